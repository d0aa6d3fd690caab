// CUDA kernels (sm_103a) and the device-side C ABI of libcbvh.
//
// Hot path: simultaneous traversal of two compressed k-DOP BVHs, Algorithm 1
// (BVHtraversal) of Tan, Weller & Zachmann, for collision detection (CD) and proximity
// query (PQ), one rigid pose of B per traversal, many poses per launch.
//
// Mapping: a persistent grid; each warp takes one pose at a time from a global counter and
// runs the traversal with an explicit node-pair stack in shared memory.  Popping (a, b)
// expands it the way Algorithm 1 recurses: the child sets of a and b (a node stands for
// itself when it is a leaf) are decoded, every child pair is tested by one lane, and a
// warp ballot compacts the survivors onto the stack; leaf pairs go to a queue that the
// warp drains 32 at a time with one triangle-triangle test per lane (checkPrimitives).
//
// Decoding (abstract; Sec. III-B): a node's slab interval is its parent's decoded interval
// corrected by b-bit deltas, so reaching a node means walking the chain of ancestors from
// its treelet's absolute root.  Each warp keeps one decoded interval per depth below the
// treelet root (tagged with the node reference); a chain walk stops at the deepest cached
// ancestor, which in depth-first order is almost always the parent.
//
// Conservative tests: B's child is its decoded axis box, moved by the pose and projected on
// each of A's directions d_j as [u_j.c + s_j - |u_j|.h, u_j.c + s_j + |u_j|.h] with
// u_j = R^T d_j, s_j = d_j.t.  Every contributing operation rounds outward (directed-rounding
// intrinsics) and the interval is widened by a bound on the rounding error of u_j, so a
// pair is pruned only if its exact bounding volumes are disjoint.  PQ uses the same
// intervals for the slab-gap lower bound max_j gap_j / |d_j|.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

constexpr int kMaxK = 13;   // directions of a 26-DOP
constexpr int kMaxM = 16;   // branching factor
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;
// Resident blocks per SM the register allocation must allow: 5 for the single-query
// collision kernel (93 registers, no spills; 20 warps per SM instead of 16), 4 otherwise
// (fewer registers would spill in the distance and batch kernels).
#ifndef CBVH_MIN_BLOCKS
#define CBVH_MIN_BLOCKS(MODE, BATCH) ((MODE) == 0 && !(BATCH) ? 5 : 4)
#endif

// ceil(2^16 / n): (i * c_inv16[n]) >> 16 == i / n for 0 <= i < 256 and 1 <= n <= 16
// (the rounding error i (c_inv16[n] - 2^16 / n) / 2^16 < 1 / 256 stays below 1 / n)
__constant__ unsigned c_inv16[kMaxM + 1] = {0,    65536, 32768, 21846, 16384, 13108, 10923, 9363, 8192,
                                            7282, 6554,  5958,  5462,  5042,  4682,  4370,  4096};

__constant__ int c_dir[kMaxK][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                    {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                    {1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};

// Device view of one BVH blob.
struct BVd {
  const uint8_t *blob;
  const unsigned long long *toff;  // treelet byte offsets
  const float4 *tris;              // 3 float4 per leaf slot
  float scale;                     // 2^e
  int K, bits, lbits, rec, root, tdepth;
  uint32_t lmask;
  uint32_t n_treelets, n_tris;  // bounds of node references and leaf slots (checked build)
};

// Per-warp shared-memory layout (byte offsets inside the warp's slice).
struct Layout {
  int tdA, tdB;  // deepest node below a treelet root, A and B (sizes the decode caches)
  // CTA region: staged treelets of A and B, their offset prefixes, one mbarrier
  int cta_bytes;
  int st_off[2], st_bytes[2], st_cnt[2], st_toff[2], o_bar;
  int warp_bytes;
  int o_stack, stack_cap;
  int o_leafq, o_leafqlb, leafq_cap;
  int o_pose;
  int o_tagA, o_latA, o_pathA;
  int o_tagB, o_latB, o_pathB;
  int o_aset, o_bset, o_bvd, o_shift, o_abox;
  int KS;      // row stride (floats) of the per-child direction arrays
  int MA, MB;  // rows of A's and of B's set arrays: E x A's branching factor, B's branching factor
  int E;       // node pairs expanded together (see the pop in traverse_kernel), E x mA <= kMaxM
};

// One work item of a batched query (see cbvh_batch_*): a pair of hierarchies, its poses and
// outputs.  Items of one launch share A's direction count and the query kind.
struct BatchItem {
  BVd A, B;
  const float *poses;
  uint8_t *hit;
  float *dist;
  uint8_t *any_hit;  // collision: per-pose flag shared by the items of one configuration set, or null
  float *min_dist;   // distance: per-pose minimum shared by the items of one configuration set, or null
  uint32_t flags, pad;
};

struct Params {
  BVd A, B;
  const BatchItem *items;              // batched query: item table, or null
  const unsigned long long *item_base; // first global pose id of each item, n_items + 1 entries
  int n_items;
  const float *poses;
  int64_t n;
  // CD
  uint8_t *hit;
  uint32_t *counts;         // per-pose pair counts (or null)
  uint32_t *triples;        // (pose, i, j) scratch
  unsigned long long cap;   // triple capacity
  unsigned long long *pair_count;
  uint32_t flags;
  // PQ
  float *dist;
  // common
  int32_t *status;
  unsigned long long *stats;  // [0] BV-pair tests, [1] leaf tests (checkPrimitives calls), [2] expansions
  const uint8_t *skip;        // PQ: poses already known to intersect (distance 0), or null
  // rounds
  int round, last_round, budget;
  uint32_t task_cap;
  unsigned int *task_next;    // this round's task cursor
  const unsigned int *count_in;
  unsigned int *count_out;
  const uint4 *tasks_in;      // (pose, a, b, 0)
  uint4 *tasks_out;
  uint2 *stacks;              // per-warp node-pair stacks, L.stack_cap entries each
  // work queue (single persistent launch): task_next points at the queue counters (see
  // queue_take); tasks_out is the queue and ready[i] != 0 once queue entry i is written
  int queue;
  uint32_t *ready;
  // polls a waiting warp (work queue) or block (staged treelets) makes before it gives up
  // and reports CBVH_ERR_TIMEOUT (CBVH_OPT_WAIT_CAP)
  long long wait_cap;
  float invn[kMaxK];
  Layout L;
};

__device__ __forceinline__ void set_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

// Checked build (compiled with CBVH_CHECKED into libcbvh_checked.so): every node reference,
// record index, cache depth, leaf slot and leaf-queue position read from a blob or computed
// by the traversal is checked before it is used; a failed check records CBVH_ERR_CHECK in the
// query's status word and the access is skipped (the set is treated as empty, the slot as
// 0), so the query ends with wrong results and a status that says so, never with an access
// outside the blob or the warp's shared memory.  The default build compiles the checks out.
#ifdef CBVH_CHECKED
__device__ __noinline__ bool check_failed(int32_t *st) {
  set_status(st, CBVH_ERR_CHECK);
  return true;
}
#define CBVH_BAD(cond, st) ((cond) && check_failed(st))
#else
#define CBVH_BAD(cond, st) false
#endif

__device__ __forceinline__ const uint8_t *treelet_base(const BVd &X, uint32_t t) { return X.blob + X.toff[t]; }
// Record of local node l in the treelet at tb: fixed-size records follow the root, Stream
// VByte records are found through the treelet's table of 2-byte offsets (4-byte units).
// VAR: the code may meet Stream VByte hierarchies (a separate compilation of the decode
// path, so that the fixed-size modes carry none of it).
template <bool VAR>
__device__ __forceinline__ const uint8_t *rec_at(const BVd &X, const uint8_t *tb, uint32_t l) {
  if (VAR && X.bits == CBVH_QUANT_SVB) return tb + 4u * (uint32_t)*reinterpret_cast<const uint16_t *>(tb + 16 + 2 * l);
  return tb + 16 + (l ? X.root + (int)(l - 1) * X.rec : 0);
}
__device__ __forceinline__ uint32_t ld32(const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Delta i of a Stream VByte record (Lemire, Kurz and Rupp 2018): its 2-bit code in the
// control word gives its length (1 to 4 bytes); its offset is i plus the codes before it,
// counted by two popcounts; the bytes are read from the one or two aligned words they span.
__device__ __forceinline__ uint32_t svb_value(const uint8_t *r, unsigned long long ctl, int i) {
  const unsigned long long below = ctl & ((1ull << (2 * i)) - 1ull);
  const int off = 16 + i + __popcll(below & 0x5555555555555555ull) + 2 * __popcll(below & 0xaaaaaaaaaaaaaaaaull);
  const int len = (int)((ctl >> (2 * i)) & 3ull) + 1;
  const uint32_t *w = reinterpret_cast<const uint32_t *>(r + (off & ~3));
  const int sh = 8 * (off & 3);
  const uint32_t v = (off & 3) + len > 4 ? __funnelshift_r(w[0], w[1], sh) : w[0] >> sh;
  return len == 4 ? v : v & ((1u << (8 * len)) - 1u);
}
// Stream VByte corrector of direction j: the exact deltas to the parent's interval.
__device__ __forceinline__ int2 svb_delta(int2 P, const uint8_t *r, int j) {
  const unsigned long long ctl = (unsigned long long)ld32(r + 8) | ((unsigned long long)ld32(r + 12) << 32);
  const uint32_t dl = svb_value(r, ctl, 2 * j), dh = svb_value(r, ctl, 2 * j + 1);
  return make_int2((int)((uint32_t)P.x + dl), (int)((uint32_t)P.y - dh));
}

// Corrector of direction j in a non-root record.
template <bool VAR>
__device__ __forceinline__ int2 apply_delta(int2 P, const uint8_t *r, int bits, int j) {
  if (VAR && bits == CBVH_QUANT_SVB) return svb_delta(P, r, j);
  uint32_t dl, dh;
  if (bits == 8) {
    uint32_t v = *reinterpret_cast<const uint16_t *>(r + 8 + 2 * j);
    dl = v & 0xffu;
    dh = v >> 8;
  } else {
    uint32_t v = ld32(r + 8 + 4 * j);
    dl = v & 0xffffu;
    dh = v >> 16;
  }
  uint32_t range = (uint32_t)P.y - (uint32_t)P.x;
  int s = max(0, (32 - __clz((int)range)) - bits);
  return make_int2((int)((uint32_t)P.x + (dl << s)), (int)((uint32_t)P.y - (dh << s)));
}
// Shift of the correctors of a child whose parent's decoded interval is P.
__device__ __forceinline__ int delta_shift(int2 P, int bits) {
  const uint32_t range = (uint32_t)P.y - (uint32_t)P.x;
  return max(0, (32 - __clz((int)range)) - bits);
}
// apply_delta with the shift already known (it depends on the parent only).
template <bool VAR>
__device__ __forceinline__ int2 apply_delta_s(int2 P, const uint8_t *r, int bits, int j, int s) {
  if (VAR && bits == CBVH_QUANT_SVB) return svb_delta(P, r, j);
  uint32_t dl, dh;
  if (bits == 8) {
    const uint32_t v = *reinterpret_cast<const uint16_t *>(r + 8 + 2 * j);
    dl = v & 0xffu;
    dh = v >> 8;
  } else {
    const uint32_t v = ld32(r + 8 + 4 * j);
    dl = v & 0xffffu;
    dh = v >> 16;
  }
  return make_int2((int)((uint32_t)P.x + (dl << s)), (int)((uint32_t)P.y - (dh << s)));
}
__device__ __forceinline__ int2 abs_lattice(const uint8_t *r, int j) {
  return *reinterpret_cast<const int2 *>(r + 8 + 8 * j);
}
__device__ __forceinline__ float2 lat_to_f(int2 L, float scale) {
  return make_float2(__fmul_rn(__int2float_rd(L.x), scale), __fmul_rn(__int2float_ru(L.y), scale));
}
// Absolute bounds (lo, hi) of direction j in a record of an FP32 (bits 0) or FP16 (bits 1)
// hierarchy; half to float conversion is exact.
__device__ __forceinline__ float2 abs_bound(const uint8_t *r, int j, int bits) {
  if (bits == 0) return *reinterpret_cast<const float2 *>(r + 8 + 8 * j);
  const uint32_t v = ld32(r + 8 + 4 * j);  // lo in the low half, hi in the high half
  return make_float2(__half2float(__ushort_as_half((unsigned short)(v & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(v >> 16))));
}

// Warp-side decode cache of one BVH: per depth below a treelet root, the reference and the
// decoded lattice interval (one column per direction) of the last node decoded there.
struct Side {
  uint32_t *tag;   // [tdepth + 1]
  int2 *lat;       // [(tdepth + 1) * nd]
  int *path;       // [tdepth + 1]
  int nd;          // directions kept (K for A, 3 for B)
  uint32_t cur_t;  // treelet whose base is cached
  const uint8_t *cur_base;
  // treelets [0, st_cnt) are staged in shared memory (see stage_treelets); st_off / st_toff
  // locate the copy and its offset prefix in the dynamic shared memory
  uint32_t st_cnt;
  int st_off, st_toff;
  int32_t *status;  // the query's status word (checked build)
};

extern __shared__ __align__(128) uint8_t g_dsmem[];

// Base of treelet t: its staged copy in shared memory when there is one, else global memory.
__device__ __forceinline__ const uint8_t *tbase(const BVd &X, const Side &S, uint32_t t) {
  if (t < S.st_cnt) {
    const unsigned long long *to = reinterpret_cast<const unsigned long long *>(g_dsmem + S.st_toff);
    return g_dsmem + S.st_off + (to[t] - to[0]);
  }
  return X.blob + X.toff[t];
}

// Decoded lattice interval of node x for direction j (lanes j < nd).  Walks up to the
// deepest cached ancestor (or the treelet root), then applies the correctors down to x,
// refreshing the cache on the way.  Returns x's record; all lanes must call it.
// w0: the first word of x's record (the caller has it); S.cur_t / cur_base must hold x's
// treelet.
template <bool VAR>
__device__ void chain_decode(const BVd &X, Side &S, uint32_t x, uint32_t w0, const uint8_t *rx, int lane,
                             int2 &P) {
  const uint32_t t = x >> X.lbits, l = x & X.lmask;
  uint32_t w = w0;
  const int d = (int)(w >> 24);
  const uint32_t tb = t << X.lbits;
  const bool act = lane < S.nd;
  // fast paths of depth-first order: x itself cached, or its parent cached (one corrector)
  if (S.tag[d] == (tb | l)) {
    if (act) P = S.lat[d * S.nd + lane];
    return;
  }
  if (d > 0 && S.tag[d - 1] == (tb | (w & 0xffffu))) {
    if (act) {
      P = apply_delta<VAR>(S.lat[(d - 1) * S.nd + lane], rx, X.bits, lane);
      S.lat[d * S.nd + lane] = P;
    }
    if (lane == 0) S.tag[d] = tb | l;
    return;  // the caller synchronises the warp before anyone reads the cache
  }
  int dd = d, start = -1;
  uint32_t ll = l;
  for (;;) {
    if (S.tag[dd] == (tb | ll)) {
      start = dd;
      break;
    }
    if (lane == 0) S.path[dd] = (int)ll;
    if (dd == 0) break;
    ll = w & 0xffffu;  // the parent: in depth-first order usually cached, so look before loading
    if (CBVH_BAD(ll >= ld32(S.cur_base), S.status)) ll = 0;
    --dd;
    if (S.tag[dd] == (tb | ll)) {
      start = dd;
      break;
    }
    w = ld32(rec_at<VAR>(X, S.cur_base, ll));  // not cached: its record leads one level up
  }
  __syncwarp();
  if (start < 0) {
    if (act) {
      P = abs_lattice(rec_at<VAR>(X, S.cur_base, 0), lane);
      S.lat[lane] = P;
    }
    if (lane == 0) S.tag[0] = tb;
    start = 0;
  } else if (act) {
    P = S.lat[start * S.nd + lane];
  }
  for (int lev = start + 1; lev <= d; ++lev) {
    const uint32_t pl = (uint32_t)S.path[lev];
    if (act) {
      P = apply_delta<VAR>(P, rec_at<VAR>(X, S.cur_base, pl), X.bits, lane);
      S.lat[lev * S.nd + lane] = P;
    }
    if (lane == 0) S.tag[lev] = tb | pl;
  }
  __syncwarp();
}

// Decode the set that Algorithm 1 expands for node x -- its children, or x itself when x is
// a leaf or `force_self` -- into per-member FP32 slab bounds (lo, hi) of directions < ND,
// written to iv (row stride KS), references to ref[], and leaf slots (or 0xffffffff) to
// leaf[].  Returns
// the number of members (warp-uniform).
template <int ND, bool VAR, bool LAT>
__device__ int decode_set(const BVd &X, Side &S, uint32_t x, bool force_self, int lane, float2 *iv, int KS,
                          uint32_t *ref, uint32_t *leaf, int *shift, bool leaf_bounds = true) {
  const uint32_t t = x >> X.lbits;
  if (CBVH_BAD(t >= X.n_treelets, S.status)) return 0;
  if (t != S.cur_t) {
    S.cur_t = t;
    S.cur_base = tbase(X, S, t);
  }
  if (CBVH_BAD((x & X.lmask) >= ld32(S.cur_base), S.status)) return 0;
  const uint8_t *rx = rec_at<VAR>(X, S.cur_base, x & X.lmask);
  const uint32_t w0 = ld32(rx), w1 = ld32(rx + 4);
  const int nc = (int)((w0 >> 16) & 31u);
  const bool ext = (w0 >> 21) & 1u;
  if (CBVH_BAD(nc > kMaxM || (int)(w0 >> 24) > X.tdepth ||
                   (nc == 0 ? w1 >= X.n_tris : (ext ? w1 + nc > X.n_treelets : w1 + nc > ld32(S.cur_base))),
               S.status))
    return 0;
  const bool self = force_self || nc == 0;
  constexpr int nd = ND;
  if (self && nc == 0 && !leaf_bounds) {  // a leaf standing for itself, bounded by its triangle
    if (lane == 0) {
      ref[0] = x;
      leaf[0] = w1;
    }
    __syncwarp();
    return 1;
  }
  if (!LAT && X.bits <= 1) {  // absolute bounds in every record
    if (self) {
      if (lane < nd) iv[lane] = abs_bound(rx, lane, X.bits);
      if (lane == 0) {
        ref[0] = x;
        leaf[0] = nc == 0 ? w1 : 0xffffffffu;
      }
    } else {
      for (int it = lane; it < nc * nd; it += 32) {
        const int i = it / nd, j = it - i * nd;
        const uint8_t *rc;
        uint32_t cref;
        if (ext) {
          cref = (w1 + i) << X.lbits;
          rc = rec_at<VAR>(X, tbase(X, S, w1 + i), 0);
        } else {
          cref = (t << X.lbits) | (w1 + i);
          rc = rec_at<VAR>(X, S.cur_base, w1 + i);
        }
        iv[i * KS + j] = abs_bound(rc, j, X.bits);
        if (j == 0) {
          const uint32_t cw0 = ld32(rc);
          uint32_t sl = ((cw0 >> 16) & 31u) == 0 ? ld32(rc + 4) : 0xffffffffu;
          if (CBVH_BAD(sl != 0xffffffffu && sl >= X.n_tris, S.status)) sl = 0;
          ref[i] = cref;
          leaf[i] = sl;
        }
      }
    }
    __syncwarp();
    return self ? 1 : nc;
  }
  int2 P = make_int2(0, 0);  // x's decoded interval (lanes < nd)
  if (self || !ext) {
    chain_decode<VAR>(X, S, x, w0, rx, lane, P);
    if (self) {
      if (lane < nd) iv[lane] = lat_to_f(P, X.scale);
      if (lane == 0) {
        ref[0] = x;
        leaf[0] = nc == 0 ? w1 : 0xffffffffu;
      }
      __syncwarp();
      return 1;
    }
  }
  const int d = (int)(w0 >> 24);
  if (!ext && lane < nd) shift[lane] = delta_shift(P, X.bits);  // the children's corrector shifts
  __syncwarp();
  for (int it = lane; it < nc * nd; it += 32) {
    const int i = it / nd, j = it - i * nd;
    const uint8_t *rc;
    uint32_t cref;
    int2 L;
    if (ext) {
      cref = (w1 + i) << X.lbits;
      rc = rec_at<VAR>(X, tbase(X, S, w1 + i), 0);
      L = abs_lattice(rc, j);
    } else {
      cref = (t << X.lbits) | (w1 + i);
      rc = rec_at<VAR>(X, S.cur_base, w1 + i);
      L = apply_delta_s<VAR>(S.lat[d * nd + j], rc, X.bits, j, shift[j]);
    }
    iv[i * KS + j] = lat_to_f(L, X.scale);
    if (j == 0) {
      const uint32_t cw0 = ld32(rc);
      uint32_t sl = ((cw0 >> 16) & 31u) == 0 ? ld32(rc + 4) : 0xffffffffu;
      if (CBVH_BAD(sl != 0xffffffffu && sl >= X.n_tris, S.status)) sl = 0;
      ref[i] = cref;
      leaf[i] = sl;
    }
  }
  __syncwarp();
  return nc;
}

// ---------------------------------------------------------------- triangle tests (FP32)
struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 axpy(V3 a, float t, V3 d) { return {fmaf(t, d.x, a.x), fmaf(t, d.y, a.y), fmaf(t, d.z, a.z)}; }

// Closed point-in-triangle test for a point on (or next to) the triangle's plane.
__device__ __forceinline__ bool inside(const V3 *T, V3 N, V3 p) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    V3 e = sub(T[(k + 1) % 3], T[k]);
    if (dot(N, cross(e, sub(p, T[k]))) < 0.f) return false;
  }
  return true;
}
__device__ __forceinline__ float orient2(float ax, float ay, float bx, float by, float cx, float cy) {
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}
__device__ __forceinline__ bool straddle(float a, float b) { return (a <= 0.f && b >= 0.f) || (a >= 0.f && b <= 0.f); }
__device__ bool coplanar_hit(const V3 *P, const V3 *Q, V3 N) {
  float ax = fabsf(N.x), ay = fabsf(N.y), az = fabsf(N.z);
  int drop = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  float p[3][2], q[3][2];
  for (int i = 0; i < 3; ++i) {
    const float a[3] = {P[i].x, P[i].y, P[i].z}, b[3] = {Q[i].x, Q[i].y, Q[i].z};
    p[i][0] = a[drop == 0 ? 1 : 0];
    p[i][1] = a[drop == 2 ? 1 : 2];
    q[i][0] = b[drop == 0 ? 1 : 0];
    q[i][1] = b[drop == 2 ? 1 : 2];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const float *a = p[i], *b = p[(i + 1) % 3], *c = q[j], *d = q[(j + 1) % 3];
      float o1 = orient2(a[0], a[1], b[0], b[1], c[0], c[1]), o2 = orient2(a[0], a[1], b[0], b[1], d[0], d[1]);
      float o3 = orient2(c[0], c[1], d[0], d[1], a[0], a[1]), o4 = orient2(c[0], c[1], d[0], d[1], b[0], b[1]);
      if (o1 == 0.f && o2 == 0.f && o3 == 0.f && o4 == 0.f) {
        bool sep = false;
        for (int c2 = 0; c2 < 2; ++c2)
          if (fmaxf(a[c2], b[c2]) < fminf(c[c2], d[c2]) || fmaxf(c[c2], d[c2]) < fminf(a[c2], b[c2])) sep = true;
        if (!sep) return true;
      } else if (straddle(o1, o2) && straddle(o3, o4)) {
        return true;
      }
    }
  auto in2 = [](const float (*t)[2], const float *x) {
    float d1 = orient2(t[0][0], t[0][1], t[1][0], t[1][1], x[0], x[1]);
    float d2 = orient2(t[1][0], t[1][1], t[2][0], t[2][1], x[0], x[1]);
    float d3 = orient2(t[2][0], t[2][1], t[0][0], t[0][1], x[0], x[1]);
    bool neg = d1 < 0.f || d2 < 0.f || d3 < 0.f, pos = d1 > 0.f || d2 > 0.f || d3 > 0.f;
    return !(neg && pos);
  };
  return in2(q, p[0]) || in2(p, q[0]);
}

// Does some edge of Q (signed plane distances dq to P's plane) meet triangle P?
__device__ __forceinline__ bool edges_meet(const V3 *P, V3 N, const V3 *Q, const float *dq) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3;
    if (dq[i] == 0.f && inside(P, N, Q[i])) return true;
    if ((dq[i] < 0.f && dq[j] > 0.f) || (dq[i] > 0.f && dq[j] < 0.f)) {
      V3 x = axpy(Q[i], __fdividef(dq[i], dq[i] - dq[j]), sub(Q[j], Q[i]));
      if (inside(P, N, x)) return true;
    }
  }
  return false;
}

// Closed triangle-triangle intersection.  Triangles that are not coplanar meet iff an edge
// of one meets the other (the ends of their common segment on the planes' intersection
// line lie on edges); each edge is cut with the other triangle's plane and the cut point
// tested against that triangle.  Coplanar triangles use a 2-D edge/containment test.
// Inputs are in coordinates local to one vertex of P, so errors scale with the local size.
__device__ bool tri_hit(const V3 *P, const V3 *Q) {
  const V3 N1 = cross(sub(P[1], P[0]), sub(P[2], P[0]));
  float dq[3], dp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) dq[i] = dot(N1, sub(Q[i], P[0]));
  if ((dq[0] > 0.f && dq[1] > 0.f && dq[2] > 0.f) || (dq[0] < 0.f && dq[1] < 0.f && dq[2] < 0.f)) return false;
  const V3 N2 = cross(sub(Q[1], Q[0]), sub(Q[2], Q[0]));
#pragma unroll
  for (int i = 0; i < 3; ++i) dp[i] = dot(N2, sub(P[i], Q[0]));
  if ((dp[0] > 0.f && dp[1] > 0.f && dp[2] > 0.f) || (dp[0] < 0.f && dp[1] < 0.f && dp[2] < 0.f)) return false;
  if (dq[0] == 0.f && dq[1] == 0.f && dq[2] == 0.f) return coplanar_hit(P, Q, N1);
  return edges_meet(P, N1, Q, dq) || edges_meet(Q, N2, P, dp);
}

__device__ __forceinline__ float pt_seg2(V3 p, V3 a, V3 b) {
  V3 ab = sub(b, a), ap = sub(p, a);
  float l2 = dot(ab, ab);
  float t = l2 > 0.f ? __saturatef(__fdividef(dot(ap, ab), l2)) : 0.f;
  V3 q = sub(axpy(a, t, ab), p);
  return dot(q, q);
}
__device__ float pt_tri2(V3 p, const V3 *T) {
  const V3 N = cross(sub(T[1], T[0]), sub(T[2], T[0]));
  if (inside(T, N, p)) {
    float s = dot(N, sub(p, T[0]));
    return __fdividef(s * s, dot(N, N));
  }
  return fminf(pt_seg2(p, T[0], T[1]), fminf(pt_seg2(p, T[1], T[2]), pt_seg2(p, T[2], T[0])));
}
// Squared distance of segments [a, b] and [c, d]: the interior stationary point when it
// lies in the unit square of parameters, else the best of the four endpoint-segment cases.
__device__ float seg_seg2(V3 a, V3 b, V3 c, V3 d) {
  V3 u = sub(b, a), v = sub(d, c), w = sub(a, c);
  float A = dot(u, u), B = dot(u, v), C = dot(v, v), D = dot(u, w), E = dot(v, w);
  float den = fmaf(A, C, -B * B);
  float best = fminf(fminf(pt_seg2(a, c, d), pt_seg2(b, c, d)), fminf(pt_seg2(c, a, b), pt_seg2(d, a, b)));
  if (den > 1e-20f * A * C) {
    float s = __fdividef(fmaf(B, E, -C * D), den), t = __fdividef(fmaf(A, E, -B * D), den);
    if (s >= 0.f && s <= 1.f && t >= 0.f && t <= 1.f) {
      V3 q = sub(axpy(w, s, u), {t * v.x, t * v.y, t * v.z});
      best = fminf(best, dot(q, q));
    }
  }
  return best;
}
// Triangle-triangle distance: 0 when they meet, else the minimum over the 6 vertex-triangle
// and 9 edge-edge cases.
__device__ float tri_dist(const V3 *P, const V3 *Q) {
  if (tri_hit(P, Q)) return 0.f;
  float d2 = INFINITY;
#pragma unroll
  for (int i = 0; i < 3; ++i) d2 = fminf(d2, fminf(pt_tri2(P[i], Q), pt_tri2(Q[i], P)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) d2 = fminf(d2, seg_seg2(P[i], P[(i + 1) % 3], Q[j], Q[(j + 1) % 3]));
  return sqrtf(d2);
}

// Load leaf triangles: A's as stored, B's moved by the pose; both shifted so that A's first
// vertex is the origin.  Returns the original triangle indices.
__device__ __forceinline__ void load_pair(const float4 *atris, const float4 *btris, const float *pose, uint32_t sa,
                                          uint32_t sb, V3 *P, V3 *Q, uint32_t &ia, uint32_t &ib) {
  const float4 a0 = atris[3 * sa], a1 = atris[3 * sa + 1], a2 = atris[3 * sa + 2];
  const float4 b0 = btris[3 * sb], b1 = btris[3 * sb + 1], b2 = btris[3 * sb + 2];
  ia = __float_as_uint(a0.w);
  ib = __float_as_uint(b0.w);
  const V3 o = {a0.x, a0.y, a0.z};
  P[0] = {0.f, 0.f, 0.f};
  P[1] = sub({a1.x, a1.y, a1.z}, o);
  P[2] = sub({a2.x, a2.y, a2.z}, o);
  const float4 bb[3] = {b0, b1, b2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V3 x;
    x.x = fmaf(pose[0], bb[c].x, fmaf(pose[1], bb[c].y, fmaf(pose[2], bb[c].z, pose[9])));
    x.y = fmaf(pose[3], bb[c].x, fmaf(pose[4], bb[c].y, fmaf(pose[5], bb[c].z, pose[10])));
    x.z = fmaf(pose[6], bb[c].x, fmaf(pose[7], bb[c].y, fmaf(pose[8], bb[c].z, pose[11])));
    Q[c] = sub(x, o);
  }
}

enum { MODE_CD = 0, MODE_PQ = 1 };

// Pose cache layout (floats): R[9], t[3], then per A-direction j, 16-byte aligned: u[3],
// |u|[3], s_lo, s_hi, eta and 3 unused
constexpr int kPoseJ = 12;
__device__ __forceinline__ float *pose_dir(float *pc, int j) { return pc + 12 + kPoseJ * j; }
constexpr int kStageBytesDefault = 0;  // per hierarchy and block: leading treelets staged in shared memory

// Conservative interval of d_j . (R x + t) over B-member i: the exact posed triangle when the
// member is a leaf, otherwise its decoded axis box, given as centre and radius bound
// bc[i] = (c, M = sum |c| + h) and half-size bh[i] = (h, 0).  q = pose_dir(pc, j).
__device__ __forceinline__ float2 project_member(const float4 *btris, const float *q, const float4 *bc,
                                                 const float4 *bh, uint32_t leaf, int i) {
  const float4 q0 = reinterpret_cast<const float4 *>(q)[0];  // u[0..2], |u|[0]
  const float4 q1 = reinterpret_cast<const float4 *>(q)[1];  // |u|[1..2], s_lo, s_hi
  const float eta = q[8];
  if (leaf != 0xffffffffu) {
    const float4 *T = btris + 3 * (size_t)leaf;
    float lo = INFINITY, hi = -INFINITY;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float4 x = T[v];
      const float l = __fmaf_rd(q0.x, x.x, __fmaf_rd(q0.y, x.y, __fmaf_rd(q0.z, x.z, q1.z)));
      const float h = __fmaf_ru(q0.x, x.x, __fmaf_ru(q0.y, x.y, __fmaf_ru(q0.z, x.z, q1.w)));
      const float sl = __fmul_ru(eta, __fadd_ru(__fadd_ru(fabsf(x.x), fabsf(x.y)), fabsf(x.z)));
      lo = fminf(lo, __fsub_rd(l, sl));
      hi = fmaxf(hi, __fadd_ru(h, sl));
    }
    return make_float2(lo, hi);
  }
  const float4 c = bc[i], h = bh[i];
  const float mlo = __fmaf_rd(q0.x, c.x, __fmaf_rd(q0.y, c.y, __fmaf_rd(q0.z, c.z, q1.z)));
  const float mhi = __fmaf_ru(q0.x, c.x, __fmaf_ru(q0.y, c.y, __fmaf_ru(q0.z, c.z, q1.w)));
  const float rad = __fmaf_ru(q0.w, h.x, __fmaf_ru(q1.x, h.y, __fmul_ru(q1.y, h.z)));
  const float sl = __fmul_ru(eta, c.w);
  return make_float2(__fsub_rd(__fsub_rd(mlo, rad), sl), __fadd_ru(__fadd_ru(mhi, rad), sl));
}

// Centre, half-size and sum |c| + h of B-member i's decoded axis box (conservative: the box
// [c - h, c + h] contains [lo, hi] and M bounds sum |c| + h from above).
__device__ __forceinline__ void member_box(const float2 *bvv, int i, float4 &bc, float4 &bh) {
  float c[3], h[3], M = 0.f;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const float2 v = bvv[i * 4 + x];
    c[x] = __fmul_rn(__fadd_rn(v.x, v.y), 0.5f);
    h[x] = fmaxf(__fsub_ru(v.y, c[x]), __fsub_ru(c[x], v.x));
    M = __fadd_ru(M, __fadd_ru(fabsf(c[x]), h[x]));
  }
  bc = make_float4(c[0], c[1], c[2], M);
  bh = make_float4(h[0], h[1], h[2], 0.f);
}

// Treelet staging (Sec. III-B clusters the hierarchy into treelets sized to a cache; here the
// cache is shared memory).  Thread 0 copies the leading treelets of A and of B -- the top of
// each hierarchy, which every traversal passes through -- with one 1-D TMA bulk copy each
// (cp.async.bulk, no multicast), completing on an mbarrier; the other threads copy the
// matching prefix of the treelet offset table.  The wait on the mbarrier is bounded: if it
// runs out the block reports CBVH_ERR_TIMEOUT and reads every treelet from global memory.
// Returns whether the staged copies may be used (uniform in the block).
constexpr long long kStageSpin = 1ll << 24;
__device__ bool stage_treelets(const Params &p, uint8_t *smem) {
  const Layout &L = p.L;
  const int nst = (L.st_bytes[0] > 0) + (L.st_bytes[1] > 0);
  if (nst == 0) return false;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.o_bar);
  const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_s), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](const BVd &X, int k) {
    if (L.st_bytes[k] <= 0) return;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem + L.st_off[k]);
    const uint8_t *src = X.blob + X.toff[0];
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"((uint32_t)L.st_bytes[k]), "r"(bar_s)
                 : "memory");
  };
  auto offsets = [&](const BVd &X, int k) {
    unsigned long long *to = reinterpret_cast<unsigned long long *>(smem + L.st_toff[k]);
    for (int t = threadIdx.x; t <= L.st_cnt[k]; t += blockDim.x) to[t] = X.toff[t];
  };
  if (threadIdx.x == 0) {
    const uint32_t total = (uint32_t)(L.st_bytes[0] + L.st_bytes[1]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(total) : "memory");
    issue(p.A, 0);
    issue(p.B, 1);
  }
  offsets(p.A, 0);
  offsets(p.B, 1);
  uint32_t done = 0;
  for (long long i = 0; i < p.wait_cap && !done; ++i)
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
        : "=r"(done)
        : "r"(bar_s), "r"(0u)
        : "memory");
  const bool ok = __syncthreads_and(done) != 0;
  if (!ok) {
    if (threadIdx.x == 0) set_status(p.status, CBVH_ERR_TIMEOUT);
    // the copies may still be in flight: give them a further bounded wait of the full default
    // length, whatever CBVH_OPT_WAIT_CAP says, before the block goes on without them (their
    // shared memory is never read)
    for (long long i = 0; i < kStageSpin && !done; ++i)
      asm volatile(
          "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
          : "=r"(done)
          : "r"(bar_s), "r"(0u)
          : "memory");
  }
  return ok;
}

// One round of the traversal.  Tasks are node pairs of one pose still to be expanded: in
// round 0 the root pair of every pose, afterwards the pairs that earlier rounds handed on.
// A warp runs Algorithm 1 depth-first from its task with an explicit stack; in a round that
// may hand work on, a task that has used its expansion budget moves its whole stack into
// the next round's task buffer, so that the node-pair tree of a heavy pose is spread over
// many warps.  The last round has no budget and finishes every task; when a task buffer is
// full, warps simply keep their work.
// Work queue of a queue round.  Counters qc: [0] cursor over the round's initial tasks (the
// poses, or the tasks an earlier round handed on), [1] tickets handed to idle warps, [2]
// queue slots reserved by donors, [3] donated tasks not yet finished (raised before slots
// are reserved), [4] initial tasks finished.  An idle warp takes one
// ticket and waits for that slot's ready flag, so waiting warps poll different addresses;
// tickets beyond the reserved slots tell donors how many warps are waiting.  Every pose
// finished and no donated task unfinished means no slot can be filled any more: the warp
// leaves.  A warp that waited p.wait_cap polls (CBVH_OPT_WAIT_CAP, default kIdleSpin)
// without either is reported as CBVH_ERR_TIMEOUT (its slot could still be filled and would
// then be lost).
constexpr long long kIdleSpin = 1ll << 24;

// Lane 0 of an idle warp: 1 and the task of its ticket, or 0 when all work is finished.
// n_poses: the number of initial tasks.
__device__ __noinline__ int queue_take(const Params &p, unsigned int *qc, uint32_t n_poses, uint4 &tk) {
  volatile unsigned int *vq = qc;
  const unsigned int h = atomicAdd(&qc[1], 1u);
  if (h >= p.task_cap) return 0;  // no slot can ever be reserved for this ticket
  volatile uint32_t *rd = p.ready;
  unsigned int nap = 64;
  for (long long it = 0; it < p.wait_cap; ++it) {
    if (rd[h]) {
      __threadfence();
      const volatile uint32_t *e = reinterpret_cast<const volatile uint32_t *>(p.tasks_out + h);
      tk = make_uint4(e[0], e[1], e[2], e[3]);
      return 1;
    }
    if ((it & 7) == 7 && vq[4] >= n_poses && vq[3] == 0) return 0;
    __nanosleep(nap);
    nap = min(nap * 2, 4096u);
  }
  set_status(p.status, CBVH_ERR_TIMEOUT);
  return 0;
}

// Work donation (work queue): a busy warp gives as many entries from the bottom of its stack
// -- its shallowest, largest subtrees -- as warps wait beyond the reserved slots, at most
// half its stack, and keeps the rest.  Returns the new stack size.  Kept out of line: it runs
// at most every 64 expansions, and the traversal's loop must stay small enough for the
// instruction cache.
template <int MODE>
__device__ __noinline__ int donate(const Params &p, unsigned int *qc, uint2 *stack, float *stack_lb, int sp,
                                   uint32_t gid, int lane) {
  int want = 0;
  if (lane == 0) {
    const int waiting = (int)(*reinterpret_cast<volatile unsigned int *>(&qc[1]) -
                              *reinterpret_cast<volatile unsigned int *>(&qc[2]));
    want = min(waiting, sp >> 1);
  }
  want = __shfl_sync(kFull, want, 0);
  if (want <= 0) return sp;
  uint32_t base = 0;
  int ok = 0;
  if (lane == 0) {
    atomicAdd(&qc[3], (unsigned int)want);  // counted before the slots exist
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(&qc[2]);
    for (int tries = 0; tries < 64; ++tries) {
      if ((unsigned long long)old + want > p.task_cap) break;
      const uint32_t prev = atomicCAS(&qc[2], old, old + (uint32_t)want);
      if (prev == old) {
        ok = 1;
        base = old;
        break;
      }
      old = prev;
    }
    if (!ok) atomicSub(&qc[3], (unsigned int)want);
    __threadfence();
  }
  ok = __shfl_sync(kFull, ok, 0);
  base = __shfl_sync(kFull, base, 0);
  if (!ok) return sp;
  // (handing out the entries just below the top instead made PQ several times slower: the
  // pieces are small and the donor runs dry)
  for (int k = lane; k < want; k += 32) {
    const uint2 e = stack[k];
    p.tasks_out[base + k] = make_uint4(gid, e.x, e.y, MODE == MODE_PQ ? __float_as_uint(stack_lb[k]) : 0u);
    __threadfence();
    *reinterpret_cast<volatile uint32_t *>(&p.ready[base + k]) = 1u;
  }
  for (int i0 = 0; i0 < sp - want; i0 += 32) {
    const bool in = i0 + lane < sp - want;
    uint2 e = make_uint2(0u, 0u);
    float l = 0.f;
    if (in) {
      e = stack[want + i0 + lane];
      if (MODE == MODE_PQ) l = stack_lb[want + i0 + lane];
    }
    __syncwarp();
    if (in) {
      stack[i0 + lane] = e;
      if (MODE == MODE_PQ) stack_lb[i0 + lane] = l;
    }
    __syncwarp();
  }
  return sp - want;
}

// Rounds: a task over its expansion budget moves its whole stack into the next round's task
// buffer.  Returns whether it did (false: the buffer is full and the warp keeps the work).
template <int MODE>
__device__ __noinline__ bool hand_on(const Params &p, const uint2 *stack, const float *stack_lb, int sp, uint32_t gid,
                                     int lane) {
  uint32_t base = 0;
  int ok = 0;
  if (lane == 0) {
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(p.count_out);
    for (int tries = 0; tries < 64; ++tries) {
      if ((unsigned long long)old + sp > p.task_cap) break;
      const uint32_t prev = atomicCAS(p.count_out, old, old + (uint32_t)sp);
      if (prev == old) {
        ok = 1;
        base = old;
        break;
      }
      old = prev;
    }
  }
  ok = __shfl_sync(kFull, ok, 0);
  base = __shfl_sync(kFull, base, 0);
  if (!ok) return false;
  for (int k = lane; k < sp; k += 32) {
    const uint2 e = stack[k];
    p.tasks_out[base + k] = make_uint4(gid, e.x, e.y, MODE == MODE_PQ ? __float_as_uint(stack_lb[k]) : 0u);
  }
  __syncwarp();
  return true;
}

// LAT: both hierarchies store predictor-corrector deltas (8 or 16 bits); the kernel then
// carries no decode path for absolute bounds, which keeps its loop small for the
// instruction cache.
template <int MODE, int KA, bool BATCH, bool VAR, bool LAT>
__global__ void __launch_bounds__(kThreads, CBVH_MIN_BLOCKS(MODE, BATCH)) traverse_kernel(const Params p) {
  uint8_t *smem = g_dsmem;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const bool staged = BATCH ? false : stage_treelets(p, smem);
  uint8_t *ws = smem + p.L.cta_bytes + wib * p.L.warp_bytes;
  uint2 *stack = reinterpret_cast<uint2 *>(reinterpret_cast<uint8_t *>(p.stacks) +
                                           ((size_t)blockIdx.x * (blockDim.x >> 5) + wib) *
                                               (size_t)((p.L.stack_cap * 12 + 15) & ~15));
  float *stack_lb = reinterpret_cast<float *>(stack + p.L.stack_cap);  // PQ: lower bound of each entry
  uint2 *leafq = reinterpret_cast<uint2 *>(ws + p.L.o_leafq);
  float *leafq_lb = reinterpret_cast<float *>(ws + p.L.o_leafqlb);
  float *pc = reinterpret_cast<float *>(ws + p.L.o_pose);
  constexpr int KS = (KA & 1) ? KA : KA + 1;
  Side SA{reinterpret_cast<uint32_t *>(ws + p.L.o_tagA),
          reinterpret_cast<int2 *>(ws + p.L.o_latA),
          reinterpret_cast<int *>(ws + p.L.o_pathA),
          KA,
          0xffffffffu,
          nullptr,
          staged ? (uint32_t)p.L.st_cnt[0] : 0u,
          p.L.st_off[0],
          p.L.st_toff[0],
          p.status};
  Side SB{reinterpret_cast<uint32_t *>(ws + p.L.o_tagB),
          reinterpret_cast<int2 *>(ws + p.L.o_latB),
          reinterpret_cast<int *>(ws + p.L.o_pathB),
          3,
          0xffffffffu,
          nullptr,
          staged ? (uint32_t)p.L.st_cnt[1] : 0u,
          p.L.st_off[1],
          p.L.st_toff[1],
          p.status};
  float2 *aiv = reinterpret_cast<float2 *>(ws + p.L.o_aset);  // A members' slabs (lo, hi) [i][KS]
  const int MA = p.L.MA, MB = p.L.MB;
  uint32_t *aref = reinterpret_cast<uint32_t *>(aiv + MA * KS);
  uint32_t *aleaf = aref + MA;
  float2 *bvv = reinterpret_cast<float2 *>(ws + p.L.o_bset);  // B members' axis slabs [i][0..2]
  float4 *bcm = reinterpret_cast<float4 *>(bvv + MB * 4);  // B members' box centre and M [i]
  float4 *bhm = bcm + MB;                                   // ... and half-size [i]
  float2 *piv = reinterpret_cast<float2 *>(bhm + MB);      // B members projected on A's directions [i][KS]
  uint32_t *bref = reinterpret_cast<uint32_t *>(piv + MB * KS);
  uint32_t *bleaf = bref + MB;
  int *shift = reinterpret_cast<int *>(ws + p.L.o_shift);
  float2 *abox = reinterpret_cast<float2 *>(ws + p.L.o_abox);  // [i][3], valid while abox_ok
  bool abox_ok = false;
  for (int i = lane; i <= p.L.tdA; i += 32) SA.tag[i] = 0xffffffffu;
  for (int i = lane; i <= p.L.tdB; i += 32) SB.tag[i] = 0xffffffffu;
  __syncwarp();
  // the query being served: fixed for a single query (read from the launch parameters), per
  // work item for a batch (the item's hierarchy views are kept in the warp's shared memory)
  BVd *bv = reinterpret_cast<BVd *>(ws + p.L.o_bvd);
  const BVd &A = BATCH ? bv[0] : p.A;
  const BVd &B = BATCH ? bv[1] : p.B;
  const float *poses = p.poses;
  uint8_t *hitp = p.hit;
  uint8_t *anyp = nullptr;  // batch items of one configuration set: "some item of this pose intersects"
  float *mindp = nullptr;   // ... and "the smallest distance any item of this pose has found"
  float *distp = p.dist;
  bool early = (p.flags & CBVH_EARLY_EXIT) != 0;
  int item = -1;
  unsigned long long item_lo = 0;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t n_in = p.round == 0 ? (uint32_t)p.n : min(*p.count_in, p.task_cap);
  const bool may_spill = !p.last_round;
  // work queue: what the task just finished was (1 a pose, 2 a donated task), and the
  // poses this warp finished since it last reported them
  unsigned int *qc = p.task_next;
  int prev_kind = 0;
  bool poses_out = false;
  unsigned int my_poses = 0;
  unsigned long long n_bv = 0, n_leaf = 0, n_exp = 0;
  int64_t cur_pose = -1;
  uint32_t keyA = 0xffffffffu, keyB = 0xffffffffu;  // node whose member set is decoded / projected
  int na_c = 0, nb_c = 0;

  for (;;) {
    uint32_t gid = 0, a = 0, b = 0;  // global pose id (equal to the pose index of a single query)
    bool root = false;
    float task_lb = 0.f;  // PQ: lower bound of the task's node pair
    if (p.queue) {
      // account for the task just finished, then take a pose, else a donated task
      if (prev_kind == 1) ++my_poses;
      if (prev_kind == 2 && lane == 0) atomicSub(&qc[3], 1u);
      prev_kind = 0;
      if (!poses_out) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(&qc[0], 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t < n_in) {
          if (p.round == 0) {
            gid = t;
            root = true;
          } else {  // the tasks the previous round handed on
            const uint4 x = p.tasks_in[t];
            gid = x.x;
            a = x.y;
            b = x.z;
            task_lb = __uint_as_float(x.w);
          }
          prev_kind = 1;
        } else {
          poses_out = true;
          if (lane == 0 && my_poses) atomicAdd(&qc[4], my_poses);
          my_poses = 0;
        }
      }
      if (prev_kind == 0) {
        uint4 tk = make_uint4(0u, 0u, 0u, 0u);
        int got = 0;
        if (lane == 0) got = queue_take(p, qc, n_in, tk);
        if (!__shfl_sync(kFull, got, 0)) break;
        gid = __shfl_sync(kFull, tk.x, 0);
        a = __shfl_sync(kFull, tk.y, 0);
        b = __shfl_sync(kFull, tk.z, 0);
        task_lb = __uint_as_float(__shfl_sync(kFull, tk.w, 0));
        prev_kind = 2;
      }
    } else {
      unsigned int task = 0;
      if (lane == 0) task = atomicAdd(p.task_next, 1u);
      task = __shfl_sync(kFull, task, 0);
      if (task >= n_in) break;
      if (p.round == 0) {
        gid = task;
        root = true;
      } else {
        const uint4 t = p.tasks_in[task];
        gid = t.x;
        a = t.y;
        b = t.z;
        task_lb = __uint_as_float(t.w);
      }
    }
    if (BATCH) {
      // find the work item holding this global pose id (uniform across the warp)
      int lo = 0, hi = p.n_items - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.item_base[mid] <= gid)
          lo = mid;
        else
          hi = mid - 1;
      }
      if (lo != item) {
        item = lo;
        const BatchItem &it = p.items[lo];
        {
          const uint32_t *src = reinterpret_cast<const uint32_t *>(&it.A);  // A and B are adjacent
          uint32_t *dst = reinterpret_cast<uint32_t *>(bv);
          for (int w = lane; w < (int)(2 * sizeof(BVd) / 4); w += 32) dst[w] = src[w];
        }
        poses = it.poses;
        hitp = it.hit;
        anyp = it.any_hit;
        mindp = it.min_dist;
        distp = it.dist;
        early = (it.flags & CBVH_EARLY_EXIT) != 0;
        item_lo = p.item_base[lo];
        // node references and projections belong to the previous pair of hierarchies
        for (int i = lane; i <= p.L.tdA; i += 32) SA.tag[i] = 0xffffffffu;
        for (int i = lane; i <= p.L.tdB; i += 32) SB.tag[i] = 0xffffffffu;
        SA.cur_t = SB.cur_t = 0xffffffffu;
        keyA = keyB = 0xffffffffu;
        cur_pose = -1;
        __syncwarp();
      }
    }
    const uint32_t pose = (uint32_t)(gid - item_lo);  // pose index within its query
    if ((int64_t)gid != cur_pose) {
      keyB = 0xffffffffu;  // projections depend on the pose
      abox_ok = false;
      // ---- pose precompute: u_j = R^T d_j, |u_j|, [s_lo, s_hi] of d_j.t, and eta_j, a
      // bound on the rounding error of each component of u_j ----
      cur_pose = gid;
      if (lane < 12) pc[lane] = poses[12 * (size_t)pose + lane];
      __syncwarp();
      if (lane < KA) {
        const int d0 = c_dir[lane][0], d1 = c_dir[lane][1], d2 = c_dir[lane][2];
        float *q = pose_dir(pc, lane);
        float smax = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float r0 = pc[c], r1 = pc[3 + c], r2 = pc[6 + c];
          const float u = __fadd_rn(__fadd_rn(d0 * r0, d1 * r1), d2 * r2);
          q[c] = u;
          q[3 + c] = fabsf(u);
          smax = fmaxf(smax, __fadd_ru(__fadd_ru(fabsf(d0 * r0), fabsf(d1 * r1)), fabsf(d2 * r2)));
        }
        q[6] = __fadd_rd(__fadd_rd(d0 * pc[9], d1 * pc[10]), d2 * pc[11]);
        q[7] = __fadd_ru(__fadd_ru(d0 * pc[9], d1 * pc[10]), d2 * pc[11]);
        q[8] = __fmul_ru(smax, 2.384185791015625e-07f);  // 2^-22
      }
      __syncwarp();
    }
    // per-pose state: the root task initialises it; later tasks update it atomically
    float best = INFINITY;
    if (root) {
      if (MODE == MODE_PQ && p.skip && p.skip[gid]) {  // intersecting: the distance is 0
        if (lane == 0) {
          distp[pose] = 0.f;
          if (BATCH && mindp) atomicMin(reinterpret_cast<unsigned int *>(&mindp[pose]), 0u);
        }
        continue;
      }
      int settled = 0;
      float v = INFINITY;
      if (lane == 0) {
        if (MODE == MODE_CD) {
          hitp[pose] = 0;
          if (p.counts) p.counts[pose] = 0;
          if (BATCH && anyp) settled = *reinterpret_cast<volatile uint8_t *>(&anyp[pose]);
        } else {
          distp[pose] = INFINITY;
          if (BATCH && mindp) v = *reinterpret_cast<volatile float *>(&mindp[pose]);
        }
      }
      if (BATCH && MODE == MODE_CD && __shfl_sync(kFull, settled, 0)) continue;  // the set's answer is known
      if (BATCH && MODE == MODE_PQ) {
        best = __shfl_sync(kFull, v, 0);  // the set's best so far bounds this item too
        if (best == 0.f) continue;
      }
    } else if (MODE == MODE_PQ) {
      float v = 0.f;
      if (lane == 0) {
        v = *reinterpret_cast<volatile float *>(&distp[pose]);
        if (BATCH && mindp) v = fminf(v, *reinterpret_cast<volatile float *>(&mindp[pose]));
      }
      best = __shfl_sync(kFull, v, 0);
      if (task_lb >= best) continue;  // a closer pair was found after this one was handed on
    } else if (early) {
      int h = 0;
      if (lane == 0) {
        h = *reinterpret_cast<volatile uint8_t *>(&hitp[pose]);
        if (BATCH && anyp) h |= *reinterpret_cast<volatile uint8_t *>(&anyp[pose]);
      }
      if (__shfl_sync(kFull, h, 0)) continue;
    }
    int sp = 0, nleaf = 0;
    uint32_t nhits = 0;
    bool done = false;
    int expansions = 0;
    int nx = 0;                         // further node pairs (ax[q], b) expanded with (a, b)
    uint32_t ax0 = 0, ax1 = 0, ax2 = 0;
    // checkPrimitives on the last `cnt` queued leaf pairs, one pair per lane
    auto drain = [&](int cnt) {
      nleaf -= cnt;
      bool h = false;
      float dl = INFINITY;
      uint32_t ia = 0, ib = 0;
      // PQ: a queued pair whose bound reached the best distance found since is skipped
      const bool test = lane < cnt && (MODE == MODE_CD || leafq_lb[nleaf + lane] < best);
      n_leaf += __popc(__ballot_sync(kFull, test));
      if (test) {
        const uint2 e = leafq[nleaf + lane];
        V3 P[3], Q[3];
        load_pair(A.tris, B.tris, pc, e.x, e.y, P, Q, ia, ib);
        if (MODE == MODE_CD)
          h = tri_hit(P, Q);
        else
          dl = tri_dist(P, Q);
      }
      __syncwarp();
      if (MODE == MODE_CD) {
        const unsigned mh = __ballot_sync(kFull, h);
        if (mh) {
          nhits += __popc(mh);
          if (p.counts) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(p.pair_count, (unsigned long long)__popc(mh));
            b0 = __shfl_sync(kFull, b0, 0);
            if (h) {
              const unsigned long long slot = b0 + __popc(mh & lt);
              if (slot < p.cap) {
                p.triples[3 * slot] = pose;
                p.triples[3 * slot + 1] = ia;
                p.triples[3 * slot + 2] = ib;
              }
            }
          }
          if (early) done = true;
        }
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dl = fminf(dl, __shfl_xor_sync(kFull, dl, o));
        // a distance this task found below every bound it knows is published at once (to the
        // set's minimum too); the pose's output only ever receives distances of its own pairs
        if (dl < best) {
          best = dl;
          if (lane == 0) {
            atomicMin(reinterpret_cast<unsigned int *>(&distp[pose]), __float_as_uint(best));
            if (BATCH && mindp) atomicMin(reinterpret_cast<unsigned int *>(&mindp[pose]), __float_as_uint(best));
          }
        }
        if (best == 0.f) done = true;
      }
    };

    for (;;) {
      // ---------------- expand (a, b) as Algorithm 1 does ----------------
      // A's member set depends on a only, B's projected set on b and the pose: in depth-first
      // order one of them is often the same as in the previous expansion and is reused.
      // Several popped pairs (a, b), (ax0, b), ... that share b expand as one: the member
      // sets of their A nodes are decoded one after another into consecutive rows, and their
      // pairs with B's members tested, compacted and pushed together, which fills the lanes
      // of the pair loop and shares the expansion's fixed costs.
      int na, nb;
      if (nx > 0 || a != keyA || root) {
        na = 0;
        for (int q = 0; q <= nx; ++q) {
          const uint32_t x = q == 0 ? a : (q == 1 ? ax0 : (q == 2 ? ax1 : ax2));
          na += decode_set<KA, VAR, LAT>(A, SA, x, root, lane, aiv + na * KS, KS, aref + na, aleaf + na, shift);
        }
        keyA = (root || nx > 0) ? 0xffffffffu : a;
        na_c = na;
        abox_ok = false;
      } else {
        na = na_c;
      }
      if (b != keyB || root) {
        nb = decode_set<3, VAR, LAT>(B, SB, b, root, lane, bvv, 4, bref, bleaf, shift, false);
        if (lane < nb && bleaf[lane] == 0xffffffffu) member_box(bvv, lane, bcm[lane], bhm[lane]);
        if (lane < 3 * nb) {  // leaf members: the exact box of their triangle
          const int i = lane / 3, x = lane - 3 * i;
          if (bleaf[i] != 0xffffffffu) {
            const float *T = reinterpret_cast<const float *>(B.tris + 3 * (size_t)bleaf[i]);
            const float v0 = T[x], v1 = T[4 + x], v2 = T[8 + x];
            bvv[i * 4 + x] = make_float2(fminf(v0, fminf(v1, v2)), fmaxf(v0, fmaxf(v1, v2)));
          }
        }
        __syncwarp();
        for (int it = lane; it < nb * KA; it += 32) {
          const int i = it / KA, j = it - i * KA;
          piv[i * KS + j] = project_member(B.tris, pose_dir(pc, j), bcm, bhm, bleaf[i], i);
        }
        __syncwarp();
        keyB = root ? 0xffffffffu : b;
        nb_c = nb;
      } else {
        nb = nb_c;
      }
      root = false;
      ++expansions;
      n_exp += 1 + nx;
      // test every member pair; survivors are compacted by ballot onto the stack (inner
      // pairs) or the leaf queue (leaf pairs)
      if (!abox_ok) {
        // A's members' axis boxes in B's frame: along B's axis k (world direction u = column k
        // of R, exact) the box projects to u.c - u.t +- |u|.h, all rounded outward
        for (int it = lane; it < 3 * na; it += 32) {
          const int i = it / 3, k = it - 3 * i;
          float c[3], h[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const float2 v = aiv[i * KS + x];
            c[x] = __fmul_rn(__fadd_rn(v.x, v.y), 0.5f);
            h[x] = fmaxf(__fsub_ru(v.y, c[x]), __fsub_ru(c[x], v.x));
          }
          const float u0 = pc[k], u1 = pc[3 + k], u2 = pc[6 + k];
          const float uc_lo = __fmaf_rd(u0, c[0], __fmaf_rd(u1, c[1], __fmul_rd(u2, c[2])));
          const float uc_hi = __fmaf_ru(u0, c[0], __fmaf_ru(u1, c[1], __fmul_ru(u2, c[2])));
          const float ut_lo = __fmaf_rd(u0, pc[9], __fmaf_rd(u1, pc[10], __fmul_rd(u2, pc[11])));
          const float ut_hi = __fmaf_ru(u0, pc[9], __fmaf_ru(u1, pc[10], __fmul_ru(u2, pc[11])));
          const float r = __fmaf_ru(fabsf(u0), h[0], __fmaf_ru(fabsf(u1), h[1], __fmul_ru(fabsf(u2), h[2])));
          abox[i * 3 + k] = make_float2(__fsub_rd(__fsub_rd(uc_lo, ut_hi), r), __fadd_ru(__fsub_ru(uc_hi, ut_lo), r));
        }
        __syncwarp();
        abox_ok = true;
      }
      const int np = na * nb;
      // pairs in B-major order: the pair popped next shares B's projected set with the one
      // before (a B change costs a decode and a projection on all of A's directions, about
      // twice an A decode)
      const unsigned inv_na = c_inv16[na];  // it / na == (it * inv_na) >> 16 for it < 256
      n_bv += np;
      float run_lb = INFINITY;  // PQ: smallest lower bound pushed by this expansion ...
      int run_pos = -1;         // ... and its stack slot
      for (int base = 0; base < np && !done; base += 32) {
        const int it = base + lane;
        bool keep = false;
        int i = 0, j = 0;
        float lb = INFINITY;
        if (it < np) {
          j = (int)(((unsigned)it * inv_na) >> 16);
          i = it - j * na;
          const float2 *av = aiv + i * KS, *pv = piv + j * KS;
          if (MODE == MODE_CD) {
            keep = true;
#pragma unroll
            for (int d = 0; d < KA; ++d) {
              const float2 x = av[d], y = pv[d];
              keep &= (x.x <= y.y) & (y.x <= x.y);
            }
            if (keep) {  // and B's own axes: A's box moved into B's frame against B's box
              const float2 *ab = abox + i * 3, *bb = bvv + j * 4;
#pragma unroll
              for (int k = 0; k < 3; ++k) keep &= (ab[k].x <= bb[k].y) & (bb[k].x <= ab[k].y);
            }
          } else {
            // three lower bounds, all rounded down: the widest slab gap over |d|, the
            // distance between the axis boxes (root of the squared x, y and z gaps), and the
            // same in B's frame
            lb = 0.f;
            float box2 = 0.f;
#pragma unroll
            for (int d = 0; d < KA; ++d) {
              const float2 x = av[d], y = pv[d];
              const float g = fmaxf(__fsub_rd(x.x, y.y), __fsub_rd(y.x, x.y));
              lb = fmaxf(lb, __fmul_rd(g, p.invn[d]));
              if (d < 3) {
                const float gp = fmaxf(g, 0.f);
                box2 = __fmaf_rd(gp, gp, box2);
              }
            }
            const float2 *ab = abox + i * 3, *bb = bvv + j * 4;  // A's box moved into B's frame
            float box2b = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const float g = fmaxf(fmaxf(__fsub_rd(ab[k].x, bb[k].y), __fsub_rd(bb[k].x, ab[k].y)), 0.f);
              box2b = __fmaf_rd(g, g, box2b);
            }
            lb = fmaxf(lb, __fsqrt_rd(fmaxf(box2, box2b)));
            keep = lb < best;
          }
        }
        const bool isleaf = keep && aleaf[i] != 0xffffffffu && bleaf[j] != 0xffffffffu;
        const unsigned ml = __ballot_sync(kFull, isleaf);
        const unsigned mi = __ballot_sync(kFull, keep && !isleaf);
        if (CBVH_BAD(nleaf + __popc(ml) > p.L.leafq_cap, p.status)) {
          done = true;
          break;
        }
        if (sp + __popc(mi) > p.L.stack_cap) {
          if (lane == 0) set_status(p.status, CBVH_ERR_STACK);
          done = true;
          break;
        }
        const int pos = sp + __popc(mi & lt);
        if (isleaf) {
          leafq[nleaf + __popc(ml & lt)] = make_uint2(aleaf[i], bleaf[j]);
          if (MODE == MODE_PQ) leafq_lb[nleaf + __popc(ml & lt)] = lb;
        }
        if (keep && !isleaf) {
          stack[pos] = make_uint2(aref[i], bref[j]);
          if (MODE == MODE_PQ) stack_lb[pos] = lb;
        }
        if (MODE == MODE_PQ && mi) {
          float mv = (keep && !isleaf) ? lb : INFINITY;
          int mp = pos;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(kFull, mv, o);
            const int op = __shfl_xor_sync(kFull, mp, o);
            if (ov < mv || (ov == mv && op < mp)) {
              mv = ov;
              mp = op;
            }
          }
          if (mv < run_lb) {
            run_lb = mv;
            run_pos = mp;
          }
        }
        nleaf += __popc(ml);
        sp += __popc(mi);
        __syncwarp();
      }
      // PQ: the most promising child pair goes on top, so that it is expanded next
      if (MODE == MODE_PQ && run_pos >= 0 && run_pos != sp - 1 && !done) {
        if (lane == 0) {
          const uint2 x = stack[run_pos];
          stack[run_pos] = stack[sp - 1];
          stack[sp - 1] = x;
          const float xl = stack_lb[run_pos];
          stack_lb[run_pos] = stack_lb[sp - 1];
          stack_lb[sp - 1] = xl;
        }
        __syncwarp();
      }
      // ---------------- leaf tests, scheduling ----------------
      // Leaf pairs are tested (checkPrimitives) 32 at a time: full batches; everything once
      // the task stops (no node pairs left, or the rest handed on); and for PQ everything
      // while no distance is known, since until then nothing can be pruned.  Between the
      // batches and the pop: donation to waiting warps, hand-off to the next round, the
      // periodic poll of the pose's shared result, and (PQ) dropping stale entries.  The
      // loop below is the one place the triangle tests are compiled in.
      bool stop = done || sp == 0;
      for (bool first = true;; first = false) {
        while (!done && nleaf > 0 && (nleaf >= 32 || stop || (MODE == MODE_PQ && best == INFINITY)))
          drain(min(nleaf, 32));
        if (done || stop || !first) break;
        if (p.queue && sp >= 2 && expansions >= p.budget && (expansions & 63) == 0)
          sp = donate<MODE>(p, qc, stack, stack_lb, sp, gid, lane);
        if (!p.queue && may_spill && expansions >= p.budget && sp >= 2 && hand_on<MODE>(p, stack, stack_lb, sp, gid, lane)) {
          sp = 0;
          stop = true;
        }
        if (!stop && (expansions & (early ? 3 : 15)) == 0) {
          if (MODE == MODE_PQ) {
            float v = 0.f;
            if (lane == 0) {
              v = *reinterpret_cast<volatile float *>(&distp[pose]);
              if (BATCH && mindp) v = fminf(v, *reinterpret_cast<volatile float *>(&mindp[pose]));
            }
            best = fminf(best, __shfl_sync(kFull, v, 0));
          } else if (early) {
            int h = 0;
            if (lane == 0) {
              h = *reinterpret_cast<volatile uint8_t *>(&hitp[pose]);
              if (BATCH && anyp) h |= *reinterpret_cast<volatile uint8_t *>(&anyp[pose]);
            }
            if (__shfl_sync(kFull, h, 0)) done = true;  // another task of the pose (or of its set) found a pair
          }
        }
        // PQ: entries whose lower bound reached the best distance found since they were
        // pushed cannot hold a closer pair and are dropped
        if (MODE == MODE_PQ && !stop) {
          while (sp > 0 && stack_lb[sp - 1] >= best) --sp;
          if (sp == 0) stop = true;
        }
        if (!stop) break;
      }
      if (done || stop) break;
      // ---------------- pop ----------------
      // the top pair, and up to E - 1 more below it with the same B node (pairs are pushed
      // B-major, so the children of one expansion with one B member lie together on top)
      const uint2 e = stack[--sp];
      a = e.x;
      b = e.y;
      nx = 0;
      if (p.L.E > 1) {
        bool more = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (more && q < p.L.E - 1 && sp > 0) {
            const uint2 f = stack[sp - 1];
            if (f.y == b && (MODE == MODE_CD || stack_lb[sp - 1] < best)) {
              if (q == 0) ax0 = f.x;
              if (q == 1) ax1 = f.x;
              if (q == 2) ax2 = f.x;
              --sp;
              ++nx;
            } else {
              more = false;
            }
          }
        }
      }
      __syncwarp();
    }
    nleaf = 0;
    if (lane == 0) {
      if (MODE == MODE_CD) {
        if (nhits) {
          hitp[pose] = 1;
          if (BATCH && anyp) anyp[pose] = 1;
          if (p.counts) atomicAdd(&p.counts[pose], nhits);
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&p.stats[0], n_bv);
    atomicAdd(&p.stats[1], n_leaf);
    atomicAdd(&p.stats[2], n_exp);
  }
}

// ---------------------------------------------------------------- output compaction
// Exclusive scan of per-pose counts into int64 offsets (one CTA, tiles of 1024 x 4);
// offsets[n] = total, also stored in *needed; flags capacity overflow in *status.
__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t *counts, int64_t n, int64_t *offsets,
                                                    int64_t *needed, unsigned long long cap, int32_t *status) {
  __shared__ long long warp_sums[32];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 4096) {
    long long v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = base + 4 * tid + k;
      v[k] = i < n ? counts[i] : 0;
      s += v[k];
    }
    long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      long long ws = warp_sums[lane], wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += y;
      }
      warp_sums[lane] = wi - ws;
    }
    __syncthreads();
    long long run = carry_s + warp_sums[wid] + incl - s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = base + 4 * tid + k;
      if (i < n) offsets[i] = run;
      run += v[k];
    }
    __syncthreads();
    if (tid == 1023) carry_s = run;
    __syncthreads();
  }
  if (tid == 0) {
    offsets[n] = carry_s;
    if (needed) *needed = carry_s;
    if ((unsigned long long)carry_s > cap) set_status(status, CBVH_ERR_CAPACITY);
  }
}

// Scatter (pose, i, j) triples into each pose's CSR segment (order within a pose arbitrary).
__global__ void scatter_kernel(const uint32_t *triples, const unsigned long long *count, unsigned long long cap,
                               const int64_t *offsets, uint32_t *cursor, int32_t *pairs) {
  const unsigned long long total = *count;
  if (total > cap) return;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t pose = triples[3 * t];
    const uint32_t slot = atomicSub(&cursor[pose], 1u) - 1u;
    const int64_t o = offsets[pose] + slot;
    pairs[2 * o] = (int32_t)triples[3 * t + 1];
    pairs[2 * o + 1] = (int32_t)triples[3 * t + 2];
  }
}

// Sort each pose's pairs by (i, j).  In shared memory: a bitonic network whose first stage of
// every merge compares mirrored elements, so that padding beyond the segment acts as
// +infinity.
constexpr int kSortSmem = 4096;
__device__ __forceinline__ void cmp_swap(unsigned long long *k, int i, int j) {
  unsigned long long a = k[i], b = k[j];
  if (a > b) {
    k[i] = b;
    k[j] = a;
  }
}
__device__ void bitonic(unsigned long long *k, int n) {
  int N = 1;
  while (N < n) N <<= 1;
  for (int size = 2; size <= N; size <<= 1) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int j = i ^ (size - 1);
      if (j > i && j < n) cmp_swap(k, i, j);
    }
    __syncthreads();
    for (int s = size >> 2; s > 0; s >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int j = i ^ s;
        if (j > i && j < n) cmp_swap(k, i, j);
      }
      __syncthreads();
    }
  }
}
// Pairs of a segment as sort keys (i << 32 | j).
__device__ __forceinline__ unsigned long long pair_key(const int32_t *pairs, int64_t q) {
  return ((unsigned long long)(uint32_t)pairs[2 * q] << 32) | (uint32_t)pairs[2 * q + 1];
}
// Merge of the sorted runs L[0, m) and R[0, r) into out[0, m + r) by the block: each thread
// finds where its share of the output starts on the merge path (binary search for the
// number of its first outputs taken from L), then merges that share sequentially.
__device__ void merge_runs(const unsigned long long *L, int m, const unsigned long long *R, int r,
                           unsigned long long *out) {
  const int total = m + r;
  const int per = (total + blockDim.x - 1) / blockDim.x;
  const int k0 = min(total, (int)threadIdx.x * per), k1 = min(total, k0 + per);
  if (k0 >= k1) return;
  int lo = max(0, k0 - r), hi = min(k0, m);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (L[mid] <= R[k0 - mid - 1])
      lo = mid + 1;
    else
      hi = mid;
  }
  int i = lo, j = k0 - lo;
  for (int k = k0; k < k1; ++k) out[k] = (j >= r || (i < m && L[i] <= R[j])) ? L[i++] : R[j++];
}
// One block per pose (grid-stride).  A segment of at most kSortSmem pairs is sorted in shared
// memory.  A longer one is sorted in runs of kSortSmem in shared memory, written to tmp (the
// triples scratch, free once the scatter has run), then merged pairwise, alternating between
// tmp and the segment itself, so that each pass reads and writes the segment once.
__global__ void __launch_bounds__(256) sort_kernel(const int64_t *offsets, int64_t n, const unsigned long long *count,
                                                   unsigned long long cap, int32_t *pairs, unsigned long long *tmp) {
  __shared__ unsigned long long keys[kSortSmem];
  if (*count > cap) return;
  for (int64_t pose = blockIdx.x; pose < n; pose += gridDim.x) {
    const int64_t o = offsets[pose];
    const int cnt = (int)(offsets[pose + 1] - o);
    if (cnt < 2) continue;
    unsigned long long *seg = reinterpret_cast<unsigned long long *>(pairs + 2 * o);
    unsigned long long *src = tmp + o, *dst = seg;
    for (int c0 = 0; c0 < cnt; c0 += kSortSmem) {
      const int len = min(kSortSmem, cnt - c0);
      for (int i = threadIdx.x; i < len; i += blockDim.x) keys[i] = pair_key(pairs, o + c0 + i);
      __syncthreads();
      bitonic(keys, len);
      if (cnt <= kSortSmem) {
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
          const unsigned long long v = keys[i];
          pairs[2 * (o + i)] = (int32_t)(v >> 32);
          pairs[2 * (o + i) + 1] = (int32_t)(v & 0xffffffffu);
        }
      } else {
        for (int i = threadIdx.x; i < len; i += blockDim.x) src[c0 + i] = keys[i];
      }
      __syncthreads();
    }
    if (cnt <= kSortSmem) continue;
    for (int w = kSortSmem; w < cnt; w *= 2) {
      for (int r0 = 0; r0 < cnt; r0 += 2 * w) {
        const int m = min(w, cnt - r0), r = max(0, min(w, cnt - r0 - w));
        merge_runs(src + r0, m, src + r0 + m, r, dst + r0);
      }
      __syncthreads();
      unsigned long long *t = src;
      src = dst;
      dst = t;
    }
    // keys back to (i, j) pairs; when they already sit in the segment, each thread rewrites
    // the 8 bytes it read
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const unsigned long long v = src[i];
      pairs[2 * (o + i)] = (int32_t)(v >> 32);
      pairs[2 * (o + i) + 1] = (int32_t)(v & 0xffffffffu);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- decode test hook
// One block per treelet; thread items (local node, direction) walk their node's chain from
// the treelet root.  Output in blob order.
__global__ void decode_all_kernel(const BVd X, int32_t *lat_out, float *f_out) {
  const uint32_t t = blockIdx.x;
  const uint8_t *tb = treelet_base(X, t);
  const uint32_t cnt = ld32(tb), first = ld32(tb + 4);
  for (uint32_t it = threadIdx.x; it < cnt * (uint32_t)X.K; it += blockDim.x) {
    const uint32_t l = it / X.K, j = it - l * X.K;
    const uint8_t *r = rec_at<true>(X, tb, l);
    float2 f;
    if (X.bits <= 1) {
      f = abs_bound(r, j, X.bits);
    } else {
      uint32_t path[64];
      int d = 0;
      for (uint32_t y = l; y != 0 && d < 64; y = ld32(rec_at<true>(X, tb, y)) & 0xffffu) path[d++] = y;
      int2 P = abs_lattice(rec_at<true>(X, tb, 0), j);
      for (int q = d - 1; q >= 0; --q) P = apply_delta<true>(P, rec_at<true>(X, tb, path[q]), X.bits, j);
      f = lat_to_f(P, X.scale);
      if (lat_out) {
        lat_out[((size_t)(first + l) * X.K + j) * 2] = P.x;
        lat_out[((size_t)(first + l) * X.K + j) * 2 + 1] = P.y;
      }
    }
    if (f_out) {
      f_out[((size_t)(first + l) * X.K + j) * 2] = f.x;
      f_out[((size_t)(first + l) * X.K + j) * 2 + 1] = f.y;
    }
  }
}

// ---------------------------------------------------------------- host side
BVd view(const cbvh_bvh *h) {
  BVd v;
  const uint8_t *b = static_cast<const uint8_t *>(h->dev_blob);
  v.blob = b;
  v.toff = reinterpret_cast<const unsigned long long *>(b + 64);
  v.tris = reinterpret_cast<const float4 *>(b + h->off_tris);
  v.scale = std::ldexp(1.0f, h->e);
  v.K = h->K;
  v.bits = h->bits;
  v.lbits = h->lbits;
  v.rec = h->rec_bytes;
  v.root = h->root_bytes;
  v.tdepth = h->max_tdepth;
  v.lmask = (h->lbits >= 32) ? 0xffffffffu : ((1u << h->lbits) - 1u);
  v.n_treelets = (uint32_t)h->n_treelets;
  v.n_tris = (uint32_t)h->n_tris;
  return v;
}

int align16(int x) { return (x + 15) & ~15; }

// Process-wide tuning options (cbvh_set_option).
std::atomic<int> g_stage_bytes{kStageBytesDefault};
std::atomic<int> g_split{4};  // work mapping, see launch_rounds
std::atomic<long long> g_launches{0};  // kernels this library has launched (cbvh_kernel_launches)
std::atomic<int> g_budget0{256};  // expansion budget of a task in round 0 (later rounds scale it)
std::atomic<long long> g_wait_cap{kIdleSpin};  // polls of a bounded device wait (CBVH_OPT_WAIT_CAP)

// Per-warp slice layout for A's direction count, the deepest nodes below a treelet root on
// either side, a stack bound and the largest branching factor on either side; no staged
// treelets.  The set arrays are sized by the branching factors, not by the largest one
// supported: shared memory taken from the SM's 256 KB is lost to L1, which caches the
// stacks and the records.
Layout warp_layout(int KA, int tdA, int tdB, int stack_cap, int mA, int mB) {
  Layout L;
  std::memset(&L, 0, sizeof L);
  L.tdA = tdA;
  L.tdB = tdB;
  L.MA = mA;
  L.MB = mB;
  L.KS = (KA & 1) ? KA : KA + 1;
  L.stack_cap = stack_cap;
  L.leafq_cap = 32 + mA * mB;  // < 32 queued before an expansion, which adds <= mA mB
  int o = 0;
  L.o_stack = -1;  // stacks live in global memory
  L.o_leafq = o;
  o = align16(o + 8 * L.leafq_cap);
  L.o_leafqlb = o;
  o = align16(o + 4 * L.leafq_cap);
  L.o_pose = o;
  o = align16(o + 4 * (12 + kPoseJ * KA));
  L.o_tagA = o;
  o = align16(o + 4 * (tdA + 1));
  L.o_latA = o;
  o = align16(o + 8 * (tdA + 1) * KA);
  L.o_pathA = o;
  o = align16(o + 4 * (tdA + 1));
  L.o_tagB = o;
  o = align16(o + 4 * (tdB + 1));
  L.o_latB = o;
  o = align16(o + 8 * (tdB + 1) * 3);
  L.o_pathB = o;
  o = align16(o + 4 * (tdB + 1));
  L.o_aset = o;
  o = align16(o + 4 * (2 * mA * L.KS + 2 * mA));
  L.o_bset = o;  // axis slabs (float2 x 4), box centre and half-size (float4 x 2), projections
  o = align16(o + 4 * (2 * mB * 4 + 8 * mB + 2 * mB * L.KS + 2 * mB));
  L.o_bvd = o;
  o = align16(o + 2 * (int)sizeof(BVd));
  L.o_shift = o;  // corrector shifts of the set being decoded, one per direction
  o = align16(o + 4 * kMaxK);
  L.o_abox = o;  // A members' axis boxes moved into B's frame, (lo, hi) per B axis
  o = align16(o + 8 * 3 * mA);
  L.warp_bytes = o;
  return L;
}

// Bytes of one warp's node-pair stack: stack_cap (A node, B node) entries, then the lower
// bound of each entry (read by the proximity query when it pops or hands on an entry).
int64_t stack_stride(int stack_cap) { return ((int64_t)stack_cap * 12 + 15) & ~int64_t(15); }

// Stack bound: every level of the node-pair tree leaves at most (mA mB - 1) siblings.
// Pairs expanded together: as many A member sets as fill kMaxM rows, at most 4.
int joint_pairs(int mA) { return std::max(1, std::min(4, kMaxM / mA)); }
// Stack bound: every level of the node-pair tree leaves at most (E mA mB - 1) siblings, E
// pairs being expanded together.
int stack_bound(const cbvh_bvh *A, const cbvh_bvh *B, int E) {
  return 1 + (A->depth + B->depth + 1) * (E * A->m * B->m - 1);
}

// mode 0: collision detection (node pairs sharing a B node expanded together); 1: proximity
// query (one pair at a time: its most promising pair goes on top of the stack and is
// expanded next, which joint expansion would dilute -- measured slower on the terrain).
Layout make_layout(const cbvh_bvh *A, const cbvh_bvh *B, int mode) {
  const int E = mode == 0 ? joint_pairs(A->m) : 1;
  Layout L = warp_layout(A->K, A->max_tdepth, B->max_tdepth, stack_bound(A, B, E), E * A->m, B->m);
  L.E = E;
  // CTA region: the leading treelets of A and B that fit the staging budget
  int o = 0;
  const cbvh_bvh *H[2] = {A, B};
  const int budget = g_stage_bytes.load();
  for (int k = 0; k < 2; ++k) {
    const uint8_t *b = H[k]->blob.data();
    auto toff = [&](int64_t t) {
      uint64_t v;
      std::memcpy(&v, b + 64 + 8 * t, 8);
      return (int64_t)v;
    };
    int cnt = 0;
    while (cnt < H[k]->n_treelets && toff(cnt + 1) - toff(0) <= budget) ++cnt;
    L.st_cnt[k] = cnt;
    L.st_bytes[k] = (int)(toff(cnt) - toff(0));
    L.st_off[k] = o;
    o += (L.st_bytes[k] + 127) & ~127;
  }
  for (int k = 0; k < 2; ++k) {
    L.st_toff[k] = o;
    o = align16(o + 8 * (L.st_cnt[k] + 1));
  }
  L.o_bar = o;
  o = align16(o + 8);
  L.cta_bytes = (o + 127) & ~127;
  return L;
}

int cuda_fail(cudaError_t e, const char *what) {
  return cbvh::fail(CBVH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Optional per-thread profiling of the traversal launches: an event pair is recorded around
// each launch on its stream and summed by cbvh_profile_collect.
struct ProfRec {
  cudaEvent_t a, b;
  int mode;
};
struct Profiler {
  bool on = false;
  std::vector<ProfRec> used, spare;
};
thread_local Profiler g_prof;

// Rounds of a query and the expansion budget of a task in each (0 = none, last round).
constexpr int kRounds = 6;
constexpr int kBudget[kRounds] = {16, 32, 64, 128, 512, 0};
// Early-exit collision queries stop a pose at its first hit; tasks handed on before then
// waste work, so their budgets start high enough for most poses to finish in round 0.
constexpr int kBudgetEarly[kRounds] = {4096, 8192, 16384, 32768, 65536, 0};
constexpr int kMaxWarpsPerSM = 64;

// Workspace layout: [0, 256) counters -- u64 pair count at 0, u64 stats[3] at 16, then the
// 24 u32 counters of pass 0 at 64 and of pass 1 at 160 (see launch_rounds) -- then the
// per-pose pair counts and (pose, i, j) triples (collide with pairs), per-pose intersection
// flags (distance), two task buffers, the ready flags of a queue round and the per-warp
// stacks.
constexpr int64_t kWsHeader = 256;
struct WsPlan {
  int64_t counts, triples, flags, tasks0, tasks1, ready, stacks, total;
  uint32_t task_cap;
  int warps_max;
};
int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }
// Entries of each task buffer.  A round whose buffer fills up stops handing tasks on, and
// the tasks that could not hand off then run to the end on one warp: measured on an arm
// link over the terrain (4,096 poses), 1M entries filled in three rounds and the query ran
// 4x slower than with room to spare.
int64_t task_capacity(int64_t n) {
  return std::min<int64_t>(std::max<int64_t>(int64_t(1) << 22, 512 * n), int64_t(1) << 28);
}
WsPlan ws_plan(const Layout &L, int64_t n, int mode, int64_t cap, int sms) {
  WsPlan w;
  int64_t o = kWsHeader;
  w.counts = o;
  if (mode == 0) o = align256(o + 4 * n);
  w.triples = o;
  if (mode == 0) o = align256(o + 12 * std::max<int64_t>(cap, 0));
  w.flags = o;
  if (mode == 1) o = align256(o + n);
  const int64_t tcap = task_capacity(n);
  w.task_cap = (uint32_t)tcap;
  w.tasks0 = o;
  o = align256(o + 16 * tcap);
  w.tasks1 = o;
  o = align256(o + 16 * tcap);
  w.ready = o;
  o = align256(o + 4 * tcap);
  w.warps_max = sms * kMaxWarpsPerSM;
  w.stacks = o;
  o = align256(o + (int64_t)w.warps_max * stack_stride(L.stack_cap));
  w.total = o;
  return w;
}

int device_sms(int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  return e == cudaSuccess ? CBVH_OK : cuda_fail(e, "device query");
}

// The traversal kernel compiled for A's number of slab directions (k = 6, 18, 24, 26).
typedef void (*TraverseFn)(const Params);
// var: a Stream VByte hierarchy takes part (single queries only; batches refuse them);
// lat: both hierarchies store 8- or 16-bit deltas (single queries).
template <int MODE, bool BATCH, bool VAR, bool LAT>
TraverseFn traverse_fn_b(int K) {
  switch (K) {
    case 3: return traverse_kernel<MODE, 3, BATCH, VAR, LAT>;
    case 9: return traverse_kernel<MODE, 9, BATCH, VAR, LAT>;
    case 12: return traverse_kernel<MODE, 12, BATCH, VAR, LAT>;
    default: return traverse_kernel<MODE, 13, BATCH, VAR, LAT>;
  }
}
template <int MODE>
TraverseFn traverse_fn(int K, bool batch, bool var, bool lat) {
  if (batch) return traverse_fn_b<MODE, true, false, false>(K);
  if (var) return traverse_fn_b<MODE, false, true, false>(K);
  return lat ? traverse_fn_b<MODE, false, false, true>(K) : traverse_fn_b<MODE, false, false, false>(K);
}
bool delta_bits(int bits) { return bits == 8 || bits == 16; }

// Launches one traversal pass.  ctr: 24 zeroed u32 counters -- [0, 8) the task cursor of
// each round, [8, 16) the task count of each round, [16, 24) the work-queue counters; buf:
// the two task buffers; ready: task_cap u32 ready flags of a queue round; stacks: per-warp
// stacks.  The work mapping (CBVH_OPT_SPLIT) decides the rounds:
//   0: one round, one warp per pose to the end;
//   1: kRounds rounds with budgets; a task over its budget hands its stack to the next
//      round, the last round runs every task to the end;
//   2: one queue round: warps take poses, then tasks that busy warps donate from the
//      bottom of their stacks while other warps wait (work donation);
//   3: the first kRounds - 1 rounds as in 1, then a queue round over the tasks they handed
//      on;
//   4 (default): 2 for collision with pair lists, 3 for early-exit collision and for
//      distance.  Measured on the terrain, the arm sweep, the clutter and the 10M-triangle
//      sphere field: the queue is 11% faster for full collision (terrain 67.6 ms against
//      75.8 ms: every hand-off restarts decode chains), rounds are 3% faster for the
//      early-exit arm sweep, and distances converge faster when rounds explore the
//      subtrees a pose handed on side by side (sphere field 596 ms against 860 ms).
// max_blocks: an upper bound on the grid (the allocation-free query has stacks for fewer
// warps than the GPU holds).
template <int MODE>
int launch_rounds(Params &p, unsigned int *ctr, uint4 *buf0, uint4 *buf1, uint32_t *ready, uint2 *stacks,
                  uint32_t task_cap, int sms, cudaStream_t s, int slot = MODE, bool early_all = false,
                  int64_t max_blocks = INT32_MAX) {
  const int smem = p.L.cta_bytes + kWarpsPerBlock * p.L.warp_bytes;
  const TraverseFn fn =
      traverse_fn<MODE>(p.A.K, p.items != nullptr, p.A.bits == CBVH_QUANT_SVB || p.B.bits == CBVH_QUANT_SVB,
                        delta_bits(p.A.bits) && delta_bits(p.B.bits));
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  if (per_sm < 1) return cbvh::fail(CBVH_ERR_ARG, "traversal state does not fit in shared memory");
  per_sm = std::min(per_sm, kMaxWarpsPerSM / kWarpsPerBlock);
  const int blocks = (int)std::min<int64_t>((int64_t)sms * per_sm, max_blocks);
  uint4 *buf[2] = {buf0, buf1};
  p.stacks = stacks;
  p.task_cap = task_cap;
  ProfRec rec{nullptr, nullptr, slot};
  if (g_prof.on) {
    if (!g_prof.spare.empty()) {
      rec = g_prof.spare.back();
      g_prof.spare.pop_back();
      rec.mode = slot;
    } else if (cudaEventCreate(&rec.a) != cudaSuccess || cudaEventCreate(&rec.b) != cudaSuccess) {
      return cbvh::fail(CBVH_ERR_CUDA, "cudaEventCreate");
    }
    cudaEventRecord(rec.a, s);
  }
  int split = g_split.load();
  if (split == 4) split = (MODE == MODE_CD && !early_all) ? 2 : 3;
  const int rounds = split == 0 ? 1 : (split == 2 ? 1 : kRounds);
  for (int r = 0; r < rounds; ++r) {
    const bool queue_round = (split == 2) || (split == 3 && r == rounds - 1);
    p.round = r;
    p.last_round = r == rounds - 1;
    p.budget = early_all ? kBudgetEarly[r] : (kBudget[r] / 16) * g_budget0.load();
    p.task_next = ctr + r;
    p.count_in = ctr + 8 + r;
    p.count_out = ctr + 8 + r + 1;
    p.tasks_in = buf[(r + 1) & 1];
    p.tasks_out = buf[r & 1];
    p.queue = 0;
    if (queue_round) {
      // the queue lives in this round's output buffer; budget = expansions before donating
      p.queue = 1;
      p.task_next = ctr + 16;
      p.ready = ready;
      p.budget = early_all ? kBudgetEarly[0] : g_budget0.load();
      e = cudaMemsetAsync(ready, 0, 4 * (size_t)task_cap, s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    fn<<<blocks, kThreads, smem, s>>>(p);
    g_launches.fetch_add(1);
  }
  e = cudaGetLastError();
  if (g_prof.on) {
    cudaEventRecord(rec.b, s);
    g_prof.used.push_back(rec);
  }
  if (e != cudaSuccess) return cuda_fail(e, "traverse launch");
  return CBVH_OK;
}

// Single query: the 24 counters of pass k (0 or 1) at ws + 64 + 96 k, buffers and stacks
// from the plan.
template <int MODE>
int launch_single(Params &p, uint8_t *ws, const WsPlan &w, int sms, cudaStream_t s, int pass = 0, int slot = MODE) {
  const bool early = MODE == MODE_CD && (p.flags & CBVH_EARLY_EXIT);
  return launch_rounds<MODE>(p, reinterpret_cast<unsigned int *>(ws + 64 + 96 * pass),
                             reinterpret_cast<uint4 *>(ws + w.tasks0), reinterpret_cast<uint4 *>(ws + w.tasks1),
                             reinterpret_cast<uint32_t *>(ws + w.ready), reinterpret_cast<uint2 *>(ws + w.stacks),
                             w.task_cap, sms, s, slot, early);
}

int check_pair(const cbvh_bvh *A, const cbvh_bvh *B) {
  if (!A || !B) return cbvh::fail(CBVH_ERR_ARG, "NULL handle");
  if (!A->dev_blob || !B->dev_blob) return cbvh::fail(CBVH_ERR_STATE, "handle has no device blob; call cbvh_attach");
  if (!A->geometry || !B->geometry)
    return cbvh::fail(CBVH_ERR_STATE, "hierarchy has no geometry (a plan before a successful cbvh_build_device)");
  return CBVH_OK;
}

void fill_params(Params &p, const cbvh_bvh *A, const cbvh_bvh *B, int mode) {
  std::memset(&p, 0, sizeof p);
  p.A = view(A);
  p.B = view(B);
  p.L = make_layout(A, B, mode);
  p.wait_cap = g_wait_cap.load();
  for (int j = 0; j < kMaxK; ++j) {
    static const int n2[kMaxK] = {1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3};
    float f = (float)(1.0 / std::sqrt((double)n2[j]));
    while ((double)f * (double)f * n2[j] > 1.0) f = std::nextafter(f, 0.0f);
    p.invn[j] = f;
  }
}

}  // namespace

extern "C" int cbvh_attach(cbvh_bvh *h, void *dev_blob, int64_t bytes, void *stream) {
  CBVH_RANGE("cbvh_attach");
  cbvh::clear_error();
  if (!h || !dev_blob) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (bytes < (int64_t)h->blob.size()) return cbvh::fail(CBVH_ERR_ARG, "device buffer smaller than the blob");
  if (h->host_stale)
    return cbvh::fail(CBVH_ERR_STATE, "host blob not updated by the device build (CBVH_BUILD_HOST_COPY not given)");
  if (reinterpret_cast<uintptr_t>(dev_blob) & 255) return cbvh::fail(CBVH_ERR_ARG, "device buffer not 256-byte aligned");
  cudaError_t e = cudaMemcpyAsync(dev_blob, h->blob.data(), h->blob.size(), cudaMemcpyHostToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  h->dev_blob = dev_blob;
  cudaGetDevice(&h->device);
  return CBVH_OK;
}

extern "C" int cbvh_decode_all(const cbvh_bvh *h, int32_t *lattice_out, float *bounds_out, void *stream) {
  CBVH_RANGE("cbvh_decode_all");
  cbvh::clear_error();
  if (!h) return cbvh::fail(CBVH_ERR_ARG, "NULL handle");
  if (!h->dev_blob) return cbvh::fail(CBVH_ERR_STATE, "handle has no device blob; call cbvh_attach");
  decode_all_kernel<<<(unsigned)h->n_treelets, 128, 0, static_cast<cudaStream_t>(stream)>>>(view(h), lattice_out,
                                                                                             bounds_out);
  g_launches.fetch_add(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBVH_OK : cuda_fail(e, "decode launch");
}

extern "C" int cbvh_workspace_bytes(const cbvh_bvh *A, const cbvh_bvh *B, int64_t n, int mode, int64_t cap,
                                    int64_t *bytes) {
  cbvh::clear_error();
  if (!A || !B || !bytes || n < 0 || (mode != 0 && mode != 1)) return cbvh::fail(CBVH_ERR_ARG, "bad argument");
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  *bytes = ws_plan(make_layout(A, B, mode), n, mode, cap, sms).total;
  return CBVH_OK;
}

extern "C" int cbvh_collide(const cbvh_bvh *A, const cbvh_bvh *B, const float *poses, int64_t n, uint8_t *hit,
                            int64_t *pair_offsets, int32_t *pairs, int64_t pair_capacity, int64_t *pairs_needed,
                            uint32_t flags, void *workspace, int64_t workspace_bytes, int32_t *status,
                            void *stream) {
  CBVH_RANGE("cbvh_collide");
  cbvh::clear_error();
  if (int rc = check_pair(A, B)) return rc;
  if (n < 0 || (n > 0 && (!poses || !hit)) || !status) return cbvh::fail(CBVH_ERR_ARG, "NULL or negative argument");
  if (n > 0x7fffffffll) return cbvh::fail(CBVH_ERR_ARG, "too many poses for one call");
  const bool want_pairs = pair_offsets != nullptr || pairs != nullptr;
  if (want_pairs && (!pair_offsets || !pairs || pair_capacity < 0))
    return cbvh::fail(CBVH_ERR_ARG, "pair_offsets and pairs must be given together");
  if (want_pairs && (flags & CBVH_EARLY_EXIT)) return cbvh::fail(CBVH_ERR_ARG, "CBVH_EARLY_EXIT returns no pairs");
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  Params p;
  fill_params(p, A, B, 0);
  const WsPlan w = ws_plan(p.L, n, 0, want_pairs ? pair_capacity : 0, sms);
  if (!workspace || workspace_bytes < w.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return cbvh::fail(CBVH_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  cudaError_t e = cudaMemsetAsync(ws, 0, kWsHeader, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (n == 0) {
    if (want_pairs) {
      e = cudaMemsetAsync(pair_offsets, 0, sizeof(int64_t), s);
      if (e == cudaSuccess && pairs_needed) e = cudaMemsetAsync(pairs_needed, 0, sizeof(int64_t), s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    return CBVH_OK;
  }
  // only the flags are asked for: each pose can stop at its first intersecting pair
  if (!want_pairs) flags |= CBVH_EARLY_EXIT;
  p.poses = poses;
  p.n = n;
  p.hit = hit;
  p.flags = flags;
  p.status = status;
  p.pair_count = reinterpret_cast<unsigned long long *>(ws);
  p.stats = reinterpret_cast<unsigned long long *>(ws + 16);
  uint32_t *counts = reinterpret_cast<uint32_t *>(ws + w.counts);
  uint32_t *triples = reinterpret_cast<uint32_t *>(ws + w.triples);
  if (want_pairs) {
    p.counts = counts;
    p.triples = triples;
    p.cap = (unsigned long long)pair_capacity;
  }
  if (int rc = launch_single<MODE_CD>(p, ws, w, sms, s)) return rc;
  if (want_pairs) {
    ProfRec rec{nullptr, nullptr, 2};
    if (g_prof.on) {
      if (!g_prof.spare.empty()) {
        rec = g_prof.spare.back();
        g_prof.spare.pop_back();
        rec.mode = 2;
      } else if (cudaEventCreate(&rec.a) != cudaSuccess || cudaEventCreate(&rec.b) != cudaSuccess) {
        return cbvh::fail(CBVH_ERR_CUDA, "cudaEventCreate");
      }
      cudaEventRecord(rec.a, s);
    }
    scan_kernel<<<1, 1024, 0, s>>>(counts, n, pair_offsets, pairs_needed, p.cap, status);
    scatter_kernel<<<1024, 256, 0, s>>>(triples, p.pair_count, p.cap, pair_offsets, counts, pairs);
    g_launches.fetch_add(2);
    if (flags & CBVH_SORT_PAIRS) {
      sort_kernel<<<(unsigned)std::min<int64_t>(n, 65535), 256, 0, s>>>(
          pair_offsets, n, p.pair_count, p.cap, pairs, reinterpret_cast<unsigned long long *>(triples));
      g_launches.fetch_add(1);
    }
    e = cudaGetLastError();
    if (g_prof.on) {
      cudaEventRecord(rec.b, s);
      g_prof.used.push_back(rec);
    }
    if (e != cudaSuccess) return cuda_fail(e, "compaction launch");
  }
  return CBVH_OK;
}

extern "C" int cbvh_distance(const cbvh_bvh *A, const cbvh_bvh *B, const float *poses, int64_t n, float *dist,
                             void *workspace, int64_t workspace_bytes, int32_t *status, void *stream) {
  CBVH_RANGE("cbvh_distance");
  cbvh::clear_error();
  if (int rc = check_pair(A, B)) return rc;
  if (n < 0 || (n > 0 && (!poses || !dist)) || !status) return cbvh::fail(CBVH_ERR_ARG, "NULL or negative argument");
  if (n > 0x7fffffffll) return cbvh::fail(CBVH_ERR_ARG, "too many poses for one call");
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  Params p;
  fill_params(p, A, B, 1);
  const WsPlan w = ws_plan(p.L, n, 1, 0, sms);
  if (!workspace || workspace_bytes < w.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return cbvh::fail(CBVH_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  cudaError_t e = cudaMemsetAsync(ws, 0, kWsHeader, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (n == 0) return CBVH_OK;
  // Pass 1: collision detection with early exit marks the poses whose distance is 0.
  // Pass 2: branch and bound on the others.  Distance 0 iff the meshes intersect, and both
  // passes decide intersection with the same triangle test, so the result is that of a
  // single branch-and-bound pass; pass 1 only finds the zeros sooner.
  Params q = p;
  q.poses = poses;
  q.n = n;
  q.hit = ws + w.flags;
  q.flags = CBVH_EARLY_EXIT;
  q.status = status;
  q.pair_count = reinterpret_cast<unsigned long long *>(ws);
  q.stats = reinterpret_cast<unsigned long long *>(ws + 16);
  if (int rc = launch_single<MODE_CD>(q, ws, w, sms, s, 0, 1)) return rc;
  p.poses = poses;
  p.n = n;
  p.dist = dist;
  p.status = status;
  p.skip = ws + w.flags;
  p.stats = reinterpret_cast<unsigned long long *>(ws + 16);
  return launch_single<MODE_PQ>(p, ws, w, sms, s, 1);
}

extern "C" int cbvh_query_stats(const void *workspace, int64_t *stats_host, void *stream) {
  cbvh::clear_error();
  if (!workspace || !stats_host) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(stats_host, static_cast<const uint8_t *>(workspace) + 16, 3 * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? CBVH_OK : cuda_fail(e, "cbvh_query_stats");
}

extern "C" int cbvh_profile_enable(int on) {
  cbvh::clear_error();
  g_prof.on = on != 0;
  return CBVH_OK;
}

extern "C" int cbvh_profile_collect(double *ms_host, int64_t *launches_host) {
  cbvh::clear_error();
  if (!ms_host || !launches_host) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  ms_host[0] = ms_host[1] = ms_host[2] = 0.0;
  launches_host[0] = launches_host[1] = launches_host[2] = 0;
  int rc = CBVH_OK;
  for (auto &r : g_prof.used) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) rc = cuda_fail(e, "cbvh_profile_collect");
    ms_host[r.mode] += ms;
    launches_host[r.mode] += 1;
    g_prof.spare.push_back(r);
  }
  g_prof.used.clear();
  return rc;
}

// ---------------------------------------------------------------- distance without allocation
// Scratch of cbvh_distance_noalloc, in one fixed array that every GPU loading this library
// holds until the process exits: the counters of both passes, the intersection flags of one
// chunk of poses, the two task buffers with the ready flags of a work-queue round, and the
// per-warp stacks.  Calls share it, so calls that overlap on the GPU race.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr uint32_t kNoAllocTasks = 1u << 20;               // entries per task buffer
constexpr int64_t kNoAllocChunk = int64_t(1) << 14;        // poses per chunk (one flag byte each)
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_addr[1024] = {};

// Device address of the scratch array on the current device, looked up once per device.
int noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 1024) return cbvh::fail(CBVH_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return CBVH_OK;
}
}  // namespace

extern "C" int cbvh_distance_noalloc(const cbvh_bvh *A, const cbvh_bvh *B, const float *poses, int64_t n, float *dist,
                                     int32_t *status, void *stream) {
  CBVH_RANGE("cbvh_distance_noalloc");
  cbvh::clear_error();
  if (int rc = check_pair(A, B)) return rc;
  if (n < 0 || (n > 0 && (!poses || !dist)) || !status) return cbvh::fail(CBVH_ERR_ARG, "NULL or negative argument");
  if (n > 0x7fffffffll) return cbvh::fail(CBVH_ERR_ARG, "too many poses for one call");
  void *scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  Params p;
  fill_params(p, A, B, 1);
  // carve the fixed array: counters, the chunk's flags, two task buffers, the ready flags,
  // then as many warp stacks as fit
  const int64_t o_flags = kWsHeader;
  const int64_t o_tasks0 = align256(o_flags + kNoAllocChunk);
  const int64_t o_tasks1 = align256(o_tasks0 + 16 * (int64_t)kNoAllocTasks);
  const int64_t o_ready = align256(o_tasks1 + 16 * (int64_t)kNoAllocTasks);
  const int64_t o_stacks = align256(o_ready + 4 * (int64_t)kNoAllocTasks);
  const int64_t per_warp = stack_stride(p.L.stack_cap);
  const int64_t warps_fit = ((int64_t)kNoAllocScratchBytes - o_stacks) / per_warp;
  if (warps_fit < kWarpsPerBlock)
    return cbvh::fail(CBVH_ERR_WORKSPACE,
                      "this pair of hierarchies needs " + std::to_string(per_warp * kWarpsPerBlock + o_stacks) +
                          " bytes of scratch; cbvh_distance_noalloc has " + std::to_string(kNoAllocScratchBytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t *ws = static_cast<uint8_t *>(scratch);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  uint4 *t0 = reinterpret_cast<uint4 *>(ws + o_tasks0), *t1 = reinterpret_cast<uint4 *>(ws + o_tasks1);
  uint32_t *rdy = reinterpret_cast<uint32_t *>(ws + o_ready);
  uint2 *st = reinterpret_cast<uint2 *>(ws + o_stacks);
  const int64_t max_blocks = warps_fit / kWarpsPerBlock;
  // the two passes of cbvh_distance with its schedule, chunk by chunk
  for (int64_t off = 0; off < n; off += kNoAllocChunk) {
    const int64_t cnt = std::min(kNoAllocChunk, n - off);
    // the counters of both passes must start at zero; everything else is written before read
    e = cudaMemsetAsync(ws, 0, kWsHeader, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    Params q = p;
    q.poses = poses + 12 * off;
    q.n = cnt;
    q.hit = ws + o_flags;
    q.flags = CBVH_EARLY_EXIT;
    q.status = status;
    q.pair_count = reinterpret_cast<unsigned long long *>(ws);
    q.stats = reinterpret_cast<unsigned long long *>(ws + 16);
    if (int rc = launch_rounds<MODE_CD>(q, reinterpret_cast<unsigned int *>(ws + 64), t0, t1, rdy, st, kNoAllocTasks,
                                        sms, s, 1, true, max_blocks))
      return rc;
    Params r = p;
    r.poses = poses + 12 * off;
    r.n = cnt;
    r.dist = dist + off;
    r.status = status;
    r.skip = ws + o_flags;
    r.stats = reinterpret_cast<unsigned long long *>(ws + 16);
    if (int rc = launch_rounds<MODE_PQ>(r, reinterpret_cast<unsigned int *>(ws + 160), t0, t1, rdy, st, kNoAllocTasks,
                                        sms, s, MODE_PQ, false, max_blocks))
      return rc;
  }
  return CBVH_OK;
}

// ---------------------------------------------------------------- batched queries
// A batch is a list of work items (A, B, kind, poses, outputs).  Items are grouped by kind and
// by A's direction count; each group runs as one pass of persistent rounds over all of its
// poses (two passes for distances: the early-exit collision pass, then branch and bound), so
// pairs of hierarchies of different sizes share the GPU and a heavy item spreads over all
// warps.  Upload writes the item table into the workspace; launch only enqueues kernels and
// memsets, so it can be captured in a CUDA graph and replayed.
struct cbvh_batch {
  struct Group {
    int mode, first, count, pre_first;
    int64_t poses, bases_at, skip_off;
    Layout L;
    BVd A0, B0;
  };
  std::vector<BatchItem> items;
  std::vector<unsigned long long> bases;
  std::vector<std::pair<uint8_t *, int64_t>> any_hit;  // distinct per-set flag arrays, cleared at launch
  std::vector<std::pair<float *, int64_t>> min_dist;   // distinct per-set distance arrays, reset at launch
  std::vector<Group> groups;
  int64_t o_ctr = 0, o_items = 0, o_bases = 0, o_tasks0 = 0, o_tasks1 = 0, o_ready = 0, o_stacks = 0, total = 0;
  uint32_t task_cap = 0;
  int sms = 0;
};

extern "C" int cbvh_batch_create(const cbvh_query_t *q, int64_t nq, cbvh_batch **out) {
  cbvh::clear_error();
  if (!out || (nq > 0 && !q) || nq < 0) return cbvh::fail(CBVH_ERR_ARG, "bad argument");
  *out = nullptr;
  for (int64_t i = 0; i < nq; ++i) {
    const cbvh_query_t &x = q[i];
    if (int rc = check_pair(x.A, x.B)) return rc;
    if (x.A->bits == CBVH_QUANT_SVB || x.B->bits == CBVH_QUANT_SVB)
      return cbvh::fail(CBVH_ERR_ARG, "batches need fixed-size records (quant_bits 0, 1, 8 or 16)");
    if ((x.mode != 0 && x.mode != 1) || x.n < 0 || (x.n > 0 && !x.poses))
      return cbvh::fail(CBVH_ERR_ARG, "query " + std::to_string(i) + ": bad mode, size or poses");
    if (x.n > 0 && ((x.mode == 0 && !x.hit) || (x.mode == 1 && !x.dist)))
      return cbvh::fail(CBVH_ERR_ARG, "query " + std::to_string(i) + ": missing output");
    if (x.mode == 1 && x.flags) return cbvh::fail(CBVH_ERR_ARG, "query " + std::to_string(i) + ": flags are for collision");
    if (x.flags & ~CBVH_EARLY_EXIT) return cbvh::fail(CBVH_ERR_ARG, "query " + std::to_string(i) + ": unknown flags");
    if (x.any_hit && x.mode != 0)
      return cbvh::fail(CBVH_ERR_ARG, "query " + std::to_string(i) + ": any_hit is for collision queries");
    if (x.min_dist && x.mode != 1)
      return cbvh::fail(CBVH_ERR_ARG, "query " + std::to_string(i) + ": min_dist is for distance queries");
    for (int64_t k = 0; k < i; ++k)
      if ((x.any_hit && q[k].any_hit == x.any_hit && q[k].n != x.n) ||
          (x.min_dist && q[k].min_dist == x.min_dist && q[k].n != x.n))
        return cbvh::fail(CBVH_ERR_ARG, "queries " + std::to_string(k) + " and " + std::to_string(i) +
                                            " share a set's array but differ in pose count");
  }
  auto b = new cbvh_batch();
  if (int rc = device_sms(&b->sms)) {
    delete b;
    return rc;
  }
  int64_t total_poses = 0, max_group = 0;
  int max_stack = 1;
  for (int mode = 0; mode < 2; ++mode)
    for (int K : {3, 9, 12, 13}) {
      std::vector<int64_t> idx;
      for (int64_t i = 0; i < nq; ++i)
        if (q[i].mode == mode && q[i].A->K == K) idx.push_back(i);
      if (idx.empty()) continue;
      cbvh_batch::Group g;
      g.mode = mode;
      g.first = (int)b->items.size();
      g.count = (int)idx.size();
      g.bases_at = (int64_t)b->bases.size();
      int tdA = 0, tdB = 0, sc = 1, mA = 2, mB = 2;
      for (int64_t i : idx) mA = std::max(mA, q[i].A->m);
      const int E = mode == 0 ? joint_pairs(mA) : 1;
      unsigned long long acc = 0;
      for (int64_t i : idx) {
        const cbvh_query_t &x = q[i];
        BatchItem it;
        std::memset(&it, 0, sizeof it);
        it.A = view(x.A);
        it.B = view(x.B);
        it.poses = x.poses;
        it.hit = x.hit;
        it.dist = x.dist;
        it.flags = x.mode == 0 ? (x.flags | CBVH_EARLY_EXIT) : 0;  // collision items return flags only
        it.any_hit = x.mode == 0 ? x.any_hit : nullptr;
        it.min_dist = x.mode == 1 ? x.min_dist : nullptr;
        b->items.push_back(it);
        b->bases.push_back(acc);
        acc += (unsigned long long)x.n;
        tdA = std::max(tdA, x.A->max_tdepth);
        tdB = std::max(tdB, x.B->max_tdepth);
        sc = std::max(sc, stack_bound(x.A, x.B, E));
        mB = std::max(mB, x.B->m);
      }
      b->bases.push_back(acc);
      g.poses = (int64_t)acc;
      g.L = warp_layout(K, tdA, tdB, sc, E * mA, mB);
      g.L.E = E;
      g.A0 = view(q[idx[0]].A);
      g.B0 = view(q[idx[0]].B);
      g.pre_first = -1;
      g.skip_off = -1;
      max_stack = std::max(max_stack, sc);
      max_group = std::max(max_group, g.poses);
      total_poses += g.poses;
      b->groups.push_back(g);
    }
  // distance groups also get a collision item table for their early-exit pass
  for (auto &g : b->groups) {
    if (g.mode != 1) continue;
    g.pre_first = (int)b->items.size();
    for (int k = 0; k < g.count; ++k) {
      BatchItem it = b->items[g.first + k];
      it.dist = nullptr;
      it.hit = nullptr;  // set at upload: the group's intersection flags + item base
      it.flags = CBVH_EARLY_EXIT;
      it.any_hit = nullptr;
      it.min_dist = nullptr;
      b->items.push_back(it);
    }
  }
  for (int64_t i = 0; i < nq; ++i) {
    if (q[i].n == 0) continue;
    bool seen = false;
    if (q[i].any_hit) {
      for (const auto &a : b->any_hit) seen |= a.first == q[i].any_hit;
      if (!seen) b->any_hit.emplace_back(q[i].any_hit, q[i].n);
    }
    seen = false;
    if (q[i].min_dist) {
      for (const auto &a : b->min_dist) seen |= a.first == q[i].min_dist;
      if (!seen) b->min_dist.emplace_back(q[i].min_dist, q[i].n);
    }
  }
  // workspace plan
  int64_t o = kWsHeader;
  b->o_ctr = o;  // per group: 24 counters of the collision pass, then 24 of the distance pass
  o = align256(o + 256 * (int64_t)b->groups.size());
  b->o_items = o;
  o = align256(o + (int64_t)sizeof(BatchItem) * (int64_t)b->items.size());
  b->o_bases = o;
  o = align256(o + 8 * (int64_t)b->bases.size());
  for (auto &g : b->groups)
    if (g.mode == 1) {
      g.skip_off = o;
      o = align256(o + g.poses);
    }
  const int64_t tcap = task_capacity(max_group);
  b->task_cap = (uint32_t)tcap;
  b->o_tasks0 = o;
  o = align256(o + 16 * tcap);
  b->o_tasks1 = o;
  o = align256(o + 16 * tcap);
  b->o_ready = o;
  o = align256(o + 4 * tcap);
  b->o_stacks = o;
  o = align256(o + (int64_t)b->sms * kMaxWarpsPerSM * stack_stride(max_stack));
  b->total = o;
  (void)total_poses;
  *out = b;
  return CBVH_OK;
}

extern "C" int cbvh_batch_free(cbvh_batch *b) {
  delete b;
  return CBVH_OK;
}

extern "C" int cbvh_batch_workspace_bytes(const cbvh_batch *b, int64_t *bytes) {
  cbvh::clear_error();
  if (!b || !bytes) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  *bytes = b->total;
  return CBVH_OK;
}

extern "C" int cbvh_batch_upload(const cbvh_batch *b, void *workspace, int64_t workspace_bytes, void *stream) {
  CBVH_RANGE("cbvh_batch_upload");
  cbvh::clear_error();
  if (!b) return cbvh::fail(CBVH_ERR_ARG, "NULL batch");
  if (!workspace || workspace_bytes < b->total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return cbvh::fail(CBVH_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  std::vector<BatchItem> items = b->items;
  for (const auto &g : b->groups)
    if (g.mode == 1)
      for (int k = 0; k < g.count; ++k)
        items[g.pre_first + k].hit = ws + g.skip_off + b->bases[g.bases_at + k];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(ws + b->o_items, items.data(), sizeof(BatchItem) * items.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + b->o_bases, b->bases.data(), 8 * b->bases.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? CBVH_OK : cuda_fail(e, "cbvh_batch_upload");
}

extern "C" int cbvh_batch_launch(const cbvh_batch *b, void *workspace, int64_t workspace_bytes, int32_t *status,
                                 void *stream) {
  CBVH_RANGE("cbvh_batch_launch");
  cbvh::clear_error();
  if (!b || !status) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (!workspace || workspace_bytes < b->total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return cbvh::fail(CBVH_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, b->o_items, s);  // header and round counters
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  for (const auto &a : b->any_hit)
    if (e == cudaSuccess) e = cudaMemsetAsync(a.first, 0, (size_t)a.second, s);
  // 0x7f7f7f7f = 3.4e38: larger than any distance, and below +inf under the unsigned
  // ordering that atomicMin applies to non-negative floats
  for (const auto &a : b->min_dist)
    if (e == cudaSuccess) e = cudaMemsetAsync(a.first, 0x7f, 4 * (size_t)a.second, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const BatchItem *dev_items = reinterpret_cast<const BatchItem *>(ws + b->o_items);
  const unsigned long long *dev_bases = reinterpret_cast<const unsigned long long *>(ws + b->o_bases);
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const auto &g = b->groups[gi];
    if (g.poses == 0) continue;
    Params p;
    std::memset(&p, 0, sizeof p);
    p.A = g.A0;
    p.B = g.B0;
    p.L = g.L;
    p.wait_cap = g_wait_cap.load();
    for (int j = 0; j < kMaxK; ++j) {
      static const int n2[kMaxK] = {1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3};
      float f = (float)(1.0 / std::sqrt((double)n2[j]));
      while ((double)f * (double)f * n2[j] > 1.0) f = std::nextafter(f, 0.0f);
      p.invn[j] = f;
    }
    p.item_base = dev_bases + g.bases_at;
    p.n_items = g.count;
    p.n = g.poses;
    p.status = status;
    p.stats = reinterpret_cast<unsigned long long *>(ws + 16);
    p.pair_count = reinterpret_cast<unsigned long long *>(ws);
    unsigned int *ctr = reinterpret_cast<unsigned int *>(ws + b->o_ctr + 256 * (int64_t)gi);
    uint32_t *rdy = reinterpret_cast<uint32_t *>(ws + b->o_ready);
    uint4 *t0 = reinterpret_cast<uint4 *>(ws + b->o_tasks0), *t1 = reinterpret_cast<uint4 *>(ws + b->o_tasks1);
    uint2 *st = reinterpret_cast<uint2 *>(ws + b->o_stacks);
    if (g.mode == 0) {
      p.items = dev_items + g.first;
      bool all_early = true;
      for (int k = 0; k < g.count; ++k) all_early &= (b->items[g.first + k].flags & CBVH_EARLY_EXIT) != 0;
      if (int rc = launch_rounds<MODE_CD>(p, ctr, t0, t1, rdy, st, b->task_cap, b->sms, s, 0, all_early)) return rc;
    } else {
      Params c = p;
      c.items = dev_items + g.pre_first;
      if (int rc = launch_rounds<MODE_CD>(c, ctr, t0, t1, rdy, st, b->task_cap, b->sms, s, 1, true)) return rc;
      p.items = dev_items + g.first;
      p.skip = ws + g.skip_off;
      if (int rc = launch_rounds<MODE_PQ>(p, ctr + 32, t0, t1, rdy, st, b->task_cap, b->sms, s)) return rc;
    }
  }
  return CBVH_OK;
}

namespace cbvh {
void count_launches(int n) { g_launches.fetch_add(n); }
}  // namespace cbvh

extern "C" int cbvh_kernel_launches(int64_t *count) {
  cbvh::clear_error();
  if (!count) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  *count = g_launches.load();
  return CBVH_OK;
}

extern "C" int cbvh_set_option(int option, int64_t value) {
  cbvh::clear_error();
  if (option == CBVH_OPT_STAGE_BYTES) {
    if (value < 0 || value > 32768) return cbvh::fail(CBVH_ERR_ARG, "stage bytes must be in [0, 32768]");
    g_stage_bytes.store((int)value);
    return CBVH_OK;
  }
  if (option == CBVH_OPT_BUDGET0) {
    if (value < 1 || value > (1 << 20)) return cbvh::fail(CBVH_ERR_ARG, "budget must be in [1, 2^20]");
    g_budget0.store((int)value);
    return CBVH_OK;
  }
  if (option == CBVH_OPT_SPLIT) {
    if (value < 0 || value > 4) return cbvh::fail(CBVH_ERR_ARG, "split must be 0, 1, 2, 3 or 4");
    g_split.store((int)value);
    return CBVH_OK;
  }
  if (option == CBVH_OPT_WAIT_CAP) {
    if (value < 1 || value > kIdleSpin) return cbvh::fail(CBVH_ERR_ARG, "wait cap must be in [1, 2^24] polls");
    g_wait_cap.store(value);
    return CBVH_OK;
  }
  if (option == CBVH_OPT_LATTICE_HEADROOM) {
    if (value < 0 || value > 8) return cbvh::fail(CBVH_ERR_ARG, "lattice headroom must be in [0, 8] bits");
    cbvh::set_lattice_headroom((int)value);
    return CBVH_OK;
  }
  if (option == CBVH_OPT_TREELET_PACKING) {
    if (value != CBVH_PACK_TOP_DOWN && value != CBVH_PACK_BOTTOM_UP)
      return cbvh::fail(CBVH_ERR_ARG, "treelet packing must be CBVH_PACK_TOP_DOWN or CBVH_PACK_BOTTOM_UP");
    cbvh::set_treelet_packing((int)value);
    return CBVH_OK;
  }
  return cbvh::fail(CBVH_ERR_ARG, "unknown option");
}
