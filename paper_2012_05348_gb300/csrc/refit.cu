// Device-side refit of an attached hierarchy for deforming meshes: new positions for the
// build's vertices, the same tree, treelets and lattice exponent.  Every node's exact
// lattice bounds are recomputed from the new vertices and the blob's bound fields and
// triangle table are rewritten in place -- the same bytes the host encoder writes for this
// tree and these vertices (the predictor-corrector of the abstract and Sec. III-B, or the
// FP16 / FP32 absolute bounds).
//
// A one-time plan (cbvh_refit_prepare) turns the blob's treelet structure into per-node
// arrays in the caller's workspace: record offset, parent, leaf slot, depth in the tree and
// below the treelet root, and two node orders (by tree depth for the bottom-up bounds, by
// treelet depth for the top-down encoding).  Each refit is then a few kernels per level:
//   0. every vertex: exact floor / ceil of d_j . v / 2^e (Shewchuk's expansion arithmetic in
//      FP64, after a fast path that decides most cases from the rounded sum);
//   1. leaves: the interval over their triangle's three vertices, the new triangle into the
//      table;
//   2. every node, deepest level first: its bounds merged into its parent's by atomicMin /
//      atomicMax (a parent's level runs after all of its children's);
//   3. treelet depth 0, 1, ...: decoded interval from the parent's (correctors rounded
//      outward exactly as the encoder does), written into the record.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <vector>

#include "internal.h"
#include "lattice.cuh"

namespace {

// ---------------------------------------------------------------- outward roundings
// Largest half <= v (down) or smallest half >= v (up), IEEE binary16 bits, for finite v:
// v's binade quantum (2^-24 below 2^-14), floor or ceil of v / quantum.
__device__ uint16_t half_pos(double v, bool up) {
  if (v > 65504.0) return up ? 0x7c00u : 0x7bffu;
  int ex = 0;
  frexp(v, &ex);
  const int E = max(ex - 1, -14);
  const double quantum = ldexp(1.0, E - 10);
  long long qi = (long long)(up ? ceil(v / quantum) : floor(v / quantum));
  if (E == -14 && qi < 1024) return (uint16_t)qi;
  int ef = E + 15;
  if (qi == 2048) {
    qi = 1024;
    ++ef;
  }
  if (ef >= 31) return 0x7c00u;
  return (uint16_t)((ef << 10) | (int)(qi - 1024));
}
__device__ uint16_t half_down(double v) {
  if (v == 0.0) return 0;
  return v > 0 ? half_pos(v, false) : (uint16_t)(0x8000u | half_pos(-v, true));
}
__device__ uint16_t half_up(double v) {
  if (v == 0.0) return 0;
  return v > 0 ? half_pos(v, true) : (uint16_t)(0x8000u | half_pos(-v, false));
}
// FP32 image of a lattice integer rounded down / up, times 2^e (exact scaling).
__device__ __forceinline__ float f32_down(int L, float scale) { return __int2float_rd(L) * scale; }
__device__ __forceinline__ float f32_up(int L, float scale) { return __int2float_ru(L) * scale; }

__device__ __forceinline__ void set_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

struct RefitArgs {
  int32_t *VL;  // [n_verts][K][2] lattice interval of every vertex
  uint8_t *blob;
  int64_t off_tris;
  const float *verts;
  const int32_t *tris;
  int64_t n_verts, n_tris;
  int K, bits, e;
  float scale;  // 2^e
  const uint64_t *rec_off;  // [nn] byte offset of the node's record
  const int32_t *parent;    // [nn] blob-order index of the parent, -1 at the root
  const int32_t *leaf;      // [nn] leaf slot, -1 for inner nodes
  const int32_t *tdepth;    // [nn] depth below the treelet root
  const int32_t *order;     // nodes of the launch's level
  int64_t begin, end;
  int32_t *C;  // [nn][K][2] exact lattice bounds
  int32_t *D;  // [nn][K][2] decoded bounds
  int32_t *status;
};

// One thread per (vertex, direction): the vertex's lattice interval.  A vertex that is not
// finite fails the refit (the builder rejects such meshes); the range rule is applied by the
// leaves, to the vertices triangles use.
__global__ void vertex_lattice(const RefitArgs a) {
  const int64_t items = a.n_verts * a.K;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = it / a.K;
    const int j = (int)(it - v * a.K);
    const float p[3] = {a.verts[3 * v], a.verts[3 * v + 1], a.verts[3 * v + 2]};
    int32_t *out = a.VL + 2 * it;
    if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) {
      set_status(a.status, CBVH_ERR_MESH);
      out[0] = INT32_MAX;
      out[1] = INT32_MIN;
      continue;
    }
    long long lo, hi;
    lattice_of(p, j, a.e, lo, hi);
    // clamp to the int32 range; anything beyond the lattice's 2^30 fails at the leaf
    out[0] = (int32_t)max(min(lo, (long long)INT32_MAX), (long long)INT32_MIN);
    out[1] = (int32_t)max(min(hi, (long long)INT32_MAX), (long long)INT32_MIN);
  }
}

__global__ void init_bounds(int32_t *C, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    C[i] = (i & 1) ? INT32_MIN : INT32_MAX;
}

// One thread per (node, direction) of one tree level: a leaf's bounds from its triangle (and
// the new triangle into the table), then every node's bounds into its parent's.
__global__ void bounds_level(const RefitArgs a) {
  const int64_t items = (a.end - a.begin) * a.K;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = it / a.K;
    const int j = (int)(it - q * a.K);
    const int32_t n = a.order[a.begin + q];
    int32_t *Cn = a.C + ((int64_t)n * a.K + j) * 2;
    const int32_t slot = a.leaf[n];
    if (slot >= 0) {
      uint8_t *T = a.blob + a.off_tris + 48 * (int64_t)slot;
      const uint32_t tri = *reinterpret_cast<const uint32_t *>(T + 12);  // original triangle index
      long long lo = LLONG_MAX, hi = LLONG_MIN;
      bool bad = tri >= (uint64_t)a.n_tris;
      for (int c = 0; c < 3 && !bad; ++c) {
        const int32_t vi = a.tris[3 * (int64_t)tri + c];
        if (vi < 0 || vi >= a.n_verts) {
          bad = true;
          break;
        }
        const int32_t *L = a.VL + ((int64_t)vi * a.K + j) * 2;
        const long long l = L[0], h = L[1];
        if (l > kLatLimit - 1 || h < -(kLatLimit - 1)) bad = true;  // the builder's range rule
        lo = min(lo, l);
        hi = max(hi, h);
        if (j == 0) {
          float *dst = reinterpret_cast<float *>(T + 16 * c);
          dst[0] = a.verts[3 * (int64_t)vi];
          dst[1] = a.verts[3 * (int64_t)vi + 1];
          dst[2] = a.verts[3 * (int64_t)vi + 2];
        }
      }
      if (bad) {
        set_status(a.status, CBVH_ERR_MESH);
        continue;
      }
      Cn[0] = (int32_t)lo;
      Cn[1] = (int32_t)hi;
    }
    const int32_t par = a.parent[n];
    if (par >= 0) {
      int32_t *Cp = a.C + ((int64_t)par * a.K + j) * 2;
      atomicMin(Cp, Cn[0]);
      atomicMax(Cp + 1, Cn[1]);
    }
  }
}

// One thread per (node, direction) at one treelet depth: the decoded interval and the
// record's bound fields.
__global__ void encode_level(const RefitArgs a) {
  const int64_t items = (a.end - a.begin) * a.K;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = it / a.K;
    const int j = (int)(it - q * a.K);
    const int32_t n = a.order[a.begin + q];
    const int32_t *Cn = a.C + ((int64_t)n * a.K + j) * 2;
    int32_t *Dn = a.D + ((int64_t)n * a.K + j) * 2;
    uint8_t *R = a.blob + a.rec_off[n];
    const int lo = Cn[0], hi = Cn[1];
    if (a.bits == 0) {
      Dn[0] = lo;
      Dn[1] = hi;
      reinterpret_cast<float *>(R + 8 + 8 * j)[0] = f32_down(lo, a.scale);
      reinterpret_cast<float *>(R + 8 + 8 * j)[1] = f32_up(hi, a.scale);
    } else if (a.bits == CBVH_QUANT_FP16) {
      Dn[0] = lo;
      Dn[1] = hi;
      const double vl = ldexp((double)lo, a.e), vh = ldexp((double)hi, a.e);
      if (fabs(vl) > 65504.0 || fabs(vh) > 65504.0) set_status(a.status, CBVH_ERR_MESH);
      reinterpret_cast<uint16_t *>(R + 8 + 4 * j)[0] = half_down(vl);
      reinterpret_cast<uint16_t *>(R + 8 + 4 * j)[1] = half_up(vh);
    } else if (a.tdepth[n] == 0) {  // treelet root: absolute lattice values
      Dn[0] = lo;
      Dn[1] = hi;
      reinterpret_cast<int32_t *>(R + 8 + 8 * j)[0] = lo;
      reinterpret_cast<int32_t *>(R + 8 + 8 * j)[1] = hi;
    } else {  // corrector against the parent's decoded interval, rounded outward
      const int32_t *Pp = a.D + ((int64_t)a.parent[n] * a.K + j) * 2;
      const long long plo = Pp[0], phi = Pp[1];
      const uint32_t dmax = (1u << a.bits) - 1u;
      const uint32_t range = (uint32_t)(phi - plo);
      int s = 0;
      while ((range >> s) > dmax) ++s;
      const uint32_t dl = (uint32_t)((long long)lo - plo) >> s;
      const uint32_t dh = (uint32_t)(phi - (long long)hi) >> s;
      Dn[0] = (int32_t)(plo + ((long long)dl << s));
      Dn[1] = (int32_t)(phi - ((long long)dh << s));
      if (a.bits == 8) {
        R[8 + 2 * j] = (uint8_t)dl;
        R[9 + 2 * j] = (uint8_t)dh;
      } else {
        reinterpret_cast<uint16_t *>(R + 8 + 4 * j)[0] = (uint16_t)dl;
        reinterpret_cast<uint16_t *>(R + 8 + 4 * j)[1] = (uint16_t)dh;
      }
    }
  }
}

int cuda_fail(cudaError_t e, const char *what) {
  return cbvh::fail(CBVH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int64_t al256(int64_t x) { return (x + 255) & ~int64_t(255); }

// Byte offsets of the plan's arrays in the workspace.
struct RefitLayout {
  int64_t rec_off, parent, leaf, tdepth, by_level, by_td, C, D, VL, total;
};
RefitLayout refit_layout(const cbvh_bvh *h) {
  const int64_t nn = h->n_nodes;
  RefitLayout L;
  int64_t o = 0;
  L.rec_off = o;
  o = al256(o + 8 * nn);
  L.parent = o;
  o = al256(o + 4 * nn);
  L.leaf = o;
  o = al256(o + 4 * nn);
  L.tdepth = o;
  o = al256(o + 4 * nn);
  L.by_level = o;
  o = al256(o + 4 * nn);
  L.by_td = o;
  o = al256(o + 4 * nn);
  L.C = o;
  o = al256(o + 8 * nn * h->K);
  L.D = o;
  o = al256(o + 8 * nn * h->K);
  L.VL = o;
  o = al256(o + 8 * h->n_verts * h->K);
  L.total = o;
  return L;
}

uint32_t rd32(const std::vector<uint8_t> &b, int64_t o) {
  uint32_t v;
  std::memcpy(&v, &b[o], 4);
  return v;
}
uint64_t rd64(const std::vector<uint8_t> &b, int64_t o) {
  uint64_t v;
  std::memcpy(&v, &b[o], 8);
  return v;
}

}  // namespace

extern "C" int cbvh_refit_workspace_bytes(const cbvh_bvh *h, int64_t *bytes) {
  cbvh::clear_error();
  if (!h || !bytes) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  *bytes = refit_layout(h).total;
  return CBVH_OK;
}

extern "C" int cbvh_refit_prepare(cbvh_bvh *h, void *workspace, int64_t workspace_bytes, void *stream) {
  CBVH_RANGE("cbvh_refit_prepare");
  cbvh::clear_error();
  if (!h || !workspace) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (h->bits == CBVH_QUANT_SVB)  // a record's size follows its deltas: no re-encoding in place
    return cbvh::fail(CBVH_ERR_ARG, "refit needs fixed-size records (quant_bits 0, 1, 8 or 16)");
  const RefitLayout L = refit_layout(h);
  if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return cbvh::fail(CBVH_ERR_WORKSPACE, "refit workspace too small or not 256-byte aligned");
  // the node plan, from the blob's treelet structure (nodes numbered in blob order)
  const std::vector<uint8_t> &b = h->blob;
  const int64_t nn = h->n_nodes, ntl = h->n_treelets;
  std::vector<int64_t> first(ntl + 1), toff(ntl);
  int64_t acc = 0;
  for (int64_t t = 0; t < ntl; ++t) {
    toff[t] = (int64_t)rd64(b, 64 + 8 * t);
    first[t] = acc;
    acc += rd32(b, toff[t]);
  }
  first[ntl] = acc;
  if (acc != nn) return cbvh::fail(CBVH_ERR_STATE, "blob node count does not match the handle");
  std::vector<uint64_t> rec(nn);
  std::vector<int32_t> parent(nn, -1), leaf(nn, -1), tdep(nn, 0), depth(nn, 0);
  std::vector<uint32_t> w0s(nn), w1s(nn);
  for (int64_t t = 0; t < ntl; ++t)
    for (int64_t l = 0; l < first[t + 1] - first[t]; ++l) {
      const int64_t n = first[t] + l;
      rec[n] = (uint64_t)(toff[t] + 16 + (l ? h->root_bytes + (l - 1) * h->rec_bytes : 0));
      w0s[n] = rd32(b, (int64_t)rec[n]);
      w1s[n] = rd32(b, (int64_t)rec[n] + 4);
      tdep[n] = (int32_t)(w0s[n] >> 24);
    }
  // children and depths, breadth-first from the root (treelet 0, local 0)
  std::deque<int64_t> queue{0};
  int max_depth = 0;
  while (!queue.empty()) {
    const int64_t n = queue.front();
    queue.pop_front();
    const uint32_t nc = (w0s[n] >> 16) & 31u;
    const bool ext = (w0s[n] >> 21) & 1u;
    if (nc == 0) {
      leaf[n] = (int32_t)w1s[n];
      continue;
    }
    int64_t t = 0;
    if (!ext) t = std::upper_bound(first.begin(), first.end(), n) - first.begin() - 1;
    for (uint32_t c = 0; c < nc; ++c) {
      const int64_t ch = ext ? first[w1s[n] + c] : first[t] + w1s[n] + c;
      parent[ch] = (int32_t)n;
      depth[ch] = depth[n] + 1;
      max_depth = std::max(max_depth, depth[ch]);
      queue.push_back(ch);
    }
  }
  std::vector<int32_t> by_level(nn), by_td(nn);
  std::vector<int64_t> level_start(max_depth + 2, 0), td_start(h->max_tdepth + 2, 0);
  for (int64_t n = 0; n < nn; ++n) {
    ++level_start[depth[n] + 1];
    ++td_start[tdep[n] + 1];
  }
  for (size_t i = 1; i < level_start.size(); ++i) level_start[i] += level_start[i - 1];
  for (size_t i = 1; i < td_start.size(); ++i) td_start[i] += td_start[i - 1];
  {
    std::vector<int64_t> fl(level_start.begin(), level_start.end() - 1), ft(td_start.begin(), td_start.end() - 1);
    for (int64_t n = 0; n < nn; ++n) {
      by_level[fl[depth[n]]++] = (int32_t)n;
      by_td[ft[tdep[n]]++] = (int32_t)n;
    }
  }
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(ws + L.rec_off, rec.data(), 8 * nn, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.parent, parent.data(), 4 * nn, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.leaf, leaf.data(), 4 * nn, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.tdepth, tdep.data(), 4 * nn, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.by_level, by_level.data(), 4 * nn, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.by_td, by_td.data(), 4 * nn, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
  if (e != cudaSuccess) return cuda_fail(e, "refit plan upload");
  h->refit_level_start = level_start;
  h->refit_td_start = td_start;
  h->refit_ws = workspace;
  return CBVH_OK;
}

extern "C" int cbvh_refit(cbvh_bvh *h, const float *verts_dev, int64_t n_verts, const int32_t *tris_dev,
                          void *workspace, int64_t workspace_bytes, int32_t *status, void *stream) {
  CBVH_RANGE("cbvh_refit");
  cbvh::clear_error();
  if (!h || !verts_dev || !tris_dev || !status || !workspace) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (!h->dev_blob) return cbvh::fail(CBVH_ERR_STATE, "handle has no device blob; call cbvh_attach");
  if (h->refit_ws != workspace) return cbvh::fail(CBVH_ERR_STATE, "workspace not prepared; call cbvh_refit_prepare");
  const RefitLayout L = refit_layout(h);
  if (workspace_bytes < L.total) return cbvh::fail(CBVH_ERR_WORKSPACE, "refit workspace too small");
  if (n_verts != h->n_verts) return cbvh::fail(CBVH_ERR_ARG, "a refit needs the build's vertex count");
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  int launches = 0;
  const int rc = cbvh::refit_launch(h, verts_dev, tris_dev, static_cast<uint8_t *>(workspace), status, stream, launches);
  cbvh::count_launches(launches);
  return rc;
}

namespace cbvh {
int64_t refit_workspace_total(const cbvh_bvh *h) { return refit_layout(h).total; }

int refit_launch(cbvh_bvh *h, const float *verts_dev, const int32_t *tris_dev, uint8_t *ws, int32_t *status,
                 void *stream, int &launches) {
  const RefitLayout L = refit_layout(h);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RefitArgs a;
  std::memset(&a, 0, sizeof a);
  a.blob = static_cast<uint8_t *>(h->dev_blob);
  a.off_tris = h->off_tris;
  a.verts = verts_dev;
  a.tris = tris_dev;
  a.n_verts = h->n_verts;
  a.n_tris = h->n_tris;
  a.K = h->K;
  a.bits = h->bits;
  a.e = h->e;
  a.scale = std::ldexp(1.0f, h->e);
  a.rec_off = reinterpret_cast<const uint64_t *>(ws + L.rec_off);
  a.parent = reinterpret_cast<const int32_t *>(ws + L.parent);
  a.leaf = reinterpret_cast<const int32_t *>(ws + L.leaf);
  a.tdepth = reinterpret_cast<const int32_t *>(ws + L.tdepth);
  a.C = reinterpret_cast<int32_t *>(ws + L.C);
  a.D = reinterpret_cast<int32_t *>(ws + L.D);
  a.status = status;
  a.VL = reinterpret_cast<int32_t *>(ws + L.VL);
  const int64_t nC = 2 * h->n_nodes * h->K;
  init_bounds<<<(unsigned)std::min<int64_t>((nC + 255) / 256, 4096), 256, 0, s>>>(a.C, nC);
  launches += 1;
  auto grid = [](int64_t items) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 65535)); };
  vertex_lattice<<<grid(h->n_verts * h->K), 256, 0, s>>>(a);
  ++launches;
  a.order = reinterpret_cast<const int32_t *>(ws + L.by_level);
  const auto &ls = h->refit_level_start;
  for (int64_t d = (int64_t)ls.size() - 2; d >= 0; --d) {  // deepest level first
    a.begin = ls[d];
    a.end = ls[d + 1];
    if (a.end > a.begin) {
      bounds_level<<<grid((a.end - a.begin) * a.K), 256, 0, s>>>(a);
      ++launches;
    }
  }
  a.order = reinterpret_cast<const int32_t *>(ws + L.by_td);
  const auto &ts = h->refit_td_start;
  for (size_t d = 0; d + 1 < ts.size(); ++d) {  // treelet roots first, parents before children
    a.begin = ts[d];
    a.end = ts[d + 1];
    if (a.end > a.begin) {
      encode_level<<<grid((a.end - a.begin) * a.K), 256, 0, s>>>(a);
      ++launches;
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CBVH_OK : cuda_fail(e, "refit launch");
}
}  // namespace cbvh
