// Device-side build of a compressed k-DOP BVH (per-frame meshes, whose topology may change
// from frame to frame).  The blob is byte-identical to cbvh_build's for the same mesh.
//
// The tree's shape -- which node has how many children, the treelets, every record's
// topology words -- depends on the triangle count and the branching alone: each node's
// triangles are halved log2(branching) times (Sec. III's median split), so the sizes of all
// groups follow from n_tris.  cbvh_build_plan lays that shape out on the host once; here the
// device fills in everything the geometry decides:
//   1. every triangle: index and area checks, centroid key (v0 + v1 + v2 in FP64, as the
//      host builder sums it); every vertex: finiteness, max |d_j . v| over the vertices in
//      use;
//   2. the lattice exponent e: the smallest with every |d_j . v| / 2^e below 2^(30 - h),
//      decided exactly (the candidates around ilogb of the rounded maximum are tested with
//      the expansion arithmetic of the refit);
//   3. three lists of the triangles, each sorted by (centroid key on one axis, index) --
//      least-significant-digit radix sort, 8-bit digits, skipping digits no key varies in;
//   4. the median splits, one round per level of the binary split tree: every segment of
//      two or more triangles picks its axis of largest centroid extent (the ends of that
//      axis's list), keeps the first half of that list on the left, and the other two lists
//      follow by a stable partition (one prefix sum over all three lists per round), so
//      each list stays sorted within every segment; once no segment holds more than 512
//      triangles, the remaining rounds run segment by segment in shared memory;
//   5. the leaves' triangles into the triangle table, then the refit kernels: leaf bounds,
//      bounds bottom-up, predictor-corrector encoding top-down.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "lattice.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256, kItems = 4, kTile = kThreads * kItems;
constexpr int kDigitBits = 8, kDigits = 1 << kDigitBits;  // radix of the sort

// mesh faults found on the device (bits of Scalars::flags)
enum : uint32_t { F_INDEX = 1u, F_DEGENERATE = 2u, F_NONFINITE = 4u, F_EXTENT = 8u, F_RANGE = 16u };
// a scatter destination outside its range (never, by construction; checked, not written)
constexpr uint32_t F_INTERNAL = 1u << 31;

struct Scalars {
  uint32_t flags;
  uint32_t fit_fail;  // bit 0: e = ex1 - 1 does not fit; bit 1: e = ex1 does not fit
  int32_t ex1;        // ilogb(max |d.v|) - 29 + headroom
  int32_t e;
  int32_t status;     // refit status (CBVH_ERR_MESH for a bound beyond the half range)
  int32_t pad;
  unsigned long long mbits;  // max |d.v| over the vertices in use, FP64 bits
  unsigned long long kor[3], kand[3];  // OR / AND of the sort keys of each axis
};

int64_t al256(int64_t x) { return (x + 255) & ~int64_t(255); }
int64_t tiles(int64_t n) { return (n + kTile - 1) / kTile; }

// Byte offsets of the build's arrays; the refit plan and scratch come first.
struct BuildLayout {
  int64_t sc, leaf_pos, dkey, ukey, tmpk, tmpv, L0, L1, X, hist, sums, seg_s, seg_n, flag, used, total;
};
BuildLayout build_layout(const cbvh_bvh *h) {
  const int64_t nt = h->n_tris, nv = h->n_verts, nblk = tiles(nt);
  BuildLayout B;
  int64_t o = al256(cbvh::refit_workspace_total(h));
  auto take = [&o](int64_t bytes) {
    const int64_t at = o;
    o = al256(o + bytes);
    return at;
  };
  B.sc = take(sizeof(Scalars));
  B.leaf_pos = take(4 * nt);
  B.dkey = take(24 * nt);
  B.ukey = take(24 * nt);
  B.tmpk = take(8 * nt);
  B.tmpv = take(4 * nt);
  B.L0 = take(12 * nt);
  B.L1 = take(12 * nt);
  B.X = take(12 * nt);
  B.hist = take(4 * kDigits * nblk);
  B.sums = take(4 * std::max(tiles(3 * nt), tiles(kDigits * nblk)));
  B.seg_s = take(4 * nt);
  B.seg_n = take(4 * nt);
  B.flag = take(nt);
  B.used = take(nv);
  B.total = o;
  return B;
}

unsigned grid(int64_t items) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 65535));
}

// ---------------------------------------------------------------- 1-2: checks, keys, e
// Order-preserving map of an FP64 key to an unsigned integer (-0 taken as +0: the host's
// split compares values, so the two zeros tie and fall back to the triangle index).
__device__ __forceinline__ unsigned long long sort_key(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d == 0.0 ? 0.0 : d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void init_scalars(Scalars *sc) {
  sc->flags = sc->fit_fail = 0;
  sc->ex1 = sc->e = sc->status = sc->pad = 0;
  sc->mbits = 0;
  for (int c = 0; c < 3; ++c) {
    sc->kor[c] = 0;
    sc->kand[c] = ~0ull;
  }
}

__global__ void tri_keys(const float *V, int64_t nv, const int32_t *T, int64_t nt, double *dkey,
                         unsigned long long *ukey, uint8_t *used, Scalars *sc) {
  unsigned long long kor[3] = {0, 0, 0}, kand[3] = {~0ull, ~0ull, ~0ull};
  uint32_t fl = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    int32_t vi[3];
    bool bad = false;
    for (int c = 0; c < 3; ++c) {
      vi[c] = T[3 * t + c];
      bad |= vi[c] < 0 || vi[c] >= nv;
    }
    double key[3] = {0.0, 0.0, 0.0};
    if (bad) {
      fl |= F_INDEX;
    } else {
      double p[3][3];
      for (int c = 0; c < 3; ++c) {
        for (int x = 0; x < 3; ++x) p[c][x] = (double)V[3 * (int64_t)vi[c] + x];
        used[vi[c]] = 1;
      }
      double a[3], b[3];
      for (int x = 0; x < 3; ++x) {
        a[x] = __dsub_rn(p[1][x], p[0][x]);
        b[x] = __dsub_rn(p[2][x], p[0][x]);
      }
      const double nx = __dsub_rn(__dmul_rn(a[1], b[2]), __dmul_rn(a[2], b[1]));
      const double ny = __dsub_rn(__dmul_rn(a[2], b[0]), __dmul_rn(a[0], b[2]));
      const double nz = __dsub_rn(__dmul_rn(a[0], b[1]), __dmul_rn(a[1], b[0]));
      if (nx == 0.0 && ny == 0.0 && nz == 0.0) fl |= F_DEGENERATE;
      for (int x = 0; x < 3; ++x) key[x] = __dadd_rn(__dadd_rn(p[0][x], p[1][x]), p[2][x]);
    }
    for (int x = 0; x < 3; ++x) {
      dkey[3 * t + x] = key[x];
      const unsigned long long u = sort_key(key[x]);
      ukey[x * nt + t] = u;
      kor[x] |= u;
      kand[x] &= u;
    }
  }
  for (int o = 16; o; o >>= 1) {
    fl |= __shfl_xor_sync(kFull, fl, o);
    for (int x = 0; x < 3; ++x) {
      kor[x] |= __shfl_xor_sync(kFull, kor[x], o);
      kand[x] &= __shfl_xor_sync(kFull, kand[x], o);
    }
  }
  if ((threadIdx.x & 31) == 0) {
    if (fl) atomicOr(&sc->flags, fl);
    for (int x = 0; x < 3; ++x) {
      atomicOr(&sc->kor[x], kor[x]);
      atomicAnd(&sc->kand[x], kand[x]);
    }
  }
}

// Every vertex finite; max over the vertices in use and the K directions of |d_j . v|, summed
// in the host builder's order ((d0 x + d1 y) + d2 z, products exact).
__global__ void vert_extent(const float *V, int64_t nv, int K, const uint8_t *used, Scalars *sc) {
  double m = 0.0;
  bool nonfinite = false;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const float x = V[3 * v], y = V[3 * v + 1], z = V[3 * v + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
      nonfinite = true;
      continue;
    }
    if (!used[v]) continue;
    for (int j = 0; j < K; ++j) {
      const double s = __dadd_rn(__dadd_rn(__dmul_rn((double)c_rdir[j][0], (double)x), __dmul_rn((double)c_rdir[j][1], (double)y)),
                                 __dmul_rn((double)c_rdir[j][2], (double)z));
      m = fmax(m, fabs(s));
    }
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  nonfinite = __any_sync(kFull, nonfinite);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&sc->mbits, (unsigned long long)__double_as_longlong(m));  // m >= 0: bits order as values
    if (nonfinite) atomicOr(&sc->flags, F_NONFINITE);
  }
}

__global__ void exponent_candidate(Scalars *sc, int headroom) {
  const double M = __longlong_as_double((long long)sc->mbits);
  if (!(M > 0.0)) {
    atomicOr(&sc->flags, F_EXTENT);
    sc->ex1 = 0;
    return;
  }
  sc->ex1 = ilogb(M) - 29 + headroom;
}

// The test at e = ex1 - 1 and e = ex1: every lattice value of a vertex in use within
// +-(2^(30 - headroom) - 1), that is |d.v| < 2^(e + 30 - headroom): below T0 = 2^ilogb(max)
// and below T1 = 2T0.  The rounded maximum is off by a few units in the last place (its
// axis terms are exact), so the exact exponent is ex1 - 1, ex1 or ex1 + 1.  The rounded
// |d.v| (two additions of exact terms, off by at most 2^-51 (|a| + |b| + |c|)) decides every
// value outside that margin of T0 and T1; the rest take the exact floor and ceil.  Most
// values never reach FP64: their terms are integers at the lattice's scale.
__global__ void exponent_fits(const float *V, int64_t nv, int K, const uint8_t *used, Scalars *sc, int headroom) {
  const int ex1 = sc->ex1;
  const double T0 = ldexp(1.0, ex1 - 1 + 30 - headroom), T1 = 2.0 * T0;
  const long long L = 1ll << (30 - headroom);
  bool f0 = false, f1 = false;
  const int64_t items = nv * K;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items; it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = it / K;
    const int j = (int)(it - v * K);
    if (!used[v]) continue;
    const float p[3] = {V[3 * v], V[3 * v + 1], V[3 * v + 2]};
    // usual case: the terms at scale 2^-(ex1 - 1) are integers and S, their int64 sum, is
    // exact; e = ex1 - 1 fits iff |S| <= L - 1 and e = ex1 iff |S / 2| < L
    long long S = 0;
    bool ints = true;
    for (int c = 0; c < 3; ++c) {
      const int d = c_rdir[j][c];
      long long x;
      if (d != 0) {
        ints = ints && scaled_int(p[c], ex1 - 1, x);
        S += ints ? d * x : 0;
      }
    }
    if (ints) {
      const long long aS = S < 0 ? -S : S;
      f0 |= aS > L - 1;
      f1 |= aS >= 2 * L;
      continue;
    }
    double a[3];
    for (int c = 0; c < 3; ++c) a[c] = __dmul_rn((double)c_rdir[j][c], (double)p[c]);
    const double s = fabs(__dadd_rn(__dadd_rn(a[0], a[1]), a[2]));
    const double m = (fabs(a[0]) + fabs(a[1]) + fabs(a[2])) * 0x1p-51;
    long long lo, hi;
    // rounding is monotone and T0, T1 are powers of two: fl(s + m) < T is certainly below,
    // fl(s - m) > T certainly above
    if (s + m >= T0) {
      if (s - m > T0) {
        f0 = true;
      } else {
        lattice_of(p, j, ex1 - 1, lo, hi);
        f0 |= lo > L - 1 || hi < -(L - 1);
      }
      if (s + m >= T1) {
        if (s - m > T1) {
          f1 = true;
        } else {
          lattice_of(p, j, ex1, lo, hi);
          f1 |= lo > L - 1 || hi < -(L - 1);
        }
      }
    }
  }
  f0 = __any_sync(kFull, f0);
  f1 = __any_sync(kFull, f1);
  if ((threadIdx.x & 31) == 0 && (f0 || f1)) atomicOr(&sc->fit_fail, (f0 ? 1u : 0u) | (f1 ? 2u : 0u));
}

__global__ void exponent_final(Scalars *sc, uint8_t *blob) {
  if (sc->flags & F_EXTENT) return;
  int e = sc->ex1 - 1;
  if (sc->fit_fail & 1u) e = (sc->fit_fail & 2u) ? sc->ex1 + 1 : sc->ex1;
  if (e < -120 || e > 96) atomicOr(&sc->flags, F_RANGE);
  sc->e = e;
  *reinterpret_cast<int32_t *>(blob + 12) = e;  // header field of the lattice exponent
}

// ---------------------------------------------------------------- prefix sums (uint32)
struct Plain {
  const uint32_t *p;
  __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
// 1 where the triangle at position i of the three concatenated lists goes left this round
struct Gathered {
  const int32_t *L;
  const uint8_t *flag;
  __device__ uint32_t operator()(int64_t i) const { return flag[L[i]]; }
};

// Exclusive prefix sum of each tile of kTile values (in place allowed), tile totals to sums.
template <class In>
__global__ void __launch_bounds__(kThreads) scan_tiles(In in, uint32_t *out, int64_t n, uint32_t *sums) {
  __shared__ uint32_t wsum[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = blockIdx.x * (int64_t)kTile + (int64_t)threadIdx.x * kItems;
  uint32_t v[kItems], acc = 0;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    v[q] = base + q < n ? in(base + q) : 0u;
    acc += v[q];
  }
  uint32_t x = acc;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    const uint32_t t = lane < kThreads / 32 ? wsum[lane] : 0u;
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane < kThreads / 32) wsum[lane] = incl - t;
  }
  __syncthreads();
  uint32_t run = wsum[w] + x - acc;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
  if (threadIdx.x == kThreads - 1) sums[blockIdx.x] = wsum[w] + x;
}

// Exclusive prefix sum of the tile totals, in place (one block of 1024 threads).
__global__ void __launch_bounds__(1024) scan_sums(uint32_t *sums, int64_t nb) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry_s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const uint32_t v = i < nb ? sums[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      const uint32_t t = wsum[lane];
      uint32_t incl = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      wsum[lane] = incl - t;
    }
    __syncthreads();
    const uint32_t excl = carry + wsum[w] + x - v;
    if (i < nb) sums[i] = excl;
    if (threadIdx.x == 1023) carry_s = excl + v;
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
}

// Value i of a scan done by scan_tiles + scan_sums: the tile's own prefix plus the tiles
// before it (the consumers add it, saving a pass over the array).
__device__ __forceinline__ uint32_t scanned(const uint32_t *X, const uint32_t *sums, int64_t i) {
  return X[i] + sums[i / kTile];
}

template <class In>
void exclusive_scan(In in, uint32_t *out, int64_t n, uint32_t *sums, cudaStream_t s, int &launches) {
  const int64_t nb = tiles(n);
  scan_tiles<In><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, sums);
  scan_sums<<<1, 1024, 0, s>>>(sums, nb);
  launches += 2;
}

// ---------------------------------------------------------------- 3: radix sort (stable LSD)
__global__ void iota_kernel(int32_t *v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

// Digit counts of each tile, digit-major: hist[d * nblk + tile].
__global__ void __launch_bounds__(kThreads) rs_hist(const unsigned long long *keys, int64_t n, int shift,
                                                   uint32_t *hist, int64_t nblk) {
  __shared__ uint32_t cnt[kDigits];
  for (int e = threadIdx.x; e < kDigits; e += kThreads) cnt[e] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kTile;
  for (int q = 0; q < kItems; ++q) {
    const int64_t i = base + q * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kDigits - 1u)], 1u);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kDigits; e += kThreads) hist[e * nblk + blockIdx.x] = cnt[e];
}

// Stable scatter by one digit: an element's destination is the scanned count of smaller
// digits and earlier tiles (base) plus the number of equal digits before it in its tile,
// counted in element order (sub-round, warp, lane).
__global__ void __launch_bounds__(kThreads) rs_scatter(const unsigned long long *kin, const int32_t *vin,
                                                      unsigned long long *kout, int32_t *vout, int64_t n,
                                                      int shift, const uint32_t *base, const uint32_t *sums,
                                                      int64_t nblk, Scalars *sc) {
  __shared__ uint32_t run[kDigits];
  __shared__ uint32_t wc[kThreads / 32][kDigits];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < kDigits; e += kThreads) run[e] = scanned(base, sums, e * nblk + blockIdx.x);
  const int64_t tb = blockIdx.x * (int64_t)kTile;
  for (int q = 0; q < kItems; ++q) {
    const int64_t i = tb + q * kThreads + threadIdx.x;
    const bool ok = i < n;
    const unsigned long long k = ok ? kin[i] : 0ull;
    const int d = ok ? (int)((k >> shift) & (kDigits - 1u)) : kDigits;
    const unsigned peers = __match_any_sync(kFull, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    for (int e = threadIdx.x; e < (kThreads / 32) * kDigits; e += kThreads) wc[e / kDigits][e % kDigits] = 0;
    __syncthreads();
    if (ok && lane == __ffs(peers) - 1) wc[w][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t pre = run[d];
      for (int u = 0; u < w; ++u) pre += wc[u][d];
      const uint32_t dst = pre + (uint32_t)rank;
      if (dst < n) {
        kout[dst] = k;
        vout[dst] = vin[i];
      } else {
        atomicOr(&sc->flags, F_INTERNAL);
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kDigits; e += kThreads) {
      uint32_t add = 0;
      for (int u = 0; u < kThreads / 32; ++u) add += wc[u][e];
      run[e] += add;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- 4: median-split rounds
__global__ void seg_init(int32_t *seg_s, int32_t *seg_n, int64_t nt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    seg_s[i] = 0;
    seg_n[i] = (int32_t)nt;
  }
}

// For every position of a segment with n >= 2: the split axis (largest centroid extent,
// lowest axis on ties, as the host builder picks it) and the side of the triangle that
// sits at this position of that axis's list.
__global__ void split_mark(const int32_t *L, int64_t nt, const double *dkey, const int32_t *seg_s,
                           const int32_t *seg_n, uint8_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t n = seg_n[i];
    if (n < 2) continue;
    const int64_t s = seg_s[i];
    double ext[3];
    for (int c = 0; c < 3; ++c)
      ext[c] = __dsub_rn(dkey[3 * (int64_t)L[c * nt + s + n - 1] + c], dkey[3 * (int64_t)L[c * nt + s] + c]);
    int ax = 0;
    if (ext[1] > ext[0]) ax = 1;
    if (ext[2] > ext[ax]) ax = 2;
    flag[L[ax * nt + i]] = (i - s) < (int64_t)(n / 2) ? 1 : 0;
  }
}

// Stable partition of each list within every segment of two or more (left half first), and
// the segments of the next round.  X holds the exclusive prefix count of left-going
// triangles over the three concatenated lists; its differences are exact modulo 2^32.
__global__ void split_move(const int32_t *Lin, int32_t *Lout, int64_t nt, const uint8_t *flag, const uint32_t *X,
                           const uint32_t *sums, int32_t *seg_s, int32_t *seg_n, Scalars *sc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t n = seg_n[i];
    const int64_t s = seg_s[i];
    for (int c = 0; c < 3; ++c) {
      const int32_t tri = Lin[c * nt + i];
      if (n < 2) {
        Lout[c * nt + i] = tri;
        continue;
      }
      const int64_t left_before = (int64_t)(uint32_t)(scanned(X, sums, c * nt + i) - scanned(X, sums, c * nt + s));
      const int64_t pos = flag[tri] ? s + left_before : s + n / 2 + (i - s - left_before);
      if (pos >= s && pos < s + n)
        Lout[c * nt + pos] = tri;
      else
        atomicOr(&sc->flags, F_INTERNAL);
    }
    if (n >= 2) {
      const int32_t half = n / 2;
      if (i - s < half) {
        seg_n[i] = half;
      } else {
        seg_s[i] = (int32_t)(s + half);
        seg_n[i] = n - half;
      }
    }
  }
}

// The last rounds, on segments of at most kLocal triangles: one block per segment, all in
// shared memory.  The segment is the one the global rounds left at position blockIdx.x of
// their binary split tree (its path of halvings, left = 0); the lists become indices into
// the segment's triangles (their keys staged beside them), and each round applies the same
// axis rule and stable partition as split_mark / split_move, with a block-wide prefix sum.
// Only list 0 is written back: after the last round all three lists agree.
constexpr int kLocal = 512;
__global__ void __launch_bounds__(kThreads) split_local(int32_t *L, int64_t nt, const double *dkey, int depth,
                                                       int32_t *loc, Scalars *sc) {
  __shared__ uint16_t ls[2][3][kLocal];
  __shared__ int32_t tri[kLocal];
  __shared__ double key[kLocal][3];
  __shared__ uint8_t flag[kLocal];
  __shared__ uint16_t ss[kLocal], sn[kLocal];
  __shared__ uint16_t X[3 * kLocal];
  __shared__ uint32_t wsum[kThreads / 32];
  int64_t s = 0, n = nt;
  for (int lev = depth - 1; lev >= 0; --lev) {
    const int64_t h = n / 2;
    if ((blockIdx.x >> lev) & 1u) {
      s += h;
      n -= h;
    } else {
      n = h;
    }
  }
  if (n <= 1) return;  // one triangle (or none): nothing to split
  if (n > kLocal) {
    if (threadIdx.x == 0) atomicOr(&sc->flags, F_INTERNAL);
    return;
  }
  const int m = (int)n;
  for (int p = threadIdx.x; p < m; p += kThreads) {
    const int32_t t = L[s + p];
    tri[p] = t;
    loc[t] = p;
    for (int c = 0; c < 3; ++c) key[p][c] = dkey[3 * (int64_t)t + c];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += kThreads) {
    ls[0][0][p] = (uint16_t)p;
    for (int c = 1; c < 3; ++c) ls[0][c][p] = (uint16_t)loc[L[c * nt + s + p]];
    ss[p] = 0;
    sn[p] = (uint16_t)m;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kPer = (3 * kLocal + kThreads - 1) / kThreads;  // scan entries per thread
  int cur = 0;
  for (int width = 1; width < m; width <<= 1) {
    for (int p = threadIdx.x; p < m; p += kThreads) {
      const int a = ss[p], len = sn[p];
      if (len < 2) continue;
      double ext[3];
      for (int c = 0; c < 3; ++c) ext[c] = __dsub_rn(key[ls[cur][c][a + len - 1]][c], key[ls[cur][c][a]][c]);
      int ax = 0;
      if (ext[1] > ext[0]) ax = 1;
      if (ext[2] > ext[ax]) ax = 2;
      flag[ls[cur][ax][p]] = (p - a) < len / 2 ? 1 : 0;
    }
    __syncthreads();
    // exclusive prefix count of left-going triangles over the three lists, in list order
    uint32_t v[kPer], acc = 0;
    for (int q = 0; q < kPer; ++q) {
      const int e = threadIdx.x * kPer + q;
      v[q] = e < 3 * m ? flag[ls[cur][e / m][e % m]] : 0u;
      acc += v[q];
    }
    uint32_t x = acc;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      const uint32_t t = lane < kThreads / 32 ? wsum[lane] : 0u;
      uint32_t incl = t;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane < kThreads / 32) wsum[lane] = incl - t;
    }
    __syncthreads();
    uint32_t run = wsum[w] + x - acc;
    for (int q = 0; q < kPer; ++q) {
      const int e = threadIdx.x * kPer + q;
      if (e < 3 * m) X[e] = (uint16_t)run;
      run += v[q];
    }
    __syncthreads();
    for (int p = threadIdx.x; p < m; p += kThreads) {
      const int a = ss[p], len = sn[p];
      for (int c = 0; c < 3; ++c) {
        const uint16_t k = ls[cur][c][p];
        if (len < 2) {
          ls[cur ^ 1][c][p] = k;
          continue;
        }
        const int lb = (int)X[c * m + p] - (int)X[c * m + a];
        const int pos = flag[k] ? a + lb : a + len / 2 + (p - a - lb);
        if (pos >= a && pos < a + len)
          ls[cur ^ 1][c][pos] = k;
        else
          atomicOr(&sc->flags, F_INTERNAL);
      }
      if (len >= 2) {
        const int half = len / 2;
        if (p - a < half) {
          sn[p] = (uint16_t)half;
        } else {
          ss[p] = (uint16_t)(a + half);
          sn[p] = (uint16_t)(len - half);
        }
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int p = threadIdx.x; p < m; p += kThreads) L[s + p] = tri[ls[cur][0][p]];
}

// ---------------------------------------------------------------- 5: triangle table
__global__ void leaf_tris(const int32_t *perm, const int32_t *leaf_pos, int64_t nt, uint8_t *blob, int64_t off_tris) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nt; q += (int64_t)gridDim.x * blockDim.x)
    *reinterpret_cast<uint32_t *>(blob + off_tris + 48 * q + 12) = (uint32_t)perm[leaf_pos[q]];
}

int cuda_fail(cudaError_t e, const char *what) {
  return cbvh::fail(CBVH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

const char *flag_message(uint32_t f) {
  if (f & F_INDEX) return "a triangle has an out-of-range vertex index";
  if (f & F_NONFINITE) return "non-finite vertex coordinate";
  if (f & F_DEGENERATE) return "a triangle is degenerate (zero area)";
  if (f & F_EXTENT) return "mesh has no extent";
  return "mesh coordinates outside the supported range";
}

}  // namespace

extern "C" int cbvh_build_device_workspace_bytes(const cbvh_bvh *h, int64_t *bytes) {
  cbvh::clear_error();
  if (!h || !bytes) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  *bytes = build_layout(h).total;
  return CBVH_OK;
}

extern "C" int cbvh_build_device(cbvh_bvh *h, const float *verts_dev, const int32_t *tris_dev, void *workspace,
                                 int64_t workspace_bytes, uint32_t flags, void *stream) {
  CBVH_RANGE("cbvh_build_device");
  cbvh::clear_error();
  if (!h || !verts_dev || !tris_dev || !workspace) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (h->leaf_pos.empty()) return cbvh::fail(CBVH_ERR_STATE, "not a plan; create the handle with cbvh_build_plan");
  if (!h->dev_blob) return cbvh::fail(CBVH_ERR_STATE, "handle has no device blob; call cbvh_attach");
  const BuildLayout BL = build_layout(h);
  if (workspace_bytes < BL.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return cbvh::fail(CBVH_ERR_WORKSPACE, "device-build workspace too small or not 256-byte aligned");
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nt = h->n_tris, nv = h->n_verts, nblk = tiles(nt);
  if (h->devbuild_ws != workspace) {  // the node plan of the refit kernels, the leaves' positions
    if (int rc = cbvh_refit_prepare(h, workspace, workspace_bytes, stream)) return rc;
    cudaError_t e = cudaMemcpyAsync(ws + BL.leaf_pos, h->leaf_pos.data(), 4 * nt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device-build plan upload");
    h->devbuild_ws = workspace;
  }
  h->geometry = false;  // until this build succeeds
  uint8_t *blob = static_cast<uint8_t *>(h->dev_blob);
  Scalars *sc = reinterpret_cast<Scalars *>(ws + BL.sc);
  double *dkey = reinterpret_cast<double *>(ws + BL.dkey);
  auto *ukey = reinterpret_cast<unsigned long long *>(ws + BL.ukey);
  auto *tmpk = reinterpret_cast<unsigned long long *>(ws + BL.tmpk);
  auto *tmpv = reinterpret_cast<int32_t *>(ws + BL.tmpv);
  auto *L0 = reinterpret_cast<int32_t *>(ws + BL.L0);
  auto *L1 = reinterpret_cast<int32_t *>(ws + BL.L1);
  auto *X = reinterpret_cast<uint32_t *>(ws + BL.X);
  auto *hist = reinterpret_cast<uint32_t *>(ws + BL.hist);
  auto *sums = reinterpret_cast<uint32_t *>(ws + BL.sums);
  auto *seg_s = reinterpret_cast<int32_t *>(ws + BL.seg_s);
  auto *seg_n = reinterpret_cast<int32_t *>(ws + BL.seg_n);
  auto *flag = ws + BL.flag;
  auto *used = ws + BL.used;
  const auto *leaf_pos = reinterpret_cast<const int32_t *>(ws + BL.leaf_pos);
  int launches = 0;

  // 1-2: checks, keys, lattice exponent
  cudaError_t e = cudaMemsetAsync(used, 0, nv, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  init_scalars<<<1, 1, 0, s>>>(sc);
  tri_keys<<<grid(nt), 256, 0, s>>>(verts_dev, nv, tris_dev, nt, dkey, ukey, used, sc);
  vert_extent<<<grid(nv), 256, 0, s>>>(verts_dev, nv, h->K, used, sc);
  exponent_candidate<<<1, 1, 0, s>>>(sc, h->headroom);
  exponent_fits<<<grid(nv * h->K), 256, 0, s>>>(verts_dev, nv, h->K, used, sc, h->headroom);
  exponent_final<<<1, 1, 0, s>>>(sc, blob);
  launches += 6;
  Scalars host_sc;
  e = cudaMemcpyAsync(&host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cbvh::count_launches(launches);
    return cuda_fail(e, "device build (checks)");
  }
  if (host_sc.flags) {
    cbvh::count_launches(launches);
    return cbvh::fail(CBVH_ERR_MESH, flag_message(host_sc.flags));
  }

  // 3: three lists sorted by (centroid key of one axis, triangle index)
  for (int c = 0; c < 3; ++c) {
    const unsigned long long vary = host_sc.kor[c] ^ host_sc.kand[c];
    unsigned long long *kin = ukey + c * nt, *kalt = tmpk;
    int32_t *vin = L0 + c * nt, *valt = tmpv;
    iota_kernel<<<grid(nt), 256, 0, s>>>(vin, nt);
    ++launches;
    for (int shift = 0; shift < 64; shift += kDigitBits) {
      if (((vary >> shift) & (kDigits - 1u)) == 0) continue;  // every key has the same digit here
      rs_hist<<<(unsigned)nblk, kThreads, 0, s>>>(kin, nt, shift, hist, nblk);
      exclusive_scan(Plain{hist}, hist, kDigits * nblk, sums, s, launches);
      rs_scatter<<<(unsigned)nblk, kThreads, 0, s>>>(kin, vin, kalt, valt, nt, shift, hist, sums, nblk, sc);
      launches += 2;
      std::swap(kin, kalt);
      std::swap(vin, valt);
    }
    if (vin != L0 + c * nt) {
      e = cudaMemcpyAsync(L0 + c * nt, vin, 4 * nt, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
  }

  // 4: one round per level of the binary split tree
  seg_init<<<grid(nt), 256, 0, s>>>(seg_s, seg_n, nt);
  ++launches;
  int32_t *Lc = L0, *Ln = L1;
  int depth = 0;  // global rounds until no segment holds more than kLocal triangles
  for (; ((nt + (int64_t(1) << depth) - 1) >> depth) > kLocal; ++depth) {
    split_mark<<<grid(nt), 256, 0, s>>>(Lc, nt, dkey, seg_s, seg_n, flag);
    exclusive_scan(Gathered{Lc, flag}, X, 3 * nt, sums, s, launches);
    split_move<<<grid(nt), 256, 0, s>>>(Lc, Ln, nt, flag, X, sums, seg_s, seg_n, sc);
    launches += 2;
    std::swap(Lc, Ln);
  }
  // the remaining rounds segment by segment in shared memory (tmpv, free after the sort,
  // maps a triangle to its index in its segment)
  split_local<<<(unsigned)(int64_t(1) << depth), kThreads, 0, s>>>(Lc, nt, dkey, depth, tmpv, sc);
  ++launches;

  // 5: triangle table, then bounds and encoding with the refit kernels
  leaf_tris<<<grid(nt), 256, 0, s>>>(Lc, leaf_pos, nt, blob, h->off_tris);
  ++launches;
  h->e = host_sc.e;
  int rc = cbvh::refit_launch(h, verts_dev, tris_dev, ws, &sc->status, stream, launches);
  cbvh::count_launches(launches);
  if (rc) return rc;
  e = cudaMemcpyAsync(&host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "device build");
  if (host_sc.flags & F_INTERNAL) return cbvh::fail(CBVH_ERR_STATE, "device build: inconsistent split order");
  if (host_sc.status)
    return cbvh::fail(CBVH_ERR_MESH, h->bits == CBVH_QUANT_FP16
                                         ? "mesh bounds exceed the half-precision range (+-65504) of quant_bits = 1"
                                         : "mesh bounds outside the lattice range");
  std::memcpy(h->blob.data() + 12, &h->e, 4);
  if (flags & CBVH_BUILD_HOST_COPY) {
    e = cudaMemcpyAsync(h->blob.data(), h->dev_blob, h->blob.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device build (host copy)");
    h->host_stale = false;
  } else {
    h->host_stale = true;
  }
  h->geometry = true;
  return CBVH_OK;
}
