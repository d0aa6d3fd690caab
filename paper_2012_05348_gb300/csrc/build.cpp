// Host-side BVH builder and treelet encoder of libcbvh.
//
// Produces the compressed blob that the CUDA kernels traverse:
//   * k-DOP bounding volumes over k/2 fixed integer directions (Table 1: "k floats" per
//     k-DOP), one triangle per leaf, `branching` children per inner node;
//   * bounds quantised on one absolute lattice of step 2^e ("we quantify BV", abstract):
//     lo = floor(d.v / 2^e), hi = ceil(d.v / 2^e) of the exact real products;
//   * predictor-corrector deltas (abstract; Sec. III-B, "predictors based on the delta to
//     the parent nodes"): a node is predicted by its parent's decoded interval and
//     corrected by b-bit unsigned deltas that round outward;
//   * treelets (Sec. III-B, "clustering BVHs into a smaller parts"): clusters of whole
//     sibling groups within a byte budget, grown top-down (breadth-first from each root) or
//     packed bottom-up (CBVH_OPT_TREELET_PACKING), each with an absolute root so that any
//     treelet is randomly accessible (abstract).
//
// Blob layout (little endian; offsets from the blob start):
//   [0, 64)     header: magic 'CBVH', version, k, K, m, bits, lbits, max treelet depth,
//               e, n_tris, n_nodes, n_treelets, record bytes, root record bytes, treelet
//               budget, tree depth, treelet packing, offset of the triangle table,
//               total bytes
//   [64, ...)   u64 treelet offsets [n_treelets + 1]
//   treelets    16-byte aligned: {u32 node count, u32 blob-order index of the root, 0, 0},
//               the root record, then fixed-size records in treelet BFS order
//   triangles   48 bytes per leaf, in leaf order: v0.xyz, original index, v1.xyz, 0, v2.xyz, 0
// Record: u32 w0 = parent local index (0xFFFF at the root) | child count << 16 |
//         children-are-treelet-roots << 21 | depth below the treelet root << 24;
//         u32 w1 = first child (local index, or treelet id when external) or, at a leaf,
//         its leaf-order triangle slot; then per direction j the pair (lo, hi): absolute
//         int32 lattice values at a treelet root, b-bit correctors elsewhere, or FP32
//         values (lo rounded down, hi rounded up) everywhere when quant_bits = 0, or FP16
//         values rounded the same way (Sec. III-A's half-float descriptors) everywhere when
//         quant_bits = 1, or (quant_bits = 2) an 8-byte Stream VByte control word and the
//         2K exact deltas to the parent's interval in 1 to 4 bytes each; such records vary in
//         size (padded to 4 bytes) and are found through a table of 2-byte offsets, in
//         4-byte units from the treelet's start, that follows the treelet header (padded
//         to 8 bytes, so that the absolute root record is 8-byte aligned).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <limits>
#include <numeric>

#include "internal.h"

namespace {

// Slab directions; the k-DOP uses the first k/2.
const int kDir[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                         {0, 1, 1},  {0, 1, -1}, {1, 1, 1},  {1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};

// ---------------------------------------------------------------- exact lattice rounding
// Exact floor of a + b + c.  Fast path: the rounded sum is far enough from an integer
// that its rounding error (at most 2u (|a| + |b| + |c|)) cannot cross one.  Otherwise the
// sum is turned into a non-overlapping expansion (Knuth's TwoSum, Shewchuk's
// Grow-Expansion) and its floor is read from the largest component down.
inline void two_sum(double a, double b, double &s, double &err) {
  s = a + b;
  double bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

int64_t exact_floor(double a, double b, double c) {
  double s = (a + b) + c;
  double slack = 4.0 * std::ldexp(std::fabs(a) + std::fabs(b) + std::fabs(c), -53);
  double f1 = std::floor(s - slack), f2 = std::floor(s + slack);
  if (f1 == f2) return (int64_t)f1;
  double x, ex, y, ey;
  two_sum(a, b, x, ex);
  two_sum(c, ex, y, ey);
  double z, ez;
  two_sum(y, x, z, ez);
  double comp[3] = {z, ez, ey};  // largest first
  int64_t acc = 0;
  for (double v : comp) {
    double fl = std::floor(v);
    if (fl != v) return acc + (int64_t)fl;
    acc += (int64_t)v;
  }
  return acc;
}
inline int64_t exact_ceil(double a, double b, double c) { return -exact_floor(-a, -b, -c); }

// RD / RU conversion of a lattice integer to FP32, then exact scaling by 2^e.
float to_f32_down(int64_t L, int e) {
  float f = (float)L;
  if ((double)f > (double)L) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
  return std::ldexp(f, e);
}
float to_f32_up(int64_t L, int e) {
  float f = (float)L;
  if ((double)f < (double)L) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return std::ldexp(f, e);
}

struct Node {
  int32_t parent = -1, first = -1, count = 0, tri = -1, depth = 0;
};

struct Builder {
  int k, K, m, bits, budget;
  const float *V;
  int64_t nv;
  const int32_t *T;
  int64_t nt;
  std::vector<double> key;  // nt x 3
  std::vector<Node> nodes;  // BFS order
  std::vector<int32_t> perm;
  int e = 0;
  std::vector<int32_t> vlat;  // per vertex, per direction: lo, hi
  std::vector<int32_t> lat;   // per node, per direction: lo, hi (exact)

  // Partition perm[s, s+n) so that its first n/2 entries are the n/2 smallest by
  // (centroid key on the axis of largest centroid extent, triangle index).
  void split(int64_t s, int64_t n) {
    double lo[3], hi[3];
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::numeric_limits<double>::infinity();
      hi[c] = -lo[c];
    }
    for (int64_t i = s; i < s + n; ++i)
      for (int c = 0; c < 3; ++c) {
        double v = key[3 * (int64_t)perm[i] + c];
        lo[c] = std::min(lo[c], v);
        hi[c] = std::max(hi[c], v);
      }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
      if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
    const double *kp = key.data();
    std::nth_element(perm.begin() + s, perm.begin() + s + n / 2, perm.begin() + s + n, [kp, ax](int32_t a, int32_t b) {
      double ka = kp[3 * (int64_t)a + ax], kb = kp[3 * (int64_t)b + ax];
      return ka < kb || (ka == kb && a < b);
    });
  }

  // shape_only: no splits; every leaf records its position in the (device-sorted) order
  // instead of a triangle, since the shape depends on the triangle count alone.
  void build_tree(bool shape_only = false) {
    perm.resize(nt);
    std::iota(perm.begin(), perm.end(), 0);
    struct Item {
      int32_t node;
      int64_t s, n;
    };
    std::deque<Item> q;
    nodes.reserve(2 * nt);
    nodes.emplace_back();
    q.push_back({0, 0, nt});
    while (!q.empty()) {
      Item it = q.front();
      q.pop_front();
      if (it.n == 1) {
        nodes[it.node].tri = perm[it.s];
        continue;
      }
      std::vector<std::pair<int64_t, int64_t>> groups{{it.s, it.n}};
      for (int r = 1; r < m; r <<= 1) {
        std::vector<std::pair<int64_t, int64_t>> next;
        for (auto [s, n] : groups) {
          if (n == 1) {
            next.push_back({s, 1});
            continue;
          }
          if (!shape_only) split(s, n);
          next.push_back({s, n / 2});
          next.push_back({s + n / 2, n - n / 2});
        }
        groups.swap(next);
      }
      int32_t first = (int32_t)nodes.size();
      nodes[it.node].first = first;
      nodes[it.node].count = (int32_t)groups.size();
      for (auto [s, n] : groups) {
        Node c;
        c.parent = it.node;
        c.depth = nodes[it.node].depth + 1;
        nodes.push_back(c);
        q.push_back({(int32_t)nodes.size() - 1, s, n});
      }
    }
  }

  // true when every |d.v| / 2^e < 2^30
  int headroom = 0;  // lattice bits kept free for refits (CBVH_OPT_LATTICE_HEADROOM)
  bool fits(int ex) const {
    const int64_t L = int64_t(1) << (30 - headroom);
    for (int64_t v = 0; v < nv; ++v)
      for (int j = 0; j < K; ++j) {
        double t[3];
        for (int c = 0; c < 3; ++c) t[c] = kDir[j][c] * std::ldexp((double)V[3 * v + c], -ex);
        if (exact_floor(t[0], t[1], t[2]) > L - 1 || exact_ceil(t[0], t[1], t[2]) < -(L - 1)) return false;
      }
    return true;
  }
};

uint32_t f32_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
void w32(std::vector<uint8_t> &b, int64_t o, uint32_t v) { std::memcpy(&b[o], &v, 4); }
void w64(std::vector<uint8_t> &b, int64_t o, uint64_t v) { std::memcpy(&b[o], &v, 8); }
void w16(std::vector<uint8_t> &b, int64_t o, uint16_t v) { std::memcpy(&b[o], &v, 2); }

// IEEE binary16 bits of the largest half-precision value <= v (down) or the smallest >= v
// (up), for a finite double v.  Values beyond the largest finite half (65504) round to it
// or to the infinity on their side, so the result always bounds v outward.  Positive v is
// q * quantum with the quantum of v's binade (2^-24 below 2^-14), q taken by floor or ceil.
uint16_t half_pos(double v, bool up) {  // v > 0
  if (v > 65504.0) return up ? 0x7c00u : 0x7bffu;
  int ex = 0;
  std::frexp(v, &ex);  // v = f 2^ex, f in [0.5, 1): binade exponent E = ex - 1
  const int E = std::max(ex - 1, -14);
  const double quantum = std::ldexp(1.0, E - 10);
  const double q = up ? std::ceil(v / quantum) : std::floor(v / quantum);  // exact: power-of-two scaling
  int64_t qi = (int64_t)q;
  if (E == -14 && qi < 1024) return (uint16_t)qi;  // subnormal (or the first normal when qi reaches 1024)
  int exp_field = E + 15;
  if (qi == 2048) {  // ceil reached the next binade
    qi = 1024;
    ++exp_field;
  }
  if (exp_field >= 31) return 0x7c00u;
  return (uint16_t)((exp_field << 10) | (qi - 1024));
}
uint16_t half_down(double v) {
  if (v == 0.0) return 0x0000u;
  return v > 0 ? half_pos(v, false) : (uint16_t)(0x8000u | half_pos(-v, true));
}
uint16_t half_up(double v) {
  if (v == 0.0) return 0x0000u;
  return v > 0 ? half_pos(v, true) : (uint16_t)(0x8000u | half_pos(-v, false));
}

// Treelets, predictor-corrector encoding and serialisation of a built tree.  `nodes` in
// BFS order (a leaf's `tri` is its triangle, or its position in the split order for a
// plan), `lat` the exact lattice bounds of every node (zeros for a plan).  With verts_host
// NULL the triangle table stays zero and the leaves' positions go to h->leaf_pos.
int layout(cbvh_bvh *h, const std::vector<Node> &nodes, const std::vector<int32_t> &lat, const float *verts_host,
           const int32_t *tris_host, int64_t n_tris) {
  const int k = h->k, K = h->K, branching = h->m, quant_bits = h->bits, treelet_bytes = h->treelet_bytes;
  const int64_t nn = (int64_t)nodes.size();
  for (const Node &nd : nodes) h->depth = std::max(h->depth, nd.depth);
  // record sizes the treelet formation assumes: Stream VByte records vary, so treelets are
  // formed with the largest record plus its offset-table entry (and the root with its entry
  // and the table's padding to 8 bytes, which keeps the absolute root record 8-byte
  // aligned), which keeps every treelet within its budget
  const bool svb = quant_bits == CBVH_QUANT_SVB;
  const int64_t form_root = h->root_bytes + (svb ? 8 : 0), form_rec = h->rec_bytes + (svb ? 2 : 0);
  // ---- treelets ----
  std::vector<int32_t> tlet(nn), local(nn), child_tlet(nn, -1);
  std::vector<uint8_t> ext(nn, 0);
  std::vector<int32_t> roots{0};
  std::vector<std::vector<int32_t>> members;
  const int packing = cbvh::treelet_packing();
  if (packing == CBVH_PACK_BOTTOM_UP) {
    // Bottom-up: `carry` counts the nodes of a subtree not yet cut off.  A node keeps its
    // children while it and everything they carry fit one treelet; else every child roots
    // a treelet of its own.  Treelets are numbered in node (BFS) order of their roots.
    const int64_t fit = (treelet_bytes - 16 - form_root) / form_rec + 1;
    std::vector<int64_t> carry(nn, 1);
    for (int64_t x = nn - 1; x >= 0; --x) {
      const Node &nd = nodes[x];
      int64_t c = 1;
      for (int i = 0; i < nd.count; ++i) c += carry[nd.first + i];
      if (c <= fit)
        carry[x] = c;
      else
        ext[x] = 1;
    }
    std::vector<int32_t> tl_of(nn, -1);
    tl_of[0] = 0;
    for (int64_t x = 1; x < nn; ++x)
      if (ext[nodes[x].parent]) {
        tl_of[x] = (int32_t)roots.size();
        roots.push_back((int32_t)x);
      }
    members.resize(roots.size());
    for (size_t t = 0; t < roots.size(); ++t) {
      std::vector<int32_t> &mem = members[t];
      mem.push_back(roots[t]);
      for (size_t i = 0; i < mem.size(); ++i) {
        const int32_t x = mem[i];
        tlet[x] = (int32_t)t;
        local[x] = (int32_t)i;
        const Node &nd = nodes[x];
        if (ext[x])
          child_tlet[x] = tl_of[nd.first];
        else
          for (int c = 0; c < nd.count; ++c) mem.push_back(nd.first + c);
      }
    }
  } else {
    // Top-down: greedy BFS from each root adding whole sibling groups inside the budget; a
    // group that does not fit makes each of its nodes a new treelet root, numbered in the
    // order of creation.
    for (size_t t = 0; t < roots.size(); ++t) {
      std::vector<int32_t> mem{roots[t]};
      tlet[roots[t]] = (int32_t)t;
      local[roots[t]] = 0;
      int64_t used_bytes = 16 + form_root;
      for (size_t i = 0; i < mem.size(); ++i) {  // `mem` doubles as the BFS queue
        const Node &nd = nodes[mem[i]];
        if (nd.count == 0) continue;
        int64_t need = (int64_t)nd.count * form_rec;
        if (used_bytes + need <= treelet_bytes) {
          used_bytes += need;
          for (int c = 0; c < nd.count; ++c) {
            tlet[nd.first + c] = (int32_t)t;
            local[nd.first + c] = (int32_t)mem.size();
            mem.push_back(nd.first + c);
          }
        } else {
          ext[mem[i]] = 1;
          child_tlet[mem[i]] = (int32_t)roots.size();
          for (int c = 0; c < nd.count; ++c) roots.push_back(nd.first + c);
        }
      }
      members.push_back(std::move(mem));
    }
  }
  const int64_t ntl = (int64_t)roots.size();
  size_t maxn = 1;
  for (auto &mm : members) maxn = std::max(maxn, mm.size());
  if (maxn > 65535) {
    return cbvh::fail(CBVH_ERR_ARG, "too many nodes in one treelet");
  }
  while (((size_t)1 << h->lbits) < maxn) ++h->lbits;
  if (h->lbits < 32 && (uint64_t)ntl >= ((uint64_t)1 << (32 - h->lbits))) {
    return cbvh::fail(CBVH_ERR_ARG, "too many treelets for 32-bit node references; use larger treelets");
  }

  // ---- predictor-corrector encoding, top-down (parents precede children in BFS) ----
  std::vector<int32_t> dec((size_t)nn * K * 2);
  std::vector<uint16_t> corr((size_t)nn * K * 2, 0);
  std::vector<uint32_t> sv(svb ? (size_t)nn * K * 2 : 0, 0);  // Stream VByte: exact deltas
  const uint32_t dmax = quant_bits >= 8 ? (1u << quant_bits) - 1 : 0;
  for (int64_t x = 0; x < nn; ++x) {
    const int32_t *C = &lat[(size_t)x * K * 2];
    int32_t *D = &dec[(size_t)x * K * 2];
    if (local[x] == 0 || quant_bits == 0 || quant_bits == CBVH_QUANT_FP16) {
      std::copy(C, C + 2 * K, D);
      continue;
    }
    if (svb) {  // lossless: the unshifted deltas to the parent's exact interval
      const int32_t *P = &lat[(size_t)nodes[x].parent * K * 2];
      for (int j = 0; j < K; ++j) {
        sv[(size_t)x * K * 2 + 2 * j] = (uint32_t)((int64_t)C[2 * j] - P[2 * j]);
        sv[(size_t)x * K * 2 + 2 * j + 1] = (uint32_t)((int64_t)P[2 * j + 1] - C[2 * j + 1]);
      }
      std::copy(C, C + 2 * K, D);
      continue;
    }
    const int32_t *P = &dec[(size_t)nodes[x].parent * K * 2];
    for (int j = 0; j < K; ++j) {
      uint32_t range = (uint32_t)((int64_t)P[2 * j + 1] - P[2 * j]);
      int s = 0;
      while ((range >> s) > dmax) ++s;
      uint32_t dl = (uint32_t)((int64_t)C[2 * j] - P[2 * j]) >> s;
      uint32_t dh = (uint32_t)((int64_t)P[2 * j + 1] - C[2 * j + 1]) >> s;
      corr[(size_t)x * K * 2 + 2 * j] = (uint16_t)dl;
      corr[(size_t)x * K * 2 + 2 * j + 1] = (uint16_t)dh;
      D[2 * j] = (int32_t)((int64_t)P[2 * j] + ((int64_t)dl << s));
      D[2 * j + 1] = (int32_t)((int64_t)P[2 * j + 1] - ((int64_t)dh << s));
    }
  }

  // ---- serialise ----
  std::vector<int64_t> toff(ntl + 1);
  int64_t pos = (64 + 8 * (ntl + 1) + 15) / 16 * 16;
  h->off_treelets = pos;
  auto svb_len = [](uint32_t v) { return v < (1u << 8) ? 1 : v < (1u << 16) ? 2 : v < (1u << 24) ? 3 : 4; };
  auto rec_size = [&](int64_t x, bool root) -> int64_t {  // bytes of x's record
    if (root) return h->root_bytes;
    if (!svb) return h->rec_bytes;
    int64_t n = 16;
    for (int i = 0; i < 2 * K; ++i) n += svb_len(sv[(size_t)x * K * 2 + i]);
    return (n + 3) / 4 * 4;
  };
  auto table_bytes = [&](int64_t count) -> int64_t { return svb ? (2 * count + 7) / 8 * 8 : 0; };
  for (int64_t t = 0; t < ntl; ++t) {
    toff[t] = pos;
    int64_t sz = 16 + table_bytes((int64_t)members[t].size());
    for (size_t l = 0; l < members[t].size(); ++l) sz += rec_size(members[t][l], l == 0);
    pos += (sz + 15) / 16 * 16;
  }
  toff[ntl] = pos;
  h->off_tris = pos;
  const int64_t total = pos + 48 * n_tris;
  std::vector<uint8_t> &b = h->blob;
  b.assign(total, 0);
  int max_td = 0;
  std::vector<int32_t> leaf_slot(nn, -1), slot_tri;
  slot_tri.reserve(n_tris);
  for (int64_t x = 0; x < nn; ++x)
    if (nodes[x].count == 0) {
      leaf_slot[x] = (int32_t)slot_tri.size();
      slot_tri.push_back(nodes[x].tri);
    }
  int64_t first_node = 0;
  for (int64_t t = 0; t < ntl; ++t) {
    const auto &mem = members[t];
    const int64_t T0 = toff[t];
    w32(b, T0, (uint32_t)mem.size());
    w32(b, T0 + 4, (uint32_t)first_node);
    first_node += (int64_t)mem.size();
    std::vector<int> tdepth(mem.size(), 0);
    int64_t at = 16 + table_bytes((int64_t)mem.size());  // next record, from the treelet start
    for (size_t l = 0; l < mem.size(); ++l) {
      const int32_t x = mem[l];
      const Node &nd = nodes[x];
      if (l) tdepth[l] = tdepth[local[nd.parent]] + 1;
      max_td = std::max(max_td, tdepth[l]);
      const int64_t R = T0 + at;
      if (svb) w16(b, T0 + 16 + 2 * (int64_t)l, (uint16_t)(at / 4));
      at += rec_size(x, l == 0);
      uint32_t w0 = (l ? (uint32_t)local[nd.parent] : 0xFFFFu) | ((uint32_t)nd.count << 16) |
                    ((uint32_t)ext[x] << 21) | ((uint32_t)tdepth[l] << 24);
      uint32_t w1 = nd.count == 0 ? (uint32_t)leaf_slot[x]
                                  : (ext[x] ? (uint32_t)child_tlet[x] : (uint32_t)local[nd.first]);
      w32(b, R, w0);
      w32(b, R + 4, w1);
      const int32_t *D = &dec[(size_t)x * K * 2];
      if (svb && l) {  // Stream VByte: control word, then each delta in its fewest bytes
        uint64_t ctl = 0;
        int64_t q = R + 16;
        for (int i = 0; i < 2 * K; ++i) {
          const uint32_t v = sv[(size_t)x * K * 2 + i];
          const int len = svb_len(v);
          ctl |= (uint64_t)(len - 1) << (2 * i);
          for (int y = 0; y < len; ++y) b[q++] = (uint8_t)(v >> (8 * y));
        }
        w64(b, R + 8, ctl);
        continue;
      }
      for (int j = 0; j < K; ++j) {
        if (quant_bits == 0) {
          w32(b, R + 8 + 8 * j, f32_bits(to_f32_down(D[2 * j], h->e)));
          w32(b, R + 12 + 8 * j, f32_bits(to_f32_up(D[2 * j + 1], h->e)));
        } else if (quant_bits == CBVH_QUANT_FP16) {  // exact lattice values, rounded outward to half
          w16(b, R + 8 + 4 * j, half_down(std::ldexp((double)D[2 * j], h->e)));
          w16(b, R + 10 + 4 * j, half_up(std::ldexp((double)D[2 * j + 1], h->e)));
        } else if (l == 0) {
          w32(b, R + 8 + 8 * j, (uint32_t)D[2 * j]);
          w32(b, R + 12 + 8 * j, (uint32_t)D[2 * j + 1]);
        } else if (quant_bits == 8) {
          b[R + 8 + 2 * j] = (uint8_t)corr[(size_t)x * K * 2 + 2 * j];
          b[R + 9 + 2 * j] = (uint8_t)corr[(size_t)x * K * 2 + 2 * j + 1];
        } else {
          w16(b, R + 8 + 4 * j, corr[(size_t)x * K * 2 + 2 * j]);
          w16(b, R + 10 + 4 * j, corr[(size_t)x * K * 2 + 2 * j + 1]);
        }
      }
    }
  }
  if (verts_host) {
    for (int64_t i = 0; i < n_tris; ++i) {
      const int64_t P = h->off_tris + 48 * i;
      const int32_t t = slot_tri[i];
      for (int c = 0; c < 3; ++c)
        for (int x = 0; x < 3; ++x) w32(b, P + 16 * c + 4 * x, f32_bits(verts_host[3 * (int64_t)tris_host[3 * (int64_t)t + c] + x]));
      w32(b, P + 12, (uint32_t)t);
    }
  } else {  // a plan: the table stays zero; slot_tri holds each leaf's position in the order
    h->leaf_pos = std::move(slot_tri);
  }
  h->max_tdepth = max_td;
  h->n_tris = n_tris;
  h->n_nodes = nn;
  h->n_treelets = ntl;
  // header
  w32(b, 0, 0x48564243u);
  w16(b, 4, 1);
  b[6] = (uint8_t)k;
  b[7] = (uint8_t)K;
  b[8] = (uint8_t)branching;
  b[9] = (uint8_t)quant_bits;
  b[10] = (uint8_t)h->lbits;
  b[11] = (uint8_t)max_td;
  w32(b, 12, (uint32_t)h->e);
  w32(b, 16, (uint32_t)n_tris);
  w32(b, 20, (uint32_t)nn);
  w32(b, 24, (uint32_t)ntl);
  w32(b, 28, (uint32_t)h->rec_bytes);
  w32(b, 32, (uint32_t)h->root_bytes);
  w32(b, 36, (uint32_t)treelet_bytes);
  w32(b, 40, (uint32_t)h->depth);
  w32(b, 44, (uint32_t)packing);
  w64(b, 48, (uint64_t)h->off_tris);
  w64(b, 56, (uint64_t)total);
  for (int64_t t = 0; t <= ntl; ++t) w64(b, 64 + 8 * t, (uint64_t)toff[t]);
  return CBVH_OK;
}

// Validated parameters and record sizes of a new handle (no mesh data yet).
int new_handle(int64_t n_verts, int64_t n_tris, int k, int branching, int quant_bits, int treelet_bytes,
               cbvh_bvh **out) {
  if (k != 6 && k != 18 && k != 24 && k != 26) return cbvh::fail(CBVH_ERR_ARG, "k must be 6, 18, 24 or 26");
  if (branching != 2 && branching != 4 && branching != 8 && branching != 16)
    return cbvh::fail(CBVH_ERR_ARG, "branching must be 2, 4, 8 or 16");
  if (quant_bits != 0 && quant_bits != CBVH_QUANT_FP16 && quant_bits != CBVH_QUANT_SVB && quant_bits != 8 &&
      quant_bits != 16)
    return cbvh::fail(CBVH_ERR_ARG, "quant_bits must be 0 (FP32), 1 (FP16), 2 (Stream VByte), 8 or 16");
  if (treelet_bytes < 4096 || treelet_bytes > 131072 || (treelet_bytes & (treelet_bytes - 1)))
    return cbvh::fail(CBVH_ERR_ARG, "treelet_bytes must be a power of two in [4096, 131072]");
  if (n_tris < 1 || n_tris > 0x7fffffff || n_verts < 3 || n_verts > 0x7fffffff)
    return cbvh::fail(CBVH_ERR_MESH, "mesh size out of range");

  const int K = k / 2;
  auto h = new cbvh_bvh();
  h->k = k;
  h->K = K;
  h->m = branching;
  h->bits = quant_bits;
  h->treelet_bytes = treelet_bytes;
  if (quant_bits == CBVH_QUANT_FP16) {  // absolute half-precision bounds in every record
    h->root_bytes = h->rec_bytes = 8 + 4 * K;
  } else if (quant_bits == CBVH_QUANT_SVB) {  // absolute root; records of at most 16 + 8K bytes
    h->root_bytes = 8 + 8 * K;
    h->rec_bytes = 16 + 8 * K;
  } else {
    h->root_bytes = 8 + 8 * K;
    h->rec_bytes = quant_bits == 0 ? h->root_bytes : (8 + 2 * K * (quant_bits / 8) + 3) / 4 * 4;
  }
  const int svb_extra = quant_bits == CBVH_QUANT_SVB ? 8 + 2 * branching : 0;  // offset-table entries
  if (16 + h->root_bytes + branching * h->rec_bytes + svb_extra > treelet_bytes) {
    delete h;
    return cbvh::fail(CBVH_ERR_ARG, "treelet_bytes too small for one sibling group");
  }
  h->n_tris = n_tris;
  h->n_verts = n_verts;
  *out = h;
  return CBVH_OK;
}


}  // namespace

extern "C" int cbvh_build(const float *verts_host, int64_t n_verts, const int32_t *tris_host, int64_t n_tris, int k,
                          int branching, int quant_bits, int treelet_bytes, cbvh_bvh **out) {
  cbvh::clear_error();
  if (!out) return cbvh::fail(CBVH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!verts_host || !tris_host) return cbvh::fail(CBVH_ERR_ARG, "NULL mesh pointer");
  cbvh_bvh *h = nullptr;
  if (int rc = new_handle(n_verts, n_tris, k, branching, quant_bits, treelet_bytes, &h)) return rc;
  const int K = h->K;

  Builder B{k, K, branching, quant_bits, treelet_bytes, verts_host, n_verts, tris_host, n_tris};
  for (int64_t i = 0; i < 3 * n_verts; ++i)
    if (!std::isfinite(verts_host[i])) {
      delete h;
      return cbvh::fail(CBVH_ERR_MESH, "non-finite vertex coordinate");
    }
  B.key.resize(3 * n_tris);
  for (int64_t t = 0; t < n_tris; ++t) {
    double p[3][3];
    for (int c = 0; c < 3; ++c) {
      int32_t vi = tris_host[3 * t + c];
      if (vi < 0 || vi >= n_verts) {
        delete h;
        return cbvh::fail(CBVH_ERR_MESH, "triangle " + std::to_string(t) + " has an out-of-range vertex index");
      }
      for (int x = 0; x < 3; ++x) p[c][x] = verts_host[3 * (int64_t)vi + x];
    }
    double a[3], b[3];
    for (int x = 0; x < 3; ++x) {
      a[x] = p[1][x] - p[0][x];
      b[x] = p[2][x] - p[0][x];
    }
    double nx = a[1] * b[2] - a[2] * b[1], ny = a[2] * b[0] - a[0] * b[2], nz = a[0] * b[1] - a[1] * b[0];
    if (nx == 0.0 && ny == 0.0 && nz == 0.0) {
      delete h;
      return cbvh::fail(CBVH_ERR_MESH, "triangle " + std::to_string(t) + " is degenerate (zero area)");
    }
    for (int x = 0; x < 3; ++x) B.key[3 * t + x] = (p[0][x] + p[1][x]) + p[2][x];
  }
  B.build_tree();
  const int64_t nn = (int64_t)B.nodes.size();

  // Lattice exponent: the smallest e with |d.v| / 2^e < 2^30 over the referenced vertices.
  // Unreferenced vertices must not influence it: restrict to vertices used by a triangle.
  std::vector<uint8_t> used(n_verts, 0);
  for (int64_t i = 0; i < 3 * n_tris; ++i) used[tris_host[i]] = 1;
  std::vector<float> UV;
  std::vector<int64_t> vmap(n_verts, -1);
  for (int64_t v = 0; v < n_verts; ++v)
    if (used[v]) {
      vmap[v] = (int64_t)UV.size() / 3;
      UV.insert(UV.end(), verts_host + 3 * v, verts_host + 3 * v + 3);
    }
  Builder E = B;
  E.V = UV.data();
  E.nv = (int64_t)UV.size() / 3;
  {
    double M = 0;
    for (int64_t v = 0; v < E.nv; ++v)
      for (int j = 0; j < K; ++j) {
        double s = kDir[j][0] * (double)UV[3 * v] + kDir[j][1] * (double)UV[3 * v + 1] + kDir[j][2] * (double)UV[3 * v + 2];
        M = std::max(M, std::fabs(s));
      }
    if (M == 0.0) {
      delete h;
      return cbvh::fail(CBVH_ERR_MESH, "mesh has no extent");
    }
    int ex = std::ilogb(M) - 29;  // 2^(ilogb M + 1) > M: fits unless rounding says otherwise
    E.headroom = cbvh::lattice_headroom();
    while (!E.fits(ex)) ++ex;
    while (E.fits(ex - 1)) --ex;
    if (ex < -120 || ex > 96) {
      delete h;
      return cbvh::fail(CBVH_ERR_MESH, "mesh coordinates outside the supported range");
    }
    h->e = ex;
  }
  // per-vertex lattice values, then node bounds bottom-up (children follow parents in BFS)
  std::vector<int32_t> vl((size_t)E.nv * K * 2);
  for (int64_t v = 0; v < E.nv; ++v)
    for (int j = 0; j < K; ++j) {
      double t[3];
      for (int c = 0; c < 3; ++c) t[c] = kDir[j][c] * std::ldexp((double)UV[3 * v + c], -h->e);
      vl[(v * K + j) * 2] = (int32_t)exact_floor(t[0], t[1], t[2]);
      vl[(v * K + j) * 2 + 1] = (int32_t)exact_ceil(t[0], t[1], t[2]);
    }
  std::vector<int32_t> lat((size_t)nn * K * 2);
  for (int64_t x = nn - 1; x >= 0; --x) {
    int32_t *L = &lat[(size_t)x * K * 2];
    for (int j = 0; j < K; ++j) {
      L[2 * j] = std::numeric_limits<int32_t>::max();
      L[2 * j + 1] = std::numeric_limits<int32_t>::min();
    }
    const Node &nd = B.nodes[x];
    if (nd.count == 0) {
      for (int c = 0; c < 3; ++c) {
        const int32_t *P = &vl[(size_t)vmap[tris_host[3 * (int64_t)nd.tri + c]] * K * 2];
        for (int j = 0; j < K; ++j) {
          L[2 * j] = std::min(L[2 * j], P[2 * j]);
          L[2 * j + 1] = std::max(L[2 * j + 1], P[2 * j + 1]);
        }
      }
    } else {
      for (int c = 0; c < nd.count; ++c) {
        const int32_t *P = &lat[(size_t)(nd.first + c) * K * 2];
        for (int j = 0; j < K; ++j) {
          L[2 * j] = std::min(L[2 * j], P[2 * j]);
          L[2 * j + 1] = std::max(L[2 * j + 1], P[2 * j + 1]);
        }
      }
    }
  }
  if (quant_bits == CBVH_QUANT_FP16)  // every bound lies inside the root's: check the root
    for (int j = 0; j < 2 * K; ++j)
      if (std::fabs(std::ldexp((double)lat[j], h->e)) > 65504.0) {
        delete h;
        return cbvh::fail(CBVH_ERR_MESH, "mesh bounds exceed the half-precision range (+-65504) of quant_bits = 1");
      }

  h->headroom = E.headroom;
  if (int rc = layout(h, B.nodes, lat, verts_host, tris_host, n_tris)) {
    delete h;
    return rc;
  }
  h->n_verts = n_verts;
  h->geometry = true;
  *out = h;
  return CBVH_OK;
}

extern "C" int cbvh_build_plan(int64_t n_verts, int64_t n_tris, int k, int branching, int quant_bits,
                               int treelet_bytes, cbvh_bvh **out) {
  cbvh::clear_error();
  if (!out) return cbvh::fail(CBVH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (quant_bits == CBVH_QUANT_SVB)
    return cbvh::fail(CBVH_ERR_ARG, "the device build needs fixed-size records (quant_bits 0, 1, 8 or 16)");
  cbvh_bvh *h = nullptr;
  if (int rc = new_handle(n_verts, n_tris, k, branching, quant_bits, treelet_bytes, &h)) return rc;
  // the tree's shape depends on n_tris and the branching alone: split nothing, keep positions
  Builder B{k, h->K, branching, quant_bits, treelet_bytes, nullptr, n_verts, nullptr, n_tris};
  B.build_tree(true);
  const std::vector<int32_t> lat((size_t)B.nodes.size() * h->K * 2, 0);
  if (int rc = layout(h, B.nodes, lat, nullptr, nullptr, n_tris)) {
    delete h;
    return rc;
  }
  h->headroom = cbvh::lattice_headroom();
  h->geometry = false;
  *out = h;
  return CBVH_OK;
}

namespace {
uint16_t rd16(const std::vector<uint8_t> &b, int64_t o) {
  uint16_t v;
  std::memcpy(&v, &b[o], 2);
  return v;
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

// Checks every part of a blob the kernels rely on and fills the handle's fields from its
// header.  Returns "" or the first failed check.
std::string check_blob(const std::vector<uint8_t> &b, cbvh_bvh *h) {
  const int64_t n = (int64_t)b.size();
  if (n < 64) return "shorter than its header";
  if (rd32(b, 0) != 0x48564243u || rd16(b, 4) != 1) return "not a version-1 hierarchy blob";
  const int k = b[6], K = b[7], m = b[8], bits = b[9], lbits = b[10], max_td = b[11];
  const int e = (int32_t)rd32(b, 12);
  const int64_t nt = rd32(b, 16), nn = rd32(b, 20), ntl = rd32(b, 24);
  const int rec = (int)rd32(b, 28), root = (int)rd32(b, 32), tb = (int)rd32(b, 36);
  const int depth = (int)rd32(b, 40), packing = (int)rd32(b, 44);
  const int64_t off_tris = (int64_t)rd64(b, 48), total = (int64_t)rd64(b, 56);
  if ((k != 6 && k != 18 && k != 24 && k != 26) || K != k / 2) return "bad k";
  if (m != 2 && m != 4 && m != 8 && m != 16) return "bad branching";
  if (bits != 0 && bits != CBVH_QUANT_FP16 && bits != CBVH_QUANT_SVB && bits != 8 && bits != 16)
    return "bad quant_bits";
  if (tb < 4096 || tb > 131072 || (tb & (tb - 1))) return "bad treelet budget";
  if (packing != CBVH_PACK_TOP_DOWN && packing != CBVH_PACK_BOTTOM_UP) return "bad treelet packing";
  if (e < -120 || e > 96) return "bad lattice exponent";
  int want_root = 8 + 8 * K, want_rec;
  if (bits == CBVH_QUANT_FP16)
    want_root = want_rec = 8 + 4 * K;
  else if (bits == CBVH_QUANT_SVB)
    want_rec = 16 + 8 * K;
  else
    want_rec = bits == 0 ? want_root : (8 + 2 * K * (bits / 8) + 3) / 4 * 4;
  if (rec != want_rec || root != want_root) return "record sizes do not match the mode";
  if (nt < 1 || nn < 1 || ntl < 1 || nn < nt) return "bad counts";
  if (lbits < 1 || lbits > 16 || (uint64_t)ntl >= ((uint64_t)1 << (32 - lbits))) return "bad node reference split";
  if (total != n) return "size does not match the header";
  const int64_t tab_end = 64 + 8 * (ntl + 1);
  if (tab_end > n) return "treelet table outside the blob";
  std::vector<int64_t> toff(ntl + 1);
  for (int64_t t = 0; t <= ntl; ++t) toff[t] = (int64_t)rd64(b, 64 + 8 * t);
  if (toff[0] != (tab_end + 15) / 16 * 16) return "first treelet misplaced";
  for (int64_t t = 0; t < ntl; ++t)
    if (toff[t + 1] <= toff[t] || (toff[t] & 15) || toff[t + 1] > n) return "treelet offsets out of order";
  if (toff[ntl] != off_tris || off_tris + 48 * nt != total) return "triangle table misplaced";
  const bool svb = bits == CBVH_QUANT_SVB;
  // depth of each treelet's root, from the external references (each treelet but the first
  // is referenced exactly once, by a node of an earlier treelet)
  std::vector<int> troot_depth(ntl, -1);
  troot_depth[0] = 0;
  std::vector<uint8_t> slot_used(nt, 0);
  int64_t nodes = 0, leaves = 0;
  int max_depth = 0, max_tdepth = 0;
  for (int64_t t = 0; t < ntl; ++t) {
    const int64_t T = toff[t], size = toff[t + 1] - T;
    if (size < 16) return "treelet too small";
    const int64_t cnt = rd32(b, T);
    if (cnt < 1 || cnt >= ((int64_t)1 << lbits)) return "bad treelet node count";
    if ((int64_t)rd32(b, T + 4) != nodes) return "treelet header: wrong first-node index";
    if (troot_depth[t] < 0) return "treelet not referenced by its parent";
    std::vector<int64_t> pos(cnt);
    if (svb) {
      const int64_t first = 16 + (2 * cnt + 7) / 8 * 8;
      if (first + root > size) return "treelet too small for its offset table";
      int64_t end = 0;
      for (int64_t l = 0; l < cnt; ++l) {
        const int64_t o = 4 * (int64_t)rd16(b, T + 16 + 2 * l);
        if ((l == 0 && o != first) || (l > 0 && o < end) || o + (l ? 16 : root) > size) return "bad record offset";
        pos[l] = o;
        if (l == 0) {
          end = o + root;
        } else {  // the record's deltas, by its control word, stay before the next record
          const uint64_t ctl = rd64(b, T + o + 8);
          int64_t bytes = 16;
          for (int i = 0; i < 2 * K; ++i) bytes += (int64_t)((ctl >> (2 * i)) & 3u) + 1;
          end = o + (bytes + 3) / 4 * 4;
          if (end > size) return "record runs past its treelet";
        }
      }
    } else {
      if (16 + root + (cnt - 1) * (int64_t)rec > size) return "treelet too small for its records";
      for (int64_t l = 0; l < cnt; ++l) pos[l] = 16 + (l ? root + (l - 1) * (int64_t)rec : 0);
    }
    std::vector<int> td(cnt, 0);
    // the node whose child range holds each node of the treelet: the decode walks a node's
    // chain through its parent field, so that field must name the node that references it,
    // and no node may be referenced twice
    std::vector<int64_t> owner(cnt, -1);
    for (int64_t l = 0; l < cnt; ++l) {
      const uint32_t w0 = rd32(b, T + pos[l]), w1 = rd32(b, T + pos[l] + 4);
      const uint32_t par = w0 & 0xffffu, nc = (w0 >> 16) & 31u, ext = (w0 >> 21) & 1u, d = w0 >> 24;
      if (l == 0 ? (par != 0xffffu || d != 0) : (par >= (uint32_t)l || d != (uint32_t)td[par] + 1))
        return "bad parent or depth";
      if (l > 0 && owner[l] != (int64_t)par) return "parent field does not name the referencing node";
      if (((w0 >> 22) & 3u) != 0 || nc > (uint32_t)m) return "bad child count";
      td[l] = (int)d;
      max_tdepth = std::max(max_tdepth, (int)d);
      const int node_depth = troot_depth[t] + (int)d;
      max_depth = std::max(max_depth, node_depth);
      if (nc == 0) {
        if (ext || w1 >= (uint64_t)nt || slot_used[w1]) return "bad leaf slot";
        slot_used[w1] = 1;
        ++leaves;
      } else if (ext) {
        if ((uint64_t)w1 + nc > (uint64_t)ntl || w1 <= (uint64_t)t) return "bad child treelet";
        for (uint32_t c = 0; c < nc; ++c) {
          if (troot_depth[w1 + c] >= 0) return "treelet referenced twice";
          troot_depth[w1 + c] = node_depth + 1;
        }
      } else if (w1 <= (uint64_t)l || (uint64_t)w1 + nc > (uint64_t)cnt) {
        return "bad child index";
      } else {
        for (uint32_t c = 0; c < nc; ++c) {
          if (owner[w1 + c] >= 0) return "node referenced twice";
          owner[w1 + c] = l;
        }
      }
    }
    nodes += cnt;
  }
  if (nodes != nn || leaves != nt) return "node or leaf count does not match the header";
  if (max_depth != depth || max_tdepth != max_td) return "depths do not match the header";
  for (int64_t i = 0; i < nt; ++i)
    if (rd32(b, off_tris + 48 * i + 12) >= (uint64_t)nt) return "bad triangle index";
  h->k = k;
  h->K = K;
  h->m = m;
  h->bits = bits;
  h->treelet_bytes = tb;
  h->e = e;
  h->lbits = lbits;
  h->max_tdepth = max_td;
  h->depth = depth;
  h->rec_bytes = rec;
  h->root_bytes = root;
  h->n_tris = nt;
  h->n_nodes = nn;
  h->n_treelets = ntl;
  h->off_treelets = toff[0];
  h->off_tris = off_tris;
  return "";
}
}  // namespace

extern "C" int cbvh_save(const cbvh_bvh *h, const char *path) {
  cbvh::clear_error();
  if (!h || !path) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (!h->geometry) return cbvh::fail(CBVH_ERR_STATE, "a plan has no geometry to save");
  if (h->host_stale)
    return cbvh::fail(CBVH_ERR_STATE, "host blob not updated by the device build (CBVH_BUILD_HOST_COPY not given)");
  FILE *f = std::fopen(path, "wb");
  if (!f) return cbvh::fail(CBVH_ERR_IO, std::string("cannot open ") + path + " for writing");
  uint8_t head[16] = {'C', 'B', 'V', 'F', 1, 0, 0, 0};
  const int64_t nv = h->n_verts;
  std::memcpy(head + 8, &nv, 8);
  bool ok = std::fwrite(head, 1, 16, f) == 16 && std::fwrite(h->blob.data(), 1, h->blob.size(), f) == h->blob.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? CBVH_OK : cbvh::fail(CBVH_ERR_IO, std::string("cannot write ") + path);
}

extern "C" int cbvh_load(const char *path, cbvh_bvh **out) {
  cbvh::clear_error();
  if (!path || !out) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) return cbvh::fail(CBVH_ERR_IO, std::string("cannot open ") + path);
  std::vector<uint8_t> data;
  uint8_t buf[1 << 16];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) data.insert(data.end(), buf, buf + got);
  const bool err = std::ferror(f) != 0;
  std::fclose(f);
  if (err) return cbvh::fail(CBVH_ERR_IO, std::string("cannot read ") + path);
  if (data.size() < 16 || std::memcmp(data.data(), "CBVF\x01\0\0\0", 8) != 0)
    return cbvh::fail(CBVH_ERR_IO, "not a saved hierarchy (bad file header)");
  int64_t nv;
  std::memcpy(&nv, data.data() + 8, 8);
  auto h = new cbvh_bvh();
  h->blob.assign(data.begin() + 16, data.end());
  const std::string why = check_blob(h->blob, h);
  if (!why.empty() || nv < 3 || nv > 0x7fffffff) {
    delete h;
    return cbvh::fail(CBVH_ERR_IO, "invalid hierarchy file: " + (why.empty() ? std::string("bad vertex count") : why));
  }
  h->n_verts = nv;
  h->geometry = true;
  *out = h;
  return CBVH_OK;
}

extern "C" int cbvh_free(cbvh_bvh *h) {
  delete h;
  return CBVH_OK;
}

extern "C" int cbvh_info(const cbvh_bvh *h, cbvh_info_t *o) {
  cbvh::clear_error();
  if (!h || !o) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  o->n_tris = h->n_tris;
  o->n_nodes = h->n_nodes;
  o->n_treelets = h->n_treelets;
  o->blob_bytes = (int64_t)h->blob.size();
  o->node_bytes = h->off_tris - h->off_treelets;
  o->k = h->k;
  o->branching = h->m;
  o->quant_bits = h->bits;
  o->treelet_bytes = h->treelet_bytes;
  o->lattice_exp = h->e;
  o->depth = h->depth;
  o->max_treelet_depth = h->max_tdepth;
  o->local_bits = h->lbits;
  return CBVH_OK;
}

extern "C" int cbvh_blob_host(const cbvh_bvh *h, const uint8_t **blob, int64_t *bytes) {
  cbvh::clear_error();
  if (!h || !blob || !bytes) return cbvh::fail(CBVH_ERR_ARG, "NULL argument");
  if (h->host_stale)
    return cbvh::fail(CBVH_ERR_STATE, "host blob not updated by the device build (CBVH_BUILD_HOST_COPY not given)");
  *blob = h->blob.data();
  *bytes = (int64_t)h->blob.size();
  return CBVH_OK;
}

namespace cbvh {
namespace {
thread_local std::string g_err;
std::atomic<int> g_packing{CBVH_PACK_TOP_DOWN};
std::atomic<int> g_headroom{0};
}  // namespace
void set_treelet_packing(int p) { g_packing.store(p); }
int treelet_packing() { return g_packing.load(); }
void set_lattice_headroom(int bits) { g_headroom.store(bits); }
int lattice_headroom() { return g_headroom.load(); }
int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
void clear_error() { g_err.clear(); }
}  // namespace cbvh

extern "C" const char *cbvh_last_error(void) { return cbvh::g_err.c_str(); }
