/*
 * oracle.c -- plain, slow FP64 CPU oracle for compressed k-DOP BVH collision detection (CD)
 * and proximity query (PQ), after Tan, Weller & Zachmann, "Compressed Bounding Volume
 * Hierarchies for Collision Detection & Proximity Query" (arXiv 2012.05348).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header, table or helper with the CUDA
 * engine; the only common ground is the written blob format and the seeded input generators.
 *
 * What it computes, and where the paper defines it:
 *   - k-DOP bounding volumes, "k floats" per node (Table 1), over fixed integer directions.
 *   - the BVH, built by recursive splitting and wrapping (Sec. I); the split rule is the
 *     engine's documented reading (median split on the longest centroid axis).
 *   - quantised bounds ("we quantify BV", abstract) on one absolute lattice per BVH, and the
 *     predictor-corrector encoding of Sec. III-B: the predictor of a node is its parent's
 *     decoded interval (itself a function of the chain of ancestors up to the treelet root,
 *     abstract and Sec. V), the corrector a small unsigned delta rounded outward.
 *   - treelets: the BVH clustered into parts of a byte budget (Sec. III-B), each root stored
 *     absolutely so every treelet is randomly accessible (abstract).
 *   - the integer-compression alternative the conclusion proposes (quant_bits = 2): the
 *     quantised bounds kept exact, each node's lattice interval stored as unsigned deltas to
 *     its parent's, written in the Stream VByte format (Lemire, Kurz and Rupp 2018).
 *   - an independent decoder of the blob bytes.
 *   - simultaneous traversal, Algorithm 1 (BVHtraversal), recursive exactly as printed, with
 *     checkPrimitives = closed triangle-triangle intersection (CD) or triangle-triangle
 *     distance (PQ); the paper leaves checkPrimitives undefined.
 *   - brute force over all triangle pairs, and the near-contact pose filter used to make
 *     FP32-vs-FP64 parity well posed.
 *
 * Everything is FP64 except where the blob format fixes FP32 (decoded float bounds).
 * Compile with -ffp-contract=off: the exact lattice arithmetic relies on unfused adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_MESH (-2)
#define OR_ERR_MEM (-8)

static char or_err[256];
const char *or_last_error(void) { return or_err; }
static int fail(int code, const char *msg) {
  snprintf(or_err, sizeof or_err, "%s", msg);
  return code;
}

/* ------------------------------------------------------------------ k-DOP directions */
/* Unnormalised integer directions; a k-DOP uses the first k/2 of them (Table 1: k values
 * per node = a [lo, hi] slab for each of k/2 directions).  k = 6 is the AABB, 18 the usual
 * 18-DOP, 26 the full 26-DOP, 24 the 26-DOP without its last corner direction. */
static const int OR_DIR[13][3] = {
    {1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, -1, 0}, {1, 0, 1},  {1, 0, -1},
    {0, 1, 1},  {0, 1, -1}, {1, 1, 1},  {1, 1, -1}, {1, -1, 1}, {-1, 1, 1},
};

/* ------------------------------------------------------------------ exact lattice */
/* Knuth/Moller TwoSum: s + e == a + b exactly (round-to-nearest, no overflow). */
static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *s = x;
  *e = (a - av) + (b - bv);
}

/* Exact floor(a + b + c) for doubles a, b, c.  Shewchuk's Grow-Expansion (1997) turns the
 * sum into a non-overlapping expansion h0 + h1 + h2 (increasing magnitude); the floor of an
 * expansion is read from its largest component down: an integer component passes through,
 * and the first non-integer one decides, because every smaller component is below its
 * lowest set bit. */
static int64_t floor3(double a, double b, double c) {
  double s1, e1, q, h0, h1;
  two_sum(a, b, &s1, &e1); /* a + b = s1 + e1, a non-overlapping expansion [e1, s1] */
  two_sum(c, e1, &q, &h0); /* Grow-Expansion by c: Q = c; (Q, h0) = TwoSum(Q, e1) */
  two_sum(q, s1, &q, &h1); /*                      (Q, h1) = TwoSum(Q, s1); h2 = Q */
  const double h[3] = {h0, h1, q};
  int64_t acc = 0;
  for (int i = 2; i >= 0; --i) {
    double f = floor(h[i]);
    if (f != h[i]) return acc + (int64_t)f;
    acc += (int64_t)h[i];
  }
  return acc;
}
static int64_t ceil3(double a, double b, double c) { return -floor3(-a, -b, -c); }

/* Lattice coordinates of d_j . v (v FP32), step 2^e: lo = floor, hi = ceil. */
static void lattice_dv(const float *v, int j, int e, int64_t *lo, int64_t *hi) {
  double t[3];
  for (int c = 0; c < 3; ++c) t[c] = (double)OR_DIR[j][c] * ldexp((double)v[c], -e);
  *lo = floor3(t[0], t[1], t[2]);
  *hi = ceil3(t[0], t[1], t[2]);
}

int64_t or_floor_sum3(double a, double b, double c) { return floor3(a, b, c); }
int64_t or_ceil_sum3(double a, double b, double c) { return ceil3(a, b, c); }
void or_lattice_dv(const float *v, int j, int e, int64_t *lo, int64_t *hi) { lattice_dv(v, j, e, lo, hi); }

/* RD / RU conversion of a lattice integer to FP32, then exact scaling by 2^e. */
static float f32_rd(int64_t L, int e) {
  float f = (float)L;
  if ((double)f > (double)L) f = nextafterf(f, -INFINITY);
  return ldexpf(f, e);
}
static float f32_ru(int64_t L, int e) {
  float f = (float)L;
  if ((double)f < (double)L) f = nextafterf(f, INFINITY);
  return ldexpf(f, e);
}

/* IEEE 754 binary16 (the half floats of Sec. III-A): value of a bit pattern, by the format's
 * definition -- sign, 5-bit exponent with bias 15, 10-bit fraction, subnormals at exponent 0,
 * infinity at exponent 31 with zero fraction. */
static double half_value(uint32_t h) {
  int sign = (h >> 15) & 1, ex = (h >> 10) & 31, fr = h & 1023;
  double v;
  if (ex == 0)
    v = ldexp((double)fr, -24);
  else if (ex == 31)
    v = INFINITY;
  else
    v = ldexp(1024.0 + fr, ex - 25);
  return sign ? -v : v;
}
/* Outward rounding of v to half precision: the largest half <= v (down) or the smallest
 * half >= v (up).  Non-negative patterns 0x0000..0x7c00 are ordered like their values, so
 * a binary search over them finds the neighbours of |v|; negative v mirrors. */
static uint32_t half_search(double a, int up) { /* a >= 0 */
  uint32_t lo = 0, hi = 0x7c00u;
  if (up) { /* smallest pattern with value >= a */
    while (lo < hi) {
      uint32_t mid = (lo + hi) / 2;
      if (half_value(mid) >= a) hi = mid; else lo = mid + 1;
    }
    return lo;
  }
  while (lo < hi) { /* largest pattern with value <= a */
    uint32_t mid = (lo + hi + 1) / 2;
    if (half_value(mid) <= a) lo = mid; else hi = mid - 1;
  }
  return lo;
}
static uint32_t half_rd(double v) { return v >= 0 ? half_search(v, 0) : (0x8000u | half_search(-v, 1)); }
static uint32_t half_ru(double v) { return v >= 0 ? half_search(v, 1) : (0x8000u | half_search(-v, 0)); }
uint32_t or_half_rd(double v) { return half_rd(v); }
uint32_t or_half_ru(double v) { return half_ru(v); }
double or_half_value(uint32_t h) { return half_value(h); }

/* ------------------------------------------------------------------ BVH */
typedef struct {
  int k, K, m, bits, budget;
  int64_t nv, nt;
  float *verts;   /* nv x 3 */
  int32_t *tris;  /* nt x 3 */
  double *key;    /* nt x 3 centroid keys (v0 + v1) + v2 */
  /* tree, BFS numbering (root 0, children of a node consecutive, in split order) */
  int64_t nn;
  int32_t *parent, *first, *nchild, *tri, *depth;
  int32_t tree_depth;
  int32_t *leaf_order; /* node -> position of its triangle in the leaf-ordered table */
  int32_t *leaf_tri;   /* leaf order -> original triangle */
  /* bounds */
  int e;
  int64_t *lat;  /* nn x K x 2 exact lattice */
  double *bnd;   /* nn x K x 2 FP64 bounds of the exact coordinates (own uncompressed BVH) */
  /* encoding */
  int32_t *tlet, *local;
  uint8_t *ext;
  int32_t *child_tlet; /* first child treelet id when ext */
  int64_t *dec;        /* nn x K x 2 decoded lattice */
  uint32_t *delta;     /* nn x K x 2 corrector values */
  float *decf;         /* nn x K x 2 decoded FP32 bounds */
  int64_t ntlet;
  int32_t *tlet_root;  /* treelet -> root node */
  int32_t *tlet_count; /* treelet -> node count */
  int32_t **tlet_nodes;
  int lbits, max_tdepth;
  int rec_bytes, root_bytes;
  int form_rec, form_root; /* record sizes the treelet formation assumes (see or_build) */
  int packing;  /* 0: treelets grown top-down; 1: packed bottom-up (see encode) */
  int headroom; /* lattice bits kept free: e is chosen for |bound| < 2^(30 - headroom) */
  uint8_t *blob;
  int64_t blob_bytes;
} or_bvh;

/* ---- build (median split on the longest centroid axis) ---- */
static const double *g_key;
static int g_axis;
static int cmp_tri(const void *pa, const void *pb) {
  int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
  double ka = g_key[3 * (int64_t)a + g_axis], kb = g_key[3 * (int64_t)b + g_axis];
  if (ka < kb) return -1;
  if (ka > kb) return 1;
  return (a > b) - (a < b);
}

typedef struct {
  int32_t *child; /* temp children */
  int32_t nchild, tri;
} tnode;

typedef struct {
  tnode *n;
  int64_t cnt, cap;
  int m;
} tbuild;

static int32_t tnew(tbuild *b) {
  if (b->cnt == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 1024;
    b->n = (tnode *)realloc(b->n, sizeof(tnode) * b->cap);
  }
  b->n[b->cnt].child = NULL;
  b->n[b->cnt].nchild = 0;
  b->n[b->cnt].tri = -1;
  return (int32_t)b->cnt++;
}

/* Split ids[0..n) in two: sort by (key on the axis of largest centroid extent, index),
 * ties between axes resolved x < y < z; the left part is the first floor(n/2). */
static void split2(const double *key, int32_t *ids, int64_t n) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      double v = key[3 * (int64_t)ids[i] + c];
      if (v < lo[c]) lo[c] = v;
      if (v > hi[c]) hi[c] = v;
    }
  int axis = 0;
  double best = hi[0] - lo[0];
  for (int c = 1; c < 3; ++c)
    if (hi[c] - lo[c] > best) {
      best = hi[c] - lo[c];
      axis = c;
    }
  g_key = key;
  g_axis = axis;
  qsort(ids, (size_t)n, sizeof(int32_t), cmp_tri);
}

static int32_t build_rec(tbuild *b, const double *key, int32_t *ids, int64_t n) {
  int32_t node = tnew(b);
  if (n == 1) {
    b->n[node].tri = ids[0];
    return node;
  }
  /* log2(m) rounds of binary splits; groups of one triangle stop splitting */
  int64_t gs[32], gn[32];
  int ng = 1;
  gs[0] = 0;
  gn[0] = n;
  for (int r = 1; r < b->m; r <<= 1) {
    int64_t ns[32], nn[32];
    int k = 0;
    for (int g = 0; g < ng; ++g) {
      if (gn[g] == 1) {
        ns[k] = gs[g];
        nn[k++] = 1;
        continue;
      }
      split2(key, ids + gs[g], gn[g]);
      int64_t l = gn[g] / 2;
      ns[k] = gs[g];
      nn[k++] = l;
      ns[k] = gs[g] + l;
      nn[k++] = gn[g] - l;
    }
    ng = k;
    memcpy(gs, ns, sizeof(int64_t) * k);
    memcpy(gn, nn, sizeof(int64_t) * k);
  }
  int32_t *ch = (int32_t *)malloc(sizeof(int32_t) * ng);
  for (int g = 0; g < ng; ++g) ch[g] = build_rec(b, key, ids + gs[g], gn[g]);
  b->n[node].child = ch;
  b->n[node].nchild = ng;
  return node;
}

void or_free(or_bvh *h);

/* Every vertex's lattice coordinates within +-lim at exponent e. */
static int lattice_fits(const or_bvh *h, int e, int64_t lim) {
  const int64_t LIM = lim;
  for (int64_t t = 0; t < h->nt; ++t)
    for (int c = 0; c < 3; ++c) {
      const float *v = h->verts + 3 * (int64_t)h->tris[3 * t + c];
      for (int j = 0; j < h->K; ++j) {
        int64_t lo, hi;
        lattice_dv(v, j, e, &lo, &hi);
        if (lo > LIM - 1 || hi < -(LIM - 1)) return 0;
      }
    }
  return 1;
}

static int encode(or_bvh *h);

/* Exact lattice bounds of every node (leaves from their three vertices, inner nodes as the
 * union of their children), and the FP64 bounds of the exact coordinates. */
static void compute_bounds(or_bvh *h) {
  int64_t nn = h->nn;
  int K = h->K;
  if (!h->lat) h->lat = (int64_t *)malloc(sizeof(int64_t) * nn * K * 2);
  if (!h->bnd) h->bnd = (double *)malloc(sizeof(double) * nn * K * 2);
  for (int64_t i = nn - 1; i >= 0; --i) {
    int64_t *L = h->lat + i * K * 2;
    double *B = h->bnd + i * K * 2;
    for (int j = 0; j < K; ++j) {
      L[2 * j] = INT64_MAX;
      L[2 * j + 1] = INT64_MIN;
      B[2 * j] = INFINITY;
      B[2 * j + 1] = -INFINITY;
    }
    if (h->nchild[i] == 0) {
      int32_t t = h->tri[i];
      for (int c = 0; c < 3; ++c) {
        const float *v = h->verts + 3 * (int64_t)h->tris[3 * (int64_t)t + c];
        for (int j = 0; j < K; ++j) {
          int64_t lo, hi;
          lattice_dv(v, j, h->e, &lo, &hi);
          if (lo < L[2 * j]) L[2 * j] = lo;
          if (hi > L[2 * j + 1]) L[2 * j + 1] = hi;
          double s = OR_DIR[j][0] * (double)v[0] + OR_DIR[j][1] * (double)v[1] + OR_DIR[j][2] * (double)v[2];
          if (s < B[2 * j]) B[2 * j] = s;
          if (s > B[2 * j + 1]) B[2 * j + 1] = s;
        }
      }
    } else {
      for (int c = 0; c < h->nchild[i]; ++c) {
        const int64_t *LC = h->lat + (int64_t)(h->first[i] + c) * K * 2;
        const double *BC = h->bnd + (int64_t)(h->first[i] + c) * K * 2;
        for (int j = 0; j < K; ++j) {
          if (LC[2 * j] < L[2 * j]) L[2 * j] = LC[2 * j];
          if (LC[2 * j + 1] > L[2 * j + 1]) L[2 * j + 1] = LC[2 * j + 1];
          if (BC[2 * j] < B[2 * j]) B[2 * j] = BC[2 * j];
          if (BC[2 * j + 1] > B[2 * j + 1]) B[2 * j + 1] = BC[2 * j + 1];
        }
      }
    }
  }
}


/* Build the BVH of a triangle mesh and its compressed blob. */
int or_build(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, int k, int m, int bits,
             int treelet_bytes, int packing, int headroom, or_bvh **out) {
  *out = NULL;
  if (packing != 0 && packing != 1) return fail(OR_ERR_ARG, "packing must be 0 or 1");
  if (headroom < 0 || headroom > 8) return fail(OR_ERR_ARG, "headroom must be in [0, 8]");
  if (k != 6 && k != 18 && k != 24 && k != 26) return fail(OR_ERR_ARG, "k must be 6, 18, 24 or 26");
  if (m != 2 && m != 4 && m != 8 && m != 16) return fail(OR_ERR_ARG, "branching must be 2, 4, 8 or 16");
  if (bits != 0 && bits != 1 && bits != 2 && bits != 8 && bits != 16)
    return fail(OR_ERR_ARG, "quant_bits must be 0 (FP32), 1 (FP16), 2 (Stream VByte), 8 or 16");
  if (treelet_bytes < 4096 || treelet_bytes > 131072 || (treelet_bytes & (treelet_bytes - 1)))
    return fail(OR_ERR_ARG, "treelet_bytes must be a power of two in [4096, 131072]");
  if (nt < 1 || nt > 0x7fffffff || nv < 3 || nv > 0x7fffffff) return fail(OR_ERR_MESH, "bad mesh size");
  or_bvh *h = (or_bvh *)calloc(1, sizeof(or_bvh));
  h->k = k;
  h->K = k / 2;
  h->m = m;
  h->bits = bits;
  h->budget = treelet_bytes;
  h->packing = packing;
  h->headroom = headroom;
  h->nv = nv;
  h->nt = nt;
  h->root_bytes = 8 + 8 * h->K;
  h->rec_bytes = bits == 0 ? h->root_bytes : ((8 + h->K * 2 * (bits / 8) + 3) / 4) * 4;
  if (bits == 1) h->root_bytes = h->rec_bytes = 8 + 4 * h->K; /* absolute halves everywhere */
  h->form_rec = h->rec_bytes;
  h->form_root = h->root_bytes;
  if (bits == 2) {
    /* Stream VByte records have variable length: 8 B of topology, an 8-byte control word
     * and 1 to 4 bytes per delta.  Treelets are formed with the largest record (16 + 8K B,
     * the header's record size) plus its 2-byte entry in the treelet's offset table, and
     * the root with its entry and the table's padding to 8 bytes (the absolute root record
     * is 8-byte aligned), so that every treelet stays within its budget whatever the deltas
     * turn out to be. */
    h->rec_bytes = 16 + 8 * h->K;
    h->form_rec = h->rec_bytes + 2;
    h->form_root = h->root_bytes + 8;
  }
  if (16 + h->form_root + m * h->form_rec > treelet_bytes) {
    or_free(h);
    return fail(OR_ERR_ARG, "treelet_bytes too small for one sibling group");
  }
  h->verts = (float *)malloc(sizeof(float) * 3 * nv);
  h->tris = (int32_t *)malloc(sizeof(int32_t) * 3 * nt);
  memcpy(h->verts, verts, sizeof(float) * 3 * nv);
  memcpy(h->tris, tris, sizeof(int32_t) * 3 * nt);
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!isfinite(h->verts[i])) {
      or_free(h);
      return fail(OR_ERR_MESH, "non-finite vertex");
    }
  h->key = (double *)malloc(sizeof(double) * 3 * nt);
  for (int64_t t = 0; t < nt; ++t) {
    double p[3][3];
    for (int c = 0; c < 3; ++c) {
      int32_t vi = h->tris[3 * t + c];
      if (vi < 0 || vi >= nv) {
        or_free(h);
        return fail(OR_ERR_MESH, "triangle index out of range");
      }
      for (int x = 0; x < 3; ++x) p[c][x] = (double)h->verts[3 * (int64_t)vi + x];
    }
    double e1[3], e2[3];
    for (int x = 0; x < 3; ++x) {
      e1[x] = p[1][x] - p[0][x];
      e2[x] = p[2][x] - p[0][x];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
    if (cx == 0.0 && cy == 0.0 && cz == 0.0) {
      or_free(h);
      return fail(OR_ERR_MESH, "degenerate (zero-area) triangle");
    }
    for (int x = 0; x < 3; ++x) h->key[3 * t + x] = (p[0][x] + p[1][x]) + p[2][x];
  }

  /* recursive build, then BFS numbering */
  tbuild b = {0};
  b.m = m;
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * nt);
  for (int64_t i = 0; i < nt; ++i) ids[i] = (int32_t)i;
  int32_t troot = build_rec(&b, h->key, ids, nt);
  free(ids);
  h->nn = b.cnt;
  int64_t nn = h->nn;
  h->parent = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->first = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->nchild = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->tri = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->depth = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * nn); /* BFS id -> temp id */
  int64_t head = 0, tail = 0;
  q[tail++] = troot;
  h->parent[0] = -1;
  h->depth[0] = 0;
  while (head < tail) {
    int64_t id = head++;
    tnode *tn = &b.n[q[id]];
    h->nchild[id] = tn->nchild;
    h->tri[id] = tn->tri;
    h->first[id] = tn->nchild ? (int32_t)tail : -1;
    for (int c = 0; c < tn->nchild; ++c) {
      h->parent[tail] = (int32_t)id;
      h->depth[tail] = h->depth[id] + 1;
      q[tail++] = tn->child[c];
    }
  }
  for (int64_t i = 0; i < b.cnt; ++i) free(b.n[i].child);
  free(b.n);
  free(q);
  h->tree_depth = 0;
  for (int64_t i = 0; i < nn; ++i)
    if (h->depth[i] > h->tree_depth) h->tree_depth = h->depth[i];
  h->leaf_order = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->leaf_tri = (int32_t *)malloc(sizeof(int32_t) * nt);
  {
    int32_t lo = 0;
    for (int64_t i = 0; i < nn; ++i) {
      h->leaf_order[i] = -1;
      if (h->nchild[i] == 0) {
        h->leaf_tri[lo] = h->tri[i];
        h->leaf_order[i] = lo++;
      }
    }
  }

  /* lattice exponent: the smallest e with |d.v| / 2^e < 2^30 for every vertex and direction */
  {
    double M = 0.0;
    for (int64_t t = 0; t < nt; ++t)
      for (int c = 0; c < 3; ++c) {
        const float *v = h->verts + 3 * (int64_t)h->tris[3 * t + c];
        for (int j = 0; j < h->K; ++j) {
          double s = OR_DIR[j][0] * (double)v[0] + OR_DIR[j][1] * (double)v[1] + OR_DIR[j][2] * (double)v[2];
          if (fabs(s) > M) M = fabs(s);
        }
      }
    if (M == 0.0) {
      or_free(h);
      return fail(OR_ERR_MESH, "mesh has no extent");
    }
    int e = ilogb(M) - 31;
    const int64_t lim = (int64_t)1 << (30 - h->headroom); /* bits kept free for refits */
    while (lattice_fits(h, e, lim)) --e;  /* walk down until it no longer fits */
    while (!lattice_fits(h, e, lim)) ++e; /* the first one that fits */
    if (e < -120 || e > 96) {
      or_free(h);
      return fail(OR_ERR_MESH, "mesh coordinates outside the supported range");
    }
    h->e = e;
  }

  compute_bounds(h);
  int K = h->K;
  if (h->bits == 1) /* half floats: every node's bounds, hence the root's, within +-65504 */
    for (int j = 0; j < 2 * K; ++j)
      if (fabs(ldexp((double)h->lat[j], h->e)) > 65504.0) {
        or_free(h);
        return fail(OR_ERR_MESH, "bounds beyond the half-precision range");
      }
  int rc = encode(h);
  if (rc) {
    or_free(h);
    return rc;
  }
  *out = h;
  return OR_OK;
}

/* Refit for deforming meshes: the same tree, treelets and lattice exponent with new
 * positions for the build's vertices.  The exact bounds are recomputed and the encoding and
 * blob redone.  Fails, leaving the handle as it was, when a new vertex is not finite, leaves
 * the lattice's range, or (half floats) puts a bound beyond +-65504. */
int or_refit(or_bvh *h, const float *verts) {
  for (int64_t i = 0; i < 3 * h->nv; ++i)
    if (!isfinite(verts[i])) return fail(OR_ERR_MESH, "non-finite vertex");
  float *old = h->verts;
  h->verts = (float *)malloc(sizeof(float) * 3 * h->nv);
  memcpy(h->verts, verts, sizeof(float) * 3 * h->nv);
  int ok = lattice_fits(h, h->e, (int64_t)1 << 30); /* a refit may use the headroom */
  if (ok && h->bits == 1)
    for (int64_t t = 0; t < h->nt && ok; ++t)
      for (int c = 0; c < 3 && ok; ++c)
        for (int j = 0; j < h->K && ok; ++j) {
          int64_t lo, hi;
          lattice_dv(h->verts + 3 * (int64_t)h->tris[3 * t + c], j, h->e, &lo, &hi);
          if (fabs(ldexp((double)lo, h->e)) > 65504.0 || fabs(ldexp((double)hi, h->e)) > 65504.0) ok = 0;
        }
  if (!ok) {
    free(h->verts);
    h->verts = old;
    return fail(OR_ERR_MESH, "refit: vertices outside the hierarchy's lattice or half range");
  }
  free(old);
  compute_bounds(h);
  /* drop the old encoding and redo it (treelets depend on the tree only) */
  free(h->tlet);
  free(h->local);
  free(h->ext);
  free(h->child_tlet);
  free(h->dec);
  free(h->delta);
  free(h->decf);
  free(h->tlet_root);
  if (h->tlet_nodes)
    for (int64_t t = 0; t < h->ntlet; ++t) free(h->tlet_nodes[t]);
  free(h->tlet_nodes);
  free(h->tlet_count);
  free(h->blob);
  h->tlet = h->local = h->child_tlet = h->tlet_root = h->tlet_count = NULL;
  h->ext = NULL;
  h->dec = NULL;
  h->delta = NULL;
  h->decf = NULL;
  h->tlet_nodes = NULL;
  h->blob = NULL;
  h->ntlet = 0;
  return encode(h);
}

/* ---- treelets and the predictor-corrector encoding ---- */
static void put32(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}
static void put16(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
}
static void put64(uint8_t *p, uint64_t v) {
  put32(p, (uint32_t)v);
  put32(p + 4, (uint32_t)(v >> 32));
}
static uint32_t f2u(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* Stream VByte (Lemire, Kurz and Rupp 2018): n unsigned 32-bit values as a 2-bit code per
 * value (its byte count minus one; value i's code in bits 2i and 2i+1 of the control bytes,
 * four codes per byte, little endian) followed by the values, little endian, each in the
 * fewest of 1 to 4 bytes.  Here the control bytes are one 8-byte word (n <= 32).  Writes
 * the control word to ctl8 and the value bytes to data; returns the number of data bytes. */
static int svb_len(uint32_t v) { return v < (1u << 8) ? 1 : v < (1u << 16) ? 2 : v < (1u << 24) ? 3 : 4; }
int or_svb_encode(const uint32_t *v, int n, uint8_t *ctl8, uint8_t *data) {
  uint64_t ctl = 0;
  int pos = 0;
  for (int i = 0; i < n; ++i) {
    const int len = svb_len(v[i]);
    ctl |= (uint64_t)(len - 1) << (2 * i);
    for (int b = 0; b < len; ++b) data[pos++] = (uint8_t)(v[i] >> (8 * b));
  }
  put64(ctl8, ctl);
  return pos;
}
/* Bytes of a Stream VByte record: topology (8), control (8), the 2K deltas, padded to 4. */
static int64_t svb_record_bytes(const or_bvh *h, int64_t x) {
  int64_t n = 16;
  for (int j = 0; j < 2 * h->K; ++j) n += svb_len(h->delta[x * h->K * 2 + j]);
  return (n + 3) / 4 * 4;
}
/* Bytes of treelet t: header, offset table (Stream VByte only), records; before padding. */
static int64_t treelet_bytes(const or_bvh *h, int64_t t) {
  if (h->bits != 2) return 16 + h->root_bytes + (int64_t)(h->tlet_count[t] - 1) * h->rec_bytes;
  int64_t sz = 16 + (2 * (int64_t)h->tlet_count[t] + 7) / 8 * 8 + h->root_bytes;
  for (int32_t l = 1; l < h->tlet_count[t]; ++l) sz += svb_record_bytes(h, h->tlet_nodes[t][l]);
  return sz;
}

/* Treelets packed bottom-up (Sec. III-B: treelets sized to the cache).  Going from the
 * deepest nodes up, each node carries the nodes of its subtree not yet cut off.  A node's
 * children stay in its treelet when the node plus everything its children carry still fits
 * one treelet (16 B header, the absolute root record, the other nodes as delta records);
 * otherwise all of its children become roots of treelets of their own.  The treelets are
 * the tree's root and every such child, numbered in node order (so siblings get consecutive
 * numbers); a treelet's nodes are listed breadth-first from its root. */
static int pack_bottom_up(or_bvh *h) {
  int64_t nn = h->nn;
  int64_t fit = (h->budget - 16 - h->form_root) / h->form_rec + 1; /* nodes per treelet */
  int64_t *carry = (int64_t *)malloc(sizeof(int64_t) * nn);
  for (int64_t x = nn - 1; x >= 0; --x) {
    int64_t sum = 1;
    for (int c = 0; c < h->nchild[x]; ++c) sum += carry[h->first[x] + c];
    if (sum <= fit) {
      carry[x] = sum;
    } else {
      carry[x] = 1;
      h->ext[x] = 1;
    }
  }
  free(carry);
  int64_t nroot = 0;
  for (int64_t x = 0; x < nn; ++x)
    if (x == 0 || h->ext[h->parent[x]]) ++nroot;
  h->ntlet = nroot;
  h->tlet_root = (int32_t *)malloc(sizeof(int32_t) * nroot);
  h->tlet_count = (int32_t *)malloc(sizeof(int32_t) * nroot);
  h->tlet_nodes = (int32_t **)malloc(sizeof(int32_t *) * nroot);
  int32_t *tlet_of = (int32_t *)malloc(sizeof(int32_t) * nn);
  int64_t t = 0;
  for (int64_t x = 0; x < nn; ++x)
    if (x == 0 || h->ext[h->parent[x]]) {
      tlet_of[x] = (int32_t)t;
      h->tlet_root[t++] = (int32_t)x;
    }
  for (int64_t x = 0; x < nn; ++x)
    if (h->ext[x]) h->child_tlet[x] = tlet_of[h->first[x]];
  free(tlet_of);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * nn);
  for (t = 0; t < nroot; ++t) {
    int64_t head = 0, tail = 0;
    queue[tail++] = h->tlet_root[t];
    while (head < tail) {
      int32_t x = queue[head++];
      if (!h->ext[x])
        for (int c = 0; c < h->nchild[x]; ++c) queue[tail++] = h->first[x] + c;
    }
    h->tlet_count[t] = (int32_t)tail;
    h->tlet_nodes[t] = (int32_t *)malloc(sizeof(int32_t) * tail);
    for (int64_t l = 0; l < tail; ++l) {
      h->tlet_nodes[t][l] = queue[l];
      h->tlet[queue[l]] = (int32_t)t;
      h->local[queue[l]] = (int32_t)l;
    }
  }
  free(queue);
  return 0;
}

static int encode(or_bvh *h) {
  int64_t nn = h->nn;
  int K = h->K;
  h->tlet = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->local = (int32_t *)malloc(sizeof(int32_t) * nn);
  h->ext = (uint8_t *)calloc(nn, 1);
  h->child_tlet = (int32_t *)malloc(sizeof(int32_t) * nn);
  for (int64_t i = 0; i < nn; ++i) h->child_tlet[i] = -1;

  if (h->packing == 1) {
    if (pack_bottom_up(h)) return 1;
  } else {
    /* Treelets (Sec. III-B): greedy BFS from each treelet root, adding whole sibling groups
     * while the treelet header, the absolute root record and the delta records fit the byte
     * budget.  A group that does not fit turns each of its nodes into the root of a new
     * treelet; new treelets are numbered in the order they are created. */
    int64_t cap = 1024;
    h->tlet_root = (int32_t *)malloc(sizeof(int32_t) * cap);
    h->tlet_root[0] = 0;
    h->ntlet = 1;
    int64_t tcap = 1024;
    h->tlet_count = (int32_t *)malloc(sizeof(int32_t) * tcap);
    h->tlet_nodes = (int32_t **)malloc(sizeof(int32_t *) * tcap);
    int32_t *bfs = (int32_t *)malloc(sizeof(int32_t) * nn);
    for (int64_t t = 0; t < h->ntlet; ++t) {
      if (t >= tcap) {
        tcap *= 2;
        h->tlet_count = (int32_t *)realloc(h->tlet_count, sizeof(int32_t) * tcap);
        h->tlet_nodes = (int32_t **)realloc(h->tlet_nodes, sizeof(int32_t *) * tcap);
      }
      int32_t r = h->tlet_root[t];
      int64_t size = 16 + h->form_root;
      int64_t cnt = 0, ncap = 64;
      int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * ncap);
      mem[cnt] = r;
      h->tlet[r] = (int32_t)t;
      h->local[r] = (int32_t)cnt++;
      int64_t bh = 0, bt = 0;
      bfs[bt++] = r;
      while (bh < bt) {
        int32_t x = bfs[bh++];
        int nc = h->nchild[x];
        if (nc == 0) continue;
        if (size + (int64_t)nc * h->form_rec <= h->budget) {
          size += (int64_t)nc * h->form_rec;
          for (int c = 0; c < nc; ++c) {
            int32_t y = h->first[x] + c;
            if (cnt == ncap) {
              ncap *= 2;
              mem = (int32_t *)realloc(mem, sizeof(int32_t) * ncap);
            }
            mem[cnt] = y;
            h->tlet[y] = (int32_t)t;
            h->local[y] = (int32_t)cnt++;
            bfs[bt++] = y;
          }
        } else {
          h->ext[x] = 1;
          h->child_tlet[x] = (int32_t)h->ntlet;
          for (int c = 0; c < nc; ++c) {
            if (h->ntlet == cap) {
              cap *= 2;
              h->tlet_root = (int32_t *)realloc(h->tlet_root, sizeof(int32_t) * cap);
            }
            h->tlet_root[h->ntlet++] = h->first[x] + c;
          }
        }
      }
      h->tlet_count[t] = (int32_t)cnt;
      h->tlet_nodes[t] = mem;
    }
    free(bfs);
  }

  int maxn = 1;
  for (int64_t t = 0; t < h->ntlet; ++t)
    if (h->tlet_count[t] > maxn) maxn = h->tlet_count[t];
  h->lbits = 1;
  while ((1 << h->lbits) < maxn) ++h->lbits;
  if (maxn > 65535) return fail(OR_ERR_ARG, "too many nodes in one treelet");
  if (h->lbits < 32 && (uint64_t)h->ntlet >= ((uint64_t)1 << (32 - h->lbits)))
    return fail(OR_ERR_ARG, "too many treelets for 32-bit node references");

  /* Predictor-corrector (abstract, Sec. III-B): a treelet root is absolute; any other node
   * is predicted by its parent's decoded interval [P_lo, P_hi] per direction.  With s the
   * smallest shift making (P_hi - P_lo) >> s fit b bits, the correctors are
   * d_lo = (C_lo - P_lo) >> s and d_hi = (P_hi - C_hi) >> s, so the decoded child
   * [P_lo + (d_lo << s), P_hi - (d_hi << s)] always contains the exact child interval. */
  h->dec = (int64_t *)malloc(sizeof(int64_t) * nn * K * 2);
  h->delta = (uint32_t *)calloc((size_t)nn * K * 2, sizeof(uint32_t));
  h->decf = (float *)malloc(sizeof(float) * nn * K * 2);
  const int64_t dmax = h->bits ? ((int64_t)1 << h->bits) - 1 : 0;
  h->max_tdepth = 0;
  for (int64_t x = 0; x < nn; ++x) {
    const int64_t *C = h->lat + x * K * 2;
    int64_t *D = h->dec + x * K * 2;
    int is_root = h->local[x] == 0;
    if (is_root || h->bits == 0 || h->bits == 1) {
      for (int j = 0; j < 2 * K; ++j) D[j] = C[j];
    } else if (h->bits == 2) {
      /* lossless: the deltas to the parent's interval, unshifted */
      const int64_t *P = h->dec + (int64_t)h->parent[x] * K * 2;
      for (int j = 0; j < K; ++j) {
        h->delta[x * K * 2 + 2 * j] = (uint32_t)(C[2 * j] - P[2 * j]);
        h->delta[x * K * 2 + 2 * j + 1] = (uint32_t)(P[2 * j + 1] - C[2 * j + 1]);
      }
      for (int j = 0; j < 2 * K; ++j) D[j] = C[j];
    } else {
      const int64_t *P = h->dec + (int64_t)h->parent[x] * K * 2;
      for (int j = 0; j < K; ++j) {
        int64_t range = P[2 * j + 1] - P[2 * j];
        int s = 0;
        while ((range >> s) > dmax) ++s;
        int64_t dlo = (C[2 * j] - P[2 * j]) >> s;
        int64_t dhi = (P[2 * j + 1] - C[2 * j + 1]) >> s;
        h->delta[x * K * 2 + 2 * j] = (uint32_t)dlo;
        h->delta[x * K * 2 + 2 * j + 1] = (uint32_t)dhi;
        D[2 * j] = P[2 * j] + (dlo << s);
        D[2 * j + 1] = P[2 * j + 1] - (dhi << s);
      }
    }
    for (int j = 0; j < K; ++j) {
      if (h->bits == 1) { /* half precision, rounded outward from the exact lattice value */
        h->decf[x * K * 2 + 2 * j] = (float)half_value(half_rd(ldexp((double)D[2 * j], h->e)));
        h->decf[x * K * 2 + 2 * j + 1] = (float)half_value(half_ru(ldexp((double)D[2 * j + 1], h->e)));
      } else {
        h->decf[x * K * 2 + 2 * j] = f32_rd(D[2 * j], h->e);
        h->decf[x * K * 2 + 2 * j + 1] = f32_ru(D[2 * j + 1], h->e);
      }
    }
  }

  /* serialise: header, treelet offsets, treelets, leaf-ordered triangles */
  int64_t off_tab = 64;
  int64_t off_t0 = (off_tab + 8 * (h->ntlet + 1) + 15) / 16 * 16;
  int64_t *toff = (int64_t *)malloc(sizeof(int64_t) * (h->ntlet + 1));
  int64_t pos = off_t0;
  for (int64_t t = 0; t < h->ntlet; ++t) {
    toff[t] = pos;
    pos += (treelet_bytes(h, t) + 15) / 16 * 16;
  }
  toff[h->ntlet] = pos;
  int64_t off_tris = pos;
  int64_t total = off_tris + 48 * h->nt;
  h->blob = (uint8_t *)calloc((size_t)total, 1);
  h->blob_bytes = total;
  uint8_t *B = h->blob;
  put32(B + 0, 0x48564243u);
  put16(B + 4, 1);
  B[6] = (uint8_t)h->k;
  B[7] = (uint8_t)K;
  B[8] = (uint8_t)h->m;
  B[9] = (uint8_t)h->bits;
  B[10] = (uint8_t)h->lbits;
  for (int64_t x = 0; x < nn; ++x) {
    int d = 0;
    for (int32_t y = (int32_t)x; h->local[y] != 0; y = h->parent[y]) ++d;
    if (d > h->max_tdepth) h->max_tdepth = d;
  }
  B[11] = (uint8_t)h->max_tdepth;
  put32(B + 12, (uint32_t)h->e);
  put32(B + 16, (uint32_t)h->nt);
  put32(B + 20, (uint32_t)nn);
  put32(B + 24, (uint32_t)h->ntlet);
  put32(B + 28, (uint32_t)h->rec_bytes);
  put32(B + 32, (uint32_t)h->root_bytes);
  put32(B + 36, (uint32_t)h->budget);
  put32(B + 40, (uint32_t)h->tree_depth);
  put32(B + 44, (uint32_t)h->packing);
  put64(B + 48, (uint64_t)off_tris);
  put64(B + 56, (uint64_t)total);
  for (int64_t t = 0; t <= h->ntlet; ++t) put64(B + off_tab + 8 * t, (uint64_t)toff[t]);
  int64_t first_node = 0;
  for (int64_t t = 0; t < h->ntlet; ++t) {
    uint8_t *T = B + toff[t];
    put32(T, (uint32_t)h->tlet_count[t]);
    put32(T + 4, (uint32_t)first_node); /* blob-order index of the treelet's root */
    first_node += h->tlet_count[t];
    /* Stream VByte: records of varying size, located by a table of 2-byte offsets (in
     * 4-byte units from the treelet's start) after the header, padded to 8 bytes */
    int64_t at = 16 + (2 * (int64_t)h->tlet_count[t] + 7) / 8 * 8;
    for (int32_t l = 0; l < h->tlet_count[t]; ++l) {
      int32_t x = h->tlet_nodes[t][l];
      uint8_t *R;
      if (h->bits == 2) {
        put16(T + 16 + 2 * l, (uint32_t)(at / 4));
        R = T + at;
        at += l == 0 ? h->root_bytes : svb_record_bytes(h, x);
      } else {
        R = T + 16 + (l == 0 ? 0 : h->root_bytes + (int64_t)(l - 1) * h->rec_bytes);
      }
      int d = 0;
      for (int32_t y = x; h->local[y] != 0; y = h->parent[y]) ++d;
      uint32_t par = l == 0 ? 0xFFFFu : (uint32_t)h->local[h->parent[x]];
      uint32_t w0 = par | ((uint32_t)h->nchild[x] << 16) | ((uint32_t)h->ext[x] << 21) | ((uint32_t)d << 24);
      uint32_t w1;
      if (h->nchild[x] == 0)
        w1 = (uint32_t)h->leaf_order[x];
      else if (h->ext[x])
        w1 = (uint32_t)h->child_tlet[x];
      else
        w1 = (uint32_t)h->local[h->first[x]];
      put32(R, w0);
      put32(R + 4, w1);
      if (h->bits == 1) {
        for (int j = 0; j < K; ++j) {
          put16(R + 8 + 4 * j, half_rd(ldexp((double)h->dec[x * K * 2 + 2 * j], h->e)));
          put16(R + 10 + 4 * j, half_ru(ldexp((double)h->dec[x * K * 2 + 2 * j + 1], h->e)));
        }
      } else if (l == 0 || h->bits == 0) {
        for (int j = 0; j < K; ++j) {
          if (h->bits == 0) {
            put32(R + 8 + 8 * j, f2u(h->decf[x * K * 2 + 2 * j]));
            put32(R + 12 + 8 * j, f2u(h->decf[x * K * 2 + 2 * j + 1]));
          } else {
            put32(R + 8 + 8 * j, (uint32_t)(int32_t)h->dec[x * K * 2 + 2 * j]);
            put32(R + 12 + 8 * j, (uint32_t)(int32_t)h->dec[x * K * 2 + 2 * j + 1]);
          }
        }
      } else if (h->bits == 2) {
        or_svb_encode(h->delta + x * K * 2, 2 * K, R + 8, R + 16);
      } else {
        for (int j = 0; j < K; ++j) {
          uint32_t dl = h->delta[x * K * 2 + 2 * j], dh = h->delta[x * K * 2 + 2 * j + 1];
          if (h->bits == 8) {
            R[8 + 2 * j] = (uint8_t)dl;
            R[9 + 2 * j] = (uint8_t)dh;
          } else {
            put16(R + 8 + 4 * j, dl);
            put16(R + 10 + 4 * j, dh);
          }
        }
      }
    }
  }
  for (int64_t i = 0; i < h->nt; ++i) {
    uint8_t *P = B + off_tris + 48 * i;
    int32_t t = h->leaf_tri[i];
    for (int c = 0; c < 3; ++c) {
      const float *v = h->verts + 3 * (int64_t)h->tris[3 * (int64_t)t + c];
      for (int x = 0; x < 3; ++x) put32(P + 16 * c + 4 * x, f2u(v[x]));
    }
    put32(P + 12, (uint32_t)t);
  }
  free(toff);
  return OR_OK;
}

void or_free(or_bvh *h) {
  if (!h) return;
  free(h->verts);
  free(h->tris);
  free(h->key);
  free(h->parent);
  free(h->first);
  free(h->nchild);
  free(h->tri);
  free(h->depth);
  free(h->leaf_order);
  free(h->leaf_tri);
  free(h->lat);
  free(h->bnd);
  free(h->tlet);
  free(h->local);
  free(h->ext);
  free(h->child_tlet);
  free(h->dec);
  free(h->delta);
  free(h->decf);
  free(h->tlet_root);
  if (h->tlet_nodes)
    for (int64_t t = 0; t < h->ntlet; ++t) free(h->tlet_nodes[t]);
  free(h->tlet_nodes);
  free(h->tlet_count);
  free(h->blob);
  free(h);
}

/* ---- accessors for tests ---- */
void or_info(const or_bvh *h, int64_t *out) {
  out[0] = h->nn;
  out[1] = h->ntlet;
  out[2] = h->e;
  out[3] = h->tree_depth;
  out[4] = h->blob_bytes;
  out[5] = h->lbits;
  out[6] = h->max_tdepth;
  out[7] = h->K;
  out[8] = h->rec_bytes;
  out[9] = h->root_bytes;
}
const uint8_t *or_blob(const or_bvh *h) { return h->blob; }
void or_tree(const or_bvh *h, int32_t *parent, int32_t *first, int32_t *nchild, int32_t *tri) {
  for (int64_t i = 0; i < h->nn; ++i) {
    parent[i] = h->parent[i];
    first[i] = h->first[i];
    nchild[i] = h->nchild[i];
    tri[i] = h->tri[i];
  }
}
void or_lattice(const or_bvh *h, int64_t *exact, int64_t *decoded, float *decf, double *bnd) {
  int64_t n = h->nn * h->K * 2;
  if (exact) memcpy(exact, h->lat, sizeof(int64_t) * n);
  if (decoded) memcpy(decoded, h->dec, sizeof(int64_t) * n);
  if (decf) memcpy(decf, h->decf, sizeof(float) * n);
  if (bnd) memcpy(bnd, h->bnd, sizeof(double) * n);
}
void or_placement(const or_bvh *h, int32_t *tlet, int32_t *local, uint8_t *ext, uint32_t *delta) {
  for (int64_t i = 0; i < h->nn; ++i) {
    tlet[i] = h->tlet[i];
    local[i] = h->local[i];
    ext[i] = h->ext[i];
  }
  if (delta) memcpy(delta, h->delta, sizeof(uint32_t) * h->nn * h->K * 2);
}

/* ------------------------------------------------------------------ independent decoder */
static uint32_t get32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint32_t get16(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint64_t get64(const uint8_t *p) { return (uint64_t)get32(p) | ((uint64_t)get32(p + 4) << 32); }

/* Decode every node of a blob, in blob order (treelet by treelet, local index order).
 * lat: n x K x 2 decoded lattice (not written for quant_bits = 0 or 1); f: n x K x 2 FP32
 * bounds; meta: n x 4 (w0, w1, treelet, local).  Returns the node count, or < 0. */
int64_t or_decode_blob(const uint8_t *blob, int64_t bytes, int32_t *lat, float *f, uint32_t *meta) {
  if (bytes < 64 || get32(blob) != 0x48564243u) return fail(OR_ERR_ARG, "not a blob");
  int K = blob[7], bits = blob[9];
  int e = (int32_t)get32(blob + 12);
  int64_t ntlet = get32(blob + 24);
  int rec = (int)get32(blob + 28), rootb = (int)get32(blob + 32);
  int64_t n = 0;
  int64_t *P = (int64_t *)malloc(sizeof(int64_t) * 2 * K * 65536);
  for (int64_t t = 0; t < ntlet; ++t) {
    int64_t off = (int64_t)get64(blob + 64 + 8 * t);
    const uint8_t *T = blob + off;
    int32_t cnt = (int32_t)get32(T);
    if ((int64_t)get32(T + 4) != n) {
      free(P);
      return fail(OR_ERR_ARG, "treelet header: wrong first-node index");
    }
    for (int32_t l = 0; l < cnt; ++l, ++n) {
      const uint8_t *R = bits == 2 ? T + 4 * (int64_t)get16(T + 16 + 2 * l)
                                   : T + 16 + (l == 0 ? 0 : rootb + (int64_t)(l - 1) * rec);
      /* Stream VByte record: the 2K deltas from the control word's 2-bit length codes */
      uint32_t sv[26];
      if (bits == 2 && l > 0) {
        const uint64_t ctl = get64(R + 8);
        const uint8_t *q = R + 16;
        for (int i = 0; i < 2 * K; ++i) {
          const int len = (int)((ctl >> (2 * i)) & 3u) + 1;
          sv[i] = 0;
          for (int b = 0; b < len; ++b) sv[i] |= (uint32_t)q[b] << (8 * b);
          q += len;
        }
      }
      uint32_t w0 = get32(R), w1 = get32(R + 4);
      int64_t *D = P + (int64_t)l * 2 * K;
      for (int j = 0; j < K; ++j) {
        if (bits == 1) {
          if (f) {
            f[n * K * 2 + 2 * j] = (float)half_value(get16(R + 8 + 4 * j));
            f[n * K * 2 + 2 * j + 1] = (float)half_value(get16(R + 10 + 4 * j));
          }
          continue;
        }
        if (bits == 0) {
          float lo, hi;
          uint32_t a = get32(R + 8 + 8 * j), b = get32(R + 12 + 8 * j);
          memcpy(&lo, &a, 4);
          memcpy(&hi, &b, 4);
          if (f) {
            f[n * K * 2 + 2 * j] = lo;
            f[n * K * 2 + 2 * j + 1] = hi;
          }
          continue;
        }
        if (l == 0) {
          D[2 * j] = (int32_t)get32(R + 8 + 8 * j);
          D[2 * j + 1] = (int32_t)get32(R + 12 + 8 * j);
        } else if (bits == 2) {
          const int64_t *Q = P + (int64_t)(w0 & 0xFFFFu) * 2 * K;
          D[2 * j] = Q[2 * j] + (int64_t)sv[2 * j];
          D[2 * j + 1] = Q[2 * j + 1] - (int64_t)sv[2 * j + 1];
        } else {
          const int64_t *Q = P + (int64_t)(w0 & 0xFFFFu) * 2 * K;
          int64_t lo = Q[2 * j], hi = Q[2 * j + 1];
          int64_t range = hi - lo;
          int s = 0;
          while ((range >> s) > ((1 << bits) - 1)) ++s;
          uint32_t dl = bits == 8 ? R[8 + 2 * j] : get16(R + 8 + 4 * j);
          uint32_t dh = bits == 8 ? R[9 + 2 * j] : get16(R + 10 + 4 * j);
          D[2 * j] = lo + ((int64_t)dl << s);
          D[2 * j + 1] = hi - ((int64_t)dh << s);
        }
        if (lat) {
          lat[n * K * 2 + 2 * j] = (int32_t)D[2 * j];
          lat[n * K * 2 + 2 * j + 1] = (int32_t)D[2 * j + 1];
        }
        if (f) {
          f[n * K * 2 + 2 * j] = f32_rd(D[2 * j], e);
          f[n * K * 2 + 2 * j + 1] = f32_ru(D[2 * j + 1], e);
        }
      }
      if (meta) {
        meta[4 * n] = w0;
        meta[4 * n + 1] = w1;
        meta[4 * n + 2] = (uint32_t)t;
        meta[4 * n + 3] = (uint32_t)l;
      }
    }
  }
  free(P);
  return n;
}

/* ------------------------------------------------------------------ geometry (FP64) */
static void sub3(const double *a, const double *b, double *o) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* 2-D helpers for the coplanar case */
static double orient2(const double *a, const double *b, const double *c) {
  return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
}
static int sgn(double x) { return (x > 0) - (x < 0); }
static int seg2_hit(const double *p1, const double *p2, const double *q1, const double *q2) {
  double o1 = orient2(p1, p2, q1), o2 = orient2(p1, p2, q2);
  double o3 = orient2(q1, q2, p1), o4 = orient2(q1, q2, p2);
  if (o1 == 0 && o2 == 0 && o3 == 0 && o4 == 0) {
    for (int c = 0; c < 2; ++c) {
      double a0 = fmin(p1[c], p2[c]), a1 = fmax(p1[c], p2[c]);
      double b0 = fmin(q1[c], q2[c]), b1 = fmax(q1[c], q2[c]);
      if (a1 < b0 || b1 < a0) return 0;
    }
    return 1;
  }
  return sgn(o1) * sgn(o2) <= 0 && sgn(o3) * sgn(o4) <= 0;
}
static int pt2_in_tri(const double *p, const double *a, const double *b, const double *c) {
  double d1 = orient2(a, b, p), d2 = orient2(b, c, p), d3 = orient2(c, a, p);
  int neg = d1 < 0 || d2 < 0 || d3 < 0, pos = d1 > 0 || d2 > 0 || d3 > 0;
  return !(neg && pos);
}
static int coplanar_hit(const double V[3][3], const double U[3][3], const double *N) {
  int drop = 0;
  if (fabs(N[1]) > fabs(N[drop])) drop = 1;
  if (fabs(N[2]) > fabs(N[drop])) drop = 2;
  int a = drop == 0 ? 1 : 0, b = drop == 2 ? 1 : 2;
  double v[3][2], u[3][2];
  for (int i = 0; i < 3; ++i) {
    v[i][0] = V[i][a];
    v[i][1] = V[i][b];
    u[i][0] = U[i][a];
    u[i][1] = U[i][b];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (seg2_hit(v[i], v[(i + 1) % 3], u[j], u[(j + 1) % 3])) return 1;
  return pt2_in_tri(v[0], u[0], u[1], u[2]) || pt2_in_tri(u[0], v[0], v[1], v[2]);
}

/* Interval of triangle X on the line L = plane(other) ∩ plane(X), as projections onto D:
 * the convex hull of X's vertices lying on the other plane and of its edge crossings. */
static void line_interval(const double X[3][3], const double *s, const double *D, double *lo, double *hi) {
  *lo = INFINITY;
  *hi = -INFINITY;
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3;
    if (s[i] == 0.0) {
      double p = dot3(D, X[i]);
      if (p < *lo) *lo = p;
      if (p > *hi) *hi = p;
    }
    if ((s[i] > 0 && s[j] < 0) || (s[i] < 0 && s[j] > 0)) {
      double t = s[i] / (s[i] - s[j]);
      double P[3];
      for (int c = 0; c < 3; ++c) P[c] = X[i][c] + (X[j][c] - X[i][c]) * t;
      double p = dot3(D, P);
      if (p < *lo) *lo = p;
      if (p > *hi) *hi = p;
    }
  }
}

/* Closed triangle-triangle intersection by Moller's interval-overlap method (1997): reject
 * when one triangle lies strictly on one side of the other's plane; otherwise both
 * triangles cut the common line L in an interval and they intersect iff the two closed
 * intervals overlap (coplanar triangles: a 2-D edge and containment test).  If margin is
 * given it receives the smallest decision margin, in length units: the unit-normal plane
 * distances of the six vertices and the separations along L of the four interval ends
 * (0 for coplanar or touching configurations); it is only meaningful when the result is 1. */
int or_tri_intersect(const double V[3][3], const double U[3][3], double *margin) {
  double e1[3], e2[3], N1[3], N2[3], du[3], dv[3], w[3];
  sub3(V[1], V[0], e1);
  sub3(V[2], V[0], e2);
  cross3(e1, e2, N1);
  for (int i = 0; i < 3; ++i) {
    sub3(U[i], V[0], w);
    du[i] = dot3(N1, w);
  }
  if ((du[0] > 0 && du[1] > 0 && du[2] > 0) || (du[0] < 0 && du[1] < 0 && du[2] < 0)) return 0;
  sub3(U[1], U[0], e1);
  sub3(U[2], U[0], e2);
  cross3(e1, e2, N2);
  for (int i = 0; i < 3; ++i) {
    sub3(V[i], U[0], w);
    dv[i] = dot3(N2, w);
  }
  if ((dv[0] > 0 && dv[1] > 0 && dv[2] > 0) || (dv[0] < 0 && dv[1] < 0 && dv[2] < 0)) return 0;
  if (du[0] == 0 && du[1] == 0 && du[2] == 0) {
    if (margin) *margin = 0.0;
    return coplanar_hit(V, U, N1);
  }
  double D[3];
  cross3(N1, N2, D);
  double a0, a1, b0, b1;
  line_interval(V, dv, D, &a0, &a1);
  line_interval(U, du, D, &b0, &b1);
  int hit = a0 <= b1 && b0 <= a1;
  if (margin) {
    double m = INFINITY, n1 = norm3(N1), n2 = norm3(N2), nd = norm3(D);
    for (int i = 0; i < 3; ++i) {
      m = fmin(m, fabs(du[i]) / n1);
      m = fmin(m, fabs(dv[i]) / n2);
    }
    if (nd > 0) {
      m = fmin(m, fabs(a0 - b0) / nd);
      m = fmin(m, fabs(a0 - b1) / nd);
      m = fmin(m, fabs(a1 - b0) / nd);
      m = fmin(m, fabs(a1 - b1) / nd);
    } else {
      m = 0.0;
    }
    *margin = m;
  }
  return hit;
}

static double pt_seg(const double *p, const double *a, const double *b) {
  double ab[3], ap[3];
  sub3(b, a, ab);
  sub3(p, a, ap);
  double l2 = dot3(ab, ab);
  double t = l2 > 0 ? dot3(ap, ab) / l2 : 0.0;
  if (t < 0) t = 0;
  if (t > 1) t = 1;
  double q[3] = {a[0] + t * ab[0] - p[0], a[1] + t * ab[1] - p[1], a[2] + t * ab[2] - p[2]};
  return norm3(q);
}

/* Distance from point p to the closed triangle T: the plane distance when p projects
 * inside T, otherwise the nearest of the three edges. */
double or_pt_tri(const double *p, const double T[3][3]) {
  double e1[3], e2[3], N[3], w[3];
  sub3(T[1], T[0], e1);
  sub3(T[2], T[0], e2);
  cross3(e1, e2, N);
  int inside = 1;
  for (int i = 0; i < 3; ++i) {
    double e[3], c[3];
    sub3(T[(i + 1) % 3], T[i], e);
    sub3(p, T[i], w);
    cross3(e, w, c);
    if (dot3(N, c) < 0) inside = 0;
  }
  if (inside) {
    sub3(p, T[0], w);
    return fabs(dot3(N, w)) / norm3(N);
  }
  double d = pt_seg(p, T[0], T[1]);
  d = fmin(d, pt_seg(p, T[1], T[2]));
  return fmin(d, pt_seg(p, T[2], T[0]));
}

/* Distance between closed segments [a, b] and [c, d]: the minimum of a convex quadratic
 * over the unit square is the unconstrained minimum when that lies inside, otherwise it is
 * on the square's boundary, i.e. one of the four endpoint-to-segment distances. */
double or_seg_seg(const double *a, const double *b, const double *c, const double *d) {
  double u[3], v[3], w[3];
  sub3(b, a, u);
  sub3(d, c, v);
  sub3(a, c, w);
  double A = dot3(u, u), B = dot3(u, v), C = dot3(v, v), Dd = dot3(u, w), E = dot3(v, w);
  double den = A * C - B * B;
  if (den > 1e-300 * (A * C + 1e-300)) {
    double s = (B * E - C * Dd) / den, t = (A * E - B * Dd) / den;
    if (s >= 0 && s <= 1 && t >= 0 && t <= 1) {
      double q[3] = {w[0] + s * u[0] - t * v[0], w[1] + s * u[1] - t * v[1], w[2] + s * u[2] - t * v[2]};
      return norm3(q);
    }
  }
  double r = pt_seg(a, c, d);
  r = fmin(r, pt_seg(b, c, d));
  r = fmin(r, pt_seg(c, a, b));
  return fmin(r, pt_seg(d, a, b));
}

/* Triangle-triangle distance: 0 when they intersect, else the minimum over the six
 * vertex-triangle and nine edge-edge distances (closest points of disjoint triangles lie on
 * such a feature pair). */
double or_tri_dist(const double V[3][3], const double U[3][3]) {
  if (or_tri_intersect(V, U, NULL)) return 0.0;
  double d = INFINITY;
  for (int i = 0; i < 3; ++i) {
    d = fmin(d, or_pt_tri(V[i], U));
    d = fmin(d, or_pt_tri(U[i], V));
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) d = fmin(d, or_seg_seg(V[i], V[(i + 1) % 3], U[j], U[(j + 1) % 3]));
  return d;
}

/* ------------------------------------------------------------------ traversal */
typedef struct {
  int32_t *ij;
  int64_t n, cap;
} pvec;
static void pv_push(pvec *v, int32_t i, int32_t j) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 16;
    v->ij = (int32_t *)realloc(v->ij, sizeof(int32_t) * 2 * v->cap);
  }
  v->ij[2 * v->n] = i;
  v->ij[2 * v->n + 1] = j;
  v->n++;
}

typedef struct {
  const or_bvh *A, *B;
  double R[9], t[3];
  double u[13][3], s[13]; /* u_j = R^T d_j, s_j = d_j . t */
  int use_decoded;        /* 0: own FP64 bounds, 1: decoded FP32 bounds of the blob */
  double eps;             /* extra inflation, length units */
  pvec *pairs;
  int hit;
  double best;
  /* near-contact */
  double min_margin;
  int near;
  int64_t bv_tests, leaf_tests;
} tctx;

static void ctx_init(tctx *c, const or_bvh *A, const or_bvh *B, const float *pose, int use_decoded, double eps) {
  memset(c, 0, sizeof *c);
  c->A = A;
  c->B = B;
  for (int i = 0; i < 9; ++i) c->R[i] = pose[i];
  for (int i = 0; i < 3; ++i) c->t[i] = pose[9 + i];
  for (int j = 0; j < A->K; ++j) {
    for (int col = 0; col < 3; ++col)
      c->u[j][col] = OR_DIR[j][0] * c->R[0 + col] + OR_DIR[j][1] * c->R[3 + col] + OR_DIR[j][2] * c->R[6 + col];
    c->s[j] = OR_DIR[j][0] * c->t[0] + OR_DIR[j][1] * c->t[1] + OR_DIR[j][2] * c->t[2];
  }
  c->use_decoded = use_decoded;
  c->eps = eps;
  c->best = INFINITY;
  c->min_margin = INFINITY;
}

static void bounds_of(const tctx *c, const or_bvh *h, int32_t x, int j, double *lo, double *hi) {
  if (c->use_decoded) {
    *lo = h->decf[(int64_t)x * h->K * 2 + 2 * j];
    *hi = h->decf[(int64_t)x * h->K * 2 + 2 * j + 1];
  } else {
    *lo = h->bnd[(int64_t)x * h->K * 2 + 2 * j];
    *hi = h->bnd[(int64_t)x * h->K * 2 + 2 * j + 1];
  }
}

/* Slab separation of A-node a and B-node b along A's direction j: the axis box of b (its
 * first three slabs), moved by the pose, is projected onto d_j as u_j.c + s_j -/+ |u_j|.h.
 * Returns the gap (<= 0 when the slabs overlap) after a relative 1e-12 slack. */
static double slab_gap(const tctx *c, int32_t a, int32_t b, int j) {
  double alo, ahi, bc[3], bh[3];
  bounds_of(c, c->A, a, j, &alo, &ahi);
  for (int i = 0; i < 3; ++i) {
    double lo, hi;
    bounds_of(c, c->B, b, i, &lo, &hi);
    bc[i] = 0.5 * (lo + hi);
    bh[i] = 0.5 * (hi - lo);
  }
  double mid = c->u[j][0] * bc[0] + c->u[j][1] * bc[1] + c->u[j][2] * bc[2] + c->s[j];
  double rad = fabs(c->u[j][0]) * bh[0] + fabs(c->u[j][1]) * bh[1] + fabs(c->u[j][2]) * bh[2];
  double blo = mid - rad, bhi = mid + rad;
  double tol = 1e-12 * (fabs(alo) + fabs(ahi) + fabs(mid) + rad) + c->eps * norm3((const double[3]){OR_DIR[j][0], OR_DIR[j][1], OR_DIR[j][2]});
  double g = fmax(alo - bhi, blo - ahi);
  return g - tol;
}

/* "a and b intersect" of Algorithm 1: every slab of A's k-DOP overlaps the projected box. */
static int bv_overlap(tctx *c, int32_t a, int32_t b) {
  c->bv_tests++;
  for (int j = 0; j < c->A->K; ++j)
    if (slab_gap(c, a, b, j) > 0) return 0;
  return 1;
}
/* Lower bound on the distance between the contents of a and b, the larger of two valid
 * bounds: max_j gap_j / |d_j| (the two contents lie in slabs gap_j / |d_j| apart), and
 * sqrt(gap_x^2 + gap_y^2 + gap_z^2) over the three axis directions, the distance between
 * A's axis box and the axis-aligned box around b's moved box, which contain the contents. */
static double bv_lower(tctx *c, int32_t a, int32_t b) {
  c->bv_tests++;
  double lb = 0.0, box2 = 0.0;
  for (int j = 0; j < c->A->K; ++j) {
    double g = slab_gap(c, a, b, j);
    double n = norm3((const double[3]){OR_DIR[j][0], OR_DIR[j][1], OR_DIR[j][2]});
    if (g / n > lb) lb = g / n;
    if (j < 3 && g > 0) box2 += g * g;
  }
  return fmax(lb, sqrt(box2));
}

static void tri_A(const or_bvh *A, int32_t t, double T[3][3]) {
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) T[c][x] = A->verts[3 * (int64_t)A->tris[3 * (int64_t)t + c] + x];
}
static void tri_B(const tctx *ctx, int32_t t, double T[3][3]) {
  const or_bvh *B = ctx->B;
  for (int c = 0; c < 3; ++c) {
    const float *v = B->verts + 3 * (int64_t)B->tris[3 * (int64_t)t + c];
    for (int r = 0; r < 3; ++r)
      T[c][r] = ctx->R[3 * r] * v[0] + ctx->R[3 * r + 1] * v[1] + ctx->R[3 * r + 2] * v[2] + ctx->t[r];
  }
}

enum { MODE_CD = 0, MODE_PQ = 1, MODE_NEAR = 2 };

static void check_primitives(tctx *c, int mode, int32_t a, int32_t b) {
  double T1[3][3], T2[3][3];
  int32_t ta = c->A->tri[a], tb = c->B->tri[b];
  tri_A(c->A, ta, T1);
  tri_B(c, tb, T2);
  c->leaf_tests++;
  if (mode == MODE_CD) {
    if (or_tri_intersect(T1, T2, NULL)) {
      c->hit = 1;
      if (c->pairs) pv_push(c->pairs, ta, tb);
    }
  } else if (mode == MODE_PQ) {
    double d = or_tri_dist(T1, T2);
    if (d < c->best) c->best = d;
  } else {
    double m;
    int amb = 0;
    if (or_tri_intersect(T1, T2, &m)) {
      if (m < c->min_margin) c->min_margin = m;
      amb = m < c->eps;
    } else {
      double d = or_tri_dist(T1, T2);
      if (d < c->min_margin) c->min_margin = d;
      amb = d <= c->eps;
    }
    if (amb) {
      c->near = 1;
      if (c->pairs) pv_push(c->pairs, ta, tb);
    }
  }
}

/* Algorithm 1, BVHtraversal(a, b), recursive as printed.  In PQ mode the test "a and b
 * intersect" is replaced by "the lower bound of (a, b) is below the best distance so far"
 * (branch and bound); the control flow is the same. */
static int pair_ok(tctx *c, int mode, int32_t a, int32_t b) {
  if (mode == MODE_PQ) return c->best > 0 && bv_lower(c, a, b) < c->best;
  return bv_overlap(c, a, b);
}
static void bvh_traversal(tctx *c, int mode, int32_t a, int32_t b) {
  const or_bvh *A = c->A, *B = c->B;
  int la = A->nchild[a] == 0, lb = B->nchild[b] == 0;
  if (la && lb) {
    check_primitives(c, mode, a, b);
  } else if (la) {
    for (int i = 0; i < B->nchild[b]; ++i) {
      int32_t bi = B->first[b] + i;
      if (pair_ok(c, mode, a, bi)) bvh_traversal(c, mode, a, bi);
    }
  } else if (lb) {
    for (int i = 0; i < A->nchild[a]; ++i) {
      int32_t ai = A->first[a] + i;
      if (pair_ok(c, mode, ai, b)) bvh_traversal(c, mode, ai, b);
    }
  } else {
    for (int i = 0; i < A->nchild[a]; ++i)
      for (int j = 0; j < B->nchild[b]; ++j) {
        int32_t ai = A->first[a] + i, bj = B->first[b] + j;
        if (pair_ok(c, mode, ai, bj)) bvh_traversal(c, mode, ai, bj);
      }
  }
}

/* Branch and bound for PQ: Algorithm 1's recursion with the overlap test replaced by
 * "lower bound below the best distance so far"; the candidate pairs of one expansion are
 * visited in increasing lower-bound order and re-checked before each descent, which changes
 * how much is visited but not the minimum found. */
typedef struct {
  double lb;
  int32_t a, b;
} cand;
static int cmp_cand(const void *x, const void *y) {
  double p = ((const cand *)x)->lb, q = ((const cand *)y)->lb;
  return (p > q) - (p < q);
}
static void bvh_pq(tctx *c, int32_t a, int32_t b) {
  const or_bvh *A = c->A, *B = c->B;
  int la = A->nchild[a] == 0, lb_ = B->nchild[b] == 0;
  if (la && lb_) {
    check_primitives(c, MODE_PQ, a, b);
    return;
  }
  int na = la ? 1 : A->nchild[a], nb = lb_ ? 1 : B->nchild[b];
  cand cs[256];
  int n = 0;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      int32_t ai = la ? a : A->first[a] + i, bj = lb_ ? b : B->first[b] + j;
      double l = bv_lower(c, ai, bj);
      if (l < c->best) cs[n++] = (cand){l, ai, bj};
    }
  qsort(cs, (size_t)n, sizeof(cand), cmp_cand);
  for (int q = 0; q < n && c->best > 0; ++q)
    if (cs[q].lb < c->best) bvh_pq(c, cs[q].a, cs[q].b);
}

typedef struct {
  int64_t n;
  pvec *v;
} or_pairs;

static int cmp_pair(const void *pa, const void *pb) {
  const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
  if (a[0] != b[0]) return (a[0] > b[0]) - (a[0] < b[0]);
  return (a[1] > b[1]) - (a[1] < b[1]);
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* CD over n poses through Algorithm 1 (the root pair is tested first).  hit: n bytes;
 * counts: n pair counts; pairs (optional): a handle with every pose's sorted (i, j) list,
 * i and j original triangle indices of A and B.  stats (optional): BV tests, leaf tests. */
or_pairs *or_collide(const or_bvh *A, const or_bvh *B, const float *poses, int64_t n, int use_decoded,
                     uint8_t *hit, int64_t *counts, int want_pairs, int64_t *stats) {
  or_pairs *P = (or_pairs *)calloc(1, sizeof(or_pairs));
  P->n = n;
  P->v = (pvec *)calloc((size_t)n, sizeof(pvec));
  int64_t bv = 0, lf = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bv, lf)
  for (int64_t p = 0; p < n; ++p) {
    tctx c;
    ctx_init(&c, A, B, poses + 12 * p, use_decoded, 0.0);
    c.pairs = want_pairs ? &P->v[p] : NULL;
    pvec tmp = {0};
    if (!want_pairs) c.pairs = &tmp;
    if (bv_overlap(&c, 0, 0)) bvh_traversal(&c, MODE_CD, 0, 0);
    hit[p] = (uint8_t)c.hit;
    counts[p] = c.pairs->n;
    if (c.pairs->n > 1) qsort(c.pairs->ij, (size_t)c.pairs->n, 2 * sizeof(int32_t), cmp_pair);
    free(tmp.ij);
    bv += c.bv_tests;
    lf += c.leaf_tests;
  }
  if (stats) {
    stats[0] = bv;
    stats[1] = lf;
  }
  return P;
}

/* PQ over n poses: branch-and-bound Algorithm 1; dist[p] = min triangle-pair distance. */
void or_distance(const or_bvh *A, const or_bvh *B, const float *poses, int64_t n, int use_decoded, double *dist,
                 int64_t *stats) {
  int64_t bv = 0, lf = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bv, lf)
  for (int64_t p = 0; p < n; ++p) {
    tctx c;
    ctx_init(&c, A, B, poses + 12 * p, use_decoded, 0.0);
    if (bv_lower(&c, 0, 0) < c.best) bvh_pq(&c, 0, 0);
    dist[p] = c.best;
    bv += c.bv_tests;
    lf += c.leaf_tests;
  }
  if (stats) {
    stats[0] = bv;
    stats[1] = lf;
  }
}

/* Near-contact filter: for each pose, every triangle pair whose bounding volumes come
 * within eps is examined; the pose is near contact when some pair is separated by at most
 * eps, or intersects with a decision margin below eps.  margin[p] = the smallest such
 * quantity seen (inf when no pair comes within eps). */
void or_near_contact(const or_bvh *A, const or_bvh *B, const float *poses, int64_t n, double eps, uint8_t *near,
                     double *margin) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n; ++p) {
    tctx c;
    ctx_init(&c, A, B, poses + 12 * p, 0, eps);
    if (bv_overlap(&c, 0, 0)) bvh_traversal(&c, MODE_NEAR, 0, 0);
    near[p] = (uint8_t)c.near;
    if (margin) margin[p] = c.min_margin;
  }
}

/* The near-contact pairs themselves: per pose, the sorted (i, j) pairs that are separated
 * by at most eps or intersect with a decision margin below eps -- the pairs for which an
 * FP32 test may legitimately decide either way. */
or_pairs *or_near_pairs(const or_bvh *A, const or_bvh *B, const float *poses, int64_t n, double eps, int64_t *counts) {
  or_pairs *P = (or_pairs *)calloc(1, sizeof(or_pairs));
  P->n = n;
  P->v = (pvec *)calloc((size_t)n, sizeof(pvec));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n; ++p) {
    tctx c;
    ctx_init(&c, A, B, poses + 12 * p, 0, eps);
    c.pairs = &P->v[p];
    if (bv_overlap(&c, 0, 0)) bvh_traversal(&c, MODE_NEAR, 0, 0);
    counts[p] = c.pairs->n;
    if (c.pairs->n > 1) qsort(c.pairs->ij, (size_t)c.pairs->n, 2 * sizeof(int32_t), cmp_pair);
  }
  return P;
}

/* Brute force over all triangle pairs (the plain definitions of CD and PQ).  A pair whose
 * triangle bounding boxes are strictly apart along some axis cannot intersect, and its box
 * gap bounds its distance from below; both shortcuts are exact. */
or_pairs *or_brute_collide(const or_bvh *A, const or_bvh *B, const float *poses, int64_t n, uint8_t *hit,
                           int64_t *counts) {
  or_pairs *P = (or_pairs *)calloc(1, sizeof(or_pairs));
  P->n = n;
  P->v = (pvec *)calloc((size_t)n, sizeof(pvec));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n; ++p) {
    tctx c;
    ctx_init(&c, A, B, poses + 12 * p, 0, 0.0);
    double (*TB)[3][3] = (double (*)[3][3])malloc(sizeof(double) * 9 * B->nt);
    double (*bb)[6] = (double (*)[6])malloc(sizeof(double) * 6 * B->nt);
    for (int64_t j = 0; j < B->nt; ++j) {
      tri_B(&c, (int32_t)j, TB[j]);
      for (int x = 0; x < 3; ++x) {
        bb[j][x] = fmin(TB[j][0][x], fmin(TB[j][1][x], TB[j][2][x]));
        bb[j][3 + x] = fmax(TB[j][0][x], fmax(TB[j][1][x], TB[j][2][x]));
      }
    }
    int h = 0;
    for (int64_t i = 0; i < A->nt; ++i) {
      double TA[3][3], lo[3], hi[3];
      tri_A(A, (int32_t)i, TA);
      for (int x = 0; x < 3; ++x) {
        lo[x] = fmin(TA[0][x], fmin(TA[1][x], TA[2][x]));
        hi[x] = fmax(TA[0][x], fmax(TA[1][x], TA[2][x]));
      }
      for (int64_t j = 0; j < B->nt; ++j) {
        if (hi[0] < bb[j][0] || bb[j][3] < lo[0] || hi[1] < bb[j][1] || bb[j][4] < lo[1] || hi[2] < bb[j][2] ||
            bb[j][5] < lo[2])
          continue;
        if (or_tri_intersect(TA, TB[j], NULL)) {
          h = 1;
          pv_push(&P->v[p], (int32_t)i, (int32_t)j);
        }
      }
    }
    hit[p] = (uint8_t)h;
    counts[p] = P->v[p].n;
    free(TB);
    free(bb);
  }
  return P;
}

void or_brute_distance(const or_bvh *A, const or_bvh *B, const float *poses, int64_t n, double *dist) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n; ++p) {
    tctx c;
    ctx_init(&c, A, B, poses + 12 * p, 0, 0.0);
    double best = INFINITY;
    for (int64_t j = 0; j < B->nt && best > 0; ++j) {
      double TB[3][3], blo[3], bhi[3];
      tri_B(&c, (int32_t)j, TB);
      for (int x = 0; x < 3; ++x) {
        blo[x] = fmin(TB[0][x], fmin(TB[1][x], TB[2][x]));
        bhi[x] = fmax(TB[0][x], fmax(TB[1][x], TB[2][x]));
      }
      for (int64_t i = 0; i < A->nt && best > 0; ++i) {
        double TA[3][3], g2 = 0.0;
        tri_A(A, (int32_t)i, TA);
        for (int x = 0; x < 3; ++x) {
          double lo = fmin(TA[0][x], fmin(TA[1][x], TA[2][x])), hi = fmax(TA[0][x], fmax(TA[1][x], TA[2][x]));
          double g = fmax(lo - bhi[x], blo[x] - hi);
          if (g > 0) g2 += g * g;
        }
        if (sqrt(g2) >= best) continue;
        double d = or_tri_dist(TA, TB);
        if (d < best) best = d;
      }
    }
    dist[p] = best;
  }
}

int64_t or_pairs_total(const or_pairs *P) {
  int64_t s = 0;
  for (int64_t p = 0; p < P->n; ++p) s += P->v[p].n;
  return s;
}
/* Copy all pose lists into offsets[n+1] / ij[2 * total]. */
void or_pairs_copy(const or_pairs *P, int64_t *offsets, int32_t *ij) {
  int64_t o = 0;
  for (int64_t p = 0; p < P->n; ++p) {
    offsets[p] = o;
    if (P->v[p].n) memcpy(ij + 2 * o, P->v[p].ij, sizeof(int32_t) * 2 * P->v[p].n);
    o += P->v[p].n;
  }
  offsets[P->n] = o;
}
void or_pairs_free(or_pairs *P) {
  if (!P) return;
  for (int64_t p = 0; p < P->n; ++p) free(P->v[p].ij);
  free(P->v);
  free(P);
}
