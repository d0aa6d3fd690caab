/*
 * cbvh.h -- C ABI of the GB300 engine for simultaneous traversal of two compressed k-DOP
 * bounding volume hierarchies: collision detection (CD) and proximity query (PQ) over many
 * rigid poses.  Method: Tan, Weller & Zachmann, "Compressed Bounding Volume Hierarchies for
 * Collision Detection & Proximity Query" (arXiv 2012.05348), Algorithm 1 and Sec. III.
 *
 * Conventions
 *   - Every call returns 0 (CBVH_OK) or a negative CBVH_ERR_* code and never throws.
 *     cbvh_last_error() returns a thread-local message for the last failing call.
 *   - Pointers are DEVICE pointers unless the parameter name ends in _host.
 *   - The library never allocates device memory.  The caller owns every device buffer:
 *     the BVH blob (cbvh_attach), outputs and a workspace sized by cbvh_workspace_bytes.
 *     A cbvh_bvh handle owns only host memory.
 *   - Query calls are asynchronous on the given cudaStream_t (a CUstream / cudaStream_t
 *     passed as void*; NULL = the legacy default stream).  Host-side argument errors are
 *     returned at once.  Errors only known on the device (capacity, stack, timeout) are
 *     written to the int32 device word `status` (0 = OK) that every query takes; read it
 *     after synchronising the stream.
 *   - Poses are n x 12 FP32, row-major: the rotation R (9 values) then the translation t
 *     (3 values).  A pose maps a point of B into A's frame: x_A = R x_B + t.  R must be a
 *     rotation (orthonormal up to FP32 rounding).
 *   - Triangle indices in outputs are the caller's original triangle indices.
 */
#ifndef CBVH_H
#define CBVH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CBVH_OK 0
#define CBVH_ERR_ARG (-1)       /* invalid argument (k, branching, bits, treelet size, sizes, pointers) */
#define CBVH_ERR_MESH (-2)      /* out-of-range index, degenerate triangle, non-finite or out-of-range coordinates */
#define CBVH_ERR_CUDA (-3)      /* a CUDA runtime call failed; see cbvh_last_error() */
#define CBVH_ERR_CAPACITY (-4)  /* device: more intersecting pairs than pair_capacity */
#define CBVH_ERR_STACK (-5)     /* device: traversal stack bound exceeded (never by construction) */
#define CBVH_ERR_TIMEOUT (-6)   /* device: a bounded wait ran out (CBVH_OPT_WAIT_CAP); results are incomplete */
#define CBVH_ERR_WORKSPACE (-7) /* workspace smaller than cbvh_workspace_bytes() */
#define CBVH_ERR_CHECK (-8)     /* device, checked build (libcbvh_checked.so) only: an index read from a blob or
                                   computed by the traversal failed its bounds check; the access was skipped and
                                   the results are not valid */
#define CBVH_ERR_STATE (-9)     /* handle has no device blob attached */
#define CBVH_ERR_IO (-10)       /* a file could not be read or written, or is not a valid hierarchy */

/* collide flags */
#define CBVH_QUANT_FP16 1 /* quant_bits value of the half-precision descriptor mode */
#define CBVH_QUANT_SVB 2  /* quant_bits value of the Stream VByte mode (exact deltas, 1-4 bytes) */
#define CBVH_EARLY_EXIT 1u /* stop each pose at its first intersecting pair (pair outputs must be NULL);
                            * implied whenever no pair outputs are requested */
#define CBVH_SORT_PAIRS 2u /* sort each pose's pair list by (i, j) */

typedef struct cbvh_bvh cbvh_bvh; /* opaque; immutable once built; concurrent reads are safe */

typedef struct {
  int64_t n_tris;
  int64_t n_nodes;
  int64_t n_treelets;
  int64_t blob_bytes;   /* bytes of the device blob, triangles included */
  int64_t node_bytes;   /* bytes of the treelets alone (the compressed hierarchy) */
  int32_t k, branching, quant_bits, treelet_bytes;
  int32_t lattice_exp;  /* e: lattice step 2^e */
  int32_t depth;        /* tree depth (edges from the root to the deepest leaf) */
  int32_t max_treelet_depth;
  int32_t local_bits;   /* node reference = (treelet << local_bits) | local index */
} cbvh_info_t;

/* Last error message of the calling thread ("" if none). */
const char *cbvh_last_error(void);

/* Build the compressed BVH of a triangle mesh on the host.
 *   verts_host: n_verts x 3 FP32; tris_host: n_tris x 3 int32 vertex indices.
 *   k: 6, 18, 24 or 26 DOP values per node (Table 1: "k floats" per k-DOP); the k/2 slab
 *      directions are fixed unnormalised integer vectors (axes, then edge diagonals, then
 *      corner diagonals).
 *   branching: 2, 4, 8 or 16 children per inner node; one triangle per leaf; each node is
 *      split by log2(branching) rounds of median splits on the longest centroid axis.
 *   quant_bits: 8 or 16 -- slab bounds quantised on one lattice of step 2^e ("we quantify
 *      BV", abstract) and stored as predictor-corrector deltas (Sec. III-B): predictor =
 *      the parent's decoded interval, corrector = outward b-bit delta; CBVH_QUANT_FP16
 *      (1) -- absolute half-precision bounds, lo rounded down and hi rounded up (the
 *      half-float descriptors of Sec. III-A; bounds beyond +-65504 become infinite); 0 --
 *      uncompressed FP32 bounds; CBVH_QUANT_SVB (2) -- the integer compression the
 *      conclusion proposes: exact lattice bounds, each node's interval stored as unsigned
 *      deltas to its parent's in the Stream VByte format (Lemire, Kurz and Rupp 2018: a
 *      2-bit length code per delta in an 8-byte control word, then 1 to 4 bytes per
 *      delta), records of varying size found through a per-treelet offset table.  Stream
 *      VByte hierarchies are not refitted, built on the device or batched
 *      (CBVH_ERR_ARG).
 *   treelet_bytes: power of two in [4096, 131072]; the hierarchy is clustered into treelets
 *      of at most this size (Sec. III-B), each with an absolute root for random access.
 * On success *out receives a handle owning host memory only; attach a device copy of its
 * blob with cbvh_attach before querying.  Errors: CBVH_ERR_ARG, CBVH_ERR_MESH. */
int cbvh_build(const float *verts_host, int64_t n_verts, const int32_t *tris_host, int64_t n_tris, int k,
               int branching, int quant_bits, int treelet_bytes, cbvh_bvh **out);

/* Free a handle (host memory only; the attached device blob stays the caller's). */
int cbvh_free(cbvh_bvh *h);

int cbvh_info(const cbvh_bvh *h, cbvh_info_t *out);

/* The host copy of the blob (read-only, owned by the handle, valid until cbvh_free). */
int cbvh_blob_host(const cbvh_bvh *h, const uint8_t **blob_host, int64_t *bytes);

/* Write a hierarchy to a file: a 16-byte header (magic "CBVF", format version 1, the
 * vertex count as int64) followed by the blob bytes of cbvh_blob_host.  Errors:
 * CBVH_ERR_ARG (NULL), CBVH_ERR_STATE (a plan without geometry, or a host copy left stale
 * by a device build), CBVH_ERR_IO. */
int cbvh_save(const cbvh_bvh *h, const char *path);
/* Read a hierarchy written by cbvh_save into a new handle (host memory only; attach it
 * before querying).  The blob is checked completely before it is accepted, so that no
 * kernel can read outside it:
 *   - the header's fields against the build rules;
 *   - the treelet offsets (ordered, inside the blob);
 *   - every record's parent, children, leaf slot and depth;
 *   - the offset tables of Stream VByte treelets;
 *   - the triangle table's indices.
 * Errors: CBVH_ERR_ARG (NULL), CBVH_ERR_IO (unreadable, or not a valid hierarchy, with the
 * first failed check in cbvh_last_error). */
int cbvh_load(const char *path, cbvh_bvh **out);

/* Copy the blob into caller-owned device memory `dev_blob` (>= blob_bytes, 256-byte
 * aligned) on `stream` and remember that address for queries.  The caller keeps the buffer
 * alive and unchanged while the handle is used.  Errors: CBVH_ERR_ARG, CBVH_ERR_CUDA. */
int cbvh_attach(cbvh_bvh *h, void *dev_blob, int64_t bytes, void *stream);

/* Test hook: decode every node on the device, in blob order (treelet by treelet, local
 * index order).  lattice_out: n_nodes x (k/2) x 2 int32 decoded lattice bounds [lo, hi]
 * (not written when quant_bits = 0 or 1; may be NULL); bounds_out: n_nodes x (k/2) x 2 FP32
 * bounds (lo rounded down, hi rounded up).  Asynchronous on `stream`. */
int cbvh_decode_all(const cbvh_bvh *h, int32_t *lattice_out, float *bounds_out, void *stream);

/* Bytes of device workspace a query needs (256-byte aligned pointer, contents need not be
 * initialised).  mode: 0 = collide, 1 = distance; pair_capacity is ignored for distance
 * and for collide without pair outputs. */
int cbvh_workspace_bytes(const cbvh_bvh *A, const cbvh_bvh *B, int64_t n_poses, int mode, int64_t pair_capacity,
                         int64_t *bytes);

/* Collision detection, Algorithm 1 with checkPrimitives = closed triangle-triangle
 * intersection, for n poses of B against A.  "a and b intersect" is tested both ways,
 * rounded outward: B's box moved by the pose against A's k-DOP slabs, then A's axis box
 * moved into B's frame against B's box (a leaf of B: its triangle's box).
 *   poses: n x 12 FP32.  hit: n bytes, 1 if any triangle of A meets a triangle of R B + t.
 *   pair_offsets (n + 1 int64) and pairs (2 x pair_capacity int32, (i, j) = (triangle of A,
 *   triangle of B)): the per-pose intersecting pairs in CSR form, or both NULL.
 *   pairs_needed: device int64 scalar receiving the total number of pairs (may be NULL
 *   when pairs are not requested).  If it exceeds pair_capacity, hit and pair_offsets are
 *   still written, pairs is not, and `status` reads CBVH_ERR_CAPACITY: reallocate and call
 *   again.  flags: CBVH_EARLY_EXIT, CBVH_SORT_PAIRS. */
int cbvh_collide(const cbvh_bvh *A, const cbvh_bvh *B, const float *poses, int64_t n, uint8_t *hit,
                 int64_t *pair_offsets, int32_t *pairs, int64_t pair_capacity, int64_t *pairs_needed, uint32_t flags,
                 void *workspace, int64_t workspace_bytes, int32_t *status, void *stream);

/* Proximity query: dist[p] = minimum distance between the triangles of A and those of
 * R_p B + t_p (0 when they intersect), by branch-and-bound Algorithm 1.  A node pair is
 * pruned when its lower bound reaches the best distance found: the largest of the widest
 * slab gap over |d_j|, the distance between the two axis boxes (root of the summed squared
 * x, y and z gaps), and the same distance in B's frame (A's box moved into it), all
 * rounded down.  A collision pass with early exit runs
 * first and settles the intersecting poses at 0.  FP32; accurate to a few ulps of the
 * scene size. */
int cbvh_distance(const cbvh_bvh *A, const cbvh_bvh *B, const float *poses, int64_t n, float *dist, void *workspace,
                  int64_t workspace_bytes, int32_t *status, void *stream);

/* Proximity query that allocates nothing and takes no workspace: the same computation and
 * results as cbvh_distance, for callers that cannot hand the library device memory at
 * query time -- for example a planner's control loop that must never block on the device
 * allocator once it runs, or a plug-in whose host application owns all device memory.
 * The paper has no counterpart; it is a packaging of the same query.
 *   Schedule: cbvh_distance's two passes (early-exit collision, then branch and bound) with
 *   its work mapping and budgets (CBVH_OPT_SPLIT, CBVH_OPT_BUDGET0), run over chunks of at
 *   most 2^14 poses (enough to fill the GPU, few enough for the task buffers below).
 *   Scratch: a fixed 64 MiB array inside the library, reserved on every GPU that loads it
 *   until the process exits.  It holds the query's counters, the intersection flags of one
 *   chunk, two task buffers of 2^20 entries (a chunk of the terrain workload hands on about
 *   52 tasks per pose; tasks that find the buffer full run on where they are, which is
 *   slower but gives the same results) and one node-pair stack per warp, as many as fit.  A
 *   pair of hierarchies whose stack bound leaves room for fewer than 4 warps would be
 *   rejected with CBVH_ERR_WORKSPACE and a message giving the bytes needed; no pair this
 *   library builds comes near that (the bound is at most 4,336 entries, 52 KB a warp).
 *   The pose count itself is not limited by the array.
 *   Set-up: the first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   Sharing: every call uses the same array and it keeps the previous call's contents (the
 *   counters are cleared at the start of each call); calls whose work overlaps on the GPU,
 *   on different streams or threads, race and give wrong results -- serialise them.
 *   Arguments, outputs and errors are those of cbvh_distance. */
int cbvh_distance_noalloc(const cbvh_bvh *A, const cbvh_bvh *B, const float *poses, int64_t n, float *dist,
                          int32_t *status, void *stream);

/* ---- batched queries (one pass of persistent launches over many work items) ----
 * A work item pairs a static hierarchy A with a posed hierarchy B for n poses and asks for
 * collision flags (mode 0; flags CBVH_EARLY_EXIT or 0, which act the same: with flags only,
 * every pose stops at its first intersecting pair) or distances (mode 1).  Items that
 * share the query kind and A's k run in one set of persistent launches, so items of very
 * different sizes (robot links against a scene, many requests) share the GPU.  Outputs and
 * semantics per item are those of cbvh_collide without pairs and of cbvh_distance. */
typedef struct {
  const cbvh_bvh *A;  /* static side (attached) */
  const cbvh_bvh *B;  /* posed side (attached) */
  int32_t mode;       /* 0 = collision detection, 1 = proximity query */
  uint32_t flags;     /* mode 0: CBVH_EARLY_EXIT or 0; mode 1: 0 */
  const float *poses; /* device, n x 12 */
  int64_t n;
  uint8_t *hit;       /* device, n bytes (mode 0) */
  float *dist;        /* device, n floats (mode 1) */
  /* device, n bytes, or NULL (mode 0 only).  Items that pass the same array form one
   * configuration set -- e.g. the links of a robot over one list of configurations, whose
   * answer is "some link collides" -- and must have the same n.  The launch clears it;
   * afterwards any_hit[i] = 1 iff pose i of some item of the set intersects.  Pose i of an
   * item stops (or is never started) once another item of the set has set any_hit[i], so
   * that item's own hit[i] is then 0: with a set, only any_hit and the items' 1s are
   * exact. */
  uint8_t *any_hit;
  /* device, n floats, or NULL (mode 1 only).  Distance items that pass the same array form
   * a configuration set (e.g. the links of a robot, whose clearance is the smallest distance
   * over its links) and must have the same n.  The launch resets it; afterwards
   * min_dist[i] is the smallest distance over the set's items at pose i, within the
   * distance tolerance of cbvh_distance.  Each item prunes with the set's best distance so
   * far, so an item's own dist[i] is then only an upper bound of its distance (a distance
   * of one of its own triangle pairs, or +inf), exact where it is the set's minimum. */
  float *min_dist;
} cbvh_query_t;

typedef struct cbvh_batch cbvh_batch; /* opaque host-side plan of a batch */

/* Plan a batch (host only; queries_host is copied).  Errors: CBVH_ERR_ARG, CBVH_ERR_STATE. */
int cbvh_batch_create(const cbvh_query_t *queries_host, int64_t n_queries, cbvh_batch **out);
int cbvh_batch_free(cbvh_batch *b);
/* Device workspace bytes the batch needs (256-byte aligned). */
int cbvh_batch_workspace_bytes(const cbvh_batch *b, int64_t *bytes);
/* Write the batch's item table into the workspace (copies and synchronises `stream`). */
int cbvh_batch_upload(const cbvh_batch *b, void *workspace, int64_t workspace_bytes, void *stream);
/* Enqueue the batch on `stream`: memsets and kernel launches only, no synchronisation and
 * no host copies, so the call can be captured in a CUDA graph and replayed (the poses and
 * outputs named at cbvh_batch_create are read and written at each replay).  Requires a
 * previous cbvh_batch_upload into the same workspace.  Device errors go to `status`. */
int cbvh_batch_launch(const cbvh_batch *b, void *workspace, int64_t workspace_bytes, int32_t *status, void *stream);

/* Process-wide tuning options; the paper has no counterpart.
 *   CBVH_OPT_STAGE_BYTES: bytes of leading treelets of each hierarchy that every thread block
 *   copies into shared memory (TMA bulk copy) before a single query, 0..32768 (default 0,
 *   off: on the terrain workload the top treelets are L1-resident anyway and staging costs
 *   occupancy).  Takes effect for queries issued afterwards. */
#define CBVH_OPT_STAGE_BYTES 1
/*   CBVH_OPT_SPLIT: work mapping (scheduling only; results do not change).
 *     0: one persistent launch in which each warp traverses whole poses (warp per pose).
 *     1: rounds of persistent launches: a task that exceeds its expansion budget hands its
 *        node-pair stack on as tasks for the next round (warp per node pair); the last
 *        round runs every task to the end.
 *     2: one launch over a work queue: warps take poses, then the tasks that busy warps
 *        donate from the bottom of their stacks while other warps wait (work donation).
 *     3: the rounds of 1, with the last round run as the work queue of 2.
 *     4 (default): 2 for collision detection with pair lists, 3 for early-exit collision
 *        detection (including every query without pair outputs) and proximity queries. */
#define CBVH_OPT_SPLIT 2
/*   CBVH_OPT_BUDGET0: node-pair expansions a task may run in round 0 before it hands the rest
 *   of its work on (default 256; later rounds allow 2, 4, 8 and 32 times as many, the last
 *   round no limit).  Queries that exit at the first hit use their own, larger budgets. */
#define CBVH_OPT_BUDGET0 3
/*   CBVH_OPT_TREELET_PACKING: how cbvh_build forms treelets (Sec. III-B sizes them to the
 *   cache; how nodes are grouped is not given).  Both keep whole sibling groups together and
 *   give each treelet an absolute root, so the blob format and every query result are the
 *   same; footprint and decode-chain length differ.  Takes effect for builds started
 *   afterwards; the value is recorded in the blob header (bytes 44..47).
 *     CBVH_PACK_TOP_DOWN (default): greedy breadth-first growth from each root; a sibling
 *     group that does not fit makes each of its nodes a new root.  Leaves many small
 *     treelets near the leaves.
 *     CBVH_PACK_BOTTOM_UP: a node's children join its treelet while the node and all the
 *     nodes its children still carry fit one treelet; otherwise each child roots a treelet.
 *     Fewer, fuller treelets and fewer absolute roots; deeper chains below a root. */
#define CBVH_OPT_TREELET_PACKING 4
/*   CBVH_OPT_LATTICE_HEADROOM: bits of the lattice range cbvh_build keeps free, 0..8
 *   (default 0): the lattice step 2^e is the smallest with every |bound| / 2^e below
 *   2^(30 - headroom) instead of 2^30.  cbvh_refit keeps e and accepts bounds up to 2^30
 *   steps, so a hierarchy built with headroom h can be refitted to a mesh up to 2^h times
 *   larger; each bit costs one bit of lattice resolution.  Takes effect for builds started
 *   afterwards. */
#define CBVH_OPT_LATTICE_HEADROOM 5
/*   CBVH_OPT_WAIT_CAP: polls a bounded device wait makes before it gives up, 1..2^24
 *   (default 2^24, about a minute with the wait's backoff).  It bounds the wait of an idle
 *   warp for donated work in a work-queue launch and a block's first wait for its staged
 *   treelets.  A wait that runs out sets `status` to CBVH_ERR_TIMEOUT and the kernel
 *   returns; that query's results are then incomplete, and later queries are unaffected.
 *   (Copies still in flight always get the full default wait before a block moves on.)
 *   A small cap makes a query report CBVH_ERR_TIMEOUT on purpose, which is how failure
 *   handling is tested.  Takes effect for queries issued afterwards. */
#define CBVH_OPT_WAIT_CAP 6
#define CBVH_PACK_TOP_DOWN 0
#define CBVH_PACK_BOTTOM_UP 1
int cbvh_set_option(int option, int64_t value);

/* ---- device refit for deforming meshes (the tree is kept, the bounds recomputed) ----
 * New positions for the build's vertices (same count, same triangles): every node's exact
 * lattice bounds are recomputed from them on the device and the attached blob's bound
 * fields and triangle table are rewritten in place.  The tree, the treelets and the
 * lattice exponent stay those of the build, so the blob is byte-identical to encoding the
 * build's tree with the new vertices (the host copy from cbvh_blob_host is not updated).
 * A deformation that reorders the median splits leaves the tree valid but less tight;
 * rebuild when it matters.
 *   cbvh_refit_workspace_bytes: device bytes of the plan and scratch (about 24 B per node,
 *     16 B per node and direction, 8 B per vertex and direction).
 *   cbvh_refit_prepare: writes the node plan into `workspace` (256-byte aligned, caller-
 *     owned, kept unchanged between refits) and synchronises `stream`; once per handle and
 *     workspace.
 *   cbvh_refit: verts_dev n_verts x 3 FP32 (n_verts: the build's vertex count) and tris_dev
 *     n_tris x 3 int32 (the build's triangles), device pointers; asynchronous on `stream`, no synchronisation, so it can
 *     be captured in a CUDA graph.  A vertex that is not finite or leaves the lattice's
 *     range (|d.v| >= 2^30 steps), or a bound beyond +-65504 for quant_bits = 1, sets
 *     `status` to CBVH_ERR_MESH; the blob is then unspecified until a successful refit.
 * Errors: CBVH_ERR_ARG, CBVH_ERR_STATE (not attached, or workspace not prepared),
 * CBVH_ERR_WORKSPACE, CBVH_ERR_CUDA. */
int cbvh_refit_workspace_bytes(const cbvh_bvh *h, int64_t *bytes);
int cbvh_refit_prepare(cbvh_bvh *h, void *workspace, int64_t workspace_bytes, void *stream);
int cbvh_refit(cbvh_bvh *h, const float *verts_dev, int64_t n_verts, const int32_t *tris_dev, void *workspace,
               int64_t workspace_bytes, int32_t *status, void *stream);

/* ---- device-side build for per-frame meshes ----
 * The same hierarchy as cbvh_build, built on the GPU from a device mesh; the blob is
 * byte-identical to cbvh_build's for the same mesh, parameters and options.  The shape of the
 * tree (child counts, treelets, topology words) follows from the triangle count and the
 * branching alone, since every node's triangles are halved log2(branching) times by the
 * median split (Sec. III); the geometry only decides which triangle ends in which leaf, the
 * lattice exponent and the bounds.
 *   cbvh_build_plan: host, no mesh data.  A handle for meshes of n_verts vertices and
 *     n_tris triangles: its blob holds the shape with zero bounds and an empty triangle table
 *     (queries refuse it with CBVH_ERR_STATE until a device build succeeds).  Treelet packing
 *     and lattice headroom are the options in force now.  Attach it (cbvh_attach) before
 *     the first device build.  Errors as cbvh_build's parameter checks.
 *   cbvh_build_device_workspace_bytes: device bytes of the build's scratch (about 110 B per
 *     triangle, plus the refit plan of cbvh_refit_workspace_bytes at its front).
 *   cbvh_build_device: verts_dev n_verts x 3 FP32, tris_dev n_tris x 3 int32 (device
 *     pointers, the plan's counts); workspace 256-byte aligned, caller-owned and kept
 *     unchanged between builds (the node plan is uploaded into it by the first build with
 *     that workspace, and again whenever another workspace is passed).  Builds into
 *     the attached blob on `stream` and synchronises it (the lattice exponent is read back
 *     once).  May be called again with new geometry of the same counts (a new frame); the
 *     workspace also serves cbvh_refit afterwards.  flags: CBVH_BUILD_HOST_COPY copies the
 *     blob back into the host copy (cbvh_blob_host); without it the host copy is stale and
 *     cbvh_blob_host / cbvh_attach refuse with CBVH_ERR_STATE.
 *   The mesh checks are cbvh_build's, reported as CBVH_ERR_MESH: an out-of-range index, a
 *   zero-area triangle, a non-finite vertex, no extent, coordinates outside the lattice's
 *   range, bounds beyond +-65504 for quant_bits = 1.  On any error the handle has no
 *   geometry until the next successful build.
 * Errors: CBVH_ERR_ARG, CBVH_ERR_STATE (not a plan, not attached), CBVH_ERR_WORKSPACE,
 * CBVH_ERR_MESH, CBVH_ERR_CUDA. */
#define CBVH_BUILD_HOST_COPY 1u
int cbvh_build_plan(int64_t n_verts, int64_t n_tris, int k, int branching, int quant_bits, int treelet_bytes,
                    cbvh_bvh **out);
int cbvh_build_device_workspace_bytes(const cbvh_bvh *h, int64_t *bytes);
int cbvh_build_device(cbvh_bvh *h, const float *verts_dev, const int32_t *tris_dev, void *workspace,
                      int64_t workspace_bytes, uint32_t flags, void *stream);

/* Kernels this library has launched in this process so far (every traversal round, every
 * compaction kernel, the decode hook); a count the caller can difference around a region.
 * Host only; no synchronisation.  Errors: CBVH_ERR_ARG (NULL). */
int cbvh_kernel_launches(int64_t *count);

/* Work counters of the last query that used `workspace`: stats_host[0] = BV-pair tests
 * (bounding-volume overlap or lower-bound tests, Algorithm 1's "a and b intersect"),
 * stats_host[1] = leaf tests (checkPrimitives calls), stats_host[2] = node-pair expansions
 * (one per recursive call of Algorithm 1 that reaches an inner node).  Copies 24 bytes to
 * the host and synchronises `stream`.  The paper has no such call; it feeds the BV-pair
 * tests/s metric. */
int cbvh_query_stats(const void *workspace, int64_t *stats_host, void *stream);

/* Profiling of the traversal kernels alone.  While enabled (on != 0), every query on this
 * host thread records pairs of library-owned CUDA events on its stream immediately around
 * its traversal launches and its output compaction.  The paper has no such call; it feeds
 * the roofline measurement. */
int cbvh_profile_enable(int on);

/* Waits for the recorded event pairs of this host thread and returns, per slot, the summed
 * time in ms (ms_host[3]) and the number of timed launch groups (launches_host[3]; a
 * distance query has two, one per pass): slot 0 = the
 * traversal kernels of collide, 1 = those of distance (both of its passes), 2 = collide's
 * output compaction (scan, scatter, sort); then forgets them. */
int cbvh_profile_collect(double *ms_host, int64_t *launches_host);

/* Machine-ceiling probe: the L2 read bandwidth against which the traversal of hierarchies
 * that stay in L2 is measured.  The paper has no counterpart.  Streams the caller's device
 * `buffer` (`bytes` >= 16 KiB, a multiple of 16, 16-byte aligned; pick a size well inside
 * L2) once to make it resident, then `reps` more times with 16-byte loads that bypass L1
 * and are cached in L2 only, from every SM, timed with CUDA events on `stream` (the call
 * synchronises).  gbs_host: bytes read / time, in GB/s.  sink: a device uint32 the kernel
 * may write (keeps its loads live).  Errors: CBVH_ERR_ARG, CBVH_ERR_CUDA. */
int cbvh_probe_l2_read(const void *buffer, int64_t bytes, int reps, uint32_t *sink, double *gbs_host, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CBVH_H */
