// Private declarations shared by the host builder and the CUDA query code of libcbvh.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "cbvh.h"

#if defined(__CUDACC__) || defined(CBVH_WITH_NVTX)
#include <nvtx3/nvToolsExt.h>
namespace cbvh {
// Named NVTX range around a host entry point, for timeline tools (Nsight Systems and the
// like); without a tool attached a push or pop is one check of a function pointer.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace cbvh
#define CBVH_RANGE(name) cbvh::NvtxRange cbvh_nvtx_range_(name)
#else
#define CBVH_RANGE(name) ((void)0)
#endif

struct cbvh_bvh {
  // parameters
  int k = 0, K = 0, m = 0, bits = 0, treelet_bytes = 0;
  // derived layout
  int e = 0;           // lattice step 2^e
  int lbits = 1;       // node reference = (treelet << lbits) | local
  int max_tdepth = 0;  // deepest node below its treelet root
  int depth = 0;       // tree depth
  int rec_bytes = 0, root_bytes = 0;
  int64_t n_tris = 0, n_nodes = 0, n_treelets = 0, n_verts = 0;
  int64_t off_treelets = 0, off_tris = 0;
  std::vector<uint8_t> blob;  // host copy of the blob
  // device copy (caller-owned memory)
  void *dev_blob = nullptr;
  int device = -1;
  // refit plan (cbvh_refit_prepare): node ranges of each tree level and each treelet depth,
  // and the workspace holding the plan's device arrays
  std::vector<int64_t> refit_level_start, refit_td_start;
  void *refit_ws = nullptr;
  // lattice bits kept free by the build (CBVH_OPT_LATTICE_HEADROOM at build or plan time)
  int headroom = 0;
  // false for a plan (cbvh_build_plan) until its first cbvh_build_device: the blob holds the
  // tree's shape, zero bounds and an empty triangle table
  bool geometry = true;
  // plan: position in the median-split order of each leaf slot's triangle
  std::vector<int32_t> leaf_pos;
  // the host blob lags the device blob (a device build without CBVH_BUILD_HOST_COPY)
  bool host_stale = false;
  // workspace holding the device build's plan arrays (cbvh_build_device)
  void *devbuild_ws = nullptr;
};

namespace cbvh {
// Records a message for cbvh_last_error() and returns `code`.
int fail(int code, const std::string &msg);
void clear_error();
// Treelet formation used by cbvh_build (CBVH_PACK_*), set by cbvh_set_option.
void set_treelet_packing(int packing);
int treelet_packing();
// Lattice bits cbvh_build keeps free (CBVH_OPT_LATTICE_HEADROOM), set by cbvh_set_option.
void set_lattice_headroom(int bits);
int lattice_headroom();
// Adds to the process-wide count of kernels launched (cbvh_kernel_launches).
void count_launches(int n);
// Workspace bytes of the refit plan and scratch (the front of a device-build workspace).
int64_t refit_workspace_total(const cbvh_bvh *h);
// The refit kernels (bounds bottom-up, encoding top-down) for lattice exponent h->e on
// `stream`, reporting into the device int32 `status`; adds to `launches`.
int refit_launch(cbvh_bvh *h, const float *verts_dev, const int32_t *tris_dev, uint8_t *workspace,
                 int32_t *status, void *stream, int &launches);
}  // namespace cbvh
