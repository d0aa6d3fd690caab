// Machine-ceiling probe of libcbvh: the L2 read bandwidth the traversal's roofline is taken
// against.  The paper has no counterpart; the traversal's hierarchies of the smaller
// workloads sit in L2, so L2 bandwidth, not HBM, is their memory ceiling.
//
// l2_read_kernel streams a buffer small enough to stay resident in L2 with 16-byte loads
// that bypass L1 (ld.global.cg), every warp reading whole 512-byte lines in turn, grid sized
// to fill every SM; the sum of what each thread read is written out so that no load is dead.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace {

__device__ __forceinline__ uint4 ld_cg(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__global__ void __launch_bounds__(512) l2_read_kernel(const uint4 *buf, int64_t n16, int reps, uint32_t *sink) {
  uint32_t acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    // start each pass at another offset so that consecutive passes of one thread do not
    // read the same line back to back
    const int64_t shift = (int64_t)r * 4096;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      int64_t j = i + shift;
      if (j >= n16) j -= n16;
      const uint4 v = ld_cg(buf + j);
      acc ^= v.x + v.y + v.z + v.w;
    }
  }
  if (acc == 0x9e3779b9u) sink[0] = acc;  // practically never; keeps the loads live
}

int cuda_fail(cudaError_t e, const char *what) {
  return cbvh::fail(CBVH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" int cbvh_probe_l2_read(const void *buffer, int64_t bytes, int reps, uint32_t *sink, double *gbs_host,
                                  void *stream) {
  cbvh::clear_error();
  if (!buffer || !sink || !gbs_host || bytes < 16 * 1024 || (bytes & 15) || reps < 1 ||
      (reinterpret_cast<uintptr_t>(buffer) & 15))
    return cbvh::fail(CBVH_ERR_ARG, "bad argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n16 = bytes / 16;
  const unsigned blocks = (unsigned)sms * 4;  // 4 x 512 threads per SM: 64 warps, full occupancy
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(e, "cudaEventCreate");
  }
  // one pass to bring the buffer into L2, then the timed passes
  l2_read_kernel<<<blocks, 512, 0, s>>>(static_cast<const uint4 *>(buffer), n16, 1, sink);
  cudaEventRecord(a, s);
  l2_read_kernel<<<blocks, 512, 0, s>>>(static_cast<const uint4 *>(buffer), n16, reps, sink);
  cudaEventRecord(b, s);
  cbvh::count_launches(2);
  e = cudaGetLastError();
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "L2 probe");
  *gbs_host = (double)bytes * reps / (ms * 1e6);
  return CBVH_OK;
}
