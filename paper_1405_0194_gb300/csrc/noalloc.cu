// Allocation-free form of the trace reduction Tr[X S] (X = DM, EDM, FDM).
//
// Some callers cannot allocate device memory at the point where they need the
// traces: code running while a stream is being captured into a CUDA graph
// (cudaMalloc is not allowed there), runtimes that hand the library a fixed
// memory arena and forbid further allocation, and real-time or serving loops
// that must not take the allocator's locks or risk an out-of-memory error in
// the middle of a request. pexsi_trace_noalloc serves them: it takes device
// inputs and a device output and uses, as scratch for its block partial sums,
// a file-scope __device__ array that exists in every GPU's memory from the
// moment the library is loaded until the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/pexsi_gb300.h"

namespace {

constexpr int kNoAllocBlocks = 1024;                     // partial-sum slots
constexpr int64_t kNoAllocMaxChunk = int64_t(1) << 20;   // entries per block, at most
constexpr int kMaxDevices = 64;

// Scratch of the reduction: 3 partial sums per block (24 KiB per device).
static __device__ __align__(256) double g_trace_scratch[3 * kNoAllocBlocks];

std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Each block sums a fixed contiguous range of entries in a fixed order, then
// a tree in shared memory; the final kernel adds the block results in block
// order, so repeated calls give bit-identical results.
__global__ void k_trace_partial_static(const double* __restrict__ dm, const double* __restrict__ edm,
                                       const double* __restrict__ fdm, const double* __restrict__ S, int64_t nnz,
                                       int64_t chunk, double* __restrict__ partials) {
  __shared__ double red[3][256];
  const int64_t lo = int64_t(blockIdx.x) * chunk;
  const int64_t hi = lo + chunk < nnz ? lo + chunk : nnz;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const double s = S[e];
    if (dm) a = fma(dm[e], s, a);
    if (edm) b = fma(edm[e], s, b);
    if (fdm) c = fma(fdm[e], s, c);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partials[3 * blockIdx.x + q] = red[q][0];
}

// Naming g_trace_scratch here also keeps the internal-linkage array in the
// device image, which cudaGetSymbolAddress needs; a pointer that is not the
// array (a host-side stand-in passed by mistake) poisons the result with NaN.
__global__ void k_trace_final_static(const double* __restrict__ partials, int nblocks, double* __restrict__ out3) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int t = 0; t < nblocks; ++t) s += partials[3 * t + threadIdx.x];
    out3[threadIdx.x] = (partials == g_trace_scratch) ? s : __longlong_as_double(0x7FF8000000000000ll);
  }
}

// Device address of the scratch array for the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_trace_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int pexsi_trace_noalloc(const double* d_dm, const double* d_edm, const double* d_fdm,
                                   const double* d_S, int64_t nnz, double* d_out3, void* stream) {
  if (!d_S || !d_out3 || nnz < 0) return PEXSI_ERR_INVALID_ARG;
  if (nnz > int64_t(kNoAllocBlocks) * kNoAllocMaxChunk) return PEXSI_ERR_INVALID_ARG;
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return PEXSI_ERR_CUDA;
  int64_t nblocks = (nnz + 4095) / 4096;
  if (nblocks < 1) nblocks = 1;
  if (nblocks > kNoAllocBlocks) nblocks = kNoAllocBlocks;
  int64_t chunk = (nnz + nblocks - 1) / nblocks;
  if (chunk < 1) chunk = 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The launches' own return codes are checked, so an error that another
  // component left pending in the runtime is neither cleared nor taken for
  // one of these launches.
  int nb = int(nblocks);
  void* args1[] = {&d_dm, &d_edm, &d_fdm, &d_S, &nnz, &chunk, &scratch};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_trace_partial_static), dim3(nb), dim3(256), args1, 0, st) !=
      cudaSuccess)
    return PEXSI_ERR_CUDA;
  void* args2[] = {&scratch, &nb, &d_out3};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_trace_final_static), dim3(1), dim3(32), args2, 0, st) !=
      cudaSuccess)
    return PEXSI_ERR_CUDA;
  return PEXSI_OK;
}
