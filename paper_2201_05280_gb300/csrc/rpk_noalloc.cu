// rpk_field_totals_noalloc: FP64 conserved totals of hydrodynamic fields that
// the caller keeps in device memory, computed without allocating anything.
//
// Who needs this: callers that are not allowed to call cudaMalloc at the point
// where they want the totals. One kind is an application whose own memory
// manager owns all of the device memory (a pooling allocator that accounts
// for every byte, or a fixed budget shared with other work) and forbids
// libraries to allocate behind its back. Another is a loop that must not
// stall: cudaMalloc and cudaFree can synchronise the device, which would
// serialise work that other streams have in flight. Such a caller already
// holds rho, u, theta_T and theta_R (for example filled by rpk_read_moments
// with on_device = 1) and only needs a reduction.
//
// Scratch: the per-block partial sums live in one file-scope __device__ array
// of kMaxChunks x kVals doubles (320 KiB). Every GPU that loads the library
// keeps that array until the process exits. Each call uses one block per chunk
// of kChunk points, so one call reduces at most kMaxChunks * kChunk points.
// Every block writes all of its own slots before the final pass reads them,
// and the final pass reads only the slots of this call's blocks, so no part
// of the array has to start at zero and nothing is cleared. All calls, on any
// stream, share the array: calls whose kernels overlap on the GPU race and
// must be ordered by the caller (same stream, or events).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "rpk_internal.h"

namespace {

constexpr int kChunk = 8192;      // points reduced by one block
constexpr int kMaxChunks = 8192;  // slots in the static scratch
constexpr int kVals = 5;          // M, Jx, Jy, Jz, E
constexpr int kThreads = 256;

static __device__ __align__(256) double g_totals_scratch[kMaxChunks * kVals];

// Host-side copy of the scratch's device address, one per device, filled at
// the first call on that device (cudaGetSymbolAddress with that device
// current). In host code the name g_totals_scratch is only a stand-in.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block b sums points [b*kChunk, min((b+1)*kChunk, n)) and writes its 5 slots.
__global__ void __launch_bounds__(kThreads)
    k_totals_partial(const double* __restrict__ rho, const double* __restrict__ u,
                     const double* __restrict__ T, const double* __restrict__ R, int64_t n,
                     double delta, double* __restrict__ scratch) {
  double acc[kVals] = {0, 0, 0, 0, 0};
  const int64_t begin = (int64_t)blockIdx.x * kChunk;
  const int64_t end = begin + kChunk < n ? begin + kChunk : n;
  for (int64_t p = begin + threadIdx.x; p < end; p += kThreads) {
    const double r = rho[p], ux = u[p], uy = u[n + p], uz = u[2 * n + p];
    acc[0] += r;
    acc[1] += r * ux;
    acc[2] += r * uy;
    acc[3] += r * uz;
    acc[4] += 0.5 * r * (ux * ux + uy * uy + uz * uz) + 1.5 * r * T[p] + 0.5 * delta * r * R[p];
  }
  __shared__ double red[kThreads / 32][kVals];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kVals; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kVals) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][threadIdx.x];
    scratch[(int64_t)blockIdx.x * kVals + threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(1024)
    k_totals_final(const double* __restrict__ scratch, int nchunks, double* __restrict__ out) {
  __shared__ double red[32][kVals];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < kVals; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nchunks; b += blockDim.x) v += scratch[(int64_t)b * kVals + k];
    v = warp_sum(v);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kVals) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w][threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// Device address of the scratch on the current device (set up on first use).
rpk_status scratch_on_current_device(double** ptr) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return rpk::cuda_fail(err, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    rpk::set_error("rpk_field_totals_noalloc supports device ordinals below 64");
    return RPK_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_totals_scratch);
    if (err != cudaSuccess) return rpk::cuda_fail(err, "cudaGetSymbolAddress(g_totals_scratch)");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return RPK_OK;
}

}  // namespace

extern "C" rpk_status rpk_field_totals_noalloc(const double* rho, const double* u,
                                               const double* theta_T, const double* theta_R,
                                               int64_t npts, double delta, void* cuda_stream,
                                               double* out) {
  if (!rho || !u || !theta_T || !theta_R || !out) {
    rpk::set_error("rpk_field_totals_noalloc: NULL pointer");
    return RPK_ERR_ARG;
  }
  if (npts < 1 || npts > (int64_t)kMaxChunks * kChunk) {
    rpk::set_error("rpk_field_totals_noalloc: npts must lie in [1, " +
                   std::to_string((int64_t)kMaxChunks * kChunk) +
                   "], the capacity of its static scratch (" +
                   std::to_string(kMaxChunks) + " chunks of " + std::to_string(kChunk) +
                   " points)");
    return RPK_ERR_ARG;
  }
  if (!(delta >= 0.0) || !std::isfinite(delta)) {
    rpk::set_error("rpk_field_totals_noalloc: delta must be finite and >= 0");
    return RPK_ERR_PARAM;
  }
  double* scratch = nullptr;
  rpk_status st = scratch_on_current_device(&scratch);
  if (st != RPK_OK) return st;
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return rpk::cuda_fail(err, "cudaGetDevice");
  // every pointer must be device memory of the current device: the kernels
  // run there and would otherwise read another GPU's or the host's memory
  const void* ptrs[5] = {rho, u, theta_T, theta_R, out};
  const char* names[5] = {"rho", "u", "theta_T", "theta_R", "out"};
  for (int k = 0; k < 5; ++k) {
    cudaPointerAttributes a{};
    err = cudaPointerGetAttributes(&a, ptrs[k]);
    if (err != cudaSuccess) {
      cudaGetLastError();
      rpk::set_error(std::string("rpk_field_totals_noalloc: ") + names[k] +
                     " is not device memory of the current device (no CUDA pointer)");
      return RPK_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice || a.device != dev) {
      rpk::set_error(std::string("rpk_field_totals_noalloc: ") + names[k] +
                     " is not device memory of the current device " + std::to_string(dev));
      return RPK_ERR_ARG;
    }
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (stream) {
    int sdev = -1;
    err = cudaStreamGetDevice(stream, &sdev);
    if (err != cudaSuccess) return rpk::cuda_fail(err, "cudaStreamGetDevice");
    if (sdev != dev) {
      rpk::set_error("rpk_field_totals_noalloc: the stream belongs to device " +
                     std::to_string(sdev) + ", not the current device " + std::to_string(dev));
      return RPK_ERR_ARG;
    }
  }
  const int nchunks = (int)((npts + kChunk - 1) / kChunk);
  k_totals_partial<<<nchunks, kThreads, 0, stream>>>(rho, u, theta_T, theta_R, npts, delta,
                                                     scratch);
  err = cudaGetLastError();
  if (err != cudaSuccess) return rpk::cuda_fail(err, "k_totals_partial");
  k_totals_final<<<1, 1024, 0, stream>>>(scratch, nchunks, out);
  err = cudaGetLastError();
  if (err != cudaSuccess) return rpk::cuda_fail(err, "k_totals_final");
  return RPK_OK;
}
