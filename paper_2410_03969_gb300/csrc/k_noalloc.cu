// Allocation-free relative trace error of a caller-provided factor.
//
// rpchol_stats computes tr(A - F F^*) / tr(A) for a context's own factor,
// using per-block partial sums in a buffer the context allocated.  Some
// callers cannot allocate device memory at all: code embedded in a host
// runtime that reserves all device memory up front in its own pool or arena
// and forbids cudaMalloc outside it, or a latency-critical loop in which an
// allocation could block or fail.  rpchol_trace_error_noalloc serves them:
// the caller passes F and the output location, and the per-tile partial
// sums live in the file-scope device array below (512 KiB; every GPU that
// loads the library holds it until the process exits).
//
// Behaviour a caller must know:
//   - Every call looks up the current device's address of the array
//     (cudaGetSymbolAddress, with that device current).  The lookup
//     enqueues no work and is not cached, so a context that was torn down
//     and created again (cudaDeviceReset) is looked up afresh.  The first
//     call on a device loads the module there; make it before any stream
//     capture on that device.
//   - Every call shares the one array; calls whose kernels overlap on the
//     GPU race on it.  Serialise them (one stream, or events).
//   - Each call overwrites every partial it reads, so nothing needs to start
//     at zero; the array keeps the last call's contents.
//   - N above kNoAllocMaxRows is rejected with RPCHOL_EINVAL.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/rpchol.h"
#include "internal.h"

namespace rpchol {
namespace {

constexpr long long kNoAllocTileRows = 128;
constexpr long long kNoAllocMaxTiles = 65536;
constexpr long long kNoAllocMaxRows = kNoAllocTileRows * kNoAllocMaxTiles;  // 8,388,608

static __device__ __align__(256) double g_trace_partials[kNoAllocMaxTiles];

// One CTA per 128-row tile: part[tile] = sum over its rows of
// (1 - ||F(r, 0:rank)||^2) (phi(0) = 1 on the diagonal of A), fixed order.
template <typename TF>
__global__ void __launch_bounds__(256) k_trace_tiles(const TF* __restrict__ F, long long ldF,
                                                     long long N, long long rank, double* part) {
  __shared__ double ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * kNoAllocTileRows;
  double acc = 0.0;
  for (long long r = r0 + warp; r < r0 + kNoAllocTileRows && r < N; r += 8) {
    double sq = 0.0;
    for (long long m = lane; m < rank; m += 32) {
      const double f = (double)F[r * ldF + m];
      sq += f * f;
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    acc += 1.0 - sq;
  }
  if (lane == 0) ws[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_trace_tiles_final(const double* __restrict__ part,
                                                           long long ntiles, long long N,
                                                           double* out) {
  __shared__ double sh[256];
  double t = 0.0;
  for (long long i = threadIdx.x; i < ntiles; i += 256) t += part[i];
  sh[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < 256; ++i) s += sh[i];
    out[0] = s / (double)N;
  }
}



}  // namespace
}  // namespace rpchol

using namespace rpchol;

extern "C" rpchol_status rpchol_trace_error_noalloc(const void* F_dev, int32_t F_dtype, int64_t N,
                                                    int64_t ldF, int64_t rank, double* out_dev,
                                                    void* stream) {
  if (!F_dev || !out_dev || N < 1 || rank < 0 || ldF < rank || ldF < 1 ||
      (F_dtype != RPCHOL_DT_F32 && F_dtype != RPCHOL_DT_F64)) {
    set_last_error(
             "rpchol_trace_error_noalloc: invalid argument (N=%lld ldF=%lld rank=%lld dtype=%d)",
             (long long)N, (long long)ldF, (long long)rank, F_dtype);
    return RPCHOL_EINVAL;
  }
  if (N > kNoAllocMaxRows) {
    set_last_error(
             "rpchol_trace_error_noalloc: N=%lld exceeds the static scratch limit of %lld rows",
             (long long)N, kNoAllocMaxRows);
    return RPCHOL_EINVAL;
  }
  // the current device's address of the array: looked up on every call (no
  // cache to go stale across a context reset; the lookup enqueues nothing)
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_trace_partials);
  if (e != cudaSuccess || !p) {
    set_last_error("rpchol_trace_error_noalloc: cudaGetSymbolAddress: %s",
                   cudaGetErrorString(e));
    return RPCHOL_ECUDA;
  }
  double* part = (double*)p;
  const long long ntiles = (N + kNoAllocTileRows - 1) / kNoAllocTileRows;
  cudaStream_t s = (cudaStream_t)stream;
  if (F_dtype == RPCHOL_DT_F32)
    k_trace_tiles<float><<<(unsigned)ntiles, 256, 0, s>>>((const float*)F_dev, ldF, N, rank, part);
  else
    k_trace_tiles<double><<<(unsigned)ntiles, 256, 0, s>>>((const double*)F_dev, ldF, N, rank,
                                                           part);
  k_trace_tiles_final<<<1, 256, 0, s>>>(part, ntiles, N, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error( "rpchol_trace_error_noalloc: launch: %s",
             cudaGetErrorString(e));
    return RPCHOL_ECUDA;
  }
  return RPCHOL_OK;
}

