// Stand-alone launch of the tensor-core column step of accelerated
// RPCholesky in mixed precision (Algorithm 2, step 3, arXiv 2410.03969):
// one persistent CTA per SM runs colstep_body (colstep_body.cuh) over the
// round's 128-row tiles.
#include <cuda.h>
#include <cuda_runtime.h>

#include "colstep_body.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

__global__ void __launch_bounds__(kTcThreads, 1)
    k_colstep_tc(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmXh,
                 const __grid_constant__ CUtensorMap tmXl, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // the TMEM address in the last 16 bytes of the allocation, beyond anything
  // the body's layout reaches (its total, alignment slack included, is at
  // most kSmemMax)
  uint32_t* tptr = (uint32_t*)(smem_raw + kSmemMax - 16);
  const DevState* st = a.st;
  const bool work = !(st->done || st->s == 0);
  if (work && (threadIdx.x >> 5) == 1) {
    tc::tmem_alloc(tptr, 512);
    tc::tmem_relinquish();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = work ? *tptr : 0u;
  colstep_body(&tmF, &tmXh, &tmXl, a, sm, tbase, (int)blockIdx.x, (int)gridDim.x);
  if (work && (threadIdx.x >> 5) == 1) tc::tmem_dealloc(tbase, 512);
}

cudaError_t launch_colstep_tc(const TcMaps& m, const DevBuffers& b, unsigned long long cond,
                              int use_cond, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_colstep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemMax);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const TcArgs a = make_tc_args(m, b, cond, use_cond);
  const long long ntiles = (b.N + kBM - 1) / kBM;
  const unsigned grid = (unsigned)(ntiles < m.num_sms ? ntiles : m.num_sms);
  // the shared-memory layout depends on s, which only the device knows: the
  // launch reserves the maximum
  k_colstep_tc<<<grid, kTcThreads, kSmemMax, s>>>(m.F, m.Xh, m.Xl, a);
  return cudaGetLastError();
}

}  // namespace rpchol
