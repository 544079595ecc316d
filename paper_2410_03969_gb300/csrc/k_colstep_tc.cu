// Stand-alone launch of the tensor-core column step of accelerated
// RPCholesky in mixed precision (Algorithm 2, step 3, arXiv 2410.03969):
// one persistent CTA per SM runs colstep_body (colstep_body.cuh) over the
// round's 128-row tiles, in clusters of kColstepMc CTAs that share each B
// operand.
#include <cuda.h>
#include <cuda_runtime.h>

#include "colstep_body.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

#ifndef RPCHOL_COLSTEP_MC
#define RPCHOL_COLSTEP_MC 2
#endif
// CTAs of a cluster sharing each B operand (bulk-copy multicast)
constexpr int kColstepMc = RPCHOL_COLSTEP_MC;

__global__ void __launch_bounds__(kTcThreads, 1)
    k_colstep_tc(const __grid_constant__ CUtensorMap tmFs, const __grid_constant__ CUtensorMap tmXh,
                 const __grid_constant__ CUtensorMap tmXl,
                 TcArgs a, int mc) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // the TMEM address in the last 16 bytes of the allocation, beyond anything
  // the body's layout reaches (its total, alignment slack included, is at
  // most kSmemMax - kTailBytes)
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
  colstep_body(&tmFs, &tmXh, &tmXl, a, sm, tbase, (int)blockIdx.x, (int)gridDim.x, mc);
  if (work && (threadIdx.x >> 5) == 1) tc::tmem_dealloc(tbase, 512);
}

cudaError_t launch_colstep_tc(const TcMaps& m, const DevBuffers& b, unsigned long long cond,
                              int use_cond, cudaStream_t s) {
  static bool attr_set = false;
  static int max_clusters = 0;  // clusters of kColstepMc resident at once
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_colstep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemMax);
    if (e != cudaSuccess) return e;
    if (kColstepMc > 1) {
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = kColstepMc;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(m.num_sms / kColstepMc * kColstepMc));
      cfg.blockDim = dim3(kTcThreads);
      cfg.dynamicSmemBytes = kSmemMax;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      e = cudaOccupancyMaxActiveClusters(&max_clusters, (void*)k_colstep_tc, &cfg);
      if (e != cudaSuccess) return e;
    }
    attr_set = true;
  }
  const TcArgs a = make_tc_args(m, b, cond, use_cond);
  const long long ntiles = (b.N + kBM - 1) / kBM;
  int grid = (int)(ntiles < m.num_sms ? ntiles : m.num_sms);
  // clusters only where every CTA of each has a tile and all are resident at once
  int mc = kColstepMc;
  if (mc > 1) {
    int g = grid / mc * mc;
    if (g > max_clusters * mc) g = max_clusters * mc;
    if (g >= mc) grid = g;
    else mc = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at;
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kTcThreads);
  // the shared-memory layout depends on s, which only the device knows: the
  // launch reserves the maximum
  cfg.dynamicSmemBytes = kSmemMax;
  cfg.stream = s;
  if (mc > 1) {
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)mc;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, k_colstep_tc, m.Fs, m.Xh, m.Xl, a, mc);
}

}  // namespace rpchol
