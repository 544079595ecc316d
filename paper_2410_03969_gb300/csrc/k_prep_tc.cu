// Per-round operand preparation for the tensor-core column step (mixed
// mode), Algorithm 2 step 3 of arXiv 2410.03969:
//   - rows j < s of the B operands: F(S_j, 0:rank) and x_{S_j}, each split
//     into TF32 head and tail planes; rows [s, 64 * ceil(s_pad / 64)) and the
//     columns [rank, 32 * ceil(rank / 32)) are zero so that padded MMA
//     columns and padded K chunks contribute nothing;
//   - ||x_{S_j}||^2;
//   - L^{-1} of the round's compact Cholesky factor, by forward substitution
//     in FP64 (one column per CTA), rounded once to FP32.
// Also the one-time split of X into head and tail planes.
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

__global__ void __launch_bounds__(256) k_prep_tc(const DevState* st, const float* __restrict__ F,
                                                 long long ldF, const float* __restrict__ X,
                                                 int xld, const float* __restrict__ nrm,
                                                 const int* __restrict__ Sacc, float* FSh,
                                                 float* FSl, float* XSh, float* XSl, float* nrmS) {
  if (st->done) return;
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const long long kpad = (rank + 31) & ~31ll;
  const int s_pad = (s + 15) & ~15;
  const int rows = (s_pad + 63) & ~63;
  const int j = blockIdx.x;
  if (j >= rows) return;
  float* fh = FSh + (long long)j * ldF;
  float* fl = FSl + (long long)j * ldF;
  float* xh = XSh + (long long)j * xld;
  float* xl = XSl + (long long)j * xld;
  if (j < s) {
    const int p = Sacc[j];
    const float* src = F + (long long)p * ldF;
    for (long long m = threadIdx.x; m < kpad; m += blockDim.x) {
      const float v = m < rank ? src[m] : 0.f;
      const float h = tc::tf32_head(v);
      fh[m] = h;
      fl[m] = v - h;
    }
    const float* xs = X + (long long)p * xld;
    for (int l = threadIdx.x; l < xld; l += blockDim.x) {
      const float v = xs[l];
      const float h = tc::tf32_head(v);
      xh[l] = h;
      xl[l] = v - h;
    }
    if (threadIdx.x == 0) nrmS[j] = nrm[p];
  } else {
    for (long long m = threadIdx.x; m < kpad; m += blockDim.x) {
      fh[m] = 0.f;
      fl[m] = 0.f;
    }
    for (int l = threadIdx.x; l < xld; l += blockDim.x) {
      xh[l] = 0.f;
      xl[l] = 0.f;
    }
    if (threadIdx.x == 0) nrmS[j] = 0.f;
  }
}

// Column c of L^{-1}: solve L x = e_c (L lower triangular, s x s, FP64).
__global__ void __launch_bounds__(32) k_linv(const DevState* st, const double* __restrict__ L,
                                             int ldL, float* Linv32) {
  __shared__ double x[kTMax];
  if (st->done) return;
  const int s = st->s;
  const int c = blockIdx.x;
  if (c >= s) return;
  const int lane = threadIdx.x;
  for (int j = lane; j < c; j += 32) Linv32[(long long)j * 256 + c] = 0.f;
  if (lane == 0) x[c] = 1.0 / L[(long long)c * ldL + c];
  __syncwarp();
  if (lane == 0) Linv32[(long long)c * 256 + c] = (float)x[c];
  for (int j = c + 1; j < s; ++j) {
    const double* Lr = L + (long long)j * ldL;
    double acc = 0.0;
    for (int l = c + lane; l < j; l += 32) acc += Lr[l] * x[l];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double v = -acc / Lr[j];
      x[j] = v;
      Linv32[(long long)j * 256 + c] = (float)v;
    }
    __syncwarp();
  }
}

__global__ void k_split_x(const float* __restrict__ X, long long n, float* Xh, float* Xl) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = X[i];
  const float h = tc::tf32_head(v);
  Xh[i] = h;
  Xl[i] = v - h;
}

cudaError_t launch_prep_tc(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  k_prep_tc<<<kTMax, 256, 0, s>>>(b.st, (const float*)b.F, b.ldF, b.X, b.xld, b.nrm, b.Sacc,
                                  m.FShp, m.FSlp, m.XShp, m.XSlp, m.nrmS);
  k_linv<<<kTMax, 32, 0, s>>>(b.st, b.L, b.Tmax, m.Linv32);
  return cudaGetLastError();
}

cudaError_t launch_split_x(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  const long long n = b.N * (long long)b.xld;
  k_split_x<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b.X, n, m.Xhp, m.Xlp);
  return cudaGetLastError();
}

}  // namespace rpchol
