// Per-round operand preparation for the tensor-core column step (mixed
// mode), Algorithm 2 step 3 of arXiv 2410.03969:
//   - rows j < s of the B operands: F(S_j, 0:rank) and x_{S_j}, each split
//     into TF32 head and tail planes; rows [s, 64 * ceil(s_pad / 64)) and the
//     columns [rank, 32 * ceil(rank / 32)) are zero so that padded MMA
//     columns and padded K chunks contribute nothing;
//   - ||x_{S_j}||^2;
//   - the blocked-substitution operand W built from the round's compact
//     Cholesky factor L in FP64 and rounded once to FP32 (k_wblk below).
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

// Blocked forward substitution operand for G L^* = R.  With the columns in
// blocks of 16 (block b covers columns j0 = 16 b .. j0 + 15) and D_b the
// 16 x 16 diagonal block of L, block b of G is
//   G_b = D_b^{-1} (R_b - G_{<j0} L(b, <j0)^*)
//       = sum_{l < j0} G(:, l) W_b(l, :) + sum_{m < 16} R(:, j0 + m) W_b(j0 + m, :)
// with W_b(l, jj) = -(D_b^{-1} L(b, <j0))(jj, l) for l < j0 and
// W_b(j0 + m, jj) = D_b^{-1}(jj, m).  All of it is formed here in FP64 from
// the FP64 L of Algorithm 1 and rounded once to FP32.  Block b occupies
// (j0 + 16) x 16 floats at offset 256 b (b + 1) / 2, row l contiguous.
// Rows and columns of L beyond s are taken as the identity, so padded
// columns of G are copies of the (zero) padded columns of R.
__global__ void __launch_bounds__(256) k_wblk(const DevState* st, const double* __restrict__ L,
                                              int ldL, float* W) {
  __shared__ double Dinv[16][17];
  __shared__ double Lb[16][kTMax];  // rows j0..j0+15 of L, columns < j0
  if (st->done) return;
  const int s = st->s;
  const int b = blockIdx.x;
  const int j0 = 16 * b;
  if (j0 >= s) return;
  const int t = threadIdx.x;
  auto Lat = [&](int r, int c) -> double {  // L with identity padding beyond s
    if (r >= s || c >= s) return r == c ? 1.0 : 0.0;
    return c <= r ? L[(long long)r * ldL + c] : 0.0;
  };
  for (int e = t; e < 16 * j0; e += blockDim.x) Lb[e / j0][e % j0] = Lat(j0 + e / j0, e % j0);
  // D_b^{-1} column m by forward substitution (16 threads)
  if (t < 16) {
    const int m = t;
    for (int r = 0; r < 16; ++r) {
      double v = (r == m) ? 1.0 : 0.0;
      for (int c = m; c < r; ++c) v -= Lat(j0 + r, j0 + c) * Dinv[c][m];
      Dinv[r][m] = r >= m ? v / Lat(j0 + r, j0 + r) : 0.0;
    }
  }
  __syncthreads();
  float* Wb = W + 256 * (long long)b * (b + 1) / 2;
  for (int e = t; e < 16 * j0; e += blockDim.x) {  // W_b(l, jj), l < j0
    const int l = e >> 4, jj = e & 15;
    double acc = 0.0;
    for (int m = 0; m <= jj; ++m) acc += Dinv[jj][m] * Lb[m][l];
    Wb[(long long)l * 16 + jj] = (float)(-acc);
  }
  for (int e = t; e < 256; e += blockDim.x) {  // W_b(j0 + m, jj) = D_b^{-1}(jj, m)
    const int m = e >> 4, jj = e & 15;
    Wb[(long long)(j0 + m) * 16 + jj] = (float)Dinv[jj][m];
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
  k_wblk<<<kTMax / 16, 256, 0, s>>>(b.st, b.L, b.Tmax, m.Linv32);
  return cudaGetLastError();
}

cudaError_t launch_split_x(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  const long long n = b.N * (long long)b.xld;
  k_split_x<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b.X, n, m.Xhp, m.Xlp);
  return cudaGetLastError();
}

}  // namespace rpchol
