// CUDA-core column step of accelerated RPCholesky (Algorithm 2, step 3,
// arXiv 2410.03969): for every row r
//   G(r, :) = (A(r, S) - F(r, :) F(S, :)^*) L^{-*},   F(r, rank:rank+s) = G(r, :),
//   d_r <- max(d_r - sum_j G(r, j)^2, 0),
// plus the tile sums of d for the next round's sampler.  This is the parity
// mode: IEEE double throughout, kernel entries by direct differences.
//
// One CTA owns 128 rows (one sampler tile).  The s new columns are produced
// in blocks of 32 with a left-looking blocked forward substitution: block c
// needs R(:, c) - G(:, <c) L(c, <c)^*, which is one dense contraction of the
// row panel [F(r, 0:rank) | G(r, 0:32c)] (contiguous in F, because G is
// written to F as it is produced) with the gathered rows
// [F(S_j, 0:rank) | L(j, 0:32c)]; the 32 x 32 diagonal block of L is then
// applied by per-row forward substitution.
#include <cuda_runtime.h>

#include "internal.h"

namespace rpchol {

namespace {
constexpr int BM = 128;  // rows per CTA
constexpr int BN = 32;   // columns per block of G
constexpr int BK = 8;    // reduction chunk (static shared memory stays under 48 KB)
}  // namespace

// q(i, j) += sum over the kn staged coordinates of |a - b| (L1: kind 4, the
// l1-Laplace) or (a - b)^2, coordinates in increasing order
template <bool L1, typename TR>
__device__ __forceinline__ void dist_tile(TR (&q)[4][4], const TR (*As)[BM + 1],
                                          const TR (*Bs)[BN + 1], int ty, int tx, int kn) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    if (kk < kn) {
      TR a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const TR t = a[i] - b[j];
          q[i][j] += L1 ? (t < (TR)0 ? -t : t) : t * t;
        }
    }
  }
}

// TR = double: the FP64 parity mode.  TR = float: the CUDA-core FP32 path of
// mixed mode (F in FP32, FP32 FMA with FP32 accumulation; L is rounded to
// FP32; d stays FP64 and the squared row norms are accumulated in FP64).
template <typename TR>
__global__ void __launch_bounds__(256) k_colstep_simt(
    const DevState* st, const float* __restrict__ X, int xld, int d, int kind, double inv_sigma,
    TR* F, long long ldF, const TR* __restrict__ Bext, long long ldB,
    const int* __restrict__ Sacc, const double* __restrict__ L, int ldL, double* dvec,
    double* tile_sums, long long N) {
  __shared__ TR As[BK][BM + 1];
  __shared__ TR Bs[BK][BN + 1];
  __shared__ TR Rb[BM][BN + 1];
  __shared__ double red[8];
  if (st->done) return;
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const long long row0 = (long long)blockIdx.x * BM;
  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;  // 32 x 8 threads, 4 x 4 outputs each
  double rsq = 0.0;                       // thread tid < 128 owns row row0 + tid

  for (int c0 = 0; c0 < s; c0 += BN) {
    const long long Kext = rank + c0;
    TR acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (TR)0;
    for (long long m0 = 0; m0 < Kext; m0 += BK) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q;
        const int r = e >> 3, kk = e & 7;
        const long long gr = row0 + r, gm = m0 + kk;
        As[kk][r] = (gr < N && gm < Kext) ? F[gr * ldF + gm] : (TR)0;
      }
      {
        const int j = tid >> 3, kk = tid & 7;
        const long long gm = m0 + kk;
        Bs[kk][j] = (c0 + j < s && gm < Kext) ? Bext[(long long)(c0 + j) * ldB + gm] : (TR)0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        TR a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
      }
      __syncthreads();
    }
    // distances q(x_r, x_{S_c}) = sum_l dist_term(x_rl - x_{S_c} l), tiled like
    // the contraction above (X rows and X(S_c) staged BK coordinates at a
    // time); every q accumulates over l in increasing order
    TR q[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) q[i][j] = (TR)0;
    for (int l0 = 0; l0 < d; l0 += BK) {
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const int e = tid + 256 * qq;
        const int r = e >> 3, kk = e & 7;
        const long long gr = row0 + r;
        As[kk][r] = (gr < N && l0 + kk < d) ? (TR)X[gr * xld + l0 + kk] : (TR)0;
      }
      {
        const int j = tid >> 3, kk = tid & 7;
        Bs[kk][j] = (c0 + j < s && l0 + kk < d) ? (TR)X[(long long)Sacc[c0 + j] * xld + l0 + kk]
                                                : (TR)0;
      }
      __syncthreads();
      const int kn = d - l0 < BK ? d - l0 : BK;
      if (kind == 4) dist_tile<true>(q, As, Bs, ty, tx, kn);
      else dist_tile<false>(q, As, Bs, ty, tx, kn);
      __syncthreads();
    }
    // R'(r, c) = kappa(x_r, x_{S_c}) - acc
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long gr = row0 + ty * 4 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + tx * 4 + j;
        TR v = (TR)0;
        if (gr < N && c < s) {
          const int p = Sacc[c];
          const TR kv = (long long)p != gr ? phi_r2<TR>(kind, (TR)inv_sigma, q[i][j]) : (TR)1;
          v = kv - acc[i][j];
        }
        Rb[ty * 4 + i][tx * 4 + j] = v;
      }
    }
    __syncthreads();
    // forward substitution with the diagonal block of L, one row per thread
    const int jmax = s - c0 < BN ? s - c0 : BN;
    if (tid < BM) {
      for (int j = 0; j < jmax; ++j) {
        const double* Lrow = L + (long long)(c0 + j) * ldL + c0;
        TR v = Rb[tid][j];
        for (int l = 0; l < j; ++l) v -= Rb[tid][l] * (TR)Lrow[l];
        v = v / (TR)Lrow[j];
        Rb[tid][j] = v;
        rsq += (double)v * (double)v;
      }
    }
    __syncthreads();
    for (int e = tid; e < BM * BN; e += 256) {
      const int r = e >> 5, j = e & 31;
      const long long gr = row0 + r;
      if (gr < N && j < jmax) F[gr * ldF + rank + c0 + j] = Rb[r][j];
    }
    __syncthreads();  // G block visible to the CTA before the next block reads it
  }
  double dn = 0.0;
  if (tid < BM) {
    const long long gr = row0 + tid;
    if (gr < N) {
      const double v = dvec[gr] - rsq;
      dn = v > d_floor<TR>() ? v : 0.0;
      dvec[gr] = dn;
    }
  }
  const double t = block_sum_fixed(dn, red);
  if (tid == 0) tile_sums[blockIdx.x] = t;
}

cudaError_t launch_colstep_f64(const DevBuffers& b, int T, cudaStream_t s) {
  (void)T;
  const long long blocks = (b.N + BM - 1) / BM;
  k_colstep_simt<double><<<(unsigned)blocks, 256, 0, s>>>(
      b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma, (double*)b.F, b.ldF, b.Bext, b.ldB, b.Sacc,
      b.L, b.Tmax, b.dvec, b.tile_sums, b.N);
  return cudaGetLastError();
}

cudaError_t launch_colstep_f32_simt(const DevBuffers& b, int T, cudaStream_t s) {
  (void)T;
  const long long blocks = (b.N + BM - 1) / BM;
  k_colstep_simt<float><<<(unsigned)blocks, 256, 0, s>>>(
      b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma, (float*)b.F, b.ldF, (const float*)b.Bext,
      b.ldB, b.Sacc, b.L, b.Tmax, b.dvec, b.tile_sums, b.N);
  return cudaGetLastError();
}

}  // namespace rpchol
