// Simple RPCholesky (Algorithm 6 of arXiv 2410.03969, appendix), the GPU
// baseline.  One step i, three kernels:
//   s ~ d / sum(d), and g_s = A(s,s) - ||F(s, 0:i)||^2     (the shared sampler,
//                                                          T = 1, k_propose)
//   g = A(:, s) - F(:, 0:i) F(s, 0:i)^*                    (k_plain_step)
//   F(:, i) = g / sqrt(g_s);  d <- max(d - F(:, i)^2, 0);
//   tile sums of d;  step bookkeeping                      (k_plain_finish)
// g_s is the pivot's entry of the freshly formed column (the literal
// Algorithm 6: the pivot row's product is the sampler's, the other rows'
// are formed here with the same arithmetic); if it is not positive
// (rounding only) the step adds no column and sets d_s = 0.  The GEMV
// streams F(:, 0:i) once per step: HBM-bound (FP64-ALU-bound in FP64 mode).
#include <cuda_runtime.h>

#include "internal.h"

namespace rpchol {

namespace {
constexpr int kPlainThreads = 256;  // 8 warps, one row each
constexpr int kPlainRows = 8;       // rows per CTA; 16 CTAs per sampler tile
}  // namespace

// One warp per row (8 rows per CTA, many CTAs resident per SM, each warp one
// 16-byte load stream over its row), F(s, 0:i) read through L1 (every warp
// reads it); lane 0 writes g to F(r, i).  Nothing here runs in FP64 in mixed
// mode: this GPU's FP64 instructions are slow, and a one-lane FP64 sequence
// per row costs as much as a full warp's.  In mixed mode (FP32 factor) the
// products accumulate in FP32 and the distance and kernel map are FP32, as
// in the accelerated column step; FP64 mode keeps every step in FP64.
template <typename TF>
__global__ void __launch_bounds__(kPlainThreads) k_plain_step(
    const DevState* st, const float* __restrict__ X, int xld, int d, int kind, double inv_sigma,
    TF* F, long long ldF, const int* __restrict__ prop, long long N) {
  using A = typename FVec<TF>::A;
  if (st->done) return;
  const long long i = st->rank;
  const int s = prop[0];
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * kPlainRows + (threadIdx.x >> 5);
  if (r >= N || r == s) return;  // the pivot's entry is the sampler's g_s
  const TF* rows[1] = {F + r * ldF};
  A acc[1];
  warp_rows_dot<TF, 1>(rows, F + (long long)s * ldF, i, lane, acc);
  A r2 = 0;
  const float* xa = X + r * xld;
  const float* xb = X + (long long)s * xld;
  for (int l = lane; l < d; l += 32) {
    const A t = (A)xa[l] - (A)xb[l];
    r2 += dist_term(kind, t);
  }
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if (lane == 0) F[r * ldF + i] = (TF)(phi_r2<A>(kind, (A)inv_sigma, r2) - acc[0]);
}

// One thread per row and one CTA per 128-row sampler tile: F(r, i) = g_r /
// sqrt(g_s) (g_s at the pivot's own entry), d <- max(d - F(r, i)^2, 0), the
// tile sum of d (fixed-order block sum); the last CTA to finish keeps the
// step's books and sets the graph's while-condition.
template <typename TF>
__global__ void __launch_bounds__(kTileRows) k_plain_finish(
    DevState* st, TF* F, long long ldF, const int* __restrict__ prop, long long* piv,
    double* dvec, double* tile_sums, long long N, int d, unsigned* ccnt,
    cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double red[kTileRows / 32];
  if (st->done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const long long i = st->rank;
  const double gs = st->gs;
  const int s = prop[0];
  const bool ok = gs > 0.0;
  const double pv = ok ? sqrt(gs) : 1.0;
  const long long r = (long long)blockIdx.x * kTileRows + threadIdx.x;
  double dn = 0.0;
  if (r < N) {
    double dv = dvec[r];
    if (ok) {
      const double g = r == s ? gs : (double)F[r * ldF + i];
      const TF f = (TF)(g / pv);
      F[r * ldF + i] = f;
      const double ff = (double)f;
      const double v = dv - ff * ff;
      dv = v > d_floor<TF>() ? v : 0.0;
    } else {
      F[r * ldF + i] = (TF)0;
      if (r == s) dv = 0.0;
    }
    dvec[r] = dv;
    dn = dv;
  }
  const double t = block_sum_fixed(dn, red);
  if (threadIdx.x == 0) {
    tile_sums[blockIdx.x] = t;
    __threadfence();
    if (atomicAdd(ccnt, 1u) == gridDim.x - 1) {
      __threadfence();
      const double n = (double)N, ic = (double)i;
      const int bF = (int)sizeof(TF);
      st->col_bytes += n * (ic * bF + bF + 4.0 * d + 16.0);
      st->col_flops += 2.0 * n * ic + 3.0 * n * d;
      if (ok) {
        piv[i] = s;
        st->rank = i + 1;
      }
      st->round += 1;
      st->proposals += 1;
      if (st->rank >= st->k) {
        st->done = 1;
      } else if (st->round >= st->max_rounds) {
        st->done = 1;
        st->status |= kStRoundLimit;
      }
      if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
      *ccnt = 0u;
    }
  }
}

cudaError_t launch_plain_step(const DevBuffers& b, cudaStream_t s) {
  const unsigned grid = (unsigned)((b.N + kPlainRows - 1) / kPlainRows);
  if (b.mixed)
    k_plain_step<float><<<grid, kPlainThreads, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                                                       (float*)b.F, b.ldF, b.prop, b.N);
  else
    k_plain_step<double><<<grid, kPlainThreads, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind,
                                                        1.0 / b.sigma, (double*)b.F, b.ldF,
                                                        b.prop, b.N);
  return cudaGetLastError();
}

cudaError_t launch_plain_tiles(const DevBuffers& b, unsigned long long cond, int use_cond,
                               cudaStream_t s) {
  const unsigned gt = (unsigned)((b.N + kTileRows - 1) / kTileRows);
  if (b.mixed)
    k_plain_finish<float><<<gt, kTileRows, 0, s>>>(b.st, (float*)b.F, b.ldF, b.prop, b.piv,
                                                   b.dvec, b.tile_sums, b.N, b.d, b.ccnt,
                                                   (cudaGraphConditionalHandle)cond, use_cond);
  else
    k_plain_finish<double><<<gt, kTileRows, 0, s>>>(b.st, (double*)b.F, b.ldF, b.prop, b.piv,
                                                    b.dvec, b.tile_sums, b.N, b.d, b.ccnt,
                                                    (cudaGraphConditionalHandle)cond, use_cond);
  return cudaGetLastError();
}

}  // namespace rpchol
