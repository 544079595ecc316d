// Simple RPCholesky (Algorithm 6 of arXiv 2410.03969, appendix), the GPU
// baseline.  One step i:
//   s ~ d / sum(d)                              (the shared sampler, T = 1)
//   g = A(:, s) - F(:, 0:i) F(s, 0:i)^*          (k_plain_col: one GEMV over F)
//   F(:, i) = g / sqrt(g_s);  d <- max(d - F(:, i)^2, 0)   (k_plain_finish)
// g_s is taken from the freshly formed column (the literal Algorithm 6);
// if it is not positive (rounding only) the step adds no column and sets
// d_s = 0.  The GEMV streams F(:, 0:i) once per step: HBM-bound.
#include <cuda_runtime.h>

#include "internal.h"

namespace rpchol {

// Accumulator type of the GEMV: double for the FP64 factor, float for the
// FP32 factor of mixed mode.
template <typename TF>
struct Acc;
template <>
struct Acc<double> {
  using T = double;
};
template <>
struct Acc<float> {
  using T = float;
};

// One warp per row: g_r = kappa(x_r, x_s) - F(r, 0:i) . F(s, 0:i).  In mixed
// mode (FP32 factor) the row of F streams as float4 and the distance and the
// kernel map are FP32, as in the accelerated column step (FP64 is slow on
// this GPU); FP64 mode keeps every step in FP64.
template <typename TF>
__global__ void __launch_bounds__(256) k_plain_col(DevState* st, const float* __restrict__ X,
                                                   int xld, int d, int kind, double inv_sigma,
                                                   TF* F, long long ldF,
                                                   const int* __restrict__ prop, long long N) {
  using A = typename Acc<TF>::T;
  if (st->done) return;
  const long long i = st->rank;
  const int s = prop[0];
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= N) return;
  const TF* fr = F + r * ldF;
  const TF* fs = F + (long long)s * ldF;
  A acc = 0;
  long long m0 = 0;
  if constexpr (sizeof(TF) == 4) {
    // rows start on 128-byte boundaries (ldF is a multiple of 32)
    const float4* fr4 = (const float4*)fr;
    const float4* fs4 = (const float4*)fs;
    const long long i4 = i >> 2;
    for (long long m = lane; m < i4; m += 32) {
      const float4 a = fr4[m], b = fs4[m];
      acc = fmaf(a.x, b.x, acc);
      acc = fmaf(a.y, b.y, acc);
      acc = fmaf(a.z, b.z, acc);
      acc = fmaf(a.w, b.w, acc);
    }
    m0 = i4 << 2;
  }
  for (long long m = m0 + lane; m < i; m += 32) acc += (A)fr[m] * (A)fs[m];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  A r2 = 0;
  if (r != s) {
    const float* xa = X + r * xld;
    const float* xb = X + (long long)s * xld;
    for (int l = lane; l < d; l += 32) {
      const A t = (A)xa[l] - (A)xb[l];
      r2 += dist_term(kind, t);
    }
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
  }
  if (lane == 0) {
    A kv = 1;
    if (r != s) kv = phi_r2<A>(kind, (A)inv_sigma, r2);
    const A g = kv - acc;
    F[r * ldF + i] = (TF)g;
    if (r == s) st->gs = (double)g;
  }
}

// F(:, i) = g / sqrt(g_s), d update, tile sums (one CTA = one sampler tile).
template <typename TF>
__global__ void __launch_bounds__(kTileRows) k_plain_finish(DevState* st, TF* F, long long ldF,
                                                            const int* __restrict__ prop,
                                                            double* dvec, double* tile_sums,
                                                            long long N) {
  __shared__ double red[kTileRows / 32];
  if (st->done) return;
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
      const double f = (double)F[r * ldF + i] / pv;
      F[r * ldF + i] = (TF)f;
      const double ff = (double)(TF)f;
      const double v = dv - ff * ff;
      dv = v > 0.0 ? v : 0.0;
    } else {
      F[r * ldF + i] = (TF)0;
      if (r == s) dv = 0.0;
    }
    dvec[r] = dv;
    dn = dv;
  }
  const double t = block_sum_fixed(dn, red);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
}

__global__ void k_plain_end(DevState* st, const int* __restrict__ prop, long long* piv,
                            cudaGraphConditionalHandle cond, int use_cond, long long N, int d,
                            int bF) {
  if (!st->done) {
    const double n = (double)N, i = (double)st->rank;
    st->col_bytes += n * (i * bF + bF + 4.0 * d + 16.0);
    st->col_flops += 2.0 * n * i + 3.0 * n * d;
    if (st->gs > 0.0) {
      piv[st->rank] = prop[0];
      st->rank += 1;
    }
    st->round += 1;
    st->proposals += 1;
    if (st->rank >= st->k) {
      st->done = 1;
    } else if (st->round >= st->max_rounds) {
      st->done = 1;
      st->status |= kStRoundLimit;
    }
  }
  if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

cudaError_t launch_plain_col(const DevBuffers& b, cudaStream_t s) {
  const unsigned gcol = (unsigned)((b.N + 7) / 8);
  if (b.mixed)
    k_plain_col<float><<<gcol, 256, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                                            (float*)b.F, b.ldF, b.prop, b.N);
  else
    k_plain_col<double><<<gcol, 256, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                                             (double*)b.F, b.ldF, b.prop, b.N);
  return cudaGetLastError();
}

cudaError_t launch_plain_finish(const DevBuffers& b, cudaStream_t s) {
  const unsigned gfin = (unsigned)((b.N + kTileRows - 1) / kTileRows);
  if (b.mixed)
    k_plain_finish<float><<<gfin, kTileRows, 0, s>>>(b.st, (float*)b.F, b.ldF, b.prop, b.dvec,
                                                     b.tile_sums, b.N);
  else
    k_plain_finish<double><<<gfin, kTileRows, 0, s>>>(b.st, (double*)b.F, b.ldF, b.prop,
                                                      b.dvec, b.tile_sums, b.N);
  return cudaGetLastError();
}

cudaError_t launch_plain_end(const DevBuffers& b, unsigned long long cond, int use_cond,
                             cudaStream_t s) {
  k_plain_end<<<1, 1, 0, s>>>(b.st, b.prop, b.piv, (cudaGraphConditionalHandle)cond, use_cond,
                              b.N, b.d, b.mixed ? 4 : 8);
  return cudaGetLastError();
}

}  // namespace rpchol
