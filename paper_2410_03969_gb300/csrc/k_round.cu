// Round kernels of accelerated RPCholesky (Algorithm 2, arXiv 2410.03969):
// reset, proposal sampler (step 1), residual submatrix H and
// RejectionSampleSubmatrix (step 2, Algorithm 1), round control, and the
// trace-error reduction.
#include <cuda_runtime.h>

#include "internal.h"

namespace rpchol {

// ------------------------------------------------------------------ reset
// d = diag A = phi(0) = 1 for every kernel here; tile sums are the tile row
// counts; state initialised for a new run.
__global__ void k_reset(DevState* st, double* dvec, double* tile_sums, long long N,
                        long long ntiles, long long k, int T, unsigned long long seed,
                        unsigned inst, int plain, long long max_rounds) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = i; r < N; r += stride) dvec[r] = 1.0;
  for (long long t = i; t < ntiles; t += stride) {
    const long long lo = t * kTileRows;
    const long long hi = lo + kTileRows < N ? lo + kTileRows : N;
    tile_sums[t] = (double)(hi - lo);
  }
  if (i == 0) {
    st->rank = 0;
    st->round = 0;
    st->k = k;
    st->max_rounds = max_rounds;
    st->proposals = 0;
    st->T = T;
    st->s = 0;
    st->done = 0;
    st->status = 0;
    st->plain = plain;
    st->seed = seed;
    st->instance = inst;
    st->W = 0.0;
    st->gs = 0.0;
    st->piv = -1;
    st->col_bytes = 0.0;
    st->col_flops = 0.0;
  }
}

cudaError_t launch_reset(const DevBuffers& b, long long k, int T, unsigned long long seed,
                         unsigned inst, int plain, long long max_rounds, cudaStream_t s) {
  long long blocks = (b.N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_reset<<<(unsigned)blocks, 256, 0, s>>>(b.st, b.dvec, b.tile_sums, b.N, b.ntiles, k, T, seed,
                                           inst, plain, max_rounds);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ sampler
__device__ __forceinline__ double warp_incl_scan(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Step 1 of Algorithm 2: T iid draws with P{j} = d_j / sum(d).  One CTA of
// 1024 threads.  The tile sums (written by the kernel that last updated d)
// are scanned into tile_prefix; each draw binary-searches the tile prefix
// and then scans its tile with a warp prefix sum: the pivot is the first j
// whose running sum exceeds U * W (the proposal map of the oracle, summed
// in tile order instead of index order).
__global__ void __launch_bounds__(1024) k_propose(DevState* st, const double* __restrict__ dvec,
                                                  const double* __restrict__ tile_sums,
                                                  double* tile_prefix, long long ntiles,
                                                  long long N, int* prop, double* uprop,
                                                  double* uacc, int use_smem) {
  extern __shared__ double pref_smem[];
  __shared__ double wsum[32];
  __shared__ double carry_sh;
  if (st->done) return;
  const int T = st->T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* P = use_smem ? pref_smem : tile_prefix;  // inclusive prefix of the tile sums
  double run = 0.0;
  for (long long base = 0; base < ntiles; base += 1024) {
    const long long t = base + tid;
    const double v = t < ntiles ? tile_sums[t] : 0.0;
    double incl = warp_incl_scan(v);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      double w = wsum[lane];
      const double wi = warp_incl_scan(w);
      wsum[lane] = wi - w;  // exclusive prefix of warp totals
      if (lane == 31) carry_sh = wi;
    }
    __syncthreads();
    incl += wsum[warp];
    if (t < ntiles) P[t] = run + incl;
    const double chunk = carry_sh;
    __syncthreads();
    run += chunk;
  }
  const double W = run;
  if (tid == 0) {
    st->W = W;
    if (!(W > 0.0)) st->done = 1;
  }
  if (!(W > 0.0)) return;
  __syncthreads();  // prefix complete and visible to the CTA

  const unsigned long long seed = st->seed;
  const unsigned round = (unsigned)st->round;
  const unsigned inst = st->instance;
  for (int j = warp; j < T; j += 32) {
    double up = 0.0, ua = 0.0;
    if (lane == 0) uniforms(seed, (unsigned)j, round, inst, &up, &ua);
    up = __shfl_sync(0xffffffffu, up, 0);
    ua = __shfl_sync(0xffffffffu, ua, 0);
    const double target = up * W;
    // first tile whose inclusive prefix exceeds the target
    long long lo = 0, hi = ntiles;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (P[mid] > target) hi = mid;
      else lo = mid + 1;
    }
    long long t = lo;
    bool fallback = false;
    if (t >= ntiles) {  // rounding left no tile: the last tile with weight
      fallback = true;
      t = ntiles - 1;
      while (t > 0 && !(tile_sums[t] > 0.0)) --t;
    }
    const long long r0 = t * kTileRows;
    const long long r1 = r0 + kTileRows < N ? r0 + kTileRows : N;
    double running = t > 0 ? P[t - 1] : 0.0;
    long long found = -1, last_pos = -1;
    for (long long c = r0; c < r1; c += 32) {
      const long long r = c + lane;
      const double v = r < r1 ? dvec[r] : 0.0;
      const double incl = warp_incl_scan(v);
      const unsigned pos = __ballot_sync(0xffffffffu, v > 0.0);
      if (pos) last_pos = c + 31 - __clz(pos);
      if (!fallback) {
        const unsigned hit = __ballot_sync(0xffffffffu, v > 0.0 && running + incl > target);
        if (hit) {
          found = c + __ffs(hit) - 1;
          break;
        }
      }
      running += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (found < 0) found = last_pos;  // rounding: the last positive weight in the tile
    if (found < 0) found = r0;         // unreachable when W > 0
    if (lane == 0) {
      prop[j] = (int)found;
      uprop[j] = dvec[found];
      uacc[j] = ua;
    }
  }
}

cudaError_t launch_propose(const DevBuffers& b, int T, cudaStream_t s) {
  (void)T;
  // the tile prefix lives in shared memory up to 20,480 tiles (N <= 2.6M)
  const size_t bytes = (size_t)b.ntiles * sizeof(double);
  const int use_smem = bytes <= 160 * 1024 ? 1 : 0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_propose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_propose<<<1, 1024, use_smem ? bytes : 0, s>>>(b.st, b.dvec, b.tile_sums, b.tile_prefix,
                                                  b.ntiles, b.N, b.prop, b.uprop, b.uacc,
                                                  use_smem);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ H
// H = A(S',S') - F(S',:) F(S',:)^*, FP64 (FP32 factors are widened; their
// products are exact in FP64).  Kernel entries by direct differences.
// 8 x 8 output tiles, lower-triangle tiles only (H is symmetric; both
// halves are written from the same value), F rows staged 32 columns at a
// time.
template <typename TF>
__global__ void __launch_bounds__(64) k_hmat(const DevState* st, const float* __restrict__ X,
                                             int xld, int d, int kind, double inv_sigma,
                                             const TF* __restrict__ F, long long ldF,
                                             const int* __restrict__ prop, double* H) {
  __shared__ double Fa[8][33];
  __shared__ double Fb[8][33];
  if (st->done) return;
  if (blockIdx.x > blockIdx.y) return;
  const int T = st->T;
  const long long rank = st->rank;
  const int a0 = blockIdx.y * 8, b0 = blockIdx.x * 8;
  if (a0 >= T) return;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  double acc = 0.0;
  for (long long m0 = 0; m0 < rank; m0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 64 * q;  // 0..255: row e >> 5, column e & 31
      const int r = e >> 5, cc = e & 31;
      const long long m = m0 + cc;
      const int ra = a0 + r < T ? prop[a0 + r] : prop[0];
      const int rb = b0 + r < T ? prop[b0 + r] : prop[0];
      Fa[r][cc] = m < rank ? (double)F[(long long)ra * ldF + m] : 0.0;
      Fb[r][cc] = m < rank ? (double)F[(long long)rb * ldF + m] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 32; ++q) acc += Fa[ty][q] * Fb[tx][q];
    __syncthreads();
  }
  const int a = a0 + ty, bcol = b0 + tx;
  if (a < T && bcol < T && bcol <= a) {
    const int pa = prop[a], pb = prop[bcol];
    double kv = 1.0;
    if (pa != pb) {
      const float* xa = X + (long long)pa * xld;
      const float* xb = X + (long long)pb * xld;
      double r2 = 0.0;
      for (int l = 0; l < d; ++l) {
        const double t = (double)xa[l] - (double)xb[l];
        r2 += t * t;
      }
      kv = phi_r2<double>(kind, inv_sigma, r2);
    }
    const double h = kv - acc;
    H[(long long)a * T + bcol] = h;
    H[(long long)bcol * T + a] = h;
  }
}

cudaError_t launch_hmat(const DevBuffers& b, int T, cudaStream_t s) {
  const int nb = (T + 7) / 8;
  dim3 grid(nb, nb);
  if (b.mixed)
    k_hmat<float><<<grid, 64, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                                      (const float*)b.F, b.ldF, b.prop, b.H);
  else
    k_hmat<double><<<grid, 64, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                                       (const double*)b.F, b.ldF, b.prop, b.H);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Algorithm 1
// RejectionSampleSubmatrix in one CTA.  The lower triangle of H lives packed
// (row j at offset j(j+1)/2) in shared memory when it fits, otherwise in a
// global scratch array.  For i = 0..T-1: accept iff u_i * U_i < h_ii with
// u_i the proposal weight d[s'_i]; on acceptance L(i:T, i) = H(i:T, i) /
// sqrt(h_ii) and the trailing triangle is downdated.  Stops once the total
// rank reaches k.  Writes the compact L, the accepted pivots and s.
__device__ __forceinline__ long long pk(int j, int l) { return (long long)j * (j + 1) / 2 + l; }

__global__ void __launch_bounds__(512) k_reject(DevState* st, const double* __restrict__ H,
                                                const double* __restrict__ uprop,
                                                const double* __restrict__ uacc,
                                                const int* __restrict__ prop, double* Lw,
                                                double* L, int ldL, int* Sacc, long long* piv,
                                                double* Hglobal, int use_smem) {
  extern __shared__ double dyn[];
  __shared__ double lc[kTMax];
  __shared__ double us[kTMax];
  __shared__ int accl[kTMax];
  if (st->done) return;
  const int T = st->T;
  const long long rank = st->rank;
  long long maxacc_ll = st->k - rank;
  const int maxacc = maxacc_ll < T ? (int)maxacc_ll : T;
  double* Hp = use_smem ? dyn : Hglobal;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int j = warp; j < T; j += nw)
    for (int l = lane; l <= j; l += 32) Hp[pk(j, l)] = H[(long long)j * T + l];
  for (int i = tid; i < T; i += nt) us[i] = uprop[i] * uacc[i];
  __syncthreads();
  int n = 0;
  for (int i = 0; i < T; ++i) {
    if (n >= maxacc) break;
    const double h = Hp[pk(i, i)];
    if (us[i] < h) {
      const double inv = 1.0 / sqrt(h);
      for (int j = i + tid; j < T; j += nt) {
        const double v = Hp[pk(j, i)] * inv;
        lc[j] = v;
        Lw[(long long)j * kTMax + n] = v;
      }
      if (tid == 0) accl[n] = i;
      __syncthreads();
      for (int j = i + 1 + warp; j < T; j += nw) {
        const double lj = lc[j];
        for (int l = i + 1 + lane; l <= j; l += 32) Hp[pk(j, l)] -= lj * lc[l];
      }
      ++n;
      __syncthreads();
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    const int a = e / n, c = e % n;
    L[(long long)a * ldL + c] = c <= a ? Lw[(long long)accl[a] * kTMax + c] : 0.0;
  }
  for (int a = tid; a < n; a += nt) {
    const int p = prop[accl[a]];
    Sacc[a] = p;
    piv[rank + a] = p;
  }
  if (tid == 0) {
    st->s = n;
    if (n > 0 && !(L[0] > 0.0)) st->status |= kStNumeric;
  }
}

cudaError_t launch_reject(const DevBuffers& b, int T, cudaStream_t s) {
  const size_t packed = (size_t)T * (T + 1) / 2 * sizeof(double);
  const size_t static_bytes = sizeof(double) * 2 * kTMax + sizeof(int) * kTMax;
  const size_t limit = 227 * 1024 - static_bytes - 1024;
  const int use_smem = packed <= limit ? 1 : 0;
  const size_t dyn = use_smem ? packed : 0;
  if (use_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_reject, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_reject<<<1, 512, dyn, s>>>(b.st, b.H, b.uprop, b.uacc, b.prop, b.Lw, b.L, b.Tmax, b.Sacc,
                               b.piv, b.Hpk, use_smem);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gather
// Rows of the extended operand of the CUDA-core column step:
//   Bext(j, m) = F(S_j, m) for m < rank,  L(j, m - rank) for rank <= m < rank + s.
template <typename TR>
__global__ void k_gather_ext(const DevState* st, const TR* __restrict__ F, long long ldF,
                             const int* __restrict__ Sacc, const double* __restrict__ L, int ldL,
                             TR* Bext, long long ldB) {
  if (st->done) return;
  const int s = st->s;
  const int j = blockIdx.x;
  if (j >= s) return;
  const long long rank = st->rank;
  const long long src = (long long)Sacc[j] * ldF;
  for (long long m = threadIdx.x; m < rank + s; m += blockDim.x)
    Bext[(long long)j * ldB + m] =
        m < rank ? F[src + m] : (TR)L[(long long)j * ldL + (m - rank)];
}

cudaError_t launch_gather_f64(const DevBuffers& b, int T, cudaStream_t s) {
  if (b.mixed)
    k_gather_ext<float><<<T, 256, 0, s>>>(b.st, (const float*)b.F, b.ldF, b.Sacc, b.L, b.Tmax,
                                          (float*)b.Bext, b.ldB);
  else
    k_gather_ext<double><<<T, 256, 0, s>>>(b.st, (const double*)b.F, b.ldF, b.Sacc, b.L, b.Tmax,
                                           b.Bext, b.ldB);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ control
__global__ void k_round_end(DevState* st, cudaGraphConditionalHandle cond, int use_cond,
                            long long N, int d, int bF) {
  if (!st->done) {
    const double n = (double)N, r = (double)st->rank, sc = (double)st->s;
    st->col_bytes += n * (r * bF + sc * bF + 4.0 * d + 16.0);
    st->col_flops += 2.0 * n * r * sc + n * sc * sc + 3.0 * n * d * sc;
    st->rank += st->s;
    st->round += 1;
    st->proposals += st->T;
    if (st->rank >= st->k) {
      st->done = 1;
    } else if (st->round >= st->max_rounds) {
      st->done = 1;
      st->status |= kStRoundLimit;
    }
  }
  if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

cudaError_t launch_round_end(const DevBuffers& b, unsigned long long cond, int use_cond,
                             cudaStream_t s) {
  k_round_end<<<1, 1, 0, s>>>(b.st, (cudaGraphConditionalHandle)cond, use_cond, b.N, b.d,
                              b.mixed ? 4 : 8);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ trace error
// red[blockIdx] = sum over the block's rows of (1 - ||F(r, 0:rank)||^2), FP64.
template <typename TF>
__global__ void __launch_bounds__(256) k_trace_part(const DevState* st, const TF* __restrict__ F,
                                                    long long ldF, long long N, double* red) {
  __shared__ double ws[8];
  const long long rank = st->rank;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (long long r = (long long)blockIdx.x * 8 + warp; r < N; r += (long long)gridDim.x * 8) {
    double sq = 0.0;
    for (long long m = lane; m < rank; m += 32) {
      const double f = (double)F[r * ldF + m];
      sq += f * f;
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if (lane == 0) acc += 1.0 - sq;
  }
  if (lane == 0) ws[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    red[1 + blockIdx.x] = t;
  }
}

__global__ void k_trace_final(double* red, int nparts, const double* dvec, long long N) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) t += red[1 + i];
  sh[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < 256; ++i) s += sh[i];
    red[0] = s;
  }
  __syncthreads();
  // clamped residual diagonal sum
  double u = 0.0;
  for (long long i = threadIdx.x; i < N; i += 256) u += dvec[i];
  sh[threadIdx.x] = u;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < 256; ++i) s += sh[i];
    red[nparts + 1] = s;
  }
}

cudaError_t launch_trace(const DevBuffers& b, cudaStream_t s) {
  int parts = (int)((b.N + 7) / 8);
  if (parts > (int)b.nred - 2) parts = (int)b.nred - 2;
  if (parts > 2048) parts = 2048;
  if (parts < 1) parts = 1;
  if (b.mixed)
    k_trace_part<float><<<parts, 256, 0, s>>>(b.st, (const float*)b.F, b.ldF, b.N, b.red);
  else
    k_trace_part<double><<<parts, 256, 0, s>>>(b.st, (const double*)b.F, b.ldF, b.N, b.red);
  k_trace_final<<<1, 256, 0, s>>>(b.red, parts, b.dvec, b.N);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ input prep
__global__ void k_convert_x64(const double* __restrict__ src, long long N, int d, float* X,
                              int xld) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * (long long)d) return;
  const long long r = i / d;
  const int c = (int)(i % d);
  X[r * xld + c] = (float)src[i];
}

cudaError_t launch_convert_x64(const double* src, long long N, int d, float* X, int xld,
                               cudaStream_t s) {
  const long long n = N * (long long)d;
  k_convert_x64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, N, d, X, xld);
  return cudaGetLastError();
}

// ||x||^2 in FP32 from the FP32 points (FP64 accumulation, rounded once).
__global__ void k_norms(const float* __restrict__ X, int xld, int d, long long N, float* nrm) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double s = 0.0;
  for (int l = 0; l < d; ++l) {
    const double v = (double)X[r * xld + l];
    s += v * v;
  }
  nrm[r] = (float)s;
}

cudaError_t launch_norms(const DevBuffers& b, cudaStream_t s) {
  k_norms<<<(unsigned)((b.N + 255) / 256), 256, 0, s>>>(b.X, b.xld, b.d, b.N,
                                                        const_cast<float*>(b.nrm));
  return cudaGetLastError();
}

__global__ void k_widen_f32(const float* __restrict__ F, long long ldF, long long N,
                            long long cols, double* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * cols) return;
  const long long r = i / cols, c = i % cols;
  out[i] = (double)F[r * ldF + c];
}

cudaError_t launch_widen_f32(const float* F, long long ldF, long long N, long long cols,
                             double* out, cudaStream_t s) {
  const long long n = N * cols;
  k_widen_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(F, ldF, N, cols, out);
  return cudaGetLastError();
}

}  // namespace rpchol
