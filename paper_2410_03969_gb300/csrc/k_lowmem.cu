// Low-memory accelerated RPCholesky (Algorithm 3, Sec. 2.4 of arXiv
// 2410.03969), FP64.  No N x k factor is stored: the context keeps the
// pivots S and the Cholesky factor L of A(S,S) (k x k, both row-major Lr and
// column-major Lc copies, so that forward and back substitution both read
// contiguous memory), regenerating kernel entries as they are needed.
//
// One round (every kernel reads rank, T and s from the device state):
//   propose     the T draws of Algorithm 2 (shared with the accelerated path)
//   k_lm_y      Y(:,j) = L^{-1} A(S, s'_j), one CTA per draw: blocked forward
//               substitution (a warp solves each 32 x 32 diagonal block, the
//               CTA updates the trailing entries)
//   k_lm_h      H = A(S',S') - Y^* Y, 16 x 16 tiles
//   reject      Algorithm 1 on H (shared): L_i, accepted pivots S_i
//   k_lm_m      M(:,a) = L^{-*} Y(:, acc_a), blocked back substitution
//   k_lm_b      B = [-M L_i^{-*}; L_i^{-*}] = the last s columns of L_new^{-*},
//               so that the new columns of the (implicit) factor are
//               G = A(:, S_new) B, with S_new = S followed by S_i
//   k_lm_col    for every 128-row tile: G = A(R, S_new) B with kernel entries
//               regenerated (direct differences, FP64), d(R) -= |G(r,:)|^2,
//               clamp at 0, tile sums for the next draw; G itself is dropped
//   k_lm_lupd   L <- [L 0; Y(:,acc)^* L_i] in both copies
//   round end   rank += s (shared)
// The listing's step 3 forms G with L_i^{-*} by substitution per row chunk;
// here the product with the s x s triangular inverse is folded into B once
// per round (same matrix in exact arithmetic), so the N-row kernel is one
// regenerate-and-contract pass without a per-row triangular solve.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "rpchol.h"

namespace rpchol {
namespace {

constexpr int kLmMaxK = 16384;  // k_max limit: one FP64 vector of rank entries per CTA in smem
constexpr int kCM = 128;        // rows per CTA of the column kernel (one sampler tile)
constexpr int kCN = 64;         // columns of G per pass
constexpr int kCK = 8;          // centres per staged chunk

__device__ __forceinline__ double kappa64(const float* __restrict__ X, int xld, int d, int kind,
                                          double inv_sigma, long long a, long long b) {
  if (a == b) return 1.0;
  const float* xa = X + a * xld;
  const float* xb = X + b * xld;
  double r2 = 0.0;
  for (int l = 0; l < d; ++l) {
    const double t = (double)xa[l] - (double)xb[l];
    r2 += dist_term(kind, t);
  }
  return phi_r2<double>(kind, inv_sigma, r2);
}

__global__ void __launch_bounds__(256)
    k_lm_y(const DevState* st, const float* __restrict__ X, int xld, int d, int kind,
           double inv_sigma, const int* __restrict__ prop, const long long* __restrict__ piv,
           const double* __restrict__ Lc, long long ldL, double* Y, long long ldY) {
  extern __shared__ double y[];
  if (st->done) return;
  const int T = st->T;
  const int j = blockIdx.x;
  if (j >= T) return;
  const long long rank = st->rank;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long pj = prop[j];
  for (long long m = tid; m < rank; m += 256) y[m] = kappa64(X, xld, d, kind, inv_sigma, piv[m], pj);
  __syncthreads();
  for (long long m0 = 0; m0 < rank; m0 += 32) {
    const int bs = rank - m0 < 32 ? (int)(rank - m0) : 32;
    if (warp == 0) {
      double v = lane < bs ? y[m0 + lane] : 0.0;
      for (int i = 0; i < bs; ++i) {
        const double yi = __shfl_sync(0xffffffffu, v, i) / Lc[(m0 + i) * ldL + m0 + i];
        if (lane == i) v = yi;
        if (lane > i && lane < bs) v -= Lc[(m0 + i) * ldL + m0 + lane] * yi;
      }
      if (lane < bs) y[m0 + lane] = v;
    }
    __syncthreads();
    for (long long mp = m0 + bs + tid; mp < rank; mp += 256) {
      double v = y[mp];
      for (int i = 0; i < bs; ++i) v -= Lc[(m0 + i) * ldL + mp] * y[m0 + i];
      y[mp] = v;
    }
    __syncthreads();
  }
  for (long long m = tid; m < rank; m += 256) Y[(long long)j * ldY + m] = y[m];
}

__global__ void __launch_bounds__(256)
    k_lm_h(const DevState* st, const float* __restrict__ X, int xld, int d, int kind,
           double inv_sigma, const int* __restrict__ prop, const double* __restrict__ Y,
           long long ldY, double* H) {
  __shared__ double Ya[16][33], Yb[16][33];
  if (st->done) return;
  const int T = st->T;
  const long long rank = st->rank;
  const int a0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
  if (a0 >= T || c0 >= T) return;
  const int tid = threadIdx.x, ta = tid >> 4, tc = tid & 15;
  double acc = 0.0;
  for (long long m0 = 0; m0 < rank; m0 += 32) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + 256 * q;
      const int r = e >> 5, mm = e & 31;
      const long long m = m0 + mm;
      Ya[r][mm] = (a0 + r < T && m < rank) ? Y[(long long)(a0 + r) * ldY + m] : 0.0;
      Yb[r][mm] = (c0 + r < T && m < rank) ? Y[(long long)(c0 + r) * ldY + m] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int mm = 0; mm < 32; ++mm) acc = fma(Ya[ta][mm], Yb[tc][mm], acc);
    __syncthreads();
  }
  const int a = a0 + ta, c = c0 + tc;
  if (a < T && c < T)
    H[(long long)a * T + c] = kappa64(X, xld, d, kind, inv_sigma, prop[a], prop[c]) - acc;
}

__global__ void __launch_bounds__(256)
    k_lm_m(const DevState* st, const int* __restrict__ prop, const int* __restrict__ Sacc,
           const double* __restrict__ Lr, long long ldL, const double* __restrict__ Y,
           long long ldY, double* Mt, int* accj) {
  extern __shared__ double z[];
  __shared__ int jsh;
  if (st->done) return;
  const int s = st->s;
  const int a = blockIdx.x;
  if (a >= s) return;
  const int T = st->T;
  const long long rank = st->rank;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    int j = 0;
    while (j < T && prop[j] != Sacc[a]) ++j;
    jsh = j < T ? j : 0;
    accj[a] = jsh;
  }
  __syncthreads();
  const int j = jsh;
  for (long long m = tid; m < rank; m += 256) z[m] = Y[(long long)j * ldY + m];
  __syncthreads();
  for (long long m1 = rank; m1 > 0; m1 -= 32) {
    const long long m0 = m1 > 32 ? m1 - 32 : 0;
    const int bs = (int)(m1 - m0);
    if (warp == 0) {
      double v = lane < bs ? z[m0 + lane] : 0.0;
      for (int i = bs - 1; i >= 0; --i) {
        const double zi = __shfl_sync(0xffffffffu, v, i) / Lr[(m0 + i) * ldL + m0 + i];
        if (lane == i) v = zi;
        if (lane < i) v -= Lr[(m0 + i) * ldL + m0 + lane] * zi;
      }
      if (lane < bs) z[m0 + lane] = v;
    }
    __syncthreads();
    for (long long mp = tid; mp < m0; mp += 256) {
      double v = z[mp];
      for (int i = 0; i < bs; ++i) v -= Lr[(m0 + i) * ldL + mp] * z[m0 + i];
      z[mp] = v;
    }
    __syncthreads();
  }
  for (long long m = tid; m < rank; m += 256) Mt[(long long)a * ldY + m] = z[m];
}

__global__ void __launch_bounds__(256)
    k_lm_b(const DevState* st, const double* __restrict__ Li, int ldLi,
           const double* __restrict__ Mt, long long ldY, double* Bt, long long ldB) {
  __shared__ double w[kTMax];
  __shared__ double ysh[kTMax];
  if (st->done) return;
  const int s = st->s;
  const int a = blockIdx.x;
  if (a >= s) return;
  const long long rank = st->rank;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // w = L_i^{-*} e_a: back substitution with the upper-triangular L_i^*
  if (warp == 0) {
    for (int c = lane; c <= a; c += 32) ysh[c] = c == a ? 1.0 : 0.0;
    __syncwarp();
    for (int l = a; l >= 0; --l) {
      const double wl = ysh[l] / Li[(long long)l * ldLi + l];
      __syncwarp();
      if (lane == 0) w[l] = wl;
      for (int c = lane; c < l; c += 32) ysh[c] -= Li[(long long)l * ldLi + c] * wl;
      __syncwarp();
    }
  }
  __syncthreads();
  for (long long m = tid; m < rank; m += 256) {
    double v = 0.0;
    for (int c = 0; c <= a; ++c) v = fma(Mt[(long long)c * ldY + m], w[c], v);
    Bt[(long long)a * ldB + m] = -v;
  }
  for (int c = tid; c < s; c += 256) Bt[(long long)a * ldB + rank + c] = c <= a ? w[c] : 0.0;
}

__global__ void __launch_bounds__(256)
    k_lm_col(const DevState* st, const float* __restrict__ X, int xld, int d, int kind,
             double inv_sigma, const long long* __restrict__ piv, const double* __restrict__ Bt,
             long long ldB, double* dvec, double* tile_sums, long long N) {
  __shared__ double Ks[kCK][kCM + 1];
  __shared__ double Bs[kCK][kCN + 1];
  __shared__ double rowsq[kCM][17];
  __shared__ double red[8];
  if (st->done) return;
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const long long nc = rank + s;  // centres: piv[0 .. rank + s)
  const long long row0 = (long long)blockIdx.x * kCM;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double rsq[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) rsq[i] = 0.0;
  for (int c0 = 0; c0 < s; c0 += kCN) {
    double acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (long long m0 = 0; m0 < nc; m0 += kCK) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q;
        const int kk = e >> 7, r = e & 127;
        const long long gr = row0 + r, m = m0 + kk;
        Ks[kk][r] = (gr < N && m < nc) ? kappa64(X, xld, d, kind, inv_sigma, gr, piv[m]) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = tid + 256 * q;
        const int kk = e >> 6, j = e & 63;
        const long long m = m0 + kk;
        Bs[kk][j] = (m < nc && c0 + j < s) ? Bt[(long long)(c0 + j) * ldB + m] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kCK; ++kk) {
        double av[8], bv[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = Ks[kk][ty * 8 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (c0 + tx * 4 + j < s) rsq[i] = fma(acc[i][j], acc[i][j], rsq[i]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) rowsq[ty * 8 + i][tx] = rsq[i];
  __syncthreads();
  double dn = 0.0;
  if (tid < kCM) {
    const long long gr = row0 + tid;
    if (gr < N) {
      double t = 0.0;
      for (int q = 0; q < 16; ++q) t += rowsq[tid][q];
      const double v = dvec[gr] - t;
      dn = v > kDFloor64 ? v : 0.0;
      dvec[gr] = dn;
    }
  }
  const double tsum = block_sum_fixed(dn, red);
  if (tid == 0) tile_sums[blockIdx.x] = tsum;
}

__global__ void __launch_bounds__(256)
    k_lm_lupd(const DevState* st, const double* __restrict__ Li, int ldLi,
              const double* __restrict__ Y, long long ldY, const int* __restrict__ accj,
              double* Lr, double* Lc, long long ldL) {
  if (st->done) return;
  const int s = st->s;
  const int a = blockIdx.x;
  if (a >= s) return;
  const long long rank = st->rank;
  const long long row = rank + a;
  const int j = accj[a];
  for (long long m = threadIdx.x; m < rank; m += blockDim.x) {
    const double v = Y[(long long)j * ldY + m];
    Lr[row * ldL + m] = v;
    Lc[m * ldL + row] = v;
  }
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    const double v = c <= a ? Li[(long long)a * ldLi + c] : 0.0;
    Lr[row * ldL + rank + c] = v;
    Lc[(rank + c) * ldL + row] = v;
  }
}

}  // namespace
}  // namespace rpchol

using namespace rpchol;

struct rpchol_lowmem {
  DevBuffers b{};
  cudaStream_t stream = nullptr;
  long long k_max = 0;
  long long ldL = 0, ldY = 0, ldB = 0;
  double* Lr = nullptr;
  double* Lc = nullptr;
  double* Y = nullptr;
  double* Mt = nullptr;
  double* Bt = nullptr;
  int* accj = nullptr;
  DevState* st_host = nullptr;
  std::vector<void*> owned;
  int has_run = 0;
};

namespace {

rpchol_status lm_cuda_fail(cudaError_t e, const char* where) {
  set_last_error("%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RPCHOL_ENOMEM : RPCHOL_ECUDA;
}

#define LMCU(call)                                            \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return lm_cuda_fail(e__, #call);  \
  } while (0)

void lm_release(rpchol_lowmem* c) {
  for (void* p : c->owned) cudaFreeAsync(p, c->stream);
  c->owned.clear();
  cudaStreamSynchronize(c->stream);
  if (c->st_host) cudaFreeHost(c->st_host);
  c->st_host = nullptr;
}

rpchol_status lm_alloc(rpchol_lowmem* c, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, c->stream);
  if (e != cudaSuccess) return lm_cuda_fail(e, "cudaMallocAsync");
  c->owned.push_back(*p);
  return RPCHOL_OK;
}

rpchol_status lm_status(const DevState& s) {
  if (s.status & kStNumeric) {
    set_last_error("non-positive pivot or non-finite value met on the device");
    return RPCHOL_ENUMERIC;
  }
  if (s.status & kStRoundLimit) {
    set_last_error("round limit reached before the target rank");
    return RPCHOL_ETIMEOUT;
  }
  if (s.status & kStTimeout) {
    set_last_error("a bounded device-side wait expired");
    return RPCHOL_ETIMEOUT;
  }
  return RPCHOL_OK;
}

cudaError_t lm_round(rpchol_lowmem* c, int T) {
  const DevBuffers& b = c->b;
  cudaStream_t s = c->stream;
  const double inv_sigma = 1.0 / b.sigma;
  const size_t vec = sizeof(double) * (size_t)c->k_max;
  cudaError_t e = launch_propose(b, T, s);
  if (e != cudaSuccess) return e;
  k_lm_y<<<T, 256, vec, s>>>(b.st, b.X, b.xld, b.d, b.kind, inv_sigma, b.prop, b.piv, c->Lc,
                             c->ldL, c->Y, c->ldY);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned ht = (unsigned)((T + 15) / 16);
  k_lm_h<<<dim3(ht, ht), 256, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, inv_sigma, b.prop, c->Y,
                                      c->ldY, b.H);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_reject(b, T, s)) != cudaSuccess) return e;
  k_lm_m<<<T, 256, vec, s>>>(b.st, b.prop, b.Sacc, c->Lr, c->ldL, c->Y, c->ldY, c->Mt, c->accj);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_lm_b<<<T, 256, 0, s>>>(b.st, b.L, b.Tmax, c->Mt, c->ldY, c->Bt, c->ldB);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_lm_col<<<(unsigned)b.ntiles, 256, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, inv_sigma, b.piv,
                                              c->Bt, c->ldB, b.dvec, b.tile_sums, b.N);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_lm_lupd<<<T, 256, 0, s>>>(b.st, b.L, b.Tmax, c->Y, c->ldY, c->accj, c->Lr, c->Lc, c->ldL);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_round_end(b, 0ull, 0, s);
}

}  // namespace

extern "C" {

rpchol_status rpchol_lowmem_create(int32_t kind, double sigma, const void* X, int64_t N,
                                   int32_t d, int32_t x_dtype, int64_t k_max, int32_t T_max,
                                   void* stream, rpchol_lowmem** out) {
  set_last_error("%s", "");
  if (!out) {
    set_last_error("out is NULL");
    return RPCHOL_EINVAL;
  }
  *out = nullptr;
  if (!X || N < 1 || d < 1 || d > 4096 || !(sigma > 0.0) || kind < 0 || kind > 4 || k_max < 1 ||
      k_max > N || k_max > kLmMaxK || T_max < 1 || T_max > kTMax ||
      (x_dtype != RPCHOL_DT_F32 && x_dtype != RPCHOL_DT_F64)) {
    set_last_error("invalid argument: N=%lld d=%d sigma=%g kind=%d k_max=%lld T_max=%d",
                   (long long)N, d, sigma, kind, (long long)k_max, T_max);
    return RPCHOL_EINVAL;
  }
  rpchol_lowmem* c = new (std::nothrow) rpchol_lowmem();
  if (!c) {
    set_last_error("host allocation failed");
    return RPCHOL_ENOMEM;
  }
  c->stream = (cudaStream_t)stream;
  c->k_max = k_max;
  c->ldL = round_up(k_max, kLdAlign);
  c->ldY = c->ldL;
  c->ldB = c->ldL + kTMax;
  DevBuffers& b = c->b;
  b.N = N;
  b.d = d;
  b.xld = (int)round_up(d, kLdAlign);
  b.kind = kind;
  b.sigma = sigma;
  b.ntiles = (N + kTileRows - 1) / kTileRows;
  b.Tmax = T_max;
  b.mixed = 0;
  b.nred = 4;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm < 1)
      nsm = 148;
    b.num_sms = nsm;
  }
  rpchol_status rs = RPCHOL_OK;
  auto fail = [&](rpchol_status s) {
    lm_release(c);
    delete c;
    return s;
  };
  cudaError_t e = cudaMallocHost((void**)&c->st_host, sizeof(DevState));
  if (e != cudaSuccess) return fail(lm_cuda_fail(e, "cudaMallocHost"));
  memset(c->st_host, 0, sizeof(DevState));
  void* p;
#define LMALLOC(dst, type, count)                                              \
  do {                                                                         \
    if ((rs = lm_alloc(c, &p, sizeof(type) * (size_t)(count))) != RPCHOL_OK)   \
      return fail(rs);                                                         \
    dst = (type*)p;                                                            \
  } while (0)
  float* Xp;
  LMALLOC(Xp, float, (size_t)N * b.xld);
  b.X = Xp;
  LMALLOC(b.dvec, double, N);
  LMALLOC(b.tile_sums, double, b.ntiles);
  LMALLOC(b.tile_prefix, double,
          b.ntiles * sizeof(double) <= 160 * 1024 ? b.ntiles : b.ntiles * (kTMax / 8));
  LMALLOC(b.piv, long long, k_max);
  LMALLOC(b.prop, int, kTMax);
  LMALLOC(b.uprop, double, kTMax);
  LMALLOC(b.uacc, double, kTMax);
  LMALLOC(b.H, double, (size_t)kTMax * kTMax);
  LMALLOC(b.Lw, double, (size_t)kTMax * kTMax);
  LMALLOC(b.L, double, (size_t)kTMax * T_max);
  LMALLOC(b.Sacc, int, kTMax);
  LMALLOC(b.red, double, b.nred);
  LMALLOC(b.st, DevState, 1);
  LMALLOC(c->Lr, double, (size_t)k_max * c->ldL);
  LMALLOC(c->Lc, double, (size_t)k_max * c->ldL);
  LMALLOC(c->Y, double, (size_t)kTMax * c->ldY);
  LMALLOC(c->Mt, double, (size_t)kTMax * c->ldY);
  LMALLOC(c->Bt, double, (size_t)kTMax * c->ldB);
  LMALLOC(c->accj, int, kTMax);
#undef LMALLOC
  e = cudaMemsetAsync((void*)b.X, 0, sizeof(float) * (size_t)N * b.xld, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.st, 0, sizeof(DevState), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.piv, 0xff, sizeof(long long) * (size_t)k_max, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->Lr, 0, sizeof(double) * (size_t)k_max * c->ldL, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->Lc, 0, sizeof(double) * (size_t)k_max * c->ldL, c->stream);
  if (e != cudaSuccess) return fail(lm_cuda_fail(e, "cudaMemsetAsync"));
  if (x_dtype == RPCHOL_DT_F32) {
    e = cudaMemcpy2DAsync((void*)b.X, sizeof(float) * b.xld, X, sizeof(float) * d,
                          sizeof(float) * d, N, cudaMemcpyDefault, c->stream);
  } else {
    void* tmp = nullptr;
    e = cudaMallocAsync(&tmp, sizeof(double) * (size_t)N * d, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp, X, sizeof(double) * (size_t)N * d, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
      e = launch_convert_x64((const double*)tmp, N, d, (float*)b.X, b.xld, c->stream);
    if (tmp) cudaFreeAsync(tmp, c->stream);
  }
  if (e != cudaSuccess) return fail(lm_cuda_fail(e, "copy of X"));
  const int vec = (int)(sizeof(double) * (size_t)k_max);
  if (vec > 48 * 1024) {
    e = cudaFuncSetAttribute(k_lm_y, cudaFuncAttributeMaxDynamicSharedMemorySize, vec);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_lm_m, cudaFuncAttributeMaxDynamicSharedMemorySize, vec);
    if (e != cudaSuccess) return fail(lm_cuda_fail(e, "cudaFuncSetAttribute"));
  }
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(lm_cuda_fail(e, "create"));
  *out = c;
  return RPCHOL_OK;
}

rpchol_status rpchol_lowmem_run(rpchol_lowmem* c, int64_t k, int32_t T, uint64_t seed) {
  set_last_error("%s", "");
  if (!c || k < 1 || k > c->k_max || T < 1 || T > c->b.Tmax) {
    set_last_error("invalid argument: k=%lld T=%d", (long long)k, T);
    return RPCHOL_EINVAL;
  }
  const long long max_rounds = 4 * k + 64;
  // rows of an earlier, longer run may hold entries right of the diagonal:
  // the copied-out factor starts from zeros
  LMCU(cudaMemsetAsync(c->Lr, 0, sizeof(double) * (size_t)c->k_max * c->ldL, c->stream));
  LMCU(launch_reset(c->b, k, T, seed, 0u, 0, max_rounds, c->stream));
  c->has_run = 1;
  for (long long it = 0; it < max_rounds + 1;) {
    for (int j = 0; j < 8; ++j, ++it) LMCU(lm_round(c, T));
    LMCU(cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevState), cudaMemcpyDeviceToHost,
                         c->stream));
    LMCU(cudaStreamSynchronize(c->stream));
    if (c->st_host->done) break;
  }
  return lm_status(*c->st_host);
}

rpchol_status rpchol_lowmem_copy(rpchol_lowmem* c, double* L_out, int64_t ld_out,
                                 int64_t* pivots_out, double* d_out, int64_t* rank_out,
                                 int64_t* rounds_out) {
  if (!c) return RPCHOL_EINVAL;
  LMCU(cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  LMCU(cudaStreamSynchronize(c->stream));
  const long long rank = c->has_run ? c->st_host->rank : 0;
  if (L_out && ld_out < rank) {
    set_last_error("ld_out %lld < rank %lld", (long long)ld_out, rank);
    return RPCHOL_EINVAL;
  }
  if (L_out && rank > 0)
    LMCU(cudaMemcpy2DAsync(L_out, sizeof(double) * ld_out, c->Lr, sizeof(double) * c->ldL,
                           sizeof(double) * rank, rank, cudaMemcpyDefault, c->stream));
  if (pivots_out && rank > 0)
    LMCU(cudaMemcpyAsync(pivots_out, c->b.piv, sizeof(long long) * rank, cudaMemcpyDefault,
                         c->stream));
  if (d_out)
    LMCU(cudaMemcpyAsync(d_out, c->b.dvec, sizeof(double) * c->b.N, cudaMemcpyDefault,
                         c->stream));
  LMCU(cudaStreamSynchronize(c->stream));
  if (rank_out) *rank_out = rank;
  if (rounds_out) *rounds_out = c->has_run ? c->st_host->round : 0;
  return c->has_run ? lm_status(*c->st_host) : RPCHOL_OK;
}

rpchol_status rpchol_lowmem_destroy(rpchol_lowmem* c) {
  if (!c) return RPCHOL_OK;
  lm_release(c);
  delete c;
  return RPCHOL_OK;
}

}  // extern "C"
