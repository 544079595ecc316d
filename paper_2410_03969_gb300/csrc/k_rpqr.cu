// Accelerated randomly pivoted QR (Algorithm 5, appendix of arXiv
// 2410.03969) of a dense M x N matrix B, FP64 on CUDA cores.  The sampler
// and Algorithm 1 are the accelerated Cholesky path's own kernels, run on
// u = squared residual column norms and on H = C^* C; every dense product is
// one strided FP64 tiled GEMM (k_dgemm).  Layout: B column-major (column j
// contiguous, ld M), Q column-major (ld M; the new columns are written in
// place), F row-major N x ldF as in the Cholesky path.
//
// One round (the host reads the accepted count after Algorithm 1):
//   propose                T draws from u (shared)
//   gather + GEMM          C = B(:,S') - Q F(S',:)^*          (M x T)
//   GEMM                   H = C^* C                          (T x T)
//   reject                 Algorithm 1 on H: S_i (its L is not used)
//   copy                   Q_perp = C(:, acc) into Q(:, rank:rank+s)
//   2 GEMMs                Q_perp -= Q (Q^* Q_perp)           (second Gram-Schmidt pass)
//   Cholesky QR, twice     Q_perp <- Q_perp R^{-1}, R^* R = Q_perp^* Q_perp
//                          (the thin-QR factor with positive diagonal)
//   GEMM                   G = B^* Q_perp into F(:, rank:rank+s)
//   update                 u <- max(u - rowsumsq(G), 0), tile sums; round end (shared)
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "rpchol.h"

namespace rpchol {
namespace {

constexpr int kGM = 64, kGN = 64, kGK = 8;

// C(i,j) = beta C(i,j) + alpha sum_k A(i,k) B(k,j) for i < m, j < n, k < K;
// X(r,c) = X[r * xr + c * xc].  Each operand's staging order follows its
// unit stride (coalesced along it).
// Split K (gridDim.z > 1): CTA z sums k in [z Kc, (z + 1) Kc) and writes
// alpha times its partial to P + z m n (dense, row-major); k_splitk_sum adds
// the partials in z order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256)
    k_dgemm(long long m, long long n, long long K, double alpha, const double* __restrict__ A,
            long long ar, long long ac, const double* __restrict__ Bm, long long br,
            long long bc, double beta, double* C, long long cr, long long cc, long long Kc,
            double* P) {
  __shared__ double As[kGK][kGM + 1];
  __shared__ double Bs[kGK][kGN + 1];
  const long long i0 = (long long)blockIdx.y * kGM, j0 = (long long)blockIdx.x * kGN;
  const long long kb = (long long)blockIdx.z * Kc;
  const long long ke = kb + Kc < K ? kb + Kc : K;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const bool a_k_fast = ac == 1, b_k_fast = br == 1;
  for (long long k0 = kb; k0 < ke; k0 += kGK) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + 256 * q;
      int r, kk;
      if (a_k_fast) { r = e >> 3; kk = e & 7; } else { r = e & 63; kk = e >> 6; }
      const long long gi = i0 + r, gk = k0 + kk;
      As[kk][r] = (gi < m && gk < ke) ? A[gi * ar + gk * ac] : 0.0;
      int c, kq;
      if (b_k_fast) { c = e >> 3; kq = e & 7; } else { c = e & 63; kq = e >> 6; }
      const long long gj = j0 + c, gkb = k0 + kq;
      Bs[kq][c] = (gj < n && gkb < ke) ? Bm[gkb * br + gj * bc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long gi = i0 + ty * 4 + i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long gj = j0 + tx * 4 + j;
      if (gj >= n) continue;
      if (P) {
        P[((long long)blockIdx.z * m + gi) * n + gj] = alpha * acc[i][j];
      } else {
        double* p = C + gi * cr + gj * cc;
        *p = beta == 0.0 ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *p);
      }
    }
  }
}

__global__ void __launch_bounds__(256)
    k_splitk_sum(long long m, long long n, int splits, const double* __restrict__ P, double beta,
                 double* C, long long cr, long long cc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const long long i = e / n, j = e % n;
  double v = 0.0;
  for (int z = 0; z < splits; ++z) v += P[(long long)z * m * n + e];
  double* p = C + i * cr + j * cc;
  *p = beta == 0.0 ? v : fma(beta, *p, v);
}

// Workspace for split-K partials (doubles), owned by the context.
struct SplitWs {
  double* p = nullptr;
  long long cap = 0;
  int num_sms = 148;
};

// C = beta C + alpha A B.  Few output tiles over a long K (the Gram-type
// products H, Q^* Q_perp, Q_perp^* Q_perp) split K across CTAs so that the
// grid covers the GPU.
cudaError_t dgemm(long long m, long long n, long long K, double alpha, const double* A,
                  long long ar, long long ac, const double* B, long long br, long long bc,
                  double beta, double* C, long long cr, long long cc, cudaStream_t s,
                  const SplitWs* ws = nullptr) {
  if (m <= 0 || n <= 0 || (K <= 0 && beta == 1.0)) return cudaSuccess;
  const long long tiles = ((n + kGN - 1) / kGN) * ((m + kGM - 1) / kGM);
  int splits = 1;
  if (ws && ws->p && K >= 1024 && tiles < ws->num_sms) {
    long long want = (2LL * ws->num_sms + tiles - 1) / tiles;
    const long long by_k = K / 256;
    const long long by_ws = ws->cap / (m * n);
    if (want > by_k) want = by_k;
    if (want > by_ws) want = by_ws;
    if (want > 64) want = 64;
    if (want > 1) splits = (int)want;
  }
  long long Kc = K;
  if (splits > 1) Kc = (((K + splits - 1) / splits) + kGK - 1) / kGK * kGK;
  if (splits > 1) splits = (int)((K + Kc - 1) / Kc);
  const dim3 grid((unsigned)((n + kGN - 1) / kGN), (unsigned)((m + kGM - 1) / kGM),
                  (unsigned)splits);
  k_dgemm<<<grid, 256, 0, s>>>(m, n, K, alpha, A, ar, ac, B, br, bc, beta, C, cr, cc,
                               splits > 1 ? Kc : (K > 0 ? K : 1), splits > 1 ? ws->p : nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  k_splitk_sum<<<(unsigned)((m * n + 255) / 256), 256, 0, s>>>(m, n, splits, ws->p, beta, C, cr,
                                                              cc);
  return cudaGetLastError();
}

// u_j = |B(:,j)|^2 and the per-tile sums of u (one CTA per 128 columns)
__global__ void __launch_bounds__(kTileRows)
    k_qr_norms(const double* __restrict__ Bc, long long M, long long N, double* u,
               double* tile_sums) {
  __shared__ double red[8];
  const long long j = (long long)blockIdx.x * kTileRows + threadIdx.x;
  double t = 0.0;
  if (j < N) {
    const double* col = Bc + j * M;
    for (long long i = 0; i < M; ++i) t = fma(col[i], col[i], t);
    u[j] = t;
  }
  const double ts = block_sum_fixed(j < N ? t : 0.0, red);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = ts;
}

// Cg(a,:) = B(:, s'_a)^T, Fg(a, 0:rank) = F(s'_a, 0:rank)
__global__ void __launch_bounds__(256)
    k_qr_gather(const int* __restrict__ prop, const double* __restrict__ Bc, long long M,
                const double* __restrict__ F, long long ldF, long long rank, double* Cg,
                double* Fg, long long ldFg) {
  const int a = blockIdx.x;
  const long long p = prop[a];
  for (long long i = threadIdx.x; i < M; i += blockDim.x) Cg[(long long)a * M + i] = Bc[p * M + i];
  for (long long m = threadIdx.x; m < rank; m += blockDim.x)
    Fg[(long long)a * ldFg + m] = F[p * ldF + m];
}

// Q(:, rank + a) = C(:, acc_a): the accepted proposal's residual column
__global__ void __launch_bounds__(256)
    k_qr_take(const DevState* st, const int* __restrict__ prop, const int* __restrict__ Sacc,
              const double* __restrict__ Cg, long long M, double* Qc, long long rank) {
  __shared__ int jsh;
  const int a = blockIdx.x;
  if (a >= st->s) return;
  if (threadIdx.x == 0) {
    const int T = st->T;
    int j = 0;
    while (j < T && prop[j] != Sacc[a]) ++j;
    jsh = j < T ? j : 0;
  }
  __syncthreads();
  const int j = jsh;
  for (long long i = threadIdx.x; i < M; i += blockDim.x)
    Qc[(rank + a) * M + i] = Cg[(long long)j * M + i];
}

// In-place Cholesky G = L L^* of an s x s matrix (row-major, ld), one CTA;
// a non-positive pivot sets the numeric status bit
__global__ void __launch_bounds__(1024) k_qr_chol(DevState* st, double* G, int s, int ld) {
  __shared__ double piv;
  for (int c = 0; c < s; ++c) {
    if (threadIdx.x == 0) {
      const double v = G[(long long)c * ld + c];
      if (!(v > 0.0)) st->status |= kStNumeric;
      piv = v > 0.0 ? sqrt(v) : 1.0;
      G[(long long)c * ld + c] = piv;
    }
    __syncthreads();
    const double p = piv;
    for (int r = c + 1 + threadIdx.x; r < s; r += blockDim.x) G[(long long)r * ld + c] /= p;
    __syncthreads();
    const int rows = s - c - 1;
    for (long long e = threadIdx.x; e < (long long)rows * rows; e += blockDim.x) {
      const int r = c + 1 + (int)(e / rows), q = c + 1 + (int)(e % rows);
      if (q <= r) G[(long long)r * ld + q] -= G[(long long)r * ld + c] * G[(long long)q * ld + c];
    }
    __syncthreads();
  }
}

// Q_perp <- Q_perp L^{-*} (columns of Q_perp at Qc + (rank + a) M): for each
// row i, forward substitution over the s columns
__global__ void __launch_bounds__(256)
    k_qr_trsm(const double* __restrict__ Lg, int ld, int s, double* Qc, long long M,
              long long rank) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double* q = Qc + rank * M + i;
  for (int a = 0; a < s; ++a) {
    double v = q[(long long)a * M];
    for (int c = 0; c < a; ++c) v -= Lg[(long long)a * ld + c] * q[(long long)c * M];
    q[(long long)a * M] = v / Lg[(long long)a * ld + a];
  }
}

// u_j <- max(u_j - sum_a F(j, rank + a)^2, 0), tile sums
__global__ void __launch_bounds__(kTileRows)
    k_qr_update(const double* __restrict__ F, long long ldF, long long rank, int s, double* u,
                double* tile_sums, long long N) {
  __shared__ double red[8];
  const long long j = (long long)blockIdx.x * kTileRows + threadIdx.x;
  double dn = 0.0;
  if (j < N) {
    double rsq = 0.0;
    for (int a = 0; a < s; ++a) {
      const double g = F[j * ldF + rank + a];
      rsq = fma(g, g, rsq);
    }
    const double v = u[j] - rsq;
    dn = v > 0.0 ? v : 0.0;
    u[j] = dn;
  }
  const double ts = block_sum_fixed(dn, red);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = ts;
}

}  // namespace
}  // namespace rpchol

using namespace rpchol;

struct rpchol_rpqr {
  DevBuffers b{};  // b.N = N columns, b.F = F, b.dvec = u
  cudaStream_t stream = nullptr;
  long long M = 0, k_max = 0;
  double* Bc = nullptr;   // N x M (column j of B at Bc + j M)
  double* Qc = nullptr;   // k_max x M (column a of Q at Qc + a M)
  double* Cg = nullptr;   // T_max x M
  double* Fg = nullptr;   // T_max x ldF
  double* Wm = nullptr;   // k_max x T_max
  double* Gs = nullptr;   // T_max x T_max
  SplitWs ws;             // split-K partials
  DevState* st_host = nullptr;
  std::vector<void*> owned;
  int has_run = 0;
};

namespace {

rpchol_status qr_fail(cudaError_t e, const char* where) {
  set_last_error("%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RPCHOL_ENOMEM : RPCHOL_ECUDA;
}

#define QRCU(call)                                         \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) return qr_fail(e__, #call);    \
  } while (0)

void qr_release(rpchol_rpqr* c) {
  for (void* p : c->owned) cudaFreeAsync(p, c->stream);
  c->owned.clear();
  cudaStreamSynchronize(c->stream);
  if (c->st_host) cudaFreeHost(c->st_host);
  c->st_host = nullptr;
}

rpchol_status qr_status(const DevState& s) {
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

rpchol_status read_st(rpchol_rpqr* c) {
  QRCU(cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevState), cudaMemcpyDeviceToHost,
                       c->stream));
  QRCU(cudaStreamSynchronize(c->stream));
  return RPCHOL_OK;
}

}  // namespace

extern "C" {

rpchol_status rpchol_rpqr_create(const double* B, int64_t M, int64_t N, int64_t ldb,
                                 int64_t k_max, int32_t T_max, void* stream, rpchol_rpqr** out) {
  set_last_error("%s", "");
  if (!out || !B || M < 1 || N < 1 || ldb < M || k_max < 1 || k_max > M || k_max > N ||
      T_max < 1 || T_max > kTMax) {
    set_last_error("invalid argument: M=%lld N=%lld ldb=%lld k_max=%lld T_max=%d", (long long)M,
                   (long long)N, (long long)ldb, (long long)k_max, T_max);
    return RPCHOL_EINVAL;
  }
  *out = nullptr;
  rpchol_rpqr* c = new (std::nothrow) rpchol_rpqr();
  if (!c) return RPCHOL_ENOMEM;
  c->stream = (cudaStream_t)stream;
  c->M = M;
  c->k_max = k_max;
  DevBuffers& b = c->b;
  b.N = N;
  b.d = 1;
  b.ntiles = (N + kTileRows - 1) / kTileRows;
  b.ldF = round_up(k_max, kLdAlign);
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
  auto fail = [&](rpchol_status s) {
    qr_release(c);
    delete c;
    return s;
  };
  cudaError_t e = cudaMallocHost((void**)&c->st_host, sizeof(DevState));
  if (e != cudaSuccess) return fail(qr_fail(e, "cudaMallocHost"));
  memset(c->st_host, 0, sizeof(DevState));
  void* p;
  auto alloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMallocAsync(&q, bytes ? bytes : 16, c->stream) != cudaSuccess) return nullptr;
    c->owned.push_back(q);
    return q;
  };
#define QRALLOC(dst, type, count)                                              \
  do {                                                                         \
    if (!(p = alloc(sizeof(type) * (size_t)(count)))) {                        \
      set_last_error("device allocation failed");                              \
      return fail(RPCHOL_ENOMEM);                                              \
    }                                                                          \
    dst = (type*)p;                                                            \
  } while (0)
  QRALLOC(c->Bc, double, (size_t)N * M);
  QRALLOC(c->Qc, double, (size_t)k_max * M);
  QRALLOC(c->Cg, double, (size_t)kTMax * M);
  QRALLOC(c->Fg, double, (size_t)kTMax * b.ldF);
  QRALLOC(c->Wm, double, (size_t)k_max * kTMax);
  QRALLOC(c->Gs, double, (size_t)kTMax * kTMax);
  // split-K partials: at least 4 splits of the largest Gram-type product
  // (k_max x 256), 64 of a 256 x 256 one
  c->ws.cap = 4 * (long long)k_max * kTMax;
  if (c->ws.cap < 64LL * kTMax * kTMax) c->ws.cap = 64LL * kTMax * kTMax;
  QRALLOC(c->ws.p, double, (size_t)c->ws.cap);
  c->ws.num_sms = b.num_sms;
  double* Fp;
  QRALLOC(Fp, double, (size_t)N * b.ldF);
  b.F = Fp;
  QRALLOC(b.dvec, double, N);
  QRALLOC(b.tile_sums, double, b.ntiles);
  QRALLOC(b.tile_prefix, double,
          b.ntiles * sizeof(double) <= 160 * 1024 ? b.ntiles : b.ntiles * (kTMax / 8));
  QRALLOC(b.piv, long long, k_max);
  QRALLOC(b.prop, int, kTMax);
  QRALLOC(b.uprop, double, kTMax);
  QRALLOC(b.uacc, double, kTMax);
  QRALLOC(b.H, double, (size_t)kTMax * kTMax);
  QRALLOC(b.Lw, double, (size_t)kTMax * kTMax);
  QRALLOC(b.L, double, (size_t)kTMax * T_max);
  QRALLOC(b.Sacc, int, kTMax);
  QRALLOC(b.red, double, b.nred);
  QRALLOC(b.st, DevState, 1);
#undef QRALLOC
  e = cudaMemcpy2DAsync(c->Bc, sizeof(double) * M, B, sizeof(double) * ldb, sizeof(double) * M,
                        N, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.F, 0, sizeof(double) * (size_t)N * b.ldF, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.st, 0, sizeof(DevState), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(qr_fail(e, "create"));
  *out = c;
  return RPCHOL_OK;
}

rpchol_status rpchol_rpqr_run(rpchol_rpqr* c, int64_t k, int32_t T, uint64_t seed) {
  set_last_error("%s", "");
  if (!c || k < 1 || k > c->k_max || T < 1 || T > c->b.Tmax) {
    set_last_error("invalid argument: k=%lld T=%d", (long long)k, T);
    return RPCHOL_EINVAL;
  }
  DevBuffers& b = c->b;
  cudaStream_t s = c->stream;
  const long long M = c->M, N = b.N, ldF = b.ldF;
  const long long max_rounds = 4 * k + 64;
  QRCU(launch_reset(b, k, T, seed, 0u, 0, max_rounds, s));
  k_qr_norms<<<(unsigned)b.ntiles, kTileRows, 0, s>>>(c->Bc, M, N, b.dvec, b.tile_sums);
  QRCU(cudaGetLastError());
  c->has_run = 1;
  long long rank = 0;
  for (long long it = 0; it <= max_rounds; ++it) {
    QRCU(launch_propose(b, T, s));
    k_qr_gather<<<T, 256, 0, s>>>(b.prop, c->Bc, M, (const double*)b.F, ldF, rank, c->Cg, c->Fg,
                                  ldF);
    QRCU(cudaGetLastError());
    // C = B(:,S') - Q F(S',:)^*, stored as rows: Cg(a,i) -= sum_m Fg(a,m) Q(i,m)
    QRCU(dgemm(T, M, rank, -1.0, c->Fg, ldF, 1, c->Qc, M, 1, 1.0, c->Cg, M, 1, s));
    // H = C^* C (ld T)
    QRCU(dgemm(T, T, M, 1.0, c->Cg, M, 1, c->Cg, 1, M, 0.0, b.H, T, 1, s, &c->ws));
    QRCU(launch_reject(b, T, s));
    rpchol_status r = read_st(c);
    if (r != RPCHOL_OK) return r;
    if (c->st_host->done) break;
    const int sa = c->st_host->s;
    if (sa > 0) {
      k_qr_take<<<sa, 256, 0, s>>>(b.st, b.prop, b.Sacc, c->Cg, M, c->Qc, rank);
      QRCU(cudaGetLastError());
      double* Qp = c->Qc + rank * M;
      // second Gram-Schmidt pass against the earlier columns
      QRCU(dgemm(rank, sa, M, 1.0, c->Qc, M, 1, Qp, 1, M, 0.0, c->Wm, kTMax, 1, s, &c->ws));
      QRCU(dgemm(sa, M, rank, -1.0, c->Wm, 1, kTMax, c->Qc, M, 1, 1.0, Qp, M, 1, s));
      // Cholesky QR twice: the thin-QR factor with positive diagonal
      for (int pass = 0; pass < 2; ++pass) {
        QRCU(dgemm(sa, sa, M, 1.0, Qp, M, 1, Qp, 1, M, 0.0, c->Gs, kTMax, 1, s, &c->ws));
        k_qr_chol<<<1, 1024, 0, s>>>(b.st, c->Gs, sa, kTMax);
        QRCU(cudaGetLastError());
        k_qr_trsm<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(c->Gs, kTMax, sa, c->Qc, M, rank);
        QRCU(cudaGetLastError());
      }
      // G = B^* Q_perp into F(:, rank:rank+s)
      QRCU(dgemm(N, sa, M, 1.0, c->Bc, M, 1, Qp, 1, M, 0.0, (double*)b.F + rank, ldF, 1, s));
      k_qr_update<<<(unsigned)b.ntiles, kTileRows, 0, s>>>((const double*)b.F, ldF, rank, sa,
                                                          b.dvec, b.tile_sums, N);
      QRCU(cudaGetLastError());
    }
    QRCU(launch_round_end(b, 0ull, 0, s));
    rank += sa;
    if ((r = read_st(c)) != RPCHOL_OK) return r;
    if (c->st_host->done) break;
  }
  if (read_st(c) != RPCHOL_OK) return RPCHOL_ECUDA;
  return qr_status(*c->st_host);
}

rpchol_status rpchol_rpqr_copy(rpchol_rpqr* c, double* Q_out, int64_t ldq, double* F_out,
                               int64_t ldf, int64_t* pivots_out, double* u_out, int64_t* rank_out,
                               int64_t* rounds_out) {
  if (!c) return RPCHOL_EINVAL;
  rpchol_status r = read_st(c);
  if (r != RPCHOL_OK) return r;
  const long long rank = c->has_run ? c->st_host->rank : 0;
  if ((Q_out && ldq < c->M) || (F_out && ldf < rank)) {
    set_last_error("leading dimension too small");
    return RPCHOL_EINVAL;
  }
  cudaStream_t s = c->stream;
  if (Q_out && rank > 0)
    QRCU(cudaMemcpy2DAsync(Q_out, sizeof(double) * ldq, c->Qc, sizeof(double) * c->M,
                           sizeof(double) * c->M, rank, cudaMemcpyDefault, s));
  if (F_out && rank > 0)
    QRCU(cudaMemcpy2DAsync(F_out, sizeof(double) * ldf, c->b.F, sizeof(double) * c->b.ldF,
                           sizeof(double) * rank, c->b.N, cudaMemcpyDefault, s));
  if (pivots_out && rank > 0)
    QRCU(cudaMemcpyAsync(pivots_out, c->b.piv, sizeof(long long) * rank, cudaMemcpyDefault, s));
  if (u_out)
    QRCU(cudaMemcpyAsync(u_out, c->b.dvec, sizeof(double) * c->b.N, cudaMemcpyDefault, s));
  QRCU(cudaStreamSynchronize(s));
  if (rank_out) *rank_out = rank;
  if (rounds_out) *rounds_out = c->has_run ? c->st_host->round : 0;
  return c->has_run ? qr_status(*c->st_host) : RPCHOL_OK;
}

rpchol_status rpchol_rpqr_destroy(rpchol_rpqr* c) {
  if (!c) return RPCHOL_OK;
  qr_release(c);
  delete c;
  return RPCHOL_OK;
}

}  // extern "C"
