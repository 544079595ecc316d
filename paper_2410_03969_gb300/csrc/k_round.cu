// Round kernels of accelerated RPCholesky (Algorithm 2, arXiv 2410.03969):
// reset, proposal sampler (step 1), residual submatrix H and
// RejectionSampleSubmatrix (step 2, Algorithm 1), round control, and the
// trace-error reduction.
#include <cuda_runtime.h>

#include "internal.h"
#include "round_body.cuh"
#include "selftest.h"

namespace rpchol {

// ------------------------------------------------------------------ reset
__global__ void k_reset(DevState* st, double* dvec, double* tile_sums, long long N,
                        long long ntiles, long long k, int T, unsigned long long seed,
                        unsigned inst, int plain, long long max_rounds) {
  reset_run(st, dvec, tile_sums, N, ntiles, k, T, seed, inst, plain, max_rounds, blockIdx.x,
            gridDim.x);
}

__global__ void k_reset_params(DevState* st, double* dvec, double* tile_sums, long long N,
                               long long ntiles, const RunParams* p) {
  reset_run(st, dvec, tile_sums, N, ntiles, p->k, p->T, p->seed, p->instance, p->plain,
            p->max_rounds, blockIdx.x, gridDim.x);
}

namespace {
unsigned reset_blocks(const DevBuffers& b) {
  long long blocks = (b.N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}
}  // namespace

cudaError_t launch_reset(const DevBuffers& b, long long k, int T, unsigned long long seed,
                         unsigned inst, int plain, long long max_rounds, cudaStream_t s) {
  k_reset<<<reset_blocks(b), 256, 0, s>>>(b.st, b.dvec, b.tile_sums, b.N, b.ntiles, k, T, seed,
                                          inst, plain, max_rounds);
  return cudaGetLastError();
}

cudaError_t add_reset_params_node(cudaGraph_t g, const DevBuffers& b, const RunParams* p,
                                  cudaGraphNode_t* out) {
  DevState* st = b.st;
  double* dvec = b.dvec;
  double* ts = b.tile_sums;
  long long N = b.N, ntiles = b.ntiles;
  void* args[] = {&st, &dvec, &ts, &N, &ntiles, (void*)&p};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_reset_params;
  kp.gridDim = dim3(reset_blocks(b));
  kp.blockDim = dim3(256);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(out, g, nullptr, 0, &kp);
}

// ------------------------------------------------------------------ sampler
__global__ void __launch_bounds__(256) k_propose(DevState* st, const double* __restrict__ dvec,
                                                 const double* __restrict__ tile_sums,
                                                 double* tile_prefix, long long ntiles,
                                                 long long N, int* prop, double* uprop,
                                                 double* uacc, int use_smem, const void* F,
                                                 long long ldF, int f_double) {
  extern __shared__ double pref_smem[];
  __shared__ double wsum[8];
  propose_body(blockIdx.x, pref_smem, wsum, st, dvec, tile_sums, tile_prefix, ntiles, N, prop,
               uprop, uacc, use_smem, F, ldF, f_double);
}

cudaError_t launch_propose(const DevBuffers& b, int T, cudaStream_t s) {
  // the tile prefix lives in shared memory up to 20,480 tiles (N <= 2.6M),
  // otherwise in a global array with one copy per CTA
  const size_t bytes = (size_t)b.ntiles * sizeof(double);
  const int use_smem = bytes <= 160 * 1024 ? 1 : 0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_propose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = (T + 7) / 8;
  k_propose<<<grid, 256, use_smem ? bytes : 0, s>>>(b.st, b.dvec, b.tile_sums, b.tile_prefix,
                                                    b.ntiles, b.N, b.prop, b.uprop, b.uacc,
                                                    use_smem, b.F, b.ldF, b.mixed ? 0 : 1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ H
template <typename TF>
__global__ void __launch_bounds__(256) k_hmat(const DevState* st, const float* __restrict__ X,
                                              int xld, int d, int kind, double inv_sigma,
                                              const TF* __restrict__ F, long long ldF,
                                              const int* __restrict__ prop, double* H,
                                              double* Hpart, int* hcnt) {
  __shared__ TF Fa[16][33];
  __shared__ TF Fb[16][33];
  __shared__ int last;
  hmat_body<TF>(blockIdx.x, blockIdx.y, gridDim.y, Fa, Fb, last, st, X, xld, d, kind, inv_sigma,
                F, ldF, prop, H, Hpart, hcnt);
}

__global__ void __launch_bounds__(256) k_hmat32(const DevState* st, const float* __restrict__ X,
                                                int xld, int d, int kind, double inv_sigma,
                                                const float* __restrict__ F, long long ldF,
                                                const int* __restrict__ prop, double* H,
                                                double* Hpart, int* hcnt) {
  __shared__ H32Smem S;
  hmat32_body(blockIdx.x, blockIdx.y, gridDim.y, S, st, X, xld, d, kind, inv_sigma, F, ldF, prop,
              H, Hpart, hcnt);
}

cudaError_t launch_hmat(const DevBuffers& b, int T, cudaStream_t s) {
  if (b.mixed) {
    const int nblk = hmat32_blocks(T);
    k_hmat32<<<dim3(nblk, hmat32_splits(nblk)), 256, 0, s>>>(
        b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma, (const float*)b.F, b.ldF, b.prop, b.H,
        b.Hpart, b.hcnt);
  } else {
    const int nb = (T + 15) / 16;
    const int ntile = nb * (nb + 1) / 2;
    const int ks = hmat_splits(ntile, b.num_sms);
    k_hmat<double><<<dim3(ntile, ks), 256, 0, s>>>(b.st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                                                   (const double*)b.F, b.ldF, b.prop, b.H,
                                                   b.Hpart, b.hcnt);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Algorithm 1
__global__ void __cluster_dims__(kRejCluster, 1, 1) __launch_bounds__(kRejectThreads)
    k_reject(DevState* st, const double* __restrict__ H, const double* __restrict__ uprop,
             const double* __restrict__ uacc, const int* __restrict__ prop, double* Lw, double* L,
             int ldL, int* Sacc, long long* piv, int fp64) {
  extern __shared__ double Hown[];  // packed rows owned by this CTA (CTAs 1..)
  __shared__ RejSmem R;
  reject_body(R, Hown, st, H, uprop, uacc, prop, Lw, L, ldL, Sacc, piv, fp64);
}

// Failure-detection self-test: one thread waits, with the cluster-scope
// bounded wait of Algorithm 1, on a barrier that nothing completes; the wait
// must give up after limit_ns.  out[0] = 1 if it gave up, out[1] = the time
// it waited (ns).
__global__ void k_wait_selftest_cluster(unsigned long long limit_ns, unsigned long long* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(&bar))
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const bool ok = wait_cluster_bounded(&bar, 0u, limit_ns);
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  out[0] = ok ? 0ull : 1ull;
  out[1] = t1 - t0;
}

cudaError_t launch_wait_selftest_cluster(unsigned long long limit_ns, unsigned long long* out,
                                         cudaStream_t s) {
  k_wait_selftest_cluster<<<1, 32, 0, s>>>(limit_ns, out);
  return cudaGetLastError();
}

cudaError_t launch_reject(const DevBuffers& b, int T, cudaStream_t s) {
  const size_t dyn = reject_own_doubles(T) * sizeof(double);
  // static and dynamic shared memory together pass the 48 KiB default for
  // T above about 200: opt in for whatever this launch needs
  static size_t attr = 0;
  if (dyn > attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_reject, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    attr = dyn;
  }
  k_reject<<<kRejCluster, kRejectThreads, dyn, s>>>(b.st, b.H, b.uprop, b.uacc, b.prop, b.Lw,
                                                    b.L, b.Tmax, b.Sacc, b.piv, b.mixed ? 0 : 1);
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
  round_end_body(st, (unsigned long long)cond, use_cond, N, d, bF);
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
