// Device-side building blocks shared by the rpchol kernels (sm_103a).
//
// Paper: Epperly, Tropp, Webber, arXiv 2410.03969.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rpchol {

// Rows per tile of the residual-diagonal partial sums that the sampler
// scans; every kernel that rewrites d also rewrites the sums of the tiles
// it owns, in a fixed order.
constexpr int kTileRows = 128;
// Largest block size T (Algorithm 2's b).
constexpr int kTMax = 256;
// Residual weights at or below the floor (relative to the kernels' unit
// diagonal) are rounding noise on an exhausted row and are set to 0 with the
// clamp d <- max(d, 0).  Without it a numerically rank-deficient kernel
// matrix keeps a few weights at the noise level whose recomputed Schur
// diagonals are far smaller, so Algorithm 1 rejects them round after round
// and the run never reaches its rank.  FP64 mode uses the oracle's floor; the
// FP32 factor of mixed mode leaves noise near 1e-7 in d.
constexpr double kDFloor64 = 1e-12;
constexpr double kDFloorMixed = 4e-6;
template <typename TF>
__host__ __device__ __forceinline__ constexpr double d_floor() {
  return sizeof(TF) == 8 ? kDFloor64 : kDFloorMixed;
}
// most ways the rank dimension of H = A(S',S') - F(S',:)F(S',:)^* is split
constexpr int kHSplitMax = 8;
constexpr int kHTilesMax = (kTMax / 16) * (kTMax / 16 + 1) / 2;
constexpr int kH32BlocksMax = (kTMax / 32) * (kTMax / 32 + 1) / 2;
// partial products of H: 16 x 16 tiles (FP64 factor) or 32 x 32 blocks (FP32 factor)
constexpr long long kHPartDoubles =
    (long long)kHTilesMax * (kHSplitMax + 1) * 256 > (long long)kH32BlocksMax * (kHSplitMax + 1) * 1024
        ? (long long)kHTilesMax * (kHSplitMax + 1) * 256
        : (long long)kH32BlocksMax * (kHSplitMax + 1) * 1024;
// Leading dimensions are padded to this many elements.
constexpr int kLdAlign = 32;

enum StatusBits : int {
  kStRoundLimit = 1,   // round limit reached before rank k
  kStNumeric = 2,      // non-finite / non-positive pivot
  kStTimeout = 4,      // a bounded device-side wait expired
  kStGateExpired = 8,  // profile mode: the stream gate gave up waiting for the host
};

// Run state, one per context, in device memory.  Written only by
// single-thread control sections of the round kernels.
struct DevState {
  long long rank;        // columns of F filled
  long long round;       // rounds (or simple steps) completed
  long long k;           // target rank of this run
  long long max_rounds;  // round limit
  long long proposals;   // pivots proposed so far
  int T;                 // proposals per round
  int s;                 // pivots accepted in the current round
  int done;              // 1 once the run has stopped
  int status;            // StatusBits
  int plain;             // 1 for simple RPCholesky
  int block;             // 1 for block RPCholesky (Algorithm 7): Algorithm 1 accepts every
                         // first draw of an index whose Schur residual is positive
  unsigned long long seed;
  unsigned int instance;
  unsigned int pad1;
  double W;              // total proposal weight of the current round
  double gs;             // simple RPCholesky: g_s of the current step
  long long piv;         // simple RPCholesky: pivot of the current step
  double col_bytes;      // algorithmic bytes of the column-step kernels so far
  double col_flops;      // algorithmic flops of the column-step kernels so far
  double mma_tf32;       // tensor-core flops the column steps executed, kind::tf32
  double mma_f16;        // tensor-core flops the column steps executed, kind::f16
};

// Parameters of one run, read by the reset kernel of a batched launch (so
// that one recorded graph serves every run of the batch).
struct RunParams {
  long long k;           // target rank
  long long max_rounds;  // round limit
  unsigned long long seed;
  int T;                 // proposals per round
  int plain;             // 1: simple RPCholesky, 2: block RPCholesky, 0: accelerated
  unsigned instance;     // Philox counter word 3
  int pad;
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)), the key advancing by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// 53-bit uniform in [0, 1 - 2^-53] from two words (27 + 26 bits).
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const unsigned long long v =
      (unsigned long long)(a >> 5) * 67108864ull + (unsigned long long)(b >> 6);
  return (double)v * (1.0 / 9007199254740992.0);
}

// Proposal and acceptance uniforms of slot `slot`, round `round`.
__device__ __forceinline__ void uniforms(unsigned long long seed, uint32_t slot, uint32_t round,
                                         uint32_t inst, double* up, double* ua) {
  const uint4 w = philox4x32_10(make_uint4(slot, round, 0u, inst), (uint32_t)(seed & 0xFFFFFFFFull),
                                (uint32_t)(seed >> 32));
  *up = u53(w.x, w.y);
  *ua = u53(w.z, w.w);
}

// ---------------------------------------------------------------- kernels
// kappa(x,y) = phi(r), r^2 = ||x-y||^2.  phi(0) = 1.
template <typename Real>
__device__ __forceinline__ Real phi_r2(int kind, Real inv_sigma, Real r2);

template <>
__device__ __forceinline__ double phi_r2<double>(int kind, double inv_sigma, double r2) {
  r2 = r2 > 0.0 ? r2 : 0.0;
  if (kind == 0) return exp(-0.5 * r2 * inv_sigma * inv_sigma);
  if (kind == 4) return exp(-r2 * inv_sigma);  // r2 holds the l1 distance
  const double r = sqrt(r2);
  if (kind == 1) return exp(-r * inv_sigma);
  if (kind == 3) {
    const double t = 1.7320508075688772935 * r * inv_sigma;  // sqrt(3) r / sigma
    return (1.0 + t) * exp(-t);
  }
  const double t = 2.2360679774997896964 * r * inv_sigma;  // sqrt(5) r / sigma
  return (1.0 + t + t * t * (1.0 / 3.0)) * exp(-t);
}

template <>
__device__ __forceinline__ float phi_r2<float>(int kind, float inv_sigma, float r2) {
  r2 = r2 > 0.f ? r2 : 0.f;
  if (kind == 0) return expf(-0.5f * r2 * inv_sigma * inv_sigma);
  if (kind == 4) return expf(-r2 * inv_sigma);  // r2 holds the l1 distance
  const float r = sqrtf(r2);
  if (kind == 1) return expf(-r * inv_sigma);
  if (kind == 3) {
    const float t = 1.7320508075688772f * r * inv_sigma;
    return (1.f + t) * expf(-t);
  }
  const float t = 2.2360679774997897f * r * inv_sigma;
  return (1.f + t + t * t * (1.f / 3.f)) * expf(-t);
}

// One coordinate's share of the distance the kernel map takes: t^2 (the
// Euclidean kernels take r^2) or |t| (the l1-Laplace takes the l1 distance).
template <typename Real>
__device__ __forceinline__ Real dist_term(int kind, Real t) {
  return kind == 4 ? (t < (Real)0 ? -t : t) : t * t;
}

// Accumulation type and 16-byte vector of a factor element type: FP32
// factors (mixed mode) accumulate in FP32, FP64 factors in FP64.
template <typename TF>
struct FVec;
template <>
struct FVec<float> {
  using V = float4;
  using A = float;
  static constexpr int E = 4;
  __device__ static float dot(const float4 a, const float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
  }
};
template <>
struct FVec<double> {
  using V = double2;
  using A = double;
  static constexpr int E = 2;
  __device__ static double dot(const double2 a, const double2 b, double acc) {
    acc = fma(a.x, b.x, acc);
    return fma(a.y, b.y, acc);
  }
};

// Dot products of R rows of a factor (16-byte aligned) with the vector v
// over n elements, by one warp: lanes stride over 16-byte vectors (the R
// rows' loads are independent), then the tail element by element, then a
// butterfly reduction.  The results are valid in every lane.
template <typename TF, int R>
__device__ __forceinline__ void warp_rows_dot(const TF* const (&rows)[R], const TF* v,
                                              long long n, int lane,
                                              typename FVec<TF>::A (&acc)[R]) {
  using V = typename FVec<TF>::V;
  constexpr int E = FVec<TF>::E;
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0;
  const long long nv = n / E;
  const V* vv = (const V*)v;
  for (long long m = lane; m < nv; m += 32) {
    const V b = vv[m];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = FVec<TF>::dot(((const V*)rows[r])[m], b, acc[r]);
  }
  for (long long m = nv * E + lane; m < n; m += 32) {
    const TF b = v[m];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += rows[r][m] * b;
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

__host__ __device__ __forceinline__ long long round_up(long long a, long long b) {
  return (a + b - 1) / b * b;
}

// The round bodies written for 256 threads (sampler, H, W blocks) use this
// barrier instead of __syncthreads: in their own 256-thread kernels it spans
// the CTA; inside a larger persistent CTA only its first 256 threads run
// them and take part.
constexpr int kBodyThreads = 256;
__device__ __forceinline__ void body_sync() { asm volatile("bar.sync 8, 256;" ::: "memory"); }

// Fixed-order block reduction of one double per thread (blockDim.x threads,
// a multiple of 32).  Result valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double* red_smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red_smem[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) t += red_smem[w];
  }
  __syncthreads();
  return t;
}

}  // namespace rpchol
