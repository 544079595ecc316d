// Tensor-core column step of accelerated RPCholesky in mixed precision
// (Algorithm 2, step 3, arXiv 2410.03969), sm_103a:
//
//   D1 = X_tile X_S^*            (fast Euclidean distances, App. A.1)
//   D2 = F_tile F(S,:)^*         (Schur complement contraction)
//   R  = kappa(||x||^2 + ||x_S||^2 - 2 D1) - D2
//   G  = R L^{-*}                (L^{-1} formed in FP64 per round, applied in FP32)
//   F(tile, rank:rank+s) = G;  d <- max(d - rowsumsq(G), 0) (FP64);  tile sums of d.
//
// Both contractions run on tcgen05.mma kind::tf32 with FP32 accumulation in
// TMEM, as three-term compensated products a_hi b_hi + a_hi b_lo + a_lo b_hi
// where hi is the TF32 head of an fp32 value and lo = value - hi (exact);
// this recovers ~fp32 accuracy and with it the cancellation in
// ||x||^2 + ||y||^2 - 2 x.y and in A - F F^*.
//
// One CTA owns a 128-row tile (one sampler tile) and all s <= 256 new
// columns.  Warp roles: warp 0 issues TMA loads (one elected lane), warp 1
// owns TMEM and issues the MMAs (one elected lane), warps 2-5 split the
// fp32 F tile into TF32 head/tail while the mainloop runs and then do the
// epilogue, one TMEM lane (= one row) per thread.  Operands stream through
// a two-stage shared-memory ring: per stage a 128 x 32 A tile (head, tail)
// and an s_pad x 32 B tile (head, tail), 128-byte swizzled, K-major.  The
// distance chunks (K = padded d) come first, then ceil(rank/32) F chunks.
// Every wait is bounded: on expiry the CTA raises an error bit, drains its
// own copies and frees its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

namespace {
constexpr int kTcThreads = 192;
constexpr int kBM = 128;
constexpr int kStageA = kBM * 32 * 4;        // 16 KiB
constexpr int kStageB = 256 * 32 * 4;        // 32 KiB (s_pad <= 256 rows)
constexpr int kStageBytes = 2 * kStageA + 2 * kStageB;
constexpr int kStages = 2;
constexpr int kBarOff = kStages * kStageBytes;  // 196608
constexpr int kSmemBytes = kBarOff + 256 + 1024;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
}  // namespace

struct TcArgs {
  const DevState* st;
  float* F;
  long long ldF;
  long long N;
  const float* nrm;     // ||x||^2, FP32
  const float* nrmS;    // ||x_{S_j}||^2
  const int* Sacc;      // accepted pivots of the round
  const float* Linv;    // L^{-1} of the round, FP32, row-major, leading dimension 256
  double* dvec;
  double* tile_sums;
  int* err;             // device status word (kStTimeout bit)
  int kind;
  float inv_sigma;
  int xld;
  const double* L;      // compact FP64 Cholesky factor of the round
  int ldL;
};

__global__ void __launch_bounds__(kTcThreads, 1)
    k_colstep_tc(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmX,
                 const __grid_constant__ CUtensorMap tmXlo,
                 const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                 const __grid_constant__ CUtensorMap tmXSh,
                 const __grid_constant__ CUtensorMap tmXSl, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + kBarOff);        // [2] TMA landed
  uint64_t* conv = full + 2;                          // [2] tail of A written
  uint64_t* empty = full + 4;                         // [2] MMAs done with the stage
  uint64_t* accf = full + 6;                          // accumulators complete
  uint32_t* tptr = (uint32_t*)(sm + kBarOff + 64);
  volatile int* abort_flag = (volatile int*)(sm + kBarOff + 128);
  double* red = (double*)(sm + kBarOff + 136);        // [4] tile-sum partials

  const DevState* st = a.st;
  if (st->done) return;
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const int s_pad = (s + 15) & ~15;
  const int nbox = (s_pad + 63) >> 6;
  const int nX = a.xld >> 5;
  const int nF = (int)((rank + 31) >> 5);
  const int nch = nX + nF;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long row0 = (long long)blockIdx.x * kBM;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&conv[i], 128);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(accf, 1);
    *abort_flag = 0;
    tc::fence_mbarrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tptr, 512);
    tc::tmem_relinquish();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tptr;
  const unsigned long long deadline = tc::globaltimer_ns() + kWaitNs;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tmap(&tmF);
      const uint32_t bbytes = (uint32_t)nbox * 64u * 128u;
      int c = 0;
      for (; c < nch; ++c) {
        const int stg = c & 1;
        if (c >= 2 && !tc::mbar_wait_bounded(&empty[stg], ((c >> 1) - 1) & 1, deadline,
                                              abort_flag))
          break;
        unsigned char* base = sm + stg * kStageBytes;
        unsigned char* sA = base;
        unsigned char* sAlo = base + kStageA;
        unsigned char* sBh = base + 2 * kStageA;
        unsigned char* sBl = sBh + kStageB;
        if (c < nX) {
          const int x = c * 32;
          tc::mbar_arrive_expect_tx(&full[stg], 2u * kStageA + 2u * bbytes);
          tc::tma_load_2d(sA, &tmX, x, (int)row0, &full[stg]);
          tc::tma_load_2d(sAlo, &tmXlo, x, (int)row0, &full[stg]);
          for (int b = 0; b < nbox; ++b) {
            tc::tma_load_2d(sBh + b * 8192, &tmXSh, x, 64 * b, &full[stg]);
            tc::tma_load_2d(sBl + b * 8192, &tmXSl, x, 64 * b, &full[stg]);
          }
        } else {
          // F chunks from the last to the first: the tensor core's FP32
          // accumulation truncates, and the factor's columns shrink with
          // their index, so adding the small late columns first and the
          // large early ones last keeps the accumulated rounding at the
          // level of FP32 FMA accumulation.
          const int x = (nF - 1 - (c - nX)) * 32;
          tc::mbar_arrive_expect_tx(&full[stg], (uint32_t)kStageA + 2u * bbytes);
          tc::tma_load_2d(sA, &tmF, x, (int)row0, &full[stg]);
          for (int b = 0; b < nbox; ++b) {
            tc::tma_load_2d(sBh + b * 8192, &tmBh, x, 64 * b, &full[stg]);
            tc::tma_load_2d(sBl + b * 8192, &tmBl, x, 64 * b, &full[stg]);
          }
        }
      }
      if (*abort_flag) {
        // drain: every issued load must land before the CTA may exit
        const unsigned long long d2 = tc::globaltimer_ns() + kWaitNs;
        volatile int dummy = 0;
        for (int q = (c > 2 ? c - 2 : 0); q < c; ++q)
          tc::mbar_wait_bounded(&full[q & 1], (q >> 1) & 1, d2, &dummy);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)s_pad);
      const uint32_t d1 = tbase;        // columns [0, 256)
      const uint32_t d2 = tbase + 256;  // columns [256, 512)
      for (int c = 0; c < nch; ++c) {
        const int stg = c & 1;
        if (!tc::mbar_wait_bounded(&conv[stg], (c >> 1) & 1, deadline, abort_flag)) break;
        tc::tc_fence_after();
        unsigned char* base = sm + stg * kStageBytes;
        const uint32_t aA = tc::smem_u32(base);
        const uint32_t aAlo = aA + kStageA;
        const uint32_t aBh = aA + 2 * kStageA;
        const uint32_t aBl = aBh + kStageB;
        const bool isX = c < nX;
        const uint32_t dt = isX ? d1 : d2;
        const bool first = (c == 0) || (c == nX);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t da = tc::smem_desc_sw128(aA + 32 * kk);
          const uint64_t dal = tc::smem_desc_sw128(aAlo + 32 * kk);
          const uint64_t dbh = tc::smem_desc_sw128(aBh + 32 * kk);
          const uint64_t dbl = tc::smem_desc_sw128(aBl + 32 * kk);
          tc::mma_tf32(dt, da, dbh, idesc, (first && kk == 0) ? 0u : 1u);
          tc::mma_tf32(dt, da, dbl, idesc, 1u);
          tc::mma_tf32(dt, dal, dbh, idesc, 1u);
        }
        tc::mma_commit(&empty[stg]);
      }
      tc::mma_commit(accf);
    }
  } else {
    // ------------------------------------------------ converter, then epilogue
    const int e = threadIdx.x - 64;  // 0..127
    for (int c = 0; c < nch; ++c) {
      const int stg = c & 1;
      if (!tc::mbar_wait_bounded(&full[stg], (c >> 1) & 1, deadline, abort_flag)) break;
      if (c >= nX) {
        // row e of the A tile: split the fp32 F values into TF32 head (in
        // place) and tail; the swizzle permutes 16-byte chunks within a row
        // only, so a row's 128 bytes are processed in place in any order.
        float4* pa = (float4*)(sm + stg * kStageBytes + e * 128);
        float4* pl = (float4*)(sm + stg * kStageBytes + kStageA + e * 128);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = (q + e) & 7;
          float4 v = pa[j];
          float4 h = make_float4(tc::tf32_head(v.x), tc::tf32_head(v.y), tc::tf32_head(v.z),
                                 tc::tf32_head(v.w));
          pa[j] = h;
          pl[j] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
        tc::fence_proxy_async_smem();
      }
      tc::mbar_arrive(&conv[stg]);
    }
  }

  // ------------------------------------------------ epilogue (warps 2-5)
  if (warp >= 2) {
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int row = q * 32 + lane;           // tile row = TMEM lane
    const long long grow = row0 + row;
    // a timed-out wait raises abort_flag before the barrier; once every
    // epilogue thread has seen the accumulators complete, the producer and
    // the MMA issuer have finished, so one thread's reading is everyone's
    tc::mbar_wait_bounded(accf, 0, deadline, abort_flag);
    volatile int* go_flag = (volatile int*)(sm + kBarOff + 132);
    asm volatile("bar.sync 1, 128;" ::: "memory");  // bar 1: the 128 epilogue threads
    if (threadIdx.x == 64) *go_flag = *abort_flag ? 0 : 1;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (*go_flag) {
      tc::tc_fence_after();
      // R tile and staged L^{-1} block reuse the (now idle) stage buffers
      const int ldR = s_pad + 1;
      float* Rt = (float*)sm;
      float* LT = (float*)(sm + 128 * 260 * 4);   // [l][16]
      const float nr = grow < a.N ? a.nrm[grow] : 0.f;
      int jpiv = -1;  // index of this row among the round's pivots, if it is one
      const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < s_pad; c0 += 16) {
        float v1[16], v2[16];
        tc::tmem_ld16_sync(tl + c0, v1);
        if (nF > 0) tc::tmem_ld16_sync(tl + 256 + c0, v2);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          float r = 0.f;
          if (c < s) {
            const int p = a.Sacc[c];
            float kv = 1.f;
            if ((long long)p == grow) {
              jpiv = c;
            } else {
              const float d2 = nr + a.nrmS[c] - 2.f * v1[j];
              kv = phi_r2<float>(a.kind, a.inv_sigma, d2);
            }
            r = kv - (nF > 0 ? v2[j] : 0.f);
          }
          Rt[row * ldR + c] = r;
        }
      }
      tc::tc_fence_before();
      // G = R L^{-*}: G(r, j) = sum_{l <= j} R(r, l) Linv(j, l), blocks of 16
      // columns from the last block down so that G overwrites R in place.
      float rsq = 0.f, rc = 0.f;  // Kahan-compensated sum of G^2
      const int nblk = (s + 15) >> 4;
      for (int bi = nblk - 1; bi >= 0; --bi) {
        const int j0 = bi * 16;
        const int lmax = min(j0 + 16, s);
        asm volatile("bar.sync 1, 128;" ::: "memory");
        for (int idx = threadIdx.x - 64; idx < lmax * 16; idx += 128) {
          const int l = idx >> 4, jj = idx & 15;
          LT[idx] = (j0 + jj < s) ? a.Linv[(long long)(j0 + jj) * 256 + l] : 0.f;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        float acc[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.f;
        const float* rrow = Rt + row * ldR;
        for (int l = 0; l < lmax; ++l) {
          const float rv = rrow[l];
          const float4* lt = (const float4*)(LT + l * 16);
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const float4 w = lt[g];
            acc[4 * g + 0] = fmaf(rv, w.x, acc[4 * g + 0]);
            acc[4 * g + 1] = fmaf(rv, w.y, acc[4 * g + 1]);
            acc[4 * g + 2] = fmaf(rv, w.z, acc[4 * g + 2]);
            acc[4 * g + 3] = fmaf(rv, w.w, acc[4 * g + 3]);
          }
        }
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          if (j0 + jj < s) {
            const float gv = acc[jj];
            Rt[row * ldR + j0 + jj] = gv;
            const float y = gv * gv - rc;
            const float t = rsq + y;
            rc = (t - rsq) - y;
            rsq = t;
          }
        }
      }
      // A pivot row of this round: in exact arithmetic R(S,:) = H(S,S) = L L^*,
      // so G(S_j,:) = L(j,:) and its residual is zero.  Write those exact
      // values (L from the FP64 Cholesky of H) instead of the rounded
      // contraction, so that a chosen pivot keeps zero proposal weight and
      // its row of F agrees with the H that later rounds form from it.
      if (jpiv >= 0) {
        for (int l = 0; l < s; ++l)
          Rt[row * ldR + l] = l <= jpiv ? (float)a.L[(long long)jpiv * a.ldL + l] : 0.f;
      }
      // residual diagonal (FP64) and the tile's sum of d
      double dn = 0.0;
      if (grow < a.N) {
        const double v = a.dvec[grow] - ((double)rsq - (double)rc);
        dn = (v > 0.0 && jpiv < 0) ? v : 0.0;
        a.dvec[grow] = dn;
      }
      double t = dn;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) red[q] = t;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (threadIdx.x == 64) a.tile_sums[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
      // write G (128 x s) to F(tile, rank : rank + s), rows by warp, columns by lane
      for (int r = q; r < kBM; r += 4) {
        const long long gr = row0 + r;
        if (gr >= a.N) break;
        float* dst = a.F + gr * a.ldF + rank;
        const float* src = Rt + r * ldR;
        for (int j = lane; j < s; j += 32) dst[j] = src[j];
      }
    } else if (threadIdx.x == 64) {
      atomicOr(a.err, (int)kStTimeout);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

cudaError_t launch_colstep_tc(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_colstep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcArgs a;
  a.st = b.st;
  a.F = (float*)b.F;
  a.ldF = b.ldF;
  a.N = b.N;
  a.nrm = b.nrm;
  a.nrmS = m.nrmS;
  a.Sacc = b.Sacc;
  a.Linv = m.Linv32;
  a.dvec = b.dvec;
  a.tile_sums = b.tile_sums;
  a.err = m.err;
  a.kind = b.kind;
  a.inv_sigma = (float)(1.0 / b.sigma);
  a.xld = b.xld;
  a.L = b.L;
  a.ldL = b.Tmax;
  const unsigned grid = (unsigned)((b.N + kBM - 1) / kBM);
  k_colstep_tc<<<grid, kTcThreads, kSmemBytes, s>>>(m.F, m.X, m.Xlo, m.FSh, m.FSl, m.XSh, m.XSl,
                                                    a);
  return cudaGetLastError();
}

}  // namespace rpchol
