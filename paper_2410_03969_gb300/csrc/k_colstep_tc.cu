// Tensor-core column step of accelerated RPCholesky in mixed precision
// (Algorithm 2, step 3, arXiv 2410.03969), sm_103a:
//
//   D1 = X_tile X_S^*            (fast Euclidean distances, App. A.1)
//   D2 = F_tile F(S,:)^*         (Schur complement contraction)
//   R  = kappa(||x||^2 + ||x_S||^2 - 2 D1) - D2
//   G L^* = R                    (forward substitution in FP32 with the FP64 L
//                                 of Algorithm 1 rounded once)
//   F(tile, rank:rank+s) = G;  d <- max(d - rowsumsq(G), 0) (FP64);  tile sums of d.
//
// Both contractions run on tcgen05.mma kind::tf32 with FP32 accumulation in
// TMEM, as three-term compensated products a_hi b_hi + a_hi b_lo + a_lo b_hi
// where hi is the TF32 head of an fp32 value (rounded to nearest) and
// lo = value - hi (exact); this recovers ~fp32 accuracy and with it the
// cancellation in ||x||^2 + ||y||^2 - 2 x.y and in A - F F^*.  The tensor
// core's FP32 accumulation truncates, so the F chunks stream from the last
// column to the first: the small late columns are added first, the large
// early ones last.
//
// Persistent kernel: one CTA per SM loops over 128-row tiles (one sampler
// tile each).  Warp roles (384 threads):
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM owner and MMA issuer (one elected lane)
//   warps 2-3   split each fp32 F tile into TF32 head (in place) and tail
//   warps 4-11  epilogue, two warps per TMEM lane quarter: the two threads of
//               a tile row (= TMEM lane) split its columns
// Operands stream through a two-stage shared-memory ring: per stage a
// 128 x 32 A tile (head, tail) and an s_pad x 32 B tile (head, tail),
// 128-byte swizzled, K-major.  The epilogue first drains both accumulators
// into an R tile in shared memory and releases TMEM, so the next tile's
// mainloop runs while this tile's substitution and write-out proceed
// (s_pad <= 128; for larger s the R tile reuses the stage buffers and the
// producer waits for the epilogue).  Every wait is bounded: on expiry the
// CTA raises the timeout bit of the run status, drains its own copies and
// frees its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

namespace {
constexpr int kTcThreads = 384;
constexpr int kBM = 128;
constexpr int kStageA = kBM * 32 * 4;  // 16 KiB
constexpr int kSmemMax = 227 * 1024;
constexpr int kSmallBytes = 4 * 1024;  // Sacc, nrmS copies, per-row scratch, barriers
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

struct Layout {
  int s_pad, nbox, stage_bytes, overlap;
  int rt_off, lt_off, small_off, total;
};

__host__ __device__ inline Layout make_layout(int s) {
  Layout L;
  L.s_pad = (s + 15) & ~15;
  L.nbox = (L.s_pad + 63) >> 6;
  L.stage_bytes = 2 * kStageA + 2 * L.nbox * 8192;
  const int stages = 2 * L.stage_bytes;
  const int rt = kBM * (L.s_pad + 1) * 4;
  const int lt = 2 * 16 * 1024;  // W blocks: two 16 KiB buffers (or all of W when it fits)
  L.overlap = (stages + rt + lt + kSmallBytes + 1024) <= kSmemMax ? 1 : 0;
  if (L.overlap) {
    L.rt_off = stages;
    L.lt_off = stages + rt;
    L.small_off = L.lt_off + lt;
  } else {
    L.rt_off = 0;
    L.lt_off = kBM * 260 * 4;  // after the largest R tile
    L.small_off = 2 * (2 * kStageA + 2 * 4 * 8192);
  }
  L.total = L.small_off + kSmallBytes + 1024;
  return L;
}
}  // namespace

struct TcArgs {
  const DevState* st;
  float* F;
  long long ldF;
  long long N;
  const float* nrm;     // ||x||^2, FP32
  const float* nrmS;    // ||x_{S_j}||^2
  const int* Sacc;      // accepted pivots of the round
  const float* W;       // blocked-substitution operand of the round (k_wblk)
  double* dvec;
  double* tile_sums;
  int* err;             // run status word
  int kind;
  float inv_sigma;
  int xld;
  const double* L;      // compact FP64 Cholesky factor of the round
  int ldL;
};

template <int KIND>  // kernel map, specialised so the epilogue has one code path
__global__ void __launch_bounds__(kTcThreads, 1)
    k_colstep_tc(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmX,
                 const __grid_constant__ CUtensorMap tmXlo,
                 const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                 const __grid_constant__ CUtensorMap tmXSh,
                 const __grid_constant__ CUtensorMap tmXSl, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const DevState* st = a.st;
  if (st->done) return;
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const Layout Lo = make_layout(s);
  const int s_pad = Lo.s_pad, nbox = Lo.nbox, SB = Lo.stage_bytes;
  const int nX = a.xld >> 5;
  const int nF = (int)((rank + 31) >> 5);
  const int nch = nX + nF;
  const long long ntiles = (a.N + kBM - 1) / kBM;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  unsigned char* small = sm + Lo.small_off;
  int* Ss = (int*)small;                  // [256] pivots of the round
  float* nrmSs = (float*)(small + 1024);  // [256] their squared norms
  int* jps = (int*)(small + 2048);        // [128] pivot index found by the second half
  float* rss = (float*)(small + 2560);    // [128] second half's sum of squares
  float* rcs = (float*)(small + 3072);    // [128] and its compensation
  uint64_t* full = (uint64_t*)(small + 3584);  // [2]
  uint64_t* conv = full + 2;                   // [2]
  uint64_t* empty = full + 4;                  // [2]
  uint64_t* accf = full + 6;                   // accumulators of a tile complete
  uint64_t* tfree = full + 7;                  // epilogue drained TMEM
  uint64_t* edone = full + 8;                  // epilogue done with shared memory
  uint32_t* tptr = (uint32_t*)(small + 3584 + 80);
  volatile int* abort_flag = (volatile int*)(small + 3584 + 84);
  volatile int* go_flag = (volatile int*)(small + 3584 + 88);
  double* red = (double*)(small + 3584 + 96);  // [4]
  float* Rt = (float*)(sm + Lo.rt_off);
  float* Wsm = (float*)(sm + Lo.lt_off);  // W of the round, whole or two 16 KiB blocks
  const int nblk_all = (s + 15) >> 4;
  // resident only when it has its own region (overlap layout) and fits 32 KiB
  const bool w_resident = Lo.overlap && 128 * nblk_all * (nblk_all + 1) <= 8192;
  const int ldR = s_pad + 1;

  for (int i = threadIdx.x; i < s_pad; i += kTcThreads) {
    Ss[i] = i < s ? a.Sacc[i] : -1;
    nrmSs[i] = i < s ? a.nrmS[i] : 0.f;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&conv[i], 2);   // one arrival per converter warp
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(accf, 1);
    tc::mbar_init(tfree, 8);        // one arrival per epilogue warp
    tc::mbar_init(edone, 8);
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

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tmap(&tmF);
      const uint32_t bbytes = (uint32_t)nbox * 8192u;
      long long g = 0;  // chunks issued so far (all tiles)
      int it = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
        if (!Lo.overlap && it > 0 &&
            !tc::mbar_wait_bounded(edone, (it - 1) & 1, tc::globaltimer_ns() + kWaitNs,
                                   abort_flag))
          break;
        const int row0 = (int)(tile * kBM);
        for (int c = 0; c < nch; ++c, ++g) {
          const int stg = (int)(g & 1);
          if (g >= 2 && !tc::mbar_wait_bounded(&empty[stg], (uint32_t)(((g >> 1) - 1) & 1),
                                               tc::globaltimer_ns() + kWaitNs, abort_flag))
            break;
          unsigned char* sA = sm + stg * SB;
          unsigned char* sAlo = sA + kStageA;
          unsigned char* sBh = sA + 2 * kStageA;
          unsigned char* sBl = sBh + nbox * 8192;
          if (c < nX) {
            const int x = c * 32;
            tc::mbar_arrive_expect_tx(&full[stg], 2u * kStageA + 2u * bbytes);
            tc::tma_load_2d(sA, &tmX, x, row0, &full[stg]);
            tc::tma_load_2d(sAlo, &tmXlo, x, row0, &full[stg]);
            for (int b = 0; b < nbox; ++b) {
              tc::tma_load_2d(sBh + b * 8192, &tmXSh, x, 64 * b, &full[stg]);
              tc::tma_load_2d(sBl + b * 8192, &tmXSl, x, 64 * b, &full[stg]);
            }
          } else {
            const int x = (nF - 1 - (c - nX)) * 32;  // last F column chunk first
            tc::mbar_arrive_expect_tx(&full[stg], (uint32_t)kStageA + 2u * bbytes);
            tc::tma_load_2d(sA, &tmF, x, row0, &full[stg]);
            for (int b = 0; b < nbox; ++b) {
              tc::tma_load_2d(sBh + b * 8192, &tmBh, x, 64 * b, &full[stg]);
              tc::tma_load_2d(sBl + b * 8192, &tmBl, x, 64 * b, &full[stg]);
            }
          }
        }
      }
      if (*abort_flag) {
        // drain: the (at most two) issued loads not yet consumed must land
        volatile int dummy = 0;
        const unsigned long long d2 = tc::globaltimer_ns() + kWaitNs;
        for (long long q = (g > 2 ? g - 2 : 0); q < g; ++q)
          tc::mbar_wait_bounded(&full[q & 1], (uint32_t)((q >> 1) & 1), d2, &dummy);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)s_pad);
      const uint32_t d1 = tbase;        // columns [0, 256)
      const uint32_t d2 = tbase + 256;  // columns [256, 512)
      long long g = 0;
      int it = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
        if (it > 0 && !tc::mbar_wait_bounded(tfree, (it - 1) & 1, tc::globaltimer_ns() + kWaitNs,
                                             abort_flag))
          break;
        tc::tc_fence_after();
        for (int c = 0; c < nch; ++c, ++g) {
          const int stg = (int)(g & 1);
          if (!tc::mbar_wait_bounded(&conv[stg], (uint32_t)((g >> 1) & 1),
                                     tc::globaltimer_ns() + kWaitNs, abort_flag))
            break;
          tc::tc_fence_after();
          const uint32_t aA = tc::smem_u32(sm + stg * SB);
          const uint32_t aAlo = aA + kStageA;
          const uint32_t aBh = aA + 2 * kStageA;
          const uint32_t aBl = aBh + nbox * 8192;
          const uint32_t dt = c < nX ? d1 : d2;
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
    }
  } else if (warp < 4) {
    // ------------------------------------------------ head/tail split of F tiles
    const int e = threadIdx.x - 64;  // 0..63: rows e and e + 64
    long long g = 0;
    for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
      for (int c = 0; c < nch; ++c, ++g) {
        const int stg = (int)(g & 1);
        if (!tc::mbar_wait_warp(&full[stg], (uint32_t)((g >> 1) & 1),
                                tc::globaltimer_ns() + kWaitNs, abort_flag))
          break;
        if (c >= nX) {
          // a row's 128 bytes are one swizzle row: process them in place in
          // any chunk order (rotated by row to spread the banks)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = e + 64 * h;
            float4* pa = (float4*)(sm + stg * SB + r * 128);
            float4* pl = (float4*)(sm + stg * SB + kStageA + r * 128);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = (q + r) & 7;
              const float4 v = pa[j];
              const float4 hd = make_float4(tc::tf32_head(v.x), tc::tf32_head(v.y),
                                            tc::tf32_head(v.z), tc::tf32_head(v.w));
              pa[j] = hd;
              pl[j] = make_float4(v.x - hd.x, v.y - hd.y, v.z - hd.z, v.w - hd.w);
            }
          }
          tc::fence_proxy_async_smem();
        }
        tc::mbar_arrive_warp(&conv[stg]);
      }
    }
  } else {
    // ------------------------------------------------ epilogue: 8 warps, two per
    // TMEM lane quarter; the two threads of a row split its columns
    const int q = warp & 3;            // TMEM lane quarter of this warp
    const int half = (warp - 4) >> 2;  // 0 for warps 4-7, 1 for warps 8-11
    const int row = q * 32 + lane;     // tile row = TMEM lane
    const int et = threadIdx.x - 128;  // 0..255
    const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16);
    float* rrow = Rt + row * ldR;
    // W_b of block b: (16 b + 16) x 16 floats at offset 128 b (b + 1)
    auto stage_w = [&](int bi, int buf) {
      const float* src = a.W + 128 * bi * (bi + 1);
      float* dst = Wsm + buf * 4096;
      const int n16 = (16 * bi + 16) * 4;  // 16-byte pieces
      for (int i = et; i < n16; i += 256) tc::cp_async16(dst + 4 * i, src + 4 * i);
      tc::cp_async_commit();
    };
    if (w_resident) {  // all of W fits: stage it once for every tile of this CTA
      const int n16 = 32 * nblk_all * (nblk_all + 1);
      for (int i = et; i < n16; i += 256) tc::cp_async16(Wsm + 4 * i, a.W + 4 * i);
      tc::cp_async_commit();
      tc::cp_async_wait<0>();
      asm volatile("bar.sync 1, 256;" ::: "memory");
    }
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const long long row0 = tile * kBM;
      const long long grow = row0 + row;
      tc::mbar_wait_warp(accf, it & 1, tc::globaltimer_ns() + kWaitNs, abort_flag);
      // one thread's reading of the abort flag decides for all 256
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (et == 0) *go_flag = *abort_flag ? 0 : 1;
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (!*go_flag) {
        if (et == 0) atomicOr(a.err, (int)kStTimeout);
        break;
      }
      tc::tc_fence_after();
      // ---- drain: R = kappa(D1) - D2 into the R tile (half h: column groups h, h+2, ...)
      const float nr = grow < a.N ? a.nrm[grow] : 0.f;
      int jpiv = -1;  // index of this row among the round's pivots, if it is one
      for (int c0 = 16 * half; c0 < s_pad; c0 += 32) {
        float v1[16], v2[16], ns[16];
        int sp[16];
        // per-column constants into registers first: with the stores to the R
        // tile below, the compiler could not otherwise reorder these loads
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          sp[j] = Ss[c0 + j];
          ns[j] = nrmSs[c0 + j];
        }
        tc::tmem_ld16_sync(tl + c0, v1);
        if (nF > 0) {
          tc::tmem_ld16_sync(tl + 256 + c0, v2);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v2[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          const bool self = (long long)sp[j] == grow;
          if (self) jpiv = c;
          const float kv = self ? 1.f : phi_r2<float>(KIND, a.inv_sigma, nr + ns[j] - 2.f * v1[j]);
          v1[j] = c < s ? kv - v2[j] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) rrow[c0 + j] = v1[j];
      }
      tc::tc_fence_before();
      tc::mbar_arrive_warp(tfree);  // TMEM may now take the next tile's accumulators
      if (half == 1) jps[row] = jpiv;
      asm volatile("bar.sync 1, 256;" ::: "memory");  // R tile complete
      if (half == 0 && jps[row] >= 0) jpiv = jps[row];
      // ---- G L^* = R, blocked: G_b = sum_{l < j0 + 16} x_l W_b(l, :) with
      // x_l = G(:, l) (final) for l < j0 and R(:, l) inside the block; one
      // small loop per block (the W_b operand is formed in FP64 per round).
      // Half h computes columns j0 + 8 h .. j0 + 8 h + 7 of the block.
      float rsq = 0.f, rc = 0.f;  // Kahan-compensated sum of G^2 (this half)
      const int nblk = (s + 15) >> 4;
      if (!w_resident) stage_w(0, 0);
      for (int bi = 0; bi < nblk; ++bi) {
        const int j0 = bi * 16;
        const float* Wb;
        if (w_resident) {
          Wb = Wsm + 128 * bi * (bi + 1);
        } else {
          if (bi + 1 < nblk) stage_w(bi + 1, (bi + 1) & 1);
          else tc::cp_async_commit();
          tc::cp_async_wait<1>();
          asm volatile("bar.sync 1, 256;" ::: "memory");
          Wb = Wsm + (bi & 1) * 4096;
        }
        Wb += 8 * half;
        float acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.f;
#pragma unroll 4
        for (int l = 0; l < j0 + 16; ++l) {
          const float xv = rrow[l];
          const float4 w0 = *(const float4*)(Wb + l * 16);
          const float4 w1 = *(const float4*)(Wb + l * 16 + 4);
          acc[0] = fmaf(xv, w0.x, acc[0]);
          acc[1] = fmaf(xv, w0.y, acc[1]);
          acc[2] = fmaf(xv, w0.z, acc[2]);
          acc[3] = fmaf(xv, w0.w, acc[3]);
          acc[4] = fmaf(xv, w1.x, acc[4]);
          acc[5] = fmaf(xv, w1.y, acc[5]);
          acc[6] = fmaf(xv, w1.z, acc[6]);
          acc[7] = fmaf(xv, w1.w, acc[7]);
        }
        // both halves have read the block's R (and the W buffer) before either
        // overwrites it
        asm volatile("bar.sync 1, 256;" ::: "memory");
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) rrow[j0 + 8 * half + jj] = acc[jj];
        // sum of squares of these 8 values (padded columns are zero), then one
        // compensated step into the running total
        float bs = 0.f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) bs = fmaf(acc[jj], acc[jj], bs);
        const float y = bs - rc;
        const float t = rsq + y;
        rc = (t - rsq) - y;
        rsq = t;
        asm volatile("bar.sync 1, 256;" ::: "memory");  // block of G visible to both halves
      }
      if (half == 1) {
        rss[row] = rsq;
        rcs[row] = rc;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (half == 0) {
        // A pivot row of this round: in exact arithmetic R(S,:) = H(S,S) = L L^*,
        // so G(S_j,:) = L(j,:) and its residual is zero.  Write those exact
        // values (L from the FP64 Cholesky of H) instead of the rounded
        // contraction, so that a chosen pivot keeps zero proposal weight and
        // its row of F agrees with the H that later rounds form from it.
        if (jpiv >= 0)
          for (int l = 0; l < s; ++l)
            rrow[l] = l <= jpiv ? (float)a.L[(long long)jpiv * a.ldL + l] : 0.f;
        // ---- residual diagonal (FP64) and the tile's sum of d
        double dn = 0.0;
        if (grow < a.N) {
          const double sq = ((double)rsq - (double)rc) + ((double)rss[row] - (double)rcs[row]);
          const double v = a.dvec[grow] - sq;
          dn = (v > 0.0 && jpiv < 0) ? v : 0.0;
          a.dvec[grow] = dn;
        }
        double t = dn;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[q] = t;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (et == 0) a.tile_sums[tile] = red[0] + red[1] + red[2] + red[3];
      // ---- write G (128 x s) to F(tile, rank : rank + s): rows by warp, columns by lane
      for (int r = warp - 4; r < kBM; r += 8) {
        const long long gr = row0 + r;
        if (gr >= a.N) break;
        float* dst = a.F + gr * a.ldF + rank;
        const float* src = Rt + r * ldR;
        for (int j = lane; j < s; j += 32) dst[j] = src[j];
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");  // R tile and red[] free again
      if (!Lo.overlap) tc::mbar_arrive_warp(edone);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

cudaError_t launch_colstep_tc(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_colstep_tc<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_colstep_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_colstep_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemMax);
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
  a.W = m.Linv32;
  a.dvec = b.dvec;
  a.tile_sums = b.tile_sums;
  a.err = m.err;
  a.kind = b.kind;
  a.inv_sigma = (float)(1.0 / b.sigma);
  a.xld = b.xld;
  a.L = b.L;
  a.ldL = b.Tmax;
  const long long ntiles = (b.N + kBM - 1) / kBM;
  const unsigned grid = (unsigned)(ntiles < m.num_sms ? ntiles : m.num_sms);
  // the shared-memory layout depends on s, which only the device knows: the
  // launch reserves the maximum
  if (b.kind == 0)
    k_colstep_tc<0><<<grid, kTcThreads, kSmemMax, s>>>(m.F, m.X, m.Xlo, m.FSh, m.FSl, m.XSh,
                                                       m.XSl, a);
  else if (b.kind == 1)
    k_colstep_tc<1><<<grid, kTcThreads, kSmemMax, s>>>(m.F, m.X, m.Xlo, m.FSh, m.FSl, m.XSh,
                                                       m.XSl, a);
  else
    k_colstep_tc<2><<<grid, kTcThreads, kSmemMax, s>>>(m.F, m.X, m.Xlo, m.FSh, m.FSl, m.XSh,
                                                       m.XSl, a);
  return cudaGetLastError();
}

}  // namespace rpchol
