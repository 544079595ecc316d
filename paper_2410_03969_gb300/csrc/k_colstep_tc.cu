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
//   warps 4-11  epilogue.  With two tiles in TMEM (s_pad <= 128) warps 4-7
//               and 8-11 form two groups taking alternate tiles, warp 4 + q
//               (8 + q) reading TMEM lane quarter q, 4 rows per thread; with
//               one tile in TMEM all eight work on it, two warps per lane
//               quarter (16 lanes each), 2 rows per thread.
// Operands stream through a ring of 2 to 4 shared-memory stages (as many as
// fit): per stage a 128 x 32 A tile (head, tail) and an s_pad x 32 B tile
// (head, tail), 128-byte swizzled, K-major.  For s_pad <= 128 the two
// accumulators of a tile take 256 TMEM columns, so TMEM holds two tiles:
// the MMAs of the next tile run while an epilogue group works on the last
// one straight from TMEM (no staging tile in shared memory).  The epilogue
// evaluates R = kappa - D2 block by block (16 columns), forms G_b with the
// W blocks, stores G_b back into TMEM over the consumed D1 block (later
// blocks read it from there) and writes it to F.  For s_pad > 128 one tile
// holds all of TMEM: tiles alternate with their epilogues, which then
// use all eight epilogue warps.  Every wait is
// bounded: on expiry the CTA raises the timeout bit of the run status,
// drains its own copies and frees its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

namespace {
constexpr int kTcThreads = 384;
constexpr int kBM = 128;
constexpr int kKc = 32;                  // K extent of a chunk (fp32 elements)
constexpr int kRowBytes = kKc * 4;       // one 128-byte swizzle row per operand row
constexpr int kStageA = kBM * kRowBytes;  // 16 KiB
constexpr int kBoxB = 64 * kRowBytes;     // one 64-row box of a B operand, 8 KiB
constexpr int kSmemMax = 227 * 1024;
constexpr int kSmallBytes = 4 * 1024;  // pivots, their norms, barriers, flags, sums
constexpr int kMaxStages = 4;
constexpr int kPrefetch = 8;          // A chunks prefetched into L2 ahead of their loads
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

struct Layout {
  int s_pad, nbox, stage_bytes, stages, nbuf, w_resident, w_off, small_off, total;
};

// Stages first, then (if room is left for at least as many stages as
// without it, or three) the whole W of the round, then the small region.
__host__ __device__ inline Layout make_layout(int s) {
  Layout L;
  L.s_pad = (s + 15) & ~15;
  L.nbox = (L.s_pad + 63) >> 6;
  L.stage_bytes = 2 * kStageA + 2 * L.nbox * kBoxB;
  L.nbuf = L.s_pad <= 128 ? 2 : 1;
  const int nblk = L.s_pad >> 4;
  const int wbytes = 512 * nblk * (nblk + 1);
  const int budget = kSmemMax - kSmallBytes - 1024;
  int st_nw = budget / L.stage_bytes;
  if (st_nw > kMaxStages) st_nw = kMaxStages;
  int st_w = (budget - wbytes) / L.stage_bytes;
  if (st_w > kMaxStages) st_w = kMaxStages;
  const int want = st_nw < 3 ? st_nw : 3;
  L.w_resident = st_w >= want ? 1 : 0;
  L.stages = L.w_resident ? st_w : st_nw;
  L.w_off = L.stages * L.stage_bytes;
  L.small_off = L.w_off + (L.w_resident ? wbytes : 0);
  L.total = L.small_off + kSmallBytes + 1024;
  return L;
}

// ---- quad layout: thread t of a warp holds NR rows x 4 columns of each
// 16-column block (NR = 4: two 16-lane halves of the warp's TMEM quarter,
// tmem_ld_quad16; NR = 2: one half, tmem_ld_half16), so that the W rows it
// needs differ between the 4 threads of a quad instead of being one
// broadcast value.
struct EpiQuad {
  uint32_t d1, d2;       // TMEM D1 / D2 of the warp's lane quarter (column 0)
  const float* W;        // W blocks of the round
  const float* nrmSs;    // squared norms of the round's pivots
  const double* L;       // FP64 Cholesky factor of the round
  float* frow[4];        // F(row ri, rank), nullptr beyond N
  float nr[4];           // squared norms of the rows
  int jpiv[4];           // index among the round's pivots, or -1
  int s, nF, kind, ldL, cq, lane, even;
  float inv_sigma;
};

// acc[ri] (columns 2cq..2cq+1 and 8+2cq..9+2cq) += sum over the 16 columns
// kappa of block X (held across the quad) of X[ri][kappa] W(kappa, col)
template <int NR>
__device__ __forceinline__ void quad_fma_block(float2 (&acc)[NR][2], const float (&X)[NR][4],
                                               const float* Wblk, int lane, int cq) {
  const int qbase = lane & ~3;
#pragma unroll
  for (int kp = 0; kp < 16; ++kp) {
    const int src = qbase | ((kp & 7) >> 1);
    const int cj = 2 * (kp >> 3) + (kp & 1);
    const float2 w01 = *(const float2*)(Wblk + 16 * kp + 2 * cq);
    const float2 w89 = *(const float2*)(Wblk + 16 * kp + 8 + 2 * cq);
#pragma unroll
    for (int ri = 0; ri < NR; ++ri) {
      const float xv = __shfl_sync(0xffffffffu, X[ri][cj], src);
      const float2 x2 = make_float2(xv, xv);
      acc[ri][0] = __ffma2_rn(x2, w01, acc[ri][0]);
      acc[ri][1] = __ffma2_rn(x2, w89, acc[ri][1]);
    }
  }
}

// The kernel map of the epilogue in FP32 with the fast exponential
// intrinsic: its error bound (2 + 1.16 |x|) ulp of exp(x) is an absolute
// error below 1e-7 for every kernel value in (0, 1], the size of the FP32
// rounding of the values it enters.
template <int KIND>
__device__ __forceinline__ float phi_fast(float inv_sigma, float r2) {
  r2 = r2 > 0.f ? r2 : 0.f;
  if (KIND == 0) return __expf(-0.5f * r2 * inv_sigma * inv_sigma);
  const float r = sqrtf(r2);
  if (KIND == 1) return __expf(-r * inv_sigma);
  if (KIND == 3) {
    const float t = 1.7320508075688772f * r * inv_sigma;
    return (1.f + t) * __expf(-t);
  }
  const float t = 2.2360679774997897f * r * inv_sigma;
  return (1.f + t + t * t * (1.f / 3.f)) * __expf(-t);
}

template <int KIND, int NR>
__device__ __forceinline__ void r_quad(const EpiQuad& e, int j0, const float (&D1v)[NR][4],
                                       const float (&D2v)[NR][4], float (&R)[NR][4]) {
#pragma unroll
  for (int cj = 0; cj < 4; ++cj) {
    const int col = j0 + 8 * (cj >> 1) + 2 * e.cq + (cj & 1);
    const float ns = e.nrmSs[col];
#pragma unroll
    for (int ri = 0; ri < NR; ++ri) {
      const float kv =
          col == e.jpiv[ri] ? 1.f : phi_fast<KIND>(e.inv_sigma, e.nr[ri] + ns - 2.f * D1v[ri][cj]);
      R[ri][cj] = col < e.s ? kv - D2v[ri][cj] : 0.f;
    }
  }
}

// G L^* = R by blocks of 16 columns in the quad layout; finished blocks of G
// go back into TMEM over the consumed D1 blocks.  Returns each row's
// Kahan-compensated partial sum of squares (this thread's 4 columns of
// every block) in rsq / rc.
template <int NR>
__device__ __forceinline__ void tmem_ld_rows(uint32_t ta, float (&v)[NR][4]) {
  if constexpr (NR == 4) tc::tmem_ld_quad16(ta, v);
  else tc::tmem_ld_half16(ta, v);
}

template <int NR>
__device__ __forceinline__ void tmem_st_rows(uint32_t ta, const float (&v)[NR][4]) {
  if constexpr (NR == 4) tc::tmem_st_quad16(ta, v);
  else tc::tmem_st_half16(ta, v);
}

template <int NR>
__device__ __forceinline__ void epi_tile_quad(const EpiQuad e, int nblk, float (&rsq)[NR],
                                              float (&rc)[NR]) {
  const int cq = e.cq;
  for (int bi = 0; bi < nblk; ++bi) {
    const int j0 = 16 * bi;
    const float* Wb = e.W + 128 * bi * (bi + 1);
    float2 acc[NR][2];
#pragma unroll
    for (int ri = 0; ri < NR; ++ri) acc[ri][0] = acc[ri][1] = make_float2(0.f, 0.f);
    for (int lb = 0; lb < bi; ++lb) {
      float X[NR][4];
      tmem_ld_rows<NR>(e.d1 + 16 * lb, X);
      quad_fma_block(acc, X, Wb + 256 * lb, e.lane, cq);
    }
    // this block of R = kappa(||x||^2 + ||x_S||^2 - 2 D1) - D2
    float R[NR][4];
    {
      float D1v[NR][4], D2v[NR][4];
      tmem_ld_rows<NR>(e.d1 + j0, D1v);
      if (e.nF > 0) {
        tmem_ld_rows<NR>(e.d2 + j0, D2v);
      } else {
#pragma unroll
        for (int ri = 0; ri < NR; ++ri)
#pragma unroll
          for (int cj = 0; cj < 4; ++cj) D2v[ri][cj] = 0.f;
      }
      // the kernel map, with the kind resolved outside the loop so that the
      // 16 evaluations interleave
      switch (e.kind) {
        case 0: r_quad<0, NR>(e, j0, D1v, D2v, R); break;
        case 1: r_quad<1, NR>(e, j0, D1v, D2v, R); break;
        case 3: r_quad<3, NR>(e, j0, D1v, D2v, R); break;
        default: r_quad<2, NR>(e, j0, D1v, D2v, R); break;
      }
    }
    quad_fma_block(acc, R, Wb + 256 * bi, e.lane, cq);
    float G[NR][4];
#pragma unroll
    for (int ri = 0; ri < NR; ++ri) {
      G[ri][0] = acc[ri][0].x;
      G[ri][1] = acc[ri][0].y;
      G[ri][2] = acc[ri][1].x;
      G[ri][3] = acc[ri][1].y;
      if (e.jpiv[ri] >= 0) {
        // A pivot row of this round: in exact arithmetic R(S,:) = L L^*, so
        // G(S_j,:) = L(j,:) and its residual is zero.  The exact values (L
        // from the FP64 Cholesky of H) replace the rounded contraction, so a
        // chosen pivot keeps zero proposal weight and its row of F agrees
        // with the H that later rounds form from it.
#pragma unroll
        for (int cj = 0; cj < 4; ++cj) {
          const int col = j0 + 8 * (cj >> 1) + 2 * cq + (cj & 1);
          G[ri][cj] = (col < e.s && col <= e.jpiv[ri])
                          ? (float)e.L[(long long)e.jpiv[ri] * e.ldL + col]
                          : 0.f;
        }
      }
    }
    tmem_st_rows<NR>(e.d1 + j0, G);  // G_b over the consumed D1 block
#pragma unroll
    for (int ri = 0; ri < NR; ++ri) {
      if (e.frow[ri]) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int col = j0 + 8 * g + 2 * cq;
          float* dst = e.frow[ri] + col;
          if (e.even && col + 1 < e.s) {
            *(float2*)dst = make_float2(G[ri][2 * g], G[ri][2 * g + 1]);
          } else {
            if (col < e.s) dst[0] = G[ri][2 * g];
            if (col + 1 < e.s) dst[1] = G[ri][2 * g + 1];
          }
        }
      }
      float bs = 0.f;
#pragma unroll
      for (int cj = 0; cj < 4; ++cj) bs = fmaf(G[ri][cj], G[ri][cj], bs);
      const float y = bs - rc[ri];
      const float t = rsq[ri] + y;
      rc[ri] = (t - rsq[ri]) - y;
      rsq[ri] = t;
    }
  }
}
}  // namespace

struct TcArgs {
  DevState* st;
  float* F;
  long long ldF;
  long long N;
  const float* nrm;     // ||x||^2, FP32
  const float* nrmS;    // ||x_{S_j}||^2
  const int* Sacc;      // accepted pivots of the round
  const float* W;       // blocked-substitution operand of the round (formed by k_prep_tc)
  double* dvec;
  double* tile_sums;
  int* err;             // run status word
  int kind;
  float inv_sigma;
  int xld;
  const double* L;      // compact FP64 Cholesky factor of the round
  int ldL;
  int d;                // point dimension (round bookkeeping)
  unsigned* ccnt;       // CTAs done with the round (zero between launches)
  unsigned long long cond;
  int use_cond;
};

__global__ void __launch_bounds__(kTcThreads, 1)
    k_colstep_tc(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmX,
                 const __grid_constant__ CUtensorMap tmXlo,
                 const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                 const __grid_constant__ CUtensorMap tmXSh,
                 const __grid_constant__ CUtensorMap tmXSl, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  DevState* st = a.st;
  // a round that ended early (nothing accepted, or the run is done) is
  // closed by one thread; otherwise the last CTA to finish closes it
  if (st->done || st->s == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) round_end_body(st, a.cond, a.use_cond, a.N, a.d, 4);
    return;
  }
  const int s = st->s;
  const long long rank = st->rank;
  const Layout Lo = make_layout(s);
  const int s_pad = Lo.s_pad, nbox = Lo.nbox, SB = Lo.stage_bytes, NS = Lo.stages;
  const int nbuf = Lo.nbuf;
  const int nX = a.xld / kKc;
  const int nF = (int)((rank + kKc - 1) / kKc);
  const int nch = nX + nF;
  const long long ntiles = (a.N + kBM - 1) / kBM;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  unsigned char* small = sm + Lo.small_off;
  int* Ss = (int*)small;                  // [256] pivots of the round (-1 beyond s)
  float* nrmSs = (float*)(small + 1024);  // [256] their squared norms
  uint64_t* full = (uint64_t*)(small + 2048);  // [kMaxStages] A operand landed
  uint64_t* conv = full + kMaxStages;          // [kMaxStages] A split into head and tail
  uint64_t* empty = conv + kMaxStages;         // [kMaxStages]
  uint64_t* fullB = empty + kMaxStages;        // [kMaxStages] B operand landed
  uint64_t* accf = fullB + kMaxStages;         // [2] accumulators of a tile complete
  uint64_t* tfree = accf + 2;                  // [2] epilogue done with a TMEM buffer
  uint32_t* tptr = (uint32_t*)(tfree + 2);
  volatile int* abort_flag = (volatile int*)(tptr + 1);
  volatile int* go_flag = abort_flag + 1;      // [2], one per epilogue group
  double* red = (double*)(small + 2048 + 512);  // [8]: [group][quarter], or [epilogue warp]
  const float* Wsm = (const float*)(sm + Lo.w_off);

  for (int i = threadIdx.x; i < s_pad; i += kTcThreads) {
    Ss[i] = i < s ? a.Sacc[i] : -1;
    nrmSs[i] = i < s ? a.nrmS[i] : 0.f;
  }
  if (Lo.w_resident) {
    const int n16 = 32 * (s_pad >> 4) * ((s_pad >> 4) + 1);  // 16-byte pieces of W
    for (int i = threadIdx.x; i < n16; i += kTcThreads)
      tc::cp_async16((float*)Wsm + 4 * i, a.W + 4 * i);
    tc::cp_async_commit();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&fullB[i], 1);
      tc::mbar_init(&conv[i], 2);   // one arrival per converter warp
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&accf[i], 1);
      tc::mbar_init(&tfree[i], nbuf == 2 ? 4 : 8);  // one arrival per epilogue warp on the tile
    }
    *abort_flag = 0;
    tc::fence_mbarrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tptr, 512);
    tc::tmem_relinquish();
  }
  tc::cp_async_wait<0>();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tptr;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tmap(&tmF);
      const uint32_t bbytes = (uint32_t)nbox * (uint32_t)kBoxB;
      // The A operands (rows of F and X, read once per round from HBM) are
      // pulled into L2 kPrefetch chunks ahead of their shared-memory loads,
      // so that a stage turns over at L2 rather than HBM latency.
      long long ptile = blockIdx.x;
      int pc = 0;
      auto prefetch_next = [&]() {
        if (ptile >= ntiles) return;
        const int prow = (int)(ptile * kBM);
        if (pc < nX) {
          tc::tma_prefetch_2d(&tmX, pc * kKc, prow);
          tc::tma_prefetch_2d(&tmXlo, pc * kKc, prow);
        } else {
          tc::tma_prefetch_2d(&tmF, (nF - 1 - (pc - nX)) * kKc, prow);
        }
        if (++pc == nch) {
          pc = 0;
          ptile += gridDim.x;
        }
      };
      for (int i = 0; i < kPrefetch; ++i) prefetch_next();
      long long g = 0;  // chunks issued so far (all tiles)
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        const int row0 = (int)(tile * kBM);
        for (int c = 0; c < nch; ++c, ++g) {
          const int stg = (int)(g % NS);
          if (g >= NS && !tc::mbar_wait_bounded(&empty[stg], (uint32_t)(((g / NS) - 1) & 1),
                                                kWaitNs, abort_flag))
            break;
          unsigned char* sA = sm + stg * SB;
          unsigned char* sAlo = sA + kStageA;
          unsigned char* sBh = sA + 2 * kStageA;
          unsigned char* sBl = sBh + nbox * kBoxB;
          if (c < nX) {
            const int x = c * kKc;
            tc::mbar_arrive_expect_tx(&full[stg], 2u * kStageA);
            tc::tma_load_2d(sA, &tmX, x, row0, &full[stg]);
            tc::tma_load_2d(sAlo, &tmXlo, x, row0, &full[stg]);
            tc::mbar_arrive_expect_tx(&fullB[stg], 2u * bbytes);
            for (int b = 0; b < nbox; ++b) {
              tc::tma_load_2d(sBh + b * kBoxB, &tmXSh, x, 64 * b, &fullB[stg]);
              tc::tma_load_2d(sBl + b * kBoxB, &tmXSl, x, 64 * b, &fullB[stg]);
            }
          } else {
            const int x = (nF - 1 - (c - nX)) * kKc;  // last F column chunk first
            tc::mbar_arrive_expect_tx(&full[stg], (uint32_t)kStageA);
            tc::tma_load_2d(sA, &tmF, x, row0, &full[stg]);
            tc::mbar_arrive_expect_tx(&fullB[stg], 2u * bbytes);
            for (int b = 0; b < nbox; ++b) {
              tc::tma_load_2d(sBh + b * kBoxB, &tmBh, x, 64 * b, &fullB[stg]);
              tc::tma_load_2d(sBl + b * kBoxB, &tmBl, x, 64 * b, &fullB[stg]);
            }
          }
          prefetch_next();
        }
      }
      if (*abort_flag) {
        // drain: the (at most NS) issued loads not yet consumed must land
        volatile int dummy = 0;
        for (long long q = (g > NS ? g - NS : 0); q < g; ++q) {
          tc::mbar_wait_bounded(&full[q % NS], (uint32_t)((q / NS) & 1), kWaitNs, &dummy);
          tc::mbar_wait_bounded(&fullB[q % NS], (uint32_t)((q / NS) & 1), kWaitNs, &dummy);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)s_pad);
      long long g = 0;
      int it = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
        const int buf = it % nbuf;
        if (it >= nbuf &&
            !tc::mbar_wait_bounded(&tfree[buf], (uint32_t)(((it / nbuf) - 1) & 1),
                                   kWaitNs, abort_flag))
          break;
        tc::tc_fence_after();
        const uint32_t d1 = tbase + (uint32_t)(buf * 256);           // D1 of this tile
        const uint32_t d2 = d1 + (nbuf == 2 ? 128u : 256u);           // D2 of this tile
        for (int c = 0; c < nch; ++c, ++g) {
          const int stg = (int)(g % NS);
          // the A split (which waited only for A) and then B
          if (!tc::mbar_wait_bounded(&conv[stg], (uint32_t)((g / NS) & 1), kWaitNs, abort_flag) ||
              !tc::mbar_wait_bounded(&fullB[stg], (uint32_t)((g / NS) & 1), kWaitNs, abort_flag))
            break;
          tc::tc_fence_after();
          const uint32_t aA = tc::smem_u32(sm + stg * SB);
          const uint32_t aAlo = aA + kStageA;
          const uint32_t aBh = aA + 2 * kStageA;
          const uint32_t aBl = aBh + nbox * kBoxB;
          const uint32_t dt = c < nX ? d1 : d2;
          const bool first = (c == 0) || (c == nX);
#pragma unroll
          for (int kk = 0; kk < kKc / 8; ++kk) {
            const uint64_t da = tc::smem_desc_sw128(aA + 32 * kk);
            const uint64_t dal = tc::smem_desc_sw128(aAlo + 32 * kk);
            const uint64_t dbh = tc::smem_desc_sw128(aBh + 32 * kk);
            const uint64_t dbl = tc::smem_desc_sw128(aBl + 32 * kk);
            // hi.hi and hi.lo share A: the second takes it from the
            // collector buffer instead of reading shared memory again
            tc::mma_tf32_keep_a(dt, da, dbh, idesc, (first && kk == 0) ? 0u : 1u);
            tc::mma_tf32_reuse_a(dt, da, dbl, idesc, 1u);
            tc::mma_tf32(dt, dal, dbh, idesc, 1u);
          }
          tc::mma_commit(&empty[stg]);
        }
        tc::mma_commit(&accf[it & 1]);
      }
    }
  } else if (warp < 4) {
    // ------------------------------------------------ head/tail split of F tiles
    const int e = threadIdx.x - 64;  // 0..63: rows e and e + 64
    long long g = 0;
    for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
      for (int c = 0; c < nch; ++c, ++g) {
        const int stg = (int)(g % NS);
        if (!tc::mbar_wait_warp(&full[stg], (uint32_t)((g / NS) & 1),
                                kWaitNs, abort_flag))
          break;
        if (c >= nX) {
          // a row's 128 bytes are one swizzle row: process them in place in
          // any chunk order (rotated by row to spread the banks); both rows
          // are read into registers before any store, so that the loads are
          // not held behind stores the compiler cannot prove apart
          float4 v[2][8];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = e + 64 * h;
            const float4* pa = (const float4*)(sm + stg * SB + r * kRowBytes);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[h][q] = pa[(q + r) & 7];
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = e + 64 * h;
            float4* pa = (float4*)(sm + stg * SB + r * kRowBytes);
            float4* pl = (float4*)(sm + stg * SB + kStageA + r * kRowBytes);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = (q + r) & 7;
              const float4 x = v[h][q];
              const float4 hd = make_float4(tc::tf32_head(x.x), tc::tf32_head(x.y),
                                            tc::tf32_head(x.z), tc::tf32_head(x.w));
              pa[j] = hd;
              pl[j] = make_float4(x.x - hd.x, x.y - hd.y, x.z - hd.z, x.w - hd.w);
            }
          }
          tc::fence_proxy_async_smem();
        }
        tc::mbar_arrive_warp(&conv[stg]);
      }
    }
  } else if (nbuf == 2) {
    // ------------------------------------------------ epilogue, two tiles in TMEM:
    // groups of four warps take alternate tiles
    const int q = warp & 3;              // TMEM lane quarter of this warp
    const int grp = (warp - 4) >> 2;     // 0: warps 4-7, 1: warps 8-11
    const int row = q * 32 + lane;       // tile row = TMEM lane
    const int gt = row;                  // thread index inside the group
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int nblk = (s + 15) >> 4;
    const int bar_id = 2 + grp;
    for (int it = grp;; it += 2) {
      const long long tile = blockIdx.x + (long long)it * gridDim.x;
      if (tile >= ntiles) break;
      const long long row0 = tile * kBM;
      // this thread's rows: ri -> 32 q + lane / 4 + 16 (ri >> 1) + 8 (ri & 1)
      const int cq = lane & 3;
      long long growv[4];
      EpiQuad eq;
#pragma unroll
      for (int ri = 0; ri < 4; ++ri) {
        growv[ri] = row0 + 32 * q + (lane >> 2) + 16 * (ri >> 1) + 8 * (ri & 1);
        const bool lv = growv[ri] < a.N;
        eq.frow[ri] = lv ? a.F + growv[ri] * a.ldF + rank : nullptr;
        eq.nr[ri] = lv ? a.nrm[growv[ri]] : 0.f;  // loaded while the accumulators fill
        eq.jpiv[ri] = -1;
      }
      // this thread updates d for row ri = cq (each row once across its quad)
      const long long grow = row0 + 32 * q + (lane >> 2) + 16 * (cq >> 1) + 8 * (cq & 1);
      const bool live = grow < a.N;
      const double dold = live ? a.dvec[grow] : 0.0;
      for (int j = 0; j < s; ++j) {
        const long long p = (long long)Ss[j];
#pragma unroll
        for (int ri = 0; ri < 4; ++ri)
          if (p == growv[ri]) eq.jpiv[ri] = j;
      }
      tc::mbar_wait_warp(&accf[grp], (uint32_t)((it >> 1) & 1), kWaitNs,
                         abort_flag);
      // one thread's reading of the abort flag decides for the whole group
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (gt == 0) go_flag[grp] = *abort_flag ? 0 : 1;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (!go_flag[grp]) {
        if (gt == 0) atomicOr(a.err, (int)kStTimeout);
        break;
      }
      tc::tc_fence_after();
      eq.d1 = tbase + lane_off + (uint32_t)(grp * 256);
      eq.d2 = eq.d1 + 128u;
      eq.W = Lo.w_resident ? Wsm : a.W;
      eq.nrmSs = nrmSs;
      eq.L = a.L;
      eq.s = s;
      eq.nF = nF;
      eq.kind = a.kind;
      eq.ldL = a.ldL;
      eq.cq = cq;
      eq.lane = lane;
      eq.even = (rank & 1) == 0;
      eq.inv_sigma = a.inv_sigma;
      float rsq[4] = {0.f, 0.f, 0.f, 0.f}, rc[4] = {0.f, 0.f, 0.f, 0.f};
      epi_tile_quad<4>(eq, nblk, rsq, rc);
      tc::tc_fence_before();
      tc::mbar_arrive_warp(&tfree[grp]);  // TMEM buffer free for tile it + 2
      // ---- row sums of G^2 across the quad (FP64), residual diagonal, tile sum
      double sq[4];
#pragma unroll
      for (int ri = 0; ri < 4; ++ri) {
        sq[ri] = (double)rsq[ri] - (double)rc[ri];
        sq[ri] += __shfl_xor_sync(0xffffffffu, sq[ri], 1);
        sq[ri] += __shfl_xor_sync(0xffffffffu, sq[ri], 2);
      }
      const double mysq = cq == 0 ? sq[0] : cq == 1 ? sq[1] : cq == 2 ? sq[2] : sq[3];
      const int myjp = cq == 0 ? eq.jpiv[0] : cq == 1 ? eq.jpiv[1] : cq == 2 ? eq.jpiv[2] : eq.jpiv[3];
      double dn = 0.0;
      if (live) {
        const double v = dold - mysq;
        dn = (v > 0.0 && myjp < 0) ? v : 0.0;
        a.dvec[grow] = dn;
      }
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
      if (lane == 0) red[grp * 4 + q] = dn;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (gt == 0)
        a.tile_sums[tile] = red[grp * 4] + red[grp * 4 + 1] + red[grp * 4 + 2] + red[grp * 4 + 3];
    }
  } else {
    // ------------------------------------------------ epilogue, one tile in TMEM:
    // all eight warps work on it (groups taking alternate tiles would leave
    // one idle): warp w takes TMEM lane quarter q = w & 3 (the quarter it
    // may access) and half h = (w - 4) >> 2 of it, 16 rows, two per thread.
    const int q = warp & 3;
    const int h = (warp - 4) >> 2;
    const int et = (warp - 4) * 32 + lane;  // 0..255
    const uint32_t lane_off = (uint32_t)(q * 32 + 16 * h) << 16;
    const int nblk = (s + 15) >> 4;
    for (int it = 0;; ++it) {
      const long long tile = blockIdx.x + (long long)it * gridDim.x;
      if (tile >= ntiles) break;
      const int buf = it % nbuf;
      const long long row0 = tile * kBM;
      // this thread's rows: ri -> 32 q + 16 h + lane / 4 + 8 ri
      const int cq = lane & 3;
      long long growv[2];
      EpiQuad eq;
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        growv[ri] = row0 + 32 * q + 16 * h + (lane >> 2) + 8 * ri;
        const bool lv = growv[ri] < a.N;
        eq.frow[ri] = lv ? a.F + growv[ri] * a.ldF + rank : nullptr;
        eq.nr[ri] = lv ? a.nrm[growv[ri]] : 0.f;  // loaded while the accumulators fill
        eq.jpiv[ri] = -1;
      }
      // threads cq = 0, 1 of a quad update d for rows ri = cq
      const long long grow = row0 + 32 * q + 16 * h + (lane >> 2) + 8 * (cq & 1);
      const bool live = cq < 2 && grow < a.N;
      const double dold = live ? a.dvec[grow] : 0.0;
      for (int j = 0; j < s; ++j) {
        const long long p = (long long)Ss[j];
#pragma unroll
        for (int ri = 0; ri < 2; ++ri)
          if (p == growv[ri]) eq.jpiv[ri] = j;
      }
      tc::mbar_wait_warp(&accf[it & 1], (uint32_t)((it >> 1) & 1), kWaitNs, abort_flag);
      // one thread's reading of the abort flag decides for all eight warps
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (et == 0) go_flag[0] = *abort_flag ? 0 : 1;
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (!go_flag[0]) {
        if (et == 0) atomicOr(a.err, (int)kStTimeout);
        break;
      }
      tc::tc_fence_after();
      eq.d1 = tbase + lane_off + (uint32_t)(buf * 256);
      eq.d2 = eq.d1 + (nbuf == 2 ? 128u : 256u);
      eq.W = Lo.w_resident ? Wsm : a.W;
      eq.nrmSs = nrmSs;
      eq.L = a.L;
      eq.s = s;
      eq.nF = nF;
      eq.kind = a.kind;
      eq.ldL = a.ldL;
      eq.cq = cq;
      eq.lane = lane;
      eq.even = (rank & 1) == 0;
      eq.inv_sigma = a.inv_sigma;
      float rsq[2] = {0.f, 0.f}, rc[2] = {0.f, 0.f};
      epi_tile_quad<2>(eq, nblk, rsq, rc);
      tc::tc_fence_before();
      tc::mbar_arrive_warp(&tfree[buf]);  // TMEM buffer free for tile it + nbuf
      // ---- row sums of G^2 across the quad (FP64), residual diagonal, tile sum
      double sq[2];
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        sq[ri] = (double)rsq[ri] - (double)rc[ri];
        sq[ri] += __shfl_xor_sync(0xffffffffu, sq[ri], 1);
        sq[ri] += __shfl_xor_sync(0xffffffffu, sq[ri], 2);
      }
      const double mysq = (cq & 1) == 0 ? sq[0] : sq[1];
      const int myjp = (cq & 1) == 0 ? eq.jpiv[0] : eq.jpiv[1];
      double dn = 0.0;
      if (live) {
        const double v = dold - mysq;
        dn = (v > 0.0 && myjp < 0) ? v : 0.0;
        a.dvec[grow] = dn;
      }
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
      if (lane == 0) red[warp - 4] = dn;
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (et == 0) {
        double ts = 0.0;
        for (int w = 0; w < 8; ++w) ts += red[w];
        a.tile_sums[tile] = ts;
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.ccnt, 1u) == gridDim.x - 1) {
      __threadfence();
      // three split products per K step, M = 128 rows per tile, N = s_pad
      const double mma = 6.0 * 128.0 * (double)ntiles * (double)s_pad * (double)(nch * kKc);
      round_end_body(st, a.cond, a.use_cond, a.N, a.d, 4, mma, 0.0);
      *a.ccnt = 0u;
    }
  }
}

cudaError_t launch_colstep_tc(const TcMaps& m, const DevBuffers& b, unsigned long long cond,
                              int use_cond, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_colstep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  a.d = b.d;
  a.ccnt = b.ccnt;
  a.cond = cond;
  a.use_cond = use_cond;
  const long long ntiles = (b.N + kBM - 1) / kBM;
  const unsigned grid = (unsigned)(ntiles < m.num_sms ? ntiles : m.num_sms);
  // the shared-memory layout depends on s, which only the device knows: the
  // launch reserves the maximum
  k_colstep_tc<<<grid, kTcThreads, kSmemMax, s>>>(m.F, m.X, m.Xlo, m.FSh, m.FSl, m.XSh, m.XSl, a);
  return cudaGetLastError();
}

}  // namespace rpchol
