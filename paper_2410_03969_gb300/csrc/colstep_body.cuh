// Tensor-core column step of accelerated RPCholesky in mixed precision
// (Algorithm 2, step 3, arXiv 2410.03969), sm_103a:
//
//   D1 = X_tile X_S^*            (fast Euclidean distances, App. A.1)
//   R  = kappa(||x||^2 + ||x_S||^2 - 2 D1) - F_tile F(S,:)^*
//   G L^* = R                    (forward substitution in FP32 with the FP64 L
//                                 of Algorithm 1 rounded once)
//   F(tile, rank:rank+s) = G;  d <- max(d - rowsumsq(G), 0) (FP64);  tile sums of d.
//
// One accumulator per 128-row tile holds, in turn, D1, then kappa(D1), then
// R: the distance contraction runs first; the epilogue maps it to kappa in
// TMEM; the Schur contraction then accumulates -F_tile F(S,:)^* onto it,
// the columns of F in forward order, so that the accumulator follows the
// Schur complement of the growing partial factorisation, whose entries
// shrink as columns are added (the tensor core's FP32 accumulation
// truncates; adding to a small accumulator keeps that error small).  With
// one accumulator of s_pad <= 256 columns per tile, TMEM (512 columns)
// holds two to four tiles, so the MMAs of later tiles run while the
// epilogue works on earlier ones, for every block size T <= 256.
//
// Precision of the contractions (FP32 accumulation throughout):
//   - distances: kind::tf32, three-term compensated products
//     a_hi b_hi + a_hi b_lo + a_lo b_hi of the TF32 head/tail planes of X,
//     for ~fp32 accuracy in ||x||^2 + ||y||^2 - 2 x.y at any scale of X;
//   - Schur part: kind::f16 (twice the TF32 rate, half the operand bytes),
//     the same three-term products of FP16 heads and tails of 4096 F: every
//     entry of F lies in [-1, 1] (its squared row norm is at most
//     kappa(x, x) = 1), so 4096 F is far inside the FP16 range and the
//     head + tail carry 22 significant bits like the TF32 pair; products
//     carry 4096^2, removed exactly in the epilogue.
//
// Persistent kernel: one CTA per SM walks its 128-row tiles (one sampler
// tile each).  Warp roles (384 threads):
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM owner and MMA issuer (one elected lane)
//   warps 2-3   no role in the column step (the CTA shape the batch engine
//               shares)
//   warps 4-11  epilogue: two groups of four warps taking alternate tiles,
//               warp 4 + q (8 + q) reading TMEM lane quarter q, 4 rows per
//               thread.
// Operands stream through a ring of shared-memory stages, each a 16 KiB A
// region (two planes of 128 rows x 64 bytes) and a B region of 2 x s_pad
// rows x 64 bytes.  A stage holds one chunk: 16 coordinates of X (TF32 head
// and tail planes) against the same 16 of X_S, or 32 columns of F (FP16
// heads and tails of 4096 F, which the epilogue writes beside F with
// every new column) against the same 32 of F(S,:).  Both A operands arrive by
// TMA ready for the MMAs: X as two planes with the 64-byte swizzle; F as
// one 128-row box of 128-byte rows (per row the 32 heads, then the 32
// tails, stored so in HBM) with the 128-byte swizzle, whose head and tail
// halves the MMAs address as K offsets 0 and 64 bytes.  The B operands of the
// round are laid out by the operand-prep kernel as the exact shared-memory
// image of each chunk and arrive with one bulk copy per chunk.  The
// producer streams the next tile's X chunks inside the current tile's F
// chunks (see Seq), so that the next tile's distances and kappa pass run
// while the current tile's Schur MMAs execute.  Every wait is bounded: on expiry
// the CTA raises the timeout bit of the run status, drains its own copies
// and frees its TMEM.
//
// This header holds the device-side body (colstep_body) and its helpers; the
// stand-alone kernel (k_colstep_tc.cu) and the persistent batch engine
// (k_batch.cu) run it.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

namespace {
constexpr int kTcThreads = 384;
constexpr int kBM = 128;
constexpr int kStageA = 16384;            // A region of a stage
constexpr int kFK = 32;                   // columns of F per chunk
constexpr int kXK = 16;                   // coordinates of X per chunk
constexpr int kSmemMax = 227 * 1024;
constexpr int kSmallBytes = 4 * 1024;     // pivots, their norms, barriers, flags, sums
// The last kTailBytes of the kSmemMax-byte allocation stay outside the
// layout (the caller's TMEM address and a persistent kernel's job slots);
// reserving them changes no stage count or W placement for any s.
constexpr int kTailBytes = 256;
constexpr int kMaxStages = 6;
constexpr int kMaxBuf = 4;                // tiles held in TMEM at once

constexpr float kFScale = 4096.f;         // the Schur operands are heads/tails of 4096 F
constexpr float kAccScale = 16777216.f;   // 4096^2: the scale of the Schur products
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

struct Layout {
  int s_pad, s_alloc, nbuf, bbytes, stage_bytes, stages, w_resident, w_off, small_off, total;
};

// Stages first, then (if room is left for at least as many stages as
// without it, or three) the whole W of the round, then the small region.
__host__ __device__ inline Layout make_layout(int s) {
  Layout L;
  L.s_pad = (s + 15) & ~15;
  L.s_alloc = (L.s_pad + 31) & ~31;
  L.nbuf = 512 / L.s_alloc;
  if (L.nbuf > kMaxBuf) L.nbuf = kMaxBuf;
  L.bbytes = 128 * L.s_pad;
  L.stage_bytes = kStageA + L.bbytes;
  const int nblk = L.s_pad >> 4;
  const int wbytes = 512 * nblk * (nblk + 1);
  const int budget = kSmemMax - kSmallBytes - 1024 - kTailBytes;
  int st_nw = budget / L.stage_bytes;
  if (st_nw > kMaxStages) st_nw = kMaxStages;
  int st_w = (budget - wbytes) / L.stage_bytes;
  if (st_w > kMaxStages) st_w = kMaxStages;
  const int want = st_nw < 3 ? st_nw : 3;
  L.w_resident = st_w >= want ? 1 : 0;
  L.stages = L.w_resident ? st_w : st_nw;
  L.w_off = L.stages * L.stage_bytes;
  L.small_off = L.w_off + (L.w_resident ? wbytes : 0);
  L.total = L.small_off + kSmallBytes + 1024 + kTailBytes;
  return L;
}

// The chunk sequence a CTA streams: the X chunks of local tile 0, then for
// each local tile t its F chunks with the X chunks of tile t + 1 inserted
// after the first `split` of them.  A tile whose round has no F columns yet
// (rank 0) gets one empty F item (kind 2), which loads nothing.  With three
// or more tiles in TMEM split = 0 (the next tile's distances and kappa pass
// run while this tile's Schur MMAs execute); with two, the next tile's
// buffer frees only when the epilogue of tile t - 1 is done, so its X chunks
// come nine tenths of the way through tile t's F chunks (measured against
// 1/2, 2/3, 3/4 and 5/6: the later the split, the longer the final pass of
// tile t - 1 may take without stalling the tensor cores, while the last
// tenth still covers the next tile's kappa pass).  Producer and MMA issuer
// walk the same sequence.
struct Seq {
  int t, ph, c;  // ph 0: F(t) before the split, 1: X(t + 1), 2: F(t) after it
  int ntl, nXc, nF, nFi, split;
  __device__ void init(int ntl_, int nbuf, int nXc_, int nF_) {
    ntl = ntl_;
    nXc = nXc_;
    nF = nF_;
    nFi = nF > 0 ? nF : 1;
    split = nbuf >= 3 ? 0 : (9 * nFi) / 10;
    t = -1;
    ph = 0;
    c = 0;
    settle();
  }
  __device__ bool done() const { return t >= ntl; }
  __device__ int kind() const { return ph == 1 ? 0 : (nF > 0 ? 1 : 2); }
  __device__ int tile() const { return ph == 1 ? t + 1 : t; }
  __device__ void settle() {
    for (;;) {
      if (t >= ntl) return;
      if (ph == 0) {
        if (t >= 0 && c < split) return;
        ph = 1;
        c = 0;
      }
      if (ph == 1) {
        if (t + 1 < ntl && c < nXc) return;
        ph = 2;
        c = t >= 0 ? split : 0;
      }
      if (t >= 0 && c < nFi) return;
      ph = 0;
      c = 0;
      ++t;
    }
  }
  __device__ void next() {
    ++c;
    settle();
  }
};

// ---- quad layout: thread t of a warp holds 4 rows x 4 columns of each
// 16-column block (two 16-lane halves of the warp's TMEM quarter,
// tmem_ld_quad16), so that the W rows it needs differ between the 4
// threads of a quad instead of being one broadcast value.
struct EpiQuad {
  uint32_t acc;          // TMEM accumulator of the warp's lane quarter (column 0)
  const float* W;        // W blocks of the round
  const float* nrmSs;    // squared norms of the round's pivots
  const double* L;       // FP64 Cholesky factor of the round
  long long fidx[4];     // element index of F(row ri, rank), -1 beyond N
  float* F;              // the factor, FP32
  __half* Fs;            // FP16 heads / tails of 4096 F, interleaved by 32-column chunk
  float nr[4];           // squared norms of the rows
  int jpiv[4];           // index among the round's pivots, or -1
  int s, kind, ldL, cq, lane, even, rank31;
  float inv_sigma;
};

// Partial products of one 16 x 16 block in the quad layout.  A thread holds
// X for its 4 rows at its own 4 columns kappa of the block (2cq, 2cq + 1,
// 8 + 2cq, 9 + 2cq), so with no exchange it can form, for every one of the
// 16 output columns, the part of sum_kappa X[ri][kappa] W(kappa, col) that
// runs over its own kappa: P[ri][q] holds output columns (2q, 2q + 1) in .x
// and (8 + 2q, 9 + 2q) in .y, the columns quad lane q finally owns.  The
// quad's four parts are added once a block of G is complete (quad_reduce).
// Row kappa of a W block keeps owner q's four columns in 16-byte group
// q ^ ((kappa >> 1) & 3), which is q ^ cq for this thread's rows, so the
// four lanes of a quad read four different bank groups.
__device__ __forceinline__ void quad_part_block(float4 (&P)[4][4], const float (&X)[4][4],
                                                const float* Wblk, int cq) {
  // the W row of the next own column is loaded before the products of the
  // current one, so its shared-memory latency overlaps them
  float4 wb[2][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) wb[0][q] = *(const float4*)(Wblk + 16 * (2 * cq) + 4 * (q ^ cq));
#pragma unroll
  for (int cj = 0; cj < 4; ++cj) {
    if (cj < 3) {
      const int cn = cj + 1;
      const float* wn = Wblk + 16 * (8 * (cn >> 1) + 2 * cq + (cn & 1));
#pragma unroll
      for (int q = 0; q < 4; ++q) wb[cn & 1][q] = *(const float4*)(wn + 4 * (q ^ cq));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 w = wb[cj & 1][q];
      const float2 w01 = make_float2(w.x, w.y), w89 = make_float2(w.z, w.w);
#pragma unroll
      for (int ri = 0; ri < 4; ++ri) {
        const float2 x2 = make_float2(X[ri][cj], X[ri][cj]);
        float2 lo = make_float2(P[ri][q].x, P[ri][q].y);
        float2 hi = make_float2(P[ri][q].z, P[ri][q].w);
        lo = __ffma2_rn(x2, w01, lo);
        hi = __ffma2_rn(x2, w89, hi);
        P[ri][q] = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
    }
  }
}

// Sum the quad's four parts of every output column onto the lane that owns
// it (two exchange steps: lanes cq ^ 2, then cq ^ 1); G[ri][cj] gets
// columns 2cq, 2cq + 1, 8 + 2cq, 9 + 2cq, the quad layout's order.
__device__ __forceinline__ void quad_reduce(const float4 (&P)[4][4], int cq, float (&G)[4][4]) {
  const bool hi = (cq & 2) != 0, lo = (cq & 1) != 0;
#pragma unroll
  for (int ri = 0; ri < 4; ++ri) {
    float4 k[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float4 snd = hi ? P[ri][q] : P[ri][q + 2];
      const float4 kp = hi ? P[ri][q + 2] : P[ri][q];
      k[q].x = kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 2);
      k[q].y = kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 2);
      k[q].z = kp.z + __shfl_xor_sync(0xffffffffu, snd.z, 2);
      k[q].w = kp.w + __shfl_xor_sync(0xffffffffu, snd.w, 2);
    }
    const float4 snd = lo ? k[0] : k[1];
    const float4 kp = lo ? k[1] : k[0];
    G[ri][0] = kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 1);
    G[ri][1] = kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 1);
    G[ri][2] = kp.z + __shfl_xor_sync(0xffffffffu, snd.z, 1);
    G[ri][3] = kp.w + __shfl_xor_sync(0xffffffffu, snd.w, 1);
  }
}

// The kernel map of the epilogue in FP32 with the fast exponential
// intrinsic: its error bound (2 + 1.16 |x|) ulp of exp(x) is an absolute
// error below 1e-7 for every kernel value in (0, 1], the size of the FP32
// rounding of the values it enters; r = r^2 rsqrt(max(r^2, 1e-30)) adds at
// most a few ulp to r (and gives 0 at r = 0).
template <int KIND>
__device__ __forceinline__ float phi_fast(float inv_sigma, float r2) {
  r2 = r2 > 0.f ? r2 : 0.f;
  if (KIND == 0) return __expf(-0.5f * r2 * inv_sigma * inv_sigma);
  const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
  if (KIND == 1) return __expf(-r * inv_sigma);
  if (KIND == 3) {
    const float t = 1.7320508075688772f * r * inv_sigma;
    return (1.f + t) * __expf(-t);
  }
  const float t = 2.2360679774997897f * r * inv_sigma;
  return (1.f + t + t * t * (1.f / 3.f)) * __expf(-t);
}

// The kappa pass: D1 -> 4096^2 kappa(||x||^2 + ||x_S||^2 - 2 D1) in place,
// columns beyond s zero, kappa(x, x) = 1 at a row's own pivot column.
// Blocks are loaded two at a time and stored without waiting; one wait at
// the end covers every store.
template <int KIND>
__device__ __forceinline__ void kappa_block(const EpiQuad& e, int j0, const float (&D1v)[4][4]) {
  float K[4][4];
#pragma unroll
  for (int cj = 0; cj < 4; ++cj) {
    const int col = j0 + 8 * (cj >> 1) + 2 * e.cq + (cj & 1);
    const float ns = e.nrmSs[col];
#pragma unroll
    for (int ri = 0; ri < 4; ++ri) {
      // evaluated for every entry (no branch around the kernel map), then
      // the row's own pivot column set to kappa(x, x) = 1
      float kv = phi_fast<KIND>(e.inv_sigma, e.nr[ri] + ns - 2.f * D1v[ri][cj]);
      kv = col == e.jpiv[ri] ? 1.f : kv;
      K[ri][cj] = col < e.s ? kv * kAccScale : 0.f;
    }
  }
  tc::tmem_st_quad16_nowait(e.acc + j0, K);
}

template <int KIND>
__device__ __forceinline__ void kappa_pass(const EpiQuad& e, int nblk) {
  for (int bi = 0; bi < nblk; bi += 2) {
    float D0[4][4], D1[4][4];
    if (bi + 1 < nblk) {
      tc::tmem_ld_quad16x2(e.acc + 16 * bi, e.acc + 16 * (bi + 1), D0, D1);
      kappa_block<KIND>(e, 16 * bi, D0);
      kappa_block<KIND>(e, 16 * (bi + 1), D1);
    } else {
      tc::tmem_ld_quad16(e.acc + 16 * bi, D0);
      kappa_block<KIND>(e, 16 * bi, D0);
    }
  }
  tc::tmem_wait_st();
}

// G L^* = R by blocks of 16 columns in the quad layout; R is the
// accumulator divided by 4096^2; finished blocks of G go back into TMEM
// over the consumed R blocks (later blocks read them from there).  Returns
// each row's Kahan-compensated partial sum of squares (this thread's 4
// columns of every block) in rsq / rc.
__device__ __forceinline__ void epi_tile_quad(const EpiQuad e, int nblk, float (&rsq)[4],
                                              float (&rc)[4]) {
  const int cq = e.cq;
  for (int bi = 0; bi < nblk; ++bi) {
    const int j0 = 16 * bi;
    const float* Wb = e.W + 128 * bi * (bi + 1);
    float4 P[4][4];
#pragma unroll
    for (int ri = 0; ri < 4; ++ri)
#pragma unroll
      for (int q = 0; q < 4; ++q) P[ri][q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int lb = 0; lb < bi; ++lb) {
      float X[4][4];
      tc::tmem_ld_quad16(e.acc + 16 * lb, X);
      quad_part_block(P, X, Wb + 256 * lb, cq);
    }
    float R[4][4];
    tc::tmem_ld_quad16(e.acc + j0, R);
#pragma unroll
    for (int ri = 0; ri < 4; ++ri)
#pragma unroll
      for (int cj = 0; cj < 4; ++cj) R[ri][cj] *= (1.f / kAccScale);
    quad_part_block(P, R, Wb + 256 * bi, cq);
    float G[4][4];
    quad_reduce(P, cq, G);
#pragma unroll
    for (int ri = 0; ri < 4; ++ri) {
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
    tc::tmem_st_quad16(e.acc + j0, G);  // G_b over the consumed R block
#pragma unroll
    for (int ri = 0; ri < 4; ++ri) {
      if (e.fidx[ri] >= 0) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int col = j0 + 8 * g + 2 * cq;
          const long long idx = e.fidx[ri] + col;  // F(row, rank + col)
          // the FP16 head and tail of 4096 G, as later rounds' Schur MMAs
          // read them: head of F(r, c) at 2 (r ldF + c) - (c mod 32), its
          // tail 32 further
          const long long hidx = 2 * idx - ((e.rank31 + col) & 31);
          const float y0 = G[ri][2 * g] * kFScale, y1 = G[ri][2 * g + 1] * kFScale;
          const __half2 h = __floats2half2_rn(y0, y1);
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn(y0 - hf.x, y1 - hf.y);
          if (e.even && col + 1 < e.s) {
            *(float2*)(e.F + idx) = make_float2(G[ri][2 * g], G[ri][2 * g + 1]);
            *(__half2*)(e.Fs + hidx) = h;
            *(__half2*)(e.Fs + hidx + 32) = l;
          } else {
            if (col < e.s) {
              e.F[idx] = G[ri][2 * g];
              e.Fs[hidx] = __low2half(h);
              e.Fs[hidx + 32] = __low2half(l);
            }
            if (col + 1 < e.s) {
              const long long hidx1 = 2 * (idx + 1) - ((e.rank31 + col + 1) & 31);
              e.F[idx + 1] = G[ri][2 * g + 1];
              e.Fs[hidx1] = __high2half(h);
              e.Fs[hidx1 + 32] = __high2half(l);
            }
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
  __half* Fs;               // FP16 heads / tails of 4096 F, written with F
  long long ldF;
  long long N;
  const float* nrm;         // ||x||^2, FP32
  const float* nrmS;        // ||x_{S_j}||^2
  const int* Sacc;          // accepted pivots of the round
  const float* W;           // blocked-substitution operand of the round (formed by k_prep_tc)
  const unsigned char* Bx;  // shared-memory images of the X_S chunks of the round
  const unsigned char* Bf;  // shared-memory images of the F(S,:) chunks of the round
  double* dvec;
  double* tile_sums;
  int* err;                 // run status word
  int kind;
  float inv_sigma;
  int xld;
  const double* L;          // compact FP64 Cholesky factor of the round
  int ldL;
  int d;                    // point dimension (round bookkeeping)
  unsigned* ccnt;           // CTAs done with the round (zero between launches)
  unsigned long long cond;
  int use_cond;
};

// The column step's arguments for a context's buffers (host side).
inline TcArgs make_tc_args(const TcMaps& m, const DevBuffers& b, unsigned long long cond,
                           int use_cond) {
  TcArgs a;
  a.st = b.st;
  a.F = (float*)b.F;
  a.Fs = (__half*)m.Fsp;
  a.ldF = b.ldF;
  a.N = b.N;
  a.nrm = b.nrm;
  a.nrmS = m.nrmS;
  a.Sacc = b.Sacc;
  a.W = m.Linv32;
  a.Bx = m.Bx;
  a.Bf = m.Bf;
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
  return a;
}

// The column step of one round on CTA `cta` of `ncta` (tiles cta, cta +
// ncta, ...), with 4 + 4 g warps (g epilogue groups), shared memory at sm
// (1024-byte aligned, kSmemMax bytes) and 512 TMEM columns at tbase
// allocated by the caller.  With mc > 1 the CTAs cta - cta % mc .. + mc - 1
// are one thread-block cluster (cluster rank cta % mc) that shares each B
// operand: every CTA loads 1/mc of it into all of them (bulk-copy
// multicast), a stage is refilled once all mc CTAs' MMAs are done with it
// (multicast commits), and all walk the same number of tiles (a CTA past
// the last tile streams zero rows and writes nothing).  The last of the
// ncta CTAs to finish closes the round; the one thread that closed it gets
// true.
__device__ __forceinline__ bool colstep_body(const CUtensorMap* tmFs, const CUtensorMap* tmXh,
                                             const CUtensorMap* tmXl,
                                             const TcArgs& a,
                                             unsigned char* sm, uint32_t tbase, int cta,
                                             int ncta, int mc = 1) {
  DevState* st = a.st;
  // a round that ended early (nothing accepted, or the run is done) is
  // closed by one thread; otherwise the last CTA to finish closes it
  if (st->done || st->s == 0) {
    if (cta == 0 && threadIdx.x == 0) {
      round_end_body(st, a.cond, a.use_cond, a.N, a.d, 4);
      return true;
    }
    return false;
  }
  const int s = st->s;
  const long long rank = st->rank;
  const Layout Lo = make_layout(s);
  const int s_pad = Lo.s_pad, SB = Lo.stage_bytes, NS = Lo.stages, nbuf = Lo.nbuf;
  const uint32_t bbytes = (uint32_t)Lo.bbytes;
  const int nXc = a.xld / kXK;
  const int nF = (int)((rank + kFK - 1) / kFK);
  const long long ntiles = (a.N + kBM - 1) / kBM;
  const int crank = cta % mc;                       // rank in the multicast cluster
  const uint16_t mc_mask = (uint16_t)((1u << mc) - 1u);
  // tiles of the cluster's first CTA: every CTA of the cluster walks as many
  const int ntl = (int)((ntiles - (cta - crank) + ncta - 1) / ncta);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = ((int)(blockDim.x >> 5) - 4) >> 2;  // epilogue groups of four warps

  unsigned char* small = sm + Lo.small_off;
  int* Ss = (int*)small;                       // [256] pivots of the round (-1 beyond s)
  float* nrmSs = (float*)(small + 1024);       // [256] their squared norms
  uint64_t* full = (uint64_t*)(small + 2048);  // [kMaxStages] A operand landed
  uint64_t* empty = full + 2 * kMaxStages;     // [kMaxStages]
  uint64_t* fullB = empty + kMaxStages;        // [kMaxStages] B operand landed
  uint64_t* d1f = fullB + kMaxStages;          // [kMaxBuf] distance MMAs of a tile done
  uint64_t* midf = d1f + kMaxBuf;              // [kMaxBuf] kappa pass of a tile done
  uint64_t* accf = midf + kMaxBuf;             // [kMaxBuf] Schur MMAs of a tile done
  uint64_t* tfree = accf + kMaxBuf;            // [kMaxBuf] epilogue done with a buffer
  volatile int* abort_flag = (volatile int*)(tfree + kMaxBuf) + 1;
  volatile int* go_flag = abort_flag + 1;       // [2], one per epilogue group
  double* red = (double*)(small + 2048 + 768);  // [8]: [group][quarter]
  const float* Wsm = (const float*)(sm + Lo.w_off);

  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    Ss[i] = i < s ? a.Sacc[i] : -1;
    nrmSs[i] = i < s ? a.nrmS[i] : 0.f;
  }
  if (Lo.w_resident) {
    const int n16 = 32 * (s_pad >> 4) * ((s_pad >> 4) + 1);  // 16-byte pieces of W
    for (int i = threadIdx.x; i < n16; i += blockDim.x)
      tc::cp_async16((float*)Wsm + 4 * i, a.W + 4 * i);
    tc::cp_async_commit();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&fullB[i], 1);
      tc::mbar_init(&empty[i], (uint32_t)mc);  // one MMA commit per CTA of the cluster
    }
    for (int i = 0; i < kMaxBuf; ++i) {
      tc::mbar_init(&d1f[i], 1);
      tc::mbar_init(&midf[i], 4);  // one arrival per warp of the tile's epilogue group
      tc::mbar_init(&accf[i], 1);
      tc::mbar_init(&tfree[i], 4);
    }
    *abort_flag = 0;
    tc::fence_mbarrier_init();
  }
  tc::cp_async_wait<0>();
  __syncthreads();
  if (mc > 1) tc::cluster_barrier();  // every barrier of the cluster is initialised
  tc::tc_fence_after();

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tmap(tmFs);
      tc::prefetch_tmap(tmXh);
      tc::prefetch_tmap(tmXl);
      // No L2 prefetch of the A operands ahead of their loads: measured, it
      // slowed the stage turnover (the prefetches compete with the loads and
      // the tensor cores' shared-memory reads for the same paths).
      // stages filled so far, g = NS pass + stg, ph = pass & 1 (kept
      // incrementally: a 64-bit division by the run-time NS on every stage
      // costs this single lane hundreds of cycles)
      long long g = 0;
      int stg = 0;
      uint32_t ph = 0;
      Seq sq;
      for (sq.init(ntl, nbuf, nXc, nF); !sq.done() && !*abort_flag; sq.next()) {
        const int kd = sq.kind();
        if (kd == 2) continue;
        if (g >= NS && !tc::mbar_wait_bounded(&empty[stg], ph ^ 1u, kWaitNs, abort_flag))
          break;
        const int row0 = (int)((cta + (long long)sq.tile() * ncta) * kBM);
        unsigned char* sA = sm + stg * SB;
        unsigned char* sB = sA + kStageA;
        tc::mbar_arrive_expect_tx(&full[stg], (uint32_t)kStageA);
        tc::mbar_arrive_expect_tx(&fullB[stg], bbytes);  // all mc slices land here
        if (kd == 0) {
          tc::tma_load_2d(sA, tmXh, sq.c * kXK, row0, &full[stg]);
          tc::tma_load_2d(sA + kStageA / 2, tmXl, sq.c * kXK, row0, &full[stg]);
        } else {
          tc::tma_load_2d(sA, tmFs, sq.c * 2 * kFK, row0, &full[stg]);
        }
        const unsigned char* srcB = (kd == 0 ? a.Bx : a.Bf) + (size_t)sq.c * bbytes;
        if (mc == 1) {
          tc::bulk_load(sB, srcB, bbytes, &fullB[stg]);
        } else {
          const uint32_t sl = bbytes / (uint32_t)mc;  // a multiple of 512
          tc::bulk_load_mc(sB + crank * sl, srcB + crank * sl, sl, &fullB[stg], mc_mask);
        }
        ++g;
        if (++stg == NS) {
          stg = 0;
          ph ^= 1u;
        }
      }
      if (mc > 1 && !*abort_flag) {
        // the last stages' releases by the other CTAs (multicast commits)
        // must have landed before this CTA's barriers are invalidated
        for (long long q = (g > NS ? g - NS : 0); q < g; ++q)
          if (!tc::mbar_wait_bounded(&empty[q % NS], (uint32_t)((q / NS) & 1), kWaitNs,
                                     abort_flag)) {
            atomicOr(a.err, (int)kStTimeout);
            break;
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
      const uint32_t id32 = tc::idesc_tf32(128, (uint32_t)s_pad);
      const uint32_t id16 = tc::idesc_f16(128, (uint32_t)s_pad);
      // ring position kept incrementally, as in the producer; the tile's
      // TMEM buffer and its use count change only with the tile
      int stg = 0;
      uint32_t ph = 0;
      int jc = -1, b = 0;
      uint32_t use = 0;
      Seq sq;
      for (sq.init(ntl, nbuf, nXc, nF); !sq.done() && !*abort_flag; sq.next()) {
        const int kd = sq.kind(), j = sq.tile();
        if (j != jc) {
          jc = j;
          b = j % nbuf;
          use = (uint32_t)(j / nbuf);
        }
        const uint32_t acc = tbase + (uint32_t)(b * Lo.s_alloc);
        if (kd == 0 && sq.c == 0 && j >= nbuf) {  // the buffer's previous tile is done
          if (!tc::mbar_wait_bounded(&tfree[b], (use - 1) & 1, kWaitNs, abort_flag)) break;
          tc::tc_fence_after();
        }
        if (kd != 0 && sq.c == 0) {  // kappa(D1) is in the accumulator
          if (!tc::mbar_wait_bounded(&midf[b], use & 1, kWaitNs, abort_flag)) break;
          tc::tc_fence_after();
        }
        if (kd == 2) {
          tc::mma_commit(&accf[b]);
          continue;
        }
        if (!tc::mbar_wait_bounded(&full[stg], ph, kWaitNs, abort_flag) ||
            !tc::mbar_wait_bounded(&fullB[stg], ph, kWaitNs, abort_flag))
          break;
        tc::tc_fence_after();
        const uint32_t aA = tc::smem_u32(sm + stg * SB);
        const uint32_t aB = aA + kStageA;
        const uint32_t aBl = aB + 64u * (uint32_t)s_pad;
        if (kd == 0) {
          // X head / tail planes (8 KiB each, 64-byte swizzle), TF32, K = 8 per MMA
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t da = tc::smem_desc(aA + 32 * kk, 512, 4);
            const uint64_t dal = tc::smem_desc(aA + kStageA / 2 + 32 * kk, 512, 4);
            const uint64_t dbh = tc::smem_desc(aB + 32 * kk, 512, 4);
            const uint64_t dbl = tc::smem_desc(aBl + 32 * kk, 512, 4);
            const uint32_t accum = (sq.c == 0 && kk == 0) ? 0u : 1u;  // a fresh tile starts at 0
            tc::mma_tf32_keep_a(acc, da, dbh, id32, accum);
            tc::mma_tf32_reuse_a(acc, da, dbl, id32, 1u);
            tc::mma_tf32(acc, dal, dbh, id32, 1u);
          }
          if (mc == 1) tc::mma_commit(&empty[stg]);
          else tc::mma_commit_mc(&empty[stg], mc_mask);
          if (sq.c == nXc - 1) tc::mma_commit(&d1f[b]);
        } else {
          // FP16 heads (bytes 0-63 of each 128-byte row) and tails (64-127) of
          // 4096 F, 128-byte swizzle, K = 16 per MMA
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t da = tc::smem_desc(aA + 32 * kk, 1024, 2);
            const uint64_t dal = tc::smem_desc(aA + 64 + 32 * kk, 1024, 2);
            const uint64_t dbh = tc::smem_desc(aB + 32 * kk, 512, 4);
            const uint64_t dbl = tc::smem_desc(aBl + 32 * kk, 512, 4);
            tc::mma_f16_keep_a(acc, da, dbh, id16, 1u);
            tc::mma_f16_reuse_a(acc, da, dbl, id16, 1u);
            tc::mma_f16(acc, dal, dbh, id16, 1u);
          }
          if (mc == 1) tc::mma_commit(&empty[stg]);
          else tc::mma_commit_mc(&empty[stg], mc_mask);
          if (sq.c == nF - 1) tc::mma_commit(&accf[b]);
        }
        if (++stg == NS) {
          stg = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp < 4) {
    // no role in the column step
  } else {
    // ------------------------------------------------ epilogue: groups of four
    // warps take alternate tiles
    const int q = warp & 3;           // TMEM lane quarter of this warp
    const int grp = (warp - 4) >> 2;  // 0: warps 4-7, 1: warps 8-11
    const int gt = q * 32 + lane;     // thread index inside the group
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int nblk = s_pad >> 4;
    const int bar_id = 2 + grp;
    const int cq = lane & 3;
    for (int j = grp; j < ntl; j += ngroups) {
      const long long tile = cta + (long long)j * ncta;
      const long long row0 = tile * kBM;
      const int b = j % nbuf;
      const uint32_t use = (uint32_t)(j / nbuf);
      // this thread's rows: ri -> 32 q + lane / 4 + 16 (ri >> 1) + 8 (ri & 1)
      long long growv[4];
      EpiQuad eq;
#pragma unroll
      for (int ri = 0; ri < 4; ++ri) {
        growv[ri] = row0 + 32 * q + (lane >> 2) + 16 * (ri >> 1) + 8 * (ri & 1);
        const bool lv = growv[ri] < a.N;
        eq.fidx[ri] = lv ? growv[ri] * a.ldF + rank : -1;
        eq.nr[ri] = lv ? a.nrm[growv[ri]] : 0.f;
        eq.jpiv[ri] = -1;
      }
      // this thread updates d for row ri = cq (each row once across its quad)
      const long long grow = row0 + 32 * q + (lane >> 2) + 16 * (cq >> 1) + 8 * (cq & 1);
      const bool live = grow < a.N;
      const double dold = live ? a.dvec[grow] : 0.0;
      for (int jj = 0; jj < s; ++jj) {
        const long long p = (long long)Ss[jj];
#pragma unroll
        for (int ri = 0; ri < 4; ++ri)
          if (p == growv[ri]) eq.jpiv[ri] = jj;
      }
      eq.acc = tbase + lane_off + (uint32_t)(b * Lo.s_alloc);
      eq.F = a.F;
      eq.Fs = a.Fs;
      eq.rank31 = (int)(rank & 31);
      eq.W = Lo.w_resident ? Wsm : a.W;
      eq.nrmSs = nrmSs;
      eq.L = a.L;
      eq.s = s;
      eq.kind = a.kind;
      eq.ldL = a.ldL;
      eq.cq = cq;
      eq.lane = lane;
      eq.even = (rank & 1) == 0;
      eq.inv_sigma = a.inv_sigma;
      // ---- the kappa pass, once the tile's distance MMAs are done; one
      // thread's reading of the abort flag decides for the whole group
      tc::mbar_wait_warp(&d1f[b], use & 1, kWaitNs, abort_flag);
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (gt == 0) go_flag[grp] = *abort_flag ? 0 : 1;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (!go_flag[grp]) {
        if (gt == 0) atomicOr(a.err, (int)kStTimeout);
        break;
      }
      tc::tc_fence_after();
      switch (eq.kind) {
        case 0: kappa_pass<0>(eq, nblk); break;
        case 1: kappa_pass<1>(eq, nblk); break;
        case 3: kappa_pass<3>(eq, nblk); break;
        default: kappa_pass<2>(eq, nblk); break;
      }
      tc::tc_fence_before();
      tc::mbar_arrive_warp(&midf[b]);
      // ---- R complete: substitution, F, d
      tc::mbar_wait_warp(&accf[b], use & 1, kWaitNs, abort_flag);
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (gt == 0) go_flag[grp] = *abort_flag ? 0 : 1;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (!go_flag[grp]) {
        if (gt == 0) atomicOr(a.err, (int)kStTimeout);
        break;
      }
      tc::tc_fence_after();
      float rsq[4] = {0.f, 0.f, 0.f, 0.f}, rc[4] = {0.f, 0.f, 0.f, 0.f};
      epi_tile_quad(eq, nblk, rsq, rc);
      tc::tc_fence_before();
      tc::mbar_arrive_warp(&tfree[b]);  // TMEM buffer free for tile j + nbuf
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
        dn = (v > kDFloorMixed && myjp < 0) ? v : 0.0;
        a.dvec[grow] = dn;
      }
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
      if (lane == 0) red[grp * 4 + q] = dn;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (gt == 0 && tile < ntiles)
        a.tile_sums[tile] = red[grp * 4] + red[grp * 4 + 1] + red[grp * 4 + 2] + red[grp * 4 + 3];
    }
  }
  tc::tc_fence_before();
  // F and d written here are read by later rounds, F also by bulk tensor
  // copies (async proxy)
  tc::fence_proxy_async_all();
  __syncthreads();
  if (mc > 1) tc::cluster_barrier();  // no CTA's copies or commits still reach another
  bool closed = false;
  if (threadIdx.x == 0) {
    // the barriers' shared memory goes back to other uses
    for (int i = 0; i < NS; ++i) {
      tc::mbar_inval(&full[i]);
      tc::mbar_inval(&fullB[i]);
      tc::mbar_inval(&empty[i]);
    }
    for (int i = 0; i < kMaxBuf; ++i) {
      tc::mbar_inval(&d1f[i]);
      tc::mbar_inval(&midf[i]);
      tc::mbar_inval(&accf[i]);
      tc::mbar_inval(&tfree[i]);
    }
    __threadfence();
    if (atomicAdd(a.ccnt, 1u) == (unsigned)ncta - 1) {
      __threadfence();
      // three split products per K step, M = 128 rows per tile, N = s_pad
      const double per = 6.0 * 128.0 * (double)ntiles * (double)s_pad;
      round_end_body(st, a.cond, a.use_cond, a.N, a.d, 4, per * (double)a.xld,
                     per * (double)(nF * kFK));
      *a.ccnt = 0u;
      closed = true;
    }
  }
  return closed;
}

}  // namespace rpchol
