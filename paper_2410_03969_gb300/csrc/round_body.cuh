// Device-side bodies of the round kernels of accelerated RPCholesky
// (Algorithm 2 and Algorithm 1 of arXiv 2410.03969): reset, proposal
// sampler, residual submatrix H and RejectionSampleSubmatrix.  Each body
// takes its block index (and shared memory) as arguments, so that the
// stand-alone kernels (k_round.cu) and the persistent batch engine
// (k_batch.cu) run the same code block by block.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace rpchol {

// ------------------------------------------------------------------ reset
// d = diag A = phi(0) = 1 for every kernel here; tile sums are the tile row
// counts; state initialised for a new run.
__device__ __forceinline__ void reset_run(DevState* st, double* dvec, double* tile_sums,
                                          long long N, long long ntiles, long long k, int T,
                                          unsigned long long seed, unsigned inst, int plain,
                                          long long max_rounds, long long blk, long long nblk) {
  const long long i = blk * blockDim.x + threadIdx.x;
  const long long stride = nblk * blockDim.x;
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
    st->plain = plain == 1;
    st->block = plain == 2;
    st->seed = seed;
    st->instance = inst;
    st->W = 0.0;
    st->gs = 0.0;
    st->piv = -1;
    st->col_bytes = 0.0;
    st->col_flops = 0.0;
    st->mma_tf32 = 0.0;
    st->mma_f16 = 0.0;
  }
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

// Step 1 of Algorithm 2: T iid draws with P{j} = d_j / sum(d).  FP64 is
// scarce on this GPU, so the draws are spread over ceil(T / 8) CTAs, one
// warp per draw, and every CTA forms the same inclusive prefix of the tile
// sums (written by the kernel that last updated d): thread t sums its run of
// consecutive tiles sequentially, then a block scan combines the runs, in a
// fixed order identical in every CTA.  A draw binary-searches the tile
// prefix and scans its tile with a warp prefix sum: the pivot is the first j
// whose running sum exceeds U * W (the proposal map of the oracle, summed in
// tile order instead of index order).
// One block `blk` of the sampler (draws 8 blk .. 8 blk + 7), 256 threads;
// pref_smem holds the tile prefix when use_smem, wsum 8 doubles.
__device__ __forceinline__ void propose_body(int blk, double* pref_smem, double* wsum, DevState* st,
                                             const double* dvec,
                                             const double* tile_sums,
                                             double* tile_prefix, long long ntiles, long long N,
                                             int* prop, double* uprop, double* uacc, int use_smem,
                                             const void* F, long long ldF, int f_double) {
  if (st->done) return;
  const int T = st->T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* P = use_smem ? pref_smem : tile_prefix + blk * ntiles;
  const long long per = (ntiles + 255) / 256;
  const long long t0 = tid * per, t1 = t0 + per < ntiles ? t0 + per : ntiles;
  double own = 0.0;
  for (long long t = t0; t < t1; ++t) own += tile_sums[t];
  double incl = warp_incl_scan(own);
  if (lane == 31) wsum[warp] = incl;
  body_sync();
  double before = 0.0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  double W = 0.0;
  for (int w = 0; w < 8; ++w) W += wsum[w];
  double run = before + (incl - own);
  for (long long t = t0; t < t1; ++t) {
    run += tile_sums[t];
    P[t] = run;
  }
  if (blk == 0 && tid == 0) {
    st->W = W;
    if (!(W > 0.0)) st->done = 1;
  }
  if (!(W > 0.0)) return;
  body_sync();  // prefix complete and visible to the CTA

  const int j = blk * 8 + warp;
  if (j >= T) return;
  const unsigned long long seed = st->seed;
  const unsigned round = (unsigned)st->round;
  const unsigned inst = st->instance;
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
    const double inc = warp_incl_scan(v);
    const unsigned pos = __ballot_sync(0xffffffffu, v > 0.0);
    if (pos) last_pos = c + 31 - __clz(pos);
    if (!fallback) {
      const unsigned hit = __ballot_sync(0xffffffffu, v > 0.0 && running + inc > target);
      if (hit) {
        found = c + __ffs(hit) - 1;
        break;
      }
    }
    running += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (found < 0) found = last_pos;  // rounding: the last positive weight in the tile
  if (found < 0) found = r0;         // unreachable when W > 0
  if (lane == 0) {
    prop[j] = (int)found;
    uprop[j] = dvec[found];
    uacc[j] = ua;
  }
  // simple RPCholesky (Algorithm 6): the pivot's entry of the new column,
  // g_s = A(s,s) - ||F(s, 0:i)||^2 (A(s,s) = 1), with the arithmetic of the
  // step's GEMV rows (FP32 accumulation for an FP32 factor)
  if (st->plain && j == 0) {
    const long long i = st->rank;
    double g;
    if (f_double) {
      const double* fr = (const double*)F + found * ldF;
      const double* rows[1] = {fr};
      double acc[1];
      warp_rows_dot<double, 1>(rows, fr, i, lane, acc);
      g = 1.0 - acc[0];
    } else {
      const float* fr = (const float*)F + found * ldF;
      const float* rows[1] = {fr};
      float acc[1];
      warp_rows_dot<float, 1>(rows, fr, i, lane, acc);
      g = (double)(1.f - acc[0]);
    }
    if (lane == 0) {
      st->gs = g;
      st->piv = found;
    }
  }
}

// ------------------------------------------------------------------ H
// Rank splits of H for ntile lower tiles on a GPU of num_sms SMs (a function
// of the problem and the GPU only, so that every launch shape sums the same
// partials in the same order).
__host__ __device__ __forceinline__ int hmat_splits(int ntile, int num_sms) {
  int ks = (4 * num_sms + ntile - 1) / ntile;
  if (ks > kHSplitMax) ks = kHSplitMax;
  if (ks < 1) ks = 1;
  return ks;
}

// H = A(S',S') - F(S',:) F(S',:)^*, FP64 (FP32 factors are widened; their
// products are exact in FP64).  Kernel entries by direct differences.
// Output tiles of 16 x 16 (lower triangle of tiles; both halves of H are
// written from the same value), one thread per entry.  FP64 throughput is
// low on this GPU, so the rank dimension is split KS = gridDim.y ways, in
// equal parts, to spread the tiles over all SMs: each CTA writes a partial
// product, and the last CTA of a tile to finish (counted with an atomic)
// adds the KS partials in the fixed order z = 0..KS-1, so the result does
// not depend on timing.  The kernel entries of a tile are shared out among
// its KS CTAs too (entries z, z + KS, ... to CTA z, computed by its first
// threads: an FP64 instruction costs the same with one lane active as with
// 32), so that no CTA evaluates the kernel after all the partials are in.
// One block (tile, z) of H: lower tile `tile` (row-major over (ta, tb),
// tb <= ta), rank split z of KS; 256 threads; Fa, Fb 16 x 33 each, `last`
// one int, all in shared memory.
template <typename TF>
__device__ __forceinline__ void hmat_body(int tile, int z, int KS, TF (*Fa)[33], TF (*Fb)[33],
                                          int& last, const DevState* st,
                                          const float* X, int xld, int d, int kind,
                                          double inv_sigma, const TF* F,
                                          long long ldF, const int* prop, double* H,
                                          double* Hpart, int* hcnt) {
  if (st->done) return;
  const int T = st->T;
  const long long rank = st->rank;
  int ta = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
  while ((ta + 1) * (ta + 2) / 2 <= tile) ++ta;
  while (ta * (ta + 1) / 2 > tile) --ta;
  const int tb = tile - ta * (ta + 1) / 2;
  const int a0 = 16 * ta, b0 = 16 * tb;
  if (a0 >= T) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long kc = (rank + KS - 1) / KS;
  const long long m_lo = z * kc < rank ? z * kc : rank;
  const long long m_hi = m_lo + kc < rank ? m_lo + kc : rank;
  // rows of this thread's two staged elements (row e >> 5, column e & 31)
  int ra[2], rb[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int r = (tid + 256 * q) >> 5;
    ra[q] = a0 + r < T ? prop[a0 + r] : prop[0];
    rb[q] = b0 + r < T ? prop[b0 + r] : prop[0];
  }
  const int cc = tid & 31;
  TF va[2], vb[2];  // the next chunk, loaded while the current one is used
  auto fetch = [&](long long m0) {
    const long long m = m0 + cc;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      va[q] = m < m_hi ? F[(long long)ra[q] * ldF + m] : (TF)0;
      vb[q] = m < m_hi ? F[(long long)rb[q] * ldF + m] : (TF)0;
    }
  };
  // kernel entry of H at (a, b), 1 on the diagonal of A
  auto kval = [&](int a, int b) -> double {
    const int pa = prop[a], pb = prop[b];
    if (pa == pb) return 1.0;
    const float* xa = X + (long long)pa * xld;
    const float* xb = X + (long long)pb * xld;
    double r2 = 0.0;
    for (int l = 0; l < d; ++l) {
      const double t = (double)xa[l] - (double)xb[l];
      r2 += dist_term(kind, t);
    }
    return phi_r2<double>(kind, inv_sigma, r2);
  };
  double acc = 0.0;
  if (m_lo < m_hi) fetch(m_lo);
  // this CTA's share of the kernel entries (slot KS of the tile's partials),
  // formed while the first chunk of F is in flight
  double* P = Hpart + (long long)tile * (KS + 1) * 256;
  if (KS > 1 && z + KS * tid < 256) {
    const int e = z + KS * tid;
    const int a = a0 + (e >> 4), bb = b0 + (e & 15);
    if (a < T && bb < T && bb <= a) P[KS * 256 + e] = kval(a, bb);
  }
  // FP32 factor (mixed mode): the products of FP32 entries are summed as
  // unevaluated float pairs (exact product by FMA, two-sum of Knuth) on the
  // FP32 pipe, which on this GPU issues far more than the FP64 one; about 48
  // bits survive, well below the FP32 rounding of F itself
  float sh = 0.f, sl = 0.f;
  for (long long m0 = m_lo; m0 < m_hi; m0 += 32) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = (tid + 256 * q) >> 5;
      Fa[r][cc] = va[q];
      Fb[r][cc] = vb[q];
    }
    body_sync();
    if (m0 + 32 < m_hi) fetch(m0 + 32);
    const int qn = m_hi - m0 < 32 ? (int)(m_hi - m0) : 32;
    if constexpr (sizeof(TF) == 4) {
#pragma unroll 8
      for (int q = 0; q < qn; ++q) {
        const float a = Fa[ty][q], b = Fb[tx][q];
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float t = __fadd_rn(sh, p);
        const float bp = __fsub_rn(t, sh);
        const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(er, e));
      }
    } else {
#pragma unroll 8
      for (int q = 0; q < qn; ++q) acc = fma(Fa[ty][q], Fb[tx][q], acc);
    }
    body_sync();
  }
  if constexpr (sizeof(TF) == 4) acc = (double)sh + (double)sl;
  double sum = acc;
  if (KS > 1) {
    P[z * 256 + tid] = acc;
    __threadfence();
    body_sync();
    if (tid == 0) last = atomicAdd(&hcnt[tile], 1) == KS - 1;
    body_sync();
    if (!last) return;
    __threadfence();
    sum = 0.0;
    for (int zz = 0; zz < KS; ++zz) sum += __ldcg(P + zz * 256 + tid);
    if (tid == 0) hcnt[tile] = 0;
  }
  const int a = a0 + ty, bcol = b0 + tx;
  if (a < T && bcol < T && bcol <= a) {
    const double kv = KS > 1 ? __ldcg(P + KS * 256 + tid) : kval(a, bcol);
    const double h = kv - sum;
    H[(long long)a * T + bcol] = h;
    H[(long long)bcol * T + a] = h;
  }
}

// H for an FP32 factor (mixed mode).  Output blocks of 32 x 32 (lower
// triangle of blocks), 256 threads, each thread four entries (rows a0 + ty
// + 16 i, columns b0 + tx + 16 j), so that four independent accumulations
// hide the latency of each.  The products of FP32 entries are summed as
// unevaluated float pairs (exact product by FMA, two-sum of Knuth) on the
// FP32 pipe, which on this GPU issues far more than the FP64 one; about 48
// bits survive, well below the FP32 rounding of F itself.  The rank
// dimension is split KS ways (hmat32_splits), each split writes its partial
// sums, and the last split of a block to finish (counted with an atomic)
// adds the KS partials in the fixed order z = 0..KS-1, so the result does
// not depend on timing or on which CTA runs which split.  The kernel
// entries of a block (FP64) are shared out among its KS splits.
__host__ __device__ __forceinline__ int hmat32_blocks(int T) {
  const int nb = (T + 31) / 32;
  return nb * (nb + 1) / 2;
}
__host__ __device__ __forceinline__ int hmat32_splits(int nblk) {
  int ks = (128 + nblk - 1) / nblk;  // about 128 CTAs: one wave over the SMs
  if (ks > kHSplitMax) ks = kHSplitMax;
  return ks < 1 ? 1 : ks;
}

struct H32Smem {
  float Fa[32][33];
  float Fb[32][33];
  int last;
};

__device__ __forceinline__ void dfloat_acc(float& sh, float& sl, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(er, e));
}

// One block (blk, z) of H for an FP32 factor: lower block `blk` (row-major
// over (ta, tb), tb <= ta), rank split z of KS; 256 threads.
__device__ __forceinline__ void hmat32_body(int blk, int z, int KS, H32Smem& S, const DevState* st,
                                            const float* X, int xld, int d, int kind,
                                            double inv_sigma, const float* F, long long ldF,
                                            const int* prop, double* H, double* Hpart,
                                            int* hcnt) {
  if (st->done) return;
  const int T = st->T;
  const long long rank = st->rank;
  int ta = (int)((sqrtf(8.f * blk + 1.f) - 1.f) * 0.5f);
  while ((ta + 1) * (ta + 2) / 2 <= blk) ++ta;
  while (ta * (ta + 1) / 2 > blk) --ta;
  const int tb = blk - ta * (ta + 1) / 2;
  const int a0 = 32 * ta, b0 = 32 * tb;
  if (a0 >= T) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long kc = (rank + KS - 1) / KS;
  const long long m_lo = z * kc < rank ? z * kc : rank;
  const long long m_hi = m_lo + kc < rank ? m_lo + kc : rank;
  // staged elements: row (tid >> 5) + 8 q, column tid & 31, q = 0..3
  const int cc = tid & 31;
  int ra[4], rb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = (tid >> 5) + 8 * q;
    ra[q] = a0 + r < T ? prop[a0 + r] : prop[0];
    rb[q] = b0 + r < T ? prop[b0 + r] : prop[0];
  }
  float va[4], vb[4];  // the next chunk, loaded while the current one is used
  auto fetch = [&](long long m0) {
    const long long m = m0 + cc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      va[q] = m < m_hi ? F[(long long)ra[q] * ldF + m] : 0.f;
      vb[q] = m < m_hi ? F[(long long)rb[q] * ldF + m] : 0.f;
    }
  };
  // kernel entry of H at (a, b), 1 on the diagonal of A
  auto kval = [&](int a, int b) -> double {
    const int pa = prop[a], pb = prop[b];
    if (pa == pb) return 1.0;
    const float* xa = X + (long long)pa * xld;
    const float* xb = X + (long long)pb * xld;
    double r2 = 0.0;
    for (int l = 0; l < d; ++l) {
      const double t = (double)xa[l] - (double)xb[l];
      r2 += dist_term(kind, t);
    }
    return phi_r2<double>(kind, inv_sigma, r2);
  };
  if (m_lo < m_hi) fetch(m_lo);
  double* P = Hpart + (long long)blk * (KS + 1) * 1024;
  if (KS > 1) {
    // this split's share of the kernel entries, formed while the first
    // chunk of F is in flight
    for (int e = z + KS * tid; e < 1024; e += KS * 256) {
      const int a = a0 + (e >> 5), bb = b0 + (e & 31);
      if (a < T && bb < T && bb <= a) P[KS * 1024 + e] = kval(a, bb);
    }
  }
  float sh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, sl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (long long m0 = m_lo; m0 < m_hi; m0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = (tid >> 5) + 8 * q;
      S.Fa[r][cc] = va[q];
      S.Fb[r][cc] = vb[q];
    }
    body_sync();
    if (m0 + 32 < m_hi) fetch(m0 + 32);
    const int qn = m_hi - m0 < 32 ? (int)(m_hi - m0) : 32;
#pragma unroll 4
    for (int q = 0; q < qn; ++q) {
      const float x0 = S.Fa[ty][q], x1 = S.Fa[ty + 16][q];
      const float y0 = S.Fb[tx][q], y1 = S.Fb[tx + 16][q];
      dfloat_acc(sh[0][0], sl[0][0], x0, y0);
      dfloat_acc(sh[0][1], sl[0][1], x0, y1);
      dfloat_acc(sh[1][0], sl[1][0], x1, y0);
      dfloat_acc(sh[1][1], sl[1][1], x1, y1);
    }
    body_sync();
  }
  double sum[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) sum[i][j] = (double)sh[i][j] + (double)sl[i][j];
  if (KS > 1) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) P[z * 1024 + (ty + 16 * i) * 32 + tx + 16 * j] = sum[i][j];
    __threadfence();
    body_sync();
    if (tid == 0) S.last = atomicAdd(&hcnt[blk], 1) == KS - 1;
    body_sync();
    if (!S.last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int e = (ty + 16 * i) * 32 + tx + 16 * j;
        double t = 0.0;
        for (int zz = 0; zz < KS; ++zz) t += __ldcg(P + zz * 1024 + e);
        sum[i][j] = t;
      }
    if (tid == 0) hcnt[blk] = 0;
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + ty + 16 * i, bcol = b0 + tx + 16 * j;
      if (a < T && bcol < T && bcol <= a) {
        const int e = (ty + 16 * i) * 32 + tx + 16 * j;
        const double kv = KS > 1 ? __ldcg(P + KS * 1024 + e) : kval(a, bcol);
        const double h = kv - sum[i][j];
        H[(long long)a * T + bcol] = h;
        H[(long long)bcol * T + a] = h;
      }
    }
}

// ------------------------------------------------------------------ Algorithm 1
// RejectionSampleSubmatrix.  For i = 0..T-1: accept iff u_i * U_i < h_ii
// (u_i the proposal weight d[s'_i], h_ii the current Schur diagonal); on
// acceptance L(i:T, i) = H(i:T, i) / sqrt(h_ii) and the trailing triangle
// is downdated.  Stops once the total rank reaches k.  Writes the compact L,
// the accepted pivots and s.
//
// FP64 issue is the limit here: a warp retires an FP64 instruction about
// every 64 cycles and an SM about every 16 to 19.  The work runs on one
// thread-block cluster of kRejCluster CTAs with a lookahead of one pivot:
//   - CTA 0 (the lead CTA) keeps the diagonal apart from H and, in the
//     iteration of accepted pivot t (index n_t), forms column t: it reads
//     H(j, n_t) from the CTA that owns row j, applies the downdate of pivot
//     t-1 to it, scales by 1/sqrt(h), sends the column to every other CTA,
//     downdates the diagonal, finds the next acceptance (warp 0, from its
//     own 32 rows unless none of them accepts) and its 1/sqrt(h);
//   - at the same time CTAs 1.. (row j lives in CTA 1 + j mod (kRejCluster -
//     1), packed) apply the downdate of pivot t-1 to their rows and columns
//     beyond n_t, the only entries later pivots read.
// One cluster barrier separates the iterations.  The lead CTA does no
// downdate work, so the lead chain has its SM's FP64 pipe to itself.
// Rejections leave H untouched, so the acceptance test looks at 32
// proposals at once.
constexpr int kRejCluster = 8;
constexpr int kRejOwners = kRejCluster - 1;
constexpr int kRejectThreads = 256;
constexpr int kLeadWarps = 4;

// offset of row j in its owner's packed rows: row j = o + kRejOwners i with
// o = j mod kRejOwners, preceded by rows o + kRejOwners i' (i' < i)
__device__ __forceinline__ int own_off(int j) {
  const int o = j % kRejOwners, i = j / kRejOwners;
  return i * (o + 1) + kRejOwners * i * (i - 1) / 2;
}

// x^{-1/2} by one Newton-Raphson step on f(y) = y^{-2} - x,
// y1 = y0 + (y0 / 2)(1 - x y0^2), from the single-precision hardware
// estimate y0: the step squares its relative error (about 2^-22) to below
// 1e-13.  The narrowing of x to float and the widening of y0 and y0/2 back
// are done on the bit patterns (exponent rebased by 1023 - 127; y0 / 2 is
// exact), so that only the three operations of the step use the FP64 pipe.
// FP64 mode takes a second step (about 1 ulp).  Arguments outside
// [1e-30, 1e30] (checked on the bit pattern) take sqrt and divide.
__device__ __forceinline__ bool rsqrt_in_range(double x) {
  // 1e-30 < x < 1e30 on the bit pattern (positive doubles order like integers)
  const long long xb = __double_as_longlong(x);
  return xb > 0x39b4484bfeebc2a0ll && xb < 0x46293e5939a08ceall;
}

// The Newton-Raphson path alone, for x with rsqrt_in_range(x).
__device__ __forceinline__ double rsqrt_core(double x, bool second) {
  const long long xb = __double_as_longlong(x);
  const float xf = __int_as_float((int)((xb >> 29) - (896ll << 23)));
  const float rf = rsqrtf(xf);
  const double y = __longlong_as_double(((long long)__float_as_int(rf) + (896ll << 23)) << 29);
  const double hy =
      __longlong_as_double(((long long)__float_as_int(0.5f * rf) + (896ll << 23)) << 29);
  const double r = fma(-x * y, y, 1.0);
  const double y1 = fma(hy, r, y);
  if (!second) return y1;
  const double r1 = fma(-x * y1, y1, 1.0);
  return fma(0.5 * y1, r1, y1);
}

__device__ __forceinline__ double rsqrt_newton(double x, bool second) {
  if (!rsqrt_in_range(x)) return 1.0 / sqrt(x);
  return rsqrt_core(x, second);
}

// u < h for u >= +0 as an integer comparison of the bit patterns (FP64
// comparisons issue at the FP64 rate); NaN h rejects, like the FP compare.
__device__ __forceinline__ bool accept_bits(long long ub, double h) {
  const long long hb = __double_as_longlong(h);
  return hb <= 0x7ff0000000000000ll && ub < hb;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_to(const void* p, uint32_t cta) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(out)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(cta));
  return out;
}

// Asynchronous store into another CTA's shared memory that completes
// `bytes` of that CTA's barrier's expected transaction count on arrival;
// both addresses already mapped into the receiving CTA's window.
__device__ __forceinline__ void st_async_f64_at(uint32_t dst, double v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(dst),
      "l"(__double_as_longlong(v)), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void st_async_s32(const void* dst, int v, uint64_t* bar,
                                             uint32_t cta) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
          map_to(dst, cta)),
      "r"(v), "r"(map_to(bar, cta))
      : "memory");
}

// This thread's arrival on a barrier of its own CTA, announcing `bytes` of
// asynchronous stores still to come in the current phase.
__device__ __forceinline__ void arrive_expect_local(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait (acquire, cluster scope) for the phase of the given parity of
// a barrier of this CTA: false once `limit_ns` of %globaltimer have passed.
// The clock is read only after the first test has failed.
__device__ __forceinline__ bool wait_cluster_bounded(uint64_t* bar, uint32_t parity,
                                                     unsigned long long limit_ns) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  unsigned long long deadline = 0;
  for (uint32_t n = 0;; ++n) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (n == 0 || (n & 15) == 15) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (n == 0) deadline = now + limit_ns;
      else if (now > deadline) return false;
    }
  }
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared memory of Algorithm 1 in every CTA of the cluster, at the same
// offset in each (the CTAs address each other's copies).
struct RejSmem {
  double lcb[2][kTMax];     // column of accepted pivot t in lcb[t & 1]
  double dg[kTMax];         // lead CTA: current Schur diagonal
  long long ub[kTMax];      // lead CTA: u_i U_i, bit pattern of a non-negative double
  double colbuf[2][kTMax];  // lead: column n_t of H through pivot t-2, pushed
  uint64_t bars[2];         // CTAs 1..: publication p complete in bars[p & 1]
  uint64_t cbar[2];         // lead: column n_t complete in cbar[t & 1]
  int accl[kTMax];
  int nxt_sh[2];
  int ok_sh;
};

// Algorithm 1 on one cluster of kRejCluster CTAs of kRejectThreads threads;
// Hown holds the packed rows this CTA owns (CTAs 1..).
__device__ __forceinline__ void reject_body(RejSmem& R, double* Hown, DevState* st,
                                            const double* H,
                                            const double* uprop,
                                            const double* uacc,
                                            const int* prop, double* Lw, double* L,
                                            int ldL, int* Sacc, long long* piv, int fp64) {
  double(&lcb)[2][kTMax] = R.lcb;
  double(&dg)[kTMax] = R.dg;
  long long(&ub)[kTMax] = R.ub;
  int(&accl)[kTMax] = R.accl;
  int(&nxt_sh)[2] = R.nxt_sh;
  uint64_t(&bars)[2] = R.bars;
  double(&colbuf)[2][kTMax] = R.colbuf;
  uint64_t(&cbar)[2] = R.cbar;
  int& ok_sh = R.ok_sh;
  // every CTA of the cluster reads the same state, so all take the same path
  if (st->done) return;
  const int T = st->T;
  const long long rank = st->rank;
  long long maxacc_ll = st->k - rank;
  const int maxacc = maxacc_ll < T ? (int)maxacc_ll : T;
  const uint32_t cr = cluster_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const bool lead = cr == 0;
  const int own = (int)cr - 1;  // owner index of the rows of this CTA (CTAs 1..)
  constexpr unsigned long long kWait = 2000000000ull;  // 2 s per wait

  if (tid == 0) {
    // one local arrival per phase (with its expected transaction bytes);
    // the data itself arrives by st.async
    uint64_t* b = lead ? cbar : bars;
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&b[i]))
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!lead) arrive_expect_local(&bars[0], 4u);  // publication 0: n_0 alone
  }
  if (lead) {
    const bool block = st->block != 0;
    for (int i = tid; i < T; i += nt) {
      dg[i] = H[(long long)i * T + i];
      long long u;
      if (block) {
        // Algorithm 7: Unique keeps the first draw of each index (threshold
        // +inf: never accepted) and the Cholesky of H takes every other draw
        // whose Schur residual is above the residual floor (a residual at
        // the rounding level is not a pivot)
        const int pi = prop[i];
        bool dup = false;
        for (int j = 0; j < i; ++j) dup |= prop[j] == pi;
        u = dup ? 0x7ff0000000000000ll : __double_as_longlong(fp64 ? kDFloor64 : kDFloorMixed);
      } else {
        u = __double_as_longlong(uprop[i] * uacc[i]);
      }
      ub[i] = u < 0 ? 0 : u;  // -0 -> +0
      lcb[1][i] = 0.0;        // "column -1": no downdate before pivot 0
    }
  } else {
    // rows j = own + kRejOwners i, one warp per row
    for (int j = own + kRejOwners * warp; j < T; j += kRejOwners * nw) {
      const int o = own_off(j);
      for (int l = lane; l <= j; l += 32) Hown[o + l] = H[(long long)j * T + l];
    }
  }
  cluster_sync_all();  // rows loaded and barriers initialised in every CTA

  // first acceptance at or after i0 (lead warp 0), T if none
  auto next_accept = [&](int i0) -> int {
    for (int c = i0; c < T; c += 32) {
      const int i = c + lane;
      const unsigned m = __ballot_sync(0xffffffffu, i < T && accept_bits(ub[i], dg[i]));
      if (m) return c + __ffs(m) - 1;
    }
    return T;
  };
  // publication p to every other CTA: column p - 1 (rows beyond n_{p-1},
  // sent by the lead warps) and n_p (lead warp 0, lane 0), each value an
  // asynchronous store that counts towards the receiver's barrier phase
  auto publish = [&](int p, int nx) {
    for (int c = 1; c < kRejCluster; ++c) st_async_s32(&nxt_sh[p & 1], nx, &bars[p & 1], c);
  };

  int t = 0;
  if (lead) {
    // lcb[0][0] and bars[0] as seen from every other CTA of the cluster
    uint32_t lcb_c[kRejCluster - 1], bars_c[kRejCluster - 1];
#pragma unroll
    for (int c = 1; c < kRejCluster; ++c) {
      lcb_c[c - 1] = map_to(&lcb[0][0], (uint32_t)c);
      bars_c[c - 1] = map_to(&bars[0], (uint32_t)c);
    }
    if (warp < kLeadWarps) {
      if (warp == 0) {
        const int nx = maxacc > 0 ? next_accept(0) : T;
        if (lane == 0) {
          nxt_sh[0] = nx;
          if (nx < T) arrive_expect_local(&cbar[0], 8u * (uint32_t)(T - nx));
          publish(0, nx);
        }
      }
      asm volatile("bar.sync 2, %0;" ::"r"(32 * kLeadWarps) : "memory");
      for (;; ++t) {
        const int n_t = nxt_sh[t & 1];
        if (n_t >= T) break;
        const double* lp = lcb[(t + 1) & 1];  // column of pivot t - 1
        const double lpn = lp[n_t];
        double* lc = lcb[t & 1];
        // 1/sqrt(h) of the pivot (every lead thread forms it from dg,
        // identically) while the rows' owners push column n_t
        const double inv = rsqrt_newton(dg[n_t], fp64);
        if (!wait_cluster_bounded(&cbar[t & 1], (uint32_t)((t >> 1) & 1), kWait)) {
          if (tid == 0) atomicOr(&st->status, (int)kStTimeout);
          break;
        }
        const double* hc = colbuf[t & 1];
        // column t below the pivot; warp 0 owns rows n_t+1..n_t+32, the ones
        // the next acceptance test looks at first
        double dwin = 0.0;
        for (int j = n_t + 1 + tid; j < T; j += 32 * kLeadWarps) {
          const double v = fma(-lp[j], lpn, hc[j]) * inv;
          const double dn = fma(-v, v, dg[j]);
          dg[j] = dn;
          if (j < n_t + 1 + 32 * kLeadWarps) dwin = dn;
          lc[j] = v;
          Lw[(long long)j * kTMax + t] = v;
          const uint32_t off = (uint32_t)(((t & 1) * kTMax + j) * 8);
          const uint32_t boff = (uint32_t)(((t + 1) & 1) * 8);
#pragma unroll
          for (int c = 1; c < kRejCluster; ++c)
            st_async_f64_at(lcb_c[c - 1] + off, v, bars_c[c - 1] + boff);
        }
        if (tid == 32 * kLeadWarps - 1) {  // the pivot's own entry, h / sqrt(h)
          const double v = fma(-lpn, lpn, hc[n_t]) * inv;
          lc[n_t] = v;
          Lw[(long long)n_t * kTMax + t] = v;
        }
        if (warp == 0) {
          // barrier 1: the lead warps' parts of column t are out; barrier 2:
          // warp 0's decision is in nxt_sh
          int nx = T;
          bool waited = false;
          if (t + 1 < maxacc) {
            const int i = n_t + 1 + lane;
            const unsigned m = __ballot_sync(0xffffffffu, i < T && accept_bits(ub[i], dwin));
            if (m) {
              const int src = __ffs(m) - 1;
              nx = n_t + 1 + src;
            } else {
              asm volatile("bar.sync 1, %0;" ::"r"(32 * kLeadWarps) : "memory");
              waited = true;
              nx = next_accept(n_t + 33);
            }
          }
          if (lane == 0) {
            accl[t] = n_t;
            // column n_{t+1} will come from the rows' owners once they have
            // n_{t+1}: expect its bytes before announcing it
            if (nx < T) arrive_expect_local(&cbar[(t + 1) & 1], 8u * (uint32_t)(T - nx));
            publish(t + 1, nx);
            nxt_sh[(t + 1) & 1] = nx;
          }
          if (!waited) asm volatile("bar.sync 1, %0;" ::"r"(32 * kLeadWarps) : "memory");
          __syncwarp();
          asm volatile("bar.arrive 2, %0;" ::"r"(32 * kLeadWarps) : "memory");
        } else {
          asm volatile("bar.arrive 1, %0;" ::"r"(32 * kLeadWarps) : "memory");
          asm volatile("bar.sync 2, %0;" ::"r"(32 * kLeadWarps) : "memory");
        }
      }
    }
  } else {
    const uint32_t colbuf_lead = map_to(&colbuf[0][0], 0u), cbar_lead = map_to(&cbar[0], 0u);
    for (;; ++t) {
      if (tid == 0) ok_sh = wait_cluster_bounded(&bars[t & 1], (uint32_t)((t >> 1) & 1), kWait)
                                ? 1
                                : 0;
      __syncthreads();
      if (!ok_sh) {
        if (tid == 0) atomicOr(&st->status, (int)kStTimeout);
        break;
      }
      const int n_t = nxt_sh[t & 1];
      if (n_t >= T) break;
      {
        // push column n_t of this CTA's rows j >= n_t (downdated through
        // pivot t - 2; the lead applies pivot t - 1 itself) into the lead's
        // colbuf: the st.async bytes complete the lead's barrier phase, which
        // also makes them visible there
        const int i0 = n_t > own ? (n_t - own + kRejOwners - 1) / kRejOwners : 0;
        const int j = own + kRejOwners * (i0 + tid);
        if (j < T)
          st_async_f64_at(colbuf_lead + (uint32_t)(((t & 1) * kTMax + j) * 8),
                          Hown[own_off(j) + n_t], cbar_lead + (uint32_t)((t & 1) * 8));
      }
      // publication t + 1 brings column t for rows n_t+1..T-1 and n_{t+1}
      if (tid == 0) arrive_expect_local(&bars[(t + 1) & 1], 8u * (uint32_t)(T - 1 - n_t) + 4u);
      if (t > 0) {
        // downdate of pivot t - 1 on this CTA's rows j > n_t, columns n_t < l <= j
        const double* lp = lcb[(t + 1) & 1];
        const int i0 = (n_t + 1 - own + kRejOwners - 1) / kRejOwners;  // first owned row > n_t
        for (int j = own + kRejOwners * (i0 + warp); j < T; j += kRejOwners * nw) {
          const int o = own_off(j);
          const double lj = lp[j];
          for (int l = n_t + 1 + lane; l <= j; l += 32) Hown[o + l] = fma(-lj, lp[l], Hown[o + l]);
        }
      }
      __syncthreads();  // the next push reads rows this downdate wrote
    }
  }
  if (lead && tid == 0) ok_sh = t;  // pivots accepted (lead warps 4.. never ran the loop)
  cluster_sync_all();  // no CTA leaves while another may still reach its shared memory
  if (tid == 0) {
    // the barriers' shared memory goes back to other uses
    uint64_t* b = lead ? cbar : bars;
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&b[i]))
                   : "memory");
  }
  if (lead) {
    const int n = ok_sh;
    for (int e = tid; e < n * n; e += nt) {
      const int a = e / n, c = e % n;
      L[(long long)a * ldL + c] = c <= a ? Lw[(long long)accl[a] * kTMax + c] : 0.0;
    }
    for (int a = tid; a < n; a += nt) {
      const int p = prop[accl[a]];
      Sacc[a] = p;
      piv[rank + a] = p;
    }
    __syncthreads();
    if (tid == 0) {
      st->s = n;
      if (n > 0 && !(L[0] > 0.0)) st->status |= kStNumeric;
    }
  }
}

// doubles of packed rows of the CTA of Algorithm 1 that owns the most
__host__ __device__ __forceinline__ size_t reject_own_doubles(int T) {
  size_t most = 0;
  for (int o = 0; o < kRejOwners; ++o) {
    size_t n = 0;
    for (int j = o; j < T; j += kRejOwners) n += (size_t)j + 1;
    if (n > most) most = n;
  }
  return most;
}

}  // namespace rpchol
