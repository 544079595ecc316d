// Per-round operand preparation for the tensor-core column step (mixed
// mode), Algorithm 2 step 3 of arXiv 2410.03969:
//   - the B operands of the round as the exact shared-memory images the
//     column step's MMAs read, one contiguous image per K chunk (loaded with
//     one bulk copy): for chunk c of the Schur part, rows j < s_pad of
//     [head | tail] of -4096 F(S_j, 32 c .. 32 c + 31) in FP16 (64-byte rows,
//     64-byte swizzle); for chunk c of the distance part, rows j < s_pad of
//     [head | tail] of x_{S_j}(16 c .. 16 c + 15) as TF32 planes (64-byte
//     rows, 64-byte swizzle).  Rows j >= s and columns >= rank are zero, so
//     padded MMA columns and the columns of F not yet formed contribute
//     nothing;
//   - ||x_{S_j}||^2;
//   - the blocked-substitution operand W built from the round's compact
//     Cholesky factor L in FP64 and rounded once to FP32 (wblk below), in
//     the same launch.
//
// Device-side bodies (block by block), shared by the stand-alone kernel
// (k_prep_tc.cu) and the persistent batch engine (k_batch.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rpchol {

// Byte offset of the 16-byte piece q (0..3) of row j in a 64-byte-row image
// with the 64-byte swizzle (piece q of row j sits at q ^ ((j >> 1) & 3)).
__device__ __forceinline__ int sw64_off(int j, int q) { return j * 64 + 16 * (q ^ ((j >> 1) & 3)); }

// Piece q (8 columns) of chunk c of row j of the F image: FP16 head and
// tail of -4096 F(S_j, 32 c + 8 q ..), zero beyond the rank or for padded
// rows (frow null).
__device__ __forceinline__ void prep_f_piece(const float* frow, long long rank, int j, int c, int q,
                                             unsigned char* Bf, size_t cb, int s_pad) {
  const long long col = 32ll * c + 8 * q;
  float v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = (frow && col + e < rank) ? -4096.f * frow[col + e] : 0.f;
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __half2 h = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
    hw[e] = *(const uint32_t*)&h;
    lw[e] = *(const uint32_t*)&l;
  }
  unsigned char* base = Bf + (size_t)c * cb + sw64_off(j, q);
  *(uint4*)base = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *(uint4*)(base + 64 * s_pad) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Piece q (4 columns) of chunk c of row j of the X image: TF32 head and tail.
__device__ __forceinline__ void prep_x_piece(const float* xrow, int j, int c, int q,
                                             unsigned char* Bx, size_t cb, int s_pad) {
  const int col = 16 * c + 4 * q;
  float h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float v = xrow ? xrow[col + e] : 0.f;
    h[e] = tc::tf32_head(v);
    l[e] = v - h[e];
  }
  unsigned char* base = Bx + (size_t)c * cb + sw64_off(j, q);
  *(float4*)base = make_float4(h[0], h[1], h[2], h[3]);
  *(float4*)(base + 64 * s_pad) = make_float4(l[0], l[1], l[2], l[3]);
}

// Row j of the B images (one CTA per row).
__device__ __forceinline__ void prep_row(const DevState* st, const float* F,
                                         long long ldF, const float* X, int xld,
                                         const float* nrm,
                                         const int* Sacc, unsigned char* Bf,
                                         unsigned char* Bx, float* nrmS, int j) {
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const int s_pad = (s + 15) & ~15;
  if (j >= s_pad) return;
  const size_t cb = 128 * (size_t)s_pad;  // bytes of one chunk image
  const int nF = (int)((rank + 31) >> 5);
  const int nXc = xld >> 4;
  const int p = j < s ? Sacc[j] : -1;
  const float* frow = p >= 0 ? F + (long long)p * ldF : nullptr;
  const float* xrow = p >= 0 ? X + (long long)p * xld : nullptr;
  for (int it = threadIdx.x; it < 4 * nF; it += blockDim.x)
    prep_f_piece(frow, rank, j, it >> 2, it & 3, Bf, cb, s_pad);
  for (int it = threadIdx.x; it < 4 * nXc; it += blockDim.x)
    prep_x_piece(xrow, j, it >> 2, it & 3, Bx, cb, s_pad);
  if (threadIdx.x == 0) nrmS[j] = p >= 0 ? nrm[p] : 0.f;
}

// Rows first, first + step, ... < s_pad of the B images in one pass of the
// whole CTA (any thread count): the bytes prep_row writes for those rows.
__device__ __forceinline__ void prep_rows_strided(const DevState* st, const float* F,
                                                  long long ldF, const float* X, int xld,
                                                  const float* nrm, const int* Sacc,
                                                  unsigned char* Bf, unsigned char* Bx,
                                                  float* nrmS, int first, int step) {
  const int s = st->s;
  if (s == 0) return;
  const long long rank = st->rank;
  const int s_pad = (s + 15) & ~15;
  if (first >= s_pad) return;
  const size_t cb = 128 * (size_t)s_pad;
  const int nF = (int)((rank + 31) >> 5);
  const int nXc = xld >> 4;
  const int nrows = (s_pad - first + step - 1) / step;
  const int per = 4 * nF + 4 * nXc;
  for (int it = threadIdx.x; it < nrows * per; it += blockDim.x) {
    const int r = it / per, k = it - r * per;
    const int j = first + r * step;
    const int p = j < s ? Sacc[j] : -1;
    if (k < 4 * nF)
      prep_f_piece(p >= 0 ? F + (long long)p * ldF : nullptr, rank, j, k >> 2, k & 3, Bf, cb,
                   s_pad);
    else
      prep_x_piece(p >= 0 ? X + (long long)p * xld : nullptr, j, (k - 4 * nF) >> 2,
                   (k - 4 * nF) & 3, Bx, cb, s_pad);
  }
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    const int j = first + r * step;
    const int p = j < s ? Sacc[j] : -1;
    nrmS[j] = p >= 0 ? nrm[p] : 0.f;
  }
}

// Blocked forward substitution operand for G L^* = R.  With the columns in
// blocks of 16 (block b covers columns j0 = 16 b .. j0 + 15) and D_b the
// 16 x 16 diagonal block of L, block b of G is
//   G_b = D_b^{-1} (R_b - G_{<j0} L(b, <j0)^*)
//       = sum_{l < j0} G(:, l) W_b(l, :) + sum_{m < 16} R(:, j0 + m) W_b(j0 + m, :)
// with W_b(l, jj) = -(D_b^{-1} L(b, <j0))(jj, l) for l < j0 and
// W_b(j0 + m, jj) = D_b^{-1}(jj, m).  All of it is formed here in FP64 from
// the FP64 L of Algorithm 1 and rounded once to FP32.  Block b occupies
// (j0 + 16) x 16 floats at offset 256 b (b + 1) / 2, row l contiguous, its
// columns in wpos order.
// Rows and columns of L beyond s are taken as the identity, so padded
// columns of G are copies of the (zero) padded columns of R.
// One CTA per block b and part of the range l < j0 (part 0 also writes the
// diagonal rows).  Each CTA forms D_b^{-1} itself, by rows (row c is final
// once rows < c are), one step per row for the whole CTA.
// Column jj of row l of a 16-column W block is stored at position
// wpos(l, jj): the four columns quad lane c of the column step's epilogue
// owns (2c, 2c + 1, 8 + 2c, 9 + 2c) form one 16-byte group, and group c
// sits at group slot c ^ ((l >> 1) & 3), so that the four lanes of a quad,
// which read four rows l two apart, hit four different bank groups.
__device__ __forceinline__ int wpos(int l, int jj) {
  return 4 * (((jj & 7) >> 1) ^ ((l >> 1) & 3)) + 2 * (jj >> 3) + (jj & 1);
}

struct WblkSmem {
  double Db[16][17];
  double acc[16][17];
  double Dinv[16][17];
  double rdiag[16];
  double Lb[16][33];  // rows j0..j0+15 of L, columns l0..l1-1
};

__device__ __forceinline__ void wblk(WblkSmem& S, const DevState* st,
                                     const double* L, int ldL, float* W, int b,
                                     int part, int nparts) {
  double(&Db)[16][17] = S.Db;
  double(&acc)[16][17] = S.acc;
  double(&Dinv)[16][17] = S.Dinv;
  double(&rdiag)[16] = S.rdiag;
  double(&Lb)[16][33] = S.Lb;
  const int s = st->s;
  const int j0 = 16 * b;
  if (j0 >= s) return;
  const int per = (j0 + nparts - 1) / nparts;  // <= 32
  const int l0 = part * per;
  const int l1 = l0 + per < j0 ? l0 + per : j0;
  if (part > 0 && l0 >= l1) return;
  const int nl = l1 > l0 ? l1 - l0 : 0;
  const int t = threadIdx.x, r = t >> 4, m = t & 15;
  auto Lat = [&](int rr, int cc) -> double {  // L with identity padding beyond s
    if (rr >= s || cc >= s) return rr == cc ? 1.0 : 0.0;
    return cc <= rr ? L[(long long)rr * ldL + cc] : 0.0;
  };
  Db[r][m] = Lat(j0 + r, j0 + m);
  acc[r][m] = r == m ? 1.0 : 0.0;
  if (t < 16) rdiag[t] = 1.0 / Lat(j0 + t, j0 + t);
  for (int e = t; e < 16 * nl; e += 256) Lb[e / nl][e % nl] = Lat(j0 + e / nl, l0 + e % nl);
  body_sync();
  // D_b^{-1}(c, :) = (e_c - sum_{c' < c} D_b(c, c') D_b^{-1}(c', :)) / D_b(c, c)
  for (int c = 0; c < 16; ++c) {
    if (r >= c) {
      const double xc = acc[c][m] * rdiag[c];
      if (r == c) Dinv[c][m] = xc;
      else acc[r][m] = fma(-Db[r][c], xc, acc[r][m]);
    }
    body_sync();
  }
  float* Wb = W + 256 * (long long)b * (b + 1) / 2;
  for (int e = t; e < 16 * nl; e += 256) {  // W_b(l, jj), l0 <= l < l1
    const int l = e >> 4, jj = e & 15;
    double a = 0.0;
    for (int mm = 0; mm <= jj; ++mm) a = fma(Dinv[jj][mm], Lb[mm][l], a);
    Wb[(long long)(l0 + l) * 16 + wpos(l0 + l, jj)] = (float)(-a);
  }
  if (part == 0)  // W_b(j0 + m, jj) = D_b^{-1}(jj, m)
    Wb[(long long)(j0 + r) * 16 + wpos(j0 + r, m)] = (float)Dinv[m][r];
}

// All of W block b in one pass of 256 threads: D_b^{-1} once, then the
// range l < j0 in pieces of 32 columns; every entry comes from the same
// FP64 operations in the same order as in wblk, so the bytes are the same.
__device__ __forceinline__ void wblk_full(WblkSmem& S, const DevState* st, const double* L,
                                          int ldL, float* W, int b) {
  double(&Db)[16][17] = S.Db;
  double(&acc)[16][17] = S.acc;
  double(&Dinv)[16][17] = S.Dinv;
  double(&rdiag)[16] = S.rdiag;
  double(&Lb)[16][33] = S.Lb;
  const int s = st->s;
  const int j0 = 16 * b;
  if (j0 >= s) return;
  const int t = threadIdx.x, r = t >> 4, m = t & 15;
  auto Lat = [&](int rr, int cc) -> double {  // L with identity padding beyond s
    if (rr >= s || cc >= s) return rr == cc ? 1.0 : 0.0;
    return cc <= rr ? L[(long long)rr * ldL + cc] : 0.0;
  };
  Db[r][m] = Lat(j0 + r, j0 + m);
  acc[r][m] = r == m ? 1.0 : 0.0;
  if (t < 16) rdiag[t] = 1.0 / Lat(j0 + t, j0 + t);
  body_sync();
  for (int c = 0; c < 16; ++c) {
    if (r >= c) {
      const double xc = acc[c][m] * rdiag[c];
      if (r == c) Dinv[c][m] = xc;
      else acc[r][m] = fma(-Db[r][c], xc, acc[r][m]);
    }
    body_sync();
  }
  float* Wb = W + 256 * (long long)b * (b + 1) / 2;
  for (int l0 = 0; l0 < j0; l0 += 32) {
    const int nl = j0 - l0 < 32 ? j0 - l0 : 32;
    for (int e = t; e < 16 * nl; e += 256) Lb[e / nl][e % nl] = Lat(j0 + e / nl, l0 + e % nl);
    body_sync();
    for (int e = t; e < 16 * nl; e += 256) {
      const int l = e >> 4, jj = e & 15;
      double a = 0.0;
      for (int mm = 0; mm <= jj; ++mm) a = fma(Dinv[jj][mm], Lb[mm][l], a);
      Wb[(long long)(l0 + l) * 16 + wpos(l0 + l, jj)] = (float)(-a);
    }
    body_sync();
  }
  Wb[(long long)(j0 + r) * 16 + wpos(j0 + r, m)] = (float)Dinv[m][r];
}

// One launch for both: CTAs [0, kTMax) prepare the rows of the B operands,
// CTAs [kTMax, kTMax + 8 kTMax / 16) form the W blocks (block b, part p at
// kTMax + 8 b + p).  The two have no data in common and run side by side.
constexpr int kWParts = 8;
constexpr int kPrepBlocks = kTMax + kWParts * (kTMax / 16);

// Block blk of the operand prep (256 threads): rows of the B images for
// blk < kTMax, W blocks after.
__device__ __forceinline__ void prep_block(int blk, WblkSmem& S, const DevState* st,
                                           const float* F, long long ldF,
                                           const float* X, int xld,
                                           const float* nrm,
                                           const int* Sacc, unsigned char* Bf,
                                           unsigned char* Bx, float* nrmS,
                                           const double* L, int ldL, float* W) {
  if (st->done) return;
  if (blk < kTMax) {
    prep_row(st, F, ldF, X, xld, nrm, Sacc, Bf, Bx, nrmS, blk);
  } else {
    const int i = blk - kTMax;
    wblk(S, st, L, ldL, W, i / kWParts, i % kWParts, kWParts);
  }
}

}  // namespace rpchol
