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
// Also the one-time split of X into TF32 head and tail planes, and the FP16
// planes of F after a checkpoint restore.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "prep_body.cuh"
#include "tc_ptx.cuh"

namespace rpchol {

__global__ void __launch_bounds__(256) k_prep_tc(const DevState* st, const float* __restrict__ F,
                                                 long long ldF, const float* __restrict__ X,
                                                 int xld, const float* __restrict__ nrm,
                                                 const int* __restrict__ Sacc, unsigned char* Bf,
                                                 unsigned char* Bx, float* nrmS,
                                                 const double* __restrict__ L, int ldL, float* W) {
  __shared__ WblkSmem S;
  prep_block((int)blockIdx.x, S, st, F, ldF, X, xld, nrm, Sacc, Bf, Bx, nrmS, L, ldL, W);
}

__global__ void k_split_x(const float* __restrict__ X, long long n, float* Xh, float* Xl) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = X[i];
  const float h = tc::tf32_head(v);
  Xh[i] = h;
  Xl[i] = v - h;
}

// FP16 head and tail of 4096 F(r, c), c < cols: the split the epilogue of
// the column step writes with every column (same operations, same place:
// the head at 2 (r ldF + c) - (c mod 32), the tail 32 further)
__global__ void k_f16_planes(const float* __restrict__ F, long long ldF, long long N,
                             long long cols, __half* Fs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * cols) return;
  const long long r = i / cols, c = i - r * cols;
  const float y = F[r * ldF + c] * 4096.f;
  const __half h = __float2half_rn(y);
  const long long hi = 2 * (r * ldF + c) - (c & 31);
  Fs[hi] = h;
  Fs[hi + 32] = __float2half_rn(y - __half2float(h));
}

cudaError_t launch_f16_planes(const TcMaps& m, const DevBuffers& b, long long cols,
                              cudaStream_t s) {
  if (cols <= 0) return cudaSuccess;
  const long long n = b.N * cols;
  k_f16_planes<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float*)b.F, b.ldF, b.N, cols,
                                                          (__half*)m.Fsp);
  return cudaGetLastError();
}

cudaError_t launch_prep_tc(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  k_prep_tc<<<kPrepBlocks, 256, 0, s>>>(
      b.st, (const float*)b.F, b.ldF, b.X, b.xld, b.nrm, b.Sacc, m.Bf, m.Bx, m.nrmS, b.L, b.Tmax,
      m.Linv32);
  return cudaGetLastError();
}

cudaError_t launch_split_x(const TcMaps& m, const DevBuffers& b, cudaStream_t s) {
  const long long n = b.N * (long long)b.xld;
  k_split_x<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b.X, n, m.Xhp, m.Xlp);
  return cudaGetLastError();
}

}  // namespace rpchol
