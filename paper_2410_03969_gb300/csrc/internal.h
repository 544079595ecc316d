// Host-side launchers of the rpchol kernels, shared by the library's
// translation units.  Not part of the public ABI (include/rpchol.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rpchol {

// Tensor maps and buffers of the tensor-core column step (mixed mode).
struct TcMaps {
  CUtensorMap Fs;       // FP16 heads / tails of 4096 F, box 64 x 128, 128-byte swizzle
  CUtensorMap Xh, Xl;   // TF32 head / tail planes of X, box 16 x 128, 64-byte swizzle
  void* Fsp;            // N x 2 ldF FP16: row r, 32-column chunk c at 64 c holds the 32
                        // heads, then the 32 tails; written with every column of F
  float* Xhp;
  float* Xlp;
  unsigned char* Bf;    // (ldF / 32) chunk images of F(S,:), 128 x kTMax bytes each
  unsigned char* Bx;    // (xld / 16) chunk images of X_S, 128 x kTMax bytes each
  float* nrmS;          // 256
  float* Linv32;        // W blocks of the round (blocked substitution operand)
  int* err;             // status word of the run state
  int num_sms;          // persistent grid size of the column step
};

cudaError_t launch_prep_tc(const TcMaps& m, const struct DevBuffers& b, cudaStream_t s);
cudaError_t launch_split_x(const TcMaps& m, const struct DevBuffers& b, cudaStream_t s);
// FP16 heads / tails of columns [0, cols) of F from the FP32 factor
// (after a checkpoint restore; the column step writes them with F otherwise)
cudaError_t launch_f16_planes(const TcMaps& m, const struct DevBuffers& b, long long cols,
                              cudaStream_t s);
// The tensor-core column step also closes the round (see round_end_body):
// `cond` / `use_cond` as for launch_round_end.
cudaError_t launch_colstep_tc(const TcMaps& m, const struct DevBuffers& b, unsigned long long cond,
                              int use_cond, cudaStream_t s);

// Buffers of one context that the round kernels touch.  All device memory.
struct DevBuffers {
  long long N;
  int d;          // point dimension
  int xld;        // leading dimension of X (d rounded up to 32, zero padded)
  int kind;       // rpchol_kernel_kind
  double sigma;
  const float* X; // N x xld, FP32
  const float* nrm;  // N, ||x||^2 in FP32 (mixed mode)
  double* dvec;      // N, residual diagonal
  double* tile_sums; // ceil(N / kTileRows)
  double* tile_prefix;
  long long ntiles;
  void* F;           // N x ldF, double (FP64) or float (mixed)
  long long ldF;
  long long* piv;    // k_max
  int* prop;         // T_max proposals of the round
  double* uprop;     // T_max proposal weights d[s'_j]
  double* uacc;      // T_max acceptance uniforms
  double* H;         // T_max x T_max, leading dimension T (of the run)
  double* Lw;        // T_max x T_max work array of Algorithm 1
  double* L;         // compact L of the round, leading dimension T_max
  double* Linv;      // L^{-1} of the round (mixed mode), leading dimension T_max
  int* Sacc;         // accepted pivots of the round
  double* Bext;      // T_max x ldB rows [F(S_j,:) | L(j,:)] (FP64 column step)
  long long ldB;
  float* Bs32;       // mixed mode: T_max x ldBs rows of the column-step operand
  long long ldBs;
  double* Hpart;     // kHPartDoubles: partial products of H, kernel entries
  int* hcnt;         // kHTilesMax arrival counters (zero between launches)
  unsigned* ccnt;    // arrival counter of the tensor-core column step and of the simple
                     // RPCholesky step (zero between launches)
  double* red;       // reduction scratch (trace error)
  long long nred;
  DevState* st;
  int Tmax;
  int mixed;         // 1: F is float
  int num_sms;
};

// End of a loop-body iteration (one round of Algorithm 2, one step of
// Algorithm 6): bookkeeping of the round, the stopping test (rank k reached,
// or the round limit), and the WHILE condition of the graph.  One thread,
// after every kernel of the round has finished with the state.
// `mma_tf32` / `mma_f16`: tensor-core flops the round's column step
// executed (zero for the CUDA-core column steps).
__device__ __forceinline__ void round_end_body(DevState* st, unsigned long long cond, int use_cond,
                                               long long N, int d, int bF, double mma_tf32 = 0.0,
                                               double mma_f16 = 0.0) {
  if (!st->done) {
    const double n = (double)N, r = (double)st->rank, sc = (double)st->s;
    st->col_bytes += n * (r * bF + sc * bF + 4.0 * d + 16.0);
    st->col_flops += 2.0 * n * r * sc + n * sc * sc + 3.0 * n * d * sc;
    st->mma_tf32 += mma_tf32;
    st->mma_f16 += mma_f16;
    st->rank += st->s;
    st->round += 1;
    st->proposals += st->T;
    if (st->rank >= st->k) {
      st->done = 1;
    } else if (st->round >= st->max_rounds) {
      st->done = 1;
      st->status |= kStRoundLimit;
    }
  }
  if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, st->done ? 0u : 1u);
}

// Thread-local message returned by rpchol_last_error (rpchol.cu).
void set_last_error(const char* fmt, ...);

// Round kernels (k_round.cu)
cudaError_t launch_reset(const DevBuffers& b, long long k, int T, unsigned long long seed,
                         unsigned inst, int plain, long long max_rounds, cudaStream_t s);
// reset kernel reading its run parameters from device memory, as a node of g
cudaError_t add_reset_params_node(cudaGraph_t g, const DevBuffers& b, const RunParams* p,
                                  cudaGraphNode_t* out);
cudaError_t launch_propose(const DevBuffers& b, int T, cudaStream_t s);
cudaError_t launch_hmat(const DevBuffers& b, int T, cudaStream_t s);
cudaError_t launch_reject(const DevBuffers& b, int T, cudaStream_t s);
cudaError_t launch_gather_f64(const DevBuffers& b, int T, cudaStream_t s);
cudaError_t launch_round_end(const DevBuffers& b, unsigned long long cond, int use_cond,
                             cudaStream_t s);
cudaError_t launch_trace(const DevBuffers& b, cudaStream_t s);  // writes red[0] = tr(A-FF*)
cudaError_t launch_convert_x64(const double* src, long long N, int d, float* X, int xld,
                               cudaStream_t s);
cudaError_t launch_norms(const DevBuffers& b, cudaStream_t s);
// out (N x cols, dense) = (double) F32(:, 0:cols)
cudaError_t launch_widen_f32(const float* F, long long ldF, long long N, long long cols,
                             double* out, cudaStream_t s);

// CUDA-core column steps (k_colstep_simt.cu): FP64, and FP32 for mixed mode
cudaError_t launch_colstep_f64(const DevBuffers& b, int T, cudaStream_t s);
cudaError_t launch_colstep_f32_simt(const DevBuffers& b, int T, cudaStream_t s);

// Persistent batch engine (k_batch.cu): whether a context can run in it
// (mixed mode with the tensor-core column step), the number of CTAs of a
// launch (whole clusters that fit at once), the device records of a batch's
// contexts, the bytes of the scheduler state (zeroed before every launch),
// and one launch over n instances admitted in the order `order`.
bool engine_supported(const DevBuffers& b, int use_tc);
cudaError_t engine_grid(int* ctas);
cudaError_t engine_setup(int n, const DevBuffers* bs, const TcMaps* ms, void** insts_dev,
                         void** maps_dev, cudaStream_t s);
size_t engine_queue_bytes(int n);
cudaError_t engine_launch(const void* insts_dev, const void* maps_dev, const RunParams* params,
                          const int* order, int n, void* queue, int ctas, cudaStream_t s);

// Simple RPCholesky (k_plain.cu)
// one step after the sampler: GEMV, new column and d; then tile sums and bookkeeping
cudaError_t launch_plain_step(const DevBuffers& b, cudaStream_t s);
cudaError_t launch_plain_tiles(const DevBuffers& b, unsigned long long cond, int use_cond,
                               cudaStream_t s);

}  // namespace rpchol
