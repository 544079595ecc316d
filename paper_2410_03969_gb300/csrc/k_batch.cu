// Persistent batch engine: many uneven instances of accelerated RPCholesky
// (Algorithm 2 with Algorithm 1, arXiv 2410.03969) in one launch.
//
// The grid is made of clusters of kEngCluster CTAs (384 threads each, one
// CTA per SM, as many clusters as fit at once).  The work of an instance's
// round splits into
//   - one control job, run by a whole cluster phase by phase with a cluster
//     barrier between phases: (reset, first round only) sampler -> H ->
//     Algorithm 1 -> operand images and W blocks;
//   - the round's column step, split into `parts` tile parts (part p takes
//     tiles p, p + parts, ...), each run by one CTA; the CTA that finishes
//     the last part closes the round and makes the next control job
//     claimable (or marks the instance finished).
// The lead warp of each cluster schedules its cluster: it claims a control
// job if one is ready (whole cluster), else up to kEngCluster tile parts
// (one per CTA, from any instances), else admits the next instance of the
// host's order (largest expected work first) and runs its first control
// job, and writes each CTA's job into that CTA's shared memory.  Admitted
// instances are scanned in admission order, so the larger ones go first.
//
// Every phase calls the block bodies of the stand-alone kernels
// (round_body.cuh, prep_body.cuh, colstep_body.cuh) with their block
// decomposition; the column step's tiles are independent of the part that
// runs them.  So an instance's result is bit-identical to rpchol_run's.
//
// Waiting: a job never waits for another cluster.  Jobs hand over through
// device-scope release / acquire (the control-job flag and the tile-part
// tickets); the waits inside the phases are bounded as in the stand-alone
// kernels.  A lead warp that finds no work sleeps and polls; after
// kIdleLimitNs without work it stops the engine and marks every unfinished
// instance's run status with the timeout bit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <new>

#include "colstep_body.cuh"
#include "internal.h"
#include "prep_body.cuh"
#include "round_body.cuh"
#include "tc_ptx.cuh"

namespace rpchol {

namespace {
constexpr int kEngThreads = kTcThreads;  // 12 warps: column step with two epilogue groups
constexpr int kEngCluster = kRejCluster;
constexpr int kMinTilesPerPart = 2;
constexpr unsigned long long kIdleLimitNs = 10ull * 1000000000ull;

static_assert(kEngThreads >= kBodyThreads, "the 256-thread bodies need their threads");

// One instance as the engine sees it (device memory).
struct EngineInst {
  DevBuffers b;
  TcArgs ta;  // column-step arguments (no graph condition)
};

// The instance's tensor maps (device memory; CUtensorMap is 64-byte aligned).
struct EngineMaps {
  CUtensorMap Fs, Xh, Xl;
};

// Scheduler state (device memory, zeroed before every launch): the header,
// then one slot per queue position.
struct EngineQueue {
  int admitted;  // queue positions handed out (may pass n)
  int finished;  // instances whose run has stopped
  int abort;     // 1: the idle limit expired, every cluster leaves
  int pad;
};
struct EngineSlot {
  unsigned long long tickets;  // (parts << 32) | next part of the open column step
  int ctrl;                    // 1: the next round's control job can be claimed
  int finished;                // 1: the run has stopped
};
static_assert(sizeof(EngineQueue) == 16 && sizeof(EngineSlot) == 16, "queue layout");

enum : int { kJobNone = 0, kJobCtrl = 1, kJobFirst = 2, kJobTile = 3, kJobExit = 4 };
struct __align__(16) Job {
  int kind, slot, part, parts;
};

// The shared-memory tail the column-step layout leaves free: two job slots
// (double-buffered by iteration), the lead's plan, the TMEM address.
struct EngineTail {
  Job jobs[2];
  Job plan[kEngCluster];
  int pad[20];
  uint32_t tptr;
  uint32_t pad2[3];
};
static_assert(sizeof(EngineTail) == kTailBytes, "tail layout");

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int atom_exch_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.exch.b32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* p,
                                                               unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
               : "=l"(old)
               : "l"(p), "l"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ void put_job(Job* local, uint32_t cta, const Job& j) {
  asm volatile("st.shared::cluster.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(map_to(local, cta)),
               "r"(j.kind), "r"(j.slot), "r"(j.part), "r"(j.parts)
               : "memory");
}

// Between two phases of a control job: every thread's generic writes are
// ordered before later bulk and tensor copies (the column step reads the
// operand images and F through the async proxy) and made visible at device
// scope (tile parts run on other clusters), then the cluster barrier.
__device__ __forceinline__ void phase_sync() {
  tc::fence_proxy_async_all();
  __threadfence();
  cluster_sync_all();
}

__device__ __forceinline__ long long engine_reset_blocks(long long N) {
  long long blocks = (N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  return blocks < 1 ? 1 : blocks;
}

// Tile parts of one round's column step: at least kMinTilesPerPart tiles a
// part, at most one part per CTA of the grid.
__device__ __forceinline__ int tile_parts(long long N, int ctas) {
  const long long ntiles = (N + kBM - 1) / kBM;
  long long per = (ntiles + ctas - 1) / ctas;
  if (per < kMinTilesPerPart) per = kMinTilesPerPart;
  const long long parts = (ntiles + per - 1) / per;
  return parts < 1 ? 1 : (int)parts;
}

// After the round end of slot a's instance (one thread): either the run has
// stopped, or the next round's control job becomes claimable.  The round
// end's state writes are released with the flag.
__device__ __forceinline__ void after_round_end(EngineQueue* q, EngineSlot* slots, int a,
                                                const DevState* st) {
  __threadfence();
  if (*(volatile const int*)&st->done) {
    st_release_s32(&slots[a].finished, 1);
    atomicAdd(&q->finished, 1);
  } else {
    st_release_s32(&slots[a].ctrl, 1);
  }
}
}  // namespace

namespace {

// The lead warp of a cluster: find the cluster's next step and write each
// CTA's job into jobs[buf] of that CTA.  `lo` is the lead warp's first queue
// position that may still be unfinished.
__device__ __noinline__ void decide(EngineQueue* q, EngineSlot* slots, const EngineInst* insts,
                                    const int* order, int n, EngineTail& tl, int buf, int& lo) {
  const int lane = threadIdx.x & 31;
  unsigned long long idle0 = 0;
  for (;;) {
    Job whole = {kJobNone, 0, 0, 0};
    int assigned = 0;
    if (ld_acquire_s32(&q->abort)) whole.kind = kJobExit;
    int A = ld_acquire_s32(&q->admitted);
    if (A > n) A = n;
    // one pass over the admitted positions from lo: the finished prefix is
    // stepped over; a control job (the whole cluster) is taken first,
    // earliest admitted first; else tile parts of open column steps, one per
    // CTA, claimed several at a time with one atomic per instance
    for (int base = lo; whole.kind == kJobNone && assigned < kEngCluster && base < A;
         base += 32) {
      const int a = base + lane;
      const bool in = a < A;
      const int fin = in ? *(volatile const int*)&slots[a].finished : 1;
      const int ctl = in ? *(volatile const int*)&slots[a].ctrl : 0;
      const unsigned long long tk = in ? ld_relaxed_u64(&slots[a].tickets) : 0ull;
      if (base == lo) {
        const unsigned mu = __ballot_sync(0xffffffffu, !fin || !in);
        if (mu != 1u) lo += (mu == 0u ? 32 : __ffs(mu) - 1);  // finished prefix
      }
      unsigned m = __ballot_sync(0xffffffffu, !fin && ctl == 1);
      while (m && assigned == 0) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        int got = 0;
        if (lane == src) got = atom_exch_acq_rel(&slots[a].ctrl, 0) == 1 ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, src);
        if (got) {
          whole = Job{kJobCtrl, base + src, 0, 0};
          break;
        }
      }
      if (whole.kind != kJobNone) break;
      const bool open = !fin && (unsigned)(tk & 0xffffffffull) < (unsigned)(tk >> 32);
      m = __ballot_sync(0xffffffffu, open);
      while (m && assigned < kEngCluster) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        if (lane == src) {
          const unsigned want = (unsigned)(kEngCluster - assigned);
          const unsigned long long old = atom_add_acq_rel(&slots[a].tickets, want);
          const unsigned p = (unsigned)(old & 0xffffffffull), parts = (unsigned)(old >> 32);
          for (unsigned i = 0; i < want && p + i < parts; ++i)
            tl.plan[assigned++] = Job{kJobTile, a, (int)(p + i), (int)parts};
        }
        assigned = __shfl_sync(0xffffffffu, assigned, src);
      }
    }
    // else admit the next instance and run its first control job
    if (whole.kind == kJobNone && assigned == 0 && A < n) {
      int a = n;
      if (lane == 0) a = atomicAdd(&q->admitted, 1);
      a = __shfl_sync(0xffffffffu, a, 0);
      if (a < n) whole = Job{kJobFirst, a, 0, 0};
    }
    if (whole.kind == kJobNone && assigned == 0 && ld_acquire_s32(&q->finished) >= n)
      whole.kind = kJobExit;
    if (whole.kind != kJobNone || assigned > 0) {
      __syncwarp();
      if (lane < kEngCluster) {
        const Job none = {kJobNone, 0, 0, 0};
        put_job(&tl.jobs[buf], (uint32_t)lane,
                whole.kind != kJobNone ? whole : (lane < assigned ? tl.plan[lane] : none));
      }
      return;
    }
    // nothing to do yet: poll, up to the idle limit
    const unsigned long long now = tc::globaltimer_ns();
    if (idle0 == 0) {
      idle0 = now;
    } else if (now - idle0 > kIdleLimitNs) {
      if (lane == 0) atomicExch(&q->abort, 1);
      for (int a = lane; a < n; a += 32)
        if (!ld_acquire_s32(&slots[a].finished))
          atomicOr(&insts[order[a]].b.st->status, (int)kStTimeout);
      continue;  // the next pass sees the abort flag
    }
    __nanosleep(256);
  }
}

// One round's control job of queue position J.slot on the whole cluster.
__device__ __forceinline__ void control_job(const Job& J, const EngineInst* insts,
                                            const RunParams* params, const int* order,
                                            EngineQueue* q, EngineSlot* slots, unsigned char* sm,
                                            uint32_t cr, int ctas) {
  const int ii = order[J.slot];
  const EngineInst& I = insts[ii];
  const DevBuffers& b = I.b;
  const RunParams& P = params[ii];
  DevState* st = b.st;
  const int tid = threadIdx.x;
  if (J.kind == kJobFirst) {  // reset: d = 1, tile sums, run state
    const long long nb = engine_reset_blocks(b.N);
    for (long long blk = cr; blk < nb; blk += kEngCluster)
      reset_run(st, b.dvec, b.tile_sums, b.N, b.ntiles, P.k, P.T, P.seed, P.instance, 0,
                P.max_rounds, blk, nb);
    phase_sync();
  }
  const int T = P.T;
  // ---- step 1: proposals (256-thread body)
  if (tid < kBodyThreads) {
    const int use_smem = b.ntiles * (long long)sizeof(double) <= 160 * 1024 ? 1 : 0;
    double* wsum = (double*)sm;
    double* pref = (double*)(sm + 64);
    for (int blk = (int)cr; blk < (T + 7) / 8; blk += kEngCluster) {
      propose_body(blk, pref, wsum, st, b.dvec, b.tile_sums, b.tile_prefix, b.ntiles, b.N,
                   b.prop, b.uprop, b.uacc, use_smem, b.F, b.ldF, 0);
      body_sync();
    }
  }
  phase_sync();
  // ---- step 2: H = A(S',S') - F(S',:) F(S',:)^* (256-thread body)
  if (tid < kBodyThreads) {
    const int nblk = hmat32_blocks(T), ks = hmat32_splits(nblk);
    H32Smem& S = *(H32Smem*)sm;
    for (int it = (int)cr; it < nblk * ks; it += kEngCluster) {
      hmat32_body(it / ks, it % ks, ks, S, st, b.X, b.xld, b.d, b.kind, 1.0 / b.sigma,
                  (const float*)b.F, b.ldF, b.prop, b.H, b.Hpart, b.hcnt);
      body_sync();
    }
  }
  phase_sync();
  // ---- Algorithm 1 on the cluster (every thread)
  {
    RejSmem& R = *(RejSmem*)sm;
    double* Hown = (double*)(sm + ((sizeof(RejSmem) + 15) & ~(size_t)15));
    reject_body(R, Hown, st, b.H, b.uprop, b.uacc, b.prop, b.Lw, b.L, b.Tmax, b.Sacc, b.piv, 0);
  }
  phase_sync();
  // a round that ended early (nothing accepted, or the sampler found no
  // weight) closes here, as the column step would close it
  if (*(volatile int*)&st->done || *(volatile int*)&st->s == 0) {
    if (cr == 0 && tid == 0) {
      round_end_body(st, I.ta.cond, I.ta.use_cond, I.ta.N, I.ta.d, 4);
      after_round_end(q, slots, J.slot, st);
    }
    return;
  }
  // ---- operand images (every thread, rows cr, cr + 8, ...) and W blocks
  // (256-thread body, blocks cr, cr + 8, ...): the bytes the stand-alone
  // prep writes
  prep_rows_strided(st, (const float*)b.F, b.ldF, b.X, b.xld, b.nrm, b.Sacc,
                    (unsigned char*)I.ta.Bf, (unsigned char*)I.ta.Bx, (float*)I.ta.nrmS, (int)cr,
                    kEngCluster);
  if (tid < kBodyThreads) {
    WblkSmem& S = *(WblkSmem*)sm;
    for (int wb = (int)cr; wb < kTMax / 16; wb += kEngCluster) {
      wblk_full(S, st, b.L, b.Tmax, (float*)I.ta.W, wb);
      body_sync();
    }
  }
  phase_sync();
  // ---- open the column step: its tile parts go to any CTA
  if (cr == 0 && tid == 0)
    st_release_u64(&slots[J.slot].tickets, (unsigned long long)tile_parts(b.N, ctas) << 32);
}
}  // namespace

__global__ void __cluster_dims__(kEngCluster, 1, 1) __launch_bounds__(kEngThreads, 1)
    k_batch_engine(const EngineInst* insts, const EngineMaps* maps, const RunParams* params,
                   const int* order, int n, EngineQueue* q) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  EngineTail& tl = *(EngineTail*)(smem_raw + kSmemMax - kTailBytes);
  EngineSlot* slots = (EngineSlot*)(q + 1);
  const uint32_t cr = cluster_rank();
  const int warp = threadIdx.x >> 5;
  const int ctas = (int)gridDim.x;
  if (warp == 1) {
    tc::tmem_alloc(&tl.tptr, 512);
    tc::tmem_relinquish();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tl.tptr;
  int lo = 0;  // lead warp's scan start
  cluster_sync_all();  // every CTA runs before the lead writes into its shared memory
  for (int it = 0;; ++it) {
    // jobs[it & 1] is rewritten two steps later, after every CTA passed the
    // barrier of the next step: one barrier a step suffices
    const int buf = it & 1;
    if (cr == 0 && warp == 0) decide(q, slots, insts, order, n, tl, buf, lo);
    cluster_sync_all();
    const Job J = tl.jobs[buf];
    if (J.kind == kJobExit) break;
    if (J.kind == kJobCtrl || J.kind == kJobFirst) {
      control_job(J, insts, params, order, q, slots, sm, cr, ctas);
    } else if (J.kind == kJobTile) {
      const int ii = order[J.slot];
      // the operand images and F were written by generic stores elsewhere
      tc::fence_proxy_async_all();
      const bool closed = colstep_body(&maps[ii].Fs, &maps[ii].Xh, &maps[ii].Xl, insts[ii].ta, sm,
                                       tbase, J.part, J.parts);
      if (closed) after_round_end(q, slots, J.slot, insts[ii].b.st);
    }
  }
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

bool engine_supported(const DevBuffers& b, int use_tc) {
  return use_tc && b.mixed && b.N >= kBM && b.Tmax <= kTMax &&
         (b.ntiles * (long long)sizeof(double) <= 160 * 1024 || b.tile_prefix != nullptr);
}

cudaError_t engine_grid(int* ctas) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_engine,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nsm / kEngCluster * kEngCluster));
  cfg.blockDim = dim3(kEngThreads);
  cfg.dynamicSmemBytes = kSmemMax;
  cfg.attrs = nullptr;  // the cluster shape is the kernel's own (__cluster_dims__)
  cfg.numAttrs = 0;
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, (void*)k_batch_engine, &cfg);
  if (e != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  *ctas = clusters * kEngCluster;
  return cudaSuccess;
}

cudaError_t engine_setup(int n, const DevBuffers* bs, const TcMaps* ms, void** insts_dev,
                         void** maps_dev, cudaStream_t s) {
  EngineInst* hi = new (std::nothrow) EngineInst[n];
  EngineMaps* hm = new (std::nothrow) EngineMaps[n];
  if (!hi || !hm) {
    delete[] hi;
    delete[] hm;
    return cudaErrorMemoryAllocation;
  }
  for (int i = 0; i < n; ++i) {
    hi[i].b = bs[i];
    hi[i].ta = make_tc_args(ms[i], bs[i], 0ull, 0);
    hm[i].Fs = ms[i].Fs;
    hm[i].Xh = ms[i].Xh;
    hm[i].Xl = ms[i].Xl;
  }
  cudaError_t e = cudaMalloc(insts_dev, sizeof(EngineInst) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(maps_dev, sizeof(EngineMaps) * (size_t)n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(*insts_dev, hi, sizeof(EngineInst) * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(*maps_dev, hm, sizeof(EngineMaps) * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  delete[] hi;
  delete[] hm;
  return e;
}

size_t engine_queue_bytes(int n) {
  return sizeof(EngineQueue) + sizeof(EngineSlot) * (size_t)(n > 0 ? n : 0);
}

cudaError_t engine_launch(const void* insts_dev, const void* maps_dev, const RunParams* params,
                          const int* order, int n, void* queue, int ctas, cudaStream_t s) {
  k_batch_engine<<<(unsigned)ctas, kEngThreads, kSmemMax, s>>>(
      (const EngineInst*)insts_dev, (const EngineMaps*)maps_dev, params, order, n,
      (EngineQueue*)queue);
  return cudaGetLastError();
}

}  // namespace rpchol
