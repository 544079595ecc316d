// C ABI and runtime of the rpchol library: contexts, device memory, the
// round loop as a CUDA graph with a device-evaluated while-condition, and
// result access.  The ABI is declared in include/rpchol.h.
//
// Paper: Epperly, Tropp, Webber, arXiv 2410.03969 (Algorithms 1, 2, 6).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <new>
#include <vector>
#include <atomic>

#include "../../include/rpchol.h"
#include "internal.h"
#include "selftest.h"

using namespace rpchol;

namespace {

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

}  // namespace

void rpchol::set_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace {

rpchol_status cuda_fail(cudaError_t e, const char* where) {
  set_err("%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RPCHOL_ENOMEM : RPCHOL_ECUDA;
}

#define CU(call)                                   \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct ProfRec {
  int slot;
  long long iter;
  cudaEvent_t a, b;
};

}  // namespace

struct rpchol_ctx {
  DevBuffers b{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to record graphs
  int precision = RPCHOL_FP64;
  int use_graph = 1;
  unsigned instance = 0;
  long long k_max = 0;
  rpchol_alloc_fn alloc = nullptr;
  rpchol_free_fn release = nullptr;
  void* alloc_user = nullptr;
  std::vector<void*> owned;
  std::map<long long, GraphEntry> graphs;  // key: plain * 1024 + T
  DevState* st_host = nullptr;             // pinned mirror
  int last_plain = 0;
  int has_run = 0;
  long long host_iters = -1;  // loop bodies the host loop launched (-1: graph)
  int profile = 0;
  std::vector<ProfRec> prof;  // events of the last profiled run
  int* gate_host = nullptr;   // profile mode: pinned, mapped release flag of the stream gate
  int* gate_dev = nullptr;
  int gate_gen = 0;
  int use_tc = 0;             // mixed mode: tensor-core column step
  TcMaps tc{};
  // rpchol_run_to_host: copy stream, pinned mapped ring of state snapshots
  // (one per round in flight) and the events that mark each round done
  cudaStream_t copy_stream = nullptr;
  DevState* snap_host = nullptr;
  cudaEvent_t snap_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t copy_ev = nullptr;
  std::atomic<long long> copies_landed{0};  // 2-D copies the copy stream has finished
};

namespace {

rpchol_status dev_alloc(rpchol_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->alloc) {
    *p = c->alloc(bytes, (void*)c->stream, c->alloc_user);
    if (!*p) {
      set_err("device allocation of %zu bytes failed", bytes);
      return RPCHOL_ENOMEM;
    }
  } else {
    cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  }
  c->owned.push_back(*p);
  return RPCHOL_OK;
}

void clear_prof(rpchol_ctx* c);

void release_all(rpchol_ctx* c) {
  clear_prof(c);
  for (auto& kv : c->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  c->graphs.clear();
  for (void* p : c->owned) {
    if (c->release) c->release(p, (void*)c->stream, c->alloc_user);
    else cudaFreeAsync(p, c->stream);
  }
  c->owned.clear();
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->st_host) cudaFreeHost(c->st_host);
  c->st_host = nullptr;
  if (c->gate_host) cudaFreeHost(c->gate_host);
  c->gate_host = nullptr;
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  c->copy_stream = nullptr;
  for (cudaEvent_t& e : c->snap_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (c->copy_ev) cudaEventDestroy(c->copy_ev);
  c->copy_ev = nullptr;
  if (c->snap_host) cudaFreeHost(c->snap_host);
  c->snap_host = nullptr;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D map over a row-major (rows x inner) FP32 (or FP16, `half`) array with
// leading dimension `inner`, box box_inner x box_rows, the given swizzle,
// zero fill.
rpchol_status make_map(CUtensorMap* m, const void* base, unsigned long long inner,
                       unsigned long long rows, unsigned box_inner, unsigned box_rows,
                       CUtensorMapSwizzle swz, bool half = false) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    set_err("cuTensorMapEncodeTiled is unavailable");
    return RPCHOL_ECUDA;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * (half ? 2ull : 4ull)};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = enc(m, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(base), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_err("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RPCHOL_ECUDA;
  }
  return RPCHOL_OK;
}

// Phases of one loop-body iteration (profile-mode event slots):
// 0 propose, 1 H, 2 Algorithm 1, 3 operand prep, 4 column step, 5 round end,
// 6 simple-RPC GEMV (new column and d), 7 simple-RPC finish (scaling, d, tile sums, step end).

struct Phase {
  int slot;
  cudaError_t (*fn)(rpchol_ctx*, int, unsigned long long, int, cudaStream_t);
};

cudaError_t ph_propose(rpchol_ctx* c, int T, unsigned long long, int, cudaStream_t s) {
  return launch_propose(c->b, T, s);
}
cudaError_t ph_hmat(rpchol_ctx* c, int T, unsigned long long, int, cudaStream_t s) {
  return launch_hmat(c->b, T, s);
}
cudaError_t ph_reject(rpchol_ctx* c, int T, unsigned long long, int, cudaStream_t s) {
  return launch_reject(c->b, T, s);
}
cudaError_t ph_prep(rpchol_ctx* c, int T, unsigned long long, int, cudaStream_t s) {
  if (c->use_tc) return launch_prep_tc(c->tc, c->b, s);
  return launch_gather_f64(c->b, T, s);
}
cudaError_t ph_colstep(rpchol_ctx* c, int T, unsigned long long cond, int use_cond,
                       cudaStream_t s) {
  if (c->precision == RPCHOL_FP64) return launch_colstep_f64(c->b, T, s);
  if (c->use_tc) return launch_colstep_tc(c->tc, c->b, cond, use_cond, s);
  return launch_colstep_f32_simt(c->b, T, s);
}
cudaError_t ph_round_end(rpchol_ctx* c, int, unsigned long long cond, int use_cond,
                         cudaStream_t s) {
  if (c->use_tc) return cudaSuccess;  // the tensor-core column step closed the round
  return launch_round_end(c->b, cond, use_cond, s);
}
cudaError_t ph_plain_step(rpchol_ctx* c, int, unsigned long long, int, cudaStream_t s) {
  return launch_plain_step(c->b, s);
}
cudaError_t ph_plain_tiles(rpchol_ctx* c, int, unsigned long long cond, int use_cond,
                           cudaStream_t s) {
  return launch_plain_tiles(c->b, cond, use_cond, s);
}

const Phase kAccelPhases[] = {{0, ph_propose}, {1, ph_hmat},    {2, ph_reject},
                              {3, ph_prep},    {4, ph_colstep}, {5, ph_round_end}};
const Phase kPlainPhases[] = {{0, ph_propose}, {6, ph_plain_step}, {7, ph_plain_tiles}};

// One iteration of the loop body: one round of Algorithm 2, or one step of
// Algorithm 6.  With `ev` (profile mode) every phase is bracketed by a pair
// of events recorded on the launch stream.
cudaError_t launch_body(rpchol_ctx* c, int plain, int T, unsigned long long cond, int use_cond,
                        cudaStream_t s, std::vector<ProfRec>* ev = nullptr, long long iter = 0) {
  const Phase* ph = plain ? kPlainPhases : kAccelPhases;
  const int n = plain ? 3 : 6;
  for (int i = 0; i < n; ++i) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (ev) {
      cudaError_t e = cudaEventCreate(&a);
      if (e == cudaSuccess) e = cudaEventCreate(&b);
      if (e != cudaSuccess) return e;
      if ((e = cudaEventRecord(a, s)) != cudaSuccess) return e;
    }
    cudaError_t e = ph[i].fn(c, T, cond, use_cond, s);
    if (e != cudaSuccess) return e;
    if (ev) {
      if ((e = cudaEventRecord(b, s)) != cudaSuccess) return e;
      ev->push_back({ph[i].slot, iter, a, b});
    }
  }
  return cudaSuccess;
}

rpchol_status get_graph(rpchol_ctx* c, int plain, int T, cudaGraphExec_t* out) {
  const long long key = (long long)plain * 1024 + T;
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    *out = it->second.exec;
    return RPCHOL_OK;
  }
  GraphEntry ge;
  CU(cudaGraphCreate(&ge.graph, 0));
  cudaGraphConditionalHandle h;
  CU(cudaGraphConditionalHandleCreate(&h, ge.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, ge.graph, nullptr, nullptr, 0, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  CU(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  cudaError_t le = launch_body(c, plain, T, (unsigned long long)h, 1, c->cap_stream);
  cudaGraph_t captured = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &captured);
  if (le != cudaSuccess) return cuda_fail(le, "capture of the round body");
  if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
  CU(cudaGraphInstantiate(&ge.exec, ge.graph, 0));
  c->graphs[key] = ge;
  *out = ge.exec;
  return RPCHOL_OK;
}

// Profile mode holds the stream at a gate until a whole chunk of rounds (the
// kernels and the events around them) is enqueued, so that the events time
// the kernels back to back rather than the host's enqueue rate.  The gate
// polls a pinned host flag for at most about a second; if it gives up, it
// sets kStGateExpired in the run status (the phase times of that run then
// include host enqueue time, and the run reports RPCHOL_ETIMEOUT).
__global__ void k_gate(const int* flag, int target, int* status) {
  for (int i = 0; i < 1000000; ++i) {
    int v;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= target) return;
    __nanosleep(1000);
  }
  atomicOr(status, (int)kStGateExpired);
}

void clear_prof(rpchol_ctx* c) {
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->prof.clear();
}

// mode 0: accelerated (Algorithm 2), 1: simple (Algorithm 6), 2: block (Algorithm 7, the
// accelerated loop body with the acceptance rule switched in the device state)
rpchol_status run_loop(rpchol_ctx* c, int plain, int T, long long max_rounds);

rpchol_status run_common(rpchol_ctx* c, int mode, long long k, int T, unsigned long long seed) {
  const int plain = mode == 1;
  const long long max_rounds = plain ? 2 * k + 64 : 4 * k + 64;
  clear_prof(c);
  CU(launch_reset(c->b, k, T, seed, c->instance, mode, max_rounds, c->stream));
  c->last_plain = plain;
  c->has_run = 1;
  return run_loop(c, plain, T, max_rounds);
}

// The round loop of a run whose device state is set (fresh or resumed).
rpchol_status run_loop(rpchol_ctx* c, int plain, int T, long long max_rounds) {
  c->host_iters = -1;
  if (c->use_graph && !c->profile) {
    cudaGraphExec_t ex;
    rpchol_status st = get_graph(c, plain, T, &ex);
    if (st != RPCHOL_OK) return st;
    CU(cudaGraphLaunch(ex, c->stream));
    return RPCHOL_OK;
  }
  if (c->profile && !c->gate_host) {
    CU(cudaHostAlloc((void**)&c->gate_host, sizeof(int), cudaHostAllocMapped));
    *(volatile int*)c->gate_host = 0;
    c->gate_gen = 0;
    CU(cudaHostGetDevicePointer((void**)&c->gate_dev, c->gate_host, 0));
  }
  // host loop: launch rounds in chunks, read the done flag between chunks
  for (long long it = 0; it < max_rounds + 1;) {
    const long long chunk = plain ? 64 : 8;
    if (c->profile) {
      k_gate<<<1, 1, 0, c->stream>>>(c->gate_dev, ++c->gate_gen,
                                     (int*)((char*)c->b.st + offsetof(DevState, status)));
      CU(cudaGetLastError());
    }
    for (long long j = 0; j < chunk; ++j, ++it) {
      cudaError_t e = launch_body(c, plain, T, 0ull, 0, c->stream,
                                  c->profile ? &c->prof : nullptr, it);
      if (e != cudaSuccess) {
        if (c->profile) __atomic_store_n(c->gate_host, c->gate_gen, __ATOMIC_RELEASE);
        return cuda_fail(e, "round launch");
      }
      c->host_iters = it + 1;
    }
    if (c->profile) __atomic_store_n(c->gate_host, c->gate_gen, __ATOMIC_RELEASE);
    CU(cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (c->st_host->done) break;
  }
  return RPCHOL_OK;
}

rpchol_status read_state(rpchol_ctx* c) {
  CU(cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return RPCHOL_OK;
}

rpchol_status status_of(const DevState& s) {
  if (s.status & kStTimeout) {
    set_err("a bounded device-side wait expired (tensor-core column step)");
    return RPCHOL_ETIMEOUT;
  }
  if (s.status & kStNumeric) {
    set_err("non-positive pivot or non-finite value met on the device");
    return RPCHOL_ENUMERIC;
  }
  if (s.status & kStGateExpired) {
    set_err("profile mode: the stream gate gave up waiting for the host, so the phase "
            "times include host enqueue time");
    return RPCHOL_ETIMEOUT;
  }
  if (s.status & kStRoundLimit) {
    set_err("round limit reached before the target rank");
    return RPCHOL_ETIMEOUT;
  }
  return RPCHOL_OK;
}

// Rounds launched ahead of the one whose end the host waits for; the
// snapshot ring holds one slot per round in flight.
constexpr int kStreamAhead = 3;
// Finished columns are copied as soon as the copy stream is idle, or once
// they make rows of at least this many bytes: the copy engine moves N rows
// of 800 bytes (one round of 200 FP32 columns) at about 120 GB/s into
// pinned host memory and rows of 3200 bytes at about 190 GB/s, the link's
// rate.  Copying whenever the engine is idle keeps it busy through the run
// (the rows grow by themselves while a copy is in flight) and leaves about
// one copy's worth of columns after the last round.
constexpr long long kFlushRowBytes = 3200;

// Host callback after each 2-D copy: counts the copies that have landed.
void CUDART_CB copy_landed(void* p) {
  ((std::atomic<long long>*)p)->fetch_add(1, std::memory_order_release);
}

// Copy of the device state into mapped pinned host memory, written by a
// kernel so that no copy engine (busy with the factor's columns) sits on
// the round stream.
__global__ void k_snapshot(const DevState* st, DevState* out) {
  const int n = (int)(sizeof(DevState) / sizeof(int));
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    ((volatile int*)out)[i] = ((const volatile int*)st)[i];
}

// The round loop of rpchol_run_to_host (device state reset): after each
// round the host reads that round's state snapshot and has the copy stream
// move the columns the round added, while later rounds run.
rpchol_status run_streaming(rpchol_ctx* c, int T, long long max_rounds, char* F_out,
                            long long ld_out, int64_t* pivots_out) {
  static_assert(kStreamAhead + 1 <= 4, "snapshot events");
  static_assert(sizeof(DevState) % sizeof(int) == 0, "state copied as ints");
  if (!c->copy_stream) {
    CU(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    CU(cudaHostAlloc((void**)&c->snap_host, sizeof(DevState) * (kStreamAhead + 1),
                     cudaHostAllocMapped));
    for (cudaEvent_t& e : c->snap_ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming));
  }
  DevState* snap_dev = nullptr;
  CU(cudaHostGetDevicePointer((void**)&snap_dev, c->snap_host, 0));
  const size_t es = c->b.mixed ? sizeof(float) : sizeof(double);
  long long launched = 0, waited = 0, copied = 0;
  long long issued = c->copies_landed.load(std::memory_order_acquire);
  for (;;) {
    while (launched < max_rounds + 1 && launched - waited <= kStreamAhead) {
      const int slot = (int)(launched % (kStreamAhead + 1));
      cudaError_t e = launch_body(c, 0, T, 0ull, 0, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "round launch");
      k_snapshot<<<1, 64, 0, c->stream>>>(c->b.st, snap_dev + slot);
      CU(cudaGetLastError());
      CU(cudaEventRecord(c->snap_ev[slot], c->stream));
      ++launched;
      c->host_iters = launched;
    }
    if (waited == launched) break;
    const int slot = (int)(waited % (kStreamAhead + 1));
    CU(cudaEventSynchronize(c->snap_ev[slot]));
    ++waited;
    const volatile DevState& sn = c->snap_host[slot];
    const long long rank = sn.rank;
    const bool last = sn.done || sn.status || waited == launched;
    const bool idle = c->copies_landed.load(std::memory_order_acquire) == issued;
    const bool flush = last || idle || (rank - copied) * (long long)es >= kFlushRowBytes;
    if (rank > copied && flush) {
      // columns [copied, rank) are final: the copy engine moves them while
      // the rounds already launched run
      CU(cudaStreamWaitEvent(c->copy_stream, c->snap_ev[slot], 0));
      CU(cudaMemcpy2DAsync(F_out + es * copied, es * ld_out, (const char*)c->b.F + es * copied,
                           es * c->b.ldF, es * (rank - copied), c->b.N, cudaMemcpyDefault,
                           c->copy_stream));
      CU(cudaLaunchHostFunc(c->copy_stream, copy_landed, &c->copies_landed));
      ++issued;
      copied = rank;
    }
    if (sn.done || sn.status) break;  // rounds still in flight find the run done
  }
  CU(cudaEventRecord(c->copy_ev, c->stream));  // every launched round
  CU(cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0));
  if (pivots_out && copied > 0)
    CU(cudaMemcpyAsync(pivots_out, c->b.piv, sizeof(long long) * copied, cudaMemcpyDefault,
                       c->copy_stream));
  CU(cudaStreamSynchronize(c->copy_stream));
  rpchol_status st = read_state(c);
  if (st != RPCHOL_OK) return st;
  if (c->st_host->rank != copied) {
    set_err("rpchol_run_to_host: rank %lld at the end, %lld columns copied",
            (long long)c->st_host->rank, copied);
    return RPCHOL_ECUDA;
  }
  return status_of(*c->st_host);
}

}  // namespace

extern "C" {

const char* rpchol_version(void) { return "rpchol-gb300 0.1 (sm_103a)"; }

const char* rpchol_last_error(void) { return g_err; }

rpchol_status rpchol_create(int32_t kind, double sigma, const void* X, int64_t N, int32_t d,
                            int32_t x_dtype, int32_t x_on_device, int64_t k_max, int32_t T_max,
                            const rpchol_opts* opts, rpchol_ctx** out) {
  g_err[0] = 0;
  if (!out) {
    set_err("out is NULL");
    return RPCHOL_EINVAL;
  }
  *out = nullptr;
  if (!X || N < 1 || d < 1 || d > 4096 || !(sigma > 0.0) || kind < 0 || kind > 4 || k_max < 1 ||
      k_max > N || T_max < 1 || T_max > kTMax || (x_dtype != RPCHOL_DT_F32 && x_dtype != RPCHOL_DT_F64) ||
      N > (1ll << 31) - 1) {
    set_err("invalid argument: N=%lld d=%d sigma=%g kind=%d k_max=%lld T_max=%d x_dtype=%d",
            (long long)N, d, sigma, kind, (long long)k_max, T_max, x_dtype);
    return RPCHOL_EINVAL;
  }
  int prec = opts ? opts->precision : RPCHOL_FP64;
  if (prec != RPCHOL_FP64 && prec != RPCHOL_MIXED) {
    set_err("invalid precision %d", prec);
    return RPCHOL_EINVAL;
  }
  rpchol_ctx* c = new (std::nothrow) rpchol_ctx();
  if (!c) {
    set_err("host allocation failed");
    return RPCHOL_ENOMEM;
  }
  c->precision = prec;
  c->use_graph = opts ? (opts->use_graph != 0) : 1;
  c->profile = opts ? (opts->profile != 0) : 0;
  c->instance = opts ? opts->instance : 0u;
  c->stream = opts ? (cudaStream_t)opts->stream : nullptr;
  c->alloc = opts ? opts->dev_alloc : nullptr;
  c->release = opts ? opts->dev_free : nullptr;
  c->alloc_user = opts ? opts->alloc_user : nullptr;
  if ((c->alloc == nullptr) != (c->release == nullptr)) {
    delete c;
    set_err("dev_alloc and dev_free must be given together");
    return RPCHOL_EINVAL;
  }
  c->k_max = k_max;
  DevBuffers& b = c->b;
  b.N = N;
  b.d = d;
  b.xld = (int)round_up(d, kLdAlign);
  b.kind = kind;
  b.sigma = sigma;
  b.ntiles = (N + kTileRows - 1) / kTileRows;
  b.ldF = round_up(k_max, kLdAlign);
  b.Tmax = T_max;
  b.mixed = prec == RPCHOL_MIXED;
  b.ldB = b.ldF + kTMax;
  b.ldBs = 0;
  b.nred = 2 + 2048 + 2;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm < 1)
      nsm = 148;
    b.num_sms = nsm;
  }

  rpchol_status rs = RPCHOL_OK;
  auto fail = [&](rpchol_status s) {
    release_all(c);
    delete c;
    return s;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate"));
  e = cudaMallocHost((void**)&c->st_host, sizeof(DevState));
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMallocHost"));
  memset(c->st_host, 0, sizeof(DevState));

  const size_t fbytes = (size_t)N * (size_t)b.ldF * (b.mixed ? sizeof(float) : sizeof(double));
  void* p;
#define ALLOC(field, type, count)                                      \
  do {                                                                 \
    if ((rs = dev_alloc(c, &p, sizeof(type) * (size_t)(count))) != RPCHOL_OK) return fail(rs); \
    b.field = (type*)p;                                                \
  } while (0)
  {
    float* Xp;
    if ((rs = dev_alloc(c, &p, sizeof(float) * (size_t)N * b.xld)) != RPCHOL_OK) return fail(rs);
    Xp = (float*)p;
    b.X = Xp;
    float* np;
    if ((rs = dev_alloc(c, &p, sizeof(float) * (size_t)N)) != RPCHOL_OK) return fail(rs);
    np = (float*)p;
    b.nrm = np;
  }
  ALLOC(dvec, double, N);
  ALLOC(tile_sums, double, b.ntiles);
  // one prefix copy per sampler CTA when the prefix does not fit in shared memory
  ALLOC(tile_prefix, double,
        b.ntiles * sizeof(double) <= 160 * 1024 ? b.ntiles : b.ntiles * (kTMax / 8));
  if ((rs = dev_alloc(c, &p, fbytes)) != RPCHOL_OK) return fail(rs);
  b.F = p;
  ALLOC(piv, long long, k_max);
  ALLOC(prop, int, kTMax);
  ALLOC(uprop, double, kTMax);
  ALLOC(uacc, double, kTMax);
  ALLOC(H, double, (size_t)kTMax * kTMax);
  ALLOC(Lw, double, (size_t)kTMax * kTMax);
  ALLOC(L, double, (size_t)kTMax * T_max);
  ALLOC(Linv, double, (size_t)kTMax * T_max);
  ALLOC(Sacc, int, kTMax);
  ALLOC(Hpart, double, (size_t)kHPartDoubles);
  ALLOC(hcnt, int, kHTilesMax);
  ALLOC(ccnt, unsigned, 1);
  ALLOC(red, double, b.nred);
  ALLOC(st, DevState, 1);
  ALLOC(Bext, double, (size_t)T_max * b.ldB);  // float rows in mixed mode
#undef ALLOC

  e = cudaMemsetAsync(b.F, 0, fbytes, c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(F)"));
  e = cudaMemsetAsync((void*)b.X, 0, sizeof(float) * (size_t)N * b.xld, c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(X)"));
  e = cudaMemsetAsync(b.ccnt, 0, sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(ccnt)"));
  e = cudaMemsetAsync(b.hcnt, 0, sizeof(int) * kHTilesMax, c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(hcnt)"));
  e = cudaMemsetAsync(b.st, 0, sizeof(DevState), c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(state)"));
  e = cudaMemsetAsync(b.piv, 0xff, sizeof(long long) * (size_t)k_max, c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(piv)"));
  if (x_dtype == RPCHOL_DT_F32) {
    e = cudaMemcpy2DAsync((void*)b.X, sizeof(float) * b.xld, X, sizeof(float) * d,
                          sizeof(float) * d, N, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "copy of X"));
  } else {
    void* tmp = nullptr;
    e = cudaMallocAsync(&tmp, sizeof(double) * (size_t)N * d, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMallocAsync(X staging)"));
    e = cudaMemcpyAsync(tmp, X, sizeof(double) * (size_t)N * d, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
      e = launch_convert_x64((const double*)tmp, N, d, (float*)b.X, b.xld, c->stream);
    cudaFreeAsync(tmp, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "conversion of X"));
  }
  e = launch_norms(b, c->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "norms"));
  if (b.mixed) {
    // tensor-core column step: needs at least one full 128-row tile; the
    // CUDA-core FP32 path serves smaller problems (and RPCHOL_COLSTEP=simt)
    const char* env = getenv("RPCHOL_COLSTEP");
    // the l1-Laplace has no inner-product form, so its distances cannot come
    // from the tensor-core contraction: the CUDA-core column step forms them
    c->use_tc = (N >= 128) && kind != RPCHOL_LAPLACE_L1 && !(env && strcmp(env, "simt") == 0);
  }
  if (c->use_tc) {
    TcMaps& m = c->tc;
    const size_t xbytes = sizeof(float) * (size_t)N * b.xld;
    // one 128 x kTMax-byte image per K chunk: ldF / 32 chunks of F(S,:), xld / 16 of X_S
    const size_t bfbytes = (size_t)(b.ldF / 32) * 128 * kTMax;
    const size_t bxbytes = (size_t)(b.xld / 16) * 128 * kTMax;
    // FP16 heads / tails of 4096 F, the Schur contraction's A operand
    const size_t fsbytes = 2 * sizeof(uint16_t) * (size_t)N * b.ldF;
    void* q;
    if ((rs = dev_alloc(c, &q, fsbytes)) != RPCHOL_OK) return fail(rs);
    m.Fsp = q;
    if ((rs = dev_alloc(c, &q, xbytes)) != RPCHOL_OK) return fail(rs);
    m.Xhp = (float*)q;
    if ((rs = dev_alloc(c, &q, xbytes)) != RPCHOL_OK) return fail(rs);
    m.Xlp = (float*)q;
    if ((rs = dev_alloc(c, &q, bfbytes)) != RPCHOL_OK) return fail(rs);
    m.Bf = (unsigned char*)q;
    if ((rs = dev_alloc(c, &q, bxbytes)) != RPCHOL_OK) return fail(rs);
    m.Bx = (unsigned char*)q;
    if ((rs = dev_alloc(c, &q, sizeof(float) * kTMax)) != RPCHOL_OK) return fail(rs);
    m.nrmS = (float*)q;
    if ((rs = dev_alloc(c, &q, sizeof(float) * kTMax * kTMax)) != RPCHOL_OK) return fail(rs);
    m.Linv32 = (float*)q;
    m.err = (int*)((char*)b.st + offsetof(DevState, status));
    m.num_sms = b.num_sms;
    // zero planes: the columns of a chunk beyond the rank meet zero B columns
    e = cudaMemsetAsync(m.Fsp, 0, fsbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.Bf, 0, bfbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.Bx, 0, bxbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.Linv32, 0, sizeof(float) * kTMax * kTMax, c->stream);
    if (e == cudaSuccess) e = launch_split_x(m, b, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "tensor-core operand setup"));
    if ((rs = make_map(&m.Fs, m.Fsp, 2ull * b.ldF, N, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B,
                       true)) != RPCHOL_OK)
      return fail(rs);
    if ((rs = make_map(&m.Xh, m.Xhp, b.xld, N, 16, 128, CU_TENSOR_MAP_SWIZZLE_64B)) != RPCHOL_OK)
      return fail(rs);
    if ((rs = make_map(&m.Xl, m.Xlp, b.xld, N, 16, 128, CU_TENSOR_MAP_SWIZZLE_64B)) != RPCHOL_OK)
      return fail(rs);
  }
  e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_fail(e, "create"));
  (void)x_on_device;
  *out = c;
  return RPCHOL_OK;
}

rpchol_status rpchol_run(rpchol_ctx* c, int64_t k, int32_t T, uint64_t seed) {
  g_err[0] = 0;
  if (!c || k < 1 || k > c->k_max || T < 1 || T > c->b.Tmax) {
    set_err("invalid argument: k=%lld T=%d", (long long)k, T);
    return RPCHOL_EINVAL;
  }
  return run_common(c, 0, k, T, seed);
}

rpchol_status rpchol_run_to_host(rpchol_ctx* c, int64_t k, int32_t T, uint64_t seed,
                                 void* F_out, int64_t ld_out, int64_t* pivots_out) {
  g_err[0] = 0;
  if (!c || k < 1 || k > c->k_max || T < 1 || T > c->b.Tmax || !F_out || ld_out < k) {
    set_err("invalid argument: k=%lld T=%d F_out=%p ld_out=%lld", (long long)k, T, F_out,
            (long long)ld_out);
    return RPCHOL_EINVAL;
  }
  const long long max_rounds = 4 * k + 64;
  clear_prof(c);
  CU(launch_reset(c->b, k, T, seed, c->instance, 0, max_rounds, c->stream));
  c->last_plain = 0;
  c->has_run = 1;
  return run_streaming(c, T, max_rounds, (char*)F_out, ld_out, pivots_out);
}

rpchol_status rpchol_run_block(rpchol_ctx* c, int64_t k, int32_t b, uint64_t seed) {
  g_err[0] = 0;
  if (!c || k < 1 || k > c->k_max || b < 1 || b > c->b.Tmax) {
    set_err("invalid argument: k=%lld b=%d", (long long)k, b);
    return RPCHOL_EINVAL;
  }
  return run_common(c, 2, k, b, seed);
}

rpchol_status rpchol_run_plain(rpchol_ctx* c, int64_t k, uint64_t seed) {
  g_err[0] = 0;
  if (!c || k < 1 || k > c->k_max) {
    set_err("invalid argument: k=%lld", (long long)k);
    return RPCHOL_EINVAL;
  }
  return run_common(c, 1, k, 1, seed);
}

rpchol_status rpchol_sync(rpchol_ctx* c) {
  if (!c) return RPCHOL_EINVAL;
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  return status_of(*c->st_host);
}

rpchol_status rpchol_factor(rpchol_ctx* c, const void** F_dev, int64_t* ldF, int32_t* F_dtype,
                            int64_t* rank, const int64_t** pivots_dev) {
  if (!c) return RPCHOL_EINVAL;
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  if (F_dev) *F_dev = c->b.F;
  if (ldF) *ldF = c->b.ldF;
  if (F_dtype) *F_dtype = c->b.mixed ? RPCHOL_DT_F32 : RPCHOL_DT_F64;
  if (rank) *rank = c->has_run ? c->st_host->rank : 0;
  if (pivots_dev) *pivots_dev = (const int64_t*)c->b.piv;
  return RPCHOL_OK;
}

rpchol_status rpchol_copy_factor(rpchol_ctx* c, double* F_out, int64_t ld_out,
                                 int64_t* pivots_out, double* d_out) {
  if (!c) return RPCHOL_EINVAL;
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  const long long rank = c->has_run ? c->st_host->rank : 0;
  if (F_out && ld_out < rank) {
    set_err("ld_out %lld < rank %lld", (long long)ld_out, rank);
    return RPCHOL_EINVAL;
  }
  if (F_out && rank > 0) {
    if (!c->b.mixed) {
      CU(cudaMemcpy2DAsync(F_out, sizeof(double) * ld_out, c->b.F, sizeof(double) * c->b.ldF,
                           sizeof(double) * rank, c->b.N, cudaMemcpyDefault, c->stream));
    } else {
      // widen FP32 -> FP64 on the device, then copy
      void* tmp = nullptr;
      CU(cudaMallocAsync(&tmp, sizeof(double) * (size_t)c->b.N * rank, c->stream));
      cudaError_t e = launch_widen_f32((const float*)c->b.F, c->b.ldF, c->b.N, rank,
                                       (double*)tmp, c->stream);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(F_out, sizeof(double) * ld_out, tmp, sizeof(double) * rank,
                              sizeof(double) * rank, c->b.N, cudaMemcpyDefault, c->stream);
      cudaFreeAsync(tmp, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "copy of F");
    }
  }
  if (pivots_out && rank > 0)
    CU(cudaMemcpyAsync(pivots_out, c->b.piv, sizeof(long long) * rank, cudaMemcpyDefault,
                       c->stream));
  if (d_out)
    CU(cudaMemcpyAsync(d_out, c->b.dvec, sizeof(double) * c->b.N, cudaMemcpyDefault, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return status_of(*c->st_host);
}

rpchol_status rpchol_copy_factor_raw(rpchol_ctx* c, void* F_out, int64_t ld_out,
                                     int64_t* pivots_out) {
  if (!c) return RPCHOL_EINVAL;
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  const long long rank = c->has_run ? c->st_host->rank : 0;
  if (F_out && ld_out < rank) {
    set_err("ld_out %lld < rank %lld", (long long)ld_out, rank);
    return RPCHOL_EINVAL;
  }
  const size_t es = c->b.mixed ? sizeof(float) : sizeof(double);
  if (F_out && rank > 0)
    CU(cudaMemcpy2DAsync(F_out, es * ld_out, c->b.F, es * c->b.ldF, es * rank, c->b.N,
                         cudaMemcpyDefault, c->stream));
  if (pivots_out && rank > 0)
    CU(cudaMemcpyAsync(pivots_out, c->b.piv, sizeof(long long) * rank, cudaMemcpyDefault,
                       c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return status_of(*c->st_host);
}

rpchol_status rpchol_stats(rpchol_ctx* c, rpchol_run_stats* out) {
  if (!c || !out) return RPCHOL_EINVAL;
  memset(out, 0, sizeof(*out));
  CU(launch_trace(c->b, c->stream));
  double host[2];
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  CU(cudaMemcpy(&host[0], c->b.red, sizeof(double), cudaMemcpyDeviceToHost));
  int parts = (int)((c->b.N + 7) / 8);
  if (parts > (int)c->b.nred - 2) parts = (int)c->b.nred - 2;
  if (parts > 2048) parts = 2048;
  if (parts < 1) parts = 1;
  CU(cudaMemcpy(&host[1], c->b.red + parts + 1, sizeof(double), cudaMemcpyDeviceToHost));
  const DevState& st = *c->st_host;
  out->rank = c->has_run ? st.rank : 0;
  out->rounds = st.round;
  out->proposals = st.proposals;
  out->accepted = st.rank;
  out->status = (int32_t)status_of(st);
  out->plain = st.plain ? 1 : (st.block ? 2 : 0);
  out->residual_trace = host[1];
  out->trace_error = host[0] / (double)c->b.N;  // tr A = N (phi(0) = 1)
  out->col_bytes = st.col_bytes;
  out->col_flops = st.col_flops;
  out->mma_flops_tf32 = st.mma_tf32;
  out->mma_flops_f16 = st.mma_f16;
  {
    // kernels of one loop body: accelerated = propose, H, Algorithm 1, operand
    // prep (prep and W blocks in one launch for the tensor-core step, the
    // gather otherwise), column step, round end (closed by the tensor-core
    // column step itself);
    // simple = propose (with g_s), GEMV and new column, tile sums and step end.
    // The graph runs the body once
    // per round; the host loop launches whole chunks of bodies.
    const long long per = c->last_plain ? 3 : (c->use_tc ? 5 : 6);
    const long long iters = c->host_iters >= 0 ? c->host_iters : st.round;
    out->kernel_launches = c->has_run ? 1 + per * iters : 0;
  }
  // profile mode: only iterations that did work (those before the final
  // round count; later ones exit at their first instruction) are counted
  for (const auto& r : c->prof) {
    if (r.iter >= st.round) continue;
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, r.a, r.b));
    out->phase_ms[r.slot] += ms;
    out->phase_launches[r.slot] += 1;
  }
  return RPCHOL_OK;
}

// ---------------------------------------------------------------- checkpoints
// Layout of a checkpoint (host memory, native byte order): SaveHeader, the
// device state, d (N doubles), the tile sums, the pivots (rank int64) and F
// (N rows x rank columns in the stored dtype, packed).
struct SaveHeader {
  char magic[8];
  int32_t version, precision, kind, d;
  int64_t N, k_max, rank, bytes;
  double sigma;
  int64_t ntiles, elem;
};

static size_t save_bytes(const rpchol_ctx* c, long long rank) {
  const size_t es = c->b.mixed ? sizeof(float) : sizeof(double);
  return sizeof(SaveHeader) + sizeof(DevState) + sizeof(double) * (size_t)c->b.N +
         sizeof(double) * (size_t)c->b.ntiles + sizeof(long long) * (size_t)rank +
         es * (size_t)c->b.N * (size_t)rank;
}

rpchol_status rpchol_save(rpchol_ctx* c, void* host_buf, size_t* bytes) {
  g_err[0] = 0;
  if (!c || !bytes) return RPCHOL_EINVAL;
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  if (!c->has_run) {
    set_err("nothing to save: the context has not run");
    return RPCHOL_EINVAL;
  }
  const DevState st = *c->st_host;
  const long long rank = st.rank;
  const size_t need = save_bytes(c, rank);
  if (!host_buf) {
    *bytes = need;
    return RPCHOL_OK;
  }
  if (*bytes < need) {
    set_err("buffer of %zu bytes, %zu needed", *bytes, need);
    *bytes = need;
    return RPCHOL_EINVAL;
  }
  char* p = (char*)host_buf;
  SaveHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "RPCHOLS1", 8);
  h.version = 1;
  h.precision = c->precision;
  h.kind = c->b.kind;
  h.d = c->b.d;
  h.N = c->b.N;
  h.k_max = c->k_max;
  h.rank = rank;
  h.bytes = (int64_t)need;
  h.sigma = c->b.sigma;
  h.ntiles = c->b.ntiles;
  h.elem = c->b.mixed ? 4 : 8;
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  memcpy(p, &st, sizeof(DevState));
  p += sizeof(DevState);
  const size_t es = (size_t)h.elem;
  CU(cudaMemcpyAsync(p, c->b.dvec, sizeof(double) * c->b.N, cudaMemcpyDeviceToHost, c->stream));
  p += sizeof(double) * c->b.N;
  CU(cudaMemcpyAsync(p, c->b.tile_sums, sizeof(double) * c->b.ntiles, cudaMemcpyDeviceToHost,
                     c->stream));
  p += sizeof(double) * c->b.ntiles;
  if (rank > 0) {
    CU(cudaMemcpyAsync(p, c->b.piv, sizeof(long long) * rank, cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(long long) * rank;
    CU(cudaMemcpy2DAsync(p, es * rank, c->b.F, es * c->b.ldF, es * rank, c->b.N,
                         cudaMemcpyDeviceToHost, c->stream));
  }
  CU(cudaStreamSynchronize(c->stream));
  *bytes = need;
  return RPCHOL_OK;
}

rpchol_status rpchol_restore(rpchol_ctx* c, const void* host_buf, size_t bytes) {
  g_err[0] = 0;
  if (!c || !host_buf || bytes < sizeof(SaveHeader) + sizeof(DevState)) return RPCHOL_EINVAL;
  const char* p = (const char*)host_buf;
  SaveHeader h;
  memcpy(&h, p, sizeof(h));
  if (memcmp(h.magic, "RPCHOLS1", 8) != 0 || h.version != 1) {
    set_err("not a checkpoint of this library");
    return RPCHOL_EINVAL;
  }
  if (h.N != c->b.N || h.d != c->b.d || h.kind != c->b.kind || h.sigma != c->b.sigma ||
      h.precision != c->precision || h.ntiles != c->b.ntiles || h.rank > c->k_max ||
      h.rank < 0 || (size_t)h.bytes != bytes || save_bytes(c, h.rank) != bytes) {
    set_err("checkpoint does not match this context (N, d, kernel, sigma, precision, k_max)");
    return RPCHOL_EINVAL;
  }
  p += sizeof(h);
  DevState st;
  memcpy(&st, p, sizeof(DevState));
  p += sizeof(DevState);
  if (st.rank != h.rank || st.T < 1 || st.T > c->b.Tmax) {
    set_err("checkpoint state does not fit this context (T_max)");
    return RPCHOL_EINVAL;
  }
  const size_t es = (size_t)h.elem;
  const long long rank = h.rank;
  CU(cudaMemcpyAsync(c->b.st, &st, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->b.dvec, p, sizeof(double) * c->b.N, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(double) * c->b.N;
  CU(cudaMemcpyAsync(c->b.tile_sums, p, sizeof(double) * c->b.ntiles, cudaMemcpyHostToDevice,
                     c->stream));
  p += sizeof(double) * c->b.ntiles;
  if (rank > 0) {
    CU(cudaMemcpyAsync(c->b.piv, p, sizeof(long long) * rank, cudaMemcpyHostToDevice, c->stream));
    p += sizeof(long long) * rank;
    CU(cudaMemcpy2DAsync(c->b.F, es * c->b.ldF, p, es * rank, es * rank, c->b.N,
                         cudaMemcpyHostToDevice, c->stream));
    if (c->use_tc) CU(launch_f16_planes(c->tc, c->b, rank, c->stream));
  }
  CU(cudaStreamSynchronize(c->stream));
  *c->st_host = st;
  c->has_run = 1;
  c->last_plain = st.plain;
  clear_prof(c);
  c->host_iters = -1;
  return RPCHOL_OK;
}

rpchol_status rpchol_resume(rpchol_ctx* c, int64_t k) {
  g_err[0] = 0;
  if (!c) return RPCHOL_EINVAL;
  rpchol_status s = read_state(c);
  if (s != RPCHOL_OK) return s;
  DevState st = *c->st_host;
  if (!c->has_run || k <= st.rank || k > c->k_max || st.status != 0) {
    set_err("invalid resume: k=%lld rank=%lld k_max=%lld status=%d", (long long)k, st.rank,
            c->k_max, st.status);
    return RPCHOL_EINVAL;
  }
  st.k = k;
  st.done = 0;
  st.max_rounds = st.round + (st.plain ? 2 * (k - st.rank) : 4 * (k - st.rank)) + 64;
  CU(cudaMemcpyAsync(c->b.st, &st, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  clear_prof(c);
  return run_loop(c, st.plain, st.T, st.max_rounds - st.round);
}

rpchol_status rpchol_selftest_wait(uint32_t limit_ms, double* waited_ms) {
  g_err[0] = 0;
  if (limit_ms < 1 || limit_ms > 2000) {
    set_err("limit_ms must be in [1, 2000]");
    return RPCHOL_EINVAL;
  }
  unsigned long long* dout = nullptr;
  unsigned long long h[4] = {0, 0, 0, 0};
  CU(cudaMalloc((void**)&dout, sizeof(h)));
  const unsigned long long lim = 1000000ull * limit_ms;
  cudaError_t e = launch_wait_selftest_cta(lim, dout, nullptr);
  if (e == cudaSuccess) e = launch_wait_selftest_cluster(lim, dout + 2, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h, dout, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(dout);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (waited_ms) {
    waited_ms[0] = (double)h[1] * 1e-6;
    waited_ms[1] = (double)h[3] * 1e-6;
  }
  if (h[0] == 1 && h[2] == 1) {
    set_err("both bounded waits gave up after %.1f and %.1f ms, as designed", h[1] * 1e-6,
            h[3] * 1e-6);
    return RPCHOL_ETIMEOUT;
  }
  set_err("a bounded wait did not report its expiry");
  return RPCHOL_ECUDA;
}

void rpchol_destroy(rpchol_ctx* c) {
  if (!c) return;
  release_all(c);
  delete c;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
struct rpchol_batch {
  std::vector<rpchol_ctx*> ctxs;
  std::vector<int> T;
  std::vector<cudaEvent_t> ready;  // per context: its stream's work so far
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  RunParams* dparams = nullptr;    // device, one per instance
  RunParams* hparams = nullptr;    // pinned staging
  cudaEvent_t copied = nullptr;    // staging copy of the last run done
  cudaEvent_t done = nullptr;      // last batch run done
  cudaStream_t cap = nullptr;      // private stream used only to record
  bool ran = false;
  // persistent engine (mode RPCHOL_BATCH_ENGINE)
  int mode = RPCHOL_BATCH_GRAPH;
  bool engine_ok = false;          // every member supports the engine
  void* insts = nullptr;           // device: instance descriptors
  void* maps = nullptr;            // device: tensor maps
  int* dorder = nullptr;           // device: queue order
  void* dqueue = nullptr;          // device: scheduler state (zeroed every run)
  int* horder = nullptr;           // pinned staging of the order
  int ctas = 0;                    // engine grid (whole clusters, all resident)
};

namespace {

void batch_release(rpchol_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ready) cudaEventDestroy(e);
  if (b->copied) cudaEventSynchronize(b->copied), cudaEventDestroy(b->copied);
  if (b->done) cudaEventSynchronize(b->done), cudaEventDestroy(b->done);
  if (b->dparams) cudaFree(b->dparams);
  if (b->hparams) cudaFreeHost(b->hparams);
  if (b->insts) cudaFree(b->insts);
  if (b->maps) cudaFree(b->maps);
  if (b->dorder) cudaFree(b->dorder);
  if (b->dqueue) cudaFree(b->dqueue);
  if (b->horder) cudaFreeHost(b->horder);
  if (b->cap) cudaStreamDestroy(b->cap);
}

// Descriptors, queue and grid of the persistent engine.
rpchol_status engine_prepare(rpchol_batch* b) {
  const int n = (int)b->ctxs.size();
  std::vector<DevBuffers> bs(n);
  std::vector<TcMaps> ms(n);
  for (int i = 0; i < n; ++i) {
    bs[i] = b->ctxs[i]->b;
    ms[i] = b->ctxs[i]->tc;
  }
  CU(engine_grid(&b->ctas));
  CU(cudaMalloc((void**)&b->dorder, sizeof(int) * (size_t)n));
  CU(cudaMalloc(&b->dqueue, engine_queue_bytes(n)));
  CU(cudaMallocHost((void**)&b->horder, sizeof(int) * (size_t)n));
  CU(engine_setup(n, bs.data(), ms.data(), &b->insts, &b->maps, b->cap));
  return RPCHOL_OK;
}

rpchol_status batch_record(rpchol_batch* b) {
  if (b->exec) return RPCHOL_OK;
  const int n = (int)b->ctxs.size();
  CU(cudaGraphCreate(&b->graph, 0));
  for (int i = 0; i < n; ++i) {
    rpchol_ctx* c = b->ctxs[i];
    cudaGraphNode_t reset;
    CU(add_reset_params_node(b->graph, c->b, b->dparams + i, &reset));
    cudaGraphConditionalHandle h;
    CU(cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CU(cudaGraphAddNode(&node, b->graph, &reset, nullptr, 1, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    CU(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    cudaError_t le = launch_body(c, 0, b->T[i], (unsigned long long)h, 1, b->cap);
    cudaGraph_t captured = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->cap, &captured);
    if (le != cudaSuccess) return cuda_fail(le, "capture of a batch branch");
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
  }
  CU(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return RPCHOL_OK;
}

}  // namespace

extern "C" {

int64_t rpchol_context_bytes(int64_t N, int32_t d, int64_t k_max, int32_t T_max,
                             int32_t precision) {
  if (N < 1 || d < 1 || k_max < 1 || T_max < 1) return 0;
  const bool mixed = precision == RPCHOL_MIXED;
  const long long xld = round_up(d, kLdAlign), ldF = round_up(k_max, kLdAlign);
  const long long ntiles = (N + kTileRows - 1) / kTileRows;
  const long long bf = mixed ? 4 : 8;
  long long b = 0;
  b += 4 * N * xld + 4 * N;                           // X, norms
  b += 8 * N + 8 * ntiles;                            // d, tile sums
  b += 8 * (ntiles * 8 <= 160 * 1024 ? ntiles : ntiles * (kTMax / 8));  // tile prefix
  b += bf * N * ldF;                                  // F
  b += 8 * k_max + 4 * kTMax + 16 * kTMax + 4 * kTMax;  // pivots, proposals, uniforms
  b += 8 * 2LL * kTMax * kTMax + 8 * 2LL * kTMax * T_max;  // H, Lw, L, Linv
  b += 8LL * kHPartDoubles + 4 * kHTilesMax + 4;  // H partials, counters
  b += 8 * (2 + 2048 + 2) + (long long)sizeof(DevState);
  b += 8LL * T_max * (ldF + kTMax);                   // extended operand rows
  if (mixed && N >= 128) {
    b += 2 * 4 * N * xld;                             // TF32 planes of X
    b += 2 * 2 * N * ldF;                             // FP16 heads / tails of 4096 F
    b += (ldF / 32) * 128LL * kTMax + (xld / 16) * 128LL * kTMax;  // chunk images of F(S,:), X_S
    b += 4LL * kTMax + 4LL * kTMax * kTMax;
  }
  return (int64_t)b;
}

rpchol_status rpchol_batch_create(rpchol_ctx* const* ctxs, int32_t n, const int32_t* T,
                                  rpchol_batch** out) {
  g_err[0] = 0;
  if (!out || !ctxs || !T || n < 1) {
    set_err("invalid argument: n=%d", n);
    return RPCHOL_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || T[i] < 1 || T[i] > ctxs[i]->b.Tmax) {
      set_err("invalid batch member %d (T=%d)", i, T[i]);
      return RPCHOL_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) {
        set_err("context %d appears twice in the batch", i);
        return RPCHOL_EINVAL;
      }
  }
  rpchol_batch* b = new (std::nothrow) rpchol_batch();
  if (!b) {
    set_err("host allocation failed");
    return RPCHOL_ENOMEM;
  }
  b->ctxs.assign(ctxs, ctxs + n);
  b->T.assign(T, T + n);
  auto fail = [&](rpchol_status s) {
    batch_release(b);
    delete b;
    return s;
  };
  cudaError_t e = cudaMalloc((void**)&b->dparams, sizeof(RunParams) * (size_t)n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->hparams, sizeof(RunParams) * (size_t)n);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ready.push_back(ev);
  }
  if (e != cudaSuccess) return fail(cuda_fail(e, "batch setup"));
  b->engine_ok = true;
  for (int i = 0; i < n; ++i) {
    const rpchol_ctx* c = ctxs[i];
    b->engine_ok = b->engine_ok && c->precision == RPCHOL_MIXED && c->use_tc &&
                   engine_supported(c->b, c->use_tc);
  }
  // the graph executor is the default: on the measured batches it is the
  // faster one (the engine is set up on first use, rpchol_batch_set_mode)
  rpchol_status rs = batch_record(b);
  b->mode = RPCHOL_BATCH_GRAPH;
  if (rs != RPCHOL_OK) return fail(rs);
  *out = b;
  return RPCHOL_OK;
}

rpchol_status rpchol_batch_set_mode(rpchol_batch* b, int32_t mode) {
  g_err[0] = 0;
  if (!b || (mode != RPCHOL_BATCH_GRAPH && mode != RPCHOL_BATCH_ENGINE)) {
    set_err("invalid argument: mode=%d", mode);
    return RPCHOL_EINVAL;
  }
  if (mode == RPCHOL_BATCH_ENGINE && !b->engine_ok) {
    set_err("the batch engine needs every member in mixed precision with the tensor-core "
            "column step (N >= 128) and T_max <= %d",
            kTMax);
    return RPCHOL_EINVAL;
  }
  if (mode == RPCHOL_BATCH_GRAPH) {
    rpchol_status rs = batch_record(b);
    if (rs != RPCHOL_OK) return rs;
  } else if (!b->insts) {
    rpchol_status rs = engine_prepare(b);
    if (rs != RPCHOL_OK) return rs;
  }
  b->mode = mode;
  return RPCHOL_OK;
}

int32_t rpchol_batch_mode(const rpchol_batch* b) { return b ? b->mode : -1; }

rpchol_status rpchol_batch_run(rpchol_batch* b, const int64_t* k, const uint64_t* seeds,
                               void* stream) {
  g_err[0] = 0;
  if (!b || !k || !seeds) {
    set_err("invalid argument");
    return RPCHOL_EINVAL;
  }
  const int n = (int)b->ctxs.size();
  for (int i = 0; i < n; ++i)
    if (k[i] < 1 || k[i] > b->ctxs[i]->k_max) {
      set_err("invalid k=%lld for batch member %d", (long long)k[i], i);
      return RPCHOL_EINVAL;
    }
  cudaStream_t s = (cudaStream_t)stream;
  if (b->ran) CU(cudaEventSynchronize(b->copied));  // staging buffer free again
  for (int i = 0; i < n; ++i) {
    RunParams& p = b->hparams[i];
    p.k = k[i];
    p.max_rounds = 4 * k[i] + 64;
    p.seed = seeds[i];
    p.T = b->T[i];
    p.plain = 0;
    p.instance = b->ctxs[i]->instance;
    p.pad = 0;
  }
  for (int i = 0; i < n; ++i) {
    rpchol_ctx* c = b->ctxs[i];
    CU(cudaEventRecord(b->ready[i], c->stream));
    CU(cudaStreamWaitEvent(s, b->ready[i], 0));
  }
  CU(cudaMemcpyAsync(b->dparams, b->hparams, sizeof(RunParams) * (size_t)n,
                     cudaMemcpyHostToDevice, s));
  if (b->mode == RPCHOL_BATCH_ENGINE) {
    // queue order: largest expected work (N k^2) first, ties in index order
    std::vector<double> w(n);
    for (int i = 0; i < n; ++i)
      w[i] = (double)b->ctxs[i]->b.N * (double)k[i] * (double)k[i];
    for (int i = 0; i < n; ++i) b->horder[i] = i;
    std::stable_sort(b->horder, b->horder + n, [&](int x, int y) { return w[x] > w[y]; });
    CU(cudaMemcpyAsync(b->dorder, b->horder, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice,
                       s));
    CU(cudaMemsetAsync(b->dqueue, 0, engine_queue_bytes(n), s));
    CU(cudaEventRecord(b->copied, s));
    CU(engine_launch(b->insts, b->maps, b->dparams, b->dorder, n, b->dqueue, b->ctas, s));
  } else {
    CU(cudaEventRecord(b->copied, s));
    CU(cudaGraphLaunch(b->exec, s));
  }
  CU(cudaEventRecord(b->done, s));
  for (int i = 0; i < n; ++i) {
    rpchol_ctx* c = b->ctxs[i];
    clear_prof(c);
    c->last_plain = 0;
    c->has_run = 1;
    c->host_iters = -1;
    CU(cudaStreamWaitEvent(c->stream, b->done, 0));
  }
  b->ran = true;
  return RPCHOL_OK;
}

void rpchol_batch_destroy(rpchol_batch* b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

}  // extern "C"
