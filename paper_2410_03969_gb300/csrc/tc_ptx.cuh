// Inline-PTX building blocks for the Blackwell (sm_103a) tensor-core path:
// mbarriers, TMA tile loads, TMEM allocation, tcgen05.mma (kind::tf32,
// cta_group::1, operands in shared memory), tcgen05.ld and tcgen05.st.
//
// Operand layout used throughout: K-major, 128-byte swizzle.  A tile of R
// rows x 32 fp32 (128 bytes per row) is stored as R rows of 128 bytes; each
// group of 8 rows forms a 1024-byte swizzle atom in which the 16-byte chunk
// j of row r sits at chunk position j ^ (r % 8).  TMA with
// CU_TENSOR_MAP_SWIZZLE_128B writes exactly this layout, and the matching
// shared-memory descriptor has stride-dimension offset 1024 bytes between
// 8-row groups.  Advancing K by 8 tf32 (32 bytes) inside the atom is done by
// advancing the descriptor's start address by 32 bytes.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpchol {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's generic-proxy accesses (all state spaces) with later
// async-proxy accesses (TMA, bulk copies) and the reverse.
__device__ __forceinline__ void fence_proxy_async_all() {
  asm volatile("fence.proxy.async;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of the phase with the given parity (no suspension).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, giving up after
// `limit_ns` of %globaltimer or when *abort is set.  Returns true when the
// phase completed.  The waiting lane spins on the non-blocking test (a
// suspending try_wait and a back-off sleep were measured 1% slower on the
// column step's operand ring); the clock is read only once the first test
// has failed, and after every 16 failed tests the lane checks the abort
// flag and the clock.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns,
                                                  volatile int* abort) {
  if (mbar_test_wait(bar, parity)) return true;
  const unsigned long long deadline = globaltimer_ns() + limit_ns;
  for (uint32_t n = 0;; ++n) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((n & 15) == 15) {
      if (*abort) return false;
      if (globaltimer_ns() > deadline) {
        *abort = 1;
        return false;
      }
    }
  }
}

// Warp-wide bounded wait: lane 0 polls, the result is broadcast.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity,
                                               unsigned long long limit_ns,
                                               volatile int* abort) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(bar, parity, limit_ns, abort) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

// One arrival per warp, by lane 0 after __syncwarp has ordered the warp's
// prior shared-memory writes.
__device__ __forceinline__ void mbar_arrive_warp(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Contiguous global -> shared copy of `bytes` (a multiple of 16, both
// addresses 16-byte aligned), completing on the mbarrier by its bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The same copy into the same shared-memory offset of every CTA of the
// cluster in `mask`; each destination's barrier at `bar`'s offset receives
// the transaction bytes.
__device__ __forceinline__ void bulk_load_mc(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Bring the box at (x, y) of a 2-D tensor map into L2 (no shared-memory
// destination, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   (unsigned long long)map),
               "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)map) : "memory");
}

// 16-byte asynchronous global -> shared copy (L2 only), with group commit
// and wait.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)),
               "l"((unsigned long long)gmem)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- TMEM
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- MMA
// Shared-memory matrix descriptor: start address >> 4 in bits [0,14),
// leading-dimension byte offset >> 4 in [16,30) (unused for swizzled
// K-major operands, set to 1), stride-dimension byte offset >> 4 in [32,46),
// descriptor version 1 in [46,48), layout 2 (128-byte swizzle) in [61,64).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// The same for any K-major swizzled layout: stride-dimension byte offset
// `sbo` between 8-row groups, layout code `lay` (2: 128-byte swizzle, 4:
// 64-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo, uint32_t lay) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)(lay & 7u) << 61;
  return d;
}

// Instruction descriptor of kind::f16 with FP16 A and B (format 0) and FP32
// accumulation (D format 1 in bits [4,6)), both operands K-major: N >> 3 in
// [17,23), M >> 4 in [24,29).
__host__ __device__ __forceinline__ uint32_t idesc_f16(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both
// operands K-major: D format F32 (1) in bits [4,6), A and B format TF32 (2)
// in [7,10) and [10,13), N >> 3 in [17,23), M >> 4 in [24,29).
__host__ __device__ __forceinline__ uint32_t idesc_tf32(uint32_t M, uint32_t N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The same, also keeping A in the tensor core's collector buffer for the
// next MMA (which must name the same A and use mma_tf32_reuse_a).
__device__ __forceinline__ void mma_tf32_keep_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// A from the collector buffer filled by the previous MMA (shared memory is
// not read for A), releasing the buffer afterwards.
__device__ __forceinline__ void mma_tf32_reuse_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                 uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// kind::f16 forms of the three MMAs above (K = 16 per instruction).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_f16_keep_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_f16_reuse_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on the mbarrier once every tcgen05.mma issued so far by this thread
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// One arrival, when this thread's MMAs so far are done, on the barrier at
// `bar`'s offset in every CTA of the cluster in `mask`.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// Barrier of every thread of the cluster (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane, loaded and
// waited for inside one asm statement so that no use of the registers can
// be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16_sync(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 16-column loads (two TMEM addresses of this thread's lane) and one
// wait.
__device__ __forceinline__ void tmem_ld16x2_sync(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, "
      "%25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[16 + i]);
  }
}

// 16 consecutive 32-bit columns of this thread's TMEM lane stored, and the
// store waited for (so that a later tcgen05.ld of the same columns sees it).
__device__ __forceinline__ void tmem_st16_sync(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane stored, without
// the wait (see tmem_wait_st).
__device__ __forceinline__ void tmem_st16_nowait(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

// 16x256b accesses: in a 16-lane half of the warp's lane quarter, thread t
// holds lanes t/4 and t/4 + 8, columns 2(t%4) and 2(t%4) + 1 of an 8-column
// group.  The quad form below covers a warp's 32 lanes and 16 columns
// (halves h = 0, 1 at lane offsets 0 and 16; groups g = 0, 1 at column
// offsets 0 and 8): thread t gets rows r = t/4 + {0, 8, 16, 24} and columns
// 2(t%4) + {0, 1, 8, 9}, as v[ri][cj] with ri = 2h + i (row offset 16h + 8i)
// and cj = 2g + e (column offset 8g + e).  One wait covers the four loads.
__device__ __forceinline__ void tmem_ld_quad16(uint32_t ta, float (&v)[4][4]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0, %1, %2, %3}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%4, %5, %6, %7}, [%17];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%8, %9, %10, %11}, [%18];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%12, %13, %14, %15}, [%19];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta), "r"(ta + 8u), "r"(ta + (16u << 16)), "r"(ta + (16u << 16) + 8u)
      : "memory");
  // load k = 2h + g holds (i, e) = (0,0), (0,1), (1,0), (1,1)
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int e = 0; e < 2; ++e) v[2 * h + i][2 * g + e] = __uint_as_float(r[4 * (2 * h + g) + 2 * i + e]);
}

__device__ __forceinline__ void tmem_st_quad16(uint32_t ta, const float (&v)[4][4]) {
  uint32_t r[16];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int e = 0; e < 2; ++e) r[4 * (2 * h + g) + 2 * i + e] = __float_as_uint(v[2 * h + i][2 * g + e]);
  asm volatile(
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%4, %5, %6, %7};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%1], {%8, %9, %10, %11};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%2], {%12, %13, %14, %15};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%3], {%16, %17, %18, %19};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(ta),
      "r"(ta + 8u), "r"(ta + (16u << 16)), "r"(ta + (16u << 16) + 8u), "r"(r[0]), "r"(r[1]),
      "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// Two blocks of the quad form (two TMEM addresses), eight loads and one wait.
__device__ __forceinline__ void tmem_ld_quad16x2(uint32_t ta, uint32_t tb, float (&va)[4][4],
                                                 float (&vb)[4][4]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0, %1, %2, %3}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%4, %5, %6, %7}, [%33];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%8, %9, %10, %11}, [%34];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%12, %13, %14, %15}, [%35];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%16, %17, %18, %19}, [%36];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%20, %21, %22, %23}, [%37];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%24, %25, %26, %27}, [%38];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%28, %29, %30, %31}, [%39];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(ta), "r"(ta + 8u), "r"(ta + (16u << 16)), "r"(ta + (16u << 16) + 8u), "r"(tb),
        "r"(tb + 8u), "r"(tb + (16u << 16)), "r"(tb + (16u << 16) + 8u)
      : "memory");
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          va[2 * h + i][2 * g + e] = __uint_as_float(r[4 * (2 * h + g) + 2 * i + e]);
          vb[2 * h + i][2 * g + e] = __uint_as_float(r[16 + 4 * (2 * h + g) + 2 * i + e]);
        }
}

// The quad-form store without its wait: the caller issues tmem_wait_st()
// before anything that must see the stored values.
__device__ __forceinline__ void tmem_st_quad16_nowait(uint32_t ta, const float (&v)[4][4]) {
  uint32_t r[16];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int e = 0; e < 2; ++e) r[4 * (2 * h + g) + 2 * i + e] = __float_as_uint(v[2 * h + i][2 * g + e]);
  asm volatile(
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%4, %5, %6, %7};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%1], {%8, %9, %10, %11};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%2], {%12, %13, %14, %15};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%3], {%16, %17, %18, %19};" ::"r"(ta),
      "r"(ta + 8u), "r"(ta + (16u << 16)), "r"(ta + (16u << 16) + 8u), "r"(r[0]), "r"(r[1]),
      "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The same for one 16-lane half (lane offset already in ta): thread t holds
// rows t/4 and t/4 + 8 of the half, columns 2 (t % 4) + {0, 1} of each
// 8-column group.
__device__ __forceinline__ void tmem_ld_half16(uint32_t ta, float (&v)[2][4]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0, %1, %2, %3}, [%8];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%4, %5, %6, %7}, [%9];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(ta), "r"(ta + 8u)
      : "memory");
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int e = 0; e < 2; ++e) v[i][2 * g + e] = __uint_as_float(r[4 * g + 2 * i + e]);
}

__device__ __forceinline__ void tmem_st_half16(uint32_t ta, const float (&v)[2][4]) {
  uint32_t r[8];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int e = 0; e < 2; ++e) r[4 * g + 2 * i + e] = __float_as_uint(v[i][2 * g + e]);
  asm volatile(
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%2, %3, %4, %5};\n\t"
      "tcgen05.st.sync.aligned.16x256b.x1.b32 [%1], {%6, %7, %8, %9};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(ta),
      "r"(ta + 8u), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
      "r"(r[7])
      : "memory");
}

// TF32 head of an fp32 value: x rounded to nearest (ties away) at 10
// explicit mantissa bits, low 13 bits zero, so that the tensor core sees it
// exactly whether it truncates or rounds its inputs; the tail x - head is
// exact in fp32 and at most half a TF32 ulp of x.  Finite inputs of the
// magnitudes met here (|x| < 2^127) cannot round up to infinity.
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

}  // namespace tc
}  // namespace rpchol
