// CTA-scope bounded-wait self-test: the same mbar_wait_bounded the
// tensor-core column step's pipeline uses, on a barrier nothing completes.
#include <cuda_runtime.h>

#include "internal.h"
#include "selftest.h"
#include "tc_ptx.cuh"

namespace rpchol {
namespace {

__global__ void k_wait_selftest_cta(unsigned long long limit_ns, unsigned long long* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  tc::mbar_init(&bar, 1);
  tc::fence_mbarrier_init();
  const unsigned long long t0 = tc::globaltimer_ns();
  const bool ok = tc::mbar_wait_bounded(&bar, 0u, limit_ns, &abort_flag);
  const unsigned long long t1 = tc::globaltimer_ns();
  out[0] = (!ok && abort_flag) ? 1ull : 0ull;
  out[1] = t1 - t0;
}

}  // namespace

cudaError_t launch_wait_selftest_cta(unsigned long long limit_ns, unsigned long long* out,
                                     cudaStream_t s) {
  k_wait_selftest_cta<<<1, 32, 0, s>>>(limit_ns, out);
  return cudaGetLastError();
}

}  // namespace rpchol
