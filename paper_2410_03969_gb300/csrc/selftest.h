// Failure-detection self-tests of the bounded device waits (internal; the
// public entry point is rpchol_selftest_wait in include/rpchol.h).  Each
// launches one thread that waits on an mbarrier nothing completes and writes
// out[0] = 1 if the wait gave up, out[1] = the time it waited (ns).
#pragma once
#include <cuda_runtime.h>

namespace rpchol {
// cluster-scope wait of Algorithm 1 (k_round.cu)
cudaError_t launch_wait_selftest_cluster(unsigned long long limit_ns, unsigned long long* out,
                                         cudaStream_t s);
// CTA-scope wait of the tensor-core column step's pipeline (k_selftest.cu)
cudaError_t launch_wait_selftest_cta(unsigned long long limit_ns, unsigned long long* out,
                                     cudaStream_t s);
}  // namespace rpchol
