// selftest.cu -- exercises the path a tensor-core kernel takes when one of its bounded device
// waits gives up, without any fault: a CTA allocates TMEM, waits on an mbarrier that nothing
// arrives on (the same bounded wait, %globaltimer-limited, that every producer / MMA / epilogue
// wait uses), records ST_TIMEOUT, frees its TMEM and returns.  The host maps the status to
// CTD_ERR_TIMEOUT and the context stays usable.
#include "ctx.cuh"
#include "umma.cuh"

namespace ctd {

__global__ void k_selftest_wait(uint64_t limit_ns, int* __restrict__ status, unsigned long long* __restrict__ waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    umma::mbar_init(&bar, 1);
    umma::mbar_fence_init();
  }
  if (warp == 0) umma::tmem_alloc(&tslot, 32);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (threadIdx.x == 0) {
    const uint64_t t0 = umma::globaltimer();
    const bool ok = umma::mbar_wait(&bar, 0, limit_ns);   // no arrival: gives up after limit_ns
    *waited_ns = umma::globaltimer() - t0;
    if (!ok) atomicOr(status, (int)ST_TIMEOUT);
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 0) umma::tmem_dealloc(tslot, 32);
}

}  // namespace ctd

using namespace ctd;

extern "C" int ctd_selftest_wait(ctd_ctx* c, double limit_ms, double* waited_ms) {
  if (!c) return CTD_ERR_INVALID_ARG;
  Bind bind_(c);
  if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) return fail(c, CTD_ERR_INVALID_ARG, "limit_ms must be in (0, 2000]");
  ENSURE(c, c->status, sizeof(int32_t) * 4);
  ENSURE(c, c->out_e, sizeof(double) * 4);
  cudaStream_t st = c->st;
  CUDA_OK(c, cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), st));
  {
    LaunchScope ls_(st);
    k_selftest_wait<<<1, 64, 0, st>>>((uint64_t)(limit_ms * 1e6), P<int>(c->status),
                                     reinterpret_cast<unsigned long long*>(c->out_e.p));
  }
  CUDA_OK(c, cudaGetLastError());
  unsigned long long ns = 0;
  CUDA_OK(c, cudaMemcpyAsync(&ns, c->out_e.p, sizeof(ns), cudaMemcpyDeviceToHost, st));
  const int r = check_status(c);   // synchronises; CTD_ERR_TIMEOUT when the wait gave up
  if (waited_ms) *waited_ms = (double)ns * 1e-6;
  return r;
}
