// selftest.cu -- the device-side failure report exercised on purpose.
//
// The persistent kernels bound every mbarrier wait; when a bound runs out
// they set a device flag word, stop issuing and return, and
// dash_device_status reports DASH_ERR_TIMEOUT.  dash_selftest_wait runs that
// path in isolation: one thread waits, with a caller-given poll bound, on a
// shared-memory mbarrier that nothing ever arrives at, so the wait always
// runs out; the kernel sets its flag word and returns.  Nothing faults and
// nothing spins without a bound: the context stays usable.
#include "dash_internal.cuh"
#include "tc_ptx.cuh"

namespace dash {
namespace {

__device__ unsigned int g_selftest_flags;

__global__ void __launch_bounds__(32) selftest_wait_kernel(uint32_t polls, unsigned int* flags) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    const uint32_t a = tc::smem_addr(&bar);
    tc::mbar_init(a, 1u);  // one arrival expected; none ever comes
    tc::mbar_init_fence();
    if (!tc::mbar_wait(a, 0u, polls)) atomicOr(flags, 1u);
  }
}

}  // namespace

namespace fused {
unsigned int* selftest_flags_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_selftest_flags) != cudaSuccess) return nullptr;
  return static_cast<unsigned int*>(p);
}
}  // namespace fused

}  // namespace dash

extern "C" int dash_selftest_wait(int64_t polls, void* stream) {
  DASH_NVTX_RANGE("dash_selftest_wait");
  using namespace dash;
  if (polls < 1 || polls > (1ll << 22)) return fail(DASH_ERR_INVALID_ARG, "polls=%lld outside [1, 2^22]", (long long)polls);
  unsigned int* flags = fused::selftest_flags_ptr();
  if (flags == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the self-test flag word");
  selftest_wait_kernel<<<1, 32, 0, as_stream(stream)>>>((uint32_t)polls, flags);
  return launch_status("selftest_wait_kernel");
}
