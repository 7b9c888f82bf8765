// probes.cu -- rate probes for the access patterns that bound the fused
// kernels, so a benchmark can put a measured ceiling beside each kernel's
// own rate (the HBM copy peak does not bind: the tables and gradients sit in
// L2).  Each probe issues `iters` operations per thread at pseudo-random
// addresses spread over a caller buffer (sized like the tables or the
// gradient buffer, so it stays L2-resident) and reports how many it issued;
// the caller times the launch.  The paper has no counterpart.
//
//   DASH_PROBE_RED8     one 8-byte FP32 vector reduction per lane, each lane
//                       its own random entry (the backward's per-corner form)
//   DASH_PROBE_RED16    one 16-byte FP32 vector reduction per lane, random
//   DASH_PROBE_RED8_PAIRED  lanes 2j and 2j+1 reduce 8 bytes each into the
//                       two halves of one 16-byte group in the same
//                       instruction (the backward's lane-paired x-neighbours
//                       when they share a sector)
//   DASH_PROBE_GATHER4  one 4-byte load per lane from a random entry (the
//                       forward's per-corner FP16 F = 2 gather)
//   DASH_PROBE_GATHER4_PAIRED  lanes 2j and 2j+1 load neighbouring 4-byte
//                       entries of one 8-byte group in the same instruction
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kProbeThreads = 256;

// A 32-bit mix (multiply-xorshift) of the thread's operation counter.
__device__ __forceinline__ uint32_t mix32(uint32_t v) {
  v ^= v >> 16;
  v *= 0x7feb352du;
  v ^= v >> 15;
  v *= 0x846ca68bu;
  v ^= v >> 16;
  return v;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(float* __restrict__ buf, uint32_t groups, int iters,
                                                              float* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  // paired kinds: both lanes of a pair draw the same group
  const uint32_t key = (KIND == DASH_PROBE_RED8_PAIRED || KIND == DASH_PROBE_GATHER4_PAIRED) ? (tid >> 1) : tid;
  float acc = 0.0f;
  for (int i = 0; i < iters; ++i) {
    const uint32_t gidx = mix32(key * 0x9E3779B1u + (uint32_t)i * 0x85EBCA77u) % groups;  // a 16-byte group
    if constexpr (KIND == DASH_PROBE_RED8) {
      red_add_v2(buf + (size_t)gidx * 4 + 2 * (mix32(key + (uint32_t)i) & 1u), 1.0f, 1.0f);
    } else if constexpr (KIND == DASH_PROBE_RED16) {
      red_add_v4(buf + (size_t)gidx * 4, 1.0f, 1.0f, 1.0f, 1.0f);
    } else if constexpr (KIND == DASH_PROBE_RED8_PAIRED) {
      red_add_v2(buf + (size_t)gidx * 4 + 2 * (lane & 1u), 1.0f, 1.0f);
    } else if constexpr (KIND == DASH_PROBE_GATHER4) {
      acc += __ldg(buf + (size_t)gidx * 4 + (mix32(key + (uint32_t)i) & 3u));
    } else {  // DASH_PROBE_GATHER4_PAIRED
      acc += __ldg(buf + (size_t)gidx * 4 + (lane & 1u));
    }
  }
  if (KIND == DASH_PROBE_GATHER4 || KIND == DASH_PROBE_GATHER4_PAIRED) sink[tid] = acc;  // keeps the loads
}

}  // namespace
}  // namespace dash

extern "C" int dash_probe_threads(int kind) {
  (void)kind;
  return dash::sm_count() * 8 * dash::kProbeThreads;
}

extern "C" int dash_probe_rate(int kind, float* buf, size_t buf_bytes, int iters, float* sink, int64_t* ops_out,
                               void* stream) {
  DASH_NVTX_RANGE("dash_probe_rate");
  using namespace dash;
  if (buf == nullptr || ops_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "buf/ops_out is NULL");
  if ((reinterpret_cast<uintptr_t>(buf) & 15u) != 0) return fail(DASH_ERR_INVALID_ARG, "buf must be 16-byte aligned");
  if (buf_bytes < 16 || buf_bytes / 16 > 0xFFFFFFFFull) return fail(DASH_ERR_INVALID_ARG, "buf_bytes out of range");
  if (iters < 1 || iters > (1 << 16)) return fail(DASH_ERR_INVALID_ARG, "iters=%d outside [1, 65536]", iters);
  const bool gather = kind == DASH_PROBE_GATHER4 || kind == DASH_PROBE_GATHER4_PAIRED;
  if (gather && sink == nullptr) return fail(DASH_ERR_INVALID_ARG, "the gather probes need a sink of one float per thread");
  const int threads = dash_probe_threads(kind);
  const unsigned blocks = (unsigned)(threads / kProbeThreads);
  const uint32_t groups = (uint32_t)(buf_bytes / 16);
  cudaStream_t st = as_stream(stream);
  switch (kind) {
    case DASH_PROBE_RED8: probe_kernel<DASH_PROBE_RED8><<<blocks, kProbeThreads, 0, st>>>(buf, groups, iters, sink); break;
    case DASH_PROBE_RED16: probe_kernel<DASH_PROBE_RED16><<<blocks, kProbeThreads, 0, st>>>(buf, groups, iters, sink); break;
    case DASH_PROBE_RED8_PAIRED:
      probe_kernel<DASH_PROBE_RED8_PAIRED><<<blocks, kProbeThreads, 0, st>>>(buf, groups, iters, sink);
      break;
    case DASH_PROBE_GATHER4: probe_kernel<DASH_PROBE_GATHER4><<<blocks, kProbeThreads, 0, st>>>(buf, groups, iters, sink); break;
    case DASH_PROBE_GATHER4_PAIRED:
      probe_kernel<DASH_PROBE_GATHER4_PAIRED><<<blocks, kProbeThreads, 0, st>>>(buf, groups, iters, sink);
      break;
    default: return fail(DASH_ERR_INVALID_ARG, "unknown probe kind %d", kind);
  }
  if (int s = launch_status("probe_kernel")) return s;
  *ops_out = (int64_t)threads * iters;
  return DASH_OK;
}
