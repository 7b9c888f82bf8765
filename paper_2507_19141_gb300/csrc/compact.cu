// compact.cu -- a1: the dynamic index list of the self-supervised
// static/dynamic split (Sec. 4.1: Gaussians above the motion threshold are
// dynamic; the 4D encoder runs on those only, Sec. 4.2).
//
// Three passes over the byte mask, CHUNK bytes per CTA:
//   count: per-CTA number of nonzero bytes -> ws[cta]
//   scan:  one CTA turns ws[] into exclusive offsets, writes the total
//   write: per-CTA exclusive scan of per-thread counts, indices staged in
//          shared memory and stored contiguously (ascending order).
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kThreads = 256;
constexpr int kBytesPerThread = 16;
constexpr int kChunk = kThreads * kBytesPerThread;  // 4096 mask bytes per CTA

// Bit 7 of each byte set iff that byte of v is nonzero.
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t v) {
  return (((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
}

// Loads this thread's 16 mask bytes as four words; bytes past n read as 0.
__device__ __forceinline__ void load16(const uint8_t* __restrict__ mask, long long n, long long start,
                                       uint32_t w[4]) {
  if (start + kBytesPerThread <= n && ((reinterpret_cast<uintptr_t>(mask + start) & 15u) == 0)) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(mask + start));
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const long long i = start + 4 * k + b;
        const uint32_t byte = i < n ? (uint32_t)mask[i] : 0u;
        v |= byte << (8 * b);
      }
      w[k] = v;
    }
  }
}

__device__ __forceinline__ int count16(const uint32_t w[4]) {
  return __popc(nonzero_bytes(w[0])) + __popc(nonzero_bytes(w[1])) + __popc(nonzero_bytes(w[2])) +
         __popc(nonzero_bytes(w[3]));
}

// Exclusive block-wide prefix sum over kThreads values; returns the total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += u;
    }
    if (lane < kThreads / 32) warp_sums[lane] = si - s;  // exclusive warp offsets
    if (lane == kThreads / 32 - 1) warp_sums[kThreads / 32] = si;
  }
  __syncthreads();
  total = warp_sums[kThreads / 32];
  return warp_sums[warp] + incl - v;
}

__global__ void __launch_bounds__(kThreads) compact_count(const uint8_t* __restrict__ mask, long long n,
                                                          int* __restrict__ cta_counts) {
  __shared__ int warp_sums[kThreads / 32 + 1];
  const long long start = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kBytesPerThread;
  uint32_t w[4];
  load16(mask, n, start, w);
  int total;
  block_exclusive_scan(count16(w), warp_sums, total);
  if (threadIdx.x == 0) cta_counts[blockIdx.x] = total;
}

// One CTA: exclusive offsets in place over nb counts, total to *count_out.
__global__ void __launch_bounds__(1024) compact_scan(int* __restrict__ cta_counts, int nb,
                                                     long long* __restrict__ count_out) {
  __shared__ int warp_sums[33];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? cta_counts[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int s = warp_sums[lane];
      int si = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += u;
      }
      warp_sums[lane] = si - s;
      if (lane == 31) warp_sums[32] = si;
    }
    __syncthreads();
    if (i < nb) cta_counts[i] = (int)(carry + warp_sums[warp] + incl - v);
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count_out = carry;
}

__global__ void __launch_bounds__(kThreads) compact_write(const uint8_t* __restrict__ mask, long long n,
                                                          const int* __restrict__ cta_offsets,
                                                          int* __restrict__ idx_out) {
  __shared__ int warp_sums[kThreads / 32 + 1];
  __shared__ int staged[kChunk];
  const long long cta_start = (long long)blockIdx.x * kChunk;
  const long long start = cta_start + (long long)threadIdx.x * kBytesPerThread;
  uint32_t w[4];
  load16(mask, n, start, w);
  int total;
  int pos = block_exclusive_scan(count16(w), warp_sums, total);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t nz = nonzero_bytes(w[k]);
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (nz & (0x80u << (8 * b))) staged[pos++] = (int)(start + 4 * k + b);
  }
  __syncthreads();
  int* dst = idx_out + cta_offsets[blockIdx.x];
  for (int i = threadIdx.x; i < total; i += kThreads) dst[i] = staged[i];
}

}  // namespace

int compact_launch(const uint8_t* mask, long long n, int* idx_out, long long* count_out, int* cta_scratch,
                   cudaStream_t st) {
  const long long nb = (n + kChunk - 1) / kChunk;
  if (nb > 0) {
    compact_count<<<(unsigned)nb, kThreads, 0, st>>>(mask, n, cta_scratch);
    if (int s = launch_status("compact_count")) return s;
  }
  compact_scan<<<1, 1024, 0, st>>>(cta_scratch, (int)nb, count_out);
  if (int s = launch_status("compact_scan")) return s;
  if (nb > 0) {
    compact_write<<<(unsigned)nb, kThreads, 0, st>>>(mask, n, cta_scratch, idx_out);
    if (int s = launch_status("compact_write")) return s;
  }
  return DASH_OK;
}

long long compact_blocks(long long n) { return (n + kChunk - 1) / kChunk; }

}  // namespace dash

extern "C" {

size_t dash_compact_workspace_size(int64_t n) {
  if (n < 0) return 0;
  const long long nb = dash::compact_blocks(n);
  return (size_t)((nb * (long long)sizeof(int) + 255) / 256 * 256) + 256;
}

int dash_compact_dynamic(const uint8_t* mask, int64_t n, int32_t* idx_out, int64_t* count_out, void* ws,
                         size_t ws_bytes, void* stream) {
  DASH_NVTX_RANGE("dash_compact_dynamic");
  using dash::fail;
  if (n < 0) return fail(DASH_ERR_INVALID_ARG, "n=%lld < 0", (long long)n);
  if (n >= (1ll << 31)) return fail(DASH_ERR_UNSUPPORTED, "n >= 2^31");
  if (count_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "count_out is NULL");
  if (n > 0 && (mask == nullptr || idx_out == nullptr)) return fail(DASH_ERR_INVALID_ARG, "mask/idx_out is NULL");
  if (ws == nullptr || ws_bytes < dash_compact_workspace_size(n))
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, dash_compact_workspace_size(n));
  return dash::compact_launch(mask, n, idx_out, reinterpret_cast<long long*>(count_out), static_cast<int*>(ws),
                              dash::as_stream(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Compaction without any allocation.  For callers that must not allocate
// device memory once they are running -- for example a render loop that owns
// all device memory and hands its plug-ins only the buffers it allocated up
// front, or code that runs inside a memory allocator's own callbacks, where a
// cudaMalloc would re-enter that allocator.  The per-CTA counts live in this
// file-scope array instead of a caller workspace; every GPU that loads the
// library holds it (256 KB) until the process exits.  Its device address is
// resolved once per device and cached for the life of the process: valid
// for the device's primary context and until a cudaDeviceReset of that
// device.  Device code is loaded lazily, so the first call on a device may
// itself allocate; callers warm up with one call per device (n >= 1).
// ---------------------------------------------------------------------------
#include <mutex>

namespace dash {
namespace {

constexpr long long kNoAllocMaxCtas = 65536;                 // 256 KB of int32 counts
constexpr long long kNoAllocMaxN = kNoAllocMaxCtas * kChunk;  // 268,435,456 mask entries

static __device__ __align__(256) int g_noalloc_cta_counts[kNoAllocMaxCtas];

std::mutex g_noalloc_mutex;
int* g_noalloc_ptr[64] = {nullptr};

// Device address of the array on the current device, resolved once per
// device (host code cannot use the symbol itself: on the host it names a
// stand-in, not device memory).
int noalloc_scratch(int** out) {
  int dev = 0;
  if (int s = cuda_status(DASH_RT(cudaGetDevice(&dev)), "cudaGetDevice")) return s;
  if (dev < 0 || dev >= 64) return fail(DASH_ERR_UNSUPPORTED, "device ordinal %d >= 64", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (int s = cuda_status(DASH_RT(cudaGetSymbolAddress(&p, g_noalloc_cta_counts)), "cudaGetSymbolAddress")) return s;
    g_noalloc_ptr[dev] = static_cast<int*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return DASH_OK;
}

}  // namespace
}  // namespace dash

extern "C" int dash_compact_dynamic_noalloc(const uint8_t* mask, int64_t n, int32_t* idx_out, int64_t* count_out,
                                            void* stream) {
  using dash::fail;
  if (n < 0) return fail(DASH_ERR_INVALID_ARG, "n=%lld < 0", (long long)n);
  if (n > dash::kNoAllocMaxN)
    return fail(DASH_ERR_UNSUPPORTED, "n=%lld exceeds the %lld-entry limit of the built-in scratch array",
                (long long)n, dash::kNoAllocMaxN);
  if (count_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "count_out is NULL");
  if (n > 0 && (mask == nullptr || idx_out == nullptr)) return fail(DASH_ERR_INVALID_ARG, "mask/idx_out is NULL");
  int* scratch = nullptr;
  if (int s = dash::noalloc_scratch(&scratch)) return s;
  // The count pass writes every slot that the scan and write passes read, so
  // what earlier calls left in the array never needs clearing.
  return dash::compact_launch(mask, n, idx_out, reinterpret_cast<long long*>(count_out), scratch,
                              dash::as_stream(stream));
}
