// replicas.cu -- replicated gradient buffers for the dense levels (F = 2).
//
// The coarsest dense levels hold few entries (44k and 122k at the paper
// shape), and every Gaussian reduces into 16 of them per level, so within a
// backward call each of their entries takes hundreds of FP32 reductions;
// the L2 applies reductions to one address one after another.  The backward
// kernels therefore reduce from CTA b into replica b % k[l] of each such
// level (see Replicas in dash_internal.cuh); this file lays the replicas
// out in the caller's workspace, clears them before the kernels and adds
// them into the gradient buffer after.  The sum is exact up to the order of
// the FP32 additions.
#include "dash_internal.cuh"

#include <string.h>

namespace dash {

constexpr long long kRepSmall = 1ll << 17;

Replicas replica_plan(const dash_layout* layout, int k, size_t* bytes) {
  Replicas r;
  memset(&r, 0, sizeof(r));
  *bytes = 0;
  if (layout == nullptr || layout->F != 2 || k < 2) return r;
  // the leading dense levels small enough for their entries to take many
  // reductions each per call: k replicas of each level of at most 2^17
  // entries (measured inside the benchmark step: replicating the next,
  // 357k-entry level as well took enough L2 room from the gradients and
  // the forward's tables to make the step slower)
  int lv = 0;
  long long off = 0;
  while (lv < layout->L && lv < kMaxRepLevels && layout->dense[lv]) {
    const long long size = layout->size[lv];
    const int kl = size <= kRepSmall ? k : 0;
    if (kl < 2) break;
    const long long stride = (size * 2 + 63) & ~63ll;  // floats; replicas start 256-byte aligned
    r.k[lv] = kl;
    r.off[lv] = off;
    r.stride[lv] = stride;
    r.size[lv] = size;
    off += stride * kl;
    ++lv;
  }
  r.levels = lv;
  *bytes = (size_t)off * sizeof(float);
  return r;
}

int replica_clear(const Replicas& rp, size_t bytes, cudaStream_t st) {
  if (rp.levels == 0 || bytes == 0) return DASH_OK;
  return cuda_status(DASH_RT(cudaMemsetAsync(rp.base, 0, bytes, st)), "cudaMemsetAsync(gradient replicas)");
}

namespace {

struct SumArgs {
  Replicas rp;
  float* grad;
  long long goff[kMaxRepLevels];     // floats from grad to level l
  long long entries[kMaxRepLevels];  // entries of level l
  long long total;                   // entries of all replicated levels
};

// One thread per entry of the replicated levels: the k replicas' float2 in
// replica order, then added to the gradient buffer (no other writer runs).
__global__ void __launch_bounds__(256) replica_sum_kernel(const __grid_constant__ SumArgs a) {
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < a.total; e += step) {
    int l = 0;
    long long i = e;
    while (l + 1 < a.rp.levels && i >= a.entries[l]) {
      i -= a.entries[l];
      ++l;
    }
    const float* src = a.rp.base + a.rp.off[l] + 2 * i;
    float sx = 0.0f, sy = 0.0f;
    for (int r = 0; r < a.rp.k[l]; ++r) {
      const float2 v = __ldcs(reinterpret_cast<const float2*>(src + (long long)r * a.rp.stride[l]));
      sx += v.x;
      sy += v.y;
    }
    float2* d = reinterpret_cast<float2*>(a.grad + a.goff[l] + 2 * i);
    float2 g = *d;
    g.x += sx;
    g.y += sy;
    *d = g;
  }
}

}  // namespace

int replica_sum(const Geom& g, const Replicas& rp, float* grad, cudaStream_t st) {
  if (rp.levels == 0) return DASH_OK;
  SumArgs a;
  memset(&a, 0, sizeof(a));
  a.rp = rp;
  a.grad = grad;
  a.total = 0;
  for (int l = 0; l < rp.levels; ++l) {
    a.goff[l] = g.offset[l] * 2;
    a.entries[l] = rp.size[l];
    a.total += a.entries[l];
  }
  const long long blocks = (a.total + 255) / 256;
  const long long cap = 4ll * sm_count();
  replica_sum_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(a);
  return launch_status("replica_sum_kernel");
}

}  // namespace dash
