// collisions.cu -- per-level hash-table occupancy of a point set: the
// distinct grid vertices V its hypervoxel corners touch, the distinct table
// entries E they occupy, and the touched vertices C that share their entry
// with another touched vertex.  This measures the collision argument of
// Sec. 4.2 (encoding only the dynamic Gaussians keeps the 4-D tables from
// being crowded) and the "w/o dec" ablation of Sec. 5.
//
// Per level: every corner's vertex id is inserted into an open-addressed set
// of 64-bit keys in the workspace; a vertex seen for the first time adds one
// to its entry's counter.  A reduction over the counters then gives
// V = sum of counts, E = number of non-zero counts, C = sum of counts >= 2.
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kEmpty = ~0ull;

struct CollWs {
  unsigned long long* set;  // [slots], kEmpty = free
  unsigned int* count;      // [max level size]
  unsigned int* flag;       // 1: a probe sequence ran out (the set was too small)
  unsigned long long slots;
};

// splitmix64's output finaliser (Steele, Lea and Flood, 2014): spreads
// consecutive vertex ids over the set's slots.
__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
  k ^= k >> 30;
  k *= 0xbf58476d1ce4e5b9ull;
  k ^= k >> 27;
  k *= 0x94d049bb133111ebull;
  k ^= k >> 31;
  return k;
}

__global__ void __launch_bounds__(kThreads) touch_kernel(Geom g, Pts pts, int l, CollWs ws) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 p = load_point(pts, i);
  uint32_t idx[16];
  float w[16];
  level_corners(g, l, p, idx, w);
  const int ns = g.res_s[l], nt = g.res_t[l];
  int c0[4];
  float fr;
  axis_cell(p.x, ns, c0[0], fr);
  axis_cell(p.y, ns, c0[1], fr);
  axis_cell(p.z, ns, c0[2], fr);
  axis_cell(p.w, nt, c0[3], fr);
  const unsigned long long R = (unsigned long long)ns + 1ull;
  const unsigned long long mask = ws.slots - 1ull;
#pragma unroll 1
  for (int b = 0; b < 16; ++b) {
    const unsigned long long cx = (unsigned long long)(c0[0] + (b & 1));
    const unsigned long long cy = (unsigned long long)(c0[1] + ((b >> 1) & 1));
    const unsigned long long cz = (unsigned long long)(c0[2] + ((b >> 2) & 1));
    const unsigned long long ct = (unsigned long long)(c0[3] + ((b >> 3) & 1));
    const unsigned long long key = cx + R * (cy + R * (cz + R * ct));
    unsigned long long slot = mix64(key) & mask;
    bool placed = false;
    for (unsigned long long probe = 0; probe < ws.slots; ++probe) {
      const unsigned long long seen = __ldcg(ws.set + slot);
      if (seen == key) {
        placed = true;
        break;
      }
      if (seen == kEmpty) {
        const unsigned long long prev = atomicCAS(ws.set + slot, kEmpty, key);
        if (prev == kEmpty) {
          atomicAdd(ws.count + idx[b], 1u);
          placed = true;
          break;
        }
        if (prev == key) {
          placed = true;
          break;
        }
      }
      slot = (slot + 1ull) & mask;
    }
    if (!placed) atomicOr(ws.flag, 1u);
  }
}

// Adds one level's V, E, C (from its entry counters) into stats[0..3).
__global__ void __launch_bounds__(kThreads) occupancy_kernel(const unsigned int* __restrict__ count, long long size,
                                                             int64_t* stats) {
  unsigned long long v = 0, e = 0, c = 0;
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < size; k += (long long)gridDim.x * kThreads) {
    const unsigned int m = count[k];
    v += m;
    e += m != 0u;
    c += m >= 2u ? m : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(0xffffffffu, v, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(stats + 0), v);
    atomicAdd(reinterpret_cast<unsigned long long*>(stats + 1), e);
    atomicAdd(reinterpret_cast<unsigned long long*>(stats + 2), c);
  }
}

// All three set to -1 if a probe sequence ran out (cannot happen with the
// workspace size below; kept as a checked failure instead of a wrong count).
__global__ void mark_overflow(const unsigned int* flag, int64_t* stats) {
  if (*flag != 0u) stats[0] = stats[1] = stats[2] = -1;
}

unsigned long long set_slots(long long n) {
  unsigned long long need = 2ull * 16ull * (unsigned long long)(n > 0 ? n : 1);
  unsigned long long s = 1024ull;
  while (s < need) s <<= 1;
  return s;
}

long long max_level_size(const dash_layout* lo) {
  long long m = 0;
  for (int l = 0; l < lo->L; ++l) m = lo->size[l] > m ? lo->size[l] : m;
  return m;
}

}  // namespace
}  // namespace dash

extern "C" {

size_t dash_collision_workspace_size(const dash_layout* layout, int64_t n) {
  using namespace dash;
  if (layout == nullptr || n < 0) return 0;
  const size_t set_bytes = (size_t)set_slots(n) * 8u;
  const size_t count_bytes = ((size_t)max_level_size(layout) * 4u + 255u) & ~(size_t)255u;
  return set_bytes + count_bytes + 256u;
}

int dash_hash4d_collision_stats(const dash_layout* layout, const dash_points* pts, int64_t* stats_out, void* ws,
                                size_t ws_bytes, void* stream) {
  DASH_NVTX_RANGE("dash_hash4d_collision_stats");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = make_geom(layout, &g)) return s;
  if (int s = make_pts(pts, &p)) return s;
  if (stats_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "stats_out is NULL");
  for (int l = 0; l < g.L; ++l) {
    const double R = (double)g.res_s[l] + 1.0, Rt = (double)g.res_t[l] + 1.0;
    if (R * R * R * Rt >= 9.2e18) return fail(DASH_ERR_UNSUPPORTED, "level %d has too many vertices for 64-bit ids", l);
  }
  const size_t need = dash_collision_workspace_size(layout, p.n);
  if (ws == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes (256-byte aligned), %zu needed", ws_bytes, need);
  cudaStream_t st = as_stream(stream);
  CollWs w;
  w.slots = set_slots(p.n);
  uint8_t* base = static_cast<uint8_t*>(ws);
  w.set = reinterpret_cast<unsigned long long*>(base);
  w.count = reinterpret_cast<unsigned int*>(base + w.slots * 8u);
  const size_t count_bytes = ((size_t)max_level_size(layout) * 4u + 255u) & ~(size_t)255u;
  w.flag = reinterpret_cast<unsigned int*>(base + w.slots * 8u + count_bytes);
  if (int s = cuda_status(DASH_RT(cudaMemsetAsync(stats_out, 0, sizeof(int64_t) * 3u * (size_t)g.L, st)), "cudaMemsetAsync"))
    return s;
  const unsigned grid = (unsigned)((p.n + kThreads - 1) / kThreads);
  for (int l = 0; l < g.L; ++l) {
    const long long size = layout->size[l];
    if (int s = cuda_status(DASH_RT(cudaMemsetAsync(w.set, 0xFF, (size_t)w.slots * 8u, st)), "cudaMemsetAsync")) return s;
    if (int s = cuda_status(DASH_RT(cudaMemsetAsync(w.count, 0, (size_t)size * 4u, st)), "cudaMemsetAsync")) return s;
    if (int s = cuda_status(DASH_RT(cudaMemsetAsync(w.flag, 0, 4u, st)), "cudaMemsetAsync")) return s;
    if (p.n > 0) {
      touch_kernel<<<grid, kThreads, 0, st>>>(g, p, l, w);
      if (int s = launch_status("touch_kernel")) return s;
    }
    long long blocks = (size + kThreads - 1) / kThreads;
    const long long cap = 4ll * sm_count();
    blocks = blocks < cap ? (blocks > 0 ? blocks : 1) : cap;
    occupancy_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(w.count, size, stats_out + 3 * l);
    if (int s = launch_status("occupancy_kernel")) return s;
    mark_overflow<<<1, 1, 0, st>>>(w.flag, stats_out + 3 * l);
    if (int s = launch_status("mark_overflow")) return s;
  }
  return DASH_OK;
}

}  // extern "C"
