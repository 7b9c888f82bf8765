// dash_internal.cuh -- device-side building blocks shared by the libdash
// kernels: level geometry, point loads, the Eq. 8 corner hash and the Eq. 9
// quadrilinear weights, plus host-side error plumbing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "dash.h"

namespace dash {

// ------------------------------------------------------------------ host --
void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
// Records a CUDA failure (launch or runtime call) and returns DASH_ERR_CUDA.
int cuda_status(cudaError_t e, const char* what);
// Fault-injection hook (dash_debug_fail_cuda_call): counts the checked CUDA
// runtime calls and returns true for the one the hook names.
bool fault_due();
// A checked CUDA runtime call: made unless the fault-injection hook names
// it, in which case it is not made and fails (cuda_status then reports an
// injected failure).  Every runtime call the library checks goes through it.
#define DASH_RT(call) (::dash::fault_due() ? ::cudaErrorUnknown : (call))
// Checks the last launch on this thread.
int launch_status(const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// An NVTX range over one C-ABI call (header-only NVTX; costs nothing
// measurable unless a profiler is attached), so timelines show which
// library entry point issued which kernels.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define DASH_NVTX_RANGE(name) ::dash::NvtxRange dash_nvtx_range_(name)

// Number of SMs of the current device (cached per device).
int sm_count();

// Kernel-form options (dash_set_option).
extern int g_opt_fwd_form;
extern int g_opt_bwd_form;
extern int g_opt_access_form;
extern int g_opt_grad_replicas;
extern int g_opt_decomp_form;

// ------------------------------------------------ kernel-side geometry ----
// Level layout in the form the kernels read it (by-value kernel argument).
struct Geom {
  int L, F;
  uint32_t mask;       // T - 1 for hashed levels
  uint32_t dense_bits; // bit l set: level l is dense
  uint32_t primes[4];
  int res_s[DASH_MAX_LEVELS];
  int res_t[DASH_MAX_LEVELS];
  long long offset[DASH_MAX_LEVELS];
};

// Validates a host layout and converts it (INVALID_ARG / UNSUPPORTED on error).
int make_geom(const dash_layout* layout, Geom* g);

// Points as the kernels read them.
struct Pts {
  const float* x;
  const float* y;
  const float* z;
  const float* t;
  long long t_stride;
  const int* idx;
  long long n;
  const long long* n_dev;
  long long rows;         // DASH_DEBUG builds: point rows must be < rows (-1: unchecked)
  unsigned int* bounds;   // DASH_DEBUG builds: flag word set by a row index out of range
};

int make_pts(const dash_points* p, Pts* out);
// The device word the bounds checks of DASH_DEBUG builds set (dash_host.cu).
unsigned int* bounds_flags_ptr();

__device__ __forceinline__ long long point_count(const Pts& p) {
  long long n = p.n;
  if (p.n_dev != nullptr) {
    long long m = *p.n_dev;
    m = m < 0 ? 0 : m;
    n = m < n ? m : n;
  }
  return n;
}

// Clamp to [0,1]; NaN maps to 0 (fmaxf returns the non-NaN operand).
__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

// The row of compact point i in the full arrays.  In DASH_DEBUG builds a row
// outside [0, rows) sets the bounds flag and comes back as -1, and every
// caller then skips the access (the check runs before it).
__device__ __forceinline__ long long point_row(const Pts& p, long long i) {
  const long long j = p.idx != nullptr ? (long long)__ldcs(p.idx + i) : i;
#ifdef DASH_DEBUG
  if (p.rows >= 0 && (j < 0 || j >= p.rows)) {
    atomicOr(p.bounds, 1u);
    return -1;
  }
#endif
  return j;
}

// Clamped (x, y, z, t) of compact point i.
__device__ __forceinline__ float4 load_point(const Pts& p, long long i) {
  const long long j = point_row(p, i);
#ifdef DASH_DEBUG
  if (j < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
#endif
  float4 r;
  // coordinates are read once per kernel: streaming loads (evict first)
  r.x = clamp01(__ldcs(p.x + j));
  r.y = clamp01(__ldcs(p.y + j));
  r.z = clamp01(__ldcs(p.z + j));
  r.w = clamp01(p.t_stride != 0 ? __ldcs(p.t + j * p.t_stride) : __ldg(p.t));
  return r;
}

// One axis of the enclosing hypervoxel (Sec. 4.2): lower corner
// i0 = min(floor(x * N), N - 1) of the FP32 round-to-nearest product, and
// the exact fractional offset from it.
__device__ __forceinline__ void axis_cell(float x, int n, int& i0, float& frac) {
  const float pos = __fmul_rn(x, (float)n);
  int c = (int)floorf(pos);
  c = c < n - 1 ? c : n - 1;
  i0 = c;
  frac = __fsub_rn(pos, (float)c);  // exact: pos and c share the binade of pos
}

// The 16 corners of level l around p (Eq. 8) and their quadrilinear weights
// (Eq. 9).  Corner b: bit d set = upper corner along axis d (x, y, z, t).
// Indices are level-local.
__device__ __forceinline__ void level_corners(const Geom& g, int l, float4 p, uint32_t idx[16],
                                              float w[16]) {
  const int ns = g.res_s[l], nt = g.res_t[l];
  int ix, iy, iz, it;
  float fx, fy, fz, ft;
  axis_cell(p.x, ns, ix, fx);
  axis_cell(p.y, ns, iy, fy);
  axis_cell(p.z, ns, iz, fz);
  axis_cell(p.w, nt, it, ft);
  if ((g.dense_bits >> l) & 1u) {
    // collision-free direct index over (N_s+1)^3 (N_t+1) vertices, x fastest
    const uint32_t R = (uint32_t)ns + 1u;
    const uint32_t base = (uint32_t)ix + R * ((uint32_t)iy + R * ((uint32_t)iz + R * (uint32_t)it));
    const uint32_t sy = R, sz = R * R, st = R * R * R;
#pragma unroll
    for (int b = 0; b < 16; ++b)
      idx[b] = base + (b & 1) + ((b >> 1) & 1) * sy + ((b >> 2) & 1) * sz + ((b >> 3) & 1) * st;
  } else {
    // XOR of coordinate * prime, wrapping at 2^32, then mod T (a mask)
    const uint32_t hx0 = (uint32_t)ix * g.primes[0], hx1 = hx0 + g.primes[0];
    const uint32_t hy0 = (uint32_t)iy * g.primes[1], hy1 = hy0 + g.primes[1];
    const uint32_t hz0 = (uint32_t)iz * g.primes[2], hz1 = hz0 + g.primes[2];
    const uint32_t ht0 = (uint32_t)it * g.primes[3], ht1 = ht0 + g.primes[3];
#pragma unroll
    for (int b = 0; b < 16; ++b)
      idx[b] = ((b & 1 ? hx1 : hx0) ^ (b & 2 ? hy1 : hy0) ^ (b & 4 ? hz1 : hz0) ^ (b & 8 ? ht1 : ht0)) &
               g.mask;
  }
  const float wx0 = 1.0f - fx, wy0 = 1.0f - fy, wz0 = 1.0f - fz, wt0 = 1.0f - ft;
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    float v = (b & 1) ? fx : wx0;
    v *= (b & 2) ? fy : wy0;
    v *= (b & 4) ? fz : wz0;
    v *= (b & 8) ? ft : wt0;
    w[b] = v;
  }
}

// The indices of the 8 corners with x bit xb (corner b = xb | 2q, q = 0..7
// over the y, z, t bits) of the level-l hypervoxel whose lower corner is
// ci, with the arithmetic of level_corners.
__device__ __forceinline__ void cell_index_x(const Geom& g, int l, const int ci[4], uint32_t xb, uint32_t idx[8]) {
  if ((g.dense_bits >> l) & 1u) {
    const uint32_t R = (uint32_t)g.res_s[l] + 1u;
    const uint32_t base =
        (uint32_t)ci[0] + R * ((uint32_t)ci[1] + R * ((uint32_t)ci[2] + R * (uint32_t)ci[3])) + xb;
    const uint32_t sy = R, sz = R * R, st = R * R * R;
#pragma unroll
    for (int q = 0; q < 8; ++q) idx[q] = base + (q & 1) * sy + ((q >> 1) & 1) * sz + ((q >> 2) & 1) * st;
  } else {
    const uint32_t hx = (uint32_t)ci[0] * g.primes[0] + (xb ? g.primes[0] : 0u);
    const uint32_t hy0 = (uint32_t)ci[1] * g.primes[1], hy1 = hy0 + g.primes[1];
    const uint32_t hz0 = (uint32_t)ci[2] * g.primes[2], hz1 = hz0 + g.primes[2];
    const uint32_t ht0 = (uint32_t)ci[3] * g.primes[3], ht1 = ht0 + g.primes[3];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      idx[q] = (hx ^ (q & 1 ? hy1 : hy0) ^ (q & 2 ? hz1 : hz0) ^ (q & 4 ? ht1 : ht0)) & g.mask;
  }
}

// The hypervoxel of level l around p: lower corners i[4] and fractional
// offsets fr[4] (axis_cell on x, y, z with N_s and t with N_t).
__device__ __forceinline__ void level_cell(const Geom& g, int l, float4 p, int i[4], float fr[4]) {
  const int ns = g.res_s[l], nt = g.res_t[l];
  axis_cell(p.x, ns, i[0], fr[0]);
  axis_cell(p.y, ns, i[1], fr[1]);
  axis_cell(p.z, ns, i[2], fr[2]);
  axis_cell(p.w, nt, i[3], fr[3]);
}

// The indices of the 8 corners of level l around p whose x bit is xb
// and the fractional offsets fr = (fx, fy, fz, ft).
__device__ __forceinline__ void level_index_x(const Geom& g, int l, float4 p, uint32_t xb, uint32_t idx[8],
                                              float fr[4]) {
  int ci[4];
  level_cell(g, l, p, ci, fr);
  cell_index_x(g, l, ci, xb, idx);
}

// Weights of the corners with x bit xb from the fractional offsets, as
// level_corners forms them: w[q] equals its w[xb | 2q] bit for bit.
__device__ __forceinline__ void level_weights_x(const float fr[4], uint32_t xb, float w[8]) {
  const float wx = xb ? fr[0] : 1.0f - fr[0], wy0 = 1.0f - fr[1], wz0 = 1.0f - fr[2], wt0 = 1.0f - fr[3];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float v = wx;
    v *= (q & 1) ? fr[1] : wy0;
    v *= (q & 2) ? fr[2] : wz0;
    v *= (q & 4) ? fr[3] : wt0;
    w[q] = v;
  }
}

// level_index_x and level_weights_x together: the 8 corners with x bit xb
// and their weights (idx[q], w[q] = level_corners' idx[xb | 2q], w[xb | 2q]).
__device__ __forceinline__ void level_corners_x(const Geom& g, int l, float4 p, uint32_t xb, uint32_t idx[8],
                                                float w[8]) {
  float fr[4];
  level_index_x(g, l, p, xb, idx, fr);
  level_weights_x(fr, xb, w);
}

// ------------------------------------------------------ value helpers ----
template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// F consecutive features of one table entry, widened to FP32.
template <typename TT, int F>
__device__ __forceinline__ void load_entry(const TT* __restrict__ p, float v[F]) {
  if constexpr (sizeof(TT) == 2 && F == 2) {
    const __half2 h = __ldg(reinterpret_cast<const __half2*>(p));
    const float2 f = __half22float2(h);
    v[0] = f.x;
    v[1] = f.y;
  } else if constexpr (sizeof(TT) == 4 && F == 2) {
    const float2 f = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = f.x;
    v[1] = f.y;
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = to_f32<TT>(p[f]);
  }
}

// Vector FP32 reductions into global memory (fire-and-forget, no return),
// with an evict-last L2 policy: the gradient buffer is updated from every tile
// and should not be pushed out of L2 by the streaming inputs.
__device__ __forceinline__ void red_add_v2(float* addr, float a, float b) {
  asm volatile(
      "{\n.reg .b64 pol;\ncreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n"
      "red.relaxed.gpu.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, pol;\n}" ::"l"(addr),
      "f"(a), "f"(b)
      : "memory");
}
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile(
      "{\n.reg .b64 pol;\ncreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n"
      "red.relaxed.gpu.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, pol;\n}" ::"l"(addr),
      "f"(a), "f"(b), "f"(c), "f"(d)
      : "memory");
}

// ------------------------------------------- corner-pair merged access ----
// Corners b and b|1 differ only in x.  With pi_x = 1 (and on dense levels)
// their entries are neighbours: c and c+1 along x hash to indices that differ
// in the low bits only, unless c ends in many one-bits.  One aligned 16-byte
// load then serves both corners, which halves the distinct addresses a warp
// presents to L1 for those pairs.  Level offsets are multiples of 8 entries
// and tables are 16-byte aligned, so the aligned group never straddles a level.

// F = 2 entry k of a 16-byte group, widened to FP32.
template <typename TT>
__device__ __forceinline__ float2 entry_in16(const uint4& v, uint32_t k);
template <>
__device__ __forceinline__ float2 entry_in16<__half>(const uint4& v, uint32_t k) {
  const uint32_t lo = (k & 1u) ? v.y : v.x;
  const uint32_t hi = (k & 1u) ? v.w : v.z;
  const uint32_t word = (k & 2u) ? hi : lo;
  return __half22float2(*reinterpret_cast<const __half2*>(&word));
}
template <>
__device__ __forceinline__ float2 entry_in16<float>(const uint4& v, uint32_t k) {
  return (k & 1u) ? make_float2(__uint_as_float(v.z), __uint_as_float(v.w))
                  : make_float2(__uint_as_float(v.x), __uint_as_float(v.y));
}

// acc[0..2) = sum_b w[b] * table[base + idx[b]] for F = 2 over NC corners
// (16 in 4-D, 8 in 3-D) whose x-neighbours come in pairs (same summation
// order as corner by corner).
template <typename TT, int NC = 16>
__device__ __forceinline__ void gather2_pairs(const TT* __restrict__ base, const uint32_t* idx, const float* w,
                                              float acc[2]) {
  constexpr uint32_t kGroup = 16u / (2u * sizeof(TT));  // entries per 16 bytes: 4 (FP16) or 2 (FP32)
  float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
  for (int p = 0; p < NC / 2; ++p) {
    const uint32_t i0 = idx[2 * p], i1 = idx[2 * p + 1];
    const uint32_t g = i0 & ~(kGroup - 1u);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(base + (size_t)g * 2));
    const float2 e0 = entry_in16<TT>(v, i0 & (kGroup - 1u));
    float2 e1;
    if ((i1 & ~(kGroup - 1u)) == g) {
      e1 = entry_in16<TT>(v, i1 & (kGroup - 1u));
    } else {
      float t[2];
      load_entry<TT, 2>(base + (size_t)i1 * 2, t);
      e1 = make_float2(t[0], t[1]);
    }
    a0 = fmaf(w[2 * p], e0.x, a0);
    a1 = fmaf(w[2 * p], e0.y, a1);
    a0 = fmaf(w[2 * p + 1], e1.x, a0);
    a1 = fmaf(w[2 * p + 1], e1.y, a1);
  }
  acc[0] = a0;
  acc[1] = a1;
}

// acc[0..2) for F = 2 exactly as gather2_pairs forms it for this lane's own
// Gaussian (the same products in the same order, so the same value bit for
// bit), with the loads issued by lane pairs: lane xb of the pair loads the
// entries of the corners whose x bit is xb for both Gaussians A (the even
// lane's, at pa) and B (the odd lane's, at pb), so an x-neighbour pair's two
// loads leave in one warp instruction and L1 serves them with one lookup
// when they share a 128-byte line (31 pairs in 32 for FP16 entries); the two
// lanes then swap the halves they loaded for each other.  pm names the
// pair's lanes.  Both lanes must call it with the same level.
template <typename TT>
__device__ __forceinline__ void gather2_level_paired(const Geom& g, int l, float4 pa, float4 pb, uint32_t xb,
                                                     const TT* __restrict__ base, unsigned int pm, float acc[2]) {
  uint32_t ia[8], ib[8];
  float fa[4], fb[4], fr[4];
  level_index_x(g, l, pa, xb, ia, fa);
  level_index_x(g, l, pb, xb, ib, fb);
#pragma unroll
  for (int k = 0; k < 4; ++k) fr[k] = xb ? fb[k] : fa[k];
  float w0[8], w1[8];  // the own Gaussian's weights of its x = 0 and x = 1 corners
  level_weights_x(fr, 0u, w0);
  level_weights_x(fr, 1u, w1);
  float a0 = 0.0f, a1 = 0.0f;
  if constexpr (sizeof(TT) == 2) {
    uint32_t ea[8], eb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ea[q] = __ldg(reinterpret_cast<const unsigned int*>(base + (size_t)ia[q] * 2));
      eb[q] = __ldg(reinterpret_cast<const unsigned int*>(base + (size_t)ib[q] * 2));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t own = xb ? eb[q] : ea[q];
      const uint32_t other = __shfl_xor_sync(pm, xb ? ea[q] : eb[q], 1);
      const uint32_t u0 = xb ? other : own, u1 = xb ? own : other;
      const float2 e0 = __half22float2(*reinterpret_cast<const __half2*>(&u0));
      const float2 e1 = __half22float2(*reinterpret_cast<const __half2*>(&u1));
      a0 = fmaf(w0[q], e0.x, a0);
      a1 = fmaf(w0[q], e0.y, a1);
      a0 = fmaf(w1[q], e1.x, a0);
      a1 = fmaf(w1[q], e1.y, a1);
    }
  } else {
    float2 ea[8], eb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ea[q] = __ldg(reinterpret_cast<const float2*>(base + (size_t)ia[q] * 2));
      eb[q] = __ldg(reinterpret_cast<const float2*>(base + (size_t)ib[q] * 2));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 own = xb ? eb[q] : ea[q];
      const float2 snd = xb ? ea[q] : eb[q];
      const float2 other = make_float2(__shfl_xor_sync(pm, snd.x, 1), __shfl_xor_sync(pm, snd.y, 1));
      const float2 e0 = xb ? other : own, e1 = xb ? own : other;
      a0 = fmaf(w0[q], e0.x, a0);
      a1 = fmaf(w0[q], e0.y, a1);
      a0 = fmaf(w1[q], e1.x, a0);
      a1 = fmaf(w1[q], e1.y, a1);
    }
  }
  acc[0] = a0;
  acc[1] = a1;
}

// F = 2 table-gradient scatter of one level for two Gaussians by a lane
// pair.  Lane xb of the pair (xb = lane & 1) issues, for both Gaussians A
// (the even lane's, at pa, gradient (a0, a1)) and B (the odd lane's, at pb,
// gradient (b0, b1)), the reductions of the corners whose x bit is xb, so an
// x-neighbour pair's two reductions leave in the same warp instruction; the
// L2 then serves them as one operation when they share a 32-byte sector
// (three pairs in four: always when the lower x coordinate is even, half the
// time otherwise), where one lane issuing both costs two whenever they do
// not form one aligned 16-byte group.  va / vb say whether A / B exist.
__device__ __forceinline__ void scatter2_level_paired(const Geom& g, int l, float4 pa, float4 pb, uint32_t xb,
                                                      bool va, bool vb, float* __restrict__ base, float a0,
                                                      float a1, float b0, float b1) {
  uint32_t ia[8], ib[8];
  float wa[8], wb[8];
  level_corners_x(g, l, pa, xb, ia, wa);
  level_corners_x(g, l, pb, xb, ib, wb);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (va) red_add_v2(base + (size_t)ia[c] * 2, wa[c] * a0, wa[c] * a1);
    if (vb) red_add_v2(base + (size_t)ib[c] * 2, wb[c] * b0, wb[c] * b1);
  }
}

// The sum of a value over the lane pair, the x = 0 lane's term first on both
// lanes (so both hold the same bits).
__device__ __forceinline__ float pair_sum(float v, uint32_t xb, unsigned int pm) {
  const float o = __shfl_xor_sync(pm, v, 1);
  return xb ? o + v : v + o;
}

// The lane pair's two points: this lane's p and its partner's, as (A, B) =
// (even lane's, odd lane's).  pm names the pair's lanes.
__device__ __forceinline__ void pair_points(float4 p, uint32_t xb, unsigned int pm, float4& pa, float4& pb) {
  const float4 q = make_float4(__shfl_xor_sync(pm, p.x, 1), __shfl_xor_sync(pm, p.y, 1),
                               __shfl_xor_sync(pm, p.z, 1), __shfl_xor_sync(pm, p.w, 1));
  pa = xb ? q : p;
  pb = xb ? p : q;
}

// One F = 2 table entry as loaded (FP16: the packed pair; FP32: two floats).
template <typename TT>
struct Entry2;
template <>
struct Entry2<__half> {
  uint32_t v;
  __device__ __forceinline__ float2 f() const { return __half22float2(*reinterpret_cast<const __half2*>(&v)); }
  __device__ __forceinline__ static Entry2 load(const __half* p) {
    return Entry2{__ldg(reinterpret_cast<const unsigned int*>(p))};
  }
};
template <>
struct Entry2<float> {
  float2 v;
  __device__ __forceinline__ float2 f() const { return v; }
  __device__ __forceinline__ static Entry2 load(const float* p) {
    return Entry2{__ldg(reinterpret_cast<const float2*>(p))};
  }
};

// ------------------------------------------- input-coordinate gradient ----
// 1 where the raw coordinate lies in [0,1] (the clamp passes the derivative),
// 0 outside and for NaN; one entry per axis x, y, z, t of compact point i.
__device__ __forceinline__ float4 coord_inside(const Pts& p, long long i) {
  const long long j = point_row(p, i);
#ifdef DASH_DEBUG
  if (j < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
#endif
  const float v[4] = {__ldg(p.x + j), __ldg(p.y + j), __ldg(p.z + j),
                      p.t_stride != 0 ? __ldg(p.t + j * p.t_stride) : __ldg(p.t)};
  float m[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) m[a] = (v[a] >= 0.0f && v[a] <= 1.0f) ? 1.0f : 0.0f;
  return make_float4(m[0], m[1], m[2], m[3]);
}

// The four axis derivatives of d . f_l (F = 2, d = (d0, d1)) at the point pp
// of a lane pair's Gaussian -- level_coord_grad's quantity before the N_l
// factor -- with the gathers issued by the lane pair: lane xb loads the
// corners whose x bit is xb, forms s = d . entry and its share of each
// derivative, and the two lanes add their shares (both end with the same
// sums).  Both lanes call it with the same pp, d0, d1.  idx / w receive this
// lane's corners and weights.  Equal to level_coord_grad up to the order of
// the additions.
template <typename TT>
__device__ __forceinline__ float4 coord_level_paired(const Geom& g, int l, float4 pp, uint32_t xb, unsigned int pm,
                                                     const TT* __restrict__ base, float d0, float d1,
                                                     uint32_t idx[8], float w[8]) {
  float fr[4], sv[8];
  level_index_x(g, l, pp, xb, idx, fr);
  level_weights_x(fr, xb, w);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float2 e = Entry2<TT>::load(base + (size_t)idx[q] * 2).f();
    sv[q] = fmaf(d1, e.y, d0 * e.x);
  }
  const float wx = xb ? fr[0] : 1.0f - fr[0];
  float gx = 0.f, gy = 0.f, gz = 0.f, gt = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float wy = (q & 1) ? fr[1] : 1.0f - fr[1];
    const float wz = (q & 2) ? fr[2] : 1.0f - fr[2];
    const float wt = (q & 4) ? fr[3] : 1.0f - fr[3];
    gx = fmaf(sv[q], wy * wz * wt, gx);
    if (!(q & 1)) gy = fmaf(sv[q | 1] - sv[q], wx * wz * wt, gy);
    if (!(q & 2)) gz = fmaf(sv[q | 2] - sv[q], wx * wy * wt, gz);
    if (!(q & 4)) gt = fmaf(sv[q | 4] - sv[q], wx * wy * wz, gt);
  }
  if (!xb) gx = -gx;  // the lower x corners enter the x derivative with a minus sign
  return make_float4(pair_sum(gx, xb, pm), pair_sum(gy, xb, pm), pair_sum(gz, xb, pm), pair_sum(gt, xb, pm));
}

// acc += d(sum_f d[f] * f_l[f]) / d(x, y, z, t) at the clamped point p for
// level l, whose corner indices idx come from level_corners.  With s_b the
// dot product of d and corner b's entry, the derivative of the quadrilinear
// interpolation along axis a is N_a times the sum over the corner pairs that
// differ only in a of (s_upper - s_lower), each weighted by the other three
// axes' weights; the hypervoxel is the one level_corners selected.
template <typename TT, int F>
__device__ __forceinline__ void level_coord_grad(const Geom& g, int l, float4 p, const TT* __restrict__ base,
                                                 const uint32_t idx[16], const float d[F], float4& acc) {
  float s[16];
  if constexpr (F == 2) {
    constexpr uint32_t kGroup = 16u / (2u * sizeof(TT));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t i0 = idx[2 * q], i1 = idx[2 * q + 1];
      const uint32_t grp = i0 & ~(kGroup - 1u);
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(base + (size_t)grp * 2));
      const float2 e0 = entry_in16<TT>(v, i0 & (kGroup - 1u));
      float2 e1;
      if ((i1 & ~(kGroup - 1u)) == grp) {
        e1 = entry_in16<TT>(v, i1 & (kGroup - 1u));
      } else {
        float t[2];
        load_entry<TT, 2>(base + (size_t)i1 * 2, t);
        e1 = make_float2(t[0], t[1]);
      }
      s[2 * q] = fmaf(d[1], e0.y, d[0] * e0.x);
      s[2 * q + 1] = fmaf(d[1], e1.y, d[0] * e1.x);
    }
  } else {
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      float e[F];
      load_entry<TT, F>(base + (size_t)idx[b] * F, e);
      float v = 0.0f;
#pragma unroll
      for (int f = 0; f < F; ++f) v = fmaf(d[f], e[f], v);
      s[b] = v;
    }
  }
  const int ns = g.res_s[l], nt = g.res_t[l];
  int i0;
  float fr[4];
  axis_cell(p.x, ns, i0, fr[0]);
  axis_cell(p.y, ns, i0, fr[1]);
  axis_cell(p.z, ns, i0, fr[2]);
  axis_cell(p.w, nt, i0, fr[3]);
  float gr[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float v = 0.0f;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      if ((b >> a) & 1) continue;  // b is the lower corner of its pair along a
      float w = 1.0f;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e != a) w *= ((b >> e) & 1) ? fr[e] : 1.0f - fr[e];
      v = fmaf(s[b | (1 << a)] - s[b], w, v);
    }
    gr[a] = v;
  }
  acc.x = fmaf(gr[0], (float)ns, acc.x);
  acc.y = fmaf(gr[1], (float)ns, acc.y);
  acc.z = fmaf(gr[2], (float)ns, acc.z);
  acc.w = fmaf(gr[3], (float)nt, acc.w);
}

// grad[base + idx[b]] += w[b] * d for F = 2 FP32 gradients over NC corners
// (16 in 4-D, 8 in 3-D): a 16-byte reduction when a pair's two entries form
// one aligned 16-byte group.
template <int NC = 16>
__device__ __forceinline__ void scatter2_pairs(float* __restrict__ base, const uint32_t* idx, const float* w, float d0,
                                               float d1) {
#pragma unroll
  for (int p = 0; p < NC / 2; ++p) {
    const uint32_t i0 = idx[2 * p], i1 = idx[2 * p + 1];
    const float u0 = w[2 * p] * d0, u1 = w[2 * p] * d1;
    const float v0 = w[2 * p + 1] * d0, v1 = w[2 * p + 1] * d1;
    if ((i0 ^ i1) == 1u) {
      if (i0 < i1) red_add_v4(base + (size_t)i0 * 2, u0, u1, v0, v1);
      else red_add_v4(base + (size_t)i1 * 2, v0, v1, u0, u1);
    } else {
      red_add_v2(base + (size_t)i0 * 2, u0, u1);
      red_add_v2(base + (size_t)i1 * 2, v0, v1);
    }
  }
}

// Replicas of the coarsest dense levels' FP32 gradients (F = 2).  Those
// levels are small and every Gaussian reduces into 16 of their entries, so
// their entries take hundreds of reductions each per call, which the L2
// serialises; CTA b reduces into replica b % k[l] of level l instead, and
// replica_sum adds the replicas into the gradient buffer afterwards.
constexpr int kMaxRepLevels = 4;
struct Replicas {
  float* base;                      // NULL / levels = 0: no replicas
  int levels;                       // levels 0 .. levels-1 are replicated
  int k[kMaxRepLevels];             // replicas of level l
  long long off[kMaxRepLevels];     // floats from base to replica 0 of level l
  long long stride[kMaxRepLevels];  // floats between consecutive replicas of level l
  long long size[kMaxRepLevels];    // entries of level l
  // where CTA blockIdx.x reduces level l's gradients ([entries][2] FP32)
  __device__ __forceinline__ float* level_base(float* grad, const Geom& g, int l) const {
    if (l < levels) return base + off[l] + (long long)(blockIdx.x % (unsigned)k[l]) * stride[l];
    return grad + g.offset[l] * 2;
  }
};

// Host: the replica layout for the leading dense levels of at most 2^17
// entries, k replicas each (none for F != 2 or k < 2), and its size in
// bytes; base unset.
Replicas replica_plan(const dash_layout* layout, int k, size_t* bytes);
// Zeroes the replicas (before the kernels that reduce into them).
int replica_clear(const Replicas& rp, size_t bytes, cudaStream_t st);
// grad[level l] += sum of the k replicas of level l, for every replicated level.
int replica_sum(const Geom& g, const Replicas& rp, float* grad, cudaStream_t st);

namespace fused {
// Device words the persistent kernels set (bit 0) when a bounded wait gives
// up (deform_fwd.cu, deform_bwd.cu, batch.cu); read by dash_device_status.
unsigned int* fwd_flags_ptr();
unsigned int* bwd_flags_ptr();
unsigned int* batch_flags_ptr();
// The same for the wait self-test (selftest.cu, dash_selftest_wait) and the
// tensor-core decomposition backward (decomp.cu).
unsigned int* selftest_flags_ptr();
unsigned int* decomp_flags_ptr();
}  // namespace fused

// Backward of the Eq. 11 smoothness term for F = 2 (smooth.cu): adds its
// table gradient into table_grad (or, for the replicated levels, into the
// replicas) and lambda_r L_r into sm->loss_out.
int launch_smooth2(const Geom& g, const Pts& pts, const void* table, int table_dtype, float* table_grad,
                   const dash_smooth* sm, const float* dfh, long long dfh_ld, const Replicas& rp, cudaStream_t st);

}  // namespace dash
