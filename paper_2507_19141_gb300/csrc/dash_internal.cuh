// dash_internal.cuh -- device-side building blocks shared by the libdash
// kernels: level geometry, point loads, the Eq. 8 corner hash and the Eq. 9
// quadrilinear weights, plus host-side error plumbing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dash.h"

namespace dash {

// ------------------------------------------------------------------ host --
void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
// Records a CUDA failure (launch or runtime call) and returns DASH_ERR_CUDA.
int cuda_status(cudaError_t e, const char* what);
// Checks the last launch on this thread.
int launch_status(const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Number of SMs of the current device (cached per device).
int sm_count();

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
};

int make_pts(const dash_points* p, Pts* out);

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

__device__ __forceinline__ long long point_row(const Pts& p, long long i) {
  return p.idx != nullptr ? (long long)__ldg(p.idx + i) : i;
}

// Clamped (x, y, z, t) of compact point i.
__device__ __forceinline__ float4 load_point(const Pts& p, long long i) {
  const long long j = point_row(p, i);
  float4 r;
  r.x = clamp01(__ldg(p.x + j));
  r.y = clamp01(__ldg(p.y + j));
  r.z = clamp01(__ldg(p.z + j));
  r.w = clamp01(p.t_stride != 0 ? __ldg(p.t + j * p.t_stride) : __ldg(p.t));
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

// Vector FP32 reductions into global memory (fire-and-forget, no return).
__device__ __forceinline__ void red_add_v2(float* addr, float a, float b) {
  asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b)
               : "memory");
}
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a),
               "f"(b), "f"(c), "f"(d)
               : "memory");
}

}  // namespace dash
