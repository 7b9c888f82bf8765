// encode.cu -- the multiresolution 4D hash encoder G_4D of Sec. 4.2 on its
// own: forward f_h = G_4D(x) (Eqs. 8-9), its transpose (the table-gradient
// scatter), the corner/weight debug view, and the plain FP32 forms used as
// the comparison baseline.  One thread per point.
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// f_h for point i: per level the weighted sum of the 16 corner entries
// (kPairs: F = 2 corner pairs fetched with one 16-byte load where possible).
template <typename TT, int F, typename OT, bool kPairs>
__global__ void __launch_bounds__(kThreads) encode_fwd_kernel(Geom g, Pts pts, const TT* __restrict__ table,
                                                              OT* __restrict__ out) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if constexpr (kPairs && F == 2) {
    // lane pairs (gather2_level_paired): both lanes of a pair stay while
    // either of their points exists
    if ((i & ~1ll) >= n) return;
    const bool valid = i < n;
    const uint32_t xb = threadIdx.x & 1u;
    const unsigned int pm = 3u << (threadIdx.x & 30u);
    const float4 p = valid ? load_point(pts, i) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pa, pb;
    pair_points(p, xb, pm, pa, pb);
    OT* row = out + i * (long long)(g.L * F);
    for (int l = 0; l < g.L; ++l) {
      float acc[2];
      gather2_level_paired<TT>(g, l, pa, pb, xb, table + g.offset[l] * 2, pm, acc);
      if (valid) {
        row[2 * l] = from_f32<OT>(acc[0]);
        row[2 * l + 1] = from_f32<OT>(acc[1]);
      }
    }
    return;
  }
  if (i >= n) return;
  const float4 p = load_point(pts, i);
  OT* row = out + i * (long long)(g.L * F);
  for (int l = 0; l < g.L; ++l) {
    uint32_t idx[16];
    float w[16];
    level_corners(g, l, p, idx, w);
    const TT* base = table + g.offset[l] * F;
    float acc[F];
    if constexpr (kPairs && F == 2) {
      gather2_pairs<TT>(base, idx, w, acc);
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] = 0.0f;
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        float v[F];
        load_entry<TT, F>(base + (size_t)idx[b] * F, v);
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f] = fmaf(w[b], v[f], acc[f]);
      }
    }
#pragma unroll
    for (int f = 0; f < F; ++f) row[l * F + f] = from_f32<OT>(acc[f]);
  }
}

// Transpose of the encoder with vector FP32 reductions (F = 2: one 8-byte
// red per corner; F = 4, 8: 16-byte reds; F = 1: scalar).
template <int F>
__global__ void __launch_bounds__(kThreads) encode_bwd_kernel(Geom g, Pts pts, const float* __restrict__ dfeat,
                                                              float* __restrict__ grad) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if constexpr (F == 2) {
    // lane pairs (scatter2_level_paired): point A = row i_a, B = row i_a + 1
    const long long ia = i & ~1ll;
    if (ia >= n) return;  // both lanes of the pair
    const bool vb = ia + 1 < n;
    const uint32_t xb = threadIdx.x & 1u;
    const unsigned int pm = 3u << (threadIdx.x & 30u);
    const float4 p = i < n ? load_point(pts, i) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pa, pb;
    pair_points(p, xb, pm, pa, pb);
    const float* da = dfeat + ia * (long long)(g.L * 2);
    const float* db = da + g.L * 2;
    for (int l = 0; l < g.L; ++l) {
      const float a0 = __ldg(da + 2 * l), a1 = __ldg(da + 2 * l + 1);
      const float b0 = vb ? __ldg(db + 2 * l) : 0.f, b1 = vb ? __ldg(db + 2 * l + 1) : 0.f;
      scatter2_level_paired(g, l, pa, pb, xb, true, vb, grad + g.offset[l] * 2, a0, a1, b0, b1);
    }
  } else {
    if (i >= n) return;
    const float4 p = load_point(pts, i);
    const float* drow = dfeat + i * (long long)(g.L * F);
    for (int l = 0; l < g.L; ++l) {
      uint32_t idx[16];
      float w[16];
      level_corners(g, l, p, idx, w);
      float d[F];
#pragma unroll
      for (int f = 0; f < F; ++f) d[f] = __ldg(drow + l * F + f);
      float* base = grad + g.offset[l] * F;
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        float* e = base + (size_t)idx[b] * F;
        if constexpr (F == 1) {
          atomicAdd(e, w[b] * d[0]);
        } else {
#pragma unroll
          for (int f = 0; f < F; f += 4)
            red_add_v4(e + f, w[b] * d[f], w[b] * d[f + 1], w[b] * d[f + 2], w[b] * d[f + 3]);
        }
      }
    }
  }
}

// d(sum dfeat . G_4D(p)) / d(x, y, z, t) of each compact point, through the
// interpolation weights; dcoord SoA [4][n_cap].
template <typename TT, int F>
__global__ void __launch_bounds__(kThreads) coord_grad_kernel(Geom g, Pts pts, const TT* __restrict__ table,
                                                              const float* __restrict__ dfeat,
                                                              float* __restrict__ dcoord) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (F == 2) {
    // lane pairs (coord_level_paired): point A = row i_a, B = row i_a + 1
    const long long i_a = i & ~1ll;
    if (i_a >= n) return;  // both lanes of the pair
    const bool vb = i_a + 1 < n;
    const uint32_t xb = threadIdx.x & 1u;
    const unsigned int pm = 3u << (threadIdx.x & 30u);
    const float4 p = i < n ? load_point(pts, i) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pa, pb;
    pair_points(p, xb, pm, pa, pb);
    for (int l = 0; l < g.L; ++l) {
      const float ns = (float)g.res_s[l], nt = (float)g.res_t[l];
#pragma unroll 1
      for (int G = 0; G < 2; ++G) {
        if (G == 1 && !vb) break;  // the same on both lanes
        const float* drow = dfeat + (i_a + G) * (long long)(g.L * 2) + 2 * l;
        uint32_t idx[8];
        float w[8];
        const float4 gr = coord_level_paired<TT>(g, l, G == 0 ? pa : pb, xb, pm, table + g.offset[l] * 2,
                                                 __ldg(drow), __ldg(drow + 1), idx, w);
        if ((uint32_t)G == xb) {
          acc.x = fmaf(gr.x, ns, acc.x);
          acc.y = fmaf(gr.y, ns, acc.y);
          acc.z = fmaf(gr.z, ns, acc.z);
          acc.w = fmaf(gr.w, nt, acc.w);
        }
      }
    }
    if (i >= n) return;
  } else {
    if (i >= n) return;
    const float4 p = load_point(pts, i);
    const float* drow = dfeat + i * (long long)(g.L * F);
    for (int l = 0; l < g.L; ++l) {
      uint32_t idx[16];
      float w[16];
      level_corners(g, l, p, idx, w);
      float d[F];
#pragma unroll
      for (int f = 0; f < F; ++f) d[f] = __ldg(drow + l * F + f);
      level_coord_grad<TT, F>(g, l, p, table + g.offset[l] * F, idx, d, acc);
    }
  }
  const float4 m = coord_inside(pts, i);
  const long long cap = pts.n;
  __stcs(dcoord + i, acc.x * m.x);
  __stcs(dcoord + cap + i, acc.y * m.y);
  __stcs(dcoord + 2 * cap + i, acc.z * m.z);
  __stcs(dcoord + 3 * cap + i, acc.w * m.w);
}

// Plain form of the transpose: one scalar FP32 atomicAdd per feature.
template <int F>
__global__ void __launch_bounds__(kThreads) plain_bwd_kernel(Geom g, Pts pts, const float* __restrict__ dfeat,
                                                             float* __restrict__ grad) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 p = load_point(pts, i);
  const float* drow = dfeat + i * (long long)(g.L * F);
  for (int l = 0; l < g.L; ++l) {
    uint32_t idx[16];
    float w[16];
    level_corners(g, l, p, idx, w);
    float* base = grad + g.offset[l] * F;
#pragma unroll
    for (int b = 0; b < 16; ++b)
#pragma unroll
      for (int f = 0; f < F; ++f) atomicAdd(base + (size_t)idx[b] * F + f, w[b] * drow[l * F + f]);
  }
}

// FP16-gradient variant of the transpose (F = 2): table_grad holds one
// f16x2 word per entry.  An x-adjacent corner pair whose two entries share an
// aligned 16-byte group goes out as one 16-byte reduction (the group's other
// entries receive +0), otherwise as two 4-byte reductions.
__device__ __forceinline__ uint32_t h2_bits(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void red_h2(__half* addr, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.noftz.f16x2 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void red_h2x4(__half* addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("red.relaxed.gpu.global.add.noftz.v4.f16x2 [%0], {%1, %2, %3, %4};" ::"l"(addr), "r"(a), "r"(b),
               "r"(c), "r"(d)
               : "memory");
}

__global__ void __launch_bounds__(kThreads) encode_bwd_half_kernel(Geom g, Pts pts, const float* __restrict__ dfeat,
                                                                   __half* __restrict__ grad) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 p = load_point(pts, i);
  const float* drow = dfeat + i * (long long)(g.L * 2);
  for (int l = 0; l < g.L; ++l) {
    uint32_t idx[16];
    float w[16];
    level_corners(g, l, p, idx, w);
    const float d0 = __ldg(drow + 2 * l), d1 = __ldg(drow + 2 * l + 1);
    __half* base = grad + g.offset[l] * 2;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t i0 = idx[2 * q], i1 = idx[2 * q + 1];
      const uint32_t u = h2_bits(w[2 * q] * d0, w[2 * q] * d1);
      const uint32_t v = h2_bits(w[2 * q + 1] * d0, w[2 * q + 1] * d1);
      if ((i0 & ~3u) == (i1 & ~3u)) {
        uint32_t word[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 4; ++k) word[k] = ((i0 & 3u) == (uint32_t)k ? u : 0u) | ((i1 & 3u) == (uint32_t)k ? v : 0u);
        red_h2x4(base + (size_t)(i0 & ~3u) * 2, word[0], word[1], word[2], word[3]);
      } else {
        red_h2(base + (size_t)i0 * 2, u);
        red_h2(base + (size_t)i1 * 2, v);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) indices_kernel(Geom g, Pts pts, uint32_t* __restrict__ idx_out,
                                                           float* __restrict__ w_out) {
  const long long n = point_count(pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 p = load_point(pts, i);
  for (int l = 0; l < g.L; ++l) {
    uint32_t idx[16];
    float w[16];
    level_corners(g, l, p, idx, w);
    const long long o = (i * g.L + l) * 16;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      if (idx_out) idx_out[o + b] = idx[b];
      if (w_out) w_out[o + b] = w[b];
    }
  }
}

template <typename TT, typename OT, bool kPairs = true>
int launch_fwd_t(const Geom& g, const Pts& p, const void* table, void* out, cudaStream_t st) {
  const unsigned grid = grid_for(p.n);
  const TT* tb = static_cast<const TT*>(table);
  OT* o = static_cast<OT*>(out);
  switch (g.F) {
    case 1: encode_fwd_kernel<TT, 1, OT, kPairs><<<grid, kThreads, 0, st>>>(g, p, tb, o); break;
    case 2: encode_fwd_kernel<TT, 2, OT, kPairs><<<grid, kThreads, 0, st>>>(g, p, tb, o); break;
    case 4: encode_fwd_kernel<TT, 4, OT, kPairs><<<grid, kThreads, 0, st>>>(g, p, tb, o); break;
    default: encode_fwd_kernel<TT, 8, OT, kPairs><<<grid, kThreads, 0, st>>>(g, p, tb, o); break;
  }
  return launch_status("encode_fwd_kernel");
}

template <typename TT>
int launch_fwd_out(const Geom& g, const Pts& p, const void* table, void* out, int feat_dtype, cudaStream_t st) {
  switch (feat_dtype) {
    case DASH_F32: return launch_fwd_t<TT, float>(g, p, table, out, st);
    case DASH_F16: return launch_fwd_t<TT, __half>(g, p, table, out, st);
    case DASH_BF16: return launch_fwd_t<TT, __nv_bfloat16>(g, p, table, out, st);
    default: return fail(DASH_ERR_UNSUPPORTED, "feat_dtype %d", feat_dtype);
  }
}

int prepare(const dash_layout* layout, const dash_points* pts, Geom* g, Pts* p) {
  if (int s = make_geom(layout, g)) return s;
  return make_pts(pts, p);
}

}  // namespace
}  // namespace dash

extern "C" {

int dash_hash4d_fwd(const dash_layout* layout, const dash_points* pts, const void* table, int table_dtype,
                    void* feat_out, int feat_dtype, void* stream) {
  DASH_NVTX_RANGE("dash_hash4d_fwd");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (p.n == 0) return DASH_OK;
  if (table == nullptr || feat_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "table/feat_out is NULL");
  if ((reinterpret_cast<uintptr_t>(table) & 15u) != 0) return fail(DASH_ERR_INVALID_ARG, "table must be 16-byte aligned");
  switch (table_dtype) {
    case DASH_F32: return launch_fwd_out<float>(g, p, table, feat_out, feat_dtype, as_stream(stream));
    case DASH_F16: return launch_fwd_out<__half>(g, p, table, feat_out, feat_dtype, as_stream(stream));
    default: return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
  }
}

int dash_hash4d_bwd(const dash_layout* layout, const dash_points* pts, const float* dfeat,
                    float* table_grad, void* stream) {
  DASH_NVTX_RANGE("dash_hash4d_bwd");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (p.n == 0) return DASH_OK;
  if (dfeat == nullptr || table_grad == nullptr) return fail(DASH_ERR_INVALID_ARG, "dfeat/table_grad is NULL");
  if ((reinterpret_cast<uintptr_t>(table_grad) & 15u) != 0)
    return fail(DASH_ERR_INVALID_ARG, "table_grad must be 16-byte aligned");
  const unsigned grid = grid_for(p.n);
  cudaStream_t st = as_stream(stream);
  switch (g.F) {
    case 1: encode_bwd_kernel<1><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
    case 2: encode_bwd_kernel<2><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
    case 4: encode_bwd_kernel<4><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
    default: encode_bwd_kernel<8><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
  }
  return launch_status("encode_bwd_kernel");
}

int dash_hash4d_coord_grad(const dash_layout* layout, const dash_points* pts, const void* table, int table_dtype,
                           const float* dfeat, float* dcoord, void* stream) {
  DASH_NVTX_RANGE("dash_hash4d_coord_grad");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (p.n == 0) return DASH_OK;
  if (table == nullptr || dfeat == nullptr || dcoord == nullptr)
    return fail(DASH_ERR_INVALID_ARG, "table/dfeat/dcoord is NULL");
  if ((reinterpret_cast<uintptr_t>(table) & 15u) != 0) return fail(DASH_ERR_INVALID_ARG, "table must be 16-byte aligned");
  const unsigned grid = grid_for(p.n);
  cudaStream_t st = as_stream(stream);
#define DASH_COORD_LAUNCH(TT)                                                                                     \
  switch (g.F) {                                                                                                 \
    case 1: coord_grad_kernel<TT, 1><<<grid, kThreads, 0, st>>>(g, p, static_cast<const TT*>(table), dfeat, dcoord); break; \
    case 2: coord_grad_kernel<TT, 2><<<grid, kThreads, 0, st>>>(g, p, static_cast<const TT*>(table), dfeat, dcoord); break; \
    case 4: coord_grad_kernel<TT, 4><<<grid, kThreads, 0, st>>>(g, p, static_cast<const TT*>(table), dfeat, dcoord); break; \
    default: coord_grad_kernel<TT, 8><<<grid, kThreads, 0, st>>>(g, p, static_cast<const TT*>(table), dfeat, dcoord); break; \
  }
  if (table_dtype == DASH_F32) {
    DASH_COORD_LAUNCH(float)
  } else if (table_dtype == DASH_F16) {
    DASH_COORD_LAUNCH(__half)
  } else {
    return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
  }
#undef DASH_COORD_LAUNCH
  return launch_status("coord_grad_kernel");
}

int dash_hash4d_bwd_half(const dash_layout* layout, const dash_points* pts, const float* dfeat, void* table_grad,
                         void* stream) {
  DASH_NVTX_RANGE("dash_hash4d_bwd_half");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (g.F != 2) return fail(DASH_ERR_UNSUPPORTED, "the FP16-gradient scatter supports F = 2");
  if (p.n == 0) return DASH_OK;
  if (dfeat == nullptr || table_grad == nullptr) return fail(DASH_ERR_INVALID_ARG, "dfeat/table_grad is NULL");
  if ((reinterpret_cast<uintptr_t>(table_grad) & 15u) != 0)
    return fail(DASH_ERR_INVALID_ARG, "table_grad must be 16-byte aligned");
  encode_bwd_half_kernel<<<grid_for(p.n), kThreads, 0, as_stream(stream)>>>(g, p, dfeat,
                                                                            static_cast<__half*>(table_grad));
  return launch_status("encode_bwd_half_kernel");
}

int dash_hash4d_indices(const dash_layout* layout, const dash_points* pts, uint32_t* idx_out, float* w_out,
                        void* stream) {
  DASH_NVTX_RANGE("dash_hash4d_indices");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (p.n == 0) return DASH_OK;
  indices_kernel<<<grid_for(p.n), kThreads, 0, as_stream(stream)>>>(g, p, idx_out, w_out);
  return launch_status("indices_kernel");
}

int dash_plain_hash4d_fwd(const dash_layout* layout, const dash_points* pts, const float* table,
                          float* feat_out, void* stream) {
  DASH_NVTX_RANGE("dash_plain_hash4d_fwd");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (p.n == 0) return DASH_OK;
  if (table == nullptr || feat_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "table/feat_out is NULL");
  return launch_fwd_t<float, float, false>(g, p, table, feat_out, as_stream(stream));
}

int dash_plain_hash4d_bwd(const dash_layout* layout, const dash_points* pts, const float* dfeat,
                          float* table_grad, void* stream) {
  DASH_NVTX_RANGE("dash_plain_hash4d_bwd");
  using namespace dash;
  Geom g;
  Pts p;
  if (int s = prepare(layout, pts, &g, &p)) return s;
  if (p.n == 0) return DASH_OK;
  if (dfeat == nullptr || table_grad == nullptr) return fail(DASH_ERR_INVALID_ARG, "dfeat/table_grad is NULL");
  const unsigned grid = grid_for(p.n);
  cudaStream_t st = as_stream(stream);
  switch (g.F) {
    case 1: plain_bwd_kernel<1><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
    case 2: plain_bwd_kernel<2><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
    case 4: plain_bwd_kernel<4><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
    default: plain_bwd_kernel<8><<<grid, kThreads, 0, st>>>(g, p, dfeat, table_grad); break;
  }
  return launch_status("plain_bwd_kernel");
}

}  // extern "C"
