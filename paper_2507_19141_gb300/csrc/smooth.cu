// smooth.cu -- the backward of the Eq. 11 smoothness term for F = 2 in a
// kernel of its own, next to the fused backward's df_h scatter:
//   L_r = (1/n) sum_i sum_{e in {e_s, e_t}} |f(p_i) - f(p_i + e)|^2,
// f = G_4D the multiresolution encoding (Eqs. 8-9), p + e clamped to [0,1].
// d(lambda_r L_r)/d table goes to the corners of p (+ scale (f(p) - f(p+e)))
// and of p + e (- scale (f(p) - f(p+e))), scale = 2 lambda_r / n; the
// perturbed encodings are recomputed here, never stored.
//
// Two lanes share two Gaussians A (the even lane's) and B (the odd lane's);
// lane xb = lane & 1 gathers and scatters the corners whose x bit is xb, so
// the two accesses of an x-neighbour pair leave in one warp instruction
// (one L1 lookup / one L2 reduction when they share a sector).  The lanes
// swap partial sums so both hold each Gaussian's full encodings.  Where p + e
// lies in p's hypervoxel (the same 16 corners) the entries loaded for f(p)
// also give f(p + e), and its gradient joins p's in one reduction per corner;
// where p + e_t lies in the next or previous temporal cell, the 8 corners of
// the face the two hypervoxels share are treated the same way.
// A thread keeps one level of one Gaussian live at a time.  Without the
// fused backward's shared-memory ring the whole L1 serves the gathers.
// Given dL/df_h (SoA [L*2][n], written by the fused backward in place of its
// scatter), p's corners take w * (dL/df_h + the Eq. 11 gradient) in one
// reduction each.
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kThreads = 256;

struct SmoothArgs {
  Geom g;
  Pts pts;
  const void* table;
  float* grad;
  float eps_s[3];
  float eps_t;
  float lambda_r;
  float* loss_out;
  const float* dfh;  // optional SoA [L*2][dfh_ld]
  long long dfh_ld;
  Replicas rep;  // the dense levels' reductions go to replicas
};

__device__ __forceinline__ float4 perturbed(float4 p, float ex, float ey, float ez, float et) {
  return make_float4(clamp01(__fadd_rn(p.x, ex)), clamp01(__fadd_rn(p.y, ey)), clamp01(__fadd_rn(p.z, ez)),
                     clamp01(__fadd_rn(p.w, et)));
}

__device__ __forceinline__ bool same_cell(const int a[4], const int b[4]) {
  return a[0] == b[0] && a[1] == b[1] && a[2] == b[2] && a[3] == b[3];
}

// sum over this lane's 8 corners of w[q] * entry[q]
template <typename TT>
__device__ __forceinline__ float2 half_sum(const float w[8], const Entry2<TT> e[8]) {
  float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float2 v = e[q].f();
    s0 = fmaf(w[q], v.x, s0);
    s1 = fmaf(w[q], v.y, s1);
  }
  return make_float2(s0, s1);
}

template <typename TT>
__global__ void __launch_bounds__(kThreads, 2) smooth_bwd_kernel(const __grid_constant__ SmoothArgs a) {
  const long long n = point_count(a.pts);
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long i_a = i & ~1ll;
  const bool has_a = i_a < n, has_b = i_a + 1 < n;  // the same on both lanes of the pair
  const uint32_t xb = threadIdx.x & 1u;
  const unsigned int pm = 3u << (threadIdx.x & 30u);
  const float4 p = i < n ? load_point(a.pts, i) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 pa, pb;
  pair_points(p, xb, pm, pa, pb);
  const float scale = 2.0f * a.lambda_r / (float)n;
  const TT* table = static_cast<const TT*>(a.table);
  float loss = 0.0f;
  for (int l = 0; has_a && l < a.g.L; ++l) {
    const TT* base = table + a.g.offset[l] * 2;
    float* gbase = a.rep.level_base(a.grad, a.g, l);
    float h0 = 0.0f, h1 = 0.0f;  // this lane's Gaussian's dL/df_h at level l
    if (a.dfh != nullptr && i < n) {
      h0 = __ldg(a.dfh + (2 * l) * a.dfh_ld + i);
      h1 = __ldg(a.dfh + (2 * l + 1) * a.dfh_ld + i);
    }
#pragma unroll 1
    for (int G = 0; G < 2; ++G) {  // one Gaussian of the pair at a time keeps the registers down
      if (G == 1 && !has_b) break;  // the same on both lanes
      const float4 pp = G == 0 ? pa : pb;
      int cp[4], cs[4], ct[4];
      float fp[4], fs[4], ft[4];
      level_cell(a.g, l, pp, cp, fp);
      level_cell(a.g, l, perturbed(pp, a.eps_s[0], a.eps_s[1], a.eps_s[2], 0.0f), cs, fs);
      level_cell(a.g, l, perturbed(pp, 0.0f, 0.0f, 0.0f, a.eps_t), ct, ft);
      const bool ss = same_cell(cs, cp), st = same_cell(ct, cp);
      // p + e_t one temporal cell up (dt = 1) or down (dt = -1): its corners
      // with t bit 0 (q < 4) are p's with t bit 1 (q + 4), or the reverse,
      // in the same lane (the x bit is unchanged)
      const int dt = (!st && ct[0] == cp[0] && ct[1] == cp[1] && ct[2] == cp[2]) ? ct[3] - cp[3] : 0;
      // ---- gather this lane's x half of p, and of p + e where it has its own corners
      float2 sp, sq_s, sq_t;
      {
        uint32_t idx[8];
        float w[8];
        Entry2<TT> e[8];
        cell_index_x(a.g, l, cp, xb, idx);
#pragma unroll
        for (int q = 0; q < 8; ++q) e[q] = Entry2<TT>::load(base + (size_t)idx[q] * 2);
        Entry2<TT> es[8], et[8];
        if (!ss) {
          cell_index_x(a.g, l, cs, xb, idx);
#pragma unroll
          for (int q = 0; q < 8; ++q) es[q] = Entry2<TT>::load(base + (size_t)idx[q] * 2);
        }
        if (!st) {
          cell_index_x(a.g, l, ct, xb, idx);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (dt == 1 && q < 4) et[q] = e[q + 4];
            else if (dt == -1 && q >= 4) et[q] = e[q - 4];
            else et[q] = Entry2<TT>::load(base + (size_t)idx[q] * 2);
          }
        }
        level_weights_x(fp, xb, w);
        sp = half_sum<TT>(w, e);
        level_weights_x(fs, xb, w);
        if (ss) sq_s = half_sum<TT>(w, e);
        else sq_s = half_sum<TT>(w, es);
        level_weights_x(ft, xb, w);
        if (st) sq_t = half_sum<TT>(w, e);
        else sq_t = half_sum<TT>(w, et);
      }
      const float p0 = pair_sum(sp.x, xb, pm), p1 = pair_sum(sp.y, xb, pm);
      const float ds0 = p0 - pair_sum(sq_s.x, xb, pm), ds1 = p1 - pair_sum(sq_s.y, xb, pm);
      const float dt0 = p0 - pair_sum(sq_t.x, xb, pm), dt1 = p1 - pair_sum(sq_t.y, xb, pm);
      if ((uint32_t)G == xb) {  // each Gaussian's loss counted by its own lane
        loss = fmaf(ds0, ds0, loss);
        loss = fmaf(ds1, ds1, loss);
        loss = fmaf(dt0, dt0, loss);
        loss = fmaf(dt1, dt1, loss);
      }
      // Gaussian G's dL/df_h lives on lane xb = G of the pair
      const float hg0 = __shfl_sync(pm, h0, (threadIdx.x & 30u) | (uint32_t)G);
      const float hg1 = __shfl_sync(pm, h1, (threadIdx.x & 30u) | (uint32_t)G);
      const float gp0 = fmaf(scale, dt0, scale * ds0) + hg0, gp1 = fmaf(scale, dt1, scale * ds1) + hg1;
      const float gs0 = -scale * ds0, gs1 = -scale * ds1, gt0 = -scale * dt0, gt1 = -scale * dt1;
      // ---- scatter: p's corners (joined by p + e where it shares them), then p + e's own
      {
        uint32_t idx[8];
        float w[8], v[8];
        cell_index_x(a.g, l, cp, xb, idx);
        level_weights_x(fp, xb, w);
        float c0[8], c1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          c0[q] = w[q] * gp0;
          c1[q] = w[q] * gp1;
        }
        if (ss) {
          level_weights_x(fs, xb, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            c0[q] = fmaf(v[q], gs0, c0[q]);
            c1[q] = fmaf(v[q], gs1, c1[q]);
          }
        }
        if (st) {
          level_weights_x(ft, xb, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            c0[q] = fmaf(v[q], gt0, c0[q]);
            c1[q] = fmaf(v[q], gt1, c1[q]);
          }
        } else if (dt == 1 || dt == -1) {  // the shared face joins p's reductions
          level_weights_x(ft, xb, v);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int qt = dt == 1 ? q : q + 4;  // p + e_t's corner on the shared face
            const int qp = dt == 1 ? q + 4 : q;  // the same corner of p
            c0[qp] = fmaf(v[qt], gt0, c0[qp]);
            c1[qp] = fmaf(v[qt], gt1, c1[qp]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) red_add_v2(gbase + (size_t)idx[q] * 2, c0[q], c1[q]);
        if (!ss) {
          cell_index_x(a.g, l, cs, xb, idx);
          level_weights_x(fs, xb, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) red_add_v2(gbase + (size_t)idx[q] * 2, v[q] * gs0, v[q] * gs1);
        }
        if (!st) {
          cell_index_x(a.g, l, ct, xb, idx);
          level_weights_x(ft, xb, v);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (!((dt == 1 && q < 4) || (dt == -1 && q >= 4)))
              red_add_v2(gbase + (size_t)idx[q] * 2, v[q] * gt0, v[q] * gt1);
        }
      }
    }
  }
  if (a.loss_out != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((threadIdx.x & 31u) == 0u && loss != 0.0f) atomicAdd(a.loss_out, a.lambda_r * loss / (float)n);
  }
}

}  // namespace

int launch_smooth2(const Geom& g, const Pts& pts, const void* table, int table_dtype, float* table_grad,
                   const dash_smooth* sm, const float* dfh, long long dfh_ld, const Replicas& rp,
                   cudaStream_t st) {
  SmoothArgs a;
  a.g = g;
  a.pts = pts;
  a.table = table;
  a.grad = table_grad;
  for (int k = 0; k < 3; ++k) a.eps_s[k] = sm->eps_s[k];
  a.eps_t = sm->eps_t;
  a.lambda_r = sm->lambda_r;
  a.loss_out = sm->loss_out;
  a.dfh = dfh;
  a.dfh_ld = dfh_ld;
  a.rep = rp;
  const unsigned grid = (unsigned)((pts.n + kThreads - 1) / kThreads);
  // two CTAs per SM (128 registers a thread): capping the registers lower to
  // fit more CTAs spills and was measured slower
  if (table_dtype == DASH_F16) smooth_bwd_kernel<__half><<<grid, kThreads, 0, st>>>(a);
  else smooth_bwd_kernel<float><<<grid, kThreads, 0, st>>>(a);
  return launch_status("smooth_bwd_kernel");
}

}  // namespace dash
