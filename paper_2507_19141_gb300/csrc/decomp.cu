// decomp.cu -- the self-supervised static/dynamic decomposition that
// produces the mask the deformation path consumes (Sec. 4.1, Eqs. 3-4):
//   f_3D = phi_p(G_3D(p)), dp = phi_l(f_3D), |dp|;  tau = top-k % of |dp|;
//   mask = |dp| > tau.
// G_3D is the 3-D multiresolution hash encoder of the Gaussian positions
// (8 corners per level, trilinear weights); phi_p is one ReLU layer D -> 64,
// phi_l one linear layer 64 -> 3.  The decoder is tiny (2.2 kflop per
// Gaussian) and runs on the CUDA cores straight from the gather registers.
// tau is found exactly by a radix select over the norms' bit patterns.
#include <math.h>

#include "deform_bwd_common.cuh"

namespace dash {
namespace {

constexpr int kThreads = 256;
constexpr int kHidden3 = 64;

// The 8 corners of level l around p (x, y, z) and their trilinear weights.
__device__ __forceinline__ void level_corners3(const Geom& g, int l, float3 p, uint32_t idx[8], float w[8]) {
  const int ns = g.res_s[l];
  int ix, iy, iz;
  float fx, fy, fz;
  axis_cell(p.x, ns, ix, fx);
  axis_cell(p.y, ns, iy, fy);
  axis_cell(p.z, ns, iz, fz);
  if ((g.dense_bits >> l) & 1u) {
    const uint32_t R = (uint32_t)ns + 1u;
    const uint32_t base = (uint32_t)ix + R * ((uint32_t)iy + R * (uint32_t)iz);
#pragma unroll
    for (int b = 0; b < 8; ++b) idx[b] = base + (b & 1) + ((b >> 1) & 1) * R + ((b >> 2) & 1) * R * R;
  } else {
    const uint32_t hx0 = (uint32_t)ix * g.primes[0], hx1 = hx0 + g.primes[0];
    const uint32_t hy0 = (uint32_t)iy * g.primes[1], hy1 = hy0 + g.primes[1];
    const uint32_t hz0 = (uint32_t)iz * g.primes[2], hz1 = hz0 + g.primes[2];
#pragma unroll
    for (int b = 0; b < 8; ++b) idx[b] = ((b & 1 ? hx1 : hx0) ^ (b & 2 ? hy1 : hy0) ^ (b & 4 ? hz1 : hz0)) & g.mask;
  }
  const float wx0 = 1.0f - fx, wy0 = 1.0f - fy, wz0 = 1.0f - fz;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    float v = (b & 1) ? fx : wx0;
    v *= (b & 2) ? fy : wy0;
    v *= (b & 4) ? fz : wz0;
    w[b] = v;
  }
}

// The indices of the 4 corners with x bit xb (corner b = xb | 2q, q over
// the y, z bits) of level l around p, and the fractional offsets, with the
// arithmetic of level_corners3.
__device__ __forceinline__ void level_index3_x(const Geom& g, int l, float3 p, uint32_t xb, uint32_t idx[4],
                                               float fr[3]) {
  const int ns = g.res_s[l];
  int ix, iy, iz;
  axis_cell(p.x, ns, ix, fr[0]);
  axis_cell(p.y, ns, iy, fr[1]);
  axis_cell(p.z, ns, iz, fr[2]);
  if ((g.dense_bits >> l) & 1u) {
    const uint32_t R = (uint32_t)ns + 1u;
    const uint32_t base = (uint32_t)ix + R * ((uint32_t)iy + R * (uint32_t)iz) + xb;
#pragma unroll
    for (int q = 0; q < 4; ++q) idx[q] = base + (q & 1) * R + ((q >> 1) & 1) * R * R;
  } else {
    const uint32_t hx = (uint32_t)ix * g.primes[0] + (xb ? g.primes[0] : 0u);
    const uint32_t hy0 = (uint32_t)iy * g.primes[1], hy1 = hy0 + g.primes[1];
    const uint32_t hz0 = (uint32_t)iz * g.primes[2], hz1 = hz0 + g.primes[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) idx[q] = (hx ^ (q & 1 ? hy1 : hy0) ^ (q & 2 ? hz1 : hz0)) & g.mask;
  }
}

// Weights of the corners with x bit xb, as level_corners3 forms them.
__device__ __forceinline__ void level_weights3_x(const float fr[3], uint32_t xb, float w[4]) {
  const float wx = xb ? fr[0] : 1.0f - fr[0], wy0 = 1.0f - fr[1], wz0 = 1.0f - fr[2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float v = wx;
    v *= (q & 1) ? fr[1] : wy0;
    v *= (q & 2) ? fr[2] : wz0;
    w[q] = v;
  }
}

// G_3D level l (F = 2) of this lane's own Gaussian, the value gather2_pairs
// forms bit for bit, with the loads issued by the lane pair: lane xb loads
// the corners with x bit xb of both Gaussians A (pa) and B (pb), and the
// lanes swap the halves they loaded for each other (as gather2_level_paired
// does in 4-D).
template <typename TT>
__device__ __forceinline__ void gather2_level3_paired(const Geom& g, int l, float3 pa, float3 pb, uint32_t xb,
                                                      const TT* __restrict__ base, unsigned int pm, float acc[2]) {
  uint32_t ia[4], ib[4];
  float fa[3], fb[3], fr[3];
  level_index3_x(g, l, pa, xb, ia, fa);
  level_index3_x(g, l, pb, xb, ib, fb);
#pragma unroll
  for (int k = 0; k < 3; ++k) fr[k] = xb ? fb[k] : fa[k];
  float w0[4], w1[4];
  level_weights3_x(fr, 0u, w0);
  level_weights3_x(fr, 1u, w1);
  Entry2<TT> ea[4], eb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ea[q] = Entry2<TT>::load(base + (size_t)ia[q] * 2);
    eb[q] = Entry2<TT>::load(base + (size_t)ib[q] * 2);
  }
  float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 own = (xb ? eb[q] : ea[q]).f();
    const float2 snd = (xb ? ea[q] : eb[q]).f();
    const float2 other = make_float2(__shfl_xor_sync(pm, snd.x, 1), __shfl_xor_sync(pm, snd.y, 1));
    const float2 e0 = xb ? other : own, e1 = xb ? own : other;
    a0 = fmaf(w0[q], e0.x, a0);
    a1 = fmaf(w0[q], e0.y, a1);
    a0 = fmaf(w1[q], e1.x, a0);
    a1 = fmaf(w1[q], e1.y, a1);
  }
  acc[0] = a0;
  acc[1] = a1;
}

template <typename TT, int F>
__global__ void __launch_bounds__(kThreads) decomp_fwd_kernel(Geom g, const float* __restrict__ xs,
                                                              const float* __restrict__ ys,
                                                              const float* __restrict__ zs, long long n,
                                                              const TT* __restrict__ table,
                                                              const float* __restrict__ params, int D,
                                                              float* __restrict__ dp_out, float* __restrict__ norm_out,
                                                              const float* __restrict__ ts, long long t_stride,
                                                              float* __restrict__ pt_out) {
  // shared: W1 transposed [D][64] (one input column's 64 weights contiguous),
  // then b1 [64], W2 [3][64], b2 [3] as packed
  extern __shared__ __align__(16) float w_s[];
  const int P = kHidden3 * D + kHidden3 + 3 * kHidden3 + 3;
  for (int e = threadIdx.x; e < P; e += kThreads) {
    const int dst = e < kHidden3 * D ? (e % D) * kHidden3 + e / D : e;
    w_s[dst] = __ldg(params + e);
  }
  __syncthreads();
  const float* W1t = w_s;
  const float* b1 = W1t + kHidden3 * D;
  const float* W2 = b1 + kHidden3;
  const float* b2 = W2 + 3 * kHidden3;
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float3 praw = make_float3(__ldcs(xs + i), __ldcs(ys + i), __ldcs(zs + i));
  const float3 p = make_float3(clamp01(praw.x), clamp01(praw.y), clamp01(praw.z));
  float h[kHidden3];
#pragma unroll
  for (int j = 0; j < kHidden3; ++j) h[j] = b1[j];
  // the gathers here are one Gaussian per lane: with lane pairs (as in the
  // backward) this ALU-heavy kernel measured slower
  for (int l = 0; l < g.L; ++l) {
    uint32_t idx[8];
    float w[8];
    level_corners3(g, l, p, idx, w);
    const TT* base = table + g.offset[l] * F;
    float f[F];
    if constexpr (F == 2) {
      gather2_pairs<TT, 8>(base, idx, w, f);  // x-neighbours share a 16-byte group when aligned
    } else {
#pragma unroll
      for (int k = 0; k < F; ++k) f[k] = 0.0f;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float e[F];
        load_entry<TT, F>(base + (size_t)idx[b] * F, e);
#pragma unroll
        for (int k = 0; k < F; ++k) f[k] = fmaf(w[b], e[k], f[k]);
      }
    }
    // phi_p: stream this level's features into the hidden pre-activations
#pragma unroll
    for (int k = 0; k < F; ++k) {
      const float4* wc = reinterpret_cast<const float4*>(W1t + (l * F + k) * kHidden3);
#pragma unroll
      for (int j4 = 0; j4 < kHidden3 / 4; ++j4) {
        const float4 wv = wc[j4];
        h[4 * j4 + 0] = fmaf(wv.x, f[k], h[4 * j4 + 0]);
        h[4 * j4 + 1] = fmaf(wv.y, f[k], h[4 * j4 + 1]);
        h[4 * j4 + 2] = fmaf(wv.z, f[k], h[4 * j4 + 2]);
        h[4 * j4 + 3] = fmaf(wv.w, f[k], h[4 * j4 + 3]);
      }
    }
  }
  float s = 0.0f;
  float dp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float a = b2[c];
#pragma unroll
    for (int j = 0; j < kHidden3; ++j) a = fmaf(W2[c * kHidden3 + j], fmaxf(h[j], 0.0f), a);
    if (dp_out != nullptr) __stcs(dp_out + (long long)c * n + i, a);
    dp[c] = a;
    s = fmaf(a, a, s);
  }
  __stcs(norm_out + i, sqrtf(s));
  if (pt_out != nullptr) {  // Eq. 4: p(t) = p + t dp, p as given
    const float t = __ldg(ts + i * t_stride);
    __stcs(pt_out + i, fmaf(t, dp[0], praw.x));
    __stcs(pt_out + n + i, fmaf(t, dp[1], praw.y));
    __stcs(pt_out + 2 * n + i, fmaf(t, dp[2], praw.z));
  }
}

// ---------------------------------------------------------- backward ------
// Gradients of  sum_i d_dp_i . dp_i + lambda_s L_s  (Eq. 5 over the static
// Gaussians of `mask`) w.r.t. the G_3D tables and the packed W1, b1, W2, b2.
// Persistent CTAs over tiles of kBwdRows Gaussians, two threads per
// Gaussian (lanes 2r and 2r + 1 of the CTA take tile row r): thread half hb
// gathers and scatters the corners whose x bit is hb (so an x-neighbour
// pair's two accesses leave in one warp instruction) and owns half of the
// hidden units of phi_p (groups of four, interleaved between the two); the two halves add their shares of the
// encoding, of phi_l and of dL/df with one shuffle each.  Per tile the CTA
// leaves f, relu(h), dz1 and the dp gradient in shared memory and contracts
// the weight gradients over the tile's Gaussians into per-thread register
// accumulators, flushed with one atomic per weight and CTA at the end.
// Splitting each Gaussian over two threads halves the per-thread registers,
// which doubles the warps an SM holds for this latency-bound work.
constexpr int kBwdRows = 128;
constexpr int kBwdThreads = 2 * kBwdRows;
constexpr int kHalfHidden = kHidden3 / 2;

struct DecompBwdArgs {
  Geom g;
  const float* x;
  const float* y;
  const float* z;
  long long n;
  const void* table;
  const float* params;
  int D;
  const float* d_dp;
  const uint8_t* mask;
  float lambda_s;
  const unsigned long long* n_static;
  float* table_grad;
  float* mlp_grad;
};

__global__ void __launch_bounds__(kThreads) count_static_kernel(const uint8_t* __restrict__ mask, long long n,
                                                                unsigned long long* out) {
  unsigned int c = 0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    c += mask[i] == 0 ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c != 0u) atomicAdd(out, (unsigned long long)c);
}

// The sum over a thread pair, the hb = 0 thread's term first on both.
__device__ __forceinline__ float half_pair_sum(float v, uint32_t hb, unsigned int pm) {
  const float o = __shfl_xor_sync(pm, v, 1);
  return hb ? o + v : v + o;
}

template <typename TT, int F>
__global__ void __launch_bounds__(kBwdThreads, 2) decomp_bwd_kernel(const __grid_constant__ DecompBwdArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int D = a.D, t = threadIdx.x;
  const int r = t >> 1;                       // tile row of this thread pair
  const uint32_t hb = (uint32_t)(t & 1);      // x half of the corners, half of the hidden units
  // this thread's hidden units: j(u) = 8 (u / 4) + 4 hb + u % 4, so the two
  // threads of a pair read neighbouring 16-byte groups of a weight row
  // (different shared-memory banks, one wavefront)
  const int u0 = 4 * (int)hb;
  const unsigned int pm = 3u << (t & 30);
  // weights: W1 transposed [D][64], b1 [64], W2 [3][64], b2 [3]; per tile:
  // f [kBwdRows][D + 4], relu(h) [kBwdRows][65], dz1 [kBwdRows][65], gdp [kBwdRows][4]
  float* W1t = sm;
  float* b1 = W1t + kHidden3 * D;
  float* W2 = b1 + kHidden3;
  float* b2 = W2 + 3 * kHidden3;
  float* s_f = b2 + 4;  // 64 D + 64 + 192 + 4 floats: a multiple of 4 (16-byte aligned rows for D % 4 == 0)
  // padded row strides: a warp's threads write 16 different rows at once,
  // which with strides of 64 or D floats would all fall in one bank
  const int SF = D + 4;            // keeps f rows 16-byte aligned for D % 4 == 0
  constexpr int SH = kHidden3 + 1;
  float* s_h = s_f + kBwdRows * SF;
  float* s_dz = s_h + kBwdRows * SH;
  float* s_g = s_dz + kBwdRows * SH;
  const int P = kHidden3 * D + kHidden3 + 3 * kHidden3 + 3;
  for (int e = t; e < P; e += kBwdThreads) {
    const int dst = e < kHidden3 * D ? (e % D) * kHidden3 + e / D : e;
    W1t[dst] = __ldg(a.params + e);
  }
  const TT* table = static_cast<const TT*>(a.table);
  const float inv_ns = (a.mask != nullptr && *a.n_static > 0ull) ? 1.0f / (float)*a.n_static : 0.0f;
  // this thread's weight-gradient outputs: dW1 row j1 = t / 4, a quarter of its columns;
  // db1[t] (t < 64) or dW2 entry t - 64 (64 <= t < 256); db2[t] (t < 3)
  const int j1 = t >> 2;
  const int kq = (D + 3) / 4, k0 = (t & 3) * kq;
  const int nk = k0 + kq <= D ? kq : (D > k0 ? D - k0 : 0);
  float acc1[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc1[q] = 0.f;
  float acc_x = 0.f, acc_b2 = 0.f;
  __syncthreads();
  const long long ntiles = (a.n + kBwdRows - 1) / kBwdRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kBwdRows + r;
    const bool valid = i < a.n;  // the same for both threads of the pair
    float h[kHalfHidden];
#pragma unroll
    for (int u = 0; u < kHalfHidden; ++u) h[u] = b1[8 * (u >> 2) + u0 + (u & 3)];
    float3 p = make_float3(0.f, 0.f, 0.f);
    if (valid) p = make_float3(clamp01(__ldg(a.x + i)), clamp01(__ldg(a.y + i)), clamp01(__ldg(a.z + i)));
    for (int l = 0; l < a.g.L; ++l) {
      float f[F];
#pragma unroll
      for (int k = 0; k < F; ++k) f[k] = 0.f;
      if (valid) {
        uint32_t idx[4];
        float fr[3], w[4];
        level_index3_x(a.g, l, p, hb, idx, fr);
        level_weights3_x(fr, hb, w);
        const TT* base = table + a.g.offset[l] * F;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float e[F];
          load_entry<TT, F>(base + (size_t)idx[q] * F, e);
#pragma unroll
          for (int k = 0; k < F; ++k) f[k] = fmaf(w[q], e[k], f[k]);
        }
#pragma unroll
        for (int k = 0; k < F; ++k) f[k] = half_pair_sum(f[k], hb, pm);
      }
#pragma unroll
      for (int k = 0; k < F; ++k) {
        const int col = l * F + k;
        if (hb == 0u) s_f[r * SF + col] = f[k];
        const float* wc = W1t + col * kHidden3 + u0;
#pragma unroll
        for (int u4 = 0; u4 < kHalfHidden / 4; ++u4) {
          const float4 wv = *reinterpret_cast<const float4*>(wc + 8 * u4);
          h[4 * u4 + 0] = fmaf(wv.x, f[k], h[4 * u4 + 0]);
          h[4 * u4 + 1] = fmaf(wv.y, f[k], h[4 * u4 + 1]);
          h[4 * u4 + 2] = fmaf(wv.z, f[k], h[4 * u4 + 2]);
          h[4 * u4 + 3] = fmaf(wv.w, f[k], h[4 * u4 + 3]);
        }
      }
    }
    // phi_l (the two halves' shares added), the dp gradient (upstream + Eq. 5), and back through phi_l
    float dp[3], s = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float v = 0.f;
#pragma unroll
      for (int u = 0; u < kHalfHidden; ++u) v = fmaf(W2[c * kHidden3 + 8 * (u >> 2) + u0 + (u & 3)], fmaxf(h[u], 0.f), v);
      v = b2[c] + half_pair_sum(v, hb, pm);
      dp[c] = v;
      s = fmaf(v, v, s);
    }
    const float norm = sqrtf(s);
    float gd[3] = {0.f, 0.f, 0.f};
    if (valid) {
      const bool stat = a.mask != nullptr && a.mask[i] == 0 && norm > 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gd[c] = a.d_dp != nullptr ? __ldg(a.d_dp + (long long)c * a.n + i) : 0.f;
        if (stat) gd[c] = fmaf(a.lambda_s * inv_ns, dp[c] / norm, gd[c]);
      }
    }
    if (hb == 0u) {
#pragma unroll
      for (int c = 0; c < 3; ++c) s_g[r * 4 + c] = gd[c];
    }
    // h -> relu(h) kept for dW2; dz1 = (W2^T gd) * [z1 > 0] kept for dW1, db1
#pragma unroll
    for (int u = 0; u < kHalfHidden; ++u) {
      const int j = 8 * (u >> 2) + u0 + (u & 3);
      const float dh = W2[j] * gd[0] + W2[kHidden3 + j] * gd[1] + W2[2 * kHidden3 + j] * gd[2];
      const float dz = h[u] > 0.f ? dh : 0.f;
      s_h[r * SH + j] = fmaxf(h[u], 0.f);
      s_dz[r * SH + j] = dz;
      h[u] = dz;  // h now holds this thread's half of dz1
    }
    // dL/df = W1^T dz1 (the halves' shares added), scattered into the tables level by level
    if (valid) {
      for (int l = 0; l < a.g.L; ++l) {
        float df[F];
#pragma unroll
        for (int k = 0; k < F; ++k) {
          const float* wc = W1t + (l * F + k) * kHidden3 + u0;
          float v = 0.f;
#pragma unroll
          for (int u4 = 0; u4 < kHalfHidden / 4; ++u4) {
            const float4 wv = *reinterpret_cast<const float4*>(wc + 8 * u4);
            v = fmaf(wv.x, h[4 * u4], v);
            v = fmaf(wv.y, h[4 * u4 + 1], v);
            v = fmaf(wv.z, h[4 * u4 + 2], v);
            v = fmaf(wv.w, h[4 * u4 + 3], v);
          }
          df[k] = half_pair_sum(v, hb, pm);
        }
        uint32_t idx[4];
        float fr[3], w[4];
        level_index3_x(a.g, l, p, hb, idx, fr);
        level_weights3_x(fr, hb, w);
        float* gbase = a.table_grad + a.g.offset[l] * F;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float* e = gbase + (size_t)idx[q] * F;
          if constexpr (F == 1) {
            atomicAdd(e, w[q] * df[0]);
          } else if constexpr (F == 2) {
            red_add_v2(e, w[q] * df[0], w[q] * df[1]);
          } else {
#pragma unroll
            for (int k = 0; k < F; k += 4)
              red_add_v4(e + k, w[q] * df[k], w[q] * df[k + 1], w[q] * df[k + 2], w[q] * df[k + 3]);
          }
        }
      }
    }
    __syncthreads();
    // weight gradients of this tile (rows of invalid Gaussians are zero)
    const bool vec4 = (kq & 3) == 0 && (D & 3) == 0;  // this thread's columns start on 16-byte boundaries
    for (int g_ = 0; g_ < kBwdRows; ++g_) {
      const float dz = s_dz[g_ * SH + j1];
      const float* fr = s_f + g_ * SF + k0;
      if (vec4) {
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          if (4 * q4 < nk) {
            const float4 fv = *reinterpret_cast<const float4*>(fr + 4 * q4);
            acc1[4 * q4 + 0] = fmaf(dz, fv.x, acc1[4 * q4 + 0]);
            acc1[4 * q4 + 1] = fmaf(dz, fv.y, acc1[4 * q4 + 1]);
            acc1[4 * q4 + 2] = fmaf(dz, fv.z, acc1[4 * q4 + 2]);
            acc1[4 * q4 + 3] = fmaf(dz, fv.w, acc1[4 * q4 + 3]);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (q < nk) acc1[q] = fmaf(dz, fr[q], acc1[q]);
      }
      if (t < kHidden3) {
        acc_x += s_dz[g_ * SH + t];
      } else {
        const int e = t - kHidden3;  // W2 entry e = c * 64 + j
        acc_x = fmaf(s_g[g_ * 4 + e / kHidden3], s_h[g_ * SH + (e % kHidden3)], acc_x);
      }
      if (t < 3) acc_b2 += s_g[g_ * 4 + t];
    }
    __syncthreads();
  }
  // flush: W1 [64][D], b1 [64], W2 [3][64], b2 [3]
  float* gW1 = a.mlp_grad;
  float* gb1 = gW1 + kHidden3 * D;
  float* gW2 = gb1 + kHidden3;
  float* gb2 = gW2 + 3 * kHidden3;
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (q < nk && acc1[q] != 0.f) atomicAdd(gW1 + j1 * D + k0 + q, acc1[q]);
  if (acc_x != 0.f) atomicAdd(t < kHidden3 ? gb1 + t : gW2 + (t - kHidden3), acc_x);
  if (t < 3 && acc_b2 != 0.f) atomicAdd(gb2 + t, acc_b2);
}

// ----------------------------------------------------------- radix select --
// State (device workspace): hist[256] | prefix | prefix_mask | rank | pad.
struct TopkState {
  unsigned int hist[256];
  unsigned int prefix;
  unsigned int prefix_mask;
  unsigned long long rank;  // ascending rank still to locate below the prefix
  double static_sum;        // Eq. 5: sum of the static norms and their number
  unsigned long long static_count;
};

// Positive floats order like their bit patterns; zeros of either sign, NaN and
// negatives all count as +0 (a norm is never negative).
__device__ __forceinline__ unsigned int norm_key(float v) { return v > 0.0f ? __float_as_uint(v) : 0u; }

__global__ void topk_init(TopkState* st, unsigned long long rank) {
  st->hist[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    st->prefix = 0u;
    st->prefix_mask = 0u;
    st->rank = rank;
    st->static_sum = 0.0;
    st->static_count = 0ull;
  }
}

__global__ void __launch_bounds__(kThreads) topk_hist(const float* __restrict__ v, long long n, TopkState* st,
                                                      int shift) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const unsigned int prefix = st->prefix, pmask = st->prefix_mask;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    const unsigned int k = norm_key(__ldg(v + i));
    if ((k & pmask) == prefix) atomicAdd(&h[(k >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x] != 0u) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

// One warp: finds the digit holding the target rank, narrows the prefix and
// clears the histogram for the next pass.
__global__ void topk_select(TopkState* st, int shift) {
  if (threadIdx.x == 0) {
    unsigned long long r = st->rank, cum = 0ull;
    unsigned int d = 255u;
    for (unsigned int b = 0; b < 256u; ++b) {
      const unsigned long long c = st->hist[b];
      if (cum + c > r) {
        d = b;
        break;
      }
      cum += c;
    }
    st->rank = r - cum;
    st->prefix |= d << shift;
    st->prefix_mask |= 0xFFu << shift;
  }
  __syncwarp();
  for (int b = threadIdx.x; b < 256; b += 32) st->hist[b] = 0u;
}

// Writes the mask; with `sums` also accumulates Eq. 5's static sum and count
// (a block reduction, then one FP64 atomic per block).
__global__ void __launch_bounds__(kThreads) topk_apply(const float* __restrict__ v, long long n, TopkState* st,
                                                       int all, uint8_t* __restrict__ mask, float* tau_out,
                                                       int sums) {
  const unsigned int tau = st->prefix;
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i == 0 && tau_out != nullptr) *tau_out = all ? -1.0f : __uint_as_float(tau);
  const unsigned int key = i < n ? norm_key(__ldg(v + i)) : 0u;
  const bool dyn = all || key > tau;
  if (i < n) mask[i] = dyn ? 1u : 0u;
  if (!sums) return;
  const bool stat = i < n && !dyn;
  double x = stat ? (double)__uint_as_float(key) : 0.0;
  unsigned int c = stat ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  __shared__ double xs[kThreads / 32];
  __shared__ unsigned int cs[kThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    xs[warp] = x;
    cs[warp] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bx = 0.0;
    unsigned int bc = 0u;
    for (int w = 0; w < kThreads / 32; ++w) {
      bx += xs[w];
      bc += cs[w];
    }
    if (bc != 0u) {
      atomicAdd(&st->static_sum, bx);
      atomicAdd(&st->static_count, (unsigned long long)bc);
    }
  }
}

__global__ void topk_static_loss(const TopkState* st, float* ls_out) {
  const unsigned long long c = st->static_count;
  *ls_out = c != 0ull ? (float)(st->static_sum / (double)c) : 0.0f;
}

// ------------------------------------------- backward on the tensor cores --
// The same gradients as decomp_bwd_kernel, with phi_p's three contractions
// on tcgen05 (BF16 operands, FP32 accumulators in TMEM), warp-specialised:
// one CTA per SM, warps 0-3 the decoder group (thread r = tile row r = TMEM
// lane r), warps 4.. kWorkers worker groups of 4 warps.  Worker group w
// takes tiles j = w, w + kWorkers, ... and owns ring stage w:
//   worker:  p -> f = G_3D(p) (FP32) -> F tile [f_hi | 1, 0.. | f_lo] of its
//            stage; arrive F-full; wait D-full; dL/df from the stage's
//            transposed [Dp][128] FP32 block -> table gradients
//   decoder: wait F-full; z = [f_hi | 1 | f_lo] [W1_hi | b1_hi | W1_hi]^T +
//            [f_hi | 1] [W1_lo | b1_lo]^T (every product but f_lo W1_lo);
//            h = relu(z), dp = W2 h + b2, |dp|, the dp gradient gd (upstream
//            + Eq. 5), dz = (W2^T gd) * [z > 0] -> dz tile [dz_hi | dz_lo];
//            dL/df = dz_hi W1_hi + dz_lo W1_hi + dz_hi W1_lo and
//            dW1^T += F^T [dz_hi | dz_lo] (accumulated in TMEM over the CTA's
//            tiles; the F tile's ones column gives db1, its lo rows are added
//            at the flush); dW2, db2 summed per warp by shuffles while those
//            MMAs run; dL/df published into the stage; arrive D-full.
// The decoder has finished reading a stage's F tile when it publishes that
// stage's dL/df, and a worker writes its stage again only after scattering,
// so each stage needs just the two barriers.  Requires L F <= 48 (the F
// tile's hi, ones and lo columns within the 128 rows of the transposed read).
namespace dtc {

using fused::kRows;
using fused::split_hi_lo8;
using fused::tile_off;
constexpr int kWorkers = 3;               // worker groups = ring stages
constexpr int kThreadsWs = (kWorkers + 1) * kRows;
constexpr uint32_t kCols = 256;           // TMEM: z 0..63, dL/df 64..111, dW1^T 128..191
constexpr uint32_t kColZ = 0, kColDF = 64, kColW = 128;
constexpr int kMaxDp = 48;

struct Args {
  Geom g;
  const float* x;
  const float* y;
  const float* z;
  long long n;
  const void* table;
  const float* params;
  int D, Dp;
  const float* d_dp;
  const uint8_t* mask;
  float lambda_s;
  const unsigned long long* n_static;
  float* table_grad;
  float* mlp_grad;
  unsigned int* flags;
  uint32_t off_w1lo, off_w2, off_dz, off_stage, stage_bytes, off_df, off_bar;
};

__device__ unsigned int g_decomp_flags;  // bit 0: a bounded wait gave up

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// F = 2 scatter of one 3-D level for a lane pair's two Gaussians: lane xb
// issues the corners with x bit xb of A (pa, gradient (a0, a1)) and of B
// (pb, (b0, b1)), so an x-neighbour pair's two reductions leave in one
// warp instruction.  va / vb: A / B exist.
__device__ __forceinline__ void scatter2_level3_paired(const Geom& g, int l, float3 pa, float3 pb, uint32_t xb,
                                                       bool va, bool vb, float* __restrict__ base, float a0,
                                                       float a1, float b0, float b1) {
  uint32_t ia[4], ib[4];
  float fa[3], fb[3], wa[4], wb[4];
  level_index3_x(g, l, pa, xb, ia, fa);
  level_weights3_x(fa, xb, wa);
  level_index3_x(g, l, pb, xb, ib, fb);
  level_weights3_x(fb, xb, wb);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (va) red_add_v2(base + (size_t)ia[q] * 2, wa[q] * a0, wa[q] * a1);
    if (vb) red_add_v2(base + (size_t)ib[q] * 2, wb[q] * b0, wb[q] * b1);
  }
}

// The sum over the warp of v[0..32) ends with lane k holding the sum of
// every lane's v[k] (a recursive-halving reduce-scatter: 31 shuffles).
__device__ __forceinline__ float warp_reduce_scatter32(float v[32], uint32_t lane) {
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool upper = (lane & (uint32_t)half) != 0u;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      // keep the half that this lane owns, send the other half to the partner
      const float send = upper ? v[k] : v[k + half];
      const float keep = upper ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return v[0];
}

template <typename TT, int F>
__global__ void __launch_bounds__(kThreadsWs, 1) decomp_bwd_ws_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int D = a.D, Dp = a.Dp, KZ = 2 * Dp + 16, KL = Dp + 16;
  constexpr int H = kHidden3;
  uint8_t* w1a = smem;                                      // [64][KZ]: W1_hi | b1_hi, 0.. | W1_hi
  uint8_t* w1lo = smem + a.off_w1lo;                        // [64][KL]: W1_lo | b1_lo, 0..
  float* W2s = reinterpret_cast<float*>(smem + a.off_w2);  // W2 [3][64], b2 [3]
  uint8_t* Dz = smem + a.off_dz;                            // [128][128]: dz_hi | dz_lo
  uint64_t* ffull = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  uint64_t* dfull = ffull + kWorkers;
  uint64_t* mma_bar = dfull + kWorkers;
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(mma_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_bar + 1) + 1;
  auto stage_f = [&](int s) { return smem + a.off_stage + (size_t)s * a.stage_bytes; };
  auto stage_df = [&](int s) { return reinterpret_cast<float*>(smem + a.off_stage + (size_t)s * a.stage_bytes + a.off_df); };

  // weight tiles: W1 [64][D] row-major, b1 [64], W2 [3][64], b2 [3]
  const float* W1 = a.params;
  const float* b1 = W1 + H * D;
  for (int e = tid; e < H * KZ; e += kThreadsWs) {
    const int nn = e / KZ, k = e % KZ;
    float v = 0.0f;
    if (k < D) v = W1[nn * D + k];
    else if (k == Dp) v = b1[nn];
    else if (k >= Dp + 16 && k - Dp - 16 < D) v = W1[nn * D + (k - Dp - 16)];
    *reinterpret_cast<uint16_t*>(w1a + tile_off(nn, k, KZ)) = bf16_bits(v);
  }
  for (int e = tid; e < H * KL; e += kThreadsWs) {
    const int nn = e / KL, k = e % KL;
    float v = 0.0f;
    if (k < D) v = W1[nn * D + k];
    else if (k == Dp) v = b1[nn];
    *reinterpret_cast<uint16_t*>(w1lo + tile_off(nn, k, KL)) = bf16_bits((k < D || k == Dp) ? v - bf16_round(v) : 0.0f);
  }
  for (int e = tid; e < 3 * H + 3; e += kThreadsWs) W2s[e] = b1[H + e];
  if (tid == 0) {
    for (int s = 0; s < kWorkers; ++s) {
      tc::mbar_init(tc::smem_addr(&ffull[s]), kRows);
      tc::mbar_init(tc::smem_addr(&dfull[s]), kRows);
    }
    tc::mbar_init(tc::smem_addr(mma_bar), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), kCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;

  const long long ntiles = (a.n + kRows - 1) / kRows;
  const long long my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int r = tid % kRows;
  const uint32_t lane = (uint32_t)(r & 31);
  float* gW1 = a.mlp_grad;
  float* gb1 = gW1 + H * D;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + 3 * H;

  if (tid < kRows) {
    // ------------------------------------------------------- decoder group
    const uint32_t trow = tbase + ((uint32_t)((r >> 5) * 32) << 16);
    const uint32_t bar = tc::smem_addr(mma_bar);
    uint32_t phase = 0;
    const float inv_ns = (a.mask != nullptr && *a.n_static > 0ull) ? 1.0f / (float)*a.n_static : 0.0f;
    const uint32_t idz = tc::idesc_bf16(kRows, H, 0, 0);
    const uint32_t iddf = tc::idesc_bf16(kRows, Dp, 0, 1);
    const uint32_t idw = tc::idesc_bf16(kRows, H, 1, 1);
    float accw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dW2 outputs 32 q + lane of this warp's rows
    float accb[3] = {0.f, 0.f, 0.f};                 // db2 (lane 0)
    bool had_tile = false;
    for (long long j = 0; j < my_tiles; ++j) {
      const int s = (int)(j % kWorkers);
      const uint32_t round = (uint32_t)(j / kWorkers);
      const long long i = (blockIdx.x + j * gridDim.x) * kRows + r;
      const bool valid = i < a.n;
      bool ok = tc::mbar_wait(tc::smem_addr(&ffull[s]), round & 1u, fused::kWaitIters);
      uint8_t* Ft = stage_f(s);
      if (tc::named_sync_any(1, kRows, !ok || *abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      if (r == 0) {
        fused::bwdk::issue(tbase + kColZ, fused::bwdk::kmajor(Ft, KZ), fused::bwdk::kmajor(w1a, KZ), KZ, idz, false);
        fused::bwdk::issue(tbase + kColZ, fused::bwdk::kmajor(Ft, KZ), fused::bwdk::kmajor(w1lo, KL), KL, idz, true);
        tc::mma_commit(bar);
      }
      ok = tc::mbar_wait(bar, phase, fused::kWaitIters);
      phase ^= 1u;
      if (tc::named_sync_any(1, kRows, !ok)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      // dp = W2 relu(z) + b2 and the ReLU mask, chunk by chunk from TMEM
      float dp[3] = {W2s[3 * H], W2s[3 * H + 1], W2s[3 * H + 2]};
      uint32_t mk[2] = {0u, 0u};
#pragma unroll
      for (int c = 0; c < H / 16; ++c) {
        float zz[16];
        tc::tmem_ld16(trow + kColZ + 16 * c, zz);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int jn = 16 * c + jj;
          if (zz[jj] > 0.0f) mk[c >> 1] |= 1u << ((c & 1) * 16 + jj);
          const float h = fmaxf(zz[jj], 0.0f);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) dp[cc] = fmaf(W2s[cc * H + jn], h, dp[cc]);
        }
      }
      const float norm = sqrtf(fmaf(dp[0], dp[0], fmaf(dp[1], dp[1], dp[2] * dp[2])));
      float gd[3] = {0.f, 0.f, 0.f};
      if (valid) {
        const bool stat = a.mask != nullptr && a.mask[i] == 0 && norm > 0.f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          gd[cc] = a.d_dp != nullptr ? __ldg(a.d_dp + (long long)cc * a.n + i) : 0.f;
          if (stat) gd[cc] = fmaf(a.lambda_s * inv_ns, dp[cc] / norm, gd[cc]);
        }
      }
      // dz = (W2^T gd) * mask -> Dz [dz_hi | dz_lo]
#pragma unroll
      for (int c8 = 0; c8 < H / 8; ++c8) {
        float d8[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int jn = 8 * c8 + jj;
          const float dh = W2s[jn] * gd[0] + W2s[H + jn] * gd[1] + W2s[2 * H + jn] * gd[2];
          d8[jj] = ((mk[jn >> 5] >> (jn & 31)) & 1u) ? dh : 0.0f;
        }
        uint4 hi, lo;
        split_hi_lo8(d8, hi, lo);
        *reinterpret_cast<uint4*>(Dz + tile_off(r, 8 * c8, 2 * H)) = hi;
        *reinterpret_cast<uint4*>(Dz + tile_off(r, H + 8 * c8, 2 * H)) = lo;
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      tc::named_sync(1, kRows);
      tc::fence_after_sync();
      if (r == 0) {
        using fused::bwdk::issue;
        using fused::bwdk::kmajor;
        using fused::bwdk::mnmajor;
        fused::bwdk::Op dzh = kmajor(Dz, 2 * H), dzl = dzh;
        dzl.addr += (uint32_t)tile_off(0, H, 2 * H);
        issue(tbase + kColDF, dzh, mnmajor(w1a, KZ), H, iddf, false);
        issue(tbase + kColDF, dzl, mnmajor(w1a, KZ), H, iddf, true);
        issue(tbase + kColDF, dzh, mnmajor(w1lo, KL), H, iddf, true);
        fused::bwdk::Op bh = mnmajor(Dz, 2 * H), bl = bh;
        bl.addr += (uint32_t)tile_off(0, H, 2 * H);
        issue(tbase + kColW, mnmajor(Ft, KZ), bh, kRows, idw, had_tile);
        issue(tbase + kColW, mnmajor(Ft, KZ), bl, kRows, idw, true);
        tc::mma_commit(bar);
      }
      // dW2 = sum over the rows of gd (x) relu(z), db2 = sum of gd: this
      // warp's 32 rows reduced by shuffles while the MMAs run (z stays in
      // TMEM columns 0..63)
#pragma unroll 1
      for (int q = 0; q < 6; ++q) {
        const int cq = q >> 1, j0 = (q & 1) * 32;
        float v[32];
        float zz[16];
        tc::tmem_ld16(trow + kColZ + j0, zz);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) v[jj] = gd[cq] * fmaxf(zz[jj], 0.0f);
        tc::tmem_ld16(trow + kColZ + j0 + 16, zz);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) v[16 + jj] = gd[cq] * fmaxf(zz[jj], 0.0f);
        accw[q] += warp_reduce_scatter32(v, lane);
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        float t = gd[cc];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        accb[cc] += t;
      }
      ok = tc::mbar_wait(bar, phase, fused::kWaitIters);
      phase ^= 1u;
      if (tc::named_sync_any(1, kRows, !ok)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      had_tile = true;
      // publish dL/df to the stage, transposed [Dp][128]
      float* dst = stage_df(s);
      for (int c = 0; c < Dp / 16; ++c) {
        float t[16];
        tc::tmem_ld16(trow + kColDF + 16 * c, t);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) dst[(16 * c + jj) * kRows + r] = t[jj];
      }
      tc::fence_before_sync();
      tc::mbar_arrive(tc::smem_addr(&dfull[s]));
    }
    // flush: dW1 rows from TMEM lanes (hi rows r < D, lo rows Dp + 16 + k,
    // the ones row Dp = db1), dW2 and db2 from the per-warp sums
    tc::named_sync(1, kRows);
    tc::fence_after_sync();
    if (had_tile && *abort_flag == 0) {
      const uint32_t trow2 = trow;
      const int col = r < D ? r : (r >= Dp + 16 && r < Dp + 16 + D ? r - Dp - 16 : -1);
#pragma unroll 1
      for (int c = 0; c < H / 16; ++c) {
        float v[16];
        tc::tmem_ld16(trow2 + kColW + 16 * c, v);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int jn = 16 * c + jj;
          if (col >= 0 && v[jj] != 0.f) atomicAdd(gW1 + jn * D + col, v[jj]);
          else if (r == Dp && v[jj] != 0.f) atomicAdd(gb1 + jn, v[jj]);
        }
      }
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (accw[q] != 0.f) atomicAdd(gW2 + 32 * q + (int)lane, accw[q]);
      if (lane == 0)
        for (int cc = 0; cc < 3; ++cc)
          if (accb[cc] != 0.f) atomicAdd(gb2 + cc, accb[cc]);
    }
  } else {
    // -------------------------------------------------------- worker groups
    const int w = tid / kRows - 1;
    const uint32_t xb = lane & 1u;
    const unsigned int pm = 3u << (lane & 30u);
    const TT* table = static_cast<const TT*>(a.table);
    uint8_t* Ft = stage_f(w);
    const float* dfs = stage_df(w);
    for (long long j = w; j < my_tiles; j += kWorkers) {
      const uint32_t round = (uint32_t)(j / kWorkers);
      const long long i = (blockIdx.x + j * gridDim.x) * kRows + r;
      const bool valid = i < a.n;
      float3 p = make_float3(0.f, 0.f, 0.f);
      if (valid) p = make_float3(clamp01(__ldg(a.x + i)), clamp01(__ldg(a.y + i)), clamp01(__ldg(a.z + i)));
      float3 pa = p, pb = p;
      bool live = valid;
      if constexpr (F == 2) {
        const float3 q = make_float3(__shfl_xor_sync(pm, p.x, 1), __shfl_xor_sync(pm, p.y, 1),
                                     __shfl_xor_sync(pm, p.z, 1));
        pa = xb ? q : p;
        pb = xb ? p : q;
        live = __shfl_xor_sync(pm, valid ? 1 : 0, 1) != 0 || valid;
      }
      // f = G_3D(p) into the stage's F tile, 8 features at a time
      constexpr int kLevelsPerChunk = 8 / F;
      for (int c = 0; c < Dp / 8; ++c) {
        float v[8];
#pragma unroll
        for (int jl = 0; jl < kLevelsPerChunk; ++jl) {
          const int l = c * kLevelsPerChunk + jl;
          float acc[F];
#pragma unroll
          for (int f = 0; f < F; ++f) acc[f] = 0.0f;
          if constexpr (F == 2) {
            if (live && l < a.g.L) {
              gather2_level3_paired<TT>(a.g, l, pa, pb, xb, table + a.g.offset[l] * 2, pm, acc);
              if (!valid) acc[0] = acc[1] = 0.0f;
            }
          } else {
            if (valid && l < a.g.L) {
              uint32_t idx[8];
              float wt[8];
              level_corners3(a.g, l, p, idx, wt);
              const TT* base = table + a.g.offset[l] * F;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                float e[F];
                load_entry<TT, F>(base + (size_t)idx[q] * F, e);
#pragma unroll
                for (int f = 0; f < F; ++f) acc[f] = fmaf(wt[q], e[f], acc[f]);
              }
            }
          }
#pragma unroll
          for (int f = 0; f < F; ++f) v[jl * F + f] = acc[f];
        }
        uint4 hi, lo;
        split_hi_lo8(v, hi, lo);
        *reinterpret_cast<uint4*>(Ft + tile_off(r, 8 * c, KZ)) = hi;
        *reinterpret_cast<uint4*>(Ft + tile_off(r, Dp + 16 + 8 * c, KZ)) = lo;
      }
      fused::write_ones(Ft, r, Dp, KZ);
      tc::fence_async_smem();
      tc::mbar_arrive(tc::smem_addr(&ffull[w]));
      if (!tc::mbar_wait(tc::smem_addr(&dfull[w]), round & 1u, fused::kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      // dL/df of this tile into the tables
      if constexpr (F == 2) {
        const long long ia0 = i - (r & 1);  // the pair's even row; both lanes agree on ia0 < n
        if (ia0 < a.n) {
          for (int l = 0; l < a.g.L; ++l) {
            const float2 f0 = *reinterpret_cast<const float2*>(dfs + (2 * l) * kRows + (r & ~1));      // (A, B)
            const float2 f1 = *reinterpret_cast<const float2*>(dfs + (2 * l + 1) * kRows + (r & ~1));  // (A, B)
            scatter2_level3_paired(a.g, l, pa, pb, xb, true, ia0 + 1 < a.n, a.table_grad + a.g.offset[l] * 2,
                                   f0.x, f1.x, f0.y, f1.y);
          }
        }
      } else {
        if (valid) {
          for (int l = 0; l < a.g.L; ++l) {
            float d[F];
#pragma unroll
            for (int f = 0; f < F; ++f) d[f] = dfs[(l * F + f) * kRows + r];
            uint32_t idx[8];
            float wt[8];
            level_corners3(a.g, l, p, idx, wt);
            float* gbase = a.table_grad + a.g.offset[l] * F;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              float* e = gbase + (size_t)idx[q] * F;
              if constexpr (F == 1) {
                atomicAdd(e, wt[q] * d[0]);
              } else {
#pragma unroll
                for (int f = 0; f < F; f += 4)
                  red_add_v4(e + f, wt[q] * d[f], wt[q] * d[f + 1], wt[q] * d[f + 2], wt[q] * d[f + 3]);
              }
            }
          }
        }
      }
    }
  }
  if (*abort_flag) atomicOr(a.flags, 1u);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, kCols);
}

}  // namespace dtc

// ---------------------------------------------- forward on the tensor cores --
// phi_p of the decomposition forward on tcgen05, warp-specialised like the
// backward: worker groups gather G_3D into F tiles, one decoder group (TMEM
// lanes) forms z = W1 f + b1 and the outputs.  To keep Delta p at FP32
// accuracy each operand is split into three BF16 parts (a = a1 + a2 + a3,
// exact for FP32) and the products of total order at most 2 are kept:
//   chain 1  [f1 | 1 1 1 | f2 | f3] x [W1 | b1 b2 b3 | W1 | W1]
//   chain 2  [f1 | 1 0 0 | f2]      x [W2 | 0 0 0    | W2]
//   chain 3  [f1]                   x [W3]
// (f2 W3, f3 W2, f3 W3 dropped: relative 2^-24).  Then on the CUDA cores:
// h = relu(z), Delta p = W2 h + b2, |Delta p| and Eq. 4's p(t).  Worker w
// owns stage w; the decoder releases a stage with tcgen05.commit once the
// z MMA has read it.
namespace dfw {

using fused::kRows;
using fused::tile_off;
constexpr int kWorkers = 4;
constexpr int kThreadsWs = (kWorkers + 1) * kRows;
constexpr uint32_t kCols = 64;  // z

struct Args {
  Geom g;
  const float* x;
  const float* y;
  const float* z;
  long long n;
  const void* table;
  const float* params;
  int D, Dp;
  float* dp_out;
  float* norm_out;
  const float* ts;
  long long t_stride;
  float* pt_out;
  unsigned int* flags;
  uint32_t off_wb, off_wc, off_w2, off_stage, stage_bytes, off_bar;
};

// v = v1 + v2 + v3 in BF16 (exact for FP32 up to the last bits of v3).
__device__ __forceinline__ void split3(float v, float& a1, float& a2, float& a3) {
  a1 = dtc::bf16_round(v);
  const float r1 = v - a1;
  a2 = dtc::bf16_round(r1);
  a3 = dtc::bf16_round(r1 - a2);
}

__device__ __forceinline__ uint32_t pack2(float a, float b) { return fused::pack_bf16x2(a, b); }

template <typename TT, int F>
__global__ void __launch_bounds__(kThreadsWs, 1) decomp_fwd_ws_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int D = a.D, Dp = a.Dp;
  const int KA = 3 * Dp + 16, KB = 2 * Dp + 16, KC = Dp;
  constexpr int H = kHidden3;
  uint8_t* wa = smem;                                      // [64][KA]
  uint8_t* wb = smem + a.off_wb;                           // [64][KB]
  uint8_t* wc = smem + a.off_wc;                           // [64][KC]
  float* W2s = reinterpret_cast<float*>(smem + a.off_w2);  // W2 [3][64], b2 [3]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  uint64_t* empty = full + kWorkers;
  uint64_t* mma_bar = empty + kWorkers;
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(mma_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_bar + 1) + 1;
  auto stage = [&](int s) { return smem + a.off_stage + (size_t)s * a.stage_bytes; };

  // weight tiles from W1 [64][D], b1 [64]
  const float* W1 = a.params;
  const float* b1 = W1 + H * D;
  for (int e = tid; e < H * KA; e += kThreadsWs) {
    const int nn = e / KA, k = e % KA;
    float v = 0.0f;
    if (k < D) {
      v = W1[nn * D + k];
      float p1, p2, p3;
      split3(v, p1, p2, p3);
      v = p1;
    } else if (k >= Dp && k < Dp + 3) {
      float p[3];
      split3(b1[nn], p[0], p[1], p[2]);
      v = p[k - Dp];
    } else if (k >= Dp + 16 && k < Dp + 16 + D) {
      float p1, p2, p3;
      split3(W1[nn * D + (k - Dp - 16)], p1, p2, p3);
      v = p1;
    } else if (k >= 2 * Dp + 16 && k < 2 * Dp + 16 + D) {
      float p1, p2, p3;
      split3(W1[nn * D + (k - 2 * Dp - 16)], p1, p2, p3);
      v = p1;
    }
    *reinterpret_cast<uint16_t*>(wa + tile_off(nn, k, KA)) = dtc::bf16_bits(v);
  }
  for (int e = tid; e < H * KB; e += kThreadsWs) {
    const int nn = e / KB, k = e % KB;
    float v = 0.0f, p1, p2, p3;
    if (k < D) {
      split3(W1[nn * D + k], p1, p2, p3);
      v = p2;
    } else if (k >= Dp + 16 && k < Dp + 16 + D) {
      split3(W1[nn * D + (k - Dp - 16)], p1, p2, p3);
      v = p2;
    }
    *reinterpret_cast<uint16_t*>(wb + tile_off(nn, k, KB)) = dtc::bf16_bits(v);
  }
  for (int e = tid; e < H * KC; e += kThreadsWs) {
    const int nn = e / KC, k = e % KC;
    float v = 0.0f, p1, p2, p3;
    if (k < D) {
      split3(W1[nn * D + k], p1, p2, p3);
      v = p3;
    }
    *reinterpret_cast<uint16_t*>(wc + tile_off(nn, k, KC)) = dtc::bf16_bits(v);
  }
  for (int e = tid; e < 3 * H + 3; e += kThreadsWs) W2s[e] = b1[H + e];
  if (tid == 0) {
    for (int s = 0; s < kWorkers; ++s) {
      tc::mbar_init(tc::smem_addr(&full[s]), kRows);
      tc::mbar_init(tc::smem_addr(&empty[s]), 1);
    }
    tc::mbar_init(tc::smem_addr(mma_bar), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), kCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;
  const long long ntiles = (a.n + kRows - 1) / kRows;
  const long long my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int r = tid % kRows;
  const uint32_t lane = (uint32_t)(r & 31);

  if (tid < kRows) {
    // ------------------------------------------------------- decoder group
    const uint32_t trow = tbase + ((uint32_t)((r >> 5) * 32) << 16);
    const uint32_t bar = tc::smem_addr(mma_bar);
    uint32_t phase = 0;
    const uint32_t idz = tc::idesc_bf16(kRows, H, 0, 0);
    for (long long j = 0; j < my_tiles; ++j) {
      const int s = (int)(j % kWorkers);
      const uint32_t round = (uint32_t)(j / kWorkers);
      const long long i = (blockIdx.x + j * gridDim.x) * kRows + r;
      bool ok = tc::mbar_wait(tc::smem_addr(&full[s]), round & 1u, fused::kWaitIters);
      if (tc::named_sync_any(1, kRows, !ok || *abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      if (r == 0) {
        uint8_t* Ft = stage(s);
        using fused::bwdk::issue;
        using fused::bwdk::kmajor;
        issue(tbase, kmajor(Ft, KA), kmajor(wa, KA), KA, idz, false);
        issue(tbase, kmajor(Ft, KA), kmajor(wb, KB), KB, idz, true);
        issue(tbase, kmajor(Ft, KA), kmajor(wc, KC), KC, idz, true);
        tc::mma_commit(bar);
        tc::mma_commit(tc::smem_addr(&empty[s]));  // the stage is free once these have read it
      }
      ok = tc::mbar_wait(bar, phase, fused::kWaitIters);
      phase ^= 1u;
      if (tc::named_sync_any(1, kRows, !ok)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      float dp[3] = {W2s[3 * H], W2s[3 * H + 1], W2s[3 * H + 2]};
#pragma unroll
      for (int c = 0; c < H / 16; ++c) {
        float zz[16];
        tc::tmem_ld16(trow + 16 * c, zz);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const float h = fmaxf(zz[jj], 0.0f);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) dp[cc] = fmaf(W2s[cc * H + 16 * c + jj], h, dp[cc]);
        }
      }
      tc::fence_before_sync();
      if (i < a.n) {
        float s2 = 0.0f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          if (a.dp_out != nullptr) __stcs(a.dp_out + (long long)cc * a.n + i, dp[cc]);
          s2 = fmaf(dp[cc], dp[cc], s2);
        }
        __stcs(a.norm_out + i, sqrtf(s2));
        if (a.pt_out != nullptr) {  // Eq. 4: p(t) = p + t dp, p as given
          const float t = __ldg(a.ts + i * a.t_stride);
          __stcs(a.pt_out + i, fmaf(t, dp[0], __ldg(a.x + i)));
          __stcs(a.pt_out + a.n + i, fmaf(t, dp[1], __ldg(a.y + i)));
          __stcs(a.pt_out + 2 * a.n + i, fmaf(t, dp[2], __ldg(a.z + i)));
        }
      }
    }
  } else {
    // -------------------------------------------------------- worker groups
    const int w = tid / kRows - 1;
    const uint32_t xb = lane & 1u;
    const unsigned int pm = 3u << (lane & 30u);
    const TT* table = static_cast<const TT*>(a.table);
    uint8_t* Ft = stage(w);
    for (long long j = w; j < my_tiles; j += kWorkers) {
      const uint32_t round = (uint32_t)(j / kWorkers);
      // the decoder's MMAs of this stage's previous tile have read it
      if (!tc::mbar_wait(tc::smem_addr(&empty[w]), (round & 1u) ^ 1u, fused::kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const long long i = (blockIdx.x + j * gridDim.x) * kRows + r;
      const bool valid = i < a.n;
      float3 p = make_float3(0.f, 0.f, 0.f);
      if (valid) p = make_float3(clamp01(__ldcs(a.x + i)), clamp01(__ldcs(a.y + i)), clamp01(__ldcs(a.z + i)));
      float3 pa = p, pb = p;
      bool live = valid;
      if constexpr (F == 2) {
        const float3 q = make_float3(__shfl_xor_sync(pm, p.x, 1), __shfl_xor_sync(pm, p.y, 1),
                                     __shfl_xor_sync(pm, p.z, 1));
        pa = xb ? q : p;
        pb = xb ? p : q;
        live = __shfl_xor_sync(pm, valid ? 1 : 0, 1) != 0 || valid;
      }
      constexpr int kLevelsPerChunk = 8 / F;
      for (int c = 0; c < Dp / 8; ++c) {
        float v[8];
#pragma unroll
        for (int jl = 0; jl < kLevelsPerChunk; ++jl) {
          const int l = c * kLevelsPerChunk + jl;
          float acc[F];
#pragma unroll
          for (int f = 0; f < F; ++f) acc[f] = 0.0f;
          if constexpr (F == 2) {
            if (live && l < a.g.L) {
              gather2_level3_paired<TT>(a.g, l, pa, pb, xb, table + a.g.offset[l] * 2, pm, acc);
              if (!valid) acc[0] = acc[1] = 0.0f;
            }
          } else {
            if (valid && l < a.g.L) {
              uint32_t idx[8];
              float wt[8];
              level_corners3(a.g, l, p, idx, wt);
              const TT* base = table + a.g.offset[l] * F;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                float e[F];
                load_entry<TT, F>(base + (size_t)idx[q] * F, e);
#pragma unroll
                for (int f = 0; f < F; ++f) acc[f] = fmaf(wt[q], e[f], acc[f]);
              }
            }
          }
#pragma unroll
          for (int f = 0; f < F; ++f) v[jl * F + f] = acc[f];
        }
        float p1[8], p2[8], p3[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split3(v[q], p1[q], p2[q], p3[q]);
        *reinterpret_cast<uint4*>(Ft + tile_off(r, 8 * c, KA)) =
            make_uint4(pack2(p1[0], p1[1]), pack2(p1[2], p1[3]), pack2(p1[4], p1[5]), pack2(p1[6], p1[7]));
        *reinterpret_cast<uint4*>(Ft + tile_off(r, Dp + 16 + 8 * c, KA)) =
            make_uint4(pack2(p2[0], p2[1]), pack2(p2[2], p2[3]), pack2(p2[4], p2[5]), pack2(p2[6], p2[7]));
        *reinterpret_cast<uint4*>(Ft + tile_off(r, 2 * Dp + 16 + 8 * c, KA)) =
            make_uint4(pack2(p3[0], p3[1]), pack2(p3[2], p3[3]), pack2(p3[4], p3[5]), pack2(p3[6], p3[7]));
      }
      // the ones block: 1 at columns Dp, Dp + 1, Dp + 2 (the bias's three parts), 0 to Dp + 15
      *reinterpret_cast<uint4*>(Ft + tile_off(r, Dp, KA)) = make_uint4(0x3F803F80u, 0x3F80u, 0u, 0u);
      *reinterpret_cast<uint4*>(Ft + tile_off(r, Dp + 8, KA)) = make_uint4(0u, 0u, 0u, 0u);
      tc::fence_async_smem();
      tc::mbar_arrive(tc::smem_addr(&full[w]));
    }
  }
  if (*abort_flag) atomicOr(a.flags, 1u);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, kCols);
}

}  // namespace dfw

}  // namespace

namespace fused {
unsigned int* decomp_flags_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, dtc::g_decomp_flags) != cudaSuccess) return nullptr;
  return static_cast<unsigned int*>(p);
}
}  // namespace fused
}  // namespace dash

extern "C" {

int dash_hash3d_layout(const dash_hash4d_cfg* cfg, dash_layout* out) {
  using dash::fail;
  if (cfg == nullptr || out == nullptr) return fail(DASH_ERR_INVALID_ARG, "cfg/out is NULL");
  if (cfg->L < 1 || cfg->L > DASH_MAX_LEVELS) return fail(DASH_ERR_UNSUPPORTED, "L=%d outside [1,32]", cfg->L);
  if (!(cfg->F == 1 || cfg->F == 2 || cfg->F == 4 || cfg->F == 8))
    return fail(DASH_ERR_UNSUPPORTED, "F=%d not in {1,2,4,8}", cfg->F);
  if (cfg->log2_T < 4 || cfg->log2_T > 28) return fail(DASH_ERR_UNSUPPORTED, "log2_T=%d outside [4,28]", cfg->log2_T);
  if (!(cfg->nmin_s >= 1.0) || !(cfg->nmax_s >= cfg->nmin_s) || cfg->nmax_s > 65535.0)
    return fail(DASH_ERR_INVALID_ARG, "resolutions must satisfy 1 <= N_min <= N_max <= 65535");
  memset(out, 0, sizeof(*out));
  out->L = cfg->L;
  out->F = cfg->F;
  out->log2_T = cfg->log2_T;
  out->dims = 3;
  for (int i = 0; i < 3; ++i) out->primes[i] = cfg->primes[i];
  const int64_t T = (int64_t)1 << cfg->log2_T;
  int64_t start = 0;
  for (int l = 0; l < cfg->L; ++l) {
    double ns_d;
    if (cfg->L == 1) {
      ns_d = floor(cfg->nmin_s + 1e-9);
    } else {
      const double growth = exp((log(cfg->nmax_s) - log(cfg->nmin_s)) / (double)(cfg->L - 1));
      ns_d = floor(cfg->nmin_s * pow(growth, (double)l) + 1e-9);
    }
    const int32_t ns = (int32_t)ns_d;
    out->res_s[l] = ns;
    out->res_t[l] = 0;
    const int64_t r = (int64_t)ns + 1;
    const int64_t vertices = r * r * r;
    out->dense[l] = vertices <= T ? 1 : 0;
    out->size[l] = out->dense[l] ? vertices : T;
    out->offset[l] = start;
    start = (start + out->size[l] + 7) & ~(int64_t)7;
  }
  out->offset[cfg->L] = start;
  return DASH_OK;
}

int dash_decomp_fwd(const dash_layout* layout, const float* x, const float* y, const float* z, int64_t n,
                    const void* table, int table_dtype, const dash_mlp* mlp, float* dp_out, float* norm_out,
                    const float* t, int64_t t_stride, float* pt_out, void* stream) {
  DASH_NVTX_RANGE("dash_decomp_fwd");
  using namespace dash;
  if (layout == nullptr || layout->dims != 3) return fail(DASH_ERR_INVALID_ARG, "needs a 3-D layout (dash_hash3d_layout)");
  dash_layout as4 = *layout;
  as4.dims = 0;
  for (int l = 0; l < as4.L; ++l) as4.res_t[l] = 1;
  Geom g;
  if (int s = make_geom(&as4, &g)) return s;
  const int D = g.L * g.F;
  if (mlp == nullptr || mlp->params == nullptr) return fail(DASH_ERR_INVALID_ARG, "mlp/params is NULL");
  if (mlp->d_in != D || mlp->d_hidden != kHidden3 || mlp->d_out != 3)
    return fail(DASH_ERR_UNSUPPORTED, "decomposition MLP must be %d -> 64 -> 3", D);
  if (D > 64) return fail(DASH_ERR_UNSUPPORTED, "L*F=%d > 64", D);
  if (n < 0) return fail(DASH_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return DASH_OK;
  if (x == nullptr || y == nullptr || z == nullptr || table == nullptr || norm_out == nullptr)
    return fail(DASH_ERR_INVALID_ARG, "NULL argument");
  if (pt_out != nullptr && (t == nullptr || t_stride < 0 || t_stride > 1))
    return fail(DASH_ERR_INVALID_ARG, "p(t) needs t with t_stride 0 or 1");
  if (n > 0x7FFFFFFFll) return fail(DASH_ERR_UNSUPPORTED, "n=%lld above 2^31 - 1", (long long)n);
  cudaStream_t st = as_stream(stream);
  if (g_opt_decomp_form == 0) {
    // phi_p on the tensor cores (dfw::decomp_fwd_ws_kernel)
    const int Dp = fused::pad16(D);
    dfw::Args b;
    b.g = g;
    b.x = x, b.y = y, b.z = z, b.n = n;
    b.table = table;
    b.params = mlp->params;
    b.D = D, b.Dp = Dp;
    b.dp_out = dp_out;
    b.norm_out = norm_out;
    b.ts = t;
    b.t_stride = t_stride;
    b.pt_out = pt_out;
    b.flags = fused::decomp_flags_ptr();
    if (b.flags == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the device flag word");
    const uint32_t KA = 3 * Dp + 16, KB = 2 * Dp + 16, KC = Dp;
    auto al = [](uint32_t v) { return (v + 127u) & ~127u; };
    b.off_wb = al(64u * KA * 2u);
    b.off_wc = al(b.off_wb + 64u * KB * 2u);
    b.off_w2 = al(b.off_wc + 64u * KC * 2u);
    b.off_stage = al(b.off_w2 + (3u * 64u + 3u) * 4u);
    b.stage_bytes = al((uint32_t)fused::kRows * KA * 2u);
    b.off_bar = al(b.off_stage + (uint32_t)dfw::kWorkers * b.stage_bytes);
    const size_t tsmem = b.off_bar + 8u * (2u * dfw::kWorkers + 1u) + 16u;
    const long long ntiles_tc = (n + fused::kRows - 1) / fused::kRows;
    long long grid_tc = sm_count();
    grid_tc = ntiles_tc < grid_tc ? ntiles_tc : grid_tc;
#define DASH_DECOMP_FWD_TC(TT, FF)                                                                                   \
  {                                                                                                                  \
    auto kern = dfw::decomp_fwd_ws_kernel<TT, FF>;                                                                   \
    if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem)), \
                            "cudaFuncSetAttribute(decomp_fwd_ws)"))                                                  \
      return s;                                                                                                      \
    kern<<<(unsigned)grid_tc, dfw::kThreadsWs, tsmem, st>>>(b);                                                      \
  }
    if (table_dtype == DASH_F16) {
      switch (g.F) {
        case 1: DASH_DECOMP_FWD_TC(__half, 1) break;
        case 2: DASH_DECOMP_FWD_TC(__half, 2) break;
        case 4: DASH_DECOMP_FWD_TC(__half, 4) break;
        default: DASH_DECOMP_FWD_TC(__half, 8) break;
      }
    } else if (table_dtype == DASH_F32) {
      switch (g.F) {
        case 1: DASH_DECOMP_FWD_TC(float, 1) break;
        case 2: DASH_DECOMP_FWD_TC(float, 2) break;
        case 4: DASH_DECOMP_FWD_TC(float, 4) break;
        default: DASH_DECOMP_FWD_TC(float, 8) break;
      }
    } else {
      return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
    }
#undef DASH_DECOMP_FWD_TC
    return launch_status("decomp_fwd_ws_kernel");
  }
  const size_t smem = sizeof(float) * (size_t)(kHidden3 * D + kHidden3 + 3 * kHidden3 + 3);
  const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
#define DASH_DECOMP_LAUNCH(TT, FF)                                                                             \
  decomp_fwd_kernel<TT, FF><<<grid, kThreads, smem, st>>>(g, x, y, z, n, static_cast<const TT*>(table),        \
                                                          mlp->params, D, dp_out, norm_out, t, t_stride, pt_out)
  if (table_dtype == DASH_F16) {
    switch (g.F) {
      case 1: DASH_DECOMP_LAUNCH(__half, 1); break;
      case 2: DASH_DECOMP_LAUNCH(__half, 2); break;
      case 4: DASH_DECOMP_LAUNCH(__half, 4); break;
      default: DASH_DECOMP_LAUNCH(__half, 8); break;
    }
  } else if (table_dtype == DASH_F32) {
    switch (g.F) {
      case 1: DASH_DECOMP_LAUNCH(float, 1); break;
      case 2: DASH_DECOMP_LAUNCH(float, 2); break;
      case 4: DASH_DECOMP_LAUNCH(float, 4); break;
      default: DASH_DECOMP_LAUNCH(float, 8); break;
    }
  } else {
    return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
  }
#undef DASH_DECOMP_LAUNCH
  return launch_status("decomp_fwd_kernel");
}

size_t dash_decomp_bwd_workspace_size(void) { return 256; }

int dash_decomp_bwd(const dash_layout* layout, const float* x, const float* y, const float* z, int64_t n,
                    const void* table, int table_dtype, const dash_mlp* mlp, const float* d_dp, const uint8_t* mask,
                    float lambda_s, float* table_grad, float* mlp_grad, void* ws, size_t ws_bytes, void* stream) {
  DASH_NVTX_RANGE("dash_decomp_bwd");
  using namespace dash;
  if (layout == nullptr || layout->dims != 3) return fail(DASH_ERR_INVALID_ARG, "needs a 3-D layout (dash_hash3d_layout)");
  dash_layout as4 = *layout;
  as4.dims = 0;
  for (int l = 0; l < as4.L; ++l) as4.res_t[l] = 1;
  DecompBwdArgs a;
  if (int s = make_geom(&as4, &a.g)) return s;
  const int D = a.g.L * a.g.F;
  if (mlp == nullptr || mlp->params == nullptr) return fail(DASH_ERR_INVALID_ARG, "mlp/params is NULL");
  if (mlp->d_in != D || mlp->d_hidden != kHidden3 || mlp->d_out != 3)
    return fail(DASH_ERR_UNSUPPORTED, "decomposition MLP must be %d -> 64 -> 3", D);
  if (D > 64) return fail(DASH_ERR_UNSUPPORTED, "L*F=%d > 64", D);
  if (n < 0 || n > 0x7FFFFFFFll) return fail(DASH_ERR_UNSUPPORTED, "n outside [0, 2^31)");
  if (ws == nullptr || ws_bytes < dash_decomp_bwd_workspace_size())
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, dash_decomp_bwd_workspace_size());
  if (n == 0) return DASH_OK;
  if (x == nullptr || y == nullptr || z == nullptr || table == nullptr || table_grad == nullptr || mlp_grad == nullptr)
    return fail(DASH_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(table) & 15u) != 0 || (reinterpret_cast<uintptr_t>(table_grad) & 15u) != 0)
    return fail(DASH_ERR_INVALID_ARG, "table and table_grad must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  a.x = x, a.y = y, a.z = z, a.n = n;
  a.table = table;
  a.params = mlp->params;
  a.D = D;
  a.d_dp = d_dp;
  a.mask = lambda_s != 0.0f ? mask : nullptr;
  a.lambda_s = lambda_s;
  a.n_static = static_cast<const unsigned long long*>(ws);
  a.table_grad = table_grad;
  a.mlp_grad = mlp_grad;
  if (a.mask != nullptr) {
    if (int s = cuda_status(DASH_RT(cudaMemsetAsync(ws, 0, 8, st)), "cudaMemsetAsync")) return s;
    long long blocks = (n + kThreads - 1) / kThreads;
    const long long cap = 4ll * sm_count();
    blocks = blocks < cap ? blocks : cap;
    count_static_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(a.mask, n, static_cast<unsigned long long*>(ws));
    if (int s = launch_status("count_static_kernel")) return s;
  }
  const int Dp = fused::pad16(D);
  if (Dp <= dtc::kMaxDp && g_opt_decomp_form == 0) {
    // phi_p's contractions on the tensor cores (dtc::decomp_bwd_ws_kernel)
    dtc::Args b;
    b.g = a.g;
    b.x = x, b.y = y, b.z = z, b.n = n;
    b.table = table;
    b.params = mlp->params;
    b.D = D, b.Dp = Dp;
    b.d_dp = d_dp;
    b.mask = a.mask;
    b.lambda_s = lambda_s;
    b.n_static = a.n_static;
    b.table_grad = table_grad;
    b.mlp_grad = mlp_grad;
    b.flags = fused::decomp_flags_ptr();
    if (b.flags == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the device flag word");
    const uint32_t KZ = 2 * Dp + 16, KL = Dp + 16;
    auto al = [](uint32_t v) { return (v + 127u) & ~127u; };
    b.off_w1lo = al(64u * KZ * 2u);
    b.off_w2 = al(b.off_w1lo + 64u * KL * 2u);
    b.off_dz = al(b.off_w2 + (3u * 64u + 3u) * 4u);
    b.off_stage = al(b.off_dz + (uint32_t)fused::kRows * 128u * 2u);
    b.off_df = al((uint32_t)fused::kRows * KZ * 2u);  // the stage's dL/df block right after its F tile
    b.stage_bytes = al(b.off_df + (uint32_t)Dp * fused::kRows * 4u);
    b.off_bar = al(b.off_stage + (uint32_t)dtc::kWorkers * b.stage_bytes);
    const size_t tsmem = b.off_bar + 8u * (2u * dtc::kWorkers + 1u) + 16u;
    const long long ntiles_tc = (n + fused::kRows - 1) / fused::kRows;
    long long grid_tc = sm_count();
    grid_tc = ntiles_tc < grid_tc ? ntiles_tc : grid_tc;
#define DASH_DECOMP_BWD_TC(TT, FF)                                                                                   \
  {                                                                                                                  \
    auto kern = dtc::decomp_bwd_ws_kernel<TT, FF>;                                                                   \
    if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem)), \
                            "cudaFuncSetAttribute(decomp_bwd_ws)"))                                                  \
      return s;                                                                                                      \
    kern<<<(unsigned)grid_tc, dtc::kThreadsWs, tsmem, st>>>(b);                                                      \
  }
    if (table_dtype == DASH_F16) {
      switch (a.g.F) {
        case 1: DASH_DECOMP_BWD_TC(__half, 1) break;
        case 2: DASH_DECOMP_BWD_TC(__half, 2) break;
        case 4: DASH_DECOMP_BWD_TC(__half, 4) break;
        default: DASH_DECOMP_BWD_TC(__half, 8) break;
      }
    } else if (table_dtype == DASH_F32) {
      switch (a.g.F) {
        case 1: DASH_DECOMP_BWD_TC(float, 1) break;
        case 2: DASH_DECOMP_BWD_TC(float, 2) break;
        case 4: DASH_DECOMP_BWD_TC(float, 4) break;
        default: DASH_DECOMP_BWD_TC(float, 8) break;
      }
    } else {
      return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
    }
#undef DASH_DECOMP_BWD_TC
    return launch_status("decomp_bwd_ws_kernel");
  }
  const size_t smem = sizeof(float) * ((size_t)kHidden3 * D + kHidden3 + 3 * kHidden3 + 4 +
                                       (size_t)kBwdRows * ((D + 4) + 2 * (kHidden3 + 1) + 4));
  const long long ntiles = (n + kBwdRows - 1) / kBwdRows;
  long long grid = 2ll * sm_count();
  grid = ntiles < grid ? ntiles : grid;
#define DASH_DECOMP_BWD(TT, FF)                                                                                     \
  {                                                                                                                 \
    auto kern = decomp_bwd_kernel<TT, FF>;                                                                          \
    if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)),     \
                            "cudaFuncSetAttribute(decomp_bwd)"))                                                     \
      return s;                                                                                                     \
    kern<<<(unsigned)grid, kBwdThreads, smem, st>>>(a);                                                             \
  }
  if (table_dtype == DASH_F16) {
    switch (a.g.F) {
      case 1: DASH_DECOMP_BWD(__half, 1) break;
      case 2: DASH_DECOMP_BWD(__half, 2) break;
      case 4: DASH_DECOMP_BWD(__half, 4) break;
      default: DASH_DECOMP_BWD(__half, 8) break;
    }
  } else if (table_dtype == DASH_F32) {
    switch (a.g.F) {
      case 1: DASH_DECOMP_BWD(float, 1) break;
      case 2: DASH_DECOMP_BWD(float, 2) break;
      case 4: DASH_DECOMP_BWD(float, 4) break;
      default: DASH_DECOMP_BWD(float, 8) break;
    }
  } else {
    return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
  }
#undef DASH_DECOMP_BWD
  return launch_status("decomp_bwd_kernel");
}

size_t dash_topk_workspace_size(void) { return (sizeof(dash::TopkState) + 255) / 256 * 256; }

int dash_topk_mask(const float* values, int64_t n, double k_percent, uint8_t* mask_out, float* tau_out,
                   float* static_loss_out, void* ws, size_t ws_bytes, void* stream) {
  DASH_NVTX_RANGE("dash_topk_mask");
  using namespace dash;
  if (n < 0 || !(k_percent >= 0.0) || k_percent > 100.0)
    return fail(DASH_ERR_INVALID_ARG, "n < 0 or k_percent outside [0, 100]");
  if (n > 0x7FFFFFFFll) return fail(DASH_ERR_UNSUPPORTED, "n=%lld above 2^31 - 1", (long long)n);
  if (n > 0 && (values == nullptr || mask_out == nullptr)) return fail(DASH_ERR_INVALID_ARG, "values/mask_out is NULL");
  if (ws == nullptr || ws_bytes < dash_topk_workspace_size())
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, dash_topk_workspace_size());
  cudaStream_t st = as_stream(stream);
  if (n == 0) {
    if (static_loss_out != nullptr && cudaMemsetAsync(static_loss_out, 0, sizeof(float), st) != cudaSuccess)
      return fail(DASH_ERR_CUDA, "cudaMemsetAsync failed");
    return DASH_OK;
  }
  TopkState* state = static_cast<TopkState*>(ws);
  long long m = (long long)floor(k_percent * (double)n / 100.0);
  m = m < 0 ? 0 : m;
  const int all = m >= n;
  const unsigned long long rank = all ? 0ull : (unsigned long long)(n - 1 - m);  // ascending rank of tau
  topk_init<<<1, 256, 0, st>>>(state, rank);
  if (int s = launch_status("topk_init")) return s;
  if (!all) {
    long long blocks = (n + kThreads - 1) / kThreads;
    const long long cap = 4ll * sm_count();
    blocks = blocks < cap ? blocks : cap;
    for (int shift = 24; shift >= 0; shift -= 8) {
      topk_hist<<<(unsigned)blocks, kThreads, 0, st>>>(values, n, state, shift);
      if (int s = launch_status("topk_hist")) return s;
      topk_select<<<1, 32, 0, st>>>(state, shift);
      if (int s = launch_status("topk_select")) return s;
    }
  }
  topk_apply<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(values, n, state, all, mask_out, tau_out,
                                                                             static_loss_out != nullptr);
  if (int s = launch_status("topk_apply")) return s;
  if (static_loss_out == nullptr) return DASH_OK;
  topk_static_loss<<<1, 1, 0, st>>>(state, static_loss_out);
  return launch_status("topk_static_loss");
}

}  // extern "C"
