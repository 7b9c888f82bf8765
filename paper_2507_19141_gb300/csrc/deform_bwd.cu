// deform_bwd.cu -- a9-a11 fused: backward of the deformation decoder and of
// the 4D hash encoder (the learnable tables of Sec. 4.2), plus the Eq. 11
// smoothness term, in one persistent kernel.
//
// Per group of 4 warps and tile of 128 Gaussians (thread r = Gaussian r =
// TMEM lane r):
//   1. f_h: the BF16 copy in the forward state, or, with the smoothness term
//      on (or no state), a fresh FP32 encoding; the perturbed points
//      p + e_s, p + e_t are encoded level by level and their gradient
//      -2 lambda/n (f(p) - f(p+e)) scattered at once (never stored).
//   2. z1 = [f_h | 1] [W1 | b1]^T, h1 = relu(z1); z2 likewise (tensor cores,
//      hi + lo operands).  The ReLU masks come from the forward state (the
//      forward's accurate pre-activations); without a state they are taken
//      from this recompute, which is then fed FP32-accurate f_h.
//   3. dh2 = ddelta W3, dz2 = dh2 * [z2 > 0]; dh1 = dz2 W2, dz1 = dh1 * [z1 > 0];
//      df_h = dz1 W1 -- the weight tiles of the forward read with the
//      transpose bit set.
//   4. dW^T += A^T dZ with the Gaussians as the contraction axis: the
//      activation tiles read MN-major; their constant-one column makes the
//      row after the last feature the bias gradient.  Accumulated in TMEM
//      over all tiles of the CTA and flushed with one atomic per weight.
//   5. table_grad[corner] += w * (df_h + smoothness term) with vector FP32
//      reductions (red.global.add.v2.f32 for F = 2).
//
// For F = 2 with a forward state the warp-specialised kernel splits this:
// a decoder group (steps 2-4) hands df_h per tile through a shared-memory
// ring to scatter groups (step 5, lane pairs); the smoothness term runs in
// smooth.cu.  With the caller's workspace the coarsest dense levels reduce
// into replicas (replicas.cu), and with the smoothness term the decoder
// group alone stores df_h there for smooth.cu to scatter with its own
// gradient.
#include "deform_bwd_common.cuh"

namespace dash {
namespace fused {
namespace {

__device__ unsigned int g_bwd_flags;  // bit 0: an MMA completion wait gave up

// tile extents, TMEM columns and MMA helpers of the backward (deform_bwd_common.cuh)
constexpr int kKH = bwdk::kKH;
constexpr int kKH2 = bwdk::kKH2;
constexpr int kKG = bwdk::kKG;
constexpr int kKO = bwdk::kKO;
constexpr uint32_t kTmemCols = bwdk::kTmemCols;
constexpr uint32_t kColS = bwdk::kColS, kColW1 = bwdk::kColW1, kColW2 = bwdk::kColW2, kColW3 = bwdk::kColW3;
using bwdk::issue;
using bwdk::kmajor;
using bwdk::mnmajor;
using bwdk::Op;
using bwdk::wait_mma;
using bwdk::scatter_levels_paired;

struct BwdArgs {
  Geom g;
  Pts pts;
  const void* table;
  const float* params;
  int D, Dp, O;
  const float* ddelta;
  long long n_cap;
  const uint8_t* state;
  float* table_grad;
  float* mlp_grad;
  float lambda_r;
  float eps_s[3];
  float eps_t;
  float* loss_out;
  float* coord_grad;  // optional SoA [4][n_cap]: d loss / d(x, y, z, t)
  unsigned int* flags;
  int paired;  // F = 2 scatter by lane pairs (no Eq. 11 term, no coordinate gradient)
  float* dfh_out;  // optional SoA [D][n_cap]: dL/df_h stored instead of scattered
  Replicas rep;    // the paired scatter's dense levels go to replicas
  uint32_t off_w2, off_w3, off_f, off_h1, off_x, off_g3, off_ring, off_bar;
};

template <int F>
__device__ __forceinline__ void scatter_level(float* __restrict__ grad, long long off, const uint32_t idx[16],
                                              const float w[16], const float d[F]) {
  float* base = grad + off * F;
  if constexpr (F == 2) {
    scatter2_pairs(base, idx, w, d[0], d[1]);
  } else {
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

// scatter_levels_paired plus the input-coordinate gradient (the quantity
// level_coord_grad computes, summed over the levels and scaled by N_l):
// lane xb gathers its x half of each Gaussian's corners, forms s = d . entry
// for them and its share of the four axis derivatives, and the lanes add
// their shares; returns the gradient of this lane's own Gaussian (before
// the clamp mask).  Matches level_coord_grad up to the order of additions.
template <typename TT>
__device__ __forceinline__ float4 scatter_coord_levels_paired(const Geom& g, const TT* __restrict__ table,
                                                              float* __restrict__ grad, const Replicas& rp,
                                                              float4 p, const float* dfp,
                                                              uint32_t xb, bool vb, unsigned int pm) {
  float4 pa, pb;
  pair_points(p, xb, pm, pa, pb);
  float4 cg = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int l = 0; l < g.L; ++l) {
    const float2 f0 = *reinterpret_cast<const float2*>(dfp + (2 * l) * kRows);
    const float2 f1 = *reinterpret_cast<const float2*>(dfp + (2 * l + 1) * kRows);
    const TT* base = table + g.offset[l] * 2;
    float* gbase = rp.level_base(grad, g, l);
    const float ns = (float)g.res_s[l], nt = (float)g.res_t[l];
#pragma unroll 1
    for (int G = 0; G < 2; ++G) {
      if (G == 1 && !vb) break;  // the same on both lanes
      const float4 pp = G == 0 ? pa : pb;
      const float d0 = G == 0 ? f0.x : f0.y, d1 = G == 0 ? f1.x : f1.y;
      uint32_t idx[8];
      float w[8];
      const float4 gr = coord_level_paired<TT>(g, l, pp, xb, pm, base, d0, d1, idx, w);
      const float gx = gr.x, gy = gr.y, gz = gr.z, gt = gr.w;
      if ((uint32_t)G == xb) {
        cg.x = fmaf(gx, ns, cg.x);
        cg.y = fmaf(gy, ns, cg.y);
        cg.z = fmaf(gz, ns, cg.z);
        cg.w = fmaf(gt, nt, cg.w);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) red_add_v2(gbase + (size_t)idx[q] * 2, w[q] * d0, w[q] * d1);
    }
  }
  return cg;
}

template <typename TT, int F>
__device__ __forceinline__ void gather_level(const TT* __restrict__ table, long long off, const uint32_t idx[16],
                                             const float w[16], float acc[F]) {
  const TT* base = table + off * F;
  if constexpr (F == 2) {
    gather2_pairs<TT>(base, idx, w, acc);
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.0f;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      float e[F];
      load_entry<TT, F>(base + (size_t)idx[b] * F, e);
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] = fmaf(w[b], e[f], acc[f]);
    }
  }
}

// Writes compact point `row`'s coordinate gradient (zero on axes the clamp blocks).
__device__ __forceinline__ void store_coord_grad(const BwdArgs& a, long long row, float4 cg) {
  const float4 m = coord_inside(a.pts, row);
  float* o = a.coord_grad;
  __stcs(o + row, cg.x * m.x);
  __stcs(o + a.n_cap + row, cg.y * m.y);
  __stcs(o + 2 * a.n_cap + row, cg.z * m.z);
  __stcs(o + 3 * a.n_cap + row, cg.w * m.w);
}

__device__ __forceinline__ float4 perturb(float4 p, float ex, float ey, float ez, float et) {
  return make_float4(clamp01(__fadd_rn(p.x, ex)), clamp01(__fadd_rn(p.y, ey)), clamp01(__fadd_rn(p.z, ez)),
                     clamp01(__fadd_rn(p.w, et)));
}

template <typename TT, int F>
__global__ void __launch_bounds__(kRows, 1) deform_bwd_kernel(const __grid_constant__ BwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int r = threadIdx.x, q = r >> 5;
  const int KF = 2 * a.Dp + 16;
  uint8_t* w1 = smem;
  uint8_t* w2 = smem + a.off_w2;
  uint8_t* w3 = smem + a.off_w3;
  uint8_t* Ft = smem + a.off_f;
  uint8_t* H1 = smem + a.off_h1;  // later reused for dz1
  uint8_t* X = smem + a.off_x;    // h2, later dz2
  uint8_t* G3 = smem + a.off_g3;
  uint64_t* bar_p = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(smem + a.off_bar + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_bar + 12);

  const float* W1 = a.params;
  const float* b1 = W1 + kHidden * a.D;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + a.O * kHidden;
  build_weight_tile(w1, kHidden, KF, a.Dp, true, a.D, kHidden, W1, b1, r, kRows);
  build_weight_tile(w2, kHidden, kKH2, kHidden, true, kHidden, kHidden, W2, b2, r, kRows);
  build_weight_tile(w3, kOutPad, kKH, kHidden, false, kHidden, a.O, W3, b3, r, kRows);
  if (r == 0) {
    tc::mbar_init(tc::smem_addr(bar_p), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (r < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), kTmemCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;
  const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16);
  const uint32_t bar = tc::smem_addr(bar_p);
  uint32_t phase = 0;

  const TT* table = static_cast<const TT*>(a.table);
  const long long n = point_count(a.pts);
  const long long ntiles = (n + kRows - 1) / kRows;
  const bool smooth = a.lambda_r != 0.0f;
  const float scale = n > 0 ? 2.0f * a.lambda_r / (float)n : 0.0f;
  float loss = 0.0f;
  bool had_tile = false;

  const uint32_t id_fwd = tc::idesc_bf16(kRows, kHidden, 0, 0);
  const uint32_t id_dh = tc::idesc_bf16(kRows, kHidden, 0, 1);
  const uint32_t id_df = tc::idesc_bf16(kRows, a.Dp, 0, 1);
  const uint32_t id_w = tc::idesc_bf16(kRows, kHidden, 1, 1);
  const uint32_t id_w3 = tc::idesc_bf16(kRows, kOutPad, 1, 1);

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row = tile * kRows + r;
    const bool valid = row < n;
    const float4 p = valid ? load_point(a.pts, row) : make_float4(0.f, 0.f, 0.f, 0.f);

    // ---- 1. f_h operand row [hi | 1 | lo], and the smoothness term's own scatters
    float dreg[64];
    constexpr int kLPC = 8 / F;
    const bool encode = smooth || a.state == nullptr;
    const uint8_t* srow = (valid && a.state != nullptr) ? a.state + row * state_stride(a.D) : nullptr;
    for (int c = 0; c < a.Dp / 8; ++c) {
      float v[8];
      if (encode) {
#pragma unroll
        for (int j = 0; j < kLPC; ++j) {
          const int l = c * kLPC + j;
          float fp[F];
#pragma unroll
          for (int f = 0; f < F; ++f) fp[f] = 0.0f;
          if (valid && l < a.g.L) {
            uint32_t idx[16];
            float w[16];
            level_corners(a.g, l, p, idx, w);
            gather_level<TT, F>(table, a.g.offset[l], idx, w, fp);
            if (smooth) {
              float dp[F];
#pragma unroll
              for (int f = 0; f < F; ++f) dp[f] = 0.0f;
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const float4 pq = e == 0 ? perturb(p, a.eps_s[0], a.eps_s[1], a.eps_s[2], 0.0f)
                                         : perturb(p, 0.0f, 0.0f, 0.0f, a.eps_t);
                level_corners(a.g, l, pq, idx, w);
                float fq[F], dq[F];
                gather_level<TT, F>(table, a.g.offset[l], idx, w, fq);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                  const float diff = fp[f] - fq[f];
                  loss = fmaf(diff, diff, loss);
                  dp[f] = fmaf(scale, diff, dp[f]);
                  dq[f] = -scale * diff;
                }
                scatter_level<F>(a.table_grad, a.g.offset[l], idx, w, dq);
              }
#pragma unroll
              for (int f = 0; f < F; ++f) dreg[(c * kLPC + j) * F + f] = dp[f];
            }
          }
          if (!(valid && l < a.g.L) && smooth) {
#pragma unroll
            for (int f = 0; f < F; ++f) dreg[(c * kLPC + j) * F + f] = 0.0f;
          }
#pragma unroll
          for (int f = 0; f < F; ++f) v[j * F + f] = fp[f];
        }
      } else {
        const __nv_bfloat16* fs = reinterpret_cast<const __nv_bfloat16*>(srow);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * c + j;
          v[j] = (srow != nullptr && k < a.D) ? __bfloat162float(__ldcs(fs + k)) : 0.0f;
        }
      }
      uint4 hi, lo;
      split_hi_lo8(v, hi, lo);
      *reinterpret_cast<uint4*>(Ft + tile_off(r, 8 * c, KF)) = hi;
      *reinterpret_cast<uint4*>(Ft + tile_off(r, a.Dp + 16 + 8 * c, KF)) = lo;
    }
    write_ones(Ft, r, a.Dp, KF);
    uint32_t m1[2] = {0u, 0u}, m2[2] = {0u, 0u};
    if (srow != nullptr) {
      const uint4 m = __ldcs(reinterpret_cast<const uint4*>(srow + state_mask_off(a.D)));
      m1[0] = m.x;
      m1[1] = m.y;
      m2[0] = m.z;
      m2[1] = m.w;
    }
    const bool own_masks = a.state == nullptr;
    tc::fence_async_smem();
    __syncthreads();
    if (*abort_flag) break;
    if (r == 0) {
      tc::fence_after_sync();
      issue(tbase + kColS, kmajor(Ft, KF), kmajor(w1, KF), KF, id_fwd, false);
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag);
    phase ^= 1u;
    tc::fence_after_sync();

    // ---- 2. h1 = relu(z1) -> H1 [hi | 1 | lo]
#pragma unroll
    for (int c = 0; c < kHidden / 16; ++c) {
      float v[16];
      tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (own_masks && v[j] > 0.0f) m1[c >> 1] |= 1u << ((c & 1) * 16 + j);
        v[j] = ((m1[c >> 1] >> ((c & 1) * 16 + j)) & 1u) ? fmaxf(v[j], 0.0f) : 0.0f;
      }
      uint4 h0, l0, h1, l1;
      split_hi_lo8(v, h0, l0);
      split_hi_lo8(v + 8, h1, l1);
      *reinterpret_cast<uint4*>(H1 + tile_off(r, 16 * c, kKH2)) = h0;
      *reinterpret_cast<uint4*>(H1 + tile_off(r, 16 * c + 8, kKH2)) = h1;
      *reinterpret_cast<uint4*>(H1 + tile_off(r, kHidden + 16 + 16 * c, kKH2)) = l0;
      *reinterpret_cast<uint4*>(H1 + tile_off(r, kHidden + 16 + 16 * c + 8, kKH2)) = l1;
    }
    write_ones(H1, r, kHidden, kKH2);
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    if (*abort_flag) break;
    if (r == 0) {
      tc::fence_after_sync();
      issue(tbase + kColS, kmajor(H1, kKH2), kmajor(w2, kKH2), kKH2, id_fwd, false);
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag);
    phase ^= 1u;
    tc::fence_after_sync();

    // ---- 3. h2 = relu(z2) -> X [h2 | 1]; ddelta -> G3
#pragma unroll
    for (int c = 0; c < kHidden / 16; ++c) {
      float v[16];
      tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (own_masks && v[j] > 0.0f) m2[c >> 1] |= 1u << ((c & 1) * 16 + j);
        v[j] = ((m2[c >> 1] >> ((c & 1) * 16 + j)) & 1u) ? fmaxf(v[j], 0.0f) : 0.0f;
      }
      uint32_t h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
      *reinterpret_cast<uint4*>(X + tile_off(r, 16 * c, kKH)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(X + tile_off(r, 16 * c + 8, kKH)) = make_uint4(h[4], h[5], h[6], h[7]);
    }
    write_ones(X, r, kHidden, kKH);
    {
      float d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) d[j] = (valid && j < a.O) ? __ldcs(a.ddelta + (long long)j * a.n_cap + row) : 0.0f;
      uint32_t h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = pack_bf16x2(d[2 * j], d[2 * j + 1]);
      *reinterpret_cast<uint4*>(G3 + tile_off(r, 0, kKO)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(G3 + tile_off(r, 8, kKO)) = make_uint4(h[4], h[5], h[6], h[7]);
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    if (*abort_flag) break;
    if (r == 0) {
      tc::fence_after_sync();
      // dh2 = ddelta W3  (B = W3 tile transposed: N = hidden unit, K = output)
      issue(tbase + kColS, kmajor(G3, kKO), mnmajor(w3, kKH), kKO, id_dh, false);
      // [dW3 | db3]^T += [h2 | 1]^T ddelta
      issue(tbase + kColW3, mnmajor(X, kKH), mnmajor(G3, kKO), kRows, id_w3, had_tile);
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag);
    phase ^= 1u;
    tc::fence_after_sync();

    // ---- 4. dz2 = dh2 * m2 -> X
#pragma unroll
    for (int c = 0; c < kHidden / 16; ++c) {
      float v[16];
      tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = ((m2[c >> 1] >> ((c & 1) * 16 + j)) & 1u) ? v[j] : 0.0f;
      uint32_t h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
      *reinterpret_cast<uint4*>(X + tile_off(r, 16 * c, kKG)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(X + tile_off(r, 16 * c + 8, kKG)) = make_uint4(h[4], h[5], h[6], h[7]);
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    if (*abort_flag) break;
    if (r == 0) {
      tc::fence_after_sync();
      issue(tbase + kColS, kmajor(X, kKG), mnmajor(w2, kKH2), kKG, id_dh, false);           // dh1 = dz2 W2
      issue(tbase + kColW2, mnmajor(H1, kKH2), mnmajor(X, kKG), kRows, id_w, had_tile);     // dW2^T += [h1|1]^T dz2
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag);
    phase ^= 1u;
    tc::fence_after_sync();

    // ---- 5. dz1 = dh1 * m1 -> H1
#pragma unroll
    for (int c = 0; c < kHidden / 16; ++c) {
      float v[16];
      tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = ((m1[c >> 1] >> ((c & 1) * 16 + j)) & 1u) ? v[j] : 0.0f;
      uint32_t h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
      *reinterpret_cast<uint4*>(H1 + tile_off(r, 16 * c, kKG)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(H1 + tile_off(r, 16 * c + 8, kKG)) = make_uint4(h[4], h[5], h[6], h[7]);
    }
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    if (*abort_flag) break;
    if (r == 0) {
      tc::fence_after_sync();
      issue(tbase + kColS, kmajor(H1, kKG), mnmajor(w1, KF), kKG, id_df, false);            // df_h = dz1 W1
      issue(tbase + kColW1, mnmajor(Ft, KF), mnmajor(H1, kKG), kRows, id_w, had_tile);     // dW1^T += [f|1]^T dz1
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag);
    phase ^= 1u;
    tc::fence_after_sync();
    had_tile = true;

    // ---- 6. scatter df_h (+ smoothness gradient at p) into the tables
    float df[64];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (16 * c < a.Dp) {
        float v[16];
        tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) df[16 * c + j] = v[j];
      }
    }
    tc::fence_before_sync();
    if (valid) {
      float4 cg = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int l = 0; l < a.g.L; ++l) {
        uint32_t idx[16];
        float w[16];
        level_corners(a.g, l, p, idx, w);
        float d[F];
#pragma unroll
        for (int f = 0; f < F; ++f) d[f] = df[l * F + f] + (smooth ? dreg[l * F + f] : 0.0f);
        scatter_level<F>(a.table_grad, a.g.offset[l], idx, w, d);
        if (a.coord_grad != nullptr) level_coord_grad<TT, F>(a.g, l, p, table + a.g.offset[l] * F, idx, d, cg);
      }
      if (a.coord_grad != nullptr) store_coord_grad(a, row, cg);
    }
  }

  // ---- flush the CTA's weight gradients (rows = input unit, columns = output unit)
  __syncthreads();
  tc::fence_after_sync();
  if (had_tile && !*abort_flag) {
    float* gW1 = a.mlp_grad;
    float* gb1 = gW1 + kHidden * a.D;
    float* gW2 = gb1 + kHidden;
    float* gb2 = gW2 + kHidden * kHidden;
    float* gW3 = gb2 + kHidden;
    float* gb3 = gW3 + a.O * kHidden;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(trow + kColW1 + 16 * c, v);
      for (int j = 0; j < 16; ++j) {
        const int o = 16 * c + j;
        if (r < a.D) atomicAdd(gW1 + o * a.D + r, v[j]);
        else if (r == a.Dp) atomicAdd(gb1 + o, v[j]);
      }
      tc::tmem_ld16(trow + kColW2 + 16 * c, v);
      for (int j = 0; j < 16; ++j) {
        const int o = 16 * c + j;
        if (r < kHidden) atomicAdd(gW2 + o * kHidden + r, v[j]);
        else if (r == kHidden) atomicAdd(gb2 + o, v[j]);
      }
    }
    {
      float v[16];
      tc::tmem_ld16(trow + kColW3, v);
      for (int j = 0; j < a.O; ++j) {
        if (r < kHidden) atomicAdd(gW3 + j * kHidden + r, v[j]);
        else if (r == kHidden) atomicAdd(gb3 + j, v[j]);
      }
    }
  }
  if (smooth && a.loss_out != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((r & 31) == 0 && n > 0) atomicAdd(a.loss_out, a.lambda_r * loss / (float)n);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (r < 32) tc::tmem_dealloc(tbase, kTmemCols);
}

// ---------------------------------------------------------------------------
// Warp-specialised backward.  Warps 0-3 (the decoder group, thread r = TMEM
// lane r) rebuild f_h from the forward state, run the decoder recompute and
// back-propagation on the tensor cores, accumulate dW in TMEM, and publish
// dL/df_h of each tile into a shared-memory ring (transposed [D][128] FP32).
// P scatter groups drain the ring: each thread takes one Gaussian, recomputes
// its corners and issues the vector reductions into the tables; with the
// smoothness term on they also encode p, p + e_s, p + e_t and scatter the
// perturbed points' gradients.  When P divides L (lane pairs, no coordinate
// gradient) every group takes every tile and scatters levels
// [g L / P, (g + 1) L / P) of it, and a stage is released once all P groups
// are done with it; this spreads each tile's reductions over the groups and
// keeps all of them busy on the last tiles.  Otherwise group g takes tiles
// g, g + P, ...  With P = 0 (no ring) the decoder group
// stores dL/df_h to a.dfh_out for the Eq. 11 kernel to scatter; that form's
// 110 KB of shared memory lets two CTAs share an SM.  Requires the forward
// state.
// ---------------------------------------------------------------------------
template <typename TT, int F, int P, int S>
__global__ void __launch_bounds__((P + 1) * kRows, 1) deform_bwd_ws_kernel(const __grid_constant__ BwdArgs a) {
  // tile j uses stage j % S.  The mbarrier waits tell phases apart only by
  // parity: with whole tiles in turn (group j % P) no two groups may wait on
  // one stage at once; with the levels split all groups wait on the same
  // phase, and the decoder refills a stage only after every group released it
  static_assert(S >= P, "the ring needs at least one stage per scatter group");
  static_assert(P > 0 || S == 0, "the store-only form has no ring");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int KF = 2 * a.Dp + 16;
  uint8_t* w1 = smem;
  uint8_t* w2 = smem + a.off_w2;
  uint8_t* w3 = smem + a.off_w3;
  uint8_t* Ft = smem + a.off_f;
  uint8_t* H1 = smem + a.off_h1;
  uint8_t* X = smem + a.off_x;
  uint8_t* G3 = smem + a.off_g3;
  float* ring = reinterpret_cast<float*>(smem + a.off_ring);  // S stages of [Dp][kRows]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  uint64_t* empty = full + S;
  uint64_t* mma_bar = empty + S;
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(mma_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_bar + 1) + 1;
  const int stage_floats = a.Dp * kRows;

  const bwdk::Tiles tl{w1, w2, w3, Ft, H1, X, G3, KF, a.D, a.Dp, a.O};
  if (tid < kRows) bwdk::build_weights(tl, a.params, tid, kRows);
  // With lane pairs and no coordinate gradient, when the groups divide the
  // levels evenly, every scatter group takes every tile and scatters its own
  // share of the levels (so the last tiles are shared by all groups);
  // otherwise the groups take whole tiles in turn.
  const bool split = F == 2 && P > 0 && a.paired && a.coord_grad == nullptr && a.g.L % (P > 0 ? P : 1) == 0;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(tc::smem_addr(&full[s]), kRows);
      tc::mbar_init(tc::smem_addr(&empty[s]), split ? P * kRows : kRows);
    }
    tc::mbar_init(tc::smem_addr(mma_bar), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), kTmemCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;

  const long long n = point_count(a.pts);
  const long long ntiles = (n + kRows - 1) / kRows;
  const long long my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const bool smooth = F != 2 && a.lambda_r != 0.0f;  // F = 2: the Eq. 11 term runs in smooth.cu
  const float scale = n > 0 ? 2.0f * a.lambda_r / (float)n : 0.0f;
  float loss = 0.0f;

  if (tid < kRows) {
    // ----------------------------------------------------- decoder group
    const int r = tid, q = tid >> 5;
    const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16);
    const uint32_t bar = tc::smem_addr(mma_bar);
    uint32_t phase = 0;
    bool had_tile = false;
    const bwdk::Ids ids = bwdk::make_ids(a.Dp);
    for (long long j = 0; j < my_tiles; ++j) {
      const long long row = (blockIdx.x + j * gridDim.x) * kRows + r;
      const bool valid = row < n;
      const uint8_t* srow = valid ? a.state + row * state_stride(a.D) : nullptr;
      if (!bwdk::decoder_tile(tl, ids, tbase, trow, r, bar, phase, a.flags, abort_flag, srow, a.ddelta + row,
                              a.n_cap, valid, had_tile))
        break;
      had_tile = true;
      if constexpr (P == 0) {
        bwdk::store_dfh(a.dfh_out, trow, a.D, a.Dp, a.n_cap, row, valid);
      } else {
        // publish dL/df_h of this tile to the scatter groups
        const int s = (int)(j % S);
        const uint32_t round = (uint32_t)(j / S);
        if (!tc::mbar_wait(tc::smem_addr(&empty[s]), (round & 1u) ^ 1u, kWaitIters)) {
          atomicOr(a.flags, 1u);
          *abort_flag = 1;
        }
        bwdk::publish(ring + (size_t)s * stage_floats, trow, r, a.Dp);
        tc::fence_before_sync();
        tc::mbar_arrive(tc::smem_addr(&full[s]));
      }
    }
    // flush the CTA's weight gradients (rows = input unit, columns = output unit)
    tc::named_sync(1, kRows);
    tc::fence_after_sync();
    if (had_tile && !*abort_flag) bwdk::flush_dw(trow, r, a.D, a.Dp, a.O, a.mlp_grad);
  } else if constexpr (P > 0) {
    // ------------------------------------------------------ scatter groups
    const int pg = tid / kRows - 1, r = tid % kRows;
    const TT* table = static_cast<const TT*>(a.table);
    const long long j0 = split ? 0 : pg, jstep = split ? 1 : P;
    const int l0 = split ? pg * a.g.L / (P > 0 ? P : 1) : 0;
    const int l1 = split ? (pg + 1) * a.g.L / (P > 0 ? P : 1) : a.g.L;
    // the point of this group's next tile is loaded one tile ahead, so the
    // index and coordinate latencies overlap the current tile's reductions
    long long next_row = (blockIdx.x + j0 * gridDim.x) * kRows + r;
    float4 p_next = (j0 < my_tiles && next_row < n) ? load_point(a.pts, next_row) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long j = j0; j < my_tiles; j += jstep) {
      const int s = (int)(j % S);
      const uint32_t round = (uint32_t)(j / S);
      const long long row = next_row;
      const float4 p = p_next;
      next_row = (blockIdx.x + (j + jstep) * gridDim.x) * kRows + r;
      if (j + jstep < my_tiles && next_row < n) p_next = load_point(a.pts, next_row);
      if (!tc::mbar_wait(tc::smem_addr(&full[s]), round & 1u, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      // dL/df_h of this tile is read from the stage level by level; the
      // stage is handed back once the tile's reductions are issued
      const float* stage = ring + (size_t)s * stage_floats;
      if (*abort_flag) break;
      bool done = false;
      if constexpr (F == 2) {
        if (a.paired) {
          const long long row_a = row - (r & 1);  // the pair's even row; both lanes agree on row_a < n
          const uint32_t xb = (uint32_t)(r & 1);
          const unsigned int pm = 3u << (r & 30);
          if (row_a < n) {
            if (a.coord_grad == nullptr) {
              scatter_levels_paired(a.g, a.table_grad, a.rep, p, stage + (r & ~1), xb, true, row_a + 1 < n, pm, l0,
                                    l1);
            } else {
              const float4 cg = scatter_coord_levels_paired<TT>(a.g, table, a.table_grad, a.rep, p, stage + (r & ~1), xb,
                                                                row_a + 1 < n, pm);
              if (row < n) store_coord_grad(a, row, cg);
            }
          }
          done = true;
        }
      }
      if (!done && row < n) {
        float4 cg = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int l = 0; l < a.g.L; ++l) {
          float d[F];
#pragma unroll
          for (int f = 0; f < F; ++f) d[f] = stage[(l * F + f) * kRows + r];
          uint32_t idx[16];
          float w[16];
          level_corners(a.g, l, p, idx, w);
          if (a.coord_grad != nullptr) level_coord_grad<TT, F>(a.g, l, p, table + a.g.offset[l] * F, idx, d, cg);
          if constexpr (F != 2) if (smooth) {
            float fp[F];
            gather_level<TT, F>(table, a.g.offset[l], idx, w, fp);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float4 pq = e == 0 ? perturb(p, a.eps_s[0], a.eps_s[1], a.eps_s[2], 0.0f)
                                       : perturb(p, 0.0f, 0.0f, 0.0f, a.eps_t);
              uint32_t qi[16];
              float qw[16];
              level_corners(a.g, l, pq, qi, qw);
              float fq[F], dq[F];
              gather_level<TT, F>(table, a.g.offset[l], qi, qw, fq);
#pragma unroll
              for (int f = 0; f < F; ++f) {
                const float diff = fp[f] - fq[f];
                loss = fmaf(diff, diff, loss);
                d[f] = fmaf(scale, diff, d[f]);
                dq[f] = -scale * diff;
              }
              scatter_level<F>(a.table_grad, a.g.offset[l], qi, qw, dq);
            }
          }
          scatter_level<F>(a.table_grad, a.g.offset[l], idx, w, d);
        }
        if (a.coord_grad != nullptr) store_coord_grad(a, row, cg);
      }
      tc::mbar_arrive(tc::smem_addr(&empty[s]));
    }
  }
  if (smooth && a.loss_out != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0 && tid >= kRows && n > 0) atomicAdd(a.loss_out, a.lambda_r * loss / (float)n);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, kTmemCols);
}

template <typename TT, int F, int P, int S>
int launch_ws(BwdArgs a, cudaStream_t st) {
  const int KF = 2 * a.Dp + 16;
  uint32_t off = (uint32_t)kHidden * KF * 2;
  a.off_w2 = (off + 127) & ~127u;
  a.off_w3 = a.off_w2 + (uint32_t)kHidden * kKH2 * 2;
  off = a.off_w3 + (uint32_t)kOutPad * kKH * 2;
  a.off_f = (off + 127) & ~127u;
  a.off_h1 = a.off_f + (uint32_t)kRows * KF * 2;
  a.off_x = a.off_h1 + (uint32_t)kRows * kKH2 * 2;
  a.off_g3 = a.off_x + (uint32_t)kRows * kKH * 2;
  a.off_ring = a.off_g3 + (uint32_t)kRows * kKO * 2;
  a.off_bar = a.off_ring + (uint32_t)S * a.Dp * kRows * 4;
  const size_t smem = a.off_bar + 8 * (2 * S + 1) + 16;
  if (smem > 227 * 1024) return fail(DASH_ERR_UNSUPPORTED, "backward form needs %zu B of shared memory", smem);
  auto kern = deform_bwd_ws_kernel<TT, F, P, S>;
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)),
                          "cudaFuncSetAttribute(deform_bwd_ws)"))
    return s;
  const long long ntiles = (a.n_cap + kRows - 1) / kRows;
  long long grid = (P == 0 ? 2 : 1) * (long long)sm_count();  // the store-only form fits two CTAs per SM
  grid = ntiles < grid ? (ntiles > 0 ? ntiles : 1) : grid;
  kern<<<(unsigned)grid, (P + 1) * kRows, smem, st>>>(a);
  return launch_status("deform_bwd_ws_kernel");
}

template <typename TT, int F>
int launch(BwdArgs a, cudaStream_t st) {
  // Tiles read transposed with M = 128 rows (F, H1, X) run past their own
  // end into the next region; G3 comes last and is read within its bounds.
  const int KF = 2 * a.Dp + 16;
  uint32_t off = (uint32_t)kHidden * KF * 2;
  a.off_w2 = (off + 127) & ~127u;
  a.off_w3 = a.off_w2 + (uint32_t)kHidden * kKH2 * 2;
  off = a.off_w3 + (uint32_t)kOutPad * kKH * 2;
  a.off_f = (off + 127) & ~127u;
  a.off_h1 = a.off_f + (uint32_t)kRows * KF * 2;
  a.off_x = a.off_h1 + (uint32_t)kRows * kKH2 * 2;
  a.off_g3 = a.off_x + (uint32_t)kRows * kKH * 2;
  a.off_bar = a.off_g3 + (uint32_t)kRows * kKO * 2;
  const size_t smem = a.off_bar + 64;
  auto kern = deform_bwd_kernel<TT, F>;
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)),
                          "cudaFuncSetAttribute(deform_bwd)"))
    return s;
  int per_sm = 0;
  if (int s = cuda_status(DASH_RT(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRows, smem)),
                          "occupancy(deform_bwd)"))
    return s;
  per_sm = per_sm < 1 ? 1 : per_sm;
  while (per_sm * (int)kTmemCols > 512) --per_sm;
  const long long ntiles = (a.n_cap + kRows - 1) / kRows;
  const long long cap = (long long)per_sm * sm_count();
  const long long grid = ntiles < cap ? ntiles : cap;
  kern<<<(unsigned)grid, kRows, smem, st>>>(a);
  return launch_status("deform_bwd_kernel");
}

template <typename TT>
int dispatch(int F, bool ws, BwdArgs& a, cudaStream_t st) {
  if (ws && F == 2 && a.Dp <= 32) {
    // warp-specialised shapes (scatter groups, ring stages); 0 = the measured best
    switch (g_opt_bwd_form) {
      case 0: return launch_ws<TT, 2, 4, 5>(a, st);
      case 10: return launch_ws<TT, 2, 3, 6>(a, st);
      case 11: return launch_ws<TT, 2, 4, 4>(a, st);
      case 12: return launch_ws<TT, 2, 2, 4>(a, st);
      case 13: return launch_ws<TT, 2, 5, 5>(a, st);
      case 14: return launch_ws<TT, 2, 3, 3>(a, st);
      default: break;
    }
  }
  if (ws) {
    if (a.Dp > 32) {
      switch (F) {
        case 1: return launch_ws<TT, 1, 2, 2>(a, st);
        case 2: return launch_ws<TT, 2, 2, 2>(a, st);
        case 4: return launch_ws<TT, 4, 2, 2>(a, st);
        default: return launch_ws<TT, 8, 2, 2>(a, st);
      }
    }
    switch (F) {
      case 1: return launch_ws<TT, 1, 3, 6>(a, st);
      case 2: return launch_ws<TT, 2, 3, 6>(a, st);
      case 4: return launch_ws<TT, 4, 3, 6>(a, st);
      default: return launch_ws<TT, 8, 3, 6>(a, st);
    }
  }
  switch (F) {
    case 1: return launch<TT, 1>(a, st);
    case 2: return launch<TT, 2>(a, st);
    case 4: return launch<TT, 4>(a, st);
    default: return launch<TT, 8>(a, st);
  }
}

}  // namespace

int check_fused_mlp(const dash_mlp* mlp, int D);

// The backward's workspace: the gradient replicas, then (with the Eq. 11
// term) dL/df_h as FP32 SoA [L*F][n], 256-byte aligned.
struct BwdWorkspace {
  Replicas rep;
  size_t rep_bytes, dfh_off, total;
};

BwdWorkspace bwd_workspace(const dash_layout* layout, long long n, bool with_dfh) {
  BwdWorkspace w;
  w.rep = replica_plan(layout, g_opt_grad_replicas, &w.rep_bytes);
  w.dfh_off = (w.rep_bytes + 255) & ~(size_t)255;
  w.total = with_dfh ? w.dfh_off + (size_t)layout->L * layout->F * (size_t)n * sizeof(float) : w.rep_bytes;
  return w;
}

unsigned int* bwd_flags_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_bwd_flags) != cudaSuccess) return nullptr;
  return static_cast<unsigned int*>(p);
}

}  // namespace fused
}  // namespace dash

extern "C" int dash_deform_mlp_bwd(const dash_layout* layout, const dash_points* pts, const void* table,
                                   int table_dtype, const dash_mlp* mlp, const float* ddelta, const void* fwd_state,
                                   float* table_grad, float* mlp_grad, const dash_smooth* smooth,
                                   float* coord_grad, void* ws_buf, size_t ws_bytes, void* stream) {
  DASH_NVTX_RANGE("dash_deform_mlp_bwd");
  using namespace dash;
  using namespace dash::fused;
  BwdArgs a;
  memset(&a, 0, sizeof(a));
  if (int s = make_geom(layout, &a.g)) return s;
  if (int s = make_pts(pts, &a.pts)) return s;
  const int D = a.g.L * a.g.F;
  if (int s = check_fused_mlp(mlp, D)) return s;
  if (a.pts.n == 0) return DASH_OK;
  if (table == nullptr || ddelta == nullptr || table_grad == nullptr || mlp_grad == nullptr)
    return fail(DASH_ERR_INVALID_ARG, "table/ddelta/table_grad/mlp_grad is NULL");
  if ((reinterpret_cast<uintptr_t>(table_grad) & 15u) != 0)
    return fail(DASH_ERR_INVALID_ARG, "table_grad must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(table) & 15u) != 0) return fail(DASH_ERR_INVALID_ARG, "table must be 16-byte aligned");
  a.table = table;
  a.params = mlp->params;
  a.D = D;
  a.Dp = pad16(D);
  a.O = mlp->d_out;
  a.ddelta = ddelta;
  a.n_cap = a.pts.n;
  a.state = static_cast<const uint8_t*>(fwd_state);
  if (fwd_state != nullptr && (reinterpret_cast<uintptr_t>(fwd_state) & 15u) != 0)
    return fail(DASH_ERR_INVALID_ARG, "fwd_state must be 16-byte aligned");
  a.table_grad = table_grad;
  a.mlp_grad = mlp_grad;
  if (smooth != nullptr) {
    a.lambda_r = smooth->lambda_r;
    for (int i = 0; i < 3; ++i) a.eps_s[i] = smooth->eps_s[i];
    a.eps_t = smooth->eps_t;
    a.loss_out = smooth->loss_out;
  }
  if (coord_grad != nullptr && a.lambda_r != 0.0f)
    return fail(DASH_ERR_UNSUPPORTED, "coordinate gradients with the Eq. 11 term on are not supported");
  a.coord_grad = coord_grad;
  a.paired = (g_opt_access_form == 0 && a.g.F == 2 && a.lambda_r == 0.0f) ? 1 : 0;
  a.flags = bwd_flags_ptr();
  if (a.flags == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the device flag word");
  cudaStream_t st = as_stream(stream);
  // the warp-specialised form needs the forward state; without it the
  // single-group form re-encodes f_h itself
  const bool ws = g_opt_bwd_form != 1 && a.state != nullptr;
  if (table_dtype != DASH_F32 && table_dtype != DASH_F16)
    return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
  // F = 2 with the warp-specialised form: the Eq. 11 term runs in its own
  // kernel after the df_h scatter (both add into table_grad)
  const bool smooth_apart = ws && a.g.F == 2 && a.lambda_r != 0.0f;
  BwdArgs b = a;
  if (smooth_apart) {
    b.lambda_r = 0.0f;
    b.loss_out = nullptr;
    b.paired = g_opt_access_form == 0 ? 1 : 0;
  }
  // the workspace: replicas of the dense levels' gradients, and dL/df_h for
  // the Eq. 11 kernel; used by the lane-paired F = 2 paths only
  const float* dfh = nullptr;
  Replicas rep;
  memset(&rep, 0, sizeof(rep));
  size_t rep_bytes = 0;
  // (not with the coordinate gradient: its table gathers share the L2 with
  // the replicas, and ncu showed 3x the DRAM traffic for no time gained)
  if (ws_buf != nullptr && ws && a.g.F == 2 && g_opt_access_form == 0 && (smooth_apart || coord_grad == nullptr)) {
    const BwdWorkspace wl = bwd_workspace(layout, a.n_cap, smooth_apart);
    if (ws_bytes < wl.total)
      return fail(DASH_ERR_WORKSPACE, "backward workspace %zu B < %zu B", ws_bytes, wl.total);
    if ((reinterpret_cast<uintptr_t>(ws_buf) & 15u) != 0)
      return fail(DASH_ERR_INVALID_ARG, "backward workspace must be 16-byte aligned");
    rep = wl.rep;
    rep.base = static_cast<float*>(ws_buf);
    rep_bytes = wl.rep_bytes;
    if (smooth_apart) {
      b.dfh_out = reinterpret_cast<float*>(static_cast<char*>(ws_buf) + wl.dfh_off);
      dfh = b.dfh_out;
    } else {
      b.rep = rep;
    }
  }
  if (int r = replica_clear(rep, rep_bytes, st)) return r;
  int s;
  if (dfh != nullptr)  // the decoder alone, dL/df_h stored for the Eq. 11 kernel
    s = table_dtype == DASH_F32 ? launch_ws<float, 2, 0, 0>(b, st) : launch_ws<__half, 2, 0, 0>(b, st);
  else
    s = table_dtype == DASH_F32 ? dispatch<float>(a.g.F, ws, b, st) : dispatch<__half>(a.g.F, ws, b, st);
  if (s == DASH_OK && smooth_apart)
    s = launch_smooth2(a.g, a.pts, table, table_dtype, table_grad, smooth, dfh, a.n_cap, rep, st);
  if (s != DASH_OK) return s;
  return replica_sum(a.g, rep, table_grad, st);
}

extern "C" size_t dash_deform_bwd_workspace_size(const dash_layout* layout, int64_t n, const dash_smooth* smooth) {
  if (layout == nullptr || layout->F != 2 || n < 0) return 0;
  return dash::fused::bwd_workspace(layout, n, smooth != nullptr && smooth->lambda_r != 0.0f).total;
}
