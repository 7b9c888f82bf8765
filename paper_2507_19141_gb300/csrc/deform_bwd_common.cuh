// deform_bwd_common.cuh -- the decoder group's share of the fused backward
// (a9: decoder recompute and back-propagation on the tensor cores), used by
// the single-scene warp-specialised backward (deform_bwd.cu) and by the
// batched one (batch.cu).  Thread r of the 128-thread decoder group owns
// tile row r = TMEM lane r.
//
// Per tile: f_h (BF16) and the ReLU masks come from the forward state; the
// decoder is recomputed (z1, z2 with hi + lo operands), then
//   dh2 = ddelta W3, dz2 = dh2 * [z2 > 0]; dh1 = dz2 W2, dz1 = dh1 * [z1 > 0];
//   df_h = dz1 W1 -- the weight tiles read with the transpose bit set --
// and dW^T += A^T dZ with the Gaussians as the contraction axis (activation
// tiles read MN-major; their constant-one column makes the row after the
// last input the bias gradient), accumulated in TMEM across tiles.
#pragma once

#include "deform_common.cuh"

namespace dash {
namespace fused {
namespace bwdk {

constexpr int kKH = kHidden + 16;        // h2 tile and W3 tile K: [h | 1, 0..]
constexpr int kKH2 = 2 * kHidden + 16;   // h1 tile and W2 tile K: [hi | 1, 0.. | lo]
constexpr int kKG = kHidden;             // dz tile K
constexpr int kKO = kOutPad;             // ddelta tile K
constexpr uint32_t kTmemCols = 256;      // S (64) | dW1 (64) | dW2 (64) | dW3 (16)
constexpr uint32_t kColS = 0, kColW1 = 64, kColW2 = 128, kColW3 = 192;

__device__ __forceinline__ bool wait_mma(uint32_t bar, uint32_t phase, unsigned int* flags, volatile int* abort) {
  if (tc::mbar_wait(bar, phase, kWaitIters)) return true;
  atomicOr(flags, 1u);
  *abort = 1;
  return false;
}

// One MMA chain over K (step 16) with per-operand descriptor strides.
struct Op {
  uint32_t addr, lbo, sbo, kstep;  // kstep: start-address advance per 16 K
};

__device__ __forceinline__ void issue(uint32_t tmem, Op a, Op b, int K, uint32_t idesc, bool accumulate) {
  for (int k = 0; k < K; k += 16) {
    const uint32_t s = (uint32_t)(k / 16);
    const uint64_t ad = tc::smem_desc(a.addr + s * a.kstep, a.lbo, a.sbo);
    const uint64_t bd = tc::smem_desc(b.addr + s * b.kstep, b.lbo, b.sbo);
    tc::mma_bf16(tmem, ad, bd, idesc, (accumulate || k > 0) ? 1u : 0u);
  }
}

// K-major operand (rows = MN axis, tile K extent KE).
__device__ __forceinline__ Op kmajor(const uint8_t* t, int KE) {
  return Op{tc::smem_addr(t), 128u, (uint32_t)KE * 16u, 256u};
}
// The same tile read transposed: its rows become the K axis.
__device__ __forceinline__ Op mnmajor(const uint8_t* t, int KE) {
  return Op{tc::smem_addr(t), (uint32_t)KE * 16u, 128u, (uint32_t)KE * 32u};
}

// The decoder group's shared-memory tiles and shapes.
struct Tiles {
  uint8_t *w1, *w2, *w3, *Ft, *H1, *X, *G3;
  int KF, D, Dp, O;
};

// Instruction descriptors of the five MMA shapes.
struct Ids {
  uint32_t fwd, dh, df, w, w3;
};
__device__ __forceinline__ Ids make_ids(int Dp) {
  return Ids{tc::idesc_bf16(kRows, kHidden, 0, 0), tc::idesc_bf16(kRows, kHidden, 0, 1),
             tc::idesc_bf16(kRows, Dp, 0, 1), tc::idesc_bf16(kRows, kHidden, 1, 1),
             tc::idesc_bf16(kRows, kOutPad, 1, 1)};
}

// BF16 weight tiles of the decoder with packed parameters `params`.
__device__ __forceinline__ void build_weights(const Tiles& t, const float* params, int tid, int nthreads) {
  const float* W1 = params;
  const float* b1 = W1 + kHidden * t.D;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + t.O * kHidden;
  build_weight_tile(t.w1, kHidden, t.KF, t.Dp, true, t.D, kHidden, W1, b1, tid, nthreads);
  build_weight_tile(t.w2, kHidden, kKH2, kHidden, true, kHidden, kHidden, W2, b2, tid, nthreads);
  build_weight_tile(t.w3, kOutPad, kKH, kHidden, false, kHidden, t.O, W3, b3, tid, nthreads);
}

// One tile on the decoder group: row r's forward state srow (NULL: a zero
// row) and upstream gradient dd[k * dd_stride], k < O (read when valid).
// Leaves dL/df_h in TMEM columns kColS.. and adds the tile's weight
// gradients into the TMEM accumulators (overwrites them when !had_tile).
// Returns false when a bounded wait gave up (abort_flag set).
__device__ __forceinline__ bool decoder_tile(const Tiles& t, const Ids& id, uint32_t tbase, uint32_t trow, int r,
                                             uint32_t bar, uint32_t& phase, unsigned int* flags,
                                             volatile int* abort_flag, const uint8_t* srow, const float* dd,
                                             long long dd_stride, bool valid, bool had_tile) {
  // the upstream gradient is loaded with the state, so that its latency
  // overlaps the state's and the first two layers instead of following them
  float d[16];
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) d[jj] = (valid && jj < t.O) ? __ldcs(dd + (long long)jj * dd_stride) : 0.0f;
  // f_h [hi | 1 | 0] from the state, masks from the forward
  const __nv_bfloat16* fs = reinterpret_cast<const __nv_bfloat16*>(srow);
  for (int c = 0; c < t.Dp / 8; ++c) {
    uint4 hv;
    if (srow != nullptr && 8 * c + 8 <= t.D) {
      hv = __ldcs(reinterpret_cast<const uint4*>(fs + 8 * c));  // rows are 16-byte aligned
    } else {
      uint32_t h[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int k = 8 * c + 2 * jj;
        const float v0 = (srow != nullptr && k < t.D) ? __bfloat162float(__ldcs(fs + k)) : 0.0f;
        const float v1 = (srow != nullptr && k + 1 < t.D) ? __bfloat162float(__ldcs(fs + k + 1)) : 0.0f;
        h[jj] = pack_bf16x2(v0, v1);
      }
      hv = make_uint4(h[0], h[1], h[2], h[3]);
    }
    *reinterpret_cast<uint4*>(t.Ft + tile_off(r, 8 * c, t.KF)) = hv;
    *reinterpret_cast<uint4*>(t.Ft + tile_off(r, t.Dp + 16 + 8 * c, t.KF)) = make_uint4(0u, 0u, 0u, 0u);
  }
  write_ones(t.Ft, r, t.Dp, t.KF);
  uint32_t m1[2] = {0u, 0u}, m2[2] = {0u, 0u};
  if (srow != nullptr) {
    const uint4 m = __ldcs(reinterpret_cast<const uint4*>(srow + state_mask_off(t.D)));
    m1[0] = m.x;
    m1[1] = m.y;
    m2[0] = m.z;
    m2[1] = m.w;
  }
  tc::fence_async_smem();
  tc::named_sync(1, kRows);
  if (*abort_flag) return false;
  if (r == 0) {
    tc::fence_after_sync();
    issue(tbase + kColS, kmajor(t.Ft, t.KF), kmajor(t.w1, t.KF), t.KF, id.fwd, false);
    tc::mma_commit(bar);
  }
  wait_mma(bar, phase, flags, abort_flag);
  phase ^= 1u;
  tc::fence_after_sync();
  // h1 = relu(z1) with the forward's mask -> H1 [hi | 1 | lo]
#pragma unroll
  for (int c = 0; c < kHidden / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj)
      v[jj] = ((m1[c >> 1] >> ((c & 1) * 16 + jj)) & 1u) ? fmaxf(v[jj], 0.0f) : 0.0f;
    uint4 h0, l0, h1, l1;
    split_hi_lo8(v, h0, l0);
    split_hi_lo8(v + 8, h1, l1);
    *reinterpret_cast<uint4*>(t.H1 + tile_off(r, 16 * c, kKH2)) = h0;
    *reinterpret_cast<uint4*>(t.H1 + tile_off(r, 16 * c + 8, kKH2)) = h1;
    *reinterpret_cast<uint4*>(t.H1 + tile_off(r, kHidden + 16 + 16 * c, kKH2)) = l0;
    *reinterpret_cast<uint4*>(t.H1 + tile_off(r, kHidden + 16 + 16 * c + 8, kKH2)) = l1;
  }
  write_ones(t.H1, r, kHidden, kKH2);
  tc::fence_before_sync();
  tc::fence_async_smem();
  tc::named_sync(1, kRows);
  if (*abort_flag) return false;
  if (r == 0) {
    tc::fence_after_sync();
    issue(tbase + kColS, kmajor(t.H1, kKH2), kmajor(t.w2, kKH2), kKH2, id.fwd, false);
    tc::mma_commit(bar);
  }
  wait_mma(bar, phase, flags, abort_flag);
  phase ^= 1u;
  tc::fence_after_sync();
  // h2 -> X [h2 | 1]; ddelta -> G3
#pragma unroll
  for (int c = 0; c < kHidden / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj)
      v[jj] = ((m2[c >> 1] >> ((c & 1) * 16 + jj)) & 1u) ? fmaxf(v[jj], 0.0f) : 0.0f;
    uint32_t h[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) h[jj] = pack_bf16x2(v[2 * jj], v[2 * jj + 1]);
    *reinterpret_cast<uint4*>(t.X + tile_off(r, 16 * c, kKH)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(t.X + tile_off(r, 16 * c + 8, kKH)) = make_uint4(h[4], h[5], h[6], h[7]);
  }
  write_ones(t.X, r, kHidden, kKH);
  {
    uint32_t h[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) h[jj] = pack_bf16x2(d[2 * jj], d[2 * jj + 1]);
    *reinterpret_cast<uint4*>(t.G3 + tile_off(r, 0, kKO)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(t.G3 + tile_off(r, 8, kKO)) = make_uint4(h[4], h[5], h[6], h[7]);
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  tc::named_sync(1, kRows);
  if (*abort_flag) return false;
  if (r == 0) {
    tc::fence_after_sync();
    issue(tbase + kColS, kmajor(t.G3, kKO), mnmajor(t.w3, kKH), kKO, id.dh, false);
    issue(tbase + kColW3, mnmajor(t.X, kKH), mnmajor(t.G3, kKO), kRows, id.w3, had_tile);
    tc::mma_commit(bar);
  }
  wait_mma(bar, phase, flags, abort_flag);
  phase ^= 1u;
  tc::fence_after_sync();
  // dz2 = dh2 * m2 -> X
#pragma unroll
  for (int c = 0; c < kHidden / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) v[jj] = ((m2[c >> 1] >> ((c & 1) * 16 + jj)) & 1u) ? v[jj] : 0.0f;
    uint32_t h[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) h[jj] = pack_bf16x2(v[2 * jj], v[2 * jj + 1]);
    *reinterpret_cast<uint4*>(t.X + tile_off(r, 16 * c, kKG)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(t.X + tile_off(r, 16 * c + 8, kKG)) = make_uint4(h[4], h[5], h[6], h[7]);
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  tc::named_sync(1, kRows);
  if (*abort_flag) return false;
  if (r == 0) {
    tc::fence_after_sync();
    issue(tbase + kColS, kmajor(t.X, kKG), mnmajor(t.w2, kKH2), kKG, id.dh, false);
    issue(tbase + kColW2, mnmajor(t.H1, kKH2), mnmajor(t.X, kKG), kRows, id.w, had_tile);
    tc::mma_commit(bar);
  }
  wait_mma(bar, phase, flags, abort_flag);
  phase ^= 1u;
  tc::fence_after_sync();
  // dz1 = dh1 * m1 -> H1
#pragma unroll
  for (int c = 0; c < kHidden / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) v[jj] = ((m1[c >> 1] >> ((c & 1) * 16 + jj)) & 1u) ? v[jj] : 0.0f;
    uint32_t h[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) h[jj] = pack_bf16x2(v[2 * jj], v[2 * jj + 1]);
    *reinterpret_cast<uint4*>(t.H1 + tile_off(r, 16 * c, kKG)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(t.H1 + tile_off(r, 16 * c + 8, kKG)) = make_uint4(h[4], h[5], h[6], h[7]);
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  tc::named_sync(1, kRows);
  if (*abort_flag) return false;
  if (r == 0) {
    tc::fence_after_sync();
    issue(tbase + kColS, kmajor(t.H1, kKG), mnmajor(t.w1, t.KF), kKG, id.df, false);
    issue(tbase + kColW1, mnmajor(t.Ft, t.KF), mnmajor(t.H1, kKG), kRows, id.w, had_tile);
    tc::mma_commit(bar);
  }
  wait_mma(bar, phase, flags, abort_flag);
  phase ^= 1u;
  tc::fence_after_sync();
  return true;
}

// dL/df_h of the tile (TMEM columns kColS..) into a ring stage, transposed
// [Dp][kRows] FP32.
__device__ __forceinline__ void publish(float* stage, uint32_t trow, int r, int Dp) {
  for (int c = 0; c < Dp / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColS + 16 * c, v);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) stage[(16 * c + jj) * kRows + r] = v[jj];
  }
}

// dL/df_h of the tile (TMEM columns kColS..) straight to global memory, SoA
// [D][ld] FP32 at column `row` (the rows of a warp are consecutive, so each
// feature's stores coalesce).  Warp-collective: every lane takes part in the
// TMEM loads; only valid rows store.
__device__ __forceinline__ void store_dfh(float* __restrict__ dst, uint32_t trow, int D, int Dp, long long ld,
                                          long long row, bool valid) {
  for (int c = 0; c < Dp / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColS + 16 * c, v);
    if (valid) {
#pragma unroll
      for (int jj = 0; jj < 16; ++jj)
        if (16 * c + jj < D) dst[(long long)(16 * c + jj) * ld + row] = v[jj];
    }
  }
}

// Adds the weight gradients accumulated in TMEM (rows = input unit, columns
// = output unit) into mlp_grad (packed as the parameters), one atomic per
// weight.
__device__ __forceinline__ void flush_dw(uint32_t trow, int r, int D, int Dp, int O, float* mlp_grad) {
  float* gW1 = mlp_grad;
  float* gb1 = gW1 + kHidden * D;
  float* gW2 = gb1 + kHidden;
  float* gb2 = gW2 + kHidden * kHidden;
  float* gW3 = gb2 + kHidden;
  float* gb3 = gW3 + O * kHidden;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tc::tmem_ld16(trow + kColW1 + 16 * c, v);
    for (int jj = 0; jj < 16; ++jj) {
      const int o = 16 * c + jj;
      if (r < D) atomicAdd(gW1 + o * D + r, v[jj]);
      else if (r == Dp) atomicAdd(gb1 + o, v[jj]);
    }
    tc::tmem_ld16(trow + kColW2 + 16 * c, v);
    for (int jj = 0; jj < 16; ++jj) {
      const int o = 16 * c + jj;
      if (r < kHidden) atomicAdd(gW2 + o * kHidden + r, v[jj]);
      else if (r == kHidden) atomicAdd(gb2 + o, v[jj]);
    }
  }
  float v[16];
  tc::tmem_ld16(trow + kColW3, v);
  for (int jj = 0; jj < O; ++jj) {
    if (r < kHidden) atomicAdd(gW3 + jj * kHidden + r, v[jj]);
    else if (r == kHidden) atomicAdd(gb3 + jj, v[jj]);
  }
}

// The F = 2 table-gradient scatter of a lane pair's two Gaussians over all
// levels l0 .. l1-1 (scatter2_level_paired; l1 < 0: to the last level).  p
// is this lane's own Gaussian; dfp points at A's column of the transposed
// [D][kRows] dL/df_h stage (B's is the next one); va / vb say whether A / B
// exist; pm names the pair's lanes.
__device__ __forceinline__ void scatter_levels_paired(const Geom& g, float* __restrict__ grad, const Replicas& rp,
                                                      float4 p, const float* dfp, uint32_t xb, bool va, bool vb,
                                                      unsigned int pm, int l0 = 0, int l1 = -1) {
  float4 pa, pb;
  pair_points(p, xb, pm, pa, pb);
  if (l1 < 0) l1 = g.L;
  for (int l = l0; l < l1; ++l) {
    const float2 f0 = *reinterpret_cast<const float2*>(dfp + (2 * l) * kRows);      // (A, B) feature 0
    const float2 f1 = *reinterpret_cast<const float2*>(dfp + (2 * l + 1) * kRows);  // (A, B) feature 1
    scatter2_level_paired(g, l, pa, pb, xb, va, vb, rp.level_base(grad, g, l), f0.x, f1.x, f0.y, f1.y);
  }
}

}  // namespace bwdk
}  // namespace fused
}  // namespace dash
