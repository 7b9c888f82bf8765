// deform_common.cuh -- operand tiles shared by the fused deformation kernels
// (encoder + decoder MLP of Sec. 4.2 on the tensor cores).
//
// Every operand tile is BF16 in the no-swizzle core-matrix layout of
// tc_ptx.cuh with LBO = 128 bytes (K-adjacent core matrices contiguous) and
// SBO = K * 16 bytes (one 8-row group = K/8 core matrices).
//
// Activation tiles hold 128 rows (one per Gaussian of the tile).  A decoder
// layer  z = W a + b  is evaluated as one K-major MMA chain by appending a
// constant-one column to the activations and the bias as an extra weight
// column.  Where the pre-activations must be accurate (they decide the ReLU
// masks the backward pass uses) activations are split into a BF16 "hi" part
// and a BF16 "lo" remainder (a = hi + lo to ~16 bits) that both multiply the
// same weights:  K = [hi (Kd) | 1, 0 x 15 | lo (Kd)].  The ones column sits
// right after hi so that, read transposed (rows = K slots), it is row Kd < 128.
#pragma once

#include "dash_internal.cuh"
#include "tc_ptx.cuh"

namespace dash {
namespace fused {

constexpr int kRows = 128;        // Gaussians per tile = MMA M
constexpr int kHidden = 64;       // H of the decoder
constexpr int kOutPad = 16;       // O padded to the MMA N granule
constexpr uint32_t kWaitIters = 1u << 22;

// Per-Gaussian forward state kept for the backward pass: f_h as BF16 (D
// values) and the two ReLU masks of the forward's accurate pre-activations
// (2 x 64 bits) at byte offset state_mask_off(D); row stride state_stride(D).
__host__ __device__ constexpr int state_mask_off(int D) { return (2 * D + 15) / 16 * 16; }
__host__ __device__ constexpr int state_stride(int D) { return state_mask_off(D) + 16; }

__host__ __device__ constexpr int pad16(int v) { return (v + 15) / 16 * 16; }

// Byte offset of element (r, k) in a tile whose K extent is `K`.
__host__ __device__ constexpr uint32_t tile_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Splits v[0..8) into hi = bf16(v) and lo = bf16(v - hi), packed 8 per uint4.
__device__ __forceinline__ void split_hi_lo8(const float v[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    const float r0 = v[2 * j] - __low2float(hb);
    const float r1 = v[2 * j + 1] - __high2float(hb);
    h[j] = *reinterpret_cast<uint32_t*>(&hb);
    l[j] = pack_bf16x2(r0, r1);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Writes the constant-one column at k = kones (and zeros up to kones + 16) of row r.
__device__ __forceinline__ void write_ones(uint8_t* tile, int r, int kones, int K) {
  const uint32_t one = 0x3F80u;  // BF16 1.0 in the low half
  *reinterpret_cast<uint4*>(tile + tile_off(r, kones, K)) = make_uint4(one, 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(tile + tile_off(r, kones + 8, K)) = make_uint4(0u, 0u, 0u, 0u);
}

// Builds a weight tile B[n][k] (N rows x KB) of  z = W a + b:
//   k < Kd: W[n][k] (0 beyond the real width kin); k = Kd: bias b[n];
//   Kd < k < Kd + 16: 0; with `dup`, Kd + 16 <= k < 2 Kd + 16 repeats W for
//   the lo operand part.  Rows n >= nout are zero.  W is row-major [nout][kin].
__device__ __forceinline__ void build_weight_tile(uint8_t* tile, int N, int KB, int Kd, bool dup, int kin, int nout,
                                                  const float* __restrict__ W, const float* __restrict__ b,
                                                  int tid, int nthreads) {
  for (int e = tid; e < N * KB; e += nthreads) {
    const int n = e / KB, k = e % KB;
    float v = 0.0f;
    if (n < nout) {
      int kk = -1;
      if (k < Kd) kk = k;
      else if (dup && k >= Kd + 16 && k < 2 * Kd + 16) kk = k - Kd - 16;
      if (kk >= 0) v = kk < kin ? __ldg(W + (size_t)n * kin + kk) : 0.0f;
      else if (k == Kd) v = __ldg(b + n);
    }
    *reinterpret_cast<__nv_bfloat16*>(tile + tile_off(n, k, KB)) = __float2bfloat16_rn(v);
  }
}

// Issues C[tmem] = A * B^T over K (multiple of 16) for K-major A (M = 128)
// and B (N rows); one thread.
__device__ __forceinline__ void mma_chain(uint32_t tmem, const uint8_t* A, int KA, const uint8_t* B, int KB, int K,
                                          int N) {
  const uint32_t idesc = tc::idesc_bf16(kRows, N, 0, 0);
  const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
  for (int k = 0; k < K; k += 16) {
    const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(k / 8) * 128u, 128u, (uint32_t)KA * 16u);
    const uint64_t bd = tc::smem_desc(b0 + (uint32_t)(k / 8) * 128u, 128u, (uint32_t)KB * 16u);
    tc::mma_bf16(tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
  }
}

constexpr int kKH = 2 * kHidden + 16;              // hidden-layer operand K (hi | ones | lo)
constexpr uint32_t kATileBytes = kRows * kKH * 2;  // 36,864 B

// Eqs. 8-9 for one point p into operand row r (K = [hi | 1 | lo], FP32
// interpolation split into BF16 hi + lo); with state_row, also the BF16 copy
// of f_h for the backward.  Invalid rows are zero features.  With `paired`
// (F = 2; uniform over the warp) the gathers are issued by lane pairs
// (gather2_level_paired) and give the same features bit for bit; both lanes
// of every pair must then call this.
template <typename TT, int F>
__device__ __forceinline__ void encode_operand_row(const Geom& g, const TT* __restrict__ table, float4 p, bool valid,
                                                   int D, int Dp, uint8_t* A, int r, uint8_t* state_row,
                                                   bool paired = false) {
  const int KA = 2 * Dp + 16;
  constexpr int kLevelsPerChunk = 8 / F;
  const int nchunks = Dp / 8;
  const uint32_t lane = threadIdx.x & 31u, xb = lane & 1u;
  const unsigned int pm = 3u << (lane & 30u);
  float4 pa = p, pb = p;
  bool live = valid;
  if constexpr (F == 2) {
    if (paired) {
      pair_points(p, xb, pm, pa, pb);
      live = __shfl_xor_sync(pm, valid ? 1 : 0, 1) != 0 || valid;  // either Gaussian of the pair exists
    }
  }
  for (int c = 0; c < nchunks; ++c) {
    float v[8];
#pragma unroll
    for (int j = 0; j < kLevelsPerChunk; ++j) {
      const int l = c * kLevelsPerChunk + j;
      float acc[F];
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] = 0.0f;
      if constexpr (F == 2) {
        if (paired) {
          if (live && l < g.L) {
            gather2_level_paired<TT>(g, l, pa, pb, xb, table + g.offset[l] * 2, pm, acc);
            if (!valid) acc[0] = acc[1] = 0.0f;
          }
#pragma unroll
          for (int f = 0; f < F; ++f) v[j * F + f] = acc[f];
          continue;
        }
      }
      if (valid && l < g.L) {
        uint32_t idx[16];
        float w[16];
        level_corners(g, l, p, idx, w);
        const TT* base = table + g.offset[l] * F;
        if constexpr (F == 2) {
          gather2_pairs<TT>(base, idx, w, acc);
        } else {
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            float e[F];
            load_entry<TT, F>(base + (size_t)idx[b] * F, e);
#pragma unroll
            for (int f = 0; f < F; ++f) acc[f] = fmaf(w[b], e[f], acc[f]);
          }
        }
      }
#pragma unroll
      for (int f = 0; f < F; ++f) v[j * F + f] = acc[f];
    }
    uint4 hi, lo;
    split_hi_lo8(v, hi, lo);
    *reinterpret_cast<uint4*>(A + tile_off(r, 8 * c, KA)) = hi;
    *reinterpret_cast<uint4*>(A + tile_off(r, Dp + 16 + 8 * c, KA)) = lo;
    if (state_row != nullptr && 8 * c < D) {
      __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(state_row) + 8 * c;
      if ((D & 7) == 0) {
        __stcs(reinterpret_cast<uint4*>(dst), hi);
      } else {
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&hi);
        for (int j = 0; j < 8 && 8 * c + j < D; ++j) dst[j] = h[j];
      }
    }
  }
  write_ones(A, r, Dp, KA);
}

// Reads this thread's 64 hidden pre-activations from TMEM, records their
// ReLU mask (bit j of mask[j / 32]), applies ReLU and writes the next
// layer's operand row [hi | 1 | lo].
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, uint8_t* A, int r, uint32_t mask[2]) {
  mask[0] = mask[1] = 0u;
#pragma unroll
  for (int c = 0; c < kHidden / 16; ++c) {
    float v[16];
    tc::tmem_ld16(trow + 16 * c, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (v[j] > 0.0f) mask[c >> 1] |= 1u << ((c & 1) * 16 + j);
      v[j] = fmaxf(v[j], 0.0f);
    }
    uint4 h0, l0, h1, l1;
    split_hi_lo8(v, h0, l0);
    split_hi_lo8(v + 8, h1, l1);
    *reinterpret_cast<uint4*>(A + tile_off(r, 16 * c, kKH)) = h0;
    *reinterpret_cast<uint4*>(A + tile_off(r, 16 * c + 8, kKH)) = h1;
    *reinterpret_cast<uint4*>(A + tile_off(r, kHidden + 16 + 16 * c, kKH)) = l0;
    *reinterpret_cast<uint4*>(A + tile_off(r, kHidden + 16 + 16 * c + 8, kKH)) = l1;
  }
  write_ones(A, r, kHidden, kKH);
}

// Decoder weights -> BF16 operand tiles in shared memory (hi | 1 | lo
// layout for the forward; bias folded in as a weight column).
__device__ __forceinline__ void build_forward_weights(uint8_t* w1, uint8_t* w2, uint8_t* w3, const float* params,
                                                      int D, int Dp, int O, int tid, int nthreads) {
  const float* W1 = params;
  const float* b1 = W1 + kHidden * D;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + O * kHidden;
  build_weight_tile(w1, kHidden, 2 * Dp + 16, Dp, true, D, kHidden, W1, b1, tid, nthreads);
  build_weight_tile(w2, kHidden, kKH, kHidden, true, kHidden, kHidden, W2, b2, tid, nthreads);
  build_weight_tile(w3, kOutPad, kKH, kHidden, true, kHidden, O, W3, b3, tid, nthreads);
}

}  // namespace fused
}  // namespace dash
