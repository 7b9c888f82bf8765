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

}  // namespace fused
}  // namespace dash
