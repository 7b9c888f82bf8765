// deform_fwd.cu -- a2-a8 fused: 4D hash encoding (Eqs. 8-9) of a tile of
// 128 dynamic Gaussians, the decoder phi_d + heads (Sec. 4.2) on the 5th-gen
// tensor cores, and the optional Eq. 10 update, in one persistent kernel.
//
// A CTA holds G independent groups of 4 warps.  In a group, thread r owns
// Gaussian r of the tile and TMEM lane r: it gathers and interpolates the
// 16 corners of every level in FP32, writes f_h as a BF16 hi+lo operand row
// to shared memory, and after each layer reads its own accumulator row back
// (tcgen05.ld 32x32b), applies ReLU and writes the next operand row.  Thread
// 0 of the group issues the MMAs (M = 128, N = 64 / 64 / 16, BF16 x BF16 ->
// FP32 in TMEM) and commits them to the group's mbarrier.
#include "deform_common.cuh"

namespace dash {
namespace fused {
namespace {

__device__ unsigned int g_fwd_flags;  // bit 0: an MMA completion wait gave up


struct FwdArgs {
  Geom g;
  Pts pts;
  const void* table;
  const float* params;
  int D, Dp, O;
  float* delta;
  long long n_cap;
  uint8_t* state;  // optional per-Gaussian forward state (row stride state_stride(D))
  const float* attrs_in;
  float* attrs_out;
  long long n_all;
  unsigned int* flags;
  int paired;  // F = 2 gathers of the warp-specialised form by lane pairs
  uint32_t off_w2, off_w3, off_a, off_bar;
};

__device__ __forceinline__ bool wait_mma(uint32_t bar, uint32_t phase, unsigned int* flags, volatile int* abort) {
  if (tc::mbar_wait(bar, phase, kWaitIters)) return true;
  atomicOr(flags, 1u);
  *abort = 1;
  return false;
}

// Encodes Gaussian `row` (Eqs. 8-9) into operand row r and keeps a BF16
// copy of f_h in the forward state.
template <typename TT, int F>
__device__ __forceinline__ void encode_row(const FwdArgs& a, bool valid, long long row, uint8_t* A, int r) {
  const float4 p = valid ? load_point(a.pts, row) : make_float4(0.f, 0.f, 0.f, 0.f);
  uint8_t* srow = (valid && a.state != nullptr) ? a.state + row * state_stride(a.D) : nullptr;
  encode_operand_row<TT, F>(a.g, static_cast<const TT*>(a.table), p, valid, a.D, a.Dp, A, r, srow);
}

template <typename TT, int F, int G>
__global__ void __launch_bounds__(G * kRows, 1) deform_fwd_kernel(const __grid_constant__ FwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, grp = tid / kRows, r = tid % kRows, q = (tid >> 5) & 3;
  const int KB1 = 2 * a.Dp + 16;
  uint8_t* w1 = smem;
  uint8_t* w2 = smem + a.off_w2;
  uint8_t* w3 = smem + a.off_w3;
  uint8_t* A = smem + a.off_a + grp * kATileBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(smem + a.off_bar + 8 * G);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_bar + 8 * G + 16);

  // decoder weights -> BF16 operand tiles (bias folded in as an extra column)
  const float* W1 = a.params;
  const float* b1 = W1 + kHidden * a.D;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + a.O * kHidden;
  build_weight_tile(w1, kHidden, KB1, a.Dp, true, a.D, kHidden, W1, b1, tid, blockDim.x);
  build_weight_tile(w2, kHidden, kKH, kHidden, true, kHidden, kHidden, W2, b2, tid, blockDim.x);
  build_weight_tile(w3, kOutPad, kKH, kHidden, true, kHidden, a.O, W3, b3, tid, blockDim.x);
  if (tid < G) {
    tc::mbar_init(tc::smem_addr(&bars[tid]), 1);
    abort_flag[tid] = 0;
  }
  if (tid == 0) tc::mbar_init_fence();
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), G * 64);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;
  const uint32_t tgrp = tbase + (uint32_t)grp * 64u;
  const uint32_t trow = tgrp + ((uint32_t)(q * 32) << 16);
  const uint32_t bar = tc::smem_addr(&bars[grp]);
  uint32_t phase = 0;

  const long long n = point_count(a.pts);
  const long long ntiles = (n + kRows - 1) / kRows;
  for (long long tile = (long long)blockIdx.x * G + grp; tile < ntiles; tile += (long long)gridDim.x * G) {
    const long long row = tile * kRows + r;
    const bool valid = row < n;
    encode_row<TT, F>(a, valid, row, A, r);
    tc::fence_async_smem();
    tc::named_sync(1 + grp, kRows);
    if (abort_flag[grp]) break;
    if (r == 0) {
      tc::fence_after_sync();
      mma_chain(tgrp, A, KB1, w1, KB1, KB1, kHidden);
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag + grp);
    phase ^= 1u;
    tc::fence_after_sync();
    uint32_t m1[2], m2[2];
    hidden_epilogue(trow, A, r, m1);
    tc::fence_before_sync();
    tc::fence_async_smem();
    tc::named_sync(1 + grp, kRows);
    if (abort_flag[grp]) break;
    if (r == 0) {
      tc::fence_after_sync();
      mma_chain(tgrp, A, kKH, w2, kKH, kKH, kHidden);
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag + grp);
    phase ^= 1u;
    tc::fence_after_sync();
    hidden_epilogue(trow, A, r, m2);
    if (valid && a.state != nullptr)
      *reinterpret_cast<uint4*>(a.state + row * state_stride(a.D) + state_mask_off(a.D)) =
          make_uint4(m1[0], m1[1], m2[0], m2[1]);
    tc::fence_before_sync();
    tc::fence_async_smem();
    tc::named_sync(1 + grp, kRows);
    if (abort_flag[grp]) break;
    if (r == 0) {
      tc::fence_after_sync();
      mma_chain(tgrp, A, kKH, w3, kKH, kKH, kOutPad);
      tc::mma_commit(bar);
    }
    wait_mma(bar, phase, a.flags, abort_flag + grp);
    phase ^= 1u;
    tc::fence_after_sync();
    float o[16];
    tc::tmem_ld16(trow, o);
    if (valid) {
      for (int j = 0; j < a.O; ++j) a.delta[(long long)j * a.n_cap + row] = o[j];
      if (a.attrs_out != nullptr) {
        const long long gi = point_row(a.pts, row);
#ifdef DASH_DEBUG
        if (gi >= 0)
#endif
        for (int j = 0; j < a.O; ++j)
          a.attrs_out[(long long)j * a.n_all + gi] = a.attrs_in[(long long)j * a.n_all + gi] + o[j];
      }
    }
    tc::fence_before_sync();
  }
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, G * 64);
}

// ---------------------------------------------------------------------------
// Warp-specialised form.  Warps 0-3 (the consumer, whose thread r owns TMEM
// lane r) run the decoder: wait for a stage of the ring, issue layer 1 from
// it (the MMA's completion releases the stage), then the epilogues and layers
// 2-3 on a private operand tile.  P producer groups of 4 warps gather and
// interpolate: producer group g fills the ring stage of every P-th tile.  The
// latency-bound gathers of the producers overlap the consumer's MMA chain.
// ---------------------------------------------------------------------------
struct WsPlan {
  size_t smem;
  uint32_t off_w2, off_w3, off_ring, off_a2, off_bar, stage_bytes;
};

template <int P, int S>
WsPlan ws_plan(int Dp) {
  WsPlan p;
  const uint32_t KA = 2 * Dp + 16;
  const uint32_t w1 = (uint32_t)kHidden * KA * 2;
  p.off_w2 = (w1 + 127) & ~127u;
  p.off_w3 = p.off_w2 + (uint32_t)kHidden * kKH * 2;
  p.off_ring = (p.off_w3 + (uint32_t)kOutPad * kKH * 2 + 127) & ~127u;
  p.stage_bytes = (uint32_t)kRows * KA * 2;
  p.off_a2 = p.off_ring + S * p.stage_bytes;
  p.off_bar = p.off_a2 + kATileBytes;
  p.smem = p.off_bar + 8 * (2 * S + 1) + 16;
  return p;
}

template <typename TT, int F, int P, int S>
__global__ void __launch_bounds__((P + 1) * kRows, 1) deform_fwd_ws_kernel(const __grid_constant__ FwdArgs a) {
  // tile j uses stage j % S and group j % P; the mbarrier waits tell phases
  // apart only by parity, so no two groups may wait on one stage at once
  static_assert(S >= P, "the ring needs at least one stage per gather group");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int KB1 = 2 * a.Dp + 16;
  uint8_t* w1 = smem;
  uint8_t* w2 = smem + a.off_w2;
  uint8_t* w3 = smem + a.off_w3;
  uint8_t* ring = smem + a.off_a;  // S stages of stage_bytes
  uint8_t* A2 = smem + a.off_a + S * (uint32_t)kRows * KB1 * 2;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  uint64_t* empty = full + S;
  uint64_t* mma_bar = empty + S;
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(mma_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_bar + 1) + 1;
  const uint32_t stage_bytes = (uint32_t)kRows * KB1 * 2;

  const float* W1 = a.params;
  const float* b1 = W1 + kHidden * a.D;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + a.O * kHidden;
  build_weight_tile(w1, kHidden, KB1, a.Dp, true, a.D, kHidden, W1, b1, tid, blockDim.x);
  build_weight_tile(w2, kHidden, kKH, kHidden, true, kHidden, kHidden, W2, b2, tid, blockDim.x);
  build_weight_tile(w3, kOutPad, kKH, kHidden, true, kHidden, a.O, W3, b3, tid, blockDim.x);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(tc::smem_addr(&full[s]), kRows);
      tc::mbar_init(tc::smem_addr(&empty[s]), 1);
    }
    tc::mbar_init(tc::smem_addr(mma_bar), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), 64);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;

  const long long n = point_count(a.pts);
  const long long ntiles = (n + kRows - 1) / kRows;
  const long long my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid < kRows) {
    // ------------------------------------------------ consumer: the decoder
    const int r = tid, q = tid >> 5;
    const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16);
    const uint32_t mb = tc::smem_addr(mma_bar);
    uint32_t phase = 0;
    for (long long j = 0; j < my_tiles; ++j) {
      const int s = (int)(j % S);
      const uint32_t round = (uint32_t)(j / S);
      const long long row = (blockIdx.x + j * gridDim.x) * kRows + r;
      const bool valid = row < n;
      // Eq. 10 inputs of this row, loaded before the wait so that the index
      // and attribute latencies overlap the wait and the three layers
      bool apply = valid && a.attrs_out != nullptr;
      const long long gi = apply ? point_row(a.pts, row) : 0;
#ifdef DASH_DEBUG
      apply = apply && gi >= 0;
#endif
      float ain[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) ain[k] = (apply && k < a.O) ? __ldcs(a.attrs_in + (long long)k * a.n_all + gi) : 0.0f;
      if (!tc::mbar_wait(tc::smem_addr(&full[s]), round & 1u, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      tc::named_sync(1, kRows);
      if (*abort_flag) break;
      if (r == 0) {
        tc::fence_after_sync();
        mma_chain(tbase, ring + s * stage_bytes, KB1, w1, KB1, KB1, kHidden);
        tc::mma_commit(tc::smem_addr(&empty[s]));  // stage free once layer 1 has read it
        tc::mma_commit(mb);
      }
      wait_mma(mb, phase, a.flags, abort_flag);
      phase ^= 1u;
      tc::fence_after_sync();
      uint32_t m1[2], m2[2];
      hidden_epilogue(trow, A2, r, m1);
      tc::fence_before_sync();
      tc::fence_async_smem();
      tc::named_sync(1, kRows);
      if (*abort_flag) break;
      if (r == 0) {
        tc::fence_after_sync();
        mma_chain(tbase, A2, kKH, w2, kKH, kKH, kHidden);
        tc::mma_commit(mb);
      }
      wait_mma(mb, phase, a.flags, abort_flag);
      phase ^= 1u;
      tc::fence_after_sync();
      hidden_epilogue(trow, A2, r, m2);
      if (valid && a.state != nullptr)
        __stcs(reinterpret_cast<uint4*>(a.state + row * state_stride(a.D) + state_mask_off(a.D)),
               make_uint4(m1[0], m1[1], m2[0], m2[1]));
      tc::fence_before_sync();
      tc::fence_async_smem();
      tc::named_sync(1, kRows);
      if (*abort_flag) break;
      if (r == 0) {
        tc::fence_after_sync();
        mma_chain(tbase, A2, kKH, w3, kKH, kKH, kOutPad);
        tc::mma_commit(mb);
      }
      wait_mma(mb, phase, a.flags, abort_flag);
      phase ^= 1u;
      tc::fence_after_sync();
      float o[16];
      tc::tmem_ld16(trow, o);
      if (valid) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (k < a.O) __stcs(a.delta + (long long)k * a.n_cap + row, o[k]);
        if (apply) {
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (k < a.O) __stcs(a.attrs_out + (long long)k * a.n_all + gi, ain[k] + o[k]);
        }
      }
      tc::fence_before_sync();
    }
  } else {
    // ------------------------------------------- producers: Eqs. 8-9 gathers
    const int pg = tid / kRows - 1, r = tid % kRows;
    for (long long j = pg; j < my_tiles; j += P) {
      const int s = (int)(j % S);
      const uint32_t round = (uint32_t)(j / S);
      const long long row = (blockIdx.x + j * gridDim.x) * kRows + r;
      const bool valid = row < n;
      // the point's loads are in flight while this group waits for its stage
      const float4 p = valid ? load_point(a.pts, row) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (!tc::mbar_wait(tc::smem_addr(&empty[s]), (round & 1u) ^ 1u, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      if (*abort_flag) break;
      uint8_t* srow = (valid && a.state != nullptr) ? a.state + row * state_stride(a.D) : nullptr;
      encode_operand_row<TT, F>(a.g, static_cast<const TT*>(a.table), p, valid, a.D, a.Dp, ring + s * stage_bytes, r,
                                srow, a.paired != 0);
      tc::fence_async_smem();
      tc::mbar_arrive(tc::smem_addr(&full[s]));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, 64);
}

template <typename TT, int F, int P, int S>
int launch_ws(FwdArgs a, cudaStream_t st) {
  const WsPlan p = ws_plan<P, S>(a.Dp);
  a.off_w2 = p.off_w2;
  a.off_w3 = p.off_w3;
  a.off_a = p.off_ring;
  a.off_bar = p.off_bar;
  auto kern = deform_fwd_ws_kernel<TT, F, P, S>;
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem)),
                          "cudaFuncSetAttribute(deform_fwd_ws)"))
    return s;
  const long long ntiles = (a.n_cap + kRows - 1) / kRows;
  long long grid = sm_count();  // one persistent CTA per SM (shared memory allows one)
  grid = ntiles < grid ? (ntiles > 0 ? ntiles : 1) : grid;
  kern<<<(unsigned)grid, (P + 1) * kRows, p.smem, st>>>(a);
  return launch_status("deform_fwd_ws_kernel");
}

struct Plan {
  size_t smem;
  uint32_t off_w2, off_w3, off_a, off_bar;
};

template <int G>
Plan plan_for(int Dp) {
  Plan p;
  const uint32_t w1 = (uint32_t)kHidden * (2 * Dp + 16) * 2;
  p.off_w2 = (w1 + 127) & ~127u;
  p.off_w3 = p.off_w2 + (uint32_t)kHidden * kKH * 2;
  p.off_a = (p.off_w3 + (uint32_t)kOutPad * kKH * 2 + 127) & ~127u;
  p.off_bar = p.off_a + (uint32_t)G * kATileBytes;
  p.smem = p.off_bar + 8 * G + 16 + 4 * G + 16;
  return p;
}

template <typename TT, int F, int G>
int launch(FwdArgs a, cudaStream_t st) {
  const Plan p = plan_for<G>(a.Dp);
  a.off_w2 = p.off_w2;
  a.off_w3 = p.off_w3;
  a.off_a = p.off_a;
  a.off_bar = p.off_bar;
  auto kern = deform_fwd_kernel<TT, F, G>;
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem)),
                          "cudaFuncSetAttribute(deform_fwd)"))
    return s;
  int per_sm = 0;
  if (int s = cuda_status(DASH_RT(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G * kRows, p.smem)),
                          "occupancy(deform_fwd)"))
    return s;
  per_sm = per_sm < 1 ? 1 : per_sm;
  while (per_sm * G * 64 > 512) --per_sm;  // TMEM columns per SM
  const long long ntiles = (a.n_cap + kRows - 1) / kRows;
  long long grid = (ntiles + G - 1) / G;
  const long long cap = (long long)per_sm * sm_count();
  grid = grid < cap ? grid : cap;
  kern<<<(unsigned)grid, G * kRows, p.smem, st>>>(a);
  return launch_status("deform_fwd_kernel");
}

template <typename TT>
int dispatch_f(int F, int Dp, int variant, FwdArgs& a, cudaStream_t st) {
  // variant 0: warp-specialised (for F = 2, L*F <= 32: 5 gather groups and 5
  // stages with FP16 tables, 3 and 3 with FP32 tables; otherwise 3 groups, 6
  // stages, 3 when D > 32); 1, 2, 4: the simple form with that many
  // independent groups per CTA
  if (F == 2 && Dp <= 32) {
    // warp-specialised shapes (gather groups, ring stages); 0 = the measured best
    switch (variant) {
      case 0:  // FP32 tables' 8-byte entries need more registers: five groups would spill
        return sizeof(TT) == 4 ? launch_ws<TT, 2, 3, 3>(a, st) : launch_ws<TT, 2, 5, 5>(a, st);
      case 15: return launch_ws<TT, 2, 2, 2>(a, st);
      case 10: return launch_ws<TT, 2, 3, 6>(a, st);
      case 11: return launch_ws<TT, 2, 3, 3>(a, st);
      case 12: return launch_ws<TT, 2, 2, 4>(a, st);
      case 13: return launch_ws<TT, 2, 5, 5>(a, st);
      case 14: return launch_ws<TT, 2, 4, 4>(a, st);
      default: break;
    }
  }
  if (variant == 0 || variant >= 10) {
    if (Dp > 32) {
      switch (F) {
        case 1: return launch_ws<TT, 1, 3, 3>(a, st);
        case 2: return launch_ws<TT, 2, 3, 3>(a, st);
        case 4: return launch_ws<TT, 4, 3, 3>(a, st);
        default: return launch_ws<TT, 8, 3, 3>(a, st);
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
    case 1: return launch<TT, 1, 2>(a, st);
    case 2:
      if (variant == 1) return launch<TT, 2, 1>(a, st);
      if (variant == 4) return launch<TT, 2, 4>(a, st);
      return launch<TT, 2, 2>(a, st);
    case 4: return launch<TT, 4, 2>(a, st);
    default: return launch<TT, 8, 2>(a, st);
  }
}

}  // namespace

unsigned int* fwd_flags_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_fwd_flags) != cudaSuccess) return nullptr;
  return static_cast<unsigned int*>(p);
}

int check_fused_mlp(const dash_mlp* mlp, int D) {
  if (mlp == nullptr || mlp->params == nullptr) return fail(DASH_ERR_INVALID_ARG, "mlp/params is NULL");
  if (mlp->d_in != D) return fail(DASH_ERR_INVALID_ARG, "mlp d_in=%d but L*F=%d", mlp->d_in, D);
  if (D > 64 || mlp->d_hidden != kHidden || mlp->d_out < 1 || mlp->d_out > kOutPad)
    return fail(DASH_ERR_UNSUPPORTED, "fused decoder supports L*F <= 64, H = 64, 1 <= O <= 16");
  return DASH_OK;
}

}  // namespace fused
}  // namespace dash

extern "C" size_t dash_deform_state_size(const dash_mlp* mlp) {
  if (mlp == nullptr || mlp->d_in < 1) return 0;
  return (size_t)dash::fused::state_stride(mlp->d_in);
}

extern "C" int dash_deform_mlp_fwd(const dash_layout* layout, const dash_points* pts, const void* table,
                                   int table_dtype, const dash_mlp* mlp, float* delta_out, void* fwd_state,
                                   const dash_apply* apply, void* stream) {
  DASH_NVTX_RANGE("dash_deform_mlp_fwd");
  using namespace dash;
  using namespace dash::fused;
  FwdArgs a;
  memset(&a, 0, sizeof(a));
  if (int s = make_geom(layout, &a.g)) return s;
  if (int s = make_pts(pts, &a.pts)) return s;
  const int D = a.g.L * a.g.F;
  if (int s = check_fused_mlp(mlp, D)) return s;
  if (a.pts.n == 0) return DASH_OK;
  if (table == nullptr || delta_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "table/delta_out is NULL");
  if ((reinterpret_cast<uintptr_t>(table) & 15u) != 0) return fail(DASH_ERR_INVALID_ARG, "table must be 16-byte aligned");
  if (fwd_state != nullptr && (reinterpret_cast<uintptr_t>(fwd_state) & 15u) != 0)
    return fail(DASH_ERR_INVALID_ARG, "fwd_state must be 16-byte aligned");
  if (apply != nullptr && (apply->attrs_in == nullptr || apply->attrs_out == nullptr || apply->n_all < 1))
    return fail(DASH_ERR_INVALID_ARG, "apply needs attrs_in, attrs_out and n_all >= 1");
  a.table = table;
  a.params = mlp->params;
  a.D = D;
  a.Dp = pad16(D);
  a.O = mlp->d_out;
  a.delta = delta_out;
  a.n_cap = a.pts.n;
  a.state = static_cast<uint8_t*>(fwd_state);
  if (apply != nullptr) {
    a.attrs_in = apply->attrs_in;
    a.attrs_out = apply->attrs_out;
    a.n_all = apply->n_all;
  }
  a.paired = (g_opt_access_form == 0 && a.g.F == 2) ? 1 : 0;
  a.flags = fwd_flags_ptr();
  if (a.flags == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the device flag word");
  cudaStream_t st = as_stream(stream);
  switch (table_dtype) {
    case DASH_F32: return dispatch_f<float>(a.g.F, a.Dp, g_opt_fwd_form, a, st);
    case DASH_F16: return dispatch_f<__half>(a.g.F, a.Dp, g_opt_fwd_form, a, st);
    default: return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", table_dtype);
  }
}
