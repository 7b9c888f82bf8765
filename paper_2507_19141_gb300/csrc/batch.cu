// batch.cu -- a12: the deformation forward for many scenes x many timestamps
// in one persistent launch, captured once in a CUDA graph and replayed.
//
// Work list: items (scene s, timestamp k, tile of 128 dynamic Gaussians),
// scene-major, then timestamp, then tile, so one scene's tables stay in L2
// while all of its timestamps run (each scene renders K frames with one
// broadcast t per frame, Sec. 5 / Table 3's per-frame rendering).  Counts are
// read from device memory at run time: the captured graph stays valid when a
// scene's dynamic count changes (e.g. written by dash_compact_dynamic).
//
// Each CTA (one per SM) is warp-specialised as in the single-scene forward:
// P gather groups fill an S-stage ring; the decoder group drains it on the
// tensor cores and rebuilds its BF16 weight tiles when the scene changes.
// With a backward the forward also writes each item's per-Gaussian state,
// and a second persistent kernel in the same graph runs the fused backward
// (a9-a10) over the same work list, between a clear of the plan's
// per-scene gradient replicas and their sum into each scene's gradients.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "deform_bwd_common.cuh"

struct dash_batch_plan;

namespace dash {
namespace fused {
namespace {

__device__ unsigned int g_batch_flags;  // bit 0: a bounded wait gave up

constexpr int kMaxScenes = DASH_MAX_SCENES;

struct SceneDev {
  const void* table;
  const float* params;
  const float* x;
  const float* y;
  const float* z;
  const float* ts;
  float* delta;
  long long n_cap;
  int K, pad;
  // backward (NULL without one): upstream gradient [K][O][n_cap], forward
  // state [K][n_cap][state_stride], FP32 table and decoder gradients
  const float* ddelta;
  uint8_t* state;
  float* table_grad;
  float* mlp_grad;
  float* rep_base;  // this scene's gradient replicas (see Replicas), or NULL
};

struct BatchArgs {
  Geom g;
  int D, Dp, O, n_scenes;
  const SceneDev* scenes;
  const long long* counts;
  unsigned int* flags;
  int paired;  // F = 2 gathers by lane pairs (fixed when the plan is created)
  uint32_t off_w2, off_w3, off_ring, off_a2, off_bar, off_tab, stage_bytes;
};

struct Item {
  int s, k;
  long long tile;
};

__device__ __forceinline__ Item decode_item(long long item, const long long* item_off, const long long* tiles,
                                            int n_scenes) {
  int s = 0;
  while (s + 1 < n_scenes && item >= item_off[s + 1]) ++s;
  const long long local = item - item_off[s];
  Item it;
  it.s = s;
  it.k = (int)(local / tiles[s]);
  it.tile = local % tiles[s];
  return it;
}

// The work list: item_off[s] = first item of scene s, tiles[s] = its tiles
// per timestamp (at least one, for decoding), item_off[n_scenes] = the total.
__device__ __forceinline__ void build_item_table(const SceneDev* scenes, const long long* counts, int n_scenes,
                                                 long long* item_off, long long* tiles) {
  long long acc = 0;
  for (int s = 0; s < n_scenes; ++s) {
    long long c = counts[s];
    const long long cap = scenes[s].n_cap;
    c = c < 0 ? 0 : (c > cap ? cap : c);
    const long long t = (c + kRows - 1) / kRows;
    tiles[s] = t > 0 ? t : 1;
    item_off[s] = acc;
    acc += t * (long long)scenes[s].K;  // an empty scene has no items
  }
  item_off[n_scenes] = acc;
}

template <typename TT, int F, int P, int S>
__global__ void __launch_bounds__((P + 1) * kRows, 1) batch_fwd_kernel(const __grid_constant__ BatchArgs a) {
  // tile j uses stage j % S and group j % P; the mbarrier waits tell phases
  // apart only by parity, so no two groups may wait on one stage at once
  static_assert(S >= P, "the ring needs at least one stage per gather group");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int KB1 = 2 * a.Dp + 16;
  uint8_t* w1 = smem;
  uint8_t* w2 = smem + a.off_w2;
  uint8_t* w3 = smem + a.off_w3;
  uint8_t* ring = smem + a.off_ring;
  uint8_t* A2 = smem + a.off_a2;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  uint64_t* empty = full + S;
  uint64_t* mma_bar = empty + S;
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(mma_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_bar + 1) + 1;
  long long* item_off = reinterpret_cast<long long*>(smem + a.off_tab);  // [n_scenes + 1]
  long long* tiles = item_off + kMaxScenes + 1;                           // [n_scenes]

  if (tid == 0) {
    build_item_table(a.scenes, a.counts, a.n_scenes, item_off, tiles);
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(tc::smem_addr(&full[s]), kRows);
      tc::mbar_init(tc::smem_addr(&empty[s]), 1);
    }
    tc::mbar_init(tc::smem_addr(mma_bar), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), 64);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;
  const long long total = item_off[a.n_scenes];
  const long long my_items = total > blockIdx.x ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid < kRows) {
    // ------------------------------------------------ consumer: the decoder
    const int r = tid, q = tid >> 5;
    const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16);
    const uint32_t mb = tc::smem_addr(mma_bar);
    uint32_t phase = 0;
    int cur_scene = -1;
    for (long long j = 0; j < my_items; ++j) {
      const Item it = decode_item(blockIdx.x + j * gridDim.x, item_off, tiles, a.n_scenes);
      const SceneDev& sc = a.scenes[it.s];
      long long cnt = a.counts[it.s];
      cnt = cnt < 0 ? 0 : (cnt > sc.n_cap ? sc.n_cap : cnt);
      if (it.s != cur_scene) {
        // the previous tile's MMAs have completed: the weight tiles are free
        build_forward_weights(w1, w2, w3, sc.params, a.D, a.Dp, a.O, r, kRows);
        tc::fence_async_smem();
        cur_scene = it.s;
      }
      const int s = (int)(j % S);
      const uint32_t round = (uint32_t)(j / S);
      if (!tc::mbar_wait(tc::smem_addr(&full[s]), round & 1u, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      tc::named_sync(1, kRows);
      if (*abort_flag) break;
      if (r == 0) {
        tc::fence_after_sync();
        mma_chain(tbase, ring + s * a.stage_bytes, KB1, w1, KB1, KB1, kHidden);
        tc::mma_commit(tc::smem_addr(&empty[s]));
        tc::mma_commit(mb);
      }
      if (!tc::mbar_wait(mb, phase, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
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
      if (!tc::mbar_wait(mb, phase, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      phase ^= 1u;
      tc::fence_after_sync();
      hidden_epilogue(trow, A2, r, m2);
      const long long row = it.tile * kRows + r;
      if (row < cnt && sc.state != nullptr)  // the ReLU masks of the state (f_h comes from the gather groups)
        __stcs(reinterpret_cast<uint4*>(sc.state + ((long long)it.k * sc.n_cap + row) * state_stride(a.D) +
                                        state_mask_off(a.D)),
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
      if (!tc::mbar_wait(mb, phase, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      phase ^= 1u;
      tc::fence_after_sync();
      float o[16];
      tc::tmem_ld16(trow, o);
      if (row < cnt) {
        float* out = sc.delta + (long long)it.k * a.O * sc.n_cap + row;
        for (int c = 0; c < a.O; ++c) __stcs(out + (long long)c * sc.n_cap, o[c]);
      }
      tc::fence_before_sync();
      tc::named_sync(1, kRows);  // all rows done with the weight tiles before a rebuild
    }
  } else {
    // ------------------------------------------- producers: Eqs. 8-9 gathers
    const int pg = tid / kRows - 1, r = tid % kRows;
    for (long long j = pg; j < my_items; j += P) {
      const Item it = decode_item(blockIdx.x + j * gridDim.x, item_off, tiles, a.n_scenes);
      const SceneDev& sc = a.scenes[it.s];
      long long cnt = a.counts[it.s];
      cnt = cnt < 0 ? 0 : (cnt > sc.n_cap ? sc.n_cap : cnt);
      const int s = (int)(j % S);
      const uint32_t round = (uint32_t)(j / S);
      if (!tc::mbar_wait(tc::smem_addr(&empty[s]), (round & 1u) ^ 1u, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      if (*abort_flag) break;
      const long long row = it.tile * kRows + r;
      const bool valid = row < cnt;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) {
        p.x = clamp01(__ldg(sc.x + row));
        p.y = clamp01(__ldg(sc.y + row));
        p.z = clamp01(__ldg(sc.z + row));
        p.w = clamp01(__ldg(sc.ts + it.k));
      }
      uint8_t* srow = (valid && sc.state != nullptr)
                          ? sc.state + ((long long)it.k * sc.n_cap + row) * state_stride(a.D)
                          : nullptr;
      encode_operand_row<TT, F>(a.g, static_cast<const TT*>(sc.table), p, valid, a.D, a.Dp,
                                ring + s * a.stage_bytes, r, srow, a.paired != 0);
      tc::fence_async_smem();
      tc::mbar_arrive(tc::smem_addr(&full[s]));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, 64);
}

// ---------------------------------------------------------------------------
// The batched backward: the warp-specialised backward of deform_bwd.cu for
// every (scene, timestamp, tile) item.  The decoder group (deform_bwd_common
// .cuh) recomputes the decoder from the item's forward state and back-
// propagates its upstream gradient; when the scene changes it adds its TMEM
// weight-gradient accumulators into the finished scene's mlp_grad and
// rebuilds its weight tiles.  The scatter groups add each tile's lane-paired
// table-gradient reductions into the item's scene.  F = 2, L*F <= 32.
// ---------------------------------------------------------------------------
struct BatchBwdArgs {
  Geom g;
  int D, Dp, O, n_scenes;
  const SceneDev* scenes;
  const long long* counts;
  unsigned int* flags;
  Replicas rep;  // replica layout; each scene's base is SceneDev::rep_base
  uint32_t off_w2, off_w3, off_f, off_h1, off_x, off_g3, off_ring, off_bar, off_tab;
};

template <typename TT, int P, int S>
__global__ void __launch_bounds__((P + 1) * kRows, 1) batch_bwd_kernel(const __grid_constant__ BatchBwdArgs a) {
  // tile j uses stage j % S and group j % P; the mbarrier waits tell phases
  // apart only by parity, so no two groups may wait on one stage at once
  static_assert(S >= P, "the ring needs at least one stage per scatter group");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int KF = 2 * a.Dp + 16;
  const bwdk::Tiles tl{smem,           smem + a.off_w2, smem + a.off_w3, smem + a.off_f, smem + a.off_h1,
                       smem + a.off_x, smem + a.off_g3, KF,              a.D,            a.Dp,
                       a.O};
  float* ring = reinterpret_cast<float*>(smem + a.off_ring);  // S stages of [Dp][kRows]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_bar);
  uint64_t* empty = full + S;
  uint64_t* mma_bar = empty + S;
  volatile uint32_t* holder = reinterpret_cast<volatile uint32_t*>(mma_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_bar + 1) + 1;
  long long* item_off = reinterpret_cast<long long*>(smem + a.off_tab);  // [n_scenes + 1]
  long long* tiles = item_off + kMaxScenes + 1;                           // [n_scenes]
  const int stage_floats = a.Dp * kRows;
  // as in the single-scene backward: when P divides L every scatter group
  // takes every tile and scatters its share of the levels, else whole tiles
  // in turn
  const bool split = a.g.L % P == 0;
  if (tid == 0) {
    build_item_table(a.scenes, a.counts, a.n_scenes, item_off, tiles);
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(tc::smem_addr(&full[s]), kRows);
      tc::mbar_init(tc::smem_addr(&empty[s]), split ? P * kRows : kRows);
    }
    tc::mbar_init(tc::smem_addr(mma_bar), 1);
    tc::mbar_init_fence();
    *abort_flag = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(const_cast<uint32_t*>(holder)), bwdk::kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *holder;
  const long long total = item_off[a.n_scenes];
  const long long my_items = total > blockIdx.x ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid < kRows) {
    // ----------------------------------------------------- decoder group
    const int r = tid, q = tid >> 5;
    const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16);
    const uint32_t bar = tc::smem_addr(mma_bar);
    uint32_t phase = 0;
    bool had_tile = false;
    int cur_scene = -1;
    const bwdk::Ids ids = bwdk::make_ids(a.Dp);
    for (long long j = 0; j < my_items; ++j) {
      const Item it = decode_item(blockIdx.x + j * gridDim.x, item_off, tiles, a.n_scenes);
      const SceneDev& sc = a.scenes[it.s];
      long long cnt = a.counts[it.s];
      cnt = cnt < 0 ? 0 : (cnt > sc.n_cap ? sc.n_cap : cnt);
      if (it.s != cur_scene) {
        // the previous tile's MMAs have completed: its scene's weight
        // gradients are final in TMEM and the weight tiles are free
        if (had_tile && !*abort_flag) bwdk::flush_dw(trow, r, a.D, a.Dp, a.O, a.scenes[cur_scene].mlp_grad);
        tc::named_sync(1, kRows);
        bwdk::build_weights(tl, sc.params, r, kRows);
        cur_scene = it.s;
        had_tile = false;
      }
      const long long row = it.tile * kRows + r;
      const bool valid = row < cnt;
      const uint8_t* srow = valid ? sc.state + ((long long)it.k * sc.n_cap + row) * state_stride(a.D) : nullptr;
      const float* dd = sc.ddelta + (long long)it.k * a.O * sc.n_cap + row;
      if (!bwdk::decoder_tile(tl, ids, tbase, trow, r, bar, phase, a.flags, abort_flag, srow, dd, sc.n_cap, valid,
                              had_tile))
        break;
      had_tile = true;
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
    tc::named_sync(1, kRows);
    tc::fence_after_sync();
    if (had_tile && !*abort_flag) bwdk::flush_dw(trow, r, a.D, a.Dp, a.O, a.scenes[cur_scene].mlp_grad);
  } else {
    // ------------------------------------------------------ scatter groups
    const int pg = tid / kRows - 1, r = tid % kRows;
    const int l0 = split ? pg * a.g.L / P : 0, l1 = split ? (pg + 1) * a.g.L / P : a.g.L;
    for (long long j = split ? 0 : pg; j < my_items; j += split ? 1 : P) {
      const int s = (int)(j % S);
      const uint32_t round = (uint32_t)(j / S);
      const Item it = decode_item(blockIdx.x + j * gridDim.x, item_off, tiles, a.n_scenes);
      const SceneDev& sc = a.scenes[it.s];
      long long cnt = a.counts[it.s];
      cnt = cnt < 0 ? 0 : (cnt > sc.n_cap ? sc.n_cap : cnt);
      const long long row = it.tile * kRows + r;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < cnt) {
        p.x = clamp01(__ldg(sc.x + row));
        p.y = clamp01(__ldg(sc.y + row));
        p.z = clamp01(__ldg(sc.z + row));
        p.w = clamp01(__ldg(sc.ts + it.k));
      }
      if (!tc::mbar_wait(tc::smem_addr(&full[s]), round & 1u, kWaitIters)) {
        atomicOr(a.flags, 1u);
        *abort_flag = 1;
      }
      if (*abort_flag) break;
      const long long row_a = row - (r & 1);  // the pair's even row; both lanes agree on row_a < cnt
      Replicas rep = a.rep;
      rep.base = sc.rep_base;
      if (rep.base == nullptr) rep.levels = 0;
      if (row_a < cnt)
        bwdk::scatter_levels_paired(a.g, sc.table_grad, rep, p, ring + (size_t)s * stage_floats + (r & ~1),
                                    (uint32_t)(r & 1), true, row_a + 1 < cnt, 3u << (r & 30), l0, l1);
      tc::mbar_arrive(tc::smem_addr(&empty[s]));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tbase, bwdk::kTmemCols);
}

// Compiled forms the autotuner chooses from: (gather groups P, ring stages S).
struct Form {
  int P, S;
};
constexpr Form kForms[] = {{4, 4}, {3, 6}, {3, 3}, {2, 4}, {2, 2}, {5, 5}};
constexpr int kNumForms = sizeof(kForms) / sizeof(kForms[0]);

size_t smem_for(int P, int S, int Dp, BatchArgs* a) {
  (void)P;
  const uint32_t KA = 2 * Dp + 16;
  a->off_w2 = ((uint32_t)kHidden * KA * 2 + 127) & ~127u;
  a->off_w3 = a->off_w2 + (uint32_t)kHidden * kKH * 2;
  a->off_ring = (a->off_w3 + (uint32_t)kOutPad * kKH * 2 + 127) & ~127u;
  a->stage_bytes = (uint32_t)kRows * KA * 2;
  a->off_a2 = a->off_ring + S * a->stage_bytes;
  a->off_bar = a->off_a2 + kATileBytes;
  a->off_tab = (a->off_bar + 8 * (2 * S + 1) + 16 + 15) & ~15u;
  return a->off_tab + sizeof(long long) * (2 * kMaxScenes + 1);
}

template <typename TT, int F, int P, int S>
int launch_form(BatchArgs a, cudaStream_t st) {
  const size_t smem = smem_for(P, S, a.Dp, &a);
  if (smem > 227 * 1024) return fail(DASH_ERR_UNSUPPORTED, "batched form P=%d S=%d needs %zu B of shared memory", P, S, smem);
  auto kern = batch_fwd_kernel<TT, F, P, S>;
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)),
                          "cudaFuncSetAttribute(batch)"))
    return s;
  kern<<<(unsigned)sm_count(), (P + 1) * kRows, smem, st>>>(a);
  return launch_status("batch_fwd_kernel");
}

template <typename TT, int F>
int launch_tt_f(int form, BatchArgs& a, cudaStream_t st) {
  switch (form) {
    case 0: return launch_form<TT, F, 4, 4>(a, st);
    case 1: return launch_form<TT, F, 3, 6>(a, st);
    case 2: return launch_form<TT, F, 3, 3>(a, st);
    case 3: return launch_form<TT, F, 2, 4>(a, st);
    case 5: return launch_form<TT, F, 5, 5>(a, st);
    default: return launch_form<TT, F, 2, 2>(a, st);
  }
}

int launch_batch(int form, int table_dtype, BatchArgs& a, cudaStream_t st) {
  if (table_dtype == DASH_F16) {
    switch (a.g.F) {
      case 1: return launch_tt_f<__half, 1>(form, a, st);
      case 2: return launch_tt_f<__half, 2>(form, a, st);
      case 4: return launch_tt_f<__half, 4>(form, a, st);
      default: return launch_tt_f<__half, 8>(form, a, st);
    }
  }
  switch (a.g.F) {
    case 1: return launch_tt_f<float, 1>(form, a, st);
    case 2: return launch_tt_f<float, 2>(form, a, st);
    case 4: return launch_tt_f<float, 4>(form, a, st);
    default: return launch_tt_f<float, 8>(form, a, st);
  }
}

// Compiled forms of the batched backward: (scatter groups P, ring stages S);
// the first is the single-scene default.
constexpr Form kBwdForms[] = {{4, 5}, {2, 2}, {2, 4}, {3, 4}, {3, 3}};
constexpr int kNumBwdForms = sizeof(kBwdForms) / sizeof(kBwdForms[0]);

template <typename TT, int P, int S>
int launch_bwd_form(BatchBwdArgs a, cudaStream_t st) {
  using bwdk::kKG;
  using bwdk::kKH;
  using bwdk::kKH2;
  using bwdk::kKO;
  const int KF = 2 * a.Dp + 16;
  uint32_t off = (uint32_t)kHidden * KF * 2;
  a.off_w2 = (off + 127) & ~127u;
  a.off_w3 = a.off_w2 + (uint32_t)kHidden * kKH2 * 2;
  off = a.off_w3 + (uint32_t)kOutPad * kKH * 2;
  // f_h, h1 and h2 tiles are read transposed with M = 128 rows past their
  // own end into the next region; G3 comes last and is read within bounds
  a.off_f = (off + 127) & ~127u;
  a.off_h1 = a.off_f + (uint32_t)kRows * KF * 2;
  a.off_x = a.off_h1 + (uint32_t)kRows * kKH2 * 2;
  a.off_g3 = a.off_x + (uint32_t)kRows * kKH * 2;
  a.off_ring = a.off_g3 + (uint32_t)kRows * kKO * 2;
  a.off_bar = a.off_ring + (uint32_t)S * a.Dp * kRows * 4;
  a.off_tab = (a.off_bar + 8 * (2 * S + 1) + 16 + 15) & ~15u;
  const size_t smem = a.off_tab + sizeof(long long) * (2 * kMaxScenes + 1);
  if (smem > 227 * 1024) return fail(DASH_ERR_UNSUPPORTED, "batched backward needs %zu B of shared memory", smem);
  auto kern = batch_bwd_kernel<TT, P, S>;
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)),
                          "cudaFuncSetAttribute(batch_bwd)"))
    return s;
  kern<<<(unsigned)sm_count(), (P + 1) * kRows, smem, st>>>(a);
  return launch_status("batch_bwd_kernel");
}

template <typename TT>
int launch_bwd_tt(int form, const BatchBwdArgs& a, cudaStream_t st) {
  switch (form) {
    case 0: return launch_bwd_form<TT, 4, 5>(a, st);
    case 1: return launch_bwd_form<TT, 2, 2>(a, st);
    case 2: return launch_bwd_form<TT, 2, 4>(a, st);
    case 3: return launch_bwd_form<TT, 3, 4>(a, st);
    default: return launch_bwd_form<TT, 3, 3>(a, st);
  }
}

int launch_batch_bwd(int form, int table_dtype, const BatchBwdArgs& a, cudaStream_t st) {
  return table_dtype == DASH_F16 ? launch_bwd_tt<__half>(form, a, st) : launch_bwd_tt<float>(form, a, st);
}

}  // namespace

unsigned int* batch_flags_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_batch_flags) != cudaSuccess) return nullptr;
  return static_cast<unsigned int*>(p);
}

}  // namespace fused
}  // namespace dash

struct dash_batch_plan {
  int device;
  int table_dtype;
  int form;
  int bform;  // backward form (plans with a backward)
  int with_bwd;
  dash::fused::BatchArgs args;
  dash::fused::BatchBwdArgs bargs;
  dash::fused::SceneDev* d_scenes;
  long long* d_counts;
  float* d_rep;      // gradient replicas of every scene (plans with a backward), or NULL
  size_t rep_bytes;  // per scene
  std::vector<dash::fused::SceneDev> h_scenes;  // host copy (gradient pointers for the autotuner)
  long long grad_floats;                         // table entries * F per scene
  long long param_floats;                        // decoder parameters per scene
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  std::string signature;
};

namespace {

void destroy_graph(dash_batch_plan* p) {
  if (p->exec != nullptr) cudaGraphExecDestroy(p->exec);
  if (p->graph != nullptr) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

// One warm-up launch, then the mean of three timed launches on st.
template <typename Launch>
int time_form(Launch launch, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  using namespace dash;
  int rc = launch();
  if (rc != DASH_OK) return rc;
  rc = cuda_status(DASH_RT(cudaEventRecord(e0, st)), "cudaEventRecord");
  for (int rep = 0; rep < 3 && rc == DASH_OK; ++rep) rc = launch();
  if (rc == DASH_OK) rc = cuda_status(DASH_RT(cudaEventRecord(e1, st)), "cudaEventRecord");
  if (rc == DASH_OK) rc = cuda_status(DASH_RT(cudaEventSynchronize(e1)), "cudaEventSynchronize");
  if (rc == DASH_OK) rc = cuda_status(DASH_RT(cudaEventElapsedTime(ms, e0, e1)), "cudaEventElapsedTime");
  return rc;
}

// Captures one launch of the current form into a graph on a private stream.
int capture(dash_batch_plan* p) {
  using namespace dash;
  destroy_graph(p);
  cudaStream_t cs = nullptr;
  if (int s = cuda_status(DASH_RT(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)), "cudaStreamCreate")) return s;
  int rc = cuda_status(DASH_RT(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)), "cudaStreamBeginCapture");
  if (rc == DASH_OK) {
    int lr = fused::launch_batch(p->form, p->table_dtype, p->args, cs);
    if (lr == DASH_OK && p->with_bwd) {
      const Replicas& rep = p->bargs.rep;
      if (p->d_rep != nullptr)
        lr = cuda_status(DASH_RT(cudaMemsetAsync(p->d_rep, 0, p->rep_bytes * p->h_scenes.size(), cs)), "cudaMemsetAsync");
      if (lr == DASH_OK) lr = fused::launch_batch_bwd(p->bform, p->table_dtype, p->bargs, cs);
      for (size_t s = 0; lr == DASH_OK && p->d_rep != nullptr && s < p->h_scenes.size(); ++s) {
        Replicas r = rep;
        r.base = p->h_scenes[s].rep_base;
        lr = replica_sum(p->bargs.g, r, p->h_scenes[s].table_grad, cs);
      }
    }
    const int er = cuda_status(cudaStreamEndCapture(cs, &p->graph), "cudaStreamEndCapture");
    rc = lr != DASH_OK ? lr : er;
  }
  if (rc == DASH_OK) rc = cuda_status(DASH_RT(cudaGraphInstantiate(&p->exec, p->graph, 0)), "cudaGraphInstantiate");
  cudaStreamDestroy(cs);
  if (rc != DASH_OK) destroy_graph(p);
  return rc;
}

}  // namespace

extern "C" {

int dash_batch_plan_create(const dash_batch_desc* desc, dash_batch_plan** out) {
  DASH_NVTX_RANGE("dash_batch_plan_create");
  using namespace dash;
  if (out == nullptr || desc == nullptr || desc->scenes == nullptr) return fail(DASH_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (desc->n_scenes < 1 || desc->n_scenes > DASH_MAX_SCENES)
    return fail(DASH_ERR_UNSUPPORTED, "n_scenes=%d outside [1, %d]", desc->n_scenes, DASH_MAX_SCENES);
  if (!(desc->table_dtype == DASH_F16 || desc->table_dtype == DASH_F32))
    return fail(DASH_ERR_UNSUPPORTED, "table_dtype %d (F32 or F16)", desc->table_dtype);
  fused::BatchArgs a;
  memset(&a, 0, sizeof(a));
  if (int s = make_geom(desc->layout, &a.g)) return s;
  const int D = a.g.L * a.g.F;
  if (desc->d_in != D) return fail(DASH_ERR_INVALID_ARG, "d_in=%d but L*F=%d", desc->d_in, D);
  if (D > 64 || desc->d_hidden != fused::kHidden || desc->d_out < 1 || desc->d_out > fused::kOutPad)
    return fail(DASH_ERR_UNSUPPORTED, "fused decoder supports L*F <= 64, H = 64, 1 <= O <= 16");
  a.D = D;
  a.Dp = fused::pad16(D);
  a.O = desc->d_out;
  a.n_scenes = desc->n_scenes;
  a.paired = (g_opt_access_form == 0 && a.g.F == 2) ? 1 : 0;
  a.flags = fused::batch_flags_ptr();
  if (a.flags == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the device flag word");
  const bool with_bwd = desc->with_backward != 0;
  if (with_bwd && (a.g.F != 2 || D > 32))
    return fail(DASH_ERR_UNSUPPORTED, "the batched backward supports F = 2 and L*F <= 32");
  fused::SceneDev host[DASH_MAX_SCENES];
  long long counts[DASH_MAX_SCENES];
  long long total_n = 0, total_k = 0;
  for (int s = 0; s < desc->n_scenes; ++s) {
    const dash_batch_scene& sc = desc->scenes[s];
    if (sc.n < 0 || sc.K < 1) return fail(DASH_ERR_INVALID_ARG, "scene %d: n < 0 or K < 1", s);
    if (sc.table == nullptr || sc.params == nullptr || sc.x == nullptr || sc.y == nullptr || sc.z == nullptr ||
        sc.timestamps == nullptr || sc.delta_out == nullptr)
      return fail(DASH_ERR_INVALID_ARG, "scene %d: NULL pointer", s);
    if ((reinterpret_cast<uintptr_t>(sc.table) & 15u) != 0)
      return fail(DASH_ERR_INVALID_ARG, "scene %d: table must be 16-byte aligned", s);
    host[s] = fused::SceneDev{sc.table, sc.params, sc.x, sc.y, sc.z, sc.timestamps, sc.delta_out, sc.n, sc.K, 0,
                              nullptr, nullptr, nullptr, nullptr, nullptr};
    if (with_bwd) {
      if (sc.ddelta == nullptr || sc.fwd_state == nullptr || sc.table_grad == nullptr || sc.mlp_grad == nullptr)
        return fail(DASH_ERR_INVALID_ARG, "scene %d: a backward pointer is NULL", s);
      if ((reinterpret_cast<uintptr_t>(sc.fwd_state) & 15u) != 0 || (reinterpret_cast<uintptr_t>(sc.table_grad) & 15u) != 0)
        return fail(DASH_ERR_INVALID_ARG, "scene %d: fwd_state and table_grad must be 16-byte aligned", s);
      host[s].ddelta = sc.ddelta;
      host[s].state = static_cast<uint8_t*>(sc.fwd_state);
      host[s].table_grad = sc.table_grad;
      host[s].mlp_grad = sc.mlp_grad;
    }
    counts[s] = sc.n;
    total_n += sc.n;
    total_k += sc.K;
  }
  dash_batch_plan* p = new dash_batch_plan();
  p->device = 0;
  cudaGetDevice(&p->device);
  p->table_dtype = desc->table_dtype;
  p->grad_floats = desc->layout->offset[a.g.L] * a.g.F;
  p->param_floats = (long long)fused::kHidden * D + fused::kHidden + (long long)fused::kHidden * fused::kHidden +
                    fused::kHidden + (long long)a.O * fused::kHidden + a.O;
  p->form = 0;
  p->bform = 0;
  p->with_bwd = with_bwd ? 1 : 0;
  p->d_scenes = nullptr;
  p->d_counts = nullptr;
  p->graph = nullptr;
  p->exec = nullptr;
  p->d_rep = nullptr;
  p->rep_bytes = 0;
  int rc = DASH_OK;
  // replicas of the coarsest dense levels' gradients, one set per scene
  // (the backward's scatter is lane-paired)
  Replicas rep;
  memset(&rep, 0, sizeof(rep));
  if (with_bwd) {
    rep = replica_plan(desc->layout, g_opt_grad_replicas, &p->rep_bytes);
    if (rep.levels > 0) {
      rc = cuda_status(DASH_RT(cudaMalloc(&p->d_rep, p->rep_bytes * desc->n_scenes)), "cudaMalloc");
      for (int s = 0; rc == DASH_OK && s < desc->n_scenes; ++s)
        host[s].rep_base = reinterpret_cast<float*>(reinterpret_cast<char*>(p->d_rep) + p->rep_bytes * s);
    }
  }
  p->h_scenes.assign(host, host + desc->n_scenes);
  if (rc == DASH_OK) rc = cuda_status(DASH_RT(cudaMalloc(&p->d_scenes, sizeof(fused::SceneDev) * desc->n_scenes)), "cudaMalloc");
  if (rc == DASH_OK) rc = cuda_status(DASH_RT(cudaMalloc(&p->d_counts, sizeof(long long) * desc->n_scenes)), "cudaMalloc");
  if (rc == DASH_OK)
    rc = cuda_status(DASH_RT(cudaMemcpy(p->d_scenes, host, sizeof(fused::SceneDev) * desc->n_scenes, cudaMemcpyHostToDevice)),
                     "cudaMemcpy");
  if (rc == DASH_OK)
    rc = cuda_status(DASH_RT(cudaMemcpy(p->d_counts, counts, sizeof(long long) * desc->n_scenes, cudaMemcpyHostToDevice)),
                     "cudaMemcpy");
  if (rc == DASH_OK) {
    a.scenes = p->d_scenes;
    a.counts = p->d_counts;
    p->args = a;
    fused::BatchBwdArgs b;
    memset(&b, 0, sizeof(b));
    b.g = a.g;
    b.D = a.D, b.Dp = a.Dp, b.O = a.O, b.n_scenes = a.n_scenes;
    b.scenes = a.scenes;
    b.counts = a.counts;
    b.flags = a.flags;
    b.rep = rep;
    p->bargs = b;
    char sig[512];
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->device);
    snprintf(sig, sizeof(sig), "%s|L%d F%d T%d D%d O%d|dt%d|S%d N%lld K%lld%s", prop.name, a.g.L, a.g.F,
             desc->layout->log2_T, D, a.O, desc->table_dtype, desc->n_scenes, total_n, total_k,
             with_bwd ? "|bwd" : "");
    p->signature = sig;
    rc = capture(p);
  }
  if (rc != DASH_OK) {
    dash_batch_plan_destroy(p);
    return rc;
  }
  *out = p;
  return DASH_OK;
}

int64_t* dash_batch_counts(dash_batch_plan* plan) {
  return plan == nullptr ? nullptr : reinterpret_cast<int64_t*>(plan->d_counts);
}

int dash_batch_run(dash_batch_plan* plan, void* stream) {
  DASH_NVTX_RANGE("dash_batch_run");
  using namespace dash;
  if (plan == nullptr || plan->exec == nullptr) return fail(DASH_ERR_INVALID_ARG, "plan is NULL or not instantiated");
  return cuda_status(DASH_RT(cudaGraphLaunch(plan->exec, as_stream(stream))), "cudaGraphLaunch");
}

int dash_batch_plan_destroy(dash_batch_plan* plan) {
  if (plan == nullptr) return DASH_OK;
  destroy_graph(plan);
  if (plan->d_scenes != nullptr) cudaFree(plan->d_scenes);
  if (plan->d_rep != nullptr) cudaFree(plan->d_rep);
  if (plan->d_counts != nullptr) cudaFree(plan->d_counts);
  delete plan;
  return DASH_OK;
}

int dash_batch_form(const dash_batch_plan* plan) { return plan == nullptr ? -1 : plan->form + 16 * plan->bform; }

int dash_batch_autotune(dash_batch_plan* plan, const char* cache_json_path, void* stream) {
  DASH_NVTX_RANGE("dash_batch_autotune");
  using namespace dash;
  if (plan == nullptr) return fail(DASH_ERR_INVALID_ARG, "plan is NULL");
  const std::string key = "\"" + plan->signature + "\": ";
  std::string cache;
  if (cache_json_path != nullptr) {
    if (FILE* f = fopen(cache_json_path, "rb")) {
      char buf[4096];
      size_t k;
      while ((k = fread(buf, 1, sizeof(buf), f)) > 0) cache.append(buf, k);
      fclose(f);
    }
    const size_t at = cache.find(key);
    if (at != std::string::npos) {
      // the entry: forward form + 16 * backward form
      const int code = atoi(cache.c_str() + at + key.size());
      const int form = code % 16, bform = code / 16;
      if (code >= 0 && form < fused::kNumForms && bform < fused::kNumBwdForms && (plan->with_bwd || bform == 0)) {
        if (form != plan->form || bform != plan->bform) {
          plan->form = form;
          plan->bform = bform;
          return capture(plan);
        }
        return DASH_OK;
      }
    }
  }
  // time every compiled form on this plan's work: one warm-up and three timed runs each
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  if (int s = cuda_status(DASH_RT(cudaEventCreate(&e0)), "cudaEventCreate")) return s;
  if (int s = cuda_status(DASH_RT(cudaEventCreate(&e1)), "cudaEventCreate")) {
    cudaEventDestroy(e0);
    return s;
  }
  int rc = DASH_OK;
  int best = plan->form;
  float best_ms = 1e30f;
  for (int form = 0; form < fused::kNumForms && rc == DASH_OK; ++form) {
    float ms = 0.0f;
    const int lr = time_form([&] { return fused::launch_batch(form, plan->table_dtype, plan->args, st); }, st, e0,
                             e1, &ms);
    if (lr == DASH_ERR_UNSUPPORTED) continue;  // does not fit this shape
    rc = lr;
    if (rc == DASH_OK && ms < best_ms) {
      best_ms = ms;
      best = form;
    }
  }
  if (rc == DASH_OK) plan->form = best;
  if (rc == DASH_OK && plan->with_bwd) {
    // the backward forms run on the state of one forward; every run adds
    // into the caller's gradients, so those are saved first and put back
    const long long per = plan->grad_floats + plan->param_floats;
    const int ns = (int)plan->h_scenes.size();
    float* saved = nullptr;
    rc = cuda_status(DASH_RT(cudaMalloc(&saved, sizeof(float) * per * ns)), "cudaMalloc");
    for (int s = 0; s < ns && rc == DASH_OK; ++s) {
      const fused::SceneDev& sc = plan->h_scenes[s];
      rc = cuda_status(DASH_RT(cudaMemcpyAsync(saved + s * per, sc.table_grad, sizeof(float) * plan->grad_floats,
                                       cudaMemcpyDeviceToDevice, st)), "cudaMemcpyAsync");
      if (rc == DASH_OK)
        rc = cuda_status(DASH_RT(cudaMemcpyAsync(saved + s * per + plan->grad_floats, sc.mlp_grad,
                                         sizeof(float) * plan->param_floats, cudaMemcpyDeviceToDevice, st)),
                         "cudaMemcpyAsync");
    }
    if (rc == DASH_OK) rc = fused::launch_batch(plan->form, plan->table_dtype, plan->args, st);
    int bbest = plan->bform;
    best_ms = 1e30f;
    for (int form = 0; form < fused::kNumBwdForms && rc == DASH_OK; ++form) {
      float ms = 0.0f;
      const int lr = time_form([&] { return fused::launch_batch_bwd(form, plan->table_dtype, plan->bargs, st); },
                               st, e0, e1, &ms);
      if (lr == DASH_ERR_UNSUPPORTED) continue;
      rc = lr;
      if (rc == DASH_OK && ms < best_ms) {
        best_ms = ms;
        bbest = form;
      }
    }
    for (int s = 0; s < ns && saved != nullptr; ++s) {  // put the gradients back, also after an error
      const fused::SceneDev& sc = plan->h_scenes[s];
      const int r1 = cuda_status(DASH_RT(cudaMemcpyAsync(sc.table_grad, saved + s * per, sizeof(float) * plan->grad_floats,
                                                 cudaMemcpyDeviceToDevice, st)), "cudaMemcpyAsync");
      const int r2 = cuda_status(DASH_RT(cudaMemcpyAsync(sc.mlp_grad, saved + s * per + plan->grad_floats,
                                                 sizeof(float) * plan->param_floats, cudaMemcpyDeviceToDevice, st)),
                                 "cudaMemcpyAsync");
      if (rc == DASH_OK) rc = r1 != DASH_OK ? r1 : r2;
    }
    if (saved != nullptr) {
      const int r = cuda_status(DASH_RT(cudaStreamSynchronize(st)), "cudaStreamSynchronize");
      if (rc == DASH_OK) rc = r;
      cudaFree(saved);
    }
    if (rc == DASH_OK) plan->bform = bbest;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DASH_OK) return rc;
  const int code = plan->form + 16 * plan->bform;
  if (cache_json_path != nullptr) {
    // keep the other entries; replace or append this signature
    std::string body;
    const size_t lb = cache.find('{'), rb = cache.rfind('}');
    if (lb != std::string::npos && rb != std::string::npos && rb > lb) body = cache.substr(lb + 1, rb - lb - 1);
    std::string entries;
    size_t pos = 0;
    while (pos < body.size()) {
      size_t nl = body.find('\n', pos);
      if (nl == std::string::npos) nl = body.size();
      std::string line = body.substr(pos, nl - pos);
      pos = nl + 1;
      while (!line.empty() && (line.back() == ',' || line.back() == ' ' || line.back() == '\r')) line.pop_back();
      const size_t first = line.find_first_not_of(' ');
      if (first == std::string::npos || line.find(key) != std::string::npos) continue;
      entries += "  " + line.substr(first) + ",\n";
    }
    char mine[512];
    snprintf(mine, sizeof(mine), "  %s%d\n", key.c_str(), code);
    if (FILE* f = fopen(cache_json_path, "wb")) {
      fprintf(f, "{\n%s%s}\n", entries.c_str(), mine);
      fclose(f);
    }
  }
  return capture(plan);
}

}  // extern "C"
