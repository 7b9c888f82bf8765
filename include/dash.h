/*
 * dash.h -- C ABI of libdash, the GB300 (sm_103a) implementation of the DASH
 * 4D-hash deformation path (arXiv 2507.19141, Sec. 4.2-4.3, Eqs. 7-11) and
 * of the steps on either side of it: the static/dynamic decomposition that
 * produces the mask (Sec. 4.1, Eqs. 3-5), the hash-table occupancy behind
 * the collision argument (Sec. 4.2, Sec. 5 "w/o dec"), and the 3D Gaussian
 * splatting renderer the deformed Gaussians are drawn with (Sec. 3, Eqs. 1-2).
 *
 * Sections below, in order: status and layouts; utilities; compaction (a1);
 * the 4-D encoder alone (a2-a6, a10); table occupancy; the fused
 * deformation forward (a2-a8) and backward (a9-a11) with the Eq. 10
 * backward; the decomposition (Eqs. 3-5); the renderer; the batched
 * persistent form (a12); the plain FP32 baseline forms.
 *
 * Conventions shared by every entry point
 *   - All pointers are DEVICE pointers unless a comment says "host".
 *   - The caller owns all memory.  Nothing here allocates device memory
 *     except dash_batch_plan_create (the plan's descriptors, graph and
 *     gradient replicas);
 *     scratch comes from caller workspaces sized by the *_workspace_size
 *     calls.
 *   - Every call is asynchronous on the CUDA stream passed as `void* stream`
 *     (a cudaStream_t; NULL = the legacy default stream).  Nothing
 *     synchronises; a kernel fault surfaces at the caller's next sync.
 *   - Every call returns a dash_status.  No exception crosses the ABI.
 *     dash_last_error() returns a thread-local message for the last failure.
 *   - Gradient outputs are ACCUMULATED (+=); the caller zeroes them.
 *   - Coordinates are normalised to [0,1]: values outside are clamped, NaN
 *     maps to 0.
 *   - Feature layout: f_h[i][l*F + f] (levels concatenated, Eq. 9).
 *   - Table layout: entry-major [offset[L]][F]; level l occupies entries
 *     [offset[l], offset[l] + size[l]).
 *   - Decoder parameters (FP32, packed): W1 [H][D], b1 [H], W2 [H][H], b2 [H],
 *     W3 [O][H], b3 [O] with D = L*F; gradients use the same packing.
 *   - Deformation output: SoA delta[k][i], k = 0-2 position, 3-6 rotation,
 *     7-9 scale (Sec. 4.2 multi-head decoder, Eq. 10).
 */
#ifndef DASH_H_
#define DASH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DASH_MAX_LEVELS 32

typedef enum dash_status {
  DASH_OK = 0,
  DASH_ERR_INVALID_ARG = -1, /* null pointer, negative size, inconsistent shapes */
  DASH_ERR_UNSUPPORTED = -2, /* valid but not implemented (F, L, MLP widths)     */
  DASH_ERR_WORKSPACE = -3,   /* workspace missing or too small                   */
  DASH_ERR_CUDA = -4,        /* a CUDA runtime call failed; see dash_last_error   */
  DASH_ERR_BOUNDS = -5,      /* a device-side check found an out-of-range value  */
  DASH_ERR_TIMEOUT = -6      /* a bounded device-side wait gave up               */
} dash_status;

typedef enum dash_dtype { DASH_F32 = 0, DASH_F16 = 1, DASH_BF16 = 2 } dash_dtype;

/* Hash-grid hyper-parameters (Sec. 4.2): L levels, F features per level,
 * hashed tables of T = 2^log2_T entries, coarsest/finest spatial (x, y, z)
 * and temporal resolutions, and the four hash primes pi_i of Eq. 8. */
typedef struct dash_hash4d_cfg {
  int32_t L, F, log2_T, reserved;
  double nmin_s, nmax_s, nmin_t, nmax_t;
  uint32_t primes[4];
} dash_hash4d_cfg;

/* Level layout derived from a cfg by dash_hash4d_layout (host struct, passed
 * to kernels by value).  res_*: N_l of Eq. 7; dense[l] != 0 when all
 * (N_s+1)^3 (N_t+1) vertices fit in T (then indexed directly, x fastest),
 * else hashed by Eq. 8 into T entries; size[l]: entries used; offset[l]:
 * first entry of level l, a multiple of 8; offset[L]: entries to allocate. */
typedef struct dash_layout {
  int32_t L, F, log2_T, dims; /* dims: 0 = 4-D (x, y, z, t), 3 = 3-D (x, y, z) */
  uint32_t primes[4];
  int32_t res_s[DASH_MAX_LEVELS];
  int32_t res_t[DASH_MAX_LEVELS];
  int32_t dense[DASH_MAX_LEVELS];
  int64_t size[DASH_MAX_LEVELS];
  int64_t offset[DASH_MAX_LEVELS + 1];
} dash_layout;

/* The points to encode: FP32 SoA coordinates of ALL Gaussians, indexed
 * through idx (compact dynamic list, NULL = identity 0..n-1).  t_stride = 1
 * reads t[j] per point, 0 broadcasts t[0] (one frame = one timestamp).
 * n is the number of points, or the capacity when n_dev is set: then the
 * kernels read the count from device memory (*n_dev, clamped to n), so a
 * captured CUDA graph needs no host-side count. */
typedef struct dash_points {
  const float* x;
  const float* y;
  const float* z;
  const float* t;
  int64_t t_stride;
  const int32_t* idx;
  int64_t n;
  const int64_t* n_dev;
} dash_points;

/* The decoder phi_d + heads (Sec. 4.2, Eq. 9): D = L*F -> H -> H -> O with
 * ReLU after the two hidden layers; params is the packed FP32 vector. */
typedef struct dash_mlp {
  int32_t d_in, d_hidden, d_out, reserved;
  const float* params;
} dash_mlp;

/* Optional Eq. 10 epilogue: attrs_out[k][j] = attrs_in[k][j] + delta[k][i]
 * for j = idx[i] (SoA [O][n_all], FP32).  Only dynamic rows are written. */
typedef struct dash_apply {
  const float* attrs_in;
  float* attrs_out;
  int64_t n_all;
} dash_apply;

/* Optional smoothness term (Eq. 11): adds lambda_r * L_r with
 * L_r = (1/n) sum_i |f(p_i) - f(p_i + e_s)|^2 + |f(p_i) - f(p_i + e_t)|^2,
 * e_s = (eps_s[0], eps_s[1], eps_s[2], 0), e_t = (0, 0, 0, eps_t); perturbed
 * coordinates are clamp(fl32(clamp(p) + e)).  The perturbed encodings are
 * recomputed by the backward, never stored.  loss_out (device
 * float, may be NULL) accumulates lambda_r * L_r. */
typedef struct dash_smooth {
  float lambda_r;
  float eps_s[3];
  float eps_t;
  float* loss_out;
} dash_smooth;

/* ----------------------------------------------------------- utilities -- */

/* Static string for a status code. */
const char* dash_status_string(int status);
/* Thread-local detail of the last failed call on this thread ("" if none). */
const char* dash_last_error(void);
/* ABI version (major * 100 + minor). */
int dash_version(void);
/* Device-side failure report: synchronises `stream`, then reads and clears
 * the flag words the persistent kernels (fused forward and backward,
 * batched plans; and the wait self-test below) set when a bounded wait (an MMA completion or a ring
 * stage, 2^22 polls) gives up — the kernel then stops issuing, frees its
 * TMEM and returns, leaving that launch's outputs incomplete.  Returns
 * DASH_ERR_TIMEOUT if any flag was set since the last call, else DASH_OK. */
int dash_device_status(void* stream);

/* Failure-path checks; the paper has no counterpart.
 *
 * dash_selftest_wait: launches one thread on `stream` that waits, with a
 * bound of `polls` (1 .. 2^22) polls, on a shared-memory mbarrier that
 * nothing arrives at -- the bounded wait of the persistent kernels, made to
 * run out.  It then sets its device flag word and returns, so the next
 * dash_device_status returns DASH_ERR_TIMEOUT (and clears the flag); the
 * context stays usable.  Errors: INVALID_ARG (polls out of range), CUDA.
 *
 * dash_debug_fail_cuda_call: fault injection on the host.  With n >= 1 the
 * n-th CUDA runtime call that the library checks from now on (counted over
 * all threads: allocations, copies, memsets, stream and graph calls,
 * launch checks) is not made and fails, so that call's entry point returns
 * DASH_ERR_CUDA with "injected failure" in dash_last_error, after releasing
 * what it had acquired.  n = 0 disarms the hook; either value restarts the
 * count that dash_debug_cuda_call_count returns (checked calls since the
 * last dash_debug_fail_cuda_call).  Not for concurrent use with other
 * library calls that must not fail. */
int dash_selftest_wait(int64_t polls, void* stream);

/* Rate probes of the access patterns that bound the fused kernels (the
 * paper has no counterpart: a measuring tool).  One launch of
 * dash_probe_threads(kind) threads (8 CTAs of 256 per SM), each issuing
 * `iters` (1 .. 65536) operations at pseudo-random 16-byte groups of buf
 * (device, 16-byte aligned, buf_bytes >= 16; size it like the tables or the
 * gradient buffer so it stays L2-resident).  *ops_out (host) receives the
 * number of lane operations issued; the caller times the launch.  The
 * reduction kinds add 1.0 into buf (its contents change); the gather kinds
 * only read buf and write one float per thread to sink (device, required
 * for them, NULL allowed otherwise).
 *   DASH_PROBE_RED8          8-byte FP32 vector reduction, each lane its own
 *                            random entry
 *   DASH_PROBE_RED16         16-byte FP32 vector reduction, random group
 *   DASH_PROBE_RED8_PAIRED   lanes 2j, 2j+1: 8 bytes each into the two halves
 *                            of one 16-byte group, same instruction
 *   DASH_PROBE_GATHER4       4-byte load, each lane its own random entry
 *   DASH_PROBE_GATHER4_PAIRED lanes 2j, 2j+1: neighbouring 4-byte entries
 * Errors: INVALID_ARG, CUDA. */
enum {
  DASH_PROBE_RED8 = 1,
  DASH_PROBE_RED16 = 2,
  DASH_PROBE_RED8_PAIRED = 3,
  DASH_PROBE_GATHER4 = 4,
  DASH_PROBE_GATHER4_PAIRED = 5
};
int dash_probe_threads(int kind);
int dash_probe_rate(int kind, float* buf, size_t buf_bytes, int iters, float* sink, int64_t* ops_out,
                    void* stream);
int dash_debug_fail_cuda_call(int64_t n);
int64_t dash_debug_cuda_call_count(void);

/* Bounds-checked build (libdash_debug.so, compiled with -DDASH_DEBUG): the
 * point rows the kernels read (dash_points.idx entries, or 0..n-1) are
 * checked against `rows`, the length of the x, y, z (and per-point t)
 * arrays, before each access: a row outside [0, rows) sets a device flag,
 * the access is skipped (the point reads as (0, 0, 0, 0) and its Eq. 10
 * update is not written), and the next dash_device_status returns
 * DASH_ERR_BOUNDS.  rows = -1 (the default) turns the check off.  The
 * release library (libdash.so) compiles no check and returns
 * DASH_ERR_UNSUPPORTED here.  Process-wide; set it before the launches it
 * should cover.  The paper has no counterpart. */
int dash_debug_set_point_rows(int64_t rows);

/* Process-wide kernel-form options (host; take effect at the next launch).
 * DASH_OPT_FWD_FORM selects the fused forward kernel: 0 = warp-specialised
 * (one decoder group fed by gather groups through a shared-memory ring;
 * default for F = 2, L*F <= 32: five groups x five stages with FP16
 * tables, enough gather warps to keep the L1's miss path busy; three x three
 * with FP32 tables, whose 8-byte entries need more registers), 1 / 2 / 4 = that many
 * independent gather+decoder groups per CTA, and for F = 2, L*F <= 32 the
 * warp-specialised shapes (gather groups, ring stages) 10 = (3, 6),
 * 11 = (3, 3), 12 = (2, 4), 13 = (5, 5), 14 = (4, 4), 15 = (2, 2).  DASH_OPT_BWD_FORM
 * selects the fused backward: 0 = warp-specialised (a decoder group feeding
 * scatter groups; default four groups x five stages for F = 2, L*F <= 32;
 * used when a forward state is given), 1 = one combined group per CTA,
 * 10..14 = the shapes (3, 6), (4, 4), (2, 4), (5, 5), (3, 3).  When the
 * number of scatter groups divides L (and there is no coordinate gradient),
 * every group scatters every tile, each its own share of the levels;
 * otherwise the groups take whole tiles in turn.  Every shape has at least
 * one ring stage per group.  Forward forms agree bit for bit, backward forms up to the
 * order of the atomic additions.  DASH_OPT_ACCESS_FORM selects how the
 * warp-specialised forward and backward kernels issue their F = 2 table
 * accesses: 0 = lane pairs (default; lanes 2j and 2j+1 take the lower and
 * upper x corner of both their Gaussians, so the two accesses of an
 * x-neighbour pair leave in one warp instruction: L1 serves two loads in
 * one 128-byte line with one lookup and L2 two reductions in one 32-byte
 * sector as one operation), 1 = one Gaussian per lane (a pair is one
 * 16-byte access when both entries share an aligned 16 bytes, else two).
 * The forward's features agree bit for bit; the backward's table gradients
 * up to the order of the additions (as are the coordinate gradients, whose
 * gathers are paired too).  A batched plan keeps the value current when it
 * was created.  (The F = 2 Eq. 11 kernel and the encoder-only kernels always
 * use lane pairs.)
 * DASH_OPT_GRAD_REPLICAS (0..64, default 16): k, the number of replicas of
 * the FP32 gradients of each leading dense level of at most 2^17 entries
 * (levels 0 and 1 at the paper shape) that dash_deform_mlp_bwd uses when it
 * is given a workspace (see there); 0 or 1 = none.  It sizes
 * dash_deform_bwd_workspace_size, so set it before sizing.
 * DASH_OPT_DECOMP_FORM (0 or 1, default 0): dash_decomp_fwd and
 * dash_decomp_bwd run phi_p's contractions on the tensor cores (0; the
 * backward for L*F <= 48) or on the CUDA cores (1; the backward always for
 * L*F > 48).  Same results up to rounding.
 * dash_get_option returns the current value (negative status for an
 * unknown option). */
enum dash_option {
  DASH_OPT_FWD_FORM = 1,
  DASH_OPT_BWD_FORM = 2,
  DASH_OPT_ACCESS_FORM = 3,
  DASH_OPT_GRAD_REPLICAS = 4,
  DASH_OPT_DECOMP_FORM = 5
};
int dash_set_option(int option, int value);
int dash_get_option(int option);

/* Eq. 7 (host): fills *out from *cfg.  N_l = floor(N_min * b^l + 1e-9),
 * b = exp((ln N_max - ln N_min) / (L - 1)), separately for space and time.
 * Errors: INVALID_ARG (null, N_min < 1, N_max < N_min), UNSUPPORTED
 * (L > 32, F not in {1,2,4,8}, log2_T outside [4, 28]). */
int dash_hash4d_layout(const dash_hash4d_cfg* cfg, dash_layout* out);

/* ------------------------------------------------- a1: compaction ------ */

/* Bytes of device workspace dash_compact_dynamic needs for n mask entries. */
size_t dash_compact_workspace_size(int64_t n);

/* Self-supervised split (Sec. 4.1): idx_out receives, in ascending order,
 * every i < n with mask[i] != 0 (the dynamic set G_d), *count_out (device
 * int64) its length.  idx_out must hold n entries.  ws: device scratch of
 * dash_compact_workspace_size(n) bytes (contents need not be initialised).
 * Errors: INVALID_ARG, WORKSPACE (ws too small), UNSUPPORTED (n >= 2^31). */
int dash_compact_dynamic(const uint8_t* mask, int64_t n, int32_t* idx_out, int64_t* count_out,
                         void* ws, size_t ws_bytes, void* stream);

/* dash_compact_dynamic without a workspace and without allocating anything.
 * The paper has no counterpart: this serves callers that must not allocate
 * device memory while they run (a render loop that owns all device memory
 * and gives its plug-ins only buffers it allocated up front, or code running
 * inside a memory allocator's own callbacks, where cudaMalloc would re-enter
 * that allocator).  The per-CTA scratch is a 256 KB array built into the
 * library, held by every GPU that loads it until the process exits; n is
 * limited to 268,435,456 mask entries (DASH_ERR_UNSUPPORTED beyond).  The
 * first call on a device resolves the array's device address (one
 * cudaGetSymbolAddress, with that device current) and, because CUDA loads
 * device code lazily, may load this part of the library onto the device --
 * and so allocate (the code and the array).  Make one warm-up call per
 * device with a nonempty mask (n >= 1, so that all three of its kernels
 * run once) before entering a region that must not allocate and before any
 * stream capture; every later call allocates nothing.  The address is
 * cached per process and per device ordinal: call from the device's primary
 * context (the runtime API's default) and do not cudaDeviceReset the device
 * between calls, which would leave the cached address pointing at memory
 * this library no longer owns.  All calls share the array: calls whose
 * kernels overlap on the GPU (other streams, other host threads) race and
 * corrupt each other's results; serialise them.  Output and errors as
 * dash_compact_dynamic. */
int dash_compact_dynamic_noalloc(const uint8_t* mask, int64_t n, int32_t* idx_out,
                                 int64_t* count_out, void* stream);

/* ---------------------------------------- a2-a6: encoder (Eqs. 8-9) ---- */

/* Debug view of Eq. 8/9: idx_out [n][L][16] level-local corner indices
 * (corner b: bit d set = upper corner along axis d of x, y, z, t) and
 * w_out [n][L][16] FP32 quadrilinear weights (either may be NULL). */
int dash_hash4d_indices(const dash_layout* layout, const dash_points* pts,
                        uint32_t* idx_out, float* w_out, void* stream);

/* Eq. 9 encoder f_h = G_4D(x): feat_out [n][L*F] of feat_dtype (F32, F16 or
 * BF16) from the table of table_dtype (F32 or F16), FP32 arithmetic. */
int dash_hash4d_fwd(const dash_layout* layout, const dash_points* pts, const void* table,
                    int table_dtype, void* feat_out, int feat_dtype, void* stream);

/* Transpose of the encoder: table_grad[offset[l] + idx][f] += w * dfeat[i][l*F+f]
 * over the 16 corners of every level.  dfeat [n][L*F] FP32, table_grad FP32
 * [offset[L]][F].  Vector FP32 atomics; summation order is not deterministic.
 * For F = 2 the reductions are issued by lane pairs (see DASH_OPT_ACCESS_FORM). */
int dash_hash4d_bwd(const dash_layout* layout, const dash_points* pts, const float* dfeat,
                    float* table_grad, void* stream);

/* The same transpose into FP16 gradients (F = 2 only): table_grad is
 * [offset[L]][2] FP16, accumulated with half2 vector atomics (an x-adjacent
 * corner pair within one aligned 16-byte group is one 16-byte reduction).
 * A reduced-precision variant: FP16 accumulation loses accuracy on entries
 * that receive many updates; the FP32 form above is the reference. */
int dash_hash4d_bwd_half(const dash_layout* layout, const dash_points* pts, const float* dfeat,
                         void* table_grad, void* stream);

/* Gradient of sum_i dfeat_i . G_4D(p_i) with respect to the coordinates
 * (x, y, z, t) of each compact point (Eq. 9 differentiated through its
 * quadrilinear weights; for canonical positions optimised through the
 * field).  d(x * N_l)/dx = N_l; at a vertex the derivative of the hypervoxel
 * above it is taken, at 1 that of the last one; the clamp passes the
 * derivative on [0,1] and gives 0 outside and for NaN.  dfeat [n][L*F] FP32
 * as dash_hash4d_bwd; dcoord SoA [4][pts->n] FP32 (rows x, y, z, t; with a
 * broadcast t, row 3 holds each point's share; rows past the device count
 * are not written).  table F32 or F16, 16-byte aligned.  One launch. */
int dash_hash4d_coord_grad(const dash_layout* layout, const dash_points* pts, const void* table,
                           int table_dtype, const float* dfeat, float* dcoord, void* stream);

/* ----------- table occupancy: the collision argument (Sec. 4.2, Sec. 5) -- */

/* Bytes of device workspace dash_hash4d_collision_stats needs for up to n
 * points: a set of 2^ceil(log2(32 n)) 64-bit vertex ids (at least 1024) plus
 * one 32-bit counter per entry of the largest level.  0 for bad arguments. */
size_t dash_collision_workspace_size(const dash_layout* layout, int64_t n);

/* Per level l, into stats_out[3 l .. 3 l + 2] (device int64 [L][3]): V, the
 * distinct grid vertices touched by the points' hypervoxel corners (Eq. 8's
 * cells); E, the distinct table entries those vertices occupy; C, the touched
 * vertices whose entry is shared with at least one other touched vertex.
 * Dense levels give E = V, C = 0.  Exact integer counts (order independent).
 * A level whose vertex set overflowed reports -1, -1, -1 (does not happen
 * with the workspace size above).  ws: 256-byte aligned, at least
 * dash_collision_workspace_size(layout, pts->n) bytes; stream-ordered memsets
 * and 3 launches per level.  The paper has no such routine: it measures how
 * crowded the tables are with and without the static/dynamic decomposition. */
int dash_hash4d_collision_stats(const dash_layout* layout, const dash_points* pts,
                                int64_t* stats_out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------- a2-a8: fused deformation forward (Eqs. 8-10) -- */

/* Bytes of forward state per Gaussian that dash_deform_mlp_fwd keeps for
 * dash_deform_mlp_bwd: f_h in BF16 (2 * d_in bytes, padded to 16) followed by
 * the two ReLU masks of the hidden layers (16 bytes). */
size_t dash_deform_state_size(const dash_mlp* mlp);

/* Encoder + decoder MLP (+ optional Eq. 10) in one kernel: gathers the
 * tables (F32 or F16), interpolates in FP32, runs the three decoder layers on
 * the tensor cores (tcgen05, BF16 operands with the activations split into a
 * hi + lo pair, FP32 accumulation in TMEM) and writes delta_out SoA [O][n]
 * FP32.  fwd_state (optional, 16-byte aligned, n * dash_deform_state_size
 * bytes) receives what the backward needs.  apply may be NULL.
 * Supported: D = L*F <= 64, H = 64, O <= 16.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int dash_deform_mlp_fwd(const dash_layout* layout, const dash_points* pts,
                        const void* table, int table_dtype, const dash_mlp* mlp,
                        float* delta_out, void* fwd_state, const dash_apply* apply,
                        void* stream);

/* Backward of the Eq. 10 update: for each compact point k (row
 * i = idx[k], or k without a list) ddelta[j][k] = dattrs[j][i] for the
 * d_out attribute rows (x, r, s for O = 10).  dattrs SoA [d_out][n_all]
 * (e.g. the renderer's gradients at the deformed attributes), ddelta SoA
 * [d_out][pts->n] as dash_deform_mlp_bwd takes it; rows past the device
 * count are not written.  One launch. */
int dash_deform_apply_bwd(const dash_points* pts, int d_out, const float* dattrs, int64_t n_all,
                          float* ddelta, void* stream);

/* ---------------------- a9-a11: fused deformation backward (+ Eq. 11) -- */

/* Backward of dash_deform_mlp_fwd for upstream ddelta SoA [O][n] FP32:
 * recomputes the decoder from fwd_state (as written by the forward, whose
 * ReLU masks it reuses; NULL = re-encode f_h in FP32 and recompute the masks),
 * back-propagates on the tensor cores (BF16 operands, FP32 accumulation),
 * accumulates mlp_grad (FP32, packed like params) and scatters dL/df_h into
 * table_grad (FP32 [offset[L]][F], 16-byte aligned) with vector atomics.
 * With smooth != NULL and lambda_r != 0 also adds the Eq. 11 term,
 * re-encoding p, p + e_s and p + e_t (for F = 2 with a forward state in a
 * second kernel launched right after, on the same stream; otherwise inside
 * the backward kernel).  Shapes as the forward.
 * coord_grad (may be NULL): SoA [4][pts->n] FP32 receives d loss / d(x, y,
 * z, t) of each compact point as dash_hash4d_coord_grad defines it (the
 * scatter step also gathers the corner entries); not available together with
 * the Eq. 11 term (DASH_ERR_UNSUPPORTED).
 * ws (device, 16-byte aligned, may be NULL) of ws_bytes >=
 * dash_deform_bwd_workspace_size bytes (DASH_ERR_WORKSPACE otherwise)
 * enables, for F = 2 with a forward state and lane-paired accesses:
 *  - replicas of the coarsest dense levels' gradients
 *    (DASH_OPT_GRAD_REPLICAS = k; not with coord_grad):
 *    the lane-paired scatter and the Eq. 11 kernel reduce from CTA b into
 *    replica b % k, which the call zeroes first and adds into table_grad
 *    last (a memset and one more kernel on the stream);
 *  - with the Eq. 11 term: the backward kernel writes dL/df_h to ws instead
 *    of scattering it, and the Eq. 11 kernel adds it to the Eq. 11 gradient
 *    at p's corners (one reduction per corner instead of two).
 * Without ws, or on other paths, the gradients are reduced straight into
 * table_grad.  The results agree up to the order of the additions. */
int dash_deform_mlp_bwd(const dash_layout* layout, const dash_points* pts,
                        const void* table, int table_dtype, const dash_mlp* mlp,
                        const float* ddelta, const void* fwd_state, float* table_grad,
                        float* mlp_grad, const dash_smooth* smooth, float* coord_grad,
                        void* ws, size_t ws_bytes, void* stream);
/* Bytes of workspace dash_deform_mlp_bwd can use for n points: the
 * gradient replicas (with the current DASH_OPT_GRAD_REPLICAS) plus, when
 * smooth has lambda_r != 0, dL/df_h as FP32 SoA [L*F][n]; 0 if neither
 * applies (F != 2). */
size_t dash_deform_bwd_workspace_size(const dash_layout* layout, int64_t n, const dash_smooth* smooth);

/* ------------- decomposition producing the mask (Sec. 4.1, Eqs. 3-5) ---- */

/* 3-D layout of the position encoder G_3D: Eq. 7 spatial resolutions,
 * levels with (N+1)^3 <= T vertices indexed directly, others hashed by Eq. 8
 * with primes[0..2]; res_t = 0, dims = 3.  Errors as dash_hash4d_layout. */
int dash_hash3d_layout(const dash_hash4d_cfg* cfg, dash_layout* out);

/* Positional deformation dp = phi_l(phi_p(G_3D(p))) of n Gaussians and its
 * norm (the motion magnitude whose top-k % makes a Gaussian dynamic).
 * x, y, z [n] FP32 in [0,1] (clamped); table of the 3-D layout (F32/F16);
 * mlp: d_in = L*F, d_hidden = 64, d_out = 3 with params packed W1 [64][D],
 * b1 [64], W2 [3][64], b2 [3] (ReLU after the first layer).  dp_out SoA
 * [3][n] (may be NULL), norm_out [n].  With pt_out (SoA [3][n], may be NULL)
 * also the Eq. 4 linear motion p(t) = p + t dp, p the unclamped x, y, z and
 * t [n] (t_stride 1) or one value for all (t_stride 0).  n <= 2^31 - 1.
 * One launch on `stream`; all pointers are device memory. */
int dash_decomp_fwd(const dash_layout* layout3, const float* x, const float* y, const float* z,
                    int64_t n, const void* table, int table_dtype, const dash_mlp* mlp,
                    float* dp_out, float* norm_out, const float* t, int64_t t_stride,
                    float* pt_out, void* stream);

/* Backward of the decomposition (Eqs. 3-5) for the loss
 *   sum_i d_dp_i . dp_i + lambda_s * L_s,  L_s = (1/N_s) sum_{mask_i = 0} |dp_i|
 * (Eq. 5 over the static Gaussians of `mask`, N_s their number):
 * recomputes G_3D, phi_p and phi_l per Gaussian and ACCUMULATES the
 * gradients of the G_3D tables (table_grad FP32 [offset[L]][F], 16-byte
 * aligned, as the table) and of the packed W1, b1, W2, b2 (mlp_grad).
 * d_dp SoA [3][n] may be NULL (no upstream term, e.g. from p(t) through
 * Eq. 4: d_dp = t dL/dp(t)); mask may be NULL or lambda_s 0 (no L_s term);
 * static Gaussians with |dp| = 0 contribute nothing.  Shapes as
 * dash_decomp_fwd.  ws: dash_decomp_bwd_workspace_size() bytes.  2-3
 * launches. */
size_t dash_decomp_bwd_workspace_size(void);
int dash_decomp_bwd(const dash_layout* layout3, const float* x, const float* y, const float* z,
                    int64_t n, const void* table, int table_dtype, const dash_mlp* mlp,
                    const float* d_dp, const uint8_t* mask, float lambda_s, float* table_grad,
                    float* mlp_grad, void* ws, size_t ws_bytes, void* stream);

/* Bytes of device workspace dash_topk_mask needs (a few hundred). */
size_t dash_topk_workspace_size(void);

/* Top-k % split: tau = the (m+1)-th largest of values[0..n) with
 * m = floor(k_percent * n / 100), found exactly by a radix select on the
 * values' bit patterns (values are norms: zeros of either sign, NaN and
 * negatives all count as +0); mask_out[i] = values[i] > tau, so ties at tau
 * are static; m = 0 marks none, m >= n marks all (tau = -1).  tau_out
 * (device float) may be NULL.  static_loss_out (device float, may be NULL)
 * receives Eq. 5's L_s = mean of the static values (0 if none is static),
 * summed in FP64.  n <= 2^31 - 1 (DASH_ERR_UNSUPPORTED above); k_percent
 * outside [0, 100] or a workspace below dash_topk_workspace_size() is an
 * error.  Launches at most 11 small kernels on `stream`; ws is reused. */
int dash_topk_mask(const float* values, int64_t n, double k_percent, uint8_t* mask_out,
                   float* tau_out, float* static_loss_out, void* ws, size_t ws_bytes,
                   void* stream);

/* ----------- the renderer the deformed Gaussians are drawn with --------
 * 3D Gaussian splatting (Sec. 3): Eq. 1 with Sigma = R S S^T R^T projected
 * to Sigma' = J W Sigma W^T J^T, spherical-harmonics colour, Eq. 2 alpha
 * blending front to back in 16 x 16 pixel tiles, into a device image.
 * Conventions: pinhole u = fx x/z + cx, v = fy y/z + cy (pixel (i, j) is
 * evaluated at (i, j)); Gaussians with z <= near_plane or det(Sigma') <= 0
 * are not drawn; `dilation` is added to Sigma''s diagonal; alpha =
 * min(0.99, opacity exp(-d^T Sigma'^-1 d / 2)), contributions below 1/255
 * are skipped and blending stops before T would fall below 1e-4; each
 * Gaussian is considered in the tiles its square of half-side
 * ceil(3 sqrt(lambda_max(Sigma'))) overlaps, in ascending depth (ties by
 * index); colour = real orthonormal SH (degree <= 3, no Condon-Shortley
 * phase) at the unit direction campos -> mean, + 0.5, clamped at 0. */

typedef struct dash_camera {
  float view[16];       /* world -> camera, row-major 4 x 4 acting on column vectors */
  float fx, fy, cx, cy; /* pixels */
  int32_t width, height;
  float near_plane;
  float dilation;       /* screen-space low-pass added to Sigma' (0.3 in 3DGS) */
  float campos[3];      /* camera centre in world coordinates */
  float bg[3];          /* background colour */
} dash_camera;

/* Device SoA attributes of n Gaussians (activations are the caller's). */
typedef struct dash_gaussians {
  const float* mean;    /* [3][n] world positions */
  const float* scale;   /* [3][n] standard deviations along the local axes */
  const float* rot;     /* [4][n] quaternion (w, x, y, z), any non-zero norm */
  const float* opacity; /* [n] */
  const float* sh;      /* [n][16][3] SH coefficients, the first (degree+1)^2 used */
  int32_t sh_degree;    /* 0..3 */
  int32_t reserved;
  int64_t n;            /* < 2^31 */
} dash_gaussians;

/* Gradient buffers, same layouts as dash_gaussians; accumulated (+=). */
typedef struct dash_gaussian_grads {
  float* mean;
  float* scale;
  float* rot;
  float* opacity;
  float* sh;
} dash_gaussian_grads;

/* Bytes of device workspace for one view of n Gaussians with room for
 * max_pairs (tile, Gaussian) pairs; 0 for bad arguments. */
size_t dash_raster_workspace_size(const dash_camera* cam, int64_t n, int64_t max_pairs);

/* Renders image [3][height][width] FP32 (device).  ws (256-byte aligned,
 * dash_raster_workspace_size bytes) keeps the view's per-Gaussian, per-tile
 * and per-pixel state for dash_raster_bwd.  pairs_needed (device int64, may
 * be NULL) receives the number of pairs the view needs; when it exceeds
 * max_pairs the image is NaN (grow the workspace and render again).  No host
 * synchronisation; 5 launches.  Errors: INVALID_ARG (NULL), UNSUPPORTED
 * (image > 16384, sh_degree > 3, n >= 2^31), WORKSPACE. */
int dash_raster_fwd(const dash_camera* cam, const dash_gaussians* gaussians, float* image, void* ws,
                    size_t ws_bytes, int64_t max_pairs, int64_t* pairs_needed, void* stream);

/* Backward of the last dash_raster_fwd on this ws (same camera, Gaussians
 * and max_pairs): accumulates dL/d(mean, scale, rot, opacity, sh) for
 * dL/dimage [3][height][width].  Culled Gaussians get no gradient; the 0.99
 * alpha clamp and the colour clamp pass none.  2 launches + 1 memset. */
int dash_raster_bwd(const dash_camera* cam, const dash_gaussians* gaussians, const float* dimage,
                    void* ws, size_t ws_bytes, int64_t max_pairs, const dash_gaussian_grads* grads,
                    void* stream);

/* ---------------- a12: many scenes x timestamps, one graph launch ------ */

#define DASH_MAX_SCENES 64

/* One scene of a batched run: its own tables and decoder, its dynamic
 * Gaussians' FP32 coordinates x, y, z [n], K normalised timestamps (device
 * [K]; one broadcast t per frame), and delta_out SoA [K][O][n] FP32.  n is the
 * capacity and initial count; the live count can be changed on the device
 * through dash_batch_counts() without rebuilding the plan.
 * With a backward (dash_batch_desc.with_backward): ddelta SoA [K][O][n] FP32
 * is the upstream gradient of each (timestamp, Gaussian); fwd_state
 * [K][n][dash_deform_state_size] (16-byte aligned) receives the forward's
 * per-Gaussian state; table_grad (FP32 [offset[L]][F], 16-byte aligned) and
 * mlp_grad (FP32, packed like params) ACCUMULATE the scene's gradients over
 * its K timestamps. */
typedef struct dash_batch_scene {
  const void* table;
  const float* params;
  const float* x;
  const float* y;
  const float* z;
  const float* timestamps;
  float* delta_out;
  int64_t n;
  int32_t K, reserved;
  const float* ddelta;
  void* fwd_state;
  float* table_grad;
  float* mlp_grad;
} dash_batch_scene;

/* All scenes share the grid layout, table dtype and decoder widths.
 * with_backward = 1 adds, after the forward, the fused backward (a9-a10:
 * decoder gradients, lane-paired table-gradient scatter) of every (scene,
 * timestamp, tile) in a second persistent kernel of the same graph; F = 2
 * and L*F <= 32 only.  The plan then also owns replicas of each scene's
 * coarsest dense levels' gradients (DASH_OPT_GRAD_REPLICAS when it is
 * created; see dash_deform_mlp_bwd), cleared before the backward kernel
 * and added into table_grad after it, inside the graph. */
typedef struct dash_batch_desc {
  const dash_layout* layout;
  int32_t table_dtype;
  int32_t d_in, d_hidden, d_out;
  int32_t n_scenes;
  const dash_batch_scene* scenes; /* host array of n_scenes */
  int32_t with_backward, reserved;
} dash_batch_desc;

typedef struct dash_batch_plan dash_batch_plan;

/* Builds a plan on the current device: copies the scene descriptors and
 * counts to device memory (the only allocation of the library) and captures
 * one persistent launch of the batched forward (Eqs. 8-9 gathers and the
 * tensor-core decoder for every (scene, timestamp, 128-Gaussian tile)) in a
 * CUDA graph.  The kernel reads the counts on the device.  Synchronous.
 * Errors: INVALID_ARG, UNSUPPORTED (n_scenes > 64, shapes), CUDA. */
int dash_batch_plan_create(const dash_batch_desc* desc, dash_batch_plan** out);
/* Device int64 [n_scenes] live counts (each clamped to its capacity). */
int64_t* dash_batch_counts(dash_batch_plan* plan);
/* Replays the captured graph on `stream`. */
int dash_batch_run(dash_batch_plan* plan, void* stream);
/* Kernel forms in use: f + 16 * b, f the forward form (index into the
 * compiled (gather groups, ring stages) forms {(4,4), (3,6), (3,3), (2,4),
 * (2,2), (5,5)}), b the backward form (into the (scatter groups, ring stages) forms
 * {(4,5), (2,2), (2,4), (3,4), (3,3)}; 0 without a backward). */
int dash_batch_form(const dash_batch_plan* plan);
/* Autotuner: if cache_json_path holds an entry for this plan's signature
 * (GPU, grid shape, scenes, counts, timestamps, with or without backward)
 * those forms are used; otherwise every compiled forward form is timed on
 * this plan's own work (one warm-up and three timed launches on `stream`)
 * and the fastest kept, then, with a backward, every backward form on the
 * state of one forward run.  The gradient buffers are copied aside before
 * the backward runs and restored after them, so tuning leaves them as they
 * were (a temporary device buffer of the scenes' gradient size).  The cache
 * file is rewritten with the choice (the value f + 16 * b) and the graph
 * re-captured for it.  Synchronous. */
int dash_batch_autotune(dash_batch_plan* plan, const char* cache_json_path, void* stream);
int dash_batch_plan_destroy(dash_batch_plan* plan);

/* ------------------------ plain FP32 form (comparison baseline) -------- */
/* One thread per point, FP32 tables, f_h stored in global memory, FP32
 * CUDA-core decoder, scalar FP32 atomics.  Same semantics as above. */
int dash_plain_hash4d_fwd(const dash_layout* layout, const dash_points* pts,
                          const float* table, float* feat_out, void* stream);
int dash_plain_hash4d_bwd(const dash_layout* layout, const dash_points* pts,
                          const float* dfeat, float* table_grad, void* stream);
/* feat [n][D] -> delta_out SoA [O][n]; n_dev optional device count. */
int dash_plain_mlp_fwd(const dash_mlp* mlp, const float* feat, int64_t n, const int64_t* n_dev,
                       float* delta_out, void* stream);
/* Bytes of workspace dash_plain_mlp_bwd needs: the materialised h1, h2,
 * dz1, dz2 (4 * H * n FP32). */
size_t dash_plain_mlp_bwd_workspace_size(const dash_mlp* mlp, int64_t n);
/* ddelta SoA [O][n] -> dfeat_out [n][D] (written), mlp_grad (accumulated).
 * ws: device scratch of dash_plain_mlp_bwd_workspace_size bytes. */
int dash_plain_mlp_bwd(const dash_mlp* mlp, const float* feat, int64_t n, const int64_t* n_dev,
                       const float* ddelta, float* dfeat_out, float* mlp_grad, void* ws, size_t ws_bytes,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DASH_H_ */
