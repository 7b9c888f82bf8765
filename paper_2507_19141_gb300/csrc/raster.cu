// raster.cu -- forward of the 3D Gaussian splatting renderer that draws the
// deformed Gaussians (Sec. 3: Eq. 1, Sigma = R S S^T R^T, the screen-space
// covariance Sigma' = J W Sigma W^T J^T, spherical-harmonics colour, Eq. 2
// alpha blending) into a device image.
//
//   1. preprocess  (thread per Gaussian): camera-space mean, Sigma', conic,
//      3-sigma extent and tile range, SH colour; counts the Gaussian in every
//      tile it overlaps.
//   2. scan        (one CTA): exclusive prefix of the per-tile counts.
//   3. emit        (thread per Gaussian): one 64-bit key per (tile, Gaussian)
//      into its tile's bucket, (depth bits << 32) | index -- unique, so the
//      order after sorting is the same whatever the atomics' order.
//   4. sort        (CTA per tile): bitonic sort of the bucket, in shared
//      memory up to 4096 keys, in global memory above.
//   5. render      (CTA per 16x16 tile): Eq. 2 front to back over the tile's
//      sorted Gaussians, staged 256 at a time in shared memory.
// No step synchronises with the host: the pairs needed are written to the
// device, and a view whose pairs exceed the workspace renders NaN.
#include "raster_common.cuh"

namespace dash {
namespace raster {
namespace {

constexpr int kThreads = 256;
constexpr int kSortSmem = 4096;

__global__ void __launch_bounds__(kThreads) preprocess_kernel(Cam c, dash_gaussians gs, Ws w) {
  const long long n = gs.n;
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  w.rect[i] = make_int4(0, 0, 0, 0);
  const float mx = gs.mean[i], my = gs.mean[n + i], mz = gs.mean[2 * n + i];
  const float tx = c.V[0] * mx + c.V[1] * my + c.V[2] * mz + c.V[3];
  const float ty = c.V[4] * mx + c.V[5] * my + c.V[6] * mz + c.V[7];
  const float tz = c.V[8] * mx + c.V[9] * my + c.V[10] * mz + c.V[11];
  if (!(tz > c.near_plane)) return;
  // Sigma = M M^T with M = R S
  float qw = gs.rot[i], qx = gs.rot[n + i], qy = gs.rot[2 * n + i], qz = gs.rot[3 * n + i];
  const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= qn, qx *= qn, qy *= qn, qz *= qn;
  float R[9];
  quat_rot(qw, qx, qy, qz, R);
  const float s[3] = {gs.scale[i], gs.scale[n + i], gs.scale[2 * n + i]};
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) M[3 * r + k] = R[3 * r + k] * s[k];
  float Sg[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) Sg[3 * r + k] = M[3 * r] * M[3 * k] + M[3 * r + 1] * M[3 * k + 1] + M[3 * r + 2] * M[3 * k + 2];
  // T = J V_r (2 x 3): rows of the projection's Jacobian times the view rotation
  const float iz = 1.f / tz;
  const float j00 = c.fx * iz, j02 = -c.fx * tx * iz * iz, j11 = c.fy * iz, j12 = -c.fy * ty * iz * iz;
  float T[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T[k] = j00 * c.V[k] + j02 * c.V[8 + k];
    T[3 + k] = j11 * c.V[4 + k] + j12 * c.V[8 + k];
  }
  float TS[6];  // T Sigma
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) TS[3 * r + k] = T[3 * r] * Sg[k] + T[3 * r + 1] * Sg[3 + k] + T[3 * r + 2] * Sg[6 + k];
  const float a = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + c.dilation;
  const float b = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
  const float cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + c.dilation;
  const float det = a * cc - b * b;
  if (!(det > 0.f)) return;
  const float idet = 1.f / det;
  const float mid = 0.5f * (a + cc);
  const float lam = mid + sqrtf(fmaxf(mid * mid - det, 0.f));
  const float r = ceilf(3.f * sqrtf(lam));
  const float u = c.fx * tx * iz + c.cx, v = c.fy * ty * iz + c.cy;
  const int x0 = (int)fminf(fmaxf(floorf((u - r) / kTile), 0.f), (float)w.tiles_x);
  const int x1 = (int)fminf(fmaxf(floorf((u + r) / kTile) + 1.f, 0.f), (float)w.tiles_x);
  const int y0 = (int)fminf(fmaxf(floorf((v - r) / kTile), 0.f), (float)w.tiles_y);
  const int y1 = (int)fminf(fmaxf(floorf((v + r) / kTile) + 1.f, 0.f), (float)w.tiles_y);
  if (x0 >= x1 || y0 >= y1) return;
  // colour: SH at the direction from the camera centre, + 0.5, clamped at 0
  float dx = mx - c.campos[0], dy = my - c.campos[1], dz = mz - c.campos[2];
  const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= dn, dy *= dn, dz *= dn;
  float Y[kMaxShCoeffs];
  sh_eval(dx, dy, dz, gs.sh_degree, Y, nullptr);
  const int K = (gs.sh_degree + 1) * (gs.sh_degree + 1);
  const float* sh = gs.sh + (size_t)i * kMaxShCoeffs * 3;
  uint32_t clampbits = 0u;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.5f;
    for (int k = 0; k < K; ++k) acc = fmaf(Y[k], sh[3 * k + ch], acc);
    if (acc < 0.f) {
      acc = 0.f;
      clampbits |= 1u << ch;
    }
    w.color[ch * n + i] = acc;
  }
  w.clamp[i] = clampbits;
  w.mean2d[i] = u;
  w.mean2d[n + i] = v;
  w.conic[i] = cc * idet;
  w.conic[n + i] = -b * idet;
  w.conic[2 * n + i] = a * idet;
  w.depth[i] = tz;
  w.rect[i] = make_int4(x0, y0, x1, y1);
  for (int ty_ = y0; ty_ < y1; ++ty_)
    for (int tx_ = x0; tx_ < x1; ++tx_) atomicAdd(w.count + ty_ * w.tiles_x + tx_, 1u);
}

// Exclusive prefix of the tile counts (one CTA of 1024 threads, chunked).
__global__ void __launch_bounds__(1024) tile_scan_kernel(Ws w) {
  __shared__ uint32_t part[32];
  __shared__ uint32_t carry;
  const int tiles = w.tiles_x * w.tiles_y;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < tiles; base += 1024) {
    const int t = base + (int)threadIdx.x;
    const uint32_t v = t < tiles ? w.count[t] : 0u;
    uint32_t x = v;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) part[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t p = part[threadIdx.x];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, p, o);
        if (threadIdx.x >= o) p += y;
      }
      part[threadIdx.x] = p;
    }
    __syncthreads();
    const uint32_t warp_off = (threadIdx.x >> 5) ? part[(threadIdx.x >> 5) - 1] : 0u;
    if (t < tiles) w.start[t] = carry + warp_off + x - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += warp_off + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.start[tiles] = carry;
    *w.pairs_needed = (long long)carry;
  }
}

__global__ void __launch_bounds__(kThreads) emit_kernel(long long n, Ws w) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const int4 rc = w.rect[i];
  if (rc.x >= rc.z) return;
  const unsigned long long key = ((unsigned long long)__float_as_uint(w.depth[i]) << 32) | (unsigned long long)i;
  for (int ty_ = rc.y; ty_ < rc.w; ++ty_)
    for (int tx_ = rc.x; tx_ < rc.z; ++tx_) {
      const int t = ty_ * w.tiles_x + tx_;
      const unsigned long long pos = (unsigned long long)w.start[t] + atomicAdd(w.cursor + t, 1u);
      if (pos < (unsigned long long)w.max_pairs) w.keys[pos] = key;
    }
}

// Bitonic network in its all-ascending form: each stage k first compares
// i with its mirror in the k-block, then half-cleans with distances k/4 .. 1.
// Pairs whose upper index is >= m are skipped (virtual +inf padding), so any
// length works in place.
template <bool kShared>
__device__ void bitonic(unsigned long long* a, int m) {
  int N = 1;
  while (N < m) N <<= 1;
  for (int k = 2; k <= N; k <<= 1) {
    for (int p = threadIdx.x; p < N / 2; p += blockDim.x) {
      const int half = k >> 1;
      const int lo = (p / half) * k + (p % half);
      const int hi = (p / half) * k + k - 1 - (p % half);
      if (hi < m) {
        const unsigned long long x = a[lo], y = a[hi];
        if (y < x) a[lo] = y, a[hi] = x;
      }
    }
    __syncthreads();
    for (int j = k >> 2; j >= 1; j >>= 1) {
      for (int p = threadIdx.x; p < N / 2; p += blockDim.x) {
        const int lo = (p / j) * 2 * j + (p % j);
        const int hi = lo + j;
        if (hi < m) {
          const unsigned long long x = a[lo], y = a[hi];
          if (y < x) a[lo] = y, a[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads) tile_sort_kernel(Ws w) {
  __shared__ unsigned long long buf[kSortSmem];
  const int t = blockIdx.x;
  const long long s0 = w.start[t];
  long long s1 = w.start[t + 1];
  if (*w.pairs_needed > w.max_pairs) return;  // overflow: nothing to sort, render writes NaN
  const int m = (int)(s1 - s0);
  if (m <= 1) return;
  if (m <= kSortSmem) {
    for (int k = threadIdx.x; k < m; k += kThreads) buf[k] = w.keys[s0 + k];
    __syncthreads();
    bitonic<true>(buf, m);
    for (int k = threadIdx.x; k < m; k += kThreads) w.keys[s0 + k] = buf[k];
  } else {
    bitonic<false>(w.keys + s0, m);
  }
}

__global__ void __launch_bounds__(kTilePix) render_kernel(Cam c, long long n, const float* __restrict__ opacity, Ws w,
                                                          float* __restrict__ image) {
  // one Gaussian's screen data per slot, packed so a pixel reads it with
  // two 16-byte and one 4-byte shared-memory loads (all lanes read the same slot)
  __shared__ float4 s_a[kTilePix];  // mean x, mean y, conic a, conic b
  __shared__ float4 s_b[kTilePix];  // conic c, opacity, colour r, colour g
  __shared__ float s_c[kTilePix];   // colour b
  const int t = blockIdx.x;
  const int tx_ = t % w.tiles_x, ty_ = t / w.tiles_x;
  const int px = tx_ * kTile + (int)(threadIdx.x % kTile), py = ty_ * kTile + (int)(threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const bool overflow = *w.pairs_needed > w.max_pairs;
  const long long s0 = w.start[t];
  const long long s1 = overflow ? s0 : (long long)w.start[t + 1];
  const float fx = (float)px, fy = (float)py;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t pos = 0, last = 0;
  bool done = !inside;
  for (long long base = s0; base < s1; base += kTilePix) {
    if (__syncthreads_count(done) == kTilePix) break;
    const long long k = base + threadIdx.x;
    if (k < s1) {
      const long long gid = (long long)(w.keys[k] & 0xffffffffull);
      s_a[threadIdx.x] = make_float4(w.mean2d[gid], w.mean2d[n + gid], w.conic[gid], w.conic[n + gid]);
      s_b[threadIdx.x] = make_float4(w.conic[2 * n + gid], opacity[gid], w.color[gid], w.color[n + gid]);
      s_c[threadIdx.x] = w.color[2 * n + gid];
    }
    __syncthreads();
    const int cnt = (int)((s1 - base) < kTilePix ? (s1 - base) : kTilePix);
    for (int j = 0; j < cnt && !done; ++j) {
      ++pos;
      const float4 A = s_a[j];
      const float dx = A.x - fx, dy = A.y - fy;
      const float4 B = s_b[j];
      const float power = -0.5f * (A.z * dx * dx + B.x * dy * dy) - A.w * dx * dy;
      if (power > 0.f) continue;
      const float alpha = fminf(kAlphaMax, B.y * expf(power));
      if (alpha < kAlphaMin) continue;
      const float tt = T * (1.f - alpha);
      if (tt < kTMin) {
        done = true;
        break;
      }
      const float wgt = alpha * T;
      C0 = fmaf(B.z, wgt, C0);
      C1 = fmaf(B.w, wgt, C1);
      C2 = fmaf(s_c[j], wgt, C2);
      T = tt;
      last = pos;
    }
  }
  if (!inside) return;
  const size_t pix = (size_t)py * c.W + px;
  const size_t plane = (size_t)c.W * c.H;
  const float nan = __int_as_float(0x7fc00000);
  image[pix] = overflow ? nan : fmaf(T, c.bg[0], C0);
  image[plane + pix] = overflow ? nan : fmaf(T, c.bg[1], C1);
  image[2 * plane + pix] = overflow ? nan : fmaf(T, c.bg[2], C2);
  w.final_T[pix] = T;
  w.n_contrib[pix] = last;
}

}  // namespace

int check_inputs(const dash_camera* cam, const dash_gaussians* g, Cam* out) {
  if (cam == nullptr || g == nullptr || out == nullptr) return fail(DASH_ERR_INVALID_ARG, "camera/gaussians is NULL");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return fail(DASH_ERR_UNSUPPORTED, "image %d x %d outside 1..16384", cam->width, cam->height);
  if (g->n < 0 || g->n > 0x7FFFFFFFll) return fail(DASH_ERR_UNSUPPORTED, "n=%lld outside [0, 2^31)", (long long)g->n);
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(DASH_ERR_UNSUPPORTED, "sh_degree %d (0..3)", g->sh_degree);
  if (g->n > 0 && (g->mean == nullptr || g->scale == nullptr || g->rot == nullptr || g->opacity == nullptr ||
                   g->sh == nullptr))
    return fail(DASH_ERR_INVALID_ARG, "a Gaussian attribute pointer is NULL");
  for (int k = 0; k < 12; ++k) out->V[k] = cam->view[k];
  out->fx = cam->fx, out->fy = cam->fy, out->cx = cam->cx, out->cy = cam->cy;
  out->W = cam->width, out->H = cam->height;
  out->near_plane = cam->near_plane, out->dilation = cam->dilation;
  for (int k = 0; k < 3; ++k) out->campos[k] = cam->campos[k], out->bg[k] = cam->bg[k];
  return DASH_OK;
}

}  // namespace raster
}  // namespace dash

extern "C" {

size_t dash_raster_workspace_size(const dash_camera* cam, int64_t n, int64_t max_pairs) {
  if (cam == nullptr || n < 0 || max_pairs < 0 || cam->width < 1 || cam->height < 1) return 0;
  return dash::raster::layout_for(n, cam->width, cam->height, max_pairs).total;
}

int dash_raster_fwd(const dash_camera* cam, const dash_gaussians* gs, float* image, void* ws, size_t ws_bytes,
                    int64_t max_pairs, int64_t* pairs_needed, void* stream) {
  DASH_NVTX_RANGE("dash_raster_fwd");
  using namespace dash;
  using namespace dash::raster;
  Cam c;
  if (int s = check_inputs(cam, gs, &c)) return s;
  if (image == nullptr) return fail(DASH_ERR_INVALID_ARG, "image is NULL");
  if (max_pairs < 0 || max_pairs > 0xFFFFFFFFll) return fail(DASH_ERR_UNSUPPORTED, "max_pairs outside [0, 2^32)");
  const size_t need = dash_raster_workspace_size(cam, gs->n, max_pairs);
  if (ws == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes (256-byte aligned), %zu needed", ws_bytes, need);
  cudaStream_t st = as_stream(stream);
  Ws w = bind(ws, gs->n, c.W, c.H, max_pairs);
  const int tiles = w.tiles_x * w.tiles_y;
  if (int s = cuda_status(DASH_RT(cudaMemsetAsync(w.count, 0, (size_t)tiles * 4u, st)), "cudaMemsetAsync")) return s;
  if (int s = cuda_status(DASH_RT(cudaMemsetAsync(w.cursor, 0, (size_t)tiles * 4u, st)), "cudaMemsetAsync")) return s;
  const unsigned grid_g = (unsigned)((gs->n + kThreads - 1) / kThreads);
  if (gs->n > 0) {
    preprocess_kernel<<<grid_g, kThreads, 0, st>>>(c, *gs, w);
    if (int s = launch_status("preprocess_kernel")) return s;
  }
  tile_scan_kernel<<<1, 1024, 0, st>>>(w);
  if (int s = launch_status("tile_scan_kernel")) return s;
  if (gs->n > 0) {
    emit_kernel<<<grid_g, kThreads, 0, st>>>(gs->n, w);
    if (int s = launch_status("emit_kernel")) return s;
  }
  tile_sort_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(w);
  if (int s = launch_status("tile_sort_kernel")) return s;
  render_kernel<<<(unsigned)tiles, kTilePix, 0, st>>>(c, gs->n, gs->opacity, w, image);
  if (int s = launch_status("render_kernel")) return s;
  if (pairs_needed != nullptr &&
      cuda_status(DASH_RT(cudaMemcpyAsync(pairs_needed, w.pairs_needed, 8u, cudaMemcpyDeviceToDevice, st)), "cudaMemcpyAsync"))
    return DASH_ERR_CUDA;
  return DASH_OK;
}

}  // extern "C"
