// raster_bwd.cu -- backward of the splatting renderer (Sec. 3): from
// dL/dimage to the gradients of every Gaussian's mean, scale, rotation,
// opacity and SH coefficients, using the forward's workspace.
//
//   1. render_bwd (CTA per tile): walks each pixel's blended Gaussians back
//      to front.  With T_i the transmittance in front of Gaussian i and
//      A_i = sum_{k>i} c_k alpha_k prod_{i<j<k} (1 - alpha_j) the colour
//      behind it, Eq. 2 gives dC/dc_i = alpha_i T_i and
//      dC/dalpha_i = T_i (c_i - A_i) - T_final bg / (1 - alpha_i).  Through
//      Eq. 1 (alpha = sigma exp(power), power = -d^T Q d / 2, d = mean' -
//      pixel) these become gradients of the screen mean, the conic Q and the
//      opacity; the 0.99 clamp passes no gradient.  All lanes of a warp visit
//      the same Gaussian together: warps none of whose pixels blended it
//      skip it, the others sum the nine values over the warp with a
//      reduce-scatter and add them with one atomic instruction.
//   2. preprocess_bwd (thread per Gaussian): conic -> Sigma' -> (J, Sigma) ->
//      camera-space mean -> world mean; Sigma = R S S^T R^T -> scale and the
//      (normalised) quaternion; colour -> SH coefficients and, through the
//      view direction, the mean.
#include "raster_common.cuh"

namespace dash {
namespace raster {
namespace {

constexpr int kThreads = 256;

// One halving step of a warp reduce-scatter: lanes whose `off` bit is clear
// keep the first H of the M values (summed with their partner's), the others
// the last M - H (padded with zero to H).  One shuffle per kept value.
template <int M, int H>
__device__ __forceinline__ void halve(float* a, unsigned lane, int off) {
  const bool up = (lane & (unsigned)off) != 0u;
  float b[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float lo = a[i];
    const float hi = i + H < M ? a[i + H] : 0.f;
    b[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, off);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) a[i] = b[i];
}

// Sums 9 values over the warp with 12 shuffles (instead of 45 for nine
// butterflies): afterwards an even lane l with scatter_index(l) >= 0 holds
// the warp total of that value in v[0] (its odd neighbour holds a copy).
__device__ __forceinline__ void warp_reduce_scatter9(float v[9], unsigned lane) {
  halve<9, 5>(v, lane, 16);
  halve<5, 3>(v, lane, 8);
  halve<3, 2>(v, lane, 4);
  halve<2, 1>(v, lane, 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Which value lane `lane` ends up with: the halving steps' (size, half, bit)
// replayed on the index range [start, start + size) this lane keeps; an upper
// half may hold fewer real values than its padded width.  -1: padding only.
__device__ __forceinline__ int scatter_index(unsigned lane) {
  const int half[4] = {5, 3, 2, 1};
  const unsigned bit[4] = {16u, 8u, 4u, 2u};
  int start = 0, size = 9;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (lane & bit[s]) {
      start += half[s];
      size = size > half[s] ? size - half[s] : 0;
    } else {
      size = size < half[s] ? size : half[s];
    }
  }
  return size >= 1 ? start : -1;
}

__global__ void __launch_bounds__(kTilePix) render_bwd_kernel(Cam c, long long n, const float* __restrict__ opacity,
                                                              Ws w, const float* __restrict__ dimage,
                                                              float* __restrict__ dopacity) {
  // one Gaussian's screen data per slot, packed as in render_kernel
  __shared__ float4 s_a[kTilePix];  // mean x, mean y, conic a, conic b
  __shared__ float4 s_b[kTilePix];  // conic c, opacity, colour r, colour g
  __shared__ float s_c[kTilePix];   // colour b
  __shared__ int s_gid[kTilePix];
  __shared__ uint32_t s_max;
  const int t = blockIdx.x;
  const int tx_ = t % w.tiles_x, ty_ = t / w.tiles_x;
  const int px = tx_ * kTile + (int)(threadIdx.x % kTile), py = ty_ * kTile + (int)(threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const size_t pix = (size_t)py * c.W + px;
  const size_t plane = (size_t)c.W * c.H;
  const long long s0 = w.start[t];
  const uint32_t last = inside ? w.n_contrib[pix] : 0u;
  if (threadIdx.x == 0) s_max = 0u;
  __syncthreads();
  atomicMax(&s_max, last);
  __syncthreads();
  const uint32_t todo = s_max;  // list positions 1..todo are visited, back to front
  const float fx = (float)px, fy = (float)py;
  const float T_final = inside ? w.final_T[pix] : 1.f;
  float T = T_final;
  float g0 = 0.f, g1 = 0.f, g2 = 0.f;
  if (inside) {
    g0 = dimage[pix];
    g1 = dimage[plane + pix];
    g2 = dimage[2 * plane + pix];
  }
  const float bg_dot = c.bg[0] * g0 + c.bg[1] * g1 + c.bg[2] * g2;
  // the gradient array this lane adds into after the warp's reduce-scatter
  const unsigned lane = threadIdx.x & 31u;
  const int red_k = scatter_index(lane);
  const bool red_lane = (lane & 1u) == 0u && red_k >= 0;
  float* red_ptr = nullptr;
  switch (red_k) {
    case 0: red_ptr = w.dmean2d; break;
    case 1: red_ptr = w.dmean2d + n; break;
    case 2: red_ptr = w.dconic; break;
    case 3: red_ptr = w.dconic + n; break;
    case 4: red_ptr = w.dconic + 2 * n; break;
    case 5: red_ptr = dopacity; break;
    case 6: red_ptr = w.dcolor; break;
    case 7: red_ptr = w.dcolor + n; break;
    case 8: red_ptr = w.dcolor + 2 * n; break;
    default: break;
  }
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;  // colour behind the current Gaussian
  float last_alpha = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;
  for (int end = (int)todo; end > 0; end -= kTilePix) {
    const int begin = end - kTilePix > 0 ? end - kTilePix : 0;
    const int cnt = end - begin;
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int k = end - 1 - (int)threadIdx.x;  // back to front
      const long long gid = (long long)(w.keys[s0 + k] & 0xffffffffull);
      s_gid[threadIdx.x] = (int)gid;
      s_a[threadIdx.x] = make_float4(w.mean2d[gid], w.mean2d[n + gid], w.conic[gid], w.conic[n + gid]);
      s_b[threadIdx.x] = make_float4(w.conic[2 * n + gid], opacity[gid], w.color[gid], w.color[n + gid]);
      s_c[threadIdx.x] = w.color[2 * n + gid];
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const uint32_t position = (uint32_t)(end - j);  // 1-based list position of this Gaussian
      float d_mx = 0.f, d_my = 0.f, d_ca = 0.f, d_cb = 0.f, d_cc = 0.f, d_op = 0.f, d_c0 = 0.f, d_c1 = 0.f,
            d_c2 = 0.f;
      bool hit = false;
      if (position <= last) {
        const float4 A = s_a[j];
        const float4 B = s_b[j];
        const float dx = A.x - fx, dy = A.y - fy;
        const float ca = A.z, cb = A.w, cc = B.x;
        const float power = -0.5f * (ca * dx * dx + cc * dy * dy) - cb * dx * dy;
        const float G = expf(power);
        const float raw = B.y * G;
        const float alpha = fminf(kAlphaMax, raw);
        if (power <= 0.f && alpha >= kAlphaMin) {
          hit = true;
          T = T / (1.f - alpha);  // transmittance in front of this Gaussian
          const float wgt = alpha * T;
          d_c0 = wgt * g0, d_c1 = wgt * g1, d_c2 = wgt * g2;
          acc0 = last_alpha * lc0 + (1.f - last_alpha) * acc0;
          acc1 = last_alpha * lc1 + (1.f - last_alpha) * acc1;
          acc2 = last_alpha * lc2 + (1.f - last_alpha) * acc2;
          const float c0 = B.z, c1 = B.w, c2 = s_c[j];
          float dL_da = ((c0 - acc0) * g0 + (c1 - acc1) * g1 + (c2 - acc2) * g2) * T;
          dL_da -= T_final / (1.f - alpha) * bg_dot;
          last_alpha = alpha, lc0 = c0, lc1 = c1, lc2 = c2;
          if (raw <= kAlphaMax) {  // the clamp passes no gradient
            const float dL_dp = dL_da * raw;  // d alpha / d power = sigma G
            d_op = dL_da * G;
            d_mx = dL_dp * (-ca * dx - cb * dy);
            d_my = dL_dp * (-cc * dy - cb * dx);
            d_ca = -0.5f * dx * dx * dL_dp;
            d_cb = -dx * dy * dL_dp;
            d_cc = -0.5f * dy * dy * dL_dp;
          }
        }
      }
      // most warps see only part of a Gaussian's footprint: skip the
      // reduction when no lane of this warp blended it
      if (!__any_sync(0xffffffffu, hit)) continue;
      float v[9] = {d_mx, d_my, d_ca, d_cb, d_cc, d_op, d_c0, d_c1, d_c2};
      warp_reduce_scatter9(v, lane);
      if (red_lane && v[0] != 0.f) atomicAdd(red_ptr + s_gid[j], v[0]);  // nine lanes, one instruction
    }
  }
}

// d rotation-matrix entries / d (w, x, y, z) of the unit quaternion, contracted
// with the gradient G_R (row-major 3x3).
__device__ __forceinline__ void quat_rot_bwd(float w, float x, float y, float z, const float G[9], float dq[4]) {
  dq[0] = 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  dq[1] = 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.f * x * G[8]);
  dq[2] = 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.f * y * G[8]);
  dq[3] = 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
}

__global__ void __launch_bounds__(kThreads) preprocess_bwd_kernel(Cam c, dash_gaussians gs, Ws w,
                                                                  dash_gaussian_grads gr) {
  const long long n = gs.n;
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const int4 rc = w.rect[i];
  if (rc.x >= rc.z) return;  // not drawn: no gradient
  const float mx = gs.mean[i], my = gs.mean[n + i], mz = gs.mean[2 * n + i];
  const float tx = c.V[0] * mx + c.V[1] * my + c.V[2] * mz + c.V[3];
  const float ty = c.V[4] * mx + c.V[5] * my + c.V[6] * mz + c.V[7];
  const float tz = c.V[8] * mx + c.V[9] * my + c.V[10] * mz + c.V[11];
  float qw = gs.rot[i], qx = gs.rot[n + i], qy = gs.rot[2 * n + i], qz = gs.rot[3 * n + i];
  const float qinv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  const float uw = qw * qinv, ux = qx * qinv, uy = qy * qinv, uz = qz * qinv;
  float R[9];
  quat_rot(uw, ux, uy, uz, R);
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
  const float iz = 1.f / tz;
  const float j00 = c.fx * iz, j02 = -c.fx * tx * iz * iz, j11 = c.fy * iz, j12 = -c.fy * ty * iz * iz;
  float T[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T[k] = j00 * c.V[k] + j02 * c.V[8 + k];
    T[3 + k] = j11 * c.V[4 + k] + j12 * c.V[8 + k];
  }
  float TS[6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) TS[3 * r + k] = T[3 * r] * Sg[k] + T[3 * r + 1] * Sg[3 + k] + T[3 * r + 2] * Sg[6 + k];
  const float a = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + c.dilation;
  const float b = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
  const float cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + c.dilation;
  const float det = a * cc - b * b;
  const float idet = 1.f / det;
  // conic Q = A^-1 (A = Sigma' + dilation): dL/dA = -Q Gq Q with Gq the
  // symmetric gradient of Q (its off-diagonal gradient is split in two halves)
  const float qa = cc * idet, qb = -b * idet, qc = a * idet;
  const float ga = w.dconic[i], gb = 0.5f * w.dconic[n + i], gc = w.dconic[2 * n + i];
  // P = Gq Q
  const float p00 = ga * qa + gb * qb, p01 = ga * qb + gb * qc, p10 = gb * qa + gc * qb, p11 = gb * qb + gc * qc;
  const float dA00 = -(qa * p00 + qb * p10), dA01 = -(qa * p01 + qb * p11), dA11 = -(qb * p01 + qc * p11);
  // Sigma' = T Sigma T^T: dL/dSigma = T^T G2 T, dL/dT = 2 G2 T Sigma (G2 symmetric = dA)
  const float G2[4] = {dA00, dA01, dA01, dA11};
  float dSg[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dSg[3 * r + k] = T[r] * (G2[0] * T[k] + G2[1] * T[3 + k]) + T[3 + r] * (G2[2] * T[k] + G2[3] * T[3 + k]);
  float dT[6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) dT[3 * r + k] = 2.f * (G2[2 * r] * TS[k] + G2[2 * r + 1] * TS[3 + k]);
  // T = J V_r: dL/dJ = dT V_r^T (only J00, J02, J11, J12 are non-zero)
  const float dJ00 = dT[0] * c.V[0] + dT[1] * c.V[1] + dT[2] * c.V[2];
  const float dJ02 = dT[0] * c.V[8] + dT[1] * c.V[9] + dT[2] * c.V[10];
  const float dJ11 = dT[3] * c.V[4] + dT[4] * c.V[5] + dT[5] * c.V[6];
  const float dJ12 = dT[3] * c.V[8] + dT[4] * c.V[9] + dT[5] * c.V[10];
  const float du = w.dmean2d[i], dv = w.dmean2d[n + i];
  const float iz2 = iz * iz, iz3 = iz2 * iz;
  float dtx = c.fx * iz * du - c.fx * iz2 * dJ02;
  float dty = c.fy * iz * dv - c.fy * iz2 * dJ12;
  float dtz = -c.fx * tx * iz2 * du - c.fy * ty * iz2 * dv - c.fx * iz2 * dJ00 + 2.f * c.fx * tx * iz3 * dJ02 -
              c.fy * iz2 * dJ11 + 2.f * c.fy * ty * iz3 * dJ12;
  float dmx = c.V[0] * dtx + c.V[4] * dty + c.V[8] * dtz;
  float dmy = c.V[1] * dtx + c.V[5] * dty + c.V[9] * dtz;
  float dmz = c.V[2] * dtx + c.V[6] * dty + c.V[10] * dtz;
  // Sigma = M M^T: dL/dM = 2 dSigma M; M = R S
  float dM[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) dM[3 * r + k] = 2.f * (dSg[3 * r] * M[k] + dSg[3 * r + 1] * M[3 + k] + dSg[3 * r + 2] * M[6 + k]);
  float dR[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) dR[3 * r + k] = dM[3 * r + k] * s[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ds = dM[k] * R[k] + dM[3 + k] * R[3 + k] + dM[6 + k] * R[6 + k];
    gr.scale[k * n + i] += ds;
  }
  float du4[4];
  quat_rot_bwd(uw, ux, uy, uz, dR, du4);
  // through q / |q|: (I - u u^T) / |q|
  const float udot = uw * du4[0] + ux * du4[1] + uy * du4[2] + uz * du4[3];
  gr.rot[i] += (du4[0] - uw * udot) * qinv;
  gr.rot[n + i] += (du4[1] - ux * udot) * qinv;
  gr.rot[2 * n + i] += (du4[2] - uy * udot) * qinv;
  gr.rot[3 * n + i] += (du4[3] - uz * udot) * qinv;
  // colour: SH coefficients, and the view direction's dependence on the mean
  float vx = mx - c.campos[0], vy = my - c.campos[1], vz = mz - c.campos[2];
  const float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
  const float ex = vx * vinv, ey = vy * vinv, ez = vz * vinv;
  float Y[kMaxShCoeffs], dY[kMaxShCoeffs][3];
  sh_eval(ex, ey, ez, gs.sh_degree, Y, dY);
  const int K = (gs.sh_degree + 1) * (gs.sh_degree + 1);
  const uint32_t cl = w.clamp[i];
  float drgb[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) drgb[ch] = (cl >> ch) & 1u ? 0.f : w.dcolor[ch * n + i];
  const float* sh = gs.sh + (size_t)i * kMaxShCoeffs * 3;
  float* gsh = gr.sh + (size_t)i * kMaxShCoeffs * 3;
  float de[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < K; ++k) {
    float dYk = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      gsh[3 * k + ch] += Y[k] * drgb[ch];
      dYk = fmaf(sh[3 * k + ch], drgb[ch], dYk);
    }
    de[0] = fmaf(dYk, dY[k][0], de[0]);
    de[1] = fmaf(dYk, dY[k][1], de[1]);
    de[2] = fmaf(dYk, dY[k][2], de[2]);
  }
  const float edot = ex * de[0] + ey * de[1] + ez * de[2];
  dmx += (de[0] - ex * edot) * vinv;
  dmy += (de[1] - ey * edot) * vinv;
  dmz += (de[2] - ez * edot) * vinv;
  gr.mean[i] += dmx;
  gr.mean[n + i] += dmy;
  gr.mean[2 * n + i] += dmz;
}

}  // namespace
}  // namespace raster
}  // namespace dash

extern "C" int dash_raster_bwd(const dash_camera* cam, const dash_gaussians* gs, const float* dimage, void* ws,
                               size_t ws_bytes, int64_t max_pairs, const dash_gaussian_grads* grads, void* stream) {
  DASH_NVTX_RANGE("dash_raster_bwd");
  using namespace dash;
  using namespace dash::raster;
  Cam c;
  if (int s = check_inputs(cam, gs, &c)) return s;
  if (dimage == nullptr || grads == nullptr || grads->mean == nullptr || grads->scale == nullptr ||
      grads->rot == nullptr || grads->opacity == nullptr || grads->sh == nullptr)
    return fail(DASH_ERR_INVALID_ARG, "dimage/grads is NULL");
  const size_t need = dash_raster_workspace_size(cam, gs->n, max_pairs);
  if (ws == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes (256-byte aligned), %zu needed", ws_bytes, need);
  if (gs->n == 0) return DASH_OK;
  cudaStream_t st = as_stream(stream);
  Ws w = bind(ws, gs->n, c.W, c.H, max_pairs);
  const Layout L = layout_for(gs->n, c.W, c.H, max_pairs);
  // dmean2d, dconic, dcolor are contiguous in the layout
  if (int s = cuda_status(DASH_RT(cudaMemsetAsync(w.dmean2d, 0, L.count - L.dmean2d, st)), "cudaMemsetAsync")) return s;
  const int tiles = w.tiles_x * w.tiles_y;
  render_bwd_kernel<<<(unsigned)tiles, kTilePix, 0, st>>>(c, gs->n, gs->opacity, w, dimage, grads->opacity);
  if (int s = launch_status("render_bwd_kernel")) return s;
  preprocess_bwd_kernel<<<(unsigned)((gs->n + kThreads - 1) / kThreads), kThreads, 0, st>>>(c, *gs, w, *grads);
  return launch_status("preprocess_bwd_kernel");
}
