// raster_common.cuh -- shared pieces of the 3D Gaussian splatting renderer
// (Sec. 3: Eq. 1, Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T, the
// spherical-harmonics colour, Eq. 2): workspace layout, constants, the
// rotation from a quaternion and the real spherical-harmonics basis with its
// gradient.
#pragma once

#include <math.h>

#include "dash_internal.cuh"

namespace dash {
namespace raster {

constexpr int kTile = 16;                   // 16 x 16 pixel tiles, one CTA each
constexpr int kTilePix = kTile * kTile;
constexpr float kAlphaMin = 1.0f / 255.0f;  // contributions below are skipped
constexpr float kAlphaMax = 0.99f;          // Eq. 1's alpha is clamped here
constexpr float kTMin = 1e-4f;              // blending stops before T drops below
constexpr int kMaxShCoeffs = 16;            // degree 3

// Device workspace of one rendered view, kept from the forward for the backward.
struct Ws {
  // per Gaussian
  float* mean2d;    // [2][n]
  float* conic;     // [3][n] (a, b, c) of Sigma'^-1
  float* color;     // [3][n]
  float* depth;     // [n]
  int4* rect;       // [n] tile range x0, y0, x1, y1 (exclusive); x0 = x1 = 0 when not drawn
  uint32_t* clamp;  // [n] bit c: colour channel c was clamped at 0
  float* dmean2d;   // [2][n] backward scratch
  float* dconic;    // [3][n]
  float* dcolor;    // [3][n]
  // per tile
  uint32_t* count;   // [tiles]
  uint32_t* start;   // [tiles + 1] exclusive prefix of count; start[tiles] = pairs needed
  uint32_t* cursor;  // [tiles]
  // pairs and pixels
  unsigned long long* keys;  // [max_pairs] (depth bits << 32) | Gaussian index
  float* final_T;            // [H * W]
  uint32_t* n_contrib;       // [H * W] list position after the last blended Gaussian
  long long* pairs_needed;   // [1]
  long long max_pairs;
  int tiles_x, tiles_y;
};

struct Cam {
  float V[12];  // rows 0-2 of the view matrix (R | t)
  float fx, fy, cx, cy;
  int W, H;
  float near_plane, dilation;
  float campos[3];
  float bg[3];
};

// Byte offsets of every array in the workspace (256-byte aligned).
struct Layout {
  size_t mean2d, conic, color, depth, rect, clamp, dmean2d, dconic, dcolor;
  size_t count, start, cursor, keys, final_T, n_contrib, pairs_needed, total;
};

inline size_t align256(size_t v) { return (v + 255u) & ~(size_t)255u; }

inline Layout layout_for(long long n, int W, int H, long long max_pairs) {
  const size_t tiles = (size_t)((W + kTile - 1) / kTile) * (size_t)((H + kTile - 1) / kTile);
  const size_t nn = (size_t)(n > 0 ? n : 1);
  Layout L;
  size_t o = 0;
  L.mean2d = o;  o = align256(o + 2 * nn * 4);
  L.conic = o;   o = align256(o + 3 * nn * 4);
  L.color = o;   o = align256(o + 3 * nn * 4);
  L.depth = o;   o = align256(o + nn * 4);
  L.rect = o;    o = align256(o + nn * 16);
  L.clamp = o;   o = align256(o + nn * 4);
  L.dmean2d = o; o = align256(o + 2 * nn * 4);
  L.dconic = o;  o = align256(o + 3 * nn * 4);
  L.dcolor = o;  o = align256(o + 3 * nn * 4);
  L.count = o;   o = align256(o + tiles * 4);
  L.start = o;   o = align256(o + (tiles + 1) * 4);
  L.cursor = o;  o = align256(o + tiles * 4);
  L.keys = o;    o = align256(o + (size_t)(max_pairs > 0 ? max_pairs : 1) * 8);
  L.final_T = o; o = align256(o + (size_t)W * H * 4);
  L.n_contrib = o; o = align256(o + (size_t)W * H * 4);
  L.pairs_needed = o; o = align256(o + 8);
  L.total = o;
  return L;
}

inline Ws bind(void* base, long long n, int W, int H, long long max_pairs) {
  const Layout L = layout_for(n, W, H, max_pairs);
  uint8_t* b = static_cast<uint8_t*>(base);
  Ws w;
  w.mean2d = reinterpret_cast<float*>(b + L.mean2d);
  w.conic = reinterpret_cast<float*>(b + L.conic);
  w.color = reinterpret_cast<float*>(b + L.color);
  w.depth = reinterpret_cast<float*>(b + L.depth);
  w.rect = reinterpret_cast<int4*>(b + L.rect);
  w.clamp = reinterpret_cast<uint32_t*>(b + L.clamp);
  w.dmean2d = reinterpret_cast<float*>(b + L.dmean2d);
  w.dconic = reinterpret_cast<float*>(b + L.dconic);
  w.dcolor = reinterpret_cast<float*>(b + L.dcolor);
  w.count = reinterpret_cast<uint32_t*>(b + L.count);
  w.start = reinterpret_cast<uint32_t*>(b + L.start);
  w.cursor = reinterpret_cast<uint32_t*>(b + L.cursor);
  w.keys = reinterpret_cast<unsigned long long*>(b + L.keys);
  w.final_T = reinterpret_cast<float*>(b + L.final_T);
  w.n_contrib = reinterpret_cast<uint32_t*>(b + L.n_contrib);
  w.pairs_needed = reinterpret_cast<long long*>(b + L.pairs_needed);
  w.max_pairs = max_pairs;
  w.tiles_x = (W + kTile - 1) / kTile;
  w.tiles_y = (H + kTile - 1) / kTile;
  return w;
}

// Validates camera and Gaussians (host), fills the kernel-side camera.
int check_inputs(const dash_camera* cam, const dash_gaussians* g, Cam* out);

// Rotation matrix (row-major 3x3) of the normalised quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Real orthonormal spherical harmonics (no Condon-Shortley phase) at the unit
// direction d, degree 0..3 ordered by degree then m = -l..l; with dY also the
// gradient of each basis function w.r.t. the (unnormalised) components.
struct ShConst {
  float c0, k1, a2, b2, c2, d1, d2, d3, d4, d5;
};

__device__ __forceinline__ ShConst sh_const() {
  const float pi = 3.14159265358979323846f;
  ShConst k;
  k.c0 = 0.5f / sqrtf(pi);
  k.k1 = sqrtf(3.f / (4.f * pi));
  k.a2 = 0.5f * sqrtf(15.f / pi);
  k.b2 = 0.25f * sqrtf(5.f / pi);
  k.c2 = 0.25f * sqrtf(15.f / pi);
  k.d1 = 0.25f * sqrtf(35.f / (2.f * pi));
  k.d2 = 0.5f * sqrtf(105.f / pi);
  k.d3 = 0.25f * sqrtf(21.f / (2.f * pi));
  k.d4 = 0.25f * sqrtf(7.f / pi);
  k.d5 = 0.25f * sqrtf(105.f / pi);
  return k;
}

__device__ __forceinline__ void sh_eval(float x, float y, float z, int degree, float Y[kMaxShCoeffs],
                                        float (*dY)[3]) {
  const ShConst k = sh_const();
  Y[0] = k.c0;
  if (dY) dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
  if (degree < 1) return;
  Y[1] = k.k1 * y;
  Y[2] = k.k1 * z;
  Y[3] = k.k1 * x;
  if (dY) {
    dY[1][0] = 0.f, dY[1][1] = k.k1, dY[1][2] = 0.f;
    dY[2][0] = 0.f, dY[2][1] = 0.f, dY[2][2] = k.k1;
    dY[3][0] = k.k1, dY[3][1] = 0.f, dY[3][2] = 0.f;
  }
  if (degree < 2) return;
  Y[4] = k.a2 * x * y;
  Y[5] = k.a2 * y * z;
  Y[6] = k.b2 * (3.f * z * z - 1.f);
  Y[7] = k.a2 * x * z;
  Y[8] = k.c2 * (x * x - y * y);
  if (dY) {
    dY[4][0] = k.a2 * y, dY[4][1] = k.a2 * x, dY[4][2] = 0.f;
    dY[5][0] = 0.f, dY[5][1] = k.a2 * z, dY[5][2] = k.a2 * y;
    dY[6][0] = 0.f, dY[6][1] = 0.f, dY[6][2] = 6.f * k.b2 * z;
    dY[7][0] = k.a2 * z, dY[7][1] = 0.f, dY[7][2] = k.a2 * x;
    dY[8][0] = 2.f * k.c2 * x, dY[8][1] = -2.f * k.c2 * y, dY[8][2] = 0.f;
  }
  if (degree < 3) return;
  const float zz5 = 5.f * z * z;
  Y[9] = k.d1 * y * (3.f * x * x - y * y);
  Y[10] = k.d2 * x * y * z;
  Y[11] = k.d3 * y * (zz5 - 1.f);
  Y[12] = k.d4 * z * (zz5 - 3.f);
  Y[13] = k.d3 * x * (zz5 - 1.f);
  Y[14] = k.d5 * z * (x * x - y * y);
  Y[15] = k.d1 * x * (x * x - 3.f * y * y);
  if (dY) {
    dY[9][0] = 6.f * k.d1 * x * y, dY[9][1] = 3.f * k.d1 * (x * x - y * y), dY[9][2] = 0.f;
    dY[10][0] = k.d2 * y * z, dY[10][1] = k.d2 * x * z, dY[10][2] = k.d2 * x * y;
    dY[11][0] = 0.f, dY[11][1] = k.d3 * (zz5 - 1.f), dY[11][2] = 10.f * k.d3 * y * z;
    dY[12][0] = 0.f, dY[12][1] = 0.f, dY[12][2] = k.d4 * (3.f * zz5 - 3.f);
    dY[13][0] = k.d3 * (zz5 - 1.f), dY[13][1] = 0.f, dY[13][2] = 10.f * k.d3 * x * z;
    dY[14][0] = 2.f * k.d5 * x * z, dY[14][1] = -2.f * k.d5 * y * z, dY[14][2] = k.d5 * (x * x - y * y);
    dY[15][0] = 3.f * k.d1 * (x * x - y * y), dY[15][1] = -6.f * k.d1 * x * y, dY[15][2] = 0.f;
  }
}

}  // namespace raster
}  // namespace dash
