// mlp_plain.cu -- plain FP32 CUDA-core form of the deformation decoder
// (Sec. 4.2: phi_d then the heads phi_x, phi_r, phi_s), the comparison
// baseline for the fused tensor-core kernels.  Unfused and materialised, the
// way a framework's Linear/ReLU layers run it:
//   forward: one thread per point, weights in shared memory;
//   backward: one thread per point recomputes the forward, back-propagates to
//   dL/df_h and stores h1, h2, dz1, dz2 (SoA [H][n]); a second kernel reduces
//   the weight gradients dW = dZ^T A over points on the CUDA cores.
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxOut = 16;

struct MlpShape {
  int D, H, O;
  long long P;  // packed parameter count
};

__host__ __device__ inline long long param_count(int D, int H, int O) {
  return (long long)H * D + H + (long long)H * H + H + (long long)O * H + O;
}

__device__ __forceinline__ long long count_of(long long n, const long long* n_dev) {
  if (n_dev == nullptr) return n;
  long long m = *n_dev;
  m = m < 0 ? 0 : m;
  return m < n ? m : n;
}

// Copies the packed parameters into shared memory.
__device__ __forceinline__ void stage_params(const float* __restrict__ params, long long P, float* s) {
  for (long long e = threadIdx.x; e < P; e += blockDim.x) s[e] = __ldg(params + e);
}

// Forward of one point with per-thread columns in shared memory:
// fcol[k*S], h1col[j*S], h2col[j*S]; returns the O outputs in out[].
__device__ __forceinline__ void point_forward(const MlpShape& m, const float* w, const float* __restrict__ feat_row,
                                              float* fcol, float* h1col, float* h2col, int S, float out[kMaxOut]) {
  const float* W1 = w;
  const float* b1 = W1 + m.H * m.D;
  const float* W2 = b1 + m.H;
  const float* b2 = W2 + m.H * m.H;
  const float* W3 = b2 + m.H;
  const float* b3 = W3 + m.O * m.H;
  for (int k = 0; k < m.D; ++k) fcol[k * S] = __ldg(feat_row + k);
  for (int j = 0; j < m.H; ++j) {
    float a = b1[j];
    for (int k = 0; k < m.D; ++k) a = fmaf(W1[j * m.D + k], fcol[k * S], a);
    h1col[j * S] = fmaxf(a, 0.0f);
  }
  for (int j = 0; j < m.H; ++j) {
    float a = b2[j];
    for (int k = 0; k < m.H; ++k) a = fmaf(W2[j * m.H + k], h1col[k * S], a);
    h2col[j * S] = fmaxf(a, 0.0f);
  }
  for (int o = 0; o < m.O; ++o) {
    float a = b3[o];
    for (int k = 0; k < m.H; ++k) a = fmaf(W3[o * m.H + k], h2col[k * S], a);
    out[o] = a;
  }
}

__global__ void __launch_bounds__(kThreads) plain_mlp_fwd_kernel(MlpShape m, const float* __restrict__ params,
                                                                 const float* __restrict__ feat, long long n,
                                                                 const long long* n_dev, float* __restrict__ delta) {
  extern __shared__ float smem[];
  float* w = smem;
  float* cols = smem + ((m.P + 3) & ~3ll);
  stage_params(params, m.P, w);
  __syncthreads();
  const long long cnt = count_of(n, n_dev);
  const int t = threadIdx.x;
  for (long long i = (long long)blockIdx.x * kThreads + t; i < cnt; i += (long long)gridDim.x * kThreads) {
    float out[kMaxOut];
    point_forward(m, w, feat + i * m.D, cols + t, cols + m.D * kThreads + t, cols + (m.D + m.H) * kThreads + t,
                  kThreads, out);
    for (int o = 0; o < m.O; ++o) delta[o * n + i] = out[o];
  }
}

// Per point: forward recompute, then back-propagation to dfeat; stores the
// activations and pre-activation gradients the weight reduction needs.
__global__ void __launch_bounds__(kThreads) plain_mlp_bwd_points(MlpShape m, const float* __restrict__ params,
                                                                 const float* __restrict__ feat, long long n,
                                                                 const long long* n_dev,
                                                                 const float* __restrict__ ddelta,
                                                                 float* __restrict__ dfeat, float* __restrict__ h1s,
                                                                 float* __restrict__ h2s, float* __restrict__ dz1s,
                                                                 float* __restrict__ dz2s) {
  extern __shared__ float smem[];
  float* w = smem;
  float* cols = smem + ((m.P + 3) & ~3ll);
  stage_params(params, m.P, w);
  __syncthreads();
  const float* W1 = w;
  const float* W2 = W1 + m.H * m.D + m.H;
  const float* W3 = W2 + m.H * m.H + m.H;
  const long long cnt = count_of(n, n_dev);
  const int t = threadIdx.x;
  float* fcol = cols + t;
  float* h1col = cols + m.D * kThreads + t;
  float* h2col = cols + (m.D + m.H) * kThreads + t;
  for (long long i = (long long)blockIdx.x * kThreads + t; i < cnt; i += (long long)gridDim.x * kThreads) {
    float out[kMaxOut];
    point_forward(m, w, feat + i * m.D, fcol, h1col, h2col, kThreads, out);
    float d[kMaxOut];
    for (int o = 0; o < m.O; ++o) d[o] = __ldg(ddelta + o * n + i);
    for (int j = 0; j < m.H; ++j) {
      h1s[j * n + i] = h1col[j * kThreads];
      h2s[j * n + i] = h2col[j * kThreads];
    }
    // dz2 = (W3^T d) * [z2 > 0]; kept in the h2 column
    for (int k = 0; k < m.H; ++k) {
      float a = 0.0f;
      for (int o = 0; o < m.O; ++o) a = fmaf(W3[o * m.H + k], d[o], a);
      a = h2col[k * kThreads] > 0.0f ? a : 0.0f;
      dz2s[k * n + i] = a;
      h2col[k * kThreads] = a;
    }
    // dz1 = (W2^T dz2) * [z1 > 0]; kept in the h1 column
    for (int k = 0; k < m.H; ++k) {
      float a = 0.0f;
      for (int j = 0; j < m.H; ++j) a = fmaf(W2[j * m.H + k], h2col[j * kThreads], a);
      a = h1col[k * kThreads] > 0.0f ? a : 0.0f;
      dz1s[k * n + i] = a;
      h1col[k * kThreads] = a;
    }
    // dfeat = W1^T dz1
    for (int k = 0; k < m.D; ++k) {
      float a = 0.0f;
      for (int j = 0; j < m.H; ++j) a = fmaf(W1[j * m.D + k], h1col[j * kThreads], a);
      dfeat[i * m.D + k] = a;
    }
  }
}

// One weight gradient: dW[a][b] += sum_p Z[p][a] A[p][b], db[a] += sum_p Z[p][a]
// with element (p, a) of Z at Z[p * zp + a * za] (likewise A).
struct WGrad {
  const float* Z;
  long long zp, za;
  int Ha;
  const float* A;
  long long ap, ab;
  int Hb;
  float* dW;
  float* db;
};

struct WGradSet {
  WGrad g[3];
};

constexpr int kWgThreads = 256;
constexpr int kChunk = 32;

__global__ void __launch_bounds__(kWgThreads) plain_wgrad_kernel(WGradSet set, long long n, const long long* n_dev) {
  __shared__ float Zs[kChunk][64];
  __shared__ float As[kChunk][64];
  const WGrad q = set.g[blockIdx.y];
  const long long cnt = count_of(n, n_dev);
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  float acc[4][4] = {};
  float bacc[4] = {};
  for (long long p0 = (long long)blockIdx.x * kChunk; p0 < cnt; p0 += (long long)gridDim.x * kChunk) {
    // walk the operand's contiguous axis with consecutive threads
    for (int e = t; e < kChunk * 64; e += kWgThreads) {
      const int p = q.zp == 1 ? e % kChunk : e / 64, c = q.zp == 1 ? e / kChunk : e % 64;
      const long long pi = p0 + p;
      Zs[p][c] = (pi < cnt && c < q.Ha) ? q.Z[pi * q.zp + c * q.za] : 0.0f;
    }
    for (int e = t; e < kChunk * 64; e += kWgThreads) {
      const int p = q.ap == 1 ? e % kChunk : e / 64, c = q.ap == 1 ? e / kChunk : e % 64;
      const long long pi = p0 + p;
      As[p][c] = (pi < cnt && c < q.Hb) ? q.A[pi * q.ap + c * q.ab] : 0.0f;
    }
    __syncthreads();
    for (int p = 0; p < kChunk; ++p) {
      float zr[4], ac[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) zr[r] = Zs[p][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) ac[c] = As[p][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        bacc[r] += zr[r];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(zr[r], ac[c], acc[r][c]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = ty * 4 + r;
    if (a >= q.Ha) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int b = tx * 4 + c;
      if (b < q.Hb) atomicAdd(q.dW + (long long)a * q.Hb + b, acc[r][c]);
    }
    if (tx == 0) atomicAdd(q.db + a, bacc[r]);
  }
}

int check_mlp(const dash_mlp* mlp, MlpShape* m) {
  if (mlp == nullptr || mlp->params == nullptr) return fail(DASH_ERR_INVALID_ARG, "mlp/params is NULL");
  if (mlp->d_in < 1 || mlp->d_hidden < 1 || mlp->d_out < 1) return fail(DASH_ERR_INVALID_ARG, "MLP widths must be >= 1");
  if (mlp->d_in > 64 || mlp->d_hidden > 64 || mlp->d_out > kMaxOut)
    return fail(DASH_ERR_UNSUPPORTED, "plain MLP supports D <= 64, H <= 64, O <= 16");
  m->D = mlp->d_in;
  m->H = mlp->d_hidden;
  m->O = mlp->d_out;
  m->P = param_count(m->D, m->H, m->O);
  return DASH_OK;
}

size_t point_smem(const MlpShape& m) {
  return (size_t)(((m.P + 3) & ~3ll) + (long long)(m.D + 2 * m.H) * kThreads) * sizeof(float);
}

int grid_points(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  const long long cap = 8ll * sm_count();
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace
}  // namespace dash

extern "C" {

int dash_plain_mlp_fwd(const dash_mlp* mlp, const float* feat, int64_t n, const int64_t* n_dev, float* delta_out,
                       void* stream) {
  DASH_NVTX_RANGE("dash_plain_mlp_fwd");
  using namespace dash;
  MlpShape m;
  if (int s = check_mlp(mlp, &m)) return s;
  if (n < 0) return fail(DASH_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return DASH_OK;
  if (feat == nullptr || delta_out == nullptr) return fail(DASH_ERR_INVALID_ARG, "feat/delta_out is NULL");
  const size_t smem = point_smem(m);
  if (int s = cuda_status(DASH_RT(cudaFuncSetAttribute(plain_mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem)),
                          "cudaFuncSetAttribute"))
    return s;
  plain_mlp_fwd_kernel<<<grid_points(n), kThreads, smem, as_stream(stream)>>>(
      m, mlp->params, feat, n, reinterpret_cast<const long long*>(n_dev), delta_out);
  return launch_status("plain_mlp_fwd_kernel");
}

size_t dash_plain_mlp_bwd_workspace_size(const dash_mlp* mlp, int64_t n) {
  if (mlp == nullptr || n < 0) return 0;
  return (size_t)4 * (size_t)mlp->d_hidden * (size_t)n * sizeof(float);
}

int dash_plain_mlp_bwd(const dash_mlp* mlp, const float* feat, int64_t n, const int64_t* n_dev,
                       const float* ddelta, float* dfeat_out, float* mlp_grad, void* ws, size_t ws_bytes,
                       void* stream) {
  DASH_NVTX_RANGE("dash_plain_mlp_bwd");
  using namespace dash;
  MlpShape m;
  if (int s = check_mlp(mlp, &m)) return s;
  if (n < 0) return fail(DASH_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return DASH_OK;
  if (feat == nullptr || ddelta == nullptr || dfeat_out == nullptr || mlp_grad == nullptr)
    return fail(DASH_ERR_INVALID_ARG, "feat/ddelta/dfeat_out/mlp_grad is NULL");
  if (ws == nullptr || ws_bytes < dash_plain_mlp_bwd_workspace_size(mlp, n))
    return fail(DASH_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes,
                dash_plain_mlp_bwd_workspace_size(mlp, n));
  cudaStream_t st = as_stream(stream);
  float* inter = static_cast<float*>(ws);
  float* h1s = inter;
  float* h2s = h1s + (size_t)m.H * n;
  float* dz1s = h2s + (size_t)m.H * n;
  float* dz2s = dz1s + (size_t)m.H * n;
  const long long* nd = reinterpret_cast<const long long*>(n_dev);
  const size_t smem = point_smem(m);
  int s = cuda_status(DASH_RT(cudaFuncSetAttribute(plain_mlp_bwd_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)),
                      "cudaFuncSetAttribute");
  if (s == DASH_OK) {
    plain_mlp_bwd_points<<<grid_points(n), kThreads, smem, st>>>(m, mlp->params, feat, n, nd, ddelta, dfeat_out, h1s,
                                                                 h2s, dz1s, dz2s);
    s = launch_status("plain_mlp_bwd_points");
  }
  if (s == DASH_OK) {
    float* gW1 = mlp_grad;
    float* gb1 = gW1 + (size_t)m.H * m.D;
    float* gW2 = gb1 + m.H;
    float* gb2 = gW2 + (size_t)m.H * m.H;
    float* gW3 = gb2 + m.H;
    float* gb3 = gW3 + (size_t)m.O * m.H;
    WGradSet set;
    // layer 1: Z = dz1 [H][n] (SoA), A = feat [n][D]
    set.g[0] = WGrad{dz1s, 1, n, m.H, feat, m.D, 1, m.D, gW1, gb1};
    // layer 2: Z = dz2, A = h1 (both SoA)
    set.g[1] = WGrad{dz2s, 1, n, m.H, h1s, 1, n, m.H, gW2, gb2};
    // layer 3: Z = ddelta [O][n], A = h2
    set.g[2] = WGrad{ddelta, 1, n, m.O, h2s, 1, n, m.H, gW3, gb3};
    long long blocks = (n + kChunk - 1) / kChunk;
    const long long cap = 2ll * sm_count();
    blocks = blocks < cap ? blocks : cap;
    plain_wgrad_kernel<<<dim3((unsigned)blocks, 3), kWgThreads, 0, st>>>(set, n, nd);
    s = launch_status("plain_wgrad_kernel");
  }
  return s;
}

}  // extern "C"
