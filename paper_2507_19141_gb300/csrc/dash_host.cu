// dash_host.cu -- host side of the libdash C ABI: status strings, the
// thread-local error message, the Eq. 7 level layout and argument checks.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>

#include "dash_internal.cuh"

namespace dash {

static thread_local char g_last_error[512] = "";

int g_opt_fwd_form = 0;
int g_opt_bwd_form = 0;
int g_opt_access_form = 0;
int g_opt_grad_replicas = 16;
int g_opt_decomp_form = 0;

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return status;
}

// Fault injection: g_fault_at > 0 names the g_fault_at-th checked runtime
// call after arming; g_rt_calls counts the checked calls since then.
static std::atomic<long long> g_fault_at{0};
static std::atomic<long long> g_rt_calls{0};
static thread_local bool g_injected = false;

bool fault_due() {
  const long long k = g_rt_calls.fetch_add(1, std::memory_order_relaxed) + 1;
  const long long at = g_fault_at.load(std::memory_order_relaxed);
  if (at > 0 && k == at) {
    g_injected = true;
    return true;
  }
  return false;
}

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DASH_OK;
  if (g_injected) {
    g_injected = false;
    return fail(DASH_ERR_CUDA, "%s: injected failure (dash_debug_fail_cuda_call), call not made", what);
  }
  return fail(DASH_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int launch_status(const char* what) { return cuda_status(DASH_RT(cudaGetLastError()), what); }

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cached[dev] = v;
  }
  return cached[dev];
}

int make_geom(const dash_layout* lo, Geom* g) {
  if (lo == nullptr || g == nullptr) return fail(DASH_ERR_INVALID_ARG, "layout is NULL");
  if (!(lo->dims == 0 || lo->dims == 4)) return fail(DASH_ERR_INVALID_ARG, "needs a 4-D layout (dims = %d)", lo->dims);
  if (lo->L < 1 || lo->L > DASH_MAX_LEVELS) return fail(DASH_ERR_UNSUPPORTED, "L=%d outside [1,32]", lo->L);
  if (!(lo->F == 1 || lo->F == 2 || lo->F == 4 || lo->F == 8))
    return fail(DASH_ERR_UNSUPPORTED, "F=%d not in {1,2,4,8}", lo->F);
  if (lo->log2_T < 4 || lo->log2_T > 28) return fail(DASH_ERR_UNSUPPORTED, "log2_T=%d outside [4,28]", lo->log2_T);
  memset(g, 0, sizeof(*g));
  g->L = lo->L;
  g->F = lo->F;
  g->mask = (uint32_t)((1ull << lo->log2_T) - 1ull);
  for (int i = 0; i < 4; ++i) g->primes[i] = lo->primes[i];
  for (int l = 0; l < lo->L; ++l) {
    if (lo->res_s[l] < 1 || lo->res_t[l] < 1) return fail(DASH_ERR_INVALID_ARG, "level %d has resolution < 1", l);
    g->res_s[l] = lo->res_s[l];
    g->res_t[l] = lo->res_t[l];
    if (lo->dense[l]) g->dense_bits |= 1u << l;
    g->offset[l] = lo->offset[l];
  }
  return DASH_OK;
}

// Point-row bounds of DASH_DEBUG builds (dash_debug_set_point_rows).
#ifdef DASH_DEBUG
static long long g_point_rows = -1;
#endif
__device__ unsigned int g_bounds_flags;

unsigned int* bounds_flags_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_bounds_flags) != cudaSuccess) return nullptr;
  return static_cast<unsigned int*>(p);
}

int make_pts(const dash_points* p, Pts* out) {
  if (p == nullptr) return fail(DASH_ERR_INVALID_ARG, "points is NULL");
  if (p->n < 0) return fail(DASH_ERR_INVALID_ARG, "n=%lld < 0", (long long)p->n);
  if (p->n > 0 && (p->x == nullptr || p->y == nullptr || p->z == nullptr || p->t == nullptr))
    return fail(DASH_ERR_INVALID_ARG, "coordinate pointer is NULL");
  if (p->t_stride < 0) return fail(DASH_ERR_INVALID_ARG, "t_stride < 0");
  if (p->n >= (1ll << 31)) return fail(DASH_ERR_UNSUPPORTED, "n >= 2^31");
  out->x = p->x;
  out->y = p->y;
  out->z = p->z;
  out->t = p->t;
  out->t_stride = p->t_stride;
  out->idx = p->idx;
  out->n = p->n;
  out->n_dev = reinterpret_cast<const long long*>(p->n_dev);
  out->rows = -1;
  out->bounds = nullptr;
#ifdef DASH_DEBUG
  if (g_point_rows >= 0) {
    out->bounds = bounds_flags_ptr();
    if (out->bounds == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the bounds flag word");
    out->rows = g_point_rows;
  }
#endif
  return DASH_OK;
}

// Eq. 7: geometric progression of resolutions between N_min and N_max.
static int32_t level_resolution(double nmin, double nmax, int L, int l) {
  if (L == 1) return (int32_t)floor(nmin + 1e-9);
  const double growth = exp((log(nmax) - log(nmin)) / (double)(L - 1));
  return (int32_t)floor(nmin * pow(growth, (double)l) + 1e-9);
}

}  // namespace dash

extern "C" {

const char* dash_status_string(int s) {
  switch (s) {
    case DASH_OK: return "DASH_OK";
    case DASH_ERR_INVALID_ARG: return "DASH_ERR_INVALID_ARG";
    case DASH_ERR_UNSUPPORTED: return "DASH_ERR_UNSUPPORTED";
    case DASH_ERR_WORKSPACE: return "DASH_ERR_WORKSPACE";
    case DASH_ERR_CUDA: return "DASH_ERR_CUDA";
    case DASH_ERR_BOUNDS: return "DASH_ERR_BOUNDS";
    case DASH_ERR_TIMEOUT: return "DASH_ERR_TIMEOUT";
    default: return "DASH_ERR_UNKNOWN";
  }
}

const char* dash_last_error(void) { return dash::g_last_error; }

int dash_debug_fail_cuda_call(int64_t n) {
  if (n < 0) return dash::fail(DASH_ERR_INVALID_ARG, "n=%lld < 0", (long long)n);
  dash::g_fault_at.store(0, std::memory_order_relaxed);
  dash::g_rt_calls.store(0, std::memory_order_relaxed);
  dash::g_fault_at.store((long long)n, std::memory_order_relaxed);
  return DASH_OK;
}

int64_t dash_debug_cuda_call_count(void) { return (int64_t)dash::g_rt_calls.load(std::memory_order_relaxed); }

int dash_debug_set_point_rows(int64_t rows) {
#ifdef DASH_DEBUG
  if (rows < -1) return dash::fail(DASH_ERR_INVALID_ARG, "rows=%lld < -1", (long long)rows);
  dash::g_point_rows = rows;
  return DASH_OK;
#else
  (void)rows;
  return dash::fail(DASH_ERR_UNSUPPORTED, "point-row bounds checks need the DASH_DEBUG build (libdash_debug.so)");
#endif
}

int dash_version(void) { return 102; }

int dash_set_option(int option, int value) {
  switch (option) {
    case DASH_OPT_FWD_FORM:
      if (!(value == 0 || value == 1 || value == 2 || value == 4 || (value >= 10 && value <= 15)))
        return dash::fail(DASH_ERR_INVALID_ARG, "forward form %d not in {0, 1, 2, 4, 10..15}", value);
      dash::g_opt_fwd_form = value;
      return DASH_OK;
    case DASH_OPT_BWD_FORM:
      if (!(value == 0 || value == 1 || (value >= 10 && value <= 14)))
        return dash::fail(DASH_ERR_INVALID_ARG, "backward form %d not in {0, 1, 10..14}", value);
      dash::g_opt_bwd_form = value;
      return DASH_OK;
    case DASH_OPT_ACCESS_FORM:
      if (!(value == 0 || value == 1))
        return dash::fail(DASH_ERR_INVALID_ARG, "access form %d not in {0, 1}", value);
      dash::g_opt_access_form = value;
      return DASH_OK;
    case DASH_OPT_GRAD_REPLICAS:
      if (value < 0 || value > 64)
        return dash::fail(DASH_ERR_INVALID_ARG, "gradient replicas %d not in [0, 64]", value);
      dash::g_opt_grad_replicas = value;
      return DASH_OK;
    case DASH_OPT_DECOMP_FORM:
      if (!(value == 0 || value == 1))
        return dash::fail(DASH_ERR_INVALID_ARG, "decomposition form %d not in {0, 1}", value);
      dash::g_opt_decomp_form = value;
      return DASH_OK;
    default: return dash::fail(DASH_ERR_INVALID_ARG, "unknown option %d", option);
  }
}

int dash_device_status(void* stream) {
  DASH_NVTX_RANGE("dash_device_status");
  using namespace dash;
  if (int s = cuda_status(DASH_RT(cudaStreamSynchronize(as_stream(stream))), "cudaStreamSynchronize")) return s;
  {
    // a point row out of range (DASH_DEBUG builds) is reported first
    unsigned int* b = bounds_flags_ptr();
    if (b == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve the bounds flag word");
    unsigned int v = 0u;
    if (int s = cuda_status(DASH_RT(cudaMemcpy(&v, b, sizeof(v), cudaMemcpyDeviceToHost)), "cudaMemcpy(bounds)")) return s;
    if (v != 0u) {
      if (int s = cuda_status(DASH_RT(cudaMemset(b, 0, sizeof(v))), "cudaMemset(bounds)")) return s;
      return fail(DASH_ERR_BOUNDS, "a point row index was outside [0, rows); those points were skipped");
    }
  }
  unsigned int* words[5] = {fused::fwd_flags_ptr(), fused::bwd_flags_ptr(), fused::batch_flags_ptr(),
                            fused::selftest_flags_ptr(), fused::decomp_flags_ptr()};
  unsigned int seen = 0u;
  for (unsigned int* w : words) {
    if (w == nullptr) return fail(DASH_ERR_CUDA, "cannot resolve a device flag word");
    unsigned int v = 0u;
    if (int s = cuda_status(DASH_RT(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost)), "cudaMemcpy(flags)")) return s;
    if (v != 0u) {
      seen |= v;
      if (int s = cuda_status(DASH_RT(cudaMemset(w, 0, sizeof(v))), "cudaMemset(flags)")) return s;
    }
  }
  if (seen != 0u) return fail(DASH_ERR_TIMEOUT, "a bounded device-side wait gave up (flags %#x); outputs of that launch are incomplete", seen);
  return DASH_OK;
}

int dash_get_option(int option) {
  switch (option) {
    case DASH_OPT_FWD_FORM: return dash::g_opt_fwd_form;
    case DASH_OPT_BWD_FORM: return dash::g_opt_bwd_form;
    case DASH_OPT_ACCESS_FORM: return dash::g_opt_access_form;
    case DASH_OPT_GRAD_REPLICAS: return dash::g_opt_grad_replicas;
    case DASH_OPT_DECOMP_FORM: return dash::g_opt_decomp_form;
    default: return dash::fail(DASH_ERR_INVALID_ARG, "unknown option %d", option);
  }
}

int dash_hash4d_layout(const dash_hash4d_cfg* cfg, dash_layout* out) {
  using dash::fail;
  if (cfg == nullptr || out == nullptr) return fail(DASH_ERR_INVALID_ARG, "cfg/out is NULL");
  if (cfg->L < 1 || cfg->L > DASH_MAX_LEVELS) return fail(DASH_ERR_UNSUPPORTED, "L=%d outside [1,32]", cfg->L);
  if (!(cfg->F == 1 || cfg->F == 2 || cfg->F == 4 || cfg->F == 8))
    return fail(DASH_ERR_UNSUPPORTED, "F=%d not in {1,2,4,8}", cfg->F);
  if (cfg->log2_T < 4 || cfg->log2_T > 28) return fail(DASH_ERR_UNSUPPORTED, "log2_T=%d outside [4,28]", cfg->log2_T);
  if (!(cfg->nmin_s >= 1.0) || !(cfg->nmax_s >= cfg->nmin_s) || !(cfg->nmin_t >= 1.0) ||
      !(cfg->nmax_t >= cfg->nmin_t) || cfg->nmax_s > 65535.0 || cfg->nmax_t > 65535.0)
    return fail(DASH_ERR_INVALID_ARG, "resolutions must satisfy 1 <= N_min <= N_max <= 65535");
  memset(out, 0, sizeof(*out));
  out->L = cfg->L;
  out->F = cfg->F;
  out->log2_T = cfg->log2_T;
  for (int i = 0; i < 4; ++i) out->primes[i] = cfg->primes[i];
  const int64_t T = (int64_t)1 << cfg->log2_T;
  int64_t start = 0;
  for (int l = 0; l < cfg->L; ++l) {
    const int32_t ns = dash::level_resolution(cfg->nmin_s, cfg->nmax_s, cfg->L, l);
    const int32_t nt = dash::level_resolution(cfg->nmin_t, cfg->nmax_t, cfg->L, l);
    out->res_s[l] = ns;
    out->res_t[l] = nt;
    const int64_t r = (int64_t)ns + 1;
    const int64_t vertices = r * r * r * ((int64_t)nt + 1);
    out->dense[l] = vertices <= T ? 1 : 0;
    out->size[l] = out->dense[l] ? vertices : T;
    out->offset[l] = start;
    start = (start + out->size[l] + 7) & ~(int64_t)7;  // next level on a multiple of 8 entries
  }
  out->offset[cfg->L] = start;
  return DASH_OK;
}

}  // extern "C"
