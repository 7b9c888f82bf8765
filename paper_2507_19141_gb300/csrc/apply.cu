// apply.cu -- backward of Eq. 10's in-place update (x' = x + dx, r' = r + dr,
// s' = s + ds at the dynamic rows): the gradient of each dynamic Gaussian's
// offsets is its rows of dL/d(attributes).  Gathers them from the full SoA
// [O][n_all] into the decoder's upstream gradient SoA [O][n] (compact order).
#include "dash_internal.cuh"

namespace dash {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) apply_bwd_kernel(Pts pts, int O, const float* __restrict__ dattrs,
                                                             long long n_all, float* __restrict__ ddelta) {
  const long long n = point_count(pts);
  const long long k = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (k >= n) return;
  const long long i = point_row(pts, k);
#ifdef DASH_DEBUG
  if (i < 0) return;
#endif
  for (int j = 0; j < O; ++j) __stcs(ddelta + (long long)j * pts.n + k, __ldg(dattrs + (long long)j * n_all + i));
}

}  // namespace
}  // namespace dash

extern "C" int dash_deform_apply_bwd(const dash_points* pts, int d_out, const float* dattrs, int64_t n_all,
                                     float* ddelta, void* stream) {
  DASH_NVTX_RANGE("dash_deform_apply_bwd");
  using namespace dash;
  Pts p;
  if (int s = make_pts(pts, &p)) return s;
  if (d_out < 1 || d_out > 16) return fail(DASH_ERR_UNSUPPORTED, "d_out=%d outside [1,16]", d_out);
  if (n_all < 0) return fail(DASH_ERR_INVALID_ARG, "n_all < 0");
  if (p.n == 0) return DASH_OK;
  if (dattrs == nullptr || ddelta == nullptr) return fail(DASH_ERR_INVALID_ARG, "dattrs/ddelta is NULL");
  apply_bwd_kernel<<<(unsigned)((p.n + kThreads - 1) / kThreads), kThreads, 0, as_stream(stream)>>>(p, d_out, dattrs,
                                                                                                    n_all, ddelta);
  return launch_status("apply_bwd_kernel");
}
