// Batched collision detection between convex shapes (Sec. 2.1) and its randomized-smoothing
// derivative (App. C): one pair per thread, FP64.
#include "ds_collision.cuh"

namespace {

template <bool kHulls>
__global__ void __launch_bounds__(128) collide_kernel(int n, const int32_t* __restrict__ type_a,
                                                      const double* __restrict__ size_a,
                                                      const double* __restrict__ pose_a,
                                                      const int32_t* __restrict__ type_b,
                                                      const double* __restrict__ size_b,
                                                      const double* __restrict__ pose_b,
                                                      const double* __restrict__ hv, int n_hv,
                                                      double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double sa[3], sb[3], pa[12], pb[12], o[DS_COLLIDE_OUT];
  for (int i = 0; i < 3; ++i) {
    sa[i] = size_a[3 * k + i];
    sb[i] = size_b[3 * k + i];
  }
  for (int i = 0; i < 12; ++i) {
    pa[i] = pose_a[12 * k + i];
    pb[i] = pose_b[12 * k + i];
  }
  ds::cd::collide<kHulls>(type_a[k], sa, pa, type_b[k], sb, pb, hv, n_hv, o);
  for (int i = 0; i < DS_COLLIDE_OUT; ++i) out[static_cast<size_t>(DS_COLLIDE_OUT) * k + i] = o[i];
}

template <bool kHulls>
__global__ void __launch_bounds__(128) collide_smoothed_kernel(
    int n, const int32_t* __restrict__ type_a, const double* __restrict__ size_a,
    const double* __restrict__ pose_a, const int32_t* __restrict__ type_b, const double* __restrict__ size_b,
    const double* __restrict__ pose_b, const double* __restrict__ hv, int n_hv, int samples,
    const double* __restrict__ eps, double sigma,
    double* __restrict__ jac) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double sa[3], sb[3], pa[12], pb[12], J[84];
  for (int i = 0; i < 3; ++i) {
    sa[i] = size_a[3 * k + i];
    sb[i] = size_b[3 * k + i];
  }
  for (int i = 0; i < 12; ++i) {
    pa[i] = pose_a[12 * k + i];
    pb[i] = pose_b[12 * k + i];
  }
  ds::cd::smoothing_jacobian<kHulls>(type_a[k], sa, pa, type_b[k], sb, pb, hv, n_hv, samples, eps, sigma, J);
  for (int i = 0; i < 84; ++i) jac[static_cast<size_t>(84) * k + i] = J[i];
}

}  // namespace

extern "C" ds_status ds_collide_smoothed(int32_t n_pairs, const int32_t* type_a, const double* size_a,
                                         const double* pose_a, const int32_t* type_b, const double* size_b,
                                         const double* pose_b, const double* hull_vertices,
                                         int32_t n_hull_vertices, int32_t n_samples, const double* eps,
                                         double sigma, double* jac, void* stream) {
  if (n_pairs < 0 || n_hull_vertices < 0) return DS_EINVAL;
  if (n_pairs == 0) return DS_OK;
  if (!type_a || !size_a || !pose_a || !type_b || !size_b || !pose_b || !eps || !jac) return DS_EINVAL;
  if (n_samples <= 0 || !(sigma > 0.0) || !(sigma < 1e300)) return DS_EINVAL;
  const int threads = 128;
  const int blocks = (n_pairs + threads - 1) / threads;
  // without a hull pool no pair can be a valid hull: the form without hulls (a tenth of the state)
  if (hull_vertices && n_hull_vertices > 0)
    collide_smoothed_kernel<true><<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_pairs, type_a, size_a, pose_a, type_b, size_b, pose_b, hull_vertices, n_hull_vertices, n_samples, eps,
        sigma, jac);
  else
    collide_smoothed_kernel<false><<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_pairs, type_a, size_a, pose_a, type_b, size_b, pose_b, nullptr, 0, n_samples, eps, sigma, jac);
  return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ECUDA;
}

extern "C" ds_status ds_collide(int32_t n_pairs, const int32_t* type_a, const double* size_a,
                                const double* pose_a, const int32_t* type_b, const double* size_b,
                                const double* pose_b, const double* hull_vertices, int32_t n_hull_vertices,
                                double* out, void* stream) {
  if (n_pairs < 0 || n_hull_vertices < 0) return DS_EINVAL;
  if (n_pairs == 0) return DS_OK;
  if (!type_a || !size_a || !pose_a || !type_b || !size_b || !pose_b || !out) return DS_EINVAL;
  const int threads = 128;
  const int blocks = (n_pairs + threads - 1) / threads;
  // without a hull pool no pair can be a valid hull: the form without hulls (a tenth of the state)
  if (hull_vertices && n_hull_vertices > 0)
    collide_kernel<true><<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_pairs, type_a, size_a, pose_a, type_b, size_b, pose_b, hull_vertices, n_hull_vertices, out);
  else
    collide_kernel<false><<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_pairs, type_a, size_a, pose_a, type_b, size_b, pose_b, nullptr, 0, out);
  return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ECUDA;
}
