// Batched collision detection between convex shapes (Sec. 2.1): one pair per thread, FP64.
#include "ds_collision.cuh"

namespace {

__global__ void __launch_bounds__(128) collide_kernel(int n, const int32_t* __restrict__ type_a,
                                                      const double* __restrict__ size_a,
                                                      const double* __restrict__ pose_a,
                                                      const int32_t* __restrict__ type_b,
                                                      const double* __restrict__ size_b,
                                                      const double* __restrict__ pose_b,
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
  ds::cd::collide(type_a[k], sa, pa, type_b[k], sb, pb, o);
  for (int i = 0; i < DS_COLLIDE_OUT; ++i) out[static_cast<size_t>(DS_COLLIDE_OUT) * k + i] = o[i];
}

}  // namespace

extern "C" ds_status ds_collide(int32_t n_pairs, const int32_t* type_a, const double* size_a,
                                const double* pose_a, const int32_t* type_b, const double* size_b,
                                const double* pose_b, double* out, void* stream) {
  if (n_pairs < 0) return DS_EINVAL;
  if (n_pairs == 0) return DS_OK;
  if (!type_a || !size_a || !pose_a || !type_b || !size_b || !pose_b || !out) return DS_EINVAL;
  const int threads = 128;
  const int blocks = (n_pairs + threads - 1) / threads;
  collide_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(n_pairs, type_a, size_a, pose_a,
                                                                              type_b, size_b, pose_b, out);
  return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ECUDA;
}
