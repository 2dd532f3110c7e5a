// FMA-throughput probe used to measure the FP64 / FP32 CUDA-core peaks of the device.
#include "ds_common.cuh"

template <typename T>
__global__ void __launch_bounds__(256) fma_probe(double* out, int iters) {
  T a0 = T(threadIdx.x) * T(1e-3), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  const T b = T(0.999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
    a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
    a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = double(a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7);
}

extern "C" ds_status ds_fma_peak(double* out, int32_t blocks, int32_t iters, int32_t fp64, void* stream) {
  if (!out || blocks <= 0 || iters <= 0) return DS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fp64) fma_probe<double><<<blocks, 256, 0, s>>>(out, iters);
  else fma_probe<float><<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ECUDA;
}
