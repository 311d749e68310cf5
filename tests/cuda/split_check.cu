// Test helper (built by tests/test_gpu_split.py): checks the integer-operation splits of
// rb_internal.cuh against the plain conversions, value by value, on the GPU.
//   df_split(v)   == (h = (float)v, l = (float)(v - (double)h))   bit for bit (NaN: both NaN)
//   f32_to_f64(x) == (double)x                                     bit for bit
#include <cuda_runtime.h>

#include "rb_internal.cuh"

namespace {

__device__ bool same_f(float a, float b) {
  return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}
__device__ bool same_d(double a, double b) {
  return (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
}

__global__ void k_check(const double *v, int n, const float *x, int nx, int *bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float h, l;
    rb::df_split(v[i], h, l);
    const float hr = (float)v[i];
    const float lr = (float)(v[i] - (double)hr);
    if (!same_f(h, hr) || !same_f(l, lr)) atomicMin(bad, i);
  }
  if (i < nx) {
    if (!same_d(rb::f32_to_f64(x[i]), (double)x[i])) atomicMin(bad + 1, i);
  }
}

}  // namespace

// Returns 0 when every value agrees; bad[0] / bad[1]: first mismatching index of v / x, or
// INT_MAX. Negative: a CUDA error.
extern "C" int split_check(const double *h_v, int n, const float *h_x, int nx, int *bad) {
  double *dv = nullptr;
  float *dx = nullptr;
  int *db = nullptr;
  const int init[2] = {0x7fffffff, 0x7fffffff};
  int rc = -1;
  if (cudaMalloc(&dv, 8 * (size_t)(n > 0 ? n : 1)) != cudaSuccess) goto done;
  if (cudaMalloc(&dx, 4 * (size_t)(nx > 0 ? nx : 1)) != cudaSuccess) goto done;
  if (cudaMalloc(&db, 8) != cudaSuccess) goto done;
  if (cudaMemcpy(dv, h_v, 8 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) goto done;
  if (cudaMemcpy(dx, h_x, 4 * (size_t)nx, cudaMemcpyHostToDevice) != cudaSuccess) goto done;
  if (cudaMemcpy(db, init, 8, cudaMemcpyHostToDevice) != cudaSuccess) goto done;
  {
    const int m = n > nx ? n : nx;
    k_check<<<(m + 255) / 256, 256>>>(dv, n, dx, nx, db);
  }
  if (cudaMemcpy(bad, db, 8, cudaMemcpyDeviceToHost) != cudaSuccess) goto done;
  rc = (bad[0] == 0x7fffffff && bad[1] == 0x7fffffff) ? 0 : 1;
done:
  cudaFree(dv);
  cudaFree(dx);
  cudaFree(db);
  return rc;
}
