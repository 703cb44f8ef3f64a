// Test probe (not part of the library): applies one float-float primitive of fm_df64.cuh to
// every input on the GPU and returns the results as float64, for tests/test_gpu_df64.py.
// Inputs are float64 values split into (hi, lo) float pairs exactly as the IP kernel's state.
#include <cuda_runtime.h>

#include "fm_df64.cuh"

using namespace fm;

__device__ __forceinline__ df split(double d) { return df_from_double(d); }

__global__ void probe(int op, const double* __restrict__ a, const double* __restrict__ b, int n,
                      double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const df x = split(a[i]);
  df r;
  switch (op) {
    case 0: r = df_add(x, split(b[i])); break;
    case 1: r = df_mul(x, split(b[i])); break;
    case 2: r = df_rcp(x); break;
    case 3: r = df_sqrt(x); break;
    case 4: r = df_rsqrt(x); break;
    default: r = df_logf(x); break;
  }
  out[i] = df_to_double(r);
}

// The float-float value the kernel saw for each input (hi + lo as float64).
__global__ void as_seen(const double* __restrict__ a, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = df_to_double(split(a[i]));
}

extern "C" int df64_probe(int op, const double* a_host, const double* b_host, int n, double* out_host,
                          double* seen_a, double* seen_b) {
  double *a = nullptr, *b = nullptr, *o = nullptr;
  const size_t bytes = (size_t)n * sizeof(double);
  if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess ||
      cudaMalloc(&o, bytes) != cudaSuccess)
    return 1;
  cudaMemcpy(a, a_host, bytes, cudaMemcpyHostToDevice);
  cudaMemcpy(b, b_host, bytes, cudaMemcpyHostToDevice);
  const int blocks = (n + 255) / 256;
  probe<<<blocks, 256>>>(op, a, b, n, o);
  cudaMemcpy(out_host, o, bytes, cudaMemcpyDeviceToHost);
  as_seen<<<blocks, 256>>>(a, n, o);
  cudaMemcpy(seen_a, o, bytes, cudaMemcpyDeviceToHost);
  as_seen<<<blocks, 256>>>(b, n, o);
  cudaMemcpy(seen_b, o, bytes, cudaMemcpyDeviceToHost);
  const int err = cudaDeviceSynchronize() != cudaSuccess;
  cudaFree(a);
  cudaFree(b);
  cudaFree(o);
  return err;
}
