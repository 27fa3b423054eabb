// Test probe: evaluates the sine/cosine, log(1 + x), exp, reciprocal and
// reciprocal square root of the
// tracing kernels (bh_common.cuh) in FP32 and FP64 on given arguments, for
// the accuracy tests in test_gpu_fastmath.py.  Test infrastructure, not part
// of the library.
#include <cuda_runtime.h>

#include "bh_common.cuh"

__global__ void probe_f32(int n, const float* x, float* s, float* c, float* l) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a, b;
  bhrt::d_sincos(x[i], &a, &b);
  s[i] = a;
  c[i] = b;
  l[i] = bhrt::d_log1p(x[i]);
}

__global__ void probe_f64(int n, const double* x, double* s, double* c, double* l, double* e,
                          double* r, double* q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a, b;
  bhrt::d_sincos(x[i], &a, &b);
  s[i] = a;
  c[i] = b;
  l[i] = bhrt::d_log1p(x[i]);
  e[i] = bhrt::d_exp(x[i]);
  r[i] = bhrt::d_rcp(x[i]);
  q[i] = x[i] > 0.0 ? bhrt::d_rsqrt(x[i]) : 0.0;
}

extern "C" int fastmath_probe_f32(int n, const float* x, float* s, float* c, float* l) {
  if (n <= 0) return 0;
  probe_f32<<<(n + 255) / 256, 256>>>(n, x, s, c, l);
  return (int)cudaDeviceSynchronize();
}

extern "C" int fastmath_probe_f64(int n, const double* x, double* s, double* c, double* l,
                                  double* e, double* r, double* q) {
  if (n <= 0) return 0;
  probe_f64<<<(n + 255) / 256, 256>>>(n, x, s, c, l, e, r, q);
  return (int)cudaDeviceSynchronize();
}
