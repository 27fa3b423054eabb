// products.cu -- image products: morphology diagnostics (Sec. 6.2-6.3,
// Eqs. 92-107) and the FP64 direct visibility sum (Sec. 6.4, Eq. 108).
//
// Diagnostics are two streaming passes over the image with FP64
// accumulation: pass 1 gives F, the centroid and the peak/mean contrast;
// pass 2 (which needs the centroid) gives the centroid-centred radial moments,
// the left/right split and the origin-centred radial profile; a one-block
// finish reduces the per-block partials in a fixed order.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace bhrt {

constexpr int kDiagThreads = 256;
constexpr int kDiagBlocks = 304;  // 2 x 152 SMs
constexpr int kP1 = 6;            // pass-1 partials per block
constexpr int kP2 = 4;            // pass-2 partials per block

struct DiagGeom {
  int nx, ny;
  double x_min, y_min, dx, dy;
  int nbins;
  double theta_g;
};

struct DiagWs {
  double* part1;   // [blocks][kP1]
  double* part2;   // [blocks][kP2]
  double* hsum;    // [nbins]
  unsigned long long* hcnt;  // [nbins]
  double* mid;     // F, X_c, Y_c
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction of n values per thread into out[0..n) (sum, or max for
// the entries flagged in max_mask).
template <int N>
__device__ __forceinline__ void block_reduce(double (&v)[N], unsigned max_mask, double* out) {
  __shared__ double s[N][kDiagThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    double x = ((max_mask >> t) & 1) ? warp_max(v[t]) : warp_sum(v[t]);
    if (lane == 0) s[t][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const int t = threadIdx.x;
    double acc = s[t][0];
    for (int k = 1; k < kDiagThreads / 32; ++k)
      acc = ((max_mask >> t) & 1) ? fmax(acc, s[t][k]) : acc + s[t][k];
    out[t] = acc;
  }
}

__global__ void __launch_bounds__(kDiagThreads) diag_pass1(const float* I, DiagGeom g, DiagWs w) {
  double v[kP1] = {0, 0, 0, 0, 0, 0};  // sum I, sum X I, sum Y I, max I, n(I>0), sum(I>0)
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(q % g.nx), j = (int)(q / g.nx);
    double x = g.x_min + (i + 0.5) * g.dx, y = g.y_min + (j + 0.5) * g.dy;
    double a = (double)I[q];
    v[0] += a;
    v[1] += x * a;
    v[2] += y * a;
    v[3] = fmax(v[3], a);
    if (a > 0.0) {
      v[4] += 1.0;
      v[5] += a;
    }
  }
  block_reduce<kP1>(v, 1u << 3, w.part1 + blockIdx.x * kP1);
}

__global__ void diag_mid(DiagGeom g, DiagWs w) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[kP1] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < kDiagBlocks; ++b)
    for (int t = 0; t < kP1; ++t)
      s[t] = (t == 3) ? fmax(s[t], w.part1[b * kP1 + t]) : s[t] + w.part1[b * kP1 + t];
  double dA = g.dx * g.dy;
  double F = s[0] * dA;                      // Eq. (92)
  w.mid[0] = F;
  w.mid[1] = s[1] * dA / F;                  // Eq. (93)
  w.mid[2] = s[2] * dA / F;
  w.mid[3] = s[3];                           // I_max
  w.mid[4] = s[4];
  w.mid[5] = s[5];
}

__global__ void __launch_bounds__(kDiagThreads) diag_pass2(const float* I, DiagGeom g, DiagWs w) {
  extern __shared__ unsigned char smem[];
  double* hs = reinterpret_cast<double*>(smem);
  unsigned* hc = reinterpret_cast<unsigned*>(hs + g.nbins);
  for (int b = threadIdx.x; b < g.nbins; b += blockDim.x) {
    hs[b] = 0.0;
    hc[b] = 0u;
  }
  __syncthreads();
  const double Xc = w.mid[1], Yc = w.mid[2];
  double v[kP2] = {0, 0, 0, 0};  // sum rho I, sum rho^2 I, F_R, F_L (pixel sums)
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(q % g.nx), j = (int)(q / g.nx);
    double x = g.x_min + (i + 0.5) * g.dx, y = g.y_min + (j + 0.5) * g.dy;
    double a = (double)I[q];
    double rho = sqrt((x - Xc) * (x - Xc) + (y - Yc) * (y - Yc));   // Eq. (95)
    v[0] += rho * a;
    v[1] += rho * rho * a;
    if (x > Xc) v[2] += a;                                         // Eq. (100)
    if (x < Xc) v[3] += a;
    double rho0 = sqrt(x * x + y * y);                             // Eq. (105)
    int b = (int)floor(rho0 / g.dx);
    if (b >= 0 && b < g.nbins) {
      atomicAdd(&hs[b], a);
      atomicAdd(&hc[b], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < g.nbins; b += blockDim.x) {
    if (hc[b]) {
      atomicAdd(&w.hsum[b], hs[b]);
      atomicAdd(&w.hcnt[b], (unsigned long long)hc[b]);
    }
  }
  block_reduce<kP2>(v, 0u, w.part2 + blockIdx.x * kP2);
}

__global__ void diag_final(DiagGeom g, DiagWs w, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[kP2] = {0, 0, 0, 0};
  for (int b = 0; b < kDiagBlocks; ++b)
    for (int t = 0; t < kP2; ++t) s[t] += w.part2[b * kP2 + t];
  const double dA = g.dx * g.dy, F = w.mid[0], Xc = w.mid[1], Yc = w.mid[2];
  const double rho_bar = s[0] * dA / F;                              // Eq. (96)
  const double var = s[1] * dA / F - rho_bar * rho_bar;              // Eq. (98)
  const double FR = s[2] * dA, FL = s[3] * dA;
  int best = -1;
  double best_v = -1.0;
  for (int b = 0; b < g.nbins; ++b) {
    if (!w.hcnt[b]) continue;
    double mean = w.hsum[b] / (double)w.hcnt[b];
    if (best < 0 || mean > best_v) {
      best_v = mean;
      best = b;
    }
  }
  const double rho_peak = (best + 0.5) * g.dx;
  out[0] = F;
  out[1] = Xc;
  out[2] = Yc;
  out[3] = sqrt(Xc * Xc + Yc * Yc);                                  // Eq. (94)
  out[4] = rho_bar;
  out[5] = 2.0 * rho_bar;                                            // Eq. (97)
  out[6] = sqrt(var > 0.0 ? var : 0.0);
  out[7] = (FR - FL) / (FR + FL);                                    // Eq. (99)
  out[8] = w.mid[3] / (w.mid[5] / w.mid[4]);                         // Eq. (101)
  out[9] = rho_peak;
  out[10] = 2.0 * rho_peak;                                          // Eq. (106)
  out[11] = 2.0 * rho_peak * g.theta_g;                              // Eq. (107)
}

// FP64 direct visibilities (Eq. 108), one block per baseline: the
// exponential factorises exactly into exp(-2 pi i u X_i) exp(-2 pi i v Y_j),
// so each block tabulates the u-phases of the image columns once and sums
// rows.  Phases use sincospi(2 u X) so the argument reduction is exact.
__global__ void __launch_bounds__(256) vis_direct_fp64(const float* I, DiagGeom g,
                                                       const double* uv, int64_t K,
                                                       double* V) {
  extern __shared__ double ph[];  // [2][nx]: cos, sin of 2 pi u X_i
  const int64_t k = blockIdx.x;
  if (k >= K) return;
  const double u = uv[2 * k], v = uv[2 * k + 1];
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
    double x = g.x_min + (i + 0.5) * g.dx, s, c;
    sincospi(2.0 * u * x, &s, &c);
    ph[i] = c;
    ph[g.nx + i] = s;
  }
  __syncthreads();
  double re = 0.0, im = 0.0;
  for (int j = threadIdx.x >> 5; j < g.ny; j += blockDim.x >> 5) {
    // warp per row: G_j = sum_i I_ji (cos - i sin)
    double gr = 0.0, gi = 0.0;
    const float* row = I + (int64_t)j * g.nx;
    for (int i = threadIdx.x & 31; i < g.nx; i += 32) {
      double a = (double)row[i];
      gr += a * ph[i];
      gi -= a * ph[g.nx + i];
    }
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    if ((threadIdx.x & 31) == 0) {
      double y = g.y_min + (j + 0.5) * g.dy, s, c;
      sincospi(2.0 * v * y, &s, &c);
      // (c - i s)(gr + i gi)
      re += c * gr + s * gi;
      im += c * gi - s * gr;
    }
  }
  __shared__ double red[2][8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = re;
    red[1][w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R = 0.0, M = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) {
      R += red[0][t];
      M += red[1][t];
    }
    const double dA = g.dx * g.dy;
    V[2 * k] = R * dA;
    V[2 * k + 1] = M * dA;
  }
}

}  // namespace bhrt

using namespace bhrt;

namespace {

bool geom_from(const bh_camera* cam, double theta_g, DiagGeom& g) {
  if (!cam || cam->nx < 1 || cam->ny < 1 || !(cam->x_max > cam->x_min) ||
      !(cam->y_max > cam->y_min) || !std::isfinite(theta_g))
    return false;
  g.nx = cam->nx;
  g.ny = cam->ny;
  g.x_min = cam->x_min;
  g.y_min = cam->y_min;
  g.dx = (cam->x_max - cam->x_min) / cam->nx;
  g.dy = (cam->y_max - cam->y_min) / cam->ny;
  double ax = std::fmax(std::fabs(cam->x_min), std::fabs(cam->x_max));
  double ay = std::fmax(std::fabs(cam->y_min), std::fabs(cam->y_max));
  g.nbins = (int)std::floor(std::sqrt(ax * ax + ay * ay) / g.dx) + 2;
  g.theta_g = theta_g;
  return g.nbins > 0 && g.nbins < (1 << 20);
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t diag_ws_layout(const DiagGeom& g, char* base, DiagWs* w) {
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o = a256(o + b);
    return base + at;
  };
  char* p1 = take(sizeof(double) * kDiagBlocks * kP1);
  char* p2 = take(sizeof(double) * kDiagBlocks * kP2);
  char* hs = take(sizeof(double) * g.nbins);
  char* hc = take(sizeof(unsigned long long) * g.nbins);
  char* mid = take(sizeof(double) * 8);
  if (w) {
    w->part1 = reinterpret_cast<double*>(p1);
    w->part2 = reinterpret_cast<double*>(p2);
    w->hsum = reinterpret_cast<double*>(hs);
    w->hcnt = reinterpret_cast<unsigned long long*>(hc);
    w->mid = reinterpret_cast<double*>(mid);
  }
  return o;
}

}  // namespace

extern "C" {

bh_status bh_diagnostics_workspace_size(const bh_camera* cam, size_t* bytes) {
  DiagGeom g;
  if (!bytes || !geom_from(cam, 1.0, g)) return BH_ERR_INVALID_ARG;
  *bytes = diag_ws_layout(g, nullptr, nullptr);
  return BH_OK;
}

bh_status bh_diagnostics(const float* I, const bh_camera* cam, double theta_g, double* out12,
                         void* workspace, size_t workspace_bytes, void* stream) {
  DiagGeom g;
  if (!I || !out12 || !geom_from(cam, theta_g, g)) return BH_ERR_INVALID_ARG;
  size_t need = diag_ws_layout(g, nullptr, nullptr);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return BH_ERR_WORKSPACE;
  // the profile histogram of pass 2 lives in shared memory: refuse or
  // configure it before anything is enqueued
  const size_t smem = (sizeof(double) + sizeof(unsigned)) * g.nbins;
  if (smem > 200 * 1024) return BH_ERR_INVALID_ARG;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(diag_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return BH_ERR_CUDA;
  DiagWs w;
  diag_ws_layout(g, static_cast<char*>(workspace), &w);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(w.hsum, 0, sizeof(double) * g.nbins, s) != cudaSuccess ||
      cudaMemsetAsync(w.hcnt, 0, sizeof(unsigned long long) * g.nbins, s) != cudaSuccess)
    return BH_ERR_CUDA;
  diag_pass1<<<kDiagBlocks, kDiagThreads, 0, s>>>(I, g, w);
  diag_mid<<<1, 32, 0, s>>>(g, w);
  diag_pass2<<<kDiagBlocks, kDiagThreads, smem, s>>>(I, g, w);
  diag_final<<<1, 32, 0, s>>>(g, w, out12);
  return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

bh_status bh_visibilities_fp64(const float* I, const bh_camera* cam, const double* uv, int64_t K,
                               double* V, void* stream) {
  DiagGeom g;
  if (!I || (K > 0 && (!uv || !V)) || K < 0 || !geom_from(cam, 1.0, g)) return BH_ERR_INVALID_ARG;
  if (K == 0) return BH_OK;
  if (K > 0x7fffffff) return BH_ERR_INVALID_ARG;
  size_t smem = sizeof(double) * 2 * g.nx;
  if (smem > 200 * 1024) return BH_ERR_INVALID_ARG;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(vis_direct_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return BH_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  vis_direct_fp64<<<(unsigned)K, 256, smem, s>>>(I, g, uv, K, V);
  return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Diagnostics without caller-provided scratch.
//
// Some callers cannot allocate device memory at the point where they need the
// diagnostics: code running inside a host framework that owns every device
// allocation through its own pool, plugins that are handed only input and
// output buffers, or loops that must not call cudaMalloc/cudaFree for timing
// reasons.  For them the scratch of the two-pass reduction (block partials
// and the radial-profile histogram) lives in a fixed file-scope device array,
// kNoAllocScratchBytes long, which every GPU that loads this library keeps
// until the process exits.  The host needs the array's device address: it is
// looked up once per device with cudaGetSymbolAddress (the host-side symbol
// is only a stand-in) and cached for the life of the process; a
// cudaDeviceReset reloads the module, which makes a cached address stale, so
// callers that reset a device must not use this entry point on it afterwards.
namespace {

constexpr size_t kNoAllocScratchBytes = 256 * 1024;
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_diag_scratch[kNoAllocScratchBytes];

namespace {

void* g_scratch_addr[kNoAllocMaxDevices];
int g_scratch_ready[kNoAllocMaxDevices];

// Device address of the scratch array on the current device (nullptr on
// failure).  The first call on a device does the lookup.
void* noalloc_scratch() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
  if (__atomic_load_n(&g_scratch_ready[dev], __ATOMIC_ACQUIRE)) return g_scratch_addr[dev];
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_diag_scratch) != cudaSuccess || !p) return nullptr;
  g_scratch_addr[dev] = p;
  __atomic_store_n(&g_scratch_ready[dev], 1, __ATOMIC_RELEASE);
  return p;
}

}  // namespace

extern "C" bh_status bh_diagnostics_noalloc(const float* I, const bh_camera* cam, double theta_g,
                                            double* out12, void* stream) {
  DiagGeom g;
  if (!I || !out12 || !geom_from(cam, theta_g, g)) return BH_ERR_INVALID_ARG;
  if (diag_ws_layout(g, nullptr, nullptr) > kNoAllocScratchBytes) return BH_ERR_WORKSPACE;
  void* scratch = noalloc_scratch();
  if (!scratch) return BH_ERR_CUDA;
  return bh_diagnostics(I, cam, theta_g, out12, scratch, kNoAllocScratchBytes, stream);
}
