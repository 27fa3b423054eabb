// scan.cu -- horizon, extremal-spin and stationary-limit scans over many
// spacetimes (Sec. 2.3, Eqs. 33-41): the parameter-space classification
// behind Figs. 2-4, one spacetime (or one spacetime and polar angle) per
// thread, in FP64.
//
// Delta(R) = R^2 H(R) + chi^2 (Eq. 33) and the stationary-limit function
// R^2 H(R) + chi^2 cos^2 theta (Eq. 40) are both R^2 H(R) plus a constant,
// so both take their minimum where R^2 H(R) does: at the extremal radius
// R_e of Eqs. 34-37, where 2 H + R H' = 0 (Eq. 36) and
// chi_e^2 = -R_e^2 H(R_e) (Eq. 37).  Each thread therefore
//   1. finds R_e as the maximiser of -R^2 H over (0, 50] (geometric scan,
//      then bisection of Eq. 36 between the neighbours of the best sample);
//   2. finds the largest root of R^2 H + c above R_e (c = chi^2 for R_+,
//      chi^2 cos^2 theta for R_s) by a downward geometric scan from R = 50
//      to the first sign change, bracketed below by R_e, where the function
//      is at its minimum, then bisection to the last representable bracket.
#include <cuda_runtime.h>

#include <algorithm>

#include "bh_common.cuh"
#include "internal.h"

namespace bhrt {

namespace {

constexpr double kScanTop = 50.0;      // no root is sought above R = 50
constexpr double kScanRatio = 0.99;    // geometric scan step
constexpr double kScanBottom = 1e-4;

__device__ __forceinline__ bool consts_of(const bh_spacetime& s, MetricConsts<double>& m) {
  if (!(fabs(s.chi) <= 1e6)) return false;  // NaN or absurd spin
  m.metric = s.metric;
  m.chi = s.chi;
  m.chi2 = s.chi * s.chi;
  m.il = 0.0;
  m.lc = s.lambda_c;
  m.ilc = 0.0;
  m.eta_lc = 0.0;
  if (s.metric == 1) {
    if (!(s.lambda_E > 0.0) || !(s.lambda_E < 1e300)) return false;
    m.il = 1.0 / s.lambda_E;
  } else if (s.metric == 2) {
    if (!(s.lambda_c > 0.0) || !(s.lambda_c < 1e300) || !(s.eta >= 0.0) || !(s.eta < 1e300))
      return false;
    m.ilc = 1.0 / s.lambda_c;
    m.eta_lc = s.eta * s.lambda_c;
  } else if (s.metric != 0) {
    return false;
  }
  return true;
}

// R^2 H(R), and Eq. (36)'s 2 H + R H' if asked; counts lapse evaluations.
__device__ __forceinline__ double r2H(const MetricConsts<double>& m, double R, double* g36,
                                      unsigned& ev) {
  ++ev;
  double H, dH;
  lapse(m, R, 1.0 / R, H, dH);
  if (g36) *g36 = 2.0 * H + R * dH;  // (R^2 H)' / R
  return R * R * H;
}

// Extremal radius and spin (Eqs. 34-37); chi_e = 0 where -R^2 H <= 0.
__device__ void extremal(const MetricConsts<double>& m, double& chi_e, double& R_e,
                         unsigned& ev) {
  double best = -INFINITY, Rb = kScanTop, R = kScanTop;
  while (R >= kScanBottom) {
    const double v = -r2H(m, R, nullptr, ev);
    if (v > best) {
      best = v;
      Rb = R;
    }
    R *= kScanRatio;
  }
  // -R^2 H rises below R_e (Eq. 36's 2H + R H' < 0) and falls above it
  double lo = Rb * kScanRatio, hi = Rb / kScanRatio;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double g;
    r2H(m, mid, &g, ev);
    if (g < 0.0) lo = mid; else hi = mid;
  }
  double Rx = 0.5 * (lo + hi);
  double v = -r2H(m, Rx, nullptr, ev);
  if (!(v >= best)) {  // the sampled maximum sits at the scan's edge
    Rx = Rb;
    v = best;
  }
  R_e = Rx;
  chi_e = v > 0.0 ? sqrt(v) : 0.0;
}

// Largest root of R^2 H(R) + c on (R_e, 50] given that R^2 H + c is at its
// minimum at R_e; returns false if there is none.
__device__ bool largest_root(const MetricConsts<double>& m, double c, double R_e, double& root,
                             unsigned& ev) {
  double hi = kScanTop;
  if (!(r2H(m, hi, nullptr, ev) + c > 0.0)) return false;
  if (!(r2H(m, R_e, nullptr, ev) + c <= 0.0)) return false;
  double lo = R_e;
  for (double R = hi * kScanRatio; R > R_e; R *= kScanRatio) {
    if (r2H(m, R, nullptr, ev) + c <= 0.0) {
      lo = R;
      break;
    }
    hi = R;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (r2H(m, mid, nullptr, ev) + c > 0.0) hi = mid; else lo = mid;
  }
  root = hi;
  return true;
}

// Warp sum of a per-thread count into *dst (one atomic per warp); every
// lane of the warp calls it.
__device__ __forceinline__ void add_count(unsigned long long* dst, unsigned v) {
  unsigned long long w = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(dst, w);
}

__global__ void __launch_bounds__(128) scan_horizon_kernel(ScanArgs a) {
  unsigned ev = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    MetricConsts<double> m;
    if (!consts_of(a.st[i], m)) {
      a.r_plus[i] = a.chi_e[i] = a.R_e[i] = 0.0;
      a.flags[i] = 2;
      continue;
    }
    double ce, Re, rp = 0.0;
    extremal(m, ce, Re, ev);
    const bool hz = largest_root(m, m.chi2, Re, rp, ev);
    a.chi_e[i] = ce;
    a.R_e[i] = Re;
    a.r_plus[i] = hz ? rp : 0.0;
    a.flags[i] = hz ? 0 : 1;
  }
  if (a.stats) add_count(&a.stats[0], ev);
}

__global__ void __launch_bounds__(128) scan_ergo_kernel(ScanArgs a) {
  unsigned ev = 0;
  const int64_t total = a.n * a.n_theta;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / a.n_theta;
    const int k = (int)(t - i * a.n_theta);
    MetricConsts<double> m;
    double rs = 0.0;
    if (consts_of(a.st[i], m)) {
      const double c = cos(a.theta[k]);
      if (!largest_root(m, m.chi2 * c * c, a.R_e[i], rs, ev)) rs = 0.0;
    }
    a.R_s[t] = rs;
  }
  if (a.stats) add_count(&a.stats[1], ev);
}

}  // namespace

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const int64_t cap = (int64_t)num_sms() * 16;
  int64_t blocks = std::min<int64_t>((a.n + 127) / 128, cap);
  scan_horizon_kernel<<<(int)blocks, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.n_theta == 0 || !a.R_s) return e;
  blocks = std::min<int64_t>((a.n * a.n_theta + 127) / 128, cap);
  scan_ergo_kernel<<<(int)blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bhrt
