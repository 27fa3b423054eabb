// scan.cu -- horizon, extremal-spin and stationary-limit scans over many
// spacetimes (Sec. 2.3, Eqs. 33-41): the parameter-space classification
// behind Figs. 2-4, one spacetime per thread, in FP64.
//
// Delta(R) = R^2 H(R) + chi^2 (Eq. 33) and the stationary-limit function
// R^2 H(R) + chi^2 cos^2 theta (Eq. 40) are both R^2 H(R) + c with c >= 0,
// so both take their minimum where R^2 H(R) does, at the extremal radius R_e
// of Eqs. 34-37 (2 H + R H' = 0, Eq. 36; chi_e^2 = -R_e^2 H(R_e), Eq. 37),
// and above the largest zero R_H of R^2 H (the equatorial static limit,
// Eq. 41) every R^2 H + c is positive.  Each thread therefore
//   1. finds R_e as the maximiser of -R^2 H over (0, 50] (geometric scan,
//      then bisection of Eq. 36 between the neighbours of the best sample);
//   2. finds R_H by a downward geometric scan from R = 50 to the first sign
//      change, stopping at R_e, where R^2 H is smallest;
//   3. finds R_+ and each R_s(theta) as the largest root of R^2 H + c in
//      [R_e, R_H] by the same downward scan started at R_H (at R = 50 when
//      R^2 H has no zero below it).
// Every root is then polished inside its bracket by Newton steps on
// d(R^2 H)/dR = R (2 H + R H'), each pushed a few units in the last place
// past the root so that both ends of the bracket close in, with bisection
// wherever Newton would leave the bracket, to the last representable
// bracket; the upper end is returned.
#include <cuda_runtime.h>

#include <algorithm>

#include "bh_common.cuh"
#include "internal.h"

namespace bhrt {

namespace {

constexpr double kScanTop = 50.0;      // no root is sought above R = 50
constexpr double kScanRatio = 0.99;    // geometric step of the root scans (1 %)
constexpr double kPeakRatio = 0.97;    // geometric step of the extremal scan (3 %)
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
    R *= kPeakRatio;
  }
  // -R^2 H rises below R_e (Eq. 36's 2H + R H' < 0) and falls above it, so
  // R_e lies between the neighbours of the best sample
  double lo = Rb * kPeakRatio, hi = Rb / kPeakRatio;
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

// Root of R^2 H + c in [lo, hi] with R^2 H(lo) + c <= 0 < R^2 H(hi) + c:
// safeguarded Newton to the last representable bracket; returns its upper end.
__device__ double polish(const MetricConsts<double>& m, double c, double lo, double hi,
                         unsigned& ev) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double g;
    const double f = r2H(m, x, &g, ev) + c;
    if (f > 0.0) hi = x; else lo = x;
    const double d = x * g;  // d(R^2 H)/dR
    double xn = x - f / d;
    const double push = 4.0 * 2.220446049250313e-16 * x;
    xn += f > 0.0 ? -push : push;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    x = xn;
  }
  return hi;
}

// Largest root of R^2 H(R) + c in (R_e, top], where R^2 H + c is smallest at
// R_e; false if there is none (R^2 H + c not positive at top, or positive at
// R_e).
__device__ bool largest_root(const MetricConsts<double>& m, double c, double R_e, double top,
                             double& root, unsigned& ev) {
  if (!(r2H(m, top, nullptr, ev) + c > 0.0)) return false;
  if (!(r2H(m, R_e, nullptr, ev) + c <= 0.0)) return false;
  double hi = top, lo = R_e;
  for (double R = hi * kScanRatio; R > R_e; R *= kScanRatio) {
    if (r2H(m, R, nullptr, ev) + c <= 0.0) {
      lo = R;
      break;
    }
    hi = R;
  }
  root = polish(m, c, lo, hi, ev);
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

__global__ void __launch_bounds__(128) scan_kernel(ScanArgs a) {
  unsigned ev_h = 0, ev_s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    MetricConsts<double> m;
    double* Rs = a.R_s ? a.R_s + i * a.n_theta : nullptr;
    if (!consts_of(a.st[i], m)) {
      a.r_plus[i] = a.chi_e[i] = a.R_e[i] = 0.0;
      a.flags[i] = 2;
      for (int k = 0; Rs && k < a.n_theta; ++k) Rs[k] = 0.0;
      continue;
    }
    double ce, Re, RH = 0.0, rp = 0.0;
    extremal(m, ce, Re, ev_h);
    // R_H: no root of any R^2 H + c (c >= 0) lies above it, so the other
    // searches start there (or at R = 50 if R^2 H has no zero below it)
    const bool hasH = largest_root(m, 0.0, Re, kScanTop, RH, ev_h);
    const double top = hasH ? RH : kScanTop;
    const bool hz = largest_root(m, m.chi2, Re, top, rp, ev_h);
    a.chi_e[i] = ce;
    a.R_e[i] = Re;
    a.r_plus[i] = hz ? rp : 0.0;
    a.flags[i] = hz ? 0 : 1;
    for (int k = 0; Rs && k < a.n_theta; ++k) {
      const double cth = cos(a.theta[k]), c = m.chi2 * cth * cth;
      double rs = 0.0;
      if (hasH && !(c > 0.0)) {
        rs = RH;
      } else if (!largest_root(m, c, Re, top, rs, ev_s)) {
        rs = 0.0;
      }
      Rs[k] = rs;
    }
  }
  if (a.stats) {
    add_count(&a.stats[0], ev_h);
    add_count(&a.stats[1], ev_s);
  }
}

}  // namespace

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((a.n + 127) / 128, (int64_t)num_sms() * 16);
  scan_kernel<<<(int)blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bhrt
