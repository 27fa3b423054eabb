// integrator.cuh -- device pieces shared by the FP64 and the mixed-precision
// trace kernels: Dormand-Prince 5(4) tableau and dense output, the launch
// from the ZAMO screen, the FP64 step with crossing events, the emitter
// redshift and emissivity, the hand-off records between precision passes and
// the terminal write of a ray's results.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace bhrt {

// Dormand & Prince (1980) RK5(4)7M tableau, FSAL; 4th-order continuous
// extension (Shampine 1986; Hairer, Norsett & Wanner, Solving ODEs I).
struct DPTab {
  double a[7][6];
  double b[7];
  double e[7];  // b - b*
  double d[7];  // dense-output correction
};
__device__ constexpr DPTab kDP = {
    {{0, 0, 0, 0, 0, 0},
     {1.0 / 5, 0, 0, 0, 0, 0},
     {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
     {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
     {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
     {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
     {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0},
    {35.0 / 384 - 5179.0 / 57600, 0, 500.0 / 1113 - 7571.0 / 16695, 125.0 / 192 - 393.0 / 640,
     -2187.0 / 6784 + 92097.0 / 339200, 11.0 / 84 - 187.0 / 2100, -1.0 / 40},
    {-12715105075.0 / 11282082432.0, 0, 87487479700.0 / 32700410799.0,
     -10690763975.0 / 1880347072.0, 701980252875.0 / 199316789632.0,
     -1453857185.0 / 822651844.0, 69997945.0 / 29380423.0}};

// The same tableau rounded to FP32 for the FP32 steps of the mixed path
// (kept as literal floats so no FP64 conversion reaches the inner loop).
struct DPTabF {
  float a[7][6];
  float b[7];
  float e[7];
  float d[7];
};
#define BH_F(x) static_cast<float>(x)
__device__ constexpr DPTabF kDPf = {
    {{0, 0, 0, 0, 0, 0},
     {BH_F(1.0 / 5), 0, 0, 0, 0, 0},
     {BH_F(3.0 / 40), BH_F(9.0 / 40), 0, 0, 0, 0},
     {BH_F(44.0 / 45), BH_F(-56.0 / 15), BH_F(32.0 / 9), 0, 0, 0},
     {BH_F(19372.0 / 6561), BH_F(-25360.0 / 2187), BH_F(64448.0 / 6561), BH_F(-212.0 / 729), 0,
      0},
     {BH_F(9017.0 / 3168), BH_F(-355.0 / 33), BH_F(46732.0 / 5247), BH_F(49.0 / 176),
      BH_F(-5103.0 / 18656), 0},
     {BH_F(35.0 / 384), 0, BH_F(500.0 / 1113), BH_F(125.0 / 192), BH_F(-2187.0 / 6784),
      BH_F(11.0 / 84)}},
    {BH_F(35.0 / 384), 0, BH_F(500.0 / 1113), BH_F(125.0 / 192), BH_F(-2187.0 / 6784),
     BH_F(11.0 / 84), 0},
    {BH_F(35.0 / 384 - 5179.0 / 57600), 0, BH_F(500.0 / 1113 - 7571.0 / 16695),
     BH_F(125.0 / 192 - 393.0 / 640), BH_F(-2187.0 / 6784 + 92097.0 / 339200),
     BH_F(11.0 / 84 - 187.0 / 2100), BH_F(-1.0 / 40)},
    {BH_F(-12715105075.0 / 11282082432.0), 0, BH_F(87487479700.0 / 32700410799.0),
     BH_F(-10690763975.0 / 1880347072.0), BH_F(701980252875.0 / 199316789632.0),
     BH_F(-1453857185.0 / 822651844.0), BH_F(69997945.0 / 29380423.0)}};
#undef BH_F

// The tableau in the order a rolled stage loop consumes it.  Once k_j is
// known, stage j + 1 + u takes q[j][u] k_j into its running input sum
// (u = 0..5), and the 5th-order update, the error estimate and the dense
// output take b_j, e_j and d_j.  Each running sum adds its terms in
// increasing j, as the unrolled sums do, so both forms round alike.  One
// copy of the right-hand side then serves all six stages, which keeps the
// stepping loop small enough for the instruction cache.
template <class T>
struct DPRolled {
  T q[7][6];
  T b[7];
  T e[7];
  T d[7];
  // nonzero coefficients as bit masks (integer tests, so that skipping a
  // zero term costs no floating-point compare): bit u of qmask[j] for
  // q[j][u]; bit j of bmask, emask, dmask
  int qmask[7];
  int bmask, emask, dmask;
};

template <class T, class Tab>
constexpr DPRolled<T> make_rolled(const Tab& t) {
  DPRolled<T> r{};
  for (int j = 0; j < 7; ++j) {
    r.qmask[j] = 0;
    for (int u = 0; u < 6; ++u) {
      const int s = j + 1 + u;
      r.q[j][u] = s <= 6 ? static_cast<T>(t.a[s][j]) : T(0);
      if (r.q[j][u] != T(0)) r.qmask[j] |= 1 << u;
    }
    r.b[j] = static_cast<T>(t.b[j]);
    r.e[j] = static_cast<T>(t.e[j]);
    r.d[j] = static_cast<T>(t.d[j]);
    if (r.b[j] != T(0)) r.bmask |= 1 << j;
    if (r.e[j] != T(0)) r.emask |= 1 << j;
    if (r.d[j] != T(0)) r.dmask |= 1 << j;
  }
  return r;
}

static __constant__ DPRolled<double> kDPr = make_rolled<double>(kDP);
// state components the right-hand side reads: R, theta, p_R, p_theta
__host__ __device__ constexpr int kQC(int x) { return x < 2 ? x + 1 : x + 2; }
static __constant__ DPRolled<float> kDPrf = make_rolled<float>(kDPf);

constexpr double kHalfPi = 1.57079632679489661923;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;
constexpr unsigned kFull = 0xffffffffu;

// Step-size factor: safety 0.9, clamp [0.2, 10], no growth right after a
// rejection; err^(-1/5) evaluated in FP32 (it only steers the step size).
__device__ __forceinline__ float step_factor(float e, bool after_reject) {
  float fac = (e == 0.f) ? 10.f : 0.9f * __powf(e, -0.2f);
  return fminf(fmaxf(fac, 0.2f), after_reject ? 1.f : 10.f);
}

// Dense output of one component: y(x0 + sig h).
__device__ __forceinline__ double dense1(double y0, double y1, double hf0, double hf1, double hd,
                                         double sig) {
  double r2 = y1 - y0;
  double r3 = hf0 - r2;
  double r4 = r2 - hf1 - r3;
  return y0 + sig * (r2 + (1.0 - sig) * (r3 + sig * (r4 + (1.0 - sig) * hd)));
}

template <class T>
__device__ __forceinline__ MetricConsts<T> metric_consts(const ImgParams& ip);
template <>
__device__ __forceinline__ MetricConsts<double> metric_consts<double>(const ImgParams& ip) {
  return ip.md;
}
template <>
__device__ __forceinline__ MetricConsts<float> metric_consts<float>(const ImgParams& ip) {
  return ip.mf;
}

// 1 / (1 + e^a) without overflow: with t = e^{-|a|} in (0, 1], it is
// t / (1 + t) for a >= 0 and 1 / (1 + t) otherwise (the tapers of
// Eqs. 85-86 as logistic functions, 0.5 (1 + tanh x) = 1 / (1 + e^{-2x})).
__device__ __forceinline__ double logistic_neg(double a) {
  const double t = d_exp(-fabs(a));
  const double s = d_rcp(1.0 + t);
  return a >= 0.0 ? t * s : s;
}

// Circular equatorial emitter at R (Eqs. 90-91 at theta = pi/2, where
// d_R g_TT = -H', d_R g_Tphi = chi H', d_R g_phph = 2R - chi^2 H') and the
// redshift g = (-p.u_obs)/(-p.u_em) with -p.u_obs = E_loc = 1 (Eq. 73).
// Returns false where no timelike prograde circular orbit exists.
// Reciprocals by d_rcp and d_rsqrt (no slow-path division).
__device__ __forceinline__ bool emitter_g(const MetricConsts<double>& m, double R, double E,
                                          double ell, double& g) {
  double iR = d_rcp(R), H, dH;
  lapse(m, R, iR, H, dH);
  double den = 2.0 * R - m.chi2 * dH;
  double disc = 2.0 * R * dH;
  if (!(disc >= 0.0) || den == 0.0) return false;
  double W = (-m.chi * dH + sqrt(disc)) * d_rcp(den);
  double gtt = -H, gtp = -m.chi * (1.0 - H), gpp = R * R + m.chi2 + m.chi2 * (1.0 - H);
  double norm = -(gtt + 2.0 * W * gtp + W * W * gpp);
  if (!(norm > 0.0)) return false;
  double uT = d_rsqrt(norm);
  g = d_rcp(uT * (E - W * ell));
  return true;
}

// Thin-disk emissivity, Eqs. (83)-(86) at z = 0, rho = R: the power and the
// exponential in log space and the tanh tapers as logistic functions
// (0.5 (1 + tanh x) = 1 / (1 + e^{-2x})), by the library's own exp and
// log1p.
__device__ __forceinline__ double emissivity_eq(const ImgParams& ip, double R) {
  const double tin = logistic_neg(-2.0 * (R - ip.R_in) * ip.isig_in);    // Eq. (85)
  const double tout = logistic_neg(2.0 * (R - ip.R_out) * ip.isig_out);  // Eq. (86)
  const double lnj = -ip.p * d_log1p(R * ip.iR_in - 1.0) - (R - ip.R_in) * ip.iR_s;
  return ip.j0 * d_exp(lnj) * tin * tout;                                // Eq. (83)
}

// Source of the volumetric intensity, Eq. (88): g^3 j at (R, theta) with the
// emissivity of Eqs. (83)-(86) (rho = R |sin theta|, z = R cos theta, so a
// trial stage past the polar axis is its mirror point) and the circular
// emitter of Eqs. (90)-(91) at the cylindrical radius rho of the equatorial
// metric (reading); 0 where no timelike circular orbit exists there.  The
// tapers are written 0.5 (1 + tanh a) = 1 / (1 + exp(-2 a)).
static __device__ __noinline__ double vol_source64(const ImgParams& ip, MetricConsts<double> m,
                                                   double E, double ell, double R, double th) {
  double s, c;
  d_sincos(th, &s, &c);
  const double rho = R * fabs(s), z = R * c;
  double g;
  if (!(rho > 0.0) || !emitter_g(m, rho, E, ell, g)) return 0.0;
  const double Hd = ip.H0 + ip.hh * rho;                        // Eq. (84)
  const double iH = d_rcp(Hd);
  const double tin = logistic_neg(-2.0 * (rho - ip.R_in) * ip.isig_in);    // Eq. (85)
  const double tout = logistic_neg(2.0 * (rho - ip.R_out) * ip.isig_out);   // Eq. (86)
  const double lnj = -ip.p * d_log1p(rho * ip.iR_in - 1.0) - (rho - ip.R_in) * ip.iR_s -
                     0.5 * (z * iH) * (z * iH);                 // Eq. (83)
  return g * g * g * ip.j0 * d_exp(lnj) * tin * tout;
}

// Redshift of a prograde circular emitter (Eqs. 89-91), FP32.
__device__ __forceinline__ bool emitter_g_f(const MetricConsts<float>& m, float R, float E,
                                            float ell, float& g) {
  float H, dH;
  lapse(m, R, __fdividef(1.f, R), H, dH);
  const float den = 2.f * R - m.chi2 * dH, disc = 2.f * R * dH;
  if (!(disc >= 0.f) || den == 0.f) return false;
  const float W = __fdividef(-m.chi * dH + sqrtf(disc), den);
  const float gtt = -H, gtp = -m.chi * (1.f - H), gpp = R * R + m.chi2 + m.chi2 * (1.f - H);
  const float norm = -(gtt + 2.f * W * gtp + W * W * gpp);
  if (!(norm > 0.f)) return false;
  g = __fdividef(sqrtf(norm), E - W * ell);
  return true;
}

// Source of the volumetric intensity (Eq. 88) in FP32: g^3 j at (R, theta),
// theta given as dth = theta - pi/2 (see dtheta_eq), as vol_source64 (mirror
// point past the polar axis, emitter at the cylindrical radius rho, tapers as
// logistic functions), from the image's FP32 emission constants.
// 1 / (1 + e^a) without overflow (see logistic_neg), FP32.
__device__ __forceinline__ float logistic_neg_f(float a) {
  const float t = __expf(-fabsf(a));
  const float s = __fdividef(1.f, 1.f + t);
  return a >= 0.f ? t * s : s;
}

static __device__ __noinline__ float vol_source32(const ImgParams& ip, MetricConsts<float> m,
                                                  float E, float ell, float R, float dth) {
  float s, c;
  d_sincos(dth, &s, &c);
  const float rho = R * fabsf(c), z = -R * s;
  float g;
  if (!(rho > 0.f) || !emitter_g_f(m, rho, E, ell, g)) return 0.f;
  const float* v = ip.vf;  // H0, hh, R_in, 1/sig_in, 1/sig_out, R_out, p, 1/R_s, j0, 1/R_in
  const float zH = __fdividef(z, v[0] + v[1] * rho);                    // Eq. (84)
  const float tin = logistic_neg_f(-2.f * (rho - v[2]) * v[3]);   // Eq. (85)
  const float tout = logistic_neg_f(2.f * (rho - v[5]) * v[4]);   // Eq. (86)
  const float lnj = -v[6] * __logf(rho * v[9]) - (rho - v[2]) * v[7] - 0.5f * zH * zH;
  return g * g * g * v[8] * __expf(lnj) * tin * tout;                    // Eq. (83)
}

// The volumetric source for an FP64 state in the mixed path's promoted pass:
// the FP32 evaluation of the FP32 legs (vol_source32) from E, ell, R and
// theta - pi/2 formed in FP64 and rounded.  The source enters only the
// intensity integral, which the mixed path holds to its bar, not the
// trajectory that the promotion protects; the all-FP64 path keeps
// vol_source64.
static __device__ __noinline__ double vol_source_mx(const ImgParams& ip, double E, double ell,
                                                    double R, double th) {
  return (double)vol_source32(ip, metric_consts<float>(ip), __double2float_rn(E),
                              __double2float_rn(ell), __double2float_rn(R),
                              __double2float_rn(th - kHalfPi));
}

// Volumetric mode (reading, as in the oracle): a step that may come within
// 5 H(rho) of the equatorial plane advances z by at most H(rho) / 2, so
// that the stages sample the Gaussian layer however thin it is.
template <class T>
__device__ __forceinline__ T layer_cap(T H0, T hh, T R, T th, T fR, T fth, T h) {
  T s, c;
  d_sincos(th, &s, &c);
  const T z = R * c, zd = fR * c - R * s * fth;
  const T Hc = H0 + hh * fabs(R * s);
  const T azd = fabs(zd);
  if (azd > T(0) && fabs(z) - azd * h < T(5) * Hc) {
    const T cap = T(0.5) * Hc * d_rcp(azd);
    if (h > cap) h = cap;
  }
  return h;
}

// Event bookkeeping common to both precisions.
struct CrossState {
  double I[4];      // I_tot, I_0, I_1, I_2
  double lam_last;  // affine parameter of the last trusted crossing
  int32_t ncross;
  bool have_trusted;
};

// Where a base ray's transfer maps go (image level 0 or points mode).
struct CrossOut {
  float* R_em;
  float* phi_em;
  float* T_em;
  float* g;
  int64_t stride, pix;   // plane stride (npix) and pixel index; pix < 0: none
  bh_ray_record* rec;    // points mode
};

// Equatorial crossing inside one accepted step, evaluated in FP64 on the
// step's dense output (Sec. 3.3 and Sec. 4.2): sign change of theta - pi/2
// (an end point exactly on the plane belongs to the step that reaches it),
// root by Illinois-modified regula falsi, trusted-crossing filter, then the
// transfer maps (Eq. 82), redshift (Eq. 89) and g^3 j (Eqs. 83, 88).
static __device__ __noinline__ void handle_crossing(const ImgParams& ip, const MetricConsts<double>& m,
                                             double E, double ell, const double* y0,
                                             const double* y1, const double* hf0,
                                             const double* hf1, const double* hd, double lam,
                                             double h, CrossState& cs, const CrossOut& co) {
  const double s0 = y0[2] - kHalfPi, s1 = y1[2] - kHalfPi;
  if (!((s0 > 0.0 && s1 <= 0.0) || (s0 < 0.0 && s1 >= 0.0))) return;
  double sig = 1.0;
  if (s1 != 0.0) {
    // theta - pi/2 on the continuous extension (dense1) written out as the
    // quartic s0 + c1 x + c2 x^2 + c3 x^3 + c4 x^4; Newton steps with its
    // derivative from the secant point, kept inside the sign-change bracket
    // by bisection, to |dx| <= 1e-15
    const double r2 = y1[2] - y0[2], A = hf0[2] - r2, Bq = r2 - hf1[2] - A, Cq = hd[2];
    const double c1 = hf0[2], c2 = Bq + Cq - A, c3 = -(Bq + 2.0 * Cq), c4 = Cq;
    double lo = 0.0, hi = 1.0, flo = s0;
    double x = s0 * d_rcp(s0 - s1);
    for (int it = 0; it < 60; ++it) {
      const double f = fma(x, fma(x, fma(x, fma(x, c4, c3), c2), c1), s0);
      if (f == 0.0) break;
      if ((f > 0.0) == (flo > 0.0)) {
        lo = x;
        flo = f;
      } else {
        hi = x;
      }
      const double d = fma(x, fma(x, fma(x, 4.0 * c4, 3.0 * c3), 2.0 * c2), c1);
      double xn = x - f * d_rcp(d);
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      const bool done = fabs(xn - x) <= 1e-15;
      x = xn;
      if (done) break;
    }
    sig = x;
  }
  double yc[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) yc[i] = dense1(y0[i], y1[i], hf0[i], hf1[i], hd[i], sig);
  double sth, cth;
  d_sincos(yc[2], &sth, &cth);
  double Sig = yc[1] * yc[1] + m.chi2 * cth * cth;
  double thdot = yc[5] * d_rcp(Sig);                            // Eq. (60)
  double lamc = lam + sig * h;
  // events count only inside the integration domain R_cap <= R <= R_esc
  bool trusted = yc[1] >= ip.R_cap && yc[1] <= ip.R_esc && fabs(thdot) >= ip.thdot_min &&
                 (!cs.have_trusted || lamc - cs.lam_last >= ip.dlam_min);
  if (!trusted) return;
  int n = cs.ncross;
  double g = 0.0, j = 0.0;
  if (emitter_g(m, yc[1], E, ell, g)) j = emissivity_eq(ip, yc[1]);
  // the volumetric mode adds no event intensity (its integral is a state)
  double In = ip.volumetric ? 0.0 : g * g * g * j;
  cs.I[0] += In;
  if (n < 3) {
    cs.I[1 + n] = In;
    // phi reduced to [0, 2 pi) by a two-part 2 pi (no slow-path fmod)
    const double qn = floor(yc[3] * 0.15915494309189533577);
    double ph = fma(-qn, 6.283185307179586232, yc[3]);
    ph = fma(-qn, 2.4492935982947064e-16, ph);
    if (ph < 0.0) ph += kTwoPi;
    if (ph >= kTwoPi) ph -= kTwoPi;
    if (co.pix >= 0) {
      int64_t o = n * co.stride + co.pix;
      if (co.R_em) co.R_em[o] = (float)yc[1];
      if (co.phi_em) co.phi_em[o] = (float)ph;
      if (co.T_em) co.T_em[o] = (float)yc[0];
      if (co.g) co.g[o] = (float)g;
    }
    if (co.rec) {
      co.rec->R_em[n] = yc[1];
      co.rec->phi_em[n] = ph;
      co.rec->T_em[n] = yc[0];
      co.rec->g[n] = g;
    }
  }
  cs.ncross = n + 1;
  cs.lam_last = lamc;
  cs.have_trusted = true;
}

// FP64 ray state.
// The FP64 right-hand side out of line, for the call sites that run once per
// ray (launch, resume, axis reflection): the stepping loop keeps the only
// inlined copy.
struct RhsD {
  double d[6];
  double W, P2;
};
static __device__ __noinline__ RhsD rhs_f64(MetricConsts<double> m, double E, double ell,
                                            double R, double th, double pR, double pth) {
  RhsD o;
  geo_rhs(m, E, ell, R, th, pR, pth, o.d, o.W, o.P2);
  return o;
}
__device__ __forceinline__ void rhs_f64_into(const MetricConsts<double>& m, double E, double ell,
                                             double R, double th, double pR, double pth,
                                             double* d) {
  const RhsD o = rhs_f64(m, E, ell, R, th, pR, pth);
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = o.d[i];
}

struct Ray64 {
  double y[6];     // T, R, th, phi, p_R, p_th
  double f[6];     // f(y) (FSAL)
  double fI;       // volumetric source g^3 j at y (FSAL of the seventh component)
  double h, lam;
  double E, ell;
  CrossState cs;
  float hdrift;
  int32_t nacc, nrej, steps;
  bool rejected;
  bool xpend;      // a crossing of this ray is parked in its XPend slot
};

// An equatorial crossing whose evaluation is deferred: the end points, the
// h f terms and the dense-output term of the accepted step that brackets
// it, everything handle_crossing reads.  A persistent FP64 warp evaluates
// parked crossings together (see trace_fp64_kernel) instead of running the
// crossing code for one or two lanes at a time.
struct XPend {
  double y0[6], y1[6], hf0[6], hf1[6], hd[6];
  double lam, h;
};

// Evaluates a parked crossing into the ray's event state.
static __device__ __noinline__ void flush_crossing(const ImgParams& ip, MetricConsts<double> m,
                                                   double E, double ell, const XPend& x,
                                                   CrossState& cs, const CrossOut& co) {
  handle_crossing(ip, m, E, ell, x.y0, x.y1, x.hf0, x.hf1, x.hd, x.lam, x.h, cs, co);
}

// Launch (Sec. 3.2): p^mu = u_o + n^(a) e_(a) with E_loc = 1 (Eq. 73),
// lowered with g_{mu nu} (Eq. 74).  With g_Tphi + omega g_phph = 0 this gives
// p_R = sqrt(g_RR) n^(R), p_th = sqrt(g_thth) n^(th), ell = sqrt(g_phph) n^(phi),
// E = N_o + omega ell.  Then the Hairer-Wanner starting step (Solving ODEs I,
// Sec. II.4) for an error estimator of order 4.  All in FP64.
__device__ __forceinline__ void ray_init64(const ImgParams& ip, const MetricConsts<double>& m,
                                           double X, double Y, Ray64& r) {
  const double id = d_rsqrt(ip.r_obs * ip.r_obs + X * X + Y * Y);
  r.y[0] = 0.0;
  r.y[1] = ip.r_obs;
  r.y[2] = ip.incl;
  r.y[3] = 0.0;
  r.y[4] = ip.sq_grr * (-ip.r_obs * id);
  r.y[5] = ip.sq_gth * (-Y * id);
  r.ell = ip.sq_gph * (-X * id);
  r.E = ip.zamo_N + ip.zamo_w * r.ell;
  rhs_f64_into(m, r.E, r.ell, r.y[1], r.y[2], r.y[4], r.y[5], r.f);
  r.fI = ip.volumetric ? vol_source64(ip, m, r.E, r.ell, r.y[1], r.y[2]) : 0.0;
  // starting-step heuristic in FP32 (it only needs a few digits)
  float d0 = 0.f, d1 = 0.f, sc[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    sc[i] = (float)(ip.atol + ip.rtol * fabs(r.y[i]));
    const float a0 = __fdividef((float)r.y[i], sc[i]), a1 = __fdividef((float)r.f[i], sc[i]);
    d0 += a0 * a0;
    d1 += a1 * a1;
  }
  d0 = sqrtf(d0 / 6.f);
  d1 = sqrtf(d1 / 6.f);
  const float h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * __fdividef(d0, d1);
  const double h0d = (double)h0;
  double f1[6];
  rhs_f64_into(m, r.E, r.ell, r.y[1] + h0d * r.f[1], r.y[2] + h0d * r.f[2],
               r.y[4] + h0d * r.f[4], r.y[5] + h0d * r.f[5], f1);
  float d2 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float q = __fdividef((float)(f1[i] - r.f[i]), sc[i]);
    d2 += q * q;
  }
  d2 = __fdividef(sqrtf(d2 / 6.f), h0);
  const float mx = fmaxf(d1, d2);
  const float h1 = (mx <= 1e-15f) ? fmaxf(1e-6f, h0 * 1e-3f) : __powf(__fdividef(0.01f, mx), 0.2f);
  r.h = (double)fminf(100.f * h0, h1);
  if (ip.volumetric)
    r.h = layer_cap(ip.H0, ip.hh, r.y[1], r.y[2], r.f[1], r.f[2], r.h);
  r.lam = 0.0;
  r.cs.lam_last = 0.0;
  r.cs.have_trusted = false;
  r.cs.ncross = 0;
  r.cs.I[0] = r.cs.I[1] = r.cs.I[2] = r.cs.I[3] = 0.0;
  r.rejected = false;
  r.xpend = false;
  r.nacc = r.nrej = r.steps = 0;
  r.hdrift = 0.f;
}

// Polar axis: a state that passed through theta = 0 or pi is mapped back
// into (0, pi) by (theta, p_th, phi) -> (-theta or 2 pi - theta, -p_th,
// phi + pi).  Returns true if it reflected.
__device__ __forceinline__ bool reflect_axis(double& th, double& pth, double& ph) {
  // 0 <= th <= pi as an unsigned compare of the bit pattern (+0 .. pi, and
  // -0), on the integer pipes; negative values and NaN order above pi
  const unsigned long long u = (unsigned long long)__double_as_longlong(th);
  if (u <= 0x400921FB54442D18ull || u == 0x8000000000000000ull) return false;
  th = th < 0.0 ? -th : kTwoPi - th;
  pth = -pth;
  ph += kPi;
  return true;
}

__device__ __forceinline__ CrossOut cross_out(const TraceArgs& a, int64_t item, uint32_t img) {
  CrossOut co;
  co.R_em = co.phi_em = co.T_em = co.g = nullptr;
  co.stride = a.npix;
  co.pix = -1;
  co.rec = nullptr;
  if (a.mode == 1) {
    co.rec = &a.rec[item];
  } else if (a.level == 0) {
    const OutPtrs& o = a.out[img];
    co.R_em = o.R_em;
    co.phi_em = o.phi_em;
    co.T_em = o.T_em;
    co.g = o.g;
    co.pix = item - (int64_t)img * a.npix;
  }
  return co;
}

// One attempted FP64 step.  Returns 0 while the ray continues, else the
// terminal status + 1 (1 escaped, 2 captured, 3 undetermined).
// A double truncated to FP32 precision by bit manipulation on the integer
// pipes (no FP64-pipe conversion): the exponent rebiased, the leading 20
// mantissa bits kept; magnitudes below 2^-126 give 0, above 2^128 the largest
// float.  Relative error below 2^-20.
__device__ __forceinline__ float f32_trunc(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 896;  // rebias 1023 -> 127
  const int sign = hi & (int)0x80000000;
  const int mag = e <= 0 ? 0 : (e >= 255 ? 0x7f7fffff : ((e << 23) | ((hi & 0xfffff) << 3)));
  return __int_as_float(sign | mag);
}

// A normal, nonzero float widened to double by bit manipulation on the
// integer pipes (exact; the step factors lie in [0.2, 10]).
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                               ((unsigned long long)(((b >> 23) & 0xff) + 896) << 52) |
                               ((unsigned long long)(b & 0x7fffff) << 29);
  return __longlong_as_double((long long)d);
}

// One component's squared scaled error (h e_i / sc_i)^2,
// sc_i = atol + rtol max(|y0_i|, |y1_i|), in FP32 from truncated operands:
// the norm only decides acceptance and the next step factor, to a few
// digits, and the FP64 pipe is the FP64 step's bottleneck.
__device__ __forceinline__ float err_term(double y0, double y1, double he, float atol,
                                          float rtol) {
  const float sc = fmaf(rtol, fmaxf(fabsf(f32_trunc(y0)), fabsf(f32_trunc(y1))), atol);
  const float q = __fdividef(f32_trunc(he), sc);
  return q * q;
}

// kVol: the build that can integrate the volumetric intensity (Eq. 88) as a
// seventh component; the thin-disk build carries none of its registers.
// kDefer: a crossing is parked in *xp (the lane's slot) for the warp to
// evaluate later; a crossing already parked there is evaluated first, so a
// ray's crossings are always evaluated in order.  kEvents = false skips the
// crossing events altogether (a caller that needs only the ray's fate: the
// fate does not depend on them).
template <bool kVol, bool kDefer = false, bool kEvents = true>
__device__ __forceinline__ int ray_step64(const ImgParams& ip, const MetricConsts<double>& m,
                                          Ray64& r, const TraceArgs& a, int64_t item,
                                          uint32_t img, XPend* xp = nullptr) {
  const double h = r.h;
  // rolled stage loop (see DPRolled): k is the latest stage derivative, q[u]
  // the running input sums of the next stages, s5/se/sd the running sums of
  // the update, the error estimate and the dense-output term; r.f keeps k_0
  // the right-hand side reads R, theta, p_R, p_theta only (T and phi are
  // cyclic), so the stage-input sums q keep those four components (kQC)
  double k[6], q[6][4], s5[6], se[6], sd[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    k[i] = r.f[i];
    s5[i] = se[i] = sd[i] = 0.0;
  }
#pragma unroll
  for (int u = 0; u < 6; ++u)
#pragma unroll
    for (int x = 0; x < 4; ++x) q[u][x] = 0.0;
  bool bad = false;
  double W = 0, P2oD = 1;
  // volumetric mode: the intensity integral is a seventh component whose
  // derivative g^3 j depends on the state only (kI, sums s5I and seI)
  const bool vol = kVol && ip.volumetric != 0;
  // the mixed path's promoted pass takes the source in FP32 (vol_source_mx)
  const bool src32 = vol && a.source == 1;
  double kI = kVol ? r.fI : 0.0, s5I = 0.0, seI = 0.0;
  const RayC<double> kc = ray_consts(m, r.E, r.ell);
#pragma unroll 1
  for (int j = 0; j < 7; ++j) {
    // zero coefficients (about a third of the triangular sums) are skipped
    // by uniform integer tests: FP64 operations are the pass's bottleneck
    if ((kDPr.bmask >> j) & 1) {
      const double bj = kDPr.b[j];
#pragma unroll
      for (int i = 0; i < 6; ++i) s5[i] = fma(bj, k[i], s5[i]);
      s5I = fma(bj, kI, s5I);
    }
    if ((kDPr.emask >> j) & 1) {
      const double ej = kDPr.e[j];
#pragma unroll
      for (int i = 0; i < 6; ++i) se[i] = fma(ej, k[i], se[i]);
      seI = fma(ej, kI, seI);
    }
    if ((kDPr.dmask >> j) & 1) {
      const double dj = kDPr.d[j];
#pragma unroll
      for (int i = 0; i < 6; ++i) sd[i] = fma(dj, k[i], sd[i]);
    }
    if (j == 6) break;
    const int qm = kDPr.qmask[j];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      if ((qm >> u) & 1) {
        const double c = kDPr.q[j][u];
#pragma unroll
        for (int x = 0; x < 4; ++x) q[u][x] = fma(c, k[kQC(x)], q[u][x]);
      }
    }
    double ys[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) ys[x] = r.y[kQC(x)] + h * q[0][x];
    double sth, cth;
    d_sincos(ys[1], &sth, &cth);
    bool ok = geo_rhs_sc(m, kc, ys[0], sth, cth, ys[2], ys[3], k, W, P2oD);
    bad |= !ok;
    if (vol)
      kI = src32 ? vol_source_mx(ip, r.E, r.ell, ys[0], ys[1])
                 : vol_source64(ip, m, r.E, r.ell, ys[0], ys[1]);
#pragma unroll
    for (int u = 0; u < 5; ++u) {
#pragma unroll
      for (int x = 0; x < 4; ++x) q[u][x] = q[u + 1][x];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) q[5][x] = 0.0;
  }
  double y1[6];
  float err2 = 0.f;
  const float fatol = f32_trunc(ip.atol), frtol = f32_trunc(ip.rtol);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    y1[i] = r.y[i] + h * s5[i];
    err2 += err_term(r.y[i], y1[i], h * se[i], fatol, frtol);
  }
  const double I1 = r.cs.I[0] + h * s5I;
  if (vol) err2 += err_term(r.cs.I[0], I1, h * seI, fatol, frtol);
  float err = sqrtf(err2 / (vol ? 7.f : 6.f));
  r.steps++;
  if (bad || !(err <= 1.f)) {
    r.h = bad ? 0.5 * h : h * f64_of_f32(step_factor(err, true));
    r.rejected = true;
    r.nrej++;
    return r.steps >= ip.max_steps ? 3 : 0;
  }
  r.nacc++;
  if (vol) {
    r.cs.I[0] = I1;
    r.fI = kI;
  }
  if (kEvents) {
    // sign tests of theta - pi/2 on the bit patterns (integer pipes; a
    // difference of two doubles is never -0 under round-to-nearest)
    const long long s0 = __double_as_longlong(r.y[2] - kHalfPi);
    const long long s1 = __double_as_longlong(y1[2] - kHalfPi);
    if ((s0 > 0 && s1 <= 0) || (s0 < 0 && s1 >= 0)) {
      double hf0[6], hf1[6], hd[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        hd[i] = h * sd[i];
        hf0[i] = h * r.f[i];
        hf1[i] = h * k[i];
      }
      if (kDefer) {
        if (r.xpend) {
          CrossState cs = r.cs;
          flush_crossing(ip, m, r.E, r.ell, *xp, cs, cross_out(a, item, img));
          r.cs = cs;
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          xp->y0[i] = r.y[i];
          xp->y1[i] = y1[i];
          xp->hf0[i] = hf0[i];
          xp->hf1[i] = hf1[i];
          xp->hd[i] = hd[i];
        }
        xp->lam = r.lam;
        xp->h = h;
        r.xpend = true;
      } else {
        // copies: the ray state must not have its address taken (it would be
        // demoted from registers to local memory for every step)
        double y0c[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) y0c[i] = r.y[i];
        CrossState cs = r.cs;
        const CrossOut co = cross_out(a, item, img);
        handle_crossing(ip, m, r.E, r.ell, y0c, y1, hf0, hf1, hd, r.lam, h, cs, co);
        r.cs = cs;
      }
    }
  }
  r.lam += h;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    r.y[i] = y1[i];
    r.f[i] = k[i];
  }
  if (reflect_axis(r.y[2], r.y[5], r.y[3])) {
    rhs_f64_into(m, r.E, r.ell, r.y[1], r.y[2], r.y[4], r.y[5], r.f);
    if (vol)
      r.fI = src32 ? vol_source_mx(ip, r.E, r.ell, r.y[1], r.y[2])
                   : vol_source64(ip, m, r.E, r.ell, r.y[1], r.y[2]);
  }
  // null-constraint monitor at the new point (stage 7 = new point, FSAL)
  // (a monitor to a few digits: FP32 from truncated operands, off the FP64 pipe)
  float hdv = __fdividef(f32_trunc(fabs(W)), f32_trunc(P2oD));
  if (hdv > r.hdrift) r.hdrift = hdv;
  // an accepted state is never NaN (a NaN stage makes the error norm
  // infinite), so R compares with the radii by bit pattern (integer pipes):
  // for R >= 0 the order of the patterns is the order of the values, and a
  // negative R has a negative pattern
  const long long rb = __double_as_longlong(r.y[1]);
  if (rb < __double_as_longlong(ip.R_cap)) return 2;
  if (rb > __double_as_longlong(ip.R_esc)) return 1;
  r.h = h * f64_of_f32(step_factor(err, r.rejected));
  if (vol) r.h = layer_cap(ip.H0, ip.hh, r.y[1], r.y[2], r.f[1], r.f[2], r.h);
  r.rejected = false;
  return r.steps >= ip.max_steps ? 3 : 0;
}

// A ray handed from one precision pass to the next.
struct alignas(16) SpillRec {
  double y[6];
  double h, lam, E, ell;
  double I[4];
  double lam_last;
  int64_t item;
  uint32_t img;
  float hdrift;
  int32_t ncross, nacc, nrej, steps;
  int32_t flags;  // bit 0 have_trusted, bit 1 rejected
  int32_t pad;
};

__device__ __forceinline__ void spill_from64(const Ray64& r, int64_t item, uint32_t img,
                                             SpillRec& s) {
#pragma unroll
  for (int i = 0; i < 6; ++i) s.y[i] = r.y[i];
  s.h = r.h;
  s.lam = r.lam;
  s.E = r.E;
  s.ell = r.ell;
#pragma unroll
  for (int i = 0; i < 4; ++i) s.I[i] = r.cs.I[i];
  s.lam_last = r.cs.lam_last;
  s.item = item;
  s.img = img;
  s.hdrift = r.hdrift;
  s.ncross = r.cs.ncross;
  s.nacc = r.nacc;
  s.nrej = r.nrej;
  s.steps = r.steps;
  s.flags = (r.cs.have_trusted ? 1 : 0) | (r.rejected ? 2 : 0);
  s.pad = 0;
}

__device__ __forceinline__ void resume64(const ImgParams& ip, const SpillRec& s,
                                         const MetricConsts<double>& m, Ray64& r) {
#pragma unroll
  for (int i = 0; i < 6; ++i) r.y[i] = s.y[i];
  r.h = s.h;
  r.lam = s.lam;
  r.E = s.E;
  r.ell = s.ell;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.cs.I[i] = s.I[i];
  r.cs.lam_last = s.lam_last;
  r.cs.ncross = s.ncross;
  r.cs.have_trusted = (s.flags & 1) != 0;
  r.rejected = (s.flags & 2) != 0;
  r.hdrift = s.hdrift;
  r.nacc = s.nacc;
  r.nrej = s.nrej;
  r.steps = s.steps;
  r.xpend = false;
  rhs_f64_into(m, r.E, r.ell, r.y[1], r.y[2], r.y[4], r.y[5], r.f);
  // a resumed ray is in the mixed path's promoted pass: FP32 source
  r.fI = ip.volumetric ? vol_source_mx(ip, r.E, r.ell, r.y[1], r.y[2]) : 0.0;
}

// Carter-type constant K = p_th^2 + Q^2, Q = ell/sin(theta) - chi E sin(theta)
// (the separation constant of Eq. 56), of the ray launched at the screen point
// (X, Y): the launch momenta of ray_init64 (Eqs. 70-74) at theta = theta_o, in
// FP64 and with the same arithmetic, so E and ell here equal the ray's own.
__device__ __forceinline__ double launch_carter(const ImgParams& ip, double X, double Y) {
  const double id = d_rsqrt(ip.r_obs * ip.r_obs + X * X + Y * Y);
  const double pth = ip.sq_gth * (-Y * id);
  const double ell = ip.sq_gph * (-X * id);
  const double E = ip.zamo_N + ip.zamo_w * ell;
  const double Q = ell * ip.isin_o - ip.chi * E * ip.sin_o;
  return pth * pth + Q * Q;
}

// Puts a state handed over by the FP32 pass back on its ray's FP64 constants
// of motion: p_th from K = p_th^2 + Q^2 and p_R from the null condition
// (Eq. 54 with Eq. 56), Delta^2 p_R^2 = P^2 - Delta K, signs kept; where
// rounding put the point just beyond a turning point, the momentum there is
// set to 0 and p_R follows from the K the state then has, so the state stays
// null.  The FP32 legs integrate with E and ell rounded to floats and round
// every operation, so their invariants arrive off by about 1e-7; near the
// photon orbit such an offset would grow exponentially over the windings,
// whereas an error in the position only shifts the phase along the exact
// geodesic.
static __device__ __noinline__ void project_invariants(MetricConsts<double> m, double E,
                                                       double ell, double K, double* y) {
  const double R = y[1];
  double s, c;
  d_sincos(y[2], &s, &c);
  if (!(fabs(s) > 1e-8) || !(R > 0.0)) return;
  double H, dH;
  lapse(m, R, d_rcp(R), H, dH);
  const double Dl = R * R * H + m.chi2;                       // Eq. (25)
  if (!(Dl > 0.0)) return;
  const double Q = ell * d_rcp(s) - m.chi * E * s;
  const double pth2 = fmax(K - Q * Q, 0.0);
  const double Ks = pth2 + Q * Q;
  const double P = (R * R + m.chi2) * E - m.chi * ell;
  const double Rr = fmax(P * P - Dl * Ks, 0.0);               // (Delta p_R)^2
  y[5] = copysign(sqrt(pth2), y[5]);
  y[4] = copysign(sqrt(Rr) * d_rcp(Dl), y[4]);
}

// Demotion of a promoted ray that has left a double root of its radial
// potential: outgoing, with Rr / P^2 = (Delta p_R)^2 / P^2 above
// kDemoteKappa times the promotion threshold kappa (see the FP32 test
// near_double_root), i.e. past the band in which it was promoted, where the
// remaining time near the orbit no longer magnifies a position error (on
// the 512^2 sweep a factor 1.2 gives the same images as 4 with 4 % fewer
// FP64 steps).  Evaluated in FP32 from truncated operands (it only decides
// where the FP32 steps resume).
constexpr float kDemoteKappa = 1.2f;
static __device__ __noinline__ bool past_double_root(const ImgParams& ip, double E, double ell,
                                                     double R, double pR) {
  const MetricConsts<float> m = metric_consts<float>(ip);
  const float Rf = f32_trunc(R);
  float H, dH;
  lapse(m, Rf, __fdividef(1.f, Rf), H, dH);
  const float R2 = Rf * Rf;
  const float Dl = R2 * H + m.chi2;
  const float P = (R2 + m.chi2) * f32_trunc(E) - m.chi * f32_trunc(ell);
  const float DpR = Dl * f32_trunc(pR);
  return DpR * DpR > kDemoteKappa * (float)ip.kappa * P * P;
}

// Resolves a fresh work item to its image, output pixel and screen point.
__device__ __forceinline__ void resolve_item(const TraceArgs& a, int64_t idx, uint32_t& img,
                                             int64_t& pix, double& X, double& Y) {
  if (a.mode == 1) {
    img = 0;
    pix = -1;
    X = a.xy[2 * idx];
    Y = a.xy[2 * idx + 1];
    return;
  }
  uint64_t key;
  if (a.level == 0) {
    img = (uint32_t)(idx / a.npix);
    pix = idx - (int64_t)img * a.npix;
    key = (uint64_t)pix << 16;
  } else {
    key = a.lv.key[idx];
    img = a.lv.img[idx];
    pix = -1;
  }
  cell_centre(a.ip[img], key, X, Y);
}

// Terminal write of a ray: the per-ray record of its level (for refinement
// and assembly), the base-ray planes, or the points-mode record.
__device__ __forceinline__ void finish_ray(const TraceArgs& a, int64_t item, uint32_t img,
                                           int status, const CrossState& cs, float hdrift,
                                           int nacc, int nrej, double E, double ell,
                                           double lam) {
  if (a.mode == 1) {
    bh_ray_record* rc = &a.rec[item];
    rc->status = status;
    rc->ncross = cs.ncross;
    rc->n_accept = nacc;
    rc->n_reject = nrej;
    rc->I_tot = cs.I[0];
    rc->I_n[0] = cs.I[1];
    rc->I_n[1] = cs.I[2];
    rc->I_n[2] = cs.I[3];
    rc->E = E;
    rc->ell = ell;
    rc->h_drift = hdrift;
    rc->lambda_end = lam;
    return;
  }
  int nc = cs.ncross > 255 ? 255 : cs.ncross;
  uint16_t cls = (uint16_t)(status | (nc << 8));
  if (a.level == 0) {
    int64_t n = (int64_t)a.n_items;
    a.base_I[item] = cs.I[0];
    a.base_I[n + item] = cs.I[1];
    a.base_I[2 * n + item] = cs.I[2];
    a.base_I[3 * n + item] = cs.I[3];
    a.base_cls[item] = cls;
    a.base_depth[item] = 0;
    const OutPtrs& o = a.out[img];
    int64_t pix = item - (int64_t)img * a.npix;
    o.status[pix] = (uint8_t)status;
    o.ncross[pix] = (uint8_t)nc;
    if (o.h_drift) o.h_drift[pix] = hdrift;
    if (o.steps) {
      o.steps[pix] = nacc;
      o.steps[a.npix + pix] = nrej;
    }
    // a ray finishing in a resumed pass (FP64 promoted, or FP32 after
    // demotion) took FP64 steps
    if (o.promoted) o.promoted[pix] = (uint8_t)(a.source == 1);
  } else {
    int64_t c = a.lv.cap;
    a.lv.I[item] = cs.I[0];
    a.lv.I[c + item] = cs.I[1];
    a.lv.I[2 * c + item] = cs.I[2];
    a.lv.I[3 * c + item] = cs.I[3];
    a.lv.cls[item] = cls;
    a.lv.depth[item] = (uint8_t)a.level;
  }
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Number of work items of this pass.
__device__ __forceinline__ int64_t pass_items(const TraceArgs& a) {
  if (a.source == 1) {
    unsigned long long c = *a.spill_in_count;
    return (int64_t)(c < (unsigned long long)a.spill_cap ? c : (unsigned long long)a.spill_cap);
  }
  if (a.mode == 0 && a.level > 0) {
    unsigned long long c = a.hdr->count[a.level];
    return (int64_t)(c < (unsigned long long)a.lv.cap ? c : (unsigned long long)a.lv.cap);
  }
  return a.n_items;
}

// Warp-aggregated claim of `need` lanes' next items from a queue cursor.
__device__ __forceinline__ int64_t claim(unsigned long long* head, bool need, int lane) {
  unsigned mask = __ballot_sync(kFull, need);
  if (!mask) return -1;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(head, (unsigned long long)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  return need ? (int64_t)base + __popc(mask & ((1u << lane) - 1u)) : -1;
}

// Whether a lane without a ray claims the next item now.  With Batch > 1 a
// free lane waits until Batch lanes of its warp are free (or none is busy),
// so that the divergent start of new rays (a resume or a launch with its
// dependent global loads) runs for several lanes at once.  All lanes of the
// warp must call it.
template <int Batch>
__device__ __forceinline__ bool refill_now(bool want, bool active) {
  if (Batch <= 1) return want;
  const unsigned wm = __ballot_sync(kFull, want);
  const unsigned am = __ballot_sync(kFull, active);
  return want && (__popc(wm) >= Batch || am == 0u);
}

// Pass timeline marks (WsHeader::t_pass): the first writer of a slot wins.
__device__ __forceinline__ void mark_first(unsigned long long* slot) {
  if (*reinterpret_cast<volatile unsigned long long*>(slot) == 0ull)
    atomicCAS(slot, 0ull, globaltimer());
}

// Warp sum of lane tallies, one atomic per warp.
__device__ __forceinline__ void flush_tally(unsigned long long* dst, unsigned long long v,
                                            int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane == 0 && v) atomicAdd(dst, v);
}

}  // namespace bhrt
