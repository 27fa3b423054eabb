// bh_common.cuh -- device-side data layout and physics shared by the CUDA
// kernels of the ray tracer (not by the CPU oracle, which is independent).
//
// Physics: the rotating Kerr-like metric of Sec. 2.2 (Eqs. 23-31) with the
// static lapses of Sec. 2.1 (Kerr, Einasto Eq. 9, cored-NFW Eq. 13), and
// Hamilton's equations of Sec. 3.1 (Eqs. 57-62) written in the
// Christoffel-free separated form obtained by multiplying the Hamiltonian
// by Sigma (the separated Hamilton-Jacobi equation, Eq. 56):
//   W = 2 Sigma H = Delta p_R^2 - P^2/Delta + p_th^2 + Q^2,
//   P = (R^2 + chi^2) E - chi ell,  Q = ell/sin(th) - chi E sin(th),
// so that dp/dlambda = -(dW)/(2 Sigma) + W dSigma/(2 Sigma^2) exactly equals
// -1/2 d(g^{ab}) p_a p_b of Eqs. (61)-(62).
#pragma once
#include <cstdint>

namespace bhrt {

constexpr int kMaxLevels = 3;

// Per-image constants, computed on the host (Sec. 2.3 horizon, Sec. 3.2
// ZAMO tetrad scalars, Sec. 5 emission), read by every ray of the image.
struct alignas(16) ImgParams {
  int32_t metric;
  int32_t max_steps;
  int32_t nx, ny;
  double chi, lamE, eta, lamc;
  double r_obs, incl;
  double x_min, y_min, dx, dy;
  // ZAMO frame at (R_o, theta_o): omega (Eq. 63), N (Eq. 65) and the
  // square roots of g_RR, g_thth, g_phph that normalise the triad (Eqs. 66-68).
  double zamo_w, zamo_N, sq_grr, sq_gth, sq_gph;
  double r_plus, R_cap, R_esc, R_in;
  double j0, p, R_s, sig_in, sig_out, R_out;
  double H0, hh;           // disk height H(rho) = H0 + hh rho (Eq. 84)
  double isig_in, isig_out, iR_s, iR_in;  // reciprocals for the emissivity (both modes)
  float vf[10];            // the same emission constants in FP32 (mixed path):
                           // H0, hh, R_in, 1/sig_in, 1/sig_out, R_out, p, 1/R_s, j0, 1/R_in
  double rtol, atol, thdot_min, dlam_min, promote_R, demote_R;
  double sin_o, isin_o;    // sin(theta_o) and its reciprocal (launch Carter constant)
  double kappa;            // mixed: near-double-root threshold of the radial potential
  int32_t promote_ncross;  // mixed: promote once N_cross reaches this inside demote_R
  int32_t volumetric;      // 1: intensity = Eq. (88) integral (seventh ODE component)
};

// Workspace header (first 256 bytes of every workspace).
struct alignas(256) WsHeader {
  int32_t status;          // bh_status written by the device
  int32_t pad0;
  unsigned long long head[kMaxLevels + 1];   // persistent-queue cursors
  unsigned long long count[kMaxLevels + 1];  // items per level
  unsigned long long t_start;                // %globaltimer at launch (ns)
  unsigned long long budget_ns;              // 0 = no budget
  unsigned long long rays[kMaxLevels + 1];   // rays finished per level
  unsigned long long accepted;               // accepted FP64 steps
  unsigned long long rejected;               // rejected FP64 steps
  unsigned long long accepted32;             // accepted FP32 steps (mixed path)
  unsigned long long rejected32;             // rejected FP32 steps (mixed path)
  unsigned long long qhead[2][kMaxLevels + 1];   // cursors: 0 promoted, 1 demoted
  unsigned long long qcount[2][kMaxLevels + 1];  // queue lengths
  unsigned long long promoted_rays;          // rays handed to FP64
  unsigned long long spill_full;             // promotions refused (queue full)
  unsigned long long max_ray_steps;          // longest ray (attempted steps)
  // Timeline of each trace pass (0 main, 1 FP64 promoted, 2 FP32 demoted)
  // per level, %globaltimer ns: [0] first warp start, [1] first warp to
  // find the queue empty, [2] last warp exit.  The span [1]..[2] is the
  // tail in which warps run with idle lanes.
  unsigned long long t_pass[3][3][kMaxLevels + 1];
  // Stepping-loop iterations of the trace kernels ([0] FP32, [1] FP64) and
  // the lanes with a ray in them: lane utilisation of the persistent loop.
  unsigned long long warp_iters[2];
  unsigned long long lane_iters[2];
};

// Structure-of-arrays records of one refinement level.
struct LevelRecs {
  uint64_t* key;      // base_id << 16 | level << 12 | digits
  uint32_t* img;      // image index
  double* I;          // [4][cap] leaf value (I_tot, I_0, I_1, I_2)
  uint16_t* cls;      // status | min(ncross,255) << 8
  int32_t* child;     // index of first child in the next level, -1 if leaf
  uint8_t* depth;     // deepest level below this cell
  int64_t cap;
};

// Lapse H(R) and dH/dR.  Kerr: 1 - 2/R; Einasto Eq. (9); cored-NFW Eq. (13).
template <class T>
struct MetricConsts {
  int metric;
  T chi, chi2, il;      // il = 1/lambda_E
  T eta_lc, lc, ilc;    // eta*lambda_c, lambda_c, 1/lambda_c
};


__device__ __forceinline__ float d_exp(float x) { return __expf(x); }

// FP32 log(1 + x) for x > -1 without a slow path: u = 1 + x = 2^e m with
// m in [sqrt(1/2), sqrt(2)), log m = 2 atanh(t), t = (m - 1)/(m + 1),
// |t| <= 0.172, by its series to t^9 (truncation below 3e-9), plus the
// first-order correction for the rounding of 1 + x.
__device__ __forceinline__ float d_log1p(float x) {
  const float u = 1.0f + x;
  const int ub = __float_as_int(u);
  // biased exponent as a float: 2^23 + e_b read back, minus 2^23 + 127
  float e = __int_as_float(0x4b000000 | ((ub >> 23) & 0xff)) - 8388735.0f;
  float m = __int_as_float((ub & 0x007fffff) | 0x3f800000);  // [1, 2)
  if (m > 1.41421356f) {
    m *= 0.5f;
    e += 1.0f;
  }
  const float t = __fdividef(m - 1.0f, m + 1.0f), t2 = t * t;
  float p = fmaf(t2, 0.111111111f, 0.142857143f);          // 1/9, 1/7
  p = fmaf(p, t2, 0.2f);                                    // 1/5
  p = fmaf(p, t2, 0.333333333f);                            // 1/3
  const float lm = 2.0f * fmaf(p * t2, t, t);
  const float corr = __fdividef(x - (u - 1.0f), u);
  return fmaf(e, 0.693147181f, lm + corr);                  // ln 2
}
// FP64 sine and cosine without a slow path, for the polar angle and trial
// stages a few radians around it: Cody & Waite reduction by the nearest
// multiple q of pi/2 with a two-part constant (exact to far below one unit
// for |q| < 2^20), sin r = r + r^3 g(r^2) and cos r = 1 - r^2/2 + r^4 h(r^2)
// on |r| <= pi/4 with g and h six-term polynomials fitted by Chebyshev
// interpolation at 40 digits (fit_sincos.py; approximation error below 1.3e-17
// for the sine and 5e-19 for the cosine, two FP64 operations fewer per sine and
// one per cosine than Taylor series of the same accuracy), then a rotation by
// q quarter turns;
// q is rounded by adding 1.5 * 2^52, whose low mantissa bits hold q mod 4.
__device__ __forceinline__ void d_sincos(double x, double* s, double* c) {
  const double qm = fma(x, 0.63661977236758134308, 6755399441055744.0);
  const double q = qm - 6755399441055744.0;
  const int iq = (int)(unsigned)__double2loint(qm);
  double r = fma(q, -1.5707963267948966192, x);            // pi/2, leading part
  r = fma(q, -6.1232339957367660359e-17, r);               // pi/2, trailing part
  const double r2 = r * r;
  double ps = fma(r2, 1.5918129294866608e-10, -2.5051131845003624e-08);  // g
  ps = fma(ps, r2, 2.755731610255244e-06);
  ps = fma(ps, r2, -0.00019841269836758574);
  ps = fma(ps, r2, 0.008333333333330948);
  ps = fma(ps, r2, -0.16666666666666666);
  const double sr = fma(ps * r2, r, r);
  double pc = fma(r2, -1.1382632425521717e-11, 2.08761462684032e-09);  // h
  pc = fma(pc, r2, -2.7557317271729793e-07);
  pc = fma(pc, r2, 2.480158729876569e-05);
  pc = fma(pc, r2, -0.0013888888888887398);
  pc = fma(pc, r2, 0.041666666666666664);
  pc = fma(pc, r2, -0.5);
  const double cr = fma(pc, r2, 1.0);
  const double so = (iq & 1) ? cr : sr, co = (iq & 1) ? sr : cr;
  *s = (iq & 2) ? -so : so;
  *c = ((iq + 1) & 2) ? -co : co;
}
// FP32 sine and cosine without a slow path (the polar angle and the trial
// stages around it stay within a few radians): Cody & Waite reduction by
// the nearest multiple q of pi/2 with a two-part constant, Taylor
// polynomials of sin r and cos r on |r| <= pi/4 (truncation below 2e-9),
// then a rotation by q quarter turns.  The argument is an unevaluated sum
// hi + lo: the leading part of q pi/2 comes off hi exactly (near a multiple
// of pi/2 the difference is representable), so the reduced argument keeps
// its relative precision near the poles theta = 0, pi even where hi + lo
// rounded to one float would carry an absolute error of half an ulp of pi.
__device__ __forceinline__ void d_sincos2(float hi, float lo, float* s, float* c) {
  // q = nearest integer to 2x/pi, rounded by adding 1.5 * 2^23 (its low
  // mantissa bits then hold q mod 4), so no conversion instruction is needed
  const float qm = fmaf(hi + lo, 0.636619772f, 12582912.0f);  // 2/pi, 1.5 * 2^23
  const float q = qm - 12582912.0f;
  const int iq = __float_as_int(qm);
  float r = fmaf(q, -1.57079637f, hi);                     // pi/2, leading part
  r = fmaf(q, 4.37113883e-8f, r + lo);                     // pi/2, trailing part
  const float r2 = r * r;
  float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);   // 1/9!, -1/7!
  ps = fmaf(ps, r2, 8.33333333e-3f);                       // 1/5!
  ps = fmaf(ps, r2, -1.66666667e-1f);                      // -1/3!
  const float sr = fmaf(ps * r2, r, r);
  float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);   // -1/10!, 1/8!
  pc = fmaf(pc, r2, -1.38888889e-3f);                      // -1/6!
  pc = fmaf(pc, r2, 4.16666667e-2f);                       // 1/4!
  pc = fmaf(pc, r2, -0.5f);
  const float cr = fmaf(pc, r2, 1.0f);
  const float so = (iq & 1) ? cr : sr, co = (iq & 1) ? sr : cr;
  *s = (iq & 2) ? -so : so;
  *c = ((iq + 1) & 2) ? -co : co;
}
__device__ __forceinline__ void d_sincos(float x, float* s, float* c) { d_sincos2(x, 0.f, s, c); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
// FP64 reciprocal without a slow path: the hardware's approximate reciprocal
// (rcp.approx.ftz.f64) refined by two Newton steps r <- r + r (1 - x r),
// within about one unit in the last place for the normal, finite x of the
// right-hand side.
__device__ __forceinline__ double d_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float d_rcp(float x) { return __fdividef(1.0f, x); }

// FP64 1/sqrt(x) for normal, finite x > 0 without a slow path: the
// hardware's approximate reciprocal square root (rsqrt.approx.ftz.f64)
// refined by two Newton steps y <- y (3 - x y^2) / 2, within about one unit
// in the last place.
__device__ __forceinline__ double d_rsqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double hx = 0.5 * x;
  y = y * fma(-hx, y * y, 1.5);
  return y * fma(-hx, y * y, 1.5);
}
// 2^(j/32) for j = 0 .. 31, each the double nearest to the exact value.
static __device__ const double kExp2Tab[32] = {
    1.0, 1.0218971486541166, 1.0442737824274138, 1.0671404006768237,
    1.0905077326652577, 1.1143867425958924, 1.1387886347566916, 1.1637248587775775,
    1.189207115002721, 1.215247359980469, 1.241857812073484, 1.2690509571917332,
    1.2968395546510096, 1.3252366431597413, 1.3542555469368927, 1.383909881963832,
    1.4142135623730951, 1.4451808069770467, 1.4768261459394993, 1.5091644275934228,
    1.5422108254079407, 1.5759808451078865, 1.6104903319492543, 1.645755478153965,
    1.681792830507429, 1.718619298122478, 1.7562521603732995, 1.7947090750031072,
    1.8340080864093424, 1.8741676341103, 1.9152065613971474, 1.9571441241754002};

// FP64 exp without a slow path: x = (32 q + j) ln2 / 32 + r with 32 q + j the
// nearest integer to 32 x / ln2 (rounded by adding 1.5 * 2^52; its low bits
// then hold it in two's complement) and r reduced by a two-part ln2 / 32
// (Cody & Waite), |r| <= ln2 / 64; e^r by its Taylor series to r^6
// (truncation below 4e-18); 2^(j/32) from the table and 2^q assembled in the
// exponent field.  Results below 2^-1022 flush to zero, above 2^1023 become
// +inf.  Twelve FP64 operations against eighteen for a Taylor series on
// |r| <= ln2 / 2.
__device__ __forceinline__ double d_exp(double x) {
  if (!(x > -708.0)) return x != x ? x : 0.0;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
  const double km = fma(x, 46.16624130844683, 6755399441055744.0);  // 32/ln2, 1.5 * 2^52
  const double k = km - 6755399441055744.0;
  const int ik = (int)(unsigned)__double2loint(km);
  double r = fma(k, -0.02166084939249829, x);   // ln2 / 32, leading part
  r = fma(k, -7.247021293269686e-19, r);         // ln2 / 32, trailing part
  double p = fma(r, 0.001388888888888889, 0.008333333333333333);  // 1/6!, 1/5!
  p = fma(p, r, 0.041666666666666664);  // 1/4!
  p = fma(p, r, 0.16666666666666666);   // 1/3!
  p = fma(p, r, 0.5);                   // 1/2!
  p = fma(p, r, 1.0);                   // 1/1!
  p = fma(p, r, 1.0);                   // 1/0!
  const double t = __ldg(&kExp2Tab[ik & 31]);
  return (t * p) * __longlong_as_double((long long)((ik >> 5) + 1023) << 52);
}

// FP64 log(1 + x) for x > -1 without a slow path: u = 1 + x = 2^e m with m in
// [sqrt(1/2), sqrt(2)); log m = 2 atanh(t), t = (m - 1)/(m + 1), |t| <= 0.172,
// by its series to t^21 (truncation below 1e-18); e ln 2 with a two-part ln 2;
// plus the first-order correction for the rounding of 1 + x.
__device__ __forceinline__ double d_log1p(double x) {
  const double u = 1.0 + x;
  const long long ub = __double_as_longlong(u);
  int e = (int)((ub >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((ub & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
  if (m > 1.4142135623730951) {
    m *= 0.5;
    e += 1;
  }
  const double t = (m - 1.0) * d_rcp(m + 1.0), t2 = t * t;
  double p = fma(t2, 0.047619047619047616, 0.05263157894736842);  // 1/21, 1/19
  p = fma(p, t2, 0.058823529411764705);  // 1/17
  p = fma(p, t2, 0.06666666666666667);  // 1/15
  p = fma(p, t2, 0.07692307692307693);  // 1/13
  p = fma(p, t2, 0.09090909090909091);  // 1/11
  p = fma(p, t2, 0.1111111111111111);  // 1/9
  p = fma(p, t2, 0.14285714285714285);  // 1/7
  p = fma(p, t2, 0.2);  // 1/5
  p = fma(p, t2, 0.3333333333333333);  // 1/3
  const double lm = 2.0 * fma(p * t2, t, t);
  const double corr = (x - (u - 1.0)) * d_rcp(u);
  const double ed = (double)e;
  return fma(ed, 0.6931471805598903, fma(ed, 5.497923018708371e-14, lm + corr));
}

__device__ __forceinline__ double d_pow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ double d_tanh(double x) { return tanh(x); }

template <class T>
__device__ __forceinline__ void lapse(const MetricConsts<T>& m, T R, T iR, T& H, T& dH) {
  const T two = T(2);
  if (m.metric == 1) {
    T e = d_exp(-R * m.il);
    T poly = two * iR + two * m.il + R * m.il * m.il;
    T dpoly = -two * iR * iR + m.il * m.il;
    H = T(1) - two * iR + poly * e;
    dH = two * iR * iR + (dpoly - poly * m.il) * e;
  } else if (m.metric == 2) {
    T q = d_rcp(R + m.lc);
    T L = d_log1p(R * m.ilc);
    T S = m.eta_lc * (q - two * iR * L);
    T dS = m.eta_lc * (-q * q + two * iR * iR * L - two * iR * q);
    T eS = d_exp(S);
    H = eS - two * iR;
    dH = eS * dS + two * iR * iR;
  } else {
    H = T(1) - two * iR;
    dH = two * iR * iR;
  }
}

// Right-hand side of Hamilton's equations (Eqs. 57-62) for the state
// (T, R, th, phi, p_R, p_th) with constants E = -p_T, ell = p_phi (Eq. 48).
// Returns false when the point is not admissible (R <= 0 or Delta <= 0).
// theta may leave (0, pi) inside a step (the equations continue through
// the polar axis; the accepted state is reflected back by the caller).
// Also returns W = 2 Sigma H and P^2/Delta for the null-constraint monitor.
// The ray's constants of motion E = -p_T, ell = p_phi (Eq. 48) with the
// products of them and the spin that the right-hand side uses, formed once
// per ray or step rather than in each of its evaluations.
template <class T>
struct RayC {
  T E, ell;
  T cE, cl, c2E, E4;  // chi E, chi ell, chi^2 E, 4 E
};
template <class T>
__device__ __forceinline__ RayC<T> ray_consts(const MetricConsts<T>& m, T E, T ell) {
  RayC<T> k;
  k.E = E;
  k.ell = ell;
  k.cE = m.chi * E;
  k.cl = m.chi * ell;
  k.c2E = m.chi2 * E;
  k.E4 = T(4) * E;
  return k;
}

// geo_rhs_sc takes sin(theta) and cos(theta) instead of theta.
template <class T>
__device__ __forceinline__ bool geo_rhs_sc(const MetricConsts<T>& m, const RayC<T>& k, T R, T s,
                                           T c, T pR, T pth, T d[6], T& W, T& P2oD) {
  T R2 = R * R;
  T Sig = R2 + m.chi2 * c * c;               // Eq. (23)
  // the lapse needs 1/R before Delta exists: 1/R and 1/Sigma from one
  // reciprocal of R Sigma, then 1/Delta and 1/sin(theta) from one more
  T iRS = d_rcp(R * Sig);
  T iR = Sig * iRS, iS = R * iRS;
  T H, dH;
  lapse(m, R, iR, H, dH);
  T Dl = R2 * H + m.chi2;                    // Eq. (25)
  T dDl = T(2) * R * H + R2 * dH;            // Eq. (35)
  T iDs = d_rcp(Dl * s);
  T iD = s * iDs, is = Dl * iDs;
  T r2a2 = R2 + m.chi2;
  T P = r2a2 * k.E - k.cl;
  T Q = k.ell * is - k.cE * s;
  T PoD = P * iD;
  P2oD = P * PoD;
  W = Dl * pR * pR - P2oD + pth * pth + Q * Q;
  d[0] = (r2a2 * PoD + (k.cl - k.c2E * (s * s))) * iS;           // Eq. (57)
  d[1] = Dl * pR * iS;                                            // Eq. (59)
  d[2] = pth * iS;                                                // Eq. (60)
  d[3] = (m.chi * PoD + k.ell * is * is - k.cE) * iS;             // Eq. (58)
  T dW_R = dDl * pR * pR - k.E4 * R * PoD + PoD * PoD * dDl;      // d(W)/dR
  T dQ = -k.ell * c * is * is - k.cE * c;                          // dQ/dth
  T iS2 = iS * iS;
  d[4] = T(-0.5) * dW_R * iS + W * R * iS2;                       // Eq. (61)
  d[5] = -Q * dQ * iS - W * m.chi2 * s * c * iS2;                 // Eq. (62)
  return (R > T(0)) && (Dl > T(0));
}
template <class T>
__device__ __forceinline__ bool geo_rhs(const MetricConsts<T>& m, T E, T ell, T R, T th, T pR,
                                        T pth, T d[6], T& W, T& P2oD) {
  T s, c;
  d_sincos(th, &s, &c);
  return geo_rhs_sc(m, ray_consts(m, E, ell), R, s, c, pR, pth, d, W, P2oD);
}

// Screen position of a cell from its key (bit-exact cell-centred
// arithmetic, no contraction: parent centre + ((k + 1/2)/4 - 1/2) width).
__device__ __forceinline__ void cell_centre(const ImgParams& ip, uint64_t key, double& X,
                                            double& Y) {
  const int64_t base = (int64_t)(key >> 16);
  const int level = (int)((key >> 12) & 0xF);
  const int i = (int)(base % ip.nx), j = (int)(base / ip.nx);
  X = __dadd_rn(ip.x_min, __dmul_rn((double)i + 0.5, ip.dx));
  Y = __dadd_rn(ip.y_min, __dmul_rn((double)j + 0.5, ip.dy));
  double wx = ip.dx, wy = ip.dy;
  for (int l = 1; l <= level; ++l) {
    int dgt = (int)((key >> (4 * (3 - l))) & 0xF);
    int cx = dgt & 3, cy = dgt >> 2;
    double ox = ((double)cx + 0.5) / 4.0 - 0.5;
    double oy = ((double)cy + 0.5) / 4.0 - 0.5;
    X = __dadd_rn(X, __dmul_rn(ox, wx));
    Y = __dadd_rn(Y, __dmul_rn(oy, wy));
    wx = wx / 4.0;
    wy = wy / 4.0;
  }
}

}  // namespace bhrt
