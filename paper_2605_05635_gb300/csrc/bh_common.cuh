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

// Constants of the lapse H(R) (Kerr: 1 - 2/R; Einasto Eq. 9; cored-NFW
// Eq. 13) in the precision of the right-hand side that reads them.
template <class T>
struct MetricConsts {
  int metric;
  T chi, chi2, il;      // il = 1/lambda_E
  T eta_lc, lc, ilc;    // eta*lambda_c, lambda_c, 1/lambda_c
};

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
  // the lapse constants in FP64 and FP32, formed once on the host (their
  // reciprocals are FP64 divisions, which the kernels would otherwise repeat
  // at every ray start and in every demotion test)
  MetricConsts<double> md;
  MetricConsts<float> mf;
};

// The lapse constants of an image from its parameters (the host fills
// ImgParams::md and ::mf with it; the kernels read those copies).
template <class T>
__host__ __device__ inline MetricConsts<T> make_metric_consts(const ImgParams& ip) {
  MetricConsts<T> m;
  m.metric = ip.metric;
  m.chi = (T)ip.chi;
  m.chi2 = (T)(ip.chi * ip.chi);
  m.il = ip.metric == 1 ? (T)(1.0 / ip.lamE) : T(0);
  m.lc = (T)ip.lamc;
  m.ilc = ip.metric == 2 ? (T)(1.0 / ip.lamc) : T(0);
  m.eta_lc = (T)(ip.eta * ip.lamc);
  return m;
}

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
  // quadrant signs by flipping the sign bit (integer pipe, not an FP64 negation)
  *s = __longlong_as_double(__double_as_longlong(so) ^ ((long long)(iq & 2) << 62));
  *c = __longlong_as_double(__double_as_longlong(co) ^ ((long long)((iq + 1) & 2) << 62));
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
  // the range tests only where |x| >= 708 (or x is inf or NaN), found by an
  // integer test of the leading word: FP64 compares take FP64-pipe slots
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40862000) {
    if (!(x > -708.0)) return x != x ? x : 0.0;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
  }
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

// FP64 log(1 + x) for x > -1 without a slow path or a division:
// u = 1 + x = 2^e m with m in [1, 2); the six leading fraction bits of m pick
// j and a table factor r_j near 1/m (gen_log_table.py), so z = m r_j - 1 (one
// fma) has |z| <= 1/64 and log u = (e + s_j) ln 2 + T_j + log(1 + z), with
// T_j = -log r_j - s_j ln 2 as two doubles and log(1 + z) by its Taylor
// series to z^9 (truncation below 6e-18 relative); the rounding of 1 + x is
// corrected to first order, (x - (u - 1)) / u, with 1/u taken as r_j 2^-e.
static __device__ const double kLogR[64] = {
    1.0, 0.9770992366412213, 0.9624060150375939, 0.9481481481481482,
    0.9343065693430657, 0.920863309352518, 0.9078014184397163, 0.8951048951048951,
    0.8827586206896552, 0.8707482993197279, 0.8590604026845637, 0.847682119205298,
    0.8366013071895425, 0.8258064516129032, 0.8152866242038217, 0.8050314465408805,
    0.7950310559006211, 0.7852760736196319, 0.7757575757575758, 0.7664670658682635,
    0.757396449704142, 0.7485380116959064, 0.7398843930635838, 0.7314285714285714,
    0.7231638418079096, 0.7150837988826816, 0.7071823204419889, 0.6994535519125683,
    0.6918918918918919, 0.6844919786096256, 0.6772486772486772, 0.6701570680628273,
    0.6632124352331606, 0.6564102564102564, 0.649746192893401, 0.6432160804020101,
    0.6368159203980099, 0.6305418719211823, 0.624390243902439, 0.6183574879227053,
    0.6124401913875598, 0.6066350710900474, 0.6009389671361502, 0.5953488372093023,
    0.5898617511520737, 0.5844748858447488, 0.579185520361991, 0.5739910313901345,
    0.5688888888888889, 0.5638766519823789, 0.5589519650655022, 0.5541125541125541,
    0.5493562231759657, 0.5446808510638298, 0.540084388185654, 0.5355648535564853,
    0.5311203319502075, 0.5267489711934157, 0.5224489795918368, 0.5182186234817814,
    0.5140562248995983, 0.5099601593625498, 0.5059288537549407, 0.5,
};
static __device__ const double kLogTHi[64] = {
    0.0, 0.023167059281534418, 0.03831886430213666, 0.05324451451881224,
    0.06795066190850778, 0.08244366921107454, 0.09672962645855114, 0.11081436634029011,
    0.12470347850095725, 0.1384023228591192, 0.151916042025842, 0.16524957289530717,
    0.17840765747281825, 0.19139485299962947, 0.20421554142869083, 0.2168739383006143,
    0.2293741010648459, 0.24171993688714513, 0.25391520998096345, 0.2659635484971379,
    0.2778684510034563, 0.2896332925830427, 0.30126133057816185, 0.3127557100038969,
    0.324119468654212, 0.3353555419211378, 0.3464667673462086, 0.3574558889218038,
    0.36832556115870757, 0.3790783529349695, 0.38971675114002524, 0.40024316412701266,
    -0.28248725557467697, -0.27217788591581565, -0.2619737157415739, -0.2518726197550701,
    -0.2418725364204867, -0.23197146543777517, -0.2221674653411543, -0.21245865121419336,
    -0.20284319251475144, -0.19331931100349606, -0.18388527877013738, -0.17453941635189965,
    -0.16528009093910292, -0.1561057146630616, -0.14701474296180975, -0.1380056730194437,
    -0.12907704227514236, -0.12022742699815989, -0.11145544092532278, -0.10275973395776894,
    -0.09413899091386191, -0.08559193033540353, -0.0771173033444312, -0.06871389254805173,
    -0.06038051098890748, -0.0521160011390141, -0.04391923393483558, -0.03578910785158529,
    -0.02772454801485477, -0.019724505347778573, -0.011787955752042173, 0.0,
};
static __device__ const double kLogTLo[64] = {
    0.0, -3.095927552179262e-19, -2.3579961573512846e-18, 1.803871134979952e-18,
    3.9239563038692484e-18, -4.707903082046854e-18, -4.0291867005826106e-18, 2.0511100808140527e-18,
    -4.6522609636496624e-18, -1.3766819196398948e-17, 4.1233095848339465e-19, -9.227573884334224e-18,
    1.2720936612962572e-17, -1.126213516780448e-17, 7.9379985298027e-18, 6.285749669211092e-18,
    -5.684839459813236e-18, 1.323779871210866e-17, -7.180735656435798e-18, 1.35209848201012e-19,
    2.2502748630777633e-17, 2.0535953219858177e-17, -1.5120043309967385e-17, -1.3650721793001109e-17,
    -4.488767429940198e-18, -1.3746739934976202e-17, -3.591951952851805e-18, -2.4269548334425144e-17,
    2.690672380132659e-17, 1.8481479367349684e-17, 2.734172667856699e-17, -1.655340963311913e-17,
    4.5622709592656976e-18, -1.859318262481925e-17, 1.878144810277299e-17, -1.2846709260565683e-17,
    -5.086688062206503e-18, 1.0705552511300431e-17, 1.1664564654755913e-17, 1.8248974208288598e-18,
    9.177560001701116e-18, 2.3084535888000873e-18, -1.51192377141417e-18, -1.2294483916404324e-17,
    1.4935930931804023e-18, 1.2806970330932863e-17, -1.6045849809178003e-18, -9.927673066865803e-18,
    1.380833506137427e-17, -6.703429385028035e-18, 4.722382936838005e-18, 5.5749926045490845e-18,
    1.9720664099579867e-18, 4.505830273858094e-18, -1.6980741255382134e-18, 5.131966502090055e-18,
    1.2896019993525642e-18, -2.445091174292264e-18, -1.7623552700046253e-18, -7.2846227792942925e-19,
    -1.6936634670586275e-19, 1.3445979863167513e-18, -2.208154666796599e-19, 0.0,
};
__device__ __forceinline__ double d_log1p(double x) {
  const double u = 1.0 + x;
  const long long ub = __double_as_longlong(u);
  const int e = (int)((ub >> 52) & 0x7ff) - 1023;
  const int j = (int)((ub >> 46) & 63);
  const double m = __longlong_as_double((ub & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
  const double r = __ldg(&kLogR[j]);
  const double z = fma(m, r, -1.0);
  double p = fma(z, 0.1111111111111111, -0.125);  // 1/9, -1/8
  p = fma(p, z, 0.14285714285714285);   // 1/7
  p = fma(p, z, -0.16666666666666666);  // -1/6
  p = fma(p, z, 0.2);                   // 1/5
  p = fma(p, z, -0.25);                 // -1/4
  p = fma(p, z, 0.3333333333333333);    // 1/3
  p = fma(p, z, -0.5);                  // -1/2
  const double lz = fma(z * z, p, z);
  const double sc = __longlong_as_double((long long)(1023 - e) << 52);  // 2^-e
  const double corr = (x - (u - 1.0)) * (r * sc);
  const double k = (double)(e + (j >> 5));
  return fma(k, 0.6931471805598903,
             __ldg(&kLogTHi[j]) + fma(k, 5.497923018708371e-14, __ldg(&kLogTLo[j]) + (lz + corr)));
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

// x > 0.  For FP64 by the bit pattern on the integer pipes (exact for every
// non-NaN x, -0 included; a NaN with a clear sign bit passes, and then fails
// the step's error test).
template <class T>
__device__ __forceinline__ bool is_pos(T x) {
  return x > T(0);
}
template <>
__device__ __forceinline__ bool is_pos<double>(double x) {
  return __double_as_longlong(x) > 0;
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
  return is_pos(R) && is_pos(Dl);
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
