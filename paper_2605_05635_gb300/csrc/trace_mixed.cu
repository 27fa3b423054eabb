// trace_mixed.cu -- FP32-bulk integrator kernel of the mixed-precision path.
//
// Same method as trace.cu (launch Eqs. 63-74, Hamilton's equations
// Eqs. 57-62, Dormand-Prince 5(4), crossings Sec. 3.3 / 4.2, redshift and
// intensity Eqs. 83-91), with the precision split that suits GB300, whose
// FP64 rate is 1/64 of FP32:
//   - the right-hand side, the stage combinations and the error estimate
//     run in FP32;
//   - the state is carried as an unevaluated sum hi + lo of two floats, so
//     each step's increment is added with ~48-bit precision (the transverse
//     position at R ~ 1000 would otherwise drift by ~R 1e-7 per step);
//   - the launch and the constants of motion (E, ell) are formed in FP64
//     and rounded; the starting step, crossing roots, transfer maps,
//     redshift, emissivity and the volumetric source run in FP32, so the
//     stepping loop issues no FP64 instruction;
//   - a ray is promoted to the FP64 kernel when it comes within promote_R of
//     the horizon, when, winding to image order n >= 2 (N_cross >= 3,
//     Sec. 4.2), it is inside demote_R, or when it nears a double root of
//     its radial potential (kappa); the FP64 pass hands it back once it is
//     outgoing beyond demote_R or past that root, and a second FP32 pass (no
//     further promotion) finishes it.  Promotion is a hand-off through a
//     queue rather than a per-lane branch, so warps never mix FP64 and FP32
//     steps.
#include <cuda_runtime.h>

#include "integrator.cuh"

namespace bhrt {

// (hi, lo) += d with round-to-nearest two-sum / fast-two-sum (no
// contraction): the pair keeps ~48 bits of the running sum.
__device__ __forceinline__ void df_add(float& hi, float& lo, float d) {
  float s = __fadd_rn(hi, d);
  float bb = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  float t = __fadd_rn(lo, e);
  float nh = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(nh, s));
  hi = nh;
}

__device__ __forceinline__ void df_from(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

__device__ __forceinline__ double df_to(float hi, float lo) { return (double)hi + (double)lo; }

// The right-hand side out of line, for the call sites that run once per ray
// (launch, resume, axis reflection): the stepping loop keeps the only
// inlined copy, so these do not grow the code the loop runs from.
struct RhsF {
  float d[6];
  float W, P2;
};
// theta is the pair th + thl (see d_sincos2).
static __device__ __noinline__ RhsF rhs_f32(MetricConsts<float> m, float E, float ell, float R,
                                            float th, float thl, float pR, float pth) {
  RhsF o;
  float s, c;
  d_sincos2(th, thl, &s, &c);
  geo_rhs_sc(m, ray_consts(m, E, ell), R, s, c, pR, pth, o.d, o.W, o.P2);
  return o;
}
__device__ __forceinline__ void rhs_f32_into(const MetricConsts<float>& m, float E, float ell,
                                             float R, float th, float thl, float pR, float pth,
                                             float* d) {
  const RhsF o = rhs_f32(m, E, ell, R, th, thl, pR, pth);
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = o.d[i];
}

// Step-size factor of the FP32 steps: safety 0.8 (0.9 in the FP64 steps),
// clamp [0.2, 10], no growth right after a rejection.  The FP32 error
// estimate fluctuates with rounding, so steps sized for 0.9 of the tolerance
// were rejected a quarter of the time; at 0.8 about 6 % are.
__device__ __forceinline__ float step_factor_mx(float e, bool after_reject) {
  float fac = (e == 0.f) ? 10.f : 0.8f * __powf(e, -0.2f);
  return fminf(fmaxf(fac, 0.2f), after_reject ? 1.f : 10.f);
}

// Free lanes that start new rays together (refill_now): a launch from the
// screen forms the ray's constants in FP64, and a resume reads a spill
// record, both divergent.  The whole warp refills at once: on the 512^2
// sweep the FP32 passes took 172 ms with groups of 16 lanes, 181 ms with
// 24 and 158 ms with 32 (the launches then run convergent).
constexpr int kMxRefillLanes = 32;

// pi/2 as a float pair hi + lo, and pi (hi part) for the axis test.
constexpr float kHalfPiHi = 1.57079637050628662109375f;
constexpr float kHalfPiLo = -4.37113900018624283e-8f;
constexpr float kPiHi = 3.1415927410125732421875f;

// theta - pi/2 from the float pair (hi + lo + extra), exact to the rounding
// of the small terms: the height z = -R sin(theta - pi/2) inside a thin layer
// keeps its relative accuracy, which theta rounded to one float would not.
__device__ __forceinline__ float dtheta_eq(float th_h, float th_l, float extra) {
  return __fadd_rn(__fsub_rn(th_h, kHalfPiHi), __fsub_rn(th_l, kHalfPiLo) + extra);
}

struct RayMx {
  float yh[6], yl[6];  // state T, R, th, phi, p_R, p_th as hi + lo
  float f[6];          // f(y) in FP32 (FSAL)
  float h;
  float lh, ll;        // affine parameter as hi + lo
  double E, ell;
  float Ef, ellf;
  CrossState cs;
  float fI;            // volumetric source at the state (FSAL of the seventh component)
  float Ih, Il;        // volumetric intensity so far as hi + lo (cs.I[0] at hand-off)
  float hdrift;
  int32_t nacc, nrej, steps;
  bool rejected;
};

__device__ __forceinline__ void mx_spill(const RayMx& x, int64_t item, uint32_t img,
                                         SpillRec& s) {
#pragma unroll
  for (int i = 0; i < 6; ++i) s.y[i] = df_to(x.yh[i], x.yl[i]);
  s.h = (double)x.h;
  s.lam = df_to(x.lh, x.ll);
  s.E = x.E;
  s.ell = x.ell;
#pragma unroll
  for (int i = 0; i < 4; ++i) s.I[i] = x.cs.I[i];
  s.lam_last = x.cs.lam_last;
  s.item = item;
  s.img = img;
  s.hdrift = x.hdrift;
  s.ncross = x.cs.ncross;
  s.nacc = x.nacc;
  s.nrej = x.nrej;
  s.steps = x.steps;
  s.flags = (x.cs.have_trusted ? 1 : 0) | (x.rejected ? 2 : 0);
  s.pad = 0;
}

template <bool kVol>
__device__ __forceinline__ void mx_resume(const ImgParams& ip, const SpillRec& s,
                                          const MetricConsts<float>& mf, RayMx& x) {
#pragma unroll
  for (int i = 0; i < 6; ++i) df_from(s.y[i], x.yh[i], x.yl[i]);
  x.h = (float)s.h;
  df_from(s.lam, x.lh, x.ll);
  x.E = s.E;
  x.ell = s.ell;
  x.Ef = (float)s.E;
  x.ellf = (float)s.ell;
#pragma unroll
  for (int i = 0; i < 4; ++i) x.cs.I[i] = s.I[i];
  x.cs.lam_last = s.lam_last;
  x.cs.ncross = s.ncross;
  x.cs.have_trusted = (s.flags & 1) != 0;
  x.rejected = (s.flags & 2) != 0;
  x.hdrift = s.hdrift;
  x.nacc = s.nacc;
  x.nrej = s.nrej;
  x.steps = s.steps;
  rhs_f32_into(mf, x.Ef, x.ellf, x.yh[1], x.yh[2], x.yl[2], x.yh[4], x.yh[5], x.f);
  if (kVol) {
    df_from(s.I[0], x.Ih, x.Il);
    x.fI = ip.volumetric
               ? vol_source32(ip, mf, x.Ef, x.ellf, x.yh[1], dtheta_eq(x.yh[2], x.yl[2], 0.f))
               : 0.f;
  }
}

struct MxConsts {
  float rtol, atol, R_cap, R_esc, promote_R, demote_R, kappa;
  int promote_nc;
};

// Radial turning point of a near-critical ray.  With the radial potential of
// the separated Hamiltonian (Eq. 56), Rr(R) = (Delta p_R)^2 = P^2 - Delta K
// (K = p_th^2 + Q^2), a ray whose Rr has a near-double root is close to the
// photon orbit and about to turn back or to plunge; there its fate and its
// number of windings depend exponentially on the constants of motion.  In
// the quadratic model Rr / P^2 = -delta + c (R - R_c)^2, c = Rr'' / (2 P^2),
// the test Rr < kappa P^2 and Rr'^2 < 2 kappa Rr'' P^2 holds for |delta| <
// kappa within sqrt(kappa / c) of R_c, and not at the turning points of rays
// far from critical (there Rr = 0 but Rr'^2 = 4 c delta P^4).  Rr'' takes
// Kerr's Delta'' = 2 (the halo lapses change it by a few percent): the test
// only decides where FP64 steps start.  FP32.
static __device__ __noinline__ bool near_double_root(MetricConsts<float> m, float E, float ell,
                                                     float R, float th, float pR, float pth,
                                                     float kappa) {
  float s, c;
  d_sincos(th, &s, &c);
  float H, dH;
  lapse(m, R, __fdividef(1.f, R), H, dH);
  const float R2 = R * R;
  const float Dl = R2 * H + m.chi2, dDl = 2.f * R * H + R2 * dH;  // Eqs. (25), (35)
  const float P = (R2 + m.chi2) * E - m.chi * ell;
  const float Q = __fdividef(ell, s) - m.chi * E * s;
  const float K = pth * pth + Q * Q;
  const float DpR = Dl * pR;
  const float Rr = DpR * DpR;
  const float Rp = 4.f * R * E * P - dDl * K;
  const float Rpp = 8.f * R2 * E * E + 4.f * E * P - 2.f * K;
  const float P2 = P * P;
  return Rr < kappa * P2 && Rpp > 0.f && Rp * Rp < 2.f * kappa * Rpp * P2;
}

// Launch of the mixed path: the constants of motion and the launch momenta
// in FP64 (Eqs. 70-74, as in ray_init64), the state as float pairs, and the
// Hairer-Wanner starting step in FP32.
template <bool kVol>
__device__ __forceinline__ void ray_init_mx(const ImgParams& ip, const MetricConsts<float>& mf,
                                            const MxConsts& c, double X, double Y, RayMx& r) {
  const double id = d_rsqrt(ip.r_obs * ip.r_obs + X * X + Y * Y);
  r.ell = ip.sq_gph * (-X * id);
  r.E = ip.zamo_N + ip.zamo_w * r.ell;
  df_from(0.0, r.yh[0], r.yl[0]);
  df_from(ip.r_obs, r.yh[1], r.yl[1]);
  df_from(ip.incl, r.yh[2], r.yl[2]);
  df_from(0.0, r.yh[3], r.yl[3]);
  df_from(ip.sq_grr * (-ip.r_obs * id), r.yh[4], r.yl[4]);
  df_from(ip.sq_gth * (-Y * id), r.yh[5], r.yl[5]);
  r.Ef = (float)r.E;
  r.ellf = (float)r.ell;
  rhs_f32_into(mf, r.Ef, r.ellf, r.yh[1], r.yh[2], r.yl[2], r.yh[4], r.yh[5], r.f);
  float d0 = 0.f, d1 = 0.f, sc[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    sc[i] = c.atol + c.rtol * fabsf(r.yh[i]);
    const float a0 = __fdividef(r.yh[i], sc[i]), a1 = __fdividef(r.f[i], sc[i]);
    d0 += a0 * a0;
    d1 += a1 * a1;
  }
  d0 = sqrtf(d0 / 6.f);
  d1 = sqrtf(d1 / 6.f);
  const float h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * __fdividef(d0, d1);
  float f1[6];
  rhs_f32_into(mf, r.Ef, r.ellf, r.yh[1] + h0 * r.f[1], r.yh[2], r.yl[2] + h0 * r.f[2],
               r.yh[4] + h0 * r.f[4], r.yh[5] + h0 * r.f[5], f1);
  float d2 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float q = __fdividef(f1[i] - r.f[i], sc[i]);
    d2 += q * q;
  }
  d2 = __fdividef(sqrtf(d2 / 6.f), h0);
  const float mx = fmaxf(d1, d2);
  const float h1 = (mx <= 1e-15f) ? fmaxf(1e-6f, h0 * 1e-3f) : __powf(__fdividef(0.01f, mx), 0.2f);
  r.h = fminf(100.f * h0, h1);
  r.fI = 0.f;
  r.Ih = r.Il = 0.f;
  if (kVol && ip.volumetric) {
    r.fI = vol_source32(ip, mf, r.Ef, r.ellf, r.yh[1], dtheta_eq(r.yh[2], r.yl[2], 0.f));
    r.h = layer_cap(ip.vf[0], ip.vf[1], r.yh[1], r.yh[2], r.f[1], r.f[2], r.h);
  }
  r.lh = r.ll = 0.f;
  r.cs.lam_last = 0.0;
  r.cs.have_trusted = false;
  r.cs.ncross = 0;
  r.cs.I[0] = r.cs.I[1] = r.cs.I[2] = r.cs.I[3] = 0.0;
  r.rejected = false;
  r.nacc = r.nrej = r.steps = 0;
  r.hdrift = 0.f;
}

// Crossing inside an accepted FP32 step: the rule of handle_crossing with an
// FP32 root of theta - pi/2 on the dense output and FP32 transfer maps,
// redshift and emissivity (Eqs. 82-91); the affine parameter of the trusted
// gap test and the intensity sums stay in FP64.
static __device__ __noinline__ void cross_f32(const ImgParams& ip, const MetricConsts<float>& m,
                                             float Ef, float ellf, const float* y0h,
                                             const float* y0l, const float* y1h,
                                             const float* y1l, const float* hf0,
                                             const float* hf1, const float* hd, double lam,
                                             float h, CrossState& cs, const CrossOut& co) {
  constexpr float kHPh = 1.57079637050628662109375f, kHPl = -4.37113900018624283e-8f;
  // dense output of one component relative to an offset (hi, lo) pair
  auto dense = [&](int i, float sig, float off_h, float off_l) {
    const float y0 = __fadd_rn(__fsub_rn(y0h[i], off_h), __fsub_rn(y0l[i], off_l));
    const float r2 = __fadd_rn(__fsub_rn(y1h[i], y0h[i]), __fsub_rn(y1l[i], y0l[i]));
    const float r3 = hf0[i] - r2, r4 = r2 - hf1[i] - r3;
    return y0 + sig * (r2 + (1.f - sig) * (r3 + sig * (r4 + (1.f - sig) * hd[i])));
  };
  const float s0 = dense(2, 0.f, kHPh, kHPl), s1 = dense(2, 1.f, kHPh, kHPl);
  float sig = 1.f;
  if (s1 != 0.f) {
    float x0 = 0.f, f0 = s0, x1 = 1.f, f1 = s1;
    for (int it = 0; it < 60; ++it) {
      float x2 = x1 - __fdividef(f1 * (x1 - x0), f1 - f0);
      if (!(x2 > fminf(x0, x1) && x2 < fmaxf(x0, x1))) x2 = 0.5f * (x0 + x1);
      const float f2 = dense(2, x2, kHPh, kHPl);
      if (f2 == 0.f) {
        x1 = x2;
        break;
      }
      if ((f2 > 0.f) != (f1 > 0.f)) {
        x0 = x1;
        f0 = f1;
      } else {
        f0 *= 0.5f;
      }
      x1 = x2;
      f1 = f2;
      if (fabsf(x1 - x0) <= 1e-7f || fabsf(f2) <= 1e-8f) break;
    }
    sig = x1;
  }
  const float Rc = dense(1, sig, 0.f, 0.f);
  const float pth = dense(5, sig, 0.f, 0.f);
  const float thdot = __fdividef(pth, Rc * Rc);  // Eq. (60) on the plane (cos theta = 0)
  const double lamc = lam + (double)(sig * h);
  if (!(Rc >= (float)ip.R_cap && Rc <= (float)ip.R_esc && fabsf(thdot) >= (float)ip.thdot_min &&
        (!cs.have_trusted || lamc - cs.lam_last >= ip.dlam_min)))
    return;
  const int n = cs.ncross;
  float g = 0.f, j = 0.f;
  if (emitter_g_f(m, Rc, Ef, ellf, g)) {
    // Eqs. (83)-(86) at z = 0 in log space, tapers as logistic functions
    const float* v = ip.vf;  // H0, hh, R_in, 1/sig_in, 1/sig_out, R_out, p, 1/R_s, j0, 1/R_in
    const float tin = logistic_neg_f(-2.f * (Rc - v[2]) * v[3]);
    const float tout = logistic_neg_f(2.f * (Rc - v[5]) * v[4]);
    j = v[8] * __expf(-v[6] * __logf(Rc * v[9]) - (Rc - v[2]) * v[7]) * tin * tout;
  }
  // the volumetric mode adds no event intensity (its integral is a state)
  const float In = ip.volumetric ? 0.f : g * g * g * j;
  cs.I[0] += (double)In;
  if (n < 3) {
    cs.I[1 + n] = (double)In;
    // phi reduced to [0, 2 pi) by a two-part 2 pi (no slow-path fmodf)
    const float phi = dense(3, sig, 0.f, 0.f);
    const float qn = floorf(phi * 0.159154943f);
    float ph = fmaf(-qn, 6.28318548f, phi);
    ph = fmaf(-qn, -1.74845553e-7f, ph);
    if (ph < 0.f) ph += 6.28318530717958647692f;
    if (ph >= 6.28318530717958647692f) ph -= 6.28318530717958647692f;
    if (co.pix >= 0) {
      const int64_t o = n * co.stride + co.pix;
      if (co.R_em) co.R_em[o] = Rc;
      if (co.phi_em) co.phi_em[o] = ph;
      if (co.T_em) co.T_em[o] = dense(0, sig, 0.f, 0.f);
      if (co.g) co.g[o] = g;
    }
    if (co.rec) {
      co.rec->R_em[n] = Rc;
      co.rec->phi_em[n] = ph;
      co.rec->T_em[n] = dense(0, sig, 0.f, 0.f);
      co.rec->g[n] = g;
    }
  }
  cs.ncross = n + 1;
  cs.lam_last = lamc;
  cs.have_trusted = true;
}

// One attempted FP32 step.  Returns 0 (continue), terminal status + 1, or 4
// when the ray must be promoted to FP64.  kVol builds in the volumetric
// intensity as a seventh component (Eq. 88; see ray_step64).
template <bool kVol>
__device__ __forceinline__ int ray_step_mx(const ImgParams& ip, const MetricConsts<float>& mf,
                                           const MxConsts& c,
                                           RayMx& r, const TraceArgs& a, int64_t item,
                                           uint32_t img, bool may_promote) {
  const float h = r.h;
  // k: the latest stage derivative; q[u]: running input sums of the next
  // stages; s5, se, sd: running sums of the update, the error estimate and
  // the dense-output term (see DPRolled).  r.f keeps k_0 until the end.
  // stage-input sums only for R, theta, p_R, p_theta (kQC): T and phi are
  // cyclic and never enter the right-hand side
  float k[6], q[6][4], s5[6], se[6], sd[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    k[i] = r.f[i];
    s5[i] = se[i] = sd[i] = 0.f;
  }
#pragma unroll
  for (int u = 0; u < 6; ++u)
#pragma unroll
    for (int x = 0; x < 4; ++x) q[u][x] = 0.f;
  bool bad = false;
  float W = 0.f, P2oD = 1.f;
  const bool vol = kVol && ip.volumetric;
  float kI = kVol ? r.fI : 0.f, s5I = 0.f, seI = 0.f;
  const RayC<float> kc = ray_consts(mf, r.Ef, r.ellf);
#pragma unroll 1
  for (int j = 0; j < 7; ++j) {
    // all coefficients, zeros included: branching around the zero terms
    // (as the FP64 step does) costs the issue-bound FP32 loop more than the
    // FMAs it saves
    const float bj = kDPrf.b[j], ej = kDPrf.e[j], dj = kDPrf.d[j];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      s5[i] = fmaf(bj, k[i], s5[i]);
      se[i] = fmaf(ej, k[i], se[i]);
      sd[i] = fmaf(dj, k[i], sd[i]);
    }
    if (kVol) {
      s5I = fmaf(bj, kI, s5I);
      seI = fmaf(ej, kI, seI);
    }
    if (j == 6) break;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const float c = kDPrf.q[j][u];
#pragma unroll
      for (int x = 0; x < 4; ++x) q[u][x] = fmaf(c, k[kQC(x)], q[u][x]);
    }
    float ys[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) ys[x] = r.yh[kQC(x)] + (r.yl[kQC(x)] + h * q[0][x]);
    // sin and cos of theta from the pair (state hi, state lo + stage offset)
    float sth, cth;
    d_sincos2(r.yh[2], r.yl[2] + h * q[0][1], &sth, &cth);
    bool ok = geo_rhs_sc(mf, kc, ys[0], sth, cth, ys[2], ys[3], k, W, P2oD);
    bad |= !ok;
    // the source depends on the state only, so its stage-input sum is not needed
    if (vol)
      kI = vol_source32(ip, mf, r.Ef, r.ellf, ys[0], dtheta_eq(r.yh[2], r.yl[2], h * q[0][1]));
#pragma unroll
    for (int u = 0; u < 5; ++u) {
#pragma unroll
      for (int x = 0; x < 4; ++x) q[u][x] = q[u + 1][x];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) q[5][x] = 0.f;
  }
  float dlt[6], err2 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    dlt[i] = h * s5[i];
    float sc = c.atol + c.rtol * fmaxf(fabsf(r.yh[i]), fabsf(r.yh[i] + dlt[i]));
    float qe = __fdividef(h * se[i], sc);
    err2 += qe * qe;
  }
  const float dI = h * s5I;
  if (vol) {
    const float sc = c.atol + c.rtol * fmaxf(fabsf(r.Ih), fabsf(r.Ih + dI));
    const float qe = __fdividef(h * seI, sc);
    err2 += qe * qe;
  }
  float err = sqrtf(vol ? err2 / 7.f : err2 / 6.f);
  r.steps++;
  if (bad || !(err <= 1.f)) {
    r.h = bad ? 0.5f * h : h * step_factor_mx(err, true);
    r.rejected = true;
    r.nrej++;
    return r.steps >= ip.max_steps ? 3 : 0;
  }
  r.nacc++;
  float nh[6], nl[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    nh[i] = r.yh[i];
    nl[i] = r.yl[i];
    df_add(nh[i], nl[i], dlt[i]);
  }
  {
    // sign of theta - pi/2 before and after, from the float pairs
    float s0 = __fadd_rn(__fsub_rn(r.yh[2], kHalfPiHi), __fsub_rn(r.yl[2], kHalfPiLo));
    float s1 = __fadd_rn(__fsub_rn(nh[2], kHalfPiHi), __fsub_rn(nl[2], kHalfPiLo));
    if ((s0 > 0.f && s1 <= 0.f) || (s0 < 0.f && s1 >= 0.f)) {
      float y0h[6], y0l[6], hf0[6], hf1[6], hd[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        y0h[i] = r.yh[i];
        y0l[i] = r.yl[i];
        hd[i] = h * sd[i];
        hf0[i] = h * r.f[i];
        hf1[i] = h * k[i];
      }
      CrossState cs = r.cs;  // copies keep the ray state in registers
      const CrossOut co = cross_out(a, item, img);
      cross_f32(ip, mf, r.Ef, r.ellf, y0h, y0l, nh, nl, hf0, hf1, hd, df_to(r.lh, r.ll), h, cs,
                co);
      r.cs = cs;
    }
  }
  df_add(r.lh, r.ll, h);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    r.yh[i] = nh[i];
    r.yl[i] = nl[i];
    r.f[i] = k[i];
  }
  if (vol) {
    df_add(r.Ih, r.Il, dI);
    r.fI = kI;
  }
  // polar axis (see reflect_axis): theta -> -theta or 2 pi - theta,
  // p_th -> -p_th, phi -> phi + pi
  if (r.yh[2] < 0.f || r.yh[2] > kPiHi) {
    double th = df_to(r.yh[2], r.yl[2]);
    double pth = df_to(r.yh[5], r.yl[5]);
    double ph = df_to(r.yh[3], r.yl[3]);
    if (reflect_axis(th, pth, ph)) {
      df_from(th, r.yh[2], r.yl[2]);
      df_from(pth, r.yh[5], r.yl[5]);
      df_from(ph, r.yh[3], r.yl[3]);
      rhs_f32_into(mf, r.Ef, r.ellf, r.yh[1], r.yh[2], r.yl[2], r.yh[4], r.yh[5], r.f);
      if (vol)
        r.fI = vol_source32(ip, mf, r.Ef, r.ellf, r.yh[1], dtheta_eq(r.yh[2], r.yl[2], 0.f));
    }
  }
  float hdv = __fdividef(fabsf(W), P2oD);
  if (hdv > r.hdrift) r.hdrift = hdv;
  const float R = r.yh[1];
  if (R < c.R_cap) return 2;
  if (R > c.R_esc) return 1;
  r.h = h * step_factor_mx(err, r.rejected);
  r.rejected = false;
  if (vol) r.h = layer_cap(ip.vf[0], ip.vf[1], r.yh[1], r.yh[2], r.f[1], r.f[2], r.h);
  // image order n = N_cross - 1 (Sec. 4.2): rays winding to n >= promote_order
  // are promoted
  if (may_promote && (R < c.promote_R || (r.cs.ncross >= c.promote_nc && R < c.demote_R)))
    return 4;
  // radial turning points of near-critical rays
  if (may_promote && c.kappa > 0.f && R < c.demote_R &&
      near_double_root(mf, r.Ef, r.ellf, R, r.yh[2], r.yh[4], r.yh[5], c.kappa))
    return 4;
  return r.steps >= ip.max_steps ? 3 : 0;
}

// MinBlocks = 0 leaves the register count to the compiler (3 blocks of 128
// threads per SM); MinBlocks = 4 caps it at 128 registers for 4 blocks at a
// small spill cost.  The autotuner picks between them.  Vol builds in the
// volumetric intensity; the thin-disk builds carry none of its registers.
template <int MinBlocks, bool Vol>
__global__ void __launch_bounds__(128, MinBlocks) trace_mixed_kernel(TraceArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n_items = pass_items(a);
  const unsigned long long budget = a.hdr->budget_ns;
  const unsigned long long t0 = a.hdr->t_start;
  const bool may_promote = a.allow_spill != 0;

  RayMx r;
  MetricConsts<float> mf;
  MxConsts c;
  const ImgParams* ip = a.ip;
  int64_t item = -1;
  uint32_t img = 0;
  bool active = false, drained = false;
  unsigned iter = 0;
  unsigned long long w_max = 0, w_iters = 0, w_lanes = 0;
  unsigned long long w_acc = 0, w_rej = 0, w_rays = 0, w_promo = 0, w_full = 0;

  const int pass = (a.source ? 2 : 0);
  if (lane == 0) mark_first(&a.hdr->t_pass[0][pass][a.level]);
  while (true) {
    const bool need = refill_now<kMxRefillLanes>(!active && !drained, active);
    int64_t idx = claim(a.head, need, lane);
    if (need) {
      if (idx < n_items) {
        if (a.source == 1) {
          const SpillRec& s = a.spill_in[idx];
          item = s.item;
          img = s.img;
          ip = &a.ip[img];
          mf = metric_consts<float>(*ip);
          mx_resume<Vol>(*ip, s, mf, r);
        } else {
          double X, Y;
          int64_t pix;
          item = idx;
          resolve_item(a, idx, img, pix, X, Y);
          ip = &a.ip[img];
          mf = metric_consts<float>(*ip);
          c.rtol = (float)fmax(ip->rtol, 1e-9);  // FP32 noise floor of the estimate
          c.atol = (float)ip->atol;
          ray_init_mx<Vol>(*ip, mf, c, X, Y, r);
        }
        c.rtol = (float)fmax(ip->rtol, 1e-9);  // FP32 noise floor of the estimate
        c.atol = (float)ip->atol;
        c.R_cap = (float)ip->R_cap;
        c.R_esc = (float)ip->R_esc;
        c.promote_R = (float)ip->promote_R;
        c.demote_R = (float)ip->demote_R;
        c.promote_nc = ip->promote_ncross;
        c.kappa = (float)ip->kappa;
        active = true;
      } else {
        drained = true;
        mark_first(&a.hdr->t_pass[1][pass][a.level]);
      }
    }
    const unsigned am = __ballot_sync(kFull, active);
    if (am == 0) {
      if (__ballot_sync(kFull, !drained) == 0) break;
      continue;
    }
    w_iters += 1ull;
    w_lanes += (unsigned long long)__popc(am);
    if (active) {
      const int acc0 = r.nacc, rej0 = r.nrej;
      int term = ray_step_mx<Vol>(*ip, mf, c, r, a, item, img, may_promote);
      // the volumetric integral rides in the float pair until hand-off
      if (Vol && term && ip->volumetric) r.cs.I[0] = df_to(r.Ih, r.Il);
      w_acc += (unsigned long long)(r.nacc - acc0);
      w_rej += (unsigned long long)(r.nrej - rej0);
      if (term == 4) {
        unsigned long long slot = atomicAdd(a.spill_out_count, 1ull);
        if (slot < (unsigned long long)a.spill_cap) {
          mx_spill(r, item, img, a.spill_out[slot]);
          active = false;
          w_promo += 1ull;
        } else {
          w_full += 1ull;  // queue full: this ray stays in FP32
        }
      } else if (term) {
        finish_ray(a, item, img, term - 1, r.cs, r.hdrift, r.nacc, r.nrej, r.E, r.ell,
                   df_to(r.lh, r.ll));
        w_rays += 1ull;
        w_max = (unsigned long long)r.steps > w_max ? (unsigned long long)r.steps : w_max;
        active = false;
      }
    }
    if (budget && ((++iter & 255u) == 0u)) {
      unsigned long long now = __shfl_sync(kFull, globaltimer(), 0);
      if (now - t0 > budget) {
        if (lane == 0) atomicCAS(&a.hdr->status, 0, (int)BH_ERR_TIMEOUT);
        break;
      }
    }
  }
  flush_tally(&a.hdr->accepted32, w_acc, lane);
  flush_tally(&a.hdr->rejected32, w_rej, lane);
  flush_tally(&a.hdr->rays[a.level], w_rays, lane);
  if (lane == 0) {
    atomicMax(&a.hdr->t_pass[2][pass][a.level], globaltimer());
    atomicAdd(&a.hdr->warp_iters[0], w_iters);
    atomicAdd(&a.hdr->lane_iters[0], w_lanes);
  }
  if (w_max) atomicMax(&a.hdr->max_ray_steps, w_max);
  flush_tally(&a.hdr->promoted_rays, w_promo, lane);
  flush_tally(&a.hdr->spill_full, w_full, lane);
}

cudaError_t launch_trace_mixed(const TraceArgs& a, LaunchShape s, cudaStream_t st) {
  if (a.any_volumetric) {
    if (s.variant == 1)
      trace_mixed_kernel<4, true><<<s.blocks, s.threads, 0, st>>>(a);
    else
      trace_mixed_kernel<0, true><<<s.blocks, s.threads, 0, st>>>(a);
  } else if (s.variant == 1) {
    trace_mixed_kernel<4, false><<<s.blocks, s.threads, 0, st>>>(a);
  } else {
    trace_mixed_kernel<0, false><<<s.blocks, s.threads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

int trace_default_blocks_per_sm(int precision, int threads, int variant) {
  int nb = 0;
  if (precision == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_fp64_kernel_ptr(variant), threads, 0);
  else if (variant == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_mixed_kernel<4, false>, threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_mixed_kernel<0, false>, threads, 0);
  return nb > 0 ? nb : 1;
}

}  // namespace bhrt
