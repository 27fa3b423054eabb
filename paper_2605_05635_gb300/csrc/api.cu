// api.cu -- the C ABI: argument validation, host-side geometry (horizon,
// extremal spin, ISCO, ZAMO frame), workspace layout and the launch
// sequence of one tracing call.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "adjoint.h"
#include "dual.cuh"
#include "internal.h"

using namespace bhrt;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxPrecision = 1;
// Mixed path: a promoted ray returns to FP32 once it is outgoing beyond this
// radius, and winding rays are promoted only inside it (reading: outside the
// photon region, whose outermost circular orbit, the retrograde equatorial
// one, lies within 4 M for Kerr spins up to 1 and moves by a few percent
// with the halos of the imaging configurations).
constexpr double kDemoteR = 5.0;

// ---------------------------------------------------------------- geometry
struct HostMetric {
  int metric;
  double chi, lamE, eta, lamc;
};

// Lapse H(R) and H'(R): Kerr 1 - 2/R, Einasto Eq. (9), cored-NFW Eq. (13).
void host_lapse(const HostMetric& m, double R, double& H, double& dH) {
  if (m.metric == BH_EINASTO) {
    double l = m.lamE, e = std::exp(-R / l);
    double poly = 2.0 / R + 2.0 / l + R / (l * l);
    H = 1.0 - 2.0 / R + poly * e;
    dH = 2.0 / (R * R) + (-2.0 / (R * R) + 1.0 / (l * l) - poly / l) * e;
  } else if (m.metric == BH_CNFW) {
    double lc = m.lamc, L = std::log1p(R / lc), q = 1.0 / (R + lc);
    double S = m.eta * lc * (q - 2.0 * L / R);
    double dS = m.eta * lc * (-q * q + 2.0 * L / (R * R) - 2.0 * q / R);
    double eS = std::exp(S);
    H = eS - 2.0 / R;
    dH = eS * dS + 2.0 / (R * R);
  } else {
    H = 1.0 - 2.0 / R;
    dH = 2.0 / (R * R);
  }
}

double host_delta(const HostMetric& m, double R) {
  double H, dH;
  host_lapse(m, R, H, dH);
  return R * R * H + m.chi * m.chi;
}

// Outer horizon (Eq. 33).  Kerr: 1 + sqrt(1 - chi^2).  Otherwise the first
// sign change of Delta met when walking inward from R = 64 on a geometric
// grid (ratio 1 - 2^-10), refined by bisection to the last bit.
bool host_horizon(const HostMetric& m, double& rp) {
  if (m.metric == BH_KERR || (m.metric == BH_CNFW && m.eta == 0.0)) {
    double d = 1.0 - m.chi * m.chi;
    if (d < 0.0) return false;
    rp = 1.0 + std::sqrt(d);
    return true;
  }
  double hi = 64.0;
  if (!(host_delta(m, hi) > 0.0)) return false;
  const double ratio = 1.0 - 1.0 / 1024.0;
  for (int k = 0; k < 40000; ++k) {
    double lo = hi * ratio;
    if (lo < 1e-6) return false;
    if (!(host_delta(m, lo) > 0.0)) {
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (host_delta(m, mid) > 0.0) hi = mid; else lo = mid;
      }
      rp = hi;
      return true;
    }
    hi = lo;
  }
  return false;
}

// Extremal spin (Eqs. 36-37): chi_e^2 = max_R [-R^2 H(R)].
double host_extremal_spin(const HostMetric& m0) {
  HostMetric m = m0;
  m.chi = 0.0;
  double best = -1e300, Rb = 1.0;
  for (int k = 0; k <= 20000; ++k) {
    double R = 1e-3 * std::pow(10.0, 4.7 * k / 20000.0);
    double H, dH;
    host_lapse(m, R, H, dH);
    double v = -R * R * H;
    if (v > best) { best = v; Rb = R; }
  }
  double a = Rb * 0.999, b = Rb * 1.001;
  for (int it = 0; it < 200; ++it) {
    double x1 = a + 0.381966011250105 * (b - a), x2 = b - 0.381966011250105 * (b - a);
    double H1, H2, d;
    host_lapse(m, x1, H1, d);
    host_lapse(m, x2, H2, d);
    if (-x1 * x1 * H1 > -x2 * x2 * H2) b = x2; else a = x1;
  }
  double R = 0.5 * (a + b), H, dH;
  host_lapse(m, R, H, dH);
  double v = -R * R * H;
  return v > 0 ? std::sqrt(v) : 0.0;
}

// Prograde circular equatorial orbit (Eqs. 90-91) -> specific energy.
bool host_circular_energy(const HostMetric& m, double R, double& E) {
  double H, dH;
  host_lapse(m, R, H, dH);
  double x2 = m.chi * m.chi;
  double den = 2.0 * R - x2 * dH, disc = 2.0 * R * dH;
  if (!(disc >= 0.0) || den == 0.0) return false;
  double W = (-m.chi * dH + std::sqrt(disc)) / den;
  double gtt = -H, gtp = -m.chi * (1.0 - H), gpp = R * R + x2 + x2 * (1.0 - H);
  double norm = -(gtt + 2.0 * W * gtp + W * W * gpp);
  if (!(norm > 0.0)) return false;
  E = -(gtt + W * gtp) / std::sqrt(norm);
  return true;
}

// r_ISCO: Kerr from Bardeen, Press & Teukolsky (1972); otherwise the
// minimiser of the circular-orbit energy (coarse scan + golden section).
bool host_isco(const HostMetric& m, double rp, double& risco) {
  if (m.metric == BH_KERR || (m.metric == BH_CNFW && m.eta == 0.0)) {
    double a = m.chi;
    double z1 = 1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
    double z2 = std::sqrt(3.0 * a * a + z1 * z1);
    double s = (a >= 0) ? 1.0 : -1.0;
    risco = 3.0 + z2 - s * std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
    return true;
  }
  double best = 1e300, Rb = -1;
  for (int k = 1; k <= 12000; ++k) {
    double R = rp + 5e-3 * k;
    double E;
    if (host_circular_energy(m, R, E) && E < best) { best = E; Rb = R; }
  }
  if (Rb < 0) return false;
  double a = Rb - 5e-3, b = Rb + 5e-3;
  for (int it = 0; it < 200; ++it) {
    double x1 = a + 0.381966011250105 * (b - a), x2 = b - 0.381966011250105 * (b - a);
    double e1 = 1e300, e2 = 1e300;
    host_circular_energy(m, x1, e1);
    host_circular_energy(m, x2, e2);
    if (e1 < e2) b = x2; else a = x1;
  }
  risco = 0.5 * (a + b);
  return true;
}

HostMetric to_metric(const bh_spacetime& s) {
  return HostMetric{s.metric, s.chi, s.lambda_E, s.eta, s.lambda_c};
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bh_status validate(const bh_spacetime& s, const bh_camera& c, const bh_emission& e,
                   const bh_integrator& g) {
  if (s.metric < 0 || s.metric > 2 || s.reserved != 0 || !std::isfinite(s.chi))
    return BH_ERR_INVALID_ARG;
  if (s.metric == BH_EINASTO && !finite_pos(s.lambda_E)) return BH_ERR_INVALID_ARG;
  if (s.metric == BH_CNFW && (!finite_pos(s.lambda_c) || !(s.eta >= 0.0) || !std::isfinite(s.eta)))
    return BH_ERR_INVALID_ARG;
  if (!finite_pos(c.r_obs) || !(c.incl > 0.0 && c.incl < kPi) || c.reserved != 0)
    return BH_ERR_INVALID_ARG;
  if (!(c.x_max > c.x_min) || !(c.y_max > c.y_min) || !std::isfinite(c.x_min) ||
      !std::isfinite(c.x_max) || !std::isfinite(c.y_min) || !std::isfinite(c.y_max))
    return BH_ERR_INVALID_ARG;
  if (c.nx < 1 || c.ny < 1 || c.nx > 16384 || c.ny > 16384) return BH_ERR_INVALID_ARG;
  if (c.refine_levels < 0 || c.refine_levels > kMaxLevels || c.refine_capacity < 0)
    return BH_ERR_INVALID_ARG;
  if ((int64_t)c.nx * c.ny > (int64_t(1) << 40)) return BH_ERR_INVALID_ARG;
  if (e.r_in_mode < 0 || e.r_in_mode > 1 || e.volumetric < 0 || e.volumetric > 1)
    return BH_ERR_INVALID_ARG;
  if (e.volumetric && !(finite_pos(e.H0) && e.h >= 0.0 && std::isfinite(e.h)))
    return BH_ERR_INVALID_ARG;
  if (!finite_pos(e.R_s) || !finite_pos(e.sigma_in) || !finite_pos(e.sigma_out) ||
      !std::isfinite(e.j0) || !std::isfinite(e.p) || !std::isfinite(e.R_out))
    return BH_ERR_INVALID_ARG;
  if (e.r_in_mode == 1 && !(e.dR_in >= 0.0)) return BH_ERR_INVALID_ARG;
  if (g.precision < 0 || g.precision > kMaxPrecision || g.max_steps < 1) return BH_ERR_INVALID_ARG;
  if (!finite_pos(g.rtol) || !finite_pos(g.atol) || !(g.cap_factor >= 1.0) ||
      !(g.esc_factor > 1.0) || !(g.thetadot_min >= 0.0) || !(g.dlambda_min >= 0.0) ||
      !(g.promote_dr >= 0.0) || !(g.time_budget_s >= 0.0) || g.promote_order < 0 ||
      g.promote_order > 1000 || g.reserved != 0 ||
      !(g.promote_turning >= 0.0 && g.promote_turning <= 1.0))
    return BH_ERR_INVALID_ARG;
  return BH_OK;
}

// Per-image device constants.
bh_status make_params(const bh_spacetime& s, const bh_camera& c, const bh_emission& e,
                      const bh_integrator& g, ImgParams& ip) {
  bh_status v = validate(s, c, e, g);
  if (v != BH_OK) return v;
  HostMetric m = to_metric(s);
  double rp;
  if (!host_horizon(m, rp)) return BH_ERR_NO_HORIZON;
  if (c.r_obs <= 10.0 * rp) return BH_ERR_OBSERVER_INSIDE;
  double R_in;
  if (e.r_in_mode == 0) {
    if (!host_isco(m, rp, R_in)) return BH_ERR_NO_ISCO;
  } else {
    R_in = rp + e.dR_in;  // Eq. (87)
  }
  std::memset(&ip, 0, sizeof(ip));
  ip.metric = s.metric;
  ip.max_steps = g.max_steps;
  ip.nx = c.nx;
  ip.ny = c.ny;
  ip.chi = s.chi;
  ip.lamE = s.lambda_E;
  ip.eta = s.eta;
  ip.lamc = s.lambda_c;
  ip.r_obs = c.r_obs;
  ip.incl = c.incl;
  ip.x_min = c.x_min;
  ip.y_min = c.y_min;
  ip.dx = (c.x_max - c.x_min) / c.nx;
  ip.dy = (c.y_max - c.y_min) / c.ny;
  // ZAMO frame at the observer (Eqs. 63-68) from the metric of Eqs. (27)-(31).
  {
    double R = c.r_obs, th = c.incl, H, dH;
    host_lapse(m, R, H, dH);
    double x2 = s.chi * s.chi, cs = std::cos(th), sn = std::sin(th), s2 = sn * sn;
    double Sig = R * R + x2 * cs * cs, F = R * R * (1.0 - H), D = R * R * H + x2;
    double gtt = -(1.0 - F / Sig), gtp = -s.chi * F * s2 / Sig;
    double grr = Sig / D, gthth = Sig, gpp = s2 * (R * R + x2 + x2 * F * s2 / Sig);
    double w = -gtp / gpp;
    double N = std::sqrt(-(gtt + 2.0 * w * gtp + w * w * gpp));
    ip.zamo_w = w;
    ip.zamo_N = N;
    ip.sq_grr = std::sqrt(grr);
    ip.sq_gth = std::sqrt(gthth);
    ip.sq_gph = std::sqrt(gpp);
  }
  ip.r_plus = rp;
  ip.R_cap = g.cap_factor * rp;
  ip.R_esc = g.esc_factor * c.r_obs;
  ip.R_in = R_in;
  ip.j0 = e.j0;
  ip.p = e.p;
  ip.R_s = e.R_s;
  ip.sig_in = e.sigma_in;
  ip.sig_out = e.sigma_out;
  ip.R_out = e.R_out;
  ip.H0 = e.H0;
  ip.hh = e.h;
  ip.volumetric = e.volumetric;
  ip.isig_in = 1.0 / e.sigma_in;
  ip.isig_out = 1.0 / e.sigma_out;
  ip.iR_s = 1.0 / e.R_s;
  ip.iR_in = 1.0 / ip.R_in;
  const double vf[10] = {e.H0, e.h, ip.R_in, ip.isig_in, ip.isig_out, e.R_out, e.p, ip.iR_s,
                         e.j0, ip.iR_in};
  for (int k = 0; k < 10; ++k) ip.vf[k] = (float)vf[k];
  ip.rtol = g.rtol;
  ip.atol = g.atol;
  ip.thdot_min = g.thetadot_min;
  ip.dlam_min = g.dlambda_min;
  ip.promote_R = rp + g.promote_dr;
  ip.demote_R = kDemoteR;
  ip.promote_ncross = g.promote_order + 1;
  ip.kappa = g.promote_turning;
  ip.sin_o = std::sin(c.incl);
  ip.isin_o = 1.0 / ip.sin_o;
  ip.md = make_metric_consts<double>(ip);
  ip.mf = make_metric_consts<float>(ip);
  return BH_OK;
}

// ---------------------------------------------------------------- workspace
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t hdr, ip, out, base_I, base_cls, base_child, base_depth, spill[2];
  int64_t spill_cap;
  size_t lv_key[kMaxLevels + 1], lv_img[kMaxLevels + 1], lv_I[kMaxLevels + 1],
      lv_cls[kMaxLevels + 1], lv_child[kMaxLevels + 1], lv_depth[kMaxLevels + 1];
  size_t total;
};

struct Caps {
  int64_t c[kMaxLevels + 1];  // cells per refinement level (index 1..3)
};

Layout make_layout(int n, int64_t npix, int levels, const Caps& caps, int precision) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  int64_t nb = (int64_t)n * npix;
  L.hdr = take(sizeof(WsHeader));
  L.ip = take(sizeof(ImgParams) * n);
  L.out = take(sizeof(OutPtrs) * n);
  L.base_I = take(sizeof(double) * 4 * nb);
  L.base_cls = take(sizeof(uint16_t) * nb);
  L.base_child = take(sizeof(int32_t) * nb);
  L.base_depth = take(nb);
  int64_t maxcap = nb;
  for (int l = 1; l <= levels; ++l) {
    const int64_t cap = caps.c[l];
    L.lv_key[l] = take(sizeof(uint64_t) * cap);
    L.lv_img[l] = take(sizeof(uint32_t) * cap);
    L.lv_I[l] = take(sizeof(double) * 4 * cap);
    L.lv_cls[l] = take(sizeof(uint16_t) * cap);
    L.lv_child[l] = take(sizeof(int32_t) * cap);
    L.lv_depth[l] = take(cap);
    if (cap > maxcap) maxcap = cap;
  }
  L.spill_cap = 0;
  L.spill[0] = L.spill[1] = 0;
  if (precision == 1) {
    L.spill_cap = maxcap;
    L.spill[0] = take(spill_record_bytes() * L.spill_cap);
    L.spill[1] = take(spill_record_bytes() * L.spill_cap);
  }
  L.total = o;
  return L;
}

// Cells per refinement level.  A caller-given capacity applies to every
// level; otherwise level L holds min(16^L, max(f_L, 2^22 / (n nx ny))) cells
// per base pixel with f = 4, 12, 24: room for 25 % of the base pixels to be
// refined and the boundary to keep growing x3 and x2 per level, and for
// every cell of a coarse screen to be refined.
Caps default_caps(int n, const bh_camera& c) {
  Caps k{};
  const int64_t nb = (int64_t)c.nx * c.ny * n;
  const int64_t f[kMaxLevels + 1] = {0, 4, 12, 24};
  int64_t full = nb;
  for (int l = 1; l <= kMaxLevels; ++l) {
    full = full > (int64_t(1) << 40) ? full : full * 16;
    int64_t cap;
    if (c.refine_capacity > 0) {
      cap = c.refine_capacity;
    } else {
      cap = f[l] * nb;
      if (cap < (int64_t(1) << 22)) cap = int64_t(1) << 22;
      if (cap > full) cap = full;
    }
    cap = (cap + 15) & ~int64_t(15);
    if (cap > (int64_t(1) << 30)) cap = int64_t(1) << 30;  // int32 child indices
    k.c[l] = cap;
  }
  return k;
}

}  // namespace

int bhrt::num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ------------------------------------------------------------------- plan
struct bh_plan_s {
  int n = 0, levels = 0, precision = 0;
  int64_t npix = 0;
  Caps caps{};
  std::vector<ImgParams> ip;
  std::vector<OutPtrs> out;
  char* ws = nullptr;
  Layout L{};
  unsigned long long budget_ns = 0;
  LaunchShape shape{0, 128};    // main trace kernel (FP64 or FP32 bulk)
  LaunchShape shape64{0, 128};  // FP64 promoted pass of the mixed path
  int refine_blocks = 0;
  bool any_keys = false;
  bool any_vol = false;   // some image integrates the volumetric intensity
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  bool timing = false;                       // events around the trace launches
  cudaEvent_t ev[2 * 3 * (kMaxLevels + 1)] = {};  // per level, per pass
  int launches = 0;                          // kernels per enqueue
};

namespace {

int count_launches(const bh_plan_s& p) {
  const int passes = p.precision == 1 ? 3 : 1;
  int k = 1 + passes * (1 + p.levels) + p.levels + (p.levels > 0 ? p.levels : 1);
  if (p.any_keys && p.levels > 0) ++k;
  return k;
}

bh_status plan_build(int32_t n, const bh_spacetime* st, const bh_camera* cam,
                     const bh_emission* em, const bh_integrator* integ, const bh_image_out* out,
                     void* ws, size_t ws_bytes, bh_plan_s& p) {
  if (n < 1 || !st || !cam || !em || !integ || !out) return BH_ERR_INVALID_ARG;
  for (int i = 1; i < n; ++i)
    if (cam[i].nx != cam[0].nx || cam[i].ny != cam[0].ny ||
        cam[i].refine_levels != cam[0].refine_levels || integ[i].precision != integ[0].precision)
      return BH_ERR_INVALID_ARG;
  p.n = n;
  p.levels = cam[0].refine_levels;
  p.precision = integ[0].precision;
  p.npix = (int64_t)cam[0].nx * cam[0].ny;
  p.caps = default_caps(n, cam[0]);
  p.ip.resize(n);
  p.out.resize(n);
  double budget = 0.0;
  for (int i = 0; i < n; ++i) {
    bh_status s = make_params(st[i], cam[i], em[i], integ[i], p.ip[i]);
    if (s != BH_OK) return s;
    const bh_image_out& o = out[i];
    if (!o.I || !o.ncross || !o.status) return BH_ERR_INVALID_ARG;
    if (o.refine_keys && o.refine_keys_cap < 0) return BH_ERR_INVALID_ARG;
    OutPtrs& d = p.out[i];
    d.I = o.I;
    d.I_n = o.I_n;
    d.ncross = o.ncross;
    d.status = o.status;
    d.refine_level = o.refine_level;
    d.R_em = o.R_em;
    d.phi_em = o.phi_em;
    d.T_em = o.T_em;
    d.g = o.g;
    d.h_drift = o.h_drift;
    d.keys = o.refine_keys;
    d.keys_cap = o.refine_keys ? o.refine_keys_cap : 0;
    d.keys_count = reinterpret_cast<unsigned long long*>(o.refine_keys_count);
    d.steps = o.steps;
    d.promoted = o.promoted;
    if (d.keys_count) p.any_keys = true;
    if (em[i].volumetric) p.any_vol = true;
    if (integ[i].time_budget_s > budget) budget = integ[i].time_budget_s;
  }
  p.budget_ns = (unsigned long long)(budget * 1e9);
  p.L = make_layout(n, p.npix, p.levels, p.caps, p.precision);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < p.L.total)
    return BH_ERR_WORKSPACE;
  p.ws = static_cast<char*>(ws);
  const int sms = num_sms();
  const int threads = 128;
  p.shape.threads = threads;
  p.shape.blocks = sms * trace_default_blocks_per_sm(p.precision, threads);
  p.shape64.threads = threads;
  p.shape64.blocks = sms * trace_default_blocks_per_sm(0, threads);
  p.refine_blocks = sms * 8;
  p.launches = count_launches(p);
  return BH_OK;
}

TraceArgs trace_args(const bh_plan_s& p, int level) {
  TraceArgs a{};
  a.hdr = reinterpret_cast<WsHeader*>(p.ws + p.L.hdr);
  a.ip = reinterpret_cast<const ImgParams*>(p.ws + p.L.ip);
  a.out = reinterpret_cast<const OutPtrs*>(p.ws + p.L.out);
  a.head = &a.hdr->head[level];
  a.level = level;
  a.mode = 0;
  a.npix = p.npix;
  a.n_items = (int64_t)p.n * p.npix;
  a.any_volumetric = p.any_vol ? 1 : 0;
  a.base_I = reinterpret_cast<double*>(p.ws + p.L.base_I);
  a.base_cls = reinterpret_cast<uint16_t*>(p.ws + p.L.base_cls);
  a.base_depth = reinterpret_cast<uint8_t*>(p.ws + p.L.base_depth);
  if (level > 0) {
    a.lv.key = reinterpret_cast<uint64_t*>(p.ws + p.L.lv_key[level]);
    a.lv.img = reinterpret_cast<uint32_t*>(p.ws + p.L.lv_img[level]);
    a.lv.I = reinterpret_cast<double*>(p.ws + p.L.lv_I[level]);
    a.lv.cls = reinterpret_cast<uint16_t*>(p.ws + p.L.lv_cls[level]);
    a.lv.child = reinterpret_cast<int32_t*>(p.ws + p.L.lv_child[level]);
    a.lv.depth = reinterpret_cast<uint8_t*>(p.ws + p.L.lv_depth[level]);
    a.lv.cap = p.caps.c[level];
  }
  return a;
}

RefineArgs refine_args(const bh_plan_s& p) {
  RefineArgs r{};
  r.hdr = reinterpret_cast<WsHeader*>(p.ws + p.L.hdr);
  r.ip = reinterpret_cast<const ImgParams*>(p.ws + p.L.ip);
  r.out = reinterpret_cast<const OutPtrs*>(p.ws + p.L.out);
  r.n_img = p.n;
  r.npix = p.npix;
  r.levels = p.levels;
  r.base_I = reinterpret_cast<double*>(p.ws + p.L.base_I);
  r.base_cls = reinterpret_cast<uint16_t*>(p.ws + p.L.base_cls);
  r.base_child = reinterpret_cast<int32_t*>(p.ws + p.L.base_child);
  r.base_depth = reinterpret_cast<uint8_t*>(p.ws + p.L.base_depth);
  for (int l = 1; l <= p.levels; ++l) r.lv[l] = trace_args(p, l).lv;
  return r;
}

bh_status upload(const bh_plan_s& p, cudaStream_t s) {
  if (cudaMemcpyAsync(p.ws + p.L.ip, p.ip.data(), sizeof(ImgParams) * p.n,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return BH_ERR_CUDA;
  if (cudaMemcpyAsync(p.ws + p.L.out, p.out.data(), sizeof(OutPtrs) * p.n,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return BH_ERR_CUDA;
  return BH_OK;
}

// Enqueues the whole tracing call (no host data is read here, so the
// sequence can be captured into a CUDA graph).
bh_status enqueue(const bh_plan_s& p, cudaStream_t s) {
  for (int i = 0; i < p.n; ++i) {
    const OutPtrs& o = p.out[i];
    size_t plane = sizeof(float) * 3 * p.npix;
    if (o.R_em && cudaMemsetAsync(o.R_em, 0, plane, s) != cudaSuccess) return BH_ERR_CUDA;
    if (o.phi_em && cudaMemsetAsync(o.phi_em, 0, plane, s) != cudaSuccess) return BH_ERR_CUDA;
    if (o.T_em && cudaMemsetAsync(o.T_em, 0, plane, s) != cudaSuccess) return BH_ERR_CUDA;
    if (o.g && cudaMemsetAsync(o.g, 0, plane, s) != cudaSuccess) return BH_ERR_CUDA;
    if (o.keys_count && cudaMemsetAsync(o.keys_count, 0, sizeof(unsigned long long), s) != cudaSuccess)
      return BH_ERR_CUDA;
    if (o.steps && cudaMemsetAsync(o.steps, 0, sizeof(int32_t) * 2 * p.npix, s) != cudaSuccess)
      return BH_ERR_CUDA;
    if (o.promoted && cudaMemsetAsync(o.promoted, 0, p.npix, s) != cudaSuccess)
      return BH_ERR_CUDA;
  }
  WsHeader* hdr = reinterpret_cast<WsHeader*>(p.ws + p.L.hdr);
  if (launch_begin(hdr, p.budget_ns, s) != cudaSuccess) return BH_ERR_CUDA;
  RefineArgs ra = refine_args(p);
  // One refinement level's tracing: one FP64 pass, or for the mixed path
  // FP32 (may promote) -> FP64 promoted (may demote) -> FP32 demoted.
  auto trace = [&](int level) {
    TraceArgs a = trace_args(p, level);
    const int passes = p.precision == 1 ? 3 : 1;
    for (int pass = 0; pass < passes; ++pass) {
      TraceArgs b = a;
      b.head = pass == 0 ? &hdr->head[level] : &hdr->qhead[pass - 1][level];
      b.source = pass == 0 ? 0 : 1;
      b.spill_cap = p.L.spill_cap;
      if (p.precision == 1) {
        SpillRec* q0 = reinterpret_cast<SpillRec*>(p.ws + p.L.spill[0]);
        SpillRec* q1 = reinterpret_cast<SpillRec*>(p.ws + p.L.spill[1]);
        if (pass == 0) {
          b.spill_out = q0;
          b.spill_out_count = &hdr->qcount[0][level];
          b.allow_spill = 1;
        } else if (pass == 1) {
          b.spill_in = q0;
          b.spill_in_count = &hdr->qcount[0][level];
          b.spill_out = q1;
          b.spill_out_count = &hdr->qcount[1][level];
          b.allow_spill = 1;
        } else {
          b.spill_in = q1;
          b.spill_in_count = &hdr->qcount[1][level];
          b.allow_spill = 0;
        }
      }
      const cudaEvent_t* ev = &p.ev[2 * (3 * level + pass)];
      if (p.timing && cudaEventRecord(ev[0], s) != cudaSuccess) return cudaErrorUnknown;
      // host-side profiler range per level and pass (no cost without a tool)
      static const char* kPassName[3] = {"main", "fp64 promoted", "fp32 demoted"};
      char label[64];
      std::snprintf(label, sizeof(label), "bhrt trace level %d %s", level,
                    p.precision == 0 ? "fp64" : kPassName[pass]);
      nvtxRangePushA(label);
      cudaError_t e = (p.precision == 0 || pass == 1) ? launch_trace_fp64(b, p.shape64, s)
                                                      : launch_trace_mixed(b, p.shape, s);
      nvtxRangePop();
      if (e == cudaSuccess && p.timing) e = cudaEventRecord(ev[1], s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (trace(0) != cudaSuccess) return BH_ERR_CUDA;
  for (int l = 0; l < p.levels; ++l) {
    nvtxRangePushA("bhrt refine mark and expand");
    cudaError_t e = launch_mark_expand(ra, l, p.refine_blocks, s);
    nvtxRangePop();
    if (e != cudaSuccess) return BH_ERR_CUDA;
    if (trace(l + 1) != cudaSuccess) return BH_ERR_CUDA;
  }
  for (int l = p.levels > 0 ? p.levels - 1 : 0; l >= 0; --l)
    if (launch_assemble(ra, l, p.refine_blocks, s) != cudaSuccess) return BH_ERR_CUDA;
  if (p.any_keys && p.levels > 0 && launch_write_keys(ra, p.refine_blocks, s) != cudaSuccess)
    return BH_ERR_CUDA;
  return BH_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* bh_status_string(bh_status s) {
  switch (s) {
    case BH_OK: return "ok";
    case BH_ERR_INVALID_ARG: return "invalid argument";
    case BH_ERR_NO_HORIZON: return "no horizon: spin beyond the extremal value";
    case BH_ERR_OBSERVER_INSIDE: return "observer too close to the black hole";
    case BH_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case BH_ERR_CUDA: return "CUDA runtime error";
    case BH_ERR_TIMEOUT: return "device time budget exceeded";
    case BH_ERR_QUEUE_OVERFLOW: return "refinement list capacity exceeded";
    case BH_ERR_NO_ISCO: return "no stable circular orbit for the inner disk edge";
  }
  return "unknown status";
}

bh_status bh_host_geometry(const bh_spacetime* st, double* r_plus, double* chi_e,
                           double* r_isco) {
  if (!st || st->metric < 0 || st->metric > 2 || !std::isfinite(st->chi))
    return BH_ERR_INVALID_ARG;
  HostMetric m = to_metric(*st);
  if (chi_e) *chi_e = host_extremal_spin(m);
  double rp;
  if (!host_horizon(m, rp)) return BH_ERR_NO_HORIZON;
  if (r_plus) *r_plus = rp;
  if (r_isco) {
    double ri;
    if (!host_isco(m, rp, ri)) return BH_ERR_NO_ISCO;
    *r_isco = ri;
  }
  return BH_OK;
}

bh_status bh_workspace_size(int32_t n, const bh_camera* cameras, const bh_integrator* integ,
                            size_t* bytes) {
  if (n < 1 || !cameras || !bytes) return BH_ERR_INVALID_ARG;
  const bh_camera& c = cameras[0];
  if (c.nx < 1 || c.ny < 1 || c.refine_levels < 0 || c.refine_levels > kMaxLevels)
    return BH_ERR_INVALID_ARG;
  for (int i = 1; i < n; ++i)
    if (cameras[i].nx != c.nx || cameras[i].ny != c.ny ||
        cameras[i].refine_levels != c.refine_levels)
      return BH_ERR_INVALID_ARG;
  int precision = integ ? integ->precision : 0;
  if (precision < 0 || precision > kMaxPrecision) return BH_ERR_INVALID_ARG;
  *bytes = make_layout(n, (int64_t)c.nx * c.ny, c.refine_levels, default_caps(n, c), precision)
               .total;
  return BH_OK;
}

bh_status bh_trace_batch(int32_t n, const bh_spacetime* st, const bh_camera* cam,
                         const bh_emission* em, const bh_integrator* integ,
                         const bh_image_out* out, void* ws, size_t ws_bytes, void* stream) {
  bh_plan_s p;
  bh_status s;
  try {
    s = plan_build(n, st, cam, em, integ, out, ws, ws_bytes, p);
  } catch (const std::bad_alloc&) {
    return BH_ERR_INVALID_ARG;
  }
  if (s != BH_OK) return s;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if ((s = upload(p, cs)) != BH_OK) return s;
  return enqueue(p, cs);
}

bh_status bh_trace_image(const bh_spacetime* st, const bh_camera* cam, const bh_emission* em,
                         const bh_integrator* integ, const bh_image_out* out, void* workspace,
                         size_t workspace_bytes, void* stream) {
  return bh_trace_batch(1, st, cam, em, integ, out, workspace, workspace_bytes, stream);
}

// Points workspace: header | image constants | two hand-off queues of n
// records each (the mixed path's FP32 -> FP64 -> FP32 passes).
bh_status bh_points_workspace_size(int64_t n, size_t* bytes) {
  if (n < 0 || !bytes) return BH_ERR_INVALID_ARG;
  *bytes = align256(sizeof(WsHeader)) + align256(sizeof(ImgParams)) +
           2 * align256(spill_record_bytes() * (size_t)n);
  return BH_OK;
}

bh_status bh_trace_points(const bh_spacetime* st, const bh_camera* cam, const bh_emission* em,
                          const bh_integrator* integ, int64_t n, const double* xy,
                          bh_ray_record* records, void* workspace, size_t workspace_bytes,
                          void* stream) {
  if (!st || !cam || !em || !integ || n < 0 || (n > 0 && (!xy || !records)))
    return BH_ERR_INVALID_ARG;
  ImgParams ip;
  bh_status s = make_params(*st, *cam, *em, *integ, ip);
  if (s != BH_OK) return s;
  size_t need;
  bh_points_workspace_size(n, &need);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return BH_ERR_WORKSPACE;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  ImgParams* dip = reinterpret_cast<ImgParams*>(ws + align256(sizeof(WsHeader)));
  if (cudaMemcpyAsync(dip, &ip, sizeof(ip), cudaMemcpyHostToDevice, cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (n > 0 && cudaMemsetAsync(records, 0, sizeof(bh_ray_record) * n, cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (launch_begin(hdr, (unsigned long long)(integ->time_budget_s * 1e9), cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (n == 0) return BH_OK;
  TraceArgs a{};
  a.hdr = hdr;
  a.ip = dip;
  a.level = 0;
  a.mode = 1;
  a.npix = 1;
  a.n_items = n;
  a.xy = xy;
  a.rec = records;
  a.head = &hdr->head[0];
  a.source = 0;
  a.allow_spill = 0;
  a.any_volumetric = em->volumetric;
  if (integ->precision == 0) {
    LaunchShape sh{num_sms() * trace_default_blocks_per_sm(0, 128), 128};
    return launch_trace_fp64(a, sh, cs) == cudaSuccess ? BH_OK : BH_ERR_CUDA;
  }
  // mixed: the image path's three passes (FP32 -> FP64 promoted -> FP32)
  char* q = ws + align256(sizeof(WsHeader)) + align256(sizeof(ImgParams));
  SpillRec* q0 = reinterpret_cast<SpillRec*>(q);
  SpillRec* q1 = reinterpret_cast<SpillRec*>(q + align256(spill_record_bytes() * (size_t)n));
  LaunchShape s32{num_sms() * trace_default_blocks_per_sm(1, 128), 128};
  LaunchShape s64{num_sms() * trace_default_blocks_per_sm(0, 128), 128};
  a.spill_cap = n;
  for (int pass = 0; pass < 3; ++pass) {
    TraceArgs b = a;
    b.head = pass == 0 ? &hdr->head[0] : &hdr->qhead[pass - 1][0];
    b.source = pass == 0 ? 0 : 1;
    b.allow_spill = pass < 2 ? 1 : 0;
    b.spill_in = pass == 1 ? q0 : q1;
    b.spill_in_count = &hdr->qcount[pass == 1 ? 0 : 1][0];
    b.spill_out = pass == 0 ? q0 : q1;
    b.spill_out_count = &hdr->qcount[pass == 0 ? 0 : 1][0];
    cudaError_t e = pass == 1 ? launch_trace_fp64(b, s64, cs) : launch_trace_mixed(b, s32, cs);
    if (e != cudaSuccess) return BH_ERR_CUDA;
  }
  return BH_OK;
}

bh_status bh_geometry_scan(int64_t n, const bh_spacetime* st, int32_t n_theta,
                           const double* theta, double* r_plus, double* chi_e, double* R_e,
                           double* R_s, int32_t* flags, int64_t* stats, void* stream) {
  if (n < 0 || n_theta < 0 || (n > 0 && (!st || !r_plus || !chi_e || !R_e || !flags)) ||
      (n > 0 && n_theta > 0 && (!theta || !R_s)))
    return BH_ERR_INVALID_ARG;
  ScanArgs a{};
  a.st = st;
  a.n = n;
  a.n_theta = n_theta;
  a.theta = theta;
  a.r_plus = r_plus;
  a.chi_e = chi_e;
  a.R_e = R_e;
  a.R_s = R_s;
  a.flags = flags;
  a.stats = reinterpret_cast<unsigned long long*>(stats);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (stats && cudaMemsetAsync(stats, 0, 2 * sizeof(int64_t), cs) != cudaSuccess)
    return BH_ERR_CUDA;
  return launch_scan(a, cs) == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

bh_status bh_shadow_workspace_size(int64_t n_psi, size_t* bytes) {
  if (n_psi < 0 || !bytes) return BH_ERR_INVALID_ARG;
  *bytes = align256(sizeof(WsHeader)) + align256(sizeof(ImgParams));
  return BH_OK;
}

bh_status bh_shadow_boundary(const bh_spacetime* st, const bh_camera* cam,
                             const bh_integrator* integ, int64_t n_psi, const double* psi,
                             double b_lo, double b_hi, double b_tol, int32_t lanes,
                             double* b_in, double* b_out, int32_t* flags, int64_t* stats,
                             void* workspace, size_t workspace_bytes, void* stream) {
  if (!st || !cam || !integ || n_psi < 0 || (n_psi > 0 && (!psi || !b_in || !b_out || !flags)))
    return BH_ERR_INVALID_ARG;
  if (lanes < 0 || lanes > 32 || (lanes & (lanes - 1)) != 0) return BH_ERR_INVALID_ARG;
  if (!(std::isfinite(b_lo) && std::isfinite(b_hi) && b_lo >= 0.0 && b_hi > b_lo &&
        b_tol > 0.0 && std::isfinite(b_tol)))
    return BH_ERR_INVALID_ARG;
  if (integ->precision != 0) return BH_ERR_INVALID_ARG;  // FP64 integrator only
  // the screen's extent and pixel counts play no part: a one-pixel screen;
  // no emission enters a ray's fate: the thin disk with R_in = R_+ + dR_in
  bh_camera c = *cam;
  c.nx = c.ny = 1;
  c.x_min = c.y_min = -1.0;
  c.x_max = c.y_max = 1.0;
  c.refine_levels = 0;
  c.refine_capacity = 0;
  bh_emission e{};
  e.r_in_mode = 1;
  e.j0 = 1.0;
  e.p = 2.0;
  e.R_s = 8.0;
  e.sigma_in = 0.2;
  e.sigma_out = 2.0;
  e.R_out = 20.0;
  e.dR_in = 0.5;
  e.H0 = 0.05;
  e.h = 0.05;
  ImgParams ip;
  bh_status s = make_params(*st, c, e, *integ, ip);
  if (s != BH_OK) return s;
  size_t need;
  bh_shadow_workspace_size(n_psi, &need);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return BH_ERR_WORKSPACE;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  ImgParams* dip = reinterpret_cast<ImgParams*>(ws + align256(sizeof(WsHeader)));
  if (cudaMemcpyAsync(dip, &ip, sizeof(ip), cudaMemcpyHostToDevice, cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (launch_begin(hdr, (unsigned long long)(integ->time_budget_s * 1e9), cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (stats && cudaMemsetAsync(stats, 0, 3 * sizeof(int64_t), cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (n_psi == 0) return BH_OK;
  // lanes per direction: the largest power of two <= 32 with directions x
  // lanes within half the resident threads (a few warps per SM keep the FP64
  // pipe busy; more lanes only trace more rays), bisection when the
  // directions alone reach that; a grid of whole warps covering every group
  // once, at most one resident wave, in one-warp blocks when four-warp
  // blocks would leave SMs without work
  const int64_t resident = shadow_resident_threads();
  int G = 1;
  while (G < 32 && n_psi * (int64_t)(4 * G) <= resident) G *= 2;
  if (lanes > 0) G = lanes;
  const int64_t warps = (n_psi * G + 31) / 32;
  const int threads = warps >= 4 * (int64_t)num_sms() ? 128 : 32;
  const int64_t max_blocks = resident / threads;
  const int64_t per_block = threads / 32;
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((warps + per_block - 1) / per_block, max_blocks));
  ShadowArgs a{};
  a.hdr = hdr;
  a.ip = dip;
  a.psi = psi;
  a.n = n_psi;
  a.b_lo = b_lo;
  a.b_hi = b_hi;
  a.tol = b_tol;
  a.b_in = b_in;
  a.b_out = b_out;
  a.flags = flags;
  a.stats = reinterpret_cast<unsigned long long*>(stats);
  a.group = G;
  return launch_shadow(a, blocks, threads, cs) == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

bh_status bh_plan_create(int32_t n, const bh_spacetime* st, const bh_camera* cam,
                         const bh_emission* em, const bh_integrator* integ,
                         const bh_image_out* out, void* ws, size_t ws_bytes, void* stream,
                         bh_plan* plan) {
  if (!plan) return BH_ERR_INVALID_ARG;
  *plan = nullptr;
  bh_plan_s* p = new (std::nothrow) bh_plan_s();
  if (!p) return BH_ERR_INVALID_ARG;
  bh_status s;
  try {
    s = plan_build(n, st, cam, em, integ, out, ws, ws_bytes, *p);
  } catch (const std::bad_alloc&) {
    s = BH_ERR_INVALID_ARG;
  }
  if (s == BH_OK) s = upload(*p, static_cast<cudaStream_t>(stream));
  if (s == BH_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
    s = BH_ERR_CUDA;
  if (s != BH_OK) {
    delete p;
    return s;
  }
  *plan = p;
  return BH_OK;
}

bh_status bh_plan_launch(bh_plan p, int32_t use_graph, void* stream) {
  if (!p) return BH_ERR_INVALID_ARG;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (!use_graph || p->timing) return enqueue(*p, cs);
  if (!cs) return BH_ERR_INVALID_ARG;  // graphs need a non-legacy stream
  if (!p->graph) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return BH_ERR_CUDA;
    bh_status s = enqueue(*p, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (s != BH_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return BH_ERR_CUDA;
    e = cudaGraphInstantiate(&p->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->graph = nullptr;
      return BH_ERR_CUDA;
    }
  }
  return cudaGraphLaunch(p->graph, cs) == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

bh_status bh_plan_set_timing(bh_plan p, int32_t enable) {
  if (!p) return BH_ERR_INVALID_ARG;
  if (enable && !p->ev[0])
    for (auto& e : p->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return BH_ERR_CUDA;
  p->timing = enable != 0;
  return BH_OK;
}

bh_status bh_plan_set_launch(bh_plan p, int32_t which, int32_t blocks, int32_t threads,
                             int32_t variant) {
  if (!p || which < 0 || which > 1 || blocks < 1 || (threads != 64 && threads != 128) ||
      variant < 0 || variant >= kKernelVariants)
    return BH_ERR_INVALID_ARG;
  LaunchShape& sh = which == 0 ? p->shape : p->shape64;
  sh = LaunchShape{blocks, threads, variant};
  if (p->graph) {
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return BH_OK;
}

bh_status bh_plan_stats(bh_plan p, void* stream, bh_run_stats* out) {
  if (!p || !out) return BH_ERR_INVALID_ARG;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  WsHeader h;
  if (cudaMemcpyAsync(&h, p->ws + p->L.hdr, sizeof(h), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return BH_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->fp32_ms = out->fp64_ms = p->timing ? 0.0 : -1.0;
  const int passes = p->precision == 1 ? 3 : 1;
  for (int l = 0; l <= kMaxLevels; ++l) {
    out->rays[l] = (int64_t)h.rays[l];
    out->cells[l] = l == 0 ? (int64_t)p->n * p->npix : (int64_t)h.count[l];
    out->trace_ms[l] = -1.0;
    if (p->timing && l <= p->levels) {
      out->trace_ms[l] = 0.0;
      for (int pass = 0; pass < passes; ++pass) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev[2 * (3 * l + pass)], p->ev[2 * (3 * l + pass) + 1]) !=
            cudaSuccess)
          continue;
        out->trace_ms[l] += ms;
        if (p->precision == 0 || pass == 1) out->fp64_ms += ms; else out->fp32_ms += ms;
      }
    }
  }
  out->accepted_fp64 = (int64_t)h.accepted;
  out->rejected_fp64 = (int64_t)h.rejected;
  out->accepted_fp32 = (int64_t)h.accepted32;
  out->rejected_fp32 = (int64_t)h.rejected32;
  out->promoted_rays = (int64_t)h.promoted_rays;
  out->spill_full = (int64_t)h.spill_full;
  out->max_ray_steps = (int64_t)h.max_ray_steps;
  out->kernel_launches = p->launches;
  out->status = h.status;
  out->trace_blocks = p->shape.blocks;
  out->trace_threads = p->shape.threads;
  for (int pass = 0; pass < 3; ++pass)
    for (int l = 0; l <= kMaxLevels; ++l) {
      const unsigned long long b = h.t_pass[0][pass][l], d = h.t_pass[1][pass][l],
                               e = h.t_pass[2][pass][l];
      const bool ok = b && d && e && d >= b && e >= d;
      out->bulk_ms[pass][l] = ok ? (double)(d - b) * 1e-6 : -1.0;
      out->tail_ms[pass][l] = ok ? (double)(e - d) * 1e-6 : -1.0;
    }
  out->lane_util_fp32 = h.warp_iters[0] ? (double)h.lane_iters[0] / (32.0 * h.warp_iters[0]) : -1.0;
  out->lane_util_fp64 = h.warp_iters[1] ? (double)h.lane_iters[1] / (32.0 * h.warp_iters[1]) : -1.0;
  return BH_OK;
}

// Autotuner: times the whole launch (all levels, all precision passes) for
// each candidate shape of the persistent trace kernel(s) and keeps the
// fastest.  Candidates: 128-thread blocks at 1..occupancy blocks per SM and
// 64-thread blocks at twice that, for the main kernel; the FP64 pass of the
// mixed path is tuned afterwards the same way.
bh_status bh_plan_autotune(bh_plan p, void* stream, bh_tune_report* rep) {
  if (!p) return BH_ERR_INVALID_ARG;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const bool was_timing = p->timing;
  if (bh_plan_set_timing(p, 1) != BH_OK) return BH_ERR_CUDA;
  if (p->graph) {
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  const int sms = num_sms();
  auto run_ms = [&](double& ms) -> bh_status {
    bh_status s = enqueue(*p, cs);
    if (s != BH_OK) return s;
    bh_run_stats st;
    s = bh_plan_stats(p, stream, &st);
    if (s != BH_OK) return s;
    if (st.status != BH_OK) return static_cast<bh_status>(st.status);
    ms = 0.0;
    for (int l = 0; l <= p->levels; ++l) ms += st.trace_ms[l];
    return BH_OK;
  };
  int tried = 0;
  for (int which = 0; which < (p->precision == 1 ? 2 : 1); ++which) {
    LaunchShape& sh = which == 0 ? p->shape : p->shape64;
    const int prec = which == 0 ? p->precision : 0;
    LaunchShape cand[24];
    int nc = 0;
    const int nvar = kKernelVariants;
    for (int v = 0; v < nvar; ++v) {
      const int occ = trace_default_blocks_per_sm(prec, 128, v);
      for (int b = (v == 0 ? 1 : occ); b <= occ && nc < 20; ++b)
        cand[nc++] = LaunchShape{sms * b, 128, v};
      cand[nc++] = LaunchShape{sms * 2 * occ, 64, v};
    }
    LaunchShape best = sh;
    double best_ms = 1e300;
    for (int c = 0; c < nc; ++c) {
      sh = cand[c];
      double ms;
      bh_status s = run_ms(ms);
      if (s != BH_OK) return s;
      ++tried;
      if (ms < best_ms) {
        best_ms = ms;
        best = cand[c];
      }
    }
    sh = best;
    if (rep) {
      rep->best_ms[which] = best_ms;
      rep->blocks[which] = best.blocks;
      rep->threads[which] = best.threads;
      rep->variant[which] = best.variant;
    }
  }
  if (rep) rep->candidates = tried;
  p->timing = was_timing;
  return BH_OK;
}

bh_status bh_plan_destroy(bh_plan p) {
  if (!p) return BH_OK;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  delete p;
  return BH_OK;
}

bh_status bh_workspace_status(const void* workspace, void* stream) {
  if (!workspace) return BH_ERR_INVALID_ARG;
  int32_t st = 0;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&st, workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (cudaStreamSynchronize(cs) != cudaSuccess) return BH_ERR_CUDA;
  return static_cast<bh_status>(st);
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint
namespace {

constexpr int kAdjThreads = 128;
constexpr int kAdjBlocksPerSM = 2;
// checkpoint room per adjoint thread in the workspace (64 checkpoints x 64
// steps = 4096 accepted steps per ray); rays of the forward image that took
// more steps get larger slabs and the adjoint runs on fewer threads
constexpr int kAdjMaxCkpt = 64;

// Lapse H(R) for any scalar type: Kerr, Eq. (9) with halo1 = lambda_E,
// Eq. (13) with halo1 = eta, halo2 = lambda_c.
template <class T>
T lapse_any(int metric, const T& R, const T& h1, const T& h2) {
  using std::exp;
  using std::log1p;
  if (metric == BH_EINASTO) {
    T e = exp(-R / h1);
    return 1.0 - 2.0 / R + (2.0 / R + 2.0 / h1 + R / (h1 * h1)) * e;
  }
  if (metric == BH_CNFW) {
    T S = h1 * h2 * (1.0 / (R + h2) - (2.0 / R) * log1p(R / h2));
    return exp(S) - 2.0 / R;
  }
  return 1.0 - 2.0 / R;
}

// Prograde circular-orbit energy -u_T (Eqs. 90-91) with H' from a dual.
double circ_energy(int metric, double R, double chi, double h1, double h2) {
  Dual<1> Hd = lapse_any(metric, Dual<1>::var(R, 0), Dual<1>(h1), Dual<1>(h2));
  const double H = Hd.v, dH = Hd.d[0], x2 = chi * chi;
  const double den = 2.0 * R - x2 * dH, disc = 2.0 * R * dH;
  const double W = (-chi * dH + std::sqrt(disc)) / den;
  const double gtt = -H, gtp = -chi * (1.0 - H), gpp = R * R + x2 + x2 * (1.0 - H);
  const double norm = -(gtt + 2.0 * W * gtp + W * W * gpp);
  return -(gtt + W * gtp) / std::sqrt(norm);
}

// Derivatives of the ZAMO frame at the observer and of R_in with respect
// to (chi, theta_o, halo1, halo2).
AdjImg adjoint_constants(const bh_spacetime& s, const bh_camera& c, const bh_emission& e,
                         const ImgParams& ip) {
  using D4 = Dual<4>;
  AdjImg aj;
  std::memset(&aj, 0, sizeof(aj));
  const bool ein = s.metric == BH_EINASTO, nfw = s.metric == BH_CNFW;
  D4 chi = D4::var(s.chi, 0), th = D4::var(c.incl, 1);
  D4 h1 = ein ? D4::var(s.lambda_E, 2) : (nfw ? D4::var(s.eta, 2) : D4(1.0));
  D4 h2 = nfw ? D4::var(s.lambda_c, 3) : D4(1.0);
  D4 R(c.r_obs);
  D4 H = lapse_any(s.metric, R, h1, h2);
  D4 cs = cos(th), sn = sin(th), s2 = sn * sn, x2 = chi * chi;
  D4 Sig = R * R + x2 * cs * cs, F = R * R * (1.0 - H), D = R * R * H + x2;
  D4 gtt = -(1.0 - F / Sig), gtp = -chi * F * s2 / Sig, grr = Sig / D, gthth = Sig;
  D4 gpp = s2 * (R * R + x2 + x2 * F * s2 / Sig);
  D4 w = -gtp / gpp;
  D4 N = sqrt(-(gtt + 2.0 * w * gtp + w * w * gpp));
  D4 sr = sqrt(grr), st = sqrt(gthth), sp = sqrt(gpp);
  for (int k = 0; k < 4; ++k) {
    aj.d_sqgrr[k] = sr.d[k];
    aj.d_sqgth[k] = st.d[k];
    aj.d_sqgph[k] = sp.d[k];
    aj.d_N[k] = N.d[k];
    aj.d_w[k] = w.d[k];
  }
  const double p1 = ein ? s.lambda_E : (nfw ? s.eta : 1.0), p2 = nfw ? s.lambda_c : 1.0;
  if (e.r_in_mode == 1) {
    // R_in = R_+ + dR_in: implicit derivative of Delta(R_+) = 0
    using D5 = Dual<5>;
    D5 Rp = D5::var(ip.r_plus, 0), ch = D5::var(s.chi, 1);
    D5 q1 = (ein || nfw) ? D5::var(p1, 3) : D5(p1), q2 = nfw ? D5::var(p2, 4) : D5(p2);
    D5 Dl = Rp * Rp * lapse_any(s.metric, Rp, q1, q2) + ch * ch;
    for (int k = 0; k < 4; ++k) aj.d_Rin[k] = k == 1 ? 0.0 : -Dl.d[1 + k] / Dl.d[0];
  } else {
    // R_in = r_ISCO: dE/dR = 0, so dR/dq = -E_Rq / E_RR (central differences)
    const double Ri = ip.R_in, dR = 1e-3;
    auto ER = [&](double rr, double ch, double a1, double a2) {
      return (circ_energy(s.metric, rr + dR, ch, a1, a2) -
              circ_energy(s.metric, rr - dR, ch, a1, a2)) / (2.0 * dR);
    };
    const double ERR = (circ_energy(s.metric, Ri + dR, s.chi, p1, p2) -
                        2.0 * circ_energy(s.metric, Ri, s.chi, p1, p2) +
                        circ_energy(s.metric, Ri - dR, s.chi, p1, p2)) / (dR * dR);
    const double base[4] = {s.chi, 0.0, p1, p2};
    for (int k = 0; k < 4; ++k) {
      if (k == 1 || (k >= 2 && !(ein || nfw)) || (k == 3 && !nfw)) continue;
      double q[4] = {base[0], 0.0, base[2], base[3]};
      const double eps = 1e-4 * std::fmax(std::fabs(base[k]), 1e-2);
      q[k] = base[k] + eps;
      const double up = ER(Ri, q[0], q[2], q[3]);
      q[k] = base[k] - eps;
      const double dn = ER(Ri, q[0], q[2], q[3]);
      aj.d_Rin[k] = -((up - dn) / (2.0 * eps)) / ERR;
    }
  }
  return aj;
}

struct BwdLayout {
  Layout fwd;
  size_t I, nc, st, G, mom, lr, hs, hc, uv, V, grad, head, status, ckpt, total;
  int nbins, threads;
};

bool bwd_layout(const bh_camera& c, BwdLayout& B) {
  if (c.nx < 1 || c.ny < 1 || c.refine_levels < 0 || c.refine_levels > kMaxLevels ||
      !(c.x_max > c.x_min))
    return false;
  const int64_t npix = (int64_t)c.nx * c.ny;
  B.fwd = make_layout(1, npix, c.refine_levels, default_caps(1, c), 0);
  const double dx = (c.x_max - c.x_min) / c.nx;
  const double ax = std::fmax(std::fabs(c.x_min), std::fabs(c.x_max));
  const double ay = std::fmax(std::fabs(c.y_min), std::fabs(c.y_max));
  B.nbins = (int)std::floor(std::sqrt(ax * ax + ay * ay) / dx) + 2;
  B.threads = num_sms() * kAdjBlocksPerSM * kAdjThreads;
  size_t o = B.fwd.total;
  auto take = [&](size_t b) {
    size_t at = o;
    o = align256(o + b);
    return at;
  };
  B.I = take(sizeof(float) * npix);
  B.nc = take(npix);
  B.st = take(npix);
  B.G = take(sizeof(double) * npix);
  B.mom = take(sizeof(double) * 3);
  B.lr = take(sizeof(double) * 2);
  B.hs = take(sizeof(double) * B.nbins);
  B.hc = take(sizeof(unsigned long long) * B.nbins);
  B.uv = take(sizeof(double) * 16);
  B.V = take(sizeof(double) * 16);
  B.grad = take(sizeof(double) * 10);
  B.head = take(sizeof(unsigned long long));
  B.status = take(sizeof(int));
  B.ckpt = take(sizeof(Ckpt) * (size_t)B.threads * kAdjMaxCkpt);
  B.total = o;
  return true;
}

}  // namespace

extern "C" {

bh_status bh_backward_workspace_size(const bh_camera* cam, size_t* bytes) {
  BwdLayout B;
  if (!cam || !bytes || !bwd_layout(*cam, B)) return BH_ERR_INVALID_ARG;
  *bytes = B.total;
  return BH_OK;
}

bh_status bh_trace_backward(const bh_spacetime* st, const bh_camera* cam, const bh_emission* em,
                            const bh_integrator* integ, const float* dL_dI,
                            const double* dL_ddiag, const double* uv8, double* grad10,
                            double* diag11, float* image_out, void* workspace,
                            size_t workspace_bytes, void* stream) {
  if (!st || !cam || !em || !integ || !grad10) return BH_ERR_INVALID_ARG;
  if (em->volumetric) return BH_ERR_INVALID_ARG;  // the adjoint covers the thin-disk events
  BwdLayout BL;
  if (!bwd_layout(*cam, BL)) return BH_ERR_INVALID_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < BL.total)
    return BH_ERR_WORKSPACE;
  char* ws = static_cast<char*>(workspace);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  bh_integrator it64 = *integ;
  it64.precision = 0;  // the adjoint differentiates the FP64 path
  const int64_t npix = (int64_t)cam->nx * cam->ny;
  float* I = reinterpret_cast<float*>(ws + BL.I);
  bh_image_out out;
  std::memset(&out, 0, sizeof(out));
  out.I = I;
  out.ncross = reinterpret_cast<uint8_t*>(ws + BL.nc);
  out.status = reinterpret_cast<uint8_t*>(ws + BL.st);
  // 1. forward image
  bh_plan_s p;
  bh_status s;
  try {
    s = plan_build(1, st, cam, em, &it64, &out, ws, BL.fwd.total, p);
  } catch (const std::bad_alloc&) {
    return BH_ERR_INVALID_ARG;
  }
  if (s != BH_OK) return s;
  if ((s = upload(p, cs)) != BH_OK) return s;
  if ((s = enqueue(p, cs)) != BH_OK) return s;
  // 2. image statistics for the diagnostics terms
  ImgAdj A;
  std::memset(&A, 0, sizeof(A));
  A.nx = cam->nx;
  A.ny = cam->ny;
  A.x_min = cam->x_min;
  A.y_min = cam->y_min;
  A.dx = (cam->x_max - cam->x_min) / cam->nx;
  A.dy = (cam->y_max - cam->y_min) / cam->ny;
  A.nbins = BL.nbins;
  double* mom = reinterpret_cast<double*>(ws + BL.mom);
  double* lr = reinterpret_cast<double*>(ws + BL.lr);
  double* hs = reinterpret_cast<double*>(ws + BL.hs);
  unsigned long long* hc = reinterpret_cast<unsigned long long*>(ws + BL.hc);
  if (cudaMemsetAsync(ws + BL.mom, 0, BL.uv - BL.mom, cs) != cudaSuccess) return BH_ERR_CUDA;
  if (launch_image_moments(I, A, mom, cs) != cudaSuccess) return BH_ERR_CUDA;
  double hm[3];
  if (cudaMemcpyAsync(hm, mom, sizeof(hm), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return BH_ERR_CUDA;
  A.S = hm[0];
  A.Xc = hm[0] != 0.0 ? hm[1] / hm[0] : 0.0;
  A.Yc = hm[0] != 0.0 ? hm[2] / hm[0] : 0.0;
  A.C = std::sqrt(A.Xc * A.Xc + A.Yc * A.Yc);
  if (launch_image_profile(I, A, lr, hs, hc, cs) != cudaSuccess) return BH_ERR_CUDA;
  std::vector<double> hsv(BL.nbins);
  std::vector<unsigned long long> hcv(BL.nbins);
  double hlr[2];
  if (cudaMemcpyAsync(hlr, lr, sizeof(hlr), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaMemcpyAsync(hsv.data(), hs, sizeof(double) * BL.nbins, cudaMemcpyDeviceToHost, cs) !=
          cudaSuccess ||
      cudaMemcpyAsync(hcv.data(), hc, sizeof(unsigned long long) * BL.nbins,
                      cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return BH_ERR_CUDA;
  A.FRs = hlr[0];
  A.FLs = hlr[1];
  const double A_LR = (A.FRs + A.FLs) != 0.0 ? (A.FRs - A.FLs) / (A.FRs + A.FLs) : 0.0;
  // radial profile peak with a parabolic vertex through the argmax bin and
  // its neighbours (differentiable reading of the bin-centre peak)
  int bstar = -1;
  double bv = 0.0;
  for (int b = 0; b < BL.nbins; ++b) {
    if (!hcv[b]) continue;
    const double m = hsv[b] / (double)hcv[b];
    if (bstar < 0 || m > bv) {
      bv = m;
      bstar = b;
    }
  }
  double delta = 0.0;
  A.bstar = bstar;
  if (bstar > 0 && bstar + 1 < BL.nbins && hcv[bstar - 1] && hcv[bstar + 1]) {
    const double mm = hsv[bstar - 1] / (double)hcv[bstar - 1], m0 = bv,
                 mp = hsv[bstar + 1] / (double)hcv[bstar + 1];
    const double Dd = mm - 2.0 * m0 + mp, Nn = 0.5 * (mm - mp);
    if (Dd != 0.0) {
      delta = Nn / Dd;
      A.drho[0] = A.dx * (0.5 * Dd - Nn) / (Dd * Dd);
      A.drho[1] = A.dx * (2.0 * Nn) / (Dd * Dd);
      A.drho[2] = A.dx * (-0.5 * Dd - Nn) / (Dd * Dd);
      for (int t = 0; t < 3; ++t) A.cnt[t] = (int)hcv[bstar - 1 + t];
    }
  }
  const double rho_peak = (bstar + 0.5 + delta) * A.dx;
  // visibility amplitudes at the given baselines
  double hv[16] = {0};
  const double dA = A.dx * A.dy;
  A.V0 = A.S * dA;
  if (uv8) {
    std::memcpy(A.uv, uv8, sizeof(double) * 16);
    if (cudaMemcpyAsync(ws + BL.uv, uv8, sizeof(double) * 16, cudaMemcpyHostToDevice, cs) !=
        cudaSuccess)
      return BH_ERR_CUDA;
    s = bh_visibilities_fp64(I, cam, reinterpret_cast<double*>(ws + BL.uv), 8,
                             reinterpret_cast<double*>(ws + BL.V), stream);
    if (s != BH_OK) return s;
    if (cudaMemcpyAsync(hv, ws + BL.V, sizeof(hv), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
      return BH_ERR_CUDA;
  }
  for (int k = 0; k < 8; ++k) {
    A.Vre[k] = hv[2 * k];
    A.Vim[k] = hv[2 * k + 1];
    A.Vabs[k] = std::sqrt(hv[2 * k] * hv[2 * k] + hv[2 * k + 1] * hv[2 * k + 1]);
  }
  if (diag11) {
    diag11[0] = A.C;
    diag11[1] = A_LR;
    diag11[2] = rho_peak;
    for (int k = 0; k < 8; ++k) diag11[3 + k] = A.V0 != 0.0 ? A.Vabs[k] / A.V0 : 0.0;
  }
  // 3. dL/dI per pixel
  A.dLdI = dL_dI;
  if (dL_ddiag) {
    A.cC = dL_ddiag[0];
    A.cA = dL_ddiag[1];
    A.cR = dL_ddiag[2];
    for (int k = 0; k < 8; ++k) A.cV[k] = uv8 ? dL_ddiag[3 + k] : 0.0;
  }
  A.G = reinterpret_cast<double*>(ws + BL.G);
  if (launch_pixel_adjoint(A, cs) != cudaSuccess) return BH_ERR_CUDA;
  // 4. rays
  AdjArgs J;
  std::memset(&J, 0, sizeof(J));
  RefineArgs ra = refine_args(p);
  J.hdr = ra.hdr;
  J.ip = ra.ip;
  J.aj = adjoint_constants(*st, *cam, *em, p.ip[0]);
  J.levels = p.levels;
  J.npix = npix;
  J.Gpix = A.G;
  J.base_child = ra.base_child;
  for (int l = 1; l <= kMaxLevels; ++l) J.lv[l] = ra.lv[l];
  J.ckpt = reinterpret_cast<Ckpt*>(ws + BL.ckpt);
  J.grad = reinterpret_cast<double*>(ws + BL.grad);
  J.head = reinterpret_cast<unsigned long long*>(ws + BL.head);
  J.status = reinterpret_cast<int*>(ws + BL.status);
  // checkpoint slab per thread from the forward image's longest ray (its
  // attempted steps bound the accepted steps the replay checkpoints): the
  // workspace's checkpoint region is divided among as many threads as it
  // can hold such slabs, up to the default grid
  unsigned long long longest = 0;
  if (cudaMemcpyAsync(&longest, &ra.hdr->max_ray_steps, sizeof(longest), cudaMemcpyDeviceToHost,
                      cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return BH_ERR_CUDA;
  const int64_t room = (int64_t)BL.threads * kAdjMaxCkpt;  // checkpoints in the region
  const int64_t per = std::max<int64_t>(kAdjMaxCkpt, (int64_t)(longest / kCkptEvery) + 2);
  int64_t threads = std::min<int64_t>(BL.threads, room / per) / kAdjThreads * kAdjThreads;
  if (threads < kAdjThreads) return BH_ERR_WORKSPACE;
  J.max_ckpt = (int)std::min<int64_t>(room / threads, 1 << 30);
  if (cudaMemsetAsync(ws + BL.grad, 0, BL.ckpt - BL.grad, cs) != cudaSuccess) return BH_ERR_CUDA;
  if (launch_adjoint(J, (int)(threads / kAdjThreads), kAdjThreads, cs) != cudaSuccess)
    return BH_ERR_CUDA;
  int dstat = 0;
  if (cudaMemcpyAsync(grad10, J.grad, sizeof(double) * 10, cudaMemcpyDeviceToHost, cs) !=
          cudaSuccess ||
      cudaMemcpyAsync(&dstat, J.status, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    return BH_ERR_CUDA;
  if (image_out &&
      cudaMemcpyAsync(image_out, I, sizeof(float) * npix, cudaMemcpyDeviceToDevice, cs) !=
          cudaSuccess)
    return BH_ERR_CUDA;
  if (cudaStreamSynchronize(cs) != cudaSuccess) return BH_ERR_CUDA;
  WsHeader h;
  if (cudaMemcpy(&h, ra.hdr, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return BH_ERR_CUDA;
  if (h.status != BH_OK) return static_cast<bh_status>(h.status);
  return static_cast<bh_status>(dstat);
}

}  // extern "C"
