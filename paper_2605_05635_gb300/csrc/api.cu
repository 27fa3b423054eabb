// api.cu -- the C ABI: argument validation, host-side geometry (horizon,
// extremal spin, ISCO, ZAMO frame), workspace layout and the launch
// sequence of one tracing call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace bhrt;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxPrecision = 1;
// Mixed path: a promoted ray returns to FP32 once it is outgoing beyond this
// radius (reading: well outside the photon region of every metric here).
constexpr double kDemoteR = 10.0;

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
  if (e.r_in_mode < 0 || e.r_in_mode > 1 || e.reserved != 0) return BH_ERR_INVALID_ARG;
  if (!finite_pos(e.R_s) || !finite_pos(e.sigma_in) || !finite_pos(e.sigma_out) ||
      !std::isfinite(e.j0) || !std::isfinite(e.p) || !std::isfinite(e.R_out))
    return BH_ERR_INVALID_ARG;
  if (e.r_in_mode == 1 && !(e.dR_in >= 0.0)) return BH_ERR_INVALID_ARG;
  if (g.precision < 0 || g.precision > kMaxPrecision || g.max_steps < 1) return BH_ERR_INVALID_ARG;
  if (!finite_pos(g.rtol) || !finite_pos(g.atol) || !(g.cap_factor >= 1.0) ||
      !(g.esc_factor > 1.0) || !(g.thetadot_min >= 0.0) || !(g.dlambda_min >= 0.0) ||
      !(g.promote_dr >= 0.0) || !(g.time_budget_s >= 0.0))
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
  ip.rtol = g.rtol;
  ip.atol = g.atol;
  ip.thdot_min = g.thetadot_min;
  ip.dlam_min = g.dlambda_min;
  ip.promote_R = rp + g.promote_dr;
  ip.demote_R = kDemoteR;
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

Layout make_layout(int n, int64_t npix, int levels, int64_t cap, int precision) {
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
  for (int l = 1; l <= levels; ++l) {
    L.lv_key[l] = take(sizeof(uint64_t) * cap);
    L.lv_img[l] = take(sizeof(uint32_t) * cap);
    L.lv_I[l] = take(sizeof(double) * 4 * cap);
    L.lv_cls[l] = take(sizeof(uint16_t) * cap);
    L.lv_child[l] = take(sizeof(int32_t) * cap);
    L.lv_depth[l] = take(cap);
  }
  L.spill_cap = 0;
  L.spill[0] = L.spill[1] = 0;
  if (precision == 1) {
    L.spill_cap = levels > 0 && cap > nb ? cap : nb;
    L.spill[0] = take(spill_record_bytes() * L.spill_cap);
    L.spill[1] = take(spill_record_bytes() * L.spill_cap);
  }
  L.total = o;
  return L;
}

int64_t default_cap(int n, const bh_camera& c) {
  int64_t cap = c.refine_capacity > 0 ? c.refine_capacity : 16 * (int64_t)c.nx * c.ny * n;
  if (c.refine_capacity == 0 && cap < 65536) cap = 65536;
  cap = (cap + 15) & ~int64_t(15);
  if (cap > (int64_t(1) << 30)) cap = int64_t(1) << 30;  // int32 child indices
  return cap;
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

// ------------------------------------------------------------------- plan
struct bh_plan_s {
  int n = 0, levels = 0, precision = 0;
  int64_t npix = 0, cap = 0;
  std::vector<ImgParams> ip;
  std::vector<OutPtrs> out;
  char* ws = nullptr;
  Layout L{};
  unsigned long long budget_ns = 0;
  LaunchShape shape{0, 128};    // main trace kernel (FP64 or FP32 bulk)
  LaunchShape shape64{0, 128};  // FP64 promoted pass of the mixed path
  int refine_blocks = 0;
  bool any_keys = false;
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
  p.cap = default_cap(n, cam[0]);
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
    if (d.keys_count) p.any_keys = true;
    if (integ[i].time_budget_s > budget) budget = integ[i].time_budget_s;
  }
  p.budget_ns = (unsigned long long)(budget * 1e9);
  p.L = make_layout(n, p.npix, p.levels, p.cap, p.precision);
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
    a.lv.cap = p.cap;
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
      cudaError_t e = (p.precision == 0 || pass == 1) ? launch_trace_fp64(b, p.shape64, s)
                                                      : launch_trace_mixed(b, p.shape, s);
      if (e == cudaSuccess && p.timing) e = cudaEventRecord(ev[1], s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (trace(0) != cudaSuccess) return BH_ERR_CUDA;
  for (int l = 0; l < p.levels; ++l) {
    if (launch_mark_expand(ra, l, p.refine_blocks, s) != cudaSuccess) return BH_ERR_CUDA;
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
  *bytes = make_layout(n, (int64_t)c.nx * c.ny, c.refine_levels, default_cap(n, c), precision)
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

bh_status bh_points_workspace_size(int64_t n, size_t* bytes) {
  if (n < 0 || !bytes) return BH_ERR_INVALID_ARG;
  *bytes = align256(sizeof(WsHeader)) + align256(sizeof(ImgParams));
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
  a.allow_spill = 0;  // points mode: the mixed kernel runs without promotion
  LaunchShape sh{num_sms() * trace_default_blocks_per_sm(integ->precision, 128), 128};
  cudaError_t e = integ->precision == 0 ? launch_trace_fp64(a, sh, cs) : launch_trace_mixed(a, sh, cs);
  return e == cudaSuccess ? BH_OK : BH_ERR_CUDA;
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
  out->kernel_launches = p->launches;
  out->status = h.status;
  out->trace_blocks = p->shape.blocks;
  out->trace_threads = p->shape.threads;
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
