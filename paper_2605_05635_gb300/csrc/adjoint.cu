// adjoint.cu -- discrete adjoint of the FP64 image path: gradients of
//   L = sum_p dL/dI_p I_p + sum_m dL/dD_m D_m,
//   D = (C, A_LR, rho_peak (parabolic vertex), |V(u_k,v_k)|/|V(0,0)|, k = 1..8)
// with respect to (chi, theta_o, halo1, halo2, j0, p, R_s, sigma_in,
// sigma_out, R_out): spin and inclination (Sec. 3.2), halo parameters
// (Einasto lambda_E as halo1; cored-NFW eta, lambda_c as halo1, halo2;
// Eqs. 9-14) and the emissivity parameters (Eqs. 83-86).
//
// The derivative is that of the algorithm as executed, with the adaptive
// decisions frozen: accepted step sizes, the refinement pattern, the trusted
// crossing choices and the termination step are held fixed; the crossing
// abscissa on the dense output is differentiated implicitly.  Per ray:
//   1. a forward replay in FP64 records a checkpoint every 64 accepted steps
//      and the crossings (step, sigma*, dI/dR_em);
//   2. the reverse sweep replays each 64-step segment from its checkpoint,
//      then walks its steps backwards: the seven stage Jacobians come from
//      forward-mode dual numbers through the same right-hand side as the
//      forward kernels, and the Runge-Kutta adjoint recursion propagates the
//      adjoint of (R, theta, p_R, p_theta) and accumulates that of (E, ell,
//      chi, halo1, halo2);
//   3. the launch (Eqs. 70-74) maps the initial adjoint to the parameters
//      through host-computed derivatives of the ZAMO frame.
// The image-level part (dL/dI per pixel from the diagnostics and the
// visibility amplitudes) is a separate per-pixel kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "adjoint.h"
#include "dual.cuh"
#include "integrator.cuh"

namespace bhrt {

struct XRec {
  int32_t step;
  double sig;
  double Rbar;
};

template <int N>
__device__ __forceinline__ MetricConsts<Dual<N>> metric_dual(const ImgParams& ip, int kchi,
                                                              int kh1, int kh2) {
  MetricConsts<Dual<N>> m;
  m.metric = ip.metric;
  m.chi = Dual<N>::var(ip.chi, kchi);
  m.chi2 = m.chi * m.chi;
  if (ip.metric == 1) {
    Dual<N> lE = Dual<N>::var(ip.lamE, kh1);
    m.il = Dual<N>(1.0) / lE;
  } else {
    m.il = Dual<N>(0.0);
  }
  if (ip.metric == 2) {
    Dual<N> eta = Dual<N>::var(ip.eta, kh1), lc = Dual<N>::var(ip.lamc, kh2);
    m.eta_lc = eta * lc;
    m.lc = lc;
    m.ilc = Dual<N>(1.0) / lc;
  } else {
    m.eta_lc = Dual<N>(ip.eta * ip.lamc);
    m.lc = Dual<N>(ip.lamc);
    m.ilc = Dual<N>(0.0);
  }
  return m;
}

// Thin-disk contribution I_c = g^3 j at a crossing radius R with tangents
// 0 R, 1 E, 2 ell, 3 chi, 4 halo1, 5 halo2, 6 R_in, 7 j0, 8 p, 9 R_s,
// 10 sigma_in, 11 sigma_out, 12 R_out (same formulas as emitter_g and
// emissivity_eq of the forward kernels, Eqs. 83-91).
using D13 = Dual<13>;
__device__ bool crossing_intensity_dual(const ImgParams& ip, double R, double E, double ell,
                                        D13& I) {
  MetricConsts<D13> m = metric_dual<13>(ip, 3, 4, 5);
  D13 r = D13::var(R, 0), e = D13::var(E, 1), l = D13::var(ell, 2);
  D13 iR = D13(1.0) / r, H, dH;
  lapse(m, r, iR, H, dH);
  D13 den = 2.0 * r - m.chi2 * dH;
  D13 disc = 2.0 * r * dH;
  if (!(disc.v >= 0.0) || den.v == 0.0) return false;
  D13 W = (-m.chi * dH + sqrt(disc)) / den;
  D13 gtt = -H, gtp = -m.chi * (1.0 - H), gpp = r * r + m.chi2 + m.chi2 * (1.0 - H);
  D13 norm = -(gtt + 2.0 * W * gtp + W * W * gpp);
  if (!(norm.v > 0.0)) return false;
  D13 uT = 1.0 / sqrt(norm);
  D13 g = 1.0 / (uT * (e - W * l));
  D13 Rin = D13::var(ip.R_in, 6), j0 = D13::var(ip.j0, 7), p = D13::var(ip.p, 8);
  D13 Rs = D13::var(ip.R_s, 9), si = D13::var(ip.sig_in, 10), so = D13::var(ip.sig_out, 11);
  D13 Ro = D13::var(ip.R_out, 12);
  D13 tin = 0.5 * (1.0 + tanh((r - Rin) / si));
  D13 tout = 0.5 * (1.0 - tanh((r - Ro) / so));
  D13 j = j0 * pow(r / Rin, -p) * exp(-(r - Rin) / Rs) * tin * tout;
  I = g * g * g * j;
  return true;
}

// One attempted FP64 step of the adjoint's own forward replay: the same
// Dormand-Prince step, crossing rule and termination as ray_step64, and it
// also reports the crossing abscissa.  Returns 0 (continue) or status + 1.
__device__ int adj_step(const ImgParams& ip, const MetricConsts<double>& m, Ray64& r,
                        bool& crossed, double& sig_out, double& Rc_out, bool& reflected) {
  crossed = false;
  reflected = false;
  const double h = r.h;
  double k[7][6];
#pragma unroll
  for (int i = 0; i < 6; ++i) k[0][i] = r.f[i];
  bool bad = false;
  double W, P2;
#pragma unroll
  for (int s = 1; s < 7; ++s) {
    double ys[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < s; ++j) acc += kDP.a[s][j] * k[j][i];
      ys[i] = r.y[i] + h * acc;
    }
    bad |= !geo_rhs(m, r.E, r.ell, ys[1], ys[2], ys[4], ys[5], k[s], W, P2);
  }
  double y1[6];
  float err2 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double a5 = 0.0, ae = 0.0;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      a5 += kDP.b[j] * k[j][i];
      ae += kDP.e[j] * k[j][i];
    }
    y1[i] = r.y[i] + h * a5;
    err2 += err_term(r.y[i], y1[i], h * ae, f32_trunc(ip.atol), f32_trunc(ip.rtol));
  }
  float err = sqrtf(err2 / 6.f);
  r.steps++;
  if (bad || !(err <= 1.f)) {
    r.h = bad ? 0.5 * h : h * (double)step_factor(err, true);
    r.rejected = true;
    r.nrej++;
    return r.steps >= ip.max_steps ? 3 : 0;
  }
  r.nacc++;
  const double s0 = r.y[2] - kHalfPi, s1 = y1[2] - kHalfPi;
  if ((s0 > 0.0 && s1 <= 0.0) || (s0 < 0.0 && s1 >= 0.0)) {
    double hd[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double a = 0.0;
#pragma unroll
      for (int j = 0; j < 7; ++j) a += kDP.d[j] * k[j][i];
      hd[i] = h * a;
    }
    double sig = 1.0;
    if (s1 != 0.0) {
      double x0 = 0.0, f0 = s0, x1 = 1.0, f1 = s1;
      for (int it = 0; it < 80; ++it) {
        double x2 = x1 - f1 * (x1 - x0) / (f1 - f0);
        if (!(x2 > fmin(x0, x1) && x2 < fmax(x0, x1))) x2 = 0.5 * (x0 + x1);
        double f2 = dense1(r.y[2], y1[2], h * k[0][2], h * k[6][2], hd[2], x2) - kHalfPi;
        if (f2 == 0.0) {
          x1 = x2;
          break;
        }
        if ((f2 > 0.0) != (f1 > 0.0)) {
          x0 = x1;
          f0 = f1;
        } else {
          f0 *= 0.5;
        }
        x1 = x2;
        f1 = f2;
        if (fabs(x1 - x0) <= 1e-15 || fabs(f2) <= 1e-15) break;
      }
      sig = x1;
    }
    const double Rc = dense1(r.y[1], y1[1], h * k[0][1], h * k[6][1], hd[1], sig);
    const double thc = dense1(r.y[2], y1[2], h * k[0][2], h * k[6][2], hd[2], sig);
    const double pthc = dense1(r.y[5], y1[5], h * k[0][5], h * k[6][5], hd[5], sig);
    const double cth = cos(thc);
    const double thdot = pthc / (Rc * Rc + m.chi2 * cth * cth);
    const double lamc = r.lam + sig * h;
    if (Rc >= ip.R_cap && Rc <= ip.R_esc && fabs(thdot) >= ip.thdot_min &&
        (!r.cs.have_trusted || lamc - r.cs.lam_last >= ip.dlam_min)) {
      crossed = true;
      sig_out = sig;
      Rc_out = Rc;
      r.cs.ncross++;
      r.cs.lam_last = lamc;
      r.cs.have_trusted = true;
    }
  }
  r.lam += h;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    r.y[i] = y1[i];
    r.f[i] = k[6][i];
  }
  if (reflect_axis(r.y[2], r.y[5], r.y[3])) {
    reflected = true;
    double Wr, Pr;
    geo_rhs(m, r.E, r.ell, r.y[1], r.y[2], r.y[4], r.y[5], r.f, Wr, Pr);
  }
  if (r.y[1] < ip.R_cap) return 2;
  if (r.y[1] > ip.R_esc) return 1;
  r.h = h * (double)step_factor(err, r.rejected);
  r.rejected = false;
  return r.steps >= ip.max_steps ? 3 : 0;
}

__device__ __forceinline__ void save_ckpt(const Ray64& r, Ckpt& c) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    c.y[i] = r.y[i];
    c.f[i] = r.f[i];
  }
  c.h = r.h;
  c.lam = r.lam;
  c.lam_last = r.cs.lam_last;
  c.nacc = r.nacc;
  c.nrej = r.nrej;
  c.steps = r.steps;
  c.ncross = r.cs.ncross;
  c.rejected = r.rejected;
  c.have_trusted = r.cs.have_trusted;
}

__device__ __forceinline__ void load_ckpt(const Ckpt& c, Ray64& r) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    r.y[i] = c.y[i];
    r.f[i] = c.f[i];
  }
  r.h = c.h;
  r.lam = c.lam;
  r.cs.lam_last = c.lam_last;
  r.nacc = c.nacc;
  r.nrej = c.nrej;
  r.steps = c.steps;
  r.cs.ncross = c.ncross;
  r.rejected = c.rejected != 0;
  r.cs.have_trusted = c.have_trusted != 0;
}

using D9 = Dual<9>;  // tangents: R, theta, p_R, p_theta, E, ell, chi, halo1, halo2

// Adjoint of one accepted step (active components R, theta, p_R, p_theta).
// ybar holds the adjoint of y_{n+1} on entry and of y_n on exit; pbar
// accumulates (E, ell, chi, halo1, halo2).
__device__ void adj_step_reverse(const ImgParams& ip, const MetricConsts<D9>& md, double E,
                                 double ell, const double* yn, double h, bool has_cross,
                                 double sig, double Rbar, double* ybar, double* pbar) {
  double kv[7][4];
  double jac[7][4][9];
  const int act[4] = {1, 2, 4, 5};
  for (int s = 0; s < 7; ++s) {
    double Y[4];
    for (int a = 0; a < 4; ++a) {
      double acc = 0.0;
      for (int j = 0; j < s; ++j) acc += kDP.a[s][j] * kv[j][a];
      Y[a] = yn[a] + h * acc;
    }
    D9 d[6], W, P2;
    geo_rhs(md, D9::var(E, 4), D9::var(ell, 5), D9::var(Y[0], 0), D9::var(Y[1], 1),
            D9::var(Y[2], 2), D9::var(Y[3], 3), d, W, P2);
    for (int a = 0; a < 4; ++a) {
      kv[s][a] = d[act[a]].v;
      for (int t = 0; t < 9; ++t) jac[s][a][t] = d[act[a]].d[t];
    }
  }
  double kbar[7][4];
  double ybar_n[4];
  for (int a = 0; a < 4; ++a) {
    ybar_n[a] = 0.0;
    for (int s = 0; s < 7; ++s) kbar[s][a] = 0.0;
  }
  if (has_cross) {
    // dense output y(sig) = c0 y_n + c1 y_{n+1} + c2 h k1 + c3 h k7 + c4 h sum d_j k_j
    const double s = sig, u = 1.0 - sig;
    const double c1 = s * s * (3.0 - 2.0 * s), c0 = 1.0 - c1, c2 = s * u * u, c3 = -s * s * u,
                 c4 = s * s * u * u;
    const double e1 = 6.0 * s * u, e0 = -e1, e2 = u * (1.0 - 3.0 * s), e3 = s * (3.0 * s - 2.0),
                 e4 = 2.0 * s * u * (1.0 - 2.0 * s);
    double y1[2], hd[2];
    for (int a = 0; a < 2; ++a) {
      double acc = 0.0, dd = 0.0;
      for (int j = 0; j < 7; ++j) {
        acc += kDP.b[j] * kv[j][a];
        dd += kDP.d[j] * kv[j][a];
      }
      y1[a] = yn[a] + h * acc;
      hd[a] = h * dd;
    }
    // derivatives of R and theta of the dense output with respect to sigma
    double dq[2];
    for (int a = 0; a < 2; ++a)
      dq[a] = e0 * yn[a] + e1 * y1[a] + e2 * h * kv[0][a] + e3 * h * kv[6][a] + e4 * hd[a];
    const double sbar = Rbar * dq[0];
    const double w[2] = {Rbar, -sbar / dq[1]};  // weights on the R and theta components
    for (int a = 0; a < 2; ++a) {
      ybar_n[a] += w[a] * c0;
      ybar[a] += w[a] * c1;  // adjoint of y_{n+1}
      kbar[0][a] += w[a] * h * c2;
      kbar[6][a] += w[a] * h * c3;
      for (int j = 0; j < 7; ++j) kbar[j][a] += w[a] * h * c4 * kDP.d[j];
    }
  }
  for (int j = 0; j < 7; ++j)
    for (int a = 0; a < 4; ++a) kbar[j][a] += h * kDP.b[j] * ybar[a];
  for (int s = 6; s >= 0; --s) {
    double Yb[4];
    for (int a = 0; a < 4; ++a) {
      double acc = 0.0;
      for (int b = 0; b < 4; ++b) acc += jac[s][b][a] * kbar[s][b];
      Yb[a] = acc;
    }
    for (int t = 0; t < 5; ++t) {
      double acc = 0.0;
      for (int b = 0; b < 4; ++b) acc += jac[s][b][4 + t] * kbar[s][b];
      pbar[t] += acc;
    }
    for (int j = 0; j < s; ++j)
      for (int a = 0; a < 4; ++a) kbar[j][a] += h * kDP.a[s][j] * Yb[a];
    for (int a = 0; a < 4; ++a) ybar_n[a] += Yb[a];
  }
  for (int a = 0; a < 4; ++a) ybar[a] += ybar_n[a];
}

__global__ void __launch_bounds__(128) adjoint_kernel(AdjArgs a) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Ckpt* ck = a.ckpt + gtid * a.max_ckpt;
  const ImgParams& ip = *a.ip;
  const MetricConsts<double> m = metric_consts<double>(ip);
  const MetricConsts<D9> md = metric_dual<9>(ip, 6, 7, 8);
  int64_t ncells[kMaxLevels + 1];
  ncells[0] = a.npix;
  for (int l = 1; l <= kMaxLevels; ++l) {
    unsigned long long c = l <= a.levels ? a.hdr->count[l] : 0ull;
    ncells[l] = (int64_t)(c < (unsigned long long)a.lv[l].cap ? c : (unsigned long long)a.lv[l].cap);
  }
  double gacc[10];
  for (int t = 0; t < 10; ++t) gacc[t] = 0.0;

  while (true) {
    int64_t idx = (int64_t)atomicAdd(a.head, 1ull);
    int level = 0;
    while (level <= kMaxLevels && idx >= ncells[level]) {
      idx -= ncells[level];
      ++level;
    }
    if (level > kMaxLevels || level > a.levels) break;
    // leaf weight and pixel
    uint64_t key;
    double w;
    if (level == 0) {
      key = (uint64_t)idx << 16;
      w = (a.levels > 0 && a.base_child[idx] >= 0) ? 0.0 : 1.0;
    } else {
      key = a.lv[level].key[idx];
      bool leaf = level == a.levels || a.lv[level].child[idx] < 0;
      w = leaf ? 1.0 / (double)(1 << (4 * level)) : 0.0;
    }
    const int64_t pix = (int64_t)(key >> 16);
    const double gI = w * a.Gpix[pix];
    if (gI == 0.0) continue;
    double X, Y;
    cell_centre(ip, key, X, Y);

    // 1. forward replay with checkpoints and crossing records
    Ray64 r;
    ray_init64(ip, m, X, Y, r);
    XRec xr[kMaxCrossAdj];
    int nx = 0;
    double pdir[13];  // direct adjoint of the crossing terms (tangents of D13)
    for (int t = 0; t < 13; ++t) pdir[t] = 0.0;
    int nck = 0;
    bool overflow = false;
    while (true) {
      if (r.nacc % kCkptEvery == 0 && r.nacc / kCkptEvery == nck && !r.rejected) {
        if (nck >= a.max_ckpt) {
          overflow = true;
          break;
        }
        save_ckpt(r, ck[nck++]);
      }
      bool crossed, refl;
      double sig, Rc;
      const double E = r.E, ell = r.ell;
      int term = adj_step(ip, m, r, crossed, sig, Rc, refl);
      if (crossed) {
        D13 Ic;
        double Rb = 0.0;
        if (crossing_intensity_dual(ip, Rc, E, ell, Ic)) {
          Rb = gI * Ic.d[0];
          for (int t = 1; t < 13; ++t) pdir[t] += gI * Ic.d[t];
        }
        if (nx < kMaxCrossAdj) xr[nx++] = XRec{r.nacc - 1, sig, Rb};
        else overflow = true;
      }
      if (term) break;
    }
    if (overflow) {
      atomicCAS(a.status, 0, (int)BH_ERR_WORKSPACE);
      continue;
    }
    if (nx == 0) continue;
    int last = xr[nx - 1].step;  // reverse sweep starts at the last crossing step
    // 2. reverse sweep over checkpoint segments
    double ybar[4] = {0, 0, 0, 0};
    double pbar[5] = {pdir[1], pdir[2], pdir[3], pdir[4], pdir[5]};  // E, ell, chi, h1, h2
    int xi = nx - 1;
    for (int seg = last / kCkptEvery; seg >= 0; --seg) {
      load_ckpt(ck[seg], r);
      const int n0 = seg * kCkptEvery;
      const int n1 = min(n0 + kCkptEvery, last + 1);
      double ys[kCkptEvery][4];
      double hs[kCkptEvery];
      bool rf[kCkptEvery];
      while (r.nacc < n1) {
        const int nb = r.nacc;
        double ya[4] = {r.y[1], r.y[2], r.y[4], r.y[5]};
        const double hh = r.h;
        bool crossed, refl;
        double sig, Rc;
        adj_step(ip, m, r, crossed, sig, Rc, refl);
        if (r.nacc > nb) {
          const int q = nb - n0;
          for (int c = 0; c < 4; ++c) ys[q][c] = ya[c];
          hs[q] = hh;
          rf[q] = refl;
        }
      }
      for (int n = n1 - 1; n >= n0; --n) {
        const int q = n - n0;
        if (rf[q]) {  // reflection applied after step n: theta -> -theta, p_th -> -p_th
          ybar[1] = -ybar[1];
          ybar[3] = -ybar[3];
        }
        bool hc = xi >= 0 && xr[xi].step == n;
        adj_step_reverse(ip, md, r.E, r.ell, ys[q], hs[q], hc, hc ? xr[xi].sig : 0.0,
                         hc ? xr[xi].Rbar : 0.0, ybar, pbar);
        if (hc) --xi;
      }
    }
    // 3. launch: theta_0 = theta_o, p_R = sqrt(g_RR) n^R, p_th = sqrt(g_thth) n^th,
    //    ell = sqrt(g_phph) n^phi, E = N + omega ell (Eqs. 63-74)
    const double d = sqrt(ip.r_obs * ip.r_obs + X * X + Y * Y);
    const double nR = -ip.r_obs / d, nth = -Y / d, nph = -X / d;
    const double ell = ip.sq_gph * nph;
    const double Eb = pbar[0], lb = pbar[1];
    for (int k = 0; k < 4; ++k) {
      const double dell = a.aj.d_sqgph[k] * nph;
      const double dE = a.aj.d_N[k] + a.aj.d_w[k] * ell + ip.zamo_w * dell;
      double gk = ybar[2] * a.aj.d_sqgrr[k] * nR + ybar[3] * a.aj.d_sqgth[k] * nth + lb * dell +
                  Eb * dE + pdir[6] * a.aj.d_Rin[k];
      if (k == 1) gk += ybar[1];
      if (k == 0) gk += pbar[2];
      if (k == 2) gk += pbar[3];
      if (k == 3) gk += pbar[4];
      gacc[k] += gk;
    }
    for (int t = 0; t < 6; ++t) gacc[4 + t] += pdir[7 + t];
  }
  for (int t = 0; t < 10; ++t)
    if (gacc[t] != 0.0) atomicAdd(&a.grad[t], gacc[t]);
}

// --------------------------------------------------------------------------
// Image-level adjoint: dL/dI per pixel.
__global__ void pixel_adjoint_kernel(ImgAdj a) {
  const int64_t n = (int64_t)a.nx * a.ny;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % a.nx), j = (int)(q / a.nx);
    const double x = a.x_min + (i + 0.5) * a.dx, y = a.y_min + (j + 0.5) * a.dy;
    double g = a.dLdI ? (double)a.dLdI[q] : 0.0;
    if (a.C > 0.0)
      g += a.cC * (a.Xc * (x - a.Xc) + a.Yc * (y - a.Yc)) / (a.C * a.S);  // Eqs. (93)-(94)
    const double T = a.FRs + a.FLs;
    if (T != 0.0) {
      const double sgn = x > a.Xc ? 1.0 : (x < a.Xc ? -1.0 : 0.0);
      g += a.cA * (sgn * T - (a.FRs - a.FLs) * fabs(sgn)) / (T * T);  // Eq. (99)
    }
    const int b = (int)floor(sqrt(x * x + y * y) / a.dx);
    for (int t = 0; t < 3; ++t)
      if (b == a.bstar - 1 + t && a.cnt[t] > 0) g += a.cR * a.drho[t] / (double)a.cnt[t];
    const double dA = a.dx * a.dy;
    for (int k = 0; k < 8; ++k) {
      if (a.cV[k] == 0.0 || a.Vabs[k] == 0.0) continue;
      double s, c;
      sincospi(2.0 * (a.uv[2 * k] * x + a.uv[2 * k + 1] * y), &s, &c);
      const double dabs = dA * (a.Vre[k] * c - a.Vim[k] * s) / a.Vabs[k];
      g += a.cV[k] * (dabs - (a.Vabs[k] / a.V0) * dA) / a.V0;        // Eq. (109)
    }
    a.G[q] = g;
  }
}

// Pixel sums needed by the image-level adjoint: S, sum X I, sum Y I.
__global__ void image_moments_kernel(const float* I, ImgAdj a, double* out3) {
  double s = 0, sx = 0, sy = 0;
  const int64_t n = (int64_t)a.nx * a.ny;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % a.nx), j = (int)(q / a.nx);
    const double x = a.x_min + (i + 0.5) * a.dx, y = a.y_min + (j + 0.5) * a.dy, v = I[q];
    s += v;
    sx += x * v;
    sy += y * v;
  }
  atomicAdd(&out3[0], s);
  atomicAdd(&out3[1], sx);
  atomicAdd(&out3[2], sy);
}

// Left / right sums about X_c and the origin-centred radial profile.
__global__ void image_profile_kernel(const float* I, ImgAdj a, double* lr, double* hs,
                                     unsigned long long* hc) {
  const int64_t n = (int64_t)a.nx * a.ny;
  double r = 0, l = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % a.nx), j = (int)(q / a.nx);
    const double x = a.x_min + (i + 0.5) * a.dx, y = a.y_min + (j + 0.5) * a.dy, v = I[q];
    if (x > a.Xc) r += v;
    if (x < a.Xc) l += v;
    const int b = (int)floor(sqrt(x * x + y * y) / a.dx);
    if (b >= 0 && b < a.nbins) {
      atomicAdd(&hs[b], v);
      atomicAdd(&hc[b], 1ull);
    }
  }
  atomicAdd(&lr[0], r);
  atomicAdd(&lr[1], l);
}



cudaError_t launch_adjoint(const AdjArgs& a, int blocks, int threads, cudaStream_t s) {
  adjoint_kernel<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_pixel_adjoint(const ImgAdj& a, cudaStream_t s) {
  pixel_adjoint_kernel<<<608, 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_image_moments(const float* I, const ImgAdj& a, double* out3, cudaStream_t s) {
  image_moments_kernel<<<608, 256, 0, s>>>(I, a, out3);
  return cudaGetLastError();
}
cudaError_t launch_image_profile(const float* I, const ImgAdj& a, double* lr, double* hs,
                                 unsigned long long* hc, cudaStream_t s) {
  image_profile_kernel<<<608, 256, 0, s>>>(I, a, lr, hs, hc);
  return cudaGetLastError();
}

}  // namespace bhrt
