/*
 * bh_oracle.c -- plain, slow, FP64 CPU oracle for the ray-tracing path of
 * "Adaptive ray tracing, image diagnostics, and photon ring signatures of
 * rotating dark-matter-dressed black holes".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it is used by tests/, by the smoke check and by the CPU
 * baseline leg of bench.py.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * Every routine follows the paper's definitions literally, one ray at a time,
 * in IEEE double precision, with FMA contraction disabled at build time.
 * Equation numbers are the paper's, counted in order of appearance.  Where the
 * paper is silent (integrator, tolerances, refinement rule, emissivity
 * constants), the routine implements a documented reading and says so.
 *
 * Parity pins: see tests/test_oracle_*.py.  Parity unpinned: the absolute
 * Table 1/2 numbers (the paper's emissivity constants and screen are not
 * printed), so nothing here claims to reproduce them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Problem description (all dimensionless, M = 1; Sec. 2, Eq. 1).            */
/* ------------------------------------------------------------------------ */
enum { ORC_KERR = 0, ORC_EINASTO = 1, ORC_CNFW = 2 };

typedef struct {
  int32_t metric;      /* ORC_KERR / ORC_EINASTO / ORC_CNFW               */
  int32_t r_in_mode;   /* 0: R_in = r_ISCO, 1: R_in = R_+ + dR_in (Eq. 87) */
  int32_t levels;      /* screen refinement levels, 0..3                  */
  int32_t max_steps;   /* attempted DP5 steps before "undetermined"       */
  int32_t nx, ny;      /* base screen resolution                          */
  int32_t volumetric;  /* 0: thin-disk events; 1: the volumetric integral
                          I = int g^3 j(R, theta) dlambda (Eq. 88)        */
  int32_t pad1;
  double chi;          /* spin a/M (Eq. 1)                                */
  double lam_E;        /* Einasto scale (Eq. 10)                          */
  double eta;          /* cored-NFW 4 pi rho0 r0^2 (Eq. 14)               */
  double lam_c;        /* cored-NFW core radius (Eq. 12)                  */
  double r_obs;        /* observer radius R_o                             */
  double incl;         /* observer inclination theta_o [rad]              */
  double x_min, x_max, y_min, y_max; /* screen extent                     */
  double j0, p, R_s, sigma_in, sigma_out, R_out, dR_in, H0, h; /* Eqs. 83-87 */
  double rtol, atol;   /* DP5 tolerances (reading)                        */
  double cap_factor;   /* capture at R < cap_factor * R_+  (Eq. 75)       */
  double esc_factor;   /* escape at R > esc_factor * R_o                  */
  double thetadot_min; /* trusted-crossing |dtheta/dlambda| floor (Sec 4.2)*/
  double dlambda_min;  /* repeated-crossing affine gap (Sec 4.2)          */
} orc_problem;

/* Per-ray record. */
typedef struct {
  int32_t status;      /* 0 escaped, 1 captured, 2 undetermined, <0 error */
  int32_t ncross;      /* trusted equatorial crossings (all orders)       */
  int32_t n_accept, n_reject;
  double I_tot;        /* sum over all trusted crossings of g^3 j         */
  double I_n[3];       /* contribution of crossing n = 0, 1, 2            */
  double R_em[3], phi_em[3], T_em[3], g[3], thdot[3], lam_cross[3];
  double R_min, R_final, lam_final;
  double h_drift;      /* max over accepted steps of |2H| / scale        */
  double E, ell;       /* constants of motion (Eq. 48)                    */
  double K0, K_final;  /* Carter-like separation constant, start / end    */
  double near_thdot;   /* min over detected crossings | |thdot|/thdot_min - 1 | */
  double near_dlam;    /* min over detected crossings | dlam/dlambda_min - 1 |  */
} orc_ray;

/* ------------------------------------------------------------------------ */
/* Lapse functions, Sec. 2.1.                                               */
/* ------------------------------------------------------------------------ */

/* H_i(R): Kerr seed 1 - 2/R (Sec. 2.2, Kerr limit); Einasto Eq. (9);
 * cored-NFW Eq. (13). */
double orc_H(const orc_problem* P, double R) {
  if (P->metric == ORC_EINASTO) {
    double l = P->lam_E;
    return 1.0 - 2.0 / R + (2.0 / R + 2.0 / l + R / (l * l)) * exp(-R / l);
  }
  if (P->metric == ORC_CNFW) {
    double lc = P->lam_c;
    double S = P->eta * lc * (1.0 / (R + lc) - (2.0 / R) * log1p(R / lc));
    return exp(S) - 2.0 / R;
  }
  return 1.0 - 2.0 / R;
}

/* dH/dR, differentiated by hand from Eqs. (9) and (13). */
double orc_dH(const orc_problem* P, double R) {
  if (P->metric == ORC_EINASTO) {
    double l = P->lam_E;
    double e = exp(-R / l);
    double poly = 2.0 / R + 2.0 / l + R / (l * l);
    double dpoly = -2.0 / (R * R) + 1.0 / (l * l);
    return 2.0 / (R * R) + dpoly * e - poly * e / l;
  }
  if (P->metric == ORC_CNFW) {
    double lc = P->lam_c;
    double S = P->eta * lc * (1.0 / (R + lc) - (2.0 / R) * log1p(R / lc));
    double dS = P->eta * lc *
                (-1.0 / ((R + lc) * (R + lc)) + (2.0 / (R * R)) * log1p(R / lc) -
                 2.0 / (R * (R + lc)));
    return exp(S) * dS + 2.0 / (R * R);
  }
  return 2.0 / (R * R);
}

/* Effective mass function mu_i = (R/2)(1 - H_i), Eq. (15). */
double orc_mu(const orc_problem* P, double R) { return 0.5 * R * (1.0 - orc_H(P, R)); }

/* Delta_i(R) = R^2 H_i + chi^2, Eq. (25). */
double orc_Delta(const orc_problem* P, double R) {
  return R * R * orc_H(P, R) + P->chi * P->chi;
}

/* ------------------------------------------------------------------------ */
/* Rotating metric, Sec. 2.2 (Eqs. 23-31) and its inverse, Sec. 3.1         */
/* (Eqs. 49-53).  Index order (T, R, theta, phi).                           */
/* ------------------------------------------------------------------------ */
void orc_metric(const orc_problem* P, double R, double th, double g[16]) {
  double chi = P->chi, c = cos(th), s = sin(th), s2 = s * s;
  double Sig = R * R + chi * chi * c * c;           /* Eq. (23) */
  double F = R * R * (1.0 - orc_H(P, R));           /* Eq. (24) */
  double D = orc_Delta(P, R);                       /* Eq. (25) */
  memset(g, 0, 16 * sizeof(double));
  g[0] = -(1.0 - F / Sig);                          /* Eq. (27) */
  g[3] = g[12] = -chi * F * s2 / Sig;               /* Eq. (28) */
  g[5] = Sig / D;                                   /* Eq. (29) */
  g[10] = Sig;                                      /* Eq. (30) */
  g[15] = s2 * (R * R + chi * chi + chi * chi * F * s2 / Sig); /* Eq. (31) */
}

/* d g_{mu nu} / dR, by hand from Eqs. (27)-(31).  Used for Omega, Eq. (91). */
void orc_dmetric_dR(const orc_problem* P, double R, double th, double dg[16]) {
  double chi = P->chi, c = cos(th), s = sin(th), s2 = s * s;
  double H = orc_H(P, R), dH = orc_dH(P, R);
  double Sig = R * R + chi * chi * c * c, dSig = 2.0 * R;
  double F = R * R * (1.0 - H), dF = 2.0 * R * (1.0 - H) - R * R * dH;
  double D = R * R * H + chi * chi, dD = 2.0 * R * H + R * R * dH;
  double FoS = F / Sig, dFoS = (dF * Sig - F * dSig) / (Sig * Sig);
  memset(dg, 0, 16 * sizeof(double));
  dg[0] = dFoS;
  dg[3] = dg[12] = -chi * s2 * dFoS;
  dg[5] = (dSig * D - Sig * dD) / (D * D);
  dg[10] = dSig;
  dg[15] = s2 * (2.0 * R + chi * chi * s2 * dFoS);
}

/* Inverse metric, Eqs. (49)-(53). */
void orc_metric_inv(const orc_problem* P, double R, double th, double gi[16]) {
  double chi = P->chi, c = cos(th), s = sin(th), s2 = s * s;
  double Sig = R * R + chi * chi * c * c;
  double F = R * R * (1.0 - orc_H(P, R));
  double D = orc_Delta(P, R);
  double A = (R * R + chi * chi) * (R * R + chi * chi) - chi * chi * D * s2;
  memset(gi, 0, 16 * sizeof(double));
  gi[0] = -A / (Sig * D);                           /* Eq. (49) */
  gi[3] = gi[12] = -chi * F / (Sig * D);            /* Eq. (50) */
  gi[5] = D / Sig;                                  /* Eq. (51) */
  gi[10] = 1.0 / Sig;                               /* Eq. (52) */
  gi[15] = (D - chi * chi * s2) / (Sig * D * s2);   /* Eq. (53) */
}

/* Partial derivatives of the inverse metric with respect to R and theta,
 * by the quotient rule applied to Eqs. (49)-(53).  These feed Eqs. (61)-(62). */
void orc_dmetric_inv(const orc_problem* P, double R, double th, double dR[16],
                     double dth[16]) {
  double chi = P->chi, c = cos(th), s = sin(th), s2 = s * s, x2 = chi * chi;
  double H = orc_H(P, R), dH = orc_dH(P, R);
  double Sig = R * R + x2 * c * c;
  double F = R * R * (1.0 - H);
  double D = R * R * H + x2;
  double Sig_R = 2.0 * R, Sig_t = -2.0 * x2 * c * s;
  double F_R = 2.0 * R * (1.0 - H) - R * R * dH;
  double D_R = 2.0 * R * H + R * R * dH;
  double s2_t = 2.0 * s * c;
  double A = (R * R + x2) * (R * R + x2) - x2 * D * s2;
  double A_R = 4.0 * R * (R * R + x2) - x2 * D_R * s2;
  double A_t = -x2 * D * s2_t;
  double SD = Sig * D, SD_R = Sig_R * D + Sig * D_R, SD_t = Sig_t * D;
  memset(dR, 0, 16 * sizeof(double));
  memset(dth, 0, 16 * sizeof(double));
  /* g^TT = -A/(Sig D) */
  dR[0] = -(A_R * SD - A * SD_R) / (SD * SD);
  dth[0] = -(A_t * SD - A * SD_t) / (SD * SD);
  /* g^Tphi = -chi F/(Sig D) */
  dR[3] = dR[12] = -chi * (F_R * SD - F * SD_R) / (SD * SD);
  dth[3] = dth[12] = chi * F * SD_t / (SD * SD);
  /* g^RR = D/Sig */
  dR[5] = (D_R * Sig - D * Sig_R) / (Sig * Sig);
  dth[5] = -D * Sig_t / (Sig * Sig);
  /* g^thth = 1/Sig */
  dR[10] = -Sig_R / (Sig * Sig);
  dth[10] = -Sig_t / (Sig * Sig);
  /* g^phph = (D - chi^2 s2)/(Sig D s2) */
  {
    double N = D - x2 * s2, N_R = D_R, N_t = -x2 * s2_t;
    double Q = Sig * D * s2, Q_R = SD_R * s2, Q_t = Sig_t * D * s2 + Sig * D * s2_t;
    dR[15] = (N_R * Q - N * Q_R) / (Q * Q);
    dth[15] = (N_t * Q - N * Q_t) / (Q * Q);
  }
}

/* 2H = g^{mu nu} p_mu p_nu, Eq. (54).  p = (p_T, p_R, p_th, p_ph). */
double orc_two_hamiltonian(const orc_problem* P, double R, double th, const double p[4]) {
  double gi[16];
  orc_metric_inv(P, R, th, gi);
  double s = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) s += gi[4 * a + b] * p[a] * p[b];
  return s;
}

/* Hamilton's equations, Eqs. (46)-(47) in the form of Eqs. (57)-(62).
 * State y = (T, R, theta, phi, p_R, p_theta); constants E = -p_T, ell = p_phi
 * (Eq. 48).  dy receives d/dlambda of the state. */
void orc_rhs(const orc_problem* P, double E, double ell, const double y[6], double dy[6]) {
  double R = y[1], th = y[2];
  double p[4] = {-E, y[4], y[5], ell};
  double gi[16], gR[16], gt[16];
  orc_metric_inv(P, R, th, gi);
  orc_dmetric_inv(P, R, th, gR, gt);
  dy[0] = gi[0] * p[0] + gi[3] * p[3];              /* Eq. (57) */
  dy[1] = gi[5] * p[1];                             /* Eq. (59) */
  dy[2] = gi[10] * p[2];                            /* Eq. (60) */
  dy[3] = gi[12] * p[0] + gi[15] * p[3];            /* Eq. (58) */
  double sR = 0.0, st = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      sR += gR[4 * a + b] * p[a] * p[b];
      st += gt[4 * a + b] * p[a] * p[b];
    }
  dy[4] = -0.5 * sR;                                /* Eq. (61) */
  dy[5] = -0.5 * st;                                /* Eq. (62) */
}

/* Carter-like separation constant read off the separated Hamilton-Jacobi
 * equation of Sec. 3.1 (Eq. 56): K = p_theta^2 + (ell/sin - chi E sin)^2. */
double orc_carter(const orc_problem* P, double E, double ell, double th, double pth) {
  double s = sin(th);
  double q = ell / s - P->chi * E * s;
  return pth * pth + q * q;
}

/* ------------------------------------------------------------------------ */
/* Horizon and extremality, Sec. 2.3.                                       */
/* ------------------------------------------------------------------------ */

/* R_+ = largest root of Delta_i(R) = 0, Eq. (33).  Scan downward from
 * R = 50 in steps of 1e-3 until Delta changes sign, then bisect to the
 * last representable bracket.  Returns 0 on success, 1 if no horizon. */
int orc_horizon(const orc_problem* P, double* r_plus) {
  const double step = 1e-3;
  double hi = 50.0, fhi = orc_Delta(P, hi);
  if (!(fhi > 0.0)) return 1;
  for (long k = 1;; ++k) {
    double lo = 50.0 - k * step;
    if (lo <= 1e-6) return 1;
    double flo = orc_Delta(P, lo);
    if (flo <= 0.0) {
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_Delta(P, mid) > 0.0) hi = mid; else lo = mid;
      }
      *r_plus = hi;
      return 0;
    }
    hi = lo;
  }
}

/* Extremal spin, Eqs. (34)-(37): the horizon exists iff chi^2 <= -R^2 H(R)
 * somewhere, so chi_e^2 = max_R [-R^2 H(R)], attained where Eq. (36) holds.
 * Dense scan on (1e-4, 50] then golden-section refinement.  Returns chi_e
 * (0 if -R^2 H never becomes positive) and the extremal radius in *R_e. */
double orc_extremal_spin(const orc_problem* P0, double* R_e) {
  orc_problem P = *P0;
  P.chi = 0.0;
  double best = -INFINITY, Rb = 0.0;
  for (long k = 1; k <= 500000; ++k) {
    double R = 1e-4 * k;
    double v = -R * R * orc_H(&P, R);
    if (v > best) { best = v; Rb = R; }
  }
  double a = Rb - 1e-4, b = Rb + 1e-4;
  const double gr = 0.5 * (sqrt(5.0) - 1.0);
  for (int it = 0; it < 200; ++it) {
    double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
    double f1 = -x1 * x1 * orc_H(&P, x1), f2 = -x2 * x2 * orc_H(&P, x2);
    if (f1 > f2) b = x2; else a = x1;
  }
  double Rx = 0.5 * (a + b);
  double v = -Rx * Rx * orc_H(&P, Rx);
  if (R_e) *R_e = Rx;
  return v > 0.0 ? sqrt(v) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Circular equatorial emitters, Sec. 5.2, Eqs. (90)-(91).                  */
/* ------------------------------------------------------------------------ */

/* Omega (Eq. 91) and u^T (normalisation u.u = -1) at theta = pi/2.
 * Returns 0 when the prograde circular orbit exists and is timelike. */
int orc_circular(const orc_problem* P, double R, double* Omega, double* uT) {
  double g[16], dg[16];
  orc_metric(P, R, 0.5 * M_PI, g);
  orc_dmetric_dR(P, R, 0.5 * M_PI, dg);
  double disc = dg[3] * dg[3] - dg[0] * dg[15];
  if (!(disc >= 0.0) || dg[15] == 0.0) return 1;
  double W = (-dg[3] + sqrt(disc)) / dg[15];
  double norm = -(g[0] + 2.0 * W * g[3] + W * W * g[15]);
  if (!(norm > 0.0)) return 1;
  *Omega = W;
  *uT = 1.0 / sqrt(norm);
  return 0;
}

/* Specific energy of the prograde circular orbit, -u_T. */
static double orc_circ_energy(const orc_problem* P, double R, int* ok) {
  double W, uT, g[16];
  if (orc_circular(P, R, &W, &uT)) { *ok = 0; return INFINITY; }
  orc_metric(P, R, 0.5 * M_PI, g);
  *ok = 1;
  return -uT * (g[0] + W * g[3]);
}

/* r_ISCO as the minimiser of the prograde circular-orbit energy (reading:
 * the paper takes R_in from Eq. 87; the ISCO default is a documented
 * reading).  Dense scan on (R_+, 60] in steps of 1e-3, golden-section
 * refinement.  Returns 0 on success. */
int orc_isco(const orc_problem* P, double* r_isco) {
  double rp;
  if (orc_horizon(P, &rp)) return 1;
  double best = INFINITY, Rb = 0.0;
  for (long k = 1; k <= 60000; ++k) {
    double R = rp + 1e-3 * k;
    if (R > 60.0) break;
    int ok;
    double e = orc_circ_energy(P, R, &ok);
    if (ok && e < best) { best = e; Rb = R; }
  }
  if (!isfinite(best)) return 1;
  double a = Rb - 1e-3, b = Rb + 1e-3;
  const double gr = 0.5 * (sqrt(5.0) - 1.0);
  for (int it = 0; it < 200; ++it) {
    double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
    int o1, o2;
    double f1 = orc_circ_energy(P, x1, &o1), f2 = orc_circ_energy(P, x2, &o2);
    if (f1 < f2) b = x2; else a = x1;
  }
  *r_isco = 0.5 * (a + b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Emissivity, Sec. 5.1, Eqs. (83)-(86), general (R, theta) form.            */
/* ------------------------------------------------------------------------ */
double orc_emissivity(const orc_problem* P, double R_in, double R, double th) {
  double rho = R * sin(th), z = R * cos(th);
  double Hd = P->H0 + P->h * rho;                                   /* Eq. (84) */
  double Tin = 0.5 * (1.0 + tanh((rho - R_in) / P->sigma_in));      /* Eq. (85) */
  double Tout = 0.5 * (1.0 - tanh((rho - P->R_out) / P->sigma_out));/* Eq. (86) */
  double vert = (z == 0.0) ? 1.0 : exp(-z * z / (2.0 * Hd * Hd));
  return P->j0 * pow(rho / R_in, -P->p) * exp(-(rho - R_in) / P->R_s) * vert * Tin *
         Tout;                                                       /* Eq. (83) */
}

/* ------------------------------------------------------------------------ */
/* Observer tetrad and launch, Sec. 3.2, Eqs. (63)-(74).                    */
/* ------------------------------------------------------------------------ */

/* Builds the ZAMO frame at (R_o, theta_o), the screen direction of pixel
 * (X, Y), the contravariant momentum (Eq. 73, E_loc = 1) and lowers it with
 * g_{mu nu} (Eq. 74).  Outputs: y0 (state), E = -p_T, ell = p_phi, and the
 * observer four-velocity u_o^mu (for the redshift numerator, Eq. 89). */
void orc_launch(const orc_problem* P, double X, double Y, double y0[6], double* E,
                double* ell, double u_o[4], double p_up[4]) {
  double Ro = P->r_obs, tho = P->incl, g[16];
  orc_metric(P, Ro, tho, g);
  double w = -g[3] / g[15];                                          /* Eq. (63) */
  double N = sqrt(-(g[0] + 2.0 * w * g[3] + w * w * g[15]));         /* Eq. (65) */
  double u[4] = {1.0 / N, 0.0, 0.0, w / N};                         /* Eq. (64) */
  double eR[4] = {0.0, 1.0 / sqrt(g[5]), 0.0, 0.0};                 /* Eq. (66) */
  double et[4] = {0.0, 0.0, 1.0 / sqrt(g[10]), 0.0};                /* Eq. (67) */
  double ep[4] = {0.0, 0.0, 0.0, 1.0 / sqrt(g[15])};                /* Eq. (68) */
  double d = sqrt(Ro * Ro + X * X + Y * Y);
  double nR = -Ro / d, nt = -Y / d, np = -X / d;                    /* Eqs. (70)-(72) */
  double pu[4], pl[4];
  for (int m = 0; m < 4; ++m) pu[m] = u[m] + nR * eR[m] + nt * et[m] + np * ep[m]; /* (73) */
  for (int m = 0; m < 4; ++m) {
    pl[m] = 0.0;
    for (int n = 0; n < 4; ++n) pl[m] += g[4 * m + n] * pu[n];      /* Eq. (74) */
  }
  y0[0] = 0.0; y0[1] = Ro; y0[2] = tho; y0[3] = 0.0; y0[4] = pl[1]; y0[5] = pl[2];
  *E = -pl[0];
  *ell = pl[3];
  if (u_o) for (int m = 0; m < 4; ++m) u_o[m] = u[m];
  if (p_up) for (int m = 0; m < 4; ++m) p_up[m] = pu[m];
}

/* ------------------------------------------------------------------------ */
/* Dormand-Prince 5(4) (Dormand & Prince 1980), FSAL, with the 4th-order     */
/* continuous extension (Shampine 1986; Hairer-Norsett-Wanner, Solving ODEs  */
/* I, Sec. II.6).  The paper names no integrator; this is the reading.       */
/* ------------------------------------------------------------------------ */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double DP_B[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784,
                               11.0 / 84, 0};
static const double DP_BS[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};
static const double DP_D[7] = {-12715105075.0 / 11282082432.0, 0,
                               87487479700.0 / 32700410799.0,
                               -10690763975.0 / 1880347072.0,
                               701980252875.0 / 199316789632.0,
                               -1453857185.0 / 822651844.0,
                               69997945.0 / 29380423.0};

typedef void (*orc_fn)(void* ctx, const double* y, double* dy);

#define ORC_NMAX 8

/* One DP5 trial step of size h from (y0, k1 = f(y0)).  Fills k[7][n] (k[0]
 * must hold f(y0) on entry), y1 and the embedded error vector.  Returns 0,
 * or 1 if a stage evaluation reported an invalid state (ok flag). */
typedef int (*orc_valid_fn)(void* ctx, const double* y);

static int orc_dp5_trial(orc_fn f, orc_valid_fn valid, void* ctx, int n, const double* y0,
                         double h, double k[7][ORC_NMAX], double* y1, double* err) {
  double ys[ORC_NMAX];
  for (int s = 1; s < 7; ++s) {
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int j = 0; j < s; ++j) acc += DP_A[s][j] * k[j][i];
      ys[i] = y0[i] + h * acc;
    }
    if (valid && !valid(ctx, ys)) return 1;
    f(ctx, ys, k[s]);
    for (int i = 0; i < n; ++i)
      if (!isfinite(k[s][i])) return 1;
  }
  for (int i = 0; i < n; ++i) {
    double a5 = 0.0, a4 = 0.0;
    for (int j = 0; j < 7; ++j) { a5 += DP_B[j] * k[j][i]; a4 += DP_BS[j] * k[j][i]; }
    y1[i] = y0[i] + h * a5;
    err[i] = h * (a5 - a4);
  }
  return 0;
}

/* Error norm: RMS over components of err_i / (atol + rtol max(|y0_i|, |y1_i|)). */
static double orc_err_norm(int n, const double* y0, const double* y1, const double* err,
                           double rtol, double atol) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double sc = atol + rtol * fmax(fabs(y0[i]), fabs(y1[i]));
    double q = err[i] / sc;
    s += q * q;
  }
  return sqrt(s / n);
}

/* Dense output y(x0 + sigma h), sigma in [0, 1]. */
static void orc_dense(int n, const double* y0, const double* y1, double h,
                      double k[7][ORC_NMAX], double sigma, double* out) {
  for (int i = 0; i < n; ++i) {
    double r2 = y1[i] - y0[i];
    double r3 = h * k[0][i] - r2;
    double r4 = r2 - h * k[6][i] - r3;
    double dd = 0.0;
    for (int j = 0; j < 7; ++j) dd += DP_D[j] * k[j][i];
    double r5 = h * dd;
    out[i] = y0[i] + sigma * (r2 + (1.0 - sigma) * (r3 + sigma * (r4 + (1.0 - sigma) * r5)));
  }
}

/* Hairer-Wanner starting step (Solving ODEs I, Sec. II.4), order 4 error
 * estimator (exponent 1/5). */
static double orc_initial_step(orc_fn f, void* ctx, int n, const double* y0, const double* f0,
                               double rtol, double atol) {
  double d0 = 0, d1 = 0, sc[ORC_NMAX];
  for (int i = 0; i < n; ++i) {
    sc[i] = atol + rtol * fabs(y0[i]);
    d0 += (y0[i] / sc[i]) * (y0[i] / sc[i]);
    d1 += (f0[i] / sc[i]) * (f0[i] / sc[i]);
  }
  d0 = sqrt(d0 / n); d1 = sqrt(d1 / n);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  double y1[ORC_NMAX], f1[ORC_NMAX];
  for (int i = 0; i < n; ++i) y1[i] = y0[i] + h0 * f0[i];
  f(ctx, y1, f1);
  double d2 = 0;
  for (int i = 0; i < n; ++i) { double q = (f1[i] - f0[i]) / sc[i]; d2 += q * q; }
  d2 = sqrt(d2 / n) / h0;
  double m = fmax(d1, d2);
  double h1 = (m <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / m, 1.0 / 5.0);
  return fmin(100.0 * h0, h1);
}

/* Step-size factor after a trial with error norm e (reading: safety 0.9,
 * clamp [0.2, 10], no growth right after a rejection). */
static double orc_step_factor(double e, int after_reject) {
  double fac = (e == 0.0) ? 10.0 : 0.9 * pow(e, -0.2);
  if (fac < 0.2) fac = 0.2;
  if (fac > 10.0) fac = 10.0;
  if (after_reject && fac > 1.0) fac = 1.0;
  return fac;
}

/* Generic fixed-endpoint driver for textbook ODE tests: integrates from x0
 * to x1 (> x0) and returns the number of accepted steps, or -1. */
typedef struct { int kind; double w; } orc_test_ode;

static void orc_test_rhs(void* ctx, const double* y, double* dy) {
  orc_test_ode* o = (orc_test_ode*)ctx;
  if (o->kind == 0) { dy[0] = y[0]; }                    /* y' = y            */
  else if (o->kind == 1) { dy[0] = y[1]; dy[1] = -o->w * o->w * y[0]; } /* oscillator */
  else { /* Kepler, (x, y, vx, vy) */
    double r = sqrt(y[0] * y[0] + y[1] * y[1]), r3 = r * r * r;
    dy[0] = y[2]; dy[1] = y[3]; dy[2] = -y[0] / r3; dy[3] = -y[1] / r3;
  }
}

int orc_dp5_solve(int kind, double w, int n, double* y, double x0, double x1, double rtol,
                  double atol, int max_steps) {
  orc_test_ode o = {kind, w};
  double k[7][ORC_NMAX], ynew[ORC_NMAX], err[ORC_NMAX];
  orc_test_rhs(&o, y, k[0]);
  double h = orc_initial_step(orc_test_rhs, &o, n, y, k[0], rtol, atol);
  double x = x0;
  int acc = 0, rej = 0;
  for (int it = 0; it < max_steps; ++it) {
    int last = 0;
    if (x + h >= x1) { h = x1 - x; last = 1; }
    orc_dp5_trial(orc_test_rhs, NULL, &o, n, y, h, k, ynew, err);
    double e = orc_err_norm(n, y, ynew, err, rtol, atol);
    if (e <= 1.0) {
      x = last ? x1 : x + h;
      for (int i = 0; i < n; ++i) { y[i] = ynew[i]; k[0][i] = k[6][i]; }
      ++acc;
      if (last) return acc;
      h *= orc_step_factor(e, rej);
      rej = 0;
    } else {
      h *= orc_step_factor(e, 1);
      rej = 1;
    }
  }
  return -1;
}

/* One step + dense output exposed for tests against an independent DP5
 * implementation: advances (y, f) by one trial step of size h and returns
 * the dense output at the requested sigmas. */
int orc_dp5_step_dense(int kind, double w, int n, const double* y0, double h, double* y1,
                       double* err, int nsig, const double* sig, double* dense) {
  orc_test_ode o = {kind, w};
  double k[7][ORC_NMAX];
  orc_test_rhs(&o, y0, k[0]);
  if (orc_dp5_trial(orc_test_rhs, NULL, &o, n, y0, h, k, y1, err)) return 1;
  for (int s = 0; s < nsig; ++s) orc_dense(n, y0, y1, h, k, sig[s], dense + s * n);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Ray tracing: Sec. 3.3 (classification) and Sec. 4.2-4.3 (crossings,     */
/* transfer maps), Sec. 5.2 (redshift, intensity).                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_problem* P;
  double E, ell;
  double num;    /* -p.u_obs (Eq. 89)                                     */
  double R_in;   /* inner disk edge (Eq. 87 or r_ISCO)                   */
} orc_geo_ctx;

/* Source of the volumetric intensity (Eq. 88): g^3 j(R, theta) with the
 * emissivity of Eqs. (83)-(86) at (R, theta) and, as the reading of the
 * emitter's motion off the plane, the circular emitter of Eqs. (90)-(91) at
 * the cylindrical radius rho = R sin(theta) of the equatorial metric; zero
 * where no timelike circular orbit exists there. */
static double orc_vol_source(const orc_geo_ctx* g, double R, double th) {
  /* a trial stage past the polar axis (theta < 0 or > pi) is the point at
   * the mirrored angle: same rho = R |sin theta| and z^2 */
  double thr = th < 0.0 ? -th : (th > M_PI ? 2.0 * M_PI - th : th);
  double rho = R * sin(thr), W, uT;
  if (!(rho > 0.0) || orc_circular(g->P, rho, &W, &uT) != 0) return 0.0;
  double gfac = g->num / (-uT * ((-g->E) + W * g->ell));
  return gfac * gfac * gfac * orc_emissivity(g->P, g->R_in, R, thr);
}

/* Volumetric mode only (reading): a step that may come within 5 H(rho) of
 * the equatorial plane advances z = R cos(theta) by at most H(rho) / 2, so
 * that the stages sample the Gaussian layer of Eq. (83) however thin it is
 * (error control alone can step over a layer that no stage lands in). */
static double orc_layer_cap(const orc_problem* P, const double* y, const double* f, double h) {
  double c = cos(y[2]), s = sin(y[2]);
  double z = y[1] * c, zd = f[1] * c - y[1] * s * f[2];
  double Hc = P->H0 + P->h * fabs(y[1] * s);               /* Eq. (84), rho = R |sin| */
  if (fabs(zd) > 0.0 && fabs(z) - fabs(zd) * h < 5.0 * Hc) {
    double cap = 0.5 * Hc / fabs(zd);
    if (h > cap) h = cap;
  }
  return h;
}

/* Hamilton's equations (Eqs. 57-62); in volumetric mode a seventh
 * component carries the accumulated intensity, d I / d lambda = g^3 j. */
static void orc_geo_rhs(void* c, const double* y, double* dy) {
  orc_geo_ctx* g = (orc_geo_ctx*)c;
  orc_rhs(g->P, g->E, g->ell, y, dy);
  if (g->P->volumetric) dy[6] = orc_vol_source(g, y[1], y[2]);
}

/* A stage is admissible only outside the horizon (Delta > 0); otherwise
 * the trial step is rejected and halved.  theta may leave (0, pi) inside a
 * step: the equations continue smoothly through the polar axis, and the
 * accepted state is reflected back (reading; see orc_trace_ray). */
static int orc_geo_valid(void* c, const double* y) {
  orc_geo_ctx* g = (orc_geo_ctx*)c;
  if (!(y[1] > 0.0) || !isfinite(y[1])) return 0;
  if (!(orc_Delta(g->P, y[1]) > 0.0)) return 0;
  for (int i = 0; i < 6; ++i) if (!isfinite(y[i])) return 0;
  return 1;
}

typedef struct {
  double r_plus, R_in, R_cap, R_esc;
} orc_geom;

int orc_geometry_setup(const orc_problem* P, orc_geom* G) {
  if (orc_horizon(P, &G->r_plus)) return 1;
  if (P->r_in_mode == 0) {
    if (orc_isco(P, &G->R_in)) return 2;
  } else {
    G->R_in = G->r_plus + P->dR_in;                  /* Eq. (87) */
  }
  G->R_cap = P->cap_factor * G->r_plus;
  G->R_esc = P->esc_factor * P->r_obs;
  return 0;
}

/* Integrate one backward ray from screen point (X, Y).
 * Optional instrumentation for gradient checks (test use):
 *   hrec != NULL: the accepted step sizes are written to hrec[0..hcap) and
 *                 their number to *nrec;
 *   hplay != NULL: "frozen" replay of nplay accepted steps of the given sizes
 *                 (no error control, no early termination): the map from
 *                 parameters to results along a fixed step sequence, whose
 *                 finite differences are smooth. */
static int orc_trace_ray_core(const orc_problem* P, const orc_geom* G, double X, double Y,
                              orc_ray* out, double* hrec, int hcap, int* nrec,
                              const double* hplay, int nplay) {
  memset(out, 0, sizeof(*out));
  out->near_thdot = INFINITY;
  out->near_dlam = INFINITY;
  double y[7], u_o[4], E, ell;
  orc_launch(P, X, Y, y, &E, &ell, u_o, NULL);
  out->E = E;
  out->ell = ell;
  out->K0 = orc_carter(P, E, ell, y[2], y[5]);
  /* Redshift numerator -p.u_obs (Eq. 89); equals E_loc = 1 by construction. */
  double num = -((-E) * u_o[0] + ell * u_o[3]);

  orc_geo_ctx ctx = {P, E, ell, num, G->R_in};
  /* reading: in volumetric mode the intensity is a seventh ODE component,
   * integrated by the same Dormand-Prince steps and included in the error
   * norm (RMS over the seven components) */
  const int nc = P->volumetric ? 7 : 6;
  double k[7][ORC_NMAX], y1[7], err[7];
  y[6] = 0.0;
  orc_geo_rhs(&ctx, y, k[0]);
  double h = orc_initial_step(orc_geo_rhs, &ctx, nc, y, k[0], P->rtol, P->atol);
  if (P->volumetric) h = orc_layer_cap(P, y, k[0], h);
  double lam = 0.0, lam_last = -INFINITY;
  int rejected = 0, have_trusted = 0;
  out->R_min = y[1];
  const double half_pi = 0.5 * M_PI;
  out->status = 2;

  if (nrec) *nrec = 0;
  for (int it = 0; it < P->max_steps; ++it) {
    if (hplay) {
      if (out->n_accept >= nplay) break;
      h = hplay[out->n_accept];
    }
    int bad = orc_dp5_trial(orc_geo_rhs, orc_geo_valid, &ctx, nc, y, h, k, y1, err);
    if (bad && !hplay) { h *= 0.5; rejected = 1; out->n_reject++; continue; }
    double e = orc_err_norm(nc, y, y1, err, P->rtol, P->atol);
    if (!hplay && !(e <= 1.0)) {
      h *= orc_step_factor(e, 1);
      rejected = 1;
      out->n_reject++;
      continue;
    }
    if (hrec && out->n_accept < hcap) hrec[out->n_accept] = h;
    out->n_accept++;
    if (nrec) *nrec = out->n_accept;
    /* Equatorial crossing test on the accepted step (Sec. 3.3, Sec. 4.2). */
    double s0 = y[2] - half_pi, s1 = y1[2] - half_pi;
    if ((s0 > 0.0 && s1 <= 0.0) || (s0 < 0.0 && s1 >= 0.0)) {
      double a = 0.0, b = 1.0, ym[6];
      if (s1 == 0.0) {
        a = 1.0;
      } else {
        for (int bi = 0; bi < 200; ++bi) {        /* bisection on the dense output */
          double m = 0.5 * (a + b);
          if (m <= a || m >= b) break;
          orc_dense(6, y, y1, h, k, m, ym);
          double sm = ym[2] - half_pi;
          if ((sm > 0.0) == (s0 > 0.0) && sm != 0.0) a = m; else b = m;
        }
      }
      double sig = (s1 == 0.0) ? 1.0 : 0.5 * (a + b);
      double yc[6];
      orc_dense(6, y, y1, h, k, sig, yc);
      double Rc = yc[1];
      /* Reading: events count only inside the integration domain
       * R_cap <= R <= R_esc, so the final step's overshoot past a
       * termination radius cannot add a crossing. */
      int in_domain = Rc >= G->R_cap && Rc <= G->R_esc;
      double Sig = Rc * Rc + P->chi * P->chi * cos(yc[2]) * cos(yc[2]);
      double thdot = yc[5] / Sig;                  /* Eq. (60) */
      double lamc = lam + sig * h;
      double rth = fabs(fabs(thdot) / P->thetadot_min - 1.0);
      if (rth < out->near_thdot) out->near_thdot = rth;
      if (have_trusted) {
        double rl = fabs((lamc - lam_last) / P->dlambda_min - 1.0);
        if (rl < out->near_dlam) out->near_dlam = rl;
      }
      int trusted = in_domain && fabs(thdot) >= P->thetadot_min &&
                    (!have_trusted || lamc - lam_last >= P->dlambda_min);
      if (trusted) {
        int n = out->ncross;
        double gfac = 0.0, jem = 0.0, W, uT;
        if (orc_circular(P, Rc, &W, &uT) == 0) {
          double den = -uT * ((-E) + W * ell);      /* -p.u_em, Eq. (89)-(90) */
          gfac = num / den;
          jem = orc_emissivity(P, G->R_in, Rc, half_pi);
        }
        /* thin-disk g^3 j (reading of Eq. 88); the volumetric mode adds no
         * event intensity (its integral is the seventh component) */
        double In = P->volumetric ? 0.0 : gfac * gfac * gfac * jem;
        out->I_tot += In;
        if (n < 3) {
          double ph = fmod(yc[3], 2.0 * M_PI);
          if (ph < 0.0) ph += 2.0 * M_PI;
          out->R_em[n] = Rc;                       /* Eq. (82) */
          out->phi_em[n] = ph;
          out->T_em[n] = yc[0];
          out->g[n] = gfac;
          out->thdot[n] = thdot;
          out->lam_cross[n] = lamc;
          out->I_n[n] = In;
        }
        out->ncross = n + 1;
        lam_last = lamc;
        have_trusted = 1;
      }
    }
    lam += h;
    for (int i = 0; i < nc; ++i) { y[i] = y1[i]; k[0][i] = k[6][i]; }
    /* Polar axis (reading): a ray that passed through theta = 0 or pi is
     * mapped back to (0, pi) by (theta, p_theta, phi) -> (-theta, -p_theta,
     * phi + pi) or (2 pi - theta, -p_theta, phi + pi). */
    if (y[2] < 0.0 || y[2] > M_PI) {
      y[2] = (y[2] < 0.0) ? -y[2] : 2.0 * M_PI - y[2];
      y[5] = -y[5];
      y[3] += M_PI;
      orc_geo_rhs(&ctx, y, k[0]);
    }
    /* Null-constraint monitor (Sec. 3.1, after Eq. 62), scaled by the
     * dominant radial term P^2/(Delta Sigma). */
    {
      double pp[4] = {-E, y[4], y[5], ell};
      double c = cos(y[2]);
      double Sig = y[1] * y[1] + P->chi * P->chi * c * c;
      double Pr = (y[1] * y[1] + P->chi * P->chi) * E - P->chi * ell;
      double scale = Pr * Pr / (orc_Delta(P, y[1]) * Sig);
      double hd = fabs(orc_two_hamiltonian(P, y[1], y[2], pp)) / scale;
      if (hd > out->h_drift) out->h_drift = hd;
    }
    if (y[1] < out->R_min) out->R_min = y[1];
    if (hplay) continue;
    if (y[1] < G->R_cap) { out->status = 1; break; }     /* Eq. (75) */
    if (y[1] > G->R_esc) { out->status = 0; break; }     /* escape, Sec. 3.3 */
    h *= orc_step_factor(e, rejected);
    if (P->volumetric) h = orc_layer_cap(P, y, k[0], h);
    rejected = 0;
  }
  if (P->volumetric) out->I_tot = y[6];
  out->R_final = y[1];
  out->lam_final = lam;
  out->K_final = orc_carter(P, E, ell, y[2], y[5]);
  return 0;
}

int orc_trace_ray(const orc_problem* P, const orc_geom* G, double X, double Y, orc_ray* out) {
  return orc_trace_ray_core(P, G, X, Y, out, NULL, 0, NULL, NULL, 0);
}

/* Points with their accepted step sequences recorded (hbuf[i*hcap ...]). */
int orc_trace_points_record(const orc_problem* P, int64_t n, const double* xy, orc_ray* out,
                            double* hbuf, int hcap, int32_t* counts) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    int nr = 0;
    orc_trace_ray_core(P, &G, xy[2 * i], xy[2 * i + 1], &out[i], hbuf + i * (int64_t)hcap, hcap,
                       &nr, NULL, 0);
    counts[i] = nr;
  }
  return 0;
}

/* Points replayed along given step sequences (frozen). */
int orc_trace_points_frozen(const orc_problem* P, int64_t n, const double* xy,
                            const double* hbuf, int hcap, const int32_t* counts, orc_ray* out) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    int np = counts[i] < hcap ? counts[i] : hcap;
    orc_trace_ray_core(P, &G, xy[2 * i], xy[2 * i + 1], &out[i], NULL, 0, NULL,
                       hbuf + i * (int64_t)hcap, np);
  }
  return 0;
}

/* Traces an explicit list of screen points (for tests and sampled parity). */
int orc_trace_points(const orc_problem* P, int64_t n, const double* xy, orc_ray* out) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) orc_trace_ray(P, &G, xy[2 * i], xy[2 * i + 1], &out[i]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adaptive screen refinement (Sec. 4, idea stated in the Introduction and  */
/* Sec. 3.3; the rule below is the reading).  Class c = (status, ncross).    */
/* A base pixel is refined iff its class differs from an on-screen          */
/* 4-neighbour; a refined cell spawns 4x4 children at cell-centred offsets;  */
/* a child at level L < levels is refined iff its class differs from one of */
/* its 4-neighbours among its 16 siblings.  Pixel value = recursive mean of */
/* its children's values; unrefined cells use their own ray.                */
/* Key = base_id << 16 | level << 12 | d1 << 8 | d2 << 4 | d3.              */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t* keys;
  int64_t count, cap;
} orc_keys;

static void orc_push_key(orc_keys* K, uint64_t key) {
#pragma omp critical(orc_keys_push)
  {
    if (K->count < K->cap) K->keys[K->count] = key;
    K->count++;
  }
}

static int orc_same_class(const orc_ray* a, const orc_ray* b) {
  return a->status == b->status && a->ncross == b->ncross;
}

/* Refines one cell centred at (Xc, Yc) of width (wx, wy) at level L; writes
 * the recursive leaf mean of (I_tot, I_0, I_1, I_2) to val[4] and returns the
 * deepest level reached. */
static int orc_refine_cell(const orc_problem* P, const orc_geom* G, double Xc, double Yc,
                           double wx, double wy, int L, uint64_t key, orc_keys* K,
                           double val[4]) {
  orc_ray ch[16];
  double cx[16], cy[16];
  int child_level = L + 1;
  for (int c = 0; c < 16; ++c) {
    int ix = c % 4, iy = c / 4;
    cx[c] = Xc + ((ix + 0.5) / 4.0 - 0.5) * wx;
    cy[c] = Yc + ((iy + 0.5) / 4.0 - 0.5) * wy;
    orc_trace_ray(P, G, cx[c], cy[c], &ch[c]);
  }
  int deepest = child_level;
  double acc[4] = {0, 0, 0, 0};
  for (int c = 0; c < 16; ++c) {
    int ix = c % 4, iy = c / 4;
    uint64_t ckey = (key & ~((uint64_t)0xF << 12)) | ((uint64_t)child_level << 12) |
                    ((uint64_t)c << (4 * (3 - child_level)));
    orc_push_key(K, ckey);
    int marked = 0;
    if (child_level < P->levels) {
      int nb[4][2] = {{ix - 1, iy}, {ix + 1, iy}, {ix, iy - 1}, {ix, iy + 1}};
      for (int q = 0; q < 4; ++q) {
        int jx = nb[q][0], jy = nb[q][1];
        if (jx < 0 || jx > 3 || jy < 0 || jy > 3) continue;
        if (!orc_same_class(&ch[c], &ch[jy * 4 + jx])) marked = 1;
      }
    }
    double v[4];
    if (marked) {
      int d = orc_refine_cell(P, G, cx[c], cy[c], wx / 4.0, wy / 4.0, child_level, ckey, K, v);
      if (d > deepest) deepest = d;
    } else {
      v[0] = ch[c].I_tot; v[1] = ch[c].I_n[0]; v[2] = ch[c].I_n[1]; v[3] = ch[c].I_n[2];
    }
    for (int q = 0; q < 4; ++q) acc[q] += v[q];
  }
  for (int q = 0; q < 4; ++q) val[q] = acc[q] / 16.0;
  return deepest;
}

/* Output planes of a traced image (row-major [ny][nx], j = row = Y index). */
typedef struct {
  double* I;        /* [ny*nx] */
  double* I_n;      /* [3][ny*nx] */
  int32_t* ncross;  /* [ny*nx] */
  int32_t* status;  /* [ny*nx] */
  int32_t* level;   /* [ny*nx] deepest refinement level */
  double* R_em;     /* [3][ny*nx] base-ray transfer maps */
  double* phi_em;
  double* T_em;
  double* g;
  double* h_drift;  /* [ny*nx] */
  uint64_t* keys;   /* refined-cell keys (unsorted) */
  int64_t keys_cap;
  int64_t keys_count;
} orc_image;

int orc_trace_image(const orc_problem* P, orc_image* out) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
  int nx = P->nx, ny = P->ny;
  int64_t np = (int64_t)nx * ny;
  double dx = (P->x_max - P->x_min) / nx, dy = (P->y_max - P->y_min) / ny;
  orc_ray* base = (orc_ray*)malloc(sizeof(orc_ray) * np);
  if (!base) return 3;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < np; ++q) {
    int i = (int)(q % nx), j = (int)(q / nx);
    double X = P->x_min + (i + 0.5) * dx, Y = P->y_min + (j + 0.5) * dy;  /* cell centres */
    orc_trace_ray(P, &G, X, Y, &base[q]);
  }
  orc_keys K = {out->keys, 0, out->keys_cap};
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < np; ++q) {
    int i = (int)(q % nx), j = (int)(q / nx);
    const orc_ray* r = &base[q];
    int marked = 0;
    if (P->levels > 0) {
      int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
      for (int t = 0; t < 4; ++t) {
        int a = nb[t][0], b = nb[t][1];
        if (a < 0 || a >= nx || b < 0 || b >= ny) continue;
        if (!orc_same_class(r, &base[(int64_t)b * nx + a])) marked = 1;
      }
    }
    double v[4] = {r->I_tot, r->I_n[0], r->I_n[1], r->I_n[2]};
    int lev = 0;
    if (marked) {
      double X = P->x_min + (i + 0.5) * dx, Y = P->y_min + (j + 0.5) * dy;
      lev = orc_refine_cell(P, &G, X, Y, dx, dy, 0, (uint64_t)q << 16, &K, v);
    }
    out->I[q] = v[0];
    for (int n = 0; n < 3; ++n) out->I_n[n * np + q] = v[1 + n];
    out->ncross[q] = r->ncross;
    out->status[q] = r->status;
    out->level[q] = lev;
    for (int n = 0; n < 3; ++n) {
      out->R_em[n * np + q] = r->R_em[n];
      out->phi_em[n * np + q] = r->phi_em[n];
      out->T_em[n * np + q] = r->T_em[n];
      out->g[n * np + q] = r->g[n];
    }
    out->h_drift[q] = r->h_drift;
  }
  out->keys_count = K.count;
  free(base);
  return 0;
}

/* One base pixel (i, j) of the image, computed on its own: traces the pixel's
 * ray, its on-screen 4-neighbours (for the refinement decision only) and the
 * refinement subtree.  Used for sampled parity at sizes where the full oracle
 * image is too slow.  val[4] = (I_tot, I_0, I_1, I_2); *level = deepest
 * level; keys of the subtree are appended to keys[0..cap). */
int orc_trace_pixel(const orc_problem* P, int i, int j, orc_ray* base_ray, double val[4],
                    int32_t* level, uint64_t* keys, int64_t cap, int64_t* count) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
  int nx = P->nx, ny = P->ny;
  double dx = (P->x_max - P->x_min) / nx, dy = (P->y_max - P->y_min) / ny;
  double X = P->x_min + (i + 0.5) * dx, Y = P->y_min + (j + 0.5) * dy;
  orc_trace_ray(P, &G, X, Y, base_ray);
  int marked = 0;
  if (P->levels > 0) {
    int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
    for (int t = 0; t < 4; ++t) {
      int a = nb[t][0], b = nb[t][1];
      if (a < 0 || a >= nx || b < 0 || b >= ny) continue;
      orc_ray nr;
      orc_trace_ray(P, &G, P->x_min + (a + 0.5) * dx, P->y_min + (b + 0.5) * dy, &nr);
      if (!orc_same_class(base_ray, &nr)) marked = 1;
    }
  }
  orc_keys K = {keys, 0, cap};
  val[0] = base_ray->I_tot; val[1] = base_ray->I_n[0];
  val[2] = base_ray->I_n[1]; val[3] = base_ray->I_n[2];
  *level = 0;
  if (marked)
    *level = orc_refine_cell(P, &G, X, Y, dx, dy, 0,
                             (uint64_t)((int64_t)j * nx + i) << 16, &K, val);
  *count = K.count;
  return 0;
}

/* Many base pixels, each with its refinement subtree (OpenMP over pixels).
 * ij[2k] = i, ij[2k+1] = j.  val4[4k..4k+3] = (I_tot, I_0, I_1, I_2),
 * level[k] = deepest level, nrays[k] = rays integrated for pixel k
 * (its own ray, its on-screen neighbours and its subtree).  Used to time the
 * oracle on a bounded sample of a workload. */
int orc_trace_pixels(const orc_problem* P, int64_t n, const int32_t* ij, double* val4,
                     int32_t* level, int64_t* nrays) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n; ++k) {
    orc_ray r;
    uint64_t keys[4096 + 256];
    int64_t cnt = 0;
    orc_trace_pixel(P, ij[2 * k], ij[2 * k + 1], &r, val4 + 4 * k, &level[k], keys, 4096 + 256,
                    &cnt);
    int i = ij[2 * k], j = ij[2 * k + 1], nb = 0;
    if (P->levels > 0) nb = (i > 0) + (i + 1 < P->nx) + (j > 0) + (j + 1 < P->ny);
    nrays[k] = 1 + nb + cnt;
  }
  return 0;
}

/* Geometry summary for tests: r_plus, R_in, R_cap, R_esc. */
int orc_geometry(const orc_problem* P, double out4[4]) {
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
  out4[0] = G.r_plus; out4[1] = G.R_in; out4[2] = G.R_cap; out4[3] = G.R_esc;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Shadow boundary (Sec. 4.1, Eqs. 78-79): for each polar direction psi of  */
/* the screen, X = b cos psi and Y = b sin psi, the impact parameter b is   */
/* varied and the transition between captured and escaping rays located.    */
/* Reading: plain bisection of [b_lo, b_hi] until the bracket is at most    */
/* tol wide; "captured" is status 1, and every other fate (escape,          */
/* undetermined) counts on the escaping side.  Per direction the final      */
/* bracket is returned (b_in on the captured side, b_out on the escaping    */
/* side) with flags: 1 if b_lo is not captured, 2 if b_hi is captured (in   */
/* either case no transition is bracketed and [b_lo, b_hi] is returned),   */
/* 4 if a traced ray was undetermined.                                      */
/* ------------------------------------------------------------------------ */
static int orc_captured(const orc_problem* P, const orc_geom* G, double b, double psi,
                        int32_t* flag) {
  orc_ray r;
  orc_trace_ray(P, G, b * cos(psi), b * sin(psi), &r);
  if (r.status == 2) *flag |= 4;
  return r.status == 1;
}

int orc_shadow_boundary(const orc_problem* P, int64_t n, const double* psi, double b_lo,
                        double b_hi, double tol, double* b_in, double* b_out, int32_t* flags) {
  if (!(b_lo >= 0.0 && b_hi > b_lo && tol > 0.0)) return -1;
  orc_geom G;
  int rc = orc_geometry_setup(P, &G);
  if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n; ++k) {
    int32_t f = 0;
    double lo = b_lo, hi = b_hi;
    if (!orc_captured(P, &G, lo, psi[k], &f)) f |= 1;
    if (orc_captured(P, &G, hi, psi[k], &f)) f |= 2;
    if (!(f & 3)) {
      while (hi - lo > tol) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_captured(P, &G, mid, psi[k], &f))
          lo = mid;
        else
          hi = mid;
      }
    }
    b_in[k] = lo;
    b_out[k] = hi;
    flags[k] = f;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Outer stationary-limit surface (Sec. 2.3, Eqs. 38-41): R_s(theta) is the */
/* largest positive root of R^2 H(R) + chi^2 cos^2 theta = 0 (Eq. 40),      */
/* found as orc_horizon finds R_+: scan downward from R = 50 in steps of    */
/* 1e-3 to the first sign change, then bisect.  Returns 0, or 1 if there    */
/* is no root.                                                               */
/* ------------------------------------------------------------------------ */
int orc_ergosurface(const orc_problem* P, double th, double* R_s) {
  const double c = cos(th), c2 = P->chi * P->chi * c * c;
  const double step = 1e-3;
  double hi = 50.0, fhi = hi * hi * orc_H(P, hi) + c2;
  if (!(fhi > 0.0)) return 1;
  for (long k = 1;; ++k) {
    double lo = 50.0 - k * step;
    if (lo <= 1e-6) return 1;
    double flo = lo * lo * orc_H(P, lo) + c2;
    if (flo <= 0.0) {
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (mid * mid * orc_H(P, mid) + c2 > 0.0) hi = mid; else lo = mid;
      }
      *R_s = hi;
      return 0;
    }
    hi = lo;
  }
}
