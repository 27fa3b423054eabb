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
  double rtol, atol, thdot_min, dlam_min, promote_R, demote_R;
  int32_t promote_ncross;  // mixed: promote once N_cross reaches this inside demote_R
  int32_t pad1;
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

__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_exp(float x) { return __expf(x); }
__device__ __forceinline__ double d_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float d_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ void d_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void d_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float d_rcp(float x) { return __frcp_rn(x); }
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
template <class T>
__device__ __forceinline__ bool geo_rhs(const MetricConsts<T>& m, T E, T ell, T R, T th, T pR,
                                        T pth, T d[6], T& W, T& P2oD) {
  T s, c;
  d_sincos(th, &s, &c);
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
  T P = r2a2 * E - m.chi * ell;
  T Q = ell * is - m.chi * E * s;
  T PoD = P * iD;
  P2oD = P * PoD;
  W = Dl * pR * pR - P2oD + pth * pth + Q * Q;
  d[0] = (r2a2 * PoD + m.chi * (ell - m.chi * E * s * s)) * iS;   // Eq. (57)
  d[1] = Dl * pR * iS;                                            // Eq. (59)
  d[2] = pth * iS;                                                // Eq. (60)
  d[3] = (m.chi * PoD + ell * is * is - m.chi * E) * iS;          // Eq. (58)
  T dW_R = dDl * pR * pR - T(4) * R * E * PoD + PoD * PoD * dDl;  // d(W)/dR
  T dQ = -ell * c * is * is - m.chi * E * c;                       // dQ/dth
  T iS2 = iS * iS;
  d[4] = T(-0.5) * dW_R * iS + W * R * iS2;                       // Eq. (61)
  d[5] = -Q * dQ * iS - W * m.chi2 * s * c * iS2;                 // Eq. (62)
  return (R > T(0)) && (Dl > T(0));
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
