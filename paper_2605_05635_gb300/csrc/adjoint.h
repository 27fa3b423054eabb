// adjoint.h -- data shared by the adjoint kernels (adjoint.cu) and the host
// orchestration of bh_trace_backward (api.cu).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace bhrt {

constexpr int kCkptEvery = 64;
constexpr int kMaxCrossAdj = 32;

// Derivatives of per-image constants with respect to (chi, theta_o, halo1,
// halo2), computed on the host.
struct AdjImg {
  double d_sqgrr[4], d_sqgth[4], d_sqgph[4], d_N[4], d_w[4], d_Rin[4];
};

struct Ckpt {
  double y[6], f[6];
  double h, lam, lam_last;
  int32_t nacc, nrej, steps, ncross;
  int32_t rejected, have_trusted, pad0, pad1;
};

struct AdjArgs {
  const WsHeader* hdr;
  const ImgParams* ip;   // [1]
  AdjImg aj;
  int levels;
  int64_t npix;
  const double* Gpix;    // [npix] dL/dI per pixel
  const int32_t* base_child;
  LevelRecs lv[kMaxLevels + 1];
  Ckpt* ckpt;            // [threads][max_ckpt]
  int max_ckpt;
  double* grad;          // [10]
  unsigned long long* head;
  int* status;
};

struct ImgAdj {
  int nx, ny;
  double x_min, y_min, dx, dy;
  const float* dLdI;    // optional
  double S, Xc, Yc, C;  // pixel sum of I, centroid
  double FRs, FLs;      // right / left pixel sums
  double cC, cA;        // dL/dC, dL/dA_LR
  int bstar, nbins;     // radial profile argmax and bins
  double drho[3];       // d rho_peak / d(mean of bins bstar-1, bstar, bstar+1)
  int cnt[3];
  double cR;            // dL/d rho_peak
  double uv[16];        // 8 baselines
  double Vre[8], Vim[8], Vabs[8], V0, cV[8];
  double* G;            // [npix] out
};


cudaError_t launch_adjoint(const AdjArgs& a, int blocks, int threads, cudaStream_t s);
cudaError_t launch_pixel_adjoint(const ImgAdj& a, cudaStream_t s);
cudaError_t launch_image_moments(const float* I, const ImgAdj& a, double* out3, cudaStream_t s);
cudaError_t launch_image_profile(const float* I, const ImgAdj& a, double* lr, double* hs,
                                 unsigned long long* hc, cudaStream_t s);

}  // namespace bhrt
