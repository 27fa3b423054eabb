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
//   - launch, constants of motion (E, ell), starting step, crossing roots,
//     transfer maps, redshift and emissivity run in FP64;
//   - a ray is promoted to the FP64 kernel when it comes within promote_R of
//     the horizon or, winding at N_cross >= 2, is inside demote_R; the FP64
//     pass hands it back once it is outgoing beyond demote_R, and a second
//     FP32 pass (no further promotion) finishes it.  Promotion is a hand-off
//     through a queue rather than a per-lane branch, so warps never mix FP64
//     and FP32 steps.
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

struct RayMx {
  float yh[6], yl[6];  // state T, R, th, phi, p_R, p_th as hi + lo
  float f[6];          // f(y) in FP32 (FSAL)
  float h;
  float lh, ll;        // affine parameter as hi + lo
  double E, ell;
  float Ef, ellf;
  CrossState cs;
  float hdrift;
  int32_t nacc, nrej, steps;
  bool rejected;
};

__device__ __forceinline__ void mx_from64(const Ray64& r, RayMx& x) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    df_from(r.y[i], x.yh[i], x.yl[i]);
    x.f[i] = (float)r.f[i];
  }
  x.h = (float)r.h;
  df_from(r.lam, x.lh, x.ll);
  x.E = r.E;
  x.ell = r.ell;
  x.Ef = (float)r.E;
  x.ellf = (float)r.ell;
  x.cs = r.cs;
  x.hdrift = r.hdrift;
  x.nacc = r.nacc;
  x.nrej = r.nrej;
  x.steps = r.steps;
  x.rejected = r.rejected;
}

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

__device__ __forceinline__ void mx_resume(const SpillRec& s, const MetricConsts<float>& mf,
                                          RayMx& x) {
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
  float W, P2;
  geo_rhs(mf, x.Ef, x.ellf, x.yh[1], x.yh[2], x.yh[4], x.yh[5], x.f, W, P2);
}

struct MxConsts {
  float rtol, atol, R_cap, R_esc, promote_R, demote_R;
};

// pi/2 as a float pair hi + lo, and pi (hi part) for the axis test.
constexpr float kHalfPiHi = 1.57079637050628662109375f;
constexpr float kHalfPiLo = -4.37113900018624283e-8f;
constexpr float kPiHi = 3.1415927410125732421875f;

// One attempted FP32 step.  Returns 0 (continue), terminal status + 1, or 4
// when the ray must be promoted to FP64.
__device__ __forceinline__ int ray_step_mx(const ImgParams& ip, const MetricConsts<float>& mf,
                                           const MetricConsts<double>& md, const MxConsts& c,
                                           RayMx& r, const CrossOut& co, bool may_promote) {
  const float h = r.h;
  float k[7][6];
#pragma unroll
  for (int i = 0; i < 6; ++i) k[0][i] = r.f[i];
  bool bad = false;
  float W = 0.f, P2oD = 1.f;
#pragma unroll
  for (int s = 1; s < 7; ++s) {
    float ys[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < s; ++j) acc += (float)kDP.a[s][j] * k[j][i];
      ys[i] = r.yh[i] + (r.yl[i] + h * acc);
    }
    bool ok = geo_rhs(mf, r.Ef, r.ellf, ys[1], ys[2], ys[4], ys[5], k[s], W, P2oD);
    bad |= !ok;
  }
  float dlt[6], err2 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float a5 = 0.f, ae = 0.f;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      a5 += (float)kDP.b[j] * k[j][i];
      ae += (float)kDP.e[j] * k[j][i];
    }
    dlt[i] = h * a5;
    float sc = c.atol + c.rtol * fmaxf(fabsf(r.yh[i]), fabsf(r.yh[i] + dlt[i]));
    float q = h * ae / sc;
    err2 += q * q;
  }
  float err = sqrtf(err2 / 6.f);
  r.steps++;
  if (bad || !(err <= 1.f)) {
    r.h = bad ? 0.5f * h : h * step_factor(err, true);
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
      double y0[6], y1[6], hf0[6], hf1[6], hd[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < 7; ++j) a += (float)kDP.d[j] * k[j][i];
        y0[i] = df_to(r.yh[i], r.yl[i]);
        y1[i] = df_to(nh[i], nl[i]);
        hd[i] = (double)h * (double)a;
        hf0[i] = (double)h * (double)k[0][i];
        hf1[i] = (double)h * (double)k[6][i];
      }
      handle_crossing(ip, md, r.E, r.ell, y0, y1, hf0, hf1, hd, df_to(r.lh, r.ll), (double)h,
                      r.cs, co);
    }
  }
  df_add(r.lh, r.ll, h);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    r.yh[i] = nh[i];
    r.yl[i] = nl[i];
    r.f[i] = k[6][i];
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
      float Wr, Pr;
      geo_rhs(mf, r.Ef, r.ellf, r.yh[1], r.yh[2], r.yh[4], r.yh[5], r.f, Wr, Pr);
    }
  }
  float hdv = fabsf(W) / P2oD;
  if (hdv > r.hdrift) r.hdrift = hdv;
  const float R = r.yh[1];
  if (R < c.R_cap) return 2;
  if (R > c.R_esc) return 1;
  r.h = h * step_factor(err, r.rejected);
  r.rejected = false;
  if (may_promote && (R < c.promote_R || (r.cs.ncross >= 2 && R < c.demote_R))) return 4;
  return r.steps >= ip.max_steps ? 3 : 0;
}

__global__ void __launch_bounds__(128) trace_mixed_kernel(TraceArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n_items = pass_items(a);
  const unsigned long long budget = a.hdr->budget_ns;
  const unsigned long long t0 = a.hdr->t_start;
  const bool may_promote = a.allow_spill != 0;

  RayMx r;
  MetricConsts<float> mf;
  MetricConsts<double> md;
  MxConsts c;
  const ImgParams* ip = a.ip;
  int64_t item = -1;
  uint32_t img = 0;
  bool active = false, drained = false;
  unsigned iter = 0;
  unsigned long long w_acc = 0, w_rej = 0, w_rays = 0, w_promo = 0, w_full = 0;

  while (true) {
    const bool need = !active && !drained;
    int64_t idx = claim(a.head, need, lane);
    if (need) {
      if (idx < n_items) {
        if (a.source == 1) {
          const SpillRec& s = a.spill_in[idx];
          item = s.item;
          img = s.img;
          ip = &a.ip[img];
          mf = metric_consts<float>(*ip);
          md = metric_consts<double>(*ip);
          mx_resume(s, mf, r);
        } else {
          double X, Y;
          int64_t pix;
          item = idx;
          resolve_item(a, idx, img, pix, X, Y);
          ip = &a.ip[img];
          mf = metric_consts<float>(*ip);
          md = metric_consts<double>(*ip);
          Ray64 r64;
          ray_init64(*ip, md, X, Y, r64);
          mx_from64(r64, r);
        }
        c.rtol = (float)fmax(ip->rtol, 1e-9);  // FP32 noise floor of the estimate
        c.atol = (float)ip->atol;
        c.R_cap = (float)ip->R_cap;
        c.R_esc = (float)ip->R_esc;
        c.promote_R = (float)ip->promote_R;
        c.demote_R = (float)ip->demote_R;
        active = true;
      } else {
        drained = true;
      }
    }
    if (__ballot_sync(kFull, active) == 0) {
      if (__ballot_sync(kFull, !drained) == 0) break;
      continue;
    }
    if (active) {
      const CrossOut co = cross_out(a, item, img);
      const int acc0 = r.nacc, rej0 = r.nrej;
      int term = ray_step_mx(*ip, mf, md, c, r, co, may_promote);
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
  flush_tally(&a.hdr->promoted_rays, w_promo, lane);
  flush_tally(&a.hdr->spill_full, w_full, lane);
}

cudaError_t launch_trace_mixed(const TraceArgs& a, LaunchShape s, cudaStream_t st) {
  trace_mixed_kernel<<<s.blocks, s.threads, 0, st>>>(a);
  return cudaGetLastError();
}

int trace_default_blocks_per_sm(int precision, int threads) {
  int nb = 0;
  if (precision == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_fp64_kernel_ptr(), threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_mixed_kernel, threads, 0);
  return nb > 0 ? nb : 1;
}

}  // namespace bhrt
