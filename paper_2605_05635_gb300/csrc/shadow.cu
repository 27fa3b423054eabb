// shadow.cu -- shadow-boundary search on the screen (Sec. 4.1, Eqs. 78-79).
//
// Along each polar direction psi of the screen (X = b cos psi, Y = b sin psi)
// the transition between captured and escaping rays is bracketed in b.  The
// paper varies b and locates the transition; a bisection traces one ray per
// round, so a few thousand directions leave most of the GPU idle for ~35
// sequential ray lifetimes.  Here a group of G lanes of one warp owns a
// direction and traces G rays per round at the interior points of a
// (G + 1)-section of the bracket: the group ballots the fates and keeps the
// sub-interval between the last captured sample and the first escaping one,
// so the bracket shrinks by G + 1 per round.  G is chosen on the host so that
// groups x G fills half the resident threads (a few warps per SM keep the
// FP64 pipe busy): many directions run as bisection (G = 1, least work), few
// directions as wide multisection (fewest rounds).
//
// Rays are traced by the FP64 integrator of the image path (ray_init64,
// ray_step64) with the caller's tolerances; crossings are located but not
// recorded.  The first round traces the two ends of the caller's bracket; a
// direction whose ends do not straddle the transition is flagged and
// returned with its bracket unchanged.
#include <cuda_runtime.h>

#include "integrator.cuh"

namespace bhrt {

// Fate of one ray: 0 escaped, 1 captured, 2 undetermined (Eq. 75, Sec. 3.3);
// its accepted and rejected steps are added to acc, rej.
__device__ __forceinline__ int ray_fate(const ImgParams& ip, const MetricConsts<double>& m,
                                        const TraceArgs& none, double X, double Y,
                                        unsigned long long& acc, unsigned long long& rej) {
  Ray64 r;
  ray_init64(ip, m, X, Y, r);
  int term = 0;
  while (term == 0) term = ray_step64<false, false, false>(ip, m, r, none, 0, 0);
  acc += (unsigned long long)r.nacc;
  rej += (unsigned long long)r.nrej;
  return term - 1;
}

__global__ void __launch_bounds__(128) shadow_kernel(ShadowArgs s) {
  const int lane = threadIdx.x & 31;
  const int G = s.group;                 // lanes per direction: 1, 2, 4, 8, 16 or 32
  const int gid = lane / G, gl = lane % G;
  const unsigned low = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const int64_t groups_per_warp = 32 / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x >> 5) * groups_per_warp;
  const ImgParams& ip = *s.ip;
  const MetricConsts<double> m = metric_consts<double>(ip);
  const unsigned long long budget = s.hdr->budget_ns, t0 = s.hdr->t_start;
  // the rays' crossing events are not evaluated (kEvents = false); the
  // arguments describe a level without per-pixel planes all the same
  TraceArgs none{};
  none.level = 1;
  none.mode = 0;

  int64_t k = warp * groups_per_warp + gid;
  double lo = s.b_lo, hi = s.b_hi;
  int phase = 0;          // 0: trace the ends (b_lo only if G = 1), 1: b_hi, 2: sections
  int32_t flags = 0;
  int rounds = 0;
  unsigned long long w_rays = 0, w_acc = 0, w_rej = 0;
  bool timed_out = false;
  while (__any_sync(kFull, k < s.n)) {
    const bool mine = k < s.n;
    double b = 0.0;
    bool sample = false;
    if (mine) {
      if (phase == 0) {
        // the ends of the bracket: lanes 0 and 1 (lane 0 twice if G = 1)
        sample = gl < 2;
        b = gl == 0 ? s.b_lo : s.b_hi;
      } else if (phase == 1) {
        sample = gl == 0;
        b = s.b_hi;
      } else {
        sample = true;
        b = lo + (hi - lo) * (double)(gl + 1) / (double)(G + 1);
      }
    }
    int fate = 0;
    if (sample) {
      double sn, cs;
      sincos(s.psi[k], &sn, &cs);
      fate = ray_fate(ip, m, none, b * cs, b * sn, w_acc, w_rej);
      ++w_rays;
    }
    const unsigned shift = (unsigned)(gid * G);
    const unsigned cap = (__ballot_sync(kFull, sample && fate == 1) >> shift) & low;
    const unsigned und = (__ballot_sync(kFull, sample && fate == 2) >> shift) & low;
    bool done = false;
    if (mine) {
      if (und) flags |= 4;
      if (phase == 0) {
        if (!(cap & 1u)) flags |= 1;
        if (G >= 2) {
          if (cap & 2u) flags |= 2;
          phase = 2;
          if (flags & 3) done = true;
        } else {
          phase = 1;  // b_hi next, whatever b_lo gave: both flags are reported
        }
      } else if (phase == 1) {
        if (cap & 1u) flags |= 2;
        phase = 2;
        if (flags & 3) done = true;
      } else {
        // first escaping sample e; [b_{e-1}, b_e] holds the transition
        const unsigned esc = ~cap & low;
        const double w0 = hi - lo;
        double nlo = lo, nhi = hi;
        if (esc == 0u) {
          nlo = lo + w0 * (double)G / (double)(G + 1);
        } else {
          const int e = __ffs(esc) - 1;
          nhi = lo + w0 * (double)(e + 1) / (double)(G + 1);
          if (e > 0) nlo = lo + w0 * (double)e / (double)(G + 1);
        }
        const bool shrank = nhi - nlo < w0;
        lo = nlo;
        hi = nhi;
        if (!shrank || hi - lo <= s.tol || ++rounds >= kShadowMaxRounds) done = true;
      }
    }
    if (budget) {
      const unsigned long long now = __shfl_sync(kFull, globaltimer(), 0);
      if (now - t0 > budget) timed_out = true;
    }
    if (mine && (done || timed_out)) {
      if (timed_out && !done) flags |= 8;
      if (gl == 0) {
        s.b_in[k] = lo;
        s.b_out[k] = hi;
        s.flags[k] = flags;
      }
      k += stride;
      lo = s.b_lo;
      hi = s.b_hi;
      phase = 0;
      flags = 0;
      rounds = 0;
    }
    if (timed_out) {
      // every direction this group still owns is reported as unfinished
      for (; k < s.n; k += stride)
        if (gl == 0) {
          s.b_in[k] = s.b_lo;
          s.b_out[k] = s.b_hi;
          s.flags[k] = 8;
        }
      if (lane == 0) atomicCAS(&s.hdr->status, 0, (int)BH_ERR_TIMEOUT);
      break;
    }
  }
  if (s.stats) {
    flush_tally(&s.stats[0], w_rays, lane);
    flush_tally(&s.stats[1], w_acc, lane);
    flush_tally(&s.stats[2], w_rej, lane);
  }
}

int shadow_resident_threads() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, shadow_kernel, 128, 0);
  return (nb > 0 ? nb : 1) * 128 * num_sms();
}

cudaError_t launch_shadow(const ShadowArgs& a, int blocks, int threads, cudaStream_t st) {
  shadow_kernel<<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bhrt
