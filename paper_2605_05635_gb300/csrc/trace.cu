// trace.cu -- persistent FP64 per-ray integrator kernel.
//
// One thread integrates one backward ray (Sec. 3-4): launch from the ZAMO
// screen (Eqs. 63-74), Dormand-Prince 5(4) steps of Hamilton's equations
// (Eqs. 57-62, separated form in bh_common.cuh), capture / escape
// (Eq. 75, Sec. 3.3), equatorial-crossing events on the dense output
// (Sec. 3.3, 4.2), transfer maps (Eq. 82), redshift (Eqs. 89-91) and the
// thin-disk intensity g^3 j (Eqs. 83-88).
//
// Scheduling: a persistent grid; every warp keeps 32 rays in flight and
// refills lanes whose ray has terminated with the next items of a global
// queue (one warp-aggregated atomic per refill), so long near-critical rays
// do not hold idle lanes hostage.  Free lanes refill in groups of
// kRefillLanes: starting a ray (above all resuming a promoted one, with its
// projection onto the launch invariants) is divergent FP64 work.
//
// In the all-FP64 path this kernel traces every ray.  In the mixed path it
// is the promoted pass: it resumes rays handed over by the FP32 kernel and,
// once a ray is outgoing beyond demote_R, hands it back for an FP32 finish.
#include <cuda_runtime.h>

#include "integrator.cuh"

namespace bhrt {

constexpr int kTraceMaxThreads = 128;  // trace blocks are 64 or 128 threads
constexpr int kXFlushLanes = 8;        // parked crossings evaluated together
constexpr int kRefillLanes = 4;        // free lanes that start new rays together

// MinBlocks = 0 leaves the register count to the compiler (2 blocks of 128
// threads per SM); MinBlocks = 3 caps it for 3 blocks at a small spill cost.
// The autotuner picks between them.  Vol = true is the build used when some
// image of the call integrates the volumetric intensity.
template <int MinBlocks, bool Vol>
__global__ void __launch_bounds__(128, MinBlocks) trace_fp64_kernel(TraceArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n_items = pass_items(a);
  const unsigned long long budget = a.hdr->budget_ns;
  const unsigned long long t0 = a.hdr->t_start;

  Ray64 r;
  MetricConsts<double> m;
  const ImgParams* ip = a.ip;
  int64_t item = -1;
  uint32_t img = 0;
  bool active = false, drained = false;
  unsigned iter = 0;
  unsigned long long w_max = 0, w_iters = 0, w_lanes = 0;
  unsigned long long w_acc = 0, w_rej = 0, w_rays = 0, w_full = 0;

  // parked crossings, one slot per thread (blocks of at most 128 threads)
  __shared__ XPend xslot[kTraceMaxThreads];
  XPend* const xp = &xslot[threadIdx.x];

  const int pass = a.source;
  if (lane == 0) mark_first(&a.hdr->t_pass[0][pass][a.level]);
  while (true) {
    const bool need = refill_now<kRefillLanes>(!active && !drained, active);
    int64_t idx = claim(a.head, need, lane);
    if (need) {
      if (idx < n_items) {
        if (a.source == 1) {
          const SpillRec& s = a.spill_in[idx];
          item = s.item;
          img = s.img;
          ip = &a.ip[img];
          m = metric_consts<double>(*ip);
          // a ray promoted from the FP32 pass continues on its exact
          // constants of motion (K from the launch point)
          double X, Y;
          int64_t pix;
          uint32_t im;
          resolve_item(a, item, im, pix, X, Y);
          SpillRec sp = s;
          project_invariants(m, s.E, s.ell, launch_carter(*ip, X, Y), sp.y);
          resume64(*ip, sp, m, r);
        } else {
          double X, Y;
          int64_t pix;
          item = idx;
          resolve_item(a, idx, img, pix, X, Y);
          ip = &a.ip[img];
          m = metric_consts<double>(*ip);
          ray_init64(*ip, m, X, Y, r);
        }
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
    int term = 0;
    bool spill = false;
    if (active) {
      const int acc0 = r.nacc, rej0 = r.nrej;
      term = ray_step64<Vol, true>(*ip, m, r, a, item, img, xp);
      w_acc += (unsigned long long)(r.nacc - acc0);
      w_rej += (unsigned long long)(r.nrej - rej0);
      // outgoing beyond the strong-field zone, or away from the double root
      // of its radial potential: finish in FP32
      // (p_R > 0 and R > demote_R as bit-pattern compares: the accepted
      // state is not NaN and R is positive)
      spill = !term && a.allow_spill && r.nacc != acc0 && __double_as_longlong(r.y[4]) > 0 &&
              (__double_as_longlong(r.y[1]) > __double_as_longlong(ip->demote_R) ||
               (ip->kappa > 0.0 && past_double_root(*ip, r.E, r.ell, r.y[1], r.y[4])));
    }
    // parked crossings: evaluated together once kXFlushLanes lanes hold one,
    // and by a lane whose ray leaves this pass now
    {
      const bool mine = active && r.xpend;
      const unsigned pm = __ballot_sync(kFull, mine);
      if (mine && (__popc(pm) >= kXFlushLanes || term || spill)) {
        CrossState cs = r.cs;
        flush_crossing(*ip, m, r.E, r.ell, *xp, cs, cross_out(a, item, img));
        r.cs = cs;
        r.xpend = false;
      }
    }
    if (term) {
      finish_ray(a, item, img, term - 1, r.cs, r.hdrift, r.nacc, r.nrej, r.E, r.ell, r.lam);
      w_rays += 1ull;
      w_max = (unsigned long long)r.steps > w_max ? (unsigned long long)r.steps : w_max;
      active = false;
    } else if (spill) {
      unsigned long long slot = atomicAdd(a.spill_out_count, 1ull);
      if (slot < (unsigned long long)a.spill_cap) {
        spill_from64(r, item, img, a.spill_out[slot]);
        active = false;
      } else {
        w_full += 1ull;
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
  flush_tally(&a.hdr->accepted, w_acc, lane);
  flush_tally(&a.hdr->rejected, w_rej, lane);
  flush_tally(&a.hdr->rays[a.level], w_rays, lane);
  if (lane == 0) {
    atomicMax(&a.hdr->t_pass[2][pass][a.level], globaltimer());
    atomicAdd(&a.hdr->warp_iters[1], w_iters);
    atomicAdd(&a.hdr->lane_iters[1], w_lanes);
  }
  if (w_max) atomicMax(&a.hdr->max_ray_steps, w_max);
  flush_tally(&a.hdr->spill_full, w_full, lane);
}

cudaError_t launch_trace_fp64(const TraceArgs& a, LaunchShape s, cudaStream_t st) {
  if (a.any_volumetric) {
    if (s.variant == 1)
      trace_fp64_kernel<3, true><<<s.blocks, s.threads, 0, st>>>(a);
    else
      trace_fp64_kernel<0, true><<<s.blocks, s.threads, 0, st>>>(a);
  } else if (s.variant == 1) {
    trace_fp64_kernel<3, false><<<s.blocks, s.threads, 0, st>>>(a);
  } else {
    trace_fp64_kernel<0, false><<<s.blocks, s.threads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

size_t spill_record_bytes() { return sizeof(SpillRec); }

const void* trace_fp64_kernel_ptr(int variant) {
  return variant == 1 ? (const void*)trace_fp64_kernel<3, false>
                      : (const void*)trace_fp64_kernel<0, false>;
}

}  // namespace bhrt
