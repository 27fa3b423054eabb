// vis_curves.cu -- visibility-amplitude curves (Sec. 6.4): the azimuthally
// averaged normalised amplitude V(q) and the horizontal cut |V(q, 0)|/|V(0,0)|
// at dense q, on a structured (u, v) set evaluated by the visibility path of
// Eq. (108) (FP64 direct sum or the split tensor-core contraction).
//
// Per curve point q_j the set holds n_phi points on the half circle,
// phi_k = (k + 1/2) pi / n_phi (|V(-u,-v)| = |V(u,v)| for a real image), then
// the cut point (q_j, 0); one (0, 0) point closes the set.  A warp per q_j
// averages the amplitudes in a fixed order (lane-strided sums, then a
// shuffle tree) and divides by |V(0, 0)| of the same evaluation, so q = 0
// gives 1 to rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

__global__ void curve_uv_kernel(const double* q, int32_t n_q, int32_t n_phi, double* uv) {
  const int64_t per = (int64_t)n_phi + 1, total = (int64_t)n_q * per + 1;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    double u = 0.0, v = 0.0;
    if (t < total - 1) {
      const int64_t j = t / per;
      const int32_t k = (int32_t)(t - j * per);
      const double qj = q[j];
      if (k < n_phi) {
        double s, c;
        sincospi(((double)k + 0.5) / (double)n_phi, &s, &c);
        u = qj * c;
        v = qj * s;
      } else {
        u = qj;
      }
    }
    uv[2 * t] = u;
    uv[2 * t + 1] = v;
  }
}

__global__ void curve_reduce_kernel(const double* V, int32_t n_q, int32_t n_phi, double* avg,
                                    double* cut) {
  const int lane = threadIdx.x & 31;
  const int64_t per = (int64_t)n_phi + 1;
  const double* V0 = V + 2 * ((int64_t)n_q * per);
  const double a0 = hypot(V0[0], V0[1]);
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n_q; j += warps) {
    const double* Vj = V + 2 * j * per;
    double s = 0.0;
    for (int32_t k = lane; k < n_phi; k += 32) s += hypot(Vj[2 * k], Vj[2 * k + 1]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      avg[j] = s / (double)n_phi / a0;
      cut[j] = hypot(Vj[2 * n_phi], Vj[2 * n_phi + 1]) / a0;
    }
  }
}

}  // namespace

extern "C" {

bh_status bh_visibility_curves_workspace_size(const bh_camera* cam, int32_t n_q, int32_t n_phi,
                                              size_t* bytes) {
  if (!cam || !bytes || n_q < 0 || n_phi < 1) return BH_ERR_INVALID_ARG;
  size_t vis;
  bh_status s = bh_visibilities_workspace_size(cam, &vis);
  if (s != BH_OK) return s;
  const size_t K = (size_t)n_q * ((size_t)n_phi + 1) + 1;
  *bytes = al256(vis) + 2 * al256(K * 2 * sizeof(double));
  return BH_OK;
}

bh_status bh_visibility_curves(const float* I, const bh_camera* cam, int32_t n_q,
                               const double* q, int32_t n_phi, int32_t mode, double image_max,
                               double* V_avg, double* V_cut, void* workspace,
                               size_t workspace_bytes, void* stream) {
  if (!I || !cam || n_q < 0 || n_phi < 1 || (n_q > 0 && (!q || !V_avg || !V_cut)) ||
      mode < 0 || mode > 2)
    return BH_ERR_INVALID_ARG;
  size_t need;
  bh_status s = bh_visibility_curves_workspace_size(cam, n_q, n_phi, &need);
  if (s != BH_OK) return s;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return BH_ERR_WORKSPACE;
  size_t vis;
  bh_visibilities_workspace_size(cam, &vis);
  const int64_t K = (int64_t)n_q * ((int64_t)n_phi + 1) + 1;
  // every argument error before anything is enqueued: the visibility
  // path's own checks (a call with no baselines enqueues nothing), its
  // baseline-count limit and the FP64 path's row limit (2 nx doubles of
  // shared memory within 200 KiB)
  s = bh_visibilities(I, cam, nullptr, 0, mode, image_max, nullptr, nullptr, 0.0, workspace,
                      vis, stream);
  if (s != BH_OK) return s;
  if (K > 0x7fffffff || (mode == 0 && (size_t)cam->nx * 2 * sizeof(double) > 200 * 1024))
    return BH_ERR_INVALID_ARG;
  char* ws = static_cast<char*>(workspace);
  double* uv = reinterpret_cast<double*>(ws + al256(vis));
  double* V = reinterpret_cast<double*>(ws + al256(vis) + al256((size_t)K * 2 * sizeof(double)));
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  // the status word leads the workspace, as for the visibility path
  if (cudaMemsetAsync(ws, 0, sizeof(int32_t), cs) != cudaSuccess) return BH_ERR_CUDA;
  const int sms = bhrt::num_sms();
  int64_t blocks = std::min<int64_t>((K + 255) / 256, (int64_t)sms * 8);
  curve_uv_kernel<<<(int)blocks, 256, 0, cs>>>(q, n_q, n_phi, uv);
  if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
  s = bh_visibilities(I, cam, uv, K, mode, image_max, V, nullptr, 0.0, ws, vis, stream);
  if (s != BH_OK) return s;
  if (n_q == 0) return BH_OK;
  blocks = std::min<int64_t>(((int64_t)n_q * 32 + 255) / 256, (int64_t)sms * 8);
  curve_reduce_kernel<<<(int)blocks, 256, 0, cs>>>(V, n_q, n_phi, V_avg, V_cut);
  return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

}  // extern "C"
