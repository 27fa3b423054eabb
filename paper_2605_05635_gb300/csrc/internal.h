// internal.h -- host-side declarations shared by the library's translation
// units (kernel launchers and the C ABI layer).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/bhrt.h"
#include "bh_common.cuh"

namespace bhrt {

// Device pointers of one image's outputs (mirrors bh_image_out).
struct OutPtrs {
  float* I;
  float* I_n;
  uint8_t* ncross;
  uint8_t* status;
  uint8_t* refine_level;
  float* R_em;
  float* phi_em;
  float* T_em;
  float* g;
  float* h_drift;
  uint64_t* keys;
  int64_t keys_cap;
  unsigned long long* keys_count;
  int32_t* steps;       // optional [2][npix] accepted, rejected steps of the base ray
  uint8_t* promoted;    // optional [npix] base ray took FP64 steps (mixed path)
};

// Everything a trace launch needs (passed by value as a kernel parameter).
struct TraceArgs {
  WsHeader* hdr;
  const ImgParams* ip;   // [n_img]
  const OutPtrs* out;    // [n_img] (image mode)
  int level;             // 0 = base screen, 1..3 = refinement list
  int mode;              // 0 = image, 1 = explicit points
  int64_t npix;          // nx * ny
  int64_t n_items;       // level 0 / points: item count; levels >= 1: read hdr->count
  // level 0 records
  double* base_I;        // [4][n_items]
  uint16_t* base_cls;
  uint8_t* base_depth;
  LevelRecs lv;          // records of `level` when level >= 1
  const double* xy;      // points mode
  bh_ray_record* rec;    // points mode
  // precision passes of the mixed path
  int source;                         // 0 fresh items, 1 resume from spill_in
  unsigned long long* head;           // cursor of this pass
  const struct SpillRec* spill_in;    // source == 1
  unsigned long long* spill_in_count;
  struct SpillRec* spill_out;         // hand-off queue (promote / demote)
  unsigned long long* spill_out_count;
  int64_t spill_cap;
  int allow_spill;                    // FP32: promote; FP64: demote
  int any_volumetric;                 // some image integrates Eq. (88): use the
                                      // kernel build that carries the integral
};

struct LaunchShape {
  int blocks;
  int threads;
  int variant = 0;  // 0 register-unbounded build; 1 capped build (FP64: 3 blocks of
                    // 128 per SM, mixed: 4)
};

// trace.cu / trace_mixed.cu
cudaError_t launch_trace_fp64(const TraceArgs& a, LaunchShape s, cudaStream_t st);
cudaError_t launch_trace_mixed(const TraceArgs& a, LaunchShape s, cudaStream_t st);
int trace_default_blocks_per_sm(int precision, int threads, int variant = 0);
constexpr int kKernelVariants = 2;
size_t spill_record_bytes();
const void* trace_fp64_kernel_ptr(int variant);

// refine.cu
struct RefineArgs {
  WsHeader* hdr;
  const ImgParams* ip;
  const OutPtrs* out;
  int n_img;
  int64_t npix;
  int levels;
  double* base_I;
  uint16_t* base_cls;
  int32_t* base_child;
  uint8_t* base_depth;
  LevelRecs lv[kMaxLevels + 1];  // lv[1..levels]
};
cudaError_t launch_mark_expand(const RefineArgs& a, int level, int blocks, cudaStream_t st);
cudaError_t launch_assemble(const RefineArgs& a, int level, int blocks, cudaStream_t st);
cudaError_t launch_write_keys(const RefineArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_begin(WsHeader* hdr, unsigned long long budget_ns, cudaStream_t st);
int num_sms();

// shadow.cu -- shadow-boundary search (Sec. 4.1, Eqs. 78-79)
constexpr int kShadowMaxRounds = 200;
struct ShadowArgs {
  WsHeader* hdr;
  const ImgParams* ip;
  const double* psi;     // [n] screen directions
  int64_t n;
  double b_lo, b_hi, tol;
  double* b_in;          // [n] captured end of the final bracket
  double* b_out;         // [n] escaping end
  int32_t* flags;        // [n]
  unsigned long long* stats;  // optional [3]: rays, accepted, rejected steps
  int group;             // lanes per direction (1, 2, 4, 8, 16, 32)
};
cudaError_t launch_shadow(const ShadowArgs& a, int blocks, int threads, cudaStream_t st);
int shadow_resident_threads();

// scan.cu -- horizon, extremal-spin and stationary-limit scans (Sec. 2.3)
struct ScanArgs {
  const bh_spacetime* st;  // [n] device
  int64_t n;
  int32_t n_theta;
  const double* theta;     // [n_theta] device
  double* r_plus;          // [n]
  double* chi_e;           // [n]
  double* R_e;             // [n]
  double* R_s;             // optional [n][n_theta]
  int32_t* flags;          // [n]
  unsigned long long* stats;  // optional [2]: lapse evaluations of the horizon
                              // and of the stationary-limit searches
};
cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st);

}  // namespace bhrt
