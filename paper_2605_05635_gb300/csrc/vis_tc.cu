// vis_tc.cu -- visibilities (Sec. 6.4, Eq. 108) as a dense image-by-phase
// contraction on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
// exp[-2 pi i (u X_i + v Y_j)] = exp(-2 pi i u X_i) exp(-2 pi i v Y_j), so with
//   C_kj = sum_i cos(2 pi u_k X_i) I_ji,   S_kj = sum_i sin(2 pi u_k X_i) I_ji
// (a GEMM: rows = baselines x {cos, sin}, columns = image rows j, reduction
// over image columns i), the visibility is
//   Re V_k = sum_j [cos(2 pi v_k Y_j) C_kj - sin(2 pi v_k Y_j) S_kj] dX dY,
//   Im V_k = -sum_j [sin(2 pi v_k Y_j) C_kj + cos(2 pi v_k Y_j) S_kj] dX dY.
// Precision: both operands are split into hi + lo parts in BF16 (or FP16)
// and the three significant products hi*hi + hi*lo + lo*hi are accumulated in
// FP32 in tensor memory.
//
// One CTA owns 64 baselines (128 accumulator rows: 64 cos + 64 sin) and
// sweeps the image rows in passes of 256 columns of tensor memory.  For each
// 64-column chunk of the reduction axis the CTA generates the phase tile once,
// on chip, straight into shared memory as its hi and lo parts in the
// 128-byte-swizzled K-major layout (a sincospif every 16 columns and a
// rotation recurrence between), while TMA brings the hi and lo parts of the
// image tile; one thread then issues the three products of the chunk.  Two
// pipeline stages overlap phase generation and TMA with the MMAs of the
// previous chunk.  The epilogue reads the accumulators with tcgen05.ld,
// applies the v-phases (the same recurrence) and reduces over j.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "internal.h"

namespace bhrt {

constexpr int kVisRows = 128;       // accumulator lanes (64 baselines x cos/sin)
constexpr int kVisUV = 64;          // baselines per CTA
constexpr int kVisKC = 64;          // reduction chunk (elements): 128 bytes of 16-bit
constexpr int kVisNP = 256;         // image rows per pass (TMEM columns)
constexpr int kGenWarps = 8;        // warps that generate phase tiles and run the epilogue
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int kVisThreads = kGenThreads + 32;  // + one warp for TMA and MMA issue
constexpr int kStages = 2;
constexpr int kATile = kVisRows * kVisKC * 2;    // 16 KB: one part (hi or lo) of A
constexpr int kBTile = kVisNP * kVisKC * 2;      // 32 KB: one part of B
constexpr int kStage = 2 * kATile + 2 * kBTile;  // 96 KB: A hi, A lo, B hi, B lo
constexpr int kVisMaxNx = 4096;    // bound of the per-CTA phase table
constexpr int kSeg = 16;            // columns per thread between sincospif reseeds
constexpr int kVisSmem = kStages * kStage + 1024 + 256 + 2048 +
                         kVisUV * (kVisMaxNx / kVisKC) * 4;
// A pipeline wait that has not completed after this long (device clock)
// is treated as a stalled pipeline.
constexpr unsigned long long kWaitNs = 2000000000ull;

// Leading 256 bytes of the visibility workspace.
struct VisHdr {
  int status;                   // bh_status of the device work
  int reserved;
  unsigned long long t_start;   // %globaltimer when the call's work began (ns)
  unsigned long long budget_ns; // 0 = no budget
};

struct VisArgs {
  const double* uv;   // [K][2]
  int64_t K;
  int nx, ny, nxp;    // nxp = nx rounded up to kVisKC
  double x_min, y_min, dx, dy;
  double scale;       // image scale applied before splitting (undone at the end)
  int fp16;           // 0: BF16 operands, 1: FP16 operands
  double* V;          // [K][2]
  VisHdr* hdr;        // status word, start time and budget
};

__device__ __forceinline__ unsigned long long vis_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// A phase in turns as a 64-bit fixed-point fraction of one turn, so that
// phases add and scale by integers modulo one turn exactly on the integer
// pipes (FP64 runs at 1/64 of the FP32 rate here, and the per-block phases
// of the epilogue and the chunk table would otherwise cost FP64 operations
// on the critical path).  x is reduced to [0, 1) in FP64 once.
__device__ __forceinline__ uint64_t turns_fixed(double x) {
  double f = x - floor(x);
  if (!(f < 1.0)) f = 0.0;  // x just below an integer rounds up to 1; NaN
  return (uint64_t)__double2ull_rz(f * 18446744073709551616.0);  // 2^64
}
// The phase as half-turns in [-1, 1) (the argument of sincospif): the
// leading 32 bits read as a signed fraction, rounded to FP32 (within
// 6e-8 half-turns, as an FP64 phase reduced to [-1, 1] and rounded).
__device__ __forceinline__ float half_turns(uint64_t t) {
  return (float)(int32_t)(uint32_t)(t >> 32) * 4.656612873077393e-10f;  // 2^-31
}

__global__ void vis_begin(VisHdr* h, unsigned long long budget_ns) {
  h->status = 0;
  h->t_start = vis_clock();
  h->budget_ns = budget_ns;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Wait on an mbarrier phase, bounded by kWaitNs of device time; returns
// false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 0u) {
      const unsigned long long now = vis_clock();
      if (it == 0) t0 = now;
      else if (now - t0 > kWaitNs) return false;
    }
  }
}

// Shared-memory matrix descriptor for tcgen05.mma: K-major operand in the
// 128-byte swizzled layout (8-row x 128-byte atoms, atoms 1024 bytes apart).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (16 B, unused)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 1024 B
  d |= (uint64_t)1 << 46;                          // descriptor version (sm_100)
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, A/B BF16 or FP16,
// both K-major, M = 128, N = 256.
__device__ __forceinline__ uint32_t instr_desc(bool fp16) {
  uint32_t d = 0;
  d |= 1u << 4;                         // D format: F32
  d |= (fp16 ? 0u : 1u) << 7;           // A format: F16 = 0, BF16 = 1
  d |= (fp16 ? 0u : 1u) << 10;          // B format
  d |= (uint32_t)(256 >> 3) << 17;      // N / 8
  d |= (uint32_t)(128 >> 4) << 24;      // M / 16
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

template <class T16>
__device__ __forceinline__ uint16_t to_bits(T16 x) {
  return *reinterpret_cast<uint16_t*>(&x);
}

__device__ __forceinline__ void split16(float v, bool fp16, uint16_t& hi, uint16_t& lo) {
  if (fp16) {
    __half h = __float2half_rn(v);
    __half l = __float2half_rn(v - __half2float(h));
    hi = to_bits(h);
    lo = to_bits(l);
  } else {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    hi = to_bits(h);
    lo = to_bits(l);
  }
}

// Image -> B2 = [hi | lo] rows of length 2 * nxp (zero padded).
__global__ void vis_prepare_image(const float* I, VisArgs a, uint16_t* Bp) {
  const int64_t n = (int64_t)a.ny * a.nxp;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    int j = (int)(q / a.nxp), i = (int)(q % a.nxp);
    float v = i < a.nx ? (float)((double)I[(int64_t)j * a.nx + i] * a.scale) : 0.f;
    uint16_t hi, lo;
    split16(v, a.fp16 != 0, hi, lo);
    uint16_t* row = Bp + (int64_t)j * 2 * a.nxp;
    row[i] = hi;
    row[a.nxp + i] = lo;
  }
}

// Wait on an mbarrier phase as one role of a warp-specialised CTA: gives up
// (returns false) when another role has flagged a failure, or after kWaitNs
// of device time, which it flags itself.
__device__ __forceinline__ bool mbar_wait_role(uint64_t* bar, unsigned parity,
                                               volatile int* fail) {
  uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63u) == 0u) {
      if (*fail) return false;
      const unsigned long long now = vis_clock();
      if (it == 0) {
        t0 = now;
      } else if (now - t0 > kWaitNs) {
        *fail = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-specialised CTA: warps 0..7 generate the phase tile of each chunk
// into its pipeline stage and run the epilogue of each pass; warp 8 (one
// lane) loads the image tiles by TMA and issues the MMAs.  Stages are handed
// over by mbarriers (no CTA-wide barrier in the main loop):
//   tma_full[s]  the stage's image tiles landed (expect_tx by the issuer),
//   gen_full[s]  the 8 generator warps wrote the stage's phase tile,
//   empty[s]     the MMAs that read the stage completed (tcgen05.commit),
//   acc_full     all MMAs of a pass completed (the accumulators are final),
//   acc_empty    the 8 epilogue warps read the accumulators.
// The time budget is checked before each chunk's copies are issued; a CTA
// that stops (budget spent, or a wait bounded by kWaitNs ran out) waits for
// the copies and products it has issued before it frees tensor memory.
__global__ void __launch_bounds__(kVisThreads, 1)
    vis_tc_kernel(const __grid_constant__ CUtensorMap bmap, VisArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* tma_full = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint64_t* gen_full = tma_full + kStages;
  uint64_t* empty = gen_full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kStages * kStage + 64);
  volatile int* fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* red = reinterpret_cast<float*>(smem + kStages * kStage + 128);  // [2][128][2]
  float* tbase = red + 512;  // [nxp / 64][64] phase table (baseline fastest: no bank conflicts)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t uv0 = (int64_t)blockIdx.x * kVisUV;
  const bool fp16 = a.fp16 != 0;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&tma_full[s], 1);
      mbar_init(&gen_full[s], kGenWarps);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kGenWarps);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kVisNP));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  // phase generation: generator thread tid fills rows kk (cos) and kk + 64
  // (sin) for baseline kk = tid % 64, columns seg * 16 .. seg * 16 + 15 of
  // each chunk
  const int kk = tid & 63;
  const int seg = (tid >> 6) & 3;          // 0..3
  const int64_t kidx = uv0 + kk;
  const double u = kidx < a.K ? a.uv[2 * kidx] : 0.0;
  const float two_u_dx = (float)(2.0 * u * a.dx);
  // phase table: 2 u X (half-turns, in [-1, 1)) at the first column of each
  // chunk, from u X = u (x_min + dx / 2) + 64 b u dx in fixed-point turns
  const int nblk = a.nxp / kVisKC;
  if (tid < kGenThreads) {
    const uint64_t ua = turns_fixed(u * (a.x_min + 0.5 * a.dx));
    const uint64_t ub = turns_fixed(u * a.dx * (double)kVisKC);
    for (int b = seg; b < nblk; b += 4) tbase[b * kVisUV + kk] = half_turns(ua + (uint64_t)b * ub);
  }
  __syncthreads();

  const int chunks = nblk;
  const int passes = (a.ny + kVisNP - 1) / kVisNP;
  const int total = passes * chunks;
  // epilogue accumulators for the thread's (row, column-half): P = sum c D, Q = sum s D
  float accP = 0.f, accQ = 0.f;
  const int erow = (warp & 3) * 32 + lane;          // TMEM lane this thread reads
  const int ehalf = (warp >> 2) & 1;                // which 128-column half

  if (warp == kGenWarps) {
    // ---------------- image tiles (TMA) and MMA issue: one lane ----------------
    if (lane == 0) {
      const uint32_t idesc = instr_desc(fp16);
      const unsigned long long t_start = a.hdr->t_start, budget = a.hdr->budget_ns;
      // per stage: TMA copies issued and waited for, MMA batches committed
      unsigned tmas[kStages] = {0, 0}, tma_done[kStages] = {0, 0}, commits[kStages] = {0, 0};
      auto issue_tma = [&](int g) -> bool {
        const int s = g % kStages;
        const unsigned use = (unsigned)(g / kStages);
        // the stage's previous products must be done before its tiles are refilled
        if (use > 0 && !mbar_wait_role(&empty[s], (use - 1) & 1, fail)) return false;
        if (budget && vis_clock() - t_start > budget) {
          *fail = 2;
          return false;
        }
        unsigned char* sB = smem + s * kStage + 2 * kATile;
        tmas[s]++;
        mbar_expect_tx(&tma_full[s], 2 * kBTile);
        tma_load_2d(sB, &bmap, (g % chunks) * kVisKC, (g / chunks) * kVisNP, &tma_full[s]);
        tma_load_2d(sB + kBTile, &bmap, a.nxp + (g % chunks) * kVisKC, (g / chunks) * kVisNP,
                    &tma_full[s]);
        return true;
      };
      bool ok = issue_tma(0);
      for (int g = 0; g < total && ok; ++g) {
        const int s = g % kStages;
        const unsigned use = (unsigned)(g / kStages);
        const int pass = g / chunks, c = g % chunks;
        if (!mbar_wait_role(&tma_full[s], use & 1, fail)) {
          ok = false;
          break;
        }
        tma_done[s] = tmas[s];
        if (!mbar_wait_role(&gen_full[s], use & 1, fail)) {
          ok = false;
          break;
        }
        // the first products of a pass overwrite the accumulators: the
        // previous pass's epilogue must have read them
        if (c == 0 && pass > 0 && !mbar_wait_role(acc_empty, (pass - 1) & 1, fail)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ah = smem_u32(smem + s * kStage), al = ah + kATile;
        const uint32_t bh = ah + 2 * kATile, bl = bh + kBTile;
#pragma unroll
        for (int k16 = 0; k16 < kVisKC / 16; ++k16) {
          const uint32_t off = k16 * 32;
          const uint64_t dah = smem_desc_sw128(ah + off), dal = smem_desc_sw128(al + off);
          const uint64_t dbh = smem_desc_sw128(bh + off), dbl = smem_desc_sw128(bl + off);
          mma_f16(tmem, dah, dbh, idesc, c > 0 || k16 > 0);   // hi x hi
          mma_f16(tmem, dah, dbl, idesc, true);               // hi x lo
          mma_f16(tmem, dal, dbh, idesc, true);               // lo x hi
        }
        mma_commit(&empty[s]);
        commits[s]++;
        if (c == chunks - 1) mma_commit(acc_full);
        if (g + 1 < total && !issue_tma(g + 1)) ok = false;
      }
      if (!ok || *fail) {
        atomicCAS(&a.hdr->status, 0, (int)BH_ERR_TIMEOUT);
        if (!*fail) *fail = 1;
        // let copies and products already issued finish (bounded) before
        // the CTA frees its tensor memory and exits
        for (int s = 0; s < kStages; ++s) {
          if (tmas[s] > tma_done[s]) mbar_wait(&tma_full[s], (tmas[s] - 1) & 1);
          if (commits[s] > 0) mbar_wait(&empty[s], (commits[s] - 1) & 1);
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------- phase tiles and the epilogue: warps 0..7 ----------------
    float rot_s, rot_c;                    // one column step of the u-phase
    sincospif(two_u_dx, &rot_s, &rot_c);
    const int64_t ek = uv0 + (erow & 63);
    const double ev = ek < a.K ? a.uv[2 * ek + 1] : 0.0;
    const float dv = (float)(2.0 * ev * a.dy);
    float vrot_s, vrot_c;
    sincospif(dv, &vrot_s, &vrot_c);
    // v Y_j in fixed-point turns: v (y_min + dy / 2) + j v dy
    const uint64_t va = turns_fixed(ev * (a.y_min + 0.5 * a.dy));
    const uint64_t vb = turns_fixed(ev * a.dy);
    for (int g = 0; g < total; ++g) {
      const int s = g % kStages;
      const unsigned use = (unsigned)(g / kStages);
      const int pass = g / chunks, c = g % chunks;
      // waits are taken by every lane and decided per warp, so that a
      // failure sends the whole warp out of the loop together
      if (use > 0 && !__all_sync(0xffffffffu, mbar_wait_role(&empty[s], (use - 1) & 1, fail)))
        break;
      unsigned char* sAh = smem + s * kStage;
      unsigned char* sAl = sAh + kATile;
      // phase tile, hi and lo parts: a sincospif at the segment start, then
      // rotations by one column step (16 steps at most between reseeds)
      {
        const float t0 = tbase[c * kVisUV + kk] + (float)(seg * kSeg) * two_u_dx;
        float sn, cs;
        sincospif(t0, &sn, &cs);
        uint16_t ch[kSeg], cl[kSeg], sh[kSeg], sl[kSeg];
#pragma unroll
        for (int q = 0; q < kSeg; ++q) {
          split16(cs, fp16, ch[q], cl[q]);
          split16(sn, fp16, sh[q], sl[q]);
          const float cn = fmaf(cs, rot_c, -sn * rot_s);
          sn = fmaf(sn, rot_c, cs * rot_s);
          cs = cn;
        }
        // 128-byte swizzle: 16-byte chunk (col / 8) xor (row % 8); this
        // thread's 16 columns are chunks 2 seg and 2 seg + 1 of its rows
        const int r0 = kk, r1 = kk + 64;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int ch16 = 2 * seg + h;
          uint4 vch, vcl, vsh, vsl;
          vch.x = ch[8 * h + 0] | ((uint32_t)ch[8 * h + 1] << 16);
          vch.y = ch[8 * h + 2] | ((uint32_t)ch[8 * h + 3] << 16);
          vch.z = ch[8 * h + 4] | ((uint32_t)ch[8 * h + 5] << 16);
          vch.w = ch[8 * h + 6] | ((uint32_t)ch[8 * h + 7] << 16);
          vcl.x = cl[8 * h + 0] | ((uint32_t)cl[8 * h + 1] << 16);
          vcl.y = cl[8 * h + 2] | ((uint32_t)cl[8 * h + 3] << 16);
          vcl.z = cl[8 * h + 4] | ((uint32_t)cl[8 * h + 5] << 16);
          vcl.w = cl[8 * h + 6] | ((uint32_t)cl[8 * h + 7] << 16);
          vsh.x = sh[8 * h + 0] | ((uint32_t)sh[8 * h + 1] << 16);
          vsh.y = sh[8 * h + 2] | ((uint32_t)sh[8 * h + 3] << 16);
          vsh.z = sh[8 * h + 4] | ((uint32_t)sh[8 * h + 5] << 16);
          vsh.w = sh[8 * h + 6] | ((uint32_t)sh[8 * h + 7] << 16);
          vsl.x = sl[8 * h + 0] | ((uint32_t)sl[8 * h + 1] << 16);
          vsl.y = sl[8 * h + 2] | ((uint32_t)sl[8 * h + 3] << 16);
          vsl.z = sl[8 * h + 4] | ((uint32_t)sl[8 * h + 5] << 16);
          vsl.w = sl[8 * h + 6] | ((uint32_t)sl[8 * h + 7] << 16);
          const int o0 = r0 * 128 + ((ch16 ^ (r0 & 7)) << 4);
          const int o1 = r1 * 128 + ((ch16 ^ (r1 & 7)) << 4);
          *reinterpret_cast<uint4*>(sAh + o0) = vch;
          *reinterpret_cast<uint4*>(sAl + o0) = vcl;
          *reinterpret_cast<uint4*>(sAh + o1) = vsh;
          *reinterpret_cast<uint4*>(sAl + o1) = vsl;
        }
      }
      // the writes reach the tensor cores' (async) proxy, then the warp's
      // share of the stage is reported
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&gen_full[s]);
      if (c == chunks - 1) {
        // epilogue of the pass: this thread reads lane erow, columns
        // ehalf * 128 .. + 128, once all of the pass's products are done
        if (!__all_sync(0xffffffffu, mbar_wait_role(acc_full, pass & 1, fail))) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int jcol0 = pass * kVisNP + ehalf * 128;
        for (int cb = 0; cb < 128; cb += 16) {
          uint32_t r[16];
          const uint32_t taddr =
              tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(ehalf * 128 + cb);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
              "%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int jb = jcol0 + cb;
          // v-phase 2 v Y_jb at the block start, then rotations over the 16 columns
          float sn, cs;
          sincospif(half_turns(va + (uint64_t)jb * vb), &sn, &cs);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float D = (jb + e < a.ny) ? __uint_as_float(r[e]) : 0.f;
            accP = fmaf(cs, D, accP);
            accQ = fmaf(sn, D, accQ);
            const float cn = fmaf(cs, vrot_c, -sn * vrot_s);
            sn = fmaf(sn, vrot_c, cs * vrot_s);
            cs = cn;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
      }
    }
  }
  __syncthreads();
  const bool ok = *fail == 0;
  // combine: rows kk (C) and kk + 64 (S), two column halves each
  if (tid < kGenThreads) {
    red[ehalf * 256 + erow * 2 + 0] = accP;
    red[ehalf * 256 + erow * 2 + 1] = accQ;
  }
  __syncthreads();
  if (tid < kVisUV && ok) {
    const int64_t k = uv0 + tid;
    if (k < a.K) {
      float P1 = 0, P2 = 0, Q1 = 0, Q2 = 0;  // sum cC, sum sC, sum sS, sum cS
      for (int hh = 0; hh < 2; ++hh) {
        P1 += red[hh * 256 + tid * 2 + 0];
        P2 += red[hh * 256 + tid * 2 + 1];
        Q2 += red[hh * 256 + (tid + 64) * 2 + 0];
        Q1 += red[hh * 256 + (tid + 64) * 2 + 1];
      }
      const double f = a.dx * a.dy / a.scale;
      a.V[2 * k] = ((double)P1 - (double)Q1) * f;
      a.V[2 * k + 1] = -((double)P2 + (double)Q2) * f;
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kVisNP));
  }
}

}  // namespace bhrt

using namespace bhrt;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Normalised amplitudes of Eq. (109), |V_k| / |V(0,0)|, with V(0,0) = F =
// sum_ij I_ij dX dY (Eq. 92) accumulated in FP64 by one block in a fixed order
// (so repeated calls agree bit for bit), then one amplitude per thread.
constexpr int kNormThreads = 1024;
__global__ void __launch_bounds__(kNormThreads) vis_norm_kernel(const float* __restrict__ I,
                                                                int64_t npix, double dA,
                                                                const double* __restrict__ V,
                                                                int64_t K, double* __restrict__ Vn) {
  __shared__ double part[kNormThreads / 32];
  __shared__ double F;
  double acc = 0.0;
  for (int64_t p = threadIdx.x; p < npix; p += kNormThreads) acc += (double)I[p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNormThreads / 32; ++w) t += part[w];
    F = fabs(t * dA);
  }
  __syncthreads();
  const double f = F;
  for (int64_t k = threadIdx.x; k < K; k += kNormThreads)
    Vn[k] = sqrt(V[2 * k] * V[2 * k] + V[2 * k + 1] * V[2 * k + 1]) / f;
}

extern "C" {

bh_status bh_visibilities_workspace_size(const bh_camera* cam, size_t* bytes) {
  if (!cam || !bytes || cam->nx < 1 || cam->ny < 1) return BH_ERR_INVALID_ARG;
  int64_t nxp = ((int64_t)cam->nx + kVisKC - 1) / kVisKC * kVisKC;
  *bytes = a256(sizeof(VisHdr)) + a256((size_t)cam->ny * 2 * nxp * 2);
  return BH_OK;
}

namespace {

bh_status vis_contraction(const float* I, const bh_camera* cam, const double* uv, int64_t K,
                          int32_t mode, double image_max, double* V, double time_budget_s,
                          void* workspace, size_t workspace_bytes, void* stream) {
  if (mode == 0) return bh_visibilities_fp64(I, cam, uv, K, V, stream);
  if (K == 0) return BH_OK;
  size_t need;
  bh_visibilities_workspace_size(cam, &need);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return BH_ERR_WORKSPACE;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return BH_ERR_CUDA;
  VisArgs a;
  a.uv = uv;
  a.K = K;
  a.nx = cam->nx;
  a.ny = cam->ny;
  a.nxp = (cam->nx + kVisKC - 1) / kVisKC * kVisKC;
  a.x_min = cam->x_min;
  a.y_min = cam->y_min;
  a.dx = (cam->x_max - cam->x_min) / cam->nx;
  a.dy = (cam->y_max - cam->y_min) / cam->ny;
  a.scale = 1.0 / image_max;
  a.fp16 = mode == 2;
  a.V = V;
  char* ws = static_cast<char*>(workspace);
  a.hdr = reinterpret_cast<VisHdr*>(ws);
  uint16_t* Bp = reinterpret_cast<uint16_t*>(ws + a256(sizeof(VisHdr)));
  // TMA map of B2: [ny rows][2 nxp] 16-bit, box 64 x 256, 128-byte swizzle
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  cuuint64_t dims[2] = {(cuuint64_t)2 * a.nxp, (cuuint64_t)a.ny};
  cuuint64_t strides[1] = {(cuuint64_t)2 * a.nxp * 2};
  cuuint32_t box[2] = {(cuuint32_t)kVisKC, (cuuint32_t)kVisNP};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = enc(&map, a.fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   2, Bp, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return BH_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  vis_begin<<<1, 1, 0, s>>>(a.hdr, (unsigned long long)(time_budget_s * 1e9));
  vis_prepare_image<<<1216, 256, 0, s>>>(I, a, Bp);
  if (cudaFuncSetAttribute(vis_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kVisSmem) != cudaSuccess)
    return BH_ERR_CUDA;
  const int64_t grid = (K + kVisUV - 1) / kVisUV;
  if (grid > 0x7fffffff) return BH_ERR_INVALID_ARG;
  vis_tc_kernel<<<(unsigned)grid, kVisThreads, kVisSmem, s>>>(map, a);
  return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

}  // namespace

bh_status bh_visibilities(const float* I, const bh_camera* cam, const double* uv, int64_t K,
                          int32_t mode, double image_max, double* V, double* Vnorm,
                          double time_budget_s, void* workspace, size_t workspace_bytes,
                          void* stream) {
  if (!(time_budget_s >= 0.0) || !std::isfinite(time_budget_s)) return BH_ERR_INVALID_ARG;
  if (!I || !cam || K < 0 || (K > 0 && (!uv || !V)) || cam->nx < 1 || cam->ny < 1 ||
      (mode != 0 && mode != 1 && mode != 2) || (mode != 0 && cam->nx > kVisMaxNx) ||
      !(cam->x_max > cam->x_min) || !(cam->y_max > cam->y_min) || !(image_max > 0.0) ||
      !std::isfinite(image_max))
    return BH_ERR_INVALID_ARG;
  bh_status st = vis_contraction(I, cam, uv, K, mode, image_max, V, time_budget_s, workspace,
                                 workspace_bytes, stream);
  if (st != BH_OK || !Vnorm || K == 0) return st;
  const double dA = ((cam->x_max - cam->x_min) / cam->nx) * ((cam->y_max - cam->y_min) / cam->ny);
  vis_norm_kernel<<<1, kNormThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      I, (int64_t)cam->nx * cam->ny, dA, V, K, Vnorm);
  return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

}  // extern "C"
