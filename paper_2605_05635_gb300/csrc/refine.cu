// refine.cu -- adaptive screen refinement and image assembly.
//
// The paper refines the screen near the shadow boundary, the critical curve
// and the higher-order image regions (Introduction; Sec. 3.3 and Sec. 4)
// without fixing a rule.  Rule implemented here (a documented reading):
//   class(cell) = (status, N_cross);
//   a base pixel is refined iff its class differs from one of its on-screen
//   4-neighbours; a refined cell spawns 4x4 children at cell-centred
//   offsets; a child at level L < levels is refined iff its class differs
//   from a 4-neighbour among its 16 siblings;
//   the pixel value is the recursive mean of its children's values, and an
//   unrefined cell takes the value of its own ray.
// Children of one parent are stored as 16 consecutive list entries in digit
// order (digit = 4*row + col), so siblings are found by index arithmetic.
// Each block compacts its marked cells in shared memory and reserves list
// space with one atomic, then writes the children cooperatively (coalesced).
#include <cuda_runtime.h>

#include "internal.h"

namespace bhrt {

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem, int& total) {
  // smem: at least blockDim.x/32 + 1 ints
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) smem[lane] = w;
  }
  __syncthreads();
  int before = (warp > 0 ? smem[warp - 1] : 0) + x - v;
  total = smem[nw - 1];
  __syncthreads();
  return before;
}

constexpr int kRefineThreads = 256;

// Marks the cells of `level` and appends 16 children per marked cell to the
// list of level + 1.
__global__ void __launch_bounds__(kRefineThreads) mark_expand_kernel(RefineArgs a, int level) {
  __shared__ int s_scan[kRefineThreads / 32 + 1];
  __shared__ uint64_t s_key[kRefineThreads];
  __shared__ uint32_t s_img[kRefineThreads];
  __shared__ unsigned long long s_base;
  const bool base_level = level == 0;
  int64_t n;
  if (base_level) {
    n = (int64_t)a.n_img * a.npix;
  } else {
    unsigned long long c = a.hdr->count[level];
    n = (int64_t)(c < (unsigned long long)a.lv[level].cap ? c : (unsigned long long)a.lv[level].cap);
  }
  LevelRecs& nxt = a.lv[level + 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t start = (int64_t)blockIdx.x * blockDim.x; start < n; start += stride) {
    int64_t q = start + threadIdx.x;
    int marked = 0;
    uint64_t key = 0;
    uint32_t img = 0;
    if (q < n) {
      if (base_level) {
        img = (uint32_t)(q / a.npix);
        int64_t pix = q - (int64_t)img * a.npix;
        const ImgParams& ip = a.ip[img];
        int i = (int)(pix % ip.nx), j = (int)(pix / ip.nx);
        const uint16_t* cls = a.base_cls + (int64_t)img * a.npix;
        uint16_t c = cls[pix];
        if (i > 0 && cls[pix - 1] != c) marked = 1;
        if (i + 1 < ip.nx && cls[pix + 1] != c) marked = 1;
        if (j > 0 && cls[pix - ip.nx] != c) marked = 1;
        if (j + 1 < ip.ny && cls[pix + ip.nx] != c) marked = 1;
        key = (uint64_t)pix << 16;
      } else {
        const LevelRecs& cur = a.lv[level];
        int dgt = (int)(q & 15);
        int64_t g0 = q - dgt;
        int cx = dgt & 3, cy = dgt >> 2;
        uint16_t c = cur.cls[q];
        if (cx > 0 && cur.cls[g0 + dgt - 1] != c) marked = 1;
        if (cx < 3 && cur.cls[g0 + dgt + 1] != c) marked = 1;
        if (cy > 0 && cur.cls[g0 + dgt - 4] != c) marked = 1;
        if (cy < 3 && cur.cls[g0 + dgt + 4] != c) marked = 1;
        key = cur.key[q];
        img = cur.img[q];
      }
    }
    int total;
    int rank = block_exclusive_scan(marked, s_scan, total);
    if (threadIdx.x == 0)
      s_base = total ? atomicAdd(&a.hdr->count[level + 1], 16ull * (unsigned long long)total) : 0ull;
    if (marked) {
      s_key[rank] = key;
      s_img[rank] = img;
    }
    __syncthreads();
    const unsigned long long base = s_base;
    if (q < n) {
      int32_t child = -1;
      if (marked) {
        unsigned long long c0 = base + 16ull * rank;
        if (c0 + 16 <= (unsigned long long)nxt.cap) child = (int32_t)c0;
        else atomicCAS(&a.hdr->status, 0, (int)BH_ERR_QUEUE_OVERFLOW);
      }
      if (base_level) a.base_child[q] = child;
      else a.lv[level].child[q] = child;
    }
    // cooperative, coalesced write of the children
    const int nchild = 16 * total;
    const uint64_t lvbits = (uint64_t)(level + 1) << 12;
    const int shift = 4 * (3 - (level + 1));
    for (int c = threadIdx.x; c < nchild; c += blockDim.x) {
      unsigned long long dst = base + (unsigned long long)c;
      if (dst >= (unsigned long long)nxt.cap) continue;
      uint64_t pk = s_key[c >> 4];
      uint64_t ck = (pk & ~((uint64_t)0xF << 12)) | lvbits | ((uint64_t)(c & 15) << shift);
      nxt.key[dst] = ck;
      nxt.img[dst] = s_img[c >> 4];
    }
    __syncthreads();
  }
}

// Bottom-up assembly: a refined cell's value becomes the mean of its 16
// children (which hold their own final values already); level 0 also
// writes the output planes.
__global__ void __launch_bounds__(kRefineThreads) assemble_kernel(RefineArgs a, int level) {
  const bool base_level = level == 0;
  int64_t n, cap;
  double* I;
  int32_t* child;
  uint8_t* depth;
  if (base_level) {
    n = (int64_t)a.n_img * a.npix;
    cap = n;
    I = a.base_I;
    child = a.base_child;
    depth = a.base_depth;
  } else {
    unsigned long long c = a.hdr->count[level];
    cap = a.lv[level].cap;
    n = (int64_t)(c < (unsigned long long)cap ? c : (unsigned long long)cap);
    I = a.lv[level].I;
    child = a.lv[level].child;
    depth = a.lv[level].depth;
  }
  const bool has_children = level < a.levels;
  const LevelRecs& nxt = a.lv[level + 1 <= kMaxLevels ? level + 1 : kMaxLevels];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    double v[4] = {I[q], I[cap + q], I[2 * cap + q], I[3 * cap + q]};
    int dpt = level;
    if (has_children) {
      int32_t c0 = child[q];
      if (c0 >= 0) {
        double acc[4] = {0, 0, 0, 0};
        const int64_t nc = nxt.cap;
        for (int c = 0; c < 16; ++c) {
#pragma unroll
          for (int t = 0; t < 4; ++t) acc[t] += nxt.I[t * nc + c0 + c];
          int d = nxt.depth[c0 + c];
          dpt = d > dpt ? d : dpt;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          v[t] = acc[t] / 16.0;
          I[t * cap + q] = v[t];
        }
      }
    }
    depth[q] = (uint8_t)dpt;
    if (base_level) {
      uint32_t img = (uint32_t)(q / a.npix);
      int64_t pix = q - (int64_t)img * a.npix;
      const OutPtrs& o = a.out[img];
      o.I[pix] = (float)v[0];
      if (o.I_n) {
        o.I_n[pix] = (float)v[1];
        o.I_n[a.npix + pix] = (float)v[2];
        o.I_n[2 * a.npix + pix] = (float)v[3];
      }
      if (o.refine_level) o.refine_level[pix] = (uint8_t)dpt;
    }
  }
}

// Copies every traced refined cell's key to its image's key list.
__global__ void __launch_bounds__(kRefineThreads) write_keys_kernel(RefineArgs a) {
  for (int level = 1; level <= a.levels; ++level) {
    const LevelRecs& lv = a.lv[level];
    unsigned long long c = a.hdr->count[level];
    int64_t n = (int64_t)(c < (unsigned long long)lv.cap ? c : (unsigned long long)lv.cap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
      const OutPtrs& o = a.out[lv.img[q]];
      if (!o.keys_count) continue;
      unsigned long long pos = atomicAdd(o.keys_count, 1ull);
      if (o.keys && pos < (unsigned long long)o.keys_cap) o.keys[pos] = lv.key[q];
    }
  }
}

__global__ void begin_kernel(WsHeader* hdr, unsigned long long budget_ns) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  hdr->t_start = t;
  hdr->budget_ns = budget_ns;
}

cudaError_t launch_mark_expand(const RefineArgs& a, int level, int blocks, cudaStream_t st) {
  mark_expand_kernel<<<blocks, kRefineThreads, 0, st>>>(a, level);
  return cudaGetLastError();
}
cudaError_t launch_assemble(const RefineArgs& a, int level, int blocks, cudaStream_t st) {
  assemble_kernel<<<blocks, kRefineThreads, 0, st>>>(a, level);
  return cudaGetLastError();
}
cudaError_t launch_write_keys(const RefineArgs& a, int blocks, cudaStream_t st) {
  write_keys_kernel<<<blocks, kRefineThreads, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_begin(WsHeader* hdr, unsigned long long budget_ns, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return e;
  begin_kernel<<<1, 1, 0, st>>>(hdr, budget_ns);
  return cudaGetLastError();
}

}  // namespace bhrt
