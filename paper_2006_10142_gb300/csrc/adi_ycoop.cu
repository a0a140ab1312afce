// adi_ycoop.cu -- pass 2 of a step (the column solves Y z = w of Eq. fr2's
// operator, fused with u^{k+1} = 2u^k - u^{k-1} + z) for long columns,
// without thread-block clusters.
//
// The cluster form (y_pipe_kernel) keeps all CTAs of a column strip in one
// cluster and joins their interface systems over distributed shared memory.
// A column of 16384 rows then needs clusters of 16 CTAs, of which only 7
// fit the GPU at a time (112 of 152 SMs).  Here the CTAs of a strip are
// independent CTAs of one persistent grid:
//   - work item = (strip of W = 16 or 32 columns, segment of R = tcol * K rows); the
//     grid's CTAs, all resident (cooperative launch), take items in
//     increasing order, item = strip * C + segment;
//   - each CTA reduces its segment of every column to a two-equation
//     summary (per-thread partition, then block cyclic reduction over the
//     column's chunks by warp shuffles, as in y_solve_cols) and writes it to
//     global memory;
//   - once all C segments of the strip have arrived (one counter per strip:
//     a release-add per column summary, an acquire poll with a bounded
//     wait), every CTA of the strip
//     solves the top systems of all W columns itself (one warp per column,
//     parallel cyclic reduction of 2C equations), so one round trip through
//     L2 per item suffices, and unwinds its own segment;
//   - the TMA pipeline of y_pipe_kernel is kept: the next item's w and m
//     tiles stream into shared memory while the current item is solved, and
//     its u^k, u^{k-1} boxes are prefetched into L2 once the current item's
//     strip is complete (prefetched a whole item ahead, a part was evicted
//     before use: 19.9 read bytes per point against 16).
// Every wait ends: a CTA waits only for the items of its own strip, and the
// lowest-numbered waiting item's missing strip-mates are either running or
// queued behind lower-numbered items on resident CTAs that do not wait for
// it.  The last CTA to finish a strip resets the strip's counters for the
// next launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "adi_bodies.cuh"
#include "adi_device.cuh"
#include "adi_internal.h"
#include "adi_sweeps.cuh"
#include "adi_tma.cuh"

namespace adi {

__device__ __forceinline__ void red_release_gpu_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared-memory layout of one CTA (byte offsets; the stage follows the
// mbarrier at the next 128-byte boundary).
struct YCoopLayout {
  int off_nodes, off_xtop, off_bar;
  size_t bytes;
};

__host__ __device__ inline YCoopLayout y_coop_layout(int W, int tcol, int K, int C) {
  const int threads = W * tcol;
  YCoopLayout L;
  size_t off = align64((size_t)threads * sizeof(Seg<float>));  // chunk summaries / end values
  L.off_nodes = (int)off;
  off += align64((size_t)(threads / 32) * 31 * sizeof(Node<float>));
  L.off_xtop = (int)off;
  off += align64((size_t)W * C * 2 * sizeof(float));          // top-system solutions
  L.off_bar = (int)off;
  off += 8 + 128 + (size_t)2 * tcol * K * W * sizeof(float);   // mbarrier, w and m tiles
  L.bytes = off;
  return L;
}

// K = 16 (and CTAs of 256 threads) run two CTAs per SM (64 registers per
// thread at 512 threads); K = 32 with 512 threads one.
template <int K, int MAXT, int W, bool ADJ>
__global__ void __launch_bounds__(MAXT, (MAXT <= 256 || K == 16) ? 2 : 1)
    y_coop_kernel(const YArgs a, const YCoop yc, const __grid_constant__ CUtensorMap tm_w,
                  const __grid_constant__ CUtensorMap tm_m, const __grid_constant__ CUtensorMap tm_uc,
                  const __grid_constant__ CUtensorMap tm_up) {
  constexpr int QG = 32 / W;  // row groups (q) per warp (W = 16 or 32)
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int lg = a.log2tcol;  // tree levels over a column's chunks (tcol <= 32)
  const int tcol = 1 << lg;
  const int R = tcol * K;     // rows of a segment (a power of two >= 64)
  const int C = yc.C;         // segments per column (<= 32)
  const int BH = R < 256 ? R : 256;
  const int nbox = R / BH;
  const int nstrips = (a.nx + W - 1) / W;
  const int nitems = nstrips * C;
  const YCoopLayout Lo = y_coop_layout(W, tcol, K, C);
  Seg<float>* csum = reinterpret_cast<Seg<float>*>(smem);
  Node<float>* nodes = reinterpret_cast<Node<float>*>(smem + Lo.off_nodes) + warp * 31;
  float* xtop = reinterpret_cast<float*>(smem + Lo.off_xtop);
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sa + (uint32_t)Lo.off_bar;
  const uint32_t st_w = (bar + 8u + 127u) & ~127u;
  const uint32_t st_m = st_w + (uint32_t)(R * W * 4);
  const float* sw = reinterpret_cast<const float*>(smem + (st_w - sa));
  const float* smv = reinterpret_cast<const float*>(smem + (st_m - sa));
  const size_t ld = (size_t)a.ld;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  // warp 0: the TMA boxes of item `it` (one box per lane)
  auto issue = [&](int it) {
    const int strip = it / C, seg = it - (it / C) * C;
    const int row0 = seg * R;
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(2 * R * W * 4));
    for (int t = lane; t < 2 * nbox; t += 32) {
      const int b = t >> 1;
      const uint32_t off = (uint32_t)(b * BH * W * 4);
      if ((t & 1) == 0) tma_load_2d(st_w + off, &tm_w, strip * W, row0 + b * BH, bar);
      else tma_load_2d(st_m + off, &tm_m, strip * W, row0 + b * BH, bar);
    }
  };
  // warp 0: L2 prefetch of the u^k and u^{k-1} boxes item `it` updates
  // (issued for the next item once the current one's strip is complete,
  // about half an item ahead of the update that reads them)
  auto prefetch_u = [&](int it) {
    const int strip = it / C, seg = it - (it / C) * C;
    const int row0 = seg * R;
    for (int t = lane; t < 2 * nbox; t += 32) {
      const int b = t >> 1;
      if ((t & 1) == 0) tma_prefetch_2d(&tm_uc, strip * W, row0 + b * BH);
      else tma_prefetch_2d(&tm_up, strip * W, row0 + b * BH);
    }
  };
  int item = blockIdx.x;
  if (tid < 32) {
    if (lane == 0) prefetch_tensormap(&tm_w);
    if (lane == 1) prefetch_tensormap(&tm_m);
    if (!ADJ && lane == 2) prefetch_tensormap(&tm_uc);
    if (!ADJ && lane == 3) prefetch_tensormap(&tm_up);
    if (item < nitems) issue(item);
  }
  const int col = tid & (W - 1);
  const int q = tid / W;
  const int qq = q & (QG - 1);
  // the column / chunk this lane reduces in the column trees
  const int tc = warp * (32 >> lg) + (lane >> lg);
  const int chunk = lane & (tcol - 1);
  uint32_t phase = 0;
  bool timed_out = false;
  bool bad = false;
  const float sc = (float)a.sc;
  for (; item < nitems; item += gridDim.x) {
    const int strip = item / C;
    const int seg = item - strip * C;
    const int i = strip * W + col;
    const bool colok = i < a.nx;
    if (!mbar_wait_bounded(bar, phase, 1000000000ull)) timed_out = true;
    phase ^= 1u;
    // rows read in blocks of QG, the two row groups of a warp in XOR order
    // (conflict-free, see y_pipe_kernel), put back in order by selects
    float d[K], s[K];
#pragma unroll
    for (int g = 0; g < K; g += QG) {
      float vw[QG], vm[QG];
#pragma unroll
      for (int r = 0; r < QG; ++r) {
        const int o = (q * K + g + (r ^ qq)) * W + col;
        vw[r] = sw[o];
        vm[r] = smv[o];
      }
#pragma unroll
      for (int b = 1; b < QG; b <<= 1) {
        const bool x = (qq & b) != 0;
#pragma unroll
        for (int r = 0; r < QG; ++r) {
          if ((r & b) == 0) {
            const float w0 = vw[r], w1 = vw[r | b], m0 = vm[r], m1 = vm[r | b];
            vw[r] = x ? w1 : w0;
            vw[r | b] = x ? w0 : w1;
            vm[r] = x ? m1 : m0;
            vm[r | b] = x ? m0 : m1;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < QG; ++r) {
        d[g + r] = colok ? (ADJ ? vm[r] * vw[r] : vw[r]) : 0.f;
        s[g + r] = colok ? sc * vm[r] : 0.f;
      }
    }
    __syncthreads();  // the stage is consumed: refill it with the next item
    const int next = item + (int)gridDim.x;
    if (tid < 32 && next < nitems) {
      fence_proxy_async_smem();
      issue(next);
    }
    // 1. partition: each thread's K rows to a two-equation summary
    Node<float> ndc;
    {
      Seg<float> S;
      chunk_reduce_split<K, float>(d, s, S, ndc);
      csum[col * tcol + q] = S;
    }
    __syncthreads();
    // 2. the segment of each column to one summary (tree over its chunks),
    // to global memory; the lane that stores a column's summary arrives on
    // the strip's counter with release semantics (its own store first), so
    // the counter reaches C * W when every summary of the strip is visible
    {
      Seg<float> S = csum[tc * tcol + chunk];
      S = warp_tree_up<float>(S, nodes, lane, lg);
      if (chunk == 0) {
        float4* dst = reinterpret_cast<float4*>(yc.tops + (((size_t)strip * W + tc) * C + seg) * 8);
        __stcg(dst, make_float4(S.f.a, S.f.b, S.f.c, S.f.d));
        __stcg(dst + 1, make_float4(S.l.a, S.l.b, S.l.c, S.l.d));
        red_release_gpu_add(yc.sync + 2 * strip, 1);
      }
    }
    if (tid == 0) {
      const int* cnt = yc.sync + 2 * strip;
      const int target = C * W;
      if (ld_acquire_gpu(cnt) < target) {
        const uint64_t t0 = global_ns();
        while (ld_acquire_gpu(cnt) < target) {
          if (global_ns() - t0 > 1000000000ull) {
            timed_out = true;
            break;
          }
          __nanosleep(32);
        }
      }
    }
    __syncthreads();
    if (!ADJ && tid < 32 && next < nitems) prefetch_u(next);
    // 3. the top systems of all W columns of the strip, one warp per column
    for (int c = warp; c < W; c += nwarps) {
      Eq<float> E0 = eq_identity<float>(), E1 = eq_identity<float>();
      if (lane < C) {
        const float4* srcp = reinterpret_cast<const float4*>(yc.tops + (((size_t)strip * W + c) * C + lane) * 8);
        const float4 f = __ldcg(srcp), l = __ldcg(srcp + 1);
        E0.a = f.x; E0.b = f.y; E0.c = f.z; E0.d = f.w;
        E1.a = l.x; E1.b = l.y; E1.c = l.z; E1.d = l.w;
      }
      pcr64<float>(E0, E1, lane, 2 * C);
      if (lane < C) {
        xtop[2 * (c * C + lane)] = div_t(E0.d, E0.b);
        xtop[2 * (c * C + lane) + 1] = div_t(E1.d, E1.b);
      }
    }
    __syncthreads();
    // every read of this strip's summaries and counter is done: the last CTA
    // of the strip resets its counters for the next launch
    // completion count of the strip (its reply is first needed after the
    // update, so the round trip overlaps the rest of the item)
    int done_before = 0;
    if (tid == 0) done_before = atomicAdd(yc.sync + 2 * strip + 1, 1);
    // 4. down the column trees to each chunk's end values, back substitution
    {
      float xa = xtop[2 * (tc * C + seg)];
      float xc = xtop[2 * (tc * C + seg) + 1];
      warp_tree_down<float>(nodes, lane, lg, xa, xc);
      float* cx = reinterpret_cast<float*>(csum + tc * tcol + chunk);
      cx[0] = xa;
      cx[1] = xc;
    }
    __syncthreads();
    {
      const float* mine = reinterpret_cast<const float*>(csum + col * tcol + q);
      chunk_backsub_split<K, float>(d, s, ndc, mine[0], mine[1]);
    }
    // 5. epilogue (as in y_pipe_kernel)
    const int j0 = seg * R + q * K;
    if (ADJ) {
      if (colok) {
        const size_t base = (size_t)j0 * ld + i;
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (j0 + k < a.ny) a.z_out[base + k * ld] = d[k] * rcp_t(__ldg(a.m + base + k * ld));
      }
    } else if (colok) {
      const size_t base = (size_t)j0 * ld + i;
      float chk = 0.f;
      if (j0 + K <= a.ny) {
        constexpr int EG = K < 16 ? K : 16;
#pragma unroll
        for (int g = 0; g < K; g += EG) {
          float uc[EG], up[EG];
#pragma unroll
          for (int k = 0; k < EG; ++k) {
            uc[k] = __ldcg(a.u_cur + base + (g + k) * ld);
            up[k] = __ldcg(a.u_prev + base + (g + k) * ld);
          }
#pragma unroll
          for (int k = 0; k < EG; ++k) {
            const float un = 2.0f * uc[k] - up[k] + d[g + k];
            a.u_prev[base + (g + k) * ld] = un;
            chk += un - un;
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (j0 + k < a.ny) {
            const float un = 2.0f * __ldcg(a.u_cur + base + k * ld) - __ldcg(a.u_prev + base + k * ld) + d[k];
            a.u_prev[base + k * ld] = un;
            chk += un - un;
          }
        }
      }
      if (a.z_out != nullptr) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (j0 + k < a.ny) a.z_out[base + k * ld] = d[k];
      }
      bad |= chk != 0.f;
    }
    if (!ADJ && item == 0 && tid == 0 && a.gd) a.gd->k += 1;
    // every CTA of the strip has read its summaries and counter: the last
    // one resets the counters for the next launch
    if (tid == 0 && done_before == C - 1) {
      yc.sync[2 * strip] = 0;
      yc.sync[2 * strip + 1] = 0;
    }
    __syncthreads();  // csum and xtop are reused by the next item
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_NUMERIC);
  if (__any_sync(0xffffffffu, timed_out) && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_TIMEOUT);
}

size_t y_coop_smem_bytes(int W, int tcol, int K, int C) { return y_coop_layout(W, tcol, K, C).bytes; }

int y_coop_segments(int ny, int tcol, int K) { return (ny + tcol * K - 1) / (tcol * K); }

template <int K, int MAXT, int W, bool ADJ>
static cudaError_t launch_y_coop_t(const YArgs& a, const YCoop& yc, const YMaps& mp, cudaStream_t st) {
  const int tcol = 1 << a.log2tcol;
  const int threads = W * tcol;
  if ((1 << a.log2W) != W || threads != MAXT || tcol > 32 || tcol * K < 64) return cudaErrorInvalidValue;
  if (yc.C < 1 || yc.C > 32 || yc.C != y_coop_segments(a.ny, tcol, K)) return cudaErrorInvalidValue;
  // scratch: summaries of every column (rounded up to the strip) and two
  // counters per strip
  const int strips = (a.nx + W - 1) / W;
  if (yc.tops == nullptr || yc.sync == nullptr || yc.cols < strips * W || yc.strips < strips)
    return cudaErrorInvalidValue;
  const size_t sm = y_coop_smem_bytes(W, tcol, K, yc.C);
  if (sm > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  auto kern = y_coop_kernel<K, MAXT, W, ADJ>;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int nitems = strips * yc.C;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(1, std::min(nitems, nsm * per_sm)), 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, yc, mp.w, mp.m, mp.uc, mp.up);
}

template <bool ADJ>
static cudaError_t launch_y_coop_any(const YArgs& a, int K, const YCoop& yc, const YMaps& mp,
                                     cudaStream_t st) {
  const int W = 1 << a.log2W;
  const int threads = W << a.log2tcol;
  if (W == 16 && K == 32 && threads == 256) return launch_y_coop_t<32, 256, 16, ADJ>(a, yc, mp, st);
  if (W == 16 && K == 32 && threads == 512) return launch_y_coop_t<32, 512, 16, ADJ>(a, yc, mp, st);
  if (W == 16 && K == 16 && threads == 512) return launch_y_coop_t<16, 512, 16, ADJ>(a, yc, mp, st);
  if (W == 32 && K == 32 && threads == 512) return launch_y_coop_t<32, 512, 32, ADJ>(a, yc, mp, st);
  if (W == 32 && K == 16 && threads == 512) return launch_y_coop_t<16, 512, 32, ADJ>(a, yc, mp, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_y_coop(const YArgs& a, int K, const YCoop& yc, const YMaps& mp, cudaStream_t st) {
  return launch_y_coop_any<false>(a, K, yc, mp, st);
}

cudaError_t launch_y_coop_adj(const YArgs& a, int K, const YCoop& yc, const CUtensorMap& lam,
                              const CUtensorMap& m, cudaStream_t st) {
  if (a.z_out == nullptr || a.m == nullptr) return cudaErrorInvalidValue;
  YMaps mp;
  mp.w = lam;
  mp.m = m;
  mp.uc = m;
  mp.up = m;
  return launch_y_coop_any<true>(a, K, yc, mp, st);
}

static cudaError_t allow(const void* kern) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

cudaError_t configure_y_coop_kernels() {
  cudaError_t e = cudaSuccess;
#define ADI_COOP_CFG(K, T, W)                                                        \
  if (e == cudaSuccess) e = allow((const void*)y_coop_kernel<K, T, W, false>);       \
  if (e == cudaSuccess) e = allow((const void*)y_coop_kernel<K, T, W, true>);
  ADI_COOP_CFG(32, 256, 16)
  ADI_COOP_CFG(32, 512, 16)
  ADI_COOP_CFG(16, 512, 16)
  ADI_COOP_CFG(32, 512, 32)
  ADI_COOP_CFG(16, 512, 32)
#undef ADI_COOP_CFG
  return e;
}

}  // namespace adi
