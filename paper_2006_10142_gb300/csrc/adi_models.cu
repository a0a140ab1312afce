// adi_models.cu -- the problem class of Section 2 beyond the workloads, and
// the paper's literal sub-schemes, on the same line solvers.
//
// mode 0, Eq. (CN1) with a time-dependent coefficient m^k = g_k m(x, y) (the
//   c(t) of Eq. f1) and a source field f^k(x, y).  CN1 weighs Lap u^{k+1} by
//   m^{k+1}/2 and Lap u^{k-1} by m^{k-1}/2; with z = u^{k+1} - 2u^k + u^{k-1}
//     (I - S Lap) z = tau^2 (g_{k+1} m Lap u^k + (g_{k-1} - g_{k+1})/2 m Lap u^{k-1} + f^k),
//   S = tau^2 g_{k+1} m / 2, factored as (I - S Lap_x)(I - S Lap_y): the x
//   pass forms the right-hand side and solves the rows, the y pass solves
//   the columns and updates u^{k+1} = 2u^k - u^{k-1} + z over u^{k-1}.
// modes 1 and 2, the two sub-problems over half time levels (Algorithm 1's
//   u, U0, Ux, Uy = u^{k-1/2}, u^k, u^{k+1/2}, u^{k+1}):
//     (I - beta S Lap_x) u^{k+1/2} = 2u^k - u^{k-1/2} + alpha S Lap_x u^{k-1/2} + tau^2 f^k
//     (I - beta S Lap_y) u^{k+1}   = 2u^{k+1/2} - u^k + alpha S Lap_y u^k + tau^2 f^{k+1/2}
//   with S = tau^2 m / 2: mode 1 (Eqs. fr1, fr2 as printed) alpha = beta = 1;
//   mode 2 (Listing 1's systems a = c = tau^2, b = 2 tau^2 + h^2 with the
//   coefficient m, right-hand side from u_old and u^k only) alpha = 0,
//   beta = 2.  The point source at the half level is the mean of the
//   samples at k and k + 1.
// The kernels load their operands directly (no TMA pipeline) and solve with
// the tree solver of adi_sweeps.cuh: rows in one CTA, columns over a
// thread-block cluster.  The level k is a kernel argument; the host advances
// the grid record's level after the step (advance_level_kernel).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "adi_device.cuh"
#include "adi_internal.h"
#include "adi_sweeps.cuh"

namespace adi {

__device__ __forceinline__ float level_hold(const float* g, int n, long long k) {
  if (g == nullptr || n <= 0) return 1.f;
  if (k < 0) return g[0];
  return k < n ? g[k] : g[n - 1];
}

__device__ __forceinline__ float wavelet_at(const GridDev* gd, long long k) {
  return (gd->wavelet != nullptr && k >= 0 && k < gd->n_wavelet) ? gd->wavelet[k] : 0.f;
}

template <int K, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 2 : 1) x_model_kernel(const ModelXArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tsys = 1 << a.log2tsys;
  const int tid = threadIdx.x;
  const int sys = tid >> a.log2tsys;
  const int p = tid & (tsys - 1);
  const int j = blockIdx.x * a.spc + sys;
  const int i0 = p * K;
  const bool active = j < a.ny && i0 < a.nx;
  const size_t ld = (size_t)a.ld;
  const size_t row = (size_t)j * ld;
  float d[K], s[K];
  if (active) {
    const float cx = (float)a.cx, cy = (float)a.cy, sc = (float)a.sc;
    float A[K], B[K], M[K];
    load_vec<K>(A, a.a + row + i0);
    load_vec<K>(M, a.m + row + i0);
    const float aL = i0 > 0 ? __ldg(a.a + row + i0 - 1) : 0.f;
    const float aR = i0 + K < a.nx ? __ldg(a.a + row + i0 + K) : 0.f;
    if (a.mode == 0) {
      // Lap u^k (B) and Lap u^{k-1} (A), both five-point
      load_vec<K>(B, a.b + row + i0);
      const float bL = i0 > 0 ? __ldg(a.b + row + i0 - 1) : 0.f;
      const float bR = i0 + K < a.nx ? __ldg(a.b + row + i0 + K) : 0.f;
      float vb[K], va[K];
#pragma unroll
      for (int k = 0; k < K; ++k) { vb[k] = 0.f; va[k] = 0.f; }
      if (j > 0) {
        float t[K];
        load_vec<K>(t, a.b + row - ld + i0);
#pragma unroll
        for (int k = 0; k < K; ++k) vb[k] += t[k];
        load_vec<K>(t, a.a + row - ld + i0);
#pragma unroll
        for (int k = 0; k < K; ++k) va[k] += t[k];
      }
      if (j + 1 < a.ny) {
        float t[K];
        load_vec<K>(t, a.b + row + ld + i0);
#pragma unroll
        for (int k = 0; k < K; ++k) vb[k] += t[k];
        load_vec<K>(t, a.a + row + ld + i0);
#pragma unroll
        for (int k = 0; k < K; ++k) va[k] += t[k];
      }
      const float gn = level_hold(a.g, a.n_g, a.level + 1);
      const float gp = level_hold(a.g, a.n_g, a.level - 1);
      const float* fk = (a.f != nullptr && a.level >= 0 && a.level < a.n_f)
                            ? a.f + (size_t)a.level * a.nx * a.ny + (size_t)j * a.nx : nullptr;
      const float tau2 = (float)a.tau2;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float bl = k > 0 ? B[k - 1] : bL, br = k < K - 1 ? B[k + 1] : bR;
        const float al = k > 0 ? A[k - 1] : aL, ar = k < K - 1 ? A[k + 1] : aR;
        const float lapc = cx * (bl + br - 2.f * B[k]) + cy * (vb[k] - 2.f * B[k]);
        const float lapp = cx * (al + ar - 2.f * A[k]) + cy * (va[k] - 2.f * A[k]);
        const bool in = i0 + k < a.nx;
        d[k] = in ? M[k] * (gn * lapc + 0.5f * (gp - gn) * lapp) + (fk ? tau2 * fk[i0 + k] : 0.f) : 0.f;
        s[k] = in ? sc * gn * M[k] : 0.f;
      }
    } else {
      load_vec<K>(B, a.b + row + i0);
      const float alpha = a.mode == 1 ? 1.f : 0.f;
      const float beta = a.mode == 1 ? 1.f : 2.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float al = k > 0 ? A[k - 1] : aL, ar = k < K - 1 ? A[k + 1] : aR;
        const bool in = i0 + k < a.nx;
        d[k] = in ? 2.f * B[k] - A[k] + alpha * sc * M[k] * (al + ar - 2.f * A[k]) : 0.f;
        s[k] = in ? beta * sc * M[k] : 0.f;
      }
    }
    // point source: tau^2 w(t_k) / (h1 h2)
    const GridDev* gd = a.gd;
    if (j == gd->src_iy && gd->src_ix >= i0 && gd->src_ix < i0 + K) {
      const float f = (float)a.src_scale * wavelet_at(gd, a.level);
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (i0 + k == gd->src_ix) d[k] += f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) { d[k] = 0.f; s[k] = 0.f; }
  }
  x_solve_rows<K, float, true>(smem, a.spc, a.log2tsys, 32, sys, p, d, s);
  if (active) store_vec<K, float>(a.out + row + i0, d);
}

template <int K, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 2 : 1) y_model_kernel(const ModelYArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int C = a.C;
  cluster_arrive_early(C);
  const int W = 1 << a.log2W;
  const int tcol = 1 << a.log2tcol;
  const int tid = threadIdx.x;
  const int col = tid & (W - 1);
  const int q = tid >> a.log2W;
  const int rank = cluster_rank(C);
  const int strip = blockIdx.x / C;
  const int gq = rank * tcol + q;
  const int i = strip * W + col;
  const int j0 = gq * K;
  const bool colok = i < a.nx;
  const size_t ld = (size_t)a.ld;
  const size_t base = (size_t)j0 * ld + i;
  const float sc = (float)a.sc;
  float d[K], s[K];
  if (a.mode == 0) {
    const float gn = level_hold(a.g, a.n_g, a.level + 1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ok = colok && j0 + k < a.ny;
      d[k] = ok ? __ldg(a.w + base + k * ld) : 0.f;
      s[k] = ok ? sc * gn * __ldg(a.m + base + k * ld) : 0.f;
    }
  } else {
    const float alpha = a.mode == 1 ? 1.f : 0.f;
    const float beta = a.mode == 1 ? 1.f : 2.f;
    float bprev = (colok && j0 > 0 && j0 - 1 < a.ny) ? __ldg(a.b + base - ld) : 0.f;
    float bcur = (colok && j0 < a.ny) ? __ldg(a.b + base) : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ok = colok && j0 + k < a.ny;
      const float bnext = (colok && j0 + k + 1 < a.ny) ? __ldg(a.b + base + (k + 1) * ld) : 0.f;
      const float mk = ok ? __ldg(a.m + base + k * ld) : 0.f;
      d[k] = ok ? 2.f * __ldg(a.w + base + k * ld) - bcur + alpha * sc * mk * (bprev + bnext - 2.f * bcur) : 0.f;
      s[k] = ok ? beta * sc * mk : 0.f;
      bprev = bcur;
      bcur = bnext;
    }
    // point source at the half level: tau^2 (w(t_k) + w(t_{k+1})) / (2 h1 h2)
    const GridDev* gd = a.gd;
    if (i == gd->src_ix && gd->src_iy >= j0 && gd->src_iy < j0 + K) {
      const float f = 0.5f * (float)a.src_scale * (wavelet_at(gd, a.level) + wavelet_at(gd, a.level + 1));
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (j0 + k == gd->src_iy) d[k] += f;
    }
  }
  y_solve_cols<K, float, true>(smem, a.log2W, a.log2tcol, C, rank, 32, col, gq, d, s);
  if (!colok) return;
  float chk = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (j0 + k < a.ny) {
      const size_t idx = base + k * ld;
      const float un = a.mode == 0 ? 2.f * __ldg(a.b + idx) - a.io[idx] + d[k] : d[k];
      a.io[idx] = un;
      chk += un - un;
    }
  }
  if (__any_sync(__activemask(), chk != 0.f) && a.err) atomicOr(a.err, ERR_NUMERIC);
}

__global__ void advance_level_kernel(GridDev* gd) { gd->k += 1; }

template <int K, int MAXT>
static cudaError_t launch_xm_t(const ModelXArgs& a, cudaStream_t st) {
  const int threads = a.spc << a.log2tsys;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;
  const size_t sm = x_smem_bytes(a.spc, 1 << a.log2tsys, false, true);
  x_model_kernel<K, MAXT><<<(a.ny + a.spc - 1) / a.spc, threads, sm, st>>>(a);
  return cudaGetLastError();
}

template <int K, int MAXT>
static cudaError_t launch_ym_t(const ModelYArgs& a, cudaStream_t st) {
  const int W = 1 << a.log2W;
  const int threads = W << a.log2tcol;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(((a.nx + W - 1) / W) * a.C, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = y_smem_bytes(W, a.C, 1 << a.log2tcol, false, true);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, y_model_kernel<K, MAXT>, a);
}

#define ADI_MODEL_DISPATCH(FN, THREADS)                   \
  switch (K) {                                            \
    case 4: return FN<4, 1024>(a, st);                    \
    case 8: return FN<8, 1024>(a, st);                    \
    case 16:                                              \
      if ((THREADS) <= 256) return FN<16, 256>(a, st);    \
      if ((THREADS) <= 512) return FN<16, 512>(a, st);    \
      return FN<16, 1024>(a, st);                         \
    case 32:                                              \
      if ((THREADS) <= 256) return FN<32, 256>(a, st);    \
      return FN<32, 512>(a, st);                          \
  }

cudaError_t launch_x_model(const ModelXArgs& a, int K, cudaStream_t st) {
  const int threads = a.spc << a.log2tsys;
  ADI_MODEL_DISPATCH(launch_xm_t, threads)
  return cudaErrorInvalidValue;
}

cudaError_t launch_y_model(const ModelYArgs& a, int K, cudaStream_t st) {
  const int threads = 1 << (a.log2W + a.log2tcol);
  ADI_MODEL_DISPATCH(launch_ym_t, threads)
  return cudaErrorInvalidValue;
}

cudaError_t launch_advance_level(GridDev* gd, cudaStream_t st) {
  advance_level_kernel<<<1, 1, 0, st>>>(gd);
  return cudaGetLastError();
}

template <typename KernT>
static cudaError_t allow_model(KernT kern) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t configure_model_kernels() {
  cudaError_t e = cudaSuccess;
#define ADI_MODEL_CFG(K, T)                                              \
  if (e == cudaSuccess) e = allow_model(x_model_kernel<K, T>);           \
  if (e == cudaSuccess) e = allow_model(y_model_kernel<K, T>);
  ADI_MODEL_CFG(4, 1024)
  ADI_MODEL_CFG(8, 1024)
  ADI_MODEL_CFG(16, 256)
  ADI_MODEL_CFG(16, 512)
  ADI_MODEL_CFG(16, 1024)
  ADI_MODEL_CFG(32, 256)
  ADI_MODEL_CFG(32, 512)
#undef ADI_MODEL_CFG
  return e;
}

}  // namespace adi
