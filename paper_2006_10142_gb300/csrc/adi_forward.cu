// adi_forward.cu -- forward-step kernels of the factored ADI scheme.
//
// One time step (Eq. CN1 in delta form, factored as in Section 2):
//   pass 1, x_sweep_kernel: r = tau^2 (m Lap u^k + f^k) fused with the row
//           solves X w = r, X = I - S Lap_x (Eq. fr1's operator);
//   pass 2, y_sweep_kernel: the column solves Y z = w, Y = I - S Lap_y
//           (Eq. fr2's operator), fused with u^{k+1} = 2u^k - u^{k-1} + z,
//           written over u^{k-1} (the buffer swap of Algorithm 1).
// Both solve their lines with the cores of adi_sweeps.cuh.  Memory traffic
// per grid point: pass 1 reads u^k and m and writes w (12 B, plus halo rows
// served by L2); pass 2 reads w, m, u^k, u^{k-1} and writes u^{k+1} (20 B).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "adi_bodies.cuh"
#include "adi_device.cuh"
#include "adi_internal.h"
#include "adi_sweeps.cuh"

namespace adi {

// ---------------------------------------------------------------------------
// pass 1: RHS assembly + x solve (adi_bodies.cuh).  CTA = `spc` rows.
// ---------------------------------------------------------------------------
// MAXT bounds the CTA size: 1024 caps a thread at 64 registers, 512 at 128,
// 256 at 128 with two CTAs per SM; the launchers pick the smallest bound that
// holds the CTA, so long chunks (K = 16, 32) keep their registers.
constexpr int min_ctas(int maxt) { return maxt <= 256 ? 2 : 1; }

template <int K, typename T, int MAXT, bool TREE>
__global__ void __launch_bounds__(MAXT, min_ctas(MAXT)) x_sweep_kernel(const XArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (!a.persist) {
    x_rows_body<K, T, TREE>(a, blockIdx.x, smem);
    return;
  }
  // persistent: loop over row blocks; prefetch the next block's rows of u^k
  // and m into L2 while this one is solved
  const int nblk = (a.ny + a.spc - 1) / a.spc;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    if (blk + (int)gridDim.x < nblk) x_prefetch_rows(a, blk + gridDim.x);
    x_rows_body<K, T, TREE>(a, blk, smem);
    __syncthreads();  // shared memory is reused by the next block
  }
}

// ---------------------------------------------------------------------------
// pass 2: y solve + update (adi_bodies.cuh).  A strip of 2^log2W columns; a
// cluster of C CTAs covers the whole column length.
// ---------------------------------------------------------------------------
template <int K, typename T, int MAXT, bool TREE>
__global__ void __launch_bounds__(MAXT, min_ctas(MAXT)) y_sweep_kernel(const YArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int rank = cluster_rank(a.C);
  if (!a.persist) {
    cluster_arrive_early(a.C);
    y_strip_body<K, T, TREE>(a, blockIdx.x / a.C, rank, blockIdx.x == 0, smem);
    return;
  }
  // persistent: each cluster loops over strips; the next strip's rows of this
  // CTA are prefetched into L2 while the current one is solved.  Every
  // iteration arrives once on the cluster barrier to pair with the wait in
  // y_solve_cols.
  const int W = 1 << a.log2W;
  const int nstrips = (a.nx + W - 1) / W;
  const int nclusters = gridDim.x / a.C;
  for (int strip = blockIdx.x / a.C; strip < nstrips; strip += nclusters) {
    cluster_arrive_early(a.C);
    if (strip + nclusters < nstrips) y_prefetch_strip(a, strip + nclusters, rank, K);
    y_strip_body<K, T, TREE>(a, strip, rank, strip == 0 && rank == 0, smem);
    __syncthreads();  // shared memory is reused by the next strip
  }
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// Receiver sampling after a step: traces[s][r] = u^{k}(rec r), s = k - k0 - 1.
__global__ void gather_kernel(const GridDev* gd, const float* __restrict__ u_new, int ld) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= gd->n_rec) return;
  const long long s = gd->k - gd->k0 - 1;
  if (s < 0 || s >= gd->steps || gd->traces == nullptr) return;
  const int ix = gd->rec[2 * r], iy = gd->rec[2 * r + 1];
  gd->traces[s * gd->n_rec + r] = u_new[(size_t)iy * ld + ix];
}

// Start-up, Eq. (CN2): u^0 = phi, u^1 = phi + tau psi (+ tau^2/2 (m Lap phi + f^0)).
__global__ void init_kernel(int nx, int ny, int ld, const float* __restrict__ m,
                            const float* __restrict__ phi, const float* __restrict__ psi,
                            float* __restrict__ u0, float* __restrict__ u1, double tau,
                            double cx_half, double cy_half, int taylor, int sx, int sy,
                            double src_half, const float* __restrict__ wavelet, int n_wavelet) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t c = (size_t)j * nx + i;
  const double ph = phi[c];
  double v = ph + (psi ? tau * (double)psi[c] : 0.0);
  if (taylor) {
    const double l = (i > 0) ? phi[c - 1] : 0.0;
    const double r = (i + 1 < nx) ? phi[c + 1] : 0.0;
    const double dn = (j > 0) ? phi[c - nx] : 0.0;
    const double up = (j + 1 < ny) ? phi[c + nx] : 0.0;
    const double mm = m[(size_t)j * ld + i];
    v += mm * (cx_half * (l + r - 2.0 * ph) + cy_half * (dn + up - 2.0 * ph));
    if (i == sx && j == sy && wavelet != nullptr && n_wavelet > 0) v += src_half * wavelet[0];
  }
  u0[(size_t)j * ld + i] = (float)ph;
  u1[(size_t)j * ld + i] = (float)v;
}

// min(m), max(m) as float bit patterns (m > 0 compares as unsigned) and a
// flag for non-finite or non-positive entries.
__global__ void scan_m_kernel(const float* __restrict__ m, int nx, int ny, int ld,
                              unsigned int* out3) {
  unsigned int lo = 0x7f7fffffu, hi = 0u, bad = 0u;
  const size_t total = (size_t)nx * ny;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t j = t / nx, i = t % nx;
    const float v = m[j * ld + i];
    if (!(v > 0.0f) || !isfinite(v)) { bad = 1u; continue; }
    const unsigned int b = __float_as_uint(v);
    lo = min(lo, b);
    hi = max(hi, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out3 + 0, lo);
    atomicMax(out3 + 1, hi);
    atomicOr(out3 + 2, bad);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

size_t x_smem_bytes(int spc, int tsys, bool fp64, bool tree) {
  if (tree) {
    const int nwarps = std::max(1, spc * tsys / 32);
    return fp64 ? XTreeSmem<double>::bytes(nwarps) : XTreeSmem<float>::bytes(nwarps);
  }
  const size_t N = 2 * (size_t)tsys;
  return fp64 ? spc * N * (sizeof(Eq<double>) + sizeof(double))
              : spc * N * (sizeof(Eq<float>) + sizeof(float));
}

size_t y_smem_bytes(int W, int C, int tcol, bool fp64, bool tree) {
  const size_t slots = (W + C - 1) / C;
  if (tree) {
    const int threads = W * tcol;
    const int G = C * std::max(1, tcol / 32);
    return fp64 ? YTreeSmem<double>::bytes(threads, (int)slots, G)
                : YTreeSmem<float>::bytes(threads, (int)slots, G);
  }
  const size_t N = 2 * (size_t)C * tcol;
  return fp64 ? slots * N * (sizeof(Eq<double>) + sizeof(double))
              : slots * N * (sizeof(Eq<float>) + sizeof(float));
}

size_t y_stage_bytes(int threads, int K) { return align64((size_t)2 * K * threads * sizeof(float)); }

template <int K, typename T, int MAXT, bool TREE>
static cudaError_t launch_x_t(const XArgs& a, cudaStream_t st) {
  const int threads = a.spc << a.log2tsys;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;  // whole warps only
  int blocks = (a.ny + a.spc - 1) / a.spc;
  const size_t sm = x_smem_bytes(a.spc, 1 << a.log2tsys, sizeof(T) == 8, TREE);
  if (a.persist) {  // one wave of resident CTAs
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, x_sweep_kernel<K, T, MAXT, TREE>, threads, sm);
    if (e != cudaSuccess) return e;
    blocks = std::max(1, std::min(blocks, nsm * std::max(per_sm, 1)));
  }
  x_sweep_kernel<K, T, MAXT, TREE><<<blocks, threads, sm, st>>>(a);
  return cudaGetLastError();
}

template <int K, typename T, int MAXT, bool TREE>
static cudaError_t launch_y_t(const YArgs& a_in, cudaStream_t st) {
  YArgs a = a_in;
  const int W = 1 << a.log2W;
  const int threads = W << a.log2tcol;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;  // whole warps only
  const int strips = (a.nx + W - 1) / W;
  const size_t ysm = align64(y_smem_bytes(W, a.C, 1 << a.log2tcol, sizeof(T) == 8, TREE));
  a.stage_off = (a.stage_mode == 2) ? -1 : (int)ysm;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(strips * a.C, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = ysm + (a.stage_off >= 0 ? y_stage_bytes(threads, K) : 0);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a.persist) {  // one wave of resident clusters
    int nc = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, y_sweep_kernel<K, T, MAXT, TREE>, &cfg);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(std::max(1, std::min(strips, nc)) * a.C, 1, 1);
  }
  return cudaLaunchKernelEx(&cfg, y_sweep_kernel<K, T, MAXT, TREE>, a);
}

// K = 4, 8 fit 64 registers; K = 16, 32 take the smallest bound that holds
// `threads` (float only; FP64 kernels are bounded at 512).
#define ADI_DISPATCH_K(FN, TT, MT, TR, ARGS)             \
  switch (K) {                                           \
    case 4: return FN<4, TT, MT, TR> ARGS;               \
    case 8: return FN<8, TT, MT, TR> ARGS;               \
    case 16: return FN<16, TT, MT, TR> ARGS;             \
    case 32: return FN<32, TT, MT, TR> ARGS;             \
  }

#define ADI_DISPATCH_KF(FN, TR, ARGS, THREADS)                       \
  switch (K) {                                                       \
    case 4: return FN<4, float, 1024, TR> ARGS;                      \
    case 8: return FN<8, float, 1024, TR> ARGS;                      \
    case 16:                                                         \
      if ((THREADS) <= 256) return FN<16, float, 256, TR> ARGS;      \
      if ((THREADS) <= 512) return FN<16, float, 512, TR> ARGS;      \
      return FN<16, float, 1024, TR> ARGS;                           \
    case 32:                                                         \
      if ((THREADS) <= 256) return FN<32, float, 256, TR> ARGS;      \
      if ((THREADS) <= 512) return FN<32, float, 512, TR> ARGS;      \
      return FN<32, float, 1024, TR> ARGS;                           \
  }

cudaError_t launch_x(const XArgs& a, int K, bool fp64, bool tree, cudaStream_t st) {
  const int threads = a.spc << a.log2tsys;
  if (fp64) {
    if (tree) { ADI_DISPATCH_K(launch_x_t, double, 512, true, (a, st)) }
    else { ADI_DISPATCH_K(launch_x_t, double, 512, false, (a, st)) }
  } else {
    if (tree) { ADI_DISPATCH_KF(launch_x_t, true, (a, st), threads) }
    else { ADI_DISPATCH_KF(launch_x_t, false, (a, st), threads) }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_y(const YArgs& a, int K, bool fp64, bool tree, cudaStream_t st) {
  const int threads = 1 << (a.log2W + a.log2tcol);
  if (fp64) {
    if (tree) { ADI_DISPATCH_K(launch_y_t, double, 512, true, (a, st)) }
    else { ADI_DISPATCH_K(launch_y_t, double, 512, false, (a, st)) }
  } else {
    if (tree) { ADI_DISPATCH_KF(launch_y_t, true, (a, st), threads) }
    else { ADI_DISPATCH_KF(launch_y_t, false, (a, st), threads) }
  }
  return cudaErrorInvalidValue;
}

template <typename KernT>
static cudaError_t allow_smem(KernT kern, bool cluster16) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxDynSmem);
  if (e != cudaSuccess) return e;
  if (cluster16) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

#define ADI_CFG4(KERN, TT, MT, TR, CL)                                   \
  if (e == cudaSuccess) e = allow_smem(KERN<4, TT, MT, TR>, CL);         \
  if (e == cudaSuccess) e = allow_smem(KERN<8, TT, MT, TR>, CL);         \
  if (e == cudaSuccess) e = allow_smem(KERN<16, TT, MT, TR>, CL);        \
  if (e == cudaSuccess) e = allow_smem(KERN<32, TT, MT, TR>, CL);

#define ADI_CFG_SMALL(KERN, TR, CL)                                      \
  if (e == cudaSuccess) e = allow_smem(KERN<16, float, 256, TR>, CL);    \
  if (e == cudaSuccess) e = allow_smem(KERN<16, float, 512, TR>, CL);    \
  if (e == cudaSuccess) e = allow_smem(KERN<32, float, 256, TR>, CL);    \
  if (e == cudaSuccess) e = allow_smem(KERN<32, float, 512, TR>, CL);

cudaError_t configure_kernels() {
  cudaError_t e = cudaSuccess;
  ADI_CFG4(x_sweep_kernel, float, 1024, true, false)
  ADI_CFG4(x_sweep_kernel, float, 1024, false, false)
  ADI_CFG4(x_sweep_kernel, double, 512, true, false)
  ADI_CFG4(x_sweep_kernel, double, 512, false, false)
  ADI_CFG4(y_sweep_kernel, float, 1024, true, true)
  ADI_CFG4(y_sweep_kernel, float, 1024, false, true)
  ADI_CFG4(y_sweep_kernel, double, 512, true, true)
  ADI_CFG4(y_sweep_kernel, double, 512, false, true)
  ADI_CFG_SMALL(x_sweep_kernel, true, false)
  ADI_CFG_SMALL(x_sweep_kernel, false, false)
  ADI_CFG_SMALL(y_sweep_kernel, true, true)
  ADI_CFG_SMALL(y_sweep_kernel, false, true)
  return e;
}

cudaError_t launch_gather(const GridDev* gd, const float* u_new, int ld, int n_rec,
                          cudaStream_t st) {
  if (n_rec <= 0) return cudaSuccess;
  const int threads = 128;
  gather_kernel<<<(n_rec + threads - 1) / threads, threads, 0, st>>>(gd, u_new, ld);
  return cudaGetLastError();
}

cudaError_t launch_init(int nx, int ny, int ld, const float* m_pitched, const float* phi,
                        const float* psi, float* u0, float* u1, double tau, double cx_half,
                        double cy_half, int taylor, int sx, int sy, double src_half,
                        const float* wavelet, int n_wavelet, cudaStream_t st) {
  dim3 block(256, 1, 1);
  dim3 grid((nx + 255) / 256, ny, 1);
  init_kernel<<<grid, block, 0, st>>>(nx, ny, ld, m_pitched, phi, psi, u0, u1, tau, cx_half,
                                      cy_half, taylor, sx, sy, src_half, wavelet, n_wavelet);
  return cudaGetLastError();
}

cudaError_t launch_scan_m(const float* m, int nx, int ny, int ld, unsigned int* out3,
                          cudaStream_t st) {
  scan_m_kernel<<<152 * 4, 256, 0, st>>>(m, nx, ny, ld, out3);
  return cudaGetLastError();
}

}  // namespace adi
