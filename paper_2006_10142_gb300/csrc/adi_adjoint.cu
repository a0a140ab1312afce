// adi_adjoint.cu -- kernels of the reverse (adjoint) time step.
//
// Forward step k (Eq. CN1 in delta form, factored as in Section 2):
//   r = tau^2 (m Lap u^k + f^k),  X w = r,  Y z = w,  u^{k+1} = 2u^k - u^{k-1} + z,
// with X = I - S Lap_x, Y = I - S Lap_y, S = diag(sigma), sigma = tau^2 m / 2.
// Reverse step (lam^j = dJ/du^j, accumulated from later steps and from the
// receiver residuals):
//   zbar = lam^{k+1};   Y^T wbar = zbar;   X^T rbar = wbar;
//   dJ/dm += (tau^2/2)(wbar . Lap_y z + rbar . Lap_x w) + tau^2 rbar . Lap u^k
//   lam^k += 2 zbar + tau^2 Lap(m . rbar);   lam^{k-1} -= zbar;
//   dJ/dw(t_k) += tau^2 rbar_src / (h1 h2).
// The transposed systems are solved with the forward line solvers through
// the similarity Y^T = S^{-1} Y S (Lap_y is symmetric):
//   wbar = m^{-1} . Y^{-1} (m . zbar),   rbar = m^{-1} . X^{-1} (m . wbar)
// (sigma is m times a constant, which cancels).  The gradient terms are
// pointwise through the forward identities Y z = w, X w = r:
//   (tau^2/2) Lap_y z = (z - w)/m,  (tau^2/2) Lap_x w = (w - r)/m,
//   tau^2 Lap u^k = (r - tau^2 f)/m,
// so  dJ/dm += (wbar (z - w) + rbar (w - tau^2 f)) / m,
// each step's increment formed in FP32 from the FP32 fields (z - w of two
// FP32 values within a factor of two of each other is exact) and added to
// an FP64 sum in the same pass: the reverse accumulation over all steps is
// FP64.
// The column solves run in y_pipe_kernel's adjoint mode (adi_forward.cu)
// when the forward y sweep is pipelined, else in y_adj_kernel below; the
// row solves in x_adj_staged_kernel (rows staged through shared memory) or
// x_adj_kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adi_adjoint.h"
#include "adi_bodies.cuh"
#include "adi_device.cuh"
#include "adi_sweeps.cuh"

namespace adi {

// MAXT bounds the CTA size: 1024 caps a thread at 64 registers, 512 at 128,
// 256 at 128 with two CTAs per SM (the launchers pick the smallest bound
// that holds the CTA).
constexpr int adj_min_ctas(int maxt) { return maxt <= 256 ? 2 : 1; }

// Dynamic shared memory the adjoint kernels are configured for.
constexpr size_t kAdjSmem = 200 * 1024;

// The source node's terms, computed in FP64 out of line: only the thread
// that holds the source node calls them, so no other warp issues FP64
// instructions.  GB300 runs FP64 at 1/64 of the FP32 rate, and predicated
// FP64 instructions inside the element loops would occupy the FP64 pipe in
// every warp.
// tau^2 f^k at the source node.
__device__ __noinline__ float source_term(double src_scale, const float* wavelet, long long level) {
  return (float)(src_scale * (double)wavelet[level]);
}
// dJ/dw(t_k) += tau^2 rbar_src / (h1 h2).
__device__ __noinline__ void add_wavelet_grad(float* gw, long long level, double src_scale, float r) {
  gw[level] += (float)(src_scale * (double)r);
}

// Y^T wbar = lam (column solves): d = m . lam, solve with Y, wbar = x / m
// (m is read again for the division rather than kept in registers).
template <int K, typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, adj_min_ctas(MAXT)) y_adj_kernel(const YAdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = 1 << a.log2W;
  const int tcol = 1 << a.log2tcol;
  const int C = a.C;
  cluster_arrive_early(C);
  const int tid = threadIdx.x;
  const int col = tid & (W - 1);
  const int q = tid >> a.log2W;
  const int rank = cluster_rank(C);
  const int strip = blockIdx.x / C;
  const int gq = rank * tcol + q;
  const int i = strip * W + col;
  const int j0 = gq * K;
  const bool colok = i < a.nx;
  const T sc = (T)a.sc;
  const size_t ld = (size_t)a.ld;
  const size_t base = (size_t)j0 * ld + i;
  const bool full = colok && j0 + K <= a.ny;
  T d[K], s[K];
  if (full) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T mk = (T)__ldg(a.m + base + k * ld);
      d[k] = mk * (T)__ldg(a.lam + base + k * ld);
      s[k] = sc * mk;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ok = colok && j0 + k < a.ny;
      const T mk = ok ? (T)__ldg(a.m + base + k * ld) : T(1);
      d[k] = ok ? mk * (T)__ldg(a.lam + base + k * ld) : T(0);
      s[k] = ok ? sc * mk : T(0);
    }
  }
  y_solve_cols<K, T, true>(smem, a.log2W, a.log2tcol, C, rank, a.pcr, col, gq, d, s);
  if (colok) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (j0 + k < a.ny) a.wbar[base + k * ld] = (float)(d[k] * (T)rcp_t(__ldg(a.m + base + k * ld)));
  }
}

// X^T rbar = wbar (row solves) fused with the FP64 gradient accumulation and
// the wavelet gradient at the source node (four unknowns at a time after
// the solve, to keep registers for the solver).
template <int K, typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, adj_min_ctas(MAXT)) x_adj_kernel(const XAdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tsys = 1 << a.log2tsys;
  const int tid = threadIdx.x;
  const int sys = tid >> a.log2tsys;
  const int p = tid & (tsys - 1);
  const int j = blockIdx.x * a.spc + sys;
  const int i0 = p * K;
  const bool active = (j < a.ny) && (i0 < a.nx);
  const size_t row = (size_t)j * a.ld;
  const T sc = (T)a.sc;
  T d[K], s[K];
  if (active) {
    float mv[K], wb[K];
    load_vec<K>(mv, a.m + row + i0);
    load_vec<K>(wb, a.wbar + row + i0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ok = (i0 + k) < a.nx;
      d[k] = ok ? (T)mv[k] * (T)wb[k] : T(0);
      s[k] = ok ? sc * (T)mv[k] : T(0);
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) { d[k] = T(0); s[k] = T(0); }
  }
  x_solve_rows<K, T, true>(smem, a.spc, a.log2tsys, a.pcr, sys, p, d, s);
  if (!active) return;
  const bool has_src = (j == a.src_iy) && a.src_ix >= i0 && a.src_ix < i0 + K;
  const bool lev_ok = a.level >= 0 && a.level < a.n_wavelet;
#pragma unroll
  for (int c = 0; c < K / 4; ++c) {
    const int e = i0 + 4 * c;
    float mv[4], wb[4], wf[4], zf[4], rb[4];
    load_vec<4>(mv, a.m + row + e);
    load_vec<4>(wb, a.wbar + row + e);
    load_vec<4>(wf, a.w + row + e);
    load_vec<4>(zf, a.z + row + e);
    float im[4], g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      im[k] = rcp_t(mv[k]);
      rb[k] = (e + k < a.nx) ? (float)(d[4 * c + k] * (T)im[k]) : 0.f;
    }
    store_vec<4, float>(a.rbar + row + e, rb);
    // the step's increment is formed in FP32 (its inputs are FP32 fields)
    // and added to the FP64 sum
    double2* g2 = reinterpret_cast<double2*>(a.g64 + row + e);
    double2 g01 = g2[0], g23 = g2[1];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g[k] = 0.f;
      if (e + k >= a.nx) continue;
      const float r_ = rb[k];
      float wsrc = wf[k];
      if (has_src && e + k == a.src_ix) {
        if (lev_ok && a.wavelet != nullptr) wsrc -= source_term(a.src_scale, a.wavelet, a.level);
        if (lev_ok && a.gw != nullptr) add_wavelet_grad(a.gw, a.level, a.src_scale, r_);
      }
      g[k] = (wb[k] * (zf[k] - wf[k]) + r_ * wsrc) * im[k];
    }
    g01.x += (double)g[0]; g01.y += (double)g[1];
    g23.x += (double)g[2]; g23.y += (double)g[3];
    g2[0] = g01;
    g2[1] = g23;
  }
}

// The same row solves and gradient terms with every global access coalesced
// (FP32): m and wbar of the CTA's rows are read in float4 groups across the
// CTA into shared memory (the 128-byte-swizzled order of swz4(), so the
// coalesced writes and the per-thread chunk reads are both conflict-free);
// after the solve each thread puts its chunk of x back, and the CTA forms
// rbar = x / m and the gradient increment in float4 groups along the rows.
// The arithmetic is that of x_adj_kernel, term for term.  Shared memory: [solver region] [x / m . wbar: spc x tsys K floats]
// [s: same] at a.stage_off.
template <int K, int MAXT>
__global__ void __launch_bounds__(MAXT, adj_min_ctas(MAXT)) x_adj_staged_kernel(const XAdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NQ = K / 4;  // float4 groups per thread
  const int threads = blockDim.x;
  const int tid = threadIdx.x;
  const int log2row = a.log2tsys + (31 - __clz(K));  // elements per CTA row = tsys * K
  const int rowlen = 1 << log2row;
  float4* sd = reinterpret_cast<float4*>(smem + a.stage_off);
  float4* ss = sd + threads * NQ;
  const float sc = (float)a.sc;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int j0 = blockIdx.x * a.spc;

#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int f = q * threads + tid;
    const int e = f << 2;
    const int col = e & (rowlen - 1);
    const int j = j0 + (e >> log2row);
    float4 m4 = z4, b4 = z4;
    if (j < a.ny && col < a.nx) {
      const size_t row = (size_t)j * a.ld;
      m4 = __ldg(reinterpret_cast<const float4*>(a.m + row + col));
      b4 = __ldg(reinterpret_cast<const float4*>(a.wbar + row + col));
    }
    const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
    const float wb[4] = {b4.x, b4.y, b4.z, b4.w};
    float d[4], s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = j < a.ny && col + k < a.nx;
      d[k] = ok ? mv[k] * wb[k] : 0.f;
      s[k] = ok ? sc * mv[k] : 0.f;
    }
    sd[swz4(f)] = make_float4(d[0], d[1], d[2], d[3]);
    ss[swz4(f)] = make_float4(s[0], s[1], s[2], s[3]);
  }
  __syncthreads();

  float d[K], s[K];
#pragma unroll
  for (int c = 0; c < NQ; ++c) {
    const float4 dv = sd[swz4(tid * NQ + c)];
    const float4 sv = ss[swz4(tid * NQ + c)];
    d[4 * c + 0] = dv.x; d[4 * c + 1] = dv.y; d[4 * c + 2] = dv.z; d[4 * c + 3] = dv.w;
    s[4 * c + 0] = sv.x; s[4 * c + 1] = sv.y; s[4 * c + 2] = sv.z; s[4 * c + 3] = sv.w;
  }
  const int sys = tid >> a.log2tsys;
  const int p = tid & ((1 << a.log2tsys) - 1);
  x_solve_rows<K, float, true>(smem, a.spc, a.log2tsys, a.pcr, sys, p, d, s);
#pragma unroll
  for (int c = 0; c < NQ; ++c)
    sd[swz4(tid * NQ + c)] = make_float4(d[4 * c + 0], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
  __syncthreads();

#pragma unroll 2
  for (int q = 0; q < NQ; ++q) {
    const int f = q * threads + tid;
    const int e = f << 2;
    const int col = e & (rowlen - 1);
    const int j = j0 + (e >> log2row);
    if (j >= a.ny || col >= a.nx) continue;
    const size_t row = (size_t)j * a.ld;
    const float4 x4 = sd[swz4(f)];
    const float4 m4 = __ldg(reinterpret_cast<const float4*>(a.m + row + col));
    const float4 b4 = __ldg(reinterpret_cast<const float4*>(a.wbar + row + col));
    const float4 w4 = __ldcs(reinterpret_cast<const float4*>(a.w + row + col));
    const float4 zz = __ldcs(reinterpret_cast<const float4*>(a.z + row + col));
    const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
    const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
    const float wb[4] = {b4.x, b4.y, b4.z, b4.w};
    const float wf[4] = {w4.x, w4.y, w4.z, w4.w};
    const float zf[4] = {zz.x, zz.y, zz.z, zz.w};
    const bool has_src = j == a.src_iy && a.src_ix >= col && a.src_ix < col + 4;
    const bool lev_ok = a.level >= 0 && a.level < a.n_wavelet;
    // FP64 sum of the increments: two 16-byte groups per four nodes (the
    // pitched rows of ld doubles keep them aligned)
    double2* g2 = reinterpret_cast<double2*>(a.g64 + row + col);
    double2 g01 = g2[0], g23 = g2[1];
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    float rb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = col + k < a.nx;
      const float im = rcp_t(mv[k]);
      rb[k] = ok ? xv[k] * im : 0.f;
      float wsrc = wf[k];
      if (ok && has_src && col + k == a.src_ix) {
        if (lev_ok && a.wavelet != nullptr) wsrc -= source_term(a.src_scale, a.wavelet, a.level);
        if (lev_ok && a.gw != nullptr) add_wavelet_grad(a.gw, a.level, a.src_scale, rb[k]);
      }
      if (ok) g[k] = (wb[k] * (zf[k] - wf[k]) + rb[k] * wsrc) * im;
    }
    *reinterpret_cast<float4*>(a.rbar + row + col) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    g01.x += (double)g[0]; g01.y += (double)g[1];
    g23.x += (double)g[2]; g23.y += (double)g[3];
    g2[0] = g01;
    g2[1] = g23;
  }
}

// lam^k += 2 lam^{k+1} + tau^2 Lap(m . rbar) (+ the previous step's receiver
// residuals);  lam^{k-1} -= lam^{k+1};  lam^{k+1} = 0.  Four nodes of a row
// per thread (16-byte accesses; nodes past nx keep their values).
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void __launch_bounds__(256) lam_update_kernel(LamArgs a) {
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y;
  if (i0 >= a.nx || j >= a.ny) return;
  const size_t c = (size_t)j * a.ld + i0;
  // receiver range of this row first, so that its load overlaps the others
  const int q0 = a.resid != nullptr ? __ldg(a.rrow + j) : 0;
  const int q1 = a.resid != nullptr ? __ldg(a.rrow + j + 1) : 0;
  auto prod = [&](size_t at) {
    const float4 m4 = __ldg(reinterpret_cast<const float4*>(a.m + at));
    const float4 r4 = __ldg(reinterpret_cast<const float4*>(a.rbar + at));
    return make_float4(m4.x * r4.x, m4.y * r4.y, m4.z * r4.z, m4.w * r4.w);
  };
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 p0 = prod(c);
  const float4 pd = j > 0 ? prod(c - a.ld) : z4;
  const float4 pu = j + 1 < a.ny ? prod(c + a.ld) : z4;
  float mr[4] = {p0.x, p0.y, p0.z, p0.w};
  const float dn[4] = {pd.x, pd.y, pd.z, pd.w};
  const float up[4] = {pu.x, pu.y, pu.z, pu.w};
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (i0 + k >= a.nx) mr[k] = 0.f;
  const float mL = i0 > 0 ? __ldg(a.m + c - 1) * __ldg(a.rbar + c - 1) : 0.f;
  const float mR = i0 + 4 < a.nx ? __ldg(a.m + c + 4) * __ldg(a.rbar + c + 4) : 0.f;
  const float4 z0 = ld4(a.L0 + c), l1 = ld4(a.L1 + c), l2 = ld4(a.L2 + c);
  const float zb[4] = {z0.x, z0.y, z0.z, z0.w};
  float v1[4] = {l1.x, l1.y, l1.z, l1.w};
  float v2[4] = {l2.x, l2.y, l2.z, l2.w};
  float v0[4] = {z0.x, z0.y, z0.z, z0.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (i0 + k >= a.nx) continue;
    const float l = k > 0 ? mr[k - 1] : mL;
    const float r = k < 3 ? mr[k + 1] : mR;
    const float lap = a.cx * (l + r - 2.f * mr[k]) + a.cy * (dn[k] + up[k] - 2.f * mr[k]);
    v1[k] += 2.f * zb[k] + lap;
    v2[k] -= zb[k];
    v0[k] = 0.f;
  }
  for (int q = q0; q < q1; ++q) {
    const int d = __ldg(a.rix + q) - i0;
    if (d >= 0 && d < 4) {
      const float rv = __ldg(a.resid + __ldg(a.rid + q));
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k == d) v1[k] += rv;
    }
  }
  st4(a.L1 + c, v1);
  st4(a.L2 + c, v2);
  st4(a.L0 + c, v0);
}

// lam[rec r] += resid[s][r] (receivers may share a node, hence the atomics).
__global__ void seed_kernel(float* lam, int ld, const int* rec, int n_rec, const float* resid) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rec) return;
  atomicAdd(lam + (size_t)rec[2 * r + 1] * ld + rec[2 * r], resid[r]);
}

// Start-up dependence (second-order start u^1 = phi + tau psi + tau^2/2 (m Lap phi + f^0)):
// dJ/dm += (tau^2/2) lam^1 . Lap phi, dJ/dw(t_0) += (tau^2/2) lam^1_src / (h1 h2).
__global__ void taylor_adj_kernel(TaylorArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const size_t c = (size_t)j * a.ld + i;
  const double ph = a.phi[c];
  const double l = (i > 0) ? a.phi[c - 1] : 0.0;
  const double r = (i + 1 < a.nx) ? a.phi[c + 1] : 0.0;
  const double dn = (j > 0) ? a.phi[c - a.ld] : 0.0;
  const double up = (j + 1 < a.ny) ? a.phi[c + a.ld] : 0.0;
  const double lam = a.lam[c];
  a.gm[(size_t)j * a.nx + i] += lam * (a.cx_half * (l + r - 2.0 * ph) + a.cy_half * (dn + up - 2.0 * ph));
  if (i == a.src_ix && j == a.src_iy && a.gw != nullptr) a.gw[a.level] += (float)(a.src_half * lam);
}

// ---------------------------------------------------------------------------
template <int K, typename T, int MAXT>
static cudaError_t launch_xa_t(const XAdjArgs& a_in, cudaStream_t st) {
  XAdjArgs a = a_in;
  const int threads = a.spc << a.log2tsys;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;
  const int blocks = (a.ny + a.spc - 1) / a.spc;
  const size_t tree = x_smem_bytes(a.spc, 1 << a.log2tsys, sizeof(T) == 8, true);
  if constexpr (sizeof(T) == 4) if (a.staged) {
    // rows of tsys * K elements that hold the row (tsys K >= nx, from the planner)
    const size_t sm = align64(tree) + x_stage_bytes(threads, K);
    if (((size_t)K << a.log2tsys) >= (size_t)a.nx && sm <= kAdjSmem) {
      a.stage_off = (int)align64(tree);
      x_adj_staged_kernel<K, MAXT><<<blocks, threads, sm, st>>>(a);
      return cudaGetLastError();
    }
  }
  x_adj_kernel<K, T, MAXT><<<blocks, threads, tree, st>>>(a);
  return cudaGetLastError();
}

template <int K, typename T, int MAXT>
static cudaError_t launch_ya_t(const YAdjArgs& a, cudaStream_t st) {
  const int W = 1 << a.log2W;
  const int threads = W << a.log2tcol;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;
  const int strips = (a.nx + W - 1) / W;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(strips * a.C, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = y_smem_bytes(W, a.C, 1 << a.log2tcol, sizeof(T) == 8, true);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, y_adj_kernel<K, T, MAXT>, a);
}

cudaError_t launch_x_adj(const XAdjArgs& a, int K, bool fp64, cudaStream_t st) {
  const int threads = a.spc << a.log2tsys;
  if (fp64) {
    switch (K) {
      case 4: return launch_xa_t<4, double, 512>(a, st);
      case 8: return launch_xa_t<8, double, 512>(a, st);
      case 16: return launch_xa_t<16, double, 512>(a, st);
      case 32: return launch_xa_t<32, double, 512>(a, st);
    }
  } else {
    switch (K) {
      case 4: return launch_xa_t<4, float, 1024>(a, st);
      case 8: return launch_xa_t<8, float, 1024>(a, st);
      case 16:
        if (threads <= 256) return launch_xa_t<16, float, 256>(a, st);
        if (threads <= 512) return launch_xa_t<16, float, 512>(a, st);
        return launch_xa_t<16, float, 1024>(a, st);
      case 32:
        if (threads <= 256) return launch_xa_t<32, float, 256>(a, st);
        if (threads <= 512) return launch_xa_t<32, float, 512>(a, st);
        return launch_xa_t<32, float, 1024>(a, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_y_adj(const YAdjArgs& a, int K, bool fp64, cudaStream_t st) {
  const int threads = 1 << (a.log2W + a.log2tcol);
  if (fp64) {
    switch (K) {
      case 4: return launch_ya_t<4, double, 512>(a, st);
      case 8: return launch_ya_t<8, double, 512>(a, st);
      case 16: return launch_ya_t<16, double, 512>(a, st);
      case 32: return launch_ya_t<32, double, 512>(a, st);
    }
  } else {
    switch (K) {
      case 4: return launch_ya_t<4, float, 1024>(a, st);
      case 8: return launch_ya_t<8, float, 1024>(a, st);
      case 16:
        if (threads <= 256) return launch_ya_t<16, float, 256>(a, st);
        if (threads <= 512) return launch_ya_t<16, float, 512>(a, st);
        return launch_ya_t<16, float, 1024>(a, st);
      case 32:
        if (threads <= 256) return launch_ya_t<32, float, 256>(a, st);
        if (threads <= 512) return launch_ya_t<32, float, 512>(a, st);
        return launch_ya_t<32, float, 1024>(a, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_lam_update(const LamArgs& a, cudaStream_t st) {
  dim3 block(256, 1, 1), grid((a.nx + 1023) / 1024, a.ny, 1);
  lam_update_kernel<<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_seed(float* lam, int ld, const int* rec, int n_rec, const float* resid,
                        cudaStream_t st) {
  if (n_rec <= 0) return cudaSuccess;
  seed_kernel<<<(n_rec + 127) / 128, 128, 0, st>>>(lam, ld, rec, n_rec, resid);
  return cudaGetLastError();
}

cudaError_t launch_taylor_adj(const TaylorArgs& a, cudaStream_t st) {
  dim3 block(256, 1, 1), grid((a.nx + 255) / 256, a.ny, 1);
  taylor_adj_kernel<<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename KernT>
static cudaError_t allow_smem(KernT kern) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t configure_adjoint_kernels() {
  cudaError_t e = cudaSuccess;
#define ADI_CFG(kern) \
  if (e == cudaSuccess) e = allow_smem(kern);
  ADI_CFG((x_adj_kernel<4, float, 1024>))
  ADI_CFG((x_adj_kernel<8, float, 1024>))
  ADI_CFG((x_adj_kernel<16, float, 1024>))
  ADI_CFG((x_adj_kernel<32, float, 1024>))
  ADI_CFG((x_adj_kernel<4, double, 512>))
  ADI_CFG((x_adj_kernel<8, double, 512>))
  ADI_CFG((x_adj_kernel<16, double, 512>))
  ADI_CFG((x_adj_kernel<32, double, 512>))
  ADI_CFG((y_adj_kernel<4, float, 1024>))
  ADI_CFG((y_adj_kernel<8, float, 1024>))
  ADI_CFG((y_adj_kernel<16, float, 1024>))
  ADI_CFG((y_adj_kernel<32, float, 1024>))
  ADI_CFG((y_adj_kernel<4, double, 512>))
  ADI_CFG((y_adj_kernel<8, double, 512>))
  ADI_CFG((y_adj_kernel<16, double, 512>))
  ADI_CFG((y_adj_kernel<32, double, 512>))
  ADI_CFG((x_adj_staged_kernel<4, 1024>))
  ADI_CFG((x_adj_staged_kernel<8, 1024>))
  ADI_CFG((x_adj_staged_kernel<16, 1024>))
  ADI_CFG((x_adj_staged_kernel<32, 1024>))
  ADI_CFG((x_adj_staged_kernel<16, 256>))
  ADI_CFG((x_adj_staged_kernel<16, 512>))
  ADI_CFG((x_adj_staged_kernel<32, 256>))
  ADI_CFG((x_adj_staged_kernel<32, 512>))
  ADI_CFG((x_adj_kernel<16, float, 256>))
  ADI_CFG((x_adj_kernel<16, float, 512>))
  ADI_CFG((x_adj_kernel<32, float, 256>))
  ADI_CFG((x_adj_kernel<32, float, 512>))
  ADI_CFG((y_adj_kernel<16, float, 256>))
  ADI_CFG((y_adj_kernel<16, float, 512>))
  ADI_CFG((y_adj_kernel<32, float, 256>))
  ADI_CFG((y_adj_kernel<32, float, 512>))
#undef ADI_CFG
  return e;
}

}  // namespace adi
