// adi_bodies.cuh -- one CTA's share of a forward step, shared by the plain
// kernels (adi_forward.cu: one launch per sweep) and the persistent batched
// kernel (adi_batch.cu: many grids, one launch per step).
//
//   x_rows_body : RHS assembly r = tau^2 (m Lap u^k + f^k) (Eq. CN1 in delta
//                 form) fused with the row solves X w = r (Eq. fr1's
//                 operator) for one block of rows;
//   y_strip_body: the column solves Y z = w (Eq. fr2's operator) for one strip
//                 of columns fused with u^{k+1} = 2u^k - u^{k-1} + z, written
//                 over u^{k-1} (Algorithm 1's buffer swap).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adi_device.cuh"
#include "adi_internal.h"
#include "adi_sweeps.cuh"

namespace adi {

// Rows blk*spc .. blk*spc+spc-1; 2^log2tsys threads per row, K contiguous
// unknowns per thread.
template <int K, typename T, bool TREE>
__device__ __forceinline__ void x_rows_body(const XArgs& a, int blk, unsigned char* smem) {
  const int tsys = 1 << a.log2tsys;
  const int tid = threadIdx.x;
  const int sys = tid >> a.log2tsys;
  const int p = tid & (tsys - 1);
  const int j = blk * a.spc + sys;
  const int i0 = p * K;
  const bool active = (j < a.ny) && (i0 < a.nx);
  const size_t row = (size_t)j * a.ld;

  T d[K], s[K];
  if (active) {
    const T cx = (T)a.cx, cy = (T)a.cy, sc = (T)a.sc;
    float uc[K], v[K];
    // vertical neighbours first, accumulated into d (halo rows j-1, j+1)
    if (j > 0) {
      load_vec<K>(v, a.u + row - a.ld + i0);
#pragma unroll
      for (int k = 0; k < K; ++k) d[k] = (T)v[k];
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) d[k] = T(0);
    }
    if (j + 1 < a.ny) {
      load_vec<K>(v, a.u + row + a.ld + i0);
#pragma unroll
      for (int k = 0; k < K; ++k) d[k] += (T)v[k];
    }
    load_vec<K>(uc, a.u + row + i0);
    load_vec<K>(v, a.m + row + i0);
    const float uL = (i0 > 0) ? __ldg(a.u + row + i0 - 1) : 0.f;
    const float uR = (i0 + K < a.nx) ? __ldg(a.u + row + i0 + K) : 0.f;
    // padding columns (i >= nx) hold zero u and zero m, so r = s = 0 there
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T c = (T)uc[k];
      const T l = (T)(k > 0 ? uc[k - 1] : uL);
      const T r = (T)(k < K - 1 ? uc[k + 1] : uR);
      const T lap = cx * (l + r - T(2) * c) + cy * (d[k] - T(2) * c);
      d[k] = (T)v[k] * lap;
      s[k] = sc * (T)v[k];
    }
    // point source f^k = w(t_k) / (h1 h2) at one node
    const GridDev* gd = a.gd;
    const int sx = gd->src_ix;
    if (j == gd->src_iy && sx >= i0 && sx < i0 + K) {
      const long long lev = gd->k;
      if (gd->wavelet != nullptr && lev >= 0 && lev < gd->n_wavelet) {
        const T f = (T)a.src_scale * (T)gd->wavelet[lev];
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (i0 + k == sx) d[k] += f;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) { d[k] = T(0); s[k] = T(0); }
  }

  x_solve_rows<K, T, TREE>(smem, a.spc, a.log2tsys, a.pcr, sys, p, d, s);
  if (active) store_vec<K, T>(a.w + row + i0, d);
}

// Staged form of x_rows_body (FP32): the CTA's rows are read with coalesced
// float4 loads (consecutive lanes, consecutive 16-byte groups), the
// right-hand side r = tau^2 (m Lap u^k + f^k) and s = sc m are formed in
// that layout -- horizontal neighbours come from the adjacent lanes by
// shuffle -- and handed to the solving threads through shared memory; the
// solution w goes back the same way and is stored coalesced.  Shared memory
// at `stage` holds [2][threads*K/4] float4 slots (r or w, then s) in the
// swizzled order of swz4(), so both access patterns are conflict-free.
// The arithmetic is that of x_rows_body, term for term.

// Slot of logical float4 index f: the 16-byte slot within each 128-byte
// row is XOR-ed with the row index.  Eight consecutive f (coalesced) and
// f = t*K/4 + c for eight consecutive t (a thread's chunk) both land in
// eight distinct slots of a 128-byte row.
__device__ __forceinline__ int swz4(int f) { return f ^ ((f >> 3) & 7); }

template <int K, bool TREE>
__device__ __forceinline__ void x_rows_body_staged(const XArgs& a, int blk, unsigned char* smem) {
  constexpr int NQ = K / 4;  // float4 groups per thread
  const int threads = blockDim.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int log2row = a.log2tsys + (31 - __clz(K));  // elements per CTA row = tsys * K
  const int rowlen = 1 << log2row;
  float4* sd = reinterpret_cast<float4*>(smem + a.stage_off);
  float4* ss = sd + threads * NQ;
  const float cx = (float)a.cx, cy = (float)a.cy, sc = (float)a.sc;
  const GridDev* gd = a.gd;
  const int sx = gd->src_ix, sy = gd->src_iy;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int f = q * threads + tid;
    const int e = f << 2;
    const int col = e & (rowlen - 1);
    const int j = blk * a.spc + (e >> log2row);
    const bool ok = j < a.ny && col < a.nx;
    const size_t row = (size_t)j * a.ld;
    float4 c4 = z4, m4 = z4, v4 = z4, w4 = z4;
    if (ok) {
      c4 = __ldg(reinterpret_cast<const float4*>(a.u + row + col));
      m4 = __ldg(reinterpret_cast<const float4*>(a.m + row + col));
      if (j > 0) v4 = __ldg(reinterpret_cast<const float4*>(a.u + row - a.ld + col));
      if (j + 1 < a.ny) w4 = __ldg(reinterpret_cast<const float4*>(a.u + row + a.ld + col));
    }
    // u at col - 1 and col + 4: the neighbouring lanes' groups (same row
    // whenever the node exists), loaded at the warp's two ends
    float uL = __shfl_up_sync(0xffffffffu, c4.w, 1);
    float uR = __shfl_down_sync(0xffffffffu, c4.x, 1);
    if (lane == 0) uL = (ok && col > 0) ? __ldg(a.u + row + col - 1) : 0.f;
    if (lane == 31) uR = (ok && col + 4 < a.nx) ? __ldg(a.u + row + col + 4) : 0.f;
    if (col == 0) uL = 0.f;
    if (col + 4 >= a.nx) uR = 0.f;
    const float uc[4] = {c4.x, c4.y, c4.z, c4.w};
    const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
    const float vs[4] = {v4.x + w4.x, v4.y + w4.y, v4.z + w4.z, v4.w + w4.w};
    float d[4], s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float c = uc[k];
      const float l = k > 0 ? uc[k - 1] : uL;
      const float r = k < 3 ? uc[k + 1] : uR;
      const float lap = cx * (l + r - 2.f * c) + cy * (vs[k] - 2.f * c);
      d[k] = mv[k] * lap;
      s[k] = sc * mv[k];
    }
    // point source f^k = w(t_k) / (h1 h2) at one node
    if (ok && j == sy && sx >= col && sx < col + 4) {
      const long long lev = gd->k;
      if (gd->wavelet != nullptr && lev >= 0 && lev < gd->n_wavelet) {
        const float fs = (float)a.src_scale * gd->wavelet[lev];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (col + k == sx) d[k] += fs;
      }
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
  x_solve_rows<K, float, TREE>(smem, a.spc, a.log2tsys, a.pcr, sys, p, d, s);

  // w: each thread rewrites its own slots, then the CTA stores coalesced
#pragma unroll
  for (int c = 0; c < NQ; ++c)
    sd[swz4(tid * NQ + c)] = make_float4(d[4 * c + 0], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int f = q * threads + tid;
    const int e = f << 2;
    const int col = e & (rowlen - 1);
    const int j = blk * a.spc + (e >> log2row);
    if (j < a.ny && col < a.nx)
      *reinterpret_cast<float4*>(a.w + (size_t)j * a.ld + col) = sd[swz4(f)];
  }
}

// One bulk L2 prefetch (TMA unit): `bytes` from `p`, both multiples of 16.
__device__ __forceinline__ void l2_prefetch_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch of what block `blk` reads: rows blk*spc-1 .. blk*spc+spc of
// u^k (the halo rows included) and rows blk*spc .. blk*spc+spc-1 of m, one
// bulk request per row.  Rows start on 128-byte boundaries (ld is a multiple
// of 32) and the request is nx*4 bytes rounded up to 16, inside the row pitch.
__device__ __forceinline__ void x_prefetch_rows(const XArgs& a, int blk) {
  const int nu = a.spc + 2;
  const uint32_t bytes = (uint32_t)((a.nx * 4 + 15) & ~15);
  for (int r = threadIdx.x; r < nu + a.spc; r += blockDim.x) {
    const bool isu = r < nu;
    const int j = isu ? blk * a.spc - 1 + r : blk * a.spc + (r - nu);
    if (j >= 0 && j < a.ny) l2_prefetch_bulk((isu ? a.u : a.m) + (size_t)j * a.ld, bytes);
  }
}

// L2 prefetch of this CTA's rows of strip `strip` (w, m, u^k, u^{k-1}): one
// bulk request of W*4 bytes per row and field.  The strip lies inside the row
// pitch (ld is a multiple of 32 >= W), so every request is in bounds.
__device__ __forceinline__ void y_prefetch_strip(const YArgs& a, int strip, int rank, int K) {
  const int log2rows = a.log2tcol + (31 - __clz(K));
  const int rows = 1 << log2rows;
  const int W = 1 << a.log2W;
  const size_t off = (size_t)strip * W;
  for (int t = threadIdx.x; t < 4 * rows; t += blockDim.x) {
    const int f = t >> log2rows;
    const int j = rank * rows + (t & (rows - 1));
    if (j < a.ny) {
      const float* base = f == 0 ? a.w : f == 1 ? a.m : f == 2 ? a.u_cur : a.u_prev;
      l2_prefetch_bulk(base + (size_t)j * a.ld + off, (uint32_t)(W * 4));
    }
  }
}

// Strip `strip` of 2^log2W columns, cluster rank `rank` of C along the
// column (C = 1 outside clusters).  `bump` advances the grid's level k (one
// CTA per grid and step does it).  A kernel with C > 1 must have executed
// cluster_arrive_early() first.
template <int K, typename T, bool TREE>
__device__ __forceinline__ void y_strip_body(const YArgs& a, int strip, int rank, bool bump,
                                             unsigned char* smem) {
  const int W = 1 << a.log2W;
  const int tcol = 1 << a.log2tcol;
  const int C = a.C;
  const int tid = threadIdx.x;
  const int col = tid & (W - 1);
  const int q = tid >> a.log2W;
  const int gq = rank * tcol + q;
  const int i = strip * W + col;
  const int j0 = gq * K;
  const bool colok = i < a.nx;
  const bool full = colok && (j0 + K <= a.ny);
  const size_t ld = (size_t)a.ld;
  const size_t base = (size_t)j0 * ld + i;
  const T sc = (T)a.sc;

  // Fetch u^k and u^{k-1} of this thread's rows now, so that their HBM
  // traffic overlaps the solve: either asynchronous copies into shared memory
  // (layout [2][K][threads], read back by the epilogue) or, with
  // stage_off < 0, prefetches into L2 (one per row segment of the strip).
  const int threads = blockDim.x;
  const bool smem_stage = a.stage_off >= 0;
  float* stage = reinterpret_cast<float*>(smem + (smem_stage ? a.stage_off : 0));
  if (!smem_stage) {
    if (col == 0) {  // base is the strip's first column here; W*4 bytes stay in the pitch
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (j0 + k < a.ny) {
          l2_prefetch_bulk(a.u_cur + base + k * ld, (uint32_t)(W * 4));
          l2_prefetch_bulk(a.u_prev + base + k * ld, (uint32_t)(W * 4));
        }
      }
    }
  } else {
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(stage + tid);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ok = colok && (j0 + k) < a.ny;
      const float* gc = ok ? a.u_cur + base + k * ld : a.u_cur;
      const float* gp = ok ? a.u_prev + base + k * ld : a.u_prev;
      const int nbytes = ok ? 4 : 0;  // 0: zero-fill without reading
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sb + 4u * (k * threads)),
                   "l"(gc), "r"(nbytes) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                   ::"r"(sb + 4u * ((K + k) * threads)), "l"(gp), "r"(nbytes) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }

  T d[K], s[K];
  if (full) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      d[k] = (T)__ldcg(a.w + base + k * ld);
      s[k] = sc * (T)__ldg(a.m + base + k * ld);
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool ok = colok && (j0 + k) < a.ny;
      d[k] = ok ? (T)__ldcg(a.w + base + k * ld) : T(0);
      s[k] = ok ? sc * (T)__ldg(a.m + base + k * ld) : T(0);
    }
  }
  y_solve_cols<K, T, TREE>(smem, a.log2W, a.log2tcol, C, rank, a.pcr, col, gq, d, s);

  if (smem_stage) asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's staged rows
  // chk accumulates un - un: zero while every new value is finite, NaN after
  // the first Inf or NaN (no fast-math, so the difference is not folded)
  float chk = 0.f;
  if (full && smem_stage) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float un = 2.0f * stage[k * threads + tid] - stage[(K + k) * threads + tid] + (float)d[k];
      a.u_prev[base + k * ld] = un;
      chk += un - un;
    }
  } else if (full) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const size_t idx = base + k * ld;
      const float un = 2.0f * __ldcg(a.u_cur + idx) - __ldcg(a.u_prev + idx) + (float)d[k];
      a.u_prev[idx] = un;
      chk += un - un;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (colok && (j0 + k) < a.ny) {
        const size_t idx = base + k * ld;
        const float uc = smem_stage ? stage[k * threads + tid] : __ldcg(a.u_cur + idx);
        const float up = smem_stage ? stage[(K + k) * threads + tid] : __ldcg(a.u_prev + idx);
        const float un = 2.0f * uc - up + (float)d[k];
        a.u_prev[idx] = un;
        chk += un - un;
      }
    }
  }
  if (a.z_out != nullptr && colok) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if ((j0 + k) < a.ny) a.z_out[base + k * ld] = (float)d[k];
  }
  const bool bad = chk != 0.f;
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_NUMERIC);
  if (bump && tid == 0 && a.gd) a.gd->k += 1;
}

}  // namespace adi
