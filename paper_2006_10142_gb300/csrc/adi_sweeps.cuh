// adi_sweeps.cuh -- the two line-solve cores shared by the forward, adjoint
// and batched kernels.  The kernels differ only in how they form the
// right-hand side (prologue) and what they do with the solution (epilogue).
//
// Solver variants (template parameter TREE):
//   TREE = true  -- per-thread partition, block cyclic reduction of the
//                   interface system across the 32 lanes of a warp (register
//                   shuffles), parallel cyclic reduction of the small system
//                   of warp summaries by one warp, back substitution down the
//                   same tree.  Two CTA barriers per line at most.
//   TREE = false -- per-thread partition, cyclic reduction of the interface
//                   system in shared memory down to `pcr` equations, PCR of
//                   those in a warp, CR back substitution (one barrier per
//                   CR level).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "adi_device.cuh"

namespace adi {

namespace cgx = cooperative_groups;

template <int K>
__device__ __forceinline__ void load_vec(float (&v)[K], const float* __restrict__ p) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    float4 t = __ldg(p4 + q);
    v[4 * q + 0] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
  }
}

template <int K, typename T>
__device__ __forceinline__ void store_vec(float* __restrict__ p, const T (&v)[K]) {
  float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int q = 0; q < K / 4; ++q)
    p4[q] = make_float4((float)v[4 * q + 0], (float)v[4 * q + 1], (float)v[4 * q + 2],
                        (float)v[4 * q + 3]);
}

__device__ __forceinline__ int ilog2_dev(int v) { return 31 - __clz(v); }

// ---------------------------------------------------------------------------
// shared-memory layouts
// ---------------------------------------------------------------------------
// Every region starts on a 64-byte boundary: Seg / Eq are stored with vector
// instructions that need their natural (16- or 32-byte) alignment.
__host__ __device__ constexpr size_t align64(size_t b) { return (b + 63) & ~size_t(63); }

template <typename T> struct XTreeSmem {
  // nodes[nwarps][31] | tops[nwarps] (one summary per warp) | xtop[nwarps][2]
  static __host__ __device__ size_t off_tops(int nwarps) {
    return align64((size_t)nwarps * 31 * sizeof(Node<T>));
  }
  static __host__ __device__ size_t off_xtop(int nwarps) {
    return off_tops(nwarps) + align64((size_t)nwarps * sizeof(Seg<T>));
  }
  static __host__ __device__ size_t bytes(int nwarps) {
    return off_xtop(nwarps) + align64((size_t)nwarps * 2 * sizeof(T));
  }
};

template <typename T> struct YTreeSmem {
  // csum[threads] (chunk summaries, later chunk end values) | nodes[nwarps][31]
  // | tops[n_slots][G] (group summaries of owned columns) | xtop[n_slots][G][2]
  static __host__ __device__ size_t off_nodes(int threads) {
    return align64((size_t)threads * sizeof(Seg<T>));
  }
  static __host__ __device__ size_t off_tops(int threads) {
    return off_nodes(threads) + align64((size_t)(threads / 32) * 31 * sizeof(Node<T>));
  }
  static __host__ __device__ size_t off_xtop(int threads, int n_slots, int G) {
    return off_tops(threads) + align64((size_t)n_slots * G * sizeof(Seg<T>));
  }
  static __host__ __device__ size_t bytes(int threads, int n_slots, int G) {
    return off_xtop(threads, n_slots, G) + align64((size_t)n_slots * G * 2 * sizeof(T));
  }
};

// ---------------------------------------------------------------------------
// x (row) solves
// ---------------------------------------------------------------------------
// The CTA holds `spc` rows of 2^log2tsys threads each; thread (sys, p) holds
// unknowns p*K .. p*K+K-1 of row sys in d (RHS) and s (off-diagonal
// magnitudes).  On return d holds the solution.  All threads of the CTA must
// call this.
template <int K, typename T, bool TREE>
__device__ __forceinline__ void x_solve_rows(unsigned char* smem, int spc, int log2tsys, int pcr,
                                             int sys, int p, T (&d)[K], T (&s)[K]) {
  if constexpr (TREE) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int levels = log2tsys < 5 ? log2tsys : 5;
    Node<T>* nodes = reinterpret_cast<Node<T>*>(smem) + warp * 31;
    Seg<T> S;
    Node<T> ndc;
    chunk_reduce_split<K, T>(d, s, S, ndc);
    S = warp_tree_up<T>(S, nodes, lane, levels);
    T xa, xc;
    if (log2tsys <= 5) {
      seg_solve_closed<T>(S, xa, xc);
    } else {
      const int nw = 1 << (log2tsys - 5);  // warps per row
      Seg<T>* tops = reinterpret_cast<Seg<T>*>(smem + XTreeSmem<T>::off_tops(nwarps));
      T* xtop = reinterpret_cast<T*>(smem + XTreeSmem<T>::off_xtop(nwarps));
      const int wis = p >> 5;
      if (lane == 0) tops[sys * nw + wis] = S;
      __syncthreads();
      for (int sy = warp; sy < spc; sy += nwarps) {
        Eq<T> E0 = eq_identity<T>(), E1 = eq_identity<T>();
        if (lane < nw) {
          E0 = tops[sy * nw + lane].f;
          E1 = tops[sy * nw + lane].l;
        }
        pcr64<T>(E0, E1, lane, 2 * nw);
        if (lane < nw) {
          xtop[2 * (sy * nw + lane)] = div_t(E0.d, E0.b);
          xtop[2 * (sy * nw + lane) + 1] = div_t(E1.d, E1.b);
        }
      }
      __syncthreads();
      xa = xtop[2 * (sys * nw + wis)];
      xc = xtop[2 * (sys * nw + wis) + 1];
    }
    warp_tree_down<T>(nodes, lane, levels, xa, xc);
    chunk_backsub_split<K, T>(d, s, ndc, xa, xc);
  } else {
    const int N = 2 << log2tsys;
    Eq<T>* red = reinterpret_cast<Eq<T>*>(smem);
    T* xs = reinterpret_cast<T*>(red + (size_t)spc * N);
    Eq<T> e0, e1;
    chunk_reduce<K, T>(d, s, e0, e1);
    red[(size_t)sys * N + 2 * p] = e0;
    red[(size_t)sys * N + 2 * p + 1] = e1;
    __syncthreads();
    reduced_solve<T>(red, xs, spc, N, log2tsys + 1, pcr);
    const T x0 = xs[(size_t)sys * N + 2 * p];
    const T xl = xs[(size_t)sys * N + 2 * p + 1];
    chunk_backsub<K, T>(d, s, x0, xl);
  }
}

// First half of the cluster start-up handshake: every CTA arrives as soon as
// it starts; y_solve_cols() waits before its first remote write.
__device__ __forceinline__ void cluster_arrive_early(int C) {
  if (C > 1) asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_started(int C) {
  if (C > 1) asm volatile("barrier.cluster.wait;" ::: "memory");
}

__device__ __forceinline__ int cluster_rank(int C) {
  return C > 1 ? (int)cgx::this_cluster().block_rank() : 0;
}

// ---------------------------------------------------------------------------
// y (column) solves
// ---------------------------------------------------------------------------
// A strip of W = 2^log2W columns, the column length spread over the C CTAs
// of a cluster (2^log2tcol threads per column per CTA, K rows per thread).
// Thread (col, q) of cluster rank `rank` holds rows gq*K .. gq*K+K-1,
// gq = rank * tcol + q, of column col.  The interface system of column col
// is reduced where its pieces live and finished in the shared memory of
// cluster rank (col mod C), reached over DSMEM.  All threads of every CTA of
// the cluster must call this; with C > 1 the caller has executed
// cluster_arrive_early() at kernel start.
// final_sync = false (tree solver only) leaves out the last cluster barrier,
// which only keeps the owners' shared memory alive until every remote read
// is done; a persistent caller may drop it because its next cluster barrier
// comes after those reads, and it must then synchronise the cluster once
// before exit.
template <int K, typename T, bool TREE>
__device__ __forceinline__ void y_solve_cols(unsigned char* smem, int log2W, int log2tcol, int C,
                                             int rank, int pcr, int col, int gq, T (&d)[K],
                                             T (&s)[K], bool final_sync = true) {
  const int W = 1 << log2W;
  // C, W, tcol and the group counts are powers of two: shifts, not divisions
  const int log2C = 31 - __clz(C);
  const int owner = col & (C - 1);
  const int slot = col >> log2C;
  const int n_slots = (W + C - 1) >> log2C;
  const int n_own = (rank < W) ? ((W - 1 - rank) >> log2C) + 1 : 0;
  if constexpr (TREE) {
    const int tcol = 1 << log2tcol;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int threads = blockDim.x;
    const int lg = log2tcol < 5 ? log2tcol : 5;  // tree levels
    const int LG = 1 << lg;                       // lanes per group
    const int gpc = tcol >> lg;                   // groups per column in this CTA
    const int G = C * gpc;                        // groups per column over the cluster (<= 32)
    Seg<T>* csum = reinterpret_cast<Seg<T>*>(smem);
    Node<T>* nodes = reinterpret_cast<Node<T>*>(smem + YTreeSmem<T>::off_nodes(threads)) + warp * 31;
    Seg<T>* tops = reinterpret_cast<Seg<T>*>(smem + YTreeSmem<T>::off_tops(threads));
    T* xtop = reinterpret_cast<T*>(smem + YTreeSmem<T>::off_xtop(threads, n_slots, G));
    const int q = gq - rank * tcol;
    Node<T> ndc;
    {
      Seg<T> S;
      chunk_reduce_split<K, T>(d, s, S, ndc);
      csum[col * tcol + q] = S;
    }
    __syncthreads();
    // re-map: each warp reduces up to 32 consecutive chunks of one column
    const int task = warp * (32 >> lg) + (lane >> lg);  // (column, group) handled by this lane
    const int tc = task >> (log2tcol - lg);
    const int tg = task & (gpc - 1);
    const int chunk = tg * LG + (lane & (LG - 1));
    Seg<T> S = csum[tc * tcol + chunk];
    S = warp_tree_up<T>(S, nodes, lane, lg);
    const int gg = rank * gpc + tg;  // global group index of this lane's group
    const int t_owner = tc & (C - 1), t_slot = tc >> log2C;
    Seg<T>* tdst = tops + t_slot * G + gg;
    if (C > 1) {
      cgx::cluster_group cl = cgx::this_cluster();
      cluster_wait_started(C);
      if ((lane & (LG - 1)) == 0) *cl.map_shared_rank(tdst, t_owner) = S;
      cl.sync();
    } else {
      if ((lane & (LG - 1)) == 0) *tdst = S;
      __syncthreads();
    }
    for (int sl = warp; sl < n_own; sl += nwarps) {
      Eq<T> E0 = eq_identity<T>(), E1 = eq_identity<T>();
      if (lane < G) {
        E0 = tops[sl * G + lane].f;
        E1 = tops[sl * G + lane].l;
      }
      pcr64<T>(E0, E1, lane, 2 * G);
      if (lane < G) {
        xtop[2 * (sl * G + lane)] = div_t(E0.d, E0.b);
        xtop[2 * (sl * G + lane) + 1] = div_t(E1.d, E1.b);
      }
    }
    T xa, xc;
    if (C > 1) {
      cgx::cluster_group cl = cgx::this_cluster();
      cl.sync();
      const T* src = cl.map_shared_rank(xtop + 2 * (t_slot * G + gg), t_owner);
      xa = src[0];
      xc = src[1];
      if (final_sync) cl.sync();  // owners keep their shared memory until every read is done
    } else {
      __syncthreads();
      xa = xtop[2 * (t_slot * G + gg)];
      xc = xtop[2 * (t_slot * G + gg) + 1];
    }
    warp_tree_down<T>(nodes, lane, lg, xa, xc);
    // hand the chunk end values back to the threads that own the chunks
    T* cx = reinterpret_cast<T*>(csum + tc * tcol + chunk);
    cx[0] = xa;
    cx[1] = xc;
    __syncthreads();
    const T* mine = reinterpret_cast<const T*>(csum + col * tcol + q);
    chunk_backsub_split<K, T>(d, s, ndc, mine[0], mine[1]);
  } else {
    const int N = (2 * C) << log2tcol;
    int log2N = log2tcol + 1;
    for (int c = C; c > 1; c >>= 1) ++log2N;
    Eq<T>* red = reinterpret_cast<Eq<T>*>(smem);
    T* xs = reinterpret_cast<T*>(red + (size_t)n_slots * N);
    Eq<T> e0, e1;
    chunk_reduce<K, T>(d, s, e0, e1);
    Eq<T>* dst = red + (size_t)slot * N + 2 * gq;
    T x0, xl;
    if (C > 1) {
      cgx::cluster_group cl = cgx::this_cluster();
      cluster_wait_started(C);
      dst = cl.map_shared_rank(dst, owner);
      dst[0] = e0;
      dst[1] = e1;
      cl.sync();
      reduced_solve<T>(red, xs, n_own, N, log2N, pcr);
      cl.sync();
      const T* src = cl.map_shared_rank(xs + (size_t)slot * N + 2 * gq, owner);
      x0 = src[0];
      xl = src[1];
      cl.sync();
    } else {
      dst[0] = e0;
      dst[1] = e1;
      __syncthreads();
      reduced_solve<T>(red, xs, W, N, log2N, pcr);
      x0 = xs[(size_t)slot * N + 2 * gq];
      xl = xs[(size_t)slot * N + 2 * gq + 1];
    }
    chunk_backsub<K, T>(d, s, x0, xl);
  }
}

// ---------------------------------------------------------------------------
// x (row) solve of one row split over a cluster of XC CTAs (FP32, tree
// solver): rank r holds the r-th part of the row, each thread K consecutive
// unknowns.  Every CTA writes its warp summaries to all XC CTAs over DSMEM;
// after one cluster barrier each CTA solves the top system (XC x warps
// segments, at most 32) itself and reads its end values locally.  The caller
// executes cluster_arrive_early(XC) once per row (the next row's wait orders
// this row's reads of `tops` before they are overwritten) and synchronises
// the cluster before exit.  Shared memory: XSplitSmem.
// ---------------------------------------------------------------------------
struct XSplitSmem {
  // nodes[nw][31] (this CTA's warps) | tops[XC * nw] | xtop[XC * nw][2]
  static __host__ __device__ size_t off_tops(int nw) {
    return align64((size_t)nw * 31 * sizeof(Node<float>));
  }
  static __host__ __device__ size_t off_xtop(int nw, int xc) {
    return off_tops(nw) + align64((size_t)xc * nw * sizeof(Seg<float>));
  }
  static __host__ __device__ size_t bytes(int nw, int xc) {
    return off_xtop(nw, xc) + align64((size_t)xc * nw * 2 * sizeof(float));
  }
};

template <int K, int XC>
__device__ __forceinline__ void x_solve_row_split(unsigned char* smem, int rank, float (&d)[K],
                                                  float (&s)[K]) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  Node<float>* nodes = reinterpret_cast<Node<float>*>(smem) + warp * 31;
  Seg<float>* tops = reinterpret_cast<Seg<float>*>(smem + XSplitSmem::off_tops(nw));
  float* xtop = reinterpret_cast<float*>(smem + XSplitSmem::off_xtop(nw, XC));
  Seg<float> S;
  Node<float> ndc;
  chunk_reduce_split<K, float>(d, s, S, ndc);
  S = warp_tree_up<float>(S, nodes, lane, 5);  // every lane holds the warp's summary
  cgx::cluster_group cl = cgx::this_cluster();
  cluster_wait_started(XC);
  if (lane < XC) *cl.map_shared_rank(tops + rank * nw + warp, lane) = S;
  cl.sync();
  if (warp == 0) {
    Eq<float> E0 = eq_identity<float>(), E1 = eq_identity<float>();
    if (lane < XC * nw) {
      E0 = tops[lane].f;
      E1 = tops[lane].l;
    }
    pcr64<float>(E0, E1, lane, 2 * XC * nw);
    if (lane < XC * nw) {
      xtop[2 * lane] = div_t(E0.d, E0.b);
      xtop[2 * lane + 1] = div_t(E1.d, E1.b);
    }
  }
  __syncthreads();
  float xa = xtop[2 * (rank * nw + warp)];
  float xc = xtop[2 * (rank * nw + warp) + 1];
  warp_tree_down<float>(nodes, lane, 5, xa, xc);
  chunk_backsub_split<K, float>(d, s, ndc, xa, xc);
}

}  // namespace adi
