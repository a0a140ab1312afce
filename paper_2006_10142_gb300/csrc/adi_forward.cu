// adi_forward.cu -- forward-step kernels of the factored ADI scheme.
//
// One time step (Eq. CN1 in delta form, factored as in Section 2):
//   pass 1, x_sweep_kernel: r = tau^2 (m Lap u^k + f^k) fused with the row
//           solves X w = r, X = I - S Lap_x (Eq. fr1's operator);
//   pass 2, y_sweep_kernel: the column solves Y z = w, Y = I - S Lap_y
//           (Eq. fr2's operator), fused with u^{k+1} = 2u^k - u^{k-1} + z,
//           written over u^{k-1} (the buffer swap of Algorithm 1).
// Both solve their lines with the cores of adi_sweeps.cuh.  Each pass also
// exists as a TMA-pipelined persistent kernel (x_pipe_kernel, y_pipe_kernel:
// the next tile streams into shared memory while the current one is
// solved), the default for FP32 tree solves.  Memory traffic per grid point:
// pass 1 reads u^k and m and writes w (12 B, plus halo rows served by L2);
// pass 2 reads w, m, u^k, u^{k-1} and writes u^{k+1} (20 B).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "adi_bodies.cuh"
#include "adi_device.cuh"
#include "adi_internal.h"
#include "adi_sweeps.cuh"
#include "adi_tma.cuh"

namespace adi {

// ---------------------------------------------------------------------------
// pass 1: RHS assembly + x solve (adi_bodies.cuh).  CTA = `spc` rows.
// ---------------------------------------------------------------------------
// MAXT bounds the CTA size: 1024 caps a thread at 64 registers, 512 at 128,
// 256 at 128 with two CTAs per SM; the launchers pick the smallest bound that
// holds the CTA, so long chunks (K = 16, 32) keep their registers.
constexpr int min_ctas(int maxt) { return maxt <= 64 ? 8 : maxt <= 128 ? 4 : maxt <= 256 ? 2 : 1; }

template <int K, typename T, int MAXT, bool TREE>
__global__ void __launch_bounds__(MAXT, min_ctas(MAXT)) x_sweep_kernel(const XArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (sizeof(T) == 4) {
    if (a.stage_off >= 0) {
      if (!a.persist) {
        x_rows_body_staged<K, TREE>(a, blockIdx.x, smem);
        return;
      }
      const int nblk = (a.ny + a.spc - 1) / a.spc;
      for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        if (blk + (int)gridDim.x < nblk) x_prefetch_rows(a, blk + gridDim.x);
        x_rows_body_staged<K, TREE>(a, blk, smem);
        __syncthreads();  // shared memory is reused by the next block
      }
      return;
    }
  }
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
// pass 1, pipelined form (FP32, tree solver): persistent CTAs loop over row
// blocks; while the rows of one block are solved, TMA brings the next
// block's rows of u^k and m into shared memory, so the loads of the next
// block overlap the solve of this one.  Halo rows (j - 1 and j + 1 of every
// row) outside the block come from L2 -- the neighbouring blocks are staged
// by the neighbouring CTAs at about the same time, and the two rows just
// outside the next block are prefetched.
//
// Shared memory: [solver region] [mbarrier at a.stage_off] [pad to 1024 B]
// [u rows: spc x rowf floats] [m rows: spc x rowf floats], rowf = tsys * K,
// every row 1024-byte aligned in the 128-byte-swizzled layout of swz4().
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void stage_vec(float (&v)[K], const float* row, int i0) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int c = 0; c < K / 4; ++c) {
    const float4 t = r4[swz4((i0 >> 2) + c)];
    v[4 * c + 0] = t.x; v[4 * c + 1] = t.y; v[4 * c + 2] = t.z; v[4 * c + 3] = t.w;
  }
}
__device__ __forceinline__ float stage_at(const float* row, int e) {
  return row[(swz4(e >> 2) << 2) | (e & 3)];
}

// XC = 2 or 4: each row is split over a cluster of XC CTAs (rank r stages
// and solves columns [r rowf, (r + 1) rowf)); one row per cluster.
template <int K, int MAXT, int XC>
__global__ void __launch_bounds__(MAXT, min_ctas(MAXT))
    x_pipe_kernel(const XArgs a, const __grid_constant__ CUtensorMap tm_u,
                  const __grid_constant__ CUtensorMap tm_m, const __grid_constant__ CUtensorMap tm_w) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NQ = K / 4;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int rank = XC > 1 ? cluster_rank(XC) : 0;
  const int tsys = 1 << a.log2tsys;        // threads per row in this CTA
  const int rowf = tsys * K;               // floats per staged row (a power of two >= 256)
  const int coff = rank * rowf;            // first column of this CTA's part of the row
  const int lines = rowf >> 5;             // 128-byte lines per staged row
  const int L = lines < 256 ? lines : 256; // lines per TMA box
  const int nchunk = lines / L;
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sa + (uint32_t)a.stage_off;
  const uint32_t st_u = (bar + 8u + 1023u) & ~1023u;
  const uint32_t st_m = st_u + (uint32_t)(a.spc * rowf * 4);
  const uint32_t st_w = st_m + (uint32_t)(a.spc * rowf * 4);
  const float* su = reinterpret_cast<const float*>(smem + (st_u - sa));
  const float* sm = su + (size_t)a.spc * rowf;
  float4* sw4 = reinterpret_cast<float4*>(smem + (st_w - sa));
  const int nblk = (a.ny + a.spc - 1) / a.spc;
  // L2 prefetch of halo rows: this CTA's part of the row, inside the pitch
  const uint32_t pf_bytes =
      XC > 1 ? (uint32_t)(max(0, min(rowf, a.ld - coff)) * 4) : (uint32_t)((a.nx * 4 + 15) & ~15);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  // warp 0: announce and start the copies of block `blk` (one box per lane)
  auto issue = [&](int blk) {
    const int j0 = blk * a.spc;
    const int nrows = min(a.spc, a.ny - j0);
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(2 * nrows * rowf * 4));
    for (int t = lane; t < 2 * nrows * nchunk; t += 32) {
      const int f = t & 1, rc = t >> 1;
      const int r = rc / nchunk, c = rc - r * nchunk;
      const uint32_t off = (uint32_t)((r * rowf + c * L * 32) * 4);
      if (f == 0) tma_load_3d(st_u + off, &tm_u, 0, c * L + rank * lines, j0 + r, bar);
      else tma_load_3d(st_m + off, &tm_m, 0, c * L + rank * lines, j0 + r, bar);
    }
  };
  const int blk0 = (int)blockIdx.x / XC;
  const int nrun = (int)gridDim.x / XC;  // CTAs (XC = 1) or clusters (XC > 1) in the grid
  if (tid < 32 && blk0 < nblk) issue(blk0);

  const int sys = tid >> a.log2tsys;
  const int p = tid & (tsys - 1);
  const int li0 = p * K;                 // first unknown of this thread within the staged part
  const int i0 = coff + li0;             // ... and within the row
  const int threads = blockDim.x;
  const int log2row = a.log2tsys + (31 - __clz(K));  // rowf = 1 << log2row
  const float* hsum = reinterpret_cast<const float*>(sw4) + (size_t)sys * rowf;
  // Halo rows: with one row per CTA and K = 32 (a thread's chunk is a whole
  // 128-byte line, so per-thread loads would touch 32 lines per warp
  // instruction) they are read coalesced and handed over through the w
  // stage; otherwise each thread loads its own chunk (interior halo rows of
  // a multi-row block come from the stage).
  const bool coalesced_halo = (K == 32) && a.spc == 1;
  uint32_t phase = 0;
  bool timed_out = false;
  for (int blk = blk0; blk < nblk; blk += nrun) {
    if constexpr (XC > 1) cluster_arrive_early(XC);
   if (coalesced_halo) {
    // The halo rows u^k_{j-1} + u^k_{j+1} of the block's rows, read with
    // coalesced float4 loads (consecutive lanes, consecutive 16-byte groups)
    // while the stage arrives, and handed to the solving threads through the
    // w stage, free until this block's solution is written.
    float4 hs[K / 4];
#pragma unroll
    for (int qi = 0; qi < K / 4; ++qi) {
      const int f = qi * threads + tid;
      const int e = f << 2;
      const int col = coff + (e & (rowf - 1));
      const int jr = blk * a.spc + (e >> log2row);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (jr < a.ny && col < a.nx) {
        if (jr > 0) v = __ldg(reinterpret_cast<const float4*>(a.u + (size_t)(jr - 1) * a.ld + col));
        if (jr + 1 < a.ny) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(a.u + (size_t)(jr + 1) * a.ld + col));
          v.x += t.x; v.y += t.y; v.z += t.z; v.w += t.w;
        }
      }
      hs[qi] = v;
    }
    if (tid < 32) bulk_wait_read();  // the previous block's w stage has been read out (per-lane groups)
    __syncthreads();
#pragma unroll
    for (int qi = 0; qi < K / 4; ++qi) sw4[swz4(qi * threads + tid)] = hs[qi];
    if (!mbar_wait_bounded(bar, phase, 1000000000ull)) timed_out = true;
    phase ^= 1u;
    __syncthreads();  // the halo sums are in place
   } else {
    if (!mbar_wait_bounded(bar, phase, 1000000000ull)) timed_out = true;
    phase ^= 1u;
   }
    const int j = blk * a.spc + sys;
    const bool active = j < a.ny && i0 < a.nx;
    float d[K], s[K];
    if (active) {
      const float cx = (float)a.cx, cy = (float)a.cy, sc = (float)a.sc;
      const float* ur = su + (size_t)sys * rowf;
      const float* mr = sm + (size_t)sys * rowf;
      float uc[K], v[K];
      if (coalesced_halo) {
        stage_vec<K>(d, hsum, li0);
      } else {
        if (sys > 0) {
          stage_vec<K>(d, ur - rowf, li0);
        } else if (j > 0) {
          load_vec<K>(d, a.u + (size_t)(j - 1) * a.ld + i0);
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) d[k] = 0.f;
        }
        if (j + 1 < a.ny) {
          if (sys + 1 < a.spc) stage_vec<K>(v, ur + rowf, li0);
          else load_vec<K>(v, a.u + (size_t)(j + 1) * a.ld + i0);
#pragma unroll
          for (int k = 0; k < K; ++k) d[k] += v[k];
        }
      }
      stage_vec<K>(uc, ur, li0);
      stage_vec<K>(v, mr, li0);
      // neighbours across the split between the two CTAs of a pair come from L2
      const size_t rowg = (size_t)j * a.ld;
      const float uL = (i0 > 0) ? (li0 > 0 ? stage_at(ur, li0 - 1) : __ldg(a.u + rowg + i0 - 1)) : 0.f;
      const float uR = (i0 + K < a.nx) ? (li0 + K < rowf ? stage_at(ur, li0 + K) : __ldg(a.u + rowg + i0 + K)) : 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float c = uc[k];
        const float l = k > 0 ? uc[k - 1] : uL;
        const float r = k < K - 1 ? uc[k + 1] : uR;
        const float lap = cx * (l + r - 2.f * c) + cy * (d[k] - 2.f * c);
        d[k] = v[k] * lap;
        s[k] = sc * v[k];
      }
      // point source f^k = w(t_k) / (h1 h2) at one node
      const GridDev* gd = a.gd;
      const int sx = gd->src_ix;
      if (j == gd->src_iy && sx >= i0 && sx < i0 + K) {
        const long long lev = gd->k;
        if (gd->wavelet != nullptr && lev >= 0 && lev < gd->n_wavelet) {
          const float f = (float)a.src_scale * gd->wavelet[lev];
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (i0 + k == sx) d[k] += f;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) { d[k] = 0.f; s[k] = 0.f; }
    }
    if (!coalesced_halo && tid < 32) bulk_wait_read();  // the previous block's w stage has been read out
    __syncthreads();  // every read of the stage is done: it may be refilled
    const int next = blk + nrun;
    if (tid < 32 && next < nblk) {
      fence_proxy_async_smem();
      issue(next);
      if (lane == 0 && pf_bytes > 0) {  // (a cluster rank wholly past the pitch prefetches nothing)
        const int jl = next * a.spc - 1, jh = next * a.spc + a.spc;
        if (jl >= 0) l2_prefetch_bulk(a.u + (size_t)jl * a.ld + coff, pf_bytes);
        if (jh < a.ny) l2_prefetch_bulk(a.u + (size_t)jh * a.ld + coff, pf_bytes);
      }
    }
    if constexpr (XC > 1) x_solve_row_split<K, XC>(smem, rank, d, s);
    else x_solve_rows<K, float, true>(smem, a.spc, a.log2tsys, a.pcr, sys, p, d, s);
    // w through the swizzled stage, stored by TMA boxes
#pragma unroll
    for (int c = 0; c < NQ; ++c)
      sw4[swz4((sys * rowf + li0) / 4 + c)] = make_float4(d[4 * c + 0], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid < 32) {
      const int j0 = blk * a.spc;
      const int nrows = min(a.spc, a.ny - j0);
      for (int t = lane; t < nrows * nchunk; t += 32) {
        const int r = t / nchunk, c = t - r * nchunk;
        // boxes that start past the pitch (a cluster rank beyond the row) are not stored
        if ((c * L + rank * lines) * 32 < a.ld)
          tma_store_3d(&tm_w, 0, c * L + rank * lines, j0 + r, st_w + (uint32_t)((r * rowf + c * L * 32) * 4));
      }
      bulk_commit();
    }
  }
  if (tid < 32) bulk_wait_all();
  if constexpr (XC > 1) cgx::this_cluster().sync();  // no CTA leaves while its shared memory may be written
  if (timed_out && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_TIMEOUT);
}


// ---------------------------------------------------------------------------
// Row solve of the band form with the CTAs of a cluster exchanging their warp
// summaries by st.async into the other CTAs' shared memory, completing on the
// receiver's mbarrier (no cluster barrier per row).  The summaries of row r
// go to buffer r & 1; a CTA writes row r + 2 into a buffer only after it has
// received every CTA's row r + 1 summaries, which those CTAs send after
// reading their row r buffer, so the two buffers never race.
// Shared memory: nodes[nw][31] | tops[2][XC * nw] | xtop[XC * nw][2] | bars[2].
// ---------------------------------------------------------------------------
struct XAsyncSmem {
  static __host__ __device__ size_t off_tops(int nw) { return align64((size_t)nw * 31 * sizeof(Node<float>)); }
  static __host__ __device__ size_t off_xtop(int nw, int xc) {
    return off_tops(nw) + align64((size_t)2 * xc * nw * sizeof(Seg<float>));
  }
  static __host__ __device__ size_t off_bars(int nw, int xc) {
    return off_xtop(nw, xc) + align64((size_t)xc * nw * 2 * sizeof(float));
  }
  static __host__ __device__ size_t bytes(int nw, int xc) { return off_bars(nw, xc) + 64; }
};

__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_async_v4(uint32_t dst, float a, float b, float c, float d, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(dst),
               "f"(a), "f"(b), "f"(c), "f"(d), "r"(bar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

template <int K, int XC>
__device__ __forceinline__ void x_solve_row_async(unsigned char* smem, int rank, int r, float (&d)[K],
                                                  float (&s)[K], bool& timed_out) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int b = r & 1;
  Node<float>* nodes = reinterpret_cast<Node<float>*>(smem) + warp * 31;
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t tops_a = sa + (uint32_t)XAsyncSmem::off_tops(nw) + (uint32_t)(b * XC * nw * sizeof(Seg<float>));
  const Seg<float>* tops = reinterpret_cast<const Seg<float>*>(smem + XAsyncSmem::off_tops(nw)) + b * XC * nw;
  float* xtop = reinterpret_cast<float*>(smem + XAsyncSmem::off_xtop(nw, XC));
  const uint32_t bar = sa + (uint32_t)XAsyncSmem::off_bars(nw, XC) + 8u * (uint32_t)b;
  Seg<float> S;
  Node<float> ndc;
  chunk_reduce_split<K, float>(d, s, S, ndc);
  S = warp_tree_up<float>(S, nodes, lane, 5);  // every lane holds the warp's summary
  if (lane < XC) {
    const uint32_t dst = mapa_shared(tops_a + (uint32_t)((rank * nw + warp) * sizeof(Seg<float>)), lane);
    const uint32_t rb = mapa_shared(bar, lane);
    st_async_v4(dst, S.f.a, S.f.b, S.f.c, S.f.d, rb);
    st_async_v4(dst + 16u, S.l.a, S.l.b, S.l.c, S.l.d, rb);
  }
  if (warp == 0) {
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(XC * nw * sizeof(Seg<float>)));
    const uint32_t par = (uint32_t)((r >> 1) & 1);
    if (!mbar_try_wait_cluster(bar, par)) {
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait_cluster(bar, par)) {
        if (global_ns() - t0 > 1000000000ull) {
          timed_out = true;
          break;
        }
      }
    }
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

// ---------------------------------------------------------------------------
// Column solves of the pipelined y sweep (one group of tcol <= 32 threads
// per column and CTA) with the CTAs of a cluster exchanging their column
// summaries by st.async instead of cluster barriers: every CTA sends the
// summary of its segment of each column to every CTA of the cluster, into
// buffer r & 1 of strip r, completing on the receiver's mbarrier, and
// solves the strip's W top systems itself.  A CTA writes strip r + 2's
// summaries only after it has received every CTA's strip r + 1 summaries,
// which those CTAs send after reading their strip r buffer, so the two
// buffers never race.
// Shared memory: [YTreeSmem csum | nodes] [tops: 2][W][C] [bars: 2].
// ---------------------------------------------------------------------------
struct YAsyncSmem {
  static __host__ __device__ size_t off_tops(int threads) { return YTreeSmem<float>::off_tops(threads); }
  static __host__ __device__ size_t off_bars(int threads, int W, int C) {
    return off_tops(threads) + align64((size_t)2 * W * C * sizeof(Seg<float>));
  }
  static __host__ __device__ size_t bytes(int threads, int W, int C) { return off_bars(threads, W, C) + 64; }
};

template <int K>
__device__ __forceinline__ void y_solve_cols_async(unsigned char* smem, int W, int log2tcol, int C, int rank,
                                                   int col, int q, int r, float (&d)[K], float (&s)[K],
                                                   bool& timed_out) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int threads = blockDim.x;
  const int lg = log2tcol;  // tree levels (tcol <= 32)
  const int tcol = 1 << lg;
  const int cpw = 32 >> lg;  // columns whose trees one warp holds
  Seg<float>* csum = reinterpret_cast<Seg<float>*>(smem);
  Node<float>* nodes = reinterpret_cast<Node<float>*>(smem + YTreeSmem<float>::off_nodes(threads)) + warp * 31;
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const int b = r & 1;
  const size_t toff = YAsyncSmem::off_tops(threads) + (size_t)b * W * C * sizeof(Seg<float>);
  const uint32_t tops_a = sa + (uint32_t)toff;
  const Seg<float>* tops = reinterpret_cast<const Seg<float>*>(smem + toff);
  const uint32_t bar = sa + (uint32_t)YAsyncSmem::off_bars(threads, W, C) + 8u * (uint32_t)b;
  Node<float> ndc;
  {
    Seg<float> S;
    chunk_reduce_split<K, float>(d, s, S, ndc);
    csum[col * tcol + q] = S;
  }
  __syncthreads();
  const int tc = warp * cpw + (lane >> lg);  // column of this lane's tree
  const int chunk = lane & (tcol - 1);
  Seg<float> S = csum[tc * tcol + chunk];
  S = warp_tree_up<float>(S, nodes, lane, lg);  // every lane of the group holds the column's summary
  for (int dst = chunk; dst < C; dst += tcol) {
    const uint32_t da = mapa_shared(tops_a + (uint32_t)((tc * C + rank) * sizeof(Seg<float>)), dst);
    const uint32_t db = mapa_shared(bar, dst);
    st_async_v4(da, S.f.a, S.f.b, S.f.c, S.f.d, db);
    st_async_v4(da + 16u, S.l.a, S.l.b, S.l.c, S.l.d, db);
  }
  if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)(W * C * sizeof(Seg<float>)));
  const uint32_t par = (uint32_t)((r >> 1) & 1);
  if (!mbar_try_wait_cluster(bar, par)) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_cluster(bar, par)) {
      if (global_ns() - t0 > 1000000000ull) {
        timed_out = true;
        break;
      }
    }
  }
  // the top systems of this warp's columns: lane l holds segment l's two
  // equations; each group takes the end values of this CTA's segment
  float xa = 0.f, xc = 0.f;
  for (int j = 0; j < cpw; ++j) {
    const int c = warp * cpw + j;
    Eq<float> E0 = eq_identity<float>(), E1 = eq_identity<float>();
    if (lane < C) {
      E0 = tops[c * C + lane].f;
      E1 = tops[c * C + lane].l;
    }
    pcr64<float>(E0, E1, lane, 2 * C);
    const float x0 = __shfl_sync(0xffffffffu, div_t(E0.d, E0.b), rank);
    const float x1 = __shfl_sync(0xffffffffu, div_t(E1.d, E1.b), rank);
    if ((lane >> lg) == j) {
      xa = x0;
      xc = x1;
    }
  }
  warp_tree_down<float>(nodes, lane, lg, xa, xc);
  float* cx = reinterpret_cast<float*>(csum + tc * tcol + chunk);
  cx[0] = xa;
  cx[1] = xc;
  __syncthreads();
  const float* mine = reinterpret_cast<const float*>(csum + col * tcol + q);
  chunk_backsub_split<K, float>(d, s, ndc, mine[0], mine[1]);
}

// ---------------------------------------------------------------------------
// pass 1, band form (FP32, tree solver, K = 16 or 32, rows split over a
// cluster of XC CTAs): each cluster walks a band of consecutive rows from top to bottom
// and keeps a ring of three rows of u^k in shared memory (rows j - 1, j,
// j + 1 of the row being solved), so the halo rows of the RHS stencil come
// from shared memory and every row of u^k and m is read from HBM once.  While
// row j is solved, TMA brings row j + 2 of u^k into the ring slot row j - 1
// has just freed, and row j + 1 of m; w goes back through a swizzled stage by
// TMA stores.  Rows outside the grid arrive as zeros (the Dirichlet ring).
// The CTAs of a cluster exchange their warp summaries with st.async
// (x_solve_row_async), so no cluster barrier runs per row (0.720 against
// 0.855 ms per 16384^2 launch with the barrier-synchronised exchange).
// The unknowns on either side of a CTA's part (the neighbouring CTAs'
// columns) come with each ring row as two 16-byte bulk copies on the same
// mbarrier, so the RHS never waits on a load from L2.
// Shared memory: [XAsyncSmem] [mbarrier at a.stage_off] [pad to 1024 B]
// [u ring: 3 x rowf] [m: rowf] [w: rowf] floats, rowf = tsys * K,
// [halo: 3 ring slots x (left, right) 16-byte groups].
// ---------------------------------------------------------------------------
template <int K, int MAXT, int XC>
__global__ void __launch_bounds__(MAXT, min_ctas(MAXT))
    x_band_kernel(const XArgs a, const __grid_constant__ CUtensorMap tm_u,
                  const __grid_constant__ CUtensorMap tm_m, const __grid_constant__ CUtensorMap tm_w) {
  static_assert((K == 16 || K == 32) && XC > 1, "band form: K = 16 or 32, rows over a cluster");
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int rank = cluster_rank(XC);
  const int tsys = 1 << a.log2tsys;        // threads of this CTA (one row part)
  const int rowf = tsys * K;               // floats per staged row part (>= 1024)
  const int coff = rank * rowf;            // first column of this CTA's part
  const int lines = rowf >> 5;             // 128-byte lines per row part
  const int L = lines < 256 ? lines : 256; // lines per TMA box
  const int nchunk = lines / L;
  const uint32_t rowb = (uint32_t)(rowf * 4);
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sa + (uint32_t)a.stage_off;
  const uint32_t st_u = (bar + 8u + 1023u) & ~1023u;  // ring slots 0, 1, 2
  const uint32_t st_m = st_u + 3u * rowb;
  const uint32_t st_w = st_m + rowb;
  const float* su = reinterpret_cast<const float*>(smem + (st_u - sa));
  const float* sm = reinterpret_cast<const float*>(smem + (st_m - sa));
  float4* sw4 = reinterpret_cast<float4*>(smem + (st_w - sa));
  const uint32_t st_h = st_w + rowb;  // halo of ring slot s at st_h + 32 s: left, right group
  const float* sh = reinterpret_cast<const float*>(smem + (st_h - sa));
  // the left group [coff - 4, coff) exists for every rank but the first; the
  // right group [coff + rowf, + 4) when a next rank's columns lie in the row
  const bool has_l = rank > 0;
  const bool has_r = rank + 1 < XC && (size_t)coff + rowf + 4 <= (size_t)a.ld;
  const int nclu = (int)gridDim.x / XC;
  const int band = (a.ny + nclu - 1) / nclu;
  const int jb = ((int)blockIdx.x / XC) * band;
  const int je = min(a.ny, jb + band);

  if (tid == 0) {
    mbar_init(bar, 1);
    const uint32_t xb = sa + (uint32_t)XAsyncSmem::off_bars((int)blockDim.x >> 5, XC);
    mbar_init(xb, 1);
    mbar_init(xb + 8u, 1);
    mbar_fence_init();
  }
  __syncthreads();
  cgx::this_cluster().sync();  // every CTA's summary barriers exist before the first st.async
  // warp 0: copies of one row part of u^k into ring slot `slot` and/or of m
  auto load_u = [&](int j, int slot) {
    for (int c = lane; c < nchunk; c += 32)
      tma_load_3d(st_u + (uint32_t)slot * rowb + (uint32_t)(c * L * 128), &tm_u, 0, c * L + rank * lines, j, bar);
  };
  auto load_m = [&](int j) {
    for (int c = lane; c < nchunk; c += 32)
      tma_load_3d(st_m + (uint32_t)(c * L * 128), &tm_m, 0, c * L + rank * lines, j, bar);
  };
  // lane 0: the halo groups of row j (rows outside the grid have none)
  auto halo_bytes = [&](int j) -> uint32_t {
    return (j >= 0 && j < a.ny) ? 16u * ((has_l ? 1u : 0u) + (has_r ? 1u : 0u)) : 0u;
  };
  auto load_halo = [&](int j, int slot) {
    if (j < 0 || j >= a.ny) return;
    const float* row = a.u + (size_t)j * a.ld;
    if (has_l) bulk_load_16(st_h + 32u * (uint32_t)slot, row + coff - 4, bar);
    if (has_r) bulk_load_16(st_h + 32u * (uint32_t)slot + 16u, row + coff + rowf, bar);
  };
  if (tid < 32 && jb < je) {
    if (lane == 0) mbar_arrive_expect_tx(bar, 4u * rowb + halo_bytes(jb - 1) + halo_bytes(jb) + halo_bytes(jb + 1));
    __syncwarp();
    load_u(jb - 1, 0);
    load_u(jb, 1);
    load_u(jb + 1, 2);
    load_m(jb);
    if (lane == 0) {
      load_halo(jb - 1, 0);
      load_halo(jb, 1);
      load_halo(jb + 1, 2);
    }
  }
  const int li0 = tid * K;          // first unknown of this thread within the part
  const int i0 = coff + li0;        // ... and within the row
  uint32_t phase = 0;
  bool timed_out = false;
  for (int j = jb; j < je; ++j) {
    const int r = j - jb;
    const int sp = r % 3, sc = (r + 1) % 3, sn = (r + 2) % 3;  // ring slots of rows j - 1, j, j + 1
    if (!mbar_wait_bounded(bar, phase, 1000000000ull)) timed_out = true;
    phase ^= 1u;
    const bool active = i0 < a.nx;
    float d[K], s[K];
    if (active) {
      const float cx = (float)a.cx, cy = (float)a.cy, scf = (float)a.sc;
      const float* up = su + (size_t)sp * rowf;
      const float* uc_row = su + (size_t)sc * rowf;
      const float* un = su + (size_t)sn * rowf;
      float uc[K], v[K];
      stage_vec<K>(d, up, li0);
      stage_vec<K>(v, un, li0);
#pragma unroll
      for (int k = 0; k < K; ++k) d[k] += v[k];
      stage_vec<K>(uc, uc_row, li0);
      stage_vec<K>(v, sm, li0);
      // neighbours across the split between the CTAs of a cluster: the
      // row's halo groups (element coff - 1 ends the left one, coff + rowf
      // starts the right one)
      const float* hs = sh + 8 * sc;
      const float uL = (i0 > 0) ? (li0 > 0 ? stage_at(uc_row, li0 - 1) : hs[3]) : 0.f;
      const float uR = (i0 + K < a.nx) ? (li0 + K < rowf ? stage_at(uc_row, li0 + K) : hs[4]) : 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float c = uc[k];
        const float l = k > 0 ? uc[k - 1] : uL;
        const float rr = k < K - 1 ? uc[k + 1] : uR;
        const float lap = cx * (l + rr - 2.f * c) + cy * (d[k] - 2.f * c);
        d[k] = v[k] * lap;
        s[k] = scf * v[k];
      }
      // point source f^k = w(t_k) / (h1 h2) at one node
      const GridDev* gd = a.gd;
      const int sx = gd->src_ix;
      if (j == gd->src_iy && sx >= i0 && sx < i0 + K) {
        const long long lev = gd->k;
        if (gd->wavelet != nullptr && lev >= 0 && lev < gd->n_wavelet) {
          const float f = (float)a.src_scale * gd->wavelet[lev];
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (i0 + k == sx) d[k] += f;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) { d[k] = 0.f; s[k] = 0.f; }
    }
    if (tid < 32) bulk_wait_read();  // the previous row's w stage has been read out
    __syncthreads();                 // slot of row j - 1 and the m stage are consumed
    if (tid < 32 && j + 1 < je) {
      fence_proxy_async_smem();
      if (lane == 0) mbar_arrive_expect_tx(bar, 2u * rowb + halo_bytes(j + 2));
      __syncwarp();
      load_u(j + 2, sp);
      load_m(j + 1);
      if (lane == 0) load_halo(j + 2, sp);
    }
    x_solve_row_async<K, XC>(smem, rank, r, d, s, timed_out);
    // w through the swizzled stage, stored by TMA boxes
#pragma unroll
    for (int c = 0; c < K / 4; ++c)
      sw4[swz4(li0 / 4 + c)] = make_float4(d[4 * c + 0], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid < 32) {
      for (int c = lane; c < nchunk; c += 32)
        if ((c * L + rank * lines) * 32 < a.ld)  // boxes past the pitch are not stored
          tma_store_3d(&tm_w, 0, c * L + rank * lines, j, st_w + (uint32_t)(c * L * 128));
      bulk_commit();
    }
  }
  if (tid < 32) bulk_wait_all();
  cgx::this_cluster().sync();  // no CTA leaves while its shared memory may be written
  if (timed_out && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_TIMEOUT);
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
// pass 2, pipelined form (FP32, tree solver, strips of W columns; launched
// with W = 16): persistent clusters loop over strips; while one strip is
// solved, each CTA loads its rows of the next strip's w and m into shared
// memory with TMA tensor boxes of W columns x BH rows (completing on an
// mbarrier) and prefetches the same boxes of u^k and u^{k-1} into L2 for the
// update.
// Shared memory: [solver region] [mbarrier at a.stage_off] [pad to 128 B]
// [w tile] [m tile], each R x W floats, R = tcol * K rows of this CTA.
// Rows beyond ny and columns beyond the row pitch arrive as zeros; columns
// beyond nx are masked.
// ADJ: the same pipeline solves the transposed column systems of the reverse
// step, Y^T wbar = lam, through Y^T = S^{-1} Y S: the first tile is lam
// (tm_w), the right-hand side is m . lam, and the epilogue writes
// wbar = x / m to z_out (m read again from global memory, one approximate
// reciprocal per node); tm_uc and tm_up
// are not used and nothing else is written.
// ---------------------------------------------------------------------------
template <int K, int MAXT, int W, bool ADJ, bool XA>
__global__ void __launch_bounds__(MAXT, min_ctas(MAXT))
    y_pipe_kernel(const YArgs a, const __grid_constant__ CUtensorMap tm_w,
                  const __grid_constant__ CUtensorMap tm_m, const __grid_constant__ CUtensorMap tm_uc,
                  const __grid_constant__ CUtensorMap tm_up) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int QG = 32 / W;  // row groups (q) per warp
  const int C = a.C;
  const int rank = cluster_rank(C);
  const int tid = threadIdx.x;
  const int tcol = 1 << a.log2tcol;
  const int R = tcol * K;              // rows of this CTA's tile (a power of two >= 64)
  const int BH = R < 256 ? R : 256;    // rows per TMA box
  const int nbox = R / BH;
  const int row0 = rank * R;
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sa + (uint32_t)a.stage_off;
  const uint32_t st_w = (bar + 8u + 127u) & ~127u;
  const uint32_t st_m = st_w + (uint32_t)(R * W * 4);
  const float* sw = reinterpret_cast<const float*>(smem + (st_w - sa));
  const float* smv = reinterpret_cast<const float*>(smem + (st_m - sa));
  const int nstrips = (a.nx + W - 1) / W;
  const int ncl = gridDim.x / C;
  const size_t ld = (size_t)a.ld;

  if (tid == 0) {
    mbar_init(bar, 1);
    if (XA) {
      const uint32_t xb = sa + (uint32_t)YAsyncSmem::off_bars((int)blockDim.x, W, C);
      mbar_init(xb, 1);
      mbar_init(xb + 8u, 1);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (XA) cgx::this_cluster().sync();  // every CTA's summary barriers exist before the first st.async
  // warp 0: copies of strip `st` (this CTA's rows) and L2 prefetch of its
  // u boxes, one box per lane
  const int lane = tid & 31;
  auto issue = [&](int st) {
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(2 * R * W * 4));
    constexpr int NF = ADJ ? 2 : 4;  // operations per box
    for (int t = lane; t < NF * nbox; t += 32) {
      const int b = t / NF, f = t % NF;
      const uint32_t off = (uint32_t)(b * BH * W * 4);
      if (f == 0) tma_load_2d(st_w + off, &tm_w, st * W, row0 + b * BH, bar);
      else if (f == 1) tma_load_2d(st_m + off, &tm_m, st * W, row0 + b * BH, bar);
      else if (f == 2) tma_prefetch_2d(&tm_uc, st * W, row0 + b * BH);
      else tma_prefetch_2d(&tm_up, st * W, row0 + b * BH);
    }
  };
  int strip = blockIdx.x / C;
  if (tid < 32) {
    if (lane == 0) prefetch_tensormap(&tm_w);
    if (lane == 1) prefetch_tensormap(&tm_m);
    if (!ADJ && lane == 2) prefetch_tensormap(&tm_uc);
    if (!ADJ && lane == 3) prefetch_tensormap(&tm_up);
    if (strip < nstrips) issue(strip);
  }
  const int col = tid & (W - 1);
  const int q = tid / W;
  const int qq = q & (QG - 1);  // this thread's row group within its warp
  const int gq = rank * tcol + q;
  const int j0 = gq * K;
  uint32_t phase = 0;
  bool timed_out = false;
  bool bad = false;
  const float sc = (float)a.sc;
  int r = 0;  // strips this cluster has solved
  for (; strip < nstrips; strip += ncl, ++r) {
    if (!XA) cluster_arrive_early(C);
    const int i = strip * W + col;
    const bool colok = i < a.nx;
    if (!mbar_wait_bounded(bar, phase, 1000000000ull)) timed_out = true;
    phase ^= 1u;
    // Rows are read in blocks of QG: row group qq takes row g + (i ^ qq) at
    // read i, so the QG groups of a warp read rows that differ modulo QG,
    // i.e. different 4W-byte slots of a 128-byte bank row (conflict-free);
    // a butterfly of selects on the bits of qq puts the values back in order.
    float d[K], s[K];
#pragma unroll
    for (int g = 0; g < K; g += QG) {
      float vw[QG], vm[QG];
#pragma unroll
      for (int i = 0; i < QG; ++i) {
        const int o = (q * K + g + (i ^ qq)) * W + col;
        vw[i] = sw[o];
        vm[i] = smv[o];
      }
#pragma unroll
      for (int b = 1; b < QG; b <<= 1) {
        const bool x = (qq & b) != 0;
#pragma unroll
        for (int i = 0; i < QG; ++i) {
          if ((i & b) == 0) {
            const float w0 = vw[i], w1 = vw[i | b], m0 = vm[i], m1 = vm[i | b];
            vw[i] = x ? w1 : w0;
            vw[i | b] = x ? w0 : w1;
            vm[i] = x ? m1 : m0;
            vm[i | b] = x ? m0 : m1;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < QG; ++i) {
        d[g + i] = colok ? (ADJ ? vm[i] * vw[i] : vw[i]) : 0.f;
        s[g + i] = colok ? sc * vm[i] : 0.f;
      }
    }
    __syncthreads();  // the stage is consumed: refill it with the next strip
    const int next = strip + ncl;
    if (tid < 32 && next < nstrips) {
      fence_proxy_async_smem();
      issue(next);
    }
    if (XA) {
      y_solve_cols_async<K>(smem, W, a.log2tcol, C, rank, col, q, r, d, s, timed_out);
    } else {
      // the cluster barrier at the top of the next strip keeps the owners'
      // shared memory alive until every remote read is done
      y_solve_cols<K, float, true>(smem, a.log2W, a.log2tcol, C, rank, a.pcr, col, gq, d, s, false);
    }
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
        // groups of EG rows: 2 EG loads in flight per thread within the register budget
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
    if (!ADJ && strip == 0 && rank == 0 && tid == 0 && a.gd) a.gd->k += 1;
    __syncthreads();  // the solver's shared memory is reused by the next strip
  }
  if (C > 1) cgx::this_cluster().sync();  // no CTA leaves while its shared memory may be read
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_NUMERIC);
  if (timed_out && (tid & 31) == 0 && a.err) atomicOr(a.err, ERR_TIMEOUT);
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
  const float phf = phi[c];
  if (!psi && !taylor) {  // u^1 = u^0 = phi: no arithmetic
    u0[(size_t)j * ld + i] = phf;
    u1[(size_t)j * ld + i] = phf;
    return;
  }
  const double ph = phf;
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
  // rows strided over the CTAs, columns over a CTA's threads (no division
  // per element)
  for (int j = blockIdx.x; j < ny; j += gridDim.x) {
    const float* row = m + (size_t)j * ld;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const float v = row[i];
      if (!(v > 0.0f) || !isfinite(v)) { bad = 1u; continue; }
      const unsigned int b = __float_as_uint(v);
      lo = min(lo, b);
      hi = max(hi, b);
    }
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
size_t x_stage_bytes(int threads, int K) { return align64((size_t)2 * K * threads * sizeof(float)); }
// tsys = threads per row in one CTA; xc > 1: the solver region holds the
// warp summaries of all CTAs of the cluster.
static size_t x_pipe_tree_bytes(int spc, int tsys, int xc) {
  return xc > 1 ? XSplitSmem::bytes(std::max(1, spc * tsys / 32), xc)
                : x_smem_bytes(spc, tsys, false, true);
}

size_t x_pipe_smem_bytes(int spc, int tsys, int K, int xc) {
  return align64(x_pipe_tree_bytes(spc, tsys, xc)) + 8 + 1024 + (size_t)3 * spc * tsys * K * 4;
}

// Tensor map of a pitched [ny][ld] FP32 field as {32, ld/32, ny} with
// 128-byte swizzle and boxes of {32, box_lines, 1} (one row segment).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static cudaError_t get_encode_fn(EncodeTiledFn* out) {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || p == nullptr) return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = fn;
  return cudaSuccess;
}

cudaError_t encode_row_map(CUtensorMap* out, const float* base, int ld, int ny, int box_lines) {
  EncodeTiledFn fn = nullptr;
  cudaError_t e = get_encode_fn(&fn);
  if (e != cudaSuccess) return e;
  if (ld % 32 != 0 || box_lines < 1 || box_lines > 256 || ((uintptr_t)base & 15) != 0)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {32, (cuuint64_t)(ld / 32), (cuuint64_t)ny};
  const cuuint64_t strides[2] = {128, (cuuint64_t)ld * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)box_lines, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int x_pipe_box_lines(int tsys, int K) {
  const int lines = tsys * K / 32;
  return lines < 256 ? lines : 256;
}

template <int K, typename T, int MAXT, bool TREE>
static cudaError_t launch_x_t(const XArgs& a_in, cudaStream_t st) {
  XArgs a = a_in;
  const int threads = a.spc << a.log2tsys;
  if (threads % 32 != 0 || threads > MAXT) return cudaErrorInvalidValue;  // whole warps only
  int blocks = (a.ny + a.spc - 1) / a.spc;
  size_t sm = x_smem_bytes(a.spc, 1 << a.log2tsys, sizeof(T) == 8, TREE);
  a.stage_off = -1;
  if (sizeof(T) == 4 && a.stage_mode == 1) {  // staging area after the solver's region
    a.stage_off = (int)align64(sm);
    sm = align64(sm) + x_stage_bytes(threads, K);
    if (sm > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  }
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
template <int K, int MAXT, int XC>
static cudaError_t launch_x_pipe_t(const XArgs& a_in, const CUtensorMap& tu, const CUtensorMap& tm,
                                   const CUtensorMap& tw, cudaStream_t st) {
  XArgs a = a_in;
  if (XC > 1) {  // the plan's threads per row are split over the cluster
    const int l2 = XC == 2 ? 1 : 2;
    if (a.spc != 1 || a.log2tsys < 5 + l2) return cudaErrorInvalidValue;
    a.log2tsys -= l2;
    if ((XC << a.log2tsys) / 32 > 32) return cudaErrorInvalidValue;  // top system of one warp
  }
  const int tsys = 1 << a.log2tsys;
  const int threads = a.spc * tsys;
  if (threads % 32 != 0 || threads > MAXT || tsys * K < 256) return cudaErrorInvalidValue;
  a.stage_off = (int)align64(x_pipe_tree_bytes(a.spc, tsys, XC));
  const size_t sm = x_pipe_smem_bytes(a.spc, tsys, K, XC);
  if (sm > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  const int nblk = (a.ny + a.spc - 1) / a.spc;
  if (XC == 1) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, x_pipe_kernel<K, MAXT, XC>, threads, sm);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(nblk, nsm * std::max(per_sm, 1)));
    x_pipe_kernel<K, MAXT, XC><<<blocks, threads, sm, st>>>(a, tu, tm, tw);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk * XC, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = XC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, x_pipe_kernel<K, MAXT, XC>, &cfg);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3(std::max(1, std::min(nblk, nc)) * XC, 1, 1);
  return cudaLaunchKernelEx(&cfg, x_pipe_kernel<K, MAXT, XC>, a, tu, tm, tw);
}

// Band form: [XAsyncSmem] [mbarrier] [pad to 1024] [u ring 3 x rowf] [m rowf] [w rowf] [halo 96 B].
size_t x_band_smem_bytes(int tsys, int K, int xc) {
  return align64(XAsyncSmem::bytes(std::max(1, tsys / 32), xc)) + 8 + 1024 + (size_t)5 * tsys * K * 4 + 128;
}

template <int K, int MAXT, int XC>
static cudaError_t launch_x_band_t(const XArgs& a_in, const CUtensorMap& tu, const CUtensorMap& tm,
                                   const CUtensorMap& tw, cudaStream_t st) {
  XArgs a = a_in;
  const int l2 = XC == 2 ? 1 : XC == 4 ? 2 : 3;
  if (a.spc != 1 || a.log2tsys < 5 + l2) return cudaErrorInvalidValue;
  a.log2tsys -= l2;                      // threads of one CTA (one row part)
  const int tsys = 1 << a.log2tsys;
  if (tsys > MAXT || tsys % 32 != 0 || tsys * K < 1024) return cudaErrorInvalidValue;
  if ((XC << a.log2tsys) / 32 > 32) return cudaErrorInvalidValue;  // top system of one warp
  a.stage_off = (int)align64(XAsyncSmem::bytes(std::max(1, tsys / 32), XC));
  const size_t sm = x_band_smem_bytes(tsys, K, XC);
  if (sm > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.ny * XC, 1, 1);
  cfg.blockDim = dim3(tsys, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = XC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, x_band_kernel<K, MAXT, XC>, &cfg);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3(std::max(1, std::min(a.ny, nc)) * XC, 1, 1);
  return cudaLaunchKernelEx(&cfg, x_band_kernel<K, MAXT, XC>, a, tu, tm, tw);
}

cudaError_t launch_x_band(const XArgs& a, int K, const CUtensorMap& tu, const CUtensorMap& tm,
                          const CUtensorMap& tw, cudaStream_t st) {
  if (K == 32) {
    if (a.xc == 2) return launch_x_band_t<32, 256, 2>(a, tu, tm, tw, st);
    if (a.xc == 4) return launch_x_band_t<32, 128, 4>(a, tu, tm, tw, st);
    if (a.xc == 8) return launch_x_band_t<32, 64, 8>(a, tu, tm, tw, st);
  } else if (K == 16) {
    if (a.xc == 2) return launch_x_band_t<16, 512, 2>(a, tu, tm, tw, st);
    if (a.xc == 4) return launch_x_band_t<16, 256, 4>(a, tu, tm, tw, st);
    if (a.xc == 8) return launch_x_band_t<16, 128, 8>(a, tu, tm, tw, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_x_pipe(const XArgs& a, int K, const CUtensorMap& tu, const CUtensorMap& tm,
                          const CUtensorMap& tw, cudaStream_t st) {
  const int threads = a.spc << a.log2tsys;
  if (a.xc == 2) return K == 32 ? launch_x_pipe_t<32, 256, 2>(a, tu, tm, tw, st) : cudaErrorInvalidValue;
  if (a.xc == 4) return K == 32 ? launch_x_pipe_t<32, 128, 4>(a, tu, tm, tw, st) : cudaErrorInvalidValue;
  switch (K) {
    case 8: return launch_x_pipe_t<8, 1024, 1>(a, tu, tm, tw, st);
    case 16:
      if (threads <= 256) return launch_x_pipe_t<16, 256, 1>(a, tu, tm, tw, st);
      if (threads <= 512) return launch_x_pipe_t<16, 512, 1>(a, tu, tm, tw, st);
      return launch_x_pipe_t<16, 1024, 1>(a, tu, tm, tw, st);
    case 32:
      if (threads <= 256) return launch_x_pipe_t<32, 256, 1>(a, tu, tm, tw, st);
      return launch_x_pipe_t<32, 512, 1>(a, tu, tm, tw, st);
  }
  return cudaErrorInvalidValue;
}

// The st.async exchange needs one group per column (tcol <= 32).  Every CTA
// solves all W top systems, so it is taken only where a warp holds at most
// two columns' trees (tcol >= 16), and for clusters of 4 to 8 CTAs: pairs
// keep the barrier form, and at 16 CTAs the exchange measured level with
// the barrier form (1.376 against 1.375 ms for y_coop_kernel at 16384^2).
static bool y_pipe_async_ok(int C, int tcol) { return C >= 4 && C <= 8 && tcol >= 16 && tcol <= 32; }

static size_t y_pipe_tree_bytes(int W, int C, int tcol) {
  const size_t t = y_smem_bytes(W, C, tcol, false, true);
  return y_pipe_async_ok(C, tcol) ? std::max(t, YAsyncSmem::bytes(W * tcol, W, C)) : t;
}

size_t y_pipe_smem_bytes(int W, int C, int tcol, int K) {
  const size_t R = (size_t)tcol * K;
  return align64(y_pipe_tree_bytes(W, C, tcol)) + 8 + 128 + 2 * R * W * 4;
}

int y_pipe_box_rows(int tcol, int K) {
  const int R = tcol * K;
  return R < 256 ? R : 256;
}

// Tensor map of a pitched [ny][ld] FP32 field as 2D {ld, ny}, boxes of
// {box_cols, box_rows} (box_cols = 4, 8, 16 or 32), no swizzle, zero fill outside.
cudaError_t encode_strip_map(CUtensorMap* out, const float* base, int ld, int ny, int box_cols,
                             int box_rows) {
  EncodeTiledFn fn = nullptr;
  cudaError_t e = get_encode_fn(&fn);
  if (e != cudaSuccess) return e;
  if (ld % 32 != 0 || box_rows < 1 || box_rows > 256 || ((uintptr_t)base & 15) != 0 ||
      (box_cols != 4 && box_cols != 8 && box_cols != 16 && box_cols != 32))
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int K, int MAXT, int W, bool ADJ>
static cudaError_t launch_y_pipe_t(const YArgs& a_in, const YMaps& mp, cudaStream_t st) {
  YArgs a = a_in;
  const int tcol = 1 << a.log2tcol;
  const int threads = W * tcol;
  if ((1 << a.log2W) != W || threads % 32 != 0 || threads > MAXT || tcol * K < 64) return cudaErrorInvalidValue;
  a.stage_off = (int)align64(y_pipe_tree_bytes(W, a.C, tcol));
  const size_t sm = y_pipe_smem_bytes(W, a.C, tcol, K);
  if (sm > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  const int strips = (a.nx + W - 1) / W;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(strips * a.C, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const bool xa = y_pipe_async_ok(a.C, tcol);
  auto kern = xa ? y_pipe_kernel<K, MAXT, W, ADJ, true> : y_pipe_kernel<K, MAXT, W, ADJ, false>;
  int nc = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3(std::max(1, std::min(strips, nc)) * a.C, 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, a, mp.w, mp.m, mp.uc, mp.up);
}

// 16-column strips (narrower strips, which fit smaller clusters, measured
// far slower: their TMA boxes and row segments are 16 or 32 bytes wide).
template <bool ADJ>
static cudaError_t launch_y_pipe_any(const YArgs& a, int K, const YMaps& mp, cudaStream_t st) {
  const int threads = 1 << (a.log2W + a.log2tcol);
  const int W = 1 << a.log2W;
  const bool small = threads <= 256;
  if (K == 16 && W == 16)
    return small ? launch_y_pipe_t<16, 256, 16, ADJ>(a, mp, st) : launch_y_pipe_t<16, 512, 16, ADJ>(a, mp, st);
  if (K == 32 && W == 16)
    return small ? launch_y_pipe_t<32, 256, 16, ADJ>(a, mp, st) : launch_y_pipe_t<32, 512, 16, ADJ>(a, mp, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_y_pipe(const YArgs& a, int K, const YMaps& mp, cudaStream_t st) {
  return launch_y_pipe_any<false>(a, K, mp, st);
}

cudaError_t launch_y_pipe_adj(const YArgs& a, int K, const CUtensorMap& lam, const CUtensorMap& m,
                              cudaStream_t st) {
  if (a.z_out == nullptr || a.m == nullptr) return cudaErrorInvalidValue;
  YMaps mp;
  mp.w = lam;
  mp.m = m;
  mp.uc = m;
  mp.up = m;
  return launch_y_pipe_any<true>(a, K, mp, st);
}

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
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 256, 16, false, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 256, 16, false, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 256, 16, true, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 256, 16, true, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 512, 16, false, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 512, 16, false, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 512, 16, true, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<16, 512, 16, true, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 256, 16, false, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 256, 16, false, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 256, 16, true, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 256, 16, true, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 512, 16, false, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 512, 16, false, true>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 512, 16, true, false>, true);
  if (e == cudaSuccess) e = allow_smem(y_pipe_kernel<32, 512, 16, true, true>, true);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<8, 1024, 1>, false);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<16, 256, 1>, false);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<16, 512, 1>, false);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<16, 1024, 1>, false);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<32, 256, 1>, false);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<32, 512, 1>, false);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<32, 256, 2>, true);
  if (e == cudaSuccess) e = allow_smem(x_pipe_kernel<32, 128, 4>, true);
  if (e == cudaSuccess) e = allow_smem(x_band_kernel<32, 256, 2>, true);
  if (e == cudaSuccess) e = allow_smem(x_band_kernel<32, 128, 4>, true);
  if (e == cudaSuccess) e = allow_smem(x_band_kernel<32, 64, 8>, true);
  if (e == cudaSuccess) e = allow_smem(x_band_kernel<16, 512, 2>, true);
  if (e == cudaSuccess) e = allow_smem(x_band_kernel<16, 256, 4>, true);
  if (e == cudaSuccess) e = allow_smem(x_band_kernel<16, 128, 8>, true);
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

__global__ void scan_init_kernel(unsigned int* out3) {
  out3[0] = 0x7f7fffffu;
  out3[1] = 0u;
  out3[2] = 0u;
}

__global__ void scan_out_kernel(const unsigned int* out3, volatile unsigned int* host3) {
  host3[0] = out3[0];
  host3[1] = out3[1];
  host3[2] = out3[2];
  __threadfence_system();
}

cudaError_t launch_scan_m(const float* m, int nx, int ny, int ld, unsigned int* out3,
                          unsigned int* host3, cudaStream_t st) {
  scan_init_kernel<<<1, 1, 0, st>>>(out3);
  scan_m_kernel<<<152 * 4, 256, 0, st>>>(m, nx, ny, ld, out3);
  scan_out_kernel<<<1, 1, 0, st>>>(out3, host3);
  return cudaGetLastError();
}

__global__ void put_gd_kernel(GridDev* dst, const GridDev v) { *dst = v; }

cudaError_t launch_put_gd(GridDev* dst, const GridDev& v, cudaStream_t st) {
  put_gd_kernel<<<1, 1, 0, st>>>(dst, v);
  return cudaGetLastError();
}

}  // namespace adi
