// adi_device.cuh -- device building blocks of the tridiagonal line solves.
//
// Every system solved here has the shape of the ADI sub-problems of
// Section 2 (Eqs. fr1, fr2) in delta form:
//     -s_i x_{i-1} + (1 + 2 s_i) x_i - s_i x_{i+1} = d_i,   s_i >= 0,
// with x outside the line equal to zero (the Dirichlet ring, Eq. CN3).  The
// matrix is a strictly diagonally dominant M-matrix, so elimination without
// pivoting is stable and the solution is unique.
//
// Section 3.1 solves each system by cyclic reduction (CR): log2 levels that
// halve the system, a 2x2 solve, and log2 levels of back substitution.  Here
// a line is spread over the threads of a CTA (or of a thread-block cluster)
// and solved in three stages:
//   1. partition: each thread owns K consecutive unknowns in registers and
//      eliminates its interior ones, leaving two interface equations per
//      thread (its first and last unknown, coupled to the neighbouring
//      threads' interface unknowns) -- chunk_reduce();
//   2. the interface system (2 equations per thread, tridiagonal) is solved
//      in shared memory by CR levels down to `pcr` equations, then by
//      parallel cyclic reduction (PCR) in one warp with shuffles, then the CR
//      back substitution -- reduced_solve();
//   3. each thread recovers its interior unknowns from its two interface
//      values -- chunk_backsub().
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace adi {

// -------------------------------------------------------------------------
// arithmetic helpers
// -------------------------------------------------------------------------

__device__ __forceinline__ float rcp_t(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

__device__ __forceinline__ float div_t(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_t(double a, double b) { return a / b; }

// One equation a x_{i-1} + b x_i + c x_{i+1} = d of a (reduced) system.
template <typename T> struct alignas(4 * sizeof(T)) Eq {
  T a, b, c, d;
};

template <typename T> __device__ __forceinline__ Eq<T> eq_identity() {
  Eq<T> e;
  e.a = T(0); e.b = T(1); e.c = T(0); e.d = T(0);
  return e;
}

// Eliminate the couplings of `e` to its neighbours `lo` (below) and `hi`
// (above) -- one step of (parallel) cyclic reduction.
template <typename T>
__device__ __forceinline__ Eq<T> cr_combine(const Eq<T>& e, const Eq<T>& lo, const Eq<T>& hi) {
  T k1 = div_t(e.a, lo.b);
  T k2 = div_t(e.c, hi.b);
  Eq<T> r;
  r.a = -lo.a * k1;
  r.c = -hi.c * k2;
  r.b = e.b - lo.c * k1 - hi.a * k2;
  r.d = e.d - lo.d * k1 - hi.d * k2;
  return r;
}

template <typename T> __device__ __forceinline__ T shfl_up_t(T v, int s) {
  return __shfl_up_sync(0xffffffffu, v, s);
}
template <typename T> __device__ __forceinline__ T shfl_down_t(T v, int s) {
  return __shfl_down_sync(0xffffffffu, v, s);
}
template <typename T> __device__ __forceinline__ Eq<T> shfl_up_eq(const Eq<T>& e, int s) {
  Eq<T> r;
  r.a = __shfl_up_sync(0xffffffffu, e.a, s); r.b = __shfl_up_sync(0xffffffffu, e.b, s);
  r.c = __shfl_up_sync(0xffffffffu, e.c, s); r.d = __shfl_up_sync(0xffffffffu, e.d, s);
  return r;
}
template <typename T> __device__ __forceinline__ Eq<T> shfl_down_eq(const Eq<T>& e, int s) {
  Eq<T> r;
  r.a = __shfl_down_sync(0xffffffffu, e.a, s); r.b = __shfl_down_sync(0xffffffffu, e.b, s);
  r.c = __shfl_down_sync(0xffffffffu, e.c, s); r.d = __shfl_down_sync(0xffffffffu, e.d, s);
  return r;
}

// -------------------------------------------------------------------------
// 1. partition step on K consecutive unknowns held by one thread
// -------------------------------------------------------------------------
// In:  d[k] right-hand side, s[k] off-diagonal magnitude (row k reads
//      -s_k x_{k-1} + (1 + 2 s_k) x_k - s_k x_{k+1} = d_k).
// Out: e0 = interface equation of unknown 0:  A x_L + B x_0 + C x_{K-1} = D
//      e1 = interface equation of unknown K-1: A x_0 + B x_{K-1} + C x_R = D
//      (x_L = the previous thread's last unknown, x_R = the next thread's
//      first), and, for chunk_backsub, d[k] <- delta_k, s[k] <- gamma_k of
//      the forward elimination of the interior rows 1..K-2:
//          x_k = delta_k - q_k x_0 - gamma_k x_{k+1},  q_1 = gamma_1,
//          q_k = -gamma_k q_{k-1}.
// The first interior unknown x_1 = Y - Q x_0 + omega_{K-1} x_{K-1} follows
// from the same forward pass through the weights omega_1 = 1,
// omega_k = -gamma_{k-1} omega_{k-1} (the back substitution unrolled), so no
// second pass over the chunk is needed.
template <int K, typename T>
__device__ __forceinline__ void chunk_reduce(T (&d)[K], T (&s)[K], Eq<T>& e0, Eq<T>& e1) {
  static_assert(K >= 4, "chunk length must be at least 4");
  T s1 = s[1];
  T g = rcp_t(T(1) + T(2) * s1);
  T gam = -s1 * g;
  T del = d[1] * g;
  T q = gam;
  T om = T(1);
  T Y = del, Q = q;
  d[1] = del;
  s[1] = gam;
#pragma unroll
  for (int k = 2; k <= K - 2; ++k) {
    T sk = s[k];
    g = rcp_t(fma(sk, T(2) + gam, T(1)));
    om = -gam * om;
    T ng = -sk * g;
    del = fma(sk, del, d[k]) * g;
    q = -ng * q;
    gam = ng;
    Y = fma(om, del, Y);
    Q = fma(om, q, Q);
    d[k] = del;
    s[k] = gam;
  }
  T omK = -gam * om;
  T s0 = s[0];
  e0.a = -s0;
  e0.b = fma(s0, T(2) + Q, T(1));
  e0.c = -s0 * omK;
  e0.d = fma(s0, Y, d[0]);
  T sl = s[K - 1];
  e1.a = sl * q;
  e1.b = fma(sl, T(2) + gam, T(1));
  e1.c = -sl;
  e1.d = fma(sl, del, d[K - 1]);
}

// 3. interior unknowns from the interface values x_0 and x_{K-1}; on return
// d[k] = x_k for k = 0..K-1.
template <int K, typename T>
__device__ __forceinline__ void chunk_backsub(T (&d)[K], const T (&s)[K], T x0, T xl) {
  T qx = s[1] * x0;
  d[1] -= qx;
#pragma unroll
  for (int k = 2; k <= K - 2; ++k) {
    qx = -s[k] * qx;
    d[k] -= qx;
  }
  T x = xl;
#pragma unroll
  for (int k = K - 2; k >= 1; --k) {
    x = fma(-s[k], x, d[k]);
    d[k] = x;
  }
  d[0] = x0;
  d[K - 1] = xl;
}

// -------------------------------------------------------------------------
// 2. interface systems: cyclic reduction in shared memory, then PCR in a warp
// -------------------------------------------------------------------------
// nsys systems of N equations (N a power of two) at red[sys * N + i]; the
// solution goes to xs[sys * N + i].  All threads of the CTA must call this
// (it contains __syncthreads); the equations must be visible (the caller
// synchronises before).  pcr = size of the system handed to PCR (a power of
// two <= 32).  Unknowns outside 0..N-1 are zero.
template <typename T>
__device__ void reduced_solve(Eq<T>* red, T* xs, int nsys, int N, int log2N, int pcr) {
  const int nthreads = blockDim.x;
  const int tid = threadIdx.x;
  int L = 0;
  while ((N >> L) > pcr) ++L;  // CR levels before the switch

  // forward CR: at level l the equations i = 2^{l+1} j + 2^{l+1} - 1 absorb
  // their neighbours at distance 2^l.
  for (int l = 0; l < L; ++l) {
    const int sft = l + 1;
    const int st = 1 << l;
    const int per_sys_log = log2N - sft;
    const int total = nsys << per_sys_log;
    for (int t = tid; t < total; t += nthreads) {
      const int sys = t >> per_sys_log;
      const int jj = t & ((1 << per_sys_log) - 1);
      const int i = (jj << sft) + (st << 1) - 1;
      Eq<T>* R = red + (size_t)sys * N;
      Eq<T> e = R[i];
      Eq<T> lo = R[i - st];
      Eq<T> hi = (i + st < N) ? R[i + st] : eq_identity<T>();
      R[i] = cr_combine(e, lo, hi);
    }
    __syncthreads();
  }

  // PCR on the M = N >> L remaining equations i = 2^L (j + 1) - 1, lane j.
  const int M = N >> L;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = nthreads >> 5;
  for (int sys = warp; sys < nsys; sys += nwarps) {
    const int i = ((lane + 1) << L) - 1;
    Eq<T> e = (lane < M) ? red[(size_t)sys * N + i] : eq_identity<T>();
    for (int st = 1; st < M; st <<= 1) {
      Eq<T> lo, hi;
      lo.a = shfl_up_t(e.a, st); lo.b = shfl_up_t(e.b, st);
      lo.c = shfl_up_t(e.c, st); lo.d = shfl_up_t(e.d, st);
      hi.a = shfl_down_t(e.a, st); hi.b = shfl_down_t(e.b, st);
      hi.c = shfl_down_t(e.c, st); hi.d = shfl_down_t(e.d, st);
      if (lane < st) lo = eq_identity<T>();
      if (lane + st >= M) hi = eq_identity<T>();
      e = cr_combine(e, lo, hi);
    }
    if (lane < M) xs[(size_t)sys * N + i] = div_t(e.d, e.b);
  }
  __syncthreads();

  // backward CR: the equations removed at level l are i = 2^{l+1} j + 2^l - 1.
  for (int l = L - 1; l >= 0; --l) {
    const int sft = l + 1;
    const int st = 1 << l;
    const int per_sys_log = log2N - sft;
    const int total = nsys << per_sys_log;
    for (int t = tid; t < total; t += nthreads) {
      const int sys = t >> per_sys_log;
      const int jj = t & ((1 << per_sys_log) - 1);
      const int i = (jj << sft) + st - 1;
      const Eq<T>* R = red + (size_t)sys * N;
      T* X = xs + (size_t)sys * N;
      Eq<T> e = R[i];
      T xl = (i - st >= 0) ? X[i - st] : T(0);
      T xr = (i + st < N) ? X[i + st] : T(0);
      X[i] = div_t(e.d - e.a * xl - e.c * xr, e.b);
    }
    __syncthreads();
  }
}

}  // namespace adi

namespace adi {

// -------------------------------------------------------------------------
// Block cyclic reduction of the interface system across the lanes of a warp
// -------------------------------------------------------------------------
// A segment [a, c] of consecutive unknowns is summarised by two equations:
//   f:  A x_{a-1} + B x_a + C x_c     = D
//   l:  A x_a     + B x_c + C x_{c+1} = D
// (a chunk's interface equations e0, e1 are such a summary).  Merging the
// adjacent segments L = [a, b] and R = [b+1, c] eliminates the interface
// unknowns x_b and x_{b+1} between them -- one level of cyclic reduction on
// the interface system -- and leaves the summary of [a, c].  The node keeps
//   x_b     = xb0 + xba x_a + xbc x_c,   x_{b+1} = y0 + yba x_a + ybc x_c
// for the back substitution.
template <typename T> struct Seg {
  Eq<T> f, l;
};

template <typename T> struct Node {
  T xb0, xba, xbc, y0, yba, ybc;
};

template <typename T>
__device__ __forceinline__ Seg<T> seg_merge(const Seg<T>& L, const Seg<T>& R, Node<T>& nd) {
  const T idet = rcp_t(L.l.b * R.f.b - L.l.c * R.f.a);
  nd.xb0 = (R.f.b * L.l.d - L.l.c * R.f.d) * idet;
  nd.xba = -(R.f.b * L.l.a) * idet;
  nd.xbc = (L.l.c * R.f.c) * idet;
  nd.y0 = (L.l.b * R.f.d - R.f.a * L.l.d) * idet;
  nd.yba = (R.f.a * L.l.a) * idet;
  nd.ybc = -(L.l.b * R.f.c) * idet;
  Seg<T> S;
  S.f.a = L.f.a;
  S.f.b = fma(L.f.c, nd.xba, L.f.b);
  S.f.c = L.f.c * nd.xbc;
  S.f.d = fma(-L.f.c, nd.xb0, L.f.d);
  S.l.a = R.l.a * nd.yba;
  S.l.b = fma(R.l.a, nd.ybc, R.l.b);
  S.l.c = R.l.c;
  S.l.d = fma(-R.l.a, nd.y0, R.l.d);
  return S;
}

template <typename T> __device__ __forceinline__ Eq<T> shfl_xor_eq(const Eq<T>& e, int m) {
  Eq<T> r;
  r.a = __shfl_xor_sync(0xffffffffu, e.a, m);
  r.b = __shfl_xor_sync(0xffffffffu, e.b, m);
  r.c = __shfl_xor_sync(0xffffffffu, e.c, m);
  r.d = __shfl_xor_sync(0xffffffffu, e.d, m);
  return r;
}

// Node slot of level t for the group of `lane` (31 slots per warp: 16 nodes
// at level 0, 8 at level 1, ...).
__device__ __forceinline__ int node_slot(int t, int lane) {
  return (32 - (32 >> t)) + (lane >> (t + 1));
}

// Up-sweep: merge the lanes' segments pairwise over `levels` levels (groups
// of 2^levels consecutive lanes).  Every lane of a group ends with the
// group's summary; node data go to nodes[0..30] (one warp's slots).
template <typename T>
__device__ __forceinline__ Seg<T> warp_tree_up(Seg<T> S, Node<T>* nodes, int lane, int levels) {
  for (int t = 0; t < levels; ++t) {
    const int m = 1 << t;
    Seg<T> P;
    P.f = shfl_xor_eq(S.f, m);
    P.l = shfl_xor_eq(S.l, m);
    // order the pair with selects (not a branch: the lanes of a warp differ)
    const bool right = (lane & m) != 0;
    Seg<T> L, R;
    L.f = right ? P.f : S.f;
    L.l = right ? P.l : S.l;
    R.f = right ? S.f : P.f;
    R.l = right ? S.l : P.l;
    Node<T> nd;
    S = seg_merge(L, R, nd);
    if ((lane & (2 * m - 1)) == 0) nodes[node_slot(t, lane)] = nd;
  }
  __syncwarp();
  return S;
}

// Down-sweep: from the group's outer values (xa, xc) to this lane's segment
// end values.
template <typename T>
__device__ __forceinline__ void warp_tree_down(const Node<T>* nodes, int lane, int levels, T& xa,
                                               T& xc) {
  for (int t = levels - 1; t >= 0; --t) {
    const Node<T> nd = nodes[node_slot(t, lane)];
    if (lane & (1 << t)) xa = fma(nd.ybc, xc, fma(nd.yba, xa, nd.y0));
    else xc = fma(nd.xbc, xc, fma(nd.xba, xa, nd.xb0));
  }
}

// Both end values of a summarised segment whose outside neighbours are zero.
template <typename T>
__device__ __forceinline__ void seg_solve_closed(const Seg<T>& S, T& xa, T& xc) {
  // f: B xa + C xc = D ;  l: A xa + B xc = D
  const T idet = rcp_t(S.f.b * S.l.b - S.f.c * S.l.a);
  xa = (S.f.d * S.l.b - S.f.c * S.l.d) * idet;
  xc = (S.f.b * S.l.d - S.l.a * S.f.d) * idet;
}

// Parallel cyclic reduction of up to 64 equations in one warp, lane l holding
// equations 2l (E0) and 2l+1 (E1); n_eq = number of real equations (lanes
// beyond hold identities).  On return E0.d / E0.b and E1.d / E1.b are the
// solution.  Unknowns outside 0..n_eq-1 are zero.
template <typename T>
__device__ __forceinline__ void pcr64(Eq<T>& E0, Eq<T>& E1, int lane, int n_eq) {
  const Eq<T> I = eq_identity<T>();
  // distance 1
  {
    Eq<T> prev1 = shfl_up_eq(E1, 1);      // equation 2l - 1
    Eq<T> next0 = shfl_down_eq(E0, 1);    // equation 2l + 2
    if (lane == 0) prev1 = I;
    if (2 * lane + 2 >= n_eq) next0 = I;
    const Eq<T> e1hi = (2 * lane + 1 < n_eq) ? E1 : I;
    const Eq<T> n0 = cr_combine(E0, prev1, e1hi);
    const Eq<T> n1 = cr_combine(E1, E0, next0);
    E0 = n0;
    E1 = n1;
  }
  // distances 2, 4, ..., 32 (lane offsets 1, 2, ..., 16); a level is needed
  // only while the coupling distance 2h is below the number of equations
  for (int h = 1; h < 32 && 2 * h < n_eq; h <<= 1) {
    const int s = 2 * h;
    Eq<T> lo0 = shfl_up_eq(E0, h), lo1 = shfl_up_eq(E1, h);
    Eq<T> hi0 = shfl_down_eq(E0, h), hi1 = shfl_down_eq(E1, h);
    if (2 * lane - s < 0) lo0 = I;
    if (2 * lane + 1 - s < 0) lo1 = I;
    if (2 * lane + s >= n_eq || lane + h >= 32) hi0 = I;
    if (2 * lane + 1 + s >= n_eq || lane + h >= 32) hi1 = I;
    const Eq<T> n0 = cr_combine(E0, lo0, hi0);
    const Eq<T> n1 = cr_combine(E1, lo1, hi1);
    E0 = n0;
    E1 = n1;
  }
}

// Partition step in two independent halves (K >= 32): each half is
// reduced to its two interface equations (two short elimination chains the
// compiler can interleave) and the halves are merged into the chunk's
// summary; `nd` keeps the merge for chunk_backsub_split.  Below K = 32 this
// is chunk_reduce itself.
template <int K, typename T>
__device__ __forceinline__ void chunk_reduce_split(T (&d)[K], T (&s)[K], Seg<T>& S, Node<T>& nd) {
  if constexpr (K >= 32) {
    constexpr int H = K / 2;
    T(&dA)[H] = *reinterpret_cast<T(*)[H]>(&d[0]);
    T(&sA)[H] = *reinterpret_cast<T(*)[H]>(&s[0]);
    T(&dB)[H] = *reinterpret_cast<T(*)[H]>(&d[H]);
    T(&sB)[H] = *reinterpret_cast<T(*)[H]>(&s[H]);
    Seg<T> A, B;
    chunk_reduce<H, T>(dA, sA, A.f, A.l);
    chunk_reduce<H, T>(dB, sB, B.f, B.l);
    S = seg_merge(A, B, nd);
  } else {
    chunk_reduce<K, T>(d, s, S.f, S.l);
  }
}

// Back substitution matching chunk_reduce_split: x_0 = xa, x_{K-1} = xc.
template <int K, typename T>
__device__ __forceinline__ void chunk_backsub_split(T (&d)[K], const T (&s)[K], const Node<T>& nd,
                                                    T xa, T xc) {
  if constexpr (K >= 32) {
    constexpr int H = K / 2;
    T(&dA)[H] = *reinterpret_cast<T(*)[H]>(&d[0]);
    const T(&sA)[H] = *reinterpret_cast<const T(*)[H]>(&s[0]);
    T(&dB)[H] = *reinterpret_cast<T(*)[H]>(&d[H]);
    const T(&sB)[H] = *reinterpret_cast<const T(*)[H]>(&s[H]);
    const T xb = fma(nd.xbc, xc, fma(nd.xba, xa, nd.xb0));  // x_{H-1}
    const T xb1 = fma(nd.ybc, xc, fma(nd.yba, xa, nd.y0));  // x_H
    chunk_backsub<H, T>(dA, sA, xa, xb);
    chunk_backsub<H, T>(dB, sB, xb1, xc);
  } else {
    chunk_backsub<K, T>(d, s, xa, xc);
  }
}

}  // namespace adi
