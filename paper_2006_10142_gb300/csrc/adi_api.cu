// adi_api.cu -- the C ABI of libadiwave.so (declared in include/adiwave.h):
// handle lifetime, validation, launch planning, the time loop with CUDA
// graph replay, state access, measurement hooks.
//
// Algorithm 1 (Section 3.1) keeps four buffers u, U0, Ux, Uy and swaps them
// after every step.  Here a grid owns two state buffers -- buf[cur] = u^k,
// buf[1-cur] = u^{k-1} -- plus one scratch field w; the y sweep writes
// u^{k+1} over u^{k-1} and `cur` flips, which is the same rotation without
// copies.  Two consecutive steps restore the orientation, so a captured
// graph of one step pair is replayed for the whole loop.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/adiwave.h"
#include "adi_internal.h"
#include "adi_run.h"
#include "adi_sweeps.cuh"

using namespace adi;

namespace adi {

static const char* kVersion = "adiwave 0.1 sm_103a";

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int fail(adi_wave* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(adi_wave* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, ADI_ECUDA, m);
}

// Launch geometry of one grid (the autotuner's knobs made concrete).
int plan_grid(Grid& G, const adi_wave_tuning& t, std::string& why) {
  const double sxm = G.dt * G.dt * G.mmax / (2.0 * G.hx * G.hx);
  const double sym = G.dt * G.dt * G.mmax / (2.0 * G.hy * G.hy);
  // dominance ratio (|a| + |c|) / |b| = 2s / (1 + 2s); weak above 0.9
  const bool weak_x = 2.0 * sxm / (1.0 + 2.0 * sxm) > kWeakDominance;
  const bool weak_y = 2.0 * sym / (1.0 + 2.0 * sym) > kWeakDominance;
  GridPlan P = G.plan;
  P.fp64x = G.fp64mode == ADI_FP64_ALWAYS || (G.fp64mode == ADI_FP64_AUTO && weak_x);
  P.fp64y = G.fp64mode == ADI_FP64_ALWAYS || (G.fp64mode == ADI_FP64_AUTO && weak_y);
  if (t.solver < ADI_SOLVER_AUTO || t.solver > ADI_SOLVER_CR_SMEM) { why = "unknown solver"; return ADI_EINVAL; }
  P.tree = t.solver != ADI_SOLVER_CR_SMEM;
  int pcr = t.pcr_size ? t.pcr_size : 32;
  if (pcr != 2 && pcr != 4 && pcr != 8 && pcr != 16 && pcr != 32) { why = "pcr_size must be 2..32, a power of two"; return ADI_EINVAL; }
  P.pcr = pcr;

  const int ct = t.cta_threads;
  const int cty = t.cta_threads_y;
  if (cty != 0 && cty != 64 && cty != 128 && cty != 256 && cty != 512 && cty != 1024) { why = "cta_threads_y must be 64..1024, a power of two"; return ADI_EINVAL; }
  if (ct != 0 && ct != 64 && ct != 128 && ct != 256 && ct != 512 && ct != 1024) { why = "cta_threads must be 64..1024, a power of two"; return ADI_EINVAL; }
  // ---- x sweep
  {
    const int maxT = std::min(P.fp64x ? 512 : 1024, ct ? ct : 1024);
    int K = t.chunk_x;
    // FP64 rows: K = 16 from 512 columns (at 4096 it ran the x sweep 1.44x
    // faster than K = 8, whose extra tree levels cost more than a few spills)
    if (K == 0) K = P.fp64x ? (G.nx >= 512 ? 16 : 8) : (G.nx >= 512 ? 16 : (G.nx >= 64 ? 8 : 4));
    // FP32 rows that fit 512 threads at 32 unknowns each: longer chunks win
    // (fewer interface equations per row, no register spills)
    // (from 2048 columns; at 1024 the adjoint's row solves run faster with K = 16)
    if (t.chunk_x == 0 && !P.fp64x && G.nx >= 2048 && next_pow2((G.nx + 31) / 32) <= std::min(maxT, 512)) K = 32;
    if (K != 4 && K != 8 && K != 16 && K != 32) { why = "chunk_x must be 4, 8, 16 or 32"; return ADI_EINVAL; }
    while (next_pow2((G.nx + K - 1) / K) > maxT && K < 32) K *= 2;
    const int tsys = next_pow2((G.nx + K - 1) / K);
    if (tsys > maxT) { why = "nx too large for one CTA per row"; return ADI_EUNSUPPORTED; }
    int spc = t.rows_per_cta;
    // default: about 256 threads per CTA (one row per CTA once a row needs
    // more), at least 256 CTAs when the grid has the rows for it
    if (spc == 0) spc = std::max(1, std::min(std::min(maxT, 256) / tsys, G.ny / 256));
    if (spc < 1 || spc * tsys > maxT) { why = "rows_per_cta too large"; return ADI_EINVAL; }
    // whole warps only: the interface solve uses full-warp shuffles
    if (tsys < 32) {
      const int q = 32 / tsys;
      spc = (spc + q - 1) / q * q;
      if (spc * tsys > maxT) spc = maxT / tsys;
    }
    if (x_smem_bytes(spc, tsys, P.fp64x, P.tree) > (size_t)kMaxDynSmem) { why = "x sweep shared memory too large"; return ADI_EUNSUPPORTED; }
    if (t.x_stage < ADI_STAGE_AUTO || t.x_stage > ADI_STAGE_BAND || t.x_stage == ADI_STAGE_COOP) { why = "unknown x_stage"; return ADI_EINVAL; }
    // TMA pipeline: FP32 tree solver, rows of >= 256 staged floats, K >= 8,
    // K = 32 only up to 512 threads (register budget)
    const bool pipe_ok = !P.fp64x && P.tree && tsys * K >= 256 && K >= 8 &&
                         (K < 32 || spc * tsys <= 512) &&
                         x_pipe_smem_bytes(spc, tsys, K, 1) <= (size_t)kMaxDynSmem;
    // a row split over a cluster of two CTAs (two pairs per SM): K = 32, one
    // row per CTA pair, at least 256 staged floats per CTA
    const bool pair_ok = pipe_ok && K == 32 && spc == 1 && tsys >= 64 &&
                         x_pipe_smem_bytes(1, tsys / 2, K, 2) <= (size_t)kMaxDynSmem;
    // four CTAs of at least one warp each (four per SM)
    const bool quad_ok = pipe_ok && K == 32 && spc == 1 && tsys >= 128 && tsys <= 512 &&
                         x_pipe_smem_bytes(1, tsys / 4, K, 4) <= (size_t)kMaxDynSmem;
    if (t.x_cluster < 0 || t.x_cluster > 8 || (t.x_cluster > 2 && t.x_cluster != 4 && t.x_cluster != 8)) { why = "x_cluster must be 0, 1, 2, 4 or 8"; return ADI_EINVAL; }
    // band form: rows of K = 16 or 32 split over 2, 4 or 8 CTAs of >= 32
    // threads (at most 512 / 256) each holding >= 1024 unknowns of the row
    auto band_ok = [&](int xc) {
      return !P.fp64x && P.tree && (K == 16 || K == 32) && spc == 1 && tsys / xc >= 32 &&
             tsys / xc <= (K == 16 ? 512 : 256) && tsys / xc * K >= 1024 &&
             xc * (tsys / xc / 32) <= 32 && x_band_smem_bytes(tsys / xc, K, xc) <= (size_t)kMaxDynSmem;
    };
    const bool smem_ok = !P.fp64x &&
                         align64(x_smem_bytes(spc, tsys, P.fp64x, P.tree)) + x_stage_bytes(spc * tsys, K) <=
                             (size_t)kMaxDynSmem;
    int xs = t.x_stage;
    // automatic: the band form over CTA pairs for rows of 256 or more
    // threads at K = 32 (8192 columns and beyond; at 16384^2 0.856 against
    // 0.942 ms for the row-block pipeline)
    if (xs == ADI_STAGE_AUTO && (t.x_cluster == 0 || t.x_cluster == 2) && tsys >= 256 && band_ok(2))
      xs = ADI_STAGE_BAND;
    if (xs == ADI_STAGE_BAND) {
      const int bxc = t.x_cluster >= 2 ? t.x_cluster : 2;
      if (!band_ok(bxc)) { why = "x band form not available for this shape"; return ADI_EUNSUPPORTED; }
      P.x_stage = xs;
      P.xc = bxc;
      P.kx = K;
      P.log2tsys = ilog2(tsys);
      P.spc = spc;
      goto x_done;
    }
    if (xs == ADI_STAGE_AUTO) xs = pipe_ok ? ADI_STAGE_TMA : ADI_STAGE_DIRECT;
    if (xs == ADI_STAGE_TMA && !pipe_ok) { why = "x TMA pipeline not available for this shape"; return ADI_EUNSUPPORTED; }
    if (xs == ADI_STAGE_SMEM && !smem_ok) {
      if (P.fp64x) xs = ADI_STAGE_DIRECT;
      else { why = "x staging does not fit shared memory"; return ADI_EUNSUPPORTED; }
    }
    P.x_stage = xs;
    int xc = 1;
    if (xs == ADI_STAGE_TMA) {
      if (t.x_cluster == 2 && !pair_ok) { why = "x_cluster = 2 needs the TMA pipeline, K = 32 and one row per CTA"; return ADI_EUNSUPPORTED; }
      if (t.x_cluster == 4 && !quad_ok) { why = "x_cluster = 4 needs the TMA pipeline, K = 32, one row per CTA and 128..512 threads per row"; return ADI_EUNSUPPORTED; }
      // automatic: rows of 512 threads (16384 unknowns at K = 32) over four
      // CTAs (measured 2 % faster than pairs at 16384^2), else pairs
      if (t.x_cluster == 2 || (t.x_cluster == 0 && pair_ok && tsys >= 512)) xc = 2;
      if (t.x_cluster == 4 || (t.x_cluster == 0 && quad_ok && tsys >= 512)) xc = 4;
    } else if (t.x_cluster >= 2) {
      why = "x_cluster = 2 needs the TMA pipeline";
      return ADI_EUNSUPPORTED;
    }
    P.xc = xc;
    P.kx = K;
    P.log2tsys = ilog2(tsys);
    P.spc = spc;
  }
x_done:
  // ---- y sweep
  {
    const int maxT = std::min(P.fp64y ? 512 : 1024, cty ? cty : 1024);
    const int maxC = 16;
    int W = t.cols_per_cta ? t.cols_per_cta : (G.nx >= 1024 && G.ny >= 1024 ? 16 : 8);
    if (W != 4 && W != 8 && W != 16 && W != 32) { why = "cols_per_cta must be 4, 8, 16 or 32"; return ADI_EINVAL; }
    int ymaxT = maxT;
    auto geom = [&](int K, int& tcol, int& C) {
      const int ttot = next_pow2((G.ny + K - 1) / K);
      tcol = std::min(ttot, ymaxT / W);
      if (W * tcol < 32) tcol = 32 / W;  // whole warps; extra chunks are empty rows
      C = std::max(1, ttot / tcol);
    };
    // the tree's top system holds at most 32 warp groups per column
    auto fits = [&](int K) {
      int tcol, C;
      geom(K, tcol, C);
      const int groups = C * std::max(1, tcol / 32);
      return C <= maxC && (!P.tree || groups <= 32);
    };
    int K = t.chunk_y;
    if (K == 0) {
      K = P.fp64y ? 8 : (G.ny >= 64 ? 8 : 4);
      // prefer portable clusters (<= 8 CTAs) and a top system that fits a warp
      while (K < 32) {
        int tcol, C;
        geom(K, tcol, C);
        if (C <= 8 && fits(K)) break;
        K *= 2;
      }
    }
    // FP32, long columns, CTA size not given: 32 rows per thread, and the
    // largest CTA (up to 512 threads, one per SM) that still leaves at least
    // 512 CTAs (strips x cluster size) in the grid; smaller grids get
    // smaller CTAs rather than idle SMs
    if (cty == 0 && t.chunk_y == 0 && !P.fp64y && G.ny >= 1024) {
      const int ttot = next_pow2((G.ny + 31) / 32);
      const int strips = (G.nx + W - 1) / W;
      int tcol = 0;
      for (int tc = std::max(1, 512 / W); tc >= std::max(1, 64 / W); tc >>= 1) {
        if (tc > ttot || ttot / tc > maxC) continue;
        tcol = tc;
        if ((long long)strips * (ttot / tc) >= 512) break;
      }
      const int groups = tcol ? (ttot / tcol) * std::max(1, tcol / 32) : 0;
      if (tcol && (!P.tree || groups <= 32)) {
        K = 32;
        ymaxT = W * tcol;
      }
    }
    if (K != 4 && K != 8 && K != 16 && K != 32) { why = "chunk_y must be 4, 8, 16 or 32"; return ADI_EINVAL; }
    if (t.y_stage < ADI_STAGE_AUTO || t.y_stage > ADI_STAGE_COOP) { why = "unknown y_stage"; return ADI_EINVAL; }
    int tcol, C;
    geom(K, tcol, C);
    // Column segments joined through global memory (adi_ycoop.cu): strips of
    // 16 columns (K = 32 with 256 or 512 threads; K = 16 with 512) or of 32
    // columns (512 threads, K = 32 or 16); at most 32 segments per column.
    // Chosen automatically for long columns (from 8192 rows, strips of 16,
    // 512 threads: the cluster form needs clusters of 8 or 16 CTAs there and
    // measured 3-6 % slower at 8192^2 and 16384^2).
    const bool coop_auto = t.y_stage == ADI_STAGE_AUTO && t.chunk_y == 0 && cty == 0 &&
                           (t.cols_per_cta == 0 || t.cols_per_cta == 16) && W == 16 &&
                           !P.fp64y && P.tree && G.ny >= 8192;
    if (t.y_stage == ADI_STAGE_COOP || coop_auto) {
      const int cW = t.cols_per_cta ? t.cols_per_cta : 16;
      const int cK = t.chunk_y ? t.chunk_y : 32;
      const int cthr = cty ? cty : 512;
      const int ctc = cthr / cW;
      const int cC = (G.ny + ctc * cK - 1) / (ctc * cK);
      const bool shape_ok = cW == 16 ? ((cK == 32 && (cthr == 256 || cthr == 512)) || (cK == 16 && cthr == 512))
                                     : (cW == 32 && cthr == 512 && (cK == 32 || cK == 16));
      const bool coop_ok = !P.fp64y && P.tree && shape_ok && cC >= 1 && cC <= 32 && ctc * cK >= 64 &&
                           y_coop_smem_bytes(cW, ctc, cK, cC) <= (size_t)kMaxDynSmem;
      if (!coop_ok && !coop_auto) {
        why = "y segments through global memory not available for this shape";
        return ADI_EUNSUPPORTED;
      }
      if (coop_ok) {
        P.y_stage = ADI_STAGE_COOP;
        P.ky = cK;
        P.log2W = ilog2(cW);
        P.log2tcol = ilog2(ctc);
        P.C = cC;
        goto y_done;
      }
    }
    if (!fits(K)) { why = "ny too large for this chunk_y (cluster or top system)"; return ADI_EUNSUPPORTED; }
    const size_t ysm = align64(y_smem_bytes(W, C, tcol, P.fp64y, P.tree));
    const size_t ystage = y_stage_bytes(W * tcol, K);
    int stage = t.y_stage;
    // pipelined strips: FP32 tree solver, 16 columns, K >= 16, <= 512 threads
    const bool ypipe_ok = !P.fp64y && P.tree && W == 16 && (K == 32 || K == 16) &&
                          W * tcol <= 512 && W * tcol >= 32 && tcol * K >= 64 &&
                          y_pipe_smem_bytes(W, C, tcol, K) <= (size_t)kMaxDynSmem;
    if (stage == ADI_STAGE_TMA && !ypipe_ok) { why = "y pipeline not available for this shape"; return ADI_EUNSUPPORTED; }
    if (stage == ADI_STAGE_AUTO && ypipe_ok) stage = ADI_STAGE_TMA;
    if (stage == ADI_STAGE_AUTO) {
      // shared-memory staging unless it would keep a second CTA off the SM
      // (kernels of <= 512 threads with K >= 16 take up to 128 registers)
      const int regs = (K >= 16 && W * tcol <= 512) ? 128 : 64;
      const int by_regs = std::max(1, 65536 / (regs * W * tcol));
      const size_t per_sm = 228 * 1024;
      stage = (std::min(by_regs, 2) * (ysm + ystage + 1024) <= per_sm) ? ADI_STAGE_SMEM : ADI_STAGE_L2;
    }
    if (stage != ADI_STAGE_TMA && ysm + (stage == ADI_STAGE_SMEM ? ystage : 0) > (size_t)kMaxDynSmem) {
      why = "y sweep shared memory too large";
      return ADI_EUNSUPPORTED;
    }
    P.y_stage = stage;
    P.ky = K;
    P.log2W = ilog2(W);
    P.log2tcol = ilog2(tcol);
    P.C = C;
  }
y_done:
  P.graph = (t.use_graph >= 0) ? 1 : 0;
  P.cta_threads = ct;
  P.cta_threads_y = cty;
  if (t.persist < -1 || t.persist > 1) { why = "persist must be -1, 0 or 1"; return ADI_EINVAL; }
  P.persist = t.persist > 0 ? 1 : 0;
  G.plan = P;
  return ADI_OK;
}

}  // namespace adi

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" const char* adi_wave_version(void) { return kVersion; }

extern "C" const char* adi_wave_strerror(int code) {
  switch (code) {
    case ADI_OK: return "ok";
    case ADI_EINVAL: return "invalid argument";
    case ADI_ENOMEM: return "out of memory";
    case ADI_ECUDA: return "CUDA runtime error";
    case ADI_ENUMERIC: return "non-finite value produced";
    case ADI_ETIMEOUT: return "bounded device wait expired";
    case ADI_ESTATE: return "call not valid in the handle's state";
    case ADI_EUNSUPPORTED: return "not supported for this shape or mode";
    default: return "unknown error code";
  }
}

// Detail of the last adi_wave_init failure on this thread (the handle is gone).
static thread_local std::string g_init_error;

// Detail of a failed handle-less call, reported by adi_wave_last_error(NULL).
void adi::set_thread_error(const std::string& msg) { g_init_error = msg; }

extern "C" const char* adi_wave_last_error(const adi_wave* h) {
  return h ? h->err.c_str() : g_init_error.c_str();
}

extern "C" int adi_wave_init(adi_wave** out, const adi_wave_desc* desc, int32_t n_shots,
                             const float* const* m, const float* const* phi,
                             const float* const* psi, const adi_source* src, void* stream) {
  if (!out) return ADI_EINVAL;
  *out = nullptr;
  if (!desc || n_shots < 1 || !m || !phi) return ADI_EINVAL;
  for (int s = 0; s < n_shots; ++s) {
    const adi_wave_desc& d = desc[s];
    if (d.nx < 1 || d.ny < 1 || d.nx > 32768 || d.ny > 32768) return ADI_EINVAL;
    if (!(d.lx > 0) || !(d.ly > 0) || !(d.dt > 0) || !std::isfinite(d.dt)) return ADI_EINVAL;
    if (d.start != ADI_START_PAPER && d.start != ADI_START_TAYLOR2) return ADI_EINVAL;
    if (d.fp64_solve < ADI_FP64_AUTO || d.fp64_solve > ADI_FP64_ALWAYS) return ADI_EINVAL;
    if (!m[s] || !phi[s]) return ADI_EINVAL;
    if (src && src[s].ix >= 0 &&
        (src[s].ix >= d.nx || src[s].iy < 0 || src[s].iy >= d.ny)) return ADI_EINVAL;
  }
  adi_wave* h = new (std::nothrow) adi_wave();
  if (!h) return ADI_ENOMEM;
  int rc = h->create(desc, n_shots, m, phi, psi, src, (cudaStream_t)stream);
  if (rc != ADI_OK) {
    g_init_error = h->err;
    delete h;
    return rc;
  }
  *out = h;
  return ADI_OK;
}

extern "C" int adi_wave_reset(adi_wave* h, const float* const* m, const float* const* phi,
                              const float* const* psi, const adi_source* src, void* stream) {
  if (!h || !phi) return ADI_EINVAL;
  return h->reset(m, phi, psi, src, (cudaStream_t)stream);
}

extern "C" int adi_wave_step(adi_wave* h, const adi_source* src, void* stream) {
  if (!h) return ADI_EINVAL;
  return h->run(1, src, nullptr, 0, nullptr, (cudaStream_t)stream, /*record=*/false);
}

extern "C" int adi_wave_run(adi_wave* h, int32_t steps, const adi_source* src,
                            const int32_t* rec_xy, int32_t n_rec, float* traces, void* stream) {
  if (!h) return ADI_EINVAL;
  return h->run(steps, src, rec_xy, n_rec, traces, (cudaStream_t)stream, /*record=*/true);
}

extern "C" int adi_wave_set_checkpointing(adi_wave* h, int32_t every) {
  if (!h || every < 0) return ADI_EINVAL;
  h->ckpt_every = every;
  return ADI_OK;
}

extern "C" int adi_wave_adjoint(adi_wave* h, const float* resid, double* grad_m,
                                float* grad_wavelet, int32_t ckpt_every, void* stream) {
  if (!h) return ADI_EINVAL;
  return h->adjoint(resid, grad_m, grad_wavelet, ckpt_every, (cudaStream_t)stream);
}

extern "C" int adi_wave_get_state(const adi_wave* h, int32_t shot, float* u_prev, float* u_cur,
                                  int64_t* k, void* stream) {
  if (!h || shot < 0 || shot >= (int)h->g.size()) return ADI_EINVAL;
  const Grid& G = h->g[shot];
  cudaStream_t st = (cudaStream_t)stream;
  const size_t wb = sizeof(float) * (size_t)G.nx;
  if (u_prev) {
    cudaError_t e = cudaMemcpy2DAsync(u_prev, wb, G.buf[1 - G.cur], sizeof(float) * G.ld, wb, G.ny,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(const_cast<adi_wave*>(h), e, "get_state");
  }
  if (u_cur) {
    cudaError_t e = cudaMemcpy2DAsync(u_cur, wb, G.buf[G.cur], sizeof(float) * G.ld, wb, G.ny,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(const_cast<adi_wave*>(h), e, "get_state");
  }
  if (k) *k = G.k;
  return ADI_OK;
}

extern "C" int adi_wave_set_state(adi_wave* h, int32_t shot, const float* u_prev,
                                  const float* u_cur, int64_t k, void* stream) {
  if (!h || shot < 0 || shot >= (int)h->g.size() || !u_prev || !u_cur) return ADI_EINVAL;
  return h->set_state(shot, u_prev, u_cur, k, (cudaStream_t)stream);
}

extern "C" int adi_wave_sync_status(adi_wave* h, void* stream) {
  if (!h) return ADI_EINVAL;
  return h->sync_status((cudaStream_t)stream);
}

extern "C" void adi_wave_destroy(adi_wave* h) { delete h; }

extern "C" int adi_wave_get_tuning(const adi_wave* h, adi_wave_tuning* t) {
  if (!h || !t) return ADI_EINVAL;
  const GridPlan& P = h->g[0].plan;
  t->chunk_x = P.kx;
  t->chunk_y = P.ky;
  t->rows_per_cta = P.spc;
  t->cols_per_cta = 1 << P.log2W;
  t->pcr_size = P.pcr;
  t->use_graph = P.graph ? 1 : -1;
  t->solver = P.tree ? ADI_SOLVER_TREE : ADI_SOLVER_CR_SMEM;
  t->cta_threads = P.cta_threads;
  t->cta_threads_y = P.cta_threads_y;
  t->y_stage = P.y_stage;
  t->persist = P.persist ? 1 : -1;
  t->x_stage = P.x_stage;
  t->x_cluster = P.xc;
  return ADI_OK;
}

extern "C" int adi_wave_set_tuning(adi_wave* h, const adi_wave_tuning* t) {
  if (!h || !t) return ADI_EINVAL;
  return h->set_tuning(*t);
}

extern "C" int adi_wave_profile(adi_wave* h, int32_t enable) {
  if (!h) return ADI_EINVAL;
  h->profile = enable != 0;
  return ADI_OK;
}

extern "C" int adi_wave_profile_read(adi_wave* h, double* ms, int64_t* launches, int32_t n_kinds) {
  if (!h || n_kinds < 0) return ADI_EINVAL;
  return h->profile_read(ms, launches, n_kinds);
}

extern "C" int64_t adi_wave_launch_count(const adi_wave* h) { return h ? h->launches : 0; }

extern "C" int adi_wave_set_batch_mode(adi_wave* h, int32_t mode) {
  if (!h || h->g.size() < 2 || mode < 0 || mode > 2) return ADI_EINVAL;
  h->batch_mode = mode;
  h->drop_graphs();
  return ADI_OK;
}

extern "C" int adi_wave_set_model(adi_wave* h, const adi_wave_model* model) {
  if (!h || !model) return ADI_EINVAL;
  return h->set_model(*model);
}

extern "C" int adi_wave_set_wait_hook(adi_wave* h, int64_t spin_limit, int32_t never_ready_shot) {
  if (!h || spin_limit < 0 || never_ready_shot < -1 || never_ready_shot >= (int)h->g.size())
    return ADI_EINVAL;
  h->spin_limit = spin_limit > 0 ? spin_limit : (1ll << 22);
  h->never_ready = never_ready_shot;
  h->drop_graphs();
  return ADI_OK;
}
