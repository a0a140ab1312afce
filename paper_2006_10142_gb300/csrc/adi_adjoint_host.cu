// adi_adjoint_host.cu -- adi_wave_adjoint: reverse sweep over the recorded
// run with checkpointing.
//
// The run kept (u^{k-1}, u^k) at every `every`-th step.  The reverse sweep
// visits the segments last to first; for each it restores the segment's
// checkpoint, recomputes the segment forward while storing the x-sweep result
// w and the y-sweep result z of every step, then runs the reverse steps of
// the segment backward (adi_adjoint.cu, and y_pipe_kernel's adjoint mode in
// adi_forward.cu for the column solves).  dJ/dm is summed in FP64 over all
// reverse steps (a pitched [ny][ld] FP64 field) and copied to the caller's
// array at the end.  Memory: 2 fields per checkpoint + 2 fields per step of
// one segment + 7 FP32 work fields + the FP64 sum.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "adi_adjoint.h"
#include "adi_internal.h"
#include "adi_run.h"

using namespace adi;

#define CKA(call, what)                                          \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail(this, e_, what);     \
  } while (0)

void adi_wave::free_adj_work() {
  cudaFree(aw.wseg);
  cudaFree(aw.zseg);
  cudaFree(aw.wb);
  cudaFree(aw.rb);
  cudaFree(aw.g64);
  for (int q = 0; q < 3; ++q) cudaFree(aw.L[q]);
  cudaFree(aw.A);
  cudaFree(aw.B);
  cudaFree(aw.gd);
  cudaFree(aw.rec);
  aw = AdjWork{};
}

int adi_wave::ensure_adj_work(Grid& G, int E, int n_rec) {
  const size_t fbytes = sizeof(float) * (size_t)G.ld * G.ny;
  if (aw.fbytes != fbytes || aw.E < E) {
    free_adj_work();
    cudaError_t e = cudaMalloc(&aw.wseg, fbytes * E);
    if (e == cudaSuccess) e = cudaMalloc(&aw.zseg, fbytes * E);
    if (e == cudaSuccess) e = cudaMalloc(&aw.wb, fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&aw.rb, fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&aw.g64, 2 * fbytes);
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaMalloc(&aw.L[q], fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&aw.A, fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&aw.B, fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&aw.gd, sizeof(GridDev));
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_adj_work();
      return fail(this, ADI_ENOMEM, "allocate adjoint workspace");
    }
    aw.fbytes = fbytes;
    aw.E = E;
  }
  // receivers [n_rec][2], then row offsets [ny + 1], columns [n_rec], indexes [n_rec]
  const int rec_ints = 4 * n_rec + G.ny + 1;
  if (rec_ints > aw.rec_cap) {
    cudaFree(aw.rec);
    aw.rec = nullptr;
    aw.rec_cap = 0;
    cudaError_t e = cudaMalloc(&aw.rec, sizeof(int) * (size_t)rec_ints);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(this, ADI_ENOMEM, "allocate adjoint receivers");
    }
    aw.rec_cap = rec_ints;
  }
  return ADI_OK;
}

int adi_wave::adjoint(const float* resid, double* grad_m, float* grad_wavelet, int every,
                      cudaStream_t st) {
  if (g.size() != 1) return fail(this, ADI_EUNSUPPORTED, "adjoint of a batched handle");
  if (model.active) return fail(this, ADI_EUNSUPPORTED, "adjoint of a non-default model");
  if (!rr.valid) return fail(this, ADI_ESTATE, "no recorded run to differentiate");
  if (rr.every <= 0)
    return fail(this, ADI_ESTATE,
                "the run kept no checkpoints: call adi_wave_set_checkpointing before adi_wave_run");
  if (every != 0 && every != rr.every)
    return fail(this, ADI_EINVAL, "ckpt_every must be 0 or the run's checkpoint interval");
  const int n_rec = (int)(rr.rec.size() / 2);
  if (!grad_m || (n_rec > 0 && !resid)) return fail(this, ADI_EINVAL, "null gradient or residual");
  Grid& G = g[0];
  const int S = rr.steps, E = rr.every;
  int rc = ensure_adj_work(G, E, n_rec);
  if (rc != ADI_OK) return rc;
  const size_t fbytes = aw.fbytes;
  const size_t ffl = (size_t)G.ld * G.ny;  // floats per field

  const bool src_on = rr.src.ix >= 0 && rr.src.wavelet != nullptr && rr.src.n_wavelet > 0;
  if (grad_wavelet && rr.src.n_wavelet > 0)
    CKA(cudaMemsetAsync(grad_wavelet, 0, sizeof(float) * (size_t)rr.src.n_wavelet, st),
        "clear grad_wavelet");
  for (int q = 0; q < 3; ++q) CKA(cudaMemsetAsync(aw.L[q], 0, fbytes, st), "clear lambda");
  CKA(cudaMemsetAsync(aw.g64, 0, 2 * fbytes, st), "clear gradient sum");
  // Receivers grouped by row: the residual of step s - 1 is added to lam at
  // the end of reverse step s (lam_update_kernel), that of the last step by
  // one seed launch before the first.
  int* d_rrow = aw.rec + 2 * n_rec;
  int* d_rix = d_rrow + G.ny + 1;
  int* d_rid = d_rix + n_rec;
  if (n_rec > 0) {
    std::vector<int>& t = aw.rtab;
    t.assign((size_t)G.ny + 1 + 2 * (size_t)n_rec, 0);
    for (int r = 0; r < n_rec; ++r) t[(size_t)rr.rec[2 * r + 1] + 1] += 1;
    for (int j = 0; j < G.ny; ++j) t[(size_t)j + 1] += t[(size_t)j];
    std::vector<int> fill(t.begin(), t.begin() + G.ny);
    for (int r = 0; r < n_rec; ++r) {  // stable: receivers of a row keep their order
      const int q = fill[rr.rec[2 * r + 1]]++;
      t[(size_t)G.ny + 1 + q] = rr.rec[2 * r];
      t[(size_t)G.ny + 1 + n_rec + q] = r;
    }
    CKA(cudaMemcpyAsync(aw.rec, rr.rec.data(), sizeof(int) * 2 * (size_t)n_rec,
                        cudaMemcpyHostToDevice, st), "copy receivers");
    CKA(cudaMemcpyAsync(d_rrow, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice, st),
        "copy receiver table");
    if (S > 0) {  // a recorded run has at least one step; the seed reads step S - 1
      CKA(launch_seed(aw.L[0], G.ld, aw.rec, n_rec, resid + (size_t)(S - 1) * n_rec, st), "seed");
      launches += 1;
    }
  }

  GridDev hg = {};
  hg.src_ix = src_on ? rr.src.ix : -1;
  hg.src_iy = src_on ? rr.src.iy : -1;
  hg.wavelet = src_on ? rr.src.wavelet : nullptr;
  hg.n_wavelet = src_on ? rr.src.n_wavelet : 0;

  const GridPlan& P = G.plan;
  // the column solves of the reverse step take the forward TMA pipeline
  // when the forward y sweep does (strip maps of m and the three lam fields)
  const bool ypipe = (P.y_stage == 3 || P.y_stage == 4) && !P.fp64y;
  CUtensorMap tl_m, tl_L[3];
  if (ypipe) {
    const int BH = y_pipe_box_rows(1 << P.log2tcol, P.ky);
    const int BW = 1 << P.log2W;
    CKA(encode_strip_map(&tl_m, G.m, G.ld, G.ny, BW, BH), "strip map m");
    for (int q = 0; q < 3; ++q) CKA(encode_strip_map(&tl_L[q], aw.L[q], G.ld, G.ny, BW, BH), "strip map lambda");
  }
  // the row solves of the reverse step stage their rows through shared
  // memory unless the forward x sweep is set to direct loads
  const bool x_adj_staged = P.x_stage != 2;
  float* L0 = aw.L[0];
  float* L1 = aw.L[1];
  float* L2 = aw.L[2];
  const int nck = (S + E - 1) / E;
  for (int c = nck - 1; c >= 0; --c) {
    const int s0 = c * E;
    const int len = std::min(E, S - s0);
    // restore the checkpoint and recompute the segment forward
    CKA(cudaMemcpyAsync(aw.A, rr.ckpt[c], fbytes, cudaMemcpyDeviceToDevice, st), "restore");
    CKA(cudaMemcpyAsync(aw.B, rr.ckpt[c] + ffl, fbytes, cudaMemcpyDeviceToDevice, st), "restore");
    hg.k = rr.k0 + s0;
    hg.k0 = hg.k;
    CKA(cudaMemcpyAsync(aw.gd, &hg, sizeof(GridDev), cudaMemcpyHostToDevice, st), "adjoint state");
    float* cur = aw.B;
    float* prev = aw.A;
    for (int i = 0; i < len; ++i) {
      rc = launch_fwd(G, cur, prev, aw.wseg + ffl * i, aw.zseg + ffl * i, aw.gd, st);
      if (rc != ADI_OK) return rc;
      std::swap(cur, prev);
    }
    // reverse steps of the segment
    for (int i = len - 1; i >= 0; --i) {
      const int s = s0 + i;
      const long long k = rr.k0 + s;
      if (ypipe) {
        YArgs ya = {};
        ya.nx = G.nx; ya.ny = G.ny; ya.ld = G.ld;
        ya.log2W = P.log2W; ya.log2tcol = P.log2tcol; ya.C = P.C; ya.pcr = P.pcr;
        ya.m = G.m; ya.z_out = aw.wb;
        ya.sc = G.dt * G.dt / (2.0 * G.hy * G.hy);
        ya.err = d_err;
        ya.stage_mode = 3;
        ya.persist = 1;
        const int q = L0 == aw.L[0] ? 0 : L0 == aw.L[1] ? 1 : 2;
        if (P.y_stage == 4) CKA(launch_y_coop_adj(ya, P.ky, G.yc, tl_L[q], tl_m, st), "adjoint y sweep");
        else CKA(launch_y_pipe_adj(ya, P.ky, tl_L[q], tl_m, st), "adjoint y sweep");
      } else {
        YAdjArgs ya;
        ya.nx = G.nx; ya.ny = G.ny; ya.ld = G.ld;
        ya.log2W = P.log2W; ya.log2tcol = P.log2tcol; ya.C = P.C; ya.pcr = P.pcr;
        ya.m = G.m; ya.lam = L0; ya.wbar = aw.wb;
        ya.sc = G.dt * G.dt / (2.0 * G.hy * G.hy);
        CKA(launch_y_adj(ya, P.ky, P.fp64y, st), "adjoint y sweep");
      }
      XAdjArgs xa;
      xa.nx = G.nx; xa.ny = G.ny; xa.ld = G.ld;
      xa.log2tsys = P.log2tsys; xa.spc = P.spc; xa.pcr = P.pcr;
      xa.m = G.m; xa.wbar = aw.wb; xa.w = aw.wseg + ffl * i; xa.z = aw.zseg + ffl * i;
      xa.rbar = aw.rb; xa.g64 = aw.g64; xa.gw = grad_wavelet; xa.level = k;
      xa.sc = G.dt * G.dt / (2.0 * G.hx * G.hx);
      xa.src_scale = G.dt * G.dt / (G.hx * G.hy);
      xa.src_ix = hg.src_ix; xa.src_iy = hg.src_iy;
      xa.wavelet = hg.wavelet; xa.n_wavelet = hg.n_wavelet;
      xa.staged = x_adj_staged ? 1 : 0; xa.stage_off = -1;
      CKA(launch_x_adj(xa, P.kx, P.fp64x, st), "adjoint x sweep");
      LamArgs la;
      la.nx = G.nx; la.ny = G.ny; la.ld = G.ld;
      la.m = G.m; la.rbar = aw.rb; la.L0 = L0; la.L1 = L1; la.L2 = L2;
      la.cx = (float)(G.dt * G.dt / (G.hx * G.hx));
      la.cy = (float)(G.dt * G.dt / (G.hy * G.hy));
      la.resid = (n_rec > 0 && s > 0) ? resid + (size_t)(s - 1) * n_rec : nullptr;
      la.rrow = d_rrow;
      la.rix = d_rix;
      la.rid = d_rid;
      CKA(launch_lam_update(la, st), "adjoint lambda update");
      launches += 3;
      float* t = L0;
      L0 = L1;
      L1 = L2;
      L2 = t;
    }
  }
  // the FP64 sum (pitched rows) into the caller's [ny][nx] array
  CKA(cudaMemcpy2DAsync(grad_m, sizeof(double) * (size_t)G.nx, aw.g64, sizeof(double) * (size_t)G.ld,
                        sizeof(double) * (size_t)G.nx, G.ny, cudaMemcpyDeviceToDevice, st),
      "copy gradient");
  // L0 = dJ/du^{k0}; the second-order start makes u^1 depend on m and f^0
  if (rr.taylor) {
    TaylorArgs ta;
    ta.nx = G.nx; ta.ny = G.ny; ta.ld = G.ld;
    ta.phi = rr.ckpt[0];  // u^0
    ta.lam = L0;
    ta.gm = grad_m;
    ta.gw = grad_wavelet;
    ta.level = 0;
    ta.cx_half = G.dt * G.dt / (2.0 * G.hx * G.hx);
    ta.cy_half = G.dt * G.dt / (2.0 * G.hy * G.hy);
    ta.src_half = G.dt * G.dt / (2.0 * G.hx * G.hy);
    ta.src_ix = hg.src_ix;
    ta.src_iy = hg.src_iy;
    CKA(launch_taylor_adj(ta, st), "start-up adjoint");
    launches += 1;
  }
  return ADI_OK;
}
