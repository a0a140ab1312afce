// adi_run.cu -- handle implementation: creation, the time loop (Algorithm 1)
// with CUDA-graph replay of step pairs, checkpoints, state access, status,
// tuning and measurement hooks.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "adi_adjoint.h"
#include "adi_internal.h"
#include "adi_run.h"

using namespace adi;

namespace {

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Kernel attributes (dynamic shared memory, cluster sizes) are per device:
// one flag per device, set under a lock.
constexpr int kMaxDevices = 64;
bool g_configured[kMaxDevices] = {};
std::mutex g_config_mu;

#define CK(call, what)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail(this, e_, what);    \
  } while (0)

}  // namespace

cudaError_t adi::configure_current_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_config_mu);
  if (g_configured[dev]) return cudaSuccess;
  e = configure_kernels();
  if (e == cudaSuccess) e = configure_adjoint_kernels();
  if (e == cudaSuccess) e = configure_y_coop_kernels();
  if (e == cudaSuccess) e = configure_model_kernels();
  if (e == cudaSuccess) g_configured[dev] = true;
  return e;
}

// Scratch of the y sweep without clusters (y_stage 4): segment summaries for
// up to 32 segments per column and two counters per strip, zeroed once.
int adi_wave::ensure_ycoop(Grid& G) {
  if (G.plan.y_stage != ADI_STAGE_COOP) return ADI_OK;
  const int cols = (G.nx + 31) / 32 * 32;
  const int strips = (G.nx + 15) / 16;
  G.yc.C = G.plan.C;
  if (G.yc.tops != nullptr && G.yc.cols >= cols && G.yc.strips >= strips) return ADI_OK;
  cudaFree(G.yc.tops);
  cudaFree(G.yc.sync);
  G.yc.tops = nullptr;
  G.yc.sync = nullptr;
  G.yc.cols = 0;
  G.yc.strips = 0;
  cudaError_t e = cudaMalloc(&G.yc.tops, sizeof(float) * 8 * 32 * (size_t)cols);
  if (e == cudaSuccess) e = cudaMalloc(&G.yc.sync, sizeof(int) * 2 * (size_t)strips);
  if (e == cudaSuccess) e = cudaMemset(G.yc.sync, 0, sizeof(int) * 2 * (size_t)strips);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(G.yc.tops);
    cudaFree(G.yc.sync);
    G.yc.tops = nullptr;
    G.yc.sync = nullptr;
    return fail(this, e == cudaErrorMemoryAllocation ? ADI_ENOMEM : ADI_ECUDA,
                std::string("y sweep scratch: ") + cudaGetErrorString(e));
  }
  G.yc.cols = cols;
  G.yc.strips = strips;
  return ADI_OK;
}

// The grid record goes to the device as a kernel argument: no copy engine
// and no host buffer that must outlive the call.
int adi_wave::upload_gd(Grid& G, cudaStream_t st) {
  CK(launch_put_gd(G.gd, G.hgd, st), "upload grid state");
  launches += 1;
  return ADI_OK;
}

int adi_wave::create(const adi_wave_desc* desc, int n, const float* const* m,
                     const float* const* phi, const float* const* psi, const adi_source* src,
                     cudaStream_t st) {
  CK(configure_current_device(), "configure kernels");
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create capture stream");
  CK(cudaMalloc(&d_err, sizeof(int)), "alloc error word");
  CK(cudaMemsetAsync(d_err, 0, sizeof(int), st), "clear error word");
  g.resize(n);
  for (int s = 0; s < n; ++s) {
    Grid& G = g[s];
    const adi_wave_desc& d = desc[s];
    G.nx = d.nx;
    G.ny = d.ny;
    G.ld = round_up(d.nx, 32);
    G.lx = d.lx;
    G.ly = d.ly;
    G.dt = d.dt;
    G.hx = d.lx / (d.nx + 1);
    G.hy = d.ly / (d.ny + 1);
    G.start = d.start;
    G.fp64mode = d.fp64_solve;
    const size_t bytes = sizeof(float) * (size_t)G.ld * G.ny;
    cudaError_t e = cudaMalloc(&G.m, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&G.buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&G.buf[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&G.w, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&G.gd, sizeof(GridDev));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(this, e == cudaErrorMemoryAllocation ? ADI_ENOMEM : ADI_ECUDA,
                  std::string("allocate grid: ") + cudaGetErrorString(e));
    }
    CK(cudaMemsetAsync(G.m, 0, bytes, st), "clear m");
    CK(cudaMemsetAsync(G.buf[0], 0, bytes, st), "clear u0");
    CK(cudaMemsetAsync(G.buf[1], 0, bytes, st), "clear u1");
    CK(cudaMemsetAsync(G.w, 0, bytes, st), "clear w");
    int rc = start_grid(s, m[s], phi[s], psi ? psi[s] : nullptr, src ? &src[s] : nullptr, st);
    if (rc != ADI_OK) return rc;
  }
  if (n > 1) return setup_batch(st);
  return ADI_OK;
}

// Batched run: every shot advances `steps` steps; one persistent launch per
// step (or the plain kernels per shot in batch mode 1), step pairs replayed
// from a captured graph.
int adi_wave::run_batch(int steps, const adi_source* src, cudaStream_t st) {
  for (size_t s = 0; s < g.size(); ++s) {
    Grid& G = g[s];
    const adi_source none = {-1, -1, nullptr, 0};
    const adi_source sr = src ? src[s] : none;
    const bool on = sr.ix >= 0 && sr.wavelet != nullptr;
    G.hgd.k = G.k;
    G.hgd.k0 = G.k;
    G.hgd.steps = steps;
    G.hgd.wavelet = on ? sr.wavelet : nullptr;
    G.hgd.n_wavelet = on ? sr.n_wavelet : 0;
    G.hgd.src_ix = on ? sr.ix : -1;
    G.hgd.src_iy = on ? sr.iy : -1;
    G.hgd.n_rec = 0;
    G.hgd.rec = nullptr;
    G.hgd.traces = nullptr;
    if (upload_gd(G, st) != ADI_OK) return ADI_ECUDA;
  }
  rr.valid = false;
  const bool use_graph = g[0].plan.graph && !profile;
  int t = 0;
  if (use_graph) {
    while (steps - t >= 2) {
      cudaGraphExec_t& ex = pair[g[0].cur][0];
      if (!ex) {
        std::vector<int> cur0;
        std::vector<long long> k0;
        for (Grid& G : g) { cur0.push_back(G.cur); k0.push_back(G.k); }
        const int64_t l0 = launches;
        CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        int rc = ADI_OK;
        if (batch_mode == 2) {
          rc = enqueue_batch_steps_parallel(2, cap);  // per-shot chains of two steps
        } else {
          rc = enqueue_batch_step(cap);
          if (rc == ADI_OK) rc = enqueue_batch_step(cap);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        for (size_t s = 0; s < g.size(); ++s) { g[s].cur = cur0[s]; g[s].k = k0[s]; }
        const int64_t per_pair = launches - l0;
        launches = l0;
        if (rc != ADI_OK) {
          if (graph) cudaGraphDestroy(graph);
          return rc;
        }
        if (e != cudaSuccess) return cuda_fail(this, e, "end capture");
        e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          ex = nullptr;
          return cuda_fail(this, e, "graph instantiate");
        }
        pair_launches = per_pair;
      }
      CK(cudaGraphLaunch(ex, st), "graph launch");
      launches += pair_launches;
      for (Grid& G : g) { G.k += 2; G.from_init = false; }
      t += 2;
    }
  }
  while (t < steps) {
    int rc = enqueue_batch_step(st);
    if (rc != ADI_OK) return rc;
    t += 1;
  }
  return ADI_OK;
}

// Copy m (optional), re-plan, and run the start-up of Eq. (CN2) for shot s.
int adi_wave::start_grid(int s, const float* m, const float* phi, const float* psi,
                         const adi_source* sr, cudaStream_t st) {
  Grid& G = g[s];
  if (m) {
    // the caller's medium is scanned before it replaces the handle's, so a
    // rejected one leaves the handle as it was
    if (!scan) CK(cudaMalloc(&scan, 3 * sizeof(unsigned int)), "alloc scan");
    if (!scan_host) {
      unsigned int* hp = nullptr;
      CK(cudaHostAlloc((void**)&hp, 4 * sizeof(unsigned int), cudaHostAllocMapped), "alloc scan result");
      scan_host = hp;
      CK(cudaHostGetDevicePointer((void**)&scan_host_dev, hp, 0), "map scan result");
    }
    CK(launch_scan_m(m, G.nx, G.ny, G.nx, scan, scan_host_dev, st), "scan m");
    CK(cudaStreamSynchronize(st), "scan sync");
    unsigned int res3[3] = {scan_host[0], scan_host[1], scan_host[2]};
    launches += 3;
    if (res3[2]) return fail(this, ADI_EINVAL, "m must be finite and > 0 everywhere");
    CK(cudaMemcpy2DAsync(G.m, sizeof(float) * G.ld, m, sizeof(float) * G.nx,
                         sizeof(float) * G.nx, G.ny, cudaMemcpyDeviceToDevice, st), "copy m");
    float lo, hi;
    memcpy(&lo, &res3[0], 4);
    memcpy(&hi, &res3[1], 4);
    G.mmin = lo;
    G.mmax = hi;
    std::string why;
    GridPlan old = G.plan;
    int rc = plan_grid(G, tuning, why);
    if (rc != ADI_OK) {
      G.plan = old;
      return fail(this, rc, why);
    }
    // the captured steps stay valid while the plan (launch shapes, kernels) is the same
    if (!(G.plan == old)) drop_graphs();
    rc = ensure_ycoop(G);
    if (rc != ADI_OK) return rc;
  }
  G.hgd = GridDev{};
  G.hgd.k = 1;
  G.hgd.k0 = 1;
  G.hgd.src_ix = -1;
  G.hgd.src_iy = -1;
  if (upload_gd(G, st) != ADI_OK) return ADI_ECUDA;
  const bool has_src = sr && sr->ix >= 0 && sr->wavelet && sr->n_wavelet > 0;
  CK(launch_init(G.nx, G.ny, G.ld, G.m, phi, psi, G.buf[0], G.buf[1], G.dt,
                 G.dt * G.dt / (2.0 * G.hx * G.hx), G.dt * G.dt / (2.0 * G.hy * G.hy),
                 G.start == ADI_START_TAYLOR2 ? 1 : 0, has_src ? sr->ix : -1,
                 has_src ? sr->iy : -1, G.dt * G.dt / (2.0 * G.hx * G.hy),
                 has_src ? sr->wavelet : nullptr, has_src ? sr->n_wavelet : 0, st),
     "init kernel");
  launches += 1;
  G.cur = 1;
  G.k = 1;
  G.from_init = true;
  rr.valid = false;
  return ADI_OK;
}

int adi_wave::reset(const float* const* m, const float* const* phi, const float* const* psi,
                    const adi_source* src, cudaStream_t st) {
  for (size_t s = 0; s < g.size(); ++s) {
    if (!phi[s]) return fail(this, ADI_EINVAL, "phi is required");
    if (src && src[s].ix >= 0 &&
        (src[s].ix >= g[s].nx || src[s].iy < 0 || src[s].iy >= g[s].ny))
      return fail(this, ADI_EINVAL, "source node outside the grid");
  }
  for (size_t s = 0; s < g.size(); ++s) {
    int rc = start_grid((int)s, m ? m[s] : nullptr, phi[s], psi ? psi[s] : nullptr,
                        src ? &src[s] : nullptr, st);
    if (rc != ADI_OK) return rc;
  }
  return ADI_OK;
}

int adi_wave::prof_begin(cudaStream_t st, cudaEvent_t* a) {
  if (ev_pool.empty()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e), "event create");
    ev_pool.push_back(e);
  }
  *a = ev_pool.back();
  ev_pool.pop_back();
  CK(cudaEventRecord(*a, st), "event record");
  return ADI_OK;
}

int adi_wave::prof_end(cudaStream_t st, cudaEvent_t a, int kind) {
  if (ev_pool.empty()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e), "event create");
    ev_pool.push_back(e);
  }
  cudaEvent_t b = ev_pool.back();
  ev_pool.pop_back();
  CK(cudaEventRecord(b, st), "event record");
  prof.push_back(ProfRec{a, b, kind});
  return ADI_OK;
}

int adi_wave::enqueue_step(Grid& G, cudaStream_t st, bool gather) {
  float* u_cur = G.buf[G.cur];
  float* u_prev = G.buf[1 - G.cur];
  int rc = launch_fwd(G, u_cur, u_prev, G.w, nullptr, G.gd, st);
  if (rc != ADI_OK) return rc;
  if (gather) {
    CK(launch_gather(G.gd, u_prev, G.ld, G.hgd.n_rec, st), "gather launch");
    launches += 1;
  }
  G.cur = 1 - G.cur;
  G.k += 1;
  G.from_init = false;
  return ADI_OK;
}

// One forward step on explicit buffers: x sweep into w, y sweep + update
// writing u^{k+1} over u_prev (and z into z_out when given).
int adi_wave::launch_fwd(Grid& G, const float* u_cur, float* u_prev, float* w, float* z_out,
                         GridDev* gd, cudaStream_t st) {
  const GridPlan& P = G.plan;
  XArgs xa;
  xa.nx = G.nx;
  xa.ny = G.ny;
  xa.ld = G.ld;
  xa.log2tsys = P.log2tsys;
  xa.spc = P.spc;
  xa.pcr = P.pcr;
  xa.m = G.m;
  xa.u = u_cur;
  xa.w = w;
  xa.cx = G.dt * G.dt / (G.hx * G.hx);
  xa.cy = G.dt * G.dt / (G.hy * G.hy);
  xa.sc = G.dt * G.dt / (2.0 * G.hx * G.hx);
  xa.src_scale = G.dt * G.dt / (G.hx * G.hy);
  xa.gd = gd;
  xa.persist = P.persist;
  xa.stage_mode = P.x_stage;
  xa.stage_off = -1;
  xa.err = d_err;
  xa.xc = P.xc;
  YArgs ya;
  ya.nx = G.nx;
  ya.ny = G.ny;
  ya.ld = G.ld;
  ya.log2W = P.log2W;
  ya.log2tcol = P.log2tcol;
  ya.C = P.C;
  ya.pcr = P.pcr;
  ya.m = G.m;
  ya.w = w;
  ya.u_cur = u_cur;
  ya.u_prev = u_prev;
  ya.z_out = z_out;
  ya.stage_mode = P.y_stage;
  ya.persist = P.persist;
  ya.stage_off = 0;
  ya.sc = G.dt * G.dt / (2.0 * G.hy * G.hy);
  ya.gd = gd;
  ya.err = d_err;

  cudaEvent_t a = nullptr;
  if (profile && prof_begin(st, &a) != ADI_OK) return ADI_ECUDA;
  if (P.x_stage == 3 || P.x_stage == 5) {
    const int L = x_pipe_box_lines((1 << P.log2tsys) / P.xc, P.kx);
    if (G.tm_lines != L) {
      CK(encode_row_map(&G.tm_buf[0], G.buf[0], G.ld, G.ny, L), "tensor map u0");
      CK(encode_row_map(&G.tm_buf[1], G.buf[1], G.ld, G.ny, L), "tensor map u1");
      CK(encode_row_map(&G.tm_m, G.m, G.ld, G.ny, L), "tensor map m");
      CK(encode_row_map(&G.tm_w, G.w, G.ld, G.ny, L), "tensor map w");
      G.tm_lines = L;
    }
    CUtensorMap tmp, tmpw;
    const CUtensorMap* tu = u_cur == G.buf[0] ? &G.tm_buf[0] : u_cur == G.buf[1] ? &G.tm_buf[1] : nullptr;
    if (tu == nullptr) {
      CK(encode_row_map(&tmp, u_cur, G.ld, G.ny, L), "tensor map u");
      tu = &tmp;
    }
    const CUtensorMap* tw = &G.tm_w;
    if (w != G.w) {
      CK(encode_row_map(&tmpw, w, G.ld, G.ny, L), "tensor map w");
      tw = &tmpw;
    }
    if (P.x_stage == 5) CK(launch_x_band(xa, P.kx, *tu, G.tm_m, *tw, st), "x sweep launch");
    else CK(launch_x_pipe(xa, P.kx, *tu, G.tm_m, *tw, st), "x sweep launch");
  } else {
    CK(launch_x(xa, P.kx, P.fp64x, P.tree, st), "x sweep launch");
  }
  if (profile && prof_end(st, a, ADI_KERNEL_X) != ADI_OK) return ADI_ECUDA;
  if (profile && prof_begin(st, &a) != ADI_OK) return ADI_ECUDA;
  if (P.y_stage == 3 || P.y_stage == 4) {
    const int BH = y_pipe_box_rows(1 << P.log2tcol, P.ky);
    const int BW = 1 << P.log2W;
    if (G.ts_rows != BH * 64 + BW) {
      CK(encode_strip_map(&G.ts_buf[0], G.buf[0], G.ld, G.ny, BW, BH), "strip map u0");
      CK(encode_strip_map(&G.ts_buf[1], G.buf[1], G.ld, G.ny, BW, BH), "strip map u1");
      CK(encode_strip_map(&G.ts_m, G.m, G.ld, G.ny, BW, BH), "strip map m");
      CK(encode_strip_map(&G.ts_w, G.w, G.ld, G.ny, BW, BH), "strip map w");
      G.ts_rows = BH * 64 + BW;
    }
    YMaps mp;
    mp.m = G.ts_m;
    const float* want[3] = {w, u_cur, u_prev};
    CUtensorMap* outm[3] = {&mp.w, &mp.uc, &mp.up};
    for (int f = 0; f < 3; ++f) {
      const float* p = want[f];
      if (p == G.w) *outm[f] = G.ts_w;
      else if (p == G.buf[0]) *outm[f] = G.ts_buf[0];
      else if (p == G.buf[1]) *outm[f] = G.ts_buf[1];
      else CK(encode_strip_map(outm[f], p, G.ld, G.ny, BW, BH), "strip map");
    }
    if (P.y_stage == 4) CK(launch_y_coop(ya, P.ky, G.yc, mp, st), "y sweep launch");
    else CK(launch_y_pipe(ya, P.ky, mp, st), "y sweep launch");
  } else {
    CK(launch_y(ya, P.ky, P.fp64y, P.tree, st), "y sweep launch");
  }
  if (profile && prof_end(st, a, ADI_KERNEL_Y) != ADI_OK) return ADI_ECUDA;
  launches += 2;
  return ADI_OK;
}

void adi_wave::drop_graphs() {
  for (int o = 0; o < 2; ++o)
    for (int q = 0; q < 2; ++q)
      if (pair[o][q]) {
        cudaGraphExecDestroy(pair[o][q]);
        pair[o][q] = nullptr;
      }
}

int adi_wave::launch_pair_graph(Grid& G, cudaStream_t st, bool gather) {
  cudaGraphExec_t& ex = pair[G.cur][gather ? 1 : 0];
  if (!ex) {
    const int cur0 = G.cur;
    const long long k0 = G.k;
    const int64_t l0 = launches;
    CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = enqueue_step(G, cap, gather);
    if (rc == ADI_OK) rc = enqueue_step(G, cap, gather);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    G.cur = cur0;
    G.k = k0;
    launches = l0;
    if (rc != ADI_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(this, e, "end capture");
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ex = nullptr;
      return cuda_fail(this, e, "graph instantiate");
    }
  }
  CK(cudaGraphLaunch(ex, st), "graph launch");
  launches += gather ? 6 : 4;
  G.k += 2;
  return ADI_OK;
}

int adi_wave::run(int steps, const adi_source* src, const int32_t* rec_xy, int n_rec,
                  float* traces, cudaStream_t st, bool record) {
  if (steps < 0 || n_rec < 0) return fail(this, ADI_EINVAL, "negative steps or receiver count");
  if (n_rec > 0 && (g.size() != 1 || !rec_xy || !traces))
    return fail(this, ADI_EINVAL, "receivers need one grid, rec_xy and traces");
  for (size_t s = 0; s < g.size(); ++s) {
    if (src && src[s].ix >= 0 &&
        (src[s].ix >= g[s].nx || src[s].iy < 0 || src[s].iy >= g[s].ny))
      return fail(this, ADI_EINVAL, "source node outside the grid");
  }
  if (g.size() != 1) return run_batch(steps, src, st);
  Grid& G = g[0];
  for (int r = 0; r < n_rec; ++r) {
    if (rec_xy[2 * r] < 0 || rec_xy[2 * r] >= G.nx || rec_xy[2 * r + 1] < 0 ||
        rec_xy[2 * r + 1] >= G.ny)
      return fail(this, ADI_EINVAL, "receiver node outside the grid");
  }
  if (steps == 0) return ADI_OK;

  // per-run device state: level, source, receivers
  if (n_rec > rec_cap) {
    if (d_rec) cudaFree(d_rec);
    d_rec = nullptr;
    rec_cap = 0;
    CK(cudaMalloc(&d_rec, sizeof(int) * 2 * (size_t)n_rec), "alloc receivers");
    rec_cap = n_rec;
  }
  if (n_rec > 0)
    CK(cudaMemcpyAsync(d_rec, rec_xy, sizeof(int) * 2 * (size_t)n_rec, cudaMemcpyHostToDevice, st),
       "copy receivers");
  const adi_source none = {-1, -1, nullptr, 0};
  const adi_source sr = src ? src[0] : none;
  G.hgd.k = G.k;
  G.hgd.k0 = G.k;
  G.hgd.steps = steps;
  G.hgd.wavelet = (sr.ix >= 0) ? sr.wavelet : nullptr;
  G.hgd.n_wavelet = (sr.ix >= 0 && sr.wavelet) ? sr.n_wavelet : 0;
  G.hgd.src_ix = (sr.ix >= 0 && sr.wavelet) ? sr.ix : -1;
  G.hgd.src_iy = (sr.ix >= 0 && sr.wavelet) ? sr.iy : -1;
  G.hgd.n_rec = n_rec;
  G.hgd.rec = d_rec;
  G.hgd.traces = traces;
  if (upload_gd(G, st) != ADI_OK) return ADI_ECUDA;

  const int every = record ? ckpt_every : 0;
  if (record) {
    rr.valid = true;
    rr.k0 = G.k;
    rr.steps = steps;
    rr.every = every;
    rr.taylor = G.start == ADI_START_TAYLOR2 && G.from_init && G.k == 1;
    rr.src = sr;
    rr.rec.assign(rec_xy ? rec_xy : (const int32_t*)nullptr,
                  rec_xy ? rec_xy + 2 * (size_t)n_rec : (const int32_t*)nullptr);
    const size_t need = every > 0 ? (size_t)((steps + every - 1) / every) : 0;
    const size_t fbytes = sizeof(float) * (size_t)G.ld * G.ny;
    if (rr.ckpt_bytes != fbytes) {
      for (float* p : rr.ckpt) cudaFree(p);
      rr.ckpt.clear();
      rr.ckpt_bytes = fbytes;
    }
    while (rr.ckpt.size() < need) {
      float* p = nullptr;
      cudaError_t e = cudaMalloc(&p, 2 * fbytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        rr.valid = false;
        return fail(this, ADI_ENOMEM, "allocate checkpoints");
      }
      rr.ckpt.push_back(p);
    }
  }

  const bool gather = n_rec > 0;
  const bool use_graph = G.plan.graph && !profile;
  const size_t fbytes = sizeof(float) * (size_t)G.ld * G.ny;
  int s = 0;
  while (s < steps) {
    int seg = steps - s;
    if (every > 0) {
      if (s % every == 0) {
        float* c = rr.ckpt[s / every];
        CK(cudaMemcpyAsync(c, G.buf[1 - G.cur], fbytes, cudaMemcpyDeviceToDevice, st), "checkpoint");
        CK(cudaMemcpyAsync(c + (size_t)G.ld * G.ny, G.buf[G.cur], fbytes, cudaMemcpyDeviceToDevice,
                           st), "checkpoint");
      }
      seg = std::min(seg, every - s % every);
    }
    int t = 0;
    if (model.active) {
      while (t < seg) {
        int rc = enqueue_model_step(G, st, gather);
        if (rc != ADI_OK) return rc;
        t += 1;
      }
    }
    if (use_graph) {
      while (seg - t >= 2) {
        int rc = launch_pair_graph(G, st, gather);
        if (rc != ADI_OK) return rc;
        t += 2;
      }
    }
    while (t < seg) {
      int rc = enqueue_step(G, st, gather);
      if (rc != ADI_OK) return rc;
      t += 1;
    }
    s += seg;
  }
  G.hgd.k = G.k;
  return ADI_OK;
}

int adi_wave::set_state(int shot, const float* u_prev, const float* u_cur, int64_t k,
                        cudaStream_t st) {
  Grid& G = g[shot];
  const size_t wb = sizeof(float) * (size_t)G.nx;
  CK(cudaMemcpy2DAsync(G.buf[1 - G.cur], sizeof(float) * G.ld, u_prev, wb, wb, G.ny,
                       cudaMemcpyDeviceToDevice, st), "set_state");
  CK(cudaMemcpy2DAsync(G.buf[G.cur], sizeof(float) * G.ld, u_cur, wb, wb, G.ny,
                       cudaMemcpyDeviceToDevice, st), "set_state");
  G.k = k;
  G.from_init = false;
  G.hgd.k = k;
  G.hgd.k0 = k;
  G.hgd.steps = 0;
  if (upload_gd(G, st) != ADI_OK) return ADI_ECUDA;
  rr.valid = false;
  return ADI_OK;
}

int adi_wave::sync_status(cudaStream_t st) {
  CK(cudaStreamSynchronize(st), "synchronize");
  int word = 0;
  CK(cudaMemcpy(&word, d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  CK(cudaMemset(d_err, 0, sizeof(int)), "clear error word");
  if (word & ERR_TIMEOUT) return fail(this, ADI_ETIMEOUT, "a bounded device wait expired");
  if (word & ERR_NUMERIC) return fail(this, ADI_ENUMERIC, "non-finite value in the wavefield");
  return ADI_OK;
}

int adi_wave::set_tuning(const adi_wave_tuning& t) {
  std::vector<GridPlan> old;
  for (auto& G : g) old.push_back(G.plan);
  for (auto& G : g) {
    std::string why;
    int rc = plan_grid(G, t, why);
    if (rc != ADI_OK) {
      for (size_t s = 0; s < g.size(); ++s) g[s].plan = old[s];
      return fail(this, rc, why);
    }
  }
  for (auto& G : g) {
    int rc = ensure_ycoop(G);
    if (rc != ADI_OK) {
      for (size_t s = 0; s < g.size(); ++s) g[s].plan = old[s];
      return rc;
    }
  }
  tuning = t;
  drop_graphs();
  return ADI_OK;
}

int adi_wave::profile_read(double* ms, int64_t* counts, int n_kinds) {
  std::vector<double> acc(ADI_KERNEL_KINDS, 0.0);
  std::vector<int64_t> cnt(ADI_KERNEL_KINDS, 0);
  for (const ProfRec& r : prof) {
    CK(cudaEventSynchronize(r.b), "event sync");
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b), "event elapsed");
    acc[r.kind] += t;
    cnt[r.kind] += 1;
    ev_pool.push_back(r.a);
    ev_pool.push_back(r.b);
  }
  prof.clear();
  for (int k = 0; k < n_kinds && k < ADI_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = acc[k];
    if (counts) counts[k] = cnt[k];
  }
  return ADI_OK;
}

adi_wave::~adi_wave() {
  cudaDeviceSynchronize();
  drop_graphs();
  for (auto& G : g) {
    cudaFree(G.m);
    cudaFree(G.buf[0]);
    cudaFree(G.buf[1]);
    cudaFree(G.w);
    cudaFree(G.gd);
    cudaFree(G.yc.tops);
    cudaFree(G.yc.sync);
  }
  for (float* p : rr.ckpt) cudaFree(p);
  free_adj_work();
  for (const ProfRec& r : prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  if (d_err) cudaFree(d_err);
  if (scan) cudaFree(scan);
  if (scan_host) cudaFreeHost(const_cast<unsigned int*>(scan_host));
  if (d_rec) cudaFree(d_rec);
  if (d_shots) cudaFree(d_shots);
  if (d_items) cudaFree(d_items);
  if (d_sync) cudaFree(d_sync);
  for (int b = 0; b < kBranches; ++b) {
    if (branch[b]) cudaStreamDestroy(branch[b]);
    if (join_ev[b]) cudaEventDestroy(join_ev[b]);
  }
  if (fork_ev) cudaEventDestroy(fork_ev);
  if (cap) cudaStreamDestroy(cap);
}


// ---------------------------------------------------------------------------
// problem class beyond the default (adi_models.cu)
// ---------------------------------------------------------------------------
int adi_wave::set_model(const adi_wave_model& mdl) {
  if (g.size() != 1) return fail(this, ADI_EUNSUPPORTED, "models need a single-grid handle");
  if (mdl.scheme < ADI_SCHEME_FACTORED || mdl.scheme > ADI_SCHEME_LISTING1)
    return fail(this, ADI_EINVAL, "unknown scheme");
  if (mdl.n_g < 0 || mdl.n_f < 0 || (mdl.g && mdl.n_g < 1) || (mdl.f && mdl.n_f < 1))
    return fail(this, ADI_EINVAL, "bad g or f length");
  if (mdl.scheme != ADI_SCHEME_FACTORED && (mdl.g || mdl.f))
    return fail(this, ADI_EINVAL, "the half-level schemes take no g or f");
  Model M;
  M.scheme = mdl.scheme;
  M.g = mdl.g;
  M.n_g = mdl.g ? mdl.n_g : 0;
  M.f = mdl.f;
  M.n_f = mdl.f ? mdl.n_f : 0;
  M.active = mdl.scheme != ADI_SCHEME_FACTORED || mdl.g != nullptr || mdl.f != nullptr;
  if (M.active) {
    // one-shot launch geometry: direct row loads, column strips over clusters
    Grid tmp = g[0];
    tmp.fp64mode = ADI_FP64_NEVER;
    adi_wave_tuning t = tuning;
    t.x_stage = ADI_STAGE_DIRECT;
    t.y_stage = ADI_STAGE_L2;
    t.solver = ADI_SOLVER_TREE;
    t.x_cluster = 0;
    std::string why;
    int rc = plan_grid(tmp, t, why);
    if (rc != ADI_OK) return fail(this, rc, "model launch geometry: " + why);
    M.plan = tmp.plan;
  }
  model = M;
  rr.valid = false;
  drop_graphs();
  return ADI_OK;
}

// One step of the active model: an x pass into the scratch field and a y pass,
// then the level advances (and the receivers sample the new field).
int adi_wave::enqueue_model_step(Grid& G, cudaStream_t st, bool gather) {
  const GridPlan& P = model.plan;
  float* A = G.buf[1 - G.cur];  // u^{k-1} (mode 0) or u^{k-1/2}
  float* B = G.buf[G.cur];      // u^k
  float* Wf = G.w;
  const int mode = model.scheme;
  ModelXArgs xa = {};
  xa.nx = G.nx; xa.ny = G.ny; xa.ld = G.ld;
  xa.log2tsys = P.log2tsys; xa.spc = P.spc; xa.mode = mode;
  xa.m = G.m; xa.a = A; xa.b = B; xa.out = Wf;
  xa.cx = G.dt * G.dt / (G.hx * G.hx);
  xa.cy = G.dt * G.dt / (G.hy * G.hy);
  xa.sc = G.dt * G.dt / (2.0 * G.hx * G.hx);
  xa.src_scale = G.dt * G.dt / (G.hx * G.hy);
  xa.tau2 = G.dt * G.dt;
  xa.g = model.g; xa.n_g = model.n_g;
  xa.f = model.f; xa.n_f = model.n_f;
  xa.level = G.k;
  xa.gd = G.gd;
  ModelYArgs ya = {};
  ya.nx = G.nx; ya.ny = G.ny; ya.ld = G.ld;
  ya.log2W = P.log2W; ya.log2tcol = P.log2tcol; ya.C = P.C; ya.mode = mode;
  ya.m = G.m; ya.w = Wf; ya.b = B; ya.io = A;
  ya.sc = G.dt * G.dt / (2.0 * G.hy * G.hy);
  ya.src_scale = G.dt * G.dt / (G.hx * G.hy);
  ya.g = model.g; ya.n_g = model.n_g;
  ya.level = G.k;
  ya.gd = G.gd;
  ya.err = d_err;
  CK(launch_x_model(xa, P.kx, st), "model x pass");
  CK(launch_y_model(ya, P.ky, st), "model y pass");
  CK(launch_advance_level(G.gd, st), "advance level");
  launches += 3;
  if (gather) {
    CK(launch_gather(G.gd, A, G.ld, G.hgd.n_rec, st), "gather launch");
    launches += 1;
  }
  if (mode == ADI_SCHEME_FACTORED) {
    G.cur = 1 - G.cur;  // u^{k+1} over u^{k-1}: the usual swap
  } else {
    // half levels: u^{k+1/2} is in the scratch field, u^{k+1} over u^{k-1/2},
    // and u^k's buffer becomes the scratch (Algorithm 1's two swaps)
    G.buf[1 - G.cur] = Wf;
    G.buf[G.cur] = A;
    G.w = B;
    G.tm_lines = 0;  // cached tensor maps name the buffers by role
    G.ts_rows = 0;
  }
  G.k += 1;
  G.from_init = false;
  return ADI_OK;
}
