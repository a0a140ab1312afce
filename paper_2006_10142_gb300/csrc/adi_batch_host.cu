// adi_batch_host.cu -- host side of the batched form: per-shot geometry for
// the persistent kernel (every item is one full CTA of K = 16 unknowns per
// thread, so items of different shots carry the same work), the work list,
// and one step.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "adi_batch.h"
#include "adi_internal.h"
#include "adi_run.h"
#include "adi_sweeps.cuh"

using namespace adi;

#define CKB(call, what)                                          \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail(this, e_, what);     \
  } while (0)

namespace {
int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
}  // namespace

int adi_wave::setup_batch(cudaStream_t st) {
  const int n = (int)g.size();
  batch_fp64 = false;
  for (const Grid& G : g) batch_fp64 |= G.plan.fp64x || G.plan.fp64y;
  const int maxT = batch_fp64 ? 512 : 1024;
  const int K = kBatchK;
  std::vector<BatchShot> shots(n);
  std::vector<int2> xitems, yitems;
  size_t smem = 0;
  for (int s = 0; s < n; ++s) {
    Grid& G = g[s];
    const int tsys = next_pow2((G.nx + K - 1) / K);
    const int tcol = next_pow2((G.ny + K - 1) / K);
    if (tsys > maxT || maxT / tcol < 4)
      return fail(this, ADI_EUNSUPPORTED, "grid too large for the batched form (nx, ny <= " +
                                               std::to_string(maxT * K / 4) + ")");
    const int spc = maxT / tsys;
    const int W = maxT / tcol;
    BatchShot& B = shots[s];
    B.x_items = (G.ny + spc - 1) / spc;
    B.y_items = (G.nx + W - 1) / W;
    const size_t ysm = align64(y_smem_bytes(W, 1, tcol, batch_fp64, true));
    smem = std::max(smem, x_smem_bytes(spc, tsys, batch_fp64, true));
    smem = std::max(smem, ysm + y_stage_bytes(maxT, K));
    for (int c = 0; c < 2; ++c) {
      XArgs& xa = B.xa[c];
      xa.nx = G.nx; xa.ny = G.ny; xa.ld = G.ld;
      xa.log2tsys = ilog2(tsys); xa.spc = spc; xa.pcr = 32;
      xa.m = G.m; xa.u = G.buf[c]; xa.w = G.w;
      xa.cx = G.dt * G.dt / (G.hx * G.hx);
      xa.cy = G.dt * G.dt / (G.hy * G.hy);
      xa.sc = G.dt * G.dt / (2.0 * G.hx * G.hx);
      xa.src_scale = G.dt * G.dt / (G.hx * G.hy);
      xa.gd = G.gd;
      xa.persist = 0;
      xa.stage_mode = 2;
      xa.stage_off = -1;
      xa.err = nullptr;
      xa.xc = 1;
      YArgs& ya = B.ya[c];
      ya.nx = G.nx; ya.ny = G.ny; ya.ld = G.ld;
      ya.log2W = ilog2(W); ya.log2tcol = ilog2(tcol); ya.C = 1; ya.pcr = 32;
      ya.m = G.m; ya.w = G.w; ya.u_cur = G.buf[c]; ya.u_prev = G.buf[1 - c]; ya.z_out = nullptr;
      ya.sc = G.dt * G.dt / (2.0 * G.hy * G.hy);
      ya.gd = G.gd; ya.err = d_err;
      ya.stage_off = (int)ysm;
      ya.stage_mode = 1;
      ya.persist = 0;
    }
    for (int i = 0; i < B.x_items; ++i) xitems.push_back(make_int2(s, i << 1));
    for (int i = 0; i < B.y_items; ++i) yitems.push_back(make_int2(s, (i << 1) | 1));
  }
  if (smem + 512 > (size_t)kMaxDynSmem)  // 512: the kernel's static shared variables
    return fail(this, ADI_EUNSUPPORTED, "batched kernel shared memory");
  std::vector<int2> items = xitems;
  items.insert(items.end(), yitems.begin(), yitems.end());
  n_items = (int)items.size();
  CKB(cudaMalloc(&d_shots, sizeof(BatchShot) * n), "alloc shot table");
  CKB(cudaMalloc(&d_items, sizeof(int2) * items.size()), "alloc work list");
  CKB(cudaMalloc(&d_sync, sizeof(int) * (1 + n)), "alloc counters");
  CKB(cudaMemcpyAsync(d_shots, shots.data(), sizeof(BatchShot) * n, cudaMemcpyHostToDevice, st),
      "upload shot table");
  CKB(cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st),
      "upload work list");
  CKB(cudaStreamSynchronize(st), "batch setup sync");
  int dev = 0, nsm = 0, b32 = 0, b64 = 0;
  CKB(cudaGetDevice(&dev), "get device");
  CKB(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  CKB(configure_batch_kernels(&b32, &b64, smem, smem), "configure batched kernel");
  const int per_sm = batch_fp64 ? b64 : b32;
  if (per_sm < 1) return fail(this, ADI_EUNSUPPORTED, "batched kernel does not fit an SM");
  batch_grid = nsm * per_sm;
  batch_smem = smem;
  return ADI_OK;
}

int adi_wave::enqueue_batch_step(cudaStream_t st) {
  const int n = (int)g.size();
  if (batch_mode == 2) return enqueue_batch_steps_parallel(1, st);
  if (batch_mode == 1) {
    for (Grid& G : g) {
      int rc = launch_fwd(G, G.buf[G.cur], G.buf[1 - G.cur], G.w, nullptr, G.gd, st);
      if (rc != ADI_OK) return rc;
    }
  } else {
    CKB(cudaMemsetAsync(d_sync, 0, sizeof(int) * (1 + n), st), "clear counters");
    BatchArgs a;
    a.shots = d_shots;
    a.items = d_items;
    a.n_items = n_items;
    a.ticket = d_sync;
    a.x_done = d_sync + 1;
    a.cur = g[0].cur;
    a.err = d_err;
    a.spin_limit = spin_limit;
    a.never_ready_shot = never_ready;
    cudaEvent_t ev = nullptr;
    if (profile && prof_begin(st, &ev) != ADI_OK) return ADI_ECUDA;
    CKB(launch_batch(a, batch_fp64, batch_grid, batch_smem, st), "batched step launch");
    if (profile && prof_end(st, ev, ADI_KERNEL_OTHER) != ADI_OK) return ADI_ECUDA;
    launches += 1;
  }
  for (Grid& G : g) {
    G.cur = 1 - G.cur;
    G.k += 1;
    G.from_init = false;
  }
  return ADI_OK;
}

// Batch mode 2: every shot's steps are a chain of the single-grid kernels on
// one of kBranches streams; the branches fork from `st` and join back into
// it, so shots of different sizes overlap and fill each other's tails, with
// no barrier between shots inside the `nsteps` steps.  Shots go to branches
// largest first, each to the branch with the fewest grid points so far, so
// that the branches end together at the join (for 64 shots of 256^2 to
// 2048^2 the fullest branch holds 1.004 of an even share, against 1.36 with
// shot s on branch s mod kBranches); they are launched in that order too.
int adi_wave::ensure_branches() {
  if (fork_ev) return ADI_OK;
  for (int b = 0; b < kBranches; ++b) {
    CKB(cudaStreamCreateWithFlags(&branch[b], cudaStreamNonBlocking), "create branch stream");
    CKB(cudaEventCreateWithFlags(&join_ev[b], cudaEventDisableTiming), "create join event");
  }
  CKB(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming), "create fork event");
  return ADI_OK;
}

int adi_wave::enqueue_batch_steps_parallel(int nsteps, cudaStream_t st) {
  int rc = ensure_branches();
  if (rc != ADI_OK) return rc;
  const int n = (int)g.size();
  const int nb = std::min(n, (int)kBranches);
  if ((int)shot_order.size() != n) {
    shot_order.resize(n);
    shot_branch.assign(n, 0);
    for (int s = 0; s < n; ++s) shot_order[s] = s;
    std::stable_sort(shot_order.begin(), shot_order.end(), [&](int a, int b) {
      return (long long)g[a].nx * g[a].ny > (long long)g[b].nx * g[b].ny;
    });
    std::vector<long long> load(nb, 0);
    for (int s : shot_order) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      shot_branch[s] = b;
      load[b] += (long long)g[s].nx * g[s].ny;
    }
  }
  CKB(cudaEventRecord(fork_ev, st), "fork");
  for (int b = 0; b < nb; ++b) CKB(cudaStreamWaitEvent(branch[b], fork_ev, 0), "branch wait");
  for (int s : shot_order) {
    Grid& G = g[s];
    cudaStream_t bs = branch[shot_branch[s]];
    int cur = G.cur;
    for (int t = 0; t < nsteps; ++t) {
      rc = launch_fwd(G, G.buf[cur], G.buf[1 - cur], G.w, nullptr, G.gd, bs);
      if (rc != ADI_OK) return rc;
      cur = 1 - cur;
    }
  }
  for (int b = 0; b < nb; ++b) {
    CKB(cudaEventRecord(join_ev[b], branch[b]), "join");
    CKB(cudaStreamWaitEvent(st, join_ev[b], 0), "join wait");
  }
  for (Grid& G : g) {
    if (nsteps & 1) G.cur = 1 - G.cur;
    G.k += nsteps;
    G.from_init = false;
  }
  return ADI_OK;
}
