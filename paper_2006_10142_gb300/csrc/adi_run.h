// adi_run.h -- the handle behind the C ABI (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/adiwave.h"
#include "adi_batch.h"
#include "adi_internal.h"

namespace adi {

// Diagonal dominance ratio above which the elimination runs in FP64.
constexpr double kWeakDominance = 0.9;

struct GridPlan {
  // x sweep
  int kx = 16, log2tsys = 0, spc = 1, pcr = 32;
  bool fp64x = false;
  // y sweep
  int ky = 8, log2W = 3, log2tcol = 0, C = 1;
  bool fp64y = false;
  int graph = 1;
  bool tree = true;  // solver variant (see adi_sweeps.cuh)
  int cta_threads = 0, cta_threads_y = 0;
  int y_stage = 1;   // 1: shared-memory staging, 2: L2 prefetch
  int persist = 0;   // 1: persistent sweeps with L2 prefetch of the next tile
  int x_stage = 2;   // 1: rows staged through shared memory, 2: direct, 3: TMA pipeline
  int xc = 1;        // TMA pipeline: CTAs per row (1 or 2)

  bool operator==(const GridPlan& o) const {
    return kx == o.kx && log2tsys == o.log2tsys && spc == o.spc && pcr == o.pcr &&
           fp64x == o.fp64x && ky == o.ky && log2W == o.log2W && log2tcol == o.log2tcol &&
           C == o.C && fp64y == o.fp64y && graph == o.graph && tree == o.tree &&
           cta_threads == o.cta_threads && cta_threads_y == o.cta_threads_y &&
           y_stage == o.y_stage && persist == o.persist && x_stage == o.x_stage && xc == o.xc;
  }
};

struct Grid {
  int nx = 0, ny = 0, ld = 0;
  double lx = 1, ly = 1, dt = 0, hx = 0, hy = 0;
  int start = 0, fp64mode = 0;
  float* m = nullptr;               // [ny][ld]
  float* buf[2] = {nullptr, nullptr};  // buf[cur] = u^k, buf[1-cur] = u^{k-1}
  float* w = nullptr;               // scratch [ny][ld]
  int cur = 1;
  long long k = 1;
  bool from_init = true;            // state is the start-up's (u^0, u^1), untouched since
  GridDev* gd = nullptr;            // device copy
  GridDev hgd = {};                 // host mirror
  double mmin = 0, mmax = 0;
  GridPlan plan;
  CUtensorMap tm_buf[2], tm_m, tm_w;  // row maps of buf[0], buf[1], m, w (pipelined x sweep)
  int tm_lines = 0;                 // box height they were encoded with, 0 = none
  CUtensorMap ts_buf[2], ts_m, ts_w;  // strip maps (pipelined y sweep)
  int ts_rows = 0;                  // 64 * box rows + box columns they were encoded with, 0 = none
  YCoop yc = {0, 0, 0, nullptr, nullptr};  // scratch of the y sweep without clusters (y_stage 4)
};

// What adi_wave_adjoint needs to replay the last run.
struct RunRecord {
  bool valid = false;
  long long k0 = 0;
  int steps = 0;
  int every = 0;
  adi_source src = {-1, -1, nullptr, 0};
  std::vector<int> rec;             // [n_rec][2] host copy
  std::vector<float*> ckpt;         // checkpoint c: 2 fields (u^{k-1}, u^k) at step c*every
  size_t ckpt_bytes = 0;
  bool taylor = false;              // run started at level 1 right after a Taylor start-up
};

// Problem class of the handle (adi_wave_set_model); the default is the
// factored delta form with a time-independent m and the point source only.
struct Model {
  int scheme = ADI_SCHEME_FACTORED;
  const float* g = nullptr;
  int n_g = 0;
  const float* f = nullptr;
  int n_f = 0;
  bool active = false;  // anything but the default
  GridPlan plan;        // one-shot launch geometry of the model kernels
};

struct ProfRec {
  cudaEvent_t a, b;
  int kind;
};

// Device workspace of adi_wave_adjoint (allocated on first use, reused).
struct AdjWork {
  size_t fbytes = 0;  // bytes of one pitched field
  int E = 0;          // segment length it was sized for
  float* wseg = nullptr;  // [E] forward x-sweep results of a segment
  float* zseg = nullptr;  // [E] forward y-sweep results of a segment
  float* wb = nullptr;    // wbar
  float* rb = nullptr;    // rbar
  double* g64 = nullptr;  // [ny][ld] FP64 sum of the dJ/dm increments
  float* L[3] = {nullptr, nullptr, nullptr};  // lam^{k+1}, lam^k, lam^{k-1}
  float* A = nullptr;     // recompute state
  float* B = nullptr;
  GridDev* gd = nullptr;
  int* rec = nullptr;     // [n_rec][2] receivers, then the per-row table (see adjoint())
  int rec_cap = 0;        // ints
  std::vector<int> rtab;  // host copy of the per-row table
};

}  // namespace adi

struct adi_wave {
  std::vector<adi::Grid> g;
  int* d_err = nullptr;
  int* d_rec = nullptr;
  unsigned int* scan = nullptr;
  // the scan's result, written by a kernel into mapped pinned host memory so
  // that reading it needs no copy engine (those may be busy with a caller's
  // large copies on other streams)
  volatile unsigned int* scan_host = nullptr;
  unsigned int* scan_host_dev = nullptr;
  int rec_cap = 0;
  cudaStream_t cap = nullptr;  // private stream used only for graph capture
  cudaGraphExec_t pair[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [orientation][gather]
  adi_wave_tuning tuning = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  int ckpt_every = 0;
  adi::RunRecord rr;
  adi::Model model;
  adi::AdjWork aw;
  bool profile = false;
  std::vector<adi::ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  int64_t launches = 0;
  std::string err;

  // batched form (n_shots > 1)
  bool batch_fp64 = false;
  int batch_mode = 2;                 // 0: persistent kernel, 1: plain kernels per shot,
                                      // 2 (default): plain kernels per shot on parallel branches
  static constexpr int kBranches = 8; // streams of batch mode 2
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kBranches] = {};
  std::vector<int> shot_order;  // batch mode 2: shots by decreasing size
  std::vector<int> shot_branch; // batch mode 2: branch of each shot
  int ensure_branches();
  int enqueue_batch_steps_parallel(int nsteps, cudaStream_t st);
  adi::BatchShot* d_shots = nullptr;
  int2* d_items = nullptr;
  int n_items = 0;
  int* d_sync = nullptr;              // [1 + n_shots]: ticket, x_done[]
  int batch_grid = 0;
  size_t batch_smem = 0;
  long long spin_limit = 1ll << 22;
  int never_ready = -1;
  int64_t pair_launches = 0;
  int setup_batch(cudaStream_t st);
  int enqueue_batch_step(cudaStream_t st);
  int run_batch(int steps, const adi_source* src, cudaStream_t st);

  int create(const adi_wave_desc* desc, int n, const float* const* m, const float* const* phi,
             const float* const* psi, const adi_source* src, cudaStream_t st);
  int reset(const float* const* m, const float* const* phi, const float* const* psi,
            const adi_source* src, cudaStream_t st);
  int start_grid(int s, const float* m, const float* phi, const float* psi, const adi_source* sr,
                 cudaStream_t st);
  int run(int steps, const adi_source* src, const int32_t* rec_xy, int n_rec, float* traces,
          cudaStream_t st, bool record);
  int adjoint(const float* resid, double* grad_m, float* grad_wavelet, int every, cudaStream_t st);
  int set_state(int shot, const float* u_prev, const float* u_cur, int64_t k, cudaStream_t st);
  int sync_status(cudaStream_t st);
  int set_tuning(const adi_wave_tuning& t);
  int profile_read(double* ms, int64_t* launches, int n_kinds);
  ~adi_wave();

  // internals
  int enqueue_step(adi::Grid& G, cudaStream_t st, bool gather);
  int launch_fwd(adi::Grid& G, const float* u_cur, float* u_prev, float* w, float* z_out,
                 adi::GridDev* gd, cudaStream_t st);
  int ensure_adj_work(adi::Grid& G, int E, int n_rec);
  void free_adj_work();
  int launch_pair_graph(adi::Grid& G, cudaStream_t st, bool gather);
  void drop_graphs();
  int prof_begin(cudaStream_t st, cudaEvent_t* a);
  int prof_end(cudaStream_t st, cudaEvent_t a, int kind);
  int upload_gd(adi::Grid& G, cudaStream_t st);
  int ensure_ycoop(adi::Grid& G);
  int set_model(const adi_wave_model& m);
  int enqueue_model_step(adi::Grid& G, cudaStream_t st, bool gather);
};

namespace adi {
int fail(adi_wave* h, int code, const std::string& msg);
int cuda_fail(adi_wave* h, cudaError_t e, const char* what);
int plan_grid(Grid& G, const adi_wave_tuning& t, std::string& why);
void set_thread_error(const std::string& msg);
}  // namespace adi
