// adi_internal.h -- host/device structures shared by the library's .cu files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace adi {

// Per-grid state read by the kernels from device memory, so that a captured
// CUDA graph picks up the current run's source and receivers on replay.
struct GridDev {
  long long k;          // time level of u_cur (u^k); the y sweep advances it
  long long k0;         // level at the start of the current run
  long long steps;      // length of the current run (bounds of traces)
  const float* wavelet; // w(t_k) samples, or null
  int n_wavelet;
  int src_ix, src_iy;   // source node, src_ix < 0 = none
  int n_rec;
  const int* rec;       // [n_rec][2] receiver nodes
  float* traces;        // [steps][n_rec]
};

// Device error word bits.
enum : int { ERR_NUMERIC = 1, ERR_TIMEOUT = 2 };

// Arguments of the fused RHS + x-sweep kernel (Eq. fr1's x operator).
struct XArgs {
  int nx, ny, ld;
  int log2tsys;   // threads per row (system) = 1 << log2tsys
  int spc;        // rows per CTA
  int pcr;        // CR -> PCR switch size
  const float* m;
  const float* u;   // u^k
  float* w;         // out: w = X^{-1} r
  double cx, cy;    // tau^2 / h1^2, tau^2 / h2^2
  double sc;        // tau^2 / (2 h1^2): s = sc * m
  double src_scale; // tau^2 / (h1 h2)
  const GridDev* gd;
  int persist;      // 1: persistent CTAs loop over row blocks (grid set by the launcher)
  int stage_mode;   // 1: rows staged through shared memory (FP32), 2: direct loads, 3: TMA pipeline
  int stage_off;    // byte offset of the staging area (set by the launcher), -1: none
  int* err;         // device error word (bounded waits), or null
  int xc;           // TMA pipeline: 2 = each row split over a cluster of two CTAs, else 1
};

// Arguments of the y-sweep + update kernel (Eq. fr2's y operator).
struct YArgs {
  int nx, ny, ld;
  int log2W;      // columns per strip = 1 << log2W
  int log2tcol;   // threads per column in one CTA
  int C;          // CTAs per cluster along the column
  int pcr;
  const float* m;
  const float* w;      // RHS
  const float* u_cur;  // u^k
  float* u_prev;       // in: u^{k-1}; out: u^{k+1}
  float* z_out;        // optional copy of z = u^{k+1} - 2u^k + u^{k-1} (adjoint recompute)
  double sc;           // tau^2 / (2 h2^2)
  GridDev* gd;         // k is advanced by one CTA
  int* err;
  int stage_off;       // byte offset of the u^k / u^{k-1} staging area in shared memory, -1: L2
  int stage_mode;      // 1: shared-memory staging, 2: L2 prefetch (launchers set stage_off)
  int persist;         // 1: persistent clusters loop over strips (grid set by the launcher)
};

// Launchers (adi_forward.cu).
cudaError_t launch_x(const XArgs& a, int K, bool fp64, bool tree, cudaStream_t st);
cudaError_t launch_y(const YArgs& a, int K, bool fp64, bool tree, cudaStream_t st);
cudaError_t launch_gather(const GridDev* gd, const float* u_new, int ld, int n_rec, cudaStream_t st);
cudaError_t launch_init(int nx, int ny, int ld, const float* m_pitched, const float* phi,
                        const float* psi, float* u0, float* u1, double tau, double cx_half,
                        double cy_half, int taylor, int src_ix, int src_iy, double src_half,
                        const float* wavelet, int n_wavelet, cudaStream_t st);
// min(m), max(m) bit patterns and a non-finite/non-positive flag into out3
// (device) and then host3 (mapped pinned host memory, device address): three
// launches, no copies.
cudaError_t launch_scan_m(const float* m, int nx, int ny, int ld, unsigned int* out3,
                          unsigned int* host3, cudaStream_t st);
// *dst = v on the stream (one-thread kernel; v travels as the argument).
cudaError_t launch_put_gd(GridDev* dst, const GridDev& v, cudaStream_t st);
size_t x_smem_bytes(int spc, int tsys, bool fp64, bool tree);
size_t y_smem_bytes(int W, int C, int tcol, bool fp64, bool tree);
size_t y_stage_bytes(int threads, int K);
size_t x_stage_bytes(int threads, int K);
size_t x_pipe_smem_bytes(int spc, int tsys, int K, int xc);
int x_pipe_box_lines(int tsys, int K);
size_t y_pipe_smem_bytes(int W, int C, int tcol, int K);
int y_pipe_box_rows(int tcol, int K);
cudaError_t encode_strip_map(CUtensorMap* out, const float* base, int ld, int ny, int box_cols,
                             int box_rows);
// Strip maps of the pipelined y sweep: w, m, u^k, u^{k-1}.
struct YMaps {
  CUtensorMap w, m, uc, up;
};
cudaError_t launch_y_pipe(const YArgs& a, int K, const YMaps& mp, cudaStream_t st);
// The same kernel on the reverse step's column systems: wbar (z_out) from
// lam (strip map `lam`) and m (a.m and strip map `m`); u fields unused.
cudaError_t launch_y_pipe_adj(const YArgs& a, int K, const CUtensorMap& lam, const CUtensorMap& m,
                              cudaStream_t st);
// Column solves without clusters (adi_ycoop.cu): persistent co-resident CTAs
// take (strip, segment) items; the C segments of a column meet through
// global memory.  Scratch of one grid:
struct YCoop {
  int C;        // segments per column (1..32)
  int cols;     // columns the summaries hold (nx rounded up to 32)
  int strips;   // strips the counters hold (nx / 16 rounded up)
  float* tops;  // [cols][C] segment summaries, 8 floats each
  int* sync;    // [strips][2] arrival / completion counters, zero between launches
};
size_t y_coop_smem_bytes(int W, int tcol, int K, int C);
int y_coop_segments(int ny, int tcol, int K);
cudaError_t launch_y_coop(const YArgs& a, int K, const YCoop& yc, const YMaps& mp, cudaStream_t st);
cudaError_t launch_y_coop_adj(const YArgs& a, int K, const YCoop& yc, const CUtensorMap& lam,
                              const CUtensorMap& m, cudaStream_t st);
cudaError_t configure_y_coop_kernels();

// The wider problem class and the literal half-level schemes (adi_models.cu).
// mode 0: Eq. CN1 with m^k = g_k m and a source field; 1: Eqs. fr1 / fr2 over
// half levels; 2: Listing 1's systems over half levels.
struct ModelXArgs {
  int nx, ny, ld, log2tsys, spc, mode;
  const float* m;
  const float* a;     // mode 0: u^{k-1}; modes 1, 2: u^{k-1/2}
  const float* b;     // u^k
  float* out;         // mode 0: w; modes 1, 2: u^{k+1/2}
  double cx, cy;      // tau^2 / h1^2, tau^2 / h2^2
  double sc;          // tau^2 / (2 h1^2)
  double src_scale;   // tau^2 / (h1 h2)
  double tau2;        // tau^2
  const float* g;     // [n_g] per-level factor of m (mode 0), or null
  int n_g;
  const float* f;     // [n_f][ny][nx] per-level source field (mode 0), or null
  int n_f;
  long long level;    // k
  const GridDev* gd;  // point source
};
struct ModelYArgs {
  int nx, ny, ld, log2W, log2tcol, C, mode;
  const float* m;
  const float* w;     // mode 0: the x pass's result; modes 1, 2: u^{k+1/2}
  const float* b;     // u^k
  float* io;          // mode 0: u^{k-1} in, u^{k+1} out; modes 1, 2: u^{k+1} out
  double sc;          // tau^2 / (2 h2^2)
  double src_scale;
  const float* g;
  int n_g;
  long long level;
  const GridDev* gd;
  int* err;
};
cudaError_t launch_x_model(const ModelXArgs& a, int K, cudaStream_t st);
cudaError_t launch_y_model(const ModelYArgs& a, int K, cudaStream_t st);
cudaError_t launch_advance_level(GridDev* gd, cudaStream_t st);
cudaError_t configure_model_kernels();
// Row tensor map for the pipelined x sweep (see adi_tma.cuh).
cudaError_t encode_row_map(CUtensorMap* out, const float* base, int ld, int ny, int box_lines);
cudaError_t launch_x_pipe(const XArgs& a, int K, const CUtensorMap& tu, const CUtensorMap& tm,
                          const CUtensorMap& tw, cudaStream_t st);
// Band form of the x sweep (x_stage 5): clusters of xc = 2, 4 or 8 CTAs walk
// bands of consecutive rows with a ring of three rows of u^k in shared memory.
size_t x_band_smem_bytes(int tsys, int K, int xc);
cudaError_t launch_x_band(const XArgs& a, int K, const CUtensorMap& tu, const CUtensorMap& tm,
                          const CUtensorMap& tw, cudaStream_t st);
constexpr int kMaxDynSmem = 227 * 1024;
cudaError_t configure_kernels();
// Kernel attributes of every kernel of the library on the current device,
// once per device (thread-safe); adi_run.cu.
cudaError_t configure_current_device();

}  // namespace adi
