// adi_adjoint.h -- arguments and launchers of the reverse-step kernels.
#pragma once

#include <cuda_runtime.h>

#include "adi_internal.h"

namespace adi {

// Column solves of Y^T wbar = lam.
struct YAdjArgs {
  int nx, ny, ld;
  int log2W, log2tcol, C, pcr;
  const float* m;
  const float* lam;  // lam^{k+1} (= zbar)
  float* wbar;       // out
  double sc;         // tau^2 / (2 h2^2)
};

// Row solves of X^T rbar = wbar + the FP64 gradient accumulation.
struct XAdjArgs {
  int nx, ny, ld;
  int log2tsys, spc, pcr;
  const float* m;
  const float* wbar;
  const float* w;    // forward x-sweep result of this step
  const float* z;    // forward y-sweep result of this step
  float* rbar;       // out
  double* g64;       // [ny][ld] FP64 sum of the dJ/dm increments of every reverse step so far
  float* gw;         // dJ/dwavelet or null
  long long level;   // k of this step
  double sc;         // tau^2 / (2 h1^2)
  double src_scale;  // tau^2 / (h1 h2)
  int src_ix, src_iy;
  const float* wavelet;
  int n_wavelet;
  int staged;     // 1: FP32 rows staged through shared memory (coalesced), when it fits
  int stage_off;  // set by the launcher
};

struct LamArgs {
  int nx, ny, ld;
  const float* m;
  const float* rbar;
  float* L0;  // lam^{k+1}, read then cleared
  float* L1;  // lam^k
  float* L2;  // lam^{k-1}
  float cx, cy;  // tau^2 / h1^2, tau^2 / h2^2
  // receiver residuals of the previous step (u^k's misfit), added to lam^k
  // at the receiver nodes, or null: the receivers of row j are
  // rrow[j] .. rrow[j+1]-1, at columns rix[], residual index rid[]
  const float* resid;
  const int* rrow;
  const int* rix;
  const int* rid;
};

struct TaylorArgs {
  int nx, ny, ld;
  const float* phi;  // u^0 (pitched)
  const float* lam;  // lam^1
  double* gm;
  float* gw;
  long long level;   // 0
  double cx_half, cy_half, src_half;
  int src_ix, src_iy;
};

cudaError_t launch_x_adj(const XAdjArgs& a, int K, bool fp64, cudaStream_t st);
cudaError_t launch_y_adj(const YAdjArgs& a, int K, bool fp64, cudaStream_t st);
cudaError_t launch_lam_update(const LamArgs& a, cudaStream_t st);
cudaError_t launch_seed(float* lam, int ld, const int* rec, int n_rec, const float* resid,
                        cudaStream_t st);
cudaError_t launch_taylor_adj(const TaylorArgs& a, cudaStream_t st);
cudaError_t configure_adjoint_kernels();

}  // namespace adi
