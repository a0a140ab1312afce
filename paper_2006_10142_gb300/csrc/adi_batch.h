// adi_batch.h -- device structures and launchers of the batched form.
#pragma once

#include <cuda_runtime.h>

#include "adi_internal.h"

namespace adi {

constexpr int kBatchK = 16;  // unknowns per thread in the batched kernels

// One shot, both buffer orientations: [c] has u^k = buf[c], u^{k-1} = buf[1-c].
struct BatchShot {
  XArgs xa[2];
  YArgs ya[2];
  int x_items;
  int y_items;
};

struct BatchArgs {
  const BatchShot* shots;
  const int2* items;     // (shot, index << 1 | kind), kind 0 = x item, 1 = y item
  int n_items;
  int* ticket;           // next item (zeroed before each launch)
  int* x_done;           // [n_shots] finished x items (zeroed before each launch)
  int cur;               // orientation of every shot this step
  int* err;
  long long spin_limit;  // bound of the dependency wait
  int never_ready_shot;  // test hook: this shot's x items never count as done (-1: none)
};

cudaError_t launch_batch(const BatchArgs& a, bool fp64, int grid, size_t smem, cudaStream_t st);
cudaError_t configure_batch_kernels(int* blocks_per_sm_f32, int* blocks_per_sm_f64, size_t smem_f32,
                                    size_t smem_f64);

}  // namespace adi
