// adi_batch.cu -- the batched form: many independent grids ("shots") of
// uneven size advanced together, one persistent kernel launch per time step.
//
// The step of every shot is cut into work items of one CTA each: x items
// (a block of rows: RHS assembly + x solve) and y items (a strip of columns:
// y solve + update).  All x items of all shots come first in the item list,
// then all y items.  Persistent CTAs take items in list order from a global
// ticket counter.  A y item of shot b may start only when every x item of
// shot b has finished (its strip reads w of all rows); each x item bumps a
// per-shot counter with release semantics and the y item waits on it with
// acquire semantics.  Because items are handed out in list order, every x
// item a y item waits for was taken earlier by a CTA that is running and
// never waits itself, so the wait always ends; it is still bounded by an
// iteration limit, after which the CTA records ERR_TIMEOUT and skips the item
// (adi_wave_sync_status reports ADI_ETIMEOUT).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "adi_batch.h"
#include "adi_bodies.cuh"

namespace adi {

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int K, typename T, int MAXT, bool TREE>
__global__ void __launch_bounds__(MAXT, 1) batch_step_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item, s_go;
  __shared__ XArgs s_xa;
  __shared__ YArgs s_ya;
  for (;;) {
    __syncthreads();  // the previous item is done with shared memory
    if (threadIdx.x == 0) {
      s_item = atomicAdd(a.ticket, 1);
      if (s_item < a.n_items) {
        const int2 it = a.items[s_item];
        if ((it.y & 1) == 0) s_xa = a.shots[it.x].xa[a.cur];
        else s_ya = a.shots[it.x].ya[a.cur];
      }
    }
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_items) return;
    const int2 it = a.items[item];
    const int idx = it.y >> 1;
    if ((it.y & 1) == 0) {
      x_rows_body<K, T, TREE>(s_xa, idx, smem);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.x_done + it.x, 1);
      }
    } else {
      if (threadIdx.x == 0) {
        const int target = a.shots[it.x].x_items + (it.x == a.never_ready_shot ? 1 : 0);
        long long n = 0;
        int go = 1;
        while (ld_acquire_gpu(a.x_done + it.x) < target) {
          if (++n > a.spin_limit) {
            atomicOr(a.err, ERR_TIMEOUT);
            go = 0;
            break;
          }
          __nanosleep(256);
        }
        s_go = go;
      }
      __syncthreads();
      if (s_go) y_strip_body<K, T, TREE>(s_ya, idx, 0, idx == 0, smem);
    }
  }
}

template <int K, typename T, int MAXT>
static cudaError_t launch_batch_t(const BatchArgs& a, int grid, size_t smem, cudaStream_t st) {
  batch_step_kernel<K, T, MAXT, true><<<grid, MAXT, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs& a, bool fp64, int grid, size_t smem, cudaStream_t st) {
  return fp64 ? launch_batch_t<kBatchK, double, 512>(a, grid, smem, st)
              : launch_batch_t<kBatchK, float, 1024>(a, grid, smem, st);
}

// The per-block limit covers static plus dynamic shared memory.
template <typename KernT>
static cudaError_t allow_dyn_smem(KernT kern) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxDynSmem - (int)fa.sharedSizeBytes);
}

cudaError_t configure_batch_kernels(int* blocks_per_sm_f32, int* blocks_per_sm_f64, size_t smem_f32,
                                    size_t smem_f64) {
  cudaError_t e = allow_dyn_smem(batch_step_kernel<kBatchK, float, 1024, true>);
  if (e == cudaSuccess) e = allow_dyn_smem(batch_step_kernel<kBatchK, double, 512, true>);
  if (e == cudaSuccess && blocks_per_sm_f32)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm_f32, batch_step_kernel<kBatchK, float, 1024, true>, 1024, smem_f32);
  if (e == cudaSuccess && blocks_per_sm_f64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm_f64, batch_step_kernel<kBatchK, double, 512, true>, 512, smem_f64);
  return e;
}

}  // namespace adi
