// adi_noalloc.cu -- adi_wave_step_noalloc: one forward step of the factored
// scheme on caller-owned buffers that allocates no device memory.
//
// A step has one intermediate field, the x sweep's result w (Eq. fr1), and
// one small device record (GridDev: time level and source) that the sweep
// kernels read.  Here both live in static device arrays of this translation
// unit, sized at build time; their addresses are looked up once per device
// with cudaGetSymbolAddress and handed to the same x / y sweep kernels the
// handle API launches.  The record's values travel to the device as a kernel
// argument (a one-thread kernel writes them into the static record), so no
// host buffer is read after the call returns.  Nothing is allocated, on the
// device or through any library, on any call.
//
// The static arrays are shared by every call on a device, so calls on one
// device must not overlap: each must be ordered after the previous one has
// finished with them (same stream, or an event between streams).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/adiwave.h"
#include "adi_internal.h"
#include "adi_run.h"
#include "adi_sweeps.cuh"

using namespace adi;

namespace {

// 4,194,304 floats (16 MiB): grids with ld * ny up to this, e.g. 2048 x 2048.
constexpr size_t kMaxElems = size_t(1) << 22;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_w_scratch[kMaxElems];
static __device__ __align__(256) GridDev g_gd_scratch;

struct DevSlot {
  bool ready = false;
  float* w = nullptr;
  GridDev* gd = nullptr;
};
DevSlot g_slots[kMaxDevices];
std::mutex g_mu;

int fail_msg(int code, const std::string& msg) {
  set_thread_error(msg);
  return code;
}

// First call on a device: kernel attributes and the scratch addresses.
int device_slot(DevSlot** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("get device: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_msg(ADI_EUNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mu);
  DevSlot& s = g_slots[dev];
  if (!s.ready) {
    e = configure_current_device();
    if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("configure kernels: ") + cudaGetErrorString(e));
    void* w = nullptr;
    void* gd = nullptr;
    e = cudaGetSymbolAddress(&w, g_w_scratch);
    if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&gd, g_gd_scratch);
    if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("grid record address: ") + cudaGetErrorString(e));
    s.w = static_cast<float*>(w);
    s.gd = static_cast<GridDev*>(gd);
    s.ready = true;
  }
  *out = &s;
  return ADI_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// The call's grid record, passed by value, into the static record.
__global__ void set_record_kernel(GridDev hg, GridDev* dst) { *dst = hg; }

}  // namespace

extern "C" int adi_wave_step_noalloc(const adi_wave_desc* desc, int32_t ld, double m_max,
                                     const float* m, const float* u_cur, float* u_prev,
                                     const adi_source* src, int64_t k, void* stream) {
  if (!desc || !m || !u_cur || !u_prev) return fail_msg(ADI_EINVAL, "null pointer");
  const adi_wave_desc& d = *desc;
  if (d.nx < 1 || d.ny < 1 || d.nx > 32768 || d.ny > 32768) return fail_msg(ADI_EINVAL, "nx, ny must be 1..32768");
  if (!(d.lx > 0) || !(d.ly > 0) || !(d.dt > 0) || !std::isfinite(d.lx) || !std::isfinite(d.ly) ||
      !std::isfinite(d.dt))
    return fail_msg(ADI_EINVAL, "lx, ly, dt must be finite and > 0");
  if (d.fp64_solve < ADI_FP64_AUTO || d.fp64_solve > ADI_FP64_ALWAYS) return fail_msg(ADI_EINVAL, "bad fp64_solve mode");
  if (ld < d.nx || ld % 32 != 0) return fail_msg(ADI_EINVAL, "ld must be a multiple of 32 and >= nx");
  if ((size_t)ld * (size_t)d.ny > kMaxElems)
    return fail_msg(ADI_EINVAL, "grid too large for the no-allocation step: ld * ny = " +
                                    std::to_string((size_t)ld * (size_t)d.ny) + " floats, at most " +
                                    std::to_string(kMaxElems));
  if (!(m_max > 0) || !std::isfinite(m_max)) return fail_msg(ADI_EINVAL, "m_max must be finite and > 0");
  if (!aligned16(m) || !aligned16(u_cur) || !aligned16(u_prev)) return fail_msg(ADI_EINVAL, "buffers must be 16-byte aligned");
  if (u_cur == u_prev) return fail_msg(ADI_EINVAL, "u_cur and u_prev must be different buffers");
  if (k < 0) return fail_msg(ADI_EINVAL, "level k must be >= 0");
  const bool on = src && src->ix >= 0 && src->wavelet != nullptr && src->n_wavelet > 0;
  if (on && (src->ix >= d.nx || src->iy < 0 || src->iy >= d.ny)) return fail_msg(ADI_EINVAL, "source node outside the grid");

  DevSlot* slot = nullptr;
  int rc = device_slot(&slot);
  if (rc != ADI_OK) return rc;

  // launch geometry: the handle API's default plan for this grid
  Grid G;
  G.nx = d.nx;
  G.ny = d.ny;
  G.ld = ld;
  G.lx = d.lx;
  G.ly = d.ly;
  G.dt = d.dt;
  G.hx = d.lx / (d.nx + 1);
  G.hy = d.ly / (d.ny + 1);
  G.fp64mode = d.fp64_solve;
  G.mmax = m_max;
  const adi_wave_tuning t = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  std::string why;
  rc = plan_grid(G, t, why);
  if (rc != ADI_OK) return fail_msg(rc, why);
  const GridPlan& P = G.plan;
  // the y sweep without clusters needs scratch of its own; the default plan
  // picks it only for grids far beyond the static array's limit
  if (P.y_stage == ADI_STAGE_COOP) return fail_msg(ADI_EUNSUPPORTED, "grid shape needs the y sweep's own scratch");

  const cudaStream_t st = (cudaStream_t)stream;
  GridDev hg = {};
  hg.k = k;
  hg.k0 = k;
  hg.steps = 1;
  hg.wavelet = on ? src->wavelet : nullptr;
  hg.n_wavelet = on ? src->n_wavelet : 0;
  hg.src_ix = on ? src->ix : -1;
  hg.src_iy = on ? src->iy : -1;
  set_record_kernel<<<1, 1, 0, st>>>(hg, slot->gd);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("grid record: ") + cudaGetErrorString(e));

  XArgs xa;
  xa.nx = d.nx;
  xa.ny = d.ny;
  xa.ld = ld;
  xa.log2tsys = P.log2tsys;
  xa.spc = P.spc;
  xa.pcr = P.pcr;
  xa.m = m;
  xa.u = u_cur;
  xa.w = slot->w;
  xa.cx = d.dt * d.dt / (G.hx * G.hx);
  xa.cy = d.dt * d.dt / (G.hy * G.hy);
  xa.sc = d.dt * d.dt / (2.0 * G.hx * G.hx);
  xa.src_scale = d.dt * d.dt / (G.hx * G.hy);
  xa.gd = slot->gd;
  xa.persist = 0;
  xa.stage_mode = P.x_stage;
  xa.stage_off = -1;
  xa.err = nullptr;
  xa.xc = P.xc;
  YArgs ya;
  ya.nx = d.nx;
  ya.ny = d.ny;
  ya.ld = ld;
  ya.log2W = P.log2W;
  ya.log2tcol = P.log2tcol;
  ya.C = P.C;
  ya.pcr = P.pcr;
  ya.m = m;
  ya.w = slot->w;
  ya.u_cur = u_cur;
  ya.u_prev = u_prev;
  ya.z_out = nullptr;
  ya.stage_mode = P.y_stage;
  ya.persist = 0;
  ya.stage_off = 0;
  ya.sc = d.dt * d.dt / (2.0 * G.hy * G.hy);
  ya.gd = slot->gd;
  ya.err = nullptr;
  if (P.x_stage == 3) {  // host-side tensor maps of the caller's buffers (no allocation)
    const int L = x_pipe_box_lines((1 << P.log2tsys) / P.xc, P.kx);
    CUtensorMap tu, tm, tw;
    e = encode_row_map(&tu, u_cur, ld, d.ny, L);
    if (e == cudaSuccess) e = encode_row_map(&tm, m, ld, d.ny, L);
    if (e == cudaSuccess) e = encode_row_map(&tw, slot->w, ld, d.ny, L);
    if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("tensor maps: ") + cudaGetErrorString(e));
    e = launch_x_pipe(xa, P.kx, tu, tm, tw, st);
  } else {
    e = launch_x(xa, P.kx, P.fp64x, P.tree, st);
  }
  if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("x sweep launch: ") + cudaGetErrorString(e));
  if (P.y_stage == 3) {
    const int BH = y_pipe_box_rows(1 << P.log2tcol, P.ky);
    const int BW = 1 << P.log2W;
    YMaps mp;
    e = encode_strip_map(&mp.w, slot->w, ld, d.ny, BW, BH);
    if (e == cudaSuccess) e = encode_strip_map(&mp.m, m, ld, d.ny, BW, BH);
    if (e == cudaSuccess) e = encode_strip_map(&mp.uc, u_cur, ld, d.ny, BW, BH);
    if (e == cudaSuccess) e = encode_strip_map(&mp.up, u_prev, ld, d.ny, BW, BH);
    if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("strip maps: ") + cudaGetErrorString(e));
    e = launch_y_pipe(ya, P.ky, mp, st);
  } else {
    e = launch_y(ya, P.ky, P.fp64y, P.tree, st);
  }
  if (e != cudaSuccess) return fail_msg(ADI_ECUDA, std::string("y sweep launch: ") + cudaGetErrorString(e));
  return ADI_OK;
}
