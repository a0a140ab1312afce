/*
 * adiwave.h -- C ABI of libadiwave.so, the GB300 (sm_103a) implementation of
 * the implicit ADI scheme for the 2D acoustic wave equation of Altybay,
 * Ruzhansky and Tokmagambetov, "A parallel hybrid implementation of the 2D
 * acoustic wave equation".
 *
 * Problem (Section 2, Eqs. f1-f5): u_tt - m (u_xx + u_yy) = f on
 * [0,T] x [0,lx] x [0,ly], u = phi and u_t = psi at t = 0, u = 0 on the
 * boundary.  The coefficient that multiplies the Laplacian is passed as
 * m = c^2 (c is the wave speed) and does not depend on time.
 *
 * Grid (Eq. f6): nx x ny interior nodes, h1 = lx / (nx + 1),
 * h2 = ly / (ny + 1); node (i, j), 0 <= i < nx, 0 <= j < ny, sits at
 * ((i + 1) h1, (j + 1) h2).  The Dirichlet ring (Eq. CN3) is implicit and
 * never stored.  Every field crossing this ABI is FP32, row-major
 * [ny][nx] with x fastest, contiguous (row stride nx), in DEVICE memory
 * unless stated otherwise.
 *
 * Time stepping: the Crank-Nicolson three-level scheme of Eq. (CN1) in
 * delta form, (I - S Lap) z = tau^2 (m Lap u^k + f^k), z = u^{k+1} - 2u^k +
 * u^{k-1}, S = diag(tau^2 m / 2), with the ADI factorisation of Section 2
 * (sub-problems Eqs. fr1 and fr2): a tridiagonal sweep along x per row,
 * then one along y per column, each solved on the GPU by a per-thread
 * partition step followed by cyclic reduction of the interface system and
 * warp-shuffle parallel cyclic reduction for its last levels (Section 3.1
 * solves the same systems by cyclic reduction).
 *
 * Point source: f^k = w(t_k) / (h1 h2) at one node (a delta-like datum
 * approximated on the grid, Section 2).  Time level k uses the sample
 * wavelet[k], t_k = k tau.
 *
 * Streams and ordering: every call enqueues its work on the CUDA stream it
 * is given (a cudaStream_t passed as void*, NULL = legacy default stream)
 * and returns without waiting for the GPU, unless stated otherwise.  Device
 * buffers passed in must stay valid until the work that reads or writes
 * them has completed in stream order.
 *
 * Errors: every int-returning call returns ADI_OK (0) or one of the
 * ADI_E* codes below; no C++ exception and no abort crosses the ABI.
 * Conditions found on the GPU (non-finite values, an expired bounded wait)
 * are recorded in a device error word and reported by
 * adi_wave_sync_status().  adi_wave_strerror() turns a code into text and
 * adi_wave_last_error() gives the detail of the last failure on a handle.
 *
 * Threads: a handle may be used by one host thread at a time.
 */
#ifndef ADIWAVE_H
#define ADIWAVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ADI_OK = 0,
    ADI_EINVAL = 1,      /* invalid argument (null pointer, size, index, mode) */
    ADI_ENOMEM = 2,      /* device or host allocation failed */
    ADI_ECUDA = 3,       /* a CUDA runtime call failed */
    ADI_ENUMERIC = 4,    /* a non-finite value was produced (device flag) */
    ADI_ETIMEOUT = 5,    /* a bounded device-side wait expired (device flag) */
    ADI_ESTATE = 6,      /* call not valid in the handle's state */
    ADI_EUNSUPPORTED = 7 /* valid request the library does not implement for this shape or mode */
};

enum { ADI_START_PAPER = 0,     /* Eq. (CN2): u^1 = phi + tau psi */
       ADI_START_TAYLOR2 = 1 }; /* u^1 = phi + tau psi + tau^2/2 (m Lap phi + f^0) */

enum { ADI_FP64_AUTO = 0,   /* FP64 elimination only where diagonal dominance is weak */
       ADI_FP64_NEVER = 1,  /* always FP32 elimination */
       ADI_FP64_ALWAYS = 2  /* always FP64 elimination (FP32 storage) */ };

typedef struct adi_wave adi_wave; /* opaque; owned by the library */

/* One grid.  nx, ny >= 1 (at most 32768 each); lx, ly > 0; dt = tau > 0. */
typedef struct {
    int32_t nx, ny;
    double lx, ly;
    double dt;
    int32_t start;      /* ADI_START_* */
    int32_t fp64_solve; /* ADI_FP64_* */
} adi_wave_desc;

/* Point source of one grid.  ix < 0 means "no source".  wavelet is a device
 * array of n_wavelet FP32 samples, wavelet[k] = w(t_k); levels k >=
 * n_wavelet get w = 0.  The array is borrowed: it must stay valid while
 * work that reads it is in flight, and until adi_wave_adjoint() returns if
 * the run is later differentiated. */
typedef struct {
    int32_t ix, iy;
    const float *wavelet;
    int32_t n_wavelet;
} adi_source;

/* Create a handle for n_shots independent grids (n_shots == 1: one grid;
 * n_shots > 1: the batched form that advances all grids together, one
 * persistent kernel launch per sweep and step).
 *   desc[s]      grid of shot s (host array of n_shots).
 *   m[s]         device pointer, [ny][nx] FP32 coefficient m = c^2 > 0.
 *   phi[s]       device pointer, [ny][nx] FP32 initial value u(0).
 *   psi          host array of n_shots device pointers to u_t(0), or NULL;
 *                entries may be NULL (= 0).
 *   src          host array of n_shots sources, or NULL; only read by the
 *                Taylor start (f^0).
 * The inputs are copied into library-owned device memory (row pitch padded
 * to 32 floats) in stream order; the caller may free them once the stream
 * has passed this call.  After init the handle holds u^0 and u^1 (time
 * level k = 1), Eq. (CN2).  Returns ADI_EINVAL for a bad size or pointer,
 * ADI_ENOMEM if device memory runs out (nothing is leaked, *out = NULL). */
int adi_wave_init(adi_wave **out, const adi_wave_desc *desc, int32_t n_shots,
                  const float *const *m, const float *const *phi,
                  const float *const *psi, const adi_source *src,
                  void *stream);

/* Re-run the start-up of Eq. (CN2) in place on an existing handle: copy new
 * coefficients m (may be NULL = keep), initial data phi (and psi, may be
 * NULL) of every shot, set the level back to k = 1 and forget the recorded
 * run.  Same pointer conventions as adi_wave_init.  A new m is scanned for
 * its range first (the plan depends on it; the host waits for the scan):
 * a coefficient that is not finite and > 0 gives ADI_EINVAL and leaves that
 * shot's medium, plan and state unchanged.  Allocates nothing, except the
 * y sweep's segment scratch the first time a new medium moves the plan to
 * ADI_STAGE_COOP. */
int adi_wave_reset(adi_wave *h, const float *const *m, const float *const *phi,
                   const float *const *psi, const adi_source *src, void *stream);

/* Advance every grid by one time step (u^{k-1}, u^k -> u^k, u^{k+1}),
 * Algorithm 1's loop body.  src: host array of n_shots sources or NULL. */
int adi_wave_step(adi_wave *h, const adi_source *src, void *stream);

/* Advance by `steps` time steps (Algorithm 1's loop).  The steps of a
 * single grid are replayed from a captured CUDA graph.
 *   src      host array of n_shots sources or NULL.
 *   rec_xy   HOST array [n_rec][2] of receiver nodes (ix, iy) of shot 0, or
 *            NULL with n_rec = 0; receivers need n_shots == 1.
 *   traces   device [steps][n_rec] FP32: traces[s][r] = u^{k0+s+1}(rec r),
 *            k0 the level at the call; NULL allowed when n_rec = 0.
 * The run is remembered (start state, steps, source, receivers) so that
 * adi_wave_adjoint() can differentiate it; with checkpointing enabled
 * (adi_wave_set_checkpointing) the states every `every` steps are kept. */
int adi_wave_run(adi_wave *h, int32_t steps, const adi_source *src,
                 const int32_t *rec_xy, int32_t n_rec, float *traces,
                 void *stream);

/* Keep (u^{k-1}, u^k) every `every` steps during adi_wave_run (0 = off).
 * The memory (2 fields per checkpoint) is allocated by the next run. */
int adi_wave_set_checkpointing(adi_wave *h, int32_t every);

/* Gradient of J = 1/2 sum_s sum_r (traces[s][r] - d[s][r])^2 for the last
 * adi_wave_run of a single grid, given resid = traces - d (device
 * [steps][n_rec] FP32).  The transposed x and y sweeps run backward in
 * time; the forward fields are recomputed from checkpoints taken every
 * ckpt_every steps (reusing the run's checkpoints when they match).
 *   grad_m        device [ny][nx] FP64, overwritten with dJ/dm (m = c^2);
 *                 each reverse step's contribution is formed in FP32 from
 *                 the FP32 fields and added to an FP64 sum (the reverse
 *                 accumulation over all steps is FP64).
 *   grad_wavelet  device [n_wavelet] FP32 dJ/dw(t_k), or NULL.
 * The handle's state (u^{k-1}, u^k) is left as it was after the run.
 * Returns ADI_ESTATE if no single-grid run was recorded. */
int adi_wave_adjoint(adi_wave *h, const float *resid, double *grad_m,
                     float *grad_wavelet, int32_t ckpt_every, void *stream);

/* Copy the state of shot `shot` out: u_prev = u^{k-1}, u_cur = u^k (device
 * [ny][nx] each, either may be NULL) and *k = k (may be NULL; the level is
 * tracked on the host, so *k is exact when the call returns).  This is the
 * state Algorithm 1 carries from one step to the next (its two time levels,
 * u^k and the previous level U0, before the swap). */
int adi_wave_get_state(const adi_wave *h, int32_t shot, float *u_prev,
                       float *u_cur, int64_t *k, void *stream);

/* Replace the state of shot `shot` (device [ny][nx] each) and its level k:
 * Algorithm 1's two time levels (u^{k-1}, u^k) from which the next step
 * starts.  Clears the recorded run. */
int adi_wave_set_state(adi_wave *h, int32_t shot, const float *u_prev,
                       const float *u_cur, int64_t k, void *stream);

/* Wait for the handle's work on `stream` and report the device error word:
 * ADI_OK, ADI_ENUMERIC or ADI_ETIMEOUT (ADI_ECUDA if the wait failed).
 * Clears the word.  This call blocks the host. */
int adi_wave_sync_status(adi_wave *h, void *stream);

/* Free everything the handle owns (device memory, graphs, events).  Waits
 * for the handle's outstanding work first.  NULL is ignored.  (Resource
 * management of this library; the paper has no counterpart.) */
void adi_wave_destroy(adi_wave *h);

/* Static text for a return code (error reporting of this library; the paper
 * has no counterpart). */
const char *adi_wave_strerror(int code);

/* Detail of the last failing call on h (empty string if none); with h = NULL,
 * the detail of the last failed adi_wave_init or adi_wave_step_noalloc on the
 * calling thread.  The returned text is owned by the library and valid until
 * the next call on h (or on the thread).  No counterpart in the paper. */
const char *adi_wave_last_error(const adi_wave *h);

/* ---- tuning (the autotuner's knobs) -------------------------------------
 * chunk_x, chunk_y: rows of a line held by one thread in the partition step
 *                   (4, 8, 16 or 32);
 * rows_per_cta:     systems (grid rows) solved by one CTA in the x sweep;
 * cols_per_cta:     columns of the strip one CTA (cluster) solves in the
 *                   y sweep (8, 16 or 32);
 * pcr_size:         ADI_SOLVER_CR_SMEM only: size of the interface system
 *                   handed from cyclic reduction in shared memory to
 *                   warp-shuffle parallel cyclic reduction (2, 4, 8, 16 or
 *                   32; the CR-to-PCR switch level);
 * use_graph:        1 = replay steps from a captured CUDA graph, -1 = never;
 * solver:           ADI_SOLVER_TREE (cyclic reduction of the interface
 *                   system across warp lanes by register shuffles, PCR of the
 *                   warp summaries) or ADI_SOLVER_CR_SMEM (cyclic reduction
 *                   level by level in shared memory, PCR for the last
 *                   `pcr_size` equations);
 * cta_threads:      upper bound on threads per CTA of the x sweep (64, 128,
 *                   256, 512 or 1024; smaller CTAs let several share an SM);
 * cta_threads_y:    the same for the y sweep;
 * y_stage:          how the y sweep fetches u^k, u^{k-1} for its update while
 *                   it solves: ADI_STAGE_SMEM (asynchronous copies into
 *                   shared memory), ADI_STAGE_L2 (prefetch into L2, no
 *                   shared memory, more CTAs per SM) or ADI_STAGE_TMA
 *                   (persistent clusters: the next strip's w and m arrive in
 *                   shared memory by bulk asynchronous copies while the
 *                   current strip is solved, and its u^k, u^{k-1} are
 *                   prefetched into L2; FP32 tree solver, 16 columns) or
 *                   ADI_STAGE_COOP (the same pipeline without clusters: a
 *                   persistent grid of co-resident CTAs takes (strip,
 *                   column segment) items and the segments of a column meet
 *                   through global memory, so long columns do not need
 *                   clusters of up to 16 CTAs; FP32 tree solver; strips
 *                   of 16 columns (chunk_y 32 with 256 or 512 threads,
 *                   chunk_y 16 with 512) or 32 columns (512 threads,
 *                   chunk_y 32 or 16); at most 32 segments per column;
 *                   the automatic choice for columns of 8192 rows or more);
 * persist:          1 = one wave of resident CTAs (clusters) loops over the
 *                   tiles of each sweep and prefetches its next tile into L2
 *                   while solving the current one; -1 = one CTA per tile;
 * x_stage:          how the x sweep reads its rows: ADI_STAGE_SMEM (coalesced
 *                   loads, right-hand side formed in that layout and handed
 *                   to the solving threads through shared memory; w written
 *                   back the same way) or ADI_STAGE_DIRECT (each thread loads
 *                   and stores its own chunk) or ADI_STAGE_TMA (persistent
 *                   CTAs; the next rows of u^k and m arrive in shared memory
 *                   by TMA tensor copies while the current rows are solved;
 *                   FP32 tree solver, rows of >= 256 floats) or
 *                   ADI_STAGE_BAND (each cluster of x_cluster = 2, 4 or 8
 *                   CTAs walks a band of consecutive rows, keeping rows
 *                   j - 1, j, j + 1 of u^k in shared memory: the halo rows
 *                   come from there and every row is read from HBM once;
 *                   K = 32, rows of at least 1024 unknowns per CTA);
 *                   FP64 elimination always reads directly;
 * x_cluster:        ADI_STAGE_TMA: 1 = one CTA per row, 2 or 4 = each row
 *                   split over a cluster of that many CTAs (K = 32, one row
 *                   per cluster; 4: CTAs of 32..128 threads, four per SM);
 *                   ADI_STAGE_BAND: 2, 4 or 8 CTAs per row.
 * Zero fields mean "choose automatically". */
enum { ADI_STAGE_AUTO = 0, ADI_STAGE_SMEM = 1, ADI_STAGE_L2 = 2, ADI_STAGE_DIRECT = 2,
       ADI_STAGE_TMA = 3, ADI_STAGE_COOP = 4 /* y_stage only */,
       ADI_STAGE_BAND = 5 /* x_stage only */ };
enum { ADI_SOLVER_AUTO = 0, ADI_SOLVER_TREE = 1, ADI_SOLVER_CR_SMEM = 2 };
typedef struct {
    int32_t chunk_x, chunk_y;
    int32_t rows_per_cta;
    int32_t cols_per_cta;
    int32_t pcr_size;
    int32_t use_graph;
    int32_t solver;
    int32_t cta_threads;
    int32_t cta_threads_y;
    int32_t y_stage;
    int32_t persist;
    int32_t x_stage;
    int32_t x_cluster;
} adi_wave_tuning;

int adi_wave_get_tuning(const adi_wave *h, adi_wave_tuning *t);
int adi_wave_set_tuning(adi_wave *h, const adi_wave_tuning *t);

/* ---- measurement --------------------------------------------------------
 * With profiling on, the single-grid forward path records a CUDA event pair
 * around every launch of each kernel kind on the launching stream and runs
 * without graphs.  adi_wave_profile_read() waits for the handle's work,
 * sums the recorded durations per kind into ms[kind] and launch counts
 * into launches[kind] for kind < n_kinds, and clears the records.  Kinds:
 * 0 = x sweep (RHS + x solve), 1 = y sweep (+ update), 2 = other (the
 * batched persistent step). */
enum { ADI_KERNEL_X = 0, ADI_KERNEL_Y = 1, ADI_KERNEL_OTHER = 2, ADI_KERNEL_KINDS = 3 };
int adi_wave_profile(adi_wave *h, int32_t enable);
int adi_wave_profile_read(adi_wave *h, double *ms, int64_t *launches,
                          int32_t n_kinds);

/* ---- batched form (n_shots > 1) -------------------------------------------
 * mode 0: every step of all shots is one persistent kernel launch that hands
 * out x-sweep and y-sweep work items of all shots from a global queue (y
 * items of a shot wait, bounded, for that shot's x items);
 * mode 1: the plain single-grid kernels (TMA-pipelined where the shape
 * allows) launched once per shot and step, one after the other;
 * mode 2 (default): the same plain kernels, each shot's steps a chain on one
 * of eight streams that fork from and join into the caller's stream
 * (parallel graph branches when replayed), so shots overlap one another's
 * launches and tails.
 * ADI_EINVAL for other modes or single-grid handles. */
int adi_wave_set_batch_mode(adi_wave *h, int32_t mode);

/* Failure-detection hook of the batched kernel.  spin_limit bounds the
 * dependency wait of a y item (iterations of ~0.25 us; 0 restores the
 * default, about one second); never_ready_shot >= 0 makes that shot's wait
 * target unreachable, so its y items time out: the kernel still finishes,
 * skips those items and adi_wave_sync_status() returns ADI_ETIMEOUT.  -1
 * disables it. */
int adi_wave_set_wait_hook(adi_wave *h, int64_t spin_limit, int32_t never_ready_shot);

/* Number of kernel launches the handle has enqueued since creation (all
 * kinds, graph replays counted per kernel node). */
int64_t adi_wave_launch_count(const adi_wave *h);

/* ---- problem class and scheme ----------------------------------------------
 * Section 2 states the problem with a coefficient c(t) that depends on time
 * (Eq. f1) and a general source f(t, x, y), and splits Eq. (CN1) into the two
 * sub-problems of Eqs. (fr1) and (fr2) over half time levels; Listing 1 sets
 * up the tridiagonal systems of a fully implicit form of them.  By default a
 * handle solves the factored delta form of Eq. (CN1) with a time-independent
 * coefficient m(x, y) and a point source (the form the benchmark workloads
 * use).  adi_wave_set_model selects, for a single-grid handle:
 *   ADI_SCHEME_FACTORED with g and/or f: Eq. (CN1) with the coefficient
 *     m^k = g[k] m(x, y) at level k (levels past the end of g keep its last
 *     value; g = NULL means 1) and a source field f^k (f = NULL means 0,
 *     levels past n_f are 0) added to the point source.  CN1 weighs
 *     Lap u^{k+1} by m^{k+1}/2 and Lap u^{k-1} by m^{k-1}/2, so a step solves
 *     (I - S Lap) z = tau^2 (g_{k+1} m Lap u^k
 *                            + (g_{k-1} - g_{k+1})/2 m Lap u^{k-1} + f^k),
 *     S = tau^2 g_{k+1} m / 2, factored into an x and a y sweep as before.
 *   ADI_SCHEME_HALF_LEVELS: Eqs. (fr1) and (fr2) as printed, over half time
 *     levels: (I - S Lap_x) u^{k+1/2} = 2u^k - u^{k-1/2} + S Lap_x u^{k-1/2}
 *     + tau^2 f^k, then (I - S Lap_y) u^{k+1} = 2u^{k+1/2} - u^k + S Lap_y u^k
 *     + tau^2 f^{k+1/2}, S = tau^2 m / 2 (Algorithm 1's buffers u, U0, Ux,
 *     Uy and its swaps).  The state reported by adi_wave_get_state is
 *     (u^{k-1/2}, u^k); the start-up's (u^0, u^1) is taken as (u^{1/2}, u^1)
 *     (with psi = 0 both equal phi, as Algorithm 1 starts).  This scheme
 *     moves the waves too fast (by about sqrt 2).
 *   ADI_SCHEME_LISTING1: the same half levels with Listing 1's systems
 *     (a = c = tau^2 m, b = 2 tau^2 m + h^2, right-hand side from u^{k-1/2}
 *     and u^k only): (I - tau^2 m Lap_x) u^{k+1/2} = 2u^k - u^{k-1/2}
 *     + tau^2 f^k and the same along y; it damps every mode.
 * The half-level schemes take no g or f (ADI_EINVAL); their point source at
 * level k + 1/2 is the mean of the samples k and k + 1.  g and f are device
 * arrays borrowed until the handle's last step that reads them; f is
 * [n_f][ny][nx] FP32, contiguous.  With any non-default model the steps run
 * as direct launches of one-shot kernels (no TMA pipeline, no graphs) with
 * FP32 elimination, and adi_wave_adjoint returns ADI_EUNSUPPORTED.  Batched
 * handles: ADI_EUNSUPPORTED.  Passing the default model restores the default
 * path. */
enum { ADI_SCHEME_FACTORED = 0, ADI_SCHEME_HALF_LEVELS = 1, ADI_SCHEME_LISTING1 = 2 };
typedef struct {
    int32_t scheme;   /* ADI_SCHEME_* */
    const float *g;   /* device [n_g] or NULL */
    int32_t n_g;
    const float *f;   /* device [n_f][ny][nx] or NULL */
    int32_t n_f;
} adi_wave_model;
int adi_wave_set_model(adi_wave *h, const adi_wave_model *model);

/* ---- one step without allocation ------------------------------------------
 * The paper has no counterpart of this call: it is a library convenience.
 *
 * One time step of the factored scheme (the same x and y sweep kernels as
 * adi_wave_step, with the plan a new handle would choose) on buffers the
 * caller owns, with no handle and no device memory allocated by the call
 * or by anything it calls.  It is meant for callers that cannot allocate
 * while they step: code whose device memory is already handed out to its
 * own pool, or a time loop that must not meet the device-wide
 * synchronisation cudaFree implies or the latency of cudaMalloc.
 *
 * The x sweep's result w, the one intermediate field of a step, lives in a
 * static device array of 4,194,304 floats (16 MiB) that the library sets
 * aside when its module loads, so grids are limited to ld * ny <= 4194304
 * (for example 2048 x 2048); larger grids get ADI_EINVAL and a message
 * from adi_wave_last_error(NULL).  The array needs no initial value.
 *
 *   desc    host pointer; nx, ny, lx, ly, dt, fp64_solve as for
 *           adi_wave_init (start is ignored).
 *   ld      row pitch in floats of m, u_cur and u_prev: a multiple of 32,
 *           >= nx.  Unlike the rest of this ABI these fields are PITCHED,
 *           [ny][ld], and their padding columns nx..ld-1 must hold zeros
 *           (the sweeps read them as the Dirichlet ring's values).
 *   m_max   the largest value of m; picks FP32 or FP64 elimination as
 *           ADI_FP64_AUTO does (it must be > 0).
 *   m       device [ny][ld] coefficient m = c^2 > 0.
 *   u_cur   device [ny][ld] u^k, read only.
 *   u_prev  device [ny][ld] u^{k-1} on entry, u^{k+1} on completion.
 *   src     host pointer to the point source or NULL; wavelet[k] is used.
 *   k       time level of u_cur (>= 0).
 * Buffers must be 16-byte aligned and u_cur != u_prev.  This call reports
 * no condition found on the GPU: non-finite values and an expired bounded
 * wait inside the sweep kernels go unreported (the handle API reports both
 * through adi_wave_sync_status).
 *
 * The first call on a device does a one-time set-up with that device
 * current: it looks up the static array's address (cudaGetSymbolAddress)
 * and sets kernel attributes.  Make that first call before any stream
 * capture.  The static array is shared by all calls on a device and keeps
 * the last call's contents: two calls whose work overlaps in time
 * (different streams without an event between them, or several host
 * threads) race on it and give wrong results.  Order them on one stream. */
int adi_wave_step_noalloc(const adi_wave_desc *desc, int32_t ld, double m_max,
                          const float *m, const float *u_cur, float *u_prev,
                          const adi_source *src, int64_t k, void *stream);

/* Library version string, e.g. "adiwave 0.1 sm_103a". */
const char *adi_wave_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADIWAVE_H */
