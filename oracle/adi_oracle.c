/*
 * adi_oracle.c -- plain FP64 CPU oracle for the factored ADI scheme of the
 * 2D acoustic wave equation (Altybay, Ruzhansky, Tokmagambetov,
 * "A parallel hybrid implementation of the 2D acoustic wave equation").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA library; both sides only receive the same seeded
 * inputs.
 *
 * Every routine is a direct, unblocked transcription of a definition:
 *   - grid and unknowns: Section 2, Eq. (f6) -- interior nodes only, the
 *     Dirichlet ring of Eq. (CN3) is implicit zero and never stored;
 *     array element [j*nx + i] is the node (x_{i+1}, y_{j+1}), x fastest.
 *   - the scheme: Eq. (CN1) with a time-independent coefficient m = c^2
 *     multiplying the Laplacian (the non-divergence form m * Lap u of
 *     Eq. (f1)).  Writing z = u^{k+1} - 2u^k + u^{k-1}, Eq. (CN1) is exactly
 *         (I - S Lap) z = tau^2 (m Lap u^k + f^k),   S = diag(tau^2 m / 2);
 *     the ADI method of Section 2 (the two sub-problems solved "in the x
 *     direction" then "in the y direction", Section 4) factors
 *     I - S Lap ~= (I - S Lap_x)(I - S Lap_y) and solves
 *         X w = r   (one tridiagonal system per row, Eq. fr1's x operator)
 *         Y z = w   (one tridiagonal system per column, Eq. fr2's y operator)
 *         u^{k+1} = 2 u^k - u^{k-1} + z.
 *   - start-up: Eq. (CN2), u^0 = phi, u^1 = phi + tau psi, and optionally
 *     the second-order Taylor start u^1 = phi + tau psi + tau^2/2 (m Lap phi + f^0).
 *   - point source: a delta-like source approximated by a grid function
 *     (Section 2, the very-weak-solution remark): f^k = w(t_k) / (h1 h2) at
 *     one node, zero elsewhere.
 *   - each tridiagonal system is solved by the Thomas algorithm (Gaussian
 *     elimination without pivoting), the textbook serial method the paper's
 *     cyclic reduction parallelises; the systems are strictly diagonally
 *     dominant so the solution is unique and pivoting is not needed.
 *   - the adjoint (reverse-mode derivative of the receiver misfit) is the
 *     transpose of each step above taken in reverse order; it is not in the
 *     paper and is derived from the scheme in the project's design notes.
 *
 * Threads: lines within one sweep are independent, so the line loops carry
 * an OpenMP "parallel for" with a caller-chosen thread count (1 = serial).
 */
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, nx) ((size_t)(j) * (size_t)(nx) + (size_t)(i))

/* Thomas algorithm for a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,
 * i = 0..n-1, a_0 and c_{n-1} ignored (the neighbours outside are the zero
 * Dirichlet values).  Workspace cp, dp of length n.  Returns 0, or 1 if a
 * pivot is exactly zero. */
static int thomas_ws(int n, const double *a, const double *b, const double *c,
                     const double *d, double *x, double *cp, double *dp)
{
    if (n <= 0) return 0;
    if (b[0] == 0.0) return 1;
    cp[0] = (n > 1 ? c[0] : 0.0) / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; ++i) {
        double den = b[i] - a[i] * cp[i - 1];
        if (den == 0.0) return 1;
        cp[i] = (i < n - 1 ? c[i] : 0.0) / den;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    return 0;
}

int oracle_thomas(int n, const double *a, const double *b, const double *c,
                  const double *d, double *x)
{
    if (n <= 0) return 0;
    double *cp = (double *)malloc(sizeof(double) * (size_t)n);
    double *dp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!cp || !dp) { free(cp); free(dp); return 2; }
    int rc = thomas_ws(n, a, b, c, d, x, cp, dp);
    free(cp); free(dp);
    return rc;
}

/* Five-point discrete Laplacian with zero Dirichlet ring, Eq. (CN1)'s
 * spatial operator: (u_{i+1,j} - 2u_{i,j} + u_{i-1,j})/h1^2 +
 * (u_{i,j+1} - 2u_{i,j} + u_{i,j-1})/h2^2. */
static double lap_x_at(const double *u, int nx, int i, int j, double hx)
{
    double c = u[IDX(i, j, nx)];
    double l = (i > 0) ? u[IDX(i - 1, j, nx)] : 0.0;
    double r = (i < nx - 1) ? u[IDX(i + 1, j, nx)] : 0.0;
    return (l - 2.0 * c + r) / (hx * hx);
}

static double lap_y_at(const double *u, int nx, int ny, int i, int j, double hy)
{
    double c = u[IDX(i, j, nx)];
    double d = (j > 0) ? u[IDX(i, j - 1, nx)] : 0.0;
    double t = (j < ny - 1) ? u[IDX(i, j + 1, nx)] : 0.0;
    return (d - 2.0 * c + t) / (hy * hy);
}

void oracle_laplacian(int nx, int ny, double hx, double hy, const double *u,
                      double *out)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            out[IDX(i, j, nx)] = lap_x_at(u, nx, i, j, hx) + lap_y_at(u, nx, ny, i, j, hy);
}

/* RHS of the delta form of Eq. (CN1): r = tau^2 (m Lap u^k + f^k), with the
 * point source f^k = wv / (h1 h2) at (sx, sy) when sx >= 0. */
static void rhs(int nx, int ny, double hx, double hy, double tau,
                const double *m, const double *u, double wv, int sx, int sy,
                double *r, int threads)
{
    (void)threads;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double lap = lap_x_at(u, nx, i, j, hx) + lap_y_at(u, nx, ny, i, j, hy);
            double f = (i == sx && j == sy) ? wv / (hx * hy) : 0.0;
            r[IDX(i, j, nx)] = tau * tau * (m[IDX(i, j, nx)] * lap + f);
        }
}

/* x sweep, Eq. (fr1)'s operator: for every row j solve
 * (I - S Lap_x) w = r, i.e. -s_i w_{i-1} + (1 + 2 s_i) w_i - s_i w_{i+1} = r_i
 * with s_i = tau^2 m_{ij} / (2 h1^2). */
static int sweep_x(int nx, int ny, double hx, double tau, const double *m,
                   const double *r, double *w, int threads)
{
    int bad = 0;
    (void)threads;
#pragma omp parallel num_threads(threads) reduction(| : bad)
    {
        double *a = (double *)malloc(sizeof(double) * (size_t)nx * 6);
        if (!a) { bad |= 2; } else {
            double *b = a + nx, *c = b + nx, *d = c + nx, *cp = d + nx, *dp = cp + nx;
#pragma omp for schedule(static)
            for (int j = 0; j < ny; ++j) {
                for (int i = 0; i < nx; ++i) {
                    double s = tau * tau * m[IDX(i, j, nx)] / (2.0 * hx * hx);
                    a[i] = -s; b[i] = 1.0 + 2.0 * s; c[i] = -s;
                    d[i] = r[IDX(i, j, nx)];
                }
                bad |= thomas_ws(nx, a, b, c, d, w + IDX(0, j, nx), cp, dp);
            }
            free(a);
        }
    }
    return bad;
}

/* y sweep, Eq. (fr2)'s operator: for every column i solve
 * (I - S Lap_y) z = w along j with s_j = tau^2 m_{ij} / (2 h2^2). */
static int sweep_y(int nx, int ny, double hy, double tau, const double *m,
                   const double *w, double *z, int threads)
{
    int bad = 0;
    (void)threads;
#pragma omp parallel num_threads(threads) reduction(| : bad)
    {
        double *a = (double *)malloc(sizeof(double) * (size_t)ny * 7);
        if (!a) { bad |= 2; } else {
            double *b = a + ny, *c = b + ny, *d = c + ny, *x = d + ny, *cp = x + ny, *dp = cp + ny;
#pragma omp for schedule(static)
            for (int i = 0; i < nx; ++i) {
                for (int j = 0; j < ny; ++j) {
                    double s = tau * tau * m[IDX(i, j, nx)] / (2.0 * hy * hy);
                    a[j] = -s; b[j] = 1.0 + 2.0 * s; c[j] = -s;
                    d[j] = w[IDX(i, j, nx)];
                }
                bad |= thomas_ws(ny, a, b, c, d, x, cp, dp);
                for (int j = 0; j < ny; ++j) z[IDX(i, j, nx)] = x[j];
            }
            free(a);
        }
    }
    return bad;
}

/* One factored-ADI step (Eq. CN1 in delta form, split as Eqs. fr1/fr2):
 * from u^{k-1} (u_prev) and u^k (u_cur) compute u^{k+1} (u_next).  Optional
 * outputs: r (RHS), w (x-sweep result), z (y-sweep result).  Returns 0 on
 * success. */
int oracle_adi_step(int nx, int ny, double hx, double hy, double tau,
                    const double *m, const double *u_prev, const double *u_cur,
                    double wv, int sx, int sy, double *u_next,
                    double *r_out, double *w_out, double *z_out, int threads)
{
    size_t N = (size_t)nx * (size_t)ny;
    double *r = r_out ? r_out : (double *)malloc(sizeof(double) * N);
    double *w = w_out ? w_out : (double *)malloc(sizeof(double) * N);
    double *z = z_out ? z_out : (double *)malloc(sizeof(double) * N);
    int rc = 0;
    if (!r || !w || !z) { rc = 2; goto done; }
    rhs(nx, ny, hx, hy, tau, m, u_cur, wv, sx, sy, r, threads);
    rc |= sweep_x(nx, ny, hx, tau, m, r, w, threads);
    rc |= sweep_y(nx, ny, hy, tau, m, w, z, threads);
    for (size_t p = 0; p < N; ++p) u_next[p] = 2.0 * u_cur[p] - u_prev[p] + z[p];
done:
    if (!r_out) free(r);
    if (!w_out) free(w);
    if (!z_out) free(z);
    return rc;
}

/* Start-up, Eq. (CN2): u^0 = phi, u^1 = phi + tau psi.  With taylor != 0 the
 * second-order start adds tau^2/2 (m Lap phi + f^0).  psi may be NULL (= 0). */
int oracle_adi_init(int nx, int ny, double hx, double hy, double tau,
                    const double *m, const double *phi, const double *psi,
                    int taylor, double wv0, int sx, int sy,
                    double *u0, double *u1)
{
    size_t N = (size_t)nx * (size_t)ny;
    for (size_t p = 0; p < N; ++p) {
        u0[p] = phi[p];
        u1[p] = phi[p] + (psi ? tau * psi[p] : 0.0);
    }
    if (taylor) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double lap = lap_x_at(phi, nx, i, j, hx) + lap_y_at(phi, nx, ny, i, j, hy);
                double f = (i == sx && j == sy) ? wv0 / (hx * hy) : 0.0;
                u1[IDX(i, j, nx)] += 0.5 * tau * tau * (m[IDX(i, j, nx)] * lap + f);
            }
    }
    return 0;
}

/* The time loop of Algorithm 1: `steps` factored-ADI steps starting from the
 * time level k0 (u_prev = u^{k0-1}, u_cur = u^{k0}).  The step that leaves
 * level k uses the source sample wavelet[k] (0 when k >= n_wavelet or sx < 0).
 * After step s the receivers sample the new field:
 * traces[s*n_rec + r] = u^{k0+s+1}(rec r).  On return u_prev/u_cur hold
 * u^{k0+steps-1} and u^{k0+steps}. */
int oracle_adi_run(int nx, int ny, double hx, double hy, double tau,
                   const double *m, double *u_prev, double *u_cur, long k0,
                   int steps, int sx, int sy, const double *wavelet,
                   int n_wavelet, const int *rec_ix, const int *rec_iy,
                   int n_rec, double *traces, int threads)
{
    size_t N = (size_t)nx * (size_t)ny;
    double *nxt = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *w = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N);
    int rc = 0;
    if (!nxt || !r || !w || !z) { rc = 2; goto done; }
    for (int s = 0; s < steps; ++s) {
        long k = k0 + s;
        double wv = (sx >= 0 && wavelet && k >= 0 && k < n_wavelet) ? wavelet[k] : 0.0;
        rc |= oracle_adi_step(nx, ny, hx, hy, tau, m, u_prev, u_cur, wv, sx, sy,
                              nxt, r, w, z, threads);
        if (rc) break;
        for (int q = 0; q < n_rec; ++q)
            traces[(size_t)s * n_rec + q] = nxt[IDX(rec_ix[q], rec_iy[q], nx)];
        memcpy(u_prev, u_cur, sizeof(double) * N);
        memcpy(u_cur, nxt, sizeof(double) * N);
    }
done:
    free(nxt); free(r); free(w); free(z);
    return rc;
}

/* Transposed sweeps.  For X = I - S Lap_x the transpose is I - Lap_x S:
 * row i of X^T reads -s_{i-1} x_{i-1} + (1 + 2 s_i) x_i - s_{i+1} x_{i+1}. */
static int sweep_x_T(int nx, int ny, double hx, double tau, const double *m,
                     const double *rhs_, double *out, int threads)
{
    int bad = 0;
    (void)threads;
#pragma omp parallel num_threads(threads) reduction(| : bad)
    {
        double *a = (double *)malloc(sizeof(double) * (size_t)nx * 6);
        if (!a) { bad |= 2; } else {
            double *b = a + nx, *c = b + nx, *d = c + nx, *cp = d + nx, *dp = cp + nx;
#pragma omp for schedule(static)
            for (int j = 0; j < ny; ++j) {
                for (int i = 0; i < nx; ++i) {
                    double k2 = tau * tau / (2.0 * hx * hx);
                    a[i] = (i > 0) ? -k2 * m[IDX(i - 1, j, nx)] : 0.0;
                    b[i] = 1.0 + 2.0 * k2 * m[IDX(i, j, nx)];
                    c[i] = (i < nx - 1) ? -k2 * m[IDX(i + 1, j, nx)] : 0.0;
                    d[i] = rhs_[IDX(i, j, nx)];
                }
                bad |= thomas_ws(nx, a, b, c, d, out + IDX(0, j, nx), cp, dp);
            }
            free(a);
        }
    }
    return bad;
}

static int sweep_y_T(int nx, int ny, double hy, double tau, const double *m,
                     const double *rhs_, double *out, int threads)
{
    int bad = 0;
    (void)threads;
#pragma omp parallel num_threads(threads) reduction(| : bad)
    {
        double *a = (double *)malloc(sizeof(double) * (size_t)ny * 7);
        if (!a) { bad |= 2; } else {
            double *b = a + ny, *c = b + ny, *d = c + ny, *x = d + ny, *cp = x + ny, *dp = cp + ny;
#pragma omp for schedule(static)
            for (int i = 0; i < nx; ++i) {
                for (int j = 0; j < ny; ++j) {
                    double k2 = tau * tau / (2.0 * hy * hy);
                    a[j] = (j > 0) ? -k2 * m[IDX(i, j - 1, nx)] : 0.0;
                    b[j] = 1.0 + 2.0 * k2 * m[IDX(i, j, nx)];
                    c[j] = (j < ny - 1) ? -k2 * m[IDX(i, j + 1, nx)] : 0.0;
                    d[j] = rhs_[IDX(i, j, nx)];
                }
                bad |= thomas_ws(ny, a, b, c, d, x, cp, dp);
                for (int j = 0; j < ny; ++j) out[IDX(i, j, nx)] = x[j];
            }
            free(a);
        }
    }
    return bad;
}

/* One sweep on its own (for tests of the operators): dir 0 solves along the
 * rows (X, spacing h = h1), dir 1 along the columns (Y, h = h2); with
 * transposed != 0 the transposed operator X^T or Y^T.  out = Op^{-1} rhs. */
int oracle_line_sweep(int dir, int transposed, int nx, int ny, double h, double tau,
                      const double *m, const double *rhs, double *out, int threads)
{
    if (dir == 0)
        return transposed ? sweep_x_T(nx, ny, h, tau, m, rhs, out, threads)
                          : sweep_x(nx, ny, h, tau, m, rhs, out, threads);
    return transposed ? sweep_y_T(nx, ny, h, tau, m, rhs, out, threads)
                      : sweep_y(nx, ny, h, tau, m, rhs, out, threads);
}

/* Reverse-mode derivative of J = 1/2 sum_s sum_r (traces[s][r] - d[s][r])^2
 * for the run oracle_adi_run(k0, steps, ...) would make from (u_prev0,
 * u_cur0).  resid[s*n_rec + r] = traces[s][r] - d[s][r] (= dJ/dtraces).
 * Outputs: grad_m[nx*ny] = dJ/dm (m = c^2), grad_wavelet[n_wavelet] =
 * dJ/dwavelet (nullable), lam_cur/lam_prev = dJ/du^{k0}, dJ/du^{k0-1}
 * (nullable).  taylor_k0 != 0 states that u^{k0} was produced by the Taylor
 * start from u^{k0-1} = phi (so the start-up's dependence on m and f^{k0-1}
 * is included).
 *
 * Forward, per level k: r = tau^2 (m Lap u^k + f^k), X w = r, Y z = w,
 * u^{k+1} = 2u^k - u^{k-1} + z.  Reverse, with lam^j = dJ/du^j accumulated
 * from later levels and the receiver residuals:
 *   zbar = lam^{k+1};  Y^T wbar = zbar;  X^T rbar = wbar;
 *   dJ/dm += (tau^2/2) (wbar . Lap_y z + rbar . Lap_x w) + tau^2 rbar . Lap u^k
 *   lam^k += 2 zbar + tau^2 Lap(m . rbar);  lam^{k-1} -= zbar;
 *   dJ/dwavelet[k] += tau^2 rbar_src / (h1 h2).
 * All forward fields are stored (the oracle runs on small grids). */
int oracle_adi_adjoint(int nx, int ny, double hx, double hy, double tau,
                       const double *m, const double *u_prev0,
                       const double *u_cur0, long k0, int steps, int sx, int sy,
                       const double *wavelet, int n_wavelet, const int *rec_ix,
                       const int *rec_iy, int n_rec, const double *resid,
                       int taylor_k0, double *grad_m, double *grad_wavelet,
                       double *lam_cur_out, double *lam_prev_out, int threads)
{
    size_t N = (size_t)nx * (size_t)ny;
    int rc = 0;
    double *U = (double *)malloc(sizeof(double) * N * (size_t)(steps + 2));
    double *r = (double *)malloc(sizeof(double) * N);
    double *w = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N);
    double *wbar = (double *)malloc(sizeof(double) * N);
    double *rbar = (double *)malloc(sizeof(double) * N);
    double *mr = (double *)malloc(sizeof(double) * N);
    double *lap = (double *)malloc(sizeof(double) * N);
    double *L0 = (double *)calloc(N, sizeof(double));
    double *L1 = (double *)calloc(N, sizeof(double));
    double *L2 = (double *)calloc(N, sizeof(double));
    if (!U || !r || !w || !z || !wbar || !rbar || !mr || !lap || !L0 || !L1 || !L2) { rc = 2; goto done; }

    memcpy(U, u_prev0, sizeof(double) * N);
    memcpy(U + N, u_cur0, sizeof(double) * N);
    for (int s = 0; s < steps; ++s) {
        long k = k0 + s;
        double wv = (sx >= 0 && wavelet && k >= 0 && k < n_wavelet) ? wavelet[k] : 0.0;
        rc |= oracle_adi_step(nx, ny, hx, hy, tau, m, U + N * (size_t)s, U + N * (size_t)(s + 1),
                              wv, sx, sy, U + N * (size_t)(s + 2), r, w, z, threads);
        if (rc) goto done;
    }

    memset(grad_m, 0, sizeof(double) * N);
    if (grad_wavelet) memset(grad_wavelet, 0, sizeof(double) * (size_t)(n_wavelet > 0 ? n_wavelet : 0));

    /* lam_next = lam^{k+1}, lam_cur = lam^k, lam_prev = lam^{k-1} */
    double *lam_next = L0, *lam_cur = L1, *lam_prev = L2;
    for (int s = steps - 1; s >= 0; --s) {
        long k = k0 + s;
        const double *uk = U + N * (size_t)(s + 1);
        for (int q = 0; q < n_rec; ++q)
            lam_next[IDX(rec_ix[q], rec_iy[q], nx)] += resid[(size_t)s * n_rec + q];
        double wv = (sx >= 0 && wavelet && k >= 0 && k < n_wavelet) ? wavelet[k] : 0.0;
        /* recompute r, w, z of this step */
        rhs(nx, ny, hx, hy, tau, m, uk, wv, sx, sy, r, threads);
        rc |= sweep_x(nx, ny, hx, tau, m, r, w, threads);
        rc |= sweep_y(nx, ny, hy, tau, m, w, z, threads);
        /* zbar = lam_next */
        rc |= sweep_y_T(nx, ny, hy, tau, m, lam_next, wbar, threads);
        rc |= sweep_x_T(nx, ny, hx, tau, m, wbar, rbar, threads);
        if (rc) goto done;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = IDX(i, j, nx);
                double lyz = lap_y_at(z, nx, ny, i, j, hy);
                double lxw = lap_x_at(w, nx, i, j, hx);
                double lu = lap_x_at(uk, nx, i, j, hx) + lap_y_at(uk, nx, ny, i, j, hy);
                grad_m[p] += 0.5 * tau * tau * (wbar[p] * lyz + rbar[p] * lxw) + tau * tau * rbar[p] * lu;
                mr[p] = m[p] * rbar[p];
            }
        if (grad_wavelet && sx >= 0 && k >= 0 && k < n_wavelet)
            grad_wavelet[k] += tau * tau * rbar[IDX(sx, sy, nx)] / (hx * hy);
        oracle_laplacian(nx, ny, hx, hy, mr, lap);
        for (size_t p = 0; p < N; ++p) {
            lam_cur[p] += 2.0 * lam_next[p] + tau * tau * lap[p];
            lam_prev[p] -= lam_next[p];
        }
        /* rotate: level k+1 is finished */
        double *t = lam_next;
        lam_next = lam_cur; lam_cur = lam_prev; lam_prev = t;
        memset(lam_prev, 0, sizeof(double) * N);
    }
    /* now lam_next = dJ/du^{k0}, lam_cur = dJ/du^{k0-1} */
    if (taylor_k0) {
        /* u^{k0} = phi + tau psi + tau^2/2 (m Lap phi + f^{k0-1}), phi = u^{k0-1} */
        oracle_laplacian(nx, ny, hx, hy, u_prev0, lap);
        for (size_t p = 0; p < N; ++p) grad_m[p] += 0.5 * tau * tau * lam_next[p] * lap[p];
        long k = k0 - 1;
        if (grad_wavelet && sx >= 0 && k >= 0 && k < n_wavelet)
            grad_wavelet[k] += 0.5 * tau * tau * lam_next[IDX(sx, sy, nx)] / (hx * hy);
    }
    if (lam_cur_out) memcpy(lam_cur_out, lam_next, sizeof(double) * N);
    if (lam_prev_out) memcpy(lam_prev_out, lam_cur, sizeof(double) * N);
done:
    free(U); free(r); free(w); free(z); free(wbar); free(rbar); free(mr); free(lap);
    free(L0); free(L1); free(L2);
    return rc;
}

int oracle_num_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Wider problem class and the paper's literal sub-schemes.
 * ------------------------------------------------------------------------ */

/* Solve (I - kfac m Lap_dir) x = rhs along every line of direction dir
 * (0: rows, spacing h1; 1: columns, spacing h2), i.e.
 * -s_i x_{i-1} + (1 + 2 s_i) x_i - s_i x_{i+1} = rhs_i, s_i = kfac m_i / h^2. */
static int sweep_coef(int dir, int nx, int ny, double h, double kfac, const double *m,
                      const double *rhs_, double *out, int threads)
{
    int bad = 0;
    int len = dir == 0 ? nx : ny;
    int lines = dir == 0 ? ny : nx;
    (void)threads;
#pragma omp parallel num_threads(threads) reduction(| : bad)
    {
        double *a = (double *)malloc(sizeof(double) * (size_t)len * 7);
        if (!a) { bad |= 2; } else {
            double *b = a + len, *c = b + len, *d = c + len, *x = d + len, *cp = x + len, *dp = cp + len;
#pragma omp for schedule(static)
            for (int l = 0; l < lines; ++l) {
                for (int t = 0; t < len; ++t) {
                    size_t p = dir == 0 ? IDX(t, l, nx) : IDX(l, t, nx);
                    double s = kfac * m[p] / (h * h);
                    a[t] = -s; b[t] = 1.0 + 2.0 * s; c[t] = -s;
                    d[t] = rhs_[p];
                }
                bad |= thomas_ws(len, a, b, c, d, x, cp, dp);
                for (int t = 0; t < len; ++t) {
                    size_t p = dir == 0 ? IDX(t, l, nx) : IDX(l, t, nx);
                    out[p] = x[t];
                }
            }
            free(a);
        }
    }
    return bad;
}

/* One step of Eq. (CN1) with a time-dependent coefficient and a source
 * field.  The coefficient of the Laplacian at level k is m^k = g_k m(x, y)
 * (the paper's c(t) of Eq. f1 times the workloads' c^2(x, y)); CN1 weighs
 * Lap u^{k+1} by m^{k+1}/2 and Lap u^{k-1} by m^{k-1}/2.  With
 * z = u^{k+1} - 2u^k + u^{k-1} it reads exactly
 *   (I - S Lap) z = tau^2 (g_{k+1} m Lap u^k
 *                          + (g_{k-1} - g_{k+1})/2 m Lap u^{k-1} + f^k),
 *   S = tau^2 g_{k+1} m / 2,
 * and the ADI method factors I - S Lap into (I - S Lap_x)(I - S Lap_y) as in
 * oracle_adi_step.  f^k = fk (a field, nullable) + wv / (h1 h2) at (sx, sy). */
int oracle_adi_step_gen(int nx, int ny, double hx, double hy, double tau,
                        const double *m, double g_prev, double g_next,
                        const double *u_prev, const double *u_cur, const double *fk,
                        double wv, int sx, int sy, double *u_next, int threads)
{
    size_t N = (size_t)nx * (size_t)ny;
    double *r = (double *)malloc(sizeof(double) * N);
    double *w = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N);
    int rc = 0;
    if (!r || !w || !z) { rc = 2; goto done; }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t p = IDX(i, j, nx);
            double lc = lap_x_at(u_cur, nx, i, j, hx) + lap_y_at(u_cur, nx, ny, i, j, hy);
            double lp = lap_x_at(u_prev, nx, i, j, hx) + lap_y_at(u_prev, nx, ny, i, j, hy);
            double f = (fk ? fk[p] : 0.0) + ((i == sx && j == sy) ? wv / (hx * hy) : 0.0);
            r[p] = tau * tau * (g_next * m[p] * lc + 0.5 * (g_prev - g_next) * m[p] * lp + f);
        }
    rc |= sweep_coef(0, nx, ny, hx, 0.5 * tau * tau * g_next, m, r, w, threads);
    rc |= sweep_coef(1, nx, ny, hy, 0.5 * tau * tau * g_next, m, w, z, threads);
    for (size_t p = 0; p < N; ++p) u_next[p] = 2.0 * u_cur[p] - u_prev[p] + z[p];
done:
    free(r); free(w); free(z);
    return rc;
}

/* The two sub-problems of Section 2 taken literally, over half time levels
 * (Algorithm 1: u, U0, Ux, Uy = u^{k-1/2}, u^k, u^{k+1/2}, u^{k+1}; after the
 * step swap(u, Ux), swap(U0, Uy)).  Coefficient m (time-independent).
 * variant 1, Eqs. fr1 and fr2 (S = tau^2 m / 2):
 *   (I - S Lap_x) u^{k+1/2} = 2u^k - u^{k-1/2} + S Lap_x u^{k-1/2} + tau^2 f^k
 *   (I - S Lap_y) u^{k+1}   = 2u^{k+1/2} - u^k + S Lap_y u^k + tau^2 f^{k+1/2}
 * variant 2, the tridiagonal systems of Listing 1 (a = c = tau^2 m,
 * b = 2 tau^2 m + h^2, right-hand side h^2 (u_old - 2 u^k) in the
 * convention a y_{i-1} - b y_i + c y_{i+1} = f), the fully implicit form:
 *   (I - tau^2 m Lap_x) u^{k+1/2} = 2u^k - u^{k-1/2} + tau^2 f^k
 *   (I - tau^2 m Lap_y) u^{k+1}   = 2u^{k+1/2} - u^k + tau^2 f^{k+1/2}
 * f^k = wv_k / (h1 h2), f^{k+1/2} = wv_half / (h1 h2) at (sx, sy) (the caller
 * passes the half-level sample).  Outputs u_half = u^{k+1/2}, u_next = u^{k+1}. */
int oracle_adi_step_halves(int variant, int nx, int ny, double hx, double hy, double tau,
                           const double *m, const double *u_half_prev, const double *u_cur,
                           double wv_k, double wv_half, int sx, int sy,
                           double *u_half, double *u_next, int threads)
{
    if (variant != 1 && variant != 2) return 3;
    size_t N = (size_t)nx * (size_t)ny;
    double *r = (double *)malloc(sizeof(double) * N);
    int rc = 0;
    if (!r) return 2;
    double kfac = variant == 1 ? 0.5 * tau * tau : tau * tau;
    double alpha = variant == 1 ? 1.0 : 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t p = IDX(i, j, nx);
            double S = 0.5 * tau * tau * m[p];
            double f = (i == sx && j == sy) ? wv_k / (hx * hy) : 0.0;
            r[p] = 2.0 * u_cur[p] - u_half_prev[p] + alpha * S * lap_x_at(u_half_prev, nx, i, j, hx)
                   + tau * tau * f;
        }
    rc |= sweep_coef(0, nx, ny, hx, kfac, m, r, u_half, threads);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t p = IDX(i, j, nx);
            double S = 0.5 * tau * tau * m[p];
            double f = (i == sx && j == sy) ? wv_half / (hx * hy) : 0.0;
            r[p] = 2.0 * u_half[p] - u_cur[p] + alpha * S * lap_y_at(u_cur, nx, ny, i, j, hy)
                   + tau * tau * f;
        }
    rc |= sweep_coef(1, nx, ny, hy, kfac, m, r, u_next, threads);
    free(r);
    return rc;
}
