/*
 * sigk_oracle.c -- plain FP64 CPU oracle for the signature kernel of
 * piecewise-linear paths.  TEST INFRASTRUCTURE ONLY: only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Three independent computations of k(x,y) = K(1,1), where K solves the
 * Goursat problem of Sec. 2.1 (Definition "Signature Kernel"):
 *
 *   orc_series_pair  -- the tile-centred local power series of Sec. 2.3
 *                       (Proposition "tile-centred expansion", proof in
 *                       App. A.6), truncated to (N+1)x(N+1) coefficient
 *                       matrices as in App. A.7, swept over anti-diagonals as
 *                       in the algorithm of App. C.1.  With N ~ 24 the
 *                       truncation error is far below FP64 rounding for the
 *                       inputs used here.
 *   orc_fd_pair      -- finite-difference Goursat scheme on a dyadically
 *                       refined grid, derived from the Volterra form of
 *                       Sec. 2.1 (trapezoid rule on each cell), plus
 *                       Richardson extrapolation in h^2.
 *   orc_chen_pair    -- the signature inner product sum_n <S^n(x), S^n(y)>
 *                       (the definition the Goursat PDE characterises, Sec.
 *                       2.1 footnote), with S(x) = exp(dx_1) (x) ... (x)
 *                       exp(dx_L) by Chen's identity, truncated at level M.
 *                       Brute force: only for tiny d^M.
 *
 * Conventions (unit local tiles): x has L1 segments with increments dx[i]
 * (row-major L1 x d), y has L2 segments dy[j].  Tile (i,j) couples x-segment i
 * (the s direction) with y-segment j (the t direction); its coefficient is
 * c_ij = <dx_i, dy_j>.  The paper writes the same problem on [0,1]^2 with the
 * density (l-1)^2 <dx, dy> and tile width 1/(l-1); rescaling every tile to the
 * unit square turns that density times the tile area into c_ij and leaves
 * K(1,1) unchanged (the kernel is invariant under reparametrisation), which
 * also covers unequal lengths without the padding of Sec. 2.1.
 *
 * All functions return 0 on success, -1 on bad arguments, -2 on allocation
 * failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static double dot_d(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int e = 0; e < d; ++e) s += a[e] * b[e];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Tile-centred expansion (Sec. 2.3).                                        */
/* ------------------------------------------------------------------------ */

/* One tile of the tile-centred expansion with truncation order N.
 *
 * Inputs: rho = c_ij; alpha[0..N] = bottom-edge series kappa(s, tau_l) in
 * powers of the local s; beta[0..N] = left-edge series kappa(sigma_k, t) in
 * powers of the local t.
 *
 * The coefficient matrix is Ct = A (.) B (.) W with
 *   A_ij = rho^min(i,j),
 *   W_ij = (max(i,j) - min(i,j))! / (max(i,j)! min(i,j)!),
 *   B_ij = beta_{j-i} if j >= i, alpha_{i-j} if i > j.
 * The orientation of B follows the proof of the proposition (App. A.6): the
 * entries with j >= i carry the left-edge (t) series beta, the entries with
 * i > j the bottom-edge (s) series alpha; the diagonal therefore uses beta_0
 * for the corner value.
 *
 * Outputs: alpha_out = Ct . eta(1) (the top edge, row sums) and
 *          beta_out  = Ct^T . eta(1) (the right edge, column sums),
 * eta(1) = (1,1,...) because the local tile width is 1.
 */
void orc_tile_map(double rho, int N, const double* alpha, const double* beta,
                  double* alpha_out, double* beta_out) {
    /* factorials and powers of rho up to N */
    double fact[64], rpow[64];
    fact[0] = 1.0;
    rpow[0] = 1.0;
    for (int k = 1; k <= N; ++k) {
        fact[k] = fact[k - 1] * (double)k;
        rpow[k] = rpow[k - 1] * rho;
    }
    for (int i = 0; i <= N; ++i) { alpha_out[i] = 0.0; beta_out[i] = 0.0; }
    for (int i = 0; i <= N; ++i) {
        for (int j = 0; j <= N; ++j) {
            int mn = i < j ? i : j;
            int mx = i < j ? j : i;
            double a_ij = rpow[mn];
            double w_ij = fact[mx - mn] / (fact[mx] * fact[mn]);
            double b_ij = (j >= i) ? beta[j - i] : alpha[i - j];
            double ct = a_ij * b_ij * w_ij;
            alpha_out[i] += ct; /* row sum: coefficient of s^i at t = 1 */
            beta_out[j] += ct;  /* column sum: coefficient of t^j at s = 1 */
        }
    }
}

/* k(x,y) by the tile-centred expansion, tiles visited diagonal by diagonal
 * (App. C.1).  alpha[i] holds the current top edge of x-segment i (the bottom
 * edge of the next tile in that column), beta[j] the current right edge of
 * y-segment j.  Both start as the boundary data K = 1, i.e. e_0. */
int orc_series_pair(const double* dx, int64_t L1, const double* dy, int64_t L2,
                    int d, int N, double* k_out) {
    if (!k_out || d < 1 || N < 1 || N > 60 || L1 < 0 || L2 < 0) return -1;
    if (L1 == 0 || L2 == 0) { *k_out = 1.0; return 0; }
    if (!dx || !dy) return -1;
    const int W = N + 1;
    double* alpha = (double*)calloc((size_t)L1 * W, sizeof(double));
    double* beta = (double*)calloc((size_t)L2 * W, sizeof(double));
    double* ta = (double*)malloc(sizeof(double) * W);
    double* tb = (double*)malloc(sizeof(double) * W);
    if (!alpha || !beta || !ta || !tb) {
        free(alpha); free(beta); free(ta); free(tb);
        return -2;
    }
    for (int64_t i = 0; i < L1; ++i) alpha[i * W] = 1.0;
    for (int64_t j = 0; j < L2; ++j) beta[j * W] = 1.0;
    for (int64_t diag = 0; diag <= L1 + L2 - 2; ++diag) {
        int64_t i_lo = diag - (L2 - 1) > 0 ? diag - (L2 - 1) : 0;
        int64_t i_hi = diag < L1 - 1 ? diag : L1 - 1;
        for (int64_t i = i_lo; i <= i_hi; ++i) {
            int64_t j = diag - i;
            double rho = dot_d(dx + i * d, dy + j * d, d);
            orc_tile_map(rho, N, alpha + i * W, beta + j * W, ta, tb);
            memcpy(alpha + i * W, ta, sizeof(double) * W);
            memcpy(beta + j * W, tb, sizeof(double) * W);
        }
    }
    /* K(1,1): the right edge of the last tile evaluated at t = 1. */
    double k = 0.0;
    for (int q = N; q >= 0; --q) k += beta[(L2 - 1) * W + q];
    *k_out = k;
    free(alpha); free(beta); free(ta); free(tb);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Finite-difference Goursat scheme (Volterra form, Sec. 2.1).               */
/* ------------------------------------------------------------------------ */

/* Each unit tile is cut into 2^lam x 2^lam square cells of side h = 2^-lam.
 * Integrating the PDE over one cell gives
 *     K11 - K10 - K01 + K00 = c h^2 * (mean of K over the cell),
 * and the trapezoid rule for the mean gives the implicit update
 *     K11 (1 - q) = K10 + K01 - K00 + q (K00 + K10 + K01),  q = c h^2 / 4,
 * which is second order in h.  K = 1 on both axes.  One grid row is kept. */
int orc_fd_pair(const double* dx, int64_t L1, const double* dy, int64_t L2,
                int d, int lam, double* k_out) {
    if (!k_out || d < 1 || lam < 0 || lam > 12 || L1 < 0 || L2 < 0) return -1;
    if (L1 == 0 || L2 == 0) { *k_out = 1.0; return 0; }
    if (!dx || !dy) return -1;
    const int64_t r = (int64_t)1 << lam;
    const int64_t n1 = L1 * r; /* cells along s */
    const double h2 = 1.0 / (double)(r * r);
    double* row = (double*)malloc(sizeof(double) * (size_t)(n1 + 1));
    double* c = (double*)malloc(sizeof(double) * (size_t)L1);
    if (!row || !c) { free(row); free(c); return -2; }
    for (int64_t p = 0; p <= n1; ++p) row[p] = 1.0; /* K(s, 0) = 1 */
    for (int64_t j = 0; j < L2; ++j) {
        for (int64_t i = 0; i < L1; ++i) c[i] = dot_d(dx + i * d, dy + j * d, d);
        for (int64_t sub = 0; sub < r; ++sub) {
            double k00 = row[0];
            row[0] = 1.0; /* K(0, t) = 1 */
            for (int64_t p = 0; p < n1; ++p) {
                double q = c[p >> lam] * h2 * 0.25;
                double k10 = row[p + 1];
                double k01 = row[p];
                double k11 = (k10 + k01 - k00 + q * (k00 + k10 + k01)) / (1.0 - q);
                k00 = k10;
                row[p + 1] = k11;
            }
        }
    }
    *k_out = row[n1];
    free(row); free(c);
    return 0;
}

/* Richardson extrapolation of orc_fd_pair over lam0, lam0+1, lam0+2: the
 * scheme's error expands in even powers of h, so two elimination steps
 * (factors 4 and 16) leave an O(h^6) remainder.  out[0..2] receive the raw
 * values, out[3] the extrapolated one. */
int orc_fd_richardson(const double* dx, int64_t L1, const double* dy, int64_t L2,
                      int d, int lam0, double* out) {
    double k[3];
    for (int t = 0; t < 3; ++t) {
        int rc = orc_fd_pair(dx, L1, dy, L2, d, lam0 + t, &k[t]);
        if (rc) return rc;
        out[t] = k[t];
    }
    double r1a = (4.0 * k[1] - k[0]) / 3.0;
    double r1b = (4.0 * k[2] - k[1]) / 3.0;
    out[3] = (16.0 * r1b - r1a) / 15.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Truncated signature inner product (Chen's identity).                      */
/* ------------------------------------------------------------------------ */

static int64_t ipow_i64(int64_t b, int e) {
    int64_t r = 1;
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}

/* S <- S (x) exp(delta) in the tensor algebra truncated at level M.  Level n
 * of S occupies d^n doubles starting at off[n].  exp(delta) has level m equal
 * to delta^{(x)m} / m!, stored in P at the same offsets. */
static void chen_step(double* S, const double* P, const int64_t* off, int d, int M) {
    for (int n = M; n >= 1; --n) {
        int64_t dn = ipow_i64(d, n);
        double* Sn = S + off[n];
        for (int k = 0; k < n; ++k) {
            int m = n - k;
            int64_t dk = ipow_i64(d, k), dm = ipow_i64(d, m);
            const double* Sk = S + off[k];
            const double* Pm = P + off[m];
            for (int64_t I = 0; I < dk; ++I) {
                double s = Sk[I];
                if (s == 0.0) continue;
                double* dst = Sn + I * dm;
                for (int64_t J = 0; J < dm; ++J) dst[J] += s * Pm[J];
            }
        }
        (void)dn;
    }
}

static int chen_signature(const double* dz, int64_t L, int d, int M, double* S,
                          double* P, const int64_t* off) {
    int64_t total = off[M + 1];
    memset(S, 0, sizeof(double) * (size_t)total);
    S[0] = 1.0;
    for (int64_t i = 0; i < L; ++i) {
        const double* delta = dz + i * d;
        /* tensor powers delta^{(x)m}/m! */
        P[0] = 1.0;
        for (int m = 1; m <= M; ++m) {
            int64_t dprev = ipow_i64(d, m - 1);
            const double* prev = P + off[m - 1];
            double* cur = P + off[m];
            for (int64_t I = 0; I < dprev; ++I)
                for (int e = 0; e < d; ++e) cur[I * d + e] = prev[I] * delta[e] / (double)m;
        }
        chen_step(S, P, off, d, M);
    }
    return 0;
}

/* k_M = sum_{n=0}^{M} <S^n(x), S^n(y)>.  levels_out (optional, M+1 doubles)
 * receives the per-level inner products so callers can check the tail. */
int orc_chen_pair(const double* dx, int64_t L1, const double* dy, int64_t L2,
                  int d, int M, double* k_out, double* levels_out) {
    if (!k_out || d < 1 || M < 0 || L1 < 0 || L2 < 0) return -1;
    int64_t off[66];
    off[0] = 0;
    for (int n = 0; n <= M; ++n) {
        off[n + 1] = off[n] + ipow_i64(d, n);
        if (off[n + 1] > ((int64_t)1 << 26)) return -1; /* brute force only */
    }
    int64_t total = off[M + 1];
    double* Sx = (double*)malloc(sizeof(double) * (size_t)total);
    double* Sy = (double*)malloc(sizeof(double) * (size_t)total);
    double* P = (double*)malloc(sizeof(double) * (size_t)total);
    if (!Sx || !Sy || !P) { free(Sx); free(Sy); free(P); return -2; }
    chen_signature(dx, L1, d, M, Sx, P, off);
    chen_signature(dy, L2, d, M, Sy, P, off);
    double k = 0.0;
    for (int n = 0; n <= M; ++n) {
        double s = 0.0;
        for (int64_t I = off[n]; I < off[n + 1]; ++I) s += Sx[I] * Sy[I];
        if (levels_out) levels_out[n] = s;
        k += s;
    }
    *k_out = k;
    free(Sx); free(Sy); free(P);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Batched forms: Gram matrix and MMD^2 over packed ragged increments.       */
/* ------------------------------------------------------------------------ */

/* Increments of path p occupy rows [off[p], off[p] + len[p]) of a packed
 * row-major (sum len) x d array; len[p] is the number of SEGMENTS. */
static void prefix_offsets(const int64_t* len, int64_t n, int64_t* off) {
    off[0] = 0;
    for (int64_t p = 0; p < n; ++p) off[p + 1] = off[p] + len[p];
}

/* G[a*n_y + b] = k(x_a, y_b) by orc_series_pair with order N; OpenMP over
 * pairs.  n_threads <= 0 keeps the runtime default. */
int orc_series_gram(const double* X, const int64_t* len_x, int64_t n_x,
                    const double* Y, const int64_t* len_y, int64_t n_y, int d,
                    int N, int n_threads, double* G) {
    if (!G || n_x < 0 || n_y < 0) return -1;
    int64_t* ox = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_x + 1));
    int64_t* oy = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_y + 1));
    if (!ox || !oy) { free(ox); free(oy); return -2; }
    prefix_offsets(len_x, n_x, ox);
    prefix_offsets(len_y, n_y, oy);
    int err = 0;
    int64_t total = n_x * n_y;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int64_t t = 0; t < total; ++t) {
        int64_t a = t / n_y, b = t % n_y;
        int rc = orc_series_pair(X + ox[a] * d, len_x[a], Y + oy[b] * d, len_y[b], d, N,
                                 &G[t]);
        if (rc) err |= 1;
    }
    free(ox); free(oy);
    return err ? -1 : 0;
}

/* Pairwise k(x_p, y_p) for p = 0..n-1 (independent pairs). */
int orc_series_pairs(const double* X, const int64_t* len_x, const double* Y,
                     const int64_t* len_y, int64_t n, int d, int N, int n_threads,
                     double* k_out) {
    if (!k_out || n < 0) return -1;
    int64_t* ox = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* oy = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!ox || !oy) { free(ox); free(oy); return -2; }
    prefix_offsets(len_x, n, ox);
    prefix_offsets(len_y, n, oy);
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int64_t p = 0; p < n; ++p) {
        int rc = orc_series_pair(X + ox[p] * d, len_x[p], Y + oy[p] * d, len_y[p], d, N,
                                 &k_out[p]);
        if (rc) err |= 1;
    }
    free(ox); free(oy);
    return err ? -1 : 0;
}

/* MMD^2 from the three Gram blocks.  unbiased != 0: U-statistic (diagonals of
 * Kxx and Kyy excluded); otherwise the V-statistic (all entries). */
double orc_mmd2_from_grams(const double* Kxx, int64_t m, const double* Kyy, int64_t n,
                           const double* Kxy, int unbiased) {
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = 0; b < m; ++b)
            if (!unbiased || a != b) sxx += Kxx[a * m + b];
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = 0; b < n; ++b)
            if (!unbiased || a != b) syy += Kyy[a * n + b];
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = 0; b < n; ++b) sxy += Kxy[a * n + b];
    double mm = unbiased ? (double)m * (double)(m - 1) : (double)m * (double)m;
    double nn = unbiased ? (double)n * (double)(n - 1) : (double)n * (double)n;
    return sxx / mm + syy / nn - 2.0 * sxy / ((double)m * (double)n);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
