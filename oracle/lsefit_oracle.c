/*
 * lsefit_oracle.c -- plain, slow, sequential FP64 oracle for the matricized
 * least-square-errors polynomial fit (Dasgupta, "An Analytical Evaluation of
 * Matricizing Least-Square-Errors Curve Fitting", arXiv 1512.08017).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA path, and the CUDA path never calls it.
 *
 * Every step follows the paper's route in the paper's order:
 *   Section II, the objective  Pi = sum_i [y_i - f(x_i)]^2  with
 *               f(x) = a_0 + a_1 x + ... + a_m x^m;
 *   Section II, the normal equations  sum_i x_i^j y_i = sum_k a_k sum_i x_i^(j+k);
 *   Section II, the matrices  A (Hankel of the power sums S_0..S_2m),
 *               B = [T_0..T_m], X = [a_0..a_m];
 *   Section II, Gaussian elimination of AX = B.
 * Readings where the paper is silent or misprinted:
 *   - the derivative printed in Section II drops the factor x_i^j inside the
 *     sum; the expanded normal equations right after it are used;
 *   - the top-left entry of A is printed "1"; it is S_0 = n;
 *   - the last row of A is printed with x^(m+2) in its second column; the
 *     Hankel rule A[j][k] = S_{j+k} is used;
 *   - "Gaussian elimination" carries no pivoting rule: partial pivoting with
 *     the first row of largest magnitude, and a pivot at or below
 *     (m+1)*eps*max|A| reported as singular, where eps is the machine epsilon
 *     of the arithmetic that formed the power sums (2^-52 for FP64, 2^-23
 *     for FP32 per-point powers: their rounding alone leaves pivots of that
 *     relative size in a rank-deficient system);
 *   - n >= 2 is only enough for m = 1: n >= m+1 is required.
 * Not in the paper (the precision extension of the method):
 *   - an affine map t = s*(x - c) of the abscissae, with c = (lo+hi)/2 and
 *     s = 2/(hi-lo) rounded to the precision in which the points are mapped
 *     (FP32 for FP32/BF16 arithmetic, FP64 otherwise); the fit runs on t and
 *     the coefficients are mapped back by the binomial expansion of
 *     (s(x - c))^k;
 *   - the adjoint of the fit (derived by the chain rule from the normal
 *     equations): with lambda solving A lambda = dL/dXt,
 *     dL/dy_i = lambda(t_i) and dL/dt_i = lambda'(t_i) r_i - lambda(t_i) f'(t_i);
 *   - two generalisations of the objective (Section V leaves higher-order
 *     fits and other solution methods open): per-point weights w_i, and the
 *     Chebyshev basis T_k(t) in place of t^k (orc_fit_general).
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared -pthread lsefit_oracle.c -lm
 * (-ffp-contract=off keeps every product and sum a separately rounded IEEE
 * operation on every host, so results do not depend on FMA contraction.)
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Oracle status values (own numbering; the test suite maps them by name). */
#define ORC_OK 0
#define ORC_N_TOO_SMALL 1
#define ORC_SINGULAR 2
#define ORC_NONFINITE 3
#define ORC_BAD_INTERVAL 4
#define ORC_BAD_ARG 5

#define ORC_MAX_M 16

int orc_max_degree(void) { return ORC_MAX_M; }

/*
 * Map constants of the affine map onto [-1, 1].  c = (lo+hi)/2 and
 * s = 2/(hi-lo), each rounded once to FP32 when fp32 != 0.
 */
int orc_map_constants(double lo, double hi, int fp32, double* c, double* s)
{
    if (!(isfinite(lo) && isfinite(hi)) || !(hi > lo)) return ORC_BAD_INTERVAL;
    double cc = (lo + hi) / 2.0;
    double ss = 2.0 / (hi - lo);
    if (fp32) {
        cc = (double)(float)cc;
        ss = (double)(float)ss;
    }
    if (!isfinite(cc) || !isfinite(ss) || ss == 0.0) return ORC_BAD_INTERVAL;
    *c = cc;
    *s = ss;
    return ORC_OK;
}

/*
 * Power sums of Section II: S[k] = sum_i t_i^k (k = 0..2m) and
 * T[k] = sum_i t_i^k y_i (k = 0..m), with t_i = x_i, or t_i = s*(x_i - c)
 * when map != NULL (map = {c, s}).  One sequential pass, i = 0..n-1, powers
 * by a running product; S[0] is the point count.
 */
void orc_powersums(const double* x, const double* y, int64_t n, int m,
                   const double* map, double* S, double* T)
{
    for (int k = 0; k <= 2 * m; ++k) S[k] = 0.0;
    for (int k = 0; k <= m; ++k) T[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = map ? map[1] * (x[i] - map[0]) : x[i];
        double p = 1.0;
        for (int k = 0; k <= 2 * m; ++k) {
            if (k > 0) S[k] += p;
            if (k <= m) T[k] += p * y[i];
            p *= t;
        }
    }
    S[0] = (double)n;
}

/* Gaussian elimination with partial pivoting of the (m+1)x(m+1) system
 * M z = r, M row-major; M and r are overwritten.  Returns ORC_SINGULAR when
 * a pivot is at or below (m+1)*eps*max|M|. */
static int orc_gauss_inplace(int m, double* M, double* r, double* z, double eps)
{
    const int N = m + 1;
    double amax = 0.0;
    for (int i = 0; i < N * N; ++i)
        if (fabs(M[i]) > amax) amax = fabs(M[i]);
    const double tol = (double)N * eps * amax;
    for (int k = 0; k < N; ++k) {
        int p = k;
        for (int i = k + 1; i < N; ++i)
            if (fabs(M[i * N + k]) > fabs(M[p * N + k])) p = i;
        if (!(fabs(M[p * N + k]) > tol)) return ORC_SINGULAR;
        if (p != k) {
            for (int j = 0; j < N; ++j) {
                double tmp = M[k * N + j];
                M[k * N + j] = M[p * N + j];
                M[p * N + j] = tmp;
            }
            double tr = r[k];
            r[k] = r[p];
            r[p] = tr;
        }
        for (int i = k + 1; i < N; ++i) {
            double f = M[i * N + k] / M[k * N + k];
            for (int j = k; j < N; ++j) M[i * N + j] -= f * M[k * N + j];
            r[i] -= f * r[k];
        }
    }
    for (int i = N - 1; i >= 0; --i) {
        double acc = r[i];
        for (int j = i + 1; j < N; ++j) acc -= M[i * N + j] * z[j];
        z[i] = acc / M[i * N + i];
    }
    for (int i = 0; i < N; ++i)
        if (!isfinite(z[i])) return ORC_SINGULAR;
    return ORC_OK;
}

/* Section II: A[j][k] = S[j+k], B[j] = T[j]; solve AX = B by Gaussian
 * elimination.  Checks finiteness of the sums first.  eps: machine epsilon
 * of the arithmetic that formed the sums (singularity threshold). */
int orc_solve(int m, const double* S, const double* T, double eps, double* X)
{
    if (m < 1 || m > ORC_MAX_M) return ORC_BAD_ARG;
    const int N = m + 1;
    for (int k = 0; k <= 2 * m; ++k)
        if (!isfinite(S[k])) return ORC_NONFINITE;
    for (int k = 0; k <= m; ++k)
        if (!isfinite(T[k])) return ORC_NONFINITE;
    double A[(ORC_MAX_M + 1) * (ORC_MAX_M + 1)];
    double B[ORC_MAX_M + 1];
    for (int j = 0; j < N; ++j) {
        for (int k = 0; k < N; ++k) A[j * N + k] = S[j + k];
        B[j] = T[j];
    }
    return orc_gauss_inplace(m, A, B, X, eps);
}

/*
 * Alternative solver (Section V names methods other than Gaussian
 * elimination as future work): A = S_{j+k} is symmetric and, for distinct
 * abscissae, positive definite (A = V^T V), so A = L L^T with L lower
 * triangular (Cholesky), then L z = B and L^T X = z.  A diagonal pivot
 * d_kk = A_kk - sum_j L_kj^2 at or below (m+1)*eps*max|A| means A is not
 * numerically positive definite: reported as singular.
 */
int orc_solve_cholesky(int m, const double* S, const double* T, double eps, double* X)
{
    if (m < 1 || m > ORC_MAX_M) return ORC_BAD_ARG;
    const int N = m + 1;
    for (int k = 0; k <= 2 * m; ++k)
        if (!isfinite(S[k])) return ORC_NONFINITE;
    for (int k = 0; k <= m; ++k)
        if (!isfinite(T[k])) return ORC_NONFINITE;
    double Lm[(ORC_MAX_M + 1) * (ORC_MAX_M + 1)];
    double amax = 0.0;
    for (int k = 0; k <= 2 * m; ++k)
        if (fabs(S[k]) > amax) amax = fabs(S[k]);
    const double tol = (double)N * eps * amax;
    for (int j = 0; j < N; ++j) {
        double d = S[2 * j];
        for (int k = 0; k < j; ++k) d -= Lm[j * N + k] * Lm[j * N + k];
        if (!(d > tol)) return ORC_SINGULAR;
        const double ljj = sqrt(d);
        Lm[j * N + j] = ljj;
        for (int i = j + 1; i < N; ++i) {
            double v = S[i + j];
            for (int k = 0; k < j; ++k) v -= Lm[i * N + k] * Lm[j * N + k];
            Lm[i * N + j] = v / ljj;
        }
    }
    double z[ORC_MAX_M + 1];
    for (int i = 0; i < N; ++i) {
        double acc = T[i];
        for (int k = 0; k < i; ++k) acc -= Lm[i * N + k] * z[k];
        z[i] = acc / Lm[i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double acc = z[i];
        for (int k = i + 1; k < N; ++k) acc -= Lm[k * N + i] * X[k];
        X[i] = acc / Lm[i * N + i];
    }
    for (int i = 0; i < N; ++i)
        if (!isfinite(X[i])) return ORC_SINGULAR;
    return ORC_OK;
}

/* Binomial coefficient C(k, j) as a double (exact for k <= 16). */
static double orc_binom(int k, int j)
{
    double b = 1.0;
    for (int i = 1; i <= j; ++i) b = b * (double)(k - j + i) / (double)i;
    return b;
}

/* Coefficients of f(x) = sum_k Xt[k] (s(x - c))^k in the monomial basis of x:
 * X[j] = sum_{k>=j} Xt[k] * C(k,j) * s^k * (-c)^(k-j). */
void orc_unmap(int m, double c, double s, const double* Xt, double* X)
{
    for (int j = 0; j <= m; ++j) {
        double acc = 0.0;
        for (int k = j; k <= m; ++k)
            acc += Xt[k] * orc_binom(k, j) * pow(s, (double)k) * pow(-c, (double)(k - j));
        X[j] = acc;
    }
}

/* Transpose of the un-map: g_t[k] = sum_{j<=k} C(k,j) s^k (-c)^(k-j) gX[j]. */
static void orc_unmap_transpose(int m, double c, double s, const double* gX, double* gt)
{
    for (int k = 0; k <= m; ++k) {
        double acc = 0.0;
        for (int j = 0; j <= k; ++j)
            acc += orc_binom(k, j) * pow(s, (double)k) * pow(-c, (double)(k - j)) * gX[j];
        gt[k] = acc;
    }
}

/*
 * The whole fit: power sums, normal equations, Gaussian elimination, un-map.
 * map = {c, s} or NULL; eps as for orc_solve.  Outputs (any may be NULL except X): X (x basis),
 * Xt (t basis), S[2m+1], T[m+1].  Returns an ORC_* status; on failure X and
 * Xt are NaN.
 */
int orc_fit(const double* x, const double* y, int64_t n, int m, const double* map, double eps,
            double* X, double* Xt, double* S_out, double* T_out)
{
    double S[2 * ORC_MAX_M + 1], T[ORC_MAX_M + 1], Z[ORC_MAX_M + 1];
    if (m < 1 || m > ORC_MAX_M) return ORC_BAD_ARG;
    orc_powersums(x, y, n, m, map, S, T);
    if (S_out) memcpy(S_out, S, sizeof(double) * (2 * m + 1));
    if (T_out) memcpy(T_out, T, sizeof(double) * (m + 1));
    int st = ORC_OK;
    if (n < m + 1) st = ORC_N_TOO_SMALL;
    else st = orc_solve(m, S, T, eps, Z);
    if (st != ORC_OK) {
        for (int j = 0; j <= m; ++j) {
            X[j] = NAN;
            if (Xt) Xt[j] = NAN;
        }
        return st;
    }
    if (Xt) memcpy(Xt, Z, sizeof(double) * (m + 1));
    if (map) orc_unmap(m, map[0], map[1], Z, X);
    else memcpy(X, Z, sizeof(double) * (m + 1));
    return ORC_OK;
}

/* Fitted values f(x_i) = sum_j X[j] x_i^j (Table V's y_f column). */
void orc_eval(int m, const double* X, const double* x, int64_t n, double* f)
{
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0, p = 1.0;
        for (int j = 0; j <= m; ++j) {
            acc += X[j] * p;
            p *= x[i];
        }
        f[i] = acc;
    }
}

/* Sum of squared residuals, Section II's Pi for coefficients X (Table V). */
double orc_sse(int m, const double* X, const double* x, const double* y, int64_t n)
{
    double sse = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0, p = 1.0;
        for (int j = 0; j <= m; ++j) {
            acc += X[j] * p;
            p *= x[i];
        }
        double e = y[i] - acc;
        sse += e * e;
    }
    return sse;
}

/*
 * Adjoint of orc_fit for a loss L(X) with gradient gX = dL/dX (x basis).
 * The map constants are held fixed.  Steps:
 *   g_t = M^T gX               (M: t-basis -> x-basis coefficient map);
 *   lambda solves A lambda = g_t (A is symmetric, so A^T = A);
 *   dy_i = lambda(t_i);
 *   dt_i = lambda'(t_i) (y_i - f(t_i)) - lambda(t_i) f'(t_i), f = sum Xt_k t^k;
 *   dx_i = s dt_i (dx_i = dt_i without a map).
 * S holds the t-basis power sums S_0..S_2m, Xt the t-basis coefficients.
 */
int orc_backward(const double* x, const double* y, int64_t n, int m, const double* map,
                 const double* S, const double* Xt, const double* gX, double eps,
                 double* dx, double* dy)
{
    double gt[ORC_MAX_M + 1], A[(ORC_MAX_M + 1) * (ORC_MAX_M + 1)], lam[ORC_MAX_M + 1];
    if (m < 1 || m > ORC_MAX_M) return ORC_BAD_ARG;
    const int N = m + 1;
    if (map) orc_unmap_transpose(m, map[0], map[1], gX, gt);
    else memcpy(gt, gX, sizeof(double) * N);
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) A[j * N + k] = S[j + k];
    int st = orc_gauss_inplace(m, A, gt, lam, eps);
    if (st != ORC_OK) return st;
    const double sc = map ? map[1] : 1.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = map ? map[1] * (x[i] - map[0]) : x[i];
        double lv = 0.0, ld = 0.0, fv = 0.0, fd = 0.0;
        double p = 1.0, pm1 = 0.0; /* t^j and t^(j-1) */
        for (int j = 0; j <= m; ++j) {
            lv += lam[j] * p;
            fv += Xt[j] * p;
            if (j > 0) {
                ld += (double)j * lam[j] * pm1;
                fd += (double)j * Xt[j] * pm1;
            }
            pm1 = p;
            p *= t;
        }
        dy[i] = lv;
        dx[i] = sc * (ld * (y[i] - fv) - lv * fd);
    }
    return ORC_OK;
}

/*
 * Generalised objective: Pi_w = sum_i w_i [y_i - f(t_i)]^2 with
 * f(t) = sum_k a_k phi_k(t), where phi_k(t) = t^k (basis 0) or the
 * Chebyshev polynomial T_k(t) (basis 1: T_0 = 1, T_1 = t,
 * T_{k+1} = 2 t T_k - T_{k-1}).  w == NULL means w_i = 1.
 * Setting dPi_w/da_j = 0 as in Section II gives the normal equations
 * G a = b with G[j][k] = sum_i w_i phi_j(t_i) phi_k(t_i) and
 * b[j] = sum_i w_i phi_j(t_i) y_i.  Written out from that definition: for
 * every point the basis values, then the double loop over (j, k).  Solved by
 * the same Gaussian elimination and singularity threshold as orc_solve, with
 * max|G| over the entries of G.
 * Outputs: Xb (coefficients a_k in the chosen basis of t), X (monomial
 * coefficients of x: the basis expanded into powers of t, then un-mapped),
 * and optionally G ((m+1)^2, row-major) and b (m+1).  n < m+1 points is
 * N_TOO_SMALL whatever the weights (zero weights show up as SINGULAR).
 */
static void orc_basis(int m, int basis, double t, double* phi)
{
    phi[0] = 1.0;
    if (m >= 1) phi[1] = t;
    for (int k = 2; k <= m; ++k)
        phi[k] = basis == 1 ? 2.0 * t * phi[k - 1] - phi[k - 2] : phi[k - 1] * t;
}

/* Monomial coefficients of sum_k a[k] T_k(t): P[k][j] = coefficient of t^j
 * in T_k, from the same recurrence applied to coefficient rows. */
void orc_cheb_to_mono(int m, const double* a, double* out)
{
    double P[(ORC_MAX_M + 1) * (ORC_MAX_M + 1)];
    const int N = m + 1;
    for (int i = 0; i < N * N; ++i) P[i] = 0.0;
    P[0] = 1.0;
    if (m >= 1) P[1 * N + 1] = 1.0;
    for (int k = 2; k <= m; ++k)
        for (int j = 0; j <= k; ++j)
            P[k * N + j] = (j > 0 ? 2.0 * P[(k - 1) * N + j - 1] : 0.0) - P[(k - 2) * N + j];
    for (int j = 0; j < N; ++j) {
        double acc = 0.0;
        for (int k = j; k < N; ++k) acc += a[k] * P[k * N + j];
        out[j] = acc;
    }
}

int orc_fit_general(const double* x, const double* y, const double* w, int64_t n, int m, int basis,
                    const double* map, double eps, double* X, double* Xb, double* G_out, double* b_out)
{
    if (m < 1 || m > ORC_MAX_M || (basis != 0 && basis != 1)) return ORC_BAD_ARG;
    const int N = m + 1;
    double G[(ORC_MAX_M + 1) * (ORC_MAX_M + 1)], b[ORC_MAX_M + 1], phi[ORC_MAX_M + 1], a[ORC_MAX_M + 1];
    for (int i = 0; i < N * N; ++i) G[i] = 0.0;
    for (int j = 0; j < N; ++j) b[j] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double t = map ? map[1] * (x[i] - map[0]) : x[i];
        const double wi = w ? w[i] : 1.0;
        orc_basis(m, basis, t, phi);
        for (int j = 0; j < N; ++j) {
            for (int k = 0; k < N; ++k) G[j * N + k] += wi * phi[j] * phi[k];
            b[j] += wi * phi[j] * y[i];
        }
    }
    if (G_out) memcpy(G_out, G, sizeof(double) * N * N);
    if (b_out) memcpy(b_out, b, sizeof(double) * N);
    int st = ORC_OK;
    if (n < m + 1) st = ORC_N_TOO_SMALL;
    for (int i = 0; st == ORC_OK && i < N * N; ++i)
        if (!isfinite(G[i])) st = ORC_NONFINITE;
    for (int j = 0; st == ORC_OK && j < N; ++j)
        if (!isfinite(b[j])) st = ORC_NONFINITE;
    if (st == ORC_OK) st = orc_gauss_inplace(m, G, b, a, eps);
    if (st != ORC_OK) {
        for (int j = 0; j < N; ++j) {
            X[j] = NAN;
            if (Xb) Xb[j] = NAN;
        }
        return st;
    }
    double Xt[ORC_MAX_M + 1];
    if (basis == 1) orc_cheb_to_mono(m, a, Xt);
    else memcpy(Xt, a, sizeof(double) * N);
    if (Xb) memcpy(Xb, a, sizeof(double) * N);
    if (map) orc_unmap(m, map[0], map[1], Xt, X);
    else memcpy(X, Xt, sizeof(double) * N);
    return ORC_OK;
}

/*
 * Residuals of a fit in the basis `basis` (Section III judges fits by their
 * residual errors, Table V): r_i = y_i - sum_k Xb[k] phi_k(t_i) with
 * t_i = s (x_i - c) (t_i = x_i without a map), SSE = sum_i r_i^2 (returned),
 * vtr[k] = sum_i phi_k(t_i) r_i (k = 0..m), and r (length n) if r_out is set.
 */
double orc_residuals_general(int m, int basis, const double* Xb, const double* map, const double* x,
                             const double* y, int64_t n, double* r_out, double* vtr)
{
    double phi[ORC_MAX_M + 1];
    double sse = 0.0;
    for (int k = 0; k <= m; ++k) vtr[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double t = map ? map[1] * (x[i] - map[0]) : x[i];
        orc_basis(m, basis, t, phi);
        double f = 0.0;
        for (int k = 0; k <= m; ++k) f += Xb[k] * phi[k];
        const double r = y[i] - f;
        if (r_out) r_out[i] = r;
        sse += r * r;
        for (int k = 0; k <= m; ++k) vtr[k] += phi[k] * r;
    }
    return sse;
}

/*
 * The power sums of orc_powersums on all host cores, for timing the oracle
 * against the GPU (not a second definition: each thread runs orc_powersums
 * itself).  Thread t of nthreads takes the fixed point range
 * [n t / nthreads, n (t+1) / nthreads); the per-thread sums are added in
 * thread order, so the result depends only on n and nthreads, and with one
 * thread it is orc_powersums bit for bit.  Returns ORC_OK, or ORC_BAD_ARG for
 * a thread count outside 1..ORC_MAX_THREADS or a thread that could not start.
 */
#define ORC_MAX_THREADS 1024

typedef struct {
    const double* x;
    const double* y;
    int64_t n;
    int m;
    const double* map;
    double S[2 * ORC_MAX_M + 1];
    double T[ORC_MAX_M + 1];
} orc_range;

static void* orc_range_main(void* arg)
{
    orc_range* r = (orc_range*)arg;
    orc_powersums(r->x, r->y, r->n, r->m, r->map, r->S, r->T);
    return NULL;
}

int orc_powersums_threads(const double* x, const double* y, int64_t n, int m, const double* map,
                          int nthreads, double* S, double* T)
{
    if (nthreads < 1 || nthreads > ORC_MAX_THREADS || m < 0 || m > ORC_MAX_M || n < 0) return ORC_BAD_ARG;
    orc_range* r = (orc_range*)calloc((size_t)nthreads, sizeof(orc_range));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    int* started = (int*)calloc((size_t)nthreads, sizeof(int));
    int st = ORC_OK;
    if (!r || !th || !started) st = ORC_BAD_ARG;
    for (int t = 0; st == ORC_OK && t < nthreads; ++t) {
        const int64_t lo = n / nthreads * t + (n % nthreads) * t / nthreads;
        const int64_t hi = n / nthreads * (t + 1) + (n % nthreads) * (t + 1) / nthreads;
        r[t].x = x + lo;
        r[t].y = y + lo;
        r[t].n = hi - lo;
        r[t].m = m;
        r[t].map = map;
        if (pthread_create(&th[t], NULL, orc_range_main, &r[t]) == 0) started[t] = 1;
        else st = ORC_BAD_ARG;
    }
    for (int t = 0; t < nthreads && started; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    if (st == ORC_OK) {
        for (int k = 0; k <= 2 * m; ++k) S[k] = 0.0;
        for (int k = 0; k <= m; ++k) T[k] = 0.0;
        for (int t = 0; t < nthreads; ++t) {
            for (int k = 0; k <= 2 * m; ++k) S[k] += r[t].S[k];  /* S[0]: the range counts, exact */
            for (int k = 0; k <= m; ++k) T[k] += r[t].T[k];
        }
    }
    free(r);
    free(th);
    free(started);
    return st;
}
