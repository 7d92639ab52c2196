/*
 * fjofc_cpu.c -- Algorithm 2 of the paper (fJOFC) in float64 on the host cores.
 *
 * TEST INFRASTRUCTURE ONLY: the CPU baseline that bench.py times beside the GPU and a
 * second float64 restatement of the method that tests/ checks against the numpy oracle.
 * The CUDA library never links or calls it, and it shares no code with it.
 *
 * What it computes (the paper's steps, in its order):
 *   - Wmod, the m x m modified weight matrix of Eq. (modW) built from the m x m weights of
 *     Eq. (W2): Wmod_jj = n w_jj + sum_{l != j} w_jl, Wmod_jl = -w_jl; its inverse by
 *     Gauss-Jordan elimination with partial pivoting (Sec. 2.1, Thm 1);
 *   - per transform, for every modality l, the diagonal block (B_l X^(l))_i =
 *     sum_{j != i, d_ij != 0} w_ll Delta_l[i][j] / d_ij (x_i - x_j) of B(X) X (Eq. B),
 *     over full rows of Delta_l;
 *   - the update X_t^(j) = sum_l [Wmod^-1]_{jl} B_l X_{t-1}^(l) (Eq. update; the J_n part
 *     of Cor. 1 is dropped because every column of B_l sums to zero, Sec. 2.1);
 *   - the raw stress of Eq. (stress): sum_l w_ll sum_{i<j} (Delta_l[i][j] - d_ij)^2 +
 *     sum_{j<l} w_jl ||X^(j) - X^(l)||_F^2;
 *   - the stopping rule of Algorithm 1/2 with the decrease reading: continue while
 *     sigma(X_{t-1}) - sigma(X_t) exceeds tol (mode 0: divided by C(mn, 2), Remark eps;
 *     mode 1: divided by sigma(X_{t-1})); tol < 0 runs exactly max_iter transforms.
 * Rows are independent within a step, so the loops over objects run in parallel
 * (OpenMP) when the compiler supports it; every sum over j is taken in index order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int fjofc_cpu_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* inverse of the m x m modified weight matrix (Eq. modW); 0 on success */
static int wmod_inverse(int m, long n, const double* W, double* winv) {
    double* A = (double*)calloc((size_t)m * 2 * m, sizeof(double));
    if (!A) return -1;
    for (int j = 0; j < m; ++j) {
        double diag = (double)n * W[j * m + j];
        for (int l = 0; l < m; ++l)
            if (l != j) {
                diag += W[j * m + l];
                A[(size_t)j * 2 * m + l] = -W[j * m + l];
            }
        A[(size_t)j * 2 * m + j] = diag;
        A[(size_t)j * 2 * m + m + j] = 1.0;
    }
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(A[(size_t)r * 2 * m + c]) > fabs(A[(size_t)piv * 2 * m + c])) piv = r;
        if (A[(size_t)piv * 2 * m + c] == 0.0) {
            free(A);
            return -1;
        }
        if (piv != c)
            for (int k = 0; k < 2 * m; ++k) {
                const double t = A[(size_t)c * 2 * m + k];
                A[(size_t)c * 2 * m + k] = A[(size_t)piv * 2 * m + k];
                A[(size_t)piv * 2 * m + k] = t;
            }
        const double inv = 1.0 / A[(size_t)c * 2 * m + c];
        for (int k = 0; k < 2 * m; ++k) A[(size_t)c * 2 * m + k] *= inv;
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * 2 * m + c];
            for (int k = 0; k < 2 * m; ++k) A[(size_t)r * 2 * m + k] -= f * A[(size_t)c * 2 * m + k];
        }
    }
    for (int j = 0; j < m; ++j)
        for (int l = 0; l < m; ++l) winv[j * m + l] = A[(size_t)j * 2 * m + m + l];
    free(A);
    return 0;
}

static double dist(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = a[k] - b[k];
        s += t * t;
    }
    return sqrt(s);
}

/* raw stress of Eq. (stress) */
static double stress(int m, long n, int d, const double* const* delta, const double* W, const double* X) {
    double fid = 0.0;
    for (int l = 0; l < m; ++l) {
        const double* Xl = X + (size_t)l * n * d;
        const double* Dl = delta[l];
        double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(dynamic, 16)
        for (long i = 0; i < n; ++i)
            for (long j = i + 1; j < n; ++j) {
                const double e = Dl[(size_t)i * n + j] - dist(Xl + (size_t)i * d, Xl + (size_t)j * d, d);
                s += e * e;
            }
        fid += W[l * m + l] * s;
    }
    double comm = 0.0;
    for (int j = 0; j < m; ++j)
        for (int l = j + 1; l < m; ++l) {
            double s = 0.0;
            for (size_t e = 0; e < (size_t)n * d; ++e) {
                const double t = X[(size_t)j * n * d + e] - X[(size_t)l * n * d + e];
                s += t * t;
            }
            comm += W[j * m + l] * s;
        }
    return fid + comm;
}

/*
 * In-sample fJOFC from X (in place).  delta: m pointers to n x n row-major float64
 * matrices; W: m x m float64 (Eq. W2); X: (m n) x d float64, rows modality-major.
 * hist (may be NULL) receives sigma(X_0) .. sigma(X_T); *iters_out = T.
 * Returns 0, -1 for invalid sizes (d <= 64) or weights, -2 when memory runs out.
 */
int fjofc_cpu_embed(int m, long n, int d, const double* const* delta, const double* W, double* X, int max_iter,
                    double tol, int tol_mode, double* hist, int* iters_out) {
    if (m < 1 || n < 2 || d < 1 || d > 64) return -1;
    double* winv = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* BX = (double*)malloc(sizeof(double) * (size_t)m * n * d);
    if (!winv || !BX) {
        free(winv);
        free(BX);
        return -2;
    }
    if (wmod_inverse(m, n, W, winv)) {
        free(winv);
        free(BX);
        return -1;
    }
    const double npairs = (double)m * n * ((double)m * n - 1.0) / 2.0;
    double prev = stress(m, n, d, delta, W, X);
    if (hist) hist[0] = prev;
    int t = 0;
    while (t < max_iter) {
        /* B_l X^(l) for every modality (Eq. B, full rows) */
        for (int l = 0; l < m; ++l) {
            const double* Xl = X + (size_t)l * n * d;
            const double* Dl = delta[l];
            const double wll = W[l * m + l];
            double* out = BX + (size_t)l * n * d;
#pragma omp parallel for schedule(dynamic, 16)
            for (long i = 0; i < n; ++i) {
                double acc[64];
                for (int k = 0; k < d; ++k) acc[k] = 0.0;
                const double* xi = Xl + (size_t)i * d;
                for (long j = 0; j < n; ++j) {
                    if (j == i) continue;
                    const double* xj = Xl + (size_t)j * d;
                    const double dij = dist(xi, xj, d);
                    if (dij == 0.0) continue;
                    const double b = wll * Dl[(size_t)i * n + j] / dij;
                    for (int k = 0; k < d; ++k) acc[k] += b * (xi[k] - xj[k]);
                }
                for (int k = 0; k < d; ++k) out[(size_t)i * d + k] = acc[k];
            }
        }
        /* X_t^(j) = sum_l [Wmod^-1]_{jl} B_l X^(l) (Eq. update) */
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j)
                for (int k = 0; k < d; ++k) {
                    double v = 0.0;
                    for (int l = 0; l < m; ++l) v += winv[j * m + l] * BX[((size_t)l * n + i) * d + k];
                    X[((size_t)j * n + i) * d + k] = v;
                }
        ++t;
        const double cur = stress(m, n, d, delta, W, X);
        if (hist) hist[t] = cur;
        if (tol >= 0.0) {
            const double dec = prev - cur;
            const int cont = (tol_mode == 1) ? (dec > tol * prev) : (dec / npairs > tol);
            if (!cont) {
                prev = cur;
                break;
            }
        }
        prev = cur;
    }
    if (iters_out) *iters_out = t;
    free(winv);
    free(BX);
    return 0;
}
