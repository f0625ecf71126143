/*
 * Plain FP64 dense linear algebra for the DC-LNO oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the oracle: a slow, direct
 * CPU statement of what the DC-LNO hot path computes.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code with the CUDA library.
 *
 * Contents (all matrices row-major, leading dimension = n unless stated):
 *   orc_cholesky      S = L L^T (lower, in place)                 [cluster solve, Sec. II.C step (iii)]
 *   orc_jacobi        cyclic Jacobi eigen-decomposition of a symmetric matrix
 *   orc_gen_eig       H c = eps S c via Cholesky, congruence, Jacobi, back-substitution
 *   orc_nonsym_eig    eigenvalues of a small nonsymmetric matrix: Householder
 *                     reduction to Hessenberg form, then Francis double-shift QR
 *                     (Golub & Van Loan, Matrix Computations, Sec. 7.4-7.5)
 *   orc_inverse_iter  eigenvector of a nonsymmetric matrix for a given (possibly
 *                     complex) eigenvalue by inverse iteration
 * The last two realise the general eigendecomposition of the nonsymmetric
 * Lambda matrix of Eq. (eigendecomp) (Sec. II.B, LNO step (ii)).
 *
 * Return codes: 0 = success; >0 = failure index (Cholesky pivot k+1);
 * -1 = not converged.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) * (size_t)(ld) + (size_t)(j))

/* ---------------------------------------------------------------------- */
/* Cholesky: A = L L^T, L stored in the lower triangle; upper set to 0.    */
/* ---------------------------------------------------------------------- */
int orc_cholesky(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[IDX(j, j, n)];
        for (int k = 0; k < j; ++k) d -= A[IDX(j, k, n)] * A[IDX(j, k, n)];
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        A[IDX(j, j, n)] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[IDX(i, j, n)];
            for (int k = 0; k < j; ++k) s -= A[IDX(i, k, n)] * A[IDX(j, k, n)];
            A[IDX(i, j, n)] = s / ljj;
        }
        for (int i = 0; i < j; ++i) A[IDX(i, j, n)] = 0.0;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Cyclic Jacobi for a symmetric matrix (Golub & Van Loan Sec. 8.5).        */
/* On exit w holds the eigenvalues in ascending order and V (n x n) the     */
/* orthonormal eigenvectors as columns.  A is destroyed.                    */
/* Sweeps stop when off(A) <= tol * ||A||_F (tol = 1e-15) or after          */
/* max_sweeps sweeps (then -1).                                             */
/* ---------------------------------------------------------------------- */
static double off_norm(int n, const double *A)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) s += A[IDX(i, j, n)] * A[IDX(i, j, n)];
    return sqrt(s);
}

int orc_jacobi(int n, double *A, double *w, double *V, int max_sweeps)
{
    double fro = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) fro += A[k] * A[k];
    fro = sqrt(fro);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
    int converged = (n <= 1);
    const double tol = 1e-15 * fro;
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        if (off_norm(n, A) <= tol) { converged = 1; break; }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[IDX(p, q, n)];
                if (fabs(apq) <= 1e-300 || fabs(apq) < 1e-18 * fro) continue;
                double app = A[IDX(p, p, n)], aqq = A[IDX(q, q, n)];
                /* 2x2 symmetric Schur decomposition: annihilate a_pq. */
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- J^T A J with J = [[c, s], [-s, c]] in the (p, q) plane. */
                for (int k = 0; k < n; ++k) {
                    double akp = A[IDX(k, p, n)], akq = A[IDX(k, q, n)];
                    A[IDX(k, p, n)] = c * akp - s * akq;
                    A[IDX(k, q, n)] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[IDX(p, k, n)], aqk = A[IDX(q, k, n)];
                    A[IDX(p, k, n)] = c * apk - s * aqk;
                    A[IDX(q, k, n)] = s * apk + c * aqk;
                }
                A[IDX(p, q, n)] = 0.0;
                A[IDX(q, p, n)] = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = V[IDX(k, p, n)], vkq = V[IDX(k, q, n)];
                    V[IDX(k, p, n)] = c * vkp - s * vkq;
                    V[IDX(k, q, n)] = s * vkp + c * vkq;
                }
            }
        }
        if (off_norm(n, A) <= tol) converged = 1;
    }
    for (int i = 0; i < n; ++i) w[i] = A[IDX(i, i, n)];
    /* selection sort of (w, columns of V), ascending */
    for (int i = 0; i < n; ++i) {
        int m = i;
        for (int j = i + 1; j < n; ++j) if (w[j] < w[m]) m = j;
        if (m != i) {
            double t = w[i]; w[i] = w[m]; w[m] = t;
            for (int k = 0; k < n; ++k) {
                double u = V[IDX(k, i, n)];
                V[IDX(k, i, n)] = V[IDX(k, m, n)];
                V[IDX(k, m, n)] = u;
            }
        }
    }
    return converged ? 0 : -1;
}

/* ---------------------------------------------------------------------- */
/* Generalised symmetric-definite problem H C = S C diag(eps), C^T S C = I.  */
/* S = L L^T;  A = L^{-1} H L^{-T};  A = Y diag(eps) Y^T;  C = L^{-T} Y.      */
/* H and S are not modified.  Returns 0, a Cholesky pivot index (>0), or -1.  */
/* ---------------------------------------------------------------------- */
int orc_gen_eig(int n, const double *H, const double *S, double *eps, double *C)
{
    size_t nn = (size_t)n * n;
    double *L = malloc(nn * sizeof(double));
    double *W = malloc(nn * sizeof(double));
    double *A = malloc(nn * sizeof(double));
    if (!L || !W || !A) { free(L); free(W); free(A); return -2; }
    memcpy(L, S, nn * sizeof(double));
    int info = orc_cholesky(n, L);
    if (info) { free(L); free(W); free(A); return info; }
    /* W = L^{-1} H: forward substitution, column by column of H. */
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = H[IDX(i, j, n)];
            for (int k = 0; k < i; ++k) s -= L[IDX(i, k, n)] * W[IDX(k, j, n)];
            W[IDX(i, j, n)] = s / L[IDX(i, i, n)];
        }
    }
    /* A = L^{-1} W^T  (= L^{-1} H L^{-T} because H is symmetric). */
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = W[IDX(j, i, n)];
            for (int k = 0; k < i; ++k) s -= L[IDX(i, k, n)] * A[IDX(k, j, n)];
            A[IDX(i, j, n)] = s / L[IDX(i, i, n)];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            double m = 0.5 * (A[IDX(i, j, n)] + A[IDX(j, i, n)]);
            A[IDX(i, j, n)] = m;
            A[IDX(j, i, n)] = m;
        }
    int rc = orc_jacobi(n, A, eps, W, 60); /* W now holds Y */
    /* C = L^{-T} Y: back substitution with the upper-triangular L^T. */
    for (int j = 0; j < n; ++j) {
        for (int i = n - 1; i >= 0; --i) {
            double s = W[IDX(i, j, n)];
            for (int k = i + 1; k < n; ++k) s -= L[IDX(k, i, n)] * C[IDX(k, j, n)];
            C[IDX(i, j, n)] = s / L[IDX(i, i, n)];
        }
    }
    free(L); free(W); free(A);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Eigenvalues of a nonsymmetric m x m matrix (m small).                    */
/* Step 1: Householder reduction to upper Hessenberg form.                  */
/* Step 2: Francis implicit double-shift QR on the active window, deflating */
/*         1x1 and 2x2 blocks from the bottom.                              */
/* wr/wi receive real and imaginary parts (unsorted).                       */
/* ---------------------------------------------------------------------- */
static void house_vec(int len, const double *x, double *v, double *beta)
{
    /* v with v[0] = 1 such that (I - beta v v^T) x = -sign(x0)||x|| e1 */
    double sigma = 0.0;
    for (int k = 1; k < len; ++k) sigma += x[k] * x[k];
    v[0] = 1.0;
    for (int k = 1; k < len; ++k) v[k] = x[k];
    if (sigma == 0.0) { *beta = 0.0; return; }
    double mu = sqrt(x[0] * x[0] + sigma);
    double v0 = (x[0] <= 0.0) ? x[0] - mu : -sigma / (x[0] + mu);
    *beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
    for (int k = 1; k < len; ++k) v[k] /= v0;
}

/* apply P = I - beta v v^T from the left to rows r0..r0+len-1, columns c0..c1 */
static void house_left(double *A, int n, int r0, int len, int c0, int c1,
                       const double *v, double beta)
{
    for (int j = c0; j <= c1; ++j) {
        double s = 0.0;
        for (int k = 0; k < len; ++k) s += v[k] * A[IDX(r0 + k, j, n)];
        s *= beta;
        for (int k = 0; k < len; ++k) A[IDX(r0 + k, j, n)] -= s * v[k];
    }
}

/* apply P from the right to columns c0..c0+len-1, rows r0..r1 */
static void house_right(double *A, int n, int c0, int len, int r0, int r1,
                        const double *v, double beta)
{
    for (int i = r0; i <= r1; ++i) {
        double s = 0.0;
        for (int k = 0; k < len; ++k) s += A[IDX(i, c0 + k, n)] * v[k];
        s *= beta;
        for (int k = 0; k < len; ++k) A[IDX(i, c0 + k, n)] -= s * v[k];
    }
}

static void eig2x2(double a, double b, double c, double d, double *r1, double *i1,
                   double *r2, double *i2)
{
    /* eigenvalues of [[a, b], [c, d]]: tr +- sqrt(p^2 + bc) with p = (a - d)/2.  The
     * discriminant is formed from p and bc, not as tr^2 - det, which cancels to zero
     * for eigenvalues closer than about sqrt(u) |tr|. */
    double tr = 0.5 * (a + d);
    double p = 0.5 * (a - d);
    double det = a * d - b * c;
    double disc = p * p + b * c;
    if (disc >= 0.0) {
        double s = sqrt(disc);
        double big = tr + (tr >= 0.0 ? s : -s);
        double small = (big != 0.0) ? det / big : tr - s;
        *r1 = big; *i1 = 0.0; *r2 = small; *i2 = 0.0;
    } else {
        double s = sqrt(-disc);
        *r1 = tr; *i1 = s; *r2 = tr; *i2 = -s;
    }
}

int orc_nonsym_eig(int m, const double *A_in, double *wr, double *wi)
{
    if (m <= 0) return 0;
    double *A = malloc((size_t)m * m * sizeof(double));
    double v[64], x[64];
    if (!A || m > 64) { free(A); return -2; }
    memcpy(A, A_in, (size_t)m * m * sizeof(double));
    /* Hessenberg reduction */
    for (int k = 0; k < m - 2; ++k) {
        int len = m - k - 1;
        for (int t = 0; t < len; ++t) x[t] = A[IDX(k + 1 + t, k, m)];
        double beta;
        house_vec(len, x, v, &beta);
        if (beta != 0.0) {
            house_left(A, m, k + 1, len, 0, m - 1, v, beta);
            house_right(A, m, k + 1, len, 0, m - 1, v, beta);
        }
        for (int t = k + 2; t < m; ++t) A[IDX(t, k, m)] = 0.0;
    }
    const double eps = 2.220446049250313e-16;
    int hi = m - 1;
    int iter = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) { wr[0] = A[0]; wi[0] = 0.0; hi = -1; break; }
        /* find the lowest lo such that H[lo..hi] is unreduced */
        int lo = hi;
        while (lo > 0) {
            double sub = fabs(A[IDX(lo, lo - 1, m)]);
            double diag = fabs(A[IDX(lo, lo, m)]) + fabs(A[IDX(lo - 1, lo - 1, m)]);
            if (diag == 0.0) diag = 1.0;
            if (sub <= eps * diag) { A[IDX(lo, lo - 1, m)] = 0.0; break; }
            --lo;
        }
        if (lo == hi) { /* 1x1 block deflated */
            wr[hi] = A[IDX(hi, hi, m)]; wi[hi] = 0.0;
            --hi; iter = 0; continue;
        }
        if (lo == hi - 1) { /* 2x2 block deflated */
            eig2x2(A[IDX(hi - 1, hi - 1, m)], A[IDX(hi - 1, hi, m)],
                   A[IDX(hi, hi - 1, m)], A[IDX(hi, hi, m)],
                   &wr[hi - 1], &wi[hi - 1], &wr[hi], &wi[hi]);
            hi -= 2; iter = 0; continue;
        }
        if (++total > 100 * m) { free(A); return -1; }
        ++iter;
        /* double shift from the trailing 2x2 block (exceptional shifts at 10, 20) */
        double s, t;
        if (iter == 10 || iter == 20) {
            double e = fabs(A[IDX(hi, hi - 1, m)]) + fabs(A[IDX(hi - 1, hi - 2, m)]);
            s = 1.5 * e + A[IDX(hi, hi, m)];
            t = e * e;
        } else {
            double a = A[IDX(hi - 1, hi - 1, m)], b = A[IDX(hi - 1, hi, m)];
            double c = A[IDX(hi, hi - 1, m)], d = A[IDX(hi, hi, m)];
            s = a + d;
            t = a * d - b * c;
        }
        /* first column of (H - s1 I)(H - s2 I) = H^2 - s H + t I */
        double h00 = A[IDX(lo, lo, m)], h01 = A[IDX(lo, lo + 1, m)];
        double h10 = A[IDX(lo + 1, lo, m)], h11 = A[IDX(lo + 1, lo + 1, m)];
        double h21 = A[IDX(lo + 2, lo + 1, m)];
        x[0] = h00 * h00 + h01 * h10 - s * h00 + t;
        x[1] = h10 * (h00 + h11 - s);
        x[2] = h10 * h21;
        /* chase the bulge */
        for (int k = lo; k <= hi - 2; ++k) {
            double beta;
            house_vec(3, x, v, &beta);
            int c0 = (k > lo) ? k - 1 : lo;
            if (beta != 0.0) {
                house_left(A, m, k, 3, c0, m - 1, v, beta);
                int r1 = (k + 3 < hi) ? k + 3 : hi;
                house_right(A, m, k, 3, 0, r1, v, beta);
            }
            if (k > lo) { A[IDX(k + 1, k - 1, m)] = 0.0; A[IDX(k + 2, k - 1, m)] = 0.0; }
            x[0] = A[IDX(k + 1, k, m)];
            x[1] = A[IDX(k + 2, k, m)];
            if (k < hi - 2) x[2] = A[IDX(k + 3, k, m)];
        }
        {
            double beta;
            house_vec(2, x, v, &beta);
            if (beta != 0.0) {
                house_left(A, m, hi - 1, 2, hi - 2, m - 1, v, beta);
                house_right(A, m, hi - 1, 2, 0, hi, v, beta);
            }
            A[IDX(hi, hi - 2, m)] = 0.0;
        }
    }
    free(A);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Inverse iteration: eigenvector x of A (m x m) for eigenvalue lr + i li.  */
/* Solves (A - (lambda + delta) I) y = x repeatedly with Gaussian            */
/* elimination and partial pivoting in complex arithmetic; delta is a tiny   */
/* relative perturbation that keeps the shifted matrix nonsingular.          */
/* Output: xr, xi (real and imaginary parts), 2-norm 1.  Returns 0.          */
/* ---------------------------------------------------------------------- */
int orc_inverse_iter(int m, const double *A, double lr, double li, double *xr, double *xi)
{
    double complex M[64 * 64], y[64], b[64];
    int piv[64];
    if (m > 64 || m <= 0) return -2;
    double anorm = 0.0;
    for (int k = 0; k < m * m; ++k) anorm += A[k] * A[k];
    anorm = sqrt(anorm);
    if (anorm == 0.0) anorm = 1.0;
    double complex lam = lr + li * I;
    double complex shift = lam + 1e-13 * anorm;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            M[i * m + j] = A[IDX(i, j, m)] - (i == j ? shift : 0.0);
    /* LU with partial pivoting */
    for (int k = 0; k < m; ++k) {
        int p = k;
        for (int i = k + 1; i < m; ++i) if (cabs(M[i * m + k]) > cabs(M[p * m + k])) p = i;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < m; ++j) { double complex t = M[k * m + j]; M[k * m + j] = M[p * m + j]; M[p * m + j] = t; }
        if (cabs(M[k * m + k]) < 1e-300) M[k * m + k] = 1e-300 * anorm;
        for (int i = k + 1; i < m; ++i) {
            double complex f = M[i * m + k] / M[k * m + k];
            M[i * m + k] = f;
            for (int j = k + 1; j < m; ++j) M[i * m + j] -= f * M[k * m + j];
        }
    }
    for (int i = 0; i < m; ++i) b[i] = 1.0 / sqrt((double)m) + 0.01 * i * I * (li != 0.0);
    for (int it = 0; it < 4; ++it) {
        for (int k = 0; k < m; ++k) y[k] = b[k];
        for (int k = 0; k < m; ++k)
            if (piv[k] != k) { double complex t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < i; ++k) y[i] -= M[i * m + k] * y[k];
        for (int i = m - 1; i >= 0; --i) {
            for (int k = i + 1; k < m; ++k) y[i] -= M[i * m + k] * y[k];
            y[i] /= M[i * m + i];
        }
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += creal(y[i] * conj(y[i]));
        nrm = sqrt(nrm);
        for (int i = 0; i < m; ++i) b[i] = y[i] / nrm;
    }
    /* fix the complex phase: make the largest component real and positive */
    int jm = 0;
    for (int i = 1; i < m; ++i) if (cabs(b[i]) > cabs(b[jm])) jm = i;
    double complex ph = conj(b[jm]) / cabs(b[jm]);
    for (int i = 0; i < m; ++i) { b[i] *= ph; xr[i] = creal(b[i]); xi[i] = cimag(b[i]); }
    return 0;
}
