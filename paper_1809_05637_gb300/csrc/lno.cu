// LNO generation (Sec. II.B, steps (i)-(iii)):
//   k_lambda   Lambda_0i = sum_Rj rho_{0i,Rj} S_{Rj,0i}   (Eq. (Lambda)); one warp per atom
//   k_lno_eig  eigenvalues of the nonsymmetric Lambda_0i (Householder-Hessenberg + Francis
//              double-shift QR), eigenvectors of the k eigenvalues of largest real part by
//              inverse iteration in real arithmetic (Eq. (eigendecomp), Eq. (apop_Lambda)),
//              returned as an S_ii-orthonormal basis of their span; one thread per atom.
// Symmetric mode (the projector form of the same selection):
//   k_projector  G_i = (S rho S)_{0i,0i} = sum_{Ra,Rb} S_{0i,Ra} rho_{Ra,Rb} S_{Rb,0i}; one CTA
//                per atom
//   k_lno_eig<true>  G_i v = lambda S_ii v for the symmetric part of G_i (Cholesky of S_ii,
//                congruence, cyclic Jacobi), the leading k eigenvectors v = L^-T y.
#include "dclno_internal.cuh"

#define MM DCLNO_MAX_M_LNO

// ---------------------------------------------------------------------------
// Lambda blocks.  S_{Rj,0i} = (S_{0i,Rj})^T, so block b of row i adds rho_b S_b^T.
// Lanes own entries (a, b) of the M_i x M_i result.
// ---------------------------------------------------------------------------
__global__ void k_lambda(int N, const int* __restrict__ norb, const long long* __restrict__ row_ptr,
                         const long long* __restrict__ key, const long long* __restrict__ blk_off,
                         const long long* __restrict__ loff, const double* __restrict__ rho,
                         const double* __restrict__ S, double* __restrict__ Lam) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int i = warp, mi = norb[i];
    double acc[MM * MM / 32];
#pragma unroll
    for (int t = 0; t < MM * MM / 32; ++t) acc[t] = 0.0;
    for (long long b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        const int j = (int)(key[b] >> 24);
        const int mj = norb[j];
        const double* rb = rho + blk_off[b];
        const double* sb = S + blk_off[b];
#pragma unroll
        for (int t = 0; t < MM * MM / 32; ++t) {
            const int e = lane + 32 * t;
            if (e < mi * mi) {
                const int a = e / mi, c = e % mi;
                double s = 0.0;
                for (int g = 0; g < mj; ++g) s = fma(rb[a * mj + g], sb[c * mj + g], s);
                acc[t] += s;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < MM * MM / 32; ++t) {
        const int e = lane + 32 * t;
        if (e < mi * mi) Lam[loff[i] + e] = acc[t];
    }
}

// ---------------------------------------------------------------------------
// Projector blocks.  rho_{Ra,Rb} = rho_{0a,(Rb-Ra)b}: block (a, t1) of row i and block
// (b, t2) of row a reach atom b in cell t1 + t2; its overlap with the centre is block
// (b, t1 + t2) of row i, transposed.  So G_i = sum_p S_p W_p with
// W_p = sum_q rho_q S_{r(q)}^T (M_a x M_i), r(q) found by binary search among row i's
// keys (held in shared memory); absent blocks contribute nothing.  Warps take the
// blocks p of row i; the lanes of a warp look up 32 blocks q at a time and then walk
// the hits in lane order, each lane owning entries of W_p and of G_i.
// ---------------------------------------------------------------------------
#define PROJ_WARPS 8

__device__ inline int add_packed_shift(int p, int q) {
    int a0, a1, a2, b0, b1, b2;
    unpack_shift(p, a0, a1, a2);
    unpack_shift(q, b0, b1, b2);
    const int s0 = a0 + b0, s1 = a1 + b1, s2 = a2 + b2;
    if (s0 < -128 || s0 > 127 || s1 < -128 || s1 > 127 || s2 < -128 || s2 > 127) return -1;
    return pack_shift(s0, s1, s2);
}

__device__ inline int find_key(const long long* keys, int len, long long want) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < want)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < len && keys[lo] == want) ? lo : -1;
}

__global__ void __launch_bounds__(PROJ_WARPS * 32)
    k_projector(const int* __restrict__ norb, const long long* __restrict__ row_ptr,
                const long long* __restrict__ key, const long long* __restrict__ blk_off,
                const long long* __restrict__ loff, const double* __restrict__ rho,
                const double* __restrict__ S, double* __restrict__ G) {
    extern __shared__ long long sh_key[];          // keys of row i, sorted
    __shared__ double sh_w[PROJ_WARPS][MM * MM];   // W_p of each warp (M_a x M_i)
    __shared__ double sh_g[PROJ_WARPS][MM * MM];   // partial G_i of each warp
    const unsigned full = 0xffffffffu;
    const int i = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r0 = row_ptr[i];
    const int len = (int)(row_ptr[i + 1] - r0);
    for (int t = threadIdx.x; t < len; t += blockDim.x) sh_key[t] = key[r0 + t];
    __syncthreads();
    const int mi = norb[i];
    double g[MM * MM / 32];
#pragma unroll
    for (int t = 0; t < MM * MM / 32; ++t) g[t] = 0.0;
    for (int p = warp; p < len; p += PROJ_WARPS) {
        const long long kp = sh_key[p];
        const int a = (int)(kp >> 24), t1 = (int)(kp & 0xffffff);
        const int ma = norb[a];
        double w[MM * MM / 32];
#pragma unroll
        for (int t = 0; t < MM * MM / 32; ++t) w[t] = 0.0;
        const long long q1 = row_ptr[a + 1];
        for (long long qb = row_ptr[a]; qb < q1; qb += 32) {
            const long long q = qb + lane;
            int r = -1, b = 0;
            if (q < q1) {
                const long long kq = key[q];
                b = (int)(kq >> 24);
                const int ps = add_packed_shift(t1, (int)(kq & 0xffffff));
                if (ps >= 0) r = find_key(sh_key, len, block_key(b, ps));
            }
            unsigned hit = __ballot_sync(full, r >= 0);
            while (hit) {
                const int src = __ffs(hit) - 1;
                hit &= hit - 1;
                const long long qs = __shfl_sync(full, q, src);
                const int rs = __shfl_sync(full, r, src);
                const int mb = norb[__shfl_sync(full, b, src)];
                const double* rq = rho + blk_off[qs];     // rho_{0a,t2 b}: M_a x M_b
                const double* sr = S + blk_off[r0 + rs];  // S_{0i,(t1+t2) b}: M_i x M_b
#pragma unroll
                for (int t = 0; t < MM * MM / 32; ++t) {
                    const int e = lane + 32 * t;
                    if (e < ma * mi) {
                        const int x = e / mi, cc = e % mi;
                        double s = 0.0;
                        for (int u = 0; u < mb; ++u) s = fma(rq[x * mb + u], sr[cc * mb + u], s);
                        w[t] += s;
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < MM * MM / 32; ++t) {
            const int e = lane + 32 * t;
            if (e < ma * mi) sh_w[warp][e] = w[t];
        }
        __syncwarp();
        const double* sp = S + blk_off[r0 + p];  // S_{0i,t1 a}: M_i x M_a
#pragma unroll
        for (int t = 0; t < MM * MM / 32; ++t) {
            const int e = lane + 32 * t;
            if (e < mi * mi) {
                const int y = e / mi, cc = e % mi;
                double s = 0.0;
                for (int x = 0; x < ma; ++x) s = fma(sp[y * ma + x], sh_w[warp][x * mi + cc], s);
                g[t] += s;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < MM * MM / 32; ++t) {
        const int e = lane + 32 * t;
        if (e < mi * mi) sh_g[warp][e] = g[t];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < mi * mi; e += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < PROJ_WARPS; ++w) s += sh_g[w][e];
        G[loff[i] + e] = s;
    }
}

// ---------------------------------------------------------------------------
// Small dense helpers for one thread (m <= 32, row-major m x m in local memory)
// ---------------------------------------------------------------------------
__device__ static void hessenberg_reduce(double* A, int m) {
    double v[MM];
    for (int k = 0; k + 2 < m; ++k) {
        // Householder vector annihilating A[k+2:, k]
        double alpha = A[(k + 1) * m + k];
        double sig = 0.0;
        for (int r = k + 2; r < m; ++r) sig += A[r * m + k] * A[r * m + k];
        if (sig == 0.0) continue;
        double nrm = sqrt(alpha * alpha + sig);
        double beta = alpha > 0 ? -nrm : nrm;  // reflect onto beta e1 with |beta| = ||x||
        double v0 = alpha - beta;
        v[k + 1] = 1.0;
        for (int r = k + 2; r < m; ++r) v[r] = A[r * m + k] / v0;
        double tau = (beta - alpha) / beta;
        // A <- P A P with P = I - tau v v^T acting on rows/cols k+1..m-1
        for (int c = 0; c < m; ++c) {
            double s = 0.0;
            for (int r = k + 1; r < m; ++r) s += v[r] * A[r * m + c];
            s *= tau;
            for (int r = k + 1; r < m; ++r) A[r * m + c] -= s * v[r];
        }
        for (int r = 0; r < m; ++r) {
            double s = 0.0;
            for (int c = k + 1; c < m; ++c) s += A[r * m + c] * v[c];
            s *= tau;
            for (int c = k + 1; c < m; ++c) A[r * m + c] -= s * v[c];
        }
        A[(k + 1) * m + k] = beta;
        for (int r = k + 2; r < m; ++r) A[r * m + k] = 0.0;
    }
}

// reflector from a 2- or 3-vector x: P = I - tau u u^T, u[0] = 1, P x = beta e1
__device__ static void small_house(int len, const double* x, double* u, double& tau) {
    double sig = 0.0;
    for (int t = 1; t < len; ++t) sig += x[t] * x[t];
    u[0] = 1.0;
    u[1] = u[2] = 0.0;
    if (sig == 0.0) {
        tau = 0.0;
        return;
    }
    double nrm = sqrt(x[0] * x[0] + sig);
    double beta = x[0] > 0 ? -nrm : nrm;
    double v0 = x[0] - beta;
    for (int t = 1; t < len; ++t) u[t] = x[t] / v0;
    tau = (beta - x[0]) / beta;
}

__device__ static void apply_small(double* A, int m, int r0, int len, int cl, int ch, int rl, int rh,
                                   const double* u, double tau) {
    if (tau == 0.0) return;
    for (int c = cl; c <= ch; ++c) {  // from the left on rows r0..r0+len-1
        double s = 0.0;
        for (int t = 0; t < len; ++t) s += u[t] * A[(r0 + t) * m + c];
        s *= tau;
        for (int t = 0; t < len; ++t) A[(r0 + t) * m + c] -= s * u[t];
    }
    for (int r = rl; r <= rh; ++r) {  // from the right on cols r0..r0+len-1
        double s = 0.0;
        for (int t = 0; t < len; ++t) s += A[r * m + r0 + t] * u[t];
        s *= tau;
        for (int t = 0; t < len; ++t) A[r * m + r0 + t] -= s * u[t];
    }
}

// Eigenvalues of an upper Hessenberg matrix by Francis double-shift QR. Returns 0 or -1.
__device__ static int francis_qr(double* A, int m, double* wr, double* wi) {
    const double eps = 2.220446049250313e-16;
    int hi = m - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            wr[0] = A[0];
            wi[0] = 0.0;
            break;
        }
        int lo = hi;
        for (; lo > 0; --lo) {
            double s = fabs(A[(lo - 1) * m + lo - 1]) + fabs(A[lo * m + lo]);
            if (s == 0.0) s = 1.0;
            if (fabs(A[lo * m + lo - 1]) <= eps * s) {
                A[lo * m + lo - 1] = 0.0;
                break;
            }
        }
        if (lo == hi) {
            wr[hi] = A[hi * m + hi];
            wi[hi] = 0.0;
            --hi;
            its = 0;
            continue;
        }
        if (lo == hi - 1) {
            double a = A[(hi - 1) * m + hi - 1], b = A[(hi - 1) * m + hi];
            double c = A[hi * m + hi - 1], d = A[hi * m + hi];
            double p = 0.5 * (a - d);
            double disc = p * p + b * c;
            double mid = 0.5 * (a + d);
            if (disc >= 0.0) {
                double r = sqrt(disc);
                double z = mid + (mid >= 0 ? r : -r);
                double det = a * d - b * c;
                wr[hi - 1] = z;
                wr[hi] = (z != 0.0) ? det / z : mid - (mid >= 0 ? r : -r);
                wi[hi - 1] = wi[hi] = 0.0;
            } else {
                double r = sqrt(-disc);
                wr[hi - 1] = wr[hi] = mid;
                wi[hi - 1] = r;
                wi[hi] = -r;
            }
            hi -= 2;
            its = 0;
            continue;
        }
        if (++total > 60 * m) return -1;
        ++its;
        double sh, dt;
        if (its % 11 == 10) {  // exceptional shift
            double w = fabs(A[hi * m + hi - 1]) + fabs(A[(hi - 1) * m + hi - 2]);
            sh = 2.0 * A[hi * m + hi] + 1.5 * w;
            dt = (A[hi * m + hi] + 0.75 * w) * (A[hi * m + hi] + 0.75 * w) - 0.4375 * w * w;
        } else {
            double a = A[(hi - 1) * m + hi - 1], b = A[(hi - 1) * m + hi];
            double c = A[hi * m + hi - 1], d = A[hi * m + hi];
            sh = a + d;
            dt = a * d - b * c;
        }
        double x[3], u[3], tau;
        const double h00 = A[lo * m + lo], h01 = A[lo * m + lo + 1];
        const double h10 = A[(lo + 1) * m + lo], h11 = A[(lo + 1) * m + lo + 1];
        const double h21 = A[(lo + 2) * m + lo + 1];
        x[0] = h00 * h00 + h01 * h10 - sh * h00 + dt;
        x[1] = h10 * (h00 + h11 - sh);
        x[2] = h10 * h21;
        for (int k = lo; k <= hi - 2; ++k) {
            small_house(3, x, u, tau);
            int cl = (k > lo) ? k - 1 : lo;
            int rh = (k + 3 < hi) ? k + 3 : hi;
            apply_small(A, m, k, 3, cl, m - 1, 0, rh, u, tau);
            if (k > lo) A[(k + 1) * m + k - 1] = A[(k + 2) * m + k - 1] = 0.0;
            x[0] = A[(k + 1) * m + k];
            x[1] = A[(k + 2) * m + k];
            x[2] = (k < hi - 2) ? A[(k + 3) * m + k] : 0.0;
        }
        small_house(2, x, u, tau);
        apply_small(A, m, hi - 1, 2, hi - 2, m - 1, 0, hi, u, tau);
        A[hi * m + hi - 2] = 0.0;
    }
    return 0;
}

// Solve M x = b in place (Gaussian elimination with partial pivoting), M n x n row-major
// in local memory (destroyed); tiny pivots are replaced by a tiny number.
__device__ static void lu_solve(double* Mx, int n, double* b, double tiny) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(Mx[r * n + k]) > fabs(Mx[p * n + k])) p = r;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = Mx[k * n + c];
                Mx[k * n + c] = Mx[p * n + c];
                Mx[p * n + c] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        if (fabs(Mx[k * n + k]) < tiny) Mx[k * n + k] = (Mx[k * n + k] < 0 ? -tiny : tiny);
        const double inv = 1.0 / Mx[k * n + k];
        for (int r = k + 1; r < n; ++r) {
            const double f = Mx[r * n + k] * inv;
            if (f == 0.0) continue;
            for (int c = k + 1; c < n; ++c) Mx[r * n + c] -= f * Mx[k * n + c];
            b[r] -= f * b[k];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int c = r + 1; c < n; ++c) s -= Mx[r * n + c] * b[c];
        b[r] = s / Mx[r * n + r];
    }
}

// Cyclic Jacobi (Golub & Van Loan, Sec. 8.5) on the symmetric m x m matrix A: the
// eigenvalues are left on its diagonal, the rotations accumulate in Y (eigenvectors in
// columns).  Returns 0 once the off-diagonal mass is below 1e-30 of the total.
__device__ static int jacobi_sym(double* A, double* Y, int m) {
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) Y[r * m + c] = (r == c) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) {
                const double v = A[r * m + c] * A[r * m + c];
                tot += v;
                if (r != c) off += v;
            }
        if (off <= 1e-30 * tot) return 0;
        for (int p = 0; p + 1 < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[p * m + q];
                if (apq == 0.0) continue;
                // rotation J (J_pp = J_qq = cs, J_pq = sn, J_qp = -sn) with (J^T A J)_pq = 0
                const double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double tn = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
                if (theta < 0.0) tn = -tn;
                const double cs = 1.0 / sqrt(tn * tn + 1.0), sn = tn * cs;
                for (int u = 0; u < m; ++u) {
                    const double up = A[u * m + p], uq = A[u * m + q];
                    A[u * m + p] = cs * up - sn * uq;
                    A[u * m + q] = sn * up + cs * uq;
                }
                for (int u = 0; u < m; ++u) {
                    const double pu = A[p * m + u], qu = A[q * m + u];
                    A[p * m + u] = cs * pu - sn * qu;
                    A[q * m + u] = sn * pu + cs * qu;
                }
                for (int u = 0; u < m; ++u) {
                    const double yp = Y[u * m + p], yq = Y[u * m + q];
                    Y[u * m + p] = cs * yp - sn * yq;
                    Y[u * m + q] = sn * yp + cs * yq;
                }
            }
    }
    return 1;
}

// ---------------------------------------------------------------------------
// One thread per atom.  SYM = false: Lam holds Lambda_0i (the paper's problem);
// SYM = true: Lam holds G_i = (S rho S)_{0i,0i} (k_projector).
// ---------------------------------------------------------------------------
template <bool SYM>
__global__ void k_lno_eig(int N, int k, int use_th, double lam_th, const int* __restrict__ norb,
                          const long long* __restrict__ loff,
                          const long long* __restrict__ moff, const long long* __restrict__ voff,
                          const long long* __restrict__ onsite, const long long* __restrict__ blk_off,
                          const double* __restrict__ S, const double* __restrict__ Lam,
                          double* __restrict__ V, double* __restrict__ lam_re, double* __restrict__ lam_im,
                          int* __restrict__ flags, int* __restrict__ kat, int* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int m = norb[i];
    double A[MM * MM], wr[MM], wi[MM];
    int ord[MM];
    const double* L = Lam + loff[i];
    double* Vi = V + voff[i];  // m x k, row-major
    const double* Sii = S + blk_off[onsite[i]];
    int fl = 0, got = 0;
    if constexpr (SYM) {
        double Lc[MM * MM], Y[MM * MM];
        // S_ii = Lc Lc^T
        for (int j = 0; j < m; ++j) {
            double s = Sii[j * m + j];
            for (int u = 0; u < j; ++u) s -= Lc[j * m + u] * Lc[j * m + u];
            if (!(s > 0.0)) {
                status[i] = ST_NOT_SPD;
                return;
            }
            Lc[j * m + j] = sqrt(s);
            for (int r = j + 1; r < m; ++r) {
                double v = Sii[r * m + j];
                for (int u = 0; u < j; ++u) v -= Lc[r * m + u] * Lc[j * m + u];
                Lc[r * m + j] = v / Lc[j * m + j];
            }
            for (int r = 0; r < j; ++r) Lc[r * m + j] = 0.0;
        }
        // A = Lc^-1 Gs Lc^-T with Gs the symmetric part of G: two forward substitutions
        // (Lc^-1 Gs, transposed, Lc^-1 again), then symmetrised
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) A[r * m + c] = 0.5 * (L[r * m + c] + L[c * m + r]);
        for (int pass = 0; pass < 2; ++pass) {
            for (int c = 0; c < m; ++c)
                for (int r = 0; r < m; ++r) {
                    double v = A[r * m + c];
                    for (int u = 0; u < r; ++u) v -= Lc[r * m + u] * A[u * m + c];
                    A[r * m + c] = v / Lc[r * m + r];
                }
            for (int r = 0; r < m; ++r)
                for (int c = r + 1; c < m; ++c) {
                    const double x = A[r * m + c];
                    A[r * m + c] = A[c * m + r];
                    A[c * m + r] = x;
                }
        }
        for (int r = 0; r < m; ++r)
            for (int c = r + 1; c < m; ++c) {
                const double x = 0.5 * (A[r * m + c] + A[c * m + r]);
                A[r * m + c] = x;
                A[c * m + r] = x;
            }
        if (jacobi_sym(A, Y, m) != 0) {
            status[i] = ST_NOT_CONVERGED;
            return;
        }
        // eigenvalues descending (ties: lower index first)
        for (int t = 0; t < m; ++t) {
            wr[t] = A[t * m + t];
            ord[t] = t;
        }
        for (int a = 1; a < m; ++a) {
            int v = ord[a], b = a - 1;
            while (b >= 0 && wr[ord[b]] < wr[v]) {
                ord[b + 1] = ord[b];
                --b;
            }
            ord[b + 1] = v;
        }
        for (int t = 0; t < m; ++t) {
            lam_re[moff[i] + t] = wr[ord[t]];
            lam_im[moff[i] + t] = 0.0;
        }
        // the leading k (with the threshold: those >= lambda_th), v = Lc^-T y
        while (got < k && got < m && !(use_th && wr[ord[got]] < lam_th)) {
            const int col = ord[got];
            double x[MM];
            for (int r = m - 1; r >= 0; --r) {
                double v = Y[r * m + col];
                for (int u = r + 1; u < m; ++u) v -= Lc[u * m + r] * x[u];
                x[r] = v / Lc[r * m + r];
            }
            for (int r = 0; r < m; ++r) Vi[r * k + got] = x[r];
            ++got;
        }
    } else {
        double anorm = 0.0;
        for (int e = 0; e < m * m; ++e) {
            A[e] = L[e];
            anorm += L[e] * L[e];
        }
        anorm = sqrt(anorm);
        if (anorm == 0.0) anorm = 1.0;
        hessenberg_reduce(A, m);
        if (francis_qr(A, m, wr, wi) != 0) {
            status[i] = ST_NOT_CONVERGED;
            return;
        }
        // order: real part descending, then imaginary part descending
        for (int t = 0; t < m; ++t) ord[t] = t;
        for (int a = 1; a < m; ++a) {
            int v = ord[a], b = a - 1;
            while (b >= 0 && (wr[ord[b]] < wr[v] || (wr[ord[b]] == wr[v] && wi[ord[b]] < wi[v]))) {
                ord[b + 1] = ord[b];
                --b;
            }
            ord[b + 1] = v;
        }
        for (int t = 0; t < m; ++t) {
            lam_re[moff[i] + t] = wr[ord[t]];
            lam_im[moff[i] + t] = wi[ord[t]];
        }
        // eigenvectors of the leading eigenvalues
        int pos = 0;
        const double tiny = 1e-300;
        while (got < k && pos < m) {
            const double lr = wr[ord[pos]], li = wi[ord[pos]];
            if (use_th && lr < lam_th) break;  // threshold selection: eigenvalues >= lambda_th only
            const double sh = lr + 1e-13 * anorm;  // shifted off the eigenvalue to keep the solve regular
            if (li == 0.0) {
                double x[MM];
                for (int r = 0; r < m; ++r) x[r] = 1.0 + 0.01 * r;
                for (int it = 0; it < 4; ++it) {
                    for (int e = 0; e < m * m; ++e) A[e] = L[e];
                    for (int r = 0; r < m; ++r) A[r * m + r] -= sh;
                    lu_solve(A, m, x, tiny * anorm);
                    double nr = 0.0;
                    for (int r = 0; r < m; ++r) nr += x[r] * x[r];
                    nr = rsqrt(nr);
                    for (int r = 0; r < m; ++r) x[r] *= nr;
                }
                for (int r = 0; r < m; ++r) Vi[r * k + got] = x[r];
                ++got;
                ++pos;
            } else {
                // (Lambda - (sh + i li) I)(x + i y) = b in real form:
                // [[Lambda - sh I, li I], [-li I, Lambda - sh I]] [x; y] = [br; bi]
                fl |= DCLNO_LNO_COMPLEX_SELECTED;
                double B[4 * MM * MM];
                double z[2 * MM];
                const int n2 = 2 * m;
                for (int r = 0; r < n2; ++r) z[r] = (r < m) ? 1.0 + 0.01 * r : 0.02 * (r - m);
                for (int it = 0; it < 4; ++it) {
                    for (int r = 0; r < m; ++r)
                        for (int c = 0; c < m; ++c) {
                            const double a = L[r * m + c] - (r == c ? sh : 0.0);
                            B[r * n2 + c] = a;
                            B[(r + m) * n2 + c + m] = a;
                            B[r * n2 + c + m] = (r == c) ? li : 0.0;
                            B[(r + m) * n2 + c] = (r == c) ? -li : 0.0;
                        }
                    lu_solve(B, n2, z, tiny * anorm);
                    double nr = 0.0;
                    for (int r = 0; r < n2; ++r) nr += z[r] * z[r];
                    nr = rsqrt(nr);
                    for (int r = 0; r < n2; ++r) z[r] *= nr;
                }
                // phase: largest-magnitude component real and positive
                int jm = 0;
                double best = -1.0;
                for (int r = 0; r < m; ++r) {
                    double a2 = z[r] * z[r] + z[r + m] * z[r + m];
                    if (a2 > best) {
                        best = a2;
                        jm = r;
                    }
                }
                const double pr = z[jm], pi = z[jm + m], pn = rsqrt(pr * pr + pi * pi);
                const double cr = pr * pn, ci = -pi * pn;  // multiply by conj(z_jm)/|z_jm|
                for (int r = 0; r < m; ++r) {
                    const double xr = z[r] * cr - z[r + m] * ci;
                    const double xi = z[r] * ci + z[r + m] * cr;
                    z[r] = xr;
                    z[r + m] = xi;
                }
                for (int r = 0; r < m; ++r) Vi[r * k + got] = z[r];
                ++got;
                if (got < k) {
                    for (int r = 0; r < m; ++r) Vi[r * k + got] = z[r + m];
                    ++got;
                } else {
                    fl |= DCLNO_LNO_PAIR_SPLIT;
                }
                pos += 2;
            }
        }
    }
    // S_ii-orthonormal basis of the span (Gram-Schmidt in eigenvalue order, twice);
    // the columns beyond this atom's count (threshold selection) are zero
    const int kk = got;
    for (int c = kk; c < k; ++c)
        for (int r = 0; r < m; ++r) Vi[r * k + c] = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < kk; ++c) {
            for (int d = 0; d < c; ++d) {
                // coefficient <v_d, v_c>_S
                double h = 0.0;
                for (int r = 0; r < m; ++r) {
                    double t = 0.0;
                    for (int s = 0; s < m; ++s) t += Sii[r * m + s] * Vi[s * k + c];
                    h += Vi[r * k + d] * t;
                }
                for (int r = 0; r < m; ++r) Vi[r * k + c] -= h * Vi[r * k + d];
            }
            double nn = 0.0;
            for (int r = 0; r < m; ++r) {
                double t = 0.0;
                for (int s = 0; s < m; ++s) t += Sii[r * m + s] * Vi[s * k + c];
                nn += Vi[r * k + c] * t;
            }
            if (!(nn > 0.0)) {
                status[i] = ST_BAD_LNO;
                return;
            }
            nn = rsqrt(nn);
            for (int r = 0; r < m; ++r) Vi[r * k + c] *= nn;
        }
    }
    for (int c = 0; c < kk; ++c) {
        int jm = 0;
        for (int r = 1; r < m; ++r)
            if (fabs(Vi[r * k + c]) > fabs(Vi[jm * k + c])) jm = r;
        if (Vi[jm * k + c] < 0.0)
            for (int r = 0; r < m; ++r) Vi[r * k + c] = -Vi[r * k + c];
    }
    flags[i] = fl;
    kat[i] = kk;
    status[i] = ST_OK;
}

// row i's keys sit in dynamic shared memory beside the 32 KB of static tiles; the
// limit is raised once per build, outside any stream capture
#define PROJ_MAX_DYN ((size_t)227 * 1024 - 2 * PROJ_WARPS * MM * MM * sizeof(double))

dclno_status prepare_lno_kernels(dclno_ctx* c) {
    DCLNO_CUDA(c, cudaFuncSetAttribute(k_projector, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PROJ_MAX_DYN));
    return DCLNO_OK;
}

dclno_status launch_lambda_lno(dclno_ctx* c, const double* rho) {
    const int N = c->N;
    const bool sym = c->lno_mode == DCLNO_LNO_SYM;
    if (sym) {
        const size_t dyn = sizeof(long long) * (size_t)std::max<long long>(c->max_row, 1);
        if (dyn > PROJ_MAX_DYN)
            return set_err(c, DCLNO_ERR_ARG, "symmetric LNO mode: a BSR row of " + std::to_string(c->max_row) +
                                                 " blocks does not fit in shared memory");
        ProfScope ps__(c, "k_projector");
        k_projector<<<N, PROJ_WARPS * 32, dyn, c->stream>>>(c->d_norb, c->d_row_ptr, c->d_key, c->d_blk_off,
                                                             c->d_loff, rho, c->S, c->d_Lambda);
    } else {
        ProfScope ps__(c, "k_lambda");
        k_lambda<<<(N * 32 + 127) / 128, 128, 0, c->stream>>>(N, c->d_norb, c->d_row_ptr, c->d_key, c->d_blk_off,
                                                          c->d_loff, rho, c->S, c->d_Lambda);
    }
    DCLNO_LAUNCHED(c);
    {
        ProfScope ps__(c, "k_lno_eig");
        const int use_th = c->lno_th_on ? 1 : 0;
        auto kern = sym ? k_lno_eig<true> : k_lno_eig<false>;
        kern<<<(N + 63) / 64, 64, 0, c->stream>>>(N, c->k_lno, use_th, c->lno_th, c->d_norb, c->d_loff, c->d_moff,
                                                 c->d_voff, c->d_onsite, c->d_blk_off, c->S, c->d_Lambda, c->d_V,
                                                 c->d_lam_re, c->d_lam_im, c->d_lflags, c->d_kat, c->d_status);
    }
    DCLNO_LAUNCHED(c);
    if (c->deferred) return launch_status_or(c);
    std::vector<int> st(N);
    DCLNO_CUDA(c, cudaMemcpyAsync(st.data(), c->d_status, sizeof(int) * N, cudaMemcpyDeviceToHost, c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < N; ++i) {
        if (st[i] == ST_NOT_CONVERGED)
            return set_err(c, DCLNO_ERR_NOT_CONVERGED, "LNO eigenvalues of atom " + std::to_string(i) + " did not converge");
        if (st[i] == ST_NOT_SPD)
            return set_err(c, DCLNO_ERR_NOT_SPD, "on-site overlap of atom " + std::to_string(i) + " is not positive definite");
        if (st[i] != ST_OK)
            return set_err(c, DCLNO_ERR_NOT_CONVERGED, "LNO basis of atom " + std::to_string(i) + " is degenerate");
    }
    if (c->lno_th_on) return relayout_clusters(c);
    return DCLNO_OK;
}
