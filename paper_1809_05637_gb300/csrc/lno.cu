// LNO generation (Sec. II.B, steps (i)-(iii)):
//   k_lambda   Lambda_0i = sum_Rj rho_{0i,Rj} S_{Rj,0i}   (Eq. (Lambda)); one warp per atom
//   k_lno_eig  eigenvalues of the nonsymmetric Lambda_0i (Householder-Hessenberg + Francis
//              double-shift QR), eigenvectors of the k eigenvalues of largest real part by
//              inverse iteration in real arithmetic (Eq. (eigendecomp), Eq. (apop_Lambda)),
//              returned as an S_ii-orthonormal basis of their span; one warp per atom
//              (lanes over the rows and columns of each update, warp sums and shuffles
//              for the norms, pivots and dot products).
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
// Small dense helpers for one warp (m <= MM, row-major m x m matrices in the warp's
// shared-memory workspace).  Lanes own the columns or rows of each update; the scalar
// control (shifts, deflation, reflector coefficients) is computed by every lane from
// shared memory, so all lanes agree; single entries are written by lane 0, and every
// write is followed by __syncwarp() before any lane reads it.
// ---------------------------------------------------------------------------
#define LNO_FULL 0xffffffffu

// Householder reduction to upper Hessenberg form (Golub & Van Loan, Sec. 7.4.3)
__device__ static void hessenberg_w(double* A, int m, double* u) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k + 2 < m; ++k) {
        // reflector annihilating A[k+2:, k]
        const double alpha = A[(k + 1) * m + k];
        const double x = (lane >= k + 2 && lane < m) ? A[lane * m + k] : 0.0;
        const double sig = warp_sum(x * x);
        if (sig == 0.0) continue;
        const double nrm = sqrt(alpha * alpha + sig);
        const double beta = alpha > 0 ? -nrm : nrm;  // reflect onto beta e1 with |beta| = ||x||
        const double v0 = alpha - beta, tau = (beta - alpha) / beta;
        if (lane < m) u[lane] = (lane < k + 1) ? 0.0 : (lane == k + 1 ? 1.0 : x / v0);
        __syncwarp();
        if (lane < m) {  // A <- P A: column `lane`
            double s = 0.0;
            for (int r = k + 1; r < m; ++r) s += u[r] * A[r * m + lane];
            s *= tau;
            for (int r = k + 1; r < m; ++r) A[r * m + lane] -= s * u[r];
        }
        __syncwarp();
        if (lane < m) {  // A <- A P: row `lane`
            double s = 0.0;
            for (int c = k + 1; c < m; ++c) s += A[lane * m + c] * u[c];
            s *= tau;
            for (int c = k + 1; c < m; ++c) A[lane * m + c] -= s * u[c];
        }
        __syncwarp();
        if (lane == k + 1) A[lane * m + k] = beta;
        else if (lane >= k + 2 && lane < m) A[lane * m + k] = 0.0;
        __syncwarp();
    }
}

// reflector from a 2- or 3-vector x: P = I - tau u u^T, u[0] = 1, P x = beta e1
// (every lane computes the same coefficients)
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

// P from the left on rows r0 .. r0+len-1, columns cl..ch (a lane per column), then from
// the right on columns r0 .. r0+len-1, rows rl..rh (a lane per row)
__device__ static void apply_small_w(double* A, int m, int r0, int len, int cl, int ch, int rl, int rh,
                                     const double* u, double tau) {
    const int lane = threadIdx.x & 31;
    if (tau == 0.0) return;
    const int c = cl + lane;
    if (c <= ch) {
        double s = 0.0;
        for (int t = 0; t < len; ++t) s += u[t] * A[(r0 + t) * m + c];
        s *= tau;
        for (int t = 0; t < len; ++t) A[(r0 + t) * m + c] -= s * u[t];
    }
    __syncwarp();
    const int r = rl + lane;
    if (r <= rh) {
        double s = 0.0;
        for (int t = 0; t < len; ++t) s += A[r * m + r0 + t] * u[t];
        s *= tau;
        for (int t = 0; t < len; ++t) A[r * m + r0 + t] -= s * u[t];
    }
    __syncwarp();
}

// lane 0 writes one entry, then the warp synchronises
__device__ __forceinline__ void lw_put(double* p, double v) {
    if ((threadIdx.x & 31) == 0) *p = v;
    __syncwarp();
}

// Eigenvalues of an upper Hessenberg matrix by Francis double-shift QR (Golub & Van
// Loan, Algorithm 7.5.1, with deflation at negligible subdiagonal entries and an
// exceptional shift every eleventh iteration).  wr, wi in shared memory.  Returns 0,
// or -1 when 60 m iterations did not suffice (the same for every lane).
__device__ static int francis_qr_w(double* A, int m, double* wr, double* wi) {
    const double eps = 2.220446049250313e-16;
    int hi = m - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            lw_put(&wr[0], A[0]);
            lw_put(&wi[0], 0.0);
            break;
        }
        int lo = hi;
        for (; lo > 0; --lo) {
            double s = fabs(A[(lo - 1) * m + lo - 1]) + fabs(A[lo * m + lo]);
            if (s == 0.0) s = 1.0;
            if (fabs(A[lo * m + lo - 1]) <= eps * s) {
                lw_put(&A[lo * m + lo - 1], 0.0);
                break;
            }
        }
        if (lo == hi) {
            lw_put(&wr[hi], A[hi * m + hi]);
            lw_put(&wi[hi], 0.0);
            --hi;
            its = 0;
            continue;
        }
        if (lo == hi - 1) {
            const double a = A[(hi - 1) * m + hi - 1], b = A[(hi - 1) * m + hi];
            const double c = A[hi * m + hi - 1], d = A[hi * m + hi];
            const double p = 0.5 * (a - d);
            const double disc = p * p + b * c;
            const double mid = 0.5 * (a + d);
            double r0, r1, i0, i1;
            if (disc >= 0.0) {
                const double r = sqrt(disc);
                const double z = mid + (mid >= 0 ? r : -r);
                const double det = a * d - b * c;
                r0 = z;
                r1 = (z != 0.0) ? det / z : mid - (mid >= 0 ? r : -r);
                i0 = i1 = 0.0;
            } else {
                const double r = sqrt(-disc);
                r0 = r1 = mid;
                i0 = r;
                i1 = -r;
            }
            if ((threadIdx.x & 31) == 0) {
                wr[hi - 1] = r0;
                wr[hi] = r1;
                wi[hi - 1] = i0;
                wi[hi] = i1;
            }
            __syncwarp();
            hi -= 2;
            its = 0;
            continue;
        }
        if (++total > 60 * m) return -1;
        ++its;
        double sh, dt;
        if (its % 11 == 10) {  // exceptional shift
            const double w = fabs(A[hi * m + hi - 1]) + fabs(A[(hi - 1) * m + hi - 2]);
            sh = 2.0 * A[hi * m + hi] + 1.5 * w;
            dt = (A[hi * m + hi] + 0.75 * w) * (A[hi * m + hi] + 0.75 * w) - 0.4375 * w * w;
        } else {
            const double a = A[(hi - 1) * m + hi - 1], b = A[(hi - 1) * m + hi];
            const double c = A[hi * m + hi - 1], d = A[hi * m + hi];
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
            const int cl = (k > lo) ? k - 1 : lo;
            const int rh = (k + 3 < hi) ? k + 3 : hi;
            apply_small_w(A, m, k, 3, cl, m - 1, 0, rh, u, tau);
            if (k > lo) {
                if ((threadIdx.x & 31) == 0) A[(k + 1) * m + k - 1] = A[(k + 2) * m + k - 1] = 0.0;
                __syncwarp();
            }
            x[0] = A[(k + 1) * m + k];
            x[1] = A[(k + 2) * m + k];
            x[2] = (k < hi - 2) ? A[(k + 3) * m + k] : 0.0;
        }
        small_house(2, x, u, tau);
        apply_small_w(A, m, hi - 1, 2, hi - 2, m - 1, 0, hi, u, tau);
        lw_put(&A[hi * m + hi - 2], 0.0);
    }
    return 0;
}

// Solve M x = b in place (Gaussian elimination with partial pivoting; a lane per row of
// each elimination step, back substitution with warp sums), M n x n (n <= 32) and b in
// shared memory; tiny pivots are replaced by a tiny number.
__device__ static void lu_solve_w(double* Mx, int n, double* b, double tiny) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < n; ++k) {
        // pivot: the first row of largest |M[r][k]|, r >= k
        double best = (lane >= k && lane < n) ? fabs(Mx[lane * n + k]) : -1.0;
        int p = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(LNO_FULL, best, o);
            const int op = __shfl_xor_sync(LNO_FULL, p, o);
            if (ob > best || (ob == best && op < p)) {
                best = ob;
                p = op;
            }
        }
        if (p != k) {
            if (lane < n) {
                const double t = Mx[k * n + lane];
                Mx[k * n + lane] = Mx[p * n + lane];
                Mx[p * n + lane] = t;
            }
            if (lane == 0) {
                const double t = b[k];
                b[k] = b[p];
                b[p] = t;
            }
            __syncwarp();
        }
        if (fabs(Mx[k * n + k]) < tiny) lw_put(&Mx[k * n + k], Mx[k * n + k] < 0 ? -tiny : tiny);
        const double inv = 1.0 / Mx[k * n + k];
        if (lane > k && lane < n) {
            const double f = Mx[lane * n + k] * inv;
            if (f != 0.0) {
                for (int c = k + 1; c < n; ++c) Mx[lane * n + c] -= f * Mx[k * n + c];
                b[lane] -= f * b[k];
            }
        }
        __syncwarp();
    }
    for (int r = n - 1; r >= 0; --r) {
        const double s = b[r] - warp_sum((lane > r && lane < n) ? Mx[r * n + lane] * b[lane] : 0.0);
        lw_put(&b[r], s / Mx[r * n + r]);
    }
}

// Cyclic Jacobi (Golub & Van Loan, Sec. 8.5) on the symmetric m x m matrix A: the
// eigenvalues are left on its diagonal, the rotations accumulate in Y (eigenvectors in
// columns), a lane per row or column of each rotation.  Returns 0 once the
// off-diagonal mass is below 1e-30 of the total, 1 after 50 sweeps without.
__device__ static int jacobi_w(double* A, double* Y, int m) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < m * m; e += 32) Y[e] = (e / m == e % m) ? 1.0 : 0.0;
    __syncwarp();
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = lane; e < m * m; e += 32) {
            const double v = A[e] * A[e];
            tot += v;
            if (e / m != e % m) off += v;
        }
        off = warp_sum(off);
        tot = warp_sum(tot);
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
                __syncwarp();  // every lane has read the entries above
                if (lane < m) {  // columns p, q: row `lane`
                    const double up = A[lane * m + p], uq = A[lane * m + q];
                    A[lane * m + p] = cs * up - sn * uq;
                    A[lane * m + q] = sn * up + cs * uq;
                }
                __syncwarp();
                if (lane < m) {  // rows p, q: column `lane`
                    const double pu = A[p * m + lane], qu = A[q * m + lane];
                    A[p * m + lane] = cs * pu - sn * qu;
                    A[q * m + lane] = sn * pu + cs * qu;
                    const double yp = Y[lane * m + p], yq = Y[lane * m + q];
                    Y[lane * m + p] = cs * yp - sn * yq;
                    Y[lane * m + q] = sn * yp + cs * yq;
                }
                __syncwarp();
            }
    }
    return 1;
}

// x <- x / ||x|| for the first n entries of x (shared memory)
__device__ static void normalise_w(double* x, int n) {
    const int lane = threadIdx.x & 31;
    const double t = lane < n ? x[lane] : 0.0;
    const double nr = rsqrt(warp_sum(t * t));
    __syncwarp();
    if (lane < n) x[lane] = t * nr;
    __syncwarp();
}

// Eigenvalue order of this atom (ord in shared memory, written by lane 0): real parts
// descending, then imaginary parts descending (insertion sort, stable)
__device__ static void order_w(const double* wr, const double* wi, int m, int* ord) {
    if ((threadIdx.x & 31) == 0) {
        for (int t = 0; t < m; ++t) ord[t] = t;
        for (int a = 1; a < m; ++a) {
            const int v = ord[a];
            int b = a - 1;
            while (b >= 0 && (wr[ord[b]] < wr[v] || (wr[ord[b]] == wr[v] && wi[ord[b]] < wi[v]))) {
                ord[b + 1] = ord[b];
                --b;
            }
            ord[b + 1] = v;
        }
    }
    __syncwarp();
}

// Per-warp shared-memory workspace of k_lno_eig (doubles): the work matrix A, the
// Cholesky factor Lc and Jacobi rotations Y (symmetric mode), the 2m x 2m system B of the
// complex inverse iteration, the basis V (m x k), the iterate z (2m), a reflector u, the
// eigenvalues (wr, wi) and their order (ints)
#define LW_A 0
#define LW_LC (LW_A + MM * MM)
#define LW_Y (LW_LC + MM * MM)
#define LW_B (LW_Y + MM * MM)
#define LW_V (LW_B + 4 * MM * MM)
#define LW_Z (LW_V + MM * MM)
#define LW_U (LW_Z + 2 * MM)
#define LW_WR (LW_U + MM)
#define LW_WI (LW_WR + MM)
#define LW_ORD (LW_WI + MM)
#define LW_DOUBLES (LW_ORD + MM)
#define LNO_WARPS 2  // atoms per CTA (34 KB of shared memory)

// ---------------------------------------------------------------------------
// One warp per atom.  SYM = false: Lam holds Lambda_0i (the paper's problem);
// SYM = true: Lam holds G_i = (S rho S)_{0i,0i} (k_projector).
// ---------------------------------------------------------------------------
template <bool SYM>
__global__ void __launch_bounds__(LNO_WARPS * 32)
    k_lno_eig(int N, int k, int use_th, double lam_th, const int* __restrict__ norb,
              const long long* __restrict__ loff, const long long* __restrict__ moff,
              const long long* __restrict__ voff, const long long* __restrict__ onsite,
              const long long* __restrict__ blk_off, const double* __restrict__ S, const double* __restrict__ Lam,
              double* __restrict__ Vout, double* __restrict__ lam_re, double* __restrict__ lam_im,
              int* __restrict__ flags, int* __restrict__ kat, int* __restrict__ status) {
    __shared__ double lw_sm[LNO_WARPS * LW_DOUBLES];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * LNO_WARPS + (threadIdx.x >> 5);
    if (i >= N) return;  // the whole warp: nothing below synchronises the CTA
    double* ws = lw_sm + (size_t)(threadIdx.x >> 5) * LW_DOUBLES;
    double* A = ws + LW_A;
    double* V = ws + LW_V;
    double* z = ws + LW_Z;
    double* wr = ws + LW_WR;
    double* wi = ws + LW_WI;
    int* ord = reinterpret_cast<int*>(ws + LW_ORD);
    const int m = norb[i];
    const double* L = Lam + loff[i];
    double* Vi = Vout + voff[i];  // m x k, row-major
    const double* Sii = S + blk_off[onsite[i]];
    int fl = 0, got = 0;
    for (int e = lane; e < MM * MM; e += 32) V[e] = 0.0;
    if constexpr (SYM) {
        double* Lc = ws + LW_LC;
        double* Y = ws + LW_Y;
        // S_ii = Lc Lc^T (column j: the diagonal from a warp sum, a lane per row below)
        for (int e = lane; e < m * m; e += 32) Lc[e] = 0.0;
        __syncwarp();
        for (int j = 0; j < m; ++j) {
            const double s = Sii[j * m + j] - warp_sum(lane < j ? Lc[j * m + lane] * Lc[j * m + lane] : 0.0);
            if (!(s > 0.0)) {
                if (lane == 0) status[i] = ST_NOT_SPD;
                return;
            }
            const double dj = sqrt(s);
            if (lane == j) Lc[j * m + j] = dj;
            if (lane > j && lane < m) {
                double v = Sii[lane * m + j];
                for (int u = 0; u < j; ++u) v -= Lc[lane * m + u] * Lc[j * m + u];
                Lc[lane * m + j] = v / dj;
            }
            __syncwarp();
        }
        // A = Lc^-1 Gs Lc^-T with Gs the symmetric part of G: two forward substitutions
        // (a lane per column; Lc^-1 Gs, transposed, Lc^-1 again), then symmetrised
        for (int e = lane; e < m * m; e += 32) {
            const int r = e / m, c = e % m;
            A[e] = 0.5 * (L[r * m + c] + L[c * m + r]);
        }
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
            if (lane < m)
                for (int r = 0; r < m; ++r) {
                    double v = A[r * m + lane];
                    for (int u = 0; u < r; ++u) v -= Lc[r * m + u] * A[u * m + lane];
                    A[r * m + lane] = v / Lc[r * m + r];
                }
            __syncwarp();
            for (int e = lane; e < m * m; e += 32) {
                const int r = e / m, c = e % m;
                if (r < c) {
                    const double x = A[r * m + c];
                    A[r * m + c] = A[c * m + r];
                    A[c * m + r] = x;
                }
            }
            __syncwarp();
        }
        for (int e = lane; e < m * m; e += 32) {
            const int r = e / m, c = e % m;
            if (r < c) {
                const double x = 0.5 * (A[r * m + c] + A[c * m + r]);
                A[r * m + c] = x;
                A[c * m + r] = x;
            }
        }
        __syncwarp();
        if (jacobi_w(A, Y, m) != 0) {
            if (lane == 0) status[i] = ST_NOT_CONVERGED;
            return;
        }
        // eigenvalues descending (ties: lower index first)
        if (lane < m) {
            wr[lane] = A[lane * m + lane];
            wi[lane] = 0.0;
        }
        __syncwarp();
        order_w(wr, wi, m, ord);
        if (lane < m) {
            lam_re[moff[i] + lane] = wr[ord[lane]];
            lam_im[moff[i] + lane] = 0.0;
        }
        // the leading k (with the threshold: those >= lambda_th), v = Lc^-T y by back
        // substitution with warp sums
        while (got < k && got < m && !(use_th && wr[ord[got]] < lam_th)) {
            const int col = ord[got];
            for (int r = m - 1; r >= 0; --r) {
                const double t = (lane > r && lane < m) ? Lc[lane * m + r] * V[lane * k + got] : 0.0;
                const double v = Y[r * m + col] - warp_sum(t);
                lw_put(&V[r * k + got], v / Lc[r * m + r]);
            }
            ++got;
        }
    } else {
        double* u = ws + LW_U;
        double* B = ws + LW_B;
        double an = 0.0;
        for (int e = lane; e < m * m; e += 32) {
            A[e] = L[e];
            an += L[e] * L[e];
        }
        double anorm = sqrt(warp_sum(an));
        if (anorm == 0.0) anorm = 1.0;
        __syncwarp();
        hessenberg_w(A, m, u);
        if (francis_qr_w(A, m, wr, wi) != 0) {
            if (lane == 0) status[i] = ST_NOT_CONVERGED;
            return;
        }
        // order: real part descending, then imaginary part descending
        order_w(wr, wi, m, ord);
        if (lane < m) {
            lam_re[moff[i] + lane] = wr[ord[lane]];
            lam_im[moff[i] + lane] = wi[ord[lane]];
        }
        // eigenvectors of the leading eigenvalues by inverse iteration
        int pos = 0;
        const double tiny = 1e-300;
        while (got < k && pos < m) {
            const double lr = wr[ord[pos]], li = wi[ord[pos]];
            if (use_th && lr < lam_th) break;  // threshold selection: eigenvalues >= lambda_th only
            const double sh = lr + 1e-13 * anorm;  // shifted off the eigenvalue to keep the solve regular
            if (li == 0.0) {
                if (lane < m) z[lane] = 1.0 + 0.01 * lane;
                __syncwarp();
                for (int it = 0; it < 4; ++it) {
                    for (int e = lane; e < m * m; e += 32) A[e] = L[e] - ((e / m == e % m) ? sh : 0.0);
                    __syncwarp();
                    lu_solve_w(A, m, z, tiny * anorm);
                    normalise_w(z, m);
                }
                if (lane < m) V[lane * k + got] = z[lane];
                __syncwarp();
                ++got;
                ++pos;
            } else {
                // (Lambda - (sh + i li) I)(x + i y) = b in real form:
                // [[Lambda - sh I, li I], [-li I, Lambda - sh I]] [x; y] = [br; bi]
                fl |= DCLNO_LNO_COMPLEX_SELECTED;
                const int n2 = 2 * m;
                if (lane < n2) z[lane] = (lane < m) ? 1.0 + 0.01 * lane : 0.02 * (lane - m);
                __syncwarp();
                for (int it = 0; it < 4; ++it) {
                    for (int e = lane; e < m * m; e += 32) {
                        const int r = e / m, c = e % m;
                        const double a = L[e] - (r == c ? sh : 0.0);
                        B[r * n2 + c] = a;
                        B[(r + m) * n2 + c + m] = a;
                        B[r * n2 + c + m] = (r == c) ? li : 0.0;
                        B[(r + m) * n2 + c] = (r == c) ? -li : 0.0;
                    }
                    __syncwarp();
                    lu_solve_w(B, n2, z, tiny * anorm);
                    normalise_w(z, n2);
                }
                // phase: the first component of largest magnitude made real and positive
                double a2 = (lane < m) ? z[lane] * z[lane] + z[lane + m] * z[lane + m] : -1.0;
                int jm = lane;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double oa = __shfl_xor_sync(LNO_FULL, a2, o);
                    const int oj = __shfl_xor_sync(LNO_FULL, jm, o);
                    if (oa > a2 || (oa == a2 && oj < jm)) {
                        a2 = oa;
                        jm = oj;
                    }
                }
                const double pr = z[jm], pi = z[jm + m], pn = rsqrt(pr * pr + pi * pi);
                const double cr = pr * pn, ci = -pi * pn;  // multiply by conj(z_jm)/|z_jm|
                if (lane < m) {
                    const double zr = z[lane], zi = z[lane + m];
                    V[lane * k + got] = zr * cr - zi * ci;
                    if (got + 1 < k) V[lane * k + got + 1] = zr * ci + zi * cr;
                }
                __syncwarp();
                ++got;
                if (got < k) ++got;
                else fl |= DCLNO_LNO_PAIR_SPLIT;
                pos += 2;
            }
        }
    }
    // S_ii-orthonormal basis of the span (Gram-Schmidt in eigenvalue order, twice; a lane
    // per row, S_ii x by rows); the columns beyond this atom's count (threshold
    // selection) stay zero
    const int kk = got;
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < kk; ++c) {
            for (int d = 0; d < c; ++d) {
                // coefficient <v_d, v_c>_S, then v_c -= h v_d
                double t = 0.0;
                if (lane < m)
                    for (int s = 0; s < m; ++s) t += Sii[lane * m + s] * V[s * k + c];
                const double h = warp_sum(lane < m ? V[lane * k + d] * t : 0.0);
                if (lane < m) V[lane * k + c] -= h * V[lane * k + d];
                __syncwarp();
            }
            double t = 0.0;
            if (lane < m)
                for (int s = 0; s < m; ++s) t += Sii[lane * m + s] * V[s * k + c];
            double nn = warp_sum(lane < m ? V[lane * k + c] * t : 0.0);
            if (!(nn > 0.0)) {
                if (lane == 0) status[i] = ST_BAD_LNO;
                return;
            }
            nn = rsqrt(nn);
            __syncwarp();
            if (lane < m) V[lane * k + c] *= nn;
            __syncwarp();
        }
    }
    // sign: the first entry of largest magnitude positive
    for (int c = 0; c < kk; ++c) {
        double a = (lane < m) ? fabs(V[lane * k + c]) : -1.0;
        int jm = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double oa = __shfl_xor_sync(LNO_FULL, a, o);
            const int oj = __shfl_xor_sync(LNO_FULL, jm, o);
            if (oa > a || (oa == a && oj < jm)) {
                a = oa;
                jm = oj;
            }
        }
        const bool neg = V[jm * k + c] < 0.0;
        __syncwarp();
        if (neg && lane < m) V[lane * k + c] = -V[lane * k + c];
        __syncwarp();
    }
    for (int e = lane; e < m * k; e += 32) Vi[e] = V[e];
    if (lane == 0) {
        flags[i] = fl;
        kat[i] = kk;
        status[i] = ST_OK;
    }
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
        kern<<<(N + LNO_WARPS - 1) / LNO_WARPS, LNO_WARPS * 32, 0, c->stream>>>(N, c->k_lno, use_th, c->lno_th, c->d_norb, c->d_loff, c->d_moff,
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
