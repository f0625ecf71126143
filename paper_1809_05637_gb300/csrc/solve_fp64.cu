// FP64 solver of the truncated-cluster eigenproblems H^(i) c = eps S^(i) c
// (Sec. II.C step (iii)), batched over all clusters.
//
//   k_cholesky     S^(i) = L L^T                 blocked right-looking, DMMA trailing updates
//   k_congruence   A = L^-1 H^(i) L^-T           two blocked right-side triangular solves
//   k_tridiag      A = Q T Q^T                   blocked Householder (DFMA symv, DMMA rank-2k);
//                                                 T torn at n/2 into two halves (Cuppen)
//   k_ql           T1, T2 = Z_k Theta_k Z_k^T    implicit QL per half; rotations logged, not accumulated
//   k_merge        (merge.cu)                    rank-one merge: eigenvalues of T and the merge matrix M
//   k_apply_q_rows P <- P Q                       central rows [L_cc^-T | L_c,:] times Q
//   k_replay_fwd   P <- P diag(Z1, Z2)            the logged rotations applied to P's columns
//   k_mgemm        P <- P M                       (Z = diag(Z1, Z2) M)
//   k_weights      q_mu = sum_a (C_c)_{a mu} (S C)_{c a, mu}, eigenvalues out
// The same kernels with EMU = true are the mixed path: the tile updates of
// Cholesky, congruence, tridiagonalisation and the merge products run on BF16
// tensor cores with FP64 emulated by 8-bit slices (emu_gemm.cuh).
//
// The central atom is the last member of its cluster, so the central rows of
// C = L^-T Q Z are L_cc^-T (Q Z)_c and those of S C = L Q Z are L_c,: Q Z: both
// need only the M_i x n strips, never the full eigenvector matrix (Eq. (Gi) is
// evaluated through these strips).
#include "dclno_internal.cuh"
#include "emu_gemm.cuh"

#define NB DCLNO_NB
#define DK_LD 33

// x L_kk^T = h for rows [r0, r1) of M (columns kb .. kb+nb-1), L_kk in smem (lower),
// reciprocals of its diagonal in invd.
__device__ static void panel_solve_rows(double* M, int ld, int kb, int nb, int r0, int r1, const double* Dk,
                                        const double* invd) {
    for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) {
        double x[NB];
        double* row = M + (size_t)r * ld + kb;
#pragma unroll
        for (int j = 0; j < NB; ++j) x[j] = (j < nb) ? row[j] : 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j < nb) {
                double s = x[j];
#pragma unroll
                for (int t = 0; t < j; ++t) s = fma(-x[t], Dk[j * DK_LD + t], s);
                x[j] = s * invd[j];
            }
        }
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j < nb) row[j] = x[j];
    }
}

// load the lower triangle of the factor's diagonal block into smem and form 1/diag
__device__ static void load_diag_block(const double* L, int ld, int kb, int nb, double* Dk, double* invd) {
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        Dk[r * DK_LD + c] = (r < nb && c <= r) ? L[(size_t)(kb + r) * ld + kb + c] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < nb) invd[threadIdx.x] = 1.0 / Dk[threadIdx.x * DK_LD + threadIdx.x];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Cholesky of S^(i) in place (lower); sets ST_NOT_SPD on a non-positive pivot.
// ---------------------------------------------------------------------------
template <int EMU>
__device__ __forceinline__ void cholesky_one(const ClusterDesc* __restrict__ cls, int ci, double* __restrict__ arena,
                                             int* __restrict__ status, TcState* tcs) {
    extern __shared__ double sm[];
    double* Dk = sm;                   // NB x DK_LD
    double* invd = sm + NB * DK_LD;    // NB
    double* G = invd + NB;             // GEMM tiles
    __shared__ int fail;
    const ClusterDesc d = cls[ci];
    const int n = d.n, ld = d.ld;
    double* L = arena + d.mat_off + (size_t)n * ld;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int kb = 0; kb < n; kb += NB) {
        const int nb = min(NB, n - kb);
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
            const int r = e / NB, c = e % NB;
            Dk[r * DK_LD + c] = (r < nb && c <= r) ? L[(size_t)(kb + r) * ld + kb + c] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            for (int j = 0; j < nb; ++j) {
                const double djj = Dk[j * DK_LD + j];
                if (!(djj > 0.0)) {
                    if (lane == 0) fail = 1;
                    break;
                }
                const double ljj = sqrt(djj), inv = 1.0 / ljj;
                __syncwarp();
                if (lane == j) {
                    Dk[j * DK_LD + j] = ljj;
                    invd[j] = inv;
                }
                if (lane > j && lane < nb) Dk[lane * DK_LD + j] *= inv;
                __syncwarp();
                if (lane > j && lane < nb) {
                    const double lij = Dk[lane * DK_LD + j];
                    for (int t = j + 1; t <= lane; ++t) Dk[lane * DK_LD + t] -= lij * Dk[t * DK_LD + j];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (fail) {
            if (threadIdx.x == 0) status[ci] = ST_NOT_SPD;
            return;
        }
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int r = e / nb, c = e % nb;
            if (c <= r) L[(size_t)(kb + r) * ld + kb + c] = Dk[r * DK_LD + c];
        }
        panel_solve_rows(L, ld, kb, nb, kb + nb, n, Dk, invd);
        __syncthreads();
        const int m2 = n - kb - nb;
        if (m2 > 0) {
            double* P = L + (size_t)(kb + nb) * ld + kb;
            tile_update<true, EMU>(P + nb, ld, P, ld, P, ld, m2, m2, nb, 0, G, tcs);
        }
    }
    if (threadIdx.x == 0) status[ci] = (EMU == 2 && tcs->failed) ? ST_TIMEOUT : ST_OK;
}


template <int EMU>
__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS, DCLNO_CTAS_PER_SM(EMU)) k_cholesky(
    const ClusterDesc* __restrict__ cls, const int* __restrict__ order, double* __restrict__ arena,
    int* __restrict__ status, int nitems, int* __restrict__ queue) {
    CUBIC_KERNEL_LOOP(EMU, cholesky_one<EMU>(cls, order[it], arena, status, &tcs))
}

// ---------------------------------------------------------------------------
// A = L^-1 H L^-T, lower triangle valid on exit (in place of H^(i)).
// Y = H L^-T (all rows), transpose, then A = Y^T L^-T restricted to the lower part.
// ---------------------------------------------------------------------------
template <int EMU>
__device__ __forceinline__ void congruence_one(const ClusterDesc* __restrict__ cls, int ci, double* __restrict__ arena,
                                               int* __restrict__ status, TcState* tcs) {
    extern __shared__ double sm[];
    double* Dk = sm;
    double* invd = sm + NB * DK_LD;
    double* G = invd + NB;
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    const int n = d.n, ld = d.ld;
    double* A = arena + d.mat_off;
    const double* L = A + (size_t)n * ld;
    for (int kb = 0; kb < n; kb += NB) {
        const int nb = min(NB, n - kb);
        load_diag_block(L, ld, kb, nb, Dk, invd);
        panel_solve_rows(A, ld, kb, nb, 0, n, Dk, invd);
        __syncthreads();
        const int n2 = n - kb - nb;
        if (n2 > 0)
            tile_update<false, EMU>(A + kb + nb, ld, A + kb, ld, L + (size_t)(kb + nb) * ld + kb, ld, n, n2, nb, 0, G,
                                    tcs);
    }
    // in-place transpose
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = 1 + warp; r < n; r += nw) {
        for (int c = lane; c < r; c += 32) {
            const double a = A[(size_t)r * ld + c], b = A[(size_t)c * ld + r];
            A[(size_t)r * ld + c] = b;
            A[(size_t)c * ld + r] = a;
        }
    }
    __syncthreads();
    for (int kb = 0; kb < n; kb += NB) {
        const int nb = min(NB, n - kb);
        load_diag_block(L, ld, kb, nb, Dk, invd);
        panel_solve_rows(A, ld, kb, nb, kb, n, Dk, invd);
        __syncthreads();
        const int m2 = n - kb - nb;
        if (m2 > 0) {
            double* C = A + (size_t)(kb + nb) * ld + kb + nb;
            tile_update<true, EMU>(C, ld, A + (size_t)(kb + nb) * ld + kb, ld, L + (size_t)(kb + nb) * ld + kb, ld, m2, m2,
                                  nb, 0, G, tcs);
        }
    }
    if (EMU == 2 && tcs->failed && threadIdx.x == 0) status[ci] = ST_TIMEOUT;
}

template <int EMU>
__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS, DCLNO_CTAS_PER_SM(EMU)) k_congruence(
    const ClusterDesc* __restrict__ cls, const int* __restrict__ order, double* __restrict__ arena,
    int* __restrict__ status, int nitems, int* __restrict__ queue) {
    CUBIC_KERNEL_LOOP(EMU, congruence_one<EMU>(cls, order[it], arena, status, &tcs))
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation of the lower triangle of A (blocked, panels of NB).
// On exit: d (diagonal), e (sub-diagonal), tau; reflector k is (1, A[k+2:, k]) acting
// on rows k+1.. (A[k+1][k] holds the unit element).
// ---------------------------------------------------------------------------
template <int EMU>
__device__ __forceinline__ void tridiag_one(const ClusterDesc* __restrict__ cls, int ci, double* __restrict__ arena,
                                            int* __restrict__ status, int skip_two_stage, TcState* tcs) {
    extern __shared__ double sm[];
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    if (skip_two_stage && two_stage_cluster(d)) return;  // reduced by k_band + k_chase instead
    const int n = d.n, ld = d.ld;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double* A = arena + d.mat_off;
    double* dv = arena + d.aux_off;  // sub-regions padded to ld (16-byte aligned)
    double* ev = dv + ld;
    double* tauv = dv + 2 * ld;
    double* W = dv + 3 * ld;  // n x NB
    double* vs = sm;                  // n
    double* ys = sm + n;              // n
    double* yw = sm + 2 * n;          // nw x n
    double* red = yw + (size_t)nw * n;  // 2*NB + 32
    double* pc = red + 32;            // NB: W^T v
    double* sc = pc + NB;             // NB: V^T v
    double* G = sm;                   // GEMM tiles alias the vectors between panels

    for (int c0 = 0; c0 < n; c0 += NB) {
        const int nb = min(NB, n - c0);
        for (int j = 0; j < nb; ++j) {
            const int c = c0 + j;
            // (1) bring column c up to date with the panel's earlier reflectors
            if (j > 0) {
                for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
                    double s = 0.0;
                    for (int t = 0; t < j; ++t)
                        s = fma(A[(size_t)r * ld + c0 + t], W[(size_t)c * NB + t],
                                fma(W[(size_t)r * NB + t], A[(size_t)c * ld + c0 + t], s));
                    A[(size_t)r * ld + c] -= s;
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) dv[c] = A[(size_t)c * ld + c];
            if (c >= n - 1) break;
            // (2) reflector for A[c+1:, c]; alpha is read before the barriers of block_sum,
            // which thread 0's overwrite of this element with the unit entry follows
            const double alpha = A[(size_t)(c + 1) * ld + c];
            double sig = 0.0;
            for (int r = c + 2 + threadIdx.x; r < n; r += blockDim.x) {
                const double a = A[(size_t)r * ld + c];
                sig = fma(a, a, sig);
            }
            sig = block_sum(sig, red);
            double tau = 0.0, beta = alpha, scale = 0.0;
            if (sig > 0.0) {
                const double nrm = sqrt(alpha * alpha + sig);
                beta = (alpha >= 0.0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            for (int r = c + 1 + threadIdx.x; r < n; r += blockDim.x) {
                double v = (r == c + 1) ? 1.0 : A[(size_t)r * ld + c] * scale;
                if (r > c + 1) A[(size_t)r * ld + c] = v;
                A[(size_t)c * ld + r] = v;  // contiguous copy in row c of the unused upper triangle
                vs[r] = v;
            }
            if (threadIdx.x == 0) {
                A[(size_t)(c + 1) * ld + c] = 1.0;
                ev[c] = beta;
                tauv[c] = tau;
            }
            __syncthreads();
            // (3) y = A22 v with A22 = A[c+1:, c+1:] (lower storage, not yet updated by this panel).
            // Row r contributes A[r][t] v_t to y_r (a sum over the warp) and A[r][t] v_r to y_t for
            // t < r (per-warp partials in shared memory).  A warp takes eight rows per pass, so each
            // shared-memory update carries eight rows' contributions and the eight row sums are
            // reduced together (warp_sum8: 9 FP64 adds per lane instead of 40).
            {
                double* yr = yw + (size_t)warp * n;
                for (int t = c + 1 + lane; t < n; t += 32) yr[t] = 0.0;
                __syncwarp();
                for (int r0 = c + 1 + warp; r0 < n; r0 += 8 * nw) {
                    int rr[8];
                    double vr[8], acc[8];
                    int rmax = r0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        rr[q] = r0 + q * nw;
                        const bool ok = rr[q] < n;
                        vr[q] = ok ? vs[rr[q]] : 0.0;
                        acc[q] = 0.0;
                        if (ok) rmax = rr[q];
                        else rr[q] = -1;
                    }
                    for (int t = c + 1 + lane; t <= rmax; t += 32) {
                        const double vt = vs[t];
                        double ysum = 0.0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (t <= rr[q]) {
                                const double a = A[(size_t)rr[q] * ld + t];
                                acc[q] = fma(a, vt, acc[q]);
                                if (t < rr[q]) ysum = fma(a, vr[q], ysum);
                            }
                        }
                        yr[t] += ysum;
                    }
                    const double a = warp_sum8(acc);  // lane L: row q = (L >> 2) & 7
                    int rq = -1;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (q == ((lane >> 2) & 7)) rq = rr[q];
                    if ((lane & 3) == 0 && rq >= 0) ys[rq] = a;
                }
            }
            __syncthreads();
            for (int t = c + 1 + threadIdx.x; t < n; t += blockDim.x) {
                double s = ys[t];
                for (int w = 0; w < nw; ++w) s += yw[(size_t)w * n + t];
                ys[t] = s;
            }
            // panel corrections: pc = W^T v, sc = V^T v over rows c+1..n-1
            for (int t = warp; t < j; t += nw) {
                double p = 0.0, q = 0.0;
                for (int r = c + 1 + lane; r < n; r += 32) {
                    p = fma(W[(size_t)r * NB + t], vs[r], p);
                    q = fma(A[(size_t)r * ld + c0 + t], vs[r], q);
                }
                p = warp_sum(p);
                q = warp_sum(q);
                if (lane == 0) {
                    pc[t] = p;
                    sc[t] = q;
                }
            }
            __syncthreads();
            double dot = 0.0;
            for (int r = c + 1 + threadIdx.x; r < n; r += blockDim.x) {
                double y = ys[r];
                for (int t = 0; t < j; ++t)
                    y = fma(-A[(size_t)r * ld + c0 + t], pc[t], fma(-W[(size_t)r * NB + t], sc[t], y));
                y *= tau;
                ys[r] = y;
                dot = fma(y, vs[r], dot);
            }
            dot = block_sum(dot, red);
            const double a2 = -0.5 * tau * dot;
            for (int r = c + 1 + threadIdx.x; r < n; r += blockDim.x) W[(size_t)r * NB + j] = fma(a2, vs[r], ys[r]);
            __syncthreads();
        }
        const int m2 = n - c0 - nb;
        if (m2 > 0) {
            double* C = A + (size_t)(c0 + nb) * ld + c0 + nb;
            const double* Vp = A + (size_t)(c0 + nb) * ld + c0;
            const double* Wp = W + (size_t)(c0 + nb) * NB;
            tile_update<true, EMU>(C, ld, Vp, ld, Wp, NB, m2, m2, nb, 0, G, tcs);
            tile_update<true, EMU>(C, ld, Wp, NB, Vp, ld, m2, m2, nb, 0, G, tcs);
        }
    }
    if (EMU == 2 && tcs->failed && threadIdx.x == 0) status[ci] = ST_TIMEOUT;
    // Cuppen's tear (tear_cluster): the segments are solved by QL and merged afterwards
    // (k_merge; for a cluster torn twice the halves first)
    __syncthreads();
    if (threadIdx.x == 0) tear_cluster(d, arena);
}

template <int EMU>
__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS, DCLNO_CTAS_PER_SM(EMU)) k_tridiag(
    const ClusterDesc* __restrict__ cls, const int* __restrict__ order, double* __restrict__ arena,
    int* __restrict__ status, int skip_two_stage, int nitems, int* __restrict__ queue) {
    CUBIC_KERNEL_LOOP(EMU, tridiag_one<EMU>(cls, order[it], arena, status, skip_two_stage, &tcs))
}

// ---------------------------------------------------------------------------
// Implicit QL on (d, e), one lane per cluster, lanes in lockstep.
// Every pass of the loop advances each lane by a burst of up to 32 plane
// rotations (phase ROT), the end of a sweep (FIN), up to 64 deflation checks
// (SEEK) and the Wilkinson-type shift of a new sweep (START), so a warp's FP64
// instructions serve all its clusters at once (an FP64 instruction costs the
// same whatever its number of active lanes).  A sweep records the two smallest
// negligible off-diagonals it leaves behind, so the next unreduced block is
// known without a scan of e; SEEK runs only at the start and after a whole
// block has converged.  Lanes are (cluster, segment) pairs of a torn problem (or
// the whole problem), with d, e and, for a torn problem, the row z = v Z of the merge
// (k_merge) kept in shared memory.  Rotations are logged as (c, s) per sweep:
// header block of a cluster = [nsweeps, (first rotation, first index i, count) x nsweeps],
// i decreasing within a sweep.
// ---------------------------------------------------------------------------
enum { QL_SEEK = 0, QL_START = 1, QL_ROT = 2, QL_FIN = 3, QL_DONE = 4 };

__device__ __forceinline__ int exp_bits(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// |e| negligible beside d_m, d_{m+1}: |e| < 2^-52 max(|d_m|, |d_{m+1}|), by exponents only
__device__ __forceinline__ bool negligible(double e, double d0, double d1) {
    if (e == 0.0) return true;
    const int ed = max(exp_bits(d0), exp_bits(d1));
    return exp_bits(e) + 53 <= ed;
}

template <bool X2>
__global__ void __launch_bounds__(32) k_ql(int ncl, int lanes, int segp, const ClusterDesc* __restrict__ cls,
                                           const int* __restrict__ order, double* __restrict__ arena,
                                           int* __restrict__ iters, int* __restrict__ status) {
    extern __shared__ double sm[];
    // lane = (problem, segment); the lane's d, e, z row and extra row live in shared memory
    // (segp each).  A problem is a cluster torn once or a half of a cluster torn twice.
    const int t = blockIdx.x * lanes + threadIdx.x;
    int phase = QL_DONE, n = 0, si = -1;
    // X2 when the problems include halves (their extra rows: four arrays per lane, else
    // three; shared memory per lane bounds how many QL chains an SM holds)
    constexpr int narr = X2 ? 4 : 3;
    double* d = sm + (size_t)threadIdx.x * narr * segp;
    double* e = d + segp;
    double* x = e + segp;   // z row of a torn problem: v diag(Z1, Z2) restricted to this segment
    double* x2 = x + segp;  // the extra row a half carries for its cluster's merge (narr = 4)
    double* dg = nullptr;   // the segment's d in global memory (eigenvalues out)
    double* zg = nullptr;   // the segment's part of z (torn problems only)
    double* x2g = nullptr;  // the segment's extra row out (halves only)
    double2* rot = nullptr;
    int* hdr = nullptr;
    int rot_cap = 0, sw_cap = 0;
    if (threadIdx.x < lanes && t < 2 * ncl) {
        const ClusterDesc dsc = cls[order[t >> 1]];
        const int sg = t & 1;
        si = dsc.sidx;
        if (status[si] == ST_OK) {
            n = seg_len(dsc, sg);
            if (n > 0) {
                dg = arena + dsc.aux_off + seg_start(dsc, sg);
                for (int k = 0; k < n; ++k) {
                    d[k] = dg[k];
                    e[k] = dg[dsc.ld + k];
                    x[k] = 0.0;
                }
                if (dsc.split) {
                    // v = e_{k-1} + sign(beta) e_k, beta kept by the tear at [n] of the z row
                    double* W = arena + dsc.w_off;
                    zg = W + seg_start(dsc, sg);
                    if (sg == 0) x[n - 1] = 1.0;
                    else x[0] = (W[dsc.n] < 0.0) ? -1.0 : 1.0;
                }
                if (X2 && ((dsc.x2_mode == 1 && sg == 0) || (dsc.x2_mode == 2 && sg == 1))) {
                    // e_first of the second half's first segment, e_last of the first half's second
                    x2g = arena + dsc.x2_off + dsc.g_row0 + seg_start(dsc, sg);
                    for (int k = 0; k < n; ++k) x2[k] = 0.0;
                    x2[dsc.x2_mode == 1 ? 0 : n - 1] = 1.0;
                }
                rot = reinterpret_cast<double2*>(arena + dsc.rot_off) + (size_t)sg * dsc.rot_cap;
                hdr = iters + dsc.it_off + (size_t)sg * dsc.it_cap;
                rot_cap = dsc.rot_cap;
                sw_cap = (dsc.it_cap - 1) / 3;
                e[n - 1] = 0.0;
                phase = (n > 1) ? QL_SEEK : QL_DONE;
                if (n <= 1) hdr[0] = 0;
            }
        }
    }
    int l = 0, m = 0, mm = 0, i = 0, it = 0, nrot = 0, nsw = 0, start = 0;
    double zx1 = 0.0;  // z row: value of the row the sweep carries (crow), updated with each rotation
    double zx2 = 0.0;  // the same for the extra row
    int crow = 0;
    // the two smallest indices in [l, m] whose e is negligible after this sweep (m counts
    // as negligible): the next unreduced block is known without scanning e again
    int lowneg = 0, low2 = 0;
    double s = 1.0, c = 1.0, p = 0.0, g = 0.0;
    double ce = 0.0, cd0 = 0.0, cd1 = 0.0;  // e[i], d[i], d[i+1] of the current rotation
    double ne = 0.0, nd = 0.0;              // e[i-1], d[i-1] loaded one rotation ahead
    double dnext = 0.0;                     // new d[i+2] written by the previous rotation
    while (__any_sync(0xffffffffu, phase != QL_DONE)) {
        // a burst of rotations: lanes outside a sweep are predicated off, the FP64
        // instructions of one rotation serve every lane that is inside one
#pragma unroll 1
        for (int u = 0; u < 32; ++u) {
            if (phase != QL_ROT) continue;
            const double f = s * ce, b = c * ce;
            const double ss = fma(f, f, g * g);
            double r;
            if (exp_bits(ss) < 64) {
                // tiny or zero: the careful hypot path (rare)
                r = hypot(f, g);
                if (r == 0.0) {
                    e[i + 1] = 0.0;
                    d[i + 1] = cd1 - p;
                    e[m] = 0.0;
                    low2 = lowneg;
                    lowneg = i + 1;  // e[i+1] = 0: the next block ends here
                    phase = QL_FIN;  // the sweep ends early, d[l] and e[l] untouched
                    continue;
                }
                s = f / r;
                c = g / r;
            } else {
                const double ti = rsqrt(ss);
                r = ss * ti;
                s = f * ti;
                c = g * ti;
            }
            e[i + 1] = r;
            g = cd1 - p;
            const double rr = fma(cd0 - g, s, (b + b) * c);
            p = s * rr;
            const double dn = g + p;
            d[i + 1] = dn;
            g = fma(c, rr, -b);
            rot[nrot++] = make_double2(c, s);
            {  // the same rotation on the z row (off the recurrence's critical path)
                const double xi = x[i];
                x[i + 1] = fma(s, xi, c * zx1);
                zx1 = fma(c, xi, -s * zx1);
                crow = i;
            }
            if (X2 && x2g) {
                const double xi = x2[i];
                x2[i + 1] = fma(s, xi, c * zx2);
                zx2 = fma(c, xi, -s * zx2);
            }
            // deflation bookkeeping for the next sweep: e[i+1], d[i+1], d[i+2] are final now
            if (i + 1 < m && negligible(r, dn, dnext)) {
                low2 = lowneg;
                lowneg = i + 1;
            }
            dnext = dn;
            if (--i < l) {
                const double dl = d[l] - p;
                d[l] = dl;
                e[l] = g;
                e[m] = 0.0;
                if (negligible(g, dl, dn)) {
                    low2 = lowneg;
                    lowneg = l;
                }
                phase = QL_FIN;
            } else {
                cd1 = cd0;
                cd0 = nd;
                ce = ne;
                if (i - 1 >= l) {
                    ne = e[i - 1];
                    nd = d[i - 1];
                }
            }
        }
        if (phase == QL_FIN) {
            x[crow] = zx1;
            if (X2 && x2g) x2[crow] = zx2;
            hdr[1 + 3 * nsw] = start;
            hdr[2 + 3 * nsw] = m - 1;
            hdr[3 + 3 * nsw] = nrot - start;
            ++nsw;
            if (lowneg > l) {
                m = lowneg;  // the unreduced block shrank: no scan needed
                phase = QL_START;
            } else {
                // d[l] converged; the block below it ends at low2 unless e[l+1] is negligible too
                ++l;
                it = 0;
                if (l >= n - 1) {
                    phase = QL_DONE;
                    hdr[0] = nsw;
                } else if (low2 > l) {
                    m = low2;
                    phase = QL_START;
                } else {
                    mm = l;
                    phase = QL_SEEK;
                }
            }
        }
        if (phase == QL_SEEK) {
#pragma unroll 1
            for (int u = 0; u < 64 && phase == QL_SEEK; ++u) {
                if (mm == n - 1 || negligible(e[mm], d[mm], d[mm + 1])) {
                    if (mm == l) {
                        ++l;
                        it = 0;
                        mm = l;
                        if (l >= n - 1) {
                            phase = QL_DONE;
                            hdr[0] = nsw;
                        }
                    } else {
                        m = mm;
                        phase = QL_START;
                    }
                } else {
                    ++mm;
                }
            }
        }
        if (phase == QL_START) {
            if (++it > 60) {
                status[si] = ST_NOT_CONVERGED;
                hdr[0] = nsw;
                phase = QL_DONE;
            } else if (nsw >= sw_cap || nrot + (m - l) > rot_cap) {
                status[si] = ST_LOG_FULL;
                hdr[0] = nsw;
                phase = QL_DONE;
            } else {
                const double dl = d[l], dl1 = d[l + 1], el = e[l], dm = d[m];
                g = (dl1 - dl) / (2.0 * el);
                const double r = hypot(g, 1.0);
                g = dm - dl + el / (g + copysign(r, g));
                s = 1.0;
                c = 1.0;
                p = 0.0;
                i = m - 1;
                start = nrot;
                lowneg = m;
                low2 = m;
                zx1 = x[m];
                if (X2 && x2g) zx2 = x2[m];
                crow = m;
                ce = e[i];
                cd0 = d[i];
                cd1 = dm;
                dnext = (m + 1 < n) ? d[m + 1] : 0.0;
                if (i - 1 >= l) {
                    ne = e[i - 1];
                    nd = d[i - 1];
                }
                phase = QL_ROT;
            }
        }
    }
    for (int k = 0; k < n; ++k) dg[k] = d[k];
    if (zg)
        for (int k = 0; k < n; ++k) zg[k] = x[k];
    if (X2 && x2g)
        for (int k = 0; k < n; ++k) x2g[k] = x2[k];
}

// ---------------------------------------------------------------------------
// Central strips: P ([n][2 mc], column t holds the 2 mc values of the strips at t)
// initialised to R1 = (L^-T)_c,: = [0 | L_cc^-T] and R2 = L_c,:, then P <- P Q with
// Q = H_0 H_1 ... H_{n-3}.  Each strip row is independent: chunks of rch rows are held
// in shared memory (row-major, stride n) and each warp applies every reflector to the
// rows it owns (q_rows_warp), so there is no block barrier per reflector.
// ---------------------------------------------------------------------------
// X <- X H_0 H_1 ... H_{n-3} on R rows owned by one warp (one-stage reduction), or
// X <- X Q1 Q2 (two-stage reduction, q2 = the chase log)
template <int R>
__device__ static void q_rows_warp(double* X, int n, const double* __restrict__ A, int ld, const double* __restrict__ tau,
                                   const double* __restrict__ q2) {
    if (q2) {
        warp_apply_two_stage<R>(X, n, A, ld, tau, q2, 0);
        return;
    }
    for (int k = 0; k + 2 < n; ++k) {
        const double tk = tau[k];
        if (tk != 0.0) warp_reflect<R>(X, n, k, n, A + (size_t)k * ld, tk);
    }
}

__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS) k_apply_q_rows(const ClusterDesc* __restrict__ cls,
                                                                      const int* __restrict__ order,
                                                                      double* __restrict__ arena,
                                                                      const int* __restrict__ status, int rch,
                                                                      int two_stage) {
    extern __shared__ double sm[];
    const int ci = order[blockIdx.x];
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    const int n = d.n, ld = d.ld, mc = d.mc, w2 = 2 * mc, c0 = n - mc;
    const double* q2 = (two_stage && two_stage_cluster(d)) ? arena + d.q2_off : nullptr;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* A = arena + d.mat_off;
    const double* L = A + (size_t)n * ld;
    const double* tau = arena + d.aux_off + 2 * ld;
    double* P = arena + d.cc_off;
    double* Li = sm;                               // mc x mc inverse of L_cc
    double* Xs = sm + DCLNO_MAX_M * DCLNO_MAX_M;   // rch x n strip rows
    // L_cc^-1 by forward substitution, one column per thread
    if (threadIdx.x < mc) {
        const int col = threadIdx.x;
        for (int r = 0; r < mc; ++r) {
            double s = (r == col) ? 1.0 : 0.0;
            for (int k = col; k < r; ++k) s -= L[(size_t)(c0 + r) * ld + c0 + k] * Li[k * DCLNO_MAX_M + col];
            Li[r * DCLNO_MAX_M + col] = (r < col) ? 0.0 : s / L[(size_t)(c0 + r) * ld + c0 + r];
        }
    }
    __syncthreads();
    for (int rc0 = 0; rc0 < w2; rc0 += rch) {
        const int rows = min(rch, w2 - rc0);
        for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
            const int r = rc0 + e / n, t = e % n;
            double v;
            if (r < mc) v = (t >= c0) ? Li[(t - c0) * DCLNO_MAX_M + r] : 0.0;  // (L_cc^-T)[r][t-c0] = Li[t-c0][r]
            else v = (t <= c0 + (r - mc)) ? L[(size_t)(c0 + r - mc) * ld + t] : 0.0;
            Xs[e] = v;
        }
        __syncthreads();
        {  // each warp owns a block of consecutive rows (at most DCLNO_RPW)
            const int rpw = (rows + nw - 1) / nw, r0 = warp * rpw, my = min(rpw, rows - r0);
            double* Xw = Xs + (size_t)max(r0, 0) * n;
            switch (my) {
                case 1: q_rows_warp<1>(Xw, n, A, ld, tau, q2); break;
                case 2: q_rows_warp<2>(Xw, n, A, ld, tau, q2); break;
                case 3: q_rows_warp<3>(Xw, n, A, ld, tau, q2); break;
                case 4: q_rows_warp<4>(Xw, n, A, ld, tau, q2); break;
                default: break;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
            const int t = e / rows, rr = e % rows;
            P[(size_t)t * w2 + rc0 + rr] = Xs[(size_t)rr * n + t];
        }
        __syncthreads();
    }
}

// P <- P diag(Z1, Z2) by the logged rotations of each segment.  Work items are
// (problem, segment, strip) with strip 0 = the mc rows of R1 and strip 1 = the mc
// rows of R2 (a problem: a cluster torn once or a half of one torn twice); a warp packs
// floor(32 / mc) items, one lane per row, so one FP64 instruction updates the rows of
// several clusters.
__global__ void k_replay_fwd(int nitems, int per_warp, int mc_max, const ClusterDesc* __restrict__ cls,
                             const int* __restrict__ order, double* __restrict__ arena,
                             const int* __restrict__ iters, const int* __restrict__ status) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int grp = lane / mc_max, row = lane % mc_max;
    if (grp >= per_warp) return;
    const int item = wid * per_warp + grp;
    if (item >= nitems) return;
    const ClusterDesc d = cls[order[item >> 2]];
    if (status[d.sidx] != ST_OK) return;
    const int sg = (item >> 1) & 1;
    if (row >= d.mc || seg_len(d, sg) == 0) return;
    const int w2 = 2 * d.mc;
    const int r = (item & 1) * d.mc + row;
    double* P = arena + d.cc_off + (size_t)seg_start(d, sg) * w2;
    const double2* rot = reinterpret_cast<const double2*>(arena + d.rot_off) + (size_t)sg * d.rot_cap;
    const int* hdr = iters + d.it_off + (size_t)sg * d.it_cap;
    const int nsw = hdr[0];
    for (int k = 0; k < nsw; ++k) {
        const int start = hdr[1 + 3 * k], i0 = hdr[2 + 3 * k], cnt = hdr[3 + 3 * k];
        if (cnt > 0) sweep_fwd<DCLNO_REPLAY_DEPTH>(P + r, w2, rot + start, i0, cnt);
    }
}

// C = X Y for a tall-skinny Y (n x w, w <= 32, row-major with stride w, staged in Ys):
// FP64 tensor-core MMA (m8n8k4); warp k of 8 owns the 8-row blocks k, k+8, ... of C
// and all its columns in 8-wide tiles, so the MMA work is padded only to a multiple
// of 8 columns.  X is n x n row-major (ld), read once.
__device__ static void tall_gemm_fp64(double* __restrict__ C, const double* __restrict__ X, int ld,
                                      const double* __restrict__ Ys, int n, int w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int fr = lane >> 2, fk = lane & 3;
    const int nt = (w + 7) >> 3;
    for (int rb = warp; rb * 8 < n; rb += nw) {
        const int r = rb * 8 + fr;
        const bool rok = r < n;
        double acc[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = 0.0;
#pragma unroll 4
        for (int k = 0; k < n; k += 4) {
            const int kk = k + fk;
            const double a = (rok && kk < n) ? X[(size_t)r * ld + kk] : 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j < nt) {  // uniform across the warp
                    const int col = 8 * j + fr;
                    const double b = (kk < n && col < w) ? Ys[(size_t)kk * w + col] : 0.0;
                    dmma_8x8x4(acc[j][0], acc[j][1], a, b);
                }
            }
        }
        if (rok) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int col = 8 * j + 2 * fk + h;
                    if (j < nt && col < w) C[(size_t)r * w + col] = acc[j][h];
                }
        }
    }
}

// Merge-matrix products of a torn cluster (one CTA per cluster):
//   dir 0: P <- M^T P   (P = [n][2 mc] central strips; X = M^T stored row-major)
//   dir 1: G <- M G     (G = [n][w] density columns in W; X = M)
// Y is first copied to scratch (W for dir 0, the M^T area for dir 1).  FP64 path:
// tall_gemm_fp64.  Mixed path: C -= X B^T on the emulated tile GEMM with B = -Y^T
// staged in the scratch and C = Y cleared.
template <int EMU>
__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS, 2) k_mgemm(const ClusterDesc* __restrict__ cls,
                                                               const int* __restrict__ order,
                                                               double* __restrict__ arena,
                                                               int* __restrict__ status, int dir, int with_e) {
    extern __shared__ double sm[];
    __shared__ TcState tcs;
    const ClusterDesc d = cls[order[blockIdx.x]];
    const int ci = d.sidx;
    if (status[ci] != ST_OK) return;
    if (!d.split) return;
    const int n = d.n, ld = d.ld;
    const int w = (dir == 0 || with_e) ? 2 * d.mc : d.mc;
    double* M = arena + d.m_off;
    double* MT = M + (size_t)n * ld;
    double* Y = (dir == 0) ? arena + d.cc_off : arena + d.gb_off + (size_t)d.g_row0 * w;
    double* Bt = (dir == 0) ? arena + d.scr_off : MT;
    const double* X = (dir == 0) ? MT : M;
    if constexpr (EMU == 0) {
        for (size_t e = threadIdx.x; e < (size_t)n * w; e += blockDim.x) Bt[e] = Y[e];
        __syncthreads();
        tall_gemm_fp64(Y, X, ld, Bt, n, w);
        return;
    } else {
    // -Y^T staged with row stride bst: n rounded up to 4 in the scratch (w x bst doubles: the
    // two halves of a cluster torn twice use disjoint parts of its W block), ld in MT
    const int bst = (dir == 0) ? ((n + 3) & ~3) : ld;
    for (size_t e = threadIdx.x; e < (size_t)n * w; e += blockDim.x) {
        const int t = (int)(e / w), a = (int)(e % w);
        Bt[(size_t)a * bst + t] = -Y[e];
    }
    __syncthreads();
    for (size_t e = threadIdx.x; e < (size_t)n * w; e += blockDim.x) Y[e] = 0.0;
    __syncthreads();
    ENGINE_BEGIN(EMU, &tcs);
    if constexpr (EMU == 2)
        cta_gemm_tc_longk<false>(Y, w, X, ld, Bt, bst, n, w, n, reinterpret_cast<unsigned char*>(sm), &tcs);
    else
        tile_update_longk<EMU>(Y, w, X, ld, Bt, bst, n, w, n, sm, &tcs);
    ENGINE_END(EMU, &tcs);
    if (EMU == 2 && tcs.failed && threadIdx.x == 0) status[ci] = ST_TIMEOUT;
    }
}

template <int EMU>
static dclno_status launch_mgemm_t(dclno_ctx* c, const int* list, int N, int dir, int with_e) {
    if (N == 0) return DCLNO_OK;
    const size_t smb = EMU ? (size_t)ENGINE_SMEM_BYTES(EMU) : 0;
    DCLNO_CUDA(c, cudaFuncSetAttribute(k_mgemm<EMU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
    k_mgemm<EMU><<<N, DCLNO_SOLVE_THREADS, smb, c->stream>>>(c->d_cl, list, c->d_arena, c->d_status, dir, with_e);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

// Y <- merge matrices of a batch: the two-segment problems' (clusters torn once and the
// halves of clusters torn twice), then the halves' merge of the clusters torn twice;
// dir 0 (strips, P <- M^T P) in that order, dir 1 (density columns, G <- M G) reversed
dclno_status launch_mgemm(dclno_ctx* c, const Batch& b, int dir, int with_e, int emu) {
    const int N1 = b.l1end - b.l1beg, N2 = b.l2end - b.l2beg;
    bool any = false;
    for (int i = b.id_lo; i < b.id_hi; ++i) any = any || c->cl[i].split;
    if (!any) return DCLNO_OK;
    ProfScope ps__(c, dir == 0 ? "k_mgemm_fwd" : "k_mgemm_rev");
    const int* l1 = c->d_l1 + b.l1beg;
    const int* l2 = c->d_l2 + b.l2beg;
    for (int pass = 0; pass < 2; ++pass) {
        const bool first = (pass == 0) == (dir == 0);
        const int* list = first ? l1 : l2;
        const int n = first ? N1 : N2;
        dclno_status st;
        if (emu == 2) st = launch_mgemm_t<2>(c, list, n, dir, with_e);
        else if (emu == 1) st = launch_mgemm_t<1>(c, list, n, dir, with_e);
        else st = launch_mgemm_t<0>(c, list, n, dir, with_e);
        if (st != DCLNO_OK) return st;
    }
    return DCLNO_OK;
}

// eigenvalues and weights: eps_mu = d_mu, q_mu = sum_a P[mu][a] P[mu][mc + a]
__global__ void k_weights(const ClusterDesc* __restrict__ cls, const int* __restrict__ order,
                          const double* __restrict__ arena, const int* __restrict__ status,
                          double* __restrict__ eps, double* __restrict__ q) {
    const int ci = order[blockIdx.y];
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    const int n = d.n, mc = d.mc;
    const double* dv = arena + d.aux_off;
    const double* P = arena + d.cc_off;
    for (int mu = blockIdx.x * blockDim.x + threadIdx.x; mu < n; mu += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < mc; ++a) s = fma(P[(size_t)mu * 2 * mc + a], P[(size_t)mu * 2 * mc + mc + a], s);
        eps[d.eig_off + mu] = dv[mu];
        q[d.eig_off + mu] = s;
    }
}


static dclno_status launch_ql(dclno_ctx* c, const int* order, int N, int segp, int narr, int lanes) {
    const size_t smq = (size_t)lanes * narr * segp * sizeof(double);
    if (narr == 4) {
        DCLNO_CUDA(c, cudaFuncSetAttribute(k_ql<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq));
        k_ql<true><<<(2 * N + lanes - 1) / lanes, 32, smq, c->stream>>>(N, lanes, segp, c->d_cl, order, c->d_arena,
                                                                       c->d_iters, c->d_status);
    } else {
        DCLNO_CUDA(c, cudaFuncSetAttribute(k_ql<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq));
        k_ql<false><<<(2 * N + lanes - 1) / lanes, 32, smq, c->stream>>>(N, lanes, segp, c->d_cl, order, c->d_arena,
                                                                        c->d_iters, c->d_status);
    }
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

// save (dir 0) or restore (dir 1) d and e of a batch's clusters (the QL input)
__global__ void k_save_de(const ClusterDesc* __restrict__ cls, const int* __restrict__ order, double* __restrict__ arena,
                          double* __restrict__ buf, int stride, int dir) {
    const ClusterDesc d = cls[order[blockIdx.x]];
    double* dv = arena + d.aux_off;
    double* bv = buf + (size_t)blockIdx.x * stride;
    for (int t = threadIdx.x; t < d.n; t += blockDim.x) {
        if (dir == 0) {
            bv[t] = dv[t];
            bv[d.n + t] = dv[d.ld + t];
        } else {
            dv[t] = bv[t];
            dv[d.ld + t] = bv[d.n + t];
        }
    }
}

// Launch-shape autotuner for k_ql: a lane is one tridiagonal segment and a warp runs
// its lanes in lockstep, so the lanes per warp trade the warp's mixed-phase overhead
// against how many warps share an SM (its FP64 pipe and shared memory).  The best
// count depends on the cluster count and segment lengths; each candidate is timed
// once on this batch's own tridiagonal matrices (d and e restored before each try;
// every lane's arithmetic is the same whatever the grouping, so the results are too).
static dclno_status tune_ql(dclno_ctx* c, const Batch& b, const int* order, int N, int segp, int narr, int fit) {
    static const int cand[DCLNO_QL_CANDIDATES] = {4, 8, 12, 16, 24, 32};
    int ldmax = 0;
    for (int i = b.id_lo; i < b.id_hi; ++i) ldmax = std::max(ldmax, c->cl[i].n);
    const int stride = 2 * ldmax;
    const size_t need = (size_t)N * stride;
    if (c->tune_doubles < need) {
        if (c->d_tune) cudaFree(c->d_tune);
        c->d_tune = nullptr;
        c->tune_doubles = 0;
        DCLNO_CUDA(c, cudaMalloc(&c->d_tune, need * sizeof(double)));
        c->tune_doubles = need;
    }
    k_save_de<<<N, 128, 0, c->stream>>>(c->d_cl, order, c->d_arena, c->d_tune, stride, 0);
    DCLNO_LAUNCHED(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DCLNO_CUDA(c, cudaEventCreate(&e0));
    DCLNO_CUDA(c, cudaEventCreate(&e1));
    int best = fit;
    float best_ms = -1.0f;
    dclno_status st = DCLNO_OK;
    for (int k = 0; k < DCLNO_QL_CANDIDATES && st == DCLNO_OK; ++k) {
        if (cand[k] > fit) continue;
        k_save_de<<<N, 128, 0, c->stream>>>(c->d_cl, order, c->d_arena, c->d_tune, stride, 1);
        c->launches++;
        cudaEventRecord(e0, c->stream);
        st = launch_ql(c, order, N, segp, narr, cand[k]);
        cudaEventRecord(e1, c->stream);
        float ms = 0.0f;
        if (st == DCLNO_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            c->ql_tune_ms[b.index * DCLNO_QL_CANDIDATES + k] = ms;
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                best = cand[k];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != DCLNO_OK) return st;
    k_save_de<<<N, 128, 0, c->stream>>>(c->d_cl, order, c->d_arena, c->d_tune, stride, 1);
    DCLNO_LAUNCHED(c);
    c->ql_lanes[b.index] = best;
    return DCLNO_OK;
}

// one cubic kernel over the clusters order[0 .. nitems) with a schedule
template <int EMU>
static dclno_status launch_cubic_t(dclno_ctx* c, int kernel, const int* order, int nitems, size_t smem, int persistent,
                                   int two) {
    const void* fn = kernel == TK_CHOL ? (const void*)k_cholesky<EMU>
                     : kernel == TK_CONG ? (const void*)k_congruence<EMU>
                                         : (const void*)k_tridiag<EMU>;
    DCLNO_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = sched_grid(c, fn, DCLNO_SOLVE_THREADS, smem, nitems, persistent != 0);
    int* q = persistent ? c->d_queue : nullptr;
    if (q) DCLNO_CUDA(c, cudaMemsetAsync(q, 0, sizeof(int), c->stream));
    if (kernel == TK_CHOL)
        k_cholesky<EMU><<<grid, DCLNO_SOLVE_THREADS, smem, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, nitems, q);
    else if (kernel == TK_CONG)
        k_congruence<EMU><<<grid, DCLNO_SOLVE_THREADS, smem, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, nitems,
                                                                         q);
    else
        k_tridiag<EMU><<<grid, DCLNO_SOLVE_THREADS, smem, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, two,
                                                                      nitems, q);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

// shared memory of a cubic kernel with engine e on clusters of dimension <= maxn
static size_t cubic_smem(int kernel, int e, int maxn) {
    const size_t g = (ENGINE_SMEM_BYTES(e) + 7) / 8;
    if (kernel == TK_TRI) return std::max(g, (size_t)(2 + DCLNO_SOLVE_THREADS / 32) * maxn + 32 + 2 * NB) * sizeof(double);
    return (size_t)(NB * DK_LD + NB + g) * sizeof(double);
}

static bool bucket_all_two_stage(const dclno_ctx* c, const Bucket& k) {
    for (int o = k.obeg; o < k.oend; ++o) {
        const ClusterDesc& d = c->cl[c->order[o]];
        if (!(d.q2_off >= 0 && d.split && d.n >= DCLNO_TWO_STAGE_MIN)) return false;
    }
    return true;
}

static dclno_status launch_solve(dclno_ctx* c, const Batch& b, bool reduce_only, bool mixed) {
    const int N = b.oend - b.obeg;  // clusters of the batch
    if (N == 0) return DCLNO_OK;
    const int maxn = b.maxn;
    const int* order = c->d_order + b.obeg;
    const int nw = DCLNO_SOLVE_THREADS / 32;
    // strip rows per shared-memory chunk of k_apply_q_rows: at most DCLNO_RPW per warp, within 200 KB
    const int rch = (int)std::min<long long>(std::min(2 * b.mcmax, DCLNO_RPW * nw),
                                             (200LL * 1024 / 8 - DCLNO_MAX_M * DCLNO_MAX_M) / std::max(maxn, 1));
    size_t sm_q = (size_t)(DCLNO_MAX_M * DCLNO_MAX_M + (size_t)std::max(rch, 1) * maxn) * sizeof(double);
    DCLNO_CUDA(c, cudaFuncSetAttribute(k_apply_q_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_q));
    if (cubic_smem(TK_TRI, 0, maxn) > 227 * 1024 || sm_q > 227 * 1024 || rch < 1)
        return set_err(c, DCLNO_ERR_ARG, "cluster dimension too large for the FP64 solver (n = " + std::to_string(maxn) + ")");
    const int two = c->solved_two ? 1 : 0;
    const bool tune = !reduce_only;
    static const char* names[3] = {"k_cholesky", "k_congruence", "k_tridiag"};
    for (int kernel = TK_CHOL; kernel <= TK_TRI; ++kernel) {
        ProfScope ps__(c, names[kernel]);
        std::vector<char> use(b.buckets.size(), 1);
        for (int k = 0; k < (int)b.buckets.size(); ++k)  // k_band + k_chase instead
            if (kernel == TK_TRI && two && bucket_all_two_stage(c, b.buckets[k])) use[k] = 0;
        for (const SchedRun& r : sched_runs(c, b, kernel, mixed, tune, use)) {
            const Sched s = r.s;
            cudaEvent_t e0 = nullptr;
            if (r.cand >= 0) {
                const dclno_status st = sched_time_begin(c, &e0);
                if (st != DCLNO_OK) return st;
            }
            const size_t smem = cubic_smem(kernel, s.engine, r.maxn);
            const int* ord = c->d_order + r.obeg;
            const int ni = r.oend - r.obeg;
            dclno_status st;
            if (s.engine == 2) st = launch_cubic_t<2>(c, kernel, ord, ni, smem, s.persistent, two);
            else if (s.engine == 1) st = launch_cubic_t<1>(c, kernel, ord, ni, smem, s.persistent, two);
            else st = launch_cubic_t<0>(c, kernel, ord, ni, smem, s.persistent, two);
            if (st == DCLNO_OK && r.cand >= 0) st = sched_time_end(c, b, r.k0, kernel, mixed, r.cand, e0);
            if (st != DCLNO_OK) return st;
        }
    }
    if (two) {
        const dclno_status st = launch_two_stage(c, b, mixed, tune);
        if (st != DCLNO_OK) return st;
    }
    if (reduce_only) {
        ProfScope ps__(c, "k_apply_q_rows");
        k_apply_q_rows<<<N, DCLNO_SOLVE_THREADS, sm_q, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, rch,
                                                                     two);
        DCLNO_LAUNCHED(c);
        return DCLNO_OK;  // statuses are read by the caller after the pole sum
    }
    // the two-segment problems: clusters torn once (or not at all), halves of those torn twice
    const int* l1 = c->d_l1 + b.l1beg;
    const int N1 = b.l1end - b.l1beg;
    {
        const int segp = b.segmax | 1;  // odd: lanes' arrays start in different banks
        const int narr = b.l2end > b.l2beg ? 4 : 3;
        const int fit = (int)std::min<long long>(32, (200LL * 1024) / (8LL * narr * segp));  // shared memory bound
        if (fit < 1) return set_err(c, DCLNO_ERR_ARG, "tridiagonal segment too long for the QL kernel");
        int& lanes = c->ql_lanes[b.index];
        if (lanes == 0 && c->autotune && !c->deferred) {
            const dclno_status st = tune_ql(c, b, l1, N1, segp, narr, fit);
            if (st != DCLNO_OK) return st;
        }
        const int use = lanes > 0 ? std::min(lanes, fit) : fit;
        ProfScope ps__(c, "k_ql");
        const dclno_status st = launch_ql(c, l1, N1, segp, narr, use);
        if (st != DCLNO_OK) return st;
    }
    {
        const dclno_status st = launch_merge(c, b);
        if (st != DCLNO_OK) return st;
    }
    {
        ProfScope ps__(c, "k_apply_q_rows");
        k_apply_q_rows<<<N, DCLNO_SOLVE_THREADS, sm_q, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, rch,
                                                                     two);
    }
    DCLNO_LAUNCHED(c);
    {
        ProfScope ps__(c, "k_replay_fwd");
        const int mcmax = b.mcmax;
        const int per_warp = std::max(1, 32 / mcmax);
        const int items = 4 * N1;
        const int warps = (items + per_warp - 1) / per_warp;
        k_replay_fwd<<<(warps * 32 + 127) / 128, 128, 0, c->stream>>>(items, per_warp, mcmax, c->d_cl, l1,
                                                                      c->d_arena, c->d_iters, c->d_status);
    }
    DCLNO_LAUNCHED(c);
    {
        const dclno_status st = launch_mgemm(c, b, 0, 0, mixed ? 2 : 0);
        if (st != DCLNO_OK) return st;
    }
    {
        ProfScope ps__(c, "k_weights");
        k_weights<<<dim3((maxn + 255) / 256, N), 256, 0, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status,
                                                                   c->d_eps, c->d_q);
    }
    DCLNO_LAUNCHED(c);
    if (c->deferred) return launch_status_or(c);
    const int nid = b.id_hi - b.id_lo;
    std::vector<int> st(nid);
    DCLNO_CUDA(c, cudaMemcpyAsync(st.data(), c->d_status + b.id_lo, sizeof(int) * nid, cudaMemcpyDeviceToHost,
                                  c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    sched_collect(c);
    for (int k = 0; k < nid; ++k) {
        const int i = b.id_lo + k;
        if (st[k] == ST_NOT_SPD)
            return set_err(c, DCLNO_ERR_NOT_SPD, "overlap of cluster " + std::to_string(i) + " is not positive definite");
        if (st[k] == ST_NOT_CONVERGED)
            return set_err(c, DCLNO_ERR_NOT_CONVERGED, "QL did not converge for cluster " + std::to_string(i));
        if (st[k] == ST_LOG_FULL)
            return set_err(c, DCLNO_ERR_NOT_CONVERGED, "QL rotation log full for cluster " + std::to_string(i));
        if (st[k] == ST_TIMEOUT)
            return set_err(c, DCLNO_ERR_TIMEOUT, "tensor-core wait ran out for cluster " + std::to_string(i));
        if (st[k] != ST_OK) return set_err(c, DCLNO_ERR_NOT_CONVERGED, "solver failed for cluster " + std::to_string(i));
    }
    return DCLNO_OK;
}

dclno_status launch_solve_fp64(dclno_ctx* c, const Batch& b, bool reduce_only) {
    return launch_solve(c, b, reduce_only, false);
}
dclno_status launch_solve_mixed(dclno_ctx* c, const Batch& b, bool reduce_only) {
    return launch_solve(c, b, reduce_only, true);
}
