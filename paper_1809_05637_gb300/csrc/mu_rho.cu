// Common chemical potential (Sec. II.C step (iv)) and density-matrix rows of the
// central atoms (Eq. (dm) with the spectral Green function of Eq. (Gi)).
//
// mu: device-wide k-section of N(mu) = 2 sum f((eps - mu)/kT) q = N_e over all
//     clusters' (eps, q) pairs; each pass evaluates KSEC interior points of the
//     current bracket, a fixed-order reduction picks the sub-interval.
// rho rows: with G = F C_c^T (n x M_i, F = diag f(eps)), the rows are
//     rho_c,:^T = L^-T Q Z G: reverse replay of the QL rotations (Z G), the
//     Householder reflectors from the left (Q .), back substitution with L^T,
//     then LNO columns are returned to PAOs through V_j and scattered into the
//     BSR pattern of row i.
#include <cmath>

#include "dclno_internal.cuh"

#define KSEC 3          // interior points per k-section pass
#define MU_BLOCKS 1024  // partial-sum blocks per pass
#define MU_PASSES 40

// f(x) = 1/(1+e^x) without overflow
__device__ __forceinline__ double fermi(double x) {
    if (x > 0.0) {
        if (x > 745.0) return 0.0;
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    if (x < -745.0) return 1.0;
    return 1.0 / (1.0 + exp(x));
}

// scal: [0] lo, [1] hi, [2] mu (result), [3] N(mu), [4] done flag, [5] kT, [6] N_e
__global__ void k_mu_bracket(long long total, const double* __restrict__ eps, double* __restrict__ part) {
    __shared__ double mn[256], mx[256];
    double a = 1e300, b = -1e300;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        a = fmin(a, eps[t]);
        b = fmax(b, eps[t]);
    }
    mn[threadIdx.x] = a;
    mx[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + s]);
            mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = mn[0];
        part[2 * blockIdx.x + 1] = mx[0];
    }
}

// Fixed-order sum of part[b * stride] over b < nblk by one warp: lane l adds the
// blocks l, l + 32, ... in order, then a butterfly over the lanes (the same order on
// every run, so the bits of N(mu) are reproducible).
__device__ __forceinline__ double warp_ordered_sum(const double* __restrict__ part, int nblk, int stride) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * stride];
    return warp_sum(s);
}

// one warp: extremes of the per-block minima and maxima, then the bracket
__global__ void k_mu_init(int nblk, const double* __restrict__ part, double* __restrict__ scal, double kT, double ne) {
    const int lane = threadIdx.x & 31;
    double a = 1e300, b = -1e300;
    for (int t = lane; t < nblk; t += 32) {
        a = fmin(a, part[2 * t]);
        b = fmax(b, part[2 * t + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane != 0) return;
    scal[0] = a - 40.0 * kT;
    scal[1] = b + 40.0 * kT;
    scal[2] = 0.5 * (scal[0] + scal[1]);
    scal[4] = 0.0;
    scal[5] = kT;
    scal[6] = ne;
}

// partial sums of N at the bracket's end points (first pass) and KSEC interior points
__global__ void k_mu_partial(long long total, const double* __restrict__ eps, const double* __restrict__ q,
                             const double* __restrict__ scal, double* __restrict__ part, int with_ends) {
    if (scal[4] != 0.0) return;
    const double lo = scal[0], hi = scal[1], kT = scal[5];
    const int np = KSEC + 2;
    double mu[KSEC + 2], acc[KSEC + 2];
#pragma unroll
    for (int p = 0; p < np; ++p) {
        mu[p] = lo + (hi - lo) * (double)p / (KSEC + 1);
        acc[p] = 0.0;
    }
    const double inv = 1.0 / kT;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const double e = eps[t], w = q[t];
#pragma unroll
        for (int p = 0; p < np; ++p) {
            if (!with_ends && (p == 0 || p == np - 1)) continue;
            acc[p] = fma(fermi((e - mu[p]) * inv), w, acc[p]);
        }
    }
    __shared__ double red[KSEC + 2][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < np; ++p) {
        double v = warp_sum(acc[p]);
        if (lane == 0) red[p][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < np) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        part[(size_t)blockIdx.x * np + threadIdx.x] = s;
    }
}

// fixed-order reduction of the partial sums (warp p sums trial point p); narrows [lo, hi]
__global__ void k_mu_update(int nblk, const double* __restrict__ part, double* __restrict__ scal, int first, int last) {
    const int np = KSEC + 2;
    __shared__ double N[KSEC + 2];
    if (scal[4] != 0.0) return;  // uniform: every thread reads the same flag
    const int warp = threadIdx.x >> 5;
    if (warp < np) {
        const double v = warp_ordered_sum(part + warp, nblk, np);
        if ((threadIdx.x & 31) == 0) N[warp] = 2.0 * v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double lo = scal[0], hi = scal[1], ne = scal[6];
    if (first) {
        scal[8] = N[0];
        scal[9] = N[np - 1];
        if (!(N[0] <= ne && ne <= N[np - 1])) {
            scal[4] = 2.0;  // no bracket
            return;
        }
    }
    const double tol = 1e-12 * fabs(ne);
    for (int p = 1; p <= KSEC; ++p) {
        const double mu = lo + (hi - lo) * (double)p / (KSEC + 1);
        if (fabs(N[p] - ne) <= tol) {
            scal[2] = mu;
            scal[3] = N[p];
            scal[4] = 1.0;
            return;
        }
    }
    int p = 1;
    while (p <= KSEC && N[p] < ne) ++p;  // first interior point with N >= ne
    const double nlo = lo + (hi - lo) * (double)(p - 1) / (KSEC + 1);
    const double nhi = lo + (hi - lo) * (double)p / (KSEC + 1);
    scal[0] = nlo;
    scal[1] = nhi;
    const double mid = 0.5 * (nlo + nhi);
    scal[2] = mid;
    if (last || !(nlo < mid && mid < nhi)) scal[4] = 3.0;  // bracket exhausted in double precision
}

// N(mu) at the final mu (exact re-evaluation, one point)
__global__ void k_mu_final_partial(long long total, const double* __restrict__ eps, const double* __restrict__ q,
                                   const double* __restrict__ scal, double* __restrict__ part) {
    const double mu = scal[2], inv = 1.0 / scal[5];
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
        acc = fma(fermi((eps[t] - mu) * inv), q[t], acc);
    __shared__ double red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_mu_final(int nblk, const double* __restrict__ part, double* __restrict__ scal) {
    const double v = warp_ordered_sum(part, nblk, 1);
    if (threadIdx.x == 0) scal[3] = 2.0 * v;
}

dclno_status launch_find_mu(dclno_ctx* c, double ne, double kT, double* mu_out, double* nmu_out) {
    const long long total = c->total_dim;
    const int nblk = MU_BLOCKS;
    {
        ProfScope ps__(c, "k_mu_bracket");
        k_mu_bracket<<<nblk, 256, 0, c->stream>>>(total, c->d_eps, c->d_mu_work);
    }
    DCLNO_LAUNCHED(c);
    {
        ProfScope ps__(c, "k_mu_init");
        k_mu_init<<<1, 32, 0, c->stream>>>(nblk, c->d_mu_work, c->d_scalars, kT, ne);
    }
    DCLNO_LAUNCHED(c);
    for (int pass = 0; pass < MU_PASSES; ++pass) {
        {
            ProfScope ps__(c, "k_mu_partial");
            k_mu_partial<<<nblk, 256, 0, c->stream>>>(total, c->d_eps, c->d_q, c->d_scalars, c->d_mu_work, pass == 0);
        }
        DCLNO_LAUNCHED(c);
        {
            ProfScope ps__(c, "k_mu_update");
            k_mu_update<<<1, 32 * (KSEC + 2), 0, c->stream>>>(nblk, c->d_mu_work, c->d_scalars, pass == 0, pass == MU_PASSES - 1);
        }
        DCLNO_LAUNCHED(c);
    }
    {
        ProfScope ps__(c, "k_mu_final_partial");
        k_mu_final_partial<<<nblk, 256, 0, c->stream>>>(total, c->d_eps, c->d_q, c->d_scalars, c->d_mu_work);
    }
    DCLNO_LAUNCHED(c);
    {
        ProfScope ps__(c, "k_mu_final");
        k_mu_final<<<1, 32, 0, c->stream>>>(nblk, c->d_mu_work, c->d_scalars);
    }
    DCLNO_LAUNCHED(c);
    if (c->deferred) return DCLNO_OK;  // mu stays in d_scalars[2]; a missing bracket is recorded by k_scf_record
    double h[10];
    DCLNO_CUDA(c, cudaMemcpyAsync(h, c->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h[4] == 2.0) {
        char b[160];
        snprintf(b, sizeof b, "dclno_find_mu: N_e = %.17g outside [%.17g, %.17g]", ne, h[8], h[9]);
        return set_err(c, DCLNO_ERR_NO_BRACKET, b);
    }
    *mu_out = h[2];
    *nmu_out = h[3];
    return DCLNO_OK;
}

// ---------------------------------------------------------------------------
// Density-matrix rows
// ---------------------------------------------------------------------------
// G[mu][a] = f(eps_mu) C_c[a][mu] and, with the energy density matrix, G[mu][mc + a] =
// f(eps_mu) eps_mu C_c[a][mu] (stored [n][w], w = mc or 2 mc, in the cluster's W area);
// band energy of the cluster
__global__ void k_rho_prep(int id_lo, const ClusterDesc* __restrict__ cls, double* __restrict__ arena,
                           const double* __restrict__ eps, const double* __restrict__ q, double mu_host,
                           const double* __restrict__ mu_dev, double kT, int with_e, double* __restrict__ eband) {
    const int ci = id_lo + blockIdx.x;
    const double mu = mu_dev ? *mu_dev : mu_host;
    const ClusterDesc d = cls[ci];
    const int n = d.n, mc = d.mc, w = with_e ? 2 * mc : mc;
    const double* P = arena + d.cc_off;
    double* G = arena + d.aux_off + 3 * d.ld;
    const double inv = 1.0 / kT;
    double eb = 0.0;
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const double e = eps[d.eig_off + m];
        const double f = fermi((e - mu) * inv);
        eb = fma(f * e, q[d.eig_off + m], eb);
        for (int a = 0; a < mc; ++a) {
            const double c = P[(size_t)m * 2 * mc + a];
            G[(size_t)m * w + a] = f * c;
            if (with_e) G[(size_t)m * w + mc + a] = f * e * c;
        }
    }
    __shared__ double red[8];
    eb = warp_sum(eb);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = eb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        eband[ci] = 2.0 * s;
    }
}

// G <- diag(Z1, Z2) G: each segment's logged rotations in reverse order acting on rows
// (i, i+1).  Work items are (problem, segment) (a cluster torn once, or a half of one
// torn twice, whose rows of G start at g_row0); a warp packs floor(32 / w) items, one
// lane per column of G.
__global__ void k_replay_rev(int nitems, int per_warp, int w_max, int with_e, const ClusterDesc* __restrict__ cls,
                             const int* __restrict__ order, double* __restrict__ arena, const int* __restrict__ iters) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int grp = lane / w_max, col = lane % w_max;
    if (grp >= per_warp) return;
    const int item = wid * per_warp + grp;
    if (item >= nitems) return;
    const ClusterDesc d = cls[order[item >> 1]];
    const int sg = item & 1;
    const int mc = with_e ? 2 * d.mc : d.mc;  // columns of G
    if (col >= mc || seg_len(d, sg) == 0) return;
    double* G = arena + d.gb_off + (size_t)(d.g_row0 + seg_start(d, sg)) * mc;
    const double2* rot = reinterpret_cast<const double2*>(arena + d.rot_off) + (size_t)sg * d.rot_cap;
    const int* hdr = iters + d.it_off + (size_t)sg * d.it_cap;
    const int nsw = hdr[0];
    for (int k = nsw - 1; k >= 0; --k) {
        const int start = hdr[1 + 3 * k], i0 = hdr[2 + 3 * k], cnt = hdr[3 + 3 * k];
        if (cnt > 0) sweep_rev<DCLNO_REPLAY_DEPTH>(G + col, mc, rot + start, i0, cnt);
    }
}

// R columns owned by one warp (rows of X, stride n): X <- H_0 ... H_{n-3} X (the
// reflectors from the last one), then L^T X_new = X by back substitution.
template <int R>
__device__ static void rho_qx_warp(double* X, int n, const double* __restrict__ A, const double* __restrict__ L,
                                   int ld, const double* __restrict__ tau, const double* __restrict__ invd,
                                   const double* __restrict__ q2) {
    const int lane = threadIdx.x & 31;
    if (q2) {
        warp_apply_two_stage<R>(X, n, A, ld, tau, q2, 1);  // Q = Q1 Q2 of the two-stage reduction
    } else {
        for (int k = n - 3; k >= 0; --k) {
            const double tk = tau[k];
            if (tk != 0.0) warp_reflect<R>(X, n, k, n, A + (size_t)k * ld, tk);
        }
    }
    // x_t = g_t / L[t][t], then g_s -= L[t][s] x_t for s < t
    for (int t = n - 1; t >= 0; --t) {
        const double it = invd[t];
        double xt[R];
#pragma unroll
        for (int j = 0; j < R; ++j) xt[j] = X[(size_t)j * n + t] * it;
        __syncwarp();
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < R; ++j) X[(size_t)j * n + t] = xt[j];
        const double* Lt = L + (size_t)t * ld;
        for (int s = lane; s < t; s += 32) {
            const double l = Lt[s];
#pragma unroll
            for (int j = 0; j < R; ++j) X[(size_t)j * n + s] = fma(-l, xt[j], X[(size_t)j * n + s]);
        }
        __syncwarp();
    }
}

// X = L^-T Q G for the columns of G ([n][w] at aux_off + 3 ld, w = mc or 2 mc): the
// reflectors applied in reverse order (Q = H_0 ... H_{n-3}), then L^T X = G by back
// substitution.  Columns are independent: chunks of rch columns are held in shared
// memory (one row of stride n per column), each warp carries its columns through all
// reflectors and the triangular solve (rho_qx_warp), with no block barriers.
__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS) k_rho_qx(const ClusterDesc* __restrict__ cls,
                                                                const int* __restrict__ order,
                                                                double* __restrict__ arena, int with_e, int rch,
                                                                int two_stage) {
    extern __shared__ double sm[];
    const ClusterDesc d = cls[order[blockIdx.x]];
    const double* q2 = (two_stage && two_stage_cluster(d)) ? arena + d.q2_off : nullptr;
    const int n = d.n, ld = d.ld, mcw = with_e ? 2 * d.mc : d.mc;  // columns of G
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* A = arena + d.mat_off;
    const double* L = A + (size_t)n * ld;
    const double* tau = arena + d.aux_off + 2 * ld;
    double* G = arena + d.aux_off + 3 * ld;
    double* invd = sm;      // n: 1 / L[t][t]
    double* Xs = sm + n;    // rch x n
    for (int t = threadIdx.x; t < n; t += blockDim.x) invd[t] = 1.0 / L[(size_t)t * ld + t];
    for (int a0 = 0; a0 < mcw; a0 += rch) {
        const int cols = min(rch, mcw - a0);
        for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
            const int t = e / cols, a = e % cols;
            Xs[(size_t)a * n + t] = G[(size_t)t * mcw + a0 + a];
        }
        __syncthreads();
        {  // each warp owns a block of consecutive columns (at most DCLNO_RPW)
            const int rpw = (cols + nw - 1) / nw, r0 = warp * rpw, my = min(rpw, cols - r0);
            double* Xw = Xs + (size_t)max(r0, 0) * n;
            switch (my) {
                case 1: rho_qx_warp<1>(Xw, n, A, L, ld, tau, invd, q2); break;
                case 2: rho_qx_warp<2>(Xw, n, A, L, ld, tau, invd, q2); break;
                case 3: rho_qx_warp<3>(Xw, n, A, L, ld, tau, invd, q2); break;
                case 4: rho_qx_warp<4>(Xw, n, A, L, ld, tau, invd, q2); break;
                default: break;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
            const int t = e / cols, a = e % cols;
            G[(size_t)t * mcw + a0 + a] = Xs[(size_t)a * n + t];
        }
        __syncthreads();
    }
}

// scatter the rows of atom i into the BSR pattern (rho from columns [0, mc) of X,
// e from [mc, 2 mc) when e_out is given); one warp per block of row i
__global__ void k_rho_scatter(int id_lo, const ClusterDesc* __restrict__ cls, const MemberDesc* __restrict__ mem,
                              const int* __restrict__ norb, const long long* __restrict__ row_ptr,
                              const long long* __restrict__ key, const long long* __restrict__ blk_off,
                              const int* __restrict__ rowblk_member, const long long* __restrict__ voff,
                              const int* __restrict__ kat, int k,
                              const double* __restrict__ V, const double* __restrict__ arena,
                              double* __restrict__ rho, double* __restrict__ e_out) {
    const int i = id_lo + blockIdx.y;
    const ClusterDesc d = cls[i];
    const int mc = d.mc, w = e_out ? 2 * mc : mc;
    const double* X = arena + d.aux_off + 3 * d.ld;  // [n][w]
    const int lane = threadIdx.x & 31;
    const long long b0 = row_ptr[i], b1 = row_ptr[i + 1];
    for (long long b = b0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < b1;
         b += (long long)gridDim.x * (blockDim.x >> 5)) {
        const int j = (int)(key[b] >> 24), mj = norb[j];
        double* out = rho + blk_off[b];
        double* oute = e_out ? e_out + blk_off[b] : nullptr;
        const int m = rowblk_member[b];
        if (m < 0) {
            for (int e = lane; e < mc * mj; e += 32) {
                out[e] = 0.0;
                if (oute) oute[e] = 0.0;
            }
            continue;
        }
        const MemberDesc md = mem[d.mbeg + m];
        const double* Vj = md.core ? nullptr : V + voff[j];
        const int kj = md.core ? 0 : kat[j];  // the member's LNO count (V rows have stride k)
        for (int e = lane; e < mc * mj; e += 32) {
            const int a = e / mj, bb = e % mj;
            double s = 0.0, se = 0.0;
            if (md.core) {
                s = X[(size_t)(md.off + bb) * w + a];
                if (oute) se = X[(size_t)(md.off + bb) * w + mc + a];
            } else {
                for (int g = 0; g < kj; ++g) {
                    const double v = Vj[bb * k + g];
                    s = fma(X[(size_t)(md.off + g) * w + a], v, s);
                    if (oute) se = fma(X[(size_t)(md.off + g) * w + mc + a], v, se);
                }
            }
            out[e] = s;
            if (oute) oute[e] = se;
        }
    }
}

dclno_status launch_density(dclno_ctx* c, const Batch& b, double mu, double kT, double* rho_out, double* e_out,
                            bool poles) {
    const int with_e = e_out ? 1 : 0;
    const int N = b.oend - b.obeg;  // clusters of the batch
    if (N == 0) return DCLNO_OK;
    const int maxn = b.maxn;
    long long maxrow = 0;
    for (int i = b.id_lo; i < b.id_hi; ++i) maxrow = std::max(maxrow, c->row_ptr[i + 1] - c->row_ptr[i]);
    if (!poles) {  // G = F C_c^T from the spectrum, then Z G (merge matrix, logged rotations)
        {
            ProfScope ps__(c, "k_rho_prep");
            k_rho_prep<<<N, 256, 0, c->stream>>>(b.id_lo, c->d_cl, c->d_arena, c->d_eps, c->d_q, mu,
                                                 c->deferred ? c->d_scalars + 2 : nullptr, kT, with_e, c->d_eband);
        }
        DCLNO_LAUNCHED(c);
        const dclno_status st = launch_mgemm(c, b, 1, with_e, c->solved_prec == DCLNO_MIXED ? 2 : 0);
        if (st != DCLNO_OK) return st;
        ProfScope ps__(c, "k_replay_rev");
        const int wmax = with_e ? 2 * b.mcmax : b.mcmax;
        const int per_warp = std::max(1, 32 / wmax);
        const int N1 = b.l1end - b.l1beg;  // two-segment problems (see launch_mgemm)
        const int warps = (2 * N1 + per_warp - 1) / per_warp;
        k_replay_rev<<<(warps * 32 + 127) / 128, 128, 0, c->stream>>>(2 * N1, per_warp, wmax, with_e, c->d_cl,
                                                                      c->d_l1 + b.l1beg, c->d_arena, c->d_iters);
        DCLNO_LAUNCHED(c);
    }
    // columns per shared-memory chunk of k_rho_qx: at most DCLNO_RPW per warp, within 200 KB
    const int wcols = with_e ? 2 * b.mcmax : b.mcmax;
    const int rch = (int)std::min<long long>(std::min(wcols, DCLNO_RPW * (DCLNO_SOLVE_THREADS / 32)),
                                             200LL * 1024 / 8 / std::max(maxn, 1) - 1);
    if (rch < 1) return set_err(c, DCLNO_ERR_ARG, "cluster dimension too large for the density kernel");
    const size_t sm = (size_t)(rch + 1) * maxn * sizeof(double);
    DCLNO_CUDA(c, cudaFuncSetAttribute(k_rho_qx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
        ProfScope ps__(c, "k_rho_qx");
        k_rho_qx<<<N, DCLNO_SOLVE_THREADS, sm, c->stream>>>(c->d_cl, c->d_order + b.obeg, c->d_arena, with_e, rch,
                                                            c->solved_two ? 1 : 0);
    }
    DCLNO_LAUNCHED(c);
    const int wpb = 8;
    const int bx = (int)std::max<long long>(1, std::min<long long>((maxrow + wpb - 1) / wpb, 64));
    {
        ProfScope ps__(c, "k_rho_scatter");
        k_rho_scatter<<<dim3(bx, N), wpb * 32, 0, c->stream>>>(b.id_lo, c->d_cl, c->d_mem, c->d_norb, c->d_row_ptr,
                                                          c->d_key, c->d_blk_off, c->d_rowblk_member, c->d_voff,
                                                          c->d_kat, c->k_lno, c->d_V, c->d_arena, rho_out, e_out);
    }
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

// ---------------------------------------------------------------------------
// SCF loop support (deferred mode): sticky status, per-step record, linear mixing
// ---------------------------------------------------------------------------
__global__ void k_status_or(int n, const int* __restrict__ status, int* __restrict__ err) {
    int w = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) w = max(w, status[i]);
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    __shared__ int red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) w = max(w, red[k]);
        if (w > err[0]) err[0] = w;
    }
}

// record mu, N(mu), E_band of this step (fixed summation order) and advance the step counter
__global__ void k_scf_record(int n, const double* __restrict__ scal, const double* __restrict__ eband,
                             int* __restrict__ err, double* __restrict__ hist, int cap) {
    if (threadIdx.x != 0) return;
    double e = 0.0;
    for (int i = 0; i < n; ++i) e += eband[i];
    const int k = err[1];
    if (k < cap) {
        hist[3 * k] = scal[2];
        hist[3 * k + 1] = scal[3];
        hist[3 * k + 2] = e;
    }
    if (scal[4] == 2.0 && err[0] < 16) err[0] = 16;  // no bracket for mu
    err[1] = k + 1;
}

// rho <- rho + alpha (rho_out - rho)
__global__ void k_mix(long long nval, double* __restrict__ rho, const double* __restrict__ rho_out, double alpha) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nval; t += (long long)gridDim.x * blockDim.x)
        rho[t] = fma(alpha, rho_out[t] - rho[t], rho[t]);
}

dclno_status launch_status_or(dclno_ctx* c) {
    k_status_or<<<1, 1024, 0, c->stream>>>(c->N, c->d_status, c->d_err);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

dclno_status launch_scf_tail(dclno_ctx* c, double* rho, const double* rho_out, double alpha) {
    k_scf_record<<<1, 32, 0, c->stream>>>(c->N, c->d_scalars, c->d_eband, c->d_err, c->d_hist, c->hist_cap);
    DCLNO_LAUNCHED(c);
    k_mix<<<c->nsm * 8, 256, 0, c->stream>>>(c->nval, rho, rho_out, alpha);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

// ---------------------------------------------------------------------------
// Chemical potential without any device allocation (dclno_find_mu_noalloc).
//
// Some callers cannot call cudaMalloc at all: applications that hand every byte
// of device memory to their own pool allocator up front, and control loops that
// must not allocate once they are running.  This variant keeps its scratch (the per-block partial
// sums of the k-section and its bracket scalars) in the file-scope array below,
// which every GPU that loads the library holds until the process exits.  The
// caller passes the (eps, q) pairs; one partial sum per block of
// 256 threads x NOALLOC_PER_THREAD pairs bounds the pair count.
// ---------------------------------------------------------------------------
#include <mutex>

#define NOALLOC_MAX_BLOCKS 4096
#define NOALLOC_PER_THREAD 8
#define NOALLOC_MAX_PAIRS ((long long)NOALLOC_MAX_BLOCKS * 256 * NOALLOC_PER_THREAD)
#define NOALLOC_SCALARS 64

// partial sums [NOALLOC_MAX_BLOCKS][KSEC + 2] followed by the bracket scalars (about 165 KB)
static __device__ __align__(256) double g_mu_scratch[NOALLOC_MAX_BLOCKS * (KSEC + 2) + NOALLOC_SCALARS];

static std::mutex g_mu_scratch_lock;
static double* g_mu_scratch_addr[128];  // device address of g_mu_scratch per device, set up once

extern "C" dclno_status dclno_find_mu_noalloc(const double* eps, const double* q, long long count, double n_electrons,
                                              double kT, double* mu_out, double* nelec_out, void* cuda_stream) {
    if (!eps || !q || count < 1 || !(kT > 0.0)) return DCLNO_ERR_ARG;
    if (count > NOALLOC_MAX_PAIRS) return DCLNO_ERR_ARG;  // more pairs than the static scratch covers
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return DCLNO_ERR_CUDA;
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu_scratch_lock);
        if (!g_mu_scratch_addr[dev]) {
            void* p = nullptr;
            // the host-side name g_mu_scratch is only a stand-in: ask the runtime for the device address
            if (cudaGetSymbolAddress(&p, g_mu_scratch) != cudaSuccess || !p) return DCLNO_ERR_CUDA;
            g_mu_scratch_addr[dev] = static_cast<double*>(p);
        }
        base = g_mu_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nblk = (int)((count + 256LL * NOALLOC_PER_THREAD - 1) / (256LL * NOALLOC_PER_THREAD));
    double* part = base;
    double* scal = base + NOALLOC_MAX_BLOCKS * (KSEC + 2);
    // every scratch word that is read is written first in this call: k_mu_init sets all
    // bracket scalars (the done flag to 0), each pass rewrites the partial sums it reads
    k_mu_bracket<<<nblk, 256, 0, st>>>(count, eps, part);
    k_mu_init<<<1, 32, 0, st>>>(nblk, part, scal, kT, n_electrons);
    for (int pass = 0; pass < MU_PASSES; ++pass) {
        k_mu_partial<<<nblk, 256, 0, st>>>(count, eps, q, scal, part, pass == 0);
        k_mu_update<<<1, 32 * (KSEC + 2), 0, st>>>(nblk, part, scal, pass == 0, pass == MU_PASSES - 1);
    }
    k_mu_final_partial<<<nblk, 256, 0, st>>>(count, eps, q, scal, part);
    k_mu_final<<<1, 32, 0, st>>>(nblk, part, scal);
    if (cudaGetLastError() != cudaSuccess) return DCLNO_ERR_CUDA;
    double h[10];
    if (cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DCLNO_ERR_CUDA;
    if (h[4] == 2.0) return DCLNO_ERR_NO_BRACKET;
    if (mu_out) *mu_out = h[2];
    if (nelec_out) *nelec_out = h[3];
    return DCLNO_OK;
}
