// Density-matrix rows from the Green function summed over the Matsubara poles (the
// paper's Appendix, Eq. (rho0j), written for a non-orthogonal basis), a second route
// to Eq. (dm) that needs no eigenvectors.  With f(x) = 1/2 + (2/beta) sum_{p>=0}
// Re 1/(i w_p - x), w_p = (2p + 1) pi kT:
//   rho^(i) = S^-1/2 + (2/beta) Re sum_p (z_p S - H)^-1,   z_p = mu + i w_p.
// The cluster reduction of the spectral route gives S = L L^T, L^-1 H L^-T = Q T Q^T, so
//   rho^(i) = L^-T Q F_P(T) Q^T L^-1,
//   F_P(T) = 1/2 + (2/beta) [ Re sum_{p<P} (z_p - T)^-1
//                              - tau_1 (T - mu) + tau_2 (T - mu)^3 - tau_3 (T - mu)^5 ],
// the poles p >= P summed from the large-|z| expansion of Re (z_p - T)^-1 with
// tau_m = sum_{p>=P} w_p^-2m = (pi kT)^-2m zeta(2m, P + 1/2) / 4^m (Hurwitz zeta).  The
// central rows are rho_c,:^T = L^-T Q G with G = F_P(T) P1, P1 = (R1 Q)^T the central
// strip the spectral route also forms (k_apply_q_rows): each pole costs complex
// tridiagonal solves (z_p - T) x = b, O(n) per column of P1.  L^-T Q G and the scatter
// into the BSR rows are the spectral route's k_rho_qx and k_rho_scatter.
//
// z_p - T has Im = w_p on its diagonal, so LU without pivoting never meets a small pivot
// (every pivot has imaginary part >= w_p).  The expansion converges only when w_P is
// above the spectral radius of T - mu: a cluster whose Gershgorin bound exceeds w_P / 3
// is refused (ST_FEW_POLES, reported with the cluster) rather than summed wrongly.
#include <cmath>

#include "dclno_internal.cuh"

#define PL 32  // poles per warp pass (one per lane)

// Hurwitz zeta(s, a) for s >= 2, a > 0: the first N terms summed, the rest by the
// Euler-Maclaurin formula with Bernoulli numbers B_2 .. B_12.
static double hurwitz_zeta(int s, double a) {
    const int N = 24;
    double sum = 0.0;
    for (int k = 0; k < N; ++k) sum += std::pow(a + k, -s);
    const double x = a + N;
    sum += std::pow(x, 1 - s) / (s - 1) + 0.5 * std::pow(x, -s);
    static const double B[6] = {1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66, -691.0 / 2730};
    double fact = 1.0;  // (2j)!
    double rise = 1.0;  // s (s+1) ... (s + 2j - 2)
    for (int j = 1; j <= 6; ++j) {
        fact *= (2.0 * j - 1) * (2.0 * j);
        rise *= (j == 1) ? s : (s + 2.0 * j - 3) * (s + 2.0 * j - 2);
        sum += B[j - 1] / fact * rise * std::pow(x, -s - 2 * j + 1);
    }
    return sum;
}

// one warp per column a of P1 (lanes = poles of a pass); scratch per warp: r = 1/pivot and
// y/x (complex) for PL lanes x n rows, [t][lane] so that a row's lanes are contiguous
__global__ void k_poles(const ClusterDesc* __restrict__ cls, const int* __restrict__ order, double* __restrict__ arena,
                        int* __restrict__ status, double mu, double kT, int npoles, double tau1, double tau2,
                        double tau3, double2* __restrict__ scratch, long long per_warp) {
    const int ci = order[blockIdx.x];
    const int a = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ClusterDesc d = cls[ci];
    __shared__ double tear[3];
    __shared__ int tk[3];
    __shared__ int refuse;
    if (threadIdx.x == 0) {
        refuse = 0;
        const double* W = arena + d.aux_off + 3 * (size_t)d.ld;
        const bool ok = status[ci] == ST_OK && d.split;
        tk[0] = ok ? d.split : -1;
        tear[0] = ok ? W[d.n] : 0.0;
        tk[1] = ok && d.split2 ? d.split1 : -1;
        tear[1] = ok && d.split2 ? W[w_row(d.ld, DCLNO_W_HALF0) + d.split] : 0.0;
        tk[2] = ok && d.split2 ? d.split3 : -1;
        tear[2] = ok && d.split2 ? W[w_row(d.ld, DCLNO_W_HALF1) + (d.n - d.split)] : 0.0;
    }
    __syncthreads();
    if (status[ci] != ST_OK) return;
    const int n = d.n, ld = d.ld, mc = d.mc;
    const double* dv = arena + d.aux_off;
    const double* ev = dv + ld;
    const double* P = arena + d.cc_off;  // [n][2 mc]: P1 = columns 0 .. mc-1
    double* G = arena + d.aux_off + 3 * ld;  // [n][mc] out (overlaps the tears' betas, read above)
    // T before Cuppen's tears (at each tear k: d[k-1], d[k] lowered by |beta|, e[k-1] = 0)
    auto dt = [&](int t) {
        double v = dv[t];
        for (int q = 0; q < 3; ++q)
            if (tk[q] > 0 && (t == tk[q] - 1 || t == tk[q])) v += fabs(tear[q]);
        return v;
    };
    auto et = [&](int t) {
        for (int q = 0; q < 3; ++q)
            if (tk[q] > 0 && t == tk[q] - 1) return tear[q];
        return ev[t];
    };
    // Gershgorin bound of |T - mu| against the first omitted pole
    double rad = 0.0;
    for (int t = lane; t < n; t += 32)
        rad = fmax(rad, fabs(dt(t) - mu) + (t > 0 ? fabs(et(t - 1)) : 0.0) + (t + 1 < n ? fabs(et(t)) : 0.0));
    for (int o = 16; o > 0; o >>= 1) rad = fmax(rad, __shfl_xor_sync(0xffffffffu, rad, o));
    const double pi_kT = 3.14159265358979323846 * kT;
    if ((2.0 * npoles + 1.0) * pi_kT < 3.0 * rad) {
        if (lane == 0) refuse = 1;
    }
    __syncthreads();
    if (refuse) {
        if (threadIdx.x == 0) status[ci] = ST_FEW_POLES;
        return;
    }
    if (a >= mc) return;
    double2* r = scratch + (size_t)(blockIdx.x * (blockDim.x >> 5) + a) * per_warp;  // [n][PL]
    double2* y = r + (size_t)n * PL;                                                 // [n][PL]
    for (int t = lane; t < n; t += 32) G[(size_t)t * mc + a] = 0.0;
    __syncwarp();
    for (int p0 = 0; p0 < npoles; p0 += PL) {
        const int p = p0 + lane;
        const double w = (p < npoles) ? (2.0 * p + 1.0) * pi_kT : 0.0;
        // forward elimination of (z - T) x = b: pivots m_t, r_t = 1/m_t, y_t
        double2 rp = make_double2(0.0, 0.0), yp = make_double2(0.0, 0.0);
        for (int t = 0; t < n; ++t) {
            const double b = P[(size_t)t * 2 * mc + a];
            const double e = (t > 0) ? et(t - 1) : 0.0;
            const double e2 = e * e;
            const double mr = (mu - dt(t)) - e2 * rp.x, mi = w - e2 * rp.y;
            const double inv = 1.0 / fma(mr, mr, mi * mi);
            const double2 rt = make_double2(mr * inv, -mi * inv);
            // y_t = b + e y_{t-1} / m_{t-1}
            const double2 yt = make_double2(fma(e, yp.x * rp.x - yp.y * rp.y, b), e * (yp.x * rp.y + yp.y * rp.x));
            r[(size_t)t * PL + lane] = rt;
            y[(size_t)t * PL + lane] = yt;
            rp = rt;
            yp = yt;
        }
        // back substitution x_t = (y_t + e_t x_{t+1}) / m_t; the real part kept in place of y
        double2 xn = make_double2(0.0, 0.0);
        for (int t = n - 1; t >= 0; --t) {
            const double e = (t + 1 < n) ? et(t) : 0.0;
            const double2 yt = y[(size_t)t * PL + lane], rt = r[(size_t)t * PL + lane];
            const double ur = fma(e, xn.x, yt.x), ui = fma(e, xn.y, yt.y);
            xn = make_double2(ur * rt.x - ui * rt.y, ur * rt.y + ui * rt.x);
            y[(size_t)t * PL + lane] = make_double2(p < npoles ? xn.x : 0.0, 0.0);
        }
        __syncwarp();
        // sum over the pass's poles, a lane per row
        for (int t = lane; t < n; t += 32) {
            double s = 0.0;
            for (int l = 0; l < PL; ++l) s += y[(size_t)t * PL + l].x;
            G[(size_t)t * mc + a] += s;
        }
        __syncwarp();
    }
    // the tail of the pole sum: (-tau1 (T-mu) + tau2 (T-mu)^3 - tau3 (T-mu)^5) b, powers
    // through the scratch (u_k = (T - mu) u_{k-1}, u_0 = b), then G = b/2 + (2/beta)(G + tail)
    double* u0 = reinterpret_cast<double*>(r);
    double* u1 = u0 + n;
    for (int t = lane; t < n; t += 32) u0[t] = P[(size_t)t * 2 * mc + a];
    __syncwarp();
    for (int pw = 1; pw <= 5; ++pw) {
        for (int t = lane; t < n; t += 32) {
            double v = (dt(t) - mu) * u0[t];
            if (t > 0) v = fma(et(t - 1), u0[t - 1], v);
            if (t + 1 < n) v = fma(et(t), u0[t + 1], v);
            u1[t] = v;
        }
        __syncwarp();
        const double c = pw == 1 ? -tau1 : pw == 3 ? tau2 : pw == 5 ? -tau3 : 0.0;
        for (int t = lane; t < n; t += 32) {
            if (c != 0.0) G[(size_t)t * mc + a] = fma(c, u1[t], G[(size_t)t * mc + a]);
            u0[t] = u1[t];
        }
        __syncwarp();
    }
    const double two_over_beta = 2.0 * kT;
    for (int t = lane; t < n; t += 32)
        G[(size_t)t * mc + a] = fma(two_over_beta, G[(size_t)t * mc + a], 0.5 * P[(size_t)t * 2 * mc + a]);
}

dclno_status launch_poles(dclno_ctx* c, const Batch& b, double mu, double kT, int npoles) {
    const int N = b.oend - b.obeg;
    if (N == 0) return DCLNO_OK;
    const double a = npoles + 0.5, pk = 3.14159265358979323846 * kT;
    const double tau1 = hurwitz_zeta(2, a) / (pk * pk * 4.0);
    const double tau2 = hurwitz_zeta(4, a) / (std::pow(pk, 4) * 16.0);
    const double tau3 = hurwitz_zeta(6, a) / (std::pow(pk, 6) * 64.0);
    const long long per_warp = 2LL * b.maxn * PL;  // double2: r and y
    const size_t need = (size_t)N * b.mcmax * per_warp * sizeof(double2);
    if (c->pole_bytes < need) {
        if (c->d_pole) cudaFree(c->d_pole);
        c->d_pole = nullptr;
        c->pole_bytes = 0;
        DCLNO_CUDA(c, cudaMalloc(&c->d_pole, need));
        c->pole_bytes = need;
    }
    ProfScope ps__(c, "k_poles");
    k_poles<<<N, 32 * b.mcmax, 0, c->stream>>>(c->d_cl, c->d_order + b.obeg, c->d_arena, c->d_status, mu, kT,
                                                npoles, tau1, tau2, tau3, reinterpret_cast<double2*>(c->d_pole),
                                                per_warp);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}
