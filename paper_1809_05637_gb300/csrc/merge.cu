// Merge of a torn tridiagonal eigenproblem (Cuppen's divide and conquer, one level).
//
// k_tridiag tears T at k = n/2: T = diag(T1, T2) + rho v v^T, rho = |beta|,
// v = e_{k-1} + sign(beta) e_k (beta = T[k][k-1]).  k_ql solves T1 = Z1 D1 Z1^T and
// T2 = Z2 D2 Z2^T as two segments and applies each rotation also to the row v, so
// that z = diag(Z1, Z2)^T v is ready in W[0, n) when it finishes.  With that z,
//     T = diag(Z1, Z2) (D + rho z z^T) diag(Z1, Z2)^T,
// and the rank-one problem D + rho z z^T = U Lambda U^T is solved here:
//   * deflation (Bunch, Nielsen and Sorensen 1978; Dongarra and Sorensen 1987):
//     a component with rho |z_i| below the tolerance leaves d_i and e_i unchanged;
//     two nearly equal d's are combined by a plane rotation that zeroes one z;
//   * the K remaining roots of the secular equation 1 + rho sum_i z_i^2/(d_i - lam) = 0,
//     one in each (d_j, d_{j+1}) and one above d_K, by a safeguarded iteration on a
//     model with the two nearest poles, with lam stored as pole + offset so that every
//     difference d_i - lam is formed without cancellation; the first model steps of
//     each root run on an FP32 preview of the sums (GB300's FP32 rate is many times
//     its FP64 rate), the bracket and the converged root on FP64 sums;
//   * z recomputed from the computed roots (Gu and Eisenstat 1995),
//     z_i^2 = prod_j (lam_j - d_i) / (rho prod_{j != i} (d_j - d_i)), which makes the
//     eigenvectors u_j = (z_i / (d_i - lam_j))_i / norm numerically orthogonal.
// The eigenvectors of T are diag(Z1, Z2) U: U (the merge matrix M, n x n, and its
// transpose) is stored for the back-transforms (k_mgemm); the eigenvalues replace d.
#include "dclno_internal.cuh"

#define MG_THREADS 256

// psi = sum_{i<=j} w_i/(d_i - lam), phi = sum_{i>j} w_i/(d_i - lam), their derivatives
// in lam and sum |terms|, at lam = d_o + tau (differences d_i - d_o formed first)
struct SecVal {
    double psi, dpsi, phi, dphi, abs;
};

// The reciprocals 1 / (d_i - lam) are also stored in the root's column of the merge
// matrix (rcol[kidx[i] * ld]): the last evaluation is at the converged root, where they
// are the eigenvector's entries up to the factor z_i.
__device__ static SecVal sec_eval(int K, const double* dk, const double* w, int o, double tau, int j, double* rcol,
                                  int ld, const int* kidx) {
    SecVal v = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double dorg = dk[o];
    for (int i = 0; i <= j; ++i) {
        const double r = 1.0 / ((dk[i] - dorg) - tau);
        rcol[(size_t)kidx[i] * ld] = r;
        const double t = w[i] * r;
        v.psi += t;
        v.dpsi = fma(t, r, v.dpsi);
        v.abs += fabs(t);
    }
    for (int i = j + 1; i < K; ++i) {
        const double r = 1.0 / ((dk[i] - dorg) - tau);
        rcol[(size_t)kidx[i] * ld] = r;
        const double t = w[i] * r;
        v.phi += t;
        v.dphi = fma(t, r, v.dphi);
        v.abs += fabs(t);
    }
    return v;
}

// FP32 preview of the same sums, for the first model steps of a root: d is held as a
// pair of floats (dh + dl = d to about 2^-48 relative), so each difference d_i - d_o
// keeps about 24 correct bits even where d_i and d_o nearly coincide.  Only the root's
// starting point comes from it; every bracket update and the final root use sec_eval.
struct SecValF {
    float psi, dpsi, phi, dphi;
};

__device__ static SecValF sec_eval_f(int K, const float* dh, const float* dl, const float* wf, int o, float tau,
                                     int j) {
    SecValF v = {0.f, 0.f, 0.f, 0.f};
    const float ho = dh[o], lo = dl[o];
    for (int i = 0; i <= j; ++i) {
        const float r = __fdividef(1.0f, ((dh[i] - ho) + (dl[i] - lo)) - tau);
        const float t = wf[i] * r;
        v.psi += t;
        v.dpsi = fmaf(t, r, v.dpsi);
    }
    for (int i = j + 1; i < K; ++i) {
        const float r = __fdividef(1.0f, ((dh[i] - ho) + (dl[i] - lo)) - tau);
        const float t = wf[i] * r;
        v.phi += t;
        v.dphi = fmaf(t, r, v.dphi);
    }
    return v;
}

// root h of A h^2 - B h + C = 0 inside (lo, hi); NaN if none (the caller bisects)
template <typename T>
__device__ static T quad_root_in(T A, T B, T C, T lo, T hi) {
    const T nan_ = T(nan(""));
    if (A == T(0)) return (B != T(0)) ? C / B : nan_;
    const T disc = fma(B, B, -T(4) * A * C);
    if (!(disc >= T(0))) return nan_;
    const T sq = sqrt(disc);
    T h1, h2;
    if (B >= T(0)) {
        h1 = (B + sq) / (T(2) * A);
        h2 = (B + sq != T(0)) ? T(2) * C / (B + sq) : nan_;
    } else {
        h1 = T(2) * C / (B - sq);
        h2 = (B - sq) / (T(2) * A);
    }
    if (h2 > lo && h2 < hi) return h2;
    if (h1 > lo && h1 < hi) return h1;
    return nan_;
}


// Root j of 1 + sum_i w_i/(d_i - lam) = 0 (d ascending, w > 0, wsum = sum w):
// lam = d_o + tau.  Returns the number of iterations (> 100: not converged).
__device__ static int sec_root(int K, const double* dk, const double* w, const float* dh, const float* dl,
                               const float* wf, double wsum, int j, double& tau_out, int& org_out, double* rcol,
                               int ld, const int* kidx) {
    const double u = 1.1102230246251565e-16;  // 2^-53
    int o;
    double lo, hi, tau;
    SecVal v;
    SecValF vf;
    if (j < K - 1) {
        const double gap = dk[j + 1] - dk[j];
        const double mid = 0.5 * gap;
        // the side of the midpoint from the FP32 sums when their sign is certain (|f|
        // well above their rounding bound, K + 8 terms of 2^-23 relative each, sum |t|
        // = phi - psi at the midpoint), else from the FP64 sums
        vf = sec_eval_f(K, dh, dl, wf, j, (float)mid, j);
        const float f32 = 1.0f + vf.psi + vf.phi;
        bool up;
        if (fabsf(f32) > 8.0f * (float)(K + 8) * 5.96e-8f * (1.0f + vf.phi - vf.psi)) {
            up = f32 >= 0.0f;
        } else {
            v = sec_eval(K, dk, w, j, mid, j, rcol, ld, kidx);
            up = 1.0 + v.psi + v.phi >= 0.0;
            vf = {(float)v.psi, (float)v.dpsi, (float)v.phi, (float)v.dphi};
        }
        if (up) {  // root in (d_j, mid]: origin d_j
            o = j;
            lo = 0.0;
            hi = mid;
            tau = mid;
        } else {   // root in (mid, d_{j+1}): origin d_{j+1}
            o = j + 1;
            lo = mid - gap;
            hi = 0.0;
            tau = mid - gap;
        }
    } else {
        o = j;
        lo = 0.0;
        hi = wsum;  // f(d_K + sum w) >= 0
        tau = 0.5 * wsum;
        vf = sec_eval_f(K, dh, dl, wf, o, (float)tau, j);
    }
    // up to three model steps on the FP32 preview from the start; the FP64 iteration
    // below then starts where they end (if that lies in its bracket)
    {
        float tf = (float)tau, lof = (float)lo, hif = (float)hi;
        const float dpj = (float)(dk[j] - dk[o]);
        const float dqj = (j < K - 1) ? (float)(dk[j + 1] - dk[o]) : 0.f;
        for (int s = 0; s < 3; ++s) {
            if (s > 0) vf = sec_eval_f(K, dh, dl, wf, o, tf, j);
            const float f = 1.0f + vf.psi + vf.phi;
            if (f < 0.f) lof = tf;
            else hif = tf;
            const float dp = dpj - tf;
            const float b1 = vf.dpsi * dp * dp, a1 = vf.psi - b1 / dp;
            float h;
            if (j < K - 1) {
                const float dq = dqj - tf;
                const float b2 = vf.dphi * dq * dq, a2 = vf.phi - b2 / dq;
                const float A = 1.0f + a1 + a2;
                h = quad_root_in<float>(A, A * (dp + dq) + b1 + b2, dp * dq * f, dp, dq);
            } else {
                h = (1.0f + a1 > 0.f) ? dp + b1 / (1.0f + a1) : nanf("");
            }
            float tn = tf + h;
            if (!(tn > lof && tn < hif)) tn = 0.5f * (lof + hif);
            if (tn == tf) break;
            tf = tn;
        }
        const double ts = (double)tf;
        if (ts > lo && ts < hi) tau = ts;
        v = sec_eval(K, dk, w, o, tau, j, rcol, ld, kidx);
    }
    int it = 0;
    for (; it < 100; ++it) {
        const double f = 1.0 + v.psi + v.phi;
        if (f < 0.0) lo = tau;
        else hi = tau;
        if (fabs(f) <= 8.0 * u * (1.0 + v.abs) || hi - lo <= 4.0 * u * fmax(fabs(lo), fabs(hi))) break;
        // model: psi ~ a1 + b1/(p - x), phi ~ a2 + b2/(q - x), values and slopes matched at tau
        const double dp = (dk[j] - dk[o]) - tau;
        const double b1 = v.dpsi * dp * dp, a1 = v.psi - b1 / dp;
        double h;
        if (j < K - 1) {
            const double dq = (dk[j + 1] - dk[o]) - tau;
            const double b2 = v.dphi * dq * dq, a2 = v.phi - b2 / dq;
            const double A = 1.0 + a1 + a2;
            h = quad_root_in(A, A * (dp + dq) + b1 + b2, dp * dq * f, dp, dq);
        } else {
            h = (1.0 + a1 > 0.0) ? dp + b1 / (1.0 + a1) : nan("");
        }
        double tn = tau + h;
        // inside the bracket; the last root may sit on its upper end (K = 1: lam = d + w exactly)
        if (!(tn > lo && (tn < hi || (j == K - 1 && tn == hi)))) tn = 0.5 * (lo + hi);
        if (tn == tau) break;
        tau = tn;
        v = sec_eval(K, dk, w, o, tau, j, rcol, ld, kidx);
    }
    tau_out = tau;
    org_out = o;
    return it + 1;
}

__global__ void __launch_bounds__(MG_THREADS) k_merge(const ClusterDesc* __restrict__ cls,
                                                      const int* __restrict__ order, double* __restrict__ arena,
                                                      int* __restrict__ status) {
    extern __shared__ double sm[];
    const ClusterDesc dc = cls[order[blockIdx.x]];
    const int ci = dc.sidx;
    if (status[ci] != ST_OK) return;
    if (!dc.split) return;
    const int n = dc.n, ld = dc.ld, tid = threadIdx.x;
    double* dv = arena + dc.aux_off;
    const double* zin = arena + dc.w_off;  // z[0, n), beta at [n]
    const double beta = zin[n];
    double* M = arena + dc.m_off;       // row = coordinate, column = eigenpair
    double* MT = M + (size_t)n * ld;    // row = eigenpair
    double* dk = sm;          // sorted d; after deflation: the K non-deflated d
    double* zk = dk + n;      // sorted normalised z; after deflation: the K non-deflated z
    double* w = zk + n;       // rho' z_k^2
    double* tau = w + n;      // root offsets
    double* zh = tau + n;     // recomputed z
    double* dev = zh + n;     // deflated eigenvalues
    double* gcs = dev + n;    // rotation c, s pairs (2 n)
    double* nrm = gcs + 2 * n;  // column norms
    int* perm = reinterpret_cast<int*>(nrm + n);  // sorted position -> coordinate
    int* kidx = perm + n;     // non-deflated entry -> coordinate
    int* org = kidx + n;      // origin pole of root j
    int* colc = org + n;      // deflated column -> coordinate
    int* gpq = colc + n;      // rotation coordinate pairs (2 n)
    float* dhf = reinterpret_cast<float*>(gpq + 2 * n);  // d as float pairs (dh + dl) and w in float
    float* dlf = dhf + n;
    float* wff = dlf + n;
    __shared__ double red[MG_THREADS / 32][2];
    __shared__ int sK, sND, sNG, sFail;
    __shared__ double sRho, sWsum;

    // norm of z and the largest |d|
    double zz = 0.0, dmax = 0.0;
    for (int t = tid; t < n; t += MG_THREADS) {
        zz = fma(zin[t], zin[t], zz);
        dmax = fmax(dmax, fabs(dv[t]));
    }
    zz = warp_sum(zz);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((tid & 31) == 0) {
        red[tid >> 5][0] = zz;
        red[tid >> 5][1] = dmax;
    }
    __syncthreads();
    zz = 0.0;
    dmax = 0.0;
    for (int k = 0; k < MG_THREADS / 32; ++k) {
        zz += red[k][0];
        dmax = fmax(dmax, red[k][1]);
    }
    const double zscale = zz > 0.0 ? 1.0 / sqrt(zz) : 0.0;
    // sort (d, coordinate) ascending by rank counting; ties by coordinate
    for (int t = tid; t < n; t += MG_THREADS) {
        const double dt = dv[t];
        int r = 0;
        for (int s = 0; s < n; ++s) {
            const double ds = dv[s];
            r += (ds < dt || (ds == dt && s < t)) ? 1 : 0;
        }
        perm[r] = t;
        dk[r] = dt;
        zk[r] = zin[t] * zscale;
    }
    __syncthreads();
    // deflation (one thread, in sorted order)
    if (tid == 0) {
        const double rho = fabs(beta) * zz;
        const double tol = 8.0 * 1.1102230246251565e-16 * fmax(dmax, rho);
        int K = 0, nd = 0, ng = 0;
        bool have = false;
        double pd = 0.0, pz = 0.0;
        int pc = -1;
        for (int j = 0; j < n; ++j) {
            const double dj = dk[j], zj = zk[j];
            const int cj = perm[j];
            if (rho * fabs(zj) <= tol) {  // z_j negligible: (d_j, e_j) is an eigenpair
                dev[nd] = dj;
                colc[nd] = cj;
                ++nd;
                continue;
            }
            if (!have) {
                have = true;
                pd = dj;
                pz = zj;
                pc = cj;
                continue;
            }
            const double t = hypot(pz, zj);
            const double c = zj / t, s = -pz / t;
            if (fabs(c * s * (dj - pd)) <= tol) {
                // rotate (pc, cj) so that the z of pc vanishes; pc deflates
                gpq[2 * ng] = pc;
                gpq[2 * ng + 1] = cj;
                gcs[2 * ng] = c;
                gcs[2 * ng + 1] = s;
                ++ng;
                dev[nd] = fma(c * c, pd, s * s * dj);
                colc[nd] = pc;
                ++nd;
                pd = fma(s * s, pd, c * c * dj);
                pz = t;
                pc = cj;
            } else {
                dk[K] = pd;  // K <= j - 1: entries not yet read are not overwritten
                zk[K] = pz;
                kidx[K] = pc;
                ++K;
                pd = dj;
                pz = zj;
                pc = cj;
            }
        }
        if (have) {
            dk[K] = pd;
            zk[K] = pz;
            kidx[K] = pc;
            ++K;
        }
        sK = K;
        sND = nd;
        sNG = ng;
        sRho = rho;
        sFail = 0;
    }
    __syncthreads();
    const int K = sK, nd = sND, ng = sNG;
    const double rho = sRho;
    for (int i = tid; i < K; i += MG_THREADS) {
        w[i] = rho * zk[i] * zk[i];
        const float h = (float)dk[i];
        dhf[i] = h;
        dlf[i] = (float)(dk[i] - (double)h);
        wff[i] = (float)w[i];
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < K; ++i) s += w[i];
        sWsum = s;
    }
    __syncthreads();
    // M = 0; the secular roots (each root's last evaluation leaves 1 / (d_i - lam_j) in
    // column j of M)
    for (size_t e = tid; e < (size_t)n * ld; e += MG_THREADS) M[e] = 0.0;
    __syncthreads();
    for (int j = tid; j < K; j += MG_THREADS) {
        double t;
        int o;
        if (sec_root(K, dk, w, dhf, dlf, wff, sWsum, j, t, o, M + j, ld, kidx) > 100) sFail = 1;
        tau[j] = t;
        org[j] = o;
    }
    __syncthreads();
    // z from the computed roots (Gu-Eisenstat): numerator and denominator products
    // accumulated separately (one division per z instead of one per factor), their
    // exponents moved into integers every 16 factors so that neither over- nor underflows
    for (int i = tid; i < K; i += MG_THREADS) {
        const double di = dk[i];
        double pn = (dk[org[K - 1]] - di) + tau[K - 1], pd = rho;
        int en = 0, ed = 0;
        for (int j = 0; j < K - 1; ++j) {
            pn *= (dk[org[j]] - di) + tau[j];
            pd *= (j < i) ? (dk[j] - di) : (dk[j + 1] - di);
            if ((j & 15) == 15) {
                int e;
                pn = frexp(pn, &e);
                en += e;
                pd = frexp(pd, &e);
                ed += e;
            }
        }
        const double prod = ldexp(pn / pd, en - ed);
        zh[i] = copysign(sqrt(fmax(prod, 0.0)), zk[i]);
    }
    __syncthreads();
    // root columns: u_j = (z_i / (d_i - lam_j))_i at the non-deflated coordinates, from the
    // reciprocals the roots' last evaluations left in M
    for (int j = tid; j < K; j += MG_THREADS) {
        const double dj = dk[org[j]], tj = tau[j];
        double s = 0.0;
        for (int i = 0; i < K; ++i) {
            double* mij = M + (size_t)kidx[i] * ld + j;
            const double uij = zh[i] * *mij;
            *mij = uij;
            s = fma(uij, uij, s);
        }
        nrm[j] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        dv[j] = dj + tj;
    }
    for (int r = tid; r < nd; r += MG_THREADS) {
        M[(size_t)colc[r] * ld + K + r] = 1.0;
        dv[K + r] = dev[r];
    }
    __syncthreads();
    for (size_t e = tid; e < (size_t)K * n; e += MG_THREADS) {
        const int i = (int)(e / K), j = (int)(e % K);
        M[(size_t)i * ld + j] *= nrm[j];
    }
    __syncthreads();
    // undo the deflation rotations (last first): rows (p, q) <- R^T rows (p, q)
    for (int g = ng - 1; g >= 0; --g) {
        const int p = gpq[2 * g], q = gpq[2 * g + 1];
        const double c = gcs[2 * g], s = gcs[2 * g + 1];
        for (int col = tid; col < n; col += MG_THREADS) {
            const double a = M[(size_t)p * ld + col], b = M[(size_t)q * ld + col];
            M[(size_t)p * ld + col] = fma(c, a, -s * b);
            M[(size_t)q * ld + col] = fma(s, a, c * b);
        }
        __syncthreads();
    }
    for (size_t e = tid; e < (size_t)n * n; e += MG_THREADS) {
        const int col = (int)(e / n), r = (int)(e % n);
        MT[(size_t)col * ld + r] = M[(size_t)r * ld + col];
    }
    if (tid == 0 && sFail) status[ci] = ST_NOT_CONVERGED;
}

// z of the merge of a cluster torn twice (one CTA per cluster): with Q_h = diag(Z_2h,
// Z_2h+1) M_h the halves' eigenvectors and v = e_{k-1} + sign(beta) e_k at the cluster's
// tear k, z = diag(Q_0, Q_1)^T v: the first half's part is M_0^T applied to the last row of
// its second quarter's eigenvectors (carried by QL), the second half's part sign(beta)
// M_1^T applied to the first row of its first quarter's.
__global__ void __launch_bounds__(MG_THREADS) k_merge_z2(const ClusterDesc* __restrict__ cls,
                                                         const int* __restrict__ order, double* __restrict__ arena,
                                                         const int* __restrict__ status, int nreal) {
    const int ci = order[blockIdx.x];
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    if (!d.split2) return;
    const int n = d.n, ld = d.ld, k = d.split;
    const ClusterDesc h0 = cls[nreal + 2 * ci], h1 = cls[nreal + 2 * ci + 1];
    double* z = arena + d.w_off;  // z[0, n), beta at [n]
    const double* x2 = arena + d.x2_off;
    const double sgn = z[n] < 0.0 ? -1.0 : 1.0;
    const double* M0 = arena + h0.m_off;  // rows: the half's coordinates, columns: its eigenpairs
    const double* M1 = arena + h1.m_off;
    const int q1 = d.split1, q3 = d.split3;  // the first half's second quarter starts at q1, the second
                                              // half's first quarter ends at q3
    for (int j = threadIdx.x; j < n; j += MG_THREADS) {
        double s = 0.0;
        if (j < k) {
            for (int r = q1; r < k; ++r) s = fma(M0[(size_t)r * ld + j], x2[r], s);
        } else {
            for (int r = k; r < q3; ++r) s = fma(M1[(size_t)(r - k) * ld + (j - k)], x2[r], s);
            s *= sgn;
        }
        z[j] = s;
    }
}

dclno_status launch_merge(dclno_ctx* c, const Batch& b) {
    const int N1 = b.l1end - b.l1beg, N2 = b.l2end - b.l2beg;
    if (N1 == 0) return DCLNO_OK;
    bool any = false;
    for (int i = b.id_lo; i < b.id_hi; ++i) any = any || c->cl[i].split;
    if (!any) return DCLNO_OK;
    const size_t sm = (size_t)b.maxn * (10 * sizeof(double) + 6 * sizeof(int) + 3 * sizeof(float));
    if (sm > 227 * 1024) return set_err(c, DCLNO_ERR_ARG, "cluster dimension too large for the merge step");
    DCLNO_CUDA(c, cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ProfScope ps__(c, "k_merge");
    // the two-segment problems (clusters torn once, halves of the others), then the halves'
    // merge of the clusters torn twice
    const size_t sm1 = (size_t)b.l1maxn * (10 * sizeof(double) + 6 * sizeof(int) + 3 * sizeof(float));
    k_merge<<<N1, MG_THREADS, sm1, c->stream>>>(c->d_cl, c->d_l1 + b.l1beg, c->d_arena, c->d_status);
    DCLNO_LAUNCHED(c);
    if (N2 > 0) {
        k_merge_z2<<<N2, MG_THREADS, 0, c->stream>>>(c->d_cl, c->d_l2 + b.l2beg, c->d_arena, c->d_status, c->N);
        DCLNO_LAUNCHED(c);
        k_merge<<<N2, MG_THREADS, sm, c->stream>>>(c->d_cl, c->d_l2 + b.l2beg, c->d_arena, c->d_status);
        DCLNO_LAUNCHED(c);
    }
    return DCLNO_OK;
}
