// Two-stage Householder tridiagonalisation of the congruence-transformed cluster
// matrix A = L^-1 H^(i) L^-T (Sec. II.C step (iii)), the alternative to the one-stage
// k_tridiag for clusters of dimension >= DCLNO_TWO_STAGE_MIN.
//
//   k_band   A = Q1 B Q1^T, B symmetric with half-bandwidth BW: panels of BW columns,
//            each a Householder QR of the block below the band (BW reflectors in
//            compact WY form I - V T V^T), then the two-sided update of the trailing
//            matrix A22 <- A22 - V W^T - W V^T with W = Y T - 1/2 V (T^T V^T Y T),
//            Y = A22 V.  Y, V^T [V | Y] and the rank-2 BW update are tile GEMMs (FP64
//            MMA, or FP64 emulated on BF16 tensor cores in the mixed path), so the
//            matrix-vector products of the one-stage reduction become matrix-matrix
//            products that read A22 once per panel instead of once per column.
//   k_chase  B = Q2 T Q2^T, T tridiagonal: Householder bulge chasing.  Sweep j
//            annihilates column j below its subdiagonal with a reflector on rows
//            [j+1, j+1+BW); its application from the right fills the block below the
//            window (the bulge), whose first column the next reflector, BW rows
//            further down, annihilates, and so on to the end of the matrix.  What
//            remains of each bulge lies in the columns that later sweeps annihilate,
//            so the matrix never grows beyond half-bandwidth 2 BW - 1.
//
// Storage (per cluster): the band and the bulges in A's lower triangle (zero below the
// band after k_band); the panel reflectors Q1 row-contiguous in A's otherwise unused
// upper triangle (reflector of column c in row c from column c + BW on, unit entry
// stored) with tau in the aux tau vector (0 where column c has none); the chase
// reflectors Q2 in the cluster's log at q2_off, one slot of BW doubles per reflector
// in generation order: [tau, v_1 .. v_{len-1}] (v_0 = 1).  The merge-matrix area, not
// used until after the tridiagonal eigensolve, is k_band's scratch.
#include "dclno_internal.cuh"
#include "emu_gemm.cuh"
#include "df32.cuh"

#define BW DCLNO_BW
#define TL (BW + 1)  // row stride of the BW x BW shared-memory blocks
static_assert(BW == 32, "the panel factorisation maps a panel column to a lane");
#define PQ 8  // panel rows per warp whose loads are issued together

// shared memory of k_band: GEMM staging (also the mirror's transpose tiles and step 8's
// operand columns), reduction scratch
__host__ __device__ inline size_t band_gemm_doubles(int emu) {
    const size_t g = (ENGINE_SMEM_BYTES(emu) + 7) / 8;
    const size_t mirror = 8 * 32 * 33;  // eight warps' 32 x 33 transpose tiles
    return g > mirror ? g : mirror;
}
__host__ __device__ inline size_t band_smem_bytes(int emu) { return (band_gemm_doubles(emu) + 64) * sizeof(double); }

// upper triangle of the trailing block [r0, n)^2 <- its lower triangle (32 x 32 tiles
// through shared memory, one tile per warp at a time)
__device__ static void mirror_lower(double* A, int ld, int r0, int n, double* tiles) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double* T = tiles + (size_t)warp * 32 * 33;
    const int nt = (n - r0 + 31) / 32;
    for (int t = warp; t < nt * (nt + 1) / 2; t += nw) {
        // tile (bi, bj) of the lower triangle, bj <= bi; copied transposed to (bj, bi)
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int bj = t - bi * (bi + 1) / 2;
        const int rb = r0 + 32 * bi, cb = r0 + 32 * bj;
        for (int r0b = 0; r0b < 32; r0b += 16) {  // 16 rows' loads in flight
            double x[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int gr = rb + r0b + i, gc = cb + lane;
                x[i] = (gr < n && gc < n && gc <= gr) ? A[(size_t)gr * ld + gc] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) T[(r0b + i) * 33 + lane] = x[i];
        }
        __syncwarp();
        // element (gr, gc), gc < gr, goes to (gc, gr): row cb + c of the upper triangle
        for (int c = 0; c < 32; ++c) {
            const int gr = rb + lane, gc = cb + c;
            if (gr < n && gc < n && gc < gr) A[(size_t)gc * ld + gr] = T[lane * 33 + c];
        }
        __syncwarp();
    }
}

template <int EMU>
__device__ __forceinline__ void band_one(const ClusterDesc* __restrict__ cls, int ci, double* __restrict__ arena,
                                         int* __restrict__ status, TcState* tcsp) {
    extern __shared__ double sm[];
    TcState& tcs = *tcsp;
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    if (!two_stage_cluster(d)) return;
    const int n = d.n, ld = d.ld;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    double* A = arena + d.mat_off;
    double* tauv = arena + d.aux_off + 2 * ld;
    // scratch in the merge-matrix area (2 n ld doubles, n >= DCLNO_TWO_STAGE_MIN)
    double* NVt = arena + d.m_off;            // BW x m (stride ld): -V^T
    double* Yt = NVt + (size_t)BW * ld;       // BW x m (stride ld): Y^T
    double* WV = NVt;                         // m x 2BW: [W | V], once -V^T and Y^T are dead
    double* Yr = Yt + (size_t)BW * ld;        // m x BW: Y = A22 V
    double* VW = Yr + (size_t)BW * ld;        // m x 2BW: [V | W]
    double* GZ = VW + (size_t)2 * BW * ld;    // [-V^T V | V^T Y], BW x 2BW (row stride gz)
    const int gz = 2 * BW + 1;
    double* Ts = GZ + BW * gz;                // T (upper triangular), BW x TL
    double* Ms = Ts + BW * TL;                // T^T (V^T Y) T, BW x TL
    double* NTt = Ms + BW * TL;               // -T^T, BW x BW
    double* HM = NTt + BW * BW;               // M / 2, BW x BW
    double* G = sm;
    double* vscale = sm + band_gemm_doubles(EMU);  // BW: the panel columns' reflector scalings
    constexpr int V2 = 2 * BW;

    for (int t = tid; t < n; t += blockDim.x) tauv[t] = 0.0;
    __syncthreads();
    for (int c0 = 0; c0 + BW < n; c0 += BW) {
        const int r0 = c0 + BW, m = n - r0;
        const int nbr = min(BW, m);  // reflectors of this panel (one per column with rows below the band)
        // (1) Householder QR of the panel block A[r0:n, c0:c0+BW]; reflector j acts on rows
        // r0+j ..  A lane per panel column, the warps over rows, one pass over the panel per
        // reflector: it applies reflector j and, on the updated rows, forms the products
        // d_l = x_{j+1}^T x_l below the next top row that reflector j+1 needs (its norm is
        // d_{j+1}; its scaling factors out of v^T x_l).  Every pass reads whole panel rows
        // (coalesced); the column sums go through shared memory, two buffers in turn.
        {
            double* cred = G;  // 2 x nw x BW partial column sums
            int cb = 0;
            double acc = 0.0;  // d_l for the first column
            for (int rb = r0 + 1 + warp; rb < n; rb += PQ * nw) {
                double x[PQ];
#pragma unroll
                for (int i = 0; i < PQ; ++i) {
                    const int r = rb + i * nw;
                    x[i] = r < n ? A[(size_t)r * ld + c0 + lane] : 0.0;
                }
#pragma unroll
                for (int i = 0; i < PQ; ++i) acc = fma(__shfl_sync(0xffffffffu, x[i], 0), x[i], acc);
            }
            cred[cb * nw * BW + warp * BW + lane] = acc;
            __syncthreads();
            double d = 0.0;  // lane l: d_l of the next reflector
            for (int q = 0; q < nw; ++q) d += cred[cb * nw * BW + q * BW + lane];
            cb ^= 1;
            for (int j = 0; j < nbr; ++j) {
                const int c = c0 + j, rs = r0 + j;
                const double alpha = A[(size_t)rs * ld + c];
                const double sig = __shfl_sync(0xffffffffu, d, j);
                double tau = 0.0, beta = alpha, scale = 0.0;
                if (sig > 0.0) {
                    const double nrm = sqrt(alpha * alpha + sig);
                    beta = (alpha >= 0.0) ? -nrm : nrm;
                    tau = (beta - alpha) / beta;
                    scale = 1.0 / (alpha - beta);
                }
                const double xtop = A[(size_t)rs * ld + c0 + lane];
                const double w = tau * fma(scale, d, xtop);  // tau v^T x_l, v = 1 on the top row
                const double ws = w * scale;                 // x_l <- x_l - ws x_j below the top row
                double na = 0.0;
                for (int rb = rs + 1 + warp; rb < n; rb += PQ * nw) {
                    double x[PQ];  // PQ rows' loads in flight before any store
#pragma unroll
                    for (int i = 0; i < PQ; ++i) {
                        const int r = rb + i * nw;
                        x[i] = r < n ? A[(size_t)r * ld + c0 + lane] : 0.0;
                    }
#pragma unroll
                    for (int i = 0; i < PQ; ++i) {
                        const int r = rb + i * nw;
                        const double xj = __shfl_sync(0xffffffffu, x[i], j);
                        if (lane > j) {
                            x[i] = fma(-ws, xj, x[i]);
                            if (r < n) A[(size_t)r * ld + c0 + lane] = x[i];
                        }
                        const double u = __shfl_sync(0xffffffffu, x[i], (j + 1) & (BW - 1));
                        if (r > rs + 1 && r < n) na = fma(u, x[i], na);
                    }
                }
                cred[cb * nw * BW + warp * BW + lane] = na;
                __syncthreads();
                d = 0.0;
                for (int q = 0; q < nw; ++q) d += cred[cb * nw * BW + q * BW + lane];
                cb ^= 1;
                // the top row, after every thread has read it (later reflectors start below it)
                if (warp == 0) {
                    if (lane > j) A[(size_t)rs * ld + c0 + lane] = xtop - w;
                    if (lane == j) {
                        A[(size_t)rs * ld + c] = beta;
                        tauv[c] = tau;
                        vscale[j] = scale;  // column j below the top row holds v / scale until step (2)
                    }
                }
            }
        }
        // (2) explicit V (unit diagonal, zero above) as [V | .] and -V^T; the reflectors'
        // row-contiguous copies for the back-transforms in the upper triangle (row c from
        // column c + BW on); the lower triangle below the band is cleared for the chase
        __syncthreads();
        for (int e = tid; e < m * BW; e += blockDim.x) {
            const int t = e / BW, j = e % BW;
            const double v =
                (j >= nbr || t < j) ? 0.0 : (t == j ? 1.0 : A[(size_t)(r0 + t) * ld + c0 + j] * vscale[j]);
            VW[(size_t)t * V2 + j] = v;
            NVt[(size_t)j * ld + t] = -v;
            if (j < nbr && t >= j) A[(size_t)(c0 + j) * ld + r0 + t] = v;
        }
        __syncthreads();
        for (int e = tid; e < m * BW; e += blockDim.x) {
            const int t = e / BW, j = e % BW;
            if (j < nbr && t > j) A[(size_t)(r0 + t) * ld + c0 + j] = 0.0;
            Yr[e] = 0.0;
        }
        // (3) the trailing block in full (upper triangle from the lower) for Y = A22 V
        mirror_lower(A, ld, r0, n, G);
        __syncthreads();
        // (4) Y = A22 V: C -= A22 (-V^T)^T; then Y^T for the next product
        double* A22 = A + (size_t)r0 * ld + r0;
        if constexpr (EMU == 2)  // one FP64 epilogue per element
            cta_gemm_tc_longk<false>(Yr, BW, A22, ld, NVt, ld, m, BW, m, reinterpret_cast<unsigned char*>(G), &tcs);
        else
            tile_update_longk<EMU>(Yr, BW, A22, ld, NVt, ld, m, BW, m, G, &tcs);
        for (int e = tid; e < BW * m; e += blockDim.x) {
            const int a = e / m, t = e % m;
            Yt[(size_t)a * ld + t] = Yr[(size_t)t * BW + a];
        }
        // (5) [-V^T V | V^T Y] = -(-V^T) [-V^T ; Y^T]^T ... as C -= A B^T with B = the 2BW rows
        // of NVt and Yt (contiguous, stride ld): C = -(V^T V) on the left, +V^T Y on the right
        for (int e = tid; e < BW * gz; e += blockDim.x) GZ[e] = 0.0;
        __syncthreads();
        if constexpr (EMU == 2)  // its transpose [-V^T V ; Y^T V] = -[-V^T ; Y^T] (-V^T)^T, written transposed
            cta_gemm_tc_longk<true>(GZ, gz, NVt, ld, NVt, ld, 2 * BW, BW, m, reinterpret_cast<unsigned char*>(G), &tcs);
        else
            tile_update_longk<EMU>(GZ, gz, NVt, ld, NVt, ld, BW, 2 * BW, m, G, &tcs);
        // (6) T (upper triangular): T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V^T V)[0:j, j]
        if (warp == 0) {
            for (int j = 0; j < BW; ++j) {
                const double tj = (j < nbr) ? tauv[c0 + j] : 0.0;
                double s = 0.0;
                if (lane < j)
                    for (int l = lane; l < j; ++l) s = fma(Ts[lane * TL + l], -GZ[l * gz + j], s);
                __syncwarp();
                if (lane < j) Ts[lane * TL + j] = -tj * s;
                if (lane == j) Ts[j * TL + j] = tj;
                if (lane > j) Ts[lane * TL + j] = 0.0;
                __syncwarp();
            }
        }
        __syncthreads();
        // (7) M = T^T (V^T Y) T  (BW x BW, symmetric): first P = (V^T Y) T into Ms, then T^T P
        for (int e = tid; e < BW * BW; e += blockDim.x) {
            const int a = e / BW, b = e % BW;
            double s = 0.0;
            for (int l = 0; l <= b; ++l) s = fma(GZ[a * gz + BW + l], Ts[l * TL + b], s);
            Ms[a * TL + b] = s;
        }
        __syncthreads();
        {
            double mv[BW / 8];
            for (int q = 0; q < BW * BW / DCLNO_SOLVE_THREADS; ++q) {
                const int e = tid + q * DCLNO_SOLVE_THREADS, a = e / BW, b = e % BW;
                double s = 0.0;
                for (int l = 0; l <= a; ++l) s = fma(Ts[l * TL + a], Ms[l * TL + b], s);
                mv[q] = s;
            }
            __syncthreads();
            for (int q = 0; q < BW * BW / DCLNO_SOLVE_THREADS; ++q) {
                const int e = tid + q * DCLNO_SOLVE_THREADS;
                Ms[(e / BW) * TL + e % BW] = mv[q];
            }
        }
        __syncthreads();
        // (8) W = Y T - 1/2 V M (m x BW) as two tile products into the right half of [V | W]:
        // B operands -T^T and M/2 (M is symmetric), both row-major with K contiguous
        for (int e = tid; e < BW * BW; e += blockDim.x) {
            const int b = e / BW, a = e % BW;
            NTt[e] = -Ts[a * TL + b];
            HM[e] = 0.5 * Ms[a * TL + b];
        }
        for (int e = tid; e < m * BW; e += blockDim.x) VW[(size_t)(e / BW) * V2 + BW + e % BW] = 0.0;
        __syncthreads();
        tile_update<false, EMU>(VW + BW, V2, Yr, BW, NTt, BW, m, BW, BW, 0, G, &tcs);
        tile_update<false, EMU>(VW + BW, V2, VW, V2, HM, BW, m, BW, BW, 0, G, &tcs);
        for (int e = tid; e < m * BW; e += blockDim.x) {
            const int t = e / BW, b = e % BW;
            WV[(size_t)t * V2 + b] = VW[(size_t)t * V2 + BW + b];
            WV[(size_t)t * V2 + BW + b] = VW[(size_t)t * V2 + b];
        }
        __syncthreads();
        // (9) A22 <- A22 - V W^T - W V^T (lower triangle).  FP64 tiles take [V | W] [W | V]^T
        // with K = 2 BW in one pass; the emulated engines take the two products apart: a
        // row of [V | W] sliced against its largest exponent would hold V (entries of
        // order 1) with as many fewer bits as W (of order |A|) is larger, and the slice
        // levels kept are relative to the product of the row maxima
        if constexpr (EMU == 0) {
            cta_gemm_nt_sub<true>(A22, ld, VW, V2, WV, V2, m, m, V2, 0, G);
        } else {
            tile_update<true, EMU>(A22, ld, VW, V2, WV, V2, m, m, BW, 0, G, &tcs);
            tile_update<true, EMU>(A22, ld, VW + BW, V2, WV + BW, V2, m, m, BW, 0, G, &tcs);
        }
    }
    if (EMU == 2 && tcs.failed && tid == 0) status[ci] = ST_TIMEOUT;
}

template <int EMU>
__global__ void __launch_bounds__(DCLNO_SOLVE_THREADS, DCLNO_CTAS_PER_SM(EMU)) k_band(
    const ClusterDesc* __restrict__ cls, const int* __restrict__ order, double* __restrict__ arena,
    int* __restrict__ status, int nitems, int* __restrict__ queue) {
    CUBIC_KERNEL_LOOP(EMU, band_one<EMU>(cls, order[it], arena, status, &tcs))
}

// ---------------------------------------------------------------------------
// Bulge chasing, one warp per cluster.  Window blocks are staged in shared memory:
// D (the symmetric diagonal block of the current reflector) and O (the block below
// the window, which the reflector fills from the right; it is carried to the next
// step, whose reflector annihilates its first column and is applied to the rest of it
// from the left).
// ---------------------------------------------------------------------------
struct Refl {
    double v, tau, beta;  // this lane's entry of v (v_0 = 1), tau, new leading entry
};

// reflector H = I - tau v v^T with H x = beta e_0 for x = (lane < len ? x : 0)
__device__ __forceinline__ Refl warp_householder(double x, int len) {
    const int lane = threadIdx.x & 31;
    const double alpha = __shfl_sync(0xffffffffu, x, 0);
    const double sig = warp_sum((lane >= 1 && lane < len) ? x * x : 0.0);
    Refl h;
    h.tau = 0.0;
    h.beta = alpha;
    h.v = (lane == 0) ? 1.0 : 0.0;
    if (sig > 0.0) {
        const double nrm = sqrt(alpha * alpha + sig);
        h.beta = (alpha >= 0.0) ? -nrm : nrm;
        h.tau = (h.beta - alpha) / h.beta;
        if (lane >= 1 && lane < len) h.v = x / (alpha - h.beta);
    }
    return h;
}

// D <- H D H for the symmetric window [p, p + len) (lower triangle in A)
__device__ static void chase_two_sided(double* A, int ld, int p, int len, const Refl& h, double* Ds) {
    const int lane = threadIdx.x & 31;
#pragma unroll 4
    for (int i = 0; i < len; ++i)
        if (lane <= i) {
            const double a = A[(size_t)(p + i) * ld + p + lane];
            Ds[i * TL + lane] = a;
            Ds[lane * TL + i] = a;
        }
    __syncwarp();
    double y0 = 0.0, y1 = 0.0;
    for (int c = 0; c < len; c += 2) {
        const double v0 = __shfl_sync(0xffffffffu, h.v, c);
        const double v1 = __shfl_sync(0xffffffffu, h.v, c + 1);
        if (lane < len) {
            y0 = fma(Ds[lane * TL + c], v0, y0);
            if (c + 1 < len) y1 = fma(Ds[lane * TL + c + 1], v1, y1);
        }
    }
    const double y = h.tau * (y0 + y1);
    const double dot = warp_sum(lane < len ? h.v * y : 0.0);
    const double w = y - 0.5 * h.tau * dot * h.v;
    // D - v w^T - w v^T on the lower triangle: the off-diagonal elements of rows i and
    // len-1-i share a warp instruction (i + (len-1-i) lanes), then the diagonal; every
    // FP64 instruction then updates up to 31 elements instead of i + 1
    for (int i = 0; 2 * i < len; ++i) {
        const int r2 = len - 1 - i;
        const bool first = lane < i;
        const int row = first ? i : r2, col = first ? lane : lane - i;
        const bool on = first || (r2 > i && col < r2);
        const double vr = __shfl_sync(0xffffffffu, h.v, row), wr = __shfl_sync(0xffffffffu, w, row);
        const double vc = __shfl_sync(0xffffffffu, h.v, col & 31), wc = __shfl_sync(0xffffffffu, w, col & 31);
        if (on) A[(size_t)(p + row) * ld + p + col] = Ds[row * TL + col] - vr * wc - wr * vc;
    }
    if (lane < len) A[(size_t)(p + lane) * ld + p + lane] = Ds[lane * TL + lane] - h.v * w - w * h.v;
    __syncwarp();
}

// Os (rows [p + len, p + len + nr) x cols [p, p + len)) loaded and multiplied by H from the right
__device__ static void chase_right(const double* A, int ld, int p, int len, int nr, const Refl& h, double* Os) {
    const int lane = threadIdx.x & 31;
#pragma unroll 4
    for (int r = 0; r < nr; ++r) Os[r * TL + lane] = (lane < len) ? A[(size_t)(p + len + r) * ld + p + lane] : 0.0;
    __syncwarp();
    double s0 = 0.0, s1 = 0.0;
    for (int c = 0; c < len; c += 2) {
        const double v0 = __shfl_sync(0xffffffffu, h.v, c);
        const double v1 = __shfl_sync(0xffffffffu, h.v, c + 1);
        if (lane < nr) {
            s0 = fma(Os[lane * TL + c], v0, s0);
            if (c + 1 < len) s1 = fma(Os[lane * TL + c + 1], v1, s1);
        }
    }
    const double s = h.tau * (s0 + s1);
    for (int r = 0; r < nr; ++r) {
        const double sr = __shfl_sync(0xffffffffu, s, r);
        if (lane < len) Os[r * TL + lane] = fma(-sr, h.v, Os[r * TL + lane]);
    }
    __syncwarp();
}

__device__ static void chase_store(double* A, int ld, int row0, int col0, int nr, int nc, const double* Os) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < nr; ++r)
        if (lane < nc) A[(size_t)(row0 + r) * ld + col0 + lane] = Os[r * TL + lane];
    __syncwarp();
}

__device__ __forceinline__ void chase_one(const ClusterDesc* __restrict__ cls, int ci, double* __restrict__ arena,
                                          const int* __restrict__ status) {
    extern __shared__ double sm[];
    double* Ds = sm;
    double* Os = sm + BW * TL;
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    if (!two_stage_cluster(d)) return;
    const int n = d.n, ld = d.ld, lane = threadIdx.x;
    double* A = arena + d.mat_off;
    double* slot = arena + d.q2_off;
    for (int j = 0; j + 2 < n; ++j) {
        const int nsteps = (int)chase_steps(n, j);
        int p = j + 1, len = min(BW, n - p);
        // step 0: column j below its subdiagonal
        Refl h = warp_householder(lane < len ? A[(size_t)(p + lane) * ld + j] : 0.0, len);
        if (lane < len) A[(size_t)(p + lane) * ld + j] = (lane == 0) ? h.beta : 0.0;
        if (lane == 0) slot[0] = h.tau;
        else if (lane < len) slot[lane] = h.v;
        slot += BW;
        chase_two_sided(A, ld, p, len, h, Ds);
        int nr = max(0, min(BW, n - p - len));
        chase_right(A, ld, p, len, nr, h, Os);
        for (int k = 1; k < nsteps; ++k) {
            // the carried block O holds rows [p + BW, ...) x cols [p, p + BW) (len == BW here)
            const int pp = p;
            p = pp + BW;
            len = min(BW, n - p);  // == nr
            h = warp_householder(lane < len ? Os[lane * TL] : 0.0, len);
            if (lane < len) Os[lane * TL] = (lane == 0) ? h.beta : 0.0;
            if (lane == 0) slot[0] = h.tau;
            else if (lane < len) slot[lane] = h.v;
            slot += BW;
            __syncwarp();
            // from the left on the carried block's other columns (lane = column)
            {
                double s0 = 0.0, s1 = 0.0;
                for (int i = 0; i < len; i += 2) {
                    const double v0 = __shfl_sync(0xffffffffu, h.v, i);
                    const double v1 = __shfl_sync(0xffffffffu, h.v, i + 1);
                    if (lane >= 1) {
                        s0 = fma(v0, Os[i * TL + lane], s0);
                        if (i + 1 < len) s1 = fma(v1, Os[(i + 1) * TL + lane], s1);
                    }
                }
                const double s = h.tau * (s0 + s1);
                for (int i = 0; i < len; ++i) {
                    const double vi = __shfl_sync(0xffffffffu, h.v, i);
                    if (lane >= 1) Os[i * TL + lane] = fma(-s, vi, Os[i * TL + lane]);
                }
                __syncwarp();
            }
            chase_store(A, ld, p, pp, len, BW, Os);
            chase_two_sided(A, ld, p, len, h, Ds);
            nr = max(0, min(BW, n - p - len));
            chase_right(A, ld, p, len, nr, h, Os);
        }
        chase_store(A, ld, p + len, p, nr, len, Os);
    }
    // the tridiagonal matrix: d, e into the aux vectors, then Cuppen's tear as in k_tridiag
    double* dv = arena + d.aux_off;
    double* ev = dv + ld;
    for (int t = lane; t < n; t += 32) {
        dv[t] = A[(size_t)t * ld + t];
        ev[t] = (t + 1 < n) ? A[(size_t)(t + 1) * ld + t] : 0.0;
    }
    __syncwarp();
    if (lane == 0) tear_cluster(d, arena);
}

// ---------------------------------------------------------------------------
// The same bulge chasing in double-float arithmetic (df32.cuh), for the mixed path.
// The band is first copied into a compact double-float layout in the merge-matrix
// area: row r holds the entries (r, r - k), k = 0 .. 2 BW - 1 (the band and the
// bulges), at Bd[r * BD + k].  The chase then takes the steps of chase_one on Bd.
// Each reflector is formed in double-float from its column (norm, square root and
// divisions: df_reflector, the steps of warp_householder) and logged in FP64 for the
// back-transforms; its application, the bulk of the work (about 6 BW^2 multiply-adds
// per reflector), runs on the FP32 pipe as well.
// The diagonal and subdiagonal go back to FP64 at the end.
//
// A cluster's band (n x 2 BW entries) and those of the other clusters in flight do not
// fit in L2, so every block a step reads comes from HBM.  Each step's two blocks are
// fetched by asynchronous copies (cp.async, one 8-byte entry per lane and row) issued
// ahead of their use: the diagonal block D of step k + 1 while step k multiplies its
// block below the window, that block O while step k updates D.  Neither region is
// written between the copy and its use: within a sweep, step k writes rows
// [p, p + BW) only, and the sweep before has finished.
// ---------------------------------------------------------------------------
#define BD (2 * BW)

__device__ __forceinline__ df32 df_zero() { return df_make(0.0f, 0.0f); }

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// copies of D's lower triangle (rows [p, p + len)) into Ds, one group
__device__ __forceinline__ void fetch_d(const df32* Bd, int p, int len, df32* Ds) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < len; ++i) cp_async8(&Ds[i * TL + lane], &Bd[(size_t)(p + i) * BD + i - lane]);
    cp_async_commit();
}

// copies of the block below the window (rows [p + len, p + len + nr) x cols [p, p + len))
// into Os, one group; columns >= len are zero
__device__ __forceinline__ void fetch_o(const df32* Bd, int p, int len, int nr, df32* Os) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < nr; ++r) {
        if (lane < len) cp_async8(&Os[r * TL + lane], &Bd[(size_t)(p + len + r) * BD + len + r - lane]);
        else Os[r * TL + lane] = df_zero();
    }
    cp_async_commit();
}

// Shared memory of a chase warp (double-float): the blocks D and O (BW x TL each), then
// the reflector v, the vector w of the two-sided update and the row scalings s (BW each)
#define CH_VS (2 * BW * TL)
#define CH_WS (CH_VS + BW)
#define CH_SS (CH_WS + BW)
#define CH_DF_ENTRIES (CH_SS + BW)

// The step functions take the window length len and the rows nr below it; FULL (len ==
// nr == BW, every step but a sweep's last one or two) fixes both at compile time, so the
// loops unroll without guards, by CH_UNROLL_DOT term pairs in the dot products and
// CH_UNROLL_UPD rows in the updates.  Measured on the 1,728-cluster rock-salt step
// (k_chase per launch): 97 ms at 4 / 8, 98-100 ms at 2-4 / 2-8, 107 ms without
// unrolling, 112-123 ms at 8-16 / 16, 144 ms fully unrolled (168 registers and spills).
constexpr int CH_UNROLL_DOT = 4;
constexpr int CH_UNROLL_UPD = 8;

// D <- H D H for the window [p, p + len) (H = I - tau v v^T); Ds holds D's lower
// triangle, Vs the reflector
template <bool FULL>
__device__ static void chase_two_sided_df(df32* Bd, int p, int len_rt, df32 v, df32 tau, const df32* Ds,
                                          const df32* Vs, df32* Ws) {
    const int lane = threadIdx.x & 31;
    const int len = FULL ? BW : len_rt;
    df_acc y0 = df_acc_zero(), y1 = df_acc_zero();
#pragma unroll(FULL ? CH_UNROLL_DOT : 1)
    for (int c = 0; c < len; c += 2) {
        if (FULL || lane < len) {
            df_acc_add(y0, Ds[c <= lane ? lane * TL + c : c * TL + lane], Vs[c]);
            if (FULL || c + 1 < len) df_acc_add(y1, Ds[c + 1 <= lane ? lane * TL + c + 1 : (c + 1) * TL + lane], Vs[c + 1]);
        }
    }
    const df32 y = df_mul(tau, df_acc_merge(y0, y1));
    const df32 dot = df_warp_sum((FULL || lane < len) ? df_mul(v, y) : df_zero());
    const df32 hc = df_mul(df_make(0.5f * tau.hi, 0.5f * tau.lo), dot);
    const df32 w = df_fma(df_neg(hc), v, y);
    Ws[lane] = w;
    __syncwarp();
    // rows i and len-1-i of the lower triangle in one pass (as in chase_two_sided)
#pragma unroll(FULL ? CH_UNROLL_DOT : 1)
    for (int i = 0; 2 * i < len; ++i) {
        const int r2 = len - 1 - i;
        const bool first = lane < i;
        const int row = first ? i : r2, col = first ? lane : lane - i;
        const bool on = first || (r2 > i && col < r2);
        if (on)
            Bd[(size_t)(p + row) * BD + row - col] = df_sub2(Ds[row * TL + col], Vs[row], Ws[col], Ws[row], Vs[col]);
    }
    if (FULL || lane < len) Bd[(size_t)(p + lane) * BD] = df_sub2(Ds[lane * TL + lane], v, w, w, v);
    __syncwarp();
}

// O <- O H for the fetched block below the window (nr rows)
template <bool FULL>
__device__ static void chase_right_df(int len_rt, int nr_rt, df32 v, df32 tau, df32* Os, const df32* Vs, df32* Ss) {
    const int lane = threadIdx.x & 31;
    const int len = FULL ? BW : len_rt, nr = FULL ? BW : nr_rt;
    df_acc s0 = df_acc_zero(), s1 = df_acc_zero();
#pragma unroll(FULL ? CH_UNROLL_DOT : 1)
    for (int c = 0; c < len; c += 2) {
        if (FULL || lane < nr) {
            df_acc_add(s0, Os[lane * TL + c], Vs[c]);
            if (FULL || c + 1 < len) df_acc_add(s1, Os[lane * TL + c + 1], Vs[c + 1]);
        }
    }
    Ss[lane] = df_neg(df_mul(tau, df_acc_merge(s0, s1)));
    __syncwarp();
#pragma unroll(FULL ? CH_UNROLL_UPD : 1)
    for (int r = 0; r < nr; ++r)
        if (FULL || lane < len) Os[r * TL + lane] = df_fma(Ss[r], v, Os[r * TL + lane]);
    __syncwarp();
}

// O <- H O on the carried block's columns 1 .. BW-1 (lane = column; len rows)
template <bool FULL>
__device__ static void chase_left_df(int len_rt, df32 tau, df32* Os, const df32* Vs) {
    const int lane = threadIdx.x & 31;
    const int len = FULL ? BW : len_rt;
    df_acc s0 = df_acc_zero(), s1 = df_acc_zero();
#pragma unroll(FULL ? CH_UNROLL_DOT : 1)
    for (int i = 0; i < len; i += 2) {
        df_acc_add(s0, Vs[i], Os[i * TL + lane]);
        if (FULL || i + 1 < len) df_acc_add(s1, Vs[i + 1], Os[(i + 1) * TL + lane]);
    }
    const df32 ns = df_neg(df_mul(tau, df_acc_merge(s0, s1)));
#pragma unroll(FULL ? CH_UNROLL_UPD : 1)
    for (int i = 0; i < len; ++i)
        if (lane >= 1) Os[i * TL + lane] = df_fma(ns, Vs[i], Os[i * TL + lane]);
    __syncwarp();
}

// rows [row0, row0 + nr) x cols [col0, col0 + nc) of the band <- Os
__device__ static void chase_store_df(df32* Bd, int row0, int col0, int nr, int nc, const df32* Os) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < nr; ++r)
        if (lane < nc) Bd[(size_t)(row0 + r) * BD + row0 + r - col0 - lane] = Os[r * TL + lane];
    __syncwarp();
}

// Reflector H = I - tau v v^T with H x = beta e_0 for this lane's entry x of the column
// (lanes >= len hold 0), as in warp_householder but in double-float (norm, square root
// and divisions included); v goes to Vs, tau and v to the FP64 log slot.
__device__ __forceinline__ void df_reflector(df32 x, int len, double* slot, df32* Vs, df32& v, df32& tau,
                                             df32& beta) {
    const int lane = threadIdx.x & 31;
    const df32 alpha = df_shfl(x, 0);
    const df32 sig = df_warp_sum((lane >= 1 && lane < len) ? df_mul(x, x) : df_zero());
    tau = df_zero();
    beta = alpha;
    v = df_make(lane == 0 ? 1.0f : 0.0f, 0.0f);
    if (sig.hi > 0.0f) {  // the same for every lane
        const df32 nrm = df_sqrt(df_fma(alpha, alpha, sig));
        beta = (alpha.hi >= 0.0f) ? df_neg(nrm) : nrm;
        const df32 am = df_add(alpha, df_neg(beta));  // alpha - beta
        tau = df_div(df_neg(am), beta);
        const df32 inv = df_div(df_make(1.0f, 0.0f), am);
        if (lane >= 1 && lane < len) v = df_mul(x, inv);
    }
    Vs[lane] = v;
    if (lane == 0) slot[0] = df_to_double(tau);
    else if (lane < len) slot[lane] = df_to_double(v);
    __syncwarp();
}

__device__ __forceinline__ void chase_one_df(const ClusterDesc* __restrict__ cls, int ci, double* __restrict__ arena,
                                             const int* __restrict__ status) {
    extern __shared__ double sm[];
    df32* Ds = reinterpret_cast<df32*>(sm);
    df32* Os = Ds + BW * TL;
    df32* Vs = Ds + CH_VS;
    df32* Ws = Ds + CH_WS;
    df32* Ss = Ds + CH_SS;
    if (status[ci] != ST_OK) return;
    const ClusterDesc d = cls[ci];
    if (!two_stage_cluster(d)) return;
    const int n = d.n, ld = d.ld, lane = threadIdx.x;
    const double* A = arena + d.mat_off;
    df32* Bd = reinterpret_cast<df32*>(arena + d.m_off);  // n x BD (merge area: 2 n ld doubles)
    double* slot = arena + d.q2_off;
    // the band (k <= BW) and zeros for the bulges, eight rows' loads in flight
    for (int r0 = 0; r0 < n; r0 += 8) {
        double x[8][2];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + q, k = lane + 32 * h, c = r - k;
                x[q][h] = (r < n && k <= BW && c >= 0) ? A[(size_t)r * ld + c] : 0.0;
            }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (r0 + q < n) Bd[(size_t)(r0 + q) * BD + lane + 32 * h] = df_from_double(x[q][h]);
    }
    __syncwarp();
    if (n > 2) fetch_d(Bd, 1, min(BW, n - 1), Ds);
    df32 v, tau, beta;
    for (int j = 0; j + 2 < n; ++j) {
        const int nsteps = (int)chase_steps(n, j);
        int p = j + 1, len = min(BW, n - p), nr = 0;
        for (int k = 0; k < nsteps; ++k) {
            if (k == 0) {
                // column j below its subdiagonal (entries (p + lane, j): k = 1 + lane)
                df32* colj = Bd + (size_t)p * BD + 1;
                df_reflector(lane < len ? colj[(size_t)lane * (BD + 1)] : df_zero(), len, slot, Vs, v, tau, beta);
                if (lane < len) colj[(size_t)lane * (BD + 1)] = (lane == 0) ? beta : df_zero();
            } else {
                // the carried block O holds rows [p + BW, ...) x cols [p, p + BW) (len == BW)
                const int pp = p;
                p = pp + BW;
                len = min(BW, n - p);  // == nr
                df_reflector(lane < len ? Os[lane * TL] : df_zero(), len, slot, Vs, v, tau, beta);
                if (lane < len) Os[lane * TL] = (lane == 0) ? beta : df_zero();
                __syncwarp();
                if (len == BW) chase_left_df<true>(len, tau, Os, Vs);
                else chase_left_df<false>(len, tau, Os, Vs);
                chase_store_df(Bd, p, pp, len, BW, Os);
            }
            slot += BW;
            // this step's block below the window into Os (free now), D (fetched ahead)
            nr = max(0, min(BW, n - p - len));
            const bool full = len == BW && nr == BW;
            fetch_o(Bd, p, len, nr, Os);
            cp_async_wait<1>();
            __syncwarp();
            if (full) chase_two_sided_df<true>(Bd, p, len, v, tau, Ds, Vs, Ws);
            else chase_two_sided_df<false>(Bd, p, len, v, tau, Ds, Vs, Ws);
            // the next step's D while this step multiplies O
            if (k + 1 < nsteps) {
                fetch_d(Bd, p + BW, min(BW, n - p - BW), Ds);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            if (full) chase_right_df<true>(len, nr, v, tau, Os, Vs, Ss);
            else chase_right_df<false>(len, nr, v, tau, Os, Vs, Ss);
        }
        chase_store_df(Bd, p + len, p, nr, len, Os);
        // the next sweep's first D (its rows are final once this sweep's stores are done)
        if (j + 3 < n) fetch_d(Bd, j + 2, min(BW, n - j - 2), Ds);
    }
    cp_async_wait<0>();
    __syncwarp();
    double* dv = arena + d.aux_off;
    double* ev = dv + ld;
    for (int t = lane; t < n; t += 32) {
        dv[t] = df_to_double(Bd[(size_t)t * BD]);
        ev[t] = (t + 1 < n) ? df_to_double(Bd[(size_t)(t + 1) * BD + 1]) : 0.0;
    }
    __syncwarp();
    if (lane == 0) tear_cluster(d, arena);
}

// one warp per cluster: a CTA per cluster, or a persistent grid on the work counter;
// DF: the double-float form (mixed path)
template <bool DF>
__global__ void __launch_bounds__(32, DF ? 12 : 1) k_chase(const ClusterDesc* __restrict__ cls, const int* __restrict__ order,
                                              double* __restrict__ arena, const int* __restrict__ status, int nitems,
                                              int* __restrict__ queue) {
    for (int it = blockIdx.x;;) {
        if (queue) {
            __syncwarp();
            int v = 0;
            if (threadIdx.x == 0) v = atomicAdd(queue, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= nitems) break;
        if constexpr (DF) chase_one_df(cls, order[it], arena, status);
        else chase_one(cls, order[it], arena, status);
        if (!queue) break;
    }
}

template <int EMU>
static dclno_status launch_band_t(dclno_ctx* c, const int* order, int nitems, int persistent) {
    const size_t smb = band_smem_bytes(EMU);
    if (smb > 227 * 1024) return set_err(c, DCLNO_ERR_ARG, "band reduction: shared memory");
    DCLNO_CUDA(c, cudaFuncSetAttribute(k_band<EMU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
    const int grid = sched_grid(c, (const void*)k_band<EMU>, DCLNO_SOLVE_THREADS, smb, nitems, persistent != 0);
    int* q = persistent ? c->d_queue : nullptr;
    if (q) DCLNO_CUDA(c, cudaMemsetAsync(q, 0, sizeof(int), c->stream));
    k_band<EMU><<<grid, DCLNO_SOLVE_THREADS, smb, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, nitems, q);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

template <bool DF>
static dclno_status launch_chase_s(dclno_ctx* c, const int* order, int nitems, int persistent) {
    static_assert(sizeof(df32) == sizeof(double), "one double-float entry takes the space of an FP64 one");
    const size_t sm2 = (DF ? CH_DF_ENTRIES : 2 * BW * TL) * sizeof(double);
    const int grid = sched_grid(c, (const void*)k_chase<DF>, 32, sm2, nitems, persistent != 0);
    int* q = persistent ? c->d_queue : nullptr;
    if (q) DCLNO_CUDA(c, cudaMemsetAsync(q, 0, sizeof(int), c->stream));
    k_chase<DF><<<grid, 32, sm2, c->stream>>>(c->d_cl, order, c->d_arena, c->d_status, nitems, q);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

// k_band then k_chase, per size bucket with the bucket's schedules (buckets without a
// two-stage cluster are skipped)
dclno_status launch_two_stage(dclno_ctx* c, const Batch& b, bool mixed, bool tune) {
    static const char* names[2] = {"k_band", "k_chase"};
    for (int kernel = TK_BAND; kernel <= TK_CHASE; ++kernel) {
        ProfScope ps__(c, names[kernel - TK_BAND]);
        std::vector<char> use(b.buckets.size(), 0);
        for (int k = 0; k < (int)b.buckets.size(); ++k) {
            const Bucket& bk = b.buckets[k];
            for (int o = bk.obeg; o < bk.oend && !use[k]; ++o) {
                const ClusterDesc& d = c->cl[c->order[o]];
                use[k] = d.q2_off >= 0 && d.split && d.n >= DCLNO_TWO_STAGE_MIN;
            }
        }
        for (const SchedRun& r : sched_runs(c, b, kernel, mixed, tune, use)) {
            const Sched s = r.s;
            cudaEvent_t e0 = nullptr;
            if (r.cand >= 0) {
                const dclno_status st = sched_time_begin(c, &e0);
                if (st != DCLNO_OK) return st;
            }
            const int* ord = c->d_order + r.obeg;
            const int ni = r.oend - r.obeg;
            dclno_status st;
            if (kernel == TK_CHASE) st = mixed ? launch_chase_s<true>(c, ord, ni, s.persistent)
                                               : launch_chase_s<false>(c, ord, ni, s.persistent);
            else if (s.engine == 2) st = launch_band_t<2>(c, ord, ni, s.persistent);
            else if (s.engine == 1) st = launch_band_t<1>(c, ord, ni, s.persistent);
            else st = launch_band_t<0>(c, ord, ni, s.persistent);
            if (st == DCLNO_OK && r.cand >= 0) st = sched_time_end(c, b, r.k0, kernel, mixed, r.cand, e0);
            if (st != DCLNO_OK) return st;
        }
    }
    return DCLNO_OK;
}
