// Ogita-Aishima refinement of batched generalised eigendecompositions H X = S X Lambda
// (Ogita & Aishima, Japan J. Indust. Appl. Math. 35 (2018), carried over to the S
// metric).  Not a step of the paper: the FP64-residual refinement a mixed-precision
// eigensolver would apply to approximate eigenpairs.  One sweep, for each pencil of
// the batch (dimension n, all FP64, row-major n x n):
//   R = I - X^T S X,   G = X^T H X,   lam_i = G_ii / (1 - R_ii),
//   delta = 2 (||G - diag(lam)||_F + max_i |lam_i| ||R||_F),
//   E_ij = (G_ij + lam_j R_ij) / (lam_j - lam_i)  where i != j and |lam_j - lam_i| > delta,
//   E_ij = R_ij / 2                                 otherwise,
//   X <- X + X E.
// Five n x n x n products per sweep (10 n^3 flops) in k_refine_gemm: 32 x 32 output
// tiles, 32-wide K chunks of both operands staged in shared memory (a transposed
// operand is read along its rows, so every global load is coalesced), FP64 fused
// multiply-adds in a fixed K order; then a CTA per pencil for lam and delta (fixed-order
// block reductions) and an elementwise pass for E.
#include <algorithm>

#include "dclno_internal.cuh"

#define RF_T 32        // output tile edge and K chunk
#define RF_THREADS 256  // 8 warps: warp w owns tile rows w, w + 8, w + 16, w + 24

enum { RF_NN = 0, RF_RESIDUAL = 1, RF_TN = 2, RF_UPDATE = 3 };

// C = op(A) B for one 32 x 32 tile of pencil blockIdx.z, with
//   RF_NN        op(A) = A,    C = A B
//   RF_RESIDUAL  op(A) = A^T,  C = I - A^T B
//   RF_TN        op(A) = A^T,  C = A^T B
//   RF_UPDATE    op(A) = A,    C = Base + A B
// C must not overlap A, B or Base.
template <int MODE>
__global__ void __launch_bounds__(RF_THREADS) k_refine_gemm(int n, const double* __restrict__ A,
                                                             const double* __restrict__ B,
                                                             const double* __restrict__ Base,
                                                             double* __restrict__ C) {
    __shared__ double As[RF_T][RF_T + 1];  // As[r][k] = op(A)[row0 + r][k0 + k]
    __shared__ double Bs[RF_T][RF_T + 1];  // Bs[k][c] = B[k0 + k][col0 + c]
    const size_t off = (size_t)blockIdx.z * n * n;
    A += off;
    B += off;
    C += off;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int row0 = blockIdx.y * RF_T, col0 = blockIdx.x * RF_T;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += RF_T) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = ty + 8 * q;
            if (MODE == RF_RESIDUAL || MODE == RF_TN) {
                // op(A)[row0 + tx][k0 + t] = A[k0 + t][row0 + tx]: lanes read along row k0 + t of A
                const int k = k0 + t, r = row0 + tx;
                As[tx][t] = (k < n && r < n) ? A[(size_t)k * n + r] : 0.0;
            } else {
                const int r = row0 + t, k = k0 + tx;
                As[t][tx] = (r < n && k < n) ? A[(size_t)r * n + k] : 0.0;
            }
            const int k = k0 + t, c = col0 + tx;
            Bs[t][tx] = (k < n && c < n) ? B[(size_t)k * n + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < RF_T; ++k) {
            const double b = Bs[k][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][k], b, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = row0 + ty + 8 * q, c = col0 + tx;
        if (r >= n || c >= n) continue;
        const size_t ix = (size_t)r * n + c;
        if (MODE == RF_RESIDUAL)
            C[ix] = (r == c ? 1.0 : 0.0) - acc[q];
        else if (MODE == RF_UPDATE)
            C[ix] = Base[off + ix] + acc[q];
        else
            C[ix] = acc[q];
    }
}

// one CTA per pencil: lam_i = G_ii / (1 - R_ii) and delta = 2 (||G - diag(lam)||_F +
// max |lam| ||R||_F); every thread sums a fixed stride of entries, then a fixed-order tree
__global__ void __launch_bounds__(RF_THREADS) k_refine_lam(int n, const double* __restrict__ G,
                                                           const double* __restrict__ R, double* __restrict__ lam,
                                                           double* __restrict__ delta) {
    const int p = blockIdx.x, t = threadIdx.x;
    const size_t off = (size_t)p * n * n;
    double sg = 0.0, sr = 0.0, mx = 0.0;
    for (int i = t; i < n; i += RF_THREADS) {
        const double gii = G[off + (size_t)i * n + i];
        const double li = gii / (1.0 - R[off + (size_t)i * n + i]);
        lam[(size_t)p * n + i] = li;
        mx = fmax(mx, fabs(li));
        sg = fma(gii - li, gii - li, sg);
    }
    const long long nn = (long long)n * n;
    for (long long idx = t; idx < nn; idx += RF_THREADS) {
        const double r = R[off + idx];
        sr = fma(r, r, sr);
        if (idx / n != idx % n) {
            const double g = G[off + idx];
            sg = fma(g, g, sg);
        }
    }
    __shared__ double s_g[RF_THREADS], s_r[RF_THREADS], s_m[RF_THREADS];
    s_g[t] = sg;
    s_r[t] = sr;
    s_m[t] = mx;
    __syncthreads();
    for (int h = RF_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) {
            s_g[t] += s_g[t + h];
            s_r[t] += s_r[t + h];
            s_m[t] = fmax(s_m[t], s_m[t + h]);
        }
        __syncthreads();
    }
    if (t == 0) delta[p] = 2.0 * (sqrt(s_g[0]) + s_m[0] * sqrt(s_r[0]));
}

// E over every entry of every pencil, written over G
__global__ void k_refine_e(int n, long long total, double* __restrict__ G, const double* __restrict__ R,
                           const double* __restrict__ lam, const double* __restrict__ delta) {
    const long long nn = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long p = idx / nn, rem = idx - p * nn;
        const int i = (int)(rem / n), j = (int)(rem - (long long)i * n);
        const double r = R[idx];
        double e = 0.5 * r;
        if (i != j) {
            const double li = lam[p * n + i], lj = lam[p * n + j];
            const double gap = lj - li;
            if (fabs(gap) > delta[p]) e = (G[idx] + lj * r) / gap;
        }
        G[idx] = e;
    }
}

extern "C" dclno_status dclno_refine_eigenpairs(const double* H, const double* S, double* X, double* lam_out,
                                                int n, int count, int nsweeps, void* cuda_stream) {
    if (!H || !S || !X || !lam_out || n < 1 || count < 1 || nsweeps < 1) return DCLNO_ERR_ARG;
    const int tiles = (n + RF_T - 1) / RF_T;
    if (tiles > 65535 || count > 65535) return DCLNO_ERR_ARG;  // grid limits of the tile launches
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t nn = (size_t)n * n, total = nn * (size_t)count;
    double* ws = nullptr;
    // W (products, then the updated X), R, G (then E), delta
    if (cudaMalloc(&ws, (3 * total + (size_t)count) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();  // clear the allocation error so it does not surface in a later call
        return DCLNO_ERR_OOM;
    }
    double *W = ws, *R = ws + total, *G = ws + 2 * total, *delta = ws + 3 * total;
    const dim3 grid(tiles, tiles, count);
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    const long long eblocks = std::min<long long>(((long long)total + 255) / 256, (long long)sms * 16);
    cudaError_t err = cudaSuccess;
    for (int s = 0; s < nsweeps && err == cudaSuccess; ++s) {
        k_refine_gemm<RF_NN><<<grid, RF_THREADS, 0, st>>>(n, S, X, nullptr, W);             // W = S X
        k_refine_gemm<RF_RESIDUAL><<<grid, RF_THREADS, 0, st>>>(n, X, W, nullptr, R);       // R = I - X^T S X
        k_refine_gemm<RF_NN><<<grid, RF_THREADS, 0, st>>>(n, H, X, nullptr, W);             // W = H X
        k_refine_gemm<RF_TN><<<grid, RF_THREADS, 0, st>>>(n, X, W, nullptr, G);             // G = X^T H X
        k_refine_lam<<<count, RF_THREADS, 0, st>>>(n, G, R, lam_out, delta);
        k_refine_e<<<(unsigned)std::max<long long>(eblocks, 1), 256, 0, st>>>(n, (long long)total, G, R, lam_out, delta);
        k_refine_gemm<RF_UPDATE><<<grid, RF_THREADS, 0, st>>>(n, X, G, X, W);               // W = X + X E
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaMemcpyAsync(X, W, total * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaFree(ws);
    return err == cudaSuccess ? DCLNO_OK : DCLNO_ERR_CUDA;
}
