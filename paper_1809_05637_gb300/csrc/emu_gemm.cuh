// FP64 tile update C -= A B^T computed on BF16 tensor cores (the mixed-precision
// path's contraction engine).
//
// GB300 runs FP64 at about 1.1 TFLOP/s (FMA and MMA alike) but BF16 mma.sync at
// about 600 TFLOP/s.  Each FP64 operand row is split into eight 8-bit integer
// slices relative to the row's largest exponent (x = sum_t s_t 2^(E_row - 7 - 8t),
// s_t in [-255, 255], exact in BF16).  For K <= 32 every partial sum of slice
// products of one level L = t + u (at most 8 x 32 x 255^2 < 2^24) is exact in the
// FP32 accumulator, the eight levels are combined exactly in 64-bit integers, and
// only the final conversion and update of C use FP64 (two FP64 instructions per
// element instead of K fused multiply-adds).  The result matches an FP64 dot
// product to about 2^-53 times the product of the row maxima.
#pragma once

#include <cuda_bf16.h>

#include "dclno_internal.cuh"

#define EG_M 64
#define EG_N 64
#define EG_K 32
#define EG_SL 8       // slices per operand
#define EG_LDS 40     // bf16 row stride of a slice tile (32 + 8: conflict-free fragment loads)
#define EG_SMEM_BYTES (2 * EG_SL * EG_M * EG_LDS * 2 + 2 * EG_M * 4)

__device__ __forceinline__ void mma_bf16_16816(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                               unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// unbiased exponent of |x| (0 for zero and subnormal inputs, which are flushed)
__device__ __forceinline__ int eg_exp(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    return e == 0 ? -100000 : e - 1023;
}

// Split rows [r0, r0+64) x k [k0, k0+32) of X (row-major, ld) into EG_SL slice tiles
// of bf16 in shared memory; expo[row] receives the row exponent.  Rows >= nrows and
// k >= K are zero.  A warp takes one row at a time, a lane one k: each element is
// read from global memory once and the row's exponent is a warp maximum.
__device__ __forceinline__ void eg_slice_tile(const double* __restrict__ X, int ld, int r0, int nrows, int k0,
                                              int K, __nv_bfloat16* sl, int* expo) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = DCLNO_SOLVE_THREADS / 32, PER = EG_M / NW;
    double xs[PER];  // the warp's rows, all loads issued before the slices are stored
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int gr = r0 + warp + i * NW, gk = k0 + lane;
        xs[i] = (gr < nrows && gk < K) ? X[(size_t)gr * ld + gk] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * NW;
        const double x = xs[i];
        const long long b = __double_as_longlong(x);
        const int ebits = (int)((b >> 52) & 0x7ff);
        int e = ebits == 0 ? -100000 : ebits - 1023;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0) expo[r] = e;
        unsigned long long al = 0ull;
        if (ebits != 0) {
            const unsigned long long man = ((unsigned long long)b & 0xfffffffffffffull) | 0x10000000000000ull;
            const int sh = e - (ebits - 1023);
            al = sh >= 64 ? 0ull : ((man << 11) >> sh);
        }
        const bool neg = b < 0;
#pragma unroll
        for (int t = 0; t < EG_SL; ++t) {
            const int v = (int)((al >> (56 - 8 * t)) & 0xffull);
            sl[(t * EG_M + r) * EG_LDS + lane] = __float2bfloat16_rn((float)(neg ? -v : v));
        }
    }
}

// C[M x N] -= A[M x K] B[N x K]^T with K <= 32 per call (callers pass panel widths
// of at most 32); LOWER and diag as in cta_gemm_nt_sub.  smem: EG_SMEM_BYTES.
// 256 threads; ends with __syncthreads().
template <bool LOWER>
__device__ void cta_gemm_nt_sub_emu(double* __restrict__ C, int ldc, const double* __restrict__ A, int lda,
                                    const double* __restrict__ B, int ldb, int M, int N, int K, int diag,
                                    unsigned char* smem) {
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* Bs = As + EG_SL * EG_M * EG_LDS;
    int* ea = reinterpret_cast<int*>(Bs + EG_SL * EG_M * EG_LDS);
    int* eb = ea + EG_M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wr = (warp >> 2) * 32;  // warp's rows in the tile (0, 32)
    const int wc = (warp & 3) * 16;   // warp's cols (0, 16, 32, 48)
    const int g = lane >> 2, tg = lane & 3;
    const int tilesM = (M + EG_M - 1) / EG_M, tilesN = (N + EG_N - 1) / EG_N;
    int sliced_ti = -1;  // A's slices stay in shared memory while the tile row is the same
    for (int tix = 0; tix < tilesM * tilesN; ++tix) {
        const int ti = tix / tilesN, tj = tix % tilesN;
        const int r0 = ti * EG_M, c0 = tj * EG_N;
        if (LOWER && r0 + EG_M - 1 + diag < c0) continue;  // uniform across the CTA
        if (ti != sliced_ti) {
            eg_slice_tile(A, lda, r0, M, 0, K, As, ea);
            sliced_ti = ti;
        }
        eg_slice_tile(B, ldb, c0, N, 0, K, Bs, eb);
        __syncthreads();
        // sum_L acc_L 2^-8L in units of 2^-32 (levels 5-7 lose bits below 2^-56 of the largest term)
        long long tot[2][2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) tot[i][j][v] = 0;
#pragma unroll
        for (int L = 0; L < EG_SL; ++L) {
            float acc[2][2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.f;
#pragma unroll 1
            for (int t = 0; t <= L; ++t) {
                const int u = L - t;
                const __nv_bfloat16* at = As + t * EG_M * EG_LDS;
                const __nv_bfloat16* bt = Bs + u * EG_M * EG_LDS;
#pragma unroll
                for (int ks = 0; ks < EG_K; ks += 16) {
                    unsigned af[2][4], bf[2][2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const __nv_bfloat16* p = at + (wr + 16 * i + g) * EG_LDS + ks + 2 * tg;
                        af[i][0] = *reinterpret_cast<const unsigned*>(p);
                        af[i][1] = *reinterpret_cast<const unsigned*>(p + 8 * EG_LDS);
                        af[i][2] = *reinterpret_cast<const unsigned*>(p + 8);
                        af[i][3] = *reinterpret_cast<const unsigned*>(p + 8 * EG_LDS + 8);
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const __nv_bfloat16* p = bt + (wc + 8 * j + g) * EG_LDS + ks + 2 * tg;
                        bf[j][0] = *reinterpret_cast<const unsigned*>(p);
                        bf[j][1] = *reinterpret_cast<const unsigned*>(p + 8);
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < 2; ++j)
                            mma_bf16_16816(acc[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bf[j][0], bf[j][1]);
                }
            }
            // integer combination of the level (exact for L <= 4)
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const long long a = (long long)__float2int_rn(acc[i][j][v]);
                        tot[i][j][v] += (L <= 4) ? (a << (32 - 8 * L)) : (a >> (8 * L - 32));
                    }
        }
        // value = 2^(ea+eb-46) tot; tot >> 3 fits the 53-bit mantissa (units of 2^(ea+eb-43));
        // C's elements are all loaded before any is stored
        double cv[2][2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = r0 + wr + 16 * i + g + (v >= 2 ? 8 : 0);
                    const int cc = c0 + wc + 8 * j + 2 * tg + (v & 1);
                    cv[i][j][v] = (r < M && cc < N && !(LOWER && r + diag < cc)) ? C[(size_t)r * ldc + cc] : 0.0;
                }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int rl = wr + 16 * i + g + (v >= 2 ? 8 : 0);
                    const int cl = wc + 8 * j + 2 * tg + (v & 1);
                    const int r = r0 + rl, cc = c0 + cl;
                    if (r >= M || cc >= N) continue;
                    if (LOWER && r + diag < cc) continue;
                    const int es = ea[rl] + eb[cl] - 43 + 1023;
                    if (es < 1 || es > 2046) continue;  // a zero row or column (or far outside range)
                    const long long q = tot[i][j][v] >> 3;
                    C[(size_t)r * ldc + cc] = fma(-(double)q, __longlong_as_double((long long)es << 52), cv[i][j][v]);
                }
        __syncthreads();
    }
}

#include "emu_tc.cuh"

// The cubic steps' tile update, by engine: EMU = 0 FP64 mma.sync tiles (FP64 path);
// EMU = 1 FP64 emulated by BF16 slices on mma.sync (register fragments); EMU = 2 the
// same emulation on tcgen05.mma with tensor-memory accumulators (tc: the CTA's state,
// set up by tc_begin).  The emulated engines take K <= 32 per call.
template <bool LOWER, int EMU>
__device__ __forceinline__ void tile_update(double* C, int ldc, const double* A, int lda, const double* B, int ldb,
                                            int M, int N, int K, int diag, double* smem, TcState* tc) {
    if constexpr (EMU == 2)
        cta_gemm_nt_sub_tc<LOWER>(C, ldc, A, lda, B, ldb, M, N, K, diag, reinterpret_cast<unsigned char*>(smem), tc);
    else if constexpr (EMU == 1)
        cta_gemm_nt_sub_emu<LOWER>(C, ldc, A, lda, B, ldb, M, N, K, diag, reinterpret_cast<unsigned char*>(smem));
    else
        cta_gemm_nt_sub<LOWER>(C, ldc, A, lda, B, ldb, M, N, K, diag, smem);
}

// C -= A B^T for any K: FP64 tiles take K whole, the emulated engines chunks of 32
// (each chunk sliced against its own row exponents and added to C in FP64).
template <int EMU>
__device__ __forceinline__ void tile_update_longk(double* C, int ldc, const double* A, int lda, const double* B,
                                                  int ldb, int M, int N, int K, double* smem, TcState* tc) {
    if constexpr (EMU == 0) {
        cta_gemm_nt_sub<false>(C, ldc, A, lda, B, ldb, M, N, K, 0, smem);
    } else {
        for (int k0 = 0; k0 < K; k0 += EG_K)
            tile_update<false, EMU>(C, ldc, A + k0, lda, B + k0, ldb, M, N, min(EG_K, K - k0), 0, smem, tc);
    }
}

// shared memory of one engine's staging (bytes)
#define ENGINE_SMEM_BYTES(EMU) ((EMU) == 2 ? TC_SMEM_BYTES : (EMU) == 1 ? EG_SMEM_BYTES : GT_SMEM_DOUBLES * 8)

// Tensor memory and barriers of an EMU == 2 kernel's CTA: tc_begin after the early
// exits, tc_end before every later exit (it waits out a timed-out engine's MMAs).
#define ENGINE_BEGIN(EMU, st) \
    do {                      \
        if ((EMU) == 2) tc_begin(st); \
    } while (0)
#define ENGINE_END(EMU, st) \
    do {                    \
        if ((EMU) == 2) tc_end(st); \
    } while (0)

// CTA-wide sum (every thread gets the result); red holds one double per warp.
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

// CTAs per SM the cubic kernels are compiled for: the FP64 tiles gain from a third
// CTA (latency hiding), the emulated ones lose by it (their slicing needs registers);
// measured on the 1728-atom step.
#define DCLNO_CTAS_PER_SM(EMU) ((EMU) ? 2 : 3)

// Work distribution of the cubic kernels.  With queue == nullptr the grid has one CTA
// per cluster (CTA b takes cluster order[b]); otherwise the grid is persistent and every
// CTA takes the next cluster from the atomic counter *queue until nitems are taken (no CTA
// waits on another).  A CTA's tensor memory (EMU == 2) is set up once for all its clusters.
#define CUBIC_KERNEL_LOOP(EMU, call)                                   \
    __shared__ TcState tcs;                                            \
    __shared__ int s_item;                                             \
    ENGINE_BEGIN(EMU, &tcs);                                           \
    for (int it = blockIdx.x;;) {                                      \
        if (queue) {                                                   \
            __syncthreads();                                           \
            if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);        \
            __syncthreads();                                           \
            it = s_item;                                               \
        }                                                              \
        if (it >= nitems) break;                                       \
        call;                                                          \
        if (!queue) break;                                             \
    }                                                                  \
    ENGINE_END(EMU, &tcs);
