// FP64 tile update C -= A B^T emulated on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory) -- the same arithmetic as
// cta_gemm_nt_sub_emu (emu_gemm.cuh): every FP64 row split into eight 8-bit slices
// relative to the row's largest exponent, the products of one level L = t + u summed
// exactly in FP32 (K <= 32), the levels combined exactly in 64-bit integers, two FP64
// instructions per output element.
//
// Tile 128 x 32 outputs, K <= 32 per call.  The slices sit in shared memory in the
// K-major core-matrix layout of the MMA (8 rows x 16 bytes per core matrix; core
// matrices 128 bytes apart along K, 512 bytes apart along M/N).  One thread issues the
// MMAs of all eight levels at once (level L: (L+1) x 2 MMAs of M = 128, N = 32, K = 16
// into its own 32 tensor-memory columns, 256 columns in all) behind one commit; after
// one wait every warp reads the eight levels of its 32 rows x 16 columns back
// (tcgen05.ld) and adds them into its integer totals.  One round trip per tile (or per
// K-chunk of the long-K product) instead of one per level.
//
// Waits on the mbarriers are bounded: on expiry the CTA's status word is set and the
// update is abandoned (its result is then garbage, the caller reports the status).
#pragma once

#include <cuda_bf16.h>

#include "dclno_internal.cuh"

#define TC_M 128
#define TC_N 32
#define TC_K 32
#define TC_SL 8
#define TC_A_SLICE_BYTES (TC_M * TC_K * 2)  // 8192
#define TC_B_SLICE_BYTES (TC_N * TC_K * 2)  // 2048
#define TC_B_REGION (TC_M * TC_N * 8)       // B slices (16 KB), or a tile of totals as doubles (32 KB)
#define TC_LBO 128                          // core matrices along K
#define TC_SBO 512                          // 8-row groups along M / N
#define TC_TMEM_COLS 256                    // eight level accumulators of TC_N columns
#define TC_SMEM_BYTES (TC_SL * TC_A_SLICE_BYTES + TC_B_REGION + (TC_M + TC_N) * 4 + 64)
// at most two such CTAs fit an SM's 228 KB of shared memory, so their tensor memory
// (2 x 256 of the SM's 512 columns) is always available to both
static_assert(3 * (TC_SMEM_BYTES + 1024) > 228 * 1024 && 2 * TC_TMEM_COLS <= 512, "tensor-memory budget");
#define TC_WAIT_LIMIT 4000000

// per-CTA state of the engine (in shared memory)
struct TcState {
    uint64_t mbar[2];    // level buffers' completion barriers
    uint32_t tmem;       // tensor-memory base address (TC_TMEM_COLS columns)
    uint32_t uses[2];    // completions of each buffer's barrier consumed so far (phase parity)
    uint32_t issued[2];  // commits issued to each buffer's barrier
    int failed;          // a bounded wait ran out
};

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Allocate the CTA's tensor memory and initialise the barriers (all threads call it).
__device__ __forceinline__ void tc_begin(TcState* st) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(&st->tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(&st->mbar[b])), "r"(1));
            st->uses[b] = 0;
            st->issued[b] = 0;
        }
        st->failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

// bounded wait for completion number `use` of a buffer's barrier (parity use & 1)
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t use) {
    const uint32_t a = tc_smem_u32(mbar);
    for (int it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p;}"
            : "=r"(done)
            : "r"(a), "r"(use & 1));
        if (done) return true;
    }
    return false;
}

// Free the tensor memory (all threads call it).  After a timed-out wait, the MMAs still
// in flight are first waited for (again bounded) so that none writes freed columns.
__device__ __forceinline__ void tc_end(TcState* st) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0 && st->failed)
        for (int b = 0; b < 2; ++b)
            while (st->uses[b] < st->issued[b] && tc_wait(&st->mbar[b], st->uses[b])) st->uses[b] += 1;
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st->tmem), "r"(TC_TMEM_COLS));
}

// Slices of rows [r0, r0 + rows_tile) x k [0, 32) of X (row-major, ld) into TC_SL slice
// tiles in the MMA layout (bf16 element (r, k) at (r/8) SBO + (k/8) LBO + (r%8) 16 + (k%8) 2
// bytes); expo[r] = the row's exponent.  Rows >= nrows and k >= K are zero.
template <int ROWS>
__device__ __forceinline__ void tc_slice_tile(const double* __restrict__ X, int ld, int r0, int nrows, int K,
                                              unsigned char* sl, int slice_bytes, int* expo) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kofs = (lane >> 3) * TC_LBO + (lane & 7) * 2;
    constexpr int NW = DCLNO_SOLVE_THREADS / 32, PER = (ROWS + NW - 1) / NW;
    double xs[PER];  // the warp's rows, all loads issued before the slices are stored
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * NW, gr = r0 + r;
        xs[i] = (r < ROWS && gr < nrows && lane < K) ? X[(size_t)gr * ld + lane] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * NW;
        if (r >= ROWS) break;
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
        unsigned char* dst = sl + (r >> 3) * TC_SBO + (r & 7) * 16 + kofs;
#pragma unroll
        for (int t = 0; t < TC_SL; ++t) {
            const int v = (int)((al >> (56 - 8 * t)) & 0xffull);
            *reinterpret_cast<__nv_bfloat16*>(dst + t * slice_bytes) = __float2bfloat16_rn((float)(neg ? -v : v));
        }
    }
}

// issue the MMAs of all levels (level L into tensor-memory columns [32 L, 32 L + 32))
// and commit them to barrier 0 (one thread)
__device__ __forceinline__ void tc_issue_levels(TcState* st, const unsigned char* As, const unsigned char* Bs) {
    const uint32_t id = tc_idesc(TC_M, TC_N);
    const uint32_t a0 = tc_smem_u32(As), b0 = tc_smem_u32(Bs);
#pragma unroll 1
    for (int L = 0; L < TC_SL; ++L) {
        const uint32_t d = st->tmem + (uint32_t)(L * TC_N);
        for (int t = 0; t <= L; ++t) {
            const int u = L - t;
#pragma unroll
            for (int ks = 0; ks < TC_K / 16; ++ks) {
                const uint64_t ad = tc_desc(a0 + t * TC_A_SLICE_BYTES + ks * 2 * TC_LBO);
                const uint64_t bd = tc_desc(b0 + u * TC_B_SLICE_BYTES + ks * 2 * TC_LBO);
                asm volatile(
                    "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}\n" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(id), "r"((t == 0 && ks == 0) ? 0 : 1));
            }
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        tc_smem_u32(&st->mbar[0])));
    st->issued[0] += 1;
}

// Issue all levels of the staged slices, wait, and add the levels of this warp's 32 rows
// (lane quarter q) x 16 columns (half h) into tot (all threads call it; it ends with a
// barrier after which the tensor memory may be reissued).  False once a wait ran out.
__device__ __forceinline__ bool tc_run_levels(TcState* st, const unsigned char* As, const unsigned char* Bs, int q,
                                              int h, long long* tot) {
    asm volatile("fence.proxy.async.shared::cta;");  // the slices, visible to the tensor cores
    __syncthreads();
    if (threadIdx.x == 0 && !st->failed) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        tc_issue_levels(st, As, Bs);
    }
    __syncthreads();
    bool ok = !st->failed && tc_wait(&st->mbar[0], st->uses[0]);
    if (!ok) st->failed = 1;  // any thread that gave up marks the CTA
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
#pragma unroll 1
        for (int L = 0; L < TC_SL; ++L) {
            uint32_t r[16];
            const uint32_t ta = st->tmem + (uint32_t)(L * TC_N + 16 * h) + ((uint32_t)(32 * q) << 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                " [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const long long v = (long long)__float2int_rn(__uint_as_float(r[j]));
                tot[j] += (L <= 4) ? (v << (32 - 8 * L)) : (v >> (8 * L - 32));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // every warp has read the accumulators
    if (threadIdx.x == 0 && !st->failed) st->uses[0] += 1;  // else tc_end waits this commit out
    __syncthreads();
    return !st->failed;
}

// C[M x N] -= A[M x K] B[N x K]^T, K <= 32; LOWER and diag as in cta_gemm_nt_sub.
// 256 threads; smem: TC_SMEM_BYTES (st lives elsewhere); ends with __syncthreads().
template <bool LOWER>
__device__ void cta_gemm_nt_sub_tc(double* __restrict__ C, int ldc, const double* __restrict__ A, int lda,
                                   const double* __restrict__ B, int ldb, int M, int N, int K, int diag,
                                   unsigned char* smem, TcState* st) {
    unsigned char* As = smem;
    unsigned char* Bs = As + TC_SL * TC_A_SLICE_BYTES;
    int* ea = reinterpret_cast<int*>(Bs + TC_B_REGION);
    int* eb = ea + TC_M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter (rows 32 q ..) and column half
    const int tilesM = (M + TC_M - 1) / TC_M, tilesN = (N + TC_N - 1) / TC_N;
    int sliced_ti = -1;
    for (int tix = 0; tix < tilesM * tilesN; ++tix) {
        const int ti = tix / tilesN, tj = tix % tilesN;
        const int r0 = ti * TC_M, c0 = tj * TC_N;
        if (LOWER && r0 + TC_M - 1 + diag < c0) continue;  // uniform across the CTA
        if (st->failed) break;
        if (ti != sliced_ti) {
            tc_slice_tile<TC_M>(A, lda, r0, M, K, As, TC_A_SLICE_BYTES, ea);
            sliced_ti = ti;
        }
        tc_slice_tile<TC_N>(B, ldb, c0, N, K, Bs, TC_B_SLICE_BYTES, eb);
        long long tot[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) tot[j] = 0;
        if (!tc_run_levels(st, As, Bs, q, h, tot)) break;
        // value = 2^(ea+eb-46) tot; tot >> 3 fits the 53-bit mantissa (units of 2^(ea+eb-43)).
        // The integer totals pass through shared memory (the B slices' region, columns
        // XOR-swizzled by the row) so that C is updated row-contiguously.
        {
            const int rl = 32 * q + lane;
            double* Vs = reinterpret_cast<double*>(Bs);  // TC_M x TC_N
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int cl = 16 * h + j;
                Vs[rl * TC_N + (cl ^ (rl & 15))] = (double)(tot[j] >> 3);
            }
            __syncthreads();
            constexpr int NW = DCLNO_SOLVE_THREADS / 32, PER = TC_M / NW;
            double cv[PER];  // C's elements of the warp's rows, loaded before any is stored
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int r = r0 + warp + i * NW, cc = c0 + lane;
                cv[i] = (r < M && cc < N && !(LOWER && r + diag < cc)) ? C[(size_t)r * ldc + cc] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int rr = warp + i * NW, r = r0 + rr, cl = lane, cc = c0 + cl;
                if (r >= M || cc >= N) continue;
                if (LOWER && r + diag < cc) continue;
                const int es = ea[rr] + eb[cl] - 43 + 1023;
                if (es < 1 || es > 2046) continue;  // a zero row or column (or far outside range)
                C[(size_t)r * ldc + cc] =
                    fma(-Vs[rr * TC_N + (cl ^ (rr & 15))], __longlong_as_double((long long)es << 52), cv[i]);
            }
        }
        __syncthreads();  // the B region may be overwritten by the next tile
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Long-K products with one FP64 epilogue: C[M x N] -= A[M x K] B[N x K]^T for any K,
// N <= 32 per tile column (tiles of 128 x 32).  Row exponents are taken over all of K
// (a first pass over the tile's rows), every K-chunk of 32 is sliced against them, and
// the integer totals of all chunks are kept in registers (|total| < 2^54 per chunk, so
// up to 500 chunks fit 64 bits); each output then costs two FP64 instructions in all,
// instead of two per chunk.  TRANS writes element (r, c) to C[c * ldc + r]; LOWER
// (without TRANS) updates only the lower triangle r >= c of C.
// smem: TC_SMEM_BYTES; tensor memory: the CTA's allocation (eight level accumulators).
// ---------------------------------------------------------------------------
#define TCL_N TC_N
#define TCL_B_SLICE_BYTES TC_B_SLICE_BYTES

// largest exponent of rows [r0, r0 + rows) of X over k < K (warp per row)
__device__ __forceinline__ void tcl_row_expo(const double* __restrict__ X, int ld, int r0, int rows, int nrows, int K,
                                             int* expo) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < rows; r += nw) {
        const int gr = r0 + r;
        int e = -100000;
        if (gr < nrows)
            for (int k = lane; k < K; k += 32) {
                const int eb = (int)((__double_as_longlong(X[(size_t)gr * ld + k]) >> 52) & 0x7ff);
                if (eb != 0) e = max(e, eb - 1023);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0) expo[r] = e;
    }
}

// rows [r0, r0 + ROWS) x k [k0, k0 + 32) of X into registers (a warp per row, a lane per
// k; warp w holds rows w, w + 8, ..)
template <int ROWS>
__device__ __forceinline__ void tcl_load_chunk(const double* __restrict__ X, int ld, int r0, int nrows, int k0, int K,
                                               double* x) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = DCLNO_SOLVE_THREADS / 32, PER = (ROWS + NW - 1) / NW;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * NW, gr = r0 + r, gk = k0 + lane;
        x[i] = (r < ROWS && gr < nrows && gk < K) ? X[(size_t)gr * ld + gk] : 0.0;
    }
}

// the loaded chunk's slices against the fixed row exponents expo[]
template <int ROWS>
__device__ __forceinline__ void tcl_store_chunk(const double* x, const int* expo, unsigned char* sl, int slice_bytes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = DCLNO_SOLVE_THREADS / 32, PER = (ROWS + NW - 1) / NW;
    const int kofs = (lane >> 3) * TC_LBO + (lane & 7) * 2;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * NW;
        if (r >= ROWS) break;
        const long long b = __double_as_longlong(x[i]);
        const int ebits = (int)((b >> 52) & 0x7ff);
        unsigned long long al = 0ull;
        if (ebits != 0) {
            const unsigned long long man = ((unsigned long long)b & 0xfffffffffffffull) | 0x10000000000000ull;
            const int sh = expo[r] - (ebits - 1023);
            al = sh >= 64 ? 0ull : ((man << 11) >> sh);
        }
        const bool neg = b < 0;
        unsigned char* dst = sl + (r >> 3) * TC_SBO + (r & 7) * 16 + kofs;
#pragma unroll
        for (int t = 0; t < TC_SL; ++t) {
            const int v = (int)((al >> (56 - 8 * t)) & 0xffull);
            *reinterpret_cast<__nv_bfloat16*>(dst + t * slice_bytes) = __float2bfloat16_rn((float)(neg ? -v : v));
        }
    }
}

template <bool TRANS, bool LOWER = false>
__device__ void cta_gemm_tc_longk(double* __restrict__ C, int ldc, const double* __restrict__ A, int lda,
                                  const double* __restrict__ B, int ldb, int M, int N, int K, unsigned char* smem,
                                  TcState* st) {
    unsigned char* As = smem;
    unsigned char* Bs = As + TC_SL * TC_A_SLICE_BYTES;
    int* ea = reinterpret_cast<int*>(Bs + TC_SL * TCL_B_SLICE_BYTES);
    int* eb = ea + TC_M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, h = warp >> 2;  // rows 32 q .., columns 16 h ..
    const int tilesM = (M + TC_M - 1) / TC_M, tilesN = (N + TCL_N - 1) / TCL_N;
    for (int tix = 0; tix < tilesM * tilesN; ++tix) {
        if (st->failed) break;
        const int ti = tix / tilesN, tj = tix % tilesN;
        const int r0 = ti * TC_M, c0 = tj * TCL_N;
        if (LOWER && r0 + TC_M - 1 < c0) continue;  // uniform across the CTA
        tcl_row_expo(A, lda, r0, TC_M, M, K, ea);
        tcl_row_expo(B, ldb, c0, TCL_N, N, K, eb);
        __syncthreads();
        long long tot[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) tot[j] = 0;
        bool ok = true;
        // the next chunk's loads are in flight while the tensor cores work on this one
        double xa[TC_M / 8], xb[TCL_N / 8];
        tcl_load_chunk<TC_M>(A, lda, r0, M, 0, K, xa);
        tcl_load_chunk<TCL_N>(B, ldb, c0, N, 0, K, xb);
        for (int k0 = 0; k0 < K && ok; k0 += TC_K) {
            tcl_store_chunk<TC_M>(xa, ea, As, TC_A_SLICE_BYTES);
            tcl_store_chunk<TCL_N>(xb, eb, Bs, TCL_B_SLICE_BYTES);
            if (k0 + TC_K < K) {
                tcl_load_chunk<TC_M>(A, lda, r0, M, k0 + TC_K, K, xa);
                tcl_load_chunk<TCL_N>(B, ldb, c0, N, k0 + TC_K, K, xb);
            }
            ok = tc_run_levels(st, As, Bs, q, h, tot);
        }
        if (!ok) break;
        // one epilogue: (tot >> 3) 2^(ea + eb - 43), staged through shared memory (the A
        // slices) for row-contiguous (or, with TRANS, column-contiguous) updates of C
        double* Vs = reinterpret_cast<double*>(As);  // TC_M x TCL_N, columns XOR-swizzled by the row
        {
            const int rl = 32 * q + lane;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int cl = 16 * h + j;
                Vs[rl * TCL_N + (cl ^ (rl & 15))] = (double)(tot[j] >> 3);
            }
        }
        __syncthreads();
        // C's elements are all loaded before any is stored (the loads overlap)
        constexpr int NW = DCLNO_SOLVE_THREADS / 32, PER = TC_M * TCL_N / DCLNO_SOLVE_THREADS;
        double cv[PER];
        if (!TRANS) {  // warp per row, lane per column
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int r = r0 + warp + i * NW, cc = c0 + lane;
                cv[i] = (r < M && cc < N && !(LOWER && r < cc)) ? C[(size_t)r * ldc + cc] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int rr = warp + i * NW, r = r0 + rr, cl = lane, cc = c0 + cl;
                if (r >= M || cc >= N || (LOWER && r < cc)) continue;
                const int es = ea[rr] + eb[cl] - 43 + 1023;
                if (es < 1 || es > 2046) continue;
                C[(size_t)r * ldc + cc] =
                    fma(-Vs[rr * TCL_N + (cl ^ (rr & 15))], __longlong_as_double((long long)es << 52), cv[i]);
            }
        } else {  // thread per row of a column
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int idx = tid + i * DCLNO_SOLVE_THREADS, cl = idx / TC_M, rr = idx % TC_M;
                const int r = r0 + rr, cc = c0 + cl;
                cv[i] = (r < M && cc < N) ? C[(size_t)cc * ldc + r] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int idx = tid + i * DCLNO_SOLVE_THREADS, cl = idx / TC_M, rr = idx % TC_M;
                const int r = r0 + rr, cc = c0 + cl;
                if (r >= M || cc >= N) continue;
                const int es = ea[rr] + eb[cl] - 43 + 1023;
                if (es < 1 || es > 2046) continue;
                C[(size_t)cc * ldc + r] =
                    fma(-Vs[rr * TCL_N + (cl ^ (rr & 15))], __longlong_as_double((long long)es << 52), cv[i]);
            }
        }
        __syncthreads();
    }
    __syncthreads();
}
