// FP64 tile update C -= A B^T emulated on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory) -- the same arithmetic as
// cta_gemm_nt_sub_emu (emu_gemm.cuh): every FP64 row split into eight 8-bit slices
// relative to the row's largest exponent, the products of one level L = t + u summed
// exactly in FP32 (K <= 32), the levels combined exactly in 64-bit integers, two FP64
// instructions per output element.
//
// Tile 128 x 64 outputs, K <= 32 per call.  The slices sit in shared memory in the
// K-major core-matrix layout of the MMA (8 rows x 16 bytes per core matrix; core
// matrices 128 bytes apart along K, 512 bytes apart along M/N).  One thread issues
// the level's (L+1) x 2 MMAs (M = 128, N = 64, K = 16) into one of two tensor-memory
// buffers of 64 FP32 columns and commits them to that buffer's mbarrier; all eight
// warps then read the level back (warp w: lanes 32 (w mod 4) .. + 31 = tile rows,
// columns 32 (w / 4) .. + 31) and add it into their integer totals, while the
// tensor cores already work on level L + 1.  A buffer is reissued (level L + 2)
// only after every warp has read it.
//
// Waits on the mbarriers are bounded: on expiry the CTA's status word is set and the
// update is abandoned (its result is then garbage, the caller reports the status).
#pragma once

#include <cuda_bf16.h>

#include "dclno_internal.cuh"

#define TC_M 128
#define TC_N 64
#define TC_K 32
#define TC_SL 8
#define TC_A_SLICE_BYTES (TC_M * TC_K * 2)  // 8192
#define TC_B_SLICE_BYTES (TC_N * TC_K * 2)  // 4096
#define TC_LBO 128                          // core matrices along K
#define TC_SBO 512                          // 8-row groups along M / N
#define TC_TMEM_COLS 128                    // two level buffers of TC_N columns
#define TC_SMEM_BYTES (TC_SL * (TC_A_SLICE_BYTES + TC_B_SLICE_BYTES) + (TC_M + TC_N) * 4 + 64)
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kofs = (lane >> 3) * TC_LBO + (lane & 7) * 2;
    for (int r = warp; r < ROWS; r += nw) {
        const int gr = r0 + r;
        const double x = (gr < nrows && lane < K) ? X[(size_t)gr * ld + lane] : 0.0;
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

// issue the MMAs of level L into buffer buf (one thread)
__device__ __forceinline__ void tc_issue_level(TcState* st, const unsigned char* As, const unsigned char* Bs, int L,
                                               int buf) {
    const uint32_t d = st->tmem + (uint32_t)(buf * TC_N);
    const uint32_t id = tc_idesc(TC_M, TC_N);
    const uint32_t a0 = tc_smem_u32(As), b0 = tc_smem_u32(Bs);
    int first = 1;
    for (int t = 0; t <= L; ++t) {
        const int u = L - t;
#pragma unroll
        for (int ks = 0; ks < TC_K / 16; ++ks) {
            const uint64_t ad = tc_desc(a0 + t * TC_A_SLICE_BYTES + ks * 2 * TC_LBO);
            const uint64_t bd = tc_desc(b0 + u * TC_B_SLICE_BYTES + ks * 2 * TC_LBO);
            asm volatile(
                "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(id), "r"(first ? 0 : 1));
            first = 0;
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        tc_smem_u32(&st->mbar[buf])));
    st->issued[buf] += 1;
}

// C[M x N] -= A[M x K] B[N x K]^T, K <= 32; LOWER and diag as in cta_gemm_nt_sub.
// 256 threads; smem: TC_SMEM_BYTES (st lives elsewhere); ends with __syncthreads().
template <bool LOWER>
__device__ void cta_gemm_nt_sub_tc(double* __restrict__ C, int ldc, const double* __restrict__ A, int lda,
                                   const double* __restrict__ B, int ldb, int M, int N, int K, int diag,
                                   unsigned char* smem, TcState* st) {
    unsigned char* As = smem;
    unsigned char* Bs = As + TC_SL * TC_A_SLICE_BYTES;
    int* ea = reinterpret_cast<int*>(Bs + TC_SL * TC_B_SLICE_BYTES);
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
        asm volatile("fence.proxy.async.shared::cta;");  // the slices, visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            tc_issue_level(st, As, Bs, 0, 0);
            tc_issue_level(st, As, Bs, 1, 1);
        }
        long long tot[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) tot[j] = 0;
        bool ok = true;
        for (int L = 0; L < TC_SL; ++L) {
            const int buf = L & 1;
            ok = ok && tc_wait(&st->mbar[buf], st->uses[buf]);
            if (!ok) st->failed = 1;  // any thread that gave up marks the CTA
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t r[32];
            if (ok) {
                const uint32_t ta = st->tmem + (uint32_t)(buf * TC_N + 32 * h) + ((uint32_t)(32 * q) << 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const long long a = (long long)__float2int_rn(__uint_as_float(r[j]));
                    tot[j] += (L <= 4) ? (a << (32 - 8 * L)) : (a >> (8 * L - 32));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();  // every warp has read buffer buf
            if (tid == 0) {
                ok = ok && !st->failed;
                st->uses[buf] += 1;
                if (ok && L + 2 < TC_SL) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    tc_issue_level(st, As, Bs, L + 2, buf);
                }
            }
            __syncthreads();
            ok = !st->failed;
        }
        if (!ok) break;
        // value = 2^(ea+eb-46) tot; tot >> 3 fits the 53-bit mantissa (units of 2^(ea+eb-43)).
        // The integer totals pass through shared memory (the B slices, 32 columns at a
        // time, columns XOR-swizzled by the row) so that C is updated row-contiguously.
        {
            const int rl = 32 * q + lane;
            double* Vs = reinterpret_cast<double*>(Bs);  // TC_M x 32
            for (int half = 0; half < TC_N / 32; ++half) {
                if (h == half)
#pragma unroll
                    for (int j = 0; j < 32; ++j) Vs[rl * 32 + (j ^ (rl & 15))] = (double)(tot[j] >> 3);
                __syncthreads();
                for (int rr = warp; rr < TC_M; rr += blockDim.x >> 5) {
                    const int r = r0 + rr, cl = 32 * half + lane, cc = c0 + cl;
                    if (r >= M || cc >= N) continue;
                    if (LOWER && r + diag < cc) continue;
                    const int es = ea[rr] + eb[cl] - 43 + 1023;
                    if (es < 1 || es > 2046) continue;  // a zero row or column (or far outside range)
                    double* pc = C + (size_t)r * ldc + cc;
                    *pc = fma(-Vs[rr * 32 + (lane ^ (rr & 15))], __longlong_as_double((long long)es << 52), *pc);
                }
                __syncthreads();
            }
        }
        __syncthreads();  // the slices may be overwritten by the next tile
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Long-K products with one FP64 epilogue: C[M x N] -= A[M x K] B[N x K]^T for any K,
// N <= 32 per tile column (tiles of 128 x 32).  Row exponents are taken over all of K
// (a first pass over the tile's rows), every K-chunk of 32 is sliced against them, and
// the integer totals of all chunks are kept in registers (|total| < 2^54 per chunk, so
// up to 500 chunks fit 64 bits); each output then costs two FP64 instructions in all,
// instead of two per chunk.  TRANS writes element (r, c) to C[c * ldc + r].
// smem: TC_SMEM_BYTES; tensor memory: columns [0, 64) of the CTA's allocation.
// ---------------------------------------------------------------------------
#define TCL_N 32
#define TCL_B_SLICE_BYTES (TCL_N * TC_K * 2)  // 2048

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

// slices of rows [r0, r0 + ROWS) x k [k0, k0 + 32) against the fixed row exponents expo[]
template <int ROWS>
__device__ __forceinline__ void tcl_slice_chunk(const double* __restrict__ X, int ld, int r0, int nrows, int k0, int K,
                                                const int* expo, unsigned char* sl, int slice_bytes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kofs = (lane >> 3) * TC_LBO + (lane & 7) * 2;
    constexpr int PER = (ROWS + 7) / 8;  // rows per warp (eight warps): loads issued together
    double x[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * nw, gr = r0 + r, gk = k0 + lane;
        x[i] = (r < ROWS && gr < nrows && gk < K) ? X[(size_t)gr * ld + gk] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = warp + i * nw;
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

__device__ __forceinline__ void tcl_issue_level(TcState* st, const unsigned char* As, const unsigned char* Bs, int L,
                                                int buf) {
    const uint32_t d = st->tmem + (uint32_t)(buf * TCL_N);
    const uint32_t id = tc_idesc(TC_M, TCL_N);
    const uint32_t a0 = tc_smem_u32(As), b0 = tc_smem_u32(Bs);
    int first = 1;
    for (int t = 0; t <= L; ++t) {
        const int u = L - t;
#pragma unroll
        for (int ks = 0; ks < TC_K / 16; ++ks) {
            const uint64_t ad = tc_desc(a0 + t * TC_A_SLICE_BYTES + ks * 2 * TC_LBO);
            const uint64_t bd = tc_desc(b0 + u * TCL_B_SLICE_BYTES + ks * 2 * TC_LBO);
            asm volatile(
                "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(id), "r"(first ? 0 : 1));
            first = 0;
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        tc_smem_u32(&st->mbar[buf])));
    st->issued[buf] += 1;
}

template <bool TRANS>
__device__ void cta_gemm_tc_longk(double* __restrict__ C, int ldc, const double* __restrict__ A, int lda,
                                  const double* __restrict__ B, int ldb, int M, int N, int K, unsigned char* smem,
                                  TcState* st) {
    unsigned char* As = smem;
    unsigned char* Bs = As + TC_SL * TC_A_SLICE_BYTES;
    int* ea = reinterpret_cast<int*>(Bs + TC_SL * TCL_B_SLICE_BYTES);
    int* eb = ea + TC_M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int q = warp & 3, h = warp >> 2;  // rows 32 q .., columns 16 h ..
    const int tilesM = (M + TC_M - 1) / TC_M, tilesN = (N + TCL_N - 1) / TCL_N;
    for (int tix = 0; tix < tilesM * tilesN; ++tix) {
        if (st->failed) break;
        const int ti = tix / tilesN, tj = tix % tilesN;
        const int r0 = ti * TC_M, c0 = tj * TCL_N;
        tcl_row_expo(A, lda, r0, TC_M, M, K, ea);
        tcl_row_expo(B, ldb, c0, TCL_N, N, K, eb);
        __syncthreads();
        long long tot[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) tot[j] = 0;
        bool ok = true;
        for (int k0 = 0; k0 < K && ok; k0 += TC_K) {
            tcl_slice_chunk<TC_M>(A, lda, r0, M, k0, K, ea, As, TC_A_SLICE_BYTES);
            tcl_slice_chunk<TCL_N>(B, ldb, c0, N, k0, K, eb, Bs, TCL_B_SLICE_BYTES);
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                tcl_issue_level(st, As, Bs, 0, 0);
                tcl_issue_level(st, As, Bs, 1, 1);
            }
            for (int L = 0; L < TC_SL; ++L) {
                const int buf = L & 1;
                ok = ok && tc_wait(&st->mbar[buf], st->uses[buf]);
                if (!ok) st->failed = 1;
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (ok) {
                    uint32_t r[16];
                    const uint32_t ta = st->tmem + (uint32_t)(buf * TCL_N + 16 * h) + ((uint32_t)(32 * q) << 16);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                        " [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long a = (long long)__float2int_rn(__uint_as_float(r[j]));
                        tot[j] += (L <= 4) ? (a << (32 - 8 * L)) : (a >> (8 * L - 32));
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                if (tid == 0) {
                    ok = ok && !st->failed;
                    st->uses[buf] += 1;
                    if (ok && L + 2 < TC_SL) {
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        tcl_issue_level(st, As, Bs, L + 2, buf);
                    }
                }
                __syncthreads();
                ok = !st->failed;
            }
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
        if (!TRANS) {
            for (int rr = warp; rr < TC_M; rr += nw) {
                const int r = r0 + rr, cl = lane, cc = c0 + cl;
                if (r >= M || cc >= N) continue;
                const int es = ea[rr] + eb[cl] - 43 + 1023;
                if (es < 1 || es > 2046) continue;
                double* pc = C + (size_t)r * ldc + cc;
                *pc = fma(-Vs[rr * TCL_N + (cl ^ (rr & 15))], __longlong_as_double((long long)es << 52), *pc);
            }
        } else {
            for (int idx = tid; idx < TC_M * TCL_N; idx += blockDim.x) {
                const int cl = idx / TC_M, rr = idx % TC_M;
                const int r = r0 + rr, cc = c0 + cl;
                if (r >= M || cc >= N) continue;
                const int es = ea[rr] + eb[cl] - 43 + 1023;
                if (es < 1 || es > 2046) continue;
                double* pc = C + (size_t)cc * ldc + r;
                *pc = fma(-Vs[rr * TCL_N + (cl ^ (rr & 15))], __longlong_as_double((long long)es << 52), *pc);
            }
        }
        __syncthreads();
    }
    __syncthreads();
}
