// Internal declarations of libdclno: device descriptors, the context, and the
// CTA-wide FP64 tile GEMM that the cluster solver's cubic steps share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dclno.h"

#define DCLNO_MAX_M 32          // largest basis of one atom (M_i)
#define DCLNO_MAX_M_LNO 16      // largest basis of an atom that carries LNOs
#define DCLNO_NB 32             // panel width of the blocked FP64 factorisations
#define DCLNO_SOLVE_THREADS 256 // threads of a per-cluster CTA

// ---------------------------------------------------------------------------
// Device descriptors
// ---------------------------------------------------------------------------
struct ClusterDesc {
    int centre;         // atom i
    int n;              // cluster dimension n_i
    int ld;             // leading dimension of the n x n work matrices (multiple of 4)
    int nmem;           // members (the centre is the last)
    long long mbeg;     // first member in the member arrays
    long long mat_off;  // arena offset (doubles) of the H^(i)/A matrix; S^(i)/L follows at + n*ld
    long long eig_off;  // offset into eps/q (sum of earlier n)
    long long cc_off;   // arena offset of the central strips P ([n][2 M_i])
    long long rot_off;  // arena offset of the QL rotation logs (2 doubles per rotation, rot_cap per segment)
    long long it_off;   // offset (ints) of the QL sweep headers (it_cap ints per segment)
    long long aux_off;  // arena offset of per-cluster vectors d, e, tau (ld each) and W (32 ld)
    int rot_cap;        // capacity of one segment's rotation log
    int it_cap;         // ints of one segment's sweep headers
    int mc;             // M of the central atom
    int split;          // tear point k of the tridiagonal matrix (segments [0,k), [k,n)); 0 = no tear
    long long pair_off; // offset of the cluster's member-pair block table (nmem x nmem ints)
    long long m_off;    // arena offset of the merge matrix M (n x ld) and its transpose (n x ld); split only
    long long q2_off;   // arena offset of the bulge-chasing reflector log of the two-stage reduction
                        // (band_refl_count(n) slots of DCLNO_BW doubles), -1 if the cluster is too small
    // Cuppen's tear applied twice (split2): each half [0, split), [split, n) is torn again at
    // split1 and split3 (absolute positions); the halves' QL, merges, rotation replays and
    // merge-matrix products run on two half descriptors (see make_halves), the cluster's
    // own merge then joins the halves.  Half descriptors describe a half's problem with
    // offsets into the cluster's workspace; kernels that take either kind index the status
    // word by sidx.
    int sidx;           // status index: the cluster itself (or, for a half, its cluster)
    int split2;         // cluster torn twice (real descriptors only)
    int split1, split3; // the halves' tears (absolute positions), split2 only
    int x2_mode;        // halves: 0 none; 1 segment 0 also carries its first row; 2 segment 1 its last row
    int g_row0;         // first row of this problem in the cluster (0, or split for the second half)
    long long w_off;    // z row of this problem's merge (n doubles) and the tear's beta at [n]
    long long gb_off;   // the cluster's density-column block G (row stride = columns of G)
    long long scr_off;  // scratch of the strips' merge-matrix product (n x 2 mc doubles)
    long long x2_off;   // the carried extra rows, indexed by row of the cluster (x2_mode != 0)
};

// Two-stage tridiagonalisation: A -> band of half-width DCLNO_BW (blocked Householder,
// k_band) -> tridiagonal (Householder bulge chasing, k_chase).  Sweep j of the chase
// (j = 0 .. n-3) uses reflectors k = 0, 1, ... acting on rows [p, p + min(BW, n - p))
// with p = j + 1 + k BW while p + 1 < n.
#define DCLNO_BW 32
#define DCLNO_TWO_STAGE_MIN 128  // clusters of at least this dimension (and torn) may use it
// the automatic choice: the mixed path's clusters of at least this dimension (measured on
// GB300 with the double-float bulge chasing: two-stage faster at n ~ 147-285 (763 against
// 827 ms per step), 231-385 (602 against 631 ms) and 654-702; the FP64 path stays one-stage)
#define DCLNO_TWO_STAGE_AUTO_MIN 128
__host__ __device__ inline long long chase_steps(int n, int j) {
    const int r = n - 2 - j;
    return r > 0 ? (r + DCLNO_BW - 1) / DCLNO_BW : 0;
}
__host__ __device__ inline long long band_refl_count(int n) {
    long long s = 0;
    for (int j = 0; j + 2 < n; ++j) s += chase_steps(n, j);
    return s;
}

// segment s (0, 1) of a cluster's tridiagonal problem: first index and length
__host__ __device__ inline int seg_start(const ClusterDesc& d, int s) { return s ? d.split : 0; }
__host__ __device__ inline int seg_len(const ClusterDesc& d, int s) {
    return d.split ? (s ? d.n - d.split : d.split) : (s ? 0 : d.n);
}
#define DCLNO_TEAR_MIN 64  // tear tridiagonal matrices of at least this dimension
// tear twice (four segments, two merge levels) in the automatic mode from this dimension on
#define DCLNO_TEAR2_MIN 512
#define DCLNO_QL_CANDIDATES 6  // QL lanes per warp tried by the autotuner: 4, 8, 12, 16, 24, 32

// The W rows of a cluster (aux_off + 3 ld, 32 ld doubles) after the reduction, each
// ld + 4 doubles long (a z row of n <= ld entries and the tear's beta at [n]): row 0 the
// cluster's merge vector z; rows 1, 2 those of the halves of a cluster torn twice; row 3
// the halves' carried extra rows.  Later the density columns G and the merge products'
// scratch reuse the block.
#define DCLNO_W_HALF0 1
#define DCLNO_W_HALF1 2
#define DCLNO_W_X2 3
__host__ __device__ inline long long w_row(int ld, int r) { return (long long)r * (ld + 4); }

// Cuppen's tear of T at k: T = diag(T1, T2) + |beta| v v^T with beta = e[k-1],
// v = e_{k-1} + sign(beta) e_k; d[k-1], d[k] are lowered by |beta|, e[k-1] = 0 and
// beta is kept in *beta_out.
__host__ __device__ inline void tear_at(double* dv, double* ev, int k, double* beta_out) {
    const double beta = ev[k - 1];
    *beta_out = beta;
    ev[k - 1] = 0.0;
    dv[k - 1] -= fabs(beta);
    dv[k] -= fabs(beta);
}
// every tear of a cluster (one thread): at split (beta in W row 0 at [n]); for a cluster
// torn twice also at split1 and split3 (betas at the halves' rows, at the half's length)
__host__ __device__ inline void tear_cluster(const ClusterDesc& d, double* arena) {
    if (!d.split) return;
    double* dv = arena + d.aux_off;
    double* ev = dv + d.ld;
    double* W = dv + 3 * (size_t)d.ld;
    tear_at(dv, ev, d.split, W + d.n);
    if (d.split2) {
        tear_at(dv, ev, d.split1, W + w_row(d.ld, DCLNO_W_HALF0) + d.split);
        tear_at(dv, ev, d.split3, W + w_row(d.ld, DCLNO_W_HALF1) + (d.n - d.split));
    }
}

struct MemberDesc {
    int atom;   // j
    int shift;  // packed cell shift (see pack_shift)
    int off;    // first basis function of the member in the cluster basis
    int core;   // 1 = PAO member (M_j functions), 0 = LNO member (k functions)
};

// cell shift (three signed bytes) packed into 24 bits of an int
__host__ __device__ inline int pack_shift(int s0, int s1, int s2) {
    return ((s0 + 128) << 16) | ((s1 + 128) << 8) | (s2 + 128);
}
__host__ __device__ inline void unpack_shift(int p, int& s0, int& s1, int& s2) {
    s0 = ((p >> 16) & 255) - 128;
    s1 = ((p >> 8) & 255) - 128;
    s2 = (p & 255) - 128;
}
// BSR search key of a block: (col, packed shift) as one sortable 64-bit integer
__host__ __device__ inline long long block_key(int col, int pshift) {
    return ((long long)col << 24) | (long long)pshift;
}

// Per-cluster status words written by kernels (0 = ok).
enum : int {
    ST_OK = 0,
    ST_NOT_SPD = 1,
    ST_NOT_CONVERGED = 2,
    ST_LOG_FULL = 3,
    ST_BAD_LNO = 4,
    ST_FEW_POLES = 5,  // the Matsubara pole sum was asked for too few poles for this cluster
    ST_TIMEOUT = 6,    // a bounded wait on the tensor cores ran out
};

// A memory-admitted batch: a contiguous range of cluster ids whose workspace is
// resident at once.  Arena offsets (mat_off, aux_off, cc_off, rot_off) and sweep
// header offsets (it_off) of its clusters are relative to the batch; eig_off and
// pair_off are global.
// A size bucket: a contiguous range of a batch's clusters in the scheduling order
// (decreasing n) whose dimensions round up to the same multiple of 64, buckets of
// fewer than two CTAs per SM merged into a neighbour (a launch ends in a tail of
// idle SMs: a bucket of a few clusters would cost the time of a whole cluster while
// the rest of the GPU waits).  Each bucket has its own schedule; consecutive
// buckets whose schedules agree run as one launch.
struct Bucket {
    int obeg = 0, oend = 0;  // positions in dclno_ctx::order
    int nround = 0;          // dimension rounded up to 64
    int maxn = 0;
};

// cubic kernels with a tuned schedule
enum { TK_CHOL = 0, TK_CONG, TK_TRI, TK_BAND, TK_CHASE, TK_COUNT };
// Schedule of one kernel on one bucket: engine of the emulated products (0 FP64 tiles,
// 1 mma.sync, 2 tcgen05) and grid form (0 one CTA per cluster, 1 persistent CTAs on an
// atomic work counter).  Every choice gives the same bits.
struct Sched {
    int engine = 0;
    int persistent = 0;
};
// One launch of a tuned kernel: consecutive buckets [k0, k1) sharing schedule s, or
// a single bucket timed for the tuner (cand >= 0).
struct SchedRun {
    int k0 = 0, k1 = 0;
    int obeg = 0, oend = 0, maxn = 0;
    Sched s;
    int cand = -1;
};
struct TuneSlot {
    int next = 0;             // next candidate to time
    int chosen = -1;          // index into the candidates once decided
    bool from_cache = false;
    int default_index = -1;   // the untuned schedule among the candidates
    std::vector<float> ms;    // timed milliseconds per cluster, per candidate (-1 = not timed)
};
struct TunePending {
    std::string slot;
    int cand;
    cudaEvent_t e0, e1;
    int clusters;
};

struct Batch {
    int id_lo = 0, id_hi = 0;       // clusters [id_lo, id_hi)
    int obeg = 0, oend = 0;         // the same clusters in `order` (by decreasing n)
    int l1beg = 0, l1end = 0;       // two-segment problems in `l1`: clusters torn once, halves of the others
    int l2beg = 0, l2end = 0;       // clusters torn twice in `l2` (their merge of the halves)
    int segmax = 1, l1maxn = 0;     // longest segment, largest problem in l1
    long long mbeg = 0, mend = 0;   // their members
    int maxn = 0, mcmax = 1;
    long long arena_doubles = 0, iters = 0;
    int index = 0;                  // position in dclno_ctx::batches
    std::vector<Bucket> buckets;
};

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct dclno_ctx {
    cudaStream_t stream = nullptr;
    std::string err;
    long long launches = 0;
    int device = 0;
    int nsm = 1;  // streaming multiprocessors of the device (grid sizes are multiples of it)

    // system (host copies of the structure, device pointers of the values)
    int N = 0;
    long long nnzb = 0, nval = 0;
    std::vector<int> norb;
    std::vector<long long> row_ptr, blk_off;
    std::vector<int> col;
    std::vector<int> pshift;  // packed shifts
    std::vector<double> pos, cell;
    int pbc[3] = {0, 0, 0};
    const double* H = nullptr;
    const double* S = nullptr;
    int* d_norb = nullptr;
    long long* d_row_ptr = nullptr;
    long long* d_key = nullptr;        // block_key per block
    long long* d_blk_off = nullptr;
    long long* d_onsite = nullptr;     // block index of S_ii per atom
    long long* d_voff = nullptr;       // offset of atom i's LNO block (M_i x k) in d_V
    long long* d_loff = nullptr;       // offset of atom i's Lambda block (M_i^2)
    long long* d_moff = nullptr;       // offset of atom i's eigenvalues lambda (M_i)

    // clusters
    bool built = false;
    double r_core = 0, r_lno = 0;
    int k_lno = 0;
    bool has_lno_region = false;
    std::vector<ClusterDesc> cl;      // one per atom, atom order
    std::vector<int> order;           // per batch, its clusters by decreasing n (scheduling)
    std::vector<Batch> batches;       // memory-admitted batches (one when everything fits)
    int resident = -1;                // batch whose solved workspace is in the arena
    dclno_precision solved_prec = DCLNO_FP64;
    // tridiagonalisation: 0 = automatic (two-stage in the mixed path, one-stage in FP64),
    // 1 = one-stage, 2 = two-stage (for the clusters that qualify); solved_two = the form
    // the last solve used (the density pass applies the same Q)
    int tridiag_mode = 0;
    int tear_mode = 0;        // 0 automatic (twice from DCLNO_TEAR2_MIN), 1 once, 2 twice where possible
    int layout_tear = -1;     // tear mode when the workspace was laid out
    int layout_mode = -1;     // tridiagonalisation mode when the workspace was laid out (-1: not yet)
    bool solved_two = false;
    // engine of the mixed path's K <= 32 tile products (Cholesky, congruence, one-stage
    // tridiagonalisation): 0 = chosen per kernel and bucket by the tuner, 1 = mma.sync,
    // 2 = tcgen05; the long-K products (band reduction, merge matrix) always use tcgen05
    int mixed_engine = 0;
    // schedules of the cubic kernels: 0 tuned, 1 one CTA per cluster, 2 persistent
    int sched_force = 0;
    int bucket_min = 0;  // minimum clusters per size bucket (0: twice the SM count)
    std::map<std::string, TuneSlot> tune_slots;  // key: batch / bucket / kernel / precision
    std::map<std::string, Sched> tune_cache;     // key: gpu | precision | kernel | rounded n
    std::string tune_cache_path, gpu_name;
    std::vector<TunePending> tune_pending;
    int* d_queue = nullptr;                      // work counter of persistent launches
    size_t ws_limit = 0;              // workspace limit in bytes (0 = free device memory)
    // launch-shape autotuner: QL lanes per warp chosen per batch by timing (0 = not yet)
    bool autotune = true;
    std::vector<int> ql_lanes;
    std::vector<float> ql_tune_ms;    // per batch: the timed candidates (lanes 4, 8, 12, 16, 24, 32)
    double* d_tune = nullptr;         // saved d, e of a batch while candidates are timed
    size_t tune_doubles = 0;
    void* d_pole = nullptr;           // scratch of the Matsubara pole sum (pivots, solutions per pole)
    size_t pole_bytes = 0;
    std::vector<MemberDesc> mem;
    long long total_dim = 0;
    ClusterDesc* d_cl = nullptr;  // N cluster descriptors, then 2 N half descriptors
    int* d_order = nullptr;
    std::vector<ClusterDesc> clh;     // half descriptors (2 per cluster; meaningful where split2)
    std::vector<int> l1, l2;          // see Batch::l1beg, l2beg (indices into d_cl)
    int* d_l1 = nullptr;
    int* d_l2 = nullptr;
    MemberDesc* d_mem = nullptr;
    int* d_mem_cl = nullptr;           // cluster of each member (atom order)
    int* d_pairblk = nullptr;          // per cluster, member pair -> BSR block (or -1)
    long long pair_total = 0;
    int* d_brow = nullptr;             // row (atom) of every BSR block
    long long* d_tblk_off = nullptr;   // per block: offset of its LNO-transformed blocks
    double* d_tblk = nullptr;          // LNO-transformed blocks (V^T X, X V, V^T X V for X = H, S)
    long long tblk_total = 0;
    int* d_rowblk_member = nullptr;    // per block of row i: member of cluster i or -1
    int* d_status = nullptr;           // per cluster
    double* d_arena = nullptr;
    size_t arena_doubles = 0;
    int* d_iters = nullptr;            // QL sweep headers
    double* d_eps = nullptr;
    double* d_q = nullptr;

    // LNOs
    bool lnos_ready = false;
    long long v_total = 0, l_total = 0;
    double* d_V = nullptr;
    double* d_lam_re = nullptr;
    double* d_lam_im = nullptr;
    double* d_Lambda = nullptr;
    int* d_lflags = nullptr;
    // threshold selection of LNOs (Sec. II.B step (iii)): per-atom counts <= k_lno; the
    // workspace is laid out for k_lno, the dimensions follow the counts of the last LNOs
    bool lno_th_on = false;
    double lno_th = 0.0;
    int* d_kat = nullptr;               // LNOs of each atom (k_lno without a threshold)
    std::vector<int> kat;
    bool relaid = false;                // the layout follows threshold-selected counts
    // LNO eigenproblem: 0 = the paper's nonsymmetric Lambda, 1 = (S rho S)_ii v = lambda S_ii v
    int lno_mode = 0;
    long long max_row = 0;              // longest BSR row (blocks)
    std::vector<char> layout_split;     // per cluster: laid out as a torn problem
    std::vector<char> layout_split2;    // per cluster: laid out as a problem torn twice

    // solve / mu
    bool solved = false;
    double* d_mu_work = nullptr;       // k-section partial sums
    double* d_scalars = nullptr;       // [lo, hi, mu, N, ...]
    double* d_eband = nullptr;         // per-cluster band energies

    // host-buffer step
    double* d_rho_in = nullptr;
    double* d_rho_out = nullptr;

    // deferred mode (SCF loop, graph capture): launchers skip every host readback;
    // statuses accumulate in d_err, mu stays on the device, per-step results go to d_hist
    bool deferred = false;
    int* d_err = nullptr;       // [0] sticky worst status of the loop, [1] step counter
    double* d_hist = nullptr;   // per step: mu, N(mu), E_band
    int hist_cap = 0;

    // optional per-kernel CUDA-event timing (dclno_set_profiling)
    struct Prof {
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
        double ms = 0.0;
        long long launches = 0;
    };
    bool prof_on = false;
    std::map<std::string, Prof> prof;
};

// Event pair around one launch when profiling is on (no-op otherwise).
struct ProfScope {
    dclno_ctx* c;
    const char* name;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ProfScope(dclno_ctx* ctx, const char* n) : c(ctx), name(n) {
        if (c->prof_on && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess)
            cudaEventRecord(e0, c->stream);
    }
    ~ProfScope() {
        if (e1) {
            cudaEventRecord(e1, c->stream);
            c->prof[name].pending.push_back({e0, e1});
        }
    }
};
void prof_collect(dclno_ctx* c);

// ---------------------------------------------------------------------------
// Error helpers
// ---------------------------------------------------------------------------
dclno_status set_err(dclno_ctx* c, dclno_status st, const std::string& msg);
dclno_status cuda_err(dclno_ctx* c, cudaError_t e, const char* where);
#define DCLNO_CUDA(ctx, call)                                            \
    do {                                                                 \
        cudaError_t e__ = (call);                                        \
        if (e__ != cudaSuccess) return cuda_err((ctx), e__, #call);      \
    } while (0)
#define DCLNO_LAUNCHED(ctx)                                              \
    do {                                                                 \
        (ctx)->launches++;                                               \
        cudaError_t e__ = cudaGetLastError();                            \
        if (e__ != cudaSuccess) return cuda_err((ctx), e__, "launch");   \
    } while (0)

// kernels' host-side launchers (one per .cu file)
dclno_status prepare_lno_kernels(dclno_ctx* c);
dclno_status launch_lambda_lno(dclno_ctx* c, const double* rho);
dclno_status relayout_clusters(dclno_ctx* c);
dclno_status launch_lno_blocks(dclno_ctx* c);
dclno_status launch_assemble(dclno_ctx* c, const Batch& b);
dclno_status launch_pair_index(dclno_ctx* c);
// reduce_only: Cholesky, congruence, tridiagonalisation and the central strips P = [R1 Q; R2 Q]
// only (the Matsubara pole route), without the tridiagonal eigensolve and the weights
dclno_status launch_solve_fp64(dclno_ctx* c, const Batch& b, bool reduce_only = false);
dclno_status launch_solve_mixed(dclno_ctx* c, const Batch& b, bool reduce_only = false);
dclno_status launch_poles(dclno_ctx* c, const Batch& b, double mu, double kT, int npoles);
dclno_status launch_merge(dclno_ctx* c, const Batch& b);
dclno_status launch_two_stage(dclno_ctx* c, const Batch& b, bool mixed, bool tune);

// scheduler (sched.cu)
void build_buckets(dclno_ctx* c, Batch& b);
// the schedule of `kernel` on bucket k of batch b; *cand >= 0 when this launch is timed
// for the tuner (then bracket it with sched_time_begin / sched_time_end)
Sched sched_pick(dclno_ctx* c, const Batch& b, int k, int kernel, bool mixed, bool tune, int* cand);
// the launches of `kernel` over the buckets with use[k] != 0
std::vector<SchedRun> sched_runs(dclno_ctx* c, const Batch& b, int kernel, bool mixed, bool tune,
                                 const std::vector<char>& use);
dclno_status sched_time_begin(dclno_ctx* c, cudaEvent_t* e0);
dclno_status sched_time_end(dclno_ctx* c, const Batch& b, int k, int kernel, bool mixed, int cand, cudaEvent_t e0);
void sched_collect(dclno_ctx* c);  // after the stream is synchronised: fold timings into the slots
void sched_reset(dclno_ctx* c);
int sched_grid(dclno_ctx* c, const void* fn, int threads, size_t smem, int nitems, bool persistent);
// Y <- X Y for the torn clusters of a batch: dir 0 = central strips P <- M^T P (after the
// forward replay), dir 1 = density columns G <- M G (before the reverse replay)
dclno_status launch_mgemm(dclno_ctx* c, const Batch& b, int dir, int with_e, int emu);
dclno_status launch_find_mu(dclno_ctx* c, double ne, double kT, double* mu, double* nmu);
// poles: the density columns G are already formed (k_poles); only L^-T Q G and the scatter
dclno_status launch_density(dclno_ctx* c, const Batch& b, double mu, double kT, double* rho_out,
                            double* e_out = nullptr, bool poles = false);
dclno_status launch_status_or(dclno_ctx* c);
dclno_status launch_scf_tail(dclno_ctx* c, double* rho, const double* rho_out, double alpha);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Householder reflector k of the tridiagonalisation, H_k = I - tau v v^T with v_{k+1} = 1
// and v_t (t > k+1) = v[t] (row k of the matrix's upper triangle, where k_tridiag keeps a
// contiguous copy), applied as x <- x - tau (x . v) v to the R consecutive rows of the
// shared-memory matrix X (row stride ldx) that this warp owns.  Each lane touches the
// entries t = lane (mod 32) only, so the rows need no synchronisation between
// successive reflectors.
#define DCLNO_RPW 4  // rows per warp at most
template <int R>
__device__ __forceinline__ void warp_reflect(double* X, int ldx, int k, int n, const double* __restrict__ v,
                                             double tau) {
    const int lane = threadIdx.x & 31;
    double u[R];
#pragma unroll
    for (int j = 0; j < R; ++j) u[j] = 0.0;
    for (int t = k + 1 + lane; t < n; t += 32) {
        const double vt = v[t];
#pragma unroll
        for (int j = 0; j < R; ++j) u[j] = fma(X[(size_t)j * ldx + t], vt, u[j]);
    }
#pragma unroll
    for (int j = 0; j < R; ++j) u[j] = tau * warp_sum(u[j]);
    for (int t = k + 1 + lane; t < n; t += 32) {
        const double vt = v[t];
#pragma unroll
        for (int j = 0; j < R; ++j) X[(size_t)j * ldx + t] = fma(-u[j], vt, X[(size_t)j * ldx + t]);
    }
}

// One logged QL sweep applied to a strided vector x_t = X[t * stride]:
// rotations u = 0 .. cnt-1 act on (i, i+1) with i = i0 - u, as column updates
//   x_{i+1} <- s x_i + c x_{i+1},  x_i <- c x_i - s x_{i+1}
// (sweep_fwd, the order they were generated: x <- x Z), or in reverse order with the
// transposed rotations (sweep_rev: x <- Z x).  Operands are loaded D rotations
// ahead: a replay is a serial chain per vector, so the load latency would
// otherwise set the time per rotation.  rot points at the sweep's first rotation.
template <int D>
__host__ __device__ __forceinline__ void sweep_fwd(double* __restrict__ X, size_t stride, const double2* __restrict__ rot,
                                          int i0, int cnt) {
    double xb[D];
    double2 cb[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        xb[q] = 0.0;
        cb[q] = make_double2(1.0, 0.0);
        if (q < cnt) {
            xb[q] = X[(size_t)(i0 - q) * stride];
            cb[q] = rot[q];
        }
    }
    double xi1 = X[(size_t)(i0 + 1) * stride];
    for (int u0 = 0; u0 < cnt; u0 += D) {
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const int u = u0 + q;
            if (u < cnt) {
                const int i = i0 - u;
                const double xi = xb[q];
                const double2 cs = cb[q];
                if (u + D < cnt) {  // row i - D is written only after rotation u + D has read it
                    xb[q] = X[(size_t)(i - D) * stride];
                    cb[q] = rot[u + D];
                }
                X[(size_t)(i + 1) * stride] = fma(cs.y, xi, cs.x * xi1);
                xi1 = fma(cs.x, xi, -cs.y * xi1);
            }
        }
    }
    X[(size_t)(i0 + 1 - cnt) * stride] = xi1;
}

template <int D>
__host__ __device__ __forceinline__ void sweep_rev(double* __restrict__ X, size_t stride, const double2* __restrict__ rot,
                                          int i0, int cnt) {
    const int ib = i0 - (cnt - 1);  // rows (ib + m, ib + m + 1) at step m = 0 .. cnt-1 (rotation cnt-1-m)
    double xb[D];
    double2 cb[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        xb[q] = 0.0;
        cb[q] = make_double2(1.0, 0.0);
        if (q < cnt) {
            xb[q] = X[(size_t)(ib + q + 1) * stride];
            cb[q] = rot[cnt - 1 - q];
        }
    }
    double wi = X[(size_t)ib * stride];
    for (int m0 = 0; m0 < cnt; m0 += D) {
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const int m = m0 + q;
            if (m < cnt) {
                const int i = ib + m;
                const double wi1 = xb[q];
                const double2 cs = cb[q];
                if (m + D < cnt) {  // row i + 1 + D is written at step m + D + 1
                    xb[q] = X[(size_t)(i + 1 + D) * stride];
                    cb[q] = rot[cnt - 1 - m - D];
                }
                X[(size_t)i * stride] = fma(cs.x, wi, cs.y * wi1);
                wi = fma(-cs.y, wi, cs.x * wi1);
            }
        }
    }
    X[(size_t)(ib + cnt) * stride] = wi;
}
#define DCLNO_REPLAY_DEPTH 1  // the replays run many warps per SM and are bound by the FP64 pipe

// A cluster reduced by the two-stage tridiagonalisation (band.cu) when that mode is on.
__device__ __forceinline__ bool two_stage_cluster(const ClusterDesc& d) {
    return d.q2_off >= 0 && d.split && d.n >= DCLNO_TWO_STAGE_MIN;
}

// Chase reflector H = I - tau v v^T of the two-stage reduction, log slot
// [tau, v_1 .. v_{len-1}] (v_0 = 1), acting on entries [p, p + len) of the R
// consecutive rows of X (row stride ldx) that this warp owns: x <- x - tau (x . v) v.
template <int R>
__device__ __forceinline__ void warp_reflect_short(double* X, int ldx, int p, int len,
                                                   const double* __restrict__ slot) {
    const int lane = threadIdx.x & 31;
    const double tau = slot[0];
    if (tau == 0.0) return;  // the same for every lane
    const double v = (lane == 0) ? 1.0 : (lane < len ? slot[lane] : 0.0);
    double u[R];
#pragma unroll
    for (int j = 0; j < R; ++j) u[j] = (lane < len) ? X[(size_t)j * ldx + p + lane] * v : 0.0;
#pragma unroll
    for (int j = 0; j < R; ++j) u[j] = tau * warp_sum(u[j]);
#pragma unroll
    for (int j = 0; j < R; ++j)
        if (lane < len) X[(size_t)j * ldx + p + lane] = fma(-u[j], v, X[(size_t)j * ldx + p + lane]);
}

// Sum over the 32 lanes of 16 values per lane at once ("transposing" reduction): each
// step halves the values a lane keeps, sending the other half to its partner, so the
// 16 sums cost 8 + 4 + 2 + 1 + 1 = 16 FP64 adds per lane instead of 16 x 5 for separate
// butterflies (on this GPU a warp-wide FP64 instruction occupies the SM's FP64 pipe for
// about 19 cycles).  On return lane L holds the sum of value (L >> 1) & 15.
__device__ __forceinline__ double warp_sum16(double (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16, cnt = 8; s >= 2; s >>= 1, cnt >>= 1) {
        const bool hi = (lane & s) != 0;  // this lane keeps the upper half of its values
#pragma unroll
        for (int i = 0; i < cnt; ++i) {
            const double send = hi ? v[i] : v[i + cnt];
            const double keep = hi ? v[i + cnt] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// The same for 8 values per lane (4 + 2 + 1 transposing adds, then 2 butterfly adds):
// on return lane L holds the sum of value (L >> 2) & 7.
__device__ __forceinline__ double warp_sum8(double (&v)[8]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16, cnt = 4; s >= 4; s >>= 1, cnt >>= 1) {
        const bool hi = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < cnt; ++i) {
            const double send = hi ? v[i] : v[i + cnt];
            const double keep = hi ? v[i + cnt] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    const double a = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
    return a + __shfl_xor_sync(0xffffffffu, a, 1);
}

// The chase reflectors of sweep j (disjoint windows [p_k, p_k + len_k), p_k = j + 1 + k BW)
// on the R rows of X owned by this warp: KW = 16 / R windows at a time, their KW x R dot
// products reduced together by warp_sum16.  Windows of one sweep commute, so the same
// code serves both directions.
template <int R>
__device__ __forceinline__ void warp_chase_sweep(double* X, int n, int j, const double* __restrict__ slot0) {
    constexpr int KW = 16 / R;
    const int lane = threadIdx.x & 31;
    const int ns = (int)chase_steps(n, j);
    for (int k0 = 0; k0 < ns; k0 += KW) {
        double v[KW], val[16];
        int p[KW];
        bool on[KW];
#pragma unroll
        for (int i = 0; i < 16; ++i) val[i] = 0.0;
#pragma unroll
        for (int w = 0; w < KW; ++w) {
            const int k = k0 + w;
            p[w] = j + 1 + k * DCLNO_BW;
            const int len = k < ns ? min(DCLNO_BW, n - p[w]) : 0;
            const double* sl = slot0 + (size_t)k * DCLNO_BW;
            on[w] = lane < len;
            const double tau = k < ns ? sl[0] : 0.0;
            v[w] = !on[w] ? 0.0 : (lane == 0 ? 1.0 : sl[lane]);
            const double vt = tau * v[w];  // the dot products come out scaled by tau
#pragma unroll
            for (int r = 0; r < R; ++r) val[w * R + r] = on[w] ? X[(size_t)r * n + p[w] + lane] * vt : 0.0;
        }
        const double mine = warp_sum16(val);  // lane L: pair (L >> 1) & 15 = w R + r
#pragma unroll
        for (int w = 0; w < KW; ++w)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const double u = __shfl_sync(0xffffffffu, mine, 2 * (w * R + r));
                if (on[w]) {
                    double* x = X + (size_t)r * n + p[w] + lane;
                    *x = fma(-u, v[w], *x);
                }
            }
    }
}

// The two-stage factor Q = Q1 Q2 (A = Q T Q^T) on the R rows of X owned by this warp:
// Q1 = the panel reflectors (reflector c in row c of A's upper triangle from column
// c + BW on, tau[c], 0 where there is none), Q2 = the chase log q2 in generation order.
// dir 0: X <- X Q (the central strips, reflectors in their order); dir 1: each row x of
// X <- Q x (the density columns stored as rows, reflectors in reverse order: each
// reflector is symmetric).
template <int R>
__device__ __forceinline__ void warp_apply_two_stage(double* X, int n, const double* __restrict__ A, int ld,
                                                     const double* __restrict__ tau, const double* __restrict__ q2,
                                                     int dir) {
    if (dir == 0) {
        for (int c = 0; c + DCLNO_BW < n; ++c) {
            const double tc = tau[c];
            if (tc != 0.0) warp_reflect<R>(X, n, c + DCLNO_BW - 1, n, A + (size_t)c * ld, tc);
        }
        const double* slot = q2;
        for (int j = 0; j + 2 < n; ++j) {
            warp_chase_sweep<R>(X, n, j, slot);
            slot += chase_steps(n, j) * DCLNO_BW;
        }
        return;
    }
    const double* slot = q2 + band_refl_count(n) * DCLNO_BW;
    for (int j = n - 3; j >= 0; --j) {
        slot -= chase_steps(n, j) * DCLNO_BW;
        warp_chase_sweep<R>(X, n, j, slot);
    }
    for (int c = n - 1 - DCLNO_BW; c >= 0; --c) {
        const double tc = tau[c];
        if (tc != 0.0) warp_reflect<R>(X, n, c + DCLNO_BW - 1, n, A + (size_t)c * ld, tc);
    }
}

// One FP64 tensor-core MMA: D(8x8) += A(8x4, row) * B(4x8, col).
// Fragments (per lane l): a = A[l/4][l%4], b = B[l%4][l/4],
// c = {C[l/4][2(l%4)], C[l/4][2(l%4)+1]}.
__device__ __forceinline__ void dmma_8x8x4(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// Shared-memory tile geometry of cta_gemm_nt: 64 x 64 outputs, K chunks of 32,
// rows padded to 36 doubles so that the 16 lanes of a half-warp hit distinct banks.
#define GT_M 64
#define GT_N 64
#define GT_K 32
#define GT_LD 36
#define GT_SMEM_DOUBLES (2 * 64 * GT_LD)

// C[M x N] -= A[M x K] * B[N x K]^T over the whole CTA (256 threads), all
// row-major in global memory with leading dimensions lda, ldb, ldc (multiples
// of 2 doubles, base pointers 16-byte aligned).  With LOWER, only elements with
// (row + diag) >= col are written and tiles wholly above that line are skipped.
// smem must hold GT_SMEM_DOUBLES doubles.  Ends with __syncthreads().
template <bool LOWER>
__device__ void cta_gemm_nt_sub(double* __restrict__ C, int ldc, const double* __restrict__ A, int lda,
                                const double* __restrict__ B, int ldb, int M, int N, int K, int diag,
                                double* smem) {
    double* As = smem;
    double* Bs = smem + GT_M * GT_LD;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 16;  // warp's row offset in the tile (0,16,32,48)
    const int wc = (warp & 1) * 32;   // warp's col offset (0,32)
    const int fr = lane >> 2, fk = lane & 3;
    const int tilesM = (M + GT_M - 1) / GT_M, tilesN = (N + GT_N - 1) / GT_N;
    for (int t = 0; t < tilesM * tilesN; ++t) {
        const int ti = t / tilesN, tj = t % tilesN;
        const int r0 = ti * GT_M, c0 = tj * GT_N;
        if (LOWER && r0 + GT_M - 1 + diag < c0) continue;  // uniform across the CTA
        double acc[2][4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
        for (int k0 = 0; k0 < K; k0 += GT_K) {
            // stage A[r0:r0+64, k0:k0+32] and B[c0:c0+64, k0:k0+32] (zero-filled); all of a
            // thread's loads are issued before its shared-memory stores
            constexpr int PER = GT_M * GT_K / 2 / DCLNO_SOLVE_THREADS;
            double2 va[PER], vb[PER];
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int e = tid + i * DCLNO_SOLVE_THREADS;
                const int r = e / (GT_K / 2), kk = (e % (GT_K / 2)) * 2;
                va[i] = vb[i] = make_double2(0.0, 0.0);
                const int gk = k0 + kk;
                if (r0 + r < M) {
                    const double* p = A + (size_t)(r0 + r) * lda + gk;
                    if (gk + 1 < K) va[i] = *reinterpret_cast<const double2*>(p);
                    else if (gk < K) va[i].x = p[0];
                }
                if (c0 + r < N) {
                    const double* p = B + (size_t)(c0 + r) * ldb + gk;
                    if (gk + 1 < K) vb[i] = *reinterpret_cast<const double2*>(p);
                    else if (gk < K) vb[i].x = p[0];
                }
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int e = tid + i * DCLNO_SOLVE_THREADS;
                const int r = e / (GT_K / 2), kk = (e % (GT_K / 2)) * 2;
                As[r * GT_LD + kk] = va[i].x;
                As[r * GT_LD + kk + 1] = va[i].y;
                Bs[r * GT_LD + kk] = vb[i].x;
                Bs[r * GT_LD + kk + 1] = vb[i].y;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < GT_K; kk += 4) {
                double a[2], b[4];
#pragma unroll
                for (int i = 0; i < 2; ++i) a[i] = As[(wr + 8 * i + fr) * GT_LD + kk + fk];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[(wc + 8 * j + fr) * GT_LD + kk + fk];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) dmma_8x8x4(acc[i][j][0], acc[i][j][1], a[i], b[j]);
            }
            __syncthreads();
        }
        // C's elements are all loaded before any is stored (the loads overlap)
        double cv[2][4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = r0 + wr + 8 * i + fr, cc = c0 + wc + 8 * j + 2 * fk + h;
                    const bool ok = r < M && cc < N && !(LOWER && r + diag < cc);
                    cv[i][j][h] = ok ? C[(size_t)r * ldc + cc] : 0.0;
                }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = r0 + wr + 8 * i + fr, cc = c0 + wc + 8 * j + 2 * fk + h;
                    if (r < M && cc < N && !(LOWER && r + diag < cc)) C[(size_t)r * ldc + cc] = cv[i][j][h] - acc[i][j][h];
                }
    }
    __syncthreads();
}

#endif  // __CUDACC__
