// C-ABI entry points of libdclno and the host-side set-up of a DC-LNO step:
// truncated clusters, device copies of the system structure, workspace layout.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "dclno_internal.cuh"

dclno_status set_err(dclno_ctx* c, dclno_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

dclno_status cuda_err(dclno_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                    ") in " + where;
    if (e == cudaErrorMemoryAllocation) return set_err(c, DCLNO_ERR_OOM, m);
    return set_err(c, DCLNO_ERR_CUDA, m);
}

template <class T>
static void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

static void free_clusters(dclno_ctx* c) {
    dfree(c->d_norb);
    dfree(c->d_row_ptr);
    dfree(c->d_key);
    dfree(c->d_blk_off);
    dfree(c->d_onsite);
    dfree(c->d_voff);
    dfree(c->d_loff);
    dfree(c->d_moff);
    dfree(c->d_cl);
    dfree(c->d_order);
    dfree(c->d_l1);
    dfree(c->d_l2);
    dfree(c->d_mem);
    dfree(c->d_mem_cl);
    dfree(c->d_pairblk);
    dfree(c->d_brow);
    dfree(c->d_tblk_off);
    dfree(c->d_tblk);
    dfree(c->d_rowblk_member);
    dfree(c->d_status);
    dfree(c->d_arena);
    dfree(c->d_iters);
    dfree(c->d_eps);
    dfree(c->d_q);
    dfree(c->d_V);
    dfree(c->d_lam_re);
    dfree(c->d_lam_im);
    dfree(c->d_Lambda);
    dfree(c->d_lflags);
    dfree(c->d_mu_work);
    dfree(c->d_scalars);
    dfree(c->d_eband);
    dfree(c->d_rho_in);
    dfree(c->d_rho_out);
    dfree(c->d_err);
    dfree(c->d_hist);
    dfree(c->d_tune);
    dfree(c->d_kat);
    dfree(c->d_queue);
    sched_reset(c);
    if (c->d_pole) cudaFree(c->d_pole);
    c->d_pole = nullptr;
    c->pole_bytes = 0;
    c->tune_doubles = 0;
    c->ql_lanes.clear();
    c->ql_tune_ms.clear();
    c->hist_cap = 0;
    c->built = c->lnos_ready = c->solved = false;
}

extern "C" dclno_status dclno_create(dclno_ctx** out, void* cuda_stream) {
    if (!out) return DCLNO_ERR_ARG;
    *out = nullptr;
    dclno_ctx* c = new (std::nothrow) dclno_ctx();
    if (!c) return DCLNO_ERR_OOM;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess || c->nsm < 1) {
        delete c;
        return DCLNO_ERR_CUDA;
    }
    c->gpu_name = prop.name;
    for (char& ch : c->gpu_name)
        if (ch == ' ' || ch == '|') ch = '_';
    *out = c;
    return DCLNO_OK;
}

void prof_collect(dclno_ctx* c) {
    for (auto& kv : c->prof) {
        for (auto& ev : kv.second.pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(ev.second) == cudaSuccess && cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
                kv.second.ms += ms;
                kv.second.launches += 1;
            }
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
        kv.second.pending.clear();
    }
}

extern "C" void dclno_destroy(dclno_ctx* c) {
    if (!c) return;
    prof_collect(c);
    free_clusters(c);
    delete c;
}

extern "C" dclno_status dclno_set_profiling(dclno_ctx* c, int on) {
    if (!c) return DCLNO_ERR_ARG;
    prof_collect(c);
    c->prof.clear();
    c->prof_on = on != 0;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_kernel_time(dclno_ctx* c, const char* name, double* total_ms, long long* launches) {
    if (!c || !name) return DCLNO_ERR_ARG;
    prof_collect(c);
    auto it = c->prof.find(name);
    if (total_ms) *total_ms = it == c->prof.end() ? 0.0 : it->second.ms;
    if (launches) *launches = it == c->prof.end() ? 0 : it->second.launches;
    return DCLNO_OK;
}

extern "C" const char* dclno_last_error(const dclno_ctx* c) { return c ? c->err.c_str() : ""; }

extern "C" long long dclno_launch_count(const dclno_ctx* c) { return c ? c->launches : 0; }

// ---------------------------------------------------------------------------
// Cluster construction
// ---------------------------------------------------------------------------
namespace {

struct Cand {
    double d;
    int atom;
    int s0, s1, s2;
};

// images (j, R) within rmax of atom i: brute force over a cell list of image points
struct ImageGrid {
    std::vector<double> px, py, pz;
    std::vector<int> atom, s0, s1, s2;
    double lo[3], cw;
    int nc[3];
    std::vector<int> head, next;

    void build(const dclno_ctx* c, double rmax) {
        int nmax[3];
        for (int d = 0; d < 3; ++d) {
            if (!c->pbc[d]) {
                nmax[d] = 0;
                continue;
            }
            const double* a = &c->cell[3 * d];
            const double* e = &c->cell[3 * ((d + 1) % 3)];
            const double* f = &c->cell[3 * ((d + 2) % 3)];
            double cr[3] = {e[1] * f[2] - e[2] * f[1], e[2] * f[0] - e[0] * f[2], e[0] * f[1] - e[1] * f[0]};
            double area = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            double h = std::fabs(a[0] * cr[0] + a[1] * cr[1] + a[2] * cr[2]) / area;
            nmax[d] = (int)std::ceil(rmax / h) + 1;
        }
        for (int a = -nmax[0]; a <= nmax[0]; ++a)
            for (int b = -nmax[1]; b <= nmax[1]; ++b)
                for (int g = -nmax[2]; g <= nmax[2]; ++g)
                    for (int j = 0; j < c->N; ++j) {
                        double x[3];
                        for (int d = 0; d < 3; ++d)
                            x[d] = c->pos[3 * j + d] + (a * c->cell[d] + b * c->cell[3 + d] + g * c->cell[6 + d]);
                        px.push_back(x[0]);
                        py.push_back(x[1]);
                        pz.push_back(x[2]);
                        atom.push_back(j);
                        s0.push_back(a);
                        s1.push_back(b);
                        s2.push_back(g);
                    }
        double hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = 1e300;
            hi[d] = -1e300;
        }
        for (size_t k = 0; k < px.size(); ++k) {
            double x[3] = {px[k], py[k], pz[k]};
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], x[d]);
                hi[d] = std::max(hi[d], x[d]);
            }
        }
        cw = std::max(rmax, 1e-3);
        for (int d = 0; d < 3; ++d) nc[d] = std::max(1, (int)((hi[d] - lo[d]) / cw) + 1);
        head.assign((size_t)nc[0] * nc[1] * nc[2], -1);
        next.assign(px.size(), -1);
        for (size_t k = 0; k < px.size(); ++k) {
            int ci = cell_of(px[k], 0), cj = cell_of(py[k], 1), ck = cell_of(pz[k], 2);
            size_t h = ((size_t)ci * nc[1] + cj) * nc[2] + ck;
            next[k] = head[h];
            head[h] = (int)k;
        }
    }
    int cell_of(double x, int d) const {
        int v = (int)std::floor((x - lo[d]) / cw);
        return std::min(std::max(v, 0), nc[d] - 1);
    }
};

}  // namespace

static dclno_status copy_to_device(dclno_ctx* c, void** dst, const void* src, size_t bytes) {
    DCLNO_CUDA(c, cudaMalloc(dst, std::max<size_t>(bytes, 16)));
    if (bytes) DCLNO_CUDA(c, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return DCLNO_OK;
}

// largest |S| of every stored block (the first-neighbour test of the region rule)
__global__ void k_block_absmax(long long nnzb, const long long* __restrict__ off, const int* __restrict__ sz,
                               const double* __restrict__ S, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; b < nnzb;
         b += ((long long)gridDim.x * blockDim.x) >> 5) {
        double m = 0.0;
        for (int e = lane; e < sz[b]; e += 32) m = fmax(m, fabs(S[off[b] + e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) out[b] = m;
    }
}

static dclno_status block_absmax(dclno_ctx* c, const double* S, std::vector<double>& out) {
    std::vector<int> sz(c->nnzb);
    for (int i = 0; i < c->N; ++i)
        for (long long b = c->row_ptr[i]; b < c->row_ptr[i + 1]; ++b) sz[b] = c->norb[i] * c->norb[c->col[b]];
    long long* d_off = nullptr;
    int* d_sz = nullptr;
    double* d_out = nullptr;
    out.assign(c->nnzb, 0.0);
    cudaError_t e;
    if ((e = cudaMalloc(&d_off, sizeof(long long) * std::max<long long>(c->nnzb, 1))) == cudaSuccess &&
        (e = cudaMalloc(&d_sz, sizeof(int) * std::max<long long>(c->nnzb, 1))) == cudaSuccess &&
        (e = cudaMalloc(&d_out, sizeof(double) * std::max<long long>(c->nnzb, 1))) == cudaSuccess &&
        (e = cudaMemcpy(d_off, c->blk_off.data(), sizeof(long long) * c->nnzb, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemcpy(d_sz, sz.data(), sizeof(int) * c->nnzb, cudaMemcpyHostToDevice)) == cudaSuccess) {
        const int grid = (int)std::min<long long>((c->nnzb * 32 + 255) / 256, (long long)c->nsm * 64);
        k_block_absmax<<<std::max(grid, 1), 256, 0, c->stream>>>(c->nnzb, d_off, d_sz, S, d_out);
        c->launches++;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = cudaMemcpy(out.data(), d_out, sizeof(double) * c->nnzb, cudaMemcpyDeviceToHost);
    }
    if (d_off) cudaFree(d_off);
    if (d_sz) cudaFree(d_sz);
    if (d_out) cudaFree(d_out);
    if (e != cudaSuccess) return cuda_err(c, e, "overlap block maxima for the region rule");
    return DCLNO_OK;
}

// Short-range radius of the region rule (Sec. III (ii)-(iii)): the shell whose sphere
// holds a number of atoms closest to N_F + kappa N_S (ties: the larger sphere).  dd:
// member distances ascending; fna: the same members' first-neighbour flags.
static double kappa_radius(const std::vector<double>& dd, const std::vector<char>& fna, double kappa, double tol) {
    long long nf = 0;
    for (char f : fna) nf += f ? 1 : 0;
    const double target = (double)nf + kappa * (double)((long long)dd.size() - nf);
    double best_r = 0.0, best_gap = 1e300;
    long long best_cnt = -1;
    for (size_t k = 0; k < dd.size(); ++k) {
        if (k > 0 && dd[k] == dd[k - 1]) continue;
        const long long cnt = std::upper_bound(dd.begin(), dd.end(), dd[k] + tol) - dd.begin();
        const double gap = std::fabs((double)cnt - target);
        if (gap < best_gap - 1e-12 || (std::fabs(gap - best_gap) <= 1e-12 && cnt > best_cnt)) {
            best_r = dd[k];
            best_gap = gap;
            best_cnt = cnt;
        }
    }
    return best_r;
}

// Tear positions of a cluster: once at n/2 (split) and, for a cluster torn twice, also at
// the middle of each half (split1, split3), by the context's tear mode.
static void set_tears(const dclno_ctx* c, ClusterDesc& d) {
    d.split2 = 0;
    d.split1 = d.split3 = 0;
    if (!d.split) return;
    const bool twice = c->tear_mode == 2 ? d.n >= DCLNO_TEAR_MIN : c->tear_mode == 0 ? d.n >= DCLNO_TEAR2_MIN : false;
    if (!twice) return;
    d.split2 = 1;
    d.split1 = d.split / 2;
    d.split3 = d.split + (d.n - d.split) / 2;
}

static long long longest_segment(const ClusterDesc& d) {
    if (!d.split) return d.n;
    if (!d.split2) return std::max(d.split, d.n - d.split);
    return std::max(std::max(d.split1, d.split - d.split1), std::max(d.split3 - d.split, d.n - d.split3));
}

// merge matrices and their transposes: the cluster's (2 n ld) and, torn twice, its halves' (2 n ld)
static long long merge_area(const ClusterDesc& d) { return d.split ? (d.split2 ? 4LL : 2LL) * d.n * d.ld : 0LL; }

// a cluster's own problem: status and W-block offsets
static void set_problem_offsets(ClusterDesc& d, int i) {
    const long long W = d.aux_off + 3LL * d.ld;
    d.sidx = i;
    d.g_row0 = 0;
    d.x2_mode = 0;
    d.w_off = W;
    d.gb_off = W;
    d.scr_off = W;
    d.x2_off = W + w_row(d.ld, DCLNO_W_X2);
}

// The two half problems of a cluster torn twice (n = 0 otherwise), in the cluster's
// workspace: d, e from the half's first row, its strips' rows, the second pair of its
// four segments' rotation logs and sweep headers for the second half, its merge matrix
// after the cluster's; its z row and the rows its QL carries in the cluster's W block.
static void make_halves(dclno_ctx* c, int i) {
    const ClusterDesc& d = c->cl[i];
    for (int h = 0; h < 2; ++h) {
        ClusterDesc& e = c->clh[2 * (size_t)i + h];
        e = ClusterDesc{};
        e.sidx = i;
        e.q2_off = -1;
        if (!d.split2) continue;
        const int r0 = h ? d.split : 0;
        const long long W = d.aux_off + 3LL * d.ld;
        e.centre = d.centre;
        e.n = h ? d.n - d.split : d.split;
        e.ld = d.ld;
        e.nmem = d.nmem;
        e.mbeg = d.mbeg;
        e.mat_off = d.mat_off;
        e.eig_off = d.eig_off + r0;
        e.cc_off = d.cc_off + (long long)r0 * 2 * d.mc;
        e.rot_off = d.rot_off + 2LL * h * 2 * d.rot_cap;  // two segments' logs of 2 doubles per rotation
        e.it_off = d.it_off + 2LL * h * d.it_cap;
        e.aux_off = d.aux_off + r0;
        e.rot_cap = d.rot_cap;
        e.it_cap = d.it_cap;
        e.mc = d.mc;
        e.split = (h ? d.split3 : d.split1) - r0;
        e.pair_off = d.pair_off;
        e.m_off = d.m_off + 2LL * d.n * d.ld + (h ? 2LL * d.split * d.ld : 0LL);
        e.g_row0 = r0;
        e.x2_mode = h ? 1 : 2;
        e.w_off = W + w_row(d.ld, h ? DCLNO_W_HALF1 : DCLNO_W_HALF0);
        e.gb_off = W;
        e.scr_off = W + (h ? 16LL * d.ld : 0LL);  // each half's strips' scratch: at most 13 ld
        e.x2_off = W + w_row(d.ld, DCLNO_W_X2);
    }
}

// per batch, in its decreasing-n order: the two-segment problems (a cluster torn at most
// once, or both halves of one torn twice) and the clusters torn twice
static void build_problem_lists(dclno_ctx* c) {
    c->l1.clear();
    c->l2.clear();
    for (Batch& b : c->batches) {
        b.l1beg = (int)c->l1.size();
        b.l2beg = (int)c->l2.size();
        b.segmax = 1;
        b.l1maxn = 1;
        for (int o = b.obeg; o < b.oend; ++o) {
            const int i = c->order[o];
            const ClusterDesc& d = c->cl[i];
            if (d.split2) {
                for (int h = 0; h < 2; ++h) {
                    const ClusterDesc& e = c->clh[2 * (size_t)i + h];
                    c->l1.push_back(c->N + 2 * i + h);
                    b.segmax = std::max(b.segmax, std::max(seg_len(e, 0), seg_len(e, 1)));
                    b.l1maxn = std::max(b.l1maxn, e.n);
                }
                c->l2.push_back(i);
            } else {
                c->l1.push_back(i);
                b.segmax = std::max(b.segmax, std::max(seg_len(d, 0), seg_len(d, 1)));
                b.l1maxn = std::max(b.l1maxn, d.n);
            }
        }
        b.l1end = (int)c->l1.size();
        b.l2end = (int)c->l2.size();
    }
}

static dclno_status build_impl(dclno_ctx* c, const dclno_system* sys, double r_core, double r_lno, int k_lno,
                               double kappa, double s_fna) {
    const bool rule = kappa >= 0.0;
    DCLNO_CUDA(c, cudaSetDevice(c->device));
    free_clusters(c);
    const bool pao_only = k_lno == 0 || (!rule && r_lno <= r_core);  // plain PAO DC: no LNO region

    const int N = sys->natoms;
    c->N = N;
    c->nnzb = sys->nnzb;
    c->nval = sys->nval;
    c->max_row = 0;
    c->norb.assign(sys->norb, sys->norb + N);
    c->row_ptr.assign(sys->row_ptr, sys->row_ptr + N + 1);
    c->col.assign(sys->col, sys->col + sys->nnzb);
    c->blk_off.assign(sys->blk_off, sys->blk_off + sys->nnzb);
    c->pos.assign(sys->pos, sys->pos + 3 * N);
    c->cell.assign(sys->cell, sys->cell + 9);
    for (int d = 0; d < 3; ++d) c->pbc[d] = sys->pbc[d] ? 1 : 0;
    c->H = sys->H;
    c->S = sys->S;
    c->r_core = r_core;
    c->r_lno = r_lno;
    c->k_lno = k_lno;

    // ---- validate the structure
    if (c->row_ptr[0] != 0 || c->row_ptr[N] != c->nnzb)
        return set_err(c, DCLNO_ERR_ARG, "row_ptr must start at 0 and end at nnzb");
    for (int i = 0; i < N; ++i) {
        if (c->norb[i] < 1 || c->norb[i] > DCLNO_MAX_M)
            return set_err(c, DCLNO_ERR_ARG, "norb must lie in 1..32 (atom " + std::to_string(i) + ")");
        if (c->row_ptr[i + 1] < c->row_ptr[i]) return set_err(c, DCLNO_ERR_ARG, "row_ptr not monotone");
    }
    c->pshift.resize(c->nnzb);
    std::vector<long long> key(c->nnzb), onsite(N, -1);
    for (int i = 0; i < N; ++i) {
        for (long long b = c->row_ptr[i]; b < c->row_ptr[i + 1]; ++b) {
            int j = c->col[b];
            if (j < 0 || j >= N) return set_err(c, DCLNO_ERR_ARG, "column index out of range");
            int s0 = sys->shift[3 * b], s1 = sys->shift[3 * b + 1], s2 = sys->shift[3 * b + 2];
            c->pshift[b] = pack_shift(s0, s1, s2);
            key[b] = block_key(j, c->pshift[b]);
            if (b > c->row_ptr[i] && key[b] <= key[b - 1])
                return set_err(c, DCLNO_ERR_ARG, "BSR rows must be sorted by (col, shift) without duplicates");
            long long sz = (long long)c->norb[i] * c->norb[j];
            if (c->blk_off[b] < 0 || c->blk_off[b] + sz > c->nval)
                return set_err(c, DCLNO_ERR_ARG, "block offset out of range");
            if (j == i && s0 == 0 && s1 == 0 && s2 == 0) onsite[i] = b;
        }
        if (onsite[i] < 0) return set_err(c, DCLNO_ERR_ARG, "missing on-site block of atom " + std::to_string(i));
        c->max_row = std::max(c->max_row, c->row_ptr[i + 1] - c->row_ptr[i]);
        if (!pao_only && (k_lno > c->norb[i] || c->norb[i] > DCLNO_MAX_M_LNO))
            return set_err(c, DCLNO_ERR_ARG, "atom " + std::to_string(i) + ": LNOs need k_lno <= M_i <= 16");
    }

    std::vector<double> bmax;
    if (rule) {
        const dclno_status st = block_absmax(c, sys->S, bmax);
        if (st != DCLNO_OK) return st;
    }

    // ---- clusters: membership by distance, order by distance descending (centre last)
    ImageGrid g;
    g.build(c, r_lno);
    const double tol = 1e-9;
    c->cl.resize(N);
    c->mem.clear();
    std::vector<int> rowblk_member(c->nnzb, -1);
    std::vector<int> mem_cl;
    c->has_lno_region = false;
    long long eig = 0, pairs = 0;
    for (int i = 0; i < N; ++i) {
        const double xi = c->pos[3 * i], yi = c->pos[3 * i + 1], zi = c->pos[3 * i + 2];
        std::vector<Cand> cand;
        int ci = g.cell_of(xi, 0), cj = g.cell_of(yi, 1), ck = g.cell_of(zi, 2);
        for (int a = std::max(ci - 1, 0); a <= std::min(ci + 1, g.nc[0] - 1); ++a)
            for (int b = std::max(cj - 1, 0); b <= std::min(cj + 1, g.nc[1] - 1); ++b)
                for (int q = std::max(ck - 1, 0); q <= std::min(ck + 1, g.nc[2] - 1); ++q)
                    for (int k = g.head[((size_t)a * g.nc[1] + b) * g.nc[2] + q]; k >= 0; k = g.next[k]) {
                        double dx = g.px[k] - xi, dy = g.py[k] - yi, dz = g.pz[k] - zi;
                        double d = std::sqrt(dx * dx + dy * dy + dz * dz);
                        if (d <= r_lno + tol) cand.push_back({d, g.atom[k], g.s0[k], g.s1[k], g.s2[k]});
                    }
        std::sort(cand.begin(), cand.end(), [](const Cand& u, const Cand& v) {
            if (u.d != v.d) return u.d > v.d;
            if (u.atom != v.atom) return u.atom < v.atom;
            if (u.s0 != v.s0) return u.s0 < v.s0;
            if (u.s1 != v.s1) return u.s1 < v.s1;
            return u.s2 < v.s2;
        });
        if (cand.empty() || cand.back().atom != i || cand.back().s0 || cand.back().s1 || cand.back().s2)
            return set_err(c, DCLNO_ERR_ARG, "cluster of atom " + std::to_string(i) + " does not end with its centre");
        double r_short = r_core;
        if (rule && !pao_only) {
            // first neighbouring atoms: stored overlap block with the centre above s_fna
            std::vector<double> dd(cand.size());
            std::vector<char> fna(cand.size());
            const auto kb = key.begin() + c->row_ptr[i], ke = key.begin() + c->row_ptr[i + 1];
            for (size_t m = 0; m < cand.size(); ++m) {
                const Cand& u = cand[cand.size() - 1 - m];  // ascending distance
                dd[m] = u.d;
                const long long want = block_key(u.atom, pack_shift(u.s0, u.s1, u.s2));
                const auto it = std::lower_bound(kb, ke, want);
                fna[m] = (it != ke && *it == want && bmax[it - key.begin()] > s_fna) ? 1 : 0;
            }
            r_short = kappa_radius(dd, fna, kappa, tol);
        }
        ClusterDesc& d = c->cl[i];
        d.centre = i;
        d.nmem = (int)cand.size();
        d.mbeg = (long long)c->mem.size();
        int off = 0;
        std::vector<std::pair<long long, int>> keys;
        keys.reserve(cand.size());
        for (size_t m = 0; m < cand.size(); ++m) {
            const Cand& u = cand[m];
            int core = (u.d <= r_short + tol) ? 1 : 0;
            if (pao_only) core = 1;
            if (!core) c->has_lno_region = true;
            MemberDesc md;
            md.atom = u.atom;
            md.shift = pack_shift(u.s0, u.s1, u.s2);
            md.off = off;
            md.core = core;
            off += core ? c->norb[u.atom] : k_lno;
            c->mem.push_back(md);
            mem_cl.push_back(i);
            keys.push_back({block_key(u.atom, md.shift), (int)m});
        }
        d.n = off;
        d.ld = (off + 3) & ~3;
        d.mc = c->norb[i];
        std::sort(keys.begin(), keys.end());
        for (long long b = c->row_ptr[i]; b < c->row_ptr[i + 1]; ++b) {
            auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(key[b], -1));
            if (it != keys.end() && it->first == key[b]) rowblk_member[b] = it->second;
        }
        d.split = d.n >= DCLNO_TEAR_MIN ? d.n / 2 : 0;
        set_tears(c, d);
        const long long sm = longest_segment(d);
        d.rot_cap = (int)std::min<long long>(3 * sm * sm / 2 + 64 * sm + 64, 2000000000LL);
        d.it_cap = (int)(24 * sm + 64);
        d.eig_off = eig;
        eig += d.n;
        d.pair_off = pairs;
        pairs += (long long)d.nmem * d.nmem;
    }
    c->total_dim = eig;
    c->pair_total = pairs;
    // LNO-transformed copies of every stored block: V_j1^T X, X V_j2, V_j1^T X V_j2 for X = H, S
    std::vector<long long> tblk_off(c->nnzb, 0), brow(c->nnzb);
    long long tb = 0;
    for (int i = 0; i < N; ++i)
        for (long long b = c->row_ptr[i]; b < c->row_ptr[i + 1]; ++b) {
            brow[b] = i;
            tblk_off[b] = tb;
            if (c->has_lno_region) {
                const long long m1 = c->norb[i], m2 = c->norb[c->col[b]], k = k_lno;
                tb += 2 * (k * m2 + m1 * k + k * k);
            }
        }
    c->tblk_total = tb;
    std::vector<int> brow32(brow.begin(), brow.end());

    // ---- memory admission: per-cluster workspace (doubles): A, L (n x ld each), d/e/tau (ld each),
    // W (32 ld), P ([n][2 mc]), rotation logs (2 rot_cap per segment), for a torn problem the merge
    // matrix and its transpose (n x ld each); 256-byte aligned.  Sweep headers: it_cap ints per segment.
    auto nseg = [](const ClusterDesc& d) { return d.split2 ? 4LL : d.split ? 2LL : 1LL; };
    c->layout_tear = c->tear_mode;
    // the two-stage reduction's chase reflectors (kept until the density rows are written),
    // laid out only when the context is in two-stage mode; it also borrows the merge-matrix
    // area as scratch, so only torn clusters qualify
    c->layout_mode = c->tridiag_mode;
    const int qmin = c->layout_mode == 2 ? DCLNO_TWO_STAGE_MIN : c->layout_mode == 0 ? DCLNO_TWO_STAGE_AUTO_MIN : 1 << 30;
    auto q2_doubles = [qmin](const ClusterDesc& d) {
        return (d.split && d.n >= qmin) ? (long long)DCLNO_BW * band_refl_count(d.n) : 0LL;
    };
    auto ws_doubles = [&](const ClusterDesc& d) {
        const long long m = 2LL * d.n * d.ld + 35LL * d.ld + 2LL * d.mc * d.ld + 2LL * d.rot_cap * nseg(d) +
                            merge_area(d) + ((q2_doubles(d) + 3) & ~3LL);
        return (m + 31) & ~31LL;
    };
    auto ws_bytes = [&](const ClusterDesc& d) { return 8 * ws_doubles(d) + 4LL * d.it_cap * nseg(d); };
    size_t free_b = 0, tot_b = 0;
    DCLNO_CUDA(c, cudaMemGetInfo(&free_b, &tot_b));
    long long msum_all = 0;
    for (int i = 0; i < N; ++i) msum_all += c->norb[i];
    const size_t other = (size_t)c->total_dim * 16 + (size_t)c->nnzb * 48 + (size_t)c->pair_total * 4 +
                         (size_t)c->tblk_total * 8 + (size_t)msum_all * (8 * k_lno + 16 + 8 * DCLNO_MAX_M) +
                         (size_t)N * 64 + c->mem.size() * 24;
    const size_t reserve = (size_t)(1u << 30) + 2 * (size_t)c->nval * sizeof(double);  // host-buffer / SCF rho copies
    long long budget;
    if (c->ws_limit) budget = (long long)c->ws_limit;
    else budget = free_b > other + reserve ? (long long)(free_b - other - reserve) : 0;
    long long total_ws = 0, max_ws = 0;
    for (int i = 0; i < N; ++i) {
        total_ws += ws_bytes(c->cl[i]);
        max_ws = std::max(max_ws, ws_bytes(c->cl[i]));
    }
    if (max_ws > budget)
        return set_err(c, DCLNO_ERR_OOM, "the workspace of one cluster (" + std::to_string(max_ws >> 20) +
                                             " MiB) exceeds the workspace budget (" + std::to_string(budget >> 20) +
                                             " MiB)");
    const long long nb_min = (total_ws + budget - 1) / budget;
    const long long target = (total_ws + nb_min - 1) / nb_min;
    c->batches.clear();
    {
        Batch cur;
        long long acc = 0;
        for (int i = 0; i < N; ++i) {
            const long long w = ws_bytes(c->cl[i]);
            if (acc > 0 && acc + w > budget) {
                cur.id_hi = i;
                c->batches.push_back(cur);
                cur = Batch();
                cur.id_lo = i;
                acc = 0;
            }
            acc += w;
            if (acc >= target && i + 1 < N) {
                cur.id_hi = i + 1;
                c->batches.push_back(cur);
                cur = Batch();
                cur.id_lo = i + 1;
                acc = 0;
            }
        }
        cur.id_hi = N;
        if (cur.id_hi > cur.id_lo) c->batches.push_back(cur);
    }
    // offsets relative to the batch; order = each batch's clusters by decreasing n
    c->order.resize(N);
    long long arena_max = 0, its_max = 0;
    for (Batch& b : c->batches) {
        long long mat = 0, its = 0;
        b.maxn = 0;
        b.mcmax = 1;
        for (int i = b.id_lo; i < b.id_hi; ++i) {
            ClusterDesc& d = c->cl[i];
            d.mat_off = mat;
            d.aux_off = mat + 2LL * d.n * d.ld;  // d, e, tau, W: each sub-region starts on a multiple of 4 doubles
            d.cc_off = d.aux_off + 35LL * d.ld;
            d.rot_off = d.cc_off + 2LL * d.mc * d.ld;
            d.m_off = d.rot_off + 2LL * d.rot_cap * nseg(d);
            d.q2_off = q2_doubles(d) ? d.m_off + merge_area(d) : -1;
            set_problem_offsets(d, i);
            mat += ws_doubles(d);
            d.it_off = its;
            its += (long long)d.it_cap * nseg(d);
            b.maxn = std::max(b.maxn, d.n);
            b.mcmax = std::max(b.mcmax, d.mc);
        }
        b.arena_doubles = mat;
        b.iters = its;
        arena_max = std::max(arena_max, mat);
        its_max = std::max(its_max, its);
        b.obeg = b.id_lo;
        b.oend = b.id_hi;
        std::iota(c->order.begin() + b.obeg, c->order.begin() + b.oend, b.id_lo);
        std::stable_sort(c->order.begin() + b.obeg, c->order.begin() + b.oend,
                         [&](int x, int y) { return c->cl[x].n > c->cl[y].n; });
        b.mbeg = c->cl[b.id_lo].mbeg;
        b.mend = b.id_hi < N ? c->cl[b.id_hi].mbeg : (long long)c->mem.size();
        build_buckets(c, b);
    }
    c->clh.assign(2 * (size_t)N, ClusterDesc{});
    for (int i = 0; i < N; ++i) make_halves(c, i);
    build_problem_lists(c);
    c->arena_doubles = (size_t)arena_max;
    c->resident = -1;
    for (size_t k = 0; k < c->batches.size(); ++k) c->batches[k].index = (int)k;
    c->ql_lanes.assign(c->batches.size(), 0);
    c->ql_tune_ms.assign(c->batches.size() * DCLNO_QL_CANDIDATES, -1.0f);

    // ---- LNO storage offsets
    std::vector<long long> voff(N + 1), loff(N + 1), moff(N + 1);
    voff[0] = loff[0] = moff[0] = 0;
    for (int i = 0; i < N; ++i) {
        voff[i + 1] = voff[i] + (long long)c->norb[i] * k_lno;
        loff[i + 1] = loff[i] + (long long)c->norb[i] * c->norb[i];
        moff[i + 1] = moff[i] + c->norb[i];
    }
    c->v_total = voff[N];
    c->l_total = loff[N];

    // ---- device memory
    const size_t need = c->arena_doubles * 8 + (size_t)its_max * 4 + other;
    if (need + (size_t)(1u << 30) > free_b) {
        free_clusters(c);
        return set_err(c, DCLNO_ERR_OOM,
                       "workspace of " + std::to_string(need >> 20) + " MiB does not fit in free device memory");
    }
    dclno_status st;
#define COPY(dst, vec)                                                                        \
    st = copy_to_device(c, (void**)&(dst), (vec).data(), (vec).size() * sizeof((vec)[0]));   \
    if (st != DCLNO_OK) {                                                                     \
        free_clusters(c);                                                                     \
        return st;                                                                            \
    }
    COPY(c->d_norb, c->norb);
    COPY(c->d_row_ptr, c->row_ptr);
    COPY(c->d_key, key);
    COPY(c->d_blk_off, c->blk_off);
    COPY(c->d_onsite, onsite);
    COPY(c->d_voff, voff);
    COPY(c->d_loff, loff);
    COPY(c->d_moff, moff);
    {
        std::vector<ClusterDesc> all(c->cl);
        all.insert(all.end(), c->clh.begin(), c->clh.end());
        COPY(c->d_cl, all);
    }
    COPY(c->d_l1, c->l1);
    COPY(c->d_l2, c->l2.empty() ? std::vector<int>{0} : c->l2);
    COPY(c->d_order, c->order);
    COPY(c->d_mem, c->mem);
    COPY(c->d_mem_cl, mem_cl);
    COPY(c->d_brow, brow32);
    COPY(c->d_tblk_off, tblk_off);
    COPY(c->d_rowblk_member, rowblk_member);
    c->kat.assign(N, k_lno);
    COPY(c->d_kat, c->kat);
    c->layout_split.resize(N);
    c->layout_split2.resize(N);
    for (int i = 0; i < N; ++i) {
        c->layout_split[i] = c->cl[i].split ? 1 : 0;
        c->layout_split2[i] = c->cl[i].split2 ? 1 : 0;
    }
#undef COPY
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_status, sizeof(int) * N)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_arena, c->arena_doubles * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_iters, sizeof(int) * std::max<long long>(its_max, 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_eps, sizeof(double) * c->total_dim)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_q, sizeof(double) * c->total_dim)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_V, sizeof(double) * std::max<long long>(c->v_total, 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_lam_re, sizeof(double) * moff[N])) != cudaSuccess ||
        (e = cudaMalloc(&c->d_lam_im, sizeof(double) * moff[N])) != cudaSuccess ||
        (e = cudaMalloc(&c->d_Lambda, sizeof(double) * std::max<long long>(loff[N], 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_lflags, sizeof(int) * N)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_eband, sizeof(double) * N)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_scalars, sizeof(double) * 64)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_mu_work, sizeof(double) * 4096 * 8)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_queue, sizeof(int) * 64)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_pairblk, sizeof(int) * std::max<long long>(c->pair_total, 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_tblk, sizeof(double) * std::max<long long>(c->tblk_total, 1))) != cudaSuccess) {
        free_clusters(c);
        return cuda_err(c, e, "cudaMalloc (cluster workspace)");
    }
    st = launch_pair_index(c);
    if (st == DCLNO_OK && c->has_lno_region) st = prepare_lno_kernels(c);
    if (st != DCLNO_OK) {
        free_clusters(c);
        return st;
    }
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    c->built = true;
    c->lnos_ready = !c->has_lno_region;
    return DCLNO_OK;
}

static dclno_status check_system(dclno_ctx* c, const dclno_system* sys, const char* who) {
    if (!sys || sys->natoms <= 0 || !sys->pos || !sys->cell || !sys->pbc || !sys->norb || !sys->row_ptr ||
        !sys->col || !sys->shift || !sys->blk_off || !sys->H || !sys->S)
        return set_err(c, DCLNO_ERR_ARG, std::string(who) + ": null or empty system");
    return DCLNO_OK;
}

extern "C" dclno_status dclno_build_clusters(dclno_ctx* c, const dclno_system* sys, double r_core,
                                             double r_lno, int k_lno) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    dclno_status st = check_system(c, sys, "dclno_build_clusters");
    if (st != DCLNO_OK) return st;
    if (!(r_core >= 0.0) || !(r_lno >= r_core) || k_lno < 0)
        return set_err(c, DCLNO_ERR_ARG, "dclno_build_clusters: need 0 <= r_core <= r_lno and k_lno >= 0");
    return build_impl(c, sys, r_core, r_lno, k_lno, -1.0, 0.0);
}

extern "C" dclno_status dclno_build_clusters_kappa(dclno_ctx* c, const dclno_system* sys, double r_lno, int k_lno,
                                                   double kappa, double s_fna) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    dclno_status st = check_system(c, sys, "dclno_build_clusters_kappa");
    if (st != DCLNO_OK) return st;
    if (!(r_lno >= 0.0) || k_lno < 0 || !(kappa >= 0.0 && kappa <= 1.0) || !(s_fna >= 0.0))
        return set_err(c, DCLNO_ERR_ARG, "dclno_build_clusters_kappa: need r_lno >= 0, k_lno >= 0, 0 <= kappa <= 1, s_fna >= 0");
    return build_impl(c, sys, 0.0, r_lno, k_lno, kappa, s_fna);
}

// Cluster dimensions after a threshold selection of LNOs: member sizes M_j (short
// range) or the atom's own LNO count; the workspace keeps the layout made for
// k_lno, every new dimension being at most the laid-out one.
dclno_status relayout_clusters(dclno_ctx* c) {
    DCLNO_CUDA(c, cudaMemcpyAsync(c->kat.data(), c->d_kat, sizeof(int) * c->N, cudaMemcpyDeviceToHost, c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    long long eig = 0;
    for (int i = 0; i < c->N; ++i) {
        ClusterDesc& d = c->cl[i];
        int off = 0;
        for (int m = 0; m < d.nmem; ++m) {
            MemberDesc& md = c->mem[d.mbeg + m];
            md.off = off;
            off += md.core ? c->norb[md.atom] : c->kat[md.atom];
        }
        if (off > d.ld) return set_err(c, DCLNO_ERR_ARG, "LNO counts exceed the laid-out cluster dimension");
        d.n = off;
        // keep tearing where the layout tore: the segment logs were sized for its segments
        d.split = (c->layout_split[i] && off >= 2) ? off / 2 : 0;
        d.split2 = 0;
        d.split1 = d.split3 = 0;
        if (c->layout_split2[i]) {
            if (off < 4) return set_err(c, DCLNO_ERR_ARG, "LNO counts leave a cluster torn twice too small");
            d.split2 = 1;
            d.split1 = d.split / 2;
            d.split3 = d.split + (off - d.split) / 2;
        }
        d.eig_off = eig;
        eig += off;
    }
    c->total_dim = eig;
    for (Batch& b : c->batches) {
        b.maxn = 0;
        for (int i = b.id_lo; i < b.id_hi; ++i) b.maxn = std::max(b.maxn, c->cl[i].n);
    }
    for (int i = 0; i < c->N; ++i) make_halves(c, i);
    build_problem_lists(c);
    std::vector<ClusterDesc> all(c->cl);
    all.insert(all.end(), c->clh.begin(), c->clh.end());
    DCLNO_CUDA(c, cudaMemcpyAsync(c->d_cl, all.data(), sizeof(ClusterDesc) * all.size(), cudaMemcpyHostToDevice,
                                  c->stream));
    DCLNO_CUDA(c, cudaMemcpyAsync(c->d_mem, c->mem.data(), sizeof(MemberDesc) * c->mem.size(),
                                  cudaMemcpyHostToDevice, c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    c->resident = -1;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_lno_threshold(dclno_ctx* c, int on, double lambda_th) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (on && !(lambda_th == lambda_th)) return set_err(c, DCLNO_ERR_ARG, "dclno_set_lno_threshold: lambda_th is NaN");
    c->lno_th_on = on != 0;
    c->lno_th = lambda_th;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_lno_mode(dclno_ctx* c, dclno_lno_mode mode) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (mode != DCLNO_LNO_PAPER && mode != DCLNO_LNO_SYM)
        return set_err(c, DCLNO_ERR_ARG, "dclno_set_lno_mode: unknown mode " + std::to_string((int)mode));
    c->lno_mode = (int)mode;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_get_lno_counts(dclno_ctx* c, int* counts) {
    if (!c) return DCLNO_ERR_ARG;
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_get_lno_counts: build clusters first");
    if (counts) std::copy(c->kat.begin(), c->kat.end(), counts);
    return DCLNO_OK;
}

extern "C" dclno_status dclno_compute_lnos(dclno_ctx* c, const double* rho) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_compute_lnos: build clusters first");
    if (!c->has_lno_region) {
        c->lnos_ready = true;
        return DCLNO_OK;
    }
    if (!rho) return set_err(c, DCLNO_ERR_ARG, "dclno_compute_lnos: rho is NULL");
    const bool counted = c->lno_th_on || c->relaid;  // the layout follows the counts of these LNOs
    const bool th = c->lno_th_on;
    dclno_status st = launch_lambda_lno(c, rho);
    if (st == DCLNO_OK && counted && !th) st = relayout_clusters(c);  // back to k_lno for every atom
    c->relaid = th;
    if (st != DCLNO_OK) return st;
    c->lnos_ready = true;
    c->solved = false;
    return DCLNO_OK;
}

// assemble and solve one batch; its workspace becomes the resident one
static dclno_status solve_batch(dclno_ctx* c, int bi, dclno_precision prec) {
    const Batch& b = c->batches[bi];
    c->resident = -1;
    dclno_status st = launch_assemble(c, b);
    if (st == DCLNO_OK) st = (prec == DCLNO_MIXED) ? launch_solve_mixed(c, b) : launch_solve_fp64(c, b);
    if (st == DCLNO_OK) c->resident = bi;
    return st;
}

// The tridiagonalisation form of a solve: mode 1 one-stage, 2 two-stage; the automatic
// mode (0) takes the form measured faster on the 1,728-atom step in each precision:
// one-stage in FP64 (2.6 against 3.3 s per step), two-stage in the mixed path (1.1
// against 1.4 s, its bulge chasing in double-float arithmetic).
// Whether the solve may use the two-stage form; which clusters do is fixed by the layout
// (a cluster takes it when its workspace holds a chase-reflector log).  Mode 0: the mixed
// path only (FP64 two-stage is slower on GB300, whose FP64 tile products barely beat its
// FP64 vector rate); mode 2: both paths.
static bool resolve_two_stage(const dclno_ctx* c, dclno_precision prec) {
    if (c->tridiag_mode == 2) return c->layout_mode == 2;
    return c->tridiag_mode == 0 && prec == DCLNO_MIXED;
}

// every batch: assemble + solve (eps and q of all clusters)
static dclno_status solve_all(dclno_ctx* c, dclno_precision prec) {
    c->solved_two = resolve_two_stage(c, prec);
    dclno_status st = launch_lno_blocks(c);
    for (int bi = 0; st == DCLNO_OK && bi < (int)c->batches.size(); ++bi) st = solve_batch(c, bi, prec);
    if (st == DCLNO_OK) c->solved_prec = prec;
    return st;
}

// density rows of every batch, the resident one first; the others are solved again
// (the same kernels on the same inputs give the same eps, q and workspace)
static dclno_status density_all(dclno_ctx* c, double mu, double kT, double* rho_out, double* e_out) {
    const int nb = (int)c->batches.size();
    const int r0 = c->resident >= 0 ? c->resident : 0;
    dclno_status st = DCLNO_OK;
    for (int k = 0; st == DCLNO_OK && k < nb; ++k) {
        const int bi = (r0 + k) % nb;
        if (bi != c->resident) st = solve_batch(c, bi, c->solved_prec);
        if (st == DCLNO_OK) st = launch_density(c, c->batches[bi], mu, kT, rho_out, e_out);
    }
    return st;
}

static dclno_status read_eband(dclno_ctx* c, double* eband_out) {
    if (!eband_out) return DCLNO_OK;
    std::vector<double> eb(c->N);
    DCLNO_CUDA(c, cudaMemcpyAsync(eb.data(), c->d_eband, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    double s = 0.0;
    for (int i = 0; i < c->N; ++i) s += eb[i];
    *eband_out = s;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_solve_clusters(dclno_ctx* c, dclno_precision prec) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_solve_clusters: build clusters first");
    if (!c->lnos_ready) return set_err(c, DCLNO_ERR_NO_LNOS, "dclno_solve_clusters: compute LNOs first");
    if (prec != DCLNO_FP64 && prec != DCLNO_MIXED)
        return set_err(c, DCLNO_ERR_ARG, "dclno_solve_clusters: unknown precision");
    c->solved = false;
    dclno_status st = solve_all(c, prec);
    if (st != DCLNO_OK) return st;
    c->solved = true;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_find_mu(dclno_ctx* c, double ne, double kT, double* mu_out, double* nelec_out) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->solved) return set_err(c, DCLNO_ERR_ARG, "dclno_find_mu: solve clusters first");
    if (!(kT > 0.0)) return set_err(c, DCLNO_ERR_ARG, "dclno_find_mu: kT must be positive");
    double mu = 0, nmu = 0;
    dclno_status st = launch_find_mu(c, ne, kT, &mu, &nmu);
    if (mu_out) *mu_out = mu;
    if (nelec_out) *nelec_out = nmu;
    return st;
}

extern "C" dclno_status dclno_density_matrix(dclno_ctx* c, double mu, double kT, double* rho_out,
                                             double* eband_out) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->solved) return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrix: solve clusters first");
    if (!(kT > 0.0) || !rho_out) return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrix: bad kT or rho_out");
    dclno_status st = density_all(c, mu, kT, rho_out, nullptr);
    if (st != DCLNO_OK) return st;
    return read_eband(c, eband_out);
}

extern "C" dclno_status dclno_density_matrices(dclno_ctx* c, double mu, double kT, double* rho_out, double* edm_out,
                                               double* eband_out) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->solved) return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrices: solve clusters first");
    if (!(kT > 0.0) || !rho_out) return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrices: bad kT or rho_out");
    if (edm_out)
        for (const auto& d : c->cl)
            if (2 * d.mc > 32)
                return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrices: the energy density matrix needs M_i <= 16");
    dclno_status st = density_all(c, mu, kT, rho_out, edm_out);
    if (st != DCLNO_OK) return st;
    return read_eband(c, eband_out);
}

// statuses of a batch after a launch sequence (host synchronisation)
static dclno_status check_batch_status(dclno_ctx* c, const Batch& b, const char* who) {
    const int nid = b.id_hi - b.id_lo;
    std::vector<int> st(nid);
    DCLNO_CUDA(c, cudaMemcpyAsync(st.data(), c->d_status + b.id_lo, sizeof(int) * nid, cudaMemcpyDeviceToHost,
                                  c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nid; ++k) {
        const int i = b.id_lo + k;
        if (st[k] == ST_OK) continue;
        const std::string id = std::string(who) + ": cluster " + std::to_string(i);
        if (st[k] == ST_NOT_SPD) return set_err(c, DCLNO_ERR_NOT_SPD, id + ": overlap not positive definite");
        if (st[k] == ST_TIMEOUT) return set_err(c, DCLNO_ERR_TIMEOUT, id + ": a tensor-core wait ran out");
        if (st[k] == ST_FEW_POLES)
            return set_err(c, DCLNO_ERR_ARG, id + ": too few poles (the first omitted pole is below three times the "
                                                  "spectral radius of the cluster about mu)");
        return set_err(c, DCLNO_ERR_NOT_CONVERGED, id + ": status " + std::to_string(st[k]));
    }
    return DCLNO_OK;
}

extern "C" dclno_status dclno_density_matrix_poles(dclno_ctx* c, double mu, double kT, int n_poles,
                                                   dclno_precision prec, double* rho_out) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrix_poles: build clusters first");
    if (!c->lnos_ready) return set_err(c, DCLNO_ERR_NO_LNOS, "dclno_density_matrix_poles: compute LNOs first");
    if (!(kT > 0.0) || n_poles < 1 || !rho_out || !(mu == mu))
        return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrix_poles: need kT > 0, n_poles >= 1, rho_out");
    if (prec != DCLNO_FP64 && prec != DCLNO_MIXED)
        return set_err(c, DCLNO_ERR_ARG, "dclno_density_matrix_poles: unknown precision");
    // the reduction overwrites the workspace of any earlier solve
    c->solved = false;
    c->resident = -1;
    c->solved_two = resolve_two_stage(c, prec);
    c->solved_prec = prec;
    dclno_status st = launch_lno_blocks(c);
    for (int bi = 0; st == DCLNO_OK && bi < (int)c->batches.size(); ++bi) {
        const Batch& b = c->batches[bi];
        st = launch_assemble(c, b);
        if (st == DCLNO_OK)
            st = (prec == DCLNO_MIXED) ? launch_solve_mixed(c, b, true) : launch_solve_fp64(c, b, true);
        if (st == DCLNO_OK) st = launch_poles(c, b, mu, kT, n_poles);
        if (st == DCLNO_OK) st = check_batch_status(c, b, "dclno_density_matrix_poles");
        if (st == DCLNO_OK) st = launch_density(c, b, mu, kT, rho_out, nullptr, true);
    }
    if (st == DCLNO_OK) DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    return st;
}

extern "C" dclno_status dclno_set_workspace_limit(dclno_ctx* c, size_t bytes) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    c->ws_limit = bytes;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_tridiag(dclno_ctx* c, int mode) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (mode < 0 || mode > 2) return set_err(c, DCLNO_ERR_ARG, "dclno_set_tridiag: mode must be 0, 1 or 2");
    if (mode == 2 && c->built && c->layout_mode != 2)
        return set_err(c, DCLNO_ERR_ARG,
                       "dclno_set_tridiag: the two-stage form keeps its chase reflectors in the cluster workspace, "
                       "laid out by dclno_build_clusters: select mode 2 before building the clusters");
    c->tridiag_mode = mode;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_tear(dclno_ctx* c, int mode) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (mode < 0 || mode > 2) return set_err(c, DCLNO_ERR_ARG, "dclno_set_tear: mode must be 0, 1 or 2");
    if (c->built && mode != c->layout_tear)
        return set_err(c, DCLNO_ERR_ARG,
                       "dclno_set_tear: the segments' logs and merge matrices are laid out by dclno_build_clusters: "
                       "select the tear mode before building the clusters");
    c->tear_mode = mode;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_mixed_engine(dclno_ctx* c, int engine) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (engine < 0 || engine > 2) return set_err(c, DCLNO_ERR_ARG, "dclno_set_mixed_engine: engine must be 0, 1 or 2");
    c->mixed_engine = engine;
    sched_reset(c);
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_autotune(dclno_ctx* c, int on) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    c->autotune = on != 0;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_get_tuning(dclno_ctx* c, int batch, int* ql_lanes, float* candidate_ms) {
    if (!c) return DCLNO_ERR_ARG;
    if (!c->built || batch < 0 || batch >= (int)c->batches.size())
        return set_err(c, DCLNO_ERR_ARG, "dclno_get_tuning: build clusters first; batch out of range");
    if (ql_lanes) *ql_lanes = c->ql_lanes[batch];
    if (candidate_ms)
        for (int k = 0; k < DCLNO_QL_CANDIDATES; ++k) candidate_ms[k] = c->ql_tune_ms[batch * DCLNO_QL_CANDIDATES + k];
    return DCLNO_OK;
}

extern "C" dclno_status dclno_batch_info(dclno_ctx* c, int* nbatches, size_t* workspace_bytes) {
    if (!c) return DCLNO_ERR_ARG;
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_batch_info: build clusters first");
    if (nbatches) *nbatches = (int)c->batches.size();
    if (workspace_bytes) *workspace_bytes = c->arena_doubles * sizeof(double);
    return DCLNO_OK;
}

extern "C" dclno_status dclno_step(dclno_ctx* c, const double* rho_in, double* rho_out, int host_buffers,
                                   dclno_precision prec, double ne, double kT, double* mu_out,
                                   double* nelec_out, double* eband_out) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_step: build clusters first");
    if (!rho_out || (!rho_in && c->has_lno_region)) return set_err(c, DCLNO_ERR_ARG, "dclno_step: null rho");
    const double* rin = rho_in;
    double* rout = rho_out;
    const size_t bytes = (size_t)c->nval * sizeof(double);
    if (host_buffers) {
        if (!c->d_rho_in) DCLNO_CUDA(c, cudaMalloc(&c->d_rho_in, bytes));
        if (!c->d_rho_out) DCLNO_CUDA(c, cudaMalloc(&c->d_rho_out, bytes));
        if (rho_in) DCLNO_CUDA(c, cudaMemcpyAsync(c->d_rho_in, rho_in, bytes, cudaMemcpyHostToDevice, c->stream));
        rin = c->d_rho_in;
        rout = c->d_rho_out;
    }
    dclno_status st = dclno_compute_lnos(c, rin);
    if (st == DCLNO_OK) st = dclno_solve_clusters(c, prec);
    double mu = 0;
    if (st == DCLNO_OK) st = dclno_find_mu(c, ne, kT, &mu, nelec_out);
    if (st == DCLNO_OK) st = dclno_density_matrix(c, mu, kT, rout, eband_out);
    if (st != DCLNO_OK) return st;
    if (mu_out) *mu_out = mu;
    if (host_buffers) {
        DCLNO_CUDA(c, cudaMemcpyAsync(rho_out, rout, bytes, cudaMemcpyDeviceToHost, c->stream));
        DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return DCLNO_OK;
}

extern "C" dclno_status dclno_cluster_info(dclno_ctx* c, int* dims, int* nmem, long long* total) {
    if (!c) return DCLNO_ERR_ARG;
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_cluster_info: build clusters first");
    for (int i = 0; i < c->N; ++i) {
        if (dims) dims[i] = c->cl[i].n;
        if (nmem) nmem[i] = c->cl[i].nmem;
    }
    if (total) *total = c->total_dim;
    return DCLNO_OK;
}

extern "C" dclno_status dclno_get_spectrum(dclno_ctx* c, double* eps, double* q) {
    if (!c) return DCLNO_ERR_ARG;
    if (!c->solved) return set_err(c, DCLNO_ERR_ARG, "dclno_get_spectrum: solve clusters first");
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    if (eps) DCLNO_CUDA(c, cudaMemcpy(eps, c->d_eps, sizeof(double) * c->total_dim, cudaMemcpyDeviceToHost));
    if (q) DCLNO_CUDA(c, cudaMemcpy(q, c->d_q, sizeof(double) * c->total_dim, cudaMemcpyDeviceToHost));
    return DCLNO_OK;
}

extern "C" dclno_status dclno_get_lnos(dclno_ctx* c, double* V, double* lre, double* lim, int* flags) {
    if (!c) return DCLNO_ERR_ARG;
    if (!c->built || !c->has_lno_region || !c->lnos_ready)
        return set_err(c, DCLNO_ERR_ARG, "dclno_get_lnos: no LNOs computed");
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    long long msum = 0;
    for (int i = 0; i < c->N; ++i) msum += c->norb[i];
    if (V) DCLNO_CUDA(c, cudaMemcpy(V, c->d_V, sizeof(double) * c->v_total, cudaMemcpyDeviceToHost));
    if (lre) DCLNO_CUDA(c, cudaMemcpy(lre, c->d_lam_re, sizeof(double) * msum, cudaMemcpyDeviceToHost));
    if (lim) DCLNO_CUDA(c, cudaMemcpy(lim, c->d_lam_im, sizeof(double) * msum, cudaMemcpyDeviceToHost));
    if (flags) DCLNO_CUDA(c, cudaMemcpy(flags, c->d_lflags, sizeof(int) * c->N, cudaMemcpyDeviceToHost));
    return DCLNO_OK;
}

// ---------------------------------------------------------------------------
// SCF loop: nsteps of (DC-LNO step, linear mixing), optionally as one CUDA graph
// ---------------------------------------------------------------------------
static dclno_status scf_one_step(dclno_ctx* c, double* rho, double alpha, dclno_precision prec, double ne, double kT) {
    dclno_status st = DCLNO_OK;
    if (c->has_lno_region) st = launch_lambda_lno(c, rho);
    if (st == DCLNO_OK) st = solve_all(c, prec);
    double mu = 0.0, nmu = 0.0;
    if (st == DCLNO_OK) st = launch_find_mu(c, ne, kT, &mu, &nmu);
    if (st == DCLNO_OK) st = density_all(c, 0.0, kT, c->d_rho_out, nullptr);
    if (st == DCLNO_OK) st = launch_scf_tail(c, rho, c->d_rho_out, alpha);
    return st;
}

extern "C" dclno_status dclno_scf_run(dclno_ctx* c, double* rho, int nsteps, double alpha, dclno_precision prec,
                                      double ne, double kT, int use_graph, double* mu_hist, double* nelec_hist,
                                      double* eband_hist) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (!c->built) return set_err(c, DCLNO_ERR_ARG, "dclno_scf_run: build clusters first");
    if (!rho || nsteps < 1 || !(kT > 0.0) || !(alpha > 0.0 && alpha <= 1.0))
        return set_err(c, DCLNO_ERR_ARG, "dclno_scf_run: need rho, nsteps >= 1, kT > 0, 0 < alpha <= 1");
    if (prec != DCLNO_FP64 && prec != DCLNO_MIXED) return set_err(c, DCLNO_ERR_ARG, "dclno_scf_run: unknown precision");
    if (c->lno_th_on && c->has_lno_region)
        return set_err(c, DCLNO_ERR_ARG, "dclno_scf_run: threshold-selected LNOs change the cluster dimensions every "
                                         "step (a host re-layout); loop over dclno_step instead");
    if (use_graph && c->stream == nullptr)
        return set_err(c, DCLNO_ERR_ARG, "dclno_scf_run: graph capture needs a context on a non-default stream");
    const size_t bytes = (size_t)c->nval * sizeof(double);
    if (!c->d_rho_out) DCLNO_CUDA(c, cudaMalloc(&c->d_rho_out, bytes));
    if (!c->d_err) DCLNO_CUDA(c, cudaMalloc(&c->d_err, 2 * sizeof(int)));
    if (c->hist_cap < nsteps) {
        if (c->d_hist) cudaFree(c->d_hist);
        c->d_hist = nullptr;
        c->hist_cap = 0;
        DCLNO_CUDA(c, cudaMalloc(&c->d_hist, 3 * sizeof(double) * nsteps));
        c->hist_cap = nsteps;
    }
    DCLNO_CUDA(c, cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int), c->stream));
    const bool prof = c->prof_on;
    c->prof_on = false;
    c->deferred = true;
    dclno_status st = DCLNO_OK;
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const long long l0 = c->launches;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) st = cuda_err(c, e, "cudaStreamBeginCapture");
        if (st == DCLNO_OK) {
            st = scf_one_step(c, rho, alpha, prec, ne, kT);
            e = cudaStreamEndCapture(c->stream, &graph);
            if (st == DCLNO_OK && e != cudaSuccess) st = cuda_err(c, e, "cudaStreamEndCapture");
        }
        if (st == DCLNO_OK) {
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) st = cuda_err(c, e, "cudaGraphInstantiate");
        }
        const long long per_step = c->launches - l0;
        for (int k = 0; st == DCLNO_OK && k < nsteps; ++k) {
            e = cudaGraphLaunch(exec, c->stream);
            if (e != cudaSuccess) st = cuda_err(c, e, "cudaGraphLaunch");
        }
        if (st == DCLNO_OK) {
            e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) st = cuda_err(c, e, "cudaStreamSynchronize");
        }
        c->launches += per_step * (nsteps - 1);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    } else {
        for (int k = 0; st == DCLNO_OK && k < nsteps; ++k) st = scf_one_step(c, rho, alpha, prec, ne, kT);
    }
    c->deferred = false;
    c->prof_on = prof;
    if (st != DCLNO_OK) return st;
    int err[2] = {0, 0};
    std::vector<double> hist(3 * (size_t)nsteps);
    DCLNO_CUDA(c, cudaMemcpyAsync(err, c->d_err, sizeof(err), cudaMemcpyDeviceToHost, c->stream));
    DCLNO_CUDA(c, cudaMemcpyAsync(hist.data(), c->d_hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost,
                                  c->stream));
    DCLNO_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nsteps; ++k) {
        if (mu_hist) mu_hist[k] = hist[3 * k];
        if (nelec_hist) nelec_hist[k] = hist[3 * k + 1];
        if (eband_hist) eband_hist[k] = hist[3 * k + 2];
    }
    c->solved = true;
    c->lnos_ready = true;
    if (err[0] == 16) return set_err(c, DCLNO_ERR_NO_BRACKET, "dclno_scf_run: N_e outside the bracket of N(mu)");
    if (err[0] == ST_NOT_SPD) return set_err(c, DCLNO_ERR_NOT_SPD, "dclno_scf_run: a cluster overlap is not positive definite");
    if (err[0] == ST_TIMEOUT) return set_err(c, DCLNO_ERR_TIMEOUT, "dclno_scf_run: a tensor-core wait ran out");
    if (err[0] != 0) return set_err(c, DCLNO_ERR_NOT_CONVERGED, "dclno_scf_run: an eigensolver failed (status " + std::to_string(err[0]) + ")");
    return DCLNO_OK;
}
