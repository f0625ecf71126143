// Cluster matrices in the mixed PAO/LNO basis (Eq. (Hi)), all clusters at once.
//
// For members m1 = (j1, R1) and m2 = (j2, R2) of cluster i, the pair block is the
// stored block X_{0 j1, (R2-R1) j2} (X = H, S; zero if absent) seen through the
// members' bases B = I (PAO member) or V_j (LNO member):
//     X^(i)[m1, m2] = B_m1^T X_{0 j1,(R2-R1) j2} B_m2.
// A stored block enters many clusters, so its LNO-transformed forms V_j1^T X,
// X V_j2 and V_j1^T X V_j2 are formed once per step (k_lno_blocks) and the
// assembly itself is a gather (k_assemble) through a member-pair -> block table
// built once with the clusters (k_pair_index).
#include "dclno_internal.cuh"

// block of row j1 holding (j2, shift): lower_bound over the sorted row, -1 if absent
__device__ __forceinline__ long long find_block(const long long* __restrict__ key, long long rb, long long re,
                                                int j2, int r0, int r1, int r2) {
    if (r0 < -128 || r0 > 127 || r1 < -128 || r1 > 127 || r2 < -128 || r2 > 127) return -1;
    const long long want = block_key(j2, pack_shift(r0, r1, r2));
    long long lo = rb, hi = re;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (key[mid] < want) lo = mid + 1;
        else hi = mid;
    }
    return (lo < re && key[lo] == want) ? lo : -1;
}

// member-pair -> block table; one CTA per (cluster, m1), warps over m2
__global__ void __launch_bounds__(128) k_pair_index(const ClusterDesc* __restrict__ cls,
                                                    const MemberDesc* __restrict__ mem,
                                                    const int* __restrict__ mem_cl,
                                                    const long long* __restrict__ row_ptr,
                                                    const long long* __restrict__ key, int* __restrict__ pairblk) {
    const long long g1 = blockIdx.x;
    const ClusterDesc d = cls[mem_cl[g1]];
    const MemberDesc a = mem[g1];
    const int m1 = (int)(g1 - d.mbeg);
    int s10, s11, s12;
    unpack_shift(a.shift, s10, s11, s12);
    const long long rb = row_ptr[a.atom], re = row_ptr[a.atom + 1];
    int* out = pairblk + d.pair_off + (long long)m1 * d.nmem;
    for (int m2 = threadIdx.x; m2 < d.nmem; m2 += blockDim.x) {
        const MemberDesc b = mem[d.mbeg + m2];
        int s20, s21, s22;
        unpack_shift(b.shift, s20, s21, s22);
        out[m2] = (int)find_block(key, rb, re, b.atom, s20 - s10, s21 - s11, s22 - s12);
    }
}

// Per stored block b (rows of atom j1, columns of atom j2) and X = H, S:
//   LP = V_j1^T X (k x M2), PL = X V_j2 (M1 x k), LL = V_j1^T X V_j2 = V_j1^T PL (k x k),
// stored at tblk + tblk_off[b] as [LP_H | LP_S | PL_H | PL_S | LL_H | LL_S].
// One warp per block: LP and PL elements over the lanes, then LL from the PL just
// written (a warp's FP64 instruction costs the same whatever its active lanes, so
// the work is spread evenly instead of recomputing X V_j2 inside every LL element).
__global__ void k_lno_blocks(long long nnzb, int k, const int* __restrict__ brow, const long long* __restrict__ key,
                             const int* __restrict__ norb, const long long* __restrict__ blk_off,
                             const long long* __restrict__ voff, const long long* __restrict__ tblk_off,
                             const double* __restrict__ H, const double* __restrict__ S,
                             const double* __restrict__ V, double* __restrict__ tblk) {
    const int lane = threadIdx.x & 31;
    for (long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; b < nnzb;
         b += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int j1 = brow[b], j2 = (int)(key[b] >> 24);
        const int M1 = norb[j1], M2 = norb[j2];
        const double* V1 = V + voff[j1];
        const double* V2 = V + voff[j2];
        const double* Xh = H + blk_off[b];
        const double* Xs = S + blk_off[b];
        double* out = tblk + tblk_off[b];
        const int nlp = k * M2, npl = M1 * k, nll = k * k;
        double* PLh = out + 2 * nlp;
        double* PLs = PLh + npl;
        for (int e = lane; e < nlp + npl; e += 32) {
            double h = 0.0, s = 0.0;
            if (e < nlp) {
                const int p = e / M2, q = e % M2;
                for (int t = 0; t < M1; ++t) {
                    const double v = V1[t * k + p];
                    h = fma(v, Xh[t * M2 + q], h);
                    s = fma(v, Xs[t * M2 + q], s);
                }
                out[e] = h;
                out[nlp + e] = s;
            } else {
                const int f = e - nlp, p = f / k, q = f % k;
                for (int t = 0; t < M2; ++t) {
                    const double v = V2[t * k + q];
                    h = fma(Xh[p * M2 + t], v, h);
                    s = fma(Xs[p * M2 + t], v, s);
                }
                PLh[f] = h;
                PLs[f] = s;
            }
        }
        __syncwarp();
        for (int f = lane; f < nll; f += 32) {
            const int p = f / k, q = f % k;
            double h = 0.0, s = 0.0;
            for (int t = 0; t < M1; ++t) {
                const double w = V1[t * k + p];
                h = fma(w, PLh[t * k + q], h);
                s = fma(w, PLs[t * k + q], s);
            }
            out[2 * nlp + 2 * npl + f] = h;
            out[2 * nlp + 2 * npl + nll + f] = s;
        }
        __syncwarp();
    }
}

// gather: one CTA per (cluster, m1) of the batch's members from mbeg, warps over m2,
// lanes over the block's elements
__global__ void __launch_bounds__(128) k_assemble(long long mbeg, const ClusterDesc* __restrict__ cls,
                                                  const MemberDesc* __restrict__ mem,
                                                  const int* __restrict__ mem_cl, const int* __restrict__ norb,
                                                  const int* __restrict__ kat,
                                                  const int* __restrict__ pairblk,
                                                  const long long* __restrict__ blk_off,
                                                  const long long* __restrict__ tblk_off, int k,
                                                  const double* __restrict__ H, const double* __restrict__ S,
                                                  const double* __restrict__ tblk, double* __restrict__ arena) {
    const long long g1 = mbeg + blockIdx.x;
    const ClusterDesc d = cls[mem_cl[g1]];
    const MemberDesc a = mem[g1];
    const int m1 = (int)(g1 - d.mbeg);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int M1 = norb[a.atom];
    const int n1 = a.core ? M1 : kat[a.atom];  // an LNO member's own count (<= k)
    double* Hc = arena + d.mat_off;
    double* Sc = Hc + (size_t)d.n * d.ld;
    const int ld = d.ld;
    const int* prow = pairblk + d.pair_off + (long long)m1 * d.nmem;
    for (int m2 = warp; m2 < d.nmem; m2 += nw) {
        const MemberDesc b = mem[d.mbeg + m2];
        const int M2 = norb[b.atom];
        const int n2 = b.core ? M2 : kat[b.atom];
        const int lds = b.core ? M2 : k;  // row length of the source block (LNO blocks are laid out for k)
        const long long blk = prow[m2];
        const double *sh = nullptr, *ss = nullptr;
        if (blk >= 0) {
            if (a.core && b.core) {
                sh = H + blk_off[blk];
                ss = S + blk_off[blk];
            } else {
                const double* t = tblk + tblk_off[blk];
                const int nlp = k * M2, npl = M1 * k, nll = k * k;
                if (!a.core && b.core) {  // V1^T X
                    sh = t;
                    ss = t + nlp;
                } else if (a.core) {  // X V2
                    sh = t + 2 * nlp;
                    ss = t + 2 * nlp + npl;
                } else {  // V1^T X V2
                    sh = t + 2 * nlp + 2 * npl;
                    ss = t + 2 * nlp + 2 * npl + nll;
                }
            }
        }
        for (int e = lane; e < n1 * n2; e += 32) {
            const int p = e / n2, q = e % n2;
            const size_t o = (size_t)(a.off + p) * ld + b.off + q;
            Hc[o] = sh ? sh[p * lds + q] : 0.0;
            Sc[o] = ss ? ss[p * lds + q] : 0.0;
        }
    }
}

dclno_status launch_pair_index(dclno_ctx* c) {
    const long long nm = (long long)c->mem.size();
    if (nm > 2147483647LL) return set_err(c, DCLNO_ERR_ARG, "too many cluster members");
    k_pair_index<<<(unsigned)nm, 128, 0, c->stream>>>(c->d_cl, c->d_mem, c->d_mem_cl, c->d_row_ptr, c->d_key,
                                                      c->d_pairblk);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

dclno_status launch_lno_blocks(dclno_ctx* c) {
    if (!c->has_lno_region) return DCLNO_OK;
    ProfScope ps__(c, "k_lno_blocks");
    const long long warps = c->nnzb;
    const int grid = (int)std::min<long long>((warps * 32 + 255) / 256, (long long)c->nsm * 64);
    k_lno_blocks<<<grid, 256, 0, c->stream>>>(c->nnzb, c->k_lno, c->d_brow, c->d_key, c->d_norb, c->d_blk_off,
                                              c->d_voff, c->d_tblk_off, c->H, c->S, c->d_V, c->d_tblk);
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}

dclno_status launch_assemble(dclno_ctx* c, const Batch& b) {
    const long long nm = b.mend - b.mbeg;
    if (nm > 2147483647LL) return set_err(c, DCLNO_ERR_ARG, "too many cluster members");
    if (nm == 0) return DCLNO_OK;
    {
        ProfScope ps__(c, "k_assemble");
        k_assemble<<<(unsigned)nm, 128, 0, c->stream>>>(b.mbeg, c->d_cl, c->d_mem, c->d_mem_cl, c->d_norb, c->d_kat,
                                                        c->d_pairblk, c->d_blk_off, c->d_tblk_off, c->k_lno, c->H,
                                                        c->S, c->d_tblk, c->d_arena);
    }
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}
