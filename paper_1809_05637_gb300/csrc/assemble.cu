// Cluster matrices in the mixed PAO/LNO basis (Eq. (Hi)), all clusters at once.
//
// For members m1 = (j1, R1) and m2 = (j2, R2) of cluster i, the pair block is the
// stored block X_{0 j1, (R2-R1) j2} (X = H, S; zero if absent) seen through the
// members' bases B = I (PAO member) or V_j (LNO member):
//     X^(i)[m1, m2] = B_m1^T X_{0 j1,(R2-R1) j2} B_m2.
// One CTA per (cluster, m1); its warps walk m2, one pair block per warp.
#include "dclno_internal.cuh"

__global__ void __launch_bounds__(128) k_assemble(const ClusterDesc* __restrict__ cls,
                                                  const MemberDesc* __restrict__ mem,
                                                  const int* __restrict__ mem_cl, const int* __restrict__ norb,
                                                  const long long* __restrict__ row_ptr,
                                                  const long long* __restrict__ key,
                                                  const long long* __restrict__ blk_off,
                                                  const long long* __restrict__ voff, int k,
                                                  const double* __restrict__ H, const double* __restrict__ S,
                                                  const double* __restrict__ V, double* __restrict__ arena) {
    const long long g1 = blockIdx.x;
    const int ci = mem_cl[g1];
    const ClusterDesc d = cls[ci];
    const MemberDesc a = mem[g1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j1 = a.atom, M1 = norb[j1];
    const int n1 = a.core ? M1 : k;
    int s10, s11, s12;
    unpack_shift(a.shift, s10, s11, s12);
    double* Hc = arena + d.mat_off;
    double* Sc = Hc + (size_t)d.n * d.ld;
    const int ld = d.ld;
    const double* V1 = a.core ? nullptr : V + voff[j1];
    const long long rb = row_ptr[j1], re = row_ptr[j1 + 1];
    for (int m2 = warp; m2 < d.nmem; m2 += nw) {
        const MemberDesc b = mem[d.mbeg + m2];
        const int j2 = b.atom, M2 = norb[j2];
        const int n2 = b.core ? M2 : k;
        int s20, s21, s22;
        unpack_shift(b.shift, s20, s21, s22);
        const int r0 = s20 - s10, r1 = s21 - s11, r2 = s22 - s12;
        long long blk = -1;
        if (r0 >= -128 && r0 <= 127 && r1 >= -128 && r1 <= 127 && r2 >= -128 && r2 <= 127) {
            const long long want = block_key(j2, pack_shift(r0, r1, r2));
            long long lo = rb, hi = re;  // lower_bound over the sorted row
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (key[mid] < want) lo = mid + 1;
                else hi = mid;
            }
            if (lo < re && key[lo] == want) blk = lo;
        }
        const double* V2 = b.core ? nullptr : V + voff[j2];
        const double* Hb = blk >= 0 ? H + blk_off[blk] : nullptr;
        const double* Sb = blk >= 0 ? S + blk_off[blk] : nullptr;
        for (int e = lane; e < n1 * n2; e += 32) {
            const int p = e / n2, q = e % n2;
            double h = 0.0, s = 0.0;
            if (blk >= 0) {
                if (a.core && b.core) {
                    h = Hb[p * M2 + q];
                    s = Sb[p * M2 + q];
                } else if (a.core) {  // X V2
                    for (int t = 0; t < M2; ++t) {
                        const double v = V2[t * k + q];
                        h = fma(Hb[p * M2 + t], v, h);
                        s = fma(Sb[p * M2 + t], v, s);
                    }
                } else if (b.core) {  // V1^T X
                    for (int t = 0; t < M1; ++t) {
                        const double v = V1[t * k + p];
                        h = fma(v, Hb[t * M2 + q], h);
                        s = fma(v, Sb[t * M2 + q], s);
                    }
                } else {  // V1^T X V2
                    for (int t = 0; t < M1; ++t) {
                        double ht = 0.0, st = 0.0;
                        for (int u = 0; u < M2; ++u) {
                            const double v = V2[u * k + q];
                            ht = fma(Hb[t * M2 + u], v, ht);
                            st = fma(Sb[t * M2 + u], v, st);
                        }
                        const double w = V1[t * k + p];
                        h = fma(w, ht, h);
                        s = fma(w, st, s);
                    }
                }
            }
            const size_t o = (size_t)(a.off + p) * ld + b.off + q;
            Hc[o] = h;
            Sc[o] = s;
        }
    }
}

dclno_status launch_assemble(dclno_ctx* c) {
    const long long nm = (long long)c->mem.size();
    if (nm > 2147483647LL) return set_err(c, DCLNO_ERR_ARG, "too many cluster members");
    {
        ProfScope ps__(c, "k_assemble");
        k_assemble<<<(unsigned)nm, 128, 0, c->stream>>>(c->d_cl, c->d_mem, c->d_mem_cl, c->d_norb, c->d_row_ptr,
                                                    c->d_key, c->d_blk_off, c->d_voff, c->k_lno, c->H, c->S,
                                                    c->d_V, c->d_arena);
    }
    DCLNO_LAUNCHED(c);
    return DCLNO_OK;
}
