// Per-space preparation for sigma (the values of the [a,b] classes of Sec. II.C):
//  - string energies  E(S) = sum_{i in S} h_ii + 1/2 sum_{i,j in S} [(ii|jj) - (ij|ji)]
//    (the same-spin part of the stored [0,0] diagonal);
//  - single-link values  sign * [h_pq + sum_{k in J} ((pq|kk) - (pk|kq))]
//    (same-spin part of the [1,0] / [0,1] classes);
//  - double-link values  sign * [(pq|rs) - (ps|rq)]  ([2,0] / [0,2]);
//  - the beta Coulomb table U[pair(p,q)][Ib] = sum_{r in Ib} (pq|rr), which
//    carries the opposite-spin part of [1,0] and of the diagonal;
//  - schedules: beta columns ordered by their single-link count and alpha rows
//    by their work, both descending, so warps and CTAs get even work.
#include <algorithm>
#include <numeric>

#include "internal.cuh"

namespace tbsci {

namespace {

__device__ __forceinline__ double eri_at(const double *__restrict__ eri, int n, int i, int j, int k, int l) {
    return __ldg(eri + (((size_t)i * n + j) * n + k) * n + l);
}

__global__ void k_string_energy(const uint64_t *__restrict__ str, int64_t l, int n, const double *__restrict__ h,
                                const double *__restrict__ eri, double *E, float *Ef) {
    int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= l) return;
    uint64_t s = str[w];
    double e = 0.0;
    for (uint64_t a = s; a; a &= a - 1) {
        int i = __ffsll((long long)a) - 1;
        e += h[i * n + i];
        for (uint64_t b = s; b; b &= b - 1) {
            int j = __ffsll((long long)b) - 1;
            e += 0.5 * (eri_at(eri, n, i, i, j, j) - eri_at(eri, n, i, j, j, i));
        }
    }
    E[w] = e;
    Ef[w] = (float)e;
}

// one warp per source row; lanes over the row's single links
__global__ void k_single_values(const uint64_t *__restrict__ str, int64_t l, int n, const int64_t *__restrict__ off,
                                const tbsci_single_link *__restrict__ ent, const double *__restrict__ h,
                                const double *__restrict__ eri, int2 *sci, double *val, float *valf) {
    int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= l) return;
    uint64_t J = str[row];
    for (int64_t k = off[row] + lane; k < off[row + 1]; k += 32) {
        tbsci_single_link e = ent[k];
        int p = e.p, q = e.q;
        double v = h[p * n + q];
        for (uint64_t a = J; a; a &= a - 1) {
            int kk = __ffsll((long long)a) - 1;
            v += eri_at(eri, n, p, q, kk, kk) - eri_at(eri, n, p, kk, kk, q);
        }
        v *= (double)e.sign;
        int pr = p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
        sci[k] = make_int2(e.target, 2 * pr + (e.sign < 0 ? 1 : 0));
        val[k] = v;
        valf[k] = (float)v;
    }
}

__global__ void k_double_values(int64_t nd, int n, const tbsci_double_link *__restrict__ ent,
                                const double *__restrict__ eri, int32_t *col, double *val, float *valf) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nd) return;
    tbsci_double_link e = ent[k];
    double v = (double)e.sign * (eri_at(eri, n, e.p, e.q, e.r, e.s) - eri_at(eri, n, e.p, e.s, e.r, e.q));
    col[k] = e.target;
    val[k] = v;
    valf[k] = (float)v;
}

// U[pair][Ib] = sum_{r in occ(Ib)} V[pair][rr]
__global__ void k_coulomb_table(const uint64_t *__restrict__ strb, int64_t lb, int npair, const double *__restrict__ V,
                                double *U, float *Uf) {
    int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int pr = blockIdx.y;
    if (ib >= lb) return;
    uint64_t s = strb[ib];
    double u = 0.0;
    for (; s; s &= s - 1) {
        int r = __ffsll((long long)s) - 1;
        u += V[(size_t)pr * npair + r * (r + 1) / 2 + r];
    }
    U[(size_t)pr * lb + ib] = u;
    Uf[(size_t)pr * lb + ib] = (float)u;
}

// Sliced-ELL copy of CSR rows taken in the column order `perm` (see Plan).
__global__ void k_sell_singles(const int32_t *__restrict__ perm, int64_t lb, const int64_t *__restrict__ off,
                               const int2 *__restrict__ sci, const double *__restrict__ sval,
                               const int64_t *__restrict__ soff, const int32_t *__restrict__ sw, int64_t nsl,
                               int zero_idx, int2 *out_ci, double *out_val, float *out_valf) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nsl * 32) return;
    const int64_t sl = t >> 5, j = t;
    const int lane = (int)(t & 31);
    const int64_t ib = j < lb ? perm[j] : 0;
    const int64_t a = j < lb ? off[ib] : 0, cnt = j < lb ? off[ib + 1] - a : 0;
    const int64_t base = soff[sl] + lane;
    const int w = sw[sl];
    for (int k = 0; k < w; ++k) {
        const int64_t pos = base + 32 * (int64_t)k;
        if (k < cnt) {
            out_ci[pos] = sci[a + k];
            if (out_val) {
                out_val[pos] = sval[a + k];
                out_valf[pos] = (float)sval[a + k];
            }
        } else {
            out_ci[pos] = make_int2((int)ib, zero_idx);
            if (out_val) {
                out_val[pos] = 0.0;
                out_valf[pos] = 0.f;
            }
        }
    }
}

__global__ void k_sell_doubles(const int32_t *__restrict__ perm, int64_t lb, const int64_t *__restrict__ off,
                               const int32_t *__restrict__ dcol, const double *__restrict__ dval,
                               const int64_t *__restrict__ soff, const int32_t *__restrict__ sw, int64_t nsl,
                               int32_t *out_col, double *out_val, float *out_valf) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nsl * 32) return;
    const int64_t sl = t >> 5, j = t;
    const int lane = (int)(t & 31);
    const int64_t ib = j < lb ? perm[j] : 0;
    const int64_t a = j < lb ? off[ib] : 0, cnt = j < lb ? off[ib + 1] - a : 0;
    const int64_t base = soff[sl] + lane;
    const int w = sw[sl];
    for (int k = 0; k < w; ++k) {
        const int64_t pos = base + 32 * (int64_t)k;
        const bool real = k < cnt;
        out_col[pos] = real ? dcol[a + k] : (int32_t)ib;
        out_val[pos] = real ? dval[a + k] : 0.0;
        out_valf[pos] = real ? (float)dval[a + k] : 0.f;
    }
}

// out[pr][j] = in[pr][perm[j]] (rows of length lb)
__global__ void k_permute_cols(const double *__restrict__ in, int64_t rows, int64_t lb, const int32_t *__restrict__ perm,
                               double *out, float *outf) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (j >= lb || r >= rows) return;
    const double v = in[r * lb + perm[j]];
    out[r * lb + j] = v;
    outf[r * lb + j] = (float)v;
}

// LBP[Jb][off(p,q)] = (Ib << 1) | (sign < 0) for each single link Ib = a+_p a_q Jb
__global__ void k_link_by_pair(int64_t lb, const int64_t *__restrict__ off, const tbsci_single_link *__restrict__ ent,
                               int npoff, int32_t *lbp) {
    const int64_t jb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (jb >= lb) return;
    for (int64_t k = off[jb]; k < off[jb + 1]; ++k) {
        const tbsci_single_link e = ent[k];
        const int hi = e.p > e.q ? e.p : e.q, lo = e.p > e.q ? e.q : e.p;
        const int x = hi * (hi - 1) / 2 + lo;
        lbp[jb * npoff + x] = (e.target << 1) | (e.sign < 0 ? 1 : 0);
    }
}

// per-slice widths and offsets of a sliced-ELL layout over `perm`
void sell_shape(const std::vector<int32_t> &perm, const std::vector<int64_t> &off, std::vector<int64_t> &soff,
                std::vector<int32_t> &sw, int64_t &total) {
    const int64_t lb = (int64_t)perm.size(), nsl = (lb + 31) / 32;
    soff.assign(nsl, 0);
    sw.assign(nsl, 0);
    total = 0;
    for (int64_t sl = 0; sl < nsl; ++sl) {
        int64_t w = 0;
        for (int64_t j = sl * 32; j < std::min(lb, sl * 32 + 32); ++j) w = std::max(w, off[perm[j] + 1] - off[perm[j]]);
        soff[sl] = total;
        sw[sl] = (int32_t)w;
        total += 32 * w;
    }
}

tbsci_status build_spin(tbsci_ctx *ctx, const tbsci_ham *ham, const tbsci_tables *t, SpinPlan &sp, cudaStream_t st) {
    const int n = ham->norb;
    sp.l = t->count;
    sp.nelec = t->nelec;
    sp.d_str = t->d_str.p;
    sp.d_soff = t->d_off1.p;
    sp.d_doff = t->d_off2.p;
    sp.h_soff = t->h_off1;
    sp.h_doff = t->h_off2;
    TB_CUDA(ctx, sp.d_E.alloc(sp.l));
    TB_CUDA(ctx, sp.d_Ef.alloc(sp.l));
    TB_CUDA(ctx, sp.d_sci.alloc(t->nsingle));
    TB_CUDA(ctx, sp.d_sval.alloc(t->nsingle));
    TB_CUDA(ctx, sp.d_svalf.alloc(t->nsingle));
    TB_CUDA(ctx, sp.d_dcol.alloc(t->ndouble));
    TB_CUDA(ctx, sp.d_dval.alloc(t->ndouble));
    TB_CUDA(ctx, sp.d_dvalf.alloc(t->ndouble));
    const double *eri = ham->d_eri.p;
    if (sp.l > 0) {
        k_string_energy<<<(unsigned)((sp.l + 127) / 128), 128, 0, st>>>(sp.d_str, sp.l, n, ham->d_h.p, eri, sp.d_E.p,
                                                                       sp.d_Ef.p);
        TB_CUDA(ctx, cudaGetLastError());
        if (t->nsingle > 0) {
            k_single_values<<<(unsigned)((sp.l * 32 + 255) / 256), 256, 0, st>>>(
                sp.d_str, sp.l, n, t->d_off1.p, t->d_ent1.p, ham->d_h.p, eri, sp.d_sci.p, sp.d_sval.p, sp.d_svalf.p);
            TB_CUDA(ctx, cudaGetLastError());
        }
        if (t->ndouble > 0) {
            k_double_values<<<(unsigned)((t->ndouble + 255) / 256), 256, 0, st>>>(t->ndouble, n, t->d_ent2.p, eri,
                                                                                 sp.d_dcol.p, sp.d_dval.p,
                                                                                 sp.d_dvalf.p);
            TB_CUDA(ctx, cudaGetLastError());
        }
    }
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    return TBSCI_OK;
}

// device bytes a prepared space holds
size_t plan_device_bytes(const Plan &P) {
    size_t b = 0;
    for (const SpinPlan *sp : {&P.A, &P.B})
        b += sp->d_sci.bytes() + sp->d_sval.bytes() + sp->d_svalf.bytes() + sp->d_dcol.bytes() + sp->d_dval.bytes() +
             sp->d_dvalf.bytes() + sp->d_E.bytes() + sp->d_Ef.bytes();
    b += P.d_U.bytes() + P.d_Uf.bytes() + P.d_permb.bytes() + P.d_permb2.bytes();
    b += P.d_s1_off.bytes() + P.d_s2_off.bytes() + P.d_d2_off.bytes() + P.d_s1_w.bytes() + P.d_s2_w.bytes() +
         P.d_d2_w.bytes() + P.d_s1_ci.bytes() + P.d_s2_ci.bytes() + P.d_s2_val.bytes() + P.d_d2_val.bytes() +
         P.d_s2_valf.bytes() + P.d_d2_valf.bytes() + P.d_d2_col.bytes();
    b += P.d_U1.bytes() + P.d_U2.bytes() + P.d_Eb2.bytes() + P.d_U1f.bytes() + P.d_U2f.bytes() + P.d_Eb2f.bytes();
    b += P.d_rowsa.bytes() + P.d_pairs.bytes() + P.d_lbp.bytes() + P.d_offpair.bytes() + P.d_tc_err.bytes();
    return b;
}

}  // namespace

tbsci_status plan_get(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b, Plan **out) {
    TB_CHECK(ctx, ham && a && b, TBSCI_EINVAL, "null handle");
    for (auto &p : ham->plans)
        if (p->ida == a->id && p->idb == b->id) {
            *out = p.get();
            return TBSCI_OK;
        }
    TB_CHECK(ctx, a->norb == ham->norb && b->norb == ham->norb, TBSCI_EINVAL,
             "tables and Hamiltonian have different norb");
    TB_CHECK(ctx, a->flags == 0 && b->flags == 0, TBSCI_EINVAL,
             "sigma needs tables built with single and double links (flags = 0)");
    cudaStream_t st = ctx->stream;
    auto plan = std::make_unique<Plan>();
    plan->ida = a->id;
    plan->idb = b->id;
    plan->norb = ham->norb;
    plan->npair = ham->npair;
    TB_TRY(build_spin(ctx, ham, a, plan->A, st));
    TB_TRY(build_spin(ctx, ham, b, plan->B, st));
    const int64_t la = a->count, lb = b->count;
    TB_CUDA(ctx, plan->d_U.alloc((size_t)ham->npair * lb));
    TB_CUDA(ctx, plan->d_Uf.alloc((size_t)ham->npair * lb));
    if (lb > 0) {
        dim3 grid((unsigned)((lb + 127) / 128), (unsigned)ham->npair);
        k_coulomb_table<<<grid, 128, 0, st>>>(b->d_str.p, lb, ham->npair, ham->d_V.p, plan->d_U.p, plan->d_Uf.p);
        TB_CUDA(ctx, cudaGetLastError());
    }
    // schedules
    std::vector<int64_t> s1b(lb), idx_b(lb);
    int64_t S1b = 0, D2b = 0;
    for (int64_t i = 0; i < lb; ++i) {
        s1b[i] = b->h_off1[i + 1] - b->h_off1[i];
        S1b += s1b[i];
        D2b += b->h_off2[i + 1] - b->h_off2[i];
    }
    std::iota(idx_b.begin(), idx_b.end(), 0);
    std::stable_sort(idx_b.begin(), idx_b.end(), [&](int64_t x, int64_t y) { return s1b[x] > s1b[y]; });
    std::vector<int32_t> permb(idx_b.begin(), idx_b.end());
    std::vector<int64_t> tot_b(lb);
    for (int64_t i = 0; i < lb; ++i) tot_b[i] = s1b[i] + (b->h_off2[i + 1] - b->h_off2[i]);
    std::iota(idx_b.begin(), idx_b.end(), 0);
    std::stable_sort(idx_b.begin(), idx_b.end(), [&](int64_t x, int64_t y) { return tot_b[x] > tot_b[y]; });
    std::vector<int32_t> permb2(idx_b.begin(), idx_b.end());
    std::vector<double> work(la);
    std::vector<int64_t> idx_a(la);
    int64_t S1a = 0, D2a = 0;
    for (int64_t i = 0; i < la; ++i) {
        int64_t s1 = a->h_off1[i + 1] - a->h_off1[i];
        int64_t d2 = a->h_off2[i + 1] - a->h_off2[i];
        S1a += s1;
        D2a += d2;
        work[i] = (double)(1 + s1) * (double)(lb + S1b) + (double)d2 * (double)lb + (double)D2b;
    }
    std::iota(idx_a.begin(), idx_a.end(), 0);
    std::stable_sort(idx_a.begin(), idx_a.end(), [&](int64_t x, int64_t y) { return work[x] > work[y]; });
    std::vector<int32_t> rowsa(idx_a.begin(), idx_a.end());
    TB_CUDA(ctx, plan->d_permb.alloc(lb));
    TB_CUDA(ctx, plan->d_permb2.alloc(lb));
    if (lb > 0) TB_CUDA(ctx, cudaMemcpy(plan->d_permb2.p, permb2.data(), lb * sizeof(int32_t), cudaMemcpyHostToDevice));
    TB_CUDA(ctx, plan->d_rowsa.alloc(la));
    if (lb > 0) TB_CUDA(ctx, cudaMemcpy(plan->d_permb.p, permb.data(), lb * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (la > 0) TB_CUDA(ctx, cudaMemcpy(plan->d_rowsa.p, rowsa.data(), la * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (la > 0 && la % 2 == 0) {
        // even alpha row starts of row pairs (2k, 2k + 1), heaviest pair first: the
        // SIMT pass of the tensor-core sigma types may serve two rows per CTA
        std::vector<int64_t> pr(la / 2);
        std::iota(pr.begin(), pr.end(), 0);
        std::stable_sort(pr.begin(), pr.end(),
                         [&](int64_t x, int64_t y) { return work[2 * x] + work[2 * x + 1] > work[2 * y] + work[2 * y + 1]; });
        std::vector<int32_t> starts(la / 2);
        for (int64_t k = 0; k < la / 2; ++k) starts[k] = (int32_t)(2 * pr[k]);
        TB_CUDA(ctx, plan->d_pairs.alloc(la / 2));
        TB_CUDA(ctx, cudaMemcpy(plan->d_pairs.p, starts.data(), (la / 2) * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    // sliced-ELL beta links and column-permuted tables
    {
        const int64_t nsl = (lb + 31) / 32;
        std::vector<int64_t> so;
        std::vector<int32_t> sw;
        int64_t tot = 0;
        const unsigned g = (unsigned)std::max<int64_t>(1, (nsl * 32 + 255) / 256);
        const int zero_idx = 2 * ham->npair;
        // singles in permb order
        sell_shape(permb, b->h_off1, so, sw, tot);
        TB_CUDA(ctx, plan->d_s1_off.alloc(nsl));
        TB_CUDA(ctx, plan->d_s1_w.alloc(nsl));
        TB_CUDA(ctx, plan->d_s1_ci.alloc(std::max<int64_t>(tot, 1)));
        if (nsl > 0) {
            TB_CUDA(ctx, cudaMemcpy(plan->d_s1_off.p, so.data(), nsl * sizeof(int64_t), cudaMemcpyHostToDevice));
            TB_CUDA(ctx, cudaMemcpy(plan->d_s1_w.p, sw.data(), nsl * sizeof(int32_t), cudaMemcpyHostToDevice));
            k_sell_singles<<<g, 256, 0, st>>>(plan->d_permb.p, lb, b->d_off1.p, plan->B.d_sci.p, nullptr,
                                              plan->d_s1_off.p, plan->d_s1_w.p, nsl, zero_idx, plan->d_s1_ci.p,
                                              nullptr, nullptr);
            TB_CUDA(ctx, cudaGetLastError());
        }
        // singles with values in permb2 order
        sell_shape(permb2, b->h_off1, so, sw, tot);
        TB_CUDA(ctx, plan->d_s2_off.alloc(nsl));
        TB_CUDA(ctx, plan->d_s2_w.alloc(nsl));
        TB_CUDA(ctx, plan->d_s2_ci.alloc(std::max<int64_t>(tot, 1)));
        TB_CUDA(ctx, plan->d_s2_val.alloc(std::max<int64_t>(tot, 1)));
        TB_CUDA(ctx, plan->d_s2_valf.alloc(std::max<int64_t>(tot, 1)));
        if (nsl > 0) {
            TB_CUDA(ctx, cudaMemcpy(plan->d_s2_off.p, so.data(), nsl * sizeof(int64_t), cudaMemcpyHostToDevice));
            TB_CUDA(ctx, cudaMemcpy(plan->d_s2_w.p, sw.data(), nsl * sizeof(int32_t), cudaMemcpyHostToDevice));
            k_sell_singles<<<g, 256, 0, st>>>(plan->d_permb2.p, lb, b->d_off1.p, plan->B.d_sci.p, plan->B.d_sval.p,
                                              plan->d_s2_off.p, plan->d_s2_w.p, nsl, zero_idx, plan->d_s2_ci.p,
                                              plan->d_s2_val.p, plan->d_s2_valf.p);
            TB_CUDA(ctx, cudaGetLastError());
        }
        // doubles in permb2 order
        sell_shape(permb2, b->h_off2, so, sw, tot);
        TB_CUDA(ctx, plan->d_d2_off.alloc(nsl));
        TB_CUDA(ctx, plan->d_d2_w.alloc(nsl));
        TB_CUDA(ctx, plan->d_d2_col.alloc(std::max<int64_t>(tot, 1)));
        TB_CUDA(ctx, plan->d_d2_val.alloc(std::max<int64_t>(tot, 1)));
        TB_CUDA(ctx, plan->d_d2_valf.alloc(std::max<int64_t>(tot, 1)));
        if (nsl > 0) {
            TB_CUDA(ctx, cudaMemcpy(plan->d_d2_off.p, so.data(), nsl * sizeof(int64_t), cudaMemcpyHostToDevice));
            TB_CUDA(ctx, cudaMemcpy(plan->d_d2_w.p, sw.data(), nsl * sizeof(int32_t), cudaMemcpyHostToDevice));
            k_sell_doubles<<<g, 256, 0, st>>>(plan->d_permb2.p, lb, b->d_off2.p, plan->B.d_dcol.p, plan->B.d_dval.p,
                                              plan->d_d2_off.p, plan->d_d2_w.p, nsl, plan->d_d2_col.p,
                                              plan->d_d2_val.p, plan->d_d2_valf.p);
            TB_CUDA(ctx, cudaGetLastError());
        }
        const int64_t np = ham->npair;
        TB_CUDA(ctx, plan->d_U1.alloc(np * lb));
        TB_CUDA(ctx, plan->d_U1f.alloc(np * lb));
        TB_CUDA(ctx, plan->d_U2.alloc(np * lb));
        TB_CUDA(ctx, plan->d_U2f.alloc(np * lb));
        TB_CUDA(ctx, plan->d_Eb2.alloc(lb));
        TB_CUDA(ctx, plan->d_Eb2f.alloc(lb));
        if (lb > 0) {
            dim3 gu((unsigned)((lb + 127) / 128), (unsigned)np);
            k_permute_cols<<<gu, 128, 0, st>>>(plan->d_U.p, np, lb, plan->d_permb.p, plan->d_U1.p, plan->d_U1f.p);
            k_permute_cols<<<gu, 128, 0, st>>>(plan->d_U.p, np, lb, plan->d_permb2.p, plan->d_U2.p, plan->d_U2f.p);
            dim3 ge((unsigned)((lb + 127) / 128), 1);
            k_permute_cols<<<ge, 128, 0, st>>>(plan->B.d_E.p, 1, lb, plan->d_permb2.p, plan->d_Eb2.p, plan->d_Eb2f.p);
            TB_CUDA(ctx, cudaGetLastError());
        }
    }
    // tensor-core alpha-beta tables (only when the off-diagonal pairs fit one 128-row tile)
    {
        const int n = ham->norb;
        plan->npoff = n * (n - 1) / 2;
        if (plan->npoff <= 128 && lb > 0) {
            TB_CUDA(ctx, plan->d_lbp.alloc((size_t)lb * plan->npoff));
            TB_CUDA(ctx, cudaMemsetAsync(plan->d_lbp.p, 0xFF, plan->d_lbp.bytes(), st));
            k_link_by_pair<<<(unsigned)((lb + 127) / 128), 128, 0, st>>>(lb, b->d_off1.p, b->d_ent1.p, plan->npoff,
                                                                          plan->d_lbp.p);
            TB_CUDA(ctx, cudaGetLastError());
            std::vector<int32_t> op(plan->npoff);
            for (int r = 1; r < n; ++r)
                for (int q = 0; q < r; ++q) op[r * (r - 1) / 2 + q] = r * (r + 1) / 2 + q;
            TB_CUDA(ctx, plan->d_offpair.alloc(plan->npoff));
            TB_CUDA(ctx, cudaMemcpy(plan->d_offpair.p, op.data(), op.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            TB_CUDA(ctx, plan->d_tc_err.alloc(1));
            TB_CUDA(ctx, cudaMemsetAsync(plan->d_tc_err.p, 0, sizeof(int), st));
        }
    }
    // work counts: non-zeros of H by class (Sec. II.C, Table I)
    tbsci_sigma_counts &c = plan->counts;
    c.ndet = la * lb;
    c.nnz_aa = (S1a + D2a) * lb;
    c.nnz_bb = (S1b + D2b) * la;
    c.nnz_ab = S1a * S1b;
    c.nnz = c.ndet + c.nnz_aa + c.nnz_bb + c.nnz_ab;
    c.bytes_tables = (int64_t)(plan->A.d_sci.bytes() + plan->A.d_sval.bytes() + plan->A.d_dcol.bytes() +
                               plan->A.d_dval.bytes() + plan->B.d_sci.bytes() + plan->B.d_sval.bytes() +
                               plan->B.d_dcol.bytes() + plan->B.d_dval.bytes() + plan->d_U.bytes());
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    const size_t bytes = plan_device_bytes(*plan);
    TB_TRY(charge(ctx, bytes, "prepared space"));  // on failure the plan is freed on return
    plan->charged = bytes;
    tune_cache_apply(ctx, plan.get(), la, lb);
    *out = plan.get();
    ham->plans.push_back(std::move(plan));
    return TBSCI_OK;
}

}  // namespace tbsci
