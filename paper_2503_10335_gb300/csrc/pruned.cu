// sigma = H.c on a pruned TBSCI space (Sec. II.A, Eq. 6): the determinants
// (w, u) of a TPB space with u in a per-alpha-string set I_w. H on the space is
// the principal submatrix of H on its determinants, so sigma on a member row is
// the TPB sigma of that row with c set to zero outside the space.
//
// One CTA owns alpha row Ia and walks its alpha terms Ja (Ia itself, its alpha
// singles, its alpha doubles) as the TPB kernel does. For each term the
// compressed c row Ja is expanded into a dense, zero-initialised shared-memory
// row (its members scattered in, then zeros scattered back after use), so every
// beta gather of the classes of Sec. II.C is a plain shared-memory read and a
// non-member reads 0: the membership test of Algorithm 1 costs nothing per link.
// Rows longer than shared memory look c(Ja, Jb) up by binary search in I_Ja.
// Each member column of Ia is owned by one thread across all terms (its sigma
// entry accumulates in place, no atomics, deterministic).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace tbsci {

namespace {

template <typename T>
struct PrArgs {
    int64_t la, lb;
    const T *C;
    T *S;
    const int64_t *off;
    const int32_t *cols, *rows;
    int npair, na;
    const uint64_t *stra;
    const int64_t *a_soff, *a_doff;
    const int2 *a_sci;
    const T *a_sval, *a_dval;
    const int32_t *a_dcol;
    const T *Ea;
    const int64_t *b_soff, *b_doff;
    const int2 *b_sci;
    const T *b_sval, *b_dval;
    const int32_t *b_dcol;
    const T *Eb;
    const T *V;  // [npair][npair]
    const T *U;  // [npair][lb]
    T ecore;
};

template <typename T>
PrArgs<T> pr_args(const tbsci_ham *ham, const Plan *P, const tbsci_pruned *pr);

template <>
PrArgs<double> pr_args<double>(const tbsci_ham *ham, const Plan *P, const tbsci_pruned *pr) {
    PrArgs<double> A{};
    A.la = P->A.l;
    A.lb = P->B.l;
    A.off = pr->d_off.p;
    A.cols = pr->d_cols.p;
    A.rows = pr->d_rows.p;
    A.npair = P->npair;
    A.na = P->A.nelec;
    A.stra = P->A.d_str;
    A.a_soff = P->A.d_soff;
    A.a_doff = P->A.d_doff;
    A.a_sci = P->A.d_sci.p;
    A.a_sval = P->A.d_sval.p;
    A.a_dcol = P->A.d_dcol.p;
    A.a_dval = P->A.d_dval.p;
    A.Ea = P->A.d_E.p;
    A.b_soff = P->B.d_soff;
    A.b_doff = P->B.d_doff;
    A.b_sci = P->B.d_sci.p;
    A.b_sval = P->B.d_sval.p;
    A.b_dcol = P->B.d_dcol.p;
    A.b_dval = P->B.d_dval.p;
    A.Eb = P->B.d_E.p;
    A.V = ham->d_V.p;
    A.U = P->d_U.p;
    A.ecore = ham->ecore;
    return A;
}

template <>
PrArgs<float> pr_args<float>(const tbsci_ham *ham, const Plan *P, const tbsci_pruned *pr) {
    PrArgs<float> A{};
    A.la = P->A.l;
    A.lb = P->B.l;
    A.off = pr->d_off.p;
    A.cols = pr->d_cols.p;
    A.rows = pr->d_rows.p;
    A.npair = P->npair;
    A.na = P->A.nelec;
    A.stra = P->A.d_str;
    A.a_soff = P->A.d_soff;
    A.a_doff = P->A.d_doff;
    A.a_sci = P->A.d_sci.p;
    A.a_sval = P->A.d_svalf.p;
    A.a_dcol = P->A.d_dcol.p;
    A.a_dval = P->A.d_dvalf.p;
    A.Ea = P->A.d_Ef.p;
    A.b_soff = P->B.d_soff;
    A.b_doff = P->B.d_doff;
    A.b_sci = P->B.d_sci.p;
    A.b_sval = P->B.d_svalf.p;
    A.b_dcol = P->B.d_dcol.p;
    A.b_dval = P->B.d_dvalf.p;
    A.Eb = P->B.d_Ef.p;
    A.V = ham->d_Vf.p;
    A.U = P->d_Uf.p;
    A.ecore = (float)ham->ecore;
    return A;
}

template <typename T>
__host__ __device__ size_t pr_head_bytes(int npair) {
    return ((2 * npair + 2) * sizeof(T) + 64 * sizeof(int) + 15) & ~size_t(15);
}

constexpr int kPrThreads = 256;

template <typename T, bool EXPAND>
__global__ void __launch_bounds__(kPrThreads) k_sigma_pruned(PrArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int npair = A.npair;
    T *sV2 = reinterpret_cast<T *>(smem_raw);  // [2 npair + 2]: coefficient by (pair, sign); last two zero
    int *sOcc = reinterpret_cast<int *>(sV2 + 2 * npair + 2);
    T *sC = reinterpret_cast<T *>(smem_raw + pr_head_bytes<T>(npair));  // [lb] when EXPAND
    const int64_t Ia = A.rows[blockIdx.x];
    const int64_t m0 = A.off[Ia], cnt = A.off[Ia + 1] - m0;
    if (cnt == 0) return;  // block-uniform, before any barrier
    const int64_t lb = A.lb;
    if (threadIdx.x == 0) {
        int k = 0;
        for (uint64_t s = A.stra[Ia]; s; s &= s - 1) {
            const int p = __ffsll((long long)s) - 1;
            sOcc[k++] = p * (p + 1) / 2 + p;
        }
        sV2[2 * npair] = T(0);
        sV2[2 * npair + 1] = T(0);
    }
    if (EXPAND)
        for (int64_t j = threadIdx.x; j < lb; j += kPrThreads) sC[j] = T(0);
    __syncthreads();
    for (int x = threadIdx.x; x < npair; x += kPrThreads) {  // W_Ia[x] = sum_{p in Ia} (pp|x)
        T w = 0;
        for (int k = 0; k < A.na; ++k) w += A.V[(size_t)sOcc[k] * npair + x];
        sV2[2 * x] = w;
        sV2[2 * x + 1] = -w;
    }
    const int64_t t0 = A.a_soff[Ia], ns = A.a_soff[Ia + 1] - t0;
    const int64_t d0 = A.a_doff[Ia], nd = A.a_doff[Ia + 1] - d0;
    const T *__restrict__ C = A.C;
    T *__restrict__ S = A.S;
    for (int64_t k = 0; k < 1 + ns + nd; ++k) {
        int64_t Ja = Ia;
        int kind = 0, pr = 0;
        T ha = T(0), sa = T(1);
        if (k >= 1 && k <= ns) {
            const int2 e = A.a_sci[t0 + k - 1];
            Ja = e.x;
            pr = e.y >> 1;
            sa = (e.y & 1) ? T(-1) : T(1);
            ha = A.a_sval[t0 + k - 1];
            kind = 1;
        } else if (k > ns) {
            Ja = A.a_dcol[d0 + k - 1 - ns];
            ha = A.a_dval[d0 + k - 1 - ns];
            kind = 2;
        }
        const int64_t j0 = A.off[Ja], jc = A.off[Ja + 1] - j0;
        if (jc == 0) continue;  // block-uniform: no member of row Ja couples
        if (kind == 1)
            for (int x = threadIdx.x; x < npair; x += kPrThreads) {
                const T vv = sa * A.V[(size_t)pr * npair + x];
                sV2[2 * x] = vv;
                sV2[2 * x + 1] = -vv;
            }
        if (EXPAND)
            for (int64_t i = threadIdx.x; i < jc; i += kPrThreads) sC[A.cols[j0 + i]] = __ldg(C + j0 + i);
        __syncthreads();
        // c(Ja, jb): expanded row, or binary search in I_Ja
        auto cv = [&](int64_t jb) -> T {
            if (EXPAND) return sC[jb];
            int64_t lo = j0, hi = j0 + jc - 1;
            while (lo <= hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int32_t x = __ldg(A.cols + mid);
                if (x == jb) return __ldg(C + mid);
                if (x < jb) lo = mid + 1;
                else hi = mid - 1;
            }
            return T(0);
        };
        for (int64_t p = threadIdx.x; p < cnt; p += kPrThreads) {
            const int64_t ib = A.cols[m0 + p];
            T acc;
            if (kind == 0) {
                T ed = A.ecore + A.Ea[Ia] + A.Eb[ib];
                for (int q = 0; q < A.na; ++q) ed += __ldg(A.U + (size_t)sOcc[q] * lb + ib);
                acc = ed * cv(ib);
                for (int64_t t = A.b_soff[ib]; t < A.b_soff[ib + 1]; ++t) {
                    const int2 e = __ldg(A.b_sci + t);
                    acc += (__ldg(A.b_sval + t) + sV2[e.y]) * cv(e.x);
                }
                for (int64_t t = A.b_doff[ib]; t < A.b_doff[ib + 1]; ++t)
                    acc += __ldg(A.b_dval + t) * cv(__ldg(A.b_dcol + t));
            } else if (kind == 1) {
                acc = S[m0 + p] + (ha + sa * __ldg(A.U + (size_t)pr * lb + ib)) * cv(ib);
                for (int64_t t = A.b_soff[ib]; t < A.b_soff[ib + 1]; ++t) {
                    const int2 e = __ldg(A.b_sci + t);
                    acc += sV2[e.y] * cv(e.x);
                }
            } else {
                acc = S[m0 + p] + ha * cv(ib);
            }
            S[m0 + p] = acc;
        }
        __syncthreads();
        if (EXPAND) {
            for (int64_t i = threadIdx.x; i < jc; i += kPrThreads) sC[A.cols[j0 + i]] = T(0);
            __syncthreads();
        }
    }
}

// diag[off[w] + p] = ecore + E_a(w) + E_b(u) + sum_{q in w} U[qq][u], u = cols[off[w] + p]
__global__ void k_diagonal_pruned(const uint64_t *__restrict__ stra, int64_t lb, const int64_t *__restrict__ off,
                                  const int32_t *__restrict__ cols, const double *__restrict__ Ea,
                                  const double *__restrict__ Eb, const double *__restrict__ U, double ecore,
                                  double *diag) {
    const int64_t w = blockIdx.x;
    const int64_t m0 = off[w], cnt = off[w + 1] - m0;
    const uint64_t sw = stra[w];
    for (int64_t p = threadIdx.x; p < cnt; p += blockDim.x) {
        const int64_t u = cols[m0 + p];
        double d = ecore + Ea[w] + Eb[u];
        for (uint64_t s = sw; s; s &= s - 1) {
            const int q = __ffsll((long long)s) - 1;
            d += U[(size_t)(q * (q + 1) / 2 + q) * lb + u];
        }
        diag[m0 + p] = d;
    }
}

template <typename T>
tbsci_status launch_pruned(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *P, const tbsci_pruned *pr, const T *c,
                           T *s, int nvec, cudaStream_t st) {
    PrArgs<T> A = pr_args<T>(ham, P, pr);
    if (pr->nd == 0 || A.la == 0) return TBSCI_OK;
    const size_t head = pr_head_bytes<T>(A.npair), full = head + (size_t)A.lb * sizeof(T);
    const bool expand = full <= ctx->smem_optin;
    for (int v = 0; v < nvec; ++v) {
        A.C = c + (size_t)v * pr->nd;
        A.S = s + (size_t)v * pr->nd;
        TraceScope tr(ctx, "k_sigma_pruned", st);
        if (expand) {
            TB_CUDA(ctx, cudaFuncSetAttribute(k_sigma_pruned<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)full));
            k_sigma_pruned<T, true><<<(unsigned)A.la, kPrThreads, full, st>>>(A);
        } else {
            k_sigma_pruned<T, false><<<(unsigned)A.la, kPrThreads, head, st>>>(A);
        }
        TB_CUDA(ctx, cudaGetLastError());
    }
    return TBSCI_OK;
}

}  // namespace

tbsci_status pruned_sigma_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const tbsci_pruned *pr,
                                 const void *c, void *s, int nvec, tbsci_dtype dt, cudaStream_t st) {
    if (dt == TBSCI_F64)
        return launch_pruned<double>(ctx, ham, plan, pr, static_cast<const double *>(c), static_cast<double *>(s),
                                     nvec, st);
    if (dt == TBSCI_F32 || dt == TBSCI_F32_TC_TF32 || dt == TBSCI_F32_TC_BF16)
        return launch_pruned<float>(ctx, ham, plan, pr, static_cast<const float *>(c), static_cast<float *>(s), nvec,
                                    st);
    return fail(ctx, TBSCI_EINVAL, "unknown dtype");
}

tbsci_status pruned_diagonal_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *P, const tbsci_pruned *pr,
                                    double *diag, cudaStream_t st) {
    if (pr->nd == 0 || P->A.l == 0) return TBSCI_OK;
    k_diagonal_pruned<<<(unsigned)P->A.l, 128, 0, st>>>(P->A.d_str, P->B.l, pr->d_off.p, pr->d_cols.p, P->A.d_E.p,
                                                       P->B.d_E.p, P->d_U.p, ham->ecore, diag);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

}  // namespace tbsci

using namespace tbsci;

extern "C" {

tbsci_status tbsci_pruned_create(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b, const int64_t *off,
                                 const int32_t *cols, tbsci_pruned **out) {
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, a && b && off && out, TBSCI_EINVAL, "tbsci_pruned_create: null argument");
    *out = nullptr;
    const int64_t la = a->count, lb = b->count;
    TB_CHECK(ctx, off[0] == 0, TBSCI_EINVAL, "tbsci_pruned_create: off[0] must be 0");
    for (int64_t w = 0; w < la; ++w)
        TB_CHECK(ctx, off[w + 1] >= off[w], TBSCI_EINVAL, "tbsci_pruned_create: off must be non-decreasing");
    const int64_t nd = off[la];
    TB_CHECK(ctx, nd == 0 || cols, TBSCI_EINVAL, "tbsci_pruned_create: null cols");
    for (int64_t w = 0; w < la; ++w)
        for (int64_t k = off[w]; k < off[w + 1]; ++k) {
            TB_CHECK(ctx, cols[k] >= 0 && cols[k] < lb, TBSCI_EINVAL,
                     "tbsci_pruned_create: beta index out of range in row " + std::to_string(w));
            TB_CHECK(ctx, k == off[w] || cols[k] > cols[k - 1], TBSCI_EINVAL,
                     "tbsci_pruned_create: beta indices of row " + std::to_string(w) + " not strictly ascending");
        }
    auto pr = std::make_unique<tbsci_pruned>();
    pr->ctx = ctx;
    pr->ida = a->id;
    pr->idb = b->id;
    pr->la = la;
    pr->lb = lb;
    pr->nd = nd;
    pr->h_off.assign(off, off + la + 1);
    // alpha rows by work, heaviest first: members x (1 + alpha singles + alpha doubles)
    std::vector<double> work(la);
    for (int64_t w = 0; w < la; ++w)
        work[w] = (double)(off[w + 1] - off[w]) *
                  (double)(1 + (a->h_off1[w + 1] - a->h_off1[w]) + (a->h_off2.empty() ? 0 : a->h_off2[w + 1] - a->h_off2[w]));
    std::vector<int32_t> rows(la);
    std::iota(rows.begin(), rows.end(), 0);
    std::stable_sort(rows.begin(), rows.end(), [&](int32_t x, int32_t y) { return work[x] > work[y]; });
    const size_t bytes = (size_t)(la + 1) * 8 + (size_t)nd * 4 + (size_t)la * 4;
    TB_TRY(charge(ctx, bytes, "pruned space"));
    pr->charged = bytes;
    cudaError_t e = pr->d_off.alloc(la + 1);
    if (e == cudaSuccess) e = pr->d_cols.alloc(nd);
    if (e == cudaSuccess) e = pr->d_rows.alloc(la);
    if (e == cudaSuccess) e = cudaMemcpy(pr->d_off.p, off, (la + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nd) e = cudaMemcpy(pr->d_cols.p, cols, nd * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && la) e = cudaMemcpy(pr->d_rows.p, rows.data(), la * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        uncharge(ctx, bytes);
        return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                    std::string("tbsci_pruned_create: ") + cudaGetErrorString(e));
    }
    *out = pr.release();
    return TBSCI_OK;
}

// Symmetry blocks (Sec. II.A): each I_w is the class of beta strings whose irrep
// is target XOR irrep(w); a string's irrep is the XOR of the labels of its
// occupied orbitals. The classes are built once and copied per alpha string.
tbsci_status tbsci_pruned_create_symmetry(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b,
                                          const int32_t *orb_irrep, int target, tbsci_pruned **out) {
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, a && b && orb_irrep && out, TBSCI_EINVAL, "tbsci_pruned_create_symmetry: null argument");
    TB_CHECK(ctx, a->norb == b->norb, TBSCI_EINVAL, "tbsci_pruned_create_symmetry: norb differs between the sets");
    TB_CHECK(ctx, target >= 0 && target < 8, TBSCI_EINVAL, "tbsci_pruned_create_symmetry: target irrep not in 0..7");
    for (int i = 0; i < a->norb; ++i)
        TB_CHECK(ctx, orb_irrep[i] >= 0 && orb_irrep[i] < 8, TBSCI_EINVAL,
                 "tbsci_pruned_create_symmetry: orbital irrep not in 0..7");
    std::vector<uint64_t> sa(a->count), sb(b->count);
    if (a->count) TB_CUDA(ctx, cudaMemcpy(sa.data(), a->d_str.p, a->count * 8, cudaMemcpyDeviceToHost));
    if (b->count) TB_CUDA(ctx, cudaMemcpy(sb.data(), b->d_str.p, b->count * 8, cudaMemcpyDeviceToHost));
    auto irrep = [&](uint64_t s) {
        int g = 0;
        for (; s; s &= s - 1) g ^= orb_irrep[__builtin_ctzll(s)];
        return g;
    };
    std::vector<int32_t> cls[8];
    for (int64_t u = 0; u < b->count; ++u) cls[irrep(sb[u])].push_back((int32_t)u);
    std::vector<int64_t> off(a->count + 1, 0);
    for (int64_t w = 0; w < a->count; ++w) off[w + 1] = off[w] + (int64_t)cls[target ^ irrep(sa[w])].size();
    std::vector<int32_t> cols((size_t)off[a->count]);
    for (int64_t w = 0; w < a->count; ++w) {
        const std::vector<int32_t> &c = cls[target ^ irrep(sa[w])];
        std::copy(c.begin(), c.end(), cols.begin() + off[w]);
    }
    return tbsci_pruned_create(ctx, a, b, off.data(), cols.empty() ? nullptr : cols.data(), out);
}

tbsci_status tbsci_pruned_count(const tbsci_pruned *pr, int64_t *ndet) {
    if (!pr || !ndet) return TBSCI_EINVAL;
    *ndet = pr->nd;
    return TBSCI_OK;
}

void tbsci_pruned_destroy(tbsci_pruned *pr) {
    if (!pr) return;
    if (pr->ctx) cudaSetDevice(pr->ctx->device);
    uncharge(pr->ctx, pr->charged);
    delete pr;
}

static tbsci_status pruned_plan(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                const tbsci_pruned *pr, Plan **p) {
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, pr && a && b, TBSCI_EINVAL, "null handle");
    TB_CHECK(ctx, pr->ida == a->id && pr->idb == b->id, TBSCI_EINVAL,
             "the pruned space was made from other tables");
    return plan_get(ctx, ham, a, b, p);
}

tbsci_status tbsci_sigma_pruned(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                const tbsci_pruned *pr, const void *c, void *sigma, int nvec, tbsci_dtype dtype,
                                tbsci_stream stream) {
    Plan *p = nullptr;
    TB_TRY(pruned_plan(ctx, ham, a, b, pr, &p));
    TB_CHECK(ctx, nvec >= 1, TBSCI_EINVAL, "nvec must be >= 1");
    if (pr->nd == 0) return TBSCI_OK;
    TB_CHECK(ctx, c && sigma && c != sigma, TBSCI_EINVAL, "bad vector pointers");
    return pruned_sigma_launch(ctx, ham, p, pr, c, sigma, nvec, dtype, (cudaStream_t)stream);
}

tbsci_status tbsci_diagonal_pruned(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                   const tbsci_pruned *pr, double *diag, tbsci_stream stream) {
    Plan *p = nullptr;
    TB_TRY(pruned_plan(ctx, ham, a, b, pr, &p));
    if (pr->nd == 0) return TBSCI_OK;
    TB_CHECK(ctx, diag, TBSCI_EINVAL, "null diag pointer");
    return pruned_diagonal_launch(ctx, ham, p, pr, diag, (cudaStream_t)stream);
}

tbsci_status tbsci_davidson_pruned(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                   const tbsci_pruned *pr, int nroots, const tbsci_davidson_opts *opts,
                                   double *energies, double *vecs, tbsci_davidson_info *info) {
    Plan *p = nullptr;
    TB_TRY(pruned_plan(ctx, ham, a, b, pr, &p));
    TB_CHECK(ctx, energies, TBSCI_EINVAL, "null energies");
    tbsci_davidson_opts o{};
    if (opts) o = *opts;
    else o.mixed = ctx->default_mixed;
    const size_t bytes = engine_device_bytes(pr->nd, nroots, &o);
    TB_TRY(charge(ctx, bytes, "Davidson vectors"));
    tbsci_status st = davidson_run(ctx, ham, p, nroots, &o, energies, vecs, info, pr);
    uncharge(ctx, bytes);
    return st;
}

}  // extern "C"
