// sigma = H.c on a TPB space (Sec. II.B, Eq. 7 on one device; the six
// Slater-Condon classes [a,b] of Sec. II.C and Algorithm 1).
//
// With alpha-block-first spin-orbital ordering, H = H_a x 1 + 1 x H_b + V_ab
// where H_a / H_b are the one-spin string Hamiltonians and
// V_ab = sum_{pq,rs} (pq|rs) E^a_pq E^b_rs. One CTA owns one alpha row Ia of
// sigma (owner computes: no atomics, deterministic) and sweeps its "alpha
// terms" -- the alpha strings Ja coupled to Ia:
//
//   Ja = Ia (classes [0,0], [0,1], [0,2] and the alpha-diagonal part of [1,1]):
//     sigma(Ia,Ib) += Hd(Ia,Ib) c(Ia,Ib)
//                   + sum_{beta singles Jb of Ib} (h_b(Ib,Jb) + s_b W_Ia[rs]) c(Ia,Jb)
//                   + sum_{beta doubles Jb of Ib} h_b(Ib,Jb) c(Ia,Jb)
//     with W_Ia[rs] = sum_{p in Ia} (pp|rs) and Hd the diagonal;
//   Ja an alpha single of Ia with orbital pair pq, sign s_a (classes [1,0], [1,1]):
//     sigma(Ia,Ib) += (h_a(Ia,Ja) + s_a U[pq][Ib]) c(Ja,Ib)
//                   + s_a sum_{beta singles Jb of Ib} s_b (pq|rs) c(Ja,Jb);
//   Ja an alpha double of Ia (class [2,0]):
//     sigma(Ia,Ib) += h_a(Ia,Ja) c(Ja,Ib).
//
// Every non-zero H_IJ costs exactly one multiply-add per vector. The c row Ja
// is staged in shared memory for the in-row beta gathers, the accumulator row
// lives in shared memory, threads own beta columns in an order sorted by
// single-link count so a warp's lanes have nearly equal trip counts.
#include <algorithm>

#include "internal.cuh"

namespace tbsci {

namespace {

template <typename T>
struct SigArgs {
    int64_t la, lb, vstride;
    const T *C;
    T *S;
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
    const int32_t *permb, *rowsa;
    T ecore;
};

constexpr int kThreads = 256;

template <typename T, int NV, bool STAGE, bool ACCS>
__global__ void __launch_bounds__(kThreads) k_sigma(SigArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int npair = A.npair;
    const int64_t lb = A.lb, vs = A.vstride;
    T *sV2 = reinterpret_cast<T *>(smem_raw);
    int *sOcc = reinterpret_cast<int *>(sV2 + 2 * npair);
    T *sC = reinterpret_cast<T *>(smem_raw + ((2 * npair * sizeof(T) + 64 * sizeof(int) + 15) & ~size_t(15)));
    T *sAcc = sC + (STAGE ? NV * lb : 0);
    const int64_t Ia = A.rowsa[blockIdx.x];
    const T *__restrict__ C = A.C;
    T *__restrict__ S = A.S;
    T *gAcc = S + Ia * lb;  // accumulator row when not in shared memory

    auto acc_ref = [&](int v, int64_t ib) -> T & { return ACCS ? sAcc[v * lb + ib] : gAcc[v * vs + ib]; };
    auto cval = [&](int v, int64_t row, int64_t col) -> T {
        return STAGE ? sC[v * lb + col] : __ldg(C + v * vs + row * lb + col);
    };
    auto stage = [&](int64_t row) {
        if (STAGE)
            for (int v = 0; v < NV; ++v) {
                const T *src = C + v * vs + row * lb;
                for (int64_t j = threadIdx.x; j < lb; j += kThreads) sC[v * lb + j] = __ldg(src + j);
            }
    };

    if (threadIdx.x == 0) {
        int k = 0;
        for (uint64_t s = A.stra[Ia]; s; s &= s - 1) {
            int p = __ffsll((long long)s) - 1;
            sOcc[k++] = p * (p + 1) / 2 + p;
        }
    }
    __syncthreads();
    const int na = A.na;
    // W_Ia[x] = sum_{p in Ia} (pp|x), stored with both signs
    for (int x = threadIdx.x; x < npair; x += kThreads) {
        T w = 0;
        for (int k = 0; k < na; ++k) w += A.V[(size_t)sOcc[k] * npair + x];
        sV2[2 * x] = w;
        sV2[2 * x + 1] = -w;
    }
    stage(Ia);
    __syncthreads();

    // ---- Ja = Ia
    const T eIa = A.ecore + A.Ea[Ia];
    for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
        const int64_t ib = A.permb[j];
        T ed = eIa + A.Eb[ib];
        for (int k = 0; k < na; ++k) ed += __ldg(A.U + (size_t)sOcc[k] * lb + ib);
        T acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = ed * cval(v, Ia, ib);
        const int64_t s0 = A.b_soff[ib], s1 = A.b_soff[ib + 1];
        for (int64_t k = s0; k < s1; ++k) {
            const int2 e = __ldg(A.b_sci + k);
            const T x = __ldg(A.b_sval + k) + sV2[e.y];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += x * cval(v, Ia, e.x);
        }
        const int64_t d0 = A.b_doff[ib], d1 = A.b_doff[ib + 1];
        for (int64_t k = d0; k < d1; ++k) {
            const int col = __ldg(A.b_dcol + k);
            const T x = __ldg(A.b_dval + k);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += x * cval(v, Ia, col);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) acc_ref(v, ib) = acc[v];
    }

    // ---- Ja = alpha singles of Ia
    const int64_t t0 = A.a_soff[Ia], t1 = A.a_soff[Ia + 1];
    for (int64_t t = t0; t < t1; ++t) {
        const int2 ea = __ldg(A.a_sci + t);
        const int64_t Ja = ea.x;
        const int pr = ea.y >> 1;
        const T sa = (ea.y & 1) ? T(-1) : T(1);
        const T ha = __ldg(A.a_sval + t);
        __syncthreads();
        for (int x = threadIdx.x; x < npair; x += kThreads) {
            const T vv = sa * A.V[(size_t)pr * npair + x];
            sV2[2 * x] = vv;
            sV2[2 * x + 1] = -vv;
        }
        stage(Ja);
        __syncthreads();
        const T *__restrict__ Urow = A.U + (size_t)pr * lb;
        for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
            const int64_t ib = A.permb[j];
            const T coef = ha + sa * __ldg(Urow + ib);
            T acc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = acc_ref(v, ib) + coef * cval(v, Ja, ib);
            const int64_t s0 = A.b_soff[ib], s1 = A.b_soff[ib + 1];
            for (int64_t k = s0; k < s1; ++k) {
                const int2 e = __ldg(A.b_sci + k);
                const T x = sV2[e.y];
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += x * cval(v, Ja, e.x);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) acc_ref(v, ib) = acc[v];
        }
    }
    __syncthreads();

    // ---- Ja = alpha doubles of Ia, natural column order, c rows read coalesced
    const int64_t u0 = A.a_doff[Ia], u1 = A.a_doff[Ia + 1];
    for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
        T acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = acc_ref(v, j);
        for (int64_t t = u0; t < u1; ++t) {
            const int64_t Ja = __ldg(A.a_dcol + t);
            const T x = __ldg(A.a_dval + t);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += x * __ldg(C + v * vs + Ja * lb + j);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) S[v * vs + Ia * lb + j] = acc[v];
    }
}

// Hd(Ia,Ib) = ecore + E_a(Ia) + E_b(Ib) + sum_{p in Ia} U[pp][Ib]
__global__ void k_diagonal(const uint64_t *__restrict__ stra, int64_t la, int64_t lb, const double *__restrict__ Ea,
                           const double *__restrict__ Eb, const double *__restrict__ U, double ecore, double *diag) {
    int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (K >= la * lb) return;
    int64_t ia = K / lb, ib = K - ia * lb;
    double d = ecore + Ea[ia] + Eb[ib];
    for (uint64_t s = stra[ia]; s; s &= s - 1) {
        int p = __ffsll((long long)s) - 1;
        d += U[(size_t)(p * (p + 1) / 2 + p) * lb + ib];
    }
    diag[K] = d;
}

template <typename T>
SigArgs<T> make_args(const tbsci_ham *ham, const Plan *P);

template <>
SigArgs<double> make_args<double>(const tbsci_ham *ham, const Plan *P) {
    SigArgs<double> A{};
    A.la = P->A.l;
    A.lb = P->B.l;
    A.vstride = A.la * A.lb;
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
    A.permb = P->d_permb.p;
    A.rowsa = P->d_rowsa.p;
    A.ecore = ham->ecore;
    return A;
}

template <>
SigArgs<float> make_args<float>(const tbsci_ham *ham, const Plan *P) {
    SigArgs<float> A{};
    A.la = P->A.l;
    A.lb = P->B.l;
    A.vstride = A.la * A.lb;
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
    A.permb = P->d_permb.p;
    A.rowsa = P->d_rowsa.p;
    A.ecore = (float)ham->ecore;
    return A;
}

template <typename T>
size_t smem_bytes(int npair, int64_t lb, int nv, bool stage, bool accs) {
    size_t head = (2 * npair * sizeof(T) + 64 * sizeof(int) + 15) & ~size_t(15);
    return head + ((stage ? 1 : 0) + (accs ? 1 : 0)) * (size_t)nv * lb * sizeof(T);
}

template <typename T, int NV, bool STAGE, bool ACCS>
tbsci_status launch_one(tbsci_ctx *ctx, SigArgs<T> A, size_t smem, cudaStream_t st) {
    auto kern = k_sigma<T, NV, STAGE, ACCS>;
    TB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)A.la, kThreads, smem, st>>>(A);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

template <typename T, int NV>
tbsci_status launch_nv(tbsci_ctx *ctx, SigArgs<T> A, cudaStream_t st) {
    const size_t limit = ctx->smem_optin;
    size_t sm;
    if ((sm = smem_bytes<T>(A.npair, A.lb, NV, true, true)) <= limit)
        return launch_one<T, NV, true, true>(ctx, A, sm, st);
    if ((sm = smem_bytes<T>(A.npair, A.lb, NV, false, true)) <= limit)
        return launch_one<T, NV, false, true>(ctx, A, sm, st);
    sm = smem_bytes<T>(A.npair, A.lb, NV, false, false);
    return launch_one<T, NV, false, false>(ctx, A, sm, st);
}

template <typename T>
tbsci_status launch_typed(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *P, const T *c, T *s, int nvec,
                          cudaStream_t st) {
    SigArgs<T> A = make_args<T>(ham, P);
    if (A.la == 0 || A.lb == 0) return TBSCI_OK;
    // vectors per CTA: as many as fit (up to 4) with staging and a shared accumulator
    int v = 0;
    while (v < nvec) {
        int rem = nvec - v;
        int nv = std::min(rem, 4);
        while (nv > 1 && smem_bytes<T>(A.npair, A.lb, nv, true, true) > ctx->smem_optin) --nv;
        A.C = c + (size_t)v * A.vstride;
        A.S = s + (size_t)v * A.vstride;
        switch (nv) {
            case 4: TB_TRY((launch_nv<T, 4>(ctx, A, st))); break;
            case 3: TB_TRY((launch_nv<T, 3>(ctx, A, st))); break;
            case 2: TB_TRY((launch_nv<T, 2>(ctx, A, st))); break;
            default: TB_TRY((launch_nv<T, 1>(ctx, A, st))); break;
        }
        v += nv;
    }
    return TBSCI_OK;
}

}  // namespace

tbsci_status sigma_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const void *c, void *s, int nvec,
                          tbsci_dtype dt, cudaStream_t st) {
    if (dt == TBSCI_F64)
        return launch_typed<double>(ctx, ham, plan, static_cast<const double *>(c), static_cast<double *>(s), nvec, st);
    if (dt == TBSCI_F32)
        return launch_typed<float>(ctx, ham, plan, static_cast<const float *>(c), static_cast<float *>(s), nvec, st);
    return fail(ctx, TBSCI_EINVAL, "unknown dtype");
}

tbsci_status diagonal_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *P, double *diag, cudaStream_t st) {
    const int64_t N = P->A.l * P->B.l;
    if (N == 0) return TBSCI_OK;
    k_diagonal<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P->A.d_str, P->A.l, P->B.l, P->A.d_E.p, P->B.d_E.p,
                                                            P->d_U.p, ham->ecore, diag);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

}  // namespace tbsci
