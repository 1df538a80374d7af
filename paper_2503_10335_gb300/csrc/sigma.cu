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
#include <cstring>
#include <vector>

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
    const int32_t *permb, *permb2, *rowsa;
    T ecore;
    // sliced-ELL beta links (see Plan): singles in permb order; singles with
    // values and doubles in permb2 order; tables with columns in those orders
    const int64_t *s1_off, *s2_off, *d2_off;
    const int32_t *s1_w, *s2_w, *d2_w;
    const int2 *s1_ci, *s2_ci;
    const T *s2_val, *d2_val;
    const int32_t *d2_col;
    const T *U1, *U2, *Eb2;
};

// One alpha row Ia of sigma (the whole body of a CTA). REST: only the classes
// the tensor-core kernel leaves out (same-spin beta singles and doubles, alpha
// doubles); the diagonal, alpha singles and every alpha-beta term are skipped.
// PAIR (with REST, NV = 2, vstride = l_beta): the CTA serves alpha rows Ia and
// Ia + 1 of one vector; the beta sweep reads each link once for both rows, the
// alpha-double sweep runs per row. Same summation order per row as NV = 1.
template <typename T, int NV, bool STAGE, bool ACCS, int kThreads, bool REST = false, bool PAIR = false>
__device__ __forceinline__ void sigma_row(const SigArgs<T> &A, const int64_t Ia, unsigned char *smem_raw) {
    const int npair = A.npair;
    const int64_t lb = A.lb, vs = A.vstride;
    T *sV2 = reinterpret_cast<T *>(smem_raw);  // [2*npair + 2], last two entries zero (padding)
    int *sOcc = reinterpret_cast<int *>(sV2 + 2 * npair + 2);
    T *sC = reinterpret_cast<T *>(smem_raw + (((2 * npair + 2) * sizeof(T) + 64 * sizeof(int) + 15) & ~size_t(15)));
    T *sAcc = sC + (STAGE ? NV * lb : 0);
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
        sV2[2 * npair] = T(0);
        sV2[2 * npair + 1] = T(0);
    }
    __syncthreads();
    const int na = A.na;
    // W_Ia[x] = sum_{p in Ia} (pp|x), stored with both signs
    for (int x = threadIdx.x; x < npair; x += kThreads) {
        T w = 0;
        if (!REST)
            for (int k = 0; k < na; ++k) w += A.V[(size_t)sOcc[k] * npair + x];
        sV2[2 * x] = w;
        sV2[2 * x + 1] = -w;
    }
    stage(Ia);
    __syncthreads();

    // ---- Ja = Ia: columns in permb2 order, beta links read as coalesced sliced-ELL rows
    const T eIa = A.ecore + A.Ea[Ia];
    for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
        const int64_t ib = A.permb2[j];
        const int64_t sl = j >> 5;
        const int lane = (int)(j & 31);
        T ed = T(0);
        if (!REST) {
            ed = eIa + __ldg(A.Eb2 + j);
            for (int k = 0; k < na; ++k) ed += __ldg(A.U2 + (size_t)sOcc[k] * lb + j);
        }
        T acc[NV], acc2[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            acc[v] = REST ? T(0) : ed * cval(v, Ia, ib);
            acc2[v] = T(0);
        }
        {
            const int2 *ci = A.s2_ci + A.s2_off[sl] + lane;
            const T *cv = A.s2_val + A.s2_off[sl] + lane;
            const int w = A.s2_w[sl];
            int k = 0;
            for (; k + 1 < w; k += 2) {
                const int2 e0 = __ldg(ci + 32 * k), e1 = __ldg(ci + 32 * (k + 1));
                const T x0 = __ldg(cv + 32 * k) + sV2[e0.y];
                const T x1 = __ldg(cv + 32 * (k + 1)) + sV2[e1.y];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    acc[v] += x0 * cval(v, Ia, e0.x);
                    acc2[v] += x1 * cval(v, Ia, e1.x);
                }
            }
            if (k < w) {
                const int2 e = __ldg(ci + 32 * k);
                const T x = __ldg(cv + 32 * k) + sV2[e.y];
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += x * cval(v, Ia, e.x);
            }
        }
        {
            const int32_t *dc = A.d2_col + A.d2_off[sl] + lane;
            const T *dv = A.d2_val + A.d2_off[sl] + lane;
            const int w = A.d2_w[sl];
            int k = 0;
            for (; k + 1 < w; k += 2) {
                const int c0 = __ldg(dc + 32 * k), c1 = __ldg(dc + 32 * (k + 1));
                const T x0 = __ldg(dv + 32 * k), x1 = __ldg(dv + 32 * (k + 1));
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    acc[v] += x0 * cval(v, Ia, c0);
                    acc2[v] += x1 * cval(v, Ia, c1);
                }
            }
            if (k < w) {
                const int col = __ldg(dc + 32 * k);
                const T x = __ldg(dv + 32 * k);
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += x * cval(v, Ia, col);
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) acc_ref(v, ib) = acc[v] + acc2[v];
    }

    // ---- Ja = alpha singles of Ia: columns in permb order
    const int64_t t0 = A.a_soff[Ia], t1 = REST ? t0 : A.a_soff[Ia + 1];
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
        const T *__restrict__ Urow = A.U1 + (size_t)pr * lb;
        for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
            const int64_t ib = A.permb[j];
            const int64_t sl = j >> 5;
            const int lane = (int)(j & 31);
            const T coef = ha + sa * __ldg(Urow + j);
            T acc[NV], acc2[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                acc[v] = acc_ref(v, ib) + coef * cval(v, Ja, ib);
                acc2[v] = T(0);
            }
            const int2 *ci = A.s1_ci + A.s1_off[sl] + lane;
            const int w = A.s1_w[sl];
            int k = 0;
            for (; k + 1 < w; k += 2) {
                const int2 e0 = __ldg(ci + 32 * k), e1 = __ldg(ci + 32 * (k + 1));
                const T x0 = sV2[e0.y], x1 = sV2[e1.y];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    acc[v] += x0 * cval(v, Ja, e0.x);
                    // FP64: one chain (the FP64 pipe, not the add latency, is the
                    // limit; the merge below would cost an add per column and term)
                    if constexpr (sizeof(T) == 8) acc[v] += x1 * cval(v, Ja, e1.x);
                    else acc2[v] += x1 * cval(v, Ja, e1.x);
                }
            }
            if (k < w) {
                const int2 e = __ldg(ci + 32 * k);
                const T x = sV2[e.y];
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += x * cval(v, Ja, e.x);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if constexpr (sizeof(T) == 8) acc_ref(v, ib) = acc[v];
                else acc_ref(v, ib) = acc[v] + acc2[v];
            }
        }
    }
    __syncthreads();

    if (PAIR) {
        // ---- alpha doubles of rows Ia and Ia + 1, each from its own link list
        for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int64_t row = Ia + v;
                const int64_t p0 = A.a_doff[row], p1 = A.a_doff[row + 1];
                T acc = acc_ref(v, j), acc2 = T(0);
                int64_t t = p0;
                for (; t + 3 < p1; t += 4) {
                    const int64_t J0 = __ldg(A.a_dcol + t), J1 = __ldg(A.a_dcol + t + 1);
                    const int64_t J2 = __ldg(A.a_dcol + t + 2), J3 = __ldg(A.a_dcol + t + 3);
                    const T x0 = __ldg(A.a_dval + t), x1 = __ldg(A.a_dval + t + 1);
                    const T x2 = __ldg(A.a_dval + t + 2), x3 = __ldg(A.a_dval + t + 3);
                    const T c0 = __ldg(C + J0 * lb + j), c1 = __ldg(C + J1 * lb + j);
                    const T c2 = __ldg(C + J2 * lb + j), c3 = __ldg(C + J3 * lb + j);
                    acc += x0 * c0;
                    acc2 += x1 * c1;
                    acc += x2 * c2;
                    acc2 += x3 * c3;
                }
                for (; t < p1; ++t) acc += __ldg(A.a_dval + t) * __ldg(C + __ldg(A.a_dcol + t) * lb + j);
                S[row * lb + j] = acc + acc2;
            }
        }
        return;
    }

    // ---- Ja = alpha doubles of Ia, natural column order, c rows read coalesced
    const int64_t u0 = A.a_doff[Ia], u1 = A.a_doff[Ia + 1];
    for (int64_t j = threadIdx.x; j < lb; j += kThreads) {
        T acc[NV], acc2[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            acc[v] = acc_ref(v, j);
            acc2[v] = T(0);
        }
        int64_t t = u0;
        for (; t + 3 < u1; t += 4) {
            const int64_t J0 = __ldg(A.a_dcol + t), J1 = __ldg(A.a_dcol + t + 1);
            const int64_t J2 = __ldg(A.a_dcol + t + 2), J3 = __ldg(A.a_dcol + t + 3);
            const T x0 = __ldg(A.a_dval + t), x1 = __ldg(A.a_dval + t + 1);
            const T x2 = __ldg(A.a_dval + t + 2), x3 = __ldg(A.a_dval + t + 3);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T c0 = __ldg(C + v * vs + J0 * lb + j), c1 = __ldg(C + v * vs + J1 * lb + j);
                const T c2 = __ldg(C + v * vs + J2 * lb + j), c3 = __ldg(C + v * vs + J3 * lb + j);
                acc[v] += x0 * c0;
                acc2[v] += x1 * c1;
                acc[v] += x2 * c2;
                acc2[v] += x3 * c3;
            }
        }
        for (; t < u1; ++t) {
            const int64_t Ja = __ldg(A.a_dcol + t);
            const T x = __ldg(A.a_dval + t);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += x * __ldg(C + v * vs + Ja * lb + j);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) S[v * vs + Ia * lb + j] = acc[v] + acc2[v];
    }
}

template <typename T, int NV, bool STAGE, bool ACCS, int kThreads, bool REST = false>
__global__ void __launch_bounds__(kThreads) k_sigma(SigArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sigma_row<T, NV, STAGE, ACCS, kThreads, REST>(A, A.rowsa[blockIdx.x], smem_raw);
}

// SIMT pass of the tensor-core sigma types over row pairs: A.rowsa holds even
// row starts, A.vstride = l_beta (see sigma_row's PAIR)
template <bool STAGE, int kThreads>
__global__ void __launch_bounds__(kThreads) k_sigma_rest_pair(SigArgs<float> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sigma_row<float, 2, STAGE, false, kThreads, true, true>(A, A.rowsa[blockIdx.x], smem_raw);
}

// One persistent launch over the alpha rows of several jobs (a job = one vector
// of one space): the grid is what fits on the GPU at once, and each CTA claims
// the next row of the concatenated job list from a device counter until the
// list is exhausted. Row b is row b - cta_off[j] of job j, the last j with
// cta_off[j] <= b; jobs are ordered heaviest rows first, each job's rows in its
// own work order. Jobs are independent, so results equal per-job launches.
template <typename T, int kThreads>
__global__ void __launch_bounds__(kThreads) k_sigma_batch(const SigArgs<T> *__restrict__ jobs,
                                                          const int64_t *__restrict__ cta_off, int njobs,
                                                          int64_t nrows, int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SigArgs<T> sA;
    __shared__ int64_t sRow, sNext;
    for (;;) {
        if (threadIdx.x == 0) sNext = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t b = sNext;
        if (b >= nrows) break;  // block-uniform
        if (threadIdx.x == 0) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cta_off[mid] <= b) lo = mid;
                else hi = mid - 1;
            }
            sA = jobs[lo];
            sRow = sA.rowsa[b - cta_off[lo]];
        }
        __syncthreads();
        sigma_row<T, 1, true, true, kThreads>(sA, sRow, smem_raw);
        __syncthreads();  // sA, sRow and shared memory are reused by the next row
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
void set_sell(SigArgs<T> &A, const Plan *P) {
    A.s1_off = P->d_s1_off.p;
    A.s2_off = P->d_s2_off.p;
    A.d2_off = P->d_d2_off.p;
    A.s1_w = P->d_s1_w.p;
    A.s2_w = P->d_s2_w.p;
    A.d2_w = P->d_d2_w.p;
    A.s1_ci = P->d_s1_ci.p;
    A.s2_ci = P->d_s2_ci.p;
    A.d2_col = P->d_d2_col.p;
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
    A.permb2 = P->d_permb2.p;
    A.rowsa = P->d_rowsa.p;
    A.ecore = ham->ecore;
    A.s2_val = P->d_s2_val.p;
    A.d2_val = P->d_d2_val.p;
    A.U1 = P->d_U1.p;
    A.U2 = P->d_U2.p;
    A.Eb2 = P->d_Eb2.p;
    set_sell(A, P);
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
    A.permb2 = P->d_permb2.p;
    A.rowsa = P->d_rowsa.p;
    A.ecore = (float)ham->ecore;
    A.s2_val = P->d_s2_valf.p;
    A.d2_val = P->d_d2_valf.p;
    A.U1 = P->d_U1f.p;
    A.U2 = P->d_U2f.p;
    A.Eb2 = P->d_Eb2f.p;
    set_sell(A, P);
    return A;
}

template <typename T>
size_t smem_bytes(int npair, int64_t lb, int nv, bool stage, bool accs) {
    size_t head = ((2 * npair + 2) * sizeof(T) + 64 * sizeof(int) + 15) & ~size_t(15);
    return head + ((stage ? 1 : 0) + (accs ? 1 : 0)) * (size_t)nv * lb * sizeof(T);
}

template <typename T, int NV, bool STAGE, bool ACCS, int TH>
tbsci_status launch_th(tbsci_ctx *ctx, SigArgs<T> A, size_t smem, cudaStream_t st) {
    auto kern = k_sigma<T, NV, STAGE, ACCS, TH>;
    TB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TraceScope tr(ctx, "k_sigma", st);
    kern<<<(unsigned)A.la, TH, smem, st>>>(A);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

// threads per CTA: 0 = by row length (16 warps on long rows, 4 on short ones)
template <typename T, int NV, bool STAGE, bool ACCS>
tbsci_status launch_one(tbsci_ctx *ctx, SigArgs<T> A, size_t smem, cudaStream_t st, int threads) {
    if (threads == 0) threads = A.lb >= 1024 ? 512 : 128;
    if (threads == 512) return launch_th<T, NV, STAGE, ACCS, 512>(ctx, A, smem, st);
    if (threads == 256) return launch_th<T, NV, STAGE, ACCS, 256>(ctx, A, smem, st);
    return launch_th<T, NV, STAGE, ACCS, 128>(ctx, A, smem, st);
}

// Shared-memory use of a launch: stage = 0 stages the c row and accumulates the
// sigma row in shared memory when both fit, else accumulates only, else neither;
// stage = 1 at most accumulates; stage = 2 keeps both in global memory (full
// occupancy on long rows). Returns 0 / 1 / 2 for the variant that runs.
template <typename T>
int stage_variant(const tbsci_ctx *ctx, int npair, int64_t lb, int nv, int stage) {
    if (stage == 0 && smem_bytes<T>(npair, lb, nv, true, true) <= ctx->smem_optin) return 0;
    if (stage <= 1 && smem_bytes<T>(npair, lb, nv, false, true) <= ctx->smem_optin) return 1;
    return 2;
}

template <typename T, int NV>
tbsci_status launch_nv(tbsci_ctx *ctx, SigArgs<T> A, cudaStream_t st, int threads, int stage) {
    switch (stage_variant<T>(ctx, A.npair, A.lb, NV, stage)) {
        case 0: return launch_one<T, NV, true, true>(ctx, A, smem_bytes<T>(A.npair, A.lb, NV, true, true), st, threads);
        case 1:
            return launch_one<T, NV, false, true>(ctx, A, smem_bytes<T>(A.npair, A.lb, NV, false, true), st, threads);
        default:
            return launch_one<T, NV, false, false>(ctx, A, smem_bytes<T>(A.npair, A.lb, NV, false, false), st,
                                                   threads);
    }
}

// nv_max / threads: 0 = defaults (as many vectors per CTA as fit with staging, up
// to 4); stage: -1 = the plan's tuned mode, else 0 (see stage_variant). rows /
// nrows: launch only these alpha rows (autotuning on a sample), NULL = all.
template <typename T>
tbsci_status launch_typed(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *P, const T *c, T *s, int nvec,
                          cudaStream_t st, int nv_max = 0, int threads = 0, int stage = -1,
                          const int32_t *rows = nullptr, int64_t nrows = 0) {
    SigArgs<T> A = make_args<T>(ham, P);
    if (A.la == 0 || A.lb == 0) return TBSCI_OK;
    const int ti = sizeof(T) == 8 ? 0 : 1;
    if (nv_max == 0 && P->tune_nv[ti] > 0) {
        nv_max = P->tune_nv[ti];
        threads = P->tune_threads[ti];
        if (stage < 0) stage = P->tune_stage[ti];
    }
    if (stage < 0) stage = 0;
    if (stage >= 3)  // rows longer than shared memory: column parts + double-class products
        return split_launch<T>(ctx, ham, const_cast<Plan *>(P), c, s, nvec, stage - 3, threads, rows, nrows, st,
                               rows ? 1 : 0);
    if (rows) {  // grid over the sample; vstride keeps the full row count
        A.rowsa = rows;
        A.la = nrows;
    }
    int v = 0;
    while (v < nvec) {
        int rem = nvec - v;
        int nv = std::min(rem, nv_max > 0 ? nv_max : 4);
        while (stage == 0 && nv > 1 && smem_bytes<T>(A.npair, A.lb, nv, true, true) > ctx->smem_optin) --nv;
        A.C = c + (size_t)v * A.vstride;
        A.S = s + (size_t)v * A.vstride;
        switch (nv) {
            case 4: TB_TRY((launch_nv<T, 4>(ctx, A, st, threads, stage))); break;
            case 3: TB_TRY((launch_nv<T, 3>(ctx, A, st, threads, stage))); break;
            case 2: TB_TRY((launch_nv<T, 2>(ctx, A, st, threads, stage))); break;
            default: TB_TRY((launch_nv<T, 1>(ctx, A, st, threads, stage))); break;
        }
        v += nv;
    }
    return TBSCI_OK;
}

constexpr int kBatchThreads = 256;  // CTA size of jobs whose space has no tuned shape

template <typename T, int TH>
tbsci_status launch_batch_th(tbsci_ctx *ctx, const SigArgs<T> *dargs, const int64_t *doff, int njobs, int64_t rows,
                             int *counter, size_t smem, cudaStream_t st) {
    auto kern = k_sigma_batch<T, TH>;
    TB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TH, smem));
    const int64_t grid = std::min<int64_t>(rows, (int64_t)std::max(1, per_sm) * ctx->num_sms);
    TB_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), st));
    TraceScope tr(ctx, "k_sigma_batch", st);
    kern<<<(unsigned)grid, TH, smem, st>>>(dargs, doff, njobs, rows, counter);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

template <typename T>
tbsci_status launch_batch_typed(tbsci_ctx *ctx, const SigmaJob *jobs, int njobs, cudaStream_t st, BatchScratch *scr) {
    const int ti = sizeof(T) == 8 ? 0 : 1;
    // one persistent launch per CTA size: each space's tuned size when it has one
    struct Item {
        SigArgs<T> a;
        double row_work;
        int threads;
    };
    std::vector<Item> items;
    size_t smem[3] = {0, 0, 0};
    for (int j = 0; j < njobs; ++j) {
        SigArgs<T> A = make_args<T>(jobs[j].ham, jobs[j].plan);
        if (A.la == 0 || A.lb == 0) continue;
        const size_t sm = smem_bytes<T>(A.npair, A.lb, 1, true, true);
        if (sm > ctx->smem_optin) {  // rows too long to stage: a launch of its own
            TB_TRY(launch_typed<T>(ctx, jobs[j].ham, jobs[j].plan, static_cast<const T *>(jobs[j].c),
                                   static_cast<T *>(jobs[j].s), jobs[j].nvec, st));
            continue;
        }
        const Plan *P = jobs[j].plan;
        int th = P->tune_threads[ti] > 0 && P->tune_threads[ti] <= 512 ? P->tune_threads[ti] : kBatchThreads;
        const int g = th == 512 ? 2 : th == 256 ? 1 : 0;
        th = g == 2 ? 512 : g == 1 ? 256 : 128;
        smem[g] = std::max(smem[g], sm);
        const double work = (double)P->counts.nnz / (double)std::max<int64_t>(1, A.la);
        for (int v = 0; v < jobs[j].nvec; ++v) {
            A.C = static_cast<const T *>(jobs[j].c) + (size_t)v * A.vstride;
            A.S = static_cast<T *>(jobs[j].s) + (size_t)v * A.vstride;
            items.push_back({A, work, th});
        }
    }
    if (items.empty()) return TBSCI_OK;
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) {
        return x.threads != y.threads ? x.threads > y.threads : x.row_work > y.row_work;
    });
    std::vector<SigArgs<T>> args;
    std::vector<int64_t> off;
    struct Group {
        int threads;
        int first, count;
        int64_t rows;
    };
    std::vector<Group> groups;
    int64_t rows = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        if (groups.empty() || groups.back().threads != items[i].threads) {
            groups.push_back({items[i].threads, (int)i, 0, 0});
            rows = 0;
        }
        args.push_back(items[i].a);
        off.push_back(rows);
        rows += items[i].a.la;
        groups.back().count++;
        groups.back().rows = rows;
    }
    const size_t abytes = args.size() * sizeof(SigArgs<T>), obytes = off.size() * sizeof(int64_t);
    const size_t aoff = (abytes + 255) & ~size_t(255), coff = (aoff + obytes + 255) & ~size_t(255);
    const size_t need = coff + 16 * sizeof(int);
    // double-buffered pinned staging: wait for the copy that last used this half
    const int half = scr->flip ^= 1;
    if (scr->h_bytes[half] < need) {
        if (scr->h_stage[half]) {
            TB_CUDA(ctx, cudaEventSynchronize(scr->copied[half]));
            cudaFreeHost(scr->h_stage[half]);
            scr->h_stage[half] = nullptr;
            scr->h_bytes[half] = 0;
        }
        TB_CUDA(ctx, cudaMallocHost(&scr->h_stage[half], 2 * need));
        scr->h_bytes[half] = 2 * need;
    }
    if (!scr->copied[half]) TB_CUDA(ctx, cudaEventCreateWithFlags(&scr->copied[half], cudaEventDisableTiming));
    TB_CUDA(ctx, cudaEventSynchronize(scr->copied[half]));
    unsigned char *h = static_cast<unsigned char *>(scr->h_stage[half]);
    std::memcpy(h, args.data(), abytes);
    std::memcpy(h + aoff, off.data(), obytes);
    if (scr->d_stage.n < need) TB_CUDA(ctx, scr->d_stage.alloc(2 * need));
    TB_CUDA(ctx, cudaMemcpyAsync(scr->d_stage.p, h, coff, cudaMemcpyHostToDevice, st));
    TB_CUDA(ctx, cudaEventRecord(scr->copied[half], st));
    const SigArgs<T> *dargs = reinterpret_cast<const SigArgs<T> *>(scr->d_stage.p);
    const int64_t *doff = reinterpret_cast<const int64_t *>(scr->d_stage.p + aoff);
    int *counters = reinterpret_cast<int *>(scr->d_stage.p + coff);
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const Group &g = groups[gi];
        const int sl = g.threads == 512 ? 2 : g.threads == 256 ? 1 : 0;
        const SigArgs<T> *ga = dargs + g.first;
        const int64_t *go = doff + g.first;
        int *ctr = counters + gi;
        TB_CHECK(ctx, g.rows <= INT32_MAX, TBSCI_EINVAL, "batched sigma: too many rows in one launch");
        if (g.threads == 512) TB_TRY((launch_batch_th<T, 512>(ctx, ga, go, g.count, g.rows, ctr, smem[sl], st)));
        else if (g.threads == 256) TB_TRY((launch_batch_th<T, 256>(ctx, ga, go, g.count, g.rows, ctr, smem[sl], st)));
        else TB_TRY((launch_batch_th<T, 128>(ctx, ga, go, g.count, g.rows, ctr, smem[sl], st)));
    }
    return TBSCI_OK;
}

}  // namespace

BatchScratch::~BatchScratch() {
    for (int i = 0; i < 2; ++i) {
        if (copied[i]) {
            cudaEventSynchronize(copied[i]);
            cudaEventDestroy(copied[i]);
        }
        if (h_stage[i]) cudaFreeHost(h_stage[i]);
    }
}

tbsci_status sigma_launch_batch(tbsci_ctx *ctx, const SigmaJob *jobs, int njobs, tbsci_dtype dt, cudaStream_t st,
                                BatchScratch *scr) {
    if (dt == TBSCI_F64) return launch_batch_typed<double>(ctx, jobs, njobs, st, scr);
    if (dt == TBSCI_F32) return launch_batch_typed<float>(ctx, jobs, njobs, st, scr);
    for (int j = 0; j < njobs; ++j)
        TB_TRY(sigma_launch(ctx, jobs[j].ham, jobs[j].plan, jobs[j].c, jobs[j].s, jobs[j].nvec, dt, st));
    return TBSCI_OK;
}

void tune_cache_record(tbsci_ctx *ctx, const Plan *plan, int64_t la, int64_t lb) {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    tbsci_ctx::TuneEntry &e = ctx->tune_cache[{plan->norb, la, lb}];
    for (int i = 0; i < 2; ++i)
        if (plan->tune_nv[i] > 0) {
            e.threads[i] = plan->tune_threads[i];
            e.nv[i] = plan->tune_nv[i];
            e.stage[i] = plan->tune_stage[i];
        }
    if (plan->tune_rest_threads > 0) {
        e.rest_mode = plan->tune_rest_mode;
        e.rest_threads = plan->tune_rest_threads;
    }
}

void tune_cache_apply(tbsci_ctx *ctx, Plan *plan, int64_t la, int64_t lb) {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    auto it = ctx->tune_cache.find({plan->norb, la, lb});
    if (it == ctx->tune_cache.end()) return;
    const tbsci_ctx::TuneEntry &e = it->second;
    for (int i = 0; i < 2; ++i)
        if (e.nv[i] > 0) {
            plan->tune_threads[i] = e.threads[i];
            plan->tune_nv[i] = e.nv[i];
            plan->tune_stage[i] = e.stage[i];
        }
    if (e.rest_threads > 0) {
        plan->tune_rest_mode = e.rest_mode;
        plan->tune_rest_threads = e.rest_threads;
    }
}

namespace {

// alpha rows per SM in the autotuner's sample of a large space: several waves of
// CTAs at every CTA size, so tail and occupancy effects match a full launch
constexpr int kTuneRowsPerSm = 64;

int rest_variant(const tbsci_ctx *ctx, int npair, int64_t lb, int mode, bool pairs);

// Tensor-core sigma types: the tensor-core kernel has one shape; this times the
// SIMT pass for the other classes over its shared-memory modes and CTA sizes (on
// a sample of 64 alpha rows per SM when one pass takes 100 ms or more), keeps the
// fastest, then runs the whole sigma once and reports its time.
tbsci_status autotune_rest(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *plan, const float *c, float *s, int nvec,
                           tbsci_dtype dt, cudaStream_t st, double *best_ms) {
    const int64_t la = plan->A.l, lb = plan->B.l;
    const int npair = ham->norb * (ham->norb + 1) / 2;
    cudaEvent_t e0, e1;
    TB_CUDA(ctx, cudaEventCreate(&e0));
    TB_CUDA(ctx, cudaEventCreate(&e1));
    auto timed = [&](auto &&launch, int reps, float *ms_out) -> tbsci_status {
        float tot = 0.f;
        for (int rep = 0; rep <= reps; ++rep) {
            TB_CUDA(ctx, cudaEventRecord(e0, st));
            TB_TRY(launch());
            TB_CUDA(ctx, cudaEventRecord(e1, st));
            TB_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            TB_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tot += ms;
        }
        *ms_out = tot / reps;
        return TBSCI_OK;
    };
    float probe = 0.f;
    tbsci_status ret = timed([&] { return sigma_launch_rest(ctx, ham, plan, c, s, nvec, st, 0, 0, nullptr, 0,
                                                            dt == TBSCI_F32_TC_BF16); }, 1, &probe);
    // a strided sample of the work-ordered rows (and of the row pairs, for the
    // pair variants: the same number of rows)
    DevBuf<int32_t> dsample, dpsample;
    const int32_t *rows = nullptr, *prows = nullptr;
    int64_t nrows = 0, nprows = 0;
    const bool pairs = plan->d_pairs.p != nullptr;
    auto sample_of = [&](const int32_t *src, int64_t n, int64_t k, DevBuf<int32_t> &dst) -> tbsci_status {
        std::vector<int32_t> all(n), sample(k);
        cudaError_t e = cudaMemcpy(all.data(), src, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
        for (int64_t j = 0; j < k; ++j) sample[j] = all[(j * n) / k];
        if (e == cudaSuccess) e = dst.alloc(k);
        if (e == cudaSuccess) e = cudaMemcpy(dst.p, sample.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? TBSCI_OK : fail(ctx, TBSCI_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    };
    if (ret == TBSCI_OK && probe >= 100.f) {
        nrows = std::min<int64_t>(la, kTuneRowsPerSm * (int64_t)ctx->num_sms);
        ret = sample_of(plan->d_rowsa.p, la, nrows, dsample);
        rows = dsample.p;
        if (ret == TBSCI_OK && pairs) {
            nprows = std::max<int64_t>(1, nrows / 2);
            ret = sample_of(plan->d_pairs.p, la / 2, nprows, dpsample);
            prows = dpsample.p;
        }
    }
    const int threads[3] = {128, 256, 512};
    float best = 1e30f;
    int bm = 0, bt = 0;
    bool seen[8] = {false, false, false, false, false, false, false, false};
    const bool bf16 = dt == TBSCI_F32_TC_BF16;
    // modes 4 (column-tiled products) and 5 (dense products) run on the whole
    // space; their time counts in proportion to the sample when the others are
    // timed on one. Mode 5 is skipped when its dense matrices do not fit the
    // context's budget or the device (the failed set-up leaves the plan as it was).
    for (int mode = 4; mode <= 5 && ret == TBSCI_OK; ++mode) {
        float ms = 0.f;
        tbsci_status r5 = timed([&] { return sigma_launch_rest(ctx, ham, plan, c, s, nvec, st, mode, 256, nullptr, 0,
                                                               bf16); }, 1, &ms);
        if (mode == 5 && r5 == TBSCI_ENOMEM) continue;
        ret = r5;
        const float scaled = rows ? ms * (float)nrows / (float)la : ms;
        if (ret == TBSCI_OK && scaled < best) {
            best = scaled;
            bm = mode;
            bt = 256;
        }
        seen[mode == 4 ? 6 : 7] = true;
    }
    for (int mode = 0; mode < 4 && ret == TBSCI_OK; ++mode) {
        const int var = rest_variant(ctx, npair, lb, mode, pairs);
        if (seen[var]) continue;
        seen[var] = true;
        const int32_t *r = var >= 4 ? prows : rows;
        const int64_t nr = var >= 4 ? nprows : nrows;
        for (int t = 0; t < 3 && ret == TBSCI_OK; ++t) {
            float ms = 0.f;
            ret = timed([&] { return sigma_launch_rest(ctx, ham, plan, c, s, nvec, st, mode, threads[t], r, nr, bf16); },
                        rows ? 1 : 2, &ms);
            if (ret == TBSCI_OK && ms < best) {
                best = ms;
                bm = mode;
                bt = threads[t];
            }
        }
    }
    if (ret == TBSCI_OK) {
        plan->tune_rest_mode = bm;
        plan->tune_rest_threads = bt;
        float ms = 0.f;
        ret = timed([&] { return sigma_launch(ctx, ham, plan, c, s, nvec, dt, st); }, 1, &ms);
        if (ret == TBSCI_OK && best_ms) *best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ret;
}

}  // namespace

namespace {

// time of the split path's parts that do not depend on the row kernel's shape
template <typename T>
tbsci_status timed_split(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *plan, const T *c, T *s, cudaStream_t st,
                         cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    TB_TRY(split_launch<T>(ctx, ham, plan, c, s, 1, 0, 512, nullptr, 0, st, 2));  // warm-up, scratch
    TB_CUDA(ctx, cudaEventRecord(e0, st));
    TB_TRY(split_launch<T>(ctx, ham, plan, c, s, 1, 0, 512, nullptr, 0, st, 2));
    TB_CUDA(ctx, cudaEventRecord(e1, st));
    TB_CUDA(ctx, cudaEventSynchronize(e1));
    TB_CUDA(ctx, cudaEventElapsedTime(ms, e0, e1));
    return TBSCI_OK;
}

}  // namespace

tbsci_status sigma_autotune(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *plan, const void *c, void *s, int nvec,
                            tbsci_dtype dt, cudaStream_t st, double *best_ms) {
    TB_CHECK(ctx, dt == TBSCI_F64 || dt == TBSCI_F32 || dt == TBSCI_F32_TC_TF32 || dt == TBSCI_F32_TC_BF16,
             TBSCI_EINVAL, "autotune: unknown dtype");
    const int64_t la = plan->A.l, lb = plan->B.l;
    if (la == 0 || lb == 0 || nvec <= 0) return TBSCI_OK;
    if (dt == TBSCI_F32_TC_TF32 || dt == TBSCI_F32_TC_BF16) {
        if (plan->npoff > 128 || !plan->d_lbp.p) dt = TBSCI_F32;  // these run on the SIMT path
        else return autotune_rest(ctx, ham, plan, static_cast<const float *>(c), static_cast<float *>(s), nvec, dt,
                                  st, best_ms);
    }
    const int ti = dt == TBSCI_F64 ? 0 : 1;
    const int npair = ham->norb * (ham->norb + 1) / 2;
    cudaEvent_t e0, e1;
    TB_CUDA(ctx, cudaEventCreate(&e0));
    TB_CUDA(ctx, cudaEventCreate(&e1));
    // runs one candidate `reps` times after one warm-up run; mean ms of the timed runs
    auto trial = [&](int nv, int th, int stage, const int32_t *rows, int64_t nrows, int reps, float *ms_out) {
        float tot = 0.f;
        for (int rep = 0; rep <= reps; ++rep) {
            TB_CUDA(ctx, cudaEventRecord(e0, st));
            TB_TRY(dt == TBSCI_F64 ? launch_typed<double>(ctx, ham, plan, static_cast<const double *>(c),
                                                          static_cast<double *>(s), nvec, st, nv, th, stage, rows,
                                                          nrows)
                                   : launch_typed<float>(ctx, ham, plan, static_cast<const float *>(c),
                                                         static_cast<float *>(s), nvec, st, nv, th, stage, rows,
                                                         nrows));
            TB_CUDA(ctx, cudaEventRecord(e1, st));
            TB_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            TB_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tot += ms;
        }
        *ms_out = tot / reps;
        return TBSCI_OK;
    };
    auto variant = [&](int nv, int stage) {
        return dt == TBSCI_F64 ? stage_variant<double>(ctx, npair, lb, nv, stage)
                               : stage_variant<float>(ctx, npair, lb, nv, stage);
    };
    const int threads[3] = {128, 256, 512};
    const int nvmax = std::min(nvec, 4);
    auto cu = [&](cudaError_t e) { return e == cudaSuccess ? TBSCI_OK : fail(ctx, TBSCI_ECUDA, std::string("autotune: ") + cudaGetErrorString(e)); };
    float best = 1e30f, probe = 0.f;
    int bt = 0, bn = 0, bs = 0;
    tbsci_status ret = trial(1, 0, 0, nullptr, 0, 1, &probe);
    if (ret == TBSCI_OK && probe < 100.f) {
        // small space: every shape on the whole space
        for (int nv = 1; nv <= nvmax && ret == TBSCI_OK; ++nv) {
            bool seen[3] = {false, false, false};
            for (int stage = 0; stage < 3 && ret == TBSCI_OK; ++stage) {
                const int var = variant(nv, stage);
                if (seen[var]) continue;
                seen[var] = true;
                for (int t = 0; t < 3 && ret == TBSCI_OK; ++t) {
                    float ms = 0.f;
                    ret = trial(nv, threads[t], stage, nullptr, 0, 2, &ms);
                    if (ret == TBSCI_OK && ms < best) {
                        best = ms;
                        bt = threads[t];
                        bn = nv;
                        bs = stage;
                    }
                }
            }
        }
    } else if (ret == TBSCI_OK) {
        // large space: time a strided sample of the work-ordered alpha rows
        // (several waves of CTAs, so tails and occupancy show as in a full launch),
        // staging mode and CTA size at one vector per CTA first,
        // then the vectors per CTA at that choice
        const int64_t nrows = std::min<int64_t>(la, kTuneRowsPerSm * (int64_t)ctx->num_sms);
        std::vector<int32_t> all(la), sample(nrows);
        DevBuf<int32_t> dsample;
        ret = cu(cudaMemcpy(all.data(), plan->d_rowsa.p, la * sizeof(int32_t), cudaMemcpyDeviceToHost));
        for (int64_t j = 0; j < nrows; ++j) sample[j] = all[(j * la) / nrows];
        if (ret == TBSCI_OK) ret = cu(dsample.alloc(nrows));
        if (ret == TBSCI_OK)
            ret = cu(cudaMemcpy(dsample.p, sample.data(), nrows * sizeof(int32_t), cudaMemcpyHostToDevice));
        bool seen[3] = {false, false, false};
        for (int stage = 0; stage < 3 && ret == TBSCI_OK; ++stage) {
            const int var = variant(1, stage);
            if (seen[var]) continue;
            seen[var] = true;
            for (int t = 0; t < 3 && ret == TBSCI_OK; ++t) {
                float ms = 0.f;
                ret = trial(1, threads[t], stage, dsample.p, nrows, 1, &ms);
                if (ret == TBSCI_OK && ms < best) {
                    best = ms;
                    bt = threads[t];
                    bn = 1;
                    bs = stage;
                }
            }
        }
        // split path (rows longer than shared memory): the row kernel is timed on
        // the sample; the double-class products, transposes and combine do not
        // depend on its shape, so their full-space time is measured once and
        // added in proportion to the sample
        if (ret == TBSCI_OK && variant(1, 0) != 0 && split_min_parts(ctx, npair, plan->norb, lb, ti == 0 ? 8 : 4, 0) >= 1) {
            float fixed = 0.f;
            ret = dt == TBSCI_F64
                      ? timed_split<double>(ctx, ham, plan, static_cast<const double *>(c), static_cast<double *>(s),
                                            st, e0, e1, &fixed)
                      : timed_split<float>(ctx, ham, plan, static_cast<const float *>(c), static_cast<float *>(s),
                                           st, e0, e1, &fixed);
            const float share = fixed * (float)nrows / (float)la;
            const int split_threads[2] = {512, 1024};
            for (int stage = 3; stage <= 6 && ret == TBSCI_OK; ++stage)
                for (int t = 0; t < 2 && ret == TBSCI_OK; ++t) {
                    float ms = 0.f;
                    ret = trial(1, split_threads[t], stage, dsample.p, nrows, 1, &ms);
                    if (ret == TBSCI_OK && ms + share < best) {
                        best = ms + share;
                        bt = split_threads[t];
                        bn = 1;
                        bs = stage;
                    }
                }
        }
        if (bs < 3)
            for (int nv = 2; nv <= nvmax && ret == TBSCI_OK; ++nv) {
                float ms = 0.f;
                ret = trial(nv, bt, bs, dsample.p, nrows, 1, &ms);
                if (ret == TBSCI_OK && ms < best) {
                    best = ms;
                    bn = nv;
                }
            }
    }
    if (ret == TBSCI_OK) {
        plan->tune_threads[ti] = bt;
        plan->tune_nv[ti] = bn;
        plan->tune_stage[ti] = bs;
        // the chosen shape on the whole space: leaves sigma computed, and its time
        float ms = 0.f;
        ret = trial(0, 0, -1, nullptr, 0, 1, &ms);
        if (ret == TBSCI_OK && best_ms) *best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ret;
}

namespace {

template <bool STAGE, bool ACCS, int TH>
tbsci_status launch_rest_th(tbsci_ctx *ctx, const SigArgs<float> &A, cudaStream_t st) {
    const size_t sm = smem_bytes<float>(A.npair, A.lb, 1, STAGE, ACCS);
    auto k = k_sigma<float, 1, STAGE, ACCS, TH, true>;
    TB_CUDA(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    TraceScope tr(ctx, "k_sigma_rest", st);
    k<<<(unsigned)A.la, TH, sm, st>>>(A);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

template <bool STAGE, int TH>
tbsci_status launch_rest_pair_th(tbsci_ctx *ctx, const SigArgs<float> &A, cudaStream_t st) {
    const size_t sm = smem_bytes<float>(A.npair, A.lb, 2, STAGE, false);
    auto k = k_sigma_rest_pair<STAGE, TH>;
    TB_CUDA(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    TraceScope tr(ctx, "k_sigma_rest_pair", st);
    k<<<(unsigned)A.la, TH, sm, st>>>(A);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

template <bool STAGE>
tbsci_status launch_rest_pair(tbsci_ctx *ctx, const SigArgs<float> &A, cudaStream_t st, int threads) {
    if (threads == 512) return launch_rest_pair_th<STAGE, 512>(ctx, A, st);
    if (threads == 256) return launch_rest_pair_th<STAGE, 256>(ctx, A, st);
    return launch_rest_pair_th<STAGE, 128>(ctx, A, st);
}

template <bool STAGE, bool ACCS>
tbsci_status launch_rest_v(tbsci_ctx *ctx, const SigArgs<float> &A, cudaStream_t st, int threads) {
    if (threads == 512) return launch_rest_th<STAGE, ACCS, 512>(ctx, A, st);
    if (threads == 256) return launch_rest_th<STAGE, ACCS, 256>(ctx, A, st);
    return launch_rest_th<STAGE, ACCS, 128>(ctx, A, st);
}

// Variant of the SIMT pass for a shared-memory mode: 0 = c row staged and sigma
// row accumulated in shared memory where both fit (else the sigma row only, else
// neither); 1 = c row only (the pass writes each sigma element once and reads it
// once, so a global accumulator costs little and frees shared memory); 2 = neither;
// 3 = two alpha rows per CTA sharing the beta links, their c rows staged where
// they fit (even l_alpha only, else as mode 1). Returns 0 (c + sigma), 1 (sigma
// only), 2 (c only), 3 (neither), 4 (row pairs, c staged) or 5 (row pairs).
int rest_variant(const tbsci_ctx *ctx, int npair, int64_t lb, int mode, bool pairs) {
    const size_t lim = ctx->smem_optin;
    if (mode == 4) return 6;  // column-tiled products (rest_products_launch)
    if (mode == 5) return 7;  // dense products on the tensor cores (rest_dense_launch)
    if (mode == 3 && pairs) return smem_bytes<float>(npair, lb, 2, true, false) <= lim ? 4 : 5;
    if (mode == 3) mode = 1;
    if (mode == 0) {
        if (smem_bytes<float>(npair, lb, 1, true, true) <= lim) return 0;
        if (smem_bytes<float>(npair, lb, 1, false, true) <= lim) return 1;
        return 3;
    }
    if (mode == 1 && smem_bytes<float>(npair, lb, 1, true, false) <= lim) return 2;
    return 3;
}

}  // namespace

// The classes the tensor-core kernel leaves out (same-spin beta singles and
// doubles, alpha doubles), FP32, one launch per vector. mode / threads: -1 / 0 =
// the plan's tuned choice (default: mode 0, 512 threads on rows of >= 1024
// columns, else 128); rows / nrows: launch only these alpha rows (tuning sample;
// for the row-pair variants: these even pair starts).
tbsci_status sigma_launch_rest(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const float *c, float *s,
                               int nvec, cudaStream_t st, int mode, int threads, const int32_t *rows, int64_t nrows,
                               bool bf16) {
    SigArgs<float> A = make_args<float>(ham, plan);
    if (A.la == 0 || A.lb == 0) return TBSCI_OK;
    if (mode < 0) {
        mode = plan->tune_rest_mode;
        threads = plan->tune_rest_threads;
    }
    if (threads == 0) threads = A.lb >= 1024 ? 512 : 128;
    const int var = rest_variant(ctx, A.npair, A.lb, mode, plan->d_pairs.p != nullptr);
    if (var == 6) return rest_products_launch(ctx, ham, const_cast<Plan *>(plan), c, s, nvec, st);
    if (var == 7) return rest_dense_launch(ctx, ham, const_cast<Plan *>(plan), c, s, nvec, bf16, st);
    if (var >= 4) {
        // row pairs: one vector per launch with vstride = l_beta, pair starts as rows
        SigArgs<float> P = A;
        P.vstride = A.lb;
        P.rowsa = rows ? rows : plan->d_pairs.p;
        P.la = rows ? nrows : A.la / 2;
        for (int v = 0; v < nvec; ++v) {
            P.C = c + (size_t)v * A.vstride;
            P.S = s + (size_t)v * A.vstride;
            if (var == 4) TB_TRY(launch_rest_pair<true>(ctx, P, st, threads));
            else TB_TRY(launch_rest_pair<false>(ctx, P, st, threads));
        }
        return TBSCI_OK;
    }
    if (rows) {
        A.rowsa = rows;
        A.la = nrows;
    }
    for (int v = 0; v < nvec; ++v) {
        A.C = c + (size_t)v * A.vstride;
        A.S = s + (size_t)v * A.vstride;
        switch (var) {
            case 0: TB_TRY((launch_rest_v<true, true>(ctx, A, st, threads))); break;
            case 1: TB_TRY((launch_rest_v<false, true>(ctx, A, st, threads))); break;
            case 2: TB_TRY((launch_rest_v<true, false>(ctx, A, st, threads))); break;
            default: TB_TRY((launch_rest_v<false, false>(ctx, A, st, threads))); break;
        }
    }
    return TBSCI_OK;
}

tbsci_status sigma_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const void *c, void *s, int nvec,
                          tbsci_dtype dt, cudaStream_t st) {
    if (dt == TBSCI_F64)
        return launch_typed<double>(ctx, ham, plan, static_cast<const double *>(c), static_cast<double *>(s), nvec, st);
    if (dt == TBSCI_F32)
        return launch_typed<float>(ctx, ham, plan, static_cast<const float *>(c), static_cast<float *>(s), nvec, st);
    if (dt == TBSCI_F32_TC_TF32 || dt == TBSCI_F32_TC_BF16) {
        const float *cf = static_cast<const float *>(c);
        float *sf = static_cast<float *>(s);
        if (plan->npoff > 128 || !plan->d_lbp.p)  // no tensor-core tile for this norb: FP32 on the SIMT path
            return launch_typed<float>(ctx, ham, plan, cf, sf, nvec, st);
        TB_TRY(sigma_launch_rest(ctx, ham, plan, cf, sf, nvec, st, -1, 0, nullptr, 0, dt == TBSCI_F32_TC_BF16));
        return sigma_tc_add(ctx, ham, plan, cf, sf, nvec, dt == TBSCI_F32_TC_BF16, st);
    }
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
