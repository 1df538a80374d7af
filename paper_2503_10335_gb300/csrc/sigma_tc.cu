// The alpha-beta classes of sigma on the 5th-generation tensor cores.
//
// For one alpha row Ia (one CTA), with K alpha terms k = (Ja_k, pq_k, s_k):
// k = 0 is Ja = Ia ("W" row: sum_{p in Ia} (pp|rs)), k >= 1 the alpha singles.
//   G[rs][Jb] = sum_k A[rs][k] * F[k][Jb],   A[rs][k] = s_k (pq_k|rs) (k >= 1),
//                                            A[rs][0] = sum_{p in Ia} (pp|rs),
//                                            F[k][Jb] = c(Ja_k, Jb)
// over the off-diagonal orbital pairs rs (one 128-row MMA tile for norb <= 16),
// then sigma(Ia, Ib) += sign * G[rs][Jb] for every beta single link
// Ib = E_rs Jb (the gather D of the classic formulation, done as a scatter from
// the accumulator rows). The beta-diagonal pairs (r = s in Ib), the alpha-single
// string-Hamiltonian values and the whole diagonal are added by the threads that
// stage F, as  (h_a(Ia,Ja_k) + s_k U[pq_k][Jb]) c(Ja_k, Jb)  and
// Hd(Ia, Jb) c(Ia, Jb). Together: classes [1,1], [1,0], [0,1] (alpha-beta
// part) and [0,0] of Sec. II.C; the rest (same-spin beta singles/doubles,
// alpha doubles) comes from the SIMT kernel run first.
//
// Operands are staged in shared memory in the K-major no-swizzle core-matrix
// layout: element (row r, k) at (r/8)*SBO + (k/E)*128 + (r%8)*16 + (k%E)*es,
// E = 16 / es elements per 16-byte core row; tcgen05.mma (cta_group::1,
// M = 128, N = 64) accumulates FP32 in TMEM; tcgen05.ld brings rows back.
// Precision: 3xTF32 (A = Ah + Al, F = Fh + Fl, G = Ah Fh + Ah Fl + Al Fh) for
// FP32-level accuracy, or one BF16 product (fast, ~3 significant digits).
// Every mbarrier wait is bounded; on timeout the CTA records an error, skips
// the rest of its row and still frees its TMEM.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace tbsci {

namespace {

// CTA size: the first half of the warps drains the accumulator, the second
// stages F. Split TF32 writes two planes per staged element and gains from 32
// warps; BF16 staging is lighter and runs best with 16.
template <bool BF16>
__host__ __device__ constexpr int tc_threads() { return BF16 ? 512 : 1024; }
constexpr int kTileN = 64;    // beta columns per MMA tile
constexpr int kTileM = 128;   // off-diagonal pair rows (norb <= 16: <= 120 used)
constexpr int kKStep = 16;    // K padding granule (a BF16 MMA step; two TF32 steps)

struct TcArgs {
    int64_t la, lb;
    const float *C;
    float *S;
    int npair, npoff, na, kmax;
    const uint64_t *stra;
    const int64_t *a_soff;
    const int2 *a_sci;
    const float *a_sval;
    const float *Vf;   // [npair][npair]
    const float *Uf;   // [npair][lb]
    const float *Ea, *Eb;
    float ecore;
    const int32_t *lbp;      // [lb][npoff]
    const int32_t *offpair;  // [npoff]
    const int32_t *rowsa;
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle, base offset 0
    return d;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of element (r, k) in a K-major no-swizzle tile with Kp columns
template <int ES>
__device__ __forceinline__ uint32_t core_off(int r, int k, int Kp) {
    constexpr int E = 16 / ES;
    return (uint32_t)((r >> 3) * (Kp / E) * 128 + (k / E) * 128 + (r & 7) * 16 + (k % E) * ES);
}

template <bool BF16>
__device__ __forceinline__ void put(unsigned char *hi, unsigned char *lo, uint32_t off_hi, uint32_t off_lo, float v) {
    if (BF16) {
        *reinterpret_cast<__nv_bfloat16 *>(hi + off_hi) = __float2bfloat16_rn(v);
    } else {
        const float h = tf32_round(v);
        *reinterpret_cast<float *>(hi + off_hi) = h;
        *reinterpret_cast<float *>(lo + off_lo) = tf32_round(v - h);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(tc_threads<BF16>()) k_sigma_ab_tc(TcArgs A) {
    constexpr int kTcThreads = tc_threads<BF16>();
    constexpr int kEpiThreads = kTcThreads / 2;
    constexpr int kEpiParts = kEpiThreads / 128;  // warps per TMEM lane quarter
    static_assert(kTileN % (16 * kEpiParts) == 0, "each draining warp reads whole 16-column TMEM chunks");
    constexpr int ES = BF16 ? 2 : 4;  // element bytes
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int sJa[256], sPq[256], sOccP[64];
    __shared__ float sSa[256], sHa[256];
    __shared__ int sAbort, sAbortTile;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t lb = A.lb;
    const int64_t Ia = A.rowsa[blockIdx.x];
    const int64_t t0 = A.a_soff[Ia];
    const int K = 1 + (int)(A.a_soff[Ia + 1] - t0);
    const int Kp = (K + kKStep - 1) / kKStep * kKStep;
    const uint32_t a_bytes = (uint32_t)kTileM * Kp * ES, b_bytes = (uint32_t)kTileN * Kp * ES;
    unsigned char *sAh = smem;
    unsigned char *sAl = sAh + (BF16 ? 0 : a_bytes);
    unsigned char *sBh = sAh + (BF16 ? 1 : 2) * a_bytes;  // two F buffers of (BF16 ? 1 : 2) planes each
    float *sAcc = reinterpret_cast<float *>(sBh + 2 * (BF16 ? 1 : 2) * b_bytes);

    // alpha terms of this row
    if (tid == 0) {
        int k = 0;
        for (uint64_t s = A.stra[Ia]; s; s &= s - 1) {
            const int p = __ffsll((long long)s) - 1;
            sOccP[k++] = p * (p + 1) / 2 + p;
        }
        sAbort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    }
    for (int k = tid; k < K; k += kTcThreads) {
        if (k == 0) {
            sJa[0] = (int)Ia;
            sPq[0] = -1;
            sSa[0] = 1.f;
            sHa[0] = 0.f;
        } else {
            const int2 e = A.a_sci[t0 + k - 1];
            sJa[k] = e.x;
            sPq[k] = e.y >> 1;
            sSa[k] = (e.y & 1) ? -1.f : 1.f;
            sHa[k] = A.a_sval[t0 + k - 1];
        }
    }
    for (int64_t j = tid; j < lb; j += kTcThreads) sAcc[j] = 0.f;
    __syncthreads();
    // A[rs][k]: rows = off-diagonal pairs, padded to 128 rows and Kp columns
    for (int x = tid; x < kTileM * Kp; x += kTcThreads) {
        const int r = x / Kp, k = x - r * Kp;
        float v = 0.f;
        if (r < A.npoff && k < K) {
            const int rs = A.offpair[r];
            if (k == 0) {
                for (int i = 0; i < A.na; ++i) v += A.Vf[(size_t)sOccP[i] * A.npair + rs];
            } else {
                v = sSa[k] * A.Vf[(size_t)sPq[k] * A.npair + rs];
            }
        }
        put<BF16>(sAh, sAl, core_off<ES>(r, k, Kp), core_off<ES>(r, k, Kp), v);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kTileN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // instruction descriptor: D F32, A/B BF16 (kind::f16) or TF32 (kind::tf32), K-major, M = 128, N = 64
    const uint32_t idesc = (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
                           ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
    const uint32_t sbo = (uint32_t)(Kp * ES / 16) * 128;
    const int ntiles = (int)((lb + kTileN - 1) / kTileN);

    // F tile t into buffer `buf` by `nth` threads starting at thread `t0`; adds the
    // diagonal, beta-diagonal and alpha-single terms of those columns into sAcc
    auto stage = [&](int t, int buf, int tid0, int nth) {
        const int me = tid - tid0;
        const int jb = me & (kTileN - 1), kstride = nth / kTileN;
        const int64_t Jb = (int64_t)t * kTileN + jb;
        const bool col_ok = Jb < lb;
        unsigned char *bh = sBh + (size_t)buf * (BF16 ? 1 : 2) * b_bytes;
        unsigned char *bl = bh + (BF16 ? 0 : b_bytes);
        float part = 0.f;
        // batches of 8 alpha terms: all loads of a batch are issued before any use
        for (int kb = me / kTileN; kb < Kp; kb += 8 * kstride) {
            float c[8], u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = kb + q * kstride;
                const bool ok = k < K && col_ok;
                c[q] = ok ? __ldg(A.C + (size_t)sJa[k] * lb + Jb) : 0.f;
                u[q] = (ok && k > 0) ? __ldg(A.Uf + (size_t)sPq[k] * lb + Jb) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = kb + q * kstride;
                if (k >= Kp) break;
                if (k < K && col_ok) {
                    float coef;
                    if (k == 0) {
                        coef = A.ecore + A.Ea[Ia] + __ldg(A.Eb + Jb);
                        for (int i = 0; i < A.na; ++i) coef += __ldg(A.Uf + (size_t)sOccP[i] * lb + Jb);
                    } else {
                        coef = sHa[k] + sSa[k] * u[q];
                    }
                    part = fmaf(coef, c[q], part);
                }
                put<BF16>(bh, bl, core_off<ES>(jb, k, Kp), core_off<ES>(jb, k, Kp), c[q]);
            }
        }
        if (col_ok && part != 0.f) atomicAdd(&sAcc[Jb], part);
        asm volatile("fence.proxy.async.shared::cta;");
    };
    auto issue = [&](int t) {
        const int buf = t & 1;
        const uint32_t d = tmem + (uint32_t)(buf * kTileN);
        const uint32_t aH = smem_u32(sAh), aL = smem_u32(sAl);
        const uint32_t bH = smem_u32(sBh + (size_t)buf * (BF16 ? 1 : 2) * b_bytes), bL = bH + (BF16 ? 0 : b_bytes);
        const int ksteps = BF16 ? Kp / 16 : Kp / 8;  // each step = two core columns = 32 bytes of K
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t o = (uint32_t)ks * 256;
            const uint32_t acc0 = ks > 0 ? 1u : 0u;
            const uint64_t dAh = smem_desc(aH + o, 128, sbo), dBh = smem_desc(bH + o, 128, sbo);
            if (BF16) {
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                    "l"(dAh), "l"(dBh), "r"(idesc), "r"(acc0));
            } else {
                const uint64_t dAl = smem_desc(aL + o, 128, sbo), dBl = smem_desc(bL + o, 128, sbo);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                    "l"(dAh), "l"(dBh), "r"(idesc), "r"(acc0));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(dAh), "l"(dBl),
                             "r"(idesc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(dAl), "l"(dBh),
                             "r"(idesc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar[buf])));
    };
    auto wait_tile = [&](int t) -> uint32_t {
        uint32_t done = 0;
        for (int it = 0; it < (1 << 22) && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(smem_u32(&mbar[t & 1])), "r"((uint32_t)((t >> 1) & 1)));
        }
        return done;
    };

    // Pipeline: while the tensor cores run tile t, the staging warps fill the other
    // F buffer with tile t+1 and the draining warps read tile t from its TMEM
    // buffer as soon as its MMAs complete; one barrier per tile.
    if (ntiles > 0) {
        stage(0, 0, 0, kTcThreads);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) issue(0);
    }
    for (int t = 0; t < ntiles; ++t) {
        if (tid >= kEpiThreads) {
            if (t + 1 < ntiles) stage(t + 1, (t + 1) & 1, kEpiThreads, kTcThreads - kEpiThreads);
        } else {
            uint32_t done = __all_sync(0xffffffffu, wait_tile(t));  // warp-uniform: tcgen05.ld is collective
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!done) {
                if (lane == 0) {
                    sAbort = 1;
                    sAbortTile = t;
                }
            } else {
                // a warp reads the TMEM lanes of its quarter (warp % 4); the warps of
                // one quarter split the tile's columns
                const int quarter = warp & 3, part = warp >> 2;
                const int rs = quarter * 32 + lane;
                const int64_t Jb0 = (int64_t)t * kTileN;
                const uint32_t dcol = (uint32_t)((t & 1) * kTileN);
                constexpr int kCols = kTileN / kEpiParts;
#pragma unroll
                for (int c0 = part * kCols; c0 < (part + 1) * kCols; c0 += 16) {
                    uint32_t r[16];
                    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + dcol + (uint32_t)c0;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (rs < A.npoff) {
                        int32_t e[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int64_t col = Jb0 + c0 + j;
                            e[j] = col < lb ? __ldg(A.lbp + col * A.npoff + rs) : -1;
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (e[j] >= 0) {
                                const float g = __uint_as_float(r[j]);
                                atomicAdd(&sAcc[e[j] >> 1], (e[j] & 1) ? -g : g);
                            }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (sAbort) break;
        if (tid == 0 && t + 1 < ntiles) issue(t + 1);
    }
    if (sAbort) {
        // only the timed-out tile's MMAs can still be in flight: give them a second
        // bounded chance to finish before TMEM is freed
        if (tid == 0) {
            wait_tile(sAbortTile);
            atomicExch(A.err, 1);
        }
    } else {
        for (int64_t j = tid; j < lb; j += kTcThreads) A.S[Ia * lb + j] += sAcc[j];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTileN));
}

}  // namespace

tbsci_status sigma_tc_add(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *P, const float *c, float *s, int nvec,
                          bool bf16, cudaStream_t st) {
    const int64_t la = P->A.l, lb = P->B.l;
    if (la == 0 || lb == 0) return TBSCI_OK;
    TB_CHECK(ctx, P->npoff <= kTileM && P->d_lbp.p, TBSCI_EINVAL, "tensor-core sigma needs norb <= 16");
    int kmax = 1;
    for (int64_t i = 0; i < la; ++i) kmax = std::max<int64_t>(kmax, 1 + P->A.h_soff[i + 1] - P->A.h_soff[i]);
    TB_CHECK(ctx, kmax <= 256, TBSCI_EINVAL, "tensor-core sigma: more than 255 alpha singles per string");
    const int kp = (kmax + kKStep - 1) / kKStep * kKStep;
    const size_t es = bf16 ? 2 : 4, planes = bf16 ? 1 : 2;
    const size_t smem = planes * ((size_t)kTileM * kp * es + 2 * (size_t)kTileN * kp * es) + (size_t)lb * sizeof(float);
    TB_CHECK(ctx, smem <= ctx->smem_optin, TBSCI_EINVAL, "tensor-core sigma: row too long for shared memory");
    TcArgs A{};
    A.la = la;
    A.lb = lb;
    A.npair = P->npair;
    A.npoff = P->npoff;
    A.na = P->A.nelec;
    A.kmax = kmax;
    A.stra = P->A.d_str;
    A.a_soff = P->A.d_soff;
    A.a_sci = P->A.d_sci.p;
    A.a_sval = P->A.d_svalf.p;
    A.Vf = ham->d_Vf.p;
    A.Uf = P->d_Uf.p;
    A.Ea = P->A.d_Ef.p;
    A.Eb = P->B.d_Ef.p;
    A.ecore = (float)ham->ecore;
    A.lbp = P->d_lbp.p;
    A.offpair = P->d_offpair.p;
    A.rowsa = P->d_rowsa.p;
    A.err = P->d_tc_err.p;
    auto kern = bf16 ? k_sigma_ab_tc<true> : k_sigma_ab_tc<false>;
    TB_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int v = 0; v < nvec; ++v) {
        A.C = c + (size_t)v * la * lb;
        A.S = s + (size_t)v * la * lb;
        TraceScope tr(ctx, "k_sigma_ab_tc", st);
        kern<<<(unsigned)la, bf16 ? tc_threads<true>() : tc_threads<false>(), smem, st>>>(A);
        TB_CUDA(ctx, cudaGetLastError());
    }
    return TBSCI_OK;
}

}  // namespace tbsci
