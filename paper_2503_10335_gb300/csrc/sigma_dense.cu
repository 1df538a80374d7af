// The same-spin classes of the tensor-core sigma types as dense products
// (rest mode 5): [0,1] + [0,2] (beta singles and doubles) and [2,0] (alpha
// doubles) of Sec. II.C, written as
//   sigma[Ia, Ib] = sum_Jb Hb[Ib, Jb] c[Ia, Jb] + sum_Ja Ha[Ia, Ja] c[Ja, Ib],
// with Hb and Ha the off-diagonal same-spin string Hamiltonians stored dense.
// On a string space close to the full one (norb <= 16, where the tensor-core
// types apply) every beta string couples to several percent of the others
// (848 of 12,870 at norb 16, 8 electrons), so the dense product does ~15x the
// multiply-adds of the sparse one but runs on the tensor cores; the autotuner
// keeps it only where it is faster. Both products are plain GEMMs, so they go
// to cuBLAS. Row-major c (l_a x l_b) is column-major c^T, so with Hb and Ha
// symmetric:  sigma^T = Hb c^T + c^T Ha. The operands are zero-padded to a
// multiple of 32 strings per dimension, so every leading dimension is 128-byte
// aligned (cuBLAS's tensor-core kernels need 16-byte aligned ones).
// Precision follows the sigma type: split TF32 (H = Hh + Hl, c = ch + cl,
// three TF32 products Hh ch + Hh cl + Hl ch, FP32 accumulation: FP32-level
// accuracy) for TBSCI_F32_TC_TF32, one BF16 product for TBSCI_F32_TC_BF16.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace tbsci {

namespace {

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

constexpr int64_t kPad = 32;
inline int64_t padded(int64_t l) { return (l + kPad - 1) / kPad * kPad; }

// One CSR row of same-spin links per thread into a dense matrix with leading
// dimension ld (zeroed before): hi / lo TF32 planes, or one BF16 plane.
__global__ void k_links_to_dense(int64_t l, int64_t ld, const int64_t *__restrict__ off,
                                 const int2 *__restrict__ sci, const int32_t *__restrict__ dcol,
                                 const double *__restrict__ val, float *hi, float *lo, __nv_bfloat16 *bf) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= l) return;
    for (int64_t t = off[r]; t < off[r + 1]; ++t) {
        const int64_t col = sci ? sci[t].x : dcol[t];
        const double v = val[t];
        const size_t at = (size_t)r * ld + col;
        if (bf) {
            bf[at] = __float2bfloat16_rn((float)v);
        } else {
            const float h = to_tf32((float)v);
            hi[at] = h;
            lo[at] = to_tf32((float)(v - (double)h));
        }
    }
}

// c (la x lb) into zero-padded lap x lbp hi / lo TF32 planes, or into BF16
__global__ void k_split_vector(const float *__restrict__ c, int64_t la, int64_t lb, int64_t lap, int64_t lbp,
                               float *hi, float *lo, __nv_bfloat16 *bf) {
    const size_t n = (size_t)lap * lbp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int64_t r = (int64_t)(i / lbp), j = (int64_t)(i - (size_t)r * lbp);
        const float x = (r < la && j < lb) ? c[(size_t)r * lb + j] : 0.f;
        if (bf) {
            bf[i] = __float2bfloat16_rn(x);
        } else {
            const float h = to_tf32(x);
            hi[i] = h;
            lo[i] = to_tf32(x - h);
        }
    }
}

// s (la x lb) = the leading block of the padded product sp (rows of lbp)
__global__ void k_unpad(const float *__restrict__ sp, int64_t la, int64_t lb, int64_t lbp, float *s) {
    const size_t n = (size_t)la * lb;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int64_t r = (int64_t)(i / lb), j = (int64_t)(i - (size_t)r * lb);
        s[i] = sp[(size_t)r * lbp + j];
    }
}

tbsci_status cublas_status(tbsci_ctx *ctx, cublasStatus_t st, const char *what) {
    if (st == CUBLAS_STATUS_SUCCESS) return TBSCI_OK;
    return fail(ctx, st == CUBLAS_STATUS_ALLOC_FAILED ? TBSCI_ENOMEM : TBSCI_ECUDA,
                std::string(what) + ": cuBLAS status " + std::to_string((int)st));
}

// Dense Hb (singles + doubles) and Ha (doubles) of the plan in the planes the
// precision needs; built once per precision.
tbsci_status ensure_dense(tbsci_ctx *ctx, Plan *P, bool bf16, cudaStream_t st) {
    const int64_t la = P->A.l, lb = P->B.l, lap = padded(la), lbp = padded(lb);
    DenseSameSpin &D = P->dense;
    if (bf16 ? D.a_bf.p != nullptr : D.a_hi.p != nullptr) return TBSCI_OK;
    const size_t planes = bf16 ? 1 : 2, es = bf16 ? 2 : 4;
    const size_t bytes = planes * es * ((size_t)lap * lap + (size_t)lbp * lbp);
    TB_TRY(charge(ctx, bytes, "dense same-spin Hamiltonians"));
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto &buf, size_t n) {
        if (e == cudaSuccess) e = buf.alloc(n);
        if (e == cudaSuccess) e = cudaMemsetAsync(buf.p, 0, buf.bytes(), st);
    };
    if (bf16) {
        alloc(D.a_bf, (size_t)lap * lap);
        alloc(D.b_bf, (size_t)lbp * lbp);
    } else {
        alloc(D.a_hi, (size_t)lap * lap);
        alloc(D.a_lo, (size_t)lap * lap);
        alloc(D.b_hi, (size_t)lbp * lbp);
        alloc(D.b_lo, (size_t)lbp * lbp);
    }
    if (e == cudaSuccess) {
        // beta: singles then doubles into the same matrix (a pair of strings is
        // either a single or a double excitation, never both); alpha: doubles
        auto fill = [&](int64_t l, int64_t ld, const int64_t *off, const int2 *sci, const int32_t *dcol,
                        const double *val, float *hi, float *lo, __nv_bfloat16 *bf) {
            if (l == 0 || e != cudaSuccess) return;
            k_links_to_dense<<<(unsigned)((l + 127) / 128), 128, 0, st>>>(l, ld, off, sci, dcol, val, hi, lo, bf);
            e = cudaGetLastError();
        };
        fill(lb, lbp, P->B.d_soff, P->B.d_sci.p, nullptr, P->B.d_sval.p, D.b_hi.p, D.b_lo.p, D.b_bf.p);
        fill(lb, lbp, P->B.d_doff, nullptr, P->B.d_dcol.p, P->B.d_dval.p, D.b_hi.p, D.b_lo.p, D.b_bf.p);
        fill(la, lap, P->A.d_doff, nullptr, P->A.d_dcol.p, P->A.d_dval.p, D.a_hi.p, D.a_lo.p, D.a_bf.p);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        if (bf16) {
            D.a_bf.release();
            D.b_bf.release();
        } else {
            D.a_hi.release();
            D.a_lo.release();
            D.b_hi.release();
            D.b_lo.release();
        }
        uncharge(ctx, bytes);
        return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                    std::string("dense same-spin Hamiltonians: ") + cudaGetErrorString(e));
    }
    P->charged += bytes;
    return TBSCI_OK;
}

}  // namespace

tbsci_status rest_dense_launch(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, const float *c, float *s, int nvec,
                               bool bf16, cudaStream_t st) {
    (void)ham;
    const int64_t la = P->A.l, lb = P->B.l;
    if (la == 0 || lb == 0) return TBSCI_OK;
    TB_CHECK(ctx, la <= INT32_MAX / 2 && lb <= INT32_MAX / 2, TBSCI_EINVAL, "dense products: too many strings");
    TB_TRY(ensure_dense(ctx, P, bf16, st));
    const int64_t lap = padded(la), lbp = padded(lb);
    // scratch: the split vector (two FP32 planes or one BF16 plane) and the
    // padded product, all lap x lbp
    const size_t np = (size_t)lap * lbp;
    const size_t need = np * (bf16 ? 2 + 4 : 3 * 4);
    DevBuf<unsigned char> &scr = P->dense.scratch;
    if (scr.n < need) {
        uncharge(ctx, scr.bytes());
        P->charged -= std::min(P->charged, scr.bytes());
        scr.release();
        TB_TRY(charge(ctx, need, "dense product scratch"));
        const cudaError_t e = scr.alloc(need);
        if (e != cudaSuccess) {
            uncharge(ctx, need);
            return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                        std::string("dense product scratch: ") + cudaGetErrorString(e));
        }
        P->charged += need;
    }
    std::lock_guard<std::mutex> g(ctx->cublas_mu);
    if (!ctx->cublas) {
        cublasHandle_t h = nullptr;
        TB_TRY(cublas_status(ctx, cublasCreate(&h), "cublasCreate"));
        ctx->cublas = h;
    }
    cublasHandle_t h = static_cast<cublasHandle_t>(ctx->cublas);
    TB_TRY(cublas_status(ctx, cublasSetStream(h, st), "cublasSetStream"));
    const DenseSameSpin &D = P->dense;
    float *sp = reinterpret_cast<float *>(scr.p);
    float *chi = sp + np, *clo = chi + np;
    __nv_bfloat16 *cbf = reinterpret_cast<__nv_bfloat16 *>(sp + np);
    const int m = (int)lbp, nn = (int)lap;
    const float one = 1.f, zero = 0.f;
    const size_t n = (size_t)la * lb;
    const int grid = (int)std::min<size_t>((np + 255) / 256, (size_t)ctx->num_sms * 8);
    for (int v = 0; v < nvec; ++v) {
        const float *cv = c + (size_t)v * n;
        float *sv = s + (size_t)v * n;
        {
            TraceScope tr(ctx, "k_split_vector", st);
            k_split_vector<<<grid, 256, 0, st>>>(cv, la, lb, lap, lbp, bf16 ? nullptr : chi, bf16 ? nullptr : clo,
                                                 bf16 ? cbf : nullptr);
            TB_CUDA(ctx, cudaGetLastError());
        }
        {
            TraceScope tr(ctx, "gemm_same_spin", st);
            if (bf16) {
                // sigma^T = Hb c^T + c^T Ha, one BF16 product each
                TB_TRY(cublas_status(ctx, cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, nn, m, &one, D.b_bf.p,
                                                       CUDA_R_16BF, m, cbf, CUDA_R_16BF, m, &zero, sp, CUDA_R_32F, m,
                                                       CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT),
                                     "beta same-spin product"));
                TB_TRY(cublas_status(ctx, cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, nn, nn, &one, cbf, CUDA_R_16BF,
                                                       m, D.a_bf.p, CUDA_R_16BF, nn, &one, sp, CUDA_R_32F, m,
                                                       CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT),
                                     "alpha double product"));
            } else {
                // split TF32: Hh ch + Hh cl + Hl ch per product (operands are exact TF32 values)
                const float *bA[3] = {D.b_hi.p, D.b_hi.p, D.b_lo.p};
                const float *bB[3] = {chi, clo, chi};
                for (int k = 0; k < 3; ++k)
                    TB_TRY(cublas_status(ctx, cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, nn, m, &one, bA[k],
                                                           CUDA_R_32F, m, bB[k], CUDA_R_32F, m, k == 0 ? &zero : &one,
                                                           sp, CUDA_R_32F, m, CUBLAS_COMPUTE_32F_FAST_TF32,
                                                           CUBLAS_GEMM_DEFAULT),
                                         "beta same-spin product"));
                const float *aA[3] = {chi, clo, chi};
                const float *aB[3] = {D.a_hi.p, D.a_hi.p, D.a_lo.p};
                for (int k = 0; k < 3; ++k)
                    TB_TRY(cublas_status(ctx, cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, nn, nn, &one, aA[k],
                                                           CUDA_R_32F, m, aB[k], CUDA_R_32F, nn, &one, sp, CUDA_R_32F,
                                                           m, CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT),
                                         "alpha double product"));
            }
        }
        TraceScope tr(ctx, "k_unpad", st);
        k_unpad<<<(int)std::min<size_t>((n + 255) / 256, (size_t)ctx->num_sms * 8), 256, 0, st>>>(sp, la, lb, lbp,
                                                                                                   sv);
        TB_CUDA(ctx, cudaGetLastError());
    }
    return TBSCI_OK;
}

void dense_context_release(tbsci_ctx *ctx) {
    if (ctx && ctx->cublas) {
        cublasDestroy(static_cast<cublasHandle_t>(ctx->cublas));
        ctx->cublas = nullptr;
    }
}

}  // namespace tbsci
