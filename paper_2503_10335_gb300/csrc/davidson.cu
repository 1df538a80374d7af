// Standard Davidson (Sec. III.A) for the lowest roots of H on a TPB space, with
// restart to the Ritz vectors when the basis is full (Sec. III.C: at most
// 2*N_max + 3 vectors are kept: basis V and images W of N_max each, plus the
// Ritz vectors, their images and the corrections, one per root).
//
// All vector work runs in FP64 on the device: block dot products with a fixed
// grid and a fixed reduction order (run-to-run deterministic), linear
// combinations, fused residual + diagonal preconditioner. The Rayleigh matrix
// (at most a few dozen rows) is diagonalised on the host by cyclic Jacobi.
// Mixed mode evaluates sigma in FP32 until the residuals reach a loose target,
// then restarts from the Ritz vectors with FP64 sigma and converges to the FP64
// tolerances; Gram-Schmidt, the subspace problem and residuals stay FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include <type_traits>

#include "internal.cuh"

namespace tbsci {

namespace {

constexpr int kDotThreads = 256;
constexpr int kMA = 8;  // rows of A per dot block
constexpr int kMB = 4;  // rows of B per dot block

// partial[b][i][j] over this block's slice of K: sum A[i][K] * B[j][K], in FP64
// whatever the storage type T of the vectors (FP32 x FP32 products are exact in
// FP64). Rows past ma / mb are skipped with block-uniform branches, so no FP64
// work goes to padding (FP64 throughput bounds these dots on this GPU).
template <typename T, int MB = kMB>
__global__ void __launch_bounds__(kDotThreads) k_dots(const T *__restrict__ A, int ma, const T *__restrict__ B, int mb,
                                                      int64_t N, double *partial, int ldp,
                                                      const int *__restrict__ skip = nullptr) {
    if (skip && *skip) return;  // a pass the device decided is not needed
    __shared__ double sh[kDotThreads / 32][kMA * MB];
    const int i0 = blockIdx.y * kMA, j0 = blockIdx.z * MB;
    const int na = min(kMA, ma - i0), nb = min(MB, mb - j0);
    double acc[kMA][MB];
#pragma unroll
    for (int i = 0; i < kMA; ++i)
#pragma unroll
        for (int j = 0; j < MB; ++j) acc[i][j] = 0.0;
    // two elements per thread per step: up to 2 * (8 + MB) independent loads in flight
    const int64_t step = (int64_t)gridDim.x * kDotThreads * 2;
    for (int64_t K0 = blockIdx.x * (int64_t)kDotThreads * 2 + threadIdx.x; K0 < N; K0 += step) {
        const int64_t K1 = K0 + kDotThreads;
        const bool h1 = K1 < N;
        double b0[MB], b1[MB];
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            b0[j] = j < nb ? (double)__ldg(B + (size_t)(j0 + j) * N + K0) : 0.0;
            b1[j] = (j < nb && h1) ? (double)__ldg(B + (size_t)(j0 + j) * N + K1) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < kMA; ++i) {
            if (i < na) {
                const double a0 = (double)__ldg(A + (size_t)(i0 + i) * N + K0);
                const double a1 = h1 ? (double)__ldg(A + (size_t)(i0 + i) * N + K1) : 0.0;
#pragma unroll
                for (int j = 0; j < MB; ++j)
                    if (j < nb) acc[i][j] = fma(a1, b1[j], fma(a0, b0[j], acc[i][j]));
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kMA; ++i)
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            double v = acc[i][j];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sh[w][i * MB + j] = v;
        }
    __syncthreads();
    if (threadIdx.x < kMA * MB) {
        int i = threadIdx.x / MB, j = threadIdx.x % MB;
        double v = 0.0;
        for (int x = 0; x < kDotThreads / 32; ++x) v += sh[x][threadIdx.x];
        if (i < na && j < nb) partial[(size_t)blockIdx.x * ldp + (size_t)(i0 + i) * mb + (j0 + j)] = v;
    }
}

// out[t] = sum_b partial[b][t] in block order
__global__ void k_reduce_partials(const double *partial, int nblocks, int ldp, int nt, double *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[(size_t)b * ldp + t];
    out[t] = v;
}

constexpr int kMaxBasis = 128;
constexpr int kMaxOut = 8;

// out[k][K] = beta * out[k][K] + yscale * sum_i Y[i][k] * A[i][K], k < KOUT,
// accumulated in FP64 and stored as TO. Each thread handles U elements spaced
// blockDim apart per step and reads two rows per unrolled pass (2U loads in
// flight); the accumulator tile KOUT x U stays small enough for 4 CTAs per SM.
// KOUT is the exact output count: a guarded output slot would still occupy the
// FP64 pipe with predicated-off multiply-adds.
template <typename TA, typename TO, int KOUT>
__global__ void __launch_bounds__(256) k_lincomb(const TA *__restrict__ A, int m, TO *out, int64_t N, double beta,
                                                 const double *__restrict__ Y, double yscale,
                                                 const int *__restrict__ skip) {
    if (skip && *skip) return;
    constexpr int U = KOUT >= 3 ? 2 : 4;
    constexpr int kout = KOUT;
    __shared__ double sY[kMaxBasis * KOUT];
    for (int x = threadIdx.x; x < m * kout; x += blockDim.x) sY[x] = yscale * Y[x];
    __syncthreads();
    const int64_t step = (int64_t)gridDim.x * blockDim.x * U;
    for (int64_t K0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x; K0 < N; K0 += step) {
        double acc[KOUT][U];
#pragma unroll
        for (int k = 0; k < KOUT; ++k)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t K = K0 + (int64_t)u * blockDim.x;
                acc[k][u] = (beta != 0.0 && K < N) ? beta * (double)out[(size_t)k * N + K] : 0.0;
            }
#pragma unroll 2
        for (int i = 0; i < m; ++i) {
            double a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t K = K0 + (int64_t)u * blockDim.x;
                a[u] = K < N ? (double)__ldg(A + (size_t)i * N + K) : 0.0;
            }
#pragma unroll
            for (int k = 0; k < KOUT; ++k) {
                const double y = sY[i * kout + k];
#pragma unroll
                for (int u = 0; u < U; ++u) acc[k][u] = fma(y, a[u], acc[k][u]);
            }
        }
#pragma unroll
        for (int k = 0; k < KOUT; ++k)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t K = K0 + (int64_t)u * blockDim.x;
                if (K < N) out[(size_t)k * N + K] = (TO)acc[k][u];
            }
    }
}

template <typename TA, typename TO>
void launch_lincomb(int grid, cudaStream_t st, const TA *A, int m, TO *out, int kout, int64_t N, double beta,
                    const double *Y, double yscale, const int *skip = nullptr) {
    switch (kout) {  // kout is 1..kMaxOut (callers split larger sets)
        case 1: k_lincomb<TA, TO, 1><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        case 2: k_lincomb<TA, TO, 2><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        case 3: k_lincomb<TA, TO, 3><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        case 4: k_lincomb<TA, TO, 4><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        case 5: k_lincomb<TA, TO, 5><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        case 6: k_lincomb<TA, TO, 6><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        case 7: k_lincomb<TA, TO, 7><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
        default: k_lincomb<TA, TO, 8><<<grid, 256, 0, st>>>(A, m, out, N, beta, Y, yscale, skip); break;
    }
}

// Second Gram-Schmidt pass needed? "Twice is enough" (Daniel-Gragg-Kaufman-
// Stewart, eta = 1/sqrt(2)): skip it when every correction kept at least half of
// its squared norm in the first pass. norms[2 j] = ||t_j||^2 before, after[j] after.
__global__ void k_gs_decide(const double *__restrict__ norms, const double *__restrict__ after, int nb, int *skip) {
    if (threadIdx.x != 0) return;
    int ok = 1;
    for (int j = 0; j < nb; ++j) ok &= (after[j * (nb + 1)] >= 0.5 * norms[2 * j]) ? 1 : 0;
    *skip = ok;
}

// y = x / sqrt(*nrm2) (zero when the norm is zero); y may be x
template <typename T>
__global__ void k_normalize(const T *x, const double *__restrict__ nrm2, T *y, int64_t N) {
    const double n2 = *nrm2;
    const double s = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    for (int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; K < N; K += (int64_t)gridDim.x * blockDim.x)
        y[K] = (T)(s * (double)x[K]);
}

// V[r][idx[j]] = M[r][j] for r < nroots, j < ncol (guess vectors on a few determinants)
template <typename T>
__global__ void k_set_guess(T *V, int64_t N, const int64_t *idx, const double *M, int nroots, int ncol) {
    const int t = threadIdx.x;
    if (t >= nroots * ncol) return;
    const int r = t / ncol, j = t - r * ncol;
    V[(size_t)r * N + idx[j]] = (T)M[t];
}

// 1/x for the diagonal preconditioner: an FP32 reciprocal as the seed, then one
// Newton-Raphson step y' = y (2 - x y) in FP64, which doubles the seed's ~23
// correct bits. |x| is clamped to [1e-8, ~1e3] by the caller, inside FP32's range.
// The preconditioned residual only sets a search direction, so ~1e-13 relative
// accuracy is ample, and it costs a fraction of a full FP64 division per element.
__device__ __forceinline__ double precond_recip(double x) {
    const double y = (double)(1.0f / (float)x);
    return y * fma(-x, y, 2.0);
}

// r = wy - theta x; t = r / clamp(theta - diag); partial norms of r (nroots <= NR)
template <int NR>
__global__ void __launch_bounds__(kDotThreads) k_residual(const double *__restrict__ X, const double *__restrict__ WY,
                                                          const double *__restrict__ diag, const double *__restrict__ theta,
                                                          int nroots, int64_t N, double *T, double *partial) {
    __shared__ double sh[kDotThreads / 32][NR];
    double acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = 0.0;
    // four elements per thread per step: 4 (2 NR + 1) loads in flight
    const int64_t step = (int64_t)gridDim.x * kDotThreads * 4;
    for (int64_t K0 = blockIdx.x * (int64_t)kDotThreads * 4 + threadIdx.x; K0 < N; K0 += step) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t K = K0 + (int64_t)u * kDotThreads;
            if (K >= N) break;
            const double d = diag[K];
#pragma unroll
            for (int k = 0; k < NR; ++k) {  // NR == nroots: no guarded FP64 slots
                const double r = WY[(size_t)k * N + K] - theta[k] * X[(size_t)k * N + K];
                acc[k] = fma(r, r, acc[k]);
                double den = theta[k] - d;
                if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
                T[(size_t)k * N + K] = r * precond_recip(den);
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < nroots) {
        double v = 0.0;
        for (int x = 0; x < kDotThreads / 32; ++x) v += sh[x][threadIdx.x];
        partial[(size_t)blockIdx.x * kMaxOut + threadIdx.x] = v;
    }
}


__global__ void k_to_f32(const double *__restrict__ x, float *y, int64_t n) {
    for (int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; K < n; K += (int64_t)gridDim.x * blockDim.x)
        y[K] = (float)x[K];
}

__global__ void k_to_f64(const float *__restrict__ x, double *y, int64_t n) {
    for (int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; K < n; K += (int64_t)gridDim.x * blockDim.x)
        y[K] = (double)x[K];
}

// per-block minimum of (value, index), skipping listed indices
__global__ void k_argmin(const double *__restrict__ d, int64_t N, const int64_t *skip, int nskip, double *bv, int64_t *bi) {
    __shared__ double sv[256];
    __shared__ int64_t si[256];
    double best = INFINITY;
    int64_t bidx = INT64_MAX;
    for (int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; K < N; K += (int64_t)gridDim.x * blockDim.x) {
        bool skipped = false;
        for (int s = 0; s < nskip; ++s) skipped |= (skip[s] == K);
        if (skipped) continue;
        double v = d[K];
        if (v < best || (v == best && K < bidx)) {
            best = v;
            bidx = K;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double v = sv[threadIdx.x + o];
            int64_t i = si[threadIdx.x + o];
            if (v < sv[threadIdx.x] || (v == sv[threadIdx.x] && i < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bv[blockIdx.x] = sv[0];
        bi[blockIdx.x] = si[0];
    }
}

// Cyclic Jacobi for a symmetric m x m matrix (row-major). On return `a` holds
// nothing useful, `w` the eigenvalues ascending and `v` the eigenvectors as
// columns (v[i*m + k] = component i of vector k).
void jacobi_eigh(std::vector<double> a, int m, std::vector<double> &w, std::vector<double> &v) {
    v.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) v[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double x = a[(size_t)i * m + j] * a[(size_t)i * m + j];
                tot += x;
                if (i != j) off += x;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = a[(size_t)p * m + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {  // rotate columns p, q
                    double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
                    a[(size_t)k * m + p] = c * akp - s * akq;
                    a[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {  // rotate rows p, q
                    double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
                    a[(size_t)p * m + k] = c * apk - s * aqk;
                    a[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    double vkp = v[(size_t)k * m + p], vkq = v[(size_t)k * m + q];
                    v[(size_t)k * m + p] = c * vkp - s * vkq;
                    v[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(m);
    for (int i = 0; i < m; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return a[(size_t)x * m + x] < a[(size_t)y * m + y]; });
    w.resize(m);
    std::vector<double> vs((size_t)m * m);
    for (int k = 0; k < m; ++k) {
        w[k] = a[(size_t)idx[k] * m + idx[k]];
        for (int i = 0; i < m; ++i) vs[(size_t)i * m + k] = v[(size_t)i * m + idx[k]];
    }
    v.swap(vs);
}

// Rayleigh-Ritz on a basis that is orthonormal only to rounding: G y = theta S y
// with S = V^T V positive definite. Cholesky S = L L^T, eigenpairs z of
// L^-1 G L^-T by Jacobi, y = L^-T z (S-orthonormal). Same output convention as
// jacobi_eigh. False when S is not positive definite.
bool gen_eigh(const std::vector<double> &G, const std::vector<double> &S, int m, std::vector<double> &w,
              std::vector<double> &y) {
    std::vector<double> L((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        double d = S[(size_t)j * m + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
        if (!(d > 0.0)) return false;
        L[(size_t)j * m + j] = std::sqrt(d);
        for (int i = j + 1; i < m; ++i) {
            double x = S[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) x -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
            L[(size_t)i * m + j] = x / L[(size_t)j * m + j];
        }
    }
    std::vector<double> A(G), B((size_t)m * m), Gh((size_t)m * m), z;
    for (int c = 0; c < m; ++c)  // A = L^-1 G
        for (int i = 0; i < m; ++i) {
            double x = A[(size_t)i * m + c];
            for (int k = 0; k < i; ++k) x -= L[(size_t)i * m + k] * A[(size_t)k * m + c];
            A[(size_t)i * m + c] = x / L[(size_t)i * m + i];
        }
    for (int c = 0; c < m; ++c)  // B = L^-1 A^T = (L^-1 G L^-T)^T
        for (int i = 0; i < m; ++i) {
            double x = A[(size_t)c * m + i];
            for (int k = 0; k < i; ++k) x -= L[(size_t)i * m + k] * B[(size_t)k * m + c];
            B[(size_t)i * m + c] = x / L[(size_t)i * m + i];
        }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Gh[(size_t)i * m + j] = 0.5 * (B[(size_t)i * m + j] + B[(size_t)j * m + i]);
    jacobi_eigh(Gh, m, w, z);
    y.assign((size_t)m * m, 0.0);
    for (int c = 0; c < m; ++c)  // y = L^-T z
        for (int i = m - 1; i >= 0; --i) {
            double x = z[(size_t)i * m + c];
            for (int k = i + 1; k < m; ++k) x -= L[(size_t)k * m + i] * y[(size_t)k * m + c];
            y[(size_t)i * m + c] = x / L[(size_t)i * m + i];
        }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Resumable Davidson engine. Each phase enqueues device work on the engine's
// stream and ends at one event; the host logic of the next phase runs once that
// event has completed. Phases per iteration:
//   NeedSigma  -> images of the newest basis vectors are wanted (driver launches sigma)
//   WaitG      -> new Rayleigh-matrix columns are on their way to the host
//   WaitR      -> Ritz vectors, residual norms and preconditioned corrections computed
//   WaitGS     -> corrections orthonormalised on the device, their norms on the way
// A driver either blocks on each phase (tbsci_davidson) or polls many engines
// and batches their sigma work (the serving loop).

struct DavEngine {
    tbsci_ctx *ctx = nullptr;
    tbsci_ham *ham = nullptr;
    Plan *plan = nullptr;
    const tbsci_pruned *pr = nullptr;  // set: the solve runs on this pruned subspace
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaEvent_t evt = nullptr;
    int nroots = 1, m_max = 0, keep = 0, max_iter = 0;
    double tol_e = 0, tol_r = 0, tol_rm = 0;
    int64_t N = 0;
    int nblocks = 0;  // blocks of the reduction kernels (fixed per problem size: deterministic sums)
    int lgrid = 0;    // blocks of the linear combinations (no reduction: sized for occupancy)
    int rgrid = 0;    // blocks of the residual kernel (fixed per problem size, like nblocks)
    DevBuf<double> V, W, X, WY, T, diag, R, partial, red, dY, dY2, dtheta, scal, coef;
    DevBuf<int> gs_skip;  // 1: the second block Gram-Schmidt pass is not needed
    DevBuf<float> v32, w32;
    // FP32-stored basis and images (basis_f32, low-precision phase only); the
    // Rayleigh problem is then solved against the overlap Sm = V^T V
    DevBuf<float> V32, W32, R32;
    bool b32 = false;
    int m_ref = 0, keep_ref = 0;  // basis size and restart of the FP64 refinement
    std::vector<double> Sm;
    double *hG = nullptr, *hY = nullptr, *hY2 = nullptr, *hR = nullptr, *hN = nullptr;  // pinned
    enum class St { NeedSigma, WaitG, WaitR, WaitGS, Done } state = St::NeedSigma;
    int m = 0, sig_lo = 0, sig_hi = 0, g_lo = 0;
    bool f32 = false, sig_prepared = false;
    bool mixed_mode = false;  // the solve has a low-precision phase
    tbsci_dtype lowp = TBSCI_F32;  // sigma type of the low-precision phase
    std::vector<double> G, theta, theta_prev, rnorm, e32, Yv;
    // the previous iteration's Ritz vectors as coefficients [i][k] over the first
    // p_rows basis vectors (later vectors have zero coefficients); kept beside the
    // lowest Ritz vectors at a restart of an FP64 basis
    std::vector<double> p_prev;
    int p_rows = 0;
    std::vector<int> todo;
    int it = 0, it32 = 0, stall32 = 0, nsig = 0, nsig32 = 0;
    double best32 = INFINITY;
    bool converged = false, failed = false;
    tbsci_status status = TBSCI_OK;
    std::chrono::steady_clock::time_point t_start;

    ~DavEngine() {
        if (hG) cudaFreeHost(hG);
        if (hY) cudaFreeHost(hY);
        if (hY2) cudaFreeHost(hY2);
        if (hR) cudaFreeHost(hR);
        if (hN) cudaFreeHost(hN);
        if (evt) cudaEventDestroy(evt);
        if (own_stream && st) cudaStreamDestroy(st);
    }

    // basis slot k of V / W in the current storage type
    size_t es() const { return b32 ? sizeof(float) : sizeof(double); }
    void *vs(int k) { return b32 ? (void *)(V32.p + (size_t)k * N) : (void *)(V.p + (size_t)k * N); }
    void *ws(int k) { return b32 ? (void *)(W32.p + (size_t)k * N) : (void *)(W.p + (size_t)k * N); }

    // out[i][j] = A_i . B_j over basis-typed rows, FP64 accumulation; skip: a
    // device flag that, when set, turns the product into no work
    tbsci_status dots(const void *A, int ma, const void *B, int mb, double *out, const int *skip = nullptr) {
        const int ldp = ma * mb;
        // columns of B per block: mb itself up to kMB (no guarded column costs
        // FP64 work), else kMB with a partial last block
        const int mbb = std::min(mb, kMB);
        const dim3 grid(nblocks, (ma + kMA - 1) / kMA, (mb + mbb - 1) / mbb);
        auto go = [&](auto mb_tag) {
            constexpr int MB = decltype(mb_tag)::value;
            if (b32)
                k_dots<float, MB><<<grid, kDotThreads, 0, st>>>((const float *)A, ma, (const float *)B, mb, N,
                                                                partial.p, ldp, skip);
            else
                k_dots<double, MB><<<grid, kDotThreads, 0, st>>>((const double *)A, ma, (const double *)B, mb, N,
                                                                 partial.p, ldp, skip);
        };
        switch (mbb) {
            case 1: go(std::integral_constant<int, 1>{}); break;
            case 2: go(std::integral_constant<int, 2>{}); break;
            case 3: go(std::integral_constant<int, 3>{}); break;
            default: go(std::integral_constant<int, 4>{}); break;
        }
        TB_CUDA(ctx, cudaGetLastError());
        k_reduce_partials<<<(ldp + 127) / 128, 128, 0, st>>>(partial.p, nblocks, ldp, ldp, out);
        TB_CUDA(ctx, cudaGetLastError());
        return TBSCI_OK;
    }
    // basis-typed out = beta * out + yscale * sum_i Y[i][k] A_i
    tbsci_status lincomb(const void *A, int mm, void *out, int kout, double beta, const double *Ydev, double yscale,
                         const int *skip = nullptr) {
        if (b32) launch_lincomb(lgrid, st, (const float *)A, mm, (float *)out, kout, N, beta, Ydev, yscale, skip);
        else launch_lincomb(lgrid, st, (const double *)A, mm, (double *)out, kout, N, beta, Ydev, yscale, skip);
        TB_CUDA(ctx, cudaGetLastError());
        return TBSCI_OK;
    }
    // FP64 out = sum_i Y[i][k] A_i over basis-typed rows (Ritz vectors and images)
    tbsci_status ritz(const void *A, int mm, double *out, int kout, const double *Ydev) {
        if (b32) launch_lincomb(lgrid, st, (const float *)A, mm, out, kout, N, 0.0, Ydev, 1.0);
        else launch_lincomb(lgrid, st, (const double *)A, mm, out, kout, N, 0.0, Ydev, 1.0);
        TB_CUDA(ctx, cudaGetLastError());
        return TBSCI_OK;
    }
    tbsci_status normalize(void *x, const double *nrm2) {
        if (b32) k_normalize<float><<<nblocks, 256, 0, st>>>((const float *)x, nrm2, (float *)x, N);
        else k_normalize<double><<<nblocks, 256, 0, st>>>((const double *)x, nrm2, (double *)x, N);
        TB_CUDA(ctx, cudaGetLastError());
        return TBSCI_OK;
    }
    tbsci_status finish_phase(St next) {
        TB_CUDA(ctx, cudaEventRecord(evt, st));
        state = next;
        return TBSCI_OK;
    }

    tbsci_status init(tbsci_ctx *c, tbsci_ham *h, Plan *p, int nr, const tbsci_davidson_opts &opt) {
        ctx = c;
        ham = h;
        plan = p;
        nroots = nr;
        t_start = std::chrono::steady_clock::now();
        m_max = opt.max_subspace > 0 ? opt.max_subspace : std::max(8 * nroots, nroots + 2);
        keep = opt.restart_keep > 0 ? opt.restart_keep : std::max(nroots, m_max / 2);
        max_iter = opt.max_iter > 0 ? opt.max_iter : 1000;
        tol_e = opt.tol_energy > 0 ? opt.tol_energy : 1e-9;
        tol_r = opt.tol_residual > 0 ? opt.tol_residual : 1e-5;
        tol_rm = opt.tol_mixed_residual > 0 ? opt.tol_mixed_residual : 5e-5;
        TB_CHECK(ctx, nroots >= 1 && nroots <= kMaxOut, TBSCI_EINVAL, "nroots must be in 1..8");
        TB_CHECK(ctx, m_max >= nroots + 1 && m_max <= kMaxBasis, TBSCI_EINVAL,
                 "max_subspace must be in nroots+1..128");
        TB_CHECK(ctx, keep >= nroots && keep < m_max, TBSCI_EINVAL, "restart_keep must be in nroots..max_subspace-1");
        N = pr ? pr->nd : plan->A.l * plan->B.l;
        TB_CHECK(ctx, N >= nroots, TBSCI_EINVAL, "space has fewer determinants than roots");
        if (opt.stream) {
            st = (cudaStream_t)opt.stream;
        } else {
            TB_CUDA(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            own_stream = true;
        }
        TB_CUDA(ctx, cudaEventCreateWithFlags(&evt, cudaEventDisableTiming));
        // small problems use fewer reduction blocks (fixed per problem size: deterministic)
        nblocks = (int)std::min<int64_t>(2 * ctx->num_sms, std::max<int64_t>(1, (N + 4095) / 4096));
        lgrid = (int)std::min<int64_t>(8 * ctx->num_sms, std::max<int64_t>(1, (N + 1023) / 1024));
        rgrid = (int)std::min<int64_t>(6 * ctx->num_sms, std::max<int64_t>(1, (N + 1023) / 1024));
        f32 = opt.mixed != 0;
        mixed_mode = f32;
        TB_CHECK(ctx, opt.mixed >= 0 && opt.mixed <= 3, TBSCI_EINVAL, "mixed must be 0..3");
        lowp = opt.mixed == 2 ? TBSCI_F32_TC_TF32 : opt.mixed == 3 ? TBSCI_F32_TC_BF16 : TBSCI_F32;
        b32 = opt.basis_f32 != 0;
        TB_CHECK(ctx, !b32 || f32, TBSCI_EINVAL, "basis_f32 needs a low-precision phase (mixed != 0)");
        m_ref = b32 ? (opt.max_subspace_refine > 0 ? opt.max_subspace_refine : std::max(nroots + 1, m_max / 2)) : m_max;
        TB_CHECK(ctx, m_ref >= nroots + 1 && m_ref <= m_max, TBSCI_EINVAL,
                 "max_subspace_refine must be in nroots+1..max_subspace");
        keep_ref = b32 ? std::max(nroots, m_ref / 2) : keep;
        TB_CUDA(ctx, partial.alloc(
                         std::max((size_t)nblocks * m_max * m_max, (size_t)std::max(nblocks, rgrid) * kMaxOut)));
        TB_CUDA(ctx, red.alloc((size_t)2 * m_max * m_max));
        TB_CUDA(ctx, dY.alloc((size_t)m_max * m_max));
        TB_CUDA(ctx, dY2.alloc((size_t)m_max * m_max));
        TB_CUDA(ctx, dtheta.alloc(kMaxOut));
        TB_CUDA(ctx, scal.alloc(2 * kMaxOut));
        TB_CUDA(ctx, coef.alloc((size_t)m_max * kMaxOut));
        TB_CUDA(ctx, gs_skip.alloc(1));
        TB_CUDA(ctx, cudaMallocHost(&hG, (size_t)2 * m_max * m_max * sizeof(double)));
        TB_CUDA(ctx, cudaMallocHost(&hY, (size_t)m_max * m_max * sizeof(double)));
        TB_CUDA(ctx, cudaMallocHost(&hY2, (size_t)m_max * m_max * sizeof(double)));
        TB_CUDA(ctx, cudaMallocHost(&hR, kMaxOut * sizeof(double)));
        TB_CUDA(ctx, cudaMallocHost(&hN, 2 * kMaxOut * sizeof(double)));
        if (b32) {
            TB_CUDA(ctx, V32.alloc((size_t)m_max * N));
            TB_CUDA(ctx, W32.alloc((size_t)m_max * N));
        } else {
            TB_CUDA(ctx, V.alloc((size_t)m_max * N));
            TB_CUDA(ctx, W.alloc((size_t)m_max * N));
        }
        TB_CUDA(ctx, X.alloc((size_t)nroots * N));
        TB_CUDA(ctx, WY.alloc((size_t)nroots * N));
        TB_CUDA(ctx, T.alloc((size_t)nroots * N));
        TB_CUDA(ctx, diag.alloc(N));
        if (f32 && !b32) {
            TB_CUDA(ctx, v32.alloc((size_t)nroots * N));
            TB_CUDA(ctx, w32.alloc((size_t)nroots * N));
        }
        G.assign((size_t)m_max * m_max, 0.0);
        Sm.assign((size_t)m_max * m_max, 0.0);
        theta.assign(nroots, 0.0);
        theta_prev.assign(nroots, INFINITY);
        rnorm.assign(nroots, INFINITY);
        e32.assign(nroots, 0.0);
        if (pr) TB_TRY(pruned_diagonal_launch(ctx, ham, plan, pr, diag.p, st));
        else TB_TRY(diagonal_launch(ctx, ham, plan, diag.p, st));
        // guess: unit vectors at the nroots lowest (H_KK, K), each mixed with the next
        // four lowest determinants so that every symmetry sector is present
        const int extra = (int)std::min<int64_t>(4, N - nroots);
        const int ncol = nroots + extra;
        std::vector<int64_t> chosen;
        DevBuf<double> bv, dM;
        DevBuf<int64_t> bi, dskip;
        TB_CUDA(ctx, bv.alloc(nblocks));
        TB_CUDA(ctx, bi.alloc(nblocks));
        TB_CUDA(ctx, dskip.alloc(kMaxOut + 4));
        TB_CUDA(ctx, dM.alloc((size_t)kMaxOut * (kMaxOut + 4)));
        std::vector<double> hv(nblocks);
        std::vector<int64_t> hi(nblocks);
        for (int r = 0; r < ncol; ++r) {
            if (!chosen.empty())
                TB_CUDA(ctx, cudaMemcpyAsync(dskip.p, chosen.data(), chosen.size() * sizeof(int64_t),
                                             cudaMemcpyHostToDevice, st));
            k_argmin<<<nblocks, 256, 0, st>>>(diag.p, N, dskip.p, (int)chosen.size(), bv.p, bi.p);
            TB_CUDA(ctx, cudaGetLastError());
            TB_CUDA(ctx, cudaMemcpyAsync(hv.data(), bv.p, nblocks * sizeof(double), cudaMemcpyDeviceToHost, st));
            TB_CUDA(ctx, cudaMemcpyAsync(hi.data(), bi.p, nblocks * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            TB_CUDA(ctx, cudaStreamSynchronize(st));
            double best = INFINITY;
            int64_t bidx = INT64_MAX;
            for (int b = 0; b < nblocks; ++b)
                if (hv[b] < best || (hv[b] == best && hi[b] < bidx)) {
                    best = hv[b];
                    bidx = hi[b];
                }
            TB_CHECK(ctx, bidx >= 0 && bidx < N, TBSCI_EINVAL, "Davidson guess: the diagonal has no finite minimum");
            chosen.push_back(bidx);
        }
        std::vector<double> M((size_t)nroots * ncol, 0.0);
        for (int k = 0; k < nroots; ++k) {
            M[(size_t)k * ncol + k] = 1.0;
            for (int j = 0; j < extra; ++j) M[(size_t)k * ncol + nroots + j] += 0.1 * (1.0 + ((j + k) % 4)) / 4.0;
        }
        for (int k = 0; k < nroots; ++k) {  // Gram-Schmidt in order, on the coefficients
            for (int i = 0; i < k; ++i) {
                double d = 0.0;
                for (int j = 0; j < ncol; ++j) d += M[(size_t)i * ncol + j] * M[(size_t)k * ncol + j];
                for (int j = 0; j < ncol; ++j) M[(size_t)k * ncol + j] -= d * M[(size_t)i * ncol + j];
            }
            double nn = 0.0;
            for (int j = 0; j < ncol; ++j) nn += M[(size_t)k * ncol + j] * M[(size_t)k * ncol + j];
            nn = std::sqrt(nn);
            for (int j = 0; j < ncol; ++j) M[(size_t)k * ncol + j] /= nn;
        }
        TB_CUDA(ctx, cudaMemsetAsync(vs(0), 0, (size_t)nroots * N * es(), st));
        TB_CUDA(ctx, cudaMemcpyAsync(dskip.p, chosen.data(), chosen.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                     st));
        TB_CUDA(ctx, cudaMemcpyAsync(dM.p, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        if (b32) k_set_guess<float><<<1, kMaxOut * (kMaxOut + 4), 0, st>>>(V32.p, N, dskip.p, dM.p, nroots, ncol);
        else k_set_guess<double><<<1, kMaxOut * (kMaxOut + 4), 0, st>>>(V.p, N, dskip.p, dM.p, nroots, ncol);
        TB_CUDA(ctx, cudaGetLastError());
        TB_CUDA(ctx, cudaStreamSynchronize(st));  // bv/bi/dskip are freed on return
        m = 0;
        sig_lo = 0;
        sig_hi = nroots;
        g_lo = 0;
        state = St::NeedSigma;
        return TBSCI_OK;
    }

    // The sigma the engine needs next (device pointers, on the engine stream).
    bool wants_sigma(const void **c, void **s, int *k, tbsci_dtype *dt) {
        if (state != St::NeedSigma) return false;
        const int kk = sig_hi - sig_lo;
        if (f32 && !b32) {
            if (!sig_prepared) {
                k_to_f32<<<nblocks, 256, 0, st>>>(V.p + (size_t)sig_lo * N, v32.p, (int64_t)kk * N);
                sig_prepared = true;
            }
            *c = v32.p;
            *s = w32.p;
        } else {  // FP64 basis with FP64 sigma, or FP32 basis with low-precision sigma in place
            *c = vs(sig_lo);
            *s = ws(sig_lo);
        }
        *dt = f32 ? lowp : TBSCI_F64;
        *k = kk;
        return true;
    }

    // Called once the sigma of wants_sigma() is enqueued on (or ordered before) the engine stream.
    tbsci_status sigma_done() {
        const int kk = sig_hi - sig_lo;
        if (f32 && !b32) {
            k_to_f64<<<nblocks, 256, 0, st>>>(w32.p, W.p + (size_t)sig_lo * N, (int64_t)kk * N);
            TB_CUDA(ctx, cudaGetLastError());
        }
        if (f32) nsig32 += kk;
        nsig += kk;
        sig_prepared = false;
        m = sig_hi;
        // Rayleigh-matrix columns g_lo..m against rows 0..m (and overlap columns for an FP32 basis)
        return fetch_G();
    }

    tbsci_status fetch_G() {
        TB_TRY(dots(vs(0), m, ws(g_lo), m - g_lo, red.p));
        const int ld = m * (m - g_lo);
        if (b32) TB_TRY(dots(vs(0), m, vs(g_lo), m - g_lo, red.p + ld));
        TB_CUDA(ctx, cudaMemcpyAsync(hG, red.p, (size_t)(b32 ? 2 : 1) * ld * sizeof(double), cudaMemcpyDeviceToHost, st));
        return finish_phase(St::WaitG);
    }

    // Iteration head: subspace eigenproblem, Ritz vectors, residuals.
    tbsci_status head() {
        ++it;
        if (f32) ++it32;
        std::vector<double> Gm((size_t)m * m), w;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) Gm[(size_t)i * m + j] = G[(size_t)i * m_max + j];
        if (b32) {
            std::vector<double> Sg((size_t)m * m);
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) Sg[(size_t)i * m + j] = Sm[(size_t)i * m_max + j];
            TB_CHECK(ctx, gen_eigh(Gm, Sg, m, w, Yv), TBSCI_ENOCONV,
                     "Davidson: the FP32 basis lost linear independence (overlap not positive definite)");
        } else {
            jacobi_eigh(Gm, m, w, Yv);
        }
        for (int k = 0; k < nroots; ++k) theta[k] = w[k];
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < nroots; ++k) hY[(size_t)i * nroots + k] = Yv[(size_t)i * m + k];
        TB_CUDA(ctx, cudaMemcpyAsync(dY.p, hY, (size_t)m * nroots * sizeof(double), cudaMemcpyHostToDevice, st));
        for (int k = 0; k < nroots; ++k) hR[k] = theta[k];
        TB_CUDA(ctx, cudaMemcpyAsync(dtheta.p, hR, nroots * sizeof(double), cudaMemcpyHostToDevice, st));
        TB_TRY(ritz(vs(0), m, X.p, nroots, dY.p));
        TB_TRY(ritz(ws(0), m, WY.p, nroots, dY.p));
        decltype(&k_residual<1>) resid = nullptr;
        switch (nroots) {
            case 1: resid = k_residual<1>; break;
            case 2: resid = k_residual<2>; break;
            case 3: resid = k_residual<3>; break;
            case 4: resid = k_residual<4>; break;
            case 5: resid = k_residual<5>; break;
            case 6: resid = k_residual<6>; break;
            case 7: resid = k_residual<7>; break;
            default: resid = k_residual<8>; break;
        }
        resid<<<rgrid, kDotThreads, 0, st>>>(X.p, WY.p, diag.p, dtheta.p, nroots, N, T.p, partial.p);
        TB_CUDA(ctx, cudaGetLastError());
        k_reduce_partials<<<1, 32, 0, st>>>(partial.p, rgrid, kMaxOut, nroots, red.p);
        TB_CUDA(ctx, cudaGetLastError());
        // hR is reused: the copy below is ordered after the upload above on the same stream
        TB_CUDA(ctx, cudaMemcpyAsync(hR, red.p, nroots * sizeof(double), cudaMemcpyDeviceToHost, st));
        return finish_phase(St::WaitR);
    }

    // End of the low-precision phase with an FP32-stored basis: release it, then
    // continue on an FP64 basis of m_ref vectors that starts from the Ritz vectors
    // (in X, FP64), orthonormalised in FP64 because the FP32 basis was orthonormal
    // only to FP32 rounding. Peak memory is the larger phase, not the sum.
    tbsci_status leave_basis32() {
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        V32.release();
        W32.release();
        R32.release();
        b32 = false;
        m_max = m_ref;
        keep = keep_ref;
        TB_CUDA(ctx, V.alloc((size_t)m_max * N));
        TB_CUDA(ctx, W.alloc((size_t)m_max * N));
        TB_CUDA(ctx, cudaMemcpyAsync(V.p, X.p, (size_t)nroots * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        for (int j = 0; j < nroots; ++j) {
            double *t = V.p + (size_t)j * N;
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                TB_TRY(dots(V.p, j, t, 1, coef.p));
                TB_TRY(lincomb(V.p, j, t, 1, 1.0, coef.p, -1.0));
            }
            TB_TRY(dots(t, 1, t, 1, scal.p));
            TB_TRY(normalize(t, scal.p));
        }
        return TBSCI_OK;
    }

    tbsci_status after_G() {
        const int cols = m - g_lo;
        for (int half = 0; half < (b32 ? 2 : 1); ++half) {
            std::vector<double> &M = half == 0 ? G : Sm;
            const double *src = hG + (size_t)half * m * cols;
            for (int i = 0; i < m; ++i)
                for (int j = g_lo; j < m; ++j) {
                    const double g = src[(size_t)i * cols + (j - g_lo)];
                    M[(size_t)i * m_max + j] = g;
                    if (i < g_lo) M[(size_t)j * m_max + i] = g;
                }
            for (int i = g_lo; i < m; ++i)
                for (int j = i + 1; j < m; ++j) {
                    const double g = 0.5 * (M[(size_t)i * m_max + j] + M[(size_t)j * m_max + i]);
                    M[(size_t)i * m_max + j] = M[(size_t)j * m_max + i] = g;
                }
        }
        return head();
    }

    tbsci_status after_R() {
        bool ok = true;
        double rmax = 0.0;
        for (int k = 0; k < nroots; ++k) {
            rnorm[k] = std::sqrt(std::max(hR[k], 0.0));
            rmax = std::max(rmax, rnorm[k]);
            const double dE = std::fabs(theta[k] - theta_prev[k]);
            if (f32) ok = ok && rnorm[k] < tol_rm;
            else ok = ok && dE < tol_e && rnorm[k] < tol_r;
        }
        if (f32) {
            // leave the FP32 phase also when its residuals stop falling (the noise
            // floor of the low-precision sigma): 30 iterations without a new best
            // residual 10% below the previous best. A slowly converging problem keeps
            // improving at that rate and stays in the cheap phase.
            if (rmax < 0.9 * best32) {
                best32 = rmax;
                stall32 = 0;
            } else if (++stall32 >= 30) {
                ok = true;
            }
        }
        theta_prev = theta;
        if (ok && f32) {
            // end of the FP32 phase: restart from the roots' Ritz vectors with FP64 sigma
            e32 = theta;
            f32 = false;
            if (b32) TB_TRY(leave_basis32());
            else TB_CUDA(ctx, cudaMemcpyAsync(V.p, X.p, (size_t)nroots * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
            p_rows = 0;
            m = 0;
            sig_lo = 0;
            sig_hi = nroots;
            g_lo = 0;
            std::fill(theta_prev.begin(), theta_prev.end(), INFINITY);
            state = St::NeedSigma;
            return TBSCI_OK;
        }
        if (ok) {
            converged = true;
            state = St::Done;
            return TBSCI_OK;
        }
        if (it >= max_iter) {
            state = St::Done;
            return TBSCI_OK;
        }
        todo.clear();
        for (int k = 0; k < nroots; ++k)
            if (rnorm[k] >= (f32 ? tol_rm : tol_r)) todo.push_back(k);
        bool restarted = false;
        // Ritz vectors of this iteration as coefficients over the current basis
        std::vector<double> p_cur((size_t)m * nroots);
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < nroots; ++k) p_cur[(size_t)i * nroots + k] = Yv[(size_t)i * m + k];
        if (m + (int)todo.size() > m_max) {
            // thick restart: keep the lowest `kk` Ritz vectors and their images, and
            // (FP64 basis) the previous iteration's Ritz vectors orthonormalised
            // against them in coefficient space, while room is left for a correction
            const int kk = std::min(keep, m);
            std::vector<double> Q((size_t)m * (kk + nroots), 0.0);  // columns of the new basis, [i][col]
            const int ldq = kk + nroots;
            for (int i = 0; i < m; ++i)
                for (int k = 0; k < kk; ++k) Q[(size_t)i * ldq + k] = Yv[(size_t)i * m + k];
            int kq = kk;
            if (!b32 && p_rows > 0) {
                for (int k = 0; k < nroots && kq + 1 < m_max; ++k) {
                    std::vector<double> z(m, 0.0);
                    for (int i = 0; i < std::min(p_rows, m); ++i) z[i] = p_prev[(size_t)i * nroots + k];
                    double z0 = 0.0;
                    for (double x : z) z0 += x * x;
                    for (int pass = 0; pass < 2; ++pass)
                        for (int c = 0; c < kq; ++c) {
                            double d = 0.0;
                            for (int i = 0; i < m; ++i) d += Q[(size_t)i * ldq + c] * z[i];
                            for (int i = 0; i < m; ++i) z[i] -= d * Q[(size_t)i * ldq + c];
                        }
                    double nz = 0.0;
                    for (double x : z) nz += x * x;
                    if (!(nz > 1e-16 * z0) || z0 == 0.0) continue;
                    nz = std::sqrt(nz);
                    for (int i = 0; i < m; ++i) Q[(size_t)i * ldq + kq] = z[i] / nz;
                    ++kq;
                }
            }
            if (b32 && !R32.p) TB_CUDA(ctx, R32.alloc((size_t)(keep + nroots) * N));
            if (!b32 && !R.p) TB_CUDA(ctx, R.alloc((size_t)(keep + nroots) * N));
            // coefficients in chunks of up to 8 columns, each chunk row-major [i][k]
            for (int k0 = 0; k0 < kq; k0 += kMaxOut) {
                const int kc = std::min(kMaxOut, kq - k0);
                for (int i = 0; i < m; ++i)
                    for (int k = 0; k < kc; ++k) hY2[(size_t)k0 * m + (size_t)i * kc + k] = Q[(size_t)i * ldq + k0 + k];
            }
            // the Ritz vectors of this iteration in the new basis: Q^T p_cur
            std::vector<double> pn((size_t)kq * nroots, 0.0);
            for (int c = 0; c < kq; ++c)
                for (int k = 0; k < nroots; ++k) {
                    double d = 0.0;
                    for (int i = 0; i < m; ++i) d += Q[(size_t)i * ldq + c] * p_cur[(size_t)i * nroots + k];
                    pn[(size_t)c * nroots + k] = d;
                }
            p_cur.swap(pn);
            TB_CUDA(ctx, cudaMemcpyAsync(dY2.p, hY2, (size_t)m * kq * sizeof(double), cudaMemcpyHostToDevice, st));
            for (int half = 0; half < 2; ++half) {
                void *src = half == 0 ? vs(0) : ws(0);
                for (int k0 = 0; k0 < kq; k0 += kMaxOut) {
                    const int kc = std::min(kMaxOut, kq - k0);
                    if (b32)
                        launch_lincomb(lgrid, st, (const float *)src, m, R32.p + (size_t)k0 * N, kc, N, 0.0,
                                       dY2.p + (size_t)k0 * m, 1.0);
                    else
                        launch_lincomb(lgrid, st, (const double *)src, m, R.p + (size_t)k0 * N, kc, N, 0.0,
                                       dY2.p + (size_t)k0 * m, 1.0);
                    TB_CUDA(ctx, cudaGetLastError());
                }
                TB_CUDA(ctx, cudaMemcpyAsync(src, b32 ? (void *)R32.p : (void *)R.p, (size_t)kq * N * es(),
                                             cudaMemcpyDeviceToDevice, st));
            }
            m = kq;
            restarted = true;
        }
        p_prev.swap(p_cur);
        p_rows = m;  // corrections appended below have zero coefficients
        // restart_keep + nroots may exceed the basis: the lowest roots' corrections
        // take the free slots (keep < max_subspace leaves at least one)
        if (m + (int)todo.size() > m_max) todo.resize(m_max - m);
        if (todo.empty()) return head();
        // Corrections into the free basis slots, then block Gram-Schmidt on the
        // device: two passes of S = V^T T, T -= V S against the basis (reads the
        // basis 4 times per iteration), then two in-block passes per vector.
        const int nb = (int)todo.size();
        void *Tb = vs(m);
        for (int j = 0; j < nb; ++j) {
            if (b32) {
                k_to_f32<<<nblocks, 256, 0, st>>>(T.p + (size_t)todo[j] * N, V32.p + (size_t)(m + j) * N, N);
                TB_CUDA(ctx, cudaGetLastError());
            } else {
                TB_CUDA(ctx, cudaMemcpyAsync(vs(m + j), T.p + (size_t)todo[j] * N, N * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
            }
            TB_TRY(dots(vs(m + j), 1, vs(m + j), 1, scal.p + 2 * j));
        }
        // block projection against the basis: S = V^T T, T -= V S; the second pass
        // runs only when the first removed more than half of a correction's
        // squared norm (decided on the device, no host round trip)
        TB_TRY(dots(vs(0), m, Tb, nb, coef.p));
        TB_TRY(lincomb(vs(0), m, Tb, nb, 1.0, coef.p, -1.0));
        TB_TRY(dots(Tb, nb, Tb, nb, red.p));
        k_gs_decide<<<1, 32, 0, st>>>(scal.p, red.p, nb, gs_skip.p);
        TB_CUDA(ctx, cudaGetLastError());
        TB_TRY(dots(vs(0), m, Tb, nb, coef.p, gs_skip.p));
        TB_TRY(lincomb(vs(0), m, Tb, nb, 1.0, coef.p, -1.0, gs_skip.p));
        for (int j = 0; j < nb; ++j) {
            void *t = vs(m + j);
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                TB_TRY(dots(Tb, j, t, 1, coef.p));
                TB_TRY(lincomb(Tb, j, t, 1, 1.0, coef.p, -1.0));
            }
            TB_TRY(dots(t, 1, t, 1, scal.p + 2 * j + 1));
            TB_TRY(normalize(t, scal.p + 2 * j + 1));
        }
        TB_CUDA(ctx, cudaMemcpyAsync(hN, scal.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        g_lo = restarted ? 0 : m;
        return finish_phase(St::WaitGS);
    }

    tbsci_status after_GS() {
        const int nb = (int)todo.size();
        // a direction that Gram-Schmidt reduced to rounding level carries nothing new
        // (FP32 storage rounds at 6e-8 of the vector's norm before projection)
        const double drop = b32 ? 1e-4 : 1e-10;
        int acc = 0;
        for (int j = 0; j < nb; ++j) {
            const double t0 = std::sqrt(std::max(hN[2 * j], 0.0)), nt = std::sqrt(std::max(hN[2 * j + 1], 0.0));
            if (!(nt > drop * t0)) continue;
            if (acc != j) TB_CUDA(ctx, cudaMemcpyAsync(vs(m + acc), vs(m + j), N * es(), cudaMemcpyDeviceToDevice, st));
            ++acc;
        }
        if (acc == 0) {
            if (g_lo == 0 && m > 0) return fetch_G();  // restarted, nothing added: refresh the Rayleigh matrix
            return head();
        }
        sig_lo = m;
        sig_hi = m + acc;
        state = St::NeedSigma;
        return TBSCI_OK;
    }

    // Runs host logic of completed phases. blocking: wait for the pending event.
    tbsci_status poll(bool blocking, bool *progressed) {
        *progressed = false;
        while (state == St::WaitG || state == St::WaitR || state == St::WaitGS) {
            if (blocking) {
                TB_CUDA(ctx, cudaEventSynchronize(evt));
            } else {
                cudaError_t q = cudaEventQuery(evt);
                if (q == cudaErrorNotReady) return TBSCI_OK;
                TB_CUDA(ctx, q);
            }
            *progressed = true;
            const St s = state;
            if (s == St::WaitG) TB_TRY(after_G());
            else if (s == St::WaitR) TB_TRY(after_R());
            else TB_TRY(after_GS());
            if (!blocking) return TBSCI_OK;  // one phase per poll keeps each scheduler pass short
        }
        return TBSCI_OK;
    }

    tbsci_status results(double *energies, double *vecs, tbsci_davidson_info *info) {
        for (int k = 0; k < nroots; ++k) energies[k] = theta[k];
        if (vecs)
            TB_CUDA(ctx, cudaMemcpyAsync(vecs, X.p, (size_t)nroots * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        if (info) {
            *info = tbsci_davidson_info{};
            info->iterations = it;
            info->converged = converged ? 1 : 0;
            info->nsigma = nsig;
            info->nsigma_f32 = nsig32;
            info->iterations_f32 = it32;
            info->precision = (int)(mixed_mode ? lowp : TBSCI_F64);
            for (int k = 0; k < nroots && k < 8; ++k) {
                info->residual[k] = rnorm[k];
                info->energy_f32[k] = e32[k];
                info->refine_delta[k] = (mixed_mode && !f32) ? theta[k] - e32[k] : 0.0;
            }
            info->seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        }
        return converged ? TBSCI_OK : fail(ctx, TBSCI_ENOCONV, "Davidson did not converge within max_iter");
    }
};

tbsci_status engine_create(tbsci_ctx *ctx, tbsci_ham *ham, Plan *plan, int nroots, const tbsci_davidson_opts *o,
                           DavEngine **out, const tbsci_pruned *pr) {
    tbsci_davidson_opts opt{};
    if (o) opt = *o;
    auto e = std::make_unique<DavEngine>();
    e->pr = pr;
    TB_TRY(e->init(ctx, ham, plan, nroots, opt));
    *out = e.release();
    return TBSCI_OK;
}

void engine_destroy(DavEngine *e) { delete e; }

void engine_set_ctx(DavEngine *e, tbsci_ctx *ctx) { e->ctx = ctx; }

bool engine_wants_sigma(DavEngine *e, const void **c, void **s, int *k, tbsci_dtype *dt) {
    return e->wants_sigma(c, s, k, dt);
}

tbsci_status engine_sigma_done(DavEngine *e) { return e->sigma_done(); }

tbsci_status engine_poll(DavEngine *e, bool blocking, bool *progressed) { return e->poll(blocking, progressed); }

bool engine_done(const DavEngine *e) { return e->state == DavEngine::St::Done; }

cudaStream_t engine_stream(const DavEngine *e) { return e->st; }

tbsci_status engine_results(DavEngine *e, double *energies, double *vecs, tbsci_davidson_info *info) {
    return e->results(energies, vecs, info);
}

size_t engine_device_bytes(int64_t N, int nroots, const tbsci_davidson_opts *o) {
    const int m_max = (o && o->max_subspace > 0) ? o->max_subspace : std::max(8 * nroots, nroots + 2);
    const int keep = (o && o->restart_keep > 0) ? o->restart_keep : std::max(nroots, m_max / 2);
    size_t vec = (size_t)(2 * m_max + keep + 4 * nroots + 1) * N * sizeof(double);
    if (o && o->mixed && o->basis_f32) {
        const int m_ref = o->max_subspace_refine > 0 ? o->max_subspace_refine : std::max(nroots + 1, m_max / 2);
        const int keep_ref = std::max(nroots, m_ref / 2);
        const size_t phase32 = (size_t)(2 * m_max + keep + nroots) * N * sizeof(float);
        const size_t phase64 = (size_t)(2 * m_ref + keep_ref + nroots) * N * sizeof(double);
        vec = std::max(phase32, phase64) + (size_t)(3 * nroots + 1) * N * sizeof(double);
    } else if (o && o->mixed) {
        vec += (size_t)2 * nroots * N * sizeof(float);
    }
    return vec + (size_t)2 * 152 * m_max * m_max * sizeof(double);
}

tbsci_status davidson_run(tbsci_ctx *ctx, tbsci_ham *ham, Plan *plan, int nroots, const tbsci_davidson_opts *o,
                          double *energies, double *vecs, tbsci_davidson_info *info, const tbsci_pruned *pr) {
    tbsci_davidson_opts opt{};
    if (o) opt = *o;
    if (!opt.stream) opt.stream = (tbsci_stream)ctx->stream;
    DavEngine *raw = nullptr;
    TB_TRY(engine_create(ctx, ham, plan, nroots, &opt, &raw, pr));
    std::unique_ptr<DavEngine> e(raw);
    cudaEvent_t s0, s1;
    TB_CUDA(ctx, cudaEventCreate(&s0));
    TB_CUDA(ctx, cudaEventCreate(&s1));
    double t_sigma = 0.0, t_sigma32 = 0.0;
    tbsci_status st = TBSCI_OK;
    while (!engine_done(e.get())) {
        const void *c;
        void *s;
        int k;
        tbsci_dtype dt;
        if (e->wants_sigma(&c, &s, &k, &dt)) {
            cudaEventRecord(s0, e->st);
            st = pr ? pruned_sigma_launch(ctx, ham, plan, pr, c, s, k, dt, e->st)
                    : sigma_launch(ctx, ham, plan, c, s, k, dt, e->st);
            if (st != TBSCI_OK) break;
            cudaEventRecord(s1, e->st);
            st = e->sigma_done();
            if (st != TBSCI_OK) break;
            cudaEventSynchronize(s1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, s0, s1);
            t_sigma += ms * 1e-3;
            if (dt != TBSCI_F64) t_sigma32 += ms * 1e-3;
        }
        bool prog;
        st = e->poll(true, &prog);
        if (st != TBSCI_OK) break;
    }
    cudaEventDestroy(s0);
    cudaEventDestroy(s1);
    if (st != TBSCI_OK) return st;
    st = e->results(energies, vecs, info);
    if (info) {
        info->seconds_sigma = t_sigma;
        info->seconds_sigma_f32 = t_sigma32;
    }
    return st;
}

tbsci_status overlap_run(tbsci_ctx *ctx, const double *A, int ma, const double *B, int mb, int64_t n, double *S,
                         cudaStream_t st) {
    TB_CHECK(ctx, ma >= 0 && mb >= 0 && n >= 0, TBSCI_EINVAL, "tbsci_overlap: negative size");
    if (ma == 0 || mb == 0) return TBSCI_OK;
    TB_CHECK(ctx, A && B && S, TBSCI_EINVAL, "tbsci_overlap: null pointer");
    TB_CHECK(ctx, (ma + kMA - 1) / kMA <= 65535 && (mb + kMB - 1) / kMB <= 65535, TBSCI_EINVAL,
             "tbsci_overlap: too many vectors");
    const int nblocks = 2 * ctx->num_sms;
    const int ldp = ma * mb;
    DevBuf<double> partial, red;
    TB_CUDA(ctx, partial.alloc((size_t)nblocks * ldp));
    TB_CUDA(ctx, red.alloc(ldp));
    dim3 grid(nblocks, (ma + kMA - 1) / kMA, (mb + kMB - 1) / kMB);
    k_dots<<<grid, kDotThreads, 0, st>>>(A, ma, B, mb, n, partial.p, ldp);
    TB_CUDA(ctx, cudaGetLastError());
    k_reduce_partials<<<(ldp + 127) / 128, 128, 0, st>>>(partial.p, nblocks, ldp, ldp, red.p);
    TB_CUDA(ctx, cudaGetLastError());
    TB_CUDA(ctx, cudaMemcpyAsync(S, red.p, (size_t)ldp * sizeof(double), cudaMemcpyDeviceToHost, st));
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    return TBSCI_OK;
}

}  // namespace tbsci

// ---------------------------------------------------------------------------
// Allocation-free overlap. Its scratch is a file-scope device array: host code
// must not use the symbol itself as a device address, so each device's address
// is looked up once with cudaGetSymbolAddress (on that device) and cached.

namespace {
constexpr int kNoAllocMaxProducts = 512;  // ma * mb
constexpr int kNoAllocMaxBlocks = 512;    // dot blocks per call
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

// partial[block][product]: 512 x 512 doubles = 2 MiB per device
static __device__ __align__(256) double g_noalloc_partial[kNoAllocMaxBlocks * kNoAllocMaxProducts];

extern "C" tbsci_status tbsci_overlap_noalloc(tbsci_ctx *ctx, const double *A, int ma, const double *B, int mb,
                                              int64_t n, double *S, tbsci_stream stream) {
    using namespace tbsci;
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, ma >= 0 && mb >= 0 && n >= 0, TBSCI_EINVAL, "tbsci_overlap_noalloc: negative size");
    if ((int64_t)ma * mb > kNoAllocMaxProducts)
        return fail(ctx, TBSCI_EINVAL,
                    "tbsci_overlap_noalloc: ma*mb = " + std::to_string((int64_t)ma * mb) +
                        " exceeds the static scratch limit of 512 products; use tbsci_overlap");
    if (ma == 0 || mb == 0) return TBSCI_OK;
    TB_CHECK(ctx, A && B && S, TBSCI_EINVAL, "tbsci_overlap_noalloc: null pointer");
    TB_CHECK(ctx, ctx->device < kNoAllocMaxDevices, TBSCI_EINVAL, "tbsci_overlap_noalloc: device index >= 64");
    double *partial = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[ctx->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
            if (e != cudaSuccess)
                return fail(ctx, TBSCI_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_addr[ctx->device] = static_cast<double *>(p);
        }
        partial = g_noalloc_addr[ctx->device];
    }
    const int nblocks = std::min(2 * ctx->num_sms, kNoAllocMaxBlocks);
    const int ldp = ma * mb;
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid(nblocks, (ma + kMA - 1) / kMA, (mb + kMB - 1) / kMB);
    k_dots<<<grid, kDotThreads, 0, st>>>(A, ma, B, mb, n, partial, ldp);
    TB_CUDA(ctx, cudaGetLastError());
    k_reduce_partials<<<(ldp + 127) / 128, 128, 0, st>>>(partial, nblocks, ldp, ldp, S);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}
