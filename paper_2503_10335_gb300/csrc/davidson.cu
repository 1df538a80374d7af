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

#include "internal.cuh"

namespace tbsci {

namespace {

constexpr int kDotThreads = 256;
constexpr int kMA = 8;  // rows of A per dot block
constexpr int kMB = 4;  // rows of B per dot block

// partial[b][i][j] over this block's slice of K: sum A[i][K] * B[j][K]
__global__ void __launch_bounds__(kDotThreads) k_dots(const double *__restrict__ A, int ma, const double *__restrict__ B,
                                                      int mb, int64_t N, double *partial, int ldp) {
    __shared__ double sh[kDotThreads / 32][kMA * kMB];
    const int i0 = blockIdx.y * kMA, j0 = blockIdx.z * kMB;
    const int na = min(kMA, ma - i0), nb = min(kMB, mb - j0);
    double acc[kMA][kMB];
#pragma unroll
    for (int i = 0; i < kMA; ++i)
#pragma unroll
        for (int j = 0; j < kMB; ++j) acc[i][j] = 0.0;
    for (int64_t K = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; K < N; K += (int64_t)gridDim.x * kDotThreads) {
        double b[kMB];
#pragma unroll
        for (int j = 0; j < kMB; ++j) b[j] = j < nb ? __ldg(B + (size_t)(j0 + j) * N + K) : 0.0;
#pragma unroll
        for (int i = 0; i < kMA; ++i) {
            if (i < na) {
                double a = __ldg(A + (size_t)(i0 + i) * N + K);
#pragma unroll
                for (int j = 0; j < kMB; ++j) acc[i][j] = fma(a, b[j], acc[i][j]);
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kMA; ++i)
#pragma unroll
        for (int j = 0; j < kMB; ++j) {
            double v = acc[i][j];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sh[w][i * kMB + j] = v;
        }
    __syncthreads();
    if (threadIdx.x < kMA * kMB) {
        int i = threadIdx.x / kMB, j = threadIdx.x % kMB;
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

// out[k][K] = beta * out[k][K] + sum_i Y[i][k] * A[i][K], k < kout <= 8
__global__ void __launch_bounds__(256) k_lincomb(const double *__restrict__ A, int m, double *out, int kout, int64_t N,
                                                 double beta, const double *__restrict__ Y) {
    __shared__ double sY[kMaxBasis * kMaxOut];
    for (int x = threadIdx.x; x < m * kout; x += blockDim.x) sY[x] = Y[x];
    __syncthreads();
    for (int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; K < N; K += (int64_t)gridDim.x * blockDim.x) {
        double acc[kMaxOut];
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k) acc[k] = (k < kout && beta != 0.0) ? beta * out[(size_t)k * N + K] : 0.0;
        for (int i = 0; i < m; ++i) {
            double a = __ldg(A + (size_t)i * N + K);
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
                if (k < kout) acc[k] = fma(sY[i * kout + k], a, acc[k]);
        }
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k)
            if (k < kout) out[(size_t)k * N + K] = acc[k];
    }
}

// r = wy - theta x; t = r / clamp(theta - diag); partial norms of r
__global__ void __launch_bounds__(kDotThreads) k_residual(const double *__restrict__ X, const double *__restrict__ WY,
                                                          const double *__restrict__ diag, const double *__restrict__ theta,
                                                          int nroots, int64_t N, double *T, double *partial) {
    __shared__ double sh[kDotThreads / 32][kMaxOut];
    double acc[kMaxOut];
#pragma unroll
    for (int k = 0; k < kMaxOut; ++k) acc[k] = 0.0;
    for (int64_t K = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; K < N; K += (int64_t)gridDim.x * kDotThreads) {
        double d = diag[K];
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k) {
            if (k < nroots) {
                double r = WY[(size_t)k * N + K] - theta[k] * X[(size_t)k * N + K];
                acc[k] = fma(r, r, acc[k]);
                double den = theta[k] - d;
                if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
                T[(size_t)k * N + K] = r / den;
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kMaxOut; ++k) {
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

__global__ void k_scale_copy(const double *__restrict__ x, double s, double *y, int64_t N) {
    for (int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; K < N; K += (int64_t)gridDim.x * blockDim.x)
        y[K] = s * x[K];
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

struct Dav {
    tbsci_ctx *ctx;
    tbsci_ham *ham;
    Plan *plan;
    cudaStream_t st;
    int64_t N;
    int nblocks;
    DevBuf<double> partial, red, dY, dtheta;
    DevBuf<float> v32, w32;
    double t_sigma = 0.0;
    int nsig = 0, nsig32 = 0;

    tbsci_status dots(const double *A, int ma, const double *B, int mb, std::vector<double> &out) {
        // out[i*mb + j] = A_i . B_j
        dim3 grid(nblocks, (ma + kMA - 1) / kMA, (mb + kMB - 1) / kMB);
        int ldp = ma * mb;
        k_dots<<<grid, kDotThreads, 0, st>>>(A, ma, B, mb, N, partial.p, ldp);
        TB_CUDA(ctx, cudaGetLastError());
        k_reduce_partials<<<(ldp + 127) / 128, 128, 0, st>>>(partial.p, nblocks, ldp, ldp, red.p);
        TB_CUDA(ctx, cudaGetLastError());
        out.resize(ldp);
        TB_CUDA(ctx, cudaMemcpyAsync(out.data(), red.p, ldp * sizeof(double), cudaMemcpyDeviceToHost, st));
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        return TBSCI_OK;
    }
    // out[0..kout) = beta*out + sum_i Y[i][k] A[i]
    tbsci_status lincomb(const double *A, int m, double *out, int kout, double beta, const std::vector<double> &Y) {
        TB_CUDA(ctx, cudaMemcpyAsync(dY.p, Y.data(), (size_t)m * kout * sizeof(double), cudaMemcpyHostToDevice, st));
        k_lincomb<<<nblocks, 256, 0, st>>>(A, m, out, kout, N, beta, dY.p);
        TB_CUDA(ctx, cudaGetLastError());
        // Y is reused by the next call: finish this one first
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        return TBSCI_OK;
    }
    tbsci_status sigma(const double *V, double *W, int k, bool f32) {
        auto t0 = std::chrono::steady_clock::now();
        if (!f32) {
            TB_TRY(sigma_launch(ctx, ham, plan, V, W, k, TBSCI_F64, st));
            nsig += k;
        } else {
            int64_t n = N * k;
            k_to_f32<<<nblocks, 256, 0, st>>>(V, v32.p, n);
            TB_CUDA(ctx, cudaGetLastError());
            TB_TRY(sigma_launch(ctx, ham, plan, v32.p, w32.p, k, TBSCI_F32, st));
            k_to_f64<<<nblocks, 256, 0, st>>>(w32.p, W, n);
            TB_CUDA(ctx, cudaGetLastError());
            nsig += k;
            nsig32 += k;
        }
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        t_sigma += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return TBSCI_OK;
    }
};

}  // namespace

tbsci_status davidson_run(tbsci_ctx *ctx, tbsci_ham *ham, Plan *plan, int nroots, const tbsci_davidson_opts *o,
                          double *energies, double *vecs, tbsci_davidson_info *info) {
    auto T0 = std::chrono::steady_clock::now();
    tbsci_davidson_opts opt{};
    if (o) opt = *o;
    const int m_max = opt.max_subspace > 0 ? opt.max_subspace : std::max(8 * nroots, nroots + 2);
    const int keep = opt.restart_keep > 0 ? opt.restart_keep : std::max(nroots, m_max / 2);
    const int max_iter = opt.max_iter > 0 ? opt.max_iter : 1000;
    const double tol_e = opt.tol_energy > 0 ? opt.tol_energy : 1e-9;
    const double tol_r = opt.tol_residual > 0 ? opt.tol_residual : 1e-5;
    const double tol_rm = opt.tol_mixed_residual > 0 ? opt.tol_mixed_residual : 5e-5;
    TB_CHECK(ctx, nroots >= 1 && nroots <= kMaxOut, TBSCI_EINVAL, "nroots must be in 1..8");
    TB_CHECK(ctx, m_max >= nroots + 1 && m_max <= kMaxBasis, TBSCI_EINVAL, "max_subspace must be in nroots+1..128");
    TB_CHECK(ctx, keep >= nroots && keep < m_max, TBSCI_EINVAL, "restart_keep must be in nroots..max_subspace-1");
    Dav D;
    D.ctx = ctx;
    D.ham = ham;
    D.plan = plan;
    D.st = opt.stream ? (cudaStream_t)opt.stream : ctx->stream;
    D.N = plan->A.l * plan->B.l;
    const int64_t N = D.N;
    TB_CHECK(ctx, N >= nroots, TBSCI_EINVAL, "space has fewer determinants than roots");
    D.nblocks = 2 * ctx->num_sms;
    // dot partials: up to max_subspace x max_subspace products per block
    TB_CUDA(ctx, D.partial.alloc((size_t)D.nblocks * kMaxBasis * kMaxBasis));
    TB_CUDA(ctx, D.red.alloc(kMaxBasis * kMaxBasis));
    TB_CUDA(ctx, D.dY.alloc(kMaxBasis * kMaxOut));
    TB_CUDA(ctx, D.dtheta.alloc(kMaxOut));
    DevBuf<double> V, W, X, WY, T, diag, R;  // R: Ritz block of a thick restart
    TB_CUDA(ctx, V.alloc((size_t)m_max * N));
    TB_CUDA(ctx, W.alloc((size_t)m_max * N));
    TB_CUDA(ctx, X.alloc((size_t)nroots * N));
    TB_CUDA(ctx, WY.alloc((size_t)nroots * N));
    TB_CUDA(ctx, T.alloc((size_t)nroots * N));
    TB_CUDA(ctx, diag.alloc(N));
    bool f32 = opt.mixed != 0;
    if (f32) {
        TB_CUDA(ctx, D.v32.alloc((size_t)nroots * N));
        TB_CUDA(ctx, D.w32.alloc((size_t)nroots * N));
    }
    cudaStream_t st = D.st;
    TB_TRY(diagonal_launch(ctx, ham, plan, diag.p, st));

    // guess: unit vectors at the lowest (H_KK, K)
    std::vector<int64_t> chosen;
    {
        DevBuf<double> bv;
        DevBuf<int64_t> bi, dskip;
        TB_CUDA(ctx, bv.alloc(D.nblocks));
        TB_CUDA(ctx, bi.alloc(D.nblocks));
        TB_CUDA(ctx, dskip.alloc(kMaxOut));
        std::vector<double> hv(D.nblocks);
        std::vector<int64_t> hi(D.nblocks);
        for (int r = 0; r < nroots; ++r) {
            if (!chosen.empty())
                TB_CUDA(ctx, cudaMemcpyAsync(dskip.p, chosen.data(), chosen.size() * sizeof(int64_t),
                                             cudaMemcpyHostToDevice, st));
            k_argmin<<<D.nblocks, 256, 0, st>>>(diag.p, N, dskip.p, (int)chosen.size(), bv.p, bi.p);
            TB_CUDA(ctx, cudaGetLastError());
            TB_CUDA(ctx, cudaMemcpyAsync(hv.data(), bv.p, D.nblocks * sizeof(double), cudaMemcpyDeviceToHost, st));
            TB_CUDA(ctx, cudaMemcpyAsync(hi.data(), bi.p, D.nblocks * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            TB_CUDA(ctx, cudaStreamSynchronize(st));
            double best = INFINITY;
            int64_t bidx = INT64_MAX;
            for (int b = 0; b < D.nblocks; ++b)
                if (hv[b] < best || (hv[b] == best && hi[b] < bidx)) {
                    best = hv[b];
                    bidx = hi[b];
                }
            chosen.push_back(bidx);
        }
    }
    TB_CUDA(ctx, cudaMemsetAsync(V.p, 0, (size_t)nroots * N * sizeof(double), st));
    const double one = 1.0;
    for (int r = 0; r < nroots; ++r)
        TB_CUDA(ctx, cudaMemcpyAsync(V.p + (size_t)r * N + chosen[r], &one, sizeof(double), cudaMemcpyHostToDevice, st));
    TB_CUDA(ctx, cudaStreamSynchronize(st));

    int m = nroots;
    TB_TRY(D.sigma(V.p, W.p, m, f32));
    std::vector<double> G((size_t)m_max * m_max, 0.0), tmp;
    auto refresh_G = [&](int lo, int hi) -> tbsci_status {
        // columns lo..hi of G against all rows < hi, mirrored
        TB_TRY(D.dots(V.p, hi, W.p + (size_t)lo * N, hi - lo, tmp));
        for (int i = 0; i < hi; ++i)
            for (int j = lo; j < hi; ++j) {
                double g = tmp[(size_t)i * (hi - lo) + (j - lo)];
                G[(size_t)i * m_max + j] = g;
                if (i < lo) G[(size_t)j * m_max + i] = g;
            }
        // symmetrise the new block
        for (int i = lo; i < hi; ++i)
            for (int j = i + 1; j < hi; ++j) {
                double g = 0.5 * (G[(size_t)i * m_max + j] + G[(size_t)j * m_max + i]);
                G[(size_t)i * m_max + j] = G[(size_t)j * m_max + i] = g;
            }
        return TBSCI_OK;
    };
    TB_TRY(refresh_G(0, m));
    std::vector<double> theta(nroots), theta_prev(nroots, INFINITY), rnorm(nroots, INFINITY);
    std::vector<double> e32(nroots, 0.0);
    int it = 0, it32 = 0;
    double best32 = INFINITY;  // FP32 phase: smallest max-residual so far
    int stall32 = 0;
    bool converged = false;
    tbsci_status result = TBSCI_OK;
    for (it = 1; it <= max_iter; ++it) {
        if (f32) ++it32;
        std::vector<double> Gm((size_t)m * m), w, Yv;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) Gm[(size_t)i * m + j] = G[(size_t)i * m_max + j];
        jacobi_eigh(Gm, m, w, Yv);
        std::vector<double> Y((size_t)m * nroots);
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < nroots; ++k) Y[(size_t)i * nroots + k] = Yv[(size_t)i * m + k];
        for (int k = 0; k < nroots; ++k) theta[k] = w[k];
        TB_TRY(D.lincomb(V.p, m, X.p, nroots, 0.0, Y));
        TB_TRY(D.lincomb(W.p, m, WY.p, nroots, 0.0, Y));
        TB_CUDA(ctx, cudaMemcpyAsync(D.dtheta.p, theta.data(), nroots * sizeof(double), cudaMemcpyHostToDevice, st));
        k_residual<<<D.nblocks, kDotThreads, 0, st>>>(X.p, WY.p, diag.p, D.dtheta.p, nroots, N, T.p, D.partial.p);
        TB_CUDA(ctx, cudaGetLastError());
        k_reduce_partials<<<1, 32, 0, st>>>(D.partial.p, D.nblocks, kMaxOut, nroots, D.red.p);
        TB_CUDA(ctx, cudaGetLastError());
        TB_CUDA(ctx, cudaMemcpyAsync(rnorm.data(), D.red.p, nroots * sizeof(double), cudaMemcpyDeviceToHost, st));
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        bool ok = true;
        double rmax = 0.0;
        for (int k = 0; k < nroots; ++k) {
            rnorm[k] = std::sqrt(rnorm[k]);
            rmax = std::max(rmax, rnorm[k]);
            double dE = std::fabs(theta[k] - theta_prev[k]);
            if (f32) ok = ok && rnorm[k] < tol_rm;
            else ok = ok && dE < tol_e && rnorm[k] < tol_r;
        }
        if (f32) {
            // leave the FP32 phase also when its residuals stop falling (FP32 noise floor)
            if (rmax < 0.9 * best32) {
                best32 = rmax;
                stall32 = 0;
            } else if (++stall32 >= 8) {
                ok = true;
            }
        }
        theta_prev = theta;
        if (ok && f32) {
            // end of the FP32 phase: restart from the Ritz vectors with FP64 sigma
            e32 = theta;
            f32 = false;
            TB_CUDA(ctx, cudaMemcpyAsync(V.p, X.p, (size_t)nroots * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
            m = nroots;
            TB_TRY(D.sigma(V.p, W.p, m, false));
            TB_TRY(refresh_G(0, m));
            std::fill(theta_prev.begin(), theta_prev.end(), INFINITY);
            continue;
        }
        if (ok) {
            converged = true;
            break;
        }
        std::vector<int> todo;
        for (int k = 0; k < nroots; ++k)
            if (rnorm[k] >= (f32 ? tol_rm : tol_r)) todo.push_back(k);
        if (m + (int)todo.size() > m_max) {
            // thick restart: keep the lowest `kk` Ritz vectors and their images
            const int kk = std::min(keep, m);
            if (!R.p) TB_CUDA(ctx, R.alloc((size_t)keep * N));
            std::vector<double> Yk;
            for (int half = 0; half < 2; ++half) {
                double *src = half == 0 ? V.p : W.p;
                for (int k0 = 0; k0 < kk; k0 += kMaxOut) {
                    const int kc = std::min(kMaxOut, kk - k0);
                    Yk.assign((size_t)m * kc, 0.0);
                    for (int i = 0; i < m; ++i)
                        for (int k = 0; k < kc; ++k) Yk[(size_t)i * kc + k] = Yv[(size_t)i * m + k0 + k];
                    TB_TRY(D.lincomb(src, m, R.p + (size_t)k0 * N, kc, 0.0, Yk));
                }
                TB_CUDA(ctx, cudaMemcpyAsync(src, R.p, (size_t)kk * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
            m = kk;
            TB_TRY(refresh_G(0, m));
        }
        const int m_old = m;
        for (int k : todo) {
            if (m >= m_max) break;  // the basis is full: remaining corrections wait for the next iteration
            double *t = T.p + (size_t)k * N;
            std::vector<double> nn;
            TB_TRY(D.dots(t, 1, t, 1, nn));
            const double t0 = std::sqrt(nn[0]);
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<double> cdot;
                TB_TRY(D.dots(V.p, m, t, 1, cdot));
                for (auto &x : cdot) x = -x;
                TB_TRY(D.lincomb(V.p, m, t, 1, 1.0, cdot));
            }
            TB_TRY(D.dots(t, 1, t, 1, nn));
            const double nt = std::sqrt(nn[0]);
            if (!(nt > 1e-10 * t0)) continue;
            k_scale_copy<<<D.nblocks, 256, 0, st>>>(t, 1.0 / nt, V.p + (size_t)m * N, N);
            TB_CUDA(ctx, cudaGetLastError());
            ++m;
        }
        if (m > m_old) {
            TB_TRY(D.sigma(V.p + (size_t)m_old * N, W.p + (size_t)m_old * N, m - m_old, f32));
            TB_TRY(refresh_G(m_old, m));
        }
    }
    if (it > max_iter) it = max_iter;
    if (!converged) result = fail(ctx, TBSCI_ENOCONV, "Davidson did not converge within max_iter");
    for (int k = 0; k < nroots; ++k) energies[k] = theta[k];
    if (vecs)
        TB_CUDA(ctx, cudaMemcpyAsync(vecs, X.p, (size_t)nroots * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    if (info) {
        *info = tbsci_davidson_info{};
        info->iterations = it;
        info->converged = converged ? 1 : 0;
        info->nsigma = D.nsig;
        info->nsigma_f32 = D.nsig32;
        info->iterations_f32 = it32;
        for (int k = 0; k < nroots && k < 8; ++k) {
            info->residual[k] = rnorm[k];
            info->energy_f32[k] = e32[k];
        }
        info->seconds_sigma = D.t_sigma;
        info->seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - T0).count();
    }
    return result;
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
