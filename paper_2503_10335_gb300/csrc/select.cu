// Bitstring selection and coefficient distributions (Sec. III.B and Fig. 3).
//
// The weight of an alpha string w in a normalised TPB vector is
// W_a(w) = sum_u c(w, u)^2 and of a beta string u is W_b(u) = sum_w c(w, u)^2;
// strings are kept when their weight is at least delta times the weight of the
// HF string (here: the string of largest weight), and the TPB space of the kept
// strings is solved again. The coefficient distribution counts |c_K| in
// logarithmic bins of |c_K / c_HF| (the caller passes the bin edges already
// scaled by |c_HF|, so both this code and a reference compare the same doubles).
// Every reduction has a fixed order: results are run-to-run identical.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace tbsci {

namespace {

constexpr int kWThreads = 256;
constexpr int kColRows = 256;  // rows per partial column sum

// rows[w] = sum_u c(w, u)^2, one CTA per row, fixed-order tree reduction
__global__ void __launch_bounds__(kWThreads) k_row_sumsq(const double *__restrict__ c, int64_t lb, double *rows) {
    __shared__ double sh[kWThreads];
    const double *r = c + (int64_t)blockIdx.x * lb;
    double acc = 0.0;
    for (int64_t u = threadIdx.x; u < lb; u += kWThreads) acc = fma(r[u], r[u], acc);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kWThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) rows[blockIdx.x] = sh[0];
}

// partial[chunk][u] = sum_{w in chunk} c(w, u)^2 over chunks of kColRows rows
__global__ void __launch_bounds__(kWThreads) k_col_sumsq(const double *__restrict__ c, int64_t la, int64_t lb,
                                                          double *partial) {
    const int64_t u = (int64_t)blockIdx.x * kWThreads + threadIdx.x;
    if (u >= lb) return;
    const int64_t w0 = (int64_t)blockIdx.y * kColRows, w1 = min(la, w0 + kColRows);
    double acc = 0.0;
    for (int64_t w = w0; w < w1; ++w) {
        const double x = c[w * lb + u];
        acc = fma(x, x, acc);
    }
    partial[(int64_t)blockIdx.y * lb + u] = acc;
}

// out[u] = sum_chunk partial[chunk][u] in chunk order
__global__ void k_col_reduce(const double *__restrict__ partial, int64_t nchunk, int64_t lb, double *out) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= lb) return;
    double acc = 0.0;
    for (int64_t k = 0; k < nchunk; ++k) acc += partial[k * lb + u];
    out[u] = acc;
}

// per-CTA counts of |x| in [edges[k], edges[k+1]): bin 0 below edges[0], bin
// nedges at or above edges[nedges-1]
__global__ void k_histogram(const double *__restrict__ x, int64_t n, const double *__restrict__ edges, int nedges,
                            unsigned long long *partial) {
    extern __shared__ unsigned long long scount[];  // [nedges + 1]
    __shared__ double sedge[257];
    for (int k = threadIdx.x; k <= nedges; k += blockDim.x) scount[k] = 0ull;
    for (int k = threadIdx.x; k < nedges; k += blockDim.x) sedge[k] = edges[k];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs(x[i]);
        int lo = 0, hi = nedges;  // first edge greater than a: the bin index
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sedge[mid] <= a) lo = mid + 1;
            else hi = mid;
        }
        atomicAdd(&scount[lo], 1ull);
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= nedges; k += blockDim.x)
        partial[(int64_t)blockIdx.x * (nedges + 1) + k] = scount[k];
}

tbsci_status weights_raw(tbsci_ctx *ctx, int64_t la, int64_t lb, const double *c, std::vector<double> &wa,
                         std::vector<double> &wb, cudaStream_t st) {
    wa.assign(la, 0.0);
    wb.assign(lb, 0.0);
    if (la == 0 || lb == 0) return TBSCI_OK;
    const int64_t nchunk = (la + kColRows - 1) / kColRows;
    DevBuf<double> rows, partial, cols;
    TB_CUDA(ctx, rows.alloc(la));
    TB_CUDA(ctx, partial.alloc((size_t)nchunk * lb));
    TB_CUDA(ctx, cols.alloc(lb));
    TB_CHECK(ctx, la <= INT32_MAX && nchunk <= 65535, TBSCI_EINVAL, "string weights: too many alpha strings");
    k_row_sumsq<<<(unsigned)la, kWThreads, 0, st>>>(c, lb, rows.p);
    TB_CUDA(ctx, cudaGetLastError());
    k_col_sumsq<<<dim3((unsigned)((lb + kWThreads - 1) / kWThreads), (unsigned)nchunk), kWThreads, 0, st>>>(
        c, la, lb, partial.p);
    TB_CUDA(ctx, cudaGetLastError());
    k_col_reduce<<<(unsigned)((lb + 255) / 256), 256, 0, st>>>(partial.p, nchunk, lb, cols.p);
    TB_CUDA(ctx, cudaGetLastError());
    TB_CUDA(ctx, cudaMemcpyAsync(wa.data(), rows.p, la * sizeof(double), cudaMemcpyDeviceToHost, st));
    TB_CUDA(ctx, cudaMemcpyAsync(wb.data(), cols.p, lb * sizeof(double), cudaMemcpyDeviceToHost, st));
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    double tot = 0.0;  // ||c||^2 from the row sums, in row order
    for (double x : wa) tot += x;
    TB_CHECK(ctx, tot > 0.0, TBSCI_EINVAL, "string weights: the vector is zero");
    for (double &x : wa) x /= tot;
    for (double &x : wb) x /= tot;
    return TBSCI_OK;
}

}  // namespace

}  // namespace tbsci

using namespace tbsci;

extern "C" {

tbsci_status tbsci_string_weights(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b, const double *c,
                                  double *wa, double *wb, tbsci_stream stream) {
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, a && b && wa && wb, TBSCI_EINVAL, "tbsci_string_weights: null argument");
    TB_CHECK(ctx, c || a->count * b->count == 0, TBSCI_EINVAL, "tbsci_string_weights: null vector");
    std::vector<double> va, vb;
    TB_TRY(weights_raw(ctx, a->count, b->count, c, va, vb, (cudaStream_t)stream));
    std::memcpy(wa, va.data(), va.size() * sizeof(double));
    std::memcpy(wb, vb.data(), vb.size() * sizeof(double));
    return TBSCI_OK;
}

tbsci_status tbsci_select_by_weight(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b, const double *c,
                                    double delta, uint64_t *sel_a, int64_t *na, uint64_t *sel_b, int64_t *nb,
                                    tbsci_stream stream) {
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, a && b && c && sel_a && na && sel_b && nb, TBSCI_EINVAL, "tbsci_select_by_weight: null argument");
    TB_CHECK(ctx, delta >= 0.0, TBSCI_EINVAL, "tbsci_select_by_weight: delta must be >= 0");
    TB_CHECK(ctx, a->count > 0 && b->count > 0, TBSCI_EINVAL, "tbsci_select_by_weight: empty space");
    std::vector<double> wa, wb;
    cudaStream_t st = (cudaStream_t)stream;
    TB_TRY(weights_raw(ctx, a->count, b->count, c, wa, wb, st));
    std::vector<uint64_t> sa(a->count), sb(b->count);
    TB_CUDA(ctx, cudaMemcpy(sa.data(), a->d_str.p, a->count * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    TB_CUDA(ctx, cudaMemcpy(sb.data(), b->d_str.p, b->count * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    auto pick = [&](const std::vector<double> &w, const std::vector<uint64_t> &s, uint64_t *out, int64_t *n) {
        const double hf = *std::max_element(w.begin(), w.end());  // the HF string: largest weight
        int64_t k = 0;
        for (size_t i = 0; i < w.size(); ++i)
            if (w[i] >= delta * hf) out[k++] = s[i];
        *n = k;
    };
    pick(wa, sa, sel_a, na);
    pick(wb, sb, sel_b, nb);
    return TBSCI_OK;
}

tbsci_status tbsci_coefficient_histogram(tbsci_ctx *ctx, const double *x, int64_t n, const double *edges, int nedges,
                                         int64_t *counts, tbsci_stream stream) {
    if (!ctx) return TBSCI_EINVAL;
    TB_CUDA(ctx, cudaSetDevice(ctx->device));
    TB_CHECK(ctx, edges && counts && n >= 0, TBSCI_EINVAL, "tbsci_coefficient_histogram: null argument");
    TB_CHECK(ctx, nedges >= 1 && nedges <= 256, TBSCI_EINVAL, "tbsci_coefficient_histogram: 1..256 edges");
    for (int k = 1; k < nedges; ++k)
        TB_CHECK(ctx, edges[k] > edges[k - 1], TBSCI_EINVAL, "tbsci_coefficient_histogram: edges must ascend");
    std::fill(counts, counts + nedges + 1, 0);
    if (n == 0) return TBSCI_OK;
    TB_CHECK(ctx, x, TBSCI_EINVAL, "tbsci_coefficient_histogram: null vector");
    cudaStream_t st = (cudaStream_t)stream;
    const int nblocks = (int)std::min<int64_t>(4 * ctx->num_sms, (n + 255) / 256);
    DevBuf<double> dedges;
    DevBuf<unsigned long long> partial;
    TB_CUDA(ctx, dedges.alloc(nedges));
    TB_CUDA(ctx, partial.alloc((size_t)nblocks * (nedges + 1)));
    TB_CUDA(ctx, cudaMemcpyAsync(dedges.p, edges, nedges * sizeof(double), cudaMemcpyHostToDevice, st));
    k_histogram<<<nblocks, 256, (nedges + 1) * sizeof(unsigned long long), st>>>(x, n, dedges.p, nedges, partial.p);
    TB_CUDA(ctx, cudaGetLastError());
    std::vector<unsigned long long> h((size_t)nblocks * (nedges + 1));
    TB_CUDA(ctx, cudaMemcpyAsync(h.data(), partial.p, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 st));
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k <= nedges; ++k) counts[k] += (int64_t)h[(size_t)b * (nedges + 1) + k];
    return TBSCI_OK;
}

}  // extern "C"
