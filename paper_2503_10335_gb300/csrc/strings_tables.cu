// String sets (Sec. II.A, Eq. 3) and their single/double excitation links
// (BETA_SINGLE_LINK / BETA_DOUBLE_LINK, Sec. II.C), built on the device.
//
// Strings: the full space is unranked in colex order (= ascending integer
// order) from the combinatorial number system; a selected list is sorted by a
// bitonic network and validated (electron count, orbital range, duplicates).
//
// Links: one warp per source string walks its candidate excitations in the
// documented order, 32 at a time; the target's index comes from the colex rank
// (full space) or a binary search (selected set), the sign from masked
// popcounts, and a ballot + prefix popcount compacts the hits in order.
// Count pass -> exclusive scan -> fill pass.
#include <algorithm>

#include "internal.cuh"

namespace tbsci {

namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ int64_t binom(const int64_t *__restrict__ B, int m, int k) {
    return (k < 0 || k > m) ? 0 : __ldg(B + m * 65 + k);
}

// k-th combination of N out of n in colex order.
__global__ void k_unrank(uint64_t *out, int64_t count, int n, int N, const int64_t *__restrict__ B) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    uint64_t s = 0;
    int64_t r = k;
    int top = n;  // next position must be below `top`
    for (int i = N; i >= 1; --i) {
        int c = i - 1;
        while (c + 1 < top && binom(B, c + 1, i) <= r) ++c;
        r -= binom(B, c, i);
        s |= 1ull << c;
        top = c;
    }
    out[k] = s;
}

__global__ void k_fill_u64(uint64_t *a, int64_t from, int64_t to, uint64_t v) {
    int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < to) a[i] = v;
}

// One compare-exchange stage of a bitonic sorting network over P = 2^m keys.
__global__ void k_bitonic(uint64_t *a, int64_t P, int64_t j, int64_t k) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= P) return;
    int64_t x = i ^ j;
    if (x <= i) return;
    uint64_t u = a[i], v = a[x];
    bool up = (i & k) == 0;
    if ((u > v) == up) {
        a[i] = v;
        a[x] = u;
    }
}

// flags: 1 wrong electron count, 2 bit >= n, 4 duplicate
__global__ void k_validate(const uint64_t *a, int64_t m, int n, int N, int *flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t s = a[i];
    int f = 0;
    if (__popcll(s) != N) f |= 1;
    if (n < 64 && (s >> n) != 0) f |= 2;
    if (i > 0 && a[i - 1] == s) f |= 4;
    if (f) atomicOr(flags, f);
}

__device__ __forceinline__ uint64_t lowmask(int k) { return (1ull << k) - 1ull; }

// Colex rank of a string of the full space.
__device__ __forceinline__ int64_t colex_rank(uint64_t s, const int64_t *__restrict__ B) {
    int64_t r = 0;
    int k = 1;
    while (s) {
        int c = __ffsll((long long)s) - 1;
        r += binom(B, c, k);
        ++k;
        s &= s - 1;
    }
    return r;
}

__device__ __forceinline__ int64_t bsearch_u64(const uint64_t *__restrict__ a, int64_t len, uint64_t s) {
    int64_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        uint64_t v = __ldg(a + mid);
        if (v == s) return mid;
        if (v < s) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

struct LinkArgs {
    const uint64_t *str;
    int64_t l;
    int n, N;
    int full;
    const int64_t *B;
    int64_t *counts;  // count pass
    const int64_t *off;  // fill pass
    tbsci_single_link *e1;
    tbsci_double_link *e2;
};

// Pair tables: pair t of m items in lexicographic (i < j) order.
__device__ void build_pairs(uint8_t *pi, uint8_t *pj, int m) {
    int t = 0;
    // every thread computes the same table slice it writes; simple serial fill by thread 0
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i)
            for (int j = i + 1; j < m; ++j) {
                pi[t] = (uint8_t)i;
                pj[t] = (uint8_t)j;
                ++t;
            }
    }
}

template <bool DBL, bool FILL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_links(LinkArgs A) {
    __shared__ uint8_t s_occ[kWarpsPerBlock][64], s_vir[kWarpsPerBlock][64];
    __shared__ uint8_t s_poi[DBL ? 2016 : 1], s_poj[DBL ? 2016 : 1];
    __shared__ uint8_t s_pvi[DBL ? 2016 : 1], s_pvj[DBL ? 2016 : 1];
    const int n = A.n, N = A.N, nv = n - N;
    if (DBL) {
        build_pairs(s_poi, s_poj, N);
        build_pairs(s_pvi, s_pvj, nv);
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (row >= A.l) return;
    const uint64_t J = A.str[row];
    // occupied / empty orbital lists, ascending
    for (int base = 0; base < n; base += 32) {
        int i = base + lane;
        bool in = i < n;
        bool occ = in && ((J >> i) & 1ull);
        unsigned mo = __ballot_sync(0xffffffffu, occ);
        unsigned mv = __ballot_sync(0xffffffffu, in && !occ);
        unsigned lt = (1u << lane) - 1u;
        int before_o = __popcll(J & lowmask(base));  // occupied below `base`
        int before_v = base - before_o;
        if (occ) s_occ[warp][before_o + __popc(mo & lt)] = (uint8_t)i;
        if (in && !occ) s_vir[warp][before_v + __popc(mv & lt)] = (uint8_t)i;
    }
    __syncwarp();
    const int64_t npo = DBL ? (int64_t)N * (N - 1) / 2 : N;
    const int64_t npv = DBL ? (int64_t)nv * (nv - 1) / 2 : nv;
    const int64_t ncand = npo * npv;
    int64_t cnt = 0;
    const int64_t base_out = FILL ? A.off[row] : 0;
    for (int64_t c0 = 0; c0 < ncand; c0 += 32) {
        int64_t c = c0 + lane;
        bool found = false;
        int64_t tgt = -1;
        int sign = 0, p = 0, q = 0, r = 0, s = 0;
        if (c < ncand) {
            int64_t to = c / npv, tv = c - to * npv;
            uint64_t T;
            if (!DBL) {
                q = s_occ[warp][to];
                p = s_vir[warp][tv];
                int lo = min(p, q), hi = max(p, q);
                uint64_t between = lowmask(hi) & ~lowmask(lo + 1);
                sign = (__popcll(J & between) & 1) ? -1 : 1;
                T = (J & ~(1ull << q)) | (1ull << p);
            } else {
                q = s_occ[warp][s_poi[to]];
                s = s_occ[warp][s_poj[to]];
                p = s_vir[warp][s_pvi[tv]];
                r = s_vir[warp][s_pvj[tv]];
                // a_q, then a_s, then a+_r, then a+_p, each sign from the
                // occupied orbitals below the operator's orbital
                uint64_t x = J;
                int par = __popcll(x & lowmask(q));
                x &= ~(1ull << q);
                par += __popcll(x & lowmask(s));
                x &= ~(1ull << s);
                par += __popcll(x & lowmask(r));
                x |= 1ull << r;
                par += __popcll(x & lowmask(p));
                x |= 1ull << p;
                sign = (par & 1) ? -1 : 1;
                T = x;
            }
            tgt = A.full ? colex_rank(T, A.B) : bsearch_u64(A.str, A.l, T);
            found = tgt >= 0;
        }
        unsigned m = __ballot_sync(0xffffffffu, found);
        if (FILL && found) {
            int64_t pos = base_out + cnt + __popc(m & ((1u << lane) - 1u));
            if (!DBL) {
                tbsci_single_link e;
                e.target = (int32_t)tgt;
                e.sign = (int8_t)sign;
                e.p = (uint8_t)p;
                e.q = (uint8_t)q;
                e.pad = 0;
                A.e1[pos] = e;
            } else {
                tbsci_double_link e;
                e.target = (int32_t)tgt;
                e.sign = (int8_t)sign;
                e.p = (uint8_t)p;
                e.r = (uint8_t)r;
                e.q = (uint8_t)q;
                e.s = (uint8_t)s;
                e.pad[0] = e.pad[1] = e.pad[2] = 0;
                A.e2[pos] = e;
            }
        }
        cnt += __popc(m);
    }
    if (!FILL && lane == 0) A.counts[row] = cnt;
}

// ---- exclusive scan (three passes: block sums, scan of sums, local scans)

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ int64_t block_scan_excl(int64_t v, int64_t *sh, int64_t *total) {
    // Hillis-Steele over warps: warp inclusive scans, then scan of warp totals.
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;  // inclusive totals of warps
    }
    __syncthreads();
    int64_t before = (w > 0 ? sh[w - 1] : 0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(const int64_t *in, int64_t n, int64_t *sums) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) v += in[i];
    }
    int64_t tot;
    block_scan_excl(v, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_top(int64_t *sums, int64_t nb, int64_t *total_out) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        int64_t tot;
        int64_t ex = block_scan_excl(v, sh, &tot);
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_local(const int64_t *in, int64_t n, const int64_t *sums,
                                                            int64_t *out) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t vals[kScanItems];
    int64_t v = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        vals[k] = i < n ? in[i] : 0;
        v += vals[k];
    }
    int64_t ex = block_scan_excl(v, sh, nullptr) + sums[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = ex;
        ex += vals[k];
    }
}

}  // namespace

tbsci_status scan_exclusive(tbsci_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    DevBuf<int64_t> sums;
    TB_CUDA(ctx, sums.alloc(std::max<int64_t>(nb, 1)));
    if (nb > 0) {
        k_scan_sums<<<(unsigned)nb, kScanBlock, 0, st>>>(in, n, sums.p);
        TB_CUDA(ctx, cudaGetLastError());
    }
    k_scan_top<<<1, kScanBlock, 0, st>>>(sums.p, nb, out + n);
    TB_CUDA(ctx, cudaGetLastError());
    if (nb > 0) {
        k_scan_local<<<(unsigned)nb, kScanBlock, 0, st>>>(in, n, sums.p, out);
        TB_CUDA(ctx, cudaGetLastError());
    }
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    return TBSCI_OK;
}

static int64_t host_binom(int m, int k) {
    if (k < 0 || k > m) return 0;
    // C(m-k+i, i) at step i; the product is formed in 128 bits
    unsigned __int128 v = 1;
    for (int i = 1; i <= k; ++i) v = v * (unsigned)(m - k + i) / (unsigned)i;
    return v > (unsigned __int128)INT64_MAX ? INT64_MAX : (int64_t)v;
}

tbsci_status strings_build(tbsci_ctx *ctx, int norb, int nelec, const uint64_t *sel, int64_t nsel,
                           tbsci_strings *out) {
    TB_CHECK(ctx, norb >= 1 && norb <= 64, TBSCI_EINVAL, "norb must be in 1..64");
    TB_CHECK(ctx, nelec >= 0 && nelec <= norb, TBSCI_EINVAL, "nelec must be in 0..norb");
    cudaStream_t st = ctx->stream;
    out->ctx = ctx;
    out->norb = norb;
    out->nelec = nelec;
    if (!sel) {
        int64_t count = host_binom(norb, nelec);
        TB_CHECK(ctx, count <= INT32_MAX, TBSCI_EINVAL, "string space exceeds 2^31-1 strings");
        out->count = count;
        out->full = true;
        TB_CUDA(ctx, out->d_str.alloc(count));
        if (count > 0) {
            k_unrank<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out->d_str.p, count, norb, nelec,
                                                                      ctx->d_binom.p);
            TB_CUDA(ctx, cudaGetLastError());
        }
        TB_CUDA(ctx, cudaStreamSynchronize(st));
        return TBSCI_OK;
    }
    TB_CHECK(ctx, nsel >= 0 && nsel <= INT32_MAX, TBSCI_EINVAL, "nsel must be in 0..2^31-1");
    out->count = nsel;
    out->full = false;
    int64_t P = 1;
    while (P < nsel) P <<= 1;
    DevBuf<uint64_t> work;
    TB_CUDA(ctx, work.alloc(std::max<int64_t>(P, 1)));
    if (nsel > 0) {
        TB_CUDA(ctx, cudaMemcpyAsync(work.p, sel, nsel * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        if (P > nsel) {
            k_fill_u64<<<(unsigned)((P - nsel + 255) / 256), 256, 0, st>>>(work.p, nsel, P, ~0ull);
            TB_CUDA(ctx, cudaGetLastError());
        }
        for (int64_t k = 2; k <= P; k <<= 1)
            for (int64_t j = k >> 1; j > 0; j >>= 1) {
                k_bitonic<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(work.p, P, j, k);
            }
        TB_CUDA(ctx, cudaGetLastError());
    }
    DevBuf<int> flags;
    TB_CUDA(ctx, flags.alloc(1));
    TB_CUDA(ctx, cudaMemsetAsync(flags.p, 0, sizeof(int), st));
    if (nsel > 0) {
        k_validate<<<(unsigned)((nsel + 255) / 256), 256, 0, st>>>(work.p, nsel, norb, nelec, flags.p);
        TB_CUDA(ctx, cudaGetLastError());
    }
    int hf = 0;
    TB_CUDA(ctx, cudaMemcpyAsync(&hf, flags.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    if (hf & 2) return fail(ctx, TBSCI_EINVAL, "selected string has a bit at or above norb");
    if (hf & 1) return fail(ctx, TBSCI_EINVAL, "selected string has the wrong electron count");
    if (hf & 4) return fail(ctx, TBSCI_EINVAL, "selected strings contain a duplicate");
    TB_CUDA(ctx, out->d_str.alloc(nsel));
    if (nsel > 0)
        TB_CUDA(ctx, cudaMemcpyAsync(out->d_str.p, work.p, nsel * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    // the set is full if it holds every string
    out->full = (nsel == host_binom(norb, nelec));
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    return TBSCI_OK;
}

tbsci_status tables_build(tbsci_ctx *ctx, const tbsci_strings *s, int flags, tbsci_tables *out) {
    TB_CHECK(ctx, (flags & ~3) == 0, TBSCI_EINVAL, "unknown table flags");
    cudaStream_t st = ctx->stream;
    const int64_t l = s->count;
    out->ctx = ctx;
    out->norb = s->norb;
    out->nelec = s->nelec;
    out->flags = flags;
    out->count = l;
    out->full = s->full;
    TB_CUDA(ctx, out->d_str.alloc(l));
    if (l > 0) TB_CUDA(ctx, cudaMemcpyAsync(out->d_str.p, s->d_str.p, l * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    DevBuf<int64_t> counts;
    TB_CUDA(ctx, counts.alloc(std::max<int64_t>(l, 1)));
    TB_CUDA(ctx, out->d_off1.alloc(l + 1));
    LinkArgs A{};
    A.str = out->d_str.p;
    A.l = l;
    A.n = s->norb;
    A.N = s->nelec;
    A.full = s->full ? 1 : 0;
    A.B = ctx->d_binom.p;
    A.counts = counts.p;
    const unsigned grid = (unsigned)((l + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const int threads = kWarpsPerBlock * 32;
    const bool want_double = !(flags & TBSCI_TABLES_SINGLES_ONLY);
    const bool fill = !(flags & TBSCI_TABLES_COUNT_ONLY);
    // singles
    if (l > 0) {
        k_links<false, false><<<grid, threads, 0, st>>>(A);
        TB_CUDA(ctx, cudaGetLastError());
    }
    TB_TRY(scan_exclusive(ctx, counts.p, out->d_off1.p, l, st));
    out->h_off1.resize(l + 1);
    TB_CUDA(ctx, cudaMemcpy(out->h_off1.data(), out->d_off1.p, (l + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    out->nsingle = out->h_off1[l];
    if (fill) {
        TB_CUDA(ctx, out->d_ent1.alloc(out->nsingle));
        A.off = out->d_off1.p;
        A.e1 = out->d_ent1.p;
        if (l > 0 && out->nsingle > 0) {
            k_links<false, true><<<grid, threads, 0, st>>>(A);
            TB_CUDA(ctx, cudaGetLastError());
        }
    }
    if (want_double) {
        TB_CUDA(ctx, out->d_off2.alloc(l + 1));
        if (l > 0) {
            k_links<true, false><<<grid, threads, 0, st>>>(A);
            TB_CUDA(ctx, cudaGetLastError());
        }
        TB_TRY(scan_exclusive(ctx, counts.p, out->d_off2.p, l, st));
        out->h_off2.resize(l + 1);
        TB_CUDA(ctx, cudaMemcpy(out->h_off2.data(), out->d_off2.p, (l + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        out->ndouble = out->h_off2[l];
        if (fill) {
            TB_CUDA(ctx, out->d_ent2.alloc(out->ndouble));
            A.off = out->d_off2.p;
            A.e2 = out->d_ent2.p;
            if (l > 0 && out->ndouble > 0) {
                k_links<true, true><<<grid, threads, 0, st>>>(A);
                TB_CUDA(ctx, cudaGetLastError());
            }
        }
    }
    TB_CUDA(ctx, cudaStreamSynchronize(st));
    return TBSCI_OK;
}

}  // namespace tbsci
