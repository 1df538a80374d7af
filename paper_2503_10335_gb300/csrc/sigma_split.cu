// sigma = H.c for spaces whose rows are longer than shared memory (Sec. II.B,
// Eq. 7; the classes of Sec. II.C), as three passes that keep every gather in
// shared memory and every read of a link table or c row inside L2:
//
//  K1 (k_sigma_parts): the diagonal, the same-spin beta singles with the
//     alpha-beta Coulomb term ([0,0], [0,1]) and the alpha singles with their
//     alpha-beta part ([1,0], [1,1]). NC CTAs serve one alpha row Ia; CTA k owns
//     every NC-th slice of 32 columns and keeps their sigma accumulators in
//     shared memory for the whole row. The c row of each alpha term is staged
//     in shared memory one column part at a time, and the beta single links of
//     every column are split by the part their target lies in (PartLayout), so
//     every gather reads shared memory and the sigma row is written once.
//  K2 (k_dbl_spmm on C): the alpha doubles ([2,0]) as a sparse x dense product
//     sigma[Ia, :] += sum_{Ja} h(Ia, Ja) c[Ja, :], in column tiles. CTAs run
//     tile by tile, so the CTAs in flight share one column tile of c in L2 and
//     read each link once per tile.
//  K3 (k_dbl_spmm on C^T): the beta doubles ([0,2]) the same way on the
//     transposed vector, sigma^T[Ib, :] = sum_{Jb} h(Ib, Jb) c^T[Jb, :],
//     then added back transposed.
// Every column is summed in a fixed order: results do not depend on the launch.
#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace tbsci {

namespace {

// A part layout link packs the target's offset in its column part (below 2^19:
// a part fits in shared memory) above the coefficient index 2 pair + sign (below
// 2^13: at most 2,080 pairs for 64 orbitals, plus the zero padding entries).
constexpr int kPartLinkBits = 13;

template <typename T>
struct SplitArgs {
    int64_t la, lb;
    const T *C;
    T *S;  // K1 output: rows in the layout's column order
    int npair, na, norb, P, NC;
    int64_t W;
    const uint64_t *stra;
    const int64_t *a_soff;
    const int2 *a_sci;
    const T *a_sval;
    const T *Ea;
    const T *V;  // [npair][npair]
    const uint64_t *pstr;  // beta string of each column, in the layout's order
    const T *pEb;          // its one-electron energy, same order
    int nbt;               // bytes of a beta string: ceil(norb / 8) lookup tables
    const int32_t *perm, *rowsa;
    T ecore;
    const int64_t *poff;
    const int32_t *pw;
    const uint32_t *pci;  // packed links: part-local target << kPartLinkBits | coefficient index
    const T *pval;
};

// shared memory ahead of the c part: the coefficient table by (pair, sign), the
// occupied pairs of the alpha string, then 256-entry lookup tables, one per byte
// of a beta string (their offset is split_tab_offset)
template <typename T>
__host__ __device__ size_t split_tab_offset(int npair) {
    return ((2 * npair + 2) * sizeof(T) + 64 * sizeof(int) + 15) & ~size_t(15);
}
template <typename T>
__host__ __device__ size_t split_head_bytes(int npair, int norb) {
    return split_tab_offset<T>(npair) + (size_t)((norb + 7) / 8) * 256 * sizeof(T);
}

// GACC: one CTA per alpha row (NC = 1) that accumulates in the output row in
// global memory (column order, coalesced), which frees shared memory for longer
// column parts; otherwise the accumulators of the CTA's slices stay in shared memory.
template <typename T, int kThreads, bool GACC, int MINB = 1>
__global__ void __launch_bounds__(kThreads, MINB) k_sigma_parts(SplitArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int npair = A.npair;
    T *sV2 = reinterpret_cast<T *>(smem_raw);  // [2 npair + 2]: coefficient by (pair, sign); last two zero
    int *sOcc = reinterpret_cast<int *>(sV2 + 2 * npair + 2);
    // sTab[256 b + v]: the column coefficient's share of the orbitals of byte b of
    // a beta string whose byte b is v (see the table build below)
    T *sTab = reinterpret_cast<T *>(smem_raw + split_tab_offset<T>(npair));
    const int nbt = A.nbt;
    T *sC = sTab + 256 * nbt;  // [W]: one part of a c row
    T *sAcc = GACC ? A.S + A.rowsa[blockIdx.x / A.NC] * A.lb  // the row itself, column order
                   : sC + A.W;  // accumulators of this CTA's column slices
    const int NC = A.NC, P = A.P;
    const int64_t Ia = A.rowsa[blockIdx.x / NC];
    const int kk = (int)(blockIdx.x % NC);
    const int64_t lb = A.lb, W = A.W;
    const int64_t nsl = (lb + 31) / 32;
    const int64_t nloc = (nsl - kk + NC - 1) / NC * 32;  // local columns: slices kk, kk + NC, ...
    const T *__restrict__ C = A.C;
    if (threadIdx.x == 0) {
        int k = 0;
        for (uint64_t s = A.stra[Ia]; s; s &= s - 1) {
            const int p = __ffsll((long long)s) - 1;
            sOcc[k++] = p * (p + 1) / 2 + p;
        }
        sV2[2 * npair] = T(0);
        sV2[2 * npair + 1] = T(0);
    }
    // zero the accumulators (in global memory only the row's lb entries exist)
    for (int64_t jl = threadIdx.x; jl < (GACC ? lb : nloc); jl += kThreads) sAcc[jl] = T(0);
    __syncthreads();
    const int na = A.na;
    const T eIa = A.ecore + A.Ea[Ia];
    const int64_t t0 = A.a_soff[Ia], t1 = A.a_soff[Ia + 1];
    // t = t0 - 1: the Ja = Ia term; then the alpha singles of Ia
    for (int64_t t = t0 - 1; t < t1; ++t) {
        const bool self = t < t0;
        int64_t Ja = Ia;
        int pr = 0;
        T sa = T(1), ha = T(0);
        if (!self) {
            const int2 ea = __ldg(A.a_sci + t);
            Ja = ea.x;
            pr = ea.y >> 1;
            sa = (ea.y & 1) ? T(-1) : T(1);
            ha = __ldg(A.a_sval + t);
        }
        const T *__restrict__ Crow = C + Ja * lb;
        for (int p = 0; p < P; ++p) {
            const int64_t base = (int64_t)p * W, len = min(W, lb - base);
            __syncthreads();  // the previous pass is done with sC and sV2
            if (p == 0)
                for (int x = threadIdx.x; x < npair; x += kThreads) {
                    T v;
                    if (self) {  // W_Ia[x] = sum_{q in Ia} (qq|x)
                        v = T(0);
                        for (int k = 0; k < na; ++k) v += A.V[(size_t)sOcc[k] * npair + x];
                    } else {
                        v = sa * A.V[(size_t)pr * npair + x];
                    }
                    sV2[2 * x] = v;
                    sV2[2 * x + 1] = -v;
                }
            // stage the part: 16-byte loads when the part starts on a 16-byte boundary
            // (four loads in flight per thread), else element by element
            const T *src = Crow + base;
            if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                constexpr int E = 16 / sizeof(T);
                const int64_t nv = len / E;
                const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
                uint4 *d4 = reinterpret_cast<uint4 *>(sC);
                int64_t q = threadIdx.x;
                for (; q + 3 * kThreads < nv; q += 4 * kThreads) {
                    const uint4 a = __ldcs(s4 + q), b = __ldcs(s4 + q + kThreads), c2 = __ldcs(s4 + q + 2 * kThreads),
                                d = __ldcs(s4 + q + 3 * kThreads);
                    d4[q] = a;
                    d4[q + kThreads] = b;
                    d4[q + 2 * kThreads] = c2;
                    d4[q + 3 * kThreads] = d;
                }
                for (; q < nv; q += kThreads) d4[q] = __ldcs(s4 + q);
                for (int64_t j = nv * E + threadIdx.x; j < len; j += kThreads) sC[j] = __ldg(src + j);
            } else {
                for (int64_t j = threadIdx.x; j < len; j += kThreads) sC[j] = __ldg(src + j);
            }
            __syncthreads();
            if (p == 0) {
                // The coefficient of a column's own c value is base + sum over the
                // orbitals l of its beta string of sV2[2 ll]: sa (pr|ll) for an
                // alpha single (base h(Ia, Ja)), sum_{q in Ia} (qq|ll) for Ja = Ia
                // (base E_core + E_a(Ia), plus E_b of the column). The sum is read
                // from one 256-entry table per byte of the string.
                const T base0 = self ? eIa : ha;
                for (int e = threadIdx.x; e < 256 * nbt; e += kThreads) {
                    const int b = e >> 8, v = e & 255;
                    T x = b == 0 ? base0 : T(0);
                    for (int i = 0; i < 8; ++i) {
                        const int l = 8 * b + i;
                        if (((v >> i) & 1) && l < A.norb) x += sV2[2 * (l * (l + 1) / 2 + l)];
                    }
                    sTab[e] = x;
                }
                __syncthreads();
            }
            // the column sweep, compiled separately for the Ja = Ia term so that the
            // singles' inner loop carries no per-link test of the term kind
            auto sweep = [&](auto self_tag) {
                constexpr bool SELF = decltype(self_tag)::value;
                for (int64_t jl = threadIdx.x; jl < nloc; jl += kThreads) {
                    const int64_t sl = (jl >> 5) * NC + kk;
                    const int lane = (int)(jl & 31);
                    const int64_t j = sl * 32 + lane;
                    if (j >= lb) continue;
                    const int64_t ib = __ldg(A.perm + j);
                    T acc = sAcc[jl];
                    if ((uint64_t)(ib - base) < (uint64_t)len) {  // the column's own c value is in this part
                        const uint64_t sb = __ldg(A.pstr + j);
                        T coef = sTab[sb & 255];
                        for (int b = 1; b < nbt; ++b) coef += sTab[256 * b + ((sb >> (8 * b)) & 255)];
                        if (SELF) coef += __ldg(A.pEb + j);
                        acc += coef * sC[ib - base];
                    }
                    const int64_t o = __ldg(A.poff + sl * P + p) + lane;
                    const int w = __ldg(A.pw + sl * P + p);
                    const uint32_t *ci = A.pci + o;
                    const T *cv = A.pval + o;
                    constexpr uint32_t kIdx = (1u << kPartLinkBits) - 1;
                    int k = 0;
                    // four links in flight per iteration: their loads overlap. One
                    // accumulator: the FP64 pipe, not the add latency, is the limit,
                    // and a second chain would cost an add per column and part
                    for (; k + 3 < w; k += 4) {
                        const uint32_t e0 = __ldg(ci + 32 * k), e1 = __ldg(ci + 32 * (k + 1));
                        const uint32_t e2 = __ldg(ci + 32 * (k + 2)), e3 = __ldg(ci + 32 * (k + 3));
                        T x0 = sV2[e0 & kIdx], x1 = sV2[e1 & kIdx], x2 = sV2[e2 & kIdx], x3 = sV2[e3 & kIdx];
                        if (SELF) {
                            x0 += __ldg(cv + 32 * k);
                            x1 += __ldg(cv + 32 * (k + 1));
                            x2 += __ldg(cv + 32 * (k + 2));
                            x3 += __ldg(cv + 32 * (k + 3));
                        }
                        acc += x0 * sC[e0 >> kPartLinkBits];
                        acc += x1 * sC[e1 >> kPartLinkBits];
                        acc += x2 * sC[e2 >> kPartLinkBits];
                        acc += x3 * sC[e3 >> kPartLinkBits];
                    }
                    for (; k < w; ++k) {
                        const uint32_t e = __ldg(ci + 32 * k);
                        T x = sV2[e & kIdx];
                        if (SELF) x += __ldg(cv + 32 * k);
                        acc += x * sC[e >> kPartLinkBits];
                    }
                    sAcc[jl] = acc;
                }
            };
            if (self)
                sweep(std::true_type{});
            else
                sweep(std::false_type{});
        }
    }
    if (GACC) return;  // the row was accumulated in place
    __syncthreads();
    T *__restrict__ S = A.S + Ia * lb;  // the row in the layout's column order
    for (int64_t jl = threadIdx.x; jl < nloc; jl += kThreads) {
        const int64_t j = ((jl >> 5) * NC + kk) * 32 + (jl & 31);
        if (j < lb) S[j] = sAcc[jl];
    }
}

constexpr int kDblRows = 16;  // rows of a CTA of the double-class product

// Y[r, cols of tile] (+)= sum_{t in row r} val[t] X[col[t], cols of tile]; X and Y
// are [rows][ld]; CTA b serves column tile b / nrb and rows (b % nrb) * kDblRows..
template <typename T, int TW>
__global__ void __launch_bounds__(TW, 1024 / TW) k_dbl_spmm(const T *__restrict__ X, T *Y, int64_t rows, int64_t ld,
                                                 const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                 const T *__restrict__ val, int64_t nrb, int accumulate) {
    __shared__ int32_t sCol[TW];
    __shared__ T sVal[TW];
    const int64_t b = blockIdx.x;
    const int64_t tile = b / nrb, rb = b - tile * nrb;
    const int64_t c = tile * TW + threadIdx.x;
    const bool ok = c < ld;
    const int64_t r0 = rb * kDblRows, r1 = min(rows, r0 + kDblRows);
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t t0 = off[r], t1 = off[r + 1];
        T acc = (accumulate && ok) ? Y[r * ld + c] : T(0), acc2 = T(0);
        for (int64_t ch = t0; ch < t1; ch += TW) {
            const int n = (int)(t1 - ch < (int64_t)TW ? t1 - ch : (int64_t)TW);
            __syncthreads();
            if (threadIdx.x < n) {
                sCol[threadIdx.x] = __ldg(col + ch + threadIdx.x);
                sVal[threadIdx.x] = __ldg(val + ch + threadIdx.x);
            }
            __syncthreads();
            if (ok) {
                const T *__restrict__ Xc = X + c;
                int k = 0;
                for (; k + 3 < n; k += 4) {
                    const T x0 = __ldg(Xc + (size_t)sCol[k] * ld), x1 = __ldg(Xc + (size_t)sCol[k + 1] * ld);
                    const T x2 = __ldg(Xc + (size_t)sCol[k + 2] * ld), x3 = __ldg(Xc + (size_t)sCol[k + 3] * ld);
                    acc += sVal[k] * x0;
                    acc2 += sVal[k + 1] * x1;
                    acc += sVal[k + 2] * x2;
                    acc2 += sVal[k + 3] * x3;
                }
                for (; k < n; ++k) acc += sVal[k] * __ldg(Xc + (size_t)sCol[k] * ld);
            }
        }
        if (ok) Y[r * ld + c] = acc + acc2;
    }
}

// out[c][r] = in[r][c] (in: rows x cols), 32 x 32 tiles through shared memory
template <typename T>
__global__ void k_transpose(const T *__restrict__ in, T *out, int64_t rows, int64_t cols) {
    __shared__ T tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][i];
    }
}

// y[r][c] = p[r][ip[c]] + z[c][r]: the K1 rows (in a layout's column order, ip its
// inverse) plus the transposed beta-double product (z: cols x rows)
template <typename T>
__global__ void k_combine(T *y, const T *__restrict__ pz, const int32_t *__restrict__ ip, const T *__restrict__ z,
                          int64_t rows, int64_t cols) {
    __shared__ T tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) tile[threadIdx.x][i] = z[c * rows + r];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) y[r * cols + c] = pz[r * cols + __ldg(ip + c)] + tile[i][threadIdx.x];
    }
}

// Part layout of the beta single links for `nparts` column parts (built on the host).
tbsci_status build_parts(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, int nparts, PartLayout **out) {
    for (auto &pl : P->parts)
        if (pl->P == nparts) {
            *out = pl.get();
            return TBSCI_OK;
        }
    const int64_t lb = P->B.l, nsl = (lb + 31) / 32;
    const int64_t W = (lb + nparts - 1) / nparts;
    TB_CHECK(ctx, W < (int64_t(1) << (32 - kPartLinkBits)) && 2 * ham->npair + 2 <= (1 << kPartLinkBits),
             TBSCI_EINVAL, "split sigma: column part or pair count too large for the packed link layout");
    const int64_t ns = P->B.h_soff.empty() ? 0 : P->B.h_soff[lb];
    std::vector<int2> sci(ns);
    std::vector<double> sval(ns);
    if (ns) {
        TB_CUDA(ctx, cudaMemcpy(sci.data(), P->B.d_sci.p, ns * sizeof(int2), cudaMemcpyDeviceToHost));
        TB_CUDA(ctx, cudaMemcpy(sval.data(), P->B.d_sval.p, ns * sizeof(double), cudaMemcpyDeviceToHost));
    }
    const std::vector<int64_t> &off = P->B.h_soff;
    // links per column and part; columns ordered by count in part 0, then 1, ... (descending)
    std::vector<int32_t> cp((size_t)lb * nparts, 0);
    for (int64_t ib = 0; ib < lb; ++ib)
        for (int64_t t = off[ib]; t < off[ib + 1]; ++t) ++cp[(size_t)ib * nparts + sci[t].x / W];
    std::vector<int32_t> perm(lb), iperm(lb);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
        for (int p = 0; p < nparts; ++p) {
            const int32_t a = cp[(size_t)x * nparts + p], b = cp[(size_t)y * nparts + p];
            if (a != b) return a > b;
        }
        return false;
    });
    for (int64_t j = 0; j < lb; ++j) iperm[perm[j]] = (int32_t)j;
    std::vector<int64_t> loff((size_t)nsl * nparts);
    std::vector<int32_t> lw((size_t)nsl * nparts);
    int64_t total = 0;
    for (int64_t sl = 0; sl < nsl; ++sl)
        for (int p = 0; p < nparts; ++p) {
            int32_t w = 0;
            for (int64_t j = sl * 32; j < std::min(lb, sl * 32 + 32); ++j)
                w = std::max(w, cp[(size_t)perm[j] * nparts + p]);
            loff[sl * nparts + p] = total;
            lw[sl * nparts + p] = w;
            total += 32 * (int64_t)w;
        }
    const int zero_idx = 2 * ham->npair;
    std::vector<uint32_t> ci(std::max<int64_t>(total, 1));
    std::vector<double> v(std::max<int64_t>(total, 1), 0.0);
    std::vector<float> vf(std::max<int64_t>(total, 1), 0.f);
    std::vector<int32_t> fill(nparts);
    for (int64_t sl = 0; sl < nsl; ++sl)
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t j = sl * 32 + lane;
            std::fill(fill.begin(), fill.end(), 0);
            if (j < lb) {
                const int64_t ib = perm[j];
                for (int64_t t = off[ib]; t < off[ib + 1]; ++t) {
                    const int p = (int)(sci[t].x / W);
                    const int64_t pos = loff[sl * nparts + p] + 32 * (int64_t)fill[p]++ + lane;
                    ci[pos] = ((uint32_t)(sci[t].x - p * W) << kPartLinkBits) | (uint32_t)sci[t].y;
                    v[pos] = sval[t];
                    vf[pos] = (float)sval[t];
                }
            }
            for (int p = 0; p < nparts; ++p)  // padding: the part's first column, zero coefficient
                for (int k = fill[p]; k < lw[sl * nparts + p]; ++k)
                    ci[loff[sl * nparts + p] + 32 * (int64_t)k + lane] = (uint32_t)zero_idx;
        }
    // beta strings and their energies in the layout's column order
    std::vector<uint64_t> hstr(lb), pstr(lb);
    std::vector<double> hE(lb), pE(lb);
    std::vector<float> pEf(lb);
    TB_CUDA(ctx, cudaMemcpy(hstr.data(), P->B.d_str, lb * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    TB_CUDA(ctx, cudaMemcpy(hE.data(), P->B.d_E.p, lb * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < lb; ++j) {
        pstr[j] = hstr[perm[j]];
        pE[j] = hE[perm[j]];
        pEf[j] = (float)pE[j];
    }
    auto pl = std::make_unique<PartLayout>();
    pl->P = nparts;
    pl->W = W;
    const size_t bytes = loff.size() * 12 + ci.size() * (sizeof(uint32_t) + 12) + (size_t)lb * 28;
    TB_TRY(charge(ctx, bytes, "column-part link layout"));
    cudaError_t e = pl->off.alloc(loff.size());
    if (e == cudaSuccess) e = pl->w.alloc(lw.size());
    if (e == cudaSuccess) e = pl->ci.alloc(ci.size());
    if (e == cudaSuccess) e = pl->val.alloc(v.size());
    if (e == cudaSuccess) e = pl->valf.alloc(vf.size());
    if (e == cudaSuccess) e = pl->perm.alloc(lb);
    if (e == cudaSuccess) e = pl->iperm.alloc(lb);
    if (e == cudaSuccess) e = pl->str.alloc(lb);
    if (e == cudaSuccess) e = pl->Eb.alloc(lb);
    if (e == cudaSuccess) e = pl->Ebf.alloc(lb);
    if (e == cudaSuccess && !loff.empty())
        e = cudaMemcpy(pl->off.p, loff.data(), loff.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !lw.empty())
        e = cudaMemcpy(pl->w.p, lw.data(), lw.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->ci.p, ci.data(), ci.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->val.p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->valf.p, vf.data(), vf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->perm.p, perm.data(), lb * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->iperm.p, iperm.data(), lb * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->str.p, pstr.data(), lb * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->Eb.p, pE.data(), lb * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->Ebf.p, pEf.data(), lb * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        uncharge(ctx, bytes);
        return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                    std::string("column-part link layout: ") + cudaGetErrorString(e));
    }
    P->charged += bytes;
    *out = pl.get();
    P->parts.push_back(std::move(pl));
    return TBSCI_OK;
}

template <typename T, int TH, bool GACC, int MINB = 1>
tbsci_status launch_parts_th(tbsci_ctx *ctx, const SplitArgs<T> &A, size_t smem, cudaStream_t st) {
    auto k = k_sigma_parts<T, TH, GACC, MINB>;
    TB_CUDA(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TraceScope tr(ctx, "k_sigma_parts", st);
    k<<<(unsigned)(A.la * A.NC), TH, smem, st>>>(A);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

template <typename T>
constexpr int dbl_tile() { return sizeof(T) == 8 ? 128 : 256; }

template <typename T>
tbsci_status launch_dbl(tbsci_ctx *ctx, const T *X, T *Y, int64_t rows, int64_t ld, const int64_t *off,
                        const int32_t *col, const T *val, bool accumulate, cudaStream_t st,
                        const char *name) {
    if (rows == 0 || ld == 0) return TBSCI_OK;
    constexpr int TW = dbl_tile<T>();
    const int64_t nrb = (rows + kDblRows - 1) / kDblRows, ntiles = (ld + TW - 1) / TW;
    TB_CHECK(ctx, nrb * ntiles <= INT32_MAX, TBSCI_EINVAL, "double-class product: grid too large");
    TraceScope tr(ctx, name, st);
    k_dbl_spmm<T, TW><<<(unsigned)(nrb * ntiles), TW, 0, st>>>(X, Y, rows, ld, off, col, val, nrb, accumulate ? 1 : 0);
    TB_CUDA(ctx, cudaGetLastError());
    return TBSCI_OK;
}

template <typename T>
SplitArgs<T> split_args(const tbsci_ham *ham, const Plan *P, const PartLayout *pl);

template <>
SplitArgs<double> split_args<double>(const tbsci_ham *ham, const Plan *P, const PartLayout *pl) {
    SplitArgs<double> A{};
    A.la = P->A.l;
    A.lb = P->B.l;
    A.npair = P->npair;
    A.na = P->A.nelec;
    A.P = pl->P;
    A.W = pl->W;
    A.stra = P->A.d_str;
    A.a_soff = P->A.d_soff;
    A.a_sci = P->A.d_sci.p;
    A.a_sval = P->A.d_sval.p;
    A.Ea = P->A.d_E.p;
    A.norb = P->norb;
    A.nbt = (P->norb + 7) / 8;
    A.V = ham->d_V.p;
    A.pstr = pl->str.p;
    A.pEb = pl->Eb.p;
    A.perm = pl->perm.p;
    A.rowsa = P->d_rowsa.p;
    A.ecore = ham->ecore;
    A.poff = pl->off.p;
    A.pw = pl->w.p;
    A.pci = pl->ci.p;
    A.pval = pl->val.p;
    return A;
}

template <>
SplitArgs<float> split_args<float>(const tbsci_ham *ham, const Plan *P, const PartLayout *pl) {
    SplitArgs<float> A{};
    A.la = P->A.l;
    A.lb = P->B.l;
    A.npair = P->npair;
    A.na = P->A.nelec;
    A.P = pl->P;
    A.W = pl->W;
    A.stra = P->A.d_str;
    A.a_soff = P->A.d_soff;
    A.a_sci = P->A.d_sci.p;
    A.a_sval = P->A.d_svalf.p;
    A.Ea = P->A.d_Ef.p;
    A.norb = P->norb;
    A.nbt = (P->norb + 7) / 8;
    A.V = ham->d_Vf.p;
    A.pstr = pl->str.p;
    A.pEb = pl->Ebf.p;
    A.perm = pl->perm.p;
    A.rowsa = P->d_rowsa.p;
    A.ecore = (float)ham->ecore;
    A.poff = pl->off.p;
    A.pw = pl->w.p;
    A.pci = pl->ci.p;
    A.pval = pl->valf.p;
    return A;
}

template <typename T>
const T *dval_of(const SpinPlan &sp);
template <>
const double *dval_of<double>(const SpinPlan &sp) { return sp.d_dval.p; }
template <>
const float *dval_of<float>(const SpinPlan &sp) { return sp.d_dvalf.p; }

}  // namespace

int split_min_parts(const tbsci_ctx *ctx, int npair, int norb, int64_t lb, size_t elem, int nc, size_t budget) {
    const size_t head = elem == 8 ? split_head_bytes<double>(npair, norb) : split_head_bytes<float>(npair, norb);
    const int64_t nsl = (lb + 31) / 32;
    const size_t acc = nc == 0 ? 0 : (size_t)((nsl + nc - 1) / nc) * 32 * elem;  // nc 0: accumulators in global memory
    const size_t lim = budget ? std::min(budget, ctx->smem_optin) : ctx->smem_optin;
    if (lim <= head + acc) return 0;
    const int64_t wmax = (int64_t)((lim - head - acc) / elem);
    if (wmax <= 0) return 0;
    return (int)std::max<int64_t>(1, (lb + wmax - 1) / wmax);
}

// mode 0: the whole sigma; 1: K1 alone on the listed alpha rows (a tuning
// sample; its output is scratch); 2: K2, K3 and the combine alone (the part of
// the time that does not depend on the K1 shape; sigma is not meaningful)
template <typename T>
tbsci_status split_launch(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, const T *c, T *s, int nvec, int variant,
                          int threads, const int32_t *rows, int64_t nrows, cudaStream_t st, int mode) {
    const int64_t la = P->A.l, lb = P->B.l;
    if (la == 0 || lb == 0) return TBSCI_OK;
    // variant 0: one CTA per alpha row accumulating in global memory, parts as
    // long as shared memory allows; 3: the same with parts short enough for two
    // CTAs per SM (one stages while the other computes); 1, 2: two or four CTAs
    // per row with their accumulators in shared memory (four when two leave no
    // room for a c part)
    const bool gacc = variant <= 0 || variant == 3;
    const size_t budget = variant == 3 ? ctx->smem_per_sm / 2 - 1024 : 0;
    int nc = gacc ? 1 : (variant == 1 ? 2 : 4), nparts = 0;
    for (; nc <= 4; nc *= 2) {
        nparts = split_min_parts(ctx, P->npair, P->norb, lb, sizeof(T), gacc ? 0 : nc, budget);
        if (nparts >= 1 || gacc) break;
    }
    TB_CHECK(ctx, nparts >= 1 && nc <= 4, TBSCI_EINVAL, "split sigma: no room for a column part in shared memory");
    TB_CHECK(ctx, (la + 31) / 32 <= 65535, TBSCI_EINVAL, "split sigma: too many alpha strings");
    nparts = (int)std::min<int64_t>(lb, nparts);
    PartLayout *pl = nullptr;
    TB_TRY(build_parts(ctx, ham, P, nparts, &pl));
    const size_t need = 2 * (size_t)la * lb * sizeof(T);
    if (P->d_trans.n < need) {
        uncharge(ctx, P->d_trans.bytes());
        P->charged -= std::min(P->charged, P->d_trans.bytes());
        P->d_trans.release();
        TB_TRY(charge(ctx, need, "split sigma scratch"));
        const cudaError_t e = P->d_trans.alloc(need);
        if (e != cudaSuccess) {
            uncharge(ctx, need);
            return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                        std::string("split sigma scratch: ") + cudaGetErrorString(e));
        }
        P->charged += need;
    }
    SplitArgs<T> A = split_args<T>(ham, P, pl);
    A.NC = nc;
    if (rows) {
        A.rowsa = rows;
        A.la = nrows;
    }
    const int64_t nsl = (lb + 31) / 32;
    const size_t smem = split_head_bytes<T>(P->npair, P->norb) + (size_t)pl->W * sizeof(T) +
                        (gacc ? 0 : (size_t)((nsl + nc - 1) / nc) * 32 * sizeof(T));
    T *ct = reinterpret_cast<T *>(P->d_trans.p), *sz = ct + (size_t)la * lb;
    const dim3 tb(32, 8), tgrid((unsigned)((lb + 31) / 32), (unsigned)((la + 31) / 32));
    for (int v = 0; v < nvec; ++v) {
        const T *cv = c + (size_t)v * la * lb;
        T *sv = s + (size_t)v * la * lb;
        if (mode != 1) {
            // [0,2]: sz = H_beta,doubles c^T (c^T in ct)
            {
                TraceScope tr(ctx, "k_transpose", st);
                k_transpose<T><<<tgrid, tb, 0, st>>>(cv, ct, la, lb);
                TB_CUDA(ctx, cudaGetLastError());
            }
            TB_TRY(launch_dbl<T>(ctx, ct, sz, lb, la, P->B.d_doff, P->B.d_dcol.p, dval_of<T>(P->B), false, st,
                                 "k_dbl_spmm_beta"));
        }
        if (mode != 2) {
            // K1 rows in the layout's column order into ct (free once c^T has been used)
            A.C = cv;
            A.S = ct;
            if (variant == 3) {  // two CTAs per SM: 512 threads at most 64 registers each
                TB_TRY((launch_parts_th<T, 512, true, 2>(ctx, A, smem, st)));
            } else if (gacc) {
                if (threads >= 1024) TB_TRY((launch_parts_th<T, 1024, true>(ctx, A, smem, st)));
                else TB_TRY((launch_parts_th<T, 512, true>(ctx, A, smem, st)));
            } else {
                if (threads >= 1024) TB_TRY((launch_parts_th<T, 1024, false>(ctx, A, smem, st)));
                else TB_TRY((launch_parts_th<T, 512, false>(ctx, A, smem, st)));
            }
        }
        if (mode == 1) continue;
        {
            TraceScope tr(ctx, "k_combine", st);
            k_combine<T><<<tgrid, tb, 0, st>>>(sv, ct, pl->iperm.p, sz, la, lb);
            TB_CUDA(ctx, cudaGetLastError());
        }
        // [2,0]: sigma += H_alpha,doubles c
        TB_TRY(launch_dbl<T>(ctx, cv, sv, la, lb, P->A.d_doff, P->A.d_dcol.p, dval_of<T>(P->A), true, st,
                             "k_dbl_spmm_alpha"));
    }
    return TBSCI_OK;
}

tbsci_status rest_products_launch(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, const float *c, float *s, int nvec,
                                  cudaStream_t st) {
    const int64_t la = P->A.l, lb = P->B.l;
    if (la == 0 || lb == 0) return TBSCI_OK;
    TB_CHECK(ctx, (la + 31) / 32 <= 65535 && (lb + 31) / 32 <= 65535, TBSCI_EINVAL,
             "product pass: too many strings");
    if (!P->d_bss_off.p) {  // merged same-spin beta links, built once
        const int64_t ns = P->B.h_soff[lb], nd = P->B.h_doff[lb];
        std::vector<int2> sci(ns);
        std::vector<float> sv(ns), dv(nd);
        std::vector<int32_t> dc(nd);
        if (ns) {
            TB_CUDA(ctx, cudaMemcpy(sci.data(), P->B.d_sci.p, ns * sizeof(int2), cudaMemcpyDeviceToHost));
            TB_CUDA(ctx, cudaMemcpy(sv.data(), P->B.d_svalf.p, ns * sizeof(float), cudaMemcpyDeviceToHost));
        }
        if (nd) {
            TB_CUDA(ctx, cudaMemcpy(dc.data(), P->B.d_dcol.p, nd * sizeof(int32_t), cudaMemcpyDeviceToHost));
            TB_CUDA(ctx, cudaMemcpy(dv.data(), P->B.d_dvalf.p, nd * sizeof(float), cudaMemcpyDeviceToHost));
        }
        std::vector<int64_t> off(lb + 1, 0);
        std::vector<int32_t> col(ns + nd);
        std::vector<float> val(ns + nd);
        int64_t k = 0;
        for (int64_t ib = 0; ib < lb; ++ib) {
            off[ib] = k;
            for (int64_t t = P->B.h_soff[ib]; t < P->B.h_soff[ib + 1]; ++t, ++k) {
                col[k] = sci[t].x;
                val[k] = sv[t];
            }
            for (int64_t t = P->B.h_doff[ib]; t < P->B.h_doff[ib + 1]; ++t, ++k) {
                col[k] = dc[t];
                val[k] = dv[t];
            }
        }
        off[lb] = k;
        const size_t bytes = (lb + 1) * 8 + (size_t)k * 8;
        TB_TRY(charge(ctx, bytes, "same-spin beta link table"));
        cudaError_t e = P->d_bss_off.alloc(lb + 1);
        if (e == cudaSuccess) e = P->d_bss_col.alloc(std::max<int64_t>(k, 1));
        if (e == cudaSuccess) e = P->d_bss_valf.alloc(std::max<int64_t>(k, 1));
        if (e == cudaSuccess) e = cudaMemcpy(P->d_bss_off.p, off.data(), (lb + 1) * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && k) e = cudaMemcpy(P->d_bss_col.p, col.data(), k * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && k) e = cudaMemcpy(P->d_bss_valf.p, val.data(), k * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            P->d_bss_off.release();
            uncharge(ctx, bytes);
            return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                        std::string("same-spin beta link table: ") + cudaGetErrorString(e));
        }
        P->charged += bytes;
    }
    const size_t need = 2 * (size_t)la * lb * sizeof(float);
    if (P->d_trans.n < need) {
        uncharge(ctx, P->d_trans.bytes());
        P->charged -= std::min(P->charged, P->d_trans.bytes());
        P->d_trans.release();
        TB_TRY(charge(ctx, need, "product pass scratch"));
        const cudaError_t e = P->d_trans.alloc(need);
        if (e != cudaSuccess) {
            uncharge(ctx, need);
            return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                        std::string("product pass scratch: ") + cudaGetErrorString(e));
        }
        P->charged += need;
    }
    float *ct = reinterpret_cast<float *>(P->d_trans.p), *sz = ct + (size_t)la * lb;
    const dim3 tb(32, 8), tg_ab((unsigned)((lb + 31) / 32), (unsigned)((la + 31) / 32)),
        tg_ba((unsigned)((la + 31) / 32), (unsigned)((lb + 31) / 32));
    for (int v = 0; v < nvec; ++v) {
        const float *cv = c + (size_t)v * la * lb;
        float *sv = s + (size_t)v * la * lb;
        {
            TraceScope tr(ctx, "k_transpose", st);
            k_transpose<float><<<tg_ab, tb, 0, st>>>(cv, ct, la, lb);
            TB_CUDA(ctx, cudaGetLastError());
        }
        TB_TRY(launch_dbl<float>(ctx, ct, sz, lb, la, P->d_bss_off.p, P->d_bss_col.p, P->d_bss_valf.p, false, st,
                                 "k_dbl_spmm_beta"));
        {
            TraceScope tr(ctx, "k_transpose", st);
            k_transpose<float><<<tg_ba, tb, 0, st>>>(sz, sv, lb, la);  // sigma = (beta classes)^T
            TB_CUDA(ctx, cudaGetLastError());
        }
        TB_TRY(launch_dbl<float>(ctx, cv, sv, la, lb, P->A.d_doff, P->A.d_dcol.p, P->A.d_dvalf.p, true, st,
                                 "k_dbl_spmm_alpha"));
    }
    return TBSCI_OK;
}

template tbsci_status split_launch<double>(tbsci_ctx *, const tbsci_ham *, Plan *, const double *, double *, int, int,
                                           int, const int32_t *, int64_t, cudaStream_t, int);
template tbsci_status split_launch<float>(tbsci_ctx *, const tbsci_ham *, Plan *, const float *, float *, int, int,
                                          int, const int32_t *, int64_t, cudaStream_t, int);

}  // namespace tbsci
