// Internal declarations shared by the CUDA translation units of libtbsci.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tbsci.h"

namespace tbsci {

// ------------------------------------------------------------ error plumbing

// Records `msg` in the context and returns `st`.
tbsci_status fail(tbsci_ctx *ctx, tbsci_status st, const std::string &msg);

// Context budget (tbsci_options.hbm_budget): charge() counts `bytes` of new
// device memory against it (ENOMEM, nothing counted, when it would be exceeded),
// uncharge() gives them back when the object is freed.
tbsci_status charge(tbsci_ctx *ctx, size_t bytes, const char *what);
void uncharge(tbsci_ctx *ctx, size_t bytes);

// A failed device allocation returns ENOMEM (the context stays usable); any
// other CUDA error returns ECUDA.
#define TB_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::tbsci::fail((ctx), e_ == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA, \
                                 std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

#define TB_CHECK(ctx, cond, st, msg)                                                         \
    do {                                                                                     \
        if (!(cond)) return ::tbsci::fail((ctx), (st), (msg));                               \
    } while (0)

#define TB_TRY(expr)                                                                         \
    do {                                                                                     \
        tbsci_status s_ = (expr);                                                            \
        if (s_ != TBSCI_OK) return s_;                                                       \
    } while (0)

// Device buffer owned by one object; freed in the destructor.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    // n is set only once the allocation succeeded: a failed alloc leaves an
    // empty buffer (p == nullptr, n == 0), so a later size check re-allocates
    cudaError_t alloc(size_t count) {
        release();
        if (count == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
    size_t bytes() const { return n * sizeof(T); }
};

}  // namespace tbsci

// ------------------------------------------------------------- public objects

struct tbsci_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;  // shared memory of one SM (all resident CTAs)
    // tbsci_options: device-memory budget of the context's objects (0 = none),
    // bytes they hold now, Davidson mode when no options are given, tune-cache file
    size_t hbm_budget = 0;
    std::atomic<size_t> hbm_used{0};
    int default_mixed = 0;
    std::string tune_path;
    cudaStream_t stream = nullptr;
    std::string err;
    uint64_t next_id = 1;
    // device buffers and copy streams of tbsci_sigma_host (streams created on first use)
    tbsci::DevBuf<double> host_c, host_s;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    // binomial table C(m, k) for m, k in 0..64, row-major [65][65]
    tbsci::DevBuf<int64_t> d_binom;
    // autotuned launch shapes keyed by (norb, l_alpha, l_beta): filled by
    // tbsci_sigma_autotune and tbsci_tune_cache_load, applied to plans created later
    struct TuneEntry {
        int threads[2] = {0, 0}, nv[2] = {0, 0}, stage[2] = {0, 0};  // F64, F32; nv 0 = not tuned
        int rest_mode = 0, rest_threads = 0;                         // threads 0 = not tuned
    };
    std::mutex tune_mu;
    std::map<std::array<int64_t, 3>, TuneEntry> tune_cache;
    // cuBLAS handle of the dense same-spin products (rest mode 5), made on first use
    void *cublas = nullptr;
    std::mutex cublas_mu;
    // kernel trace (tbsci_trace_enable): while on, each sigma-path launch is
    // bracketed by two events recorded on its own stream; tbsci_trace_read
    // turns them into durations, oldest first
    struct TraceRec {
        const char *kernel;
        cudaEvent_t start, end;
    };
    std::atomic<bool> trace_on{false};
    std::mutex trace_mu;
    std::vector<TraceRec> trace;
    int64_t trace_dropped = 0;
};

struct tbsci_strings {
    tbsci_ctx *ctx = nullptr;
    size_t charged = 0;  // bytes counted against the context's budget
    int norb = 0, nelec = 0;
    int64_t count = 0;
    bool full = false;  // the full C(norb, nelec) space (combinatorial rank applies)
    tbsci::DevBuf<uint64_t> d_str;
};

struct tbsci_tables {
    tbsci_ctx *ctx = nullptr;
    size_t charged = 0;
    uint64_t id = 0;
    int norb = 0, nelec = 0, flags = 0;
    int64_t count = 0;
    bool full = false;
    int64_t nsingle = 0, ndouble = 0;
    tbsci::DevBuf<uint64_t> d_str;
    tbsci::DevBuf<int64_t> d_off1, d_off2;
    tbsci::DevBuf<tbsci_single_link> d_ent1;
    tbsci::DevBuf<tbsci_double_link> d_ent2;
    std::vector<int64_t> h_off1, h_off2;  // host copies of the row offsets
};

namespace tbsci {

// Records the launches made in its scope in the context's kernel trace when
// tracing is on (nothing otherwise, and nothing while `st` is being captured
// into a graph). `kernel` must be a string literal.
class TraceScope {
  public:
    TraceScope(tbsci_ctx *ctx, const char *kernel, cudaStream_t st);
    ~TraceScope();
    TraceScope(const TraceScope &) = delete;
    TraceScope &operator=(const TraceScope &) = delete;

  private:
    tbsci_ctx *ctx_;
    const char *kernel_;
    cudaStream_t st_;
    cudaEvent_t start_ = nullptr;
};

// Per-spin data of one prepared space (values depend on the Hamiltonian).
struct SpinPlan {
    int64_t l = 0;
    int nelec = 0;
    const uint64_t *d_str = nullptr;  // owned by the tables
    const int64_t *d_soff = nullptr, *d_doff = nullptr;
    DevBuf<int2> d_sci;      // singles: {target, 2*pair(p,q) + (sign < 0)}
    DevBuf<double> d_sval;   // singles: signed string-Hamiltonian value
    DevBuf<float> d_svalf;
    DevBuf<int32_t> d_dcol;  // doubles: target
    DevBuf<double> d_dval;   // doubles: signed value (pq|rs) - (ps|rq)
    DevBuf<float> d_dvalf;
    DevBuf<double> d_E;      // string energies
    DevBuf<float> d_Ef;
    std::vector<int64_t> h_soff, h_doff;
};

// Beta single links split by the column part their target lies in (part p =
// columns [p W, (p + 1) W)), for a c row staged in shared memory one part at a
// time. Columns are taken in their own order `perm` (by link count in part 0,
// then part 1, ..., descending) so the 32 columns of a slice have similar counts
// in every part; per slice and part a sliced-ELL block (offset, width) whose
// padding entries point at the part's first column with a zero coefficient.
// U is the beta Coulomb table with its columns in `perm` order.
struct PartLayout {
    int P = 0;
    int64_t W = 0;
    DevBuf<int32_t> perm, iperm;  // column order and its inverse
    DevBuf<int64_t> off;          // [nslices * P]
    DevBuf<int32_t> w;            // [nslices * P]
    // one 32-bit link: (target - part start) << kPartLinkBits | (2 * pair + (sign < 0))
    DevBuf<uint32_t> ci;
    DevBuf<double> val;           // same-spin string-Hamiltonian value
    DevBuf<float> valf;
    DevBuf<uint64_t> str;         // beta string of each column, in perm order
    DevBuf<double> Eb;            // its one-electron energy, same order
    DevBuf<float> Ebf;
};

// Dense off-diagonal same-spin string Hamiltonians (rest mode 5): beta singles
// + doubles and alpha doubles, each zero-padded to a multiple of 32 strings per
// side; split-TF32 planes or BF16.
struct DenseSameSpin {
    DevBuf<float> a_hi, a_lo, b_hi, b_lo;
    DevBuf<__nv_bfloat16> a_bf, b_bf;
    DevBuf<unsigned char> scratch;  // padded split vector and product
};

struct Plan {
    uint64_t ida = 0, idb = 0;
    int norb = 0, npair = 0;
    SpinPlan A, B;
    DevBuf<double> d_U;      // [npair][l_b]: sum_{r in occ(Ib)} (pair|rr)
    DevBuf<float> d_Uf;
    DevBuf<int32_t> d_permb; // beta columns ordered by single-link count (descending)
    DevBuf<int32_t> d_permb2; // beta columns ordered by single + double link count (descending)
    // Beta links in sliced-ELL layout: per slice of 32 consecutive columns of a
    // column order, entry k of lane i at off[slice] + 32 k + i, padded to the
    // slice's longest list with zero-coefficient entries (coalesced warp loads).
    DevBuf<int64_t> d_s1_off, d_s2_off, d_d2_off;
    DevBuf<int32_t> d_s1_w, d_s2_w, d_d2_w;
    DevBuf<int2> d_s1_ci, d_s2_ci;       // singles {target, 2*pair + neg}; s1: permb order, s2: permb2 order
    DevBuf<double> d_s2_val, d_d2_val;   // string-Hamiltonian values (permb2 order)
    DevBuf<float> d_s2_valf, d_d2_valf;
    DevBuf<int32_t> d_d2_col;            // doubles target (permb2 order)
    DevBuf<double> d_U1, d_U2, d_Eb2;    // Coulomb table / beta energies with columns in permb / permb2 order
    DevBuf<float> d_U1f, d_U2f, d_Eb2f;
    DevBuf<int32_t> d_rowsa; // alpha rows ordered by work (descending)
    DevBuf<int32_t> d_pairs; // even l_alpha only: starts 2k of row pairs, heaviest pair first
    // Tensor-core alpha-beta path (norb <= 16): beta single links indexed by
    // (source string Jb, off-diagonal orbital pair r > s): (Ib << 1 | sign<0) or -1,
    // and the map from off-diagonal pair index to the full pair index.
    int npoff = 0;
    DevBuf<int32_t> d_lbp, d_offpair;
    DevBuf<int> d_tc_err;
    // autotuned launch shape per sigma type (index = tbsci_dtype F64 / F32): threads per CTA, vectors per CTA
    int tune_threads[2] = {0, 0}, tune_nv[2] = {0, 0}, tune_stage[2] = {0, 0};
    // autotuned SIMT pass of the tensor-core sigma types (shared-memory mode, threads; 0 = default)
    int tune_rest_mode = 0, tune_rest_threads = 0;
    // split path for rows longer than shared memory: part layouts by part count,
    // and the transposed c / sigma scratch of the beta-double class
    std::vector<std::unique_ptr<PartLayout>> parts;
    DevBuf<unsigned char> d_trans;
    // same-spin beta links (singles, then doubles, per source string) with FP32
    // values: the beta classes of the tensor-core types' product pass
    DevBuf<int64_t> d_bss_off;
    DevBuf<int32_t> d_bss_col;
    DevBuf<float> d_bss_valf;
    DenseSameSpin dense;
    tbsci_sigma_counts counts{};
    size_t charged = 0;  // device bytes counted against the context's budget
};

}  // namespace tbsci

// A pruned TBSCI space (Sec. II.A, Eq. 6): per alpha string w the ascending
// beta indices I_w, CSR off[la + 1] / cols[nd]; compressed vectors [nd].
struct tbsci_pruned {
    tbsci_ctx *ctx = nullptr;
    uint64_t ida = 0, idb = 0;  // the tables of the TPB space it is taken from
    int64_t la = 0, lb = 0, nd = 0;
    tbsci::DevBuf<int64_t> d_off;
    tbsci::DevBuf<int32_t> d_cols;
    tbsci::DevBuf<int32_t> d_rows;  // alpha rows ordered by work (descending)
    std::vector<int64_t> h_off;
    size_t charged = 0;
};

struct tbsci_ham {
    tbsci_ctx *ctx = nullptr;
    int norb = 0, npair = 0;
    double ecore = 0.0;
    tbsci::DevBuf<double> d_h, d_V, d_eri;  // h[n][n], V[npair][npair] = (pq|rs) pair-packed, eri[n^4]
    tbsci::DevBuf<float> d_Vf;
    std::vector<double> h_h, h_eri;
    std::vector<std::unique_ptr<tbsci::Plan>> plans;
};

namespace tbsci {

inline int pair_index(int p, int q) { return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p; }

// strings.cu
tbsci_status strings_build(tbsci_ctx *ctx, int norb, int nelec, const uint64_t *sel, int64_t nsel,
                           tbsci_strings *out);
// tables.cu
tbsci_status tables_build(tbsci_ctx *ctx, const tbsci_strings *s, int flags, tbsci_tables *out);
// plan.cu
tbsci_status plan_get(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                      Plan **out);
// sigma.cu
tbsci_status sigma_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const void *c, void *s,
                          int nvec, tbsci_dtype dt, cudaStream_t st);
// One sigma of a batch: nvec vectors of one prepared space.
struct SigmaJob {
    const tbsci_ham *ham;
    const Plan *plan;
    const void *c;
    void *s;
    int nvec;
};
// Device/pinned staging of batched launches (owned by the caller, reused).
struct BatchScratch {
    DevBuf<unsigned char> d_stage;
    void *h_stage[2] = {nullptr, nullptr};
    size_t h_bytes[2] = {0, 0};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    int flip = 0;
    BatchScratch() = default;
    BatchScratch(const BatchScratch &) = delete;
    BatchScratch &operator=(const BatchScratch &) = delete;
    ~BatchScratch();
};
// All jobs (same dtype) in one launch on `st`; jobs whose rows do not fit the
// staged variant get launches of their own.
tbsci_status sigma_launch_batch(tbsci_ctx *ctx, const SigmaJob *jobs, int njobs, tbsci_dtype dt, cudaStream_t st,
                                BatchScratch *scr);
// FP32 sigma without the diagonal, alpha singles and alpha-beta classes (the
// part the tensor-core kernel does not cover); overwrites s.
// Times every launch shape of the SIMT kernel on (c, s) and keeps the fastest in the plan.
// copy a plan's tuned shape into the context's cache / a cached shape into a new plan
void tune_cache_record(tbsci_ctx *ctx, const Plan *plan, int64_t la, int64_t lb);
void tune_cache_apply(tbsci_ctx *ctx, Plan *plan, int64_t la, int64_t lb);
tbsci_status sigma_autotune(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *plan, const void *c, void *s, int nvec,
                            tbsci_dtype dt, cudaStream_t st, double *best_ms);
tbsci_status sigma_launch_rest(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const float *c, float *s,
                               int nvec, cudaStream_t st, int mode = -1, int threads = 0,
                               const int32_t *rows = nullptr, int64_t nrows = 0, bool bf16 = false);
// sigma_split.cu: sigma for rows longer than shared memory (column parts + the
// same-spin double classes as column-tiled products); see the file head
// smallest number of column parts of a c row that fits in shared memory beside
// the accumulators of 1/nc of a sigma row (0: none fits)
int split_min_parts(const tbsci_ctx *ctx, int npair, int norb, int64_t lb, size_t elem, int nc, size_t budget = 0);
// variant: 0 one CTA per alpha row (global accumulators), 1, 2 two or four CTAs
// per row (shared-memory accumulators), 3 as 0 with parts for two CTAs per SM
template <typename T>
tbsci_status split_launch(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, const T *c, T *s, int nvec, int variant,
                          int threads, const int32_t *rows, int64_t nrows, cudaStream_t st, int mode);
// The classes the tensor-core kernel leaves out (same-spin beta singles and
// doubles, alpha doubles) as column-tiled products: beta on the transposed
// vector, alpha on c; overwrites s (rest mode 4).
tbsci_status rest_products_launch(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, const float *c, float *s, int nvec,
                                  cudaStream_t st);
// sigma_dense.cu: the same classes as dense products on the tensor cores (cuBLAS;
// split TF32, or BF16 when bf16); overwrites s (rest mode 5). The context's
// cuBLAS handle is released by dense_context_release.
tbsci_status rest_dense_launch(tbsci_ctx *ctx, const tbsci_ham *ham, Plan *P, const float *c, float *s, int nvec,
                               bool bf16, cudaStream_t st);
void dense_context_release(tbsci_ctx *ctx);
// sigma_tc.cu: the diagonal, alpha singles and all alpha-beta classes on the
// tensor cores (3xTF32 or BF16 products, FP32 accumulation), added into s.
tbsci_status sigma_tc_add(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const float *c, float *s, int nvec,
                          bool bf16, cudaStream_t st);
tbsci_status diagonal_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, double *diag,
                             cudaStream_t st);

// davidson.cu: resumable Davidson engine (one solve) and its drivers
struct DavEngine;
// pr != NULL: the solve runs on that pruned subspace of the plan's space
tbsci_status engine_create(tbsci_ctx *ctx, tbsci_ham *ham, Plan *plan, int nroots, const tbsci_davidson_opts *o,
                           DavEngine **out, const tbsci_pruned *pr = nullptr);
void engine_destroy(DavEngine *e);
// the context whose error slot and device the engine uses from now on (a
// server builds an engine on its set-up thread and drives it from the scheduler)
void engine_set_ctx(DavEngine *e, tbsci_ctx *ctx);
// The sigma the engine needs next: c/s device pointers ([k][N], dtype dt), on the engine stream.
bool engine_wants_sigma(DavEngine *e, const void **c, void **s, int *k, tbsci_dtype *dt);
// Call once that sigma is enqueued on, or ordered before, the engine stream.
tbsci_status engine_sigma_done(DavEngine *e);
tbsci_status engine_poll(DavEngine *e, bool blocking, bool *progressed);
bool engine_done(const DavEngine *e);
cudaStream_t engine_stream(const DavEngine *e);
tbsci_status engine_results(DavEngine *e, double *energies, double *vecs, tbsci_davidson_info *info);
size_t engine_device_bytes(int64_t N, int nroots, const tbsci_davidson_opts *o);
tbsci_status davidson_run(tbsci_ctx *ctx, tbsci_ham *ham, Plan *plan, int nroots, const tbsci_davidson_opts *o,
                          double *energies, double *vecs, tbsci_davidson_info *info,
                          const tbsci_pruned *pr = nullptr);
// pruned.cu: sigma and diagonal on a pruned space (compressed vectors [nvec][nd])
tbsci_status pruned_sigma_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const tbsci_pruned *pr,
                                 const void *c, void *s, int nvec, tbsci_dtype dt, cudaStream_t st);
tbsci_status pruned_diagonal_launch(tbsci_ctx *ctx, const tbsci_ham *ham, const Plan *plan, const tbsci_pruned *pr,
                                    double *diag, cudaStream_t st);

tbsci_status overlap_run(tbsci_ctx *ctx, const double *A, int ma, const double *B, int mb, int64_t n, double *S,
                         cudaStream_t st);

// Exclusive scan of n int64 counts into out[0..n] (out[n] = total), on stream st.
tbsci_status scan_exclusive(tbsci_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, cudaStream_t st);

}  // namespace tbsci
