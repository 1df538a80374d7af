// extern "C" entry points of libtbsci (declared in include/tbsci.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

namespace tbsci {

tbsci_status fail(tbsci_ctx *ctx, tbsci_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

tbsci_status charge(tbsci_ctx *ctx, size_t bytes, const char *what) {
    if (!ctx || bytes == 0) return TBSCI_OK;
    size_t cur = ctx->hbm_used.load();
    for (;;) {
        if (ctx->hbm_budget && cur + bytes > ctx->hbm_budget)
            return fail(ctx, TBSCI_ENOMEM,
                        std::string(what) + ": " + std::to_string(bytes) + " device bytes would exceed the context's "
                        "budget (" + std::to_string(cur) + " of " + std::to_string(ctx->hbm_budget) + " in use)");
        if (ctx->hbm_used.compare_exchange_weak(cur, cur + bytes)) return TBSCI_OK;
    }
}

void uncharge(tbsci_ctx *ctx, size_t bytes) {
    if (ctx && bytes) ctx->hbm_used.fetch_sub(std::min(bytes, ctx->hbm_used.load()));
}

constexpr size_t kTraceCap = 1 << 16;  // launches held before the oldest unread ones are dropped

TraceScope::TraceScope(tbsci_ctx *ctx, const char *kernel, cudaStream_t st) : ctx_(ctx), kernel_(kernel), st_(st) {
    if (!ctx || !ctx->trace_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&start_) != cudaSuccess) {
        start_ = nullptr;
        return;
    }
    if (cudaEventRecord(start_, st) != cudaSuccess) {
        cudaEventDestroy(start_);
        start_ = nullptr;
    }
}

TraceScope::~TraceScope() {
    if (!start_) return;
    cudaEvent_t end = nullptr;
    if (cudaEventCreate(&end) != cudaSuccess || cudaEventRecord(end, st_) != cudaSuccess) {
        if (end) cudaEventDestroy(end);
        cudaEventDestroy(start_);
        return;
    }
    std::lock_guard<std::mutex> g(ctx_->trace_mu);
    if (ctx_->trace.size() >= kTraceCap) {
        cudaEventDestroy(ctx_->trace.front().start);
        cudaEventDestroy(ctx_->trace.front().end);
        ctx_->trace.erase(ctx_->trace.begin());
        ++ctx_->trace_dropped;
    }
    ctx_->trace.push_back({kernel_, start_, end});
}

}  // namespace tbsci

using namespace tbsci;

#define TB_GUARD_CTX(ctx)                                    \
    do {                                                     \
        if (!(ctx)) return TBSCI_EINVAL;                     \
        cudaError_t e_ = cudaSetDevice((ctx)->device);       \
        if (e_ != cudaSuccess)                               \
            return fail((ctx), TBSCI_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

extern "C" {

const char *tbsci_status_string(tbsci_status st) {
    switch (st) {
        case TBSCI_OK: return "ok";
        case TBSCI_EINVAL: return "invalid argument";
        case TBSCI_ENOMEM: return "out of memory";
        case TBSCI_ECUDA: return "CUDA error";
        case TBSCI_ENOCONV: return "not converged";
        case TBSCI_EAGAIN: return "try again";
        case TBSCI_ETIMEOUT: return "timed out";
        case TBSCI_EBUSY: return "busy";
    }
    return "unknown status";
}

tbsci_status tbsci_create_ex(const tbsci_options *opts, tbsci_ctx **out) {
    if (!out) return TBSCI_EINVAL;
    *out = nullptr;
    tbsci_options o{};
    if (opts) o = *opts;
    if (o.default_mixed < 0 || o.default_mixed > 3) return TBSCI_EINVAL;
    const int device = o.device;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return TBSCI_EINVAL;
    tbsci_ctx *ctx = new (std::nothrow) tbsci_ctx();
    if (!ctx) return TBSCI_ENOMEM;
    ctx->device = device;
    ctx->hbm_budget = o.hbm_budget;
    ctx->default_mixed = o.default_mixed;
    if (o.tune_cache) ctx->tune_path = o.tune_cache;
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        delete ctx;
        return true;
    };
    if (bad(cudaSetDevice(device))) return TBSCI_ECUDA;
    cudaDeviceProp prop;
    if (bad(cudaGetDeviceProperties(&prop, device))) return TBSCI_ECUDA;
    ctx->num_sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    ctx->smem_per_sm = prop.sharedMemPerMultiprocessor;
    if (bad(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking))) return TBSCI_ECUDA;
    // binomials by Pascal's rule (no intermediate overflow up to C(64, 32))
    std::vector<int64_t> B(65 * 65, 0);
    for (int m = 0; m <= 64; ++m) {
        B[m * 65] = 1;
        for (int k = 1; k <= m; ++k) B[m * 65 + k] = B[(m - 1) * 65 + k - 1] + (k <= m - 1 ? B[(m - 1) * 65 + k] : 0);
    }
    if (bad(ctx->d_binom.alloc(B.size()))) return TBSCI_ENOMEM;
    if (bad(cudaMemcpy(ctx->d_binom.p, B.data(), B.size() * sizeof(int64_t), cudaMemcpyHostToDevice))) return TBSCI_ECUDA;
    if (!ctx->tune_path.empty()) {
        FILE *f = std::fopen(ctx->tune_path.c_str(), "r");
        if (f) {
            std::fclose(f);
            if (tbsci_tune_cache_load(ctx, ctx->tune_path.c_str()) != TBSCI_OK) {
                ctx->tune_path.clear();  // not written back on destroy
                tbsci_destroy(ctx);
                return TBSCI_EINVAL;
            }
        }
    }
    *out = ctx;
    return TBSCI_OK;
}

tbsci_status tbsci_create(int device, tbsci_ctx **out) {
    tbsci_options o{};
    o.device = device;
    return tbsci_create_ex(&o, out);
}

tbsci_status tbsci_hbm_used(const tbsci_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return TBSCI_EINVAL;
    *bytes = ctx->hbm_used.load();
    return TBSCI_OK;
}

void tbsci_destroy(tbsci_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_out) cudaStreamSynchronize(ctx->copy_out);
    if (!ctx->tune_path.empty()) tbsci_tune_cache_save(ctx, ctx->tune_path.c_str());
    for (auto &r : ctx->trace) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.end);
    }
    ctx->trace.clear();
    dense_context_release(ctx);
    ctx->host_c.release();
    ctx->host_s.release();
    ctx->d_binom.release();
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    delete ctx;
}

const char *tbsci_last_error(const tbsci_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tbsci_status tbsci_trace_enable(tbsci_ctx *ctx, int on) {
    if (!ctx) return TBSCI_EINVAL;
    ctx->trace_on.store(on != 0);
    return TBSCI_OK;
}

tbsci_status tbsci_trace_read(tbsci_ctx *ctx, tbsci_trace_entry *out, int64_t cap, int64_t *n, int64_t *dropped) {
    TB_GUARD_CTX(ctx);
    TB_CHECK(ctx, n && cap >= 0 && (out || cap == 0), TBSCI_EINVAL, "tbsci_trace_read: null argument");
    *n = 0;
    std::vector<tbsci_ctx::TraceRec> take;
    {
        std::lock_guard<std::mutex> g(ctx->trace_mu);
        const size_t k = std::min(ctx->trace.size(), (size_t)cap);
        take.assign(ctx->trace.begin(), ctx->trace.begin() + k);
        ctx->trace.erase(ctx->trace.begin(), ctx->trace.begin() + k);
        if (dropped) *dropped = ctx->trace_dropped;
        ctx->trace_dropped = 0;
    }
    tbsci_status st = TBSCI_OK;
    for (size_t i = 0; i < take.size(); ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(take[i].end);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, take[i].start, take[i].end);
        if (e != cudaSuccess && st == TBSCI_OK)
            st = fail(ctx, TBSCI_ECUDA, std::string("tbsci_trace_read: ") + cudaGetErrorString(e));
        out[i].kernel = take[i].kernel;
        out[i].ms = ms;
        cudaEventDestroy(take[i].start);
        cudaEventDestroy(take[i].end);
    }
    *n = (int64_t)take.size();
    return st;
}

tbsci_status tbsci_build_strings(tbsci_ctx *ctx, int norb, int nelec, const uint64_t *selected, int64_t nsel,
                                 tbsci_strings **out) {
    TB_GUARD_CTX(ctx);
    if (!out) return fail(ctx, TBSCI_EINVAL, "out is NULL");
    *out = nullptr;
    tbsci_strings *s = new (std::nothrow) tbsci_strings();
    if (!s) return fail(ctx, TBSCI_ENOMEM, "host allocation failed");
    tbsci_status st = strings_build(ctx, norb, nelec, selected, nsel, s);
    if (st == TBSCI_OK) st = charge(ctx, s->d_str.bytes(), "string set");
    if (st != TBSCI_OK) {
        delete s;
        return st;
    }
    s->charged = s->d_str.bytes();
    *out = s;
    return TBSCI_OK;
}

tbsci_status tbsci_strings_count(const tbsci_strings *s, int64_t *count) {
    if (!s || !count) return TBSCI_EINVAL;
    *count = s->count;
    return TBSCI_OK;
}

tbsci_status tbsci_strings_export(tbsci_ctx *ctx, const tbsci_strings *s, uint64_t *out) {
    TB_GUARD_CTX(ctx);
    if (!s || !out) return fail(ctx, TBSCI_EINVAL, "null argument");
    if (s->count > 0) TB_CUDA(ctx, cudaMemcpy(out, s->d_str.p, s->count * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return TBSCI_OK;
}

void tbsci_strings_destroy(tbsci_strings *s) {
    if (!s) return;
    if (s->ctx) cudaSetDevice(s->ctx->device);
    uncharge(s->ctx, s->charged);
    delete s;
}

tbsci_status tbsci_build_excitation_tables(tbsci_ctx *ctx, const tbsci_strings *s, int flags, tbsci_tables **out) {
    TB_GUARD_CTX(ctx);
    if (!s || !out) return fail(ctx, TBSCI_EINVAL, "null argument");
    *out = nullptr;
    tbsci_tables *t = new (std::nothrow) tbsci_tables();
    if (!t) return fail(ctx, TBSCI_ENOMEM, "host allocation failed");
    t->id = ctx->next_id++;
    tbsci_status st = tables_build(ctx, s, flags, t);
    const size_t bytes = t->d_str.bytes() + t->d_off1.bytes() + t->d_off2.bytes() + t->d_ent1.bytes() +
                         t->d_ent2.bytes();
    if (st == TBSCI_OK) st = charge(ctx, bytes, "excitation tables");
    if (st != TBSCI_OK) {
        delete t;
        return st;
    }
    t->charged = bytes;
    *out = t;
    return TBSCI_OK;
}

tbsci_status tbsci_tables_counts(const tbsci_tables *t, int64_t *nsingle, int64_t *ndouble) {
    if (!t) return TBSCI_EINVAL;
    if (nsingle) *nsingle = t->nsingle;
    if (ndouble) *ndouble = t->ndouble;
    return TBSCI_OK;
}

tbsci_status tbsci_tables_export(tbsci_ctx *ctx, const tbsci_tables *t, int64_t *off1, tbsci_single_link *ent1,
                                 int64_t *off2, tbsci_double_link *ent2) {
    TB_GUARD_CTX(ctx);
    if (!t) return fail(ctx, TBSCI_EINVAL, "null tables");
    const bool stored = !(t->flags & TBSCI_TABLES_COUNT_ONLY);
    const bool doubles = !(t->flags & TBSCI_TABLES_SINGLES_ONLY);
    if (ent1 && !stored) return fail(ctx, TBSCI_EINVAL, "tables hold no single-link entries");
    if (off2 && !doubles) return fail(ctx, TBSCI_EINVAL, "tables hold no double links");
    if (ent2 && !(stored && doubles)) return fail(ctx, TBSCI_EINVAL, "tables hold no double-link entries");
    if (off1) std::memcpy(off1, t->h_off1.data(), t->h_off1.size() * sizeof(int64_t));
    if (off2) std::memcpy(off2, t->h_off2.data(), t->h_off2.size() * sizeof(int64_t));
    if (ent1 && t->nsingle > 0)
        TB_CUDA(ctx, cudaMemcpy(ent1, t->d_ent1.p, t->nsingle * sizeof(tbsci_single_link), cudaMemcpyDeviceToHost));
    if (ent2 && t->ndouble > 0)
        TB_CUDA(ctx, cudaMemcpy(ent2, t->d_ent2.p, t->ndouble * sizeof(tbsci_double_link), cudaMemcpyDeviceToHost));
    return TBSCI_OK;
}

void tbsci_tables_destroy(tbsci_tables *t) {
    if (!t) return;
    if (t->ctx) cudaSetDevice(t->ctx->device);
    uncharge(t->ctx, t->charged);
    delete t;
}

tbsci_status tbsci_hamiltonian_create(tbsci_ctx *ctx, int norb, const double *h, const double *eri, double ecore,
                                      tbsci_ham **out) {
    TB_GUARD_CTX(ctx);
    if (!out || !h || !eri) return fail(ctx, TBSCI_EINVAL, "null argument");
    *out = nullptr;
    if (norb < 1 || norb > 64) return fail(ctx, TBSCI_EINVAL, "norb must be in 1..64");
    const int n = norb;
    const size_t n2 = (size_t)n * n, n4 = n2 * n2;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (!std::isfinite(h[i * n + j])) return fail(ctx, TBSCI_EINVAL, "h has a non-finite entry");
            if (std::fabs(h[i * n + j] - h[j * n + i]) > 1e-12) return fail(ctx, TBSCI_EINVAL, "h is not symmetric");
        }
    auto E = [&](int i, int j, int k, int l) { return eri[(((size_t)i * n + j) * n + k) * n + l]; };
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l < n; ++l) {
                    double v = E(i, j, k, l);
                    if (!std::isfinite(v)) return fail(ctx, TBSCI_EINVAL, "eri has a non-finite entry");
                    if (std::fabs(v - E(j, i, k, l)) > 1e-12 || std::fabs(v - E(i, j, l, k)) > 1e-12 ||
                        std::fabs(v - E(k, l, i, j)) > 1e-12)
                        return fail(ctx, TBSCI_EINVAL, "eri lacks the 8-fold symmetry of real orbitals");
                }
    tbsci_ham *H = new (std::nothrow) tbsci_ham();
    if (!H) return fail(ctx, TBSCI_ENOMEM, "host allocation failed");
    H->ctx = ctx;
    H->norb = n;
    H->npair = n * (n + 1) / 2;
    H->ecore = ecore;
    H->h_h.assign(h, h + n2);
    H->h_eri.assign(eri, eri + n4);
    const int P = H->npair;
    std::vector<double> V((size_t)P * P);
    std::vector<float> Vf((size_t)P * P);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q <= p; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s <= r; ++s) {
                    size_t idx = (size_t)pair_index(p, q) * P + pair_index(r, s);
                    V[idx] = E(p, q, r, s);
                    Vf[idx] = (float)V[idx];
                }
    auto cleanup = [&](tbsci_status st, const char *msg) {
        delete H;
        return fail(ctx, st, msg);
    };
    if (H->d_h.alloc(n2) != cudaSuccess || H->d_V.alloc(V.size()) != cudaSuccess ||
        H->d_Vf.alloc(Vf.size()) != cudaSuccess || H->d_eri.alloc(n4) != cudaSuccess)
        return cleanup(TBSCI_ENOMEM, "device allocation failed");
    if (cudaMemcpy(H->d_h.p, h, n2 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_V.p, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_Vf.p, Vf.data(), Vf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(H->d_eri.p, eri, n4 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(TBSCI_ECUDA, "copy of integrals failed");
    *out = H;
    return TBSCI_OK;
}

void tbsci_hamiltonian_destroy(tbsci_ham *ham) {
    if (!ham) return;
    if (ham->ctx) cudaSetDevice(ham->ctx->device);
    for (auto &p : ham->plans) uncharge(ham->ctx, p->charged);
    delete ham;
}

tbsci_status tbsci_prepare(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b) {
    TB_GUARD_CTX(ctx);
    Plan *p = nullptr;
    return plan_get(ctx, ham, a, b, &p);
}

tbsci_status tbsci_sigma(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b, const void *c,
                         void *sigma, int nvec, tbsci_dtype dtype, tbsci_stream stream) {
    TB_GUARD_CTX(ctx);
    if (nvec < 1) return fail(ctx, TBSCI_EINVAL, "nvec must be >= 1");
    Plan *p = nullptr;
    TB_TRY(plan_get(ctx, ham, a, b, &p));
    if (p->A.l * p->B.l == 0) return TBSCI_OK;  // empty space: nothing to read or write
    if (!c || !sigma) return fail(ctx, TBSCI_EINVAL, "null vector pointer");
    if (c == sigma) return fail(ctx, TBSCI_EINVAL, "c and sigma must not overlap");
    return sigma_launch(ctx, ham, p, c, sigma, nvec, dtype, (cudaStream_t)stream);
}

tbsci_status tbsci_sigma_autotune(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                  const void *c, void *sigma, int nvec, tbsci_dtype dtype, tbsci_stream stream,
                                  double *best_ms) {
    TB_GUARD_CTX(ctx);
    if (nvec < 1) return fail(ctx, TBSCI_EINVAL, "nvec must be >= 1");
    Plan *p = nullptr;
    TB_TRY(plan_get(ctx, ham, a, b, &p));
    if (p->A.l * p->B.l == 0) return TBSCI_OK;
    if (!c || !sigma || c == sigma) return fail(ctx, TBSCI_EINVAL, "bad vector pointers");
    TB_TRY(sigma_autotune(ctx, ham, p, c, sigma, nvec, dtype, (cudaStream_t)stream, best_ms));
    tune_cache_record(ctx, p, p->A.l, p->B.l);
    return TBSCI_OK;
}

// Tune cache file: a header line "tbsci-tune 1", then one line per space shape:
// norb l_alpha l_beta  f64_threads f64_nv f64_stage  f32_threads f32_nv f32_stage
// rest_mode rest_threads  (nv or threads 0 = not tuned).
tbsci_status tbsci_tune_cache_save(tbsci_ctx *ctx, const char *path) {
    TB_GUARD_CTX(ctx);
    if (!path) return fail(ctx, TBSCI_EINVAL, "null path");
    std::string text = "tbsci-tune 1\n";
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        char line[256];
        for (const auto &kv : ctx->tune_cache) {
            const auto &e = kv.second;
            std::snprintf(line, sizeof line, "%lld %lld %lld %d %d %d %d %d %d %d %d\n", (long long)kv.first[0],
                          (long long)kv.first[1], (long long)kv.first[2], e.threads[0], e.nv[0], e.stage[0],
                          e.threads[1], e.nv[1], e.stage[1], e.rest_mode, e.rest_threads);
            text += line;
        }
    }
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(ctx, TBSCI_EINVAL, std::string("tune cache: cannot write ") + path);
    const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return fail(ctx, TBSCI_EINVAL, std::string("tune cache: write failed: ") + path);
    return TBSCI_OK;
}

tbsci_status tbsci_tune_cache_load(tbsci_ctx *ctx, const char *path) {
    TB_GUARD_CTX(ctx);
    if (!path) return fail(ctx, TBSCI_EINVAL, "null path");
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(ctx, TBSCI_EINVAL, std::string("tune cache: cannot read ") + path);
    std::map<std::array<int64_t, 3>, tbsci_ctx::TuneEntry> got;
    char buf[512];
    int lineno = 0;
    std::string bad;
    auto threads_ok = [](int t) { return t == 0 || t == 128 || t == 256 || t == 512 || t == 1024; };
    while (std::fgets(buf, sizeof buf, f)) {
        ++lineno;
        if (lineno == 1) {
            if (std::strncmp(buf, "tbsci-tune 1", 12) != 0) bad = "missing header";
            if (!bad.empty()) break;
            continue;
        }
        long long k0, k1, k2;
        tbsci_ctx::TuneEntry e;
        const int n = std::sscanf(buf, "%lld %lld %lld %d %d %d %d %d %d %d %d", &k0, &k1, &k2, &e.threads[0],
                                  &e.nv[0], &e.stage[0], &e.threads[1], &e.nv[1], &e.stage[1], &e.rest_mode,
                                  &e.rest_threads);
        bool ok = n == 11 && k0 >= 1 && k0 <= 64 && k1 >= 0 && k2 >= 0 && threads_ok(e.rest_threads) &&
                  e.rest_mode >= 0 && e.rest_mode <= 5;
        for (int i = 0; i < 2 && ok; ++i)
            ok = threads_ok(e.threads[i]) && e.nv[i] >= 0 && e.nv[i] <= 4 && e.stage[i] >= 0 && e.stage[i] <= 6 &&
                 (e.stage[i] < 3 ? e.threads[i] != 1024 : (e.threads[i] == 0 || e.threads[i] >= 512));
        if (!ok) {
            bad = "malformed line " + std::to_string(lineno);
            break;
        }
        got[{k0, k1, k2}] = e;
    }
    std::fclose(f);
    if (lineno == 0) bad = "empty file";
    if (!bad.empty()) return fail(ctx, TBSCI_EINVAL, std::string("tune cache ") + path + ": " + bad);
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    for (const auto &kv : got) ctx->tune_cache[kv.first] = kv.second;
    return TBSCI_OK;
}

tbsci_status tbsci_tune_cache_size(tbsci_ctx *ctx, int64_t *entries) {
    TB_GUARD_CTX(ctx);
    if (!entries) return fail(ctx, TBSCI_EINVAL, "null out");
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    *entries = (int64_t)ctx->tune_cache.size();
    return TBSCI_OK;
}

tbsci_status tbsci_sigma_host(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                              const double *c, double *sigma, int nvec) {
    TB_GUARD_CTX(ctx);
    if (nvec < 1) return fail(ctx, TBSCI_EINVAL, "nvec must be >= 1");
    Plan *p = nullptr;
    TB_TRY(plan_get(ctx, ham, a, b, &p));
    const size_t n = (size_t)nvec * p->A.l * p->B.l;
    if (n == 0) return TBSCI_OK;
    if (!c || !sigma) return fail(ctx, TBSCI_EINVAL, "null vector pointer");
    if (ctx->host_c.n < n || ctx->host_s.n < n) {
        // both buffers are re-made together; a failure leaves them empty
        uncharge(ctx, ctx->host_c.bytes() + ctx->host_s.bytes());
        ctx->host_c.release();
        ctx->host_s.release();
        TB_TRY(charge(ctx, 2 * n * sizeof(double), "tbsci_sigma_host buffers"));
        cudaError_t e = ctx->host_c.alloc(n);
        if (e == cudaSuccess) e = ctx->host_s.alloc(n);
        if (e != cudaSuccess) {
            ctx->host_c.release();
            uncharge(ctx, 2 * n * sizeof(double));
            return fail(ctx, e == cudaErrorMemoryAllocation ? TBSCI_ENOMEM : TBSCI_ECUDA,
                        std::string("tbsci_sigma_host buffers: ") + cudaGetErrorString(e));
        }
    }
    if (!ctx->copy_in) TB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
    if (!ctx->copy_out) TB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
    // Vectors go through in the launch groups of the (tuned) kernel: group i is
    // evaluated while group i+1 is copied in and group i-1 copied out, on two copy
    // streams ordered by events. Vectors are independent and every launch shape
    // sums a column in the same order, so the result equals one launch over all.
    const int64_t N = p->A.l * p->B.l;
    const int g = p->tune_nv[0] > 0 ? p->tune_nv[0] : std::min(nvec, 4);
    const int ngroups = (nvec + g - 1) / g;
    std::vector<cudaEvent_t> evs((size_t)2 * ngroups, nullptr);
    auto cleanup = [&] {
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
    };
    tbsci_status ret = TBSCI_OK;
    cudaError_t ce = cudaSuccess;
    for (size_t i = 0; i < evs.size() && ce == cudaSuccess; ++i)
        ce = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
    cudaStream_t st = ctx->stream;
    for (int gi = 0; gi < ngroups && ce == cudaSuccess && ret == TBSCI_OK; ++gi) {
        const int v0 = gi * g, k = std::min(g, nvec - v0);
        const size_t off = (size_t)v0 * N, cnt = (size_t)k * N;
        ce = cudaMemcpyAsync(ctx->host_c.p + off, c + off, cnt * sizeof(double), cudaMemcpyHostToDevice,
                             ctx->copy_in);
        if (ce == cudaSuccess) ce = cudaEventRecord(evs[2 * gi], ctx->copy_in);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, evs[2 * gi], 0);
        if (ce != cudaSuccess) break;
        ret = sigma_launch(ctx, ham, p, ctx->host_c.p + off, ctx->host_s.p + off, k, TBSCI_F64, st);
        if (ret != TBSCI_OK) break;
        ce = cudaEventRecord(evs[2 * gi + 1], st);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->copy_out, evs[2 * gi + 1], 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sigma + off, ctx->host_s.p + off, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->copy_out);
    }
    // drain every stream this call used before its events are destroyed
    const cudaError_t s1 = cudaStreamSynchronize(ctx->copy_in), s2 = cudaStreamSynchronize(st),
                      s3 = cudaStreamSynchronize(ctx->copy_out);
    cleanup();
    if (ret != TBSCI_OK) return ret;
    for (cudaError_t e : {ce, s1, s2, s3})
        if (e != cudaSuccess) return fail(ctx, TBSCI_ECUDA, std::string("tbsci_sigma_host: ") + cudaGetErrorString(e));
    return TBSCI_OK;
}

tbsci_status tbsci_diagonal(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b, double *diag,
                            tbsci_stream stream) {
    TB_GUARD_CTX(ctx);
    Plan *p = nullptr;
    TB_TRY(plan_get(ctx, ham, a, b, &p));
    if (p->A.l * p->B.l == 0) return TBSCI_OK;
    if (!diag) return fail(ctx, TBSCI_EINVAL, "null diag pointer");
    return diagonal_launch(ctx, ham, p, diag, (cudaStream_t)stream);
}

tbsci_status tbsci_sigma_counts_get(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                    tbsci_sigma_counts *out) {
    TB_GUARD_CTX(ctx);
    if (!out) return fail(ctx, TBSCI_EINVAL, "null out");
    Plan *p = nullptr;
    TB_TRY(plan_get(ctx, ham, a, b, &p));
    *out = p->counts;
    for (int i = 0; i < 2; ++i) {
        out->tuned_threads[i] = p->tune_threads[i];
        out->tuned_nv[i] = p->tune_nv[i];
        out->tuned_stage[i] = p->tune_stage[i];
    }
    out->tuned_rest[0] = p->tune_rest_mode;
    out->tuned_rest[1] = p->tune_rest_threads;
    return TBSCI_OK;
}

tbsci_status tbsci_davidson(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b, int nroots,
                            const tbsci_davidson_opts *opts, double *energies, double *vecs,
                            tbsci_davidson_info *info) {
    TB_GUARD_CTX(ctx);
    if (!energies) return fail(ctx, TBSCI_EINVAL, "null energies");
    Plan *p = nullptr;
    TB_TRY(plan_get(ctx, ham, a, b, &p));
    tbsci_davidson_opts o{};
    if (opts) o = *opts;
    else o.mixed = ctx->default_mixed;
    const size_t bytes = engine_device_bytes(p->A.l * p->B.l, nroots, &o);
    TB_TRY(charge(ctx, bytes, "Davidson vectors"));
    tbsci_status st = davidson_run(ctx, ham, p, nroots, &o, energies, vecs, info);
    uncharge(ctx, bytes);
    return st;
}

tbsci_status tbsci_overlap(tbsci_ctx *ctx, const double *A, int ma, const double *B, int mb, int64_t n, double *S,
                           tbsci_stream stream) {
    TB_GUARD_CTX(ctx);
    return overlap_run(ctx, A, ma, B, mb, n, S, (cudaStream_t)stream);
}

}  // extern "C"
