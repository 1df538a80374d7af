/*
 * tbsci.h -- C ABI of the GB300 TBSCI library: the Hamiltonian-times-vector
 * product sigma = H.c over a tensor-product bitstring (TPB) determinant space
 * and the Davidson eigensolver that drives it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns a tbsci_status; nothing aborts or exits. On an error
 *    tbsci_last_error() of the context gives a one-line reason.
 *  - Strings are uint64 occupation bitstrings: bit i (LSB = 0) is spatial
 *    orbital i, norb <= 64. A string set is kept in ascending integer order and
 *    a string's index is its 0-based rank in that order.
 *  - A determinant is an alpha string times a beta string (Sec. II.A, Eq. 2-3);
 *    as a spin-orbital determinant it is a+_{alpha occ} a+_{beta occ} |0> with
 *    ascending indices inside each block, so a beta excitation carries only its
 *    own string sign. Determinant index K = w * l_beta + u (beta fastest,
 *    Sec. II.A, Eq. 4-5), so a CI vector is a row-major l_alpha x l_beta matrix.
 *  - Vectors passed to sigma/davidson are DEVICE pointers owned by the caller,
 *    layout [nvec][l_alpha][l_beta], contiguous. Host arrays passed in are copied
 *    before the call returns. Objects the library creates are opaque handles
 *    that own their device memory and are freed by the matching *_destroy.
 *  - Objects belong to the context that made them; one context is used by one
 *    host thread at a time. Calls take a stream where they launch work on a
 *    caller's stream; otherwise they run on the context's own stream and return
 *    when the work is complete.
 */
#ifndef TBSCI_H
#define TBSCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tbsci_status {
    TBSCI_OK = 0,
    TBSCI_EINVAL = 1,   /* invalid argument or input data */
    TBSCI_ENOMEM = 2,   /* device or host allocation failed / over budget */
    TBSCI_ECUDA = 3,    /* a CUDA call failed (message in tbsci_last_error) */
    TBSCI_ENOCONV = 4,  /* Davidson reached max_iter; best estimates returned */
    TBSCI_EAGAIN = 5,   /* serving: queue full / result not ready */
    TBSCI_ETIMEOUT = 6, /* serving: poll timed out */
    TBSCI_EBUSY = 7     /* object in use */
} tbsci_status;

/* Arithmetic of a sigma evaluation. F64 and F32: c, sigma and all arithmetic
 * in that type (SIMT). F32_TC_TF32 / F32_TC_BF16: c and sigma FP32; the
 * alpha-beta classes, alpha singles and the diagonal run on the tensor cores
 * with FP32 accumulation, their products from split TF32 (3 products per term,
 * FP32-level accuracy) or from single BF16 values (about 3 significant digits);
 * the other classes on the FP32 SIMT path. Tensor-core modes need norb <= 16
 * and otherwise fall back to F32. */
typedef enum tbsci_dtype {
    TBSCI_F64 = 0,
    TBSCI_F32 = 1,
    TBSCI_F32_TC_TF32 = 2,
    TBSCI_F32_TC_BF16 = 3
} tbsci_dtype;

/* Same object as cudaStream_t; NULL = the legacy default stream. */
typedef struct CUstream_st *tbsci_stream;

typedef struct tbsci_ctx tbsci_ctx;
typedef struct tbsci_strings tbsci_strings;
typedef struct tbsci_tables tbsci_tables;
typedef struct tbsci_ham tbsci_ham;

/* One single-excitation link of a source string J (8 bytes): the target string
 * I = a+_p a_q |J> of the same set, and sign = <I|a+_p a_q|J>. This is the
 * BETA_SINGLE_LINK entry of Sec. II.C (the paper packs the same fields into
 * 7 bytes, Sec. III.C). */
typedef struct tbsci_single_link {
    int32_t target;
    int8_t sign;
    uint8_t p; /* created orbital */
    uint8_t q; /* annihilated orbital */
    uint8_t pad;
} tbsci_single_link;

/* One double-excitation link (12 bytes, BETA_DOUBLE_LINK of Sec. II.C):
 * I = a+_p a+_r a_s a_q |J>, q < s annihilated, p < r created, sign =
 * <I|a+_p a+_r a_s a_q|J>. */
typedef struct tbsci_double_link {
    int32_t target;
    int8_t sign;
    uint8_t p, r, q, s;
    uint8_t pad[3];
} tbsci_double_link;

/* ------------------------------------------------------------- context */

/* Options of a context (tbsci_create_ex). */
typedef struct tbsci_options {
    int device;             /* CUDA device (made current for the calls of this context) */
    size_t hbm_budget;      /* device bytes the context's objects may hold: string sets,
                               link tables, prepared spaces, Davidson vectors and the
                               buffers of tbsci_sigma_host; a call whose objects would
                               exceed it frees what it made and returns ENOMEM.
                               0 = no limit */
    int default_mixed;      /* mixed mode of tbsci_davidson when its opts is NULL
                               (0..3, as tbsci_davidson_opts.mixed) */
    const char *tune_cache; /* NULL, or a tune-cache file (tbsci_tune_cache_save format):
                               loaded at creation when it exists, written back by
                               tbsci_destroy; the path is copied */
} tbsci_options;

/* Creates a context from options (NULL = device 0, no budget, FP64 Davidson, no
 * tune-cache file). Errors: EINVAL (bad device, default_mixed outside 0..3, an
 * existing tune-cache file that does not parse), ENOMEM, ECUDA. The paper has no
 * counterpart: the settings of one GPU process. */
tbsci_status tbsci_create_ex(const tbsci_options *opts, tbsci_ctx **out);
/* tbsci_create_ex with only the device set. Errors: EINVAL (bad device), ECUDA. */
tbsci_status tbsci_create(int device, tbsci_ctx **out);
/* Device bytes the context's live objects hold against its budget. */
tbsci_status tbsci_hbm_used(const tbsci_ctx *ctx, size_t *bytes);
void tbsci_destroy(tbsci_ctx *ctx);
/* Last error message of this context ("" when none). Valid until the next call. */
const char *tbsci_last_error(const tbsci_ctx *ctx);
const char *tbsci_status_string(tbsci_status st);

/* Kernel trace: the device time of each launch of the sigma path (the fused
 * row kernel, the split path's row kernel, double-class products, transposes
 * and combine, the tensor-core kernel and its SIMT pass, the dense same-spin
 * products of rest mode 5 (one entry for the cuBLAS calls of a vector, plus
 * the split and unpad passes), the pruned kernel).
 * While tracing is on, every such launch made through this context is
 * bracketed by two CUDA events recorded on its own stream (launches made while
 * that stream is being captured into a graph are not traced). The trace keeps
 * the last 65,536 launches. tbsci_trace_enable: on != 0 starts, 0 stops
 * (entries already recorded stay until read). */
tbsci_status tbsci_trace_enable(tbsci_ctx *ctx, int on);
typedef struct tbsci_trace_entry {
    const char *kernel; /* static name of the kernel, valid for the library's lifetime */
    double ms;          /* device time between the events around the launch */
} tbsci_trace_entry;
/* Moves up to `cap` of the oldest entries into the HOST array out[cap] (waiting
 * for their end events) and sets *n to their number; *dropped (may be NULL)
 * receives the entries lost to the cap since the last read. Errors: EINVAL
 * (null n, negative cap, null out with cap > 0), ECUDA (an event failed; the
 * entries are still removed). */
tbsci_status tbsci_trace_read(tbsci_ctx *ctx, tbsci_trace_entry *out, int64_t cap, int64_t *n, int64_t *dropped);

/* --------------------------------------------------------------- strings */

/* Builds a string set (Sec. II.A, Eq. 3: the sets {S^alpha}, {S^beta}).
 * selected == NULL: all C(norb, nelec) strings (full string space; nsel is
 * ignored). Otherwise `selected` is a HOST array of nsel strings in any order;
 * the set is sorted ascending on the device.
 * Errors: EINVAL when norb is outside 1..64, nelec outside 0..norb, a selected
 * string has the wrong electron count, a bit at or above norb, or appears
 * twice, or the set would exceed 2^31 - 1 strings; ENOMEM; ECUDA. */
tbsci_status tbsci_build_strings(tbsci_ctx *ctx, int norb, int nelec, const uint64_t *selected,
                                 int64_t nsel, tbsci_strings **out);
tbsci_status tbsci_strings_count(const tbsci_strings *s, int64_t *count);
/* Copies the sorted set into host memory `out` (count entries). */
tbsci_status tbsci_strings_export(tbsci_ctx *ctx, const tbsci_strings *s, uint64_t *out);
void tbsci_strings_destroy(tbsci_strings *s);

/* ---------------------------------------------------------- link tables */

#define TBSCI_TABLES_SINGLES_ONLY 1 /* build no double links */
#define TBSCI_TABLES_COUNT_ONLY 2   /* count links, store no entries */

/* Builds the single and double excitation links of every string of the set
 * within the set (BETA_SINGLE_LINK / BETA_DOUBLE_LINK, Sec. II.C; the paper
 * builds them for beta, this library for both spins). Rows are CSR by source
 * string; inside a row singles are ordered by (q, p) and doubles by
 * (q, s, p, r), ascending. The target index comes from the combinatorial rank
 * (full string space) or a binary search (selected set). Sign from masked
 * popcounts. The tables keep their own copy of the strings.
 * Errors: EINVAL (flags), ENOMEM, ECUDA. */
tbsci_status tbsci_build_excitation_tables(tbsci_ctx *ctx, const tbsci_strings *s, int flags,
                                           tbsci_tables **out);
tbsci_status tbsci_tables_counts(const tbsci_tables *t, int64_t *nsingle, int64_t *ndouble);
/* Copies the tables into host arrays: off1[l+1], ent1[nsingle], off2[l+1],
 * ent2[ndouble]; any pointer may be NULL to skip that array. EINVAL when entries
 * are requested from a COUNT_ONLY or SINGLES_ONLY table that has none. */
tbsci_status tbsci_tables_export(tbsci_ctx *ctx, const tbsci_tables *t, int64_t *off1,
                                 tbsci_single_link *ent1, int64_t *off2, tbsci_double_link *ent2);
void tbsci_tables_destroy(tbsci_tables *t);

/* ----------------------------------------------------------- Hamiltonian */

/* Creates a Hamiltonian from HOST integrals (the FCIDUMP content the paper
 * reads, Sec. III.A): h[norb*norb] row-major one-electron integrals and
 * eri[norb^4] two-electron integrals in chemists' notation (ij|kl) at
 * ((i*n + j)*n + k)*n + l, plus the constant ecore. H = ecore +
 * sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps).
 * Errors: EINVAL when norb is outside 1..64, h is not symmetric or eri lacks
 * the 8-fold symmetry of real orbitals (tolerance 1e-12 absolute); ENOMEM; ECUDA. */
tbsci_status tbsci_hamiltonian_create(tbsci_ctx *ctx, int norb, const double *h, const double *eri,
                                      double ecore, tbsci_ham **out);
void tbsci_hamiltonian_destroy(tbsci_ham *ham);

/* Prepares (and caches inside `ham`) the per-space data sigma needs: string
 * Hamiltonian values of every link, per-string energies, the beta Coulomb
 * table and the work schedules. Called implicitly by tbsci_sigma; exposed to
 * keep set-up out of timed regions. `a` and `b` must have double links and
 * the same norb as `ham`. Errors: EINVAL, ENOMEM, ECUDA. */
tbsci_status tbsci_prepare(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b);

/* sigma = H.c over the space a x b (Sec. II.B, Eq. 7, on one device; the six
 * Slater-Condon classes of Sec. II.C, Eq. 8 and Algorithm 1). c and sigma are
 * DEVICE arrays [nvec][l_a][l_b] of `dtype`, must not overlap; sigma is
 * overwritten. Work is enqueued on `stream`; the call returns without waiting.
 * Errors: EINVAL (null pointers, nvec < 1, norb mismatch, tables without
 * double links), ENOMEM, ECUDA. */
tbsci_status tbsci_sigma(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                         const void *c, void *sigma, int nvec, tbsci_dtype dtype, tbsci_stream stream);

/* Autotuner of the SIMT sigma kernel (F64 or F32): times launch shapes (4, 8
 * or 16 warps per CTA x 1..4 vectors per CTA x shared-memory use: c row and
 * sigma row in shared memory, sigma row only, or neither) on the caller's c and
 * sigma, keeps the fastest for this space and type (later tbsci_sigma calls use
 * it) and leaves sigma = H c computed. When one sigma takes 100 ms or more, the
 * shapes are timed on a strided sample of 64 alpha rows per SM (staging and CTA
 * size at one vector per CTA, then the vectors per CTA), else every shape on the
 * whole space. Each column is summed in the same order in every shape, so
 * tuning never changes results. For F32_TC_TF32 / F32_TC_BF16 the tensor-core
 * kernel has one shape; the SIMT pass for the classes it leaves out is tuned
 * (shared-memory mode x CTA size) and the whole sigma is then run once.
 * *best_ms: the chosen shape's time on the whole space (may be NULL).
 * Synchronises `stream`. Errors as tbsci_sigma. */
tbsci_status tbsci_sigma_autotune(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                  const void *c, void *sigma, int nvec, tbsci_dtype dtype, tbsci_stream stream,
                                  double *best_ms);

/* Autotune cache of the context: launch shapes keyed by the space's shape
 * (norb, l_alpha, l_beta). tbsci_sigma_autotune records the shape it chooses
 * (F64 / F32 SIMT shape, or the SIMT pass of the tensor-core types); a space
 * prepared afterwards on this context with the same shape starts with it, so
 * same-shaped spaces (another geometry, another Hamiltonian) need no tuning.
 * save writes the cache as text ("tbsci-tune 1", then one line per shape:
 * norb l_alpha l_beta, threads / vectors per CTA / shared-memory mode for F64
 * and for F32, then mode / threads of the tensor-core types' SIMT pass; 0 = not
 * tuned); load merges such a file into the cache, replacing equal keys, and
 * applies to spaces prepared after it. Errors: EINVAL (null path, unreadable or
 * unwritable file, missing header, a malformed or out-of-range line, with its
 * number in tbsci_last_error; nothing is merged then). Not part of the paper:
 * tile shapes for this GPU. */
tbsci_status tbsci_tune_cache_save(tbsci_ctx *ctx, const char *path);
tbsci_status tbsci_tune_cache_load(tbsci_ctx *ctx, const char *path);
tbsci_status tbsci_tune_cache_size(tbsci_ctx *ctx, int64_t *entries);

/* Same product with HOST vectors (pinned memory lets the copies overlap): copies
 * c in, evaluates in FP64, copies sigma out and returns when done. The vectors go
 * through in the kernel's launch groups, each group's copies overlapping the
 * evaluation of its neighbours (two copy streams of the context); the result is
 * the same as one evaluation of all vectors. Uses device buffers and streams
 * owned by the context, so calls on one context must not overlap. */
tbsci_status tbsci_sigma_host(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a,
                              const tbsci_tables *b, const double *c, double *sigma, int nvec);

/* Diagonal H_KK (the [0,0] class, Sec. II.C) into the DEVICE array diag[l_a*l_b]
 * (FP64), enqueued on `stream`. */
tbsci_status tbsci_diagonal(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                            double *diag, tbsci_stream stream);

/* Work counts of one sigma per vector: nnz = number of non-zero H_IJ of the
 * space (each costs one multiply-add per vector), and the split by class. */
typedef struct tbsci_sigma_counts {
    int64_t ndet;
    int64_t nnz;         /* total non-zeros of H */
    int64_t nnz_aa;      /* alpha singles + doubles (classes [1,0] and [2,0]) */
    int64_t nnz_bb;      /* beta singles + doubles ([0,1], [0,2]) */
    int64_t nnz_ab;      /* alpha-single x beta-single ([1,1]) */
    int64_t bytes_tables;
    int32_t tuned_threads[2]; /* autotuned CTA size for F64 / F32 (0 = not tuned) */
    int32_t tuned_nv[2];      /* autotuned vectors per CTA for F64 / F32 */
    int32_t tuned_stage[2];   /* autotuned shared-memory use for F64 / F32: 0 c row
                                 staged and sigma row accumulated in shared memory
                                 where they fit, 1 sigma row only, 2 neither;
                                 3, 4, 5: the split path for rows longer than shared
                                 memory with 1, 2 or 4 CTAs per alpha row (the row
                                 kernel stages c rows in column parts and keeps its
                                 share of the sigma row in shared memory; the
                                 same-spin double classes run as column-tiled
                                 products) */
    int32_t tuned_rest[2];    /* tensor-core types: autotuned mode and CTA size of
                                 the SIMT pass for the classes the tensor cores
                                 leave out (0, 0 = defaults). Modes: 0 c row and
                                 sigma row in shared memory where they fit, 1 c row
                                 only, 2 neither, 3 two alpha rows per CTA sharing
                                 the beta links (even l_alpha; else as 1), 4 the
                                 column-tiled products of the split path (beta
                                 classes on the transposed vector, alpha doubles on
                                 c), 5 dense products on the tensor cores through
                                 cuBLAS (off-diagonal same-spin Hamiltonians stored
                                 dense, sides padded to multiples of 32: about
                                 8 (l_a^2 + l_b^2) bytes for the TF32 type and
                                 2 (l_a^2 + l_b^2) for BF16, plus 12 or 6 bytes
                                 per determinant of scratch; split-TF32 or BF16
                                 products with the type) */
} tbsci_sigma_counts;
tbsci_status tbsci_sigma_counts_get(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a,
                                    const tbsci_tables *b, tbsci_sigma_counts *out);

/* -------------------------------------------------------------- Davidson */

typedef struct tbsci_davidson_opts {
    int max_subspace;    /* basis size before restart; 0 -> max(8*nroots, nroots+2) */
    int restart_keep;    /* Ritz vectors kept at a restart; 0 -> max(nroots, max_subspace/2) */
    int max_iter;        /* 0 -> 1000 */
    double tol_energy;   /* |theta - theta_prev| per root; 0 -> 1e-9 */
    double tol_residual; /* ||r||_2 per root; 0 -> 1e-5 */
    int mixed;           /* 0: FP64 sigma throughout. 1 (F32), 2 (F32_TC_TF32) or
                            3 (F32_TC_BF16): that low-precision sigma until every
                            residual is below tol_mixed_residual (or the largest
                            has not set a new best 10% below the previous one for
                            30 iterations), then restart from the roots' Ritz
                            vectors with FP64 sigma and converge to the FP64
                            tolerances; everything else in FP64 */
    double tol_mixed_residual; /* residual target of the FP32 phase; 0 -> 5e-5 */
    tbsci_stream stream; /* stream for all work; NULL -> the context's stream */
    int basis_f32;       /* 1 (needs mixed != 0): during the low-precision phase the
                            basis and its sigma images are stored in FP32 and sigma
                            reads and writes them in place; dot products and linear
                            combinations accumulate in FP64, and the Rayleigh matrix
                            is solved against the measured overlap V^T V (Cholesky),
                            so rounding of the stored basis does not bias the Ritz
                            values. The FP32 basis is then released and the FP64
                            refinement restarts from the Ritz vectors, orthonormalised
                            in FP64, on a basis of max_subspace_refine vectors.
                            0: FP64 basis throughout */
    int max_subspace_refine; /* FP64 basis size after an FP32 basis (restart keeps
                            max(nroots, max_subspace_refine / 2));
                            0 -> max(nroots + 1, max_subspace / 2) */
} tbsci_davidson_opts;

typedef struct tbsci_davidson_info {
    int iterations;
    int converged;
    int nsigma;          /* sigma vector evaluations, FP64 + FP32 */
    int nsigma_f32;
    int iterations_f32;
    double residual[8];  /* final ||r|| per root (first 8) */
    double energy_f32[8];/* energies at the end of the FP32 phase (mixed mode) */
    double seconds_total;
    double seconds_sigma;     /* device time of all sigma evaluations (blocking call) */
    double seconds_sigma_f32; /* of which the low-precision phase's */
    int precision;            /* sigma type of the low-precision phase (a tbsci_dtype);
                                 TBSCI_F64 when the solve ran in FP64 throughout */
    double refine_delta[8];   /* mixed mode: final FP64-refined energy minus the energy
                                 at the end of the low-precision phase, per root
                                 (the low-precision phase's energy error); 0 otherwise */
} tbsci_davidson_info;

/* Lowest nroots (1..8) eigenpairs of H on a x b by standard Davidson (Sec. III.A)
 * with restart to the lowest restart_keep Ritz vectors when the basis is full
 * (Sec. III.C); an FP64 basis also keeps the previous iteration's Ritz vectors
 * at a restart (orthonormalised against the kept ones, while a slot is left for
 * a correction). Memory: 2 * max_subspace + restart_keep + 4 * nroots + 1 FP64
 * vectors (+ 2 * nroots FP32 in mixed mode); with basis_f32, 3 * nroots + 1 FP64
 * vectors plus the larger of 2 * max_subspace + restart_keep + nroots FP32
 * vectors and 2 * m_ref + m_ref / 2 + nroots FP64 vectors (m_ref = the
 * refinement basis size). Guess: guess k is the unit vector
 * at the k-th lowest H_KK (ties by K) plus 0.1 (1 + ((j + k) mod 4)) / 4 times
 * the unit vector at the (nroots + j)-th lowest, j < 4, orthonormalised, so
 * every symmetry sector is present. Each iteration: Rayleigh
 * matrix, its eigenpairs, Ritz vectors and residuals, stop when every root has
 * |dE| < tol_energy and ||r|| < tol_residual, else precondition residuals by
 * (theta - H_KK)^-1 (|denominator| clamped at 1e-8), orthonormalise twice
 * against the basis (FP64 Gram-Schmidt) and add. energies: HOST array
 * [nroots]. vecs: DEVICE array [nroots][l_a][l_b] FP64 or NULL.
 * opts == NULL: defaults, with the context's default_mixed mode.
 * Errors: EINVAL, ENOMEM, ECUDA; ENOCONV when max_iter is reached (energies
 * and vecs hold the last estimates). Blocks until done. */
tbsci_status tbsci_davidson(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                            int nroots, const tbsci_davidson_opts *opts, double *energies, double *vecs,
                            tbsci_davidson_info *info);

/* --------------------------------------------------------- pruned spaces */

/* The general TBSCI space D_TBSCI (Sec. II.A, Eq. 6): inside the TPB space of
 * tables a x b, determinant (w, u) is kept when beta index u is in the set I_w
 * of alpha string w (the membership test of Algorithm 1, Sec. II.C). I_w is
 * given as CSR: `off` HOST [l_a + 1] (off[0] = 0, non-decreasing) and `cols`
 * HOST [off[l_a]] with each row's beta indices strictly ascending in
 * 0..l_b-1. Determinant (w, u) has the compressed index off[w] + (position of
 * u in I_w); vectors on a pruned space are DEVICE arrays [nvec][off[l_a]].
 * H on the space is the principal submatrix of H on its determinants. Arrays
 * are copied. Errors: EINVAL (null pointers, a malformed CSR, an index out of
 * range or not ascending), ENOMEM, ECUDA. */
typedef struct tbsci_pruned tbsci_pruned;
tbsci_status tbsci_pruned_create(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b, const int64_t *off,
                                 const int32_t *cols, tbsci_pruned **out);
/* Point-group symmetry blocking (Sec. II.A): the pruned space of the
 * determinants of irrep `target` in an abelian point group (D2h or a subgroup,
 * irrep labels 0..7 multiplying as bitwise XOR). orb_irrep: HOST [norb] labels
 * of the orbitals; a string's irrep is the XOR of its occupied orbitals'
 * labels, and (w, u) is kept when irrep(w) XOR irrep(u) = target. The paper
 * sorts the beta strings by irrep so that each I_w is one interval; here the
 * strings keep ascending order and I_w is the irrep class of beta strings,
 * passed to tbsci_pruned_create. With integrals of that symmetry, H couples no
 * two blocks, so the blocks' spectra together are the spectrum of H.
 * Errors: EINVAL (labels or target outside 0..7), ENOMEM, ECUDA. */
tbsci_status tbsci_pruned_create_symmetry(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b,
                                          const int32_t *orb_irrep, int target, tbsci_pruned **out);
tbsci_status tbsci_pruned_count(const tbsci_pruned *pr, int64_t *ndet);
void tbsci_pruned_destroy(tbsci_pruned *pr);

/* sigma = H.c on a pruned space (Sec. II.A, Eq. 6; the classes of Sec. II.C):
 * c and sigma are compressed DEVICE arrays [nvec][ndet] of F64 or F32 (the
 * tensor-core types run as F32 here); sigma is overwritten. Enqueued on
 * `stream`. `pr` must come from the tables a and b. Errors: EINVAL, ENOMEM,
 * ECUDA. */
tbsci_status tbsci_sigma_pruned(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                const tbsci_pruned *pr, const void *c, void *sigma, int nvec, tbsci_dtype dtype,
                                tbsci_stream stream);
/* Diagonal H_KK of the pruned space into the DEVICE array diag[ndet] (FP64). */
tbsci_status tbsci_diagonal_pruned(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                   const tbsci_pruned *pr, double *diag, tbsci_stream stream);
/* tbsci_davidson on a pruned space: vecs is a DEVICE array [nroots][ndet]
 * (compressed) or NULL; options, guess and errors as tbsci_davidson. */
tbsci_status tbsci_davidson_pruned(tbsci_ctx *ctx, tbsci_ham *ham, const tbsci_tables *a, const tbsci_tables *b,
                                   const tbsci_pruned *pr, int nroots, const tbsci_davidson_opts *opts,
                                   double *energies, double *vecs, tbsci_davidson_info *info);

/* ---------------------------------------------------- bitstring selection */

/* Weights of the strings of a TPB vector (Sec. III.B): with c normalised,
 * W_a(w) = sum_u c(w, u)^2 and W_b(u) = sum_w c(w, u)^2. c: DEVICE FP64
 * [l_a][l_b] (need not be normalised); wa, wb: HOST [l_a], [l_b]. Fixed
 * reduction order (run-to-run identical). Blocks until done.
 * Errors: EINVAL (null pointers, a zero vector), ENOMEM, ECUDA. */
tbsci_status tbsci_string_weights(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b, const double *c,
                                  double *wa, double *wb, tbsci_stream stream);
/* Bitstring selection by weight (Sec. III.B): the alpha (beta) strings whose
 * weight in c is at least delta times the weight of the HF string, read as the
 * string of largest weight. sel_a / sel_b: HOST arrays of capacity l_a / l_b
 * that receive the kept strings in ascending order; *na / *nb their counts.
 * The kept sets define the next TPB space. Errors: EINVAL (null pointers,
 * delta < 0, an empty space, a zero vector), ENOMEM, ECUDA. */
tbsci_status tbsci_select_by_weight(tbsci_ctx *ctx, const tbsci_tables *a, const tbsci_tables *b, const double *c,
                                    double delta, uint64_t *sel_a, int64_t *na, uint64_t *sel_b, int64_t *nb,
                                    tbsci_stream stream);
/* Coefficient distribution (Fig. 3): counts[k] = number of entries of the DEVICE
 * FP64 array x[n] with edges[k-1] <= |x| < edges[k] (counts[0]: |x| < edges[0];
 * counts[nedges]: |x| >= edges[nedges-1]). edges: HOST, strictly ascending,
 * 1..256 values; for the paper's bins of |c_K / c_HF| on a logarithmic scale
 * pass edges 10^e |c_HF|. counts: HOST [nedges + 1]. Exact integer counts.
 * Errors: EINVAL, ENOMEM, ECUDA. */
tbsci_status tbsci_coefficient_histogram(tbsci_ctx *ctx, const double *x, int64_t n, const double *edges, int nedges,
                                         int64_t *counts, tbsci_stream stream);

/* --------------------------------------------------------------- serving */

/* A request loop for many solves (no counterpart in the paper, which runs one
 * solve at a time): requests of any norb, electron counts and string sets are
 * submitted from any thread; a scheduler thread admits them against an HBM
 * budget in arrival order, builds their strings, tables and Hamiltonian on the
 * device, and advances all admitted solves together -- continuous batching:
 * a request that arrives while others run joins as soon as a slot and memory
 * are free, its sigma work goes into the same batched launches and its vector
 * work overlaps on its own stream. Each solve is the Davidson of tbsci_davidson,
 * so a result does not depend on what else was running (batched sigma launches
 * compute every job exactly as a launch of its own would). */
typedef struct tbsci_server tbsci_server;

typedef struct tbsci_server_opts {
    int device;
    size_t hbm_budget; /* bytes the admitted solves may hold; 0 -> 60 GiB */
    int max_active;    /* solves advanced together; 0 -> 64 */
    int max_queue;     /* submitted but not yet admitted; 0 -> 4096 (then EAGAIN) */
    int fuse_sigma;    /* 0 or 1: one batched sigma launch per precision per
                          scheduler round; -1: one launch per solve */
    int fail_admission_at; /* test hook: the n-th admission (1-based) fails with ENOMEM; 0 = off */
    const char *tune_cache; /* NULL, or a file of tbsci_tune_cache_save loaded into
                               the server's context: solves of a cached shape that
                               are launched on their own use its tuned shape */
} tbsci_server_opts;

typedef struct tbsci_request {
    int norb, nalpha, nbeta;
    const double *h;   /* HOST [norb*norb], copied at submit */
    const double *eri; /* HOST [norb^4] chemists' order, copied at submit */
    double ecore;
    const uint64_t *alpha; /* HOST selected alpha strings or NULL (full space) */
    int64_t n_alpha;
    const uint64_t *beta;  /* HOST selected beta strings or NULL (full space) */
    int64_t n_beta;
    int nroots;            /* 1..8 */
    int mixed;             /* 0: FP64 throughout; 1, 2, 3: FP32, FP32 + split-TF32
                              tensor-core or FP32 + BF16 tensor-core sigma, then FP64
                              refinement (the mixed modes of tbsci_davidson_opts);
                              other values: EINVAL */
    double tol_energy, tol_residual; /* 0 -> the tbsci_davidson defaults */
    int max_iter;          /* 0 -> 1000 */
} tbsci_request;

typedef struct tbsci_result {
    tbsci_status status;   /* OK, ENOCONV, EINVAL, ENOMEM, ECUDA */
    int nroots;
    double energies[8];
    double residual[8];
    int iterations, nsigma, nsigma_f32;
    int64_t ndet;
    /* seconds since the server was created */
    double t_submit, t_admit, t_first_sigma, t_done;
} tbsci_result;

/* Starts a server (its own context and scheduler thread) on opts->device.
 * Errors: EINVAL, ENOMEM, ECUDA. */
tbsci_status tbsci_server_create(const tbsci_server_opts *opts, tbsci_server **out);
/* Queues a solve; copies every host array before returning. *ticket identifies
 * it in tbsci_poll. Errors: EINVAL (bad sizes or null arrays), EAGAIN (queue
 * full), EBUSY (server shutting down). */
tbsci_status tbsci_submit(tbsci_server *srv, const tbsci_request *req, uint64_t *ticket);
/* Waits up to timeout_ms (0: do not wait, < 0: forever) for the ticket. OK with
 * *out filled (the ticket is then released), ETIMEOUT when not finished in time,
 * EINVAL for an unknown ticket. */
tbsci_status tbsci_poll(tbsci_server *srv, uint64_t ticket, int timeout_ms, tbsci_result *out);
/* Number of queued and of admitted (running) requests. */
tbsci_status tbsci_server_load(tbsci_server *srv, int *queued, int *active);
/* Stops the scheduler after the running solves finish; queued requests are
 * dropped with EBUSY results. Frees everything. */
void tbsci_server_destroy(tbsci_server *srv);

/* Overlaps of FP64 DEVICE vectors: S[i*mb + j] = sum_K A[i][K] * B[j][K] for
 * i < ma, j < mb, each vector n long (CI vectors of a space: n = l_a * l_b; the
 * Rayleigh-matrix and Gram-Schmidt products of the Davidson of Sec. III.A). S is
 * a HOST array [ma*mb]. Fixed grid and fixed reduction order: the result is
 * run-to-run bit-identical. Scratch of (2 * SM count + 1) * ma * mb doubles is
 * allocated and freed inside the call. Blocks until done.
 * Errors: EINVAL (null pointers, ma or mb < 0, n < 0), ENOMEM, ECUDA. */
tbsci_status tbsci_overlap(tbsci_ctx *ctx, const double *A, int ma, const double *B, int mb, int64_t n,
                           double *S, tbsci_stream stream);

/* Allocation-free form of tbsci_overlap, for callers that must not allocate
 * device memory while they run: for example a framework that has handed all
 * free HBM to its own caching pool (a cudaMalloc would fail or break its
 * accounting), or a latency-bound serving loop where cudaMalloc/cudaFree would
 * synchronise the device and stall other streams. The paper has no counterpart.
 *
 * Same product as tbsci_overlap, but S is a DEVICE array [ma*mb] written on
 * `stream`, and the call returns without waiting. The per-block partial sums
 * live in a 2 MiB array of static device memory that the library holds on every
 * GPU that loads it until the process exits; it limits ma * mb to 512
 * (larger requests return EINVAL and launch nothing). Every partial is
 * rewritten by each call, so nothing needs clearing between calls, but all calls
 * share the one array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * The first call on each device resolves the array's device address (and may
 * load the library's device code); make that first call during set-up, before
 * any stream capture. That address is kept for the rest of the process: after
 * a cudaDeviceReset of the device it is stale, so a process that resets a
 * device must not call this entry point on it again. No call allocates: no
 * cudaMalloc, cudaFree or allocating library routine. Errors: EINVAL, ECUDA. */
tbsci_status tbsci_overlap_noalloc(tbsci_ctx *ctx, const double *A, int ma, const double *B, int mb, int64_t n,
                                   double *S, tbsci_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TBSCI_H */
