/*
 * Plain FP64 CPU oracle for the TBSCI sigma = H.c product (test infrastructure
 * only: tests, the smoke check and the bench's CPU-baseline leg use it; the
 * CUDA library never links or calls it, and this file includes nothing of it).
 *
 * Everything here follows textbook definitions, one step at a time:
 *
 *  - A determinant of the TPB space (Sec. II.A, Eq. 2-5) is the product of an
 *    alpha string S_w and a beta string S_u, index K = w * l_beta + u (0-based,
 *    beta fastest). As a spin-orbital determinant it is
 *        a+_{alpha occupations, ascending} a+_{beta occupations, ascending} |0>,
 *    i.e. spin orbital P < n is alpha orbital P, P >= n is beta orbital P - n,
 *    and creation/annihilation signs count occupied spin orbitals below P in
 *    that order.
 *  - The Hamiltonian is H = ecore + sum_PQ h_PQ a+_P a_Q
 *                        + 1/4 sum_PQRS <PQ||RS> a+_P a+_Q a_S a_R,
 *    with <PQ|RS> = (pr|qs) delta(spin P, spin R) delta(spin Q, spin S) built
 *    from chemists' spatial integrals, and <PQ||RS> = <PQ|RS> - <PQ|SR>.
 *  - Matrix elements follow the Slater-Condon rules (Sec. II.C, Eq. 8: only
 *    determinants that differ by at most two spin orbitals couple):
 *      diagonal      ecore + sum_i h_ii + 1/2 sum_ij <ij||ij>
 *      single i->a   sgn * (h_ai + sum_{k in J} <ak||ik>)
 *      double ij->ab sgn * <ab||ij>
 *    where sgn is obtained by applying the operators one at a time to the
 *    source determinant, each sign a counted loop over lower occupied orbitals.
 *  - Excitations are enumerated over spin orbitals; a target is kept only when
 *    both of its strings are in the selected sets (binary search).
 *
 * String enumeration and the per-string link tables (BETA_SINGLE_LINK /
 * BETA_DOUBLE_LINK, Sec. II.C and Sec. III.C) are produced here by explicit
 * loops in the conventions the library documents, for bit-exact comparison.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ bits */

static int bit_of(uint64_t s, int i) { return (int)((s >> i) & 1u); }

static int count_bits(uint64_t s, int n)
{
    int c = 0;
    for (int i = 0; i < n; i++) c += bit_of(s, i);
    return c;
}

/* sorted-set membership by binary search; -1 when absent */
static int64_t find_string(const uint64_t *set, int64_t len, uint64_t s)
{
    int64_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (set[mid] == s) return mid;
        if (set[mid] < s) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------- strings */

/* All C(n, N) strings in ascending integer order: the positions array walks
 * combinations in colexicographic order, which is ascending integer order. */
int64_t orc_fci_strings(int n, int N, uint64_t *out, int64_t cap)
{
    int pos[64];
    int64_t m = 0;
    if (N < 0 || N > n || n > 64) return -1;
    for (int k = 0; k < N; k++) pos[k] = k;
    for (;;) {
        uint64_t s = 0;
        for (int k = 0; k < N; k++) s |= (uint64_t)1 << pos[k];
        if (out && m < cap) out[m] = s;
        m++;
        /* next combination in colex order: find the lowest k whose position can
         * move up by one without colliding with position k+1 */
        int k = 0;
        while (k < N && ((k + 1 < N) ? (pos[k] + 1 == pos[k + 1]) : (pos[k] + 1 == n))) k++;
        if (k >= N) break;
        pos[k]++;
        for (int j = 0; j < k; j++) pos[j] = j;
    }
    return m;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Sorted copy of a selected string list. Returns 0, or 1 = wrong electron
 * count, 2 = bit at or above n, 3 = duplicate string. */
int orc_sort_validate(int n, int N, const uint64_t *in, int64_t m, uint64_t *out)
{
    for (int64_t i = 0; i < m; i++) {
        if (n < 64 && (in[i] >> n) != 0) return 2;
        if (count_bits(in[i], 64) != N) return 1;
    }
    memcpy(out, in, (size_t)m * sizeof(uint64_t));
    qsort(out, (size_t)m, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 1; i < m; i++)
        if (out[i] == out[i - 1]) return 3;
    return 0;
}

/* ---------------------------------------------------- operator algebra */

/* a_P on a string (one spin): returns sign, 0 when P is empty. */
static int str_annihilate(uint64_t *s, int P)
{
    if (!bit_of(*s, P)) return 0;
    int below = 0;
    for (int Q = 0; Q < P; Q++) below += bit_of(*s, Q);
    *s &= ~((uint64_t)1 << P);
    return (below & 1) ? -1 : 1;
}

/* a+_P on a string (one spin): returns sign, 0 when P is occupied. */
static int str_create(uint64_t *s, int P)
{
    if (bit_of(*s, P)) return 0;
    int below = 0;
    for (int Q = 0; Q < P; Q++) below += bit_of(*s, Q);
    *s |= (uint64_t)1 << P;
    return (below & 1) ? -1 : 1;
}

/* ----------------------------------------------------------- link tables */

/* Single links of each source string J (row = J): targets I = a+_p a_q |J>
 * inside the set, with sign <I|a+_p a_q|J>, in ascending (q, p) order. When
 * tgt is NULL only the row offsets are written. Returns the total count. */
int64_t orc_links_single(int n, const uint64_t *strs, int64_t l, int64_t *off,
                         int32_t *tgt, int8_t *sign, uint8_t *p_out, uint8_t *q_out)
{
    int64_t total = 0;
    for (int64_t j = 0; j < l; j++) {
        off[j] = total;
        for (int q = 0; q < n; q++) {
            for (int p = 0; p < n; p++) {
                uint64_t s = strs[j];
                int sg = str_annihilate(&s, q);
                if (!sg) continue;
                if (p == q) continue;
                int sc = str_create(&s, p);
                if (!sc) continue;
                int64_t i = find_string(strs, l, s);
                if (i < 0) continue;
                if (tgt) {
                    tgt[total] = (int32_t)i;
                    sign[total] = (int8_t)(sg * sc);
                    p_out[total] = (uint8_t)p;
                    q_out[total] = (uint8_t)q;
                }
                total++;
            }
        }
    }
    off[l] = total;
    return total;
}

/* Double links of each source string J: targets I = a+_p a+_r a_s a_q |J> with
 * q < s annihilated, p < r created (p, r empty in J), sign
 * <I|a+_p a+_r a_s a_q|J> (a_q applied first), ascending (q, s, p, r). */
int64_t orc_links_double(int n, const uint64_t *strs, int64_t l, int64_t *off,
                         int32_t *tgt, int8_t *sign, uint8_t *p_out, uint8_t *r_out,
                         uint8_t *q_out, uint8_t *s_out)
{
    int64_t total = 0;
    for (int64_t j = 0; j < l; j++) {
        off[j] = total;
        uint64_t J = strs[j];
        for (int q = 0; q < n; q++) {
            if (!bit_of(J, q)) continue;
            for (int s = q + 1; s < n; s++) {
                if (!bit_of(J, s)) continue;
                for (int p = 0; p < n; p++) {
                    if (bit_of(J, p)) continue;
                    for (int r = p + 1; r < n; r++) {
                        if (bit_of(J, r)) continue;
                        uint64_t x = J;
                        int sg = str_annihilate(&x, q);
                        sg *= str_annihilate(&x, s);
                        sg *= str_create(&x, r);
                        sg *= str_create(&x, p);
                        int64_t i = find_string(strs, l, x);
                        if (i < 0) continue;
                        if (tgt) {
                            tgt[total] = (int32_t)i;
                            sign[total] = (int8_t)sg;
                            p_out[total] = (uint8_t)p;
                            r_out[total] = (uint8_t)r;
                            q_out[total] = (uint8_t)q;
                            s_out[total] = (uint8_t)s;
                        }
                        total++;
                    }
                }
            }
        }
    }
    off[l] = total;
    return total;
}

/* ------------------------------------------------- spin-orbital algebra */

typedef struct {
    uint64_t a, b; /* alpha string, beta string */
} det_t;

typedef struct {
    int n;
    const double *h;   /* [n][n] */
    const double *eri; /* [n][n][n][n], (ij|kl) */
    double ecore;
} ham_t;

static int so_occ(const det_t *d, int n, int P)
{
    return P < n ? bit_of(d->a, P) : bit_of(d->b, P - n);
}

static void so_flip(det_t *d, int n, int P)
{
    if (P < n) d->a ^= (uint64_t)1 << P;
    else d->b ^= (uint64_t)1 << (P - n);
}

/* number of occupied spin orbitals strictly below P (alpha block first) */
static int so_below(const det_t *d, int n, int P)
{
    int c = 0;
    for (int Q = 0; Q < P; Q++) c += so_occ(d, n, Q);
    return c;
}

static int so_annihilate(det_t *d, int n, int P)
{
    if (!so_occ(d, n, P)) return 0;
    int c = so_below(d, n, P);
    so_flip(d, n, P);
    return (c & 1) ? -1 : 1;
}

static int so_create(det_t *d, int n, int P)
{
    if (so_occ(d, n, P)) return 0;
    int c = so_below(d, n, P);
    so_flip(d, n, P);
    return (c & 1) ? -1 : 1;
}

static int spin_of(int n, int P) { return P < n ? 0 : 1; }
static int orb_of(int n, int P) { return P < n ? P : P - n; }

static double chem(const ham_t *H, int i, int j, int k, int l)
{
    int n = H->n;
    return H->eri[(((size_t)i * n + j) * n + k) * n + l];
}

static double h_so(const ham_t *H, int P, int Q)
{
    int n = H->n;
    if (spin_of(n, P) != spin_of(n, Q)) return 0.0;
    return H->h[orb_of(n, P) * n + orb_of(n, Q)];
}

/* physicists' <PQ|RS> = (pr|qs) with spin deltas */
static double g_so(const ham_t *H, int P, int Q, int R, int S)
{
    int n = H->n;
    if (spin_of(n, P) != spin_of(n, R) || spin_of(n, Q) != spin_of(n, S)) return 0.0;
    return chem(H, orb_of(n, P), orb_of(n, R), orb_of(n, Q), orb_of(n, S));
}

static double ga_so(const ham_t *H, int P, int Q, int R, int S)
{
    return g_so(H, P, Q, R, S) - g_so(H, P, Q, S, R);
}

static double diag_element(const ham_t *H, const det_t *d)
{
    int n = H->n, M = 2 * n;
    double e = H->ecore;
    for (int i = 0; i < M; i++) {
        if (!so_occ(d, n, i)) continue;
        e += h_so(H, i, i);
        for (int j = 0; j < M; j++) {
            if (!so_occ(d, n, j)) continue;
            e += 0.5 * ga_so(H, i, j, i, j);
        }
    }
    return e;
}

typedef struct {
    const uint64_t *sa, *sb;
    int64_t la, lb;
} space_t;

/* Appends (column, value) for every determinant of the space coupled to row
 * K = (w, u), diagonal first. Returns the count. Columns are distinct. */
static int64_t row_elements(const ham_t *H, const space_t *sp, int64_t K,
                            int64_t *cols, double *vals)
{
    int n = H->n, M = 2 * n;
    int64_t w = K / sp->lb, u = K % sp->lb;
    det_t J = {sp->sa[w], sp->sb[u]};
    int64_t m = 0;
    cols[m] = K;
    vals[m] = diag_element(H, &J);
    m++;
    /* singles i -> a */
    for (int i = 0; i < M; i++) {
        if (!so_occ(&J, n, i)) continue;
        for (int a = 0; a < M; a++) {
            if (so_occ(&J, n, a)) continue;
            if (spin_of(n, a) != spin_of(n, i)) continue; /* keeps N_alpha, N_beta */
            det_t I = J;
            int sg = so_annihilate(&I, n, i);
            sg *= so_create(&I, n, a);
            int64_t wi = find_string(sp->sa, sp->la, I.a);
            if (wi < 0) continue;
            int64_t ui = find_string(sp->sb, sp->lb, I.b);
            if (ui < 0) continue;
            double v = h_so(H, a, i);
            for (int k = 0; k < M; k++)
                if (so_occ(&J, n, k)) v += ga_so(H, a, k, i, k);
            cols[m] = wi * sp->lb + ui;
            vals[m] = sg * v;
            m++;
        }
    }
    /* doubles ij -> ab, i < j, a < b */
    for (int i = 0; i < M; i++) {
        if (!so_occ(&J, n, i)) continue;
        for (int j = i + 1; j < M; j++) {
            if (!so_occ(&J, n, j)) continue;
            for (int a = 0; a < M; a++) {
                if (so_occ(&J, n, a)) continue;
                for (int b = a + 1; b < M; b++) {
                    if (so_occ(&J, n, b)) continue;
                    /* keep the number of electrons of each spin */
                    int nin = (spin_of(n, i) == 0) + (spin_of(n, j) == 0);
                    int nout = (spin_of(n, a) == 0) + (spin_of(n, b) == 0);
                    if (nin != nout) continue;
                    det_t I = J;
                    I.a = J.a; I.b = J.b;
                    int sg = so_annihilate(&I, n, i);
                    sg *= so_annihilate(&I, n, j);
                    sg *= so_create(&I, n, b);
                    sg *= so_create(&I, n, a);
                    int64_t wi = find_string(sp->sa, sp->la, I.a);
                    if (wi < 0) continue;
                    int64_t ui = find_string(sp->sb, sp->lb, I.b);
                    if (ui < 0) continue;
                    cols[m] = wi * sp->lb + ui;
                    vals[m] = sg * ga_so(H, a, b, i, j);
                    m++;
                }
            }
        }
    }
    return m;
}

/* Upper bound on the number of elements of one row. */
int64_t orc_row_capacity(int n, int na, int nb)
{
    int64_t occ = na + nb, vir = 2 * n - occ;
    return 1 + occ * vir + (occ * (occ - 1) / 2) * (vir * (vir - 1) / 2);
}

/* Row K of H restricted to the space: writes cols/vals, returns the count. */
int64_t orc_row(int n, const uint64_t *sa, int64_t la, const uint64_t *sb, int64_t lb,
                const double *h, const double *eri, double ecore, int64_t K,
                int64_t *cols, double *vals)
{
    ham_t H = {n, h, eri, ecore};
    space_t sp = {sa, sb, la, lb};
    return row_elements(&H, &sp, K, cols, vals);
}

/* sigma_K = sum_J H_KJ c_J for the rows listed in `rows` (all when rows is
 * NULL and nrows = la*lb). C is [nvec][la*lb]; out is [nvec][nrows]. When
 * bound is not NULL it receives sum_J |H_KJ| |c_J| (same layout). */
void orc_sigma_rows(int n, int na, int nb, const uint64_t *sa, int64_t la,
                    const uint64_t *sb, int64_t lb, const double *h, const double *eri,
                    double ecore, const double *C, int nvec, const int64_t *rows,
                    int64_t nrows, double *out, double *bound, int nthreads)
{
    ham_t H = {n, h, eri, ecore};
    space_t sp = {sa, sb, la, lb};
    int64_t N = la * lb;
    int64_t cap = orc_row_capacity(n, na, nb);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        int64_t *cols = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        double *vals = (double *)malloc((size_t)cap * sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nrows; r++) {
            int64_t K = rows ? rows[r] : r;
            int64_t m = row_elements(&H, &sp, K, cols, vals);
            for (int v = 0; v < nvec; v++) {
                const double *c = C + (size_t)v * N;
                double acc = 0.0, ab = 0.0;
                for (int64_t t = 0; t < m; t++) {
                    acc += vals[t] * c[cols[t]];
                    ab += (vals[t] < 0 ? -vals[t] : vals[t]) * (c[cols[t]] < 0 ? -c[cols[t]] : c[cols[t]]);
                }
                out[(size_t)v * nrows + r] = acc;
                if (bound) bound[(size_t)v * nrows + r] = ab;
            }
        }
        free(cols);
        free(vals);
    }
}

/* ----------------------------------------------- pruned spaces (D_TBSCI) */

/* A pruned space (Sec. II.A, Eq. 6): for each alpha string w the ascending list
 * of allowed beta indices I_w = cols[off[w] .. off[w+1]). Determinant (w, u)
 * with u in I_w has the compressed index off[w] + (position of u in I_w). */
typedef struct {
    const int64_t *off; /* [la + 1] */
    const int32_t *cols;
    int64_t la, nd;
} pruned_t;

/* compressed index of (w, u); -1 when u is not in I_w (binary search) */
static int64_t pruned_index(const pruned_t *pr, int64_t w, int64_t u)
{
    int64_t lo = pr->off[w], hi = pr->off[w + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (pr->cols[mid] == u) return mid;
        if (pr->cols[mid] < u) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* alpha string of compressed index K: the last w with off[w] <= K */
static int64_t pruned_row_of(const pruned_t *pr, int64_t K)
{
    int64_t lo = 0, hi = pr->la - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (pr->off[mid] <= K) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* sigma over a pruned space: for every listed compressed row K (all when rows
 * is NULL, nrows = nd), sigma_K = sum_{J in D} H_KJ c_J. The elements are the
 * full TPB row of the Slater-Condon rules, kept when the coupled determinant is
 * a member (H restricted to D is the principal submatrix of H on D's
 * determinants). C is [nvec][nd], out / bound [nvec][nrows]. */
void orc_sigma_pruned(int n, int na, int nb, const uint64_t *sa, int64_t la, const uint64_t *sb, int64_t lb,
                      const int64_t *off, const int32_t *pcols, const double *h, const double *eri, double ecore,
                      const double *C, int nvec, const int64_t *rows, int64_t nrows, double *out, double *bound,
                      int nthreads)
{
    ham_t H = {n, h, eri, ecore};
    space_t sp = {sa, sb, la, lb};
    pruned_t pr = {off, pcols, la, off[la]};
    int64_t cap = orc_row_capacity(n, na, nb);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        int64_t *cols = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        double *vals = (double *)malloc((size_t)cap * sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nrows; r++) {
            int64_t Kp = rows ? rows[r] : r;
            int64_t w = pruned_row_of(&pr, Kp);
            int64_t K = w * lb + pcols[Kp];
            int64_t m = row_elements(&H, &sp, K, cols, vals);
            for (int v = 0; v < nvec; v++) {
                const double *c = C + (size_t)v * pr.nd;
                double acc = 0.0, ab = 0.0;
                for (int64_t t = 0; t < m; t++) {
                    int64_t Jp = pruned_index(&pr, cols[t] / lb, cols[t] % lb);
                    if (Jp < 0) continue;
                    acc += vals[t] * c[Jp];
                    ab += (vals[t] < 0 ? -vals[t] : vals[t]) * (c[Jp] < 0 ? -c[Jp] : c[Jp]);
                }
                out[(size_t)v * nrows + r] = acc;
                if (bound) bound[(size_t)v * nrows + r] = ab;
            }
        }
        free(cols);
        free(vals);
    }
}

/* Diagonal of a pruned space for the listed compressed rows (all when rows is NULL). */
void orc_diagonal_pruned(int n, const uint64_t *sa, int64_t la, const uint64_t *sb, const int64_t *off,
                         const int32_t *pcols, const double *h, const double *eri, double ecore,
                         const int64_t *rows, int64_t nrows, double *out)
{
    ham_t H = {n, h, eri, ecore};
    pruned_t pr = {off, pcols, la, off[la]};
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t Kp = rows ? rows[r] : r;
        det_t d = {sa[pruned_row_of(&pr, Kp)], sb[pcols[Kp]]};
        out[r] = diag_element(&H, &d);
    }
}

/* Diagonal H_KK for the listed rows (all when rows is NULL). */
void orc_diagonal(int n, const uint64_t *sa, int64_t la, const uint64_t *sb, int64_t lb,
                  const double *h, const double *eri, double ecore, const int64_t *rows,
                  int64_t nrows, double *out)
{
    ham_t H = {n, h, eri, ecore};
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t K = rows ? rows[r] : r;
        det_t d = {sa[K / lb], sb[K % lb]};
        out[r] = diag_element(&H, &d);
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
