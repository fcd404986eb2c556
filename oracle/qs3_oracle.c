/*
 * qs3_oracle.c -- plain, slow CPU restatement of the QS^3 method
 * (Ueda, Yunoki, Shimokawa, "Quantum spin solver near saturation: QS^3").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle of the GPU
 * library.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA path and never calls it.
 *
 * Conventions follow the paper, not the GPU path:
 *   - sites are 1-based, 1 <= n_1 < ... < n_Nd <= N  (Sec. "Representation of
 *     states with the U(1) symmetry");
 *   - the state index a is 1-based, a = F(n) = 1 + sum_m C(n_m - 1, m)
 *     (Eq. a_of_n);
 *   - a site r is spin s of the unit cell at (x, y, z), with
 *     r - 1 = s + n_sub (x + Lx (y + Ly z)) (n_sub spins per cell, 1 for a
 *     Bravais lattice), and the translation T^t moves every cell by +t modulo
 *     (Lx, Ly, Lz), keeping s; the group has Lx Ly Lz elements.
 *   - the momentum sector K = (Kx, Ky, Kz) means k.a_alpha = 2 pi K_alpha/L_alpha
 *     (input parameters KX, KY, KZ).
 *
 * Everything is fp64.  Complex vectors are C99 double complex (interleaved
 * re, im pairs for a caller using plain double arrays).
 *
 * Readings of garbled or silent passages (each one is listed in the design
 * notes as well):
 *   R1  norm ratio in Alg. 8/9/11: sqrt(N_a'/N_a) as in Eq. (hak2), i.e. the
 *       ratio of normalisation factors, not of their square roots R.
 *   R3  Alg. 3, f = True branch: the site entering the list is r' (r leaves).
 *   R4  Alg. 1/2: binary_search returns p = ls - 1 + #{k : s_k <= s0}; the
 *       column search of Alg. 1 therefore yields max{k : C(k,m) <= s-1},
 *       which is >= m-1 because C(k,m) = 0 for k < m.
 *   R6  Alg. 7 keeps the last translation with the minimum index ("<=");
 *       translations are visited with tx fastest, then ty, then tz.
 *   R9  site field: -sum_r h_r s^z_r adds sum_{r in n} h_r - (1/2) sum_r h_r
 *       to the diagonal (the paper drops a uniform field as a constant).
 *   R-N Alg. 6 keeps a state when N_{a,k} exceeds 1e-8 (it is either >= N or
 *       zero up to rounding of the phase sum).
 *   Duplicate bond pairs add their couplings (Eq. (1) sums each pair once).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXND 16

typedef double complex zdbl;

typedef struct {
    int N, nd, nb;
    const int *r, *rp;           /* bond end points, 1-based, normalised r < r' */
    const double *jxy, *jz;
    const double *h;             /* per-site field or NULL */
    int L[3];
    int nsub;                    /* spins per unit cell */
    int ncell;                   /* Lx Ly Lz: the order of the translation group */
    uint64_t *C;                 /* (N+1) x (nd+1) table of binomials */
} orc_ctx;

/* ---------------------------------------------------------------- binomials */

/* Pascal's rule; returns -1 on uint64 overflow beyond 2^63. */
static int make_binom(orc_ctx *c)
{
    int N = c->N, nd = c->nd;
    c->C = (uint64_t *)calloc((size_t)(N + 1) * (nd + 1), sizeof(uint64_t));
    if (!c->C) return -1;
    for (int k = 0; k <= N; ++k) {
        c->C[(size_t)k * (nd + 1) + 0] = 1;
        for (int m = 1; m <= nd; ++m) {
            if (k == 0) { c->C[m] = 0; continue; }
            uint64_t a = c->C[(size_t)(k - 1) * (nd + 1) + m - 1];
            uint64_t b = c->C[(size_t)(k - 1) * (nd + 1) + m];
            uint64_t s = a + b;
            if (s < a || s > ((uint64_t)1 << 63)) return -1;
            c->C[(size_t)k * (nd + 1) + m] = s;
        }
    }
    return 0;
}

static uint64_t Cb(const orc_ctx *c, int k, int m)
{
    if (m < 0 || k < m || k < 0) return 0;
    return c->C[(size_t)k * (c->nd + 1) + m];
}

static int ctx_init(orc_ctx *c, int N, int nd, int nb, const int *r, const int *rp,
                    const double *jxy, const double *jz, const double *h, const int *L)
{
    memset(c, 0, sizeof(*c));
    c->N = N; c->nd = nd; c->nb = nb; c->r = r; c->rp = rp;
    c->jxy = jxy; c->jz = jz; c->h = h;
    /* L: Lx, Ly, Lz, n_sub (four ints) */
    c->nsub = 1;
    if (L) { c->L[0] = L[0]; c->L[1] = L[1]; c->L[2] = L[2]; c->nsub = L[3] > 0 ? L[3] : 1; }
    c->ncell = c->L[0] * c->L[1] * c->L[2];
    if (nd < 0 || nd > ORC_MAXND || nd > N) return -1;
    return make_binom(c);
}

static void ctx_free(orc_ctx *c) { free(c->C); c->C = NULL; }

/* ------------------------------------------------------- Eq. (a_of_n), Alg 1-3 */

/* Eq. (a_of_n): a = 1 + sum_{m=1}^{Nd} C(r_m - 1, m). */
static uint64_t F(const orc_ctx *c, const int *n)
{
    uint64_t a = 1;
    for (int m = 1; m <= c->nd; ++m) a += Cb(c, n[m - 1] - 1, m);
    return a;
}

/* Alg. 2 over the integer vector n (1-based view n[1..nd] = n0[0..nd-1]). */
static int binary_search_int(int s0, const int *n0, int ls, int le, int *f)
{
    /* largest p in [ls-1, le] with s_p <= s0 (s_{ls-1} = -inf) */
    int lo = ls - 1, hi = le;
    while (lo < hi) {
        int mid = lo + (hi - lo + 1) / 2;
        if (n0[mid - 1] <= s0) lo = mid; else hi = mid - 1;
    }
    *f = (lo >= ls && n0[lo - 1] == s0);
    return lo;
}

/* Alg. 2 over a sorted uint64 vector (sigma), 1-based view. */
static int64_t binary_search_u64(uint64_t s0, const uint64_t *s, int64_t ls, int64_t le, int *f)
{
    int64_t lo = ls - 1, hi = le;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (s[mid - 1] <= s0) lo = mid; else hi = mid - 1;
    }
    *f = (lo >= ls && s[lo - 1] == s0);
    return lo;
}

/* Inverse of Eq. (a_of_n) (the paper's F_bar, Alg. 1): the sorted list n
 * with F(n) = a.  Every list whose largest site is below r has an index
 * below 1 + C(r - 1, Nd), so the largest site of n is the largest r with
 * C(r - 1, Nd) <= a - 1; the remaining sites are the inverse, for Nd - 1
 * sites below r, of what is left of a - 1.  Each site is found by scanning
 * down from the previous one.  trace (optional) records the paper's running
 * value s = (what is left) + 1 after each of the sites n_Nd .. n_2. */
static void f_bar(const orc_ctx *c, uint64_t a, int *n, uint64_t *trace)
{
    uint64_t left = a - 1;
    int top = c->N;
    int t = 0;
    for (int m = c->nd; m >= 1; --m) {
        int r = top;
        while (r > m && Cb(c, r - 1, m) > left) --r;
        n[m - 1] = r;
        left -= Cb(c, r - 1, m);
        top = r - 1;
        if (trace && m >= 2) trace[t++] = left + 1;
    }
}

/* membership of site r in the sorted list n */
static int contains(const int *n, int nd, int r)
{
    for (int i = 0; i < nd; ++i)
        if (n[i] == r) return 1;
    return 0;
}

/* Alg. 3 by its definition (reading R3): on a bond (r, r') with exactly one
 * down spin, the exchange moves that spin to the other end.  np = the list
 * without the site it leaves, with the site it enters, in ascending order.
 * Returns 0 (np untouched) when both ends or neither end hold a down spin. */
static int hop_target(int nd, const int *n, int r, int rp, int *np)
{
    const int in_r = contains(n, nd, r), in_rp = contains(n, nd, rp);
    if (in_r == in_rp) return 0;
    const int leave = in_r ? r : rp, enter = in_r ? rp : r;
    int k = 0;
    for (int i = 0; i < nd; ++i)
        if (n[i] != leave) np[k++] = n[i];
    np[k] = enter;
    for (int i = 1; i < nd; ++i) {            /* insertion sort */
        int v = np[i], j = i - 1;
        while (j >= 0 && np[j] > v) { np[j + 1] = np[j]; --j; }
        np[j + 1] = v;
    }
    return 1;
}

/* --------------------------------------------------------------- translations */

/* site r -> spin s of the cell at (x, y, z) */
static void site_xyz(const orc_ctx *c, int r, int *s, int *x, int *y, int *z)
{
    int q = r - 1;
    *s = q % c->nsub; q /= c->nsub;
    *x = q % c->L[0]; q /= c->L[0];
    *y = q % c->L[1]; *z = q / c->L[1];
}

static int xyz_site(const orc_ctx *c, int s, int x, int y, int z)
{
    return 1 + s + c->nsub * (x + c->L[0] * (y + c->L[1] * z));
}

static void insertion_sort(int *n, int nd)
{
    for (int i = 1; i < nd; ++i) {
        int v = n[i], j = i - 1;
        while (j >= 0 && n[j] > v) { n[j + 1] = n[j]; --j; }
        n[j + 1] = v;
    }
}

/* n' = insertion_sort(T^t n) */
static void translate(const orc_ctx *c, const int *n, const int *t, int *out)
{
    for (int m = 0; m < c->nd; ++m) {
        int s, x, y, z;
        site_xyz(c, n[m], &s, &x, &y, &z);
        x = (x + t[0]) % c->L[0];
        y = (y + t[1]) % c->L[1];
        z = (z + t[2]) % c->L[2];
        out[m] = xyz_site(c, s, x, y, z);
    }
    insertion_sort(out, c->nd);
}

/* k . t = 2 pi sum_alpha K_alpha t_alpha / L_alpha */
static double kdot(const orc_ctx *c, const int *K, const int *t)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += (double)K[a] * (double)t[a] / (double)c->L[a];
    return 2.0 * M_PI * s;
}

/* Alg. 5: N_{a,k} of state a, or 0 when a is not the representative / not
 * compatible with k. */
static double check_state(const orc_ctx *c, uint64_t a, const int *K)
{
    int n[ORC_MAXND], nt[ORC_MAXND];
    f_bar(c, a, n, NULL);
    zdbl cs = 0.0;
    int nc = 0;
    int t[3];
    for (t[2] = 0; t[2] < c->L[2]; ++t[2])
        for (t[1] = 0; t[1] < c->L[1]; ++t[1])
            for (t[0] = 0; t[0] < c->L[0]; ++t[0]) {
                translate(c, n, t, nt);
                uint64_t ap = F(c, nt);
                if (ap < a) return 0.0;
                if (ap == a) { cs += cexp(I * kdot(c, K, t)); nc += 1; }
            }
    double ab = cabs(cs);
    return ab * ab * (double)c->ncell / (double)nc;
}

/* Alg. 7: representative (minimum index over all translations) and the
 * translation l with T^l a' = rep (reading R6). */
static uint64_t representative(const orc_ctx *c, uint64_t ap, int *l)
{
    int n[ORC_MAXND], nt[ORC_MAXND];
    f_bar(c, ap, n, NULL);
    uint64_t rep = ap;
    int t[3];
    l[0] = l[1] = l[2] = 0;
    for (t[2] = 0; t[2] < c->L[2]; ++t[2])
        for (t[1] = 0; t[1] < c->L[1]; ++t[1])
            for (t[0] = 0; t[0] < c->L[0]; ++t[0]) {
                translate(c, n, t, nt);
                uint64_t a = F(c, nt);
                if (a <= rep) { rep = a; l[0] = t[0]; l[1] = t[1]; l[2] = t[2]; }
            }
    return rep;
}

/* -------------------------------------------------------- diagonal of Eq. (1) */

/* sum over bonds of J^z s^z s^z plus the site field (reading R9) for state n */
static double diag_elem(const orc_ctx *c, const int *n)
{
    double e = 0.0;
    for (int b = 0; b < c->nb; ++b) {
        int f, fp;
        f = contains(n, c->nd, c->r[b]);
        fp = contains(n, c->nd, c->rp[b]);
        e += (f == fp) ? c->jz[b] / 4.0 : -c->jz[b] / 4.0;
    }
    if (c->h) {
        for (int i = 1; i <= c->N; ++i) {
            int f;
            f = contains(n, c->nd, i);
            e += f ? 0.5 * c->h[i - 1] : -0.5 * c->h[i - 1];
        }
    }
    return e;
}

/* ============================================================ exported API */

#define ORC_LAT int N, int nd, int nb, const int *r, const int *rp, const double *jxy, \
                const double *jz, const double *h, const int *L
#define ORC_LAT_ARGS N, nd, nb, r, rp, jxy, jz, h, L

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* C(N, nd) or 0 on overflow */
uint64_t orc_binom(int N, int nd)
{
    orc_ctx c;
    if (ctx_init(&c, N, nd, 0, NULL, NULL, NULL, NULL, NULL, NULL)) { ctx_free(&c); return 0; }
    uint64_t v = Cb(&c, N, nd);
    ctx_free(&c);
    return v;
}

/* Eq. (a_of_n) on a 1-based sorted list */
uint64_t orc_F(int N, int nd, const int *n)
{
    orc_ctx c;
    if (ctx_init(&c, N, nd, 0, NULL, NULL, NULL, NULL, NULL, NULL)) { ctx_free(&c); return 0; }
    uint64_t a = F(&c, n);
    ctx_free(&c);
    return a;
}

/* Alg. 1; trace receives the nd-1 intermediate s values (may be NULL) */
int orc_f_bar(int N, int nd, uint64_t a, int *n, uint64_t *trace)
{
    orc_ctx c;
    if (ctx_init(&c, N, nd, 0, NULL, NULL, NULL, NULL, NULL, NULL)) { ctx_free(&c); return -1; }
    if (a < 1 || a > Cb(&c, N, nd)) { ctx_free(&c); return -1; }
    f_bar(&c, a, n, trace);
    ctx_free(&c);
    return 0;
}

/* all lists in index order: out[(a-1)*nd + m], 1-based sites */
int orc_unrank_all(int N, int nd, int *out)
{
    orc_ctx c;
    if (ctx_init(&c, N, nd, 0, NULL, NULL, NULL, NULL, NULL, NULL)) { ctx_free(&c); return -1; }
    uint64_t D = Cb(&c, N, nd);
#pragma omp parallel for schedule(static)
    for (int64_t a = 1; a <= (int64_t)D; ++a) f_bar(&c, (uint64_t)a, out + (size_t)(a - 1) * nd, NULL);
    ctx_free(&c);
    return 0;
}

/* Alg. 3 exposed for tests: returns F(n') */
uint64_t orc_spin_exchange(int N, int nd, const int *n, int r, int rp)
{
    orc_ctx c;
    if (ctx_init(&c, N, nd, 0, NULL, NULL, NULL, NULL, NULL, NULL)) { ctx_free(&c); return 0; }
    int f, fp, np[ORC_MAXND];
    f = contains(n, nd, r);
    fp = contains(n, nd, rp);
    uint64_t a = 0;
    if (f != fp) { hop_target(nd, n, r, rp, np); a = F(&c, np); }
    ctx_free(&c);
    return a;
}

/* Alg. 4 (plus reading R9): dense U(1) block, row-major D x D */
int orc_dense_u1(ORC_LAT, double *H)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    uint64_t D = Cb(&c, N, nd);
    memset(H, 0, sizeof(double) * D * D);
    for (uint64_t a = 1; a <= D; ++a) {
        int n[ORC_MAXND], np[ORC_MAXND];
        f_bar(&c, a, n, NULL);
        for (int b = 0; b < nb; ++b) {
            int f, fp;
            f = contains(n, nd, r[b]);
            fp = contains(n, nd, rp[b]);
            if (f == fp) {
                H[(a - 1) * D + (a - 1)] += jz[b] / 4.0;
            } else {
                H[(a - 1) * D + (a - 1)] -= jz[b] / 4.0;
                hop_target(nd, n, r[b], rp[b], np);
                uint64_t ap = F(&c, np);
                H[(a - 1) * D + (ap - 1)] += jxy[b] / 2.0;
            }
        }
        if (h) {
            for (int i = 1; i <= N; ++i) {
                int f;
                f = contains(n, nd, i);
                H[(a - 1) * D + (a - 1)] += f ? 0.5 * h[i - 1] : -0.5 * h[i - 1];
            }
        }
    }
    ctx_free(&c);
    return 0;
}

/* one row of the U(1) product psi = H phi (Alg. 4 applied on the fly) */
static zdbl hphi_u1_row(const orc_ctx *c, uint64_t a, const zdbl *phi, int64_t *terms)
{
    int n[ORC_MAXND], np[ORC_MAXND];
    f_bar(c, a, n, NULL);
    zdbl acc = diag_elem(c, n) * phi[a - 1];
    *terms += 1;
    for (int b = 0; b < c->nb; ++b) {
        int f, fp;
        f = contains(n, c->nd, c->r[b]);
        fp = contains(n, c->nd, c->rp[b]);
        if (f != fp) {
            hop_target(c->nd, n, c->r[b], c->rp[b], np);
            uint64_t ap = F(c, np);
            acc += (c->jxy[b] / 2.0) * phi[ap - 1];
            *terms += 1;
        }
    }
    return acc;
}

/* U(1) HPhi over all rows (complex vectors; a real vector is the case im = 0) */
int orc_hphi_u1(ORC_LAT, const double *phi, double *psi)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    uint64_t D = Cb(&c, N, nd);
    const zdbl *p = (const zdbl *)phi;
    zdbl *q = (zdbl *)psi;
    int64_t terms = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : terms)
    for (int64_t a = 1; a <= (int64_t)D; ++a) q[a - 1] = hphi_u1_row(&c, (uint64_t)a, p, &terms);
    ctx_free(&c);
    return 0;
}

/* U(1) HPhi on a list of 0-based rows only (sampled parity / CPU timing);
 * *nterms (may be NULL) receives the number of matrix terms applied */
int orc_hphi_u1_rows(ORC_LAT, const double *phi, int64_t nrows, const int64_t *rows, double *psi_rows,
                     int64_t *nterms)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    const zdbl *p = (const zdbl *)phi;
    zdbl *q = (zdbl *)psi_rows;
    int64_t terms = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : terms)
    for (int64_t i = 0; i < nrows; ++i) q[i] = hphi_u1_row(&c, (uint64_t)rows[i] + 1, p, &terms);
    if (nterms) *nterms = terms;
    ctx_free(&c);
    return 0;
}

/* Alg. 5 + 6: representative list for sector K.  First call with sigma = NULL
 * returns the dimension d; second call fills sigma (1-based indices a) and
 * Nak (normalisation factors N_{a,k}). */
int64_t orc_mk_list(ORC_LAT, const int *K, uint64_t *sigma, double *Nak)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    uint64_t D = Cb(&c, N, nd);
    int64_t d = 0;
    for (uint64_t a = 1; a <= D; ++a) {
        double nak = check_state(&c, a, K);
        if (nak > 1e-8) {
            if (sigma) { sigma[d] = a; Nak[d] = nak; }
            ++d;
        }
    }
    ctx_free(&c);
    return d;
}

/* Alg. 7 exposed: returns rep index, writes l[3] */
uint64_t orc_representative(ORC_LAT, uint64_t a, int *l)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return 0; }
    uint64_t rep = representative(&c, a, l);
    ctx_free(&c);
    return rep;
}

/* all translates F(T^t rep), t in the order tx fastest (N entries) */
int orc_orbit(ORC_LAT, uint64_t a, uint64_t *out)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    int n[ORC_MAXND], nt[ORC_MAXND], t[3];
    f_bar(&c, a, n, NULL);
    int i = 0;
    for (t[2] = 0; t[2] < c.L[2]; ++t[2])
        for (t[1] = 0; t[1] < c.L[1]; ++t[1])
            for (t[0] = 0; t[0] < c.L[0]; ++t[0]) {
                translate(&c, n, t, nt);
                out[i++] = F(&c, nt);
            }
    ctx_free(&c);
    return 0;
}

/* one row of Alg. 9 (readings R1, R6) */
static zdbl hphi_k_row(const orc_ctx *c, const int *K, const uint64_t *sigma, const double *Nak,
                       int64_t d, int64_t row /*1-based*/, const zdbl *phi, int64_t *terms)
{
    int n[ORC_MAXND], np[ORC_MAXND];
    f_bar(c, sigma[row - 1], n, NULL);
    zdbl acc = 0.0;
    *terms += 1;
    for (int b = 0; b < c->nb; ++b) {
        int f, fp;
        f = contains(n, c->nd, c->r[b]);
        fp = contains(n, c->nd, c->rp[b]);
        if (f == fp) {
            acc += (c->jz[b] / 4.0) * phi[row - 1];
        } else {
            acc -= (c->jz[b] / 4.0) * phi[row - 1];
            hop_target(c->nd, n, c->r[b], c->rp[b], np);
            uint64_t ap = F(c, np);
            int l[3];
            uint64_t rep = representative(c, ap, l);
            int found;
            int64_t col = binary_search_u64(rep, sigma, 1, d, &found);
            if (found) {
                zdbl ph = cexp(I * kdot(c, K, l));
                acc += (c->jxy[b] / 2.0) * ph * sqrt(Nak[col - 1] / Nak[row - 1]) * phi[col - 1];
                *terms += 1;
            }
        }
    }
    if (c->h) {
        double e = 0.0;
        for (int i = 1; i <= c->N; ++i) {
            int f;
            f = contains(n, c->nd, i);
            e += f ? 0.5 * c->h[i - 1] : -0.5 * c->h[i - 1];
        }
        acc += e * phi[row - 1];
    }
    return acc;
}

/* Alg. 9: psi = H phi in sector K (complex interleaved vectors of length d) */
int orc_hphi_k(ORC_LAT, const int *K, const uint64_t *sigma, const double *Nak, int64_t d,
               const double *phi, double *psi)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    const zdbl *p = (const zdbl *)phi;
    zdbl *q = (zdbl *)psi;
    int64_t terms = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : terms)
    for (int64_t row = 1; row <= d; ++row) q[row - 1] = hphi_k_row(&c, K, sigma, Nak, d, row, p, &terms);
    ctx_free(&c);
    return 0;
}

int orc_hphi_k_rows(ORC_LAT, const int *K, const uint64_t *sigma, const double *Nak, int64_t d,
                    const double *phi, int64_t nrows, const int64_t *rows, double *psi_rows, int64_t *nterms)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    const zdbl *p = (const zdbl *)phi;
    zdbl *q = (zdbl *)psi_rows;
    int64_t terms = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : terms)
    for (int64_t i = 0; i < nrows; ++i) q[i] = hphi_k_row(&c, K, sigma, Nak, d, rows[i] + 1, p, &terms);
    if (nterms) *nterms = terms;
    ctx_free(&c);
    return 0;
}

/* Alg. 8: dense symmetry-adapted block (row-major d x d complex) */
int orc_dense_k(ORC_LAT, const int *K, const uint64_t *sigma, const double *Nak, int64_t d, double *Hout)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    zdbl *H = (zdbl *)Hout;
    memset(H, 0, sizeof(zdbl) * d * d);
    for (int64_t row = 1; row <= d; ++row) {
        int n[ORC_MAXND], np[ORC_MAXND];
        f_bar(&c, sigma[row - 1], n, NULL);
        for (int b = 0; b < nb; ++b) {
            int f, fp;
            f = contains(n, nd, r[b]);
            fp = contains(n, nd, rp[b]);
            if (f == fp) {
                H[(row - 1) * d + (row - 1)] += jz[b] / 4.0;
            } else {
                H[(row - 1) * d + (row - 1)] -= jz[b] / 4.0;
                hop_target(nd, n, r[b], rp[b], np);
                uint64_t ap = F(&c, np);
                int l[3];
                uint64_t rep = representative(&c, ap, l);
                int found;
                int64_t col = binary_search_u64(rep, sigma, 1, d, &found);
                if (found)
                    H[(row - 1) * d + (col - 1)] +=
                        (jxy[b] / 2.0) * cexp(I * kdot(&c, K, l)) * sqrt(Nak[col - 1] / Nak[row - 1]);
            }
        }
        if (h) {
            double e = 0.0;
            for (int i = 1; i <= N; ++i) {
                int f;
                f = contains(n, nd, i);
                e += f ? 0.5 * h[i - 1] : -0.5 * h[i - 1];
            }
            H[(row - 1) * d + (row - 1)] += e;
        }
    }
    ctx_free(&c);
    return 0;
}

/* Alg. 11 (push form, reading R1): psi2 = S^-_q phi, from sector (nd, K) to
 * sector (nd+1, K+Q).  Q is the wave vector in units of 2 pi / L_alpha
 * (integers), pos are the 3 N site positions r used in e^{-i q.r} (NULL:
 * the lattice coordinates), so that q.r = 2 pi sum_alpha Q_alpha r_alpha / L_alpha. */
int orc_smq(ORC_LAT, const int *K, const uint64_t *sigma, const double *Nak, int64_t d,
            const double *phi, const int *Q, const double *pos,
            const uint64_t *sigma2, const double *Nak2, int64_t d2, double *psi2)
{
    orc_ctx c, c2;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1; }
    if (ctx_init(&c2, N, nd + 1, nb, r, rp, jxy, jz, h, L)) { ctx_free(&c); ctx_free(&c2); return -1; }
    const zdbl *p = (const zdbl *)phi;
    zdbl *q = (zdbl *)psi2;
    memset(q, 0, sizeof(zdbl) * d2);
    int K2[3] = {K[0] + Q[0], K[1] + Q[1], K[2] + Q[2]};
    for (int rr = 1; rr <= N; ++rr) {
        int sb, x, y, z;
        site_xyz(&c, rr, &sb, &x, &y, &z);
        double qr;
        if (pos) {
            qr = 2.0 * M_PI * (Q[0] * pos[3 * (rr - 1)] / L[0] + Q[1] * pos[3 * (rr - 1) + 1] / L[1] +
                               Q[2] * pos[3 * (rr - 1) + 2] / L[2]);
        } else {
            int t[3] = {x, y, z};
            qr = kdot(&c, Q, t);
        }
        for (int64_t row = 1; row <= d; ++row) {
            int n[ORC_MAXND], np[ORC_MAXND];
            f_bar(&c, sigma[row - 1], n, NULL);
            int f;
            int pidx = binary_search_int(rr, n, 1, nd, &f);
            if (f) continue;
            int k = 0;
            for (int i = 1; i <= pidx; ++i) np[k++] = n[i - 1];
            np[k++] = rr;
            for (int i = pidx + 1; i <= nd; ++i) np[k++] = n[i - 1];
            uint64_t b = F(&c2, np);
            int l[3];
            uint64_t repb = representative(&c2, b, l);
            int found;
            int64_t col = binary_search_u64(repb, sigma2, 1, d2, &found);
            if (!found) continue;
            double ph = -(qr + kdot(&c, K2, l));
            q[col - 1] += sqrt(Nak2[col - 1] / (Nak[row - 1] * N)) * cexp(I * ph) * p[row - 1];
        }
    }
    ctx_free(&c);
    ctx_free(&c2);
    return 0;
}

/* Two-point functions of a U(1) vector (complex, length C(N,nd)):
 * szsz[i*N+j] = <s^z_i s^z_j>, spsm[(i*N+j)] (complex) = <s^+_i s^-_j>,
 * sz[i] = <s^z_i>; sites 0-based in the output arrays.  Definition of
 * L916-style local operators applied directly in the unsymmetrised basis. */
int orc_corr_u1(int N, int nd, const double *phi, double *szsz, double *spsm, double *sz)
{
    orc_ctx c;
    if (ctx_init(&c, N, nd, 0, NULL, NULL, NULL, NULL, NULL, NULL)) { ctx_free(&c); return -1; }
    uint64_t D = Cb(&c, N, nd);
    const zdbl *p = (const zdbl *)phi;
    zdbl *pm = (zdbl *)spsm;
    memset(szsz, 0, sizeof(double) * N * N);
    memset(pm, 0, sizeof(zdbl) * N * N);
    memset(sz, 0, sizeof(double) * N);
    double *szv = (double *)malloc(sizeof(double) * N);
    for (uint64_t a = 1; a <= D; ++a) {
        int n[ORC_MAXND], np[ORC_MAXND];
        f_bar(&c, a, n, NULL);
        double w = creal(p[a - 1] * conj(p[a - 1]));
        for (int i = 1; i <= N; ++i) {
            int f;
            f = contains(n, nd, i);
            szv[i - 1] = f ? -0.5 : 0.5;
        }
        for (int i = 0; i < N; ++i) {
            sz[i] += w * szv[i];
            for (int j = 0; j < N; ++j) szsz[i * N + j] += w * szv[i] * szv[j];
            /* s^+_i s^-_i is the projector on spin up at i */
            if (szv[i] > 0) pm[i * N + i] += w;
        }
        /* s^+_i s^-_j |a> for i in n, j not in n: i leaves, j enters */
        for (int m = 0; m < nd; ++m) {
            int i = n[m];
            for (int j = 1; j <= N; ++j) {
                if (szv[j - 1] < 0) continue;
                int k = 0;
                for (int u = 0; u < nd; ++u) if (u != m) np[k++] = n[u];
                np[k++] = j;
                insertion_sort(np, nd);
                uint64_t ap = F(&c, np);
                pm[(i - 1) * N + (j - 1)] += conj(p[ap - 1]) * p[a - 1];
            }
        }
    }
    free(szv);
    ctx_free(&c);
    return 0;
}

/* One row of Alg. 9 for the representative with 1-based index a, without a
 * precomputed representative list: the representative of every hop target
 * comes from Alg. 7 and its normalisation factor (zero when incompatible)
 * from Alg. 5.  Writes up to max_terms off-diagonal terms (target
 * representative index, 1-based, and complex coefficient) and the diagonal
 * element (bonds plus site field); returns the number of terms, or -1 when a
 * is not a representative compatible with K.  For sampled rows of sectors
 * too large for Alg. 6. */
int64_t orc_row_terms_k(ORC_LAT, const int *K, uint64_t a, int64_t max_terms, uint64_t *targets, double *coef,
                        double *diag)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -2; }
    const double Na = check_state(&c, a, K);
    if (!(Na > 1e-8)) { ctx_free(&c); return -1; }
    int n[ORC_MAXND], np[ORC_MAXND];
    f_bar(&c, a, n, NULL);
    double dg = 0.0;
    int64_t nt = 0;
    zdbl *cf = (zdbl *)coef;
    for (int b = 0; b < nb; ++b) {
        int f, fp;
        f = contains(n, nd, r[b]);
        fp = contains(n, nd, rp[b]);
        if (f == fp) {
            dg += jz[b] / 4.0;
        } else {
            dg -= jz[b] / 4.0;
            hop_target(nd, n, r[b], rp[b], np);
            uint64_t ap = F(&c, np);
            int l[3];
            uint64_t rep = representative(&c, ap, l);
            const double Nr = check_state(&c, rep, K);
            if (Nr > 1e-8 && nt < max_terms) {
                targets[nt] = rep;
                cf[nt] = (jxy[b] / 2.0) * cexp(I * kdot(&c, K, l)) * sqrt(Nr / Na);
                ++nt;
            }
        }
    }
    if (h) {
        for (int i = 1; i <= N; ++i) {
            int f;
            f = contains(n, nd, i);
            dg += f ? 0.5 * h[i - 1] : -0.5 * h[i - 1];
        }
    }
    *diag = dg;
    ctx_free(&c);
    return nt;
}

/* N_{a,k} of Alg. 5 for the 1-based index a (0 when a is not the
 * representative of its orbit or not compatible with K) */
double orc_check_state(ORC_LAT, const int *K, uint64_t a)
{
    orc_ctx c;
    if (ctx_init(&c, ORC_LAT_ARGS)) { ctx_free(&c); return -1.0; }
    const double v = check_state(&c, a, K);
    ctx_free(&c);
    return v;
}
