/*
 * fci_oracle.c -- plain, slow, determinant-by-determinant configuration interaction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header or table with the
 * CUDA path and follows the textbook definition of the problem the paper solves
 * ("Methods", Eqs. sigmaL/sigmaL1e/sigmaL2e define sigma = H C for
 *  H = sum_PQ h_PQ a+_P a_Q + 1/2 sum_PQRS (PQ|RS) a+_P a+_R a_S a_Q ).
 *
 * Everything is written over spin orbitals (or spinors) with complex arithmetic; the
 * real spin-free case is the special case with zero imaginary parts and integrals that
 * vanish between different spins.  A determinant is a bit mask over at most 64 spin
 * orbitals, meaning a+_{P1} a+_{P2} ... a+_{Pk} |0> with P1 < P2 < ... < Pk.
 * Fermion signs are obtained by applying one operator at a time and counting the
 * occupied spin orbitals it has to pass (Jordan-Wigner ordering); no closed-form
 * phase formula is used anywhere.
 *
 * Matrix elements follow the Slater-Condon rules:
 *   <I|H|I>  = sum_P h_PP + 1/2 sum_{P,R in I} [(PP|RR) - (PR|RP)]
 *   single   = sgn * [h_PQ + sum_{R in J, R != Q} ((PQ|RR) - (PR|RQ))]
 *   double   = sgn * [(PQ|RS) - (PS|RQ)],  sgn = <I| a+_P a+_R a_S a_Q |J>
 * sigma_I = sum_J H_IJ C_J runs over J = I and every single and double replacement of
 * I that lies in the given determinant list (so a list that is a subset of the full
 * space gives P H P, the projected Hamiltonian).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} cplx;

static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx csub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
static inline cplx cmul(cplx a, cplx b) {
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}
static inline cplx cscale(cplx a, double s) { cplx r = {a.re * s, a.im * s}; return r; }

static inline int popcount64(uint64_t x) { return __builtin_popcountll(x); }

/* Annihilate spin orbital p in *m.  Returns 0 if p is empty, else the sign (+1/-1). */
static int op_annihilate(uint64_t *m, int p) {
    uint64_t bit = (uint64_t)1 << p;
    if (!(*m & bit)) return 0;
    int below = popcount64(*m & (bit - 1));
    *m &= ~bit;
    return (below & 1) ? -1 : 1;
}

/* Create spin orbital p in *m.  Returns 0 if p is occupied, else the sign. */
static int op_create(uint64_t *m, int p) {
    uint64_t bit = (uint64_t)1 << p;
    if (*m & bit) return 0;
    int below = popcount64(*m & (bit - 1));
    *m |= bit;
    return (below & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------ strings */

/* All masks of m bits with ne bits set, ascending as integers, by scanning every mask.
 * Returns the count.  out may be NULL (count only). */
int64_t orc_enumerate_strings(int m, int ne, uint64_t *out) {
    if (m < 0 || m > 30 || ne < 0 || ne > m) return -1;
    int64_t k = 0;
    uint64_t lim = (uint64_t)1 << m;
    for (uint64_t x = 0; x < lim; ++x) {
        if (popcount64(x) == ne) {
            if (out) out[k] = x;
            ++k;
        }
    }
    return k;
}

static int64_t bsearch_u64(const uint64_t *a, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] == key) return mid;
        if (a[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Single-replacement list of every string S of a sorted string list (the one-electron
 * excitation list of the paper's Introduction, n_e (n_h + 1) entries per string).
 * For S, entries run over occupied a ascending, then over b ascending among the empty
 * orbitals of S together with b = a.  Each entry is T = S - a + b together with
 * <S| a+_a a_b |T>, evaluated by applying a_b and then a+_a to T.
 * Outputs (n_str * n_ent each): target index of T, a, b, sign.  Returns n_ent or -1. */
int orc_replacement_table(int m, int ne, const uint64_t *strings, int64_t n_str,
                          int32_t *target, int32_t *a_out, int32_t *b_out, int8_t *sign) {
    int n_ent = ne * (m - ne + 1);
    for (int64_t i = 0; i < n_str; ++i) {
        uint64_t S = strings[i];
        int e = 0;
        for (int a = 0; a < m; ++a) {
            if (!((S >> a) & 1)) continue;
            for (int b = 0; b < m; ++b) {
                if (b != a && ((S >> b) & 1)) continue;
                uint64_t T = (S & ~((uint64_t)1 << a)) | ((uint64_t)1 << b);
                uint64_t w = T;
                int s1 = op_annihilate(&w, b);
                int s2 = op_create(&w, a);
                if (s1 == 0 || s2 == 0 || w != S) return -1;
                int64_t t = bsearch_u64(strings, n_str, T);
                if (t < 0) return -1;
                int64_t o = i * n_ent + e;
                target[o] = (int32_t)t;
                a_out[o] = a;
                b_out[o] = b;
                sign[o] = (int8_t)(s1 * s2);
                ++e;
            }
        }
        if (e != n_ent) return -1;
    }
    return n_ent;
}

/* ------------------------------------------------------------- hamiltonian */

typedef struct {
    int nso;
    const cplx *h;  /* nso x nso */
    const cplx *g;  /* nso^4, (PQ|RS) at ((P*nso+Q)*nso+R)*nso+S */
} ham_t;

static inline cplx G(const ham_t *H, int P, int Q, int R, int S) {
    int n = H->nso;
    return H->g[(((size_t)P * n + Q) * n + R) * n + S];
}

static cplx h_diag(const ham_t *H, uint64_t I) {
    cplx e = {0.0, 0.0};
    int n = H->nso;
    for (int P = 0; P < n; ++P) {
        if (!((I >> P) & 1)) continue;
        e = cadd(e, H->h[P * n + P]);
        for (int R = 0; R < n; ++R) {
            if (!((I >> R) & 1)) continue;
            cplx t = csub(G(H, P, P, R, R), G(H, P, R, R, P));
            e = cadd(e, cscale(t, 0.5));
        }
    }
    return e;
}

/* <I|H|J> for two determinants over the same spin-orbital set. */
static cplx h_elem(const ham_t *H, uint64_t I, uint64_t J) {
    cplx zero = {0.0, 0.0};
    uint64_t diff = I ^ J;
    int nd = popcount64(diff);
    if (popcount64(I) != popcount64(J)) return zero;
    if (nd == 0) return h_diag(H, I);
    int n = H->nso;
    if (nd == 2) {
        int P = __builtin_ctzll(I & diff);
        int Q = __builtin_ctzll(J & diff);
        uint64_t w = J;
        int s = op_annihilate(&w, Q);
        s *= op_create(&w, P);
        if (s == 0 || w != I) return zero;
        cplx e = H->h[P * n + Q];
        for (int R = 0; R < n; ++R) {
            if (R == Q || !((J >> R) & 1)) continue;
            e = cadd(e, csub(G(H, P, Q, R, R), G(H, P, R, R, Q)));
        }
        return cscale(e, (double)s);
    }
    if (nd == 4) {
        uint64_t ip = I & diff, jp = J & diff;
        int P = __builtin_ctzll(ip);
        int R = __builtin_ctzll(ip & (ip - 1));
        int Q = __builtin_ctzll(jp);
        int S = __builtin_ctzll(jp & (jp - 1));
        /* sgn = <I| a+_P a+_R a_S a_Q |J>: rightmost operator acts first */
        uint64_t w = J;
        int s = op_annihilate(&w, Q);
        s *= op_annihilate(&w, S);
        s *= op_create(&w, R);
        s *= op_create(&w, P);
        if (s == 0 || w != I) return zero;
        cplx e = csub(G(H, P, Q, R, S), G(H, P, S, R, Q));
        return cscale(e, (double)s);
    }
    return zero;
}

/* ------------------------------------------------------------- lookup table */

typedef struct {
    uint64_t *keys;
    int64_t *vals;
    uint64_t mask;
} lut_t;

static inline uint64_t mix64(uint64_t z) {
    z ^= z >> 33; z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33; z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}

static int lut_build(lut_t *t, const uint64_t *dets, int64_t n) {
    uint64_t cap = 1;
    while (cap < (uint64_t)(2 * n + 2)) cap <<= 1;
    t->keys = (uint64_t *)malloc(cap * sizeof(uint64_t));
    t->vals = (int64_t *)malloc(cap * sizeof(int64_t));
    if (!t->keys || !t->vals) { free(t->keys); free(t->vals); return -1; }
    t->mask = cap - 1;
    for (uint64_t i = 0; i < cap; ++i) t->vals[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = dets[i], p = mix64(k) & t->mask;
        while (t->vals[p] >= 0) {
            if (t->keys[p] == k) return -2; /* duplicate determinant */
            p = (p + 1) & t->mask;
        }
        t->keys[p] = k;
        t->vals[p] = i;
    }
    return 0;
}

static inline int64_t lut_find(const lut_t *t, uint64_t k) {
    uint64_t p = mix64(k) & t->mask;
    while (t->vals[p] >= 0) {
        if (t->keys[p] == k) return t->vals[p];
        p = (p + 1) & t->mask;
    }
    return -1;
}

static void lut_free(lut_t *t) { free(t->keys); free(t->vals); }

/* -------------------------------------------------------------- public API */

/* H_II for every determinant.  h, g: interleaved complex.  diag: interleaved complex. */
int orc_diag(int nso, const double *h, const double *g, int64_t ndet, const uint64_t *dets,
             double *diag) {
    ham_t H = {nso, (const cplx *)h, (const cplx *)g};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ndet; ++i) {
        cplx e = h_diag(&H, dets[i]);
        diag[2 * i] = e.re;
        diag[2 * i + 1] = e.im;
    }
    return 0;
}

/* One matrix element <I|H|J>. */
int orc_hij(int nso, const double *h, const double *g, uint64_t I, uint64_t J, double *out) {
    ham_t H = {nso, (const cplx *)h, (const cplx *)g};
    cplx e = h_elem(&H, I, J);
    out[0] = e.re;
    out[1] = e.im;
    return 0;
}

/* Dense H (row-major ndet x ndet, interleaved complex) for tiny determinant lists. */
int orc_dense_h(int nso, const double *h, const double *g, int64_t ndet, const uint64_t *dets,
                double *Hout) {
    ham_t H = {nso, (const cplx *)h, (const cplx *)g};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < ndet; ++i) {
        for (int64_t j = 0; j < ndet; ++j) {
            cplx e = h_elem(&H, dets[i], dets[j]);
            Hout[2 * (i * ndet + j)] = e.re;
            Hout[2 * (i * ndet + j) + 1] = e.im;
        }
    }
    return 0;
}

/* sigma_I = e_core C_I + sum_J H_IJ C_J for the rows listed in `rows` (all rows when
 * rows == NULL, in which case nrows must equal ndet).  sigma has nrows entries,
 * in the order of `rows`.  C and sigma are interleaved complex.
 * J runs over I itself and all single and double replacements of I (every pair of
 * occupied spin orbitals replaced by every pair of empty ones) that are present in
 * the determinant list, found through the lookup table `lut` of that list. */
static int sigma_rows(const lut_t *lut, int nso, const double *h, const double *g, double e_core, int64_t ndet,
                      const uint64_t *dets, const double *Cin, const int64_t *rows, int64_t nrows, double *sigma) {
    ham_t H = {nso, (const cplx *)h, (const cplx *)g};
    const cplx *C = (const cplx *)Cin;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows ? rows[r] : r;
        if (i < 0 || i >= ndet) { bad = 1; continue; }
        uint64_t I = dets[i];
        int occ[64], vir[64], no = 0, nv = 0;
        for (int P = 0; P < nso; ++P) {
            if ((I >> P) & 1) occ[no++] = P; else vir[nv++] = P;
        }
        cplx acc = cscale(C[i], e_core);
        acc = cadd(acc, cmul(h_diag(&H, I), C[i]));
        /* singles */
        for (int a = 0; a < no; ++a) {
            for (int v = 0; v < nv; ++v) {
                uint64_t J = (I & ~((uint64_t)1 << occ[a])) | ((uint64_t)1 << vir[v]);
                int64_t j = lut_find(lut, J);
                if (j < 0) continue;
                acc = cadd(acc, cmul(h_elem(&H, I, J), C[j]));
            }
        }
        /* doubles */
        for (int a = 0; a < no; ++a) {
            for (int b = a + 1; b < no; ++b) {
                uint64_t I2 = I & ~((uint64_t)1 << occ[a]) & ~((uint64_t)1 << occ[b]);
                for (int v = 0; v < nv; ++v) {
                    for (int w = v + 1; w < nv; ++w) {
                        uint64_t J = I2 | ((uint64_t)1 << vir[v]) | ((uint64_t)1 << vir[w]);
                        int64_t j = lut_find(lut, J);
                        if (j < 0) continue;
                        acc = cadd(acc, cmul(h_elem(&H, I, J), C[j]));
                    }
                }
            }
        }
        sigma[2 * r] = acc.re;
        sigma[2 * r + 1] = acc.im;
    }
    return bad ? -3 : 0;
}

/* sigma over a determinant list (see sigma_rows), with a lookup table built for this
 * call. */
int orc_sigma(int nso, const double *h, const double *g, double e_core, int64_t ndet,
              const uint64_t *dets, const double *Cin, const int64_t *rows, int64_t nrows,
              double *sigma) {
    lut_t lut;
    int rc = lut_build(&lut, dets, ndet);
    if (rc != 0) return rc;
    rc = sigma_rows(&lut, nso, h, g, e_core, ndet, dets, Cin, rows, nrows, sigma);
    lut_free(&lut);
    return rc;
}

/* The lookup table of a determinant list, built once for many orc_sigma_table calls on
 * the same list (NULL on failure or duplicate determinants). */
void *orc_table_new(int64_t ndet, const uint64_t *dets) {
    lut_t *t = (lut_t *)malloc(sizeof(lut_t));
    if (!t) return NULL;
    if (lut_build(t, dets, ndet) != 0) { free(t); return NULL; }
    return t;
}

void orc_table_free(void *t) {
    if (!t) return;
    lut_free((lut_t *)t);
    free(t);
}

/* orc_sigma with a table from orc_table_new for the same determinant list. */
int orc_sigma_table(const void *t, int nso, const double *h, const double *g, double e_core, int64_t ndet,
                    const uint64_t *dets, const double *Cin, const int64_t *rows, int64_t nrows,
                    double *sigma) {
    if (!t) return -1;
    return sigma_rows((const lut_t *)t, nso, h, g, e_core, ndet, dets, Cin, rows, nrows, sigma);
}

/* Number of threads OpenMP will use (for reporting the CPU baseline's core count). */
int orc_num_threads(void) {
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
