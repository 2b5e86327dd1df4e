/*
 * wick_oracle.c -- plain, slow, FP64 CPU reference for the nuclear two-point
 * correlator of arXiv:2411.08962 (plane-wave sink / block algorithm).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA product library.
 *
 * What it computes, each function citing the passage it follows:
 *
 *   oracle_blocks        single-product baryon blocks
 *                          Bhat_s(c1,c2,c3) = sum_x sum_e w_e S1[x](r1_e,c1) S1[x](r2_e,c2) S2[x](r3_e,c3)
 *                        i.e. the summand of Eq. 2.4/2.5 before its antisymmetrisation,
 *                        summed over sink sites (zero momentum, plane-wave sink, Sec. V.A).
 *   oracle_raw_correlator the plain Wick sum (Eq. 2.6, generalised in App. D):
 *                          C(t) = scale sum_{sink} W sum_{source} C' sum_{sigma_u, sigma_d}
 *                                 sgn(sigma_u) sgn(sigma_d) prod_k Bhat_k(chi'_{sigma(k,1..3)})
 *                        with the fermion sign of each term the parity of the whole quark
 *                        pairing (sink quark (k, slot) -> source position), i.e.
 *                        sgn(sigma_u) sgn(sigma_d) eta with eta the parity of the identity
 *                        flavour pairing (Eq. 2.8); the pairing of every sink quark with the
 *                        source quark listed in the same place counts +1 (the two-term
 *                        proton expression of App. B).
 *   oracle_dedup         the randomised minimal-set search (Sec. III.B "Computation of
 *                        non-redundant minimal set"; App. C): every raw term is
 *                        evaluated as a polynomial at random integer points modulo
 *                        p = 2^61 - 1 using the antisymmetric blocks of Eq. 2.4, equal
 *                        values (up to sign, R.1) are grouped and their integer weights
 *                        summed.  mode 1 replaces the hash by the exact symbolic
 *                        canonical form (sort each block's like-flavour pair with a sign,
 *                        sort the blocks), the "inspection" alternative of Sec. III.B.
 *   oracle_table_correlator  C(t) = scale sum_u w_u prod_k B[id_{u,k}] with the
 *                        antisymmetric blocks B = Bhat(c1,c2,c3) - Bhat(c2,c1,c3) (Eq. 2.4).
 *   oracle_modp_raw / oracle_modp_table  the raw sum and the reduced sum evaluated
 *                        exactly modulo p at a fresh random integer propagator
 *                        (Theorem 1, App. C), used to pin the reduced table.
 *
 * Raw terms of the reduction (method B of Sec. III.C: antisymmetrise the source
 * coefficients first).  A source tuple whose u (or d) indices repeat cancels
 * in the sum over sigma; every other tuple m is a signed reordering of the
 * sorted multiset pair M = (sorted u indices, sorted d indices):
 *   C'(M) = sum_{m -> M} C'_m sgn(sort_u(m)) sgn(sort_d(m)).
 * Nonzero multisets are listed in lexicographic order; the raw terms are
 *   j = ((i_sink * n_M + M) * n_u! + rank(tau_u)) * n_d! + rank(tau_d)
 * where tau assigns sorted index tau(q) to the sink quark of flavour-ordinal q,
 * with coefficient sink_w * eta * C'(M) * sgn(tau_u) * sgn(tau_d).  Summed with
 * the same products this equals the plain sum over source tuples and sigma.
 * A reduced term keeps the raw term of smallest j in its class as
 * representative (its block ids and its sign), its weight is
 * sum_{j in class} c_j * (term_j / term_rep) / 2^A, and terms are listed by
 * increasing representative.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* problem description (mirrors the Python side, plain arrays)               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n_ops;
    const int32_t *op_f1;    /* flavour of slots 1,2 (0 = u, 1 = d); slot 3 is 1 - f1 */
    const int32_t *op_off;   /* n_ops + 1 offsets into ent / ent_w */
    const int8_t *ent;       /* (s, r1, r2, r3) per entry, r = 4*colour + spin */
    const int32_t *ent_w;
    int n_spin, n_chi;
    const int8_t *chi;       /* source indices chi' kept in the block layout */
    int A, n_sink;
    const int8_t *sink_type; /* n_sink x A */
    const int8_t *sink_spin; /* n_sink x A */
    const int64_t *sink_w;
    int n_src;
    const int8_t *src_chi;   /* n_src x 3A */
    const int64_t *src_w;
    const int8_t *src_flav;  /* 3A */
} problem;

enum { OK = 0, EINVAL_ = -1, ENOMEM_ = -2, ECAP_ = -4, EOVF_ = -5 };

/* ------------------------------------------------------------------------- */
/* compensated (Neumaier) summation                                          */
/* ------------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------- */
/* permutations in lexicographic order                                       */
/* ------------------------------------------------------------------------- */
static int64_t fact(int n) { int64_t f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* r-th permutation of 0..n-1 in lexicographic order; sign = (-1)^(inversions).
 * The Lehmer digit d_i counts later entries smaller than perm[i], so the
 * number of inversions is the digit sum. */
static void perm_unrank(int n, int64_t r, int *perm, int *sign) {
    int used[32] = {0};
    int inv = 0;
    for (int i = 0; i < n; ++i) {
        int64_t f = fact(n - 1 - i);
        int d = (int)(r / f);
        r %= f;
        inv += d;
        int cnt = -1;
        for (int v = 0; v < n; ++v) {
            if (!used[v]) { ++cnt; if (cnt == d) { perm[i] = v; used[v] = 1; break; } }
        }
    }
    *sign = (inv & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------------- */
/* raw-term enumeration context                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    const problem *P;
    int nq, nu, nd;
    int ju[32], jd[32];          /* source positions of u / d antiquarks */
    int64_t fu, fd;              /* n_u!, n_d! */
    int *pu, *pd;                /* permutation tables */
    int *su, *sd;                /* their signs */
    int cidx[12];                /* chi' -> index in the block layout, -1 if absent */
    int *fslot;                  /* n_sink x nq: flavour-ordinal of sink quark (k,slot) */
    int *sflav;                  /* n_sink x nq: flavour of sink quark (k,slot) */
    int *eta;                    /* n_sink: parity of the identity flavour pairing */
    int64_t n_raw;               /* sink x source tuples x sigma_u x sigma_d (plain sum) */
    int64_t n_M;                 /* nonzero antisymmetrised source multisets */
    int8_t *Mu, *Md;             /* n_M x nu, n_M x nd: sorted layout indices */
    int64_t *CM;                 /* n_M: C'(M) */
    int64_t n_red;               /* raw terms of the reduction: sink x n_M x n_u! x n_d! */
} ctx;

static void ctx_free(ctx *c) { free(c->pu); free(c->pd); free(c->su); free(c->sd); free(c->fslot); free(c->sflav); free(c->eta); free(c->Mu); free(c->Md); free(c->CM); }

/* ------------------------------------------------------------------------- */
/* antisymmetrised source: sorted multisets with their summed signed weights */
/* ------------------------------------------------------------------------- */
typedef struct { int8_t v[24]; int64_t w; } msrec;
static int ms_len;  /* nu + nd of the records being compared */
static int cmp_ms(const void *a, const void *b) {
    return memcmp(((const msrec *)a)->v, ((const msrec *)b)->v, (size_t)ms_len);
}

/* sort x[0..n) ascending by insertion; return -1 if two entries are equal,
 * else the parity (+1/-1) of the sorting permutation */
static int sort_sign(int8_t *x, int n) {
    int sgn = 1;
    for (int a = 1; a < n; ++a)
        for (int b = a; b > 0 && x[b - 1] >= x[b]; --b) {
            if (x[b - 1] == x[b]) return 0;
            int8_t t = x[b]; x[b] = x[b - 1]; x[b - 1] = t;
            sgn = -sgn;
        }
    for (int a = 1; a < n; ++a) if (x[a - 1] == x[a]) return 0;
    return sgn;
}

static int ms_build(ctx *c) {
    const problem *P = c->P;
    msrec *r = malloc(sizeof(msrec) * (size_t)P->n_src);
    if (!r) return ENOMEM_;
    int64_t n = 0;
    for (int m = 0; m < P->n_src; ++m) {
        msrec x;
        memset(&x, 0, sizeof(x));
        for (int k = 0; k < c->nu; ++k) x.v[k] = (int8_t)c->cidx[(int)P->src_chi[m * c->nq + c->ju[k]]];
        for (int k = 0; k < c->nd; ++k) x.v[c->nu + k] = (int8_t)c->cidx[(int)P->src_chi[m * c->nq + c->jd[k]]];
        const int su = sort_sign(x.v, c->nu), sd = sort_sign(x.v + c->nu, c->nd);
        if (su == 0 || sd == 0) continue;    /* repeated index within a flavour: cancels */
        x.w = P->src_w[m] * su * sd;
        r[n++] = x;
    }
    ms_len = c->nu + c->nd;
    qsort(r, (size_t)n, sizeof(msrec), cmp_ms);
    int64_t k = 0;
    for (int64_t a = 0; a < n; ) {
        int64_t b = a, w = 0;
        while (b < n && memcmp(r[b].v, r[a].v, (size_t)ms_len) == 0) w += r[b++].w;
        if (w != 0) { r[k] = r[a]; r[k].w = w; ++k; }
        a = b;
    }
    c->n_M = k;
    c->Mu = malloc((size_t)(k ? k : 1) * (c->nu ? c->nu : 1));
    c->Md = malloc((size_t)(k ? k : 1) * (c->nd ? c->nd : 1));
    c->CM = malloc(sizeof(int64_t) * (size_t)(k ? k : 1));
    if (!c->Mu || !c->Md || !c->CM) { free(r); return ENOMEM_; }
    for (int64_t q = 0; q < k; ++q) {
        memcpy(c->Mu + q * c->nu, r[q].v, (size_t)c->nu);
        memcpy(c->Md + q * c->nd, r[q].v + c->nu, (size_t)c->nd);
        c->CM[q] = r[q].w;
    }
    c->n_red = (int64_t)P->n_sink * k * c->fu * c->fd;
    free(r);
    return OK;
}

static int ctx_init(ctx *c, const problem *P) {
    memset(c, 0, sizeof(*c));
    c->P = P;
    c->nq = 3 * P->A;
    if (P->A < 1 || P->A > 8 || P->n_sink < 1 || P->n_src < 1) return EINVAL_;
    for (int q = 0; q < c->nq; ++q) {
        if (P->src_flav[q] == 0) c->ju[c->nu++] = q; else c->jd[c->nd++] = q;
    }
    if (c->nu > 12 || c->nd > 12) return EINVAL_;
    c->fu = fact(c->nu); c->fd = fact(c->nd);
    c->pu = malloc(sizeof(int) * (size_t)(c->fu * (c->nu ? c->nu : 1)));
    c->pd = malloc(sizeof(int) * (size_t)(c->fd * (c->nd ? c->nd : 1)));
    c->su = malloc(sizeof(int) * (size_t)c->fu);
    c->sd = malloc(sizeof(int) * (size_t)c->fd);
    c->fslot = malloc(sizeof(int) * (size_t)(P->n_sink * c->nq));
    c->sflav = malloc(sizeof(int) * (size_t)(P->n_sink * c->nq));
    c->eta = malloc(sizeof(int) * (size_t)P->n_sink);
    if (!c->pu || !c->pd || !c->su || !c->sd || !c->fslot || !c->sflav || !c->eta) return ENOMEM_;
    for (int64_t r = 0; r < c->fu; ++r) perm_unrank(c->nu, r, c->pu + r * c->nu, c->su + r);
    for (int64_t r = 0; r < c->fd; ++r) perm_unrank(c->nd, r, c->pd + r * c->nd, c->sd + r);
    for (int i = 0; i < 12; ++i) c->cidx[i] = -1;
    for (int i = 0; i < P->n_chi; ++i) c->cidx[(int)P->chi[i]] = i;
    for (int i = 0; i < P->n_sink; ++i) {
        int mu = 0, md = 0;
        for (int k = 0; k < P->A; ++k) {
            int o = P->sink_type[i * P->A + k];
            if (o < 0 || o >= P->n_ops) return EINVAL_;
            int f1 = P->op_f1[o];
            for (int sl = 0; sl < 3; ++sl) {
                int f = (sl < 2) ? f1 : 1 - f1;
                c->sflav[i * c->nq + 3 * k + sl] = f;
                c->fslot[i * c->nq + 3 * k + sl] = (f == 0) ? mu++ : md++;
            }
        }
        if (mu != c->nu || md != c->nd) return EINVAL_;
        /* eta_i: parity of the pairing q -> source position of the same-flavour
         * quark with the same ordinal (Eq. 2.8's eta); +1 when the source lists
         * the quarks in the sink's flavour order. */
        int pi[32], inv = 0;
        for (int q = 0; q < c->nq; ++q) {
            int f = c->sflav[i * c->nq + q], ord = c->fslot[i * c->nq + q];
            pi[q] = (f == 0) ? c->ju[ord] : c->jd[ord];
        }
        for (int a = 0; a < c->nq; ++a)
            for (int b = a + 1; b < c->nq; ++b) inv += pi[a] > pi[b];
        c->eta[i] = (inv & 1) ? -1 : 1;
    }
    for (int m = 0; m < P->n_src * c->nq; ++m)
        if (P->src_chi[m] < 0 || P->src_chi[m] > 11 || c->cidx[(int)P->src_chi[m]] < 0) return EINVAL_;
    c->n_raw = (int64_t)P->n_sink * P->n_src * c->fu * c->fd;
    return ms_build(c);
}

static inline int blk_id(const problem *P, int o, int s, int i1, int i2, int i3) {
    return (((o * P->n_spin + s) * P->n_chi + i1) * P->n_chi + i2) * P->n_chi + i3;
}

/* Decode term j of the plain sum (sink, source tuple, sigma_u, sigma_d): its
 * integer coefficient and, per nucleon k, the (op, spin, i1, i2, i3) of the
 * block it multiplies. */
static void raw_decode(const ctx *c, int64_t j, int64_t *coef, int *bo, int *bs, int *bi) {
    const problem *P = c->P;
    int64_t rd = j % c->fd; j /= c->fd;
    int64_t ru = j % c->fu; j /= c->fu;
    int64_t m = j % P->n_src;
    int64_t i = j / P->n_src;
    const int *pu = c->pu + ru * c->nu, *pd = c->pd + rd * c->nd;
    for (int k = 0; k < P->A; ++k) {
        bo[k] = P->sink_type[i * P->A + k];
        bs[k] = P->sink_spin[i * P->A + k];
        for (int sl = 0; sl < 3; ++sl) {
            int q = 3 * k + sl;
            int f = c->sflav[i * c->nq + q], ord = c->fslot[i * c->nq + q];
            int pos = (f == 0) ? c->ju[pu[ord]] : c->jd[pd[ord]];
            bi[3 * k + sl] = c->cidx[(int)P->src_chi[m * c->nq + pos]];
        }
    }
    *coef = P->sink_w[i] * P->src_w[m] * c->su[ru] * c->sd[rd] * c->eta[i];
}

/* Decode raw term j of the reduction (sink, multiset M, tau_u, tau_d). */
static void term_decode(const ctx *c, int64_t j, int64_t *coef, int *bo, int *bs, int *bi) {
    const problem *P = c->P;
    int64_t rd = j % c->fd; j /= c->fd;
    int64_t ru = j % c->fu; j /= c->fu;
    int64_t M = j % c->n_M;
    int64_t i = j / c->n_M;
    const int *pu = c->pu + ru * c->nu, *pd = c->pd + rd * c->nd;
    for (int k = 0; k < P->A; ++k) {
        bo[k] = P->sink_type[i * P->A + k];
        bs[k] = P->sink_spin[i * P->A + k];
        for (int sl = 0; sl < 3; ++sl) {
            int q = 3 * k + sl;
            int f = c->sflav[i * c->nq + q], ord = c->fslot[i * c->nq + q];
            bi[3 * k + sl] = (f == 0) ? c->Mu[M * c->nu + pu[ord]] : c->Md[M * c->nd + pd[ord]];
        }
    }
    *coef = P->sink_w[i] * c->CM[M] * c->su[ru] * c->sd[rd] * c->eta[i];
}

/* ------------------------------------------------------------------------- */
/* blocks (Eq. 2.4/2.5 summand, zero-momentum sum over sink sites)           */
/* ------------------------------------------------------------------------- */
/* S arrays: [src][t][x][12 sink chi][12 source chi] complex, interleaved.
 * out:     [src][t][n_blk] complex, n_blk = n_ops * n_spin * n_chi^3. */
int oracle_blocks(const double *Su, const double *Sd, int n_src, int T, int V,
                  const problem *P, double *out) {
    const int nc = P->n_chi, nc3 = nc * nc * nc;
    const int n_blk = P->n_ops * P->n_spin * nc3;
    const int64_t nslice = (int64_t)n_src * T;
    int err = OK;
#pragma omp parallel for collapse(3) schedule(dynamic)
    for (int64_t sl = 0; sl < nslice; ++sl)
        for (int o = 0; o < P->n_ops; ++o)
            for (int s = 0; s < P->n_spin; ++s) {
                nsum *acc = calloc((size_t)nc3 * 2, sizeof(nsum));
                if (!acc) { err = ENOMEM_; continue; }
                const double *S1 = (P->op_f1[o] == 0) ? Su : Sd;
                const double *S2 = (P->op_f1[o] == 0) ? Sd : Su;
                for (int x = 0; x < V; ++x) {
                    const int64_t base = (sl * V + x) * 144;
                    for (int e = P->op_off[o]; e < P->op_off[o + 1]; ++e) {
                        if (P->ent[4 * e] != s) continue;
                        const int r1 = P->ent[4 * e + 1], r2 = P->ent[4 * e + 2], r3 = P->ent[4 * e + 3];
                        const double w = (double)P->ent_w[e];
                        for (int i1 = 0; i1 < nc; ++i1) {
                            const int64_t a1 = 2 * (base + r1 * 12 + P->chi[i1]);
                            cplx v1 = (S1[a1] + I * S1[a1 + 1]) * w;
                            for (int i2 = 0; i2 < nc; ++i2) {
                                const int64_t a2 = 2 * (base + r2 * 12 + P->chi[i2]);
                                cplx v12 = v1 * (S1[a2] + I * S1[a2 + 1]);
                                for (int i3 = 0; i3 < nc; ++i3) {
                                    const int64_t a3 = 2 * (base + r3 * 12 + P->chi[i3]);
                                    cplx v = v12 * (S2[a3] + I * S2[a3 + 1]);
                                    int id = (i1 * nc + i2) * nc + i3;
                                    nadd(&acc[2 * id], creal(v));
                                    nadd(&acc[2 * id + 1], cimag(v));
                                }
                            }
                        }
                    }
                }
                double *dst = out + 2 * (sl * n_blk + (int64_t)(o * P->n_spin + s) * nc3);
                for (int id = 0; id < nc3; ++id) {
                    dst[2 * id] = nval(&acc[2 * id]);
                    dst[2 * id + 1] = nval(&acc[2 * id + 1]);
                }
                free(acc);
            }
    return err;
}

/* ------------------------------------------------------------------------- */
/* plain Wick sum over raw terms with single-product blocks                  */
/* ------------------------------------------------------------------------- */
int oracle_raw_correlator(const problem *P, const double *Bhat, int n_slices, double scale, double *out) {
    ctx c;
    int err = ctx_init(&c, P);
    if (err) { ctx_free(&c); return err; }
    const int n_blk = P->n_ops * P->n_spin * P->n_chi * P->n_chi * P->n_chi;
#pragma omp parallel for schedule(dynamic)
    for (int sl = 0; sl < n_slices; ++sl) {
        const double *B = Bhat + 2 * (int64_t)sl * n_blk;
        nsum re = {0, 0}, im = {0, 0};
        int bo[8], bs[8], bi[24];
        int64_t coef;
        for (int64_t j = 0; j < c.n_raw; ++j) {
            raw_decode(&c, j, &coef, bo, bs, bi);
            cplx prod = (double)coef;
            for (int k = 0; k < P->A; ++k) {
                int id = blk_id(P, bo[k], bs[k], bi[3 * k], bi[3 * k + 1], bi[3 * k + 2]);
                prod *= B[2 * id] + I * B[2 * id + 1];
            }
            nadd(&re, creal(prod));
            nadd(&im, cimag(prod));
        }
        out[2 * sl] = scale * nval(&re);
        out[2 * sl + 1] = scale * nval(&im);
    }
    ctx_free(&c);
    return OK;
}

/* C(t) from a reduced table, antisymmetric blocks built from Bhat (Eq. 2.4). */
int oracle_table_correlator(const problem *P, const double *Bhat, int n_slices, double scale,
                            int64_t U, const uint16_t *ids, const int64_t *w, double *out) {
    const int nc = P->n_chi, n_blk = P->n_ops * P->n_spin * nc * nc * nc;
    const int A = P->A;
#pragma omp parallel for schedule(dynamic)
    for (int sl = 0; sl < n_slices; ++sl) {
        const double *B = Bhat + 2 * (int64_t)sl * n_blk;
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t u = 0; u < U; ++u) {
            cplx prod = (double)w[u];
            for (int k = 0; k < A; ++k) {
                int id = ids[u * A + k];
                int i3 = id % nc, i2 = (id / nc) % nc, i1 = (id / (nc * nc)) % nc, os = id / (nc * nc * nc);
                int sw = (os * nc + i2) * nc * nc + i1 * nc + i3;
                prod *= (B[2 * id] - B[2 * sw]) + I * (B[2 * id + 1] - B[2 * sw + 1]);
            }
            nadd(&re, creal(prod));
            nadd(&im, cimag(prod));
        }
        out[2 * sl] = scale * nval(&re);
        out[2 * sl + 1] = scale * nval(&im);
    }
    return OK;
}

/* ------------------------------------------------------------------------- */
/* exact arithmetic modulo the Mersenne prime p = 2^61 - 1                   */
/* ------------------------------------------------------------------------- */
#define PMOD ((uint64_t)0x1FFFFFFFFFFFFFFFull)
static inline uint64_t mred(unsigned __int128 x) {       /* x < 2^122 */
    uint64_t lo = (uint64_t)(x & PMOD), hi = (uint64_t)(x >> 61);
    uint64_t r = lo + hi;                                 /* 2^61 == 1 (mod p) */
    r = (r & PMOD) + (r >> 61);
    return r >= PMOD ? r - PMOD : r;
}
static inline uint64_t mmul(uint64_t a, uint64_t b) { return mred((unsigned __int128)a * b); }
static inline uint64_t madd(uint64_t a, uint64_t b) { uint64_t r = a + b; return r >= PMOD ? r - PMOD : r; }
static inline uint64_t msub(uint64_t a, uint64_t b) { return a >= b ? a - b : a + PMOD - b; }
static inline uint64_t mfrom(int64_t v) {
    if (v >= 0) return (uint64_t)v % PMOD;
    uint64_t m = (uint64_t)(-(v + 1)) % PMOD;             /* |v| - 1 */
    return msub(PMOD - 1, m);                             /* p - |v| */
}

/* SplitMix64 (Steele, Lea, Flood 2014), counter-based use */
static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t sm_at(uint64_t key, uint64_t i) { return sm_mix(key + (i + 1) * 0x9E3779B97F4A7C15ull); }

/* Block values modulo p at V0 random integer sites: R[id] (antisymmetric,
 * Eq. 2.4) when antisym != 0, else the single product. */
static void modp_blocks(const problem *P, uint64_t seed, int V0, int antisym, uint64_t *R) {
    const int nc = P->n_chi, nc3 = nc * nc * nc;
    uint64_t *S = malloc(sizeof(uint64_t) * 2 * (size_t)V0 * 144);
    for (int f = 0; f < 2; ++f)
        for (int v = 0; v < V0; ++v) {
            uint64_t key = sm_mix(seed ^ sm_mix(0x5151ull + (uint64_t)(f * 1000003 + v)));
            for (int e = 0; e < 144; ++e) {
                uint64_t r = sm_at(key, (uint64_t)e) >> 3;        /* 61 random bits */
                S[((size_t)f * V0 + v) * 144 + e] = (r == PMOD) ? 0 : r;
            }
        }
    for (int o = 0; o < P->n_ops; ++o)
        for (int s = 0; s < P->n_spin; ++s)
            for (int i1 = 0; i1 < nc; ++i1)
                for (int i2 = 0; i2 < nc; ++i2)
                    for (int i3 = 0; i3 < nc; ++i3) {
                        uint64_t acc = 0;
                        const int f1 = P->op_f1[o], f2 = 1 - f1;
                        const int c1 = P->chi[i1], c2 = P->chi[i2], c3 = P->chi[i3];
                        for (int v = 0; v < V0; ++v) {
                            const uint64_t *S1 = S + ((size_t)f1 * V0 + v) * 144;
                            const uint64_t *S2 = S + ((size_t)f2 * V0 + v) * 144;
                            for (int e = P->op_off[o]; e < P->op_off[o + 1]; ++e) {
                                if (P->ent[4 * e] != s) continue;
                                int r1 = P->ent[4 * e + 1], r2 = P->ent[4 * e + 2], r3 = P->ent[4 * e + 3];
                                uint64_t t = mmul(S1[r1 * 12 + c1], S1[r2 * 12 + c2]);
                                if (antisym) t = msub(t, mmul(S1[r1 * 12 + c2], S1[r2 * 12 + c1]));
                                t = mmul(mmul(t, S2[r3 * 12 + c3]), mfrom(P->ent_w[e]));
                                acc = madd(acc, t);
                            }
                        }
                        R[(o * P->n_spin + s) * nc3 + (i1 * nc + i2) * nc + i3] = acc;
                    }
    free(S);
}

/* ------------------------------------------------------------------------- */
/* grouping map: 128-bit key -> (summed weight, smallest raw index)          */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t k0, k1; int64_t W; int64_t rep; } slot_t;
typedef struct { slot_t *s; int64_t cap, n; } map_t;
#define EMPTY_K0 UINT64_MAX

static int map_init(map_t *m, int64_t cap) {
    m->cap = cap; m->n = 0;
    m->s = malloc(sizeof(slot_t) * (size_t)cap);
    if (!m->s) return ENOMEM_;
    for (int64_t i = 0; i < cap; ++i) m->s[i].k0 = EMPTY_K0;
    return OK;
}
static inline uint64_t khash(uint64_t k0, uint64_t k1) { return sm_mix(k0 * 0x9E3779B97F4A7C15ull ^ k1); }
static int map_put(map_t *m, uint64_t k0, uint64_t k1, int64_t W, int64_t rep);
static int map_grow(map_t *m) {
    map_t n2;
    if (map_init(&n2, m->cap * 2)) return ENOMEM_;
    for (int64_t i = 0; i < m->cap; ++i)
        if (m->s[i].k0 != EMPTY_K0) map_put(&n2, m->s[i].k0, m->s[i].k1, m->s[i].W, m->s[i].rep);
    free(m->s);
    *m = n2;
    return OK;
}
static int map_put(map_t *m, uint64_t k0, uint64_t k1, int64_t W, int64_t rep) {
    if (2 * (m->n + 1) > m->cap && map_grow(m)) return ENOMEM_;
    uint64_t h = khash(k0, k1) & (uint64_t)(m->cap - 1);
    for (;;) {
        slot_t *s = &m->s[h];
        if (s->k0 == EMPTY_K0) { s->k0 = k0; s->k1 = k1; s->W = W; s->rep = rep; m->n++; return OK; }
        if (s->k0 == k0 && s->k1 == k1) {
            s->W += W;
            if (rep < s->rep) s->rep = rep;
            return OK;
        }
        h = (h + 1) & (uint64_t)(m->cap - 1);
    }
}

/* canonical key of raw term j: returns 0 for an identically vanishing term */
static int term_key(const ctx *c, int mode, int trials, const uint64_t *R, int n_blk,
                    int64_t j, int64_t *coef, uint64_t *k0, uint64_t *k1, int *eps) {
    const problem *P = c->P;
    int bo[8], bs[8], bi[24];
    term_decode(c, j, coef, bo, bs, bi);
    if (mode == 0) {
        uint64_t h[2] = {1, 1};
        for (int r = 0; r < trials; ++r)
            for (int k = 0; k < P->A; ++k)
                h[r] = mmul(h[r], R[r * n_blk + blk_id(P, bo[k], bs[k], bi[3 * k], bi[3 * k + 1], bi[3 * k + 2])]);
        if (trials == 1) h[1] = 0;
        int first = (h[0] != 0) ? 0 : (h[1] != 0 ? 1 : -1);
        if (first < 0) return 0;
        *eps = 1;
        if (h[first] > (PMOD - 1) / 2) {
            *eps = -1;
            for (int r = 0; r < 2; ++r) h[r] = h[r] ? PMOD - h[r] : 0;
        }
        *k0 = h[0]; *k1 = h[1];
        return 1;
    }
    /* exact symbolic canonical form */
    int sign = 1;
    uint16_t id[8];
    for (int k = 0; k < P->A; ++k) {
        int a = bi[3 * k], b = bi[3 * k + 1];
        if (a == b) return 0;
        if (a > b) { int t = a; a = b; b = t; sign = -sign; }
        id[k] = (uint16_t)blk_id(P, bo[k], bs[k], a, b, bi[3 * k + 2]);
    }
    for (int x = 1; x < P->A; ++x)            /* insertion sort: the product commutes */
        for (int y = x; y > 0 && id[y - 1] > id[y]; --y) { uint16_t t = id[y]; id[y] = id[y - 1]; id[y - 1] = t; }
    uint64_t a0 = 0, a1 = 0;
    for (int k = 0; k < P->A; ++k) {
        if (k < 4) a0 |= (uint64_t)id[k] << (16 * k); else a1 |= (uint64_t)id[k] << (16 * (k - 4));
    }
    *k0 = a0 ^ 0x8000000000000000ull;          /* never equal to EMPTY_K0 */
    *k1 = a1;
    *eps = sign;
    return 1;
}

typedef struct { int64_t rep, w; } outrec;
static int cmp_rep(const void *a, const void *b) {
    int64_t x = ((const outrec *)a)->rep, y = ((const outrec *)b)->rep;
    return (x > y) - (x < y);
}

/* stats: [0] raw terms, [1] identically-zero terms, [2] classes, [3] kept terms */
int oracle_dedup(const problem *P, uint64_t seed, int trials, int V0, int mode, int64_t cap,
                 int64_t *out_rep, int64_t *out_w, uint16_t *out_ids, int64_t *stats) {
    ctx c;
    int err = ctx_init(&c, P);
    if (err) { ctx_free(&c); return err; }
    if (trials < 1 || trials > 2 || V0 < 1) { ctx_free(&c); return EINVAL_; }
    const int nc = P->n_chi, n_blk = P->n_ops * P->n_spin * nc * nc * nc;
    uint64_t *R = malloc(sizeof(uint64_t) * 2 * (size_t)n_blk);
    for (int r = 0; r < trials; ++r) modp_blocks(P, sm_mix(seed + 77ull * (uint64_t)r), V0, 1, R + (size_t)r * n_blk);

    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    map_t *loc = calloc((size_t)nth, sizeof(map_t));
    int64_t *nzero = calloc((size_t)nth, sizeof(int64_t));
    for (int t = 0; t < nth; ++t) map_init(&loc[t], 1 << 12);
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 4096)
        for (int64_t j = 0; j < c.n_red; ++j) {
            int64_t coef; uint64_t k0, k1; int eps;
            if (!term_key(&c, mode, trials, R, n_blk, j, &coef, &k0, &k1, &eps)) { nzero[tid]++; continue; }
            if (map_put(&loc[tid], k0, k1, eps * coef, j)) err = ENOMEM_;
        }
    }
    map_t g;
    map_init(&g, 1 << 12);
    int64_t nz = 0;
    for (int t = 0; t < nth; ++t) {
        nz += nzero[t];
        for (int64_t i = 0; i < loc[t].cap; ++i)
            if (loc[t].s[i].k0 != EMPTY_K0) map_put(&g, loc[t].s[i].k0, loc[t].s[i].k1, loc[t].s[i].W, loc[t].s[i].rep);
        free(loc[t].s);
    }
    free(loc); free(nzero);
    int64_t U = 0;
    outrec *rec = malloc(sizeof(outrec) * (size_t)(g.n ? g.n : 1));
    const int64_t two_a = (int64_t)1 << P->A;
    for (int64_t i = 0; i < g.cap; ++i) {
        if (g.s[i].k0 == EMPTY_K0 || g.s[i].W == 0) continue;
        int64_t coef; uint64_t k0, k1; int eps;
        term_key(&c, mode, trials, R, n_blk, g.s[i].rep, &coef, &k0, &k1, &eps);
        int64_t w = g.s[i].W * eps;
        if (w % two_a != 0) err = EOVF_;   /* cannot happen: classes are unions of pair-swap orbits */
        rec[U].rep = g.s[i].rep;
        rec[U].w = w / two_a;
        ++U;
    }
    qsort(rec, (size_t)U, sizeof(outrec), cmp_rep);
    if (U > cap) err = err ? err : ECAP_;
    for (int64_t u = 0; u < U && u < cap; ++u) {
        int64_t coef; int bo[8], bs[8], bi[24];
        term_decode(&c, rec[u].rep, &coef, bo, bs, bi);
        out_rep[u] = rec[u].rep;
        out_w[u] = rec[u].w;
        for (int k = 0; k < P->A; ++k)
            out_ids[u * P->A + k] = (uint16_t)blk_id(P, bo[k], bs[k], bi[3 * k], bi[3 * k + 1], bi[3 * k + 2]);
    }
    stats[0] = c.n_red; stats[1] = nz; stats[2] = g.n; stats[3] = U;
    free(rec); free(g.s); free(R);
    ctx_free(&c);
    return err;
}

/* Raw Wick sum (single-product blocks) at a random integer propagator, mod p. */
int oracle_modp_raw(const problem *P, uint64_t seed, uint64_t *out) {
    ctx c;
    int err = ctx_init(&c, P);
    if (err) { ctx_free(&c); return err; }
    const int nc = P->n_chi, n_blk = P->n_ops * P->n_spin * nc * nc * nc;
    uint64_t *R = malloc(sizeof(uint64_t) * (size_t)n_blk);
    modp_blocks(P, seed, 1, 0, R);
    uint64_t total = 0;
#pragma omp parallel
    {
        uint64_t part = 0;
#pragma omp for schedule(dynamic, 4096)
        for (int64_t j = 0; j < c.n_raw; ++j) {
            int64_t coef; int bo[8], bs[8], bi[24];
            raw_decode(&c, j, &coef, bo, bs, bi);
            uint64_t v = mfrom(coef);
            for (int k = 0; k < P->A; ++k)
                v = mmul(v, R[blk_id(P, bo[k], bs[k], bi[3 * k], bi[3 * k + 1], bi[3 * k + 2])]);
            part = madd(part, v);
        }
#pragma omp critical
        total = madd(total, part);
    }
    *out = total;
    free(R);
    ctx_free(&c);
    return OK;
}

/* Reduced sum (antisymmetric blocks) at the same kind of point, mod p. */
int oracle_modp_table(const problem *P, uint64_t seed, int64_t U, const uint16_t *ids, const int64_t *w,
                      uint64_t *out) {
    const int nc = P->n_chi, n_blk = P->n_ops * P->n_spin * nc * nc * nc;
    uint64_t *R = malloc(sizeof(uint64_t) * (size_t)n_blk);
    modp_blocks(P, seed, 1, 1, R);
    uint64_t total = 0;
    for (int64_t u = 0; u < U; ++u) {
        uint64_t v = mfrom(w[u]);
        for (int k = 0; k < P->A; ++k) v = mmul(v, R[ids[u * P->A + k]]);
        total = madd(total, v);
    }
    *out = total;
    free(R);
    return OK;
}

/* The antisymmetrised source table: counts[0] = n_M, counts[1] = raw terms
 * of the reduction; Mu/Md/CM filled up to cap entries. */
int oracle_source_multisets(const problem *P, int64_t cap, int8_t *Mu, int8_t *Md, int64_t *CM, int64_t *counts) {
    ctx c;
    int err = ctx_init(&c, P);
    if (err) { ctx_free(&c); return err; }
    counts[0] = c.n_M;
    counts[1] = c.n_red;
    for (int64_t q = 0; q < c.n_M && q < cap; ++q) {
        memcpy(Mu + q * c.nu, c.Mu + q * c.nu, (size_t)c.nu);
        memcpy(Md + q * c.nd, c.Md + q * c.nd, (size_t)c.nd);
        CM[q] = c.CM[q];
    }
    ctx_free(&c);
    return c.n_M > cap ? ECAP_ : OK;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
