/* CPU reference for the point-sink determinant algorithm (test infrastructure
 * only: the tests, the smoke check and the benchmark's CPU-baseline leg use it;
 * the GPU product path never does).  Plain FP64 C, OpenMP over sites.
 *
 * Eq. 2.9 of Sec. III.A, with the sink and source coefficient tables
 * antisymmetrised within each flavour (Sec. III.C, method A):
 *     G(t) = sum_x sum_{M, M'} C[M] C'[M'] det M^u(x; M_u, M'_u) det M^d(x; M_d, M'_d)
 *     M^f_ij = S_f(x, t)(chi_i, chi'_j)   (sink index chi_i, source index chi'_j)
 * The caller lists the distinct (row set, column set) pairs of each flavour and,
 * per (M, M'), the pair indices and the weight C[M] C'[M']; each determinant
 * of a site is evaluated once (memoisation) by its definition, the Leibniz sum
 * over permutations.  Sums are Neumaier-compensated; the sum over sites is
 * taken per thread and the thread sums are added in a fixed order.
 *
 * Three-point functions (Sec. "Three-point functions", Eq. Proton3pt_seq,
 * generalised to nuclei): the current on flavour f through a sequential
 * propagator Sig replaces, in every Wick term, one f-quark line by Sig, summed
 * over the lines -- each f determinant becomes the sum over its rows of the
 * determinant with that row taken from Sig.
 *
 * Also: determinants modulo p = 2^61 - 1 of a random integer matrix (the
 * identity testing of App. C applied to determinants, Sec. III.B).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* permutations of 0..n-1 (lexicographic) with their signs */
static int det_perms(int n, int8_t **perm, int8_t **sign) {
    int np = 1;
    for (int i = 2; i <= n; ++i) np *= i;
    *perm = (int8_t *)malloc((size_t)np * (n > 0 ? n : 1));
    *sign = (int8_t *)malloc((size_t)np);
    int8_t cur[8];
    for (int i = 0; i < n; ++i) cur[i] = (int8_t)i;
    for (int k = 0; k < np; ++k) {
        memcpy(*perm + (size_t)k * n, cur, (size_t)n);
        int inv = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) inv += cur[i] > cur[j];
        (*sign)[k] = (int8_t)(inv & 1 ? -1 : 1);
        /* next permutation in lexicographic order */
        int i = n - 2;
        while (i >= 0 && cur[i] > cur[i + 1]) --i;
        if (i < 0) break;
        int j = n - 1;
        while (cur[j] < cur[i]) --j;
        int8_t t = cur[i]; cur[i] = cur[j]; cur[j] = t;
        for (int a = i + 1, b = n - 1; a < b; ++a, --b) { t = cur[a]; cur[a] = cur[b]; cur[b] = t; }
    }
    return np;
}

/* det of S[rows][cols] (S a 12 x 12 complex matrix, row = sink chi, column = source chi') */
static cplx det_leibniz(const cplx *S, const int8_t *rows, const int8_t *cols, int n, const int8_t *perm,
                        const int8_t *sign, int np) {
    double sr = 0, cr = 0, si = 0, ci = 0;  /* Neumaier sums of both parts */
    for (int k = 0; k < np; ++k) {
        cplx p = sign[k];
        for (int i = 0; i < n; ++i) p *= S[rows[i] * 12 + cols[perm[(size_t)k * n + i]]];
        double v[2] = {creal(p), cimag(p)};
        double *acc[2] = {&sr, &si}, *cmp[2] = {&cr, &ci};
        for (int q = 0; q < 2; ++q) {
            double t = *acc[q] + v[q];
            if (fabs(*acc[q]) >= fabs(v[q])) *cmp[q] += (*acc[q] - t) + v[q];
            else *cmp[q] += (v[q] - t) + *acc[q];
            *acc[q] = t;
        }
    }
    return (sr + cr) + I * (si + ci);
}

/* derivative of det S[rows][cols] in the direction Sig (Jacobi's formula written as a sum over the row
 * replaced): sum_i det(S with row i taken from Sig), each by the Leibniz sum */
static cplx det_leibniz_deriv(const cplx *S, const cplx *Sig, const int8_t *rows, const int8_t *cols, int n,
                              const int8_t *perm, const int8_t *sign, int np) {
    double sr = 0, cr = 0, si = 0, ci = 0;
    for (int k = 0; k < np; ++k)
        for (int rep = 0; rep < n; ++rep) {
            cplx p = sign[k];
            for (int i = 0; i < n; ++i) p *= (i == rep ? Sig : S)[rows[i] * 12 + cols[perm[(size_t)k * n + i]]];
            double v[2] = {creal(p), cimag(p)};
            double *acc[2] = {&sr, &si}, *cmp[2] = {&cr, &ci};
            for (int q = 0; q < 2; ++q) {
                double t = *acc[q] + v[q];
                if (fabs(*acc[q]) >= fabs(v[q])) *cmp[q] += (*acc[q] - t) + v[q];
                else *cmp[q] += (v[q] - t) + *acc[q];
                *acc[q] = t;
            }
        }
    return (sr + cr) + I * (si + ci);
}

static void neumaier(double *s, double *c, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

/* S_f[slice][x][a][alpha][b][beta] complex128 (interleaved doubles); out[slice] complex. */
static int point_sum(const double *Su, const double *Sd, const double *Sig, int sig_flavour, int V, int n_slices,
                     int n_u, int n_d, int64_t n_pu, const int8_t *pu_rows, const int8_t *pu_cols, int64_t n_pd,
                     const int8_t *pd_rows, const int8_t *pd_cols, int64_t n_terms, const int64_t *t_pu,
                     const int64_t *t_pd, const double *t_w, double *out);

int oracle_point_correlator(const double *Su, const double *Sd, int V, int n_slices, int n_u, int n_d,
                            int64_t n_pu, const int8_t *pu_rows, const int8_t *pu_cols, int64_t n_pd,
                            const int8_t *pd_rows, const int8_t *pd_cols, int64_t n_terms, const int64_t *t_pu,
                            const int64_t *t_pd, const double *t_w, double *out) {
    return point_sum(Su, Sd, NULL, -1, V, n_slices, n_u, n_d, n_pu, pu_rows, pu_cols, n_pd, pd_rows, pd_cols,
                     n_terms, t_pu, t_pd, t_w, out);
}

/* Three-point function with the current on flavour sig_flavour (0 = u, 1 = d) through the sequential
 * propagator Sig (same layout as S): every determinant of that flavour becomes the sum over the row
 * whose propagator line is replaced by Sig (the derivative of Eq. 2.9 in the direction Sig). */
int oracle_point_3pt(const double *Su, const double *Sd, const double *Sig, int sig_flavour, int V, int n_slices,
                     int n_u, int n_d, int64_t n_pu, const int8_t *pu_rows, const int8_t *pu_cols, int64_t n_pd,
                     const int8_t *pd_rows, const int8_t *pd_cols, int64_t n_terms, const int64_t *t_pu,
                     const int64_t *t_pd, const double *t_w, double *out) {
    if (!Sig || (sig_flavour != 0 && sig_flavour != 1)) return -1;
    return point_sum(Su, Sd, Sig, sig_flavour, V, n_slices, n_u, n_d, n_pu, pu_rows, pu_cols, n_pd, pd_rows,
                     pd_cols, n_terms, t_pu, t_pd, t_w, out);
}

static int point_sum(const double *Su, const double *Sd, const double *Sig, int sig_flavour, int V, int n_slices,
                     int n_u, int n_d, int64_t n_pu, const int8_t *pu_rows, const int8_t *pu_cols, int64_t n_pd,
                     const int8_t *pd_rows, const int8_t *pd_cols, int64_t n_terms, const int64_t *t_pu,
                     const int64_t *t_pd, const double *t_w, double *out) {
    if (n_u < 0 || n_u > 7 || n_d < 0 || n_d > 7) return -1;
    int8_t *pmu, *smu, *pmd, *smd;
    const int npu = det_perms(n_u, &pmu, &smu), npd = det_perms(n_d, &pmd, &smd);
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *part = (double *)calloc((size_t)nth * 4, sizeof(double));
    for (int sl = 0; sl < n_slices; ++sl) {
        memset(part, 0, sizeof(double) * 4 * (size_t)nth);
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            cplx *U = (cplx *)malloc(sizeof(cplx) * (size_t)(n_pu > 0 ? n_pu : 1));
            cplx *Dt = (cplx *)malloc(sizeof(cplx) * (size_t)(n_pd > 0 ? n_pd : 1));
            double sr = 0, cr = 0, si = 0, ci = 0;
#pragma omp for schedule(static)
            for (int x = 0; x < V; ++x) {
                const cplx *su = (const cplx *)(Su + ((size_t)sl * V + x) * 288);
                const cplx *sd = (const cplx *)(Sd + ((size_t)sl * V + x) * 288);
                const cplx *sg = Sig ? (const cplx *)(Sig + ((size_t)sl * V + x) * 288) : NULL;
                for (int64_t k = 0; k < n_pu; ++k)
                    U[k] = sig_flavour == 0
                               ? det_leibniz_deriv(su, sg, pu_rows + k * n_u, pu_cols + k * n_u, n_u, pmu, smu, npu)
                               : det_leibniz(su, pu_rows + k * n_u, pu_cols + k * n_u, n_u, pmu, smu, npu);
                for (int64_t k = 0; k < n_pd; ++k)
                    Dt[k] = sig_flavour == 1
                                ? det_leibniz_deriv(sd, sg, pd_rows + k * n_d, pd_cols + k * n_d, n_d, pmd, smd, npd)
                                : det_leibniz(sd, pd_rows + k * n_d, pd_cols + k * n_d, n_d, pmd, smd, npd);
                for (int64_t t = 0; t < n_terms; ++t) {
                    const cplx v = t_w[t] * U[t_pu[t]] * Dt[t_pd[t]];
                    neumaier(&sr, &cr, creal(v));
                    neumaier(&si, &ci, cimag(v));
                }
            }
            part[4 * tid + 0] = sr; part[4 * tid + 1] = cr;
            part[4 * tid + 2] = si; part[4 * tid + 3] = ci;
            free(U);
            free(Dt);
        }
        double sr = 0, cr = 0, si = 0, ci = 0;
        for (int t = 0; t < nth; ++t) {
            neumaier(&sr, &cr, part[4 * t]);
            neumaier(&sr, &cr, part[4 * t + 1]);
            neumaier(&si, &ci, part[4 * t + 2]);
            neumaier(&si, &ci, part[4 * t + 3]);
        }
        out[2 * sl] = sr + cr;
        out[2 * sl + 1] = si + ci;
    }
    free(part); free(pmu); free(smu); free(pmd); free(smd);
    return 0;
}

/* ---- determinants mod p = 2^61 - 1 ---- */
static const uint64_t P61 = (1ull << 61) - 1;
static uint64_t mulmod61(uint64_t a, uint64_t b) {
    unsigned __int128 z = (unsigned __int128)a * b;
    uint64_t lo = (uint64_t)z & P61, hi = (uint64_t)(z >> 61);
    uint64_t s = lo + hi;
    return s >= P61 ? s - P61 : s;
}

/* M: 12 x 12 entries in [0, p); det of M[rows][cols] for each pair, Leibniz sum mod p */
int oracle_det_modp(const uint64_t *M, int n, int64_t n_pairs, const int8_t *rows, const int8_t *cols,
                    uint64_t *out) {
    if (n < 0 || n > 7) return -1;
    int8_t *perm, *sign;
    const int np = det_perms(n, &perm, &sign);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n_pairs; ++k) {
        uint64_t acc = 0;
        for (int q = 0; q < np; ++q) {
            uint64_t prod = 1;
            for (int i = 0; i < n; ++i) prod = mulmod61(prod, M[rows[k * n + i] * 12 + cols[k * n + perm[(size_t)q * n + i]]]);
            acc = sign[q] > 0 ? (acc + prod) % P61 : (acc + P61 - prod) % P61;
        }
        out[k] = acc;
    }
    free(perm);
    free(sign);
    return 0;
}
