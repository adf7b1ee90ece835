/*
 * fbn_oracle.c -- plain, sequential CPU oracle for the PC-stable skeleton with
 * the G^2 conditional-independence test (Fast-BNS, Sections III-B and III-C).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * GPU path is compared against.  It shares no code with the GPU library, and
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It is deliberately slow and literal: one sample at a time, one
 * test at a time, every floating-point step in double precision.
 *
 * Conventions (each is a reading of the paper where it is silent):
 *   - contingency-table layout: counts[(z * r_x + x) * r_y + y], where z is the
 *     mixed-radix index of the conditioning values with S[0] most significant;
 *   - G^2 uses the natural logarithm; cells with N_xyz = 0 contribute 0;
 *   - df = (r_x - 1)(r_y - 1) * prod_{k in S} r_k over declared arities;
 *   - independence is accepted iff p > alpha (strictly);
 *   - at depth d >= 1 the edge i<j first tries every S subset of a(i)\{j} in
 *     lexicographic order, then every S subset of a(j)\{i} (grouping of the two
 *     endpoints, Section IV-C); a subset present on both sides is tried twice;
 *   - at depth 0 each pair gets exactly one marginal test (Section IV-B);
 *   - the separating set is the first accepting S in that order;
 *   - the depth loop stops when no edge of the current snapshot has a side
 *     with at least d candidates, or when d exceeds max_depth (>= 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* Contingency table (Section III-B; generation as described in Section IV-A:
 * visit every sample, find its cell from the values of X, Y and S, add one). */
int64_t oracle_ci_table(const uint8_t* data, int64_t ld, int64_t n_samples,
                        const uint8_t* arities, int32_t x, int32_t y,
                        const int32_t* S, int32_t d, int64_t* counts, int64_t cap)
{
    int64_t cells = (int64_t)arities[x] * arities[y];
    for (int32_t k = 0; k < d; k++) cells *= arities[S[k]];
    if (cells > cap) return ORACLE_EINVAL;
    memset(counts, 0, (size_t)cells * sizeof(int64_t));
    for (int64_t s = 0; s < n_samples; s++) {
        int64_t z = 0;
        for (int32_t k = 0; k < d; k++)
            z = z * arities[S[k]] + data[(int64_t)S[k] * ld + s];
        int64_t cell = (z * arities[x] + data[(int64_t)x * ld + s]) * arities[y]
                       + data[(int64_t)y * ld + s];
        counts[cell] += 1;
    }
    return cells;
}

/* ------------------------------------------------------------------------ */
/* G^2 = 2 sum_{x,y,z} N_xyz ln(N_xyz / E_xyz), E_xyz = N_x+z N_+yz / N_++z
 * (Section III-B, equations for G^2 and E).
 *
 * The ratio N_xyz / E_xyz equals the integer ratio a / b with
 * a = N_xyz * N_++z and b = N_x+z * N_+yz.  Both products are exact in 64-bit
 * integers (counts < 2^31), so ln(a/b) is taken as log1p((a - b) / b) with the
 * difference formed exactly; this is the same quantity as the textbook term,
 * only evaluated without a rounding step inside the logarithm. */
double oracle_g2(const int64_t* counts, int32_t rx, int32_t ry, int64_t nz)
{
    double g2 = 0.0;
    for (int64_t z = 0; z < nz; z++) {
        const int64_t* t = counts + z * rx * ry;
        int64_t nzz = 0;
        for (int32_t i = 0; i < rx * ry; i++) nzz += t[i];
        for (int32_t x = 0; x < rx; x++) {
            int64_t nxz = 0;
            for (int32_t y = 0; y < ry; y++) nxz += t[x * ry + y];
            for (int32_t y = 0; y < ry; y++) {
                int64_t nxyz = t[x * ry + y];
                if (nxyz == 0) continue;            /* 0 ln 0 = 0 */
                int64_t nyz = 0;
                for (int32_t xx = 0; xx < rx; xx++) nyz += t[xx * ry + y];
                int64_t a = nxyz * nzz;
                int64_t b = nxz * nyz;
                g2 += (double)nxyz * log1p((double)(a - b) / (double)b);
            }
        }
    }
    return 2.0 * g2;
}

/* Pearson's X^2 of the same table (the chi-square statistic the paper names
 * next to G^2, Section III-B): sum over cells with E_xyz > 0 of
 * (N_xyz - E_xyz)^2 / E_xyz.  With E = N_x+z N_+yz / N_++z each term is
 * (N_xyz N_++z - N_x+z N_+yz)^2 / (N_++z N_x+z N_+yz): the numerator's
 * difference is an exact 64-bit integer.  Empty cells with E > 0 count. */
double oracle_x2(const int64_t* counts, int32_t rx, int32_t ry, int64_t nz)
{
    double x2 = 0.0;
    for (int64_t z = 0; z < nz; z++) {
        const int64_t* t = counts + z * rx * ry;
        int64_t nzz = 0;
        for (int32_t i = 0; i < rx * ry; i++) nzz += t[i];
        if (nzz == 0) continue;
        for (int32_t x = 0; x < rx; x++) {
            int64_t nxz = 0;
            for (int32_t y = 0; y < ry; y++) nxz += t[x * ry + y];
            if (nxz == 0) continue;
            for (int32_t y = 0; y < ry; y++) {
                int64_t nyz = 0;
                for (int32_t xx = 0; xx < rx; xx++) nyz += t[xx * ry + y];
                if (nyz == 0) continue;
                double diff = (double)(t[x * ry + y] * nzz - nxz * nyz);
                x2 += diff * diff / ((double)nzz * (double)nxz * (double)nyz);
            }
        }
    }
    return x2;
}

/* Degrees of freedom adjusted to the observed table: the sum over strata with
 * N_++z > 0 of (r'_x - 1)(r'_y - 1), r'_x counting the values of X with
 * N_x+z > 0 in the stratum and r'_y those of Y with N_+yz > 0 (the variant of
 * df that drops structurally empty rows, columns and strata). */
double oracle_df_adjusted(const int64_t* counts, int32_t rx, int32_t ry, int64_t nz)
{
    double df = 0.0;
    for (int64_t z = 0; z < nz; z++) {
        const int64_t* t = counts + z * rx * ry;
        int32_t ax = 0, ay = 0;
        for (int32_t x = 0; x < rx; x++) {
            int64_t s = 0;
            for (int32_t y = 0; y < ry; y++) s += t[x * ry + y];
            ax += s > 0;
        }
        for (int32_t y = 0; y < ry; y++) {
            int64_t s = 0;
            for (int32_t x = 0; x < rx; x++) s += t[x * ry + y];
            ay += s > 0;
        }
        if (ax > 0 && ay > 0) df += (double)(ax - 1) * (double)(ay - 1);
    }
    return df;
}

/* Degrees of freedom (Section III-B, read as the conditional form; see header). */
double oracle_df(const uint8_t* arities, int32_t x, int32_t y, const int32_t* S, int32_t d)
{
    double df = (double)(arities[x] - 1) * (double)(arities[y] - 1);
    for (int32_t k = 0; k < d; k++) df *= (double)arities[S[k]];
    return df;
}

/* Chi-square survival function Q(k/2, x/2) for integer k >= 1, from the exact
 * finite sums that hold for integer degrees of freedom (t = x/2):
 *   k = 2m     : Q = sum_{i=0}^{m-1} e^{-t} t^i / i!
 *   k = 2m + 1 : Q = erfc(sqrt t) + sum_{i=0}^{m-1} e^{-t} t^{i+1/2} / Gamma(i + 3/2)
 * Every term is positive; the sum is formed in log space, scaled by its
 * largest term, so neither e^{-t} nor t^i overflows or underflows early. */
double oracle_chisq_sf(int64_t k, double x)
{
    if (!(x > 0.0)) return 1.0;
    double t = 0.5 * x;
    double lt = log(t);
    int64_t m = k / 2;
    int odd = (int)(k & 1);
    double head = odd ? erfc(sqrt(t)) : 0.0;
    if (m == 0) return head;
    double lmax = -INFINITY;
    for (int64_t i = 0; i < m; i++) {
        double li = odd ? (-t + ((double)i + 0.5) * lt - lgamma((double)i + 1.5))
                        : (-t + (double)i * lt - lgamma((double)i + 1.0));
        if (li > lmax) lmax = li;
    }
    double s = 0.0;
    for (int64_t i = 0; i < m; i++) {
        double li = odd ? (-t + ((double)i + 0.5) * lt - lgamma((double)i + 1.5))
                        : (-t + (double)i * lt - lgamma((double)i + 1.0));
        s += exp(li - lmax);
    }
    double q = head + exp(lmax) * s;
    return q > 1.0 ? 1.0 : q;
}

/* One CI test I(X, Y | S): table, statistic, df and p (Section III-B).
 * stat: 0 = G^2, 1 = Pearson X^2; df_mode: 0 = declared arities, 1 = adjusted
 * to the observed table.  With no degrees of freedom left the test cannot
 * reject: p = 1. */
int oracle_ci_test_ex(const uint8_t* data, int64_t ld, int64_t n_samples, const uint8_t* arities,
                      int32_t x, int32_t y, const int32_t* S, int32_t d, int32_t stat, int32_t df_mode,
                      double* stat_out, double* df_out, double* p_out)
{
    int64_t cells = (int64_t)arities[x] * arities[y];
    for (int32_t k = 0; k < d; k++) cells *= arities[S[k]];
    int64_t* counts = (int64_t*)malloc((size_t)cells * sizeof(int64_t));
    if (!counts) return ORACLE_ENOMEM;
    oracle_ci_table(data, ld, n_samples, arities, x, y, S, d, counts, cells);
    const int64_t nz = cells / ((int64_t)arities[x] * arities[y]);
    double st = stat == 1 ? oracle_x2(counts, arities[x], arities[y], nz) : oracle_g2(counts, arities[x], arities[y], nz);
    double df = df_mode == 1 ? oracle_df_adjusted(counts, arities[x], arities[y], nz) : oracle_df(arities, x, y, S, d);
    free(counts);
    *stat_out = st;
    *df_out = df;
    *p_out = df > 0.0 ? oracle_chisq_sf((int64_t)df, st) : 1.0;
    return ORACLE_OK;
}

int oracle_ci_test(const uint8_t* data, int64_t ld, int64_t n_samples, const uint8_t* arities,
                   int32_t x, int32_t y, const int32_t* S, int32_t d,
                   double* g2_out, double* df_out, double* p_out)
{
    return oracle_ci_test_ex(data, ld, n_samples, arities, x, y, S, d, 0, 0, g2_out, df_out, p_out);
}

/* ------------------------------------------------------------------------ */
/* q-subsets of {0..p-1} in lexicographic order (Section IV-C generates the
 * conditioning sets in this order).  first: c = (0, 1, ..., q-1).  next:
 * raise the right-most position that can still move, reset the ones after it. */
int oracle_first_subset(int32_t p, int32_t q, int32_t* c)
{
    if (q > p || q < 0) return 0;
    for (int32_t k = 0; k < q; k++) c[k] = k;
    return 1;
}

int oracle_next_subset(int32_t p, int32_t q, int32_t* c)
{
    int32_t k = q - 1;
    while (k >= 0 && c[k] == p - q + k) k--;
    if (k < 0) return 0;
    c[k] += 1;
    for (int32_t l = k + 1; l < q; l++) c[l] = c[l - 1] + 1;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* PC-stable skeleton (Algorithm 1). */
typedef struct {
    int32_t n;
    uint8_t* adj;            /* n*n */
    int32_t* sep_len;        /* n*n, -1 while adjacent */
    int32_t** sep;           /* n*n pointers, stored for i<j and mirrored */
    int32_t depths;          /* depths that ran at least the snapshot */
    int64_t tests[64];       /* tests per depth (depths >= 64 fold into 63) */
    int64_t removed[64];
    /* tests whose p lies within near_tol of alpha: (i, j, d, p) */
    int64_t n_near, cap_near;
    int32_t* near_ijd;
    double* near_p;
} oracle_result;

static int near_push(oracle_result* r, int32_t i, int32_t j, int32_t d, double p)
{
    if (r->n_near == r->cap_near) {
        int64_t cap = r->cap_near ? 2 * r->cap_near : 64;
        int32_t* a = (int32_t*)realloc(r->near_ijd, (size_t)cap * 3 * sizeof(int32_t));
        if (!a) return ORACLE_ENOMEM;
        r->near_ijd = a;
        double* b = (double*)realloc(r->near_p, (size_t)cap * sizeof(double));
        if (!b) return ORACLE_ENOMEM;
        r->near_p = b;
        r->cap_near = cap;
    }
    r->near_ijd[3 * r->n_near + 0] = i;
    r->near_ijd[3 * r->n_near + 1] = j;
    r->near_ijd[3 * r->n_near + 2] = d;
    r->near_p[r->n_near] = p;
    r->n_near++;
    return ORACLE_OK;
}

void oracle_result_free(oracle_result* r)
{
    if (!r) return;
    if (r->sep)
        for (int64_t k = 0; k < (int64_t)r->n * r->n; k++) free(r->sep[k]);
    free(r->sep);
    free(r->sep_len);
    free(r->adj);
    free(r->near_ijd);
    free(r->near_p);
    free(r);
}

oracle_result* oracle_pc_stable_ex(const uint8_t* data, int64_t ld, int32_t n, int64_t n_samples,
                                   const uint8_t* arities, double alpha, int32_t max_depth, double near_tol,
                                   int32_t stat, int32_t df_mode)
{
    oracle_result* r = (oracle_result*)calloc(1, sizeof(oracle_result));
    if (!r) return NULL;
    int64_t nn = (int64_t)n * n;
    r->n = n;
    r->adj = (uint8_t*)malloc((size_t)nn);
    r->sep_len = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    r->sep = (int32_t**)calloc((size_t)nn, sizeof(int32_t*));
    int32_t* nbr = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    int32_t* deg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* cand = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* c = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t* S = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    uint8_t* remove = (uint8_t*)malloc((size_t)nn);
    if (!r->adj || !r->sep_len || !r->sep || !nbr || !deg || !cand || !c || !S || !remove) {
        free(nbr); free(deg); free(cand); free(c); free(S); free(remove);
        oracle_result_free(r);
        return NULL;
    }
    /* Algorithm 1 starts from the complete undirected graph. */
    for (int32_t i = 0; i < n; i++)
        for (int32_t j = 0; j < n; j++) {
            r->adj[(int64_t)i * n + j] = (uint8_t)(i != j);
            r->sep_len[(int64_t)i * n + j] = -1;
        }

    for (int32_t d = 0;; d++) {
        if (max_depth >= 0 && d > max_depth) break;
        /* Snapshot a(V_i) of every node, ascending (Algorithm 1). */
        for (int32_t i = 0; i < n; i++) {
            deg[i] = 0;
            for (int32_t j = 0; j < n; j++)
                if (r->adj[(int64_t)i * n + j]) nbr[(int64_t)i * n + deg[i]++] = j;
        }
        /* Termination test of Algorithm 1, evaluated on this depth's snapshot:
         * does any edge have a side with at least d candidates? */
        int any = 0;
        for (int32_t i = 0; i < n && !any; i++)
            for (int32_t k = 0; k < deg[i]; k++)
                if (deg[i] - 1 >= d) { any = 1; break; }
        if (!any) break;
        int32_t slot = d < 63 ? d : 63;
        r->depths = d + 1;
        memset(remove, 0, (size_t)nn);

        /* Every edge i<j of the snapshot (Algorithm 1). */
        for (int32_t i = 0; i < n; i++) {
            for (int32_t kk = 0; kk < deg[i]; kk++) {
                int32_t j = nbr[(int64_t)i * n + kk];
                if (j <= i) continue;
                int found = 0;
                int sides = (d == 0) ? 1 : 2;     /* depth 0: one marginal test */
                for (int side = 0; side < sides && !found; side++) {
                    int32_t a = side == 0 ? i : j, b = side == 0 ? j : i;
                    int32_t p = 0;
                    for (int32_t t = 0; t < deg[a]; t++) {
                        int32_t v = nbr[(int64_t)a * n + t];
                        if (v != b) cand[p++] = v;
                    }
                    if (!oracle_first_subset(p, d, c)) continue;
                    do {
                        for (int32_t k = 0; k < d; k++) S[k] = cand[c[k]];
                        double g2, df, pv;
                        if (oracle_ci_test_ex(data, ld, n_samples, arities, i, j, S, d, stat, df_mode, &g2, &df,
                                              &pv)) {
                            free(nbr); free(deg); free(cand); free(c); free(S); free(remove);
                            oracle_result_free(r);
                            return NULL;
                        }
                        r->tests[slot]++;
                        if (fabs(pv - alpha) <= near_tol) near_push(r, i, j, d, pv);
                        if (pv > alpha) {               /* independent: remove, keep S */
                            found = 1;
                            remove[(int64_t)i * n + j] = 1;
                            int32_t* s = (int32_t*)malloc((size_t)(d > 0 ? d : 1) * sizeof(int32_t));
                            for (int32_t k = 0; k < d; k++) s[k] = S[k];
                            r->sep[(int64_t)i * n + j] = s;
                            r->sep_len[(int64_t)i * n + j] = d;
                            r->sep_len[(int64_t)j * n + i] = d;
                        }
                    } while (!found && oracle_next_subset(p, d, c));
                }
            }
        }
        /* Removals take effect after the depth (PC-stable: tests read the snapshot). */
        for (int32_t i = 0; i < n; i++)
            for (int32_t j = i + 1; j < n; j++)
                if (remove[(int64_t)i * n + j]) {
                    r->adj[(int64_t)i * n + j] = 0;
                    r->adj[(int64_t)j * n + i] = 0;
                    r->removed[slot]++;
                }
    }
    free(nbr); free(deg); free(cand); free(c); free(S); free(remove);
    return r;
}

oracle_result* oracle_pc_stable(const uint8_t* data, int64_t ld, int32_t n, int64_t n_samples,
                                const uint8_t* arities, double alpha, int32_t max_depth, double near_tol)
{
    return oracle_pc_stable_ex(data, ld, n, n_samples, arities, alpha, max_depth, near_tol, 0, 0);
}

void oracle_result_adjacency(const oracle_result* r, uint8_t* out)
{
    memcpy(out, r->adj, (size_t)r->n * r->n);
}

int32_t oracle_result_sepset(const oracle_result* r, int32_t i, int32_t j, int32_t* buf, int32_t cap)
{
    if (i > j) { int32_t t = i; i = j; j = t; }
    int32_t len = r->sep_len[(int64_t)i * r->n + j];
    if (len < 0) return -1;
    for (int32_t k = 0; k < len && k < cap; k++) buf[k] = r->sep[(int64_t)i * r->n + j][k];
    return len;
}

int32_t oracle_result_depths(const oracle_result* r) { return r->depths; }
int64_t oracle_result_tests(const oracle_result* r, int32_t d) { return (d >= 0 && d < 64) ? r->tests[d] : 0; }
int64_t oracle_result_removed(const oracle_result* r, int32_t d) { return (d >= 0 && d < 64) ? r->removed[d] : 0; }
int64_t oracle_result_near_count(const oracle_result* r) { return r->n_near; }

void oracle_result_near(const oracle_result* r, int32_t* ijd, double* p)
{
    memcpy(ijd, r->near_ijd, (size_t)r->n_near * 3 * sizeof(int32_t));
    memcpy(p, r->near_p, (size_t)r->n_near * sizeof(double));
}
