/*
 * CPU oracle for literal-weighted model counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this file; only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (Dudek & Vardi, "Parallel Weighted Model Counting with
 * Tensor Networks"):
 *
 *   W(phi) = sum over all assignments tau of phi(tau) * prod_x W(x, tau(x))
 *
 * the literal-weighted model count of Def. 2.1.  Two independent routes:
 *
 *   oracle_brute_force   enumerates every tau in {0,1}^n (Def. 2.1 verbatim),
 *                        long double accumulation with Neumaier compensation,
 *                        plus an exact uint64 count of satisfying tau.
 *   oracle_bucket_elim   classic variable (bucket) elimination over the
 *                        clause indicator factors and the per-variable weight
 *                        factors: multiply the factors that mention x, sum x
 *                        out, repeat.  It evaluates Eq. (1) for the network
 *                        of Thm 3.2 with every COPY tensor already contracted
 *                        into its variable, which equals Def. 2.1 by
 *                        distributivity.  Tables are long double (64-bit
 *                        mantissa, decimal exponent range about +-4930), so
 *                        counts down to 1e-4900 need no rescaling.
 *   oracle_bucket_exact  the same elimination in unsigned __int128 with all
 *                        weights 1: the exact unweighted count (constant W,
 *                        Sec. 2.1), valid while the count is below 2^128.
 *   oracle_contract_pair one pairwise tensor contraction A . B evaluated
 *                        entry by entry from Eq. (1) for the two-tensor
 *                        network {A, B} (Sec. 2.3), long double sums.
 *
 * Readings where the paper is silent: a clause is evaluated directly from
 * its literals, so repeated literals and tautologies need no special case
 * and an empty clause is a rank-0 factor equal to 0; a variable in no clause
 * contributes W(x,0) + W(x,1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ETOOWIDE -3

/* ------------------------------------------------------------------ */
/* O1a: brute force over {0,1}^n (Def. 2.1)                              */
/* ------------------------------------------------------------------ */

typedef struct { long double s, c; } neumaier_t;

static void neu_add(neumaier_t *acc, long double v) {
    long double t = acc->s + v;
    if (fabsl(acc->s) >= fabsl(v)) acc->c += (acc->s - t) + v;
    else acc->c += (v - t) + acc->s;
    acc->s = t;
}

/* n <= 40.  For each clause two bit masks: the variables that appear
 * positively and negatively.  tau satisfies the clause when some positive
 * literal's variable is 1 or some negative literal's variable is 0. */
int oracle_brute_force(int32_t n, int64_t m, const int32_t *lits,
                       const int64_t *off, const double *wpos,
                       const double *wneg, double *mant, int64_t *exp2,
                       uint64_t *count) {
    if (n < 0 || n > 40 || m < 0) return ORC_EINVAL;
    uint64_t *pos = (uint64_t *)calloc((size_t)(m ? m : 1), sizeof(uint64_t));
    uint64_t *neg = (uint64_t *)calloc((size_t)(m ? m : 1), sizeof(uint64_t));
    if (!pos || !neg) { free(pos); free(neg); return ORC_ENOMEM; }
    for (int64_t c = 0; c < m; ++c) {
        for (int64_t i = off[c]; i < off[c + 1]; ++i) {
            int32_t l = lits[i];
            int32_t v = l > 0 ? l : -l;
            if (v < 1 || v > n) { free(pos); free(neg); return ORC_EINVAL; }
            if (l > 0) pos[c] |= 1ull << (v - 1);
            else neg[c] |= 1ull << (v - 1);
        }
    }
    const uint64_t total = 1ull << n;
    /* Fixed chunking so the summation order does not depend on the number
     * of threads. */
    const int64_t n_chunks = total < 256 ? (int64_t)total : 256;
    const uint64_t chunk = total / (uint64_t)n_chunks;
    neumaier_t *part = (neumaier_t *)calloc((size_t)n_chunks, sizeof(neumaier_t));
    uint64_t *cnt = (uint64_t *)calloc((size_t)n_chunks, sizeof(uint64_t));
    if (!part || !cnt) { free(pos); free(neg); free(part); free(cnt); return ORC_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < n_chunks; ++ch) {
        neumaier_t acc = {0.0L, 0.0L};
        uint64_t k = 0;
        for (uint64_t tau = ch * chunk; tau < (ch + 1) * chunk; ++tau) {
            int sat = 1;
            for (int64_t c = 0; c < m; ++c) {
                if (!((tau & pos[c]) || (~tau & neg[c]))) { sat = 0; break; }
            }
            if (!sat) continue;
            ++k;
            long double p = 1.0L;
            for (int32_t x = 0; x < n; ++x)
                p *= ((tau >> x) & 1) ? (long double)wpos[x] : (long double)wneg[x];
            neu_add(&acc, p);
        }
        part[ch] = acc;
        cnt[ch] = k;
    }
    neumaier_t tot = {0.0L, 0.0L};
    uint64_t k = 0;
    for (int64_t ch = 0; ch < n_chunks; ++ch) {
        neu_add(&tot, part[ch].s);
        neu_add(&tot, part[ch].c);
        k += cnt[ch];
    }
    long double v = tot.s + tot.c;
    int e = 0;
    long double fr = frexpl(v, &e);
    *mant = (double)fr;
    *exp2 = (v == 0.0L) ? 0 : e;
    *count = k;
    free(pos); free(neg); free(part); free(cnt);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* O1b: bucket elimination                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t r;        /* number of variables */
    int32_t *vars;    /* bit j of a table offset is variable vars[j] */
    void *tab;        /* 2^r entries */
    int alive;
} factor_t;

/* The oracle's own elimination order: minimum degree on the primal graph,
 * ties broken by the lowest variable id.  Variables are 1-based. */
static int min_degree_order(int32_t n, int64_t m, const int32_t *lits,
                            const int64_t *off, int32_t *order) {
    uint8_t *adj = (uint8_t *)calloc((size_t)n * (size_t)n, 1);
    int32_t *deg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    if (!adj || !deg || !done) { free(adj); free(deg); free(done); return ORC_ENOMEM; }
    for (int64_t c = 0; c < m; ++c)
        for (int64_t i = off[c]; i < off[c + 1]; ++i)
            for (int64_t j = off[c]; j < off[c + 1]; ++j) {
                int32_t a = abs(lits[i]) - 1, b = abs(lits[j]) - 1;
                if (a != b && !adj[(size_t)a * n + b]) {
                    adj[(size_t)a * n + b] = 1;
                    deg[a]++;
                }
            }
    for (int32_t step = 0; step < n; ++step) {
        int32_t best = -1;
        for (int32_t v = 0; v < n; ++v)
            if (!done[v] && (best < 0 || deg[v] < deg[best])) best = v;
        order[step] = best + 1;
        done[best] = 1;
        /* connect the neighbours of best into a clique, then drop best */
        for (int32_t a = 0; a < n; ++a) {
            if (done[a] || !adj[(size_t)best * n + a]) continue;
            for (int32_t b = 0; b < n; ++b) {
                if (b == a || done[b] || !adj[(size_t)best * n + b]) continue;
                if (!adj[(size_t)a * n + b]) { adj[(size_t)a * n + b] = 1; deg[a]++; }
            }
        }
        for (int32_t a = 0; a < n; ++a)
            if (adj[(size_t)best * n + a]) { adj[(size_t)a * n + best] = 0; deg[a]--; }
    }
    free(adj); free(deg); free(done);
    return ORC_OK;
}

/* Clause indicator over the clause's distinct variables (sorted), evaluated
 * literal by literal. */
static int clause_vars(const int32_t *lits, int64_t lo, int64_t hi, int32_t *vars) {
    int32_t r = 0;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t v = abs(lits[i]);
        int seen = 0;
        for (int32_t j = 0; j < r; ++j) seen |= (vars[j] == v);
        if (!seen) vars[r++] = v;
    }
    for (int32_t i = 1; i < r; ++i)   /* insertion sort */
        for (int32_t j = i; j > 0 && vars[j - 1] > vars[j]; --j) {
            int32_t t = vars[j]; vars[j] = vars[j - 1]; vars[j - 1] = t;
        }
    return r;
}

static int clause_value(const int32_t *lits, int64_t lo, int64_t hi,
                        const int32_t *vars, int32_t r, uint64_t assign) {
    for (int64_t i = lo; i < hi; ++i) {
        int32_t v = abs(lits[i]);
        int32_t j = 0;
        while (vars[j] != v) ++j;
        int bit = (int)((assign >> j) & 1);
        if ((lits[i] > 0 && bit) || (lits[i] < 0 && !bit)) return 1;
    }
    (void)r;
    return 0;
}

/* The elimination is written once as a macro and instantiated for long
 * double (weighted) and unsigned __int128 (exact unweighted). */
#define DEFINE_BUCKET_ELIM(NAME, T)                                            \
static int NAME(int32_t n, int64_t m, const int32_t *lits, const int64_t *off, \
                const double *wpos, const double *wneg, const int32_t *order,  \
                int32_t max_width, T *result, int32_t *width_out) {            \
    int64_t nf = m + n;                                                        \
    factor_t *f = (factor_t *)calloc((size_t)(nf + n + 1), sizeof(factor_t));  \
    int32_t *tmpv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));      \
    if (!f || !tmpv) { free(f); free(tmpv); return ORC_ENOMEM; }               \
    int64_t cnt = 0;                                                           \
    for (int64_t c = 0; c < m; ++c) {                                          \
        int32_t r = clause_vars(lits, off[c], off[c + 1], tmpv);               \
        if (r > max_width) { cnt = -1; break; }                                \
        factor_t *F = &f[cnt++];                                               \
        F->r = r; F->alive = 1;                                                \
        F->vars = (int32_t *)malloc(sizeof(int32_t) * (size_t)(r ? r : 1));    \
        memcpy(F->vars, tmpv, sizeof(int32_t) * (size_t)r);                    \
        F->tab = malloc(sizeof(T) << r);                                       \
        for (uint64_t a = 0; a < (1ull << r); ++a)                             \
            ((T *)F->tab)[a] = (T)clause_value(lits, off[c], off[c + 1],       \
                                               F->vars, r, a);                 \
    }                                                                          \
    if (cnt < 0) { free(tmpv); return ORC_ETOOWIDE; }                          \
    for (int32_t x = 1; x <= n; ++x) {                                         \
        factor_t *F = &f[cnt++];                                               \
        F->r = 1; F->alive = 1;                                                \
        F->vars = (int32_t *)malloc(sizeof(int32_t));                          \
        F->vars[0] = x;                                                        \
        F->tab = malloc(sizeof(T) * 2);                                        \
        ((T *)F->tab)[0] = (T)wneg[x - 1];                                     \
        ((T *)F->tab)[1] = (T)wpos[x - 1];                                     \
    }                                                                          \
    int32_t width = 0;                                                         \
    int rc = ORC_OK;                                                           \
    for (int32_t step = 0; step < n && rc == ORC_OK; ++step) {                 \
        int32_t x = order[step];                                               \
        /* union U of the variables of the factors that mention x */          \
        int32_t R = 0;                                                         \
        for (int64_t i = 0; i < cnt; ++i) {                                    \
            if (!f[i].alive) continue;                                         \
            int has = 0;                                                       \
            for (int32_t j = 0; j < f[i].r; ++j) has |= (f[i].vars[j] == x);   \
            if (!has) continue;                                                \
            for (int32_t j = 0; j < f[i].r; ++j) {                             \
                int seen = 0;                                                  \
                for (int32_t k = 0; k < R; ++k) seen |= (tmpv[k] == f[i].vars[j]); \
                if (!seen) tmpv[R++] = f[i].vars[j];                           \
            }                                                                  \
        }                                                                      \
        if (R == 0) continue;                                                  \
        if (R > width) width = R;                                              \
        if (R > max_width) { rc = ORC_ETOOWIDE; break; }                       \
        /* U minus x, in the order collected; x handled separately */         \
        int32_t *uv = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);          \
        int32_t ru = 0;                                                        \
        for (int32_t k = 0; k < R; ++k) if (tmpv[k] != x) uv[ru++] = tmpv[k];  \
        /* the bucket: factor ids, and for each the offset bit of every      \
         * union variable (0 if absent) and of x */                          \
        int32_t nb = 0;                                                        \
        int64_t *bid = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt);      \
        for (int64_t i = 0; i < cnt; ++i) {                                    \
            if (!f[i].alive) continue;                                         \
            for (int32_t j = 0; j < f[i].r; ++j)                               \
                if (f[i].vars[j] == x) { bid[nb++] = i; break; }               \
        }                                                                      \
        uint64_t *ubit = (uint64_t *)calloc((size_t)nb * (size_t)(ru + 1), sizeof(uint64_t)); \
        uint64_t *xbit = (uint64_t *)calloc((size_t)nb, sizeof(uint64_t));     \
        for (int32_t b = 0; b < nb; ++b) {                                     \
            factor_t *F = &f[bid[b]];                                          \
            for (int32_t j = 0; j < F->r; ++j) {                               \
                if (F->vars[j] == x) { xbit[b] = 1ull << j; continue; }        \
                for (int32_t k = 0; k < ru; ++k)                               \
                    if (uv[k] == F->vars[j]) ubit[(size_t)b * ru + k] = 1ull << j; \
            }                                                                  \
        }                                                                      \
        T *out = (T *)calloc((size_t)1 << ru, sizeof(T));                      \
        const uint64_t total = 1ull << ru;                                     \
        const int64_t nch = total < 1024 ? 1 : 1024;                           \
        const uint64_t chunk = total / (uint64_t)nch;                          \
        _Pragma("omp parallel for schedule(static)")                           \
        for (int64_t ch = 0; ch < nch; ++ch) {                                 \
            uint64_t *offs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nb ? nb : 1)); \
            uint64_t u0 = (uint64_t)ch * chunk;                                \
            /* direct offsets of the chunk's first assignment */              \
            for (int32_t b = 0; b < nb; ++b) {                                 \
                offs[b] = 0;                                                   \
                for (int32_t k = 0; k < ru; ++k)                               \
                    if ((u0 >> k) & 1) offs[b] |= ubit[(size_t)b * ru + k];    \
            }                                                                  \
            for (uint64_t u = u0; u < u0 + chunk; ++u) {                       \
                if (u != u0) {                                                 \
                    /* u-1 -> u flips the trailing ones of u-1 and one bit */ \
                    uint64_t flips = u ^ (u - 1);                              \
                    for (int32_t k = 0; k < ru; ++k) {                         \
                        if (!((flips >> k) & 1)) continue;                     \
                        for (int32_t b = 0; b < nb; ++b)                       \
                            offs[b] ^= ubit[(size_t)b * ru + k];               \
                    }                                                          \
                }                                                              \
                T s = 0;                                                       \
                for (int xv = 0; xv < 2; ++xv) {                               \
                    T p = 1;                                                   \
                    for (int32_t b = 0; b < nb; ++b) {                         \
                        uint64_t o = offs[b] | (xv ? xbit[b] : 0);             \
                        p *= ((T *)f[bid[b]].tab)[o];                          \
                    }                                                          \
                    s += p;                                                    \
                }                                                              \
                out[u] = s;                                                    \
            }                                                                  \
            free(offs);                                                        \
        }                                                                      \
        for (int32_t b = 0; b < nb; ++b) {                                     \
            factor_t *F = &f[bid[b]];                                          \
            F->alive = 0; free(F->tab); free(F->vars);                         \
            F->tab = NULL; F->vars = NULL;                                     \
        }                                                                      \
        factor_t *G = &f[cnt++];                                               \
        G->r = ru; G->vars = uv; G->tab = out; G->alive = 1;                   \
        free(bid); free(ubit); free(xbit);                                     \
    }                                                                          \
    T res = 1;                                                                 \
    for (int64_t i = 0; i < cnt; ++i) {                                        \
        if (!f[i].alive) continue;                                             \
        if (rc == ORC_OK && f[i].r != 0) rc = ORC_EINVAL; /* order missed a var */ \
        if (rc == ORC_OK) res *= ((T *)f[i].tab)[0];                           \
        free(f[i].tab); free(f[i].vars);                                       \
    }                                                                          \
    free(f); free(tmpv);                                                       \
    *result = res;                                                             \
    if (width_out) *width_out = width;                                         \
    return rc;                                                                 \
}

DEFINE_BUCKET_ELIM(bucket_elim_ld, long double)
DEFINE_BUCKET_ELIM(bucket_elim_u128, unsigned __int128)

static int check_order(int32_t n, const int32_t *order) {
    uint8_t *seen = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!seen) return ORC_ENOMEM;
    for (int32_t i = 0; i < n; ++i) {
        if (order[i] < 1 || order[i] > n || seen[order[i]]) { free(seen); return ORC_EINVAL; }
        seen[order[i]] = 1;
    }
    free(seen);
    return ORC_OK;
}

static int check_cnf(int32_t n, int64_t m, const int32_t *lits, const int64_t *off) {
    if (n < 0 || m < 0) return ORC_EINVAL;
    for (int64_t c = 0; c < m; ++c) {
        if (off[c + 1] < off[c]) return ORC_EINVAL;
        for (int64_t i = off[c]; i < off[c + 1]; ++i) {
            int32_t v = abs(lits[i]);
            if (lits[i] == 0 || v > n) return ORC_EINVAL;
        }
    }
    return ORC_OK;
}

/* order: n variable ids (1-based) or NULL for the oracle's own min-degree
 * order.  width_out: the largest bucket (number of variables multiplied
 * together), i.e. the induced width + 1. */
int oracle_bucket_elim(int32_t n, int64_t m, const int32_t *lits,
                       const int64_t *off, const double *wpos,
                       const double *wneg, const int32_t *order,
                       int32_t max_width, double *mant, int64_t *exp2,
                       int32_t *width_out) {
    int rc = check_cnf(n, m, lits, off);
    if (rc) return rc;
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!ord) return ORC_ENOMEM;
    if (order) { memcpy(ord, order, sizeof(int32_t) * (size_t)n); rc = check_order(n, ord); }
    else rc = min_degree_order(n, m, lits, off, ord);
    if (rc) { free(ord); return rc; }
    long double v = 0;
    rc = bucket_elim_ld(n, m, lits, off, wpos, wneg, ord, max_width, &v, width_out);
    free(ord);
    if (rc) return rc;
    int e = 0;
    long double fr = frexpl(v, &e);
    *mant = (double)fr;
    *exp2 = (v == 0.0L) ? 0 : e;
    return ORC_OK;
}

/* Exact unweighted count (all weights 1) as two 64-bit halves. */
int oracle_bucket_exact(int32_t n, int64_t m, const int32_t *lits,
                        const int64_t *off, const int32_t *order,
                        int32_t max_width, uint64_t *lo, uint64_t *hi,
                        int32_t *width_out) {
    int rc = check_cnf(n, m, lits, off);
    if (rc) return rc;
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double *ones = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!ord || !ones) { free(ord); free(ones); return ORC_ENOMEM; }
    for (int32_t i = 0; i < n; ++i) ones[i] = 1.0;
    if (order) { memcpy(ord, order, sizeof(int32_t) * (size_t)n); rc = check_order(n, ord); }
    else rc = min_degree_order(n, m, lits, off, ord);
    unsigned __int128 v = 0;
    if (!rc) rc = bucket_elim_u128(n, m, lits, off, ones, ones, ord, max_width, &v, width_out);
    free(ord); free(ones);
    if (rc) return rc;
    *lo = (uint64_t)v;
    *hi = (uint64_t)(v >> 64);
    return ORC_OK;
}

/* The oracle's own min-degree order, exported for tests. */
int oracle_min_degree_order(int32_t n, int64_t m, const int32_t *lits,
                            const int64_t *off, int32_t *order) {
    int rc = check_cnf(n, m, lits, off);
    if (rc) return rc;
    return min_degree_order(n, m, lits, off, order);
}

/* ------------------------------------------------------------------ */
/* Pairwise contraction C = A . B, entry by entry (Eq. (1), two tensors) */
/* ------------------------------------------------------------------ */

/* Labels are nonnegative ints < 4096.  Bit j of a tensor's linear offset
 * is the index labels[j].  Summed indices are the labels of A or B absent
 * from C.  out_offsets lists the C offsets to evaluate (n_out of them); if
 * NULL, all 2^rc offsets are evaluated in order. */
int oracle_contract_pair(int32_t ra, const int32_t *la, const double *a,
                         int32_t rb, const int32_t *lb, const double *b,
                         int32_t rc, const int32_t *lc, int64_t n_out,
                         const int64_t *out_offsets, double *out) {
    if (ra < 0 || rb < 0 || rc < 0 || ra > 40 || rb > 40 || rc > 40) return ORC_EINVAL;
    enum { MAXL = 4096 };
    int32_t summed[80];
    int32_t ks = 0;
    for (int32_t i = 0; i < ra + rb; ++i) {
        int32_t l = i < ra ? la[i] : lb[i - ra];
        if (l < 0 || l >= MAXL) return ORC_EINVAL;
        int inc = 0, dup = 0;
        for (int32_t j = 0; j < rc; ++j) inc |= (lc[j] == l);
        for (int32_t j = 0; j < ks; ++j) dup |= (summed[j] == l);
        if (!inc && !dup) summed[ks++] = l;
    }
    for (int32_t j = 0; j < rc; ++j) {
        int found = 0;
        for (int32_t i = 0; i < ra; ++i) found |= (la[i] == lc[j]);
        for (int32_t i = 0; i < rb; ++i) found |= (lb[i] == lc[j]);
        if (!found) return ORC_EINVAL;
    }
    if (ks > 30) return ORC_EINVAL;
    const int64_t total = n_out;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < total; ++t) {
        uint64_t o = out_offsets ? (uint64_t)out_offsets[t] : (uint64_t)t;
        int8_t val[MAXL];
        for (int32_t j = 0; j < rc; ++j) val[lc[j]] = (int8_t)((o >> j) & 1);
        long double acc = 0.0L;
        for (uint64_t s = 0; s < (1ull << ks); ++s) {
            for (int32_t j = 0; j < ks; ++j) val[summed[j]] = (int8_t)((s >> j) & 1);
            uint64_t oa = 0, ob = 0;
            for (int32_t i = 0; i < ra; ++i) oa |= (uint64_t)val[la[i]] << i;
            for (int32_t i = 0; i < rb; ++i) ob |= (uint64_t)val[lb[i]] << i;
            acc += (long double)a[oa] * (long double)b[ob];
        }
        out[t] = (double)acc;
    }
    return ORC_OK;
}

int oracle_num_threads(void) { return omp_get_max_threads(); }
