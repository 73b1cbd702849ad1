/*
 * kp_oracle.c -- plain, slow, FP64 CPU oracle for the dual-decomposition
 * knapsack method of "Solving Billion-Scale Knapsack Problems"
 * (Zhang, Qi, Hua, Yang; WWW 2020, arXiv 2002.00352).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may link, import or call this file.  It exists so
 * that the tests, the smoke check and the CPU-baseline leg of the benchmark
 * can compare the GPU path against an implementation that a reader can check
 * against the paper by eye.  It shares no code, header, table or constant
 * with the GPU path.
 *
 * Every routine follows the paper's steps in its order and notation, in
 * double precision, with no blocking, fusion or reordering:
 *
 *   kpo_reduced_costs   cost-adjusted profit  p~_ij = p_ij - sum_k lam_k b_ijk
 *                       (Sec. 4.2, the display before Algorithm 1)
 *   kpo_greedy          Algorithm 1 (greedy for hierarchical local
 *                       constraints), literally: initialise x_j = [p~_j > 0],
 *                       sort items by non-increasing p~, then for each set S_l
 *                       in topological order of the inclusion DAG keep only
 *                       the top C_l still-selected items of S_l.
 *   kpo_brute_force     exhaustive 2^M search of the per-user IP,
 *                       Eq. (11)-(13) -- the pin for Proposition 1.
 *   kpo_user_pass       the Map of Algorithm 2 for every user plus the
 *                       Reduce R_k = sum_i v_ik, and the dual / primal sums.
 *   kpo_dd_update       Eq. (14).
 *   kpo_scd_map_user    Algorithm 3 (candidate lambda_k values) and the Map of
 *                       Algorithm 4.
 *   kpo_scd_reduce      the Reduce of Algorithm 4.
 *   kpo_scd_step        one synchronous coordinate-descent iteration
 *                       (Algorithm 4's loop body).
 *   kpo_postprocess     Sec. 5.4, post-processing for feasibility.
 *   kpo_alg5_map_user   Algorithm 5 (Sec. 5.1): the linear-time Map for one
 *                       item per knapsack (M = K, b_ijk = 0 for j != k) and
 *                       one cap Q on the number of items of a user.
 *   kpo_alg5_step       one iteration of Algorithm 4 with Algorithm 5 as Map.
 *
 * Readings of passages that are ambiguous in the paper (each listed in the
 * design notes of the repository):
 *   R1  Algorithm 1 sorts in non-increasing order of p~ (the surrounding prose
 *       says "non-decreasing"; only the algorithm's order is optimal).
 *   R2  "until their sum exceeds C_l" is read as: at most C_l selected items
 *       per set, i.e. constraint (3) is a count.
 *   R3  Equal p~ are ordered by lower item index first; an item is selected
 *       initially only if p~ > 0 strictly (Algorithm 1, first step).
 *   R4  Algorithm 4 re-solves the greedy "at" each candidate.  At a candidate
 *       the lines tie, so the greedy is evaluated on the open interval just
 *       below the candidate (here: at the midpoint between the candidate and
 *       the next smaller candidate, or half the smallest candidate).  The
 *       emitted pair (v1, v2) therefore means: when lambda_k decreases
 *       through v1, this user's k-consumption grows by v2.
 *   R5  Candidates <= 0 are dropped (lambda >= 0, Eq. (10)); parallel lines
 *       have no crossing; a horizontal line (b_jk = 0) has no zero crossing.
 *   R6  The Reduce's "minimal threshold v such that sum_{v1 >= v} v2 <= B_k"
 *       has no minimum over the reals; it is read as the infimum
 *           lambda_k = min { v in {emitted v1} : sum_{v1' > v} v2 <= B_k },
 *       i.e. the emitted value at which the mass accumulated from the top,
 *       including that value's own mass, first exceeds B_k.  If the whole
 *       mass fits, lambda_k = 0.
 *   R7  Post-processing zeroes users in non-decreasing order of the
 *       cost-adjusted group profit (ties: lower user index first), every
 *       user in that order, until all global constraints hold.
 *   R12 Algorithm 5's n-th largest adjusted profit, for n larger than the
 *       number of items K, is 0 (the adjusted profits are clamped at 0, so
 *       missing ranks act as items of profit 0); an item with b_ikk = 0 has
 *       no candidate (as R5 for parallel lines).
 *
 * Layout: p is [N][M], b is dense [N][M][K] with k fastest, lam and B are
 * [K]; local constraints are L item sets given as bitmasks S[l] over the M
 * items (M <= 64) with caps C[l].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "kp_oracle.h"

/* ------------------------------------------------------------------------ */
/* Sec. 4.2: cost-adjusted profit, k summed in ascending order.              */
/* ------------------------------------------------------------------------ */
void kpo_reduced_costs(int M, int K, const double *p, const double *b,
                       const double *lam, double *pt)
{
    for (int j = 0; j < M; ++j) {
        double s = 0.0;
        for (int k = 0; k < K; ++k)
            s += lam[k] * b[(size_t)j * K + k];
        pt[j] = p[j] - s;
    }
}

/* Topological order of the inclusion DAG of the local-constraint sets
 * (Sec. 2.1): a subset comes before any superset.  Ordering by set size,
 * ties by index, is such an order. */
void kpo_topo_order(int L, const uint64_t *S, int *topo)
{
    for (int l = 0; l < L; ++l)
        topo[l] = l;
    for (int a = 1; a < L; ++a) {
        int v = topo[a], b = a - 1;
        int sv = __builtin_popcountll(S[v]);
        while (b >= 0 && __builtin_popcountll(S[topo[b]]) > sv) {
            topo[b + 1] = topo[b];
            --b;
        }
        topo[b + 1] = v;
    }
}

/* Sec. 2.1, Definition 1: every pair of sets is either disjoint or nested. */
int kpo_is_hierarchical(int L, const uint64_t *S)
{
    for (int a = 0; a < L; ++a)
        for (int b = a + 1; b < L; ++b) {
            uint64_t i = S[a] & S[b];
            if (i != 0 && i != S[a] && i != S[b])
                return 0;
        }
    return 1;
}

/* Stable ordering of the items by non-increasing value (R1, R3). */
static void order_desc(int M, const double *v, int *order)
{
    for (int j = 0; j < M; ++j)
        order[j] = j;
    for (int a = 1; a < M; ++a) {
        int t = order[a], b = a - 1;
        while (b >= 0 && v[order[b]] < v[t]) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = t;
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1.                                                              */
/* ------------------------------------------------------------------------ */
void kpo_greedy(int M, int L, const uint64_t *S, const int *C, const int *topo,
                const double *pt, int *x)
{
    int order[64];
    /* first step: x_j = 1 iff p~_j > 0 */
    for (int j = 0; j < M; ++j)
        x[j] = pt[j] > 0.0 ? 1 : 0;
    /* second step: sort items by non-increasing p~ */
    order_desc(M, pt, order);
    /* third step: for each S_l in topological order keep its top C_l
     * still-selected items */
    for (int t = 0; t < L; ++t) {
        int l = topo[t], kept = 0;
        for (int r = 0; r < M; ++r) {
            int j = order[r];
            if (!((S[l] >> j) & 1u) || !x[j])
                continue;
            if (kept < C[l])
                ++kept;
            else
                x[j] = 0;
        }
    }
}

/* Exhaustive search of Eq. (11)-(13) for one user (M <= 24).  Returns the
 * optimal objective sum_j p~_j x_j; x receives the first optimal subset in
 * increasing bitmask order. */
double kpo_brute_force(int M, int L, const uint64_t *S, const int *C,
                       const double *pt, int *x)
{
    double best = 0.0;
    uint64_t bestmask = 0;
    uint64_t nmask = (uint64_t)1 << M;
    for (uint64_t mask = 0; mask < nmask; ++mask) {
        int ok = 1;
        for (int l = 0; l < L && ok; ++l)
            if (__builtin_popcountll(mask & S[l]) > C[l])
                ok = 0;
        if (!ok)
            continue;
        double v = 0.0;
        for (int j = 0; j < M; ++j)
            if ((mask >> j) & 1u)
                v += pt[j];
        if (v > best) {
            best = v;
            bestmask = mask;
        }
    }
    for (int j = 0; j < M; ++j)
        x[j] = (int)((bestmask >> j) & 1u);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, Map + Reduce at a fixed lambda (also the state of Alg. 4).   */
/*   x      optional [N][M] decisions                                        */
/*   R      [K]   R_k = sum_i sum_j b_ijk x_ij                               */
/*   dual   sum_i sum_j p~_ij x_ij   (Eq. (5) without the lambda.B term)     */
/*   primal sum_i sum_j p_ij x_ij    (Eq. (1))                               */
/* Users are split statically over threads; per-thread partial sums are      */
/* combined in thread order.                                                 */
/* ------------------------------------------------------------------------ */
void kpo_user_pass(int64_t N, int M, int K, const double *p, const double *b,
                   int L, const uint64_t *S, const int *C, const double *lam,
                   int *x, double *R, double *dual, double *primal)
{
    int topo[64];
    kpo_topo_order(L, S, topo);
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *partR = (double *)calloc((size_t)nth * K, sizeof(double));
    double *partD = (double *)calloc((size_t)nth, sizeof(double));
    double *partP = (double *)calloc((size_t)nth, sizeof(double));
#pragma omp parallel num_threads(nth)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double pt[64];
        int xi[64];
        double *myR = partR + (size_t)tid * K;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            const double *pi = p + (size_t)i * M;
            const double *bi = b + (size_t)i * M * K;
            kpo_reduced_costs(M, K, pi, bi, lam, pt);
            kpo_greedy(M, L, S, C, topo, pt, xi);
            for (int j = 0; j < M; ++j) {
                if (x)
                    x[(size_t)i * M + j] = xi[j];
                if (!xi[j])
                    continue;
                partD[tid] += pt[j];
                partP[tid] += pi[j];
                for (int k = 0; k < K; ++k)
                    myR[k] += bi[(size_t)j * K + k];
            }
        }
    }
    for (int k = 0; k < K; ++k)
        R[k] = 0.0;
    *dual = 0.0;
    *primal = 0.0;
    for (int t = 0; t < nth; ++t) {
        for (int k = 0; k < K; ++k)
            R[k] += partR[(size_t)t * K + k];
        *dual += partD[t];
        *primal += partP[t];
    }
    free(partR);
    free(partD);
    free(partP);
}

/* Eq. (14): lam_k <- max(lam_k + alpha (R_k - B_k), 0). */
void kpo_dd_update(int K, const double *lam, const double *R, const double *B,
                   double alpha, double *lam_next)
{
    for (int k = 0; k < K; ++k) {
        double v = lam[k] + alpha * (R[k] - B[k]);
        lam_next[k] = v > 0.0 ? v : 0.0;
    }
}

/* Dual objective Eq. (5) at lam:  g = sum_i max_x sum_j p~_ij x_ij
 *                                     + sum_k lam_k B_k.                    */
double kpo_dual_value(int64_t N, int M, int K, const double *p,
                      const double *b, int L, const uint64_t *S, const int *C,
                      const double *lam, const double *B)
{
    double *R = (double *)malloc(sizeof(double) * (size_t)K);
    double dual, primal;
    kpo_user_pass(N, M, K, p, b, L, S, C, lam, NULL, R, &dual, &primal);
    double g = dual;
    for (int k = 0; k < K; ++k)
        g += lam[k] * B[k];
    free(R);
    return g;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 + Map of Algorithm 4 for one user.                            */
/* For each k: the lines z_j(lam_k) = a_j - lam_k b_jk with                  */
/* a_j = p_j - sum_{k' != k} lam_k' b_jk'; candidates are their zero         */
/* crossings and pairwise crossings (R5), unique, sorted decreasingly; the   */
/* greedy is re-solved below each candidate (R4) and the increments of the   */
/* k-consumption are emitted.                                                */
/* Emissions are appended to (ek, ev1, ev2) from position *n; the arrays     */
/* must hold K * (M + M(M-1)/2) more entries.                                */
/* ------------------------------------------------------------------------ */
static int cmp_desc(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a < b) - (a > b);
}

void kpo_scd_map_user(int M, int K, const double *pi, const double *bi, int L,
                      const uint64_t *S, const int *C, const int *topo,
                      const double *lam, int64_t *n, int32_t *ek, double *ev1,
                      double *ev2)
{
    double a[64], s[64], pt[64];
    int x[64];
    int maxc = M + M * (M - 1) / 2;
    double *cand = (double *)malloc(sizeof(double) * (size_t)(maxc > 0 ? maxc : 1));
    for (int k = 0; k < K; ++k) {
        /* the M lines for coordinate k */
        for (int j = 0; j < M; ++j) {
            double o = 0.0;
            for (int kk = 0; kk < K; ++kk)
                if (kk != k)
                    o += lam[kk] * bi[(size_t)j * K + kk];
            a[j] = pi[j] - o;
            s[j] = bi[(size_t)j * K + k];
        }
        /* Algorithm 3: candidate set */
        int nc = 0;
        for (int j = 0; j < M; ++j) {
            if (s[j] > 0.0) {
                double v = a[j] / s[j];
                if (v > 0.0)
                    cand[nc++] = v;
            }
            for (int jj = j + 1; jj < M; ++jj) {
                if (s[j] != s[jj]) {
                    double v = (a[j] - a[jj]) / (s[j] - s[jj]);
                    if (v > 0.0)
                        cand[nc++] = v;
                }
            }
        }
        /* unique values, decreasing */
        qsort(cand, (size_t)nc, sizeof(double), cmp_desc);
        int nu = 0;
        for (int c = 0; c < nc; ++c)
            if (nu == 0 || cand[c] != cand[nu - 1])
                cand[nu++] = cand[c];
        /* Map of Algorithm 4 */
        double prev = 0.0;
        for (int c = 0; c < nu; ++c) {
            double lo = (c + 1 < nu) ? cand[c + 1] : 0.0;
            double at = 0.5 * (cand[c] + lo); /* R4: just below cand[c] */
            for (int j = 0; j < M; ++j)
                pt[j] = a[j] - at * s[j];
            kpo_greedy(M, L, S, C, topo, pt, x);
            double cur = 0.0;
            for (int j = 0; j < M; ++j)
                if (x[j])
                    cur += s[j];
            if (cur > prev) {
                ek[*n] = k;
                ev1[*n] = cand[c];
                ev2[*n] = cur - prev;
                ++*n;
                prev = cur;
            }
        }
    }
    free(cand);
}

/* ------------------------------------------------------------------------ */
/* Reduce of Algorithm 4 for one knapsack (R6).  v1/v2 are permuted.         */
/* ------------------------------------------------------------------------ */
typedef struct {
    double v1, v2;
} pair_t;

static int cmp_pair_desc(const void *x, const void *y)
{
    double a = ((const pair_t *)x)->v1, b = ((const pair_t *)y)->v1;
    return (a < b) - (a > b);
}

double kpo_scd_reduce(int64_t n, const double *v1, const double *v2, double Bk)
{
    double total = 0.0;
    for (int64_t e = 0; e < n; ++e)
        total += v2[e];
    if (total <= Bk)
        return 0.0;
    pair_t *pr = (pair_t *)malloc(sizeof(pair_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t e = 0; e < n; ++e) {
        pr[e].v1 = v1[e];
        pr[e].v2 = v2[e];
    }
    qsort(pr, (size_t)n, sizeof(pair_t), cmp_pair_desc);
    double cum = 0.0, ans = 0.0;
    int64_t e = 0;
    while (e < n) {
        double v = pr[e].v1, mass = 0.0;
        while (e < n && pr[e].v1 == v)
            mass += pr[e++].v2;
        if (cum + mass > Bk) {
            ans = v;
            break;
        }
        cum += mass;
    }
    free(pr);
    return ans;
}

/* ------------------------------------------------------------------------ */
/* One iteration of Algorithm 4: Map over all users, Reduce over all k.      */
/* Returns the number of emitted pairs, or -1 on allocation failure.         */
/* Optional per-k outputs: nemit[k] (pairs emitted for k), mass[k] (their    */
/* total v2).                                                                */
/* ------------------------------------------------------------------------ */
int64_t kpo_scd_step(int64_t N, int M, int K, const double *p, const double *b,
                     int L, const uint64_t *S, const int *C, const double *lam,
                     const double *B, double *lam_next, int64_t *nemit,
                     double *mass)
{
    int topo[64];
    kpo_topo_order(L, S, topo);
    int64_t per_user = (int64_t)K * (M + (int64_t)M * (M - 1) / 2);
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    /* per-thread emission lists, concatenated in thread order afterwards */
    int64_t *cnt = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int32_t **tk = (int32_t **)calloc((size_t)nth, sizeof(int32_t *));
    double **t1 = (double **)calloc((size_t)nth, sizeof(double *));
    double **t2 = (double **)calloc((size_t)nth, sizeof(double *));
    int64_t *cap = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int failed = 0;
#pragma omp parallel num_threads(nth)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            if (cnt[tid] + per_user > cap[tid]) {
                int64_t nc = 2 * cap[tid] + 4 * per_user;
                int32_t *nk = (int32_t *)realloc(tk[tid], sizeof(int32_t) * (size_t)nc);
                double *n1 = (double *)realloc(t1[tid], sizeof(double) * (size_t)nc);
                double *n2 = (double *)realloc(t2[tid], sizeof(double) * (size_t)nc);
                if (!nk || !n1 || !n2) {
                    failed = 1;
                    continue;
                }
                tk[tid] = nk;
                t1[tid] = n1;
                t2[tid] = n2;
                cap[tid] = nc;
            }
            kpo_scd_map_user(M, K, p + (size_t)i * M, b + (size_t)i * M * K, L,
                             S, C, topo, lam, &cnt[tid], tk[tid], t1[tid],
                             t2[tid]);
        }
    }
    int64_t total = 0;
    for (int t = 0; t < nth; ++t)
        total += cnt[t];
    if (failed) {
        total = -1;
        goto done;
    }
    /* Reduce: group the emissions by key k */
    {
        int64_t *nk = (int64_t *)calloc((size_t)K, sizeof(int64_t));
        for (int t = 0; t < nth; ++t)
            for (int64_t e = 0; e < cnt[t]; ++e)
                nk[tk[t][e]]++;
        for (int k = 0; k < K; ++k) {
            double *v1 = (double *)malloc(sizeof(double) * (size_t)(nk[k] + 1));
            double *v2 = (double *)malloc(sizeof(double) * (size_t)(nk[k] + 1));
            int64_t m = 0;
            double ms = 0.0;
            for (int t = 0; t < nth; ++t)
                for (int64_t e = 0; e < cnt[t]; ++e)
                    if (tk[t][e] == k) {
                        v1[m] = t1[t][e];
                        v2[m] = t2[t][e];
                        ms += t2[t][e];
                        ++m;
                    }
            lam_next[k] = kpo_scd_reduce(m, v1, v2, B[k]);
            if (nemit)
                nemit[k] = m;
            if (mass)
                mass[k] = ms;
            free(v1);
            free(v2);
        }
        free(nk);
    }
done:
    for (int t = 0; t < nth; ++t) {
        free(tk[t]);
        free(t1[t]);
        free(t2[t]);
    }
    free(tk);
    free(t1);
    free(t2);
    free(cnt);
    free(cap);
    return total;
}

/* ------------------------------------------------------------------------ */
/* The Map of Algorithm 4 for every user (kpo_scd_map_user per user, users   */
/* split over threads, lists concatenated in thread order, so users ascend): */
/* writes (user, k, v1, v2) of every emission when the total fits in cap and */
/* returns the total (or -1 on allocation failure); no Reduce.               */
/* ------------------------------------------------------------------------ */
int64_t kpo_scd_map_all(int64_t N, int M, int K, const double *p, const double *b,
                        int L, const uint64_t *S, const int *C, const double *lam,
                        int64_t cap_out, int64_t *eu, int32_t *ek, double *ev1,
                        double *ev2)
{
    int topo[64];
    kpo_topo_order(L, S, topo);
    int64_t per_user = (int64_t)K * (M + (int64_t)M * (M - 1) / 2);
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    int64_t *cnt = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int64_t **tu = (int64_t **)calloc((size_t)nth, sizeof(int64_t *));
    int32_t **tk = (int32_t **)calloc((size_t)nth, sizeof(int32_t *));
    double **t1 = (double **)calloc((size_t)nth, sizeof(double *));
    double **t2 = (double **)calloc((size_t)nth, sizeof(double *));
    int64_t *cap = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int failed = 0;
#pragma omp parallel num_threads(nth)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            if (cnt[tid] + per_user > cap[tid]) {
                int64_t nc = 2 * cap[tid] + 4 * per_user;
                int64_t *nu = (int64_t *)realloc(tu[tid], sizeof(int64_t) * (size_t)nc);
                if (nu) tu[tid] = nu;
                int32_t *nk = (int32_t *)realloc(tk[tid], sizeof(int32_t) * (size_t)nc);
                if (nk) tk[tid] = nk;
                double *n1 = (double *)realloc(t1[tid], sizeof(double) * (size_t)nc);
                if (n1) t1[tid] = n1;
                double *n2 = (double *)realloc(t2[tid], sizeof(double) * (size_t)nc);
                if (n2) t2[tid] = n2;
                if (!nu || !nk || !n1 || !n2) {
                    failed = 1;
                    continue;
                }
                cap[tid] = nc;
            }
            int64_t before = cnt[tid];
            kpo_scd_map_user(M, K, p + (size_t)i * M, b + (size_t)i * M * K, L,
                             S, C, topo, lam, &cnt[tid], tk[tid], t1[tid],
                             t2[tid]);
            for (int64_t e = before; e < cnt[tid]; ++e)
                tu[tid][e] = i;
        }
    }
    int64_t total = 0;
    for (int t = 0; t < nth; ++t)
        total += cnt[t];
    if (failed) {
        total = -1;
    } else if (total <= cap_out) {
        int64_t o = 0;
        for (int t = 0; t < nth; ++t)
            for (int64_t e = 0; e < cnt[t]; ++e, ++o) {
                eu[o] = tu[t][e];
                ek[o] = tk[t][e];
                ev1[o] = t1[t][e];
                ev2[o] = t2[t][e];
            }
    }
    for (int t = 0; t < nth; ++t) {
        free(tu[t]);
        free(tk[t]);
        free(t1[t]);
        free(t2[t]);
    }
    free(tu);
    free(tk);
    free(t1);
    free(t2);
    free(cnt);
    free(cap);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Sec. 5.4: post-processing for feasibility (R7).  x is [N][M], modified in */
/* place.  Returns the number of users reset.                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    double key;
    int64_t i;
} ukey_t;

static int cmp_ukey(const void *x, const void *y)
{
    const ukey_t *a = (const ukey_t *)x, *b = (const ukey_t *)y;
    if (a->key < b->key)
        return -1;
    if (a->key > b->key)
        return 1;
    return (a->i > b->i) - (a->i < b->i);
}

int64_t kpo_postprocess(int64_t N, int M, int K, const double *p,
                        const double *b, const double *lam, const double *B,
                        int *x)
{
    double *R = (double *)calloc((size_t)K, sizeof(double));
    ukey_t *u = (ukey_t *)malloc(sizeof(ukey_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        double gp = 0.0;
        for (int j = 0; j < M; ++j) {
            if (!x[(size_t)i * M + j])
                continue;
            gp += p[(size_t)i * M + j];
            for (int k = 0; k < K; ++k) {
                double bk = b[((size_t)i * M + j) * K + k];
                gp -= lam[k] * bk;
                R[k] += bk;
            }
        }
        u[i].key = gp;
        u[i].i = i;
    }
    qsort(u, (size_t)N, sizeof(ukey_t), cmp_ukey);
    int64_t reset = 0;
    for (int64_t r = 0; r < N; ++r) {
        int feasible = 1;
        for (int k = 0; k < K; ++k)
            if (R[k] > B[k])
                feasible = 0;
        if (feasible)
            break;
        int64_t i = u[r].i;
        for (int j = 0; j < M; ++j) {
            if (!x[(size_t)i * M + j])
                continue;
            for (int k = 0; k < K; ++k)
                R[k] -= b[((size_t)i * M + j) * K + k];
            x[(size_t)i * M + j] = 0;
        }
        ++reset;
    }
    free(R);
    free(u);
    return reset;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 5 (Sec. 5.1): Map of one user when item k is the only item that */
/* consumes knapsack k (M = K) and one local constraint allows at most Q     */
/* items.  pi[k] = p_ik, bi[k] = b_ikk.  Emits at most one (k, v1, v2) per k */
/* into ek / ev1 / ev2; *n receives their number.                            */
/* ------------------------------------------------------------------------ */
static int cmp_double_desc(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a < b) - (a > b);
}

/* n-th largest of the K adjusted profits (n >= 1); 0 beyond K (R12) */
static double nth_largest(const double *sorted_desc, int K, int n)
{
    return n <= K ? sorted_desc[n - 1] : 0.0;
}

void kpo_alg5_map_user(int K, const double *pi, const double *bi, int Q,
                       const double *lam, int64_t *n, int32_t *ek,
                       double *ev1, double *ev2)
{
    double *adj = (double *)malloc(sizeof(double) * (size_t)K);
    double *srt = (double *)malloc(sizeof(double) * (size_t)K);
    for (int k = 0; k < K; ++k) {
        double a = pi[k] - lam[k] * bi[k];
        adj[k] = a > 0.0 ? a : 0.0;
        srt[k] = adj[k];
    }
    qsort(srt, (size_t)K, sizeof(double), cmp_double_desc);
    const double q_th = nth_largest(srt, K, Q);
    const double q1_th = nth_largest(srt, K, Q + 1);
    int64_t m = 0;
    for (int k = 0; k < K; ++k) {
        const double pbar = adj[k] >= q_th ? q1_th : q_th;
        if (pi[k] > pbar && bi[k] > 0.0) {
            ek[m] = k;
            ev1[m] = (pi[k] - pbar) / bi[k];
            ev2[m] = bi[k];
            ++m;
        }
    }
    *n = m;
    free(adj);
    free(srt);
}

/* One iteration of Algorithm 4 with Algorithm 5 as its Map: p and bd are    */
/* [N][K] (bd[i][k] = b_ikk); lam_next[k] = the Reduce of the pairs of k.    */
/* Returns the number of emitted pairs, or -1 on allocation failure.         */
int64_t kpo_alg5_step(int64_t N, int K, const double *p, const double *bd,
                      int Q, const double *lam, const double *B,
                      double *lam_next)
{
    int64_t cap = N * (int64_t)K;
    int32_t *ek = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    double *v1 = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    double *v2 = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    if (!ek || !v1 || !v2 || !cnt) {
        free(ek);
        free(v1);
        free(v2);
        free(cnt);
        return -1;
    }
    int64_t total = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t m = 0;
        kpo_alg5_map_user(K, p + i * K, bd + i * K, Q, lam, &m, ek + total,
                          v1 + total, v2 + total);
        total += m;
    }
    /* group the pairs by k (the shuffle of the MapReduce), then Reduce */
    for (int64_t e = 0; e < total; ++e)
        cnt[ek[e] + 1]++;
    for (int k = 0; k < K; ++k)
        cnt[k + 1] += cnt[k];
    double *g1 = (double *)malloc(sizeof(double) * (size_t)(total > 0 ? total : 1));
    double *g2 = (double *)malloc(sizeof(double) * (size_t)(total > 0 ? total : 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    if (!g1 || !g2 || !pos) {
        free(ek);
        free(v1);
        free(v2);
        free(cnt);
        free(g1);
        free(g2);
        free(pos);
        return -1;
    }
    for (int k = 0; k < K; ++k)
        pos[k] = cnt[k];
    for (int64_t e = 0; e < total; ++e) {
        const int64_t s = pos[ek[e]]++;
        g1[s] = v1[e];
        g2[s] = v2[e];
    }
    for (int k = 0; k < K; ++k)
        lam_next[k] = kpo_scd_reduce(cnt[k + 1] - cnt[k], g1 + cnt[k], g2 + cnt[k], B[k]);
    free(ek);
    free(v1);
    free(v2);
    free(cnt);
    free(g1);
    free(g2);
    free(pos);
    return total;
}

int kpo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
