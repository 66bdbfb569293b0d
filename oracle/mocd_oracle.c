/*
 * mocd_oracle.c -- plain, slow, single-threaded CPU oracle for HP-MOCD
 * (arXiv 2506.01752): one NSGA-II generation of Alg. 1 and every step in it.
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg are the only code that may load
 * this file. The CUDA library never links, loads or calls it, and the two
 * share no source, header, table or helper. Every floating-point expression
 * here is a single IEEE operation on values that both sides compute exactly,
 * compiled with -ffp-contract=off.
 *
 * What each function follows:
 *   philox4x32_10      Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers:
 *                      As Easy as 1, 2, 3" (SC'11), Philox4x32 with 10 rounds.
 *   objectives         Eq. (objectives), Sec. 4.1: f1 = 1 - sum_c |E(c)|/m,
 *                      f2 = sum_c (sum_{v in c} deg v / 2m)^2, kept as the
 *                      exact integers intra = sum_c |E(c)| and S = sum_c D_c^2.
 *   nondominated_sort  Deb et al. 2002 fast non-dominated sort (Alg. 1,
 *                      FastNonDominatedSort; dominance as defined in Sec. 2.2).
 *   crowding           Deb et al. 2002 crowding distance (Alg. 1,
 *                      CrowdingDistanceAssignment; Sec. 4.5.1).
 *   sort_rank_crowd    Alg. 1, SortByRankAndDistance.
 *   select_parents     Alg. 1, TournamentSelection(P, E_S, k = 2).
 *   crossover          Sec. 4.3.1 and Alg. 2 (majority vote, random tie-break,
 *                      skip branch x > C_P copies a random parent).
 *   mutation           Sec. 4.3.2 (nodes with r_v < M_P take the most frequent
 *                      label among their neighbours, random tie-break).
 *   env_select         Alg. 1, R = P u Q and EnvironmentalSelection(R, N_p).
 *   pareto_front       Alg. 1, F_1 = {p : rank(p) = 1}; Alg. 3 SelectSolution
 *                      with Q = 1 - f1 - f2 (Eq. selection).
 *   community_stats    Sec. 4.4 alternative criteria: community count, size
 *                      spread, conductance (definitions at the function).
 *   select_solution    Alg. 3 and the Sec. 4.4 alternatives over a front.
 *
 * Readings where the paper is silent (each one a definition both sides follow):
 *   - E_S parents per crossover (Alg. 1 and the parameter table), chosen by E_S
 *     independent binary tournaments with replacement over P sorted by
 *     (rank asc, crowding desc, position asc); the winner of positions a, b in
 *     that order is position min(a, b).
 *   - Uniform draws are 32-bit words u. Crossover happens iff
 *     u <= floor(C_P * 2^32); node v mutates iff u < floor(M_P * 2^32).
 *     An integer pick in [0, k) is floor(u * k / 2^32).
 *   - "Uniformly at random" among tied labels: the tied labels in ascending
 *     order, index pick(u, t).
 *   - Mutation is synchronous: every selected node reads the post-crossover
 *     child; a node of degree 0 keeps its label.
 *   - Ranks and crowding for the tournament are recomputed on P (Alg. 1).
 *   - Crowding per front and objective: order by (key, position); both ends
 *     +inf; interior += (double)(k[i+1] - k[i-1]) / (double)(k_max - k_min) on
 *     the integer keys, objective 1 then objective 2; zero range adds 0; fronts
 *     of at most two members are all +inf.
 *   - Environmental selection orders R = P positions, then Q positions, by
 *     (rank asc, crowding desc, R index asc) and keeps the first N_p, in that
 *     order, as the next P.
 *   - Dominance keys are the integers (m - intra, S); f1 = (m - intra)/m and
 *     f2 = S/(4 m^2), each one division in double.
 *   - SelectSolution minimises 4 m (m - intra) + S (the same order as Q);
 *     the first member of the front in P order wins ties.
 *   - Initialisation ("random hash-map partitions", "hybrid initialization"):
 *     init_mode 0: label uniform in [0, n), pick(INIT word, n); init_mode 1:
 *     every node starts as its own community (label v), then one synchronous
 *     full-rate neighbour-majority sweep with the INIT word as tie-break.
 *   - Random stream layout (Philox4x32-10, key = (seed low, seed high)):
 *       per individual i and node v:   counter (v, i / 4, g, stage), word i % 4
 *         stage 1 INIT  (g = 0)  initial label pick(u, n)
 *         stage 3 XTIE           crossover tie-break
 *         stage 4 MCOIN          mutation coin r_v
 *         stage 5 MTIE           mutation tie-break
 *       per child i:               counter (w / 4, i, g, 2 SELECT), word w % 4
 *         w = 2j, 2j+1: tournament j draws a, b; w = 2 E_S: crossover coin x;
 *         w = 2 E_S + 1: the parent copied when crossover is skipped.
 *
 * Pins (tests/test_oracle_*.py): Philox published test vectors; objectives of
 * the paper's Fig. 2 and App. E examples, closed forms, networkx modularity;
 * the sort against brute-force Pareto fronts of every partition of small
 * graphs and the longest-dominance-chain rank; crowding closed forms;
 * tournament winner distribution; the App. E crossover / mutation example;
 * planted-partition recovery by a whole run. The exact trajectory of a run
 * depends on the stream layout above, which the paper does not fix: that
 * layout is a definition, not a result, and is pinned only through those
 * properties.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-6)

enum { ST_INIT = 1, ST_SELECT = 2, ST_XTIE = 3, ST_MCOIN = 4, ST_MTIE = 5 };

/* ------------------------------------------------------------------------- */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------- */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t draw_node(uint64_t seed, uint32_t stage, uint32_t gen, uint32_t ind, uint32_t v)
{
    uint32_t ctr[4] = { v, ind / 4u, gen, stage };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[ind % 4u];
}

static uint32_t draw_select(uint64_t seed, uint32_t gen, uint32_t child, uint32_t w)
{
    uint32_t ctr[4] = { w / 4u, child, gen, ST_SELECT };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[w % 4u];
}

/* Integer pick in [0, k) from a 32-bit word: floor(u * k / 2^32). */
uint32_t orc_pick(uint32_t u, uint32_t k)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)k) >> 32);
}

/* floor(p * 2^32) for p in [0, 1]; multiplying by a power of two is exact. */
uint64_t orc_threshold(double p)
{
    return (uint64_t)floor(p * 4294967296.0);
}

/* ------------------------------------------------------------------------- */
/* Objectives, Eq. (objectives)                                              */
/* ------------------------------------------------------------------------- */

/*
 * For one labelling lab[0..n): intra = sum_c |E(c)| (each undirected edge
 * {u, v} with lab[u] == lab[v] counted once) and S = sum_c D_c^2 with
 * D_c = sum_{v : lab[v] = c} deg(v). Labels must lie in [0, n).
 */
int orc_objectives(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                   const int32_t *lab, int64_t *intra_out, int64_t *sumsq_out)
{
    int64_t intra = 0, sumsq = 0;
    int64_t *D = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!D) return ORC_ENOMEM;
    for (int64_t v = 0; v < n; ++v) {
        if (lab[v] < 0 || (int64_t)lab[v] >= n) { free(D); return ORC_EINVAL; }
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int64_t u = col_idx[e];
            if (u > v && lab[u] == lab[v]) intra += 1;
        }
        D[lab[v]] += row_ptr[v + 1] - row_ptr[v];
    }
    for (int64_t c = 0; c < n; ++c) sumsq += D[c] * D[c];
    free(D);
    *intra_out = intra;
    *sumsq_out = sumsq;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* NSGA-II: dominance, non-dominated sort, crowding, ordering                */
/* ------------------------------------------------------------------------- */

/* a dominates b (Sec. 2.2, minimisation of both keys). */
static int dominates(int64_t a1, int64_t a2, int64_t b1, int64_t b2)
{
    return a1 <= b1 && a2 <= b2 && (a1 < b1 || a2 < b2);
}

/*
 * Deb's fast non-dominated sort: n_p = number of points dominating p; the
 * first front is {p : n_p = 0}; removing a front decrements n_q for every q
 * its members dominate; points reaching 0 form the next front. rank[] is
 * 1-based. The dominated sets S_p are recomputed rather than stored.
 */
int orc_nondominated_sort(int32_t N, const int64_t *k1, const int64_t *k2, int32_t *rank)
{
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!cnt || !cur || !nxt) { free(cnt); free(cur); free(nxt); return ORC_ENOMEM; }
    int32_t ncur = 0;
    for (int32_t p = 0; p < N; ++p) {
        cnt[p] = 0;
        for (int32_t q = 0; q < N; ++q)
            if (dominates(k1[q], k2[q], k1[p], k2[p])) cnt[p] += 1;
        if (cnt[p] == 0) { rank[p] = 1; cur[ncur++] = p; }
    }
    int32_t r = 1;
    while (ncur > 0) {
        int32_t nnxt = 0;
        for (int32_t a = 0; a < ncur; ++a) {
            int32_t p = cur[a];
            for (int32_t q = 0; q < N; ++q) {
                if (dominates(k1[p], k2[p], k1[q], k2[q])) {
                    cnt[q] -= 1;
                    if (cnt[q] == 0) { rank[q] = r + 1; nxt[nnxt++] = q; }
                }
            }
        }
        int32_t *t = cur; cur = nxt; nxt = t;
        ncur = nnxt;
        r += 1;
    }
    free(cnt); free(cur); free(nxt);
    return ORC_OK;
}

/* qsort helpers: members ordered by (key, position). The comparators read
 * their keys through thread-local pointers, so that several host threads may
 * run the oracle at once (the tests split one generation's children over
 * threads). */
static _Thread_local const int64_t *g_sort_key;
static int cmp_key_pos(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_sort_key[a] < g_sort_key[b]) return -1;
    if (g_sort_key[a] > g_sort_key[b]) return 1;
    return (a > b) - (a < b);
}

/* Crowding distance per front (reading in the file header). */
int orc_crowding(int32_t N, const int64_t *k1, const int64_t *k2, const int32_t *rank, double *crowd)
{
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!mem) return ORC_ENOMEM;
    int32_t maxr = 0;
    for (int32_t p = 0; p < N; ++p) if (rank[p] > maxr) maxr = rank[p];
    for (int32_t r = 1; r <= maxr; ++r) {
        int32_t F = 0;
        for (int32_t p = 0; p < N; ++p) if (rank[p] == r) mem[F++] = p;
        if (F == 0) continue;
        if (F <= 2) {
            for (int32_t a = 0; a < F; ++a) crowd[mem[a]] = INFINITY;
            continue;
        }
        for (int32_t a = 0; a < F; ++a) crowd[mem[a]] = 0.0;
        for (int obj = 0; obj < 2; ++obj) {
            const int64_t *key = obj == 0 ? k1 : k2;
            g_sort_key = key;
            qsort(mem, (size_t)F, sizeof(int32_t), cmp_key_pos);
            int64_t range = key[mem[F - 1]] - key[mem[0]];
            crowd[mem[0]] = INFINITY;
            crowd[mem[F - 1]] = INFINITY;
            if (range > 0) {
                for (int32_t a = 1; a < F - 1; ++a) {
                    double term = (double)(key[mem[a + 1]] - key[mem[a - 1]]) / (double)range;
                    crowd[mem[a]] = crowd[mem[a]] + term;
                }
            }
        }
    }
    free(mem);
    return ORC_OK;
}

static _Thread_local const int32_t *g_rank;
static _Thread_local const double *g_crowd;
static int cmp_rank_crowd(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_rank[a] != g_rank[b]) return g_rank[a] < g_rank[b] ? -1 : 1;
    if (g_crowd[a] > g_crowd[b]) return -1;
    if (g_crowd[a] < g_crowd[b]) return 1;
    return (a > b) - (a < b);
}

/* order[0..N) = positions sorted by (rank asc, crowding desc, position asc). */
int orc_sort_rank_crowd(int32_t N, const int32_t *rank, const double *crowd, int32_t *order)
{
    for (int32_t p = 0; p < N; ++p) order[p] = p;
    g_rank = rank;
    g_crowd = crowd;
    qsort(order, (size_t)N, sizeof(int32_t), cmp_rank_crowd);
    return ORC_OK;
}

/* Rank, crowding and the (rank, crowding) order of a population's keys. */
int orc_rank_crowd_order(int32_t N, const int64_t *k1, const int64_t *k2,
                         int32_t *rank, double *crowd, int32_t *order)
{
    int rc = orc_nondominated_sort(N, k1, k2, rank);
    if (rc) return rc;
    rc = orc_crowding(N, k1, k2, rank, crowd);
    if (rc) return rc;
    return orc_sort_rank_crowd(N, rank, crowd, order);
}

/* ------------------------------------------------------------------------- */
/* Operators                                                                 */
/* ------------------------------------------------------------------------- */

static int cmp_i32(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/*
 * Most frequent value of x[0..k) (Eq. arg_max). After sorting, equal labels are
 * adjacent and a label's count is the length of its run; the labels whose
 * count is maximal come out in ascending order in ties[0..t). Returns t.
 * scratch must hold k values.
 */
static int32_t mode_ties(int32_t k, const int32_t *x, int32_t *scratch, int32_t *ties)
{
    memcpy(scratch, x, sizeof(int32_t) * (size_t)k);
    qsort(scratch, (size_t)k, sizeof(int32_t), cmp_i32);
    int32_t best = 0, t = 0;
    int32_t a = 0;
    while (a < k) {
        int32_t b = a;
        while (b < k && scratch[b] == scratch[a]) ++b;
        int32_t run = b - a;
        if (run > best) { best = run; t = 0; }
        if (run == best) ties[t++] = scratch[a];
        a = b;
    }
    return t;
}

/* Mode of x[0..k) with the tie among the t most frequent labels broken by u. */
int32_t orc_mode_pick(int32_t k, const int32_t *x, uint32_t u)
{
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * k + 2));
    if (!s) return -1;
    int32_t t = mode_ties(k, x, s, s + k);
    int32_t r = s[k + (int32_t)orc_pick(u, (uint32_t)t)];
    free(s);
    return r;
}

typedef struct {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col_idx;
} orc_graph;

/*
 * Crossover of one child (Alg. 2) from the E parents' label vectors
 * par[j][0..n): per node, the majority label, ties broken by the XTIE word of
 * (child, node). Used only when the crossover coin said "cross".
 */
static int crossover_child(int64_t n, int32_t E, const int32_t *const *par,
                           uint64_t seed, uint32_t gen, uint32_t child, int32_t *out)
{
    int32_t x[64], s[64], ties[64];
    if (E > 64) return ORC_EINVAL;
    for (int64_t v = 0; v < n; ++v) {
        for (int32_t j = 0; j < E; ++j) x[j] = par[j][v];
        int32_t t = mode_ties(E, x, s, ties);
        int32_t pickix = 0;
        if (t > 1) pickix = (int32_t)orc_pick(draw_node(seed, ST_XTIE, gen, child, (uint32_t)v), (uint32_t)t);
        out[v] = ties[pickix];
    }
    return ORC_OK;
}

/*
 * Mutation of one child (Sec. 4.3.2): a node whose MCOIN word is below the
 * threshold, and whose degree is positive, takes the most frequent label among
 * its neighbours in the post-crossover child; ties broken by the MTIE word.
 */
static int mutate_child(const orc_graph *g, const int32_t *child, uint64_t thr_m,
                        uint64_t seed, uint32_t gen, uint32_t ind, int32_t *out)
{
    int64_t dmax = 0;
    for (int64_t v = 0; v < g->n; ++v) {
        int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
        if (d > dmax) dmax = d;
    }
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * dmax + 3));
    if (!x) return ORC_ENOMEM;
    int32_t *s = x + dmax + 1, *ties = s + dmax + 1;
    for (int64_t v = 0; v < g->n; ++v) {
        out[v] = child[v];
        uint32_t coin = draw_node(seed, ST_MCOIN, gen, ind, (uint32_t)v);
        int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
        if ((uint64_t)coin < thr_m && d > 0) {
            for (int64_t e = 0; e < d; ++e) x[e] = child[g->col_idx[g->row_ptr[v] + e]];
            int32_t t = mode_ties((int32_t)d, x, s, ties);
            int32_t pickix = 0;
            if (t > 1) pickix = (int32_t)orc_pick(draw_node(seed, ST_MTIE, gen, ind, (uint32_t)v), (uint32_t)t);
            out[v] = ties[pickix];
        }
    }
    free(x);
    return ORC_OK;
}

/*
 * The App. E worked example with forced draws: crossover of E parents with
 * given tie words (tie[v] used only for ties), then mutation of the nodes with
 * sel[v] != 0 using mtie[v]. Outputs child (post-crossover) and q (mutated).
 */
int orc_operators_forced(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                         int32_t E, const int32_t *parents /* [E][n] */,
                         const uint32_t *xtie, const uint8_t *sel, const uint32_t *mtie,
                         int32_t *child, int32_t *q)
{
    int32_t x[64];
    if (E < 1 || E > 64) return ORC_EINVAL;
    for (int64_t v = 0; v < n; ++v) {
        for (int32_t j = 0; j < E; ++j) x[j] = parents[(int64_t)j * n + v];
        child[v] = orc_mode_pick(E, x, xtie[v]);
    }
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        q[v] = child[v];
        if (sel[v] && d > 0) {
            int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)d);
            if (!nb) return ORC_ENOMEM;
            for (int64_t e = 0; e < d; ++e) nb[e] = child[col_idx[row_ptr[v] + e]];
            q[v] = orc_mode_pick((int32_t)d, nb, mtie[v]);
            free(nb);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Population, tournament, one generation                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t pop_size;    /* N_p */
    int32_t n_parents;   /* E_S */
    double p_crossover;  /* C_P */
    double p_mutation;   /* M_P */
    uint64_t seed;
    int32_t init_mode;
} orc_params;

static int check_params(const orc_params *pr)
{
    if (pr->pop_size < 1 || pr->n_parents < 1 || pr->n_parents > 64) return ORC_EINVAL;
    if (!(pr->p_crossover >= 0.0 && pr->p_crossover <= 1.0)) return ORC_EINVAL;
    if (!(pr->p_mutation >= 0.0 && pr->p_mutation <= 1.0)) return ORC_EINVAL;
    if (pr->init_mode != 0 && pr->init_mode != 1) return ORC_EINVAL;
    return ORC_OK;
}

/* InitializePopulation (Alg. 1) for init_mode 0: label of node v in
 * individual i is pick(INIT word, n), i.e. uniform in [0, n). P is [N_p][n]. */
int orc_init_population(int64_t n, const orc_params *pr, int32_t *P)
{
    int rc = check_params(pr);
    if (rc) return rc;
    if (pr->init_mode != 0) return ORC_EINVAL;
    for (int32_t i = 0; i < pr->pop_size; ++i)
        for (int64_t v = 0; v < n; ++v)
            P[(int64_t)i * n + v] = (int32_t)orc_pick(draw_node(pr->seed, ST_INIT, 0, (uint32_t)i, (uint32_t)v), (uint32_t)n);
    return ORC_OK;
}

/* init_mode 1: singletons (label v), then one synchronous neighbour-majority
 * sweep of every node of positive degree (the mutation rule of Sec. 4.3.2 at
 * rate 1), ties broken by the INIT word of (individual, node). */
int orc_init_population_sweep(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                              const orc_params *pr, int32_t *P)
{
    int rc = check_params(pr);
    if (rc) return rc;
    int64_t dmax = 0;
    for (int64_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] - row_ptr[v] > dmax) dmax = row_ptr[v + 1] - row_ptr[v];
    int32_t *single = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * dmax + 3));
    if (!single || !x) { free(single); free(x); return ORC_ENOMEM; }
    int32_t *s = x + dmax + 1, *ties = s + dmax + 1;
    for (int64_t v = 0; v < n; ++v) single[v] = (int32_t)v;
    for (int32_t i = 0; i < pr->pop_size; ++i) {
        for (int64_t v = 0; v < n; ++v) {
            int64_t d = row_ptr[v + 1] - row_ptr[v];
            int32_t lab = single[v];
            if (d > 0) {
                for (int64_t e = 0; e < d; ++e) x[e] = single[col_idx[row_ptr[v] + e]];
                int32_t t = mode_ties((int32_t)d, x, s, ties);
                int32_t k = t > 1 ? (int32_t)orc_pick(draw_node(pr->seed, ST_INIT, 0, (uint32_t)i, (uint32_t)v), (uint32_t)t) : 0;
                lab = ties[k];
            }
            P[(int64_t)i * n + v] = lab;
        }
    }
    free(single); free(x);
    return ORC_OK;
}

/*
 * TournamentSelection for every child of generation gen: P (keys in P order)
 * is ranked, crowded and sorted; parent j of child i is the winner of the
 * binary tournament between sorted positions a and b, i.e. sorted position
 * min(a, b). Outputs: par[i*E + j] = P position, xo[i] = 1 if crossover
 * happens, skip[i] = index j of the parent copied when it does not.
 */
int orc_select_parents(const orc_params *pr, uint32_t gen, const int64_t *k1, const int64_t *k2,
                       int32_t *par, int32_t *xo, int32_t *skip)
{
    int32_t Np = pr->pop_size, E = pr->n_parents;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)Np);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)Np);
    double *crowd = (double *)malloc(sizeof(double) * (size_t)Np);
    if (!rank || !order || !crowd) { free(rank); free(order); free(crowd); return ORC_ENOMEM; }
    int rc = orc_rank_crowd_order(Np, k1, k2, rank, crowd, order);
    if (rc) { free(rank); free(order); free(crowd); return rc; }
    uint64_t thr_c = orc_threshold(pr->p_crossover);
    for (int32_t i = 0; i < Np; ++i) {
        for (int32_t j = 0; j < E; ++j) {
            uint32_t a = orc_pick(draw_select(pr->seed, gen, (uint32_t)i, (uint32_t)(2 * j)), (uint32_t)Np);
            uint32_t b = orc_pick(draw_select(pr->seed, gen, (uint32_t)i, (uint32_t)(2 * j + 1)), (uint32_t)Np);
            uint32_t win = a < b ? a : b;
            par[i * E + j] = order[win];
        }
        uint32_t x = draw_select(pr->seed, gen, (uint32_t)i, (uint32_t)(2 * E));
        xo[i] = (uint64_t)x <= thr_c ? 1 : 0;
        skip[i] = (int32_t)orc_pick(draw_select(pr->seed, gen, (uint32_t)i, (uint32_t)(2 * E + 1)), (uint32_t)E);
    }
    free(rank); free(order); free(crowd);
    return ORC_OK;
}

/*
 * Offspring generation (Alg. 1 parallel map, done here one child after the
 * other) and evaluation: Q[i] = mutation(crossover(parents of i)), with keys,
 * for the children i0 <= i < i1 (Q, qk1, qk2 are indexed by child).
 */
int orc_make_offspring_range(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             const orc_params *pr, uint32_t gen, const int32_t *P,
                             const int64_t *k1, const int64_t *k2, int32_t i0, int32_t i1,
                             int32_t *Q, int64_t *qk1, int64_t *qk2)
{
    int32_t Np = pr->pop_size, E = pr->n_parents;
    orc_graph g = { n, row_ptr, col_idx };
    int64_t m = row_ptr[n] / 2;
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)(Np * E));
    int32_t *xo = (int32_t *)malloc(sizeof(int32_t) * (size_t)Np);
    int32_t *skip = (int32_t *)malloc(sizeof(int32_t) * (size_t)Np);
    int32_t *child = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    const int32_t *pp[64];
    if (!par || !xo || !skip || !child) { free(par); free(xo); free(skip); free(child); return ORC_ENOMEM; }
    int rc = orc_select_parents(pr, gen, k1, k2, par, xo, skip);
    uint64_t thr_m = orc_threshold(pr->p_mutation);
    if (i0 < 0) i0 = 0;
    if (i1 > Np) i1 = Np;
    for (int32_t i = i0; i < i1 && rc == ORC_OK; ++i) {
        for (int32_t j = 0; j < E; ++j) pp[j] = P + (int64_t)par[i * E + j] * n;
        if (xo[i]) rc = crossover_child(n, E, pp, pr->seed, gen, (uint32_t)i, child);
        else memcpy(child, pp[skip[i]], sizeof(int32_t) * (size_t)n);
        if (rc) break;
        rc = mutate_child(&g, child, thr_m, pr->seed, gen, (uint32_t)i, Q + (int64_t)i * n);
        if (rc) break;
        int64_t intra, sumsq;
        rc = orc_objectives(n, row_ptr, col_idx, Q + (int64_t)i * n, &intra, &sumsq);
        qk1[i] = m - intra;
        qk2[i] = sumsq;
    }
    free(par); free(xo); free(skip); free(child);
    return rc;
}

/* All N_p children of generation gen (the "parallel map" of Alg. 1). */
int orc_make_offspring(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const orc_params *pr, uint32_t gen, const int32_t *P,
                       const int64_t *k1, const int64_t *k2,
                       int32_t *Q, int64_t *qk1, int64_t *qk2)
{
    return orc_make_offspring_range(n, row_ptr, col_idx, pr, gen, P, k1, k2, 0, pr->pop_size, Q, qk1, qk2);
}

/*
 * EnvironmentalSelection (Alg. 1): R = P (R index 0..N_p-1) then Q (N_p..),
 * ranked and crowded as one population, ordered by (rank, crowding desc,
 * R index); the first N_p form the next P. keep[k] = R index of new P[k].
 */
int orc_env_select(int32_t Np, const int64_t *rk1, const int64_t *rk2, int32_t *keep)
{
    int32_t N = 2 * Np;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *crowd = (double *)malloc(sizeof(double) * (size_t)N);
    if (!rank || !order || !crowd) { free(rank); free(order); free(crowd); return ORC_ENOMEM; }
    int rc = orc_rank_crowd_order(N, rk1, rk2, rank, crowd, order);
    if (rc == ORC_OK) for (int32_t k = 0; k < Np; ++k) keep[k] = order[k];
    free(rank); free(order); free(crowd);
    return rc;
}

/*
 * G generations of Alg. 1 starting after generation gen0 (the first one run
 * is gen0 + 1). P [N_p][n] and its keys (k1 = m - intra, k2 = S) are updated
 * in place and stay in P order.
 */
int orc_run(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const orc_params *pr,
            uint32_t gen0, int32_t G, int32_t *P, int64_t *k1, int64_t *k2)
{
    int rc = check_params(pr);
    if (rc) return rc;
    int32_t Np = pr->pop_size;
    size_t cells = (size_t)Np * (size_t)(n > 0 ? n : 1);
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * cells);
    int32_t *Pn = (int32_t *)malloc(sizeof(int32_t) * cells);
    int64_t *rk1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * Np));
    int64_t *rk2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * Np));
    int32_t *keep = (int32_t *)malloc(sizeof(int32_t) * (size_t)Np);
    if (!Q || !Pn || !rk1 || !rk2 || !keep) { rc = ORC_ENOMEM; goto done; }
    for (int32_t step = 0; step < G; ++step) {
        uint32_t gen = gen0 + 1u + (uint32_t)step;
        rc = orc_make_offspring(n, row_ptr, col_idx, pr, gen, P, k1, k2, Q, rk1 + Np, rk2 + Np);
        if (rc) goto done;
        memcpy(rk1, k1, sizeof(int64_t) * (size_t)Np);
        memcpy(rk2, k2, sizeof(int64_t) * (size_t)Np);
        rc = orc_env_select(Np, rk1, rk2, keep);
        if (rc) goto done;
        for (int32_t k = 0; k < Np; ++k) {
            int32_t r = keep[k];
            const int32_t *src = r < Np ? P + (int64_t)r * n : Q + (int64_t)(r - Np) * n;
            memcpy(Pn + (int64_t)k * n, src, sizeof(int32_t) * (size_t)n);
            k1[k] = rk1[r];
            k2[k] = rk2[r];
        }
        memcpy(P, Pn, sizeof(int32_t) * cells);
    }
done:
    free(Q); free(Pn); free(rk1); free(rk2); free(keep);
    return rc;
}

/* Initial population and its evaluation (Alg. 1, phases 1 and 2). */
int orc_population_init(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                        const orc_params *pr, int32_t *P, int64_t *k1, int64_t *k2)
{
    int rc = pr->init_mode == 1 ? orc_init_population_sweep(n, row_ptr, col_idx, pr, P)
                                : orc_init_population(n, pr, P);
    if (rc) return rc;
    int64_t m = row_ptr[n] / 2;
    for (int32_t i = 0; i < pr->pop_size; ++i) {
        int64_t intra, sumsq;
        rc = orc_objectives(n, row_ptr, col_idx, P + (int64_t)i * n, &intra, &sumsq);
        if (rc) return rc;
        k1[i] = m - intra;
        k2[i] = sumsq;
    }
    return ORC_OK;
}

/*
 * Phase 4 of Alg. 1: F_1 = members of P with rank 1 (P recomputed on its own
 * keys), listed in P order; best = index into that list of the member that
 * minimises 4 m k1 + k2 (maximises Q = 1 - f1 - f2, Alg. 3), first one on
 * ties.
 */
int orc_pareto_front(int32_t Np, const int64_t *k1, const int64_t *k2, int64_t m,
                     int32_t *count, int32_t *members, int32_t *best)
{
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)Np);
    if (!rank) return ORC_ENOMEM;
    int rc = orc_nondominated_sort(Np, k1, k2, rank);
    if (rc) { free(rank); return rc; }
    int32_t c = 0, b = -1;
    int64_t bestK = 0;
    for (int32_t p = 0; p < Np; ++p) {
        if (rank[p] != 1) continue;
        int64_t K = 4 * m * k1[p] + k2[p];
        if (b < 0 || K < bestK) { b = c; bestK = K; }
        members[c++] = p;
    }
    *count = c;
    *best = b;
    free(rank);
    return ORC_OK;
}

/* f1 and f2 from the integer keys: one IEEE division each. */
void orc_objective_values(int64_t m, int64_t k1, int64_t k2, double *f1, double *f2)
{
    *f1 = (double)k1 / (double)m;
    *f2 = (double)k2 / (double)(4 * m * m);
}

/*
 * Community statistics of `count` labelings (Sec. 4.4, the alternative
 * criteria Alg. 3 leaves to the user). For labeling i and its communities
 * V_c: k = number of non-empty communities; sumsq = sum_c |V_c|^2;
 * phi_c = cut_c / min(vol_c, 2m - vol_c) as one IEEE division (0 if cut_c is
 * 0), cut_c = edges with one endpoint in V_c, vol_c = sum of degrees in V_c;
 * mean_phi = (exact sum_c phi_c, rounded once to nearest double) / k;
 * max_phi = max_c phi_c. The exact sum: every phi_c is a double in
 * [2^-30, 1] or 0, so phi_c * 2^88 is an integer below 2^89; those integers
 * are added in 128 bits and the total converted once.
 */
int orc_community_stats(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int32_t count,
                        const int32_t *labels, int64_t *k_out, int64_t *sumsq_out,
                        double *mean_phi, double *max_phi)
{
    int64_t *size = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *vol = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *cut = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!size || !vol || !cut) { free(size); free(vol); free(cut); return ORC_ENOMEM; }
    const int64_t two_m = row_ptr[n];
    for (int32_t i = 0; i < count; ++i) {
        const int32_t *L = labels + (int64_t)i * n;
        memset(size, 0, sizeof(int64_t) * (size_t)n);
        memset(vol, 0, sizeof(int64_t) * (size_t)n);
        memset(cut, 0, sizeof(int64_t) * (size_t)n);
        for (int64_t v = 0; v < n; ++v) {
            if (L[v] < 0 || (int64_t)L[v] >= n) { free(size); free(vol); free(cut); return ORC_EINVAL; }
            size[L[v]] += 1;
            vol[L[v]] += row_ptr[v + 1] - row_ptr[v];
            for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
                if (L[col_idx[e]] != L[v]) cut[L[v]] += 1;
        }
        int64_t k = 0, sq = 0;
        unsigned __int128 sum = 0;
        double mx = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            if (!size[c]) continue;
            k += 1;
            sq += size[c] * size[c];
            if (!cut[c]) continue;
            const int64_t den = vol[c] < two_m - vol[c] ? vol[c] : two_m - vol[c];
            const double phi = (double)cut[c] / (double)den;
            if (phi > mx) mx = phi;
            sum += (unsigned __int128)ldexp(phi, 88);
        }
        k_out[i] = k;
        sumsq_out[i] = sq;
        mean_phi[i] = ldexp((double)sum, -88) / (double)k;
        max_phi[i] = mx;
    }
    free(size); free(vol); free(cut);
    return ORC_OK;
}

/* Sign of var_a - var_b, var = (k sumsq - n^2) / k^2, exactly: integer parts
 * of the two quotients first, then the remainders cross-multiplied (each
 * remainder is below k^2 < 2^60, so the products fit in 128 bits). */
static int variance_cmp(int64_t n, int64_t ka, int64_t sa, int64_t kb, int64_t sb)
{
    const unsigned __int128 n2 = (unsigned __int128)n * (unsigned __int128)n;
    const unsigned __int128 na = (unsigned __int128)ka * (unsigned __int128)sa - n2;
    const unsigned __int128 nb = (unsigned __int128)kb * (unsigned __int128)sb - n2;
    const unsigned __int128 da = (unsigned __int128)ka * (unsigned __int128)ka;
    const unsigned __int128 db = (unsigned __int128)kb * (unsigned __int128)kb;
    const unsigned __int128 qa = na / da, qb = nb / db;
    if (qa != qb) return qa < qb ? -1 : 1;
    const unsigned __int128 ra = (na % da) * db, rb = (nb % db) * da;
    return ra < rb ? -1 : ra > rb ? 1 : 0;
}

/*
 * Index of the member a selection criterion prefers among `count` front
 * members (Alg. 3 and the alternatives of Sec. 4.4): criterion 0 largest Q
 * (the least 4 m k1 + k2), 1 number of communities nearest `target`, 2 least
 * community-size variance, 3 least mean conductance, 4 least maximum
 * conductance; ties go to the larger Q, then to the earlier member.
 */
int32_t orc_select_solution(int32_t count, int64_t m, int64_t n, const int64_t *k1, const int64_t *k2,
                            const int64_t *k, const int64_t *sumsq, const double *mean_phi,
                            const double *max_phi, int32_t criterion, int64_t target)
{
    int32_t best = -1;
    for (int32_t a = 0; a < count; ++a) {
        if (best < 0) { best = a; continue; }
        const int32_t b = best;
        int d = 0;
        if (criterion == 1) {
            const int64_t xa = k[a] > target ? k[a] - target : target - k[a];
            const int64_t xb = k[b] > target ? k[b] - target : target - k[b];
            d = xa < xb ? -1 : xa > xb ? 1 : 0;
        } else if (criterion == 2) {
            d = variance_cmp(n, k[a], sumsq[a], k[b], sumsq[b]);
        } else if (criterion == 3) {
            d = mean_phi[a] < mean_phi[b] ? -1 : mean_phi[a] > mean_phi[b] ? 1 : 0;
        } else if (criterion == 4) {
            d = max_phi[a] < max_phi[b] ? -1 : max_phi[a] > max_phi[b] ? 1 : 0;
        }
        if (d == 0) {
            const int64_t Ka = 4 * m * k1[a] + k2[a], Kb = 4 * m * k1[b] + k2[b];
            d = Ka < Kb ? -1 : 0;
        }
        if (d < 0) best = a;
    }
    return best;
}
