/*
 * CPU oracle for Monte Carlo simulation of the independent cascade (IC) and
 * linear threshold (LT) diffusion models.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C written to be read
 * against the paper (CyNetDiff, arXiv 2404.17059).  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never calls it, and the two share no code.  It shares with the GPU path only
 * the *definition* of the random numbers (a Philox4x32-10 counter layout,
 * below), implemented here independently.
 *
 * What is computed (Sec. 2, "Diffusion Models"; Sec. 3, "Algorithms"):
 *   IC: from seed set S, a node v newly active at step t gets one chance to
 *       activate each inactive out-neighbour w, succeeding with probability
 *       p_{v,w}; success makes w active at t+1; runs until no activation.
 *   LT: node v draws a threshold theta_v uniform on [0,1]; at each step every
 *       inactive node whose active in-neighbours' total weight reaches its
 *       threshold becomes active; runs until no activation.
 *   Observation 1 (Sec. 3): a non-seed node activated at t has an in-neighbour
 *   activated at t-1, so only out-neighbours of the previous step's newly
 *   active nodes are examined: a FIFO breadth-first traversal per trial.
 *   A second, deliberately different "full sweep" mode loops over every edge
 *   (IC) / recomputes every node's active in-weight (LT) at every step, the
 *   per-step whole-graph loop the paper attributes to NDlib (Sec. 1).
 *
 * Readings fixed where the paper is silent or ambiguous:
 *   R1 random numbers: Philox4x32-10 (Salmon et al., SC'11), key =
 *      (lo32(rng_seed), hi32(rng_seed)).  For trial t (g = t >> 2, j = t & 3):
 *        IC coin of edge e   = philox(e, lo32(g), 0, hi32(g))[j]
 *        LT threshold of v   = philox(v, lo32(g), 1, hi32(g))[j]
 *      e is the index of the edge in the caller's CSR `col` array.
 *   R2 IC probability p (fp32) becomes thr = floor(p * 2^32) for p < 1 and
 *      thr = 0xFFFFFFFF ("always") for p == 1; the edge is live in trial t iff
 *      thr == 0xFFFFFFFF or coin < thr.  Live probability is exactly thr/2^32.
 *   R3 LT weights are uint32 fixed point with in-weight sums <= 2^32 - 1; v
 *      activates iff (sum of active in-weights) > theta (theta a uint32), so
 *      P(activate | sum) = sum / 2^32, and a node with no active in-weight
 *      never activates.
 *   R4 Spread counts the seeds; duplicate seeds count once.
 *   R5 edge checks = sum over trials of sum over active nodes of out-degree.
 *   R6 levels: seeds are level 0; a node's level is its activation step.
 *      With max_levels >= 1, nodes at level max_levels are not expanded and
 *      their existence is reported as "limit hit".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_OK 0
#define ORACLE_LIMIT 1
#define ORACLE_EINVAL (-1)
#define ORACLE_EOVERFLOW (-2)
#define ORACLE_ENOMEM (-3)

/* ---------------------------------------------------------------- Philox */
/* Philox4x32 round: two 32x32->64 multiplications, the high halves xored with
 * the other counter words and the round key (Salmon et al. SC'11, Sec. 4). */
static void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t r0 = (uint32_t)(prod1 >> 32) ^ c[1] ^ k0;
    uint32_t r1 = (uint32_t)prod1;
    uint32_t r2 = (uint32_t)(prod0 >> 32) ^ c[3] ^ k1;
    uint32_t r3 = (uint32_t)prod0;
    c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}

/* Ten rounds; the key is bumped by the Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], uint64_t rng_seed, uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = (uint32_t)(rng_seed & 0xFFFFFFFFu);
    uint32_t k1 = (uint32_t)(rng_seed >> 32);
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c, k0, k1);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Many blocks at once (for tests): ctr is count x 4, out is count x 4. */
void oracle_philox_many(const uint32_t *ctr, int64_t count, uint64_t rng_seed, uint32_t *out)
{
    for (int64_t i = 0; i < count; ++i)
        oracle_philox4x32_10(ctr + 4 * i, rng_seed, out + 4 * i);
}

/* R1: the uint32 drawn for (trial, index, domain). */
static uint32_t draw(uint64_t rng_seed, int64_t trial, int64_t index, uint32_t domain)
{
    uint64_t g = (uint64_t)trial >> 2;
    uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(g & 0xFFFFFFFFu), domain, (uint32_t)(g >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, rng_seed, out);
    return out[trial & 3];
}

uint32_t oracle_ic_coin(uint64_t rng_seed, int64_t trial, int64_t edge)
{
    return draw(rng_seed, trial, edge, 0u);
}

uint32_t oracle_lt_theta(uint64_t rng_seed, int64_t trial, int64_t node)
{
    return draw(rng_seed, trial, node, 1u);
}

/* R2 */
#define ALWAYS 0xFFFFFFFFu
uint32_t oracle_ic_threshold(float p)
{
    if (p == 1.0f) return ALWAYS;
    return (uint32_t)floor((double)p * 4294967296.0);
}

static int ic_live(uint64_t rng_seed, int64_t trial, int64_t edge, uint32_t thr)
{
    if (thr == ALWAYS) return 1;
    return oracle_ic_coin(rng_seed, trial, edge) < thr;
}

/* ---------------------------------------------------------------- checks */
static int check_csr(int32_t n, const int32_t *row_ptr, const int32_t *col)
{
    if (n <= 0 || row_ptr == NULL) return 0;
    if (row_ptr[0] != 0) return 0;
    for (int32_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u]) return 0;
    int32_t m = row_ptr[n];
    if (m > 0 && col == NULL) return 0;
    for (int32_t e = 0; e < m; ++e)
        if (col[e] < 0 || col[e] >= n) return 0;
    return 1;
}

/* ---------------------------------------------------------------- one trial */
/* Each trial routine fills level[0..n) (activation step or -1) and returns 1 if
 * the level cap was reached (R6). */

static int ic_trial_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *thr,
                        const int32_t *seeds, int32_t n_seeds, uint64_t rng_seed, int64_t t,
                        int32_t max_levels, int32_t *level, int32_t *queue)
{
    int64_t head = 0, tail = 0;
    for (int32_t v = 0; v < n; ++v) level[v] = -1;
    for (int32_t i = 0; i < n_seeds; ++i) {
        int32_t s = seeds[i];
        if (level[s] < 0) { level[s] = 0; queue[tail++] = s; }
    }
    int limit = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        if (max_levels > 0 && level[u] >= max_levels) { limit = 1; continue; }
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] < 0 && ic_live(rng_seed, t, e, thr[e])) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    return limit;
}

static int lt_trial_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w,
                        const int32_t *seeds, int32_t n_seeds, uint64_t rng_seed, int64_t t,
                        int32_t max_levels, int32_t *level, int32_t *queue, uint64_t *acc)
{
    int64_t head = 0, tail = 0;
    for (int32_t v = 0; v < n; ++v) { level[v] = -1; acc[v] = 0; }
    for (int32_t i = 0; i < n_seeds; ++i) {
        int32_t s = seeds[i];
        if (level[s] < 0) { level[s] = 0; queue[tail++] = s; }
    }
    int limit = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        if (max_levels > 0 && level[u] >= max_levels) { limit = 1; continue; }
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] >= 0) continue;
            acc[v] += w[e];
            if (acc[v] > (uint64_t)oracle_lt_theta(rng_seed, t, v)) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    return limit;
}

static int ic_trial_sweep(int32_t n, int32_t m, const int32_t *src, const int32_t *col, const uint32_t *thr,
                          const int32_t *seeds, int32_t n_seeds, uint64_t rng_seed, int64_t t,
                          int32_t max_levels, int32_t *level)
{
    for (int32_t v = 0; v < n; ++v) level[v] = -1;
    for (int32_t i = 0; i < n_seeds; ++i) level[seeds[i]] = 0;
    for (int32_t L = 0;; ++L) {
        if (max_levels > 0 && L >= max_levels) break;
        int any = 0;
        for (int32_t e = 0; e < m; ++e) {
            if (level[src[e]] != L) continue;
            int32_t v = col[e];
            if (level[v] >= 0) continue;
            if (ic_live(rng_seed, t, e, thr[e])) { level[v] = L + 1; any = 1; }
        }
        if (!any) break;
    }
    int limit = 0;
    if (max_levels > 0)
        for (int32_t v = 0; v < n; ++v)
            if (level[v] == max_levels) limit = 1;
    return limit;
}

static int lt_trial_sweep(int32_t n, int32_t m, const int32_t *src, const int32_t *col, const uint32_t *w,
                          const int32_t *seeds, int32_t n_seeds, uint64_t rng_seed, int64_t t,
                          int32_t max_levels, int32_t *level, uint64_t *sum)
{
    for (int32_t v = 0; v < n; ++v) level[v] = -1;
    for (int32_t i = 0; i < n_seeds; ++i) level[seeds[i]] = 0;
    for (int32_t L = 0;; ++L) {
        if (max_levels > 0 && L >= max_levels) break;
        /* total weight of in-neighbours active by the end of step L, from scratch */
        for (int32_t v = 0; v < n; ++v) sum[v] = 0;
        for (int32_t e = 0; e < m; ++e)
            if (level[src[e]] >= 0) sum[col[e]] += w[e];
        int any = 0;
        for (int32_t v = 0; v < n; ++v) {
            if (level[v] >= 0) continue;
            if (sum[v] > (uint64_t)oracle_lt_theta(rng_seed, t, v)) { level[v] = L + 1; any = 1; }
        }
        if (!any) break;
    }
    int limit = 0;
    if (max_levels > 0)
        for (int32_t v = 0; v < n; ++v)
            if (level[v] == max_levels) limit = 1;
    return limit;
}

/* ---------------------------------------------------------------- driver */
/*
 * model: 0 = IC (uses ic_prob), 1 = LT (uses lt_weight).
 * mode:  0 = breadth-first traversal, 1 = full sweep.
 * Trials first_trial .. first_trial+n_trials-1.  Every output may be NULL:
 *   spread_out[i]        spread of trial first_trial+i (R4)
 *   node_count_out[v]    number of these trials in which v is active
 *   edge_checks_out[0]   R5 summed over these trials
 *   level_counts_out[L]  number of (trial, node) pairs activated at step L, L < level_counts_len
 *   active_out[i*n+v]    1 if v is active in trial first_trial+i
 *   level_out[i*n+v]     activation step of v in that trial, or -1
 * Returns ORACLE_OK, ORACLE_LIMIT (some trial reached max_levels), or < 0 on bad input.
 */
int32_t oracle_simulate(int32_t model, int32_t mode, int32_t n, const int32_t *row_ptr, const int32_t *col,
                        const float *ic_prob, const uint32_t *lt_weight,
                        const int32_t *seeds, int32_t n_seeds,
                        int64_t first_trial, int64_t n_trials, uint64_t rng_seed, int32_t max_levels,
                        int32_t *spread_out, int32_t *node_count_out, int64_t *edge_checks_out,
                        int64_t *level_counts_out, int32_t level_counts_len,
                        uint8_t *active_out, int32_t *level_out)
{
    if (!check_csr(n, row_ptr, col)) return ORACLE_EINVAL;
    if (n_trials < 0 || first_trial < 0 || n_seeds < 0 || (n_seeds > 0 && seeds == NULL)) return ORACLE_EINVAL;
    for (int32_t i = 0; i < n_seeds; ++i)
        if (seeds[i] < 0 || seeds[i] >= n) return ORACLE_EINVAL;
    int32_t m = row_ptr[n];

    uint32_t *thr = NULL;
    if (model == 0) {
        if (ic_prob == NULL && m > 0) return ORACLE_EINVAL;
        thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
        if (!thr) return ORACLE_ENOMEM;
        for (int32_t e = 0; e < m; ++e) {
            float p = ic_prob[e];
            if (!(p >= 0.0f && p <= 1.0f)) { free(thr); return ORACLE_EINVAL; }  /* also rejects NaN */
            thr[e] = oracle_ic_threshold(p);
        }
    } else if (model == 1) {
        if (lt_weight == NULL && m > 0) return ORACLE_EINVAL;
        uint64_t *in_sum = (uint64_t *)calloc((size_t)n, sizeof(uint64_t));
        if (!in_sum) return ORACLE_ENOMEM;
        for (int32_t e = 0; e < m; ++e) in_sum[col[e]] += lt_weight[e];
        int over = 0;
        for (int32_t v = 0; v < n; ++v) if (in_sum[v] > 0xFFFFFFFFull) over = 1;
        free(in_sum);
        if (over) return ORACLE_EOVERFLOW;
    } else {
        return ORACLE_EINVAL;
    }

    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *acc = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!level || !queue || !acc || !src) {
        free(level); free(queue); free(acc); free(src); free(thr);
        return ORACLE_ENOMEM;
    }
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) src[e] = u;

    if (node_count_out) memset(node_count_out, 0, sizeof(int32_t) * (size_t)n);
    if (level_counts_out && level_counts_len > 0) memset(level_counts_out, 0, sizeof(int64_t) * (size_t)level_counts_len);
    int64_t checks = 0;
    int any_limit = 0;

    for (int64_t i = 0; i < n_trials; ++i) {
        int64_t t = first_trial + i;
        int lim;
        if (model == 0 && mode == 0)
            lim = ic_trial_bfs(n, row_ptr, col, thr, seeds, n_seeds, rng_seed, t, max_levels, level, queue);
        else if (model == 0)
            lim = ic_trial_sweep(n, m, src, col, thr, seeds, n_seeds, rng_seed, t, max_levels, level);
        else if (mode == 0)
            lim = lt_trial_bfs(n, row_ptr, col, lt_weight, seeds, n_seeds, rng_seed, t, max_levels, level, queue, acc);
        else
            lim = lt_trial_sweep(n, m, src, col, lt_weight, seeds, n_seeds, rng_seed, t, max_levels, level, acc);
        any_limit |= lim;

        int32_t spread = 0;
        for (int32_t v = 0; v < n; ++v) {
            int32_t L = level[v];
            if (L < 0) continue;
            spread += 1;
            checks += row_ptr[v + 1] - row_ptr[v];
            if (node_count_out) node_count_out[v] += 1;
            if (level_counts_out && L < level_counts_len) level_counts_out[L] += 1;
        }
        if (spread_out) spread_out[i] = spread;
        if (active_out)
            for (int32_t v = 0; v < n; ++v) active_out[i * (int64_t)n + v] = (uint8_t)(level[v] >= 0);
        if (level_out)
            memcpy(level_out + i * (int64_t)n, level, sizeof(int32_t) * (size_t)n);
    }
    if (edge_checks_out) edge_checks_out[0] = checks;

    free(level); free(queue); free(acc); free(src); free(thr);
    return any_limit ? ORACLE_LIMIT : ORACLE_OK;
}
