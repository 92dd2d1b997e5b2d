/*
 * cnd.h -- C ABI of the GB300 (sm_103a) Monte Carlo engine for the independent
 * cascade (IC) and linear threshold (LT) diffusion models.
 *
 * The models are the ones stated in CyNetDiff (arXiv 2404.17059), Sec. 2
 * "Diffusion Models"; the graph is a directed CSR graph (Sec. 3 "Data
 * Structures"); the quantity estimated is sigma(S), the expected number of
 * active nodes when the process started from seed set S stops (Sec. 2
 * "Influence Maximization").  One call runs many independent trials from one
 * seed set and reports, per trial, how many nodes ended active (the spread)
 * and, per node, in how many trials it ended active (the data of the paper's
 * activation heatmap, Sec. 4 "Visualizations").
 *
 * Definitions that bind every entry point (the paper fixes no random number
 * generator or rounding; these are this library's readings):
 *
 *   Random numbers.  Philox4x32-10 (Salmon et al., SC'11) with key
 *   (lo32(rng_seed), hi32(rng_seed)).  For trial t let g = t >> 2, j = t & 3:
 *     IC coin of edge e      = Philox(e, lo32(g), 0, hi32(g))[j]
 *     LT threshold of node v = Philox(v, lo32(g), 1, hi32(g))[j]
 *   e is the position of the edge in the caller's `col` array.  A trial is
 *   therefore a pure function of (graph, seeds, rng_seed, t): results do not
 *   depend on how trials are grouped, on traversal order or on direction.
 *
 *   IC.  Probability p (fp32, 0 <= p <= 1) becomes the threshold
 *   thr = floor(p * 2^32) for p < 1 and thr = 0xFFFFFFFF ("always") for
 *   p == 1.  Edge e is live in trial t iff thr == 0xFFFFFFFF or coin < thr, so
 *   its live probability is exactly thr / 2^32.  Because every edge's coin is
 *   fixed per trial, the set of active nodes is the set reachable from S over
 *   live edges (each newly active node gets one chance per inactive
 *   out-neighbour, Sec. 2).
 *
 *   LT.  Weights are uint32 fixed point: the weight w of edge u->v is the
 *   influence of u on v, and for every node the in-weights sum to at most
 *   2^32 - 1 (the fixed-point form of "sum <= 1", Sec. 2).  Node v becomes
 *   active in the step after the summed weight of its active in-neighbours
 *   exceeds its threshold theta (a uint32): activation probability given total
 *   W is exactly W / 2^32, and a node with no active in-weight never activates.
 *
 *   Steps.  Seeds are active at step 0 (duplicates count once); a node
 *   activated at step L+1 has an in-neighbour activated at step L (Sec. 3,
 *   Observation 1).  Expansion is level-synchronous, so a node's step is its
 *   activation time in the paper's process.
 *
 *   Spread counts the seeds.  Edge checks (throughput unit) = sum over trials
 *   of sum over active nodes of out-degree: every active node examines its
 *   out-row once per trial (Sec. 3 "Algorithms": work proportional to the
 *   edges incident to activated nodes).
 *
 * Conventions.  Inputs are copied: the caller keeps ownership of its arrays.
 * Outputs are caller-allocated.  Unless `device_ptrs` is set in the options,
 * seeds and outputs are host pointers and the call returns after the results
 * are written.  Every function returns a cnd_status; on failure
 * cnd_last_error() describes the failure in a thread-local string.  Calls on
 * one graph from several host threads are allowed when they use distinct
 * streams.  Nothing here falls back to the CPU.
 */
#ifndef CND_H
#define CND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cnd_graph cnd_graph; /* opaque; device copy owned by the library */
typedef int32_t cnd_status;

#define CND_OK 0
#define CND_EINVAL (-1)    /* bad argument or malformed graph */
#define CND_ENOMEM (-2)    /* device or host allocation failed */
#define CND_ECUDA (-3)     /* CUDA runtime error (no device, launch failure, ...) */
#define CND_ELIMIT (-4)    /* some trial still had newly active nodes at step max_levels */
#define CND_ETIMEOUT (-5)  /* time limit (timeout_s) reached; outputs are not valid */
#define CND_EOVERFLOW (-6) /* LT in-weights of a node sum above 2^32 - 1 */

#define CND_DIR_AUTO 0 /* push or pull per step, by frontier size (see pull_permille) */
#define CND_DIR_PUSH 1
#define CND_DIR_PULL 2

/* Optional measurements of one *_ex call (cnd_sim_opts.stats).  The caller
 * sets `flags`; every other field is written by the call. */
#define CND_STATS_TIMING 1 /* CUDA-event time the expansion and finalize kernels */
#define CND_STATS_COUNT 2  /* count the work terms below in the kernels (adds atomics) */
typedef struct cnd_sim_stats {
    int32_t flags;             /* in: CND_STATS_* */
    int32_t passes;            /* passes over the trials */
    int32_t word_bits;         /* trials held per node per pass */
    int32_t levels;            /* expansion steps, summed over passes */
    int64_t launches;          /* kernels launched by the call */
    int64_t expand_launches;   /* IC push / LT accumulate kernels */
    double expand_ms;          /* their summed CUDA-event time (CND_STATS_TIMING) */
    int64_t finalize_launches; /* frontier finalize / LT threshold kernels */
    double finalize_ms;
    int64_t frontier_slots;    /* (node, step) frontier entries */
    int64_t work_items;        /* (node, step, edge chunk) work items */
    /* CND_STATS_COUNT only: */
    int64_t edges_scanned;     /* frontier out-edges read by the expansion kernels */
    int64_t frontier_words;    /* frontier words loaded by the expansion kernels */
    int64_t word_checks;       /* (edge, word) pairs with frontier bits: target word read */
    int64_t draws;             /* Philox blocks drawn (IC coins; LT thresholds) */
    int64_t updates;           /* IC: (edge, target word) pairs with live coins for inactive trials
                                  (each or-ed into the target's words); LT: accumulator adds, or
                                  counter-plane updates in the counting form */
    int64_t pull_steps;        /* expansion steps run in the pull direction */
    int32_t lt_counters;       /* 1: LT ran in the counting form (see lt_accumulate) */
    int32_t pad0;
    double setup_ms;           /* CUDA-event time of the per-pass set-up: state zero fills and, in
                                  the counting form, the counter start values (CND_STATS_TIMING) */
    int32_t graph_reused;      /* graph mode: 1 if the call updated an executable graph cached by an
                                  earlier call of the same shape on this host thread, 0 if it
                                  instantiated one */
    int32_t pad1;
} cnd_sim_stats;

/* Options of the *_ex entry points.  Zero-initialise (cnd_sim_opts_init). */
typedef struct cnd_sim_opts {
    int64_t first_trial;       /* id of the first trial; a multiple of 64 (default 0) */
    int32_t max_levels;        /* <= 0: no cap; else steps 1..max_levels are expanded and
                                  a node activated at step max_levels yields CND_ELIMIT
                                  (outputs are still written) */
    int32_t direction;         /* CND_DIR_* */
    int32_t word_bits;         /* trials held per node per pass: 0 = automatic, else a multiple
                                  of 64 up to 131072 (pulling passes hold at most 16384) */
    int32_t device_ptrs;       /* 1: seeds and all outputs are device pointers; the work runs
                                  on `stream`, and the call returns once it is complete */
    void *stream;              /* cudaStream_t to run on; NULL = legacy default stream */
    int64_t *edge_checks_out;  /* NULL or 1 value: edge checks summed over the trials */
    int64_t *level_counts_out; /* NULL or level_counts_len values: [L] = number of
                                  (trial, node) pairs activated at step L */
    int32_t level_counts_len;
    int32_t pull_permille;     /* IC, AUTO: pull when the frontier's out-edges exceed this many
                                  thousandths of m; 0 = push only (the measured default).  LT
                                  always pushes */
    int32_t chunk_edges;       /* edges per push work item (0 = automatic) */
    int32_t defer_bits;        /* > 0: a node's word with fewer newly active trials than this may
                                  wait for more before its out-edges are examined; the spreads,
                                  counts and edge checks are unchanged (IC: reachability, LT: the
                                  least fixed point do not depend on the order of expansion), but
                                  steps no longer are activation times, so level counts and
                                  max_levels are refused (CND_EINVAL); 0 = off, at most 64 */
    double timeout_s;          /* > 0: give up with CND_ETIMEOUT after this many seconds (checked
                                  between steps: by the host, or in a CUDA-graph call by the
                                  step-control kernel on the GPU's global timer) */
    cnd_sim_stats *stats;      /* NULL or host struct filled by the call */
    int32_t defer_steps;       /* with defer_bits: a word waits at most this many steps (0 = until
                                  nothing else is left to expand) */
    int32_t graph;             /* 1: run the whole call as one CUDA graph launch -- every pass
                                  and its step loop (a device-side WHILE node whose condition a
                                  one-thread control kernel sets after each step), no host round
                                  trip per step; ignored with CND_STATS_TIMING.  Each host thread
                                  keeps the executable graphs of its recent call shapes (up to 16)
                                  and updates a matching one in place rather than instantiating */
    int32_t autotune;          /* 1: take word_bits, chunk_edges, pull_permille and graph from the
                                  autotuner's cache for this graph, model and problem size class,
                                  tuning (cnd_autotune on a sample of this call) on a miss */
    int32_t lt_accumulate;     /* LT only.  0 (default): where every node's non-zero in-weights are
                                  equal (the weighted cascade), keep per (node, trial) a count of
                                  active in-neighbours, bit-sliced over ceil(log2(k_v + 1)) planes
                                  of 64 trials (k_v the node's in-edges of non-zero weight), since
                                  k * w_v > theta <=> k > floor(theta / w_v); elsewhere, and with 1,
                                  keep the 32-bit in-weight sum per (node, trial).  Both compute
                                  exactly the same results */
    int64_t reserved[1];
} cnd_sim_opts;

void cnd_sim_opts_init(cnd_sim_opts *opts);

/*
 * Build the device copy of a directed CSR graph (Sec. 3 "Data Structures":
 * out-neighbours of u are col[row_ptr[u] .. row_ptr[u+1]-1]).
 *   n > 0 nodes, m >= 0 edges; row_ptr has n+1 entries, row_ptr[0] = 0,
 *   non-decreasing, row_ptr[n] = m; 0 <= col[e] < n.
 *   ic_prob: m fp32 IC probabilities in [0, 1] (NaN rejected), or NULL if the
 *            graph is only used for LT.
 *   lt_weight_fx: m uint32 LT weights, in-weights of every node summing to at
 *            most 2^32 - 1 (else CND_EOVERFLOW), or NULL if only used for IC.
 *   Self-loops and parallel edges are accepted.  All arrays are host memory
 *   and are copied.  The graph lives on the device that is current.
 *   *out receives the handle (NULL on failure).
 */
cnd_status cnd_graph_create(int32_t n, int32_t m, const int32_t *row_ptr, const int32_t *col,
                            const float *ic_prob, const uint32_t *lt_weight_fx, cnd_graph **out);

/* Release a graph (NULL-safe).  No call on it may be in flight. */
void cnd_graph_destroy(cnd_graph *g);

/* n, m and which models the graph carries (any output may be NULL). */
cnd_status cnd_graph_info(const cnd_graph *g, int32_t *n, int32_t *m, int32_t *has_ic, int32_t *has_lt);

/*
 * Monte Carlo IC simulation (Sec. 2 "Diffusion Models", first model): trials
 * 0 .. n_trials-1 from seed set `seeds` (n_seeds ids in [0, n); duplicates
 * count once; n_seeds = 0 gives spread 0).
 *   spread_out:     NULL or n_trials int32, spread of each trial.
 *   node_count_out: NULL or n int32, number of trials in which each node is active.
 * 0 <= n_trials <= 2^31 - 1.  CND_EINVAL if the graph carries no IC probabilities.
 */
cnd_status cnd_ic_simulate(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                           uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out);

/* Monte Carlo LT simulation (Sec. 2, second model); arguments as cnd_ic_simulate.
 * CND_EINVAL if the graph carries no LT weights. */
cnd_status cnd_lt_simulate(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                           uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out);

/* As above with options (opts may be NULL = defaults).  Trial ids run from
 * opts->first_trial; spread_out[i] is trial first_trial + i. */
cnd_status cnd_ic_simulate_ex(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                              uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out,
                              const cnd_sim_opts *opts);
cnd_status cnd_lt_simulate_ex(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                              uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out,
                              const cnd_sim_opts *opts);

/*
 * Batched simulation: n_items independent problems in one call, each with its
 * own seed set, trial count and key -- the workload of evaluating many
 * candidate seed sets, e.g. the marginal gains of greedy / CELF influence
 * maximisation (Sec. 2 "Influence Maximization").  Item i has seeds
 * seeds[seed_off[i] .. seed_off[i+1]), trials 0 .. n_trials[i]-1 (plus
 * opts->first_trial) and rng_seed[i]; its results are exactly those of
 * cnd_ic_simulate / cnd_lt_simulate on that item alone.  The trials of all
 * items are packed into shared passes (64-trial words of different items side
 * by side), so small items keep the whole GPU busy.
 *   seed_off (n_items+1 int64), n_trials (n_items int32, each 0 .. 2^31-1) and
 *   rng_seed (n_items uint64) are host arrays whatever opts->device_ptrs says:
 *   they drive the packing.  seeds and the outputs follow device_ptrs.
 *   spread_out:     NULL or sum(n_trials) int32; trial t of item i is at
 *                   n_trials[0] + ... + n_trials[i-1] + t.
 *   node_count_out: NULL or n_items * n int32; row i counts item i's trials.
 * Edge checks and level counts (opts) are summed over all items.
 */
cnd_status cnd_ic_simulate_batch(const cnd_graph *g, int32_t n_items, const int64_t *seed_off, const int32_t *seeds,
                                 const int32_t *n_trials, const uint64_t *rng_seed, int32_t *spread_out,
                                 int32_t *node_count_out, const cnd_sim_opts *opts);
cnd_status cnd_lt_simulate_batch(const cnd_graph *g, int32_t n_items, const int64_t *seed_off, const int32_t *seeds,
                                 const int32_t *n_trials, const uint64_t *rng_seed, int32_t *spread_out,
                                 int32_t *node_count_out, const cnd_sim_opts *opts);

/*
 * Autotuner: times candidate settings of the engine on a sample of the given
 * work (at most 4,096 trials of a single seed set, or the first 4 items of a
 * batch with at most 512 trials each) and writes the fastest into *best_out
 * (a copy of *base with word_bits, chunk_edges, pull_permille and graph set).
 * The candidates: the widest pass that fits (up to 2,048 words), 64 and 16
 * words (single seed sets; the widest for batches); 0 (by frontier words),
 * 32 and 512 edges per work item; push only or pull above 25 % of m (IC);
 * host loop or one CUDA graph per call.  The result is cached per (graph,
 * model, single or batch, log2 trials, log2 seeds) for opts.autotune.
 * model: 0 IC, 1 LT.  Single seed set: n_items = 0, seed_off NULL, n_trials[0]
 * and rng_seed[0] describe it.  Arrays as in the simulate calls; best_ms_out
 * (may be NULL) receives the sample time of the winner in milliseconds.
 * Every candidate computes the same results, so tuning never changes outputs.
 */
cnd_status cnd_autotune(const cnd_graph *g, int32_t model, int32_t n_items, const int64_t *seed_off,
                        const int32_t *seeds, int32_t n_seeds, const int32_t *n_trials, const uint64_t *rng_seed,
                        const cnd_sim_opts *base, cnd_sim_opts *best_out, double *best_ms_out);

/*
 * Influence maximisation by lazy greedy (CELF, Leskovec et al. 2007) on the
 * batched engine (Sec. 2 "Influence Maximization": choose |S| = k maximising
 * sigma(S); the paper applies CELF in Sec. 4 "Influence Maximization").
 *
 * sigma is estimated with common random numbers: every evaluation of a set X
 * runs trials first_trial .. first_trial + n_trials - 1 of key rng_seed, and
 * the value used is the exact integer F(X) = sum over those trials of the
 * spread.  For IC, F is a coverage function of the trials' live-edge graphs,
 * hence submodular, and the result equals plain greedy's.  The rule, which
 * fixes the result for both models:
 *   round 0: gain(v) = F({v}) for every candidate (a candidate with no
 *            out-edges has F({v}) = n_trials without simulation);
 *   round j: entries are ordered by (gain descending, node id ascending);
 *            while the first entry was last evaluated before round j, the
 *            stale entries that precede the first fresh one (at most
 *            eval_batch of them, in order) are re-evaluated in one batched
 *            call, gain(v) = F(S + v) - F(S); the first entry, once fresh, is
 *            chosen and F(S) grows by its gain.
 *   k:              seeds to choose, 1 <= k <= number of candidates.
 *   n_trials:       trials per evaluation, 1 .. 2^31 - 1.
 *   candidates:     host array of n_candidates distinct node ids, or NULL for
 *                   all nodes (n_candidates ignored).
 *   eval_batch:     0 = 64.  max_items: items per batched call, 0 = 8192;
 *                   also capped so that items x n_trials <= 2^28 (the
 *                   per-trial spreads of one call stay within 1 GiB).
 *   sim:            engine settings for the batched calls (NULL = defaults;
 *                   its first_trial, a multiple of 64 as for every batched
 *                   call, is used; device_ptrs, stream and output pointers
 *                   are ignored).
 *   stream:         cudaStream_t for the work (NULL = legacy default stream).
 * Outputs (host): seeds_out[j] = j-th chosen node; f_out (may be NULL)[j] =
 * F(first j+1 seeds) (sigma estimate = f_out[j] / n_trials); evaluations_out
 * and edge_checks_out (may be NULL) count the sets simulated and their edge
 * checks.  Returns when the results are written.
 */
typedef struct {
    int32_t k;
    int32_t eval_batch;
    int64_t n_trials;
    uint64_t rng_seed;
    const int32_t *candidates;
    int32_t n_candidates;
    int32_t max_items;
    const cnd_sim_opts *sim;
    void *stream;
    int64_t *evaluations_out;
    int64_t *edge_checks_out;
    int64_t reserved[4];
} cnd_im_opts;

void cnd_im_opts_init(cnd_im_opts *o);
cnd_status cnd_ic_im_celf(const cnd_graph *g, const cnd_im_opts *o, int32_t *seeds_out, int64_t *f_out);
cnd_status cnd_lt_im_celf(const cnd_graph *g, const cnd_im_opts *o, int32_t *seeds_out, int64_t *f_out);

/*
 * Learned surrogate of IC activation frequencies, for screening candidate
 * seeds in greedy influence maximisation (Sec. 2 "Influence Maximization";
 * the paper has no learned component -- the exact simulator above makes
 * every decision).  A 3-layer message-passing network, hidden width 64, maps a seed
 * set S to yhat_v, a prediction of the fraction of trials in which node v
 * ends active (the per-node counts of the paper's activation heatmap, Sec. 4,
 * over the trial count):
 *
 *   q_e    = fp32(thr_e) * 2^-32, the live probability of edge e (thr_e the
 *            IC threshold defined above; "always" gives 1)
 *   x_v    = bf16([s_v, ln(1 + indeg v), ln(1 + outdeg v), 0 x 13])  (16 wide)
 *   a^l_v  = bf16(sum over in-edges e = (u -> v) of q_e h^{l-1}_u)
 *   h^l_v  = bf16(relu(W_s^l h^{l-1}_v + W_n^l a^l_v + b^l)),  h^0 = x, l = 1..3
 *   yhat_v = s_v + (1 - s_v) sigmoid(w_o . h^3_v + b_o)
 *   loss   = mean over v of (yhat_v - y_v)^2
 *
 * W_s, W_n are used as bf16 (tensor-core operands, fp32 accumulation); biases,
 * w_o and b_o as fp32; the fp32 masters are what get_params returns.  The
 * backward rounds dz = d loss / d z to bf16 before its products, like the
 * forward's operands.  Parameters are one fp32 vector of CND_SUR_N_PARAMS
 * values: [W_s^1 (64x16), W_n^1 (64x16), b^1 (64), W_s^2 (64x64), W_n^2,
 * b^2, W_s^3, W_n^3, b^3, w_o (64), b_o (1)], matrices row-major (out x in).
 *
 * Host arrays throughout; a surrogate lives on its graph's device and owns
 * its working memory (about 0.5 KB per node).  The graph needs IC
 * probabilities.  Seed ids must lie in [0, n); duplicates count once.
 *
 * Bit-reproducible: every sum runs in a fixed order (in-edge sums of high
 * in-degree nodes split over several warps, gradients split over blocks and
 * the predicted spread are added up from partial sums in index order; the
 * seed channel of a^1 is an exact fixed-point sum), so the same calls on the
 * same device give the same bits.  Simulation results above are exact.
 */
#define CND_SUR_N_PARAMS 18689
typedef struct cnd_sur cnd_sur;

/* params: host, CND_SUR_N_PARAMS fp32 values (required).  Adam state starts at zero. */
cnd_status cnd_sur_create(const cnd_graph *g, const float *params, cnd_sur **out);
void cnd_sur_destroy(cnd_sur *s); /* NULL-safe */
cnd_status cnd_sur_set_params(cnd_sur *s, const float *params); /* also resets the Adam state */
cnd_status cnd_sur_get_params(const cnd_sur *s, float *params_out);

/* yhat_out: NULL or n floats; spread_out: NULL or sum of yhat (the predicted sigma(S)). */
cnd_status cnd_sur_forward(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, float *yhat_out, double *spread_out);

/* Loss for targets y (n floats) and its gradient (CND_SUR_N_PARAMS floats); either output may be NULL. */
cnd_status cnd_sur_loss_grad(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, const float *y, double *loss_out,
                             float *grad_out);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; Kingma and Ba 2015) on the
 * fp32 masters with the given gradient (host, CND_SUR_N_PARAMS floats). */
cnd_status cnd_sur_adam(cnd_sur *s, const float *grad, float lr);

/* Screening scores: score_out[c] (n floats) = the first-order gain of the predicted spread
 * P = sum_v yhat_v when c joins S, (1 - s_c)(1 - sigmoid(o_c)) + d P / d x_c[0] through the
 * network.  Seeds themselves get (1 - s_c) = 0 for the direct term. */
cnd_status cnd_sur_scores(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, float *score_out);

/* One-hop expected gain under the prediction yhat = yhat(S): score_out[c] (n floats) =
 * (1 - yhat_c) (1 + sum over out-edges (c -> w) of q_e (1 - yhat_w)). */
cnd_status cnd_sur_onehop(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, float *score_out);

/*
 * Training on pairs the simulator generates on the fly: pair i is a seed set
 * of size U{set_size_lo..set_size_hi} of distinct nodes (uniform, or with
 * hub_frac partly in proportion to out-degree; drawn from a splitmix64 stream of
 * data_seed and i), with targets y_v = (trials in which
 * v ends active) / n_trials from n_trials exact IC trials under key
 * rng_seed + i (cnd_ic_simulate_batch).  Adam steps on the mean loss of
 * batch_sets pairs; pairs first_pair .. first_pair + n_pairs - 1.
 * loss_out: NULL or ceil(n_pairs / batch_sets) doubles, the mean loss of each
 * step's batch (before the step).
 */
typedef struct {
    int64_t first_pair;
    int64_t n_pairs;
    int32_t set_size_lo, set_size_hi;
    int32_t n_trials;
    int32_t batch_sets;   /* 0 = 16 */
    int32_t sim_chunk;    /* pairs simulated per batched call, 0 = 256 */
    float lr;             /* 0 = 1e-3 */
    uint64_t data_seed;
    uint64_t rng_seed;
    void *stream;
    double *sim_ms_out;   /* NULL or time spent in the simulator, ms */
    double *train_ms_out; /* NULL or time spent in forward / backward / Adam, ms */
    float hub_frac;       /* 0 (default): seeds uniform over the nodes; in (0, 1]: each seed is, with
                             this probability, the source of a uniform random edge instead (drawn in
                             proportion to out-degree), so that training sets contain hubs the way
                             the sets a greedy seed selection scores do (its earlier picks) */
    int32_t pad;
    int64_t reserved[3];
} cnd_sur_train_opts;

void cnd_sur_train_opts_init(cnd_sur_train_opts *o);
cnd_status cnd_sur_train(cnd_sur *s, const cnd_sur_train_opts *o, double *loss_out);

/*
 * Greedy influence maximisation with the surrogate as a screen (IC).  Each of
 * the k rounds, with S the seeds chosen so far:
 *   1. score every candidate c not in S and keep the n_screen best (ties:
 *      lower id).  mode 0: cnd_sur_scores (one forward and one backward
 *      pass); mode 1: the expected one-hop gain under the network's
 *      prediction yhat = yhat(S) (one forward pass),
 *        (1 - yhat_c) (1 + sum over out-edges (c -> w) of q_e (1 - yhat_w));
 *      mode 2: out-degree (no network: the screen without the surrogate);
 *      mode 3: the n_exact candidates are taken alternately from the best
 *      by the mode-0 score and the best by out-degree (repeats skipped;
 *      n_screen unused): the network proposes half of what is simulated;
 *   2. if n_screen > n_exact, re-rank those by the surrogate's predicted
 *      spread of S + c (one forward each) and keep the n_exact best (mode 2
 *      keeps the n_exact best by out-degree directly; s may then be NULL);
 *   3. evaluate F(S + c) exactly for the survivors with the batched Monte
 *      Carlo engine (common random numbers as in CELF: trials first_trial ..
 *      first_trial + n_trials - 1 of key rng_seed) and choose the best
 *      (ties: lower id).
 * The simulator makes every choice; the network only decides which
 * candidates it sees.  o->k, n_trials, rng_seed, candidates, max_items, sim,
 * stream, evaluations_out and edge_checks_out as for CELF (eval_batch
 * unused).  seeds_out[j], f_out[j] (may be NULL) as for CELF.
 */
typedef struct {
    int32_t n_screen;     /* candidates kept by the first score, >= n_exact (0 = n_exact) */
    int32_t n_exact;      /* candidates simulated per round, >= 1 */
    int32_t mode;         /* first score: 0 gradient, 1 one-hop gain, 2 out-degree, 3 gradient and
                             out-degree alternately */
    int32_t pad;
    double *sur_ms_out;   /* NULL or wall time in the surrogate, ms */
    double *sim_ms_out;   /* NULL or wall time in the simulator, ms */
    int64_t reserved[3];
} cnd_screen_opts;

cnd_status cnd_ic_im_screened(const cnd_graph *g, cnd_sur *s, const cnd_im_opts *o, const cnd_screen_opts *so,
                              int32_t *seeds_out, int64_t *f_out);

/*
 * Weighted-cascade LT weights for a CSR graph (Sec. 4 "Benchmarks", WC model:
 * the weight of every edge entering v is 1/in-degree(v)) in fixed point:
 * w_out[e] = floor((2^32 - 1) / in-degree(col[e])), so in-weights sum to at
 * most 2^32 - 1.  Host arrays: col has m entries in [0, n), w_out m entries.
 */
cnd_status cnd_lt_weights_wc(int32_t n, int32_t m, const int32_t *col, uint32_t *w_out);

/*
 * The engine's device Philox4x32-10 (the generator defined above), for
 * checking: out[4i..4i+3] = Philox(ctr[4i..4i+3]) under key rng_seed, for
 * i < count.  Host arrays of 4*count uint32 each.
 */
cnd_status cnd_philox4x32_10(uint64_t rng_seed, const uint32_t *ctr, int64_t count, uint32_t *out);

/*
 * Throughput of the engine's Philox4x32-10 (the generator above) on the current device, for the
 * roofline of the coin-drawing kernels (measurement only; the paper has no counterpart): one
 * launch of as many 256-thread blocks as are resident on all SMs, each thread computing 2 x iters
 * blocks in registers with the same code and precomputed round keys the expansion kernels use,
 * timed with CUDA events on `stream` (NULL = legacy default stream) after one short warm-up
 * launch.  *blocks_per_s_out = Philox blocks per second; ms_out (may be NULL) = the launch time.
 * iters >= 1 (about 4096 keeps the launch near 100 ms on a GB300).  Allocates 1 KB per block.
 */
cnd_status cnd_philox_rate(int32_t iters, void *stream, double *blocks_per_s_out, double *ms_out);

/*
 * Rate of random 8-byte memory operations on the current device, the ceiling of the
 * expansion kernels' scattered target-word accesses (measurement only; the paper has no
 * counterpart).  Allocates a region of the largest power of two of 8-byte words that fits
 * in region_bytes (zeroed; freed before return).  One launch of as many 256-thread blocks
 * as are resident on all SMs; each thread makes iters accesses at uniformly random words
 * of the region, each address derived from the value the previous access returned.
 * op 0: 8-byte reads through L2 (ld.global.cg); op 1: 8-byte atomic XOR with return.
 * A region well inside L2 (e.g. 32 MiB) gives the L2 rate, one far above it (e.g.
 * 4 GiB) the DRAM rate.  Timed with CUDA events on `stream` (NULL = legacy default
 * stream) after one short warm-up launch.  *ops_per_s_out = accesses per second;
 * ms_out (may be NULL) = the launch time.  region_bytes >= 64, iters >= 1 (about 256
 * keeps the launch in milliseconds); CND_ENOMEM if the region cannot be allocated.
 */
cnd_status cnd_random_access_rate(int64_t region_bytes, int32_t op, int32_t iters, void *stream,
                                  double *ops_per_s_out, double *ms_out);

/*
 * Allocation-free IC simulation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory while a
 * simulation runs -- for example code that runs on a device whose memory is
 * entirely reserved by another allocator (a framework's caching pool), or a
 * latency-critical loop that must not wait on the CUDA allocator.  It
 * computes exactly what cnd_ic_simulate computes, and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Its working state lives in one file-scope device array of
 * CND_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads this library
 * reserves until the process exits.  Graphs whose state does not fit even
 * with 64 trials per pass are rejected with CND_EINVAL and a message giving
 * the bytes needed.  The caller passes inputs and outputs:
 *   seeds:          device pointer, n_seeds ids (duplicates count once)
 *   spread_out:     device pointer, n_trials int32 (required if n_trials > 0)
 *   node_count_out: device pointer, n int32 (required)
 *   stream:         cudaStream_t the work runs on (NULL = legacy default stream)
 * The graph must live on the current device.  The call returns when the
 * results are complete.  The first call on a device looks up the array's
 * device address (once per device); make that first call before any stream
 * capture.  Every call shares the array, which keeps the last call's
 * contents (the call clears what must start at zero): calls that overlap on
 * the GPU -- from several host threads or on several streams -- race and
 * must be serialised by the caller.
 */
#define CND_NOALLOC_SCRATCH_BYTES (64u << 20)
cnd_status cnd_ic_simulate_noalloc(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                                   uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out, void *stream);

/* Message describing the last failure on this host thread ("" if none). */
const char *cnd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CND_H */
