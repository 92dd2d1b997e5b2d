// Bit-parallel, level-synchronous Monte Carlo engine for the IC and LT models
// on sm_103a.
//
// Layout.  Trials are packed 64 to a uint64 word; a pass holds B <= 2048
// consecutive words (64*B trials) and every node owns B contiguous words of
// each state array (node-major), so the state of one node in all of the pass's
// trials is one contiguous run of 8*B bytes:
//   vis[v*B + w]   bit b set <=> node v is active in trial 64*(w0+w) + b
//   nxt[v*B + w]   IC: bits first activated in the current step
//                  LT: trials whose accumulator grew in the current step
//   dmask[v*nq+q]  bit w%64 of word q set <=> nxt[v*B + w] != 0 (nq = ceil(B/64))
//   acc[(v*B + w)*64 + b]   LT: active in-weight of v in that trial (uint32)
//   planes[cnt_off[v]*B + w*L_v + i]   LT, counting form (every node's non-zero
//                  in-weights equal, as in the weighted cascade): bit i of a
//                  64-lane bit-sliced counter per (node, word), L_v planes
//
// Frontier.  In a step, a node is newly active in only some of the pass's
// trials, and those trials are scattered over its words; the frontier keeps
// only the words that carry bits: a list of slots (node, pair offset, pair
// count) over a pool of (word index, frontier bits) pairs.  Work items
// (slot, edge offset) cover about kTasks (edge, pair) tasks each, and a warp
// spreads the tasks of an item evenly over its lanes, so hubs are split over
// many warps and no lane idles on empty words.
//
// Steps (Sec. 3 "Algorithms": only out-neighbours of nodes newly active in
// the previous step are examined, Observation 1):
//   seeds      every valid word of every distinct seed
//   IC push    task (edge u->v, pair (w, f)): c = f & ~vis_v[w]; coins are
//              drawn only for the 4-trial blocks with a bit in c; live bits are
//              or-ed into vis_v and nxt_v; v is listed once per step
//   LT push    task: for each trial of f & ~vis_v[w], add w(u,v) to acc and
//              mark the word touched; v is listed once per step
//              (counting form: one bit-sliced increment of v's counter word by
//              the trials of f & ~vis_v[w]; a carry out of the top plane is
//              the activation, see k_lt_init)
//   collect    per listed node: IC and the LT counting form take the dirty
//              words of nxt (k_collect; k_finalize where words wait); the LT
//              accumulate form draws the thresholds of the touched trials and
//              activates where acc > theta (k_finalize<2>); the non-empty
//              words become the next frontier
// then the per-trial spread and per-node counts are reduced from vis.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "cnd_common.cuh"

namespace cnd {

constexpr int kMaxB = 2048;  // words per node per pass (dirty mask: one 64-bit word per lane)
// Occupancy of the step kernels (all latency-bound on scattered word traffic): the push runs
// 8 blocks of 256 threads per SM (32 registers), k_collect 6, the block-cooperative finalize
// 6 (IC) or 4 (LT accumulate form, which converts accumulator rows and needs more registers).
// Measured on GB300: against one block minimum, BA n=100k IC -21 %, LT -15 %, a sparse
// 256-set batch -17 %.
constexpr int kPushMinBlocks = 8;
constexpr int kStageB = 64;  // pairs of a push work item staged in shared memory (more: read from the pool)
constexpr int kPullMaxB = 256;  // words per node the pull kernel keeps in registers
constexpr int kTasks = 256;  // (edge, pair) tasks per push work item
// AUTO without pull_permille: push only -- the pull step measured 1.3x to 3.7x
// slower than push on every GB300 workload here (hub in-rows scanned by one warp)
constexpr int kPullPermille = 1001;
constexpr int kWarps = 8;    // warps per block
constexpr int kBlock = 32 * kWarps;

struct Frontier {
    int32_t *node = nullptr;   // [n] node of each slot
    int32_t *poff = nullptr;   // [n] first pair of each slot in the pool
    int32_t *pk = nullptr;     // [n] number of pairs of each slot
    uint16_t *pw = nullptr;    // [n*B] pool: word index
    uint64_t *pb = nullptr;    // [n*B] pool: frontier bits
    int2 *work = nullptr;      // [work_cap] (slot, first edge of the item within the row)
    int32_t *cnt = nullptr;    // device [4]: pool pairs, slots (one 64-bit word), work items, out-edges of the slots
};

// Step state of a run whose step loop executes on the device (CUDA-graph mode).
struct Ctl {
    int32_t level;   // step being run: frontier fr[level & 1] -> fr[(level + 1) & 1]; -1: the seed step
    uint32_t stamp;  // stamp of that step
    int32_t force;   // 1: every waiting word is expanded now
    int32_t pull;    // 1: this step pulls (IC)
    int32_t limit;   // a pass stopped at max_levels with trials still active
    int32_t timed_out;  // the device loop stopped at its time limit
    unsigned long long slots, items, levels, pull_steps;
    unsigned long long t0;  // global timer (ns) when the call's first step began
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Params {
    int32_t n, B, nq;
    int32_t chunk;             // > 0: fixed edges per work item
    const int32_t *row_ptr;
    const uint2 *edge;         // {col, IC threshold} or {col, LT weight}
    uint64_t *vis, *nxt, *dmask;
    uint64_t *cvt;             // LT: [v*nq+q] bit w%64 set <=> acc row (v, w) holds ~theta + sum
    uint32_t *acc;
    // LT counting form (nodes with equal in-weights): bit-sliced counters, plane i of node v
    // and word w at planes[cnt_off[v] * B + w * L_v + i], L_v = cnt_off[v+1] - cnt_off[v]
    uint64_t *planes;
    const int32_t *cnt_off;
    const uint32_t *unit_w;
    uint32_t *mark;            // [n] last stamp that listed the node
    int32_t *lin, *lin_cnt;    // [n] nodes the current step finalizes (its push lists them here)
    int32_t *lnext, *lnext_cnt;// [n] nodes whose words wait for the next step (deferral)
    Frontier in, out;
    uint32_t stamp;            // stamp of the current step; stamp + 1 is the next step's
    int32_t tau;               // > 0: words with fewer new bits than tau may wait (not when force)
    int32_t max_wait;          // > 0: ... for at most max_wait steps
    uint8_t *age;              // [n*B] steps the word has waited (deferral)
    int32_t force;             // 1: expand every pending word
    RoundKeys rk;              // Philox round keys of rng_seed (all words share one key)
    const uint2 *wkey;         // [B] per-word Philox key (batches: words of different items)
    // pull direction (IC): the frontier of the step, node-indexed
    const int32_t *in_row_ptr;
    const uint4 *in_edge;      // {src, edge id, IC threshold, LT weight}
    uint64_t *fdense;          // [n*B] frontier words by node (zero outside the frontier)
    uint32_t *fbits;           // [ceil(n/32)] frontier nodes
    const uint64_t *wg0;       // [B] per-word trial-block index of bit 0
    uint64_t g_base;           // trial-block index (trial >> 2) of bit 0 of word 0
    unsigned long long *level_counts;
    int32_t lc_len;
    int32_t level;             // step whose frontier is being produced
    const uint64_t *valid;     // [B] valid-trial mask of each word
    int32_t nvalid;            // words of this pass that hold trials
    unsigned long long *ctr;   // null, or [C_N] work counters (CND_STATS_COUNT)
    // graph mode: the step's frontiers, lists and stamp come from ctl (resolve())
    Ctl *ctl;
    Frontier fr[2];
    int32_t *lists[2];
    int32_t *lcnt;             // [2] list counters
};

// In graph mode, point the step fields of p at this step's buffers.
__device__ __forceinline__ void resolve(Params &p) {
    if (!p.ctl) return;
    const int L = p.ctl->level;
    const bool odd = (L & 1) != 0;
    p.in = odd ? p.fr[1] : p.fr[0];
    p.out = odd ? p.fr[0] : p.fr[1];
    p.lin = odd ? p.lists[1] : p.lists[0];
    p.lin_cnt = p.lcnt + (odd ? 1 : 0);
    p.lnext = odd ? p.lists[0] : p.lists[1];
    p.lnext_cnt = p.lcnt + (odd ? 0 : 1);
    p.stamp = p.ctl->stamp;
    p.force = p.ctl->force;
    p.level = L + 1;
}

enum { C_EDGES, C_FWORDS, C_WCHECKS, C_DRAWS, C_UPDATES, C_N };

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ void count_add(const Params &p, int i, unsigned long long v) {
    if (!p.ctr) return;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane_id() == 0 && v) atomicAdd(&p.ctr[i], v);
}

__device__ __forceinline__ void add_level_count(const Params &p, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane_id() == 0 && v && p.level < p.lc_len) atomicAdd(&p.level_counts[p.level], v);
}

// Edges per work item for a slot with k pairs.
__device__ __forceinline__ int edges_per_item(const Params &p, int k) {
    return p.chunk > 0 ? p.chunk : max(1, kTasks / max(k, 1));
}

// t / k for t < 2^32 / k (k <= kMaxB): multiply by ceil-ish reciprocal.
__device__ __forceinline__ uint32_t div_by(uint32_t t, uint32_t k, uint32_t magic) {
    return k == 1 ? t : __umulhi(t, magic);
}

// Position of the r-th (0-based) set bit of x; x has more than r set bits.
__device__ __forceinline__ int nth_set_bit(uint64_t x, int r) {
    const uint32_t lo = (uint32_t)x;
    const int c = __popc(lo);
    if (r < c) return (int)__fns(lo, 0, r + 1);
    return 32 + (int)__fns((uint32_t)(x >> 32), 0, r - c + 1);
}

// Philox block (index, trial block g, domain) of word w: one key for the whole
// pass, or (batches) the key of the item that owns the word.
template <bool PERWORD>
__device__ __forceinline__ U4 draw(const Params &p, int w, uint32_t index, uint64_t g, uint32_t domain) {
    if (PERWORD) {
        const uint2 k = p.wkey[w];
        return philox4x32_10(index, (uint32_t)g, domain, (uint32_t)(g >> 32), k.x, k.y);
    }
    return philox4x32_10(index, (uint32_t)g, domain, (uint32_t)(g >> 32), p.rk);
}

template <bool PERWORD>
__device__ __forceinline__ uint64_t word_g0(const Params &p, int w) {
    return PERWORD ? p.wg0[w] : p.g_base + 16ull * (uint64_t)w;
}

// Per-warp staging of the nodes a push lists for the collect / finalize kernel: one
// global atomic per 32 or more nodes instead of one per warp iteration.
struct ListBuf {
    int32_t *buf;  // 64 entries in shared memory
    int n;         // warp-uniform fill level

    __device__ __forceinline__ void flush(const Params &p) {
        __syncwarp();
        int base = 0;
        if (lane_id() == 0) base = atomicAdd(p.lin_cnt, n);
        base = __shfl_sync(kFull, base, 0);
        for (int j = lane_id(); j < n; j += 32) p.lin[base + j] = buf[j];
        __syncwarp();
        n = 0;
    }

    // List v once per step (the stamp in mark[v] says whether it already is).
    __device__ __forceinline__ void add(const Params &p, bool want, int v) {
        put(p, want && __ldcg(&p.mark[v]) != p.stamp && atomicExch(&p.mark[v], p.stamp) != p.stamp, v);
    }

    // Append v for the lanes with need set (the caller has claimed mark[v] for this step).
    __device__ __forceinline__ void put(const Params &p, bool need, int v) {
        const unsigned nm = __ballot_sync(kFull, need);
        if (nm) {
            if (need) buf[n + __popc(nm & ((1u << lane_id()) - 1u))] = v;
            n += __popc(nm);
            if (n >= 32) flush(p);
        }
    }
};

// Mark word w of v dirty the first time nxt[v][w] gains bits in this step.
__device__ __forceinline__ void mark_dirty(const Params &p, int v, int w, uint64_t old_nxt) {
    if (old_nxt == 0) atomicOr((unsigned long long *)(p.dmask + (size_t)v * p.nq + (w >> 6)), 1ull << (w & 63));
}

// ---------------------------------------------------------------- seeds
// A run of word columns of one item and the range of that item's seeds.
struct SeedSeg {
    int32_t s_begin, s_end;  // seeds[s_begin .. s_end)
    int32_t col0, cnt;       // word columns [col0, col0 + cnt) of the pass
};

// Step 0: every seed is active in every valid trial of its item's words.  The
// words go to nxt (dirty) and the seed to the list, so the seed step is then
// finalized like an IC step.  Duplicate seeds write the same words.
__global__ void k_seed(Params p_, const SeedSeg *__restrict__ segs, int32_t n_segs, const int32_t *__restrict__ seeds,
                       int32_t *__restrict__ bad) {
    Params p = p_;
    resolve(p);
    for (int j = blockIdx.x; j < n_segs; j += gridDim.x) {
        const SeedSeg sg = segs[j];
        for (int i = sg.s_begin + (int)threadIdx.x; i < sg.s_end; i += blockDim.x) {
            const int s = seeds[i];
            if (s < 0 || s >= p.n) {
                atomicExch(bad, 1);
                continue;
            }
            for (int w = sg.col0; w < sg.col0 + sg.cnt; ++w) {
                const size_t idx = (size_t)s * p.B + w;
                const uint64_t x = p.valid[w];
                p.vis[idx] = x;
                p.nxt[idx] = x;
                atomicOr((unsigned long long *)(p.dmask + (size_t)s * p.nq + (w >> 6)), 1ull << (w & 63));
            }
            if (atomicExch(&p.mark[s], p.stamp) != p.stamp) p.lin[atomicAdd(p.lin_cnt, 1)] = s;
        }
    }
}

// ---------------------------------------------------------------- finalize
// Word index of the r-th word listed in a node's dirty mask.  Lane q holds mask word q
// (nq <= 32) in `mine` and the inclusive count of listed words up to it in `incl`; each
// lane asks for its own r (0 <= r < listed words), so every lane must call this.
__device__ __forceinline__ int word_at(uint64_t mine, int incl, int r) {
    int q = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int x = __shfl_sync(kFull, incl, q + step - 1);
        if (x <= r) q += step;
    }
    const uint64_t wq = __shfl_sync(kFull, mine, q);
    const int before = __shfl_sync(kFull, incl, q) - __popcll(wq);
    return 64 * q + nth_set_bit(wq, r - before);
}

// Placement of the slots of the nodes a block finalizes together: a block
// scan gives each node its slot, pool offset and first work item, with one
// 64-bit atomic for (slots, pool pairs) and one for work items per block
// iteration.  cnt = {pool pairs, slots, work items, listed nodes}; the pool
// count stays below 2^31 (n * B < 2^31), so it never carries into the slots.
constexpr int kNPW = 2;                 // nodes per warp per block iteration
constexpr int kNPB = kWarps * kNPW;     // nodes per block iteration

// Block-cooperative finalize: each warp takes kNPW listed nodes per block
// iteration, collects their words with frontier bits into slots, and emits
// their work items.
//   MODE 1 (IC, and the seed step of both models): the dirty words of nxt.
//   MODE 2 (LT):    rows touched for the first time in this pass are converted
//                   (64 thresholds drawn once; acc = sum + ~theta; activation
//                   where sum > theta); rows converted earlier carry the
//                   activations their push detected.
// With deferral (tau > 0, not force) a word with fewer than tau new bits stays
// in nxt, still dirty, and its node is listed for the next step: expanding it
// later, merged with later bits, leaves reachability (IC) and the least fixed
// point (LT) unchanged.
template <int MODE, bool PERWORD>
__global__ void __launch_bounds__(kBlock, MODE == 2 ? 4 : 6) k_finalize(Params p_) {
    Params p = p_;
    resolve(p);
    __shared__ int s_kept[kNPB], s_nch[kNPB], s_def[kNPB], s_deg[kNPB];
    __shared__ int s_off[kNPB], s_slot[kNPB], s_wb[kNPB], s_dpos[kNPB];
    const int lane = lane_id();
    const int wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int count = *p.lin_cnt;
    const int B = p.B, nq = p.nq;
    const int tau = p.force ? 0 : p.tau;
    unsigned long long pc = 0;
    uint32_t n_dr = 0;
    for (int base = blockIdx.x * kNPB; base < count; base += gridDim.x * kNPB) {
        int vv[kNPW], KK[kNPW], dinc[kNPW];
        uint64_t dmine[kNPW];
#pragma unroll
        for (int h = 0; h < kNPW; ++h) {
            const int i = base + wid * kNPW + h;
            const bool act = i < count;
            vv[h] = act ? p.lin[i] : 0;
            dmine[h] = (act && lane < nq) ? p.dmask[(size_t)vv[h] * nq + lane] : 0ull;
            if (act && lane < nq) p.dmask[(size_t)vv[h] * nq + lane] = 0ull;
            int c = __popcll(dmine[h]);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(kFull, c, o);
                if (lane >= o) c += x;
            }
            dinc[h] = c;
            KK[h] = __shfl_sync(kFull, c, 31);
        }
#pragma unroll
        for (int h = 0; h < kNPW; ++h) {
            const int v = vv[h], K = KK[h];
            int kept = K, deferred = 0;
            if (K > 0) {
                // the new bits of every listed word (LT: after the threshold test);
                // words that wait go back into the dirty mask
                kept = 0;
                for (int r0 = 0; r0 < K; r0 += 32) {
                    const int r = r0 + lane;
                    uint64_t nb = 0;
                    const int w = word_at(dmine[h], dinc[h], min(r, K - 1));
                    const size_t idx = (size_t)v * B + w;
                    if (MODE == 1) {
                        if (r < K) nb = p.nxt[idx];
                    } else {
                        // LT: a row converted earlier in this pass carries the activations its push
                        // detected; a row touched for the first time is converted here by a
                        // half-warp (one lane per 4-trial block, coalesced 256-byte row)
                        uint64_t *cw = p.cvt + (size_t)v * nq + (w >> 6);
                        const bool conv = r < K && ((*cw >> (w & 63)) & 1ull);
                        const uint64_t x = r < K ? p.nxt[idx] : 0ull;
                        if (conv) nb = x;
                        unsigned need = __ballot_sync(kFull, r < K && !conv);
                        const int hl = lane & 15;
                        while (need) {
                            const int l0 = __ffs(need) - 1;
                            need &= need - 1;
                            const int l1 = need ? __ffs(need) - 1 : -1;
                            if (need) need &= need - 1;
                            const int own = lane < 16 ? l0 : (l1 >= 0 ? l1 : l0);
                            const bool act = lane < 16 || l1 >= 0;
                            const int ow = __shfl_sync(kFull, w, own);
                            const size_t oidx = (size_t)v * B + ow;
                            uint64_t bits = 0;
                            if (act) {
                                ++n_dr;
                                const U4 th = draw<PERWORD>(p, ow, (uint32_t)v, word_g0<PERWORD>(p, ow) + (uint64_t)hl, 1u);
                                uint4 *a4 = reinterpret_cast<uint4 *>(p.acc + oidx * 64) + hl;
                                uint4 s4 = *a4;
                                bits = ((uint64_t)(s4.x > th.x) | ((uint64_t)(s4.y > th.y) << 1) |
                                        ((uint64_t)(s4.z > th.z) << 2) | ((uint64_t)(s4.w > th.w) << 3))
                                       << (4 * hl);
                                s4.x += ~th.x;
                                s4.y += ~th.y;
                                s4.z += ~th.z;
                                s4.w += ~th.w;
                                *a4 = s4;
                            }
                            // or the 16 lanes' 4-bit pieces within each half-warp
#pragma unroll
                            for (int o = 1; o < 16; o <<= 1) bits |= __shfl_xor_sync(kFull, bits, o);
                            const uint64_t b0 = __shfl_sync(kFull, bits, 0), b1 = __shfl_sync(kFull, bits, 16);
                            if (lane == l0 || lane == l1) {
                                const uint64_t vis = p.vis[idx];
                                nb = (lane == l0 ? b0 : b1) & ~vis;
                                if (nb) p.vis[idx] = vis | nb;
                                atomicOr((unsigned long long *)cw, 1ull << (w & 63));
                            }
                        }
                        if (r < K) p.nxt[idx] = nb;
                    }
                    bool wait = nb != 0ull && __popcll(nb) < tau;
                    if (nb != 0ull && tau > 0 && p.max_wait > 0) {
                        uint8_t *ag = p.age + (size_t)v * B + w;
                        const int a = *ag;
                        wait = wait && a < p.max_wait;
                        *ag = wait ? (uint8_t)(a + 1) : (uint8_t)0;
                    }
                    if (wait) atomicOr((unsigned long long *)(p.dmask + (size_t)v * nq + (w >> 6)), 1ull << (w & 63));
                    kept += __popc(__ballot_sync(kFull, nb != 0ull && !wait));
                    deferred |= __any_sync(kFull, wait) ? 1 : 0;
                }
            }
            const int deg = kept > 0 ? p.row_ptr[v + 1] - p.row_ptr[v] : 0;
            const int ne = edges_per_item(p, kept);
            if (lane == 0) {
                s_kept[wid * kNPW + h] = kept;
                s_nch[wid * kNPW + h] = deg > 0 ? (deg + ne - 1) / ne : 0;
                s_def[wid * kNPW + h] = deferred;
                s_deg[wid * kNPW + h] = deg;
            }
        }
        __syncthreads();
        if (wid == 0) {
            const int kk = lane < kNPB ? s_kept[lane] : 0;
            const int hs = kk > 0 ? 1 : 0;
            const int cc = lane < kNPB ? s_nch[lane] : 0;
            const int dd = lane < kNPB ? s_def[lane] : 0;
            int sk = kk, sh = hs, sc = cc, sd = dd;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int a1 = __shfl_up_sync(kFull, sk, o), a2 = __shfl_up_sync(kFull, sh, o),
                          a3 = __shfl_up_sync(kFull, sc, o), a4 = __shfl_up_sync(kFull, sd, o);
                if (lane >= o) {
                    sk += a1;
                    sh += a2;
                    sc += a3;
                    sd += a4;
                }
            }
            unsigned long long ps0 = 0;
            int item0 = 0, d0 = 0;
            // out-edges of the new frontier (direction choice of the next step)
            int dg = lane < kNPB ? s_deg[lane] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dg += __shfl_xor_sync(kFull, dg, o);
            if (lane == 0 && dg) atomicAdd(&p.out.cnt[3], dg);
            if (lane == 31) {
                if (sk) ps0 = atomicAdd((unsigned long long *)p.out.cnt, ((unsigned long long)sh << 32) | (unsigned)sk);
                if (sc) item0 = atomicAdd(&p.out.cnt[2], sc);
                if (sd) d0 = atomicAdd(p.lnext_cnt, sd);
            }
            ps0 = __shfl_sync(kFull, ps0, 31);
            item0 = __shfl_sync(kFull, item0, 31);
            d0 = __shfl_sync(kFull, d0, 31);
            if (lane < kNPB) {
                s_off[lane] = (int)(uint32_t)ps0 + sk - kk;
                s_slot[lane] = (int)(ps0 >> 32) + sh - hs;
                s_wb[lane] = item0 + sc - cc;
                s_dpos[lane] = d0 + sd - dd;
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < kNPW; ++h) {
            const int e = wid * kNPW + h;
            const int v = vv[h], K = KK[h];
            if (s_def[e] && lane == 0) {
                // the node's waiting words are expanded by a later step
                p.mark[v] = p.stamp + 1u;
                p.lnext[s_dpos[e]] = v;
            }
            const int kept = s_kept[e];
            if (kept == 0) continue;
            const int off = s_off[e], slot = s_slot[e];
            if (lane == 0) {
                p.out.node[slot] = v;
                p.out.poff[slot] = off;
                p.out.pk[slot] = kept;
            }
            int pos = 0;
            for (int r0 = 0; r0 < K; r0 += 32) {
                const int r = r0 + lane;
                uint64_t x = 0;
                const int w = word_at(dmine[h], dinc[h], min(r, K - 1));
                if (r < K) {
                    const size_t idx = (size_t)v * B + w;
                    x = p.nxt[idx];
                    // a word that waits got its dirty bit back in the pass above
                    if (tau > 0 && ((p.dmask[(size_t)v * nq + (w >> 6)] >> (w & 63)) & 1ull)) x = 0ull;
                    else p.nxt[idx] = 0ull;
                    pc += __popcll(x);
                }
                const unsigned bm = __ballot_sync(kFull, x != 0ull);
                if (x) {
                    const int q = pos + __popc(bm & below);
                    p.out.pw[off + q] = (uint16_t)w;
                    p.out.pb[off + q] = x;
                }
                pos += __popc(bm);
            }
            const int nch = s_nch[e], wb = s_wb[e];
            const int ne = edges_per_item(p, kept);
            for (int c = lane; c < nch; c += 32) p.out.work[wb + c] = make_int2(slot, c * ne);
        }
    }
    add_level_count(p, pc);
    count_add(p, C_DRAWS, n_dr);
}

// Frontier collect when no word waits (tau = 0) and a node's words fit kCollectNq
// dirty-mask words (B <= 256): every dirty word then holds new bits, so a node keeps
// all of them.  A warp takes 32 listed nodes, one per lane, places their slots, pool
// pairs and work items with one atomic each per 32 nodes, then its lanes go over the
// 32 nodes' (word, bits) pairs and work items together, each lane finding the node of
// its entry by a binary search of the warp's prefix sums.  No block barrier; the loads
// of 32 nodes are in flight at once, and each lane issues the nxt loads of two pairs
// before it stores either.  Same outputs as k_finalize<1> up to the order of the
// slots, pairs and work items in the pool.
constexpr int kCollectNq = 4;

__device__ __forceinline__ int owner_of(const int *pre, int q) {  // largest j < 32 with pre[j] <= q
    int j = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (pre[j + step] <= q) j += step;
    return j;
}

template <bool ONE_WORD>  // nq == 1
__global__ void __launch_bounds__(kBlock) k_collect(Params p_) {
    constexpr int kU = 2;  // pairs per lane whose loads go out together
    Params p = p_;
    resolve(p);
    __shared__ int s_pp[kWarps][33], s_ip[kWarps][33];
    __shared__ int s_v[kWarps][32], s_slot[kWarps][32], s_ne[kWarps][32];
    __shared__ uint64_t s_dm[kWarps][kCollectNq][32];
    const int lane = lane_id();
    const int wid = threadIdx.x >> 5;
    const int count = *p.lin_cnt;
    const int B = p.B, nq = ONE_WORD ? 1 : p.nq;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long pc = 0;
    if (lane == 0) {
        s_pp[wid][0] = 0;
        s_ip[wid][0] = 0;
    }
    for (int base = warp * 32; base < count; base += n_warps * 32) {
        const int i = base + lane;
        int v = 0, K = 0, deg = 0;
        if (i < count) v = p.lin[i];
        for (int q = 0; q < nq; ++q) {
            uint64_t dm = 0;
            if (i < count) {
                uint64_t *d = p.dmask + (size_t)v * nq + q;
                dm = *d;
                if (dm) *d = 0ull;
            }
            s_dm[wid][q][lane] = dm;
            K += __popcll(dm);
        }
        if (K) deg = p.row_ptr[v + 1] - p.row_ptr[v];
        const int ne = edges_per_item(p, K);
        const int hs = K > 0 ? 1 : 0;
        const int nch = deg > 0 ? (deg + ne - 1) / ne : 0;
        int sk = K, sh = hs, sc = nch, dg = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a1 = __shfl_up_sync(kFull, sk, o), a2 = __shfl_up_sync(kFull, sh, o),
                      a3 = __shfl_up_sync(kFull, sc, o);
            if (lane >= o) {
                sk += a1;
                sh += a2;
                sc += a3;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dg += __shfl_xor_sync(kFull, dg, o);
        unsigned long long ps0 = 0;
        int item0 = 0;
        if (lane == 31) {
            if (sk) ps0 = atomicAdd((unsigned long long *)p.out.cnt, ((unsigned long long)sh << 32) | (unsigned)sk);
            if (sc) item0 = atomicAdd(&p.out.cnt[2], sc);
        }
        if (lane == 0 && dg) atomicAdd(&p.out.cnt[3], dg);
        ps0 = __shfl_sync(kFull, ps0, 31);
        item0 = __shfl_sync(kFull, item0, 31);
        const int n_pairs = __shfl_sync(kFull, sk, 31), n_items = __shfl_sync(kFull, sc, 31);
        const int pool0 = (int)(uint32_t)ps0;
        const int slot = (int)(ps0 >> 32) + sh - hs;
        if (K) {
            p.out.node[slot] = v;
            p.out.poff[slot] = pool0 + sk - K;
            p.out.pk[slot] = K;
        }
        s_pp[wid][lane + 1] = sk;
        s_ip[wid][lane + 1] = sc;
        s_v[wid][lane] = v;
        s_slot[wid][lane] = slot;
        s_ne[wid][lane] = ne;
        __syncwarp();
        for (int q0 = 0; q0 < n_pairs; q0 += 32 * kU) {
            uint64_t x[kU];
            size_t idx[kU];
            int w[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + 32 * u + lane;
                x[u] = 0ull;
                idx[u] = 0;
                w[u] = 0;
                if (q < n_pairs) {
                    // the r-th listed word of node j
                    const int j = owner_of(s_pp[wid], q);
                    int r = q - s_pp[wid][j], qq = 0;
                    uint64_t dm = s_dm[wid][0][j];
                    while (!ONE_WORD && r >= __popcll(dm)) {
                        r -= __popcll(dm);
                        dm = s_dm[wid][++qq][j];
                    }
                    w[u] = 64 * qq + nth_set_bit(dm, r);
                    idx[u] = (size_t)s_v[wid][j] * B + w[u];
                    x[u] = __ldcg((const unsigned long long *)p.nxt + idx[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + 32 * u + lane;
                if (q < n_pairs) {
                    p.nxt[idx[u]] = 0ull;
                    p.out.pw[pool0 + q] = (uint16_t)w[u];
                    p.out.pb[pool0 + q] = x[u];
                    pc += __popcll(x[u]);
                }
            }
        }
        for (int q = lane; q < n_items; q += 32) {
            const int j = owner_of(s_ip[wid], q);
            p.out.work[item0 + q] = make_int2(s_slot[wid][j], (q - s_ip[wid][j]) * s_ne[wid][j]);
        }
        __syncwarp();
    }
    add_level_count(p, pc);
}

// ---------------------------------------------------------------- LT counting form
// Set-up of a pass in the counting form (every node's non-zero in-weights equal w_v).  With k
// active in-neighbours, v activates iff k * w_v > theta, i.e. iff k > q = floor(theta / w_v).
// Each (node, word) keeps one counter per trial, bit-sliced over L_v planes (plane i holds bit i
// of the 64 trials' counters), started at c0 = 2^L_v - 1 - q (0 when q >= 2^L_v - 1): the k-th
// increment then carries out of the top plane exactly when k > q.  Since k never exceeds
// k_v <= 2^L_v - 1, c0 + k < 2^(L_v+1) and the carry happens at most once per trial, so the
// push can take it as the activation.  One warp per node; each iteration fills two words:
// lanes 0-15 draw the 64 thresholds of the first (one Philox block of 4 trials per lane),
// lanes 16-31 those of the second.
template <bool PERWORD>
__global__ void __launch_bounds__(kBlock) k_lt_init(Params p) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    const int h = lane >> 4, j = lane & 15;
    uint32_t n_dr = 0;
    for (int v = warp; v < p.n; v += n_warps) {
        const int32_t o0 = p.cnt_off[v];
        const int L = p.cnt_off[v + 1] - o0;
        if (L == 0) continue;
        const uint32_t wv = p.unit_w[v];
        const uint32_t top = (L >= 32) ? 0xFFFFFFFFu : ((1u << L) - 1u);
        uint64_t *base0 = p.planes + (size_t)o0 * B;
        for (int w0 = 0; w0 < B; w0 += 2) {
            // the counter starts of this lane's 4-trial block
            const int wh = min(w0 + h, B - 1);
            const U4 th = draw<PERWORD>(p, wh, (uint32_t)v, word_g0<PERWORD>(p, wh) + (uint64_t)j, 1u);
            if (w0 + h < B) ++n_dr;
            uint32_t c0[4];
            const uint32_t tv[4] = {th.x, th.y, th.z, th.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t q = tv[k] / wv;
                c0[k] = q < top ? top - q : 0u;
            }
            // trial t of a word sits in component t & 3 of the block drawn by lane t >> 2 of its
            // half; this lane gathers trials lane and lane + 32 of both words
            uint32_t a[4];  // {word 0 trial lane, word 0 trial lane+32, word 1 trial lane, word 1 trial lane+32}
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                const int src = 16 * (q4 >> 1) + 8 * (q4 & 1) + (lane >> 2);
                const uint32_t x0 = __shfl_sync(kFull, c0[0], src), x1 = __shfl_sync(kFull, c0[1], src),
                               x2 = __shfl_sync(kFull, c0[2], src), x3 = __shfl_sync(kFull, c0[3], src);
                const int cmp = lane & 3;
                a[q4] = cmp == 0 ? x0 : cmp == 1 ? x1 : cmp == 2 ? x2 : x3;
            }
            // planes of word w0 then of w0 + 1 are one contiguous run of 2L words: element e of
            // the run is kept by lane e % 32 in slot e / 32
            uint64_t s0 = 0, s1 = 0;
            for (int i = 0; i < L; ++i) {
                const uint64_t P0 = (uint64_t)__ballot_sync(kFull, (a[0] >> i) & 1u) |
                                    ((uint64_t)__ballot_sync(kFull, (a[1] >> i) & 1u) << 32);
                const uint64_t P1 = (uint64_t)__ballot_sync(kFull, (a[2] >> i) & 1u) |
                                    ((uint64_t)__ballot_sync(kFull, (a[3] >> i) & 1u) << 32);
                const int e0 = i, e1 = L + i;
                if ((e0 & 31) == lane) {
                    if (e0 < 32) s0 = P0;
                    else s1 = P0;
                }
                if ((e1 & 31) == lane) {
                    if (e1 < 32) s0 = P1;
                    else s1 = P1;
                }
            }
            const int run = (w0 + 1 < B) ? 2 * L : L;
            uint64_t *out = base0 + (size_t)w0 * L;
            if (lane < run) out[lane] = s0;
            if (32 + lane < run) out[32 + lane] = s1;
        }
    }
    count_add(p, C_DRAWS, n_dr);
}

// ---------------------------------------------------------------- push
// One warp per work item: the item's (edge, pair) tasks are spread over the
// lanes, task t = (edge t / k, pair t % k).
// Nibble j of x non-zero -> bit j of the result (16 bits).
__device__ __forceinline__ uint32_t nibble_mask(uint64_t x) {
    uint64_t m = (x | (x >> 1) | (x >> 2) | (x >> 3)) & 0x1111111111111111ull;
    m = (m | (m >> 3)) & 0x0303030303030303ull;
    m = (m | (m >> 6)) & 0x000F000F000F000Full;
    m = (m | (m >> 12)) & 0x000000FF000000FFull;
    m = (m | (m >> 24)) & 0xFFFFull;
    return (uint32_t)m;
}

// Per-warp queue that spreads the Philox calls of 32 IC tasks evenly over the
// lanes: a task with many 4-trial blocks to draw no longer stalls the warp.
struct DrawQueue {
    uint16_t q[32 * 16];  // (lane << 4) | block
    uint8_t res[32 * 16]; // live bits of the block's four trials
    uint64_t g0[32];
    uint32_t e[32], thr[32];
    uint16_t w[32];
};

template <int MODEL, bool PERWORD>
__global__ void __launch_bounds__(kBlock, kPushMinBlocks) k_push(Params p_) {
    Params p = p_;
    resolve(p);
    if (p.ctl && p.ctl->pull) return;  // graph mode: this step pulls
    __shared__ uint64_t s_b[kWarps][kStageB];
    __shared__ uint16_t s_w[kWarps][kStageB];
    __shared__ int32_t s_list[kWarps][64];
    __shared__ DrawQueue s_dq[MODEL == 0 ? kWarps : 1];
    const int lane = lane_id();
    const int wid = threadIdx.x >> 5;
    ListBuf lb{s_list[wid], 0};
    const int n_work = p.in.cnt[2];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    uint32_t n_edges = 0, n_fw = 0, n_wc = 0, n_dr = 0, n_up = 0;
    for (int wi = warp; wi < n_work; wi += n_warps) {
        const int2 it = p.in.work[wi];
        const int u = p.in.node[it.x];
        const int off = p.in.poff[it.x];
        const int k = p.in.pk[it.x];
        const int row0 = p.row_ptr[u];
        const int deg = p.row_ptr[u + 1] - row0;
        const int ne = edges_per_item(p, k);
        const int e_begin = row0 + it.y;
        const int e_cnt = min(ne, deg - it.y);
        const bool staged = k <= kStageB;
        if (staged)
            for (int j = lane; j < k; j += 32) {
                s_b[wid][j] = p.in.pb[off + j];
                s_w[wid][j] = p.in.pw[off + j];
            }
        __syncwarp();
        if (lane == 0) {
            n_edges += e_cnt;
            n_fw += k;
        }
        const uint32_t T = (uint32_t)e_cnt * (uint32_t)k;
        const uint32_t magic = 0xFFFFFFFFu / (uint32_t)k + 1u;
        for (uint32_t t0 = 0; t0 < T; t0 += 32) {
            const uint32_t t = t0 + lane;
            bool hit = false, claimed = false;  // claimed: this lane took mark[v] for the step
            int v = 0;
            uint64_t ic_c = 0;
            uint32_t ic_thr = 0;
            int ic_e = 0, ic_w = 0, ic_v = 0;
            size_t ic_idx = 0;
            if (t < T) {
                const uint32_t el = div_by(t, (uint32_t)k, magic);
                const int j = (int)(t - el * (uint32_t)k);
                const int e = e_begin + (int)el;
                const uint2 ed = __ldg(&p.edge[e]);
                v = (int)ed.x;
                const int w = staged ? (int)s_w[wid][j] : (int)p.in.pw[off + j];
                const uint64_t f = staged ? s_b[wid][j] : p.in.pb[off + j];
                const size_t idx = (size_t)v * B + w;
                if (MODEL == 0) {
                    ic_c = 0;
                    ic_thr = ed.y;
                    ic_e = e;
                    ic_w = w;
                    ic_v = v;
                    ic_idx = idx;
                    if (ic_thr != 0u) {
                        ++n_wc;
                        ic_c = f & ~(uint64_t)__ldcg((const unsigned long long *)p.vis + idx);
                    }
                } else if (MODEL == 2) {
                    // counting form: add 1 to the counters of the trials of c (bit-sliced ripple
                    // carry, plane by plane, atomically); what carries out of the top plane
                    // activates (see k_lt_init)
                    const uint32_t tag = ed.y;
                    if (tag != 0u) {
                        ++n_wc;
                        uint64_t carry = f & ~(uint64_t)__ldcg((const unsigned long long *)p.vis + idx);
                        if (carry) {
                            const uint32_t L = tag & 31u;
                            unsigned long long *pl =
                                (unsigned long long *)p.planes + ((size_t)(tag >> 5) * B + (size_t)w * L);
                            for (uint32_t i = 0; i < L && carry; ++i) {
                                ++n_up;
                                carry &= (uint64_t)atomicXor(pl + i, (unsigned long long)carry);
                            }
                            if (carry) {
                                // the update of nxt and the claim of the node's listing go out together
                                atomicOr((unsigned long long *)p.vis + idx, (unsigned long long)carry);
                                const uint64_t old =
                                    atomicOr((unsigned long long *)p.nxt + idx, (unsigned long long)carry);
                                claimed = atomicExch(&p.mark[v], p.stamp) != p.stamp;
                                mark_dirty(p, v, w, old);
                                hit = true;
                            }
                        }
                    }
                } else {
                    const uint32_t wt = ed.y;
                    if (wt != 0u) {
                        ++n_wc;
                        uint64_t c = f & ~(uint64_t)__ldcg((const unsigned long long *)p.vis + idx);
                        if (c) {
                            n_up += __popcll(c);
                            uint32_t *a = p.acc + idx * 64;
                            const bool conv = (__ldg((const unsigned long long *)p.cvt + (size_t)v * p.nq + (w >> 6)) >>
                                               (w & 63)) & 1ull;
                            if (!conv) {
                                // first touches of the row: plain sums, converted by the finalize
                                const uint64_t old =
                                    atomicOr((unsigned long long *)p.nxt + idx, (unsigned long long)c);
                                mark_dirty(p, v, w, old);
                                while (c) {
                                    const int b = __ffsll((long long)c) - 1;
                                    c &= c - 1;
                                    atomicAdd(a + b, wt);
                                }
                                hit = true;
                            } else {
                                // acc = ~theta + sum: the add that carries out of 32 bits is the
                                // one that lifts the sum above theta (at most one carry ever,
                                // since in-weights sum to at most 2^32 - 1)
                                uint64_t nb = 0;
                                while (c) {
                                    int bb[4];
                                    uint32_t ob[4];
#pragma unroll
                                    for (int q = 0; q < 4; ++q) {
                                        bb[q] = c ? __ffsll((long long)c) - 1 : -1;
                                        if (c) c &= c - 1;
                                    }
#pragma unroll
                                    for (int q = 0; q < 4; ++q) ob[q] = bb[q] >= 0 ? atomicAdd(a + bb[q], wt) : 0u;
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        if (bb[q] >= 0 && ob[q] + wt < ob[q]) nb |= 1ull << bb[q];
                                }
                                if (nb) {
                                    atomicOr((unsigned long long *)p.vis + idx, (unsigned long long)nb);
                                    const uint64_t old =
                                        atomicOr((unsigned long long *)p.nxt + idx, (unsigned long long)nb);
                                    mark_dirty(p, v, w, old);
                                    hit = true;
                                }
                            }
                        }
                    }
                }
            }
            if (MODEL == 0) {
                // coins: the 4-trial blocks of c that need a draw, queued and drawn
                // by all lanes; then the live bits go to vis / nxt
                DrawQueue &dq = s_dq[MODEL == 0 ? wid : 0];
                const uint64_t need = (ic_thr != kAlways) ? ic_c : 0ull;
                const uint32_t nm = nibble_mask(need);
                const int d = __popc(nm);
                int base = d;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int x = __shfl_up_sync(kFull, base, o);
                    if (lane >= o) base += x;
                }
                const int D = __shfl_sync(kFull, base, 31);
                base -= d;
                if (D > 0) {
                    dq.g0[lane] = word_g0<PERWORD>(p, ic_w);
                    dq.e[lane] = (uint32_t)ic_e;
                    dq.thr[lane] = ic_thr;
                    dq.w[lane] = (uint16_t)ic_w;
                    {
                        uint32_t mm = nm;
                        int r = base;
                        while (mm) {
                            const int j = __ffs(mm) - 1;
                            mm &= mm - 1;
                            dq.q[r++] = (uint16_t)((lane << 4) | j);
                        }
                    }
                    __syncwarp();
                    for (int qi = lane; qi < D; qi += 32) {
                        const uint32_t ent = dq.q[qi];
                        const int o = (int)(ent >> 4), j = (int)(ent & 15u);
                        const uint32_t th = dq.thr[o];
                        const U4 r = draw<PERWORD>(p, dq.w[o], dq.e[o], dq.g0[o] + (uint64_t)j, 0u);
                        dq.res[qi] = (uint8_t)((uint32_t)(r.x < th) | ((uint32_t)(r.y < th) << 1) |
                                               ((uint32_t)(r.z < th) << 2) | ((uint32_t)(r.w < th) << 3));
                        ++n_dr;
                    }
                    __syncwarp();
                }
                uint64_t nb = 0;
                if (ic_c) {
                    if (ic_thr == kAlways) {
                        nb = ic_c;
                    } else {
                        uint64_t live = 0;
                        uint32_t mm = nm;
                        int r = base;
                        while (mm) {
                            const int j = __ffs(mm) - 1;
                            mm &= mm - 1;
                            live |= (uint64_t)dq.res[r++] << (4 * j);
                        }
                        nb = ic_c & live;
                    }
                }
                if (nb) {
                    // vis: a reduction without return (no round trip); bits another task of this
                    // step has just set are or-ed again into nxt, which is idempotent
                    atomicOr((unsigned long long *)p.vis + ic_idx, (unsigned long long)nb);
                    const uint64_t old = atomicOr((unsigned long long *)p.nxt + ic_idx, (unsigned long long)nb);
                    claimed = atomicExch(&p.mark[ic_v], p.stamp) != p.stamp;
                    mark_dirty(p, ic_v, ic_w, old);
                    ++n_up;
                    hit = true;
                }
                __syncwarp();
            }
            if (MODEL == 1) lb.add(p, hit, v);
            else lb.put(p, claimed, v);
        }
        __syncwarp();
    }
    if (lb.n) lb.flush(p);
    count_add(p, C_EDGES, n_edges);
    count_add(p, C_FWORDS, n_fw);
    count_add(p, C_WCHECKS, n_wc);
    count_add(p, C_DRAWS, n_dr);
    count_add(p, C_UPDATES, n_up);
}

// ---------------------------------------------------------------- pull (IC)
// Scatter (SET) or clear (!SET) the step's frontier in node-indexed form: one
// warp per slot, lanes over its (word, bits) pairs.
template <bool SET>
__global__ void __launch_bounds__(kBlock) k_frontier_dense(Params p_) {
    Params p = p_;
    resolve(p);
    if (p.ctl && !p.ctl->pull) return;
    const int lane = lane_id();
    const int slots = p.in.cnt[1];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    for (int sl = warp; sl < slots; sl += n_warps) {
        const int u = p.in.node[sl];
        const int off = p.in.poff[sl], k = p.in.pk[sl];
        for (int j = lane; j < k; j += 32) p.fdense[(size_t)u * p.B + p.in.pw[off + j]] = SET ? p.in.pb[off + j] : 0ull;
        if (lane == 0) {
            if (SET) atomicOr(&p.fbits[u >> 5], 1u << (u & 31));
            else atomicAnd(&p.fbits[u >> 5], ~(1u << (u & 31)));
        }
    }
}

// Pull step of IC: one warp per node v with trials where it is still inactive;
// lanes own words.  The warp walks v's in-edges; for an in-neighbour u in the
// frontier it draws the coins of edge (u, v) only for the trials where u is
// newly active and v is still inactive -- trials activated by an earlier
// in-edge in this step need no further coin -- and stops once every trial of
// v is active.  v's words are written by this warp alone (no atomics).
template <bool PERWORD>
__global__ void __launch_bounds__(kBlock) k_pull_ic(Params p_) {
    Params p = p_;
    resolve(p);
    if (p.ctl && !p.ctl->pull) return;
    constexpr int NW = kPullMaxB / 32;
    __shared__ int32_t s_list[kWarps][64];
    const int lane = lane_id();
    const int wid = threadIdx.x >> 5;
    ListBuf lb{s_list[wid], 0};
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    uint32_t n_edges = 0, n_wc = 0, n_dr = 0, n_up = 0;
    for (int v = warp; v < p.n; v += n_warps) {
        uint64_t U[NW], nb[NW];
        bool open = false;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int w = lane + 32 * k;
            U[k] = w < B ? p.valid[w] & ~(uint64_t)p.vis[(size_t)v * B + w] : 0ull;
            nb[k] = 0ull;
            open |= U[k] != 0ull;
        }
        if (!__any_sync(kFull, open)) continue;
        const int e0 = p.in_row_ptr[v], e1 = p.in_row_ptr[v + 1];
        bool done = false;
        for (int eb = e0; eb < e1 && !done; eb += 32) {
            uint4 ie = make_uint4(0u, 0u, 0u, 0u);
            if (eb + lane < e1) ie = __ldg(&p.in_edge[eb + lane]);
            const bool fr = eb + lane < e1 && ie.z != 0u && ((p.fbits[ie.x >> 5] >> (ie.x & 31)) & 1u);
            unsigned todo = __ballot_sync(kFull, fr);
            if (lane == 0) n_edges += min(32, e1 - eb);
            while (todo) {
                const int sidx = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t u = __shfl_sync(kFull, ie.x, sidx);
                const uint32_t e = __shfl_sync(kFull, ie.y, sidx);
                const uint32_t thr = __shfl_sync(kFull, ie.z, sidx);
                bool still = false;
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    if (U[k] == 0ull) continue;
                    const int w = lane + 32 * k;
                    const uint64_t f = p.fdense[(size_t)u * B + w] & U[k];
                    ++n_wc;
                    if (f) {
                        uint64_t live = f;
                        if (thr != kAlways) {
                            live = 0;
                            const uint64_t g0 = word_g0<PERWORD>(p, w);
                            uint64_t c = f;
                            while (c) {
                                ++n_dr;
                                const int j = (__ffsll((long long)c) - 1) >> 2;
                                const U4 r = draw<PERWORD>(p, w, e, g0 + (uint64_t)j, 0u);
                                const uint32_t nib = (uint32_t)(r.x < thr) | ((uint32_t)(r.y < thr) << 1) |
                                                     ((uint32_t)(r.z < thr) << 2) | ((uint32_t)(r.w < thr) << 3);
                                live |= (uint64_t)nib << (4 * j);
                                c &= ~(0xFull << (4 * j));
                            }
                            live &= f;
                        }
                        nb[k] |= live;
                        U[k] &= ~live;
                    }
                    still |= U[k] != 0ull;
                }
                if (!__any_sync(kFull, still)) {
                    done = true;
                    break;
                }
            }
        }
        bool hit = false;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            if (nb[k] == 0ull) continue;
            const int w = lane + 32 * k;
            const size_t idx = (size_t)v * B + w;
            p.vis[idx] |= nb[k];
            p.nxt[idx] = nb[k];
            atomicOr((unsigned long long *)(p.dmask + (size_t)v * p.nq + (w >> 6)), 1ull << (w & 63));
            ++n_up;
            hit = true;
        }
        const bool any_hit = __any_sync(kFull, hit);
        lb.add(p, lane == 0 && any_hit, v);
    }
    if (lb.n) lb.flush(p);
    count_add(p, C_EDGES, n_edges);
    count_add(p, C_WCHECKS, n_wc);
    count_add(p, C_DRAWS, n_dr);
    count_add(p, C_UPDATES, n_up);
}

// ---------------------------------------------------------------- device step loop
// Start of a pass in graph mode: the seed step (-1) with a fresh stamp.
__global__ void k_pass_begin(Params p) {
    Ctl *c = p.ctl;
    c->level = -1;
    c->stamp += 1u;
    c->force = 1;
    c->pull = 0;
}

// The host loop's decision, on the device: run step L (the first step of a
// pass, or the one after the step just finalized)?  Prepares its counters and
// sets the WHILE condition of the pass's step loop.
// The device loop's step control (one thread): census of the frontier the last step produced,
// stop at an empty frontier, the level cap or the time limit (timeout_ns > 0, measured on the GPU's
// global timer from the call's first step), else set up the next step.
__global__ void k_ctl(Params p, cudaGraphConditionalHandle h, int32_t first, int32_t max_levels, int32_t may_pull,
                      int32_t pull_always, int32_t permille, int64_t m, int32_t tau,
                      unsigned long long timeout_ns) {
    Ctl *c = p.ctl;
    const unsigned long long now = global_ns();
    if (c->t0 == 0ull) c->t0 = now;
    const int L = first ? 0 : c->level + 1;
    const bool odd = (L & 1) != 0;
    const int32_t *cnt = odd ? p.fr[1].cnt : p.fr[0].cnt;
    const int32_t slots = cnt[1], items = cnt[2], fedges = cnt[3];
    const int32_t waiting = p.lcnt[odd ? 1 : 0];
    c->slots += (unsigned long long)slots;
    c->items += (unsigned long long)items;
    int go = 1;
    if (c->timed_out || (timeout_ns > 0ull && now - c->t0 > timeout_ns)) {
        c->timed_out = 1;
        go = 0;
    } else if (slots == 0 && waiting == 0) {
        go = 0;
    } else if (max_levels > 0 && L >= max_levels) {
        c->limit = 1;
        go = 0;
    } else if (items == 0 && waiting == 0) {
        go = 0;
    }
    if (go) {
        int32_t *ncnt = odd ? p.fr[0].cnt : p.fr[1].cnt;
        ncnt[0] = ncnt[1] = ncnt[2] = ncnt[3] = 0;
        p.lcnt[odd ? 0 : 1] = 0;
        c->level = L;
        c->stamp += 1u;
        c->force = items == 0 ? 1 : 0;
        c->pull = (may_pull && items > 0 && tau == 0 &&
                   (pull_always || (int64_t)fedges * 1000 > (int64_t)permille * m))
                      ? 1
                      : 0;
        c->levels += 1ull;
        c->pull_steps += (unsigned long long)c->pull;
    }
    cudaGraphSetConditional(h, (unsigned)go);
}

// ---------------------------------------------------------------- outputs
// Per-trial spread: warp k of a block owns word w and reduces 32 nodes at a
// time with one ballot per trial bit; trial b of word w lands at
// spread[wout[w] + b] (wout < 0: the word holds no trials).
__global__ void __launch_bounds__(256) k_spread(const uint64_t *__restrict__ vis, int32_t n, int32_t B,
                                                int32_t nwords, int32_t nodes_per_block,
                                                const int64_t *__restrict__ wout, int32_t *__restrict__ spread) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w >= nwords) return;
    const int64_t out = wout[w];
    if (out < 0) return;
    const int v0 = blockIdx.y * nodes_per_block;
    const int v1 = min(n, v0 + nodes_per_block);
    uint32_t lo = 0, hi = 0;
    for (int vb = v0; vb < v1; vb += 32) {
        const int v = vb + lane;
        const uint64_t x = (v < v1) ? __ldcs((const unsigned long long *)vis + (size_t)v * B + w) : 0ull;
        const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            const uint32_t ml = __ballot_sync(kFull, (xl >> b) & 1u);
            const uint32_t mh = __ballot_sync(kFull, (xh >> b) & 1u);
            if (lane == b) {
                lo += __popc(ml);
                hi += __popc(mh);
            }
        }
    }
    if (lo) atomicAdd(&spread[out + lane], (int)lo);
    if (hi) atomicAdd(&spread[out + 32 + lane], (int)hi);
}

// Per-node activation counts (accumulated over passes) and edge checks; one
// warp per node, lanes over words.  witem == null: one count row; else the
// count of word w goes to row witem[w] (one row per batch item).
__global__ void __launch_bounds__(256) k_counts(const uint64_t *__restrict__ vis, int32_t n, int32_t B,
                                                const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ witem,
                                                int32_t *__restrict__ count, unsigned long long *__restrict__ checks) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ck = 0;
    for (int v = warp; v < n; v += n_warps) {
        int s = 0;
        for (int w = lane; w < B; w += 32) {
            const int c = __popcll(__ldcs((const unsigned long long *)vis + (size_t)v * B + w));
            s += c;
            if (witem && c && count) atomicAdd(&count[(size_t)witem[w] * n + v], c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0 && s) {
            if (!witem && count) count[v] += s;
            ck += (unsigned long long)s * (unsigned long long)(row_ptr[v + 1] - row_ptr[v]);
        }
    }
    if (lane == 0 && ck) atomicAdd(checks, ck);
}

// ---------------------------------------------------------------- dispatch
static cudaError_t launch(const void *fn, int blocks, cudaStream_t st, Params &p) {
    void *args[] = {&p};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(kBlock), args, 0, st);
}

static int resident_blocks(const void *fn) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kBlock, 0) != cudaSuccess || b < 1) b = 1;
    return b;
}

// ---------------------------------------------------------------- driver
// Instantiated call graphs of recent call shapes, per host thread.  Every graph-mode call captures
// its graph (cheap: API calls only); when a cached executable of the same shape exists it is
// updated in place with the new capture's parameters (cudaGraphExecUpdate) instead of a new
// instantiation.  The capture stream is kept too.  Per thread, so that two host threads never
// share an executable; a call waits for its launch to finish before it returns, so the next call
// of the thread may update it.
struct ExecCache {
    struct Entry {
        uint64_t key;
        int device;
        cudaGraphExec_t x;
    };
    std::vector<Entry> e;
    cudaStream_t cs = nullptr;
    int cs_device = -1;
    ~ExecCache() {
        for (auto &q : e) cudaGraphExecDestroy(q.x);
        if (cs) cudaStreamDestroy(cs);
    }
};
static thread_local ExecCache t_exec;
constexpr size_t kExecCacheSize = 16;

static uint64_t mix_key(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h;
}

struct Work {
    cudaStream_t st = nullptr;
    std::vector<void *> allocs;
    ~Work() {
        for (void *q : allocs) cudaFreeAsync(q, st);
    }
    template <class T>
    cudaError_t alloc(T **ptr, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e == cudaSuccess) allocs.push_back(q);
        *ptr = (T *)q;
        return e;
    }
};

struct PinnedCounters {
    int32_t *h = nullptr;
    ~PinnedCounters() {
        if (h) cudaFreeHost(h);
    }
};
static thread_local PinnedCounters t_pinned;

// Keep up to a quarter of the device's memory cached in the stream-ordered
// pool between calls, so repeated simulations do not go back to the driver.
static void keep_pool(int device) {
    static bool done[64] = {};
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        uint64_t thr = total_b / 4;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[device] = true;
}

static int blocks_for(int64_t warps, int max_blocks) {
    const int64_t b = (warps + kWarps - 1) / kWarps;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, max_blocks));
}

// One simulation problem: a seed set, a trial count and a Philox key.
struct ItemDesc {
    int64_t seed_begin, seed_end;  // range in the seed array
    int64_t trials;
    int64_t out0;                  // position of its first trial in the spread output
    uint64_t key;
};

// Pass layout: runs of word columns, each from one item.
struct Seg {
    int32_t item;
    int64_t lw0;  // first word of the item in this run
    int32_t col0, cnt;
};

template <int MODEL, bool PERWORD>
static const void *push_fn() {
    return (const void *)k_push<MODEL, PERWORD>;
}

// Runs the items' trials: words of all items are packed into passes of B
// word columns (an item may span passes; trials are independent), and each
// pass runs the level loop over all its columns at once.
//   seeds_dev: all seeds on the device; items index into it.
//   spread: device, zeroed, sum of trials entries; counts: device, zeroed,
//   n x (batched ? items : 1) entries, or null.
static cnd_status run_items(int model, const cnd_graph_dev &G, const char *fn, std::vector<ItemDesc> items,
                            const int32_t *seeds_dev, bool batched, int32_t *d_spread, int32_t *d_count,
                            unsigned long long *d_checks, unsigned long long *d_lc, int32_t *d_bad,
                            const cnd_sim_opts &o, Work &W, bool &limit_hit) {
    cudaStream_t st = W.st;
    const int32_t n = G.n;
    // LT in the counting form where the graph allows it (unless the caller asks for the sums)
    const bool lt_cnt = model == 1 && G.lt_cnt_edge != nullptr && !o.lt_accumulate;
    const uint2 *edge = model == 0 ? G.ic_edge : (lt_cnt ? G.lt_cnt_edge : G.lt_edge);
    int64_t total_words = 0;
    for (const auto &it : items) total_words += (it.trials + 63) / 64;
    cnd_sim_stats *S = o.stats;
    if (total_words == 0) return CND_OK;
    const bool timing = S && (S->flags & CND_STATS_TIMING);
    unsigned long long *d_ctr = nullptr;
    if (S && (S->flags & CND_STATS_COUNT)) {
        CND_CUDA_TRY(W.alloc(&d_ctr, C_N));
        CND_CUDA_TRY(cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long) * C_N, st));
    }
    struct Events {
        cudaEvent_t e[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        ~Events() {
            for (auto x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    if (timing)
        for (auto &x : ev.e) CND_CUDA_TRY(cudaEventCreate(&x));
    bool timing_pending = false, setup_pending = false;
    auto collect_timing = [&]() -> cnd_status {
        if (setup_pending) {
            float c = 0.f;
            CND_CUDA_TRY(cudaEventElapsedTime(&c, ev.e[4], ev.e[5]));
            S->setup_ms += c;
            setup_pending = false;
        }
        if (!timing_pending) return CND_OK;
        float a = 0.f, b = 0.f;
        CND_CUDA_TRY(cudaEventElapsedTime(&a, ev.e[0], ev.e[1]));
        CND_CUDA_TRY(cudaEventElapsedTime(&b, ev.e[2], ev.e[3]));
        S->expand_ms += a;
        S->finalize_ms += b;
        timing_pending = false;
        return CND_OK;
    };

    // ---- pass width
    size_t free_b = 0, total_b = 0;
    CND_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const double budget = 0.6 * (double)free_b;
    // bytes per word column: vis, nxt, two pair pools (+ LT accumulators or counter planes)
    const double per_word = (double)n * (2 * 8 + 2 * 10 + (model == 1 && !lt_cnt ? 256 : 0)) +
                            (lt_cnt ? 8.0 * (double)G.lt_planes : 0.0);
    // pulling (IC) happens only when asked for: by direction, or by a switch threshold
    const bool may_pull = model == 0 && G.m > 0 &&
                          (o.direction == CND_DIR_PULL || (o.direction == CND_DIR_AUTO && o.pull_permille > 0));
    int64_t bmax = o.word_bits ? o.word_bits / 64 : kMaxB;
    bmax = std::min<int64_t>(bmax, std::max<int64_t>(1, (int64_t)(budget / per_word)));
    bmax = std::min<int64_t>(bmax, may_pull ? kPullMaxB : kMaxB);
    bmax = std::min<int64_t>(bmax, std::max<int64_t>(1, (int64_t)0x7FFFFFFF / std::max(n, 1)));
    const int64_t n_pass = (total_words + bmax - 1) / bmax;
    const int B = (int)((total_words + n_pass - 1) / n_pass);
    const int nq = (B + 63) / 64;

    // ---- pass layout: items by decreasing size, runs of columns
    std::vector<int32_t> order(items.size());
    for (size_t i = 0; i < items.size(); ++i) order[i] = (int32_t)i;
    if (batched)
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return items[a].trials > items[b].trials; });
    std::vector<std::vector<Seg>> passes(1);
    {
        int32_t col = 0;
        for (int32_t it : order) {
            int64_t words = (items[it].trials + 63) / 64, lw = 0;
            while (words > 0) {
                if (col == B) {
                    passes.emplace_back();
                    col = 0;
                }
                const int32_t take = (int32_t)std::min<int64_t>(words, B - col);
                passes.back().push_back(Seg{it, lw, col, take});
                col += take;
                lw += take;
                words -= take;
            }
        }
    }

    const size_t nB = (size_t)n * B;
    const int chunk = std::min(o.chunk_edges, 16384);  // task index < 2^32 / k in k_push's division
    const size_t work_cap = chunk > 0 ? (size_t)n + (size_t)G.m / chunk + 1
                                      : (size_t)n + 2 * (size_t)G.m * (size_t)B / kTasks + (size_t)G.m + 1;
    Params P{};
    P.n = n;
    P.B = B;
    P.nq = nq;
    P.chunk = chunk;
    P.row_ptr = G.row_ptr;
    P.edge = edge;
    P.rk = round_keys(items[0].key);
    P.level_counts = d_lc;
    P.lc_len = o.level_counts_len;
    Frontier fr[2];
    CND_CUDA_TRY(W.alloc(&P.vis, nB));
    CND_CUDA_TRY(W.alloc(&P.nxt, nB));
    CND_CUDA_TRY(W.alloc(&P.dmask, (size_t)n * nq));
    CND_CUDA_TRY(W.alloc(&P.mark, (size_t)n));
    int32_t *lists[2] = {nullptr, nullptr}, *d_lcnt = nullptr;
    CND_CUDA_TRY(W.alloc(&lists[0], (size_t)n));
    CND_CUDA_TRY(W.alloc(&lists[1], (size_t)n));
    CND_CUDA_TRY(W.alloc(&d_lcnt, 2));
    // column descriptors of every pass, uploaded as one block; pass i's part:
    // valid[B] | wg0[B] | wout[B] | wkey[B] | witem[B] (+pad) | seed runs
    size_t max_runs = 0;
    for (const auto &ps : passes) max_runs = std::max(max_runs, ps.size());
    const size_t desc_words = 4 * (size_t)B + (size_t)(B + 1) / 2 + 2 * max_runs;
    const size_t n_pass_all = passes.size();
    uint64_t *d_desc = nullptr;
    CND_CUDA_TRY(W.alloc(&d_desc, desc_words * n_pass_all));
    std::vector<uint64_t> h_desc(desc_words * n_pass_all, 0);
    struct PassInfo {
        int32_t nw_here;
        bool perword;
        uint64_t key, g_base;
    };
    std::vector<PassInfo> pinfo(n_pass_all);
    for (size_t pass = 0; pass < n_pass_all; ++pass) {
        const std::vector<Seg> &ps = passes[pass];
        uint64_t *hv = h_desc.data() + pass * desc_words, *hg = hv + B;
        int64_t *ho = (int64_t *)(hg + B);
        uint2 *hk = (uint2 *)(ho + B);
        int32_t *hi = (int32_t *)(hk + B);
        SeedSeg *hs = (SeedSeg *)(hv + 4 * (size_t)B + (size_t)(B + 1) / 2);
        bool one_key = true;
        int32_t nw_here = 0;
        for (size_t r = 0; r < ps.size(); ++r) {
            const Seg &sg = ps[r];
            const ItemDesc &it = items[sg.item];
            one_key = one_key && it.key == items[ps[0].item].key;
            for (int32_t c = 0; c < sg.cnt; ++c) {
                const int32_t col = sg.col0 + c;
                const int64_t lw = sg.lw0 + c;
                const int64_t left = it.trials - 64 * lw;
                hv[col] = left >= 64 ? ~0ull : ((1ull << left) - 1ull);
                hg[col] = (uint64_t)(o.first_trial + 64 * lw) >> 2;
                ho[col] = it.out0 + 64 * lw;
                hk[col] = make_uint2((uint32_t)it.key, (uint32_t)(it.key >> 32));
                hi[col] = sg.item;
            }
            hs[r] = SeedSeg{(int32_t)it.seed_begin, (int32_t)it.seed_end, sg.col0, sg.cnt};
            nw_here = std::max(nw_here, sg.col0 + sg.cnt);
        }
        for (int32_t col = nw_here; col < B; ++col) ho[col] = -1;
        // one key and consecutive trial blocks: the key goes in the launch parameters
        bool uniform = one_key;
        for (int32_t col = 1; col < nw_here && uniform; ++col) uniform = hg[col] == hg[0] + 16ull * col;
        pinfo[pass] = PassInfo{nw_here, !uniform, items[ps[0].item].key, hg[0]};
    }
    CND_CUDA_TRY(cudaMemcpyAsync(d_desc, h_desc.data(), sizeof(uint64_t) * h_desc.size(), cudaMemcpyHostToDevice, st));
    // launch parameters of pass i's kernels
    auto pass_params = [&](size_t pass, Params q) {
        uint64_t *dv = d_desc + pass * desc_words;
        q.valid = dv;
        q.wg0 = dv + B;
        q.wkey = (const uint2 *)(dv + 3 * (size_t)B);
        q.rk = round_keys(pinfo[pass].key);
        q.g_base = pinfo[pass].g_base;
        q.nvalid = pinfo[pass].nw_here;
        return q;
    };
    auto pass_wout = [&](size_t pass) { return (const int64_t *)(d_desc + pass * desc_words + 2 * (size_t)B); };
    auto pass_witem = [&](size_t pass) { return (const int32_t *)(d_desc + pass * desc_words + 4 * (size_t)B); };
    auto pass_segs = [&](size_t pass) {
        return (const SeedSeg *)(d_desc + pass * desc_words + 4 * (size_t)B + (size_t)(B + 1) / 2);
    };

    P.tau = o.defer_bits;
    P.max_wait = o.defer_steps;
    if (o.defer_bits > 0 && o.defer_steps > 0) CND_CUDA_TRY(W.alloc(&P.age, nB));
    if (lt_cnt) {
        CND_CUDA_TRY(W.alloc(&P.planes, (size_t)G.lt_planes * (size_t)B));
        P.cnt_off = G.lt_cnt_off;
        P.unit_w = G.lt_unit_w;
    } else if (model == 1) {
        CND_CUDA_TRY(W.alloc(&P.acc, nB * 64));
        CND_CUDA_TRY(W.alloc(&P.cvt, (size_t)n * nq));
    }
    // pull direction (IC only): node-indexed frontier and frontier-node bitmap
    const int permille = o.pull_permille > 0 ? o.pull_permille : kPullPermille;
    if (may_pull) {
        CND_CUDA_TRY(W.alloc(&P.fdense, nB));
        CND_CUDA_TRY(W.alloc(&P.fbits, (size_t)(n + 31) / 32));
        CND_CUDA_TRY(cudaMemsetAsync(P.fdense, 0, sizeof(uint64_t) * nB, st));
        CND_CUDA_TRY(cudaMemsetAsync(P.fbits, 0, sizeof(uint32_t) * ((size_t)(n + 31) / 32), st));
        P.in_row_ptr = G.in_row_ptr;
        P.in_edge = G.in_edge;
    }
    for (int i = 0; i < 2; ++i) {
        CND_CUDA_TRY(W.alloc(&fr[i].node, (size_t)n));
        CND_CUDA_TRY(W.alloc(&fr[i].poff, (size_t)n));
        CND_CUDA_TRY(W.alloc(&fr[i].pk, (size_t)n));
        CND_CUDA_TRY(W.alloc(&fr[i].pw, nB));
        CND_CUDA_TRY(W.alloc(&fr[i].pb, nB));
        CND_CUDA_TRY(W.alloc(&fr[i].work, work_cap));
        CND_CUDA_TRY(W.alloc(&fr[i].cnt, 4));
    }
    P.ctr = d_ctr;
    if (S) {
        S->passes = (int32_t)passes.size();
        S->word_bits = 64 * B;
        S->lt_counters = lt_cnt ? 1 : 0;
    }
    CND_CUDA_TRY(cudaMemsetAsync(P.mark, 0xFF, sizeof(uint32_t) * (size_t)n, st));
    CND_CUDA_TRY(cudaMemsetAsync(P.nxt, 0, sizeof(uint64_t) * nB, st));
    CND_CUDA_TRY(cudaMemsetAsync(P.dmask, 0, sizeof(uint64_t) * (size_t)n * nq, st));
    if (!t_pinned.h) CND_CUDA_TRY(cudaMallocHost(&t_pinned.h, 6 * sizeof(int32_t)));
    int32_t *hcnt = t_pinned.h;

    // a pass whose columns share one key takes it as launch parameters
    // (the counting form's push draws nothing and its finalize only collects, like IC's)
    const void *k_push_pw = model == 0 ? push_fn<0, true>() : lt_cnt ? push_fn<2, false>() : push_fn<1, true>();
    const void *k_push_uk = model == 0 ? push_fn<0, false>() : lt_cnt ? push_fn<2, false>() : push_fn<1, false>();
    const void *k_fin_pw = model == 0 ? (const void *)k_finalize<1, true>
                           : lt_cnt   ? (const void *)k_finalize<1, false>
                                      : (const void *)k_finalize<2, true>;
    const void *k_fin_uk = model == 0 ? (const void *)k_finalize<1, false>
                           : lt_cnt   ? (const void *)k_finalize<1, false>
                                      : (const void *)k_finalize<2, false>;
    // nothing waits and a node's words fit one dirty-mask word: the barrier-free collect
    const bool flat = P.tau == 0 && nq <= kCollectNq;
    const void *k_col = nq == 1 ? (const void *)k_collect<true> : (const void *)k_collect<false>;
    if (flat && (model == 0 || lt_cnt)) k_fin_pw = k_fin_uk = k_col;
    const void *k_init_pw = (const void *)k_lt_init<true>, *k_init_uk = (const void *)k_lt_init<false>;
    const int init_blocks = G.num_sms * resident_blocks(k_init_uk);
    const void *k_seedfin = nq <= kCollectNq ? k_col : (const void *)k_finalize<1, false>;
    const int push_blocks = G.num_sms * resident_blocks(k_push_uk);
    const void *k_pull_pw = (const void *)k_pull_ic<true>, *k_pull_uk = (const void *)k_pull_ic<false>;
    const int pull_blocks = G.num_sms * resident_blocks(k_pull_uk);
    const int dense_blocks = G.num_sms * resident_blocks((const void *)k_frontier_dense<true>);
    const int fin_blocks = G.num_sms * resident_blocks(k_fin_uk);
    const int seed_blocks = G.num_sms * resident_blocks(k_seedfin);
    uint32_t stamp = 0;
    int64_t launches = 0;
    const auto t0 = std::chrono::steady_clock::now();

    const bool graph_mode = o.graph != 0 && !timing;
    for (size_t pass = 0; pass < passes.size() && !graph_mode; ++pass) {
        const std::vector<Seg> &ps = passes[pass];
        P = pass_params(pass, P);
        const int32_t nw_here = pinfo[pass].nw_here;
        const bool pw = pinfo[pass].perword;
        const int64_t *d_wout = pass_wout(pass);
        const int32_t *d_witem = pass_witem(pass);
        const SeedSeg *d_segs = pass_segs(pass);
        if (timing) CND_CUDA_TRY(cudaEventRecord(ev.e[4], st));
        CND_CUDA_TRY(cudaMemsetAsync(P.vis, 0, sizeof(uint64_t) * nB, st));
        if (P.age) CND_CUDA_TRY(cudaMemsetAsync(P.age, 0, nB, st));
        if (lt_cnt) {
            CND_CUDA_TRY(launch(pw ? k_init_pw : k_init_uk, init_blocks, st, P));
            launches += 1;
        } else if (model == 1) {
            CND_CUDA_TRY(cudaMemsetAsync(P.acc, 0, sizeof(uint32_t) * nB * 64, st));
            CND_CUDA_TRY(cudaMemsetAsync(P.cvt, 0, sizeof(uint64_t) * (size_t)n * nq, st));
        }
        if (timing) {
            CND_CUDA_TRY(cudaEventRecord(ev.e[5], st));
            setup_pending = true;
        }
        const void *k_push_fn = pw ? k_push_pw : k_push_uk;
        const void *k_fin_fn = pw ? k_fin_pw : k_fin_uk;

        // step 0: seeds (finalized from list 1 like an IC step; nothing waits)
        int cur = 0;
        CND_CUDA_TRY(cudaMemsetAsync(fr[cur].cnt, 0, 4 * sizeof(int32_t), st));
        CND_CUDA_TRY(cudaMemsetAsync(d_lcnt, 0, 2 * sizeof(int32_t), st));
        P.out = fr[cur];
        P.lin = lists[1];
        P.lin_cnt = d_lcnt + 1;
        P.lnext = lists[0];
        P.lnext_cnt = d_lcnt;
        P.force = 1;
        P.stamp = stamp++;
        P.level = 0;
        k_seed<<<std::max<int>(1, (int)ps.size()), 128, 0, st>>>(P, d_segs, (int32_t)ps.size(), seeds_dev, d_bad);
        CND_CUDA_TRY(cudaGetLastError());
        CND_CUDA_TRY(launch(k_seedfin, seed_blocks, st, P));
        launches += 2;
        P.force = 0;
        for (int L = 0;; ++L) {
            CND_CUDA_TRY(cudaMemcpyAsync(hcnt, fr[cur].cnt, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CND_CUDA_TRY(cudaMemcpyAsync(hcnt + 4, d_lcnt + (L & 1), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CND_CUDA_TRY(cudaStreamSynchronize(st));
            if (timing) {
                const cnd_status ts = collect_timing();
                if (ts != CND_OK) return ts;
            }
            // slots / work items of step L's frontier; nodes whose words wait
            const int32_t slots = hcnt[1], n_items_w = hcnt[2], front_edges = hcnt[3], waiting = hcnt[4];
            if (S) {
                S->frontier_slots += slots;
                S->work_items += n_items_w;
            }
            if (slots == 0 && waiting == 0) break;
            if (o.max_levels > 0 && L >= o.max_levels) {
                limit_hit = true;
                break;
            }
            if (n_items_w == 0 && waiting == 0) break;
            if (o.timeout_s > 0) {
                const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (el > o.timeout_s) {
                    set_error("%s: timed out after %.3f s", fn, el);
                    cudaStreamSynchronize(st);
                    return CND_ETIMEOUT;
                }
            }
            const int nx = cur ^ 1;
            CND_CUDA_TRY(cudaMemsetAsync(fr[nx].cnt, 0, 4 * sizeof(int32_t), st));
            CND_CUDA_TRY(cudaMemsetAsync(d_lcnt + ((L + 1) & 1), 0, sizeof(int32_t), st));
            P.in = fr[cur];
            P.out = fr[nx];
            P.lin = lists[L & 1];
            P.lin_cnt = d_lcnt + (L & 1);
            P.lnext = lists[(L + 1) & 1];
            P.lnext_cnt = d_lcnt + ((L + 1) & 1);
            P.stamp = stamp++;
            P.level = L + 1;
            // nothing to expand in this step: every waiting word goes now
            P.force = n_items_w == 0 ? 1 : 0;
            // direction: pull when the frontier's out-edges are a large share of m
            const bool pull = may_pull && n_items_w > 0 && P.tau == 0 &&
                              (o.direction == CND_DIR_PULL ||
                               (int64_t)front_edges * 1000 > (int64_t)permille * (int64_t)G.m);
            if (timing) CND_CUDA_TRY(cudaEventRecord(ev.e[0], st));
            if (pull) {
                CND_CUDA_TRY(launch((const void *)k_frontier_dense<true>, dense_blocks, st, P));
                CND_CUDA_TRY(launch(pw ? k_pull_pw : k_pull_uk, pull_blocks, st, P));
                CND_CUDA_TRY(launch((const void *)k_frontier_dense<false>, dense_blocks, st, P));
                launches += 3;
                if (S) S->pull_steps += 1;
            } else if (n_items_w > 0) {
                CND_CUDA_TRY(launch(k_push_fn, blocks_for(n_items_w, push_blocks), st, P));
                launches += 1;
            }
            if (timing) {
                CND_CUDA_TRY(cudaEventRecord(ev.e[1], st));
                CND_CUDA_TRY(cudaEventRecord(ev.e[2], st));
            }
            CND_CUDA_TRY(launch(k_fin_fn, fin_blocks, st, P));
            if (timing) {
                CND_CUDA_TRY(cudaEventRecord(ev.e[3], st));
                timing_pending = true;
            }
            launches += 1;
            if (S) {
                S->levels += 1;
                S->expand_launches += n_items_w > 0 ? 1 : 0;
                S->finalize_launches += 1;
            }
            cur = nx;
        }
        // outputs of this pass
        const int npb = 4096;
        dim3 grid((unsigned)((nw_here + 7) / 8), (unsigned)((n + npb - 1) / npb));
        k_spread<<<grid, 256, 0, st>>>(P.vis, n, B, nw_here, npb, d_wout, d_spread);
        CND_CUDA_TRY(cudaGetLastError());
        k_counts<<<blocks_for(n, G.num_sms * 8), 256, 0, st>>>(P.vis, n, B, G.row_ptr, batched ? d_witem : nullptr,
                                                                d_count, d_checks);
        CND_CUDA_TRY(cudaGetLastError());
        launches += 2;
    }
    if (graph_mode) {
        // ---- the whole run as one CUDA graph: per pass its set-up, the seed
        // step, a WHILE node over the steps (condition set on the device by
        // k_ctl) and its outputs; one launch
        Ctl *d_ctl = nullptr;
        CND_CUDA_TRY(W.alloc(&d_ctl, 1));
        CND_CUDA_TRY(cudaMemsetAsync(d_ctl, 0, sizeof(Ctl), st));
        P.ctl = d_ctl;
        P.fr[0] = fr[0];
        P.fr[1] = fr[1];
        P.lists[0] = lists[0];
        P.lists[1] = lists[1];
        P.lcnt = d_lcnt;
        struct Graph {
            cudaGraph_t g = nullptr;
            ~Graph() {
                if (g) cudaGraphDestroy(g);
            }
        } gr;
        if (!t_exec.cs || t_exec.cs_device != G.device) {
            if (t_exec.cs) cudaStreamDestroy(t_exec.cs);
            t_exec.cs = nullptr;
            CND_CUDA_TRY(cudaStreamCreateWithFlags(&t_exec.cs, cudaStreamNonBlocking));
            t_exec.cs_device = G.device;
        }
        CND_CUDA_TRY(cudaGraphCreate(&gr.g, 0));
        cudaStream_t cs = t_exec.cs;
        // shape of the call graph: what decides its nodes and their kinds (launch dimensions and
        // parameters may differ between calls of one shape)
        uint64_t shape = mix_key(0, (uint64_t)model);
        shape = mix_key(shape, lt_cnt ? 1 : 0);
        shape = mix_key(shape, (uint64_t)passes.size());
        shape = mix_key(shape, may_pull ? 1 : 0);
        shape = mix_key(shape, P.age ? 1 : 0);
        shape = mix_key(shape, (uint64_t)B);
        shape = mix_key(shape, (uint64_t)n);
        for (size_t pass = 0; pass < passes.size(); ++pass) shape = mix_key(shape, pinfo[pass].perword ? 1 : 0);
        std::vector<cudaGraphNode_t> tail;
        auto cap_begin = [&](cudaGraph_t target, const std::vector<cudaGraphNode_t> &deps) -> cudaError_t {
            return cudaStreamBeginCaptureToGraph(cs, target, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                                 cudaStreamCaptureModeRelaxed);
        };
        auto cap_end = [&](std::vector<cudaGraphNode_t> *tail_out) -> cudaError_t {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
            if (e != cudaSuccess) return e;
            if (tail_out) tail_out->assign(deps, deps + nd);
            cudaGraph_t gout = nullptr;
            return cudaStreamEndCapture(cs, &gout);
        };
        const int body_kernels = (may_pull ? 3 : 0) + 3;
        const unsigned long long timeout_ns =
            o.timeout_s > 0 ? (unsigned long long)std::max(1.0, std::min(o.timeout_s * 1e9, 1.8e19)) : 0ull;
        for (size_t pass = 0; pass < passes.size(); ++pass) {
            const std::vector<Seg> &ps = passes[pass];
            Params Q = pass_params(pass, P);
            const bool pw = pinfo[pass].perword;
            const int32_t nw_here = pinfo[pass].nw_here;
            cudaGraphConditionalHandle h;
            CND_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, gr.g, 0, 0));
            // set-up and seed step
            CND_CUDA_TRY(cap_begin(gr.g, tail));
            CND_CUDA_TRY(cudaMemsetAsync(P.vis, 0, sizeof(uint64_t) * nB, cs));
            if (P.age) CND_CUDA_TRY(cudaMemsetAsync(P.age, 0, nB, cs));
            if (lt_cnt) {
                CND_CUDA_TRY(launch(pw ? k_init_pw : k_init_uk, init_blocks, cs, Q));
                launches += 1;
            } else if (model == 1) {
                CND_CUDA_TRY(cudaMemsetAsync(P.acc, 0, sizeof(uint32_t) * nB * 64, cs));
                CND_CUDA_TRY(cudaMemsetAsync(P.cvt, 0, sizeof(uint64_t) * (size_t)n * nq, cs));
            }
            CND_CUDA_TRY(cudaMemsetAsync(fr[0].cnt, 0, 4 * sizeof(int32_t), cs));
            CND_CUDA_TRY(cudaMemsetAsync(d_lcnt, 0, 2 * sizeof(int32_t), cs));
            k_pass_begin<<<1, 1, 0, cs>>>(Q);
            k_seed<<<std::max<int>(1, (int)ps.size()), 128, 0, cs>>>(Q, pass_segs(pass), (int32_t)ps.size(),
                                                                      seeds_dev, d_bad);
            CND_CUDA_TRY(launch(k_seedfin, seed_blocks, cs, Q));
            k_ctl<<<1, 1, 0, cs>>>(Q, h, 1, o.max_levels, may_pull ? 1 : 0, o.direction == CND_DIR_PULL ? 1 : 0,
                                   permille, (int64_t)G.m, P.tau, timeout_ns);
            CND_CUDA_TRY(cudaGetLastError());
            CND_CUDA_TRY(cap_end(&tail));
            // the step loop
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t loop_node;
            CND_CUDA_TRY(cudaGraphAddNode(&loop_node, gr.g, tail.data(), nullptr, tail.size(), &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            CND_CUDA_TRY(cap_begin(body, {}));
            if (may_pull) {
                CND_CUDA_TRY(launch((const void *)k_frontier_dense<true>, dense_blocks, cs, Q));
                CND_CUDA_TRY(launch(pw ? k_pull_pw : k_pull_uk, pull_blocks, cs, Q));
                CND_CUDA_TRY(launch((const void *)k_frontier_dense<false>, dense_blocks, cs, Q));
            }
            CND_CUDA_TRY(launch(pw ? k_push_pw : k_push_uk, push_blocks, cs, Q));
            CND_CUDA_TRY(launch(pw ? k_fin_pw : k_fin_uk, fin_blocks, cs, Q));
            k_ctl<<<1, 1, 0, cs>>>(Q, h, 0, o.max_levels, may_pull ? 1 : 0, o.direction == CND_DIR_PULL ? 1 : 0,
                                   permille, (int64_t)G.m, P.tau, timeout_ns);
            CND_CUDA_TRY(cudaGetLastError());
            CND_CUDA_TRY(cap_end(nullptr));
            tail.assign(1, loop_node);
            // outputs of the pass
            CND_CUDA_TRY(cap_begin(gr.g, tail));
            const int npb = 4096;
            dim3 grid((unsigned)((nw_here + 7) / 8), (unsigned)((n + npb - 1) / npb));
            k_spread<<<grid, 256, 0, cs>>>(P.vis, n, B, nw_here, npb, pass_wout(pass), d_spread);
            k_counts<<<blocks_for(n, G.num_sms * 8), 256, 0, cs>>>(P.vis, n, B, G.row_ptr,
                                                                    batched ? pass_witem(pass) : nullptr, d_count,
                                                                    d_checks);
            CND_CUDA_TRY(cudaGetLastError());
            CND_CUDA_TRY(cap_end(&tail));
            launches += 6;
        }
        cudaGraphExec_t gx = nullptr;
        size_t slot = t_exec.e.size();
        for (size_t i = 0; i < t_exec.e.size(); ++i)
            if (t_exec.e[i].key == shape && t_exec.e[i].device == G.device) slot = i;
        if (slot < t_exec.e.size()) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(t_exec.e[slot].x, gr.g, &info) == cudaSuccess) {
                gx = t_exec.e[slot].x;
                if (S) S->graph_reused = 1;
            } else {
                cudaGetLastError();  // a refused update is not an error of the call
                cudaGraphExecDestroy(t_exec.e[slot].x);
                t_exec.e.erase(t_exec.e.begin() + (ptrdiff_t)slot);
            }
        }
        if (!gx) {
            CND_CUDA_TRY(cudaGraphInstantiate(&gx, gr.g, 0));
            if (t_exec.e.size() >= kExecCacheSize) {
                cudaGraphExecDestroy(t_exec.e.front().x);
                t_exec.e.erase(t_exec.e.begin());
            }
            t_exec.e.push_back(ExecCache::Entry{shape, G.device, gx});
        }
        CND_CUDA_TRY(cudaGraphLaunch(gx, st));
        Ctl hc;
        CND_CUDA_TRY(cudaMemcpyAsync(&hc, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CND_CUDA_TRY(cudaStreamSynchronize(st));
        if (hc.timed_out) {
            set_error("%s: timed out after %.3f s (device loop)", fn, o.timeout_s);
            return CND_ETIMEOUT;
        }
        if (hc.limit) limit_hit = true;
        launches += (int64_t)hc.levels * body_kernels;
        if (S) {
            S->levels = (int32_t)hc.levels;
            S->frontier_slots = (int64_t)hc.slots;
            S->work_items = (int64_t)hc.items;
            S->pull_steps = (int64_t)hc.pull_steps;
            S->expand_launches = (int64_t)hc.levels;
            S->finalize_launches = (int64_t)hc.levels;
        }
    }
    if (S) S->launches = launches;
    if (d_ctr) {
        unsigned long long hctr[C_N] = {0, 0, 0, 0, 0};
        CND_CUDA_TRY(cudaMemcpyAsync(hctr, d_ctr, sizeof(hctr), cudaMemcpyDeviceToHost, st));
        CND_CUDA_TRY(cudaStreamSynchronize(st));
        S->edges_scanned = (int64_t)hctr[C_EDGES];
        S->frontier_words = (int64_t)hctr[C_FWORDS];
        S->word_checks = (int64_t)hctr[C_WCHECKS];
        S->draws = (int64_t)hctr[C_DRAWS];
        S->updates = (int64_t)hctr[C_UPDATES];
    }
    CND_CUDA_TRY(cudaStreamSynchronize(st));
    if (timing) return collect_timing();
    return CND_OK;
}

// ---------------------------------------------------------------- autotuner
struct TuneVal {
    int32_t word_bits, chunk_edges, pull_permille, graph;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<const void *, int, int, int, int>, TuneVal> g_tune_cache;

static int log2_bucket(int64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

static cnd_status simulate_common(int model, const cnd_graph *g, const char *fn, int32_t n_items,
                                  const int64_t *seed_off, const int32_t *seeds, const int32_t *n_trials_arr,
                                  int64_t n_trials_one, const uint64_t *keys, uint64_t key_one, int32_t *spread_out,
                                  int32_t *count_out, const cnd_sim_opts *opts);

// Times the candidates on a sample; returns the best settings.
static cnd_status tune(int model, const cnd_graph *g, int32_t n_items, const int64_t *seed_off, const int32_t *seeds,
                       const int32_t *n_trials_arr, int64_t n_trials_one, const uint64_t *keys, uint64_t key_one,
                       bool batched, const cnd_sim_opts &base, TuneVal &best, double &best_ms) {
    // the sample: its own copies of the (small) item metadata
    int32_t ns_items = batched ? std::min(n_items, 4) : 1;
    std::vector<int32_t> tr((size_t)ns_items);
    int64_t total = 0;
    for (int32_t i = 0; i < ns_items; ++i) {
        tr[i] = batched ? std::min<int32_t>(n_trials_arr[i], 512) : (int32_t)std::min<int64_t>(n_trials_one, 4096);
        total += tr[i];
    }
    if (total == 0) {
        best = TuneVal{0, 0, 0, 0};
        best_ms = 0.0;
        return CND_OK;
    }
    const int64_t total_words = batched ? 0 : (total + 63) / 64;
    std::vector<int32_t> widths = {0};  // 0 = widest pass that fits
    for (int wb : {64 * 64, 16 * 64})
        if (!batched && wb < 64 * total_words) widths.push_back(wb);
    const std::vector<int32_t> chunks = {0, 32, 512};
    std::vector<int32_t> pulls = {0};
    if (model == 0) pulls.push_back(250);
    cnd_sim_opts o = base;
    o.autotune = 0;
    o.stats = nullptr;
    o.edge_checks_out = nullptr;
    o.level_counts_out = nullptr;
    o.level_counts_len = 0;
    o.max_levels = 0;
    o.direction = CND_DIR_AUTO;
    const bool dev = o.device_ptrs != 0;
    // outputs of the sample runs
    int32_t *d_sp = nullptr;
    std::vector<int32_t> h_sp;
    if (dev) {
        if (cudaMalloc(&d_sp, sizeof(int32_t) * (size_t)total) != cudaSuccess) {
            set_error("cnd_autotune: allocation failed");
            return CND_ENOMEM;
        }
    } else {
        h_sp.resize((size_t)total);
    }
    int32_t *sp = dev ? d_sp : h_sp.data();
    best_ms = 1e300;
    // one untimed run first (first-call costs: pool growth, module load)
    cnd_status st = simulate_common(model, g, "cnd_autotune", batched ? ns_items : 1, seed_off, seeds,
                                    batched ? tr.data() : nullptr, batched ? 0 : tr[0], keys, key_one, sp, nullptr, &o);
    for (int32_t wb : widths)
        for (int32_t ch : chunks)
            for (int32_t pm : pulls)
                for (int32_t gr : {0, 1}) {
                    o.word_bits = wb;
                    o.chunk_edges = ch;
                    o.pull_permille = pm;
                    o.graph = gr;
                    double t_best = 1e300;
                    for (int rep = 0; rep < 1 && st == CND_OK; ++rep) {
                        const auto t0 = std::chrono::steady_clock::now();
                        st = simulate_common(model, g, "cnd_autotune", batched ? ns_items : 1, seed_off, seeds,
                                             batched ? tr.data() : nullptr, batched ? 0 : tr[0], keys, key_one, sp,
                                             nullptr, &o);
                        if (st == CND_OK && dev) st = cudaStreamSynchronize((cudaStream_t)o.stream) == cudaSuccess
                                                          ? CND_OK
                                                          : CND_ECUDA;
                        const double ms =
                            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                        t_best = std::min(t_best, ms);
                    }
                    if (st != CND_OK) break;
                    if (t_best < best_ms) {
                        best_ms = t_best;
                        best = TuneVal{wb, ch, pm, gr};
                    }
                }
    if (d_sp) cudaFree(d_sp);
    return st;
}

static cnd_status apply_autotune(int model, const cnd_graph *g, int32_t n_items, const int64_t *seed_off,
                                 const int32_t *seeds, const int32_t *n_trials_arr, int64_t n_trials_one,
                                 const uint64_t *keys, uint64_t key_one, bool batched, cnd_sim_opts &o) {
    int64_t total = 0, n_seeds = 0;
    for (int32_t i = 0; i < (batched ? n_items : 1); ++i) {
        total += batched ? n_trials_arr[i] : n_trials_one;
        n_seeds += batched ? seed_off[i + 1] - seed_off[i] : seed_off[1];
    }
    const auto key = std::make_tuple((const void *)g, model, batched ? 1 : 0, log2_bucket(total),
                                     log2_bucket(std::max<int64_t>(1, n_seeds / std::max(1, batched ? n_items : 1))));
    TuneVal tv{};
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            tv = it->second;
            hit = true;
        }
    }
    if (!hit) {
        double ms = 0.0;
        const cnd_status st =
            tune(model, g, n_items, seed_off, seeds, n_trials_arr, n_trials_one, keys, key_one, batched, o, tv, ms);
        if (st != CND_OK) return st;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = tv;
    }
    o.word_bits = tv.word_bits;
    o.chunk_edges = tv.chunk_edges;
    o.pull_permille = tv.pull_permille;
    o.graph = tv.graph;
    return CND_OK;
}

// Shared front end of the single and batched entry points.
static cnd_status simulate_common(int model, const cnd_graph *g, const char *fn, int32_t n_items,
                                  const int64_t *seed_off, const int32_t *seeds, const int32_t *n_trials_arr,
                                  int64_t n_trials_one, const uint64_t *keys, uint64_t key_one, int32_t *spread_out,
                                  int32_t *count_out, const cnd_sim_opts *opts) {
    clear_error();
    cnd_sim_opts o;
    cnd_sim_opts_init(&o);
    if (opts) o = *opts;
    const bool batched = n_trials_arr != nullptr;
    if (!g) {
        set_error("%s: graph is NULL", fn);
        return CND_EINVAL;
    }
    const cnd_graph_dev &G = g->d;
    const uint2 *edge = model == 0 ? G.ic_edge : G.lt_edge;
    if (!edge && G.m > 0) {
        set_error("%s: graph was created without %s", fn, model == 0 ? "IC probabilities" : "LT weights");
        return CND_EINVAL;
    }
    if (n_items < 0 || (batched && n_items > 0 && (!seed_off || !keys)) || o.first_trial < 0 ||
        (o.first_trial & 63) || o.word_bits < 0 || (o.word_bits & 63) || o.word_bits > 64 * kMaxB ||
        o.level_counts_len < 0 || (o.level_counts_len > 0 && !o.level_counts_out) || o.chunk_edges < 0 ||
        o.direction < 0 || o.direction > 2 || o.defer_bits < 0 || o.defer_bits > 64 || o.defer_steps < 0 ||
        o.defer_steps > 255 || o.lt_accumulate < 0 || o.lt_accumulate > 1) {
        set_error("%s: bad arguments (items, first_trial %% 64, word_bits, level_counts, chunk, defer)", fn);
        return CND_EINVAL;
    }
    if (o.defer_bits > 0 && (o.level_counts_len > 0 || o.max_levels > 0)) {
        set_error("%s: defer_bits changes activation steps; it cannot be combined with level counts or max_levels", fn);
        return CND_EINVAL;
    }
    if (o.autotune) {
        const cnd_status ts = apply_autotune(model, g, n_items, seed_off, seeds, n_trials_arr, n_trials_one, keys,
                                             key_one, batched, o);
        if (ts != CND_OK) return ts;
        o.autotune = 0;
    }
    // ---- items
    std::vector<ItemDesc> items((size_t)n_items);
    int64_t total_trials = 0, n_seeds_total = 0;
    for (int32_t i = 0; i < n_items; ++i) {
        ItemDesc &it = items[i];
        it.seed_begin = batched ? seed_off[i] : 0;
        it.seed_end = batched ? seed_off[i + 1] : seed_off[1];
        it.trials = batched ? n_trials_arr[i] : n_trials_one;
        it.key = batched ? keys[i] : key_one;
        it.out0 = total_trials;
        if (it.seed_begin < 0 || it.seed_end < it.seed_begin || it.seed_end > 0x7FFFFFFFll || it.trials < 0 ||
            it.trials > 0x7FFFFFFFll) {
            set_error("%s: item %d: bad seed range or trial count", fn, i);
            return CND_EINVAL;
        }
        total_trials += it.trials;
        n_seeds_total = std::max(n_seeds_total, it.seed_end);
    }
    if (n_seeds_total > 0 && !seeds) {
        set_error("%s: seeds is NULL", fn);
        return CND_EINVAL;
    }
    const bool dev = o.device_ptrs != 0;
    if (!dev)
        for (int64_t i = 0; i < n_seeds_total; ++i)
            if (seeds[i] < 0 || seeds[i] >= G.n) {
                set_error("%s: seed %d out of range", fn, seeds[i]);
                return CND_EINVAL;
            }
    int prev_dev = 0;
    CND_CUDA_TRY(cudaGetDevice(&prev_dev));
    if (prev_dev != G.device) CND_CUDA_TRY(cudaSetDevice(G.device));
    struct Restore {
        int d, cur;
        ~Restore() {
            if (d != cur) cudaSetDevice(d);
        }
    } restore{prev_dev, G.device};

    keep_pool(G.device);
    Work W;
    W.st = (cudaStream_t)o.stream;
    cudaStream_t st = W.st;
    const int32_t n = G.n;
    const size_t count_rows = batched ? (size_t)n_items : 1;

    // ---- outputs on the device
    int32_t *d_spread = nullptr, *d_count = nullptr, *d_bad = nullptr;
    const int32_t *d_seeds = nullptr;
    unsigned long long *d_lc = nullptr, *d_checks = nullptr;
    const int lc_len = o.level_counts_len;
    if (dev && spread_out) d_spread = spread_out;
    else CND_CUDA_TRY(W.alloc(&d_spread, (size_t)std::max<int64_t>(total_trials, 1)));
    if (count_out) {
        if (dev) d_count = count_out;
        else CND_CUDA_TRY(W.alloc(&d_count, (size_t)n * count_rows));
    }
    CND_CUDA_TRY(W.alloc(&d_lc, (size_t)std::max(lc_len, 1)));
    CND_CUDA_TRY(W.alloc(&d_checks, 1));
    CND_CUDA_TRY(W.alloc(&d_bad, 1));
    if (dev) {
        d_seeds = seeds;
    } else {
        int32_t *tmp = nullptr;
        CND_CUDA_TRY(W.alloc(&tmp, (size_t)std::max<int64_t>(n_seeds_total, 1)));
        if (n_seeds_total)
            CND_CUDA_TRY(cudaMemcpyAsync(tmp, seeds, sizeof(int32_t) * n_seeds_total, cudaMemcpyHostToDevice, st));
        d_seeds = tmp;
    }
    if (total_trials) CND_CUDA_TRY(cudaMemsetAsync(d_spread, 0, sizeof(int32_t) * (size_t)total_trials, st));
    if (d_count) CND_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int32_t) * (size_t)n * count_rows, st));
    CND_CUDA_TRY(cudaMemsetAsync(d_lc, 0, sizeof(unsigned long long) * (size_t)std::max(lc_len, 1), st));
    CND_CUDA_TRY(cudaMemsetAsync(d_checks, 0, sizeof(unsigned long long), st));
    CND_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), st));

    cnd_sim_stats *S = o.stats;
    if (S) {
        const int32_t flags = S->flags;
        memset(S, 0, sizeof(*S));
        S->flags = flags;
    }
    bool limit_hit = false;
    const cnd_status rs =
        run_items(model, G, fn, items, d_seeds, batched, d_spread, d_count, d_checks, d_lc, d_bad, o, W, limit_hit);
    if (rs != CND_OK) return rs;

    // ---- results
    int32_t hbad = 0;
    CND_CUDA_TRY(cudaMemcpyAsync(&hbad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    std::vector<unsigned long long> hlc((size_t)std::max(lc_len, 1));
    unsigned long long hchecks = 0;
    if (dev) {
        if (o.edge_checks_out)
            CND_CUDA_TRY(cudaMemcpyAsync(o.edge_checks_out, d_checks, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        if (lc_len)
            CND_CUDA_TRY(cudaMemcpyAsync(o.level_counts_out, d_lc, sizeof(int64_t) * lc_len, cudaMemcpyDeviceToDevice, st));
    } else {
        if (spread_out && total_trials)
            CND_CUDA_TRY(cudaMemcpyAsync(spread_out, d_spread, sizeof(int32_t) * total_trials, cudaMemcpyDeviceToHost, st));
        if (count_out)
            CND_CUDA_TRY(cudaMemcpyAsync(count_out, d_count, sizeof(int32_t) * (size_t)n * count_rows,
                                         cudaMemcpyDeviceToHost, st));
        CND_CUDA_TRY(cudaMemcpyAsync(&hchecks, d_checks, sizeof(hchecks), cudaMemcpyDeviceToHost, st));
        if (lc_len)
            CND_CUDA_TRY(cudaMemcpyAsync(hlc.data(), d_lc, sizeof(unsigned long long) * lc_len, cudaMemcpyDeviceToHost, st));
    }
    CND_CUDA_TRY(cudaStreamSynchronize(st));
    if (!dev) {
        if (o.edge_checks_out) *o.edge_checks_out = (int64_t)hchecks;
        for (int i = 0; i < lc_len; ++i) o.level_counts_out[i] = (int64_t)hlc[i];
    }
    if (hbad) {
        set_error("%s: a seed id is out of range", fn);
        return CND_EINVAL;
    }
    if (limit_hit) {
        set_error("%s: trials still active at step max_levels = %d", fn, o.max_levels);
        return CND_ELIMIT;
    }
    return CND_OK;
}

static cnd_status simulate(int model, const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                           uint64_t rng_seed, int32_t *spread_out, int32_t *count_out, const cnd_sim_opts *opts) {
    const char *fn = model == 0 ? "cnd_ic_simulate" : "cnd_lt_simulate";
    if (n_seeds < 0 || (n_seeds > 0 && !seeds) || n_trials < 0 || n_trials > 0x7FFFFFFFll) {
        clear_error();
        set_error("%s: bad arguments (n_seeds, seeds, n_trials)", fn);
        return CND_EINVAL;
    }
    const int64_t off[2] = {0, n_seeds};
    return simulate_common(model, g, fn, 1, off, seeds, nullptr, n_trials, nullptr, rng_seed, spread_out, count_out,
                           opts);
}

static cnd_status simulate_batch(int model, const cnd_graph *g, int32_t n_items, const int64_t *seed_off,
                                 const int32_t *seeds, const int32_t *n_trials, const uint64_t *rng_seed,
                                 int32_t *spread_out, int32_t *count_out, const cnd_sim_opts *opts) {
    const char *fn = model == 0 ? "cnd_ic_simulate_batch" : "cnd_lt_simulate_batch";
    if (n_items < 0 || (n_items > 0 && (!seed_off || !n_trials || !rng_seed))) {
        clear_error();
        set_error("%s: bad arguments (n_items, seed_off, n_trials, rng_seed)", fn);
        return CND_EINVAL;
    }
    if (n_items == 0) {
        clear_error();
        return CND_OK;
    }
    return simulate_common(model, g, fn, n_items, seed_off, seeds, n_trials, 0, rng_seed, 0, spread_out, count_out,
                           opts);
}

}  // namespace cnd

using namespace cnd;

extern "C" {

cnd_status cnd_ic_simulate(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                           uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out) {
    return simulate(0, g, seeds, n_seeds, n_trials, rng_seed, spread_out, node_count_out, nullptr);
}

cnd_status cnd_lt_simulate(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                           uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out) {
    return simulate(1, g, seeds, n_seeds, n_trials, rng_seed, spread_out, node_count_out, nullptr);
}

cnd_status cnd_ic_simulate_ex(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                              uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out,
                              const cnd_sim_opts *opts) {
    return simulate(0, g, seeds, n_seeds, n_trials, rng_seed, spread_out, node_count_out, opts);
}

cnd_status cnd_lt_simulate_ex(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                              uint64_t rng_seed, int32_t *spread_out, int32_t *node_count_out,
                              const cnd_sim_opts *opts) {
    return simulate(1, g, seeds, n_seeds, n_trials, rng_seed, spread_out, node_count_out, opts);
}

cnd_status cnd_autotune(const cnd_graph *g, int32_t model, int32_t n_items, const int64_t *seed_off,
                        const int32_t *seeds, int32_t n_seeds, const int32_t *n_trials, const uint64_t *rng_seed,
                        const cnd_sim_opts *base, cnd_sim_opts *best_out, double *best_ms_out) {
    clear_error();
    if (!g || (model != 0 && model != 1) || n_items < 0 || !n_trials || !rng_seed || !best_out ||
        (n_items > 0 && !seed_off) || (n_items == 0 && n_seeds < 0)) {
        set_error("cnd_autotune: bad arguments");
        return CND_EINVAL;
    }
    cnd_sim_opts o;
    cnd_sim_opts_init(&o);
    if (base) o = *base;
    const bool batched = n_items > 0;
    const int64_t off1[2] = {0, n_seeds};
    TuneVal tv{};
    double ms = 0.0;
    const cnd_status st = tune(model, g, batched ? n_items : 1, batched ? seed_off : off1, seeds,
                               batched ? n_trials : nullptr, batched ? 0 : n_trials[0], rng_seed,
                               batched ? 0 : rng_seed[0], batched, o, tv, ms);
    if (st != CND_OK) return st;
    o.word_bits = tv.word_bits;
    o.chunk_edges = tv.chunk_edges;
    o.pull_permille = tv.pull_permille;
    o.graph = tv.graph;
    o.autotune = 0;
    *best_out = o;
    if (best_ms_out) *best_ms_out = ms;
    return CND_OK;
}

cnd_status cnd_ic_simulate_batch(const cnd_graph *g, int32_t n_items, const int64_t *seed_off, const int32_t *seeds,
                                 const int32_t *n_trials, const uint64_t *rng_seed, int32_t *spread_out,
                                 int32_t *node_count_out, const cnd_sim_opts *opts) {
    return simulate_batch(0, g, n_items, seed_off, seeds, n_trials, rng_seed, spread_out, node_count_out, opts);
}

cnd_status cnd_lt_simulate_batch(const cnd_graph *g, int32_t n_items, const int64_t *seed_off, const int32_t *seeds,
                                 const int32_t *n_trials, const uint64_t *rng_seed, int32_t *spread_out,
                                 int32_t *node_count_out, const cnd_sim_opts *opts) {
    return simulate_batch(1, g, n_items, seed_off, seeds, n_trials, rng_seed, spread_out, node_count_out, opts);
}

}  // extern "C"

// ============================================================================
// Allocation-free IC simulation (cnd_ic_simulate_noalloc).
//
// For callers that must not allocate device memory during a simulation call:
// the working state lives in one file-scope device array of fixed size,
// reserved when the library is loaded.  The kernels are the ones above; only
// the placement of their working arrays differs.
// ============================================================================
namespace cnd {

constexpr size_t kStaticScratchBytes = (size_t)CND_NOALLOC_SCRATCH_BYTES;

// Scratch shared by every cnd_ic_simulate_noalloc call on this device.  In
// host code this name is a host-side stand-in; kernels get the device
// address from cudaGetSymbolAddress (see static_scratch_ptr).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static unsigned char *g_static_ptr[64] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this; that call should come before
// any stream capture).
static cnd_status static_scratch_ptr(int device, unsigned char **out) {
    if (device < 0 || device >= 64) {
        set_error("cnd_ic_simulate_noalloc: device %d out of range", device);
        return CND_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[device]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("cnd_ic_simulate_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return CND_ECUDA;
        }
        g_static_ptr[device] = (unsigned char *)ptr;
    }
    *out = g_static_ptr[device];
    return CND_OK;
}

// Bump placement of the working arrays inside the static scratch.
struct Arena {
    unsigned char *base;
    size_t cap, used;
    template <class T>
    T *take(size_t count) {
        const size_t bytes = ((std::max<size_t>(count, 1) * sizeof(T)) + 255) & ~(size_t)255;
        T *p = (used + bytes <= cap) ? (T *)(base + used) : nullptr;
        used += bytes;
        return p;
    }
};

// Working arrays for a pass of B words: fills P and fr when `a.base` is set,
// and returns the bytes they need either way.
static size_t place_static(Arena &a, Params &P, Frontier (&fr)[2], int32_t n, int32_t m, int B,
                           uint64_t **d_valid, unsigned long long **d_checks, int32_t **d_bad) {
    const int nq = (B + 63) / 64;
    const size_t nB = (size_t)n * B;
    const size_t work_cap = (size_t)n + 2 * (size_t)m * (size_t)B / kTasks + (size_t)m + 1;
    P.vis = a.take<uint64_t>(nB);
    P.nxt = a.take<uint64_t>(nB);
    P.dmask = a.take<uint64_t>((size_t)n * nq);
    P.mark = a.take<uint32_t>((size_t)n);
    P.lin = a.take<int32_t>((size_t)n);
    P.lnext = a.take<int32_t>((size_t)n);
    P.lin_cnt = a.take<int32_t>(2);
    P.lnext_cnt = P.lin_cnt ? P.lin_cnt + 1 : nullptr;
    *d_valid = a.take<uint64_t>(2 * (size_t)B + 2);  // valid[B] | wout[B] | one seed run
    *d_checks = a.take<unsigned long long>(1);
    *d_bad = a.take<int32_t>(1);
    for (int i = 0; i < 2; ++i) {
        fr[i].node = a.take<int32_t>((size_t)n);
        fr[i].poff = a.take<int32_t>((size_t)n);
        fr[i].pk = a.take<int32_t>((size_t)n);
        fr[i].pw = a.take<uint16_t>(nB);
        fr[i].pb = a.take<uint64_t>(nB);
        fr[i].work = a.take<int2>(work_cap);
        fr[i].cnt = a.take<int32_t>(4);
    }
    return a.used;
}

static cnd_status simulate_noalloc(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                                   uint64_t rng_seed, int32_t *spread_out, int32_t *count_out, void *stream) {
    clear_error();
    const char *fn = "cnd_ic_simulate_noalloc";
    if (!g) {
        set_error("%s: graph is NULL", fn);
        return CND_EINVAL;
    }
    const cnd_graph_dev &G = g->d;
    if (!G.ic_edge && G.m > 0) {
        set_error("%s: graph was created without IC probabilities", fn);
        return CND_EINVAL;
    }
    if (n_seeds < 0 || (n_seeds > 0 && !seeds) || n_trials < 0 || n_trials > 0x7FFFFFFFll ||
        (n_trials > 0 && !spread_out) || !count_out) {
        set_error("%s: bad arguments (seeds, n_trials, spread_out and node_count_out are required)", fn);
        return CND_EINVAL;
    }
    int cur_dev = 0;
    CND_CUDA_TRY(cudaGetDevice(&cur_dev));
    if (cur_dev != G.device) {
        set_error("%s: the graph lives on device %d but device %d is current", fn, G.device, cur_dev);
        return CND_EINVAL;
    }
    const int32_t n = G.n;
    const int64_t total_words = (n_trials + 63) / 64;
    // the widest pass that fits the scratch
    Params P{};
    Frontier fr[2];
    uint64_t *d_valid = nullptr;
    unsigned long long *d_checks = nullptr;
    int32_t *d_bad = nullptr;
    int B = (int)std::min<int64_t>(std::max<int64_t>(total_words, 1), kMaxB);
    for (;; --B) {
        Arena probe{nullptr, kStaticScratchBytes, 0};
        if (place_static(probe, P, fr, n, G.m, B, &d_valid, &d_checks, &d_bad) <= kStaticScratchBytes) break;
        if (B == 1) {
            set_error("%s: a graph with n = %d, m = %d needs %zu bytes of scratch; the static scratch holds %zu",
                      fn, n, G.m, place_static(probe, P, fr, n, G.m, 1, &d_valid, &d_checks, &d_bad),
                      kStaticScratchBytes);
            return CND_EINVAL;
        }
    }
    unsigned char *base = nullptr;
    const cnd_status sst = static_scratch_ptr(G.device, &base);
    if (sst != CND_OK) return sst;
    Arena arena{base, kStaticScratchBytes, 0};
    place_static(arena, P, fr, n, G.m, B, &d_valid, &d_checks, &d_bad);

    cudaStream_t st = (cudaStream_t)stream;
    // the scratch keeps the previous call's contents: clear what must start at zero
    CND_CUDA_TRY(cudaMemsetAsync(spread_out, 0, sizeof(int32_t) * (size_t)n_trials, st));
    CND_CUDA_TRY(cudaMemsetAsync(count_out, 0, sizeof(int32_t) * (size_t)n, st));
    CND_CUDA_TRY(cudaMemsetAsync(d_checks, 0, sizeof(unsigned long long), st));
    CND_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), st));
    if (total_words > 0) {
        const int nq = (B + 63) / 64;
        const size_t nB = (size_t)n * B;
        const int64_t n_pass = (total_words + B - 1) / B;
        P.n = n;
        P.B = B;
        P.nq = nq;
        P.chunk = 0;
        P.tau = 0;
        P.max_wait = 0;
        P.force = 0;
        P.row_ptr = G.row_ptr;
        P.edge = G.ic_edge;
        P.rk = round_keys(rng_seed);
        P.level_counts = nullptr;
        P.lc_len = 0;
        P.valid = d_valid;
        P.ctr = nullptr;
        CND_CUDA_TRY(cudaMemsetAsync(P.mark, 0xFF, sizeof(uint32_t) * (size_t)n, st));
        CND_CUDA_TRY(cudaMemsetAsync(P.nxt, 0, sizeof(uint64_t) * nB, st));
        CND_CUDA_TRY(cudaMemsetAsync(P.dmask, 0, sizeof(uint64_t) * (size_t)n * nq, st));
        const void *k_push_fn = (const void *)k_push<0, false>;
        // nothing waits here (tau = 0): the barrier-free collect where a node's words fit its masks
        const void *k_fin_fn = nq == 1 ? (const void *)k_collect<true>
                               : nq <= kCollectNq ? (const void *)k_collect<false>
                                                  : (const void *)k_finalize<1, false>;
        const int push_blocks = G.num_sms * resident_blocks(k_push_fn);
        const int fin_blocks = G.num_sms * resident_blocks(k_fin_fn);
        uint64_t desc[2 * kMaxB + 2];  // valid[B] | wout[B] | one seed run
        uint64_t *valid = desc;
        int64_t *wout = (int64_t *)(desc + B);
        const int64_t *d_wout = (const int64_t *)(d_valid + B);
        const SeedSeg *d_seg = (const SeedSeg *)(d_valid + 2 * B);
        int32_t hcnt[4];
        uint32_t stamp = 0;
        for (int64_t pass = 0; pass < n_pass; ++pass) {
            const int64_t w0 = pass * B;
            const int64_t nw_here = std::min<int64_t>(B, total_words - w0);
            for (int w = 0; w < B; ++w) {
                const int64_t left = n_trials - (w0 + w) * 64;
                valid[w] = w >= nw_here ? 0ull : (left >= 64 ? ~0ull : ((1ull << left) - 1ull));
                wout[w] = w >= nw_here ? -1 : 64 * (w0 + w);
            }
            *(SeedSeg *)(desc + 2 * B) = SeedSeg{0, n_seeds, 0, (int32_t)nw_here};
            P.nvalid = (int32_t)nw_here;
            CND_CUDA_TRY(cudaMemcpyAsync(d_valid, desc, sizeof(uint64_t) * (2 * B + 2), cudaMemcpyHostToDevice, st));
            CND_CUDA_TRY(cudaMemsetAsync(P.vis, 0, sizeof(uint64_t) * nB, st));
            P.g_base = (uint64_t)(64 * w0) >> 2;
            int cur = 0;
            CND_CUDA_TRY(cudaMemsetAsync(fr[cur].cnt, 0, 4 * sizeof(int32_t), st));
            CND_CUDA_TRY(cudaMemsetAsync(P.lin_cnt, 0, 2 * sizeof(int32_t), st));
            P.out = fr[cur];
            P.stamp = stamp++;
            P.level = 0;
            P.force = 1;
            k_seed<<<1, 128, 0, st>>>(P, d_seg, 1, seeds, d_bad);
            CND_CUDA_TRY(cudaGetLastError());
            CND_CUDA_TRY(launch(k_fin_fn, fin_blocks, st, P));
            P.force = 0;
            for (;;) {
                CND_CUDA_TRY(cudaMemcpyAsync(hcnt, fr[cur].cnt, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                CND_CUDA_TRY(cudaStreamSynchronize(st));
                if (hcnt[1] == 0 || hcnt[2] == 0) break;
                const int nx = cur ^ 1;
                CND_CUDA_TRY(cudaMemsetAsync(fr[nx].cnt, 0, 4 * sizeof(int32_t), st));
                CND_CUDA_TRY(cudaMemsetAsync(P.lin_cnt, 0, sizeof(int32_t), st));
                P.in = fr[cur];
                P.out = fr[nx];
                P.stamp = stamp++;
                P.level += 1;
                CND_CUDA_TRY(launch(k_push_fn, blocks_for(hcnt[2], push_blocks), st, P));
                CND_CUDA_TRY(launch(k_fin_fn, fin_blocks, st, P));
                cur = nx;
            }
            const int npb = 4096;
            dim3 grid((unsigned)((nw_here + 7) / 8), (unsigned)((n + npb - 1) / npb));
            k_spread<<<grid, 256, 0, st>>>(P.vis, n, B, (int)nw_here, npb, d_wout, spread_out);
            CND_CUDA_TRY(cudaGetLastError());
            k_counts<<<blocks_for(n, G.num_sms * 8), 256, 0, st>>>(P.vis, n, B, G.row_ptr, nullptr, count_out,
                                                                    d_checks);
            CND_CUDA_TRY(cudaGetLastError());
        }
    }
    int32_t hbad = 0;
    CND_CUDA_TRY(cudaMemcpyAsync(&hbad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CND_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) {
        set_error("%s: a seed id is out of range", fn);
        return CND_EINVAL;
    }
    return CND_OK;
}

}  // namespace cnd

extern "C" cnd_status cnd_ic_simulate_noalloc(const cnd_graph *g, const int32_t *seeds, int32_t n_seeds,
                                              int64_t n_trials, uint64_t rng_seed, int32_t *spread_out,
                                              int32_t *node_count_out, void *stream) {
    return cnd::simulate_noalloc(g, seeds, n_seeds, n_trials, rng_seed, spread_out, node_count_out, stream);
}
