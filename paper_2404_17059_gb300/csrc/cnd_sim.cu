// Bit-parallel, level-synchronous Monte Carlo engine for the IC and LT models
// on sm_103a.
//
// Layout.  Trials are packed 64 to a uint64 word; a pass ("slab") holds B
// consecutive words, i.e. 64*B trials, and every node owns B contiguous words
// of each state array (node-major), so the state of one node in all of the
// slab's trials is one contiguous run of 8*B bytes:
//   vis[v*B + w]   bit b set <=> node v is active in trial 64*(w0+w) + b
//   nxt[v*B + w]   IC: bits first activated in the current step
//                  LT: bits whose accumulator grew in the current step
//   acc[(v*B + w)*64 + b]   LT: active in-weight of v in that trial (uint32)
// The frontier of a step is a compact list of (node, B frontier words)
// "slots" plus work items (slot, edge chunk) that split long rows into chunks
// of `chunk` edges, so that hubs are spread over many warps.
//
// Steps (Sec. 3 "Algorithms": only out-neighbours of nodes newly active in
// the previous step are examined, Observation 1):
//   seed select + finalize  -> step-0 frontier (seeds in every valid trial)
//   IC:  push       for every frontier edge (u,v) and word: c = f_u & ~vis_v;
//                   coins are drawn only for the 4-trial groups that have a
//                   bit in c; live bits are or-ed into vis_v and nxt_v
//        finalize   nxt -> next frontier slots, nxt cleared
//   LT:  push       for every frontier edge (u,v) and word: for each trial in
//                   f_u & ~vis_v add w(u,v) to acc; mark the word touched
//        finalize   for every touched word, draw the thresholds of the
//                   touched trials and activate where acc > theta
// then the per-trial spread and per-node counts are reduced from vis.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "cnd_common.cuh"

namespace cnd {

struct Frontier {
    int32_t *node = nullptr;  // [cap] node of each slot
    uint64_t *bits = nullptr; // [cap * B] frontier words of each slot
    int2 *work = nullptr;     // [work_cap] (slot, chunk index)
    int32_t *cnt = nullptr;   // device [2]: slots, work items
};

struct Params {
    int32_t n;
    int32_t B;
    int32_t chunk;
    const int32_t *row_ptr;
    const uint2 *edge;        // {col, IC threshold} or {col, LT weight}
    uint64_t *vis;
    uint64_t *nxt;
    uint32_t *acc;
    uint32_t *mark;           // [n] last stamp that enqueued the node
    Frontier in, out, tmp;
    uint32_t stamp;
    uint32_t k0, k1;          // Philox key
    uint64_t g_base;          // trial-group index (trial >> 2) of bit 0 of word 0
    unsigned long long *level_counts;
    int32_t lc_len;
    int32_t level;            // step whose frontier is being produced
    const uint64_t *valid;    // [B] valid-trial mask of each word
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t ld_cg(const uint64_t *p) { return __ldcg((const unsigned long long *)p); }

// IC: bits of `c` (trials of one word) whose edge e is live.  Coins come in
// blocks of four trials, one Philox call per block that has a bit in c.
__device__ __forceinline__ uint64_t ic_live_bits(uint32_t e, uint64_t g0, uint64_t c, uint32_t thr, uint32_t k0,
                                                 uint32_t k1) {
    uint64_t live = 0;
    while (c) {
        const int j = (__ffsll((long long)c) - 1) >> 2;
        const uint64_t g = g0 + (uint64_t)j;
        const U4 r = philox4x32_10(e, (uint32_t)g, 0u, (uint32_t)(g >> 32), k0, k1);
        const uint32_t nib = (uint32_t)(r.x < thr) | ((uint32_t)(r.y < thr) << 1) | ((uint32_t)(r.z < thr) << 2) |
                             ((uint32_t)(r.w < thr) << 3);
        live |= (uint64_t)nib << (4 * j);
        c &= ~(0xFull << (4 * j));
    }
    return live;
}

__device__ __forceinline__ void add_level_count(const Params &p, unsigned long long v) {
    // one atomic per warp
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v && p.level < p.lc_len) atomicAdd(&p.level_counts[p.level], v);
}

// Append the work items of the slots held by group leaders (`lead`) of this warp.
__device__ __forceinline__ void emit_work(const Params &p, bool lead, int slot, int v) {
    int nch = 0;
    if (lead) {
        const int deg = p.row_ptr[v + 1] - p.row_ptr[v];
        nch = (deg + p.chunk - 1) / p.chunk;
    }
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(kFull, nch > 0);
    while (pending) {
        const int src = __ffs(pending) - 1;
        pending &= pending - 1;
        const int nc = __shfl_sync(kFull, nch, src);
        const int sl = __shfl_sync(kFull, slot, src);
        int base = 0;
        if (lane == 0) base = atomicAdd(&p.out.cnt[1], nc);
        base = __shfl_sync(kFull, base, 0);
        for (int c = lane; c < nc; c += 32) p.out.work[base + c] = make_int2(sl, c);
    }
}

// ---------------------------------------------------------------- seeds
__global__ void k_seed_select(Params p, const int32_t *__restrict__ seeds, int32_t n_seeds, int32_t *__restrict__ bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_seeds; i += gridDim.x * blockDim.x) {
        const int s = seeds[i];
        if (s < 0 || s >= p.n) {
            atomicExch(bad, 1);
            continue;
        }
        if (atomicExch(&p.mark[s], p.stamp) != p.stamp) {
            const int slot = atomicAdd(&p.out.cnt[0], 1);
            p.out.node[slot] = s;
        }
    }
}

// Fill the frontier words of the out-list slots.  SEED: from the valid masks
// (and set vis); IC: from nxt (cleared on the way).  Emits the work items.
template <int LPE, int NW, bool SEED>
__global__ void __launch_bounds__(256) k_finalize(Params p) {
    constexpr int G = 32 / LPE;
    const int lane = threadIdx.x & 31, sub = lane % LPE, grp = lane / LPE;
    const int count = p.out.cnt[0];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    unsigned long long pc = 0;
    for (int base = warp * G; base < count; base += n_warps * G) {
        const int slot = base + grp;
        const bool act = slot < count;
        const int v = act ? p.out.node[slot] : 0;
        if (act) {
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const int w = sub + k * LPE;
                if (w >= B) break;
                const size_t idx = (size_t)v * B + w;
                uint64_t x;
                if (SEED) {
                    x = p.valid[w];
                    p.vis[idx] = x;
                } else {
                    x = p.nxt[idx];
                    p.nxt[idx] = 0;
                }
                p.out.bits[(size_t)slot * B + w] = x;
                pc += __popcll(x);
            }
        }
        emit_work(p, act && sub == 0, slot, v);
    }
    add_level_count(p, pc);
}

// ---------------------------------------------------------------- IC push
template <int LPE, int NW>
__global__ void __launch_bounds__(256) k_ic_push(Params p) {
    constexpr int EPW = 32 / LPE;
    const int lane = threadIdx.x & 31, sub = lane % LPE, grp = lane / LPE;
    const unsigned gmask = (LPE == 32) ? kFull : (((1u << LPE) - 1u) << (grp * LPE));
    const int n_work = p.in.cnt[1];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    for (int wi = warp; wi < n_work; wi += n_warps) {
        const int2 it = p.in.work[wi];
        const int u = p.in.node[it.x];
        const int e_begin = p.row_ptr[u] + it.y * p.chunk;
        const int e_end = min(p.row_ptr[u + 1], e_begin + p.chunk);
        uint64_t f[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int w = sub + k * LPE;
            f[k] = (w < B) ? p.in.bits[(size_t)it.x * B + w] : 0ull;
        }
        for (int e0 = e_begin; e0 < e_end; e0 += EPW) {
            const int e = e0 + grp;
            bool fresh = false;
            int v = 0;
            if (e < e_end) {
                const uint2 ed = __ldg(&p.edge[e]);
                v = (int)ed.x;
                const uint32_t thr = ed.y;
                if (thr != 0u) {
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        if (f[k] == 0) continue;
                        const int w = sub + k * LPE;
                        uint64_t *vp = p.vis + (size_t)v * B + w;
                        const uint64_t c = f[k] & ~ld_cg(vp);
                        if (c == 0) continue;
                        uint64_t nb = c;
                        if (thr != kAlways) nb &= ic_live_bits((uint32_t)e, p.g_base + 16ull * w, c, thr, p.k0, p.k1);
                        if (nb == 0) continue;
                        nb &= ~(uint64_t)atomicOr((unsigned long long *)vp, (unsigned long long)nb);
                        if (nb == 0) continue;
                        atomicOr((unsigned long long *)(p.nxt + (size_t)v * B + w), (unsigned long long)nb);
                        fresh = true;
                    }
                }
            }
            const unsigned fb = __ballot_sync(kFull, fresh);
            bool need = (sub == 0) && (fb & gmask);
            if (need) need = atomicExch(&p.mark[v], p.stamp) != p.stamp;
            const unsigned nm = __ballot_sync(kFull, need);
            if (nm) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&p.out.cnt[0], __popc(nm));
                base = __shfl_sync(kFull, base, 0);
                if (need) p.out.node[base + __popc(nm & ((1u << lane) - 1u))] = v;
            }
        }
    }
}

// ---------------------------------------------------------------- LT push
// Phase A of an LT step: accumulate the weight of every frontier in-neighbour
// into the trials where the target is still inactive; list the targets in tmp.
template <int LPE, int NW>
__global__ void __launch_bounds__(256) k_lt_push(Params p) {
    constexpr int EPW = 32 / LPE;
    const int lane = threadIdx.x & 31, sub = lane % LPE, grp = lane / LPE;
    const unsigned gmask = (LPE == 32) ? kFull : (((1u << LPE) - 1u) << (grp * LPE));
    const int n_work = p.in.cnt[1];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    for (int wi = warp; wi < n_work; wi += n_warps) {
        const int2 it = p.in.work[wi];
        const int u = p.in.node[it.x];
        const int e_begin = p.row_ptr[u] + it.y * p.chunk;
        const int e_end = min(p.row_ptr[u + 1], e_begin + p.chunk);
        uint64_t f[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int w = sub + k * LPE;
            f[k] = (w < B) ? p.in.bits[(size_t)it.x * B + w] : 0ull;
        }
        for (int e0 = e_begin; e0 < e_end; e0 += EPW) {
            const int e = e0 + grp;
            bool touched = false;
            int v = 0;
            if (e < e_end) {
                const uint2 ed = __ldg(&p.edge[e]);
                v = (int)ed.x;
                const uint32_t wt = ed.y;
                if (wt != 0u) {
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        if (f[k] == 0) continue;
                        const int w = sub + k * LPE;
                        const size_t idx = (size_t)v * B + w;
                        uint64_t c = f[k] & ~p.vis[idx];
                        if (c == 0) continue;
                        uint32_t *a = p.acc + idx * 64;
                        atomicOr((unsigned long long *)(p.nxt + idx), (unsigned long long)c);
                        while (c) {
                            const int b = __ffsll((long long)c) - 1;
                            c &= c - 1;
                            atomicAdd(a + b, wt);
                        }
                        touched = true;
                    }
                }
            }
            const unsigned fb = __ballot_sync(kFull, touched);
            bool need = (sub == 0) && (fb & gmask);
            if (need) need = atomicExch(&p.mark[v], p.stamp) != p.stamp;
            const unsigned nm = __ballot_sync(kFull, need);
            if (nm) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&p.tmp.cnt[0], __popc(nm));
                base = __shfl_sync(kFull, base, 0);
                if (need) p.tmp.node[base + __popc(nm & ((1u << lane) - 1u))] = v;
            }
        }
    }
}

// Phase B of an LT step: threshold test of every touched (node, trial).
template <int LPE, int NW>
__global__ void __launch_bounds__(256) k_lt_finalize(Params p) {
    constexpr int G = 32 / LPE;
    const int lane = threadIdx.x & 31, sub = lane % LPE, grp = lane / LPE;
    const int count = p.tmp.cnt[0];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int B = p.B;
    unsigned long long pc = 0;
    for (int base = warp * G; base < count; base += n_warps * G) {
        const int ts = base + grp;
        const bool act = ts < count;
        const int v = act ? p.tmp.node[ts] : 0;
        uint64_t nbw[NW];
        bool any = false;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            nbw[k] = 0;
            const int w = sub + k * LPE;
            if (!act || w >= B) continue;
            const size_t idx = (size_t)v * B + w;
            const uint64_t tb = p.nxt[idx];
            if (tb == 0) continue;
            p.nxt[idx] = 0;
            const uint64_t vis = p.vis[idx];
            uint64_t cand = tb & ~vis;
            const uint32_t *a = p.acc + idx * 64;
            uint64_t nb = 0;
            while (cand) {
                const int j = (__ffsll((long long)cand) - 1) >> 2;
                const uint64_t g = p.g_base + 16ull * w + (uint64_t)j;
                const U4 r = philox4x32_10((uint32_t)v, (uint32_t)g, 1u, (uint32_t)(g >> 32), p.k0, p.k1);
                const uint32_t th[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int b = 4 * j + q;
                    if ((cand >> b) & 1ull)
                        if (a[b] > th[q]) nb |= 1ull << b;
                }
                cand &= ~(0xFull << (4 * j));
            }
            if (nb) {
                p.vis[idx] = vis | nb;
                nbw[k] = nb;
                any = true;
                pc += __popcll(nb);
            }
        }
        // group-wide "any new bit" -> one slot per activated node
        const unsigned ab = __ballot_sync(kFull, any);
        const unsigned gmask = (LPE == 32) ? kFull : (((1u << LPE) - 1u) << (grp * LPE));
        const bool lead = act && sub == 0 && (ab & gmask);
        const unsigned lm = __ballot_sync(kFull, lead);
        int slot = 0;
        if (lm) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(&p.out.cnt[0], __popc(lm));
            b0 = __shfl_sync(kFull, b0, 0);
            if (lead) {
                slot = b0 + __popc(lm & ((1u << lane) - 1u));
                p.out.node[slot] = v;
            }
        }
        slot = __shfl_sync(kFull, slot, grp * LPE);
        const bool has = (ab & gmask) && act;
        if (has) {
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const int w = sub + k * LPE;
                if (w < B) p.out.bits[(size_t)slot * B + w] = nbw[k];
            }
        }
        emit_work(p, lead, slot, v);
    }
    add_level_count(p, pc);
}

// ---------------------------------------------------------------- outputs
// Per-trial spread: warp k of a block owns word w and reduces 32 nodes at a
// time with one ballot per trial bit.
__global__ void __launch_bounds__(256) k_spread(const uint64_t *__restrict__ vis, int32_t n, int32_t B,
                                                int32_t nwords, int32_t nodes_per_block, int32_t *__restrict__ spread) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w >= nwords) return;
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
    if (lo) atomicAdd(&spread[w * 64 + lane], (int)lo);
    if (hi) atomicAdd(&spread[w * 64 + 32 + lane], (int)hi);
}

// Per-node activation counts (accumulated over passes) and edge checks.
template <int LPE>
__global__ void __launch_bounds__(256) k_counts(const uint64_t *__restrict__ vis, int32_t n, int32_t B,
                                                const int32_t *__restrict__ row_ptr, int32_t *__restrict__ count,
                                                unsigned long long *__restrict__ checks) {
    constexpr int G = 32 / LPE;
    const int lane = threadIdx.x & 31, sub = lane % LPE, grp = lane / LPE;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ck = 0;
    for (int base = warp * G; base < n; base += n_warps * G) {
        const int v = base + grp;
        int s = 0;
        if (v < n)
            for (int w = sub; w < B; w += LPE) s += __popcll(vis[(size_t)v * B + w]);
#pragma unroll
        for (int o = LPE / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (v < n && sub == 0 && s) {
            count[v] += s;
            ck += (unsigned long long)s * (unsigned long long)(row_ptr[v + 1] - row_ptr[v]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) ck += __shfl_xor_sync(kFull, ck, o);
    if (lane == 0 && ck) atomicAdd(checks, ck);
}

// ---------------------------------------------------------------- dispatch
struct Shape {
    int lpe, nw;
};

static Shape shape_for(int B) {
    int lpe = 1;
    while (lpe < B && lpe < 32) lpe <<= 1;
    int nw = (B + lpe - 1) / lpe;
    int r = 1;
    while (r < nw) r <<= 1;
    return Shape{lpe, r};
}

#define CND_SHAPES(X)  \
    X(1, 1)            \
    X(2, 1)            \
    X(4, 1)            \
    X(8, 1)            \
    X(16, 1)           \
    X(32, 1)           \
    X(32, 2)           \
    X(32, 4)           \
    X(32, 8)

enum Kern { K_FIN_SEED, K_FIN_IC, K_IC_PUSH, K_LT_PUSH, K_LT_FIN };

static const void *kernel_ptr(Kern k, Shape s) {
#define PICK(L, N)                                                  \
    if (s.lpe == L && s.nw == N) {                                  \
        switch (k) {                                                \
            case K_FIN_SEED: return (const void *)k_finalize<L, N, true>;  \
            case K_FIN_IC: return (const void *)k_finalize<L, N, false>;   \
            case K_IC_PUSH: return (const void *)k_ic_push<L, N>;          \
            case K_LT_PUSH: return (const void *)k_lt_push<L, N>;          \
            case K_LT_FIN: return (const void *)k_lt_finalize<L, N>;       \
        }                                                           \
    }
    CND_SHAPES(PICK)
#undef PICK
    return nullptr;
}

static const void *counts_ptr(int lpe) {
    switch (lpe) {
        case 1: return (const void *)k_counts<1>;
        case 2: return (const void *)k_counts<2>;
        case 4: return (const void *)k_counts<4>;
        case 8: return (const void *)k_counts<8>;
        case 16: return (const void *)k_counts<16>;
        default: return (const void *)k_counts<32>;
    }
}

static cudaError_t launch(const void *fn, int blocks, cudaStream_t st, Params &p) {
    void *args[] = {&p};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(256), args, 0, st);
}

// ---------------------------------------------------------------- driver
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

static int blocks_for(int items_per_warp_unit, int64_t items, int max_blocks) {
    const int64_t warps = (items + items_per_warp_unit - 1) / items_per_warp_unit;
    const int64_t b = (warps + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, max_blocks));
}

static cnd_status simulate(int model, const cnd_graph *g, const int32_t *seeds, int32_t n_seeds, int64_t n_trials,
                           uint64_t rng_seed, int32_t *spread_out, int32_t *count_out, const cnd_sim_opts *opts) {
    clear_error();
    cnd_sim_opts o;
    cnd_sim_opts_init(&o);
    if (opts) o = *opts;
    const char *fn = model == 0 ? "cnd_ic_simulate" : "cnd_lt_simulate";
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
    if (n_seeds < 0 || (n_seeds > 0 && !seeds) || n_trials < 0 || n_trials > 0x7FFFFFFFll || o.first_trial < 0 ||
        (o.first_trial & 63) || o.word_bits < 0 || (o.word_bits & 63) || o.word_bits > 16384 ||
        o.level_counts_len < 0 || (o.level_counts_len > 0 && !o.level_counts_out) || o.chunk_edges < 0 ||
        o.direction < 0 || o.direction > 2) {
        set_error("%s: bad arguments (n_seeds, n_trials, first_trial %% 64, word_bits, level_counts, chunk)", fn);
        return CND_EINVAL;
    }
    const bool dev = o.device_ptrs != 0;
    if (!dev) {
        for (int32_t i = 0; i < n_seeds; ++i)
            if (seeds[i] < 0 || seeds[i] >= G.n) {
                set_error("%s: seed %d out of range", fn, seeds[i]);
                return CND_EINVAL;
            }
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

    // ---- outputs on the device
    const int64_t total_words = (n_trials + 63) / 64;
    int32_t *d_spread = nullptr, *d_count = nullptr, *d_seeds = nullptr, *d_bad = nullptr;
    unsigned long long *d_lc = nullptr, *d_checks = nullptr;
    const int lc_len = o.level_counts_len;
    CND_CUDA_TRY(W.alloc(&d_spread, (size_t)std::max<int64_t>(total_words, 1) * 64));
    if (dev && count_out) d_count = count_out;
    else CND_CUDA_TRY(W.alloc(&d_count, (size_t)n));
    CND_CUDA_TRY(W.alloc(&d_lc, (size_t)std::max(lc_len, 1)));
    CND_CUDA_TRY(W.alloc(&d_checks, 1));
    CND_CUDA_TRY(W.alloc(&d_bad, 1));
    if (dev) d_seeds = (int32_t *)seeds;
    else {
        CND_CUDA_TRY(W.alloc(&d_seeds, (size_t)std::max(n_seeds, 1)));
        if (n_seeds) CND_CUDA_TRY(cudaMemcpyAsync(d_seeds, seeds, sizeof(int32_t) * n_seeds, cudaMemcpyHostToDevice, st));
    }
    CND_CUDA_TRY(cudaMemsetAsync(d_spread, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(total_words, 1) * 64, st));
    CND_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int32_t) * (size_t)n, st));
    CND_CUDA_TRY(cudaMemsetAsync(d_lc, 0, sizeof(unsigned long long) * (size_t)std::max(lc_len, 1), st));
    CND_CUDA_TRY(cudaMemsetAsync(d_checks, 0, sizeof(unsigned long long), st));
    CND_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), st));

    bool limit_hit = false;
    if (total_words > 0) {
        // ---- pass width
        size_t free_b = 0, total_b = 0;
        CND_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const double budget = 0.6 * (double)free_b;
        // bytes per word column: vis, nxt, two frontier buffers (+ LT accumulators)
        const double per_word = (double)n * (4 * 8 + (model == 1 ? 256 : 0));
        int64_t bmax = o.word_bits ? o.word_bits / 64 : 256;
        bmax = std::min<int64_t>(bmax, std::max<int64_t>(1, (int64_t)(budget / per_word)));
        bmax = std::min<int64_t>(bmax, 256);
        const int64_t n_pass = (total_words + bmax - 1) / bmax;
        const int B = (int)((total_words + n_pass - 1) / n_pass);
        const Shape shp = shape_for(B);
        const int chunk = o.chunk_edges > 0 ? o.chunk_edges : std::max(32, (32 / shp.lpe) * 8);

        const size_t nB = (size_t)n * B;
        const size_t work_cap = (size_t)n + (size_t)G.m / chunk + 1;
        Params P{};
        P.n = n;
        P.B = B;
        P.chunk = chunk;
        P.row_ptr = G.row_ptr;
        P.edge = edge;
        P.k0 = (uint32_t)rng_seed;
        P.k1 = (uint32_t)(rng_seed >> 32);
        P.level_counts = d_lc;
        P.lc_len = lc_len;
        uint64_t *d_valid = nullptr;
        Frontier fr[3];
        CND_CUDA_TRY(W.alloc(&P.vis, nB));
        CND_CUDA_TRY(W.alloc(&P.nxt, nB));
        CND_CUDA_TRY(W.alloc(&P.mark, (size_t)n));
        CND_CUDA_TRY(W.alloc(&d_valid, (size_t)B));
        if (model == 1) CND_CUDA_TRY(W.alloc(&P.acc, nB * 64));
        for (int i = 0; i < 3; ++i) {
            if (i == 2 && model == 0) break;
            CND_CUDA_TRY(W.alloc(&fr[i].node, (size_t)n));
            CND_CUDA_TRY(W.alloc(&fr[i].cnt, 2));
            if (i < 2) {
                CND_CUDA_TRY(W.alloc(&fr[i].bits, nB));
                CND_CUDA_TRY(W.alloc(&fr[i].work, work_cap));
            }
        }
        P.valid = d_valid;
        CND_CUDA_TRY(cudaMemsetAsync(P.mark, 0xFF, sizeof(uint32_t) * (size_t)n, st));
        CND_CUDA_TRY(cudaMemsetAsync(P.nxt, 0, sizeof(uint64_t) * nB, st));
        if (!t_pinned.h) CND_CUDA_TRY(cudaMallocHost(&t_pinned.h, 4 * sizeof(int32_t)));
        int32_t *hcnt = t_pinned.h;

        const int max_blocks = G.num_sms * 8;
        uint32_t stamp = 0;
        std::vector<uint64_t> valid((size_t)B);
        const auto t0 = std::chrono::steady_clock::now();

        for (int64_t pass = 0; pass < n_pass; ++pass) {
            const int64_t w0 = pass * B;
            const int64_t nw_here = std::min<int64_t>(B, total_words - w0);
            for (int w = 0; w < B; ++w) {
                const int64_t word = w0 + w;
                if (w >= nw_here) valid[w] = 0;
                else {
                    const int64_t left = n_trials - word * 64;
                    valid[w] = left >= 64 ? ~0ull : ((1ull << left) - 1ull);
                }
            }
            CND_CUDA_TRY(cudaMemcpyAsync(d_valid, valid.data(), sizeof(uint64_t) * B, cudaMemcpyHostToDevice, st));
            CND_CUDA_TRY(cudaMemsetAsync(P.vis, 0, sizeof(uint64_t) * nB, st));
            if (model == 1) CND_CUDA_TRY(cudaMemsetAsync(P.acc, 0, sizeof(uint32_t) * nB * 64, st));
            P.g_base = (uint64_t)(o.first_trial + 64 * w0) >> 2;

            // step 0: seeds
            int cur = 0;
            CND_CUDA_TRY(cudaMemsetAsync(fr[cur].cnt, 0, 2 * sizeof(int32_t), st));
            P.out = fr[cur];
            P.stamp = stamp++;
            P.level = 0;
            if (n_seeds > 0) {
                k_seed_select<<<std::max(1, std::min((n_seeds + 255) / 256, max_blocks)), 256, 0, st>>>(P, d_seeds,
                                                                                                    n_seeds, d_bad);
                CND_CUDA_TRY(cudaGetLastError());
                CND_CUDA_TRY(launch(kernel_ptr(K_FIN_SEED, shp), blocks_for(32 / shp.lpe, n_seeds, max_blocks), st, P));
            }
            for (int L = 0;; ++L) {
                CND_CUDA_TRY(cudaMemcpyAsync(hcnt, fr[cur].cnt, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                CND_CUDA_TRY(cudaStreamSynchronize(st));
                const int32_t slots = hcnt[0], items = hcnt[1];
                if (slots == 0) break;
                if (o.max_levels > 0 && L >= o.max_levels) {
                    limit_hit = true;
                    break;
                }
                if (items == 0) break;
                if (o.timeout_s > 0) {
                    const double el =
                        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                    if (el > o.timeout_s) {
                        set_error("%s: timed out after %.3f s", fn, el);
                        cudaStreamSynchronize(st);
                        return CND_ETIMEOUT;
                    }
                }
                const int nxt = cur ^ 1;
                CND_CUDA_TRY(cudaMemsetAsync(fr[nxt].cnt, 0, 2 * sizeof(int32_t), st));
                P.in = fr[cur];
                P.out = fr[nxt];
                P.stamp = stamp++;
                P.level = L + 1;
                const int pb = blocks_for(1, items, max_blocks);
                if (model == 0) {
                    CND_CUDA_TRY(launch(kernel_ptr(K_IC_PUSH, shp), pb, st, P));
                    CND_CUDA_TRY(launch(kernel_ptr(K_FIN_IC, shp), max_blocks, st, P));
                } else {
                    CND_CUDA_TRY(cudaMemsetAsync(fr[2].cnt, 0, 2 * sizeof(int32_t), st));
                    P.tmp = fr[2];
                    CND_CUDA_TRY(launch(kernel_ptr(K_LT_PUSH, shp), pb, st, P));
                    CND_CUDA_TRY(launch(kernel_ptr(K_LT_FIN, shp), max_blocks, st, P));
                }
                cur = nxt;
            }
            // outputs of this pass
            {
                const int npb = 4096;
                dim3 grid((unsigned)((nw_here + 7) / 8), (unsigned)((n + npb - 1) / npb));
                k_spread<<<grid, 256, 0, st>>>(P.vis, n, B, (int)nw_here, npb, d_spread + w0 * 64);
                CND_CUDA_TRY(cudaGetLastError());
                void *args[] = {&P.vis, (void *)&n, (void *)&B, (void *)&G.row_ptr, &d_count, &d_checks};
                const int cb = blocks_for(32 / shp.lpe, n, max_blocks);
                CND_CUDA_TRY(cudaLaunchKernel(counts_ptr(shp.lpe), dim3(cb), dim3(256), args, 0, st));
            }
        }
    }

    // ---- results
    int32_t hbad = 0;
    CND_CUDA_TRY(cudaMemcpyAsync(&hbad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    std::vector<unsigned long long> hlc((size_t)std::max(lc_len, 1));
    unsigned long long hchecks = 0;
    if (dev) {
        if (spread_out && n_trials)
            CND_CUDA_TRY(cudaMemcpyAsync(spread_out, d_spread, sizeof(int32_t) * n_trials, cudaMemcpyDeviceToDevice, st));
        if (o.edge_checks_out)
            CND_CUDA_TRY(cudaMemcpyAsync(o.edge_checks_out, d_checks, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        if (lc_len)
            CND_CUDA_TRY(cudaMemcpyAsync(o.level_counts_out, d_lc, sizeof(int64_t) * lc_len, cudaMemcpyDeviceToDevice, st));
    } else {
        if (spread_out && n_trials)
            CND_CUDA_TRY(cudaMemcpyAsync(spread_out, d_spread, sizeof(int32_t) * n_trials, cudaMemcpyDeviceToHost, st));
        if (count_out) CND_CUDA_TRY(cudaMemcpyAsync(count_out, d_count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
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

}  // extern "C"
