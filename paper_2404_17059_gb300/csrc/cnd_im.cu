// Influence maximisation by lazy greedy (CELF) over the batched engine
// (Sec. 2 "Influence Maximization"; the paper runs CELF in Sec. 4).
//
// A client of the public batched entry points: each re-evaluation step packs
// the stale candidates' sets S + v into one cnd_*_simulate_batch call on the
// device (common random numbers: every item uses the same key and trial
// range), a small kernel sums every item's per-trial spreads, and only those
// sums come back to the host, where the lazy-greedy queue lives.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <queue>
#include <vector>

#include "cnd_common.cuh"

namespace cnd {

// sums[i] = sum of spread[i * T .. (i + 1) * T)
__global__ void k_item_sums(const int32_t *__restrict__ spread, int32_t n_items, int64_t T,
                            long long *__restrict__ sums) {
    __shared__ long long part[32];
    for (int32_t i = blockIdx.x; i < n_items; i += gridDim.x) {
        long long s = 0;
        const int32_t *row = spread + (int64_t)i * T;
        for (int64_t t = threadIdx.x; t < T; t += blockDim.x) s += row[t];
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
            for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) sums[i] = s;
        }
        __syncthreads();
    }
}

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

struct DeviceGuard {
    int prev = -1;
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct Entry {
    int64_t gain;
    int32_t node;
    int32_t round;  // round of the last evaluation
};

// priority: larger gain first, then lower node id
struct Lower {
    bool operator()(const Entry &a, const Entry &b) const {
        return a.gain != b.gain ? a.gain < b.gain : a.node > b.node;
    }
};

class Evaluator {
  public:
    Evaluator(int model, const cnd_graph *g, const cnd_im_opts &o, cudaStream_t st)
        : model_(model), g_(g), o_(o), st_(st) {}

    cnd_status init(int32_t k) {
        T_ = o_.n_trials;
        const int64_t cap_by_trials = std::max<int64_t>(1, ((int64_t)1 << 28) / T_);
        items_ = (int32_t)std::min<int64_t>(o_.max_items > 0 ? o_.max_items : 8192, cap_by_trials);
        CND_CUDA_TRY(cudaMalloc(&seeds_.p, sizeof(int32_t) * (size_t)items_ * (size_t)k));
        CND_CUDA_TRY(cudaMalloc(&spread_.p, sizeof(int32_t) * (size_t)items_ * (size_t)T_));
        CND_CUDA_TRY(cudaMalloc(&sums_.p, sizeof(long long) * ((size_t)items_ + 1)));
        trials_.assign((size_t)items_, (int32_t)T_);
        keys_.assign((size_t)items_, o_.rng_seed);
        cnd_sim_opts_init(&so_);
        if (o_.sim) so_ = *o_.sim;
        so_.device_ptrs = 1;
        so_.stream = st_;
        so_.level_counts_out = nullptr;
        so_.level_counts_len = 0;
        so_.stats = nullptr;
        so_.edge_checks_out = reinterpret_cast<int64_t *>(static_cast<long long *>(sums_.p) + items_);
        return CND_OK;
    }

    // F(S + v) for every v in nodes, in order
    cnd_status eval(const std::vector<int32_t> &S, const std::vector<int32_t> &nodes, std::vector<int64_t> &F) {
        F.resize(nodes.size());
        const size_t w = S.size() + 1;
        std::vector<int64_t> off;
        std::vector<int32_t> hs;
        std::vector<long long> hsums;
        for (size_t b = 0; b < nodes.size(); b += (size_t)items_) {
            const int32_t cnt = (int32_t)std::min<size_t>((size_t)items_, nodes.size() - b);
            off.resize((size_t)cnt + 1);
            hs.resize((size_t)cnt * w);
            for (int32_t i = 0; i < cnt; ++i) {
                off[i] = (int64_t)i * (int64_t)w;
                std::copy(S.begin(), S.end(), hs.begin() + (size_t)i * w);
                hs[(size_t)i * w + S.size()] = nodes[b + (size_t)i];
            }
            off[cnt] = (int64_t)cnt * (int64_t)w;
            CND_CUDA_TRY(cudaMemcpyAsync(seeds_.p, hs.data(), sizeof(int32_t) * hs.size(), cudaMemcpyHostToDevice, st_));
            const cnd_status s = model_ == 0
                ? cnd_ic_simulate_batch(g_, cnt, off.data(), static_cast<int32_t *>(seeds_.p), trials_.data(),
                                        keys_.data(), static_cast<int32_t *>(spread_.p), nullptr, &so_)
                : cnd_lt_simulate_batch(g_, cnt, off.data(), static_cast<int32_t *>(seeds_.p), trials_.data(),
                                        keys_.data(), static_cast<int32_t *>(spread_.p), nullptr, &so_);
            if (s != CND_OK) return s;
            const int blocks = std::min<int32_t>(cnt, 4 * std::max(1, g_->d.num_sms));
            k_item_sums<<<blocks, 256, 0, st_>>>(static_cast<int32_t *>(spread_.p), cnt, T_,
                                                 static_cast<long long *>(sums_.p));
            CND_CUDA_TRY(cudaGetLastError());
            hsums.resize((size_t)cnt + 1);
            CND_CUDA_TRY(cudaMemcpyAsync(hsums.data(), static_cast<long long *>(sums_.p), sizeof(long long) * cnt,
                                         cudaMemcpyDeviceToHost, st_));
            CND_CUDA_TRY(cudaMemcpyAsync(&hsums[cnt], static_cast<long long *>(sums_.p) + items_, sizeof(long long),
                                         cudaMemcpyDeviceToHost, st_));
            CND_CUDA_TRY(cudaStreamSynchronize(st_));
            for (int32_t i = 0; i < cnt; ++i) F[b + (size_t)i] = hsums[i];
            checks_ += hsums[cnt];
            evals_ += cnt;
        }
        return CND_OK;
    }

    int64_t evaluations() const { return evals_; }
    int64_t edge_checks() const { return checks_; }

  private:
    int model_;
    const cnd_graph *g_;
    const cnd_im_opts &o_;
    cudaStream_t st_;
    int64_t T_ = 0;
    int32_t items_ = 0;
    DevBuf seeds_, spread_, sums_;
    std::vector<int32_t> trials_;
    std::vector<uint64_t> keys_;
    cnd_sim_opts so_{};
    int64_t evals_ = 0, checks_ = 0;
};

cnd_status candidates_of(const cnd_graph_dev &G, const cnd_im_opts *o, const char *fn, std::vector<int32_t> &cand);

cnd_status celf(int model, const cnd_graph *g, const cnd_im_opts *o, int32_t *seeds_out, int64_t *f_out) {
    const char *fn = model == 0 ? "cnd_ic_im_celf" : "cnd_lt_im_celf";
    clear_error();
    if (!g || !o || !seeds_out) {
        set_error("%s: graph, options and seeds_out are required", fn);
        return CND_EINVAL;
    }
    const cnd_graph_dev &G = g->d;
    if ((model == 0 ? G.ic_edge : G.lt_edge) == nullptr && G.m > 0) {
        set_error("%s: graph was created without %s", fn, model == 0 ? "IC probabilities" : "LT weights");
        return CND_EINVAL;
    }
    if (o->n_trials < 1 || o->n_trials > INT32_MAX) {
        set_error("%s: n_trials must be in 1 .. 2^31-1", fn);
        return CND_EINVAL;
    }
    std::vector<int32_t> cand;
    {
        const cnd_status cs = candidates_of(G, o, fn, cand);
        if (cs != CND_OK) return cs;
    }
    if (o->k < 1 || (size_t)o->k > cand.size()) {
        set_error("%s: k = %d must be in 1 .. number of candidates (%zu)", fn, (int)o->k, cand.size());
        return CND_EINVAL;
    }
    int dev = 0;
    DeviceGuard guard;
    CND_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != G.device) {
        CND_CUDA_TRY(cudaSetDevice(G.device));
        guard.prev = dev;
    }
    cudaStream_t st = static_cast<cudaStream_t>(o->stream);

    std::vector<int32_t> row_ptr((size_t)G.n + 1);
    CND_CUDA_TRY(cudaMemcpy(row_ptr.data(), G.row_ptr, sizeof(int32_t) * row_ptr.size(), cudaMemcpyDeviceToHost));

    Evaluator ev(model, g, *o, st);
    cnd_status s = ev.init(o->k);
    if (s != CND_OK) return s;
    const int32_t B = o->eval_batch > 0 ? o->eval_batch : 64;

    // round 0: F({v}) for all candidates; a node without out-edges spreads to itself alone
    std::vector<int32_t> S, todo;
    std::vector<int64_t> F;
    std::priority_queue<Entry, std::vector<Entry>, Lower> q;
    for (int32_t v : cand) {
        if (row_ptr[(size_t)v + 1] == row_ptr[(size_t)v])
            q.push({o->n_trials, v, 0});
        else
            todo.push_back(v);
    }
    s = ev.eval(S, todo, F);
    if (s != CND_OK) return s;
    for (size_t i = 0; i < todo.size(); ++i) q.push({F[i], todo[i], 0});

    int64_t fS = 0;
    for (int32_t j = 0; j < o->k; ++j) {
        while (q.top().round != j) {
            todo.clear();
            std::vector<Entry> popped;
            while (!q.empty() && q.top().round != j && (int32_t)todo.size() < B) {
                popped.push_back(q.top());
                todo.push_back(q.top().node);
                q.pop();
            }
            s = ev.eval(S, todo, F);
            if (s != CND_OK) return s;
            for (size_t i = 0; i < todo.size(); ++i) q.push({F[i] - fS, todo[i], j});
        }
        const Entry e = q.top();
        q.pop();
        S.push_back(e.node);
        fS += e.gain;
        seeds_out[j] = e.node;
        if (f_out) f_out[j] = fS;
    }
    if (o->evaluations_out) *o->evaluations_out = ev.evaluations();
    if (o->edge_checks_out) *o->edge_checks_out = ev.edge_checks();
    return CND_OK;
}

cnd_status candidates_of(const cnd_graph_dev &G, const cnd_im_opts *o, const char *fn, std::vector<int32_t> &cand) {
    std::vector<char> seen((size_t)G.n, 0);
    if (o->candidates) {
        if (o->n_candidates < 0) {
            set_error("%s: n_candidates < 0", fn);
            return CND_EINVAL;
        }
        cand.assign(o->candidates, o->candidates + o->n_candidates);
        for (int32_t v : cand) {
            if (v < 0 || v >= G.n || seen[(size_t)v]) {
                set_error("%s: candidate %d out of range or repeated", fn, (int)v);
                return CND_EINVAL;
            }
            seen[(size_t)v] = 1;
        }
    } else {
        cand.resize((size_t)G.n);
        std::iota(cand.begin(), cand.end(), 0);
    }
    return CND_OK;
}

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

// indices of the best `keep` entries by (value descending, node ascending)
std::vector<int32_t> top_by(const std::vector<int32_t> &nodes, const std::vector<double> &val, size_t keep) {
    std::vector<size_t> idx(nodes.size());
    std::iota(idx.begin(), idx.end(), 0);
    keep = std::min(keep, idx.size());
    auto better = [&](size_t a, size_t b) { return val[a] != val[b] ? val[a] > val[b] : nodes[a] < nodes[b]; };
    std::partial_sort(idx.begin(), idx.begin() + keep, idx.end(), better);
    std::vector<int32_t> out(keep);
    for (size_t i = 0; i < keep; ++i) out[i] = nodes[idx[i]];
    return out;
}

cnd_status screened(const cnd_graph *g, cnd_sur *sur, const cnd_im_opts *o, const cnd_screen_opts *so,
                    int32_t *seeds_out, int64_t *f_out) {
    const char *fn = "cnd_ic_im_screened";
    clear_error();
    if (!g || !o || !so || !seeds_out || (!sur && so->mode != 2)) {
        set_error("%s: graph, surrogate (modes 0, 1, 3), options and seeds_out are required", fn);
        return CND_EINVAL;
    }
    const cnd_graph_dev &G = g->d;
    if (!G.ic_edge && G.m > 0) {
        set_error("%s: graph was created without IC probabilities", fn);
        return CND_EINVAL;
    }
    if (o->n_trials < 1 || o->n_trials > INT32_MAX || so->n_exact < 1 ||
        (so->n_screen != 0 && so->n_screen < so->n_exact) || so->mode < 0 || so->mode > 3) {
        set_error("%s: need 1 <= n_trials <= 2^31-1, n_exact >= 1, n_screen 0 or >= n_exact, mode 0..3", fn);
        return CND_EINVAL;
    }
    std::vector<int32_t> cand;
    cnd_status s = candidates_of(G, o, fn, cand);
    if (s != CND_OK) return s;
    if (o->k < 1 || (size_t)o->k > cand.size()) {
        set_error("%s: k = %d must be in 1 .. number of candidates (%zu)", fn, (int)o->k, cand.size());
        return CND_EINVAL;
    }
    int dev = 0;
    DeviceGuard guard;
    CND_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != G.device) {
        CND_CUDA_TRY(cudaSetDevice(G.device));
        guard.prev = dev;
    }
    Evaluator ev(0, g, *o, static_cast<cudaStream_t>(o->stream));
    s = ev.init(o->k);
    if (s != CND_OK) return s;
    const size_t n_screen = (size_t)(so->n_screen > 0 ? so->n_screen : so->n_exact);
    const size_t n_exact = (size_t)so->n_exact;
    std::vector<char> is_cand((size_t)G.n, 0);
    for (int32_t v : cand) is_cand[(size_t)v] = 1;
    std::vector<int32_t> S, pool, one;
    std::vector<float> score((size_t)G.n), degree;
    if (so->mode == 2 || so->mode == 3) {
        std::vector<int32_t> rp((size_t)G.n + 1);
        CND_CUDA_TRY(cudaMemcpy(rp.data(), G.row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost));
        degree.resize((size_t)G.n);
        for (int32_t v = 0; v < G.n; ++v) degree[(size_t)v] = (float)(rp[(size_t)v + 1] - rp[(size_t)v]);
        if (so->mode == 2) score = degree;
    }
    std::vector<double> val, val2;
    std::vector<int64_t> F;
    double sur_ms = 0.0, sim_ms = 0.0;
    int64_t fS = 0;
    for (int32_t j = 0; j < o->k; ++j) {
        auto t0 = Clock::now();
        if (so->mode == 0 || so->mode == 3)
            s = cnd_sur_scores(sur, S.data(), (int32_t)S.size(), score.data());
        else if (so->mode == 1)
            s = cnd_sur_onehop(sur, S.data(), (int32_t)S.size(), score.data());
        if (s != CND_OK) return s;
        pool.clear();
        val.clear();
        for (int32_t v : cand)
            if (is_cand[(size_t)v]) {
                pool.push_back(v);
                val.push_back((double)score[(size_t)v]);
            }
        // without a network (mode 2) the first score alone picks the candidates to simulate; mode 3
        // takes them alternately from the network's ranking and the out-degree ranking
        std::vector<int32_t> keep;
        if (so->mode == 3) {
            val2.clear();
            for (int32_t v : pool) val2.push_back((double)degree[(size_t)v]);
            const std::vector<int32_t> a = top_by(pool, val, n_exact), b = top_by(pool, val2, n_exact);
            size_t ia = 0, ib = 0;
            while (keep.size() < std::min(n_exact, pool.size())) {
                const bool from_a = (keep.size() % 2 == 0 && ia < a.size()) || ib >= b.size();
                const int32_t c = from_a ? a[ia++] : b[ib++];
                if (std::find(keep.begin(), keep.end(), c) == keep.end()) keep.push_back(c);
            }
        } else {
            keep = top_by(pool, val, so->mode == 2 ? n_exact : n_screen);
        }
        if (keep.size() > n_exact) {
            val.assign(keep.size(), 0.0);
            for (size_t i = 0; i < keep.size(); ++i) {
                one = S;
                one.push_back(keep[i]);
                double pred = 0.0;
                s = cnd_sur_forward(sur, one.data(), (int32_t)one.size(), nullptr, &pred);
                if (s != CND_OK) return s;
                val[i] = pred;
            }
            keep = top_by(keep, val, n_exact);
        }
        sur_ms += ms_since(t0);
        t0 = Clock::now();
        s = ev.eval(S, keep, F);
        if (s != CND_OK) return s;
        sim_ms += ms_since(t0);
        size_t best = 0;
        for (size_t i = 1; i < keep.size(); ++i)
            if (F[i] > F[best] || (F[i] == F[best] && keep[i] < keep[best])) best = i;
        S.push_back(keep[best]);
        is_cand[(size_t)keep[best]] = 0;
        fS = F[best];
        seeds_out[j] = keep[best];
        if (f_out) f_out[j] = fS;
    }
    if (o->evaluations_out) *o->evaluations_out = ev.evaluations();
    if (o->edge_checks_out) *o->edge_checks_out = ev.edge_checks();
    if (so->sur_ms_out) *so->sur_ms_out = sur_ms;
    if (so->sim_ms_out) *so->sim_ms_out = sim_ms;
    return CND_OK;
}

}  // namespace
}  // namespace cnd

extern "C" {

cnd_status cnd_ic_im_screened(const cnd_graph *g, cnd_sur *s, const cnd_im_opts *o, const cnd_screen_opts *so,
                              int32_t *seeds_out, int64_t *f_out) {
    return cnd::screened(g, s, o, so, seeds_out, f_out);
}

void cnd_im_opts_init(cnd_im_opts *o) {
    if (!o) return;
    *o = cnd_im_opts{};
    o->n_trials = 1024;
    o->rng_seed = 1;
}

cnd_status cnd_ic_im_celf(const cnd_graph *g, const cnd_im_opts *o, int32_t *seeds_out, int64_t *f_out) {
    return cnd::celf(0, g, o, seeds_out, f_out);
}

cnd_status cnd_lt_im_celf(const cnd_graph *g, const cnd_im_opts *o, int32_t *seeds_out, int64_t *f_out) {
    return cnd::celf(1, g, o, seeds_out, f_out);
}

}  // extern "C"
