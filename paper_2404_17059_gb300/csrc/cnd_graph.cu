// Graph ingest (CSR upload, IC probability -> threshold, LT weights, in-CSR),
// option defaults, error strings and the device Philox check entry point.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "cnd_common.cuh"

namespace cnd {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// IC probability -> fixed-point threshold (floor(p * 2^32), p == 1 -> always).
// p * 2^32 is exact in fp32 (a power-of-two scaling of a value below 1 stays
// below 2^32), and the float -> uint conversion truncates, i.e. floors.
__global__ void k_build_ic_edges(int32_t m, const int32_t *__restrict__ col, const float *__restrict__ p,
                                 uint2 *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const float x = p[e];
        const uint32_t thr = (x == 1.0f) ? kAlways : __float2uint_rz(x * 4294967296.0f);
        out[e] = make_uint2((uint32_t)col[e], thr);
    }
}

__global__ void k_build_lt_edges(int32_t m, const int32_t *__restrict__ col, const uint32_t *__restrict__ w,
                                 uint2 *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = make_uint2((uint32_t)col[e], w[e]);
}

// Counting-form LT edges: {col, tag}; tag = (first plane of the target << 5) | its plane count,
// or 0 for an edge of zero weight (it adds nothing, so the push skips it).
__global__ void k_build_lt_cnt_edges(int32_t m, const int32_t *__restrict__ col, const uint32_t *__restrict__ w,
                                     const int32_t *__restrict__ cnt_off, uint2 *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = col[e];
        const uint32_t L = (uint32_t)(cnt_off[v + 1] - cnt_off[v]);
        out[e] = make_uint2((uint32_t)v, w[e] ? (((uint32_t)cnt_off[v] << 5) | L) : 0u);
    }
}

// in_edge[k] = {src, edge id, IC threshold, LT weight} for the k-th in-edge.
__global__ void k_build_in_edges(int32_t m, const int32_t *__restrict__ in_src, const int32_t *__restrict__ in_eid,
                                 const uint2 *__restrict__ ic, const uint2 *__restrict__ lt, uint4 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = in_eid[k];
        out[k] = make_uint4((uint32_t)in_src[k], (uint32_t)e, ic ? ic[e].y : 0u, lt ? lt[e].y : 0u);
    }
}

__global__ void k_philox(uint32_t k0, uint32_t k1, const uint4 *__restrict__ ctr, int64_t count, uint4 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 c = ctr[i];
        const U4 r = philox4x32_10(c.x, c.y, c.z, c.w, k0, k1);
        out[i] = make_uint4(r.x, r.y, r.z, r.w);
    }
}

// Philox throughput probe: every thread computes `iters` blocks in registers, in two independent
// chains (each block's counter taken from the previous block's output), with the engine's own
// Philox4x32-10 (precomputed round keys, as the expansion kernels use it); one word per thread is
// stored so that nothing is optimised away.
__global__ void __launch_bounds__(256) k_philox_rate(RoundKeys rk, int32_t iters, uint32_t *__restrict__ sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    U4 a{t, 0u, 0u, 0u}, b{t, 1u, 0u, 0u};
    for (int32_t i = 0; i < iters; ++i) {
        a = philox4x32_10(a.x, a.y ^ (uint32_t)i, a.z, a.w, rk);
        b = philox4x32_10(b.x, b.y ^ (uint32_t)i, b.z, b.w, rk);
    }
    sink[t] = a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
}

// Random 8-byte accesses over a region of 2^k words (mask = 2^k - 1): each thread
// follows one chain, the next address derived from the value the previous access
// returned (a splitmix64 step, Steele, Lea and Flood 2014), so every access waits
// for the one before it, as the expansion kernels' do.  OP 0: ld.global.cg read;
// OP 1: atomic XOR with return.
template <int OP>
__global__ void __launch_bounds__(256) k_random_rate(unsigned long long *__restrict__ region, uint64_t mask,
                                                     int32_t iters, uint64_t *__restrict__ sink) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t x = t;
    for (int32_t i = 0; i < iters; ++i) {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const uint64_t r = OP == 0 ? (uint64_t)__ldcg(region + (z & mask)) : (uint64_t)atomicXor(region + (z & mask), 1ull);
        x += r;
    }
    sink[t] = x;
}

static void free_dev(cnd_graph_dev &d) {
    cudaFree(d.row_ptr);
    cudaFree(d.ic_edge);
    cudaFree(d.lt_edge);
    cudaFree(d.in_row_ptr);
    cudaFree(d.in_edge);
    cudaFree(d.lt_cnt_edge);
    cudaFree(d.lt_cnt_off);
    cudaFree(d.lt_unit_w);
    d = cnd_graph_dev{};
}

}  // namespace cnd

using namespace cnd;

extern "C" {

const char *cnd_last_error(void) { return g_err; }

void cnd_sim_opts_init(cnd_sim_opts *o) {
    if (o) memset(o, 0, sizeof(*o));
}

cnd_status cnd_lt_weights_wc(int32_t n, int32_t m, const int32_t *col, uint32_t *w_out) {
    clear_error();
    if (n <= 0 || m < 0 || (m > 0 && (!col || !w_out))) {
        set_error("cnd_lt_weights_wc: bad arguments");
        return CND_EINVAL;
    }
    std::vector<int64_t> indeg((size_t)n, 0);
    for (int64_t e = 0; e < m; ++e) {
        if (col[e] < 0 || col[e] >= n) {
            set_error("cnd_lt_weights_wc: col[%lld] out of range", (long long)e);
            return CND_EINVAL;
        }
        indeg[col[e]]++;
    }
    for (int64_t e = 0; e < m; ++e) w_out[e] = (uint32_t)(0xFFFFFFFFull / (uint64_t)indeg[col[e]]);
    return CND_OK;
}

cnd_status cnd_graph_create(int32_t n, int32_t m, const int32_t *row_ptr, const int32_t *col, const float *ic_prob,
                            const uint32_t *lt_weight_fx, cnd_graph **out) {
    clear_error();
    if (!out) {
        set_error("cnd_graph_create: out is NULL");
        return CND_EINVAL;
    }
    *out = nullptr;
    // ---- host-side validation: nothing touches the device before the input is known good
    if (n <= 0 || m < 0 || !row_ptr || (m > 0 && !col)) {
        set_error("cnd_graph_create: need n > 0, m >= 0, row_ptr and col");
        return CND_EINVAL;
    }
    if (row_ptr[0] != 0 || row_ptr[n] != m) {
        set_error("cnd_graph_create: row_ptr[0] must be 0 and row_ptr[n] must equal m");
        return CND_EINVAL;
    }
    int32_t max_deg = 0;
    for (int32_t u = 0; u < n; ++u) {
        const int32_t d = row_ptr[u + 1] - row_ptr[u];
        if (d < 0) {
            set_error("cnd_graph_create: row_ptr decreases at node %d", u);
            return CND_EINVAL;
        }
        if (d > max_deg) max_deg = d;
    }
    std::vector<int64_t> indeg((size_t)n, 0);
    for (int32_t e = 0; e < m; ++e) {
        if (col[e] < 0 || col[e] >= n) {
            set_error("cnd_graph_create: col[%d] = %d out of range", e, col[e]);
            return CND_EINVAL;
        }
        indeg[col[e]]++;
    }
    if (ic_prob) {
        for (int32_t e = 0; e < m; ++e) {
            const float p = ic_prob[e];
            if (!(p >= 0.0f && p <= 1.0f)) {
                set_error("cnd_graph_create: ic_prob[%d] = %g is not in [0, 1]", e, (double)p);
                return CND_EINVAL;
            }
        }
    }
    // LT counting form: possible when, at every node, the in-edges of non-zero weight all carry
    // the same weight w_v.  Then the active in-weight of v in a trial is k * w_v for k active
    // in-neighbours over such edges, and k * w_v > theta  <=>  k > floor(theta / w_v): a count
    // of at most k_v <= 2^L_v - 1 replaces the 32-bit sum.
    std::vector<int32_t> cnt_off;
    std::vector<uint32_t> unit_w;
    int64_t planes = 0;
    if (lt_weight_fx) {
        std::vector<uint64_t> insum((size_t)n, 0);
        for (int32_t e = 0; e < m; ++e) insum[col[e]] += lt_weight_fx[e];
        for (int32_t v = 0; v < n; ++v)
            if (insum[v] > 0xFFFFFFFFull) {
                set_error("cnd_graph_create: LT in-weights of node %d sum to %llu > 2^32-1", v,
                          (unsigned long long)insum[v]);
                return CND_EOVERFLOW;
            }
        unit_w.assign((size_t)n, 0u);
        std::vector<int64_t> k((size_t)n, 0);
        bool equal = true;
        for (int32_t e = 0; e < m && equal; ++e) {
            const uint32_t x = lt_weight_fx[e];
            if (x == 0u) continue;
            const int32_t v = col[e];
            if (unit_w[v] == 0u) unit_w[v] = x;
            equal = unit_w[v] == x;
            k[v]++;
        }
        if (equal) {
            cnt_off.assign((size_t)n + 1, 0);
            for (int32_t v = 0; v < n; ++v) {
                int32_t L = 0;
                while (L < 32 && (k[v] >> L) != 0) ++L;  // bits of k_v: 2^L - 1 >= k_v
                planes += L;
                // the edge tag holds the first plane in 27 bits
                if (planes >= ((int64_t)1 << 27)) break;
                cnt_off[v + 1] = (int32_t)planes;
            }
            if (planes >= ((int64_t)1 << 27)) {
                cnt_off.clear();
                planes = 0;
            }
        }
    }
    // ---- in-CSR permutation (counting sort by target, stable in edge id)
    std::vector<int32_t> in_row_ptr((size_t)n + 1, 0);
    for (int32_t v = 0; v < n; ++v) in_row_ptr[v + 1] = in_row_ptr[v] + (int32_t)indeg[v];
    std::vector<int32_t> in_src((size_t)(m > 0 ? m : 1)), in_eid((size_t)(m > 0 ? m : 1));
    {
        std::vector<int32_t> cursor(in_row_ptr.begin(), in_row_ptr.end() - 1);
        for (int32_t u = 0; u < n; ++u)
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                const int32_t k = cursor[col[e]]++;
                in_src[k] = u;
                in_eid[k] = e;
            }
    }

    cnd_graph *g = new (std::nothrow) cnd_graph();
    if (!g) {
        set_error("cnd_graph_create: host allocation failed");
        return CND_ENOMEM;
    }
    cnd_graph_dev &d = g->d;
    d.n = n;
    d.m = m;
    d.max_out_degree = max_deg;
    int32_t *d_col = nullptr, *d_tmp_a = nullptr, *d_tmp_b = nullptr;
    float *d_p = nullptr;
    uint32_t *d_w = nullptr;
    cnd_status st = CND_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        set_error("cnd_graph_create: %s: %s", what, cudaGetErrorString(e));
        st = (e == cudaErrorMemoryAllocation) ? CND_ENOMEM : CND_ECUDA;
    };
    do {
        cudaError_t e;
        if ((e = cudaGetDevice(&d.device)) != cudaSuccess) { fail(e, "cudaGetDevice"); break; }
        if ((e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, d.device)) != cudaSuccess) {
            fail(e, "attribute");
            break;
        }
        const size_t mb = (size_t)(m > 0 ? m : 1);
        if ((e = cudaMalloc(&d.row_ptr, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) { fail(e, "alloc row_ptr"); break; }
        if ((e = cudaMalloc(&d.in_row_ptr, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) { fail(e, "alloc in_row_ptr"); break; }
        if ((e = cudaMalloc(&d_col, sizeof(int32_t) * mb)) != cudaSuccess) { fail(e, "alloc col"); break; }
        if ((e = cudaMemcpy(d.row_ptr, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy row_ptr"); break; }
        if ((e = cudaMemcpy(d.in_row_ptr, in_row_ptr.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy in_row_ptr"); break; }
        if (m > 0 && (e = cudaMemcpy(d_col, col, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy col"); break; }
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>(((int64_t)m + threads - 1) / threads + 1, (int64_t)d.num_sms * 8);
        if (ic_prob) {
            if ((e = cudaMalloc(&d.ic_edge, sizeof(uint2) * mb)) != cudaSuccess) { fail(e, "alloc ic_edge"); break; }
            if ((e = cudaMalloc(&d_p, sizeof(float) * mb)) != cudaSuccess) { fail(e, "alloc p"); break; }
            if (m > 0 && (e = cudaMemcpy(d_p, ic_prob, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy p"); break; }
            k_build_ic_edges<<<blocks, threads>>>(m, d_col, d_p, d.ic_edge);
        }
        if (lt_weight_fx) {
            if ((e = cudaMalloc(&d.lt_edge, sizeof(uint2) * mb)) != cudaSuccess) { fail(e, "alloc lt_edge"); break; }
            if ((e = cudaMalloc(&d_w, sizeof(uint32_t) * mb)) != cudaSuccess) { fail(e, "alloc w"); break; }
            if (m > 0 && (e = cudaMemcpy(d_w, lt_weight_fx, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy w"); break; }
            k_build_lt_edges<<<blocks, threads>>>(m, d_col, d_w, d.lt_edge);
            if (!cnt_off.empty()) {
                if ((e = cudaMalloc(&d.lt_cnt_edge, sizeof(uint2) * mb)) != cudaSuccess) { fail(e, "alloc lt_cnt_edge"); break; }
                if ((e = cudaMalloc(&d.lt_cnt_off, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) { fail(e, "alloc lt_cnt_off"); break; }
                if ((e = cudaMalloc(&d.lt_unit_w, sizeof(uint32_t) * (size_t)n)) != cudaSuccess) { fail(e, "alloc lt_unit_w"); break; }
                if ((e = cudaMemcpy(d.lt_cnt_off, cnt_off.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy lt_cnt_off"); break; }
                if ((e = cudaMemcpy(d.lt_unit_w, unit_w.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy lt_unit_w"); break; }
                k_build_lt_cnt_edges<<<blocks, threads>>>(m, d_col, d_w, d.lt_cnt_off, d.lt_cnt_edge);
                d.lt_planes = planes;
            }
        }
        if ((e = cudaMalloc(&d.in_edge, sizeof(uint4) * mb)) != cudaSuccess) { fail(e, "alloc in_edge"); break; }
        if ((e = cudaMalloc(&d_tmp_a, sizeof(int32_t) * mb)) != cudaSuccess) { fail(e, "alloc tmp"); break; }
        if ((e = cudaMalloc(&d_tmp_b, sizeof(int32_t) * mb)) != cudaSuccess) { fail(e, "alloc tmp"); break; }
        if (m > 0) {
            if ((e = cudaMemcpy(d_tmp_a, in_src.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy in_src"); break; }
            if ((e = cudaMemcpy(d_tmp_b, in_eid.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy in_eid"); break; }
            k_build_in_edges<<<blocks, threads>>>(m, d_tmp_a, d_tmp_b, d.ic_edge, d.lt_edge, d.in_edge);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "launch"); break; }
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) { fail(e, "sync"); break; }
    } while (0);
    cudaFree(d_col);
    cudaFree(d_p);
    cudaFree(d_w);
    cudaFree(d_tmp_a);
    cudaFree(d_tmp_b);
    if (st != CND_OK) {
        free_dev(d);
        delete g;
        return st;
    }
    *out = g;
    return CND_OK;
}

void cnd_graph_destroy(cnd_graph *g) {
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->d.device);
    free_dev(g->d);
    cudaSetDevice(prev);
    delete g;
}

cnd_status cnd_graph_info(const cnd_graph *g, int32_t *n, int32_t *m, int32_t *has_ic, int32_t *has_lt) {
    clear_error();
    if (!g) {
        set_error("cnd_graph_info: graph is NULL");
        return CND_EINVAL;
    }
    if (n) *n = g->d.n;
    if (m) *m = g->d.m;
    if (has_ic) *has_ic = g->d.ic_edge != nullptr;
    if (has_lt) *has_lt = g->d.lt_edge != nullptr;
    return CND_OK;
}

cnd_status cnd_philox4x32_10(uint64_t rng_seed, const uint32_t *ctr, int64_t count, uint32_t *out) {
    clear_error();
    if (count < 0 || (count > 0 && (!ctr || !out))) {
        set_error("cnd_philox4x32_10: bad arguments");
        return CND_EINVAL;
    }
    if (count == 0) return CND_OK;
    uint4 *dc = nullptr, *dout = nullptr;
    cnd_status st = CND_OK;
    do {
        cudaError_t e;
        if ((e = cudaMalloc(&dc, sizeof(uint4) * count)) != cudaSuccess ||
            (e = cudaMalloc(&dout, sizeof(uint4) * count)) != cudaSuccess ||
            (e = cudaMemcpy(dc, ctr, sizeof(uint4) * count, cudaMemcpyHostToDevice)) != cudaSuccess) {
            set_error("cnd_philox4x32_10: %s", cudaGetErrorString(e));
            st = CND_ECUDA;
            break;
        }
        const int blocks = (int)std::min<int64_t>((count + 255) / 256, 4096);
        k_philox<<<blocks, 256>>>((uint32_t)rng_seed, (uint32_t)(rng_seed >> 32), dc, count, dout);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpy(out, dout, sizeof(uint4) * count, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            set_error("cnd_philox4x32_10: %s", cudaGetErrorString(e));
            st = CND_ECUDA;
        }
    } while (0);
    cudaFree(dc);
    cudaFree(dout);
    return st;
}

cnd_status cnd_philox_rate(int32_t iters, void *stream, double *blocks_per_s_out, double *ms_out) {
    clear_error();
    if (iters <= 0 || !blocks_per_s_out) {
        set_error("cnd_philox_rate: bad arguments");
        return CND_EINVAL;
    }
    int dev = 0, sms = 0, per_sm = 0;
    CND_CUDA_TRY(cudaGetDevice(&dev));
    CND_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CND_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_philox_rate, 256, 0));
    const int blocks = sms * std::max(per_sm, 1);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *sink = nullptr;
    CND_CUDA_TRY(cudaMalloc(&sink, sizeof(uint32_t) * 256 * (size_t)blocks));
    const RoundKeys rk = round_keys(0x0123456789ABCDEFull);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cnd_status rs = CND_OK;
    do {
        cudaError_t e;
        if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
            set_error("cnd_philox_rate: %s", cudaGetErrorString(e));
            rs = CND_ECUDA;
            break;
        }
        k_philox_rate<<<blocks, 256, 0, st>>>(rk, std::min(iters, 16), sink);  // warm-up
        cudaEventRecord(e0, st);
        k_philox_rate<<<blocks, 256, 0, st>>>(rk, iters, sink);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            set_error("cnd_philox_rate: %s", cudaGetErrorString(e));
            rs = CND_ECUDA;
            break;
        }
        *blocks_per_s_out = 2.0 * 256.0 * (double)blocks * (double)iters / (ms * 1e-3);
        if (ms_out) *ms_out = ms;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rs;
}

cnd_status cnd_random_access_rate(int64_t region_bytes, int32_t op, int32_t iters, void *stream,
                                  double *ops_per_s_out, double *ms_out) {
    clear_error();
    if (region_bytes < 64 || op < 0 || op > 1 || iters <= 0 || !ops_per_s_out) {
        set_error("cnd_random_access_rate: bad arguments");
        return CND_EINVAL;
    }
    uint64_t words = 8;
    while (words * 2 <= (uint64_t)region_bytes / 8) words *= 2;
    const void *fn = op == 0 ? (const void *)k_random_rate<0> : (const void *)k_random_rate<1>;
    int dev = 0, sms = 0, per_sm = 0;
    CND_CUDA_TRY(cudaGetDevice(&dev));
    CND_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CND_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0));
    const int blocks = sms * std::max(per_sm, 1);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *region = nullptr;
    uint64_t *sink = nullptr;
    if (cudaMalloc(&region, words * 8) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(uint64_t) * 256 * (size_t)blocks) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(region);
        set_error("cnd_random_access_rate: cannot allocate %llu bytes", (unsigned long long)(words * 8));
        return CND_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cnd_status rs = CND_OK;
    do {
        cudaError_t e;
        if ((e = cudaMemsetAsync(region, 0, words * 8, st)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
            (e = cudaEventCreate(&e1)) != cudaSuccess) {
            set_error("cnd_random_access_rate: %s", cudaGetErrorString(e));
            rs = CND_ECUDA;
            break;
        }
        const uint64_t mask = words - 1;
        if (op == 0) k_random_rate<0><<<blocks, 256, 0, st>>>(region, mask, std::min(iters, 16), sink);  // warm-up
        else k_random_rate<1><<<blocks, 256, 0, st>>>(region, mask, std::min(iters, 16), sink);
        cudaEventRecord(e0, st);
        if (op == 0) k_random_rate<0><<<blocks, 256, 0, st>>>(region, mask, iters, sink);
        else k_random_rate<1><<<blocks, 256, 0, st>>>(region, mask, iters, sink);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            set_error("cnd_random_access_rate: %s", cudaGetErrorString(e));
            rs = CND_ECUDA;
            break;
        }
        *ops_per_s_out = 256.0 * (double)blocks * (double)iters / (ms * 1e-3);
        if (ms_out) *ms_out = ms;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(region);
    cudaFree(sink);
    return rs;
}

}  // extern "C"
