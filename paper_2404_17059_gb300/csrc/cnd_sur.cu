// Learned surrogate of IC activation frequencies: forward, backward, screening
// scores, Adam and the on-the-fly training loop (definition in include/cnd.h).
//
// Layout: activations are node-major rows (h: n x 64 bf16, 128 B per node;
// layer-1 inputs x, a^1: n x 16 bf16).  Each layer is two kernels:
//   k_spmm_in    a = A_q h over the in-CSR (warp per work item of <= 256
//                in-edges; a node with more in-edges is split over several
//                items, each writing its partial row, summed in item order
//                and rounded afterwards);
//   k_dense_fwd  the 64 x (2 DIN) dense map on the tensor cores
//                (mma.sync m16n8k16 bf16 -> fp32, a warp per 16-row tile) with
//                bias, relu and bf16 rounding fused; the last layer also
//                computes the head o = w_o . h^3 + b_o.
// Backward mirrors it: k_dense_bwd (mask, head, bias gradient, dX = e W on the
// tensor cores, e kept as A operand straight from the accumulator layout),
// k_dw (split-K dW = e^T [h | a] on the tensor cores) and k_spmm_out (the
// transpose aggregation over the out-CSR).  The seed-dependent channel of
// layer 1 (x_v[0] = s_v and a^1_v[0]) is patched in place from the seeds'
// out-edges; the static channels are built once.
// Every reduction runs in a fixed order (partial rows and per-block partial
// sums are added up in index order by a second kernel; the seed channel sums
// fixed-point integers), so results do not depend on scheduling.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "cnd_common.cuh"

namespace cnd {
namespace sur {

constexpr int H = 64;
constexpr int D0 = 16;
// parameter offsets of layer l = 0, 1, 2 (W_s, W_n, b)
__host__ __device__ constexpr int off_ws(int l) { return l == 0 ? 0 : (l == 1 ? 2112 : 10368); }
__host__ __device__ constexpr int off_wn(int l) { return l == 0 ? 1024 : (l == 1 ? 6208 : 14464); }
__host__ __device__ constexpr int off_b(int l) { return l == 0 ? 2048 : (l == 1 ? 10304 : 18560); }
constexpr int OFF_WO = 18624;
constexpr int OFF_BO = 18688;
constexpr int N_PARAMS = 18689;
constexpr int kItemEdges = 256;
constexpr float kQScale = 2.3283064365386963e-10f;  // 2^-32

static_assert(N_PARAMS == CND_SUR_N_PARAMS, "parameter count");

__device__ __forceinline__ float edge_q(uint32_t thr) { return __uint2float_rn(thr) * kQScale; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t u) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162 *>(&u);
    return __bfloat1622float2(v);
}

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// D += A B for one m16n8k16 tile (A row-major 16x16 bf16, B col-major 16x8 bf16, fp32 accumulators)
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// --------------------------------------------------------------------------- setup kernels
// x_v = [0, ln(1 + indeg), ln(1 + outdeg), 0...] (the seed channel is patched per call)
__global__ void k_features(int32_t n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ in_row_ptr,
                           __nv_bfloat16 *__restrict__ x) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float li = log1pf((float)(in_row_ptr[v + 1] - in_row_ptr[v]));
        const float lo = log1pf((float)(row_ptr[v + 1] - row_ptr[v]));
        uint4 *row = reinterpret_cast<uint4 *>(x + (size_t)v * D0);
        uint4 r0;
        r0.x = pack_bf16(0.0f, li);
        r0.y = pack_bf16(lo, 0.0f);
        r0.z = 0u;
        r0.w = 0u;
        row[0] = r0;
        row[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// compact in-edges {src, thr} from the graph's {src, eid, thr, w}
__global__ void k_in_compact(int32_t m, const uint4 *__restrict__ in_edge, uint2 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const uint4 e = in_edge[k];
        out[k] = make_uint2(e.x, e.z);
    }
}

// static channels of a^1 (channel 0, the seed channel, stays 0 here): a thread per node
__global__ void k_a1_static(int32_t n, const int32_t *__restrict__ in_row_ptr, const uint2 *__restrict__ in_c,
                            const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ a1) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        float s1 = 0.0f, s2 = 0.0f;
        for (int32_t k = in_row_ptr[v]; k < in_row_ptr[v + 1]; ++k) {
            const uint2 e = in_c[k];
            const float q = edge_q(e.y);
            const float2 f = unpack_bf16(ld_u32(x + (size_t)e.x * D0));      // channels 0, 1
            const float2 f2 = unpack_bf16(ld_u32(x + (size_t)e.x * D0 + 2));  // channels 2, 3
            s1 += q * f.y;
            s2 += q * f2.x;
        }
        uint4 *row = reinterpret_cast<uint4 *>(a1 + (size_t)v * D0);
        uint4 r0;
        r0.x = pack_bf16(0.0f, s1);
        r0.y = pack_bf16(s2, 0.0f);
        r0.z = 0u;
        r0.w = 0u;
        row[0] = r0;
        row[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// fp32 masters -> bf16 operand layouts: wcat[l][o][i] = [W_s | W_n][o][i], wt[l][i][o] (its transpose)
__global__ void k_pack_weights(const float *__restrict__ p, __nv_bfloat16 *__restrict__ wcat,
                               __nv_bfloat16 *__restrict__ wt) {
    // layer 0: 64 x 32, layers 1, 2: 64 x 128; offsets in elements
    const int base[3] = {0, 64 * 32, 64 * 32 + 64 * 128};
    const int tot = 64 * 32 + 2 * 64 * 128;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
        const int l = idx < base[1] ? 0 : (idx < base[2] ? 1 : 2);
        const int din = l == 0 ? D0 : H;
        const int k = idx - base[l];
        const int o = k / (2 * din), i = k % (2 * din);
        const float w = i < din ? p[off_ws(l) + o * din + i] : p[off_wn(l) + o * din + (i - din)];
        const __nv_bfloat16 b = __float2bfloat16_rn(w);
        wcat[base[l] + o * 2 * din + i] = b;
        wt[base[l] + i * H + o] = b;
    }
}

// --------------------------------------------------------------------------- seed channel
// phase 1: x_u[0] = 1 for seeds; acc0[w] += q * 2^32 over the seeds' out-edges.  q = fp32(thr) 2^-32
// with fp32(thr) an integer below 2^33, so the sums are exact integers: their order does not matter.
__global__ void k_seed_scatter(const int32_t *__restrict__ seeds, int32_t ns, const int32_t *__restrict__ row_ptr,
                               const uint2 *__restrict__ ic_edge, __nv_bfloat16 *__restrict__ x,
                               unsigned long long *__restrict__ acc0) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < ns; i += nwarps) {
        const int32_t u = seeds[i];
        if (lane == 0) x[(size_t)u * D0] = __float2bfloat16_rn(1.0f);
        for (int32_t e = row_ptr[u] + lane; e < row_ptr[u + 1]; e += 32) {
            const uint2 ed = ic_edge[e];
            atomicAdd(acc0 + ed.x, (unsigned long long)__uint2float_rn(ed.y));
        }
    }
}

// phase 2: a^1_w[0] = bf16(acc0[w] 2^-32) (exact in fp64, one rounding) for the seeds' out-neighbours;
// mode 1 clears everything phase 1 set
template <int CLEAR>
__global__ void k_seed_finish(const int32_t *__restrict__ seeds, int32_t ns, const int32_t *__restrict__ row_ptr,
                              const uint2 *__restrict__ ic_edge, __nv_bfloat16 *__restrict__ x,
                              __nv_bfloat16 *__restrict__ a1, unsigned long long *__restrict__ acc0) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < ns; i += nwarps) {
        const int32_t u = seeds[i];
        if (CLEAR && lane == 0) x[(size_t)u * D0] = __float2bfloat16_rn(0.0f);
        for (int32_t e = row_ptr[u] + lane; e < row_ptr[u + 1]; e += 32) {
            const uint32_t w = ic_edge[e].x;
            if (CLEAR) {
                a1[(size_t)w * D0] = __float2bfloat16_rn(0.0f);
                acc0[w] = 0ull;
            } else {
                a1[(size_t)w * D0] = __double2bfloat16((double)acc0[w] * 2.3283064365386963e-10);
            }
        }
    }
}

// --------------------------------------------------------------------------- aggregation
struct Item {
    int32_t node, begin, end, slot;  // slot >= 0: this item's partial row of a split node (scratch row index)
};

// a[v] = bf16(sum over in-edges of q h[src]) for 64-wide bf16 rows; a warp per item.  The warp
// gathers 4 rows per load instruction (8 lanes x 16 B per 128-byte row), 16 rows in flight, and
// folds the 4 partial sums of each feature at the end.
__global__ void __launch_bounds__(256) k_spmm_in(int32_t n_items, const Item *__restrict__ items,
                                                 const uint2 *__restrict__ in_c, const __nv_bfloat16 *__restrict__ h,
                                                 __nv_bfloat16 *__restrict__ a, float *__restrict__ scratch) {
    const int lane = threadIdx.x & 31;
    const int sub = lane >> 3;       // which of 4 edges
    const int f8 = (lane & 7) * 8;   // first of this lane's 8 features
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int it = warp; it < n_items; it += nwarps) {
        const Item item = items[it];
        float acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.0f;
        for (int32_t b = item.begin; b < item.end; b += 32) {
            const int cnt = min(32, item.end - b);
            uint2 my = make_uint2(0u, 0u);
            if (lane < cnt) my = in_c[b + lane];
            const float myq = edge_q(my.y);
            for (int j = 0; j < cnt; j += 16) {
                // edges j + sub + 4 r, r = 0..3 (q = 0 past the end: row 0 read, nothing added)
                uint4 rr[4];
                float qq[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int e = j + sub + 4 * r;
                    const uint32_t u = __shfl_sync(0xffffffffu, my.x, e & 31);
                    const float q = __shfl_sync(0xffffffffu, myq, e & 31);
                    qq[r] = e < cnt ? q : 0.0f;
                    rr[r] = *reinterpret_cast<const uint4 *>(h + (size_t)(e < cnt ? u : 0u) * H + f8);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t w4[4] = {rr[r].x, rr[r].y, rr[r].z, rr[r].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 x = unpack_bf16(w4[i]);
                        acc[2 * i] += qq[r] * x.x;
                        acc[2 * i + 1] += qq[r] * x.y;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 8);
            acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 16);
        }
        if (lane < 8) {
            if (item.slot < 0) {
                uint4 o;
                o.x = pack_bf16(acc[0], acc[1]);
                o.y = pack_bf16(acc[2], acc[3]);
                o.z = pack_bf16(acc[4], acc[5]);
                o.w = pack_bf16(acc[6], acc[7]);
                *reinterpret_cast<uint4 *>(a + (size_t)item.node * H + f8) = o;
            } else {
                float4 *pr = reinterpret_cast<float4 *>(scratch + (size_t)item.slot * H + f8);
                pr[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                pr[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
            }
        }
    }
}

// rows of split nodes: add the partial rows of node i (slots first[i] .. first[i+1]-1) in order,
// round into a
__global__ void k_split_finish(int32_t n_split, const int32_t *__restrict__ split_node,
                               const int32_t *__restrict__ first, const float *__restrict__ scratch,
                               __nv_bfloat16 *__restrict__ a) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n_split; i += nwarps) {
        float2 f = make_float2(0.0f, 0.0f);
        for (int32_t j = first[i]; j < first[i + 1]; ++j) {
            const float2 x = reinterpret_cast<const float2 *>(scratch + (size_t)j * H)[lane];
            f.x += x.x;
            f.y += x.y;
        }
        *reinterpret_cast<uint32_t *>(a + (size_t)split_node[i] * H + 2 * lane) = pack_bf16(f.x, f.y);
    }
}

// out-rows of split nodes: dh[node i] += the partial rows of node i, in order
__global__ void k_split_out_finish(int32_t n_split, const int32_t *__restrict__ split_node,
                                   const int32_t *__restrict__ first, const float *__restrict__ scratch,
                                   float *__restrict__ dh) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n_split; i += nwarps) {
        float2 f = make_float2(0.0f, 0.0f);
        for (int32_t j = first[i]; j < first[i + 1]; ++j) {
            const float2 x = reinterpret_cast<const float2 *>(scratch + (size_t)j * H)[lane];
            f.x += x.x;
            f.y += x.y;
        }
        float2 *row = reinterpret_cast<float2 *>(dh + (size_t)split_node[i] * H) + lane;
        float2 v = *row;
        v.x += f.x;
        v.y += f.y;
        *row = v;
    }
}

// dh[u] += sum over out-edges (u -> w) of q da[w], 64-wide fp32 rows; a warp per item of the out-CSR,
// 2 rows per load instruction (16 lanes x 16 B per 256-byte row), 8 rows in flight.  An item of a
// split node writes its partial row (k_split_out_finish adds them in order); a single-item node is
// read-modify-written by its warp.
__global__ void __launch_bounds__(256) k_spmm_out(int32_t n_items, const Item *__restrict__ items,
                                                  const uint2 *__restrict__ ic_edge, const float *__restrict__ da,
                                                  float *__restrict__ dh, float *__restrict__ scratch) {
    const int lane = threadIdx.x & 31;
    const int sub = lane >> 4;       // which of 2 edges
    const int f4 = (lane & 15) * 4;  // first of this lane's 4 features
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int it = warp; it < n_items; it += nwarps) {
        const Item item = items[it];
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int32_t b = item.begin; b < item.end; b += 32) {
            const int cnt = min(32, item.end - b);
            uint2 my = make_uint2(0u, 0u);
            if (lane < cnt) my = ic_edge[b + lane];
            const float myq = edge_q(my.y);
            for (int j = 0; j < cnt; j += 8) {
                float4 xx[4];
                float qq[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int e = j + sub + 2 * r;
                    const uint32_t w = __shfl_sync(0xffffffffu, my.x, e & 31);
                    const float q = __shfl_sync(0xffffffffu, myq, e & 31);
                    qq[r] = e < cnt ? q : 0.0f;
                    xx[r] = *reinterpret_cast<const float4 *>(da + (size_t)(e < cnt ? w : 0u) * H + f4);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc.x += qq[r] * xx[r].x;
                    acc.y += qq[r] * xx[r].y;
                    acc.z += qq[r] * xx[r].z;
                    acc.w += qq[r] * xx[r].w;
                }
            }
        }
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, 16);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, 16);
        if (lane < 16) {
            float4 *row = reinterpret_cast<float4 *>(dh + (size_t)item.node * H + f4);
            if (item.slot < 0) {
                float4 v = *row;
                v.x += acc.x;
                v.y += acc.y;
                v.z += acc.z;
                v.w += acc.w;
                *row = v;
            } else {
                *reinterpret_cast<float4 *>(scratch + (size_t)item.slot * H + f4) = acc;
            }
        }
    }
}

// scalar transpose aggregation: ds[u] += sum over out-edges of q da[w]; a thread per node
__global__ void k_spmm_out_scalar(int32_t n, const int32_t *__restrict__ row_ptr, const uint2 *__restrict__ ic_edge,
                                  const float *__restrict__ da, float *__restrict__ ds) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            const uint2 ed = ic_edge[e];
            s += edge_q(ed.y) * da[ed.x];
        }
        ds[u] += s;
    }
}

// --------------------------------------------------------------------------- dense layers
// Per warp a 16-row tile; lane = 4 g + t (g = lane / 4 row group, t = lane % 4).
template <int DIN>
struct WTile {
    static constexpr int K = 2 * DIN;       // input width [h | a]
    static constexpr int LDW = K + 8;       // padded row of wcat (bank-conflict free fragment loads)
    static constexpr int LDT = H + 8;       // padded row of wt
};

// h_out = bf16(relu([h_in | a] W^T + b)); HEAD: also o = w_o . h_out + b_o
template <int DIN, bool HEAD>
__global__ void __launch_bounds__(128) k_dense_fwd(int32_t n, const __nv_bfloat16 *__restrict__ hin,
                                                   const __nv_bfloat16 *__restrict__ ain,
                                                   const __nv_bfloat16 *__restrict__ wcat,
                                                   const float *__restrict__ params, int layer,
                                                   __nv_bfloat16 *__restrict__ hout, float *__restrict__ o_out) {
    using T = WTile<DIN>;
    __shared__ __align__(16) __nv_bfloat16 sw[H * T::LDW];
    __shared__ float sb[H], swo[H];
    for (int i = threadIdx.x; i < H * T::K; i += blockDim.x) sw[(i / T::K) * T::LDW + i % T::K] = wcat[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        sb[i] = params[off_b(layer) + i];
        swo[i] = params[OFF_WO + i];
    }
    __syncthreads();
    const float bo = params[OFF_BO];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int tiles = (n + 15) >> 4;
    for (int tile = warp; tile < tiles; tile += nwarps) {
        const int rA = tile * 16 + g, rB = rA + 8;
        const bool okA = rA < n, okB = rB < n;
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < T::K / 16; ++kk) {
            const __nv_bfloat16 *src = (kk * 16 < DIN) ? hin : ain;
            const int c = (kk * 16) % DIN + 2 * t;
            const uint32_t a0 = okA ? ld_u32(src + (size_t)rA * DIN + c) : 0u;
            const uint32_t a1 = okB ? ld_u32(src + (size_t)rB * DIN + c) : 0u;
            const uint32_t a2 = okA ? ld_u32(src + (size_t)rA * DIN + c + 8) : 0u;
            const uint32_t a3 = okB ? ld_u32(src + (size_t)rB * DIN + c + 8) : 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __nv_bfloat16 *wr = sw + (j * 8 + g) * T::LDW + kk * 16 + 2 * t;
                mma16816(acc[j], a0, a1, a2, a3, ld_u32(wr), ld_u32(wr + 8));
            }
        }
        float pA = 0.0f, pB = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = j * 8 + 2 * t;
            const float z0 = round_bf16(fmaxf(acc[j][0] + sb[col], 0.0f));
            const float z1 = round_bf16(fmaxf(acc[j][1] + sb[col + 1], 0.0f));
            const float z2 = round_bf16(fmaxf(acc[j][2] + sb[col], 0.0f));
            const float z3 = round_bf16(fmaxf(acc[j][3] + sb[col + 1], 0.0f));
            if (okA) *reinterpret_cast<uint32_t *>(hout + (size_t)rA * H + col) = pack_bf16(z0, z1);
            if (okB) *reinterpret_cast<uint32_t *>(hout + (size_t)rB * H + col) = pack_bf16(z2, z3);
            if (HEAD) {
                pA += z0 * swo[col] + z1 * swo[col + 1];
                pB += z2 * swo[col] + z3 * swo[col + 1];
            }
        }
        if (HEAD) {
            pA += __shfl_xor_sync(0xffffffffu, pA, 1);
            pA += __shfl_xor_sync(0xffffffffu, pA, 2);
            pB += __shfl_xor_sync(0xffffffffu, pB, 1);
            pB += __shfl_xor_sync(0xffffffffu, pB, 2);
            if (t == 0) {
                if (okA) o_out[rA] = pA + bo;
                if (okB) o_out[rB] = pB + bo;
            }
        }
    }
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// Head gradient g_v of the objective w.r.t. o_v.  MODE 1: loss (targets y, or counts * inv_t);
// MODE 2: the predicted spread sum_v yhat_v.
struct HeadArgs {
    const float *o;
    const __nv_bfloat16 *x;  // x_v[0] = s_v
    const float *y;          // MODE 1 targets, or null: cnt * inv_t
    const int32_t *cnt;
    float inv_t;
    float scale;             // MODE 1: 2 / n / batch
    double *loss;            // MODE 1: sum of (yhat - y)^2 / n / batch
    float loss_scale;
};

template <int MODE>
__device__ __forceinline__ float head_grad(const HeadArgs &ha, int r, bool ok, float &lossterm) {
    lossterm = 0.0f;
    if (!ok) return 0.0f;
    const float s = __bfloat162float(ha.x[(size_t)r * D0]);
    const float sg = sigmoidf_(ha.o[r]);
    if (MODE == 2) return (1.0f - s) * sg * (1.0f - sg);
    const float y = ha.y ? ha.y[r] : (float)ha.cnt[r] * ha.inv_t;
    const float yh = s + (1.0f - s) * sg;
    lossterm = (yh - y) * (yh - y);
    return ha.scale * (yh - y) * (1.0f - s) * sg * (1.0f - sg);
}

// Backward of one layer.  dz = dh * [h_out > 0] (MODE 0: dh read from memory; MODE 1, 2: dh = g w_o
// from the head).  GRADS: e = bf16(dz) stored for k_dw, bias (and head) gradients accumulated.
// XOUT 1: dX = e [W_s | W_n] -> dh_prev (first DIN columns) and da (last DIN); XOUT 2: column 0 of
// each half only -> ds0, da0 (the seed channel, for screening).
// GRADS: block b writes its partial sums to part[b * kBwdPart ..] (bias 64, w_o 64, b_o 1, loss 1);
// k_reduce_bwd adds them up in block order.
constexpr int kBwdPart = 2 * H + 2;
template <int DIN, int MODE, int XOUT, bool GRADS>
__global__ void __launch_bounds__(128) k_dense_bwd(int32_t n, const __nv_bfloat16 *__restrict__ hout,
                                                   const float *__restrict__ dh, HeadArgs ha,
                                                   const __nv_bfloat16 *__restrict__ wt, int layer,
                                                   const float *__restrict__ params, __nv_bfloat16 *__restrict__ e_out,
                                                   float *__restrict__ dprev, float *__restrict__ da,
                                                   float *__restrict__ part) {
    using T = WTile<DIN>;
    __shared__ __align__(16) __nv_bfloat16 swt[(XOUT ? T::K : 1) * T::LDT];
    __shared__ float swo[H];
    if (XOUT)
        for (int i = threadIdx.x; i < T::K * H; i += blockDim.x) swt[(i / H) * T::LDT + i % H] = wt[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) swo[i] = params[OFF_WO + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int tiles = (n + 15) >> 4;
    float db[16], dwo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) db[i] = dwo[i] = 0.0f;
    float dbo = 0.0f, lsum = 0.0f;
    for (int tile = warp; tile < tiles; tile += nwarps) {
        const int rA = tile * 16 + g, rB = rA + 8;
        const bool okA = rA < n, okB = rB < n;
        float gA = 0.0f, gB = 0.0f;
        if (MODE != 0) {
            float lA, lB;
            gA = head_grad<MODE>(ha, rA, okA, lA);
            gB = head_grad<MODE>(ha, rB, okB, lB);
            if (t == 0) lsum += lA + lB;
            if (t == 0) dbo += gA + gB;
        }
        uint32_t e[8][2];  // bf16 pairs of dz: [j][0] row A cols (2t, 2t+1), [j][1] row B
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = j * 8 + 2 * t;
            const float2 hA = okA ? unpack_bf16(ld_u32(hout + (size_t)rA * H + col)) : make_float2(0.f, 0.f);
            const float2 hB = okB ? unpack_bf16(ld_u32(hout + (size_t)rB * H + col)) : make_float2(0.f, 0.f);
            float2 dA, dB;
            if (MODE == 0) {
                dA = okA ? *reinterpret_cast<const float2 *>(dh + (size_t)rA * H + col) : make_float2(0.f, 0.f);
                dB = okB ? *reinterpret_cast<const float2 *>(dh + (size_t)rB * H + col) : make_float2(0.f, 0.f);
            } else {
                dA = make_float2(gA * swo[col], gA * swo[col + 1]);
                dB = make_float2(gB * swo[col], gB * swo[col + 1]);
                if (GRADS) {
                    dwo[2 * j] += gA * hA.x + gB * hB.x;
                    dwo[2 * j + 1] += gA * hA.y + gB * hB.y;
                }
            }
            const float z0 = hA.x > 0.0f ? dA.x : 0.0f, z1 = hA.y > 0.0f ? dA.y : 0.0f;
            const float z2 = hB.x > 0.0f ? dB.x : 0.0f, z3 = hB.y > 0.0f ? dB.y : 0.0f;
            if (GRADS) {
                db[2 * j] += z0 + z2;
                db[2 * j + 1] += z1 + z3;
            }
            e[j][0] = pack_bf16(z0, z1);
            e[j][1] = pack_bf16(z2, z3);
            if (GRADS) {
                if (okA) *reinterpret_cast<uint32_t *>(e_out + (size_t)rA * H + col) = e[j][0];
                if (okB) *reinterpret_cast<uint32_t *>(e_out + (size_t)rB * H + col) = e[j][1];
            }
        }
        if (XOUT) {
            // dX[r][i] = sum_o e[r][o] W[o][i]: A = e (accumulator layout reused as A fragments), B[k=o][n=i] = wt[i][o]
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                constexpr int NT = DIN / 8;
                float acc[NT][4];
#pragma unroll
                for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        if (XOUT == 2 && j > 0) continue;
                        const __nv_bfloat16 *wr = swt + (half * DIN + j * 8 + g) * T::LDT + kk * 16 + 2 * t;
                        mma16816(acc[j], e[2 * kk][0], e[2 * kk][1], e[2 * kk + 1][0], e[2 * kk + 1][1],
                                 ld_u32(wr), ld_u32(wr + 8));
                    }
                }
                float *dst = half == 0 ? dprev : da;
                if (XOUT == 1) {
#pragma unroll
                    for (int j = 0; j < NT; ++j) {
                        const int col = j * 8 + 2 * t;
                        if (okA) *reinterpret_cast<float2 *>(dst + (size_t)rA * DIN + col) = make_float2(acc[j][0], acc[j][1]);
                        if (okB) *reinterpret_cast<float2 *>(dst + (size_t)rB * DIN + col) = make_float2(acc[j][2], acc[j][3]);
                    }
                } else if (t == 0) {  // column 0 lives in lanes with t == 0, n-tile 0
                    if (okA) dst[rA] = acc[0][0];
                    if (okB) dst[rB] = acc[0][2];
                }
            }
        }
    }
    if (GRADS) {
        // reduce over the 8 row groups (lanes with equal t), then over the block's warps in shared
        // memory, in a fixed order; the block's sums go to its partial row
        __shared__ float s_db[4][H], s_dwo[4][H], s_misc[4][2];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            for (int off = 4; off < 32; off <<= 1) {
                db[i] += __shfl_xor_sync(0xffffffffu, db[i], off);
                if (MODE == 1) dwo[i] += __shfl_xor_sync(0xffffffffu, dwo[i], off);
            }
        }
        const int wib = threadIdx.x >> 5;
        if (g == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = j * 8 + 2 * t;
                s_db[wib][col] = db[2 * j];
                s_db[wib][col + 1] = db[2 * j + 1];
                s_dwo[wib][col] = dwo[2 * j];
                s_dwo[wib][col + 1] = dwo[2 * j + 1];
            }
        }
        if (MODE == 1) {
            for (int off = 1; off < 32; off <<= 1) {
                dbo += __shfl_xor_sync(0xffffffffu, dbo, off);
                lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
            }
            if (lane == 0) {
                s_misc[wib][0] = dbo;
                s_misc[wib][1] = lsum;
            }
        }
        __syncthreads();
        const int nw = blockDim.x >> 5;
        float *pb = part + (size_t)blockIdx.x * kBwdPart;
        if (threadIdx.x < H) {
            float a = 0.0f, b = 0.0f;
            for (int w = 0; w < nw; ++w) {
                a += s_db[w][threadIdx.x];
                b += s_dwo[w][threadIdx.x];
            }
            pb[threadIdx.x] = a;
            pb[H + threadIdx.x] = MODE == 1 ? b : 0.0f;
        }
        if (threadIdx.x == 0) {
            float a = 0.0f, b = 0.0f;
            if (MODE == 1)
                for (int w = 0; w < nw; ++w) {
                    a += s_misc[w][0];
                    b += s_misc[w][1];
                }
            pb[2 * H] = a;
            pb[2 * H + 1] = b;
        }
    }
}

// dW[o][i] = sum_r e[r][o] X[r][i], X = [h_prev | a] (split-K over row chunks; 8 warps per block,
// warp w owns outputs o in [16 (w % 4), +16) and inputs i in [K/2 (w / 4), +K/2)); block b writes its
// partial dW (64 x 2 DIN, row-major) to part[b * 128 DIN ..], added up in block order by k_reduce_dw
template <int DIN>
__global__ void __launch_bounds__(256) k_dw(int32_t n, const __nv_bfloat16 *__restrict__ e,
                                            const __nv_bfloat16 *__restrict__ hprev,
                                            const __nv_bfloat16 *__restrict__ ain, float *__restrict__ part,
                                            int rows_per_block) {
    constexpr int K = 2 * DIN;
    constexpr int LE = H + 8, LX = K + 8;
    constexpr int NT = K / 2 / 8;  // n-tiles per warp
    constexpr int RC = 32;         // rows per chunk
    __shared__ __align__(16) __nv_bfloat16 se[RC * LE];
    __shared__ __align__(16) __nv_bfloat16 sx[RC * LX];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int o0 = 16 * (w & 3), i0 = (K / 2) * (w >> 2);
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    const int rb = blockIdx.x * rows_per_block;
    const int re = min(n, rb + rows_per_block);
    for (int r0 = rb; r0 < re; r0 += RC) {
        // stage e rows (64 bf16 = 8 x 16 B) and X rows (K bf16 = K/8 x 16 B)
        for (int i = threadIdx.x; i < RC * 8; i += blockDim.x) {
            const int r = i >> 3, c = (i & 7) * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r0 + r < re) v = *reinterpret_cast<const uint4 *>(e + (size_t)(r0 + r) * H + c);
            *reinterpret_cast<uint4 *>(se + r * LE + c) = v;
        }
        for (int i = threadIdx.x; i < RC * (K / 8); i += blockDim.x) {
            const int r = i / (K / 8), c = (i % (K / 8)) * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r0 + r < re)
                v = c < DIN ? *reinterpret_cast<const uint4 *>(hprev + (size_t)(r0 + r) * DIN + c)
                            : *reinterpret_cast<const uint4 *>(ain + (size_t)(r0 + r) * DIN + (c - DIN));
            *reinterpret_cast<uint4 *>(sx + r * LX + c) = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < RC / 16; ++ks) {
            const int r = ks * 16;
            auto E = [&](int rr, int oo) { return se[(r + rr) * LE + o0 + oo]; };
            auto pk = [](__nv_bfloat16 lo, __nv_bfloat16 hi) {
                return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            };
            const uint32_t a0 = pk(E(2 * t, g), E(2 * t + 1, g));
            const uint32_t a1 = pk(E(2 * t, g + 8), E(2 * t + 1, g + 8));
            const uint32_t a2 = pk(E(2 * t + 8, g), E(2 * t + 9, g));
            const uint32_t a3 = pk(E(2 * t + 8, g + 8), E(2 * t + 9, g + 8));
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int col = i0 + j * 8 + g;
                const uint32_t b0 = pk(sx[(r + 2 * t) * LX + col], sx[(r + 2 * t + 1) * LX + col]);
                const uint32_t b1 = pk(sx[(r + 2 * t + 8) * LX + col], sx[(r + 2 * t + 9) * LX + col]);
                mma16816(acc[j], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncthreads();
    }
    float *pb = part + (size_t)blockIdx.x * (H * K);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int o = o0 + g + (q >= 2 ? 8 : 0);
            const int i = i0 + j * 8 + 2 * t + (q & 1);
            pb[o * K + i] = acc[j][q];
        }
    }
}

// grad += the blocks' partial dW of layer `layer`, added in block order (a thread per weight)
__global__ void k_reduce_dw(int32_t nblocks, int32_t din, const float *__restrict__ part, int layer,
                            float *__restrict__ grad) {
    const int K = 2 * din;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < H * K; idx += gridDim.x * blockDim.x) {
        float sum = 0.0f;
        for (int b = 0; b < nblocks; ++b) sum += part[(size_t)b * H * K + idx];
        const int o = idx / K, i = idx % K;
        grad[i < din ? off_ws(layer) + o * din + i : off_wn(layer) + o * din + (i - din)] += sum;
    }
}

// grad (bias of `layer`; MODE 1 also w_o, b_o and the loss) += the blocks' partial sums, in block order
__global__ void k_reduce_bwd(int32_t nblocks, const float *__restrict__ part, int layer, int head,
                             float *__restrict__ grad, double *__restrict__ loss, float loss_scale) {
    const int c = threadIdx.x;  // 0 .. 2 H + 1
    if (c >= kBwdPart || (!head && c >= H)) return;
    if (c < 2 * H + 1) {
        float sum = 0.0f;
        for (int b = 0; b < nblocks; ++b) sum += part[(size_t)b * kBwdPart + c];
        grad[c < H ? off_b(layer) + c : (c < 2 * H ? OFF_WO + (c - H) : OFF_BO)] += sum;
    } else {
        double sum = 0.0;
        for (int b = 0; b < nblocks; ++b) sum += (double)part[(size_t)b * kBwdPart + c];
        *loss += sum * (double)loss_scale;
    }
}

// yhat and the predicted spread; screening scores
// yhat, and each block's sum of it in part[block] (256 threads; k_sum_parts adds the blocks in order)
__global__ void __launch_bounds__(256) k_yhat(int32_t n, const float *__restrict__ o,
                                              const __nv_bfloat16 *__restrict__ x, float *__restrict__ yhat,
                                              double *__restrict__ part) {
    __shared__ double s_w[8];
    double local = 0.0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float s = __bfloat162float(x[(size_t)v * D0]);
        const float y = s + (1.0f - s) * sigmoidf_(o[v]);
        if (yhat) yhat[v] = y;
        local += y;
    }
    for (int off = 16; off; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; ++w) b += s_w[w];
        part[blockIdx.x] = b;
    }
}

__global__ void k_sum_parts(int32_t nblocks, const double *__restrict__ part, double *__restrict__ out) {
    double sum = 0.0;
    for (int b = 0; b < nblocks; ++b) sum += part[b];
    *out = sum;
}

__global__ void k_scores(int32_t n, const float *__restrict__ o, const __nv_bfloat16 *__restrict__ x,
                         const float *__restrict__ ds0, float *__restrict__ score) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float s = __bfloat162float(x[(size_t)v * D0]);
        score[v] = (1.0f - s) * (1.0f - sigmoidf_(o[v])) + ds0[v];
    }
}

// (1 - yhat_c) (1 + sum over out-edges of q (1 - yhat_w)); a thread per node
__global__ void k_onehop(int32_t n, const int32_t *__restrict__ row_ptr, const uint2 *__restrict__ ic_edge,
                         const float *__restrict__ yhat, float *__restrict__ score) {
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        float s = 1.0f;
        for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
            const uint2 ed = ic_edge[e];
            s += edge_q(ed.y) * (1.0f - yhat[ed.x]);
        }
        score[c] = (1.0f - yhat[c]) * s;
    }
}

__global__ void k_adam(int32_t np, float *__restrict__ p, const float *__restrict__ grad, float gscale,
                       float *__restrict__ m, float *__restrict__ v, float lr, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float gr = grad[i] * gscale;
        const float mi = 0.9f * m[i] + 0.1f * gr;
        const float vi = 0.999f * v[i] + 0.001f * gr * gr;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

}  // namespace sur
}  // namespace cnd

// =========================================================================== host object
using namespace cnd;
using namespace cnd::sur;

struct cnd_sur {
    const cnd_graph *g = nullptr;
    int32_t n = 0;
    int device = 0;
    int num_sms = 0;
    // parameters
    float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *wcat = nullptr, *wt = nullptr;
    int64_t adam_t = 0;
    // graph-side
    uint2 *in_c = nullptr;
    Item *items_in = nullptr, *items_out = nullptr;
    int32_t n_items_in = 0, n_items_out = 0;
    int32_t *split_node = nullptr, *split_first = nullptr;  // in-CSR split nodes, first partial row of each
    int32_t n_split = 0;
    float *scratch = nullptr;                                 // partial rows of the in-aggregation
    int32_t *split_out_node = nullptr, *split_out_first = nullptr;
    int32_t n_split_out = 0;
    float *scratch_out = nullptr;                             // partial rows of the out-aggregation
    float *part = nullptr;                                    // per-block partial sums of the backward
    double *part_d = nullptr;                                 // per-block partial sums of the spread
    int32_t part_blocks = 0;                                  // blocks the backward's partials allow
    // activations
    __nv_bfloat16 *x = nullptr, *a1 = nullptr, *h[3] = {nullptr, nullptr, nullptr}, *a[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *e = nullptr;
    unsigned long long *acc0 = nullptr;
    float *o = nullptr, *dhA = nullptr, *dhB = nullptr, *da = nullptr, *ds0 = nullptr,
          *da0 = nullptr, *yv = nullptr;
    int32_t *seeds = nullptr;
    int32_t seeds_cap = 0;
    std::vector<int32_t> row_ptr_h;  // host copy of the out-CSR offsets (training-set sampler)
    double *dsum = nullptr;  // [0] spread, [1] loss
    std::vector<void *> allocs;
};

namespace {

template <class T>
cudaError_t dalloc(cnd_sur *s, T **p, size_t count) {
    void *q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(T));
    if (e == cudaSuccess) {
        s->allocs.push_back(q);
        *p = static_cast<T *>(q);
    }
    return e;
}

void free_all(cnd_sur *s) {
    for (void *q : s->allocs) cudaFree(q);
    s->allocs.clear();
}

// work items of <= kItemEdges edges per node; a row with more edges is split, each of its items
// getting a partial-row slot of its own (consecutive per node): split[i] is the i-th split node and
// first[i] .. first[i+1]-1 its slots
void make_items(const std::vector<int32_t> &rp, std::vector<Item> &items, std::vector<int32_t> &split,
                std::vector<int32_t> &first) {
    const int32_t n = (int32_t)rp.size() - 1;
    items.clear();
    split.clear();
    first.assign(1, 0);
    int32_t slot = 0;
    for (int32_t v = 0; v < n; ++v) {
        const int32_t b = rp[v], e = rp[v + 1];
        if (e - b <= kItemEdges) {
            items.push_back({v, b, e, -1});
        } else {
            split.push_back(v);
            for (int32_t k = b; k < e; k += kItemEdges) items.push_back({v, k, std::min(e, k + kItemEdges), slot++});
            first.push_back(slot);
        }
    }
}

int grid_for(int64_t work, int per_block, int num_sms, int max_per_sm = 8) {
    const int64_t blocks = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * max_per_sm));
}

struct DevGuard {
    int prev = -1;
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

cnd_status enter(const cnd_sur *s, DevGuard &gd) {
    int dev = 0;
    CND_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != s->device) {
        CND_CUDA_TRY(cudaSetDevice(s->device));
        gd.prev = dev;
    }
    return CND_OK;
}

cnd_status upload_seeds(cnd_sur *s, const int32_t *seeds, int32_t ns, int32_t &ns_out, cudaStream_t st,
                        const char *fn) {
    if (ns < 0 || (ns > 0 && !seeds)) {
        set_error("%s: bad seed list", fn);
        return CND_EINVAL;
    }
    std::vector<int32_t> u(seeds, seeds + ns);
    for (int32_t x : u)
        if (x < 0 || x >= s->n) {
            set_error("%s: seed %d out of range", fn, (int)x);
            return CND_EINVAL;
        }
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    if ((int32_t)u.size() > s->seeds_cap) {
        set_error("%s: more distinct seeds than nodes", fn);
        return CND_EINVAL;
    }
    if (!u.empty())
        CND_CUDA_TRY(cudaMemcpyAsync(s->seeds, u.data(), sizeof(int32_t) * u.size(), cudaMemcpyHostToDevice, st));
    ns_out = (int32_t)u.size();
    return CND_OK;
}

void seed_set(cnd_sur *s, const int32_t *d_seeds, int32_t ns, cudaStream_t st) {
    if (ns == 0) return;
    const cnd_graph_dev &G = s->g->d;
    const int blocks = grid_for((int64_t)ns * 32, 256, s->num_sms);
    k_seed_scatter<<<blocks, 256, 0, st>>>(d_seeds, ns, G.row_ptr, G.ic_edge, s->x, s->acc0);
    k_seed_finish<0><<<blocks, 256, 0, st>>>(d_seeds, ns, G.row_ptr, G.ic_edge, s->x, s->a1, s->acc0);
}

void seed_clear(cnd_sur *s, const int32_t *d_seeds, int32_t ns, cudaStream_t st) {
    if (ns == 0) return;
    const cnd_graph_dev &G = s->g->d;
    const int blocks = grid_for((int64_t)ns * 32, 256, s->num_sms);
    k_seed_finish<1><<<blocks, 256, 0, st>>>(d_seeds, ns, G.row_ptr, G.ic_edge, s->x, s->a1, s->acc0);
}

void aggregate_in(cnd_sur *s, const __nv_bfloat16 *hin, __nv_bfloat16 *aout, cudaStream_t st) {
    const int blocks = grid_for((int64_t)s->n_items_in * 32, 256, s->num_sms);
    k_spmm_in<<<blocks, 256, 0, st>>>(s->n_items_in, s->items_in, s->in_c, hin, aout, s->scratch);
    if (s->n_split)
        k_split_finish<<<grid_for((int64_t)s->n_split * 32, 256, s->num_sms), 256, 0, st>>>(
            s->n_split, s->split_node, s->split_first, s->scratch, aout);
}

void forward(cnd_sur *s, cudaStream_t st) {
    const int32_t n = s->n;
    const int tb = grid_for(((int64_t)n + 15) / 16 * 32, 128, s->num_sms, 16);
    k_dense_fwd<D0, false><<<tb, 128, 0, st>>>(n, s->x, s->a1, s->wcat, s->p, 0, s->h[0], nullptr);
    aggregate_in(s, s->h[0], s->a[1], st);
    k_dense_fwd<H, false><<<tb, 128, 0, st>>>(n, s->h[0], s->a[1], s->wcat + 64 * 32, s->p, 1, s->h[1], nullptr);
    aggregate_in(s, s->h[1], s->a[2], st);
    k_dense_fwd<H, true><<<tb, 128, 0, st>>>(n, s->h[1], s->a[2], s->wcat + 64 * 32 + 64 * 128, s->p, 2, s->h[2],
                                             s->o);
}

void aggregate_out(cnd_sur *s, const float *da, float *dh, cudaStream_t st) {
    const int blocks = grid_for((int64_t)s->n_items_out * 32, 256, s->num_sms);
    k_spmm_out<<<blocks, 256, 0, st>>>(s->n_items_out, s->items_out, s->g->d.ic_edge, da, dh, s->scratch_out);
    if (s->n_split_out)
        k_split_out_finish<<<grid_for((int64_t)s->n_split_out * 32, 256, s->num_sms), 256, 0, st>>>(
            s->n_split_out, s->split_out_node, s->split_out_first, s->scratch_out, dh);
}

// the predicted spread (sum of yhat) into *spread, summed in a fixed order
void spread_sum(cnd_sur *s, double *spread, cudaStream_t st) {
    const int nb = grid_for(s->n, 256, s->num_sms);
    k_yhat<<<nb, 256, 0, st>>>(s->n, s->o, s->x, s->yv, s->part_d);
    k_sum_parts<<<1, 1, 0, st>>>(nb, s->part_d, spread);
}

// training backward: gradients accumulate into s->grad; loss adds into s->dsum[1]
void backward_loss(cnd_sur *s, const float *y, const int32_t *cnt, float inv_t, float batch, cudaStream_t st) {
    const int32_t n = s->n;
    const int tb = grid_for(((int64_t)n + 15) / 16 * 32, 128, s->num_sms, 16);
    const int tbb = grid_for(((int64_t)n + 15) / 16 * 32, 128, s->num_sms, 4);  // backward: few blocks, few atomics
    const int rpb = (int)std::max<int64_t>(512, (((int64_t)n + 2 * s->num_sms - 1) / (2 * s->num_sms) + 31) / 32 * 32);
    const int db = (int)std::max<int64_t>(1, ((int64_t)n + rpb - 1) / rpb);
    HeadArgs ha{s->o, s->x, y, cnt, inv_t, 2.0f / (float)n / batch, s->dsum + 1, 1.0f / (float)n / batch};
    HeadArgs none{};
    __nv_bfloat16 *wt2 = s->wt + 64 * 32 + 64 * 128, *wt1 = s->wt + 64 * 32;
    // each gradient kernel writes per-block partial sums; the reduce kernels add them up in block order
    auto bias = [&](int layer, int head) {
        k_reduce_bwd<<<1, 2 * H + 2, 0, st>>>(tbb, s->part, layer, head, s->grad, ha.loss, ha.loss_scale);
    };
    auto weights = [&](int layer, int din) {
        k_reduce_dw<<<grid_for(H * 2 * din, 256, s->num_sms), 256, 0, st>>>(db, din, s->part, layer, s->grad);
    };
    k_dense_bwd<H, 1, 1, true><<<tbb, 128, 0, st>>>(n, s->h[2], nullptr, ha, wt2, 2, s->p, s->e, s->dhA, s->da, s->part);
    bias(2, 1);
    k_dw<H><<<db, 256, 0, st>>>(n, s->e, s->h[1], s->a[2], s->part, rpb);
    weights(2, H);
    aggregate_out(s, s->da, s->dhA, st);
    k_dense_bwd<H, 0, 1, true><<<tbb, 128, 0, st>>>(n, s->h[1], s->dhA, none, wt1, 1, s->p, s->e, s->dhB, s->da, s->part);
    bias(1, 0);
    k_dw<H><<<db, 256, 0, st>>>(n, s->e, s->h[0], s->a[1], s->part, rpb);
    weights(1, H);
    aggregate_out(s, s->da, s->dhB, st);
    k_dense_bwd<D0, 0, 0, true><<<tbb, 128, 0, st>>>(n, s->h[0], s->dhB, none, s->wt, 0, s->p, s->e, nullptr, nullptr,
                                                     s->part);
    bias(0, 0);
    k_dw<D0><<<db, 256, 0, st>>>(n, s->e, s->x, s->a1, s->part, rpb);
    weights(0, D0);
}

void pack_weights(cnd_sur *s, cudaStream_t st) {
    k_pack_weights<<<grid_for(64 * 32 + 2 * 64 * 128, 256, s->num_sms), 256, 0, st>>>(s->p, s->wcat, s->wt);
}

cnd_status check_sur(const cnd_sur *s, const char *fn) {
    if (!s) {
        set_error("%s: surrogate is NULL", fn);
        return CND_EINVAL;
    }
    return CND_OK;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

cnd_status cnd_sur_create(const cnd_graph *g, const float *params, cnd_sur **out) {
    clear_error();
    if (!g || !params || !out) {
        set_error("cnd_sur_create: graph, params and out are required");
        return CND_EINVAL;
    }
    const cnd_graph_dev &G = g->d;
    if (!G.ic_edge && G.m > 0) {
        set_error("cnd_sur_create: graph was created without IC probabilities");
        return CND_EINVAL;
    }
    *out = nullptr;
    cnd_sur *s = new cnd_sur();
    s->g = g;
    s->n = G.n;
    s->device = G.device;
    s->num_sms = std::max(1, G.num_sms);
    DevGuard gd;
    cnd_status st = enter(s, gd);
    if (st != CND_OK) {
        delete s;
        return st;
    }
    auto fail = [&](cudaError_t e, const char *what) {
        set_error("cnd_sur_create: %s: %s", what, cudaGetErrorString(e));
        free_all(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? CND_ENOMEM : CND_ECUDA;
    };
    const int32_t n = G.n, m = G.m;
    std::vector<int32_t> rp((size_t)n + 1), irp((size_t)n + 1);
    cudaError_t e;
    if ((e = cudaMemcpy(rp.data(), G.row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(e, "row_ptr");
    if ((e = cudaMemcpy(irp.data(), G.in_row_ptr, sizeof(int32_t) * irp.size(), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
        return fail(e, "in_row_ptr");
    std::vector<Item> it_in, it_out;
    std::vector<int32_t> split, first, split_out, first_out;
    make_items(irp, it_in, split, first);
    make_items(rp, it_out, split_out, first_out);
    s->row_ptr_h = rp;
    s->n_items_in = (int32_t)it_in.size();
    s->n_items_out = (int32_t)it_out.size();
    s->n_split = (int32_t)split.size();
    s->n_split_out = (int32_t)split_out.size();
    // per-block partials: the backward's blocks (bias rows, dW blocks), the spread's blocks
    const int bwd_blocks = grid_for(((int64_t)n + 15) / 16 * 32, 128, s->num_sms, 4);
    const int rpb0 = (int)std::max<int64_t>(512, (((int64_t)n + 2 * s->num_sms - 1) / (2 * s->num_sms) + 31) / 32 * 32);
    const int dw_blocks = (int)std::max<int64_t>(1, ((int64_t)n + rpb0 - 1) / rpb0);
    const size_t part_floats = std::max<size_t>((size_t)bwd_blocks * kBwdPart, (size_t)dw_blocks * H * 2 * H);
    s->part_blocks = bwd_blocks;
    s->seeds_cap = n;
    const size_t nr = (size_t)n;
#define SUR_ALLOC(ptr, count)                                               \
    if ((e = dalloc(s, &(ptr), (size_t)(count))) != cudaSuccess) return fail(e, "alloc " #ptr);
    SUR_ALLOC(s->p, N_PARAMS);
    SUR_ALLOC(s->m, N_PARAMS);
    SUR_ALLOC(s->v, N_PARAMS);
    SUR_ALLOC(s->grad, N_PARAMS);
    SUR_ALLOC(s->wcat, 64 * 32 + 2 * 64 * 128);
    SUR_ALLOC(s->wt, 64 * 32 + 2 * 64 * 128);
    SUR_ALLOC(s->in_c, m);
    SUR_ALLOC(s->items_in, it_in.size());
    SUR_ALLOC(s->items_out, it_out.size());
    SUR_ALLOC(s->split_node, split.size());
    SUR_ALLOC(s->split_first, first.size());
    SUR_ALLOC(s->scratch, (size_t)first.back() * H);
    SUR_ALLOC(s->split_out_node, split_out.size());
    SUR_ALLOC(s->split_out_first, first_out.size());
    SUR_ALLOC(s->scratch_out, (size_t)first_out.back() * H);
    SUR_ALLOC(s->part, part_floats);
    SUR_ALLOC(s->part_d, (size_t)grid_for(n, 256, s->num_sms));
    SUR_ALLOC(s->x, nr * D0);
    SUR_ALLOC(s->a1, nr * D0);
    for (int l = 0; l < 3; ++l) SUR_ALLOC(s->h[l], nr * H);
    SUR_ALLOC(s->a[1], nr * H);
    SUR_ALLOC(s->a[2], nr * H);
    SUR_ALLOC(s->e, nr * H);
    SUR_ALLOC(s->o, nr);
    SUR_ALLOC(s->acc0, nr);
    SUR_ALLOC(s->dhA, nr * H);
    SUR_ALLOC(s->dhB, nr * H);
    SUR_ALLOC(s->da, nr * H);
    SUR_ALLOC(s->ds0, nr);
    SUR_ALLOC(s->da0, nr);
    SUR_ALLOC(s->yv, nr);
    SUR_ALLOC(s->seeds, nr);
    SUR_ALLOC(s->dsum, 2);
#undef SUR_ALLOC
    if ((e = cudaMemcpy(s->items_in, it_in.data(), sizeof(Item) * it_in.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "items");
    if ((e = cudaMemcpy(s->items_out, it_out.data(), sizeof(Item) * it_out.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return fail(e, "items");
    auto up = [&](int32_t *dst, const std::vector<int32_t> &src) {
        return src.empty() ? cudaSuccess : cudaMemcpy(dst, src.data(), sizeof(int32_t) * src.size(), cudaMemcpyHostToDevice);
    };
    if ((e = up(s->split_node, split)) != cudaSuccess || (e = up(s->split_first, first)) != cudaSuccess ||
        (e = up(s->split_out_node, split_out)) != cudaSuccess || (e = up(s->split_out_first, first_out)) != cudaSuccess)
        return fail(e, "split rows");
    if ((e = cudaMemset(s->acc0, 0, sizeof(unsigned long long) * nr)) != cudaSuccess) return fail(e, "memset");
    const int sms = s->num_sms;
    if (m > 0) k_in_compact<<<grid_for(m, 256, sms), 256>>>(m, G.in_edge, s->in_c);
    k_features<<<grid_for(n, 256, sms), 256>>>(n, G.row_ptr, G.in_row_ptr, s->x);
    k_a1_static<<<grid_for(n, 256, sms), 256>>>(n, G.in_row_ptr, s->in_c, s->x, s->a1);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "setup kernels");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "setup");
    *out = s;
    st = cnd_sur_set_params(s, params);
    if (st != CND_OK) {
        free_all(s);
        delete s;
        *out = nullptr;
    }
    return st;
}

void cnd_sur_destroy(cnd_sur *s) {
    if (!s) return;
    DevGuard gd;
    enter(s, gd);
    free_all(s);
    delete s;
}

cnd_status cnd_sur_set_params(cnd_sur *s, const float *params) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_set_params");
    if (st != CND_OK) return st;
    if (!params) {
        set_error("cnd_sur_set_params: params is NULL");
        return CND_EINVAL;
    }
    for (int i = 0; i < N_PARAMS; ++i)
        if (!std::isfinite(params[i])) {
            set_error("cnd_sur_set_params: parameter %d is not finite", i);
            return CND_EINVAL;
        }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    CND_CUDA_TRY(cudaMemcpy(s->p, params, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice));
    CND_CUDA_TRY(cudaMemset(s->m, 0, sizeof(float) * N_PARAMS));
    CND_CUDA_TRY(cudaMemset(s->v, 0, sizeof(float) * N_PARAMS));
    s->adam_t = 0;
    pack_weights(s, nullptr);
    CND_CUDA_TRY(cudaGetLastError());
    CND_CUDA_TRY(cudaDeviceSynchronize());
    return CND_OK;
}

cnd_status cnd_sur_get_params(const cnd_sur *s, float *params_out) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_get_params");
    if (st != CND_OK) return st;
    if (!params_out) {
        set_error("cnd_sur_get_params: params_out is NULL");
        return CND_EINVAL;
    }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    CND_CUDA_TRY(cudaMemcpy(params_out, s->p, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost));
    return CND_OK;
}

cnd_status cnd_sur_forward(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, float *yhat_out, double *spread_out) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_forward");
    if (st != CND_OK) return st;
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    cudaStream_t cs = nullptr;
    int32_t ns = 0;
    if ((st = upload_seeds(s, seeds, n_seeds, ns, cs, "cnd_sur_forward")) != CND_OK) return st;
    seed_set(s, s->seeds, ns, cs);
    forward(s, cs);
    spread_sum(s, s->dsum, cs);
    seed_clear(s, s->seeds, ns, cs);
    CND_CUDA_TRY(cudaGetLastError());
    if (yhat_out) CND_CUDA_TRY(cudaMemcpyAsync(yhat_out, s->yv, sizeof(float) * s->n, cudaMemcpyDeviceToHost, cs));
    double sp = 0.0;
    CND_CUDA_TRY(cudaMemcpyAsync(&sp, s->dsum, sizeof(double), cudaMemcpyDeviceToHost, cs));
    CND_CUDA_TRY(cudaStreamSynchronize(cs));
    if (spread_out) *spread_out = sp;
    return CND_OK;
}

cnd_status cnd_sur_loss_grad(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, const float *y, double *loss_out,
                             float *grad_out) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_loss_grad");
    if (st != CND_OK) return st;
    if (!y) {
        set_error("cnd_sur_loss_grad: targets are required");
        return CND_EINVAL;
    }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    cudaStream_t cs = nullptr;
    int32_t ns = 0;
    if ((st = upload_seeds(s, seeds, n_seeds, ns, cs, "cnd_sur_loss_grad")) != CND_OK) return st;
    CND_CUDA_TRY(cudaMemcpyAsync(s->yv, y, sizeof(float) * s->n, cudaMemcpyHostToDevice, cs));
    CND_CUDA_TRY(cudaMemsetAsync(s->grad, 0, sizeof(float) * N_PARAMS, cs));
    CND_CUDA_TRY(cudaMemsetAsync(s->dsum, 0, 2 * sizeof(double), cs));
    seed_set(s, s->seeds, ns, cs);
    forward(s, cs);
    backward_loss(s, s->yv, nullptr, 0.0f, 1.0f, cs);
    seed_clear(s, s->seeds, ns, cs);
    CND_CUDA_TRY(cudaGetLastError());
    double ls[2] = {0.0, 0.0};
    CND_CUDA_TRY(cudaMemcpyAsync(ls, s->dsum, 2 * sizeof(double), cudaMemcpyDeviceToHost, cs));
    if (grad_out) CND_CUDA_TRY(cudaMemcpyAsync(grad_out, s->grad, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, cs));
    CND_CUDA_TRY(cudaStreamSynchronize(cs));
    if (loss_out) *loss_out = ls[1];
    return CND_OK;
}

cnd_status cnd_sur_adam(cnd_sur *s, const float *grad, float lr) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_adam");
    if (st != CND_OK) return st;
    if (!grad || !(lr >= 0.0f)) {
        set_error("cnd_sur_adam: gradient required and lr >= 0");
        return CND_EINVAL;
    }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    CND_CUDA_TRY(cudaMemcpy(s->grad, grad, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice));
    s->adam_t += 1;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)s->adam_t);
    const float c2 = 1.0f - (float)std::pow(0.999, (double)s->adam_t);
    k_adam<<<grid_for(N_PARAMS, 256, s->num_sms), 256>>>(N_PARAMS, s->p, s->grad, 1.0f, s->m, s->v, lr, c1, c2);
    pack_weights(s, nullptr);
    CND_CUDA_TRY(cudaGetLastError());
    CND_CUDA_TRY(cudaDeviceSynchronize());
    return CND_OK;
}

cnd_status cnd_sur_scores(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, float *score_out) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_scores");
    if (st != CND_OK) return st;
    if (!score_out) {
        set_error("cnd_sur_scores: score_out is NULL");
        return CND_EINVAL;
    }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    cudaStream_t cs = nullptr;
    int32_t ns = 0;
    if ((st = upload_seeds(s, seeds, n_seeds, ns, cs, "cnd_sur_scores")) != CND_OK) return st;
    const int32_t n = s->n;
    const int tb = grid_for(((int64_t)n + 15) / 16 * 32, 128, s->num_sms, 16);
    seed_set(s, s->seeds, ns, cs);
    forward(s, cs);
    HeadArgs ha{s->o, s->x, nullptr, nullptr, 0.0f, 0.0f, nullptr, 0.0f};
    HeadArgs none{};
    __nv_bfloat16 *wt2 = s->wt + 64 * 32 + 64 * 128, *wt1 = s->wt + 64 * 32;
    k_dense_bwd<H, 2, 1, false><<<tb, 128, 0, cs>>>(n, s->h[2], nullptr, ha, wt2, 2, s->p, nullptr, s->dhA, s->da,
                                                    nullptr);
    aggregate_out(s, s->da, s->dhA, cs);
    k_dense_bwd<H, 0, 1, false><<<tb, 128, 0, cs>>>(n, s->h[1], s->dhA, none, wt1, 1, s->p, nullptr, s->dhB, s->da,
                                                    nullptr);
    aggregate_out(s, s->da, s->dhB, cs);
    k_dense_bwd<D0, 0, 2, false><<<tb, 128, 0, cs>>>(n, s->h[0], s->dhB, none, s->wt, 0, s->p, nullptr, s->ds0,
                                                     s->da0, nullptr);
    const cnd_graph_dev &G = s->g->d;
    k_spmm_out_scalar<<<grid_for(n, 256, s->num_sms), 256, 0, cs>>>(n, G.row_ptr, G.ic_edge, s->da0, s->ds0);
    k_scores<<<grid_for(n, 256, s->num_sms), 256, 0, cs>>>(n, s->o, s->x, s->ds0, s->yv);
    seed_clear(s, s->seeds, ns, cs);
    CND_CUDA_TRY(cudaGetLastError());
    CND_CUDA_TRY(cudaMemcpyAsync(score_out, s->yv, sizeof(float) * n, cudaMemcpyDeviceToHost, cs));
    CND_CUDA_TRY(cudaStreamSynchronize(cs));
    return CND_OK;
}

cnd_status cnd_sur_onehop(cnd_sur *s, const int32_t *seeds, int32_t n_seeds, float *score_out) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_onehop");
    if (st != CND_OK) return st;
    if (!score_out) {
        set_error("cnd_sur_onehop: score_out is NULL");
        return CND_EINVAL;
    }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    cudaStream_t cs = nullptr;
    int32_t ns = 0;
    if ((st = upload_seeds(s, seeds, n_seeds, ns, cs, "cnd_sur_onehop")) != CND_OK) return st;
    const int32_t n = s->n;
    seed_set(s, s->seeds, ns, cs);
    forward(s, cs);
    spread_sum(s, s->dsum, cs);
    const cnd_graph_dev &G = s->g->d;
    k_onehop<<<grid_for(n, 256, s->num_sms), 256, 0, cs>>>(n, G.row_ptr, G.ic_edge, s->yv, s->ds0);
    seed_clear(s, s->seeds, ns, cs);
    CND_CUDA_TRY(cudaGetLastError());
    CND_CUDA_TRY(cudaMemcpyAsync(score_out, s->ds0, sizeof(float) * n, cudaMemcpyDeviceToHost, cs));
    CND_CUDA_TRY(cudaStreamSynchronize(cs));
    return CND_OK;
}

void cnd_sur_train_opts_init(cnd_sur_train_opts *o) {
    if (!o) return;
    *o = cnd_sur_train_opts{};
    o->set_size_lo = 1;
    o->set_size_hi = 50;
    o->n_trials = 1024;
    o->batch_sets = 16;
    o->sim_chunk = 256;
    o->lr = 1e-3f;
    o->data_seed = 1;
    o->rng_seed = 1;
}

}  // extern "C"

// --------------------------------------------------------------------------- training loop
namespace {

uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// uniform integer in [0, range) from a counter-based stream (rejection on the top bits)
struct Stream {
    uint64_t key, ctr = 0;
    uint64_t next() { return splitmix64(key ^ splitmix64(ctr++)); }
    uint32_t below(uint32_t range) {
        const uint64_t lim = (0x100000000ull / range) * range;
        for (;;) {
            const uint64_t r = next() >> 32;
            if (r < lim) return (uint32_t)(r % range);
        }
    }
};

// seed set of pair i: size U{lo..hi}, distinct nodes.  hub_frac == 0: uniform (Floyd's sampling);
// else each seed is, with probability hub_frac, the source of a uniform random edge (row_ptr is
// the host copy of the out-CSR offsets: out-degree prefix sums), else a uniform node; repeats are
// drawn again (and, should draws keep repeating, the lowest free ids fill the set).
void pair_seeds(uint64_t data_seed, int64_t i, int32_t n, int32_t lo, int32_t hi, float hub_frac,
                const std::vector<int32_t> &row_ptr, std::vector<int32_t> &out) {
    Stream r{splitmix64(data_seed) ^ splitmix64(0x5EEDull + (uint64_t)i)};
    const int32_t k = std::min(n, lo + (int32_t)r.below((uint32_t)(hi - lo + 1)));
    out.clear();
    const int32_t m = row_ptr.empty() ? 0 : row_ptr.back();
    if (hub_frac <= 0.0f || m == 0) {
        for (int32_t j = n - k; j < n; ++j) {
            const int32_t t = (int32_t)r.below((uint32_t)j + 1);
            bool dup = std::find(out.begin(), out.end(), t) != out.end();
            out.push_back(dup ? j : t);
        }
        return;
    }
    const uint64_t cut = (uint64_t)((double)hub_frac * 16777216.0);  // hub_frac in 2^-24 units
    for (int64_t tries = 0; (int32_t)out.size() < k && tries < 64 * (int64_t)k + 1024; ++tries) {
        int32_t u;
        if ((r.next() >> 40) < cut) {
            const int32_t e = (int32_t)r.below((uint32_t)m);
            u = (int32_t)(std::upper_bound(row_ptr.begin(), row_ptr.end(), e) - row_ptr.begin()) - 1;
        } else {
            u = (int32_t)r.below((uint32_t)n);
        }
        if (std::find(out.begin(), out.end(), u) == out.end()) out.push_back(u);
    }
    for (int32_t u = 0; (int32_t)out.size() < k && u < n; ++u)
        if (std::find(out.begin(), out.end(), u) == out.end()) out.push_back(u);
}

}  // namespace

extern "C" cnd_status cnd_sur_train(cnd_sur *s, const cnd_sur_train_opts *o, double *loss_out) {
    clear_error();
    cnd_status st = check_sur(s, "cnd_sur_train");
    if (st != CND_OK) return st;
    if (!o || o->n_pairs < 0 || o->first_pair < 0 || o->set_size_lo < 1 || o->set_size_hi < o->set_size_lo ||
        o->n_trials < 1 || !(o->hub_frac >= 0.0f && o->hub_frac <= 1.0f)) {
        set_error("cnd_sur_train: bad options");
        return CND_EINVAL;
    }
    DevGuard gd;
    if ((st = enter(s, gd)) != CND_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(o->stream);
    const int32_t n = s->n;
    const int32_t B = o->batch_sets > 0 ? o->batch_sets : 16;
    int32_t chunk = o->sim_chunk > 0 ? o->sim_chunk : 256;
    chunk = std::max(B, (chunk / B) * B);
    const float lr = o->lr > 0.0f ? o->lr : 1e-3f;
    const int32_t T = o->n_trials;
    // device buffers for one chunk: seeds (all sets) and node counts (sets x n)
    int32_t *d_seeds = nullptr, *d_cnt = nullptr;
    const size_t max_seeds = (size_t)chunk * (size_t)std::min(n, o->set_size_hi);
    CND_CUDA_TRY(cudaMalloc(&d_seeds, sizeof(int32_t) * std::max<size_t>(1, max_seeds)));
    cudaError_t e = cudaMalloc(&d_cnt, sizeof(int32_t) * (size_t)chunk * (size_t)n);
    if (e != cudaSuccess) {
        cudaFree(d_seeds);
        set_error("cnd_sur_train: alloc counts: %s", cudaGetErrorString(e));
        return CND_ENOMEM;
    }
    double *d_loss = nullptr;
    e = cudaMalloc(&d_loss, sizeof(double) * (size_t)((chunk + B - 1) / B));
    if (e != cudaSuccess) {
        cudaFree(d_seeds);
        cudaFree(d_cnt);
        set_error("cnd_sur_train: alloc: %s", cudaGetErrorString(e));
        return CND_ENOMEM;
    }
    struct Free {
        int32_t *a, *b;
        double *c;
        ~Free() {
            cudaFree(a);
            cudaFree(b);
            cudaFree(c);
        }
    } fr{d_seeds, d_cnt, d_loss};
    std::vector<int32_t> hs, one;
    std::vector<int64_t> off;
    std::vector<int32_t> trials;
    std::vector<uint64_t> keys;
    double sim_ms = 0.0, train_ms = 0.0;
    int64_t step = 0;
    cnd_sim_opts so;
    cnd_sim_opts_init(&so);
    so.device_ptrs = 1;
    so.stream = cs;
    so.graph = 1;
    for (int64_t c0 = 0; c0 < o->n_pairs; c0 += chunk) {
        const int32_t cnt = (int32_t)std::min<int64_t>(chunk, o->n_pairs - c0);
        hs.clear();
        off.assign(1, 0);
        trials.assign((size_t)cnt, T);
        keys.resize((size_t)cnt);
        for (int32_t i = 0; i < cnt; ++i) {
            const int64_t pid = o->first_pair + c0 + i;
            pair_seeds(o->data_seed, pid, n, o->set_size_lo, o->set_size_hi, o->hub_frac, s->row_ptr_h, one);
            hs.insert(hs.end(), one.begin(), one.end());
            off.push_back((int64_t)hs.size());
            keys[(size_t)i] = o->rng_seed + (uint64_t)pid;
        }
        const auto t0 = std::chrono::steady_clock::now();
        CND_CUDA_TRY(cudaMemcpyAsync(d_seeds, hs.data(), sizeof(int32_t) * hs.size(), cudaMemcpyHostToDevice, cs));
        st = cnd_ic_simulate_batch(s->g, cnt, off.data(), d_seeds, trials.data(), keys.data(), nullptr, d_cnt, &so);
        if (st != CND_OK) return st;
        CND_CUDA_TRY(cudaStreamSynchronize(cs));
        const auto t1 = std::chrono::steady_clock::now();
        // seed lists hold distinct nodes by construction; a step's loss is kept on the device
        const int64_t step0 = step;
        for (int32_t b0 = 0; b0 < cnt; b0 += B) {
            const int32_t nb = std::min(B, cnt - b0);
            CND_CUDA_TRY(cudaMemsetAsync(s->grad, 0, sizeof(float) * N_PARAMS, cs));
            CND_CUDA_TRY(cudaMemsetAsync(s->dsum, 0, 2 * sizeof(double), cs));
            for (int32_t i = b0; i < b0 + nb; ++i) {
                const int32_t *sd = d_seeds + off[(size_t)i];
                const int32_t ns = (int32_t)(off[(size_t)i + 1] - off[(size_t)i]);
                seed_set(s, sd, ns, cs);
                forward(s, cs);
                backward_loss(s, nullptr, d_cnt + (size_t)i * (size_t)n, 1.0f / (float)T, (float)nb, cs);
                seed_clear(s, sd, ns, cs);
            }
            s->adam_t += 1;
            const float c1 = 1.0f - (float)std::pow(0.9, (double)s->adam_t);
            const float c2 = 1.0f - (float)std::pow(0.999, (double)s->adam_t);
            k_adam<<<grid_for(N_PARAMS, 256, s->num_sms), 256, 0, cs>>>(N_PARAMS, s->p, s->grad, 1.0f, s->m, s->v, lr,
                                                                        c1, c2);
            pack_weights(s, cs);
            CND_CUDA_TRY(cudaGetLastError());
            CND_CUDA_TRY(cudaMemcpyAsync(d_loss + (step - step0), s->dsum + 1, sizeof(double), cudaMemcpyDeviceToDevice,
                                         cs));
            ++step;
        }
        if (loss_out)
            CND_CUDA_TRY(cudaMemcpyAsync(loss_out + step0, d_loss, sizeof(double) * (size_t)(step - step0),
                                         cudaMemcpyDeviceToHost, cs));
        CND_CUDA_TRY(cudaStreamSynchronize(cs));
        const auto t2 = std::chrono::steady_clock::now();
        sim_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
        train_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
    }
    if (o->sim_ms_out) *o->sim_ms_out = sim_ms;
    if (o->train_ms_out) *o->train_ms_out = train_ms;
    return CND_OK;
}
