// Shared definitions of the sm_103a IC/LT engine: device Philox, graph layout,
// error plumbing.  See include/cnd.h for the definitions every kernel follows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cnd.h"

namespace cnd {

constexpr uint32_t kAlways = 0xFFFFFFFFu;  // IC threshold of an edge with p == 1
constexpr uint32_t kFull = 0xFFFFFFFFu;    // full warp mask

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11).  One call yields four
// uint32 for the counter (c0, c1, c2, c3) under key (k0, k1): ten rounds, each
// multiplying c0 and c2 by the two round constants (32x32 -> 64), xoring the
// high halves into the other two words and the round key, and bumping the key
// by the two Weyl constants.
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                     uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t a = (uint64_t)0xD2511F53u * c0;
        const uint64_t b = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)b;
        c3 = (uint32_t)a;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// The ten round keys of one Philox key, precomputed once per call so that
// kernels take them as launch parameters instead of re-deriving them.
struct RoundKeys {
    uint32_t k[20];  // round r uses (k[2r], k[2r+1])
};

inline RoundKeys round_keys(uint64_t key) {
    RoundKeys rk;
    uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return rk;
}

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const RoundKeys &rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t a = (uint64_t)0xD2511F53u * c0;
        const uint64_t b = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ rk.k[2 * r];
        const uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ rk.k[2 * r + 1];
        c1 = (uint32_t)b;
        c3 = (uint32_t)a;
        c0 = n0;
        c2 = n2;
    }
    return U4{c0, c1, c2, c3};
}

// ---------------------------------------------------------------- graph
// Device copy of the caller's CSR.  Edges keep the caller's order, so the
// edge id of the coin definition is the position in these arrays.
struct cnd_graph_dev {
    int32_t n = 0, m = 0;
    int device = 0;
    int32_t *row_ptr = nullptr;   // [n+1]
    uint2 *ic_edge = nullptr;     // [m] {col, IC threshold}, or null
    uint2 *lt_edge = nullptr;     // [m] {col, LT weight}, or null
    int32_t *in_row_ptr = nullptr;  // [n+1] in-CSR (pull direction)
    uint4 *in_edge = nullptr;       // [m] {src, edge id, IC threshold, LT weight}
    int32_t max_out_degree = 0;
    int num_sms = 0;
    // LT counting form, set when every node's non-zero in-weights are equal (the weighted
    // cascade): node v keeps, per 64-trial word, L_v = bits(k_v) bit-sliced counter planes
    // (k_v its in-edges of non-zero weight) at planes [cnt_off[v] * B + w * L_v, + L_v)
    uint2 *lt_cnt_edge = nullptr;   // [m] {col, (cnt_off[col] << 5) | L_col}, 0 for a zero-weight edge
    int32_t *lt_cnt_off = nullptr;  // [n+1] prefix sums of L_v
    uint32_t *lt_unit_w = nullptr;  // [n] the common in-weight of v (0: no in-edge of non-zero weight)
    int64_t lt_planes = 0;          // sum of L_v (planes per word column)
};

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();

}  // namespace cnd

struct cnd_graph {
    cnd::cnd_graph_dev d;
};

#define CND_CUDA_TRY(expr)                                                                    \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess) {                                                              \
            cnd::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
            return _e == cudaErrorMemoryAllocation ? CND_ENOMEM : CND_ECUDA;                  \
        }                                                                                     \
    } while (0)
