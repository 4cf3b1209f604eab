// Geometry of the swept tiles shared by the kernel translation units
// (swept.cu, register.cu): stencil radius and variables per equation, node
// partition of [0, N), tile windows, periodic wrap.  Internal header.
#pragma once

#include <cstdint>

#include "scheme.cuh"

namespace swp {

// Slot q of a node window stands for global point g0 + q (mod N).
template <int EQ> struct Shape {
    static constexpr int RAD = EQ == HEAT ? 1 : 2;
    static constexpr int NV = EQ == EULER ? 3 : 1;
};

__host__ __device__ __forceinline__ int window_width(int n, int rad) { return n + 2 * rad; }

// First point of node k of the K nodes of n points (plus the remainder d
// spread over them) that partition [0, N).
__host__ __device__ __forceinline__ int64_t node_start(int64_t k, int n, int K, int d)
{
    return k * n + (k * d) / K;
}

// Window of the tile of node k in a phase: global point of slot 0 and the
// tile's width nk (slots [rad, rad + nk) are its points).  Odd phases: n
// points centred on the node boundary b_k; even phases: the whole node.
__device__ __forceinline__ void tile_window(int k, int odd, int n, int K, int d, int rad, int64_t& g0, int& nk)
{
    const int64_t b = node_start(k, n, K, d);
    if (odd) {
        g0 = b - n / 2 - rad;
        nk = n;
    } else {
        g0 = b - rad;
        nk = (int)(node_start(k + 1, n, K, d) - b);
    }
}

__device__ __forceinline__ int64_t wrap(int64_t g, int64_t N)
{
    return g < 0 ? g + N : (g >= N ? g - N : g);
}

}  // namespace swp
