// The paper's Register variant of the swept rule (Section 5.1), and its form
// on one thread-block cluster.  A node is one warp of 32 points whose levels
// stay in registers; stencil neighbours come from warp shuffles.
#include <cooperative_groups.h>

#include "geometry.cuh"
#include "launch.h"

namespace swp {

namespace {

// ---------------------------------------------------------------------------
// Register variant (Section 5.1): a node is one warp of 32 points; lane l
// holds window slot rad + l of both level rows in registers, and the odd row's
// halo slots (the rad outermost on each side) are held by every lane.  Stencil
// neighbours come from warp shuffles (all 32 lanes always take part, so lanes
// outside the shrinking triangle still supply their values), and levels are
// warp-synchronous: no shared memory and no block barrier.  Periodic problems.
// ---------------------------------------------------------------------------
constexpr int kRegNode = 32;

// Levels j_lo..j_hi of one warp node (lane l holds window slot rad + l: a0 of
// the even-level row, a1 of the odd-level row; hl / hr the odd row's halo
// slots, held by every lane).  Shared by the per-phase Register kernel and
// its cluster form, so both produce the same bits.
template <typename R, int EQ>
__device__ __forceinline__ void warp_node_levels(R& a0, R& a1, const R (&hl)[Shape<EQ>::RAD],
                                                 const R (&hr)[Shape<EQ>::RAD], int j_lo, int j_hi, int H,
                                                 const Coefs<R>& c)
{
    constexpr int RAD = Shape<EQ>::RAD;
    constexpr int n = kRegNode;
    const int lane = threadIdx.x & 31;
    const int cs = n / 2 + RAD;
    for (int j = j_lo; j <= j_hi; ++j) {
        const int w = RAD * (j <= H ? j : 2 * H - j);
        const bool odd_level = j & 1;
        const R src = odd_level ? a0 : a1;
        // stencil values v[RAD + d] = slot lane + d: the lane's own value,
        // neighbours by shuffle up / down, and beyond the warp's ends the odd
        // row's halo (slot -RAD + i is hl[i], slot n + i is hr[i]; the even
        // row never needs its halo: its stencils stay inside)
        R v[2 * RAD + 1];
        v[RAD] = src;
#pragma unroll
        for (int d = 1; d <= RAD; ++d) {
            R lo_v = __shfl_up_sync(0xffffffffu, src, d);
            R hi_v = __shfl_down_sync(0xffffffffu, src, d);
#pragma unroll
            for (int l = 0; l < d; ++l) {
                if (lane == l) lo_v = hl[RAD - d + l];
                if (lane == n - d + l) hi_v = hr[l];
            }
            v[RAD - d] = lo_v;
            v[RAD + d] = hi_v;
        }
        const int slot = RAD + lane;
        if (slot >= cs - w && slot < cs + w) {
            if constexpr (EQ == HEAT) {
                const R o = heat_point(v[0], v[1], v[2], c.fo);
                if (odd_level) a1 = o;
                else a0 = o;
            } else {
                const R o = ks_point(v[0], v[1], v[2], v[3], v[4], a0,
                                     odd_level ? c.a1[0] : c.a1[1], odd_level ? c.a4[0] : c.a4[1],
                                     odd_level ? c.beta[0] : c.beta[1], odd_level ? c.gam[0] : c.gam[1]);
                if (odd_level) a1 = o;
                else a0 = o;
            }
        }
    }
}

template <typename R, int EQ>
__global__ void __launch_bounds__(256) swept_register_kernel(R* A, R* B, PhaseGeom g, Coefs<R> c)
{
    constexpr int RAD = Shape<EQ>::RAD;
    constexpr int n = kRegNode;
    const int lane = threadIdx.x & 31;
    const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= g.K) return;   // whole warps only: K nodes, one per warp
    const int H = g.H;
    const int64_t xc = g.odd ? (int64_t)k * n : (int64_t)k * n + n / 2;
    const int64_t g0 = xc - n / 2 - RAD;   // global point of window slot 0
    const int64_t gl = wrap(g0 + RAD + lane, g.N);
    R a0 = A[gl];
    R a1 = R(0), hl[RAD], hr[RAD];
#pragma unroll
    for (int i = 0; i < RAD; ++i) hl[i] = hr[i] = R(0);
    if (g.j_lo <= H) {
        a1 = B[gl];
#pragma unroll
        for (int i = 0; i < RAD; ++i) {
            hl[i] = B[wrap(g0 + i, g.N)];
            hr[i] = B[wrap(g0 + n + RAD + i, g.N)];
        }
    }
    warp_node_levels<R, EQ>(a0, a1, hl, hr, g.j_lo, g.j_hi, H, c);
    A[gl] = a0;
    if (lane >= RAD && lane < n - RAD) B[gl] = a1;
}

// ---------------------------------------------------------------------------
// The Register variant on one thread-block cluster, for small problems.  The
// per-phase form pays a kernel boundary and a round trip of every node
// window through global memory per phase; at N ~ 10^3 those cost as much as
// the phase's levels.  Here the whole advance is one launch of one cluster of
// C blocks: block r keeps points [r P, (r + 1) P) of both level rows in its
// shared memory, a warp (one 32-point node, as above) reads and writes its
// window through distributed shared memory (the owning block of each point),
// and a cluster barrier separates phases, so the state never leaves the chip
// until the end.  Tiles of one phase write disjoint slots and read no slot
// another tile of the phase writes (as in the per-phase form), so one barrier
// per phase suffices.  Every thread runs every phase's barrier.
// ---------------------------------------------------------------------------
template <typename R, int EQ>
__global__ void __launch_bounds__(256) swept_cluster_kernel(R* A, R* B, ClusterGeom g, Coefs<R> c)
{
    namespace cg = cooperative_groups;
    constexpr int RAD = Shape<EQ>::RAD;
    constexpr int n = kRegNode;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    R* rowA = reinterpret_cast<R*>(smem_raw);   // this block's points of row A
    R* rowB = rowA + g.portion;                 // and of row B
    const int rank = (int)cluster.block_rank();
    const int64_t p0 = (int64_t)rank * g.portion;
    for (int i = threadIdx.x; i < g.portion; i += blockDim.x) {
        rowA[i] = A[p0 + i];
        rowB[i] = B[p0 + i];
    }
    const int lane = threadIdx.x & 31;
    // one node per warp (the host makes the cluster's warps equal the nodes)
    const int k = rank * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    const int H = g.H;
    // the slot of global point x (within one period of [0, N)) in the owning
    // block's row; the tile of node k starts at k n (even phases) or
    // k n - n / 2 (odd phases), so each lane's slots are found once here
    const int N = (int)g.N;
    auto at = [&](R* row, int x) -> R* {
        const int gx = x < 0 ? x + N : (x >= N ? x - N : x);
        return cluster.map_shared_rank(row, (unsigned)(gx / g.portion)) + gx % g.portion;
    };
    R *pa[2], *pb[2], *phl[2][RAD], *phr[2][RAD];
#pragma unroll
    for (int odd = 0; odd < 2; ++odd) {
        const int x0 = odd ? k * n - n / 2 : k * n;
        pa[odd] = at(rowA, x0 + lane);
        pb[odd] = at(rowB, x0 + lane);
#pragma unroll
        for (int i = 0; i < RAD; ++i) {
            phl[odd][i] = at(rowB, x0 - RAD + i);
            phr[odd][i] = at(rowB, x0 + n + i);
        }
    }
    cluster.sync();
    for (int64_t ph = 0; ph < g.n_phases; ++ph) {
        const int odd = (int)(ph & 1);
        const int j_lo = ph == 0 ? H + 1 : 1;
        const int j_hi = ph < g.Q ? 2 * H - 1 : (ph == g.Q ? H + (int)g.r : (int)g.r);
        R* const a_ptr = odd ? pa[1] : pa[0];
        R* const b_ptr = odd ? pb[1] : pb[0];
        R a0 = *a_ptr;
        R a1 = R(0), hl[RAD], hr[RAD];
#pragma unroll
        for (int i = 0; i < RAD; ++i) hl[i] = hr[i] = R(0);
        if (j_lo <= H) {
            a1 = *b_ptr;
#pragma unroll
            for (int i = 0; i < RAD; ++i) {
                hl[i] = *(odd ? phl[1][i] : phl[0][i]);
                hr[i] = *(odd ? phr[1][i] : phr[0][i]);
            }
        }
        warp_node_levels<R, EQ>(a0, a1, hl, hr, j_lo, j_hi, H, c);
        *a_ptr = a0;
        if (lane >= RAD && lane < n - RAD) *b_ptr = a1;
        cluster.sync();
    }
    for (int i = threadIdx.x; i < g.portion; i += blockDim.x) {
        A[p0 + i] = rowA[i];
        B[p0 + i] = rowB[i];
    }
}

template <typename R, int EQ>
cudaError_t register_launch_eq(R* A, R* B, const PhaseGeom& g, const Coefs<R>& c, int threads,
                               cudaStream_t s)
{
    const int64_t warps_per_block = threads / 32;
    const int64_t blocks = (g.K + warps_per_block - 1) / warps_per_block;
    swept_register_kernel<R, EQ><<<(unsigned)blocks, threads, 0, s>>>(A, B, g, c);
    return cudaGetLastError();
}

template <typename R, int EQ>
cudaLaunchConfig_t cluster_config(const ClusterGeom& g, int ctas, int threads, cudaStream_t s,
                                  cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 2 * sizeof(R) * (size_t)g.portion;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <typename R, int EQ>
cudaError_t cluster_launch_eq(R* A, R* B, const ClusterGeom& g, const Coefs<R>& c, int ctas, int threads,
                              cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute((const void*)swept_cluster_kernel<R, EQ>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config<R, EQ>(g, ctas, threads, s, attr);
    return cudaLaunchKernelEx(&cfg, swept_cluster_kernel<R, EQ>, A, B, g, c);
}

template <typename R, int EQ>
int cluster_fits_eq(const ClusterGeom& g, int ctas, int threads)
{
    if (cudaFuncSetAttribute((const void*)swept_cluster_kernel<R, EQ>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) != cudaSuccess)
        return 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config<R, EQ>(g, ctas, threads, nullptr, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)swept_cluster_kernel<R, EQ>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return clusters;
}

}  // namespace

template <typename R>
cudaError_t launch_swept_register(int eq, R* A, R* B, const PhaseGeom& g, const Coefs<R>& c,
                                  int threads, cudaStream_t s)
{
    if (eq == HEAT) return register_launch_eq<R, HEAT>(A, B, g, c, threads, s);
    return register_launch_eq<R, KS>(A, B, g, c, threads, s);
}

template cudaError_t launch_swept_register<double>(int, double*, double*, const PhaseGeom&,
                                                   const Coefs<double>&, int, cudaStream_t);
template cudaError_t launch_swept_register<float>(int, float*, float*, const PhaseGeom&,
                                                  const Coefs<float>&, int, cudaStream_t);

template <typename R>
cudaError_t launch_swept_cluster(int eq, R* A, R* B, const ClusterGeom& g, const Coefs<R>& c, int ctas,
                                 int threads, cudaStream_t s)
{
    if (eq == HEAT) return cluster_launch_eq<R, HEAT>(A, B, g, c, ctas, threads, s);
    return cluster_launch_eq<R, KS>(A, B, g, c, ctas, threads, s);
}

template <typename R>
int swept_cluster_fits(int eq, const ClusterGeom& g, int ctas, int threads)
{
    if (eq == HEAT) return cluster_fits_eq<R, HEAT>(g, ctas, threads);
    return cluster_fits_eq<R, KS>(g, ctas, threads);
}

template cudaError_t launch_swept_cluster<double>(int, double*, double*, const ClusterGeom&, const Coefs<double>&,
                                                  int, int, cudaStream_t);
template cudaError_t launch_swept_cluster<float>(int, float*, float*, const ClusterGeom&, const Coefs<float>&, int,
                                                 int, cudaStream_t);
template int swept_cluster_fits<double>(int, const ClusterGeom&, int, int);
template int swept_cluster_fits<float>(int, const ClusterGeom&, int, int);

}  // namespace swp
