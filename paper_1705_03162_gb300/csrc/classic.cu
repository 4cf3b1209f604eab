// Classic decomposition (arXiv:1705.03162 Section 5.1): one kernel launch per
// sub-timestep, every point advanced from the previous sub-timestep's full
// array in global memory.  GB300 forms: heat and KS stream 16-byte vectors
// with neighbours exchanged by warp shuffle (bandwidth form); otherwise each
// block stages its tile plus a stencil halo (boundary condition applied while
// loading) in shared memory.  Both evaluate the shared point update of
// scheme.cuh.
// Euler evaluates each interface flux once per tile (P per cell, G per
// interface) instead of twice per cell, and reuses each cell's velocity,
// specific energy and sqrt(rho) on the interface sides the limiter leaves
// first order.
#include "launch.h"

namespace swp {

namespace {

constexpr int kClassicPointsPerThread = 2;

// Value of variable v at global point g in [-rad, N + rad) with the boundary
// condition outside [0, N): periodic wrap, mirror about the end points
// (Appendix A Eq. heatcond), or the Dirichlet ghost states (Appendix C).
template <typename R>
__device__ __forceinline__ R bc_load(const R* arr, int64_t g, int64_t N, int bc, int v,
                                     const Coefs<R>& c)
{
    if (g >= 0 && g < N) return arr[v * N + g];
    if (bc == PERIODIC) return arr[v * N + (g < 0 ? g + N : g - N)];
    if (bc == REFLECTIVE) return arr[v * N + (g < 0 ? -g : 2 * (N - 1) - g)];
    return g < 0 ? c.ghost_l[v] : c.ghost_r[v];
}

template <typename R, int EQ>
__global__ void __launch_bounds__(256) classic_kernel(const R* __restrict__ src, const R* base,
                                                      R* out, int64_t N, int stage, int bc,
                                                      Coefs<R> c)
{
    constexpr int RAD = EQ == HEAT ? 1 : 2;
    constexpr int NV = EQ == EULER ? 3 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const int T = blockDim.x;
    const int TILE = T * kClassicPointsPerThread;
    const int SW = TILE + 2 * RAD;
    const int64_t t0 = (int64_t)blockIdx.x * TILE;

    for (int s = threadIdx.x; s < SW; s += T) {
        int64_t g = t0 - RAD + s;
#pragma unroll
        for (int v = 0; v < NV; ++v)
            sm[v * SW + s] = (g < N + RAD) ? bc_load(src, g, N, bc, v, c) : R(0);
    }
    __syncthreads();

    if constexpr (EQ == EULER) {
        R* P = sm + NV * SW;        // pressure of every staged cell
        R* G = P + SW;              // G[v][l]: interface between tile cells l-1 and l
        const int GW = TILE + 1;
        R* Cc = G + 3 * GW;         // cached (u, e, sqrt(rho)) of staged cell s at Cc[k SW + s]
        for (int s = threadIdx.x; s < SW; s += T) {
            P[s] = euler_cell(sm[s], sm[SW + s], sm[2 * SW + s], c.gm1, Cc[s], Cc[SW + s], Cc[2 * SW + s]);
        }
        __syncthreads();
        for (int l = threadIdx.x; l < GW; l += T) {
            if (t0 + l > N) break;
            const int sb = RAD + l;
            R qa[3] = {sm[sb - 1], sm[SW + sb - 1], sm[2 * SW + sb - 1]};
            R qb[3] = {sm[sb], sm[SW + sb], sm[2 * SW + sb]};
            const R ca[3] = {Cc[sb - 1], Cc[SW + sb - 1], Cc[2 * SW + sb - 1]};
            const R cb[3] = {Cc[sb], Cc[SW + sb], Cc[2 * SW + sb]};
            R g3[3];
            euler_interface_cached(qa, qb, P[sb - 2], P[sb - 1], P[sb], P[sb + 1], ca, cb, c.gm1, c.ggm1, g3);
            G[l] = g3[0];
            G[GW + l] = g3[1];
            G[2 * GW + l] = g3[2];
        }
        __syncthreads();
        const R kh = c.kh[stage];
        for (int l = threadIdx.x; l < TILE; l += T) {
            const int64_t i = t0 + l;
            if (i >= N) break;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const R b = stage == 0 ? sm[v * SW + RAD + l] : base[v * N + i];   // predictor: base = source
                out[v * N + i] = euler_update(G[v * GW + l + 1], G[v * GW + l], b, kh);
            }
        }
    } else {
        for (int l = threadIdx.x; l < TILE; l += T) {
            const int64_t i = t0 + l;
            if (i >= N) break;
            const int s = RAD + l;
            if constexpr (EQ == HEAT) {
                out[i] = heat_point(sm[s - 1], sm[s], sm[s + 1], c.fo);
            } else {
                const R b = stage == 0 ? sm[s] : base[i];   // predictor: base = source
                out[i] = ks_point(sm[s - 2], sm[s - 1], sm[s], sm[s + 1], sm[s + 2], b,
                                  c.a1[stage], c.a4[stage], c.beta[stage], c.gam[stage]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Bandwidth form for heat and KS (N a multiple of the vector width): every
// thread moves 16-byte vectors (float4 / double2), U of them in flight (U = 4
// when the grid still covers every SM twice, else 1); stencil neighbours come from the adjacent lanes by warp shuffle, and
// only the first and last lane of a warp row load a halo vector.
// ---------------------------------------------------------------------------
template <typename R> struct Vec16;
template <> struct Vec16<float> {
    using T = float4;
    static constexpr int W = 4;
};
template <> struct Vec16<double> {
    using T = double2;
    static constexpr int W = 2;
};


template <typename R>
__device__ __forceinline__ void vec_to(const typename Vec16<R>::T& v, R* a)
{
    const R* p = reinterpret_cast<const R*>(&v);
#pragma unroll
    for (int i = 0; i < Vec16<R>::W; ++i) a[i] = p[i];
}

// The VW values of vector vi of a level (vi may lie outside [0, nvec): the
// boundary condition supplies them).
template <typename R>
__device__ __forceinline__ void vec_load_bc(const R* arr, int64_t vi, int64_t nvec, int64_t N, int bc,
                                            const Coefs<R>& c, R* a)
{
    constexpr int VW = Vec16<R>::W;
    using T = typename Vec16<R>::T;
    if (vi >= 0 && vi < nvec) {
        vec_to<R>(reinterpret_cast<const T*>(arr)[vi], a);
        return;
    }
#pragma unroll
    for (int i = 0; i < VW; ++i) a[i] = bc_load(arr, vi * VW + i, N, bc, 0, c);
}

template <typename R, int EQ, int U>
__global__ void __launch_bounds__(256) classic_vec_kernel(const R* __restrict__ src, const R* base,
                                                          R* out, int64_t N, int stage, int bc,
                                                          Coefs<R> c)
{
    constexpr int VW = Vec16<R>::W;
    using T = typename Vec16<R>::T;
    const int lane = threadIdx.x & 31;
    const int64_t nvec = N / VW;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t row0 = warp_global * (32 * U);
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t vi = row0 + u * 32 + lane;
        if (vi < nvec) v[u] = reinterpret_cast<const T*>(src)[vi];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t vi = row0 + u * 32 + lane;
        R a[3 * VW];   // left vector, own vector, right vector
        vec_to<R>(v[u], a + VW);
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            a[i] = __shfl_up_sync(0xffffffffu, a[VW + i], 1);
            a[2 * VW + i] = __shfl_down_sync(0xffffffffu, a[VW + i], 1);
        }
        if (vi >= nvec) continue;
        if (lane == 0 || vi == 0) vec_load_bc<R>(src, vi - 1, nvec, N, bc, c, a);
        if (lane == 31 || vi == nvec - 1) vec_load_bc<R>(src, vi + 1, nvec, N, bc, c, a + 2 * VW);
        R o[VW];
        if constexpr (EQ == HEAT) {
#pragma unroll
            for (int i = 0; i < VW; ++i) o[i] = heat_point(a[VW + i - 1], a[VW + i], a[VW + i + 1], c.fo);
        } else {
            R b[VW];
            if (stage == 0) {   // predictor: the base is the source vector itself
#pragma unroll
                for (int i = 0; i < VW; ++i) b[i] = a[VW + i];
            } else {
                vec_to<R>(reinterpret_cast<const T*>(base)[vi], b);
            }
#pragma unroll
            for (int i = 0; i < VW; ++i)
                o[i] = ks_point(a[VW + i - 2], a[VW + i - 1], a[VW + i], a[VW + i + 1], a[VW + i + 2], b[i],
                                c.a1[stage], c.a4[stage], c.beta[stage], c.gam[stage]);
        }
        reinterpret_cast<T*>(out)[vi] = *reinterpret_cast<const T*>(o);
    }
}

template <typename R, int EQ>
cudaError_t classic_launch_eq(int bc, const R* src, const R* base, R* out, int64_t N, int stage,
                              const Coefs<R>& c, int threads, cudaStream_t s)
{
    if constexpr (EQ != EULER) {
        constexpr int VW = Vec16<R>::W;
        if (N % VW == 0 && N / VW >= 32) {
            const int64_t nvec = N / VW;
            const int64_t blocks4 = (nvec + 4 * (int64_t)threads - 1) / (4 * (int64_t)threads);
            if (blocks4 >= 2 * 152) {
                classic_vec_kernel<R, EQ, 4><<<(unsigned)blocks4, threads, 0, s>>>(src, base, out, N, stage, bc, c);
            } else {
                const int64_t blocks1 = (nvec + threads - 1) / threads;
                classic_vec_kernel<R, EQ, 1><<<(unsigned)blocks1, threads, 0, s>>>(src, base, out, N, stage, bc, c);
            }
            return cudaGetLastError();
        }
    }
    constexpr int RAD = EQ == HEAT ? 1 : 2;
    constexpr int NV = EQ == EULER ? 3 : 1;
    const int tile = threads * kClassicPointsPerThread;
    const int sw = tile + 2 * RAD;
    size_t smem = sizeof(R) * (size_t)NV * sw;
    if (EQ == EULER) smem += sizeof(R) * ((size_t)sw + 3 * (size_t)(tile + 1) + 3 * (size_t)sw);
    const int64_t blocks = (N + tile - 1) / tile;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(classic_kernel<R, EQ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    classic_kernel<R, EQ><<<(unsigned)blocks, threads, smem, s>>>(src, base, out, N, stage, bc, c);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_classic(int eq, int bc, const R* src, const R* base, R* out, int64_t N,
                           int stage, const Coefs<R>& c, int threads, cudaStream_t s)
{
    if (threads <= 0) threads = 256;
    switch (eq) {
    case HEAT: return classic_launch_eq<R, HEAT>(bc, src, base, out, N, stage, c, threads, s);
    case KS: return classic_launch_eq<R, KS>(bc, src, base, out, N, stage, c, threads, s);
    default: return classic_launch_eq<R, EULER>(bc, src, base, out, N, stage, c, threads, s);
    }
}

template cudaError_t launch_classic<double>(int, int, const double*, const double*, double*,
                                            int64_t, int, const Coefs<double>&, int, cudaStream_t);
template cudaError_t launch_classic<float>(int, int, const float*, const float*, float*, int64_t,
                                           int, const Coefs<float>&, int, cudaStream_t);

}  // namespace swp
