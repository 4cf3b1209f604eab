// Classic decomposition (arXiv:1705.03162 Section 5.1): one kernel launch per
// sub-timestep, every point advanced from the previous sub-timestep's full
// array in global memory.  GB300 form: each block stages its tile plus a
// stencil halo (boundary condition applied while loading) in shared memory
// with coalesced loads, then evaluates the shared point update of scheme.cuh.
// Euler evaluates each interface flux once per tile (P per cell, G per
// interface) instead of twice per cell.
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
        for (int s = threadIdx.x; s < SW; s += T) {
            R u;
            P[s] = euler_pressure(sm[s], sm[SW + s], sm[2 * SW + s], c.gm1, u);
        }
        __syncthreads();
        for (int l = threadIdx.x; l < GW; l += T) {
            if (t0 + l > N) break;
            const int sb = RAD + l;
            R qa[3] = {sm[sb - 1], sm[SW + sb - 1], sm[2 * SW + sb - 1]};
            R qb[3] = {sm[sb], sm[SW + sb], sm[2 * SW + sb]};
            R g3[3];
            euler_interface(qa, qb, P[sb - 2], P[sb - 1], P[sb], P[sb + 1], c.gm1, c.ggm1, g3);
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
            for (int v = 0; v < 3; ++v)
                out[v * N + i] = euler_update(G[v * GW + l + 1], G[v * GW + l], base[v * N + i], kh);
        }
    } else {
        for (int l = threadIdx.x; l < TILE; l += T) {
            const int64_t i = t0 + l;
            if (i >= N) break;
            const int s = RAD + l;
            if constexpr (EQ == HEAT) {
                out[i] = heat_point(sm[s - 1], sm[s], sm[s + 1], c.fo);
            } else {
                out[i] = ks_point(sm[s - 2], sm[s - 1], sm[s], sm[s + 1], sm[s + 2], base[i],
                                  c.a1[stage], c.a4[stage], c.beta[stage], c.gam[stage]);
            }
        }
    }
}

template <typename R, int EQ>
cudaError_t classic_launch_eq(int bc, const R* src, const R* base, R* out, int64_t N, int stage,
                              const Coefs<R>& c, int threads, cudaStream_t s)
{
    constexpr int RAD = EQ == HEAT ? 1 : 2;
    constexpr int NV = EQ == EULER ? 3 : 1;
    const int tile = threads * kClassicPointsPerThread;
    const int sw = tile + 2 * RAD;
    size_t smem = sizeof(R) * (size_t)NV * sw;
    if (EQ == EULER) smem += sizeof(R) * ((size_t)sw + 3 * (size_t)(tile + 1));
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
