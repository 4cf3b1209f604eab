// Swept time-space decomposition (arXiv:1705.03162 Sections 4.2-4.3) for
// GB300.
//
// Geometry.  Nodes of n points, stencil radius rad (1 heat, 2 KS/Euler),
// H = n / (2 rad) sub-timestep levels per half-cycle.  A phase is one kernel
// of the paper: every node advances a space-time tile centred at x_c (node
// centres in even phases, node boundaries in odd phases).  Relative to the
// phase's base level the tile computes level j on the points
// [x_c - w(j), x_c + w(j)) with w(j) = rad * min(j, 2H - j): levels 1..H grow
// (inverted triangle), levels H+1..2H-1 shrink (upright triangle).  Phase 0 is
// the upright triangle alone (levels H+1..2H-1 above the initial row); the
// last phase is the closing inverted triangle (levels 1..H, or 1..r for a
// final partial half-cycle, in which case the phase before it stops its
// upright triangle at level H + r).
//
// Working set.  As in the paper, a node keeps two rows: even levels (heat
// steps / RK2 final values) and odd levels (predictor values).  Each level's
// outermost 2 rad values survive in these rows because even and odd levels'
// edges never overlap (Fig. 2), and the two rows' surviving edges are exactly
// what the neighbouring nodes of the next phase need.  Here the edges are
// exchanged through two full-length rows in global memory, A (even levels)
// and B (odd levels), at their absolute positions: a node loads its window
// [x_c - n/2 - rad, x_c + n/2 + rad) of A and B into shared memory, runs its
// levels with one barrier per level, and writes the window back.  Nodes of one
// phase touch disjoint parts of A and B, so a phase needs no synchronisation
// inside itself; a node of phase p depends only on its two overlapping nodes
// of phase p-1.  At the end A (or B, when the last level is odd) holds the
// full state.
//
// Any N.  The paper's nodes all have n points, so N must be a multiple of n.
// Here N = K n + d with 0 <= d < n: node k covers [b_k, b_{k+1}) with
// b_k = k n + floor(k d / K), so d nodes are one point (or a few points)
// wider.  Odd-phase tiles keep width n, centred on the node boundaries b_k;
// an even-phase tile spans its whole node and computes level j on
// [b_k + rad |j - H|, b_{k+1} - rad |j - H|): a triangle for a node of n
// points, a trapezoid for a wider one, which also computes level 2H on its
// middle points (the gap between the two odd tiles beside it).  Locally the
// geometry is the equal-width one, so the two rows still hold, at every
// position, the latest level of each parity that the next tile reads.
//
// Boundaries.  Periodic problems wrap the window modulo N.  For reflective or
// Dirichlet ends, the node straddling x = 0 (first node of odd phases, the
// paper's split node) and the first/last nodes of even phases (whose widest
// level reaches the ends) evaluate points next to a wall through a
// boundary-aware gather.
#include "geometry.cuh"
#include "launch.h"

namespace swp {

namespace {

// Stencil value at slot q + d for the point at slot q, applying the boundary
// condition when the stencil crosses a domain end: mirror about the end point
// (u_{-k} = u_k, u_{N-1+k} = u_{N-1-k}) or the Dirichlet ghost state.
template <typename R>
__device__ __forceinline__ R wall_fetch(const R* row, int W, int q, int d, int v, int64_t g0,
                                        int64_t N, int bc, const Coefs<R>& c)
{
    const int64_t gp = wrap(g0 + q, N);
    const int64_t gt = gp + d;
    if (gt < 0) {
        if (bc == REFLECTIVE) return row[v * W + (int)(q - 2 * gp - d)];
        return c.ghost_l[v];
    }
    if (gt >= N) {
        if (bc == REFLECTIVE) return row[v * W + (int)(q + 2 * (N - 1 - gp) - d)];
        return c.ghost_r[v];
    }
    return row[v * W + q + d];
}

// 16-byte vectors of the working precision.
template <typename R> struct Vec16;
template <> struct Vec16<double> {
    using T = double2;
    static constexpr int W = 2;
};
template <> struct Vec16<float> {
    using T = float4;
    static constexpr int W = 4;
};

template <typename R, bool CG>
__device__ __forceinline__ typename Vec16<R>::T load_vec(const R* p)
{
    using T = typename Vec16<R>::T;
    return CG ? __ldcg(reinterpret_cast<const T*>(p)) : *reinterpret_cast<const T*>(p);
}

template <typename R, bool CG>
__device__ __forceinline__ void store_vec(R* p, const typename Vec16<R>::T& v)
{
    using T = typename Vec16<R>::T;
    if (CG) __stcg(reinterpret_cast<T*>(p), v);
    else *reinterpret_cast<T*>(p) = v;
}

// Move `count` consecutive points of a global row (period N) starting at
// global point g into shared memory at s (IN) or back (OUT).  The range is
// split where it wraps; inside each piece the block moves 16-byte vectors
// from the first 16-byte-aligned address on, and single values before and
// after.
template <typename R, bool CG, bool IN>
__device__ __forceinline__ void row_copy(R* row, int64_t N, int64_t g, int count, R* s)
{
    constexpr int VW = Vec16<R>::W;
    g = wrap(g, N);
    for (int done = 0; done < count;) {
        const int len = (int)min((int64_t)(count - done), N - g);
        R* gp = row + g;
        R* sp = s + done;
        const int head = min(len, (int)(((16 - (reinterpret_cast<uintptr_t>(gp) & 15)) & 15) / sizeof(R)));
        const int body = (len - head) / VW;
        const int tail = len - head - body * VW;
        for (int t = threadIdx.x; t < head + tail; t += blockDim.x) {
            const int q = t < head ? t : head + body * VW + (t - head);
            if (IN) sp[q] = CG ? __ldcg(gp + q) : gp[q];
            else if (CG) __stcg(gp + q, sp[q]);
            else gp[q] = sp[q];
        }
        for (int i = threadIdx.x; i < body; i += blockDim.x) {
            const int q = head + i * VW;
            if (IN) {
                const typename Vec16<R>::T v = load_vec<R, CG>(gp + q);
                const R* e = reinterpret_cast<const R*>(&v);
#pragma unroll
                for (int k = 0; k < VW; ++k) sp[q + k] = e[k];
            } else {
                typename Vec16<R>::T v;
                R* e = reinterpret_cast<R*>(&v);
#pragma unroll
                for (int k = 0; k < VW; ++k) e[k] = sp[q + k];
                store_vec<R, CG>(gp + q, v);
            }
        }
        done += len;
        g = 0;
    }
}

// Load the window of a tile of n points from rows A / B (global, [NV][N])
// into shared memory.  Row 0 (A) occupies slots [rad, rad + n); row 1 (B)
// all W = n + 2 rad slots.  Coalesced 16-byte vector loads (row_copy).
template <typename R, int EQ, bool CG>
__device__ __forceinline__ void window_load(const R* A, const R* B, R* row0, R* row1, int n,
                                            int64_t g0, int64_t N, bool need_b)
{
    constexpr int RAD = Shape<EQ>::RAD, NV = Shape<EQ>::NV;
    const int W = window_width(n, RAD);
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
        row_copy<R, CG, true>(const_cast<R*>(A) + v * N, N, g0 + RAD, n, row0 + v * W + RAD);
        if (need_b) row_copy<R, CG, true>(const_cast<R*>(B) + v * N, N, g0, W, row1 + v * W);
    }
}

// Write back what a tile of n points may have changed: row 0 slots
// [rad, rad + n) and row 1 slots [2 rad, n) (the odd levels of its upright
// triangle).
template <typename R, int EQ, bool CG>
__device__ __forceinline__ void window_store(R* A, R* B, const R* row0, const R* row1, int n,
                                             int64_t g0, int64_t N)
{
    constexpr int RAD = Shape<EQ>::RAD, NV = Shape<EQ>::NV;
    const int W = window_width(n, RAD);
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
        row_copy<R, CG, false>(A + v * N, N, g0 + RAD, n, const_cast<R*>(row0) + v * W + RAD);
        row_copy<R, CG, false>(B + v * N, N, g0 + 2 * RAD, n - 2 * RAD, const_cast<R*>(row1) + v * W + 2 * RAD);
    }
}

// One heat / KS level of cnt points from slot lo (source row src, result row
// dst; KS stage 1 takes its base values from dst, which is row 0 then), each
// thread sweeping a contiguous run of the points with the stencil window in
// registers: one shared-memory load per point instead of 2 rad + 1.  The runs
// have odd length, so the threads of a warp address distinct banks while they
// step together: the sweep goes 2 rad + 1 points at a time (the window turns
// over once, so no register moves), then point by point; only a shorter last
// run can fall out of step, in its last few points.  Each point takes the
// same update from the same operands as in the strided loop.
// tsh: log2 of the block size when that is a power of two, else -1.
template <typename R, int EQ, int STAGE>
__device__ __forceinline__ R run_point(const R (&v)[2 * Shape<EQ>::RAD + 1], const R* dst, int q,
                                       const Coefs<R>& c)
{
    if constexpr (EQ == HEAT) {
        return heat_point(v[0], v[1], v[2], c.fo);
    } else {
        const R base = STAGE == 0 ? v[2] : dst[q];
        return ks_point(v[0], v[1], v[2], v[3], v[4], base, c.a1[STAGE], c.a4[STAGE], c.beta[STAGE],
                        c.gam[STAGE]);
    }
}

template <typename R, int EQ, int STAGE>
__device__ __forceinline__ void level_runs(const R* src, R* dst, int lo, int cnt, int tsh, const Coefs<R>& c)
{
    constexpr int RAD = Shape<EQ>::RAD, U = 2 * RAD + 1;
    const int T = blockDim.x, m = cnt + T - 1;
    const int len = (tsh >= 0 ? m >> tsh : m / T) | 1;
    int q = lo + (int)threadIdx.x * len;
    const int end = min(q + len, lo + cnt);
    if (q >= end) return;
    R v[U];
#pragma unroll
    for (int k = 0; k < U - 1; ++k) v[k] = src[q - RAD + k];
    for (; q + U <= end; q += U) {
        // the block's loads first (the rows may alias as far as the compiler knows)
        R nv[U], base[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            nv[u] = src[q + u + RAD];
            base[u] = STAGE == 1 ? dst[q + u] : R(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[U - 1] = nv[u];
            if constexpr (EQ == HEAT)
                dst[q + u] = heat_point(v[0], v[1], v[2], c.fo);
            else
                dst[q + u] = ks_point(v[0], v[1], v[2], v[3], v[4], STAGE == 0 ? v[2] : base[u], c.a1[STAGE],
                                      c.a4[STAGE], c.beta[STAGE], c.gam[STAGE]);
#pragma unroll
            for (int k = 0; k < U - 1; ++k) v[k] = v[k + 1];
        }
    }
    for (; q < end; ++q) {
        v[U - 1] = src[q + RAD];
        dst[q] = run_point<R, EQ, STAGE>(v, dst, q, c);
#pragma unroll
        for (int k = 0; k < U - 1; ++k) v[k] = v[k + 1];
    }
}

// Advance levels j_lo..j_hi of one tile of nk points in shared memory.
//   row0 / row1 : [NV][W] even / odd level rows, W = nk + 2 rad
//   P, G        : Euler scratch, W pressures, [3][W + 1] + 3 interface values, 14 ghost values,
//                 [3][W] cached cell values (euler_cell)
//   wall        : the node may evaluate points next to a non-periodic end
//   RUNS        : FP32 heat / KS levels sweep contiguous runs (level_runs)
template <typename R, int EQ, bool RUNS>
__device__ __forceinline__ void tile_levels(R* row0, R* row1, R* P, R* G, int nk, int H, int j_lo,
                                            int j_hi, int64_t g0, int64_t N, bool wall, int bc,
                                            const Coefs<R>& c)
{
    constexpr int RAD = Shape<EQ>::RAD;
    const int W = window_width(nk, RAD);
    const int T = blockDim.x;
    const int tsh = (T & (T - 1)) == 0 ? __ffs(T) - 1 : -1;
    for (int j = j_lo; j <= j_hi; ++j) {
        // level j on slots [rad (1 + |j - H|), rad + nk - rad |j - H|): for a
        // tile of n = 2 rad H points, the 2 rad min(j, 2H - j) points around
        // its centre
        const int a = RAD * (j <= H ? H - j : j - H);
        const int lo = RAD + a, cnt = nk - 2 * a;
        R* dst = (j & 1) ? row1 : row0;
        const R* src = (j & 1) ? row0 : row1;
        const int stage = (EQ == HEAT) ? 0 : ((j & 1) ? 0 : 1);
        if constexpr (EQ == HEAT) {
            if (RUNS && sizeof(R) == 4 && !wall) {
                level_runs<R, EQ, 0>(src, dst, lo, cnt, tsh, c);
                __syncthreads();
                continue;
            }
            for (int t = threadIdx.x; t < cnt; t += T) {
                const int q = lo + t;
                R tm, tp;
                if (wall) {
                    tm = wall_fetch(src, W, q, -1, 0, g0, N, bc, c);
                    tp = wall_fetch(src, W, q, 1, 0, g0, N, bc, c);
                } else {
                    tm = src[q - 1];
                    tp = src[q + 1];
                }
                dst[q] = heat_point(tm, src[q], tp, c.fo);
            }
        } else if constexpr (EQ == KS) {
            // KS problems are periodic: the window is already wrapped.  (The
            // stage picks by value: c may be a copy in registers.)
            if constexpr (RUNS && sizeof(R) == 4) {
                if (stage) level_runs<R, EQ, 1>(src, dst, lo, cnt, tsh, c);
                else level_runs<R, EQ, 0>(src, dst, lo, cnt, tsh, c);
                __syncthreads();
                continue;
            }
            const R a1 = stage ? c.a1[1] : c.a1[0], a4 = stage ? c.a4[1] : c.a4[0];
            const R beta = stage ? c.beta[1] : c.beta[0], gam = stage ? c.gam[1] : c.gam[0];
            for (int t = threadIdx.x; t < cnt; t += T) {
                const int q = lo + t;
                const R base = stage == 0 ? src[q] : row0[q];
                dst[q] = ks_point(src[q - 2], src[q - 1], src[q], src[q + 1], src[q + 2], base, a1,
                                  a4, beta, gam);
            }
        } else {
            const R kh = c.kh[stage];
            // pressures (and the cell values euler_cell caches) of cells
            // [lo-2, hi+2), interfaces [lo, hi], then cells
            const int GW = W + 1;
            R* Gx = G + 3 * GW;   // wall nodes: the interface between cell N-1 and the right ghost
            // ghost states, variable v of the left / right end at Gh[2v] /
            // Gh[2v + 1], their pressures at Gh[6] / Gh[7] and their cached
            // (u, e, sqrt(rho)) at Gh[8 + 2k] / Gh[9 + 2k]
            R* Gh = Gx + 3;
            R* Cc = Gh + 14;      // cached (u, e, sqrt(rho)) of slot s at Cc[k W + s]
            // Slots wrap modulo N; next to a Dirichlet end s0 is the slot of
            // cell 0 (W when the window does not wrap), so slots below s0 hold
            // cells ..., N-2, N-1.  Periodic ends: no slot is special.
            int s0 = INT_MIN / 2;
            if (wall) {
                const int64_t w0 = wrap(-g0, N);
                s0 = w0 < W ? (int)w0 : W;
            }
            if (wall && threadIdx.x < 2) {
                const R* gs = threadIdx.x ? c.ghost_r : c.ghost_l;
                Gh[threadIdx.x] = gs[0];
                Gh[2 + threadIdx.x] = gs[1];
                Gh[4 + threadIdx.x] = gs[2];
                Gh[6 + threadIdx.x] = euler_cell(gs[0], gs[1], gs[2], c.gm1, Gh[8 + threadIdx.x],
                                                 Gh[10 + threadIdx.x], Gh[12 + threadIdx.x]);
            }
            for (int t = threadIdx.x; t < cnt + 4; t += T) {
                const int s = lo - 2 + t;
                P[s] = euler_cell(src[s], src[W + s], src[2 * W + s], c.gm1, Cc[s], Cc[W + s], Cc[2 * W + s]);
            }
            __syncthreads();
            for (int t = threadIdx.x; t <= cnt; t += T) {
                const int sb = lo + t;   // interface between slots sb-1 and sb
                // Where cell 0 sits at slot sb == s0, the slot boundary stands
                // for two interfaces: -1 | 0 (in G) and N-1 | N (in Gx).
                const int reps = sb == s0 ? 2 : 1;
                for (int rep = 0; rep < reps; ++rep) {
                    // interface among cells 0, 1, ... (slots >= s0) or among
                    // ..., N-2, N-1 (slots < s0); a stencil cell on the other
                    // side of s0 is the ghost state of that end
                    const bool left_end = rep == 0 && sb >= s0;
                    R q[2][3], p[4], cc[2][3];
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int s = sb + d - 2;
                        const bool lg = left_end && s < s0, rg = !left_end && s >= s0;
                        const bool gh = lg || rg;
                        const R* cell = gh ? Gh + (rg ? 1 : 0) : src + s;
                        const R* cache = gh ? Gh + 8 + (rg ? 1 : 0) : Cc + s;
                        const int vs = gh ? 2 : W;
                        p[d] = gh ? Gh[6 + (rg ? 1 : 0)] : P[s];
                        if (d == 1 || d == 2) {
#pragma unroll
                            for (int v = 0; v < 3; ++v) {
                                q[d - 1][v] = cell[v * vs];
                                cc[d - 1][v] = cache[v * vs];
                            }
                        }
                    }
                    R g3[3];
                    euler_interface_cached(q[0], q[1], p[0], p[1], p[2], p[3], cc[0], cc[1], c.gm1, c.ggm1, g3);
                    R* o = rep ? Gx : G + sb;
                    const int os = rep ? 1 : GW;
                    o[0] = g3[0];
                    o[os] = g3[1];
                    o[2 * os] = g3[2];
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < cnt; t += T) {
                const int q = lo + t;
                const bool last = q == s0 - 1;   // cell N-1: right interface in Gx
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const R base = stage == 0 ? src[v * W + q] : row0[v * W + q];
                    const R gp = last ? Gx[v] : G[v * GW + q + 1];
                    dst[v * W + q] = euler_update(gp, G[v * GW + q], base, kh);
                }
            }
        }
        __syncthreads();
    }
}

// One level of the register-blocked form (below), of parity ODD: odd levels
// hold predictor values (KS stage 0, base = the source value), even levels the
// heat step or the KS final values (stage 1, base = the level-j-2 value of the
// same slot, i.e. the destination register before it is overwritten).
template <typename R, int EQ, int P, bool ODD>
__device__ __forceinline__ void reg_level(const R (&src)[P], R (&dst)[P], R* xb, const R (&hl)[Shape<EQ>::RAD],
                                          const R (&hr)[Shape<EQ>::RAD], int j, int H, int cs, int s0,
                                          const Coefs<R>& c)
{
    constexpr int RAD = Shape<EQ>::RAD;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int w = RAD * (j <= H ? j : 2 * H - j);
    const int lo = cs - w, hi = cs + w;   // slots of level j
    // source values of the RAD slots left and right of this thread's range
    R L[RAD], Rt[RAD];
#pragma unroll
    for (int k = 0; k < RAD; ++k) {
        L[k] = __shfl_up_sync(0xffffffffu, src[P - RAD + k], 1);
        Rt[k] = __shfl_down_sync(0xffffffffu, src[k], 1);
    }
    R* x = xb + (ODD ? 2 * 32 * RAD : 0);   // [warp][first | last][RAD]
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < RAD; ++k) x[(2 * warp) * RAD + k] = src[k];
    }
    if (lane == 31) {
#pragma unroll
        for (int k = 0; k < RAD; ++k) x[(2 * warp + 1) * RAD + k] = src[P - RAD + k];
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < RAD; ++k) L[k] = warp > 0 ? x[(2 * warp - 1) * RAD + k] : hl[k];
    }
    if (lane == 31) {
#pragma unroll
        for (int k = 0; k < RAD; ++k) Rt[k] = warp < nw - 1 ? x[(2 * warp + 2) * RAD + k] : hr[k];
    }
    if (s0 + P <= lo || s0 >= hi) return;   // no slot of this thread on level j
    constexpr int stage = ODD ? 0 : 1;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        // stencil value at local index i + d
        auto at = [&](int d) -> R {
            const int q = i + d;
            return q < 0 ? L[RAD + q] : (q >= P ? Rt[q - P] : src[q]);
        };
        R v;
        if constexpr (EQ == HEAT) {
            v = heat_point(at(-1), at(0), at(1), c.fo);
        } else {
            const R base = ODD ? src[i] : dst[i];
            v = ks_point(at(-2), at(-1), at(0), at(1), at(2), base, c.a1[stage], c.a4[stage], c.beta[stage],
                         c.gam[stage]);
        }
        const int q = s0 + i;
        dst[i] = (q >= lo && q < hi) ? v : dst[i];
    }
}

// Register-blocked levels j_lo..j_hi (heat and KS nodes that do not touch a
// non-periodic end; blockDim.x * P == n).  Thread t keeps slots rad + tP ..
// rad + tP + P - 1 of both rows in registers; stencil neighbours come from
// the adjacent lanes by warp shuffle and, at warp edges, through the exchange
// buffer xb (one barrier per level).  The same point updates in the same
// order as tile_levels, so the bits are the same; the rows go back to shared
// memory at the end.  j_lo is always odd (H + 1 or 1, H even).
template <typename R, int EQ, int P>
__device__ __forceinline__ void tile_levels_reg(R* row0, R* row1, R* xb, int n, int H, int j_lo, int j_hi,
                                                const Coefs<R>& c)
{
    constexpr int RAD = Shape<EQ>::RAD;
    static_assert(P >= RAD, "a thread must own at least rad slots");
    const int cs = n / 2 + RAD;
    const int s0 = RAD + threadIdx.x * P;
    R r0[P], r1[P], hl[RAD], hr[RAD];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        r0[i] = row0[s0 + i];
        r1[i] = row1[s0 + i];
    }
    // row 1's window halo, read by the widest level (j = H, even: its source is row 1)
#pragma unroll
    for (int k = 0; k < RAD; ++k) {
        hl[k] = row1[k];
        hr[k] = row1[n + RAD + k];
    }
    for (int j = j_lo; j <= j_hi; j += 2) {
        reg_level<R, EQ, P, true>(r0, r1, xb, hl, hr, j, H, cs, s0, c);
        if (j + 1 <= j_hi) reg_level<R, EQ, P, false>(r1, r0, xb, hl, hr, j + 1, H, cs, s0, c);
    }
#pragma unroll
    for (int i = 0; i < P; ++i) {
        row0[s0 + i] = r0[i];
        row1[s0 + i] = r1[i];
    }
    __syncthreads();
}

// Exchange buffer of the register-blocked levels: per level parity, per warp
// (at most 32), the first and the last rad values of the warp's source row.
template <int EQ>
constexpr int kExchangeElems = 2 * 32 * 2 * Shape<EQ>::RAD;

template <int EQ>
__host__ __device__ __forceinline__ size_t smem_elems(int n)
{
    constexpr int RAD = Shape<EQ>::RAD, NV = Shape<EQ>::NV;
    const size_t W = (size_t)window_width(n, RAD);
    size_t e = 2 * NV * W;
    if (EQ == EULER) e += W + 3 * (W + 1) + 17 + 3 * W;   // P, G, Gx, Gh, cached cell values
    else e += kExchangeElems<EQ>;   // warp-edge exchange of the register-blocked levels
    return e;
}

template <typename R, int EQ>
__device__ __forceinline__ void smem_rows(unsigned char* raw, int n, R*& row0, R*& row1, R*& P,
                                          R*& G)
{
    constexpr int RAD = Shape<EQ>::RAD, NV = Shape<EQ>::NV;
    const int W = window_width(n, RAD);
    R* sm = reinterpret_cast<R*>(raw);
    row0 = sm;
    row1 = sm + NV * W;
    P = row1 + NV * W;
    G = P + W;
}

// Which nodes may evaluate a point next to a non-periodic domain end: the
// node centred on x = 0 and the first / last node of a phase.
__device__ __forceinline__ bool node_near_wall(int bc, int k, int K)
{
    return bc != PERIODIC && (k == 0 || k == K - 1);
}

// Levels j_lo..j_hi of one tile of nk points (nodes of n).  PR > 0:
// register-blocked with PR slots per thread (heat and KS tiles of n points
// away from non-periodic ends; blockDim.x * PR == n, the host picks it);
// otherwise in shared memory.
template <typename R, int EQ, int PR>
__device__ __forceinline__ void run_levels(R* row0, R* row1, R* P, R* G, int n, int nk, int H, int j_lo,
                                           int j_hi, int64_t g0, int64_t N, bool wall, int bc, const Coefs<R>& c)
{
    if constexpr (PR > 0 && EQ != EULER) {
        if (!wall && nk == n) {
            tile_levels_reg<R, EQ, PR>(row0, row1, P, n, H, j_lo, j_hi, c);
            return;
        }
    }
    // (tiles of the register-blocked kernels that fall back here, wider or
    // next to a wall, keep the strided loop: fewer registers for the kernel)
    tile_levels<R, EQ, PR == 0>(row0, row1, P, G, nk, H, j_lo, j_hi, g0, N, wall, bc, c);
}

template <typename R, int EQ, int PR>
__global__ void __launch_bounds__(EQ == EULER ? 256 : 1024) swept_phase_kernel(R* A, R* B, PhaseGeom g, int bc,
                                                           Coefs<R> c)
{
    constexpr int RAD = Shape<EQ>::RAD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = blockIdx.x;
    int64_t g0;
    int nk;
    tile_window(k, g.odd, g.n, g.K, g.d, RAD, g0, nk);
    R *row0, *row1, *P, *G;
    smem_rows<R, EQ>(smem_raw, nk, row0, row1, P, G);
    const bool need_b = g.j_lo <= g.H;   // every phase but the first reads odd-level edges
    window_load<R, EQ, false>(A, B, row0, row1, nk, g0, g.N, need_b);
    __syncthreads();
    run_levels<R, EQ, PR>(row0, row1, P, G, g.n, nk, g.H, g.j_lo, g.j_hi, g0, g.N,
                          node_near_wall(bc, k, g.K), bc, c);
    window_store<R, EQ, false>(A, B, row0, row1, nk, g0, g.N);
}

// ---------------------------------------------------------------------------
// Flags between the items of a persistent (dataflow) launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int* p)
{
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Hard cap on polls of one wait, in case the global timer does not advance.
constexpr uint32_t kMaxPolls = 1u << 26;

// ---------------------------------------------------------------------------
// Persistent dataflow form: one launch runs every phase of one or many
// problems (a single problem's SWP_LAUNCH_PERSISTENT advance is a batch of
// one).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One (instance, node, phase) item of a batch.  REG: heat / KS nodes away
// from non-periodic ends run register-blocked at n / blockDim.x slots per
// thread when that is 2, 4, 8 (or, FP32, 16), else in shared memory.
template <typename R, int EQ, bool REG>
__device__ __forceinline__ void batch_item(const BatchInst<R>& in, int k, int64_t p,
                                           unsigned char* smem_raw)
{
    constexpr int RAD = Shape<EQ>::RAD;
    const int H = in.H, n = in.n;
    const int odd = (int)(p & 1);
    const int j_lo = p == 0 ? H + 1 : 1;
    // even phases of a partition with wider nodes also compute level 2H (the
    // wider nodes' middle points)
    const int j_hi = p < in.Q ? 2 * H - 1 + (!odd && in.d ? 1 : 0) : (p == in.Q ? H + (int)in.r : (int)in.r);
    int64_t g0;
    int nk;
    tile_window(k, odd, n, in.K, in.d, RAD, g0, nk);
    R *row0, *row1, *P, *G;
    smem_rows<R, EQ>(smem_raw, nk, row0, row1, P, G);
    window_load<R, EQ, true>(in.A, in.B, row0, row1, nk, g0, in.N, j_lo <= H);
    // heat / KS: the point-update coefficients in registers for all levels,
    // rather than re-read from the instance table after every level barrier
    Coefs<R> cr{};
    if constexpr (EQ != EULER) {
        cr.fo = in.c.fo;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            cr.a1[s] = in.c.a1[s];
            cr.a4[s] = in.c.a4[s];
            cr.beta[s] = in.c.beta[s];
            cr.gam[s] = in.c.gam[s];
        }
    }
    const Coefs<R>& c = EQ != EULER ? cr : in.c;
    __syncthreads();
    bool done = false;
    if constexpr (REG && EQ != EULER) {
        // (the launch is register-blocked when some instance's nodes split
        // evenly over the block; this instance's may not)
        done = !node_near_wall(in.bc, k, in.K) && nk == n && n % (int)blockDim.x == 0;
        if (done) switch (n / (int)blockDim.x) {
        case 2: tile_levels_reg<R, EQ, 2>(row0, row1, P, n, H, j_lo, j_hi, c); break;
        case 4: tile_levels_reg<R, EQ, 4>(row0, row1, P, n, H, j_lo, j_hi, c); break;
        case 8: tile_levels_reg<R, EQ, 8>(row0, row1, P, n, H, j_lo, j_hi, c); break;
        case 16:
            if constexpr (sizeof(R) == 4) {
                tile_levels_reg<R, EQ, 16>(row0, row1, P, n, H, j_lo, j_hi, c);
                break;
            }
            done = false;
            break;
        default: done = false; break;
        }
    }
    if (!done)
        run_levels<R, EQ, 0>(row0, row1, P, G, n, nk, H, j_lo, j_hi, g0, in.N, node_near_wall(in.bc, k, in.K),
                             in.bc, c);
    window_store<R, EQ, true>(in.A, in.B, row0, row1, nk, g0, in.N);
}

// Value of variable v at global point g (within rad of [0, N)) of a [NV][N]
// row, through the boundary condition; read past L1, since other blocks of
// the launch write the rows.
template <typename R>
__device__ __forceinline__ R row_bc_load(const R* row, int64_t g, int64_t N, int bc, int v, const Coefs<R>& c)
{
    if (g < 0 || g >= N) {
        if (bc == DIRICHLET) return g < 0 ? c.ghost_l[v] : c.ghost_r[v];
        if (bc == PERIODIC) g = g < 0 ? g + N : g - N;
        else g = g < 0 ? -g : 2 * (N - 1) - g;
    }
    return __ldcg(row + v * N + g);
}

// One (instance, chunk, sub-step) item of a classic instance (Section 5.1:
// one sub-timestep over the whole grid, here over chunk k of the balanced
// partition of [0, N) into K chunks).  Even sub-steps read row A, odd ones
// row B: heat alternates A -> B -> A; KS and Euler run the predictor A -> B
// and the final step B -> A in place, with base values from A.
template <typename R, int EQ>
__device__ __forceinline__ void classic_item(const BatchInst<R>& in, int k, int64_t p, unsigned char* smem_raw)
{
    constexpr int RAD = Shape<EQ>::RAD, NV = Shape<EQ>::NV;
    const int64_t N = in.N;
    // chunk k is [floor(kN/K), floor((k+1)N/K)), with kN split so that it
    // cannot overflow (N < 2^35, K < 2^30)
    const int64_t q = N / in.K, rem = N % in.K;
    const int64_t x0 = (int64_t)k * q + (int64_t)k * rem / in.K;
    const int64_t x1 = (int64_t)(k + 1) * q + (int64_t)(k + 1) * rem / in.K;
    const int cnt = (int)(x1 - x0);
    const int W = cnt + 2 * RAD;
    R* sm = reinterpret_cast<R*>(smem_raw);   // [NV][W]: the chunk and its halo
    const bool even = (p & 1) == 0;
    const R* src = even ? in.A : in.B;
    R* dst = even ? in.B : in.A;
    const int stage = even ? 0 : 1;
    const int T = blockDim.x;
    for (int s = threadIdx.x; s < W; s += T) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sm[v * W + s] = row_bc_load(src, x0 - RAD + s, N, in.bc, v, in.c);
    }
    __syncthreads();
    if constexpr (EQ == HEAT) {
        for (int l = threadIdx.x; l < cnt; l += T)
            __stcg(dst + x0 + l, heat_point(sm[l], sm[l + 1], sm[l + 2], in.c.fo));
    } else if constexpr (EQ == KS) {
        const R a1 = in.c.a1[stage], a4 = in.c.a4[stage], beta = in.c.beta[stage], gam = in.c.gam[stage];
        for (int l = threadIdx.x; l < cnt; l += T) {
            const int q = RAD + l;
            const R base = stage == 0 ? sm[q] : __ldcg(in.A + x0 + l);
            __stcg(dst + x0 + l, ks_point(sm[q - 2], sm[q - 1], sm[q], sm[q + 1], sm[q + 2], base, a1, a4, beta, gam));
        }
    } else {
        R* P = sm + NV * W;   // pressure of every staged cell
        R* G = P + W;         // G[v][l]: interface between chunk cells l-1 and l
        const int GW = cnt + 1;
        R* Cc = G + 3 * GW;   // cached (u, e, sqrt(rho)) of staged cell s at Cc[k W + s]
        for (int s = threadIdx.x; s < W; s += T)
            P[s] = euler_cell(sm[s], sm[W + s], sm[2 * W + s], in.c.gm1, Cc[s], Cc[W + s], Cc[2 * W + s]);
        __syncthreads();
        for (int l = threadIdx.x; l <= cnt; l += T) {
            const int sb = RAD + l;
            const R qa[3] = {sm[sb - 1], sm[W + sb - 1], sm[2 * W + sb - 1]};
            const R qb[3] = {sm[sb], sm[W + sb], sm[2 * W + sb]};
            const R ca[3] = {Cc[sb - 1], Cc[W + sb - 1], Cc[2 * W + sb - 1]};
            const R cb[3] = {Cc[sb], Cc[W + sb], Cc[2 * W + sb]};
            R g3[3];
            euler_interface_cached(qa, qb, P[sb - 2], P[sb - 1], P[sb], P[sb + 1], ca, cb, in.c.gm1, in.c.ggm1, g3);
            G[l] = g3[0];
            G[GW + l] = g3[1];
            G[2 * GW + l] = g3[2];
        }
        __syncthreads();
        const R kh = in.c.kh[stage];
        for (int l = threadIdx.x; l < cnt; l += T) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const R base = stage == 0 ? sm[v * W + RAD + l] : __ldcg(in.A + v * N + x0 + l);
                __stcg(dst + v * N + x0 + l, euler_update(G[v * GW + l + 1], G[v * GW + l], base, kh));
            }
        }
    }
}

// MODE HEAT: heat and KS instances (chosen per item); MODE EULER: Euler.
// CLS: the launch holds classic instances too (their items are compiled in
// only then, so that swept-only launches keep fewer registers: Euler 80
// against 63 without).
template <typename R, int MODE, bool REG, bool CLS>
__global__ void __launch_bounds__(MODE == EULER ? 256 : 1024) swept_batch_kernel(const BatchInst<R>* insts,
                                                                                BatchWork w)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int task_s, node_s, abort_s;
    for (;;) {
        if (threadIdx.x == 0) {
            // claim the next node of the first task with unclaimed nodes
            int t = ld_relaxed(w.cur_task), k = -1;
            while (t < w.ntasks) {
                const int K = insts[w.tasks[t].x].K;
                k = atomicAdd(w.task_ctr + t, 1);
                if (k < K) break;
                atomicCAS(w.cur_task, t, t + 1);
                t = ld_relaxed(w.cur_task);
            }
            task_s = t;
            node_s = k;
            abort_s = 0;
        }
        __syncthreads();
        const int t = task_s;
        if (t >= w.ntasks) break;
        const int2 tk = w.tasks[t];
        const BatchInst<R>& in = insts[tk.x];
        const int64_t p = tk.y;
        const int k = node_s, K = in.K;
        if (p > in.phase_lo && threadIdx.x == 0) {
            // items of the previous phase this one reads: swept, the two
            // overlapping nodes; classic, the chunk and its neighbours
            int kl, km, kr;
            if (!CLS || in.kind == BATCH_SWEPT) {
                const int odd = (int)(p & 1);
                kl = odd ? (k + K - 1) % K : k;
                kr = odd ? k : (k + 1) % K;
                km = kl;
            } else {
                const bool per = in.bc == PERIODIC;
                kl = k > 0 ? k - 1 : (per ? K - 1 : k);
                km = k;
                kr = k < K - 1 ? k + 1 : (per ? 0 : k);
            }
            const uint32_t need = (uint32_t)(p - in.phase_lo) + w.wait_offset;
            const uint32_t* f = w.flags + in.flag_off;
            const uint64_t t_start = global_ns();
            uint32_t polls = 0, backoff = 32;
            while (ld_acquire(f + kl) < need || ld_acquire(f + kr) < need || ld_acquire(f + km) < need) {
                if (ld_volatile(w.status) != 0 || ++polls > kMaxPolls ||
                    global_ns() - t_start > w.wait_limit_ns) {
                    atomicExch(w.status, 1);
                    abort_s = 1;
                    break;
                }
                __nanosleep(backoff);
                if (backoff < 1024) backoff *= 2;
            }
        }
        __syncthreads();
        if (abort_s) break;
        if (!CLS || in.kind == BATCH_SWEPT) {
            if constexpr (MODE == EULER) batch_item<R, EULER, false>(in, k, p, smem_raw);
            else if (in.eq == HEAT) batch_item<R, HEAT, REG>(in, k, p, smem_raw);
            else batch_item<R, KS, REG>(in, k, p, smem_raw);
        } else if constexpr (CLS) {
            if constexpr (MODE == EULER) classic_item<R, EULER>(in, k, p, smem_raw);
            else if (in.eq == HEAT) classic_item<R, HEAT>(in, k, p, smem_raw);
            else classic_item<R, KS>(in, k, p, smem_raw);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(w.flags + in.flag_off + k, (uint32_t)(p - in.phase_lo) + 1);
    }
}

template <typename R, int EQ>
cudaError_t set_smem(const void* fn, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Slots per thread of the register-blocked levels for node width n and
// block size threads, or 0 for the shared-memory levels.
// FP32 only: in FP64 the FP64 pipe bounds both forms, and the register-blocked
// kernel's larger register file cost (fewer resident nodes) made it slower.
template <typename R, int EQ>
int reg_slots(int n, int threads)
{
    if (EQ == EULER || sizeof(R) != 4 || threads <= 0 || n % threads) return 0;
    const int p = n / threads;
    return (p == 2 || p == 4 || p == 8 || (p == 16 && sizeof(R) == 4)) ? p : 0;
}

template <typename R, int EQ, int PR>
cudaError_t phase_launch_pr(int bc, R* A, R* B, const PhaseGeom& g, const Coefs<R>& c, int threads,
                            cudaStream_t s)
{
    const size_t smem = sizeof(R) * smem_elems<EQ>(g.n + (g.d + g.K - 1) / g.K);   // the widest node
    cudaError_t e = set_smem<R, EQ>((const void*)swept_phase_kernel<R, EQ, PR>, smem);
    if (e != cudaSuccess) return e;
    swept_phase_kernel<R, EQ, PR><<<g.K, threads, smem, s>>>(A, B, g, bc, c);
    return cudaGetLastError();
}

template <typename R, int EQ>
cudaError_t phase_launch_eq(int bc, R* A, R* B, const PhaseGeom& g, const Coefs<R>& c, int threads,
                            cudaStream_t s)
{
    if constexpr (EQ != EULER) {
        switch (reg_slots<R, EQ>(g.n, threads)) {
        case 2: return phase_launch_pr<R, EQ, 2>(bc, A, B, g, c, threads, s);
        case 4: return phase_launch_pr<R, EQ, 4>(bc, A, B, g, c, threads, s);
        case 8: return phase_launch_pr<R, EQ, 8>(bc, A, B, g, c, threads, s);
        case 16:
            if constexpr (sizeof(R) == 4) return phase_launch_pr<R, EQ, 16>(bc, A, B, g, c, threads, s);
            break;
        default: break;
        }
    }
    return phase_launch_pr<R, EQ, 0>(bc, A, B, g, c, threads, s);
}

template <typename R, int MODE, bool REG, bool CLS>
cudaError_t batch_launch_mode(const BatchInst<R>* insts, const BatchWork& w, int threads, int blocks,
                              cudaStream_t s)
{
    cudaError_t e = set_smem<R, MODE>((const void*)swept_batch_kernel<R, MODE, REG, CLS>, w.smem_bytes);
    if (e != cudaSuccess) return e;
    swept_batch_kernel<R, MODE, REG, CLS><<<blocks, threads, w.smem_bytes, s>>>(insts, w);
    return cudaGetLastError();
}

template <typename R, int MODE, bool REG, bool CLS>
int batch_bps_mode(size_t smem, int threads)
{
    if (set_smem<R, MODE>((const void*)swept_batch_kernel<R, MODE, REG, CLS>, smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, swept_batch_kernel<R, MODE, REG, CLS>, threads, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

}  // namespace

size_t batch_classic_smem_bytes(int eq, int m, int elem_bytes)
{
    const size_t rad = eq == HEAT ? 1 : 2, nv = eq == EULER ? 3 : 1;
    const size_t W = (size_t)m + 2 * rad;
    size_t e = nv * W;
    if (eq == EULER) e += W + 3 * ((size_t)m + 1) + 3 * W;   // P, G, cached cell values
    return (size_t)elem_bytes * e;
}

size_t swept_smem_bytes(int eq, int n, int elem_bytes)
{
    switch (eq) {
    case HEAT: return (size_t)elem_bytes * smem_elems<HEAT>(n);
    case KS: return (size_t)elem_bytes * smem_elems<KS>(n);
    default: return (size_t)elem_bytes * smem_elems<EULER>(n);
    }
}

template <typename R>
cudaError_t launch_swept_phase(int eq, int bc, R* A, R* B, const PhaseGeom& g, const Coefs<R>& c,
                               int threads, cudaStream_t s)
{
    switch (eq) {
    case HEAT: return phase_launch_eq<R, HEAT>(bc, A, B, g, c, threads, s);
    case KS: return phase_launch_eq<R, KS>(bc, A, B, g, c, threads, s);
    default: return phase_launch_eq<R, EULER>(bc, A, B, g, c, threads, s);
    }
}


template cudaError_t launch_swept_phase<double>(int, int, double*, double*, const PhaseGeom&,
                                                const Coefs<double>&, int, cudaStream_t);
template cudaError_t launch_swept_phase<float>(int, int, float*, float*, const PhaseGeom&,
                                               const Coefs<float>&, int, cudaStream_t);
template <typename R>
cudaError_t launch_swept_batch(int mode, bool reg, bool cls, const BatchInst<R>* insts, const BatchWork& w,
                               int threads, int blocks, cudaStream_t s)
{
    if (mode == EULER)
        return cls ? batch_launch_mode<R, EULER, false, true>(insts, w, threads, blocks, s)
                   : batch_launch_mode<R, EULER, false, false>(insts, w, threads, blocks, s);
    if (reg)
        return cls ? batch_launch_mode<R, HEAT, true, true>(insts, w, threads, blocks, s)
                   : batch_launch_mode<R, HEAT, true, false>(insts, w, threads, blocks, s);
    return cls ? batch_launch_mode<R, HEAT, false, true>(insts, w, threads, blocks, s)
               : batch_launch_mode<R, HEAT, false, false>(insts, w, threads, blocks, s);
}

template <typename R>
int swept_batch_blocks_per_sm(int mode, bool reg, bool cls, size_t smem_bytes, int threads)
{
    if (mode == EULER)
        return cls ? batch_bps_mode<R, EULER, false, true>(smem_bytes, threads)
                   : batch_bps_mode<R, EULER, false, false>(smem_bytes, threads);
    if (reg)
        return cls ? batch_bps_mode<R, HEAT, true, true>(smem_bytes, threads)
                   : batch_bps_mode<R, HEAT, true, false>(smem_bytes, threads);
    return cls ? batch_bps_mode<R, HEAT, false, true>(smem_bytes, threads)
               : batch_bps_mode<R, HEAT, false, false>(smem_bytes, threads);
}

int swept_reg_slots(int eq, int n, int threads, int elem_bytes)
{
    if (eq == EULER) return 0;
    if (elem_bytes == 4) return eq == HEAT ? reg_slots<float, HEAT>(n, threads) : reg_slots<float, KS>(n, threads);
    return eq == HEAT ? reg_slots<double, HEAT>(n, threads) : reg_slots<double, KS>(n, threads);
}

template cudaError_t launch_swept_batch<double>(int, bool, bool, const BatchInst<double>*, const BatchWork&,
                                                int, int, cudaStream_t);
template cudaError_t launch_swept_batch<float>(int, bool, bool, const BatchInst<float>*, const BatchWork&, int,
                                               int, cudaStream_t);
template int swept_batch_blocks_per_sm<double>(int, bool, bool, size_t, int);
template int swept_batch_blocks_per_sm<float>(int, bool, bool, size_t, int);

}  // namespace swp
