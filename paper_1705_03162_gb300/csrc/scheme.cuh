// Point updates of the three test problems (arXiv:1705.03162, Appendices
// A-C), shared by the classic and the swept kernels so that both produce the
// same bits.  Every operation is an explicit round-to-nearest intrinsic, so
// the compiler neither contracts nor reorders: the rounding sequence is the
// one written here.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace swp {

enum Eq : int { HEAT = 0, KS = 1, EULER = 2 };
enum Bc : int { PERIODIC = 0, REFLECTIVE = 1, DIRICHLET = 2 };

// Round-to-nearest arithmetic in the working precision.
template <typename R> struct Fp;
template <> struct Fp<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
    static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double abs(double a) { return fabs(a); }
};
template <> struct Fp<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
    static __device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
};

// Per-problem constants, formed on the host in double and rounded once to R.
template <typename R> struct Coefs {
    R fo;                 // heat: Fourier number alpha dt / dx^2
    R a1[2], a4[2], beta[2], gam[2];  // KS stage s (0 predictor h = dt/2, 1 final h = dt):
                          // a1 = -h/(4dx), a4 = -h/dx^4, beta = a2 - 4 a4,
                          // gam = 6 a4 - 2 a2, a2 = -h/dx^2
    R kh[2];              // Euler stage s: -(h/dx)/2 (G below is twice the flux)
    R gm1, ggm1;          // gamma - 1, gamma (gamma - 1)
    R ghost_l[3], ghost_r[3];  // Dirichlet end states, conserved
};

// ---------------------------------------------------------------------------
// Heat, FTCS (Appendix A, Eq. heatdisc):
//   T' = Fo (T_{i+1} + T_{i-1}) + (1 - 2 Fo) T_i = T_i + Fo (T_{i+1} - 2 T_i + T_{i-1})
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R heat_point(R tm, R t0, R tp, R fo)
{
    using F = Fp<R>;
    R lap = F::fma(R(-2), t0, F::add(tp, tm));
    return F::fma(fo, lap, t0);
}

// ---------------------------------------------------------------------------
// Kuramoto-Sivashinsky, one midpoint-RK2 stage (Appendix B, Eqs. KSDisc, RKm,
// RKf): out = base + h f(v), base = u^m, h = dt/2 (predictor) or dt (final).
// The Laplacian (1, -2, 1)/dx^2 and the fourth difference (1, -4, 6, -4, 1)/dx^4
// combine into one five-point stencil with weights a4 (v++, v--),
// beta = a2 - 4 a4 (v+, v-) and gam = 6 a4 - 2 a2 (v); the nonlinear term
// a1 (v+^2 - v-^2) = a1 (v+ - v-)(v+ + v-) shares the factor v+ + v-, so
//   h f = gam v + a4 (v++ + v--) + (beta + a1 (v+ - v-)) (v+ + v-),
// with a1 = -h/(4dx), a2 = -h/dx^2, a4 = -h/dx^4.  Seven FP operations; the
// dependent chain is three deep.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R ks_point(R vmm, R vm, R v0, R vp, R vpp, R base,
                                      R a1, R a4, R beta, R gam)
{
    using F = Fp<R>;
    const R t = F::fma(a1, F::sub(vp, vm), beta);
    R acc = F::fma(gam, v0, base);
    acc = F::fma(a4, F::add(vpp, vmm), acc);
    return F::fma(t, F::add(vp, vm), acc);
}

// ---------------------------------------------------------------------------
// Euler (Appendix C).  Conserved Q = (rho, rho u, E), E total energy per volume.
// ---------------------------------------------------------------------------

// Velocity and pressure, Eq. EulerP: u = (rho u)/rho, P = (gamma-1)(E - (rho u) u / 2),
// dividing by rho as a multiplication by the correctly rounded 1/rho (ir).
template <typename R>
__device__ __forceinline__ R euler_pressure(R r, R m, R E, R gm1, R& u, R& ir)
{
    using F = Fp<R>;
    ir = F::rcp(r);
    u = F::mul(m, ir);
    return F::mul(gm1, F::fma(F::mul(R(-0.5), m), u, E));
}

template <typename R>
__device__ __forceinline__ R euler_pressure(R r, R m, R E, R gm1)
{
    R u, ir;
    return euler_pressure(r, m, E, gm1, u, ir);
}

// Sign and magnitude tests on the IEEE bit patterns (integer pipe; GB300's
// FP64 pipe would spend a full slot on each comparison).  Equal to the
// floating-point comparisons for every non-NaN value.
__device__ __forceinline__ uint64_t fbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ uint32_t fbits(float x) { return (uint32_t)__float_as_uint(x); }

// (a > 0 && b > 0) || (a < 0 && b < 0): both nonzero, equal sign bits
template <typename R>
__device__ __forceinline__ bool same_sign(R a, R b)
{
    const auto ua = fbits(a), ub = fbits(b);
    constexpr int top = 8 * sizeof(R) - 1;
    return (ua << 1) != 0 && (ub << 1) != 0 && ((ua ^ ub) >> top) == 0;
}

// min(num/den, 1) for num, den nonzero with the same sign.  When
// |num| >= |den| the quotient rounds to >= 1, so the division is skipped.
template <typename R>
__device__ __forceinline__ R limited_ratio(R num, R den)
{
    const auto mag = ~(decltype(fbits(num)))0 >> 1;
    return (fbits(num) & mag) >= (fbits(den) & mag) ? R(1) : Fp<R>::div(num, den);
}

// Limited states at the interface between cells a (left) and b (right)
// (Eqs. Pratio, limitleft, limitright): the ratio at cell a is
// (pb - pa)/(pa - pam) and gives QL = Qa + min(ratio, 1)/2 (Qb - Qa) when it
// lies in (0, inf); the inverse ratio at cell b, (pb - pa)/(pbp - pb), gives
// QR = Qb + min(inverse, 1)/2 (Qa - Qb); otherwise first order.
// lfirst / rfirst: the side was left first order (a copy of its cell).
template <typename R>
__device__ __forceinline__ void euler_reconstruct(const R qa[3], const R qb[3], R pam, R pa,
                                                  R pb, R pbp, R ql[3], R qr[3], bool& lfirst, bool& rfirst)
{
    using F = Fp<R>;
    R num = F::sub(pb, pa), den = F::sub(pa, pam);
    lfirst = !same_sign(num, den);
    if (!lfirst) {
        R h = F::mul(R(0.5), limited_ratio(num, den));
#pragma unroll
        for (int c = 0; c < 3; ++c) ql[c] = F::fma(h, F::sub(qb[c], qa[c]), qa[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) ql[c] = qa[c];
    }
    R num2 = F::sub(pbp, pb);
    rfirst = !same_sign(num2, num);
    if (!rfirst) {
        R h = F::mul(R(0.5), limited_ratio(num, num2));
#pragma unroll
        for (int c = 0; c < 3; ++c) qr[c] = F::fma(h, F::sub(qa[c], qb[c]), qb[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) qr[c] = qb[c];
    }
}

template <typename R>
__device__ __forceinline__ void euler_reconstruct(const R qa[3], const R qb[3], R pam, R pa,
                                                  R pb, R pbp, R ql[3], R qr[3])
{
    bool lfirst, rfirst;
    euler_reconstruct(qa, qb, pam, pa, pb, pbp, ql, qr, lfirst, rfirst);
}

// G = 2 Flux from the limited states: F(QR) + F(QL) + r_sp (QL - QR), with
// F(Q) = (rho u, rho u^2 + P, u (E + P)) (Eq. EulerF) and spectral radius
// r_sp = sqrt(gamma (gamma-1) (e_sp - u_sp^2/2)) + |u_sp| from sqrt(rho)-weighted
// Roe averages of u and of e = E/rho (gamma P_sp / rho_sp with
// P_sp = (gamma-1) rho_sp (e_sp - u_sp^2/2)).  Divisions by rho and by the
// weight sum are multiplications by correctly rounded reciprocals.
template <typename R>
__device__ __forceinline__ void euler_flux(const R ql[3], const R qr[3], R gm1, R ggm1, R G[3])
{
    using F = Fp<R>;
    R ul, ur, irl, irr;
    R pl = euler_pressure(ql[0], ql[1], ql[2], gm1, ul, irl);
    R pr = euler_pressure(qr[0], qr[1], qr[2], gm1, ur, irr);
    R fl1 = F::fma(ql[1], ul, pl);
    R fl2 = F::mul(ul, F::add(ql[2], pl));
    R fr1 = F::fma(qr[1], ur, pr);
    R fr2 = F::mul(ur, F::add(qr[2], pr));
    R sl = F::sqrt(ql[0]);
    R sr = F::sqrt(qr[0]);
    R iw = F::rcp(F::add(sl, sr));
    R usp = F::mul(F::fma(sl, ul, F::mul(sr, ur)), iw);
    R el = F::mul(ql[2], irl);
    R er = F::mul(qr[2], irr);
    R esp = F::mul(F::fma(sl, el, F::mul(sr, er)), iw);
    R c2 = F::mul(ggm1, F::fma(F::mul(R(-0.5), usp), usp, esp));
    R rsp = F::add(F::sqrt(c2), F::abs(usp));
    G[0] = F::fma(rsp, F::sub(ql[0], qr[0]), F::add(qr[1], ql[1]));
    G[1] = F::fma(rsp, F::sub(ql[1], qr[1]), F::add(fr1, fl1));
    G[2] = F::fma(rsp, F::sub(ql[2], qr[2]), F::add(fr2, fl2));
}

// Interface value from the four cells around it and their pressures.
template <typename R>
__device__ __forceinline__ void euler_interface(const R qa[3], const R qb[3], R pam, R pa, R pb,
                                                R pbp, R gm1, R ggm1, R G[3])
{
    R ql[3], qr[3];
    euler_reconstruct(qa, qb, pam, pa, pb, pbp, ql, qr);
    euler_flux(ql, qr, gm1, ggm1, G);
}

// ---------------------------------------------------------------------------
// The same interface value with per-cell values reused.  Where the limiter
// leaves a side first order (uniform regions: the pressure difference is 0),
// the side state is its cell's state, and the flux's pressure, velocity,
// specific energy e = E/rho and sqrt(rho) of that side are the cell's own.
// euler_cell forms them once per cell with exactly the operations euler_flux
// applies to a side state, so reusing them gives the same bits; a limited
// side is computed as in euler_flux.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R euler_cell(R r, R m, R E, R gm1, R& u, R& e, R& s)
{
    R ir;
    const R p = euler_pressure(r, m, E, gm1, u, ir);
    e = Fp<R>::mul(E, ir);
    s = Fp<R>::sqrt(r);
    return p;
}

// Pressure, velocity, e and sqrt(rho) of a limited side state q.
template <typename R>
__device__ __forceinline__ R euler_side(const R q[3], R gm1, R& u, R& e, R& s)
{
    return euler_cell(q[0], q[1], q[2], gm1, u, e, s);
}

// ca / cb: (u, e, sqrt(rho)) of cells a and b (as euler_cell forms them).
template <typename R>
__device__ __forceinline__ void euler_interface_cached(const R qa[3], const R qb[3], R pam, R pa, R pb,
                                                       R pbp, const R ca[3], const R cb[3], R gm1, R ggm1,
                                                       R G[3])
{
    using F = Fp<R>;
    R ql[3], qr[3];
    bool lfirst, rfirst;
    euler_reconstruct(qa, qb, pam, pa, pb, pbp, ql, qr, lfirst, rfirst);
    R pl, ul, el, sl, pr, ur, er, sr;
    if (lfirst) {
        pl = pa;
        ul = ca[0];
        el = ca[1];
        sl = ca[2];
    } else {
        pl = euler_side(ql, gm1, ul, el, sl);
    }
    if (rfirst) {
        pr = pb;
        ur = cb[0];
        er = cb[1];
        sr = cb[2];
    } else {
        pr = euler_side(qr, gm1, ur, er, sr);
    }
    R fl1 = F::fma(ql[1], ul, pl);
    R fl2 = F::mul(ul, F::add(ql[2], pl));
    R fr1 = F::fma(qr[1], ur, pr);
    R fr2 = F::mul(ur, F::add(qr[2], pr));
    R iw = F::rcp(F::add(sl, sr));
    R usp = F::mul(F::fma(sl, ul, F::mul(sr, ur)), iw);
    R esp = F::mul(F::fma(sl, el, F::mul(sr, er)), iw);
    R c2 = F::mul(ggm1, F::fma(F::mul(R(-0.5), usp), usp, esp));
    R rsp = F::add(F::sqrt(c2), F::abs(usp));
    G[0] = F::fma(rsp, F::sub(ql[0], qr[0]), F::add(qr[1], ql[1]));
    G[1] = F::fma(rsp, F::sub(ql[1], qr[1]), F::add(fr1, fl1));
    G[2] = F::fma(rsp, F::sub(ql[2], qr[2]), F::add(fr2, fl2));
}

// Finite-volume RK2 stage: out = base - (h/dx)(Flux_{i+1/2} - Flux_{i-1/2})
// = fma(kh, G_{i+1/2} - G_{i-1/2}, base).
template <typename R>
__device__ __forceinline__ R euler_update(R gp, R gm, R base, R kh)
{
    return Fp<R>::fma(kh, Fp<R>::sub(gp, gm), base);
}

}  // namespace swp
