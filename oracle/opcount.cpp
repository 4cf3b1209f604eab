/*
 * Operation-counting build of the CPU oracle (TEST INFRASTRUCTURE, like
 * swept_oracle.c; the CUDA library never uses it).
 *
 * scheme.inc is compiled a third time, with REAL = Counted: a double that
 * counts every floating-point operation done on it (additions and
 * subtractions, multiplications, fused multiply-adds, divisions, square
 * roots).  Comparisons, absolute values and copies are not counted.  Running
 * the oracle's classic scheme on a problem then counts, exactly, the
 * operations of its point updates as written in scheme.inc, and the pieces of
 * the Euler update (pressure, interface, cell update) are counted alone, so
 * that the algorithmic count of one cell sub-step (one pressure per cell, one
 * interface per interface) can be told apart from the plain oracle's (which
 * evaluates each interface twice and each pressure five times).
 *
 * Build: g++ -O1 -std=c++17 -ffp-contract=off -shared -fPIC.
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

extern "C" {
#include "oracle.h"
}

namespace {

struct OpCounts {
    long long add, mul, fma, div, sqrt;
};
OpCounts g_ops;

struct Counted {
    double v;
    Counted() = default;
    Counted(double x) : v(x) {}
};

inline Counted operator+(Counted a, Counted b) { ++g_ops.add; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_ops.add; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { ++g_ops.mul; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_ops.div; return Counted(a.v / b.v); }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<(Counted a, int b) { return a.v < b; }
inline bool operator>(Counted a, int b) { return a.v > b; }
inline Counted cnt_fma(Counted a, Counted b, Counted c) { ++g_ops.fma; return Counted(std::fma(a.v, b.v, c.v)); }
inline Counted cnt_sqrt(Counted a) { ++g_ops.sqrt; return Counted(std::sqrt(a.v)); }
inline Counted cnt_fabs(Counted a) { return Counted(std::fabs(a.v)); }

#define REAL Counted
#define SFX(x) x##_cnt
#define FMA cnt_fma
#define SQRT cnt_sqrt
#define FABS cnt_fabs
#include "scheme.inc"
#undef REAL
#undef SFX
#undef FMA
#undef SQRT
#undef FABS

void take(long long* out)
{
    out[0] = g_ops.add;
    out[1] = g_ops.mul;
    out[2] = g_ops.fma;
    out[3] = g_ops.div;
    out[4] = g_ops.sqrt;
    std::memset(&g_ops, 0, sizeof(g_ops));
}

}  // namespace

extern "C" {

/* Count the operations of `steps` classic timesteps of the problem from the
 * FP64 state (nv x N, not modified).  out[0..4]: additions (and
 * subtractions), multiplications, FMAs, divisions, square roots. */
int orc_opcount_classic(const orc_problem* pb, const double* state, int64_t steps, long long* out)
{
    if (!pb || !state || !out || steps < 0 || pb->n_points <= 4) return ORC_EINVAL;
    const int nv = pb->eq == ORC_EULER ? 3 : 1;
    const size_t count = (size_t)nv * (size_t)pb->n_points;
    Counted* u = (Counted*)std::malloc(sizeof(Counted) * count);
    if (!u) return ORC_ENOMEM;
    for (size_t i = 0; i < count; ++i) u[i] = Counted(state[i]);
    std::memset(&g_ops, 0, sizeof(g_ops));
    const int e = classic_cnt(pb, u, steps);
    take(out);
    std::free(u);
    return e;
}

/* Operations of one Euler pressure evaluation (Eq. EulerP). */
int orc_opcount_euler_pressure(long long* out)
{
    if (!out) return ORC_EINVAL;
    std::memset(&g_ops, 0, sizeof(g_ops));
    Counted u, ir;
    euler_pressure_cnt(Counted(1.0), Counted(0.5), Counted(2.5), Counted(0.4), &u, &ir);
    take(out);
    return ORC_OK;
}

/* Operations of one Euler cell update at the five cells q (5 x 3,
 * conserved) with base values base: out_point counts the whole update as the
 * oracle evaluates it (five pressures, two interfaces, the cell update);
 * out_interfaces the two interface evaluations alone, done again on the same
 * cells.  The cell update's own share is out_point - 5 pressures -
 * out_interfaces. */
int orc_opcount_euler_point(const double* q, const double* base, double gamma, double kh, long long* out_point,
                            long long* out_interfaces)
{
    if (!q || !base || !out_point || !out_interfaces) return ORC_EINVAL;
    Counted qc[15], bc[3], o[3], p[5], gm[3], gp[3];
    for (int i = 0; i < 15; ++i) qc[i] = Counted(q[i]);
    for (int i = 0; i < 3; ++i) bc[i] = Counted(base[i]);
    const Counted gm1(gamma - 1.0), ggm1(gamma * (gamma - 1.0));
    for (int k = 0; k < 5; ++k)
        p[k] = euler_pressure_cnt(qc[3 * k], qc[3 * k + 1], qc[3 * k + 2], gm1, NULL, NULL);
    std::memset(&g_ops, 0, sizeof(g_ops));
    euler_point_cnt(qc, bc, Counted(kh), gm1, ggm1, o);
    take(out_point);
    euler_interface_cnt(qc + 3, qc + 6, p[0], p[1], p[2], p[3], gm1, ggm1, gm);
    euler_interface_cnt(qc + 6, qc + 9, p[1], p[2], p[3], p[4], gm1, ggm1, gp);
    take(out_interfaces);
    return ORC_OK;
}

}  // extern "C"
