/*
 * CPU oracle for the swept time-space decomposition of Magee & Niemeyer,
 * "Accelerating solutions of one-dimensional unsteady PDEs with GPU-based
 * swept time-space decomposition" (arXiv:1705.03162).
 *
 * TEST INFRASTRUCTURE.  This is a plain, slow, single-threaded restatement of
 * the paper's schemes, used only by the tests, the package smoke check and the
 * benchmark's CPU-baseline leg to check and time the CUDA library.  The
 * product path never calls it and shares no code with it.
 *
 * Contents (all in the precision the caller selects, FP64 or FP32):
 *  - classic decomposition (Section 5.1): one sub-timestep at a time over the
 *    whole grid, double-buffered;
 *  - swept decomposition restated on the CPU (Sections 4.2-4.3): nodes,
 *    upright triangles, diamonds, edge arrays passed between nodes, closing
 *    triangle;
 *  - schemes: heat FTCS (Appendix A), Kuramoto-Sivashinsky with central
 *    differences and midpoint RK2 (Appendix B), Euler equations with the
 *    limited second-order finite-volume scheme and RK2 (Appendix C);
 *  - boundary conditions: periodic, reflective (insulated, Appendix A) and
 *    Dirichlet ghost cells (Appendix C).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off (no contraction of a*b+c into FMA:
 * every FMA is written out), no fast-math, -lm; the same source with
 * -fopenmp is the all-core build, whose classic loops split each
 * sub-timestep's points over threads (the bits do not change).
 */
#include "oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* FP64 instantiation */
#define REAL double
#define SFX(x) x##_f64
#define FMA fma
#define SQRT sqrt
#define FABS fabs
#include "scheme.inc"
#undef REAL
#undef SFX
#undef FMA
#undef SQRT
#undef FABS

/* FP32 instantiation */
#define REAL float
#define SFX(x) x##_f32
#define FMA fmaf
#define SQRT sqrtf
#define FABS fabsf
#include "scheme.inc"
#undef REAL
#undef SFX
#undef FMA
#undef SQRT
#undef FABS

static int check_problem(const orc_problem* pb)
{
    if (!pb || pb->n_points <= 0) return ORC_EINVAL;
    if (pb->eq < ORC_HEAT || pb->eq > ORC_EULER) return ORC_EINVAL;
    if (pb->bc < ORC_BC_PERIODIC || pb->bc > ORC_BC_DIRICHLET) return ORC_EINVAL;
    if (!(pb->dx > 0) || !(pb->dt > 0)) return ORC_EINVAL;
    int rad = pb->eq == ORC_HEAT ? 1 : 2;
    if (pb->n_points < 2 * rad + 1) return ORC_EINVAL;
    /* the paper's pairings: heat periodic/reflective, KS periodic, Euler
     * Dirichlet (periodic also allowed for Euler) */
    if (pb->eq == ORC_HEAT && pb->bc == ORC_BC_DIRICHLET) return ORC_EUNSUPPORTED;
    if (pb->eq == ORC_KS && pb->bc != ORC_BC_PERIODIC) return ORC_EUNSUPPORTED;
    if (pb->eq == ORC_EULER && pb->bc == ORC_BC_REFLECTIVE) return ORC_EUNSUPPORTED;
    return ORC_OK;
}

/* Threads of the classic loops in the OpenMP build (built with -fopenmp);
 * the serial build ignores the request.  Returns the count in use. */
int orc_set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* Advance `state` (nv x N, SoA, in place) by `steps` timesteps with the
 * classic decomposition. */
int orc_classic(const orc_problem* pb, int32_t dtype, void* state, int64_t steps)
{
    int e = check_problem(pb);
    if (e) return e;
    if (!state || steps < 0) return ORC_EINVAL;
    if (dtype == ORC_F64) return classic_f64(pb, (double*)state, steps);
    if (dtype == ORC_F32) return classic_f32(pb, (float*)state, steps);
    return ORC_EINVAL;
}

/* Advance `state` by `steps` timesteps with the swept decomposition, nodes of
 * n points (N % n == 0, n / (2 rad) even). */
int orc_swept(const orc_problem* pb, int32_t dtype, void* state, int64_t steps, int64_t n)
{
    int e = check_problem(pb);
    if (e) return e;
    if (!state || steps < 0) return ORC_EINVAL;
    if (dtype == ORC_F64) return swept_f64(pb, (double*)state, steps, n);
    if (dtype == ORC_F32) return swept_f32(pb, (float*)state, steps, n);
    return ORC_EINVAL;
}

/* The swept geometry the oracle runs, for the pins against the paper's
 * figures: out = (H, W, Q, r, kernels, timesteps per triangle). */
int orc_swept_geometry(int32_t eq, int64_t n, int64_t steps, int64_t* out)
{
    if (!out || eq < ORC_HEAT || eq > ORC_EULER) return ORC_EINVAL;
    orc_geometry g;
    int e = swept_geometry(eq == ORC_HEAT ? 1 : 2, eq == ORC_HEAT ? 1 : 2, n, steps, &g);
    if (e) return e;
    out[0] = g.H;
    out[1] = g.W;
    out[2] = g.Q;
    out[3] = g.r;
    out[4] = g.kernels;
    out[5] = g.triangle_steps;
    return ORC_OK;
}

/* One sub-timestep at one point (FP64), as the classic scheme evaluates it:
 * the problem's coefficients (formed as for a whole run) and the point update
 * of stage `stage` (0 predictor, 1 final; heat has only stage 0).
 *   st   : the 2 rad + 1 stencil values, point-major (nv values per point)
 *   base : nv values of the point at the start of the timestep (KS / Euler)
 *   out  : nv values
 * For the pins that compare one stage with the paper's formula in exact
 * arithmetic. */
int orc_stage_f64(const orc_problem* pb, int32_t stage, const double* st, const double* base, double* out)
{
    int e = check_problem(pb);
    if (e) return e;
    if (!st || !base || !out || stage < 0 || stage > 1) return ORC_EINVAL;
    coefs_f64 c;
    make_coefs_f64(pb, &c);
    point_update_f64(&c, stage, st, base, out);
    return ORC_OK;
}

/* Pieces of the Euler scheme, exposed for the pins that check them on
 * hand-worked states (FP64).  q: conserved (rho, rho u, E) triples. */
double orc_euler_pressure_f64(const double* q, double gamma)
{
    return euler_pressure_f64(q[0], q[1], q[2], gamma - 1.0, NULL, NULL);
}

/* q: 4 cells (a-1, a, b, b+1) x 3; outputs the reconstructed left and right
 * states at the interface between a and b. */
int orc_euler_reconstruct_f64(const double* q, double gamma, double* ql, double* qr)
{
    double gm1 = gamma - 1.0, p[4];
    for (int k = 0; k < 4; ++k) p[k] = euler_pressure_f64(q[3 * k], q[3 * k + 1], q[3 * k + 2], gm1, NULL, NULL);
    euler_reconstruct_f64(q + 3, q + 6, p[0], p[1], p[2], p[3], ql, qr);
    return ORC_OK;
}

/* G = 2 Flux at the interface between cells a and b of the 4 cells q. */
int orc_euler_interface_f64(const double* q, double gamma, double* G)
{
    double gm1 = gamma - 1.0, ggm1 = gamma * (gamma - 1.0);
    double p[4];
    for (int k = 0; k < 4; ++k) p[k] = euler_pressure_f64(q[3 * k], q[3 * k + 1], q[3 * k + 2], gm1, NULL, NULL);
    euler_interface_f64(q + 3, q + 6, p[0], p[1], p[2], p[3], gm1, ggm1, G);
    return ORC_OK;
}
