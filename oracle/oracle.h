/*
 * Definitions shared by the CPU oracle's builds (test infrastructure only):
 * swept_oracle.c (FP64 and FP32, serial or OpenMP) and opcount.cpp (the
 * operation-counting build).  See swept_oracle.c.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EUNSUPPORTED 5

#define ORC_HEAT 0
#define ORC_KS 1
#define ORC_EULER 2

#define ORC_BC_PERIODIC 0
#define ORC_BC_REFLECTIVE 1
#define ORC_BC_DIRICHLET 2

#define ORC_F64 0
#define ORC_F32 1

/* Problem description (mirrors the fields a user gives when creating a
 * problem: equation, boundary condition, grid size, dx, dt, parameters). */
typedef struct {
    int32_t eq;
    int32_t bc;
    int64_t n_points;
    double dx;
    double dt;
    double alpha;      /* heat: thermal diffusivity */
    double gamma;      /* Euler: heat capacity ratio */
    double left[3];    /* Euler Dirichlet end states, primitive (rho, u, p) */
    double right[3];
} orc_problem;

/* Geometry of the swept plan (Sections 4.2-4.3) for nodes of n points and a
 * stencil of radius rad (sub sub-timesteps per timestep): H sub-timestep
 * levels per half-cycle, so an upright triangle of H - 1 levels above its base
 * advances H / sub timesteps; each node works in two rows of W = n + 2 rad
 * slots; `steps` timesteps take Q full half-cycles plus r remaining levels,
 * in `kernels` kernels (triangle, diamonds, closing triangle). */
typedef struct {
    int64_t H, W, Q, r, kernels, triangle_steps;
} orc_geometry;

static int swept_geometry(int rad, int sub, int64_t n, int64_t steps, orc_geometry* g)
{
    if (n <= 0 || n % (2 * rad) || steps < 0) return ORC_EINVAL;
    g->H = n / (2 * rad);
    /* H even keeps the level parity of every kernel's base level even, so the
     * predictor / final alternation and the two rows line up in every node */
    if (g->H & 1) return ORC_EINVAL;
    g->W = n + 2 * rad;
    int64_t T = steps * sub;
    g->Q = T / g->H;
    g->r = T % g->H;
    g->kernels = T == 0 ? 0 : (g->r > 0 ? g->Q + 2 : g->Q + 1);
    g->triangle_steps = g->H / sub;
    return ORC_OK;
}

#endif /* ORACLE_H */
