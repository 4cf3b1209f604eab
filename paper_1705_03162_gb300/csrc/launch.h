// Internal launch interface between the C-ABI layer (api.cu) and the kernel
// translation units (classic.cu, swept.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "scheme.cuh"
#include "../../include/swept.h"

struct swp_problem;
struct swp_batch;

namespace swp {

// One sub-timestep of the classic decomposition over all N points (Section
// 5.1): out = stage(src) with base values from `base` (KS / Euler).
//   heat : src -> out                       (stage ignored)
//   KS/Euler predictor (stage 0): src = base = u^m,      out = u^{m+1/2}
//   KS/Euler final     (stage 1): src = u^{m+1/2}, base = u^m, out = u^m (in place)
template <typename R>
cudaError_t launch_classic(int eq, int bc, const R* src, const R* base, R* out, int64_t N,
                           int stage, const Coefs<R>& c, int threads, cudaStream_t s);

// Geometry of one swept phase (one kernel of the paper's Sections 4.2-4.3).
struct PhaseGeom {
    int64_t N;      // points
    int n;          // node width (points per node)
    int H;          // sub-timestep levels per half-cycle, n / (2 radius)
    int K;          // nodes, floor(N / n)
    int d;          // N - K n: node k starts at k n + floor(k d / K)
    int j_lo, j_hi; // levels computed, relative to the phase's base level
    int odd;        // 1: tiles centred on node boundaries; 0: a tile per node
};

// Shared memory a swept phase kernel needs for tiles of at most n points.
size_t swept_smem_bytes(int eq, int n, int elem_bytes);

// One phase over all K nodes: every block loads its node's window of the two
// level rows A (even levels) and B (odd levels), advances levels j_lo..j_hi in
// shared memory and writes the window back.
template <typename R>
cudaError_t launch_swept_phase(int eq, int bc, R* A, R* B, const PhaseGeom& g, const Coefs<R>& c,
                               int threads, cudaStream_t s);

// Register variant of one phase (heat / KS, periodic): node width 32, one
// warp per node, levels in registers with warp-shuffle neighbours.
template <typename R>
cudaError_t launch_swept_register(int eq, R* A, R* B, const PhaseGeom& g, const Coefs<R>& c,
                                  int threads, cudaStream_t s);

// The Register variant's whole advance on one thread-block cluster of ctas
// blocks (small periodic heat / KS problems): block r keeps points
// [r portion, (r + 1) portion) of both level rows in shared memory, a warp is
// a node of 32 points, phases are separated by cluster barriers.
struct ClusterGeom {
    int64_t N;
    int H, K;             // levels per half-cycle (32-point nodes), nodes N / 32
    int64_t Q, r, n_phases;
    int portion;          // points per block, N / ctas
    int warps;            // warps of the cluster
};
template <typename R>
cudaError_t launch_swept_cluster(int eq, R* A, R* B, const ClusterGeom& g, const Coefs<R>& c, int ctas,
                                 int threads, cudaStream_t s);
// Clusters of this shape that fit on the device at once (0: it cannot run).
template <typename R>
int swept_cluster_fits(int eq, const ClusterGeom& g, int ctas, int threads);

// ---------------------------------------------------------------------------
// Batched advance: many independent problems of one precision in one
// persistent launch (heat and KS together; Euler in its own launch).  Work is
// a table of (instance, phase) tasks, each instance's phases in order; a block
// claims one item (node or chunk) of the current task at a time, so items are
// claimed in dependency order, and waits (bounded) for the items of the
// instance's previous phase that it reads.  A swept instance's phase is a
// triangle / diamond over nodes of n points; a classic instance's phase is
// one sub-timestep over K chunks (the balanced partition of [0, N)).
// ---------------------------------------------------------------------------
enum BatchKind : int { BATCH_SWEPT = 0, BATCH_CLASSIC = 1 };

template <typename R> struct BatchInst {
    R* A;                 // swept: even-level row; classic: the state u ([nv][N])
    R* B;                 // swept: odd-level row; classic: the other row
    int64_t N;
    int n, H, K, bc;      // classic: n = widest chunk, H unused, K chunks
    int d;                // swept: N - K n (wider nodes, see PhaseGeom); classic: 0
    int64_t Q, r, n_phases;  // classic: n_phases = sub-timesteps, Q = r = 0
    int64_t phase_lo;     // first phase of this launch (the earlier ones ran in earlier launches)
    int flag_off;         // first flag of this instance
    int eq;               // HEAT or KS (heat / KS launch), EULER
    int kind;             // BatchKind
    Coefs<R> c;
};

// Shared memory of a classic batch item over a chunk of m points.
size_t batch_classic_smem_bytes(int eq, int m, int elem_bytes);

struct BatchWork {
    const int2* tasks;    // (instance, phase), each instance's phases in order
    int* task_ctr;        // nodes claimed per task (zeroed per launch)
    int* cur_task;        // first task with unclaimed nodes (zeroed per launch)
    int ntasks;
    size_t smem_bytes;    // dynamic shared memory of the launch (widest node)
    uint32_t* flags;      // phases completed in this launch per (instance, node or chunk), zeroed per launch
    int* status;          // != 0: a wait gave up
    uint64_t wait_limit_ns;
    uint32_t wait_offset; // 0; a test hook sets it so that no wait can succeed
};

// mode: HEAT for a heat / KS launch, EULER for an Euler launch.  reg: the
// heat / KS launch runs its nodes' levels register-blocked where
// swept_reg_slots allows (nodes next to non-periodic ends stay in shared
// memory).  cls: the launch holds classic instances (else the kernel is the
// one compiled without them).
template <typename R>
cudaError_t launch_swept_batch(int mode, bool reg, bool cls, const BatchInst<R>* insts, const BatchWork& w,
                               int threads, int blocks, cudaStream_t s);

template <typename R>
int swept_batch_blocks_per_sm(int mode, bool reg, bool cls, size_t smem_bytes, int threads);

// Slots per thread of the register-blocked swept levels for node width n and
// block size threads (2, 4, 8 or, FP32, 16), or 0 when the levels run in
// shared memory (Euler, or n not split that way).
int swept_reg_slots(int eq, int n, int threads, int elem_bytes);

// Open advances in pieces (the serving loop): a range runs phases
// [p_lo, p_hi) of the plan for `steps` timesteps: swept at node width n, or
// (kind BATCH_CLASSIC, for N too small for any node width) classic in chunks
// of n points, a phase per sub-timestep.  Between pieces the problem's two
// rows hold the open state (triangle edges, or the predictor row); it is
// complete, and bit-identical to one swp_advance of `steps` with that scheme,
// after the plan's last phase has run.  All pieces of one problem use the
// same (kind, steps, n) and run in order on the batch's stream.
struct PhaseRange {
    swp_problem* p;
    int n;
    int64_t steps;
    int64_t p_lo, p_hi;
    int kind;   // BatchKind
};
int swept_width(const swp_problem* p);    // the tuned or default dataflow node width (0: none)
int classic_chunk(const swp_problem* p);  // the default classic chunk width
int64_t phase_count(const swp_problem* p, int64_t steps, int kind, int n);
swp_status batch_advance_phases(swp_batch* b, const PhaseRange* ranges, int count, int threads);
// The same for one problem, as per-phase launches on its own stream.
swp_status advance_phases(swp_problem* p, int n, int64_t steps, int64_t p_lo, int64_t p_hi);

}  // namespace swp
