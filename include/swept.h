/*
 * swept.h -- C ABI of the GB300 (sm_103a) swept time-space decomposition
 * library, libswept.so.
 *
 * The library solves the paper's three explicit 1D test problems
 * (Magee & Niemeyer, arXiv:1705.03162, Section 5.2 and Appendices A-C):
 *   heat  u_t = alpha u_xx, FTCS                          (Appendix A)
 *   KS    u_t + u u_x + u_xx + u_xxxx = 0, central
 *         differences, midpoint RK2                       (Appendix B)
 *   Euler Sod shock tube, limited second-order finite
 *         volume, Rusanov flux, midpoint RK2              (Appendix C)
 * with either the classic decomposition (one kernel per sub-timestep,
 * Section 5.1) or the swept decomposition (upright triangle, diamonds, closing
 * triangle; Sections 4.2-4.3).  Both schemes evaluate every point update with
 * the same device function, so for the same problem they produce the same
 * bits.
 *
 * Conventions
 *  - Layout: the state is structure-of-arrays [nv][N] of double (SWP_F64) or
 *    float (SWP_F32), nv = 3 for Euler (rho, rho u, E), else 1.
 *  - Ownership: the library owns all device memory of a problem (allocated in
 *    swp_create, freed in swp_destroy).  Caller buffers are only read or
 *    written during the call that receives them (host buffers) or during the
 *    stream work that call enqueues (device buffers).
 *  - Streams: every call enqueues its GPU work on the problem's stream (the
 *    one given to swp_create; NULL = the legacy default stream).  Calls with a
 *    host buffer synchronise that stream before returning.
 *  - Errors: every call returns a swp_status; nothing throws across the ABI.
 *    swp_last_error() returns a thread-local description of the last error.
 *  - Threading: a problem may be used from one host thread at a time.
 */
#ifndef SWEPT_H
#define SWEPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SWP_OK = 0,
    SWP_EINVAL = 1,        /* invalid argument (null, size, node width, ...) */
    SWP_ENOMEM = 2,        /* device or host allocation failed */
    SWP_EBUDGET = 3,       /* request exceeds the caller-set memory budget */
    SWP_ECUDA = 4,         /* a CUDA runtime call failed */
    SWP_EUNSUPPORTED = 5,  /* equation / boundary / precision not supported */
    SWP_ETIMEOUT = 6,      /* a device-side bounded wait gave up */
    SWP_EDEVICE = 7        /* no usable sm_103 device */
} swp_status;

typedef enum { SWP_HEAT = 0, SWP_KS = 1, SWP_EULER = 2 } swp_equation;

/* Boundary conditions: periodic; reflective (insulated ends, mirror about the
 * end points: u_{-k} = u_k, u_{N-1+k} = u_{N-1-k}, Appendix A Eq. heatcond);
 * Dirichlet (two ghost cells per side holding the end states, Appendix C).
 * Supported pairs: heat periodic/reflective, KS periodic, Euler
 * Dirichlet/periodic. */
typedef enum { SWP_BC_PERIODIC = 0, SWP_BC_REFLECTIVE = 1, SWP_BC_DIRICHLET = 2 } swp_bc;

typedef enum { SWP_F64 = 0, SWP_F32 = 1 } swp_dtype;   /* Euler: SWP_F64 only */

/* SWP_SCHEME_AUTO: the scheme (and width) swp_autotune measured faster for
 * the problem's (equation, dtype, n_points); swept at the tuned or default
 * width when none was measured; classic when N is too small for any swept
 * node width. */
typedef enum { SWP_CLASSIC = 0, SWP_SWEPT = 1, SWP_SCHEME_AUTO = 2 } swp_scheme;

/* Problem description.
 *   n_points : N grid points (cells for Euler), N >= 5
 *   dx, dt   : grid spacing and timestep (> 0)
 *   alpha    : heat diffusivity (Fourier number alpha dt / dx^2)
 *   gamma    : Euler heat capacity ratio
 *   left, right : Euler Dirichlet end states, primitive (rho, u, p) */
typedef struct {
    int32_t eq;        /* swp_equation */
    int32_t bc;        /* swp_bc */
    int32_t dtype;     /* swp_dtype */
    int32_t reserved;  /* must be 0 */
    int64_t n_points;
    double dx;
    double dt;
    double alpha;
    double gamma;
    double left[3];
    double right[3];
} swp_desc;

/* How swp_advance_ex runs the swept scheme. */
typedef enum {
    SWP_LAUNCH_AUTO = 0,        /* library choice, from measurement, with
                                   the default width: for periodic heat and
                                   KS with N a multiple of 32, CLUSTER up to
                                   N = 2048 (FP64) or 4096 (FP32), then
                                   REGISTER up to 2^15 for FP64 heat, 2^14
                                   for FP64 KS, 2^18 for FP32 heat, 2^17 for
                                   FP32 KS;
                                   otherwise in FP64 GRAPH
                                   below 2^17 and PERSISTENT from 2^17
                                   (Euler: from 2^13), in FP32 PER_PHASE */
    SWP_LAUNCH_PER_PHASE = 1,   /* one kernel per triangle / diamond phase;
                                   nodes synchronise at kernel boundaries */
    SWP_LAUNCH_PERSISTENT = 2,  /* one dataflow kernel for the whole advance
                                   (the batched kernel with this problem
                                   alone); each node waits (bounded) on its
                                   two neighbours of the previous phase */
    SWP_LAUNCH_GRAPH = 3,       /* the per-phase (swept) or per-sub-step (classic)
                                   launches as a CUDA graph, captured on first use
                                   for (scheme, n_steps, width, threads) and
                                   replayed afterwards */
    SWP_LAUNCH_REGISTER = 4,    /* the paper's Register variant (Section 5.1):
                                   one warp per node of 32 points, levels in
                                   registers, neighbours by warp shuffle; one
                                   kernel per phase, replayed as a CUDA graph
                                   like SWP_LAUNCH_GRAPH; periodic heat and KS
                                   only (points_per_block 32 or 0) */
    SWP_LAUNCH_CLUSTER = 5      /* the Register variant's nodes on one
                                   thread-block cluster: the whole advance in
                                   one launch, the level rows in the blocks'
                                   shared memory (distributed shared memory),
                                   a cluster barrier between phases; for small
                                   periodic heat and KS problems: N a multiple
                                   of 32 with N / 32 = blocks (<= 16) x warps
                                   per block (<= 8), i.e. N <= 4096; threads =
                                   32 x warps per block (0 = the most
                                   blocks).
                                   SWP_EUNSUPPORTED when such a cluster cannot
                                   run on the device */
} swp_launch;

typedef struct {
    int32_t scheme;            /* swp_scheme */
    int32_t points_per_block;  /* swept node width n (0 = auto); classic: unused */
    int32_t launch;            /* swp_launch (classic: AUTO / PER_PHASE = stream
                                  launches, GRAPH = graph replay) */
    int32_t threads;           /* threads per block (0 = auto; multiple of 32) */
} swp_advance_opts;

/* A problem handle is used by one host thread at a time (calls on different
 * problems may run concurrently; the server's problems belong to its own
 * scheduler thread). */
typedef struct swp_problem swp_problem;

/* Create a problem on the current CUDA device and copy its initial state.
 *   desc         : problem description (copied)
 *   u0           : nv * N values of the dtype, layout [nv][N]
 *   u0_on_device : 0 = u0 is host memory, 1 = device memory
 *   cuda_stream  : cudaStream_t for all work of this problem (NULL = default)
 *   out          : receives the handle
 * Errors: SWP_EINVAL (null / bad sizes), SWP_EUNSUPPORTED (bad pairing),
 * SWP_EBUDGET (see swp_set_memory_budget), SWP_ENOMEM, SWP_EDEVICE, SWP_ECUDA. */
swp_status swp_create(const swp_desc* desc, const void* u0, int u0_on_device,
                      void* cuda_stream, swp_problem** out);

/* Replace the state by nv * N values from src (bytes = nv * N * sizeof(dtype)). */
swp_status swp_write(swp_problem* p, const void* src, size_t src_bytes, int src_on_device);

/* Advance n_steps timesteps (any n_steps >= 0) with `scheme`.
 * Swept: points_per_block = n must be a multiple of 4 * radius (radius 1 for
 * heat, 2 for KS/Euler) and leave every node's working set in shared memory.
 * N need not be a multiple of n (the paper's nodes, Section 4.2, need it):
 * the N = K n + d points form K = floor(N / n) nodes, node k starting at
 * k n + floor(k d / K), so some are wider (by at most ceil(d / K) points);
 * such a split needs K >= 2.
 * 0 picks a width (the tuned one, else a default); when N is too small for
 * any (fewer than two nodes of 4 * radius points) the advance runs the
 * classic scheme, whose result is the same.  The advance ends on a closing triangle, so
 * the state is complete afterwards (Section 4.2: output only at closing
 * triangles); a final partial half-cycle is closed exactly.
 * Asynchronous on the problem's stream.  SWP_ETIMEOUT reports a persistent
 * launch whose bounded neighbour wait gave up (the state is then invalid).
 * Each such wait gives up after 2 s of device global time, or after the
 * number of nanoseconds (1 to 10^12) in the environment variable
 * SWP_WAIT_LIMIT_NS, read once per process: raise it to run persistent
 * launches under a tool that pauses or replays kernels (a profiler's
 * multi-pass replay). */
swp_status swp_advance(swp_problem* p, int64_t n_steps, int32_t scheme, int32_t points_per_block);
swp_status swp_advance_ex(swp_problem* p, int64_t n_steps, const swp_advance_opts* opts);

/* Copy the current state (nv * N values, [nv][N]) to dst.  dst_bytes must be
 * at least nv * N * sizeof(dtype).  Host dst: synchronises the stream. */
swp_status swp_read(swp_problem* p, void* dst, size_t dst_bytes, int dst_on_device);

/* Wait for the problem's stream; reports a deferred device-side error. */
swp_status swp_synchronize(swp_problem* p);

/* Free all device memory of the problem.  NULL is accepted (no-op). */
swp_status swp_destroy(swp_problem* p);

/* Number of points N, variables nv and element size of a problem. */
swp_status swp_shape(const swp_problem* p, int64_t* n_points, int32_t* nv, int32_t* elem_bytes);

/* Kernels launched by this problem since creation (for launch accounting). */
int64_t swp_kernel_launches(const swp_problem* p);

/* Device memory a problem of this description would allocate, in bytes. */
swp_status swp_required_bytes(const swp_desc* desc, size_t* bytes);

/* Process-wide device-memory budget for swp_create (0 = unlimited): a create
 * whose allocation would push the library's live total above it fails with
 * SWP_EBUDGET. */
swp_status swp_set_memory_budget(size_t bytes);
size_t swp_memory_in_use(void);

/* ---- Batched advance (many independent problems, one launch) ----
 * Advancing many small problems one by one leaves most of the GPU idle and
 * pays a launch per phase each.  A batch advances every problem given to it
 * in one persistent launch per precision (heat and KS together, Euler in a
 * launch of its own): work is a table of (problem, phase) tasks ordered by
 * estimated start time (each problem's phases in order); each block claims
 * one item of the current task at a time and waits, bounded, for the items
 * of the problem's previous phase that it reads (the paper's kernel-boundary
 * synchronisation of Section 3, done per item instead of per grid).
 *   swept problem   : a phase is a triangle / diamond, an item one node;
 *   classic problem : a phase is one sub-timestep (Section 5.1), an item one
 *                     chunk of the balanced partition of [0, N) into
 *                     ceil(N / m) chunks of at most m points.
 * Each problem's result is bit-identical to swp_advance with the same scheme
 * (and, swept, the same node width).  The table costs 12 bytes of device
 * memory per (problem, phase) task; this workspace is not counted against
 * swp_set_memory_budget.  A batch, like its problems, is used by one host
 * thread at a time.  The paper has no batched form. */
typedef struct swp_batch swp_batch;

/* A batch runs its work on cuda_stream (NULL = legacy default stream); every
 * problem given to it must have been created with that stream. */
swp_status swp_batch_create(void* cuda_stream, swp_batch** out);

/* Advance problems[i] by n_steps[i] timesteps (swept), i < count.
 * points_per_block: per-problem node widths (any width swp_advance accepts),
 * or NULL / 0 entries for the tuned width of swp_autotune_width (else the
 * default rule; a problem too small for any node width runs as classic
 * items, with the same result).  threads: block
 * size (0 = 128 for FP64 and 32 for FP32; Euler at most 256).  Problems must be distinct.  Asynchronous;
 * SWP_ETIMEOUT surfaces at swp_batch_synchronize (wait bound as for
 * swp_advance's persistent launch, SWP_WAIT_LIMIT_NS included). */
swp_status swp_batch_advance(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps,
                             int32_t count, const int32_t* points_per_block, int32_t threads);

/* Like swp_batch_advance, with a scheme per problem and a launch form.
 *   schemes          : SWP_SWEPT, SWP_CLASSIC or SWP_SCHEME_AUTO per problem
 *                      (NULL = all SWP_SCHEME_AUTO)
 *   points_per_block : swept node width / classic chunk width m (4 <= m <= N)
 *                      per problem; NULL or 0 = the tuned width, else the
 *                      default (classic: min(N, 1024), Euler min(N, 256);
 *                      swept as for swp_batch_advance)
 *   launch           : SWP_LAUNCH_AUTO or _PERSISTENT (upload the task table
 *                      and launch), or SWP_LAUNCH_GRAPH: the launch is
 *                      captured as a CUDA graph with tables of its own on the
 *                      first advance of these problems, in their current
 *                      rows, with these plans, and replayed when the same
 *                      advance comes again (at most 8 graphs per batch, the
 *                      oldest dropped first).
 * Errors as swp_batch_advance; SWP_ENOMEM when the tables do not fit. */
swp_status swp_batch_advance_ex(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps,
                                int32_t count, const int32_t* schemes, const int32_t* points_per_block,
                                int32_t threads, int32_t launch);
swp_status swp_batch_synchronize(swp_batch* b);
swp_status swp_batch_destroy(swp_batch* b);
int64_t swp_batch_kernel_launches(const swp_batch* b);

/* Node-width autotuner.  Times batch_count copies of the problem (initial
 * state u0_host, host memory) advanced `steps` timesteps in one batch for
 * every power-of-two node width up to 1024 that fits, keeps the fastest for the
 * (equation, dtype, n_points) of desc, and returns it in best_n.  Later
 * batches use it for problems of that key.  Allocates and frees its own
 * trial problems; synchronises the device. */
swp_status swp_autotune_width(const swp_desc* desc, const void* u0_host, int32_t batch_count,
                              int64_t steps, int32_t* best_n);
/* The tuned swept width for desc's (equation, dtype, n_points), or 0 if none. */
swp_status swp_tuned_width(const swp_desc* desc, int32_t* n);

/* Scheme autotuner.  Times the swept widths as swp_autotune_width does and
 * the classic scheme in the same batched form (chunks of 256, 1024 and 4096
 * points, capped at N), keeps whichever is faster for desc's (equation,
 * dtype, n_points) and returns it: best_scheme SWP_SWEPT or SWP_CLASSIC,
 * best_n its node or chunk width.  SWP_SCHEME_AUTO advances (single or
 * batched) of problems with that key then use it.  Allocates and frees its
 * own trial problems; synchronises the device. */
swp_status swp_autotune(const swp_desc* desc, const void* u0_host, int32_t batch_count, int64_t steps,
                        int32_t* best_scheme, int32_t* best_n);
/* The tuned choice for desc's key: scheme and width (SWP_SWEPT, 0 if none). */
swp_status swp_tuned(const swp_desc* desc, int32_t* scheme, int32_t* n);

/* Node width for n_points points of equation eq from a target width:
 * n_points split into K = max(2, ceil(n_points / target)) nearly equal nodes,
 * the width a multiple of 4 rad (rad 1 for heat, 2 for KS and Euler), so that
 * the remainder (Section 4.2's nodes all have n points; here any N is split)
 * widens some nodes by at most 4 rad and no node is wider than
 * target + 4 rad.  *n = 0 when n_points has no two nodes of 4 rad points.
 * Host arithmetic only; SWP_EINVAL for an unknown eq, n_points or target <= 0,
 * or n NULL. */
swp_status swp_fit_width(int32_t eq, int64_t n_points, int32_t target, int32_t* n);

/* Node widths for a mixed batch, measured on the batch itself.  For each of
 * the n_candidates target widths, every problem's width is fitted to its N
 * (swp_fit_width; 0, the default rule, where the fitted width is not valid
 * for the problem) and problems[0..count) are advanced once by n_steps[i]
 * (swept, one persistent launch per group, block size `threads` as for
 * swp_batch_advance), timed with CUDA events on the batch's stream (the
 * span includes the host building and uploading the task tables, as a
 * plain advance would).  A problem listed twice is rejected by the advance
 * (SWP_EINVAL) after the states are saved, and put back.  The
 * fastest candidate's per-problem widths are written to widths_out[count],
 * its index to *best (may be NULL), and each candidate's milliseconds to
 * ms_out[n_candidates] (may be NULL).  The per-bucket autotuner
 * (swp_autotune_width) times copies of one problem alone; in a mixed batch
 * every block is sized for the widest node, which can change the order.
 * The problems' states are saved to a device buffer this call allocates (the
 * sum of their state sizes, not counted against swp_set_memory_budget) and
 * put back after every trial, so the call leaves them as it found them.
 * Synchronises the batch's stream.  Errors: SWP_EINVAL (NULL arguments,
 * count or n_candidates <= 0, a candidate <= 0, a problem on another stream),
 * SWP_ENOMEM (the save buffer), and those of swp_batch_advance_ex and
 * swp_batch_synchronize, after the states are put back. */
swp_status swp_batch_tune_width(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps, int32_t count,
                                const int32_t* candidates, int32_t n_candidates, int32_t threads,
                                int32_t* widths_out, float* ms_out, int32_t* best);

/* ---- Serving with continuous batching ----
 * A server owns a scheduler thread that admits solve requests as they arrive
 * (in order, while its device-memory budget and slot count allow), keeps their
 * states resident on the device, and advances all admitted requests together
 * in rounds of batched launches; requests arriving meanwhile join the next
 * round.  A round runs every request whose remaining work fits in
 * round_target_ms to its end; longer ones run in order of their remaining
 * work less the work done while they waited (shortest remaining first, aged,
 * so that none is passed indefinitely), as many as fill the GPU.  Each result
 * is bit-identical to solving the request alone.  The paper has no serving
 * layer. */
typedef struct swp_server swp_server;

typedef struct {
    size_t hbm_budget_bytes;  /* device bytes the server may hold (0 = no limit);
                                 a request needing more than all of it fails
                                 with SWP_EBUDGET */
    int32_t max_active;       /* requests admitted at once (> 0) */
    int32_t threads;          /* block size of the batched launches (0 = the batch
                                 defaults: 128 in FP64, 32 in FP32) */
    double round_target_ms;   /* GPU time aimed at per round (> 0) */
} swp_server_config;

typedef struct {
    int64_t completed, rounds, kernel_launches, pending, active;
    size_t device_bytes_in_use;
    double point_updates;     /* grid points x timesteps completed */
    double busy_span_s;       /* first submission to last completion */
} swp_server_statistics;

/* Start a server whose GPU work runs on cuda_stream of the current device. */
swp_status swp_server_create(const swp_server_config* cfg, void* cuda_stream, swp_server** out);
/* Queue a solve of n_steps (>= 1) timesteps from u0_host (copied before the
 * call returns); request_id receives its id.  Any N is served: swept at the
 * tuned or default width (wider nodes take the remainder), classic when N is
 * too small for any node width.  Thread-safe. */
swp_status swp_server_submit(swp_server* s, const swp_desc* desc, const void* u0_host, int64_t n_steps,
                             int64_t* request_id);
/* done = 1 once the request has finished (successfully or not). */
swp_status swp_server_poll(swp_server* s, int64_t request_id, int32_t* done);
/* Block until the request finishes; copy its final state to dst_host (NULL:
 * discard) and its latency (submission to completion, seconds) to latency_s.
 * Returns the request's status; the id is released. */
swp_status swp_server_wait(swp_server* s, int64_t request_id, void* dst_host, size_t dst_bytes,
                           double* latency_s);
swp_status swp_server_stats(swp_server* s, swp_server_statistics* out);
/* Finish admitted work, fail unadmitted requests, stop the thread, free all. */
swp_status swp_server_destroy(swp_server* s);

/* Fault-injection hook for tests of the persistent launch's bounded waits.
 * withhold != 0 makes every neighbour wait of later SWP_LAUNCH_PERSISTENT
 * advances of this problem wait for a flag value no node ever publishes, so
 * each wait gives up after wait_limit_ns nanoseconds (device global timer),
 * the kernel returns without computing, and the next swp_synchronize /
 * swp_read reports SWP_ETIMEOUT (the state is then invalid).  withhold = 0
 * restores normal waits; wait_limit_ns (in (0, 1e10]) bounds every wait of
 * later persistent advances either way (default 2 s).  Nothing faults, traps
 * or hangs.  The paper has no counterpart: its nodes synchronise only at
 * kernel boundaries (Section 3). */
swp_status swp_debug_withhold_flags(swp_problem* p, int withhold, int64_t wait_limit_ns);

/* Swept advance that allocates nothing.  The paper has no counterpart: it is
 * here for callers that cannot call cudaMalloc -- code whose device memory is
 * owned by a pool or arena, loops that forbid allocation once running, or
 * hosts that hand the library only pre-allocated buffers.
 *   desc             : problem description (as for swp_create)
 *   state            : DEVICE buffer of nv * N values ([nv][N], the dtype),
 *                      read as the initial state and overwritten with the
 *                      state after n_steps timesteps; owned by the caller.
 *                      The call has no size argument: the buffer must hold
 *                      exactly that many values.  A pointer that is not
 *                      device memory of the current device fails with
 *                      SWP_EINVAL.
 *   points_per_block : node width as for swp_advance (0 = auto)
 *   threads          : threads per block (0 = auto)
 *   cuda_stream      : stream for the work (NULL = legacy default stream)
 * The swept scheme's scratch (its odd-level row) is a fixed 8 MiB array built
 * into the library, so the state may hold at most 8 MiB (for example 2^20
 * FP64 points); larger states fail with SWP_EINVAL.  Every GPU that loads the
 * library holds that array until the process exits.  The first call on a
 * device looks up the array's device address (set-up, once per device, with
 * that device current), so make that first call before any stream capture.
 * That address belongs to the device's primary context: after
 * cudaDeviceReset (or anything else that destroys that context) it is stale,
 * so do not call this entry point on that device again in the process.
 * All calls share the one array, so calls whose GPU work overlaps (other
 * streams, other host threads) race and must be serialised by the caller.
 * No scratch value is read before the call writes it, so nothing needs
 * clearing between calls.  Asynchronous on cuda_stream; no synchronisation. */
swp_status swp_swept_noalloc(const swp_desc* desc, void* state, int64_t n_steps,
                             int32_t points_per_block, int32_t threads, void* cuda_stream);

const char* swp_status_str(swp_status s);
const char* swp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SWEPT_H */
