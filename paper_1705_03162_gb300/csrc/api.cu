// C ABI of libswept.so (declared in include/swept.h).  Host-side driver of the
// classic (one launch per sub-timestep, arXiv:1705.03162 Section 5.1) and the
// swept (triangle / diamond / closing phases, Sections 4.2-4.3) schemes.
// Built with host FP contraction off so the coefficients below round exactly
// as written.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "../../include/swept.h"
#include "launch.h"

using namespace swp;

struct swp_problem {
    swp_desc desc;
    uint64_t id = 0;   // unique per created problem (keys of cached batch graphs)
    int nv = 1, rad = 1, sub = 1, esize = 8;
    int64_t N = 0;
    void* rows[2] = {nullptr, nullptr};   // level rows / classic ping-pong, [nv][N] each
    int cur = 0;                          // which row holds the state
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 0;
    int64_t launches = 0;
    size_t bytes = 0;
    Coefs<double> cd{};
    Coefs<float> cf{};
    // persistent swept launch: a batch of this one problem (the dataflow
    // kernel), with its own status word for bounded-wait failures
    swp_batch* batch = nullptr;
    int* status = nullptr;
    int inject_withheld_flags = 0;            // test hook: waits never succeed
    uint64_t wait_limit_ns = 2000000000ull;   // bound of one neighbour wait
    // CUDA graphs of launch sequences (SWP_LAUNCH_GRAPH), replayed on `stream`
    struct Graph {
        int scheme, n, threads, cur_before, cur_after;
        int64_t steps;
        int64_t kernels;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    cudaStream_t capture_stream = nullptr;
};

namespace {

thread_local std::string g_last_error;
std::atomic<size_t> g_in_use{0};
std::atomic<size_t> g_budget{0};
std::atomic<uint64_t> g_next_id{1};

swp_status fail(swp_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

swp_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(SWP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Bound of one neighbour wait of a persistent launch: 2 s, or the value of
// SWP_WAIT_LIMIT_NS (nanoseconds, 1 .. 10^12; read once), for tools that
// pause or replay kernels (a profiler's multi-pass replay stretches waits).
uint64_t default_wait_limit_ns()
{
    static const uint64_t v = [] {
        const char* s = std::getenv("SWP_WAIT_LIMIT_NS");
        if (!s || !*s) return (uint64_t)2000000000ull;
        char* end = nullptr;
        const unsigned long long x = std::strtoull(s, &end, 10);
        if (*end != '\0' || x == 0 || x > 1000000000000ull) return (uint64_t)2000000000ull;
        return (uint64_t)x;
    }();
    return v;
}

int radius_of(int eq) { return eq == SWP_HEAT ? 1 : 2; }
int nv_of(int eq) { return eq == SWP_EULER ? 3 : 1; }
int esize_of(int dtype) { return dtype == SWP_F32 ? 4 : 8; }

swp_status check_desc(const swp_desc* d)
{
    if (!d) return fail(SWP_EINVAL, "desc is NULL");
    if (d->eq < SWP_HEAT || d->eq > SWP_EULER) return fail(SWP_EINVAL, "unknown equation %d", d->eq);
    if (d->bc < SWP_BC_PERIODIC || d->bc > SWP_BC_DIRICHLET)
        return fail(SWP_EINVAL, "unknown boundary condition %d", d->bc);
    if (d->dtype != SWP_F64 && d->dtype != SWP_F32) return fail(SWP_EINVAL, "unknown dtype %d", d->dtype);
    if (d->reserved != 0) return fail(SWP_EINVAL, "reserved field must be 0");
    if (d->n_points < 5) return fail(SWP_EINVAL, "n_points must be >= 5 (got %lld)", (long long)d->n_points);
    if (d->n_points > (int64_t)1 << 34) return fail(SWP_EINVAL, "n_points too large");
    if (!(d->dx > 0) || !(d->dt > 0) || !std::isfinite(d->dx) || !std::isfinite(d->dt))
        return fail(SWP_EINVAL, "dx and dt must be finite and > 0");
    if (d->eq == SWP_HEAT && d->bc == SWP_BC_DIRICHLET)
        return fail(SWP_EUNSUPPORTED, "heat supports periodic and reflective ends");
    if (d->eq == SWP_KS && d->bc != SWP_BC_PERIODIC)
        return fail(SWP_EUNSUPPORTED, "KS supports periodic ends");
    if (d->eq == SWP_EULER && d->bc == SWP_BC_REFLECTIVE)
        return fail(SWP_EUNSUPPORTED, "Euler supports Dirichlet and periodic ends");
    if (d->eq == SWP_EULER && d->dtype != SWP_F64)
        return fail(SWP_EUNSUPPORTED, "Euler runs in FP64 only");
    if (d->eq == SWP_HEAT && !std::isfinite(d->alpha)) return fail(SWP_EINVAL, "alpha must be finite");
    if (d->eq == SWP_EULER && !(d->gamma > 1.0)) return fail(SWP_EINVAL, "gamma must be > 1");
    return SWP_OK;
}

size_t state_bytes(const swp_desc* d) { return (size_t)nv_of(d->eq) * d->n_points * esize_of(d->dtype); }

// Coefficients of the point updates, formed in double and rounded once.
template <typename R>
void make_coefs(const swp_desc* d, Coefs<R>& c)
{
    std::memset(&c, 0, sizeof(c));
    const double fo = d->alpha * d->dt / (d->dx * d->dx);
    c.fo = (R)fo;
    for (int s = 0; s < 2; ++s) {
        const double h = s == 0 ? 0.5 * d->dt : d->dt;
        const double c1 = 1.0 / (4.0 * d->dx);
        const double c2 = 1.0 / (d->dx * d->dx);
        const double c4 = c2 * c2;
        const double a1 = -(h * c1), a2 = -(h * c2), a4 = -(h * c4);
        c.a1[s] = (R)a1;
        c.a4[s] = (R)a4;
        c.beta[s] = (R)(a2 - 4.0 * a4);
        c.gam[s] = (R)(6.0 * a4 - 2.0 * a2);
        const double lam = d->dt / d->dx;
        const double lamh = s == 0 ? 0.5 * lam : lam;
        c.kh[s] = (R)(-(0.5 * lamh));
    }
    const double g = d->gamma;
    c.gm1 = (R)(g - 1.0);
    c.ggm1 = (R)(g * (g - 1.0));
    const double* st[2] = {d->left, d->right};
    R* gh[2] = {c.ghost_l, c.ghost_r};
    for (int s = 0; s < 2; ++s) {
        const double r = st[s][0], u = st[s][1], p = st[s][2];
        gh[s][0] = (R)r;
        gh[s][1] = (R)(r * u);
        gh[s][2] = (R)(p / (g - 1.0) + 0.5 * r * u * u);
    }
}

// Largest shared memory a block may use on this device.
size_t max_smem(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return (size_t)v;
}

// Widest tile of nodes of n points over N: K = floor(N / n) nodes, the
// remainder d = N - K n spread over them (node k starts at k n + floor(k d / K)).
int64_t widest_node(int64_t N, int n)
{
    const int64_t K = N / n, d = N - K * n;
    return K > 0 ? n + (d + K - 1) / K : 0;
}

// A swept node width must be a multiple of 4 rad (so that H is even), give at
// least one node (two when it does not divide N: the wider nodes' tiles then
// never meet themselves across the periodic wrap) and fit the widest node's
// working set in shared memory.  It need not divide N: the remainder widens
// some nodes.
swp_status check_width(const swp_problem* p, int n)
{
    const int step = 4 * p->rad;
    if (n < step || n % step) return fail(SWP_EINVAL, "points_per_block %d must be a positive multiple of %d", n, step);
    const int64_t K = p->N / n, d = p->N % n;
    if (K < 1) return fail(SWP_EINVAL, "points_per_block %d exceeds n_points %lld", n, (long long)p->N);
    if (d != 0 && K < 2)
        return fail(SWP_EINVAL, "points_per_block %d leaves one node for n_points %lld, which it does not divide", n,
                    (long long)p->N);
    if (K > 0x7FFFFFFF) return fail(SWP_EINVAL, "points_per_block %d gives more than 2^31 - 1 nodes", n);
    const int64_t wide = widest_node(p->N, n);
    if (wide > (1 << 20) || swept_smem_bytes(p->desc.eq, (int)wide, p->esize) > max_smem(p->device))
        return fail(SWP_EINVAL, "points_per_block %d (widest node %lld) needs more shared memory than a block has", n,
                    (long long)wide);
    return SWP_OK;
}

// Default node width, from the widths measured fastest on GB300 for single
// problems: about N / 512 in the persistent dataflow launch, and otherwise
// N / 1024 points for heat and KS in FP64, N / 128 in FP32 (at least 128, at
// most 1024) and N / 256 for Euler (64 to 512).  The nearest width down to half the target that divides N and
// is a multiple of 4 rad; else the target itself (rounded down to a multiple
// of 4 rad), whose remainder widens some nodes; 0 when N is too small for
// any (fewer than two nodes of 4 rad points).
int default_width(const swp_problem* p, bool dataflow = false)
{
    const int step = 4 * p->rad;
    const bool euler = p->desc.eq == SWP_EULER;
    const int lo = euler ? 64 : 128;
    const int cap = euler ? 512 : 1024;
    // FP32 per-phase nodes: about N / 128 (2^17 heat: 1024-point nodes 287
    // against 252 G point-updates/s for 128)
    const bool f32 = p->desc.dtype == SWP_F32;
    int64_t target = p->N / (dataflow ? 512 : (euler ? 256 : (f32 ? 128 : 1024)));
    if (target < lo) target = lo;
    if (target > cap) target = cap;
    if (target > p->N / 2) target = p->N / 2;
    for (int64_t n = target; n >= step && 2 * n >= target; --n)
        if (n % step == 0 && p->N % n == 0 && check_width(p, (int)n) == SWP_OK) return (int)n;
    for (int64_t n = target / step * step; n >= step; n -= step)
        if (check_width(p, (int)n) == SWP_OK) return (int)n;
    return 0;
}

// Choices measured by the autotuners, per (equation, dtype, n_points).
struct Tuned {
    int scheme = SWP_SWEPT;   // the faster scheme (swp_autotune)
    int n = 0;                // its width: swept node or classic chunk
    int n_swept = 0;          // the fastest swept node width
};
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int64_t>, Tuned> g_tuned;

bool tuned_of(const swp_desc& d, Tuned* t)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(std::make_tuple(d.eq, d.dtype, d.n_points));
    if (it == g_tuned.end()) return false;
    *t = it->second;
    return true;
}

// Swept node width for a problem: the tuned one if measured, else the
// default rule (for the dataflow launch, or for per-phase launches).
int width_for(const swp_problem* p, bool dataflow = false)
{
    Tuned t;
    if (tuned_of(p->desc, &t) && t.n_swept > 0 && check_width(p, t.n_swept) == SWP_OK) return t.n_swept;
    return default_width(p, dataflow);
}

// Classic chunk width of a batched classic advance (points per item).
int default_chunk(const swp_problem* p)
{
    return (int)std::min<int64_t>(p->N, p->desc.eq == SWP_EULER ? 256 : 1024);
}

// SWP_SCHEME_AUTO: the scheme swp_autotune measured faster (with its width),
// else swept at width_for, else (N too small for any node width) classic.
void choice_for(const swp_problem* p, int* scheme, int* n)
{
    Tuned t;
    if (tuned_of(p->desc, &t) && t.scheme == SWP_CLASSIC && t.n > 0) {
        *scheme = SWP_CLASSIC;
        *n = t.n;
        return;
    }
    *scheme = SWP_SWEPT;
    *n = width_for(p);
    if (*n == 0) {
        *scheme = SWP_CLASSIC;
        *n = default_chunk(p);
    }
}

template <typename R>
const Coefs<R>& coefs_of(const swp_problem* p);
template <>
const Coefs<double>& coefs_of<double>(const swp_problem* p) { return p->cd; }
template <>
const Coefs<float>& coefs_of<float>(const swp_problem* p) { return p->cf; }

template <typename R>
swp_status run_classic(swp_problem* p, int64_t steps, int threads)
{
    if (threads <= 0) threads = 256;
    if (threads > 256 || threads % 32) return fail(SWP_EINVAL, "classic threads must be a multiple of 32 <= 256");
    const Coefs<R>& c = coefs_of<R>(p);
    const int eq = p->desc.eq, bc = p->desc.bc;
    for (int64_t m = 0; m < steps; ++m) {
        R* u = (R*)p->rows[p->cur];
        R* o = (R*)p->rows[1 - p->cur];
        cudaError_t e;
        if (eq == SWP_HEAT) {
            e = launch_classic<R>(eq, bc, u, u, o, p->N, 0, c, threads, p->stream);
            p->launches++;
            if (e != cudaSuccess) return cuda_fail(e, "classic heat launch");
            p->cur = 1 - p->cur;
        } else {
            e = launch_classic<R>(eq, bc, u, u, o, p->N, 0, c, threads, p->stream);
            p->launches++;
            if (e != cudaSuccess) return cuda_fail(e, "classic predictor launch");
            e = launch_classic<R>(eq, bc, o, u, u, p->N, 1, c, threads, p->stream);
            p->launches++;
            if (e != cudaSuccess) return cuda_fail(e, "classic final launch");
        }
    }
    return SWP_OK;
}

struct SweptPlan {
    int n, H, K;
    int d;     // N - K n, spread over the nodes (0 when n divides N)
    int64_t T, Q, r, n_phases;
    int top;   // relative level of the last phase's top row
};

SweptPlan plan_swept(const swp_problem* p, int64_t steps, int n)
{
    SweptPlan s;
    s.n = n;
    s.H = n / (2 * p->rad);
    s.K = (int)(p->N / n);
    s.d = (int)(p->N - (int64_t)s.K * n);
    s.T = steps * p->sub;
    s.Q = s.T / s.H;
    s.r = s.T % s.H;
    s.n_phases = s.r > 0 ? s.Q + 2 : s.Q + 1;
    s.top = s.r > 0 ? (int)s.r : s.H;
    return s;
}

// Geometry of phase ph of a plan.  Even phases of a plan with wider nodes
// (d > 0) also compute level 2H, the wider nodes' middle points.
PhaseGeom phase_geom(const swp_problem* p, const SweptPlan& s, int64_t ph)
{
    PhaseGeom g;
    g.N = p->N;
    g.n = s.n;
    g.H = s.H;
    g.K = s.K;
    g.d = s.d;
    g.odd = (int)(ph & 1);
    g.j_lo = ph == 0 ? s.H + 1 : 1;
    g.j_hi = ph < s.Q ? 2 * s.H - 1 + (!g.odd && s.d ? 1 : 0) : (ph == s.Q ? s.H + (int)s.r : (int)s.r);
    return g;
}

template <typename R>
swp_status run_swept_register(swp_problem* p, const SweptPlan& s, int threads)
{
    R* A = (R*)p->rows[p->cur];
    R* B = (R*)p->rows[1 - p->cur];
    const Coefs<R>& c = coefs_of<R>(p);
    for (int64_t ph = 0; ph < s.n_phases; ++ph) {
        const PhaseGeom g = phase_geom(p, s, ph);
        cudaError_t e = launch_swept_register<R>(p->desc.eq, A, B, g, c, threads, p->stream);
        p->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "register swept launch");
    }
    return SWP_OK;
}

template <typename R>
swp_status run_swept_phases(swp_problem* p, const SweptPlan& s, int threads, int64_t p_lo = 0,
                            int64_t p_hi = -1)
{
    R* A = (R*)p->rows[p->cur];
    R* B = (R*)p->rows[1 - p->cur];
    const Coefs<R>& c = coefs_of<R>(p);
    if (p_hi < 0) p_hi = s.n_phases;
    for (int64_t ph = p_lo; ph < p_hi; ++ph) {
        const PhaseGeom g = phase_geom(p, s, ph);
        cudaError_t e = launch_swept_phase<R>(p->desc.eq, p->desc.bc, A, B, g, c, threads, p->stream);
        p->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "swept phase launch");
    }
    return SWP_OK;
}

// The persistent launch of one problem is the batched dataflow kernel with
// this problem alone (defined with the batch code below).
swp_status persistent_via_batch(swp_problem* p, const SweptPlan& s, int threads);

template <typename R>
swp_status run_swept_persistent(swp_problem* p, const SweptPlan& s, int threads)
{
    if (!p->status) {
        cudaError_t e = cudaMalloc((void**)&p->status, sizeof(int));
        if (e != cudaSuccess) return fail(SWP_ENOMEM, "status word: %s", cudaGetErrorString(e));
        e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "status memset");
    }
    return persistent_via_batch(p, s, threads);
}

// Reads the device status word of persistent launches (stream must be idle).
swp_status check_device_status(swp_problem* p)
{
    if (!p->status) return SWP_OK;
    int st = 0;
    cudaError_t e = cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st != 0) {
        cudaMemset(p->status, 0, sizeof(int));
        return fail(SWP_ETIMEOUT, "a node's bounded wait for its neighbours gave up; the state is invalid");
    }
    return SWP_OK;
}

// Graph cache key of the Register variant's phase launches (beside
// SWP_CLASSIC and SWP_SWEPT).
constexpr int kGraphRegister = 100;

// Run the launch sequence of an advance as a CUDA graph: captured once per
// (scheme, steps, node width, threads, starting row) on a private stream,
// then replayed on the problem's stream.
template <typename R>
swp_status run_graph(swp_problem* p, int64_t steps, int scheme, int n, int threads,
                     const SweptPlan* s)
{
    for (auto& g : p->graphs)
        if (g.scheme == scheme && g.steps == steps && g.n == n && g.threads == threads &&
            g.cur_before == p->cur) {
            cudaError_t e = cudaGraphLaunch(g.exec, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            p->cur = g.cur_after;
            p->launches += g.kernels;
            return SWP_OK;
        }
    cudaError_t e;
    if (!p->capture_stream) {
        e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
    swp_problem::Graph g;
    g.scheme = scheme;
    g.steps = steps;
    g.n = n;
    g.threads = threads;
    g.cur_before = p->cur;
    const cudaStream_t user = p->stream;
    const int64_t launches0 = p->launches;
    e = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    p->stream = p->capture_stream;
    swp_status st = scheme == SWP_CLASSIC    ? run_classic<R>(p, steps, threads)
                    : scheme == kGraphRegister ? run_swept_register<R>(p, *s, threads)
                                               : run_swept_phases<R>(p, *s, threads);
    p->stream = user;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->capture_stream, &graph);
    if (st != SWP_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        p->cur = g.cur_before;
        p->launches = launches0;
        return st != SWP_OK ? st : cuda_fail(e, "end capture");
    }
    if (scheme != SWP_CLASSIC && (s->top & 1)) p->cur = 1 - p->cur;
    g.cur_after = p->cur;
    g.kernels = p->launches - launches0;
    p->launches = launches0;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        p->cur = g.cur_before;
        return cuda_fail(e, "graph instantiate");
    }
    if (p->graphs.size() >= 8) {
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back(g);
    e = cudaGraphLaunch(g.exec, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    p->launches += g.kernels;
    return SWP_OK;
}

// The Register variant's whole advance on one thread-block cluster
// (SWP_LAUNCH_CLUSTER).
template <typename R>
swp_status run_swept_cluster(swp_problem* p, int64_t steps, const swp_advance_opts& o)
{
    if (p->desc.eq == SWP_EULER || p->desc.bc != SWP_BC_PERIODIC)
        return fail(SWP_EUNSUPPORTED, "the cluster variant runs periodic heat and KS");
    if (o.points_per_block != 0 && o.points_per_block != 32)
        return fail(SWP_EINVAL, "the cluster variant's node is one warp: points_per_block 32 (or 0)");
    if (p->N % 32 || p->N < 64) return fail(SWP_EINVAL, "the cluster variant needs n_points a multiple of 32, >= 64");
    const int K = (int)std::min<int64_t>(p->N / 32, 1 << 20);
    // one warp per node: the most blocks (at most 16) that split the
    // nodes evenly with at most 8 warps each (measured: 16 blocks of 2
    // warps ran N = 1024 faster than 8 of 4), or as many as `threads` asks
    int ctas = 0, warps = 0;
    if (o.threads != 0) {
        warps = o.threads / 32;
        if (o.threads % 32 || warps < 1 || warps > 8 || K % warps || K / warps > 16)
            return fail(SWP_EINVAL, "cluster threads must be 32 w (w <= 8) with n_points / 32 = w x (blocks <= 16)");
        ctas = K / warps;
    } else {
        for (int cc = 16; cc >= 1; --cc)
            if (K % cc == 0 && K / cc <= 8) {
                ctas = cc;
                warps = K / cc;
                break;
            }
        if (ctas == 0)
            return fail(SWP_EINVAL, "the cluster variant holds at most 16 blocks of 8 nodes (n_points %lld)",
                        (long long)p->N);
    }
    const SweptPlan s = plan_swept(p, steps, 32);
    if (s.T == 0) return SWP_OK;
    ClusterGeom g;
    g.N = p->N;
    g.H = s.H;
    g.K = K;
    g.Q = s.Q;
    g.r = s.r;
    g.n_phases = s.n_phases;
    g.portion = (int)(p->N / ctas);
    g.warps = ctas * warps;
    if (swept_cluster_fits<R>(p->desc.eq, g, ctas, 32 * warps) <= 0)
        return fail(SWP_EUNSUPPORTED, "a cluster of %d blocks of %d threads does not fit this device", ctas,
                    32 * warps);
    cudaError_t e = launch_swept_cluster<R>(p->desc.eq, (R*)p->rows[p->cur], (R*)p->rows[1 - p->cur], g,
                                            coefs_of<R>(p), ctas, 32 * warps, p->stream);
    p->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "cluster swept launch");
    if (s.top & 1) p->cur = 1 - p->cur;
    return SWP_OK;
}

template <typename R>
swp_status advance_typed(swp_problem* p, int64_t steps, const swp_advance_opts& o_in)
{
    swp_advance_opts o = o_in;
    if (o.scheme == SWP_SCHEME_AUTO) {
        int n = 0;
        choice_for(p, &o.scheme, &n);
        if (o.scheme == SWP_SWEPT && o.points_per_block == 0) o.points_per_block = n;
    }
    if (o.scheme == SWP_SWEPT && o.points_per_block == 0 && o.launch != SWP_LAUNCH_REGISTER &&
        o.launch != SWP_LAUNCH_CLUSTER && default_width(p) == 0) {
        // N is too small for two nodes of 4 rad points: the classic scheme,
        // whose result is the same
        o.scheme = SWP_CLASSIC;
        if (o.launch != SWP_LAUNCH_GRAPH) o.launch = SWP_LAUNCH_AUTO;
    }
    if (o.scheme == SWP_CLASSIC) {
        if (o.launch == SWP_LAUNCH_GRAPH) {
            const int thr = o.threads <= 0 ? 256 : o.threads;
            if (thr > 256 || thr % 32) return fail(SWP_EINVAL, "classic threads must be a multiple of 32 <= 256");
            return run_graph<R>(p, steps, SWP_CLASSIC, 0, thr, nullptr);
        }
        return run_classic<R>(p, steps, o.threads);
    }
    // AUTO for small periodic heat and KS, where phases are short and launch
    // gaps and global round trips count (measured fastest on GB300): the
    // cluster form up to 2048 points in FP64 and 4096 in FP32 (heat FP32
    // N = 1024: 11.9 G point-updates/s against 2.2 for per-phase launches),
    // then the Register variant (graph) up to 2^15 (heat) and 2^14 (KS) in
    // FP64, and in FP32 for heat up to 2^18 (2^18: 566 against 528) and KS up
    // to 2^17; a cluster that cannot run falls through
    if (o.launch == SWP_LAUNCH_AUTO && o.points_per_block == 0 && o.threads == 0 && p->desc.eq != SWP_EULER &&
        p->desc.bc == SWP_BC_PERIODIC && p->N % 32 == 0 && p->N >= 64) {
        const bool f32 = p->desc.dtype == SWP_F32;
        if (p->N <= (f32 ? 4096 : 2048)) {
            swp_advance_opts oc = o;
            oc.launch = SWP_LAUNCH_CLUSTER;
            swp_status st = run_swept_cluster<R>(p, steps, oc);
            if (st != SWP_EUNSUPPORTED && st != SWP_EINVAL) return st;   // else no cluster shape fits N
        }
        const int64_t reg_max = f32 ? ((int64_t)1 << (p->desc.eq == SWP_HEAT ? 18 : 17))
                                    : ((int64_t)1 << (p->desc.eq == SWP_HEAT ? 15 : 14));
        if (p->N <= reg_max) o.launch = SWP_LAUNCH_REGISTER;
    }
    if (o.launch == SWP_LAUNCH_CLUSTER) return run_swept_cluster<R>(p, steps, o);
    if (o.launch == SWP_LAUNCH_REGISTER) {
        if (p->desc.eq == SWP_EULER || p->desc.bc != SWP_BC_PERIODIC)
            return fail(SWP_EUNSUPPORTED, "the register variant runs periodic heat and KS");
        if (o.points_per_block != 0 && o.points_per_block != 32)
            return fail(SWP_EINVAL, "the register variant's node is one warp: points_per_block 32 (or 0)");
        if (p->N % 32 || p->N < 64) return fail(SWP_EINVAL, "the register variant needs n_points a multiple of 32, >= 64");
        // two nodes per block by default: small problems then spread over
        // more SMs (heat N = 1024: 2.9 G upd/s against 2.0 with 8 per block)
        const int thr = o.threads == 0 ? 64 : o.threads;
        if (thr < 32 || thr > 256 || thr % 32) return fail(SWP_EINVAL, "threads must be a multiple of 32 in [32, 256]");
        const SweptPlan s = plan_swept(p, steps, 32);
        if (s.T == 0) return SWP_OK;
        // its phases are short (16 levels of KS, 32 of heat), so they replay
        // as a CUDA graph rather than pay a stream launch each
        return run_graph<R>(p, steps, kGraphRegister, 32, thr, &s);
    }
    // AUTO: in FP64 the dataflow (persistent) launch from N = 2^17 up (Euler
    // from 2^13: Sod 2^17, 256-cell nodes, 3.21 against 2.81 G
    // point-updates/s for the best per-phase form), where it measured faster
    // than per-phase launches, and below that the per-phase launches replayed
    // as a CUDA graph (captured on the first advance of a step count;
    // measured 5-10 % faster than stream launches); in FP32 per-phase
    // launches, where the per-phase kernels' register-blocked levels win
    const bool euler = p->desc.eq == SWP_EULER;
    const int launch = o.launch != SWP_LAUNCH_AUTO ? o.launch
                       : p->desc.dtype != SWP_F64                      ? SWP_LAUNCH_PER_PHASE
                       : p->N >= ((int64_t)1 << (euler ? 13 : 17))     ? SWP_LAUNCH_PERSISTENT
                                                                       : SWP_LAUNCH_GRAPH;
    int n = o.points_per_block;
    if (n == 0) {
        n = default_width(p, launch == SWP_LAUNCH_PERSISTENT);
        if (n == 0) return fail(SWP_EINVAL, "no valid node width for n_points %lld", (long long)p->N);
    }
    swp_status st = check_width(p, n);
    if (st != SWP_OK) return st;
    int threads = o.threads;
    if (threads == 0) {
        if (p->desc.dtype == SWP_F32)   // about 8 points per thread (register-blocked levels)
            threads = std::max(64, std::min(256, n / 8)) / 32 * 32;
        else if (launch == SWP_LAUNCH_PERSISTENT)   // measured: 256 from 256-point nodes up (Euler: always)
            threads = (n >= 256 || p->desc.eq == SWP_EULER) ? 256 : (n >= 128 ? 128 : 64);
        else
            threads = n >= 512 ? 256 : (n >= 128 ? 128 : 64);
    }
    const int max_threads = p->desc.eq == SWP_EULER ? 256 : 1024;
    if (threads < 32 || threads > max_threads || threads % 32)
        return fail(SWP_EINVAL, "threads must be a multiple of 32 in [32, %d]", max_threads);
    const SweptPlan s = plan_swept(p, steps, n);
    if (s.T == 0) return SWP_OK;
    if (launch == SWP_LAUNCH_GRAPH) return run_graph<R>(p, steps, SWP_SWEPT, n, threads, &s);
    if (launch == SWP_LAUNCH_PERSISTENT) st = run_swept_persistent<R>(p, s, threads);
    else if (launch == SWP_LAUNCH_PER_PHASE) st = run_swept_phases<R>(p, s, threads);
    else return fail(SWP_EINVAL, "unknown launch mode %d", o.launch);
    if (st != SWP_OK) return st;
    if (s.top & 1) p->cur = 1 - p->cur;   // last level odd: the state is in row B
    return SWP_OK;
}

}  // namespace

extern "C" {

swp_status swp_required_bytes(const swp_desc* desc, size_t* bytes)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!bytes) return fail(SWP_EINVAL, "bytes is NULL");
    *bytes = 2 * state_bytes(desc);
    return SWP_OK;
}

swp_status swp_set_memory_budget(size_t bytes)
{
    g_budget.store(bytes);
    return SWP_OK;
}

size_t swp_memory_in_use(void) { return g_in_use.load(); }

swp_status swp_create(const swp_desc* desc, const void* u0, int u0_on_device, void* cuda_stream,
                      swp_problem** out)
{
    if (!out) return fail(SWP_EINVAL, "out is NULL");
    *out = nullptr;
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!u0) return fail(SWP_EINVAL, "u0 is NULL");
    // admission against the memory budget comes first (host-side decision)
    const size_t sbytes = state_bytes(desc);
    const size_t need = 2 * sbytes;
    const size_t budget = g_budget.load();
    size_t cur = g_in_use.load();
    for (;;) {
        if (budget && cur + need > budget)
            return fail(SWP_EBUDGET, "problem needs %zu bytes, %zu of the %zu-byte budget in use", need, cur, budget);
        if (g_in_use.compare_exchange_weak(cur, cur + need)) break;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) {
        g_in_use -= need;
        return fail(SWP_EDEVICE, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    if (prop.major != 10 || prop.minor != 3) {
        g_in_use -= need;
        return fail(SWP_EDEVICE, "libswept is built for sm_103 (device is sm_%d%d)", prop.major, prop.minor);
    }
    swp_problem* p = new (std::nothrow) swp_problem();
    if (!p) {
        g_in_use -= need;
        return fail(SWP_ENOMEM, "host allocation failed");
    }
    p->desc = *desc;
    p->id = g_next_id.fetch_add(1);
    p->wait_limit_ns = default_wait_limit_ns();
    p->nv = nv_of(desc->eq);
    p->rad = radius_of(desc->eq);
    p->sub = desc->eq == SWP_HEAT ? 1 : 2;
    p->esize = esize_of(desc->dtype);
    p->N = desc->n_points;
    p->stream = (cudaStream_t)cuda_stream;
    p->device = dev;
    p->sms = prop.multiProcessorCount;
    p->bytes = need;
    void* mem = nullptr;
    e = cudaMalloc(&mem, need);
    if (e != cudaSuccess) {
        g_in_use -= need;
        delete p;
        return fail(SWP_ENOMEM, "device allocation of %zu bytes failed: %s", need, cudaGetErrorString(e));
    }
    p->rows[0] = mem;
    p->rows[1] = (char*)mem + sbytes;
    make_coefs<double>(desc, p->cd);
    make_coefs<float>(desc, p->cf);
    e = cudaMemsetAsync(p->rows[1], 0, sbytes, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->rows[0], u0, sbytes,
                            u0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess && !u0_on_device) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        swp_destroy(p);
        return cuda_fail(e, "initial state copy");
    }
    *out = p;
    return SWP_OK;
}

swp_status swp_write(swp_problem* p, const void* src, size_t src_bytes, int src_on_device)
{
    if (!p || !src) return fail(SWP_EINVAL, "problem or src is NULL");
    const size_t sbytes = (size_t)p->nv * p->N * p->esize;
    if (src_bytes != sbytes) return fail(SWP_EINVAL, "src_bytes %zu != state bytes %zu", src_bytes, sbytes);
    cudaError_t e = cudaMemcpyAsync(p->rows[p->cur], src, sbytes,
                                    src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    p->stream);
    if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state write");
    return SWP_OK;
}

swp_status swp_advance_ex(swp_problem* p, int64_t n_steps, const swp_advance_opts* opts)
{
    if (!p || !opts) return fail(SWP_EINVAL, "problem or opts is NULL");
    if (n_steps < 0) return fail(SWP_EINVAL, "n_steps must be >= 0");
    if (opts->scheme != SWP_CLASSIC && opts->scheme != SWP_SWEPT && opts->scheme != SWP_SCHEME_AUTO)
        return fail(SWP_EINVAL, "unknown scheme %d", opts->scheme);
    if (n_steps == 0) return SWP_OK;
    if (n_steps > ((int64_t)1 << 40)) return fail(SWP_EINVAL, "n_steps too large");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return fail(SWP_EINVAL, "current device %d differs from the problem's device %d", dev, p->device);
    if (p->desc.dtype == SWP_F64) return advance_typed<double>(p, n_steps, *opts);
    return advance_typed<float>(p, n_steps, *opts);
}

swp_status swp_advance(swp_problem* p, int64_t n_steps, int32_t scheme, int32_t points_per_block)
{
    swp_advance_opts o;
    o.scheme = scheme;
    o.points_per_block = points_per_block;
    o.launch = SWP_LAUNCH_AUTO;
    o.threads = 0;
    return swp_advance_ex(p, n_steps, &o);
}

swp_status swp_synchronize(swp_problem* p)
{
    if (!p) return fail(SWP_EINVAL, "problem is NULL");
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return check_device_status(p);
}

swp_status swp_read(swp_problem* p, void* dst, size_t dst_bytes, int dst_on_device)
{
    if (!p || !dst) return fail(SWP_EINVAL, "problem or dst is NULL");
    const size_t sbytes = (size_t)p->nv * p->N * p->esize;
    if (dst_bytes < sbytes) return fail(SWP_EINVAL, "dst_bytes %zu < state bytes %zu", dst_bytes, sbytes);
    cudaError_t e = cudaMemcpyAsync(dst, p->rows[p->cur], sbytes,
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state read");
    if (!dst_on_device) return swp_synchronize(p);
    return SWP_OK;
}

swp_status swp_destroy(swp_problem* p)
{
    if (!p) return SWP_OK;
    cudaError_t e = cudaSuccess;
    if (p->rows[0]) e = cudaFree(p->rows[0]);
    if (p->batch) swp_batch_destroy(p->batch);
    if (p->status) cudaFree(p->status);
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
    if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
    g_in_use -= p->bytes;
    delete p;
    if (e != cudaSuccess) return cuda_fail(e, "free");
    return SWP_OK;
}

swp_status swp_shape(const swp_problem* p, int64_t* n_points, int32_t* nv, int32_t* elem_bytes)
{
    if (!p) return fail(SWP_EINVAL, "problem is NULL");
    if (n_points) *n_points = p->N;
    if (nv) *nv = p->nv;
    if (elem_bytes) *elem_bytes = p->esize;
    return SWP_OK;
}

int64_t swp_kernel_launches(const swp_problem* p) { return p ? p->launches : -1; }

swp_status swp_debug_withhold_flags(swp_problem* p, int withhold, int64_t wait_limit_ns)
{
    if (!p) return fail(SWP_EINVAL, "problem is NULL");
    if (wait_limit_ns <= 0 || wait_limit_ns > 10000000000ll)
        return fail(SWP_EINVAL, "wait_limit_ns must be in (0, 1e10]");
    p->inject_withheld_flags = withhold ? 1 : 0;
    p->wait_limit_ns = (uint64_t)wait_limit_ns;
    return SWP_OK;
}

const char* swp_status_str(swp_status s)
{
    switch (s) {
    case SWP_OK: return "SWP_OK";
    case SWP_EINVAL: return "SWP_EINVAL";
    case SWP_ENOMEM: return "SWP_ENOMEM";
    case SWP_EBUDGET: return "SWP_EBUDGET";
    case SWP_ECUDA: return "SWP_ECUDA";
    case SWP_EUNSUPPORTED: return "SWP_EUNSUPPORTED";
    case SWP_ETIMEOUT: return "SWP_ETIMEOUT";
    case SWP_EDEVICE: return "SWP_EDEVICE";
    }
    return "SWP_UNKNOWN";
}

const char* swp_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched advance (swept and classic instances in one persistent launch) and
// the autotuners.
// ---------------------------------------------------------------------------
namespace {

// Device tables of one persistent batch launch.
struct BatchTables {
    void* insts = nullptr;     size_t insts_cap = 0;
    int2* tasks = nullptr;     size_t tasks_cap = 0;
    int* ctr = nullptr;        size_t ctr_cap = 0;     // [0] = cur_task, [1..] = task counters
    uint32_t* flags = nullptr; size_t flags_cap = 0;
    void release()
    {
        if (insts) cudaFree(insts);
        if (tasks) cudaFree(tasks);
        if (ctr) cudaFree(ctr);
        if (flags) cudaFree(flags);
        *this = BatchTables();
    }
};

// A batch launch captured as a CUDA graph (zero the counters and flags, run
// the persistent kernel), with tables of its own; replayed when the same
// problems, in the same rows, advance by the same plans again.
struct BatchGraph {
    std::vector<int64_t> key;
    BatchTables t;
    cudaGraphExec_t exec = nullptr;
    std::vector<swp_problem*> flip;   // problems whose state ends in the other row
    std::vector<swp_problem*> all;
};

}  // namespace

struct swp_batch {
    cudaStream_t stream = nullptr;
    int device = 0, sms = 0;
    int64_t launches = 0;
    BatchTables t;                     // plain launches, grown on demand
    int* status = nullptr;             // != 0: a bounded wait gave up (sticky until synchronize)
    void* stage = nullptr;             // pinned staging of the table uploads
    size_t stage_cap = 0;
    cudaEvent_t staged = nullptr;      // the last upload out of `stage` has finished
    std::vector<BatchGraph> graphs;    // at most 8, oldest first
    cudaStream_t capture_stream = nullptr;
    uint64_t wait_limit_ns = 2000000000ull;
};

namespace {

swp_status grow(void** p, size_t* cap, size_t bytes)
{
    if (*cap >= bytes) return SWP_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = bytes + bytes / 2 + 256;
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) return fail(SWP_ENOMEM, "batch workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    *cap = want;
    return SWP_OK;
}

swp_status grow_tables(BatchTables& t, size_t inst_bytes, size_t ntasks, size_t nflags)
{
    swp_status st;
    if ((st = grow(&t.insts, &t.insts_cap, inst_bytes)) != SWP_OK) return st;
    if ((st = grow((void**)&t.tasks, &t.tasks_cap, sizeof(int2) * ntasks)) != SWP_OK) return st;
    if ((st = grow((void**)&t.ctr, &t.ctr_cap, sizeof(int) * (ntasks + 1))) != SWP_OK) return st;
    return grow((void**)&t.flags, &t.flags_cap, sizeof(uint32_t) * nflags);
}

struct BatchItem {
    swp_problem* p;
    int kind;       // BATCH_SWEPT / BATCH_CLASSIC
    SweptPlan s;    // swept plan; classic: n = widest chunk, K = chunks, n_phases = sub-steps
    int64_t p_lo, p_hi;   // phases of the plan this launch runs
    bool flip;      // the state ends in the other row (the plan's last phase runs)
};

// Classic instance of a batch: K = ceil(N / m) chunks of the balanced
// partition (each at least N / K >= m / 2 >= rad points, so a point's stencil
// stays within its chunk's two neighbours), one phase per sub-timestep.
SweptPlan plan_classic(const swp_problem* p, int64_t steps, int m)
{
    SweptPlan s{};
    s.K = (int)((p->N + m - 1) / m);
    s.n = (int)((p->N + s.K - 1) / s.K);
    s.T = steps * p->sub;
    s.n_phases = s.T;
    return s;
}

swp_status check_chunk(const swp_problem* p, int m)
{
    if (m < 4 || m > p->N) return fail(SWP_EINVAL, "classic chunk width %d must be in [4, n_points]", m);
    if ((p->N + m - 1) / m >= ((int64_t)1 << 30))
        return fail(SWP_EINVAL, "classic chunk width %d gives 2^30 or more chunks", m);
    if (batch_classic_smem_bytes(p->desc.eq, m, p->esize) > max_smem(p->device))
        return fail(SWP_EINVAL, "classic chunk width %d does not fit shared memory", m);
    return SWP_OK;
}

// Estimated FP64-pipe operations per point of one level (sub-timestep).
double level_cost(int eq) { return eq == SWP_HEAT ? 3.0 : (eq == SWP_KS ? 7.0 : 100.0); }

// One persistent launch of the items (one equation group and dtype).  status,
// wait_offset and wait_limit override the batch's status word and bounded-wait
// settings (the single-problem persistent launch and its test hook).
template <typename R>
swp_status batch_group(swp_batch* b, const std::vector<BatchItem>& items, int mode, int threads, bool graph,
                       int* status = nullptr, uint32_t wait_offset = 0, uint64_t wait_limit = 0,
                       int max_blocks_per_sm = 0)
{
    std::vector<int64_t> key;
    if (graph) {
        key.reserve(items.size() * 5 + 2);
        key.push_back(mode);
        key.push_back(threads);
        for (const auto& it : items) {
            // the id, not the address: a new problem may reuse a destroyed one's
            key.push_back((int64_t)it.p->id);
            key.push_back(it.p->cur);
            key.push_back(it.kind);
            key.push_back(it.s.n);
            key.push_back(it.s.T);
            key.push_back(it.p_lo);
            key.push_back(it.p_hi);
        }
        for (auto& g : b->graphs)
            if (g.key == key) {
                cudaError_t e = cudaGraphLaunch(g.exec, b->stream);
                if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
                b->launches++;
                for (auto* p : g.all) p->launches++;
                for (auto* p : g.flip) p->cur = 1 - p->cur;
                return SWP_OK;
            }
    }
    std::vector<BatchInst<R>> insts(items.size());
    int64_t flags = 0, items_total = 0;
    size_t smem = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        const BatchItem& it = items[i];
        BatchInst<R>& in = insts[i];
        in.A = (R*)it.p->rows[it.p->cur];
        in.B = (R*)it.p->rows[1 - it.p->cur];
        in.N = it.p->N;
        in.n = it.s.n;
        in.H = it.s.H;
        in.K = it.s.K;
        in.d = it.kind == BATCH_SWEPT ? it.s.d : 0;
        in.bc = it.p->desc.bc;
        in.Q = it.s.Q;
        in.r = it.s.r;
        in.n_phases = it.s.n_phases;
        in.phase_lo = it.p_lo;
        in.flag_off = (int)flags;
        in.eq = it.p->desc.eq;
        in.kind = it.kind;
        in.c = coefs_of<R>(it.p);
        flags += it.s.K;
        items_total += (it.p_hi - it.p_lo) * it.s.K;
        smem = std::max(smem, it.kind == BATCH_SWEPT
                                  ? swept_smem_bytes(it.p->desc.eq, (int)widest_node(it.p->N, it.s.n), it.p->esize)
                                                     : batch_classic_smem_bytes(it.p->desc.eq, it.s.n, it.p->esize));
    }
    // (instance, phase) tasks in order of estimated start: phase p of instance
    // i at p * c_i, with c_i the cost of one of its items (levels times FP64
    // operations per point, times the warp rows of its widest level).  Each
    // instance keeps its phases in order, so every item depends only on items
    // of earlier tasks; instances with short items run ahead instead of
    // waiting, phase by phase, for instances with long ones.
    struct Key {
        double start;
        int inst, phase;
    };
    std::vector<Key> keys;
    keys.reserve((size_t)std::min<int64_t>(items_total, (int64_t)1 << 30));
    for (size_t i = 0; i < items.size(); ++i) {
        const auto& s = items[i].s;
        const double rows = std::max(1.0, (double)s.n / 256.0);
        const double levels = items[i].kind == BATCH_SWEPT ? 2.0 * s.H - 1.0 : 1.0;
        const double cost = levels * level_cost(items[i].p->desc.eq) * rows;
        const int64_t lo = items[i].p_lo, hi = items[i].p_hi;
        if ((int64_t)keys.size() + (hi - lo) >= ((int64_t)1 << 30))
            return fail(SWP_EINVAL, "batch too large for one launch");
        for (int64_t ph = lo; ph < hi; ++ph) keys.push_back(Key{(double)(ph - lo) * cost, (int)i, (int)ph});
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
        return x.start < y.start || (x.start == y.start && x.phase < y.phase);
    });
    if (flags >= (int64_t)1 << 30) return fail(SWP_EINVAL, "batch too large for one launch");
    const size_t ntasks = keys.size();
    const size_t inst_bytes = sizeof(BatchInst<R>) * insts.size();
    const size_t task_bytes = sizeof(int2) * ntasks;

    BatchGraph gnew;
    BatchTables& t = graph ? gnew.t : b->t;
    swp_status st = grow_tables(t, inst_bytes, ntasks, (size_t)flags);
    if (st != SWP_OK) {
        if (graph) gnew.t.release();
        return st;
    }
    // upload through the pinned staging buffer once its previous upload is done
    cudaError_t e = cudaEventSynchronize(b->staged);
    if (e == cudaSuccess && b->stage_cap < inst_bytes + task_bytes) {
        if (b->stage) cudaFreeHost(b->stage);
        b->stage = nullptr;
        b->stage_cap = 0;
        const size_t want = inst_bytes + task_bytes + (inst_bytes + task_bytes) / 2 + 256;
        e = cudaMallocHost(&b->stage, want);
        if (e == cudaSuccess) b->stage_cap = want;
    }
    if (e == cudaSuccess) {
        unsigned char* stg = (unsigned char*)b->stage;
        std::memcpy(stg, insts.data(), inst_bytes);
        int2* tk = (int2*)(stg + inst_bytes);
        for (size_t i = 0; i < ntasks; ++i) tk[i] = make_int2(keys[i].inst, keys[i].phase);
        e = cudaMemcpyAsync(t.insts, stg, inst_bytes, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(t.tasks, tk, task_bytes, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->staged, b->stream);
    }
    if (e != cudaSuccess) {
        if (graph) gnew.t.release();
        return cuda_fail(e, "batch table upload");
    }
    BatchWork w;
    w.tasks = t.tasks;
    w.cur_task = t.ctr;
    w.task_ctr = t.ctr + 1;
    w.status = status ? status : b->status;
    w.ntasks = (int)ntasks;
    w.smem_bytes = smem;
    w.flags = t.flags;
    w.wait_limit_ns = wait_limit ? wait_limit : b->wait_limit_ns;
    w.wait_offset = wait_offset;
    bool reg = false, cls = false;
    for (const auto& it : items) {
        if (it.kind == BATCH_SWEPT && swept_reg_slots(it.p->desc.eq, it.s.n, threads, it.p->esize) > 0) reg = true;
        if (it.kind == BATCH_CLASSIC) cls = true;
    }
    int bps = swept_batch_blocks_per_sm<R>(mode, reg, cls, smem, threads);
    if (max_blocks_per_sm > 0 && bps > max_blocks_per_sm) bps = max_blocks_per_sm;
    if (bps <= 0) {
        if (graph) gnew.t.release();
        return fail(SWP_EINVAL, "batch kernel does not fit (%zu bytes of shared memory, threads=%d)", smem, threads);
    }
    int64_t blocks = (int64_t)b->sms * bps;
    if (blocks > items_total) blocks = items_total;
    const BatchInst<R>* dinsts = (const BatchInst<R>*)t.insts;
    if (!graph) {
        e = cudaMemsetAsync(t.ctr, 0, sizeof(int) * (ntasks + 1), b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.flags, 0, sizeof(uint32_t) * (size_t)flags, b->stream);
        if (e == cudaSuccess) e = launch_swept_batch<R>(mode, reg, cls, dinsts, w, threads, (int)blocks, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    } else {
        // the uploads above are ordinary stream work; the graph holds the rest
        if (!b->capture_stream) {
            e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                gnew.t.release();
                return cuda_fail(e, "capture stream");
            }
        }
        cudaGraph_t cg = nullptr;
        e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(t.ctr, 0, sizeof(int) * (ntasks + 1), b->capture_stream);
            if (e1 == cudaSuccess)
                e1 = cudaMemsetAsync(t.flags, 0, sizeof(uint32_t) * (size_t)flags, b->capture_stream);
            if (e1 == cudaSuccess) e1 = launch_swept_batch<R>(mode, reg, cls, dinsts, w, threads, (int)blocks, b->capture_stream);
            e = cudaStreamEndCapture(b->capture_stream, &cg);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gnew.exec, cg, 0);
        if (cg) cudaGraphDestroy(cg);
        if (e == cudaSuccess) e = cudaGraphLaunch(gnew.exec, b->stream);
        if (e != cudaSuccess) {
            if (gnew.exec) cudaGraphExecDestroy(gnew.exec);
            cudaStreamSynchronize(b->stream);
            gnew.t.release();
            return cuda_fail(e, "batch graph capture");
        }
        gnew.key = std::move(key);
        for (const auto& it : items) {
            gnew.all.push_back(it.p);
            if (it.flip) gnew.flip.push_back(it.p);
        }
        if (b->graphs.size() >= 8) {
            // its last replay may still run: wait before freeing its tables
            cudaStreamSynchronize(b->stream);
            cudaGraphExecDestroy(b->graphs.front().exec);
            b->graphs.front().t.release();
            b->graphs.erase(b->graphs.begin());
        }
        b->graphs.push_back(std::move(gnew));
    }
    b->launches++;
    for (const auto& it : items) {
        it.p->launches++;
        if (it.flip) it.p->cur = 1 - it.p->cur;
    }
    return SWP_OK;
}

swp_status persistent_via_batch(swp_problem* p, const SweptPlan& s, int threads)
{
    if (!p->batch) {
        swp_status st = swp_batch_create(p->stream, &p->batch);
        if (st != SWP_OK) return st;
    }
    std::vector<BatchItem> items(1);
    items[0].p = p;
    items[0].kind = BATCH_SWEPT;
    items[0].s = s;
    items[0].p_lo = 0;
    items[0].p_hi = s.n_phases;
    items[0].flip = false;   // the caller moves the state's row
    const int mode = p->desc.eq == SWP_EULER ? SWP_EULER : SWP_HEAT;
    const uint32_t withhold = p->inject_withheld_flags ? (1u << 30) : 0u;
    // at most 768 threads (24 warps) per SM: with fewer nodes in flight each
    // finishes sooner and the phase chain advances faster (KS 2^20, 1024-point
    // nodes: 40.0 against 36.8 G upd/s with 5 blocks of 256 per SM)
    const int max_bps = std::max(1, 768 / threads);
    const int64_t l0 = p->launches;
    swp_status st = p->desc.dtype == SWP_F64
                        ? batch_group<double>(p->batch, items, mode, threads, false, p->status, withhold,
                                              p->wait_limit_ns, max_bps)
                        : batch_group<float>(p->batch, items, mode, threads, false, p->status, withhold,
                                             p->wait_limit_ns, max_bps);
    if (st == SWP_OK && p->launches != l0 + 1) p->launches = l0 + 1;
    return st;
}

// One group launch per (equation group, dtype) of the given items.
swp_status launch_groups(swp_batch* b, std::vector<BatchItem> (&groups)[2][2], int threads, bool graph)
{
    for (int g = 0; g < 2; ++g)
        for (int dt = 0; dt < 2; ++dt) {
            if (groups[g][dt].empty()) continue;
            const int mode = g == 1 ? SWP_EULER : SWP_HEAT;
            // default block, measured on the batched heat+KS workload: 128
            // threads in FP64; one warp per node in FP32, where a level's
            // barrier is the cost that matters
            int thr = threads ? threads : (dt == SWP_F32 ? 32 : 128);
            if (g == 1 && thr > 256) thr = 256;
            swp_status st = dt == SWP_F64 ? batch_group<double>(b, groups[g][dt], mode, thr, graph)
                                          : batch_group<float>(b, groups[g][dt], mode, thr, graph);
            if (st != SWP_OK) return st;
        }
    return SWP_OK;
}

swp_status batch_advance(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps, int32_t count,
                         const int32_t* schemes, int default_scheme, const int32_t* points_per_block,
                         int32_t threads, int32_t launch)
{
    if (!b || !problems || !n_steps) return fail(SWP_EINVAL, "batch, problems or n_steps is NULL");
    if (count < 0) return fail(SWP_EINVAL, "count must be >= 0");
    if (launch != SWP_LAUNCH_AUTO && launch != SWP_LAUNCH_PERSISTENT && launch != SWP_LAUNCH_GRAPH)
        return fail(SWP_EINVAL, "batch launch must be SWP_LAUNCH_AUTO, _PERSISTENT or _GRAPH");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return fail(SWP_EINVAL, "current device differs from the batch's device");
    std::vector<BatchItem> groups[2][2];   // [heat+KS | Euler][dtype]
    int max_threads = 1024;
    for (int32_t i = 0; i < count; ++i) {
        swp_problem* p = problems[i];
        if (!p) return fail(SWP_EINVAL, "problem %d is NULL", i);
        if (p->device != b->device) return fail(SWP_EINVAL, "problem %d is on another device", i);
        if (p->stream != b->stream) return fail(SWP_EINVAL, "problem %d uses another stream than the batch", i);
        if (n_steps[i] < 0 || n_steps[i] > ((int64_t)1 << 40)) return fail(SWP_EINVAL, "n_steps[%d] out of range", i);
        for (int32_t j = 0; j < i; ++j)
            if (problems[j] == p) return fail(SWP_EINVAL, "problem %d appears twice", i);
        int scheme = schemes ? schemes[i] : default_scheme;
        if (scheme != SWP_CLASSIC && scheme != SWP_SWEPT && scheme != SWP_SCHEME_AUTO)
            return fail(SWP_EINVAL, "unknown scheme %d for problem %d", scheme, i);
        if (n_steps[i] == 0) continue;
        int n = points_per_block ? points_per_block[i] : 0;
        if (scheme == SWP_SCHEME_AUTO) {
            int tn = 0;
            choice_for(p, &scheme, &tn);
            if (n == 0) n = tn;
        }
        BatchItem it;
        it.p = p;
        if (scheme == SWP_SWEPT && n == 0) {
            n = width_for(p);
            if (n == 0) scheme = SWP_CLASSIC;   // N too small for any node width: classic items
        }
        if (scheme == SWP_SWEPT) {
            swp_status st = check_width(p, n);
            if (st != SWP_OK) return st;
            it.kind = BATCH_SWEPT;
            it.s = plan_swept(p, n_steps[i], n);
            it.flip = (it.s.top & 1) != 0;
        } else {
            if (n == 0) n = default_chunk(p);
            swp_status st = check_chunk(p, n);
            if (st != SWP_OK) return st;
            it.kind = BATCH_CLASSIC;
            it.s = plan_classic(p, n_steps[i], n);
            it.flip = p->desc.eq == SWP_HEAT && (it.s.T & 1);
        }
        it.p_lo = 0;
        it.p_hi = it.s.n_phases;
        groups[p->desc.eq == SWP_EULER ? 1 : 0][p->desc.dtype].push_back(it);
        if (p->desc.eq == SWP_EULER) max_threads = 256;
    }
    if (threads < 0 || threads > max_threads || threads % 32)
        return fail(SWP_EINVAL, "threads must be 0 or a multiple of 32 in [32, %d]", max_threads);
    return launch_groups(b, groups, threads, launch == SWP_LAUNCH_GRAPH);
}

// Node width for N points from a target width w: N split into
// K = max(2, ceil(N / w)) nearly equal nodes, the width a multiple of 4 rad,
// so that the remainder widens some nodes by at most 4 rad and no node is
// wider than w + 4 rad (a batch sizes its blocks for its widest node); 0 when
// N has no two nodes of 4 rad points.
int64_t fitted_width(int rad, int64_t N, int64_t w)
{
    const int64_t step = 4 * rad;
    if (w < step || N < 2 * step) return 0;
    const int64_t K = std::max<int64_t>(2, (N + w - 1) / w);
    return std::max<int64_t>(step, (N / K) / step * step);
}

// Time two advances (the second timed) of `steps` timesteps of `count`
// copies of a problem in one batch with the given scheme and width; returns
// point-updates per second, or < 0.
double time_batch(const swp_desc* desc, const void* u0, int count, int64_t steps, int scheme, int n, int threads)
{
    std::vector<swp_problem*> probs;
    double rate = -1.0;
    swp_batch* b = nullptr;
    std::vector<int64_t> st(count, steps);
    std::vector<int32_t> nn(count, n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (swp_batch_create(nullptr, &b) != SWP_OK) return -1.0;
    for (int i = 0; i < count; ++i) {
        swp_problem* p = nullptr;
        if (swp_create(desc, u0, 0, nullptr, &p) != SWP_OK) goto done;
        probs.push_back(p);
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0, nullptr);
        if (batch_advance(b, probs.data(), st.data(), count, nullptr, scheme, nn.data(), threads, SWP_LAUNCH_AUTO) !=
            SWP_OK)
            goto done;
        if (rep == 1) cudaEventRecord(e1, nullptr);
        if (swp_batch_synchronize(b) != SWP_OK) goto done;
    }
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f) rate = (double)count * desc->n_points * steps / (ms * 1e-3);
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (auto* p : probs) swp_destroy(p);
    swp_batch_destroy(b);
    return rate;
}

// Fastest swept node width (powers of two that fit) for the description.
swp_status tune_swept(const swp_desc* desc, const void* u0_host, int32_t count, int64_t steps, int* best_n,
                      double* best_rate)
{
    swp_problem probe;   // for the width checks only
    probe.desc = *desc;
    probe.rad = radius_of(desc->eq);
    probe.nv = nv_of(desc->eq);
    probe.sub = desc->eq == SWP_HEAT ? 1 : 2;
    probe.esize = esize_of(desc->dtype);
    probe.N = desc->n_points;
    if (cudaGetDevice(&probe.device) != cudaSuccess) return fail(SWP_EDEVICE, "no CUDA device");
    // wider nodes won in isolation but lost in mixed batches (fewer, longer items)
    const int cap = 1024;
    *best_n = 0;
    *best_rate = -1.0;
    for (int n = 32; n <= cap && n <= probe.N; n *= 2) {
        if (check_width(&probe, n) != SWP_OK || probe.N / n < 2) continue;
        const int threads = desc->dtype == SWP_F32 ? 32 : 128;   // the batch defaults
        const double rate = time_batch(desc, u0_host, count, steps, SWP_SWEPT, n, threads);
        if (rate > *best_rate) {
            *best_rate = rate;
            *best_n = n;
        }
    }
    if (*best_n == 0) return fail(SWP_EINVAL, "no node width could be timed for n_points %lld", (long long)probe.N);
    return SWP_OK;
}

}  // namespace

namespace swp {

int swept_width(const swp_problem* p) { return width_for(p, true); }

int classic_chunk(const swp_problem* p) { return default_chunk(p); }

int64_t phase_count(const swp_problem* p, int64_t steps, int kind, int n)
{
    return kind == BATCH_CLASSIC ? plan_classic(p, steps, n).n_phases : plan_swept(p, steps, n).n_phases;
}

swp_status batch_advance_phases(swp_batch* b, const PhaseRange* ranges, int count, int threads)
{
    if (!b || (count > 0 && !ranges)) return fail(SWP_EINVAL, "batch or ranges is NULL");
    std::vector<BatchItem> groups[2][2];
    for (int i = 0; i < count; ++i) {
        const PhaseRange& r = ranges[i];
        swp_problem* p = r.p;
        if (!p || p->device != b->device || p->stream != b->stream)
            return fail(SWP_EINVAL, "range %d: problem NULL or on another device / stream", i);
        const bool classic = r.kind == BATCH_CLASSIC;
        swp_status st = classic ? check_chunk(p, r.n) : check_width(p, r.n);
        if (st != SWP_OK) return st;
        BatchItem it;
        it.p = p;
        it.kind = classic ? BATCH_CLASSIC : BATCH_SWEPT;
        it.s = classic ? plan_classic(p, r.steps, r.n) : plan_swept(p, r.steps, r.n);
        if (r.p_lo < 0 || r.p_hi > it.s.n_phases || r.p_lo > r.p_hi)
            return fail(SWP_EINVAL, "range %d: phases [%lld, %lld) outside the plan", i, (long long)r.p_lo,
                        (long long)r.p_hi);
        if (r.p_lo == r.p_hi) continue;
        it.p_lo = r.p_lo;
        it.p_hi = r.p_hi;
        // the state moves to the other row once the whole plan has run: swept
        // when its last level is odd, classic heat after an odd step count
        it.flip = r.p_hi == it.s.n_phases &&
                  (classic ? (p->desc.eq == SWP_HEAT && (it.s.T & 1)) : (it.s.top & 1) != 0);
        groups[p->desc.eq == SWP_EULER ? 1 : 0][p->desc.dtype].push_back(it);
    }
    return launch_groups(b, groups, threads, false);
}

swp_status set_error(swp_status s, const char* msg) { return fail(s, "%s", msg); }

swp_status advance_phases(swp_problem* p, int n, int64_t steps, int64_t p_lo, int64_t p_hi)
{
    if (!p) return fail(SWP_EINVAL, "problem is NULL");
    swp_status st = check_width(p, n);
    if (st != SWP_OK) return st;
    const SweptPlan s = plan_swept(p, steps, n);
    if (p_lo < 0 || p_hi > s.n_phases || p_lo > p_hi)
        return fail(SWP_EINVAL, "phases [%lld, %lld) outside the plan", (long long)p_lo, (long long)p_hi);
    if (p_lo == p_hi) return SWP_OK;
    // the same per-phase kernels and block size as swp_advance's per-phase launch
    const int threads = n >= 512 ? 256 : (n >= 128 ? 128 : 64);
    const int thr = p->desc.dtype == SWP_F32 ? std::max(64, std::min(256, n / 8)) / 32 * 32 : threads;
    st = p->desc.dtype == SWP_F64 ? run_swept_phases<double>(p, s, thr, p_lo, p_hi)
                                  : run_swept_phases<float>(p, s, thr, p_lo, p_hi);
    if (st != SWP_OK) return st;
    if (p_hi == s.n_phases && (s.top & 1)) p->cur = 1 - p->cur;
    return SWP_OK;
}

}  // namespace swp

extern "C" {

swp_status swp_batch_create(void* cuda_stream, swp_batch** out)
{
    if (!out) return fail(SWP_EINVAL, "out is NULL");
    *out = nullptr;
    swp_batch* b = new (std::nothrow) swp_batch();
    if (!b) return fail(SWP_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->wait_limit_ns = default_wait_limit_ns();
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        delete b;
        return fail(SWP_EDEVICE, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    e = cudaMalloc((void**)&b->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        swp_batch_destroy(b);
        return cuda_fail(e, "batch create");
    }
    *out = b;
    return SWP_OK;
}

swp_status swp_batch_advance(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps,
                             int32_t count, const int32_t* points_per_block, int32_t threads)
{
    return batch_advance(b, problems, n_steps, count, nullptr, SWP_SWEPT, points_per_block, threads,
                         SWP_LAUNCH_AUTO);
}

swp_status swp_batch_advance_ex(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps,
                                int32_t count, const int32_t* schemes, const int32_t* points_per_block,
                                int32_t threads, int32_t launch)
{
    return batch_advance(b, problems, n_steps, count, schemes, SWP_SCHEME_AUTO, points_per_block, threads, launch);
}

swp_status swp_batch_synchronize(swp_batch* b)
{
    if (!b) return fail(SWP_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronize");
    int st = 0;
    e = cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "batch status read");
    if (st != 0) {
        cudaMemset(b->status, 0, sizeof(int));
        return fail(SWP_ETIMEOUT, "a node's bounded wait gave up; the batch's states are invalid");
    }
    return SWP_OK;
}

swp_status swp_batch_destroy(swp_batch* b)
{
    if (!b) return SWP_OK;
    if (b->stream || b->status) cudaStreamSynchronize(b->stream);
    b->t.release();
    for (auto& g : b->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.t.release();
    }
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->status) cudaFree(b->status);
    if (b->stage) cudaFreeHost(b->stage);
    if (b->staged) cudaEventDestroy(b->staged);
    delete b;
    return SWP_OK;
}

int64_t swp_batch_kernel_launches(const swp_batch* b) { return b ? b->launches : -1; }

swp_status swp_autotune_width(const swp_desc* desc, const void* u0_host, int32_t batch_count,
                              int64_t steps, int32_t* best_n)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!u0_host || !best_n || batch_count <= 0 || steps <= 0)
        return fail(SWP_EINVAL, "u0_host / best_n NULL or count, steps <= 0");
    *best_n = 0;
    int n = 0;
    double rate = 0.0;
    if ((st = tune_swept(desc, u0_host, batch_count, steps, &n, &rate)) != SWP_OK) return st;
    *best_n = n;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    Tuned& t = g_tuned[std::make_tuple(desc->eq, desc->dtype, desc->n_points)];
    t.n_swept = n;
    if (t.scheme == SWP_SWEPT) t.n = n;
    return SWP_OK;
}

swp_status swp_autotune(const swp_desc* desc, const void* u0_host, int32_t batch_count, int64_t steps,
                        int32_t* best_scheme, int32_t* best_n)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!u0_host || !best_scheme || !best_n || batch_count <= 0 || steps <= 0)
        return fail(SWP_EINVAL, "u0_host / best_scheme / best_n NULL or count, steps <= 0");
    *best_scheme = SWP_SWEPT;
    *best_n = 0;
    int n = 0;
    double swept_rate = 0.0;
    if ((st = tune_swept(desc, u0_host, batch_count, steps, &n, &swept_rate)) != SWP_OK) return st;
    // classic in the same batched form: chunks of 256 .. 4096 points
    int cm = 0;
    double classic_rate = -1.0;
    swp_problem probe;
    probe.desc = *desc;
    probe.esize = esize_of(desc->dtype);
    probe.N = desc->n_points;
    probe.device = 0;
    cudaGetDevice(&probe.device);
    for (int m = 256; m <= 4096; m *= 4) {
        const int mm = (int)std::min<int64_t>(m, desc->n_points);
        if (check_chunk(&probe, mm) != SWP_OK) continue;
        const double r = time_batch(desc, u0_host, batch_count, steps, SWP_CLASSIC, mm, 256);
        if (r > classic_rate) {
            classic_rate = r;
            cm = mm;
        }
        if (mm == desc->n_points) break;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    Tuned& t = g_tuned[std::make_tuple(desc->eq, desc->dtype, desc->n_points)];
    t.n_swept = n;
    if (cm > 0 && classic_rate > swept_rate) {
        t.scheme = SWP_CLASSIC;
        t.n = cm;
    } else {
        t.scheme = SWP_SWEPT;
        t.n = n;
    }
    *best_scheme = t.scheme;
    *best_n = t.n;
    return SWP_OK;
}

swp_status swp_tuned_width(const swp_desc* desc, int32_t* n)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!n) return fail(SWP_EINVAL, "n is NULL");
    Tuned t;
    *n = tuned_of(*desc, &t) ? t.n_swept : 0;
    return SWP_OK;
}

swp_status swp_fit_width(int32_t eq, int64_t n_points, int32_t target, int32_t* n)
{
    if (!n) return fail(SWP_EINVAL, "n is NULL");
    *n = 0;
    if (eq != SWP_HEAT && eq != SWP_KS && eq != SWP_EULER) return fail(SWP_EINVAL, "unknown equation %d", eq);
    if (n_points <= 0 || target <= 0) return fail(SWP_EINVAL, "n_points and target must be > 0");
    *n = (int32_t)fitted_width(eq == SWP_HEAT ? 1 : 2, n_points, target);
    return SWP_OK;
}

swp_status swp_batch_tune_width(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps, int32_t count,
                                const int32_t* candidates, int32_t n_candidates, int32_t threads,
                                int32_t* widths_out, float* ms_out, int32_t* best)
{
    if (!b || !problems || !n_steps || !candidates || !widths_out)
        return fail(SWP_EINVAL, "batch, problems, n_steps, candidates or widths_out is NULL");
    if (count <= 0 || n_candidates <= 0) return fail(SWP_EINVAL, "count and n_candidates must be > 0");
    for (int32_t k = 0; k < n_candidates; ++k)
        if (candidates[k] <= 0) return fail(SWP_EINVAL, "candidate width %d must be > 0", k);
    for (int32_t i = 0; i < count; ++i) {
        if (!problems[i]) return fail(SWP_EINVAL, "problem %d is NULL", i);
        if (problems[i]->stream != b->stream) return fail(SWP_EINVAL, "problem %d uses another stream than the batch", i);
    }
    // the states, saved once and put back after every trial
    std::vector<size_t> off(count), bytes(count);
    std::vector<int> cur(count);
    size_t total = 0;
    for (int32_t i = 0; i < count; ++i) {
        const swp_problem* p = problems[i];
        bytes[i] = (size_t)p->nv * (size_t)p->N * (size_t)p->esize;
        off[i] = total;
        total += (bytes[i] + 255) / 256 * 256;
        cur[i] = p->cur;
    }
    char* saved = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&saved, total);
    if (e != cudaSuccess) return fail(SWP_ENOMEM, "no device memory to save the states (%zu bytes)", total);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int32_t i = 0; i < count && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(saved + off[i], problems[i]->rows[cur[i]], bytes[i], cudaMemcpyDeviceToDevice, b->stream);
    swp_status st = e == cudaSuccess ? SWP_OK : cuda_fail(e, "save states");
    std::vector<int32_t> w(count), best_w;
    float best_ms = 0.0f;
    int32_t best_k = -1;
    for (int32_t k = 0; k < n_candidates && st == SWP_OK; ++k) {
        for (int32_t i = 0; i < count; ++i) {
            swp_problem* p = problems[i];
            const int64_t n = fitted_width(p->rad, p->N, candidates[k]);
            w[i] = n > 0 && n <= INT32_MAX && check_width(p, (int)n) == SWP_OK ? (int32_t)n : 0;
        }
        e = cudaEventRecord(e0, b->stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "tune event"); break; }
        st = batch_advance(b, problems, n_steps, count, nullptr, SWP_SWEPT, w.data(), threads, SWP_LAUNCH_PERSISTENT);
        if (st == SWP_OK && (e = cudaEventRecord(e1, b->stream)) != cudaSuccess) st = cuda_fail(e, "tune event");
        if (st == SWP_OK) st = swp_batch_synchronize(b);
        float ms = 0.0f;
        if (st == SWP_OK && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) st = cuda_fail(e, "tune timing");
        // back to the saved states, whatever the trial did
        for (int32_t i = 0; i < count; ++i) {
            swp_problem* p = problems[i];
            const cudaError_t er = cudaMemcpyAsync(p->rows[cur[i]], saved + off[i], bytes[i], cudaMemcpyDeviceToDevice,
                                                   b->stream);
            if (er != cudaSuccess && st == SWP_OK) st = cuda_fail(er, "restore states");
            p->cur = cur[i];
        }
        if (st != SWP_OK) break;
        if (ms_out) ms_out[k] = ms;
        if (best_k < 0 || ms < best_ms) {
            best_ms = ms;
            best_k = k;
            best_w = w;
        }
    }
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess && st == SWP_OK) st = cuda_fail(e, "tune synchronize");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(saved);
    if (st != SWP_OK) return st;
    std::copy(best_w.begin(), best_w.end(), widths_out);
    if (best) *best = best_k;
    return SWP_OK;
}

swp_status swp_tuned(const swp_desc* desc, int32_t* scheme, int32_t* n)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!scheme || !n) return fail(SWP_EINVAL, "scheme or n is NULL");
    Tuned t;
    if (tuned_of(*desc, &t)) {
        *scheme = t.scheme;
        *n = t.n;
    } else {
        *scheme = SWP_SWEPT;
        *n = 0;
    }
    return SWP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Swept advance without allocation.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool or
// arena that owns all device memory, real-time loops that forbid allocation
// after start-up, or host environments that hand the library only
// pre-allocated device buffers.  swp_swept_noalloc serves them: the caller
// passes the state buffer, and the swept scheme's one piece of scratch, the
// odd-level row, lives in the file-scope array below.  It is sized for at
// most kNoAllocScratchBytes of state (8 MiB: 2^20 FP64 values), and every
// GPU that loads this library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// What the entry point needs to know about a device, looked up once per
// device under the mutex: the scratch array's device address and the SM
// count (the compute capability is checked at that time).
struct NoAllocDevice {
    void* scratch = nullptr;
    int sms = 0;
};
std::mutex g_noalloc_mutex;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// Set-up for the current device `dev`, once per device.  In host code the
// array's name only stands in for the symbol; the kernel must be given the
// address that cudaGetSymbolAddress returns with that device current.
swp_status noalloc_device(int dev, NoAllocDevice* out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SWP_EDEVICE, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.scratch) {
        int major = 0, minor = 0, sms = 0;
        cudaError_t e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(SWP_EDEVICE, "no usable CUDA device: %s", cudaGetErrorString(e));
        if (major != 10 || minor != 3)
            return fail(SWP_EDEVICE, "libswept is built for sm_103 (device is sm_%d%d)", major, minor);
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "scratch symbol address");
        d.sms = sms;
        d.scratch = ptr;
    }
    *out = d;
    return SWP_OK;
}

}  // namespace

extern "C" swp_status swp_swept_noalloc(const swp_desc* desc, void* state, int64_t n_steps,
                                        int32_t points_per_block, int32_t threads, void* cuda_stream)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!state) return fail(SWP_EINVAL, "state is NULL");
    if (n_steps < 0 || n_steps > ((int64_t)1 << 40)) return fail(SWP_EINVAL, "n_steps out of range");
    const size_t sbytes = state_bytes(desc);
    if (sbytes > kNoAllocScratchBytes)
        return fail(SWP_EINVAL, "state of %zu bytes exceeds the %zu-byte scratch of swp_swept_noalloc; "
                    "use swp_create / swp_advance for larger problems", sbytes, kNoAllocScratchBytes);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SWP_EDEVICE, "no usable CUDA device: %s", cudaGetErrorString(e));
    NoAllocDevice nd;
    st = noalloc_device(dev, &nd);
    if (st != SWP_OK) return st;
    void* scratch = nd.scratch;
    // the state must be device memory of the current device (the kernels
    // would otherwise read and write memory the caller did not mean)
    cudaPointerAttributes pa;
    e = cudaPointerGetAttributes(&pa, state);
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear the (non-sticky) error this query recorded
        return fail(SWP_EINVAL, "state is not a CUDA pointer: %s", cudaGetErrorString(e));
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
        return fail(SWP_EINVAL, "state must be device memory of the current device %d", dev);
    if (n_steps == 0) return SWP_OK;

    // a problem record on the stack whose two level rows are the caller's
    // state (even levels) and the scratch array (odd levels)
    swp_problem p;
    p.desc = *desc;
    p.nv = nv_of(desc->eq);
    p.rad = radius_of(desc->eq);
    p.sub = desc->eq == SWP_HEAT ? 1 : 2;
    p.esize = esize_of(desc->dtype);
    p.N = desc->n_points;
    p.rows[0] = state;
    p.rows[1] = scratch;
    p.cur = 0;
    p.stream = (cudaStream_t)cuda_stream;
    p.device = dev;
    p.sms = nd.sms;
    make_coefs<double>(desc, p.cd);
    make_coefs<float>(desc, p.cf);
    swp_advance_opts o;
    o.scheme = SWP_SWEPT;
    o.points_per_block = points_per_block;
    o.launch = SWP_LAUNCH_PER_PHASE;
    o.threads = threads;
    st = desc->dtype == SWP_F64 ? advance_typed<double>(&p, n_steps, o) : advance_typed<float>(&p, n_steps, o);
    if (st != SWP_OK) return st;
    if (p.cur == 1) {
        // the last level was odd: the result sits in the scratch row
        e = cudaMemcpyAsync(state, scratch, sbytes, cudaMemcpyDeviceToDevice, p.stream);
        if (e != cudaSuccess) return cuda_fail(e, "result copy from scratch");
    }
    return SWP_OK;
}
