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
#include <cstring>
#include <new>
#include <string>

#include "../../include/swept.h"
#include "launch.h"

using namespace swp;

struct swp_problem {
    swp_desc desc;
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
    // persistent swept launch
    uint32_t* flags = nullptr;
    int flags_k = 0;          // capacity of flags
    int flags_last_k = -1;    // node count the flags were last used with
    uint32_t flag_base = 0;
    int inject_withheld_flags = 0;            // test hook: waits never succeed
    uint64_t wait_limit_ns = 2000000000ull;   // bound of one neighbour wait
    unsigned int* counter = nullptr;
    int* status = nullptr;
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

// A swept node width must divide N, be a multiple of 4 rad (so that H is
// even) and fit the node's working set in shared memory.
swp_status check_width(const swp_problem* p, int n)
{
    const int step = 4 * p->rad;
    if (n < step || n % step) return fail(SWP_EINVAL, "points_per_block %d must be a positive multiple of %d", n, step);
    if (p->N % n) return fail(SWP_EINVAL, "points_per_block %d must divide n_points %lld", n, (long long)p->N);
    if (p->N / n > 0x7FFFFFFF) return fail(SWP_EINVAL, "points_per_block %d gives more than 2^31 - 1 nodes", n);
    if (swept_smem_bytes(p->desc.eq, n, p->esize) > max_smem(p->device))
        return fail(SWP_EINVAL, "points_per_block %d needs %zu bytes of shared memory (max %zu)", n,
                    swept_smem_bytes(p->desc.eq, n, p->esize), max_smem(p->device));
    return SWP_OK;
}

// Default node width, from the widths measured fastest on GB300 for single
// problems: about N / 1024 points for heat and KS (at least 64 and 128, at
// most 1024) and N / 256 for Euler (64 to 512); the nearest width that
// divides N, is a multiple of 4 rad and fits shared memory.
int default_width(const swp_problem* p)
{
    const int step = 4 * p->rad;
    const bool euler = p->desc.eq == SWP_EULER;
    const int lo = (p->desc.eq == SWP_HEAT || euler) ? 64 : 128;
    const int cap = euler ? 512 : 1024;
    int64_t target = p->N / (euler ? 256 : 1024);
    if (target < lo) target = lo;
    if (target > cap) target = cap;
    if (target > p->N / 2) target = p->N / 2;
    for (int64_t n = target; n >= step; --n)
        if (n % step == 0 && p->N % n == 0 && check_width(p, (int)n) == SWP_OK) return (int)n;
    for (int64_t n = target + 1; n <= cap && n <= p->N; ++n)
        if (n % step == 0 && p->N % n == 0 && check_width(p, (int)n) == SWP_OK) return (int)n;
    return 0;
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
    int64_t T, Q, r, n_phases;
    int top;   // relative level of the last phase's top row
};

SweptPlan plan_swept(const swp_problem* p, int64_t steps, int n)
{
    SweptPlan s;
    s.n = n;
    s.H = n / (2 * p->rad);
    s.K = (int)(p->N / n);
    s.T = steps * p->sub;
    s.Q = s.T / s.H;
    s.r = s.T % s.H;
    s.n_phases = s.r > 0 ? s.Q + 2 : s.Q + 1;
    s.top = s.r > 0 ? (int)s.r : s.H;
    return s;
}

template <typename R>
swp_status run_swept_register(swp_problem* p, const SweptPlan& s, int threads)
{
    R* A = (R*)p->rows[p->cur];
    R* B = (R*)p->rows[1 - p->cur];
    const Coefs<R>& c = coefs_of<R>(p);
    for (int64_t ph = 0; ph < s.n_phases; ++ph) {
        PhaseGeom g;
        g.N = p->N;
        g.n = s.n;
        g.H = s.H;
        g.K = s.K;
        g.j_lo = ph == 0 ? s.H + 1 : 1;
        g.j_hi = ph < s.Q ? 2 * s.H - 1 : (ph == s.Q ? s.H + (int)s.r : (int)s.r);
        g.odd = (int)(ph & 1);
        cudaError_t e = launch_swept_register<R>(p->desc.eq, A, B, g, c, threads, p->stream);
        p->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "register swept launch");
    }
    return SWP_OK;
}

template <typename R>
swp_status run_swept_phases(swp_problem* p, const SweptPlan& s, int threads)
{
    R* A = (R*)p->rows[p->cur];
    R* B = (R*)p->rows[1 - p->cur];
    const Coefs<R>& c = coefs_of<R>(p);
    for (int64_t ph = 0; ph < s.n_phases; ++ph) {
        PhaseGeom g;
        g.N = p->N;
        g.n = s.n;
        g.H = s.H;
        g.K = s.K;
        g.j_lo = ph == 0 ? s.H + 1 : 1;
        g.j_hi = ph < s.Q ? 2 * s.H - 1 : (ph == s.Q ? s.H + (int)s.r : (int)s.r);
        g.odd = (int)(ph & 1);
        cudaError_t e = launch_swept_phase<R>(p->desc.eq, p->desc.bc, A, B, g, c, threads, p->stream);
        p->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "swept phase launch");
    }
    return SWP_OK;
}

swp_status ensure_persistent_state(swp_problem* p, int K)
{
    if (p->flags && p->flags_k >= K) return SWP_OK;
    if (p->flags) cudaFree(p->flags);
    p->flags = nullptr;
    cudaError_t e = cudaMalloc(&p->flags, sizeof(uint32_t) * (size_t)K);
    if (e != cudaSuccess) return fail(SWP_ENOMEM, "flags: %s", cudaGetErrorString(e));
    e = cudaMemsetAsync(p->flags, 0, sizeof(uint32_t) * (size_t)K, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "flags memset");
    p->flags_k = K;
    p->flag_base = 0;
    if (!p->counter) {
        e = cudaMalloc(&p->counter, sizeof(unsigned int) + sizeof(int) * 4);
        if (e != cudaSuccess) return fail(SWP_ENOMEM, "counter: %s", cudaGetErrorString(e));
        p->status = reinterpret_cast<int*>(p->counter + 1);
        e = cudaMemsetAsync(p->counter, 0, sizeof(unsigned int) + sizeof(int) * 4, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "status memset");
    }
    return SWP_OK;
}

template <typename R>
swp_status run_swept_persistent(swp_problem* p, const SweptPlan& s, int threads)
{
    swp_status st = ensure_persistent_state(p, s.K);
    if (st != SWP_OK) return st;
    // flags count completed phases per node; restart the count when the node
    // layout changes or the count would wrap
    if (p->flags_last_k != s.K || (uint64_t)p->flag_base + (uint64_t)s.n_phases >= (1ull << 30)) {
        cudaError_t e = cudaMemsetAsync(p->flags, 0, sizeof(uint32_t) * (size_t)p->flags_k, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "flags reset");
        p->flag_base = 0;
        p->flags_last_k = s.K;
    }
    const int64_t total = s.n_phases * (int64_t)s.K;
    if (total >= ((int64_t)1 << 31)) return fail(SWP_EINVAL, "advance too long for one persistent launch");
    const int bps = swept_persistent_blocks_per_sm<R>(p->desc.eq, s.n, threads);
    if (bps <= 0) return fail(SWP_EINVAL, "persistent kernel does not fit (n=%d, threads=%d)", s.n, threads);
    // enough blocks for about two phases in flight: more would only poll the
    // flags of phases that cannot start yet
    int64_t blocks = (int64_t)p->sms * bps;
    if (blocks > 2 * (int64_t)s.K) blocks = 2 * (int64_t)s.K > p->sms ? 2 * (int64_t)s.K : p->sms;
    if (blocks > total) blocks = total;
    PersistentPlan plan;
    plan.N = p->N;
    plan.n = s.n;
    plan.H = s.H;
    plan.K = s.K;
    plan.Q = s.Q;
    plan.r = s.r;
    plan.n_phases = s.n_phases;
    plan.flag_base = p->flag_base;
    plan.wait_offset = p->inject_withheld_flags ? (1u << 30) : 0u;
    plan.wait_limit_ns = p->wait_limit_ns;
    cudaError_t e = launch_swept_persistent<R>(p->desc.eq, p->desc.bc, (R*)p->rows[p->cur],
                                               (R*)p->rows[1 - p->cur], plan, coefs_of<R>(p), p->flags,
                                               p->counter, p->status, threads, (int)blocks, p->stream);
    p->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "persistent swept launch");
    p->flag_base += (uint32_t)s.n_phases;
    return SWP_OK;
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
        p->flags_last_k = -1;   // flags are inconsistent: restart them next time
        return fail(SWP_ETIMEOUT, "a node's bounded wait for its neighbours gave up; the state is invalid");
    }
    return SWP_OK;
}

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
    swp_status st = scheme == SWP_CLASSIC ? run_classic<R>(p, steps, threads) : run_swept_phases<R>(p, *s, threads);
    p->stream = user;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->capture_stream, &graph);
    if (st != SWP_OK) {
        if (graph) cudaGraphDestroy(graph);
        p->cur = g.cur_before;
        p->launches = launches0;
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    if (scheme == SWP_SWEPT && (s->top & 1)) p->cur = 1 - p->cur;
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

template <typename R>
swp_status advance_typed(swp_problem* p, int64_t steps, const swp_advance_opts& o)
{
    if (o.scheme == SWP_CLASSIC) {
        if (o.launch == SWP_LAUNCH_GRAPH) {
            const int thr = o.threads <= 0 ? 256 : o.threads;
            if (thr > 256 || thr % 32) return fail(SWP_EINVAL, "classic threads must be a multiple of 32 <= 256");
            return run_graph<R>(p, steps, SWP_CLASSIC, 0, thr, nullptr);
        }
        return run_classic<R>(p, steps, o.threads);
    }
    if (o.launch == SWP_LAUNCH_REGISTER) {
        if (p->desc.eq == SWP_EULER || p->desc.bc != SWP_BC_PERIODIC)
            return fail(SWP_EUNSUPPORTED, "the register variant runs periodic heat and KS");
        if (o.points_per_block != 0 && o.points_per_block != 32)
            return fail(SWP_EINVAL, "the register variant's node is one warp: points_per_block 32 (or 0)");
        if (p->N % 32 || p->N < 64) return fail(SWP_EINVAL, "the register variant needs n_points a multiple of 32, >= 64");
        const int thr = o.threads == 0 ? 256 : o.threads;
        if (thr < 32 || thr > 256 || thr % 32) return fail(SWP_EINVAL, "threads must be a multiple of 32 in [32, 256]");
        const SweptPlan s = plan_swept(p, steps, 32);
        if (s.T == 0) return SWP_OK;
        swp_status st = run_swept_register<R>(p, s, thr);
        if (st != SWP_OK) return st;
        if (s.top & 1) p->cur = 1 - p->cur;
        return SWP_OK;
    }
    int n = o.points_per_block;
    if (n == 0) {
        n = default_width(p);
        if (n == 0) return fail(SWP_EINVAL, "no valid node width for n_points %lld", (long long)p->N);
    }
    swp_status st = check_width(p, n);
    if (st != SWP_OK) return st;
    int threads = o.threads;
    if (threads == 0) threads = n >= 512 ? 256 : (n >= 128 ? 128 : 64);
    const int max_threads = p->desc.eq == SWP_EULER ? 256 : 1024;
    if (threads < 32 || threads > max_threads || threads % 32)
        return fail(SWP_EINVAL, "threads must be a multiple of 32 in [32, %d]", max_threads);
    const SweptPlan s = plan_swept(p, steps, n);
    if (s.T == 0) return SWP_OK;
    int launch = o.launch == SWP_LAUNCH_AUTO ? SWP_LAUNCH_PER_PHASE : o.launch;
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
    if (opts->scheme != SWP_CLASSIC && opts->scheme != SWP_SWEPT)
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
    if (p->flags) cudaFree(p->flags);
    if (p->counter) cudaFree(p->counter);
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
// Batched swept advance and node-width autotuner.
// ---------------------------------------------------------------------------
struct swp_batch {
    cudaStream_t stream = nullptr;
    int device = 0, sms = 0;
    int64_t launches = 0;
    // device workspace, grown on demand
    void* insts = nullptr;   size_t insts_cap = 0;
    int2* tasks = nullptr;   size_t tasks_cap = 0;
    int* ctr = nullptr;      size_t ctr_cap = 0;     // [0] = cur_task, [1] = status, [2..] = task counters
    uint32_t* flags = nullptr; size_t flags_cap = 0;
    uint64_t wait_limit_ns = 2000000000ull;
};

namespace {

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int64_t>, int> g_tuned;   // (eq, dtype, N) -> node width

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

// Node width for a problem: the tuned value for (eq, dtype, N) if the tuner
// measured one, else the default rule.
int width_for(const swp_problem* p)
{
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(std::make_tuple(p->desc.eq, p->desc.dtype, p->N));
        if (it != g_tuned.end() && check_width(p, it->second) == SWP_OK) return it->second;
    }
    return default_width(p);
}

struct BatchItem {
    swp_problem* p;
    SweptPlan s;
};

template <typename R>
swp_status batch_group(swp_batch* b, const std::vector<BatchItem>& items, int mode, int threads)
{
    std::vector<BatchInst<R>> insts(items.size());
    int64_t flags = 0, max_phases = 0;
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
        in.bc = it.p->desc.bc;
        in.Q = it.s.Q;
        in.r = it.s.r;
        in.n_phases = it.s.n_phases;
        in.flag_off = (int)flags;
        in.eq = it.p->desc.eq;
        in.c = coefs_of<R>(it.p);
        flags += it.s.K;
        max_phases = std::max(max_phases, it.s.n_phases);
        smem = std::max(smem, swept_smem_bytes(it.p->desc.eq, it.s.n, it.p->esize));
    }
    // (instance, phase) tasks in order of estimated start: phase p of instance
    // i at p * c_i, with c_i the cost of one of its phase items (levels times
    // FP64 operations per point, times the warp rows of its widest level).
    // Each instance keeps its phases in order, so every item depends only on
    // items of earlier tasks; instances with short items run ahead instead of
    // waiting, phase by phase, for instances with long ones.
    struct Key {
        double start;
        int inst, phase;
    };
    std::vector<Key> keys;
    for (size_t i = 0; i < items.size(); ++i) {
        const auto& s = items[i].s;
        const double ops = items[i].p->desc.eq == SWP_HEAT ? 3.0 : (items[i].p->desc.eq == SWP_KS ? 7.0 : 260.0);
        const double rows = std::max(1.0, (double)s.n / 256.0);
        const double cost = (2.0 * s.H - 1.0) * ops * rows;
        for (int64_t ph = 0; ph < s.n_phases; ++ph) keys.push_back(Key{(double)ph * cost, (int)i, (int)ph});
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
        return x.start < y.start || (x.start == y.start && x.phase < y.phase);
    });
    std::vector<int2> tasks(keys.size());
    for (size_t t = 0; t < keys.size(); ++t) tasks[t] = make_int2(keys[t].inst, keys[t].phase);
    if (tasks.size() >= (size_t)1 << 30 || flags >= (int64_t)1 << 30)
        return fail(SWP_EINVAL, "batch too large for one launch");
    swp_status st;
    if ((st = grow(&b->insts, &b->insts_cap, sizeof(BatchInst<R>) * insts.size())) != SWP_OK) return st;
    if ((st = grow((void**)&b->tasks, &b->tasks_cap, sizeof(int2) * tasks.size())) != SWP_OK) return st;
    if ((st = grow((void**)&b->ctr, &b->ctr_cap, sizeof(int) * (tasks.size() + 2))) != SWP_OK) return st;
    if ((st = grow((void**)&b->flags, &b->flags_cap, sizeof(uint32_t) * (size_t)flags)) != SWP_OK) return st;
    cudaError_t e = cudaMemcpyAsync(b->insts, insts.data(), sizeof(BatchInst<R>) * insts.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tasks, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctr, 0, sizeof(int) * (tasks.size() + 2), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->flags, 0, sizeof(uint32_t) * (size_t)flags, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch table upload");
    // the staging vectors die at return: wait for the copies out of them
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch table upload");
    BatchWork w;
    w.tasks = b->tasks;
    w.cur_task = b->ctr;
    w.status = b->ctr + 1;
    w.task_ctr = b->ctr + 2;
    w.ntasks = (int)tasks.size();
    w.smem_bytes = smem;
    w.flags = b->flags;
    w.wait_limit_ns = b->wait_limit_ns;
    const int bps = swept_batch_blocks_per_sm<R>(mode, smem, threads);
    if (bps <= 0) return fail(SWP_EINVAL, "batch kernel does not fit (%zu bytes of shared memory, threads=%d)", smem, threads);
    int64_t blocks = (int64_t)b->sms * bps;
    int64_t items_total = 0;
    for (auto& it : items) items_total += it.s.n_phases * it.s.K;
    if (blocks > items_total) blocks = items_total;
    e = launch_swept_batch<R>(mode, (const BatchInst<R>*)b->insts, w, threads, (int)blocks, b->stream);
    b->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    for (auto& it : items) {
        it.p->launches++;
        if (it.s.top & 1) it.p->cur = 1 - it.p->cur;
    }
    return SWP_OK;
}

// Time `reps` advances of `steps` timesteps of `count` copies of a problem in
// one batch at node width n; returns point-updates per second or < 0.
double time_width(const swp_desc* desc, const void* u0, int count, int64_t steps, int n, int threads,
                  cudaStream_t stream)
{
    std::vector<swp_problem*> probs;
    double rate = -1.0;
    swp_batch* b = nullptr;
    std::vector<int64_t> st(count, steps);
    std::vector<int32_t> nn(count, n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (swp_batch_create(stream, &b) != SWP_OK) return -1.0;
    for (int i = 0; i < count; ++i) {
        swp_problem* p = nullptr;
        if (swp_create(desc, u0, 0, stream, &p) != SWP_OK) goto done;
        probs.push_back(p);
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    if (swp_batch_advance(b, probs.data(), st.data(), count, nn.data(), threads) != SWP_OK) goto done;
    if (swp_batch_synchronize(b) != SWP_OK) goto done;
    cudaEventRecord(e0, stream);
    if (swp_batch_advance(b, probs.data(), st.data(), count, nn.data(), threads) != SWP_OK) goto done;
    cudaEventRecord(e1, stream);
    if (swp_batch_synchronize(b) == SWP_OK) {
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

}  // namespace

extern "C" {

swp_status swp_batch_create(void* cuda_stream, swp_batch** out)
{
    if (!out) return fail(SWP_EINVAL, "out is NULL");
    *out = nullptr;
    swp_batch* b = new (std::nothrow) swp_batch();
    if (!b) return fail(SWP_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        delete b;
        return fail(SWP_EDEVICE, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    *out = b;
    return SWP_OK;
}

swp_status swp_batch_advance(swp_batch* b, swp_problem* const* problems, const int64_t* n_steps,
                             int32_t count, const int32_t* points_per_block, int32_t threads)
{
    if (!b || !problems || !n_steps) return fail(SWP_EINVAL, "batch, problems or n_steps is NULL");
    if (count < 0) return fail(SWP_EINVAL, "count must be >= 0");
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
        if (n_steps[i] == 0) continue;
        int n = points_per_block ? points_per_block[i] : 0;
        if (n == 0) n = width_for(p);
        if (n == 0) return fail(SWP_EINVAL, "no valid node width for problem %d", i);
        swp_status st = check_width(p, n);
        if (st != SWP_OK) return st;
        BatchItem it;
        it.p = p;
        it.s = plan_swept(p, n_steps[i], n);
        groups[p->desc.eq == SWP_EULER ? 1 : 0][p->desc.dtype].push_back(it);
        if (p->desc.eq == SWP_EULER) max_threads = 256;
    }
    if (threads == 0) threads = 256;
    if (threads < 32 || threads > max_threads || threads % 32)
        return fail(SWP_EINVAL, "threads must be a multiple of 32 in [32, %d]", max_threads);
    for (int g = 0; g < 2; ++g)
        for (int dt = 0; dt < 2; ++dt) {
            if (groups[g][dt].empty()) continue;
            const int mode = g == 1 ? SWP_EULER : SWP_HEAT;
            const int thr = (g == 1 && threads > 256) ? 256 : threads;
            swp_status st = dt == SWP_F64 ? batch_group<double>(b, groups[g][dt], mode, thr)
                                          : batch_group<float>(b, groups[g][dt], mode, thr);
            if (st != SWP_OK) return st;
        }
    return SWP_OK;
}

swp_status swp_batch_synchronize(swp_batch* b)
{
    if (!b) return fail(SWP_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronize");
    if (b->ctr) {
        int st = 0;
        e = cudaMemcpy(&st, b->ctr + 1, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "batch status read");
        if (st != 0) {
            cudaMemset(b->ctr + 1, 0, sizeof(int));
            return fail(SWP_ETIMEOUT, "a node's bounded wait gave up; the batch's states are invalid");
        }
    }
    return SWP_OK;
}

swp_status swp_batch_destroy(swp_batch* b)
{
    if (!b) return SWP_OK;
    if (b->insts) cudaFree(b->insts);
    if (b->tasks) cudaFree(b->tasks);
    if (b->ctr) cudaFree(b->ctr);
    if (b->flags) cudaFree(b->flags);
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
    swp_problem probe;   // for the width checks only
    probe.desc = *desc;
    probe.rad = radius_of(desc->eq);
    probe.nv = nv_of(desc->eq);
    probe.esize = esize_of(desc->dtype);
    probe.N = desc->n_points;
    if (cudaGetDevice(&probe.device) != cudaSuccess) return fail(SWP_EDEVICE, "no CUDA device");
    const int cap = desc->eq == SWP_EULER ? 1024 : 4096;
    double best = -1.0;
    for (int n = 32; n <= cap && n <= probe.N; n *= 2) {
        if (check_width(&probe, n) != SWP_OK || probe.N / n < 2) continue;
        const int threads = desc->eq == SWP_EULER ? 128 : (n >= 512 ? 256 : 128);
        const double rate = time_width(desc, u0_host, batch_count, steps, n, threads, nullptr);
        if (rate > best) {
            best = rate;
            *best_n = n;
        }
    }
    if (*best_n == 0) return fail(SWP_EINVAL, "no node width could be timed for n_points %lld", (long long)probe.N);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[std::make_tuple(desc->eq, desc->dtype, desc->n_points)] = *best_n;
    return SWP_OK;
}

swp_status swp_tuned_width(const swp_desc* desc, int32_t* n)
{
    swp_status st = check_desc(desc);
    if (st != SWP_OK) return st;
    if (!n) return fail(SWP_EINVAL, "n is NULL");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(std::make_tuple(desc->eq, desc->dtype, desc->n_points));
    *n = it == g_tuned.end() ? 0 : it->second;
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

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device `dev`, looked up
// once per device.  In host code the array's name only stands in for the
// symbol; the kernel must be given this address.
swp_status noalloc_scratch(int dev, void** out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SWP_EDEVICE, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "scratch symbol address");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
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
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return fail(SWP_EDEVICE, "no usable CUDA device: %s", cudaGetErrorString(e));
    if (prop.major != 10 || prop.minor != 3)
        return fail(SWP_EDEVICE, "libswept is built for sm_103 (device is sm_%d%d)", prop.major, prop.minor);
    void* scratch = nullptr;
    st = noalloc_scratch(dev, &scratch);
    if (st != SWP_OK) return st;
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
    p.sms = prop.multiProcessorCount;
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
