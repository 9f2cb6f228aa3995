// C-ABI of libasicp (declared in include/asicp.h): context, inputs, the
// iteration loop of Algorithm 1 and result read-back.  Host code only; every
// arithmetic step of the method runs in the kernels of k_match.cu,
// k_collision.cu and k_update.cu.
//
// A context holds n_objects objects (one grasp set each) that are optimised
// together: every kernel covers the particles of all objects, each particle
// matched against its own object's cloud.  Particles are numbered object by
// object, preshape by preshape (groups g = o * P + p of K_g particles).
#include "../../include/asicp.h"
#include "asicp_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <utility>
#include <vector>

using namespace asicp;
static_assert(kFwdVariants == ASICP_FWD_SHAPES, "kernel shape count differs from the header");

namespace {

struct Err {
    asicp_status st;
    std::string msg;
};

[[noreturn]] void fail(asicp_status st, const std::string &msg) { throw Err{st, msg}; }

void ck(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(ASICP_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    fail(ASICP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device allocation owned by the context; grows on demand, never shrinks.
struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    ~DevMem() { if (p) cudaFree(p); }
    void ensure(size_t want, const char *what)
    {
        if (want <= bytes && p) return;
        if (p) { cudaFree(p); p = nullptr; bytes = 0; }
        if (want == 0) want = 16;
        ck(cudaMalloc(&p, want), what);
        bytes = want;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct ObjBufs {
    DevMem R, Rx, Rt, C;      // C stays empty when the collision cloud is R itself
    int M = 0, Mpad = 0, Mc = 0;
    bool set = false;
};

enum { kTimeMatch = 0, kTimeCollide = 1, kTimeCollideNN = 2, kTimeFinalize = 3, kTimeStein = 4, kTimeExact = 5,
       kTimeKinds = 6 };
static_assert(kTimeKinds == ASICP_KERNEL_KINDS, "kernel kinds");

}  // namespace

struct asicp_ctx {
    asicp_config cfg{};
    cudaStream_t st = nullptr;
    std::string err;
    int N = 0;
    int nobj = 1;
    std::vector<int> Kg;              // particles per group, [nobj * P]
    std::vector<ObjBufs> objs;
    bool theta_set = false, stepped = false, run_done = false;
    std::vector<char> pre_set;
    std::vector<SdfMeta> meta;
    std::vector<DevMem> grids;
    std::vector<DevMem> cells;         // corner-packed grids
    int k_next = 0;

    // mini-batches of the object cloud per iteration (Table I), one object only
    std::vector<int> mb_off;          // [iters + 1] on the host (sizes are fixed at capture)
    long long mb_version = 0;         // bumped by every asicp_set_minibatch
    DevMem mb_idx, mb_R, mb_Rx;

    int fwd_variant = 0;              // forward-matching kernel shape (autotuner's choice)
    bool tuned = false;
    bool expire_test = false;         // the float32 matching kernels' first copy waits expire (testing)

    // layout (rebuilt when objects, particle counts or N change)
    bool layout_dirty = true;
    int T = 0, G = 0, n_items = 0;
    long long colidx_total = 0, csum_total = 0;
    std::vector<int> grp_off_h;
    std::vector<ObjMeta> objmeta_h;

    DevMem partgrp, grpoff, objmeta, items, ctaoff, com, frame, colitems, collist, box, stage, S, pconst, dmeta, theta, fsums,
        csums, ncol, colidx, cost, grad, prev, frozen, phi, h, order, errw, out7, outc, outi, nnidx, tccand, dbg_d2, dbg_sp,
        dbg_colnn;

    // profiling: events recorded around launches (kind, start, stop)
    struct Ev { int kind; cudaEvent_t a, b; };
    std::vector<Ev> events;
    std::vector<cudaEvent_t> pool;
    double acc_ms[kTimeKinds] = {};
    long long acc_n[kTimeKinds] = {};

    // CUDA graph of asicp_run's iteration loop (captured once per buffer layout)
    cudaStream_t cap_st = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    std::vector<const void *> loop_key;
    std::vector<Ev> graph_events;     // event pairs inside the graph (profile = 1)
    bool graph_pending = false;       // a replay's events have not been accumulated yet
    bool capturing = false;

    bool inputs_ready() const
    {
        if (N == 0) return false;
        for (const auto &o : objs) if (!o.set) return false;
        for (char c : pre_set) if (!c) return false;
        return true;
    }
    Layout layout() const
    {
        Layout L;
        L.P = cfg.P;
        L.N = N;
        L.G = G;
        L.nobj = nobj;
        L.T = T;
        L.part_grp = partgrp.as<int>();
        L.grp_off = grpoff.as<int>();
        L.obj = objmeta.as<ObjMeta>();
        L.com = com.as<double>();
        L.frame = frame.as<float4>();
        return L;
    }
    cudaEvent_t take_event()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        ck(cudaEventCreate(&e), "cudaEventCreate");
        return e;
    }
    ~asicp_ctx()
    {
        for (auto &e : events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
        for (auto &e : graph_events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
        for (auto e : pool) cudaEventDestroy(e);
        if (loop_exec) cudaGraphExecDestroy(loop_exec);
        if (cap_st) cudaStreamDestroy(cap_st);
    }
};

namespace {

template <class F>
asicp_status guarded(asicp_ctx *ctx, F &&f)
{
    if (!ctx) return ASICP_ERR_INVALID_ARG;
    try {
        f();
        ctx->err.clear();
        return ASICP_OK;
    } catch (const Err &e) {
        ctx->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        ctx->err = "host allocation failed";
        return ASICP_ERR_OOM;
    } catch (...) {
        ctx->err = "unexpected internal error";
        return ASICP_ERR_CUDA;
    }
}

void sync_and_check_err(asicp_ctx *c, const char *what)
{
    ck(cudaStreamSynchronize(c->st), what);
    int e = 0;
    ck(cudaMemcpy(&e, c->errw.p, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (e == kDevNonFinite) {
        ck(cudaMemsetAsync(c->errw.p, 0, sizeof(int), c->st), "clear error word");
        fail(ASICP_ERR_INVALID_ARG, std::string(what) + ": non-finite value in the input");
    }
    if (e == kDevTimeout) {
        ck(cudaMemsetAsync(c->errw.p, 0, sizeof(int), c->st), "clear error word");
        fail(ASICP_ERR_TIMEOUT, std::string(what) + ": a bounded device wait expired");
    }
}

double gamma_of(const asicp_config &c, int k)
{
    if (c.schedule == 1) {
        if (c.k_max <= 1) return c.g1;
        return c.g0 + (double)(c.g1 - c.g0) * k / (double)(c.k_max - 1);
    }
    const double period = (double)c.k_max / c.C_cycles;          // Eq. 11 with T = k_max
    return std::pow(std::fmod((double)k, period) / period, (double)c.p_exp);
}

// Offsets, work items and buffers for the current objects, particle counts and N.
// Work plan of the forward matching for kernel shape v.  Items are whole
// multiples of the shape's CTA size (at most threads x queries per thread) of one
// object, sized so that about kPlanRounds items of equal cost fall to each CTA
// of the persistent grid; they are dealt out longest first, each to the CTA
// with the least work so far (cost = queries x padded object points), and
// every CTA gets a contiguous range of the item table.
void plan_fwd_items(asicp_ctx *c, int v)
{
    constexpr int kPlanRounds = 3;
    const int grid = fwd_shape_grid(v), threads = fwd_shape_threads(v), qmax = fwd_shape_queries(v), N = c->N;
    const std::vector<ObjMeta> &om = c->objmeta_h;
    double W = 0.0;
    for (const ObjMeta &m : om) W += (double)m.np * N * m.Mpad;
    const double unit = W / ((double)grid * kPlanRounds);
    std::vector<FwdItem> items;
    for (int o = 0; o < (int)om.size(); ++o) {
        const ObjMeta &m = om[o];
        long long nq = (long long)std::ceil(unit / std::max(1, m.Mpad) / threads) * threads;
        nq = std::min<long long>(std::max<long long>(nq, threads), qmax);
        const long long q0 = (long long)m.pfirst * N, q1 = (long long)(m.pfirst + m.np) * N;
        for (long long q = q0; q < q1; q += nq) {
            FwdItem it;
            it.q0 = q;
            it.nq = (int)std::min<long long>(nq, q1 - q);
            it.obj = o;
            items.push_back(it);
        }
    }
    auto cost = [&](const FwdItem &x) { return (long long)x.nq * om[x.obj].Mpad; };
    std::stable_sort(items.begin(), items.end(), [&](const FwdItem &x, const FwdItem &y) { return cost(x) > cost(y); });
    // least-loaded CTA first (ties: lowest CTA index)
    using Slot = std::pair<long long, int>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int b = 0; b < grid; ++b) heap.push({0, b});
    std::vector<int> owner(items.size());
    std::vector<int> count(grid + 1, 0);
    for (size_t i = 0; i < items.size(); ++i) {
        Slot s = heap.top();
        heap.pop();
        owner[i] = s.second;
        ++count[s.second + 1];
        heap.push({s.first + cost(items[i]), s.second});
    }
    std::vector<int> off(grid + 1, 0);
    for (int b = 0; b < grid; ++b) off[b + 1] = off[b] + count[b + 1];
    std::vector<FwdItem> placed(items.size());
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (size_t i = 0; i < items.size(); ++i) placed[fill[owner[i]]++] = items[i];

    c->items.ensure(sizeof(FwdItem) * std::max<size_t>(1, placed.size()), "matching work items");
    c->ctaoff.ensure(sizeof(int) * (grid + 1), "matching work plan");
    if (!placed.empty())
        ck(cudaMemcpyAsync(c->items.p, placed.data(), sizeof(FwdItem) * placed.size(), cudaMemcpyHostToDevice, c->st),
           "work items");
    ck(cudaMemcpyAsync(c->ctaoff.p, off.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice, c->st),
       "work plan");
    ck(cudaStreamSynchronize(c->st), "work plan");
    c->n_items = (int)placed.size();
}

void build_layout(asicp_ctx *c)
{
    if (!c->layout_dirty) return;
    if (!c->inputs_ready()) fail(ASICP_ERR_STATE, "objects and every preshape must be set first");
    const int P = c->cfg.P, G = c->nobj * P, N = c->N;
    std::vector<int> off(G + 1, 0);
    for (int g = 0; g < G; ++g) off[g + 1] = off[g] + c->Kg[g];
    const int T = off[G];
    std::vector<int> part_grp(T);
    for (int g = 0; g < G; ++g)
        for (int i = off[g]; i < off[g + 1]; ++i) part_grp[i] = g;
    std::vector<ObjMeta> om(c->nobj);
    long long colidx_total = 0, csum_total = 0;
    for (int o = 0; o < c->nobj; ++o) {
        const ObjBufs &b = c->objs[o];
        ObjMeta &m = om[o];
        m.R = b.R.as<float4>();
        m.Rx = b.Rx.as<ulonglong2>();
        m.Rt = b.Rt.as<float>();
        m.C = b.C.p ? b.C.as<float4>() : b.R.as<float4>();
        m.M = b.M;
        m.Mpad = b.Mpad;
        m.Mc = b.Mc;
        m.chunks = (b.Mc + kColChunk - 1) / kColChunk;
        m.pfirst = off[o * P];
        m.np = off[(o + 1) * P] - off[o * P];
        m.colidx_base = colidx_total;
        m.csum_base = csum_total;
        colidx_total += (long long)m.np * m.Mc;
        csum_total += (long long)m.np * m.chunks;
    }

    if (T != c->T) {
        c->theta_set = false;
        c->run_done = false;
    }
    c->T = T;
    c->G = G;
    c->colidx_total = colidx_total;
    c->csum_total = csum_total;
    c->grp_off_h = off;
    c->objmeta_h = om;

    c->partgrp.ensure(sizeof(int) * T, "particle groups");
    c->grpoff.ensure(sizeof(int) * (G + 1), "group offsets");
    c->objmeta.ensure(sizeof(ObjMeta) * c->nobj, "object table");
    c->theta.ensure(sizeof(float) * 8 * (size_t)T, "poses");
    c->fsums.ensure(sizeof(double) * T * kFwdSums, "fsums");
    c->csums.ensure(sizeof(double) * std::max<long long>(1, csum_total) * kColSums, "csums");
    c->colitems.ensure(sizeof(int) * 2, "collision work counters");
    c->collist.ensure(sizeof(int) * 2 * std::max<long long>(1, csum_total), "collision work list");
    c->nnidx.ensure(sizeof(int) * (size_t)T * N, "nn_idx");
    c->tccand.ensure(sizeof(int4) * (size_t)T * N, "tensor-core candidate chunks");
    c->ncol.ensure(sizeof(int) * T, "ncol");
    c->colidx.ensure(sizeof(int) * std::max<long long>(1, colidx_total), "colidx");
    c->cost.ensure(sizeof(double) * T, "cost");
    c->grad.ensure(sizeof(double) * T * 8, "grad");
    c->prev.ensure(sizeof(double) * T, "prev_cost");
    c->frozen.ensure(sizeof(int) * T, "frozen");
    c->phi.ensure(sizeof(float) * T * 8, "phi");
    c->h.ensure(sizeof(float) * G, "h");
    c->order.ensure(sizeof(int) * T, "order");
    c->out7.ensure(sizeof(float) * T * 8, "out7");
    c->outc.ensure(sizeof(float) * T, "outc");
    c->outi.ensure(sizeof(int) * T, "outi");
    if (c->cfg.debug) {
        c->dbg_d2.ensure(sizeof(float) * (size_t)T * N, "dbg_d2");
        c->dbg_sp.ensure(sizeof(float) * (size_t)T * N * 3, "dbg_sp");
        c->dbg_colnn.ensure(sizeof(int) * std::max<long long>(1, colidx_total), "dbg_colnn");
    }
    // device tables (pageable sources: the copies complete before returning)
    ck(cudaMemcpyAsync(c->partgrp.p, part_grp.data(), sizeof(int) * T, cudaMemcpyHostToDevice, c->st), "particle groups");
    ck(cudaMemcpyAsync(c->grpoff.p, off.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, c->st), "group offsets");
    ck(cudaMemcpyAsync(c->objmeta.p, om.data(), sizeof(ObjMeta) * c->nobj, cudaMemcpyHostToDevice, c->st),
       "object table");
    ck(cudaStreamSynchronize(c->st), "layout");
    c->layout_dirty = false;
    plan_fwd_items(c, c->fwd_variant);
}

__global__ void reset_convergence_kernel(double *prev, int *frozen, float *phi, int T, int *col_items)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) { col_items[0] = 0; col_items[1] = 0; }
    if (i >= T) return;
    prev[i] = -1.0;     // no previous cost
    frozen[i] = 0;
    for (int a = 0; a < 8; ++a) phi[(size_t)i * 8 + a] = 0.f;
}

// Stream the iteration kernels go to: the capture stream while a graph is being
// recorded, else the caller's stream.
cudaStream_t work_stream(const asicp_ctx *c) { return c->capturing ? c->cap_st : c->st; }

void reset_convergence(asicp_ctx *c)
{
    reset_convergence_kernel<<<(c->T + 255) / 256, 256, 0, work_stream(c)>>>(
        c->prev.as<double>(), c->frozen.as<int>(), c->phi.as<float>(), c->T, c->colitems.as<int>());
    ck(cudaGetLastError(), "reset convergence state");
}

template <class L>
void timed(asicp_ctx *c, int kind, L &&launch, const char *what)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st = work_stream(c);
    // inside a capture, an external record makes the event a graph node that every
    // replay records (a plain record would only express a capture dependency)
    const unsigned flags = c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    // profile 1: every kernel; 2: the forward-matching (screening) kernel only.  Each event
    // record is a node of the captured loop and costs a few microseconds of the replay.
    const bool on = c->cfg.profile == 1 || (c->cfg.profile == 2 && kind == kTimeMatch);
    if (on) {
        a = c->take_event();
        b = c->take_event();
        ck(cudaEventRecordWithFlags(a, st, flags), "cudaEventRecord");
    }
    ck(launch(st), what);
    if (on) {
        ck(cudaEventRecordWithFlags(b, st, flags), "cudaEventRecord");
        (c->capturing ? c->graph_events : c->events).push_back({kind, a, b});
    }
}

// Add the device times of the last graph replay (its events are re-recorded by
// every replay, so they are read before the next one).
void accumulate_graph_events(asicp_ctx *c)
{
    if (!c->graph_pending) return;
    for (auto &e : c->graph_events) {
        float t = 0.f;
        ck(cudaEventSynchronize(e.b), "cudaEventSynchronize");
        ck(cudaEventElapsedTime(&t, e.a, e.b), "cudaEventElapsedTime");
        c->acc_ms[e.kind] += t;
        c->acc_n[e.kind] += 1;
    }
    c->graph_pending = false;
}

// One pass of cost/gradient evaluation (+ update for mode 1/2).
// Object 0's table points at the mini-batch of iteration k (k < the number of
// mini-batches) or back at the whole cloud (otherwise), on the work stream.
void select_minibatch(asicp_ctx *c, int k)
{
    if (c->mb_off.empty()) return;
    cudaStream_t st = work_stream(c);
    ObjMeta m = c->objmeta_h[0];
    if (k >= 0 && k + 1 < (int)c->mb_off.size()) {
        const int first = c->mb_off[k], cnt = c->mb_off[k + 1] - first;
        const int Mpad = (cnt + kRefTilePts - 1) / kRefTilePts * kRefTilePts;
        ck(launch_gather_points(c->objs[0].R.as<float4>(), c->mb_idx.as<int>() + first, cnt, c->mb_R.as<float4>(), st),
           "mini-batch gather");
        // the mini-batch keeps the whole object's frame (its points are a subset)
        ck(launch_ref_prep(c->mb_R.as<float4>(), cnt, Mpad, c->mb_Rx.p, c->frame.as<float4>(), false, st),
           "mini-batch prep");
        m.R = c->mb_R.as<float4>();
        m.Rx = c->mb_Rx.as<ulonglong2>();
        m.M = cnt;
        m.Mpad = Mpad;
    }
    ck(launch_store_meta(c->objmeta.as<ObjMeta>(), m, st), "object table");
}

void iterate(asicp_ctx *c, int mode, float gamma, int k)
{
    select_minibatch(c, k);
    const Layout L = c->layout();
    FwdArgs fa{};
    fa.L = L;
    fa.S = c->S.as<float4>();
    fa.theta = c->theta.as<float>();
    fa.items = c->items.as<FwdItem>();
    fa.cta_off = c->ctaoff.as<int>();
    fa.n_items = c->n_items;
    fa.err = c->errw.as<int>();
    fa.nn_idx = c->nnidx.as<int>();
    fa.cand = c->tccand.as<int4>();
    fa.variant = c->fwd_variant;
    fa.expire_test = c->expire_test ? 1 : 0;
    if (c->cfg.debug) {
        fa.dbg_d2 = c->dbg_d2.as<float>();
        fa.dbg_sp = c->dbg_sp.as<float>();
    }
    timed(c, kTimeMatch, [&](cudaStream_t st) { return launch_fwd_match(fa, st); }, "forward matching kernel");
    if (fwd_has_exact_kernel(fa.variant))
        timed(c, kTimeExact, [&](cudaStream_t st) { return launch_fwd_exact(fa, st); }, "exact choice kernel");

    CollideArgs ca{};
    ca.L = L;
    ca.theta = c->theta.as<float>();
    ca.meta = c->dmeta.as<SdfMeta>();
    ca.S = c->S.as<float4>();
    ca.nn_idx = c->nnidx.as<int>();
    ca.ncol = c->ncol.as<int>();
    ca.colidx = c->colidx.as<int>();
    ca.fsums = c->fsums.as<double>();
    ca.csums = c->csums.as<double>();
    ca.col_items = c->colitems.as<int>();
    ca.col_list = c->collist.as<int>();
    ca.err = c->errw.as<int>();
    if (c->cfg.debug) ca.dbg_colnn = c->dbg_colnn.as<int>();
    timed(c, kTimeCollide, [&](cudaStream_t st) { return launch_collide(ca, st); }, "collision kernel");
    timed(c, kTimeCollideNN, [&](cudaStream_t st) { return launch_collide_nn(ca, st); }, "collision matching kernel");

    UpdateArgs ua{};
    ua.L = L;
    ua.theta = c->theta.as<float>();
    ua.fsums = c->fsums.as<double>();
    ua.csums = c->csums.as<double>();
    ua.ncol = c->ncol.as<int>();
    ua.pconst = c->pconst.as<double>();
    ua.w_com = c->cfg.w_com;
    ua.mode = mode;
    ua.gamma = gamma;
    ua.eta_svgd = c->cfg.eta_svgd > 0.f ? c->cfg.eta_svgd : 1.f / (float)c->N;
    ua.eta_sgd = c->cfg.eta_sgd;
    ua.bandwidth_mode = c->cfg.bandwidth_mode;
    ua.h_fixed = c->cfg.h_fixed;
    ua.conv_tol = c->cfg.conv_tol;
    ua.cost = c->cost.as<double>();
    ua.grad = c->grad.as<double>();
    ua.prev_cost = c->prev.as<double>();
    ua.frozen = c->frozen.as<int>();
    ua.phi = c->phi.as<float>();
    ua.h = c->h.as<float>();
    ua.col_items = c->colitems.as<int>();
    ua.err = c->errw.as<int>();
    ua.prior_t_sigma = c->cfg.prior_t_sigma;
    ua.prior_q_kappa = c->cfg.prior_q_kappa;
    {
        const float *m = c->cfg.prior_q_mean;
        const double n =
            std::sqrt((double)m[0] * m[0] + (double)m[1] * m[1] + (double)m[2] * m[2] + (double)m[3] * m[3]);
        for (int a = 0; a < 4; ++a) ua.prior_q_mean[a] = n > 0.0 ? (float)(m[a] / n) : (a == 0 ? 1.f : 0.f);
    }
    timed(c, kTimeFinalize, [&](cudaStream_t st) { return launch_finalize(ua, st); }, "finalize kernel");
    if (mode == 1)
        timed(c, kTimeStein, [&](cudaStream_t st) { return launch_stein(ua, st); }, "Stein kernel");
}

void step_impl(asicp_ctx *c, int k)
{
    const int mode = k < c->cfg.k_stein ? 1 : 2;
    iterate(c, mode, (float)gamma_of(c->cfg, k), k);
    c->k_next = k + 1;
    c->stepped = true;
}

// Everything asicp_run does after the initial poses: convergence reset, k_max
// iterations, final evaluation and ranking.
void run_loop(asicp_ctx *c)
{
    reset_convergence(c);
    for (int k = 0; k < c->cfg.k_max; ++k) step_impl(c, k);
    iterate(c, 0, 0.f, -1);   // final evaluation at the last poses (whole object cloud)
    ck(launch_select(c->layout(), c->cost.as<double>(), c->ncol.as<int>(), c->order.as<int>(), work_stream(c)),
       "select");
}

// Buffers and sizes the captured graph depends on (the tables they hold are
// read at replay, so new objects of the same sizes reuse the graph).
std::vector<const void *> loop_key(const asicp_ctx *c)
{
    return {c->partgrp.p, c->grpoff.p, c->objmeta.p, c->items.p, c->ctaoff.p, c->com.p, c->frame.p, c->colitems.p, c->collist.p,
            c->S.p, c->pconst.p, c->dmeta.p, c->theta.p, c->fsums.p, c->csums.p, c->ncol.p, c->colidx.p, c->cost.p,
            c->grad.p, c->prev.p, c->frozen.p, c->phi.p, c->h.p, c->order.p, c->errw.p, c->nnidx.p, c->tccand.p, c->dbg_d2.p,
            c->dbg_sp.p, c->dbg_colnn.p, c->mb_idx.p, c->mb_R.p, c->mb_Rx.p,
            reinterpret_cast<const void *>((size_t)c->mb_version), reinterpret_cast<const void *>((size_t)c->T),
            reinterpret_cast<const void *>((size_t)c->G), reinterpret_cast<const void *>((size_t)c->n_items),
            reinterpret_cast<const void *>((size_t)c->N), reinterpret_cast<const void *>((size_t)c->fwd_variant),
            reinterpret_cast<const void *>((size_t)c->expire_test)};
}

// Replay the captured loop on the caller's stream, capturing it first when the
// buffers changed.  Kernel arguments (buffer pointers, per-iteration gamma) are
// fixed at capture; the buffers' contents are read at replay.
void run_loop_graph(asicp_ctx *c)
{
    std::vector<const void *> key = loop_key(c);
    if (!c->loop_exec || key != c->loop_key) {
        if (c->loop_exec) {
            cudaGraphExecDestroy(c->loop_exec);
            c->loop_exec = nullptr;
        }
        for (auto &e : c->graph_events) { c->pool.push_back(e.a); c->pool.push_back(e.b); }
        c->graph_events.clear();
        c->graph_pending = false;
        if (!c->cap_st) ck(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking), "capture stream");
        ck(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal), "begin capture");
        c->capturing = true;
        cudaGraph_t g = nullptr;
        try {
            run_loop(c);
        } catch (...) {
            c->capturing = false;
            cudaStreamEndCapture(c->cap_st, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        c->capturing = false;
        ck(cudaStreamEndCapture(c->cap_st, &g), "end capture");
        cudaError_t e = cudaGraphInstantiate(&c->loop_exec, g, 0);
        cudaGraphDestroy(g);
        ck(e, "instantiate graph");
        c->loop_key = key;
    }
    accumulate_graph_events(c);
    ck(cudaGraphLaunch(c->loop_exec, c->st), "graph launch");
    c->graph_pending = c->cfg.profile != 0;
}

void copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st, const char *what)
{
    if (!dst || bytes == 0) return;
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st), what);
}

__global__ void repack_kernel(const float *src8, int n, float *dst7)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 7; ++a) dst7[(size_t)i * 7 + a] = src8[(size_t)i * 8 + a];
}

__global__ void repack_f64_kernel(const double *src8, int n, double *dst7)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 7; ++a) dst7[(size_t)i * 7 + a] = src8[(size_t)i * 8 + a];
}

__global__ void gather_best_kernel(const int *order, int first, int n, const int *part_grp, int P, const float *theta8,
                                   const double *cost, float *o7, float *oc, int *oi)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int i = order[first + r];
    for (int a = 0; a < 7; ++a) o7[(size_t)r * 7 + a] = theta8[(size_t)i * 8 + a];
    oc[r] = (float)cost[i];
    oi[r] = part_grp[i] % P;
}

// Time every forward-matching kernel shape on the context's current work (poses
// as they are) and keep the fastest.  ms[v] receives the mean launch time.
void autotune_impl(asicp_ctx *c, float *ms_out)
{
    const int reps = 3;
    cudaEvent_t e0 = c->take_event(), e1 = c->take_event();
    float best = 0.f;
    int best_v = 0;
    for (int v = 0; v < kFwdVariants; ++v) {
        if (v == 7 && !c->mb_off.empty()) {   // the tensor-core kernel has no mini-batch tiles
            if (ms_out) ms_out[v] = 0.f;
            continue;
        }
        plan_fwd_items(c, v);
        FwdArgs fa{};
        fa.L = c->layout();
        fa.S = c->S.as<float4>();
        fa.theta = c->theta.as<float>();
        fa.items = c->items.as<FwdItem>();
        fa.cta_off = c->ctaoff.as<int>();
        fa.n_items = c->n_items;
        fa.err = c->errw.as<int>();
        fa.nn_idx = c->nnidx.as<int>();
        fa.cand = c->tccand.as<int4>();
        fa.variant = v;
        ck(launch_fwd_match(fa, c->st), "autotune warm-up");
        if (fwd_has_exact_kernel(v)) ck(launch_fwd_exact(fa, c->st), "autotune warm-up");
        ck(cudaEventRecord(e0, c->st), "cudaEventRecord");
        for (int r = 0; r < reps; ++r) {
            ck(launch_fwd_match(fa, c->st), "autotune launch");
            if (fwd_has_exact_kernel(v)) ck(launch_fwd_exact(fa, c->st), "autotune launch");
        }
        ck(cudaEventRecord(e1, c->st), "cudaEventRecord");
        ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float t = 0.f;
        ck(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime");
        t /= reps;
        if (ms_out) ms_out[v] = t;
        if (v == 0 || t < best) { best = t; best_v = v; }
    }
    c->pool.push_back(e0);
    c->pool.push_back(e1);
    sync_and_check_err(c, "autotune");
    c->fwd_variant = best_v;
    plan_fwd_items(c, best_v);
    c->tuned = true;
}

void set_object_impl(asicp_ctx *ctx, int o, const float *R_xyz, int M, const float *C_xyz, int Mc)
{
    if (o < 0 || o >= ctx->nobj) fail(ASICP_ERR_INVALID_ARG, "set_object: object index out of range");
    if (!R_xyz || M < 1) fail(ASICP_ERR_INVALID_ARG, "set_object: R must be non-NULL with M >= 1");
    if (C_xyz && Mc < 1) fail(ASICP_ERR_INVALID_ARG, "set_object: Mc must be >= 1 when C is given");
    ObjBufs &b = ctx->objs[o];
    const int mc = C_xyz ? Mc : M;
    if (!ctx->mb_off.empty()) {   // mini-batches index the previous cloud
        ctx->mb_off.clear();
        ++ctx->mb_version;
    }
    // what the layout (object table, work plan) and the captured loop depend on
    const bool was_set = b.set;
    const void *was[4] = {b.R.p, b.Rx.p, b.Rt.p, b.C.p};
    const int was_M = b.M, was_Mc = b.Mc, was_Mpad = b.Mpad;
    b.set = false;
    ctx->run_done = false;
    ctx->stage.ensure(sizeof(float) * 3 * (size_t)(M > mc ? M : mc), "staging");
    b.R.ensure(sizeof(float4) * M, "object cloud");
    ck(cudaMemcpyAsync(ctx->stage.p, R_xyz, sizeof(float) * 3 * (size_t)M, cudaMemcpyDefault, ctx->st), "copy R");
    ck(launch_pack_points(ctx->stage.as<float>(), M, b.R.as<float4>(), ctx->errw.as<int>(), ctx->st), "pack R");
    if (C_xyz) {
        b.C.ensure(sizeof(float4) * mc, "collision cloud");
        ck(cudaMemcpyAsync(ctx->stage.p, C_xyz, sizeof(float) * 3 * (size_t)mc, cudaMemcpyDefault, ctx->st), "copy C");
        ck(launch_pack_points(ctx->stage.as<float>(), mc, b.C.as<float4>(), ctx->errw.as<int>(), ctx->st), "pack C");
    } else {
        b.C.release();
    }
    ck(launch_centroid(b.R.as<float4>(), M, ctx->com.as<double>() + 3 * o, ctx->st), "centroid");
    const int Mpad = (M + kRefTilePts - 1) / kRefTilePts * kRefTilePts;
    b.Rx.ensure(sizeof(float4) * (size_t)Mpad, "screening layout");
    ck(launch_ref_prep(b.R.as<float4>(), M, Mpad, b.Rx.p, ctx->frame.as<float4>() + o, true, ctx->st), "ref prep");
    b.Rt.ensure(tc_ref_bytes(Mpad), "tensor-core object tiles");
    ck(launch_tc_ref_prep(b.R.as<float4>(), M, Mpad, ctx->frame.as<float4>() + o, b.Rt.p, ctx->st),
       "tensor-core ref prep");
    sync_and_check_err(ctx, "set_object");
    b.M = M;
    b.Mpad = Mpad;
    b.Mc = mc;
    b.set = true;
    // a new object of the same sizes in the same buffers keeps the layout, the poses
    // and the captured loop (whose kernels read the object's data at replay)
    if (!was_set || M != was_M || mc != was_Mc || Mpad != was_Mpad || b.R.p != was[0] || b.Rx.p != was[1] ||
        b.Rt.p != was[2] || b.C.p != was[3])
        ctx->layout_dirty = true;
}

}  // namespace

// ---------------------------------------------------------------------- ABI
extern "C" {

void asicp_config_default(asicp_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->P = 1;
    cfg->K = 32;
    cfg->k_max = 40;
    cfg->k_stein = 15;          // Table I: 15 SVGD + 25 SGD iterations
    cfg->schedule = 0;
    cfg->C_cycles = 5.f;        // Table I annealing factor (mod(k, k_max/5) / (k_max/5))^2
    cfg->p_exp = 2.f;
    cfg->g0 = 0.1f;
    cfg->g1 = 1.f;
    cfg->eta_sgd = 1.f;         // Table I learning rate
    cfg->eta_svgd = 0.f;        // 1/N
    cfg->w_com = 1.f;           // Table I cost weights
    cfg->bandwidth_mode = 0;
    cfg->h_fixed = 1.f;
    cfg->conv_tol = 2e-4f;      // Table I convergence criterion 0.02 %
    cfg->init_radius = 0.15f;
    cfg->debug = 0;
    cfg->profile = 0;
    cfg->cuda_stream = nullptr;
    cfg->n_objects = 1;
    cfg->autotune = 0;
    cfg->fwd_shape = 0;
}

asicp_status asicp_create(const asicp_config *cfg, asicp_ctx **out)
{
    if (!cfg || !out) return ASICP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->P < 1 || cfg->P > 64 || cfg->K < 1 || cfg->K > kMaxK || cfg->k_max < 0 || cfg->k_stein < 0 ||
        cfg->k_stein > cfg->k_max || (cfg->schedule != 0 && cfg->schedule != 1) ||
        (cfg->schedule == 0 && !(cfg->C_cycles > 0.f)) || !(cfg->eta_sgd >= 0.f) ||
        (cfg->bandwidth_mode == 1 && !(cfg->h_fixed > 0.f)) || !std::isfinite(cfg->w_com) ||
        !(cfg->init_radius >= 0.f) || cfg->n_objects < 1 || cfg->n_objects > 4096 ||
        cfg->fwd_shape < 0 || cfg->fwd_shape >= kFwdVariants || cfg->init_mode < 0 || cfg->init_mode > 1 ||
        !std::isfinite(cfg->prior_t_sigma) || !std::isfinite(cfg->prior_q_kappa) ||
        (cfg->prior_q_kappa > 0.f && !(std::fabs(cfg->prior_q_mean[0]) + std::fabs(cfg->prior_q_mean[1]) +
                                       std::fabs(cfg->prior_q_mean[2]) + std::fabs(cfg->prior_q_mean[3]) > 0.f)))
        return ASICP_ERR_INVALID_ARG;
    asicp_ctx *c = new (std::nothrow) asicp_ctx();
    if (!c) return ASICP_ERR_OOM;
    c->cfg = *cfg;
    c->st = static_cast<cudaStream_t>(cfg->cuda_stream);
    c->nobj = cfg->n_objects;
    c->fwd_variant = cfg->fwd_shape;
    c->pre_set.assign(cfg->P, 0);
    c->meta.assign(cfg->P, SdfMeta{});
    c->grids.resize(cfg->P);
    c->cells.resize(cfg->P);
    c->objs.resize(c->nobj);
    c->Kg.assign((size_t)c->nobj * cfg->P, cfg->K);
    asicp_status s = guarded(c, [&] {
        // one-time kernel attributes, set outside any graph capture
        fwd_grid_size();
        ck(init_collision_attributes(), "collision kernel attributes");
        ck(init_update_attributes(), "update kernel attributes");
        c->com.ensure(sizeof(double) * 3 * c->nobj, "com");
        c->frame.ensure(sizeof(float4) * c->nobj, "screening frames");
        c->pconst.ensure(sizeof(double) * 12 * cfg->P, "pconst");
        c->dmeta.ensure(sizeof(SdfMeta) * cfg->P, "sdf meta");
        c->errw.ensure(sizeof(int), "error word");
        ck(cudaMemsetAsync(c->errw.p, 0, sizeof(int), c->st), "clear error word");
        ck(cudaStreamSynchronize(c->st), "create");
    });
    if (s != ASICP_OK) {
        delete c;
        return s;
    }
    *out = c;
    return ASICP_OK;
}

asicp_status asicp_destroy(asicp_ctx *ctx)
{
    if (!ctx) return ASICP_OK;
    cudaStreamSynchronize(ctx->st);
    delete ctx;
    return ASICP_OK;
}

asicp_status asicp_set_object(asicp_ctx *ctx, const float *R_xyz, int M, const float *C_xyz, int Mc)
{
    return guarded(ctx, [&] { set_object_impl(ctx, 0, R_xyz, M, C_xyz, Mc); });
}

asicp_status asicp_set_object_at(asicp_ctx *ctx, int object, const float *R_xyz, int M, const float *C_xyz, int Mc)
{
    return guarded(ctx, [&] { set_object_impl(ctx, object, R_xyz, M, C_xyz, Mc); });
}

asicp_status asicp_set_particle_counts(asicp_ctx *ctx, const int *K, int n)
{
    return guarded(ctx, [&] {
        if (!K || n != ctx->nobj * ctx->cfg.P)
            fail(ASICP_ERR_INVALID_ARG, "set_particle_counts: need n_objects * P counts");
        std::vector<int> k(n);
        ck(cudaMemcpy(k.data(), K, sizeof(int) * n, cudaMemcpyDefault), "copy particle counts");
        for (int v : k)
            if (v < 1 || v > kMaxK) fail(ASICP_ERR_INVALID_ARG, "set_particle_counts: every count must be in [1, 1024]");
        ctx->Kg = k;
        ctx->layout_dirty = true;
        ctx->theta_set = false;
        ctx->run_done = false;
    });
}

asicp_status asicp_set_minibatch(asicp_ctx *ctx, const int *offsets, const int *indices, int iters)
{
    return guarded(ctx, [&] {
        ++ctx->mb_version;
        if (!offsets) {
            ctx->mb_off.clear();
            return;
        }
        if (ctx->nobj != 1) fail(ASICP_ERR_INVALID_ARG, "set_minibatch: one object per context");
        if (!ctx->objs[0].set) fail(ASICP_ERR_STATE, "set_minibatch: set the object first");
        if (!indices || iters < 1) fail(ASICP_ERR_INVALID_ARG, "set_minibatch: NULL indices or iters < 1");
        if (ctx->fwd_variant == 7) fail(ASICP_ERR_INVALID_ARG, "set_minibatch: not with the tensor-core kernel shape");
        const int M = ctx->objs[0].M;
        std::vector<int> off(iters + 1);
        ck(cudaMemcpy(off.data(), offsets, sizeof(int) * (iters + 1), cudaMemcpyDefault), "copy mini-batch offsets");
        if (off[0] != 0) fail(ASICP_ERR_INVALID_ARG, "set_minibatch: offsets must start at 0");
        for (int k = 0; k < iters; ++k)
            if (off[k + 1] - off[k] < 1 || off[k + 1] - off[k] > M)
                fail(ASICP_ERR_INVALID_ARG, "set_minibatch: every mini-batch needs 1..M points");
        std::vector<int> idx(off[iters]);
        ck(cudaMemcpy(idx.data(), indices, sizeof(int) * idx.size(), cudaMemcpyDefault), "copy mini-batch indices");
        for (int k = 0; k < iters; ++k)
            for (int i = off[k]; i < off[k + 1]; ++i)
                if (idx[i] < 0 || idx[i] >= M || (i > off[k] && idx[i] <= idx[i - 1]))
                    fail(ASICP_ERR_INVALID_ARG, "set_minibatch: indices must be ascending within [0, M)");
        const int Mpad = (M + kRefTilePts - 1) / kRefTilePts * kRefTilePts;
        ctx->mb_idx.ensure(sizeof(int) * idx.size(), "mini-batch indices");
        ctx->mb_R.ensure(sizeof(float4) * M, "mini-batch points");
        ctx->mb_Rx.ensure(sizeof(float4) * Mpad, "mini-batch screening layout");
        ck(cudaMemcpy(ctx->mb_idx.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice), "upload indices");
        ctx->mb_off = off;
        ctx->run_done = false;
    });
}

asicp_status asicp_set_gripper_sdf(asicp_ctx *ctx, int preshape, const float *S_xyz, int N, const float *sdf,
                                   int nx, int ny, int nz, const float origin[3], float voxel)
{
    return guarded(ctx, [&] {
        if (preshape < 0 || preshape >= ctx->cfg.P) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: preshape out of range");
        if (!S_xyz || !sdf || !origin) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: NULL array");
        if (N < 1 || N > kMaxN) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: N must be in [1, 6144]");
        if (nx < 2 || ny < 2 || nz < 2) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: every grid dimension must be >= 2");
        if (!(voxel > 0.f) || !std::isfinite(voxel)) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: voxel must be > 0");
        float org[3];
        ck(cudaMemcpy(org, origin, sizeof(org), cudaMemcpyDefault), "copy origin");
        for (float o : org)
            if (!std::isfinite(o)) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: non-finite origin");
        bool any_set = false;
        for (char s : ctx->pre_set) any_set = any_set || s;
        if (any_set && N != ctx->N) fail(ASICP_ERR_INVALID_ARG, "set_gripper_sdf: every preshape must have the same N");
        if (N != ctx->N) {
            ctx->N = N;
            ctx->layout_dirty = true;
        }
        ctx->pre_set[preshape] = 0;
        ctx->run_done = false;
        ctx->S.ensure(sizeof(float4) * (size_t)ctx->cfg.P * N, "gripper clouds");
        ctx->stage.ensure(sizeof(float) * 3 * (size_t)N, "staging");
        ck(cudaMemcpyAsync(ctx->stage.p, S_xyz, sizeof(float) * 3 * (size_t)N, cudaMemcpyDefault, ctx->st), "copy S");
        float4 *Sp = ctx->S.as<float4>() + (size_t)preshape * N;
        ck(launch_pack_points(ctx->stage.as<float>(), N, Sp, ctx->errw.as<int>(), ctx->st), "pack S");
        ck(launch_preshape_consts(Sp, N, ctx->pconst.as<double>() + 12 * preshape, ctx->st), "preshape sums");
        const size_t nv = (size_t)nx * ny * nz;
        ctx->grids[preshape].ensure(sizeof(float) * nv, "sdf grid");
        ck(cudaMemcpyAsync(ctx->grids[preshape].p, sdf, sizeof(float) * nv, cudaMemcpyDefault, ctx->st), "copy sdf");
        ck(launch_check_finite(ctx->grids[preshape].as<float>(), (long long)nv, ctx->errw.as<int>(), ctx->st), "check sdf");
        ctx->cells[preshape].ensure(sdf_cells_bytes(nx, ny, nz), "corner-packed sdf grid");
        ck(launch_sdf_pack_cells(ctx->grids[preshape].as<float>(), nx, ny, nz, ctx->cells[preshape].as<float4>(), ctx->st),
           "pack sdf cells");
        // index box of the positive nodes -> gripper-frame box holding every cell that
        // has a positive corner (trilinear values outside it cannot be > 0)
        ctx->box.ensure(sizeof(int) * 6, "sdf box");
        const int box_init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
        ck(cudaMemcpyAsync(ctx->box.p, box_init, sizeof(box_init), cudaMemcpyHostToDevice, ctx->st), "init sdf box");
        ck(launch_sdf_box(ctx->grids[preshape].as<float>(), nx, ny, nz, ctx->box.as<int>(), ctx->st), "sdf box");
        int box6[6];
        ck(cudaMemcpyAsync(box6, ctx->box.p, sizeof(box6), cudaMemcpyDeviceToHost, ctx->st), "read sdf box");
        sync_and_check_err(ctx, "set_gripper_sdf");
        SdfMeta m{};
        m.grid = ctx->grids[preshape].as<float>();
        m.cells = ctx->cells[preshape].as<float4>();
        m.nx = nx; m.ny = ny; m.nz = nz;
        m.ox = org[0]; m.oy = org[1]; m.oz = org[2];
        m.voxel = voxel;
        for (int a = 0; a < 3; ++a) {
            if (box6[a] == INT_MAX) {            // no positive node: nothing can collide
                m.lo[a] = 1.f;
                m.hi[a] = -1.f;
            } else {
                const double margin = 1e-3 * voxel;
                m.lo[a] = (float)(org[a] + (double)voxel * (box6[a] - 1) - margin);
                m.hi[a] = (float)(org[a] + (double)voxel * (box6[3 + a] + 1) + margin);
            }
        }
        ctx->meta[preshape] = m;
        ck(cudaMemcpyAsync(ctx->dmeta.as<SdfMeta>() + preshape, &ctx->meta[preshape], sizeof(SdfMeta),
                           cudaMemcpyHostToDevice, ctx->st), "copy sdf meta");
        ck(cudaStreamSynchronize(ctx->st), "set_gripper_sdf");
        ctx->pre_set[preshape] = 1;
    });
}

asicp_status asicp_set_state(asicp_ctx *ctx, const float *theta, int k)
{
    return guarded(ctx, [&] {
        if (!ctx->inputs_ready()) fail(ASICP_ERR_STATE, "set_state: objects and every preshape must be set first");
        if (!theta || k < 0 || k > ctx->cfg.k_max) fail(ASICP_ERR_INVALID_ARG, "set_state: bad theta or k");
        build_layout(ctx);
        const size_t T = ctx->T;
        ctx->stage.ensure(sizeof(float) * 7 * T, "staging");
        ck(cudaMemcpyAsync(ctx->stage.p, theta, sizeof(float) * 7 * T, cudaMemcpyDefault, ctx->st), "copy theta");
        ck(launch_set_theta(ctx->stage.as<float>(), (int)T, ctx->theta.as<float>(), ctx->errw.as<int>(), ctx->st),
           "set theta");
        reset_convergence(ctx);
        sync_and_check_err(ctx, "set_state");
        ctx->k_next = k;
        ctx->theta_set = true;
        ctx->stepped = false;
        ctx->run_done = false;
    });
}

asicp_status asicp_set_convergence(asicp_ctx *ctx, const double *prev_cost, const int *frozen)
{
    return guarded(ctx, [&] {
        if (!ctx->theta_set || ctx->layout_dirty) fail(ASICP_ERR_STATE, "set_convergence: set the poses first");
        const size_t T = ctx->T;
        if (prev_cost)
            ck(cudaMemcpyAsync(ctx->prev.p, prev_cost, sizeof(double) * T, cudaMemcpyDefault, ctx->st),
               "copy prev_cost");
        if (frozen)
            ck(cudaMemcpyAsync(ctx->frozen.p, frozen, sizeof(int) * T, cudaMemcpyDefault, ctx->st), "copy frozen");
        ck(cudaStreamSynchronize(ctx->st), "set_convergence");
    });
}

asicp_status asicp_step(asicp_ctx *ctx, int k)
{
    return guarded(ctx, [&] {
        if (!ctx->inputs_ready() || !ctx->theta_set) fail(ASICP_ERR_STATE, "step: inputs and poses must be set first");
        if (ctx->layout_dirty) fail(ASICP_ERR_STATE, "step: inputs changed since the poses were set");
        if (k < 0 || k >= ctx->cfg.k_max) fail(ASICP_ERR_INVALID_ARG, "step: k out of [0, k_max)");
        step_impl(ctx, k);
        ctx->run_done = false;
    });
}

asicp_status asicp_run(asicp_ctx *ctx, const float *theta0)
{
    return guarded(ctx, [&] {
        if (!ctx->inputs_ready()) fail(ASICP_ERR_STATE, "run: objects and every preshape must be set first");
        build_layout(ctx);
        const int T = ctx->T;
        if (theta0) {
            ctx->stage.ensure(sizeof(float) * 7 * T, "staging");
            ck(cudaMemcpyAsync(ctx->stage.p, theta0, sizeof(float) * 7 * (size_t)T, cudaMemcpyDefault, ctx->st),
               "copy theta0");
            ck(launch_set_theta(ctx->stage.as<float>(), T, ctx->theta.as<float>(), ctx->errw.as<int>(), ctx->st),
               "set theta0");
            sync_and_check_err(ctx, "run");
        } else {
            ck(launch_fibonacci(ctx->layout(), ctx->cfg.init_radius, ctx->cfg.init_mode, ctx->theta.as<float>(),
                                ctx->st),
               "initial poses");
        }
        ctx->theta_set = true;
        if (ctx->cfg.autotune && !ctx->tuned) autotune_impl(ctx, nullptr);
        run_loop_graph(ctx);
        ctx->k_next = ctx->cfg.k_max;
        ctx->stepped = true;
        ctx->run_done = true;
    });
}

asicp_status asicp_best_grasps_at(asicp_ctx *ctx, int object, int topk, float *theta, float *cost, int *preshape,
                                  int *n_out)
{
    return guarded(ctx, [&] {
        if (!ctx->run_done) fail(ASICP_ERR_STATE, "best_grasps: no completed run");
        if (topk < 0) fail(ASICP_ERR_INVALID_ARG, "best_grasps: topk < 0");
        if (object < 0 || object >= ctx->nobj) fail(ASICP_ERR_INVALID_ARG, "best_grasps: object index out of range");
        const ObjMeta &om = ctx->objmeta_h[object];
        const int n = topk < om.np ? topk : om.np;
        if (n > 0) {
            gather_best_kernel<<<(n + 127) / 128, 128, 0, ctx->st>>>(ctx->order.as<int>(), om.pfirst, n,
                                                                     ctx->partgrp.as<int>(), ctx->cfg.P,
                                                                     ctx->theta.as<float>(), ctx->cost.as<double>(),
                                                                     ctx->out7.as<float>(), ctx->outc.as<float>(),
                                                                     ctx->outi.as<int>());
            ck(cudaGetLastError(), "gather best");
            copy_out(theta, ctx->out7.p, sizeof(float) * 7 * n, ctx->st, "copy best theta");
            copy_out(cost, ctx->outc.p, sizeof(float) * n, ctx->st, "copy best cost");
            copy_out(preshape, ctx->outi.p, sizeof(int) * n, ctx->st, "copy best preshape");
        }
        sync_and_check_err(ctx, "best_grasps");
        if (n_out) *n_out = n;
    });
}

asicp_status asicp_best_grasps(asicp_ctx *ctx, int topk, float *theta, float *cost, int *preshape, int *n_out)
{
    return asicp_best_grasps_at(ctx, 0, topk, theta, cost, preshape, n_out);
}

asicp_status asicp_get_state(asicp_ctx *ctx, const asicp_state_view *v)
{
    return guarded(ctx, [&] {
        if (!v) fail(ASICP_ERR_INVALID_ARG, "get_state: NULL view");
        if (!ctx->theta_set) fail(ASICP_ERR_STATE, "get_state: no poses yet");
        const bool dbg = v->nn_idx || v->nn_d2 || v->s_prime || v->col_list || v->col_nn;
        if (dbg && !ctx->cfg.debug) fail(ASICP_ERR_STATE, "get_state: debug arrays need config.debug = 1");
        const int T = ctx->T;
        if (v->theta) {
            repack_kernel<<<(T + 127) / 128, 128, 0, ctx->st>>>(ctx->theta.as<float>(), T, ctx->out7.as<float>());
            ck(cudaGetLastError(), "repack theta");
            copy_out(v->theta, ctx->out7.p, sizeof(float) * 7 * T, ctx->st, "copy theta");
            ck(cudaStreamSynchronize(ctx->st), "get_state");
        }
        if (v->phi) {
            repack_kernel<<<(T + 127) / 128, 128, 0, ctx->st>>>(ctx->phi.as<float>(), T, ctx->out7.as<float>());
            ck(cudaGetLastError(), "repack phi");
            copy_out(v->phi, ctx->out7.p, sizeof(float) * 7 * T, ctx->st, "copy phi");
            ck(cudaStreamSynchronize(ctx->st), "get_state");
        }
        if (v->grad) {
            ctx->stage.ensure(sizeof(double) * 7 * T, "staging");
            repack_f64_kernel<<<(T + 127) / 128, 128, 0, ctx->st>>>(ctx->grad.as<double>(), T, ctx->stage.as<double>());
            ck(cudaGetLastError(), "repack grad");
            copy_out(v->grad, ctx->stage.p, sizeof(double) * 7 * T, ctx->st, "copy grad");
            ck(cudaStreamSynchronize(ctx->st), "get_state");
        }
        if (ctx->stepped || ctx->run_done) {
            copy_out(v->cost, ctx->cost.p, sizeof(double) * T, ctx->st, "copy cost");
            copy_out(v->ncol, ctx->ncol.p, sizeof(int) * T, ctx->st, "copy ncol");
            copy_out(v->h, ctx->h.p, sizeof(float) * ctx->G, ctx->st, "copy h");
            if (ctx->cfg.debug) {
                copy_out(v->nn_idx, ctx->nnidx.p, sizeof(int) * (size_t)T * ctx->N, ctx->st, "copy nn_idx");
                copy_out(v->nn_d2, ctx->dbg_d2.p, sizeof(float) * (size_t)T * ctx->N, ctx->st, "copy nn_d2");
                copy_out(v->s_prime, ctx->dbg_sp.p, sizeof(float) * 3 * (size_t)T * ctx->N, ctx->st, "copy s_prime");
                copy_out(v->col_list, ctx->colidx.p, sizeof(int) * (size_t)ctx->colidx_total, ctx->st, "copy col_list");
                copy_out(v->col_nn, ctx->dbg_colnn.p, sizeof(int) * (size_t)ctx->colidx_total, ctx->st, "copy col_nn");
            }
        } else if (v->cost || v->ncol || v->h || dbg) {
            fail(ASICP_ERR_STATE, "get_state: no step has run since the poses were set");
        }
        copy_out(v->frozen, ctx->frozen.p, sizeof(int) * T, ctx->st, "copy frozen");
        sync_and_check_err(ctx, "get_state");
    });
}

asicp_status asicp_autotune(asicp_ctx *ctx, int *chosen, float *ms)
{
    return guarded(ctx, [&] {
        if (!ctx->inputs_ready()) fail(ASICP_ERR_STATE, "autotune: objects and every preshape must be set first");
        build_layout(ctx);
        if (!ctx->theta_set) {
            ck(launch_fibonacci(ctx->layout(), ctx->cfg.init_radius, ctx->cfg.init_mode, ctx->theta.as<float>(),
                                ctx->st),
               "initial poses");
            ctx->theta_set = true;
            ctx->stepped = false;
        }
        autotune_impl(ctx, ms);
        if (chosen) *chosen = ctx->fwd_variant;
    });
}

asicp_status asicp_test_expire_waits(asicp_ctx *ctx, int on)
{
    return guarded(ctx, [&] { ctx->expire_test = on != 0; });
}

asicp_status asicp_kernel_times(asicp_ctx *ctx, double ms[ASICP_KERNEL_KINDS], long long launches[ASICP_KERNEL_KINDS],
                                int reset)
{
    return guarded(ctx, [&] {
        if (!ctx->cfg.profile) fail(ASICP_ERR_STATE, "kernel_times: config.profile is 0");
        ck(cudaStreamSynchronize(ctx->st), "kernel_times");
        accumulate_graph_events(ctx);
        for (auto &e : ctx->events) {
            float t = 0.f;
            ck(cudaEventElapsedTime(&t, e.a, e.b), "cudaEventElapsedTime");
            ctx->acc_ms[e.kind] += t;
            ctx->acc_n[e.kind] += 1;
            ctx->pool.push_back(e.a);
            ctx->pool.push_back(e.b);
        }
        ctx->events.clear();
        for (int i = 0; i < kTimeKinds; ++i) {
            if (ms) ms[i] = ctx->acc_ms[i];
            if (launches) launches[i] = ctx->acc_n[i];
        }
        if (reset)
            for (int i = 0; i < kTimeKinds; ++i) { ctx->acc_ms[i] = 0; ctx->acc_n[i] = 0; }
    });
}

const char *asicp_last_error(const asicp_ctx *ctx)
{
    if (!ctx) return "NULL context";
    return ctx->err.c_str();
}

}  // extern "C"
