// C ABI entry points (include/sph.h): context, argument checks, stage timing,
// error word, and the step driver.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "sph_internal.cuh"

using namespace sph;

namespace {

const char *status_text(sph_status s)
{
    switch (s) {
    case SPH_OK: return "ok";
    case SPH_ERR_INVALID_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA error";
    case SPH_ERR_NOMEM: return "out of memory or tree capacity exceeded";
    case SPH_ERR_NOT_CONVERGED: return "h-rho Newton iteration did not converge";
    case SPH_ERR_TILE_OVERFLOW: return "tree-walk stack or neighbour-list overflow";
    case SPH_ERR_NONFINITE: return "non-finite or non-positive input (pos, vel, m, h)";
    case SPH_ERR_NEGATIVE_U: return "negative internal energy";
    case SPH_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown";
}

sph_status fail(Ctx &c, sph_status s, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", status_text(s), what);
    c.last_error = buf;
    return s;
}

sph_status cuda_fail(Ctx &c, cudaError_t e, const char *what)
{
    char buf[320];
    snprintf(buf, sizeof(buf), "CUDA error in %s: %s", what, cudaGetErrorString(e));
    c.last_error = buf;
    return SPH_ERR_CUDA;
}

template <class T>
cudaError_t dalloc(T *&p, size_t count)
{
    return cudaMalloc((void **)&p, sizeof(T) * (count > 0 ? count : 1));
}

// an event pair from the pool (created when the pool is empty)
bool take_event_pair(Ctx &c, Ctx::EvPair &ev)
{
    if (c.ev_free.empty()) {
        Ctx::EvPair p{};
        if (cudaEventCreate(&p.a) != cudaSuccess) return false;
        if (cudaEventCreate(&p.b) != cudaSuccess) {
            cudaEventDestroy(p.a);
            return false;
        }
        c.ev_free.push_back(p);
    }
    ev = c.ev_free.back();
    c.ev_free.pop_back();
    return true;
}

struct StageScope {
    Ctx &c;
    int stage;
    cudaStream_t st;
    Ctx::EvPair ev{};
    bool on = false;
    StageScope(Ctx &c_, int stage_, cudaStream_t st_, int launches) : c(c_), stage(stage_), st(st_)
    {
        (c.capturing ? c.capture_launches : c.pending_launches)[stage] += launches;
        if (!c.timing) return;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        // a graph the caller records holds no timing events of ours
        if (!c.capturing && (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone))
            return;
        if (!take_event_pair(c, ev)) return;
        ev.stage = stage;
        on = record(ev.a);
        if (!on) c.ev_free.push_back(ev);
    }
    ~StageScope()
    {
        if (!on) return;
        record(ev.b);
        (c.capturing ? c.capture_ev : c.ev_pending).push_back(ev);
    }
    // while a step graph is recorded, as an event-record node of the graph
    bool record(cudaEvent_t e)
    {
        return (c.capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                            : cudaEventRecord(e, st)) == cudaSuccess;
    }
};

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

sph_status check_state(Ctx &c, const sph_state *s, bool need_outputs)
{
    if (!s) return fail(c, SPH_ERR_INVALID_ARG, "state is NULL");
    if (s->n < 0 || s->n > c.max_n) return fail(c, SPH_ERR_INVALID_ARG, "n out of range [0, max_n]");
    if (s->n == 0) return SPH_OK;
    if (!s->pos || !s->vel || !s->h || !s->perm || !s->keys)
        return fail(c, SPH_ERR_INVALID_ARG, "NULL state array");
    if (need_outputs && (!s->acc || !s->rho || !s->omega || !s->drhodt || !s->vsigmax))
        return fail(c, SPH_ERR_INVALID_ARG, "NULL output array");
    if (!aligned16(s->pos) || !aligned16(s->vel) || (s->acc && !aligned16(s->acc)))
        return fail(c, SPH_ERR_INVALID_ARG, "pos/vel/acc must be 16-byte aligned");
    return SPH_OK;
}

sph_status check_params(Ctx &c, const sph_params *p)
{
    if (!p) return fail(c, SPH_ERR_INVALID_ARG, "params is NULL");
    if (!(p->gamma > 1.f) || !(p->hfact > 0.f) || !(p->h_tol > 0.f) || !(p->c_cour > 0.f) ||
        !(p->alpha_av >= 0.f) || !(p->beta_av >= 0.f) || !(p->alpha_u >= 0.f))
        return fail(c, SPH_ERR_INVALID_ARG, "parameter out of range");
    if (p->kernel < 0 || p->kernel > 2)
        return fail(c, SPH_ERR_INVALID_ARG, "kernel must be 0 (M4), 1 (M6) or 2 (Wendland C6)");
    if (p->n_leaf < 1 || p->n_leaf > 64 || p->n_group < 1 || p->n_group > 32)
        return fail(c, SPH_ERR_INVALID_ARG, "n_leaf must be 1..64 and n_group 1..32");
    if (p->tile < 0 || p->tile > 128 || p->max_h_iter < 1 || p->density_iters < 0)
        return fail(c, SPH_ERR_INVALID_ARG, "tile 0..128, max_h_iter >= 1, density_iters >= 0");
    const int t = p->pair_targets, w = p->pair_warps, u = p->pair_unroll;
    if (!(t == 0 || t == 4 || t == 8 || t == 16) || !(w == 0 || w == 1 || w == 2 || w == 4 || w == 8) ||
        !(u == 0 || u == 2 || u == 4))
        return fail(c, SPH_ERR_INVALID_ARG, "pair_targets 0/4/8/16, pair_warps 0/1/2/4/8, pair_unroll 0/2/4");
    for (int a = 0; a < 3; ++a)
        if (!(p->box_len[a] >= 0.f) || !std::isfinite(p->box_len[a]) || !std::isfinite(p->box_lo[a]))
            return fail(c, SPH_ERR_INVALID_ARG, "box_len must be finite and >= 0, box_lo finite");
    if (!(p->grav_G >= 0.f) || !std::isfinite(p->grav_G))
        return fail(c, SPH_ERR_INVALID_ARG, "grav_G must be finite and >= 0");
    if (p->grav_G > 0.f) {
        if (!(p->grav_eps > 0.f) || !std::isfinite(p->grav_eps) || !(p->grav_theta > 0.f) ||
            !(p->grav_theta <= 0.57f))
            return fail(c, SPH_ERR_INVALID_ARG, "gravity needs grav_eps > 0 and 0 < grav_theta <= 0.57");
        if (p->box_len[0] > 0.f || p->box_len[1] > 0.f || p->box_len[2] > 0.f)
            return fail(c, SPH_ERR_INVALID_ARG, "gravity with periodic boundaries is not built");
    }
    return SPH_OK;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

constexpr int kTreeLaunches = 33;
constexpr int kPrepLaunches = 1;

// tree_fresh: the tree was just built from this state (node and group h_max
// hold the current h); inside a step (c.drhodt_in_force) the density pass
// reads positions only, so the packed records need not be current
sph_status do_density(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                      bool tree_fresh)
{
    if (!tree_fresh) {
        // node and group h_max of the starting h, for the list walk
        StageScope sc(c, ST_PREP, st, 3);
        CK(update_hmax(c, s, p, st), "update_hmax");
        CK(pack_records(c, s, st), "pack");
    }
    {
        StageScope sc(c, ST_LISTS, st, 1);
        CK(density_lists(c, s, p, st, nullptr, false), "neighbour lists");
    }
    StageScope sc(c, ST_DENSITY, st, 2);
    CK(density_solve(c, s, p, st), "density");
    return SPH_OK;
}

// records_fresh: the packed particle records hold the current pos, vel (the
// density pass of the same step ran on this state)
sph_status do_force(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                    bool records_fresh)
{
    {
        StageScope sc(c, ST_PREP, st, kPrepLaunches + (records_fresh ? 0 : 1));
        CK(force_prep(c, s, p, st), "force_prep");
        if (!records_fresh) CK(pack_records(c, s, st), "pack");
    }
    {
        // relist (h_max refresh 2, list kernel 1), list kernel, h_max refresh 2, walking fallback
        StageScope sc(c, ST_FORCE, st, 7);
        CK(force_pass(c, s, p, st), "force");
    }
    if (p.grav_G > 0.f) {
        StageScope sc(c, ST_GRAVITY, st, 2);  // moments, walk
        CK(gravity_pass(c, s, p, (float4 *)s.acc, nullptr, st), "gravity");
    }
    return SPH_OK;
}

sph_status do_tree(Ctx &c, const sph_state &s, const sph_params &p, bool full, cudaStream_t st)
{
    StageScope sc(c, ST_TREE, st, kTreeLaunches);
    CK(build_tree(c, s, p, full, st), "build_tree");
    return SPH_OK;
}

// Host buffers that receive a step's outputs (sph_step_host's last step):
// each output is copied on the context's copy stream as soon as it is final,
// while the rest of the step runs.
struct HostOut {
    const sph_state *hs;
    float *h_dt;
};

// queue the device-to-host copies of `fields` (bit k: field k of
// sph_state after n, in declaration order) behind what st has queued so far
cudaError_t copy_out(Ctx &c, const sph_state &d, const HostOut &o, unsigned fields, cudaStream_t st,
                     int ev)
{
    const size_t n = (size_t)d.n;
    void *const dst[10] = {o.hs->pos, o.hs->vel, o.hs->acc, o.hs->h, o.hs->rho,
                           o.hs->omega, o.hs->drhodt, o.hs->vsigmax, o.hs->perm, o.hs->keys};
    const void *const src[10] = {d.pos, d.vel, d.acc, d.h, d.rho, d.omega, d.drhodt, d.vsigmax, d.perm, d.keys};
    const size_t size[10] = {16, 16, 16, 4, 4, 4, 4, 4, 4, 8};
    cudaError_t e = cudaEventRecord(c.copy_ev[ev], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.copy_stream, c.copy_ev[ev], 0);
    for (int k = 0; k < 10 && e == cudaSuccess; ++k)
        if (fields & (1u << k))
            e = cudaMemcpyAsync(dst[k], src[k], n * size[k], cudaMemcpyDeviceToHost, c.copy_stream);
    return e;
}

// one leapfrog step (kick-drift, tree, density, force, closing kick, Courant dt)
sph_status enqueue_step(Ctx &c, const sph_state &s, const sph_params &p, float *d_dt,
                        double *d_time, cudaStream_t st, const HostOut *out = nullptr)
{
    sph_status r;
    {
        StageScope sc(c, ST_LEAPFROG, st, 1);
        CK(kick_drift(c, s, p, d_dt, st), "kick_drift");
    }
    if ((r = do_tree(c, s, p, false, st)) != SPH_OK) return r;
    // final from here on: pos (the closing kick changes v only), perm, keys
    if (out) CK(copy_out(c, s, *out, 1u | 1u << 8 | 1u << 9, st, 0), "copy out");
    {
        DrhodtInForce fused(c);
        if ((r = do_density(c, s, p, st, true)) != SPH_OK) return r;
        if (out) CK(copy_out(c, s, *out, 1u << 3 | 1u << 4 | 1u << 5, st, 1), "copy out");
        if ((r = do_force(c, s, p, st, true)) != SPH_OK) return r;
    }
    // acc, drhodt, vsigmax
    if (out) CK(copy_out(c, s, *out, 1u << 2 | 1u << 6 | 1u << 7, st, 2), "copy out");
    {
        StageScope sc(c, ST_LEAPFROG, st, 1);
        CK(kick_close(c, s, d_dt, d_time, st), "kick_close");
    }
    {
        StageScope sc(c, ST_REDUCE, st, 2);
        CK(courant_dt(c, s, p, d_dt, st), "timestep");
    }
    if (out) {
        CK(copy_out(c, s, *out, 1u << 1, st, 4), "copy out");  // vel
        CK(cudaMemcpyAsync(out->h_dt, d_dt, sizeof(float), cudaMemcpyDeviceToHost, c.copy_stream), "copy out");
        CK(cudaEventRecord(c.copy_ev[3], c.copy_stream), "copy join");
        CK(cudaStreamWaitEvent(st, c.copy_ev[3], 0), "copy join");
    }
    return SPH_OK;
}

void free_step_graph(Ctx::StepGraph &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = Ctx::StepGraph{};
}

// Record one step into g (on the context's private stream: the caller's may
// be the legacy default stream, which cannot be captured).  With timing on,
// the stage scopes become event-record nodes; their events go back to the
// pool, and every launch points the nodes at fresh ones.
sph_status record_step_graph(Ctx &c, Ctx::StepGraph &g, const sph_state &s, const sph_params &p,
                             float *d_dt, double *d_time, const HostOut *out)
{
    free_step_graph(g);
    CK(configure_density_kernels(p.kernel), "configure density");
    CK(configure_force_kernels(p.kernel), "configure force");
    CK(configure_nlist_kernels(), "configure lists");
    CK(configure_gravity_kernels(), "configure gravity");
    if (!c.capture_stream)
        CK(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking), "capture stream");
    cudaStream_t cs = c.capture_stream;
    c.capture_ev.clear();
    for (auto &x : c.capture_launches) x = 0;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    c.capturing = true;
    const sph_status r = enqueue_step(c, s, p, d_dt, d_time, cs, out);
    c.capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    for (auto &ev : c.capture_ev) c.ev_free.push_back(ev);
    if (r != SPH_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        c.capture_ev.clear();
        return r != SPH_OK ? r : cuda_fail(c, e, "end capture");
    }
    g.graph = graph;
    g.ev_nodes.assign(c.capture_ev.size(), Ctx::StepGraph::EvNode{nullptr, nullptr, 0});
    for (size_t q = 0; q < c.capture_ev.size(); ++q) g.ev_nodes[q].stage = c.capture_ev[q].stage;
    size_t nn = 0;
    cudaError_t e2 = cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e2 == cudaSuccess && nn) e2 = cudaGraphGetNodes(graph, nodes.data(), &nn);
    for (size_t k = 0; e2 == cudaSuccess && k < nn; ++k) {
        cudaGraphNodeType t;
        if ((e2 = cudaGraphNodeGetType(nodes[k], &t)) != cudaSuccess || t != cudaGraphNodeTypeEventRecord)
            continue;
        cudaEvent_t ev = nullptr;
        if ((e2 = cudaGraphEventRecordNodeGetEvent(nodes[k], &ev)) != cudaSuccess) break;
        for (size_t q = 0; q < c.capture_ev.size(); ++q) {
            if (c.capture_ev[q].a == ev) g.ev_nodes[q].a = nodes[k];
            if (c.capture_ev[q].b == ev) g.ev_nodes[q].b = nodes[k];
        }
    }
    c.capture_ev.clear();
    for (const auto &en : g.ev_nodes)
        if (e2 == cudaSuccess && (!en.a || !en.b)) e2 = cudaErrorInvalidResourceHandle;
    if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e2 != cudaSuccess) {
        free_step_graph(g);
        return cuda_fail(c, e2, "step graph");
    }
    for (int k = 0; k < ST_N; ++k) g.launches[k] = c.capture_launches[k];
    return SPH_OK;
}

}  // namespace

extern "C" {

void sph_params_default(sph_params *p)
{
    if (!p) return;
    p->gamma = 5.0f / 3.0f;
    p->hfact = 1.2f;
    p->alpha_av = 1.0f;
    p->beta_av = 2.0f;
    p->alpha_u = 1.0f;
    p->c_cour = 0.3f;
    p->h_tol = 1e-6f;
    p->kernel = 0;
    p->n_leaf = 16;
    p->n_group = 8;
    p->tile = 0;
    p->max_h_iter = 50;
    p->density_iters = 0;
    p->pair_targets = 8;
    p->pair_warps = 4;
    p->pair_unroll = 2;
    for (int a = 0; a < 3; ++a) {
        p->box_lo[a] = 0.f;
        p->box_len[a] = 0.f;
    }
    p->grav_G = 0.f;
    p->grav_eps = 0.01f;
    p->grav_theta = 0.5f;
}

sph_status sph_create(sph_ctx **out, int64_t max_n, int device)
{
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_n < 1 || max_n >= (int64_t)1 << 31) return SPH_ERR_INVALID_ARG;
    sph_ctx *h = new (std::nothrow) sph_ctx();
    if (!h) return SPH_ERR_NOMEM;
    Ctx &c = h->impl;
    c.device = device;
    c.max_n = max_n;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete h;
        return SPH_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete h;
        return SPH_ERR_CUDA;
    }
    c.num_sms = prop.multiProcessorCount;
    const size_t n = (size_t)max_n;
    c.ntiles_cap = div_up(max_n, 2048);
    int nbchop = div_up(max_n, kChopBlock);
    int64_t scan_n = max_n > (int64_t)kLevels * nbchop ? max_n : (int64_t)kLevels * nbchop;
    c.scan_part_cap = div_up(scan_n, 2048) + 16;
    c.red_cap = c.num_sms * 16;
    Tree &t = c.tree;
    t.cap_nodes = (int)(2 * n + 1024 < (size_t)INT32_MAX ? 2 * n + 1024 : INT32_MAX);
    t.cap_groups = (int)n;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(c.keys_alt, n));
    A(dalloc(c.idx_a, n));
    A(dalloc(c.idx_b, n));
    A(dalloc(c.rs_ghist, 10 * 256));
    A(dalloc(c.rs_gstart, 10 * 256));
    A(dalloc(c.rs_status, (size_t)kRsSlots * 256 * c.ntiles_cap));
    A(dalloc(c.rs_tiles, kRsSlots + 1));
    for (int k = 0; k < 4; ++k) A(dalloc(c.tmp4[k], n));
    for (int k = 0; k < 5; ++k) A(dalloc(c.tmp1[k], n));
    A(dalloc(c.tmp_perm, n));
    A(dalloc(t.node_first, t.cap_nodes));
    A(dalloc(t.node_count, t.cap_nodes));
    A(dalloc(t.node_level, t.cap_nodes));
    A(dalloc(t.node_child, t.cap_nodes));
    A(dalloc(t.node_nchild, t.cap_nodes));
    A(dalloc(t.node_parent, t.cap_nodes));
    A(dalloc(t.node_arrive, t.cap_nodes));
    A(dalloc(t.node_lo, t.cap_nodes));
    A(dalloc(t.node_hi, t.cap_nodes));
    A(dalloc(t.node_ref, t.cap_nodes));
    A(dalloc(t.level_start, kLevels + 1));
    A(dalloc(t.grp_ref, t.cap_groups));
    A(dalloc(t.grp_lo, t.cap_groups));
    A(dalloc(t.grp_hi, t.cap_groups));
    A(dalloc(c.nl_idx, n * kNbrCapMax));  // 768 B per particle
    A(dalloc(c.nl_len, n));
    A(dalloc(c.fallback, n));
    A(dalloc(t.rec_ctl, 2));
    if (e == cudaSuccess) e = cudaMemset(t.rec_ctl, 0xff, 2 * sizeof(int));  // no lists yet
    A(dalloc(t.rec_bad, kMaxInstances));
    A(dalloc(t.lv_tree, n));
    A(dalloc(t.lv_grp, n));
    A(dalloc(t.blk_cnt, (size_t)kLevels * nbchop));
    A(dalloc(c.rec, 2 * n));
    A(dalloc(c.prop, n));
    A(dalloc(c.frec, 3 * n));
    A(dalloc(c.vhalf, n));
    A(dalloc(c.active, n));
    A(dalloc(c.g_com, t.cap_nodes));
    A(dalloc(c.g_q0, t.cap_nodes));
    A(dalloc(c.g_q1, t.cap_nodes));
    A(dalloc(c.inst, n));
    A(dalloc(c.bbox_inst, (size_t)6 * kMaxInstances));
    A(dalloc(c.dtmin_inst, kMaxInstances));
    A(dalloc(c.bbox, 8));
    A(dalloc(c.scan_part, c.scan_part_cap));
    A(dalloc(c.red_f, c.red_cap));
    A(dalloc(c.red_d, (size_t)8 * c.red_cap));
    A(dalloc(c.d_err, 1));
    A(dalloc(c.d_counters, C_N));
    A(dalloc(c.d_sizes, SZ_N));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c.h_pinned, 64);
    if (e == cudaSuccess) e = cudaMemset(c.d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c.d_counters, 0, sizeof(unsigned long long) * C_N);
    if (e == cudaSuccess) e = cudaMemset(c.d_sizes, 0, sizeof(int) * SZ_N);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sph_destroy(h);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SPH_ERR_NOMEM : SPH_ERR_CUDA;
    }
    *out = h;
    return SPH_OK;
}

void sph_destroy(sph_ctx *h)
{
    if (!h) return;
    Ctx &c = h->impl;
    cudaSetDevice(c.device);
    cudaDeviceSynchronize();
    release_rollout(c);
    void *ptrs[] = {c.keys_alt, c.idx_a, c.idx_b, c.rs_ghist, c.rs_gstart, c.rs_status, c.rs_tiles, c.tmp4[0], c.tmp4[1], c.tmp4[2],
                    c.tmp4[3], c.tmp1[0], c.tmp1[1], c.tmp1[2], c.tmp1[3], c.tmp1[4], c.tmp_perm,
                    c.tree.node_first, c.tree.node_count, c.tree.node_level, c.tree.node_child,
                    c.tree.node_nchild, c.tree.node_parent, c.tree.node_arrive, c.tree.node_lo,
                    c.tree.node_hi, c.tree.node_ref, c.tree.level_start, c.tree.grp_ref,
                    c.tree.grp_lo, c.tree.grp_hi, c.tree.lv_tree, c.tree.lv_grp, c.tree.blk_cnt,
                    c.nl_idx, c.nl_len, c.fallback,
                    c.tree.rec_ctl, c.tree.rec_bad,
                    c.rec, c.prop, c.frec, c.vhalf, c.active, c.g_com, c.g_q0, c.g_q1, c.inst, c.bbox_inst,
                    c.dtmin_inst,
                    c.bbox, c.scan_part, c.red_f, c.red_d, c.d_err, c.d_counters,
                    c.d_sizes, c.mirror.pos, c.mirror.vel, c.mirror.acc, c.mirror.h, c.mirror.rho,
                    c.mirror.omega, c.mirror.drhodt, c.mirror.vsigmax, c.mirror.perm,
                    c.mirror.keys, c.mirror_dt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c.h_pinned) cudaFreeHost(c.h_pinned);
    if (c.batch_graph) cudaGraphExecDestroy(c.batch_graph);
    for (auto &g : c.step_graph) free_step_graph(g);
    if (c.copy_stream) cudaStreamDestroy(c.copy_stream);
    for (auto &ev : c.copy_ev)
        if (ev) cudaEventDestroy(ev);
    if (c.capture_stream) cudaStreamDestroy(c.capture_stream);
    for (auto &p : c.ev_free) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto &p : c.ev_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    delete h;
}

sph_status sph_build_tree(sph_ctx *h, sph_state *s, const sph_params *p, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (s->n == 0) return SPH_OK;
    return do_tree(c, *s, *p, true, (cudaStream_t)stream);
}

sph_status sph_density(sph_ctx *h, sph_state *s, const sph_params *p, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (s->n == 0) return SPH_OK;
    return do_density(c, *s, *p, (cudaStream_t)stream, false);
}

sph_status sph_force(sph_ctx *h, sph_state *s, const sph_params *p, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (s->n == 0) return SPH_OK;
    return do_force(c, *s, *p, (cudaStream_t)stream, false);
}

sph_status sph_gravity(sph_ctx *h, const sph_state *s, const sph_params *p, float *d_out4,
                       void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, false);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (!(p->grav_G > 0.f)) return fail(c, SPH_ERR_INVALID_ARG, "sph_gravity needs grav_G > 0");
    if (!d_out4 || ((uintptr_t)d_out4 & 15)) return fail(c, SPH_ERR_INVALID_ARG, "d_out4 NULL or not 16-byte aligned");
    if (s->n == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    StageScope sc(c, ST_GRAVITY, st, 2);
    CK(gravity_pass(c, *s, *p, nullptr, (float4 *)d_out4, st), "gravity");
    return SPH_OK;
}

sph_status sph_block_levels(sph_ctx *h, const sph_state *s, const sph_params *p, int max_level,
                            float *d_dt_min, int32_t *d_level, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (max_level < 0 || max_level > kMaxBlockLevel)
        return fail(c, SPH_ERR_INVALID_ARG, "max_level out of range [0, 16]");
    if (!d_dt_min || !d_level) return fail(c, SPH_ERR_INVALID_ARG, "d_dt_min or d_level is NULL");
    if (s->n == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    StageScope sc(c, ST_REDUCE, st, 3);
    CK(courant_dt(c, *s, *p, d_dt_min, st), "block levels: dt");
    CK(block_levels(c, *s, *p, max_level, d_dt_min, d_level, st), "block levels");
    return SPH_OK;
}

sph_status sph_step_block(sph_ctx *h, sph_state *s, const sph_params *p, int max_level,
                          const int32_t *d_level, const float *d_dt_min, double *d_time, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (max_level < 0 || max_level > kMaxBlockLevel)
        return fail(c, SPH_ERR_INVALID_ARG, "max_level out of range [0, 16]");
    if (!d_level || !d_dt_min) return fail(c, SPH_ERR_INVALID_ARG, "d_level or d_dt_min is NULL");
    if (p->grav_G > 0.f) return fail(c, SPH_ERR_INVALID_ARG, "block time steps with gravity are not built");
    if (s->n == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the block starts from a sorted tree: every per-particle array in curve order
    if ((r = do_tree(c, *s, *p, true, st)) != SPH_OK) return r;
    for (int j = 0; j < (1 << max_level); ++j) {
        {
            StageScope sc(c, ST_LEAPFROG, st, 1);
            CK(block_substep(c, *s, *p, d_level, j, max_level, d_dt_min, st), "block substep");
        }
        {
            StageScope sc(c, ST_TREE, st, 2);
            CK(refit_tree(c, *s, st), "refit");
        }
        c.mask = c.active;
        {
            DrhodtInForce fused(c);
            r = do_density(c, *s, *p, st, true);
            if (r == SPH_OK) r = do_force(c, *s, *p, st, true);
        }
        c.mask = nullptr;
        if (r != SPH_OK) return r;
        StageScope sc(c, ST_LEAPFROG, st, 1);
        CK(block_close(c, *s, d_level, max_level, d_dt_min, d_time, st), "block close");
    }
    return SPH_OK;
}

sph_status sph_timestep(sph_ctx *h, const sph_state *s, const sph_params *p, float *d_dt,
                        void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (!d_dt) return fail(c, SPH_ERR_INVALID_ARG, "d_dt is NULL");
    if (s->n == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    StageScope sc(c, ST_REDUCE, st, 2);
    CK(courant_dt(c, *s, *p, d_dt, st), "timestep");
    return SPH_OK;
}

namespace {

// Launch one step as the recorded graph for these arguments (recorded on
// first use; the context keeps the last kStepGraphs).
sph_status step_launch(Ctx &c, const sph_state &s, const sph_params &p, float *d_dt, double *d_time,
                       cudaStream_t st, const HostOut *out)
{
    sph_status r;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap), "capture query");
    if (cap != cudaStreamCaptureStatusNone)  // the caller records a graph of its own
        return enqueue_step(c, s, p, d_dt, d_time, st, out);
    // the graph is valid for exactly these pointers, sizes, parameters and timing mode
    std::vector<unsigned char> key(2 * sizeof(sph_state) + sizeof(sph_params) + 4 * sizeof(void *));
    unsigned char *kp = key.data();
    memcpy(kp, &s, sizeof(sph_state)); kp += sizeof(sph_state);
    const sph_state none{};
    memcpy(kp, out ? out->hs : &none, sizeof(sph_state)); kp += sizeof(sph_state);
    memcpy(kp, &p, sizeof(sph_params)); kp += sizeof(sph_params);
    const void *extra[4] = {d_dt, d_time, out ? out->h_dt : nullptr, (const void *)(intptr_t)(c.timing ? 1 : 0)};
    memcpy(kp, extra, sizeof(extra));
    Ctx::StepGraph *g = nullptr;
    for (auto &x : c.step_graph)
        if (x.exec && x.key == key) g = &x;
    if (!g) {
        g = &c.step_graph[0];  // the least recently used slot
        for (auto &x : c.step_graph)
            if (x.used < g->used) g = &x;
        if ((r = record_step_graph(c, *g, s, p, d_dt, d_time, out)) != SPH_OK) return r;
        g->key = key;
    }
    g->used = ++c.step_graph_clock;
    if (c.timing) {
        for (const auto &en : g->ev_nodes) {
            Ctx::EvPair ev{};
            if (!take_event_pair(c, ev)) return cuda_fail(c, cudaErrorMemoryAllocation, "timing events");
            ev.stage = en.stage;
            CK(cudaGraphExecEventRecordNodeSetEvent(g->exec, en.a, ev.a), "timing event node");
            CK(cudaGraphExecEventRecordNodeSetEvent(g->exec, en.b, ev.b), "timing event node");
            c.ev_pending.push_back(ev);
        }
    }
    for (int k = 0; k < ST_N; ++k) c.pending_launches[k] += g->launches[k];
    CK(cudaGraphLaunch(g->exec, st), "step graph launch");
    // the graph rebuilt the lists for p.kernel
    c.nl_kernel = p.kernel;
    c.nl_stride = list_cap(p.kernel);
    return SPH_OK;
}

}  // namespace

sph_status sph_step(sph_ctx *h, sph_state *s, const sph_params *p, float *d_dt, double *d_time,
                    void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (!d_dt) return fail(c, SPH_ERR_INVALID_ARG, "d_dt is NULL");
    if (s->n == 0) return SPH_OK;
    return step_launch(c, *s, *p, d_dt, d_time, (cudaStream_t)stream, nullptr);
}

sph_status sph_step_host(sph_ctx *h, sph_state *hs, const sph_params *p, int n_steps, float *h_dt,
                         void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    if (!hs || !h_dt || n_steps < 0) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    sph_status r = check_params(c, p);
    if (r != SPH_OK) return r;
    if (hs->n < 0 || hs->n > c.max_n) return fail(c, SPH_ERR_INVALID_ARG, "n out of range");
    const int64_t n = hs->n;
    if (n == 0) return SPH_OK;
    if (!hs->pos || !hs->vel || !hs->acc || !hs->h || !hs->rho || !hs->omega || !hs->drhodt ||
        !hs->vsigmax || !hs->perm || !hs->keys)
        return fail(c, SPH_ERR_INVALID_ARG, "NULL host array");
    cudaStream_t st = (cudaStream_t)stream;
    if (c.mirror_n < n) {
        sph_state &m = c.mirror;
        void *old[] = {m.pos, m.vel, m.acc, m.h, m.rho, m.omega, m.drhodt, m.vsigmax, m.perm, m.keys};
        for (void *q : old)
            if (q) cudaFree(q);
        m = sph_state{};
        cudaError_t e = cudaSuccess;
        auto A = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
        size_t nn = (size_t)c.max_n;
        A(cudaMalloc((void **)&m.pos, nn * 16));
        A(cudaMalloc((void **)&m.vel, nn * 16));
        A(cudaMalloc((void **)&m.acc, nn * 16));
        A(cudaMalloc((void **)&m.h, nn * 4));
        A(cudaMalloc((void **)&m.rho, nn * 4));
        A(cudaMalloc((void **)&m.omega, nn * 4));
        A(cudaMalloc((void **)&m.drhodt, nn * 4));
        A(cudaMalloc((void **)&m.vsigmax, nn * 4));
        A(cudaMalloc((void **)&m.perm, nn * 4));
        A(cudaMalloc((void **)&m.keys, nn * 8));
        if (!c.mirror_dt) A(cudaMalloc((void **)&c.mirror_dt, sizeof(float)));
        if (e != cudaSuccess) return cuda_fail(c, e, "step_host mirror allocation");
        c.mirror_n = c.max_n;
    }
    sph_state d = c.mirror;
    d.n = n;
    const cudaMemcpyKind H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(d.pos, hs->pos, n * 16, H2D, st), "H2D pos");
    CK(cudaMemcpyAsync(d.vel, hs->vel, n * 16, H2D, st), "H2D vel");
    CK(cudaMemcpyAsync(d.acc, hs->acc, n * 16, H2D, st), "H2D acc");
    CK(cudaMemcpyAsync(d.h, hs->h, n * 4, H2D, st), "H2D h");
    CK(cudaMemcpyAsync(d.perm, hs->perm, n * 4, H2D, st), "H2D perm");
    CK(cudaMemcpyAsync(c.mirror_dt, h_dt, sizeof(float), H2D, st), "H2D dt");
    // With all host buffers pinned, the last step copies each output back as
    // soon as it is final, on the copy stream, while the step runs on.
    bool pinned = true;
    for (const void *q : {(const void *)hs->pos, (const void *)hs->vel, (const void *)hs->acc,
                          (const void *)hs->h, (const void *)hs->rho, (const void *)hs->omega,
                          (const void *)hs->drhodt, (const void *)hs->vsigmax, (const void *)hs->perm,
                          (const void *)hs->keys}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess || at.type != cudaMemoryTypeHost) pinned = false;
    }
    (void)cudaGetLastError();  // an unregistered pointer may leave an error behind
    if (pinned && !c.copy_stream) {
        CK(cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking), "copy stream");
        for (auto &ev : c.copy_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "copy events");
    }
    float *dt_pinned = reinterpret_cast<float *>(c.h_pinned + 8);  // the next dt, read after the sync
    for (int k = 0; k < n_steps; ++k) {
        const HostOut out{hs, dt_pinned};
        const bool last = k == n_steps - 1 && pinned;
        if ((r = step_launch(c, d, *p, c.mirror_dt, nullptr, st, last ? &out : nullptr)) != SPH_OK) return r;
    }
    if (n_steps > 0 && pinned) {
        if ((r = sph_sync(h, stream)) != SPH_OK) return r;
        *h_dt = *dt_pinned;
        return SPH_OK;
    }
    CK(cudaMemcpyAsync(hs->pos, d.pos, n * 16, D2H, st), "D2H pos");
    CK(cudaMemcpyAsync(hs->vel, d.vel, n * 16, D2H, st), "D2H vel");
    CK(cudaMemcpyAsync(hs->acc, d.acc, n * 16, D2H, st), "D2H acc");
    CK(cudaMemcpyAsync(hs->h, d.h, n * 4, D2H, st), "D2H h");
    CK(cudaMemcpyAsync(hs->rho, d.rho, n * 4, D2H, st), "D2H rho");
    CK(cudaMemcpyAsync(hs->omega, d.omega, n * 4, D2H, st), "D2H omega");
    CK(cudaMemcpyAsync(hs->drhodt, d.drhodt, n * 4, D2H, st), "D2H drhodt");
    CK(cudaMemcpyAsync(hs->vsigmax, d.vsigmax, n * 4, D2H, st), "D2H vsigmax");
    CK(cudaMemcpyAsync(hs->perm, d.perm, n * 4, D2H, st), "D2H perm");
    CK(cudaMemcpyAsync(hs->keys, d.keys, n * 8, D2H, st), "D2H keys");
    CK(cudaMemcpyAsync(h_dt, c.mirror_dt, sizeof(float), D2H, st), "D2H dt");
    return sph_sync(h, stream);
}

namespace {

sph_status check_batch(Ctx &c, const sph_state *s, const int64_t *d_offsets, int n_inst)
{
    if (!d_offsets) return fail(c, SPH_ERR_INVALID_ARG, "d_offsets is NULL");
    if (n_inst < 1 || n_inst > kMaxInstances)
        return fail(c, SPH_ERR_INVALID_ARG, "n_inst must be 1..65536");
    if (s->n < n_inst) return fail(c, SPH_ERR_INVALID_ARG, "every instance needs a particle");
    return SPH_OK;
}

// enqueue one leapfrog step of every instance of a batch (no host sync)
cudaError_t enqueue_batch_step(Ctx &c, const sph_state &s, const sph_params &p, const Batch &b,
                               float *d_dt, double *d_time, cudaStream_t st)
{
    cudaError_t e = kick_drift(c, s, p, d_dt, st, &b);
    if (e == cudaSuccess) e = build_tree(c, s, p, false, st, &b);
    {
        DrhodtInForce fused(c);
        if (e == cudaSuccess) e = density_pass(c, s, p, st, &b);
        if (e == cudaSuccess) e = force_prep(c, s, p, st);
        if (e == cudaSuccess) e = force_pass(c, s, p, st, &b);
    }
    if (e == cudaSuccess && p.grav_G > 0.f) e = gravity_pass(c, s, p, (float4 *)s.acc, nullptr, st, &b);
    if (e == cudaSuccess) e = kick_close(c, s, d_dt, d_time, st, &b);
    if (e == cudaSuccess) e = courant_dt(c, s, p, d_dt, st, &b);
    return e;
}

}  // namespace

sph_status sph_batch_evaluate(sph_ctx *h, sph_state *s, const int64_t *d_offsets, int n_inst,
                              const sph_params *p, float *d_dt, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if ((r = check_batch(c, s, d_offsets, n_inst)) != SPH_OK) return r;
    if (!d_dt) return fail(c, SPH_ERR_INVALID_ARG, "d_dt is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    Batch b{d_offsets, n_inst};
    const int n = (int)s->n;
    CK(instance_map(c, d_offsets, n_inst, n, st), "instance map");
    CK(build_tree(c, *s, *p, true, st, &b), "batch build_tree");
    CK(density_pass(c, *s, *p, st, &b), "batch density");
    CK(force_prep(c, *s, *p, st), "batch force_prep");
    CK(force_pass(c, *s, *p, st, &b), "batch force");
    // with self-gravity on, acc takes its term as in sph_force and the batched step
    if (p->grav_G > 0.f) CK(gravity_pass(c, *s, *p, (float4 *)s->acc, nullptr, st, &b), "batch gravity");
    CK(courant_dt(c, *s, *p, d_dt, st, &b), "batch timestep");
    return SPH_OK;
}

sph_status sph_batch_step(sph_ctx *h, sph_state *s, const int64_t *d_offsets, int n_inst,
                          int n_steps, const sph_params *p, float *d_dt, double *d_time,
                          void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, true);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if ((r = check_batch(c, s, d_offsets, n_inst)) != SPH_OK) return r;
    if (!d_dt || n_steps < 0) return fail(c, SPH_ERR_INVALID_ARG, "d_dt is NULL or n_steps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    Batch b{d_offsets, n_inst};
    CK(instance_map(c, d_offsets, n_inst, (int)s->n, st), "instance map");
    // the graph is valid for exactly these pointers, sizes and parameters
    std::vector<unsigned char> key(sizeof(sph_state) + sizeof(sph_params) + 4 * sizeof(void *));
    unsigned char *kp = key.data();
    memcpy(kp, s, sizeof(sph_state)); kp += sizeof(sph_state);
    memcpy(kp, p, sizeof(sph_params)); kp += sizeof(sph_params);
    const void *extra[4] = {d_offsets, d_dt, d_time, (const void *)(intptr_t)n_inst};
    memcpy(kp, extra, sizeof(extra));
    if (!c.batch_graph || key != c.batch_graph_key) {
        if (c.batch_graph) {
            cudaGraphExecDestroy(c.batch_graph);
            c.batch_graph = nullptr;
        }
        CK(configure_density_kernels(p->kernel), "configure density");
        CK(configure_force_kernels(p->kernel), "configure force");
        CK(configure_nlist_kernels(), "configure lists");
        CK(configure_gravity_kernels(), "configure gravity");
        // record on a private stream: the caller's may be the legacy default
        // stream, which cannot be captured
        if (!c.capture_stream)
            CK(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking), "capture stream");
        cudaStream_t cs = c.capture_stream;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = enqueue_batch_step(c, *s, *p, b, d_dt, d_time, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) return cuda_fail(c, e, "batch step capture");
        if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
        cudaError_t e3 = cudaGraphInstantiate(&c.batch_graph, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            c.batch_graph = nullptr;
            return cuda_fail(c, e3, "graph instantiate");
        }
        c.batch_graph_key = key;
    }
    for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(c.batch_graph, st), "graph launch");
    // the graph rebuilt the lists for p->kernel
    c.nl_kernel = p->kernel;
    c.nl_stride = list_cap(p->kernel);
    return SPH_OK;
}

sph_status sph_conserved(sph_ctx *h, const sph_state *s, double *d_out8, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, false);
    if (r != SPH_OK) return r;
    if (!d_out8) return fail(c, SPH_ERR_INVALID_ARG, "d_out8 is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (s->n == 0) {
        CK(cudaMemsetAsync(d_out8, 0, 8 * sizeof(double), st), "memset");
        return SPH_OK;
    }
    StageScope sc(c, ST_REDUCE, st, 2);
    CK(conserved(c, *s, d_out8, st), "conserved");
    return SPH_OK;
}

sph_status sph_neighbours(sph_ctx *h, const sph_state *s, const sph_params *p, int mode,
                          int64_t *d_off, int32_t *d_idx, int64_t cap, int64_t *h_total,
                          void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    sph_status r = check_state(c, s, false);
    if (r != SPH_OK) return r;
    if ((r = check_params(c, p)) != SPH_OK) return r;
    if (mode < 0 || mode > 3 || !d_off || !h_total)
        return fail(c, SPH_ERR_INVALID_ARG, "mode must be 0..3; d_off and h_total required");
    cudaStream_t st = (cudaStream_t)stream;
    if (s->n == 0) {
        *h_total = 0;
        CK(cudaMemsetAsync(d_off, 0, sizeof(int64_t), st), "memset");
        return sph_sync(h, stream);
    }
    if (mode >= 2) {
        int missing = 0;
        CK(list_sets(c, *s, *p, mode - 2, d_off, d_idx, cap, h_total, &missing, st), "list sets");
        sph_status r2 = sph_sync(h, stream);
        if (r2 != SPH_OK) return r2;
        if (missing > 0) {
            char buf[96];
            snprintf(buf, sizeof(buf), "%d particles have no neighbour list (overflow)", missing);
            return fail(c, SPH_ERR_TILE_OVERFLOW, buf);
        }
        return SPH_OK;
    }
    // the force set needs the current h in the node/group bounds
    CK(update_hmax(c, *s, *p, st), "update_hmax");
    CK(neighbour_lists(c, *s, *p, mode, d_off, d_idx, cap, h_total, st), "neighbours");
    return sph_sync(h, stream);
}

sph_status sph_get_tree(sph_ctx *h, int32_t *h_level, int32_t *h_first, int32_t *h_count,
                        int32_t *h_nchild, int32_t *h_child, int64_t node_cap,
                        int32_t *h_gfirst, int32_t *h_gcount, int64_t group_cap,
                        int64_t *n_nodes, int64_t *n_groups)
{
    if (!h || !n_nodes || !n_groups) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    int sz[SZ_N];
    CK(cudaDeviceSynchronize(), "tree sync");
    CK(cudaMemcpy(sz, c.d_sizes, sizeof(sz), cudaMemcpyDeviceToHost), "sizes copy");
    *n_nodes = sz[SZ_NODES];
    *n_groups = sz[SZ_GROUPS];
    const Tree &t = c.tree;
    if (sz[SZ_NODES] <= node_cap) {
        size_t b = sizeof(int32_t) * (size_t)sz[SZ_NODES];
        if (h_level) CK(cudaMemcpy(h_level, t.node_level, b, cudaMemcpyDeviceToHost), "copy");
        if (h_first) CK(cudaMemcpy(h_first, t.node_first, b, cudaMemcpyDeviceToHost), "copy");
        if (h_count) CK(cudaMemcpy(h_count, t.node_count, b, cudaMemcpyDeviceToHost), "copy");
        if (h_nchild) CK(cudaMemcpy(h_nchild, t.node_nchild, b, cudaMemcpyDeviceToHost), "copy");
        if (h_child) CK(cudaMemcpy(h_child, t.node_child, b, cudaMemcpyDeviceToHost), "copy");
    }
    if (sz[SZ_GROUPS] <= group_cap && sz[SZ_GROUPS] > 0) {
        std::vector<int2> g((size_t)sz[SZ_GROUPS]);
        CK(cudaMemcpy(g.data(), t.grp_ref, sizeof(int2) * g.size(), cudaMemcpyDeviceToHost), "copy");
        for (size_t k = 0; k < g.size(); ++k) {
            if (h_gfirst) h_gfirst[k] = g[k].x;
            if (h_gcount) h_gcount[k] = g[k].y;
        }
    }
    return SPH_OK;
}

sph_status sph_test_lookback_timeout(sph_ctx *h, int spin_cap, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    if (spin_cap < 1 || spin_cap > (1 << 20)) return fail(c, SPH_ERR_INVALID_ARG, "spin_cap must be 1..2^20");
    CK(sort_lookback_probe(c, spin_cap, (cudaStream_t)stream), "look-back probe");
    return SPH_OK;
}

sph_status sph_get_stats(sph_ctx *h, sph_stats *out)
{
    if (!h || !out) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    unsigned long long v[C_N];
    int sz[SZ_N];
    CK(cudaDeviceSynchronize(), "stats sync");
    CK(cudaMemcpy(v, c.d_counters, sizeof(v), cudaMemcpyDeviceToHost), "stats copy");
    CK(cudaMemcpy(sz, c.d_sizes, sizeof(sz), cudaMemcpyDeviceToHost), "sizes copy");
    CK(cudaMemset(c.d_counters, 0, sizeof(v)), "stats reset");
    out->density_pairs = v[C_DENS_PAIRS];
    out->density_candidates = v[C_DENS_CAND];
    out->force_pairs = v[C_FORCE_PAIRS];
    out->force_candidates = v[C_FORCE_CAND];
    out->newton_iters = v[C_NEWTON];
    out->density_rewalks = v[C_REWALK];
    out->streamed_groups = v[C_STREAMED];
    out->list_entries = v[C_LIST_ENTRIES];
    out->list_overflows = v[C_LIST_OVERFLOW];
    out->force_rewalks = v[C_FORCE_FB];
    out->gravity_cells = v[C_GRAV_CELLS];
    out->gravity_particles = v[C_GRAV_PARTS];
    out->n_nodes = (uint64_t)sz[SZ_NODES];
    out->n_groups = (uint64_t)sz[SZ_GROUPS];
    return SPH_OK;
}

sph_status sph_set_timing(sph_ctx *h, int enable)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    h->impl.timing = enable != 0;
    return SPH_OK;
}

sph_status sph_get_timing(sph_ctx *h, double *ms, int64_t *launches)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    for (auto &p : c.ev_pending) {
        CK(cudaEventSynchronize(p.b), "timing sync");
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, p.a, p.b), "timing elapsed");
        c.stage_ms[p.stage] += t;
        c.ev_free.push_back(p);
    }
    c.ev_pending.clear();
    for (int k = 0; k < ST_N; ++k) {
        if (ms) ms[k] = c.stage_ms[k];
        if (launches) launches[k] = c.pending_launches[k];
        c.stage_ms[k] = 0;
        c.pending_launches[k] = 0;
    }
    return SPH_OK;
}

sph_status sph_sync(sph_ctx *h, void *stream)
{
    if (!h) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st), "sync");
    CK(cudaMemcpy(c.h_pinned, c.d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    int w = c.h_pinned[0];
    if (w == 0) return SPH_OK;
    CK(cudaMemset(c.d_err, 0, sizeof(int)), "error reset");
    std::string msg = "device reported:";
    sph_status first = SPH_OK;
    for (int k = 1; k <= (int)SPH_ERR_TIMEOUT; ++k)
        if (w & (1 << k)) {
            msg += " ";
            msg += status_text((sph_status)k);
            msg += ";";
            if (first == SPH_OK) first = (sph_status)k;
        }
    c.last_error = msg;
    return first;
}

const char *sph_last_error(sph_ctx *h)
{
    if (!h) return "NULL context";
    return h->impl.last_error.c_str();
}

}  // extern "C"
