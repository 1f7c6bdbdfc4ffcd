// Internal definitions shared by the library's translation units.
// Not part of the public ABI (include/sph.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "sph.h"

namespace sph {

constexpr int kMaxLevel = 21;        // 21 bits per axis, 63-bit keys
constexpr int kLevels = 22;          // levels 0..21
constexpr int kWarp = 32;
constexpr int kMaxInstances = 65536;  // instances in one batch
constexpr int kRsSlots = 14;         // radix passes of one sort at most (4 + 8 + 2)
// Neighbour-list entries per particle (also the lists' stride): at least
// twice the mean list length of the kernel at its usual hfact (list radius
// (1 + pad) R max(h_i, h_j): about 63 entries for M4 at hfact 1.2, 80 for
// Wendland C6 at 1.3, 90 for M6 at 0.9); multiples of 4 for the 16-byte list
// loads.  The list array is allocated for the largest.
constexpr int kNbrCapMax = 192;
constexpr int kMaxBlockLevel = 16;  // deepest level of the block time steps
inline int list_cap(int kernel) { return kernel == 0 ? 128 : 192; }
constexpr float kListPad = 0.03f;    // neighbour-list radius margin, relative to h

// stage ids for the per-stage timers
enum Stage {
    ST_TREE = 0, ST_DENSITY = 1, ST_FORCE = 2, ST_REDUCE = 3, ST_LEAPFROG = 4, ST_PREP = 5, ST_LISTS = 6,
    ST_GRAVITY = 7, ST_N = 8
};

// device error word: bit (1 << status) per condition seen
__device__ __forceinline__ void raise_error(int *err, sph_status code)
{
    atomicOr(err, 1 << (int)code);
}

// device counters (indices into Ctx::d_counters)
enum Counter {
    C_DENS_PAIRS = 0,
    C_DENS_CAND = 1,
    C_FORCE_PAIRS = 2,
    C_FORCE_CAND = 3,
    C_NEWTON = 4,
    C_REWALK = 5,
    C_STREAMED = 6,
    C_LIST_ENTRIES = 7,
    C_LIST_OVERFLOW = 8,
    C_FORCE_FB = 9,
    C_GRAV_CELLS = 10,
    C_GRAV_PARTS = 11,
    C_N = 12
};

// tree-size scalars on the device (Ctx::d_sizes)
// SZ_WORK / SZ_WORK2: work counters of the persistent kernels; SZ_FALLBACK:
// entries in Ctx::fallback; SZ_BAD_OFFSETS: the batch offsets failed their check
enum Size { SZ_NODES = 0, SZ_GROUPS = 1, SZ_WORK = 3, SZ_FALLBACK = 4, SZ_WORK2 = 5, SZ_BAD_OFFSETS = 6,
            SZ_N = 8 };

struct Tree {
    int cap_nodes = 0;
    int cap_groups = 0;
    // nodes, level-major, first-particle order inside a level
    int *node_first = nullptr, *node_count = nullptr, *node_level = nullptr;
    int *node_child = nullptr, *node_nchild = nullptr, *node_parent = nullptr;
    int *node_arrive = nullptr;
    float4 *node_lo = nullptr;   // x, y, z, h_max
    float4 *node_hi = nullptr;   // x, y, z, unused
    int2 *node_ref = nullptr;    // leaf: (first, count); internal: (child_first, -nchild)
    int *level_start = nullptr;  // [kLevels + 1]
    // groups: terminal nodes of the n_group chop
    int2 *grp_ref = nullptr;     // (first, count)
    float4 *grp_lo = nullptr;    // x, y, z, h_max
    float4 *grp_hi = nullptr;
    // Validity of the neighbour lists built by the density pass:
    // rec_ctl[1] != 0: lists stale (tree rebuilt since the density pass);
    // rec_bad[k] != 0: an h of instance k (0 without a batch) outgrew its pad;
    // rec_ctl[0] != 0: some rec_bad[k] is set (the relist pass's gate).
    int *rec_ctl = nullptr;
    int *rec_bad = nullptr;
    // chop scratch
    int *lv_tree = nullptr, *lv_grp = nullptr;
    int *blk_cnt = nullptr;      // [kLevels][nb]
};

// a batch of independent instances packed back to back
struct Batch {
    const int64_t *offsets;  // device [n_inst + 1]
    int n_inst;
};

struct Ctx {
    int device = 0;
    int64_t max_n = 0;
    int num_sms = 0;
    std::string last_error;

    // sort scratch
    uint64_t *keys_alt = nullptr;
    uint32_t *idx_a = nullptr, *idx_b = nullptr;
    uint32_t *rs_ghist = nullptr;   // [10][256] digit counts of every pass
    uint32_t *rs_gstart = nullptr;  // [10][256] their exclusive scans
    uint32_t *rs_status = nullptr;  // [kRsSlots][ntiles][256] look-back words, one slot per pass
    int *rs_tiles = nullptr;        // [kRsSlots] tile counters, then the full-sort flag
    int ntiles_cap = 0;

    // gather scratch
    float4 *tmp4[4] = {nullptr, nullptr, nullptr, nullptr};
    float *tmp1[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t *tmp_perm = nullptr;

    Tree tree;

    // Neighbour lists (curve order): particle i owns nl_idx[i * nl_stride ...],
    // nl_len[i] entries (-1: none).  Entry j is in i's list if
    // r_ij < R (1 + pad) max(h_i, h_j) at the h the density pass started from,
    // R the support radius of kernel nl_kernel, the kernel of the last full
    // build (-1: none); nl_stride = list_cap(nl_kernel).  A pass with another
    // kernel treats the lists as stale.
    int *nl_idx = nullptr;
    int *nl_len = nullptr;
    int nl_stride = 128;
    int nl_kernel = -1;
    // Inside a step the force pass writes drho/dt (its pressure-work sum is
    // the same sum up to a per-particle factor) and the density pass gathers
    // positions only; standalone density passes write drho/dt themselves.
    bool drhodt_in_force = false;
    int2 *fallback = nullptr;  // (group, first batch slot) handed to the walk kernels

    // per-particle scratch
    float4 *rec = nullptr;    // [2 n]: pos, vel of each particle side by side (32-byte records)
    float4 *prop = nullptr;   // h, rho, 1/(rho Omega), c_s
    // [3 n]: the force record of each particle: (x, m), (v, (gamma - 1) u),
    // ((R h)^2, G C / (h^4 rho Omega), alpha_AV c_s, rho)
    float4 *frec = nullptr;
    float4 *vhalf = nullptr;  // half-step v, u of the leapfrog
    // [n] block time steps: per-slot flag of the particles whose step ends in
    // the current substep; mask points at it while the passes run for those
    // particles only (nullptr otherwise)
    uint8_t *active = nullptr;
    const uint8_t *mask = nullptr;
    // [cap_nodes] gravity moments: (centre of mass, M), (Qxx, Qyy, Qzz, r_open^2),
    // (Qxy, Qxz, Qyz, -)
    float4 *g_com = nullptr, *g_q0 = nullptr, *g_q1 = nullptr;
    float *bbox = nullptr;    // [8]: lo xyz, size, then scratch
    // batches
    int *inst = nullptr;       // [max_n] instance of each slot
    int *bbox_inst = nullptr;  // [6 * kMaxInstances] per-instance boxes
    int *dtmin_inst = nullptr; // [kMaxInstances] per-instance min h / vsigmax (ordered ints)
    cudaGraphExec_t batch_graph = nullptr;
    cudaStream_t capture_stream = nullptr;  // graphs are recorded here, launched on the caller's
    cudaStream_t copy_stream = nullptr;     // sph_step_host's output copies (inside its graph)
    cudaEvent_t copy_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<unsigned char> batch_graph_key;

    // scan scratch
    int *scan_part = nullptr;
    int scan_part_cap = 0;

    // reductions
    float *red_f = nullptr;     // block minima
    double *red_d = nullptr;    // block partial sums [8][nb]
    int red_cap = 0;

    int *d_err = nullptr;
    unsigned long long *d_counters = nullptr;
    int *d_sizes = nullptr;
    int *h_pinned = nullptr;  // small pinned host buffer

    // work buffers of sph_rollout (allocated on its first call, released by
    // sph_destroy through release_rollout)
    void *rollout = nullptr;

    // host-buffer mirror (sph_step_host)
    sph_state mirror{};
    float *mirror_dt = nullptr;
    int64_t mirror_n = 0;

    // timing
    bool timing = false;
    struct EvPair { cudaEvent_t a, b; int stage; };
    std::vector<EvPair> ev_free, ev_pending;
    double stage_ms[ST_N] = {};
    int64_t stage_launches[ST_N] = {};
    int64_t pending_launches[ST_N] = {};

    // sph_step recorded as CUDA graphs, one per (state, params, dt, time,
    // timing) seen last; with timing on, the graph holds the stage events as
    // event-record nodes, pointed at fresh events before every launch
    struct StepGraph {
        std::vector<unsigned char> key;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        struct EvNode { cudaGraphNode_t a, b; int stage; };
        std::vector<EvNode> ev_nodes;
        int64_t launches[ST_N] = {};
        uint64_t used = 0;
    };
    static constexpr int kStepGraphs = 4;
    StepGraph step_graph[kStepGraphs];
    uint64_t step_graph_clock = 0;
    bool capturing = false;  // stage scopes record into the capture lists below
    std::vector<EvPair> capture_ev;
    int64_t capture_launches[ST_N] = {};
};

// Periods of the axes for periodic boundaries (0: open axis), and the lower
// corner of the periodic box.
struct Period {
    float x, y, z;
    __host__ __device__ bool any() const { return x > 0.f || y > 0.f || z > 0.f; }
};
inline Period period_of(const sph_params &p) { return Period{p.box_len[0], p.box_len[1], p.box_len[2]}; }
inline float3 box_lo_of(const sph_params &p) { return make_float3(p.box_lo[0], p.box_lo[1], p.box_lo[2]); }

// ---------------------------------------------------------------------------
// launchers (host functions) implemented in the .cu files
// ---------------------------------------------------------------------------
// tree.cu
cudaError_t build_tree(Ctx &c, const sph_state &s, const sph_params &p, bool full_permute,
                       cudaStream_t st, const Batch *batch = nullptr);
cudaError_t instance_map(Ctx &c, const int64_t *d_offsets, int n_inst, int n, cudaStream_t st);
// node and group h_max of the current h; gate != nullptr: only if *gate != 0
cudaError_t update_hmax(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                        const int *gate = nullptr);
// c.rec from the state's pos and vel (build_tree writes it too)
cudaError_t pack_records(Ctx &c, const sph_state &s, cudaStream_t st);
cudaError_t scan_exclusive_int(Ctx &c, const int *in, int *out, int n, int *total_dev,
                               cudaStream_t st);
// test hook: a sort pass whose look-back predecessor never publishes
cudaError_t sort_lookback_probe(Ctx &c, int spin_cap, cudaStream_t st);
// nlist.cu
cudaError_t nlist_pass(Ctx &c, const sph_state &s, const sph_params &p, float pad,
                       cudaStream_t st, const Batch *batch = nullptr);
// After the density pass: rebuild, at the final h, the lists of the
// instances where an h outgrew the list pad (rec_bad), so the force pass and
// the adjoint passes read lists instead of walking; returns at once (gated
// launches) when no h outgrew its pad.
cudaError_t relist_pass(Ctx &c, const sph_state &s, const sph_params &p, float pad,
                        cudaStream_t st, const Batch *batch = nullptr);
// lists built for another kernel than p.kernel are marked stale (the passes
// then walk the tree)
cudaError_t check_list_kernel(Ctx &c, const sph_params &p, cudaStream_t st);
cudaError_t configure_nlist_kernels();
// density.cu (density_pass = density_lists + density_solve; density_pass
// expects the node and group h_max of the current h, as build_tree leaves them)
cudaError_t density_lists(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                          const Batch *batch = nullptr, bool refresh_hmax = true);
cudaError_t density_solve(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                          const Batch *batch = nullptr);
cudaError_t density_pass(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                         const Batch *batch = nullptr);
cudaError_t neighbour_lists(Ctx &c, const sph_state &s, const sph_params &p, int mode,
                            int64_t *d_off, int32_t *d_idx, int64_t cap, int64_t *h_total,
                            cudaStream_t st);
// the same sets read from the neighbour lists that the density and force
// passes use (built here at the current h); *h_missing = particles whose
// list overflowed (their rows are empty)
cudaError_t list_sets(Ctx &c, const sph_state &s, const sph_params &p, int mode, int64_t *d_off,
                      int32_t *d_idx, int64_t cap, int64_t *h_total, int *h_missing,
                      cudaStream_t st);
// force.cu
// hmax_now: also refresh node and group h_max (force_pass refreshes them
// itself, only when a batch falls back to a walk)
cudaError_t force_prep(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                       bool hmax_now = false);
cudaError_t force_pass(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                       const Batch *batch = nullptr);
// kernel attributes and occupancy of the pair kernels of smoothing kernel
// `kernel` (before any graph capture)
cudaError_t configure_density_kernels(int kernel);
cudaError_t configure_force_kernels(int kernel);
// gravity.cu: the moments pass and the Barnes-Hut walk; adds G a to acc.xyz
// and/or writes (G a, G phi) to out (either may be null)
cudaError_t gravity_pass(Ctx &c, const sph_state &s, const sph_params &p, float4 *acc, float4 *out,
                         cudaStream_t st, const Batch *batch = nullptr);
cudaError_t configure_gravity_kernels();
// integrate.cu
// with a batch, d_dt and d_time hold one value per instance
// (drifted positions wrap into the periodic box of p)
cudaError_t kick_drift(Ctx &c, const sph_state &s, const sph_params &p, const float *d_dt,
                       cudaStream_t st, const Batch *batch = nullptr);
// block time steps (integrate.cu): substep j's kicks, drift, prediction and
// due flags; the closing kicks of the due particles; the levels from Eq. 8
cudaError_t block_substep(Ctx &c, const sph_state &s, const sph_params &p, const int *d_level, int j,
                          int max_level, const float *d_dt_min, cudaStream_t st);
cudaError_t block_close(Ctx &c, const sph_state &s, const int *d_level, int max_level,
                        const float *d_dt_min, double *d_time, cudaStream_t st);
cudaError_t block_levels(Ctx &c, const sph_state &s, const sph_params &p, int max_level,
                         const float *d_dt_min, int *d_level, cudaStream_t st);
// node and group boxes and h_max from the current positions and h, without
// re-sorting (tree.cu)
cudaError_t refit_tree(Ctx &c, const sph_state &s, cudaStream_t st);
cudaError_t kick_close(Ctx &c, const sph_state &s, const float *d_dt, double *d_time,
                       cudaStream_t st, const Batch *batch = nullptr);
cudaError_t courant_dt(Ctx &c, const sph_state &s, const sph_params &p, float *d_dt,
                       cudaStream_t st, const Batch *batch = nullptr);
cudaError_t conserved(Ctx &c, const sph_state &s, double *d_out8, cudaStream_t st);
// rollout.cu
void release_rollout(Ctx &c);

// helpers
inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Launch shape of the list pair kernels (density and force), from sph_params
// (0 selects the default): targets per warp batch (4, 8 or 16; a target gets
// 32 / targets lanes), warps per block (1, 2, 4 or 8) and list entries per
// lane and iteration of the force kernel (2 or 4).
struct PairShape {
    int targets, warps, unroll;
};
inline PairShape pair_shape(const sph_params &p)
{
    return PairShape{p.pair_targets ? p.pair_targets : 8, p.pair_warps ? p.pair_warps : 4,
                     p.pair_unroll ? p.pair_unroll : 2};
}

// drho/dt from the force pass while in scope (the density and force passes of a step)
struct DrhodtInForce {
    Ctx &c;
    explicit DrhodtInForce(Ctx &cc) : c(cc) { c.drhodt_in_force = true; }
    ~DrhodtInForce() { c.drhodt_in_force = false; }
};

// lanes per target for a batch of nt targets (a power of two, nt * L <= 32)
__host__ __device__ inline int lanes_per_target(int nt)
{
    return nt > 8 ? 2 : nt > 4 ? 4 : nt > 2 ? 8 : nt > 1 ? 16 : 32;
}

// number of blocks used by the chop's per-block counting (1024 particles each)
constexpr int kChopBlock = 1024;

}  // namespace sph

struct sph_ctx {
    sph::Ctx impl;
};
