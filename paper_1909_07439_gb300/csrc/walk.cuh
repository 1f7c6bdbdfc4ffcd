// Group-wise tree walk (Sect. 3.2): one warp walks the tree for one group of
// particles (Barnes' vectorisation).  Nodes are tested 32 at a time, one per
// lane; opened internal nodes push their child range (first, count) on a
// warp-private stack in shared memory, opened leaves queue their particle
// range (the compressed (first, count) tuple of the paper, expanded here one
// 32-particle chunk at a time).  Each chunk is handed to the caller's
// functor with one candidate particle per lane, so candidate loads are
// coalesced (a leaf's particles are contiguous in curve order).
//
// The stack is LIFO, which keeps it short; the paper's walk is breadth first.
// The set of leaves visited is the same.
#pragma once

#include "sph_internal.cuh"

namespace sph {

constexpr int kStack = 224;  // node-range stack entries per warp
constexpr int kRQ = 64;      // leaf-range queue entries per warp
constexpr float kOpenSlack = 1.0f + 1e-5f;  // keeps FP32 box tests conservative

// Nearest-image separation along one axis: d - L if d > L/2, d + L if
// d < -L/2.  Positions lie in one period, so |d| < L and, with
// L/2 <= |d| < L, the correction is exact; L = 0 (open axis) leaves d as it is.
__device__ __forceinline__ float wrap_sep(float d, float L)
{
    const float hL = 0.5f * L;
    d = d > hL ? __fsub_rn(d, L) : d;
    return d < -hL ? __fadd_rn(d, L) : d;
}

struct WalkTree {
    const float4 *__restrict__ node_lo;   // x, y, z, h_max
    const float4 *__restrict__ node_hi;
    const int2 *__restrict__ node_ref;    // leaf (first, count) / internal (child, -nchild)
    Period per;                           // periodic axes (box distances over images)
};

struct WalkSmem {
    int2 stk[kStack];
    int2 rq[kRQ];
    int nodes[32];
};

__device__ __forceinline__ unsigned lane_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

__device__ __forceinline__ int warp_sum_i(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// L2 policy for particle data that neighbouring groups read again soon: keep
// it in L2 while the neighbour lists stream through.
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Particle i's position/mass and velocity/energy as one 32-byte record
// (rec[2 i], rec[2 i + 1]), read with a single 256-bit load.
__device__ __forceinline__ void ld_rec(const float4 *rec, int i, uint64_t pol, float4 &p, float4 &v)
{
    asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=f"(p.x), "=f"(p.y), "=f"(p.z), "=f"(p.w), "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(rec + 2 * (size_t)i), "l"(pol));
}

__device__ __forceinline__ float4 ld_keep(const float4 *a, int i, uint64_t pol)
{
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(a + i), "l"(pol));
    return v;
}

// canonical FP32 squared distance: (dx*dx + dy*dy) + dz*dz, no fusion
__device__ __forceinline__ float canon_r2(float xi, float yi, float zi, float xj, float yj, float zj)
{
    float dx = __fsub_rn(xi, xj), dy = __fsub_rn(yi, yj), dz = __fsub_rn(zi, zj);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// the same with the nearest image on the periodic axes of P
__device__ __forceinline__ float canon_r2p(float xi, float yi, float zi, float xj, float yj, float zj,
                                           const Period &P)
{
    float dx = wrap_sep(__fsub_rn(xi, xj), P.x), dy = wrap_sep(__fsub_rn(yi, yj), P.y),
          dz = wrap_sep(__fsub_rn(zi, zj), P.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// The same canonical squared distance for two targets at once with the
// packed FP32x2 instructions: every element is rounded to nearest exactly as
// in canon_r2 (x - y is formed as x + (-y), which is the same operation).
__device__ __forceinline__ float2 canon_r2_x2(float2 tx, float2 ty, float2 tz, float xj, float yj,
                                              float zj)
{
    const float2 dx = __fadd2_rn(tx, make_float2(-xj, -xj));
    const float2 dy = __fadd2_rn(ty, make_float2(-yj, -yj));
    const float2 dz = __fadd2_rn(tz, make_float2(-zj, -zj));
    return __fadd2_rn(__fadd2_rn(__fmul2_rn(dx, dx), __fmul2_rn(dy, dy)), __fmul2_rn(dz, dz));
}

// canon_r2_x2 with the nearest image on the periodic axes of P
__device__ __forceinline__ float2 canon_r2_x2p(float2 tx, float2 ty, float2 tz, float xj, float yj,
                                               float zj, const Period &P)
{
    float2 dx = __fadd2_rn(tx, make_float2(-xj, -xj));
    float2 dy = __fadd2_rn(ty, make_float2(-yj, -yj));
    float2 dz = __fadd2_rn(tz, make_float2(-zj, -zj));
    dx = make_float2(wrap_sep(dx.x, P.x), wrap_sep(dx.y, P.x));
    dy = make_float2(wrap_sep(dy.x, P.y), wrap_sep(dy.y, P.y));
    dz = make_float2(wrap_sep(dz.x, P.z), wrap_sep(dz.y, P.z));
    return __fadd2_rn(__fadd2_rn(__fmul2_rn(dx, dx), __fmul2_rn(dy, dy)), __fmul2_rn(dz, dz));
}

// Targets of a warp's batch as coordinate pairs for canon_r2_x2: element t of
// the batch is component (t & 1) of pair t >> 1; unused slots sit far away.
template <int TB>
struct TargetPairs {
    float2 x[TB / 2], y[TB / 2], z[TB / 2];
    __device__ __forceinline__ void set(int t, float4 p)
    {
        reinterpret_cast<float *>(x)[t] = p.x;
        reinterpret_cast<float *>(y)[t] = p.y;
        reinterpret_cast<float *>(z)[t] = p.z;
    }
};

// squared distance between two axis-aligned boxes (0 if they overlap)
__device__ __forceinline__ float box_dist2(float4 alo, float4 ahi, float4 blo, float4 bhi)
{
    float dx = fmaxf(0.f, fmaxf(blo.x - ahi.x, alo.x - bhi.x));
    float dy = fmaxf(0.f, fmaxf(blo.y - ahi.y, alo.y - bhi.y));
    float dz = fmaxf(0.f, fmaxf(blo.z - ahi.z, alo.z - bhi.z));
    return dx * dx + dy * dy + dz * dz;
}

// Gap along one axis between [alo, ahi] and the nearest of the images of
// [blo, bhi] shifted by 0, +L, -L (L > 0).  The shifted gaps are lower
// bounds (rounded down), so a box test on them stays conservative.
__device__ __forceinline__ float gap_periodic(float alo, float ahi, float blo, float bhi, float L)
{
    const float g0 = fmaxf(0.f, fmaxf(blo - ahi, alo - bhi));
    const float gp = fmaxf(0.f, fmaxf(__fsub_rd(__fadd_rd(blo, L), ahi), __fsub_rd(alo, __fadd_ru(bhi, L))));
    const float gm = fmaxf(0.f, fmaxf(__fsub_rd(__fsub_rd(blo, L), ahi), __fsub_rd(alo, __fsub_ru(bhi, L))));
    return fminf(g0, fminf(gp, gm));
}

// box_dist2 over the nearest images on the periodic axes of the walk's tree
__device__ __forceinline__ float box_dist2_t(const WalkTree &T, float4 alo, float4 ahi, float4 blo,
                                             float4 bhi)
{
    if (!T.per.any()) return box_dist2(alo, ahi, blo, bhi);
    float dx = T.per.x > 0.f ? gap_periodic(alo.x, ahi.x, blo.x, bhi.x, T.per.x)
                             : fmaxf(0.f, fmaxf(blo.x - ahi.x, alo.x - bhi.x));
    float dy = T.per.y > 0.f ? gap_periodic(alo.y, ahi.y, blo.y, bhi.y, T.per.y)
                             : fmaxf(0.f, fmaxf(blo.y - ahi.y, alo.y - bhi.y));
    float dz = T.per.z > 0.f ? gap_periodic(alo.z, ahi.z, blo.z, bhi.z, T.per.z)
                             : fmaxf(0.f, fmaxf(blo.z - ahi.z, alo.z - bhi.z));
    return dx * dx + dy * dy + dz * dz;
}

// box_dist2_t with the periodicity known at compile time: PER = false takes
// the open-box distance without the run-time check (the same value then)
template <bool PER>
__device__ __forceinline__ float box_dist2_c(const WalkTree &T, float4 alo, float4 ahi, float4 blo, float4 bhi)
{
    return PER ? box_dist2_t(T, alo, ahi, blo, bhi) : box_dist2(alo, ahi, blo, bhi);
}

// One step of a walk: pop whole stack entries from the top (at most 32
// nodes), test the nodes one per lane, and push the child ranges of opened
// internal nodes.  On return this lane's opened leaf, if any, is in
// (leaf = true, ref = (first, count), node).  Sets ok = false if the stack
// overflowed.
//   force_mode = false: open a node if dist < sqrt(reach2 / kOpenSlack)
//   force_mode = true : open a node if dist < 2 max(hgroup, node_scale h_max(node))
__device__ __forceinline__ void walk_step(const WalkTree &T, float4 glo, float4 ghi, float reach2,
                                          bool force_mode, float hgroup, float node_scale,
                                          WalkSmem &sm, int &sp, bool &ok, bool &leaf, int2 &ref,
                                          int &node)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    int2 e = lane < sp ? sm.stk[sp - 1 - lane] : make_int2(0, 0);
    int sz = lane < sp ? e.y : 0;
    int inc = sz;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    unsigned take = __ballot_sync(0xffffffffu, lane < sp && inc <= 32);
    int k = __popc(take);
    int total = __shfl_sync(0xffffffffu, inc, k - 1);
    if (lane < k)
        for (int q = 0, ex = inc - sz; q < sz; ++q) sm.nodes[ex + q] = e.x + q;
    sp -= k;
    __syncwarp();
    node = lane < total ? sm.nodes[lane] : -1;
    __syncwarp();
    bool open = false;
    leaf = false;
    ref = make_int2(0, 0);
    if (node >= 0) {
        float4 lo = __ldg(&T.node_lo[node]);
        float4 hi = __ldg(&T.node_hi[node]);
        ref = __ldg(&T.node_ref[node]);
        float d2 = box_dist2_t(T, glo, ghi, lo, hi);
        float r2 = reach2;
        if (force_mode) {
            float R = 2.0f * fmaxf(hgroup, lo.w * node_scale);
            r2 = R * R * kOpenSlack;
        }
        open = d2 < r2;
        leaf = ref.y >= 0;
    }
    unsigned bint = __ballot_sync(0xffffffffu, open && !leaf);
    if (open && !leaf) {
        int p = sp + __popc(bint & lt);
        if (p < kStack) sm.stk[p] = make_int2(ref.x, -ref.y);
    }
    sp += __popc(bint);
    if (sp > kStack) {
        ok = false;
        sp = kStack;
    }
    leaf = open && leaf;
}

// Walk the tree below node `root` for a group with box [glo, ghi].
//   force_mode = false: open a node if dist < reach (reach = 2 * padded h of the group)
//   force_mode = true : open a node if dist < 2 max(h_group, node_scale h_max(node))
// chunk(j): called warp-uniformly with this lane's candidate j (-1: none).
// Returns false if the stack overflowed (results then incomplete).
template <class ChunkFn>
__device__ bool walk_group(const WalkTree &T, int root, float4 glo, float4 ghi, float reach,
                           bool force_mode, float hgroup, WalkSmem &sm, ChunkFn &&chunk,
                           float node_scale = 1.f)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    bool ok = true;
    int sp = 1;
    if (lane == 0) sm.stk[0] = make_int2(root, 1);  // the group's (instance) root
    int rq_head = 0, rq_tail = 0, rq_off = 0, pending = 0;
    const float reach2 = reach * reach * kOpenSlack;
    __syncwarp();
    while (sp > 0 || pending > 0) {
        if (sp > 0) {
            bool leaf;
            int2 ref;
            int node;
            walk_step(T, glo, ghi, reach2, force_mode, hgroup, node_scale, sm, sp, ok, leaf, ref, node);
            unsigned bleaf = __ballot_sync(0xffffffffu, leaf);
            if (leaf) sm.rq[(rq_tail + __popc(bleaf & lt)) % kRQ] = ref;
            rq_tail += __popc(bleaf);
            pending += warp_sum_i(leaf ? ref.y : 0);
            __syncwarp();
        }
        // hand out full chunks; the tail too once the stack is empty
        while (pending >= 32 || (sp == 0 && pending > 0)) {
            int filled = 0, myj = -1;
            while (filled < 32 && pending > 0) {
                int2 r = sm.rq[rq_head % kRQ];
                if (r.y - rq_off <= 0) {  // never happens for a valid tree; no spinning
                    ++rq_head;
                    rq_off = 0;
                    if (rq_head > rq_tail) pending = 0;
                    continue;
                }
                int take = min(r.y - rq_off, 32 - filled);
                if (lane >= filled && lane < filled + take) myj = r.x + rq_off + (lane - filled);
                filled += take;
                rq_off += take;
                pending -= take;
                if (rq_off == r.y) {
                    ++rq_head;
                    rq_off = 0;
                }
            }
            chunk(myj);
        }
    }
    __syncwarp();
    return ok;
}

// Walk the tree below `root` for the box [glo, ghi] in force mode and store
// every opened leaf as (node, first particle) in out[0 .. cap).  Returns the
// number of leaves, or -1 if they did not fit or the stack overflowed.
__device__ __forceinline__ int walk_leaves(const WalkTree &T, int root, float4 glo, float4 ghi,
                                           float hgroup, float node_scale, WalkSmem &sm, int2 *out,
                                           int cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    bool ok = true;
    int sp = 1, nout = 0;
    if (lane == 0) sm.stk[0] = make_int2(root, 1);
    __syncwarp();
    while (sp > 0) {
        bool leaf;
        int2 ref;
        int node;
        walk_step(T, glo, ghi, 0.f, true, hgroup, node_scale, sm, sp, ok, leaf, ref, node);
        const unsigned bleaf = __ballot_sync(0xffffffffu, leaf);
        if (leaf) {
            const int p = nout + __popc(bleaf & lt);
            if (p < cap) out[p] = make_int2(node, ref.x);
        }
        nout += __popc(bleaf);
        __syncwarp();
    }
    return ok && nout <= cap ? nout : -1;
}

// Shared memory of a wide walk: W nodes per lane and step.
template <int W, int STK>
struct WalkSmemW {
    int2 stk[STK];
    int nodes[32 * W];
};

// walk_leaves with W nodes tested per lane and step (fewer, wider steps: the
// node loads of a step are independent, so a step costs about one memory
// latency whatever W is).  Same opening test and result set as walk_leaves;
// the order of `out` differs.
template <int W, int STK, bool PER = true>
__device__ __forceinline__ int walk_leaves_wide(const WalkTree &T, int root, float4 glo, float4 ghi,
                                                float hgroup, float node_scale, WalkSmemW<W, STK> &sm,
                                                int2 *out, int cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    bool ok = true;
    int sp = 1, nout = 0;
    if (lane == 0) sm.stk[0] = make_int2(root, 1);
    __syncwarp();
    while (sp > 0) {
        // pop whole entries from the top, at most 32 W nodes
        const int2 e = lane < sp ? sm.stk[sp - 1 - lane] : make_int2(0, 0);
        const int sz = lane < sp ? e.y : 0;
        int inc = sz;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const unsigned take = __ballot_sync(0xffffffffu, lane < sp && inc <= 32 * W);
        const int k = __popc(take);
        const int total = __shfl_sync(0xffffffffu, inc, k - 1);
        if (lane < k)
            for (int q = 0, ex = inc - sz; q < sz; ++q) sm.nodes[ex + q] = e.x + q;
        sp -= k;
        __syncwarp();
        int node[W];
        float4 lo[W], hi[W];
        int2 ref[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            node[w] = w * 32 + lane < total ? sm.nodes[w * 32 + lane] : -1;
            lo[w] = hi[w] = make_float4(0.f, 0.f, 0.f, 0.f);
            ref[w] = make_int2(0, 0);
            if (node[w] >= 0) {
                lo[w] = __ldg(&T.node_lo[node[w]]);
                hi[w] = __ldg(&T.node_hi[node[w]]);
                ref[w] = __ldg(&T.node_ref[node[w]]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int w = 0; w < W; ++w) {
            bool open = false;
            if (node[w] >= 0) {
                const float d2 = box_dist2_c<PER>(T, glo, ghi, lo[w], hi[w]);
                const float R = 2.0f * fmaxf(hgroup, lo[w].w * node_scale);
                open = d2 < R * R * kOpenSlack;
            }
            const bool leaf = open && ref[w].y >= 0, inner = open && ref[w].y < 0;
            const unsigned bint = __ballot_sync(0xffffffffu, inner);
            if (inner) {
                const int p = sp + __popc(bint & lt);
                if (p < STK) sm.stk[p] = make_int2(ref[w].x, -ref[w].y);
            }
            sp += __popc(bint);
            if (sp > STK) {
                ok = false;
                sp = STK;
            }
            const unsigned bleaf = __ballot_sync(0xffffffffu, leaf);
            if (leaf) {
                const int p = nout + __popc(bleaf & lt);
                if (p < cap) out[p] = make_int2(node[w], ref[w].x);
            }
            nout += __popc(bleaf);
        }
        __syncwarp();
        if (nout > cap) break;  // the result is -1 whatever else the walk finds
    }
    return ok && nout <= cap ? nout : -1;
}

// Hand a batch of cnt targets of group g, from its target b0 on, to the
// walking kernels, in items of at most 8 targets (their batch size):
// item = (g, first target | count << 16).  Called by one lane.
__device__ __forceinline__ void push_fallback_batch(int2 *fallback, int *n_fallback, int g, int b0,
                                                    int cnt)
{
    for (int k = 0; k < cnt; k += 8)
        fallback[atomicAdd(n_fallback, 1)] = make_int2(g, (b0 + k) | (min(8, cnt - k) << 16));
}

// Candidate slots of a group: runs[m] = (first particle, first slot) for
// m < nrun and runs[nrun] = (-1, number of candidates).  Slot k belongs to the
// run r with runs[r].y <= k < runs[r + 1].y; r only moves forward, so a lane
// visiting ascending slots keeps its r between calls.
__device__ __forceinline__ int slot_particle(const int2 *runs, int &r, int k)
{
    while (runs[r + 1].y <= k) ++r;
    return runs[r].x + (k - runs[r].y);
}

}  // namespace sph
