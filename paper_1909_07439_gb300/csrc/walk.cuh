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

struct WalkTree {
    const float4 *__restrict__ node_lo;   // x, y, z, h_max
    const float4 *__restrict__ node_hi;
    const int2 *__restrict__ node_ref;    // leaf (first, count) / internal (child, -nchild)
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

// canonical FP32 squared distance: (dx*dx + dy*dy) + dz*dz, no fusion
__device__ __forceinline__ float canon_r2(float xi, float yi, float zi, float xj, float yj, float zj)
{
    float dx = __fsub_rn(xi, xj), dy = __fsub_rn(yi, yj), dz = __fsub_rn(zi, zj);
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

// Walk the tree below node `root` for a group with box [glo, ghi].
//   force_mode = false: open a node if dist < reach (reach = 2 * padded h of the group)
//   force_mode = true : open a node if dist < 2 max(h_group, h_max(node))
// chunk(j): called warp-uniformly with this lane's candidate j (-1: none).
// Returns false if the stack overflowed (results then incomplete).
// Opened leaves are appended, in order, to rec[0 .. *rec_n) when rec is
// given (*rec_n = -1 once more than rec_cap were opened).  In force mode a
// node's h_max is scaled by node_scale.
template <class ChunkFn>
__device__ bool walk_group(const WalkTree &T, int root, float4 glo, float4 ghi, float reach,
                           bool force_mode, float hgroup, WalkSmem &sm, ChunkFn &&chunk,
                           float node_scale = 1.f, int2 *rec = nullptr, int *rec_n = nullptr,
                           int rec_cap = 0)
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
            // pop whole entries from the top, at most 32 nodes
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
            int node = lane < total ? sm.nodes[lane] : -1;
            __syncwarp();
            bool open = false, leaf = false;
            int2 ref = make_int2(0, 0);
            if (node >= 0) {
                float4 lo = __ldg(&T.node_lo[node]);
                float4 hi = __ldg(&T.node_hi[node]);
                ref = __ldg(&T.node_ref[node]);
                float d2 = box_dist2(glo, ghi, lo, hi);
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
            unsigned bleaf = __ballot_sync(0xffffffffu, open && leaf);
            if (open && leaf) sm.rq[(rq_tail + __popc(bleaf & lt)) % kRQ] = ref;
            if (rec) {
                int nr = *rec_n;
                if (nr >= 0) {
                    if (nr + __popc(bleaf) > rec_cap) {
                        nr = -1;
                    } else {
                        if (open && leaf) rec[nr + __popc(bleaf & lt)] = ref;
                        nr += __popc(bleaf);
                    }
                }
                __syncwarp();
                if (lane == 0) *rec_n = nr;
                __syncwarp();
            }
            rq_tail += __popc(bleaf);
            pending += warp_sum_i(open && leaf ? ref.y : 0);
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

// Hand the particles of recorded leaf ranges (global, in walk order) to
// chunk() in 32-particle chunks, as walk_group would.
template <class ChunkFn>
__device__ void replay_ranges(const int2 *__restrict__ ranges, int count, ChunkFn &&chunk)
{
    const int lane = threadIdx.x & 31;
    int filled = 0, myj = -1;
    for (int b = 0; b < count; b += 32) {
        const int2 mine = b + lane < count ? __ldg(&ranges[b + lane]) : make_int2(0, 0);
        const int nb = min(32, count - b);
        for (int k = 0; k < nb; ++k) {
            const int first = __shfl_sync(0xffffffffu, mine.x, k);
            const int cnt = __shfl_sync(0xffffffffu, mine.y, k);
            int off = 0;
            while (off < cnt) {
                const int take = min(cnt - off, 32 - filled);
                if (lane >= filled && lane < filled + take) myj = first + off + (lane - filled);
                filled += take;
                off += take;
                if (filled == 32) {
                    chunk(myj);
                    filled = 0;
                    myj = -1;
                }
            }
        }
    }
    if (filled > 0) chunk(myj);
    __syncwarp();
}

}  // namespace sph
