// Self-gravity: the a_grav term of Eq. 9 by the Barnes-Hut walk (Sect. 2.4
// and 3.2) on the octree the hydro passes use, with Plummer softening eps.
//
// gravity_moments_kernel: per node the mass M, the centre of mass X, the
// traceless quadrupole Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab) (d = x - X)
// and the opening radius r_open = l / theta + delta (l the longest edge of
// the node's box, delta the distance from X to the box centre).  Leaves sum
// their particles; a parent is formed by the last of its children to finish
// (an arrival counter per node, no waiting) from the children's moments,
// Q shifted by the parallel-axis rule.
//
// gravity_kernel: one warp per group (Barnes' vectorisation, as in the
// paper's walk): the warp tests 32 nodes at a time; a node whose centre of
// mass is farther than r_open from the group's box is accepted for the whole
// group (a cell: monopole + quadrupole), an opened leaf contributes its
// particles one by one (softened pair sum), an opened internal node pushes
// its children.  Cells and particles are staged in per-warp lists in shared
// memory and evaluated 32 at a time, each target's sum split over
// 32 / (targets) lanes and combined by shuffles at the end.
//   cell:      phi = -M/r - (d.Q.d) / (2 r^5),
//              a   = -M d / r^3 + Q d / r^5 - 5 (d.Q.d) d / (2 r^7)
//   particle:  phi = -m/r,  a = -m d / r^3
// with d = x_i - X (or x_i - x_j) and r^2 = |d|^2 + eps^2.  FP32 throughout.
#include "walk.cuh"

namespace sph {

constexpr int kGWarps = 4;     // warps per block
constexpr int kGStack = 256;   // node-range stack entries per warp
constexpr int kGRQ = 64;       // leaf-range queue entries per warp
constexpr int kGCell = 64;     // cell list entries per warp

struct GravSmem {
    int2 stk[kGStack];
    int nodes[32];
    int2 rq[kGRQ];
    float4 c_com[kGCell];   // X, M
    float4 c_q0[kGCell];    // Qxx, Qyy, Qzz, unused
    float4 c_q1[kGCell];    // Qxy, Qxz, Qyz, unused
    float4 p_pos[32];
    int p_idx[32];
};

struct GravArgs {
    const float4 *pos;
    const int2 *node_ref;
    const float4 *com, *q0, *q1;  // q0.w = r_open^2
    const int2 *grp_ref;
    const float4 *grp_lo, *grp_hi;
    const int *sizes;
    int *work;
    const int *inst;
    float4 *acc;   // += G a (xyz), or nullptr
    float4 *out;   // = (G a, G phi), or nullptr
    float G, eps2;
    int *err;
    unsigned long long *counters;
};

__global__ void gravity_moments_kernel(const float4 *__restrict__ pos, Tree t, float4 *com, float4 *q0,
                                       float4 *q1, const int *sizes, float theta)
{
    const int nn = sizes[SZ_NODES];
    auto finish = [&](int k, float M, float3 X, float Q[6]) {
        const float4 lo = t.node_lo[k], hi = t.node_hi[k];
        const float l = fmaxf(hi.x - lo.x, fmaxf(hi.y - lo.y, hi.z - lo.z));
        const float cx = 0.5f * (lo.x + hi.x) - X.x, cy = 0.5f * (lo.y + hi.y) - X.y,
                    cz = 0.5f * (lo.z + hi.z) - X.z;
        const float r_open = l / theta + sqrtf(cx * cx + cy * cy + cz * cz);
        com[k] = make_float4(X.x, X.y, X.z, M);
        q0[k] = make_float4(Q[0], Q[1], Q[2], r_open * r_open);
        q1[k] = make_float4(Q[3], Q[4], Q[5], 0.f);
    };
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
        if (t.node_nchild[k] != 0) continue;
        const int s = t.node_first[k], e = s + t.node_count[k];
        float M = 0.f;
        float3 X = make_float3(0.f, 0.f, 0.f);
        for (int i = s; i < e; ++i) {
            const float4 p = pos[i];
            M += p.w;
            X.x += p.w * p.x; X.y += p.w * p.y; X.z += p.w * p.z;
        }
        X.x /= M; X.y /= M; X.z /= M;
        float Q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int i = s; i < e; ++i) {
            const float4 p = pos[i];
            const float dx = p.x - X.x, dy = p.y - X.y, dz = p.z - X.z, d2 = dx * dx + dy * dy + dz * dz;
            Q[0] += p.w * (3.f * dx * dx - d2);
            Q[1] += p.w * (3.f * dy * dy - d2);
            Q[2] += p.w * (3.f * dz * dz - d2);
            Q[3] += p.w * 3.f * dx * dy;
            Q[4] += p.w * 3.f * dx * dz;
            Q[5] += p.w * 3.f * dy * dz;
        }
        finish(k, M, X, Q);
        // the last child to arrive forms its parent (and so on up)
        int cur = k;
        while (true) {
            const int p = t.node_parent[cur];
            if (p < 0) break;
            __threadfence();
            const int old = atomicAdd(&t.node_arrive[p], 1);
            if (old != t.node_nchild[p] - 1) break;
            t.node_arrive[p] = 0;  // ready for the next pass
            __threadfence();
            const int cf = t.node_child[p], nc = t.node_nchild[p];
            float Mp = 0.f;
            float3 Xp = make_float3(0.f, 0.f, 0.f);
            for (int q = cf; q < cf + nc; ++q) {
                const float4 c = __ldcg(&com[q]);
                Mp += c.w;
                Xp.x += c.w * c.x; Xp.y += c.w * c.y; Xp.z += c.w * c.z;
            }
            Xp.x /= Mp; Xp.y /= Mp; Xp.z /= Mp;
            float Qp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int q = cf; q < cf + nc; ++q) {
                const float4 c = __ldcg(&com[q]), a = __ldcg(&q0[q]), b = __ldcg(&q1[q]);
                const float dx = c.x - Xp.x, dy = c.y - Xp.y, dz = c.z - Xp.z,
                            d2 = dx * dx + dy * dy + dz * dz;
                Qp[0] += a.x + c.w * (3.f * dx * dx - d2);
                Qp[1] += a.y + c.w * (3.f * dy * dy - d2);
                Qp[2] += a.z + c.w * (3.f * dz * dz - d2);
                Qp[3] += b.x + c.w * 3.f * dx * dy;
                Qp[4] += b.y + c.w * 3.f * dx * dz;
                Qp[5] += b.z + c.w * 3.f * dy * dz;
            }
            finish(p, Mp, Xp, Qp);
            cur = p;
        }
    }
}

__global__ void __launch_bounds__(kGWarps * 32) gravity_kernel(GravArgs a)
{
    __shared__ GravSmem smv[kGWarps];
    GravSmem &sm = smv[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int ng = a.sizes[SZ_GROUPS];
    unsigned long long n_cell = 0, n_part = 0;

    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.work, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int2 gr = a.grp_ref[g];
        const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        const int nt = min(gr.y, 32);
        const int L = nt > 16 ? 1 : nt > 8 ? 2 : nt > 4 ? 4 : nt > 2 ? 8 : nt > 1 ? 16 : 32;
        const int t = lane / L, sub = lane % L;
        const bool act = t < nt;
        const int i = gr.x + (act ? t : 0);
        const float4 xt = a.pos[i];
        float ax = 0.f, ay = 0.f, az = 0.f, phi = 0.f;

        auto eval_cells = [&](int nc) {
            __syncwarp();
#pragma unroll 4
            for (int e = sub; e < nc; e += L) {
                const float4 c = sm.c_com[e], qa = sm.c_q0[e], qb = sm.c_q1[e];
                const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z;
                const float rinv = rsqrtf(dx * dx + dy * dy + dz * dz + a.eps2);
                const float rinv2 = rinv * rinv, rinv3 = rinv * rinv2, rinv5 = rinv3 * rinv2;
                const float qx = qa.x * dx + qb.x * dy + qb.y * dz;
                const float qy = qb.x * dx + qa.y * dy + qb.z * dz;
                const float qz = qb.y * dx + qb.z * dy + qa.z * dz;
                const float dqd = dx * qx + dy * qy + dz * qz;
                const float s = -c.w * rinv3 - 2.5f * dqd * rinv5 * rinv2;
                ax += s * dx + qx * rinv5;
                ay += s * dy + qy * rinv5;
                az += s * dz + qz * rinv5;
                phi -= c.w * rinv + 0.5f * dqd * rinv5;
            }
            if (act && sub == 0) n_cell += (unsigned long long)nc;
            __syncwarp();
        };
        auto eval_parts = [&](int np) {
            __syncwarp();
#pragma unroll 4
            for (int e = sub; e < np; e += L) {
                const float4 pj = sm.p_pos[e];
                const bool self = sm.p_idx[e] == i;
                const float dx = xt.x - pj.x, dy = xt.y - pj.y, dz = xt.z - pj.z;
                const float rinv = rsqrtf(dx * dx + dy * dy + dz * dz + a.eps2);
                const float mr = self ? 0.f : pj.w * rinv;
                const float mr3 = mr * rinv * rinv;
                ax -= mr3 * dx;
                ay -= mr3 * dy;
                az -= mr3 * dz;
                phi -= mr;
            }
            if (act && sub == 0) n_part += (unsigned long long)np;
            __syncwarp();
        };

        int sp = 1, ncell = 0, rq_head = 0, rq_tail = 0, rq_off = 0, pending = 0;
        bool ok = true;
        if (lane == 0) sm.stk[0] = make_int2(a.inst ? a.inst[gr.x] : 0, 1);
        __syncwarp();
        while (sp > 0 || pending > 0 || ncell > 0) {
            if (sp > 0) {
                // pop whole stack entries from the top, at most 32 nodes
                const int2 e = lane < sp ? sm.stk[sp - 1 - lane] : make_int2(0, 0);
                const int sz = lane < sp ? e.y : 0;
                int inc = sz;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const unsigned take = __ballot_sync(0xffffffffu, lane < sp && inc <= 32);
                const int k = __popc(take);
                const int total = __shfl_sync(0xffffffffu, inc, k - 1);
                if (lane < k)
                    for (int q = 0, ex = inc - sz; q < sz; ++q) sm.nodes[ex + q] = e.x + q;
                sp -= k;
                __syncwarp();
                const int node = lane < total ? sm.nodes[lane] : -1;
                __syncwarp();
                bool cell = false, leaf = false, inner = false;
                int2 ref = make_int2(0, 0);
                float4 c = make_float4(0.f, 0.f, 0.f, 0.f), qa = c, qb = c;
                if (node >= 0) {
                    c = __ldg(&a.com[node]);
                    qa = __ldg(&a.q0[node]);
                    ref = __ldg(&a.node_ref[node]);
                    // distance from the group's box to the node's centre of mass
                    const float dx = fmaxf(0.f, fmaxf(glo.x - c.x, c.x - ghi.x));
                    const float dy = fmaxf(0.f, fmaxf(glo.y - c.y, c.y - ghi.y));
                    const float dz = fmaxf(0.f, fmaxf(glo.z - c.z, c.z - ghi.z));
                    cell = dx * dx + dy * dy + dz * dz > qa.w;
                    leaf = !cell && ref.y >= 0;
                    inner = !cell && ref.y < 0;
                    if (cell) qb = __ldg(&a.q1[node]);
                }
                const unsigned bint = __ballot_sync(0xffffffffu, inner);
                if (inner) {
                    const int p = sp + __popc(bint & lt);
                    if (p < kGStack) sm.stk[p] = make_int2(ref.x, -ref.y);
                }
                sp += __popc(bint);
                if (sp > kGStack) {
                    ok = false;
                    sp = kGStack;
                }
                const unsigned bcell = __ballot_sync(0xffffffffu, cell);
                if (cell) {
                    const int p = ncell + __popc(bcell & lt);
                    sm.c_com[p] = c;
                    sm.c_q0[p] = qa;
                    sm.c_q1[p] = qb;
                }
                ncell += __popc(bcell);
                const unsigned bleaf = __ballot_sync(0xffffffffu, leaf);
                if (leaf) sm.rq[(rq_tail + __popc(bleaf & lt)) % kGRQ] = ref;
                rq_tail += __popc(bleaf);
                pending += warp_sum_i(leaf ? ref.y : 0);
                __syncwarp();
            }
            if (ncell >= 32 || (sp == 0 && ncell > 0)) {
                eval_cells(ncell);
                ncell = 0;
            }
            // particles of opened leaves, 32 at a time (the tail once the walk is done)
            while (pending >= 32 || (sp == 0 && pending > 0)) {
                int filled = 0, myj = -1;
                while (filled < 32 && pending > 0) {
                    const int2 r = sm.rq[rq_head % kGRQ];
                    if (r.y - rq_off <= 0) {  // never for a valid tree; no spinning
                        ++rq_head;
                        rq_off = 0;
                        if (rq_head > rq_tail) pending = 0;
                        continue;
                    }
                    const int take = min(r.y - rq_off, 32 - filled);
                    if (lane >= filled && lane < filled + take) myj = r.x + rq_off + (lane - filled);
                    filled += take;
                    rq_off += take;
                    pending -= take;
                    if (rq_off == r.y) {
                        ++rq_head;
                        rq_off = 0;
                    }
                }
                __syncwarp();
                if (lane < filled) {
                    sm.p_pos[lane] = __ldg(&a.pos[myj]);
                    sm.p_idx[lane] = myj;
                }
                eval_parts(filled);
            }
        }
        if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
        for (int o = L >> 1; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            az += __shfl_xor_sync(0xffffffffu, az, o);
            phi += __shfl_xor_sync(0xffffffffu, phi, o);
        }
        if (act && sub == 0) {
            if (a.out) a.out[i] = make_float4(a.G * ax, a.G * ay, a.G * az, a.G * phi);
            if (a.acc) {
                float4 v = a.acc[i];
                v.x += a.G * ax;
                v.y += a.G * ay;
                v.z += a.G * az;
                a.acc[i] = v;
            }
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_cell += __shfl_xor_sync(0xffffffffu, n_cell, o);
        n_part += __shfl_xor_sync(0xffffffffu, n_part, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_GRAV_CELLS], n_cell);
        atomicAdd(&a.counters[C_GRAV_PARTS], n_part);
    }
}

static cudaError_t configure_gravity(int &blocks)
{
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int nb_cached = 1;
    if (!configured) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gravity_kernel, kGWarps * 32, 0);
        if (e != cudaSuccess) return e;
        nb_cached = nb > 0 ? nb : 1;
        configured = true;
    }
    blocks = nb_cached;
    return cudaSuccess;
}

cudaError_t configure_gravity_kernels()
{
    int b;
    return configure_gravity(b);
}

cudaError_t gravity_pass(Ctx &c, const sph_state &s, const sph_params &p, float4 *acc, float4 *out,
                         cudaStream_t st, const Batch *batch)
{
    int blocks = 1;
    cudaError_t e = configure_gravity(blocks);
    if (e != cudaSuccess) return e;
    const int n = (int)s.n;
    int mgrid = (int)((c.tree.cap_nodes + 255) / 256);
    if (mgrid > c.num_sms * 16) mgrid = c.num_sms * 16;
    gravity_moments_kernel<<<mgrid, 256, 0, st>>>((const float4 *)s.pos, c.tree, c.g_com, c.g_q0, c.g_q1,
                                                  c.d_sizes, p.grav_theta);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GravArgs a{};
    a.pos = (const float4 *)s.pos;
    a.node_ref = c.tree.node_ref;
    a.com = c.g_com;
    a.q0 = c.g_q0;
    a.q1 = c.g_q1;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.inst = batch ? c.inst : nullptr;
    a.acc = acc;
    a.out = out;
    a.G = p.grav_G;
    a.eps2 = p.grav_eps * p.grav_eps;
    a.err = c.d_err;
    a.counters = c.d_counters;
    (void)n;
    e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    gravity_kernel<<<c.num_sms * blocks, kGWarps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sph
