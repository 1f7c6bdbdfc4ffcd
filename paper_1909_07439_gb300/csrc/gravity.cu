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
#include "kernels.cuh"
#include "walk.cuh"

namespace sph {

constexpr int kGWarps = 4;     // warps per block
constexpr int kGStack = 256;   // node-range stack entries per warp
constexpr int kGRQ = 64;       // leaf-range queue entries per warp
constexpr int kGCell = 64;     // cell list entries per warp

// Staged cells and particles are stored in pairs, component by component
// (element 2k and 2k + 1 of the list side by side), so that a lane evaluates
// two of them against its target with the packed FP32x2 instructions.
struct GravSmem {
    int2 stk[kGStack];
    int nodes[32];
    int2 rq[kGRQ];
    float4 c0[kGCell / 2];  // (X_a, X_b, Y_a, Y_b)
    float4 c1[kGCell / 2];  // (Z_a, Z_b, M_a, M_b)
    float4 c2[kGCell / 2];  // (Qxx_a, Qxx_b, Qyy_a, Qyy_b)
    float4 c3[kGCell / 2];  // (Qzz_a, Qzz_b, Qxy_a, Qxy_b)
    float4 c4[kGCell / 2];  // (Qxz_a, Qxz_b, Qyz_a, Qyz_b)
    float4 p0[16];          // (x_a, x_b, y_a, y_b)
    float4 p1[16];          // (z_a, z_b, m_a, m_b)
    int pidx[32];           // slot of each staged particle (the target's own is skipped)
};

// element e of a pair-staged list: component c (0..1 of a float4) of slot e
__device__ __forceinline__ void put_pair(float4 *arr, int e, int c, float v)
{
    reinterpret_cast<float *>(&arr[e >> 1])[2 * c + (e & 1)] = v;
}

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
        const int t = lane >> (__ffs(L) - 1), sub = lane & (L - 1);  // L a power of two
        const bool act = t < nt;
        const int i = gr.x + (act ? t : 0);
        const float4 xt = a.pos[i];

        // Two staged entries per lane and iteration in FP32x2 (element 0 the
        // even entry, 1 the odd one), with d' = X - x_i = -d: the potential is
        // even in d, and
        //   a = d' (M / r^3 + 5/2 (d'.Q.d') / r^7) - Q d' / r^5.
        // The sums are combined (and phi negated) at the end.
        const float2 tx = f2(xt.x), ty = f2(xt.y), tz = f2(xt.z), e2 = f2(a.eps2);
        float2 ax2 = f2(0.f), ay2 = f2(0.f), az2 = f2(0.f), nphi2 = f2(0.f);  // nphi2: -phi
        auto eval_cells = [&](int nc) {
            if ((nc & 1) && lane == 0) {  // an odd list gets a massless partner far away
                put_pair(sm.c0, nc, 0, 1e18f); put_pair(sm.c0, nc, 1, 1e18f);
                put_pair(sm.c1, nc, 0, 1e18f); put_pair(sm.c1, nc, 1, 0.f);
                put_pair(sm.c2, nc, 0, 0.f); put_pair(sm.c2, nc, 1, 0.f);
                put_pair(sm.c3, nc, 0, 0.f); put_pair(sm.c3, nc, 1, 0.f);
                put_pair(sm.c4, nc, 0, 0.f); put_pair(sm.c4, nc, 1, 0.f);
            }
            __syncwarp();
            const int np2 = (nc + 1) >> 1;
#pragma unroll 2
            for (int e = sub; e < np2; e += L) {
                const float4 A = sm.c0[e], B = sm.c1[e], Q0 = sm.c2[e], Q1 = sm.c3[e], Q2 = sm.c4[e];
                const float2 dx = add2(make_float2(A.x, A.y), mul2(tx, f2(-1.f)));
                const float2 dy = add2(make_float2(A.z, A.w), mul2(ty, f2(-1.f)));
                const float2 dz = add2(make_float2(B.x, B.y), mul2(tz, f2(-1.f)));
                const float2 M = make_float2(B.z, B.w);
                const float2 qxx = make_float2(Q0.x, Q0.y), qyy = make_float2(Q0.z, Q0.w);
                const float2 qzz = make_float2(Q1.x, Q1.y), qxy = make_float2(Q1.z, Q1.w);
                const float2 qxz = make_float2(Q2.x, Q2.y), qyz = make_float2(Q2.z, Q2.w);
                const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e2)));
                const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                const float2 rinv2 = mul2(rinv, rinv), rinv3 = mul2(rinv, rinv2), rinv5 = mul2(rinv3, rinv2);
                const float2 qx = fma2(qxx, dx, fma2(qxy, dy, mul2(qxz, dz)));
                const float2 qy = fma2(qxy, dx, fma2(qyy, dy, mul2(qyz, dz)));
                const float2 qz = fma2(qxz, dx, fma2(qyz, dy, mul2(qzz, dz)));
                const float2 dqd = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
                const float2 s = fma2(M, rinv3, mul2(mul2(f2(2.5f), dqd), mul2(rinv5, rinv2)));
                const float2 nr5 = mul2(rinv5, f2(-1.f));
                ax2 = fma2(s, dx, fma2(qx, nr5, ax2));
                ay2 = fma2(s, dy, fma2(qy, nr5, ay2));
                az2 = fma2(s, dz, fma2(qz, nr5, az2));
                nphi2 = fma2(M, rinv, fma2(mul2(f2(0.5f), dqd), rinv5, nphi2));
            }
            if (act && sub == 0) n_cell += (unsigned long long)nc;
            __syncwarp();
        };
        // particles: a = m d' / r^3, phi = -m / r (the target's own slot gets m = 0)
        auto eval_parts = [&](int np) {
            if ((np & 1) && lane == 0) {
                put_pair(sm.p0, np, 0, 1e18f); put_pair(sm.p0, np, 1, 1e18f);
                put_pair(sm.p1, np, 0, 1e18f); put_pair(sm.p1, np, 1, 0.f);
                sm.pidx[np] = -1;
            }
            __syncwarp();
            const int np2 = (np + 1) >> 1;
#pragma unroll 2
            for (int e = sub; e < np2; e += L) {
                const float4 A = sm.p0[e], B = sm.p1[e];
                const int2 js = reinterpret_cast<const int2 *>(sm.pidx)[e];
                const float2 m = make_float2(js.x == i ? 0.f : B.z, js.y == i ? 0.f : B.w);
                const float2 dx = add2(make_float2(A.x, A.y), mul2(tx, f2(-1.f)));
                const float2 dy = add2(make_float2(A.z, A.w), mul2(ty, f2(-1.f)));
                const float2 dz = add2(make_float2(B.x, B.y), mul2(tz, f2(-1.f)));
                const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e2)));
                const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                const float2 mr = mul2(m, rinv);
                const float2 mr3 = mul2(mr, mul2(rinv, rinv));
                ax2 = fma2(mr3, dx, ax2);
                ay2 = fma2(mr3, dy, ay2);
                az2 = fma2(mr3, dz, az2);
                nphi2 = add2(nphi2, mr);
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
                    put_pair(sm.c0, p, 0, c.x); put_pair(sm.c0, p, 1, c.y);
                    put_pair(sm.c1, p, 0, c.z); put_pair(sm.c1, p, 1, c.w);
                    put_pair(sm.c2, p, 0, qa.x); put_pair(sm.c2, p, 1, qa.y);
                    put_pair(sm.c3, p, 0, qa.z); put_pair(sm.c3, p, 1, qb.x);
                    put_pair(sm.c4, p, 0, qb.y); put_pair(sm.c4, p, 1, qb.z);
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
                    const float4 pj = __ldg(&a.pos[myj]);
                    put_pair(sm.p0, lane, 0, pj.x); put_pair(sm.p0, lane, 1, pj.y);
                    put_pair(sm.p1, lane, 0, pj.z);
                    put_pair(sm.p1, lane, 1, pj.w);
                    sm.pidx[lane] = myj;
                }
                eval_parts(filled);
            }
        }
        if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
        float ax = ax2.x + ax2.y, ay = ay2.x + ay2.y, az = az2.x + az2.y, phi = -(nphi2.x + nphi2.y);
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
