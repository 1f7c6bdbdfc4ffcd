// Density pass (Sect. 2.2, Eqs. 1-4) with the smoothing-length solve.
//
// One warp per group of particles (up to 8 targets at a time).  The warp
// walks the tree once with a padded search radius 2 h (1 + pad) per target
// and keeps, per target, the list of candidates inside that radius in shared
// memory as (r^2, m_j, j).  The Newton iterations on
//     g(h) = sum_j m_j W(r_ij, h) - m_i (hfact / h)^3
// then run over those lists only: r_ij does not depend on h, so an iteration
// is a pure pair sum with no memory traffic.  If a target's h leaves its
// padded radius the group is walked again; if a list would overflow the
// shared-memory tile, the group falls back to walking the tree for every
// sweep ("streamed"), accumulating partial sums as the tile fills.
//
// Lane layout for the sums: L = 32 / pow2ceil(targets) lanes per target,
// lane = t * L + sub; partial sums are reduced across the L lanes with xor
// shuffles, so every lane of a target holds the full sums and takes the
// same Newton step.
#include "walk.cuh"

namespace sph {

constexpr int kTB = 8;           // targets per batch
constexpr int kDensWarps = 4;    // warps per block
constexpr float kPad = 0.05f;    // padded list radius, relative to h

template <int CAP>
struct DensSmem {
    WalkSmem w;
    float4 tp[kTB];        // target x, y, z, m
    float tr2[kTB];        // list radius^2
    int tlen[kTB];
    float2 erm[kTB][CAP];  // (r^2, m_j)
    int ej[kTB][CAP];
};

struct DensArgs {
    const float4 *pos;
    const float4 *vel;
    float *h, *rho, *omega, *drhodt;
    float4 *prop;  // h, rho, 1/(rho Omega), c_s  (for the force pass)
    const int2 *grp_ref;
    float4 *grp_lo;  // .w <- h_max of the group after the solve
    const float4 *grp_hi;
    const int *sizes;
    int *work;
    WalkTree tree;
    float hfact, tol, gamma;
    int max_iter, fixed_iters;
    int *err;
    unsigned long long *counters;
};

__device__ __forceinline__ void m4_f_df(float q, float &f, float &df)
{
    if (q < 1.f) {
        f = 1.f + q * q * (-1.5f + 0.75f * q);
        df = q * (-3.f + 2.25f * q);
    } else if (q < 2.f) {
        float t = 2.f - q;
        f = 0.25f * t * t * t;
        df = -0.75f * t * t;
    } else {
        f = 0.f;
        df = 0.f;
    }
}

__device__ __forceinline__ float seg_sum(float v, int L)
{
    for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int CAP>
__global__ void __launch_bounds__(kDensWarps * 32) density_kernel(DensArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    DensSmem<CAP> &sm = reinterpret_cast<DensSmem<CAP> *>(dsm_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int ng = a.sizes[SZ_GROUPS];
    const float hf3 = a.hfact * a.hfact * a.hfact;
    unsigned long long n_pairs = 0, n_cand = 0, n_newton = 0, n_rewalk = 0, n_stream = 0;

    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.work, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int2 gr = a.grp_ref[g];
        const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        float ghmax = 0.f;
        for (int b0 = 0; b0 < gr.y; b0 += kTB) {
            const int nt = min(kTB, gr.y - b0);
            const int L = nt > 4 ? 4 : nt > 2 ? 8 : nt > 1 ? 16 : 32;
            const int t = lane / L, sub = lane % L;
            const bool act = t < nt;
            const int i = gr.x + b0 + (act ? t : 0);
            if (lane < nt) sm.tp[lane] = a.pos[gr.x + b0 + lane];
            float h = a.h[i];
            const float mi = a.pos[i].w;
            const float M = mi * hf3;
            float hlo = 0.f, hhi = INFINITY;
            float hw = h * (1.f + kPad);  // list radius is 2 hw
            bool valid = false;           // lists cover the current h
            bool streamed = false;        // group overflowed the tile
            bool conv = !act;
            int it = 0;
            const int limit = a.fixed_iters > 0 ? a.fixed_iters : a.max_iter;
            bool final_pass = false;
            float s0, s1, s2;
            int cnt;
            __syncwarp();
            while (true) {
                // ---- one sweep: sums at the current h of every target
                s0 = 0.f; s1 = 0.f; s2 = 0.f; cnt = 0;
                const float hinv = 1.f / h;
                const float R = 2.f * h;
                const float R2 = R * R;
                const float4 ti = act ? sm.tp[t] : make_float4(0, 0, 0, 0);
                const float4 vi = (act && final_pass) ? a.vel[i] : make_float4(0, 0, 0, 0);
                auto list_sums = [&]() {
                    if (act) {
                        const int len = min(sm.tlen[t], CAP);
                        for (int e = sub; e < len; e += L) {
                            float2 rm = sm.erm[t][e];
                            if (!(rm.x < R2)) continue;
                            ++cnt;
                            float r = sqrtf(rm.x);
                            float q = r * hinv, f, df;
                            m4_f_df(q, f, df);
                            s0 += rm.y * f;
                            s1 += rm.y * (3.f * f + q * df);
                            if (final_pass && r > 0.f) {
                                int j = sm.ej[t][e];
                                float4 pj = __ldg(&a.pos[j]);
                                float4 vj = __ldg(&a.vel[j]);
                                float vr = ((vi.x - vj.x) * (ti.x - pj.x) + (vi.y - vj.y) * (ti.y - pj.y) +
                                            (vi.z - vj.z) * (ti.z - pj.z)) / r;
                                s2 += rm.y * vr * df;
                            }
                        }
                    }
                    __syncwarp();
                };
                if (!valid) {
                    // (re)build the candidate lists with a walk
                    if (lane < nt) {
                        sm.tlen[lane] = 0;
                    }
                    // radius per target: padded unless streaming
                    float myr = streamed ? R : 2.f * hw;
                    if (act && sub == 0) sm.tr2[t] = myr * myr;
                    float reach = 0.f;
                    {
                        float rr = act ? myr : 0.f;
                        for (int o = 16; o > 0; o >>= 1) rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, o));
                        reach = rr;
                    }
                    __syncwarp();
                    bool overflow = false;
                    auto chunk = [&](int j) {
                        float4 pj = j >= 0 ? __ldg(&a.pos[j]) : make_float4(0, 0, 0, 0);
                        float r2s[kTB];
                        unsigned bs[kTB];
                        bool over = false;
#pragma unroll
                        for (int tt = 0; tt < kTB; ++tt) {
                            if (tt < nt) {
                                float4 tq = sm.tp[tt];
                                r2s[tt] = canon_r2(tq.x, tq.y, tq.z, pj.x, pj.y, pj.z);
                                bs[tt] = __ballot_sync(0xffffffffu, j >= 0 && r2s[tt] < sm.tr2[tt]);
                                over |= sm.tlen[tt] + __popc(bs[tt]) > CAP;
                            }
                        }
                        // a list would overflow: sum what is there at the current h, start over
                        if (over) {
                            overflow = true;
                            list_sums();
                            if (lane < nt) sm.tlen[lane] = 0;
                            __syncwarp();
                        }
#pragma unroll
                        for (int tt = 0; tt < kTB; ++tt) {
                            if (tt < nt) {
                                int base = sm.tlen[tt];
                                if ((bs[tt] >> lane) & 1u) {
                                    int p = base + __popc(bs[tt] & lt);
                                    sm.erm[tt][p] = make_float2(r2s[tt], pj.w);
                                    sm.ej[tt][p] = j;
                                }
                                __syncwarp();
                                if (lane == 0) sm.tlen[tt] = base + __popc(bs[tt]);
                                __syncwarp();
                            }
                        }
                        n_cand += (unsigned long long)nt * 32;
                    };
                    bool ok = walk_group(a.tree, glo, ghi, reach, false, 0.f, sm.w, chunk);
                    if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
                    list_sums();
                    if (overflow) {
                        if (!streamed) ++n_stream;
                        streamed = true;
                        valid = false;
                    } else {
                        valid = !streamed;
                        if (!streamed && it > 0) ++n_rewalk;
                    }
                } else {
                    list_sums();
                }
                s0 = seg_sum(s0, L);
                s1 = seg_sum(s1, L);
                float cf = seg_sum((float)cnt, L);
                if (sub == 0 && act) n_pairs += (unsigned long long)cf;
                if (final_pass) {
                    s2 = seg_sum(s2, L);
                    break;
                }
                // ---- Newton step on g(h) (bracketed)
                if (act && !conv) {
                    float gt = kCNorm * s0 - M;          // g h^3
                    float gp = 3.f * M - kCNorm * s1;    // g' h^4
                    float hn;
                    if (gt == 0.f) {
                        hn = h;
                        conv = a.fixed_iters <= 0;
                    } else {
                        if (gt < 0.f) hlo = h; else hhi = h;
                        hn = h * (1.f - gt / gp);
                        bool ok = gp > 0.f && hn >= hlo && hn <= hhi && hn >= 0.5f * h && hn <= 2.f * h;
                        if (!ok) {
                            if (hlo > 0.f && hhi < INFINITY) hn = 0.5f * (hlo + hhi);
                            else if (gt < 0.f) hn = 2.f * h;
                            else hn = 0.5f * h;
                        }
                        double rel = fabs((double)hn - (double)h) / (double)h;
                        if (a.fixed_iters <= 0 && rel < (double)a.tol) conv = true;
                    }
                    h = hn;
                    if (sub == 0) ++n_newton;
                    if (h > hw) {  // outgrew the padded list
                        hw = h * (1.f + kPad);
                        valid = false;
                    }
                }
                ++it;
                bool need_walk = __any_sync(0xffffffffu, !valid && act);
                if (need_walk) valid = false;
                bool all_conv = __all_sync(0xffffffffu, conv);
                if (a.fixed_iters > 0 ? it >= a.fixed_iters : (all_conv || it >= limit)) {
                    if (!all_conv && a.fixed_iters <= 0 && lane == 0)
                        raise_error(a.err, SPH_ERR_NOT_CONVERGED);
                    final_pass = true;
                    // the final sweep at the accepted h needs the lists to cover h
                    if (__any_sync(0xffffffffu, act && h > hw)) valid = false;
                }
                __syncwarp();
            }
            // ---- outputs at the accepted h
            if (act && sub == 0) {
                float hinv = 1.f / h;
                float rho = M * hinv * hinv * hinv;
                float om = 1.f - kCNorm * s1 / (3.f * M);
                float F4 = kCNorm * hinv * hinv * hinv * hinv;
                a.h[i] = h;
                a.rho[i] = rho;
                a.omega[i] = om;
                a.drhodt[i] = F4 * s2 / om;
                float u = a.vel[i].w;
                float cs = sqrtf(fmaxf(a.gamma * (a.gamma - 1.f) * u, 0.f));
                a.prop[i] = make_float4(h, rho, 1.f / (rho * om), cs);
            }
            float hm = act ? h : 0.f;
            for (int o = 16; o > 0; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
            ghmax = fmaxf(ghmax, hm);
            __syncwarp();
        }
        if (lane == 0) a.grp_lo[g].w = ghmax;
    }
    // counters: one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        n_pairs += __shfl_xor_sync(0xffffffffu, n_pairs, o);
        n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
        n_newton += __shfl_xor_sync(0xffffffffu, n_newton, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_DENS_PAIRS], n_pairs);
        atomicAdd(&a.counters[C_DENS_CAND], n_cand / 32);  // n_cand counted on all lanes
        atomicAdd(&a.counters[C_NEWTON], n_newton);
        atomicAdd(&a.counters[C_REWALK], n_rewalk);
        atomicAdd(&a.counters[C_STREAMED], n_stream);
    }
}

// ------------------------------------------------------------ neighbour lists
struct NbrArgs {
    const float4 *pos;
    const float *h;
    const int2 *grp_ref;
    const float4 *grp_lo, *grp_hi;
    const int *sizes;
    int *work;
    WalkTree tree;
    int mode;          // 0 density set, 1 force set
    int64_t *off;      // [n+1]
    int32_t *idx;      // nullptr: count pass
    int *err;
};

struct NbrSmem {
    WalkSmem w;
    float4 tp[kTB];
    float th[kTB];
    int tcnt[kTB];
};

__global__ void __launch_bounds__(128) neighbour_kernel(NbrArgs a)
{
    __shared__ NbrSmem smv[4];
    NbrSmem &sm = smv[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int ng = a.sizes[SZ_GROUPS];
    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.work, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        int2 gr = a.grp_ref[g];
        float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        for (int b0 = 0; b0 < gr.y; b0 += kTB) {
            int nt = min(kTB, gr.y - b0);
            if (lane < nt) {
                sm.tp[lane] = a.pos[gr.x + b0 + lane];
                sm.th[lane] = a.h[gr.x + b0 + lane];
                sm.tcnt[lane] = 0;
            }
            __syncwarp();
            float hmx = lane < nt ? sm.th[lane] : 0.f;
            for (int o = 16; o > 0; o >>= 1) hmx = fmaxf(hmx, __shfl_xor_sync(0xffffffffu, hmx, o));
            auto chunk = [&](int j) {
                float4 pj = j >= 0 ? __ldg(&a.pos[j]) : make_float4(0, 0, 0, 0);
                float hj = j >= 0 ? __ldg(&a.h[j]) : 0.f;
                for (int tt = 0; tt < nt; ++tt) {
                    float4 tq = sm.tp[tt];
                    float ht = sm.th[tt];
                    int it = gr.x + b0 + tt;
                    float r2 = canon_r2(tq.x, tq.y, tq.z, pj.x, pj.y, pj.z);
                    float Rr = a.mode == 0 ? 2.0f * ht : 2.0f * fmaxf(ht, hj);
                    bool hit = j >= 0 && r2 < Rr * Rr && (a.mode == 0 || j != it);
                    unsigned b = __ballot_sync(0xffffffffu, hit);
                    int base = sm.tcnt[tt];
                    if (hit && a.idx) a.idx[a.off[it] + base + __popc(b & lt)] = j;
                    __syncwarp();
                    if (lane == 0) sm.tcnt[tt] = base + __popc(b);
                    __syncwarp();
                }
            };
            bool ok = walk_group(a.tree, glo, ghi, 2.f * hmx, a.mode == 1, hmx, sm.w, chunk);
            if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
            if (lane < nt && !a.idx) a.off[gr.x + b0 + lane] = sm.tcnt[lane];
            __syncwarp();
        }
    }
}

__global__ void scan_i64_kernel(int64_t *off, int n)
{
    // single block exclusive scan of counts (test-only path, not timed)
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < n; b += blockDim.x) {
        int i = b + threadIdx.x;
        int64_t v = i < n ? off[i] : 0;
        // naive block scan via shared memory
        __shared__ int64_t buf[1024];
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int64_t y = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < n) off[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

// ------------------------------------------------------------------ host side
template <int CAP>
static cudaError_t launch_density(Ctx &c, const DensArgs &a, cudaStream_t st)
{
    size_t smem = sizeof(DensSmem<CAP>) * kDensWarps;
    static bool configured = false;
    static int g_dens_blocks = 0;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(density_kernel<CAP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, density_kernel<CAP>, kDensWarps * 32, smem);
        if (e != cudaSuccess) return e;
        g_dens_blocks = nb > 0 ? nb : 1;
        configured = true;
    }
    int grid = c.num_sms * g_dens_blocks;
    density_kernel<CAP><<<grid, kDensWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t density_pass(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st)
{
    DensArgs a{};
    a.pos = (const float4 *)s.pos;
    a.vel = (const float4 *)s.vel;
    a.h = s.h;
    a.rho = s.rho;
    a.omega = s.omega;
    a.drhodt = s.drhodt;
    a.prop = c.prop;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + 3;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref};
    a.hfact = p.hfact;
    a.tol = p.h_tol;
    a.gamma = p.gamma;
    a.max_iter = p.max_h_iter;
    a.fixed_iters = p.density_iters;
    a.err = c.d_err;
    a.counters = c.d_counters;
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int cap = p.tile > 0 ? p.tile : 96;
    if (cap <= 64) return launch_density<64>(c, a, st);
    if (cap <= 96) return launch_density<96>(c, a, st);
    return launch_density<128>(c, a, st);
}

cudaError_t neighbour_lists(Ctx &c, const sph_state &s, const sph_params &p, int mode,
                            int64_t *d_off, int32_t *d_idx, int64_t cap, int64_t *h_total,
                            cudaStream_t st)
{
    (void)p;
    NbrArgs a{};
    a.pos = (const float4 *)s.pos;
    a.h = s.h;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + 3;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref};
    a.mode = mode;
    a.off = d_off;
    a.idx = nullptr;
    a.err = c.d_err;
    int grid = c.num_sms * 4;
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    neighbour_kernel<<<grid, 128, 0, st>>>(a);
    scan_i64_kernel<<<1, 1024, 0, st>>>(d_off, (int)s.n);
    e = cudaMemcpyAsync(h_total, d_off + s.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (d_idx && *h_total <= cap) {
        a.idx = d_idx;
        e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        neighbour_kernel<<<grid, 128, 0, st>>>(a);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace sph
