// Density pass (Sect. 2.2, Eqs. 1-4) with the smoothing-length solve.
//
// The h-rho relation is solved per particle with a bracketed Newton iteration
// on
//     g(h) = sum_j m_j W(r_ij, h) - m_i (hfact / h)^3
// (Sect. 3.2.1).  r_ij does not depend on h, so every sweep is a pure pair sum
// over a candidate list.
//
// density_list_kernel: one warp per batch of up to 8 targets of a group, L
// lanes per target, reading each target's neighbour list (built by
// nlist_kernel at the starting h with a (1 + pad) margin).  A batch whose h
// leaves that margin, or whose list overflowed, is handed to
// density_walk_kernel, which starts the batch over: it walks the tree with a
// padded search radius 2 h (1 + pad) per target and keeps the candidates as
// (r^2, m_j, (v_i - v_j).(x_i - x_j)) in shared memory, walking again if h
// leaves the pad and falling back to summing while walking ("streamed") if a
// list would overflow the shared-memory tile.
//
// Lane layout for the sums: L = 32 / pow2ceil(targets) lanes per target,
// lane = t * L + sub; partial sums are reduced across the L lanes with xor
// shuffles, so every lane of a target holds the full sums and takes the
// same Newton step.
#include "kernels.cuh"
#include "walk.cuh"

namespace sph {

constexpr int kTB = 8;           // targets per batch
constexpr int kDensWarps = 4;    // warps per block
constexpr float kPad = kListPad; // padded list radius, relative to h
constexpr int kRound = 2;        // groups per warp per work grab of the list kernel

template <int CAP>
struct DensSmem {
    WalkSmem w;
    float4 tp[kTB];        // target x, y, z, m
    float4 tv[kTB];        // target vx, vy, vz, u
    TargetPairs<kTB> tq;   // target coordinates in pairs for the packed distance test
    float tr2[kTB];        // list radius^2
    int tlen[kTB];
    // list entries: r^2, m_j, (v_i - v_j).(x_i - x_j)
    float er2[kTB][CAP];
    float em[kTB][CAP];
    float evd[kTB][CAP];
};

struct DensArgs {
    const float4 *pos;
    const float4 *vel;
    const float4 *rec;  // pos, vel side by side
    float *h, *rho, *omega, *drhodt;
    float4 *prop;  // h, rho, 1/(rho Omega), c_s  (for the force pass)
    const int2 *grp_ref;
    const float4 *grp_lo, *grp_hi;
    const int *sizes;
    int *work, *work2;
    WalkTree tree;
    const int *inst;  // instance of each slot (batches), or nullptr
    const int *nl_idx, *nl_len;
    int nl_stride;
    const uint8_t *active;  // only these targets are solved and written (nullptr: all)
    int2 *fallback;   // batches handed to the walking kernel
    int *n_fallback;
    int *rec_bad;     // per instance: an h outgrew the pad of the lists
    int *rec_any;     // set with rec_bad: some instance outgrew its pad
    float h_in_scale; // 1 + pad
    float hfact, tol, gamma;
    int tb;           // targets per batch of the list kernel (4, 8 or 16)
    int vd;           // 1: drho/dt here (Eq. 3); 0: the force pass of the step writes it
    int max_iter, fixed_iters;
    int *err;
    unsigned long long *counters;
};

__device__ __forceinline__ float seg_sum(float v, int L)
{
    for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of one pair at smoothing length 1/hinv (kernel K, whose f and f'
// vanish beyond its support):
//   s0 += m_j f(q), s1 += m_j (3 f + q f'), s2 += m_j vd f' / r
// (h^3 rho = C s0, -h^4 d(rho)/dh = C s1, Eq. 3 numerator x h^4 / C = s2).
template <int K, bool VD = true>
__device__ __forceinline__ void pair_sums(float r2, float mj, float vd, float hinv, float &s0,
                                          float &s1, float &s2)
{
    // r = 0 (the particle itself, or a padding entry) gives q = 0 and vd = 0
    const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
    const float q = r2 * rinv * hinv;
    float f, df;
    SphKernel<K>::f_df(q, f, df);
    s0 += mj * f;
    s1 += mj * (3.f * f + q * df);
    if (VD) s2 += mj * vd * df * rinv;
}

// One bracketed Newton update of h from the sums at h; g h^3 = C s0 - M,
// g' h^4 = 3 M - C s1 with M = m_i hfact^3.  Convergence |h_new - h| < tol h
// is decided exactly: h_new - h is exact in FP32 for h_new in [h/2, 2h] and
// the rounding error of tol h is recovered with an FMA.
__device__ __forceinline__ void newton_update(float &h, float &hlo, float &hhi, bool &conv,
                                              float s0, float s1, float M, bool fixed, float tol,
                                              float C)
{
    const float gt = C * s0 - M;
    const float gp = 3.f * M - C * s1;
    if (gt == 0.f) {
        conv = !fixed;
        return;
    }
    if (gt < 0.f) hlo = h; else hhi = h;
    float hn = h * (1.f - gt / gp);
    const bool ok = gp > 0.f && hn >= hlo && hn <= hhi && hn >= 0.5f * h && hn <= 2.f * h;
    if (!ok) {
        if (hlo > 0.f && hhi < INFINITY) hn = 0.5f * (hlo + hhi);
        else if (gt < 0.f) hn = 2.f * h;
        else hn = 0.5f * h;
    }
    const float d = fabsf(hn - h);
    const float th = tol * h;
    const float th_err = fmaf(tol, h, -th);  // tol h = th + th_err exactly
    if (!fixed && (d < th || (d == th && th_err > 0.f))) conv = true;  // sums are at this h
    else h = hn;
}

// outputs at the accepted h (Eqs. 1-4) and the force pass's per-particle terms
// (drho/dt only with vd: otherwise the force pass of the step writes it)
__device__ __forceinline__ void density_outputs(const DensArgs &a, int i, float h, float M, float s1,
                                                float s2, float u, float C, bool vd = true)
{
    const float hinv = 1.f / h;
    const float rho = M * hinv * hinv * hinv;
    const float om = 1.f - C * s1 / (3.f * M);
    const float F4 = C * hinv * hinv * hinv * hinv;
    a.h[i] = h;
    a.rho[i] = rho;
    a.omega[i] = om;
    if (vd) a.drhodt[i] = F4 * s2 / om;
    const float cs = sqrtf(fmaxf(a.gamma * (a.gamma - 1.f) * u, 0.f));
    a.prop[i] = make_float4(h, rho, 1.f / (rho * om), cs);
}

__device__ __forceinline__ void push_fallback(const DensArgs &a, int g, int b0, int nt)
{
    if ((threadIdx.x & 31) == 0) push_fallback_batch(a.fallback, a.n_fallback, g, b0, nt);
}

// Launch shape (run-time): a.tb targets per batch (32 / a.tb lanes per
// target), blockDim.x / 32 warps per block; NPER list entries per lane and
// iteration; registers capped for 1024 resident threads per SM.  VD: the
// sums of drho/dt too, over 32-byte records (position, velocity); without,
// the neighbours' 16-byte positions alone are gathered.
template <int NPER, int K, bool PER, bool VD>
__global__ void __launch_bounds__(256, 4) density_list_kernel(DensArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t keep = l2_keep_policy();
    const int ng = a.sizes[SZ_GROUPS];
    const float hf3 = a.hfact * a.hfact * a.hfact;
    const bool fixed = a.fixed_iters > 0;
    const int limit = fixed ? a.fixed_iters : a.max_iter;
    unsigned long long n_pairs = 0, n_newton = 0;
    // The block takes kRound consecutive groups per warp at a time, warp w the
    // groups base + w + nw k: the warps of a block work on neighbouring groups
    // together and share their candidates in L1.
    __shared__ int s_base;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

    while (true) {
        if (threadIdx.x == 0) s_base = atomicAdd(a.work, nw * kRound);
        __syncthreads();
        const int base = s_base;
        __syncthreads();
        if (base >= ng) break;
        for (int kr = 0; kr < kRound; ++kr) {
            const int gq = base + warp + nw * kr;
            if (gq >= ng) break;
            const int g = ng - 1 - gq;  // last group first: its lists were written last (in L2)
            const int2 gr = a.grp_ref[g];
            for (int b0 = 0; b0 < gr.y; b0 += a.tb) {
                const int nt = min(a.tb, gr.y - b0);
                const int L = lanes_per_target(nt);
                const int t = lane >> (__ffs(L) - 1), sub = lane & (L - 1);  // L a power of two
                const bool act = t < nt;
                const int i = gr.x + b0 + (act ? t : 0);
                const bool on = act && (!a.active || a.active[i]);
                if (!__any_sync(0xffffffffu, on)) continue;  // no target of the batch is due
                const int len = act ? a.nl_len[i] : 0;
                if (__any_sync(0xffffffffu, len < 0)) {  // no list (overflow, or too many leaves)
                    push_fallback(a, g, b0, nt);
                    continue;
                }
                const int *__restrict__ lst = a.nl_idx + (size_t)i * a.nl_stride;
                const float4 xi = a.pos[i], vi = a.vel[i];
                float h = a.h[i];
                const float hw = h * a.h_in_scale;  // the lists hold every pair with r < R hw
                const float M = xi.w * hf3;
                float hlo = 0.f, hhi = INFINITY;
                bool conv = !on, outside = false, final_pass = false;
                int it = 0;
                float s0, s1, s2;
                while (true) {
                    s0 = 0.f; s1 = 0.f; s2 = 0.f;
                    int cnt = 0;
                    const float hinv = 1.f / h;
                    const float R = SphKernel<K>::R * h;
                    const float R2 = R * R;
                    // NPER consecutive entries per lane and iteration (one 8- or
                    // 16-byte load of the list, fetched an iteration ahead: the
                    // lists come from DRAM), no branch on the distance: f and f'
                    // vanish for q >= R, so entries beyond R h add nothing.  A
                    // missing entry repeats the first with zero mass.
                    auto entry = [&](float4 pj, float4 vj, float mj) {
                        float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
                        if (PER) {  // nearest images on the periodic axes
                            dx = wrap_sep(dx, a.tree.per.x);
                            dy = wrap_sep(dy, a.tree.per.y);
                            dz = wrap_sep(dz, a.tree.per.z);
                        }
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const float vd =
                            VD ? (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz : 0.f;
                        cnt += (mj > 0.f && r2 < R2) ? 1 : 0;
                        pair_sums<K, VD>(r2, mj, vd, hinv, s0, s1, s2);
                    };
                    // neighbour j's position (and velocity with VD)
                    auto load = [&](int j, float4 &pj, float4 &vj) {
                        if (VD) {
                            ld_rec(a.rec, j, keep, pj, vj);
                        } else {
                            pj = ld_keep(a.pos, j, keep);
                            vj = make_float4(0.f, 0.f, 0.f, 0.f);  // not read without VD
                        }
                    };
                    if (NPER == 4) {
                        int e = 4 * sub;
                        int4 jn = e < len ? __ldcs(reinterpret_cast<const int4 *>(lst + e)) : make_int4(0, 0, 0, 0);
                        for (; e < len; e += 4 * L) {
                            const int4 jj = jn;
                            if (e + 4 * L < len) jn = __ldcs(reinterpret_cast<const int4 *>(lst + e + 4 * L));
                            const bool b1 = e + 1 < len, b2 = e + 2 < len, b3 = e + 3 < len;
                            float4 p0, v0, p1, v1, p2, v2, p3, v3;
                            load(jj.x, p0, v0);
                            load(b1 ? jj.y : jj.x, p1, v1);
                            load(b2 ? jj.z : jj.x, p2, v2);
                            load(b3 ? jj.w : jj.x, p3, v3);
                            entry(p0, v0, p0.w);
                            entry(p1, v1, b1 ? p1.w : 0.f);
                            entry(p2, v2, b2 ? p2.w : 0.f);
                            entry(p3, v3, b3 ? p3.w : 0.f);
                        }
                    } else {
                        int e = 2 * sub;
                        int2 jn = e < len ? __ldcs(reinterpret_cast<const int2 *>(lst + e)) : make_int2(0, 0);
                        for (; e < len; e += 2 * L) {
                            const int2 jj = jn;
                            if (e + 2 * L < len) jn = __ldcs(reinterpret_cast<const int2 *>(lst + e + 2 * L));
                            const bool b1 = e + 1 < len;
                            float4 p0, v0, p1, v1;
                            load(jj.x, p0, v0);
                            load(b1 ? jj.y : jj.x, p1, v1);
                            entry(p0, v0, p0.w);
                            entry(p1, v1, b1 ? p1.w : 0.f);
                        }
                    }
                    s0 = seg_sum(s0, L);
                    s1 = seg_sum(s1, L);
                    s2 = seg_sum(s2, L);
                    const float cf = seg_sum((float)cnt, L);
                    if (sub == 0 && on) {
                        n_pairs += (unsigned long long)cf;
                        ++n_newton;
                    }
                    if (final_pass) break;
                    if (on && !conv) {
                        newton_update(h, hlo, hhi, conv, s0, s1, M, fixed, a.tol, SphKernel<K>::C);
                        outside = h > hw;
                    }
                    ++it;
                    if (__any_sync(0xffffffffu, outside)) break;  // the lists no longer cover h
                    if (fixed) {
                        if (it >= limit) final_pass = true;   // one more sweep at the last h
                    } else if (__all_sync(0xffffffffu, conv)) {
                        break;                                // every target's sums are at its h
                    } else if (it >= limit) {
                        if (lane == 0) raise_error(a.err, SPH_ERR_NOT_CONVERGED);
                        final_pass = true;
                    }
                }
                if (__any_sync(0xffffffffu, outside)) {  // start the batch over with walks
                    push_fallback(a, g, b0, nt);
                    continue;
                }
                if (on && sub == 0) density_outputs(a, i, h, M, s1, s2, vi.w, SphKernel<K>::C, VD);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_pairs += __shfl_xor_sync(0xffffffffu, n_pairs, o);
        n_newton += __shfl_xor_sync(0xffffffffu, n_newton, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_DENS_PAIRS], n_pairs);
        atomicAdd(&a.counters[C_NEWTON], n_newton);
    }
}

// Batches the list kernel handed over, each solved from its starting h with
// tree walks.
template <int CAP, int K>
__global__ void __launch_bounds__(kDensWarps * 32) density_walk_kernel(DensArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    DensSmem<CAP> &sm = reinterpret_cast<DensSmem<CAP> *>(dsm_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int nfb = *a.n_fallback;
    if (nfb == 0) return;  // nothing handed over (the usual case): no atomics
    const float hf3 = a.hfact * a.hfact * a.hfact;
    const bool fixed = a.fixed_iters > 0;
    const int limit = fixed ? a.fixed_iters : a.max_iter;
    unsigned long long n_pairs = 0, n_cand = 0, n_newton = 0, n_rewalk = 0, n_stream = 0;

    while (true) {
        int k = 0;
        if (lane == 0) k = atomicAdd(a.work2, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nfb) break;
        const int2 fb = a.fallback[k];
        const int g = fb.x, b0 = fb.y & 0xffff, cnt = fb.y >> 16;  // cnt <= kTB
        const int2 gr = a.grp_ref[g];
        const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        const int root = a.inst ? a.inst[gr.x] : 0;
        ++n_rewalk;
        {
            const int nt = min(cnt, gr.y - b0);
            const int L = lanes_per_target(nt);
            const int t = lane >> (__ffs(L) - 1), sub = lane & (L - 1);  // L a power of two
            const bool act = t < nt;
            const int i = gr.x + b0 + (act ? t : 0);
            const bool on = act && (!a.active || a.active[i]);
            if (lane < kTB) {
                const float4 p = lane < nt ? a.pos[gr.x + b0 + lane] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                sm.tp[lane] = p;
                sm.tq.set(lane, p);
                if (lane < nt) sm.tv[lane] = a.vel[gr.x + b0 + lane];
            }
            __syncwarp();
            float h = a.h[i];
            const float h_in = h;
            const float M = sm.tp[act ? t : 0].w * hf3;  // m_i hfact^3
            float hlo = 0.f, hhi = INFINITY;
            float hw = h * (1.f + kPad);  // list radius is R hw
            bool valid = false;           // lists cover the current h
            bool streamed = false;        // batch overflowed the tile
            bool conv = !on;
            bool final_pass = false;
            int it = 0;
            float s0, s1, s2;
            while (true) {
                // ---- one sweep: sums at the current h of every target
                s0 = 0.f; s1 = 0.f; s2 = 0.f;
                int cnt = 0;
                const float hinv = 1.f / h;
                const float R = SphKernel<K>::R * h;
                const float R2 = R * R;
                auto list_sums = [&]() {
                    if (act) {
                        const int len = sm.tlen[t];
                        for (int e = sub; e < len; e += L) {
                            const float r2 = sm.er2[t][e];
                            if (!(r2 < R2)) continue;
                            ++cnt;
                            pair_sums<K>(r2, sm.em[t][e], sm.evd[t][e], hinv, s0, s1, s2);
                        }
                    }
                    __syncwarp();
                };
                if (!valid) {
                    // (re)build the candidate lists with a walk
                    const float myr = streamed ? R : SphKernel<K>::R * hw;  // padded unless streaming
                    if (act && sub == 0) sm.tr2[t] = myr * myr;
                    if (lane < kTB) sm.tlen[lane] = 0;
                    float reach = act ? myr : 0.f;
                    for (int o = 16; o > 0; o >>= 1) reach = fmaxf(reach, __shfl_xor_sync(0xffffffffu, reach, o));
                    __syncwarp();
                    bool overflow = false;
                    auto chunk = [&](int j) {
                        const float4 pj = j >= 0 ? __ldg(&a.pos[j]) : make_float4(0, 0, 0, 0);
                        const float4 vj = j >= 0 ? __ldg(&a.vel[j]) : make_float4(0, 0, 0, 0);
                        unsigned bs[kTB];
                        float r2s[kTB];
                        int base[kTB];
                        bool over = false;
#pragma unroll
                        for (int q = 0; q < kTB / 2; ++q) {
                            const int t0 = 2 * q, t1 = 2 * q + 1;
                            bs[t0] = bs[t1] = 0u;
                            base[t0] = base[t1] = 0;
                            r2s[t0] = r2s[t1] = 0.f;
                            if (t0 < nt) {
                                const float2 r2 = canon_r2_x2p(sm.tq.x[q], sm.tq.y[q], sm.tq.z[q], pj.x,
                                                               pj.y, pj.z, a.tree.per);
                                r2s[t0] = r2.x;
                                r2s[t1] = r2.y;
                                bs[t0] = __ballot_sync(0xffffffffu, j >= 0 && r2.x < sm.tr2[t0]);
                                bs[t1] = __ballot_sync(0xffffffffu, j >= 0 && t1 < nt && r2.y < sm.tr2[t1]);
                                base[t0] = sm.tlen[t0];
                                base[t1] = sm.tlen[t1];
                                over |= base[t0] + __popc(bs[t0]) > CAP;
                                over |= base[t1] + __popc(bs[t1]) > CAP;
                            }
                        }
                        if (over) {
                            // a list would overflow: sum what is there at the current h, start over
                            overflow = true;
                            list_sums();
                            if (lane < nt) sm.tlen[lane] = 0;
                            __syncwarp();
#pragma unroll
                            for (int tt = 0; tt < kTB; ++tt) base[tt] = 0;
                        }
#pragma unroll
                        for (int tt = 0; tt < kTB; ++tt) {
                            if (tt < nt) {
                                if ((bs[tt] >> lane) & 1u) {
                                    const float4 tq = sm.tp[tt], tv = sm.tv[tt];
                                    const float vdot = (tv.x - vj.x) * wrap_sep(tq.x - pj.x, a.tree.per.x) +
                                                       (tv.y - vj.y) * wrap_sep(tq.y - pj.y, a.tree.per.y) +
                                                       (tv.z - vj.z) * wrap_sep(tq.z - pj.z, a.tree.per.z);
                                    const int pe = base[tt] + __popc(bs[tt] & lt);
                                    sm.er2[tt][pe] = r2s[tt];
                                    sm.em[tt][pe] = pj.w;
                                    sm.evd[tt][pe] = vdot;
                                }
                                if (lane == tt) sm.tlen[tt] = base[tt] + __popc(bs[tt]);
                            }
                        }
                        __syncwarp();
                        n_cand += (unsigned long long)nt;
                    };
                    bool ok = walk_group(a.tree, root, glo, ghi, reach, false, 0.f, sm.w, chunk);
                    if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
                    list_sums();
                    if (overflow) {
                        if (!streamed) ++n_stream;
                        streamed = true;
                        valid = false;
                    } else {
                        valid = !streamed;
                    }
                } else {
                    list_sums();
                }
                s0 = seg_sum(s0, L);
                s1 = seg_sum(s1, L);
                s2 = seg_sum(s2, L);
                const float cf = seg_sum((float)cnt, L);
                if (sub == 0 && on) {
                    n_pairs += (unsigned long long)cf;
                    ++n_newton;
                }
                if (final_pass) break;
                if (on && !conv) {
                    newton_update(h, hlo, hhi, conv, s0, s1, M, fixed, a.tol, SphKernel<K>::C);
                    if (h > hw) {  // outgrew the padded list
                        hw = h * (1.f + kPad);
                        valid = false;
                    }
                }
                ++it;
                if (__any_sync(0xffffffffu, !valid)) valid = false;
                if (fixed) {
                    if (it >= limit) final_pass = true;   // one more sweep at the last h
                } else if (__all_sync(0xffffffffu, conv)) {
                    break;                                // every target's sums are at its h
                } else if (it >= limit) {
                    if (lane == 0) raise_error(a.err, SPH_ERR_NOT_CONVERGED);
                    final_pass = true;
                }
                __syncwarp();
            }
            if (on && sub == 0) density_outputs(a, i, h, M, s1, s2, sm.tv[t].w, SphKernel<K>::C);
            // the neighbour lists hold while no h grew beyond their pad
            if (__any_sync(0xffffffffu, on && h > a.h_in_scale * h_in) && lane == 0) {
                atomicOr(a.rec_bad + root, 1);  // root = this group's instance
                atomicOr(a.rec_any, 1);
            }
            __syncwarp();
        }
    }
    // counters: one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        n_pairs += __shfl_xor_sync(0xffffffffu, n_pairs, o);
        n_newton += __shfl_xor_sync(0xffffffffu, n_newton, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_DENS_PAIRS], n_pairs);
        atomicAdd(&a.counters[C_DENS_CAND], n_cand * 32);
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
    const int *inst;
    int mode;          // 0 density set, 1 force set
    float kr;          // support radius in units of h
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
                    float r2 = canon_r2p(tq.x, tq.y, tq.z, pj.x, pj.y, pj.z, a.tree.per);
                    float Rr = a.mode == 0 ? a.kr * ht : a.kr * fmaxf(ht, hj);
                    bool hit = j >= 0 && r2 < Rr * Rr && (a.mode == 0 || j != it);
                    unsigned b = __ballot_sync(0xffffffffu, hit);
                    int base = sm.tcnt[tt];
                    if (hit && a.idx) a.idx[a.off[it] + base + __popc(b & lt)] = j;
                    __syncwarp();
                    if (lane == 0) sm.tcnt[tt] = base + __popc(b);
                    __syncwarp();
                }
            };
            bool ok = walk_group(a.tree, a.inst ? a.inst[gr.x] : 0, glo, ghi, a.kr * hmx, a.mode == 1,
                                 0.5f * a.kr * hmx, sm.w, chunk, 0.5f * a.kr);
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

// Test export: the density (mode 0) or force (mode 1) set of every particle
// taken from its neighbour list with the canonical FP32 test, one thread per
// particle.  out == nullptr: row counts into off[i] (and particles without a
// list into *missing); otherwise the rows are written at off[i].
__global__ void list_set_kernel(const float4 *__restrict__ pos, const float *__restrict__ h,
                                const int *__restrict__ idx, const int *__restrict__ len, int n,
                                int stride, int mode, float kr, Period per, int64_t *off,
                                int32_t *out, int *missing)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = len[i];
        if (l < 0) {
            if (!out) {
                off[i] = 0;
                atomicAdd(missing, 1);
            }
            continue;
        }
        const float4 pi = pos[i];
        const float hi = h[i];
        int64_t w = out ? off[i] : 0;
        int cnt = 0;
        for (int e = 0; e < l; ++e) {
            const int j = idx[(size_t)i * stride + e];
            const float4 pj = pos[j];
            const float r2 = canon_r2p(pi.x, pi.y, pi.z, pj.x, pj.y, pj.z, per);
            const float R = mode == 0 ? kr * hi : kr * fmaxf(hi, h[j]);
            if (r2 < R * R && (mode == 0 || j != i)) {
                if (out) out[w++] = j;
                ++cnt;
            }
        }
        if (!out) off[i] = cnt;
    }
}

// ------------------------------------------------------------------ host side
// one-time kernel attributes and occupancy (also called before graph capture)
template <int CAP, int K>
static cudaError_t configure_density(int &blocks)
{
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int nb_cached = 1;
    if (!configured) {
        size_t smem = sizeof(DensSmem<CAP>) * kDensWarps;
        cudaError_t e = cudaFuncSetAttribute(density_walk_kernel<CAP, K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, density_walk_kernel<CAP, K>,
                                                          kDensWarps * 32, smem);
        if (e != cudaSuccess) return e;
        nb_cached = nb > 0 ? nb : 1;
        configured = true;
    }
    blocks = nb_cached;
    return cudaSuccess;
}

// resident blocks per SM of the list kernel for 1, 2, 4 and 8 warps per block
// (the smallest over its variants)
template <int K>
static cudaError_t configure_density_list(int blocks[4])
{
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int nb_cached[4];
    if (!configured) {
        const void *fns[8] = {(const void *)density_list_kernel<2, K, false, true>,
                              (const void *)density_list_kernel<2, K, true, true>,
                              (const void *)density_list_kernel<4, K, false, true>,
                              (const void *)density_list_kernel<4, K, true, true>,
                              (const void *)density_list_kernel<2, K, false, false>,
                              (const void *)density_list_kernel<2, K, true, false>,
                              (const void *)density_list_kernel<4, K, false, false>,
                              (const void *)density_list_kernel<4, K, true, false>};
        for (int w = 0; w < 4; ++w) {
            int nb = 1 << 30;
            for (const void *f : fns) {
                int b = 0;
                cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, 32 << w, 0);
                if (e != cudaSuccess) return e;
                nb = b < nb ? b : nb;
            }
            nb_cached[w] = nb > 0 ? nb : 1;
        }
        configured = true;
    }
    for (int w = 0; w < 4; ++w) blocks[w] = nb_cached[w];
    return cudaSuccess;
}

template <int CAP, int K>
static cudaError_t launch_density_walk(Ctx &c, const DensArgs &a, cudaStream_t st)
{
    int blocks = 1;
    cudaError_t e = configure_density<CAP, K>(blocks);
    if (e != cudaSuccess) return e;
    size_t smem = sizeof(DensSmem<CAP>) * kDensWarps;
    density_walk_kernel<CAP, K><<<c.num_sms * blocks, kDensWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int K>
static cudaError_t configure_density_k()
{
    int b, bl[4];
    cudaError_t e = configure_density_list<K>(bl);
    if (e == cudaSuccess) e = configure_density<64, K>(b);
    if (e == cudaSuccess) e = configure_density<80, K>(b);
    if (e == cudaSuccess) e = configure_density<96, K>(b);
    if (e == cudaSuccess) e = configure_density<128, K>(b);
    return e;
}

cudaError_t configure_density_kernels(int kernel)
{
    return kernel == 1 ? configure_density_k<1>() : kernel == 2 ? configure_density_k<2>()
                                                                : configure_density_k<0>();
}

// the list kernel, then the walking kernel for the batches it handed over
template <int K>
static cudaError_t density_solve_k(Ctx &c, DensArgs &a, const sph_params &p, cudaStream_t st)
{
    int bl[4];
    cudaError_t e = configure_density_list<K>(bl);
    if (e != cudaSuccess) return e;
    const PairShape ps = pair_shape(p);
    a.tb = ps.targets;
    const int wl = ps.warps == 8 ? 3 : ps.warps == 4 ? 2 : ps.warps == 2 ? 1 : 0;
    const dim3 grid(c.num_sms * bl[wl]), block(32 * ps.warps);
    const bool per = a.tree.per.any();
    if (a.vd) {
        if (ps.unroll == 4 && per) density_list_kernel<4, K, true, true><<<grid, block, 0, st>>>(a);
        else if (ps.unroll == 4) density_list_kernel<4, K, false, true><<<grid, block, 0, st>>>(a);
        else if (per) density_list_kernel<2, K, true, true><<<grid, block, 0, st>>>(a);
        else density_list_kernel<2, K, false, true><<<grid, block, 0, st>>>(a);
    } else {
        if (ps.unroll == 4 && per) density_list_kernel<4, K, true, false><<<grid, block, 0, st>>>(a);
        else if (ps.unroll == 4) density_list_kernel<4, K, false, false><<<grid, block, 0, st>>>(a);
        else if (per) density_list_kernel<2, K, true, false><<<grid, block, 0, st>>>(a);
        else density_list_kernel<2, K, false, false><<<grid, block, 0, st>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // default tile: the mean density set (about 58 for M4 at hfact 1.2, 82 for
    // M6 at 0.9, 74 for Wendland C6 at 1.3) with room to spare
    int cap = p.tile > 0 ? p.tile : K == 0 ? 80 : 128;
    if (cap <= 64) return launch_density_walk<64, K>(c, a, st);
    if (cap <= 80) return launch_density_walk<80, K>(c, a, st);
    if (cap <= 96) return launch_density_walk<96, K>(c, a, st);
    return launch_density_walk<128, K>(c, a, st);
}

cudaError_t density_lists(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                          const Batch *batch, bool refresh_hmax)
{
    cudaError_t e = cudaSuccess;
    // node and group h_max of the starting h: the list walk's opening test needs them
    if (refresh_hmax) e = update_hmax(c, s, p, st);
    if (e != cudaSuccess) return e;
    // fresh lists: valid unless an h outgrows its pad
    e = cudaMemsetAsync(c.tree.rec_ctl, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c.tree.rec_bad, 0, sizeof(int) * (batch ? batch->n_inst : 1), st);
    if (e != cudaSuccess) return e;
    c.nl_kernel = p.kernel;
    c.nl_stride = list_cap(p.kernel);
    return nlist_pass(c, s, p, kPad, st, batch);
}

cudaError_t density_solve(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                          const Batch *batch)
{
    DensArgs a{};
    a.inst = batch ? c.inst : nullptr;
    a.h_in_scale = 1.f + kPad;
    a.nl_idx = c.nl_idx;
    a.nl_len = c.nl_len;
    a.nl_stride = c.nl_stride;
    a.active = c.mask;
    a.fallback = c.fallback;
    a.n_fallback = c.d_sizes + SZ_FALLBACK;
    a.rec_bad = c.tree.rec_bad;
    a.rec_any = c.tree.rec_ctl;
    a.pos = (const float4 *)s.pos;
    a.vel = (const float4 *)s.vel;
    a.rec = c.rec;
    a.vd = c.drhodt_in_force ? 0 : 1;
    a.h = s.h;
    a.rho = s.rho;
    a.omega = s.omega;
    a.drhodt = s.drhodt;
    a.prop = c.prop;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.work2 = c.d_sizes + SZ_WORK2;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref, period_of(p)};
    a.hfact = p.hfact;
    a.tol = p.h_tol;
    a.gamma = p.gamma;
    a.max_iter = p.max_h_iter;
    a.fixed_iters = p.density_iters;
    a.err = c.d_err;
    a.counters = c.d_counters;
    static_assert(SZ_FALLBACK == SZ_WORK + 1 && SZ_WORK2 == SZ_WORK + 2, "work counters adjacent");
    cudaError_t e = cudaMemsetAsync(a.work, 0, 3 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (p.kernel == 1) return density_solve_k<1>(c, a, p, st);
    if (p.kernel == 2) return density_solve_k<2>(c, a, p, st);
    return density_solve_k<0>(c, a, p, st);
}

cudaError_t density_pass(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                         const Batch *batch)
{
    cudaError_t e = density_lists(c, s, p, st, batch, false);
    if (e != cudaSuccess) return e;
    return density_solve(c, s, p, st, batch);
}

cudaError_t list_sets(Ctx &c, const sph_state &s, const sph_params &p, int mode, int64_t *d_off,
                      int32_t *d_idx, int64_t cap, int64_t *h_total, int *h_missing,
                      cudaStream_t st)
{
    // the production lists at the current h: node and group h_max refreshed,
    // then the list-building kernel of the density pass
    cudaError_t e = density_lists(c, s, p, st, nullptr, true);
    if (e != cudaSuccess) return e;
    const int n = (int)s.n;
    int *missing = c.d_sizes + SZ_WORK2;
    e = cudaMemsetAsync(missing, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int grid = c.num_sms * 8;
    const float kr = kernel_support(p.kernel);
    list_set_kernel<<<grid, 256, 0, st>>>((const float4 *)s.pos, s.h, c.nl_idx, c.nl_len, n,
                                          c.nl_stride, mode, kr, period_of(p),
                                          d_off, nullptr, missing);
    scan_i64_kernel<<<1, 1024, 0, st>>>(d_off, n);
    e = cudaMemcpyAsync(h_total, d_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.h_pinned + 4, missing, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *h_missing = c.h_pinned[4];
    if (d_idx && *h_total <= cap) {
        list_set_kernel<<<grid, 256, 0, st>>>((const float4 *)s.pos, s.h, c.nl_idx, c.nl_len, n,
                                              c.nl_stride, mode,
                                              kr, period_of(p), d_off, d_idx, missing);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t neighbour_lists(Ctx &c, const sph_state &s, const sph_params &p, int mode,
                            int64_t *d_off, int32_t *d_idx, int64_t cap, int64_t *h_total,
                            cudaStream_t st)
{
    NbrArgs a{};
    a.kr = kernel_support(p.kernel);
    a.pos = (const float4 *)s.pos;
    a.h = s.h;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref, period_of(p)};
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
