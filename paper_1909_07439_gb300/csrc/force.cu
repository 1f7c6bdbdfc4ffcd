// Hydro force pass (Sect. 2.4-2.6, Eqs. 9-15), no gravity.
//
// The pair set of a particle is every j with r_ij < R max(h_i, h_j), R the
// support radius of the kernel in units of h: a pair is found whenever either
// particle reaches the other (Sect. 3.2).  The pair kernels are templates on
// the smoothing kernel K (SphKernel<K>).
//
// force_list_kernel: one warp per batch of up to 8 targets of a group, L
// lanes per target, reading each target's neighbour list from the density
// pass (a superset of the pair set while no h outgrew the list pad) and
// applying the exact test with the canonical FP32 distance.  Batches whose
// lists are unusable (overflowed, stale, or an h of the instance outgrew the
// pad) go to force_walk_kernel, which walks the tree: it opens a node if its
// box is within R max(h_max(group), h_max(node)) of the group box, tests
// each candidate chunk against every target and compacts the hits with
// ballots into per-target lists in shared memory; the pair arithmetic then
// runs over those lists with L lanes per target, flushing whenever a list
// could overflow.
#include "kernels.cuh"
#include "walk.cuh"

namespace sph {

constexpr int kFTB = 8;          // targets per batch
constexpr int kForceWarps = 4;   // warps per block
constexpr int kRound = 2;        // groups per warp per work grab of the list kernel

template <int CAP>
struct ForceSmem {
    WalkSmem w;
    float4 tp[kFTB];   // x, y, z, m
    float4 tv[kFTB];   // vx, vy, vz, u
    float4 tq[kFTB];   // h, rho, 1/(rho Omega), c
    TargetPairs<kFTB> tc;  // target coordinates in pairs for the packed distance test
    float th[kFTB];    // target h (0 for unused slots)
    int tlen[kFTB];
    int ej[kFTB][CAP];
};

struct ForceArgs {
    const float4 *pos, *vel, *prop;
    const float4 *frec;  // [3 n] force records of the list kernel
    int tb;              // targets per batch of the list kernel (4, 8 or 16)
    float4 *acc;
    float *vsigmax;
    float *drhodt;  // written too (Eq. 3, the pressure-work sum over m_j F_i), or nullptr
    const int2 *grp_ref;
    const float4 *grp_lo, *grp_hi;
    const int *sizes;
    int *work, *work2;
    WalkTree tree;
    const int *inst;  // instance of each slot (batches), or nullptr
    const int *nl_idx, *nl_len;
    int nl_stride;
    const uint8_t *active;  // only these targets are computed and written (nullptr: all)
    const int *rec_ctl, *rec_bad;
    int2 *fallback;
    int *n_fallback;
    float gm1, alpha, beta, alpha_u;
    int *err;
    unsigned long long *counters;
};

// Per-target state of the pair sums: the target's constants and the
// accumulated acceleration (Eq. 9 with Eq. 13), the three du/dt terms
// (Eqs. 10, 14, 15) and the signal-velocity maximum (Eq. 12).
template <int K>
struct ForceTarget {
    float4 xi, vi, qi;  // x, m / v, u / h, rho, A = 1/(rho Omega), c
    float hinv_i, cf_i, Pi, pres_i;
    float ax, ay, az, dup, duav, duc, vsmax;
    int cnt;

    __device__ __forceinline__ void init(float4 x, float4 v, float4 q, const ForceArgs &a)
    {
        xi = x; vi = v; qi = q;
        hinv_i = 1.f / qi.x;
        cf_i = SphKernel<K>::C * hinv_i * hinv_i * hinv_i * hinv_i;  // F_i = f'(q_i) C / h_i^4
        pres_i = a.gm1 * vi.w;  // P_i / rho_i
        Pi = pres_i * qi.y;      // formed as P_j is
        ax = ay = az = dup = duav = duc = 0.f;
        vsmax = a.alpha * qi.w;
        cnt = 0;
    }

    // One pair.  `in` = j is in the pair set; all other contributions scale
    // with mj, which callers set to 0 for a padding entry.  Square roots and
    // quotients use the hardware approximations (a few ulp), the pair-set
    // decision is made by the caller with the canonical distance.
    __device__ __forceinline__ void pair(float4 pj, float4 vj, float4 qj, float mj, bool in,
                                         const ForceArgs &a)
    {
        // nearest images on the periodic axes (open axes: unchanged)
        const float dx = wrap_sep(xi.x - pj.x, a.tree.per.x), dy = wrap_sep(xi.y - pj.y, a.tree.per.y),
                    dz = wrap_sep(xi.z - pj.z, a.tree.per.z);
        pair_d(dx, dy, dz, dx * dx + dy * dy + dz * dz, vj, qj, mj, in, a);
    }

    // the same with the separation x_i - x_j and its squared length given
    __device__ __forceinline__ void pair_d(float dx, float dy, float dz, float r2, float4 vj, float4 qj,
                                           float mj, bool in, const ForceArgs &a)
    {
        const float Ai = qi.z, ci = qi.w;
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float r = r2 * rinv;
        const float hinv_j = __fdividef(1.f, qj.x);
        const float hinv2_j = hinv_j * hinv_j;
        const float Fi = SphKernel<K>::df(r * hinv_i) * cf_i;
        const float Fj = SphKernel<K>::C * SphKernel<K>::df(r * hinv_j) * hinv2_j * hinv2_j;
        const float vr = ((vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz) * rinv;
        const float avr = fabsf(vr);
        const float vsi = a.alpha * ci + a.beta * avr;
        const float mu = vr < 0.f ? -0.5f * vr : 0.f;  // viscosity acts on approaching pairs
        const float avi = mu * vsi;
        const float avj = mu * (a.alpha * qj.w + a.beta * avr);
        duav += mj * vsi * vr * (-2.f * mu) * Fi;
        const float Aj = qj.z;
        const float pres_j = a.gm1 * vj.w;  // P_j / rho_j
        const float coef = mj * (Ai * (pres_i + avi) * Fi + Aj * (pres_j + avj) * Fj);
        const float cr = coef * rinv;
        ax -= cr * dx;
        ay -= cr * dy;
        az -= cr * dz;
        dup += mj * vr * Fi;
        const float Pj = pres_j * qj.y;
        const float x = __fdividef(2.f * fabsf(Pi - Pj), qi.y + qj.y);
        const float vsu = x > 0.f ? x * rsqrtf(x) : 0.f;
        duc += mj * vsu * (vi.w - vj.w) * (Fi * Ai + Fj * Aj);
        vsmax = in ? fmaxf(vsmax, vsi) : vsmax;
        cnt += in ? 1 : 0;
    }

    // reduce over the L lanes of each target; lane sub == 0 writes
    __device__ __forceinline__ void finish(int L, bool write, int i, const ForceArgs &a)
    {
        for (int o = L >> 1; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            az += __shfl_xor_sync(0xffffffffu, az, o);
            dup += __shfl_xor_sync(0xffffffffu, dup, o);
            duav += __shfl_xor_sync(0xffffffffu, duav, o);
            duc += __shfl_xor_sync(0xffffffffu, duc, o);
            vsmax = fmaxf(vsmax, __shfl_xor_sync(0xffffffffu, vsmax, o));
        }
        if (write) {
            const float Ai = qi.z;
            const float du = pres_i * Ai * dup - 0.5f * Ai * duav + 0.5f * a.alpha_u * duc;
            a.acc[i] = make_float4(ax, ay, az, du);
            a.vsigmax[i] = vsmax;
            // drho/dt = (1 / Omega) sum m_j v_ij.rhat_ij F(r, h_i) = rho A dup
            if (a.drhodt) a.drhodt[i] = qi.y * Ai * dup;
        }
    }
};

// Pair sums of the list kernel for one target, written for few instructions
// per pair with the per-particle factors taken from the force records:
//   F(r, h) = C f'(q) / h^4 = G C / h^4 g_p(p),  p = q / R = r rsqrt((R h)^2)
// (for M4, G = -3 and g_p(p) = max(1 - p, 0)^2 - max(1 - 2 p, 0)^2: the
// derivative -3 q + 9/4 q^2 for q < 1, -3/4 (2 - q)^2 for 1 <= q < 2, 0
// beyond).  With A = 1 / (rho Omega) and AK = G C A / h^4, A F = AK g_p.  A
// neighbour is one 48-byte record (three 16-byte loads from one address):
// (x, y, z, m), (vx, vy, vz, (gamma - 1) u), ((R h)^2, AK, alpha c, rho).
// The L1 data path is what bounds this kernel: the gathers deliver about
// 48 bytes per wavefront, so the record holds only what the pair needs.
// Per pair
// (Eqs. 9-15, w = min(v_ij . rhat_ij, 0), hw = -w / 2):
//   (P_i + q^i) / (rho_i^2 Omega_i) F_i = (P_i / rho_i + hw vsig_i) AK_i g_i
//   du/dt terms: sum m_j vr g_i, sum m_j vsig_i hw^2 g_i and the conduction
//   sum m_j |dP| rsqrt(|dP| (rho_i + rho_j)) (P_i/rho_i - P_j/rho_j) (AK_i g_i + AK_j g_j),
// whose constant factors are applied once per target at the end.
template <int K, bool PER>
struct ForceSums {
    float xi, yi, zi, vxi, vyi, vzi, pri;   // position, velocity, (gamma - 1) u
    float R2i, AKi, aci, rhoi, Pi;          // (R h)^2, AK, alpha c, rho, P
    float ax, ay, az, sp, sv, sc, vsmax;
    int cnt;

    __device__ __forceinline__ void init(const float4 *rec)
    {
        const float4 p = rec[0], v = rec[1], q = rec[2];
        xi = p.x; yi = p.y; zi = p.z;
        vxi = v.x; vyi = v.y; vzi = v.z; pri = v.w;
        R2i = q.x; AKi = q.y; aci = q.z; rhoi = q.w;
        Pi = pri * rhoi;
        ax = ay = az = sp = sv = sc = 0.f;
        vsmax = aci;
        cnt = 0;
    }

    // one list entry with record (p, v, q); valid = false for padding; PER:
    // nearest images on the periodic axes of P
    __device__ __forceinline__ void pair(const float4 p, const float4 v, const float4 q, bool valid,
                                         float beta, const Period &P)
    {
        const float prj = v.w;
        // canonical separation: decides the pair set, feeds the pair terms
        float dx = __fsub_rn(xi, p.x), dy = __fsub_rn(yi, p.y), dz = __fsub_rn(zi, p.z);
        if (PER) {
            dx = wrap_sep(dx, P.x);
            dy = wrap_sep(dy, P.y);
            dz = wrap_sep(dz, P.z);
        }
        const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        // r < R max(h_i, h_j) as r^2 < max((R h_i)^2, (R h_j)^2): squaring is monotone
        const bool in = valid && r2 > 0.f && r2 < fmaxf(R2i, q.x);
        const float mj = in ? p.w : 0.f;
        const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
        const float r = r2 * rinv;
        const float pi = r * rsqrtf(R2i), pj = r * rsqrtf(q.x);   // q / R of each side
        const float gi = SphKernel<K>::g_p(pi), gj = SphKernel<K>::g_p(pj);
        const float Ti = AKi * gi, Tj = q.y * gj;
        const float dvx = vxi - v.x, dvy = vyi - v.y, dvz = vzi - v.z, dpr = pri - prj;
        const float vr = fmaf(dvz, dz, fmaf(dvy, dy, dvx * dx)) * rinv;
        const float avr = fabsf(vr);
        const float vsi = fmaf(beta, avr, aci);
        const float hw = -0.5f * fminf(vr, 0.f);
        const float pi_ = fmaf(hw, vsi, pri);
        const float pj_ = fmaf(hw, fmaf(beta, avr, q.z), prj);
        const float cr = fmaf(pi_, Ti, pj_ * Tj) * (mj * rinv);
        ax = fmaf(-cr, dx, ax);
        ay = fmaf(-cr, dy, ay);
        az = fmaf(-cr, dz, az);
        const float mg = mj * gi;
        sp = fmaf(mg, vr, sp);
        sv = fmaf(mg, vsi * (hw * hw), sv);
        const float dP = fabsf(Pi - prj * q.w);
        const float vu = dP * rsqrtf(fmaxf(dP * (rhoi + q.w), 1e-30f));
        sc = fmaf(mj * (vu * dpr), Ti + Tj, sc);
        vsmax = fmaxf(vsmax, in ? vsi : 0.f);
        cnt += in ? 1 : 0;
    }

    // reduce over the L lanes of the target; lane sub == 0 writes
    __device__ __forceinline__ void finish(int L, bool write, int i, float gm1, float alpha_u,
                                           float4 *acc, float *vsig, float *drhodt)
    {
        for (int o = L >> 1; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            az += __shfl_xor_sync(0xffffffffu, az, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
            sc += __shfl_xor_sync(0xffffffffu, sc, o);
            vsmax = fmaxf(vsmax, __shfl_xor_sync(0xffffffffu, vsmax, o));
        }
        if (write) {
            // Eq. 10 pressure work, Eq. 13 viscous heating (sv holds w^2 / 4) and
            // conduction: vsig_u = sqrt(2) |dP| rsqrt(|dP| (rho_i + rho_j)), u = pr / (gamma - 1)
            const float du = AKi * (pri * sp - 2.f * sv) + (0.70710678118654752f * alpha_u / gm1) * sc;
            acc[i] = make_float4(ax, ay, az, du);
            vsig[i] = vsmax;
            // drho/dt = (1 / Omega) sum m_j v_ij.rhat_ij F(r, h_i) = rho AK sp
            if (drhodt) drhodt[i] = rhoi * AKi * sp;
        }
    }
};

// Launch shape (run-time): a.tb targets per batch (32 / a.tb lanes per
// target), blockDim.x / 32 warps per block; NPER list entries per lane and
// iteration.  Registers are capped for 768 resident threads per SM.
template <int NPER, int K, bool PER>
__global__ void __launch_bounds__(256, 3) force_list_kernel(ForceArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t keep = l2_keep_policy();
    const int ng = a.sizes[SZ_GROUPS];
    const bool lists_fresh = a.rec_ctl[1] == 0;
    unsigned long long n_pairs = 0, n_cand = 0, n_fb = 0;
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
            const int g = base + warp + nw * kr;
            if (g >= ng) break;
            const int2 gr = a.grp_ref[g];
            const int root = a.inst ? a.inst[gr.x] : 0;
            const bool usable = lists_fresh && a.rec_bad[root] == 0;
            for (int b0 = 0; b0 < gr.y; b0 += a.tb) {
                const int nt = min(a.tb, gr.y - b0);
                const int L = lanes_per_target(nt);
                const int t = lane >> (__ffs(L) - 1), sub = lane & (L - 1);  // L a power of two
                const bool act = t < nt;
                const int i = gr.x + b0 + (act ? t : 0);
                const bool on = act && (!a.active || a.active[i]);
                if (!__any_sync(0xffffffffu, on)) continue;  // no target of the batch is due
                const int len = usable && act ? a.nl_len[i] : 0;
                if (!usable || __any_sync(0xffffffffu, len < 0)) {
                    if (lane == 0) push_fallback_batch(a.fallback, a.n_fallback, g, b0, nt);
                    ++n_fb;
                    continue;
                }
                ForceSums<K, PER> T;
                T.init(a.frec + 3 * (size_t)i);
                const int *__restrict__ lst = a.nl_idx + (size_t)i * a.nl_stride;
                // Four consecutive entries per lane and iteration (one 16-byte
                // load of the list, fetched an iteration ahead), no branch: an
                // entry outside the pair set (or padding) gets zero mass.  The
                // particle itself (r = 0) is left out; a distinct particle at
                // r = 0 would add nothing either (every term carries f'(0) = 0 or
                // v_ij.r_ij / r = 0).
                auto entry = [&](int j, bool valid) {
                    const float4 *rj = a.frec + 3 * (size_t)j;
                    T.pair(ld_keep(rj, 0, keep), ld_keep(rj, 1, keep), ld_keep(rj, 2, keep), valid,
                           a.beta, a.tree.per);
                };
                if (NPER == 4) {
                    int e = 4 * sub;
                    int4 jn = e < len ? __ldcs(reinterpret_cast<const int4 *>(lst + e)) : make_int4(0, 0, 0, 0);
                    for (; e < len; e += 4 * L) {
                        const int4 jj = jn;
                        if (e + 4 * L < len) jn = __ldcs(reinterpret_cast<const int4 *>(lst + e + 4 * L));
                        const bool b1 = e + 1 < len, b2 = e + 2 < len, b3 = e + 3 < len;
                        entry(jj.x, true);
                        entry(b1 ? jj.y : jj.x, b1);
                        entry(b2 ? jj.z : jj.x, b2);
                        entry(b3 ? jj.w : jj.x, b3);
                    }
                } else {
                    int e = 2 * sub;
                    int2 jn = e < len ? __ldcs(reinterpret_cast<const int2 *>(lst + e)) : make_int2(0, 0);
                    for (; e < len; e += 2 * L) {
                        const int2 jj = jn;
                        if (e + 2 * L < len) jn = __ldcs(reinterpret_cast<const int2 *>(lst + e + 2 * L));
                        const bool b1 = e + 1 < len;
                        entry(jj.x, true);
                        entry(b1 ? jj.y : jj.x, b1);
                    }
                }
                T.finish(L, on && sub == 0, i, a.gm1, a.alpha_u, a.acc, a.vsigmax, a.drhodt);
                n_pairs += on ? T.cnt : 0;
                n_cand += on && sub == 0 ? (unsigned long long)len : 0ull;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_pairs += __shfl_xor_sync(0xffffffffu, n_pairs, o);
        n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_FORCE_PAIRS], n_pairs);
        atomicAdd(&a.counters[C_FORCE_CAND], n_cand);
        if (n_fb) atomicAdd(&a.counters[C_FORCE_FB], n_fb);  // warp-uniform count
    }
}

// Batches the list kernel handed over, with tree walks.
template <int CAP, int K>
__global__ void __launch_bounds__(kForceWarps * 32) force_walk_kernel(ForceArgs a)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    ForceSmem<CAP> &sm = reinterpret_cast<ForceSmem<CAP> *>(fsm_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int nfb = *a.n_fallback;
    if (nfb == 0) return;  // nothing handed over (the usual case): no atomics
    unsigned long long n_pairs = 0, n_cand = 0;

    while (true) {
        int k = 0;
        if (lane == 0) k = atomicAdd(a.work2, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nfb) break;
        const int2 fb = a.fallback[k];
        const int g = fb.x, b0 = fb.y & 0xffff, cnt = fb.y >> 16;  // cnt <= kFTB
        const int2 gr = a.grp_ref[g];
        const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        {
            const int nt = min(cnt, gr.y - b0);
            const int L = lanes_per_target(nt);
            const int t = lane >> (__ffs(L) - 1), sub = lane & (L - 1);  // L a power of two
            const bool act = t < nt;
            const int i0 = gr.x + b0;
            if (lane < kFTB) {
                const float4 p = lane < nt ? a.pos[i0 + lane] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                sm.tc.set(lane, p);
                sm.th[lane] = lane < nt ? a.prop[i0 + lane].x : 0.f;
                sm.tlen[lane] = 0;
                if (lane < nt) {
                    sm.tp[lane] = p;
                    sm.tv[lane] = a.vel[i0 + lane];
                    sm.tq[lane] = a.prop[i0 + lane];
                }
            }
            __syncwarp();
            ForceTarget<K> T;
            T.init(sm.tp[act ? t : 0], sm.tv[act ? t : 0], sm.tq[act ? t : 0], a);

            auto flush = [&]() {
                if (act) {
                    const int len = sm.tlen[t];
                    for (int e = sub; e < len; e += L) {
                        const int j = sm.ej[t][e];
                        const float4 pj = __ldg(&a.pos[j]);
                        T.pair(pj, __ldg(&a.vel[j]), __ldg(&a.prop[j]), pj.w, true, a);
                    }
                }
                __syncwarp();
                if (lane < nt) sm.tlen[lane] = 0;
                __syncwarp();
            };
            auto chunk = [&](int j) {
                const float4 pj = j >= 0 ? __ldg(&a.pos[j]) : make_float4(0, 0, 0, 0);
                const float hj = j >= 0 ? __ldg(&a.prop[j].x) : 0.f;
                unsigned bs[kFTB];
                int base[kFTB];
                bool over = false;
#pragma unroll
                for (int q = 0; q < kFTB / 2; ++q) {
                    const int t0 = 2 * q, t1 = 2 * q + 1;
                    bs[t0] = bs[t1] = 0u;
                    base[t0] = base[t1] = 0;
                    if (t0 < nt) {
                        const float2 r2 = canon_r2_x2p(sm.tc.x[q], sm.tc.y[q], sm.tc.z[q], pj.x, pj.y, pj.z,
                                                       a.tree.per);
                        const float R0 = SphKernel<K>::R * fmaxf(sm.th[t0], hj);
                        const float R1 = SphKernel<K>::R * fmaxf(sm.th[t1], hj);
                        bs[t0] = __ballot_sync(0xffffffffu, j >= 0 && j != i0 + t0 && r2.x < R0 * R0);
                        bs[t1] = __ballot_sync(0xffffffffu, j >= 0 && t1 < nt && j != i0 + t1 && r2.y < R1 * R1);
                        base[t0] = sm.tlen[t0];
                        base[t1] = sm.tlen[t1];
                        over |= base[t0] + __popc(bs[t0]) > CAP;
                        over |= base[t1] + __popc(bs[t1]) > CAP;
                    }
                }
                if (over) {  // run the pairs listed so far, then start over
                    flush();
#pragma unroll
                    for (int tt = 0; tt < kFTB; ++tt) base[tt] = 0;
                }
#pragma unroll
                for (int tt = 0; tt < kFTB; ++tt) {
                    if (tt < nt) {
                        if ((bs[tt] >> lane) & 1u) sm.ej[tt][base[tt] + __popc(bs[tt] & lt)] = j;
                        if (lane == tt) sm.tlen[tt] = base[tt] + __popc(bs[tt]);
                    }
                }
                __syncwarp();
                n_cand += (unsigned long long)nt;
            };
            const int root = a.inst ? a.inst[gr.x] : 0;
            // opens a node within R max(h_max(group), h_max(node)) of the group box
            constexpr float hr = 0.5f * SphKernel<K>::R;
            bool ok = walk_group(a.tree, root, glo, ghi, 0.f, true, hr * glo.w, sm.w, chunk, hr);
            if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
            flush();
            const bool on = act && (!a.active || a.active[i0 + t]);
            T.finish(L, on && sub == 0, i0 + t, a);
            n_pairs += on ? T.cnt : 0;
            __syncwarp();
        }
    }
    for (int o = 16; o > 0; o >>= 1) n_pairs += __shfl_xor_sync(0xffffffffu, n_pairs, o);
    if (lane == 0) {
        atomicAdd(&a.counters[C_FORCE_PAIRS], n_pairs);
        atomicAdd(&a.counters[C_FORCE_CAND], n_cand * 32);  // 32 lanes per chunk-target
    }
}

// prop = (h, rho, 1/(rho Omega), c_s) and the force records from the state
// (kr = R, gc = G C of the kernel); checks vel and u
__global__ void force_prep_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                  const float *__restrict__ h, const float *__restrict__ rho,
                                  const float *__restrict__ omega, float4 *__restrict__ prop,
                                  float4 *__restrict__ frec, int n, float gamma, float alpha, float kr,
                                  float gc, float h_lim, int *err)
{
    bool bad = false, neg = false, wide = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 v = vel[i];
        const float r = rho[i], o = omega[i], hi = h[i];
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w) && isfinite(r) &&
                 isfinite(o));
        neg |= v.w < 0.f;
        wide |= !(hi < h_lim);  // the support would reach a second periodic image
        const float cs = sqrtf(fmaxf(gamma * (gamma - 1.f) * v.w, 0.f));
        const float A = 1.f / (r * o);
        prop[i] = make_float4(hi, r, A, cs);
        const float R = kr * hi;
        const float hinv = 1.f / hi, hinv2 = hinv * hinv;
        frec[3 * (size_t)i] = pos[i];
        frec[3 * (size_t)i + 1] = make_float4(v.x, v.y, v.z, (gamma - 1.f) * v.w);
        frec[3 * (size_t)i + 2] = make_float4(R * R, gc * A * hinv2 * hinv2, alpha * cs, r);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_NONFINITE);
    if (__any_sync(0xffffffffu, neg) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_NEGATIVE_U);
    if (__any_sync(0xffffffffu, wide) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_INVALID_ARG);
}

// one-time kernel attributes and occupancy (also called before graph capture)
template <int CAP, int K>
static cudaError_t configure_force(int &blocks)
{
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int nb_cached = 1;
    if (!configured) {
        size_t smem = sizeof(ForceSmem<CAP>) * kForceWarps;
        cudaError_t e = cudaFuncSetAttribute(force_walk_kernel<CAP, K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, force_walk_kernel<CAP, K>, kForceWarps * 32,
                                                          smem);
        if (e != cudaSuccess) return e;
        nb_cached = nb > 0 ? nb : 1;
        configured = true;
    }
    blocks = nb_cached;
    return cudaSuccess;
}

// Resident blocks per SM of the list kernel for each (entries per lane,
// warps per block): computed once, before any graph capture.
template <int K>
static cudaError_t configure_force_list(int blocks[2][4])
{
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int nb_cached[2][4];
    if (!configured) {
        for (int u = 0; u < 2; ++u)
            for (int w = 0; w < 4; ++w) {
                int nb = 0;
                const int threads = 32 << w;  // 1, 2, 4, 8 warps
                cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &nb, u ? force_list_kernel<4, K, false> : force_list_kernel<2, K, false>, threads, 0);
                int nbp = 0;
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &nbp, u ? force_list_kernel<4, K, true> : force_list_kernel<2, K, true>, threads, 0);
                if (e != cudaSuccess) return e;
                nb = nbp < nb ? nbp : nb;
                nb_cached[u][w] = nb > 0 ? nb : 1;
            }
        configured = true;
    }
    for (int u = 0; u < 2; ++u)
        for (int w = 0; w < 4; ++w) blocks[u][w] = nb_cached[u][w];
    return cudaSuccess;
}

template <int CAP, int K>
static cudaError_t launch_force_walk(Ctx &c, const ForceArgs &a, cudaStream_t st)
{
    int blocks = 1;
    cudaError_t e = configure_force<CAP, K>(blocks);
    if (e != cudaSuccess) return e;
    size_t smem = sizeof(ForceSmem<CAP>) * kForceWarps;
    force_walk_kernel<CAP, K><<<c.num_sms * blocks, kForceWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int K>
static cudaError_t configure_force_k()
{
    int b, bl[2][4];
    cudaError_t e = configure_force_list<K>(bl);
    if (e == cudaSuccess) e = configure_force<64, K>(b);
    if (e == cudaSuccess) e = configure_force<96, K>(b);
    if (e == cudaSuccess) e = configure_force<128, K>(b);
    return e;
}

cudaError_t configure_force_kernels(int kernel)
{
    return kernel == 1 ? configure_force_k<1>() : kernel == 2 ? configure_force_k<2>()
                                                              : configure_force_k<0>();
}

cudaError_t force_prep(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                       bool hmax_now)
{
    const int n = (int)s.n;
    int grid = (n + 255) / 256;
    if (grid > c.num_sms * 16) grid = c.num_sms * 16;
    force_prep_kernel<<<grid, 256, 0, st>>>((const float4 *)s.pos, (const float4 *)s.vel, s.h, s.rho,
                                            s.omega, c.prop, c.frec, n, p.gamma, p.alpha_av,
                                            kernel_support(p.kernel), kernel_gc(p.kernel),
                                            periodic_h_limit(p), c.d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return hmax_now ? update_hmax(c, s, p, st) : cudaSuccess;
}

// the list kernel, then the walking kernel for the batches it handed over
template <int K>
static cudaError_t force_launch_k(Ctx &c, ForceArgs &a, const sph_params &p, const sph_state &s,
                                  cudaStream_t st)
{
    int bl[2][4];
    cudaError_t e = configure_force_list<K>(bl);
    if (e != cudaSuccess) return e;
    const PairShape ps = pair_shape(p);
    a.tb = ps.targets;
    const int u = ps.unroll == 4 ? 1 : 0, wl = ps.warps == 8 ? 3 : ps.warps == 4 ? 2 : ps.warps == 2 ? 1 : 0;
    const int grid = c.num_sms * bl[u][wl];
    const bool per = a.tree.per.any();
    if (u && per) force_list_kernel<4, K, true><<<grid, 32 * ps.warps, 0, st>>>(a);
    else if (u) force_list_kernel<4, K, false><<<grid, 32 * ps.warps, 0, st>>>(a);
    else if (per) force_list_kernel<2, K, true><<<grid, 32 * ps.warps, 0, st>>>(a);
    else force_list_kernel<2, K, false><<<grid, 32 * ps.warps, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the walking kernel needs node and group h_max of the final h; refreshed
    // only when some batch was handed over
    e = update_hmax(c, s, p, st, a.n_fallback);
    if (e != cudaSuccess) return e;
    int cap = p.tile > 0 ? p.tile : K == 0 ? 96 : 128;
    if (cap <= 64) return launch_force_walk<64, K>(c, a, st);
    if (cap <= 96) return launch_force_walk<96, K>(c, a, st);
    return launch_force_walk<128, K>(c, a, st);
}

cudaError_t force_pass(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                       const Batch *batch)
{
    cudaError_t e;
    ForceArgs a{};
    a.inst = batch ? c.inst : nullptr;
    a.nl_idx = c.nl_idx;
    a.nl_len = c.nl_len;
    a.nl_stride = c.nl_stride;
    a.active = c.mask;
    a.rec_ctl = c.tree.rec_ctl;
    a.rec_bad = c.tree.rec_bad;
    a.fallback = c.fallback;
    a.n_fallback = c.d_sizes + SZ_FALLBACK;
    a.pos = (const float4 *)s.pos;
    a.vel = (const float4 *)s.vel;
    a.prop = c.prop;
    a.frec = c.frec;
    a.acc = (float4 *)s.acc;
    a.vsigmax = s.vsigmax;
    a.drhodt = c.drhodt_in_force ? s.drhodt : nullptr;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.work2 = c.d_sizes + SZ_WORK2;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref, period_of(p)};
    a.gm1 = p.gamma - 1.f;
    a.alpha = p.alpha_av;
    a.beta = p.beta_av;
    a.alpha_u = p.alpha_u;
    a.err = c.d_err;
    a.counters = c.d_counters;
    e = check_list_kernel(c, p, st);
    if (e != cudaSuccess) return e;
    // lists of instances where an h outgrew the pad are rebuilt at the final h
    e = relist_pass(c, s, p, kListPad, st, batch);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.work, 0, 3 * sizeof(int), st);  // work, fallback count, work2
    if (e != cudaSuccess) return e;
    if (p.kernel == 1) return force_launch_k<1>(c, a, p, s, st);
    if (p.kernel == 2) return force_launch_k<2>(c, a, p, s, st);
    return force_launch_k<0>(c, a, p, s, st);
}

}  // namespace sph
