// Adjoint (reverse-mode) kernels of the density and force passes, for the
// differentiable rollout.  Not part of the paper's method; they differentiate
// Eqs. 1-4 and 9-15 as implemented by density.cu and force.cu.
//
// All backward passes are "pull" passes: a warp walks the tree for a group of
// targets, collects each target's neighbours (force set, or density set), and
// every target sums the cotangent contributions that land on ITS inputs, from
// its own equations and from its neighbours' equations.  No atomics, so the
// results are deterministic.
//
// Force backward: the vector-Jacobian product of the pair term T_ij (the
// contribution of j to a_i and du_i/dt, Eqs. 9-15 as the force pass computes
// them) is a hand-written reverse sweep (force_pair_vjp), one sweep per pair
// and side, in FP32 only (this GPU's FP64 rate is a small fraction of FP32's).
//
// Density backward (implicit-function theorem): h_i solves
// g_i = sum_j m_j W(r_ij, h_i) - M_i / h_i^3 = 0, M_i = m_i hfact^3, with
// dg_i/dh_i = 3 rho_i Omega_i / h_i and dg_i/dr_ij = m_j F(r_ij, h_i);
// rho_i = M_i / h_i^3 and Omega_i = 1 + h_i^4 S_i / (3 M_i),
// S_i = sum_j m_j dW/dh(r_ij, h_i).
//
// The pair operations are templates on the smoothing kernel K (SphKernel<K>:
// f, f', f'' and the support radius R).
#include "kernels.cuh"
#include "walk.cuh"

namespace sph {

// ------------------------------------------------------- generic pair walk
struct PairWalkArgs {
    const float4 *pos;
    const float *h;
    const int2 *grp_ref;
    const float4 *grp_lo, *grp_hi;
    const int *sizes;
    int *work;
    WalkTree tree;
    const int *inst;
    int dens_set;  // 1: density set r < R h_i (self included); 0: force set r < R max(h_i, h_j)
    float kr;      // R, the kernel's support radius in units of h
    // neighbour lists of the last density pass (a superset of both pair sets
    // while they are fresh and no h of the instance outgrew the list pad)
    const int *nl_idx, *nl_len, *rec_ctl, *rec_bad;
    int nl_stride;
    int *err;
};

constexpr int kPW_TB = 8;

template <int CAP>
struct PairWalkSmem {
    WalkSmem w;
    float4 tp[kPW_TB];
    float th[kPW_TB];
    int tlen[kPW_TB];
    int ej[kPW_TB][CAP];
};

// Op: struct with  Acc;  init(i, Acc&);  pair(i, j, Acc&);  reduce(Acc&, L);  store(i, Acc&)
template <int CAP, class Op>
__global__ void __launch_bounds__(128) pairwalk_kernel(PairWalkArgs a, Op op)
{
    extern __shared__ __align__(16) unsigned char pw_raw[];
    PairWalkSmem<CAP> &sm = reinterpret_cast<PairWalkSmem<CAP> *>(pw_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int ng = a.sizes[SZ_GROUPS];
    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.work, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int2 gr = a.grp_ref[g];
        const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        const int root = a.inst ? a.inst[gr.x] : 0;
        for (int b0 = 0; b0 < gr.y; b0 += kPW_TB) {
            const int nt = min(kPW_TB, gr.y - b0);
            const int L = nt > 4 ? 4 : nt > 2 ? 8 : nt > 1 ? 16 : 32;
            const int t = lane >> (__ffs(L) - 1), sub = lane & (L - 1);  // L a power of two
            const bool act = t < nt;
            const int i0 = gr.x + b0;
            const int i = i0 + (act ? t : 0);
            if (lane < nt) {
                sm.tp[lane] = a.pos[i0 + lane];
                sm.th[lane] = a.h[i0 + lane];
                sm.tlen[lane] = 0;
            }
            __syncwarp();
            typename Op::Acc acc;
            op.init(i, acc);
            float hmx = lane < nt ? sm.th[lane] : 0.f;
            for (int o = 16; o > 0; o >>= 1) hmx = fmaxf(hmx, __shfl_xor_sync(0xffffffffu, hmx, o));
            auto flush = [&]() {
                if (act) {
                    const int len = sm.tlen[t];
                    for (int e = sub; e < len; e += L) op.pair(i, sm.ej[t][e], acc);
                }
                __syncwarp();
                if (lane < nt) sm.tlen[lane] = 0;
                __syncwarp();
            };
            auto chunk = [&](int j) {
                const float4 pj = j >= 0 ? __ldg(&a.pos[j]) : make_float4(0, 0, 0, 0);
                const float hj = j >= 0 ? __ldg(&a.h[j]) : 0.f;
                unsigned bs[kPW_TB];
                int base[kPW_TB];
                bool over = false;
#pragma unroll
                for (int tt = 0; tt < kPW_TB; ++tt) {
                    bs[tt] = 0u;
                    base[tt] = 0;
                    if (tt < nt) {
                        const float4 tp = sm.tp[tt];
                        const float r2 = canon_r2p(tp.x, tp.y, tp.z, pj.x, pj.y, pj.z, a.tree.per);
                        bool hit;
                        if (a.dens_set) {
                            const float R = a.kr * sm.th[tt];
                            hit = j >= 0 && r2 < R * R;
                        } else {
                            const float R = a.kr * fmaxf(sm.th[tt], hj);
                            hit = j >= 0 && j != i0 + tt && r2 < R * R;
                        }
                        bs[tt] = __ballot_sync(0xffffffffu, hit);
                        base[tt] = sm.tlen[tt];
                        over |= base[tt] + __popc(bs[tt]) > CAP;
                    }
                }
                if (over) {
                    flush();
#pragma unroll
                    for (int tt = 0; tt < kPW_TB; ++tt) base[tt] = 0;
                }
#pragma unroll
                for (int tt = 0; tt < kPW_TB; ++tt) {
                    if (tt < nt) {
                        if ((bs[tt] >> lane) & 1u) sm.ej[tt][base[tt] + __popc(bs[tt] & lt)] = j;
                        if (lane == tt) sm.tlen[tt] = base[tt] + __popc(bs[tt]);
                    }
                }
                __syncwarp();
            };
            const int len = act ? a.nl_len[i] : 0;
            const bool lists = a.rec_ctl[1] == 0 && a.rec_bad[root] == 0 &&
                               !__any_sync(0xffffffffu, len < 0);
            if (lists) {
                // the pair set from the target's list, with the same exact tests
                if (act) {
                    const int *__restrict__ lst = a.nl_idx + (size_t)i * a.nl_stride;
                    const float4 tp = sm.tp[t];
                    const float ht = sm.th[t];
                    for (int e = sub; e < len; e += L) {
                        const int j = __ldcs(lst + e);
                        const float4 pj = __ldg(&a.pos[j]);
                        const float r2 = canon_r2p(tp.x, tp.y, tp.z, pj.x, pj.y, pj.z, a.tree.per);
                        const float R = a.dens_set ? a.kr * ht : a.kr * fmaxf(ht, __ldg(&a.h[j]));
                        if (r2 < R * R && (a.dens_set || j != i)) op.pair(i, j, acc);
                    }
                }
                __syncwarp();
            } else {
                const float hr = 0.5f * a.kr;
                bool ok = a.dens_set ? walk_group(a.tree, root, glo, ghi, a.kr * hmx, false, 0.f, sm.w, chunk)
                                     : walk_group(a.tree, root, glo, ghi, 0.f, true, hr * hmx, sm.w, chunk, hr);
                if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
                flush();
            }
            op.reduce(acc, L);
            if (act && sub == 0) op.store(i, acc);
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------ force backward
// Inputs of one particle in a pair term.
struct PairIn {
    float x[3], v[3], u, h, rho, om;
};

// P_i - P_j = (gamma - 1)(rho_i u_i - rho_j u_j) without FP64 (whose rate is
// a small fraction of FP32's on this GPU): each product's rounding error is
// recovered exactly with an FMA, and when the pressures are close the
// difference of the rounded products is exact (Sterbenz), so the difference
// keeps about twice FP32's precision.  The conduction speed's derivative
// carries 1 / sqrt(|P_i - P_j|), so the difference must not be swamped by
// the rounding of the two pressures.
__device__ __forceinline__ float pressure_diff(float gm1, float ri, float ui, float rj, float uj)
{
    const float a = ri * ui, b = rj * uj;
    const float ea = fmaf(ri, ui, -a), eb = fmaf(rj, uj, -b);
    return gm1 * ((a - b) + (ea - eb));
}

// sqrt(x) for x >= 0 through the hardware reciprocal square root (0 at 0)
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// Reverse-mode derivative of the pair term T_ij (particle I in the role of
// i, J in the role of j, the same operations as the force pass): given the
// cotangent w of (a_i xyz, du_i/dt), adds w . dT_ij / d(inputs of I) to g
// and w . dT_ij / d alpha to *galpha (WANT_I), or w . dT_ij / d(inputs of J)
// to g (otherwise).  r = 0 gives no term, the viscous terms act for vr < 0
// only, |x| has derivative +1 at 0, and sqrt has derivative 0 at 0 (at equal
// pressures the conduction term carries u_i - u_j times a zero speed).
// Quotients and roots use the hardware approximations (a few ulp).
template <bool WANT_I, int K>
__device__ __forceinline__ void force_pair_vjp(const PairIn &I, const PairIn &J, float mj, float alpha,
                                               float beta, float alpha_u, float gamma, float4 w,
                                               const Period &P, PairIn &g, float &galpha)
{
    const float gm1 = gamma - 1.f;
    // nearest images on the periodic axes (the wrap's derivative is 1)
    const float dx = wrap_sep(I.x[0] - J.x[0], P.x), dy = wrap_sep(I.x[1] - J.x[1], P.y),
                dz = wrap_sep(I.x[2] - J.x[2], P.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 > 0.f)) return;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    // ---- forward values
    const float hiinv = __fdividef(1.f, I.h), hjinv = __fdividef(1.f, J.h);
    const float qi = r * hiinv, qj = r * hjinv;
    const float dfi = SphKernel<K>::df(qi), dfj = SphKernel<K>::df(qj);
    const float h2i = hiinv * hiinv, h2j = hjinv * hjinv;
    const float Ki = SphKernel<K>::C * h2i * h2i, Kj = SphKernel<K>::C * h2j * h2j;  // C / h^4
    const float Fi = dfi * Ki, Fj = dfj * Kj;
    const float dvx = I.v[0] - J.v[0], dvy = I.v[1] - J.v[1], dvz = I.v[2] - J.v[2];
    const float sd = dvx * dx + dvy * dy + dvz * dz;
    const float vr = sd * rinv;
    const float avr = fabsf(vr);
    const float ci = fast_sqrt(gamma * gm1 * I.u), cj = fast_sqrt(gamma * gm1 * J.u);
    const float vsi = alpha * ci + beta * avr;
    const bool visc = vr < 0.f;
    const float vsj = alpha * cj + beta * avr;
    const float avi = visc ? -0.5f * (vsi * vr) : 0.f;
    const float avj = visc ? -0.5f * (vsj * vr) : 0.f;
    const float duav = visc ? 0.5f * (vsi * vr * vr * Fi) : 0.f;
    const float rhoinv_i = __fdividef(1.f, I.rho), rhoinv_j = __fdividef(1.f, J.rho);
    const float Ai = rhoinv_i * __fdividef(1.f, I.om), Aj = rhoinv_j * __fdividef(1.f, J.om);
    const float pi_ = gm1 * I.u + avi, pj_ = gm1 * J.u + avj;
    const float Ti = Ai * pi_ * Fi, Tj = Aj * pj_ * Fj;
    const float coef = mj * (Ti + Tj);
    const float PD = pressure_diff(gm1, I.rho, I.u, J.rho, J.u);
    const float APD = fabsf(PD);
    const float Sinv = __fdividef(2.f, I.rho + J.rho);   // 1 / (rho_i + rho_j) / 2
    const float X = APD * Sinv;
    const float vsu = fast_sqrt(X);
    const float du = I.u - J.u;
    const float AF = Fi * Ai + Fj * Aj;
    // ---- reverse sweep
    float bui = 0.f, bhi = 0.f, brhoi = 0.f, bomi = 0.f;
    float buj = 0.f, bhj = 0.f, brhoj = 0.f, bomj = 0.f;
    float bal = 0.f;
    // out_a = -coef rinv d
    const float Wd = w.x * dx + w.y * dy + w.z * dz;
    const float bcr = -Wd;
    const float cri = -coef * rinv;
    float bdx = cri * w.x, bdy = cri * w.y, bdz = cri * w.z;
    float brinv = bcr * coef;
    const float bcoef = bcr * rinv;
    // out_u = mj E, E = gm1 u_i A_i vr F_i - A_i duav + 0.5 alpha_u vsu (u_i - u_j) AF
    const float bE = w.w * mj;
    const float hau = 0.5f * alpha_u * bE;
    bui += bE * gm1 * Ai * vr * Fi + hau * vsu * AF;
    buj += -hau * vsu * AF;
    float bAi = bE * (gm1 * I.u * vr * Fi - duav);
    float bvr = bE * gm1 * I.u * Ai * Fi;
    float bFi = bE * gm1 * I.u * Ai * vr;
    const float bduav = -bE * Ai;
    const float bvsu = hau * du * AF;
    const float bAF = hau * vsu * du;
    // AF = F_i A_i + F_j A_j
    bFi += bAF * Ai;
    bAi += bAF * Fi;
    float bFj = bAF * Aj;
    float bAj = bAF * Fj;
    // vsu = sqrt(|PD| / Srho), Srho = (rho_i + rho_j) / 2
    const float bX = vsu > 0.f ? __fdividef(0.5f * bvsu, vsu) : 0.f;
    const float bAPD = bX * Sinv;
    const float bSrho = -bX * X * Sinv;
    const float bPD = PD < 0.f ? -bAPD : bAPD;
    brhoi += bPD * gm1 * I.u + 0.5f * bSrho;
    bui += bPD * gm1 * I.rho;
    brhoj += -bPD * gm1 * J.u + 0.5f * bSrho;
    buj += -bPD * gm1 * J.rho;
    // coef = mj (T_i + T_j), T = A p F
    const float bT = bcoef * mj;
    bAi += bT * pi_ * Fi;
    bFi += bT * Ai * pi_;
    const float bpi = bT * Ai * Fi;
    bAj += bT * pj_ * Fj;
    bFj += bT * Aj * pj_;
    const float bpj = bT * Aj * Fj;
    bui += bpi * gm1;
    buj += bpj * gm1;
    float bavr = 0.f, bci = 0.f, bcj = 0.f;
    if (visc) {
        // avi = -vsi vr / 2, avj = -vsj vr / 2, duav = vsi vr^2 F_i / 2
        const float bvsi = bpi * (-0.5f * vr) + bduav * 0.5f * vr * vr * Fi;
        const float bvsj = bpj * (-0.5f * vr);
        bvr += bpi * (-0.5f * vsi) + bpj * (-0.5f * vsj) + bduav * vsi * vr * Fi;
        bFi += bduav * 0.5f * vsi * vr * vr;
        bal += bvsi * ci + bvsj * cj;
        bci += bvsi * alpha;
        bcj += bvsj * alpha;
        bavr += (bvsi + bvsj) * beta;
    }
    // A = 1 / (rho Omega)
    brhoi += -bAi * Ai * rhoinv_i;
    bomi += -bAi * Ai * __fdividef(1.f, I.om);
    brhoj += -bAj * Aj * rhoinv_j;
    bomj += -bAj * Aj * __fdividef(1.f, J.om);
    // c = sqrt(gamma gm1 u)
    bui += ci > 0.f ? __fdividef(bci * gamma * gm1 * 0.5f, ci) : 0.f;
    buj += cj > 0.f ? __fdividef(bcj * gamma * gm1 * 0.5f, cj) : 0.f;
    // avr = |vr| (derivative +1 at 0)
    bvr += vr < 0.f ? -bavr : bavr;
    // vr = sd rinv
    const float bsd = bvr * rinv;
    brinv += bvr * sd;
    bdx += bsd * dvx;
    bdy += bsd * dvy;
    bdz += bsd * dvz;
    // F = C f'(q) / h^4, q = r / h
    float br = 0.f;
    {
        const float bq = bFi * Ki * SphKernel<K>::d2f(qi);
        bhi += -4.f * bFi * Fi * hiinv - bq * qi * hiinv;
        br += bq * hiinv;
    }
    {
        const float bq = bFj * Kj * SphKernel<K>::d2f(qj);
        bhj += -4.f * bFj * Fj * hjinv - bq * qj * hjinv;
        br += bq * hjinv;
    }
    // rinv = 1 / r, r = |d|
    br += -brinv * rinv * rinv;
    bdx += br * rinv * dx;
    bdy += br * rinv * dy;
    bdz += br * rinv * dz;
    if (WANT_I) {
        g.x[0] += bdx;
        g.x[1] += bdy;
        g.x[2] += bdz;
        g.v[0] += bsd * dx;
        g.v[1] += bsd * dy;
        g.v[2] += bsd * dz;
        g.u += bui;
        g.h += bhi;
        g.rho += brhoi;
        g.om += bomi;
        galpha += bal;
    } else {
        // d = x_i - x_j, dv = v_i - v_j
        g.x[0] -= bdx;
        g.x[1] -= bdy;
        g.x[2] -= bdz;
        g.v[0] -= bsd * dx;
        g.v[1] -= bsd * dy;
        g.v[2] -= bsd * dz;
        g.u += buj;
        g.h += bhj;
        g.rho += brhoj;
        g.om += bomj;
    }
}

template <int KER>
struct ForceBwdOp {
    const float4 *pos, *vel, *gacc;  // gacc: (dL/da xyz, dL/d(du/dt))
    const float *h, *rho, *omega;
    float4 *gpos, *gvel;             // out: dL/dx (xyz, 0), dL/dv (xyz), dL/du (w)
    float *gh, *grho, *gom;          // out
    double *galpha;                  // out: accumulated (one atomic per target)
    float alpha, beta, alpha_u, gamma;
    Period per;
    struct Acc {
        PairIn K;     // the target's own inputs, loaded once
        float mk;
        float4 wk;    // the target's cotangent
        PairIn g;
        float ga;
    };
    __device__ PairIn load(int k) const
    {
        const float4 p = pos[k], v = vel[k];
        return PairIn{{p.x, p.y, p.z}, {v.x, v.y, v.z}, v.w, h[k], rho[k], omega[k]};
    }
    __device__ void init(int k, Acc &c) const
    {
        c.K = load(k);
        c.mk = pos[k].w;
        c.wk = gacc[k];
        c.g = PairIn{{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, 0.f, 0.f, 0.f, 0.f};
        c.ga = 0.f;
    }
    // the terms that land on k's inputs: from k's own equations (T_kj with
    // cotangent gacc[k]) and from j's (T_jk with cotangent gacc[j])
    __device__ void pair(int k, int j, Acc &c) const
    {
        (void)k;
        const PairIn J = load(j);
        force_pair_vjp<true, KER>(c.K, J, pos[j].w, alpha, beta, alpha_u, gamma, c.wk, per, c.g, c.ga);
        float unused = 0.f;
        force_pair_vjp<false, KER>(J, c.K, c.mk, alpha, beta, alpha_u, gamma, gacc[j], per, c.g, unused);
    }
    __device__ void reduce(Acc &c, int L) const
    {
        for (int o = L >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                c.g.x[a] += __shfl_xor_sync(0xffffffffu, c.g.x[a], o);
                c.g.v[a] += __shfl_xor_sync(0xffffffffu, c.g.v[a], o);
            }
            c.g.u += __shfl_xor_sync(0xffffffffu, c.g.u, o);
            c.g.h += __shfl_xor_sync(0xffffffffu, c.g.h, o);
            c.g.rho += __shfl_xor_sync(0xffffffffu, c.g.rho, o);
            c.g.om += __shfl_xor_sync(0xffffffffu, c.g.om, o);
            c.ga += __shfl_xor_sync(0xffffffffu, c.ga, o);
        }
    }
    __device__ void store(int k, Acc &c) const
    {
        gpos[k] = make_float4(c.g.x[0], c.g.x[1], c.g.x[2], 0.f);
        gvel[k] = make_float4(c.g.v[0], c.g.v[1], c.g.v[2], c.g.u);
        gh[k] = c.g.h;
        grho[k] = c.g.rho;
        gom[k] = c.g.om;
        atomicAdd(galpha, (double)c.ga);
    }
};

// --------------------------------------------------------- density backward
// kernel pieces f, f', f'' at q (all 0 beyond the support)
template <int K>
__device__ __forceinline__ void kernel_all(float q, float &f, float &df, float &d2f)
{
    SphKernel<K>::f_df(q, f, df);
    d2f = SphKernel<K>::d2f(q);
}

// pass 1: per target, S = sum m dW/dh and S2 = sum m d2W/dh2 over the density
// set; then lambda (the IFT multiplier) and omega-coefficient per particle.
template <int K>
struct DensBwd1Op {
    const float4 *pos;
    const float *h, *rho, *omega;
    const float *gh, *grho, *gom;  // cotangents of h, rho, Omega
    float2 *coef;                  // out: (lambda, w)
    float hf3;
    Period per;
    struct Acc { float S, S2; };
    __device__ void init(int, Acc &c) const { c.S = 0.f; c.S2 = 0.f; }
    __device__ void pair(int i, int j, Acc &c) const
    {
        float4 pi = pos[i], pj = pos[j];
        float dx = wrap_sep(pi.x - pj.x, per.x), dy = wrap_sep(pi.y - pj.y, per.y),
              dz = wrap_sep(pi.z - pj.z, per.z);
        float r = fast_sqrt(dx * dx + dy * dy + dz * dz);
        float hi = h[i], hinv = __fdividef(1.f, hi);
        float q = r * hinv, f, df, d2f;
        kernel_all<K>(q, f, df, d2f);
        float h4 = hinv * hinv * hinv * hinv;
        constexpr float C = SphKernel<K>::C;
        c.S += pj.w * (-C * (3.f * f + q * df) * h4);
        c.S2 += pj.w * (C * (12.f * f + 8.f * q * df + q * q * d2f) * h4 * hinv);
    }
    __device__ void reduce(Acc &c, int L) const
    {
        for (int o = L >> 1; o > 0; o >>= 1) {
            c.S += __shfl_xor_sync(0xffffffffu, c.S, o);
            c.S2 += __shfl_xor_sync(0xffffffffu, c.S2, o);
        }
    }
    __device__ void store(int i, Acc &c) const
    {
        float hi = h[i], M = pos[i].w * hf3;
        float h3 = hi * hi * hi, h4 = h3 * hi;
        float domdh = (4.f * h3 * c.S + h4 * c.S2) / (3.f * M);
        float htot = gh[i] - 3.f * rho[i] / hi * grho[i] + gom[i] * domdh;
        float lambda = htot * hi / (3.f * rho[i] * omega[i]);
        coef[i] = make_float2(lambda, gom[i] * h4 / (3.f * M));
    }
};

// pass 2 (force set): gx_k += sum_j (c_kj + c_jk) rhat_kj,
// c_ij = -lambda_i m_j F(r, h_i) + w_i m_j d2W/dh dr(r, h_i)
template <int K>
struct DensBwd2Op {
    const float4 *pos;
    const float *h;
    const float2 *coef;
    float4 *gpos;  // accumulated (+=)
    Period per;
    struct Acc { float g[3]; };
    __device__ void init(int, Acc &c) const { c.g[0] = c.g[1] = c.g[2] = 0.f; }
    __device__ static float cterm(float r, float hh, float lam, float w, float m)
    {
        float hinv = __fdividef(1.f, hh), q = r * hinv, f, df, d2f;
        kernel_all<K>(q, f, df, d2f);
        float h4 = hinv * hinv * hinv * hinv;
        constexpr float C = SphKernel<K>::C;
        float F = C * df * h4;
        float Whr = -C * (4.f * df + q * d2f) * h4 * hinv;
        return m * (-lam * F + w * Whr);
    }
    __device__ void pair(int k, int j, Acc &c) const
    {
        float4 pk = pos[k], pj = pos[j];
        float dx = wrap_sep(pk.x - pj.x, per.x), dy = wrap_sep(pk.y - pj.y, per.y),
              dz = wrap_sep(pk.z - pj.z, per.z);
        float r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 > 0.f)) return;
        float rinv = rsqrtf(r2), r = r2 * rinv;
        float2 ck = coef[k], cj = coef[j];
        float s = (cterm(r, h[k], ck.x, ck.y, pj.w) + cterm(r, h[j], cj.x, cj.y, pk.w)) * rinv;
        c.g[0] += s * dx;
        c.g[1] += s * dy;
        c.g[2] += s * dz;
    }
    __device__ void reduce(Acc &c, int L) const
    {
        for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) c.g[a] += __shfl_xor_sync(0xffffffffu, c.g[a], o);
    }
    __device__ void store(int k, Acc &c) const
    {
        float4 g = gpos[k];
        gpos[k] = make_float4(g.x + c.g[0], g.y + c.g[1], g.z + c.g[2], g.w);
    }
};

// ------------------------------------------------------------------ launch
template <int CAP, class Op>
static cudaError_t launch_pairwalk(Ctx &c, const sph_state &s, bool dens_set, float kr, Period per,
                                   const Op &op, cudaStream_t st, const Batch *batch)
{
    size_t smem = sizeof(PairWalkSmem<CAP>) * 4;
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int blocks = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(pairwalk_kernel<CAP, Op>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pairwalk_kernel<CAP, Op>, 128, smem);
        if (e != cudaSuccess) return e;
        blocks = nb > 0 ? nb : 1;
        configured = true;
    }
    PairWalkArgs a{};
    a.pos = (const float4 *)s.pos;
    a.h = s.h;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref, per};
    a.inst = batch ? c.inst : nullptr;
    a.dens_set = dens_set ? 1 : 0;
    a.kr = kr;
    a.nl_idx = c.nl_idx;
    a.nl_len = c.nl_len;
    a.nl_stride = c.nl_stride;
    a.rec_ctl = c.tree.rec_ctl;
    a.rec_bad = c.tree.rec_bad;
    a.err = c.d_err;
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    pairwalk_kernel<CAP, Op><<<c.num_sms * blocks, 128, smem, st>>>(a, op);
    return cudaGetLastError();
}

template <int K>
static cudaError_t force_bwd_k(Ctx &c, const sph_state &s, const sph_params &p, const float4 *gacc,
                               float4 *gpos, float4 *gvel, float *gh, float *grho, float *gom,
                               double *galpha, cudaStream_t st)
{
    ForceBwdOp<K> op;
    op.pos = (const float4 *)s.pos;
    op.vel = (const float4 *)s.vel;
    op.gacc = gacc;
    op.h = s.h;
    op.rho = s.rho;
    op.omega = s.omega;
    op.gpos = gpos;
    op.gvel = gvel;
    op.gh = gh;
    op.grho = grho;
    op.gom = gom;
    op.galpha = galpha;
    op.alpha = p.alpha_av;
    op.beta = p.beta_av;
    op.alpha_u = p.alpha_u;
    op.gamma = p.gamma;
    op.per = period_of(p);
    // the force-set walk needs node and group h_max of the current h
    cudaError_t e = check_list_kernel(c, p, st);
    if (e == cudaSuccess) e = update_hmax(c, s, p, st);
    if (e != cudaSuccess) return e;
    return launch_pairwalk<96>(c, s, false, SphKernel<K>::R, op.per, op, st, nullptr);
}

cudaError_t force_bwd(Ctx &c, const sph_state &s, const sph_params &p, const float4 *gacc,
                      float4 *gpos, float4 *gvel, float *gh, float *grho, float *gom,
                      double *galpha, cudaStream_t st)
{
    if (p.kernel == 1) return force_bwd_k<1>(c, s, p, gacc, gpos, gvel, gh, grho, gom, galpha, st);
    if (p.kernel == 2) return force_bwd_k<2>(c, s, p, gacc, gpos, gvel, gh, grho, gom, galpha, st);
    return force_bwd_k<0>(c, s, p, gacc, gpos, gvel, gh, grho, gom, galpha, st);
}

template <int K>
static cudaError_t density_bwd_k(Ctx &c, const sph_state &s, const sph_params &p, const float *gh,
                                 const float *grho, const float *gom, float4 *gpos, float2 *coef,
                                 cudaStream_t st, bool refresh_hmax)
{
    DensBwd1Op<K> op1;
    op1.pos = (const float4 *)s.pos;
    op1.h = s.h;
    op1.rho = s.rho;
    op1.omega = s.omega;
    op1.gh = gh;
    op1.grho = grho;
    op1.gom = gom;
    op1.coef = coef;
    op1.hf3 = p.hfact * p.hfact * p.hfact;
    op1.per = period_of(p);
    // pass 2 opens nodes by their h_max (force set) where it walks: refresh it
    // for the current h (unless the caller just did)
    cudaError_t e = check_list_kernel(c, p, st);
    if (e == cudaSuccess && refresh_hmax) e = update_hmax(c, s, p, st);
    if (e != cudaSuccess) return e;
    e = launch_pairwalk<96>(c, s, true, SphKernel<K>::R, op1.per, op1, st, nullptr);
    if (e != cudaSuccess) return e;
    DensBwd2Op<K> op2;
    op2.pos = (const float4 *)s.pos;
    op2.h = s.h;
    op2.coef = coef;
    op2.gpos = gpos;
    op2.per = op1.per;
    return launch_pairwalk<96>(c, s, false, SphKernel<K>::R, op2.per, op2, st, nullptr);
}

cudaError_t density_bwd(Ctx &c, const sph_state &s, const sph_params &p, const float *gh,
                        const float *grho, const float *gom, float4 *gpos, float2 *coef,
                        cudaStream_t st, bool refresh_hmax)
{
    if (p.kernel == 1) return density_bwd_k<1>(c, s, p, gh, grho, gom, gpos, coef, st, refresh_hmax);
    if (p.kernel == 2) return density_bwd_k<2>(c, s, p, gh, grho, gom, gpos, coef, st, refresh_hmax);
    return density_bwd_k<0>(c, s, p, gh, grho, gom, gpos, coef, st, refresh_hmax);
}

}  // namespace sph
