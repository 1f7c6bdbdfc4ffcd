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
// Force backward: the pair term T_ij (the contribution of j to a_i and du_i)
// is written once as a template over the scalar type; forward-mode dual
// numbers give its derivatives with respect to one particle's inputs
// (x, v, u, h, rho, Omega) and alpha_AV, in passes of 4 derivative slots.
//
// Density backward (implicit-function theorem): h_i solves
// g_i = sum_j m_j W(r_ij, h_i) - M_i / h_i^3 = 0, M_i = m_i hfact^3, with
// dg_i/dh_i = 3 rho_i Omega_i / h_i and dg_i/dr_ij = m_j F(r_ij, h_i);
// rho_i = M_i / h_i^3 and Omega_i = 1 + h_i^4 S_i / (3 M_i),
// S_i = sum_j m_j dW/dh(r_ij, h_i).
#include "walk.cuh"

namespace sph {

// ------------------------------------------------------------ dual numbers
template <int N>
struct Dual {
    float v;
    float d[N];
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(float x) : v(x)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = 0.f;
    }
};

template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N> &a, const Dual<N> &b)
{
    Dual<N> r;
    float inv = 1.f / b.v;
    r.v = a.v * inv;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(float s, const Dual<N> &a)
{
    Dual<N> r;
    r.v = s * a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = s * a.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a)
{
    return (-1.f) * a;
}
template <int N>
__device__ __forceinline__ Dual<N> dsqrt(const Dual<N> &a)
{
    Dual<N> r;
    r.v = sqrtf(a.v);
    // sqrt at 0: zero derivative (the only places this happens are the
    // conduction speed of two particles at equal pressure, times u_i - u_j)
    float g = r.v > 0.f ? 0.5f / r.v : 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = g * a.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> dabs(const Dual<N> &a)
{
    return a.v < 0.f ? -a : a;
}

__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float dabs(float a) { return fabsf(a); }
__device__ __forceinline__ float val(float a) { return a; }
template <int N>
__device__ __forceinline__ float val(const Dual<N> &a) { return a.v; }

// (gamma-1)(rho_i u_i - rho_j u_j): the value in FP64, because the two
// pressures are often nearly equal and the conduction speed's derivative
// carries 1 / sqrt(|P_i - P_j|)
__device__ __forceinline__ float pdiff(float gm1, float ri, float ui, float rj, float uj)
{
    return (float)((double)gm1 * ((double)ri * (double)ui - (double)rj * (double)uj));
}
template <int N>
__device__ __forceinline__ Dual<N> pdiff(float gm1, const Dual<N> &ri, const Dual<N> &ui,
                                         const Dual<N> &rj, const Dual<N> &uj)
{
    Dual<N> r;
    r.v = pdiff(gm1, ri.v, ui.v, rj.v, uj.v);
#pragma unroll
    for (int k = 0; k < N; ++k)
        r.d[k] = gm1 * (ri.d[k] * ui.v + ri.v * ui.d[k] - rj.d[k] * uj.v - rj.v * uj.d[k]);
    return r;
}

// M4 f'(q), piecewise on the value of q
template <class S>
__device__ __forceinline__ S m4_dfq(const S &q)
{
    if (val(q) < 1.f) return q * (S(-3.f) + 2.25f * q);
    if (val(q) < 2.f) {
        S t = S(2.f) - q;
        return (-0.75f) * (t * t);
    }
    return S(0.f);
}

// Contribution of neighbour j to a_i (xyz) and du_i/dt (Eqs. 9-15), the same
// arithmetic as the force pass.
template <class S>
__device__ __forceinline__ void force_pair(const S xi[3], const S vi[3], const S &ui, const S &hi,
                                           const S &rhoi, const S &omi, const S xj[3],
                                           const S vj[3], const S &uj, const S &hj,
                                           const S &rhoj, const S &omj, float mj, const S &alpha,
                                           float beta, float alpha_u, float gamma, S out[4])
{
    const float gm1 = gamma - 1.f;
    S dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
    S r = dsqrt(dx * dx + dy * dy + dz * dz);
    if (!(val(r) > 0.f)) {
        out[0] = out[1] = out[2] = out[3] = S(0.f);
        return;
    }
    S rinv = S(1.f) / r;
    S h2i = hi * hi, h2j = hj * hj;
    S Fi = (kCNorm * m4_dfq(r / hi)) / (h2i * h2i);
    S Fj = (kCNorm * m4_dfq(r / hj)) / (h2j * h2j);
    S vr = ((vi[0] - vj[0]) * dx + (vi[1] - vj[1]) * dy + (vi[2] - vj[2]) * dz) * rinv;
    S avr = dabs(vr);
    S ci = dsqrt(gamma * gm1 * ui), cj = dsqrt(gamma * gm1 * uj);
    S vsi = alpha * ci + beta * avr;
    S avi(0.f), avj(0.f), duav(0.f);
    if (val(vr) < 0.f) {
        S vsj = alpha * cj + beta * avr;
        avi = (-0.5f) * (vsi * vr);
        avj = (-0.5f) * (vsj * vr);
        duav = 0.5f * (vsi * vr * vr * Fi);
    }
    S Ai = S(1.f) / (rhoi * omi), Aj = S(1.f) / (rhoj * omj);
    S coef = mj * (Ai * (gm1 * ui + avi) * Fi + Aj * (gm1 * uj + avj) * Fj);
    S cr = coef * rinv;
    out[0] = -(cr * dx);
    out[1] = -(cr * dy);
    out[2] = -(cr * dz);
    S vsu = dsqrt(dabs(pdiff(gm1, rhoi, ui, rhoj, uj)) / (0.5f * (rhoi + rhoj)));
    out[3] = mj * (gm1 * (ui * Ai * vr * Fi) - Ai * duav +
                   0.5f * alpha_u * (vsu * (ui - uj) * (Fi * Ai + Fj * Aj)));
}

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
    int dens_set;  // 1: density set r < 2 h_i (self included); 0: force set
    // neighbour lists of the last density pass (a superset of both pair sets
    // while they are fresh and no h of the instance outgrew the list pad)
    const int *nl_idx, *nl_len, *rec_ctl, *rec_bad;
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
            const int t = lane / L, sub = lane % L;
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
                        const float r2 = canon_r2(tp.x, tp.y, tp.z, pj.x, pj.y, pj.z);
                        bool hit;
                        if (a.dens_set) {
                            const float R = 2.0f * sm.th[tt];
                            hit = j >= 0 && r2 < R * R;
                        } else {
                            const float R = 2.0f * fmaxf(sm.th[tt], hj);
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
                    const int *__restrict__ lst = a.nl_idx + (size_t)i * kNbrCap;
                    const float4 tp = sm.tp[t];
                    const float ht = sm.th[t];
                    for (int e = sub; e < len; e += L) {
                        const int j = __ldcs(lst + e);
                        const float4 pj = __ldg(&a.pos[j]);
                        const float r2 = canon_r2(tp.x, tp.y, tp.z, pj.x, pj.y, pj.z);
                        const float R = a.dens_set ? 2.0f * ht : 2.0f * fmaxf(ht, __ldg(&a.h[j]));
                        if (r2 < R * R && (a.dens_set || j != i)) op.pair(i, j, acc);
                    }
                }
                __syncwarp();
            } else {
                bool ok = a.dens_set ? walk_group(a.tree, root, glo, ghi, 2.f * hmx, false, 0.f, sm.w, chunk)
                                     : walk_group(a.tree, root, glo, ghi, 0.f, true, hmx, sm.w, chunk);
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
struct ForceBwdOp {
    const float4 *pos, *vel, *gacc;  // gacc: (dL/da xyz, dL/d(du/dt))
    const float *h, *rho, *omega;
    float4 *gpos, *gvel;             // out: dL/dx (xyz, 0), dL/dv (xyz), dL/du (w)
    float *gh, *grho, *gom;          // out
    double *galpha;                  // out: accumulated (one atomic per target)
    float alpha, beta, alpha_u, gamma;
    struct Acc {
        float g[10];  // x0 x1 x2 v0 v1 v2 u h rho om
        float ga;
    };
    __device__ void init(int, Acc &c) const
    {
#pragma unroll
        for (int k = 0; k < 10; ++k) c.g[k] = 0.f;
        c.ga = 0.f;
    }
    // side: 0 -> derivatives of T_kj w.r.t. k's inputs (k = "i" of the pair);
    //       1 -> derivatives of T_jk w.r.t. k's inputs (k = "j" of the pair)
    template <int P>
    __device__ void pass(int k, int j, int side, Acc &c) const
    {
        typedef Dual<4> D;
        const int base = 4 * P;  // input slots base .. base+3 of (x0..om, alpha)
        float4 pk = pos[k], vk = vel[k], pj = pos[j], vj = vel[j];
        float fk[11] = {pk.x, pk.y, pk.z, vk.x, vk.y, vk.z, vk.w, h[k], rho[k], omega[k], alpha};
        float fj[10] = {pj.x, pj.y, pj.z, vj.x, vj.y, vj.z, vj.w, h[j], rho[j], omega[j]};
        D dk[11], dj[10];
#pragma unroll
        for (int s = 0; s < 11; ++s) {
            dk[s] = D(fk[s]);
            if (s >= base && s < base + 4 && (s < 10 || side == 0)) dk[s].d[s - base] = 1.f;
        }
#pragma unroll
        for (int s = 0; s < 10; ++s) dj[s] = D(fj[s]);
        D out[4];
        const D al = dk[10];
        if (side == 0)
            force_pair(dk, dk + 3, dk[6], dk[7], dk[8], dk[9], dj, dj + 3, dj[6], dj[7], dj[8], dj[9],
                       pj.w, al, beta, alpha_u, gamma, out);
        else
            force_pair(dj, dj + 3, dj[6], dj[7], dj[8], dj[9], dk, dk + 3, dk[6], dk[7], dk[8], dk[9],
                       pk.w, D(alpha), beta, alpha_u, gamma, out);
        const float4 w = gacc[side == 0 ? k : j];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float v = w.x * out[0].d[s] + w.y * out[1].d[s] + w.z * out[2].d[s] + w.w * out[3].d[s];
            int slot = base + s;
            if (slot < 10) c.g[slot] += v;
            else if (slot == 10 && side == 0) c.ga += v;
        }
    }
    __device__ void pair(int k, int j, Acc &c) const
    {
        pass<0>(k, j, 0, c);
        pass<1>(k, j, 0, c);
        pass<2>(k, j, 0, c);
        pass<0>(k, j, 1, c);
        pass<1>(k, j, 1, c);
        pass<2>(k, j, 1, c);
    }
    __device__ void reduce(Acc &c, int L) const
    {
        for (int o = L >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 10; ++k) c.g[k] += __shfl_xor_sync(0xffffffffu, c.g[k], o);
            c.ga += __shfl_xor_sync(0xffffffffu, c.ga, o);
        }
    }
    __device__ void store(int k, Acc &c) const
    {
        gpos[k] = make_float4(c.g[0], c.g[1], c.g[2], 0.f);
        gvel[k] = make_float4(c.g[3], c.g[4], c.g[5], c.g[6]);
        gh[k] = c.g[7];
        grho[k] = c.g[8];
        gom[k] = c.g[9];
        atomicAdd(galpha, (double)c.ga);
    }
};

// --------------------------------------------------------- density backward
// M4 pieces: f, f', f''
__device__ __forceinline__ void m4_all(float q, float &f, float &df, float &d2f)
{
    if (q < 1.f) {
        f = 1.f + q * q * (-1.5f + 0.75f * q);
        df = q * (-3.f + 2.25f * q);
        d2f = -3.f + 4.5f * q;
    } else if (q < 2.f) {
        float t = 2.f - q;
        f = 0.25f * t * t * t;
        df = -0.75f * t * t;
        d2f = 1.5f * t;
    } else {
        f = df = d2f = 0.f;
    }
}

// pass 1: per target, S = sum m dW/dh and S2 = sum m d2W/dh2 over the density
// set; then lambda (the IFT multiplier) and omega-coefficient per particle.
struct DensBwd1Op {
    const float4 *pos;
    const float *h, *rho, *omega;
    const float *gh, *grho, *gom;  // cotangents of h, rho, Omega
    float2 *coef;                  // out: (lambda, w)
    float hf3;
    struct Acc { float S, S2; };
    __device__ void init(int, Acc &c) const { c.S = 0.f; c.S2 = 0.f; }
    __device__ void pair(int i, int j, Acc &c) const
    {
        float4 pi = pos[i], pj = pos[j];
        float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        float r = sqrtf(dx * dx + dy * dy + dz * dz);
        float hi = h[i], hinv = 1.f / hi;
        float q = r * hinv, f, df, d2f;
        m4_all(q, f, df, d2f);
        float h4 = hinv * hinv * hinv * hinv;
        c.S += pj.w * (-kCNorm * (3.f * f + q * df) * h4);
        c.S2 += pj.w * (kCNorm * (12.f * f + 8.f * q * df + q * q * d2f) * h4 * hinv);
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
struct DensBwd2Op {
    const float4 *pos;
    const float *h;
    const float2 *coef;
    float4 *gpos;  // accumulated (+=)
    struct Acc { float g[3]; };
    __device__ void init(int, Acc &c) const { c.g[0] = c.g[1] = c.g[2] = 0.f; }
    __device__ static float cterm(float r, float hh, float lam, float w, float m)
    {
        float hinv = 1.f / hh, q = r * hinv, f, df, d2f;
        m4_all(q, f, df, d2f);
        float h4 = hinv * hinv * hinv * hinv;
        float F = kCNorm * df * h4;
        float Whr = -kCNorm * (4.f * df + q * d2f) * h4 * hinv;
        return m * (-lam * F + w * Whr);
    }
    __device__ void pair(int k, int j, Acc &c) const
    {
        float4 pk = pos[k], pj = pos[j];
        float dx = pk.x - pj.x, dy = pk.y - pj.y, dz = pk.z - pj.z;
        float r = sqrtf(dx * dx + dy * dy + dz * dz);
        if (!(r > 0.f)) return;
        float2 ck = coef[k], cj = coef[j];
        float s = (cterm(r, h[k], ck.x, ck.y, pj.w) + cterm(r, h[j], cj.x, cj.y, pk.w)) / r;
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
static cudaError_t launch_pairwalk(Ctx &c, const sph_state &s, bool dens_set, const Op &op,
                                   cudaStream_t st, const Batch *batch)
{
    size_t smem = sizeof(PairWalkSmem<CAP>) * 4;
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
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref};
    a.inst = batch ? c.inst : nullptr;
    a.dens_set = dens_set ? 1 : 0;
    a.nl_idx = c.nl_idx;
    a.nl_len = c.nl_len;
    a.rec_ctl = c.tree.rec_ctl;
    a.rec_bad = c.tree.rec_bad;
    a.err = c.d_err;
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    pairwalk_kernel<CAP, Op><<<c.num_sms * blocks, 128, smem, st>>>(a, op);
    return cudaGetLastError();
}

cudaError_t force_bwd(Ctx &c, const sph_state &s, const sph_params &p, const float4 *gacc,
                      float4 *gpos, float4 *gvel, float *gh, float *grho, float *gom,
                      double *galpha, cudaStream_t st)
{
    ForceBwdOp op;
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
    // the force-set walk needs node and group h_max of the current h
    cudaError_t e = update_hmax(c, s, p, st);
    if (e != cudaSuccess) return e;
    return launch_pairwalk<96>(c, s, false, op, st, nullptr);
}

cudaError_t density_bwd(Ctx &c, const sph_state &s, const sph_params &p, const float *gh,
                        const float *grho, const float *gom, float4 *gpos, float2 *coef,
                        cudaStream_t st)
{
    DensBwd1Op op1;
    op1.pos = (const float4 *)s.pos;
    op1.h = s.h;
    op1.rho = s.rho;
    op1.omega = s.omega;
    op1.gh = gh;
    op1.grho = grho;
    op1.gom = gom;
    op1.coef = coef;
    op1.hf3 = p.hfact * p.hfact * p.hfact;
    // pass 2 opens nodes by their h_max (force set): refresh it for the current h
    cudaError_t e = update_hmax(c, s, p, st);
    if (e != cudaSuccess) return e;
    e = launch_pairwalk<96>(c, s, true, op1, st, nullptr);
    if (e != cudaSuccess) return e;
    DensBwd2Op op2;
    op2.pos = (const float4 *)s.pos;
    op2.h = s.h;
    op2.coef = coef;
    op2.gpos = gpos;
    return launch_pairwalk<96>(c, s, false, op2, st, nullptr);
}

}  // namespace sph
