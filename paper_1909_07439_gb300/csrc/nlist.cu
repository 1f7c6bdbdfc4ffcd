// Neighbour lists for the density and force passes.
//
// One tree walk per group (Sect. 3.2) finds, for every particle i, the
// particles j with
//     r_ij < 2 (1 + pad) max(h_i, h_j)          (h at the start of the pass)
// and stores them in i's fixed-size slot of nl_idx (curve order, walk order).
// That set holds both pair sets of the step as long as no smoothing length
// grows by more than the pad during the h-rho solve:
//   density (Eq. 1):       r_ij < 2 h_i,           h_i <= (1 + pad) h_i,in
//   force   (Eqs. 9-15):   r_ij < 2 max(h_i, h_j), both h <= (1 + pad) h_in
// so the density Newton sweeps and the force pass read lists instead of
// walking; the few particles that leave the pad (and lists that overflow
// kNbrCap) are handed to the walking kernels.
//
// The walk opens a node if its box is within max(reach of the batch,
// 2 (1 + pad) h_max(node)) of the group box, so every j of the set is a
// candidate.  Each 32-candidate chunk is tested against up to 16 targets
// with the canonical FP32 squared distance (two targets per packed
// instruction); hits go straight to the lists in global memory.
#include "walk.cuh"

namespace sph {

constexpr int kNlTB = 16;       // targets per walk
constexpr int kNlWarps = 4;     // warps per block
constexpr float kListSlack = 1.0f + 1e-5f;  // list radius margin over the FP32 pad checks

struct NlistSmem {
    WalkSmem w;
    TargetPairs<kNlTB> tc;
    float tr[kNlTB];  // list radius factor x h_i (0 for unused slots)
};

struct NlistArgs {
    const float4 *pos;
    const float *h;
    const int2 *grp_ref;
    const float4 *grp_lo, *grp_hi;
    const int *sizes;
    int *work;
    WalkTree tree;
    const int *inst;
    float rscale;  // list radius = rscale * max(h_i, h_j)
    int *idx, *len;
    int *err;
    unsigned long long *counters;
};

__global__ void __launch_bounds__(kNlWarps * 32) nlist_kernel(NlistArgs a)
{
    __shared__ NlistSmem smv[kNlWarps];
    NlistSmem &sm = smv[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int ng = a.sizes[SZ_GROUPS];
    unsigned long long n_cand = 0, n_entries = 0, n_over = 0;

    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(a.work, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const int2 gr = a.grp_ref[g];
        const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
        const int root = a.inst ? a.inst[gr.x] : 0;
        for (int b0 = 0; b0 < gr.y; b0 += kNlTB) {
            const int nt = min(kNlTB, gr.y - b0);
            const int i0 = gr.x + b0;
            float rt = 0.f;
            if (lane < kNlTB) {
                const float4 p = lane < nt ? a.pos[i0 + lane] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                sm.tc.set(lane, p);
                rt = lane < nt ? a.rscale * a.h[i0 + lane] : 0.f;
                sm.tr[lane] = rt;
            }
            for (int o = 16; o > 0; o >>= 1) rt = fmaxf(rt, __shfl_xor_sync(0xffffffffu, rt, o));
            __syncwarp();
            int len[kNlTB];
#pragma unroll
            for (int tt = 0; tt < kNlTB; ++tt) len[tt] = 0;
            auto chunk = [&](int j) {
                const float4 pj = j >= 0 ? __ldg(&a.pos[j]) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float rj = j >= 0 ? a.rscale * __ldg(&a.h[j]) : 0.f;
#pragma unroll
                for (int q = 0; q < kNlTB / 2; ++q) {
                    const int t0 = 2 * q, t1 = t0 + 1;
                    if (t0 < nt) {
                        const float2 r2 = canon_r2_x2(sm.tc.x[q], sm.tc.y[q], sm.tc.z[q], pj.x, pj.y, pj.z);
                        const float R0 = fmaxf(sm.tr[t0], rj), R1 = fmaxf(sm.tr[t1], rj);
                        const bool hit0 = j >= 0 && r2.x < R0 * R0;
                        const bool hit1 = j >= 0 && t1 < nt && r2.y < R1 * R1;
                        const unsigned m0 = __ballot_sync(0xffffffffu, hit0);
                        const unsigned m1 = __ballot_sync(0xffffffffu, hit1);
                        if (hit0) {
                            const int e = len[t0] + __popc(m0 & lt);
                            if (e < kNbrCap) a.idx[(size_t)(i0 + t0) * kNbrCap + e] = j;
                        }
                        if (hit1) {
                            const int e = len[t1] + __popc(m1 & lt);
                            if (e < kNbrCap) a.idx[(size_t)(i0 + t1) * kNbrCap + e] = j;
                        }
                        len[t0] += __popc(m0);
                        len[t1] += __popc(m1);
                    }
                }
                n_cand += (unsigned long long)(nt * __popc(__ballot_sync(0xffffffffu, j >= 0)));
            };
            // open a node within max(rt, rscale h_max(node)) of the group box
            const bool ok = walk_group(a.tree, root, glo, ghi, 0.f, true, 0.5f * rt, sm.w, chunk,
                                       0.5f * a.rscale);
            if (!ok && lane == 0) raise_error(a.err, SPH_ERR_TILE_OVERFLOW);
            int mine = 0;
#pragma unroll
            for (int tt = 0; tt < kNlTB; ++tt)
                if (lane == tt) mine = len[tt];
            const bool fits = ok && mine <= kNbrCap;
            if (lane < nt) {
                a.len[i0 + lane] = fits ? mine : -1;
                n_entries += (unsigned long long)min(mine, kNbrCap);
                n_over += fits ? 0ull : 1ull;
            }
            __syncwarp();
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_entries += __shfl_xor_sync(0xffffffffu, n_entries, o);
        n_over += __shfl_xor_sync(0xffffffffu, n_over, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_DENS_CAND], n_cand);  // candidate x target tests
        atomicAdd(&a.counters[C_LIST_ENTRIES], n_entries);
        atomicAdd(&a.counters[C_LIST_OVERFLOW], n_over);
    }
}

static cudaError_t configure_nlist(int &blocks)
{
    static bool configured = false;
    static int nb_cached = 1;
    if (!configured) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, nlist_kernel, kNlWarps * 32, 0);
        if (e != cudaSuccess) return e;
        nb_cached = nb > 0 ? nb : 1;
        configured = true;
    }
    blocks = nb_cached;
    return cudaSuccess;
}

cudaError_t configure_nlist_kernels()
{
    int b;
    return configure_nlist(b);
}

cudaError_t nlist_pass(Ctx &c, const sph_state &s, const sph_params &p, float pad, cudaStream_t st,
                       const Batch *batch)
{
    (void)p;
    int blocks = 1;
    cudaError_t e = configure_nlist(blocks);
    if (e != cudaSuccess) return e;
    NlistArgs a{};
    a.pos = (const float4 *)s.pos;
    a.h = s.h;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref};
    a.inst = batch ? c.inst : nullptr;
    a.rscale = 2.f * (1.f + pad) * kListSlack;
    a.idx = c.nl_idx;
    a.len = c.nl_len;
    a.err = c.d_err;
    a.counters = c.d_counters;
    e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    nlist_kernel<<<c.num_sms * blocks, kNlWarps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sph
