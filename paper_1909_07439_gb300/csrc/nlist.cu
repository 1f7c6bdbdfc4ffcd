// Neighbour lists for the density and force passes.
//
// For every particle i the list holds the particles j with
//     r_ij < 2 (1 + pad) max(h_i, h_j)          (h at the start of the pass)
// in i's fixed-size slot of nl_idx (curve order).  That set holds both pair
// sets of the step as long as no smoothing length grows by more than the pad
// during the h-rho solve:
//   density (Eq. 1):       r_ij < 2 h_i,           h_i <= (1 + pad) h_i,in
//   force   (Eqs. 9-15):   r_ij < 2 max(h_i, h_j), both h <= (1 + pad) h_in
// so the density Newton sweeps and the force pass read lists instead of
// walking; the few particles that leave the pad (and lists that overflow
// their capacity, or groups whose walk finds more than kSGLeaves leaves) are handed
// to the walking kernels.
//
// Candidates come from the group walk of Sect. 3.2: a leaf is opened for a
// group if its box is within max(reach of the group, 2 (1 + pad) h_max(leaf))
// of the group box.  One persistent kernel, nlist_kernel: each warp takes up
// to kSG consecutive groups at a time.  Runs of those groups of one instance
// whose h_max agree within kShareH share one tree walk for the union of their
// boxes and their largest h (2 nodes per lane and walk step); the walk's
// leaves are ranked by first particle.  A node that passes the opening test
// for a box passes it for any box containing it, so each group then picks its
// own leaves from that list with its own test and gets the candidates its own
// walk would give, in particle order; while a shared walk finds more than
// kSGLeaves leaves, its range of groups is halved.  A group's targets are
// taken in batches of up to kNlTB; the candidates within reach of a batch's
// box are queued, and every 32 queued candidates are tested against the
// batch's targets with the canonical FP32 squared distance (two targets per
// packed instruction); hits go straight to the lists in global memory.
#include "kernels.cuh"
#include "walk.cuh"

namespace sph {

constexpr int kNlTB = 8;        // targets per candidate test batch
constexpr int kNlWarps = 4;     // warps per block
constexpr int kSG = 8;          // consecutive groups that may share one tree walk
constexpr int kSGLeaves = 320;  // leaves one walk may find
constexpr int kMaxRuns = 128;   // candidate runs of one group (plus a sentinel)
constexpr int kLWWide = 2;      // nodes per lane and walk step
constexpr int kLWStack = 320;   // stack entries of a wide walk
constexpr float kShareH = 2.f;  // groups share a walk if their h_max differ by less
constexpr float kListSlack = 1.0f + 1e-5f;  // list radius margin over the FP32 pad checks

struct NlistWalkPart {
    WalkSmemW<kLWWide, kLWStack> w;
    int2 lv[kSGLeaves];        // walk output (node, first); then a group's leaves (first, count)
};

// A batch's candidates that pass its box test, waiting to be tested against
// its targets in chunks of 32 (in slot order)
struct NlistQueue {
    float4 p[64];              // x, y, z, (list radius factor x h_j)^2
    int j[64];
};

struct NlistSmem {
    // the walk's scratch is free while a group's batches are tested
    union {
        NlistWalkPart wp;
        NlistQueue q;
    } u;
    int leaves[kSGLeaves];     // the walk's leaves (nodes) in particle order
    int2 runs[kMaxRuns + 1];   // a group's candidate runs: (first particle, first slot), sentinel
    TargetPairs<kNlTB> tc;
    float tr2[kNlTB];          // (list radius factor x h_i)^2 (0 for unused slots)
    float4 blo, bhi;           // the batch's box; bhi.w: its largest tr2
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
    int cap;       // entries per list (and the lists' stride)
    const uint8_t *active;  // lists only for groups holding one of these targets (nullptr: all)
    int *idx;
    int *len;
    // relist mode: the kernel returns at once unless *gate != 0, and builds the
    // lists only of groups whose instance k has only_bad[k] != 0
    const int *gate, *only_bad;
    int *err;
    unsigned long long *counters;
};

// Walk for the box [blo, bhi] (h_max blo.w) and put the leaves, in particle
// order, in sm.leaves.  Returns their number, or -1 if more than kSGLeaves.
template <bool PER>
__device__ __forceinline__ int walk_sorted(const NlistArgs &a, NlistSmem &sm, int root, float4 blo,
                                           float4 bhi)
{
    const int lane = threadIdx.x & 31;
    const int n = walk_leaves_wide<kLWWide, kLWStack, PER>(a.tree, root, blo, bhi, 0.5f * (a.rscale * blo.w), 0.5f * a.rscale,
                                   sm.u.wp.w, sm.u.wp.lv, kSGLeaves);
    __syncwarp();
    // rank sort by first particle (leaves hold disjoint particle ranges)
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        const int2 me = k < n ? sm.u.wp.lv[k] : make_int2(-1, 0x7fffffff);
        int rank = 0;
        for (int m = 0; m < n; ++m) rank += sm.u.wp.lv[m].y < me.y ? 1 : 0;
        if (k < n) sm.leaves[rank] = me.x;
    }
    __syncwarp();
    return n;
}

// The group's candidates: the leaves of sm.leaves that pass the group's own
// opening test (the test of walk_step for the group box and hgroup = rscale
// h_max(group) / 2), in particle order, merged into maximal contiguous runs
// of particles numbered by slot: sm.runs[m] = (first particle, first slot),
// sm.runs[nrun] = (-1, number of slots).  A node that passes the test for a
// box passes it for any box containing it, so when sm.leaves comes from a
// walk shared with other groups (union box, largest h) the result is the same
// as for the group's own walk.  Returns nrun, or -1 if more than max_runs.
template <bool PER>
__device__ __forceinline__ int group_candidates(const NlistArgs &a, NlistSmem &sm, int nleaf,
                                                float4 glo, float4 ghi, int max_runs)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const float hgroup = 0.5f * (a.rscale * glo.w), node_scale = 0.5f * a.rscale;
    int nsel = 0;
    for (int k0 = 0; k0 < nleaf; k0 += 32) {
        const int k = k0 + lane;
        const int node = k < nleaf ? sm.leaves[k] : -1;
        bool open = false;
        int2 ref = make_int2(0, 0);
        if (node >= 0) {
            const float4 lo = __ldg(&a.tree.node_lo[node]);
            const float4 hi = __ldg(&a.tree.node_hi[node]);
            ref = __ldg(&a.tree.node_ref[node]);
            const float d2 = box_dist2_c<PER>(a.tree, glo, ghi, lo, hi);
            const float R = 2.0f * fmaxf(hgroup, lo.w * node_scale);
            open = d2 < R * R * kOpenSlack;
        }
        const unsigned m = __ballot_sync(0xffffffffu, open);
        __syncwarp();
        if (open) sm.u.wp.lv[nsel + __popc(m & lt)] = ref;
        nsel += __popc(m);
    }
    __syncwarp();
    // merge: a leaf starts a run unless its particles continue the previous one's
    int nrun = 0, slot = 0;
    for (int k0 = 0; k0 < nsel; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < nsel;
        const int2 cur = valid ? sm.u.wp.lv[k] : make_int2(0, 0);
        const bool st = valid && (k == 0 || sm.u.wp.lv[k - 1].x + sm.u.wp.lv[k - 1].y != cur.x);
        const unsigned bst = __ballot_sync(0xffffffffu, st);
        int inc = cur.y;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int p = nrun + __popc(bst & lt);
        if (st && p < max_runs) sm.runs[p] = make_int2(cur.x, slot + inc - cur.y);
        nrun += __popc(bst);
        slot += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0 && nrun <= max_runs) sm.runs[nrun] = make_int2(-1, slot);
    __syncwarp();
    return nrun <= max_runs ? nrun : -1;
}

// Test up to 32 queued candidates (entries [0, cnt) of sm.u.q, one per lane)
// against the batch's targets (TB slots, the unused ones far away: no
// candidate hits them, and a missing candidate, also far away, hits no
// target) and append the hits to the targets' lists.
template <int TB, bool PER, int CAP>
__device__ __forceinline__ void test_queued(const NlistArgs &a, const NlistSmem &sm, int cnt, int *tbase,
                                            int (&len)[TB])
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const bool v = lane < cnt;
    const float4 pj = v ? sm.u.q.p[lane] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
    const int j = v ? sm.u.q.j[lane] : -1;
#pragma unroll
    for (int q = 0; q < TB / 2; ++q) {
        const int t0 = 2 * q, t1 = t0 + 1;
        // r < max(R_i, R_j) as r^2 < max(R_i^2, R_j^2): squaring is
        // monotone, so both compare the same rounded values
        const float2 r2 = PER ? canon_r2_x2p(sm.tc.x[q], sm.tc.y[q], sm.tc.z[q], pj.x, pj.y, pj.z, a.tree.per)
                              : canon_r2_x2(sm.tc.x[q], sm.tc.y[q], sm.tc.z[q], pj.x, pj.y, pj.z);
        const bool hit0 = r2.x < fmaxf(sm.tr2[t0], pj.w);
        const bool hit1 = r2.y < fmaxf(sm.tr2[t1], pj.w);
        const unsigned m0 = __ballot_sync(0xffffffffu, hit0);
        const unsigned m1 = __ballot_sync(0xffffffffu, hit1);
        // past CAP hits the last entry is overwritten: such a list is
        // discarded (its length is set to -1) anyway.  Stores kept in L2 (the
        // density pass reads the last groups' lists first).
        if (hit0) __stcg(tbase + t0 * CAP + min(len[t0] + __popc(m0 & lt), CAP - 1), j);
        if (hit1) __stcg(tbase + t1 * CAP + min(len[t1] + __popc(m1 & lt), CAP - 1), j);
        len[t0] += __popc(m0);
        len[t1] += __popc(m1);
    }
}

// The lists of a batch of targets (sm.tc, sm.tr2, box [sm.blo, sm.bhi],
// largest (list radius factor x h_i)^2 sm.bhi.w) from the group's candidate slots,
// 32 per chunk (one per lane; the next chunk's candidates are loaded while
// one is handled).  A candidate enters the queue only if it is within
// max(its own list radius, the batch's largest) of the batch box: a
// candidate that hits a target is always that close (the box test rounds to
// the conservative side within kOpenSlack), so the lists are the same as
// from testing every candidate against every target, with fewer tests when
// the batch is smaller than the group or h varies across the group.  Every
// 32 queued candidates are tested against the batch's targets.  Returns the
// list length of target `lane` (lane < TB).  PER: nearest images on the
// periodic axes.
template <int TB, bool PER, int CAP>
__device__ __forceinline__ int test_chunks(const NlistArgs &a, NlistSmem &sm, int ncand, int i0)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    int len[TB];
#pragma unroll
    for (int tt = 0; tt < TB; ++tt) len[tt] = 0;
    int *const tbase = a.idx + (size_t)i0 * CAP;  // the batch's first list
    int qn = 0;  // queued candidates
    int r = 0;
    int jn = lane < ncand ? slot_particle(sm.runs, r, lane) : -1;
    float4 pn = jn >= 0 ? __ldg(&a.pos[jn]) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
    float hn = jn >= 0 ? __ldg(&a.h[jn]) : 0.f;
    for (int c0 = 0;;) {
        if (c0 < ncand) {  // the chunk's candidates near the batch box into the queue
            const int k = c0 + lane;
            const int j = jn;
            const float4 pj = pn;
            const float rj = a.rscale * hn;
            const float rj2 = rj * rj;
            if (c0 + 32 < ncand) {
                jn = k + 32 < ncand ? slot_particle(sm.runs, r, k + 32) : -1;
                pn = jn >= 0 ? __ldg(&a.pos[jn]) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                hn = jn >= 0 ? __ldg(&a.h[jn]) : 0.f;
            }
            const float4 blo = sm.blo, bhi = sm.bhi;
            const bool keep = j >= 0 && box_dist2_c<PER>(a.tree, blo, bhi, pj, pj) < fmaxf(bhi.w, rj2) * kOpenSlack;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int slot = qn + __popc(m & lt);
                sm.u.q.p[slot] = make_float4(pj.x, pj.y, pj.z, rj2);
                sm.u.q.j[slot] = j;
            }
            qn += __popc(m);
            c0 += 32;
            __syncwarp();
        }
        const bool last = c0 >= ncand;
        if (qn >= 32 || (last && qn > 0)) {
            const int cnt = min(qn, 32);
            test_queued<TB, PER, CAP>(a, sm, cnt, tbase, len);
            // the rest (fewer than 32) to the front of the queue
            const int rest = qn - cnt;
            float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
            int jv = 0;
            if (lane < rest) {
                pv = sm.u.q.p[32 + lane];
                jv = sm.u.q.j[32 + lane];
            }
            __syncwarp();
            if (lane < rest) {
                sm.u.q.p[lane] = pv;
                sm.u.q.j[lane] = jv;
            }
            __syncwarp();
            qn = rest;
        }
        if (last && qn == 0) break;
    }
    int mine = 0;
#pragma unroll
    for (int tt = 0; tt < TB; ++tt)
        if (lane == tt) mine = len[tt];
    return mine;
}

// CAP: the lists' stride (list_cap of their kernel), a constant so that the
// hit stores' addresses need no multiplication
template <bool PER, int CAP>
__global__ void __launch_bounds__(kNlWarps * 32, 7) nlist_kernel(NlistArgs a)
{
    __shared__ NlistSmem smv[kNlWarps];
    NlistSmem &sm = smv[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lane_lt();
    const int ng = a.sizes[SZ_GROUPS];
    if (a.gate && *a.gate == 0) return;  // relist mode, nothing outgrew its pad
    // per-warp tallies (32 bits: a warp's share of a launch stays far below 2^32)
    unsigned n_cand = 0, n_entries = 0, n_over = 0;

    while (true) {
        // kSG groups at a time, kSG / 2 in the last quarter (shorter tail);
        // with a due mask (block steps) kSG / 2 throughout: the due groups are
        // few and clustered, and smaller grabs spread them over more warps
        int gf = 0, grab = kSG;
        if (lane == 0) {
            grab = a.active || *(volatile int *)a.work >= ng - (ng >> 2) ? kSG / 2 : kSG;
            gf = atomicAdd(a.work, grab);
        }
        gf = __shfl_sync(0xffffffffu, gf, 0);
        grab = __shfl_sync(0xffffffffu, grab, 0);
        if (gf >= ng) break;
        const int sgn = min(grab, ng - gf);
        const bool have = lane < sgn;
        const int2 grl = have ? a.grp_ref[gf + lane] : make_int2(0, 0);
        const float hml = have ? a.grp_lo[gf + lane].w : 0.f;  // the group's h_max
        const int ins = a.inst && have ? a.inst[grl.x] : 0;
        // a group starts a new run unless it is of the same instance as the
        // previous one and their h_max agree within kShareH
        const int ins_p = __shfl_up_sync(0xffffffffu, ins, 1);
        const float hm_p = __shfl_up_sync(0xffffffffu, hml, 1);
        const bool starts = have && (lane == 0 || ins != ins_p || hml > kShareH * hm_p ||
                                     hm_p > kShareH * hml);
        const unsigned bstart = __ballot_sync(0xffffffffu, starts);
        // with a due-target mask (block steps): the groups holding a due target
        unsigned bdue = 0xffffffffu;
        if (a.active) {
            bool due = false;
            if (have)
                for (int k = 0; k < grl.y && !due; ++k) due = a.active[grl.x + k] != 0;
            bdue = __ballot_sync(0xffffffffu, due);
        }
        for (int s = 0; s < sgn;) {
            const unsigned later = bstart & ~((2u << s) - 1u);  // starts after s
            int e = later ? min(__ffs(later) - 1, sgn) : sgn;
            const int root = __shfl_sync(0xffffffffu, ins, s);
            if (a.only_bad && a.only_bad[root] == 0) {  // relist mode: this instance's lists hold
                s = e;
                continue;
            }
            const unsigned run = (e >= 32 ? 0xffffffffu : ((1u << e) - 1u)) & ~((1u << s) - 1u);
            if ((bdue & run) == 0) {  // no group of the run is due: no walk
                s = e;
                continue;
            }
            // One walk for the groups [s, e) of the run; while its leaves do
            // not fit, the range is halved (a group alone that does not fit
            // gets no lists), so whether a group gets lists depends on the
            // group alone.
            int nshared;
            while (true) {
                const bool mine = lane >= s && lane < e;
                float4 ulo = mine ? a.grp_lo[gf + lane] : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
                float4 uhi = mine ? a.grp_hi[gf + lane] : make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
                for (int o = 16; o > 0; o >>= 1) {
                    ulo.x = fminf(ulo.x, __shfl_xor_sync(0xffffffffu, ulo.x, o));
                    ulo.y = fminf(ulo.y, __shfl_xor_sync(0xffffffffu, ulo.y, o));
                    ulo.z = fminf(ulo.z, __shfl_xor_sync(0xffffffffu, ulo.z, o));
                    ulo.w = fmaxf(ulo.w, __shfl_xor_sync(0xffffffffu, ulo.w, o));  // h_max
                    uhi.x = fmaxf(uhi.x, __shfl_xor_sync(0xffffffffu, uhi.x, o));
                    uhi.y = fmaxf(uhi.y, __shfl_xor_sync(0xffffffffu, uhi.y, o));
                    uhi.z = fmaxf(uhi.z, __shfl_xor_sync(0xffffffffu, uhi.z, o));
                }
                nshared = walk_sorted<PER>(a, sm, root, ulo, uhi);
                if (nshared >= 0 || e - s == 1) break;
                e = s + (e - s + 1) / 2;
            }
            for (int gi = s; gi < e; ++gi) {
                const int g = gf + gi;
                const int2 gr = a.grp_ref[g];
                if (a.active && !__any_sync(0xffffffffu, lane < gr.y && a.active[gr.x + lane]))
                    continue;  // no target of the group is due: its lists are not read
                const float4 glo = a.grp_lo[g], ghi = a.grp_hi[g];
                const int nleaf = nshared;
                const int nrun = nleaf >= 0 ? group_candidates<PER>(a, sm, nleaf, glo, ghi, kMaxRuns) : -1;
                const bool ok = nrun >= 0;
                const int ncand = ok ? sm.runs[nrun].y : 0;
                for (int b0 = 0; b0 < gr.y; b0 += kNlTB) {
                    const int nt = min(kNlTB, gr.y - b0);
                    const int i0 = gr.x + b0;
                    // the batch's targets, their box and largest list radius
                    float4 blo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
                    float4 bhi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
                    float tr2max = 0.f;
                    if (lane < kNlTB) {
                        const float4 p = lane < nt ? a.pos[i0 + lane] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                        sm.tc.set(lane, p);
                        const float rt = lane < nt ? a.rscale * a.h[i0 + lane] : 0.f;
                        sm.tr2[lane] = rt * rt;
                        if (lane < nt) {
                            blo = make_float4(p.x, p.y, p.z, 0.f);
                            bhi = blo;
                            tr2max = rt * rt;
                        }
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        blo.x = fminf(blo.x, __shfl_xor_sync(0xffffffffu, blo.x, o));
                        blo.y = fminf(blo.y, __shfl_xor_sync(0xffffffffu, blo.y, o));
                        blo.z = fminf(blo.z, __shfl_xor_sync(0xffffffffu, blo.z, o));
                        bhi.x = fmaxf(bhi.x, __shfl_xor_sync(0xffffffffu, bhi.x, o));
                        bhi.y = fmaxf(bhi.y, __shfl_xor_sync(0xffffffffu, bhi.y, o));
                        bhi.z = fmaxf(bhi.z, __shfl_xor_sync(0xffffffffu, bhi.z, o));
                        tr2max = fmaxf(tr2max, __shfl_xor_sync(0xffffffffu, tr2max, o));
                    }
                    if (lane == 0) {
                        sm.blo = blo;
                        sm.bhi = make_float4(bhi.x, bhi.y, bhi.z, tr2max);
                    }
                    __syncwarp();
                    int mlen = 0;
                    if (ncand > 0) {
                        if (nt <= 4) mlen = test_chunks<4, PER, CAP>(a, sm, ncand, i0);
                        else if (nt <= 8) mlen = test_chunks<8, PER, CAP>(a, sm, ncand, i0);
                        else mlen = test_chunks<kNlTB, PER, CAP>(a, sm, ncand, i0);
                        n_cand += (unsigned)nt * (unsigned)ncand;
                    }
                    // a group without lists is left to the walking kernels
                    const bool fits = ok && mlen <= CAP;
                    if (lane < nt) {
                        a.len[i0 + lane] = fits ? mlen : -1;
                        n_entries += (unsigned)min(mlen, CAP);
                        n_over += fits ? 0u : 1u;
                    }
                    __syncwarp();
                }
            }
            s = e;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_entries += __shfl_xor_sync(0xffffffffu, n_entries, o);
        n_over += __shfl_xor_sync(0xffffffffu, n_over, o);
    }
    if (lane == 0) {
        atomicAdd(&a.counters[C_DENS_CAND], (unsigned long long)n_cand);  // candidate x target tests
        atomicAdd(&a.counters[C_LIST_ENTRIES], (unsigned long long)n_entries);
        atomicAdd(&a.counters[C_LIST_OVERFLOW], (unsigned long long)n_over);
    }
}

static cudaError_t configure_nlist(int &blocks)
{
    static std::mutex mu;  // first calls may come from several host threads
    std::lock_guard<std::mutex> lock(mu);
    static bool configured = false;
    static int nb_cached = 1;
    if (!configured) {  // the smallest over the variants
        const void *fns[4] = {(const void *)nlist_kernel<false, 128>, (const void *)nlist_kernel<true, 128>,
                              (const void *)nlist_kernel<false, 192>, (const void *)nlist_kernel<true, 192>};
        int nb = 1 << 30;
        for (const void *f : fns) {
            int b = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kNlWarps * 32, 0);
            if (e != cudaSuccess) return e;
            nb = b < nb ? b : nb;
        }
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

// the variant for the lists' stride and the periodicity
static cudaError_t launch_nlist(Ctx &c, const NlistArgs &a, int blocks, cudaStream_t st)
{
    static_assert(kNbrCapMax == 192, "list strides are 128 and 192");
    const dim3 grid(c.num_sms * blocks), block(kNlWarps * 32);
    const bool per = a.tree.per.any();
    if (a.cap == 128) {
        if (per) nlist_kernel<true, 128><<<grid, block, 0, st>>>(a);
        else nlist_kernel<false, 128><<<grid, block, 0, st>>>(a);
    } else if (a.cap == 192) {
        if (per) nlist_kernel<true, 192><<<grid, block, 0, st>>>(a);
        else nlist_kernel<false, 192><<<grid, block, 0, st>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static NlistArgs nlist_args(Ctx &c, const sph_state &s, const sph_params &p, float pad,
                            const Batch *batch)
{
    NlistArgs a{};
    a.pos = (const float4 *)s.pos;
    a.h = s.h;
    a.grp_ref = c.tree.grp_ref;
    a.grp_lo = c.tree.grp_lo;
    a.grp_hi = c.tree.grp_hi;
    a.sizes = c.d_sizes;
    a.work = c.d_sizes + SZ_WORK;
    a.tree = WalkTree{c.tree.node_lo, c.tree.node_hi, c.tree.node_ref, period_of(p)};
    a.inst = batch ? c.inst : nullptr;
    // the radius and capacity of the lists' kernel (a relist keeps them)
    a.rscale = kernel_support(c.nl_kernel >= 0 ? c.nl_kernel : p.kernel) * (1.f + pad) * kListSlack;
    a.cap = c.nl_stride;
    a.active = c.mask;
    a.idx = c.nl_idx;
    a.len = c.nl_len;
    a.err = c.d_err;
    a.counters = c.d_counters;
    return a;
}

cudaError_t nlist_pass(Ctx &c, const sph_state &s, const sph_params &p, float pad, cudaStream_t st,
                       const Batch *batch)
{
    int blocks = 1;
    cudaError_t e = configure_nlist(blocks);
    if (e != cudaSuccess) return e;
    NlistArgs a = nlist_args(c, s, p, pad, batch);
    e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    return launch_nlist(c, a, blocks, st);
}

cudaError_t check_list_kernel(Ctx &c, const sph_params &p, cudaStream_t st)
{
    if (c.nl_kernel == p.kernel) return cudaSuccess;
    return cudaMemsetAsync(c.tree.rec_ctl + 1, 0xff, sizeof(int), st);
}

cudaError_t relist_pass(Ctx &c, const sph_state &s, const sph_params &p, float pad, cudaStream_t st,
                        const Batch *batch)
{
    int blocks = 1;
    cudaError_t e = configure_nlist(blocks);
    if (e != cudaSuccess) return e;
    int *any = c.tree.rec_ctl;  // rec_ctl[0]: some instance outgrew its pad
    // node and group h_max of the final h (the list walk's opening test)
    e = update_hmax(c, s, p, st, any);
    if (e != cudaSuccess) return e;
    NlistArgs a = nlist_args(c, s, p, pad, batch);
    a.gate = any;
    a.only_bad = c.tree.rec_bad;
    e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    e = launch_nlist(c, a, blocks, st);
    if (e != cudaSuccess) return e;
    // the rebuilt lists cover the pair sets at the final h
    e = cudaMemsetAsync(c.tree.rec_bad, 0, sizeof(int) * (batch ? batch->n_inst : 1), st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(any, 0, sizeof(int), st);
}

}  // namespace sph
