// Tree build (Sect. 3.1): bounding box, Morton keys, radix sort, in-place
// permutation into curve order, octree chop and group chop, node bounds.
//
// Chop: the paper builds the tree level by level, splitting every curve
// section with more than N_leaf particles.  Here the same node set is found
// with O(log T) work per particle instead of one pass per level.  With d(s) the
// first level at which key[s] differs from key[s-1] (s starts a run at every
// level >= d(s)), the nodes that start at particle s are the levels
// d(s) .. Lmax(s), provided the run containing s at level d(s)-1 holds more
// than T particles; Lmax(s) = max(d(s), min(c + 1, 21)), where c is the number
// of leading 3-bit digits key[s] shares with key[s+T] (the run starting at s
// holds more than T particles exactly at the levels <= c).  A node is terminal
// at Lmax(s), so the terminal nodes (the groups, for T = N_group) start at the
// particles with any node at all.  Nodes are numbered level by level and by
// first particle inside a level, the order of the level-by-level chop.  Both
// tests reduce to window minima and maxima of the shared prefixes of
// neighbouring keys (chop_flags_kernel).
#include "sph_internal.cuh"

namespace sph {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int ord_of(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float float_of(int o)
{
    return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff);
}

// number of equal leading 3-bit digits of two 63-bit keys (0..21)
__device__ __forceinline__ int common_digits(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return kMaxLevel;
    int hb = 63 - __clzll((long long)x);
    return (62 - hb) / 3;
}

__device__ __forceinline__ uint64_t spread21(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// ------------------------------------------------------------ bbox + checks
__global__ void bbox_init_kernel(int *bb)
{
    if (threadIdx.x < 3) bb[threadIdx.x] = 0x7fffffff;           // min of ordered ints
    else if (threadIdx.x < 6) bb[threadIdx.x] = (int)0x80000000; // max
}

__global__ void bbox_kernel(const float4 *__restrict__ pos, const float *__restrict__ h, int n,
                            int *bb, int *err)
{
    int mn[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff};
    int mx[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 p = pos[i];
        float hh = h[i];
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) &&
                 isfinite(hh) && p.w > 0.f && hh > 0.f);
        int o0 = ord_of(p.x), o1 = ord_of(p.y), o2 = ord_of(p.z);
        mn[0] = min(mn[0], o0); mx[0] = max(mx[0], o0);
        mn[1] = min(mn[1], o1); mx[1] = max(mx[1], o1);
        mn[2] = min(mn[2], o2); mx[2] = max(mx[2], o2);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_NONFINITE);
    // block-level combine first: one set of 6 atomics per block
    __shared__ int sb[6][32];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            sb[a][w] = mn[a];
            sb[3 + a][w] = mx[a];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        int k = threadIdx.x, v = sb[k][0];
        for (int q = 1; q < nw; ++q) v = k < 3 ? min(v, sb[k][q]) : max(v, sb[k][q]);
        if (k < 3) atomicMin(bb + k, v); else atomicMax(bb + k, v);
    }
}

// batch: one box per instance (6 ordered ints each), warp-combined atomics
__global__ void bbox_batch_init_kernel(int *bb, int n_inst)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 6 * n_inst; k += gridDim.x * blockDim.x)
        bb[k] = (k % 6) < 3 ? 0x7fffffff : (int)0x80000000;
}

__global__ void bbox_batch_kernel(const float4 *__restrict__ pos, const float *__restrict__ h,
                                  const int *__restrict__ inst, int n, int *bb, int *err)
{
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
        int i = i0 + threadIdx.x;
        bool in = i < n;
        float4 p = in ? pos[i] : make_float4(0, 0, 0, 0);
        float hh = in ? h[i] : 1.f;
        int k = in ? inst[i] : -1;
        bool bad = in && !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) &&
                           isfinite(hh) && p.w > 0.f && hh > 0.f);
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_NONFINITE);
        int o[3] = {ord_of(p.x), ord_of(p.y), ord_of(p.z)};
        int k0 = __shfl_sync(0xffffffffu, k, 0);
        if (__all_sync(0xffffffffu, k == k0)) {  // whole warp in one instance
            int mn[3] = {o[0], o[1], o[2]}, mx[3] = {o[0], o[1], o[2]};
            for (int s = 16; s > 0; s >>= 1)
                for (int a = 0; a < 3; ++a) {
                    mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], s));
                    mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], s));
                }
            if ((threadIdx.x & 31) == 0 && k0 >= 0)
                for (int a = 0; a < 3; ++a) {
                    atomicMin(bb + 6 * k0 + a, mn[a]);
                    atomicMax(bb + 6 * k0 + 3 + a, mx[a]);
                }
        } else if (in) {
            for (int a = 0; a < 3; ++a) {
                atomicMin(bb + 6 * k + a, o[a]);
                atomicMax(bb + 6 * k + 3 + a, o[a]);
            }
        }
    }
}

// canonical FP32 quantisation, see include/sph.h
__device__ __forceinline__ void box_scale(const int *bb, float lo[3], float &s)
{
    float size = 0.f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = float_of(bb[a]);
        float e = __fsub_rn(float_of(bb[3 + a]), lo[a]);
        size = e > size ? e : size;
    }
    s = size > 0.f ? __fdiv_rn(2097152.0f, size) : 0.f;
}

// (also checks that positions lie in [plo, plo + L) on the periodic axes)
__global__ void morton_kernel(const float4 *__restrict__ pos, const int *__restrict__ inst, int n,
                              const int *bb, uint64_t *__restrict__ keys, uint32_t *__restrict__ idx,
                              Period per, float3 plo, int *err)
{
    float lo[3], s;
    box_scale(bb, lo, s);
    const float L[3] = {per.x, per.y, per.z}, pl[3] = {plo.x, plo.y, plo.z};
    bool outside = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (inst) box_scale(bb + 6 * inst[i], lo, s);
        float4 p = pos[i];
        float x[3] = {p.x, p.y, p.z};
        for (int a = 0; a < 3; ++a)
            outside |= L[a] > 0.f && !(x[a] >= pl[a] && x[a] < pl[a] + L[a]);
        uint32_t c[3];
        for (int a = 0; a < 3; ++a) {
            float t = __fmul_rn(__fsub_rn(x[a], lo[a]), s);
            uint32_t v = (uint32_t)floorf(t);
            c[a] = v > 2097151u ? 2097151u : v;
        }
        keys[i] = (spread21(c[0]) << 2) | (spread21(c[1]) << 1) | spread21(c[2]);
        idx[i] = (uint32_t)i;
    }
    if (__any_sync(0xffffffffu, outside) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_INVALID_ARG);
}

// ------------------------------------------------------------- radix sort
// Stable LSD radix sort of (key, index) with 8-bit digits.  Few particles
// share the key's top 32 bits (a cell of 2^-10 of the box per axis), so four
// passes sort by bits 32..63 and a fix-up pass orders each run of equal top
// bits by its low 32 bits; if some run is longer than kFixRun, eight passes
// over the whole word follow (they return at once otherwise).  Two
// more passes on the instance id in a batch.  The digit counts of
// every pass are taken in one histogram pass up front (the multiset of keys
// does not change between passes).  Each pass is then one kernel: tiles are
// numbered in launch order by an atomic counter, each ranks its keys (warp
// match + per-warp counts, in input order, so the sort is stable), publishes
// its per-digit counts and adds up its predecessors' counts by looking back
// through their published words (decoupled look-back), then writes its keys
// out digit run by digit run from a digit-ordered copy in shared memory.
constexpr int RS_T = 256, RS_I = 8, RS_TILE = RS_T * RS_I;
constexpr uint32_t RS_AGG = 1u << 30, RS_INC = 2u << 30, RS_CNT = RS_AGG - 1u;
constexpr int RS_SPIN = 1 << 22;  // look-back polls before giving up (error, no hang)
constexpr int RS_LB = 4;           // predecessor tiles read together in the look-back

// block-wide exclusive scan helper for 256 threads, returns the block total
__device__ __forceinline__ uint32_t block_scan_256(uint32_t v, uint32_t &excl, uint32_t *ws)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < 8 ? ws[lane] : 0;
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < 8) ws[lane] = t;
    }
    __syncthreads();
    uint32_t wbase = w > 0 ? ws[w - 1] : 0;
    uint32_t total = ws[7];
    excl = wbase + x - v;
    __syncthreads();
    return total;
}

// digit counts of all passes: ghist[p][d] for the 8 key digits and, with
// inst, the 2 instance-id digits.  Each thread counts RS_GE consecutive
// keys, adding runs of one digit with one shared atomic: the keys are nearly
// in curve order, so the high digits come in long runs, and a run that spans
// the whole warp is added once for the warp.  Four blocks per SM: each adds
// its shared counts to ghist once, which keeps the global atomics few.
constexpr int RS_GE = 8;
__global__ void __launch_bounds__(256) rs_ghist_kernel(const uint64_t *__restrict__ keys,
                                                       const int *__restrict__ inst, int n,
                                                       uint32_t *ghist)
{
    __shared__ uint32_t h[10][256];
    for (int k = threadIdx.x; k < 10 * 256; k += 256) (&h[0][0])[k] = 0;
    __syncthreads();
    const int np = inst ? 10 : 8;
    for (int b = blockIdx.x * 256 * RS_GE; b < n; b += gridDim.x * 256 * RS_GE) {
        const int s0 = b + threadIdx.x * RS_GE;
        uint32_t cur[10], cnt[10];
#pragma unroll
        for (int p = 0; p < 10; ++p) { cur[p] = 0; cnt[p] = 0; }
        for (int e = 0; e < RS_GE && s0 + e < n; ++e) {
            const uint64_t key = keys[s0 + e];
            const uint32_t iv = inst ? (uint32_t)inst[s0 + e] : 0u;
#pragma unroll
            for (int p = 0; p < 10; ++p) {
                if (p >= np) break;
                const uint32_t d = p < 8 ? (uint32_t)((key >> (8 * p)) & 255u) : (iv >> (8 * (p - 8))) & 255u;
                if (cnt[p] != 0 && d != cur[p]) {
                    atomicAdd(&h[p][cur[p]], cnt[p]);
                    cnt[p] = 0;
                }
                cur[p] = d;
                ++cnt[p];
            }
        }
#pragma unroll
        for (int p = 0; p < 10; ++p) {
            if (p >= np) break;
            const uint32_t c0 = __shfl_sync(0xffffffffu, cur[p], 0);
            if (__all_sync(0xffffffffu, cnt[p] == 0 || cur[p] == c0)) {
                const uint32_t tot = __reduce_add_sync(0xffffffffu, cnt[p]);
                if ((threadIdx.x & 31) == 0 && tot != 0) atomicAdd(&h[p][c0], tot);
            } else if (cnt[p] != 0) {
                atomicAdd(&h[p][cur[p]], cnt[p]);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < np * 256; k += 256) {
        const uint32_t v = (&h[0][0])[k];
        if (v) atomicAdd(&ghist[k], v);
    }
}

// gstart[p][d] = exclusive scan of ghist[p][.]   (block p)
__global__ void __launch_bounds__(256) rs_gscan_kernel(const uint32_t *ghist, uint32_t *gstart)
{
    __shared__ uint32_t ws[8];
    uint32_t ex;
    block_scan_256(ghist[blockIdx.x * 256 + threadIdx.x], ex, ws);
    gstart[blockIdx.x * 256 + threadIdx.x] = ex;
}

// One pass: warp w of a tile owns the contiguous keys [w * 256, (w + 1) * 256)
// of the tile and ranks them in 8 rounds of 32: the lanes holding the same
// digit are found with one ballot per digit bit, and a warp-private digit
// counter row accumulates; tile order is (warp, round, lane), so equal digits
// keep their input order.
__global__ void __launch_bounds__(RS_T, 4) rs_onesweep_kernel(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const int *__restrict__ inst, int n, int shift,
    const uint32_t *__restrict__ gstart, uint32_t *status, int *tile_counter, int *err,
    const int *gate, int spin_cap)
{
    if (gate && *gate == 0) return;  // a pass of the full sort that is not needed
    __shared__ uint32_t gbase[256];   // first output slot of each digit for this tile
    __shared__ uint32_t tstart[256];  // first slot of each digit in the sorted tile
    __shared__ uint32_t wcnt[8][256];
    __shared__ uint32_t ws[8];
    __shared__ int s_tile;
    __shared__ uint64_t skey[RS_TILE];
    __shared__ uint32_t sval[RS_TILE];
    __shared__ uint8_t sdig[RS_TILE];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1);
    uint32_t *flat = &wcnt[0][0];
#pragma unroll
    for (int k = 0; k < 8; ++k) flat[k * 256 + tid] = 0;
    __syncthreads();
    const int tile = s_tile;
    const uint32_t lt = (1u << lane) - 1u;
    const int tile0 = tile * RS_TILE;
    const int wbase = tile0 + w * (RS_TILE / 8);
    uint64_t key[RS_I];
    uint32_t val[RS_I], dig[RS_I], rank[RS_I];
#pragma unroll
    for (int r = 0; r < RS_I; ++r) {
        const int s = wbase + r * 32 + lane;
        const bool valid = s < n;
        key[r] = valid ? kin[s] : 0;
        val[r] = valid ? vin[s] : 0;
        uint32_t d = valid ? (inst ? ((uint32_t)inst[val[r]] >> shift) & 255u
                                   : (uint32_t)((key[r] >> shift) & 255u))
                           : 256u + lane;
        dig[r] = d;
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        const uint32_t old = valid ? wcnt[w][d] : 0u;
        rank[r] = old + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[w][d] = old + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t cnt;  // keys of digit tid in this tile
    {
        uint32_t acc = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            const uint32_t c = wcnt[ww][tid];
            wcnt[ww][tid] = acc;
            acc += c;
        }
        cnt = acc;
        uint32_t ex;
        block_scan_256(acc, ex, ws);  // digit starts inside the sorted tile
        tstart[tid] = ex;
    }
    // publish this tile's count of digit tid, then add up the predecessors'
    volatile uint32_t *st = status;
    st[(size_t)tile * 256 + tid] = (tile == 0 ? RS_INC : RS_AGG) | cnt;
    // predecessors are read RS_LB at a time, so a long look-back costs one
    // memory latency per RS_LB tiles; tiles before tile 0 count as inclusive zeros
    uint32_t excl = 0;
    bool done = tile == 0;
    for (int t0 = tile - 1; !done; t0 -= RS_LB) {
        uint32_t v[RS_LB];
#pragma unroll
        for (int k = 0; k < RS_LB; ++k)
            v[k] = t0 - k >= 0 ? (uint32_t)st[(size_t)(t0 - k) * 256 + tid] : (uint32_t)(RS_INC + 0u);
#pragma unroll
        for (int k = 0; k < RS_LB; ++k) {
            if (done) break;
            int spin = 0;
            while ((v[k] & ~RS_CNT) == 0u) {
                if (++spin > spin_cap) {  // a predecessor never published: report, do not hang
                    raise_error(err, SPH_ERR_TIMEOUT);
                    v[k] = RS_INC;
                    break;
                }
                __nanosleep(32);
                v[k] = st[(size_t)(t0 - k) * 256 + tid];
            }
            excl += v[k] & RS_CNT;
            done = (v[k] & RS_INC) != 0u;
        }
    }
    if (tile > 0) st[(size_t)tile * 256 + tid] = RS_INC | (excl + cnt);
    gbase[tid] = gstart[tid] + excl;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_I; ++r) {
        if (wbase + r * 32 + lane < n) {
            const uint32_t d = dig[r];
            const uint32_t lp = tstart[d] + wcnt[w][d] + rank[r];
            skey[lp] = key[r];
            sval[lp] = val[r];
            sdig[lp] = (uint8_t)d;
        }
    }
    __syncthreads();
    const int valid_n = min(RS_TILE, n - tile0);
    for (int i = tid; i < valid_n; i += RS_T) {
        const uint32_t d = sdig[i];
        const uint32_t pos = gbase[d] + (uint32_t)i - tstart[d];
        kout[pos] = skey[i];
        vout[pos] = sval[i];
    }
}

// Runs of keys with equal bits 32..63 (after the passes on those bits, in
// input order) sorted by their low 32 bits: one thread per run, stable
// insertion sort.  A run longer than kFixRun raises *full instead.  Threads
// that are not at a run's start read only the top bits of their neighbours,
// which the sort inside a run does not change.
constexpr int kFixRun = 32;
__global__ void rs_fixup_kernel(uint64_t *keys, uint32_t *vals, int n, int *full)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint64_t top = keys[s] >> 32;
        if (s > 0 && (keys[s - 1] >> 32) == top) continue;        // inside a run
        if (s + 1 >= n || (keys[s + 1] >> 32) != top) continue;   // a run of one
        int e = s + 2;
        while (e < n && e - s <= kFixRun && (keys[e] >> 32) == top) ++e;
        if (e - s > kFixRun) {
            atomicOr(full, 1);
            continue;
        }
        for (int i = s + 1; i < e; ++i) {
            const uint64_t k = keys[i];
            const uint32_t v = vals[i];
            int j = i - 1;
            while (j >= s && (uint32_t)keys[j] > (uint32_t)k) {
                keys[j + 1] = keys[j];
                vals[j + 1] = vals[j];
                --j;
            }
            keys[j + 1] = k;
            vals[j + 1] = v;
        }
    }
}

// ------------------------------------------------------------------ gather
struct GatherArgs {
    const uint32_t *order;
    float4 *a4[4];
    float4 *t4[4];
    float *a1[5];
    float *t1[5];
    uint32_t *perm, *tperm;
    float4 *rec;  // a4[0], a4[1] (pos, vel) side by side, or nullptr
    const uint64_t *keys_sorted;  // if not null: copied to keys_out
    uint64_t *keys_out;
    int n4, n1;
};

__global__ void gather_kernel(GatherArgs g, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        uint32_t o = g.order[k];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (a < g.n4) {
                const float4 v = g.a4[a][o];
                g.t4[a][k] = v;
                if (a < 2 && g.rec) g.rec[2 * (size_t)k + a] = v;
            }
        }
#pragma unroll
        for (int a = 0; a < 5; ++a)
            if (a < g.n1) g.t1[a][k] = g.a1[a][o];
        g.tperm[k] = g.perm[o];
        if (g.keys_sorted) g.keys_out[k] = g.keys_sorted[k];
    }
}

// -------------------------------------------------------------------- scan
constexpr int SC_T = 256, SC_I = 8, SC_CHUNK = SC_T * SC_I;

__device__ __forceinline__ int scan_in(const int *in, int i, int n, int mode)
{
    if (i >= n) return 0;
    int v = in[i];
    return mode == 0 ? v : (v >= 0 ? 1 : 0);
}

__global__ void __launch_bounds__(SC_T) scan_reduce_kernel(const int *in, int n, int mode, int *part)
{
    __shared__ uint32_t ws[8];
    int base = blockIdx.x * SC_CHUNK + threadIdx.x * SC_I;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SC_I; ++k) s += scan_in(in, base + k, n, mode);
    uint32_t ex;
    uint32_t tot = block_scan_256((uint32_t)s, ex, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = (int)tot;
}

__global__ void __launch_bounds__(SC_T) scan_part_kernel(int *part, int nb, int *total)
{
    __shared__ uint32_t ws[8];
    uint32_t carry = 0;
    for (int b = 0; b < nb; b += SC_T) {
        int i = b + threadIdx.x;
        uint32_t v = i < nb ? (uint32_t)part[i] : 0, ex;
        uint32_t tot = block_scan_256(v, ex, ws);
        if (i < nb) part[i] = (int)(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = (int)carry;
}

__global__ void __launch_bounds__(SC_T) scan_down_kernel(const int *in, int *out, int n, int mode,
                                                         const int *part)
{
    __shared__ uint32_t ws[8];
    int base = blockIdx.x * SC_CHUNK + threadIdx.x * SC_I;
    int v[SC_I], s = 0;
#pragma unroll
    for (int k = 0; k < SC_I; ++k) { v[k] = scan_in(in, base + k, n, mode); s += v[k]; }
    uint32_t ex;
    block_scan_256((uint32_t)s, ex, ws);
    int run = part[blockIdx.x] + (int)ex;
#pragma unroll
    for (int k = 0; k < SC_I; ++k)
        if (base + k < n) { out[base + k] = run; run += v[k]; }
}

// mode 0: out[i] = sum_{k<i} in[k]; mode 1: counts in[k] >= 0
static cudaError_t scan_mode(Ctx &c, const int *in, int *out, int n, int mode, int *total_dev,
                             cudaStream_t st)
{
    int nb = div_up(n, SC_CHUNK);
    if (nb < 1) nb = 1;
    if (nb > c.scan_part_cap) return cudaErrorInvalidValue;
    scan_reduce_kernel<<<nb, SC_T, 0, st>>>(in, n, mode, c.scan_part);
    scan_part_kernel<<<1, SC_T, 0, st>>>(c.scan_part, nb, total_dev);
    scan_down_kernel<<<nb, SC_T, 0, st>>>(in, out, n, mode, c.scan_part);
    return cudaGetLastError();
}

cudaError_t scan_exclusive_int(Ctx &c, const int *in, int *out, int n, int *total_dev,
                               cudaStream_t st)
{
    return scan_mode(c, in, out, n, 0, total_dev, st);
}

// -------------------------------------------------------------------- chop
// Shared leading digits of the keys of slots a and b; -1 when the slots
// belong to different instances of a batch (inst != nullptr): instances never
// share a node, each has its own root at level 0.
__device__ __forceinline__ int cd_slots(const uint64_t *__restrict__ keys,
                                        const int *__restrict__ inst, int a, int b)
{
    if (inst && inst[a] != inst[b]) return -1;
    return common_digits(keys[a], keys[b]);
}

// Node starts of the chop with threshold T: lv[s] = d | (Lmax << 8) if the
// nodes of levels d..Lmax start at slot s, else -1.  With
//   b[z] = cd(z - 1, z)    (-1 at slot 0, at an instance boundary and past
//                           the last slot),
// sorted keys give cd(x, y) = min(b[x+1 .. y]) for x < y, so
//   q[x] = cd(x, x + T) = min(b[x+1 .. x+T])      (-1 if x + T >= n).
// Slot s with 0 <= b[s] < kMaxLevel starts a cell of level d = b[s] + 1
// inside the cell P of level b[s] that holds s - 1 and s; the cell is a node
// iff P has more than T slots (P is split), i.e. iff q[x] >= b[s] for some x
// in [s - T, s] (then x and x + T lie in one cell of level b[s], which holds
// s, so it is P; conversely the first slot of P, or s - T, is such an x).
// Its descendants starting at s are nodes down to the first one with at most
// T slots: Lmax = max(d, min(q[s] + 1, kMaxLevel)).  b[s] = -1 is a root
// (d = 0), b[s] = kMaxLevel a key equal to the previous one (no node).
//
// One block per tile of kCfTile slots, with halos of kCfHalo > T slots on
// both sides in shared memory (one byte per slot); the window minima and
// maxima by doubling.
constexpr int kCfTile = 2048, kCfHalo = 65, kCfR = kCfTile + 2 * kCfHalo;

// dst[i] = min (or max) of src[i + off .. i + off + len - 1] for i in [lo, hi);
// needs lo + off >= 0 and hi + off + len <= kCfR, and reads src only there.
// t0, t1: scratch.
template <bool MAX>
__device__ __forceinline__ void cf_window(const signed char *src, signed char *dst, signed char *t0,
                                          signed char *t1, int lo, int hi, int off, int len)
{
    // cur[j] = op(src[j .. j + w - 1]) for j in [lo + off, hi + off + len - w)
    const signed char *cur = src;
    signed char *out = t0;
    int w = 1;
    while (2 * w <= len) {
        for (int j = lo + off + threadIdx.x; j < hi + off + len - 2 * w; j += blockDim.x) {
            const int a = cur[j], b = cur[j + w];
            out[j] = (signed char)(MAX ? max(a, b) : min(a, b));
        }
        __syncthreads();
        cur = out;
        out = out == t0 ? t1 : t0;
        w *= 2;
    }
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int a = cur[i + off], b = cur[i + off + len - w];  // two windows of w cover len
        dst[i] = (signed char)(MAX ? max(a, b) : min(a, b));
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) chop_flags_kernel(const uint64_t *__restrict__ keys,
                                                         const int *__restrict__ inst, int n,
                                                         int t_leaf, int t_group, int *lv_tree,
                                                         int *lv_grp)
{
    // local index i <-> slot t0 - kCfHalo + i
    __shared__ signed char sb[kCfR], sq[kCfR], sm[kCfR], s0[kCfR], s1[kCfR];
    const int ntile = (n + kCfTile - 1) / kCfTile;
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int t0 = tile * kCfTile;
        for (int i = threadIdx.x; i < kCfR; i += blockDim.x) {
            const int x = t0 - kCfHalo + i;
            sb[i] = (signed char)(x <= 0 || x >= n ? -1 : cd_slots(keys, inst, x - 1, x));
        }
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            const int T = pass == 0 ? t_leaf : t_group;
            int *lv = pass == 0 ? lv_tree : lv_grp;
            if (pass == 0 || t_group != t_leaf) {
                // q over [-T, kCfTile) relative to t0, then the maxima over [s - T, s]
                cf_window<false>(sb, sq, s0, s1, kCfHalo - T, kCfHalo + kCfTile, 1, T);
                cf_window<true>(sq, sm, s0, s1, kCfHalo, kCfHalo + kCfTile, -T, T + 1);
            }
            for (int k = threadIdx.x; k < kCfTile && t0 + k < n; k += blockDim.x) {
                const int i = kCfHalo + k;
                const int bs = sb[i], qs = sq[i];
                int v;
                if (bs < 0) v = max(0, min(qs + 1, kMaxLevel)) << 8;  // root
                else if (bs == kMaxLevel || sm[i] < bs) v = -1;
                else v = (bs + 1) | (max(bs + 1, min(qs + 1, kMaxLevel)) << 8);
                lv[t0 + k] = v;
            }
            __syncthreads();  // sq, sm and (next tile) sb are rewritten next
        }
    }
}

// The node levels [d, lm] that start at the slots of warp w of a 256-thread
// block: warp w owns the block's slots [w * 128, (w + 1) * 128), 4 per lane,
// slot base + 32 r + lane for r = 0..3 (no node: an empty range).  Returns
// the range of levels over the warp in [wlo, whi] (wlo > whi if none).
constexpr int kCwR = kChopBlock / 256;
__device__ __forceinline__ int chop_warp_levels(const int *__restrict__ lv, int n, int base,
                                                int (&d)[kCwR], int (&lm)[kCwR], int &whi)
{
    const int lane = threadIdx.x & 31;
    int dmin = kLevels, lmx = -1;
#pragma unroll
    for (int r = 0; r < kCwR; ++r) {
        const int s = base + 32 * r + lane;
        const int v = s < n ? lv[s] : -1;
        d[r] = v >= 0 ? (v & 0xff) : kLevels;
        lm[r] = v >= 0 ? (v >> 8) : -1;
        dmin = min(dmin, d[r]);
        lmx = max(lmx, lm[r]);
    }
    whi = __reduce_max_sync(0xffffffffu, lmx);
    return __reduce_min_sync(0xffffffffu, dmin);
}

// per block of kChopBlock particles: number of nodes per level
__global__ void __launch_bounds__(256) chop_count_kernel(const int *__restrict__ lv, int n,
                                                         int *blk_cnt, int nb)
{
    __shared__ int cnt[kLevels];
    if (threadIdx.x < kLevels) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int d[kCwR], lm[kCwR], whi;
    const int wlo = chop_warp_levels(lv, n, blockIdx.x * kChopBlock + w * 32 * kCwR, d, lm, whi);
    for (int L = wlo; L <= whi; ++L) {
        int c = 0;
#pragma unroll
        for (int r = 0; r < kCwR; ++r) c += __popc(__ballot_sync(0xffffffffu, d[r] <= L && L <= lm[r]));
        if (lane == 0 && c != 0) atomicAdd(&cnt[L], c);
    }
    __syncthreads();
    if (threadIdx.x < kLevels) blk_cnt[threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Node k of level L gets index level offset + its rank among the level-L
// nodes in slot order: per warp and level the count, one scan over the
// warps, then per warp and level the ballots again for the ranks.
__global__ void __launch_bounds__(256) chop_write_kernel(const int *__restrict__ lv, int n,
                                                         const int *__restrict__ blk_off, int nb,
                                                         Tree t, int *err)
{
    __shared__ int wcnt[kLevels][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int base = blockIdx.x * kChopBlock + w * 32 * kCwR;
    int d[kCwR], lm[kCwR], whi;
    const int wlo = chop_warp_levels(lv, n, base, d, lm, whi);
    if (lane < kLevels) wcnt[lane][w] = 0;
    __syncwarp();
    for (int L = wlo; L <= whi; ++L) {
        int c = 0;
#pragma unroll
        for (int r = 0; r < kCwR; ++r) c += __popc(__ballot_sync(0xffffffffu, d[r] <= L && L <= lm[r]));
        if (lane == 0) wcnt[L][w] = c;
    }
    __syncthreads();
    if (threadIdx.x < kLevels) {  // exclusive scan over the warps from the block's offset
        int acc = blk_off[threadIdx.x * nb + blockIdx.x];
        for (int ww = 0; ww < 8; ++ww) {
            const int cc = wcnt[threadIdx.x][ww];
            wcnt[threadIdx.x][ww] = acc;
            acc += cc;
        }
    }
    __syncthreads();
    for (int L = wlo; L <= whi; ++L) {
        int off = wcnt[L][w];
#pragma unroll
        for (int r = 0; r < kCwR; ++r) {
            const bool on = d[r] <= L && L <= lm[r];
            const unsigned b = __ballot_sync(0xffffffffu, on);
            if (on) {
                const int idx = off + __popc(b & lt);
                if (idx < t.cap_nodes) {
                    t.node_first[idx] = base + 32 * r + lane;
                    t.node_level[idx] = L;
                    t.node_arrive[idx] = 0;
                } else {
                    raise_error(err, SPH_ERR_NOMEM);
                }
            }
            off += __popc(b);
        }
    }
}

__global__ void level_start_kernel(const int *blk_off, int nb, const int *total, Tree t,
                                   int *sizes)
{
    int L = threadIdx.x;
    if (L < kLevels) t.level_start[L] = blk_off[L * nb];
    if (L == kLevels) {
        t.level_start[kLevels] = *total;
        sizes[SZ_NODES] = min(*total, t.cap_nodes);
    }
}

// end of the run at level L that starts at s (galloping search).  The
// root run of a batch instance is its slots (the sort keeps each instance's
// slots together), found from the instance ids, so the tree stays inside
// [0, n) whatever the caller's offsets hold.
__device__ int run_end(const uint64_t *__restrict__ keys, const int *__restrict__ inst, int n, int s,
                       int L)
{
    if (L == 0 && !inst) return n;
    int step = 1, lo = s;  // slot lo is in the run
    while (s + step < n && cd_slots(keys, inst, s + step, s) >= L) {
        lo = s + step;
        step <<= 1;
    }
    int hi = min(s + step, n);  // slot hi is not in the run (or hi == n)
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (cd_slots(keys, inst, mid, s) >= L) lo = mid; else hi = mid;
    }
    return hi;
}

__global__ void node_finish_kernel(const uint64_t *__restrict__ keys, const int *__restrict__ inst,
                                   int n, int T, Tree t, const int *sizes)
{
    int nn = sizes[SZ_NODES];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
        int L = t.node_level[k], s = t.node_first[k];
        int cnt = run_end(keys, inst, n, s, L) - s;
        t.node_count[k] = cnt;
        if (L == 0) t.node_parent[k] = -1;
        int cf = -1, nc = 0;
        if (cnt > T && L < kMaxLevel) {
            int lo = t.level_start[L + 1], hi = min(t.level_start[L + 2], nn);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (t.node_first[mid] < s) lo = mid + 1; else hi = mid;
            }
            cf = lo;
            int e = min(t.level_start[L + 2], nn);
            while (cf + nc < e && t.node_first[cf + nc] < s + cnt) {
                t.node_parent[cf + nc] = k;
                ++nc;
            }
        }
        t.node_child[k] = cf;
        t.node_nchild[k] = nc;
        t.node_ref[k] = nc > 0 ? make_int2(cf, -nc) : make_int2(s, cnt);
    }
}

// Bottom-up bounds: leaves from particles, parents from children; the last
// child to finish (arrival counter, reset by that child) computes its parent.
// gate != nullptr: do nothing unless *gate != 0.  what = 0: AABB of
// positions and h_max; what = 1: h_max only.
__global__ void node_bounds_kernel(const float4 *__restrict__ pos, const float *__restrict__ h,
                                   Tree t, const int *sizes, int what, const int *gate)
{
    if (gate && *gate == 0) return;
    int nn = sizes[SZ_NODES];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
        if (t.node_nchild[k] != 0) continue;
        int s = t.node_first[k], e = s + t.node_count[k];
        if (what == 0) {
            float3 lo = make_float3(INFINITY, INFINITY, INFINITY);
            float3 hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
            float hm = 0.f;
            for (int i = s; i < e; ++i) {
                float4 p = pos[i];
                lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
                hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
                hm = fmaxf(hm, h[i]);
            }
            t.node_lo[k] = make_float4(lo.x, lo.y, lo.z, hm);
            t.node_hi[k] = make_float4(hi.x, hi.y, hi.z, 0.f);
        } else {
            float hm = 0.f;
            for (int i = s; i < e; ++i) hm = fmaxf(hm, h[i]);
            t.node_lo[k].w = hm;
        }
        int cur = k;
        while (true) {
            int p = t.node_parent[cur];
            if (p < 0) break;
            __threadfence();
            int old = atomicAdd(&t.node_arrive[p], 1);
            if (old != t.node_nchild[p] - 1) break;
            t.node_arrive[p] = 0;  // the last child: ready for the next pass
            __threadfence();
            int cf = t.node_child[p], nc = t.node_nchild[p];
            if (what == 0) {
                float3 lo = make_float3(INFINITY, INFINITY, INFINITY);
                float3 hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
                float hm = 0.f;
                for (int q = cf; q < cf + nc; ++q) {
                    float4 a = __ldcg(&t.node_lo[q]), b = __ldcg(&t.node_hi[q]);
                    lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
                    hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
                    hm = fmaxf(hm, a.w);
                }
                __stcg(&t.node_lo[p], make_float4(lo.x, lo.y, lo.z, hm));
                __stcg(&t.node_hi[p], make_float4(hi.x, hi.y, hi.z, 0.f));
            } else {
                float hm = 0.f;
                for (int q = cf; q < cf + nc; ++q) hm = fmaxf(hm, __ldcg(&t.node_lo[q].w));
                __stcg(&t.node_lo[p].w, hm);
            }
            cur = p;
        }
    }
}

// groups: first particle of each terminal node of the group chop
__global__ void group_write_kernel(const int *__restrict__ lv_grp, const int *__restrict__ gidx,
                                   int n, Tree t)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        if (lv_grp[s] >= 0) t.grp_ref[gidx[s]] = make_int2(s, 0);
}

// what = 0: count + AABB (h_max too); what = 1: h_max only
__global__ void group_bounds_kernel(const float4 *__restrict__ pos, const float *__restrict__ h,
                                    int n, Tree t, const int *sizes, int what, const int *gate)
{
    if (gate && *gate == 0) return;
    int ng = sizes[SZ_GROUPS];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        int s = t.grp_ref[g].x;
        int e = g + 1 < ng ? t.grp_ref[g + 1].x : n;
        float hm = 0.f;
        if (what == 0) {
            float3 lo = make_float3(INFINITY, INFINITY, INFINITY);
            float3 hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
            for (int i = s; i < e; ++i) {
                float4 p = pos[i];
                lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
                hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
                hm = fmaxf(hm, h[i]);
            }
            t.grp_ref[g].y = e - s;
            t.grp_lo[g] = make_float4(lo.x, lo.y, lo.z, hm);
            t.grp_hi[g] = make_float4(hi.x, hi.y, hi.z, 0.f);
        } else {
            for (int i = s; i < e; ++i) hm = fmaxf(hm, h[i]);
            t.grp_lo[g].w = hm;
        }
    }
}

// inst[k] = instance owning slot k (offsets ascending, every instance non-empty)
// *bad = 1 (and SPH_ERR_INVALID_ARG) unless 0 = offs[0] < offs[1] < ... <
// offs[n_inst] = n (one block)
__global__ void offsets_check_kernel(const int64_t *__restrict__ offs, int n_inst, int n, int *bad, int *err)
{
    bool b = false;
    for (int k = threadIdx.x; k <= n_inst; k += blockDim.x)
        b |= k == 0 ? offs[0] != 0
           : k == n_inst ? offs[k] != (int64_t)n || offs[k - 1] >= offs[k]
                         : offs[k - 1] >= offs[k];
    b = __syncthreads_or(b);
    if (threadIdx.x == 0) {
        *bad = b ? 1 : 0;
        if (b) raise_error(err, SPH_ERR_INVALID_ARG);
    }
}

// inst[k] = the instance of particle k (caller order).  With offsets that
// failed their check, instance i < n_inst - 1 gets particle i alone and the
// last one the rest (n >= n_inst): every instance keeps a particle, so the
// instances' roots are the first n_inst nodes as the walks assume, and no
// kernel leaves the state's slots.
__global__ void instance_map_kernel(const int64_t *__restrict__ offs, int n_inst, int n, const int *bad,
                                    int *inst)
{
    const bool valid = *bad == 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (!valid) {
            inst[k] = min(k, n_inst - 1);
            continue;
        }
        int lo = 0, hi = n_inst - 1;  // largest i with offs[i] <= k
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= k) lo = mid; else hi = mid - 1;
        }
        inst[k] = lo;
    }
}

// ------------------------------------------------------------- host driver
static int grid_for(const Ctx &c, int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)c.num_sms * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

#define SPH_TRY(x)                                  \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

cudaError_t instance_map(Ctx &c, const int64_t *d_offsets, int n_inst, int n, cudaStream_t st)
{
    int *bad = c.d_sizes + SZ_BAD_OFFSETS;
    offsets_check_kernel<<<1, 1024, 0, st>>>(d_offsets, n_inst, n, bad, c.d_err);
    instance_map_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(d_offsets, n_inst, n, bad, c.inst);
    return cudaGetLastError();
}

cudaError_t refit_tree(Ctx &c, const sph_state &s, cudaStream_t st)
{
    const int n = (int)s.n;
    Tree &t = c.tree;
    const float4 *pos = (const float4 *)s.pos;
    group_bounds_kernel<<<grid_for(c, n, 128), 128, 0, st>>>(pos, s.h, n, t, c.d_sizes, 0, nullptr);
    node_bounds_kernel<<<grid_for(c, t.cap_nodes, 128), 128, 0, st>>>(pos, s.h, t, c.d_sizes, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t build_tree(Ctx &c, const sph_state &s, const sph_params &p, bool full_permute,
                       cudaStream_t st, const Batch *batch)
{
    const int n = (int)s.n;
    Tree &t = c.tree;
    float4 *pos = (float4 *)s.pos;
    const int *inst = batch ? c.inst : nullptr;
    int *bb = batch ? c.bbox_inst : (int *)c.bbox;
    // Within a step (full_permute = false) kick_drift has left the kicked pos,
    // vel, v_half, h and perm in the temporaries: keys come from there and
    // the gather writes the state straight back in curve order.
    const bool kicked = !full_permute;
    float4 *pos_in = kicked ? c.tmp4[0] : pos;
    const float *h_in = kicked ? c.tmp1[0] : s.h;
    // 1. bounding box (per instance in a batch) and input checks
    if (batch) {
        bbox_batch_init_kernel<<<div_up(6 * batch->n_inst, 256), 256, 0, st>>>(bb, batch->n_inst);
        bbox_batch_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(pos_in, h_in, inst, n, bb, c.d_err);
    } else {
        bbox_init_kernel<<<1, 32, 0, st>>>(bb);
        bbox_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(pos_in, h_in, n, bb, c.d_err);
    }
    // 2. keys
    morton_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(pos_in, inst, n, bb, s.keys, c.idx_a,
                                                      period_of(p), box_lo_of(p), c.d_err);
    // 3. radix sort (key, slot); a batch adds stable passes on the instance id,
    //    which puts every instance back on its own slots
    const int ntiles = div_up(n, RS_TILE);
    uint64_t *kin = s.keys, *kout = c.keys_alt;
    uint32_t *vin = c.idx_a, *vout = c.idx_b;
    const int ndigit = batch ? 10 : 8;  // digits 0..7 of the key, 8..9 of the instance id
    const int nslot = 4 + 8 + (batch ? 2 : 0);
    int *full = c.rs_tiles + kRsSlots;  // the fix-up found a long run: sort all 64 bits
    // digit counts of all passes, their scans, fresh look-back words, tile counters, flag
    SPH_TRY(cudaMemsetAsync(c.rs_ghist, 0, sizeof(uint32_t) * 10 * 256, st));
    SPH_TRY(cudaMemsetAsync(c.rs_tiles, 0, sizeof(int) * (kRsSlots + 1), st));
    SPH_TRY(cudaMemsetAsync(c.rs_status, 0, sizeof(uint32_t) * 256 * (size_t)ntiles * nslot, st));
    const int gh_grid = (int)std::max<int64_t>(1, std::min<int64_t>(div_up(n, 256 * RS_GE), 4 * (int64_t)c.num_sms));
    rs_ghist_kernel<<<gh_grid, 256, 0, st>>>(kin, inst, n, c.rs_ghist);
    rs_gscan_kernel<<<ndigit, 256, 0, st>>>(c.rs_ghist, c.rs_gstart);
    int slot = 0;
    auto pass = [&](int digit, const int *gate) {
        const int *dinst = digit >= 8 ? inst : nullptr;
        const int shift = digit >= 8 ? 8 * (digit - 8) : 8 * digit;
        rs_onesweep_kernel<<<ntiles, RS_T, 0, st>>>(kin, vin, kout, vout, dinst, n, shift,
                                                    c.rs_gstart + 256 * digit,
                                                    c.rs_status + (size_t)256 * ntiles * slot,
                                                    c.rs_tiles + slot, c.d_err, gate, RS_SPIN);
        ++slot;
        std::swap(kin, kout);  // a gated pass that returns moves nothing, but
        std::swap(vin, vout);  // the gated passes come in an even number
    };
    for (int digit = 4; digit < 8; ++digit) pass(digit, nullptr);
    rs_fixup_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(kin, vin, n, full);
    for (int digit = 0; digit < 8; ++digit) pass(digit, full);
    if (batch) {
        pass(8, nullptr);
        pass(9, nullptr);
    }
    // the sorted (key, slot) pairs are in (kin, vin)
    // 4. permute the state into curve order
    GatherArgs g{};
    g.order = vin;
    // the packed (pos, vel) records serve the standalone density pass after a
    // full build; the density pass of a step gathers positions alone
    g.rec = kicked ? nullptr : c.rec;
    if (kin != s.keys) {
        g.keys_sorted = kin;
        g.keys_out = s.keys;
    }
    if (kicked) {
        float4 *src4[3] = {c.tmp4[0], c.tmp4[1], c.tmp4[2]};
        float4 *dst4[3] = {(float4 *)s.pos, (float4 *)s.vel, c.vhalf};
        for (int a = 0; a < 3; ++a) { g.a4[a] = src4[a]; g.t4[a] = dst4[a]; }
        g.a1[0] = c.tmp1[0];
        g.t1[0] = s.h;
        g.perm = c.tmp_perm;
        g.tperm = s.perm;
        g.n4 = 3;
        g.n1 = 1;
        gather_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(g, n);
    } else {
        // gather into the temporaries, then copy back
        float4 *arr4[4] = {(float4 *)s.pos, (float4 *)s.vel, (float4 *)s.acc, nullptr};
        float *arr1[5] = {s.h, s.rho, s.omega, s.drhodt, s.vsigmax};
        const int n4 = 3, n1 = 5;
        for (int a = 0; a < n4; ++a) { g.a4[a] = arr4[a]; g.t4[a] = c.tmp4[a]; }
        for (int a = 0; a < n1; ++a) { g.a1[a] = arr1[a]; g.t1[a] = c.tmp1[a]; }
        g.perm = s.perm;
        g.tperm = c.tmp_perm;
        g.n4 = n4;
        g.n1 = n1;
        gather_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(g, n);
        for (int a = 0; a < n4; ++a)
            SPH_TRY(cudaMemcpyAsync(arr4[a], c.tmp4[a], (size_t)n * 16, cudaMemcpyDeviceToDevice, st));
        for (int a = 0; a < n1; ++a)
            SPH_TRY(cudaMemcpyAsync(arr1[a], c.tmp1[a], (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        SPH_TRY(cudaMemcpyAsync(s.perm, c.tmp_perm, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    // recorded leaf ranges refer to the previous tree: mark them invalid
    SPH_TRY(cudaMemsetAsync(t.rec_ctl + 1, 0xff, sizeof(int), st));
    // 5. chop: tree (n_leaf) and groups (n_group)
    chop_flags_kernel<<<grid_for(c, n, kCfTile), 256, 0, st>>>(s.keys, inst, n, p.n_leaf, p.n_group,
                                                                t.lv_tree, t.lv_grp);
    // groups
    int *gidx = (int *)c.tmp1[1];  // scratch: tmp1[1..] are free once copied back
    SPH_TRY(scan_mode(c, t.lv_grp, gidx, n, 1, c.d_sizes + SZ_GROUPS, st));
    group_write_kernel<<<grid_for(c, n, 256), 256, 0, st>>>(t.lv_grp, gidx, n, t);
    group_bounds_kernel<<<grid_for(c, n, 128), 128, 0, st>>>(pos, s.h, n, t, c.d_sizes, 0, nullptr);
    // nodes
    int nb = div_up(n, kChopBlock);
    int *blk_off = (int *)c.tmp1[2];
    int *ntotal = c.d_sizes + 2;
    chop_count_kernel<<<nb, 256, 0, st>>>(t.lv_tree, n, t.blk_cnt, nb);
    SPH_TRY(scan_mode(c, t.blk_cnt, blk_off, kLevels * nb, 0, ntotal, st));
    chop_write_kernel<<<nb, 256, 0, st>>>(t.lv_tree, n, blk_off, nb, t, c.d_err);
    level_start_kernel<<<1, 32, 0, st>>>(blk_off, nb, ntotal, t, c.d_sizes);
    node_finish_kernel<<<grid_for(c, t.cap_nodes, 256), 256, 0, st>>>(s.keys, inst, n, p.n_leaf, t,
                                                                       c.d_sizes);
    node_bounds_kernel<<<grid_for(c, t.cap_nodes, 128), 128, 0, st>>>(pos, s.h, t, c.d_sizes, 0, nullptr);
    return cudaGetLastError();
}

__global__ void pack_records_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                    float4 *__restrict__ rec, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        rec[2 * (size_t)i] = pos[i];
        rec[2 * (size_t)i + 1] = vel[i];
    }
}

cudaError_t pack_records(Ctx &c, const sph_state &s, cudaStream_t st)
{
    pack_records_kernel<<<grid_for(c, s.n, 256), 256, 0, st>>>((const float4 *)s.pos,
                                                                (const float4 *)s.vel, c.rec, (int)s.n);
    return cudaGetLastError();
}

cudaError_t update_hmax(Ctx &c, const sph_state &s, const sph_params &p, cudaStream_t st,
                        const int *gate)
{
    (void)p;
    Tree &t = c.tree;
    node_bounds_kernel<<<grid_for(c, t.cap_nodes, 128), 128, 0, st>>>((const float4 *)s.pos, s.h, t,
                                                                       c.d_sizes, 1, gate);
    group_bounds_kernel<<<grid_for(c, s.n, 128), 128, 0, st>>>((const float4 *)s.pos, s.h,
                                                               (int)s.n, t, c.d_sizes, 1, gate);
    return cudaGetLastError();
}

// Test hook for the bounded look-back: one block of a sort pass that takes
// the place of tile 1 while tile 0 never publishes its counts.  The tile
// holds no keys (n = RS_TILE), so the block reads and writes no key; its
// look-back polls tile 0's zeroed status word spin_cap times, raises
// SPH_ERR_TIMEOUT in the error word and returns.
__global__ void set_int_kernel(int *p, int v) { *p = v; }

cudaError_t sort_lookback_probe(Ctx &c, int spin_cap, cudaStream_t st)
{
    // status words of tiles 0 and 1 (the buffer holds at least kRsSlots tiles)
    SPH_TRY(cudaMemsetAsync(c.rs_status, 0, sizeof(uint32_t) * 256 * 2, st));
    set_int_kernel<<<1, 1, 0, st>>>(c.rs_tiles, 1);  // the block draws tile 1
    rs_onesweep_kernel<<<1, RS_T, 0, st>>>(c.keys_alt, c.idx_a, c.keys_alt, c.idx_b, nullptr, RS_TILE,
                                          0, c.rs_gstart, c.rs_status, c.rs_tiles, c.d_err, nullptr,
                                          spin_cap);
    return cudaGetLastError();
}

}  // namespace sph
