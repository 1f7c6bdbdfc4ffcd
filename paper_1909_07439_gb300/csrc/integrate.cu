// Particle integration (Sect. 3.3): one thread per particle.
// Leapfrog of Eqs. 5-7 in kick-drift-kick form, the Courant step (Eq. 8) and
// the FP64 conserved quantities used for the energy error (Eq. 16).
#include "sph_internal.cuh"

namespace sph {

static int grid_n(const Ctx &c, int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)c.num_sms * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// v_half = v + a dt/2, u_half = u + du dt/2 (into vhalf);
// predicted v1p = v + a dt, u1p = u + du dt (Eq. 6) into vel1;
// r1 = r + v_half dt = r + v dt + a dt^2/2 (Eq. 5) into pos1, moved back
// into [lo, lo + L) on the periodic axes (by -L or +L; should rounding leave
// it outside, it becomes lo, its image within an ulp); h and perm copied
// along.  The outputs are the context's temporaries, from which the tree
// build gathers the state back in the new curve order.
__global__ void kick_drift_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                  const float4 *__restrict__ acc, const float *__restrict__ h,
                                  const uint32_t *__restrict__ perm, float4 *__restrict__ pos1,
                                  float4 *__restrict__ vel1, float4 *__restrict__ vhalf,
                                  float *__restrict__ h1, uint32_t *__restrict__ perm1, int n,
                                  const float *d_dt, const int *__restrict__ inst, Period per,
                                  float3 plo)
{
    auto wrap = [](float x, float L, float lo) {
        if (L > 0.f) {
            const float hi = lo + L;
            x = x >= hi ? x - L : x < lo ? x + L : x;
            x = (x >= lo && x < hi) ? x : lo;
        }
        return x;
    };
    float dt = *d_dt, hdt = 0.5f * dt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (inst) {
            dt = d_dt[inst[i]];
            hdt = 0.5f * dt;
        }
        float4 v = vel[i], a = acc[i], p = pos[i];
        float4 vh = make_float4(v.x + hdt * a.x, v.y + hdt * a.y, v.z + hdt * a.z, v.w + hdt * a.w);
        vhalf[i] = vh;
        vel1[i] = make_float4(v.x + dt * a.x, v.y + dt * a.y, v.z + dt * a.z, v.w + dt * a.w);
        pos1[i] = make_float4(wrap(p.x + dt * vh.x, per.x, plo.x), wrap(p.y + dt * vh.y, per.y, plo.y),
                              wrap(p.z + dt * vh.z, per.z, plo.z), p.w);
        h1[i] = h[i];
        perm1[i] = perm[i];
    }
}

// v1 = v_half + a1 dt/2 (equal to Eq. 7 applied to the Eq. 6 prediction)
__global__ void kick_close_kernel(float4 *__restrict__ vel, const float4 *__restrict__ acc,
                                  const float4 *__restrict__ vhalf, int n, const float *d_dt,
                                  double *d_time, int *err, const int *__restrict__ inst)
{
    float dt = *d_dt, hdt = 0.5f * dt;
    bool neg = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (inst) {
            dt = d_dt[inst[i]];
            hdt = 0.5f * dt;
        }
        float4 vh = vhalf[i], a = acc[i];
        float4 v = make_float4(vh.x + hdt * a.x, vh.y + hdt * a.y, vh.z + hdt * a.z, vh.w + hdt * a.w);
        neg |= !(v.w >= 0.f);
        vel[i] = v;
    }
    if (__any_sync(0xffffffffu, neg) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_NEGATIVE_U);
    if (!inst && d_time && blockIdx.x == 0 && threadIdx.x == 0) *d_time += (double)*d_dt;
}

// per-instance simulation time
__global__ void time_batch_kernel(const float *d_dt, double *d_time, int n_inst)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_inst; k += gridDim.x * blockDim.x)
        d_time[k] += (double)d_dt[k];
}

// per-instance minimum of h / vsigmax: ordered-int atomics, combined per warp
// when the warp lies inside one instance (positive floats order as ints)
__global__ void dt_batch_init_kernel(int *dtmin, int n_inst)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_inst; k += gridDim.x * blockDim.x)
        dtmin[k] = 0x7f800000;  // +inf
}

__global__ void dt_batch_kernel(const float *__restrict__ h, const float *__restrict__ vs,
                                const int *__restrict__ inst, int n, int *dtmin)
{
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
        int i = i0 + threadIdx.x;
        bool in = i < n;
        float m = in ? h[i] / vs[i] : INFINITY;
        int k = in ? inst[i] : -1;
        int k0 = __shfl_sync(0xffffffffu, k, 0);
        if (__all_sync(0xffffffffu, k == k0)) {
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0 && k0 >= 0) atomicMin(dtmin + k0, __float_as_int(m));
        } else if (in) {
            atomicMin(dtmin + k, __float_as_int(m));
        }
    }
}

__global__ void dt_batch_final_kernel(const int *dtmin, int n_inst, float c_cour, float *d_dt)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_inst; k += gridDim.x * blockDim.x)
        d_dt[k] = c_cour * __int_as_float(dtmin[k]);
}

// block minima of h / vsigmax
__global__ void __launch_bounds__(256) dt_block_kernel(const float *__restrict__ h,
                                                       const float *__restrict__ vs, int n,
                                                       float *blockmin)
{
    __shared__ float sm[8];
    float m = INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = fminf(m, h[i] / vs[i]);
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = sm[0];
        for (int w = 1; w < 8; ++w) r = fminf(r, sm[w]);
        blockmin[blockIdx.x] = r;
    }
}

__global__ void dt_final_kernel(const float *blockmin, int nb, float c_cour, float *d_dt)
{
    float m = INFINITY;
    for (int b = threadIdx.x; b < nb; b += 32) m = fminf(m, blockmin[b]);
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *d_dt = c_cour * m;
}

// FP64 sums in a fixed order: each thread owns a fixed strided subset, the
// block combines by a fixed tree, the final kernel adds block sums in order.
__global__ void __launch_bounds__(256) conserved_block_kernel(const float4 *__restrict__ pos,
                                                              const float4 *__restrict__ vel, int n,
                                                              double *part, int nb)
{
    __shared__ double sm[8][256];
    double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 p = pos[i], v = vel[i];
        double m = p.w, x = p.x, y = p.y, z = p.z, vx = v.x, vy = v.y, vz = v.z;
        e[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        e[1] += m * (double)v.w;
        e[2] += m * vx;
        e[3] += m * vy;
        e[4] += m * vz;
        e[5] += m * (y * vz - z * vy);
        e[6] += m * (z * vx - x * vz);
        e[7] += m * (x * vy - y * vx);
    }
    for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] = e[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 8) part[threadIdx.x * nb + blockIdx.x] = sm[threadIdx.x][0];
}

__global__ void conserved_final_kernel(const double *part, int nb, double *out8)
{
    int k = threadIdx.x;
    if (k < 8) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[k * nb + b];
        out8[k] = s;
    }
}

// ------------------------------------------------------------ block steps
// Individual power-of-two time steps: particle i (slot k, caller index
// perm[k]) steps with dt_i = dt_min 2^L_i, L_i = level[perm[k]]; substep j of
// the block spans [j, j + 1) dt_min.
//
// Substep j, before the passes: a particle whose step starts (j mod 2^L = 0)
// gets its opening half kick from its last acceleration (v_half = v + a dt/2,
// also u); every particle drifts with its half-step velocity (wrapped into a
// periodic box) and its velocity and u are predicted to the substep's end,
// v = v_half + a ((j mod 2^L + 1) dt_min - dt/2); the particles whose step ends
// there ((j + 1) mod 2^L = 0) are flagged for the density and force passes.

// a particle's level, checked: outside [0, max_level] it counts as 0 (and
// the substep kernel reports SPH_ERR_INVALID_ARG)
__device__ __forceinline__ int block_level(const int *level, const uint32_t *perm, int i, int max_level,
                                           bool &bad)
{
    const int L = level[perm[i]];
    bad = L < 0 || L > max_level;
    return bad ? 0 : L;
}

__global__ void block_substep_kernel(float4 *__restrict__ pos, float4 *__restrict__ vel,
                                     const float4 *__restrict__ acc, float4 *__restrict__ vhalf,
                                     uint8_t *__restrict__ due,
                                     const uint32_t *__restrict__ perm, const int *__restrict__ level,
                                     int n, int j, int max_level, const float *d_dt_min, Period per,
                                     float3 plo, int *err)
{
    bool any_bad = false;
    const float dtm = *d_dt_min;
    auto wrap = [](float x, float L, float lo) {
        if (L > 0.f) {
            const float hi = lo + L;
            x = x >= hi ? x - L : x < lo ? x + L : x;
            x = (x >= lo && x < hi) ? x : lo;
        }
        return x;
    };
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        bool bad;
        const int L = block_level(level, perm, i, max_level, bad);
        any_bad |= bad;
        const int mask = (1 << L) - 1;
        const float dt = dtm * (float)(1 << L);
        const float4 a = acc[i];
        float4 vh;
        if ((j & mask) == 0) {
            const float4 v = vel[i];
            const float hdt = 0.5f * dt;
            vh = make_float4(v.x + hdt * a.x, v.y + hdt * a.y, v.z + hdt * a.z, v.w + hdt * a.w);
            vhalf[i] = vh;
        } else {
            vh = vhalf[i];
        }
        const float4 p = pos[i];
        const float4 q = make_float4(wrap(p.x + dtm * vh.x, per.x, plo.x), wrap(p.y + dtm * vh.y, per.y, plo.y),
                                     wrap(p.z + dtm * vh.z, per.z, plo.z), p.w);
        const float into = (float)((j & mask) + 1) * dtm - 0.5f * dt;
        const float4 w = make_float4(vh.x + into * a.x, vh.y + into * a.y, vh.z + into * a.z, vh.w + into * a.w);
        pos[i] = q;
        vel[i] = w;
        due[i] = ((j + 1) & mask) == 0 ? 1 : 0;
    }
    if (__any_sync(0xffffffffu, any_bad) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_INVALID_ARG);
}

// the closing half kick of the particles whose step ended: v = v_half + a dt/2
__global__ void block_close_kernel(float4 *__restrict__ vel, const float4 *__restrict__ acc,
                                   const float4 *__restrict__ vhalf, const uint8_t *__restrict__ due,
                                   const uint32_t *__restrict__ perm, const int *__restrict__ level,
                                   int n, int max_level, const float *d_dt_min, double *d_time, int *err)
{
    const float dtm = *d_dt_min;
    bool neg = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!due[i]) continue;
        bool bad;
        const float hdt = 0.5f * dtm * (float)(1 << block_level(level, perm, i, max_level, bad));
        const float4 vh = vhalf[i], a = acc[i];
        const float4 v = make_float4(vh.x + hdt * a.x, vh.y + hdt * a.y, vh.z + hdt * a.z, vh.w + hdt * a.w);
        neg |= !(v.w >= 0.f);
        vel[i] = v;
    }
    if (__any_sync(0xffffffffu, neg) && (threadIdx.x & 31) == 0) raise_error(err, SPH_ERR_NEGATIVE_U);
    if (d_time && blockIdx.x == 0 && threadIdx.x == 0) *d_time += (double)dtm;
}

// level of each particle (caller order): the largest L <= max_level with
// dt_min 2^L <= c_cour min(h / vsigmax, u / |du/dt|) (Eq. 8 per particle and
// the same fraction of the time in which u changes by itself; FP32)
__global__ void block_levels_kernel(const float *__restrict__ h, const float *__restrict__ vs,
                                    const float4 *__restrict__ vel, const float4 *__restrict__ acc,
                                    const uint32_t *__restrict__ perm, int n, float c_cour,
                                    int max_level, const float *d_dt_min, int *level)
{
    const float dtm = *d_dt_min;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float du = fabsf(acc[i].w);
        const float tu = du > 0.f ? vel[i].w / du : INFINITY;
        const float dtc = c_cour * fminf(h[i] / vs[i], tu);
        int L = 0;
        while (L < max_level && dtm * (float)(2 << L) <= dtc) ++L;
        level[perm[i]] = L;
    }
}

cudaError_t block_substep(Ctx &c, const sph_state &s, const sph_params &p, const int *d_level, int j,
                          int max_level, const float *d_dt_min, cudaStream_t st)
{
    const int n = (int)s.n;
    block_substep_kernel<<<grid_n(c, n, 256), 256, 0, st>>>(
        (float4 *)s.pos, (float4 *)s.vel, (const float4 *)s.acc, c.vhalf, c.active, s.perm,
        d_level, n, j, max_level, d_dt_min, period_of(p), box_lo_of(p), c.d_err);
    return cudaGetLastError();
}

cudaError_t block_close(Ctx &c, const sph_state &s, const int *d_level, int max_level,
                        const float *d_dt_min, double *d_time, cudaStream_t st)
{
    const int n = (int)s.n;
    block_close_kernel<<<grid_n(c, n, 256), 256, 0, st>>>((float4 *)s.vel, (const float4 *)s.acc,
                                                          c.vhalf, c.active, s.perm, d_level, n,
                                                          max_level, d_dt_min, d_time, c.d_err);
    return cudaGetLastError();
}

cudaError_t block_levels(Ctx &c, const sph_state &s, const sph_params &p, int max_level,
                         const float *d_dt_min, int *d_level, cudaStream_t st)
{
    const int n = (int)s.n;
    block_levels_kernel<<<grid_n(c, n, 256), 256, 0, st>>>(s.h, s.vsigmax, (const float4 *)s.vel,
                                                           (const float4 *)s.acc, s.perm, n, p.c_cour,
                                                           max_level, d_dt_min, d_level);
    return cudaGetLastError();
}

cudaError_t kick_drift(Ctx &c, const sph_state &s, const sph_params &p, const float *d_dt,
                       cudaStream_t st, const Batch *batch)
{
    int n = (int)s.n;
    kick_drift_kernel<<<grid_n(c, n, 256), 256, 0, st>>>(
        (const float4 *)s.pos, (const float4 *)s.vel, (const float4 *)s.acc, s.h, s.perm, c.tmp4[0],
        c.tmp4[1], c.tmp4[2], c.tmp1[0], c.tmp_perm, n, d_dt, batch ? c.inst : nullptr,
        period_of(p), box_lo_of(p));
    return cudaGetLastError();
}

cudaError_t kick_close(Ctx &c, const sph_state &s, const float *d_dt, double *d_time,
                       cudaStream_t st, const Batch *batch)
{
    int n = (int)s.n;
    kick_close_kernel<<<grid_n(c, n, 256), 256, 0, st>>>((float4 *)s.vel, (const float4 *)s.acc,
                                                         c.vhalf, n, d_dt, d_time, c.d_err,
                                                         batch ? c.inst : nullptr);
    if (batch && d_time)
        time_batch_kernel<<<div_up(batch->n_inst, 256), 256, 0, st>>>(d_dt, d_time, batch->n_inst);
    return cudaGetLastError();
}

cudaError_t courant_dt(Ctx &c, const sph_state &s, const sph_params &p, float *d_dt,
                       cudaStream_t st, const Batch *batch)
{
    int n = (int)s.n;
    if (batch) {
        const int ni = batch->n_inst;
        dt_batch_init_kernel<<<div_up(ni, 256), 256, 0, st>>>(c.dtmin_inst, ni);
        dt_batch_kernel<<<grid_n(c, n, 256), 256, 0, st>>>(s.h, s.vsigmax, c.inst, n, c.dtmin_inst);
        dt_batch_final_kernel<<<div_up(ni, 256), 256, 0, st>>>(c.dtmin_inst, ni, p.c_cour, d_dt);
        return cudaGetLastError();
    }
    int nb = grid_n(c, n, 256);
    dt_block_kernel<<<nb, 256, 0, st>>>(s.h, s.vsigmax, n, c.red_f);
    dt_final_kernel<<<1, 32, 0, st>>>(c.red_f, nb, p.c_cour, d_dt);
    return cudaGetLastError();
}

cudaError_t conserved(Ctx &c, const sph_state &s, double *d_out8, cudaStream_t st)
{
    int n = (int)s.n;
    int nb = grid_n(c, n, 256);
    conserved_block_kernel<<<nb, 256, 0, st>>>((const float4 *)s.pos, (const float4 *)s.vel, n,
                                               c.red_d, nb);
    conserved_final_kernel<<<1, 32, 0, st>>>(c.red_d, nb, d_out8);
    return cudaGetLastError();
}

}  // namespace sph
