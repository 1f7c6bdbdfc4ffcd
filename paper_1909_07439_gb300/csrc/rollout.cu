// Differentiable rollout (not part of the paper's method): a loss after
// n_steps leapfrog steps and its gradient by the adjoint method.
//
// Forward: initial evaluation, then n_steps sph_step-equivalent steps with
// the Courant dt of each step recorded (the dt sequence is held fixed in the
// gradient: no derivative through the minimum of Eq. 8).  The state before
// every ckpt-th step is kept (checkpoint); with gradients, the states of the
// last window after their force passes are kept too.  Loss L = mean over
// probe particles (by the caller's index) of rho^2 after the last step.
//
// Backward, window by window from the last checkpoint: the window's steps
// are recomputed from its checkpoint (deterministic: the same trees and
// neighbour sets; the last window's were kept by the forward) and each
// step's state after its force pass is kept; then,
// from the last step of the window down, a step's state is restored, its
// tree and neighbour lists are rebuilt (the state is in that tree's order, so
// the sort is the identity) and the step is differentiated: closing kick,
// force (adjoint kernels), density (implicit-function theorem), opening kick
// and drift.  Between steps
// the cotangents live in the caller's particle order; each step gathers them
// into its own curve order through perm and scatters them back, so the sort
// permutations need no bookkeeping.  Finally the initial force evaluation is
// differentiated for dL/dv0, dL/du0; dL/dalpha_AV accumulates in FP64.
#include <cstring>

#include "sph_internal.cuh"

namespace sph {

cudaError_t force_bwd(Ctx &c, const sph_state &s, const sph_params &p, const float4 *gacc,
                      float4 *gpos, float4 *gvel, float *gh, float *grho, float *gom,
                      double *galpha, cudaStream_t st);
cudaError_t density_bwd(Ctx &c, const sph_state &s, const sph_params &p, const float *gh,
                        const float *grho, const float *gom, float4 *gpos, float2 *coef,
                        cudaStream_t st, bool refresh_hmax = true);

static int grid_r(const Ctx &c, int64_t n)
{
    int64_t g = (n + 255) / 256, cap = (int64_t)c.num_sms * 16;
    return (int)(g < 1 ? 1 : g > cap ? cap : g);
}

__global__ void iota_kernel(uint32_t *p, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

__global__ void probe_flag_kernel(const int64_t *probes, int np, int n, unsigned char *flag)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        int64_t p = probes[k];
        if (p >= 0 && p < n) flag[p] = 1;
    }
}

// per-block partial sums of rho^2 over probe slots (fixed order), then total / np
__global__ void loss_block_kernel(const float *rho, const uint32_t *perm,
                                  const unsigned char *flag, int n, double *part)
{
    __shared__ double sm[256];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (flag[perm[i]]) s += (double)rho[i] * (double)rho[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void loss_final_kernel(const double *part, int nb, int np, double *loss)
{
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *loss = s / (double)np;
    }
}

// cotangent of (a1, du1) from the closing kick v1 = vh + a1 dt/2:
// gacc_s = ga + dt/2 gv (gathered from the caller's order)
__global__ void gather_cot_kernel(const uint32_t *perm, const float4 *ga, const float4 *gv,
                                  const float *dts, int k, int n, float4 *gacc_s)
{
    const float hdt = 0.5f * dts[k];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint32_t o = perm[s];
        float4 a = ga[o], v = gv[o];
        gacc_s[s] = make_float4(a.x + hdt * v.x, a.y + hdt * v.y, a.z + hdt * v.z, a.w + hdt * v.w);
    }
}

// loss cotangent on rho at the last step: 2 rho / np on probe slots
__global__ void loss_grho_kernel(const float *rho, const uint32_t *perm, const unsigned char *flag,
                                 int n, int np, float *grho)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        if (flag[perm[s]]) grho[s] += 2.f * rho[s] / (float)np;
}

// Backward of the opening kick and drift, from the step's slot order to the
// caller's order.  x1 = x + dt vh, vh = v + dt/2 a, vp = v + dt a (same for u).
__global__ void scatter_cot_kernel(const uint32_t *perm, const float4 *gpos_s, const float4 *gvel_s,
                                   const float *dts, int k, int n, float4 *gx, float4 *gv,
                                   float4 *ga)
{
    const float dt = dts[k], hdt = 0.5f * dt;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint32_t o = perm[s];
        float4 gp = gpos_s[s], gvp = gvel_s[s], x0 = gx[o], v0 = gv[o];
        float x1x = gp.x + x0.x, x1y = gp.y + x0.y, x1z = gp.z + x0.z;  // dL/dx1
        float vhx = v0.x + dt * x1x, vhy = v0.y + dt * x1y, vhz = v0.z + dt * x1z;  // dL/dvh
        float uh = v0.w;                                                         // dL/duh
        gx[o] = make_float4(x1x, x1y, x1z, 0.f);
        gv[o] = make_float4(vhx + gvp.x, vhy + gvp.y, vhz + gvp.z, uh + gvp.w);
        ga[o] = make_float4(hdt * vhx + dt * gvp.x, hdt * vhy + dt * gvp.y, hdt * vhz + dt * gvp.z,
                            hdt * uh + dt * gvp.w);
    }
}

__global__ void final_grad_kernel(const uint32_t *perm, const float4 *gv, const float4 *gvel_s,
                                  int n, float *out)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint32_t o = perm[s];
        float4 a = gv[o], b = gvel_s[s];
        reinterpret_cast<float4 *>(out)[o] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
}

// ------------------------------------------------------------ buffers
struct StateBuf {
    float4 *pos = nullptr, *vel = nullptr, *acc = nullptr;
    float *h = nullptr, *rho = nullptr, *omega = nullptr;
    uint32_t *perm = nullptr;
};

static cudaError_t alloc_sb(StateBuf &b, size_t n)
{
    cudaError_t e = cudaMalloc(&b.pos, n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&b.vel, n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&b.acc, n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&b.h, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b.rho, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b.omega, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b.perm, n * 4);
    return e;
}

static void free_sb(StateBuf &b)
{
    cudaFree(b.pos);
    cudaFree(b.vel);
    cudaFree(b.acc);
    cudaFree(b.h);
    cudaFree(b.rho);
    cudaFree(b.omega);
    cudaFree(b.perm);
    b = StateBuf{};
}

static cudaError_t save(const sph_state &w, StateBuf &b, size_t n, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(b.pos, w.pos, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.vel, w.vel, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.acc, w.acc, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.h, w.h, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.rho, w.rho, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.omega, w.omega, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.perm, w.perm, n * 4, cudaMemcpyDeviceToDevice, st);
    return e;
}

static cudaError_t restore(sph_state &w, const StateBuf &b, size_t n, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(w.pos, b.pos, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.vel, b.vel, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.acc, b.acc, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.h, b.h, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.rho, b.rho, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.omega, b.omega, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.perm, b.perm, n * 4, cudaMemcpyDeviceToDevice, st);
    return e;
}

struct RolloutBuf {
    int64_t n = 0;
    int n_ckpt = 0, win = 0, n_steps = 0;
    sph_state w{};                 // working state (all arrays)
    std::vector<StateBuf> ckpt;    // state before step k * ckpt
    std::vector<StateBuf> window;  // pre-step states of one window
    float *dts = nullptr;
    float *d_dt = nullptr;
    double *d_loss = nullptr, *d_galpha = nullptr, *part = nullptr;
    float4 *gx = nullptr, *gv = nullptr, *ga = nullptr;
    float4 *gacc_s = nullptr, *gpos_s = nullptr, *gvel_s = nullptr;
    float *gh_s = nullptr, *grho_s = nullptr, *gom_s = nullptr;
    float2 *coef = nullptr;
    unsigned char *flag = nullptr;
};

}  // namespace sph

using namespace sph;

namespace {

struct RB {
    RolloutBuf b;
    ~RB()
    {
        sph_state &w = b.w;
        void *p[] = {w.pos, w.vel, w.acc, w.h, w.rho, w.omega, w.drhodt, w.vsigmax, w.perm, w.keys,
                     b.dts, b.d_dt, b.d_loss, b.d_galpha, b.part, b.gx, b.gv, b.ga, b.gacc_s,
                     b.gpos_s, b.gvel_s, b.gh_s, b.grho_s, b.gom_s, b.coef, b.flag};
        for (void *q : p)
            if (q) cudaFree(q);
        for (auto &s : b.ckpt) free_sb(s);
        for (auto &s : b.window) free_sb(s);
    }
};

// The context owns its rollout buffers (Ctx::rollout); sph_destroy releases
// them through release_rollout.
cudaError_t ensure_rb(Ctx &c, int64_t n, int n_steps, int ck, RB **out)
{
    RB *rb = static_cast<RB *>(c.rollout);
    int n_ckpt = (n_steps + ck - 1) / ck;
    // dts holds n_steps + 1 entries, so a longer rollout needs new buffers
    if (rb && rb->b.n >= n && rb->b.n_ckpt >= n_ckpt && rb->b.win >= ck && rb->b.n_steps >= n_steps) {
        *out = rb;
        return cudaSuccess;
    }
    if (rb) {
        c.rollout = nullptr;
        delete rb;
    }
    rb = new RB();
    RolloutBuf &b = rb->b;
    size_t N = (size_t)c.max_n;
    b.n = c.max_n;
    b.n_ckpt = n_ckpt;
    b.win = ck;
    b.n_steps = n_steps;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(cudaMalloc((void **)&b.w.pos, N * 16));
    A(cudaMalloc((void **)&b.w.vel, N * 16));
    A(cudaMalloc((void **)&b.w.acc, N * 16));
    A(cudaMalloc((void **)&b.w.h, N * 4));
    A(cudaMalloc((void **)&b.w.rho, N * 4));
    A(cudaMalloc((void **)&b.w.omega, N * 4));
    A(cudaMalloc((void **)&b.w.drhodt, N * 4));
    A(cudaMalloc((void **)&b.w.vsigmax, N * 4));
    A(cudaMalloc((void **)&b.w.perm, N * 4));
    A(cudaMalloc((void **)&b.w.keys, N * 8));
    b.ckpt.resize(n_ckpt);
    for (auto &s : b.ckpt) A(alloc_sb(s, N));
    b.window.resize(ck);
    for (auto &s : b.window) A(alloc_sb(s, N));
    A(cudaMalloc((void **)&b.dts, sizeof(float) * (size_t)(n_steps + 1)));
    A(cudaMalloc((void **)&b.d_dt, sizeof(float)));
    A(cudaMalloc((void **)&b.d_loss, sizeof(double)));
    A(cudaMalloc((void **)&b.d_galpha, sizeof(double)));
    A(cudaMalloc((void **)&b.part, sizeof(double) * (size_t)c.num_sms * 16));
    A(cudaMalloc((void **)&b.gx, N * 16));
    A(cudaMalloc((void **)&b.gv, N * 16));
    A(cudaMalloc((void **)&b.ga, N * 16));
    A(cudaMalloc((void **)&b.gacc_s, N * 16));
    A(cudaMalloc((void **)&b.gpos_s, N * 16));
    A(cudaMalloc((void **)&b.gvel_s, N * 16));
    A(cudaMalloc((void **)&b.gh_s, N * 4));
    A(cudaMalloc((void **)&b.grho_s, N * 4));
    A(cudaMalloc((void **)&b.gom_s, N * 4));
    A(cudaMalloc((void **)&b.coef, N * 8));
    A(cudaMalloc((void **)&b.flag, N));
    if (e != cudaSuccess) {
        delete rb;
        return e;
    }
    c.rollout = rb;
    *out = rb;
    return cudaSuccess;
}

#define RT(x)                             \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// initial evaluation of the working state: tree, density, force, Courant dt
cudaError_t evaluate(Ctx &c, sph_state &w, const sph_params &p, float *d_dt, cudaStream_t st)
{
    RT(build_tree(c, w, p, true, st));
    RT(density_pass(c, w, p, st));
    RT(force_prep(c, w, p, st));
    RT(force_pass(c, w, p, st));
    return courant_dt(c, w, p, d_dt, st);
}

// leapfrog step with dt = dts[k]; up to the force pass if partial
cudaError_t step(Ctx &c, sph_state &w, const sph_params &p, const float *dt, bool partial,
                 float *d_dt_next, cudaStream_t st)
{
    RT(kick_drift(c, w, p, dt, st));
    RT(build_tree(c, w, p, false, st));
    {
        DrhodtInForce fused(c);  // as in sph_step: drho/dt from the force pass
        RT(density_pass(c, w, p, st));
        RT(force_prep(c, w, p, st));
        RT(force_pass(c, w, p, st));
    }
    if (partial) return cudaSuccess;
    RT(kick_close(c, w, dt, nullptr, st));
    return courant_dt(c, w, p, d_dt_next, st);
}

cudaError_t load_init(Ctx &c, sph_state &w, const sph_state &init, cudaStream_t st)
{
    size_t n = (size_t)init.n;
    RT(cudaMemcpyAsync(w.pos, init.pos, n * 16, cudaMemcpyDeviceToDevice, st));
    RT(cudaMemcpyAsync(w.vel, init.vel, n * 16, cudaMemcpyDeviceToDevice, st));
    RT(cudaMemcpyAsync(w.h, init.h, n * 4, cudaMemcpyDeviceToDevice, st));
    RT(cudaMemsetAsync(w.acc, 0, n * 16, st));
    iota_kernel<<<grid_r(c, n), 256, 0, st>>>(w.perm, (int)n);
    return cudaGetLastError();
}

cudaError_t rollout(Ctx &c, RolloutBuf &b, const sph_state &init, const sph_params &p, int K,
                    int ck, const int64_t *probes, int np, bool grad, cudaStream_t st)
{
    const int n = (int)init.n;
    sph_state w = b.w;
    w.n = n;
    const int nb = grid_r(c, n);
    // ---- forward (with gradients, the last window's states after their
    // force passes are kept on the way: its backward needs no recompute)
    const int nwin = (K + ck - 1) / ck;
    const int k_last = (nwin - 1) * ck;
    RT(load_init(c, w, init, st));
    RT(evaluate(c, w, p, b.d_dt, st));
    for (int k = 0; k < K; ++k) {
        if (k % ck == 0) RT(save(w, b.ckpt[k / ck], n, st));
        RT(cudaMemcpyAsync(b.dts + k, b.d_dt, sizeof(float), cudaMemcpyDeviceToDevice, st));
        if (grad && k >= k_last) {
            RT(step(c, w, p, b.dts + k, true, nullptr, st));
            RT(save(w, b.window[k - k_last], n, st));
            RT(kick_close(c, w, b.dts + k, nullptr, st));
            RT(courant_dt(c, w, p, b.d_dt, st));
        } else {
            RT(step(c, w, p, b.dts + k, false, b.d_dt, st));
        }
    }
    RT(cudaMemsetAsync(b.flag, 0, n, st));
    probe_flag_kernel<<<grid_r(c, np), 256, 0, st>>>(probes, np, n, b.flag);
    loss_block_kernel<<<nb, 256, 0, st>>>(w.rho, w.perm, b.flag, n, b.part);
    loss_final_kernel<<<1, 32, 0, st>>>(b.part, nb, np, b.d_loss);
    if (!grad) return cudaGetLastError();
    // ---- backward
    RT(cudaMemsetAsync(b.gx, 0, (size_t)n * 16, st));
    RT(cudaMemsetAsync(b.gv, 0, (size_t)n * 16, st));
    RT(cudaMemsetAsync(b.ga, 0, (size_t)n * 16, st));
    RT(cudaMemsetAsync(b.d_galpha, 0, sizeof(double), st));
    for (int cw = nwin - 1; cw >= 0; --cw) {
        const int k0 = cw * ck, k1 = std::min(k0 + ck, K);
        const bool kept = cw == nwin - 1;  // the forward kept this window's states
        if (!kept) {
            // recompute the window from its checkpoint, keeping each step's state
            // after its force pass (what the step's backward differentiates)
            RT(restore(w, b.ckpt[cw], n, st));
            for (int k = k0; k < k1; ++k) {
                RT(step(c, w, p, b.dts + k, true, nullptr, st));
                RT(save(w, b.window[k - k0], n, st));
                if (k < k1 - 1) RT(kick_close(c, w, b.dts + k, nullptr, st));
            }
        }
        for (int k = k1 - 1; k >= k0; --k) {
            if (k < k1 - 1 || kept) RT(restore(w, b.window[k - k0], n, st));
            // the step's tree (the state is already in its curve order: the
            // permutation is the identity) and its neighbour lists at the final h
            RT(build_tree(c, w, p, true, st));
            RT(density_lists(c, w, p, st, nullptr, false));
            gather_cot_kernel<<<nb, 256, 0, st>>>(w.perm, b.ga, b.gv, b.dts, k, n, b.gacc_s);
            RT(force_bwd(c, w, p, b.gacc_s, b.gpos_s, b.gvel_s, b.gh_s, b.grho_s, b.gom_s,
                         b.d_galpha, st));
            if (k == K - 1)
                loss_grho_kernel<<<nb, 256, 0, st>>>(w.rho, w.perm, b.flag, n, np, b.grho_s);
            // force_bwd refreshed node and group h_max for this h
            RT(density_bwd(c, w, p, b.gh_s, b.grho_s, b.gom_s, b.gpos_s, b.coef, st, false));
            scatter_cot_kernel<<<nb, 256, 0, st>>>(w.perm, b.gpos_s, b.gvel_s, b.dts, k, n, b.gx,
                                                   b.gv, b.ga);
        }
    }
    // ---- the initial force evaluation: (a0, du0) depend on v0, u0 and alpha
    RT(load_init(c, w, init, st));
    RT(evaluate(c, w, p, b.d_dt, st));
    gather_cot_kernel<<<nb, 256, 0, st>>>(w.perm, b.ga, b.gv, b.dts, K, n, b.gacc_s);
    return cudaGetLastError();
}

}  // namespace

void sph::release_rollout(Ctx &c)
{
    delete static_cast<RB *>(c.rollout);
    c.rollout = nullptr;
}

// parameters the adjoint passes take: a built kernel, no gravity (its
// a_grav term is not differentiated)
static bool adjoint_params_ok(const sph_params *p)
{
    return p->kernel >= 0 && p->kernel <= 2 && p->grav_G == 0.f;
}

extern "C" sph_status sph_rollout(sph_ctx *h, const sph_state *init, const sph_params *p,
                                  int n_steps, int ckpt, const int64_t *d_probes, int n_probes,
                                  double *h_loss, float *d_gvel, double *h_galpha, void *stream)
{
    if (!h || !init || !p || !h_loss || !d_probes) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    if (init->n < 1 || init->n > c.max_n || !init->pos || !init->vel || !init->h)
        return SPH_ERR_INVALID_ARG;
    if (n_steps < 1 || ckpt < 1 || n_probes < 1 || !adjoint_params_ok(p)) return SPH_ERR_INVALID_ARG;
    if ((d_gvel == nullptr) != (h_galpha == nullptr)) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    RB *rb = nullptr;
    cudaError_t e = ensure_rb(c, init->n, n_steps, ckpt, &rb);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SPH_ERR_NOMEM : SPH_ERR_CUDA;
    RolloutBuf &b = rb->b;
    const bool grad = d_gvel != nullptr;
    if (grad) {
        // dts[n_steps] = 0: the gather for the initial evaluation adds no kick term
        e = cudaMemsetAsync(b.dts + n_steps, 0, sizeof(float), st);
        if (e != cudaSuccess) return SPH_ERR_CUDA;
    }
    e = rollout(c, b, *init, *p, n_steps, ckpt, d_probes, n_probes, grad, st);
    if (e != cudaSuccess) return SPH_ERR_CUDA;
    if (grad) {
        sph_state w = b.w;
        w.n = init->n;
        const int n = (int)init->n;
        e = force_bwd(c, w, *p, b.gacc_s, b.gpos_s, b.gvel_s, b.gh_s, b.grho_s, b.gom_s,
                      b.d_galpha, st);
        if (e != cudaSuccess) return SPH_ERR_CUDA;
        final_grad_kernel<<<grid_r(c, n), 256, 0, st>>>(w.perm, b.gv, b.gvel_s, n, d_gvel);
        if (cudaMemcpyAsync(h_galpha, b.d_galpha, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return SPH_ERR_CUDA;
    }
    if (cudaMemcpyAsync(h_loss, b.d_loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SPH_ERR_CUDA;
    return sph_sync(h, stream);
}

extern "C" sph_status sph_force_bwd(sph_ctx *h, const sph_state *s, const sph_params *p,
                                    const float *d_gacc, float *d_gpos, float *d_gvel, float *d_gh,
                                    float *d_grho, float *d_gomega, double *d_galpha, void *stream)
{
    if (!h || !s || !p || !d_gacc || !d_gpos || !d_gvel || !d_gh || !d_grho || !d_gomega ||
        !d_galpha)
        return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    if (s->n < 1 || s->n > c.max_n || !adjoint_params_ok(p)) return SPH_ERR_INVALID_ARG;
    cudaError_t e = force_bwd(c, *s, *p, (const float4 *)d_gacc, (float4 *)d_gpos, (float4 *)d_gvel,
                              d_gh, d_grho, d_gomega, d_galpha, (cudaStream_t)stream);
    return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

extern "C" sph_status sph_density_bwd(sph_ctx *h, const sph_state *s, const sph_params *p,
                                      const float *d_gh, const float *d_grho, const float *d_gomega,
                                      float *d_gpos, void *stream)
{
    if (!h || !s || !p || !d_gh || !d_grho || !d_gomega || !d_gpos) return SPH_ERR_INVALID_ARG;
    Ctx &c = h->impl;
    if (s->n < 1 || s->n > c.max_n || !adjoint_params_ok(p)) return SPH_ERR_INVALID_ARG;
    // the per-particle multipliers use context scratch (one float2 per particle)
    cudaError_t e = density_bwd(c, *s, *p, d_gh, d_grho, d_gomega, (float4 *)d_gpos,
                                reinterpret_cast<float2 *>(c.tmp4[3]), (cudaStream_t)stream);
    return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
