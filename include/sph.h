/*
 * sph.h - C ABI of the GB300 (sm_103a) SPH neighbour-sum library.
 *
 * The library implements the per-step hot path of Bonsai-SPH
 * (arXiv 1909.07439): space-filling-curve octree build (Sect. 3.1), the
 * group-wise tree walk (Sect. 3.2), the smoothing-length / density solve
 * (Sect. 2.2, Eqs. 1-4), the hydro force with artificial viscosity and
 * conductivity (Sect. 2.4-2.6, Eqs. 9-15) and the leapfrog step with the
 * Courant time step (Sect. 2.4, Eqs. 5-8), for the M4 cubic spline
 * (Sect. 2.3).  Self-gravity is not part of this library.
 *
 * Conventions for every entry point:
 *  - All array pointers in sph_state are DEVICE pointers (unless an entry
 *    point says otherwise), owned by the caller, 16-byte aligned, and must
 *    stay valid until the work enqueued on `stream` has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Calls are asynchronous.  Argument errors are returned synchronously.
 *    Conditions found on the device (non-finite input, a density solve that
 *    did not converge, a scratch overflow, negative internal energy) are
 *    recorded in the context's device error word and returned by the next
 *    sph_sync(); sph_last_error() gives the text.
 *  - A context owns all scratch memory, allocated once by sph_create for at
 *    most max_n particles; no later call allocates device memory, except
 *    sph_step_host (host-buffer mirror, allocated on its first call).
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_ERR_INVALID_ARG = 1,   /* bad pointer, size, or parameter                    */
    SPH_ERR_CUDA = 2,          /* a CUDA runtime call failed                         */
    SPH_ERR_NOMEM = 3,         /* allocation failed, or tree capacity exceeded       */
    SPH_ERR_NOT_CONVERGED = 4, /* h-rho Newton did not reach h_tol in max_h_iter     */
    SPH_ERR_TILE_OVERFLOW = 5, /* a tree-walk stack or a neighbour list overflowed  */
    SPH_ERR_NONFINITE = 6,     /* non-finite position, velocity, mass or h; m<=0; h<=0 */
    SPH_ERR_NEGATIVE_U = 7,    /* internal energy became negative                    */
    SPH_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up                 */
} sph_status;

/* Method parameters.  Defaults (sph_params_default) are the paper's
 * (Sect. 4: gamma = 5/3, alpha_AV = 1, beta_AV = 2, alpha_u = 1, C_cour = 0.3,
 * M4 kernel; Sect. 4.6: N_leaf = 16, N_crit = N_group = 8) and hfact = 1.2. */
typedef struct {
    float gamma;         /* adiabatic index; P = (gamma-1) rho u                       */
    float hfact;         /* h = hfact (m/rho)^(1/3)  (Eq. 2)                            */
    float alpha_av;      /* alpha^AV  (Eq. 12)                                          */
    float beta_av;       /* beta^AV   (Eq. 12)                                          */
    float alpha_u;       /* alpha_u, artificial conductivity (Eq. 13)                   */
    float c_cour;        /* Courant factor (Eq. 8)                                      */
    float h_tol;         /* Newton stops when |dh| < h_tol h (decided exactly)         */
    int32_t kernel;      /* smoothing kernel (Sect. 2.3), support radius R in units of h:
                            0 = M4 cubic spline (R = 2), 1 = M6 quintic spline
                            (R = 3), 2 = Wendland C6 (R = 2); other values are
                            SPH_ERR_INVALID_ARG.  hfact should suit the kernel
                            (about 1.2, 0.9 and 1.3 respectively)             */
    int32_t n_leaf;      /* max particles per tree leaf  (1..64)                        */
    int32_t n_group;     /* max particles per walk group (1..32)                        */
    int32_t tile;        /* shared-memory list capacity per target of the walking
                            fallback kernels, 0 = default (80 density, 96 force
                            for M4; 128 for the other kernels)                 */
    int32_t max_h_iter;  /* Newton iteration cap (>= 1)                                 */
    int32_t density_iters; /* 0: iterate to h_tol; k > 0: exactly k updates (Sect. 3.2.1) */
    /* Launch shape of the neighbour-list density and force kernels (results
     * do not depend on it beyond FP32 summation order; 0 = default):       */
    int32_t pair_targets;  /* targets per warp batch: 4, 8 (default) or 16;
                              each target gets 32 / pair_targets lanes       */
    int32_t pair_warps;    /* warps per block: 1, 2, 4 (default) or 8       */
    int32_t pair_unroll;   /* list entries per lane and iteration of the
                              density and force kernels: 2 (default) or 4 */
    /* Periodic boundaries (the tube tests of Sect. 4.1-4.2 are periodic in y
     * and z).  box_len[a] > 0 makes axis a periodic with period box_len[a]
     * (0 = open axis, the default): positions must lie in
     * [box_lo[a], box_lo[a] + box_len[a]) (sph_build_tree checks this,
     * SPH_ERR_INVALID_ARG), every pair separation along the axis is the
     * nearest image (d - L if d > L/2, d + L if d < -L/2, exact in FP32),
     * and sph_step wraps drifted positions back into the box.  The support
     * R h of every particle must stay below box_len[a] / 2 (the force pass
     * reports SPH_ERR_INVALID_ARG otherwise).                              */
    float box_lo[3];
    float box_len[3];
    /* Self-gravity, the a_grav term of Eq. 9 (Sect. 2.4): grav_G > 0 adds the
     * Newtonian acceleration of every particle, with Plummer softening
     * grav_eps, to acc in every force pass, by a Barnes-Hut walk of the same
     * tree (a node whose centre of mass lies farther than
     * l / grav_theta + delta from a group's box acts on the group through its
     * monopole and quadrupole; l its longest edge, delta the offset of its
     * centre of mass from its box centre).  grav_G = 0 (default): no gravity.
     * With grav_G > 0: grav_eps > 0, 0 < grav_theta <= 0.57 (no node that
     * holds a target is ever accepted), and no periodic axis; the adjoint
     * entry points reject it (gravity is not differentiated).             */
    float grav_G;
    float grav_eps;
    float grav_theta;
} sph_params;

/* Particle state, structure of arrays, n particles, device memory.
 * After sph_build_tree the arrays are in space-filling-curve order and
 * perm[k] is the caller's original index of slot k. */
typedef struct {
    int64_t n;
    float *pos;      /* [n][4]  x, y, z, m                                   in    */
    float *vel;      /* [n][4]  vx, vy, vz, u                                in    */
    float *acc;      /* [n][4]  ax, ay, az, du/dt                            out   */
    float *h;        /* [n]     smoothing length                             in/out */
    float *rho;      /* [n]     density                                      out   */
    float *omega;    /* [n]     grad-h term Omega (Eq. 4)                    out   */
    float *drhodt;   /* [n]     drho/dt (Eq. 3)                              out   */
    float *vsigmax;  /* [n]     max signal speed (Eq. 8)                     out   */
    uint32_t *perm;  /* [n]     original index of each slot                  in/out */
    uint64_t *keys;  /* [n]     63-bit Morton key of each slot               out   */
} sph_state;

/* Fill *p with the defaults listed above. */
void sph_params_default(sph_params *p);

/* Create a context on CUDA device `device` for up to max_n particles
 * (max_n >= 1, < 2^31).  All scratch is allocated here.
 * Errors: SPH_ERR_INVALID_ARG, SPH_ERR_CUDA, SPH_ERR_NOMEM. */
sph_status sph_create(sph_ctx **out, int64_t max_n, int device);

/* Release a context and its scratch (synchronises its device first). */
void sph_destroy(sph_ctx *ctx);

/* Tree build (Sect. 3.1): bounding box, 63-bit Morton keys (21 bits per axis,
 * canonical FP32 quantisation), stable LSD radix sort of (key, slot), in-place
 * permutation of pos, vel, acc, h, rho, omega, drhodt, vsigmax and perm into
 * curve order, octree chop (nodes of at most n_leaf particles) and group chop
 * (groups of at most n_group particles), with node/group bounding boxes.
 * The caller initialises perm once (identity for "original order").
 * Validates inputs: non-finite pos/h, m <= 0 or h <= 0 set SPH_ERR_NONFINITE. */
sph_status sph_build_tree(sph_ctx *ctx, sph_state *s, const sph_params *p, void *stream);

/* Density pass (Eqs. 1-4): for every particle, Newton iteration on
 * g(h) = sum_j m_j W(r_ij, h) - m (hfact/h)^3 from the input h, over the
 * group walk of the tree built by the last sph_build_tree on this state.
 * Writes h, rho = m (hfact/h)^3, omega (Eq. 4) and drhodt (Eq. 3, with vel). */
sph_status sph_density(sph_ctx *ctx, sph_state *s, const sph_params *p, void *stream);

/* Hydro force pass (Eqs. 9-15), no gravity: writes acc (xyz and du/dt) and
 * vsigmax.  Needs h, rho, omega from sph_density and the current vel.
 * A pair interacts if r < R max(h_i, h_j), R the kernel's support radius
 * in units of h (Sect. 3.2). */
sph_status sph_force(sph_ctx *ctx, sph_state *s, const sph_params *p, void *stream);

/* Courant step (Eq. 8): *d_dt = c_cour * min_i h_i / vsigmax_i (device float). */
sph_status sph_timestep(sph_ctx *ctx, const sph_state *s, const sph_params *p, float *d_dt,
                        void *stream);

/* One leapfrog step (Eqs. 5-7 in kick-drift-kick form) with dt = *d_dt:
 * kick/drift with the acc already in the state, tree build, density and force
 * at the new positions with predicted v and u, closing kick, then the next
 * Courant step is written to *d_dt.  Inside a step drhodt comes from the
 * force pass (Eq. 3 is, up to the factor rho_i A_i, the pair sum of the
 * energy equation's pressure work), so the density pass gathers positions
 * only.  If d_time is not NULL, *d_time += dt
 * (device double).  Nothing returns to the host inside the call.
 * The first call for a given (state arrays, n, params, d_dt, d_time, timing
 * on/off) records the step's kernels into a CUDA graph (the context keeps the
 * last four); later calls with the same arguments launch that graph on
 * `stream`.  Inside a capture that the caller records on `stream`, the kernels
 * are enqueued directly and the stage timers skip the step. */
sph_status sph_step(sph_ctx *ctx, sph_state *s, const sph_params *p, float *d_dt,
                    double *d_time, void *stream);

/* Batched form (not in the paper): n_inst independent SPH problems packed
 * back to back in one state; instance k owns slots [d_offsets[k],
 * d_offsets[k+1]) (device int64 [n_inst+1], ascending, d_offsets[0] = 0,
 * d_offsets[n_inst] = n, every instance non-empty, n_inst <= 65536; other
 * offsets are reported as SPH_ERR_INVALID_ARG through the error word, and
 * no kernel then reads or writes outside the state's n slots).  Each
 * instance gets its own bounding box, keys, tree and groups (the sort keeps
 * every instance on its own slots), its own Courant step and its own time:
 * d_dt is a device float [n_inst], d_time a device double [n_inst] (or NULL).
 * The results for an instance equal those of the single-instance calls on
 * that instance alone.
 * sph_batch_evaluate: tree build, density, force (with self-gravity when
 * grav_G > 0, as sph_force) and Courant step of every instance (the initial
 * evaluation before stepping).
 * sph_batch_step: n_steps leapfrog steps of every instance.  The first call
 * for a given (state, offsets, params, d_dt, d_time) records one step into a
 * CUDA graph (stream capture); every step is a replay of that graph, whose
 * density and force kernels are persistent launches pulling the groups of
 * all instances from one work queue.  Asynchronous. */
sph_status sph_batch_evaluate(sph_ctx *ctx, sph_state *s, const int64_t *d_offsets, int n_inst,
                              const sph_params *p, float *d_dt, void *stream);
sph_status sph_batch_step(sph_ctx *ctx, sph_state *s, const int64_t *d_offsets, int n_inst,
                          int n_steps, const sph_params *p, float *d_dt, double *d_time,
                          void *stream);

/* Adjoint of the force pass (not in the paper): given the cotangents
 * d_gacc [n][4] = (dL/da xyz, dL/d(du/dt)) of the outputs of the LAST
 * sph_force on this state (same tree and neighbour sets), writes dL/dx
 * (d_gpos [n][4], xyz), dL/dv and dL/du (d_gvel [n][4]), dL/dh, dL/drho,
 * dL/dOmega (d_gh, d_grho, d_gomega [n]) of every particle, and ADDS
 * dL/dalpha_AV to *d_galpha (device double).  Deterministic: each particle
 * sums the terms landing on its inputs (no atomics on particle data). */
sph_status sph_force_bwd(sph_ctx *ctx, const sph_state *s, const sph_params *p,
                         const float *d_gacc, float *d_gpos, float *d_gvel, float *d_gh,
                         float *d_grho, float *d_gomega, double *d_galpha, void *stream);

/* Adjoint of the density pass (not in the paper): given cotangents of h,
 * rho and Omega from the LAST sph_density on this state, ADDS dL/dx to
 * d_gpos [n][4] (xyz).  The h-rho fixed point is differentiated by the
 * implicit-function theorem: dh_i = -(dg_i/dx) dx / (dg_i/dh_i),
 * g_i = sum_j m_j W(r_ij, h_i) - m_i (hfact/h_i)^3 (Eqs. 1, 2, 4). */
sph_status sph_density_bwd(sph_ctx *ctx, const sph_state *s, const sph_params *p,
                           const float *d_gh, const float *d_grho, const float *d_gomega,
                           float *d_gpos, void *stream);

/* Differentiable rollout (not in the paper).  From the initial state init
 * (device arrays pos, vel, h in the caller's order, n particles; not
 * modified): initial evaluation, then n_steps leapfrog steps with the Courant
 * dt of each step recorded; loss L = mean over the n_probes particles
 * d_probes (device int64, caller's indices) of rho^2 after the last step,
 * written to *h_loss (host).  If d_gvel (device float [n][4]) is not NULL,
 * also writes dL/dv0 (xyz) and dL/du0 (w) of every particle in the caller's
 * order and dL/dalpha_AV to *h_galpha (host), by the adjoint method: the dt
 * sequence is held fixed, the state before every ckpt-th step is
 * checkpointed, and each window of ckpt steps is recomputed from its
 * checkpoint during the backward sweep.  Work buffers (about 12 state copies
 * plus ckpt + n_steps/ckpt checkpoints) are allocated on the first call and
 * kept by the context.  Synchronous. */
sph_status sph_rollout(sph_ctx *ctx, const sph_state *init, const sph_params *p, int n_steps,
                       int ckpt, const int64_t *d_probes, int n_probes, double *h_loss,
                       float *d_gvel, double *h_galpha, void *stream);

/* Same step for a state held in HOST memory (pinned for best speed): copies
 * the state in, runs n_steps steps, copies it back; *h_dt (host) is read as
 * the first dt and receives the next one.  Allocates a device mirror on the
 * first call.  With every array of *hs pinned, the last step copies each
 * output back on a second stream as soon as it is final (pos, perm, keys
 * after the tree build; h, rho, omega after the density pass; acc, drhodt,
 * vsigmax after the force pass), so those copies overlap the rest of the
 * step.  Synchronous. */
sph_status sph_step_host(sph_ctx *ctx, sph_state *host_state, const sph_params *p, int n_steps,
                         float *h_dt, void *stream);

/* FP64 conserved quantities (Sect. 4.5, Eq. 16), deterministic reduction:
 * d_out8 = { E_kin, E_th, px, py, pz, Lx, Ly, Lz } (device doubles). */
sph_status sph_conserved(sph_ctx *ctx, const sph_state *s, double *d_out8, void *stream);

/* Conserved quantities for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a library convenience.
 * Same result as sph_conserved (FP64 {E_kin, E_th, px, py, pz, Lx, Ly, Lz},
 * summation order differs, so values agree to FP64 rounding), but it needs
 * no context: sph_create allocates, and some callers cannot call cudaMalloc
 * (a host framework that owns all device memory and only lends its particle
 * arrays, or code that must not risk the device-wide synchronisation an
 * allocation can cause).  d_pos, d_vel: device [n][4] float arrays as in
 * sph_state, 16-byte aligned; d_out8: device double[8]; stream as above.
 * Its scratch is a fixed 256 KB array inside the library, held on every GPU
 * that loads the library until the process exits; no call allocates.
 * The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make
 * that first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) while the library is loaded: the kept address would then
 * be stale.
 * All calls share the array and it keeps the last call's partial sums: calls
 * whose kernels overlap on the GPU (unordered streams) race; calls ordered on
 * one stream are safe.  Returns SPH_ERR_INVALID_ARG if n < 0 or
 * n > SPH_CONSERVED_NOALLOC_MAX_N, for NULL pointers, for d_pos or d_vel not
 * 16-byte aligned or d_out8 not 8-byte aligned, or a
 * current device index >= 64; SPH_ERR_CUDA if a launch or the address
 * lookup fails.  Asynchronous otherwise. */
#define SPH_CONSERVED_NOALLOC_MAX_N 16777216
sph_status sph_conserved_noalloc(int64_t n, const float *d_pos, const float *d_vel,
                                 double *d_out8, void *stream);

/* Block (individual) time steps: the kick-drift-kick leapfrog of sph_step
 * with a step of its own per particle, dt_i = dt_min 2^L_i (the paper's code
 * has such steps and leaves them unused, Sect. 2.4).
 *
 * sph_block_levels: *d_dt_min = c_cour min_i h_i / vsigmax_i (Eq. 8, as
 * sph_timestep) and d_level[i] (caller order, int32, device) = the largest
 * L <= max_level with dt_min 2^L <= c_cour min(h_i / vsigmax_i, u_i / |du_i/dt|)
 * (FP32; the second term keeps a long step from driving u negative).  Needs
 * h, vsigmax, u and du/dt of the current state.
 *
 * sph_step_block: one block of 2^max_level substeps of *d_dt_min (device
 * float) with the levels d_level (caller order, each in [0, max_level],
 * fixed for the block; a level outside that range counts as 0 and is
 * reported as SPH_ERR_INVALID_ARG through the error word).  It first sorts the state into curve order (as
 * sph_build_tree: acc, h, rho, omega, drhodt, vsigmax move along), then per
 * substep j: particles whose step starts (j mod 2^L = 0) get their opening
 * half kick from their last acceleration; all drift with their half-step
 * velocity (wrapped into a periodic box) and have velocity and u predicted
 * to the substep's end; the tree's boxes are refitted to the new positions
 * (no re-sort); the particles whose step ends ((j + 1) mod 2^L = 0) get the
 * density pass (Newton from their last h) and the force pass against all
 * particles at their predicted velocities and last h, rho, Omega, then
 * their closing half kick.  After the block every particle is synchronised
 * with fresh forces.  *d_time (device double, may be NULL) advances by
 * dt_min per substep.  Needs acc, vsigmax, h, rho, omega of the current
 * state (after sph_force, sph_step or sph_step_block).  0 <= max_level <= 16;
 * not with gravity (SPH_ERR_INVALID_ARG).  Asynchronous. */
sph_status sph_block_levels(sph_ctx *ctx, const sph_state *s, const sph_params *p, int max_level,
                            float *d_dt_min, int32_t *d_level, void *stream);
sph_status sph_step_block(sph_ctx *ctx, sph_state *s, const sph_params *p, int max_level,
                          const int32_t *d_level, const float *d_dt_min, double *d_time,
                          void *stream);

/* Self-gravity alone (the a_grav term of Eq. 9, see sph_params.grav_G):
 * d_out4[4 k .. 4 k + 3] = (a_x, a_y, a_z, phi) of slot k, G included, by
 * the Barnes-Hut walk of the tree built by the last sph_build_tree on this
 * state (positions unchanged since).  The potential energy is
 * 1/2 sum_k m_k phi_k.  d_out4: device, 16-byte aligned, n float4.
 * SPH_ERR_INVALID_ARG unless grav_G > 0 and the gravity parameters are
 * valid.  Asynchronous. */
sph_status sph_gravity(sph_ctx *ctx, const sph_state *s, const sph_params *p, float *d_out4,
                       void *stream);

/* Neighbour sets of the current tree/state (Sect. 3.2), for testing.
 * mode 0: density set {j : r2 < (R h_i)^2} (includes i);
 * mode 1: force set {j != i : r2 < (R max(h_i, h_j))^2};
 * R the support radius of p->kernel (2 M4, 3 M6, 2 Wendland C6) and R h
 * rounded to FP32;
 * r2 = (dx*dx + dy*dy) + dz*dz in FP32, round-to-nearest, no fusion.
 * Modes 0 and 1 use a separate tree walk.  Modes 2 and 3 give the same two
 * sets taken from the neighbour lists that sph_density and sph_force read:
 * the list-building walk of the density pass runs at the current h (its
 * lists replace the context's), and each list is filtered with the test
 * above (mode 2: density set, mode 3: force set).  If a particle's list
 * overflowed, its row is empty and the call returns SPH_ERR_TILE_OVERFLOW.
 * The tree must be the one built from the current positions.
 * d_off: device int64 [n+1] row offsets (always written);
 * d_idx: device int32 [cap] slot indices (written if non-NULL and total <= cap).
 * *h_total receives the total (host).  Synchronous. */
sph_status sph_neighbours(sph_ctx *ctx, const sph_state *s, const sph_params *p, int mode,
                          int64_t *d_off, int32_t *d_idx, int64_t cap, int64_t *h_total,
                          void *stream);

/* Copy the tree and groups of the last sph_build_tree to HOST arrays, for
 * testing.  Nodes are in level-major order (first particle order inside a
 * level): level, first particle, particle count, number of children, and the
 * index of the first child (-1 for a leaf; children are contiguous).  Groups:
 * first particle and count.  *n_nodes / *n_groups receive the counts; the
 * arrays are filled only when the counts fit node_cap / group_cap (any array
 * may be NULL).  Synchronous. */
sph_status sph_get_tree(sph_ctx *ctx, int32_t *h_level, int32_t *h_first, int32_t *h_count,
                        int32_t *h_nchild, int32_t *h_child, int64_t node_cap,
                        int32_t *h_gfirst, int32_t *h_gcount, int64_t group_cap,
                        int64_t *n_nodes, int64_t *n_groups);

/* Test hook for the bounded device-side waits: enqueues one block of a
 * radix-sort pass that waits, in its decoupled look-back, on a predecessor
 * tile that never publishes (the real passes wait only on tiles that are
 * already running).  After spin_cap polls (1..2^20) the block records
 * SPH_ERR_TIMEOUT in the error word and returns, reading and writing no
 * particle data; the next sph_sync returns SPH_ERR_TIMEOUT and clears it.
 * Uses the context's sort scratch, so do not overlap it with a tree build. */
sph_status sph_test_lookback_timeout(sph_ctx *ctx, int spin_cap, void *stream);

/* Work counters accumulated since the last call (then reset).  Synchronous. */
typedef struct {
    uint64_t density_pairs;       /* true-neighbour pairs summed, all Newton sweeps   */
    uint64_t density_candidates;  /* particle-pair distance tests in list-building and
                                     density walks                                     */
    uint64_t force_pairs;         /* pairs in the force sets                           */
    uint64_t force_candidates;    /* list entries scanned plus pair tests of force walks */
    uint64_t newton_iters;        /* Newton updates summed over particles              */
    uint64_t density_rewalks;     /* target batches solved by the walking fallback
                                     (an h outgrew the list pad or a list overflowed) */
    uint64_t streamed_groups;     /* fallback batches whose lists overflowed the tile  */
    uint64_t n_nodes;             /* tree nodes of the last build                      */
    uint64_t n_groups;            /* groups of the last build                          */
    uint64_t list_entries;        /* neighbour-list entries written                    */
    uint64_t list_overflows;      /* particles whose list exceeded its capacity        */
    uint64_t force_rewalks;       /* target batches of the force pass solved by the
                                     walking fallback (lists stale, overflowed, or an
                                     h of the instance outgrew the list pad)          */
    uint64_t gravity_cells;       /* target-node (multipole) gravity interactions      */
    uint64_t gravity_particles;   /* target-particle gravity interactions             */
} sph_stats;
sph_status sph_get_stats(sph_ctx *ctx, sph_stats *out);

/* Per-stage device timing (CUDA events on the launching stream).
 * Stages: 0 tree build, 1 density (h-rho solve), 2 force, 3 reductions
 * (dt, conserved), 4 leapfrog kicks/drift, 5 force preparation (per-particle
 * sound speed and node/group h_max, also refreshed before the density pass),
 * 6 neighbour lists (the list-building tree walk of the density pass),
 * 7 self-gravity (multipole moments and the Barnes-Hut walk).
 * sph_get_timing synchronises and returns the milliseconds summed since the
 * last call, and the number of kernels launched per stage (also counted when
 * timing is off); both arrays hold SPH_N_STAGES entries. */
#define SPH_N_STAGES 8
sph_status sph_set_timing(sph_ctx *ctx, int enable);
sph_status sph_get_timing(sph_ctx *ctx, double *ms_by_stage, int64_t *launches_by_stage);

/* FP32 throughput probe (a measurement utility, not part of the method):
 * enqueues `blocks` blocks of 256 threads, each thread running `iters`
 * iterations of 8 independent fused multiply-add chains, as scalar FP32
 * FMAs (packed = 0: 16 FLOP per thread and iteration) or packed FP32x2 FMAs
 * (packed = 1: 32 FLOP per thread and iteration).  The caller times it with
 * events on `stream`; d_sink is one device float that is never written in
 * practice.  SPH_ERR_INVALID_ARG for bad arguments, SPH_ERR_CUDA if the
 * launch fails; asynchronous otherwise. */
sph_status sph_fp32_probe(float *d_sink, int blocks, int iters, int packed, void *stream);

/* Synchronise `stream` and return (then clear) the device error word. */
sph_status sph_sync(sph_ctx *ctx, void *stream);

/* Text of the last error on this context (never NULL). */
const char *sph_last_error(sph_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
