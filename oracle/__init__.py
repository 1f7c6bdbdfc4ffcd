"""Plain CPU oracle for the Bonsai-SPH hot path (arXiv 1909.07439).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The product package never imports
this module, and the C library here shares no code with the CUDA path.

The arithmetic lives in ``sph_oracle.c`` (FP64 brute force, canonical FP32
for keys and neighbour sets); this module builds it with gcc, marshals numpy
arrays, and composes the leapfrog step (Sect. 2.4, Eqs. 5-8) and the
Sedov-Taylor similarity constant (Sect. 4.3) on top of it.

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute-force enumeration or textbook values; none of
the functions is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available, no FP contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c11", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.orc_kernel_eval.argtypes = [P, P, i64, P, P, P, ctypes.c_int]
            lib.orc_bbox.argtypes = [P, i64, P]
            lib.orc_morton_keys.argtypes = [P, i64, P]
            lib.orc_sort_order.argtypes = [P, i64, P]
            lib.orc_sort_order.restype = ctypes.c_int
            lib.orc_chop.argtypes = [P, i64, i32, P, P, P, P, P, i64]
            lib.orc_chop.restype = i64
            lib.orc_neighbour_counts.argtypes = [P, P, i64, ctypes.c_int, P, i64, P, ctypes.c_int, P]
            lib.orc_neighbour_lists.argtypes = [P, P, i64, ctypes.c_int, P, i64, P, P, ctypes.c_int,
                                                P]
            lib.orc_density.argtypes = [P, P, P, i64, P, i64, P, f64, f64, i32, i32,
                                        P, P, P, P, P, P, ctypes.c_int, P]
            lib.orc_density.restype = i64
            lib.orc_force.argtypes = [P, P, P, P, P, P, P, i64, P, i64, f64, f64, f64,
                                      f64, f64, P, P, P, P, ctypes.c_int, P]
            lib.orc_conserved.argtypes = [P, P, P, P, i64, P]
            lib.orc_gravity.argtypes = [P, P, i64, P, i64, f64, f64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _box(box, dtype):
    """Periods (Lx, Ly, Lz), 0 for an open axis, as a C array; None: all open."""
    if box is None:
        return None
    b = np.ascontiguousarray(np.asarray(box, dtype).reshape(3))
    return b if np.any(b > 0) else None


def _bptr(b):
    return None if b is None else _ptr(b)


def _f32(a, shape_last=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape_last is not None:
        assert a.shape[-1] == shape_last
    return a


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _targets(targets, n):
    if targets is None:
        return np.arange(n, dtype=np.int64)
    return np.ascontiguousarray(targets, dtype=np.int64)


# --------------------------------------------------------------------------
# Smoothing kernels (Sect. 2.3, Eq. 14): 0 = M4 cubic, 1 = M6 quintic,
# 2 = Wendland C6; SUPPORT[k] = support radius in units of h
# --------------------------------------------------------------------------
M4, M6, WC6 = 0, 1, 2
SUPPORT = {M4: 2.0, M6: 3.0, WC6: 2.0}


def kernel_eval(r, h, kernel=M4):
    """Return (W, F = dW/dr, dW/dh) of the 3D kernel at (r, h)."""
    r, h = np.broadcast_arrays(_f64(r), _f64(h))
    r, h = _f64(r.ravel()), _f64(h.ravel())
    w, F, dh = (np.empty_like(r) for _ in range(3))
    _load().orc_kernel_eval(_ptr(r), _ptr(h), r.size, _ptr(w), _ptr(F), _ptr(dh), int(kernel))
    return w, F, dh


# --------------------------------------------------------------------------
# Keys, sort, chop (Sect. 3.1)
# --------------------------------------------------------------------------
def bbox(pos4):
    pos4 = _f32(pos4, 4)
    out = np.zeros(4, np.float32)
    _load().orc_bbox(_ptr(pos4), pos4.shape[0], _ptr(out))
    return out


def morton_keys(pos4):
    pos4 = _f32(pos4, 4)
    keys = np.zeros(pos4.shape[0], np.uint64)
    _load().orc_morton_keys(_ptr(pos4), pos4.shape[0], _ptr(keys))
    return keys


def sort_order(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    order = np.zeros(keys.size, np.int64)
    if _load().orc_sort_order(_ptr(keys), keys.size, _ptr(order)) != 0:
        raise MemoryError("oracle sort")
    return order


@dataclass
class Chop:
    level: np.ndarray
    first: np.ndarray
    count: np.ndarray
    child_first: np.ndarray
    nchild: np.ndarray


def chop(sorted_keys, thresh):
    """Level-by-level chop of the sorted curve into nodes (Sect. 3.1)."""
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    n = k.size
    cap = max(16, 4 * n + 64)
    lvl = np.zeros(cap, np.int32)
    first = np.zeros(cap, np.int64)
    count = np.zeros(cap, np.int64)
    cf = np.zeros(cap, np.int64)
    nc = np.zeros(cap, np.int32)
    nn = _load().orc_chop(_ptr(k), n, int(thresh), _ptr(lvl), _ptr(first), _ptr(count),
                          _ptr(cf), _ptr(nc), cap)
    if nn < 0:
        raise RuntimeError("oracle chop capacity")
    return Chop(lvl[:nn].copy(), first[:nn].copy(), count[:nn].copy(), cf[:nn].copy(),
                nc[:nn].copy())


# --------------------------------------------------------------------------
# Neighbour sets (Sect. 3.2), canonical FP32
# --------------------------------------------------------------------------
def neighbours(pos4, h, mode, targets=None, kernel=M4, box=None):
    """CSR (offsets, indices) of the density (mode 0) or force (mode 1) sets;
    box: periods of the periodic axes (0: open), compared in FP32."""
    pos4 = _f32(pos4, 4)
    h = _f32(h)
    b = _box(box, np.float32)
    n = pos4.shape[0]
    t = _targets(targets, n)
    cnt = np.zeros(t.size, np.int64)
    lib = _load()
    lib.orc_neighbour_counts(_ptr(pos4), _ptr(h), n, int(mode), _ptr(t), t.size, _ptr(cnt),
                             int(kernel), _bptr(b))
    off = np.zeros(t.size + 1, np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.zeros(max(1, int(off[-1])), np.int64)
    lib.orc_neighbour_lists(_ptr(pos4), _ptr(h), n, int(mode), _ptr(t), t.size, _ptr(off),
                            _ptr(idx), int(kernel), _bptr(b))
    return off, idx[: off[-1]]


# --------------------------------------------------------------------------
# Density / smoothing length (Eqs. 1-4) and force (Eqs. 9-15)
# --------------------------------------------------------------------------
@dataclass
class Density:
    h: np.ndarray
    rho: np.ndarray
    omega: np.ndarray
    drhodt: np.ndarray
    nngb: np.ndarray
    iters: np.ndarray
    failures: int


def density(x, v, m, h0, targets=None, hfact=1.2, tol=1e-12, max_iter=200, fixed_iters=0,
            kernel=M4, box=None):
    """Solve the h-rho fixed point for each target (FP64, brute force);
    box: periods of the periodic axes (0: open)."""
    x, v, m, h0 = _f64(x), _f64(v), _f64(m), _f64(h0)
    b = _box(box, np.float64)
    n = m.size
    assert x.shape == (n, 3) and v.shape == (n, 3) and h0.shape == (n,)
    t = _targets(targets, n)
    h, rho, om, dr = (np.zeros(t.size) for _ in range(4))
    nngb = np.zeros(t.size, np.int32)
    iters = np.zeros(t.size, np.int32)
    fails = _load().orc_density(_ptr(x), _ptr(v), _ptr(m), n, _ptr(t), t.size, _ptr(h0),
                                float(hfact), float(tol), int(max_iter), int(fixed_iters),
                                _ptr(h), _ptr(rho), _ptr(om), _ptr(dr), _ptr(nngb),
                                _ptr(iters), int(kernel), _bptr(b))
    return Density(h, rho, om, dr, nngb, iters, int(fails))


@dataclass
class Force:
    acc: np.ndarray
    dudt: np.ndarray
    vsigmax: np.ndarray
    nforce: np.ndarray


def force(x, v, m, u, h, rho, omega, targets=None, gamma=5.0 / 3.0, alpha=1.0, beta=2.0,
          alpha_u=1.0, vsig_scale=1.0, kernel=M4, box=None):
    """Accelerations, du/dt and max signal speed for each target (FP64);
    box: periods of the periodic axes (0: open)."""
    x, v, m, u, h, rho, omega = (_f64(a) for a in (x, v, m, u, h, rho, omega))
    b = _box(box, np.float64)
    n = m.size
    t = _targets(targets, n)
    acc = np.zeros((t.size, 3))
    dudt, vsig = np.zeros(t.size), np.zeros(t.size)
    nf = np.zeros(t.size, np.int32)
    _load().orc_force(_ptr(x), _ptr(v), _ptr(m), _ptr(u), _ptr(h), _ptr(rho), _ptr(omega), n,
                      _ptr(t), t.size, float(gamma), float(alpha), float(beta),
                      float(alpha_u), float(vsig_scale), _ptr(acc), _ptr(dudt), _ptr(vsig),
                      _ptr(nf), int(kernel), _bptr(b))
    return Force(acc, dudt, vsig, nf)


def gravity(x, m, G=1.0, eps=0.01, targets=None):
    """Softened self-gravity by direct summation (the a_grav of Eq. 9):
    returns (acc [nt, 3], phi [nt]) for the targets."""
    x, m = _f64(x), _f64(m)
    n = m.size
    t = _targets(targets, n)
    out = np.zeros((t.size, 4))
    _load().orc_gravity(_ptr(x), _ptr(m), n, _ptr(t), t.size, float(G), float(eps), _ptr(out))
    return out[:, :3].copy(), out[:, 3].copy()


def conserved(x, v, m, u):
    """{E_kin, E_th, px, py, pz, Lx, Ly, Lz} (Sect. 4.5, Eq. 16 uses E = E_kin + E_th)."""
    x, v, m, u = _f64(x), _f64(v), _f64(m), _f64(u)
    out = np.zeros(8)
    _load().orc_conserved(_ptr(x), _ptr(v), _ptr(m), _ptr(u), m.size, _ptr(out))
    return out


# --------------------------------------------------------------------------
# Leapfrog (Sect. 2.4, Eqs. 5-8) in kick-drift-kick form
# --------------------------------------------------------------------------
@dataclass
class Params:
    gamma: float = 5.0 / 3.0
    hfact: float = 1.2
    alpha: float = 1.0
    beta: float = 2.0
    alpha_u: float = 1.0
    c_cour: float = 0.3
    tol: float = 1e-12
    max_iter: int = 200
    kernel: int = M4
    box: tuple = None       # periods (Lx, Ly, Lz), 0 for an open axis
    box_lo: tuple = None    # lower corner of the periodic box (positions wrap into it)


@dataclass
class SphState:
    x: np.ndarray      # (n,3)
    v: np.ndarray      # (n,3)
    u: np.ndarray      # (n,)
    m: np.ndarray      # (n,)
    h: np.ndarray      # (n,)
    rho: np.ndarray = None
    omega: np.ndarray = None
    drhodt: np.ndarray = None
    acc: np.ndarray = None
    dudt: np.ndarray = None
    vsigmax: np.ndarray = None


def evaluate(s: SphState, p: Params = Params()):
    """Density solve then force pass at the current state (in place)."""
    d = density(s.x, s.v, s.m, s.h, hfact=p.hfact, tol=p.tol, max_iter=p.max_iter, kernel=p.kernel,
                box=p.box)
    if d.failures:
        raise RuntimeError(f"oracle density: {d.failures} targets did not converge")
    s.h, s.rho, s.omega, s.drhodt = d.h, d.rho, d.omega, d.drhodt
    f = force(s.x, s.v, s.m, s.u, s.h, s.rho, s.omega, gamma=p.gamma, alpha=p.alpha,
              beta=p.beta, alpha_u=p.alpha_u, kernel=p.kernel, box=p.box)
    s.acc, s.dudt, s.vsigmax = f.acc, f.dudt, f.vsigmax
    return s


def courant_dt(s: SphState, p: Params = Params()):
    """Global step dt = C_cour min_i h_i / vsigmax_i (Eq. 8)."""
    return float(p.c_cour * np.min(s.h / s.vsigmax))


def kdk_step(s: SphState, dt: float, p: Params = Params()):
    """One leapfrog step; equal to Eqs. 5-7 written as kick-drift-kick.

    r1 = r0 + v0 dt + a0 dt^2/2 (Eq. 5); v1p = v0 + a0 dt (Eq. 6) feeds the
    force pass; v1 = v1p + (a1 - a0) dt/2 (Eq. 7).  The internal energy uses
    the same predictor/corrector.
    """
    vh = s.v + 0.5 * dt * s.acc
    uh = s.u + 0.5 * dt * s.dudt
    x1 = wrap_positions(s.x + dt * vh, p)
    v1p = s.v + dt * s.acc
    u1p = s.u + dt * s.dudt
    n = SphState(x=x1, v=v1p, u=u1p, m=s.m, h=s.h)
    evaluate(n, p)
    n.v = vh + 0.5 * dt * n.acc
    n.u = uh + 0.5 * dt * n.dudt
    return n


def wrap_positions(x, p: Params):
    """Positions moved back into the periodic box [lo, lo + L) on each
    periodic axis (x - L above it, x + L below it)."""
    if p.box is None:
        return x
    x = np.array(x, np.float64, copy=True)
    for a in range(3):
        L = float(p.box[a])
        if L > 0:
            lo = float(p.box_lo[a]) if p.box_lo is not None else 0.0
            x[:, a] = np.where(x[:, a] >= lo + L, x[:, a] - L, x[:, a])
            x[:, a] = np.where(x[:, a] < lo, x[:, a] + L, x[:, a])
    return x


def block_step(s: SphState, levels, dt_min: float, max_level: int, p: Params = Params()):
    """One block step of individual (power-of-two) time steps, the block-time-step
    form of the leapfrog the paper leaves unused (footnote in Sect. 2.4), in the
    same kick-drift-kick form as kdk_step.

    Particle i steps with dt_i = dt_min 2^levels[i] (levels fixed for the block);
    the block lasts dt_min 2^max_level, in substeps of dt_min.  In substep k
    (k = 0 .. 2^max_level - 1) a particle whose step starts (k mod 2^levels[i]
    = 0) gets its opening half kick from its last acceleration; every
    particle drifts with its half-step velocity; every particle's velocity and
    u are predicted to the substep's end (half-step value plus acceleration
    times the time past the step's middle); the particles whose step ends
    there ((k + 1) mod 2^levels[i] = 0) get their density solved (from their
    last h) and their force computed, against all particles at their
    predicted velocities and last h, rho, Omega, then the closing half kick.
    The state must hold the accelerations of its positions (an evaluate)."""
    lv = np.asarray(levels, np.int64)
    x, v, u = s.x.copy(), s.v.copy(), s.u.copy()
    h, rho, om, drho = s.h.copy(), s.rho.copy(), s.omega.copy(), s.drhodt.copy()
    acc, dudt, vs = s.acc.copy(), s.dudt.copy(), s.vsigmax.copy()
    dti = dt_min * 2.0 ** lv
    vh, uh = v.copy(), u.copy()
    for k in range(2 ** max_level):
        period = 2 ** lv
        start = (k % period) == 0
        vh[start] = v[start] + 0.5 * dti[start, None] * acc[start]
        uh[start] = u[start] + 0.5 * dti[start] * dudt[start]
        x = wrap_positions(x + dt_min * vh, p)
        into = ((k % period) + 1) * dt_min - 0.5 * dti
        v = vh + into[:, None] * acc
        u = uh + into * dudt
        end = np.where(((k + 1) % period) == 0)[0]
        d = density(x, v, s.m, h, targets=end, hfact=p.hfact, tol=p.tol, max_iter=p.max_iter,
                    kernel=p.kernel, box=p.box)
        if d.failures:
            raise RuntimeError(f"oracle density: {d.failures} targets did not converge")
        h[end], rho[end], om[end], drho[end] = d.h, d.rho, d.omega, d.drhodt
        f = force(x, v, s.m, u, h, rho, om, targets=end, gamma=p.gamma, alpha=p.alpha,
                  beta=p.beta, alpha_u=p.alpha_u, kernel=p.kernel, box=p.box)
        acc[end], dudt[end], vs[end] = f.acc, f.dudt, f.vsigmax
        v[end] = vh[end] + 0.5 * dti[end, None] * acc[end]
        u[end] = uh[end] + 0.5 * dti[end] * dudt[end]
    return SphState(x=x, v=v, u=u, m=s.m, h=h, rho=rho, omega=om, drhodt=drho, acc=acc,
                    dudt=dudt, vsigmax=vs)


def block_levels(s: SphState, dt_min: float, max_level: int, p: Params = Params()):
    """Level of each particle for a block step: the largest k <= max_level with
    dt_min 2^k <= C_cour min(h_i / vsigmax_i, u_i / |du_i/dt|) (Eq. 8 per
    particle, and the same fraction of the time in which u changes by
    itself, which keeps a long step from driving u negative)."""
    with np.errstate(divide="ignore"):
        tu = np.where(s.dudt != 0.0, s.u / np.abs(s.dudt), np.inf)
    dtc = p.c_cour * np.minimum(s.h / s.vsigmax, tu)
    k = np.zeros(len(dtc), np.int64)
    for j in range(1, max_level + 1):
        k = np.where(dt_min * 2.0 ** j <= dtc, j, k)
    return k


def total_energy(s: SphState):
    c = conserved(s.x, s.v, s.m, s.u)
    return c[0] + c[1]


# --------------------------------------------------------------------------
# Sedov-Taylor similarity solution (Sect. 4.3)
# --------------------------------------------------------------------------
def sedov_xi0(gamma: float) -> float:
    """Constant xi0 of the spherical blast radius R = xi0 (E t^2 / rho0)^(1/5).

    Self-similar ansatz u = Rdot f(l), rho = rho0 g(l), p = rho0 Rdot^2 k(l),
    l = r / R, R ~ t^(2/5).  Mass, momentum and entropy conservation give
      (f-l) g' + g (f' + 2 f / l) = 0
      -3/2 f + (f-l) f' + k'/g = 0
      -3 + (f-l) (k'/k - gamma g'/g) = 0
    with strong-shock values f = k = 2/(gamma+1), g = (gamma+1)/(gamma-1) at
    l = 1.  Energy: 1 = (16 pi / 25) xi0^5 int_0^1 l^2 (g f^2/2 + k/(gamma-1)) dl.
    """
    from scipy.integrate import solve_ivp

    def rhs(l, y):
        f, g, k, _ = y
        a = f - l
        A = np.array([[g, a, 0.0],
                      [a, 0.0, 1.0 / g],
                      [0.0, -gamma * a / g, a / k]])
        b = np.array([-2.0 * g * f / l, 1.5 * f, 3.0])
        df, dg, dk = np.linalg.solve(A, b)
        dI = l * l * (0.5 * g * f * f + k / (gamma - 1.0))
        return [df, dg, dk, dI]

    y0 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0), 0.0]
    sol = solve_ivp(rhs, (1.0, 1e-6), y0, method="LSODA", rtol=1e-11, atol=1e-14)
    I = -sol.y[3, -1]  # integrated from 1 down to ~0
    return float((25.0 / (16.0 * np.pi * I)) ** 0.2)


def sedov_radius(E: float, rho0: float, t: float, gamma: float) -> float:
    return sedov_xi0(gamma) * (E * t * t / rho0) ** 0.2


def shock_radius_from_profile(x, rho, centre, nbins=64, rmax=None):
    """Radius of the peak of the radially binned mean density (analysis helper)."""
    r = np.linalg.norm(_f64(x) - np.asarray(centre, np.float64), axis=1)
    rmax = rmax or float(r.max())
    edges = np.linspace(0.0, rmax, nbins + 1)
    which = np.clip(np.digitize(r, edges) - 1, 0, nbins - 1)
    s = np.bincount(which, weights=_f64(rho), minlength=nbins)
    c = np.bincount(which, minlength=nbins)
    prof = np.where(c > 0, s / np.maximum(c, 1), 0.0)
    k = int(np.argmax(prof))
    return 0.5 * (edges[k] + edges[k + 1]), prof, edges
