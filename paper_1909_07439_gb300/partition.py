"""Domain decomposition of one SPH problem over ranks (Sect. 3.4).

The paper splits the particles along the space-filling curve and exchanges
the parts of the tree other domains need.  Here each rank owns one
contiguous range of the global Morton order with an equal number of
particles, and receives as halo every particle of the other ranks that can
interact with one of its own:

1. global bounding box (all-reduce of min and max, exact in FP32) and the
   63-bit Morton key of every particle with the same canonical FP32
   quantisation as the tree build (21 bits per axis);
2. the global order is (key, global id); rank r owns positions
   [r N / P, (r + 1) N / P) of it.  The boundaries are found by bisection,
   first on the key, then on the id among particles of the boundary key,
   each round one all-reduce of P - 1 counts;
3. particles move to their owners by point-to-point messages;
4. halo selection: particle j of rank r goes to rank q if
   dist(x_j, box_q) < R max(h_max,q, h_j) (1 + pad), box_q and h_max,q the
   bounding box and largest h of q's own particles, R the kernel's support
   radius in units of h (2 for M4 and Wendland C6, 3 for M6).  Every j with
   |x_i - x_j| < R max(h_i, h_j) for some i of q satisfies it, since
   dist(x_j, box_q) <= |x_i - x_j|: the halo holds the density sets
   (r < R h_i, Eq. 1) and the force sets (r < R max(h_i, h_j), Sect. 3.2) of
   q's particles as long as no h grows by more than the pad;
5. after the density pass the owners send h, rho and Omega of their halo
   particles (the force pass needs them, Eqs. 9-15), and an all-reduced flag
   says whether an h outgrew the pad (then the halo is selected again).

The collectives are torch.distributed calls (gloo on CPU ranks); the
arithmetic here is host-side bookkeeping, no SPH sums.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KEY_BITS = 21


def bounding_box(pos4: np.ndarray, group=None):
    """Global (lo[3], size) of all ranks' positions: FP32 min / max all-reduced
    (exact), size = max over axes of (hi - lo) in FP32, as the tree build."""
    import torch
    import torch.distributed as dist
    x = np.asarray(pos4, np.float32)[:, :3]
    lo = torch.tensor(x.min(0) if len(x) else np.full(3, np.inf, np.float32))
    hi = torch.tensor(x.max(0) if len(x) else np.full(3, -np.inf, np.float32))
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    lo, hi = lo.numpy().astype(np.float32), hi.numpy().astype(np.float32)
    ext = (hi - lo).astype(np.float32)
    return lo, np.float32(ext.max())


def _spread(c: np.ndarray) -> np.ndarray:
    """Bits k of c moved to bit 3 k (21-bit coordinates)."""
    c = c.astype(np.uint64) & np.uint64(0x1FFFFF)
    c = (c | (c << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    c = (c | (c << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    c = (c | (c << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    c = (c | (c << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    c = (c | (c << np.uint64(2))) & np.uint64(0x1249249249249249)
    return c


def morton_keys(pos4: np.ndarray, lo: np.ndarray, size: np.float32) -> np.ndarray:
    """63-bit keys: c_a = min(floor((x_a - lo_a) * s), 2^21 - 1) with
    s = 2^21 / size, every operation an FP32 round-to-nearest step; x in bit
    3k + 2, y in bit 3k + 1, z in bit 3k."""
    x = np.asarray(pos4, np.float32)[:, :3]
    s = np.float32(2097152.0) / size if size > 0 else np.float32(0.0)
    with np.errstate(invalid="ignore", over="ignore"):
        t = np.floor((x - lo[None, :].astype(np.float32)) * np.float32(s))
    c = np.minimum(t, np.float32(2097151.0)).astype(np.uint64)
    return (_spread(c[:, 0]) << np.uint64(2)) | (_spread(c[:, 1]) << np.uint64(1)) | _spread(c[:, 2])


def _allreduce_counts(vals: np.ndarray, group=None) -> np.ndarray:
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals.astype(np.int64))
    dist.all_reduce(t, group=group)
    return t.numpy()


def split_points(keys: np.ndarray, gid: np.ndarray, n_total: int, n_ranks: int, group=None):
    """Boundaries (key_b, id_b) of the equal-count split of the global
    (key, id) order: rank r owns (key, id) with b_r <= (key, id) < b_{r+1},
    b_0 = (0, 0), b_P = (2^63, 0).  Bisection on the key for each target
    position t_r = r N / P, then on the id among the particles of the
    boundary key; every rank runs the same rounds (one all-reduce each)."""
    m = n_ranks - 1
    targets = np.array([(r + 1) * n_total // n_ranks for r in range(m)], np.int64)
    if m == 0:
        return []
    ks = np.sort(keys)
    lo_k = np.zeros(m, np.uint64)
    hi_k = np.full(m, np.uint64(1) << np.uint64(63), np.uint64)
    # smallest key k with count(key <= k) > t: then count(key < k) <= t
    while True:
        active = hi_k - lo_k > np.uint64(0)
        if not active.any():
            break
        mid = lo_k + (hi_k - lo_k) // np.uint64(2)
        below_eq = np.searchsorted(ks, mid, side="right").astype(np.int64)
        cnt = _allreduce_counts(below_eq, group)
        go_left = cnt > targets
        hi_k = np.where(active & go_left, mid, hi_k)
        lo_k = np.where(active & ~go_left, mid + np.uint64(1), lo_k)
    kb = lo_k                                          # the boundary key of each target
    below = _allreduce_counts(np.searchsorted(ks, kb, side="left").astype(np.int64), group)
    need = targets - below                             # particles of key kb before the boundary
    # among particles of key kb, the boundary id b: count(id < b) == need
    # (the smallest b with count(id < b) >= need; ids are distinct)
    ids = [np.sort(gid[keys == kb[q]]) for q in range(m)]
    lo_i = np.zeros(m, np.int64)
    hi_i = np.full(m, np.int64(1) << np.int64(62))
    while True:
        active = hi_i > lo_i
        if not active.any():
            break
        mid = lo_i + (hi_i - lo_i) // 2
        c = np.array([np.searchsorted(ids[q], mid[q], side="left") for q in range(m)], np.int64)
        cnt = _allreduce_counts(c, group)
        go_left = cnt >= need
        hi_i = np.where(active & go_left, mid, hi_i)
        lo_i = np.where(active & ~go_left, mid + 1, lo_i)
    return [(np.uint64(kb[q]), int(lo_i[q])) for q in range(m)]


def owner_of(keys: np.ndarray, gid: np.ndarray, bounds) -> np.ndarray:
    """Rank of each particle under the split boundaries."""
    own = np.zeros(len(keys), np.int64)
    for kb, ib in bounds:
        after = (keys > kb) | ((keys == kb) & (gid >= ib))
        own += after.astype(np.int64)
    return own


def _exchange(send: list, group=None):
    """Point-to-point all-to-all of float64 / int64 numpy arrays: send[q] goes
    to rank q; returns the list of arrays received from each rank."""
    import torch
    import torch.distributed as dist
    rank, size = dist.get_rank(group), dist.get_world_size(group)
    sizes = torch.tensor([a.size for a in send], dtype=torch.int64)
    all_sizes = [torch.zeros(size, dtype=torch.int64) for _ in range(size)]
    dist.all_gather(all_sizes, sizes, group=group)
    recv = [None] * size
    reqs = []
    bufs = {}
    for q in range(size):
        if q == rank:
            recv[q] = send[q].copy()
            continue
        n_in = int(all_sizes[q][rank])
        bufs[q] = torch.empty(n_in, dtype=torch.float64)
        reqs.append(dist.irecv(bufs[q], src=q, group=group))
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(send[q], np.float64)), dst=q,
                               group=group))
    for r in reqs:
        r.wait()
    for q, b in bufs.items():
        recv[q] = b.numpy()
    return recv


@dataclass
class Domain:
    """One rank's particles after the decomposition: owned first, then halo.

    pos, vel [n, 4] float32 (x, y, z, m / vx, vy, vz, u), h [n] float32,
    gid [n] global ids, n_own owned particles (a contiguous range of the
    global (key, id) order), halo_from[k] the rank that owns halo particle k."""
    pos: np.ndarray
    vel: np.ndarray
    h: np.ndarray
    gid: np.ndarray
    keys: np.ndarray
    n_own: int
    halo_from: np.ndarray
    box_lo: np.ndarray
    box_hi: np.ndarray
    h_max: float
    pad: float
    support: float = 2.0


def _pack(pos, vel, h, gid):
    return np.concatenate([pos.astype(np.float64), vel.astype(np.float64), h[:, None].astype(np.float64),
                           gid[:, None].astype(np.float64)], axis=1)


def _unpack(a):
    a = a.reshape(-1, 10)
    return (a[:, 0:4].astype(np.float32), a[:, 4:8].astype(np.float32), a[:, 8].astype(np.float32),
            a[:, 9].astype(np.int64))


def box_distance(x: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Euclidean distance of each point to the box [lo, hi] (0 inside)."""
    d = np.maximum(0.0, np.maximum(lo[None, :] - x, x - hi[None, :]))
    return np.sqrt(np.sum(d * d, axis=1))


def decompose(pos, vel, h, gid, pad=0.03, group=None, support=2.0) -> Domain:
    """Redistribute this rank's particles (any initial split) into the
    equal-count Morton ranges and attach the halo (support: the kernel's
    support radius in units of h)."""
    import torch.distributed as dist
    rank, size = dist.get_rank(group), dist.get_world_size(group)
    pos = np.asarray(pos, np.float32)
    vel = np.asarray(vel, np.float32)
    h = np.asarray(h, np.float32)
    gid = np.asarray(gid, np.int64)
    lo, ext = bounding_box(pos, group)
    keys = morton_keys(pos, lo, ext)
    n_total = int(_allreduce_counts(np.array([len(pos)], np.int64), group)[0])
    bounds = split_points(keys, gid, n_total, size, group)
    own = owner_of(keys, gid, bounds)
    send = [_pack(pos[own == q], vel[own == q], h[own == q], gid[own == q]).ravel() for q in range(size)]
    recv = _exchange(send, group)
    p_, v_, h_, g_ = zip(*[_unpack(a) for a in recv])
    pos, vel, h, gid = (np.concatenate(p_), np.concatenate(v_), np.concatenate(h_), np.concatenate(g_))
    keys = morton_keys(pos, lo, ext)
    order = np.lexsort((gid, keys))
    pos, vel, h, gid, keys = pos[order], vel[order], h[order], gid[order], keys[order]
    return attach_halo(pos, vel, h, gid, keys, pad, group, support)


def attach_halo(pos, vel, h, gid, keys, pad=0.03, group=None, support=2.0) -> Domain:
    """Select and exchange the halo of owned particles (pos ... keys) with
    the rule of the module docstring."""
    import torch
    import torch.distributed as dist
    rank, size = dist.get_rank(group), dist.get_world_size(group)
    x = pos[:, :3].astype(np.float64)
    box_lo = x.min(0) if len(x) else np.full(3, np.inf)
    box_hi = x.max(0) if len(x) else np.full(3, -np.inf)
    h_max = float(h.max()) if len(h) else 0.0
    mine = torch.tensor(np.concatenate([box_lo, box_hi, [h_max]]))
    allb = [torch.zeros(7, dtype=torch.float64) for _ in range(size)]
    dist.all_gather(allb, mine, group=group)
    send = []
    for q in range(size):
        if q == rank:
            send.append(np.zeros(0))
            continue
        b = allb[q].numpy()
        reach = support * np.maximum(b[6], h.astype(np.float64)) * (1.0 + pad)
        sel = box_distance(x, b[0:3], b[3:6]) < reach
        send.append(_pack(pos[sel], vel[sel], h[sel], gid[sel]).ravel())
    recv = _exchange(send, group)
    halo = [(_unpack(recv[q]), q) for q in range(size) if q != rank]
    hp = [a[0] for a, _ in halo]
    hv = [a[1] for a, _ in halo]
    hh = [a[2] for a, _ in halo]
    hg = [a[3] for a, _ in halo]
    hf = [np.full(len(a[3]), q, np.int64) for a, q in halo]
    cat = lambda own, extra: np.concatenate([own] + extra) if extra else own
    return Domain(pos=cat(pos, hp), vel=cat(vel, hv), h=cat(h, hh), gid=cat(gid, hg), keys=keys,
                  n_own=len(pos), halo_from=cat(np.zeros(0, np.int64), hf), box_lo=box_lo,
                  box_hi=box_hi, h_max=h_max, pad=pad, support=support)


def refresh_halo(dom: Domain, fields: dict, h_start: np.ndarray, group=None):
    """After a pass over the owned particles, send each halo particle's new
    per-particle values (fields: name -> array over the owned particles,
    e.g. h, rho, omega) from its owner to the ranks holding it.  Returns
    (halo values by field, outgrew) where outgrew is True on every rank if
    some owned h anywhere grew past h_start (1 + pad): the halo selection
    then no longer covers the sets and must be redone."""
    import torch.distributed as dist
    rank, size = dist.get_rank(group), dist.get_world_size(group)
    names = sorted(fields)
    own_vals = np.stack([np.asarray(fields[k], np.float64) for k in names], axis=1)
    grew = np.any(np.asarray(fields.get("h", h_start)) > h_start[: dom.n_own] * (1.0 + dom.pad))
    flag = int(_allreduce_counts(np.array([1 if grew else 0], np.int64), group)[0]) > 0
    # requests: each rank asks the owners for the ids of its halo particles
    want = [dom.gid[dom.n_own:][dom.halo_from == q].astype(np.float64) for q in range(size)]
    asked = _exchange(want, group)
    index = {int(g): k for k, g in enumerate(dom.gid[: dom.n_own])}
    reply = []
    for q in range(size):
        ids = asked[q].astype(np.int64)
        reply.append(own_vals[[index[int(g)] for g in ids]].ravel() if len(ids) else np.zeros(0))
    got = _exchange(reply, group)
    out = {k: np.zeros(len(dom.gid) - dom.n_own) for k in names}
    for q in range(size):
        if q == rank:
            continue
        sel = np.where(dom.halo_from == q)[0]
        vals = got[q].reshape(-1, len(names)) if len(sel) else np.zeros((0, len(names)))
        for c, k in enumerate(names):
            out[k][sel] = vals[:, c]
    return out, flag
