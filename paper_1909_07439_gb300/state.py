"""Device particle state held in torch tensors, marshalled to ``sph_state``.

PyTorch is used for device memory and streams only; all computation runs
in libsph.
"""
from __future__ import annotations

import numpy as np

from . import native


class DeviceState:
    """Structure-of-arrays particle state on a CUDA device.

    pos [n,4] = (x, y, z, m), vel [n,4] = (vx, vy, vz, u), acc [n,4] =
    (ax, ay, az, du/dt), h/rho/omega/drhodt/vsigmax [n] float32,
    perm [n] int32 (original index of each slot), keys [n] int64 (Morton keys).
    """

    FIELDS4 = ("pos", "vel", "acc")
    FIELDS1 = ("h", "rho", "omega", "drhodt", "vsigmax")

    def __init__(self, n: int, device="cuda"):
        import torch
        self.n = int(n)
        self.device = torch.device(device)
        z4 = lambda: torch.zeros((max(self.n, 1), 4), dtype=torch.float32, device=self.device)
        z1 = lambda: torch.zeros(max(self.n, 1), dtype=torch.float32, device=self.device)
        self.pos, self.vel, self.acc = z4(), z4(), z4()
        self.h, self.rho, self.omega, self.drhodt, self.vsigmax = z1(), z1(), z1(), z1(), z1()
        self.perm = torch.arange(max(self.n, 1), dtype=torch.int32, device=self.device)
        self.keys = torch.zeros(max(self.n, 1), dtype=torch.int64, device=self.device)

    @classmethod
    def from_arrays(cls, pos, vel, h, device="cuda"):
        import torch
        s = cls(len(pos), device)
        if s.n:
            s.pos.copy_(torch.as_tensor(np.ascontiguousarray(pos, np.float32)))
            s.vel.copy_(torch.as_tensor(np.ascontiguousarray(vel, np.float32)))
            s.h.copy_(torch.as_tensor(np.ascontiguousarray(h, np.float32)))
        return s

    @property
    def c(self) -> native.sph_state:
        st = native.sph_state()
        st.n = self.n
        for f in self.FIELDS4 + self.FIELDS1 + ("perm", "keys"):
            setattr(st, f, getattr(self, f).data_ptr())
        return st

    def numpy(self, field):
        return getattr(self, field)[: self.n].cpu().numpy()

    def in_original_order(self, field):
        """Field values re-indexed by the particles' original index."""
        a = self.numpy(field)
        out = np.empty_like(a)
        out[self.numpy("perm")] = a
        return out
