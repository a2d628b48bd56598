"""Device buffers for one particle set: torch CUDA tensors for the inputs and outputs, wrapped
into the C structs of evol.py.  Allocation and copies only; the computation is in libevol.so."""
from __future__ import annotations

import numpy as np
import torch

from . import evol as E

OUT_LEN_GAS = {"rho", "P", "c", "omega", "zeta", "dudt", "dalpha", "dalpha_u"}


class DeviceSet:
    """Inputs of a workload on `device` plus output tensors, and the matching C structs."""

    def __init__(self, w, params=None, device="cuda:0", outputs=None, precision=None, pinned_host=False):
        self.w = w
        self.n, self.n_gas = w.n, w.n_gas
        p = params or w.params
        self.params_py = p
        self.params = E.make_params(p)
        if precision is not None:
            self.params.precision = int(precision)
        self.device = torch.device(device)
        self.inp = {}
        for k, a in w.arrays().items():
            t = torch.from_numpy(np.ascontiguousarray(a, np.float32))
            if k in ("u", "h"):
                t = t[: max(self.n_gas, 1)].clone() if self.n_gas > 0 else t[:1].clone()
            self.inp[k] = t.to(self.device)
        for k in ("alpha", "alpha_u"):        # per-particle dissipation inputs (gas), when the workload has them
            a = getattr(w, k, None)
            if a is not None and self.n_gas > 0:
                self.inp[k] = torch.from_numpy(np.ascontiguousarray(a[: self.n_gas], np.float32)).to(self.device)
        names = outputs if outputs is not None else E.OUTPUT_FIELDS
        self.out = {}
        for k in names:
            ln = self.n_gas if k in OUT_LEN_GAS else self.n
            self.out[k] = torch.zeros(max(ln, 1), dtype=torch.float32, device=self.device)
        self.particles = E.make_particles(self.n, self.n_gas, self.inp)
        self.outputs = E.make_outputs(self.out)
        # the starting guesses of h and eps, kept on the device: restoring them before a step is a
        # device copy, which needs no host synchronisation between steps
        self._start = {k: self.inp[k].clone() for k in ("h", "eps")}

    def reset_lengths(self):
        """Restore the caller's starting guesses for h and eps (the step overwrites them)."""
        for k in ("h", "eps"):
            self.inp[k].copy_(self._start[k])

    def numpy(self) -> dict:
        res = {k: v.detach().cpu().numpy().astype(np.float64)[: (self.n_gas if k in OUT_LEN_GAS else self.n)]
               for k, v in self.out.items()}
        res["h"] = self.inp["h"].cpu().numpy().astype(np.float64)[: self.n_gas]
        res["eps"] = self.inp["eps"].cpu().numpy().astype(np.float64)
        return res
