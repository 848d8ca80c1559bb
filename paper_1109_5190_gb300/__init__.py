"""GB300-native Barnes-Hut hot path (arXiv:1109.5190).

The computation lives in the CUDA library ``libbh.so`` (C ABI in
``include/bh.h``); :mod:`.binding` is its thin ctypes binding and
:class:`System` a small convenience wrapper.  There is no CPU fallback:
importing the binding fails if the library has not been built.
"""
from __future__ import annotations

from . import binding
from .binding import BHError  # noqa: F401

__all__ = ["binding", "System", "BHError"]


class System:
    """One N-body system resident on the GPU (wraps bh_create / bh_step / ...)."""

    def __init__(self, pos_mass, vel=None, G=1.0, eps=0.01, theta=0.5, potential=False,
                 kahan=True, stream=None):
        flags = (binding.BH_POTENTIAL if potential else 0) | (0 if kahan else binding.BH_NO_KAHAN)
        self.n = (pos_mass.numel() if binding._is_torch(pos_mass) else pos_mass.size) // 4
        self._h = binding.bh_create(binding.params(G, eps, theta, flags), pos_mass, vel, stream)

    def close(self):
        if getattr(self, "_h", None):
            binding.bh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def compute_accel(self, out=None):
        import numpy as np
        if out is None:
            out = np.zeros((self.n, 4), np.float32)
        binding.bh_compute_accel(self._h, out)
        return out

    def build_tree(self):
        binding.bh_build_tree(self._h)

    def tree(self):
        return binding.bh_get_tree(self._h, self.n)

    def step(self, nsteps, dt, use_graph=False):
        binding.bh_step(self._h, nsteps, dt, use_graph)

    def state(self):
        import numpy as np
        pm = np.zeros((self.n, 4), np.float32)
        v = np.zeros((self.n, 4), np.float32)
        a = np.zeros((self.n, 4), np.float32)
        binding.bh_get_state(self._h, pm, v, a)
        return pm, v, a

    def set_state(self, pos_mass, vel=None, acc=None):
        binding.bh_set_state(self._h, pos_mass, vel, acc)

    def diagnostics(self):
        return binding.bh_diagnostics(self._h)

    def interaction_count(self):
        return binding.bh_interaction_count(self._h, self.n)

    def autotune(self):
        return binding.bh_autotune(self._h)

    def set_tuning(self, ppl=2, warps_per_block=8, blocks_per_sm=0):
        binding.bh_set_tuning(self._h, ppl, warps_per_block, blocks_per_sm)
