"""Error measures used by the parity tests.

Per-particle acceleration error against the FP64 oracle:
  e_i = |a_gpu,i - a_ref,i| / |a_ref,i|                (for the p99 gate)
  e_max = max_i |a_gpu,i - a_ref,i| / max(|a_ref,i|, 1e-3 rms|a_ref|)
The floor keeps particles with near-zero net force (where any absolute
error is a large relative one) from dominating the max.
"""
import numpy as np

P99_TOL = 1e-5
MAX_TOL = 1e-3


def accel_errors(a_gpu, a_ref):
    a_gpu = np.asarray(a_gpu, dtype=np.float64)[:, :3]
    a_ref = np.asarray(a_ref, dtype=np.float64)[:, :3]
    d = np.linalg.norm(a_gpu - a_ref, axis=1)
    r = np.linalg.norm(a_ref, axis=1)
    if r.size == 0:
        return 0.0, 0.0
    rms = np.sqrt(np.mean(r * r))

    def ratio(num, den):
        # 0/0 (an exactly zero force reproduced exactly) is no error
        out = np.zeros_like(num)
        nz = num > 0
        with np.errstate(divide="ignore"):
            out[nz] = num[nz] / den[nz]
        return out

    rel = ratio(d, r)
    relmax = ratio(d, np.maximum(r, 1e-3 * rms))
    return float(np.percentile(rel, 99)), float(relmax.max())


def assert_accel_close(a_gpu, a_ref, p99=P99_TOL, mx=MAX_TOL, what=""):
    e99, emax = accel_errors(a_gpu, a_ref)
    assert e99 <= p99 and emax <= mx, f"{what}: p99 {e99:.3e} (tol {p99}), max {emax:.3e} (tol {mx})"
    return e99, emax
