"""Test helper: the FP64 oracle with every operator output rounded to FP32.

Used to size tolerances where a fixed FIRLS schedule is ill-conditioned: the
error this emulation shows against the plain FP64 oracle is the error any
FP32 evaluation of the same algorithm incurs on that input.  Test
infrastructure only (imports the oracle; never used by the library).
"""
import numpy as np

from oracle import firls_oracle as O


def r32(x):
    if np.iscomplexobj(x):
        return x.astype(np.complex64).astype(np.complex128)
    return x.astype(np.float32).astype(np.float64)


class System32(O.System):
    def apply_S(self, x):
        return r32(super().apply_S(r32(x)))

    def apply_Pinv(self, r):
        return r32(super().apply_Pinv(r32(r)))

    def update_weights(self, x):
        super().update_weights(r32(x))
        if self.w is not None:
            self.w = r32(self.w)
        if self.pinv is not None:
            self.pinv = r32(self.pinv)


def one_outer_step_fp32_error(p, x, inner):
    """Relative difference between an FP32-rounded and an FP64 outer step from x."""
    out = []
    for cls in (O.System, System32):
        s = cls(p.mask, p.real, p.psi, p.levels, p.lam, p.lam_tv, p.groups)
        rhs = O.op_AH(p.mask * p.b, p.mask.astype(float), p.real)
        xx = x
        if cls is System32:
            rhs, xx = r32(rhs), r32(x)
        s.update_weights(xx)
        y, _ = O.pcg(s, rhs, xx, inner, 0.0, 1.0)
        out.append(y)
    return float(np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]))
