"""Element-wise comparison of an FP32 GPU step with the FP64 oracle, allowing
for the one hard decision of the step: the Shamov gate (Eq. 5), which turns
the Grass load (Eq. 3) on when |v|^6 > C_Sh^6 d50^2 H.

The GPU takes that decision in FP32, the oracle in FP64; a cell whose
transport velocity sits within FP32 rounding of the critical velocity can be
gated differently, and its load, O(A_J v_k^3), then moves the bed of it and
its neighbours by far more than rounding.  So the oracle is also evaluated
at the two edges of the decision band -- the sixth-power criterion scaled by
1 -/+ 3e-5 (C_Sh scaled by 1 -/+ 5e-6), wider than the FP32 error of that
chain (a few 1e-6) -- and an element passes when it lies within the bound of
any of the three results.  Away from the band the three results coincide,
so everywhere else this is the plain element-wise bound.
"""
import dataclasses

import numpy as np

C_SH_BAND = 5e-6


def band_params(p):
    """The oracle parameters at the threshold and at the band's two edges."""
    return [p] + [dataclasses.replace(p, C_Sh=p.C_Sh * f) for f in (1.0 - C_SH_BAND, 1.0 + C_SH_BAND)]


def fp32_bound(ref_q, q):
    """Per-step FP32 bound: 4e-5 m on H and b, 4e-5 m^2/s + 2e-5 |Hu| on momenta."""
    return 4e-5 + (2e-5 * np.abs(ref_q) if q in (1, 2) else 0.0)


def band_error(got, outs, q):
    """Per element, the smallest excess over the bound among the oracle
    results in outs (lists of 4 arrays); <= 0 passes.  Also returns the plain
    error against outs[0]."""
    g = np.asarray(got, dtype=np.float64)
    excess = None
    for o in outs:
        e = np.abs(g - o[q]) - fp32_bound(o[q], q)
        excess = e if excess is None else np.minimum(excess, e)
    return excess, np.abs(g - outs[0][q])
