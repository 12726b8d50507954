"""Shared helpers of the parity tests (inputs from workloads.py, expected
values from the oracle only)."""
import numpy as np

import workloads as W
from oracle import pipeline as opipe
from oracle.sft import true_coefficients


def coeff_arrays(dct):
    keys = sorted(dct)
    return np.array(keys, np.int64).reshape(len(keys), -1), np.array([dct[k] for k in keys], np.complex128)


def true_a(inst):
    """Exact Fourier coefficients of the workload's a (oracle definition)."""
    return coeff_arrays(true_coefficients(inst.a.freq, inst.a.coef))


def true_f(inst):
    """Exact Fourier coefficients of f: the given sum, or the oracle's
    convolution for manufactured instances (exact zeros dropped)."""
    if inst.f is not None:
        return coeff_arrays(true_coefficients(inst.f.freq, inst.f.coef))
    ff, fv = opipe.forcing(inst)
    keep = np.abs(fv) > 0
    return ff[keep], fv[keep]


def stamp_inputs(name_or_inst):
    inst = W.CONFIGS[name_or_inst]() if isinstance(name_or_inst, str) else name_or_inst
    af, av = true_a(inst)
    ff, fv = true_f(inst)
    return inst, af, av, ff, fv


def rel_l2(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))
