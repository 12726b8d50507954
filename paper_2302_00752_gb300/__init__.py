"""Single-GPU (sm_103a) sparse spectral method of Gross & Iwen (arXiv 2302.00752)
for -div(a grad u) = f on the d-torus.

The compute path is the CUDA library libsparse_spectral.so (C ABI in
include/sparse_spectral.h); ``binding`` exposes it with the same names and
``pipeline`` strings the calls together as Algorithm 1.  The binding is loaded
on first use of one of its names (``build`` can run before the library exists).
"""
import importlib

_EXPORTS = ("SS_FP32", "SS_FP64", "SS_DF64", "Batch", "SSError", "Stamp", "galerkin_apply", "lattice_cbc", "lattice_check",
            "lattice_random", "lattice_sample", "lattice_size", "sft_recover", "sft_identify", "sft_identify_samples", "sft_recover_samples", "solve",
            "stamp_build", "stamp_build_adr", "version", "proxy_residual", "proxy_mc", "solve_noalloc",
            "sparse_spectral_solve")

__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        return getattr(importlib.import_module(".binding", __name__), name)
    raise AttributeError(name)
