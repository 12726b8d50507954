"""The allocation-free solve (solve_noalloc) against the regular solve.

solve_noalloc exists for callers that may not allocate device memory while
they run (plug-ins inside a host application that owns all device memory, loops
that must not stall on an allocation, fixed device-memory budgets): its workspace is one fixed library
array, sized for stamping sets of at most 32,768 padded rows, shared by every
call.  This file runs last (pytest collects it after the other test files) so
that a failure here leaves every other test already run."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.helpers import rel_l2, stamp_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the solve tolerance of the other parity tests


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_equals_solve_on_two_calls(B, prec):
    inst, af, av, ff, fv = stamp_inputs("cfg1")
    small = W.make_tiny(3, d=3, n_cos=2, n_u=3, N=2)
    _, saf, sav, sff, sfv = stamp_inputs(small)
    with B.stamp_build(af, av, ff, inst.N) as s, B.stamp_build(saf, sav, sff, small.N) as s2:
        f_on, _ = s.scatter(ff, fv)
        f2, _ = s2.scatter(sff, sfv)
        ref, _ = B.solve(s, f_on, 1e-12, 500, prec)
        ref2, _ = B.solve(s2, f2, 1e-12, 500, prec)
        out = torch.empty_like(f_on)
        out2 = torch.empty_like(f2)
        torch.cuda.synchronize()
        for _ in range(2):
            n0 = B.alloc_count()
            u, st = B.solve_noalloc(s, f_on, out, 1e-12, 500, prec)
            # a different, smaller set in between: the shared array is re-initialised
            u2, _ = B.solve_noalloc(s2, f2, out2, 1e-12, 500, prec)
            assert B.alloc_count() == n0, "solve_noalloc called an allocating routine"
            assert st["status"] == "SS_OK"
            assert rel_l2(u.cpu().numpy(), ref.cpu().numpy()) <= TOL
            assert rel_l2(u2.cpu().numpy(), ref2.cpu().numpy()) <= TOL


def test_noalloc_rejects_sets_beyond_its_workspace(B):
    from paper_2302_00752_gb300.binding import SSError
    inst, af, av, ff, fv = stamp_inputs("cfg3")          # |S| = 86,272 > 32,768
    with B.stamp_build(af, av, ff, inst.N) as s:
        f_on, _ = s.scatter(ff, fv)
        with pytest.raises(SSError) as e:
            B.solve_noalloc(s, f_on, torch.empty_like(f_on), 1e-12, 500, "fp64")
        assert e.value.name == "SS_ERR_INVALID"


def test_noalloc_checks_buffer_sizes(B):
    # buffers shorter than |S| (or on another device) are rejected before any
    # kernel could write past them
    inst, af, av, ff, fv = stamp_inputs("cfg1")
    with B.stamp_build(af, av, ff, inst.N) as s:
        f_on, _ = s.scatter(ff, fv)
        with pytest.raises(ValueError):
            B.solve_noalloc(s, f_on, torch.empty(s.size - 1, dtype=torch.complex128, device="cuda"))
        with pytest.raises(ValueError):
            B.solve_noalloc(s, f_on[:-1].contiguous(), torch.empty_like(f_on))
        with pytest.raises(ValueError):
            B.solve(s, f_on, out=torch.empty(s.size - 1, dtype=torch.complex128, device="cuda"))
