"""Batched persistent solve: many instances of uneven d, |supp a_hat| and |S| in
one cooperative launch (optionally replayed from a CUDA graph) give the same
solutions as the oracle, instance by instance (relative l2 <= 1e-10)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pipeline as opipe
from tests.helpers import rel_l2, stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def instances():
    # small members of the batched workload family (|S| from 100 to 3000)
    return [W.make_batch_instance(7, i, lo=100, hi=3000) for i in range(12)]


@pytest.fixture(scope="module")
def built(B, instances):
    stamps, fs, refs = [], [], []
    for inst in instances:
        _, af, av, ff, fv = stamp_inputs(inst)
        s = B.stamp_build(af, av, ff, inst.N)
        f_on, _ = s.scatter(ff, fv)
        stamps.append(s)
        fs.append(f_on)
        refs.append(opipe.solve_recovered(inst.N, af, av, ff, fv, tol=1e-14))
    yield stamps, fs, refs
    for s in stamps:
        s.destroy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(B, built, prec, use_graph):
    stamps, fs, refs = built
    batch = B.Batch(stamps)
    us, stats = batch.solve(fs, tol=1e-12, max_iter=500, precision=prec, use_graph=use_graph)
    for u, st, ref in zip(us, stats, refs):
        assert st["status"] == "SS_OK"
        assert rel_l2(u.cpu().numpy(), ref.u) < 1e-10
    # a second call replays (graph) and is bit-identical
    us2, _ = batch.solve(fs, tol=1e-12, max_iter=500, precision=prec, use_graph=use_graph)
    for a, b in zip(us, us2):
        assert torch.equal(a, b)
    batch.destroy()


def test_batch_equals_single_solves(B, built):
    stamps, fs, _ = built
    batch = B.Batch(stamps)
    us, _ = batch.solve(fs, tol=1e-12, max_iter=500, precision="fp64", use_graph=False)
    for s, f, u in zip(stamps, fs, us):
        u1, _ = B.solve(s, f, 1e-12, 500, "fp64")
        assert rel_l2(u.cpu().numpy(), u1.cpu().numpy()) < 1e-11
    batch.destroy()


def test_autotune_and_config(B, built):
    stamps, fs, refs = built
    batch = B.Batch(stamps)
    ms, cfg = batch.autotune(fs, tol=1e-12, max_iter=500, precision="fp32")
    assert ms > 0 and cfg["block"] in (128, 256, 512) and cfg["grid"] >= 1
    us, stats = batch.solve(fs, tol=1e-12, max_iter=500, precision="fp32", use_graph=True)
    for u, ref in zip(us, refs):
        assert rel_l2(u.cpu().numpy(), ref.u) < 1e-10
    batch.set_config(128, 1, 2)
    us, stats = batch.solve(fs, tol=1e-12, max_iter=500, precision="fp32", use_graph=False)
    for u, ref in zip(us, refs):
        assert rel_l2(u.cpu().numpy(), ref.u) < 1e-10
    batch.destroy()


def test_half_batch_equals_full_batch(B, built):
    stamps, fs, refs = built
    batch = B.Batch(stamps)
    try:
        for prec in ("fp64", "fp32"):
            us_h, st_h = batch.solve(fs, tol=1e-12, precision=prec)
            batch.set_symmetry(False)
            us_f, st_f = batch.solve(fs, tol=1e-12, precision=prec)
            batch.set_symmetry(True)
            assert all(s["half_system"] for s in st_h) and not any(s["half_system"] for s in st_f)
            for uh, uf, s in zip(us_h, us_f, st_h):
                assert s["status"] == "SS_OK"
                assert rel_l2(uh.cpu().numpy(), uf.cpu().numpy()) < 1e-11
    finally:
        batch.destroy()


def test_half_batch_falls_back_for_a_non_hermitian_f(B, built):
    stamps, fs, refs = built
    fs2 = [f.clone() for f in fs]
    nz = torch.nonzero(fs2[3].abs() > 0).flatten()
    fs2[3][nz[0]] *= 1 + 1e-9
    batch = B.Batch(stamps)
    try:
        us, st = batch.solve(fs2, tol=1e-12, precision="fp64")
        assert not any(s["half_system"] for s in st)
        batch.set_symmetry(False)
        us_f, _ = batch.solve(fs2, tol=1e-12, precision="fp64")
        for a, b in zip(us, us_f):
            assert torch.equal(a, b)
    finally:
        batch.destroy()
