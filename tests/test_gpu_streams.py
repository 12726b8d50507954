"""Library calls on alternating CUDA streams give the same bits as on the
default stream: the per-thread scratch that holds call-local temporaries of
the lattice, recovery and stamping paths is reused in stream order, and a
call on another stream first waits for the previous stream's use of it."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import lattice as olat
from oracle import pipeline as opipe
from tests.helpers import stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def test_recovery_and_stamp_on_alternating_streams(B):
    inst = W.make_cfg3()
    cand = opipe.candidates(inst, inst.f.freq)
    z, M, _ = olat.random_lattice(cand, inst.lattice)
    _, af, av, ff, fv = stamp_inputs(inst)

    def run():
        out = []
        for trig in (inst.a, inst.f):
            gf, gv = B.sft_recover(z, M, trig.freq, trig.coef, cand, tau=1e-9)
            out += [gf.clone(), gv.clone()]
        s = B.stamp_build(af, av, ff, inst.N)
        S, lv = s.export()
        out += [S.clone(), lv.clone()]
        s.destroy()
        return out

    ref = run()
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(6):
        st = streams[k % 2]
        with torch.cuda.stream(st):
            got = run()
        st.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)


def test_one_call_pipeline_on_alternating_streams(B):
    from paper_2302_00752_gb300 import pipeline as gp
    p = gp.prepare(W.make_cfg1())
    ref = gp.run_fused(p)
    ref_u = ref.u.clone()
    ref.stamp.destroy()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(4):
        st = streams[k % 2]
        with torch.cuda.stream(st):
            r = gp.run_fused(p)
            u = r.u.clone()
        st.synchronize()
        try:
            assert r.stats["status"] == "SS_OK" and torch.equal(u, ref_u)
        finally:
            r.stamp.destroy()
