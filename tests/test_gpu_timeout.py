"""Failure detection of the bounded device-side waits, without a GPU fault.

Kernels that wait on an mbarrier for their own bulk/TMA copies (the
two-rows-per-warp row pass, the pipelined column pass and the warp row pass
of complex fields) bound every wait;
a wait that runs out sets the time-out bit of the context's status word, lets
its copies in flight land and returns, and the next synchronising call reports
SFT_ETIMEOUT.  SFT_WAIT_LIMIT=-1 in the environment of a new context gives its
waits no iterations at all, so the first wait of a launch runs out while its
(ordinary, in-bounds) copy is still in flight.  Afterwards the device must
still answer: a new context with the default limit steps and matches the
oracle.
"""
import numpy as np
import pytest

import sft_inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sft():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_22510_gb300 as m
    m.load_library()
    return m


def stepper(sft, w):
    return sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)


@pytest.mark.parametrize("plan", [[3, 0, 4, 0], [0, 0, 4, 1]], ids=["tma_row_pass", "pipelined_column_pass"])
def test_wait_runs_out_and_the_device_stays_usable(sft, oracle_mod, plan, monkeypatch):
    w = W.model_b_1024(replicas=2, sigma0=0.3)
    f0 = W.initial_fields(w).astype(np.float32)
    monkeypatch.setenv("SFT_WAIT_LIMIT", "-1")
    g = stepper(sft, w)
    sft.sft_set_plan(g.ctx, plan)
    g.set_field(f0)
    with pytest.raises(sft.SftError) as ei:
        g.step(1)
        g.sync()
    assert ei.value.status == sft.SFT_ETIMEOUT
    g.close()
    monkeypatch.delenv("SFT_WAIT_LIMIT")
    g = stepper(sft, w)
    sft.sft_set_plan(g.ctx, plan)
    g.set_field(f0)
    g.step(3)
    got = g.field()
    g.close()
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(w.replicas):
        o.set_field(r, f0[r].astype(np.float64))
    o.step(3)
    for r in range(w.replicas):
        ref = o.field(r)
        assert np.linalg.norm(got[r] - ref) / np.linalg.norm(ref) <= 1e-5


def test_complex_warp_row_pass_wait_runs_out(sft, oracle_mod, monkeypatch):
    """The same on the complex (CGL) step at 1024^2 under 2/3 truncation, whose
    row pass loads its tiles by TMA."""
    w = W.cgl_2048(n=[1024, 1024], replicas=2)
    f0 = W.initial_fields(w).astype(np.complex64)
    monkeypatch.setenv("SFT_WAIT_LIMIT", "-1")
    g = stepper(sft, w)
    g.set_field(f0)
    with pytest.raises(sft.SftError) as ei:
        g.step(1)
        g.sync()
    assert ei.value.status == sft.SFT_ETIMEOUT
    g.close()
    monkeypatch.delenv("SFT_WAIT_LIMIT")
    g = stepper(sft, w)
    g.set_field(f0)
    g.step(3)
    got = g.field().astype(np.complex128)
    g.close()
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(w.replicas):
        o.set_field(r, f0[r].astype(np.complex128))
    o.step(3)
    for r in range(w.replicas):
        ref = o.field(r)
        assert np.linalg.norm(got[r] - ref) / np.linalg.norm(ref) <= 1e-5
