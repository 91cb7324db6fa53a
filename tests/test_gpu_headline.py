"""Field parity on the headline lattice over the full 100-step horizon.

Model B, 1024^2, h = 0.05, two replicas, each scheme (SETD-EM, SETD1, SETD2),
stepped 100 times on the GPU and by the FP64 oracle from the same FP32 initial
fields, under every schedule a run can take on this lattice: the one the plan
autotuner picks (what the bench times), the default schedule, and each
row-pass schedule built for 1024-point rows.

Bounds (the method's FP32 accuracy gate, Sec. IV with the FP32 path): relative
L2 of the real-space field <= 1e-5 per replica, and, so that one wrong mode
cannot hide under the norm, every stored mode within 1e-4 of the RMS mode
amplitude: max_a |Phi_gpu - Phi_oracle| / rms_a |Phi_oracle| <= 1e-4.

The oracle runs one context per replica (replica offsets 0 and 1) in threads;
its C library is entered through ctypes, which releases the GIL.
"""
import threading

import numpy as np
import pytest

import sft_inputs as W

pytestmark = pytest.mark.gpu

NSTEPS = 100


@pytest.fixture(scope="module")
def sft():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_22510_gb300 as m
    m.load_library()
    return m


def half_xmajor(full):
    nx = full.shape[-1]
    return np.moveaxis(full[..., : nx // 2 + 1], -1, 0)


def oracle_run(oracle_mod, w, f32):
    """Step one R = 1 oracle per replica in parallel threads; return (fields, spectra)."""
    R = f32.shape[0]
    out = [None] * R
    errs = []

    def one(r):
        try:
            o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                                  replica0=r)
            o.set_field(0, f32[r].astype(np.float64))
            o.step(NSTEPS)
            out[r] = (o.field(0), half_xmajor(o.spectrum(0)))
        except Exception as ex:  # reported in the main thread
            errs.append(ex)

    th = [threading.Thread(target=one, args=(r,)) for r in range(R)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return out


def check(got_field, got_spec, ref_field, ref_spec, tag):
    e = float(np.linalg.norm(got_field - ref_field) / np.linalg.norm(ref_field))
    rms = float(np.sqrt(np.mean(np.abs(ref_spec) ** 2)))
    emax = float(np.max(np.abs(got_spec - ref_spec))) / rms
    assert e <= 1e-5, (tag, "relative L2", e)
    assert emax <= 1e-4, (tag, "max mode error / rms", emax)
    return e, emax


@pytest.mark.parametrize("scheme", [0, 1, 2], ids=["setd_em", "setd1", "setd2"])
def test_headline_100_steps(sft, oracle_mod, scheme):
    w = W.model_b_1024(replicas=2, h=0.05, scheme=scheme)
    f32 = W.initial_fields(w).astype(np.float32)
    ref = oracle_run(oracle_mod, w, f32)
    plans = [None, [0, 0, 4, 0]]  # None: the autotuner's choice
    probe = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for row, col in [(1, 0), (2, 0), (3, 0), (0, 3), (3, 3)]:
        try:
            sft.sft_set_plan(probe.ctx, [row, col, 2, 0])
            plans.append([row, col, 2, 0])
        except sft.SftError:
            pass
    probe.close()
    # the two-rows-per-warp row pass and the warp-per-column column pass are built for 1024-point lines
    assert [3, 0, 2, 0] in plans and [0, 3, 2, 0] in plans and [3, 3, 2, 0] in plans
    for plan in plans:
        g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
        g.set_field(f32)
        if plan is not None:
            sft.sft_set_plan(g.ctx, plan)
        g.step(NSTEPS)
        field, spec = g.field(), g.spectrum()
        used = sft.sft_get_plan(g.ctx)
        g.close()
        for r in range(w.replicas):
            check(field[r], spec[r], ref[r][0], ref[r][1], (scheme, plan, used, r))
