"""The plan autotuner and the schedule variants of the 2-D step.

Every schedule variant (row-pass block shape; column-pass radix schedule and
block shape; replicas per column block; pipelined column pass) computes the
same step, so all of them must agree with the default schedule to FP32
rounding, and the default with the oracle (checked by the parity tests, which
run with whatever schedule the autotuner picks).  The autotuner must leave the
context's state untouched and cache its choice per configuration.
"""
import itertools

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


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def stepper(sft, w):
    return sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)


PLAN_CASES = [
    ("model_b_1024_setd2_R3", W.model_b_1024(replicas=3, scheme=2, h=0.025, sigma0=0.3)),
    ("kpz_2d_512_R5", W.kpz_2d(n=[512, 512], replicas=5, sigma0=0.5)),
    ("model_a_64_R9", W.model_a_64(replicas=9, sigma0=0.3)),
]


@pytest.mark.parametrize("name,w", PLAN_CASES, ids=[c[0] for c in PLAN_CASES])
def test_schedule_variants_agree(sft, name, w):
    f0 = W.initial_fields(w).astype(np.float32)
    ref = stepper(sft, w)
    ref.set_field(f0)
    sft.sft_set_plan(ref.ctx, [0, 0, 4, 0])
    ref.step(20)
    want = ref.field()
    ref.close()
    ncol = 3 if w.n[1] >= 512 else 1
    if w.n[1] == 1024 and w.model != W.KPZ:
        ncol = 4  # column schedule 3: one warp per 1024-point column (cubic term)
    pipes = [0, 1] if (w.n[0], w.n[1]) in ((1024, 1024), (2048, 2048)) and w.model != W.KPZ else [0]
    # row schedule 3 (two rows per warp, TMA tiles) is built for 1024-point rows with the cubic term
    nrow = 4 if w.n[0] == 1024 and w.model != W.KPZ else 3
    for row, col, rpb, pipe in itertools.product(range(nrow), range(ncol), (1, 2, 4, 8), pipes):
        if pipe and (col or rpb != 4):
            continue  # the pipelined column pass has one schedule
        g = stepper(sft, w)
        g.set_field(f0)
        sft.sft_set_plan(g.ctx, [row, col, rpb, pipe])
        assert sft.sft_get_plan(g.ctx) == [row, col, rpb, pipe]
        g.step(20)
        got = g.field()
        g.close()
        for r in range(w.replicas):
            assert rel_l2(got[r], want[r]) <= 2e-6, (name, row, col, rpb, pipe, r)


def test_autotuner_leaves_state_and_caches(sft):
    w = W.model_b_1024(n=[512, 512], replicas=4, sigma0=0.3)
    f0 = W.initial_fields(w).astype(np.float32)
    g = stepper(sft, w)
    g.set_field(f0)
    spec0 = g.spectrum()
    plan = sft.sft_get_plan(g.ctx)
    assert 0 <= plan[0] < 3 and 0 <= plan[1] < 3 and plan[2] in (1, 2, 4, 8) and plan[3] in (0, 1)
    assert np.array_equal(g.spectrum(), spec0)
    assert g.step_count == 0
    g2 = stepper(sft, w)
    assert sft.sft_get_plan(g2.ctx) == plan  # cached for the configuration
    g.step(10)
    g2.set_field(f0)
    sft.sft_set_plan(g2.ctx, [0, 0, 4, 0])
    g2.step(10)
    for r in range(w.replicas):
        assert rel_l2(g.field(r), g2.field(r)) <= 2e-6
    with pytest.raises(sft.SftError):
        sft.sft_set_plan(g.ctx, [3, 0, 4, 0])
    with pytest.raises(sft.SftError):
        sft.sft_set_plan(g.ctx, [0, 3, 4, 0])
    g.close()
    g2.close()
