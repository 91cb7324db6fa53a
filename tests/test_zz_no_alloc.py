"""The allocation-free 2-D step entry point, for callers that cannot call
cudaMalloc (their runtime owns the allocator, or allocation is forbidden after
start-up).  Through the C ABI it must give what the context-based entry point
gives on the same input, on two calls in a row (the second continuing the
first: later noise counters, SETD2 history carried in the caller's buffer).
Both run the same kernels with the same tables when the context is held to the
default schedule, so the comparison is bit for bit; a replica offset (the
noise counter of sharded runs) and a state that turns non-finite are covered
too.

This file is collected last on purpose, and passes alone in a fresh process
as well as after every other test."""
import numpy as np
import pytest

import sft_inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_22510_gb300 as m
    m.load_library()
    return m, torch


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("w,rep0", [
    (W.model_b_1024(n=[64, 64], replicas=3, sigma0=0.3, scheme=2, h=0.025), 0),
    (W.kpz_2d(n=[32, 32], replicas=2, sigma0=0.4), 0),
    (W.model_a_64(n=[128, 128], replicas=2, scheme=0), 0),
    (W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3), 3),
], ids=["model_b_64_setd2_R3", "kpz_32_setd1_R2", "model_a_128_em_R2", "model_b_64_setd1_replica0_3"])
def test_noalloc_matches_context_entry_point_on_two_calls(env, w, rep0):
    m, torch = env
    f0 = W.initial_fields(w).astype(np.float32)
    ref = m.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                    replica0=rep0)
    m.sft_set_plan(ref.ctx, [0, 0, 4, 0])  # the schedule the allocation-free path launches
    ref.set_field(f0)
    spec0 = ref.spectrum()
    # caller-owned device buffers: the state and (SETD2) the history
    phi = torch.from_numpy(spec0.copy()).cuda()
    fprev = torch.zeros_like(phi) if w.scheme == 2 else None
    cfg = m.make_config(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, w.dealias,
                        replica0=rep0)
    torch.cuda.synchronize()
    done = 0
    for call, n in enumerate((7, 11)):
        m.sft_step2d_noalloc(cfg, phi.data_ptr(), None if fprev is None else fprev.data_ptr(),
                             1 if call > 0 else 0, done, n)
        ref.step(n)
        done += n
        torch.cuda.synchronize()
        got = phi.cpu().numpy()
        want = ref.spectrum()
        for r in range(w.replicas):
            assert np.array_equal(got[r], want[r]), (call, r, rel(got[r], want[r]))
    ref.close()


def test_noalloc_reports_a_nonfinite_state(env):
    """Model A far below its critical point with a huge step: the cubic term
    overflows within a few steps, and the entry point says so."""
    m, torch = env
    w = W.model_a_64(n=[32, 32], replicas=1, p=[1.0, -50.0, 1.0, 0.5], h=0.5, sigma0=5.0)
    ref = m.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    ref.set_field(W.initial_fields(w).astype(np.float32))
    phi = torch.from_numpy(ref.spectrum().copy()).cuda()
    ref.close()
    cfg = m.make_config(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, w.dealias)
    torch.cuda.synchronize()
    with pytest.raises(m.SftError) as ei:
        m.sft_step2d_noalloc(cfg, phi.data_ptr(), None, 0, 0, 20)
    assert ei.value.status == m.SFT_ENONFINITE


def test_noalloc_applies_the_context_checks(env):
    """Configurations sft_create refuses are refused here too, before any device work."""
    m, torch = env
    w = W.model_b_1024(n=[32, 32], replicas=1)
    phi = torch.zeros((1, 17, 32), dtype=torch.complex64, device="cuda")
    for h, rep0 in ((w.h, -1), (float("inf"), 0)):
        cfg = m.make_config(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, h, w.seed, w.dealias, replica0=rep0)
        with pytest.raises(m.SftError) as ei:
            m.sft_step2d_noalloc(cfg, phi.data_ptr(), None, 0, 0, 1)
        assert ei.value.status == m.SFT_EINVAL, (h, rep0)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    m, torch = env
    w = W.model_b_1024(replicas=1)  # 1024 points per axis: above the 512-point limit
    cfg = m.make_config(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, w.dealias)
    phi = torch.zeros((1, 513, 1024), dtype=torch.complex64, device="cuda")
    with pytest.raises(m.SftError) as ei:
        m.sft_step2d_noalloc(cfg, phi.data_ptr(), None, 0, 0, 1)
    assert ei.value.status == m.SFT_EINVAL
    w = W.model_b_1024(n=[512, 512], replicas=2)  # 2 * 257 * 512 modes > 262144
    cfg = m.make_config(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, w.dealias)
    phi = torch.zeros((2, 257, 512), dtype=torch.complex64, device="cuda")
    with pytest.raises(m.SftError) as ei:
        m.sft_step2d_noalloc(cfg, phi.data_ptr(), None, 0, 0, 1)
    assert ei.value.status == m.SFT_EINVAL
