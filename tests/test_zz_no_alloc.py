"""The allocation-free 2-D step entry point, for callers that cannot call
cudaMalloc (their runtime owns the allocator, or allocation is forbidden after
start-up).  Through the C ABI it must give what the context-based entry point
gives on the same input, on two calls in a row (the second continuing the
first: later noise counters, SETD2 history carried in the caller's buffer).

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


@pytest.mark.parametrize("w", [
    W.model_b_1024(n=[64, 64], replicas=3, sigma0=0.3, scheme=2, h=0.025),
    W.kpz_2d(n=[32, 32], replicas=2, sigma0=0.4),
    W.model_a_64(n=[128, 128], replicas=2, scheme=0),
], ids=["model_b_64_setd2_R3", "kpz_32_setd1_R2", "model_a_128_em_R2"])
def test_noalloc_matches_context_entry_point_on_two_calls(env, w):
    m, torch = env
    f0 = W.initial_fields(w).astype(np.float32)
    ref = m.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    ref.set_field(f0)
    spec0 = ref.spectrum()
    # caller-owned device buffers: the state and (SETD2) the history
    phi = torch.from_numpy(spec0.copy()).cuda()
    fprev = torch.zeros_like(phi) if w.scheme == 2 else None
    cfg = m.make_config(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, w.dealias)
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
            assert rel(got[r], want[r]) <= 1e-5, (call, r, rel(got[r], want[r]))
    ref.close()


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
