"""Shell sums taken in a fixed order with compensated FP64 summation.

* Bit-identical: the same state observed twice, and the same ensemble run in
  two contexts, give the same bits of S(k), of the per-replica S(k) and of the
  roughness (no atomics decide the summation order).
* The device time accumulator of S(k, t) (SFT_OBS_SK_ACCUM, read back by
  SFT_OBS_SK_TIME_MEAN) equals the mean of the individual S(k) observations it
  accumulated, and counts them; SFT_OBS_SK_RESET clears it.
* The shell sums agree with the oracle's App. C estimator on the same state
  (the parity test of every observable is in test_gpu_parity.py).
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


@pytest.mark.parametrize("w", [
    W.model_b_1024(n=[256, 256], replicas=8, sigma0=0.3),
    W.model_a_128_3d(n=[32, 32, 32], replicas=3, sigma0=0.3),
    W.cgl_2048(n=[128, 128], replicas=2),
], ids=["model_b_256_R8", "model_a_3d_32_R3", "cgl_128_R2"])
def test_repeated_observations_are_bit_identical(sft, w):
    f0 = W.initial_fields(w)
    f0 = f0.astype(np.complex64 if w.complex_field else np.float32)
    runs = []
    for _ in range(2):
        g = stepper(sft, w)
        g.set_field(f0)
        g.step(40)
        first = (g.observe(sft.SFT_OBS_SK), g.observe(sft.SFT_OBS_SK_REPLICAS))
        again = (g.observe(sft.SFT_OBS_SK), g.observe(sft.SFT_OBS_SK_REPLICAS))
        for a, b in zip(first, again):
            assert np.array_equal(a, b)
        if not w.complex_field:
            first = first + (g.observe(sft.SFT_OBS_ROUGHNESS),)
        runs.append(first)
        g.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_time_accumulator_is_the_mean_of_the_observations(sft):
    w = W.model_b_1024(n=[128, 128], replicas=4, sigma0=0.3)
    g = stepper(sft, w)
    g.set_field(W.initial_fields(w).astype(np.float32))
    ns = g.nshells()
    g.observe(sft.SFT_OBS_SK_RESET)
    snaps = []
    for _ in range(5):
        g.step(20)
        snaps.append(g.observe(sft.SFT_OBS_SK)[:ns])
        g.observe(sft.SFT_OBS_SK_ACCUM)
    out = g.observe(sft.SFT_OBS_SK_TIME_MEAN)
    assert out[ns] == 5
    want = np.mean(snaps, axis=0)
    assert np.allclose(out[:ns], want, rtol=1e-13, atol=0)
    g.observe(sft.SFT_OBS_SK_RESET)
    out = g.observe(sft.SFT_OBS_SK_TIME_MEAN)
    assert out[ns] == 0 and np.all(out[:ns] == 0)
    g.close()


def test_shell_sums_match_the_oracle(sft, oracle_mod):
    w = W.model_a_64(n=[64, 64], replicas=3, sigma0=0.3)
    f0 = W.initial_fields(w).astype(np.float32)
    g = stepper(sft, w)
    g.set_field(f0)
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(w.replicas):
        o.set_field(r, f0[r].astype(np.float64))
    g.step(30)
    o.step(30)
    got = g.observe(sft.SFT_OBS_SK)
    ns = g.nshells()
    ref, cnt = o.shells(0)
    assert np.array_equal(got[ns:2 * ns], cnt)
    assert np.allclose(got[:ns], ref, rtol=2e-5, atol=1e-12 * np.max(np.abs(ref)))
    g.close()
