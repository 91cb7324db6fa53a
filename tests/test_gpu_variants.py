"""The variants of the 2-D real step (real-space noise, phase-shift dealiasing,
lattices of p x 2^k points) through the rest of the C ABI: checkpoint resume
bit for bit, the schedule they run with, per-pass profiling and the launch
count claimed for each step."""
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


VARIANTS = [
    ("real_space_noise", W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3, scheme=2, h=0.025), dict(noise_space=1)),
    ("phase_shift", W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3, scheme=2, h=0.025, dealias=2), {}),
    ("lattice_96", W.model_b_1024(n=[96, 96], replicas=2, sigma0=0.3, scheme=2, h=0.025), {}),
    ("lattice_80_kpz", W.kpz_2d(n=[80, 80], replicas=2, sigma0=0.3), {}),
]


def make(sft, w, extra):
    return sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, **extra)


@pytest.mark.parametrize("name,w,extra", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_checkpoint_resume_bit_identical(sft, name, w, extra):
    a = make(sft, w, extra)
    a.set_field(W.initial_fields(w).astype(np.float32))
    a.step(20)
    blob = a.checkpoint()
    a.step(37)
    ref = a.spectrum().copy()
    b = make(sft, w, extra)
    b.restore(blob)
    b.step(37)
    assert np.array_equal(b.spectrum().view(np.uint64), ref.view(np.uint64))
    a.close()
    b.close()


@pytest.mark.parametrize("name,w,extra", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_schedule_profile_and_launch_count(sft, name, w, extra):
    g = make(sft, w, extra)
    g.set_field(W.initial_fields(w).astype(np.float32))
    plan = sft.sft_get_plan(g.ctx)
    if name != "real_space_noise":  # phase shifts and p x 2^k lattices keep the default schedule
        assert plan[0] == 0 and plan[1] == 0 and plan[3] == 0
    if "lattice" in name:  # only the default schedule is built for p x 2^k lattices
        with pytest.raises(sft.SftError) as ei:
            sft.sft_set_plan(g.ctx, [1, 0, 2, 0])
        assert ei.value.status == sft.SFT_EINVAL
    prof = sft.sft_profile(g.ctx, 5)
    assert len(prof) == 3 and np.all(prof > 0) and abs(prof[0] + prof[1] - prof[2]) < 1e-6 * prof[2] + 1e-9
    per = sft.sft_launches_per_step(g.ctx)
    assert per == (4 if extra.get("noise_space") else 2)
    n0 = sft.sft_kernel_launches(g.ctx)
    g.step(40)  # graph chunks and plain steps
    g.sync()
    assert sft.sft_kernel_launches(g.ctx) - n0 >= 40 * per
    g.close()
