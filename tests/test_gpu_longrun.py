"""Long-run statistics of interacting models, GPU against the oracle.  After
many steps the two sides are no longer comparable point by point (the
dynamics amplify rounding), so each side runs its own independent ensembles:
8 seeds per side (the GPU's and the oracle's seeds differ, and so do their
initial fields), several replicas per seed.  The ensemble means of the
observables must agree within 3 combined standard errors:
- Model B critical quench (the headline workload's parameters): shell averages
  of |phi_a|^2 (App. C) for the first shells, 32^2 after 400 steps and 128^2
  after 2000 steps;
- KPZ in 1-D (the ensemble workload's parameters, 256 sites): the width w^2;
- CGL (the 2-D workload's parameters, 32^2, SETD2): the mean |A|^2 and the
  shell average of |A_a|^2 of the first shells.
The oracle replicas run one per thread (its C library releases the GIL)."""
import threading
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


def shell_means(full, nshell):
    """Per-replica shell averages of |F_a|^2 (F: (R, ny, nx) full spectra), shells j = ceil(|a|) = 1..nshell."""
    R, ny, nx = full.shape
    ay, ax = np.meshgrid(np.fft.fftfreq(ny, 1.0 / ny), np.fft.fftfreq(nx, 1.0 / nx), indexing="ij")
    j = np.ceil(np.sqrt(ax ** 2 + ay ** 2) - 1e-12).astype(int)
    p = np.abs(full) ** 2
    return np.stack([p[:, j == s].mean(axis=1) for s in range(1, nshell + 1)], axis=1)


def agree(x, y, z_max=3.0):
    """Ensemble means of x and y (samples along axis 0) within z_max combined standard errors."""
    se = np.sqrt(x.var(axis=0, ddof=1) / len(x) + y.var(axis=0, ddof=1) / len(y))
    z = (x.mean(axis=0) - y.mean(axis=0)) / se
    assert np.all(np.abs(z) < z_max), z
    return z


GPU_SEEDS = [201, 202, 203, 204, 205, 206, 207, 208]
ORACLE_SEEDS = [301, 302, 303, 304, 305, 306, 307, 308]


def run_pair(sft, oracle_mod, w, nsteps, R):
    """Final fields of len(seeds) x R replicas on each side: (GPU, oracle)."""
    dt = np.complex64 if w.complex_field else np.float32
    dt64 = np.complex128 if w.complex_field else np.float64
    a = []
    for k, seed in enumerate(GPU_SEEDS):
        g = sft.Stepper(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, seed, dealias=w.dealias)
        g.set_field(W.initial_fields(w, replicas=R, seed_offset=k).astype(dt))
        g.step(nsteps)
        a.append(g.field().astype(dt64))
        g.close()
    jobs = [(k, seed, r) for k, seed in enumerate(ORACLE_SEEDS) for r in range(R)]
    out = [None] * len(jobs)

    def one(i):
        k, seed, r = jobs[i]
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, seed, dealias=w.dealias, replica0=r)
        f = W.initial_fields(w, replicas=R, seed_offset=1000 + k)[r]
        o.set_field(0, f.astype(dt).astype(dt64))
        o.step(nsteps)
        out[i] = o.field(0)

    for i0 in range(0, len(jobs), 16):
        th = [threading.Thread(target=one, args=(i,)) for i in range(i0, min(len(jobs), i0 + 16))]
        for t in th:
            t.start()
        for t in th:
            t.join()
    return np.concatenate(a), np.stack(out)


def test_model_b_quench_structure_factor(sft, oracle_mod):
    w = W.model_b_1024(n=[32, 32], h=0.05, sigma0=0.1)
    a, b = run_pair(sft, oracle_mod, w, 400, 4)
    agree(shell_means(np.fft.fft2(a), 6), shell_means(np.fft.fft2(b), 6))


def test_model_b_quench_128_long(sft, oracle_mod):
    """The headline workload's quench (Model B, r = -1, T = 0.1, h = 0.05) on
    128^2 over 2000 steps (100 time units of coarsening)."""
    w = W.model_b_1024(n=[128, 128], h=0.05, sigma0=0.1)
    a, b = run_pair(sft, oracle_mod, w, 2000, 2)
    agree(shell_means(np.fft.fft2(a), 8), shell_means(np.fft.fft2(b), 8))


def test_kpz_1d_width(sft, oracle_mod):
    w = W.kpz_1d(256, sigma0=0.0)
    a, b = run_pair(sft, oracle_mod, w, 1000, 4)
    wa = (a - a.mean(axis=1, keepdims=True)) ** 2
    wb = (b - b.mean(axis=1, keepdims=True)) ** 2
    agree(wa.mean(axis=1)[:, None], wb.mean(axis=1)[:, None])


def test_cgl_amplitude_and_spectrum(sft, oracle_mod):
    w = W.cgl_2048(n=[32, 32], sigma0=0.01)
    a, b = run_pair(sft, oracle_mod, w, 300, 2)
    agree((np.abs(a) ** 2).mean(axis=(1, 2))[:, None], (np.abs(b) ** 2).mean(axis=(1, 2))[:, None])
    agree(shell_means(np.fft.fft2(a), 4), shell_means(np.fft.fft2(b), 4))
