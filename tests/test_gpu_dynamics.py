"""Dynamic correlation C(k, omega), noise-inferred susceptibility chi(k, omega)
and the deviation from the FDT (App. C, Sec. V.A) on the GPU.

* Parity: the GPU's C_ab, chi_ab and Dbar equal the oracle's App. C
  estimators (oracle.dyn_estimators, pinned in test_oracle_dynamics.py) on the
  series recorded from the oracle (its state and its nonlinear force F at every
  sampled step), with the oracle's own c_a and D_a.
* For a linear model (u = 0) the deterministic force is K = c phi, so every
  sample gives phi conj(-i omega phi - c phi) = (i omega - c) |phi|^2 and the
  estimator obeys 2 Im chi = (omega / D) C exactly: a check of the whole sign
  convention of the time transform.
* Interacting Model A in equilibrium: the average absolute deviation from the
  FDT falls as 1/sqrt(S) with the ensemble size, and its signed mean is far
  below it (Sec. V.A).
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


def model_a_c_D(w):
    G, r, u, T = w.p
    nx, ny = w.n
    dk = 2 * np.pi / (nx * w.dx[0])
    ax = np.arange(nx // 2 + 1)[:, None]
    ay = np.fft.fftfreq(ny, 1.0 / ny)[None, :]
    k2 = dk * dk * (ax * ax + ay * ay)
    return (-G * (r + k2)).ravel(), np.full(k2.size, G * T)


def half_layout(full):
    """(ny, nx) full spectrum -> the library's x-major half layout, flattened (a = a_x ny + a_y)."""
    nx = full.shape[1]
    return full[:, : nx // 2 + 1].T.ravel()


def test_dynamics_against_oracle(sft, oracle_mod):
    w = W.model_a_64(n=[16, 16], replicas=4, sigma0=0.3, h=0.02)
    M, every = 32, 2
    f0 = W.initial_fields(w).astype(np.float32)
    g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    g.set_field(f0)
    g.step(10)
    sft.sft_dyn_start(g.ctx, M, every)
    g.step(M * every)
    nm = (w.n[0] // 2 + 1) * w.n[1]
    C, chi, dbar = sft.sft_dyn_result(g.ctx, nm, M)
    g.step(3)  # stepping goes on after the recording ends
    g.close()
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(w.replicas):
        o.set_field(r, f0[r].astype(np.float64))
    o.step(10)
    phi = np.zeros((w.replicas, nm, M), complex)
    F = np.zeros_like(phi)
    for m in range(M):
        for r in range(w.replicas):
            phi[r, :, m] = half_layout(o.spectrum(r))
            F[r, :, m] = half_layout(o.force(r))
        o.step(every)
    c_full, D_full = o.mode_operators()
    c, D = half_layout(c_full), half_layout(D_full)
    T = M * every * w.h
    norm = (w.dx[0] / w.n[0]) ** 2
    Co, chio, dbar_o = oracle_mod.dyn_estimators(phi, F, c, D, T, norm)
    assert np.linalg.norm(C - Co) <= 1e-4 * np.linalg.norm(Co)
    assert np.linalg.norm(chi - chio) <= 1e-4 * np.linalg.norm(chio)
    assert abs(dbar - dbar_o) <= 1e-3 * dbar_o
    # the GPU's Dbar is its own C and chi summarised the same way
    om = 2 * np.pi * np.fft.fftfreq(M, 1.0 / M) / T
    dev = np.abs(2 * chi.imag - om[None, :] / D[:, None] * C)
    assert abs(dbar - dev.mean()) <= 1e-9 * (1 + dev.mean())


def test_linear_model_obeys_the_fdt_identically(sft):
    w = W.model_a_64(n=[32, 32], replicas=64, p=[1.0, 0.5, 0.0, 0.5], sigma0=0.5, h=0.05)
    g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    g.set_field(W.initial_fields(w).astype(np.float32))
    g.step(100)
    M = 64
    sft.sft_dyn_start(g.ctx, M, 1)
    g.step(M)
    nm = (w.n[0] // 2 + 1) * w.n[1]
    C, chi, dbar = sft.sft_dyn_result(g.ctx, nm, M)
    g.close()
    _, D = model_a_c_D(w)
    om = 2 * np.pi * np.fft.fftfreq(M, 1.0 / M) / (M * w.h)
    rhs = om[None, :] / D[:, None] * C
    assert np.max(np.abs(2 * chi.imag - rhs)) <= 1e-9 * np.max(np.abs(rhs))
    assert dbar <= 1e-9 * np.mean(np.abs(rhs))


def test_fdt_deviation_falls_with_the_ensemble(sft):
    """Interacting Model A (u = 1, r = 0.5: disordered, fast relaxation) in
    equilibrium: Dbar(S) ~ 1/sqrt(S) (S = 256 -> 1024 halves it, within 30 %)
    and the signed mean deviation stays far below Dbar."""
    out = {}
    for R in (256, 1024):
        w = W.model_a_64(n=[32, 32], replicas=R, p=[1.0, 0.5, 1.0, 0.5], sigma0=0.5, h=0.02)
        g = sft.Stepper(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
        g.set_field(W.initial_fields(w).astype(np.float32))
        g.step(500)
        M = 128
        sft.sft_dyn_start(g.ctx, M, 1)
        g.step(M)
        nm = (w.n[0] // 2 + 1) * w.n[1]
        C, chi, dbar = sft.sft_dyn_result(g.ctx, nm, M)
        g.close()
        _, D = model_a_c_D(w)
        om = 2 * np.pi * np.fft.fftfreq(M, 1.0 / M) / (M * w.h)
        dev = 2 * chi.imag - om[None, :] / D[:, None] * C
        out[R] = (dbar, float(np.mean(dev)))
    ratio = out[256][0] / out[1024][0]
    assert 1.4 < ratio < 2.6, (ratio, out)
    for R, (dbar, mean) in out.items():
        assert abs(mean) < 0.1 * dbar, (R, mean, dbar)
