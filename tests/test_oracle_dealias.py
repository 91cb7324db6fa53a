"""Pins of the oracle's phase-shift dealiasing (Sec. IV step 1 names it as the
alternative to 2/3 truncation): the nonlinear term averaged over the 2^d grids
shifted by half a cell must equal the alias-free nonlinear term, computed here
independently with numpy on a grid refined twice per axis (no aliasing reaches
the kept modes there), for every mode but the Nyquist ones; without
dealiasing the same inputs do alias."""
import numpy as np
import pytest

import sft_inputs as W


def band_limited_spectrum(shape, seed, amp=1.0):
    """Full spectrum of a random real field with every Nyquist mode zeroed."""
    rng = np.random.default_rng(seed)
    S = np.fft.fftn(amp * rng.standard_normal(shape))
    for ax, n in enumerate(shape):
        sl = [slice(None)] * len(shape)
        sl[ax] = n // 2
        S[tuple(sl)] = 0.0
    return S


def refined_nonlinear_dft(S, kind, dx):
    """DFT (on the N grid's modes) of q = psi^3 or sum_j (d_j psi)^2, psi the
    band-limited field of spectrum S, evaluated on the 2N grid."""
    shape = S.shape
    fine = tuple(2 * n for n in shape)
    maps = [np.array([a if a < n // 2 else a + n for a in range(n)]) for n in shape]
    P = np.zeros(fine, dtype=complex)
    P[np.ix_(*maps)] = S
    scale = np.prod(fine) / np.prod(shape)
    if kind == "cubic":
        q = (np.fft.ifftn(P).real * scale) ** 3
    else:
        q = np.zeros(fine)
        for ax in range(len(shape)):
            k = 2 * np.pi * np.fft.fftfreq(fine[ax], dx / 2)
            k = k.reshape([-1 if i == ax else 1 for i in range(len(shape))])
            q += (np.fft.ifftn(1j * k * P).real * scale) ** 2
    return np.fft.fftn(q)[np.ix_(*maps)] / scale


def nyquist_mask(shape):
    m = np.ones(shape)
    for ax, n in enumerate(shape):
        sl = [slice(None)] * len(shape)
        sl[ax] = n // 2
        m[tuple(sl)] = 0.0
    return m


CASES = [
    ("model_a_1d_32", W.model_a_64(d=1, n=[32], dx=[1.0]), "cubic", -1.0),
    ("model_a_2d_16", W.model_a_64(n=[16, 16], dx=[0.7, 0.7]), "cubic", -1.0),
    ("model_a_3d_8", W.model_a_128_3d(n=[8, 8, 8]), "cubic", -1.0),
    ("kpz_2d_16", W.kpz_2d(n=[16, 16], dx=[0.5, 0.5]), "grad2", 1.0),
]


@pytest.mark.parametrize("name,w,kind,s", CASES, ids=[c[0] for c in CASES])
def test_phase_shift_dealiasing_is_alias_free(oracle_mod, name, w, kind, s):
    shape = tuple(reversed(w.n))
    S = band_limited_spectrum(shape, 7)
    want = nyquist_mask(shape) * s * refined_nonlinear_dft(S, kind, w.dx[0])
    got = {}
    for dealias in (0, 2):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=dealias)
        o.set_spectrum(0, S)
        got[dealias] = o.force(0)
    err = np.max(np.abs(got[2] - want)) / np.max(np.abs(want))
    assert err < 1e-12, (name, err)
    # the plain product on the N grid aliases the same input
    assert np.max(np.abs(got[0] - want)) / np.max(np.abs(want)) > 1e-3


def test_quadratic_term_truncation_and_phase_shift_agree_inside_the_band(oracle_mod):
    """KPZ (quadratic): for an input inside the 2/3 band the sum of two modes
    aliases only to modes outside the band, so the truncated and the
    phase-shifted terms agree on it."""
    w = W.kpz_2d(n=[16, 16])
    shape = tuple(reversed(w.n))
    ky, kx = np.meshgrid(np.fft.fftfreq(16, 1 / 16), np.fft.fftfreq(16, 1 / 16), indexing="ij")
    band = (3 * np.abs(kx) < 16) & (3 * np.abs(ky) < 16)
    S = band_limited_spectrum(shape, 11) * band
    F = {}
    for dealias in (1, 2):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=dealias)
        o.set_spectrum(0, S)
        F[dealias] = o.force(0)
    assert np.max(np.abs(F[1][band] - F[2][band])) < 1e-12 * np.max(np.abs(F[2]))


def test_phase_shift_dealiasing_complex_cgl_term(oracle_mod):
    """|A|^2 A of a complex band-limited field (CGL, no Hermitian symmetry): the
    mean over the four half-cell-shifted grids equals the alias-free term from the
    twice-refined grid, s = -(1 + i beta)."""
    w = W.cgl_2048(n=[16, 16], dx=[0.5, 0.5])
    shape = tuple(reversed(w.n))
    rng = np.random.default_rng(3)
    S = np.fft.fftn(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    mask = nyquist_mask(shape)
    S = S * mask
    fine = tuple(2 * n for n in shape)
    maps = [np.array([a if a < n // 2 else a + n for a in range(n)]) for n in shape]
    P = np.zeros(fine, dtype=complex)
    P[np.ix_(*maps)] = S
    scale = np.prod(fine) / np.prod(shape)
    A = np.fft.ifftn(P) * scale
    Q = np.fft.fftn(np.abs(A) ** 2 * A)[np.ix_(*maps)] / scale
    want = mask * (-(1 + 1j * w.p[1])) * Q
    o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=2)
    o.set_spectrum(0, S)
    got = o.force(0)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-12
