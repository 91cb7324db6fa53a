"""Pins of the oracle's general Fourier-space model (tables c, D and s over
q = |a|^2, the form of Sec. IV that the built-in models specialise), each
against a closed form or an independent integrator, never against the
oracle's built-in models:

- noise-free linear propagation: with D = 0 and no nonlinearity every mode
  evolves as e^{c(|a|^2) n h} exactly (Sec. II, Eq. setd-beg with F = 0), for
  irregular tables that a wrong index (|a| for |a|^2, a flattened index, a
  missing axis) would read at the wrong entry; real and complex c, d = 1..3;
- the noise amplitude per mode: g^2 / (1 - |f1|^2) is the exact stationary
  variance (N^2/L)^d D_q / (-Re c_q) of the linear SDE for SETD1 / SETD2, and
  (N^2/L)^d D_q h / sinh(-Re c_q h) for SETD-EM (Sec. II);
- nonlinear dynamics: with D = 0 the table-driven step converges with order 1
  (SETD1) and 2 (SETD2) to scipy's DOP853 on the semi-discrete equation
  dPhi/dt = c Phi + s M DFT[q(IDFT M Phi)], written here with numpy, for the
  cubic, gradient-squared and |A|^2 A nonlinearities with irregular s tables."""
import math

import numpy as np
import pytest

import sft_inputs as W


def a2_grid(shape):
    """|a|^2 of every mode of the full spectrum (numpy's signed indices)."""
    ax = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    return np.rint(sum(a * a for a in ax)).astype(int)


def table_len(d, n):
    return d * (n // 2) ** 2 + 1


def irregular(q, a, b, c):
    """A smooth-looking but irregular function of the table index: neighbouring
    entries differ, so an index off by one or by a factor shows."""
    q = np.asarray(q, dtype=np.float64)
    return a + b * np.sin(0.7 * q + 0.3) ** 2 + c * np.cos(1.9 * q)


def make(oracle_mod, d, n, dx, scheme, h, nl, cplx, c_re, c_im=None, D=None, s_re=None, s_im=None, dealias=1):
    ntab = table_len(d, n)
    D = np.zeros(ntab) if D is None else D
    return oracle_mod.Oracle(d, [n] * d, [dx] * d, 1, oracle_mod.CUSTOM, [], scheme, h, 17, dealias=dealias, nl=nl,
                             complex_field=cplx, c_re=c_re, c_im=c_im, noise_D=D, nl_re=s_re, nl_im=s_im)


@pytest.mark.parametrize("d,n,cplx", [(1, 32, 0), (2, 8, 0), (3, 8, 0), (1, 16, 1), (2, 8, 1)])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_custom_noise_free_linear_propagation(oracle_mod, d, n, cplx, scheme):
    ntab = table_len(d, n)
    q = np.arange(ntab)
    c_re = -irregular(q, 0.2, 0.9, 0.3) - 0.05 * q
    c_im = irregular(q, 0.0, 0.8, 0.5) if cplx else None
    h, nst = 0.07, 25
    o = make(oracle_mod, d, n, 0.6, scheme, h, oracle_mod.NL_NONE, cplx, c_re, c_im)
    shape = (n,) * d
    rng = np.random.default_rng(3)
    f0 = rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0)
    o.set_field(0, f0)
    S0 = np.fft.fftn(f0)
    o.step(nst)
    qq = a2_grid(shape)
    c = c_re[qq] + (1j * c_im[qq] if cplx else 0)
    expect = S0 * np.exp(c * nst * h)
    got = o.spectrum(0)
    err = np.abs(got - expect) / np.abs(expect)
    assert err.max() <= nst * 8 * 2.2e-16 + 1e-13, err.max()


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_custom_noise_amplitude_is_the_exact_stationary_variance(oracle_mod, scheme):
    d, n, dx = 2, 8, 0.8
    ntab = table_len(d, n)
    q = np.arange(ntab)
    c_re = -irregular(q, 0.3, 1.1, 0.2)
    c_im = irregular(q, 0.0, 0.6, 0.4)
    D = irregular(q, 0.1, 0.7, 0.05)
    for h, cplx in ((0.02, 0), (0.9, 0), (0.3, 1)):
        o = make(oracle_mod, d, n, dx, scheme, h, oracle_mod.NL_NONE, cplx, c_re, c_im if cplx else None, D)
        qq = a2_grid((n, n)).reshape(-1)
        nf2 = (n / dx) ** d
        for idx in range(n * n):
            f1, a, b, g = o.mode_coefs(idx)
            cr, Dq = c_re[qq[idx]], D[qq[idx]]
            var = abs(g) ** 2 / (1 - abs(f1) ** 2)
            ref = nf2 * Dq * h / math.sinh(-cr * h) if scheme == 0 else nf2 * Dq / (-cr)
            assert abs(var - ref) <= 1e-12 * ref, (h, cplx, idx)


def semi_discrete_rhs(shape, dx, nl, c, s, cplx):
    """dPhi/dt = c Phi + s M DFT[q(psi)], psi = IDFT[M Phi], as a real-space
    right-hand side for scipy (M: the 2/3 box mask; q: psi^3, sum_j (d_j psi)^2
    with the Nyquist derivative set to zero, or |psi|^2 psi)."""
    M = np.ones(shape)
    for ax, n in enumerate(shape):
        a = np.fft.fftfreq(n) * n
        sh = [1] * len(shape)
        sh[ax] = n
        M = M * (3 * np.abs(a) < n).reshape(sh)
    ks = []
    for ax, n in enumerate(shape):
        k = 2 * np.pi * np.fft.fftfreq(n, d=dx)
        k[n // 2] = 0.0
        sh = [1] * len(shape)
        sh[ax] = n
        ks.append(k.reshape(sh))

    def rhs(t, y):
        f = (y[: y.size // 2] + 1j * y[y.size // 2:]).reshape(shape) if cplx else y.reshape(shape)
        Phi = np.fft.fftn(f)
        psi = np.fft.ifftn(M * Phi)
        if nl == 1:
            qf = psi.real ** 3
        elif nl == 2:
            qf = sum(np.fft.ifftn(1j * k * M * Phi).real ** 2 for k in ks)
        else:
            qf = np.abs(psi) ** 2 * psi
        out = np.fft.ifftn(c * Phi + s * M * np.fft.fftn(qf))
        if cplx:
            out = out.reshape(-1)
            return np.concatenate([out.real, out.imag])
        return out.real.reshape(-1)

    return rhs


@pytest.mark.parametrize("nl,cplx", [(1, 0), (2, 0), (3, 1)], ids=["cubic", "grad2", "cgl"])
def test_custom_nonlinear_convergence_orders(oracle_mod, nl, cplx):
    from scipy.integrate import solve_ivp
    d, n, dx, T = 1, 16, 0.6, 0.4
    ntab = table_len(d, n)
    q = np.arange(ntab)
    c_re = -irregular(q, 0.1, 0.6, 0.2) - 0.08 * q
    c_im = irregular(q, 0.0, 0.5, 0.3) if cplx else None
    s_re = -irregular(q, 0.5, 0.4, 0.2) if nl != 2 else irregular(q, 0.6, 0.5, 0.2)
    s_im = irregular(q, 0.0, 0.7, 0.3) if cplx else None
    shape = (n,)
    qq = a2_grid(shape)
    c = c_re[qq] + (1j * c_im[qq] if cplx else 0)
    s = s_re[qq] + (1j * s_im[qq] if cplx else 0)
    w = W.Workload("custom", d, [n], [dx], W.CUSTOM, [], 1, 0.01, seed=0, sigma0=0.0)
    if cplx:
        w = w.with_(model=W.CGL)  # complex smooth field of the same band
    f0 = W.smooth_field(w, amplitude=0.6, seed=13)[0]
    rhs = semi_discrete_rhs(shape, dx, nl, c, s, cplx)
    y0 = np.concatenate([f0.real, f0.imag]) if cplx else f0.reshape(-1)
    ref = solve_ivp(rhs, (0, T), y0, method="DOP853", rtol=1e-12, atol=1e-13).y[:, -1]
    if cplx:
        ref = ref[: n] + 1j * ref[n:]
    errs = {}
    for scheme in (1, 2):
        e = []
        for nst in (40, 80, 160):
            o = make(oracle_mod, d, n, dx, scheme, T / nst, nl, cplx, c_re, c_im, None, s_re, s_im)
            o.set_field(0, f0)
            o.step(nst)
            e.append(np.abs(o.field(0).reshape(-1) - ref).max())
        errs[scheme] = e
        order = math.log2(e[1] / e[2])
        assert abs(order - (1 if scheme == 1 else 2)) < 0.15, (nl, scheme, e)
    assert errs[2][2] < errs[1][2]
