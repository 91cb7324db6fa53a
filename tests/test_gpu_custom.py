"""The general Fourier-space model (SFT_CUSTOM: c, D and the nonlinear prefactor
s as tables over |a|^2, Sec. IV) on the GPU.

A custom model whose tables restate Model A, KPZ or CGL must step like the
built-in model (to FP32 rounding: the library folds s into the FP64 SETD
coefficients instead of multiplying in FP32), and custom operators that no
built-in model has must match the oracle's own table-driven model.
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


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def a2_grid(w):
    return np.arange(sum((n // 2) ** 2 for n in w.n[: w.d]) + 1, dtype=np.float64)


def dk2(w):
    return (2 * np.pi / (w.n[0] * w.dx[0])) ** 2


def run_pair(sft, a, b, f0, nsteps):
    for g in (a, b):
        g.set_field(f0)
        g.step(nsteps)
    out = a.field(), b.field()
    a.close()
    b.close()
    return out


def test_custom_restating_model_a(sft):
    w = W.model_a_64(replicas=2, sigma0=0.3)
    G, r, u, T = w.p
    q = a2_grid(w)
    tab = dict(nl=sft.SFT_NL_CUBIC, c=-G * (r + dk2(w) * q), D=np.full(q.size, G * T), s=np.full(q.size, -G * u))
    f0 = W.initial_fields(w).astype(np.float32)
    got, want = run_pair(sft, sft.Stepper(w.d, w.n, w.dx, 2, sft.SFT_CUSTOM, [], w.scheme, w.h, w.seed, custom=tab),
                         sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed), f0, 100)
    for rr in range(2):
        assert rel_l2(got[rr], want[rr]) <= 1e-5


def test_custom_restating_kpz_and_cgl(sft):
    w = W.kpz_2d(n=[64, 64], replicas=2, sigma0=0.5)
    nu, lam, D = w.p
    q = a2_grid(w)
    tab = dict(nl=sft.SFT_NL_GRAD2, c=-nu * dk2(w) * q, D=np.full(q.size, D), s=np.full(q.size, 0.5 * lam))
    f0 = W.initial_fields(w).astype(np.float32)
    got, want = run_pair(sft, sft.Stepper(w.d, w.n, w.dx, 2, sft.SFT_CUSTOM, [], w.scheme, w.h, w.seed, custom=tab),
                         sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed), f0, 100)
    for rr in range(2):
        assert rel_l2(got[rr], want[rr]) <= 1e-5
    w = W.cgl_2048(n=[64, 64], replicas=2, p=[2.0, -0.5, 1e-3])
    al, be, eps = w.p
    q = a2_grid(w)
    tab = dict(nl=sft.SFT_NL_CGL, complex_field=1, c=1.0 - (1.0 + 1j * al) * dk2(w) * q, D=np.full(q.size, eps),
               s=np.full(q.size, -(1.0 + 1j * be)))
    f0 = W.initial_fields(w).astype(np.complex64)
    got, want = run_pair(sft, sft.Stepper(w.d, w.n, w.dx, 2, sft.SFT_CUSTOM, [], w.scheme, w.h, w.seed, custom=tab),
                         sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed), f0, 100)
    for rr in range(2):
        assert rel_l2(got[rr], want[rr]) <= 1e-5


CUSTOM_CASES = [
    # Swift-Hohenberg-like linear operator with a wavenumber-dependent noise, cubic term
    ("sh_2d_cubic", 2, [64, 64], 0, "cubic", lambda k2: -(0.3 + (1.0 - k2) ** 2), lambda k2: 0.05 * (1 + k2),
     lambda k2: -np.ones_like(k2), 1),
    ("ou_2d_none_setd2", 2, [32, 32], 0, "none", lambda k2: -(0.2 + k2 ** 2), lambda k2: 0.1 + 0 * k2, None, 2),
    ("grad2_1d", 1, [256], 0, "grad2", lambda k2: -0.8 * k2 - 0.1 * k2 ** 2, lambda k2: 0.3 + 0 * k2,
     lambda k2: 0.7 + 0.1 * k2, 1),
    ("cubic_3d_em", 3, [16, 16, 16], 0, "cubic", lambda k2: -(0.5 + k2), lambda k2: 0.2 + 0.1 * k2,
     lambda k2: -0.8 + 0 * k2, 0),
    ("cgl_like_2d", 2, [32, 32], 1, "cgl", lambda k2: 0.5 - (1 + 0.7j) * k2, lambda k2: 1e-3 + 0 * k2,
     lambda k2: -(1 - 0.3j) + 0.01 * k2, 1),
    ("complex_none_1d", 1, [128], 1, "none", lambda k2: -0.1 - (1 + 2j) * k2, lambda k2: 0.01 + 0 * k2, None, 1),
]


@pytest.mark.parametrize("name,d,n,cplx,nl,c,D,s,scheme", CUSTOM_CASES, ids=[c[0] for c in CUSTOM_CASES])
def test_custom_against_oracle(sft, oracle_mod, name, d, n, cplx, nl, c, D, s, scheme):
    nls = {"none": (sft.SFT_NL_NONE, oracle_mod.NL_NONE), "cubic": (sft.SFT_NL_CUBIC, oracle_mod.NL_CUBIC),
           "grad2": (sft.SFT_NL_GRAD2, oracle_mod.NL_GRAD2), "cgl": (sft.SFT_NL_CGL, oracle_mod.NL_CGL)}[nl]
    dx = [1.0] * d
    w = W.Workload(name, d, n, dx, W.CUSTOM, [], scheme, 0.02, seed=4242, replicas=2, sigma0=0.3)
    q = a2_grid(w)
    k2 = dk2(w) * q
    ct, Dt = c(k2), D(k2)
    st = None if s is None else s(k2)
    tab = dict(nl=nls[0], complex_field=cplx, c=ct, D=Dt, s=st)
    g = sft.Stepper(d, n, dx, 2, sft.SFT_CUSTOM, [], scheme, w.h, w.seed, custom=tab)
    ct = np.asarray(ct, dtype=np.complex128)
    st = np.zeros_like(ct) if st is None else np.asarray(st, dtype=np.complex128)
    o = oracle_mod.Oracle(d, n, dx, 2, oracle_mod.CUSTOM, [], scheme, w.h, w.seed, nl=nls[1], complex_field=cplx,
                          c_re=np.ascontiguousarray(ct.real), c_im=np.ascontiguousarray(ct.imag),
                          noise_D=np.ascontiguousarray(Dt, dtype=np.float64),
                          nl_re=np.ascontiguousarray(st.real), nl_im=np.ascontiguousarray(st.imag))
    f0 = W.initial_fields(w.with_(model=W.CGL) if cplx else w)  # complex fields draw complex initial values
    g.set_field(f0.astype(np.complex64 if cplx else np.float32))
    for r in range(2):
        o.set_field(r, f0[r].astype(np.complex64 if cplx else np.float32).astype(np.complex128 if cplx else np.float64))
    g.step(60)
    o.step(60)
    got = g.field()
    for r in range(2):
        assert rel_l2(got[r], o.field(r)) <= 1e-5, (name, r)
    g.close()
