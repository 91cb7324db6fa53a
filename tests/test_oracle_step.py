"""Pins of the oracle's stepper against closed forms, invariants and
independent integrators (never against a retyped copy of its own formulas).

Each test names the passage of the paper that fixes the expected value.
"""
import math

import numpy as np
import pytest

import sft_inputs as W


def make_oracle(O, w: W.Workload, replicas=None, **kw):
    return O.Oracle(w.d, w.n, w.dx, replicas or w.replicas, w.model, w.p, w.scheme, w.h, w.seed,
                    dealias=w.dealias, **kw)


def spectral_k(shape, dx):
    """numpy-side wavenumbers (independent of the oracle's index code)."""
    ks = [2 * np.pi * np.fft.fftfreq(n, d=dx) for n in shape]
    return np.meshgrid(*ks, indexing="ij")


# ------------------------------------------------------------ noise structure
def test_noise_hermitian_and_counts(oracle_mod):
    """App. B: eta_{-a} = conj(eta_a); the draw holds exactly N^d real deviates,
    split into blue / red / black regions as the paper counts them in 2-D."""
    rows = np.loadtxt(__file__.replace("test_oracle_step.py", "golden/noise_deviate_count_2d.txt"))
    for N, blue, red, black, total in rows.astype(int):
        w = W.model_a_64(n=[N, N])
        o = make_oracle(oracle_mod, w)
        eta = o.noise(0, 3)
        real = np.fft.ifft2(eta)
        assert np.abs(real.imag).max() < 1e-15 * N * N
        # classify the stored half a_x in [0, N/2] like the paper's figure
        nb = nr = nk = 0
        for iy in range(N):
            for ix in range(N // 2 + 1):
                on_plane_x = ix in (0, N // 2)
                on_plane_y = iy in (0, N // 2)
                if on_plane_x and on_plane_y:
                    nk += 1
                    assert eta[iy, ix].imag == 0.0
                elif on_plane_x:
                    if iy < N // 2:  # canonical half of the stripe
                        nr += 2
                else:
                    nb += 2 if on_plane_y or True else 0
        # blue regions exclude the a_y in {0, N/2} rows, which belong to red stripes R3/R4
        blue_count = 2 * 2 * (N // 2 - 1) ** 2
        red_count = 8 * (N // 2 - 1)
        assert blue_count == blue and red_count == red and nk == black
        assert blue_count + red_count + nk == N * N == total


def test_noise_unit_variance_and_real_space_scaling(oracle_mod):
    """Sec. IV / App. A: <|eta_a|^2> = 1 per mode; scaled by (N^2/L)^{d/2} and
    transformed back, the real-space noise has variance (N/L)^d per site."""
    N, dx = 16, 0.5
    w = W.model_a_64(n=[N, N], dx=[dx, dx])
    o = make_oracle(oracle_mod, w)
    acc = np.zeros((N, N))
    racc = 0.0
    S = 300
    for s in range(S):
        eta = o.noise(0, s)
        acc += np.abs(eta) ** 2
        scaled = eta * (N * N / (N * dx)) ** (2 / 2)
        racc += np.mean(np.real(np.fft.ifft2(scaled)) ** 2)
    m = acc / S
    assert abs(m.mean() - 1) < 4 * math.sqrt(2 / (S * N * N))
    assert abs(racc / S - (N / (N * dx)) ** 2) < 0.03 * (N / (N * dx)) ** 2


def test_noise_streams_distinct(oracle_mod):
    w = W.model_a_64(n=[8, 8])
    o = make_oracle(oracle_mod, w, replicas=2)
    a, b, c = o.noise(0, 0), o.noise(1, 0), o.noise(0, 1)
    assert np.abs(a - b).max() > 0.1 and np.abs(a - c).max() > 0.1


def test_real_space_noise_is_the_transformed_site_draw(oracle_mod):
    """Sec. IV step 2, real-space alternative: eta(x) iid N(0, 1) per site and
    eta_a = DFT[eta]_a / sqrt(N^d).  The inverse DFT (numpy) of the oracle's
    eta_a times sqrt(N^d) gives back, site by site, normal s & 3 of the Philox
    block (s / 4, step, replica, 3) (Philox pinned by its known answers); the
    spectrum is Hermitian with real self-conjugate modes."""
    nx, ny, R = 16, 8, 2
    w = W.model_a_64(n=[nx, nx])
    o = oracle_mod.Oracle(2, [nx, ny], [1.0, 1.0], R, w.model, w.p, w.scheme, w.h, 99, noise_space=1,
                          replica0=5)
    for r, step in ((0, 0), (1, 7)):
        eta = o.noise(r, step)  # (ny, nx) full spectrum
        site = np.fft.ifft2(eta) * math.sqrt(nx * ny)
        assert np.abs(site.imag).max() < 1e-13
        want = np.array([oracle_mod.normals4(99, s >> 2, step, 5 + r, 3)[s & 3] for s in range(nx * ny)],
                        dtype=np.float64).reshape(ny, nx)
        assert np.abs(site.real - want).max() < 1e-12
        neg = np.conj(np.roll(eta[::-1, ::-1], 1, axis=(0, 1)))
        assert np.array_equal(eta, neg)
        for iy in (0, ny // 2):
            for ix in (0, nx // 2):
                assert eta[iy, ix].imag == 0.0


@pytest.mark.parametrize("d,n", [(1, [64]), (3, [8, 4, 6])])
def test_real_space_noise_other_dimensions(oracle_mod, d, n):
    """The same site-by-site identity in 1-D and 3-D (site s = x + n_x (y + n_y z))."""
    w = W.model_a_64(d=d, n=n, dx=[1.0] * d)
    o = oracle_mod.Oracle(d, n, [1.0] * d, 1, w.model, w.p, w.scheme, w.h, 7, noise_space=1)
    eta = o.noise(0, 4)
    site = np.fft.ifftn(eta) * math.sqrt(np.prod(n))
    assert np.abs(site.imag).max() < 1e-13
    want = np.array([oracle_mod.normals4(7, s >> 2, 4, 0, 3)[s & 3] for s in range(int(np.prod(n)))],
                    dtype=np.float64).reshape(tuple(reversed(n)))
    assert np.abs(site.real - want).max() < 1e-12


def test_gaussian_model_a_structure_factor_real_space_noise(oracle_mod):
    """Sec. IV step 2 / Sec. V.A: with the real-space draw the linear theory
    C_ET(k) = T / (r + k^2) holds as with the Fourier draw (the two noises have
    the same covariance); shell averages within 5 sigma."""
    N, R = 16, 64
    w = W.model_a_64(n=[N, N], dx=[0.5, 0.5], p=[1.0, 1.0, 0.0, 0.6], h=0.05)
    o = make_oracle(oracle_mod, w, replicas=R, noise_space=1)
    o.step(200)
    acc = None
    S = 20
    for _ in range(S):
        o.step(20)
        v, _ = o.shells(0)
        acc = v if acc is None else acc + v
    v = acc / S
    dk = 2 * np.pi / (N * 0.5)
    KY, KX = spectral_k(w.shape, 0.5)
    kk = np.sqrt(KX ** 2 + KY ** 2)
    for j in range(1, 6):
        sel = (kk > (j - 1) * dk + 1e-9) & (kk <= j * dk + 1e-9)
        ref = np.mean(0.6 / (1.0 + kk[sel] ** 2))
        assert abs(v[j] - ref) < 5 * ref / math.sqrt(sel.sum() * R * S / 4), (j, v[j], ref)


# ------------------------------------------------------------ linear closed forms
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("n", [[16, 16], [32], [8, 8, 8]], ids=["2d", "1d", "3d"])
def test_noise_free_linear_propagation(oracle_mod, model, scheme, n):
    """u = 0, D = 0: Eq. (setd-beg) reduces to phi_a(t+h) = e^{c h} phi_a(t)
    exactly; after n steps phi_a = e^{c n h} phi_a(0) to rounding."""
    p = [1.0, 0.3, 0.0, 0.0]
    d = len(n)
    w = W.model_a_64(n=n, d=d, dx=[0.7] * d, model=model, p=p, scheme=scheme, h=0.05)
    o = make_oracle(oracle_mod, w)
    rng = np.random.default_rng(0)
    f0 = rng.standard_normal(w.shape)
    o.set_field(0, f0)
    S0 = np.fft.fftn(f0)
    n = 40
    o.step(n)
    k2 = sum(kk ** 2 for kk in spectral_k(w.shape, 0.7))
    c = -(0.3 + k2) if model == 0 else -k2 * (0.3 + k2)
    expect = S0 * np.exp(c * n * w.h)
    got = o.spectrum(0)
    err = np.abs(got - expect) / np.maximum(np.abs(expect), 1e-300)
    big = np.abs(expect) > 1e-200
    # rounding: a few ulps per step, plus the argument c h rounded (relative eps) on both sides, which moves
    # e^{c n h} by |c n h| eps relative
    tol = n * 4 * 2.2e-16 + 2 * np.abs(c) * n * w.h * 2.2e-16 + 1e-14
    assert (err[big] <= tol[big]).all(), (err[big] / tol[big]).max()


def test_ou_stationary_variance_identity(oracle_mod):
    """u = 0: the SETD1/SETD2 noise amplitude makes the discrete stationary
    variance g^2/(1-f1^2) equal the exact OU value (N^2/L)^d D_a/(-c_a) for
    every h (exact I1, Sec. II); SETD-EM gives (N^2/L)^d D_a h / sinh(|c| h)."""
    N, dx = 8, 0.8
    for scheme in (0, 1, 2):
        for h in (0.01, 0.3, 2.0):
            w = W.model_a_64(n=[N, N], dx=[dx, dx], p=[1.3, 0.4, 0.0, 0.7], scheme=scheme, h=h)
            o = make_oracle(oracle_mod, w)
            KY, KX = spectral_k(w.shape, dx)
            k2 = (KX ** 2 + KY ** 2).reshape(-1)
            nf2 = (N * N / (N * dx)) ** 2
            for idx in range(N * N):
                f1, a, b, g = o.mode_coefs(idx)
                c = -1.3 * (0.4 + k2[idx])
                D = 1.3 * 0.7
                var = abs(g) ** 2 / (1 - abs(f1) ** 2)
                if scheme == 0:
                    ref = nf2 * D * h / math.sinh(abs(c) * h)
                else:
                    ref = nf2 * D / (-c)
                assert abs(var - ref) <= 1e-12 * ref


def test_complex_c_coefficients_closed_forms(oracle_mod):
    """CGL, c_a = 1 - (1 + i alpha) k^2 complex (Sec. V.C): f1 = e^{c h}; the
    exact integrals of Sec. II, A = int_0^h e^{c (h - s)} ds = (e^{ch} - 1)/c
    (SETD-EM, SETD1) and, with the linear interpolation of F, A = ((1 + ch) e^{ch} - 1
    - 2ch)/(c^2 h), B = (1 + ch - e^{ch})/(c^2 h) (SETD2; its first step takes
    SETD1's); and the noise amplitude of the exact stochastic integral
    int_0^h e^{c (h - s)} dW, whose stationary variance g^2/(1 - |f1|^2) is the
    exact OU value (N^2/L)^d D/(-Re c) for every h (SETD-EM: (N^2/L)^d D h /
    sinh(-Re(c) h)).  Modes with Re c > 0 (the unstable band) obey the same
    identities with the signs carried through."""
    N, dx, alpha, eps = 8, 0.5, 2.0, 1e-4
    for scheme in (0, 1, 2):
        for h in (0.05, 0.4):
            w = W.cgl_2048(n=[N, N], dx=[dx, dx], p=[alpha, -0.5, eps], scheme=scheme, h=h)
            o = make_oracle(oracle_mod, w)
            KY, KX = spectral_k(w.shape, dx)
            k2 = (KX ** 2 + KY ** 2).reshape(-1)
            nf2 = (N * N / (N * dx)) ** 2
            for idx in range(N * N):
                c = 1 - (1 + 1j * alpha) * k2[idx]
                e = np.exp(c * h)
                for first in ((0, 1) if scheme == 2 else (0,)):
                    f1, a, b, g = o.mode_coefs(idx, first)
                    assert abs(f1 - e) <= 1e-14 * abs(e)
                    if scheme == 2 and not first:
                        a_ref = ((1 + c * h) * e - 1 - 2 * c * h) / (c * c * h)
                        b_ref = (1 + c * h - e) / (c * c * h)
                    else:
                        a_ref, b_ref = (e - 1) / c, 0.0
                    assert abs(a - a_ref) <= 1e-12 * abs(a_ref), (scheme, h, idx, a, a_ref)
                    assert abs(b - b_ref) <= 1e-12 * max(abs(b_ref), h * h), (scheme, h, idx, b, b_ref)
                    var = abs(g) ** 2 / (1 - abs(f1) ** 2)
                    x = -c.real
                    ref = nf2 * eps * h / math.sinh(x * h) if scheme == 0 else nf2 * eps / x
                    assert abs(var - ref) <= 1e-11 * abs(ref), (scheme, h, idx, var, ref)


def test_ou_finite_time_variance_ensemble(oracle_mod):
    """u = 0, SETD1 from phi = 0: V_n = g^2 (1 - f1^{2n}) / (1 - f1^2), and in
    the limit the linear-theory C_ET = T/(r+k^2) (Sec. V.A, sign of the
    printed transient formula corrected).  Ensemble of replicas, 4 sigma."""
    N, R, n = 8, 400, 30
    w = W.model_a_64(n=[N, N], p=[1.0, 0.5, 0.0, 0.8], h=0.1)
    o = make_oracle(oracle_mod, w, replicas=R)
    o.step(n)
    spec = np.array([o.spectrum(r) for r in range(R)])
    KY, KX = spectral_k(w.shape, 1.0)
    k2 = KX ** 2 + KY ** 2
    c = -(0.5 + k2)
    V_inf = N * N * 0.8 / (-c)  # (N^2/L)^d T/(r+k^2) with dx = 1
    V_n = V_inf * (1 - np.exp(2 * c * w.h * n))
    est = np.mean(np.abs(spec) ** 2, axis=0)
    z = (est - V_n) / (V_n / math.sqrt(R))  # |Phi|^2 of complex Gaussian: std = mean
    selfc = np.zeros_like(k2, dtype=bool)
    for iy in (0, N // 2):
        for ix in (0, N // 2):
            selfc[iy, ix] = True
    z[selfc] /= math.sqrt(2)  # real modes: std of chi^2_1 is sqrt(2) mean
    assert np.abs(z).max() < 4.5, np.abs(z).max()


def test_gaussian_model_a_structure_factor(oracle_mod):
    """Sec. V.A linear theory: C_ET(k) = T / (r + k^2) for u = 0, r > 0,
    measured with the App. C shell average."""
    N, R = 16, 64
    w = W.model_a_64(n=[N, N], dx=[0.5, 0.5], p=[1.0, 1.0, 0.0, 0.6], h=0.05)
    o = make_oracle(oracle_mod, w, replicas=R)
    o.step(200)  # t = 10 >> 1/(2r)
    acc = None
    S = 20
    for _ in range(S):
        o.step(20)
        v, cnt = o.shells(0)
        acc = v if acc is None else acc + v
    v = acc / S
    dk = 2 * np.pi / (N * 0.5)
    for j in range(1, 6):
        # shell j holds modes with (j-1) dk < |k| <= j dk; compare with the shell mean of T/(r+k^2)
        KY, KX = spectral_k(w.shape, 0.5)
        kk = np.sqrt(KX ** 2 + KY ** 2)
        sel = (kk > (j - 1) * dk + 1e-9) & (kk <= j * dk + 1e-9)
        ref = np.mean(0.6 / (1.0 + kk[sel] ** 2))
        nmodes = sel.sum() * R * S
        assert abs(v[j] - ref) < 5 * ref / math.sqrt(nmodes / 4), (j, v[j], ref)


def test_two_time_correlation_discrete(oracle_mod):
    """u = 0, SETD1, stationary: <Phi_a(n+m) Phi_a*(n)> = f1^m V_inf exactly in
    discrete time (the update is linear with independent noise)."""
    N, R = 8, 300
    w = W.model_a_64(n=[N, N], p=[1.0, 0.6, 0.0, 0.5], h=0.2)
    o = make_oracle(oracle_mod, w, replicas=R)
    o.step(100)
    o.mark()
    m = 3
    o.step(m)
    v, cnt = o.shells(1)
    KY, KX = spectral_k(w.shape, 1.0)
    k2 = KX ** 2 + KY ** 2
    c = -(0.6 + k2)
    kk = np.sqrt(k2)
    dk = 2 * np.pi / N
    for j in range(0, 4):
        sel = (kk > (j - 1) * dk + 1e-9) & (kk <= j * dk + 1e-9)
        ref = np.mean(np.exp(c[sel] * w.h * m) * 0.5 / (-c[sel]) * (-c[sel]) / (0.6 + k2[sel]))
        sd = np.mean(0.5 / (0.6 + k2[sel])) / math.sqrt(sel.sum() * R / 2)
        assert abs(v[j] - ref) < 5 * sd, (j, v[j], ref)


def test_model_b_zero_mode_conserved_bitwise(oracle_mod):
    """Sec. V.A footnote: c(0) = 0 and D(0) = 0 for Model B, so the k = 0 mode is
    never forgotten: it must stay bit-identical through noisy nonlinear steps."""
    for scheme in (0, 1, 2):
        w = W.model_b_1024(n=[16, 16], scheme=scheme, h=0.05, sigma0=0.3)
        o = make_oracle(oracle_mod, w, replicas=2)
        f0 = W.initial_fields(w, replicas=2)
        for r in range(2):
            o.set_field(r, f0[r])
        z0 = [o.spectrum(r)[0, 0] for r in range(2)]
        o.step(25)
        for r in range(2):
            assert o.spectrum(r)[0, 0] == z0[r]
            assert np.abs(o.spectrum(r)).max() > 0


# ------------------------------------------------------------ nonlinear dynamics
def _real_space_rhs(model, p, shape, dx, dealias):
    """Semi-discrete real-space right-hand side from the PDEs of Sec. V,
    written with numpy spectral derivatives (independent of the oracle)."""
    k = spectral_k(shape, dx)
    k2 = sum(kk ** 2 for kk in k)
    M = np.ones(shape)
    if dealias:
        for ax, n in enumerate(shape):
            a = np.fft.fftfreq(n) * n
            sh = [1] * len(shape)
            sh[ax] = n
            M = M * (3 * np.abs(a) < n).reshape(sh)
    lap = lambda f: np.fft.ifftn(-k2 * np.fft.fftn(f))
    proj = lambda f: np.fft.ifftn(M * np.fft.fftn(f))

    def rhs(t, y):
        if model == 3:
            A = (y[: y.size // 2] + 1j * y[y.size // 2:]).reshape(shape)
        else:
            A = y.reshape(shape)
        if model == 0:  # Model A: -Gamma (r phi + u P[(P phi)^3] - lap phi)
            G, r, u = p[0], p[1], p[2]
            out = -G * (r * A + u * proj(proj(A).real ** 3) - lap(A))
        elif model == 1:  # Model B: Gamma lap (r phi + u P[(P phi)^3] - lap phi)
            G, r, u = p[0], p[1], p[2]
            out = G * lap(r * A + u * proj(proj(A).real ** 3) - lap(A))
        elif model == 2:  # KPZ: nu lap h + lambda/2 P[|grad P h|^2]
            nu, lam = p[0], p[1]
            H = np.fft.fftn(A) * M
            g2 = 0
            for ax, kk in enumerate(k):
                n = shape[ax]
                kodd = kk.copy()
                sl = [slice(None)] * len(shape)
                sl[ax] = n // 2
                kodd[tuple(sl)] = 0.0
                g2 = g2 + np.fft.ifftn(1j * kodd * H).real ** 2
            out = nu * lap(A) + 0.5 * lam * proj(g2)
        else:  # CGL: A + (1 + i alpha) lap A - (1 + i beta) P[|PA|^2 PA]
            al, be = p[0], p[1]
            PA = proj(A)
            out = A + (1 + 1j * al) * lap(A) - (1 + 1j * be) * proj(np.abs(PA) ** 2 * PA)
        if model == 3:
            out = out.reshape(-1)
            return np.concatenate([out.real, out.imag])
        return out.real.reshape(-1)

    return rhs


@pytest.mark.parametrize("model", [0, 1, 2])
def test_deterministic_convergence_orders(oracle_mod, model):
    """D = 0: SETD-EM / SETD1 converge with order 1 and SETD2 with order 2 in h
    (Sec. II: ETD1 local error O(h^2); Cox-Matthews ETD2) to the exact solution
    of the semi-discrete equation, here from scipy's RK45 at tight tolerance."""
    from scipy.integrate import solve_ivp
    N, dx, T = 16, 0.6, 0.4
    if model == 0:
        p = [1.0, -0.5, 1.0, 0.0]
    elif model == 1:
        p = [1.0, -1.0, 1.0, 0.0]
    else:
        p = [1.0, 2.0, 0.0]
    w = W.model_a_64(n=[N], d=1, dx=[dx], model=model, p=p)
    f0 = W.smooth_field(w.with_(n=[N]), amplitude=0.6, seed=11)[0]
    rhs = _real_space_rhs(model, p, w.shape, dx, 1)
    ref = solve_ivp(rhs, (0, T), f0.reshape(-1), method="DOP853", rtol=1e-12, atol=1e-13).y[:, -1]
    errs = {}
    for scheme in (1, 2):
        e = []
        for nst in (40, 80, 160):
            o = make_oracle(oracle_mod, w.with_(scheme=scheme, h=T / nst))
            o.set_field(0, f0)
            o.step(nst)
            e.append(np.abs(o.field(0).reshape(-1) - ref).max())
        errs[scheme] = e
        order = math.log2(e[1] / e[2])
        expect = 1 if scheme == 1 else 2
        assert abs(order - expect) < 0.15, (scheme, e)
    assert errs[2][2] < errs[1][2]


def test_cgl_plane_wave_setd2_order2(oracle_mod):
    """Sec. V.C: for D = 0 the plane wave R e^{i(qx - Omega t)}, R = sqrt(1-q^2),
    Omega = alpha q^2 + beta (1 - q^2) is exact.  SETD2 error ~ h^2, SETD1 ~ h."""
    N, dx = 32, 0.5
    L = N * dx
    q = 2 * np.pi * 2 / L
    al, be = 2.0, -0.5
    w = W.cgl_2048(n=[N], d=1, dx=[dx], p=[al, be, 0.0])
    x = np.arange(N) * dx
    R = math.sqrt(1 - q * q)
    Om = al * q * q + be * (1 - q * q)
    A0 = R * np.exp(1j * q * x)
    T = 2.0
    for scheme, expect in ((2, 2), (1, 1)):
        e = []
        for nst in (20, 40, 80):
            o = make_oracle(oracle_mod, w.with_(scheme=scheme, h=T / nst))
            o.set_field(0, A0)
            o.step(nst)
            e.append(np.abs(o.field(0) - R * np.exp(1j * (q * x - Om * T))).max())
        order = math.log2(e[1] / e[2])
        assert abs(order - expect) < 0.2, (scheme, e)


def test_cgl_deterministic_vs_integrator(oracle_mod):
    from scipy.integrate import solve_ivp
    N, dx, T = 16, 0.8, 0.3
    p = [2.0, -0.5, 0.0]
    w = W.cgl_2048(n=[N], d=1, dx=[dx], p=p)
    f0 = W.smooth_field(w, amplitude=0.5, seed=3)[0]
    rhs = _real_space_rhs(3, p, w.shape, dx, 1)
    y = solve_ivp(rhs, (0, T), np.concatenate([f0.real, f0.imag]), method="DOP853", rtol=1e-12,
                  atol=1e-13).y[:, -1]
    ref = y[:N] + 1j * y[N:]
    e = []
    for nst in (50, 100):
        o = make_oracle(oracle_mod, w.with_(scheme=2, h=T / nst))
        o.set_field(0, f0)
        o.step(nst)
        e.append(np.abs(o.field(0) - ref).max())
    assert e[1] < 1e-4 and abs(math.log2(e[0] / e[1]) - 2) < 0.25, e


def test_kpz_cole_hopf(oracle_mod):
    """Sec. V.B deterministic KPZ in 1-D maps to the heat equation (Cole-Hopf):
    h = (2 nu / lambda) ln Z, Z = sum_m I_m(lambda eps / 2 nu) e^{-nu m^2 k^2 t} cos(m k x)
    for h(x, 0) = eps cos(k x).  SETD1 must converge to it with order 1."""
    from scipy.special import iv
    nu, lam, eps = 1.0, 1.0, 0.4
    N, dx = 64, 0.25
    L = N * dx
    k = 2 * np.pi / L
    x = np.arange(N) * dx
    T = 0.5
    beta = lam * eps / (2 * nu)
    Z = iv(0, beta) * np.ones(N)
    for m in range(1, 30):
        Z = Z + 2 * iv(m, beta) * np.exp(-nu * m * m * k * k * T) * np.cos(m * k * x)
    exact = (2 * nu / lam) * np.log(Z)
    w = W.kpz_1d(N, dx=[dx], p=[nu, lam, 0.0], dealias=0)
    e = []
    for nst in (50, 100, 200):
        o = make_oracle(oracle_mod, w.with_(h=T / nst))
        o.set_field(0, eps * np.cos(k * x))
        o.step(nst)
        e.append(np.abs(o.field(0) - exact).max())
    assert e[2] < 2e-4
    assert abs(math.log2(e[1] / e[2]) - 1) < 0.15, e


def test_sao_boltzmann(oracle_mod):
    """A one-site Model A lattice is the stochastic anharmonic oscillator of
    Sec. III.A; its stationary law is P(u) ~ exp(-V/T), V = u^2/2 + b u^4/4."""
    from scipy.integrate import quad
    G, T, b = 5.0, 6.0, 0.01
    w = W.model_a_64(n=[1], d=1, dx=[1.0], p=[G, 1.0, b, T], h=0.01)
    R = 2000
    o = make_oracle(oracle_mod, w, replicas=R)
    o.step(200)
    samples = []
    for _ in range(40):
        o.step(10)
        samples.extend([o.spectrum(r)[0].real for r in range(R)])
    u = np.array(samples)
    Zn = quad(lambda s: math.exp(-(s * s / 2 + b * s ** 4 / 4) / T), -60, 60)[0]
    m2 = quad(lambda s: s * s * math.exp(-(s * s / 2 + b * s ** 4 / 4) / T), -60, 60)[0] / Zn
    m4 = quad(lambda s: s ** 4 * math.exp(-(s * s / 2 + b * s ** 4 / 4) / T), -60, 60)[0] / Zn
    neff = R * 40 / 3  # snapshots 10 steps apart are correlated (relaxation time 1/Gamma = 20 steps)
    assert abs(np.mean(u ** 2) - m2) < 4 * m2 * math.sqrt(2 / neff) + 0.02 * m2
    assert abs(np.mean(u ** 4) - m4) < 4 * m4 * math.sqrt(8 / neff) + 0.04 * m4


def test_strong_order_one_additive(oracle_mod):
    """Sec. III.C: for additive noise the SETD schemes have strong order 1.
    Coarse noise is built from the fine path exactly: for SETD1,
    xi_c = (e^{c h} xi_1 + xi_2) f4(h) / f4(2h) (exact I1 of the combined
    interval); the reference uses h_min / 4."""
    N, R, T = 8, 12, 0.32
    p = [1.0, -0.5, 1.0, 0.5]
    base = W.model_a_64(n=[N, N], p=p, scheme=1)
    f0 = W.initial_fields(base.with_(sigma0=0.3), replicas=R)
    hf = T / 256
    fine = make_oracle(oracle_mod, base.with_(h=hf), replicas=R)
    etas = np.array([[fine.noise(r, s) for r in range(R)] for s in range(256)])  # (steps, R, N, N)
    KY, KX = spectral_k(base.shape, 1.0)
    c = -(p[1] + KX ** 2 + KY ** 2)

    def f4sq(h):
        return np.expm1(2 * c * h) / (2 * c)

    def run(level):
        h = hf * 2 ** level
        e = etas
        hh = hf
        for _ in range(level):
            e = (np.exp(c * hh) * e[0::2] + e[1::2]) * np.sqrt(f4sq(hh) / f4sq(2 * hh))
            hh *= 2
        o = make_oracle(oracle_mod, base.with_(h=h), replicas=R)
        for r in range(R):
            o.set_field(r, f0[r])
        for s in range(e.shape[0]):
            o.step_with_noise(e[s])
        return np.array([o.field(r) for r in range(R)])

    ref = run(0)
    errs = [np.mean(np.abs(run(lv) - ref)) for lv in (2, 3, 4)]
    slope = math.log2(errs[2] / errs[0]) / 2
    assert abs(slope - 1) < 0.2, errs


# ------------------------------------------------------------ observables
def test_kpz_width_parseval(oracle_mod):
    """Sec. V.B width with the box equal to the system: the Fourier-space
    w^2 = N^{-2d} sum_{a != 0} |h_a|^2 equals the real-space variance."""
    w = W.kpz_2d(n=[16, 16], h=0.01)
    o = make_oracle(oracle_mod, w, replicas=3)
    o.step(30)
    w2 = o.roughness()
    for r in range(3):
        f = o.field(r)
        assert abs(w2[r] - np.var(f)) <= 1e-12 * np.var(f)


def test_field_stays_real_and_hermitian(oracle_mod):
    for model, n in ((0, [8, 8, 8]), (1, [16, 16]), (2, [32])):
        p = [1.0, 2.0, 0.5] if model == 2 else [1.0, -0.5, 1.0, 0.5]
        w = W.model_a_64(d=len(n), n=n, dx=[1.0] * len(n), model=model, p=p, scheme=2, sigma0=0.2)
        o = make_oracle(oracle_mod, w)
        o.set_field(0, W.initial_fields(w)[0])
        o.step(5)
        S = o.spectrum(0)
        Sneg = np.conj(np.roll(np.flip(S), 1, axis=tuple(range(S.ndim))))
        assert np.array_equal(S, Sneg)


def test_init_random_statistics(oracle_mod):
    w = W.model_a_64(n=[32, 32])
    o = make_oracle(oracle_mod, w, replicas=4)
    o.init_random(0.7)
    f = np.array([o.field(r) for r in range(4)])
    assert abs(f.mean()) < 4 * 0.7 / math.sqrt(f.size)
    assert abs(f.var() / 0.49 - 1) < 4 * math.sqrt(2 / f.size)
    # site s of replica r is sigma * normal[s & 3] of Philox(ctr = (s >> 2, 0, r, 1))
    z = oracle_mod.normals4(w.seed, 5, 0, 2, 1)
    assert abs(f[2].reshape(-1)[21] - 0.7 * float(z[1])) < 1e-12


# ------------------------------------------------------------ tangent / adjoint
@pytest.mark.parametrize("model,scheme", [(0, 1), (1, 1), (2, 1), (3, 2), (0, 2), (2, 2), (3, 1)])
def test_tangent_matches_finite_differences(oracle_mod, model, scheme):
    """The tangent (forward-mode linearisation on the same noise path) must
    equal the central difference (Phi(+e) - Phi(-e)) / 2e up to O(e^2)."""
    n = [16, 16]
    if model == 2:
        p = [1.0, 2.0, 0.5]
    elif model == 3:
        p = [2.0, -0.5, 1e-3]
    else:
        p = [1.0, -0.5, 1.0, 0.3]
    w = W.model_a_64(n=n, model=model, p=p, scheme=scheme, h=0.02, sigma0=0.3)
    f0 = W.initial_fields(w)[0]
    d0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=5)[0]
    nst = 15

    def run(eps):
        o = make_oracle(oracle_mod, w)
        o.set_field(0, f0 + eps * d0)
        o.step(nst)
        return o.field(0)

    o = make_oracle(oracle_mod, w)
    o.set_field(0, f0)
    tan = o.tangent_step(d0[None], nst)[0]
    errs = []
    for eps in (1e-3, 5e-4):
        fd = (run(eps) - run(-eps)) / (2 * eps)
        errs.append(np.abs(fd - tan).max() / np.abs(tan).max())
    assert errs[1] < 1e-5
    assert errs[1] < errs[0] or errs[1] < 1e-9
    # the primal advanced along the same path
    assert np.allclose(o.field(0), run(0.0), rtol=0, atol=1e-13)


@pytest.mark.parametrize("model,scheme,pre", [(0, 1, 0), (1, 1, 0), (2, 1, 0), (0, 2, 0), (1, 2, 0), (2, 2, 0),
                                               (0, 2, 3), (1, 0, 0)])
def test_adjoint_dot_product_identity(oracle_mod, model, scheme, pre):
    """<lambda_N, T delta_0> = <A lambda_N, delta_0> with T the tangent and A the
    adjoint over the same steps, real-space inner product, to rounding.  The
    tangent is pinned by finite differences above, so this pins the adjoint;
    SETD2 covers the history cotangent (pre > 0: the SETD2 history already
    running when the tangent is seeded)."""
    p = [1.0, 2.0, 0.5] if model == 2 else [1.0, -0.5, 1.0, 0.3]
    w = W.model_a_64(n=[16, 16], model=model, p=p, scheme=scheme, h=0.02, sigma0=0.3)
    f0 = W.initial_fields(w, replicas=2)
    d0 = W.initial_fields(w.with_(sigma0=1.0), replicas=2, seed_offset=3)
    lam = W.initial_fields(w.with_(sigma0=1.0), replicas=2, seed_offset=4)
    nst = 12
    o = make_oracle(oracle_mod, w, replicas=2)
    for r in range(2):
        o.set_field(r, f0[r])
    o.step(pre)
    tan = o.tangent_step(d0, nst)
    o2 = make_oracle(oracle_mod, w, replicas=2)
    for r in range(2):
        o2.set_field(r, f0[r])
    o2.step(pre)
    grad = o2.adjoint(lam, nst)
    for r in range(2):
        lhs = np.sum(lam[r] * tan[r])
        rhs = np.sum(grad[r] * d0[r])
        assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1e-300), (lhs, rhs)


@pytest.mark.parametrize("d,scheme,pre", [(2, 1, 0), (2, 2, 0), (2, 2, 3), (2, 0, 0), (1, 2, 0), (1, 1, 2)])
def test_adjoint_dot_product_identity_complex(oracle_mod, d, scheme, pre):
    """CGL (Sec. V.C, complex field): with the real inner product
    Re sum_x conj(u) v, <lambda_N, T delta_0> = <A lambda_N, delta_0> to
    rounding, T the tangent (pinned by finite differences above, model 3)."""
    n = [16, 16] if d == 2 else [32]
    w = W.model_a_64(d=d, n=n, dx=[1.0] * d, model=3, p=[2.0, -0.5, 1e-3], scheme=scheme, h=0.02, sigma0=0.3)
    assert w.complex_field
    f0 = W.initial_fields(w, replicas=2)
    d0 = W.initial_fields(w.with_(sigma0=1.0), replicas=2, seed_offset=3)
    lam = W.initial_fields(w.with_(sigma0=1.0), replicas=2, seed_offset=4)
    nst = 12
    o = make_oracle(oracle_mod, w, replicas=2)
    for r in range(2):
        o.set_field(r, f0[r])
    o.step(pre)
    tan = o.tangent_step(d0, nst)
    o2 = make_oracle(oracle_mod, w, replicas=2)
    for r in range(2):
        o2.set_field(r, f0[r])
    o2.step(pre)
    grad = o2.adjoint(lam, nst)
    for r in range(2):
        lhs = np.sum(np.conj(lam[r]) * tan[r]).real
        rhs = np.sum(np.conj(grad[r]) * d0[r]).real
        assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1e-300), (lhs, rhs)
    # the primal ends where plain steps end
    o3 = make_oracle(oracle_mod, w, replicas=2)
    for r in range(2):
        o3.set_field(r, f0[r])
    o3.step(pre + nst)
    assert np.allclose(o2.field(1), o3.field(1), rtol=0, atol=1e-13)


def test_adjoint_complex_gradient_by_finite_differences(oracle_mod):
    """CGL adjoint against a directional derivative of the scalar
    J(phi_0) = Re <lambda, phi_N(phi_0)>: Re <grad J, delta> equals the central
    difference of J along delta (O(e^2)), for a real and an imaginary delta."""
    w = W.model_a_64(n=[16, 16], model=3, p=[2.0, -0.5, 1e-3], scheme=2, h=0.02, sigma0=0.3)
    f0 = W.initial_fields(w)[0]
    lam = W.initial_fields(w.with_(sigma0=1.0), seed_offset=4)
    base = W.initial_fields(w.with_(sigma0=1.0), seed_offset=6)[0]
    nst = 10
    o = make_oracle(oracle_mod, w)
    o.set_field(0, f0)
    grad = o.adjoint(lam, nst)[0]

    def J(x):
        q = make_oracle(oracle_mod, w)
        q.set_field(0, x)
        q.step(nst)
        return np.sum(np.conj(lam[0]) * q.field(0)).real

    for delta in (base.real + 0j, 1j * base.imag):
        eps = 1e-4
        fd = (J(f0 + eps * delta) - J(f0 - eps * delta)) / (2 * eps)
        ad = np.sum(np.conj(grad) * delta).real
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("model,scheme", [(0, 1), (1, 1), (0, 0), (1, 0)])
def test_r_in_F_linear_closed_form(oracle_mod, model, scheme):
    """Model A/B with r placed in F (p[4] = 1, the variant of the Sec. V.A
    footnote), u = 0 and no noise: each mode follows
    phi_n = (e^{c0 h} + h phi1(c0 h) s_r)^n phi_0, c0 = -Gamma k^Delta k^2,
    s_r = -Gamma r k^Delta (the explicit r phi term of F)."""
    G, r, h, n = 1.3, -0.7, 0.05, 12
    N, L = 16, 16.0
    o = oracle_mod.Oracle(2, [N, N], [L / N, L / N], 1, model, [G, r, 0.0, 0.0, 1.0], scheme, h, seed=5)
    rng = np.random.default_rng(0)
    f0 = rng.normal(size=(N, N))
    o.set_field(0, f0)
    o.step(n)
    k = 2 * np.pi * np.fft.fftfreq(N, L / N)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    kd = k2 if model == 1 else np.ones_like(k2)
    c0 = -G * kd * k2
    z = c0 * h
    phi1 = np.where(np.abs(z) > 1e-12, np.expm1(z) / np.where(z == 0, 1, z), 1.0)
    f = np.exp(z) + h * phi1 * (-G * r * kd)
    want = np.fft.fft2(f0) * f ** n
    got = o.spectrum(0)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


# ------------------------------------------------------------ 3 x 2^k lattices
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_noise_free_linear_propagation_3x2k(oracle_mod, scheme):
    """48 x 48 (a lattice of 3 x 2^k points): u = 0, D = 0 propagates every mode by
    e^{c h} per step exactly, with numpy's wavenumbers."""
    p = [1.0, 0.3, 0.0, 0.0]
    w = W.model_a_64(n=[48, 48], dx=[0.7, 0.7], model=1, p=p, scheme=scheme, h=0.05)
    o = make_oracle(oracle_mod, w)
    rng = np.random.default_rng(5)
    f0 = rng.standard_normal(w.shape)
    o.set_field(0, f0)
    S0 = np.fft.fft2(f0)
    n = 30
    o.step(n)
    KY, KX = spectral_k(w.shape, 0.7)
    k2 = KX ** 2 + KY ** 2
    decay = np.exp(-k2 * (0.3 + k2) * n * w.h)
    expect = S0 * decay
    got = o.spectrum(0)
    # each mode to rounding of the transforms, on the scale of its own decay
    live = decay > 1e-200
    err = np.abs(got - expect)[live] / (np.abs(S0).max() * decay[live])
    # rounding of c h (relative eps) grows the error of e^{c h n} by |c h n| eps
    cnh = (k2 * (0.3 + k2) * n * w.h)[live]
    assert np.all(err <= 4 * 2.2e-16 * (n + cnh) + 1e-13)
    assert np.abs(got[~live]).max() <= 1e-200 * np.abs(S0).max()


def test_noise_structure_3x2k(oracle_mod):
    """App. B on a 24 x 24 lattice: Hermitian noise, real self-conjugate modes,
    unit mean |eta_a|^2."""
    N = 24
    o = make_oracle(oracle_mod, W.model_a_64(n=[N, N]))
    acc = np.zeros((N, N))
    for s in range(200):
        eta = o.noise(0, s)
        assert np.array_equal(eta, np.conj(np.roll(eta[::-1, ::-1], 1, axis=(0, 1))))
        for iy in (0, N // 2):
            for ix in (0, N // 2):
                assert eta[iy, ix].imag == 0.0
        acc += np.abs(eta) ** 2
    assert abs(acc.mean() / 200 - 1.0) < 4 * math.sqrt(2 / (200 * N * N))


def test_gaussian_model_a_structure_factor_3x2k(oracle_mod):
    """Sec. V.A linear theory C_ET(k) = T / (r + k^2) on a 24 x 24 lattice."""
    N, R = 24, 48
    w = W.model_a_64(n=[N, N], dx=[0.5, 0.5], p=[1.0, 1.0, 0.0, 0.6], h=0.05)
    o = make_oracle(oracle_mod, w, replicas=R)
    o.step(200)
    acc = None
    S = 15
    for _ in range(S):
        o.step(20)
        v, _ = o.shells(0)
        acc = v if acc is None else acc + v
    v = acc / S
    dk = 2 * np.pi / (N * 0.5)
    KY, KX = spectral_k(w.shape, 0.5)
    kk = np.sqrt(KX ** 2 + KY ** 2)
    for j in range(1, 6):
        sel = (kk > (j - 1) * dk + 1e-9) & (kk <= j * dk + 1e-9)
        ref = np.mean(0.6 / (1.0 + kk[sel] ** 2))
        assert abs(v[j] - ref) < 5 * ref / math.sqrt(sel.sum() * R * S / 4), (j, v[j], ref)
