"""Pin of the oracle's linear-response observable (the tangent seeded by an
impulse dphi(t0), projected per shell onto the seed: the response R(k, t) of
Sec. V.A with the shells of App. C).  In the linear model (u = 0) the tangent
of the step is the step's own propagator, so dPhi_a(t0 + n h) = e^{c_a n h}
dPhi_a(t0) exactly for every scheme (Sec. II with F = 0), and the per-shell
response is sum_a e^{c_a n h} |dPhi_a(t0)|^2 / sum_a |dPhi_a(t0)|^2 over the
modes of the shell, computed here from numpy's wavenumbers and shells
(ceil(|k| / dk), App. C)."""
import numpy as np
import pytest

import sft_inputs as W


@pytest.mark.parametrize("model,scheme", [(0, 0), (0, 1), (0, 2), (1, 1)])
def test_linear_response_is_the_propagator(oracle_mod, model, scheme):
    N, dx, h, nst, R = 16, 0.7, 0.04, 30, 2
    p = [1.2, 0.4, 0.0, 0.5]  # u = 0: linear; T > 0, so the primal carries noise the tangent must not see
    w = W.model_a_64(n=[N, N], dx=[dx, dx], model=model, p=p, scheme=scheme, h=h, sigma0=0.3, replicas=R)
    o = oracle_mod.Oracle(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    f0 = W.initial_fields(w)
    for r in range(R):
        o.set_field(r, f0[r])
    seed = W.initial_fields(w.with_(sigma0=1.0), seed_offset=9)
    o.tangent_step(seed, nst)
    k = [2 * np.pi * np.fft.fftfreq(N, d=dx)] * 2
    KY, KX = np.meshgrid(*k, indexing="ij")
    k2 = KX ** 2 + KY ** 2
    c = -p[0] * (p[1] + k2) if model == 0 else -p[0] * k2 * (p[1] + k2)
    prop = np.exp(c * nst * h)
    S0 = np.fft.fft2(seed)
    for r in range(R):
        got = o.tangent_spectrum(r)
        np.testing.assert_allclose(got, prop * S0[r], rtol=0, atol=1e-12 * np.abs(S0[r]).max())
    dk = 2 * np.pi / (N * dx)
    shell = np.ceil(np.sqrt(k2) / dk - 1e-9).astype(int)
    resp = o.response()
    for j in range(resp.size):
        sel = shell == j
        den = sum(np.sum(np.abs(S0[r][sel]) ** 2) for r in range(R))
        if den == 0:
            continue
        ref = sum(np.sum(prop[sel] * np.abs(S0[r][sel]) ** 2) for r in range(R)) / den
        assert abs(resp[j] - ref) <= 1e-12, (j, resp[j], ref)
