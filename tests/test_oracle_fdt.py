"""Pin of the oracle's interacting dynamics by the fluctuation-dissipation
relation (Sec. V.A): in equilibrium Model A (Gamma = 1, noise strength D = T),
the response of mode k to an impulse in its own amplitude at t0 and the
two-time correlation satisfy R(k, tau) = -(1/T) dC(k, tau)/dtau, here in the
integrated form

    int_0^tau R(k, s) ds = (C(k, 0) - C(k, tau)) / T.

R comes from the oracle's tangent (the linearised step on the same noise
path, seeded by a random impulse dphi(t0); its projection on the seed,
shell by shell), C from the oracle's states (App. C shells and
normalisation).  Nothing here restates the step: the relation ties the
noise amplitude, the linear operator and the linearised cubic term together,
so a wrong amplitude, temperature or tangent term breaks it.  Model A 16^2,
r = 0.5, u = 4 (strong enough that the response differs from the free one),
T = 1, SETD2, h = 0.02 (the scheme's bias stays below the statistical error),
192 replicas x 4 windows of 40 steps after a burn-in of 8 time units, shells
1-5 at tau = 0.2, 0.4, 0.8: every mean deviation within 4 standard errors.
The same data fail by far with the temperature off by 15 %, or with the free
response e^{-(r + k^2) tau} (a tangent without the cubic term) in place of the
oracle's."""
import numpy as np

import sft_inputs as W

N, R, H, T = 16, 192, 0.02, 1.0
WINDOWS, M, TAUS, SHELLS = 4, 40, (10, 20, 40), range(1, 6)


def test_fluctuation_dissipation_relation_interacting_model_a(oracle_mod):
    r0 = 0.5
    w = W.model_a_64(n=[N, N], p=[1.0, r0, 4.0, T], scheme=2, h=H, sigma0=0.5, replicas=R)
    o = oracle_mod.Oracle(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    f0 = W.initial_fields(w)
    for r in range(R):
        o.set_field(r, f0[r])
    o.step(400)
    k = 2 * np.pi * np.fft.fftfreq(N)
    KY, KX = np.meshgrid(k, k, indexing="ij")
    shell = np.ceil(np.sqrt(KX ** 2 + KY ** 2) / (2 * np.pi / N) - 1e-9).astype(int)
    masks = [shell == j for j in SHELLS]
    k2 = KX ** 2 + KY ** 2
    nrm = (1.0 / N) ** 2  # (dx / N)^d, App. C
    D, D0, rhs = [], [], []
    for win in range(WINDOWS):
        S0 = np.array([o.spectrum(r) for r in range(R)])
        seed = W.initial_fields(w.with_(sigma0=1.0), seed_offset=100 + win)
        s = np.fft.fft2(seed)
        C, Rs, R0 = [], [], []
        for m in range(M + 1):
            o.tangent_step(seed if m == 0 else None, 0 if m == 0 else 1)
            Sm = np.array([o.spectrum(r) for r in range(R)])
            dm = np.array([o.tangent_spectrum(r) for r in range(R)])
            C.append([[nrm * np.mean((Sm[r] * np.conj(S0[r])).real[q]) for q in masks] for r in range(R)])
            Rs.append([[np.sum((dm[r] * np.conj(s[r])).real[q]) / np.sum(np.abs(s[r][q]) ** 2) for q in masks]
                       for r in range(R)])
            # the free response, for the power check only
            R0.append([[np.sum(np.exp(-(r0 + k2[q]) * m * H) * np.abs(s[r][q]) ** 2) / np.sum(np.abs(s[r][q]) ** 2)
                        for q in masks] for r in range(R)])
        C, Rs, R0 = np.array(C), np.array(Rs), np.array(R0)  # (M + 1, R, shells)
        # trapezoidal integral of the response over the steps (its error is O(h^2) of the decay)
        D.append([H * (0.5 * Rs[0] + Rs[1:m].sum(0) + 0.5 * Rs[m]) for m in TAUS])
        D0.append([H * (0.5 * R0[0] + R0[1:m].sum(0) + 0.5 * R0[m]) for m in TAUS])
        rhs.append([C[0] - C[m] for m in TAUS])
        o.step(100)  # decorrelate the windows
    pool = lambda a: np.array(a).transpose(1, 0, 2, 3).reshape(len(TAUS), WINDOWS * R, len(SHELLS))
    I, I0, dC = pool(D), pool(D0), pool(rhs)

    def zscores(integral, temp):
        dev = integral - dC / temp
        return dev.mean(1) / (dev.std(1, ddof=1) / np.sqrt(dev.shape[1]))

    z = zscores(I, T)
    assert np.abs(z).max() < 4.0, np.round(z, 2)
    assert np.abs(zscores(I, 1.15 * T)).max() > 8.0
    assert np.abs(zscores(I0, T)).max() > 8.0
