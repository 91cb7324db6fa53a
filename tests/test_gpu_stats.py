"""Long-run statistics of the GPU stepper against exact results.

Gaussian Model A and Model B (u = 0) are Ornstein-Uhlenbeck processes per
Fourier mode.  SETD1 (Sec. II) integrates each exactly in distribution, so the
stationary equal-time structure factor is S(k) = T / (r + k^2) for every mode
(Sec. V.A; Model B's conserved noise and k^2 mobility cancel), at any h.  The
test runs 8 independent ensembles (8 seeds, 8 replicas each) to equilibrium and
samples the per-replica shell averages (App. C) at well separated times.  The
shells are pooled into 8 bands of consecutive shells (mode-count weights);
every band must agree with the exact band average within 3 standard errors
(estimated from the samples).  Every single shell must lie within 4.5 standard
errors (with up to 47 shells a 3-sigma cut per shell would fail a correct
stepper about one time in eight), and the mean squared z-score of the shells
must be that of a unit normal.
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


def exact_shells(n, L, r, T):
    """Shell average of T / (r + k^2) over the full-spectrum modes of shell
    j = ceil(|a|), k = 2 pi |a| / L, and the mode counts."""
    a = np.fft.fftfreq(n, 1.0 / n)
    ax, ay = np.meshgrid(a, a, indexing="ij")
    mag = np.sqrt(ax ** 2 + ay ** 2)
    shell = np.ceil(mag - 1e-12).astype(int)
    k2 = (2 * np.pi / L) ** 2 * mag ** 2
    val = T / (r + k2)
    ns = shell.max() + 1
    counts = np.bincount(shell.ravel(), minlength=ns)
    sums = np.bincount(shell.ravel(), weights=val.ravel(), minlength=ns)
    return sums / np.maximum(counts, 1), counts


SEEDS = [11, 12, 13, 14, 15, 16, 17, 18]

CASES = [
    # relaxation time of the slowest mode: 20 steps (Model A, 1 / (Gamma r h));
    # 20 steps (Model B 16^2, 1 / (Gamma k1^2 (r + k1^2) h)); samples 5 of them apart
    ("model_a", W.model_a_64(p=[1.0, 0.5, 0.0, 0.5], h=0.1, replicas=8, sigma0=0.0), 1000, 100),
    ("model_b", W.model_b_1024(n=[16, 16], p=[1.0, 0.5, 0.0, 0.5], h=0.5, replicas=8, sigma0=0.0), 2000, 100),
]


@pytest.mark.parametrize("name,w,n_eq,gap", CASES, ids=[c[0] for c in CASES])
def test_gaussian_structure_factor(sft, name, w, n_eq, gap):
    samples = []
    for seed in SEEDS:
        g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, seed, dealias=w.dealias)
        g.set_field(np.zeros((w.replicas,) + w.shape, dtype=np.float32))
        g.step(n_eq)
        ns = g.nshells()
        for _ in range(20):
            g.step(gap)
            samples.append(g.observe(sft.SFT_OBS_SK_REPLICAS).reshape(w.replicas, ns))
        counts = g.observe(sft.SFT_OBS_SK)[ns:]
        g.close()
    S = np.concatenate(samples)
    exp, exp_counts = exact_shells(w.n[0], w.n[0] * w.dx[0], w.p[1], w.p[3])
    assert len(exp) == ns and np.array_equal(counts, exp_counts)
    first = 0 if name == "model_a" else 1  # Model B conserves the k = 0 mode (zero here)
    if first:
        assert np.all(S[:, 0] == 0.0)
    mean = S.mean(axis=0)[first:]
    se = S.std(axis=0, ddof=1)[first:] / np.sqrt(S.shape[0])
    z = (mean - exp[first:]) / se
    assert np.all(np.abs(z) < 4.5), (name, np.argmax(np.abs(z)) + first, z[np.argmax(np.abs(z))])
    assert 0.5 < float(np.mean(z ** 2)) < 1.6, (name, float(np.mean(z ** 2)))
    # 8 bands of consecutive shells, each the mode-count-weighted mean of its shells
    shells = np.arange(first, ns)
    for band in np.array_split(shells, 8):
        wts = counts[band] / counts[band].sum()
        b = S[:, band] @ wts
        zb = (b.mean() - float(exp[band] @ wts)) / (b.std(ddof=1) / np.sqrt(len(b)))
        assert abs(zb) < 3.0, (name, band[0], band[-1], zb)
