"""0-d SDE ensembles (Sec. III) on the GPU through the C ABI: bit-identical to
the oracle for every problem and scheme (FP64, every operation one correctly
rounded IEEE operation in the same order, the same Philox normals), and the
strong orders of convergence on a large ensemble."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_22510_gb300 as m
    m.load_library()
    return m, torch


PROBLEMS = [("sao", 0, [5.0, 6.0, 0.01]), ("gbm", 1, [2.0, 1.0, 1.0]), ("gbm_exact_drift", 1, [-1.0, 0.7, 0.0])]


@pytest.mark.parametrize("name,kind,p", PROBLEMS, ids=[x[0] for x in PROBLEMS])
@pytest.mark.parametrize("scheme", range(5), ids=["EM", "Milstein", "SETD-EM", "SETD-Milstein", "SETD1"])
def test_sde0d_bit_identical_to_oracle(env, oracle_mod, name, kind, p, scheme):
    m, torch = env
    S, h, n, sub = 1003, 0.05, 40, 3  # a path count that is not a multiple of 4
    u0 = np.linspace(0.5, 1.5, S)
    u = torch.from_numpy(u0.copy()).cuda()
    w = torch.zeros(S, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for step0 in (0, n):  # two calls in a row continue the same Wiener path
        m.sft_sde0d(kind, p, scheme, h, n, u.data_ptr(), S, seed=77, substeps=sub, step0=step0,
                    w_dev_ptr=w.data_ptr())
    torch.cuda.synchronize()
    uo, wo = oracle_mod.sde0d(kind, p, scheme, h, 2 * n, u0, seed=77, substeps=sub)
    assert np.array_equal(u.cpu().numpy(), uo)
    assert np.array_equal(w.cpu().numpy(), wo)


def test_sde0d_strong_orders_on_the_gpu(env):
    """GBM (lambda = 2, mu = 1, delta = 1) at t = 1 against the exact solution on
    the same Wiener path: strong order 1/2 (EM, SETD-EM) and 1 (Milstein,
    SETD-Milstein), on 2^18 paths."""
    m, torch = env
    lam, mu, delta = 2.0, 1.0, 1.0
    S, kmax = 1 << 18, 8
    for scheme, order in ((0, 0.5), (1, 1.0), (2, 0.5), (3, 1.0)):
        hs, errs = [], []
        for k in range(4, kmax + 1):
            h = 2.0 ** -k
            u = torch.ones(S, dtype=torch.float64, device="cuda")
            w = torch.zeros(S, dtype=torch.float64, device="cuda")
            m.sft_sde0d(1, [lam, mu, delta], scheme, h, 2 ** k, u.data_ptr(), S, seed=3, substeps=2 ** (kmax - k),
                        w_dev_ptr=w.data_ptr())
            exact = torch.exp((lam - 0.5 * mu * mu) + mu * w)
            errs.append(float(torch.mean(torch.abs(u - exact))))
            hs.append(h)
        slope = float(np.polyfit(np.log(hs), np.log(errs), 1)[0])
        assert abs(slope - order) < 0.1, (scheme, slope, errs)


def test_sde0d_arguments(env):
    m, torch = env
    u = torch.ones(8, dtype=torch.float64, device="cuda")
    m.sft_sde0d(0, [5.0, 6.0, 0.0], 4, 0.1, 0, u.data_ptr(), 8, seed=1)  # zero steps: nothing changes
    m.sft_sde0d(0, [5.0, 6.0, 0.0], 4, 0.1, 5, 0, 0, seed=1)             # zero paths: nothing to do
    torch.cuda.synchronize()
    assert torch.all(u == 1.0)
    for kw in (dict(kind=2), dict(scheme=5), dict(h=0.0), dict(substeps=0)):
        args = dict(kind=0, p=[5.0, 6.0, 0.0], scheme=4, h=0.1, nsteps=3, u_dev_ptr=u.data_ptr(), npaths=8, seed=1)
        args.update(kw)
        with pytest.raises(m.SftError) as ei:
            m.sft_sde0d(**args)
        assert ei.value.status == m.SFT_EINVAL
