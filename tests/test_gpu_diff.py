"""GPU parity of the differentiated step: the tangent (forward mode, advanced
with the primal on the same noise path) and the checkpointed adjoint, through
the C ABI with device buffers, against the FP64 oracle (whose tangent is pinned
by finite differences and whose adjoint by the dot-product identity)."""
import numpy as np
import pytest

import sft_inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_22510_gb300 as m
    m.load_library()
    return m, torch


def make_pair(m, oracle_mod, w, f0):
    g = m.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    g.set_field(f0.astype(np.float32))
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(w.replicas):
        o.set_field(r, f0[r].astype(np.float32).astype(np.float64))
    return g, o


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    ("model_a_64", W.model_a_64(n=[64, 64], replicas=2, sigma0=0.3, h=0.02)),
    ("model_b_32_em", W.model_b_1024(n=[32, 32], replicas=2, sigma0=0.3, scheme=0, h=0.02)),
    ("model_a_1d_256", W.model_a_64(d=1, n=[256], dx=[1.0], replicas=3, sigma0=0.3, h=0.02)),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_tangent_parity(env, oracle_mod, name, w):
    m, torch = env
    f0 = W.initial_fields(w)
    d0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=9)
    g, o = make_pair(m, oracle_mod, w, f0)
    nst = 20
    dev_in = torch.from_numpy(d0.astype(np.float32)).cuda()
    dev_out = torch.zeros_like(dev_in)
    torch.cuda.synchronize()
    m.sft_tangent_step(g.ctx, dev_in.data_ptr(), nst, dev_out.data_ptr())
    torch.cuda.synchronize()
    tan_o = o.tangent_step(d0, nst)
    tan_g = dev_out.cpu().numpy()
    for r in range(w.replicas):
        assert rel(tan_g[r], tan_o[r]) <= 1e-5, (name, r, rel(tan_g[r], tan_o[r]))
        assert rel(g.field()[r], o.field(r)) <= 1e-5
    # response observable (shell-resolved projection on the seed)
    resp = g.observe(m.SFT_OBS_RESPONSE)
    ro = o.response()
    assert np.allclose(resp, ro, rtol=1e-4, atol=1e-6)
    g.close()


def test_tangent_matches_gpu_finite_differences(env):
    m, torch = env
    w = W.model_b_1024(n=[64, 64], replicas=1, sigma0=0.3, h=0.02)
    f0 = W.initial_fields(w).astype(np.float32)
    d0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=2).astype(np.float32)
    nst = 15

    def run(eps):
        g = m.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed)
        g.set_field((f0.astype(np.float64) + eps * d0).astype(np.float32))
        g.step(nst)
        out = g.field().astype(np.float64)
        g.close()
        return out

    g = m.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed)
    g.set_field(f0)
    dev_in = torch.from_numpy(d0).cuda()
    dev_out = torch.zeros_like(dev_in)
    torch.cuda.synchronize()
    m.sft_tangent_step(g.ctx, dev_in.data_ptr(), nst, dev_out.data_ptr())
    torch.cuda.synchronize()
    tan = dev_out.cpu().numpy().astype(np.float64)
    eps = 1e-2
    fd = (run(eps) - run(-eps)) / (2 * eps)
    assert rel(fd, tan) < 2e-3
    g.close()


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_adjoint_dot_product_and_parity(env, oracle_mod, name, w):
    """<lambda, T delta> = <A lambda, delta> on the GPU, and the GPU gradient
    against the oracle's; checkpoint segments of 7 steps over a 20-step horizon
    force the recompute of the primal from checkpoints."""
    m, torch = env
    f0 = W.initial_fields(w)
    d0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=3).astype(np.float32)
    lam = W.initial_fields(w.with_(sigma0=1.0), seed_offset=4).astype(np.float32)
    nst = 20
    g1, o = make_pair(m, oracle_mod, w, f0)
    din = torch.from_numpy(d0).cuda()
    dout = torch.zeros_like(din)
    torch.cuda.synchronize()
    m.sft_tangent_step(g1.ctx, din.data_ptr(), nst, dout.data_ptr())
    g2, _ = make_pair(m, oracle_mod, w, f0)
    m.sft_set_checkpoint_interval(g2.ctx, 7)
    lin = torch.from_numpy(lam).cuda()
    grad = torch.zeros_like(lin)
    torch.cuda.synchronize()
    m.sft_adjoint(g2.ctx, lin.data_ptr(), nst, grad.data_ptr())
    torch.cuda.synchronize()
    tan = dout.cpu().numpy().astype(np.float64)
    gr = grad.cpu().numpy().astype(np.float64)
    for r in range(w.replicas):
        lhs = float(np.sum(lam[r].astype(np.float64) * tan[r]))
        rhs = float(np.sum(gr[r] * d0[r].astype(np.float64)))
        assert abs(lhs - rhs) <= 2e-5 * (abs(lhs) + abs(rhs)), (name, lhs, rhs)
    go = o.adjoint(lam.astype(np.float64), nst)
    for r in range(w.replicas):
        assert rel(gr[r], go[r]) <= 1e-5, (name, r, rel(gr[r], go[r]))
    # the primal ends where nsteps of plain stepping end
    g3, _ = make_pair(m, oracle_mod, w, f0)
    g3.step(nst)
    assert g2.step_count == nst
    assert np.array_equal(g2.spectrum(), g3.spectrum())
    for x in (g1, g2, g3):
        x.close()
