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
    dt, dt64 = (np.complex64, np.complex128) if w.complex_field else (np.float32, np.float64)
    g.set_field(f0.astype(dt))
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(w.replicas):
        o.set_field(r, f0[r].astype(dt).astype(dt64))
    return g, o


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    ("model_a_64", W.model_a_64(n=[64, 64], replicas=2, sigma0=0.3, h=0.02)),
    ("model_b_32_em", W.model_b_1024(n=[32, 32], replicas=2, sigma0=0.3, scheme=0, h=0.02)),
    ("model_a_1d_256", W.model_a_64(d=1, n=[256], dx=[1.0], replicas=3, sigma0=0.3, h=0.02)),
    ("model_a_3d_16", W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3, h=0.02)),
    ("model_b_3d_16_em", W.model_a_128_3d(n=[16, 16, 16], model=1, p=[1.0, -0.5, 1.0, 0.2], scheme=0, h=0.02,
                                          sigma0=0.3)),
]


# SETD2 (Eq. SETD2): the tangent carries its own history dF_prev, zero at the seed; KPZ (Sec. V.B):
# dq = 2 grad h . grad dh; CGL (Sec. V.C): dq = 2 |A|^2 dA + A^2 conj(dA), complex seeds
TAN_CASES = CASES + [
    ("model_a_64_setd2", W.model_a_64(n=[64, 64], replicas=2, sigma0=0.3, h=0.02, scheme=2)),
    ("model_b_1d_128_setd2", W.model_b_1024(d=1, n=[128], dx=[1.0], replicas=2, sigma0=0.3, h=0.02, scheme=2)),
    ("model_a_3d_16_setd2", W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3, h=0.02, scheme=2)),
    ("kpz_1d_256_setd1", W.kpz_1d(256, replicas=3, sigma0=0.5)),
    ("kpz_1d_512_setd2", W.kpz_1d(512, replicas=2, sigma0=0.5, scheme=2)),
    ("cgl_1d_128_setd2", W.cgl_2048(d=1, n=[128], dx=[0.5], replicas=2, p=[2.0, -0.5, 1e-3])),
    ("cgl_1d_256_setd1", W.cgl_2048(d=1, n=[256], dx=[0.5], replicas=2, scheme=1, p=[0.5, 0.3, 1e-2])),
    ("kpz_2d_32_setd1", W.kpz_2d(n=[32, 32], replicas=2, sigma0=0.5)),
    ("kpz_2d_64_setd2", W.kpz_2d(n=[64, 64], replicas=2, sigma0=0.5, scheme=2)),
    ("cgl_2d_32_setd2", W.cgl_2048(n=[32, 32], replicas=2, p=[2.0, -0.5, 1e-3])),
    ("cgl_2d_64_setd1", W.cgl_2048(n=[64, 64], replicas=2, scheme=1, p=[0.5, 0.3, 1e-2])),
]


@pytest.mark.parametrize("name,w", TAN_CASES, ids=[c[0] for c in TAN_CASES])
def test_tangent_parity(env, oracle_mod, name, w):
    m, torch = env
    f0 = W.initial_fields(w)
    d0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=9)
    g, o = make_pair(m, oracle_mod, w, f0)
    nst = 20
    dev_in = torch.from_numpy(d0.astype(np.complex64 if w.complex_field else np.float32)).cuda()
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


ADJ_CASES = CASES + [
    ("kpz_1d_256_setd1", W.kpz_1d(256, replicas=3, sigma0=0.5)),
    ("model_a_64_setd2", W.model_a_64(n=[64, 64], replicas=2, sigma0=0.3, h=0.02, scheme=2)),
    ("model_b_1d_128_setd2", W.model_b_1024(d=1, n=[128], dx=[1.0], replicas=2, sigma0=0.3, h=0.02, scheme=2)),
    ("model_a_3d_16_setd2", W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3, h=0.02, scheme=2)),
    ("kpz_1d_512_setd2", W.kpz_1d(512, replicas=2, sigma0=0.5, scheme=2)),
    ("kpz_2d_32_setd1", W.kpz_2d(n=[32, 32], replicas=2, sigma0=0.5)),
    ("kpz_2d_64_setd2", W.kpz_2d(n=[64, 64], replicas=2, sigma0=0.5, scheme=2)),
    ("kpz_2d_128_em_nodeal", W.kpz_2d(n=[128, 128], replicas=2, sigma0=0.5, scheme=0, dealias=0)),
    # CGL (Sec. V.C): the transpose for the real inner product Re sum conj(u) v, complex cotangents
    ("cgl_1d_128_setd2", W.cgl_2048(d=1, n=[128], dx=[0.5], replicas=2, p=[2.0, -0.5, 1e-3])),
    ("cgl_1d_256_setd1", W.cgl_2048(d=1, n=[256], dx=[0.5], replicas=2, scheme=1, p=[0.5, 0.3, 1e-2])),
    ("cgl_2d_32_setd2", W.cgl_2048(n=[32, 32], replicas=2, p=[2.0, -0.5, 1e-3])),
    ("cgl_2d_64_setd1", W.cgl_2048(n=[64, 64], replicas=2, scheme=1, p=[0.5, 0.3, 1e-2])),
    ("cgl_2d_64_em_nodeal", W.cgl_2048(n=[64, 64], replicas=2, scheme=0, dealias=0, p=[0.5, 0.3, 1e-2])),
]


@pytest.mark.parametrize("name,w", ADJ_CASES, ids=[c[0] for c in ADJ_CASES])
def test_adjoint_dot_product_and_parity(env, oracle_mod, name, w):
    """<lambda, T delta> = <A lambda, delta> on the GPU, and the GPU gradient
    against the oracle's; checkpoint segments of 7 steps over a 20-step horizon
    force the recompute of the primal from checkpoints."""
    m, torch = env
    dt = np.complex64 if w.complex_field else np.float32
    f0 = W.initial_fields(w)
    d0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=3).astype(dt)
    lam = W.initial_fields(w.with_(sigma0=1.0), seed_offset=4).astype(dt)
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
    dt64 = np.complex128 if w.complex_field else np.float64
    tan = dout.cpu().numpy().astype(dt64)
    gr = grad.cpu().numpy().astype(dt64)
    for r in range(w.replicas):
        # the real inner product (complex fields: Re sum conj(u) v)
        lhs = float(np.vdot(lam[r].astype(dt64), tan[r]).real)
        rhs = float(np.vdot(gr[r], d0[r].astype(dt64)).real)
        assert abs(lhs - rhs) <= 2e-5 * (abs(lhs) + abs(rhs)), (name, lhs, rhs)
    go = o.adjoint(lam.astype(dt64), nst)
    for r in range(w.replicas):
        assert rel(gr[r], go[r]) <= 1e-5, (name, r, rel(gr[r], go[r]))
    # the primal ends where nsteps of plain stepping end
    g3, _ = make_pair(m, oracle_mod, w, f0)
    g3.step(nst)
    assert g2.step_count == nst
    assert np.array_equal(g2.spectrum(), g3.spectrum())
    for x in (g1, g2, g3):
        x.close()


def test_fluctuation_dissipation_model_a_3d(env):
    """Equilibrium Model A (Gamma = 1, D = T): the response to an impulse in the
    mode k0 obeys R(k0, tau) = -(1/T) dC(k0, tau)/dtau (the time-domain form of
    the FDT of Sec. V.A), checked in integrated form
    int_0^tau R = (C(k0, 0) - C(k0, tau)) / T over an ensemble of replicas, with
    the tangent on the same noise paths as the correlations.  Tolerance: 4
    standard errors (batch means over replica groups) plus the O(h) bias."""
    m, torch = env
    T = 1.0
    w = W.model_a_128_3d(n=[16, 16, 16], replicas=512, p=[1.0, 0.5, 1.0, T], h=0.01)
    g = m.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed)
    g.init_random(0.5)
    g.step(1500)
    ns = g.nshells()
    g.observe(m.SFT_OBS_MARK)
    N = 16
    x = np.arange(N)
    seed = np.cos(2 * np.pi * x / N)[None, None, None, :] * np.ones((w.replicas, N, N, N))
    din = torch.from_numpy(seed.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    taus, resp, corr = [0.0], [1.0], []
    c0 = m.sft_observe(g.ctx, m.SFT_OBS_SK_REPLICAS, w.replicas * ns).reshape(w.replicas, ns)[:, 1]
    corr.append(c0)
    chunk = 5
    first = True
    for i in range(40):
        m.sft_tangent_step(g.ctx, din.data_ptr() if first else None, chunk, None)
        first = False
        taus.append((i + 1) * chunk * w.h)
        resp.append(g.observe(m.SFT_OBS_RESPONSE)[1])
        # two-time correlation per replica in shell 1 (|a| = 1: exactly the modes +-k0 on each axis)
        ck = m.sft_observe(g.ctx, m.SFT_OBS_CKT, 2 * ns)
        corr.append(ck[1])
    taus = np.array(taus)
    resp = np.array(resp)
    cmean0 = float(np.mean(corr[0]))
    ctau = np.array([cmean0] + [float(c) for c in corr[1:]])
    integ = np.concatenate([[0.0], np.cumsum(0.5 * (resp[1:] + resp[:-1]) * np.diff(taus))])
    lhs = integ
    rhs = (ctau[0] - ctau) / T
    # statistical error of C(0) - C(tau): scale from the spread of C(0) over replica groups
    groups = corr[0].reshape(16, -1).mean(axis=1)
    sem = float(np.std(groups) / np.sqrt(16))
    for j in (10, 20, 40):
        assert abs(lhs[j] - rhs[j]) <= 4 * sem + 0.03 * abs(rhs[j]) + 0.02 * taus[j], (taus[j], lhs[j], rhs[j], sem)
    g.close()


AUTOGRAD_CASES = [
    ("model_a_32", W.model_a_64(n=[32, 32], replicas=2, sigma0=0.3, h=0.02)),
    ("model_b_3d_16_em", W.model_a_128_3d(n=[16, 16, 16], model=1, p=[1.0, -0.5, 1.0, 0.2], scheme=0, h=0.02,
                                          sigma0=0.3)),
    ("kpz_2d_32_setd2", W.kpz_2d(n=[32, 32], replicas=2, sigma0=0.5, scheme=2)),
    ("cgl_2d_32_setd2", W.cgl_2048(n=[32, 32], replicas=2, p=[2.0, -0.5, 1e-3])),
]


@pytest.mark.parametrize("name,w", AUTOGRAD_CASES, ids=[c[0] for c in AUTOGRAD_CASES])
def test_autograd_function(env, oracle_mod, name, w):
    """torch.autograd over the tangent/adjoint pair: forward = J v (the oracle's
    tangent), backward = J^T g (the oracle's adjoint); <J v, g> = <v, J^T g>;
    the backward pass leaves the stepper where the forward left it."""
    m, torch = env
    from paper_2511_22510_gb300.response import propagate
    dt, dt64 = (np.complex64, np.complex128) if w.complex_field else (np.float32, np.float64)
    f0 = W.initial_fields(w)
    v0 = W.initial_fields(w.with_(sigma0=1.0), seed_offset=5).astype(dt)
    gw = W.initial_fields(w.with_(sigma0=1.0), seed_offset=6).astype(dt)
    nst = 15
    g, o = make_pair(m, oracle_mod, w, f0)
    m.sft_set_checkpoint_interval(g.ctx, 6)
    v = torch.from_numpy(v0).cuda().requires_grad_(True)
    out = propagate(v, g, nst)
    after_forward = g.spectrum()
    gt = torch.from_numpy(gw).cuda()
    # a real loss: Re sum conj(g) J v (complex fields), sum g J v (real fields)
    loss = (out * gt.conj()).sum()
    (loss.real if w.complex_field else loss).backward()
    assert np.array_equal(g.spectrum(), after_forward)
    assert g.step_count == nst
    jv = out.detach().cpu().numpy().astype(dt64)
    jtg = v.grad.cpu().numpy().astype(dt64)
    tan_o = o.tangent_step(v0.astype(dt64), nst)
    o2 = make_pair(m, oracle_mod, w, f0)[1]
    adj_o = o2.adjoint(gw.astype(dt64), nst)
    for r in range(w.replicas):
        assert rel(jv[r], tan_o[r]) <= 1e-5, (name, r)
        assert rel(jtg[r], adj_o[r]) <= 1e-5, (name, r)
        lhs = float(np.vdot(gw[r].astype(dt64), jv[r]).real)
        rhs = float(np.vdot(jtg[r], v0[r].astype(dt64)).real)
        assert abs(lhs - rhs) <= 2e-5 * (abs(lhs) + abs(rhs)), (name, lhs, rhs)
    # linear in v, same noise path: a second propagation from the same start doubles with 2 v
    g2, _ = make_pair(m, oracle_mod, w, f0)
    out2 = propagate(2.0 * v.detach(), g2, nst)
    assert rel(out2.cpu().numpy().astype(dt64), 2.0 * jv) <= 1e-6
    for x in (g, g2):
        x.close()


def test_autograd_rejects_host_tensors(env):
    m, torch = env
    from paper_2511_22510_gb300.response import propagate
    w = W.model_a_64(n=[16, 16], replicas=1)
    g = m.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed)
    with pytest.raises(ValueError):
        propagate(torch.zeros((1, 16, 16)), g, 1)
    with pytest.raises(ValueError):
        propagate(torch.zeros((2, 16, 16), device="cuda"), g, 1)
    g.close()
