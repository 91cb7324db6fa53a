"""Batched execution: a batch of uneven lattices (1-D KPZ members of several
lengths in one persistent launch, a 2-D member and a 32768-point member on the
forked branch of the same graph) must evolve every member as a stand-alone
context of the same configuration does (same arithmetic compiled into another
kernel: equal up to floating-point contraction, relative 1e-6), and match the
oracle."""
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


MEMBERS = [W.kpz_1d(1024, replicas=5), W.kpz_1d(2048, replicas=3), W.kpz_1d(16384, replicas=2),
           W.kpz_1d(4096, replicas=17), W.kpz_2d(n=[64, 64], replicas=2), W.kpz_1d(32768, replicas=1),
           W.kpz_1d(65536, replicas=2)]


def cfg_of(sft, w, replica0=0):
    return sft.make_config(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, w.dealias,
                           replica0=replica0)


def start_fields(w, k):
    return (0.3 * np.random.default_rng(100 + k).standard_normal((w.replicas,) + w.shape)).astype(np.float32)


@pytest.mark.parametrize("plain", [False, True], ids=["graph", "plain"])
def test_batch_matches_standalone_members(sft, plain):
    batch = sft.Batch([cfg_of(sft, w) for w in MEMBERS])
    singles = []
    off = 0
    for k, w in enumerate(MEMBERS):
        f = start_fields(w, k)
        for r in range(w.replicas):
            batch.set_field(off + r, f[r])
        g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed)
        g.set_field(f)
        singles.append((g, off))
        off += w.replicas
    nst = 37
    if plain:
        batch.step_plain(nst)
    else:
        batch.step(nst)
    for (g, o), w in zip(singles, MEMBERS):
        g.step(nst)
        ref = g.field()
        for r in range(w.replicas):
            got = batch.field(o + r, w.shape)
            err = float(np.linalg.norm(got - ref[r]) / np.linalg.norm(ref[r]))
            assert err <= 1e-6, (w.name, r, err)
        g.close()
    rough = batch.roughness()
    assert rough.shape == (batch.R,) and np.all(rough > 0)
    batch.close()


def test_batch_member_against_oracle(sft, oracle_mod):
    members = [W.kpz_1d(512, replicas=3), W.kpz_1d(2048, replicas=2)]
    batch = sft.Batch([cfg_of(sft, w) for w in members])
    f = [start_fields(w, k) for k, w in enumerate(members)]
    batch.set_field(-1, np.concatenate([x.reshape(-1) for x in f]))
    batch.step(40)
    off = 0
    for w, f0 in zip(members, f):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed)
        for r in range(w.replicas):
            o.set_field(r, f0[r].astype(np.float64))
        o.step(40)
        for r in range(w.replicas):
            got = batch.field(off + r, w.shape)
            ref = o.field(r)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        off += w.replicas
    batch.close()


# members with a step variant or p x 2^k points run their own kernels on graph branches of the batch step
VARIANT_MEMBERS = [(W.kpz_1d(1024, replicas=3), dict(noise_space=1)),
                   (W.kpz_1d(2048, replicas=2, sigma0=0.5), dict(dealias=2)),
                   (W.kpz_1d(768, replicas=2), {}),
                   (W.kpz_1d(4096, replicas=5), {}),
                   (W.kpz_2d(n=[64, 64], replicas=2), dict(noise_space=1))]


def test_batch_with_variant_members(sft, oracle_mod):
    cfgs = []
    for w, kw in VARIANT_MEMBERS:
        kw = dict(kw)
        dealias = kw.pop("dealias", w.dealias)
        cfgs.append(sft.make_config(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias, **kw))
    batch = sft.Batch(cfgs)
    fields = [start_fields(w, k) for k, (w, _) in enumerate(VARIANT_MEMBERS)]
    off = 0
    for (w, _), f in zip(VARIANT_MEMBERS, fields):
        for r in range(w.replicas):
            batch.set_field(off + r, f[r])
        off += w.replicas
    nst = 29
    batch.step(nst)
    off = 0
    for k, ((w, kw), f) in enumerate(zip(VARIANT_MEMBERS, fields)):
        kw = dict(kw)
        dealias = kw.pop("dealias", w.dealias)
        g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=dealias, **kw)
        g.set_field(f)
        g.step(nst)
        ref = g.field()
        g.close()
        for r in range(w.replicas):
            got = batch.field(off + r, w.shape)
            assert np.linalg.norm(got - ref[r]) / np.linalg.norm(ref[r]) <= 1e-6, (k, r)
        if k == 0:
            # the real-space-noise member against the oracle
            o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=dealias,
                                  **kw)
            for r in range(w.replicas):
                o.set_field(r, f[r].astype(np.float64))
            o.step(nst)
            for r in range(w.replicas):
                got = batch.field(off + r, w.shape)
                assert np.linalg.norm(got - o.field(r)) / np.linalg.norm(o.field(r)) <= 1e-5, (k, r)
        off += w.replicas
    batch.close()
