"""The multi-rank path on the CPU (gloo, world size 2).

With one process per GPU, bench.py shards an ensemble of replicas over the
ranks: rank r advances R replicas whose Philox replica counters start at
r R (so no two ranks draw the same noise) and the job's time is the maximum
over the ranks.  The path has no data-path collective.  Here two gloo ranks
step their shares with the oracle; together they must reproduce a single run
of the whole ensemble bit for bit, and the time reduction must return the
slowest rank's time.
"""
import socket

import numpy as np
import pytest

import sft_inputs as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _whole_ensemble(oracle_mod, w, f0, nsteps):
    ref = oracle_mod.Oracle(w.d, w.n, w.dx, len(f0), w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    for r in range(len(f0)):
        ref.set_field(r, f0[r])
    ref.step(nsteps)
    return np.stack([ref.field(r) for r in range(len(f0))])


def test_replica_offset_splits_an_ensemble(oracle_mod):
    """Two contexts of 2 replicas at replica offsets 0 and 2 = one context of 4."""
    w = W.model_b_1024(n=[16, 16], sigma0=0.3)
    f0 = W.initial_fields(w, replicas=4)
    want = _whole_ensemble(oracle_mod, w, f0, 6)
    got = []
    for r0 in (0, 2):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, replica0=r0)
        for r in range(2):
            o.set_field(r, f0[r0 + r])
        o.step(6)
        got += [o.field(r) for r in range(2)]
    assert np.array_equal(np.stack(got), want)
    # and the offset does change the noise: replica 2 of the whole run is not replica 0 of a fresh one
    o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed)
    o.set_field(0, f0[2])
    o.step(6)
    assert not np.array_equal(o.field(0), want[2])


@pytest.mark.parametrize("name,w,extra", [
    ("real_space_noise", W.model_b_1024(n=[16, 16], sigma0=0.3), dict(noise_space=1)),
    ("phase_shift", W.model_a_64(n=[16, 16], sigma0=0.3, dealias=2), {}),
    ("lattice_24", W.model_a_64(n=[24, 24], sigma0=0.3), {}),
], ids=["real_space_noise", "phase_shift", "lattice_24"])
def test_replica_offset_splits_an_ensemble_for_the_variants(oracle_mod, name, w, extra):
    """The variants shard the same way: their noise is keyed by the global replica index too."""
    f0 = W.initial_fields(w, replicas=4)
    ref = oracle_mod.Oracle(w.d, w.n, w.dx, 4, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, **extra)
    for r in range(4):
        ref.set_field(r, f0[r])
    ref.step(6)
    want = np.stack([ref.field(r) for r in range(4)])
    got = []
    for r0 in (0, 2):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                              replica0=r0, **extra)
        for r in range(2):
            o.set_field(r, f0[r0 + r])
        o.step(6)
        got += [o.field(r) for r in range(2)]
    assert np.array_equal(np.stack(got), want)


def test_two_gloo_ranks_reproduce_one_ensemble(oracle_mod, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import multirank_worker

    ws, R, nsteps = 2, 2, 5
    out = str(tmp_path / "rank0.npz")
    mp.start_processes(multirank_worker.run_rank, args=(ws, _free_port(), R, nsteps, out), nprocs=ws,
                       start_method="spawn", join=True)
    d = np.load(out)
    assert float(d["tmax"]) == 11.0  # the slowest rank's time
    w = W.model_a_64(n=[16, 16], sigma0=0.3)
    f0 = W.initial_fields(w, replicas=ws * R)
    assert np.array_equal(d["fields"], _whole_ensemble(oracle_mod, w, f0, nsteps))
