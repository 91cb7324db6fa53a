"""The complex 2-D step (CGL, Sec. V.C) on columns and rows of 1024 and 2048
points, whose passes hold each line in one or two warps (warp-resident
1024-point transforms; the 2048-point lines split across two warps), against
the FP64 oracle from the same FP32 initial fields: relative L2 <= 1e-5 per
replica and every mode within 1e-4 of the RMS mode amplitude, for SETD-EM,
SETD1 and SETD2, with and without 2/3 truncation (the warp row pass runs under
truncation, the general row pass without).  The oracle runs one context per
replica in threads (its C library releases the GIL)."""
import threading

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


CASES = [
    ("cgl_1024_setd2_R2", W.cgl_2048(n=[1024, 1024], replicas=2), 20),
    ("cgl_1024_setd1_nodeal", W.cgl_2048(n=[1024, 1024], replicas=1, scheme=1, dealias=0), 20),
    ("cgl_2048_setd2", W.cgl_2048(replicas=1), 8),
    ("cgl_2048_em_nodeal", W.cgl_2048(replicas=1, scheme=0, dealias=0, p=[0.5, 0.3, 1e-2]), 6),
]


@pytest.mark.parametrize("name,w,nsteps", CASES, ids=[c[0] for c in CASES])
def test_complex_warp_columns_against_oracle(sft, oracle_mod, name, w, nsteps):
    R = w.replicas
    f0 = W.initial_fields(w).astype(np.complex64)
    g = sft.Stepper(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    g.set_field(f0)
    g.step(nsteps)
    got = g.field().astype(np.complex128)
    g.close()
    want = [None] * R

    def one(r):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                              replica0=r)
        o.set_field(0, f0[r].astype(np.complex128))
        o.step(nsteps)
        want[r] = o.field(0)

    th = [threading.Thread(target=one, args=(r,)) for r in range(R)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for r in range(R):
        rel = np.linalg.norm(got[r] - want[r]) / np.linalg.norm(want[r])
        a, b = np.fft.fft2(got[r]), np.fft.fft2(want[r])  # every mode, not just the norm
        worst = np.abs(a - b).max() / np.sqrt(np.mean(np.abs(b) ** 2))
        assert rel <= 1e-5, (name, r, rel)
        assert worst <= 1e-4, (name, r, worst)


def test_complex_warp_columns_graph_and_plain_bit_identical(sft):
    w = W.cgl_2048(n=[1024, 1024], replicas=2)
    mk = lambda: sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed)
    a, b = mk(), mk()
    f = W.initial_fields(w).astype(np.complex64)
    a.set_field(f)
    b.set_field(f)
    a.step(17)
    b.step_plain(17)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    for s in (a, b):
        s.close()
