"""Precision of the FP32 path over a 100-step horizon (the CGL workload's
parameters, SETD2, h = 0.05) against the FP64 oracle from the same FP32 initial
field: the relative L2 error of the field after 10, 50 and 100 steps, next to
the intrinsic sensitivity floor of the dynamics (oracle twin runs one FP32 ulp
apart, 5.5e-7 at 128^2)."""
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


@pytest.mark.parametrize("n", [256, 512])
def test_cgl_fp32_error_over_100_steps(sft, oracle_mod, n):
    w = W.cgl_2048(n=[n, n], replicas=1)
    f0 = W.initial_fields(w).astype(np.complex64)
    g = sft.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    g.set_field(f0)
    o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    o.set_field(0, f0[0].astype(np.complex128))
    errs = {}
    done = 0
    for k in (10, 50, 100):
        g.step(k - done)
        o.step(k - done)
        done = k
        ref = o.field(0)
        errs[k] = float(np.linalg.norm(g.field()[0] - ref) / np.linalg.norm(ref))
    g.close()
    print("CGL %d^2 FP32 vs FP64 rel L2:" % n, errs)
    assert errs[100] <= 1e-5, errs
    assert errs[10] <= errs[100] * 10


def test_split_bf16x3_tensor_core_study(sft, oracle_mod):
    """The split-BF16x3 tensor-core transforms (sft_config.precision = 1) against
    the FP32 path and the FP64 oracle over the 100-step horizon, CGL 1024^2
    (the workload's parameters and SETD2).  The study reports both errors; the
    FP32 path meets the 1e-5 bound; the tensor-core path stays an option that
    is kept off by default unless it meets the bound as well.  Its first step
    agrees with the FP32 path to the bf16x3 rounding level, which checks the
    transform itself."""
    w = W.cgl_2048(n=[1024, 1024], replicas=1)
    f0 = W.initial_fields(w).astype(np.complex64)
    runs = {}
    for prec in (0, 1):
        g = sft.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, precision=prec)
        g.set_field(f0)
        g.step(1)
        one = g.field()[0]
        g.step(99)
        runs[prec] = (one, g.field()[0])
        g.close()
    d1 = float(np.linalg.norm(runs[1][0] - runs[0][0]) / np.linalg.norm(runs[0][0]))
    assert d1 <= 1e-4, d1
    o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    o.set_field(0, f0[0].astype(np.complex128))
    o.step(100)
    ref = o.field(0)
    e32 = float(np.linalg.norm(runs[0][1] - ref) / np.linalg.norm(ref))
    etc = float(np.linalg.norm(runs[1][1] - ref) / np.linalg.norm(ref))
    print("CGL 1024^2 after 100 steps, rel L2 vs FP64: FP32 %.3e, split-BF16x3 %.3e; one step apart %.3e"
          % (e32, etc, d1))
    assert e32 <= 1e-5, e32
    assert etc <= 1e-2, etc
