"""Intrinsic sensitivity floor of the workloads: two oracle runs whose initial
fields differ by one FP32 ulp per site drift apart by the dynamics alone.  The
relative L2 distance after 100 steps is the floor below which no FP32
implementation can be compared pointwise with the FP64 oracle; the parity
target (1e-5 after 100 steps) is meaningful where the floor is well below it.
Model A (64^2, the SETD1 workload), Model B (the critical quench of the
headline, at 128^2) and the CGL workload's parameters (at 128^2, SETD2)."""
import numpy as np
import pytest

import sft_inputs as W


def floor_after(oracle_mod, w, nsteps):
    f0 = W.initial_fields(w, replicas=1)[0]
    if w.complex_field:
        a = f0.astype(np.complex64)
        b = (np.nextafter(a.real, np.float32(np.inf)) + 1j * a.imag).astype(np.complex64)
        cast = np.complex128
    else:
        a = f0.astype(np.float32)
        b = np.nextafter(a, np.float32(np.inf))
        cast = np.float64
    out = []
    for f in (a, b):
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
        o.set_field(0, f.astype(cast))
        o.step(nsteps)
        out.append(o.field(0))
    return float(np.linalg.norm(out[0] - out[1]) / np.linalg.norm(out[1]))


@pytest.mark.parametrize("name,w,bound", [
    ("model_a_64_setd1", W.model_a_64(), 1e-6),
    ("model_b_128_setd1", W.model_b_1024(n=[128, 128]), 1e-6),
    ("cgl_128_setd2", W.cgl_2048(n=[128, 128]), 1e-6),
])
def test_sensitivity_floor_below_the_parity_target(oracle_mod, name, w, bound):
    d = floor_after(oracle_mod, w, 100)
    assert 0.0 < d < bound, (name, d)
