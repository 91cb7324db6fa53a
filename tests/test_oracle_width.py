"""Pins of the oracle's width over boxes (Sec. V.B) against numpy: the box
variance averaged over the boxes of a reshaped field, 0 for single-site boxes,
and for the whole lattice the real-space variance, which Parseval ties to the
spectral roughness."""
import numpy as np
import pytest

import sft_inputs as W


def numpy_box_width(f, ell):
    d = f.ndim
    shp = []
    for n in f.shape:
        shp += [n // ell, ell]
    b = f.reshape(shp)
    axes = tuple(range(1, 2 * d, 2))
    return float(np.mean(b.var(axis=axes)))


@pytest.mark.parametrize("w,ells", [
    (W.kpz_1d(64, replicas=2, sigma0=0.7), [1, 2, 8, 64]),
    (W.kpz_2d(n=[16, 16], replicas=2, sigma0=0.7), [1, 4, 16]),
    (W.model_a_128_3d(n=[8, 8, 8], replicas=1, sigma0=0.7), [2, 8]),
])
def test_box_width(oracle_mod, w, ells):
    o = oracle_mod.Oracle(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    f0 = W.initial_fields(w)
    for r in range(w.replicas):
        o.set_field(r, f0[r])
    o.step(3)
    for ell in ells:
        got = o.box_width(ell)
        for r in range(w.replicas):
            f = o.field(r)
            assert abs(got[r] - numpy_box_width(f, ell)) <= 1e-12 * (1 + abs(got[r]))
            if ell == 1:
                assert got[r] == 0.0
            if ell == w.n[0]:
                assert abs(got[r] - f.var()) <= 1e-12 * f.var()
                assert abs(got[r] - o.roughness()[r]) <= 1e-10 * f.var()
