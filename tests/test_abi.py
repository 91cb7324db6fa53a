"""The C-ABI library loads without a GPU and exports every entry point that
include/sft.h declares; configuration validation needs no device."""
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sft_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2511_22510_gb300 as sft
    from paper_2511_22510_gb300 import _build
    _build.build()
    return sft


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sft_create", "sft_step", "sft_observe", "sft_tangent_step", "sft_adjoint", "sft_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.load_library()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(lib.ABI_FUNCTIONS) == _declared()


@pytest.mark.parametrize("bad", [
    dict(d=4), dict(n=[40, 40]), dict(n=[1536, 1536]), dict(replicas=0), dict(h=0.0), dict(h=float("nan")), dict(model=9),
    dict(scheme=5), dict(dealias=3), dict(dealias=-1),
])
def test_invalid_configs_rejected_before_any_device_call(lib, bad):
    kw = dict(d=2, n=[64, 64], dx=[1.0, 1.0], replicas=1, model=0, p=[1, -0.5, 1, 0.5], scheme=1, h=0.01,
              seed=1)
    kw.update(bad)
    cfg = lib.make_config(min(kw["d"], 2), kw["n"], kw["dx"], kw["replicas"], kw["model"], kw["p"],
                          kw["scheme"], kw["h"], kw["seed"], dealias=kw.get("dealias", 1))
    if bad.get("d") == 4:
        cfg.d = 4
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == lib.SFT_EINVAL


def test_unsupported_configs_report_unsupported(lib):
    cfg = lib.make_config(2, [64, 32], [1.0, 1.0], 1, 0, [1, -0.5, 1, 0.5], 1, 0.01, 1)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == lib.SFT_EUNSUPPORTED


def _custom(lib, n=16, **over):
    q = 2 * (n // 2) ** 2 + 1
    tab = dict(nl=lib.SFT_NL_CUBIC, complex_field=0, c=-(0.5 + np.arange(q) * 0.01), D=np.full(q, 0.1),
               s=np.full(q, -1.0))
    tab.update(over)
    return tab


@pytest.mark.parametrize("over", [
    dict(c=None), dict(D=None), dict(D=-np.ones(2 * 8 ** 2 + 1)), dict(nl=7),
    dict(c=-(0.5 + 0.1j) * np.ones(2 * 8 ** 2 + 1)),          # complex c on a real field
    dict(s=(-1.0 + 0.5j) * np.ones(2 * 8 ** 2 + 1)),          # complex s on a real field
    dict(nl=3),                                               # |A|^2 A on a real field
    dict(complex_field=1, nl=1),                              # psi^3 on a complex field
    dict(c=np.full(2 * 8 ** 2 + 1, np.nan)),
])
def test_invalid_custom_models_rejected_before_any_device_call(lib, over):
    tab = _custom(lib, **over)
    if tab["c"] is None or tab["D"] is None:
        cfg = lib.make_config(2, [16, 16], [1.0, 1.0], 1, lib.SFT_CUSTOM, [], 1, 0.01, 1,
                              custom=dict(tab, c=np.zeros(1) if tab["c"] is None else tab["c"],
                                          D=np.zeros(1) if tab["D"] is None else tab["D"]))
        if tab["c"] is None:
            cfg.c_re = None
        else:
            cfg.noise_D = None
    else:
        cfg = lib.make_config(2, [16, 16], [1.0, 1.0], 1, lib.SFT_CUSTOM, [], 1, 0.01, 1, custom=tab)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == lib.SFT_EINVAL


def test_r_in_F_with_setd2_unsupported(lib):
    cfg = lib.make_config(2, [64, 64], [1.0, 1.0], 1, 0, [1, -0.5, 1, 0.5, 1.0], 2, 0.01, 1)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == lib.SFT_EUNSUPPORTED


@pytest.mark.parametrize("d,n,model,space,status", [
    (2, 16, 0, 2, "SFT_EINVAL"),          # no such noise space
    (1, 32768, 0, 1, "SFT_EUNSUPPORTED"), # real-space noise: 2-D real fields and 1-D lines up to 16384 points
    (1, 128, 3, 1, "SFT_EUNSUPPORTED"),   # complex line (CGL)
    (2, 16, 3, 1, "SFT_EUNSUPPORTED"),    # complex field (CGL)
])
def test_real_space_noise_limits(lib, d, n, model, space, status):
    n = [n] * d
    cfg = lib.make_config(d, n, [1.0] * d, 1, model, [1, -0.5, 1, 0.5], 1, 0.01, 1, noise_space=space)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == getattr(lib, status)


@pytest.mark.parametrize("d,n,model,space", [
    (1, 32768, 0, 0), (3, 128, 0, 0),  # phase shifts: 2-D real fields, 1-D lines up to 16384 points, 3-D up to 64^3
    (1, 128, 3, 0),                   # complex lines (CGL; 2-D complex fields are built)
    (2, 16, 0, 1), (1, 256, 0, 1),    # with real-space noise
])
def test_phase_shift_dealiasing_limits(lib, d, n, model, space):
    cfg = lib.make_config(d, [n] * d, [1.0] * d, 1, model, [1, -0.5, 1, 0.5], 1, 0.01, 1, dealias=2,
                          noise_space=space)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == lib.SFT_EUNSUPPORTED


@pytest.mark.parametrize("d,model,extra", [
    (3, 0, {}),                               # p x 2^k lattices are built for 1-D and 2-D real fields
    (2, 3, {}),                               # complex field (CGL)
    (2, 0, dict(dealias=2)), (2, 0, dict(noise_space=1)),
])
def test_3x2k_lattice_limits(lib, d, model, extra):
    cfg = lib.make_config(d, [48] * d, [1.0] * d, 1, model, [1, -0.5, 1, 0.5], 1, 0.01, 1, **extra)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create(cfg)
    assert ei.value.status == lib.SFT_EUNSUPPORTED


@pytest.mark.parametrize("case,status", [
    (dict(n=[1024, 1024]), "SFT_EINVAL"),                   # above the 512-point scratch limit
    (dict(n=[512, 512], replicas=2), "SFT_EINVAL"),         # 2 x 257 x 512 modes > 262144
    (dict(scheme=2, fprev=None), "SFT_EINVAL"),             # SETD2 without its history buffer
    (dict(h=float("inf")), "SFT_EINVAL"),                   # the checks of sft_create
    (dict(replica0=-1), "SFT_EINVAL"),
    (dict(model=3, p=[2.0, -0.5, 1e-4]), "SFT_EUNSUPPORTED"),  # complex field
    (dict(d=1, n=[64]), "SFT_EUNSUPPORTED"),
    (dict(dealias=2), "SFT_EUNSUPPORTED"),
    (dict(nsteps=-1), "SFT_EINVAL"),
    (dict(step0=(1 << 32) - 5, nsteps=10), "SFT_EINVAL"),  # past the 32-bit noise step counter
], ids=["n1024", "modes", "setd2_nohist", "h_inf", "replica0", "cgl", "1d", "phase_shift", "nsteps", "counter"])
def test_noalloc_refusals_need_no_device(lib, case, status):
    """The allocation-free entry point refuses these before it touches the device:
    the device pointers given here are never dereferenced."""
    kw = dict(d=2, n=[64, 64], replicas=1, model=1, p=[1.0, -1.0, 1.0, 0.1], scheme=1, h=0.05, dealias=1,
              replica0=0, fprev=4096, step0=0, nsteps=3)
    kw.update(case)
    d = kw["d"]
    cfg = lib.make_config(d, kw["n"], [1.0] * d, kw["replicas"], kw["model"], kw["p"], kw["scheme"], kw["h"], 7,
                          kw["dealias"], replica0=kw["replica0"])
    with pytest.raises(lib.SftError) as ei:
        lib.sft_step2d_noalloc(cfg, 4096, kw["fprev"], 0, kw["step0"], kw["nsteps"])
    assert ei.value.status == getattr(lib, status)


@pytest.mark.parametrize("case", [
    dict(kind=7), dict(scheme=9), dict(h=0.0), dict(h=float("inf")), dict(substeps=0), dict(nsteps=-1),
    dict(npaths=-1), dict(step0=-1), dict(kind=0, p=[0.0, 1.0, 1.0]), dict(kind=0, p=[1.0, -1.0, 1.0]),
    dict(step0=1 << 31, nsteps=1 << 31, substeps=2), dict(u=None),
], ids=["kind", "scheme", "h0", "hinf", "substeps", "nsteps", "npaths", "step0", "sao_a0", "sao_b", "counter",
        "no_u"])
def test_sde0d_refusals_need_no_device(lib, case):
    """The 0-d SDE ensemble entry point refuses bad arguments before any launch
    (the device pointers given here are never dereferenced)."""
    kw = dict(kind=1, p=[2.0, 1.0, 1.0], scheme=3, h=2.0 ** -8, nsteps=4, npaths=16, substeps=1, step0=0, u=4096)
    kw.update(case)
    with pytest.raises(lib.SftError) as ei:
        lib.sft_sde0d(kw["kind"], kw["p"], kw["scheme"], kw["h"], kw["nsteps"], kw["u"], kw["npaths"], seed=1,
                      substeps=kw["substeps"], step0=kw["step0"])
    assert ei.value.status == lib.SFT_EINVAL


def test_sde0d_empty_work_is_a_no_op(lib):
    # no paths or no steps: nothing to launch, nothing dereferenced
    lib.sft_sde0d(1, [2.0, 1.0, 1.0], 3, 0.01, 5, None, 0, seed=1)
    lib.sft_sde0d(1, [2.0, 1.0, 1.0], 3, 0.01, 0, 4096, 8, seed=1)


def test_batch_members_must_share_model_and_scheme(lib):
    a = lib.make_config(1, [1024], [1.0], 2, 2, [1.0, 2.0, 0.5], 1, 0.01, 3)
    b = lib.make_config(1, [2048], [1.0], 2, 2, [1.0, 2.0, 0.5], 2, 0.01, 3)  # another scheme
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create_batch([a, b])
    assert ei.value.status == lib.SFT_EUNSUPPORTED
    bad = lib.make_config(1, [1000], [1.0], 2, 2, [1.0, 2.0, 0.5], 1, 0.01, 3)  # not a built lattice size
    with pytest.raises(lib.SftError) as ei:
        lib.sft_create_batch([a, bad])
    assert ei.value.status == lib.SFT_EINVAL
