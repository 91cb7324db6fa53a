"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances: noise normals bit-identical; fields relative L2 <= 1e-5 after the
stated number of steps (the FP32 target of the method's accuracy gate);
transforms and observables at FP32 rounding (<= 2e-6 relative); the Model B
zero mode and graph-vs-plain / checkpoint resumes bit-identical.
"""
import numpy as np
import pytest

import sft_inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_22510_gb300 as m
    m.load_library()
    return m


def gpu_stepper(sft, w, replicas=None):
    return sft.Stepper(w.d, w.n, w.dx, replicas or w.replicas, w.model, w.p, w.scheme, w.h, w.seed,
                       dealias=w.dealias)


def oracle_for(oracle_mod, w, replicas=None):
    return oracle_mod.Oracle(w.d, w.n, w.dx, replicas or w.replicas, w.model, w.p, w.scheme, w.h, w.seed,
                             dealias=w.dealias)


def half_xmajor(full, complex_field):
    """Oracle full spectrum (shape (..., ny, nx)) -> the library's stored layout
    (HX, [nz,] [ny]) with x-major ordering."""
    nx = full.shape[-1]
    hx = nx if complex_field else nx // 2 + 1
    h = full[..., :hx]
    return np.moveaxis(h, -1, 0)


def start_pair(sft, oracle_mod, w, replicas=None, fields=None):
    R = replicas or w.replicas
    f0 = W.initial_fields(w, replicas=R) if fields is None else fields
    dt = np.complex64 if w.complex_field else np.float32
    f32 = f0.astype(dt)
    g = gpu_stepper(sft, w, R)
    g.set_field(f32)
    o = oracle_for(oracle_mod, w, R)
    for r in range(R):
        o.set_field(r, f32[r].astype(np.complex128 if w.complex_field else np.float64))
    return g, o


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ noise bits
@pytest.mark.parametrize("w", [
    W.model_a_64(n=[16, 16], replicas=3),
    W.model_b_1024(n=[32, 32], replicas=2),
    W.kpz_1d(64, replicas=2),
    W.cgl_2048(n=[32], d=1, dx=[0.5], replicas=2),
    W.model_a_128_3d(n=[16, 16, 16], replicas=2),
    W.cgl_2048(n=[16, 16], replicas=2),
], ids=["2d16", "2d32", "1d64", "cgl1d32", "3d16", "cgl2d16"])
def test_noise_normals_bit_identical(sft, oracle_mod, w):
    g = gpu_stepper(sft, w)
    o = oracle_for(oracle_mod, w)
    hx = g.hx
    ny = w.n[1] if w.d > 1 else 1
    nz = w.n[2] if w.d > 2 else 1
    nx = w.n[0]
    # self-conjugate stored modes of a real field (App. B): a_x in {0, nx/2}, a_z in {0, nz/2}, a_y in {0, ny/2}
    selfc = np.zeros((hx, nz, ny), dtype=bool)
    if not w.complex_field:
        for ax in (0, nx // 2):
            for az in ({0, nz // 2} if nz > 1 else {0}):
                for ay in ({0, ny // 2} if ny > 1 else {0}):
                    selfc[ax, az, ay] = True
    selfc = selfc.reshape(g.spec_shape[1:])
    r2 = np.float32(float.fromhex('0x1.6a09e6p-1'))
    for step in (0, 7, 123456):
        eg = g.noise(step)
        for r in range(w.replicas):
            eo = half_xmajor(o.noise(r, step), w.complex_field)
            # the oracle widens the float normals: self-conjugate eta = z_a, others (z_a + i z_b)/sqrt2;
            # recover z_a, z_b exactly and apply the library's single-precision scaling.
            za = np.where(selfc, eo.real, eo.real * np.sqrt(2.0)).astype(np.float32)
            zb = (eo.imag * np.sqrt(2.0)).astype(np.float32)
            exp_re = np.where(selfc, za, za * r2).astype(np.float32)
            exp_im = np.where(selfc, np.float32(0), zb * r2).astype(np.float32)
            got = eg[r]
            assert np.array_equal(got.real, exp_re), np.abs(got.real - exp_re).max()
            assert np.array_equal(got.imag, exp_im), np.abs(got.imag - exp_im).max()
    g.close()


# ------------------------------------------------------------------ transforms
@pytest.mark.parametrize("w", [
    W.model_a_64(n=[64, 64], replicas=3), W.model_a_64(n=[256, 256]), W.kpz_1d(1024, replicas=2, sigma0=1.0),
    W.cgl_2048(n=[128], d=1, dx=[0.5], replicas=2), W.model_a_128_3d(n=[32, 32, 32], replicas=2),
    W.model_a_128_3d(n=[128, 128, 128], replicas=1), W.cgl_2048(n=[64, 64], replicas=2),
], ids=["2d64", "2d256", "1d1024", "cgl1d", "3d32", "3d128", "cgl2d64"])
def test_forward_transform_and_roundtrip(sft, oracle_mod, w):
    w = w.with_(sigma0=1.0)
    g, o = start_pair(sft, oracle_mod, w)
    spec = g.spectrum()
    for r in range(w.replicas):
        ref = half_xmajor(o.spectrum(r), w.complex_field)
        assert rel_l2(spec[r], ref) < 2e-6
    back = g.field()
    f0 = W.initial_fields(w).astype(np.complex64 if w.complex_field else np.float32)
    assert rel_l2(back, f0) < 2e-6
    g.close()


# ------------------------------------------------------------------ step parity
CASES = [
    ("cfg1_model_a_64_setd1", W.model_a_64(replicas=2), 100),
    ("model_a_64_em", W.model_a_64(scheme=0, replicas=1), 100),
    ("model_a_64_setd2", W.model_a_64(scheme=2, replicas=1), 100),
    ("model_b_64_setd1", W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3), 100),
    ("model_b_64_em_h01", W.model_b_1024(n=[64, 64], scheme=0, h=0.1, sigma0=0.3), 100),
    ("model_b_64_setd2", W.model_b_1024(n=[64, 64], scheme=2, h=0.025, sigma0=0.3), 100),
    ("model_b_128_setd1_R3", W.model_b_1024(n=[128, 128], replicas=3, sigma0=0.3), 40),
    ("kpz_2d_32", W.kpz_2d(n=[32, 32], replicas=2), 100),
    ("model_a_64_r_in_F", W.model_a_64(p=[1.0, -0.5, 1.0, 0.5, 1.0], replicas=2, sigma0=0.3), 100),
    ("model_b_64_r_in_F_em", W.model_b_1024(n=[64, 64], p=[1.0, -1.0, 1.0, 0.1, 1.0], scheme=0, h=0.02,
                                            sigma0=0.3), 100),
    ("kpz_2d_512", W.kpz_2d(n=[512, 512], replicas=2), 10),
    ("model_a_2048_setd1", W.model_a_64(n=[2048, 2048], replicas=1, sigma0=0.3), 3),
    ("model_b_4096_setd2", W.model_b_1024(n=[4096, 4096], scheme=2, h=0.025, sigma0=0.3), 2),
    ("kpz_1d_256", W.kpz_1d(256, replicas=3), 100),
    ("kpz_1d_4096", W.kpz_1d(4096, replicas=1), 50),
    ("kpz_1d_65536_cluster_R3", W.kpz_1d(65536, replicas=3, sigma0=0.2), 30),
    ("kpz_1d_16384_cluster_R3", W.kpz_1d(16384, replicas=3, sigma0=0.2), 30),
    ("model_a_1d_32768_setd2_cluster", W.model_a_64(d=1, n=[32768], dx=[1.0], scheme=2, sigma0=0.3), 30),
    # at twice the SM count in replicas the 16384-point lines take the one-block-per-replica kernel
    ("kpz_1d_16384_single_block_R304", W.kpz_1d(16384, replicas=304, sigma0=0.2), 3),
    ("model_a_1d_65536_setd2", W.model_a_64(d=1, n=[65536], dx=[1.0], scheme=2, sigma0=0.3), 30),
    ("model_a_1d_128", W.model_a_64(d=1, n=[128], dx=[1.0], replicas=2), 100),
    ("cgl_1d_64_setd2", W.cgl_2048(n=[64], d=1, dx=[0.5], replicas=2, p=[2.0, -0.5, 1e-3]), 100),
    ("model_a_16_nodealias", W.model_a_64(n=[16, 16], dealias=0), 100),
    ("cgl_2d_64_setd2", W.cgl_2048(n=[64, 64], replicas=2, p=[2.0, -0.5, 1e-3]), 100),
    ("cgl_2d_128_em", W.cgl_2048(n=[128, 128], scheme=0, h=0.02, p=[2.0, -0.5, 1e-3]), 50),
    ("cgl_2d_32_setd1_nodealias", W.cgl_2048(n=[32, 32], scheme=1, dealias=0, p=[0.5, 0.3, 1e-2]), 60),
    ("model_a_3d_16_setd1", W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3), 60),
    ("model_a_3d_32_setd2", W.model_a_128_3d(n=[32, 32, 32], replicas=1, sigma0=0.3, scheme=2), 30),
    ("model_b_3d_32_em", W.model_a_128_3d(n=[32, 32, 32], model=1, p=[1.0, -0.5, 1.0, 0.2], scheme=0, h=0.02,
                                          sigma0=0.3), 30),
]


@pytest.mark.parametrize("name,w,nsteps", CASES, ids=[c[0] for c in CASES])
def test_step_parity(sft, oracle_mod, name, w, nsteps):
    g, o = start_pair(sft, oracle_mod, w)
    g.step(nsteps)
    o.step(nsteps)
    got = g.field()
    for r in range(w.replicas):
        e = rel_l2(got[r], o.field(r))
        assert e <= 1e-5, (name, r, e)
    spec = g.spectrum()
    for r in range(w.replicas):
        assert rel_l2(spec[r], half_xmajor(o.spectrum(r), w.complex_field)) <= 1e-5
    g.close()


def test_full_size_model_b_1024(sft, oracle_mod):
    """The headline lattice (Model B 1024^2) in the bench's launch configuration:
    a few steps, whole field against the oracle."""
    w = W.model_b_1024(replicas=1, h=0.05)
    g, o = start_pair(sft, oracle_mod, w)
    g.step(4)
    o.step(4)
    assert rel_l2(g.field()[0], o.field(0)) <= 1e-5
    g.close()


@pytest.mark.parametrize("w", [
    W.model_b_1024(replicas=3, scheme=2, h=0.025, sigma0=0.3),
    W.kpz_2d(n=[1024, 1024], replicas=2, sigma0=0.5),
], ids=["model_b_1024_setd2_R3", "kpz_1024_R2"])
def test_pipelined_column_pass_parity(sft, oracle_mod, w):
    """Lattices with 1024-point columns run the bulk-copy pipelined column pass;
    several replicas exercise its (column, replica) work distribution."""
    g, o = start_pair(sft, oracle_mod, w)
    g.step(3)
    o.step(3)
    got = g.field()
    for r in range(w.replicas):
        assert rel_l2(got[r], o.field(r)) <= 1e-5
    g.close()


def test_full_size_model_a_128_3d(sft, oracle_mod):
    """The 3-D linear-response lattice (Model A 128^3) for a few steps."""
    w = W.model_a_128_3d(replicas=2, sigma0=0.3)
    g, o = start_pair(sft, oracle_mod, w)
    g.step(3)
    o.step(3)
    got = g.field()
    for r in range(2):
        assert rel_l2(got[r], o.field(r)) <= 1e-5
    g.close()


def test_full_size_cgl_2048(sft, oracle_mod):
    """The CGL lattice (2048^2, dx = 0.5, SETD2) for two steps."""
    w = W.cgl_2048(replicas=1)
    g, o = start_pair(sft, oracle_mod, w)
    g.step(2)
    o.step(2)
    assert rel_l2(g.field()[0], o.field(0)) <= 1e-5
    g.close()


def test_model_b_zero_mode_bitwise(sft):
    w = W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3)
    g = gpu_stepper(sft, w)
    g.set_field(W.initial_fields(w).astype(np.float32))
    s0 = g.spectrum()[:, 0, 0].copy()
    g.step(37)
    s1 = g.spectrum()[:, 0, 0]
    assert np.array_equal(s0.view(np.uint64), s1.view(np.uint64))
    g.close()


def test_graph_and_plain_launches_bit_identical(sft):
    w = W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3, scheme=2)
    a = gpu_stepper(sft, w)
    b = gpu_stepper(sft, w)
    f = W.initial_fields(w).astype(np.float32)
    a.set_field(f)
    b.set_field(f)
    a.step(53)
    b.step_plain(53)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    a.close()
    b.close()


def test_checkpoint_resume_bit_identical(sft):
    w = W.model_a_64(n=[64, 64], replicas=2, scheme=2)
    a = gpu_stepper(sft, w)
    a.set_field(W.initial_fields(w).astype(np.float32))
    a.step(20)
    blob = a.checkpoint()
    a.step(30)
    ref = a.spectrum().copy()
    b = gpu_stepper(sft, w)
    b.restore(blob)
    assert b.step_count == 20
    b.step(30)
    assert np.array_equal(b.spectrum().view(np.uint64), ref.view(np.uint64))
    # a checkpoint of another configuration is refused
    c = gpu_stepper(sft, w.with_(h=0.02))
    with pytest.raises(sft.SftError) as ei:
        c.restore(blob)
    assert ei.value.status == sft.SFT_ECHECKPOINT
    for x in (a, b, c):
        x.close()


def test_nonfinite_state_is_reported(sft):
    w = W.model_a_64(n=[32, 32])
    g = gpu_stepper(sft, w)
    f = W.initial_fields(w).astype(np.float32)
    f[0, 3, 5] = np.nan
    g.set_field(f)
    g.step(3)
    with pytest.raises(sft.SftError) as ei:
        g.sync()
    assert ei.value.status == sft.SFT_ENONFINITE
    g.close()


def test_init_random_parity(sft, oracle_mod):
    for w in (W.model_a_64(n=[64, 64], replicas=2), W.cgl_2048(n=[64], d=1, dx=[0.5], replicas=2)):
        g = gpu_stepper(sft, w)
        g.init_random(0.37)
        o = oracle_for(oracle_mod, w)
        o.init_random(0.37)
        spec = g.spectrum()
        for r in range(w.replicas):
            assert rel_l2(spec[r], half_xmajor(o.spectrum(r), w.complex_field)) < 2e-6
        g.close()


# ------------------------------------------------------------------ observables
def test_structure_factor_twotime_roughness(sft, oracle_mod):
    w = W.kpz_2d(n=[64, 64], replicas=3, sigma0=0.5)
    g, o = start_pair(sft, oracle_mod, w)
    g.step(10)
    o.step(10)
    sk = g.observe(sft.SFT_OBS_SK)
    ns = g.nshells()
    ov, oc = o.shells(0)
    assert np.array_equal(sk[ns:], oc)
    assert np.allclose(sk[:ns], ov, rtol=2e-5, atol=1e-12 * np.abs(ov).max())
    per = g.observe(sft.SFT_OBS_SK_REPLICAS).reshape(3, ns)
    assert np.allclose(per.mean(0), sk[:ns], rtol=1e-9, atol=1e-15)
    g.observe(sft.SFT_OBS_MARK)
    o.mark()
    g.step(5)
    o.step(5)
    ck = g.observe(sft.SFT_OBS_CKT)
    oc2, _ = o.shells(1)
    assert np.allclose(ck[:ns], oc2, rtol=3e-5, atol=1e-9 * np.abs(oc2).max())
    rough = g.observe(sft.SFT_OBS_ROUGHNESS)
    assert np.allclose(rough, o.roughness(), rtol=2e-5)
    g.close()


def test_observables_large_shell_count(sft, oracle_mod):
    """A 65536-point line has 32769 shells: the shell sums no longer fit shared
    memory and accumulate in global memory instead."""
    w = W.kpz_1d(65536, replicas=2, sigma0=0.3)
    g, o = start_pair(sft, oracle_mod, w)
    g.step(5)
    o.step(5)
    ns = g.nshells()
    sk = g.observe(sft.SFT_OBS_SK)
    ov, oc = o.shells(0)
    assert ns == len(ov) and np.array_equal(sk[ns:], oc)
    assert np.allclose(sk[:ns], ov, rtol=2e-5, atol=1e-12 * np.abs(ov).max())
    assert np.allclose(g.observe(sft.SFT_OBS_ROUGHNESS), o.roughness(), rtol=2e-5)
    g.close()


def test_replica_offset_shards_one_ensemble(sft, oracle_mod):
    """Two contexts of 2 replicas at replica offsets 0 and 2 (as bench.py gives
    two ranks) reproduce one context of 4 bit for bit (same schedule), and each
    matches the oracle at the same offset."""
    w = W.model_b_1024(n=[64, 64], replicas=4, sigma0=0.3)
    f0 = W.initial_fields(w).astype(np.float32)
    whole = sft.Stepper(w.d, w.n, w.dx, 4, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    whole.set_field(f0)
    sft.sft_set_plan(whole.ctx, [0, 0, 4, 0])
    whole.step(20)
    want = whole.field()
    whole.close()
    for r0 in (0, 2):
        g = sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, replica0=r0)
        g.set_field(f0[r0:r0 + 2])
        sft.sft_set_plan(g.ctx, [0, 0, 4, 0])
        g.step(20)
        got = g.field()
        g.close()
        assert np.array_equal(got, want[r0:r0 + 2])
        o = oracle_mod.Oracle(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, replica0=r0)
        for r in range(2):
            o.set_field(r, f0[r0 + r].astype(np.float64))
        o.step(20)
        for r in range(2):
            assert rel_l2(got[r], o.field(r)) <= 1e-5


# ------------------------------------------------------------------ real-space noise
RSN_CASES = [
    ("model_a_64_setd1_R2", W.model_a_64(replicas=2, sigma0=0.3), 100),
    ("model_b_64_setd2", W.model_b_1024(n=[64, 64], scheme=2, h=0.025, sigma0=0.3), 100),
    ("kpz_2d_32_em", W.kpz_2d(n=[32, 32], replicas=2, scheme=0), 100),
    ("model_b_128_setd1_R3", W.model_b_1024(n=[128, 128], replicas=3, sigma0=0.3), 40),
    ("model_b_1024_setd1_R2", W.model_b_1024(replicas=2, h=0.05), 3),
    # 1-D lines: the draw and its transform inside the line kernel
    ("model_a_1d_256_setd1_R3", W.model_a_64(d=1, n=[256], dx=[1.0], replicas=3, sigma0=0.3), 100),
    ("model_b_1d_2048_setd2", W.model_b_1024(d=1, n=[2048], dx=[1.0], replicas=2, h=0.025, sigma0=0.3), 100),
    ("kpz_1d_1024_em_R2", W.kpz_1d(1024, replicas=2, scheme=0), 100),
    ("kpz_1d_16384_setd1", W.kpz_1d(16384, replicas=2), 20),
    ("model_a_1d_32_nodeal", W.model_a_64(d=1, n=[32], dx=[1.0], replicas=2, sigma0=0.3, dealias=0), 100),
    # 3-D: the row pass draws and transforms along x, the plane pass transforms along y and z, the step's plane
    # pass reads the result
    ("model_a_3d_16_setd1_R2", W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3), 100),
    ("model_b_3d_32_setd2", W.model_a_128_3d(n=[32, 32, 32], model=1, p=[1.0, -0.5, 1.0, 0.2], scheme=2, h=0.01,
                                             sigma0=0.3), 40),
]


@pytest.mark.parametrize("name,w,nsteps", RSN_CASES, ids=[c[0] for c in RSN_CASES])
def test_real_space_noise_step_parity(sft, oracle_mod, name, w, nsteps):
    """Sec. IV step 2, real-space draw: the per-site Philox draw, its forward
    transform and the step that reads eta_a = DFT[eta]_a / sqrt(N^d) against the
    oracle (FP64 DFT of the same normals); replica0 = 3 checks the replica word."""
    R = w.replicas
    f32 = W.initial_fields(w, replicas=R).astype(np.float32)
    g = sft.Stepper(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, replica0=3,
                    noise_space=1)
    g.set_field(f32)
    o = oracle_mod.Oracle(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                          replica0=3, noise_space=1)
    for r in range(R):
        o.set_field(r, f32[r].astype(np.float64))
    g.step(nsteps)
    o.step(nsteps)
    got = g.field()
    for r in range(R):
        assert rel_l2(got[r], o.field(r)) <= 1e-5, (name, r)
    g.close()


def test_real_space_noise_graph_and_plain_bit_identical(sft):
    w = W.model_a_64(n=[64, 64], replicas=2, sigma0=0.3)
    mk = lambda: sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, noise_space=1)
    a, b = mk(), mk()
    f = W.initial_fields(w).astype(np.float32)
    a.set_field(f)
    b.set_field(f)
    a.step(53)
    b.step_plain(53)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    # the two noises are different streams: a Fourier-noise run ends elsewhere
    c = sft.Stepper(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed)
    c.set_field(f)
    c.step(53)
    assert rel_l2(c.field(), a.field()) > 1e-2
    for s in (a, b, c):
        s.close()


# ------------------------------------------------------------------ phase-shift dealiasing
PS_CASES = [
    ("model_a_16_setd1", W.model_a_64(n=[16, 16], replicas=2, sigma0=0.3), 100),
    ("model_a_64_em", W.model_a_64(replicas=2, scheme=0, sigma0=0.3), 100),
    ("model_b_64_setd2", W.model_b_1024(n=[64, 64], scheme=2, h=0.025, sigma0=0.3), 100),
    ("model_b_128_setd1_R3", W.model_b_1024(n=[128, 128], replicas=3, sigma0=0.3), 40),
    ("model_a_512_setd1", W.model_a_64(n=[512, 512], replicas=1, sigma0=0.3), 10),
    ("model_b_1024_setd1_R2", W.model_b_1024(replicas=2, h=0.05), 3),
    ("kpz_2d_32_setd1_R2", W.kpz_2d(n=[32, 32], replicas=2), 100),
    ("kpz_2d_64_setd2", W.kpz_2d(n=[64, 64], scheme=2, h=0.005), 100),
    ("kpz_2d_256_em_R3", W.kpz_2d(n=[256, 256], replicas=3, scheme=0, sigma0=0.5), 20),
    ("kpz_2d_1024_setd1", W.kpz_2d(n=[1024, 1024], sigma0=0.5), 3),
    # 1-D lines: both grids evaluated by the line kernel
    ("model_a_1d_256_setd1_R3", W.model_a_64(d=1, n=[256], dx=[1.0], replicas=3, sigma0=0.3), 100),
    ("model_b_1d_2048_setd2", W.model_b_1024(d=1, n=[2048], dx=[1.0], replicas=2, h=0.025, sigma0=0.3), 100),
    ("kpz_1d_1024_em_R2", W.kpz_1d(1024, replicas=2, scheme=0, sigma0=0.5), 100),
    ("kpz_1d_16384_setd1", W.kpz_1d(16384, replicas=2, sigma0=0.5), 20),
    ("model_a_1d_32_setd2", W.model_a_64(d=1, n=[32], dx=[1.0], replicas=2, sigma0=0.3, scheme=2), 100),
    # 3-D: four copies of P (shifts of y and z), each row averaged over its two x shifts (eight grids in all)
    ("model_a_3d_16_setd1_R2", W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3), 100),
    ("model_b_3d_32_setd2", W.model_a_128_3d(n=[32, 32, 32], model=1, p=[1.0, -0.5, 1.0, 0.2], scheme=2, h=0.01,
                                             sigma0=0.3), 40),
    ("model_a_3d_64_em", W.model_a_128_3d(n=[64, 64, 64], scheme=0, sigma0=0.3), 10),
    # complex fields (CGL): the complex row pass averages its two x shifts, the column pass the two y copies
    ("cgl_32_setd2_R2", W.cgl_2048(n=[32, 32], replicas=2), 100),
    ("cgl_256_setd1", W.cgl_2048(n=[256, 256], scheme=1, p=[0.5, 0.3, 1e-2]), 40),
    ("cgl_64_em", W.cgl_2048(n=[64, 64], scheme=0, p=[0.5, 0.3, 1e-2], sigma0=0.3), 100),
    ("cgl_2048_setd2", W.cgl_2048(replicas=1), 3),
]


@pytest.mark.parametrize("name,w,nsteps", PS_CASES, ids=[c[0] for c in PS_CASES])
def test_phase_shift_dealiasing_step_parity(sft, oracle_mod, name, w, nsteps):
    """Phase-shift dealiasing (dealias = 2): the row pass over both y copies of
    P with its two x shifts, the column pass combining the y copies, against
    the oracle's mean over the four half-cell-shifted grids."""
    w = w.with_(dealias=2)
    g, o = start_pair(sft, oracle_mod, w)
    g.step(nsteps)
    o.step(nsteps)
    got = g.field()
    for r in range(w.replicas):
        assert rel_l2(got[r], o.field(r)) <= 1e-5, (name, r)
    g.close()


@pytest.mark.parametrize("variant", ["phase_shift", "real_space_noise"])
def test_line_variants_graph_plain_and_rejections(sft, variant):
    """1-D variants: graph and plain launches agree bit for bit; lines longer
    than 16384 points and complex lines are refused before any device work."""
    kw = {"dealias": 2} if variant == "phase_shift" else {"noise_space": 1}
    w = W.kpz_1d(512, replicas=3, sigma0=0.5)
    mk = lambda: sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, **kw)
    a, b = mk(), mk()
    f = W.initial_fields(w).astype(np.float32)
    a.set_field(f)
    b.set_field(f)
    a.step(37)
    b.step_plain(37)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    for s in (a, b):
        s.close()
    long_w = W.kpz_1d(32768, replicas=1)
    with pytest.raises(sft.SftError):
        sft.Stepper(long_w.d, long_w.n, long_w.dx, 1, long_w.model, long_w.p, long_w.scheme, long_w.h, 1, **kw)
    c = W.cgl_2048(d=1, n=[128], dx=[0.5], replicas=1)
    with pytest.raises(sft.SftError):
        sft.Stepper(c.d, c.n, c.dx, 1, c.model, c.p, c.scheme, c.h, 1, **kw)


def test_phase_shift_3d_graph_and_plain_bit_identical(sft):
    w = W.model_a_128_3d(n=[16, 16, 16], replicas=2, sigma0=0.3, scheme=2, dealias=2)
    a, b = gpu_stepper(sft, w), gpu_stepper(sft, w)
    f = W.initial_fields(w).astype(np.float32)
    a.set_field(f)
    b.set_field(f)
    a.step(23)
    b.step_plain(23)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    for s in (a, b):
        s.close()


def test_phase_shift_graph_plain_and_checkpoint(sft):
    w = W.model_b_1024(n=[64, 64], replicas=2, sigma0=0.3, scheme=2, dealias=2)
    a, b = gpu_stepper(sft, w), gpu_stepper(sft, w)
    f = W.initial_fields(w).astype(np.float32)
    a.set_field(f)
    b.set_field(f)
    a.step(53)
    b.step_plain(53)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    # the Model B zero mode stays fixed bit for bit with the phase-shifted force too
    s0 = gpu_stepper(sft, w)
    s0.set_field(f)
    z0 = s0.spectrum()[:, 0, 0].copy()
    s0.step(40)
    assert np.array_equal(s0.spectrum()[:, 0, 0].view(np.uint64), z0.view(np.uint64))
    for s in (a, b, s0):
        s.close()


# ------------------------------------------------------------------ lattices of p x 2^k points (p = 3, 5, 7)
MIXED_CASES = [
    ("model_a_48_setd1_R2", W.model_a_64(n=[48, 48], replicas=2, sigma0=0.3), 100),
    ("model_b_96_setd2", W.model_b_1024(n=[96, 96], scheme=2, h=0.025, sigma0=0.3), 100),
    ("kpz_2d_96_em_R2", W.kpz_2d(n=[96, 96], replicas=2, scheme=0), 100),
    ("model_a_192_nodealias", W.model_a_64(n=[192, 192], dealias=0, sigma0=0.3), 40),
    ("model_b_384_setd1_R3", W.model_b_1024(n=[384, 384], replicas=3, sigma0=0.3), 10),
    ("model_b_768_setd1", W.model_b_1024(n=[768, 768], h=0.05), 3),
    ("model_a_80_setd1_R2", W.model_a_64(n=[80, 80], replicas=2, sigma0=0.3), 100),
    ("kpz_2d_160_setd2", W.kpz_2d(n=[160, 160], scheme=2, h=0.005), 60),
    ("model_b_640_setd1", W.model_b_1024(n=[640, 640], h=0.05), 3),
    ("model_a_112_em_R2", W.model_a_64(n=[112, 112], replicas=2, scheme=0, sigma0=0.3), 100),
    ("model_b_448_setd2", W.model_b_1024(n=[448, 448], scheme=2, h=0.025, sigma0=0.3), 5),
    ("kpz_1d_96_R3", W.kpz_1d(96, replicas=3), 100),
    ("model_a_1d_48_setd2", W.model_a_64(d=1, n=[48], dx=[1.0], scheme=2, replicas=2, sigma0=0.3), 100),
    ("kpz_1d_640_em", W.kpz_1d(640, replicas=2, scheme=0), 100),
    ("model_b_1d_448", W.model_b_1024(d=1, n=[448], dx=[1.0], replicas=2, sigma0=0.3), 100),
    ("kpz_1d_768_R200", W.kpz_1d(768, replicas=200, sigma0=0.2), 20),
]


@pytest.mark.parametrize("name,w,nsteps", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_3x2k_lattice_step_parity(sft, oracle_mod, name, w, nsteps):
    """Lattices of p x 2^k points: the radix-p + radix-4/2 Stockham transforms of
    the row and column passes against the oracle's split-radix transform."""
    g, o = start_pair(sft, oracle_mod, w)
    g.step(nsteps)
    o.step(nsteps)
    got = g.field()
    spec = g.spectrum()
    for r in range(w.replicas):
        assert rel_l2(got[r], o.field(r)) <= 1e-5, (name, r)
        assert rel_l2(spec[r], half_xmajor(o.spectrum(r), False)) <= 1e-5
    g.close()


def test_3x2k_graph_plain_and_observables(sft, oracle_mod):
    w = W.model_a_64(n=[96, 96], replicas=2, sigma0=0.3)
    a, b = gpu_stepper(sft, w), gpu_stepper(sft, w)
    f = W.initial_fields(w).astype(np.float32)
    a.set_field(f)
    b.set_field(f)
    a.step(53)
    b.step_plain(53)
    assert np.array_equal(a.spectrum().view(np.uint64), b.spectrum().view(np.uint64))
    a.close()
    b.close()
    # S(k) shells, their mode counts and the roughness against the oracle
    g, o = start_pair(sft, oracle_mod, w)
    g.step(10)
    o.step(10)
    sk = g.observe(sft.SFT_OBS_SK)
    ns = g.nshells()
    ov, oc = o.shells(0)
    assert np.array_equal(sk[ns:], oc)
    assert np.allclose(sk[:ns], ov, rtol=2e-5, atol=1e-12 * np.abs(ov).max())
    assert np.allclose(g.observe(sft.SFT_OBS_ROUGHNESS), o.roughness(), rtol=2e-5)
    g.close()
