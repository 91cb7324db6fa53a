"""Host-side check of the 1024-point warp kernels of the 2-D real step (the
headline lattice), restated here in float64 from their sources:

- fft1024_warp (csrc/sft_warpfft.cuh): a 1024-point line held by one warp as
  lane t, slot e = index t + 32 e; a 32-point radix-2 DIF DFT over the slots
  (with the bit-reversal permutation), the twiddle W_1024^{t k1} as the product
  of S_j = W^{t j} and B_g = W^{8 g t} (slot k1 = 8 g + j), a transpose through
  the XOR-swizzled buffer (element (t, k1) at t 32 + (k1 ^ (2 t mod 32))) and a
  second 32-point DFT over the lanes;
- that swizzle is free of shared-memory bank conflicts for the 16-byte stores
  (quarter warps) and the 8-byte loads (half warps) the transpose issues;
- the slots a transform skips as zero (ZIN) hold only modes outside the 2/3
  band, in every lane;
- k2_rows_pair (csrc/sft_k2d_pair.cu): two real rows per warp as one complex
  transform, read from and written to the 128-byte-swizzled TMA tile, unpacked
  with the mirrored mode of lane (32 - t) mod 32;
- k2_cols_warp (csrc/sft_k2d_colwarp.cu): forward transform of Q along y, the
  SETD update with the coefficient row of |a_x| indexed by |a_y|, the Hermitian
  fix-up on the self-conjugate columns, and P = IFFT_y(M phi / N^2).

Two noise-free steps of Model A and Model B at 1024^2 (temperature 0, so the
noise amplitude g is zero and nothing random is involved), chained through
P and Q exactly as the kernels chain them, equal the FP64 oracle's two steps
(Sec. IV boxed algorithm) to rounding, with and without 2/3 truncation and
for SETD1 and SETD2 (whose history F_prev the column pass carries).  The
column pass's noise map (which lane evaluates which Philox counter and the
lane exchange that hands each mode its pair) reproduces the oracle's noise of
App. B on columns on and off the self-conjugate planes, and the complex
column pass's map (one or two warps per column, csrc/sft_k2c_colwarp.cu)
reproduces the oracle's complex draw."""
import numpy as np
import pytest

import sft_inputs as W

NY = 1024


# ------------------------------------------------------------ warp transform
def _bitrev5(k):
    return int("{:05b}".format(k)[::-1], 2)


def dft32(x, inv):
    """The in-register 32-point DFT of the last axis: radix-2 decimation in
    frequency (span 16 down to 1, twiddle W_32^{i 16 / span} on the
    difference), then the bit-reversal permutation."""
    x = np.array(x, dtype=np.complex128)
    w = np.exp((2j if inv else -2j) * np.pi * np.arange(32) / 32)
    span = 16
    while span >= 1:
        for blk in range(0, 32, 2 * span):
            for i in range(span):
                a, b = x[..., blk + i].copy(), x[..., blk + i + span].copy()
                x[..., blk + i] = a + b
                x[..., blk + i + span] = (a - b) * w[i * (16 // span)]
        span //= 2
    return x[..., [_bitrev5(k) for k in range(32)]]


def tw32_table():
    """tw32[k1 32 + t] = W_1024^{t k1}, forward sign (the table k_twiddles32 builds)."""
    i = np.arange(1024)
    return np.exp(-2j * np.pi * ((i >> 5) * (i & 31)) / 1024)


def swz(t, k1):
    """Offset (in 8-byte elements) of element (lane t, slot k1) in the transpose buffer."""
    return t * 32 + (k1 ^ ((2 * t) & 31))


def warp_twiddle_transpose(v, inv):
    """v[..., lane, slot] -> twiddled and transposed through the swizzled buffer."""
    tw = tw32_table()
    if inv:
        tw = np.conj(tw)
    lanes = np.arange(32)
    out = v.copy()
    S = [None] + [tw[j * 32 + lanes] for j in range(1, 8)]
    B = [None] + [tw[8 * g * 32 + lanes] for g in range(1, 4)]
    for k1 in range(1, 32):
        g, j = k1 >> 3, k1 & 7
        if j:
            out[..., k1] = out[..., k1] * S[j]
        if g:
            out[..., k1] = out[..., k1] * B[g]
    xb = np.zeros(v.shape[:-2] + (1024,), dtype=np.complex128)
    for t in range(32):
        for k1 in range(0, 32, 2):  # one 16-byte store of the pair (k1, k1 + 1)
            p = swz(t, k1)
            assert p % 2 == 0 and swz(t, k1 + 1) == p + 1
            xb[..., p] = out[..., t, k1]
            xb[..., p + 1] = out[..., t, k1 + 1]
    res = np.empty_like(v)
    for lane in range(32):
        for t in range(32):
            res[..., lane, t] = xb[..., t * 32 + (lane ^ ((2 * t) & 31))]
    return res


def fft1024_warp(v, inv):
    """Unnormalised 1024-point transform of v[..., lane, slot] = x[lane + 32 slot]."""
    return dft32(warp_twiddle_transpose(dft32(v, inv), inv), inv)


def to_warp(x):
    """x[..., 1024] -> v[..., lane, slot]."""
    return np.swapaxes(x.reshape(x.shape[:-1] + (32, 32)), -1, -2)


def from_warp(v):
    return np.swapaxes(v, -1, -2).reshape(v.shape[:-2] + (1024,))


def test_fft1024_warp_matches_numpy():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((3, 1024)) + 1j * rng.standard_normal((3, 1024))
    np.testing.assert_allclose(from_warp(fft1024_warp(to_warp(x), False)), np.fft.fft(x), rtol=0, atol=1e-10)
    np.testing.assert_allclose(from_warp(fft1024_warp(to_warp(x), True)), 1024 * np.fft.ifft(x), rtol=0, atol=1e-10)


def test_twiddle_factoring_and_bitrev():
    tw = tw32_table()
    t = np.arange(32)
    for k1 in range(32):
        g, j = k1 >> 3, k1 & 7
        np.testing.assert_allclose(tw[j * 32 + t] * tw[8 * g * 32 + t], np.exp(-2j * np.pi * t * k1 / 1024),
                                   atol=1e-14)
    assert sorted(_bitrev5(k) for k in range(32)) == list(range(32))


def test_transpose_swizzle_is_bank_conflict_free():
    # 32 banks of 4 bytes.  A 16-byte store is served a quarter warp (8 lanes, 128 bytes) at a time, an 8-byte
    # load a half warp (16 lanes) at a time: each phase must touch every bank once.
    for k1 in range(0, 32, 2):
        for q in range(4):
            banks = set()
            for t in range(8 * q, 8 * q + 8):
                b0 = (8 * swz(t, k1) // 4) % 32
                banks.update(range(b0, b0 + 4))
            assert len(banks) == 32, (k1, q)
    for t in range(32):
        for hlf in range(2):
            banks = set()
            for lane in range(16 * hlf, 16 * hlf + 16):
                b0 = (8 * (t * 32 + (lane ^ ((2 * t) & 31))) // 4) % 32
                banks.update((b0, b0 + 1))
            assert len(banks) == 32, (t, hlf)
    # every element has its own slot of the 1024-element buffer
    assert len({swz(t, k) for t in range(32) for k in range(32)}) == 1024


ZIN = 0x001FF800  # slots 11..20


def test_skipped_slots_hold_only_masked_modes():
    for e in range(32):
        if (ZIN >> e) & 1:
            for lane in range(32):
                k = lane + 32 * e
                ks = k if k < 512 else k - 1024
                assert 3 * abs(ks) >= 1024, (e, lane)


# ------------------------------------------------------------ row pass
PAIR_ROWS, BOXC = 16, 176


def tile_pos(c, j):
    """Float2 offset of chunk j (rows 2j, 2j + 1) of column c in the tile (the kernel's tile_pos)."""
    return c * 16 + ((j ^ (c & 7)) << 1)


def tma_swizzle_128b(c, j):
    """Where a TMA load with CU_TENSOR_MAP_SWIZZLE_128B puts 16-byte chunk j of box row c (128-byte rows, the
    chunk index XORed with the row's position in its 1024-byte atom), in float2 units."""
    return (c * 128 + ((j ^ (c % 8)) * 16)) // 8


def row_pass_pair(P, ncols, deal):
    """k2_rows_pair on one replica: P[c, y] (c < ncols) -> Q[c, y], every block of
    16 rows at once (axis 0 of the arrays below is the block)."""
    nc = 1024 // 3 + 1 if deal else 513
    assert ncols == nc
    tilew = -(-nc // BOXC) * BOXC
    nblk = NY // PAIR_ROWS
    zin = ZIN if deal else 0
    c = np.arange(tilew)[:, None]
    j = np.arange(8)[None, :]
    pos = tile_pos(c, j)  # (tilew, 8)
    assert np.array_equal(pos, tma_swizzle_128b(c, j))
    assert len(np.unique(pos)) == pos.size and pos.max() + 1 < tilew * 16
    # the TMA load (columns beyond ncols are filled with zeros): chunk j of column c = rows 2j, 2j + 1
    tile = np.zeros((nblk, tilew * 16), dtype=np.complex128)
    rows = P.reshape(ncols, nblk, 8, 2).transpose(1, 0, 2, 3)  # [block, c, j, row of the pair]
    tile[:, pos[:ncols]] = rows[..., 0]
    tile[:, pos[:ncols] + 1] = rows[..., 1]
    # Z[k] for k = lane + 32 e: the stored column k (e < 16) or the mirror 1024 - k
    lane = np.arange(32)[:, None]
    e = np.arange(32)[None, :]
    lo = e < 16
    col = np.where(lo, lane + 32 * e, 32 * (32 - e) - lane)  # (lane, slot)
    live = (((zin >> e) & 1) == 0) & (col < tilew)
    colc = np.where(live, col, 0)
    v = np.zeros((nblk, 8, 32, 32), dtype=np.complex128)
    for warp in range(8):
        xa = tile[:, tile_pos(colc, warp)]
        xb = tile[:, tile_pos(colc, warp) + 1]
        z = np.where(lo, xa + 1j * xb, np.conj(xa) + 1j * np.conj(xb))
        v[:, warp] = np.where(live, z, 0)
    v = fft1024_warp(v, True)
    v = v.real ** 3 + 1j * v.imag ** 3
    v = fft1024_warp(v, False)
    # unpack: W[1024 - k] from lane (32 - lane) mod 32, slot 31 - e (lane 0: slot (32 - e) mod 32)
    eout = (nc - 1) // 32
    for ee in range(eout + 1):
        k = np.arange(32) + 32 * ee
        src = (32 - np.arange(32)) & 31
        slot = np.where(src == 0, (32 - ee) & 31, 31 - ee)
        assert np.all((src + 32 * slot) % 1024 == (1024 - k) % 1024)
        ok = k < nc
        for warp in range(8):
            w = v[:, warp, np.arange(32), ee]
            wm = v[:, warp, src, slot]
            qa = 0.5 * (w + np.conj(wm))
            qb = 0.5 * ((w.imag + wm.imag) + 1j * (wm.real - w.real))
            tile[:, tile_pos(k[ok], warp)] = qa[:, ok]
            tile[:, tile_pos(k[ok], warp) + 1] = qb[:, ok]
    # the TMA store of the same tile
    out = np.empty((nblk, ncols, 8, 2), dtype=np.complex128)
    out[..., 0] = tile[:, pos[:ncols]]
    out[..., 1] = tile[:, pos[:ncols] + 1]
    return out.transpose(1, 0, 2, 3).reshape(ncols, NY)


def test_row_pass_pair_is_the_cubic_term_along_x():
    rng = np.random.default_rng(5)
    for deal in (True, False):
        nc = 342 if deal else 513
        # rows of real fields: a_x = 0 and the Nyquist column real
        P = rng.standard_normal((513, NY)) + 1j * rng.standard_normal((513, NY))
        P[0].imag = 0
        P[512].imag = 0
        if deal:
            P[nc:] = 0
        Pc = P[:nc].copy()
        Q = row_pass_pair(Pc, nc, deal)
        psi = 1024 * np.fft.irfft(P.T, n=1024, axis=1)  # unnormalised inverse, [y, x]
        ref = np.fft.rfft(psi ** 3, axis=1).T[:nc]
        err = np.max(np.abs(Q - ref)) / np.max(np.abs(ref))
        assert err < 1e-12, (deal, err)


# ------------------------------------------------------------ column pass
def column_pass_warp(Q, phi, fprev, coef, w, deal, first, prime=False):
    """k2_cols_warp on one replica (x-major: phi[a_x, a_y]); returns the new
    phi, F_prev and P.  coef[a_x, a_y] = (f1, A, B, g) of the oracle, read
    by (|a_x|, |a_y|) as the kernel's coefficient rows are."""
    nx = w.n[0]
    hx = nx // 2 + 1
    ncols = sum(1 for c in range(hx) if not deal or 3 * c < nx)
    dk = 2 * np.pi / (nx * w.dx[0])
    mb = w.model == W.MODEL_B
    s0 = -w.p[0] * w.p[2]
    sB = s0 * dk * dk if mb else s0
    scale = 1.0 / (nx * NY)
    ay = np.arange(NY)
    ays = np.where(ay < NY // 2, ay, ay - NY)
    aya = np.abs(ays)
    inm = (3 * aya < NY) if deal else np.ones(NY, bool)  # the 2/3 mask along y
    phi, fprev = phi.copy(), (None if fprev is None else fprev.copy())
    P = np.zeros((ncols, NY), dtype=np.complex128)
    for cc in range(hx):
        has_f = cc < ncols
        plane = cc == 0 or 2 * cc == nx
        if prime:
            xb = np.where(inm, phi[cc] * scale, 0) if has_f else None
        else:
            X = from_warp(fft1024_warp(to_warp(Q[cc]), False)) if has_f else np.zeros(NY, complex)
            f1, A, B, g = (coef[cc, aya, i] for i in range(4))
            if has_f:
                sq = sB * (cc * cc + ays * ays) if mb else np.full(NY, sB)
                F = np.where(inm, X * sq, 0)
            else:
                F = np.zeros(NY, complex)
            if w.scheme == 2 and has_f:
                Ae, Be = (A + B, 0 * B) if first else (A, B)  # the first SETD2 step takes the SETD1 pair
                out = f1 * phi[cc] + Ae * F + Be * fprev[cc]
                fprev[cc] = F
            else:
                Ae = A + B if (w.scheme == 2 and first) else A
                out = f1 * phi[cc] + Ae * F  # g eta = 0: temperature 0
            if plane:
                wv = np.where(2 * ay > NY, np.conj(out[(NY - ay) % NY]), out)
                wv = np.where((ay == 0) | (2 * ay == NY), wv.real + 0j, wv)
                out = wv
            phi[cc] = out
            xb = np.where(inm, out * scale, 0) if has_f else None
        if has_f:
            v = to_warp(xb)
            if deal:
                for e in range(32):
                    if (ZIN >> e) & 1:
                        assert np.all(v[:, e] == 0)
            P[cc] = from_warp(fft1024_warp(v, True))
    return phi, fprev, P


def oracle_coefs(o, nx, first):
    """(f1, A, B, g) of every (|a_x|, |a_y|) from the oracle (real parts: real c)."""
    hy = NY // 2 + 1
    coef = np.zeros((nx // 2 + 1, hy, 4))
    for ax in range(nx // 2 + 1):
        for ay in range(hy):
            f1, A, B, g = o.mode_coefs(ay * nx + ax, first)
            coef[ax, ay] = (f1.real, A.real, B.real, g.real)
    return coef


def half_xmajor(full):
    nx = full.shape[-1]
    return np.moveaxis(full[..., : nx // 2 + 1], -1, 0)


@pytest.mark.parametrize("model,scheme,deal", [
    ("b", 1, True), ("b", 2, True), ("a", 1, True), ("b", 1, False),
], ids=["model_b_setd1", "model_b_setd2", "model_a_setd1", "model_b_setd1_no_dealias"])
def test_two_noise_free_steps_match_the_oracle(oracle_mod, model, scheme, deal):
    if model == "b":
        w = W.model_b_1024(replicas=1, scheme=scheme, sigma0=0.3)
        w = w.with_(p=[w.p[0], w.p[1], w.p[2], 0.0])
    else:
        w = W.model_a_64(n=[1024, 1024], replicas=1, scheme=scheme, sigma0=0.3)
        w = w.with_(p=[w.p[0], w.p[1], w.p[2], 0.0])
    w = w.with_(dealias=1 if deal else 0)
    f0 = W.initial_fields(w)[0].astype(np.float64)
    o = oracle_mod.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    o.set_field(0, f0)
    phi = half_xmajor(o.spectrum(0)).copy()
    coef = oracle_coefs(o, w.n[0], 0)
    assert np.all(coef[:, :, 3] == 0)  # temperature 0: no noise
    if scheme == 2:
        # the kernel's first step reads the SETD2 row as A + B and B = 0: the oracle's first-step coefficients
        c1 = oracle_coefs(o, w.n[0], 1)
        np.testing.assert_allclose(c1[:, :, 1], coef[:, :, 1] + coef[:, :, 2], rtol=1e-13, atol=0)
        assert np.all(c1[:, :, 2] == 0)
    fprev = np.zeros_like(phi) if scheme == 2 else None
    _, _, P = column_pass_warp(None, phi, fprev, coef, w, deal, False, prime=True)
    nc = P.shape[0]
    for s in range(2):
        first = scheme == 2 and s == 0
        Q = row_pass_pair(P, nc, deal)
        phi, fprev, P = column_pass_warp(Q, phi, fprev, coef, w, deal, first)
    o.step(2)
    ref = half_xmajor(o.spectrum(0))
    err = np.max(np.abs(phi - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2))
    assert err < 1e-11, err


# ------------------------------------------------------------ noise map of the column pass
def column_noise_warp(oracle_mod, seed, cc, step, rep):
    """eta of column cc as k2_cols_warp draws it (team_normal_pair_ks with 32
    lanes): the trip over slots (e, e + 1), e even; lane t evaluates Philox at
    j = cc NY + t + 32 (e + (t odd)), counter (j >> 1, step, replica, 0); even
    lanes keep the first pair for slot e and hand the second to lane t + 1,
    odd lanes hand the first to lane t - 1 and keep the second for slot e + 1."""
    eta = np.zeros(NY, dtype=np.complex128)
    plane = cc in (0, NY // 2)  # a_x = 0 or nx / 2 (nx = NY = 1024)
    r2 = np.float32(0.70710677)  # 0x1.6a09e6p-1f
    for e in range(0, 32, 2):
        p = {}
        for t in range(32):
            j = cc * NY + t + 32 * (e + (t & 1))
            z = oracle_mod.normals4(seed, j >> 1, step, rep, 0)
            p[t] = (z[0:2], z[2:4])
        for t in range(32):
            odd = t & 1
            recv = p[t ^ 1][1] if odd else p[t ^ 1][0]  # the partner lane's send (even lanes: p1, odd: p0)
            z0 = recv if odd else p[t][0]
            z1 = p[t][1] if odd else recv
            for h, z in ((0, z0), (1, z1)):
                ay = t + 32 * (e + h)
                if plane and (ay == 0 or ay == NY // 2):
                    eta[ay] = float(z[0])
                else:
                    eta[ay] = complex(np.float32(z[0]) * r2, np.float32(z[1]) * r2)
    return eta


def test_column_pass_noise_map_is_the_oracles(oracle_mod):
    w = W.model_b_1024(replicas=1)
    step, rep = 7, 3
    o = oracle_mod.Oracle(w.d, w.n, w.dx, rep + 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    ref = half_xmajor(o.noise(rep, step))
    ay = np.arange(NY)
    for cc in (0, 1, 2, 341, 342, 511, 512):
        got = column_noise_warp(oracle_mod, w.seed, cc, step, rep)
        keep = (2 * ay <= NY) if cc in (0, NY // 2) else np.ones(NY, bool)  # plane partners: the fix-up's
        np.testing.assert_allclose(got[keep], ref[cc][keep], rtol=2e-7, atol=0, err_msg=str(cc))


def complex_noise_convention(oracle_mod, seed, nyq, cols, step, rep):
    """eta of the complex-field modes (a_x, a_y) by the counter map of App. B's
    complex draw: mode j = a_x n_y + a_y takes the pair (j & 1) of
    Philox(ctr = (j >> 1, step, replica, 0)), eta = (z0 + i z1) / sqrt 2."""
    r2 = np.float32(0.70710677)
    out = np.zeros((len(cols), nyq), dtype=np.complex128)
    for i, c in enumerate(cols):
        for ay in range(nyq):
            j = c * nyq + ay
            z = oracle_mod.normals4(seed, j >> 1, step, rep, 0)[2 * (j & 1): 2 * (j & 1) + 2]
            out[i, ay] = complex(np.float32(z[0]) * r2, np.float32(z[1]) * r2)
    return out


def complex_column_noise_warp(oracle_mod, seed, c, H, step, rep):
    """eta of column c as k2c_cols_warp draws it: warp h of the H warps holds
    a_y = 1024 h + t + 32 e and calls team_normal_pair_ks with the base
    j = c NY + 1024 h (the same lane exchange as the real column pass)."""
    ny = 1024 * H
    r2 = np.float32(0.70710677)
    eta = np.zeros(ny, dtype=np.complex128)
    for h in range(H):
        jb = c * ny + 1024 * h
        for e in range(0, 32, 2):
            p = {}
            for t in range(32):
                j = jb + t + 32 * (e + (t & 1))
                z = oracle_mod.normals4(seed, j >> 1, step, rep, 0)
                p[t] = (z[0:2], z[2:4])
            for t in range(32):
                odd = t & 1
                recv = p[t ^ 1][1] if odd else p[t ^ 1][0]
                z0 = recv if odd else p[t][0]
                z1 = p[t][1] if odd else recv
                for hh, z in ((0, z0), (1, z1)):
                    eta[1024 * h + t + 32 * (e + hh)] = complex(np.float32(z[0]) * r2, np.float32(z[1]) * r2)
    return eta


def test_complex_column_pass_noise_map(oracle_mod):
    # the convention is the oracle's (a 64^2 complex field: every mode drawn, no Hermitian partner)
    w = W.cgl_2048(n=[64, 64], replicas=2)
    step, rep = 5, 1
    o = oracle_mod.Oracle(w.d, w.n, w.dx, 2, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    ref = np.moveaxis(o.noise(rep, step), -1, 0)  # [a_x][a_y]
    cols = [0, 1, 31, 32, 63]
    np.testing.assert_allclose(complex_noise_convention(oracle_mod, w.seed, 64, cols, step, rep), ref[cols],
                               rtol=2e-7, atol=0)
    # the warp column pass on 1024- and 2048-point columns (one or two warps per column) follows it
    for H in (1, 2):
        ny = 1024 * H
        for c in (0, 3, ny // 3, ny - 1):
            got = complex_column_noise_warp(oracle_mod, w.seed, c, H, step, rep)
            want = complex_noise_convention(oracle_mod, w.seed, ny, [c], step, rep)[0]
            np.testing.assert_array_equal(got, want, err_msg=str((H, c)))
