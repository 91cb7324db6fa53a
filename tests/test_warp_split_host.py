"""Host-side check of the 2048-point lines split over two warps (the complex
warp row and column passes, csrc/sft_k2c_rowwarp.cu and
csrc/sft_k2c_colwarp.cu), restated here in float64:

- the row pass's swizzled shared tile: every (column, row) of a block's tile
  has its own 8-byte slot inside the tile, and the per-lane base plus a step of
  32 columns that the kernel uses equals the direct swizzled offset;
- the twiddle factoring W_2048^{t + 32 e} = W_2048^{t + 32 (e mod 2)} W_32^{e div 2};
- the transform split: decimation in frequency on the way in (halves combined,
  two 1024-point inverse transforms give the even and odd samples), decimation
  in time on the way out (parity classes transformed, combined with W^k), which
  reproduces numpy's 2048-point transforms, and the row pass's |A|^2 A on top.
This is the check that ran before the first GPU launch of these kernels."""
import numpy as np
import pytest


def cr_off(H, c, r):
    """Byte offset of (column c, row r): pieces of 64 / H bytes, SWIZZLE_32B (H = 2) or SWIZZLE_64B (H = 1)."""
    piece = (8 // H) * 8
    o = c * piece + r * 8
    return o ^ (((o >> 7) & 1) << 4) if H == 2 else o ^ (((o >> 7) & 3) << 4)


@pytest.mark.parametrize("H", [1, 2])
def test_row_tile_layout(H):
    NX, ROWS = 1024 * H, 8 // H
    NC, M = 2 * (NX // 3) + 1, NX // 3 + 1
    BOXC = 128 if H == 2 else 176
    TILE = -(-NC // BOXC) * BOXC * ROWS * 8
    ESTEP, CSH = 32 * ROWS * 8, NX - NC
    EH = -(-(NX - M + 1) // 32)
    offs = {(c, r): cr_off(H, c, r) for c in range(NC) for r in range(ROWS)}
    assert len(set(offs.values())) == len(offs)
    assert all(0 <= o and o + 8 <= TILE for o in offs.values())
    assert 2 * (1024 + TILE + 8 * 8192 + 16 + 1024) <= 233472  # two blocks per SM
    col = lambda ax: ax if ax < M else ax - CSH
    written = set()
    for warp in range(8):
        r, h = warp // H, warp % H
        for lane in range(32):
            blo = cr_off(H, lane, r)
            bhi = cr_off(H, lane + 32 * EH - CSH, r) if H == 1 else cr_off(H, lane + 1024 - CSH, r)
            for e in range(32):
                k = lane + 32 * e
                if H == 1:
                    if k < M:
                        assert blo + ESTEP * e == offs[(k, r)]
                    elif k >= NX - M + 1:
                        assert bhi + ESTEP * (e - EH) == offs[(col(k), r)]
                else:
                    if k < M:
                        assert blo + ESTEP * e == offs[(k, r)]
                    if k + 1024 >= NX - M + 1:
                        assert bhi + ESTEP * e == offs[(col(k + 1024), r)]
                ax = 1024 * h + k
                if ax < M or ax >= NX - M + 1:
                    assert (col(ax), r) not in written
                    written.add((col(ax), r))
    assert len(written) == NC * ROWS


def tw(n, k):
    return np.exp(-2j * np.pi * k / n)


def test_twiddle_factoring():
    t = np.arange(32)[:, None]
    e = np.arange(32)[None, :]
    direct = tw(2048, t + 32 * e)
    factored = tw(2048, t + 32 * (e % 2)) * tw(32, e // 2)
    assert np.abs(direct - factored).max() < 1e-15


def split_inverse(X):
    """A = sum_k X[k] e^{+2 pi i k x / 2048}: warp 0 -> A(2n), warp 1 -> A(2n + 1)."""
    k = np.arange(1024)
    w0 = X[:1024] + X[1024:]
    w1 = (X[:1024] - X[1024:]) * np.conj(tw(2048, k))
    return np.fft.ifft(w0) * 1024, np.fft.ifft(w1) * 1024


def split_forward(a_even, a_odd):
    """X = FFT_2048 of the interleaved samples: warp 0 -> X[k], warp 1 -> X[k + 1024]."""
    k = np.arange(1024)
    E, O = np.fft.fft(a_even), np.fft.fft(a_odd) * tw(2048, k)
    return E + O, E - O


def test_split_transforms_match_numpy():
    rng = np.random.default_rng(7)
    X = rng.standard_normal(2048) + 1j * rng.standard_normal(2048)
    ae, ao = split_inverse(X)
    A = np.fft.ifft(X) * 2048
    assert np.allclose(ae, A[0::2], atol=1e-10) and np.allclose(ao, A[1::2], atol=1e-10)
    x0, x1 = split_forward(A[0::2], A[1::2])
    assert np.allclose(np.concatenate([x0, x1]), np.fft.fft(A), atol=1e-9)


def test_split_row_pass_cubic_term():
    # the row pass's Q on the carried columns: DFT_x(|A|^2 A), A = IDFT_x(P) (unnormalised), P zero off the band
    rng = np.random.default_rng(11)
    nx = 2048
    a = np.arange(nx)
    carried = 3 * np.minimum(a, nx - a) < nx
    P = np.where(carried, rng.standard_normal(nx) + 1j * rng.standard_normal(nx), 0) / nx
    ae, ao = split_inverse(P)
    x0, x1 = split_forward(ae * np.abs(ae) ** 2, ao * np.abs(ao) ** 2)
    A = np.fft.ifft(P) * nx
    want = np.fft.fft(A * np.abs(A) ** 2)
    got = np.concatenate([x0, x1])
    assert np.abs(got - want)[carried].max() < 1e-9 * np.abs(want).max()
