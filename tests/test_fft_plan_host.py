"""Host-side check of the Stockham plans of the CUDA line FFT (FftPlan in
csrc/sft_device.cuh), restated here: for every line length the library
instantiates (powers of two with 8 or 16 values per thread, and p x 2^k with
p = 3, 5, 7), the radix sequence multiplies to N and divides the values per
thread, every exchange-buffer and twiddle index stays inside its buffer, and a
float64 emulation of the passes (the kernel's index arithmetic, thread by
thread) reproduces numpy's FFT in both directions.  This is the check that ran
before the first GPU launch of each new plan."""
import numpy as np
import pytest


def log2(v):
    return 0 if v <= 1 else 1 + log2(v // 2)


def plan(N, EM=16):
    PR = 3 if N % 3 == 0 else (5 if N % 5 == 0 else (7 if N % 7 == 0 else 1))
    mixed = PR > 1
    L = log2(N // PR if mixed else N)
    E = 4 * PR if mixed else (N if N <= 16 else (EM if N >= 512 else (N if (N <= 32 and EM >= 32) else 16)))
    R0 = PR if mixed else E
    E2 = 4 if mixed else E
    LE = log2(E2)
    LR = L if mixed else L - log2(R0)
    P = 1 + (LR + LE - 1) // LE

    def radix(p):
        return R0 if p == 0 else (E2 if p < P - 1 else (E2 if LR % LE == 0 else (1 << (LR % LE))))

    PAD = R0 if R0 >= 16 else 16
    return dict(E=E, T=N // E, radices=[radix(p) for p in range(P)], PAD=PAD, BUF=N + N // PAD + 1)


def emulate(N, x, inv, EM):
    pl = plan(N, EM)
    E, T = pl["E"], pl["T"]
    sign = 1 if inv else -1
    tw = np.exp(-2j * np.pi * np.arange(N) / N)
    xpos = lambda i: i + i // pl["PAD"]
    v = np.array([[x[t + T * e] for e in range(E)] for t in range(T)])
    buf = np.full(pl["BUF"], np.nan + 0j)
    NS = 1
    for p, R in enumerate(pl["radices"]):
        NB = E // R
        xs = np.zeros((T, NB, R), complex)
        for t in range(T):
            for b in range(NB):
                j = t + T * b
                for r in range(R):
                    if p == 0:
                        xs[t, b, r] = v[t, b + r * NB]
                    else:
                        i = xpos(j + r * (N // R))
                        assert i < pl["BUF"]
                        xs[t, b, r] = buf[i]
                if p > 0:
                    k = j % NS
                    for r in range(1, R):
                        ti = r * k * (N // (NS * R))
                        assert 0 <= ti < N
                        xs[t, b, r] *= np.conj(tw[ti]) if inv else tw[ti]
                m = np.arange(R)
                xs[t, b] = np.exp(sign * 2j * np.pi * np.outer(m, m) / R) @ xs[t, b]
        if NS * R == N:
            for t in range(T):
                for b in range(NB):
                    for s in range(R):
                        v[t, b + s * NB] = xs[t, b, s]
            break
        buf[:] = np.nan
        for t in range(T):
            for b in range(NB):
                j = t + T * b
                k = j % NS
                base = (j // NS) * NS * R + k
                for s in range(R):
                    i = xpos(base + s * NS)
                    assert i < pl["BUF"]
                    buf[i] = xs[t, b, s]
        NS *= R
    return np.array([v[n % T, n // T] for n in range(N)])


SIZES = ([(n, 16) for n in (16, 32, 64, 128, 256)] + [(n, em) for n in (512, 1024, 2048, 4096) for em in (8, 16)]
         + [(n, 16) for n in (24, 48, 96, 192, 384, 768, 40, 80, 160, 320, 640, 56, 112, 224, 448)])


@pytest.mark.parametrize("N,EM", SIZES, ids=["%d_e%d" % s for s in SIZES])
def test_stockham_plan(N, EM):
    pl = plan(N, EM)
    assert int(np.prod(pl["radices"])) == N
    assert all(pl["E"] % r == 0 for r in pl["radices"])
    assert pl["T"] * pl["E"] == N
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = np.fft.fft(x)
    assert np.abs(emulate(N, x, False, EM) - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(emulate(N, x, True, EM) - np.fft.ifft(x) * N).max() <= 1e-12 * np.abs(ref).max()
