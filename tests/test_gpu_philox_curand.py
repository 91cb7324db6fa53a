"""The oracle's Philox4x32-10 against cuRAND's device implementation
(curand_Philox4x32_10, a library call on the GPU): bit for bit on random
counters and keys, including the counter words the noise map uses (tags 0-3).
The GPU path's normals are bit-identical to the oracle's (test_gpu_parity), so
this pins both to a third implementation besides the published known answers."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def xcheck():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = os.path.join(HERE, "_build", "libphilox_xcheck.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "philox_xcheck.cu"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.curand_philox_words.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    return lib


def test_oracle_philox_matches_curand(xcheck, oracle_mod):
    rng = np.random.default_rng(17)
    n = 2000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:400, 3] = np.arange(400) % 4          # the tags of the noise map
    ctr[400:800, 1:3] = 0                      # small step and replica words
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    out = np.zeros((n, 4), dtype=np.uint32)
    rc = xcheck.curand_philox_words(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, n)
    assert rc == 0
    for i in range(n):
        assert oracle_mod.philox4x32_10([int(x) for x in ctr[i]], [int(x) for x in key[i]]) == \
            [int(x) for x in out[i]], i
