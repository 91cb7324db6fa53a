"""FP64 CPU oracle of the pseudo-spectral stochastic-ETD step (test infrastructure).

This package is the independent reference that the CUDA library is checked
against.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product path never does.  It shares no code
with the CUDA library: the C source ``sft_oracle.c`` is compiled here with gcc
(``-ffp-contract=off`` so the single-precision noise recipe is evaluated
operation by operation) and driven through ctypes.

The C file's header lists the paper passages each part follows (Sec. II
schemes, Sec. IV algorithm, Sec. V models, App. A-C conventions) and the
readings taken where the paper is silent.  Parity unpinned: the noise counter
map (which Philox counter each mode or site takes), a convention of this
implementation; the structure and statistics of the noise are pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sft_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsft_oracle.so")
_lock = threading.Lock()
_lib = None

MODEL_A, MODEL_B, KPZ, CGL, CUSTOM = 0, 1, 2, 3, 4
NL_NONE, NL_CUBIC, NL_GRAD2, NL_CGL = 0, 1, 2, 3
EM, SETD1, SETD2 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP contraction off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3),
        ("replicas", C.c_int), ("model", C.c_int), ("p", C.c_double * 8),
        ("nl", C.c_int), ("complex_field", C.c_int),
        ("c_re", C.POINTER(C.c_double)), ("c_im", C.POINTER(C.c_double)),
        ("noise_D", C.POINTER(C.c_double)), ("nl_re", C.POINTER(C.c_double)),
        ("nl_im", C.POINTER(C.c_double)),
        ("scheme", C.c_int), ("h", C.c_double), ("seed", C.c_uint64),
        ("dealias", C.c_int), ("replica0", C.c_int), ("noise_space", C.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            vp = C.c_void_p
            L.or_box_width.argtypes = [vp, C.c_int, dp]
            L.or_box_width.restype = C.c_int
            L.or_force.argtypes = [vp, C.c_int, dp]
            L.or_force.restype = C.c_int
            L.or_mode_operators.argtypes = [vp, dp]
            L.or_dyn_estimators.argtypes = [C.c_int, C.c_long, C.c_int, dp, dp, dp, dp, C.c_double, C.c_double, dp,
                                            dp, dp]
            L.or_dyn_estimators.restype = C.c_int
            L.or_sde0d.argtypes = [C.c_int, dp, C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_int64, C.c_int64,
                                   C.c_int64, dp, dp]
            L.or_sde0d.restype = C.c_int
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.or_bm_log.argtypes = [C.c_float]
            L.or_bm_log.restype = C.c_float
            L.or_bm_sincos_turn.argtypes = [C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.or_bm_pair.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.or_normals4.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.POINTER(C.c_float)]
            L.or_fft_nd.argtypes = [C.c_int, C.POINTER(C.c_int), dp, C.c_int]
            L.or_dft_naive.argtypes = [C.c_int, C.POINTER(C.c_int), dp, dp, C.c_int]
            L.or_phi12.argtypes = [C.c_double, C.c_double, dp]
            L.or_create.argtypes = [C.POINTER(_Cfg)]
            L.or_create.restype = vp
            L.or_destroy.argtypes = [vp]
            L.or_ntot.argtypes = [vp]
            L.or_ntot.restype = C.c_size_t
            L.or_get_step.argtypes = [vp]
            L.or_get_step.restype = C.c_int64
            L.or_set_step.argtypes = [vp, C.c_int64]
            for name in ("or_set_field", "or_get_field", "or_get_spectrum", "or_set_spectrum", "or_get_fprev",
                         "or_get_tangent_spectrum"):
                getattr(L, name).argtypes = [vp, C.c_int, dp]
            L.or_init_random.argtypes = [vp, C.c_double]
            L.or_step.argtypes = [vp, C.c_int64]
            L.or_noise.argtypes = [vp, C.c_int, C.c_int64, dp]
            L.or_mode_coefs.argtypes = [vp, C.c_size_t, C.c_int, dp]
            L.or_nshells.argtypes = [vp]
            L.or_observe_shells.argtypes = [vp, C.c_int, dp, dp]
            L.or_mark.argtypes = [vp]
            L.or_roughness.argtypes = [vp, dp]
            L.or_tangent_step.argtypes = [vp, dp, C.c_int64, dp]
            L.or_observe_response.argtypes = [vp, dp]
            L.or_adjoint.argtypes = [vp, dp, C.c_int64, dp]
            L.or_step_noise.argtypes = [vp, dp]
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------------------
# Stand-alone primitives
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) of one 128-bit counter."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def bm_log(x: float) -> float:
    return float(lib().or_bm_log(C.c_float(x)))


def bm_sincos_turn(k24: int):
    s, c = C.c_float(), C.c_float()
    lib().or_bm_sincos_turn(C.c_uint32(k24), C.byref(s), C.byref(c))
    return s.value, c.value


def bm_pair(wa: int, wb: int):
    z0, z1 = C.c_float(), C.c_float()
    lib().or_bm_pair(C.c_uint32(wa), C.c_uint32(wb), C.byref(z0), C.byref(z1))
    return np.float32(z0.value), np.float32(z1.value)


def normals4(seed: int, c0: int, c1: int, c2: int, c3: int) -> np.ndarray:
    out = (C.c_float * 4)()
    lib().or_normals4(C.c_uint64(seed), c0 & 0xFFFFFFFF, c1 & 0xFFFFFFFF, c2 & 0xFFFFFFFF,
                      c3 & 0xFFFFFFFF, out)
    return np.array(list(out), dtype=np.float32)


def _dims(shape):
    # numpy shape (..., y, x) -> C dims x, y, z
    return list(reversed(shape))


def fft_nd(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised radix-2 FFT (sign -1 forward, +1 inverse) of a complex array."""
    x = np.ascontiguousarray(a, dtype=np.complex128).copy()
    dims = _dims(x.shape)
    n = (C.c_int * 3)(*(dims + [1] * (3 - len(dims))))
    rc = lib().or_fft_nd(len(dims), n, x.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)), sign)
    if rc != 0:
        raise ValueError("oracle FFT needs power-of-two sizes")
    return x


def dft_naive(a: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.complex128)
    out = np.empty_like(x)
    dims = _dims(x.shape)
    n = (C.c_int * 3)(*(dims + [1] * (3 - len(dims))))
    lib().or_dft_naive(len(dims), n, x.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)),
                       out.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)), sign)
    return out


def phi12(z: complex):
    out = np.zeros(4)
    lib().or_phi12(float(np.real(z)), float(np.imag(z)), _dptr(out))
    return complex(out[0], out[1]), complex(out[2], out[3])


# --------------------------------------------------------------------------
# Stepper
# --------------------------------------------------------------------------
def dyn_estimators(phi, F, c, D, T, norm):
    """App. C estimators from an ensemble of recorded series.

    phi, F: complex arrays (S, n, M) -- state and nonlinear term of n modes at M
    sample times spanning T, for S replicas; c (complex) and D: (n,) linear
    operator and noise strength; norm = (L/N^2)^d.  Returns (C, chi, Dbar) with
    C, chi of shape (n, M) over the DFT frequency index b (omega_b = 2 pi b / T,
    b signed) and Dbar the mean |2 Im chi - (omega / D) C| over modes with D > 0.
    """
    phi = np.ascontiguousarray(phi, dtype=np.complex128)
    F = np.ascontiguousarray(F, dtype=np.complex128)
    S, n, M = phi.shape
    c = np.ascontiguousarray(np.broadcast_to(np.asarray(c, dtype=np.complex128), (n,)))
    D = np.ascontiguousarray(np.broadcast_to(np.asarray(D, dtype=np.float64), (n,)))
    Cout = np.zeros((n, M))
    chi = np.zeros((n, M), dtype=np.complex128)
    dbar = np.zeros(1)
    rc = lib().or_dyn_estimators(S, n, M, _dptr(phi.view(np.float64)), _dptr(F.view(np.float64)),
                                 _dptr(c.view(np.float64)), _dptr(D), float(T), float(norm), _dptr(Cout),
                                 _dptr(chi.view(np.float64)), _dptr(dbar))
    if rc != 0:
        raise ValueError("dyn_estimators: bad arguments")
    return Cout, chi, float(dbar[0])


class Oracle:
    """One oracle context: R replicas of a d-dimensional periodic field.

    ``n`` and ``dx`` are given x-first (x is the fastest real-space axis).
    Fields are numpy arrays of shape ``(R, [nz,] [ny,] nx)``.  Spectra are the
    FULL complex DFT with the same shape.
    """

    def __init__(self, d, n, dx, replicas, model, p, scheme, h, seed, dealias=1,
                 nl=NL_NONE, complex_field=0, c_re=None, c_im=None, noise_D=None,
                 nl_re=None, nl_im=None, replica0=0, noise_space=0):
        cfg = _Cfg()
        cfg.replica0 = int(replica0)
        cfg.noise_space = int(noise_space)
        cfg.d = d
        for i in range(3):
            cfg.n[i] = int(n[i]) if i < d else 1
            cfg.dx[i] = float(dx[i]) if i < d else 1.0
        cfg.replicas = replicas
        cfg.model = model
        for i, v in enumerate(p):
            cfg.p[i] = float(v)
        cfg.nl = nl
        cfg.complex_field = complex_field
        self._keep = []
        for name, arr in (("c_re", c_re), ("c_im", c_im), ("noise_D", noise_D), ("nl_re", nl_re),
                          ("nl_im", nl_im)):
            if arr is not None:
                a = np.ascontiguousarray(arr, dtype=np.float64)
                self._keep.append(a)
                setattr(cfg, name, _dptr(a))
        cfg.scheme = scheme
        cfg.h = h
        cfg.seed = seed
        cfg.dealias = dealias
        self._cfg = cfg
        self._p = lib().or_create(C.byref(cfg))
        if not self._p:
            raise ValueError("oracle rejected the configuration")
        self.d, self.R = d, replicas
        self.n = [int(n[i]) for i in range(d)]
        self.shape = tuple(reversed(self.n))
        self.complex_field = model == CGL or (model == CUSTOM and complex_field)
        self.ntot = int(np.prod(self.n))

    def __del__(self):
        if getattr(self, "_p", None):
            lib().or_destroy(self._p)
            self._p = None

    @property
    def step_count(self):
        return int(lib().or_get_step(self._p))

    @step_count.setter
    def step_count(self, v):
        lib().or_set_step(self._p, int(v))

    def set_field(self, r, field):
        if self.complex_field:
            a = np.ascontiguousarray(field, dtype=np.complex128).reshape(-1).view(np.float64)
        else:
            a = np.ascontiguousarray(field, dtype=np.float64).reshape(-1)
        lib().or_set_field(self._p, r, _dptr(a))

    def init_random(self, sigma):
        lib().or_init_random(self._p, sigma)

    def field(self, r):
        if self.complex_field:
            out = np.zeros(self.ntot, dtype=np.complex128)
            lib().or_get_field(self._p, r, _dptr(out.view(np.float64)))
        else:
            out = np.zeros(self.ntot)
            lib().or_get_field(self._p, r, _dptr(out))
        return out.reshape(self.shape)

    def spectrum(self, r):
        out = np.zeros(self.ntot, dtype=np.complex128)
        lib().or_get_spectrum(self._p, r, _dptr(out.view(np.float64)))
        return out.reshape(self.shape)

    def set_spectrum(self, r, spec):
        a = np.ascontiguousarray(spec, dtype=np.complex128).reshape(-1)
        lib().or_set_spectrum(self._p, r, _dptr(a.view(np.float64)))

    def fprev(self, r):
        out = np.zeros(self.ntot, dtype=np.complex128)
        lib().or_get_fprev(self._p, r, _dptr(out.view(np.float64)))
        return out.reshape(self.shape)

    def step(self, nsteps=1):
        lib().or_step(self._p, int(nsteps))

    def step_with_noise(self, eta):
        """One step with caller-supplied full-spectrum noise of shape (R,) + shape."""
        a = np.ascontiguousarray(eta, dtype=np.complex128).reshape(-1)
        lib().or_step_noise(self._p, _dptr(a.view(np.float64)))

    def noise(self, r, step):
        out = np.zeros(self.ntot, dtype=np.complex128)
        lib().or_noise(self._p, r, int(step), _dptr(out.view(np.float64)))
        return out.reshape(self.shape)

    def mode_coefs(self, idx, first=0):
        out = np.zeros(8)
        lib().or_mode_coefs(self._p, int(idx), int(first), _dptr(out))
        return complex(out[0], out[1]), complex(out[2], out[3]), complex(out[4], out[5]), complex(out[6], out[7])

    def nshells(self):
        return int(lib().or_nshells(self._p))

    def shells(self, kind=0):
        ns = self.nshells()
        out, cnt = np.zeros(ns), np.zeros(ns)
        lib().or_observe_shells(self._p, kind, _dptr(out), _dptr(cnt))
        return out, cnt

    def mark(self):
        lib().or_mark(self._p)

    def roughness(self):
        out = np.zeros(self.R)
        lib().or_roughness(self._p, _dptr(out))
        return out

    def tangent_step(self, dphi0, nsteps):
        if self.complex_field:
            out = np.zeros(self.R * self.ntot, dtype=np.complex128)
            seed = None if dphi0 is None else np.ascontiguousarray(dphi0, dtype=np.complex128).reshape(-1)
            lib().or_tangent_step(self._p, None if seed is None else _dptr(seed.view(np.float64)), int(nsteps),
                                  _dptr(out.view(np.float64)))
        else:
            out = np.zeros(self.R * self.ntot)
            seed = None if dphi0 is None else np.ascontiguousarray(dphi0, dtype=np.float64).reshape(-1)
            lib().or_tangent_step(self._p, None if seed is None else _dptr(seed), int(nsteps), _dptr(out))
        return out.reshape((self.R,) + self.shape)

    def tangent_spectrum(self, r):
        out = np.zeros(self.ntot, dtype=np.complex128)
        lib().or_get_tangent_spectrum(self._p, r, _dptr(out.view(np.float64)))
        return out.reshape(self.shape)

    def response(self):
        out = np.zeros(self.nshells())
        lib().or_observe_response(self._p, _dptr(out))
        return out

    def force(self, r):
        """Nonlinear term F_a of replica r at the current state (full spectrum)."""
        out = np.zeros(self.ntot, dtype=np.complex128)
        lib().or_force(self._p, int(r), _dptr(out.view(np.float64)))
        return out.reshape(self.shape)

    def mode_operators(self):
        """(c_a, D_a) over the full spectrum (shape of a spectrum): the model's linear
        operator and noise strength (Sec. V)."""
        out = np.zeros(3 * self.ntot)
        lib().or_mode_operators(self._p, _dptr(out))
        out = out.reshape(self.ntot, 3)
        return (out[:, 0] + 1j * out[:, 1]).reshape(self.shape), out[:, 2].reshape(self.shape)

    def box_width(self, ell):
        """w_ell^2 per replica: mean over boxes of ell^d sites of the in-box variance (Sec. V.B)."""
        out = np.zeros(self.R)
        if lib().or_box_width(self._p, int(ell), _dptr(out)) != 0:
            raise ValueError("box width: real field and a box size dividing every n_i")
        return out

    def adjoint(self, lam, nsteps):
        """Gradient of <lam, field after nsteps> with respect to the field now (the transpose of the
        tangent for the real inner product; complex fields: Re sum conj(u) v).  Advances the state."""
        cf = np.iscomplexobj(lam) or self.complex_field
        if cf:
            a = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128)).view(np.float64).reshape(-1)
        else:
            a = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
        out = np.zeros(self.R * self.ntot * (2 if cf else 1))
        rc = lib().or_adjoint(self._p, _dptr(a), int(nsteps), _dptr(out))
        if rc != 0:
            raise ValueError("adjoint: truncation or no dealiasing; complex fields with the |A|^2 A term only")
        if cf:
            return out.view(np.complex128).reshape((self.R,) + self.shape)
        return out.reshape((self.R,) + self.shape)


SDE_SAO, SDE_GBM = 0, 1
SDE_EM, SDE_MILSTEIN, SDE_SETD_EM, SDE_SETD_MILSTEIN, SDE_SETD1 = 0, 1, 2, 3, 4


def sde0d(kind, p, scheme, h, nsteps, u0, seed, substeps=1, step0=0, w0=None):
    """0-d SDE ensemble (Sec. III): advances the paths u0 (array) by nsteps steps of
    size h (each the sum of `substeps` fine Wiener increments); returns (u, W)."""
    u = np.array(u0, dtype=np.float64, copy=True).reshape(-1)
    w = np.zeros_like(u) if w0 is None else np.array(w0, dtype=np.float64, copy=True).reshape(-1)
    pv = np.zeros(8)
    pv[:len(p)] = p
    rc = lib().or_sde0d(int(kind), _dptr(pv), int(scheme), float(h), int(substeps), int(seed), int(step0),
                        int(nsteps), int(u.size), _dptr(u), _dptr(w))
    if rc != 0:
        raise ValueError("or_sde0d: invalid arguments")
    return u, w
