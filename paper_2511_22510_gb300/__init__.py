"""Python binding of the GB300 stochastic-ETD stepper (libsft.so).

Argument marshalling only: every step of the method runs in the CUDA library
behind the C ABI of ``include/sft.h``.  The functions below carry the same
names as the C entry points; ``Stepper`` is a small convenience wrapper that
accepts numpy arrays (host buffers) and torch CUDA tensors (device buffers).

There is no fallback: if ``libsft.so`` is missing or cannot be loaded the
import of the library raises, and every call fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SFT_LIB", os.path.join(_HERE, "libsft.so"))

SFT_OK, SFT_EINVAL, SFT_ENOMEM, SFT_ECUDA, SFT_ENONFINITE, SFT_ETIMEOUT, SFT_EUNSUPPORTED, SFT_ECHECKPOINT = range(8)
SFT_MODEL_A, SFT_MODEL_B, SFT_KPZ, SFT_CGL, SFT_CUSTOM = 0, 1, 2, 3, 4
SFT_NL_NONE, SFT_NL_CUBIC, SFT_NL_GRAD2, SFT_NL_CGL = 0, 1, 2, 3
SFT_SETD_EM, SFT_SETD1, SFT_SETD2 = 0, 1, 2
(SFT_OBS_SK, SFT_OBS_SK_REPLICAS, SFT_OBS_MARK, SFT_OBS_CKT, SFT_OBS_ROUGHNESS, SFT_OBS_RESPONSE,
 SFT_OBS_NSHELLS, SFT_OBS_SK_ACCUM, SFT_OBS_SK_TIME_MEAN, SFT_OBS_SK_RESET) = range(10)

_STATUS_NAMES = {0: "SFT_OK", 1: "SFT_EINVAL", 2: "SFT_ENOMEM", 3: "SFT_ECUDA", 4: "SFT_ENONFINITE",
                 5: "SFT_ETIMEOUT", 6: "SFT_EUNSUPPORTED", 7: "SFT_ECHECKPOINT"}

# every function declared in include/sft.h
ABI_FUNCTIONS = [
    "sft_create", "sft_create_batch", "sft_set_field", "sft_init_random", "sft_get_field", "sft_get_spectrum",
    "sft_set_spectrum", "sft_step", "sft_prepare", "sft_step_plain", "sft_sync", "sft_observe", "sft_tangent_step",
    "sft_adjoint", "sft_set_checkpoint_interval", "sft_checkpoint", "sft_restore", "sft_get_step",
    "sft_launches_per_step", "sft_kernel_launches", "sft_draw_noise", "sft_profile", "sft_step2d_noalloc",
    "sft_get_plan", "sft_set_plan", "sft_sde0d", "sft_box_width", "sft_dyn_start", "sft_dyn_result", "sft_last_error",
    "sft_destroy",
]


class SftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class sft_config(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3), ("replicas", C.c_int),
        ("model", C.c_int), ("p", C.c_double * 8), ("scheme", C.c_int), ("h", C.c_double),
        ("seed", C.c_uint64), ("dealias", C.c_int), ("precision", C.c_int), ("stream", C.c_void_p),
        ("replica0", C.c_int), ("custom_nl", C.c_int), ("complex_field", C.c_int),
        ("c_re", C.POINTER(C.c_double)), ("c_im", C.POINTER(C.c_double)), ("noise_D", C.POINTER(C.c_double)),
        ("nl_re", C.POINTER(C.c_double)), ("nl_im", C.POINTER(C.c_double)), ("noise_space", C.c_int),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsft.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libsft.so not found at %s; build it with `python -c 'import __graft_entry__ as g; "
                          "g.build()'`" % path)
    L = C.CDLL(path)
    vp, sz, i64 = C.c_void_p, C.c_size_t, C.c_int64
    L.sft_create.argtypes = [C.POINTER(sft_config), C.POINTER(vp)]
    L.sft_create_batch.argtypes = [C.POINTER(sft_config), C.c_int, C.POINTER(vp)]
    L.sft_set_field.argtypes = [vp, C.c_int, vp, sz]
    L.sft_init_random.argtypes = [vp, C.c_double]
    L.sft_get_field.argtypes = [vp, C.c_int, vp, sz]
    L.sft_get_spectrum.argtypes = [vp, vp, sz]
    L.sft_set_spectrum.argtypes = [vp, vp, sz]
    L.sft_step.argtypes = [vp, i64]
    L.sft_step_plain.argtypes = [vp, i64]
    L.sft_prepare.argtypes = [vp]
    L.sft_sync.argtypes = [vp]
    L.sft_observe.argtypes = [vp, C.c_int, C.POINTER(C.c_double), sz, C.POINTER(sz)]
    L.sft_tangent_step.argtypes = [vp, vp, i64, vp]
    L.sft_adjoint.argtypes = [vp, vp, i64, vp]
    L.sft_set_checkpoint_interval.argtypes = [vp, C.c_int]
    L.sft_checkpoint.argtypes = [vp, vp, sz, C.POINTER(sz)]
    L.sft_restore.argtypes = [vp, vp, sz]
    L.sft_get_step.argtypes = [vp, C.POINTER(i64)]
    L.sft_launches_per_step.argtypes = [vp, C.POINTER(C.c_int)]
    L.sft_draw_noise.argtypes = [vp, i64, vp, sz]
    L.sft_kernel_launches.argtypes = [vp, C.POINTER(i64)]
    L.sft_step2d_noalloc.argtypes = [C.POINTER(sft_config), vp, vp, C.c_int, i64, i64]
    L.sft_profile.argtypes = [vp, i64, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]
    L.sft_get_plan.argtypes = [vp, C.POINTER(C.c_int), C.c_int]
    L.sft_box_width.argtypes = [vp, C.c_int, C.POINTER(C.c_double), sz, C.POINTER(sz)]
    L.sft_dyn_start.argtypes = [vp, C.c_int, C.c_int]
    L.sft_dyn_result.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), sz, C.POINTER(C.c_double)]
    L.sft_sde0d.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_int, C.c_uint64, i64, i64, i64,
                            vp, vp, vp]
    L.sft_set_plan.argtypes = [vp, C.POINTER(C.c_int), C.c_int]
    L.sft_last_error.argtypes = [vp]
    L.sft_last_error.restype = C.c_char_p
    L.sft_destroy.argtypes = [vp]
    L.sft_destroy.restype = None
    for name in ABI_FUNCTIONS:
        fn = getattr(L, name)
        if name not in ("sft_last_error", "sft_destroy"):
            fn.restype = C.c_int
    _lib = L
    return L


def _check(ctx, status: int):
    if status != SFT_OK:
        msg = load_library().sft_last_error(ctx).decode() if ctx else ""
        raise SftError(status, msg)


# ---------------------------------------------------------------- thin wrappers
def make_config(d: int, n: Sequence[int], dx: Sequence[float], replicas: int, model: int, p: Sequence[float],
                scheme: int, h: float, seed: int, dealias: int = 1, stream: Optional[int] = None,
                replica0: int = 0, custom: Optional[dict] = None, noise_space: int = 0,
                precision: int = 0) -> sft_config:
    """custom (SFT_CUSTOM): {"nl": SFT_NL_*, "complex_field": 0/1, "c": c(|a|^2), "D": D(|a|^2),
    "s": s(|a|^2) or None}, arrays over q = 0 .. sum_i (n_i/2)^2 (complex c or s for complex fields)."""
    cfg = sft_config()
    cfg.d = d
    for i in range(3):
        cfg.n[i] = int(n[i]) if i < d else 1
        cfg.dx[i] = float(dx[i]) if i < d else 1.0
    cfg.replicas = replicas
    cfg.model = model
    for i, v in enumerate(p):
        cfg.p[i] = float(v)
    cfg.scheme = scheme
    cfg.h = float(h)
    cfg.seed = int(seed)
    cfg.dealias = dealias
    cfg.precision = int(precision)
    cfg.stream = stream
    cfg.replica0 = replica0
    cfg.noise_space = int(noise_space)
    if custom is not None:
        keep = []

        def put(name, arr):
            if arr is None:
                return
            a = np.ascontiguousarray(arr, dtype=np.float64)
            keep.append(a)
            setattr(cfg, name, a.ctypes.data_as(C.POINTER(C.c_double)))

        cfg.custom_nl = int(custom.get("nl", SFT_NL_NONE))
        cfg.complex_field = int(custom.get("complex_field", 0))
        c = np.asarray(custom["c"])
        put("c_re", c.real)
        put("c_im", c.imag if np.iscomplexobj(c) else None)
        put("noise_D", np.asarray(custom["D"], dtype=np.float64))
        sv = custom.get("s")
        if sv is not None:
            sv = np.asarray(sv)
            put("nl_re", sv.real)
            put("nl_im", sv.imag if np.iscomplexobj(sv) else None)
        cfg._keep = keep  # the tables live until sft_create has copied them
    return cfg


def sft_create(cfg: sft_config):
    ctx = C.c_void_p()
    _check(None, load_library().sft_create(C.byref(cfg), C.byref(ctx)))
    return ctx


def sft_create_batch(cfgs):
    arr = (sft_config * len(cfgs))(*cfgs)
    ctx = C.c_void_p()
    _check(None, load_library().sft_create_batch(arr, len(cfgs), C.byref(ctx)))
    return ctx


def sft_destroy(ctx):
    load_library().sft_destroy(ctx)


def sft_step(ctx, nsteps: int):
    _check(ctx, load_library().sft_step(ctx, int(nsteps)))


def sft_step_plain(ctx, nsteps: int):
    _check(ctx, load_library().sft_step_plain(ctx, int(nsteps)))


def sft_prepare(ctx):
    _check(ctx, load_library().sft_prepare(ctx))


def sft_sync(ctx):
    _check(ctx, load_library().sft_sync(ctx))


def sft_init_random(ctx, sigma: float):
    _check(ctx, load_library().sft_init_random(ctx, float(sigma)))


def sft_set_field(ctx, replica: int, host: np.ndarray):
    a = np.ascontiguousarray(host)
    _check(ctx, load_library().sft_set_field(ctx, int(replica), a.ctypes.data, a.nbytes))


def sft_get_field(ctx, replica: int, out: np.ndarray):
    assert out.flags.c_contiguous
    _check(ctx, load_library().sft_get_field(ctx, int(replica), out.ctypes.data, out.nbytes))
    return out


def sft_get_spectrum(ctx, out: np.ndarray):
    _check(ctx, load_library().sft_get_spectrum(ctx, out.ctypes.data, out.nbytes))
    return out


def sft_set_spectrum(ctx, host: np.ndarray):
    a = np.ascontiguousarray(host, dtype=np.complex64)
    _check(ctx, load_library().sft_set_spectrum(ctx, a.ctypes.data, a.nbytes))


def sft_observe(ctx, kind: int, cap: int) -> np.ndarray:
    out = np.zeros(max(cap, 1), dtype=np.float64)
    w = C.c_size_t()
    _check(ctx, load_library().sft_observe(ctx, int(kind), out.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                           C.byref(w)))
    return out[: w.value]


def sft_tangent_step(ctx, dphi0_dev_ptr: Optional[int], nsteps: int, dphi_out_dev_ptr: Optional[int]):
    _check(ctx, load_library().sft_tangent_step(ctx, dphi0_dev_ptr, int(nsteps), dphi_out_dev_ptr))


def sft_adjoint(ctx, cot_dev_ptr: int, nsteps: int, grad_dev_ptr: int):
    _check(ctx, load_library().sft_adjoint(ctx, cot_dev_ptr, int(nsteps), grad_dev_ptr))


def sft_set_checkpoint_interval(ctx, segment: int):
    _check(ctx, load_library().sft_set_checkpoint_interval(ctx, int(segment)))


def sft_checkpoint(ctx) -> bytes:
    need = C.c_size_t()
    _check(ctx, load_library().sft_checkpoint(ctx, None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value)
    _check(ctx, load_library().sft_checkpoint(ctx, buf, need.value, C.byref(need)))
    return buf.raw


def sft_restore(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(ctx, load_library().sft_restore(ctx, buf, len(blob)))


def sft_get_step(ctx) -> int:
    v = C.c_int64()
    _check(ctx, load_library().sft_get_step(ctx, C.byref(v)))
    return v.value


def sft_step2d_noalloc(cfg: sft_config, phi_dev_ptr: int, fprev_dev_ptr: Optional[int], history_valid: int,
                       step0: int, nsteps: int):
    """Context-free 2-D step on caller-owned device buffers; allocates nothing."""
    _check(None, load_library().sft_step2d_noalloc(C.byref(cfg), phi_dev_ptr, fprev_dev_ptr, int(history_valid),
                                                   int(step0), int(nsteps)))


def sft_kernel_launches(ctx) -> int:
    v = C.c_int64()
    _check(ctx, load_library().sft_kernel_launches(ctx, C.byref(v)))
    return v.value


def sft_get_plan(ctx) -> list:
    """[row shape, column shape, replicas per column block, pipelined column pass]"""
    out = (C.c_int * 4)()
    _check(ctx, load_library().sft_get_plan(ctx, out, 4))
    return list(out)


def sft_set_plan(ctx, plan: Sequence[int]):
    v = (C.c_int * 4)(*[int(x) for x in plan])
    _check(ctx, load_library().sft_set_plan(ctx, v, 4))


def sft_box_width(ctx, ell: int, replicas: int) -> np.ndarray:
    """w_ell^2 per replica: mean over boxes of ell^d sites of the in-box variance."""
    out = np.zeros(replicas)
    n = C.c_size_t()
    _check(ctx, load_library().sft_box_width(ctx, int(ell), out.ctypes.data_as(C.POINTER(C.c_double)), replicas,
                                             C.byref(n)))
    return out


def sft_dyn_start(ctx, M: int, every: int = 1):
    _check(ctx, load_library().sft_dyn_start(ctx, int(M), int(every)))


def sft_dyn_result(ctx, nmodes: int, M: int):
    """(C [nmodes, M], chi [nmodes, M] complex, dbar) of App. C; b at index b mod M."""
    Cv = np.zeros(nmodes * M)
    chi = np.zeros(2 * nmodes * M)
    db = C.c_double()
    dp = C.POINTER(C.c_double)
    _check(ctx, load_library().sft_dyn_result(ctx, Cv.ctypes.data_as(dp), chi.ctypes.data_as(dp), nmodes * M,
                                              C.byref(db)))
    return Cv.reshape(nmodes, M), chi.view(np.complex128).reshape(nmodes, M), db.value


SFT_SDE_SAO, SFT_SDE_GBM = 0, 1
SFT_SDE_EM, SFT_SDE_MILSTEIN, SFT_SDE_SETD_EM, SFT_SDE_SETD_MILSTEIN, SFT_SDE_SETD1 = 0, 1, 2, 3, 4


def sft_sde0d(kind: int, p: Sequence[float], scheme: int, h: float, nsteps: int, u_dev_ptr: int, npaths: int,
              seed: int, substeps: int = 1, step0: int = 0, w_dev_ptr: Optional[int] = None,
              stream: Optional[int] = None):
    """0-d SDE ensemble (Sec. III) on device arrays of npaths doubles (u in/out, W accumulated)."""
    pv = (C.c_double * 8)(*([float(x) for x in p] + [0.0] * (8 - len(p))))
    st = load_library().sft_sde0d(int(kind), pv, int(scheme), float(h), int(substeps), int(seed), int(step0),
                                  int(nsteps), int(npaths), u_dev_ptr, w_dev_ptr, stream)
    _check(None, st)


def sft_launches_per_step(ctx) -> int:
    v = C.c_int()
    _check(ctx, load_library().sft_launches_per_step(ctx, C.byref(v)))
    return v.value


def sft_draw_noise(ctx, step: int, out: np.ndarray):
    _check(ctx, load_library().sft_draw_noise(ctx, int(step), out.ctypes.data, out.nbytes))
    return out


def sft_profile(ctx, nsteps: int):
    """Mean per-kernel and per-step durations (ms) over nsteps plain launches."""
    out = np.zeros(8)
    nk = C.c_int()
    _check(ctx, load_library().sft_profile(ctx, int(nsteps), out.ctypes.data_as(C.POINTER(C.c_double)), 8,
                                           C.byref(nk)))
    return out[: nk.value + 1]


# ---------------------------------------------------------------- convenience
class Batch:
    """Several configurations (same model and scheme, uneven lattice sizes)
    advanced together: 1-D members in one persistent launch, the others on a
    parallel branch of the same CUDA graph.  Replicas are numbered member by
    member."""

    def __init__(self, cfgs):
        self.cfgs = list(cfgs)
        self.ctx = sft_create_batch(self.cfgs)
        self.R = sum(c.replicas for c in self.cfgs)

    def close(self):
        if getattr(self, "ctx", None):
            sft_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        sft_step(self.ctx, n)

    def step_plain(self, n=1):
        sft_step_plain(self.ctx, n)

    def sync(self):
        sft_sync(self.ctx)

    def set_field(self, replica: int, field: np.ndarray):
        sft_set_field(self.ctx, replica, np.ascontiguousarray(field, dtype=np.float32))

    def field(self, replica: int, shape) -> np.ndarray:
        out = np.zeros(shape, dtype=np.float32)
        sft_get_field(self.ctx, replica, out)
        return out

    def init_random(self, sigma):
        sft_init_random(self.ctx, sigma)

    def roughness(self) -> np.ndarray:
        return sft_observe(self.ctx, SFT_OBS_ROUGHNESS, self.R)


class Stepper:
    """R replicas of one field behind one sft context.

    ``n``/``dx`` are x-first.  Real-space fields are numpy arrays of shape
    (R,) + (nz, ny, nx)[-d:]; spectra come back in the library's x-major
    layout with shape (R, HX, nz, ny) squeezed to (R, HX[, nz], ny) style
    arrays (see ``spectrum``).
    """

    def __init__(self, d, n, dx, replicas, model, p, scheme, h, seed, dealias=1, stream=None, replica0=0,
                 custom=None, noise_space=0, precision=0):
        self.cfg = make_config(d, n, dx, replicas, model, p, scheme, h, seed, dealias, stream, replica0, custom,
                               noise_space, precision)
        self.ctx = sft_create(self.cfg)
        self.d, self.R = d, replicas
        self.n = [int(n[i]) for i in range(d)]
        self.shape = tuple(reversed(self.n))
        self.complex_field = model == SFT_CGL or (model == SFT_CUSTOM and bool(custom.get("complex_field", 0)))
        self.sites = int(np.prod(self.n))
        nx = self.n[0]
        self.hx = nx if self.complex_field else nx // 2 + 1
        rest = self.n[1:] if d > 1 else []
        self.spec_shape = (replicas, self.hx) + tuple(reversed(rest))  # (R, HX, [nz,] [ny])

    def close(self):
        if getattr(self, "ctx", None):
            sft_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def field_dtype(self):
        return np.complex64 if self.complex_field else np.float32

    def set_field(self, fields: np.ndarray, replica: int = -1):
        sft_set_field(self.ctx, replica, np.ascontiguousarray(fields, dtype=self.field_dtype))

    def init_random(self, sigma: float):
        sft_init_random(self.ctx, sigma)

    def field(self, replica: int = -1) -> np.ndarray:
        R = self.R if replica < 0 else 1
        out = np.zeros((R,) + self.shape, dtype=self.field_dtype)
        sft_get_field(self.ctx, replica, out)
        return out if replica < 0 else out[0]

    def spectrum(self) -> np.ndarray:
        out = np.zeros(self.spec_shape, dtype=np.complex64)
        return sft_get_spectrum(self.ctx, out)

    def set_spectrum(self, spec: np.ndarray):
        sft_set_spectrum(self.ctx, spec)

    def step(self, n: int = 1):
        sft_step(self.ctx, n)

    def noise(self, step: int) -> np.ndarray:
        out = np.zeros(self.spec_shape, dtype=np.complex64)
        return sft_draw_noise(self.ctx, step, out)

    def step_plain(self, n: int = 1):
        sft_step_plain(self.ctx, n)

    def prepare(self):
        sft_prepare(self.ctx)

    def sync(self):
        sft_sync(self.ctx)

    def nshells(self) -> int:
        return int(sft_observe(self.ctx, SFT_OBS_NSHELLS, 1)[0])

    def observe(self, kind: int) -> np.ndarray:
        ns = self.nshells()
        cap = {SFT_OBS_SK: 2 * ns, SFT_OBS_SK_REPLICAS: self.R * ns, SFT_OBS_MARK: 0, SFT_OBS_CKT: 2 * ns,
               SFT_OBS_ROUGHNESS: self.R, SFT_OBS_RESPONSE: ns, SFT_OBS_SK_ACCUM: 0, SFT_OBS_SK_TIME_MEAN: ns + 1,
               SFT_OBS_SK_RESET: 0}[kind]
        return sft_observe(self.ctx, kind, cap)

    @property
    def step_count(self) -> int:
        return sft_get_step(self.ctx)

    def checkpoint(self) -> bytes:
        return sft_checkpoint(self.ctx)

    def restore(self, blob: bytes):
        sft_restore(self.ctx, blob)
