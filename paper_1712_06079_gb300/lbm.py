"""ctypes binding of ``liblbm.so`` (C ABI in ``include/lbm.h``).

Argument marshalling only: every step of the lattice update runs in the CUDA
kernels of the library.  If the library has not been built this module raises
on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

OK, E_INVALID, E_NOMEM, E_CUDA, E_UNSTABLE, E_TIMEOUT, E_STATE, E_IO = range(8)
EOS = {"vdw": 0, "cs": 1, "pr": 2, "rk": 3, "rks": 4, "psi_exp": 5}
FORCE = {"sc": 0, "zc": 1}
GRAD = {"hdm": 0, "cdm": 1}
PREC = {"f32": 0, "f64": 1}
FLAG_TWO_PASS = 1
FLAG_WALLS_Y = 2
FLAG_F32_ARITH = 4
FLAG_STAGED_HOST = 8
GROUPS_BALANCED = -1   # lbm_batch_set_groups: cap at the largest 8-CTA slice

_lib = None
_lock = threading.Lock()


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("prec", ctypes.c_int), ("eos", ctypes.c_int),
                ("force", ctypes.c_int), ("grad", ctypes.c_int), ("hdm_radius", ctypes.c_int),
                ("flags", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("R", ctypes.c_double), ("omega", ctypes.c_double), ("Tr", ctypes.c_double),
                ("Tc", ctypes.c_double), ("k", ctypes.c_double), ("tau", ctypes.c_double),
                ("G", ctypes.c_double), ("rho0", ctypes.c_double), ("stream", ctypes.c_void_p)]


class _Obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("mom_x", ctypes.c_double), ("mom_y", ctypes.c_double),
                ("max_speed", ctypes.c_double), ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double)]


class _Timing(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("launches", ctypes.c_longlong),
                ("ms_kernel", ctypes.c_double * 4), ("count_kernel", ctypes.c_longlong * 4)]


# kernel slots of lbm_timing
KERNEL_SLOTS = ("potential", "collide", "fused_step", "unused")

# name -> (restype, argtypes) of every entry point declared in include/lbm.h
_D = ctypes.POINTER(ctypes.c_double)
_V = ctypes.c_void_p
SIGNATURES = {
    "lbm_critical_point": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]),
    "lbm_hdm_weights": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(_Params), ctypes.POINTER(_V)]),
    "lbm_init_density": (ctypes.c_int, [_V, _D, _D, _D]),
    "lbm_init_density_device": (ctypes.c_int, [_V, _V, _V, _V]),
    "lbm_set_f": (ctypes.c_int, [_V, _D]),
    "lbm_get_f": (ctypes.c_int, [_V, _D]),
    "lbm_step": (ctypes.c_int, [_V, ctypes.c_int]),
    "lbm_sync": (ctypes.c_int, [_V]),
    "lbm_moments": (ctypes.c_int, [_V, _D, _D, _D]),
    "lbm_moments_device": (ctypes.c_int, [_V, _V, _V, _V]),
    "lbm_observables": (ctypes.c_int, [_V, ctypes.POINTER(_Obs)]),
    "lbm_set_timing": (ctypes.c_int, [_V, ctypes.c_int]),
    "lbm_get_timing": (ctypes.c_int, [_V, ctypes.POINTER(_Timing)]),
    "lbm_step_noalloc": (ctypes.c_int, [ctypes.POINTER(_Params), _V, _V]),
    "lbm_maxwell": (ctypes.c_int, [ctypes.POINTER(_Params), _D, _D]),
    "lbm_adjoint_forward": (ctypes.c_int, [_V, _V, ctypes.c_int, ctypes.c_int, _V]),
    "lbm_set_segment_rows": (ctypes.c_int, [_V, ctypes.c_int]),
    "lbm_get_segment_rows": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int)]),
    "lbm_tune_segment_rows": (ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lbm_gradient": (ctypes.c_int, [_V, _D, ctypes.c_double, _D, _D]),
    "lbm_adjoint_backward": (ctypes.c_int, [_V, _V, _V, _D, _D, _D]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(_Params), ctypes.c_int, ctypes.POINTER(_V)]),
    "lbm_batch_init_density": (ctypes.c_int, [_V, _D]),
    "lbm_batch_set_f": (ctypes.c_int, [_V, _D]),
    "lbm_batch_get_f": (ctypes.c_int, [_V, _D]),
    "lbm_batch_step": (ctypes.c_int, [_V, ctypes.c_int]),
    "lbm_batch_sync": (ctypes.c_int, [_V]),
    "lbm_batch_density": (ctypes.c_int, [_V, _D]),
    "lbm_batch_moments": (ctypes.c_int, [_V, _D, _D, _D]),
    "lbm_batch_set_launch": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_get_launch": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_set_cluster": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_get_cluster": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_set_groups": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_get_groups": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_tune": (ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_debug_skip_barrier": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_V]),
    "lbm_batch_destroy": (None, [_V]),
    "lbm_debug_alloc_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_debug_check_canaries": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_destroy": (None, [_V]),
    "lbm_last_error": (ctypes.c_char_p, [_V]),
    "lbm_host_in_place": (ctypes.c_int, [_V]),
    "lbm_save": (ctypes.c_int, [_V, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_V, ctypes.c_char_p]),
}


def library_path() -> str:
    """The library this process loads: ``_build/liblbm.so``, or the
    bounds-checked build when the environment sets LBM_CHECKED=1 (tests)."""
    return _build.LIB_CHECKED if os.environ.get("LBM_CHECKED") == "1" else _build.LIB


def load():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_1712_06079_gb300.build.build() "
                                   "(or __graft_entry__.build()); there is no CPU fallback")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def alloc_stats():
    """(live device allocations, live pinned host allocations) of the library."""
    d, h = ctypes.c_longlong(), ctypes.c_longlong()
    st = load().lbm_debug_alloc_stats(ctypes.byref(d), ctypes.byref(h))
    if st != OK:
        raise LBMError(st, "lbm_debug_alloc_stats failed")
    return d.value, h.value


def damaged_canaries() -> int:
    """Device allocations whose canary (the bytes past their end, in the
    bounds-checked build) was overwritten; -1 in the normal build."""
    n = ctypes.c_longlong()
    st = load().lbm_debug_check_canaries(ctypes.byref(n))
    if st != OK:
        raise LBMError(st, "lbm_debug_check_canaries failed")
    return n.value


def critical_point(eos: str, a: float, b: float, R: float = 1.0):
    Tc, rc = ctypes.c_double(), ctypes.c_double()
    st = load().lbm_critical_point(EOS[eos], a, b, R, ctypes.byref(Tc), ctypes.byref(rc))
    if st != OK:
        raise LBMError(st, "lbm_critical_point failed")
    return Tc.value, rc.value


def step_noalloc(params: "Params", f_in_ptr: int, f_out_ptr: int) -> int:
    """One step from device array f_in to device array f_out through
    lbm_step_noalloc (no device allocation; see include/lbm.h).  Returns the
    lbm_status code."""
    return load().lbm_step_noalloc(ctypes.byref(params.c()), f_in_ptr, f_out_ptr)


def maxwell(params: "Params"):
    """(rho_g, rho_l) of the Maxwell construction for params' EOS at params.Tr."""
    g, l = ctypes.c_double(), ctypes.c_double()
    st = load().lbm_maxwell(ctypes.byref(params.c()), ctypes.byref(g), ctypes.byref(l))
    if st != OK:
        raise LBMError(st, "lbm_maxwell failed (no van der Waals loop?)")
    return g.value, l.value


def hdm_weights(n: int, radius: int):
    w = np.zeros(radius + 1)
    k = ctypes.c_int()
    st = load().lbm_hdm_weights(n, radius, _dp(w), ctypes.byref(k))
    if st != OK:
        raise LBMError(st, "lbm_hdm_weights failed")
    return w, k.value


@dataclasses.dataclass
class Params:
    nx: int
    ny: int
    eos: str = "cs"
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    omega: float = 0.0
    Tr: float = 0.8
    Tc: float = 0.0
    k: float = 1.0
    tau: float = 1.0
    force: str = "sc"
    grad: str = "hdm"
    prec: str = "f32"
    hdm_radius: int = 0
    two_pass: bool = False  # LBM_FLAG_TWO_PASS: never use the single-pass FP32 kernel
    walls: bool = False     # LBM_FLAG_WALLS_Y: no-slip walls below row 0 and above row ny-1
    f32_arith: bool = False  # LBM_FLAG_F32_ARITH: FP32 arithmetic in the two-pass kernels of an FP32 lattice
    staged_host: bool = False  # LBM_FLAG_STAGED_HOST: host arrays through the pinned staging buffer
    G: float = 0.0     # eos "psi_exp": interaction strength of Eq. 4
    rho0: float = 1.0  # eos "psi_exp": reference density of psi = 1 - exp(-rho/rho0)
    stream: int = 0  # cudaStream_t as an integer (torch.cuda.Stream.cuda_stream), 0 = default

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, PREC[self.prec], EOS[self.eos], FORCE[self.force], GRAD[self.grad],
                       self.hdm_radius,
                       (FLAG_TWO_PASS if self.two_pass else 0) | (FLAG_WALLS_Y if self.walls else 0) |
                       (FLAG_F32_ARITH if self.f32_arith else 0) | (FLAG_STAGED_HOST if self.staged_host else 0),
                       self.a, self.b, self.R, self.omega, self.Tr, self.Tc, self.k,
                       self.tau, self.G, self.rho0, ctypes.c_void_p(self.stream or None))


class Lattice:
    """One periodic D2Q9 lattice behind an ``lbm_ctx``."""

    def __init__(self, params: Params):
        self.params = params
        self._lib = load()
        h = ctypes.c_void_p()
        st = self._lib.lbm_create(ctypes.byref(params.c()), ctypes.byref(h))
        if st != OK:
            raise LBMError(st, self._lib.lbm_last_error(None).decode())
        self._h = h
        self.shape = (params.ny, params.nx)
        self.dtype = np.float64 if params.prec == "f64" else np.float32

    def _check(self, st: int):
        if st != OK:
            raise LBMError(st, self._lib.lbm_last_error(self._h).decode())

    @property
    def handle(self) -> int:
        return self._h.value

    def init_density(self, rho, ux=None, uy=None):
        c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
        rho, ux, uy = c(rho), c(ux), c(uy)
        self._check(self._lib.lbm_init_density(self._h, _dp(rho), _dp(ux), _dp(uy)))

    def init_density_device(self, rho_ptr: int, ux_ptr: int = 0, uy_ptr: int = 0):
        self._check(self._lib.lbm_init_density_device(self._h, rho_ptr or None, ux_ptr or None, uy_ptr or None))

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((9,) + self.shape)
        self._check(self._lib.lbm_set_f(self._h, _dp(f)))

    def get_f(self) -> np.ndarray:
        f = np.empty((9,) + self.shape)
        self._check(self._lib.lbm_get_f(self._h, _dp(f)))
        return f

    def step(self, n: int = 1):
        self._check(self._lib.lbm_step(self._h, int(n)))

    def sync(self):
        self._check(self._lib.lbm_sync(self._h))

    def moments(self, out=None):
        """(rho, vx, vy) as FP64 host arrays; ``out``: three C-contiguous FP64
        arrays of the lattice's shape to write into (reused buffers spare the
        page population of fresh ones)."""
        if out is None:
            out = tuple(np.empty(self.shape) for _ in range(3))
        elif len(out) != 3 or any(not isinstance(o, np.ndarray) or o.dtype != np.float64 or o.shape != self.shape
                                  or not o.flags.c_contiguous or not o.flags.writeable for o in out):
            raise ValueError(f"out must be three writeable C-contiguous float64 arrays of shape {self.shape}")
        r, vx, vy = out
        self._check(self._lib.lbm_moments(self._h, _dp(r), _dp(vx), _dp(vy)))
        return r, vx, vy

    def save(self, path):
        """Write the current state (and the single-pass kernel's stencil field) to a file."""
        self._check(self._lib.lbm_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Resume from a file written by save() (same nx, ny and precision)."""
        self._check(self._lib.lbm_load(self._h, os.fsencode(path)))

    def host_in_place(self) -> bool:
        """True if the device reads and writes this context's host arrays in place
        where it can (results: into arrays whose pages are all resident)."""
        return self._lib.lbm_host_in_place(self._h) == 1

    def moments_device(self, rho_ptr: int, vx_ptr: int, vy_ptr: int):
        self._check(self._lib.lbm_moments_device(self._h, rho_ptr, vx_ptr, vy_ptr))

    def gradient(self, q, h: float = 1.0):
        """The context's gradient operator (HDM Eq. 20 or CDM Eq. 15) of a (ny, nx)
        field on a grid of spacing h: returns (d/dx, d/dy) as FP64 arrays."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        if q.shape != self.shape:
            raise ValueError(f"q must have shape {self.shape}")
        gx, gy = np.empty(self.shape), np.empty(self.shape)
        self._check(self._lib.lbm_gradient(self._h, _dp(q), float(h), _dp(gx), _dp(gy)))
        return gx, gy

    def observables(self) -> dict:
        o = _Obs()
        self._check(self._lib.lbm_observables(self._h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in _Obs._fields_}

    def set_segment_rows(self, rows: int):
        """Rows per CTA segment of the single-pass FP32 step (0: automatic)."""
        self._check(self._lib.lbm_set_segment_rows(self._h, int(rows)))

    def segment_rows(self) -> int:
        r = ctypes.c_int()
        self._check(self._lib.lbm_get_segment_rows(self._h, ctypes.byref(r)))
        return r.value

    def tune_segment_rows(self, trials: int = 3) -> int:
        """Time the single-pass step at every segment height 8k - 2 on the current
        state (which is kept), keep the fastest and return it (0: two-pass step)."""
        r = ctypes.c_int()
        self._check(self._lib.lbm_tune_segment_rows(self._h, int(trials), ctypes.byref(r)))
        return r.value

    def adjoint_forward(self, rho0_ptr: int, nsteps: int, checkpoint_interval: int, rhoT_ptr: int):
        self._check(self._lib.lbm_adjoint_forward(self._h, rho0_ptr, int(nsteps), int(checkpoint_interval), rhoT_ptr))

    def adjoint_backward(self, grad_rhoT_ptr: int, grad_rho0_ptr: int):
        """Writes dL/drho0 and returns (dL/dT, dL/d(T/Tc), dL/dG)."""
        gT, gTr, gG = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm_adjoint_backward(self._h, grad_rhoT_ptr, grad_rho0_ptr, ctypes.byref(gT),
                                                   ctypes.byref(gTr), ctypes.byref(gG)))
        return gT.value, gTr.value, gG.value

    def set_timing(self, enable: bool):
        self._check(self._lib.lbm_set_timing(self._h, 1 if enable else 0))

    def timing(self) -> dict:
        t = _Timing()
        self._check(self._lib.lbm_get_timing(self._h, ctypes.byref(t)))
        return {"steps": t.steps, "launches": t.launches,
                "kernels": {KERNEL_SLOTS[i]: {"ms": t.ms_kernel[i], "count": t.count_kernel[i]}
                            for i in range(4) if t.count_kernel[i]}}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent lattices advanced together (``lbm_batch``): one
    persistent launch per ``step`` call, replayed from a CUDA graph."""

    def __init__(self, params: list):
        self._lib = load()
        self.params = list(params)
        arr = (_Params * len(self.params))(*[p.c() for p in self.params])
        h = ctypes.c_void_p()
        st = self._lib.lbm_batch_create(arr, len(self.params), ctypes.byref(h))
        if st != OK:
            raise LBMError(st, "lbm_batch_create failed")
        self._h = h
        self.shapes = [(p.ny, p.nx) for p in self.params]
        self.cells = [p.nx * p.ny for p in self.params]

    def _check(self, st: int):
        if st != OK:
            raise LBMError(st, self._lib.lbm_batch_last_error(self._h).decode())

    def _split(self, flat, per):
        out, o = [], 0
        for n, shp in zip(self.cells, self.shapes):
            out.append(flat[o:o + per * n].reshape((per,) + shp if per > 1 else shp))
            o += per * n
        return out

    def init_density(self, rhos: list):
        flat = np.ascontiguousarray(np.concatenate([np.asarray(r, dtype=np.float64).ravel() for r in rhos]))
        self._check(self._lib.lbm_batch_init_density(self._h, _dp(flat)))

    def set_f(self, fs: list):
        flat = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in fs]))
        self._check(self._lib.lbm_batch_set_f(self._h, _dp(flat)))

    def get_f(self) -> list:
        flat = np.empty(9 * sum(self.cells))
        self._check(self._lib.lbm_batch_get_f(self._h, _dp(flat)))
        return self._split(flat, 9)

    def step(self, n: int = 1):
        self._check(self._lib.lbm_batch_step(self._h, int(n)))

    def sync(self):
        self._check(self._lib.lbm_batch_sync(self._h))

    def density(self) -> list:
        flat = np.empty(sum(self.cells))
        self._check(self._lib.lbm_batch_density(self._h, _dp(flat)))
        return self._split(flat, 1)

    def moments(self) -> tuple:
        """(rho, vx, vy) per instance: density and the Eq. 11 velocity."""
        out = [np.empty(sum(self.cells)) for _ in range(3)]
        self._check(self._lib.lbm_batch_moments(self._h, *(_dp(a) for a in out)))
        return tuple(self._split(a, 1) for a in out)

    def set_launch(self, block_threads: int, blocks_per_sm: int):
        self._check(self._lib.lbm_batch_set_launch(self._h, block_threads, blocks_per_sm))

    def launch(self):
        t, g = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.lbm_batch_get_launch(self._h, ctypes.byref(t), ctypes.byref(g)))
        return t.value, g.value

    def set_cluster(self, cluster: int, block_threads: int = 256):
        """One cluster of ``cluster`` CTAs per instance, state in shared memory
        (``cluster = 0``: the grid form)."""
        self._check(self._lib.lbm_batch_set_cluster(self._h, int(cluster), int(block_threads)))

    def cluster(self) -> int:
        """0: grid form; 2, 4, 8: the cluster form's cluster size; -1: grouped."""
        c = ctypes.c_int()
        self._check(self._lib.lbm_batch_get_cluster(self._h, ctypes.byref(c)))
        return c.value

    def set_groups(self, max_smem_bytes: int = GROUPS_BALANCED, block_threads: int = 1024):
        """Grouped cluster form: each instance on the smallest cluster (2, 4, 8)
        whose slices fit ``max_smem_bytes`` of shared memory (0: the opt-in
        maximum; GROUPS_BALANCED: the largest 8-CTA slice's), one launch per
        cluster size on its own stream."""
        self._check(self._lib.lbm_batch_set_groups(self._h, int(max_smem_bytes), int(block_threads)))

    def groups(self, smem: bool = False):
        """[(cluster size, instance count)] of the grouped form ([] otherwise),
        with the shared memory per CTA as a third entry when ``smem``."""
        n = ctypes.c_int()
        cl = (ctypes.c_int * 3)()
        ct = (ctypes.c_int * 3)()
        sm = (ctypes.c_int * 3)()
        self._check(self._lib.lbm_batch_get_groups(self._h, ctypes.byref(n), cl, ct, sm))
        return [(cl[g], ct[g], sm[g]) if smem else (cl[g], ct[g]) for g in range(n.value)]

    def tune(self, trial_steps: int = 50):
        t, g = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.lbm_batch_tune(self._h, int(trial_steps), ctypes.byref(t), ctypes.byref(g)))
        return t.value, g.value

    def debug_skip_barrier(self, block: int, limit_seconds: float):
        self._check(self._lib.lbm_batch_debug_skip_barrier(self._h, int(block), float(limit_seconds)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lbm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
