"""FP64 CPU oracle for the Oregonator reaction-diffusion step (Eq. 1, §2).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and this package imports nothing from the product package.

The arithmetic lives in ``rdc_oracle.c`` (plain C, FP64, compiled with
``-O2 -ffp-contract=off``).  This module compiles it with gcc on first use
and wraps it with ctypes and NumPy.

Parity status of the functions (what pins each one is in ``tests/``):
  * rest_state / rest_field  -- pinned (cubic roots, fixed point of the step)
  * step / run               -- pinned (cosine eigenmodes, conservation,
                                analytic Jacobian, symmetries, 1-D reduction,
                                AND-gate and diode behaviour of §4)
  * seed_disk                -- pinned (Gauss circle counts)
  * draw_line / snap_segment -- pinned (line widths of the §3 presets, end
                                caps, snapped angles and preserved length)
  * render / timelapse       -- pinned (channel assignment of §3.1, clamping,
                                round-half-even codes, the green threshold's
                                edge, running maximum and its reset)
  * arrival times in run     -- pinned by brute force (the recorded crossing
                                of theta and its linear interpolation equal
                                those of separate runs to the two steps
                                around it); the paper prints no wave speeds or
                                arrival times to compare the values with.
  * round_stoch              -- pinned (exact unbiasedness over all 2^16
                                random values, both neighbours on the target
                                grid, round-to-nearest cases)
  * round_stoch_cells        -- pinned by properties (every counter field and
                                the key change the draws, u and v and the
                                cells of a quad draw different bits, position
                                independence, unbiasedness over steps); which
                                half-word goes to u is a convention
  * philox4x32_10            -- pinned (the published known-answer vectors
                                of Philox4x32-10; bijectivity in each counter
                                word, avalanche and uniformity of the output
                                bits)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rdc_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

# Table 1 of the paper.
EPS = 0.0243
F = 1.4
PHI_ACTIVE = 0.054
PHI_PASSIVE = 0.0975
Q = 0.002
DU = 0.45
DT = 0.001
DX = 0.25

DIFFUSION_ONLY = 1
REACTION_ONLY = 2

OK = 0
EINVAL = 1
ENOMEM = 2
ENONFINITE = 4

GCC_FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
             "-shared", "-fPIC"]


class _OrcParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("f", ctypes.c_double),
                ("q", ctypes.c_double), ("Du", ctypes.c_double),
                ("dt", ctypes.c_double), ("dx", ctypes.c_double),
                ("flags", ctypes.c_int32), ("pad_", ctypes.c_int32)]


@dataclasses.dataclass
class Params:
    """Model parameters; defaults are Table 1."""
    eps: float = EPS
    f: float = F
    q: float = Q
    Du: float = DU
    dt: float = DT
    dx: float = DX
    flags: int = 0

    def _c(self) -> _OrcParams:
        return _OrcParams(self.eps, self.f, self.q, self.Du, self.dt, self.dx,
                          int(self.flags), 0)


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH,
                   openmp: bool = True, extra: list[str] | None = None) -> str:
    """Compiles ``src`` into a shared library at ``out`` and returns the path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    flags = list(GCC_FLAGS)
    if openmp:
        flags.append("-fopenmp")
    if extra:
        flags += extra
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *flags, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def _stale(lib: str, src: str) -> bool:
    return (not os.path.exists(lib)) or os.path.getmtime(lib) < os.path.getmtime(src)


_LOCK = threading.Lock()
_DEFAULT: "Oracle | None" = None


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """ctypes wrapper around one compiled copy of the oracle."""

    def __init__(self, lib_path: str):
        self.path = lib_path
        lib = ctypes.CDLL(lib_path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_rest_state.argtypes = [ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, dp]
        lib.orc_rest_state.restype = ctypes.c_int
        lib.orc_rest_field.argtypes = [ctypes.c_int64, dp, ctypes.c_double,
                                       ctypes.c_double, dp, dp]
        lib.orc_rest_field.restype = ctypes.c_int
        lib.orc_seed_disk.argtypes = [ctypes.c_int32, ctypes.c_int32, dp,
                                      ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]
        lib.orc_seed_disk.restype = ctypes.c_int64
        lib.orc_step.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                 ctypes.POINTER(_OrcParams), dp, dp, dp, dp,
                                 dp, ctypes.c_int32, i64p]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_run.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(_OrcParams), dp, dp, dp,
                                ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                i64p, ctypes.c_double, dp, i64p, i64p]
        lib.orc_run.restype = ctypes.c_int
        fp = ctypes.POINTER(ctypes.c_float)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.orc_render.argtypes = [ctypes.c_int64, fp, fp, dp, fp, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_double, u8p]
        lib.orc_render.restype = None
        lib.orc_timelapse.argtypes = [ctypes.c_int64, fp, fp, ctypes.c_int32]
        lib.orc_timelapse.restype = None
        lib.orc_snap_segment.argtypes = [ctypes.c_double] * 5 + [dp, dp]
        lib.orc_snap_segment.restype = ctypes.c_int
        lib.orc_draw_line.argtypes = [ctypes.c_int32, ctypes.c_int32, dp] + [ctypes.c_double] * 6
        lib.orc_draw_line.restype = ctypes.c_int64
        lib.orc_max_threads.argtypes = []
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_round_stoch.argtypes = [ctypes.c_float, ctypes.c_uint32, ctypes.c_int32]
        lib.orc_round_stoch.restype = ctypes.c_float
        fp = ctypes.POINTER(ctypes.c_float)
        lib.orc_round_stoch_cells.argtypes = [ctypes.c_int64, fp, ctypes.c_uint32, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              fp, fp]
        lib.orc_round_stoch_cells.restype = None
        lib.orc_max_threads.restype = ctypes.c_int32
        self.lib = lib

    # -- rest state ---------------------------------------------------------
    def rest_state(self, phi: float, f: float = F, q: float = Q) -> float:
        out = ctypes.c_double()
        rc = self.lib.orc_rest_state(phi, f, q, ctypes.byref(out))
        if rc != OK:
            raise ValueError(f"no positive rest state for phi={phi}, f={f}, q={q}")
        return out.value

    def rest_field(self, phi: np.ndarray, f: float = F, q: float = Q):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        u = np.empty_like(phi)
        v = np.empty_like(phi)
        rc = self.lib.orc_rest_field(phi.size, _dptr(phi), f, q, _dptr(u), _dptr(v))
        if rc != OK:
            raise ValueError("rest_field: invalid phi / f / q")
        return u, v

    # -- stimulation --------------------------------------------------------
    def seed_disk(self, u: np.ndarray, cx: float, cy: float, r: float,
                  value: float) -> int:
        """In place: u := value inside the disk; returns the cell count."""
        assert u.dtype == np.float64 and u.flags.c_contiguous and u.ndim == 2
        H, W = u.shape
        n = self.lib.orc_seed_disk(W, H, _dptr(u), cx, cy, r, value)
        if n < 0:
            raise ValueError("seed_disk: invalid arguments")
        return int(n)

    # -- stepping -----------------------------------------------------------
    def step(self, phi, u, v, params: Params | None = None, nthreads: int = 1):
        """One Euler step; returns (u1, v1, status, bad_index)."""
        params = params or Params()
        phi, u, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (phi, u, v))
        H, W = u.shape
        u1 = np.empty_like(u)
        v1 = np.empty_like(v)
        bad = ctypes.c_int64(-1)
        cp = params._c()
        rc = self.lib.orc_step(W, H, ctypes.byref(cp), _dptr(phi), _dptr(u),
                               _dptr(v), _dptr(u1), _dptr(v1), nthreads,
                               ctypes.byref(bad))
        if rc == EINVAL:
            raise ValueError("orc_step: invalid arguments")
        return u1, v1, rc, bad.value

    def run(self, phi, u, v, nsteps: int, params: Params | None = None,
            nthreads: int = 1, probes=None, theta: float = 0.3):
        """nsteps Euler steps on copies of (u, v).

        Returns a dict with u, v, status, bad_step, bad_index and (when
        probes are given, as flat cell indices) t_arr in steps.
        """
        params = params or Params()
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        u = np.array(u, dtype=np.float64, order="C", copy=True)
        v = np.array(v, dtype=np.float64, order="C", copy=True)
        H, W = u.shape
        if probes is None:
            pr = np.zeros(0, dtype=np.int64)
        else:
            pr = np.ascontiguousarray(probes, dtype=np.int64)
        t_arr = np.full(max(len(pr), 1), -1.0)
        bs = ctypes.c_int64(-1)
        bi = ctypes.c_int64(-1)
        cp = params._c()
        rc = self.lib.orc_run(W, H, ctypes.byref(cp), _dptr(phi), _dptr(u),
                              _dptr(v), int(nsteps), int(nthreads), len(pr),
                              pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              float(theta), _dptr(t_arr), ctypes.byref(bs),
                              ctypes.byref(bi))
        if rc == EINVAL:
            raise ValueError("orc_run: invalid arguments")
        if rc == ENOMEM:
            raise MemoryError("orc_run: out of memory")
        return {"u": u, "v": v, "status": rc, "bad_step": bs.value,
                "bad_index": bi.value, "t_arr": t_arr[:len(pr)]}

    # -- drawing (§3) -----------------------------------------------------------
    def snap_segment(self, x0, y0, x1, y1, snap=15.0):
        a = ctypes.c_double()
        b = ctypes.c_double()
        rc = self.lib.orc_snap_segment(x0, y0, x1, y1, snap, ctypes.byref(a), ctypes.byref(b))
        if rc != OK:
            raise ValueError("snap_segment: invalid arguments")
        return a.value, b.value

    def draw_line(self, phi, x0, y0, x1, y1, width, value, snap=0.0):
        """In place on a float64 H x W map; returns the number of cells set."""
        assert phi.dtype == np.float64 and phi.flags.c_contiguous
        if snap > 0:
            x1, y1 = self.snap_segment(x0, y0, x1, y1, snap)
        H, W = phi.shape
        return int(self.lib.orc_draw_line(W, H, _dptr(phi), x0, y0, x1, y1, width, value))

    # -- outputs (§3.1) --------------------------------------------------------
    def render(self, u, v, phi, u_scale=1.0, v_scale=1.0, thr=0.07575, tl=None):
        """RGBA8 image (H, W, 4) of float32 u, v (or of the timelapse tl)."""
        fp = ctypes.POINTER(ctypes.c_float)
        u = np.ascontiguousarray(u, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        H, W = u.shape
        out = np.empty((H, W, 4), dtype=np.uint8)
        tlp = None
        if tl is not None:
            tl = np.ascontiguousarray(tl, dtype=np.float32)
            tlp = tl.ctypes.data_as(fp)
        self.lib.orc_render(u.size, u.ctypes.data_as(fp), v.ctypes.data_as(fp), _dptr(phi), tlp,
                            float(u_scale), float(v_scale), float(thr),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return out

    def timelapse(self, u, tl=None):
        """Returns the record updated with float32 u (a new record if tl is None)."""
        fp = ctypes.POINTER(ctypes.c_float)
        u = np.ascontiguousarray(u, dtype=np.float32)
        reset = tl is None
        tl = np.empty_like(u) if reset else np.array(tl, dtype=np.float32, copy=True)
        self.lib.orc_timelapse(u.size, u.ctypes.data_as(fp), tl.ctypes.data_as(fp), int(reset))
        return tl

    def max_threads(self) -> int:
        return int(self.lib.orc_max_threads())

    # -- stochastic rounding to 16-bit storage ---------------------------------
    def philox4x32_10(self, ctr, key):
        """Four 32-bit output words of Philox4x32-10 for counter ctr[4], key[2]."""
        u32p = ctypes.POINTER(ctypes.c_uint32)
        c = np.ascontiguousarray(ctr, dtype=np.uint32)
        k = np.ascontiguousarray(key, dtype=np.uint32)
        out = np.empty(4, dtype=np.uint32)
        self.lib.orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p),
                                   out.ctypes.data_as(u32p))
        return out

    def round_stoch(self, x: float, r16: int, fmt: str) -> float:
        """x (a float32 value) rounded stochastically to "bf16" or "f16" with
        the 16-bit random value r16; returned as a Python float."""
        return float(self.lib.orc_round_stoch(float(np.float32(x)), int(r16),
                                              0 if fmt == "bf16" else 1))

    def round_stoch_cells(self, x, seed: int, step: int, row: int, col0: int, fmt: str):
        """The rounding of the u and v of cells (col0 + i, row) writing state
        `step` with key `seed`; float32 arrays (u, v)."""
        fp = ctypes.POINTER(ctypes.c_float)
        x = np.ascontiguousarray(x, dtype=np.float32).ravel()
        u = np.empty_like(x)
        v = np.empty_like(x)
        self.lib.orc_round_stoch_cells(x.size, x.ctypes.data_as(fp), int(seed) & 0xFFFFFFFF,
                                       int(step), int(row), int(col0),
                                       0 if fmt == "bf16" else 1,
                                       u.ctypes.data_as(fp), v.ctypes.data_as(fp))
        return u, v


def load(force_rebuild: bool = False) -> Oracle:
    """Returns the default oracle, compiling it first when needed."""
    global _DEFAULT
    with _LOCK:
        if _DEFAULT is None or force_rebuild:
            if force_rebuild or _stale(_LIB_PATH, _SRC):
                compile_oracle()
            _DEFAULT = Oracle(_LIB_PATH)
        return _DEFAULT


def build() -> str:
    """Compiles the oracle library (used by the build entry point)."""
    return compile_oracle()
