"""FP64 CPU oracle for the phase-field LB freezing step (arXiv 2403.16122).

TEST INFRASTRUCTURE. This package wraps ``lbm_oracle.c``, a plain, slow
restatement of the paper's scheme (Sections 2-3) in double precision. Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the CUDA library never links or calls it, and it
imports nothing from the CUDA side.

Arrays use the lattice layout ``[..., ny, nx]`` (site (x, y) at ``[y, x]``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

OBS_NAMES = (
    "volume", "solid", "enthalpy", "mass", "condensed_mass", "mdot",
    "phi_mdot", "solid_col", "solid_row", "umax", "nonfinite",
)
FIELD_NAMES = ("phi", "H", "T", "fs", "mdot", "rho", "ux", "uy", "p", "S")
DERIVED_NAMES = (
    "L", "Hs", "Hl", "tau_g", "kappa", "beta", "rho_g", "rho_s", "mu_l",
    "mu_g", "mu_s", "tan_w",
)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction), with
    OpenMP over the lattice rows of the site loops when the compiler has it
    (the thread count changes no value: every site's result depends only on
    the previous state)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(__file__))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("dirichlet_x_lo", ctypes.c_int32), ("dirichlet_x_hi", ctypes.c_int32),
        ("dirichlet_y_lo", ctypes.c_int32), ("dirichlet_y_hi", ctypes.c_int32),
        ("st_mask_liquid", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("W", ctypes.c_double), ("sigma", ctypes.c_double),
        ("mobility", ctypes.c_double), ("tau_f_liquid", ctypes.c_double),
        ("tau_h", ctypes.c_double), ("rho_l", ctypes.c_double),
        ("rho_ratio_lg", ctypes.c_double), ("rho_ratio_sl", ctypes.c_double),
        ("mu_ratio_lg", ctypes.c_double), ("Ste", ctypes.c_double),
        ("Cp", ctypes.c_double), ("Cp_ref", ctypes.c_double),
        ("T_m", ctypes.c_double), ("T_w", ctypes.c_double),
        ("theta_deg", ctypes.c_double), ("pc_ramp", ctypes.c_double),
        ("normal_eps", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("beta_T", ctypes.c_double), ("T_ref", ctypes.c_double),
        ("rho_0", ctypes.c_double),
        ("Cp_ratio_sl", ctypes.c_double), ("Cp_ratio_gl", ctypes.c_double),
        ("k_ratio_sl", ctypes.c_double), ("k_ratio_gl", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        vp = ctypes.c_void_p
        dp = P(d)
        lib.oracle_create.argtypes = [P(OracleParams), P(vp)]
        lib.oracle_create.restype = ctypes.c_int
        lib.oracle_destroy.argtypes = [vp]
        lib.oracle_init.argtypes = [vp, dp, dp]
        lib.oracle_step.argtypes = [vp, i64]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        lib.oracle_mdot_integral.argtypes = [vp]
        lib.oracle_mdot_integral.restype = d
        lib.oracle_step_count.argtypes = [vp]
        lib.oracle_step_count.restype = i64
        lib.oracle_get_state.argtypes = [vp, dp, dp]
        lib.oracle_set_state.argtypes = [vp, dp, dp]
        lib.oracle_fields.argtypes = [vp, dp]
        lib.oracle_observables.argtypes = [vp, dp]
        lib.oracle_derived.argtypes = [vp, dp]
        lib.oracle_lattice.argtypes = [P(i32), P(i32), dp, P(i32)]
        lib.oracle_geq.argtypes = [d, d, d, dp]
        lib.oracle_heq.argtypes = [d, d, d, d, d, d, dp]
        lib.oracle_feq.argtypes = [d, d, d, d, dp]
        lib.oracle_force_F.argtypes = [d, d, d, d, d, d, d, dp]
        lib.oracle_source_G.argtypes = [d, d, d, d, d, d, d, dp]
        lib.oracle_closure.argtypes = [vp, d, d, dp, dp]
        lib.oracle_stencil.argtypes = [vp, dp, i32, i32, i32, dp, dp, dp]
        lib.oracle_ghost.argtypes = [vp, dp, i32, i32, i32]
        lib.oracle_ghost.restype = d
        _lib = lib
        return lib


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's site loops (n > 0 sets them); returns the
    count in effect (1 when built without OpenMP)."""
    return int(_load().oracle_set_threads(int(n)))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(cfg: dict) -> OracleParams:
    p = OracleParams()
    for name, _ in OracleParams._fields_:
        if name == "reserved":
            continue
        setattr(p, name, cfg[name])
    return p


def lattice():
    """D2Q9 tables of the oracle: (cx, cy, w, opp)."""
    lib = _load()
    cx = (ctypes.c_int32 * 9)()
    cy = (ctypes.c_int32 * 9)()
    w = (ctypes.c_double * 9)()
    opp = (ctypes.c_int32 * 9)()
    lib.oracle_lattice(cx, cy, w, opp)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:]))


def _call9(fn, *args):
    out = np.zeros(9)
    fn(*[float(a) for a in args], _dptr(out))
    return out


def geq(phi, ux, uy):
    return _call9(_load().oracle_geq, phi, ux, uy)


def heq(H, T, Cp, Cp_ref, ux, uy):
    return _call9(_load().oracle_heq, H, T, Cp, Cp_ref, ux, uy)


def feq(p, rho, ux, uy):
    return _call9(_load().oracle_feq, p, rho, ux, uy)


def force_F(S, fx, fy, ux, uy, Ftx, Fty):
    return _call9(_load().oracle_force_F, S, fx, fy, ux, uy, Ftx, Fty)


def source_G(phi, mdot, dtx, dty, lam, nx, ny):
    return _call9(_load().oracle_source_G, phi, mdot, dtx, dty, lam, nx, ny)


class OracleError(RuntimeError):
    pass


class Oracle:
    """One lattice advanced by the FP64 oracle."""

    def __init__(self, cfg: dict):
        self._lib = _load()
        self.cfg = dict(cfg)
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self._p = _params(cfg)
        h = ctypes.c_void_p()
        rc = self._lib.oracle_create(ctypes.byref(self._p), ctypes.byref(h))
        if rc != 0:
            raise OracleError(f"oracle_create failed ({rc}): invalid parameters" if rc == -1
                              else f"oracle_create failed ({rc})")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.ny, self.nx)

    def _grid(self, a) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != self.shape:
            raise ValueError(f"expected shape {self.shape}, got {a.shape}")
        return a

    def init(self, phi0, T0):
        phi0, T0 = self._grid(phi0), self._grid(T0)
        self._lib.oracle_init(self._h, _dptr(phi0), _dptr(T0))
        return self

    def step(self, n: int = 1):
        self._lib.oracle_step(self._h, int(n))
        return self

    @property
    def step_count(self) -> int:
        return int(self._lib.oracle_step_count(self._h))

    @property
    def mdot_integral(self) -> float:
        """Sum of mdot over every step since init/set_state and every site."""
        return float(self._lib.oracle_mdot_integral(self._h))

    def solid_profile(self):
        """Sum over y of f_s per column (the frozen shape seen from a wall
        below), from the last step's fields."""
        return self.fields()["fs"].sum(axis=0)

    def get_state(self):
        pops = np.zeros((27, self.ny, self.nx))
        aux = np.zeros((5, self.ny, self.nx))
        self._lib.oracle_get_state(self._h, _dptr(pops), _dptr(aux))
        return pops, aux

    def set_state(self, pops, aux):
        pops = np.ascontiguousarray(np.asarray(pops, dtype=np.float64)).reshape(27, self.ny, self.nx)
        aux = np.ascontiguousarray(np.asarray(aux, dtype=np.float64)).reshape(5, self.ny, self.nx)
        self._lib.oracle_set_state(self._h, _dptr(pops), _dptr(aux))
        return self

    def fields(self) -> dict:
        out = np.zeros((len(FIELD_NAMES), self.ny, self.nx))
        self._lib.oracle_fields(self._h, _dptr(out))
        return {k: out[j] for j, k in enumerate(FIELD_NAMES)}

    def observables(self) -> dict:
        out = np.zeros(len(OBS_NAMES))
        self._lib.oracle_observables(self._h, _dptr(out))
        return {k: float(out[j]) for j, k in enumerate(OBS_NAMES)}

    def derived(self) -> dict:
        out = np.zeros(len(DERIVED_NAMES))
        self._lib.oracle_derived(self._h, _dptr(out))
        return {k: float(out[j]) for j, k in enumerate(DERIVED_NAMES)}

    def closure(self, H, phihat):
        fs = ctypes.c_double()
        T = ctypes.c_double()
        self._lib.oracle_closure(self._h, float(H), float(phihat),
                                 ctypes.byref(fs), ctypes.byref(T))
        return fs.value, T.value

    def stencil(self, field, x, y, kind=0):
        field = self._grid(field)
        gx, gy, lap = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._lib.oracle_stencil(self._h, _dptr(field), int(x), int(y), int(kind),
                                 ctypes.byref(gx), ctypes.byref(gy), ctypes.byref(lap))
        return gx.value, gy.value, lap.value

    def ghost(self, field, x, y, kind=0):
        field = self._grid(field)
        return float(self._lib.oracle_ghost(self._h, _dptr(field), int(x), int(y), int(kind)))
