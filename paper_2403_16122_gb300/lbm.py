"""ctypes binding of liblbmfreeze (include/lbm.h).

The functions ``lbm_*`` mirror the C-ABI one to one (argument marshalling
only); :class:`Lattice` is a convenience owner of a handle whose device
workspace is a torch uint8 tensor on the current CUDA device and whose stream
is torch's current stream. Every computation runs in the library's CUDA
kernels; there is no fallback: if the library is missing or no GPU is present
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "liblbmfreeze.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_EUNSTABLE, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
LBM_ETOOLARGE = -7
LBM_NOALLOC_MAX_TILES = 8192
LBM_STORE_FP32, LBM_STORE_FP16, LBM_STORE_BF16 = 0, 1, 2
OBS_NAMES = (
    "volume", "solid", "enthalpy", "mass", "condensed_mass", "mdot",
    "phi_mdot", "solid_col", "solid_row", "umax", "nonfinite",
)
LBM_OBS_COUNT = len(OBS_NAMES)
FRZ_NAMES = ("step", "mdot_integral", "freeze_step", "solid_fraction")
LBM_FRZ_COUNT = len(FRZ_NAMES)
LBM_FREEZE_FRACTION = 0.99


class lbm_params(ctypes.Structure):
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


class LbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lbm_error_string(code)} ({code})")
        self.code = code


_lib = None
_lock = threading.Lock()

# Exported C-ABI symbols (the set include/lbm.h declares).
SYMBOLS = (
    "lbm_workspace_size", "lbm_create", "lbm_init_fields", "lbm_step",
    "lbm_observables", "lbm_observables_all", "lbm_get_state", "lbm_set_state",
    "lbm_step_count", "lbm_launch_count", "lbm_destroy", "lbm_error_string",
    "lbm_set_kernel", "lbm_get_kernel", "lbm_autotune", "lbm_step_noalloc",
    "lbm_set_exec", "lbm_get_exec", "lbm_barrier_selftest", "lbm_set_thermal_walls",
    "lbm_freezing", "lbm_solid_profile",
)
LBM_KERNEL_TILE, LBM_KERNEL_STRIP, LBM_KERNEL_STAGED, LBM_KERNEL_BLOCK = 0, 1, 2, 3
LBM_EXEC_LAUNCH, LBM_EXEC_GRAPH, LBM_EXEC_PERSISTENT = 0, 1, 2


def load(path: str | None = None):
    """Load liblbmfreeze (raises OSError when it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"liblbmfreeze not built: {p} is missing "
                          "(run paper_2403_16122_gb300.build.build())")
        lib = ctypes.CDLL(p)
        P = ctypes.POINTER
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        dp = P(ctypes.c_double)
        lib.lbm_workspace_size.argtypes = [P(lbm_params), i32, i32, P(u64)]
        lib.lbm_create.argtypes = [P(lbm_params), i32, i32, vp, u64, vp, P(vp)]
        lib.lbm_init_fields.argtypes = [vp, i32, dp, dp]
        lib.lbm_step.argtypes = [vp, i64]
        lib.lbm_observables.argtypes = [vp, i32, dp]
        lib.lbm_observables_all.argtypes = [vp, dp]
        lib.lbm_get_state.argtypes = [vp, i32, dp, dp]
        lib.lbm_set_state.argtypes = [vp, i32, dp, dp]
        lib.lbm_step_count.argtypes = [vp]
        lib.lbm_step_count.restype = i64
        lib.lbm_launch_count.argtypes = [vp]
        lib.lbm_launch_count.restype = i64
        lib.lbm_destroy.argtypes = [vp]
        lib.lbm_destroy.restype = None
        lib.lbm_set_kernel.argtypes = [vp, i32, i32, i32, i32]
        lib.lbm_set_kernel.restype = ctypes.c_int
        lib.lbm_get_kernel.argtypes = [vp, P(i32)]
        lib.lbm_get_kernel.restype = ctypes.c_int
        lib.lbm_autotune.argtypes = [vp, i32, dp, i32, P(i32)]
        lib.lbm_autotune.restype = ctypes.c_int
        lib.lbm_step_noalloc.argtypes = [P(lbm_params), vp, vp, vp, vp, i32, vp, vp]
        lib.lbm_step_noalloc.restype = ctypes.c_int
        lib.lbm_set_exec.argtypes = [vp, i32, i32]
        lib.lbm_get_exec.argtypes = [vp, P(i32)]
        lib.lbm_barrier_selftest.argtypes = [vp, u64, P(i32)]
        lib.lbm_set_thermal_walls.argtypes = [vp, i32, i32, i32, i32, i32]
        lib.lbm_freezing.argtypes = [vp, i32, dp]
        lib.lbm_solid_profile.argtypes = [vp, i32, dp]
        lib.lbm_error_string.argtypes = [ctypes.c_int]
        lib.lbm_error_string.restype = ctypes.c_char_p
        for name in ("lbm_workspace_size", "lbm_create", "lbm_init_fields", "lbm_step",
                     "lbm_observables", "lbm_observables_all", "lbm_get_state", "lbm_set_state",
                     "lbm_freezing", "lbm_solid_profile"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(cfg: dict) -> lbm_params:
    p = lbm_params()
    for name, _ in lbm_params._fields_:
        setattr(p, name, 0 if name == "reserved" else cfg[name])
    return p


# ---- one-to-one wrappers of the C-ABI ---------------------------------------

def lbm_error_string(code: int) -> str:
    return load().lbm_error_string(int(code)).decode()


def lbm_workspace_size(params, storage: int = LBM_STORE_FP32) -> int:
    arr = (lbm_params * len(params))(*[make_params(c) for c in params])
    out = ctypes.c_uint64()
    rc = load().lbm_workspace_size(arr, len(params), int(storage), ctypes.byref(out))
    if rc:
        raise LbmError(rc, "lbm_workspace_size")
    return int(out.value)


def lbm_create(params, storage, d_workspace: int, nbytes: int, stream: int):
    arr = (lbm_params * len(params))(*[make_params(c) for c in params])
    h = ctypes.c_void_p()
    rc = load().lbm_create(arr, len(params), int(storage), ctypes.c_void_p(d_workspace),
                           int(nbytes), ctypes.c_void_p(stream), ctypes.byref(h))
    if rc:
        raise LbmError(rc, "lbm_create")
    return h


def lbm_init_fields(h, inst: int, phi0: np.ndarray, T0: np.ndarray):
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    rc = load().lbm_init_fields(h, int(inst), _dptr(phi0), _dptr(T0))
    if rc:
        raise LbmError(rc, "lbm_init_fields")


def lbm_step(h, n: int):
    rc = load().lbm_step(h, int(n))
    if rc:
        raise LbmError(rc, "lbm_step")


def lbm_observables(h, inst: int, check: bool = True) -> np.ndarray:
    out = np.zeros(LBM_OBS_COUNT)
    rc = load().lbm_observables(h, int(inst), _dptr(out))
    if rc and (check or rc != LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_observables")
    return out


def lbm_observables_all(h, n_inst: int, check: bool = True) -> np.ndarray:
    out = np.zeros((n_inst, LBM_OBS_COUNT))
    rc = load().lbm_observables_all(h, _dptr(out))
    if rc and (check or rc != LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_observables_all")
    return out


def lbm_freezing(h, inst: int) -> np.ndarray:
    out = np.zeros(LBM_FRZ_COUNT)
    rc = load().lbm_freezing(h, int(inst), _dptr(out))
    if rc:
        raise LbmError(rc, "lbm_freezing")
    return out


def lbm_solid_profile(h, inst: int, nx: int) -> np.ndarray:
    out = np.zeros(nx)
    rc = load().lbm_solid_profile(h, int(inst), _dptr(out))
    if rc:
        raise LbmError(rc, "lbm_solid_profile")
    return out


def lbm_get_state(h, inst: int, nx: int, ny: int):
    pops = np.zeros((27, ny, nx))
    aux = np.zeros((5, ny, nx))
    rc = load().lbm_get_state(h, int(inst), _dptr(pops), _dptr(aux))
    if rc:
        raise LbmError(rc, "lbm_get_state")
    return pops, aux


def lbm_set_state(h, inst: int, pops: np.ndarray, aux: np.ndarray):
    pops = np.ascontiguousarray(pops, dtype=np.float64)
    aux = np.ascontiguousarray(aux, dtype=np.float64)
    rc = load().lbm_set_state(h, int(inst), _dptr(pops), _dptr(aux))
    if rc:
        raise LbmError(rc, "lbm_set_state")


def lbm_step_count(h) -> int:
    return int(load().lbm_step_count(h))


def lbm_launch_count(h) -> int:
    return int(load().lbm_launch_count(h))


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_set_kernel(h, kind: int, a: int, b: int, c: int = 0):
    rc = load().lbm_set_kernel(h, int(kind), int(a), int(b), int(c))
    if rc:
        raise LbmError(rc, "lbm_set_kernel")


def lbm_step_noalloc(cfg: dict, pops_in: int, aux_in: int, pops_out: int, aux_out: int,
                     pitch: int, d_obs: int, stream: int):
    """One time step of one lattice on caller-owned device buffers (integer
    device addresses), with no handle and no device allocation."""
    p = make_params(cfg)
    rc = load().lbm_step_noalloc(ctypes.byref(p), ctypes.c_void_p(pops_in), ctypes.c_void_p(aux_in),
                                 ctypes.c_void_p(pops_out), ctypes.c_void_p(aux_out), int(pitch),
                                 ctypes.c_void_p(d_obs), ctypes.c_void_p(stream))
    if rc:
        raise LbmError(rc, "lbm_step_noalloc")


def lbm_autotune(h, steps: int, cap: int = 64):
    times = np.zeros(cap)
    n = ctypes.c_int32()
    rc = load().lbm_autotune(h, int(steps), _dptr(times), int(cap), ctypes.byref(n))
    if rc:
        raise LbmError(rc, "lbm_autotune")
    return times[: n.value].copy()


def lbm_get_kernel(h):
    out = (ctypes.c_int32 * 4)()
    rc = load().lbm_get_kernel(h, out)
    if rc:
        raise LbmError(rc, "lbm_get_kernel")
    return tuple(out[:])


def lbm_set_exec(h, mode: int, chunk: int = 64):
    rc = load().lbm_set_exec(h, int(mode), int(chunk))
    if rc:
        raise LbmError(rc, "lbm_set_exec")


def lbm_get_exec(h):
    """(mode, chunk, CTAs of one persistent launch)."""
    out = (ctypes.c_int32 * 3)()
    rc = load().lbm_get_exec(h, out)
    if rc:
        raise LbmError(rc, "lbm_get_exec")
    return tuple(out[:])


def lbm_set_thermal_walls(h, inst: int, x_lo: int, x_hi: int, y_lo: int, y_hi: int):
    rc = load().lbm_set_thermal_walls(h, int(inst), int(x_lo), int(x_hi), int(y_lo), int(y_hi))
    if rc:
        raise LbmError(rc, "lbm_set_thermal_walls")


def lbm_barrier_selftest(h, limit_ns: int) -> int:
    flag = ctypes.c_int32()
    rc = load().lbm_barrier_selftest(h, ctypes.c_uint64(int(limit_ns)), ctypes.byref(flag))
    if rc:
        raise LbmError(rc, "lbm_barrier_selftest")
    return int(flag.value)


# ---- convenience owner --------------------------------------------------------

class Lattice:
    """Handle over one or more lattices with a torch-owned device workspace."""

    def __init__(self, params, storage: int = LBM_STORE_FP32, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblbmfreeze needs a CUDA GPU; none is visible")
        load()
        if isinstance(params, dict):
            params = [params]
        self.params = [dict(p) for p in params]
        self.n_inst = len(self.params)
        self.storage = storage
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = lbm_workspace_size(self.params, storage)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._h = lbm_create(self.params, storage, self.workspace.data_ptr(), nbytes,
                             self.stream.cuda_stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lbm_destroy(self._h)
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

    def init(self, phi0, T0, inst: int = 0):
        lbm_init_fields(self._h, inst, phi0, T0)
        return self

    def step(self, n: int = 1):
        lbm_step(self._h, n)
        return self

    def observables(self, inst: int = 0, check: bool = True) -> dict:
        v = lbm_observables(self._h, inst, check)
        return {k: float(v[j]) for j, k in enumerate(OBS_NAMES)}

    def observables_all(self, check: bool = True) -> np.ndarray:
        return lbm_observables_all(self._h, self.n_inst, check)

    def freezing(self, inst: int = 0) -> dict:
        """Freezing record of the run: last observable step, the FP64
        mass-source integral over every step, the first observed step with
        solidified fraction >= 0.99 (-1 before) and the fraction itself."""
        v = lbm_freezing(self._h, inst)
        out = {k: float(v[j]) for j, k in enumerate(FRZ_NAMES)}
        out["step"] = int(out["step"])
        out["freeze_step"] = int(out["freeze_step"])
        return out

    def solid_profile(self, inst: int = 0) -> np.ndarray:
        """Sum over y of f_s per column at the last observable step."""
        return lbm_solid_profile(self._h, inst, self.params[inst]["nx"])

    def get_state(self, inst: int = 0):
        p = self.params[inst]
        return lbm_get_state(self._h, inst, p["nx"], p["ny"])

    def set_state(self, pops, aux, inst: int = 0):
        lbm_set_state(self._h, inst, pops, aux)
        return self

    def set_kernel(self, kind: int, a: int, b: int, c: int = 0):
        lbm_set_kernel(self._h, kind, a, b, c)
        return self

    def autotune(self, steps: int = 20):
        return lbm_autotune(self._h, steps)

    def set_thermal_walls(self, x_lo=0, x_hi=0, y_lo=0, y_hi=0, inst: int = 0):
        """Switch the thermal wall types of one lattice (for example from
        adiabatic during the isothermal relaxation to the contact angle to a
        cold substrate)."""
        lbm_set_thermal_walls(self._h, inst, x_lo, x_hi, y_lo, y_hi)
        self.params[inst].update(dirichlet_x_lo=x_lo, dirichlet_x_hi=x_hi,
                                 dirichlet_y_lo=y_lo, dirichlet_y_hi=y_hi)
        return self

    def set_exec(self, mode: int, chunk: int = 64):
        lbm_set_exec(self._h, mode, chunk)
        return self

    @property
    def exec(self):
        return lbm_get_exec(self._h)

    @property
    def kernel(self):
        return lbm_get_kernel(self._h)

    @property
    def step_count(self) -> int:
        return lbm_step_count(self._h)

    @property
    def launch_count(self) -> int:
        return lbm_launch_count(self._h)
