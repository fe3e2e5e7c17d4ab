"""Seeded synthetic workloads for the freezing step.

This module only states problems: parameter sets and initial fields (order
parameter phi0 and temperature T0 on the lattice). It holds none of the
scheme's arithmetic, so the FP64 oracle and the CUDA library can both be fed
from it. Every random draw goes through ``numpy.random.default_rng(seed)``.

Parameter dictionaries carry the paper's own problem statement (Sections 4.1,
4.2 and 4.3 of arXiv 2403.16122): lattice size, walls, relaxation times,
density/viscosity ratios, Stefan number, rho_s/rho_l, contact angle, wall
temperature. Values the paper leaves open are fixed here once: sigma = 0.01,
rho_l = 1, Cp = Cp_ref = 1, T_m = 0, a phase-change ramp width of 0.2 and an
interface-normal regularisation of 1e-3.

Arrays use the lattice layout [ny, nx]; site (x, y) is element [y, x]. Walls
sit half a link outside the first and last lattice rows/columns, so a wall
below row 0 is at y = -1/2.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20240324

BASE = dict(
    nx=64, ny=64,
    periodic_x=1, periodic_y=1,
    dirichlet_x_lo=0, dirichlet_x_hi=0, dirichlet_y_lo=0, dirichlet_y_hi=0,
    st_mask_liquid=0,
    W=4.0, sigma=0.01, mobility=0.02,
    tau_f_liquid=0.8, tau_h=0.8,
    rho_l=1.0, rho_ratio_lg=10.0, rho_ratio_sl=0.9, mu_ratio_lg=10.0,
    Ste=0.1, Cp=1.0, Cp_ref=1.0, T_m=0.0, T_w=-1.0,
    theta_deg=90.0, pc_ramp=0.2, normal_eps=1e-3,
    gx=0.0, gy=0.0, beta_T=0.0, T_ref=0.0, rho_0=1.0,  # Boussinesq force off
    Cp_ratio_sl=1.0, Cp_ratio_gl=1.0, k_ratio_sl=1.0, k_ratio_gl=1.0,  # uniform thermal props
)


def params(**over) -> dict:
    """BASE with overrides; unknown keys are an error."""
    bad = set(over) - set(BASE)
    if bad:
        raise KeyError(f"unknown parameter(s): {sorted(bad)}")
    p = dict(BASE)
    p.update(over)
    p["nx"], p["ny"] = int(p["nx"]), int(p["ny"])
    return p


# ----------------------------------------------------------------------------
# Initial order-parameter profiles
# ----------------------------------------------------------------------------

def coords(nx: int, ny: int):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def flat_column(nx: int, ny: int, H0: float, W: float, axis: str = "x") -> np.ndarray:
    """Liquid layer of thickness H0 on a wall at -1/2 (Eq. 43 shifted so that
    the liquid occupies exactly H0 cells from the wall)."""
    x, y = coords(nx, ny)
    d = x if axis == "x" else y
    return 0.5 + 0.5 * np.tanh(2.0 * (H0 - 0.5 - d) / W)


def slab(nx: int, ny: int, x0: float, x1: float, W: float) -> np.ndarray:
    """Periodic liquid slab between x0 and x1 (two flat interfaces)."""
    x, _ = coords(nx, ny)
    return 0.5 * (np.tanh(2.0 * (x - x0) / W) - np.tanh(2.0 * (x - x1) / W))


def disk(nx: int, ny: int, xc: float, yc: float, R: float, W: float) -> np.ndarray:
    """Circular drop of radius R (Eq. 45 with the square root restored)."""
    x, y = coords(nx, ny)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / W)


def cap(nx: int, ny: int, R: float, theta_deg: float, W: float, xc: float | None = None) -> np.ndarray:
    """Drop of radius R cut by the wall at y = -1/2 so that it meets the wall at
    contact angle theta: circle centre at y = -1/2 - R cos(theta)."""
    if xc is None:
        xc = 0.5 * (nx - 1)
    yc = -0.5 - R * math.cos(math.radians(theta_deg))
    return disk(nx, ny, xc, yc, R, W)


def place_bubbles(rng, nx, ny, R, theta_deg, W, n_bub, r_lo, r_hi, xc=None, tries=20000):
    """Rejection-sample n_bub bubble centres inside a cap drop, each bubble at
    least W away from the drop surface, the wall and the other bubbles."""
    if xc is None:
        xc = 0.5 * (nx - 1)
    yc = -0.5 - R * math.cos(math.radians(theta_deg))
    out = []
    for _ in range(tries):
        if len(out) == n_bub:
            break
        r = rng.uniform(r_lo, r_hi)
        bx = rng.uniform(xc - R, xc + R)
        by = rng.uniform(-0.5, yc + R)
        if math.hypot(bx - xc, by - yc) > R - r - W:
            continue
        if by - r - W < -0.5:
            continue
        if any(math.hypot(bx - q[0], by - q[1]) < r + q[2] + W for q in out):
            continue
        out.append((bx, by, r))
    return out


def with_bubbles(phi: np.ndarray, bubbles, W: float) -> np.ndarray:
    ny, nx = phi.shape
    x, y = coords(nx, ny)
    out = phi.copy()
    for bx, by, r in bubbles:
        d = np.sqrt((x - bx) ** 2 + (y - by) ** 2)
        out *= 0.5 + 0.5 * np.tanh(2.0 * (d - r) / W)
    return out


# ----------------------------------------------------------------------------
# The five workloads (plus scaled versions used by the tests)
# ----------------------------------------------------------------------------

def stefan(nx=256, ny=8, H0=128, Ste=0.1, rho_ratio_sl=0.9, **over):
    """Three-phase Stefan problem (Section 4.1): cold Dirichlet wall at x = -1/2,
    closed adiabatic wall at the far end, periodic in y; liquid on the first H0
    columns, gas beyond; T0 = T_m."""
    p = params(nx=nx, ny=ny, periodic_x=0, periodic_y=1, dirichlet_x_lo=1,
               rho_ratio_lg=10.0, mu_ratio_lg=10.0, Ste=Ste,
               rho_ratio_sl=rho_ratio_sl, **over)
    phi0 = flat_column(nx, ny, H0, p["W"], axis="x")
    T0 = np.full((ny, nx), p["T_m"])
    return p, phi0, T0


def sessile(nx=256, ny=256, R=64.0, theta_deg=90.0, **over):
    """Sessile drop on a cold no-slip wall at y = -1/2 with wetting angle theta;
    adiabatic no-slip top wall; periodic in x (Section 4.2)."""
    kw = dict(rho_ratio_lg=1000.0, mu_ratio_lg=100.0, rho_ratio_sl=0.9, Ste=0.1)
    kw.update(over)
    p = params(nx=nx, ny=ny, periodic_x=1, periodic_y=0, dirichlet_y_lo=1,
               theta_deg=theta_deg, **kw)
    phi0 = cap(nx, ny, R, theta_deg, p["W"])
    T0 = np.full((ny, nx), p["T_m"])
    return p, phi0, T0


def bubbles_drop(n=1024, R=None, seed=DEFAULT_SEED, n_bub=8, r_lo=4.0, r_hi=12.0, **over):
    """Drop with gas bubbles on a cold wall (Section 4.3 structure): contact
    angle drawn from U[60, 120] degrees, bubbles placed without overlap,
    surface tension restricted to the liquid; ratios as in the Stefan case."""
    rng = np.random.default_rng(seed)
    theta = float(rng.uniform(60.0, 120.0))
    if R is None:
        R = 320.0 * n / 1024.0
    kw = dict(rho_ratio_lg=10.0, mu_ratio_lg=10.0, rho_ratio_sl=0.9, Ste=0.1)
    kw.update(over)
    p = params(nx=n, ny=n, periodic_x=1, periodic_y=0, dirichlet_y_lo=1,
               theta_deg=theta, st_mask_liquid=1, **kw)
    phi = cap(n, n, R, theta, p["W"])
    bub = place_bubbles(rng, n, n, R, theta, p["W"], n_bub, r_lo, r_hi)
    phi = with_bubbles(phi, bub, p["W"])
    T0 = np.full((n, n), p["T_m"])
    return p, phi, T0


def column_bubbles(l=32, g=1e-4, beta_T=1.0, **over):
    """Liquid column with three gas bubbles freezing from a cold bottom wall
    (Section 4.3 geometry: a 4l x 3l box, periodic in x, walls at the bottom
    and the top; liquid up to 1.8 l; bubbles of radii 0.2 l, 0.24 l, 0.3 l at
    (l, 0.3 l), (2 l, l), (3 l, 0.4 l)), with the Boussinesq buoyancy
    F_g = -rho_0 g beta_T (T - T_ref), gravity pointing to -y and T_ref the
    initial temperature. Thermal properties uniform (one C_p and tau_h)."""
    nx, ny = 4 * l, 3 * l
    kw = dict(rho_ratio_lg=10.0, mu_ratio_lg=10.0, rho_ratio_sl=0.9, Ste=0.1)
    kw.update(over)
    p = params(nx=nx, ny=ny, periodic_x=1, periodic_y=0, dirichlet_y_lo=1, st_mask_liquid=1,
               gx=0.0, gy=-g, beta_T=beta_T, rho_0=1.0, **kw)
    p["T_ref"] = p["T_m"]
    phi = flat_column(nx, ny, 1.8 * l, p["W"], axis="y")
    bub = [(1.0 * l, 0.3 * l, 0.2 * l), (2.0 * l, 1.0 * l, 0.24 * l), (3.0 * l, 0.4 * l, 0.3 * l)]
    phi = with_bubbles(phi, bub, p["W"])
    T0 = np.full((ny, nx), p["T_m"])
    return p, phi, T0


def batched_sweep(n_inst=256, seed=DEFAULT_SEED, sizes=(128, 192, 256, 384, 512)):
    """Independent sessile drops of uneven size and wetting: square grids drawn
    from `sizes`, R ~ U[0.15, 0.3] grid, theta ~ U[30, 150] deg,
    rho_s/rho_l ~ U[0.88, 0.95], Ste ~ U[0.05, 0.2]; ratios 1000/100."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        g = int(rng.choice(sizes))
        R = float(rng.uniform(0.15, 0.3)) * g
        th = float(rng.uniform(30.0, 150.0))
        sl = float(rng.uniform(0.88, 0.95))
        ste = float(rng.uniform(0.05, 0.2))
        out.append(sessile(g, g, R, th, rho_ratio_sl=sl, Ste=ste))
    return out


def batched_bubbles(n_inst=1024, seed=DEFAULT_SEED, lo=64, hi=256):
    """Independent drops with 0-4 bubbles (r ~ U[3, 10]) on uneven grids
    nx, ny ~ U{lo..hi}, theta ~ U[60, 120] deg, R ~ U[0.15, 0.3] min(nx, ny);
    other parameters as in the bubble drop."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        nx = int(rng.integers(lo, hi + 1))
        ny = int(rng.integers(lo, hi + 1))
        th = float(rng.uniform(60.0, 120.0))
        R = float(rng.uniform(0.15, 0.3)) * min(nx, ny)
        nb = int(rng.integers(0, 5))
        p = params(nx=nx, ny=ny, periodic_x=1, periodic_y=0, dirichlet_y_lo=1,
                   theta_deg=th, st_mask_liquid=1, rho_ratio_lg=10.0,
                   mu_ratio_lg=10.0, rho_ratio_sl=0.9, Ste=0.1)
        phi = cap(nx, ny, R, th, p["W"])
        bub = place_bubbles(rng, nx, ny, R, th, p["W"], nb, 3.0, 10.0)
        phi = with_bubbles(phi, bub, p["W"])
        out.append((p, phi, np.full((ny, nx), p["T_m"])))
    return out


def random_state(p: dict, seed: int, amp: float = 1e-3):
    """Perturbed initial fields for parity cases that must exercise every term:
    a droplet-like phi with small noise and a temperature field that crosses
    T_m. Returns (phi0, T0)."""
    rng = np.random.default_rng(seed)
    nx, ny = p["nx"], p["ny"]
    phi = disk(nx, ny, 0.5 * (nx - 1), 0.4 * ny, 0.3 * min(nx, ny), p["W"])
    phi = np.clip(phi + amp * rng.standard_normal(phi.shape), 0.0, 1.0)
    x, y = coords(nx, ny)
    T0 = p["T_m"] + 0.2 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    return phi, T0
