"""Pins of the oracle's pointwise pieces against what the paper and the
mathematics fix: the D2Q9 lattice of Eqs. 22-23, the moments the equilibria and
source terms of Eqs. 24, 25, 28, 31-33 must carry, the isotropic stencils of
Eq. 38, the wetting ghost of Eqs. 39-41, the enthalpy closure of Eqs. 8-9 and
the parameter relations of Eqs. 13 and 42."""
import math

import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def lat(oracle_mod):
    cx, cy, w, opp = oracle_mod.lattice()
    return cx.astype(float), cy.astype(float), w, opp


def test_lattice_matches_eq23_and_eq22(lat):
    cx, cy, w, opp = lat
    # Eq. 23 written with cos/sin (c = 1): axis links then diagonal links.
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        assert cx[i] == pytest.approx(math.cos(a), abs=1e-12)
        assert cy[i] == pytest.approx(math.sin(a), abs=1e-12)
    for i in range(5, 9):
        a = (2 * i - 9) * math.pi / 4
        assert cx[i] == pytest.approx(math.sqrt(2) * math.cos(a), abs=1e-12)
        assert cy[i] == pytest.approx(math.sqrt(2) * math.sin(a), abs=1e-12)
    assert (cx[0], cy[0]) == (0.0, 0.0)
    assert w[0] == pytest.approx(4 / 9)
    assert np.allclose(w[1:5], 1 / 9, rtol=0, atol=1e-16)
    assert np.allclose(w[5:], 1 / 36, rtol=0, atol=1e-16)
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]


def test_lattice_isotropy(lat):
    """Moments up to fourth order that the equilibria rely on."""
    cx, cy, w, _ = lat
    c = np.stack([cx, cy])
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose((w * c).sum(1), 0.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ai,bi->ab", w, c, c), CS2 * np.eye(2), atol=1e-15)
    assert np.allclose(np.einsum("i,ai,bi,ci->abc", w, c, c, c), 0.0, atol=1e-15)
    d = np.eye(2)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ai,bi,ci,di->abcd", w, c, c, c, c), iso4, atol=1e-15)


def _draws(n, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, size=12) for _ in range(n)]


def _moments(vals, lat):
    cx, cy, _, _ = lat
    c = np.stack([cx, cy])
    return vals.sum(), c @ vals, np.einsum("ai,bi,i->ab", c, c, vals)


def test_geq_moments(oracle_mod, lat):
    for r in _draws(50, 1):
        phi, ux, uy = 0.5 + 0.5 * r[0], 0.1 * r[1], 0.1 * r[2]
        m0, m1, _ = _moments(oracle_mod.geq(phi, ux, uy), lat)
        assert m0 == pytest.approx(phi, abs=1e-14)
        assert np.allclose(m1, [phi * ux, phi * uy], atol=1e-14)


def test_heq_moments(oracle_mod, lat):
    """Sum h^eq = H, sum c h^eq = Cp T u, sum cc h^eq = cs2 Cp_ref T I + Cp T uu
    (the moments that recover the total-enthalpy equation, Eq. 7)."""
    for r in _draws(50, 2):
        H, T = 10 * r[0], r[1]
        Cp, Cpr = 1.0 + 0.5 * abs(r[2]), 1.0 + 0.3 * abs(r[3])
        u = 0.1 * r[4:6]
        m0, m1, m2 = _moments(oracle_mod.heq(H, T, Cp, Cpr, u[0], u[1]), lat)
        assert m0 == pytest.approx(H, abs=1e-13)
        assert np.allclose(m1, Cp * T * u, atol=1e-14)
        assert np.allclose(m2, CS2 * Cpr * T * np.eye(2) + Cp * T * np.outer(u, u), atol=1e-14)


def test_feq_moments(oracle_mod, lat):
    """Pressure-based equilibrium: sum = 0, sum c = rho u, sum cc = p I + rho uu,
    and the i != 0 sum that Eq. 36 inverts."""
    for r in _draws(50, 3):
        p, rho = 0.01 * r[0], 1.0 + 0.9 * r[1]
        u = 0.1 * r[2:4]
        f = oracle_mod.feq(p, rho, u[0], u[1])
        m0, m1, m2 = _moments(f, lat)
        assert m0 == pytest.approx(0.0, abs=1e-14)
        assert np.allclose(m1, rho * u, atol=1e-14)
        assert np.allclose(m2, p * np.eye(2) + rho * np.outer(u, u), atol=1e-14)
        w0 = 4 / 9
        s0 = w0 * (-(u @ u) / (2 * CS2))
        assert f[1:].sum() == pytest.approx((1 - w0) * p / CS2 - rho * s0, abs=1e-14)


def test_force_moments(oracle_mod, lat):
    """Sum F_i = S, sum c F_i = F + rho f, sum cc F_i = cs2 S I + u F~ + F~ u."""
    for r in _draws(50, 4):
        S = 0.01 * r[0]
        fvec = 0.01 * r[1:3]
        u = 0.1 * r[3:5]
        ft = 0.01 * r[5:7]
        Fi = oracle_mod.force_F(S, fvec[0], fvec[1], u[0], u[1], ft[0], ft[1])
        m0, m1, m2 = _moments(Fi, lat)
        assert m0 == pytest.approx(S, abs=1e-15)
        assert np.allclose(m1, fvec, atol=1e-15)
        assert np.allclose(m2, CS2 * S * np.eye(2) + np.outer(u, ft) + np.outer(ft, u), atol=1e-15)


def test_source_moments(oracle_mod, lat):
    """Sum G_i = phi div u, sum c G_i = d_t(phi u) + cs2 lambda n (Eq. 25)."""
    for r in _draws(50, 5):
        phi, md = 0.5 + 0.5 * r[0], 0.01 * r[1]
        dt = 0.01 * r[2:4]
        lam = abs(r[4])
        n = r[5:7] / np.linalg.norm(r[5:7])
        G = oracle_mod.source_G(phi, md, dt[0], dt[1], lam, n[0], n[1])
        m0, m1, _ = _moments(G, lat)
        assert m0 == pytest.approx(phi * md, abs=1e-15)
        assert np.allclose(m1, dt + CS2 * lam * n, atol=1e-15)


# ---------------------------------------------------------------------------
# Stencils (Eq. 38) and ghosts (Eqs. 39-41)
# ---------------------------------------------------------------------------

def _state(oracle_mod, **over):
    p = inputs.params(**over)
    return oracle_mod.Oracle(p)


def test_stencil_exact_on_quadratics(oracle_mod):
    o = _state(oracle_mod, nx=16, ny=16)
    x, y = inputs.coords(16, 16)
    rng = np.random.default_rng(7)
    for _ in range(5):
        a = rng.uniform(-1, 1, 6)
        Z = a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y
        for (px, py) in [(3, 4), (8, 8), (12, 5)]:
            gx, gy, lap = o.stencil(Z, px, py)
            assert gx == pytest.approx(a[1] + 2 * a[3] * px + a[4] * py, abs=1e-11)
            assert gy == pytest.approx(a[2] + a[4] * px + 2 * a[5] * py, abs=1e-11)
            assert lap == pytest.approx(2 * a[3] + 2 * a[5], abs=1e-11)


def test_stencil_second_order_on_periodic_waves(oracle_mod):
    errs = []
    for n in (16, 32, 64):
        o = _state(oracle_mod, nx=n, ny=n)
        x, y = inputs.coords(n, n)
        k = 2 * np.pi / n
        Z = np.sin(k * x + 0.3) * np.cos(2 * k * y + 0.7)
        px, py = 0, n // 8  # a periodic edge site exercises the wrap
        gx, gy, lap = o.stencil(Z, px, py)
        ex = k * np.cos(k * px + 0.3) * np.cos(2 * k * py + 0.7)
        ey = -2 * k * np.sin(k * px + 0.3) * np.sin(2 * k * py + 0.7)
        el = -5 * k * k * Z[py, px]
        errs.append((abs(gx - ex) / k, abs(gy - ey) / k + abs(lap - el) / k ** 2))
    for j in range(2):
        assert errs[0][j] / errs[1][j] > 3.5 and errs[1][j] / errs[2][j] > 3.5


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
def test_wetting_ghost_linear_field(oracle_mod, theta):
    """For phi = a + b x + c y the tangential derivative at the wall is b for
    every second-order formula, so Eq. 39 fixes the ghost exactly."""
    nx, ny = 12, 10
    o = _state(oracle_mod, nx=nx, ny=ny, periodic_x=0, periodic_y=0, theta_deg=theta)
    x, y = inputs.coords(nx, ny)
    a, b, c = 0.4, -0.03, 0.02
    Z = a + b * x + c * y
    t = math.tan(math.pi / 2 - math.radians(theta))
    for px in range(2, nx - 2):
        # wall below row 0: n_w = +y, n_w.grad = Z(x,0) - Z(x,-1) = -t |b|
        assert o.ghost(Z, px, -1, 1) == pytest.approx(Z[0, px] + t * abs(b), abs=1e-14)
        # wall above row ny-1: n_w = -y, Z(x,ny-1) - Z(x,ny) = -t |b|
        assert o.ghost(Z, px, ny, 1) == pytest.approx(Z[ny - 1, px] + t * abs(b), abs=1e-14)
    for py in range(2, ny - 2):
        assert o.ghost(Z, -1, py, 1) == pytest.approx(Z[py, 0] + t * abs(c), abs=1e-14)
        assert o.ghost(Z, nx, py, 1) == pytest.approx(Z[py, nx - 1] + t * abs(c), abs=1e-14)
    # copy ghosts
    assert o.ghost(Z, 3, -1, 0) == Z[0, 3]
    assert o.ghost(Z, -1, -1, 1) == Z[0, 0]


def test_wetting_ghost_uses_second_layer(oracle_mod):
    """Eq. 40b extrapolates the tangential derivative from the first two
    layers: 1.5 d_x phi(x,0) - 0.5 d_x phi(x,1)."""
    nx, ny = 12, 8
    o = _state(oracle_mod, nx=nx, ny=ny, periodic_x=1, periodic_y=0, theta_deg=45.0)
    x, y = inputs.coords(nx, ny)
    Z = np.sin(0.5 * x) * (1.0 + 0.3 * y)  # the two layers differ
    px = 5
    d0 = 0.5 * (Z[0, px + 1] - Z[0, px - 1])
    d1 = 0.5 * (Z[1, px + 1] - Z[1, px - 1])
    assert o.ghost(Z, px, -1, 1) == pytest.approx(Z[0, px] + 1.0 * abs(1.5 * d0 - 0.5 * d1), abs=1e-14)
    # periodic wrap of the tangential neighbours at the lattice edge
    d0 = 0.5 * (Z[0, 1] - Z[0, nx - 1])
    d1 = 0.5 * (Z[1, 1] - Z[1, nx - 1])
    assert o.ghost(Z, 0, -1, 1) == pytest.approx(Z[0, 0] + abs(1.5 * d0 - 0.5 * d1), abs=1e-14)


# ---------------------------------------------------------------------------
# Enthalpy closure (Eqs. 8-9) and derived parameters (Eqs. 13, 42)
# ---------------------------------------------------------------------------

def _paper_closure(H, Cp, Tm, L):
    """Eq. 9 for a pure substance (T_s = T_l = T_m, H_s = Cp T_m, H_l = H_s + L)."""
    Hs, Hl = Cp * Tm, Cp * Tm + L
    if H <= Hs:
        fl = 0.0
    elif H >= Hl:
        fl = 1.0
    else:
        fl = (H - Hs) / (Hl - Hs)
    Ts = Tl = Tm
    if H < Hs:
        T = H / Cp
    elif H <= Hl:
        T = Ts + (H - Hs) / (Hl - Hs) * (Tl - Ts)
    else:
        T = Tl + (H - Hl) / Cp
    return fl, T


@pytest.mark.parametrize("Tm,Tw,Ste,Cp", [(0.0, -1.0, 0.1, 1.0), (0.5, -1.5, 0.2, 1.3)])
def test_closure_liquid_matches_eq9(oracle_mod, Tm, Tw, Ste, Cp):
    o = _state(oracle_mod, T_m=Tm, T_w=Tw, Ste=Ste, Cp=Cp)
    L = o.derived()["L"]
    assert L == pytest.approx(Cp * (Tm - Tw) / Ste)
    for H in np.linspace(Cp * Tm - 3, Cp * Tm + L + 3, 97):
        fs, T = o.closure(H, 1.0)
        fl, Tp = _paper_closure(H, Cp, Tm, L)
        assert 1 - fs == pytest.approx(fl, abs=1e-13)
        assert T == pytest.approx(Tp, abs=1e-12)
        # Eq. 8 with f_l = 1 - f_s
        assert H == pytest.approx(Cp * T + L * (1 - fs), abs=1e-12)


def test_closure_temperature_ignores_phase_field_and_solid_is_masked(oracle_mod):
    """The thermal model of Section 2.2 has no phi: T follows Eq. 9b for every
    phihat. Solid forms only in the liquid content: f_s = 0 in gas, f_s =
    1 - f_l in liquid, continuous in between with slope <= 1 / pc_ramp."""
    o = _state(oracle_mod)
    L = o.derived()["L"]
    ramp = inputs.BASE["pc_ramp"]
    for H in np.linspace(-3, L + 3, 41):
        fl, Tp = _paper_closure(H, 1.0, 0.0, L)
        for q in (-0.05, 0.0, 0.2, 0.5 - ramp / 2):
            fs, T = o.closure(H, q)
            assert fs == pytest.approx(0.0, abs=1e-15)
            assert T == pytest.approx(Tp, abs=1e-12)
        for q in (0.5 + ramp / 2, 0.8, 1.0, 1.05):
            fs, T = o.closure(H, q)
            assert fs == pytest.approx(1.0 - fl, abs=1e-13)
            assert T == pytest.approx(Tp, abs=1e-12)
    ph = np.linspace(-0.1, 1.1, 121)
    for H in np.linspace(-2, L + 2, 31):
        fl, _ = _paper_closure(H, 1.0, 0.0, L)
        fs = np.array([o.closure(H, q)[0] for q in ph])
        assert (fs >= 0).all() and (fs <= 1.0 - fl + 1e-15).all()
        assert np.abs(np.diff(fs)).max() <= (ph[1] - ph[0]) / ramp + 1e-12
        assert (np.diff(fs) >= -1e-15).all()  # more liquid content, more solid


def test_derived_parameters(oracle_mod):
    o = _state(oracle_mod, sigma=0.013, W=5.0, mobility=0.05, tau_f_liquid=0.9,
               rho_ratio_lg=1000.0, mu_ratio_lg=100.0, rho_ratio_sl=1.1)
    d = o.derived()
    # Eq. 13 and its inverse
    assert math.sqrt(2 * d["kappa"] * d["beta"]) / 6 == pytest.approx(0.013)
    assert math.sqrt(8 * d["kappa"] / d["beta"]) == pytest.approx(5.0)
    # mobility relation of Section 3.1 read with tau_g
    assert CS2 * (d["tau_g"] - 0.5) == pytest.approx(0.05)
    assert d["rho_g"] == pytest.approx(1e-3) and d["rho_s"] == pytest.approx(1.1)
    assert d["mu_l"] / d["mu_g"] == pytest.approx(100.0)
    assert d["mu_l"] == pytest.approx(CS2 * 0.4)


def test_invalid_parameters_rejected(oracle_mod):
    for bad in (dict(nx=2), dict(tau_h=0.5), dict(mobility=0.0), dict(theta_deg=180.0),
                dict(T_w=0.0), dict(Ste=0.0), dict(rho_ratio_lg=-1.0), dict(normal_eps=0.0),
                dict(k_ratio_gl=0.0), dict(Cp_ratio_sl=-0.5)):
        with pytest.raises(oracle_mod.OracleError):
            _state(oracle_mod, **bad)
