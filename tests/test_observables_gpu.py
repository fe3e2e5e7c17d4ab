"""Run-spanning observables of the CUDA path against the FP64 oracle: the
mass-source integral (the sum of mdot of Eq. 19 over every step and site,
accumulated in FP64 on the device while the steps run), the solid height
profile (sum over y of f_s per column, the frozen shape of Section 4.2) and
the freezing time (first observed step with solidified fraction >= 0.99,
Sections 4.2-4.3), through every kernel layout and execution form."""
import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-5  # observables of the FP32 path against the oracle (relative)


@pytest.fixture(scope="module")
def lbm():
    from paper_2403_16122_gb300 import build, lbm as _lbm
    build.build()
    _lbm.load()
    return _lbm


def _check(lat, o, inst=0):
    fr = lat.freezing(inst)
    assert fr["step"] == o.step_count
    md_o = o.mdot_integral
    assert fr["mdot_integral"] == pytest.approx(md_o, rel=REL, abs=1e-7), (fr, md_o)
    ob = o.observables()
    X_o = ob["solid"] / ob["volume"]
    assert fr["solid_fraction"] == pytest.approx(X_o, rel=REL, abs=1e-9)
    # each column sums ny sites; at the freezing front a site's f_s follows
    # FP32 rounding of H over the run (f_l = (H - H_s) / L), so each is held
    # to 2e-5
    prof = lat.solid_profile(inst)
    assert np.abs(prof - o.solid_profile()).max() <= 2e-5 * lat.params[inst]["ny"]
    return fr, X_o


def test_freezing_record_tile_kernel_to_completion(lbm, oracle_mod):
    """A liquid column frozen from a cold wall (walls in x: the tile kernel)
    until the solidified fraction passes 0.99: the integral, the profile and
    the fraction after every 100-step call, and the freezing step."""
    p, phi0, T0 = inputs.stefan(nx=24, ny=4, H0=8, Ste=0.25, rho_ratio_sl=0.9)
    lat = lbm.Lattice([p]).init(phi0, T0)
    assert lat.kernel[0] == lbm.LBM_KERNEL_TILE
    o = oracle_mod.Oracle(p).init(phi0, T0)
    want = -1
    for k in range(1, 25):
        lat.step(100)
        o.step(100)
        fr, X = _check(lat, o)
        if want < 0 and X >= lbm.LBM_FREEZE_FRACTION:
            want = o.step_count
        assert fr["freeze_step"] == want
    assert want > 0 and o.mdot_integral > 0.5


@pytest.mark.parametrize("kind", ["staged", "strip"])
def test_freezing_record_strip_kernels(lbm, oracle_mod, kind):
    """A sessile drop on a cold wall (periodic x: the strip layouts), ragged
    strips: integral and profile after each 250-step call."""
    p, phi0, T0 = inputs.sessile(nx=70, ny=44, R=16.0, theta_deg=100.0)
    lat = lbm.Lattice([p]).init(phi0, T0)
    lat.set_kernel(lbm.LBM_KERNEL_STAGED if kind == "staged" else lbm.LBM_KERNEL_STRIP, 4, 0, 168)
    o = oracle_mod.Oracle(p).init(phi0, T0)
    for _ in range(4):
        lat.step(250)
        o.step(250)
        fr, _ = _check(lat, o)
    assert o.mdot_integral > 1.0 and fr["freeze_step"] == -1


def test_integral_survives_table_changes(lbm, oracle_mod):
    """The device sums live in the slots of the current tile or strip table;
    switching layouts (lbm_set_kernel, lbm_autotune) mid-run folds them into
    the lattice's total, so the integral still covers every step."""
    p, phi0, T0 = inputs.sessile(nx=64, ny=40, R=14.0)
    lat = lbm.Lattice([p]).init(phi0, T0)
    o = oracle_mod.Oracle(p).init(phi0, T0)
    lat.step(150)
    o.step(150)
    _check(lat, o)
    lat.set_kernel(lbm.LBM_KERNEL_STRIP, 8, 6, 128)
    lat.step(150)
    lat.set_kernel(lbm.LBM_KERNEL_TILE, 32, 8)
    lat.step(100)
    o.step(250)
    _check(lat, o)
    lat.autotune(steps=2)  # advances the lattice by the steps it times
    n = lat.step_count - o.step_count
    o.step(n)
    lat.step(50)
    o.step(50)
    _check(lat, o)


@pytest.mark.parametrize("mode", ["graph", "persistent"])
def test_freezing_record_batched_forms(lbm, oracle_mod, mode):
    """Two uneven drops in one handle, the body steps replayed from a graph or
    run by the persistent kernel: each lattice's record against its own
    oracle run; re-initialising one lattice restarts only its record."""
    cases = [inputs.sessile(nx=64, ny=40, R=14.0),
             inputs.sessile(nx=50, ny=36, R=11.0, theta_deg=70.0)]
    lat = lbm.Lattice([c[0] for c in cases])
    for k, (_, phi0, T0) in enumerate(cases):
        lat.init(phi0, T0, inst=k)
    lat.set_exec(lbm.LBM_EXEC_GRAPH if mode == "graph" else lbm.LBM_EXEC_PERSISTENT, 40)
    ors = [oracle_mod.Oracle(p).init(phi0, T0) for p, phi0, T0 in cases]
    for _ in range(3):
        lat.step(101)
        for k, o in enumerate(ors):
            o.step(101)
            _check(lat, o, inst=k)
    p1, phi1, T1 = cases[1]
    lat.init(phi1, T1, inst=1)
    ors[1] = oracle_mod.Oracle(p1).init(phi1, T1)
    lat.step(101)
    ors[0].step(101)
    ors[1].step(101)
    fr0, fr1 = lat.freezing(0), lat.freezing(1)
    assert fr0["step"] == 404 and fr1["step"] == 101
    assert fr1["mdot_integral"] == pytest.approx(ors[1].mdot_integral, rel=REL, abs=1e-7)
    assert fr0["mdot_integral"] == pytest.approx(ors[0].mdot_integral, rel=REL, abs=1e-7)


def test_records_need_a_step(lbm):
    p, phi0, T0 = inputs.sessile(nx=40, ny=24, R=8.0)
    lat = lbm.Lattice([p]).init(phi0, T0)
    for call in (lat.freezing, lat.solid_profile):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.code == lbm.LBM_ESTATE
    lat.step(1)
    assert lat.freezing()["step"] == 1
