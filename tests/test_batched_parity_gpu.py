"""Oracle parity of the batched forms (many independent lattices in one
handle): every lattice of a handle of uneven drops, advanced by one launch per
step, by replayed CUDA graphs of launches, or by the cooperative persistent
kernel, against its own FP64 oracle run, element by element (Section 3's
update, Section 4.2-4.3 drop set-ups); and the 16-bit storage forms of the
same batch against the oracle at the reduced-precision bar."""
import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs
from parity_util import compare_state

pytestmark = pytest.mark.gpu


def _batch():
    """Three uneven lattices, all periodic in x (the strip layouts): a sessile
    drop at density ratio 1000 and wetting at 70 deg on a ragged 70 x 44
    lattice; a drop with two gas bubbles and the liquid-masked surface
    tension at 110 deg on 96 x 64; a small drop at 45 deg on 40 x 30."""
    rng = np.random.default_rng(7)
    a = inputs.sessile(nx=70, ny=44, R=16.0, theta_deg=70.0)
    p = inputs.params(nx=96, ny=64, periodic_x=1, periodic_y=0, dirichlet_y_lo=1,
                      theta_deg=110.0, st_mask_liquid=1, rho_ratio_lg=10.0, mu_ratio_lg=10.0,
                      rho_ratio_sl=0.9, Ste=0.1)
    phi = inputs.cap(96, 64, 26.0, 110.0, p["W"])
    phi = inputs.with_bubbles(phi, inputs.place_bubbles(rng, 96, 64, 26.0, 110.0, p["W"], 2,
                                                        4.0, 6.0), p["W"])
    b = (p, phi, np.full((64, 96), p["T_m"]))
    c = inputs.sessile(nx=40, ny=30, R=10.0, theta_deg=45.0, rho_ratio_lg=100.0,
                       mu_ratio_lg=30.0)
    return [a, b, c]


@pytest.fixture(scope="module")
def oracle_runs(oracle_mod):
    """Each lattice's state and observables after 1000 oracle steps."""
    out = []
    for p, phi0, T0 in _batch():
        o = oracle_mod.Oracle(p).init(phi0, T0)
        o.step(1000)
        out.append((o.get_state(), o.observables(), o.mdot_integral))
    return out


@pytest.mark.parametrize("mode", ["launch", "graph", "persistent"])
def test_batched_forms_match_oracle_1000_steps(oracle_runs, mode):
    from paper_2403_16122_gb300 import lbm

    cases = _batch()
    lat = lbm.Lattice([c[0] for c in cases])
    for k, (_, phi0, T0) in enumerate(cases):
        lat.init(phi0, T0, inst=k)
    ex = {"launch": lbm.LBM_EXEC_LAUNCH, "graph": lbm.LBM_EXEC_GRAPH,
          "persistent": lbm.LBM_EXEC_PERSISTENT}[mode]
    lat.set_exec(ex, 64)
    lat.step(1000)
    assert lat.exec[0] == ex
    for k, (state, ob_o, md_o) in enumerate(oracle_runs):
        d = compare_state(lat.get_state(k), state)
        print(mode, "lattice", k, d)
        ob = lat.observables(k)
        assert ob["solid"] == pytest.approx(ob_o["solid"], rel=1e-5)
        assert ob["volume"] == pytest.approx(ob_o["volume"], rel=5e-6)
        assert lat.freezing(k)["mdot_integral"] == pytest.approx(md_o, rel=1e-5, abs=1e-7)
    lat.close()


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_batched_persistent_observables_match_oracle(oracle_mod, storage):
    """The same batch in 16-bit storage, persistent form, 2000 steps: solid
    amount and drop volume within 1 % and the front height at the centre
    column within 0.5 lattice units of the FP64 oracle."""
    from paper_2403_16122_gb300 import lbm

    st = lbm.LBM_STORE_FP16 if storage == "fp16" else lbm.LBM_STORE_BF16
    cases = _batch()
    lat = lbm.Lattice([c[0] for c in cases], storage=st)
    for k, (_, phi0, T0) in enumerate(cases):
        lat.init(phi0, T0, inst=k)
    lat.set_exec(lbm.LBM_EXEC_PERSISTENT, 100)
    lat.step(2000)
    for k, (p, phi0, T0) in enumerate(cases):
        o = oracle_mod.Oracle(p).init(phi0, T0)
        o.step(2000)
        ob_o, ob = o.observables(), lat.observables(k)
        print(storage, k, {j: (ob[j], ob_o[j]) for j in ("solid", "volume", "solid_col")})
        assert ob_o["solid"] > 20
        assert ob["solid"] == pytest.approx(ob_o["solid"], rel=0.01)
        assert ob["volume"] == pytest.approx(ob_o["volume"], rel=0.01)
        assert abs(ob["solid_col"] - ob_o["solid_col"]) <= 0.5
    lat.close()
