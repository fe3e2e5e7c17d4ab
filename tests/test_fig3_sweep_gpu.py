"""The final height of a frozen liquid column against the density ratio of
solid and liquid (Section 4.1, Eq. 44, the sweep of Fig. 3) on the GPU: one
batched handle of short columns, one per rho_s / rho_l, each frozen from its
cold wall until it stops freezing. Mass conservation through the phase
change gives H_f / H_0 = rho_l / rho_s."""
import pytest

from paper_2403_16122_gb300 import inputs

pytestmark = pytest.mark.gpu

RATIOS = (0.8, 0.85, 0.9, 0.95, 1.0, 1.05, 1.1)
H0 = 16


def test_final_height_against_density_ratio():
    from paper_2403_16122_gb300 import lbm

    cases = []
    for sl in RATIOS:
        # closed column of 48 cells (cold Dirichlet wall at one end, adiabatic
        # wall at the other, periodic across), liquid on the first H0 cells,
        # gas of density ratio 1000 above it
        p, phi0, T0 = inputs.stefan(nx=48, ny=4, H0=H0, Ste=0.25, rho_ratio_sl=sl)
        p.update(rho_ratio_lg=1000.0, mu_ratio_lg=100.0)
        cases.append((p, phi0, T0))
    lat = lbm.Lattice([c[0] for c in cases])
    for k, (_, phi0, T0) in enumerate(cases):
        lat.init(phi0, T0, inst=k)
    lat.set_exec(lbm.LBM_EXEC_GRAPH, 100)
    done = [None] * len(RATIOS)
    for _ in range(60):
        lat.step(500)
        obs = lat.observables_all()
        for k in range(len(RATIOS)):
            v, s, md = (obs[k, lbm.OBS_NAMES.index(n)] for n in ("volume", "solid", "mdot"))
            # frozen: almost all of the drop solid and no more phase change
            if done[k] is None and s / v > 0.97 and abs(md) < 1e-4:
                done[k] = v / cases[k][0]["ny"]
        if all(d is not None for d in done):
            break
    for sl, hf in zip(RATIOS, done):
        print(f"rho_s/rho_l {sl}: H_f/H_0 {hf / H0:.5f}, rho_l/rho_s {1 / sl:.5f}")
        assert hf is not None
        assert hf / H0 == pytest.approx(1.0 / sl, rel=0.01)
    lat.close()
