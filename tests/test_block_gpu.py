"""The block kernel (one warp per 32-site column of row blocks, rows staged by
bulk copies) against the FP64 oracle and the other layouts: walls with
bounce-back and anti-bounce-back, wetting at several angles, partial last
blocks (nx not a multiple of 32, down to one site), lattices narrower than a
block, periodic y, bubbles with the liquid-masked surface tension, 16-bit
storage, and the graph and persistent forms."""
import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs
from parity_util import compare_state, max_abs

pytestmark = pytest.mark.gpu

VARIANTS = [(4, 168), (4, 128), (8, 128)]


@pytest.fixture(scope="module")
def lbm():
    from paper_2403_16122_gb300 import build, lbm as _lbm
    build.build()
    _lbm.load()
    return _lbm


def _block(lbm, params, fields, warps=4, regs=168, rows=0, storage=0):
    lat = lbm.Lattice(params, storage=storage)
    for k, (phi0, T0) in enumerate(fields):
        lat.init(phi0, T0, inst=k)
    lat.set_kernel(lbm.LBM_KERNEL_BLOCK, warps, rows, regs)
    return lat


@pytest.mark.parametrize("warps,regs", VARIANTS)
def test_block_sessile_ragged_1000_steps(lbm, oracle_mod, warps, regs):
    """Sessile drop, density ratio 1000, cold Dirichlet wall below, wetting at
    100 deg, 70 x 44 (the last block holds 6 columns): the 1000-step bar."""
    p, phi0, T0 = inputs.sessile(nx=70, ny=44, R=16.0, theta_deg=100.0)
    lat = _block(lbm, [p], [(phi0, T0)], warps, regs, rows=8)
    lat.step(1000)
    o = oracle_mod.Oracle(p).init(phi0, T0).step(1000)
    d = compare_state(lat.get_state(), o.get_state())
    print(warps, regs, d)
    ob, obo = lat.observables(), o.observables()
    assert obo["solid"] > 10
    assert ob["solid"] == pytest.approx(obo["solid"], rel=1e-5)
    assert ob["volume"] == pytest.approx(obo["volume"], rel=5e-6)


@pytest.mark.parametrize("nx,ny,py,theta", [(33, 20, 0, 45.0), (4, 9, 1, 90.0), (31, 12, 0, 120.0),
                                            (64, 17, 1, 90.0)])
def test_block_edge_cases(lbm, oracle_mod, nx, ny, py, theta):
    """Blocks of one site (nx = 33), lattices narrower than a block (4, 31),
    periodic y, exact multiples of 32; perturbed drop-like fields, 300
    steps."""
    p = inputs.params(nx=nx, ny=ny, periodic_x=1, periodic_y=py, dirichlet_y_lo=0 if py else 1,
                      theta_deg=theta, rho_ratio_lg=100.0, mu_ratio_lg=30.0, rho_ratio_sl=0.92)
    phi0, T0 = inputs.random_state(p, seed=11)
    lat = _block(lbm, [p], [(phi0, T0)], rows=4)
    lat.step(300)
    o = oracle_mod.Oracle(p).init(phi0, T0).step(300)
    d = compare_state(lat.get_state(), o.get_state())
    print(nx, ny, py, d)


def test_block_bubbles_masked_surface_tension(lbm, oracle_mod):
    """Bubbles in a drop with the liquid-masked surface tension, 500 steps."""
    rng = np.random.default_rng(3)
    p = inputs.params(nx=96, ny=64, periodic_x=1, periodic_y=0, dirichlet_y_lo=1, theta_deg=80.0,
                      st_mask_liquid=1)
    phi = inputs.cap(96, 64, 26.0, 80.0, p["W"])
    phi = inputs.with_bubbles(phi, inputs.place_bubbles(rng, 96, 64, 26.0, 80.0, p["W"], 3, 4.0,
                                                        6.0), p["W"])
    T0 = np.full((64, 96), p["T_m"])
    lat = _block(lbm, [p], [(phi, T0)])
    lat.step(500)
    o = oracle_mod.Oracle(p).init(phi, T0).step(500)
    compare_state(lat.get_state(), o.get_state())


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_block_matches_staged_one_step_full_size(lbm, storage):
    """One step of the 1024 x 1024 bubble drop from a common state: block
    against the row-staged strips, every site (FP32 rounding; 16-bit storage
    decodes the same stored words)."""
    st = {"fp32": lbm.LBM_STORE_FP32, "fp16": lbm.LBM_STORE_FP16, "bf16": lbm.LBM_STORE_BF16}[storage]
    p, phi0, T0 = inputs.bubbles_drop(n=1024)
    a = lbm.Lattice([p], storage=st).init(phi0, T0)
    a.set_kernel(lbm.LBM_KERNEL_STAGED, 4, 0, 168)
    a.step(20)
    pops, aux = a.get_state()
    b = lbm.Lattice([p], storage=st).set_state(pops, aux)
    b.set_kernel(lbm.LBM_KERNEL_BLOCK, 4, 0, 168)
    a.set_state(pops, aux)
    a.step(1)
    b.step(1)
    ga, gb = a.get_state(), b.get_state()
    tol = 2e-6 if storage == "fp32" else 5e-4
    assert max_abs(ga[0], gb[0]) <= tol
    assert max_abs(ga[1], gb[1]) <= tol
    oa, ob_ = a.observables(), b.observables()
    assert ob_["volume"] == pytest.approx(oa["volume"], rel=1e-6)
    assert ob_["solid"] == pytest.approx(oa["solid"], rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_block_16bit_observables_match_oracle(lbm, oracle_mod, storage):
    """16-bit storage in the block kernel: a sessile drop and a drop with
    bubbles after 2000 steps within the reduced-precision bar of the FP64
    oracle (front height 0.5 lu, solid and volume 1 %)."""
    st = lbm.LBM_STORE_FP16 if storage == "fp16" else lbm.LBM_STORE_BF16
    p, phi0, T0 = inputs.sessile(nx=96, ny=64, R=24.0, theta_deg=100.0, rho_ratio_lg=10.0,
                                 mu_ratio_lg=10.0)
    lat = _block(lbm, [p], [(phi0, T0)], storage=st)
    lat.step(2000)
    o = oracle_mod.Oracle(p).init(phi0, T0).step(2000)
    ob, obo = lat.observables(), o.observables()
    print(storage, {k: (ob[k], obo[k]) for k in ("solid", "volume", "solid_col")})
    assert ob["solid"] == pytest.approx(obo["solid"], rel=0.01)
    assert ob["volume"] == pytest.approx(obo["volume"], rel=0.01)
    assert abs(ob["solid_col"] - obo["solid_col"]) <= 0.5


@pytest.mark.parametrize("mode", ["graph", "persistent"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_block_execution_forms(lbm, mode, storage):
    """Several uneven lattices in one handle: graph replay equals per-step
    launches bit for bit; the persistent form (a separately compiled kernel)
    agrees to FP32 rounding."""
    st = lbm.LBM_STORE_FP32 if storage == "fp32" else lbm.LBM_STORE_FP16
    cases = [inputs.sessile(nx=70, ny=44, R=16.0, theta_deg=100.0),
             inputs.sessile(nx=40, ny=30, R=10.0, theta_deg=60.0)]
    ref = _block(lbm, [c[0] for c in cases], [c[1:] for c in cases], storage=st)
    ref.step(120)
    lat = _block(lbm, [c[0] for c in cases], [c[1:] for c in cases], storage=st)
    lat.set_exec(lbm.LBM_EXEC_GRAPH if mode == "graph" else lbm.LBM_EXEC_PERSISTENT, 16)
    lat.step(120)
    tol = 0.0 if mode == "graph" else (1e-6 if storage == "fp32" else 1e-3)
    for k in range(2):
        a, b = ref.get_state(k), lat.get_state(k)
        assert max_abs(a[0], b[0]) <= tol and max_abs(a[1], b[1]) <= tol, (k, max_abs(a[0], b[0]))
