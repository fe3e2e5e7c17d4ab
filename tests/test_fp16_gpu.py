"""FP16 shifted-distribution storage (FP32 arithmetic) against the FP64 oracle
and the FP32 path: front height within 0.5 lattice units, solidified amount and
drop volume within 1 % after thousands of steps; state round trip and
single-step accuracy."""
import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs
from parity_util import gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_16122_gb300 import build
    build.build()


def _cases():
    return {
        "sessile": inputs.sessile(nx=96, ny=64, R=24.0, theta_deg=100.0),
        "bubbles": inputs.bubbles_drop(n=96, n_bub=2, r_lo=4.0, r_hi=6.0, seed=21),
    }


@pytest.mark.parametrize("case", ["sessile", "bubbles"])
def test_fp16_observables_match_oracle(oracle_mod, case):
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = _cases()[case]
    steps = 2000
    h16 = gpu_run([p], [(phi0, T0)], steps, storage=lbm.LBM_STORE_FP16)
    o = oracle_run(oracle_mod, p, phi0, T0, steps)
    g, r = h16.observables(), o.observables()
    f = gpu_run([p], [(phi0, T0)], steps).observables()
    print(case, {k: (g[k], f[k], r[k]) for k in ("volume", "solid", "solid_col", "enthalpy")})
    assert r["solid"] > 5.0
    assert g["volume"] == pytest.approx(r["volume"], rel=0.01)
    assert g["solid"] == pytest.approx(r["solid"], rel=0.01)
    assert abs(g["solid_col"] - r["solid_col"]) <= 0.5   # centre freezing height
    assert g["nonfinite"] == 0.0
    # populations stay close to the FP64 state
    gp, _ = h16.get_state()
    op, _ = o.get_state()
    assert np.abs(gp - op).max() < 2e-3


def test_fp16_one_step_from_common_state(oracle_mod):
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = inputs.sessile(nx=80, ny=60, R=20.0, theta_deg=60.0)
    o = oracle_run(oracle_mod, p, phi0, T0, 200)
    pops, aux = o.get_state()
    lat = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_FP16)
    lat.set_state(pops, aux)
    back = lat.get_state()
    # encoding error of the stored deviations
    assert np.abs(back[0] - pops).max() < 2e-5
    lat.step(1)
    o.step(1)
    gp, ga = lat.get_state()
    op, oa = o.get_state()
    assert np.abs(gp - op).max() < 5e-5
    assert np.abs(ga - oa).max() < 5e-5


def test_fp16_requires_periodic_x_and_strip_layout():
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = inputs.stefan(nx=64)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_size([p], lbm.LBM_STORE_FP16)
    p, phi0, T0 = inputs.sessile(nx=64, ny=48, R=16.0)
    lat = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_FP16)
    assert lat.kernel[0] == lbm.LBM_KERNEL_STAGED
    with pytest.raises(lbm.LbmError):
        lat.set_kernel(lbm.LBM_KERNEL_TILE, 32, 8)
    for v in [(4, 16, 168), (4, 8, 128), (4, 16, 255)]:
        lat.set_kernel(lbm.LBM_KERNEL_STRIP, *v)
        lat.step(5)
    assert np.isfinite(lat.get_state()[0]).all()


STAGED_VARIANTS = [(4, 16, 168), (4, 3, 128), (8, 32, 128), (2, 2, 128), (4, 5, 255), (4, 0, 168)]


@pytest.mark.parametrize("case", ["sessile", "bubbles", "periodic"])
def test_fp16_staged_matches_plain_strip(case):
    """The row-staged strip layout decodes the same 16-bit words as the plain
    one, for every variant, over 60 steps. The kernels are compiled apart and
    may fuse a different a * b + c into one rounding, so a stored deviation
    can round to the neighbouring 16-bit value and the two runs drift apart
    at the moving interface (measured up to 1e-4); a slip in the layout (a
    word of the wrong plane, half or reference) is an error of 1e-2 or more.
    The one-step test below bounds the per-step difference itself."""
    from paper_2403_16122_gb300 import lbm

    if case == "periodic":
        p = inputs.params(nx=71, ny=33, periodic_x=1, periodic_y=1)
        phi0, T0 = inputs.random_state(p, seed=6)
    else:
        p, phi0, T0 = _cases()[case]
    ref = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_FP16)
    ref.set_kernel(lbm.LBM_KERNEL_STRIP, 4, 16, 168)
    ref.step(60)
    want = ref.get_state()
    for v in STAGED_VARIANTS:
        lat = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_FP16)
        lat.set_kernel(lbm.LBM_KERNEL_STAGED, *v)
        lat.step(60)
        got = lat.get_state()
        d = (np.abs(got[0] - want[0]).max(), np.abs(got[1] - want[1]).max())
        print(case, v, "max |dpop|, |daux| after 60 steps:", d)
        assert d[0] <= 1e-3 and d[1] <= 1e-3, (v, d)


def test_fp16_staged_matches_plain_strip_one_step(oracle_mod):
    """One step of every staged variant and of the plain strip from one stored
    FP16 state (the oracle's after 200 steps of a drop with flow): the
    kernels evaluate the same expressions, so they differ by FP32 rounding
    and, where that moves a value across a 16-bit rounding boundary, by one
    unit in the last place of a stored deviation, 2^-10 of it at most (the
    deviations here stay below 0.02)."""
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = inputs.sessile(nx=80, ny=60, R=20.0, theta_deg=60.0)
    o = oracle_run(oracle_mod, p, phi0, T0, 200)
    pops, aux = o.get_state()
    ref = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_FP16)
    ref.set_kernel(lbm.LBM_KERNEL_STRIP, 4, 16, 168)
    ref.set_state(pops, aux)
    ref.step(1)
    want = ref.get_state()
    for v in STAGED_VARIANTS:
        lat = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_FP16)
        lat.set_kernel(lbm.LBM_KERNEL_STAGED, *v)
        lat.set_state(pops, aux)  # the same words as ref's
        lat.step(1)
        got = lat.get_state()
        d = (np.abs(got[0] - want[0]).max(), np.abs(got[1] - want[1]).max())
        print(v, "max |dpop|, |daux| after one step:", d)
        assert d[0] <= 2e-5 and d[1] <= 2e-5, (v, d)


def _crossing_times(t, X, thr):
    """Per lattice: first time X reaches thr, linear between observations
    (nan if it never does)."""
    out = np.full(X.shape[1], np.nan)
    for k in range(X.shape[1]):
        idx = np.nonzero(X[:, k] >= thr)[0]
        if len(idx) == 0 or idx[0] == 0:
            continue
        j = idx[0]
        x0, x1 = X[j - 1, k], X[j, k]
        out[k] = t[j - 1] + (thr - x0) / (x1 - x0) * (t[j] - t[j - 1])
    return out


def test_fp16_batched_freezing_time_within_one_percent():
    """A batch of small drops with bubbles, advanced in one persistent launch
    per 250 steps: in FP16 storage each drop reaches solidified fractions
    X = solid / volume of 0.5 and 0.9 within 1 % of the time it takes in FP32
    storage (the FP32 path itself is held to the oracle elsewhere)."""
    from paper_2403_16122_gb300 import lbm

    cases = inputs.batched_bubbles(n_inst=6, lo=40, hi=56, seed=11)
    every, n_obs = 250, 80
    i_s, i_v = lbm.OBS_NAMES.index("solid"), lbm.OBS_NAMES.index("volume")

    def run(storage):
        lat = lbm.Lattice([c[0] for c in cases], storage=storage)
        for k, (_, phi0, T0) in enumerate(cases):
            lat.init(phi0, T0, inst=k)
        lat.set_exec(lbm.LBM_EXEC_PERSISTENT, every - 1)
        X = []
        for _ in range(n_obs):
            o = lat.step(every).observables_all()
            X.append(o[:, i_s] / o[:, i_v])
        lat.close()
        return np.array(X)

    t = every * np.arange(1, n_obs + 1, dtype=float)
    X32, X16 = run(lbm.LBM_STORE_FP32), run(lbm.LBM_STORE_FP16)
    checked = 0
    for thr in (0.5, 0.9):
        t32, t16 = _crossing_times(t, X32, thr), _crossing_times(t, X16, thr)
        print("X =", thr, "t32", np.round(t32, 1), "t16", np.round(t16, 1))
        for a, b in zip(t32, t16):
            if np.isnan(a):
                continue
            assert not np.isnan(b)
            assert abs(b - a) <= 0.01 * a, (thr, a, b)
            checked += 1
    assert checked >= 6  # every drop crosses 0.5 within the run


@pytest.mark.parametrize("case", ["sessile", "bubbles"])
def test_bf16_observables_match_oracle(oracle_mod, case):
    """BF16 storage (7-bit mantissa) in the same shifted arrangement: the
    freezing observables after 2000 steps hold the reduced-precision bar
    (volume and solidified amount within 1 %, centre front height within
    0.5 lattice units)."""
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = _cases()[case]
    steps = 2000
    hb = gpu_run([p], [(phi0, T0)], steps, storage=lbm.LBM_STORE_BF16)
    assert hb.kernel[0] == lbm.LBM_KERNEL_STAGED
    o = oracle_run(oracle_mod, p, phi0, T0, steps)
    g, r = hb.observables(), o.observables()
    print(case, "bf16", {k: (g[k], r[k]) for k in ("volume", "solid", "solid_col")})
    assert g["volume"] == pytest.approx(r["volume"], rel=0.01)
    assert g["solid"] == pytest.approx(r["solid"], rel=0.01)
    assert abs(g["solid_col"] - r["solid_col"]) <= 0.5
    assert g["nonfinite"] == 0.0


def test_bf16_one_step_from_common_state(oracle_mod):
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = inputs.sessile(nx=80, ny=60, R=20.0, theta_deg=60.0)
    o = oracle_run(oracle_mod, p, phi0, T0, 200)
    pops, aux = o.get_state()
    lat = gpu_run([p], [(phi0, T0)], 0, storage=lbm.LBM_STORE_BF16)
    lat.set_state(pops, aux)
    # 8 significant bits of each deviation from its rest equilibrium
    assert np.abs(lat.get_state()[0] - pops).max() < 2e-4
    lat.step(1)
    o.step(1)
    gp, ga = lat.get_state()
    op, oa = o.get_state()
    assert np.abs(gp - op).max() < 4e-4
    assert np.abs(ga - oa).max() < 4e-4
    with pytest.raises(lbm.LbmError):
        lat.set_kernel(lbm.LBM_KERNEL_STRIP, 4, 16, 168)  # BF16: staged strips only


def test_16bit_storage_at_benchmark_size():
    """The precision bar at the benchmark's own size and length: the 1024 x
    1024 drop with 8 bubbles on the cold wall, 100,000 steps (the front moves
    some 40 cells), in FP16 and BF16 storage against FP32 storage on the same
    GPU: front height at the centre column within 0.5 lu, solidified amount
    and volume within 1 %."""
    from paper_2403_16122_gb300 import lbm

    p, phi0, T0 = inputs.bubbles_drop(n=1024)
    steps = 100_000
    res = {}
    for name, st in (("fp32", lbm.LBM_STORE_FP32), ("fp16", lbm.LBM_STORE_FP16),
                     ("bf16", lbm.LBM_STORE_BF16)):
        lat = gpu_run([p], [(phi0, T0)], 0, storage=st)
        lat.step(steps)
        res[name] = lat.observables()
        lat.close()
    ref = res["fp32"]
    assert ref["solid_col"] > 30 and ref["nonfinite"] == 0
    for name in ("fp16", "bf16"):
        o = res[name]
        d = {"front": o["solid_col"] - ref["solid_col"],
             "solid": o["solid"] / ref["solid"] - 1.0,
             "volume": o["volume"] / ref["volume"] - 1.0}
        print(name, "after", steps, "steps at 1024x1024 against FP32:", d,
              {k: (o[k], ref[k]) for k in ("solid_col", "solid", "volume")})
        assert abs(d["front"]) <= 0.5, (name, d)
        assert abs(d["solid"]) <= 0.01 and abs(d["volume"]) <= 0.01, (name, d)
