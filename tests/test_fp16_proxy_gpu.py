"""Reduced-precision storage against the FP64 oracle at the scale of the
bubble-drop benchmark's accuracy proxy: the 256 x 256 drop with 8 gas bubbles
freezing on a cold wall (Section 4.3's structure) for 20000 steps, observed
every 2000 steps. The oracle's values come from tests/golden/
bubble_drop_256_oracle.txt (written by make_bubble_drop_256.py beside it,
which calls only the oracle). Bar for FP16 and BF16 storage: front height at
the centre column within 0.5 lattice units, solidified amount and drop volume
within 1 %; FP32 storage is held far tighter."""
import os

import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bubble_drop_256_oracle.txt")


def _golden():
    rows = [list(map(float, line.split())) for line in open(GOLDEN)
            if line.strip() and not line.startswith("#")]
    return {int(r[0]): dict(volume=r[1], solid=r[2], solid_col=r[3], enthalpy=r[4],
                            mdot_integral=r[5]) for r in rows}


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_bubble_drop_256_against_oracle_20000_steps(storage):
    from paper_2403_16122_gb300 import lbm

    gold = _golden()
    assert max(gold) == 20000
    st = {"fp32": lbm.LBM_STORE_FP32, "fp16": lbm.LBM_STORE_FP16,
          "bf16": lbm.LBM_STORE_BF16}[storage]
    p, phi0, T0 = inputs.bubbles_drop(n=256)
    lat = lbm.Lattice([p], storage=st).init(phi0, T0)
    worst = dict(front=0.0, solid=0.0, volume=0.0)
    for step in sorted(gold):
        lat.step(step - lat.step_count)
        ob, g = lat.observables(), gold[step]
        worst["front"] = max(worst["front"], abs(ob["solid_col"] - g["solid_col"]))
        worst["solid"] = max(worst["solid"], abs(ob["solid"] / g["solid"] - 1))
        worst["volume"] = max(worst["volume"], abs(ob["volume"] / g["volume"] - 1))
        fr = lat.freezing()
        if storage == "fp32":
            assert fr["mdot_integral"] == pytest.approx(g["mdot_integral"], rel=1e-4)
    print(storage, "worst over 2000..20000 steps:", worst, "final front",
          gold[20000]["solid_col"])
    assert gold[20000]["solid_col"] > 15  # the front travels well over the bar's scale
    if storage == "fp32":
        assert worst["front"] <= 0.01 and worst["solid"] <= 1e-4 and worst["volume"] <= 1e-4
    else:
        assert worst["front"] <= 0.5 and worst["solid"] <= 0.01 and worst["volume"] <= 0.01
    assert np.isfinite(lat.get_state()[0]).all()
