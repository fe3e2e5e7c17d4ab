"""Write tests/golden/bubble_drop_256_oracle.txt: observables of the FP64
oracle on the 256 x 256 version of the bubble-drop workload (a drop of radius
80 with 8 gas bubbles freezing on a cold wall, Section 4.3's structure),
every 2000 steps up to 20000. The reduced-precision GPU tests compare 16-bit
storage against these values. Calls only the oracle and the input generator:

    python tests/golden/make_bubble_drop_256.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2403_16122_gb300 import inputs  # noqa: E402

N, STEPS, EVERY = 256, 20000, 2000
OUT = os.path.join(HERE, "bubble_drop_256_oracle.txt")


def main():
    oracle.build()
    threads = oracle.set_threads(0)
    p, phi0, T0 = inputs.bubbles_drop(n=N)
    o = oracle.Oracle(p).init(phi0, T0)
    t0 = time.perf_counter()
    lines = ["# FP64 oracle, inputs.bubbles_drop(n=256) (seed 20240324): step volume solid "
             "solid_col enthalpy mdot_integral",
             "# volume = sum phi, solid = sum f_s, solid_col = sum_y f_s at x = nx/2 (front "
             "height at the centre column), enthalpy = sum H, mdot_integral = sum over steps "
             "and sites of mdot (Eq. 19)"]
    while o.step_count < STEPS:
        o.step(EVERY)
        ob = o.observables()
        lines.append(f"{o.step_count} {ob['volume']!r} {ob['solid']!r} {ob['solid_col']!r} "
                     f"{ob['enthalpy']!r} {o.mdot_integral!r}")
        print(lines[-1], f"({time.perf_counter() - t0:.0f} s, {threads} threads)", flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
