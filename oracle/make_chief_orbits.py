"""Write the three periodic chief orbits used by the paper-scale workload.

Calls only the oracle (its DOPRI5 propagator and the differential corrector in
``oracle/periodic.py``).  Output: ``paper_2207_13175_gb300/chief_orbits.json``.
Run from the repository root:  python -m oracle.make_chief_orbits
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import jacobi
from . import periodic as P

MU = 0.01215058560962404


def main() -> None:
    orbits = {}
    for name, fn in (("lyapunov", P.lyapunov_l1), ("halo", P.halo_l2_north), ("dro", P.dro)):
        s0, thalf = fn(MU)
        period = 2.0 * thalf
        ret = float(np.max(np.abs(P.state_at(MU, s0, period) - s0)))
        orbits[name] = {"state": [float(v) for v in s0], "period_tu": float(period),
                        "jacobi": float(jacobi(MU, s0)), "return_error": ret}
    doc = {"mu": MU, "written_by": "python -m oracle.make_chief_orbits",
           "family": {"lyapunov": "L1 planar Lyapunov, x0 = x_L1 - 0.02",
                      "halo": "L2 northern halo, z0 = +0.05 at the far x-axis crossing",
                      "dro": "distant retrograde orbit, x0 = 1 - mu + 0.2, vy0 < 0"},
           "orbits": orbits}
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = os.path.join(root, "paper_2207_13175_gb300", "chief_orbits.json")
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
