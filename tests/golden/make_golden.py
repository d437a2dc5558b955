"""Write tests/golden/oracle_regression.json from the FP64 oracle alone.

The paper prints no worked example, so the stored values are the oracle's own
output on a small seeded case (16 packets, 4^3 grid, CIC and TSC, 10 steps in
the config-1 fields B = x, E = 0.01 z, c = 1, c~ = 0.1, dt = 0.2 / c~).  They
are a regression guard: a later change to the oracle's arithmetic must name the
passage of the paper that justifies it before this file is regenerated.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import rsol_inputs as ri  # noqa: E402


def case(shape):
    grid = (4, 4, 4)
    F = ri.field_grid(grid, B0=1.0, u_gas=(0.0, 0.01, 0.0))
    parts = ri.make_particles(16, grid, seed=1)
    p = oracle.params(grid, shape=shape, dt=2.0, c=1.0, c_tilde=0.1)
    P = oracle.Particles(parts)
    G = None
    for _ in range(10):
        G = oracle.step(p, F, P)
    return {"shape": shape, "cell": P.cell.tolist(), "off": P.off.tolist(), "u": P.u.tolist(),
            "deposit_last_step_sums": G.sum(axis=(1, 2, 3)).tolist(),
            "deposit_last_step_node0": G[:, 0, 0, 0].tolist()}


if __name__ == "__main__":
    out = {"source": "oracle/rsol_oracle.c via tests/golden/make_golden.py",
           "cases": [case(1), case(2)]}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
