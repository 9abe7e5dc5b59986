"""Writes oracle_regression.txt: one Algorithm 1 call of the oracle on three
small seeded scenes (iterations, searches, sum of |P|, contacts and a SHA-256
of x^{t+1}).  It calls only oracle/ and the seeded input generator.  Run it
after an intentional change of the oracle's arithmetic, and name the reading
that justifies the change in the commit message.

    python tests/golden/make_oracle_regression.py
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2211_04045_gb300 import scenes  # noqa: E402

CASES = {
    "cloth_sphere": lambda: scenes.cloth_over_sphere(n=10, side=0.5, sphere_subdiv=1, sphere_r=0.15, noise=0.3,
                                                     seed=1),
    "two_cloths": lambda: scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2),
    "hair_sand": lambda: scenes.hair_sand(n_strands=36, segs=8, n_points=120, grain_r=0.002, bowl_r=0.12,
                                          bowl_subdiv=2, seg_len=0.01, seed=4),
}
VARIANTS = {"gs": {}, "gs_greedy": {"colouring": 0}, "jacobi": {"solver": 1}, "jacobi3": {"solver": 1, "gs_sweeps": 3},
            "gap": {"constraint_form": 1}, "ccd_rule": {"step_rule": 1}}


def record(name, variant):
    sc = CASES[name]()
    x, xt, _ = scenes.initial(sc)
    prm = oracle.params_for(sc, max_iters=200, **VARIANTS[variant])
    xn, st, _ = oracle.handle_step(oracle.OracleScene(sc), prm, x, xt)
    h = hashlib.sha256(np.ascontiguousarray(xn, dtype="<f8").tobytes()).hexdigest()
    return (f"{name} {variant} iterations={st['iterations']} searches={st['searches']} "
            f"pairs={st['pairs_evaluated']} contacts={st['active_contacts']} sha256={h}")


def lines():
    return [record(n, v) for n in CASES for v in VARIANTS]


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as f:
        f.write("# written by make_oracle_regression.py; one line per scene and variant (backward step or step rule)\n")
        for line in lines():
            f.write(line + "\n")
