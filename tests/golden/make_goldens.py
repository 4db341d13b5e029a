"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (oracle/) on seeded inputs from wmcgen.

    python tests/golden/make_goldens.py

grid_24x200.json: W(phi) of the 24x200 grid CNF (seeds 0 and 1) with
w(x) ~ U(0.05, 0.95), w(~x) = 1 - w(x) (weight seed = formula seed), by
long-double bucket elimination along the column sweep.  Too slow to
recompute inside the test suite.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import wmcgen  # noqa: E402


def grid_golden(H, W, seeds):
    out = []
    for seed in seeds:
        cnf = wmcgen.grid_cnf(H, W, seed)
        wp, wn = wmcgen.weights_complementary(H * W, seed, 0.05, 0.95)
        col = [i * W + j + 1 for j in range(W) for i in range(H)]
        t = time.time()
        v, width = oracle.bucket_elim(cnf, wp, wn, order=col, return_width=True)
        out.append({"seed": seed, "mant": v.mant, "exp2": v.exp2, "log10": v.log10(),
                    "oracle_width": width, "oracle_seconds": round(time.time() - t, 1),
                    "oracle_threads": oracle.num_threads()})
        print(out[-1], flush=True)
    return out


if __name__ == "__main__":
    data = {
        "what": "W(phi) of grid_cnf(24, 200, seed) with weights_complementary(4800, seed, 0.05, 0.95)",
        "method": "oracle.bucket_elim, long double, column-sweep order",
        "values": grid_golden(24, 200, [0, 1]),
    }
    with open(os.path.join(HERE, "grid_24x200.json"), "w") as f:
        json.dump(data, f, indent=1)
