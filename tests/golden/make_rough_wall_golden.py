"""Write the stored oracle values of the full-size rough-wall parity test.

    python tests/golden/make_rough_wall_golden.py [steps]

Runs the FP64 CPU oracle (``oracle/``, nothing else of this repository but
the seeded input generator) for 20 time steps of the 2,082,816-node
rough-wall droplet (width 2048, 1017 body-fitted rows on the wall
y = 8 + 4 sin(2 pi x / 64), jitter 0.2h from seed 4, R 300, contact angle
60 degrees, density ratio 100, dt 0.1) and stores g and h at a seeded
sample of nodes -- 4,096 drawn uniformly from default_rng(2024) plus every
8th node of the rough wall -- with the global diagnostics, in
``rough_wall_20_steps.npz`` beside this script.  The oracle takes minutes
and several GB here, which is why the parity test compares against these
stored values instead of running it.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import OracleMesh, OracleSim, params_from_physical  # noqa: E402
from paper_1708_04678_gb300 import inputs as I  # noqa: E402


def sample_nodes(mesh):
    n = len(mesh["xy"])
    rng = np.random.default_rng(2024)
    rand = rng.choice(n, size=4096, replace=False)
    wall = np.unique(mesh["wall_edges"][mesh["wall_id"] == 0].reshape(-1))[::8]
    return np.unique(np.concatenate([rand, wall])).astype(np.int64)


def main(steps=20):
    w = I.rough_wall_droplet()
    m = w["mesh"]
    t0 = time.time()
    sim = OracleSim(OracleMesh(m["xy"], m["tri"], m["wall_edges"], m["wall_id"], m["period"]),
                    params_from_physical(w["phys"]), w["C0"])
    print(f"oracle mesh: {time.time() - t0:.1f} s", flush=True)
    for k in range(steps):
        t1 = time.time()
        sim.step(1)
        print(f"step {k + 1}: {time.time() - t1:.1f} s, PCG iterations {sim.last_iters}", flush=True)
    nodes = sample_nodes(m)
    d = sim.diagnostics(w["centre"], w["R"], w["phys"]["xi"], 0)
    np.savez_compressed(os.path.join(HERE, "rough_wall_20_steps.npz"), steps=steps, nodes=nodes,
                        g=sim.g[:, nodes], h=sim.h[:, nodes],
                        diag_names=np.array(sorted(d)), diag_values=np.array([d[k] for k in sorted(d)]))
    print(f"wrote {len(nodes)} nodes after {steps} steps in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 20)
