"""Writes search_c3_reduced.json: the oracle's exact uniform-cost search
(Sec. IV-B with h0 = 0 and w = 1; set-keyed states, Sec. IV-A) on the
heavy-occlusion setting (640x480, three of the eight uneven 2k-50k-triangle
meshes, one object more than 30% hidden behind a taller one) with a coarse
pose grid of 8 x 8 positions x 4 yaws, for two seeded scenes. The GPU search
must return the same cost and scene (tests/test_gpu_search_c2.py). Only
oracle/ computes the values; the seeded inputs come from the generator
package.

    python tests/golden/make_search_c3_reduced.py      (minutes per scene on 8 cores)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import search  # noqa: E402
from paper_1510_05613_gb300 import synth  # noqa: E402

GRID = dict(x0=-0.49, step=0.14, n=8, n_yaw=4)
SCENES = (0, 2)


def main():
    out = {"what": "oracle uniform-cost search, 640x480 heavy-occlusion setting with three of the uneven "
                   "meshes, pose grid reduced to 8 x 8 positions (x0 -0.49 m, step 0.14 m) x 4 yaws",
           "grid": GRID, "scenes": []}
    for scene in SCENES:
        grid = synth.pose_grid(GRID["x0"], GRID["step"], GRID["n"], GRID["n_yaw"])
        wl = synth.workload_c3_reduced(scene=scene, grid=grid)
        w = oracle.World.of(wl)
        t0 = time.time()
        cost, key, expansions = search.uniform_cost_search(w, wl.depth, wl.grid, wl.mesh_multiset)
        out["scenes"].append({"scene": scene, "cost": int(cost), "key": [list(map(int, o)) for o in key],
                              "occlusion": [round(float(x), 3) for x in wl.extra["occlusion"]],
                              "oracle_expansions": int(expansions), "oracle_seconds": round(time.time() - t0, 1)})
        print(out["scenes"][-1], flush=True)
    with open(os.path.join(HERE, "search_c3_reduced.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
