"""Count the work of each benchmark frame with the CPU oracle.

For every benchmark workload (the same seeded sets and cameras the benchmark
renders) the oracle counts the active particles, the covered (particle, pixel)
pairs (one Gaussian kernel evaluation each, Section 2.1) and the (particle,
tile) pairs of the tile rule (Section 3.2.1) at the default tile edge.  The
benchmark divides the splat's algorithmic arithmetic, stated per covered pair,
by its measured time; these counts fix the number of units, independently of
the kernels.  FP16 workloads are counted on FP16-rounded attributes, as the
GPU renders them.

Writes ``work_units.json`` beside this script.  Run once; the counts are frozen.
    python tests/golden/freeze_work.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1606_04427_gb300 import synth  # noqa: E402

TILE = 32


def main():
    res = {"tile": TILE, "units": "active particles; covered (particle, pixel) pairs; (particle, tile) pairs"}
    t0 = time.time()
    big = synth.two_species_set(70_000_000, 30_000_000, 2)
    cam = synth.front_camera(2048, 2048)
    res["two_species_f16"] = oracle.count_work(big, cam, storage="f16", tile=TILE)
    res["two_species_f32"] = oracle.count_work(big, cam, storage="f32", tile=TILE)
    del big
    small = synth.two_species_set(7_000_000, 3_000_000, 2)
    res["two_species_small"] = oracle.count_work(small, cam, storage="f16", tile=TILE)
    del small
    res["clustered"] = oracle.count_work(synth.clustered_set(10_000_000, 1), synth.front_camera(1024, 1024),
                                         storage="f32", tile=TILE)
    res["plain"] = oracle.count_work(synth.plain_set(100_000, 0), synth.front_camera(256, 256), tile=TILE)
    batched = synth.clustered_set(20_000_000, 3)
    views = [oracle.count_work(batched, c, storage="f16", tile=TILE) for c in synth.orbit_cameras(64, 1024, 1024)]
    res["batched_f16"] = {k: sum(v[k] for v in views) for k in views[0]}
    res["seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, "work_units.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
