"""Freeze the brightness of each synthetic workload from the CPU oracle.

Rule: with brightness 1 the oracle renders the workload's reference frame; the
brightness of each species is set so that the 99th-percentile pixel (largest
channel of the accumulation a) reaches a = 3, so the final transform 1 - exp(-a)
is neither trivially dark nor saturated everywhere and parity stays informative.
Species are rendered alone to set their own brightness.  The served sets share
the clustered distribution; since a grows linearly with the particle count for a
fixed distribution, set k gets the 1 M-particle value times 1e6 / N_k.

Writes ``brightness.json`` beside this script.  Run once; the values are frozen.
    python tests/golden/freeze_brightness.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1606_04427_gb300 import synth  # noqa: E402


def a99(ps, cam):
    a = oracle.render(ps.with_brightness(np.ones(ps.n_types)), cam)
    return float(np.percentile(a.max(axis=2), 99.0))


def per_species(ps, cam):
    out = []
    for t in range(ps.n_types):
        idx = np.arange(ps.type_begin[t], ps.type_begin[t + 1])
        out.append(3.0 / a99(ps.subset(idx), cam))
    return out


def main():
    res = {"rule": "99th-percentile pixel (max channel of a) = 3 under the FP64 oracle, per species"}
    t0 = time.time()
    res["plain"] = per_species(synth.plain_set(100_000, 0), synth.front_camera(256, 256))
    res["clustered"] = per_species(synth.clustered_set(10_000_000, 1), synth.front_camera(1024, 1024))
    res["batched"] = per_species(synth.clustered_set(20_000_000, 3), synth.orbit_cameras(64, 1024, 1024)[0])
    served1m = per_species(synth.clustered_set(1_000_000, 4), synth.front_camera(1024, 1024))[0]
    res["served"] = [served1m * 1e6 / n for n in synth.served_set_sizes()]
    res["two_species"] = per_species(synth.two_species_set(70_000_000, 30_000_000, 2),
                                     synth.front_camera(2048, 2048))
    res["seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, "brightness.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
