"""Writes the oracle's analysis of the two full-size single-clip workloads
(1920x1080 interlaced, 1500 frames; 1920x1080 3:2 pulldown, 1800 frames) to
tests/golden/oracle_<workload>.json.gz: every decision and every reported
measure (integer record and FP64 values).  Only the oracle and the seeded
input generator run here; the GPU tests compare the library's results with
these files value by value.

    python tests/golden/make_full_size_oracle.py [--workers N]
"""
from __future__ import annotations

import argparse
import gzip
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = ("interlaced_1080p", "pulldown_1080p")


def spec_of(name):
    from paper_2502_09202_gb300 import synth
    return {"interlaced_1080p": synth.config_interlaced, "pulldown_1080p": synth.config_pulldown}[name]()


def path_of(name):
    return os.path.join(HERE, f"oracle_{name}.json.gz")


def main():
    from oracle import analyser as OA
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for name in WORKLOADS:
        spec = spec_of(name)
        t0 = time.time()
        r = OA.analyse_spec(spec, workers=args.workers)
        measures = [[k[0], k[1], k[2], {f: (v.hex() if isinstance(v, float) else v) for f, v in m.items()}]
                    for k, m in r["measures"].items()]
        out = {"workload": spec.name, "frames": spec.nframes, "width": spec.width, "height": spec.height,
               "cuts": r["cuts"], "dissolves": [list(d) for d in r["dissolves"]], "keyframes": r["keyframes"],
               "shots": r["shots"], "label": r["label"], "field_order": r["field_order"],
               "pulldown_phase": r["pulldown_phase"], "measures": measures}
        with gzip.open(path_of(name), "wt") as f:
            json.dump(out, f, separators=(",", ":"))
        print(f"{name}: {len(measures)} measures, cuts {r['cuts']}, dissolves {r['dissolves']}, "
              f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
