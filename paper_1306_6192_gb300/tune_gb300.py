"""Generates the shipped tuning table of the split path on a GB300.

Runs the library's autotuner (mm_tune: times every candidate tile width, K
depth / pipeline depth, raster band height and tail split on or off on the
device) for one
representative size per bucket and writes the table next to this file
(tune_gb300.txt), which the binding loads at mm_init.  Buckets are
(ceil(log2 n), ceil(log2 m), ceil(log2 p)).

  python paper_1306_6192_gb300/tune_gb300.py [--reps 3]
"""
from __future__ import annotations

import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_1306_6192_gb300 as mm  # noqa: E402

TABLE = os.path.join(HERE, "tune_gb300.txt")

# Single-product shapes: the square sizes, the rectangular and the skinny
# workload.  Buckets of the grouped range (dims 32..1024) are left to the
# built-in choice: their K is below 2237, so they take the three-part split,
# whose layout is fixed (128-wide tiles, 32 bf16 of K per stage, four stages),
# and the knobs left (raster band height, grid) were timed on the whole
# 4096-instance mix on GB300 (band 1 to 16, grid 148 or 152: 97.6 to 99.2
# TFLOP/s against 98.4 for the built-in choice, within the run-to-run spread).
SHAPES = ([(s, s, s) for s in (256, 512, 1024, 2048, 4096, 8192)] +
          [(8192, 512, 8192), (64, 16384, 64), (16384, 16384, 16384)])


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    for (n, m, p) in SHAPES:
        st = mm.mm_tune(n, m, p, args.reps)
        mm.check_status(st, "mm_tune %dx%dx%d" % (n, m, p))
        q = mm.mm_tune_query(n, m, p)
        print("%5d %5d %5d -> bn %d bk %d stages %d group_m %d" % ((n, m, p) + q[1:]), flush=True)
    mm.check_status(mm.mm_tune_save(TABLE), "mm_tune_save")
    mm.mm_shutdown()
    print("wrote", TABLE)
    return 0


if __name__ == "__main__":
    sys.exit(main())
