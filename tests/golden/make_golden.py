"""Writes tests/golden/oracle_small_clip.json from the oracle alone.

The values are the oracle's per-frame cut value, mask area and prior/saliency
sums on the seeded 160x120 red-disk clip.  They guard the oracle against
unintended change; they are not a pin of its correctness (the pins live in
tests/test_oracle_pins.py).  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1008_0502_b300 import synth  # noqa: E402


def main():
    frames, gt = synth.clip_small()
    sg = O.Segmenter(120, 160, O.CONFIG_SMALL)
    rows = []
    for t in range(len(frames)):
        sal, pr, mask, cut = sg.push(frames[t])
        rows.append({"t": t, "cut": cut, "mask_area": int(mask.sum()),
                     "mask_gt_overlap": int((mask & gt[t]).sum()),
                     "saliency_sum": float(sal.sum()), "prior_sum": float(pr.sum())})
    with open(os.path.join(HERE, "oracle_small_clip.json"), "w") as f:
        json.dump({"workload": "160x120 red-disk clip, seed 10080502+1, 10 frames",
                   "frames": rows}, f, indent=1)


if __name__ == "__main__":
    main()
