"""Writes the golden files of tests/golden/ from the oracle alone.

oracle_small_clip.json: the oracle's per-frame cut value, mask area and
prior/saliency sums on the seeded 160x120 red-disk clip.  They guard the
oracle against unintended change; they are not a pin of its correctness (the
pins live in tests/test_oracle_pins.py).

oracle_vga_state_f195.json: the oracle's temporal state (Sec. 6: previous
mask and Kalman variance, frame index) after frames 0..194 of the seeded
640x480 clip, so that a parity test can start both sides at frame 195 (the
ambiguous frames where the fading disk's labelling flips) without running the
slow oracle through the whole clip.  Run:  python tests/golden/make_golden.py
(add --vga-state for the second file; it takes a few minutes).
"""
import base64
import json
import os
import sys
import zlib

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


def vga_state(t_stop=195):
    import itertools

    import numpy as np
    sg = O.Segmenter(480, 640, O.CONFIG_VGA)
    # frames 0..t_stop-1 of the 300-frame clip (the clip's frames depend on its length)
    for f, _ in itertools.islice(synth.clip_vga_frames(300), t_stop):
        sg.push(f)
    bits = np.packbits(sg.prev.ravel())
    with open(os.path.join(HERE, f"oracle_vga_state_f{t_stop}.json"), "w") as fh:
        json.dump({"workload": "640x480 clip of 300 frames (synth.clip_vga_frames), seed 10080502+2, oracle run over frames "
                   f"0..{t_stop - 1}", "t": sg.t, "P_hex": float(sg.P_var).hex(), "H": 480, "W": 640,
                   "prev_mask_packbits_zlib_b64": base64.b64encode(zlib.compress(bits.tobytes(), 9)).decode()},
                  fh, indent=1)


if __name__ == "__main__":
    if "--vga-state" in sys.argv:
        vga_state()
    else:
        main()
