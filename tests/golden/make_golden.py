"""Write the oracle regression fixture for config 1 (2,000 atoms, 256x256).

The paper prints no per-pixel values, so this fixture is not a paper value: it
freezes the oracle's own output on 96 fixed pixels so that an accidental
change to the oracle's arithmetic shows up in the CPU test suite.  It calls
only ``oracle`` and the seeded scene generator.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2501_12750_gb300 import scenes  # noqa: E402


def main():
    s = scenes.config1()
    rng = np.random.default_rng(123)
    # half the pixels inside the cube's footprint, half anywhere
    pix = np.concatenate([np.stack([rng.integers(90, 166, 48), rng.integers(90, 166, 48)], 1),
                          np.stack([rng.integers(0, 256, 48), rng.integers(0, 256, 48)], 1)]).astype(np.int32)
    h = oracle.render_pixels(s, 0, pix)
    out = {
        "what": "oracle output on 96 fixed pixels of config 1 (regression fixture, not a paper value)",
        "writer": "tests/golden/make_golden.py (calls only oracle/)",
        "pix": pix.tolist(),
        "id": h.id.tolist(),
        "depth": np.where(np.isfinite(h.depth), h.depth, -1.0).tolist(),
        "rgb": h.rgb.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_oracle_pixels.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print("wrote", path, "covered", int((h.id != oracle.NO_ID).sum()))


if __name__ == "__main__":
    main()
