"""Writes the small EDT fixtures in this folder.  Calls only the oracle's brute-force
EDT (the definition of Sec. III-C: nearest occupied voxel of every voxel), never the
CUDA path.  Run:  python tests/golden/make_golden.py"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

CASES = {
    # name: (dims (X, Y, Z), occupied voxels (x, y, z))
    "three_sites_6x5x4": ((6, 5, 4), [(0, 0, 0), (5, 4, 3), (2, 3, 1)]),
    "plane_and_point_9x7x5": ((9, 7, 5), [(x, y, 0) for x in range(9) for y in range(7)] + [(4, 3, 4)]),
    "corner_row_17x3x2": ((17, 3, 2), [(16, 2, 1)]),
}


def main():
    for name, (dims, sites) in CASES.items():
        X, Y, Z = dims
        occ = np.zeros((Z, Y, X), dtype=np.uint8)
        for (x, y, z) in sites:
            occ[z, y, x] = 1
        sq, _ = oracle.edt_brute(occ)
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump({"source": "oracle.edt_brute (definition of the EDT, Sec. III-C)",
                       "dims": list(dims), "sites": [list(s) for s in sites],
                       "sqdist_zyx": sq.reshape(Z, Y, X).tolist()}, f)


if __name__ == "__main__":
    main()
