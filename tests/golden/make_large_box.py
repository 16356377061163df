"""Write the oracle's energies, virial and pair count of the 3,000,000-atom box.

Run once on the host (about three hours on 8 cores, twenty minutes on 16
Arm cores):

    python tests/golden/make_large_box.py

It calls only the FP64 oracle (oracle/nb_oracle.c, the plain O(N^2)
minimum-image pair sum) and the seeded input generator, on the box the
benchmark times: 1,000,000 rigid three-site waters in L = 31.0 nm, seed 3,
Lennard-Jones + Ewald real space (beta = 3.12 nm^-1), rc = 1.0 nm.  The
result goes to tests/golden/large_box_seed3.json with the SHA-256 of the
float32 inputs, so that a test on another machine can tell whether its
generator produced the very same atoms.

The paper's Section 3.2 states that the cluster-pair list only adds
interactions that are zero, so the cluster-pair method must reach exactly
this plain sum; these values pin that claim at full size.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1506_00716_gb300 import waterbox as wb  # noqa: E402

OUT = os.path.join(HERE, "large_box_seed3.json")


def input_digest(s) -> str:
    """SHA-256 over the float32 coordinates, charges, types and exclusions."""
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(s.x, dtype=np.float32), np.ascontiguousarray(s.q, dtype=np.float32),
              np.ascontiguousarray(s.type, dtype=np.int32), np.ascontiguousarray(s.excl_index, dtype=np.int32),
              np.ascontiguousarray(s.excl_atoms, dtype=np.int32), np.asarray(s.box, dtype=np.float64)):
        h.update(a.tobytes())
    return h.hexdigest()


def main():
    seed = 3
    s = wb.large_box(seed=seed)
    p = wb.params_ewald()
    oracle.build()
    t0 = time.time()
    ev = oracle.energy_virial(s, p)
    wall = time.time() - t0
    rec = {
        "what": "FP64 O(N^2) oracle sums of the 3,000,000-atom water box (LJ + Ewald real space)",
        "generator": "paper_1506_00716_gb300.waterbox.large_box(seed=3)",
        "seed": seed,
        "natoms": int(s.n),
        "box_nm": [float(v) for v in s.box],
        "params": {"rc": p.rc, "coul": "ewald", "beta": p.beta, "eps_r": p.eps_r, "fcoul": p.fcoul,
                   "c6_OO": float(p.c6[0]), "c12_OO": float(p.c12[0]), "modifiers": 0},
        "input_sha256": input_digest(s),
        "e_lj": float(ev["e_lj"]),
        "e_coul": float(ev["e_coul"]),
        "virial": [float(v) for v in ev["virial"].reshape(-1)],
        "npairs": int(ev["npairs"]),
        "e12": float(ev["e12"]),
        "e6": float(ev["e6"]),
        "oracle_threads": oracle.num_threads(),
        "oracle_wall_s": round(wall, 1),
    }
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
