"""Write the oracle's energies, virial and pair count of the 3,000,000-atom box.

Run once on the host (about three and a half hours on 8 cores):

    python tests/golden/make_large_box.py

The O(N^2) sum is taken in 64 row ranges of about equal pair counts; the
sums of finished ranges are kept in large_box_seed3.partial.json beside the
output, so an interrupted run resumes where it stopped (and the file is
removed at the end).  `--add-moments` adds the input moments (see
input_moments) to an existing output without the O(N^2) work.

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
PARTIAL = os.path.join(HERE, "large_box_seed3.partial.json")
N_RANGES = 64


def input_digest(s) -> str:
    """SHA-256 over the float32 coordinates, charges, types and exclusions."""
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(s.x, dtype=np.float32), np.ascontiguousarray(s.q, dtype=np.float32),
              np.ascontiguousarray(s.type, dtype=np.int32), np.ascontiguousarray(s.excl_index, dtype=np.int32),
              np.ascontiguousarray(s.excl_atoms, dtype=np.int32), np.asarray(s.box, dtype=np.float64)):
        h.update(a.tobytes())
    return h.hexdigest()


def input_moments(s) -> list:
    """Float64 sums of the float32 coordinates and of their squares, per axis,
    and of the charges: a fingerprint of the atoms that a few last-bit
    differences of the generator on another machine (fused multiply-adds,
    libm) leave equal to about 1e-12, where the SHA-256 would change."""
    x = np.asarray(s.x, dtype=np.float64)
    return [float(v) for v in np.concatenate([x.sum(0), (x * x).sum(0), [np.asarray(s.q, np.float64).sum()]])]


def add_moments():
    """Add the input moments to an existing output (no O(N^2) work)."""
    with open(OUT) as fh:
        rec = json.load(fh)
    s = wb.large_box(seed=rec["seed"])
    if input_digest(s) != rec["input_sha256"]:
        raise SystemExit("the generator made other atoms than the stored run")
    rec["input_moments"] = input_moments(s)
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")


def main():
    seed = 3
    s = wb.large_box(seed=seed)
    p = wb.params_ewald()
    oracle.build()
    digest = input_digest(s)
    # row ranges of about equal pair counts: row i holds n - 1 - i pairs, so
    # the rows before i hold i (2n - 1 - i) / 2; bound k of N_RANGES solves
    # that for k / N_RANGES of all pairs
    n = s.n
    tot = n * (n - 1) / 2.0
    bounds = [0]
    for k in range(1, N_RANGES):
        t = tot * k / N_RANGES
        i = int((2 * n - 1 - ((2 * n - 1) ** 2 - 8 * t) ** 0.5) / 2)
        bounds.append(min(max(i, bounds[-1]), n))
    bounds.append(n)
    done = {}
    if os.path.exists(PARTIAL):
        with open(PARTIAL) as fh:
            prev = json.load(fh)
        if prev.get("input_sha256") == digest and prev.get("bounds") == bounds:
            done = {int(k): v for k, v in prev["ranges"].items()}
    wall = sum(v["wall_s"] for v in done.values())
    for k in range(N_RANGES):
        if k in done:
            continue
        t0 = time.time()
        out, np_k = oracle.energy_virial_rows(s, p, bounds[k], bounds[k + 1])
        done[k] = {"sums": [float(v) for v in out], "npairs": np_k, "wall_s": round(time.time() - t0, 1)}
        wall += done[k]["wall_s"]
        with open(PARTIAL + ".tmp", "w") as fh:
            json.dump({"input_sha256": digest, "bounds": bounds, "ranges": done}, fh)
        os.replace(PARTIAL + ".tmp", PARTIAL)
        print(f"rows {bounds[k]}..{bounds[k + 1]}: {done[k]['wall_s']} s ({len(done)}/{N_RANGES})", flush=True)
    sums = np.zeros(15)
    npairs = 0
    for k in range(N_RANGES):
        sums += np.asarray(done[k]["sums"])
        npairs += done[k]["npairs"]
    ev = oracle.ev_from_sums(sums, npairs)
    rec = {
        "what": "FP64 O(N^2) oracle sums of the 3,000,000-atom water box (LJ + Ewald real space)",
        "generator": "paper_1506_00716_gb300.waterbox.large_box(seed=3)",
        "seed": seed,
        "natoms": int(s.n),
        "box_nm": [float(v) for v in s.box],
        "params": {"rc": p.rc, "coul": "ewald", "beta": p.beta, "eps_r": p.eps_r, "fcoul": p.fcoul,
                   "c6_OO": float(p.c6[0]), "c12_OO": float(p.c12[0]), "modifiers": 0},
        "input_sha256": digest,
        "input_moments": input_moments(s),
        "e_lj": float(ev["e_lj"]),
        "e_coul": float(ev["e_coul"]),
        "virial": [float(v) for v in ev["virial"].reshape(-1)],
        "npairs": int(ev["npairs"]),
        "e12": float(ev["e12"]),
        "e6": float(ev["e6"]),
        "oracle_threads": oracle.num_threads(),
        "oracle_wall_s": round(wall, 1),
        "row_ranges": N_RANGES,
    }
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    os.remove(PARTIAL)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    if sys.argv[1:] == ["--add-moments"]:
        add_moments()
    else:
        main()
