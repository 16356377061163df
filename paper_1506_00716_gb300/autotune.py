"""Autotuner for the launch parameters of the cluster-pair path.

Tuned per (electrostatics, system size):
  max_entries       work-item split: (i-cluster, shift) runs of list entries
                    longer than this become several items, so that the
                    persistent force kernel balances well on small systems
                    (list-splitting threshold);
  force_min_blocks  force-kernel register budget / block residency (block
                    shape): 1, 2 or 3 resident 256-thread blocks per SM, or
                    4: two 320-thread blocks (96 registers);
  search_mode       cluster-pair search: a warp per i-cluster (1) or a
                    thread per i-cluster (2);
  energy_mode       evaluations with energies: a separate double-float energy
                    kernel (0) or the energies fused into the force kernel (1);
  jcluster          cluster geometry M x N (Section 3.2): 8 x 8, or 8 x 4 with
                    the z-halves of the 8-atom clusters as j-clusters, two per
                    list entry (fewer computed pair slots, more entries).

For every (max_entries, force_min_blocks) candidate the tuner builds the list
and times one build (search + prune) plus EVALS force evaluations with the
library's per-stage CUDA events, and keeps the fastest; at that setting it
times the same with each cluster geometry and keeps the faster, then times
the build with each search kernel, and one evaluation with energies and
virial with each energy path.  The result is a JSON table keyed by GPU name;
lookup() picks the entry of the nearest size (in log atoms).

    python -m paper_1506_00716_gb300.autotune [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

from . import nb
from . import waterbox as wb

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning.json")
SIZES_MOL = [1000, 8000, 64000, 1_000_000]
MAX_ENTRIES = [8, 16, 32, 64, 128]
MIN_BLOCKS = [1, 2, 3, 4]
SEARCH_MODES = [1, 2]
ENERGY_MODES = [0, 1]
JCLUSTERS = [8, 4]
EVALS = 10


def _time_build(ctx, h, s, me, mb, search_mode, jc: int = 8, reps: int = 3) -> float:
    """Fastest list build (search + prune), ms."""
    nb.nb_ctx_set_tuning(ctx, me, mb, search_mode, 0, jc)
    nb.nb_grid_put(h, s.xq(), s.type)
    nb.nb_pairlist_build(h)
    best = None
    for _ in range(reps):
        nb.nb_ctx_timing(ctx, reset=True)
        nb.nb_ctx_set_timing(ctx, True)
        nb.nb_pairlist_build(h)
        nb.nb_ctx_set_timing(ctx, False)
        st = nb.nb_ctx_timing(ctx, reset=True)
        t = st["search"][0] + st["prune"][0]
        best = t if best is None else min(best, t)
    return best


def _time_energy_eval(ctx, h, s, me, mb, search_mode, energy_mode, jc: int = 8, reps: int = 3) -> float:
    """Fastest evaluation with energies and virial (force + energy stages), ms."""
    nb.nb_ctx_set_tuning(ctx, me, mb, search_mode, energy_mode, jc)
    nb.nb_grid_put(h, s.xq(), s.type)
    nb.nb_pairlist_build(h)
    flags = nb.NB_F_ENERGY | nb.NB_F_VIRIAL
    import numpy as np

    e = np.zeros(2)
    v = np.zeros(9)
    nb.nb_forces(h, None, None, e, v, flags)
    best = None
    for _ in range(reps):
        nb.nb_ctx_timing(ctx, reset=True)
        nb.nb_ctx_set_timing(ctx, True)
        nb.nb_forces(h, None, None, e, v, flags)
        nb.nb_ctx_set_timing(ctx, False)
        st = nb.nb_ctx_timing(ctx, reset=True)
        t = st["forces"][0] + st["energy"][0]
        best = t if best is None else min(best, t)
    return best


def _time_config(ctx, h, s, max_entries, min_blocks, jc: int = 8, reps: int = 2) -> dict:
    nb.nb_ctx_set_tuning(ctx, max_entries, min_blocks, 0, 0, jc)
    xq, ty = s.xq(), s.type
    nb.nb_grid_put(h, xq, ty)
    nb.nb_pairlist_build(h)
    for _ in range(2):
        nb.nb_forces(h, None, None, None, None, 0)
    best = None
    for _ in range(reps):
        nb.nb_ctx_timing(ctx, reset=True)
        nb.nb_ctx_set_timing(ctx, True)
        nb.nb_pairlist_build(h)
        for _ in range(EVALS):
            nb.nb_forces(h, None, None, None, None, 0)
        nb.nb_ctx_set_timing(ctx, False)
        st = nb.nb_ctx_timing(ctx, reset=True)
        total = st["search"][0] + st["prune"][0] + st["forces"][0] + st["zero"][0] + st["final"][0]
        rec = {"total_ms": total, "forces_ms": st["forces"][0] / EVALS,
               "build_ms": st["search"][0] + st["prune"][0],
               "slots": 64 * nb.nb_pairlist_info(h)["n_entries"]}
        if best is None or rec["total_ms"] < best["total_ms"]:
            best = rec
    return best


def tune(sizes=SIZES_MOL, device: int = 0, verbose: bool = True) -> dict:
    import torch

    torch.cuda.set_device(device)
    gpu = torch.cuda.get_device_name(device)
    ctx = nb.nb_ctx_create(device, torch.cuda.current_stream(), 0)
    entries = []
    try:
        for coul, params in (("rf", wb.params_rf()), ("ewald", wb.params_ewald())):
            for m in sizes:
                s = wb.water_box(m, None, seed=11)
                h = nb.nb_sys_create(ctx, params, s.n, s.box)
                nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
                results = []
                for me in MAX_ENTRIES:
                    for mb in MIN_BLOCKS:
                        r = _time_config(ctx, h, s, me, mb)
                        results.append({"max_entries": me, "force_min_blocks": mb, **r})
                best = min(results, key=lambda r: r["total_ms"])
                me, mb = best["max_entries"], best["force_min_blocks"]
                geo = {jc: (best if jc == 8 else _time_config(ctx, h, s, me, mb, jc)) for jc in JCLUSTERS}
                jc = min(geo, key=lambda k: geo[k]["total_ms"])
                best = geo[jc]
                build = {sm: _time_build(ctx, h, s, me, mb, sm, jc) for sm in SEARCH_MODES}
                search_mode = min(build, key=build.get)
                energy = {em: _time_energy_eval(ctx, h, s, me, mb, search_mode, em, jc) for em in ENERGY_MODES}
                energy_mode = min(energy, key=energy.get)
                nb.nb_sys_destroy(h)
                default = next(r for r in results if r["max_entries"] == 32 and r["force_min_blocks"] == 3)
                entries.append({"coul": coul, "atoms": s.n, "max_entries": me, "force_min_blocks": mb,
                                "search_mode": search_mode, "energy_mode": energy_mode, "jcluster": jc,
                                "by_jcluster": {str(k): {"total_ms": round(v["total_ms"], 5),
                                                         "forces_ms": round(v["forces_ms"], 5),
                                                         "build_ms": round(v["build_ms"], 5), "slots": v["slots"]}
                                                for k, v in geo.items()},
                                "build_ms_by_search_mode": {str(k): round(v, 5) for k, v in build.items()},
                                "energy_eval_ms_by_energy_mode": {str(k): round(v, 5) for k, v in energy.items()},
                                "total_ms": round(best["total_ms"], 5),
                                "default_total_ms": round(default["total_ms"], 5),
                                "sweep": [{k: (round(v, 5) if isinstance(v, float) else v)
                                           for k, v in r.items()} for r in results]})
                if verbose:
                    print(f"{coul:5s} {s.n:8d} atoms: best max_entries={me} min_blocks={mb} jcluster={jc} "
                          f"{best['total_ms']:.4f} ms (default {default['total_ms']:.4f} ms); "
                          f"geometry { {k: round(v['total_ms'], 4) for k, v in geo.items()} }; search {build}; "
                          f"energy {energy}", flush=True)
    finally:
        nb.nb_ctx_destroy(ctx)
    return {"gpu": gpu, "evals_per_build": EVALS, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
            "entries": entries}


def load(path: str = DEFAULT_TABLE) -> dict | None:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def lookup(table: dict | None, coul: str, natoms: int, gpu: str | None = None) -> dict:
    """Tuning for a system: the table entry of the same electrostatics and nearest size."""
    default = {"max_entries": 32, "force_min_blocks": 3, "search_mode": 0, "energy_mode": 0, "jcluster": 8}
    if not table or (gpu is not None and table.get("gpu") != gpu):
        return default
    cands = [e for e in table.get("entries", []) if e["coul"] == coul]
    if not cands:
        return default
    e = min(cands, key=lambda e: abs(math.log(e["atoms"]) - math.log(max(natoms, 1))))
    return {"max_entries": int(e["max_entries"]), "force_min_blocks": int(e["force_min_blocks"]),
            "search_mode": int(e.get("search_mode", 0)), "energy_mode": int(e.get("energy_mode", 0)),
            "jcluster": int(e.get("jcluster", 8))}


def apply(ctx, coul: str, natoms: int, table: dict | None = None, gpu: str | None = None) -> dict:
    t = lookup(table if table is not None else load(), coul, natoms, gpu)
    nb.nb_ctx_set_tuning(ctx, t["max_entries"], t["force_min_blocks"], t["search_mode"], t["energy_mode"],
                         t["jcluster"])
    return t


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    args = ap.parse_args()
    from . import build as nbbuild

    nbbuild.build()
    table = tune()
    with open(args.out, "w") as fh:
        json.dump(table, fh, indent=1)
    print(args.out)


if __name__ == "__main__":
    main()
