"""Error of every result against the FP64 oracle, as a markdown table.

Not a test: a report, run on a GPU machine after `__graft_entry__.build()`:

    python tests/report_errors.py          # both tables
    python tests/report_errors.py --pme    # the long-range table only

Per workload it evaluates through the C ABI and prints RMS(dF)/RMS(F), the
relative errors of E_LJ and E_C, the largest virial component error relative to
the virial's Frobenius norm, and whether the interacting-pair count equals the
oracle's.  The 3M-atom box gets forces of 10^4 sampled atoms (the oracle's
per-atom loop) and its energies, virial and pair count against the oracle's
O(N^2) sums stored in tests/golden/large_box_seed3.json; the ensemble goes
through the batched path.  A second table
gives the long-range (PME) part against oracle/pme.py, the virial error
relative to the sum of the reciprocal and excluded-pair virials' norms.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from paper_1506_00716_gb300 import autotune, nb  # noqa: E402
from paper_1506_00716_gb300 import waterbox as wb  # noqa: E402
from _support import rel_rms  # noqa: E402

FLAGS = nb.NB_F_ENERGY | nb.NB_F_VIRIAL


def _eval(ctx, s, p):
    h = nb.nb_sys_create(ctx, p, s.n, s.box)
    try:
        nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
        nb.nb_grid_put(h, s.xq(), s.type)
        nb.nb_pairlist_build(h)
        f = np.zeros((s.n, 3), dtype=np.float32)
        e = np.zeros(2)
        v = np.zeros(9)
        nb.nb_forces(h, None, f, e, v, FLAGS)
        npairs = nb.nb_eval_info(h)["n_pairs"]
    finally:
        nb.nb_sys_destroy(h)
    return f, e, v, npairs


def _row(name, f_err, e, v, npairs, ref):
    if ref is None:
        return f"| {name} | {f_err:.2e} | — | — | — | — |"
    vr = ref["virial"].reshape(-1)
    ref_pairs = ref["npairs"]
    count = "equal" if npairs == ref_pairs else f"{npairs} vs {ref_pairs}"
    return (f"| {name} | {f_err:.2e} | {abs(e[0] - ref['e_lj']) / abs(ref['e_lj']):.2e} | "
            f"{abs(e[1] - ref['e_coul']) / abs(ref['e_coul']):.2e} | "
            f"{np.abs(v - vr).max() / np.linalg.norm(vr):.2e} | {count} |")


def main():
    import torch

    from paper_1506_00716_gb300 import build as nbbuild

    nbbuild.build()
    torch.cuda.set_device(0)
    gpu = torch.cuda.get_device_name(0)
    ctx = nb.nb_ctx_create(0, None, 0)
    rows = ["| workload | RMS(dF)/RMS(F) | E_LJ rel | E_C rel | virial / norm | pair count |",
            "|---|---:|---:|---:|---:|---|"]
    for name, s in (("small (1,944 atoms)", wb.small_box(seed=1)), ("mid (24,000 atoms)", wb.mid_box(seed=2))):
        for cname, p in (("RF", wb.params_rf()), ("Ewald", wb.params_ewald())):
            autotune.apply(ctx, "rf" if cname == "RF" else "ewald", s.n, gpu=gpu)
            f, e, v, npairs = _eval(ctx, s, p)
            ref = oracle.energy_virial(s, p)
            rows.append(_row(f"{name}, {cname}", rel_rms(f, oracle.forces(s, p)), e, v, npairs, ref))
            print(rows[-1], flush=True)
    for name, s in (("small (1,944 atoms)", wb.small_box(seed=1)), ("mid (24,000 atoms)", wb.mid_box(seed=2))):
        for cname, coul, mods, label in (
                ("RF", wb.COUL_RF, nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_RF_EXCL, "LJ shift + RF exclusion correction"),
                ("Ewald", wb.COUL_EWALD, nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_EWALD_SHIFT, "LJ + Ewald shifts")):
            p = wb.Params(coul=coul, modifiers=mods)
            autotune.apply(ctx, "rf" if cname == "RF" else "ewald", s.n, gpu=gpu)
            f, e, v, npairs = _eval(ctx, s, p)
            ref = oracle.energy_virial(s, p)
            rows.append(_row(f"{name}, {cname}, {label}", rel_rms(f, oracle.forces(s, p)), e, v, npairs, ref))
            print(rows[-1], flush=True)
    s = wb.large_box(seed=3)
    p = wb.params_ewald()
    autotune.apply(ctx, "ewald", s.n, gpu=gpu)
    f, e, v, npairs = _eval(ctx, s, p)
    sel = np.sort(np.random.default_rng(31).choice(s.n, size=10_000, replace=False)).astype(np.int32)
    # the oracle's O(N^2) sums of this box, written once by tests/golden/make_large_box.py
    gold_path = os.path.join(HERE, "golden", "large_box_seed3.json")
    ref = None
    if os.path.exists(gold_path):
        import json

        with open(gold_path) as fh:
            g = json.load(fh)
        ref = {"e_lj": g["e_lj"], "e_coul": g["e_coul"], "virial": np.array(g["virial"]), "npairs": g["npairs"]}
    rows.append(_row("large (3,000,000 atoms), Ewald: golden sums; forces of 10^4 sampled atoms",
                     rel_rms(f[sel], oracle.forces(s, p, sel)), e, v, npairs, ref))
    print(rows[-1], flush=True)
    nb.nb_ctx_destroy(ctx)

    # ensemble through the batched path: worst case over the systems
    systems = wb.ensemble(64, 1000, 32000, seed=4)
    p = wb.params_rf()
    stream = torch.cuda.Stream()
    ctx = nb.nb_ctx_create(0, stream, 0)
    autotune.apply(ctx, "rf", sum(x.n for x in systems) // len(systems), gpu=gpu)
    hs = []
    for x in systems:
        h = nb.nb_sys_create(ctx, p, x.n, x.box)
        nb.nb_set_exclusions(h, x.excl_index, x.excl_atoms)
        nb.nb_sys_set_coords(h, x.xq(), x.type)
        hs.append(h)
    b = nb.nb_batch_create(ctx, hs)
    for attempt in range(3):
        try:
            nb.nb_batch_poll(b, nb.nb_batch_submit(b, FLAGS), 60_000_000)
            break
        except nb.NbError as exc:
            if exc.status != 9:
                raise
    rng = np.random.default_rng(32)
    order = np.argsort([x.n for x in systems])
    worst = np.zeros(4)
    for k in range(len(systems)):
        x, h = systems[k], hs[k]
        f = np.zeros((x.n, 3), dtype=np.float32)
        e = np.zeros(2)
        v = np.zeros(9)
        nb.nb_sys_results(h, f, e, v)
        sel = np.sort(rng.choice(x.n, size=48, replace=False)).astype(np.int32)
        worst[0] = max(worst[0], rel_rms(f[sel], oracle.forces(x, p, sel)))
        if k in set(order[:12].tolist()):
            ref = oracle.energy_virial(x, p)
            vr = ref["virial"].reshape(-1)
            worst[1] = max(worst[1], abs(e[0] - ref["e_lj"]) / abs(ref["e_lj"]))
            worst[2] = max(worst[2], abs(e[1] - ref["e_coul"]) / abs(ref["e_coul"]))
            worst[3] = max(worst[3], np.abs(v - vr).max() / np.linalg.norm(vr))
    rows.append(f"| ensemble (64 boxes, batched), RF: worst system; energies of the 12 smallest | "
                f"{worst[0]:.2e} | {worst[1]:.2e} | {worst[2]:.2e} | {worst[3]:.2e} | — |")
    print(rows[-1], flush=True)
    nb.nb_batch_destroy(b)
    for h in hs:
        nb.nb_sys_destroy(h)
    nb.nb_ctx_destroy(ctx)
    print("\n".join(rows))
    print()
    print("\n".join(pme_rows(gpu)))


def pme_rows(gpu):
    """The long-range part (nb_pme_forces) against oracle/pme.py."""
    from oracle import pme as opme

    rows = ["| workload | mesh, order | RMS(dF)/RMS(F) | E_rec rel | E_self rel | E_excl rel | virial / scale |",
            "|---|---|---:|---:|---:|---:|---:|"]
    ctx = nb.nb_ctx_create(0, None, 0)
    p = wb.params_ewald()
    cases = [("small (1,944 atoms)", wb.small_box(seed=1), (24, 24, 24), 4, None),
             ("small (1,944 atoms)", wb.small_box(seed=1), (25, 27, 45), 6, None),
             ("small (1,944 atoms)", wb.small_box(seed=1), (32, 30, 20), 8, None),
             ("mid (24,000 atoms)", wb.mid_box(seed=2), (54, 50, 60), 4, None),
             ("mid (24,000 atoms)", wb.mid_box(seed=2), (64, 64, 64), 6, None),
             ("rhombic dodecahedron (2,100 atoms)", wb.rhombic_dodecahedron_box(648, seed=5), (24, 30, 18), 4, None),
             ("rhombic dodecahedron (2,100 atoms)", wb.rhombic_dodecahedron_box(648, seed=5), (16, 20, 12), 6, None),
             ("rhombic dodecahedron (23,232 atoms)", wb.rhombic_dodecahedron_box(7744, seed=6), (60, 60, 40), 4, None),
             ("large (3,000,000 atoms), 192 sampled forces", wb.large_box(seed=3), (256, 256, 256), 4, 192)]
    for name, s, grid, order, nsel in cases:
        h = nb.nb_sys_create(ctx, p, s.n, s.box, getattr(s, "skew", None))
        try:
            nb.nb_set_exclusions(h, s.excl_index, s.excl_atoms)
            nb.nb_grid_put(h, s.xq(), s.type)
            nb.nb_pairlist_build(h)
            nb.nb_pme_init(h, grid, order)
            f = np.zeros((s.n, 3), dtype=np.float32)
            e = np.zeros(3)
            v = np.zeros(9)
            nb.nb_pme_forces(h, None, f, e, v, FLAGS)
        finally:
            nb.nb_sys_destroy(h)
        sel = None if nsel is None else np.sort(np.random.default_rng(31).choice(s.n, size=nsel, replace=False))
        rec = opme.pme(s, p, grid=grid, order=order, sel=sel)
        ex = opme.ewald_exclusions(s, p)
        rf = rec["forces"] + (ex["forces"] if sel is None else ex["forces"][sel])
        fg = f if sel is None else f[sel]
        re = [rec["energy"], opme.ewald_self(s, p), ex["energy"]]
        rv = rec["virial"] + ex["virial"]
        scale = np.linalg.norm(rec["virial"]) + np.linalg.norm(ex["virial"])
        rows.append(f"| {name} | {grid[0]}x{grid[1]}x{grid[2]}, {order} | {rel_rms(fg, rf):.2e} | "
                    + " | ".join(f"{abs(e[k] - re[k]) / abs(re[k]):.2e}" for k in range(3))
                    + f" | {np.abs(v.reshape(3, 3) - rv).max() / scale:.2e} |")
        print(rows[-1], flush=True)
    nb.nb_ctx_destroy(ctx)
    return rows


if __name__ == "__main__":
    if "--pme" in sys.argv[1:]:
        print("\n".join(pme_rows(None)))
    else:
        main()
