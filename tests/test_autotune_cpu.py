"""The autotuner's committed GB300 table and its lookup (host logic, no GPU).

The tuner (paper_1506_00716_gb300/autotune.py) picks per electrostatics and
system size the cluster geometry (8 x 8 or 8 x 4 j-clusters), the work-item
split, the force kernel's register budget, the search kernel and the energy
path.  These tests check that the committed table is well formed and
consistent with the tuner's own rules, and that lookup() takes the entry of
the nearest size and falls back to the defaults for another GPU.
"""
import math

from paper_1506_00716_gb300 import autotune

TABLE = autotune.load()


def test_table_is_present_and_covers_both_electrostatics():
    assert TABLE is not None
    for coul in ("rf", "ewald"):
        sizes = sorted(e["atoms"] for e in TABLE["entries"] if e["coul"] == coul)
        assert sizes == [3000, 24000, 192000, 3000000]


def test_entries_hold_valid_choices():
    for e in TABLE["entries"]:
        assert e["jcluster"] in (8, 4)
        assert e["force_min_blocks"] in (1, 2, 3, 4)
        assert e["max_entries"] in autotune.MAX_ENTRIES
        assert e["search_mode"] in (1, 2)
        assert e["energy_mode"] in (0, 1)


def test_each_choice_is_the_fastest_the_tuner_measured():
    for e in TABLE["entries"]:
        # geometry: the faster of the two build + 10 evaluation times
        g = e["by_jcluster"]
        assert set(g) == {"8", "4"}
        assert g[str(e["jcluster"])]["total_ms"] == min(v["total_ms"] for v in g.values())
        # 8 x 4 computes fewer pair slots than 8 x 8 on every size
        assert g["4"]["slots"] < g["8"]["slots"]
        # item split and register budget: the fastest of the sweep (at 8 x 8)
        best = min(e["sweep"], key=lambda r: r["total_ms"])
        assert (best["max_entries"], best["force_min_blocks"]) == (e["max_entries"], e["force_min_blocks"])
        b = e["build_ms_by_search_mode"]
        assert b[str(e["search_mode"])] == min(b.values())
        en = e["energy_eval_ms_by_energy_mode"]
        assert en[str(e["energy_mode"])] == min(en.values())


def test_lookup_takes_the_nearest_size_in_log_atoms():
    gpu = TABLE["gpu"]
    for coul in ("rf", "ewald"):
        entries = [e for e in TABLE["entries"] if e["coul"] == coul]
        for n in (1000, 3000, 9000, 24000, 70000, 500000, 3000000, 9000000):
            want = min(entries, key=lambda e: abs(math.log(e["atoms"]) - math.log(n)))
            got = autotune.lookup(TABLE, coul, n, gpu)
            assert got == {"max_entries": want["max_entries"], "force_min_blocks": want["force_min_blocks"],
                           "search_mode": want["search_mode"], "energy_mode": want["energy_mode"],
                           "jcluster": want["jcluster"]}


def test_lookup_defaults_for_another_gpu_or_no_table():
    default = {"max_entries": 32, "force_min_blocks": 3, "search_mode": 0, "energy_mode": 0, "jcluster": 8}
    assert autotune.lookup(TABLE, "rf", 24000, "another GPU") == default
    assert autotune.lookup(None, "ewald", 24000) == default
