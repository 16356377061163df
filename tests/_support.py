"""Test helpers: run the CUDA path through the C ABI and expand its pair list.

Test infrastructure; the expansion reads the list exactly as the kernels do
(bit 8*i + t of an entry's mask = pair (i-slot i, j-slot t XOR i), j-slot j
at sorted slot jslot[e, j // 4] + j % 4, the i-cluster displaced by the
item's periodic shift), for either j-cluster geometry.
"""
import numpy as np

from paper_1506_00716_gb300 import nb


def gpu_eval(ctx, sys, params, flags=nb.NB_F_ENERGY | nb.NB_F_VIRIAL, keep=False):
    """Grid put, list build and one evaluation; returns (f, energy, virial, handle-or-None)."""
    h = nb.nb_sys_create(ctx, params, sys.n, sys.box, getattr(sys, "skew", None))
    nb.nb_set_exclusions(h, sys.excl_index, sys.excl_atoms)
    nb.nb_grid_put(h, np.ascontiguousarray(sys.xq()), np.ascontiguousarray(sys.type))
    nb.nb_pairlist_build(h)
    f = np.zeros((sys.n, 3), dtype=np.float32)
    e = np.zeros(2)
    v = np.zeros(9)
    nb.nb_forces(h, None, f, e, v, flags)
    if keep:
        return f, e, v, h
    nb.nb_sys_destroy(h)
    return f, e, v, None


def export_list(h):
    info = nb.nb_pairlist_info(h)
    perm = np.zeros(info["n_clusters"] * 8, dtype=np.int32)
    items = np.zeros((max(info["n_items"], 1), 4), dtype=np.int32)
    ne = nb.nb_pairlist_export_slots(h)  # the entry arrays' extent (the largest item end)
    jslot = np.zeros((max(ne, 1), 2), dtype=np.int32)
    mask = np.zeros(max(ne, 1), dtype=np.uint64)
    nb.nb_pairlist_export_slots(h, perm, items, jslot, mask)
    return info, perm, items[: info["n_items"]], jslot, mask


def expand_pairs(sys, perm, items, jslot, mask, r_cut, chunk=20000):
    """Atom pairs (i<j keys) of the list whose distance under the entry's shift is < r_cut
    (float64), plus the number of such (pair, shift) occurrences (duplicates > 0 = double count)."""
    n = sys.n
    x = sys.x.astype(np.float64)
    L = sys.box
    ent_item = np.zeros(0, dtype=np.int64)
    ent_idx = np.zeros(0, dtype=np.int64)
    lens = items[:, 2] - items[:, 1]
    ent_item = np.repeat(np.arange(items.shape[0]), lens)
    ent_idx = np.concatenate([np.arange(a, b) for a, b in zip(items[:, 1], items[:, 2])]) \
        if items.shape[0] else np.zeros(0, dtype=np.int64)
    keys_all = []
    count = 0
    bits = np.arange(64, dtype=np.uint64)
    for s in range(0, ent_idx.shape[0], chunk):
        e = ent_idx[s:s + chunk]
        it = items[ent_item[s:s + chunk]]
        m = mask[e]
        on = ((m[:, None] >> bits[None, :]) & np.uint64(1)).astype(bool)
        er, bit = np.nonzero(on)
        i = bit // 8
        j = (bit % 8) ^ i
        ci = it[er, 0]
        sh = it[er, 3]
        a = perm[ci * 8 + i]
        b = perm[jslot[e[er], j // 4] + j % 4]
        ok = (a >= 0) & (b >= 0)
        a, b, sh = a[ok], b[ok], sh[ok]
        sx, sy, sz = sh // 9 - 1, (sh // 3) % 3 - 1, sh % 3 - 1
        bx, cx, cy = getattr(sys, "skew", np.zeros(3))
        S = np.stack([sx * L[0] + sy * bx + sz * cx, sy * L[1] + sz * cy, sz * L[2]], axis=1)
        d = x[a] + S - x[b]
        r2 = (d * d).sum(1)
        w = r2 < r_cut * r_cut
        a, b = a[w], b[w]
        count += a.shape[0]
        keys_all.append(np.minimum(a, b).astype(np.int64) * n + np.maximum(a, b))
    keys = np.unique(np.concatenate(keys_all)) if keys_all else np.zeros(0, dtype=np.int64)
    return keys, count


def rel_rms(f, ref):
    return float(np.sqrt(((f - ref) ** 2).mean()) / np.sqrt((ref ** 2).mean()))


def expand_pairs_of_rows(sys, perm, items, jslot, mask, r_cut, sel, chunk=200000):
    """Atom pairs (min * n + max keys, unique, sorted) of the list that touch an
    atom of `sel` and lie closer than r_cut under their entry's shift (float64
    distance of the float32 inputs), and the number of (pair, shift)
    occurrences among them (more than the unique keys = a pair listed twice).

    Only the entries whose i- or j-cluster holds a selected atom are expanded,
    so a list of tens of millions of entries stays within seconds."""
    n = sys.n
    x = sys.x.astype(np.float64)
    L = sys.box
    bx, cx, cy = getattr(sys, "skew", np.zeros(3))
    sel = np.asarray(sel, dtype=np.int64)
    is_sel = np.zeros(n, dtype=bool)
    is_sel[sel] = True
    ncl = perm.shape[0] // 8
    slot_atom = perm.reshape(ncl, 8)
    cl_sel = ((slot_atom >= 0) & is_sel[np.maximum(slot_atom, 0)]).any(1)
    lens = (items[:, 2] - items[:, 1]).astype(np.int64)
    total = int(lens.sum())
    ent_item = np.repeat(np.arange(items.shape[0]), lens)
    offs = np.cumsum(lens) - lens
    ent_idx = np.arange(total, dtype=np.int64) - np.repeat(offs, lens) + np.repeat(items[:, 1].astype(np.int64), lens)
    keep = cl_sel[items[ent_item, 0]] | cl_sel[jslot[ent_idx, 0] // 8] | cl_sel[jslot[ent_idx, 1] // 8]
    ent_item, ent_idx = ent_item[keep], ent_idx[keep]
    bits = np.arange(64, dtype=np.uint64)
    keys_all = []
    count = 0
    for s in range(0, ent_idx.shape[0], chunk):
        e = ent_idx[s:s + chunk]
        it = items[ent_item[s:s + chunk]]
        on = ((mask[e][:, None] >> bits[None, :]) & np.uint64(1)).astype(bool)
        er, bit = np.nonzero(on)
        i = bit // 8
        j = (bit % 8) ^ i
        a = perm[it[er, 0] * 8 + i]
        b = perm[jslot[e[er], j // 4] + j % 4]
        sh = it[er, 3]
        ok = (a >= 0) & (b >= 0)
        a, b, sh = a[ok], b[ok], sh[ok]
        ok = is_sel[a] | is_sel[b]
        a, b, sh = a[ok], b[ok], sh[ok]
        sx, sy, sz = sh // 9 - 1, (sh // 3) % 3 - 1, sh % 3 - 1
        S = np.stack([sx * L[0] + sy * bx + sz * cx, sy * L[1] + sz * cy, sz * L[2]], axis=1)
        d = x[a] + S - x[b]
        w = (d * d).sum(1) < r_cut * r_cut
        a, b = a[w], b[w]
        count += a.shape[0]
        keys_all.append(np.minimum(a, b).astype(np.int64) * n + np.maximum(a, b))
    keys = np.unique(np.concatenate(keys_all)) if keys_all else np.zeros(0, dtype=np.int64)
    return keys, count
