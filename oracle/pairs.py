"""DM-gas pair set (oracle, FP64).

The overlap g_ij is non-zero exactly when d_ij < h_i + h_j (the kernel has
support [0, h), Sec. 2.4; App. D notes g = 0 for d > h_i + h_j).  The paper finds
these pairs with GIZMO's tree by searching 2h from both sides (Sec. 2.4); the
set is the same, so the oracle enumerates it directly:

    pairs = {(i, j) : |x_i - x_j| < h_i + h_j}   (strict; minimum image if periodic)

Reading: each pair appears once; equal h needs no tie-break because this is a set.

Parity: pinned by construction (brute force is the definition); the cell list
is checked against brute force in tests/test_oracle_pairs.py.
"""
import numpy as np


def min_image(dx, box):
    """Minimum-image displacement for a periodic box of sides box[3]."""
    box = np.asarray(box, dtype=np.float64)
    return dx - box * np.round(dx / box)


def pair_distance(dm_pos, gas_pos, periodic, box):
    dx = dm_pos - gas_pos
    if periodic:
        dx = min_image(dx, box)
    return np.sqrt(np.sum(dx * dx, axis=-1))


def pairs_bruteforce(dm, gas, periodic=False, box=None, dm_subset=None, gas_subset=None,
                     block=2048):
    """All (i, j) with d_ij < h_i + h_j; i indexes dm, j indexes gas.

    dm_subset / gas_subset restrict the query to those indices (used to check
    sampled particles of very large inputs).  Returned sorted by (i, j).
    """
    ii = np.arange(len(dm["h"])) if dm_subset is None else np.asarray(dm_subset)
    jj = np.arange(len(gas["h"])) if gas_subset is None else np.asarray(gas_subset)
    gp = gas["pos"][jj]
    gh = gas["h"][jj]
    out_i, out_j = [], []
    for s in range(0, len(ii), block):
        blk = ii[s:s + block]
        dx = dm["pos"][blk][:, None, :] - gp[None, :, :]
        if periodic:
            dx = min_image(dx, box)
        d2 = np.sum(dx * dx, axis=-1)
        r = dm["h"][blk][:, None] + gh[None, :]
        a, b = np.nonzero(d2 < r * r)
        # d2 < r^2 and d < r agree except where rounding of the square root decides;
        # keep the definition d < r exactly.
        keep = np.sqrt(d2[a, b]) < r[a, b]
        out_i.append(blk[a[keep]])
        out_j.append(jj[b[keep]])
    if not out_i:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    pi = np.concatenate(out_i).astype(np.int64)
    pj = np.concatenate(out_j).astype(np.int64)
    order = np.lexsort((pj, pi))
    return pi[order], pj[order]


def pairs_celllist(dm, gas, periodic, box, lo=None):
    """The same set with a plain uniform cell list (cell side >= max h_i + max h_j).

    Intended for uniform boxes where a single cell size fits every particle.
    """
    box = np.asarray(box, dtype=np.float64)
    rmax = dm["h"].max() + gas["h"].max()
    lo = np.zeros(3) if lo is None else np.asarray(lo, dtype=np.float64)
    ncell = np.maximum(np.floor(box / rmax).astype(np.int64), 1)
    if np.any(ncell < 3) or not periodic:
        return pairs_bruteforce(dm, gas, periodic, box)
    side = box / ncell

    def cell_of(p):
        c = np.floor((p - lo) / side).astype(np.int64)
        return np.mod(c, ncell)

    cd = cell_of(dm["pos"])
    cg = cell_of(gas["pos"])
    key_g = (cg[:, 0] * ncell[1] + cg[:, 1]) * ncell[2] + cg[:, 2]
    order_g = np.argsort(key_g, kind="stable")
    sorted_keys = key_g[order_g]
    ncells_total = int(np.prod(ncell))
    starts = np.searchsorted(sorted_keys, np.arange(ncells_total), side="left")
    ends = np.searchsorted(sorted_keys, np.arange(ncells_total), side="right")
    out_i, out_j = [], []
    for off in np.ndindex(3, 3, 3):
        o = np.array(off) - 1
        nb = np.mod(cd + o, ncell)
        key = (nb[:, 0] * ncell[1] + nb[:, 1]) * ncell[2] + nb[:, 2]
        cnt = ends[key] - starts[key]
        rep_i = np.repeat(np.arange(len(cd)), cnt)
        base = np.repeat(starts[key], cnt)
        within = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        jj = order_g[base + within]
        d = pair_distance(dm["pos"][rep_i], gas["pos"][jj], True, box)
        keep = d < dm["h"][rep_i] + gas["h"][jj]
        out_i.append(rep_i[keep])
        out_j.append(jj[keep])
    pi = np.concatenate(out_i).astype(np.int64)
    pj = np.concatenate(out_j).astype(np.int64)
    # with >= 3 cells per side the 27 offsets are distinct cells, so no duplicates
    order = np.lexsort((pj, pi))
    return pi[order], pj[order]
