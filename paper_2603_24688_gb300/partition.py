"""Spatial decomposition of the interaction step over ranks: slabs and ghost imports.

Rank r owns the particles of slab r, a range of x chosen so that every slab holds about the
same number of particles, and imports as ghosts the particles of both species within
R = max h_DM + max h_gas of its slab (through the periodic faces when the box is periodic).
It runs the step on its owned and ghost particles and keeps the outputs of its owned
particles only:

* the mean field of an owned gas particle sums over all its DM partners, and every partner
  lies within h_i + h_j <= R of it, so inside the slab or its ghost zone;
* the Monte Carlo of an owned DM particle draws over all its gas partners, likewise;
* the random numbers key on global ids and the step number (never on an index), so the owned
  outputs equal those of the whole step;
* the step's conservation sums are sums over particles (and the pair count a sum over gas
  rows), so they are the sum over ranks of the owned particles' terms: one allreduce of 16
  doubles, the only exchange besides the ghost import.

Local arrays keep the particles in increasing global index, so a rank's rows list their
partners in the same relative order as the whole step does.  This module only selects
particles; it holds none of the method's arithmetic.
"""
import numpy as np


def slab_edges(x, nparts):
    """Interior slab boundaries: nparts - 1 quantiles of the x coordinates of all particles."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    return np.quantile(np.asarray(x, dtype=np.float64), np.arange(1, nparts) / nparts)


def interaction_range(dm, gas):
    """R = max h_DM + max h_gas: no pair is farther apart than this."""
    hd = float(np.max(dm["h"])) if len(dm["h"]) else 0.0
    hg = float(np.max(gas["h"])) if len(gas["h"]) else 0.0
    return hd + hg


def _slab_bounds(edges, r):
    lo = -np.inf if r == 0 else edges[r - 1]
    hi = np.inf if r == len(edges) else edges[r]
    return lo, hi


def owned(x, edges, r):
    """Mask of the particles (x coordinates) owned by rank r."""
    lo, hi = _slab_bounds(edges, r)
    return (x >= lo) & (x < hi)


def ghosts(x, edges, r, R, periodic=False, L=None):
    """Mask of the particles not owned by rank r that lie within R of its slab in x."""
    lo, hi = _slab_bounds(edges, r)
    own = (x >= lo) & (x < hi)
    if not periodic:
        near = ((x >= lo - R) & (x < lo)) | ((x >= hi) & (x < hi + R))
        return near & ~own
    L = float(L)
    # distance along x to the slab through the periodic faces (slab bounds wrapped into [0, L))
    a = 0.0 if not np.isfinite(lo) else lo
    b = L if not np.isfinite(hi) else hi
    to_lo = np.mod(a - x, L)          # from x forward to the slab's lower face
    from_hi = np.mod(x - b, L)        # from the slab's upper face forward to x
    return (np.minimum(to_lo, from_hi) < R) & ~own


def subset(particles, idx):
    """The particles at the global indices idx (increasing), as a new dict of arrays."""
    return {k: v[idx] for k, v in particles.items()}


def rank_view(dm, gas, edges, r, periodic=False, box=None):
    """Local particles of rank r: global index arrays (owned and ghosts, increasing) of each
    species and the masks of the owned ones among them."""
    R = interaction_range(dm, gas)
    L = None if not periodic else float(np.asarray(box)[0])
    out = {}
    for name, sp in (("dm", dm), ("gas", gas)):
        x = sp["pos"][:, 0]
        if periodic:
            x = np.mod(x, L)
        own = owned(x, edges, r)
        take = own | ghosts(x, edges, r, R, periodic, L)
        idx = np.nonzero(take)[0]
        out[name] = idx
        out[name + "_owned"] = own[idx]
    return out
