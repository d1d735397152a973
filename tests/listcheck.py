"""Entry-level check of the FP32 interaction-list entries (Sec. 3.1.1: positions relative
to the group's centre, single precision) against values derived from the oracle.

For an index entry (kind, index, image shift) of group g the oracle gives the position
exactly in FP64: the sorted particle's wrapped position, or the node's centre of mass
(Sec. 3.1.2), plus shift * L.  The FP32 entry must hold (that position - centre of the
group's cell) / r_cut within a few FP32 roundings, and the mass: a particle's exactly,
a node's total mass rounded to FP32 (within one unit in the last place, since the two
sides sum the FP64 moments in different orders).
"""
import numpy as np

# |FP32 entry - FP64 value| <= REL_TOL * (|value|_inf + 1), per component.  The entry is
# (integer cell offset) * fl(u / r_cut) + (FP32 offset from the cell's centre): a handful
# of FP32 roundings of terms of magnitude below |value| + 1 (offsets within a cell are
# below one r_cut for every accepted node), far below any misplaced cell (one finest
# cell, L / 2^21, is 2e-5 r_cut at the 256^3 workload's r_cut = 3/256).
REL_TOL = 2.0 ** -21


def expected_entries(T, L, r_cut, groups, offsets, index_entries):
    """FP64 expected (rel [E,3], mass [E], kind [E]) for the index entries of the selected
    groups (oracle tree T; groups in the same order as the dump)."""
    nodes, mom, grp = T.nodes(), T.moments(), T.groups()
    _, _, xyz, ms = T.sorted()
    gn = grp[np.asarray(groups)]
    side = L / (2.0 ** nodes[gn, 0])
    centre = (nodes[gn, 1:4].astype(np.float64) + 0.5) * side[:, None]
    lens = np.diff(offsets)
    cen = np.repeat(centre, lens, axis=0)
    kind, idx, sh = index_entries[:, 0], index_entries[:, 1], index_entries[:, 2:5].astype(np.float64)
    part = kind == 0
    pos = np.empty((len(kind), 3))
    pos[part] = xyz[idx[part]]
    pos[~part] = mom[idx[~part], 1:]
    pos += sh * L
    mass = np.empty(len(kind))
    mass[part] = ms[idx[part]].astype(np.float64)
    mass[~part] = mom[idx[~part], 0]
    return (pos - cen) / r_cut, mass, kind


def check_entries(f32, rel, mass, kind):
    """Asserts the FP32 entries [E,4] against the expected values; returns the largest
    component error in units of REL_TOL * (|value| + 1)."""
    assert f32.shape == (len(kind), 4)
    scale = np.abs(rel).max(axis=1, keepdims=True) + 1.0
    err = np.abs(f32[:, :3].astype(np.float64) - rel) / scale
    worst = float(err.max() / REL_TOL) if len(err) else 0.0
    assert worst <= 1.0, worst
    part = kind == 0
    assert np.array_equal(f32[part, 3], mass[part].astype(np.float32))
    m32 = mass[~part].astype(np.float32)
    ulp = np.spacing(np.abs(m32))
    assert np.all(np.abs(f32[~part, 3].astype(np.float64) - m32) <= ulp)
    return worst
