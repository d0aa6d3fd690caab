"""The split order of the device build, checked on the CPU against the oracle's tree.

The device build does not run the median split (Sec. III) as a recursion.  It sorts three
lists of the triangles once, by (centroid key on one axis, triangle index), then runs one
round per level of the binary split tree.  In each round every segment of two or more
triangles takes the axis of largest centroid extent (read from the ends of the three
lists), keeps the first half of that axis's list on the left, and lets the other two
lists follow by a stable partition, so that every list stays sorted inside every segment.
This test runs those steps in numpy, in the device's order.  The leaves it yields, in
breadth-first order, must be the oracle's own: ties, signed zeros, ragged counts and
every branching included."""
from collections import deque

import numpy as np
import pytest

import oracle
import synth


def _leaf_positions(nt, m):
    """Position in the final split order of each leaf, leaves in breadth-first order (the
    shape alone: every node's triangles halved log2(m) times)."""
    q, leaves = deque([(0, nt)]), []
    while q:
        s, n = q.popleft()
        if n == 1:
            leaves.append(s)
            continue
        groups, r = [(s, n)], 1
        while r < m:
            groups = [g for a, b in groups for g in (((a, 1),) if b == 1 else ((a, b // 2), (a + b // 2, b - b // 2)))]
            r <<= 1
        q.extend(groups)
    return np.array(leaves)


def _split_order(v, t):
    nt = len(t)
    p = v[t].astype(np.float64)
    key = (p[:, 0] + p[:, 1]) + p[:, 2]  # the builder's centroid key, summed in this order
    idx = np.arange(nt)
    # stable sort by the key (np.lexsort: the last key is the primary one); +0 and -0 tie
    L = np.stack([np.lexsort((idx, key[:, c] + 0.0)) for c in range(3)])
    seg_s, seg_n = np.zeros(nt, np.int64), np.full(nt, nt, np.int64)
    flag = np.zeros(nt, np.int64)
    width = 1
    while width < nt:
        act = seg_n >= 2
        s, n = seg_s, seg_n
        ends = np.minimum(s + n - 1, nt - 1)
        ext = np.stack([key[L[c, ends], c] - key[L[c, s], c] for c in range(3)])
        ax = np.zeros(nt, np.int64)
        ax[ext[1] > ext[0]] = 1
        ax[ext[2] > ext[ax, idx]] = 2
        flag[L[ax[act], idx[act]]] = ((idx - s) < n // 2)[act]
        X = np.concatenate([[0], np.cumsum(flag[L.reshape(-1)])[:-1]]).reshape(3, nt)
        Ln = np.empty_like(L)
        for c in range(3):
            lb = X[c] - X[c, s]
            pos = np.where(flag[L[c]] == 1, s + lb, s + n // 2 + (idx - s - lb))
            Ln[c, np.where(act, pos, idx)] = L[c]
        half = n // 2
        left = (idx - s) < half
        seg_s = np.where(act & ~left, s + half, s)
        seg_n = np.where(act, np.where(left, half, n - half), n)
        L = Ln
        width <<= 1
    assert (L[0] == L[1]).all() and (L[0] == L[2]).all()  # every segment is one triangle
    return L[0]


def _signed_zeros():
    v, t = synth.heightfield(20, 4.0, seed=6)[:2]
    v = v.copy()
    v[v == 0.0] = -0.0
    v[::7, 2] = 0.0
    return v, t


MESHES = {
    "sphere": lambda: synth.icosphere(3, 1.0, 0.15, seed=9),
    "terrain_ties": lambda: synth.heightfield(40, 4.0, seed=4)[:2],
    "signed_zero": _signed_zeros,
    "ragged": lambda: (synth.icosphere(3, 1.0, 0.15, seed=3)[0], synth.icosphere(3, 1.0, 0.15, seed=3)[1][:1111]),
    "three": lambda: (synth.icosphere(1)[0], synth.icosphere(1)[1][5:8]),
}


@pytest.mark.parametrize("m", [2, 4, 8, 16])
@pytest.mark.parametrize("mesh", list(MESHES))
def test_split_rounds_give_the_oracle_leaves(mesh, m):
    v, t = MESHES[mesh]()
    order = _split_order(np.asarray(v, np.float32), np.asarray(t, np.int32))
    tr = oracle.BVH(v, t, 18, m, 8, 4096).tree()
    leaves = tr["tri"][tr["nchild"] == 0]  # nodes are numbered breadth-first
    assert (order[_leaf_positions(len(t), m)] == leaves).all()
