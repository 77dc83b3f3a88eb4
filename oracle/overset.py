"""Overset assembly and inverse-distance interpolation (test infrastructure).

Plain FP64 numpy restatement of Sec. 3.1 (assembly) and Sec. 3.2
(interpolation).  Every predicate uses FP64 add / multiply / divide /
compare only, evaluated in the order written here, so a device
implementation evaluating the same expressions in the same order without
fused multiply-add reproduces the result bit for bit.

Readings (the node-classification sentence of Sec. 3.1 is garbled):
  O1 wall distance of a node to a zone = min over that zone's wall segments
     (squared Euclidean distance to the segment, compared squared); a zone
     without walls has distance +inf.
  O2 a node p of zone Z is inactive if it lies strictly inside the wall
     polygon of another zone (a body), or if another zone D has a "core"
     cell containing p (inclusive edges) and d_D(p) < d_Z(p), ties going to
     the higher priority.  Core cells exclude the fringe and gap layers along
     a zone's overset outer edge.  Nodes with no such zone stay active.
  O3 cells: inactive (HOLE) if all nodes are inactive, boundary if mixed;
     cells in the n_fringe layers along an overset outer edge are boundary;
     the buffer layer is every active face neighbour of a boundary (mixed)
     or hole cell.  Receptors = boundary + buffer; the rest are FIELD.
  O4 donor of a receptor (its vertex centre at t^{n+1}) = a cell of another
     zone containing it: FIELD cells first, then RECEPTOR cells; within each
     class by (higher priority, lower block index, lower cell index); none ->
     orphan.
  O5 interpolation stencil (Sec. 3.2) = the donor and its logical face
     neighbours that are not holes, order (donor, i-1, i+1, j-1, j+1),
     weights d^-2 / sum d^-2 summed in that order; a zero distance takes that
     cell's value.  All receptors read their donors' values from before the
     pass (Jacobi), so chained receptors are well defined and lag one pass.
  O6 cells uncovered by the motion (HOLE before, FIELD now) are initialised
     once per step from donors found the same way.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .mesh import NB_CELL, Topology
from .ugks import FIELD, HOLE, RECEPTOR, State
from paper_2604_09984_gb300.workloads import BC_OVERSET, BC_WALL


@dataclass
class Connectivity:
    status: np.ndarray        # (nc,) FIELD / RECEPTOR / HOLE
    node_active: np.ndarray   # (nn,) bool
    receptors: np.ndarray     # (nr,) cell ids, ascending
    donors: np.ndarray        # (nr, 5) stencil cell ids, -1 unused
    weights: np.ndarray       # (nr, 5)
    fresh: np.ndarray         # (nfr,) cell ids
    fresh_donors: np.ndarray
    fresh_weights: np.ndarray
    n_orphan: int


def block_side_nodes(blk, X, side):
    if side == 0:
        return X[0, :, :]
    if side == 1:
        return X[blk.ni, :, :]
    if side == 2:
        return X[:, 0, :]
    return X[:, blk.nj, :]


def wall_segments(blk, X):
    segs = []
    for side in range(4):
        if blk.bc[side] == BC_WALL:
            P = block_side_nodes(blk, X, side)
            segs.append(np.stack([P[:-1], P[1:]], axis=1))
    if not segs:
        return np.zeros((0, 2, 2))
    return np.concatenate(segs, axis=0)


def body_polygon(blk, X):
    """Closed wall ring of a body-fitted periodic block (its j = 0 side)."""
    if blk.periodic_i and blk.bc[2] == BC_WALL:
        return X[:blk.ni, 0, :]
    return None


def wall_dist2(p, segs):
    """Squared distance from points p (N, 2) to the nearest segment (reading O1)."""
    if segs.shape[0] == 0:
        return np.full(p.shape[0], np.inf)
    ax = segs[None, :, 0, 0]
    ay = segs[None, :, 0, 1]
    ex = segs[None, :, 1, 0] - ax
    ey = segs[None, :, 1, 1] - ay
    px = p[:, None, 0] - ax
    py = p[:, None, 1] - ay
    t = (px * ex + py * ey) / (ex * ex + ey * ey)
    t = np.minimum(np.maximum(t, 0.0), 1.0)
    dx = px - t * ex
    dy = py - t * ey
    return (dx * dx + dy * dy).min(axis=1)


def inside_quads(p, quads):
    """(N, C) inclusive point-in-convex-quad test: every edge cross product of
    the counter-clockwise quad is >= 0."""
    ok = np.ones((p.shape[0], quads.shape[0]), dtype=bool)
    for e in range(4):
        a = quads[None, :, e, :]
        b = quads[None, :, (e + 1) % 4, :]
        cr = ((b[..., 0] - a[..., 0]) * (p[:, None, 1] - a[..., 1])
              - (b[..., 1] - a[..., 1]) * (p[:, None, 0] - a[..., 0]))
        ok &= cr >= 0.0
    return ok


def inside_polygon(p, poly):
    """Crossing-number point-in-polygon (strict interior up to ties)."""
    inside = np.zeros(p.shape[0], dtype=bool)
    M = poly.shape[0]
    for i in range(M):
        a = poly[i]
        b = poly[(i + 1) % M]
        crosses = (a[1] > p[:, 1]) != (b[1] > p[:, 1])
        dy = b[1] - a[1]
        safe = np.where(crosses, dy, 1.0)
        xint = a[0] + (p[:, 1] - a[1]) * (b[0] - a[0]) / safe
        inside ^= crosses & (p[:, 0] < xint)
    return inside


def _core_mask(blk):
    """Cells of a block usable to cut holes: not within n_fringe + n_gap
    layers of an overset outer side."""
    m = np.ones((blk.ni, blk.nj), dtype=bool)
    L = blk.n_fringe + blk.n_gap
    for side in range(4):
        if blk.bc[side] == BC_OVERSET:
            if side == 0:
                m[:L, :] = False
            elif side == 1:
                m[blk.ni - L:, :] = False
            elif side == 2:
                m[:, :L] = False
            else:
                m[:, blk.nj - L:] = False
    return m.T.ravel()        # cell order j*ni + i


def _fringe_mask(blk):
    m = np.zeros((blk.ni, blk.nj), dtype=bool)
    L = blk.n_fringe
    for side in range(4):
        if blk.bc[side] == BC_OVERSET:
            if side == 0:
                m[:L, :] = True
            elif side == 1:
                m[blk.ni - L:, :] = True
            elif side == 2:
                m[:, :L] = True
            else:
                m[:, blk.nj - L:] = True
    return m.T.ravel()


def _quads(topo, Xn, bi):
    c0, c1 = topo.cell_off[bi], topo.cell_off[bi + 1]
    return Xn[topo.cell_nodes[c0:c1]]      # (C, 4, 2)


def _first_containing(p, quads, allowed, chunk=2048):
    """Index of the lowest-numbered allowed quad containing each point, -1 if
    none."""
    res = np.full(p.shape[0], -1, dtype=np.int64)
    idx = np.nonzero(allowed)[0]
    if idx.size == 0:
        return res
    Q = quads[idx]
    for s in range(0, p.shape[0], chunk):
        ok = inside_quads(p[s:s + chunk], Q)
        anyk = ok.any(axis=1)
        first = ok.argmax(axis=1)
        r = np.where(anyk, idx[first], -1)
        res[s:s + chunk] = r
    return res


def connect(topo: Topology, X_new_list, prev_status=None) -> Connectivity:
    """Overset assembly at t^{n+1} (Sec. 3.1; readings O1-O6)."""
    blocks = topo.blocks
    nb = len(blocks)
    Xn = topo.concat_nodes(X_new_list)
    segs = [wall_segments(b, X) for b, X in zip(blocks, X_new_list)]
    polys = [body_polygon(b, X) for b, X in zip(blocks, X_new_list)]
    cores = [_core_mask(b) for b in blocks]
    node_active = np.ones(topo.nn, dtype=bool)
    for z in range(nb):
        n0, n1 = topo.node_off[z], topo.node_off[z + 1]
        p = Xn[n0:n1]
        dz = wall_dist2(p, segs[z])
        inact = np.zeros(p.shape[0], dtype=bool)
        for d in range(nb):
            if d == z:
                continue
            if polys[d] is not None:
                inact |= inside_polygon(p, polys[d])
            hit = _first_containing(p, _quads(topo, Xn, d), cores[d]) >= 0
            dd = wall_dist2(p, segs[d])
            wins = (dd < dz) | ((dd == dz) & (blocks[d].priority > blocks[z].priority))
            inact |= hit & wins
        node_active[n0:n1] = ~inact
    # cell classification (reading O3)
    act = node_active[topo.cell_nodes]          # (nc, 4)
    nact = act.sum(axis=1)
    status = np.full(topo.nc, FIELD, dtype=np.int64)
    mixed = (nact > 0) & (nact < 4)
    status[nact == 0] = HOLE
    status[mixed] = RECEPTOR
    fringe = np.concatenate([_fringe_mask(b) for b in blocks])
    status[fringe & (nact > 0)] = RECEPTOR
    seed = mixed | (status == HOLE)
    buf = np.zeros(topo.nc, dtype=bool)
    for d in range(4):
        m = topo.nb_kind[:, d] == NB_CELL
        nbid = np.where(m, topo.nb_id[:, d], 0)
        buf |= m & seed[nbid]
    status[(status == FIELD) & buf] = RECEPTOR

    xc_new = 0.25 * ((Xn[topo.cell_nodes[:, 0]] + Xn[topo.cell_nodes[:, 1]])
                     + (Xn[topo.cell_nodes[:, 2]] + Xn[topo.cell_nodes[:, 3]]))
    receptors = np.nonzero(status == RECEPTOR)[0]
    if prev_status is None:
        fresh = np.zeros(0, dtype=np.int64)
    else:
        fresh = np.nonzero((prev_status == HOLE) & (status == FIELD))[0]
    rd, rw, no1 = _donors(topo, Xn, xc_new, status, receptors)
    fd, fw, no2 = _donors(topo, Xn, xc_new, status, fresh)
    return Connectivity(status, node_active, receptors, rd, rw, fresh, fd, fw, no1 + no2)


def _donors(topo, Xn, xc_new, status, cells):
    """Donor search (O4) and IDW stencil weights (O5) for the given cells."""
    blocks = topo.blocks
    nb = len(blocks)
    n = cells.size
    donors = np.full((n, 5), -1, dtype=np.int64)
    weights = np.zeros((n, 5))
    if n == 0:
        return donors, weights, 0
    order = sorted(range(nb), key=lambda b: (-blocks[b].priority, b))
    found = np.full(n, -1, dtype=np.int64)
    cb = topo.cell_block[cells]
    p = xc_new[cells]
    for cls in (FIELD, RECEPTOR):
        for d in order:
            todo = (found < 0) & (cb != d)
            if not todo.any():
                continue
            c0 = topo.cell_off[d]
            allowed = status[c0:topo.cell_off[d + 1]] == cls
            loc = _first_containing(p[todo], _quads(topo, Xn, d), allowed)
            hit = loc >= 0
            idx = np.nonzero(todo)[0]
            found[idx[hit]] = c0 + loc[hit]
    orphan = int((found < 0).sum())
    for r in range(n):
        dnr = found[r]
        if dnr < 0:
            continue
        st = [dnr]
        for d in range(4):
            if topo.nb_kind[dnr, d] == NB_CELL:
                c = topo.nb_id[dnr, d]
                if status[c] != HOLE:
                    st.append(c)
        x = p[r]
        d2 = [(x[0] - xc_new[c, 0]) * (x[0] - xc_new[c, 0])
              + (x[1] - xc_new[c, 1]) * (x[1] - xc_new[c, 1]) for c in st]
        donors[r, :len(st)] = st
        zero = [k for k, v in enumerate(d2) if v == 0.0]
        if zero:
            weights[r, zero[0]] = 1.0
            continue
        inv = [1.0 / v for v in d2]
        tot = 0.0
        for v in inv:
            tot = tot + v
        for k, v in enumerate(inv):
            weights[r, k] = v / tot
    return donors, weights, orphan


def interpolate(st: State, cells, donors, weights):
    """phi_r = sum_j w_rj phi_j (Sec. 3.2) for f, W and q, summed in stencil
    order; donors read the values before this pass (Jacobi)."""
    if cells.size == 0:
        return
    f0, W0, q0 = st.f.copy(), st.W.copy(), st.q.copy()
    for r, c in enumerate(cells):
        if donors[r, 0] < 0:
            continue
        af = np.zeros_like(f0[0])
        aW = np.zeros(4)
        aq = np.zeros(2)
        for k in range(5):
            d = donors[r, k]
            if d < 0:
                continue
            af = af + weights[r, k] * f0[d]
            aW = aW + weights[r, k] * W0[d]
            aq = aq + weights[r, k] * q0[d]
        st.f[c] = af
        st.W[c] = aW
        st.q[c] = aq
