"""Structured-block topology and ALE geometry (test infrastructure).

Blocks are logically rectangular quad meshes (ni x nj cells, node array
(ni+1, nj+1, 2); periodic blocks repeat column 0 as column ni, the difference
being the period vector: zero for an O-grid, the channel length for a
periodic channel).  Cell (i, j) has the counter-clockwise nodes
(i,j), (i+1,j), (i+1,j+1), (i,j+1); global cell id = offset + j*ni + i.

Readings of the paper (which says nothing about how moving geometry enters
the Crank-Nicolson step, Sec. 2.2):
  * face length S, normal n and centre, and cell centres are taken at the
    mid-time nodes x^{n+1/2} = (x^n + x^{n+1})/2;
  * the face velocity U_f is the mean of its two node velocities
    (x^{n+1} - x^n)/dt and S U.n = U_f . (S n)_{mid}; this equals the area
    swept by the face over the step divided by dt, so
    Omega^{n+1} - Omega^n = dt sum_faces S U.n (discrete GCL);
  * cell volumes Omega^n, Omega^{n+1} by the shoelace formula; the cell
    centre is the vertex mean.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from paper_2604_09984_gb300.workloads import BC_FARFIELD, BC_NONE, BC_OUTFLOW

NB_CELL, NB_GHOST, NB_NONE = 0, 1, 2
IM, IP, JM, JP = 0, 1, 2, 3


class Topology:
    def __init__(self, blocks):
        self.blocks = blocks
        self.cell_off = np.cumsum([0] + [b.ni * b.nj for b in blocks])
        self.node_off = np.cumsum([0] + [(b.ni + 1) * (b.nj + 1) for b in blocks])
        self.nc = int(self.cell_off[-1])
        self.nn = int(self.node_off[-1])
        nc = self.nc
        self.cell_block = np.empty(nc, dtype=np.int64)
        self.cell_i = np.empty(nc, dtype=np.int64)
        self.cell_j = np.empty(nc, dtype=np.int64)
        self.cell_nodes = np.empty((nc, 4), dtype=np.int64)
        self.cell_row_nodes = np.empty((nc, 2), dtype=np.int64)  # nodes (0,j),(ni,j)
        self.nb_kind = np.full((nc, 4), NB_NONE, dtype=np.int64)
        self.nb_id = np.full((nc, 4), -1, dtype=np.int64)
        self.nb_shift = np.zeros((nc, 4), dtype=np.int64)
        self.cell_faces = np.full((nc, 4), -1, dtype=np.int64)

        fL, fR, fa, fb, fkind, fside, fblock, fshL, fTw = ([] for _ in range(9))

        def add_face(L, R, a, b, kind, side, blk, shL, Tw):
            fL.append(L); fR.append(R); fa.append(a); fb.append(b)
            fkind.append(kind); fside.append(side); fblock.append(blk)
            fshL.append(shL); fTw.append(Tw)
            return len(fL) - 1

        for bi, blk in enumerate(blocks):
            ni, nj = blk.ni, blk.nj
            co, no = int(self.cell_off[bi]), int(self.node_off[bi])

            def cid(i, j):
                return co + j * ni + i

            def nid(i, j):
                return no + j * (ni + 1) + i

            for j in range(nj):
                for i in range(ni):
                    c = cid(i, j)
                    self.cell_block[c] = bi
                    self.cell_i[c] = i
                    self.cell_j[c] = j
                    self.cell_nodes[c] = (nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1))
                    self.cell_row_nodes[c] = (nid(0, j), nid(ni, j))
            # i-faces
            for j in range(nj):
                irange = range(ni) if blk.periodic_i else range(ni + 1)
                for i in irange:
                    if blk.periodic_i:
                        L = cid((i - 1) % ni, j)
                        R = cid(i, j)
                        f = add_face(L, R, nid(i, j), nid(i, j + 1), BC_NONE, -1, bi,
                                     -1 if i == 0 else 0, 0.0)
                        self.cell_faces[L, IP] = f
                        self.cell_faces[R, IM] = f
                    elif i == 0:
                        c = cid(0, j)
                        f = add_face(c, -1, nid(0, j + 1), nid(0, j), blk.bc[0], 0, bi, 0,
                                     blk.wall_T[0])
                        self.cell_faces[c, IM] = f
                    elif i == ni:
                        c = cid(ni - 1, j)
                        f = add_face(c, -1, nid(ni, j), nid(ni, j + 1), blk.bc[1], 1, bi, 0,
                                     blk.wall_T[1])
                        self.cell_faces[c, IP] = f
                    else:
                        L, R = cid(i - 1, j), cid(i, j)
                        f = add_face(L, R, nid(i, j), nid(i, j + 1), BC_NONE, -1, bi, 0, 0.0)
                        self.cell_faces[L, IP] = f
                        self.cell_faces[R, IM] = f
            # j-faces
            for i in range(ni):
                for j in range(nj + 1):
                    if j == 0:
                        c = cid(i, 0)
                        f = add_face(c, -1, nid(i, 0), nid(i + 1, 0), blk.bc[2], 2, bi, 0,
                                     blk.wall_T[2])
                        self.cell_faces[c, JM] = f
                    elif j == nj:
                        c = cid(i, nj - 1)
                        f = add_face(c, -1, nid(i + 1, nj), nid(i, nj), blk.bc[3], 3, bi, 0,
                                     blk.wall_T[3])
                        self.cell_faces[c, JP] = f
                    else:
                        L, R = cid(i, j - 1), cid(i, j)
                        f = add_face(L, R, nid(i + 1, j), nid(i, j), BC_NONE, -1, bi, 0, 0.0)
                        self.cell_faces[L, JP] = f
                        self.cell_faces[R, JM] = f
            # logical neighbours for reconstruction
            for j in range(nj):
                for i in range(ni):
                    c = cid(i, j)
                    for d, (di, dj, side) in enumerate(((-1, 0, 0), (1, 0, 1), (0, -1, 2), (0, 1, 3))):
                        ii, jj = i + di, j + dj
                        if 0 <= ii < ni and 0 <= jj < nj:
                            self.nb_kind[c, d] = NB_CELL
                            self.nb_id[c, d] = cid(ii, jj)
                        elif di != 0 and blk.periodic_i:
                            self.nb_kind[c, d] = NB_CELL
                            self.nb_id[c, d] = cid(ii % ni, jj)
                            self.nb_shift[c, d] = di
                        else:
                            kind = blk.bc[side]
                            if kind in (BC_FARFIELD, BC_OUTFLOW):
                                self.nb_kind[c, d] = NB_GHOST
                                self.nb_id[c, d] = self.cell_faces[c, d]
                            else:
                                self.nb_kind[c, d] = NB_NONE
        self.face_L = np.array(fL, dtype=np.int64)
        self.face_R = np.array(fR, dtype=np.int64)
        self.face_a = np.array(fa, dtype=np.int64)
        self.face_b = np.array(fb, dtype=np.int64)
        self.face_kind = np.array(fkind, dtype=np.int64)
        self.face_side = np.array(fside, dtype=np.int64)
        self.face_block = np.array(fblock, dtype=np.int64)
        self.face_shiftL = np.array(fshL, dtype=np.int64)
        self.face_Tw = np.array(fTw, dtype=np.float64)
        self.nf = self.face_L.size
        # orientation of each cell face: +1 if the cell is the face's L side
        self.cell_face_sign = np.where(self.face_L[self.cell_faces] == np.arange(nc)[:, None], 1, -1)

    def concat_nodes(self, X_list):
        return np.concatenate([X.transpose(1, 0, 2).reshape(-1, 2) for X in X_list], axis=0)


def shoelace(p1, p2, p3, p4):
    """Area of the quad p1 p2 p3 p4 (counter-clockwise positive):
    (1/2) (p3 - p1) x (p4 - p2)."""
    return 0.5 * ((p3[..., 0] - p1[..., 0]) * (p4[..., 1] - p2[..., 1])
                  - (p3[..., 1] - p1[..., 1]) * (p4[..., 0] - p2[..., 0]))


def vertex_centre(p1, p2, p3, p4):
    return 0.25 * ((p1 + p2) + (p3 + p4))


@dataclass
class Geometry:
    vol_old: np.ndarray     # (nc,) Omega^n
    vol_new: np.ndarray     # (nc,) Omega^{n+1}
    xc: np.ndarray          # (nc, 2) mid-time cell centres
    xc_new: np.ndarray      # (nc, 2) cell centres at t^{n+1}
    period: np.ndarray      # (nc, 2) period vector of the cell's row (mid-time)
    Sn: np.ndarray          # (nf, 2) S n at mid time (L -> R, or outward)
    S: np.ndarray           # (nf,)
    n: np.ndarray           # (nf, 2)
    xf: np.ndarray          # (nf, 2) mid-time face centre
    Uf: np.ndarray          # (nf, 2) face velocity
    SUn: np.ndarray         # (nf,) S U.n
    X_new: np.ndarray       # (nn, 2) nodes at t^{n+1}


def geometry(topo: Topology, X_old_list, X_new_list, dt: float) -> Geometry:
    Xo = topo.concat_nodes(X_old_list)
    Xn = topo.concat_nodes(X_new_list)
    Xm = 0.5 * (Xo + Xn)
    cn = topo.cell_nodes
    vol_old = shoelace(Xo[cn[:, 0]], Xo[cn[:, 1]], Xo[cn[:, 2]], Xo[cn[:, 3]])
    vol_new = shoelace(Xn[cn[:, 0]], Xn[cn[:, 1]], Xn[cn[:, 2]], Xn[cn[:, 3]])
    xc = vertex_centre(Xm[cn[:, 0]], Xm[cn[:, 1]], Xm[cn[:, 2]], Xm[cn[:, 3]])
    xc_new = vertex_centre(Xn[cn[:, 0]], Xn[cn[:, 1]], Xn[cn[:, 2]], Xn[cn[:, 3]])
    period = Xm[topo.cell_row_nodes[:, 1]] - Xm[topo.cell_row_nodes[:, 0]]
    a, b = topo.face_a, topo.face_b
    e = Xm[b] - Xm[a]
    Sn = np.stack([e[:, 1], -e[:, 0]], axis=-1)
    S = np.sqrt(e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1])
    n = Sn / S[:, None]
    xf = 0.5 * (Xm[a] + Xm[b])
    Uf = 0.5 * ((Xn[a] - Xo[a]) + (Xn[b] - Xo[b])) / dt
    SUn = Uf[:, 0] * Sn[:, 0] + Uf[:, 1] * Sn[:, 1]
    return Geometry(vol_old, vol_new, xc, xc_new, period, Sn, S, n, xf, Uf, SUn, Xn)
