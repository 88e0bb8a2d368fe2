"""Periodic mesh, DOF numbering and per-element PUFE basis lists (oracle).

Implements the discrete basis of Sec. 4 (eq. pufebasis): the classical FE
functions phi_i on every node of the periodic tricubic grid, plus
phi_j^PU Psi_alpha for every enrichment alpha and every PU vertex j within
the support radius r_e of alpha's atom (Sec. 5.1, "all nodes that lie within
the support radius r_e of the atom are enriched").

Numbering (shared convention with the library's interface, written again
here from its definition):
* elements e = ex + nel (ey + nel ez), box [ex h, (ex+1) h] x ...;
* FE nodes on the (3 nel)^3 periodic grid, index gx + 3nel (gy + 3nel gz);
  element-local node (a, b, c) in {0..3}^3 -> g = 3 e + (a, b, c) mod 3 nel;
* PU vertices on the nel^3 periodic grid, element-local vertex
  (a, b, c) in {0,1}^3 -> (e + (a, b, c)) mod nel;
* enrichments alpha in (atom, orbital) order; enrichment DOFs follow the FE
  DOFs, ordered by (atom, orbital, enriched vertex index).

Classical FE space: the tricubic Lagrange space (64 nodes per element) or
the cubic serendipity space (32 nodes per element, the paper's choice in its
PUFE runs, Sec. 6): the workload key "fe" = "lagrange64" (default) or
"serendipity32".  Serendipity DOFs are the grid nodes with at most one
coordinate off the vertex planes (vertices and inner edge nodes), numbered
compactly in grid order; an element's FE columns follow fe.SERENDIPITY_LOCAL.

Readings: a vertex is enriched when its minimum-image distance to the atom is
<= r_e + 1e-12 bohr.  The column phi_v^PU Psi_alpha is kept on element e only
when some image of alpha's atom lies at distance < r_c from the element box
(otherwise Psi_alpha vanishes identically there); a DOF left with no element
is dropped.  Within an element the enrichment columns are ordered by global
DOF, then by local vertex.

General (triclinic) cells, the paper's CeAl geometry (Sec. 6.2, eq.
ceal-primitive): a workload with a "lattice" entry (rows a_1, a_2, a_3)
divides the cell into nel^3 parallelepipeds in lattice coordinates,
s_d in [e_d / nel, (e_d + 1) / nel]; an element maps the reference cube by
x = x_0 + J (xi + 1), J = [a_1, a_2, a_3] / (2 nel) (columns), so the FE and
PU functions keep their reference form and physical gradients are
J^-T grad_xi.  Minimum-image distances search the neighbouring images of the
lattice-coordinate rounding; the distance from an atom image to an element
is the exact minimum over the parallelepiped (a box-constrained least-squares
problem solved on each of its 27 faces).

Pins: through the assembled matrices (tests/test_oracle_assembly.py) --
partition of unity, empty-lattice spectrum, PU reproduction, translation;
for general cells (tests/test_oracle_triclinic.py) the partition of unity on
mapped elements, the empty-lattice spectrum |G|^2/2 of a sheared cell on the
reciprocal lattice, and the cubic cell written as a lattice.
"""
from __future__ import annotations

import numpy as np

from .enrich import image_vectors
from .fe import SERENDIPITY_LOCAL, serendipity32, tricubic


def parallelepiped_dist(x0, M, P):
    """Distances from points P (m, 3) to {x0 + M t : t in [0, 1]^3}.

    The squared distance is a convex quadratic in t; its minimiser over the
    box lies in the relative interior of one of the box's 27 faces (each
    coordinate free, at 0 or at 1).  On every face the free coordinates solve
    a small least-squares problem; a face whose minimiser stays inside the
    box gives a point of the parallelepiped, and the smallest such distance
    is the exact one (the true minimiser is among them).
    """
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    best = np.full(len(P), np.inf)
    for code in range(27):
        st = [(code // 3 ** d) % 3 for d in range(3)]   # 0 free, 1 at 0, 2 at 1
        t = np.zeros((len(P), 3))
        fixed = np.array([0.0 if c == 1 else 1.0 for c in st])
        free = [d for d in range(3) if st[d] == 0]
        base = x0 + M @ np.where(np.array(st) == 0, 0.0, fixed)
        r = P - base
        if free:
            Mf = M[:, free]
            sol = np.linalg.lstsq(Mf, r.T, rcond=None)[0].T
            ok = ((sol >= 0.0) & (sol <= 1.0)).all(axis=1)
            q = base + sol @ Mf.T
        else:
            ok = np.ones(len(P), dtype=bool)
            q = np.broadcast_to(base, P.shape)
        d = np.sqrt(((P - q) ** 2).sum(axis=1))
        best = np.where(ok, np.minimum(best, d), best)
        del t
    return best


def box_distance(lo, hi, p):
    """Euclidean distance from point p to the axis-aligned box [lo, hi]."""
    d = np.maximum(np.maximum(lo - p, p - hi), 0.0)
    return float(np.sqrt((d * d).sum()))


class Mesh:
    def __init__(self, wl):
        self.wl = wl
        self.nel = int(wl["nel"])
        self.general = "lattice" in wl
        if self.general:
            self.L = np.array(wl["lattice"], dtype=np.float64).reshape(3, 3)   # rows a_d
            self.a = None            # no cubic edge: cubic-only code paths fail loudly
            self.h = None
            self.J = self.L.T / (2.0 * self.nel)                               # columns a_d / 2nel
            self.Jinv = np.linalg.inv(self.J)
            self.detJ = abs(float(np.linalg.det(self.J)))
            self.lattice = self.L
        else:
            self.a = float(wl["a"])
            self.h = self.a / self.nel
            self.lattice = self.a
        self.nelem = self.nel ** 3
        self.nfe_axis = 3 * self.nel
        # classical FE space: "lagrange64" (tricubic) or "serendipity32"
        self.fe = wl.get("fe", "lagrange64")
        m = self.nfe_axis
        if self.fe == "lagrange64":
            self.fe_local = np.arange(64)
            self.n_fe = m ** 3
            self._gmap = np.arange(m ** 3)
        elif self.fe == "serendipity32":
            # nodes of the periodic tricubic grid with at most one coordinate
            # off the vertex planes, numbered compactly in grid order
            self.fe_local = SERENDIPITY_LOCAL
            g = np.arange(m ** 3)
            gx, gy, gz = g % m, (g // m) % m, g // (m * m)
            keep = (gx % 3 != 0).astype(int) + (gy % 3 != 0) + (gz % 3 != 0) <= 1
            self._gmap = np.full(m ** 3, -1, dtype=np.int64)
            self._gmap[keep] = np.arange(int(keep.sum()))
            self.n_fe = int(keep.sum())
        else:
            raise ValueError(f"unknown FE space {self.fe!r}")
        self.nfe_e = len(self.fe_local)
        self.species = wl["species"]
        self.atoms = [(int(s), np.array(t, dtype=np.float64)) for s, t in wl["atoms"]]
        # enrichment functions alpha = (atom, orbital)
        self.alphas = []
        for ia, (s, tau) in enumerate(self.atoms):
            sp = self.species[s]
            for io, orb in enumerate(sp["orbitals"]):
                self.alphas.append(dict(atom=ia, orb=tuple(orb), rc=sp["r_c"], tau=tau))
        self._images = image_vectors(self.lattice)
        self._build()

    # -- geometry helpers --------------------------------------------------
    def elem_coords(self, e):
        n = self.nel
        return e % n, (e // n) % n, e // (n * n)

    def elem_box(self, e):
        ex, ey, ez = self.elem_coords(e)
        lo = np.array([ex, ey, ez], dtype=np.float64) * self.h
        return lo, lo + self.h

    def elem_origin(self, e):
        """Corner x_0 of element e (the image of xi = (-1, -1, -1))."""
        if not self.general:
            return self.elem_box(e)[0]
        return self.L.T @ (np.array(self.elem_coords(e), dtype=np.float64) / self.nel)

    def to_reference(self, e, pts):
        """Reference coordinates xi in [-1, 1]^3 of physical points of element e."""
        if not self.general:
            lo, _ = self.elem_box(e)
            return 2.0 * (pts - lo) / self.h - 1.0
        return (np.asarray(pts) - self.elem_origin(e)) @ self.Jinv.T - 1.0

    def grad_to_physical(self, dN):
        """Physical gradients (3, Q, k) from reference gradients (3, Q, k)."""
        if not self.general:
            return dN * (2.0 / self.h)
        return np.einsum("kd,kqj->dqj", self.Jinv, dN)

    def vertex_pos(self, v):
        n = self.nel
        g = np.array([v % n, (v // n) % n, v // (n * n)], dtype=np.float64)
        if not self.general:
            return g * self.h
        return self.L.T @ (g / n)

    def min_image_dist(self, x, tau):
        d = x - tau
        if not self.general:
            d = d - self.a * np.round(d / self.a)
            return float(np.sqrt((d * d).sum()))
        # round in lattice coordinates, then search the neighbouring images
        s = np.linalg.solve(self.L.T, d)
        d0 = self.L.T @ (s - np.round(s))
        off = np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")).reshape(3, -1).T
        dd = d0 + off @ self.L
        return float(np.sqrt((dd * dd).sum(axis=1)).min())

    def atom_box_dist(self, ia, e):
        """Smallest distance from any image tau + R of atom ia to element e."""
        if not self.general:
            lo, hi = self.elem_box(e)
            P = self.atoms[ia][1] + self._images
            d = np.maximum(np.maximum(lo - P, P - hi), 0.0)
            return float(np.sqrt((d * d).sum(axis=1)).min())
        return float(parallelepiped_dist(self.elem_origin(e), 2.0 * self.J,
                                         self.atoms[ia][1] + self._images).min())

    # -- numbering -----------------------------------------------------------
    def fe_dofs(self, e):
        """Global FE DOFs of the element's FE columns (local nodes fe_local)."""
        ex, ey, ez = self.elem_coords(e)
        m = self.nfe_axis
        out = np.empty(len(self.fe_local), dtype=np.int64)
        for j, loc in enumerate(self.fe_local):
            a, b, c = loc & 3, (loc >> 2) & 3, loc >> 4
            gx, gy, gz = (3 * ex + a) % m, (3 * ey + b) % m, (3 * ez + c) % m
            out[j] = self._gmap[gx + m * (gy + m * gz)]
        return out

    def fe_functions(self, xi):
        """The element's FE functions and reference gradients at xi (Q, 3)."""
        return tricubic(xi) if self.fe == "lagrange64" else serendipity32(xi)

    def elem_vertices(self, e):
        ex, ey, ez = self.elem_coords(e)
        n = self.nel
        out = []
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    out.append(((ex + a) % n) + n * (((ey + b) % n) + n * ((ez + c) % n)))
        return out

    def _build(self):
        nv = self.nel ** 3
        # element/atom proximity: atom image within r_c of the element box
        self.near = np.zeros((self.nelem, len(self.atoms)), dtype=bool)
        for e in range(self.nelem):
            for ia, (s, _) in enumerate(self.atoms):
                self.near[e, ia] = self.atom_box_dist(ia, e) < self.species[s]["r_c"]
        # enriched vertices per atom
        enr_verts = []
        for ia, (s, tau) in enumerate(self.atoms):
            re = self.species[s]["r_e"]
            enr_verts.append([v for v in range(nv)
                              if self.min_image_dist(self.vertex_pos(v), tau) <= re + 1e-12])
        # candidate DOFs (atom, orbital, vertex) and the elements that keep them
        vert_elems = [[] for _ in range(nv)]
        for e in range(self.nelem):
            for lv, v in enumerate(self.elem_vertices(e)):
                vert_elems[v].append((e, lv))
        dof = self.n_fe
        self.enr_dof_info = []      # (alpha, vertex)
        cols = [[] for _ in range(self.nelem)]  # (dof, lv, alpha)
        for k, al in enumerate(self.alphas):
            ia = al["atom"]
            for v in enr_verts[ia]:
                keep = [(e, lv) for (e, lv) in vert_elems[v] if self.near[e, ia]]
                if not keep:
                    continue
                for (e, lv) in keep:
                    cols[e].append((dof, lv, k))
                self.enr_dof_info.append((k, v))
                dof += 1
        self.n_dof = dof
        self.n_enr = dof - self.n_fe
        self.elem_cols = [sorted(c) for c in cols]

    # -- per-element basis description ------------------------------------
    def elem_dofs(self, e):
        """Global DOFs of the element's columns: the FE ones (64 or 32), then
        the enrichments."""
        enr = np.array([c[0] for c in self.elem_cols[e]], dtype=np.int64)
        return np.concatenate([self.fe_dofs(e), enr])

    def elem_alphas(self, e):
        """Enrichments that appear in the element's columns (sorted)."""
        return sorted({c[2] for c in self.elem_cols[e]})
