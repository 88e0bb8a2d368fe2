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

Readings: a vertex is enriched when its minimum-image distance to the atom is
<= r_e + 1e-12 bohr.  The column phi_v^PU Psi_alpha is kept on element e only
when some image of alpha's atom lies at distance < r_c from the element box
(otherwise Psi_alpha vanishes identically there); a DOF left with no element
is dropped.  Within an element the enrichment columns are ordered by global
DOF, then by local vertex.

Pins: through the assembled matrices (tests/test_oracle_assembly.py) --
partition of unity, empty-lattice spectrum, PU reproduction, translation.
"""
from __future__ import annotations

import numpy as np

from .enrich import image_vectors


def box_distance(lo, hi, p):
    """Euclidean distance from point p to the axis-aligned box [lo, hi]."""
    d = np.maximum(np.maximum(lo - p, p - hi), 0.0)
    return float(np.sqrt((d * d).sum()))


class Mesh:
    def __init__(self, wl):
        self.wl = wl
        self.a = float(wl["a"])
        self.nel = int(wl["nel"])
        self.h = self.a / self.nel
        self.nelem = self.nel ** 3
        self.nfe_axis = 3 * self.nel
        self.n_fe = self.nfe_axis ** 3
        self.species = wl["species"]
        self.atoms = [(int(s), np.array(t, dtype=np.float64)) for s, t in wl["atoms"]]
        # enrichment functions alpha = (atom, orbital)
        self.alphas = []
        for ia, (s, tau) in enumerate(self.atoms):
            sp = self.species[s]
            for io, orb in enumerate(sp["orbitals"]):
                self.alphas.append(dict(atom=ia, orb=tuple(orb), rc=sp["r_c"], tau=tau))
        self._images = image_vectors(self.a)
        self._build()

    # -- geometry helpers --------------------------------------------------
    def elem_coords(self, e):
        n = self.nel
        return e % n, (e // n) % n, e // (n * n)

    def elem_box(self, e):
        ex, ey, ez = self.elem_coords(e)
        lo = np.array([ex, ey, ez], dtype=np.float64) * self.h
        return lo, lo + self.h

    def vertex_pos(self, v):
        n = self.nel
        return np.array([v % n, (v // n) % n, v // (n * n)], dtype=np.float64) * self.h

    def min_image_dist(self, x, tau):
        d = x - tau
        d = d - self.a * np.round(d / self.a)
        return float(np.sqrt((d * d).sum()))

    def atom_box_dist(self, ia, e):
        """Smallest distance from any image tau + R of atom ia to element e."""
        lo, hi = self.elem_box(e)
        P = self.atoms[ia][1] + self._images
        d = np.maximum(np.maximum(lo - P, P - hi), 0.0)
        return float(np.sqrt((d * d).sum(axis=1)).min())

    # -- numbering -----------------------------------------------------------
    def fe_dofs(self, e):
        ex, ey, ez = self.elem_coords(e)
        m = self.nfe_axis
        out = np.empty(64, dtype=np.int64)
        for c in range(4):
            for b in range(4):
                for a in range(4):
                    gx, gy, gz = (3 * ex + a) % m, (3 * ey + b) % m, (3 * ez + c) % m
                    out[a + 4 * b + 16 * c] = gx + m * (gy + m * gz)
        return out

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
        """Global DOFs of the element's columns: 64 FE, then enrichments."""
        enr = np.array([c[0] for c in self.elem_cols[e]], dtype=np.int64)
        return np.concatenate([self.fe_dofs(e), enr])

    def elem_alphas(self, e):
        """Enrichments that appear in the element's columns (sorted)."""
        return sorted({c[2] for c in self.elem_cols[e]})
