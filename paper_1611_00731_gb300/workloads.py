"""Workload definitions and seeded synthetic inputs for the PUFE hot path.

This module holds *data only*: the cells, atoms, enrichment orbitals and
quadrature options of the synthetic workloads, and seeded random generators
for the arrays that feed the hot path (the local potential at quadrature
points ``V_q``, coefficient blocks ``C`` and occupations ``f``).  It contains
none of the method's arithmetic, so that both the CUDA library and the
independent CPU oracle can consume the very same inputs.

Units are atomic (bohr, hartree).  Positions are Cartesian.

Orbital exponents ``zeta`` are stated explicitly.  They were chosen once, by
hand, with Slater's screening rules (Z_eff / n with the integer principal
quantum number) for the heavy atoms, and the hydrogenic values Z / n for the
hydrogen-like atom; nothing below derives them at run time.
"""
from __future__ import annotations

import numpy as np

# quadrature modes (same numbering as the C header)
QUAD_FIXED = 0   # p_near^3 Gauss on elements that meet an r_c ball, p_far^3 elsewhere
QUAD_PADAPT = 1  # per element, smallest p in [p_min, p_max] passing the tolerance test
QUAD_HADAPT = 2  # recursive octree subdivision (5^3 vs 8^3 test), depth-limited


def _orbs(*spec):
    """spec entries: (n, l, zeta); expands every l into m = -l..l."""
    out = []
    for n, l, zeta in spec:
        for m in range(-l, l + 1):
            out.append((n, l, m, zeta))
    return out


# --- species -------------------------------------------------------------
# Z and sigma define the local pseudopotential -Z erf(r/sigma)/r.
H_LIKE_1S = dict(name="H", Z=1.0, sigma=0.5, orbitals=_orbs((1, 0, 1.0)))
LI_LIKE_1S2S2P = dict(name="Li", Z=3.0, sigma=0.8,
                      orbitals=_orbs((1, 0, 2.70), (2, 0, 0.65), (2, 1, 0.65)))
H_LIKE_1S2S2P = dict(name="H", Z=1.0, sigma=0.5,
                     orbitals=_orbs((1, 0, 1.0), (2, 0, 0.5), (2, 1, 0.5)))
# Ce-like: 1s..4f (30 orbitals), Slater exponents for Z = 58
CE_LIKE = dict(name="Ce", Z=58.0, sigma=0.3,
               orbitals=_orbs((1, 0, 57.70), (2, 0, 26.925), (2, 1, 26.925),
                              (3, 0, 15.583333333333334), (3, 1, 15.583333333333334),
                              (3, 2, 12.283333333333333),
                              (4, 0, 7.5625), (4, 1, 7.5625), (4, 2, 4.7125),
                              (4, 3, 3.0)))
# Al-like: 1s..3p (9 orbitals), Slater exponents for Z = 13
AL_LIKE = dict(name="Al", Z=13.0, sigma=0.8,
               orbitals=_orbs((1, 0, 12.70), (2, 0, 4.425), (2, 1, 4.425),
                              (3, 0, 1.1666666666666667), (3, 1, 1.1666666666666667)))


def _species(base, r_c, r_e):
    d = dict(base)
    d["r_c"] = float(r_c)
    d["r_e"] = float(r_e)
    return d


def workload(name: str) -> dict:
    """Return the definition of a named workload.

    Keys: ``a`` (cubic lattice constant, bohr), ``nel`` (elements per axis),
    ``species`` (list of dicts with Z, sigma, orbitals [(n,l,m,zeta)], r_c,
    r_e), ``atoms`` (list of (species index, Cartesian position)),
    ``quad`` (dict: mode, p_far, p_near, p_min, p_max, tol, max_depth),
    ``nocc`` (occupied states used for density runs), ``nelec``.
    """
    if name == "c1_two_atom_4cube":
        # simple-cubic a=4 bohr, two atoms, 4^3 tricubic elements, fixed Gauss
        a = 4.0
        sp = [_species(H_LIKE_1S, 1.5, 1.5), _species(LI_LIKE_1S2S2P, 1.5, 1.5)]
        atoms = [(0, (0.0, 0.0, 0.0)), (1, (a / 2, a / 2, a / 2))]
        return dict(name=name, a=a, nel=4, species=sp, atoms=atoms,
                    quad=dict(mode=QUAD_FIXED, p_far=4, p_near=8, p_min=0,
                              p_max=0, tol=1e-6, max_depth=0),
                    nocc=2, nelec=4.0)
    if name.startswith("c2_rocksalt"):
        # LiH-like rocksalt conventional cube a=7.6, 8 atoms; nel from the name
        # ("c2_rocksalt_12cube" is the full size, smaller meshes for tests)
        nel = int(name.split("_")[2].replace("cube", "")) if name.count("_") >= 2 else 12
        a = 7.6
        sp = [_species(H_LIKE_1S2S2P, 2.0, 2.0), _species(LI_LIKE_1S2S2P, 2.0, 2.0)]
        fcc = [(0.0, 0.0, 0.0), (0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)]
        atoms = [(0, tuple(a * c for c in f)) for f in fcc]
        atoms += [(1, tuple(a * ((c + s) % 1.0) for c, s in zip(f, (0.5, 0.0, 0.0))))
                  for f in fcc]
        return dict(name=name, a=a, nel=nel, species=sp, atoms=atoms,
                    quad=dict(mode=QUAD_PADAPT, p_far=6, p_near=10, p_min=6,
                              p_max=10, tol=1e-6, max_depth=0),
                    nocc=8, nelec=16.0)
    if name.startswith("c5_rocksalt_2x2x2"):
        # 2x2x2 supercell of the LiH-like rocksalt cube (64 atoms, a = 15.2);
        # the name gives the elements per conventional cube ("..._16cube":
        # 32^3 elements in all, the equation-of-state configuration)
        per = int(name.split("_")[3].replace("cube", "")) if name.count("_") >= 3 else 16
        c = workload(f"c2_rocksalt_{per}cube")
        a0 = c["a"]
        atoms = [(s, tuple(t[d] + a0 * m[d] for d in range(3)))
                 for m in [(i, j, k) for k in range(2) for j in range(2) for i in range(2)]
                 for s, t in c["atoms"]]
        return dict(name=name, a=2 * a0, nel=2 * per, species=c["species"], atoms=atoms,
                    quad=c["quad"], nocc=64, nelec=128.0)
    if name.startswith("c3_cscl"):
        # CsCl-type a=5.8, Ce-like + Al-like, 16^3 elements, h-adaptive depth 1
        nel = int(name.split("_")[2].replace("cube", "")) if name.count("_") >= 2 else 16
        a = 5.8
        sp = [_species(CE_LIKE, 2.5, 0.37), _species(AL_LIKE, 2.5, 0.37)]
        atoms = [(0, (0.0, 0.0, 0.0)), (1, (a / 2, a / 2, a / 2))]
        return dict(name=name, a=a, nel=nel, species=sp, atoms=atoms,
                    quad=dict(mode=QUAD_HADAPT, p_far=4, p_near=8, p_min=5,
                              p_max=8, tol=1e-6, max_depth=1),
                    nocc=36, nelec=71.0)
    raise KeyError(name)


def small_two_atom(nel: int = 2, a: float = 4.0, quad_p: int = 4,
                   r_c: float = 1.5, r_e: float = 1.5) -> dict:
    """A cut-down C1-like cell for fast tests: same species, fewer elements."""
    sp = [_species(H_LIKE_1S, r_c, r_e), _species(LI_LIKE_1S2S2P, r_c, r_e)]
    atoms = [(0, (0.0, 0.0, 0.0)), (1, (a / 2, a / 2, a / 2))]
    return dict(name=f"two_atom_{nel}cube", a=a, nel=nel, species=sp, atoms=atoms,
                quad=dict(mode=QUAD_FIXED, p_far=quad_p, p_near=quad_p, p_min=0,
                          p_max=0, tol=1e-6, max_depth=0),
                nocc=2, nelec=4.0)


# The triclinic CeAl cell of Sec. 6.2 (eq. ceal-primitive): lattice vectors
# and atom positions in lattice coordinates as printed, in units of a.
CEAL_A = 5.75
CEAL_LATTICE = ((1.00, 0.02, -0.04), (0.01, 0.98, 0.03), (0.03, -0.06, 1.09))
CEAL_TAU_LATTICE = ((0.01, 0.02, 0.03), (0.51, 0.47, 0.55))


def ceal_like(nel: int = 2, quad_p: int = 6, r_c: float = 2.5, r_e: float = 2.0,
              full_orbitals: bool = False) -> dict:
    """The CeAl geometry with the synthetic Ce-like and Al-like species (a
    reduced orbital set unless `full_orbitals`): a general cell given by its
    lattice (rows a_1, a_2, a_3, bohr), nel^3 elements in lattice
    coordinates, a fixed p^3 rule on every element."""
    L = [[CEAL_A * c for c in row] for row in CEAL_LATTICE]
    ce, al = dict(CE_LIKE), dict(AL_LIKE)
    if not full_orbitals:   # 4s 4p (Ce-like), 3s 3p (Al-like)
        ce["orbitals"] = [o for o in CE_LIKE["orbitals"] if o[0] == 4 and o[1] <= 1]
        al["orbitals"] = [o for o in AL_LIKE["orbitals"] if o[0] == 3]
    sp = [_species(ce, r_c, r_e), _species(al, r_c, r_e)]
    atoms = [(i, tuple(sum(s[k] * L[k][d] for k in range(3)) for d in range(3)))
             for i, s in enumerate(CEAL_TAU_LATTICE)]
    return dict(name=f"ceal_like_{nel}cube", lattice=L, a=None, nel=nel, species=sp,
                atoms=atoms,
                quad=dict(mode=QUAD_FIXED, p_far=quad_p, p_near=quad_p, p_min=0, p_max=0,
                          tol=1e-6, max_depth=0),
                nocc=4, nelec=8.0)


def sheared_empty(nel: int = 3, p: int = 4) -> dict:
    """No atoms, no enrichment, the CeAl lattice: the tricubic space on a
    general cell (its empty-lattice spectrum is |G|^2 / 2 on the reciprocal
    lattice)."""
    L = [[CEAL_A * c for c in row] for row in CEAL_LATTICE]
    return dict(name=f"sheared_empty_{nel}cube", lattice=L, a=None, nel=nel, species=[],
                atoms=[],
                quad=dict(mode=QUAD_FIXED, p_far=p, p_near=p, p_min=0, p_max=0, tol=1e-6,
                          max_depth=0),
                nocc=1, nelec=2.0)


def empty_lattice(nel: int = 2, a: float = 4.0, p: int = 4) -> dict:
    """No atoms, no enrichment: the classical tricubic space on its own."""
    return dict(name=f"empty_{nel}cube", a=a, nel=nel, species=[], atoms=[],
                quad=dict(mode=QUAD_FIXED, p_far=p, p_near=p, p_min=0, p_max=0,
                          tol=1e-6, max_depth=0),
                nocc=1, nelec=2.0)


# --- seeded arrays -----------------------------------------------------------

def random_potential(nq: int, seed: int = 0) -> np.ndarray:
    """V_q ~ U(-1, 0), float64, one value per quadrature point."""
    return np.random.default_rng(seed).uniform(-1.0, 0.0, size=nq)


def random_coefficients(n: int, nocc: int, seed: int = 0) -> np.ndarray:
    """C ~ N(0, 1), float64, shape (n, nocc), column-major friendly copy."""
    return np.random.default_rng(seed).standard_normal((n, nocc))


def random_occupations(nocc: int, seed: int = 0) -> np.ndarray:
    """f ~ U(0, 2), float64 (occupations lie in [0, 2])."""
    return np.random.default_rng(seed + 1).uniform(0.0, 2.0, size=nocc)


def random_symmetric_values(nnz: int, seed: int = 0) -> np.ndarray:
    """Values ~ N(0,1) for a sparse matrix pattern (caller symmetrises)."""
    return np.random.default_rng(seed + 2).standard_normal(nnz)
