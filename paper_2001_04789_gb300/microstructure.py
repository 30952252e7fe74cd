"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds INPUT fields (moduli, eigenstrain, boundary data) for
the elasticity problem of Section 2.1, Eq. (1a)-(1d).  It contains none of the
solver's arithmetic (no finite differences, no smoothing, no transfers) and is
the one module that both the CUDA path's callers and the CPU oracle import.

Field conventions shared by every consumer:

* A grid has ``n = (nx, ny, nz)`` nodes.  In a non-periodic direction the
  nodes include both boundary planes and ``h = (hi - lo) / (n - 1)``; in a
  periodic direction ``n`` counts the unique nodes and ``h = (hi - lo) / n``.
* Scalar fields are numpy arrays of shape ``(nz, ny, nx)`` (x fastest), so a
  node's flat index is ``i + nx * (j + ny * k)``.
* Vector fields are ``(3, nz, ny, nx)``; symmetric second-order tensors
  (eigenstrain, mean strain) are 6 tensor components in the order
  11, 22, 33, 23, 31, 12 (tensor shears, not doubled).
* Isotropic moduli are ``(2, nz, ny, nx)`` = (lambda, mu).  General moduli are
  the 21 upper-triangle entries of the 6x6 Voigt matrix (Section 4.3, the
  Voigt form of the cubic tensor, Voigt order 11, 22, 33, 23, 31, 12), stored
  row by row: C11 C12 C13 C14 C15 C16 C22 C23 ... C66, shape
  ``(21, nz, ny, nx)``.
* Boundary faces are numbered 0..5 = -x, +x, -y, +y, -z, +z; each face carries
  one (type, value) pair per displacement component.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional

import numpy as np

# boundary-row types (Section 2.1, Eq. 1b-1d)
DIRICHLET = 1
TRACTION = 2
NEUMANN = 3

MODULI_ISO = 2
MODULI_GEN21 = 21

_VOIGT = ((0, 5, 4), (5, 1, 3), (4, 3, 2))


@dataclasses.dataclass
class Problem:
    """One elasticity problem on a single uniform node grid."""
    n: tuple                      # (nx, ny, nz)
    periodic: tuple = (False, False, False)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    moduli_kind: int = MODULI_ISO
    moduli: Optional[np.ndarray] = None          # (2|21, nz, ny, nx)
    eigenstrain: Optional[np.ndarray] = None     # (6, nz, ny, nx)
    body_force: Optional[np.ndarray] = None      # (3, nz, ny, nx)
    mean_strain: Optional[np.ndarray] = None     # (6,), fully periodic grids only
    # bc[face][comp] = (type, uniform value)
    bc: list = dataclasses.field(default_factory=list)
    dirichlet_values: Optional[np.ndarray] = None  # (3, nz, ny, nx) overrides face values
    # face_values[f] = (3, nz, ny, nx): per-node boundary data of face f (its
    # Dirichlet value, traction or normal derivative), read on that face only
    face_values: Optional[dict] = None
    name: str = ""

    @property
    def h(self):
        out = []
        for d in range(3):
            span = self.hi[d] - self.lo[d]
            out.append(span / self.n[d] if self.periodic[d] else span / (self.n[d] - 1))
        return tuple(out)

    def coords(self):
        """Node coordinates X, Y, Z, each (nz, ny, nx)."""
        h = self.h
        ax = [self.lo[d] + h[d] * np.arange(self.n[d]) for d in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return X, Y, Z


def lame(E, nu):
    E = np.asarray(E, dtype=np.float64)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def tanh_profile(s, w):
    """Diffuse indicator: 1 well inside (s < 0), 0 well outside, width w."""
    return 0.5 * (1.0 - np.tanh(2.0 * s / w))


def all_faces(kind, value=0.0):
    return [[(kind, value)] * 3 for _ in range(6)]


# --------------------------------------------------------------------------
# moduli tensors used only to build inputs (Section 4.3)
# --------------------------------------------------------------------------

def cubic_voigt(c11, c12, c44):
    V = np.zeros((6, 6))
    V[:3, :3] = c12
    for a in range(3):
        V[a, a] = c11
        V[a + 3, a + 3] = c44
    return V


def voigt_to_tensor(V):
    T = np.zeros((3, 3, 3, 3))
    for i, j, k, l in itertools.product(range(3), repeat=4):
        T[i, j, k, l] = V[_VOIGT[i][j], _VOIGT[k][l]]
    return T


def tensor_to_upper21(T):
    V = np.zeros((6, 6))
    for i, j, k, l in itertools.product(range(3), repeat=4):
        V[_VOIGT[i][j], _VOIGT[k][l]] = T[i, j, k, l]
    return np.array([V[a, b] for a in range(6) for b in range(a, 6)])


def rotate_tensor(T, R):
    """Rotated modulus tensor of Section 4.3: C'_pqst = R_pi R_qj C_ijkl R_sk R_tl."""
    return np.einsum("pi,qj,sk,tl,ijkl->pqst", R, R, R, R, T)


def random_rotation(rng):
    """Uniform random rotation from a uniform unit quaternion (Shoemake, 1992)."""
    u1, u2, u3 = rng.random(3)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.array([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def iso_to_upper21(lam, mu):
    """Isotropic (lambda, mu) fields written as the 21 Voigt components."""
    lam = np.asarray(lam)
    out = np.zeros((21,) + lam.shape)
    k = 0
    for a in range(6):
        for b in range(a, 6):
            if a < 3 and b < 3:
                out[k] = lam + (2.0 * mu if a == b else 0.0)
            elif a == b:
                out[k] = mu
            k += 1
    return out


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def eshelby_sphere(n=33, radius=0.2, width_cells=3.0, E_matrix=1.0, E_incl=2.0, nu=0.3,
                   eps_star=1e-3, centre=(0.5, 0.5, 0.5), box=None, width=None):
    """Spherical Eshelby inhomogeneity on the unit cube (Section 4.1 analogue):
    tanh-blended isotropic moduli, eigenstrain eps_star * phi * I, u = 0 on all faces.
    ``box = (n3, lo3, hi3)`` evaluates the same fields on a sub-box (AMR levels); the
    profile width is then ``width`` (physical), else width_cells node spacings."""
    if box is None:
        p = Problem(n=(n, n, n), name=f"eshelby_sphere_{n}")
    else:
        p = Problem(n=tuple(box[0]), lo=tuple(box[1]), hi=tuple(box[2]), name="eshelby_sphere_box")
    X, Y, Z = p.coords()
    w = width if width is not None else width_cells * p.h[0]
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    phi = tanh_profile(r - radius, w)
    lam, mu = lame(E_matrix * (1.0 - phi) + E_incl * phi, nu)
    p.moduli_kind = MODULI_ISO
    p.moduli = np.stack([lam, mu])
    eps = np.zeros((6,) + phi.shape)
    eps[0] = eps[1] = eps[2] = eps_star * phi
    p.eigenstrain = eps
    p.bc = all_faces(DIRICHLET, 0.0)
    return p


def eshelby_ellipsoid(n=129, half_width=4.0, axes=(1.0, 0.75, 0.5), E=210.0, nu=0.3, eps_star=1e-3,
                      width=0.1):
    """Ellipsoidal Eshelby inclusion of Section 4.1: an 8 x 8 x 8 box (half width 4) with
    u = 0 on all faces, homogeneous moduli E = 210, nu = 0.3, and the dilatational
    eigenstrain eps_star I inside the ellipsoid with semi-axes (1, 0.75, 0.5), blended by
    the error-function profile of width 0.1.  The indicator as printed is garbled; the
    reading taken: eta = 1 inside, A = diag(a_i^-2) and the argument
    (x^T A x - 1) / (2 width |A x|), so that eta = 1/2 on the sharp ellipsoid."""
    from scipy.special import erf
    p = Problem(n=(n, n, n), lo=(-half_width,) * 3, hi=(half_width,) * 3, name=f"eshelby_ellipsoid_{n}")
    X, Y, Z = p.coords()
    a = np.asarray(axes, dtype=float)
    q = (X / a[0]) ** 2 + (Y / a[1]) ** 2 + (Z / a[2]) ** 2
    ax = np.sqrt((X / a[0] ** 2) ** 2 + (Y / a[1] ** 2) ** 2 + (Z / a[2] ** 2) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        arg = np.where(ax > 0, (q - 1.0) / (2.0 * width * np.maximum(ax, 1e-300)), -np.inf)
    eta = 0.5 * (1.0 - erf(arg))
    lam, mu = lame(np.full(X.shape, E), nu)
    p.moduli_kind = MODULI_ISO
    p.moduli = np.stack([lam, mu])
    eps = np.zeros((6,) + X.shape)
    eps[0] = eps[1] = eps[2] = eps_star * eta
    p.eigenstrain = eps
    p.bc = all_faces(DIRICHLET, 0.0)
    return p


def polycrystal(n=257, grains=20, seed=0, c11=1.68, c12=1.21, c44=0.75, width_cells=4.0,
                strain=1e-3, box=None, width=None, clamp=False):
    """Voronoi polycrystal (Section 4.3 analogue): rotated cubic grains blended by the
    linear mixture rule over tanh grain-boundary profiles; u_x = -+strain/2 on the x
    faces, zero shear traction there, traction-free y and z faces (with ``clamp`` the
    x faces hold u_y = u_z = 0 too, leaving no rigid modes).  ``box = (n3, lo3, hi3)``
    evaluates the same grains on a sub-box (AMR levels), profile width ``width``."""
    rng = np.random.default_rng(seed)
    if box is None:
        p = Problem(n=(n, n, n), name=f"polycrystal_{n}_{grains}g")
    else:
        p = Problem(n=tuple(box[0]), lo=tuple(box[1]), hi=tuple(box[2]), name="polycrystal_box")
    centres = rng.random((grains, 3))
    rots = [random_rotation(rng) for _ in range(grains)]
    base = voigt_to_tensor(cubic_voigt(c11, c12, c44))
    grain_c = np.stack([tensor_to_upper21(rotate_tensor(base, R)) for R in rots])
    w = width if width is not None else width_cells * p.h[0]
    X, Y, Z = p.coords()
    shape = X.shape
    # distance-squared to every centre, one z-slab at a time to bound memory
    C = np.zeros((21,) + shape)
    for k0 in range(0, shape[0], 16):
        sl = slice(k0, min(shape[0], k0 + 16))
        pts = np.stack([X[sl], Y[sl], Z[sl]], axis=-1)
        d2 = np.stack([np.sum((pts - c) ** 2, axis=-1) for c in centres])
        nearest = np.argmin(d2, axis=0)
        cn = centres[nearest]
        d2n = np.min(d2, axis=0)
        s = np.empty_like(d2)
        for g in range(grains):
            sep = np.linalg.norm(centres[g] - cn, axis=-1)
            with np.errstate(divide="ignore", invalid="ignore"):
                s[g] = np.where(sep > 0, (d2[g] - d2n) / (2.0 * np.where(sep > 0, sep, 1.0)), np.inf)
        s_other = np.where(np.arange(grains)[:, None, None, None] == nearest[None], np.inf, s)
        s_near = -np.min(s_other, axis=0)
        s = np.where(np.arange(grains)[:, None, None, None] == nearest[None], s_near[None], s)
        eta = tanh_profile(s, w)
        tot = eta.sum(axis=0)
        C[:, sl] = np.einsum("gc,g...->c...", grain_c, eta) / tot
    p.moduli_kind = MODULI_GEN21
    p.moduli = C
    bc = all_faces(TRACTION, 0.0)
    lat = DIRICHLET if clamp else TRACTION
    bc[0] = [(DIRICHLET, -0.5 * strain), (lat, 0.0), (lat, 0.0)]
    bc[1] = [(DIRICHLET, +0.5 * strain), (lat, 0.0), (lat, 0.0)]
    p.bc = bc
    return p


def crack_indicator(X, Y, Z, radius=0.25, width=3.0 / 256):
    """Diffuse penny-crack indicator: 1 on the disc (radius, plane z = 0.5), decaying
    as 1 - tanh^2(d / width) with the distance d to the disc."""
    rho = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
    d = np.sqrt(np.maximum(rho - radius, 0.0) ** 2 + (Z - 0.5) ** 2)
    return 1.0 - np.tanh(d / width) ** 2


def penny_crack(n=65, radius=0.25, width=3.0 / 256, E=1.0, nu=0.3, soft=1e-2, strain=1e-3,
                clamp_lateral=False, box=None):
    """Penny-shaped diffuse crack (Section 4.2 analogue) in the plane z = 0.5:
    E is reduced to soft * E inside the crack profile, soft capped at 1 % of the
    matrix modulus as Section 4.2 does for numerical stability; u_z = -+strain/2 on
    the z faces (u_x = u_y = 0 there too when clamp_lateral, else zero shear
    traction), traction-free x and y faces.  ``box = (n3, lo3, hi3)`` evaluates the
    same fields on a sub-box of the unit cube."""
    if box is None:
        p = Problem(n=(n, n, n), name=f"penny_crack_{n}")
    else:
        p = Problem(n=tuple(box[0]), lo=tuple(box[1]), hi=tuple(box[2]), name="penny_crack_box")
    X, Y, Z = p.coords()
    phi = crack_indicator(X, Y, Z, radius, width)
    lam, mu = lame(E * ((1.0 - phi) + soft * phi), nu)
    p.moduli_kind = MODULI_ISO
    p.moduli = np.stack([lam, mu])
    bc = all_faces(TRACTION, 0.0)
    lat = DIRICHLET if clamp_lateral else TRACTION
    bc[4] = [(lat, 0.0), (lat, 0.0), (DIRICHLET, -0.5 * strain)]
    bc[5] = [(lat, 0.0), (lat, 0.0), (DIRICHLET, +0.5 * strain)]
    p.bc = bc
    return p


# --------------------------------------------------------------------------
# block-structured AMR layouts (Section 3.1: levels of refinement by 2, tagged
# where the indicator varies fast; one box per level, properly nested)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class AmrLevel:
    """One AMR level.  Node indices are global in the level's own index space
    (node i of level l sits at lo + i * h_l).  The level's grid is its valid box plus
    one ghost layer on every coarse/fine face; ``problem`` lives on that grid, with
    Dirichlet rows on the ghost faces (their values come from the coarser level)."""
    level: int
    h: float
    valid_lo: tuple
    valid_hi: tuple
    grid_lo: tuple
    ghost: tuple            # 6 flags: face has a coarse/fine ghost layer
    problem: Problem


def _tag_box(phi, h, thresh, block, parent_lo, parent_hi, n_level):
    """Box (in the next finer level's global node indices) covering every aligned
    block of `block` fine cells that contains a tagged coarse cell, i.e. a coarse
    cell with a corner node where |grad phi| h > thresh; clipped to stay one coarse
    cell inside the parent box except on the physical boundary."""
    g = np.gradient(phi, h)
    tag = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2) * h > thresh   # (z, y, x)
    if not tag.any():
        return None
    idx = np.argwhere(tag)
    lo_c = idx.min(axis=0)[::-1] + np.array(parent_lo)     # coarse global (x, y, z)
    hi_c = idx.max(axis=0)[::-1] + np.array(parent_lo)
    lo_f = 2 * np.maximum(lo_c - 1, 0)
    hi_f = 2 * (hi_c + 1)
    lo_f = (lo_f // block) * block
    hi_f = -(-hi_f // block) * block
    nmax = 2 * (n_level - 1)
    lo_f = np.maximum(lo_f, 0)
    hi_f = np.minimum(hi_f, nmax)
    for d in range(3):
        if parent_lo[d] > 0:
            lo_f[d] = max(lo_f[d], 2 * (parent_lo[d] + 1))
        if parent_hi[d] < n_level - 1:
            hi_f[d] = min(hi_f[d], 2 * (parent_hi[d] - 1))
    if np.any(hi_f - lo_f < 4):
        return None
    return tuple(int(v) for v in lo_f), tuple(int(v) for v in hi_f)


def amr_layout(make_box_problem, base_n, nlevels, indicator, thresh=0.1, block=32, ghost_layers=1):
    """Build the AMR levels of a unit-cube workload.  ``make_box_problem(n3, lo3, hi3)``
    returns the workload's Problem on a node box; ``indicator(X, Y, Z)`` is the field
    whose gradient tags cells for refinement.  Fine grids carry ``ghost_layers`` node
    layers beyond each coarse/fine face (1 for reading R1, 2 for reading R2)."""
    base = make_box_problem((base_n,) * 3, (0.0,) * 3, (1.0,) * 3)
    levels = [AmrLevel(0, 1.0 / (base_n - 1), (0, 0, 0), (base_n - 1,) * 3, (0, 0, 0),
                       (False,) * 6, base)]
    n_level = base_n
    for l in range(1, nlevels):
        par = levels[-1]
        X, Y, Z = par.problem.coords()
        gl, gh = par.grid_lo, tuple(par.grid_lo[d] + par.problem.n[d] - 1 for d in range(3))
        phi = indicator(X, Y, Z)
        box = _tag_box(phi, par.h, thresh, block, par.valid_lo, par.valid_hi, n_level)
        if box is None:
            break
        n_level = 2 * (n_level - 1) + 1
        h = par.h / 2.0
        vlo, vhi = box
        ghost = []
        for f in range(6):
            d = f // 2
            ghost.append(vlo[d] > 0 if f % 2 == 0 else vhi[d] < n_level - 1)
        glo = tuple(vlo[d] - (ghost_layers if ghost[2 * d] else 0) for d in range(3))
        ghi = tuple(vhi[d] + (ghost_layers if ghost[2 * d + 1] else 0) for d in range(3))
        n3 = tuple(ghi[d] - glo[d] + 1 for d in range(3))
        lo3 = tuple(glo[d] * h for d in range(3))
        hi3 = tuple(ghi[d] * h for d in range(3))
        prob = make_box_problem(n3, lo3, hi3)
        prob.bc = [list(prob.bc[f]) if not ghost[f] else [(DIRICHLET, 0.0)] * 3 for f in range(6)]
        levels.append(AmrLevel(l, h, vlo, vhi, glo, tuple(ghost), prob))
    return levels


def amr_penny_crack(base_n=65, nlevels=3, block=32, thresh=0.1, width=3.0 / 256, ghost_layers=1, **kw):
    """Penny crack on a 3-level layout, ratio 2 (laterally clamped z grips)."""
    mk = lambda n3, lo3, hi3: penny_crack(width=width, clamp_lateral=True, box=(n3, lo3, hi3), **kw)
    ind = lambda X, Y, Z: crack_indicator(X, Y, Z, width=width)
    return amr_layout(mk, base_n, nlevels, ind, thresh, block, ghost_layers)


def amr_request_layout(kind, base_n, nlevels=2, block=32, seed=0, ghost_layers=1):
    """Two-level (by default) AMR layouts of the served microstructures: an Eshelby
    sphere, a laterally clamped penny crack and a clamped polycrystal, each refined where
    its indicator varies fast; profile widths fixed in physical units (3 or 4 spacings of
    the finest level)."""
    hf = 1.0 / ((base_n - 1) * 2 ** (nlevels - 1))
    if kind == "sphere":
        w = 3.0 * hf
        mk = lambda n3, lo3, hi3: eshelby_sphere(box=(n3, lo3, hi3), width=w)
        r = lambda X, Y, Z: np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
        ind = lambda X, Y, Z: tanh_profile(r(X, Y, Z) - 0.2, w)
        return amr_layout(mk, base_n, nlevels, ind, 0.1, block, ghost_layers)
    if kind == "crack":
        return amr_penny_crack(base_n, nlevels, block, 0.1, width=3.0 * hf, ghost_layers=ghost_layers)
    w = 4.0 * hf
    mk = lambda n3, lo3, hi3: polycrystal(grains=12, seed=seed, box=(n3, lo3, hi3), width=w, clamp=True)
    ind = lambda X, Y, Z: mk(X.shape[::-1], (X.min(), Y.min(), Z.min()), (X.max(), Y.max(), Z.max())).moduli[0] / 1.68
    return amr_layout(mk, base_n, nlevels, ind, 0.1, block, ghost_layers)


def ellipsoid_rve(n, seed, nu=0.3, width_cells=3.0, strain_norm=1e-3):
    """Periodic RVE with 1-8 random ellipsoidal inclusions (semi-axes 0.05-0.2,
    uniform orientation, stiffness ratio 0.5-4) under a random symmetric mean strain
    of Frobenius norm strain_norm.  ``n`` counts the node planes including the
    duplicated periodic face, so the grid keeps n - 1 unique nodes per direction.
    Distances use the nearest periodic image (the inclusions are smaller than half
    the cell)."""
    rng = np.random.default_rng(seed)
    m = n - 1
    p = Problem(n=(m, m, m), periodic=(True, True, True), name=f"rve_{n}_{seed}")
    X, Y, Z = p.coords()
    h = p.h[0]
    w = width_cells * h
    E = np.ones(X.shape)
    for _ in range(int(rng.integers(1, 9))):
        axes = rng.uniform(0.05, 0.2, 3)
        R = random_rotation(rng)
        c = rng.random(3)
        ratio = rng.uniform(0.5, 4.0)
        dx = X - c[0]
        dy = Y - c[1]
        dz = Z - c[2]
        dx -= np.round(dx)
        dy -= np.round(dy)
        dz -= np.round(dz)
        q = [R[0, a] * dx + R[1, a] * dy + R[2, a] * dz for a in range(3)]
        rad = np.sqrt(sum((q[a] / axes[a]) ** 2 for a in range(3)))
        s = (rad - 1.0) * axes.min()
        phi = tanh_profile(s, w)
        E = E * (1.0 - phi) + ratio * phi
    lam, mu = lame(E, nu)
    p.moduli_kind = MODULI_ISO
    p.moduli = np.stack([lam, mu])
    G = rng.normal(size=(3, 3))
    S = 0.5 * (G + G.T)
    S *= strain_norm / np.linalg.norm(S)
    p.mean_strain = np.array([S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[2, 0], S[0, 1]])
    p.bc = []
    return p


def batch_sizes(count=256, seed=0, choices=(33, 65, 97, 129)):
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(choices, size=count)]
