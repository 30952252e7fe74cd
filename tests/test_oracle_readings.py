"""Readings of the paper that rest on a measurement, repeated with the CPU oracle.

* Penny crack (Section 4.2): the modulus inside the crack is capped at 1 % of the bulk
  modulus, the stabilising floor the paper keeps, not the 1e-4 a sharper model would
  take.  With 1e-4 the product-rule operator's V(2,2) cycle diverges on a 17^3 crack
  (the residual grows by about 10^8 per cycle); with the 1 % floor it converges.
* Singular problems (Section 2.1.1 product rule): loads outside the operator's range,
  hence the equilibrating load of the solve."""
import numpy as np

from paper_2001_04789_gb300 import microstructure as M
from oracle import multigrid as MG


def test_crack_modulus_floor_of_one_percent_converges_and_1e4_diverges():
    with np.errstate(all="ignore"):
        _, soft = MG.solve(M.penny_crack(17, width=3.0 / 16, soft=1e-4), tol=1e-8, max_cycles=4)
        _, capped = MG.solve(M.penny_crack(17, width=3.0 / 16, soft=1e-2), tol=1e-8, max_cycles=40)
    hist = np.asarray(soft.rel_history, dtype=float)
    assert not np.all(np.isfinite(hist)) or hist[-1] > 1e6 * hist[1]      # diverging
    assert capped.rel_residual <= 1e-8 and capped.cycles < 40
    c = np.asarray(capped.rel_history[1:], dtype=float)
    assert np.all(c[1:] < c[:-1])                                          # monotone contraction


def _left_null(p):
    """The free rows and the left null space of the assembled operator of problem p (its
    dimension is the number of free rigid modes), with the singular values around that gap."""
    from oracle import stencil as S
    L = MG.build_hierarchy(S.level_from_problem(p))[0]
    free, A = MG.assemble_dense(L.level, L.types)
    U, s, _ = np.linalg.svd(A)
    k = L.null.shape[0]
    return L, free, U[:, -k:], s[-k] / s[0], s[-k - 1] / s[0]


def _share(p, L, free, W):
    """Share of p's effective load (the residual of the Dirichlet-filled zero field on the
    free rows) in the left null space W: the operator depends on the moduli and boundary
    types only, so one factorisation serves every load."""
    from oracle import stencil as S
    f = S.rhs(L.level, p)
    uD = S.dirichlet_values(L.level, p.dirichlet_values)
    b = S.residual(L.level, uD, f, L.types)[free]
    return np.linalg.norm(W.T @ b) / np.linalg.norm(b)


def _iso_tensor():
    lam, mu = M.lame(1.0, 0.3)
    return M.voigt_to_tensor(M.cubic_voigt(lam + 2 * mu, lam, mu))


def _periodic_inclusion(n):
    """Fully periodic cell: a smooth rotated-cubic sphere in an isotropic matrix."""
    p = M.Problem(n=(n, n, n), periodic=(True, True, True))
    X, Y, Z = p.coords()
    c = [(a.max() + a.min()) / 2 for a in (X, Y, Z)]
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    phi = 0.5 * (1 - np.tanh((r - 0.25) / (2 * p.h[0])))
    Cin = M.rotate_tensor(M.voigt_to_tensor(M.cubic_voigt(1.68, 1.21, 0.75)),
                          M.random_rotation(np.random.default_rng(3)))
    up = lambda C: M.tensor_to_upper21(C)[:, None, None, None]
    p.moduli_kind = M.MODULI_GEN21
    p.moduli = up(_iso_tensor()) * (1 - phi) + up(Cin) * phi
    p.bc = []
    return p, phi


def test_loads_outside_the_range_of_the_product_rule_operator():
    """Singular problems (free rigid modes): the product-rule operator is not in divergence
    form, so its left null vectors are not the rigid modes and a load need not be in its
    range; the solve therefore carries an equilibrating load.  Measured by SVD of the
    assembled operator: the polycrystal with traction-free faces puts a few 1e-4 of its
    load outside the range, the same boundary conditions with constant moduli none; on a
    periodic cell the mean-strain and eigenstrain loads lie in the range, a zero-mean body
    force does not.  The oracle's solve converges on the incompatible problem with a
    nonzero equilibrating load."""
    p = M.polycrystal(5, grains=3, seed=2)
    L, free, W, gap_lo, gap_hi = _left_null(p)
    assert gap_lo < 1e-12 and gap_hi > 1e-4           # rigid modes: a clean null space
    assert _share(p, L, free, W) > 1e-5
    _, info = MG.solve(p, tol=1e-10, max_cycles=200)
    assert info.converged and np.abs(np.asarray(info.lam)).max() > 0
    q = M.polycrystal(5, grains=3, seed=2)
    q.moduli = M.tensor_to_upper21(_iso_tensor())[:, None, None, None] * np.ones((1,) + q.moduli.shape[1:])
    assert _share(q, *_left_null(q)[:3]) < 1e-12
    cell, phi = _periodic_inclusion(6)
    L, free, W, _, _ = _left_null(cell)
    cell.mean_strain = np.array([0.7, -0.4, 0.25, 0.5, -0.35, 0.6]) * 1e-3
    assert _share(cell, L, free, W) < 1e-12
    cell.mean_strain = None
    cell.eigenstrain = np.array([1.0, 0.5, -0.3, 0.2, 0.0, 0.1])[:, None, None, None] * 1e-3 * phi[None]
    assert _share(cell, L, free, W) < 1e-12
    cell.eigenstrain = None
    b = np.random.default_rng(1).normal(size=(3,) + phi.shape)
    cell.body_force = b - b.mean(axis=(1, 2, 3), keepdims=True)
    assert _share(cell, L, free, W) > 1e-5
