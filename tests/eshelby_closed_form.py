"""Closed forms of Eshelby's inclusion problem used to validate the solver (test
infrastructure, not part of the method).

Eshelby tensor of an ellipsoid with semi-axes a_1, a_2, a_3 in an isotropic body of
Poisson ratio nu (Eshelby 1957, in the notation of Mura's *Micromechanics of Defects in
Solids*, Section 11): with Delta(s) = sqrt((a_1^2 + s)(a_2^2 + s)(a_3^2 + s)),

  I_i  = 2 pi a_1 a_2 a_3 int_0^inf ds / ((a_i^2 + s) Delta(s)),
  I_ij = 2 pi a_1 a_2 a_3 int_0^inf ds / ((a_i^2 + s)(a_j^2 + s) Delta(s)),
  S_iiii = 3 a_i^2 I_ii / (8 pi (1 - nu)) + (1 - 2 nu) I_i / (8 pi (1 - nu)),
  S_iijj = a_j^2 I_ij / (8 pi (1 - nu)) - (1 - 2 nu) I_i / (8 pi (1 - nu))   (i != j).

Inside a homogeneous inclusion the strain is uniform, eps = S : eps*, and the stress is
C : (eps - eps*).  The integrals are evaluated by adaptive quadrature."""
import numpy as np


def eshelby_integrals(a):
    from scipy.integrate import quad
    a = np.asarray(a, dtype=float)
    pref = 2 * np.pi * a[0] * a[1] * a[2]
    delta = lambda s: np.sqrt((a[0] ** 2 + s) * (a[1] ** 2 + s) * (a[2] ** 2 + s))
    I = np.array([pref * quad(lambda s, i=i: 1.0 / ((a[i] ** 2 + s) * delta(s)), 0, np.inf, limit=200)[0]
                  for i in range(3)])
    Iij = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            Iij[i, j] = pref * quad(lambda s: 1.0 / ((a[i] ** 2 + s) * (a[j] ** 2 + s) * delta(s)), 0, np.inf,
                                    limit=200)[0]
    return I, Iij


def normal_eshelby_block(a, nu):
    """S_iijj (3 x 3) of the ellipsoid a: the part a dilatational eigenstrain sees."""
    a = np.asarray(a, dtype=float)
    I, Iij = eshelby_integrals(a)
    c = 1.0 / (8 * np.pi * (1 - nu))
    S = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                S[i, j] = c * (3 * a[i] ** 2 * Iij[i, i] + (1 - 2 * nu) * I[i])
            else:
                S[i, j] = c * (a[j] ** 2 * Iij[i, j] - (1 - 2 * nu) * I[i])
    return S


def interior_stress_dilatational(a, E, nu, eps_star):
    """Normal stresses (s11, s22, s33) inside a homogeneous ellipsoidal inclusion with
    eigenstrain eps_star I (the shear stresses vanish)."""
    S = normal_eshelby_block(a, nu)
    eps = S @ np.full(3, eps_star)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    d = eps - eps_star
    return lam * d.sum() + 2 * mu * d
