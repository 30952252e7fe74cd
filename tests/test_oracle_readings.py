"""Readings of the paper that rest on a measurement, repeated with the CPU oracle.

Penny crack (Section 4.2): the modulus inside the crack is capped at 1 % of the bulk
modulus, the stabilising floor the paper keeps, not the 1e-4 a sharper model would
take.  With 1e-4 the product-rule operator's V(2,2) cycle diverges on a 17^3 crack
(the residual grows by about 10^8 per cycle); with the 1 % floor it converges."""
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
