"""The synthetic inputs are seeded: the same seed gives the same arrays, in this process
and in a fresh one (no hidden global state), and different seeds give different ones.
The random rotations of the polycrystal and RVE grains are proper rotations."""
import hashlib
import os
import subprocess
import sys

import numpy as np

from paper_2001_04789_gb300 import microstructure as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _digest(kind, n, seed):
    if kind == "poly":
        p = M.polycrystal(n, grains=4, seed=seed)
        arrays = [p.moduli]
    elif kind == "rve":
        p = M.ellipsoid_rve(n, seed=seed)
        arrays = [p.moduli, p.mean_strain]
    else:
        arrays = [np.asarray(M.batch_sizes(64, seed=seed))]
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


CASES = [("poly", 13, 2), ("rve", 13, 3), ("sizes", 0, 5)]


def test_same_seed_same_inputs_across_processes():
    here = [_digest(*c) for c in CASES]
    assert here == [_digest(*c) for c in CASES]
    code = ("import sys; sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[2]); "
            "import test_inputs_cpu as T; print(' '.join(T._digest(*c) for c in T.CASES))")
    out = subprocess.run([sys.executable, "-c", code, ROOT, os.path.join(ROOT, "tests")],
                         capture_output=True, text=True, check=True, timeout=300).stdout.split()
    assert out == here


def test_different_seeds_differ_and_sizes_come_from_the_choices():
    assert _digest("poly", 13, 2) != _digest("poly", 13, 3)
    assert _digest("rve", 13, 3) != _digest("rve", 13, 4)
    sizes = M.batch_sizes(256, seed=0)
    assert set(sizes) <= {33, 65, 97, 129} and len(set(sizes)) == 4


def test_random_rotations_are_proper():
    rng = np.random.default_rng(9)
    for _ in range(200):
        R = M.random_rotation(rng)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
