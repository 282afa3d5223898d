"""CPU checks of the C-ABI library: it builds, loads, exports every declared symbol, and its
host-side reference element and mesh counts agree with closed forms and the oracle."""
import math
import os
import re

import numpy as np
import pytest

import paper_2410_09790_gb300 as H
from oracle import Mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, 'include', 'hdg.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(hdg_[a-z_]+)\s*\(', src)))


def test_library_exports_every_declared_symbol():
    lib = H.load()
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    lib = H.load()
    for s in range(7):
        assert lib.hdg_status_string(s)


@pytest.mark.parametrize('px,py', [(False, False), (True, False), (True, True)])
def test_mesh_counts_match_oracle(px, py):
    for n in (1, 3, 8):
        for k in (1, 4):
            m = Mesh(n, periodic_x=px, periodic_y=py)
            assert H.hdg_mesh_counts(n, k, px, py) == (m.ncells, m.nfacets)


def test_invalid_arguments_rejected():
    with pytest.raises(H.HdgError):
        H.hdg_mesh_counts(0, 2)
    with pytest.raises(H.HdgError):
        H.hdg_mesh_counts(4, 5)
    with pytest.raises(H.HdgError):
        H.hdg_reference_rule(0, 0)


@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_reference_volume_rule_exact(k):
    pts, w = H.hdg_reference_rule(k, 0)
    deg = 3 * k + 2
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b) - exact) < 1e-15


@pytest.mark.parametrize('k', [1, 2, 3, 4])
def test_reference_facet_rule_is_gauss_legendre(k):
    t, w = H.hdg_reference_rule(k, 1)
    n = len(w)
    assert n == (3 * k + 5) // 2
    x, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(t[:, 0]), (x + 1) / 2, atol=1e-15)
    assert np.allclose(np.sort(w), np.sort(wr / 2), atol=1e-15)


@pytest.mark.parametrize('m', [0, 1, 2, 3, 4, 5])
def test_reference_basis_orthonormal_and_hierarchical(m):
    pts, w = H.hdg_reference_rule(4, 0)           # exact to degree 14 >= 2m
    V = H.hdg_reference_basis(m, pts)
    G = (V.T * w) @ V
    assert np.abs(G - np.eye(V.shape[1])).max() < 1e-13
    if m > 0:
        Vlow = H.hdg_reference_basis(m - 1, pts)
        assert np.abs(V[:, :Vlow.shape[1]] - Vlow).max() < 1e-13   # P_{m-1} basis is a prefix
    # spans P_m: reproduces the monomials by least squares exactly
    mono = np.stack([pts[:, 0] ** a * pts[:, 1] ** (d - a) for d in range(m + 1) for a in range(d + 1)], 1)
    coef = np.linalg.lstsq(V, mono, rcond=None)[0]
    assert np.abs(V @ coef - mono).max() < 1e-12
