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


def struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/hdg.h."""
    src = open(os.path.join(ROOT, 'include', 'hdg.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    body = re.search(r'typedef struct \{([^{}]*)\}\s*' + name + r'\s*;', src).group(1)
    out = []
    for decl in body.split(';'):
        decl = decl.strip()
        if decl:
            parts = decl.split(',')           # "type a, b": a is the last word of the first part
            names = [parts[0].split()[-1]] + [q.strip() for q in parts[1:]]
            out += [v.lstrip('*').split('[')[0] for v in names]
    return out


@pytest.mark.parametrize('name', ['hdg_params', 'hdg_stats', 'hdg_mesh_desc'])
def test_ctypes_mirrors_match_header(name):
    # the binding's ctypes structures list the header's fields in the header's order
    assert [f[0] for f in getattr(H.hdg, name)._fields_] == struct_fields(name)


def test_default_params():
    # hdg_default_params (host code) fills the documented defaults, the GB300 options on
    p = H.hdg.hdg_default_params()
    assert p.alpha == 1.0 and p.tau == 1.0 and p.delta_up == 1.0 and p.n_richardson == 2
    assert p.trace_rtol == 1e-12 and p.stepI_rtol == 1e-10
    assert (p.stage_krylov, p.trace_mg, p.device_loops, p.inner_trace_vcycles) == (1, 1, 1, 1)
    assert (p.inner_trace_fp32, p.trace_fp32_vcycle, p.inner_gs, p.precision) == (1, 1, 1, 1)
    assert p.inner_stepI_rtol == 2e-2 and p.inner_trace_rtol == 1e-1
    assert p.timeout_ms == 0.0 and p.relax_eta == 1e-5


def test_status_strings():
    lib = H.load()
    for s in range(8):
        assert lib.hdg_status_string(s).decode() != 'unknown status'


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


def test_memory_estimate_host_only():
    # hdg_estimate_bytes (host code, used by the server's admission): positive, growing with the
    # mesh and the degree, the stage FGMRES bases counted only when stages are solved to tolerance,
    # the FP32 cell maps only in mixed precision; 0 for an invalid degree
    est = lambda n, k, **kw: H.hdg_estimate_bytes(n, k, tableau='ARS343', **kw)
    assert est(16, 2) > 0
    assert est(32, 2) > 3.5 * est(16, 2) and est(32, 3) > est(32, 2) > est(32, 1)
    assert est(32, 3, n_richardson=0, stage_krylov=1) > est(32, 3, n_richardson=2)
    assert est(32, 3, n_richardson=0, precision='MIXED') > est(32, 3, n_richardson=0, precision='FP64')
    # the FP32 copy of the diagonal blocks (relaxed products): 4 NU^2 bytes per cell and more
    nu, nc = 2 * 10, 2 * 32 * 32
    d = est(32, 3, n_richardson=0, precision='MIXED') - est(32, 3, n_richardson=0, precision='MIXED', relax_eta=0.0)
    assert d >= 4 * nu * nu * nc
    assert H.hdg_estimate_bytes(16, 5) == 0.0
