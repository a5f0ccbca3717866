"""C-ABI library: loads, exports every declared symbol, and its host logic (quadrature,
bases, table products, expanded mesh) agrees with the independent oracle.  CPU only: no
call here touches the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import basis, hdg as ohdg, quadrature
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, kuhn_cube

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_1489_gb300 import _lib, build
    build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1305_1489_gb300 import _lib
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.exported_symbols())


def _table(lib, k, name):
    size = C.c_int64(0)
    assert lib.hdg_host_table(k, name.encode(), None, 0, C.byref(size)) == 0
    out = np.zeros(size.value)
    assert lib.hdg_host_table(k, name.encode(), out.ctypes.data, size.value, C.byref(size)) == 0
    return out


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_host_tables_match_oracle(lib, k):
    tab = ohdg.Tables(k)
    n, d2 = tab.n, tab.d2
    assert np.allclose(_table(lib, k, "vol_pts").reshape(-1, 3), tab.p, atol=1e-15, rtol=0)
    assert np.allclose(_table(lib, k, "vol_w"), tab.w, atol=1e-15, rtol=0)
    assert np.allclose(_table(lib, k, "face_pts").reshape(-1, 2), tab.qf, atol=1e-15, rtol=0)
    assert np.allclose(_table(lib, k, "face_w"), tab.varpi, atol=1e-15, rtol=0)
    tol = 1e-12
    assert np.abs(_table(lib, k, "P").reshape(-1, n) - tab.P).max() < tol
    assert np.abs(_table(lib, k, "Pd").reshape(3, -1, n) - tab.Pstar).max() < 1e-11
    assert np.abs(_table(lib, k, "Chat").reshape(3, n, n) - tab.Chat).max() < tol
    assert np.abs(_table(lib, k, "Pl").reshape(4, -1, n) - tab.Pl).max() < tol
    assert np.abs(_table(lib, k, "D").reshape(-1, d2) - tab.D).max() < tol
    assert np.abs(_table(lib, k, "Dmu").reshape(6, -1, d2) - tab.Dmu).max() < tol
    S = np.stack([(tab.varpi[:, None] * tab.Pl[l]).T @ tab.Pl[l] for l in range(4)])
    assert np.abs(_table(lib, k, "S").reshape(4, n, n) - S).max() < tol
    E = np.stack([[(tab.varpi[:, None] * tab.Dmu[mu]).T @ tab.Pl[l] for mu in range(6)] for l in range(4)])
    assert np.abs(_table(lib, k, "E").reshape(4, 6, d2, n) - E).max() < tol
    n1 = basis.d3(k + 1)
    assert np.abs(_table(lib, k, "P1").reshape(-1, n1) - basis.dubiner3(k + 1, tab.p)).max() < tol
    assert np.abs(_table(lib, k, "G1").reshape(3, -1, n1) - basis.dubiner3_grad(k + 1, tab.p)).max() < 1e-11


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_host_symmetric_rule_tables_match_oracle(lib, k):
    """The library's own Grundmann-Moller rule (tables.cpp) against the oracle's
    (quadrature.symmetric_volume_rule): same nodes in the same order, same weights, and the
    volume basis tables built on them."""
    tab = ohdg.Tables(k, "symmetric")
    n = tab.n
    assert np.allclose(_table(lib, k, "vol_pts:sym").reshape(-1, 3), tab.p, atol=1e-15, rtol=0)
    assert np.allclose(_table(lib, k, "vol_w:sym"), tab.w, atol=1e-14, rtol=0)
    assert np.abs(_table(lib, k, "P:sym").reshape(-1, n) - tab.P).max() < 1e-12
    assert np.abs(_table(lib, k, "Pd:sym").reshape(3, -1, n) - tab.Pstar).max() < 1e-11
    # C_hat is a volume integral of degree 2k - 1: the same on either rule
    assert np.abs(_table(lib, k, "Chat:sym") - _table(lib, k, "Chat")).max() < 1e-12


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_host_sum_factorisation_reproduces_oracle_masses(lib, k):
    """The library's sum-factorisation tables, summed in three passes as the double-float K1
    does, give the oracle's direct quadrature sum_q g_q P_a P_b for an arbitrary weight g."""
    tab = ohdg.Tables(k)
    n, d2, nn = tab.n, tab.d2, k + 2
    AA = _table(lib, k, "sfAA").reshape(-1, nn)
    BB = _table(lib, k, "sfBB").reshape(-1, nn)
    CC = _table(lib, k, "sfCC").reshape(-1, nn)
    p2to1 = _table(lib, k, "sfp2to1").astype(int)
    p3to2 = _table(lib, k, "sfp3to2").astype(int)
    assert AA.shape[0] == (k + 1) * (k + 2) // 2 and BB.shape[0] == d2 * (d2 + 1) // 2
    assert CC.shape[0] == n * (n + 1) // 2
    g = np.random.default_rng(k).uniform(0.5, 2.0, size=tab.nq).reshape(nn, nn, nn)  # [i, j, l]
    T1 = np.einsum("ijl,pl->pij", g, AA)
    T2 = np.einsum("pj,pij->pi", BB, T1[p2to1])
    lib_mass = np.einsum("ti,ti->t", CC, T2[p3to2])
    ia, ib = np.triu_indices(n)  # the row-major (a <= b) order of the 3-D pairs
    ref = np.einsum("q,qt,qt->t", g.ravel(), tab.P[:, ia], tab.P[:, ib])
    assert np.abs(lib_mass - ref).max() < 1e-12 * np.abs(ref).max()


def _expand(lib, c, e, d, nn):
    nelt = len(e)
    nfc = C.c_int64(0)
    faces = np.zeros((4 * nelt, 4), np.int32)
    fbe = np.zeros((nelt, 4), np.int32)
    perm = np.zeros((nelt, 4), np.int32)
    c = np.ascontiguousarray(c, np.float64)
    e = np.ascontiguousarray(e, np.int32)
    d = np.ascontiguousarray(d, np.int32)
    nn = np.ascontiguousarray(nn, np.int32)
    rc = lib.hdg_host_expand_mesh(c.ctypes.data, len(c), e.ctypes.data, nelt,
                                  d.ctypes.data if len(d) else None, len(d),
                                  nn.ctypes.data if len(nn) else None, len(nn),
                                  C.byref(nfc), faces.ctypes.data, fbe.ctypes.data, perm.ctypes.data)
    return rc, faces[:nfc.value], fbe, perm


@pytest.mark.parametrize("s,jit", [(2, 0.0), (3, 0.2)])
def test_host_expanded_mesh_matches_oracle(lib, s, jit):
    c, e = kuhn_cube(s, jitter=jit, seed=1)
    d, n = boundary_faces(c, e, lambda ax, v: "D" if ax == 2 else "N")
    rc, faces, fbe, perm = _expand(lib, c, e, d, n)
    assert rc == 0
    m = ExpandedMesh(c, e, d, n)
    assert np.array_equal(faces[:, :3], m.faces)
    assert np.array_equal(faces[:, 3], m.facetype)
    assert np.array_equal(fbe, m.facebyele)
    assert np.array_equal(perm, m.perm)


def test_host_mesh_errors(lib):
    c, e = kuhn_cube(1)
    d, n = boundary_faces(c, e, lambda ax, v: "D")
    rc, *_ = _expand(lib, c, e, d[:-1], n)
    assert rc == 3  # HDG_ERR_NONCONFORMING: a boundary face is in neither list
    e2 = e.copy()
    e2[0, [2, 3]] = e2[0, [3, 2]]
    rc, *_ = _expand(lib, c, e2, d, n)
    assert rc == 2  # HDG_ERR_ORIENTATION
    size = C.c_int64(0)
    assert lib.hdg_host_table(7, b"P", None, 0, C.byref(size)) == 9  # HDG_ERR_UNSUPPORTED


# C structs of include/hdg.h and their ctypes mirrors in the binding
_STRUCTS = {"hdg_mesh_info": "MeshInfo", "hdg_tuning": "Tuning", "hdg_host_inputs": "HostInputs"}


def _struct_fields(src, name):
    """Field names of `typedef struct [tag] { ... } name;` in declaration order."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct\s*\w*\s*\{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [re.sub(r"[\s*]", "", v) for v in re.sub(r"^(const\s+)?\w+", "", decl).split(",")]
    return names


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's fields in its order, at the offsets
    and with the sizes a C compiler gives them (gcc compiles a probe against include/hdg.h)."""
    import shutil
    import subprocess
    from paper_1305_1489_gb300 import _lib
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hdg.h"', "int main(void) {"]
    expect = []
    for cname, pyname in _STRUCTS.items():
        fields = _struct_fields(src, cname)
        py = getattr(_lib, pyname)
        assert [f for f, _ in py._fields_] == fields, cname
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(C.sizeof(py))
        for f in fields:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            expect.append(getattr(py, f).offset)
    lines += ["  return 0;", "}"]
    (tmp_path / "probe.c").write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(tmp_path / "probe.c"), "-o", str(exe)],
                   check=True, capture_output=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
