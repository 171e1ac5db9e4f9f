"""The C-ABI library builds, loads and exports every function include/vlb.h
declares; the host-only lattice query agrees with the paper's velocity set.
No GPU needed (no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    return vlb.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "vlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(vlb_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        # and it is a real exported function
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_binding_covers_the_header():
    from paper_2401_17183_gb300 import vlb
    lib = vlb.load()
    for n in _declared():
        assert getattr(lib, n).argtypes is not None or n == "vlb_last_error", n


def test_lattice_matches_paper_set_and_pairs():
    from oracle import lattice as olat
    from paper_2401_17183_gb300 import vlb
    for q in (9, 19, 39):
        c, w = vlb.lattice(q)
        co, wo, _ = olat(q)
        assert len({tuple(v) for v in c}) == q
        assert sorted(map(tuple, c)) == sorted(map(tuple, co))
        # weights agree direction by direction
        for a in range(q):
            b = [k for k in range(q) if tuple(co[k]) == tuple(c[a])][0]
            assert w[a] == wo[b]
        # the library's pairing: direction a + H is -c_a
        H = (q - 1) // 2
        for a in range(1, H + 1):
            assert np.array_equal(c[a + H], -c[a])


def test_errors_without_gpu_work(lib):
    from paper_2401_17183_gb300 import vlb
    with pytest.raises(vlb.VlbError) as e:
        vlb.lattice(15)
    assert e.value.code == "EINVAL"
    d = vlb.vlb_mesh_desc()
    d.dim = 2
    d.lattice = 19          # D3Q19 in 2D is rejected before any device work
    h = ctypes.c_void_p()
    x = np.zeros(8)
    d.x = x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n[0], d.n[1], d.n[2] = 2, 2, 1
    rc = lib.vlb_mesh_create(ctypes.byref(d), ctypes.byref(h))
    assert rc == vlb.VLB_EINVAL and not h.value
    assert b"lattice" in lib.vlb_last_error()


def test_empty_and_degenerate_sizes_are_rejected_on_the_host(lib):
    """Sizes the method has no meaning for are refused by the host-side checks,
    before any device work: an empty axis, a wall axis of one node (it has no
    interior row to extrapolate a ghost from), a 2D mesh with n[2] != 1, a
    D3Q39 axis shorter than its three-cell links, and a negative step count or
    a missing simulation."""
    from paper_2401_17183_gb300 import vlb
    x = np.zeros(64 * 3)

    def create(dim, q, n, bc):
        d = vlb.vlb_mesh_desc()
        d.dim, d.lattice = dim, q
        d.x = x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        for a in range(3):
            d.n[a] = n[a]
            d.bc[a] = bc[a]
        h = ctypes.c_void_p()
        rc = lib.vlb_mesh_create(ctypes.byref(d), ctypes.byref(h))
        assert not h.value
        return rc, lib.vlb_last_error()

    P, Wl = vlb.VLB_PERIODIC, vlb.VLB_WALL
    cases = [
        ((2, 9, (0, 4, 1), (P, P, P)), b"n[0]"),
        ((3, 19, (4, 4, 0), (P, P, P)), b"n[2]"),
        ((3, 19, (4, -3, 4), (P, P, P)), b"n[1]"),
        ((2, 9, (4, 1, 1), (P, Wl, P)), b"wall axis"),
        ((2, 9, (4, 4, 2), (P, P, P)), b"n[2] must be 1"),
        ((3, 39, (4, 2, 4), (P, P, P)), b"D3Q39"),
        ((3, 39, (4, 4, 4), (P, Wl, P)), b"D3Q39"),
    ]
    for args, msg in cases:
        rc, err = create(*args)
        assert rc == vlb.VLB_EINVAL, args
        assert msg in err, (args, err)
    assert lib.vlb_step(None, 1) == vlb.VLB_EINVAL
