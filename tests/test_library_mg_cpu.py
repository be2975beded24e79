"""CPU checks of the multigrid hierarchy of the pressure-correction solve
(host logic of the library, no GPU): coarse grids, level counts and the
prolongation weights against what the construction fixes -- every coarse
face is a fine face, the coarse cells tile the axis, and linear
interpolation between coarse centres reproduces constants everywhere and
linear functions at every fine centre between the first and last coarse
centre."""
import ctypes

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_08521_gb300._lib import lib
    return lib


MAPS = {"sine0975": 0, "cosine": 1, "uniform": 2}


def axis(lib, n, kind, level):
    nout = ctypes.c_int()
    assert lib.fv_host_mg_axis(n, MAPS[kind], level, ctypes.byref(nout), None, None, None) == 0
    m = nout.value
    faces = np.empty(m + 1)
    pc0 = np.empty(m, dtype=np.int32)
    pw1 = np.empty(m)
    assert lib.fv_host_mg_axis(n, MAPS[kind], level, ctypes.byref(nout), faces.ctypes.data,
                               pc0.ctypes.data, pw1.ctypes.data) == 0
    return faces, pc0, pw1


@pytest.mark.parametrize("n,expect", [((100, 100, 100), 6), ((256, 256, 256), 7),
                                      ((150, 150, 150), 7), ((4, 4, 4), 1), ((5, 4, 4), 2),
                                      ((112, 112, 8), 6)])
def test_level_count(lib, n, expect):
    assert lib.fv_host_mg_levels(*n) == expect


@pytest.mark.parametrize("n", [4, 5, 7, 13, 100, 150, 256])
@pytest.mark.parametrize("kind", ["cosine", "sine0975", "uniform"])
def test_coarse_axes_and_prolongation(lib, n, kind):
    fine = synth.map_faces(n, kind)
    prev = None
    for level in range(10):
        faces, pc0, pw1 = axis(lib, n, kind, level)
        m = len(faces) - 1
        if level == 0:
            assert np.array_equal(faces, fine)
        else:
            # every other face of the level above and its last one
            pf = prev
            want = np.append(pf[:-1:2], pf[-1]) if len(pf) - 1 > 2 else pf
            assert np.array_equal(faces, want)
        assert np.all(np.diff(faces) > 0) and faces[0] == 0.0 and faces[-1] == 1.0
        # prolongation from the next level to this one
        cf, _, _ = axis(lib, n, kind, level + 1)
        xc = 0.5 * (faces[1:] + faces[:-1])
        Xc = 0.5 * (cf[1:] + cf[:-1])
        assert np.all((pw1 >= 0) & (pw1 <= 1))
        assert np.all((pc0 >= 0) & (pc0 < len(Xc)))
        assert np.all(pc0[pw1 > 0] + 1 < len(Xc))
        if len(Xc) == m:                     # axis not coarsened: the identity
            assert np.array_equal(pc0, np.arange(m)) and np.all(pw1 == 0)
        else:
            lin = lambda x: 2.0 - 3.0 * x       # noqa: E731
            hi = np.minimum(pc0 + 1, len(Xc) - 1)
            interp = (1 - pw1) * lin(Xc[pc0]) + pw1 * lin(Xc[hi])
            inside = (xc >= Xc[0]) & (xc <= Xc[-1])
            assert np.allclose(interp[inside], lin(xc[inside]), rtol=0, atol=1e-13)
            # outside the first / last coarse centre: the nearest centre's value
            assert np.all(pw1[~inside] == 0)
            assert np.all(pc0[xc < Xc[0]] == 0) and np.all(pc0[xc > Xc[-1]] == len(Xc) - 1)
        prev = faces
        if m <= 2:
            break


def test_bad_arguments(lib):
    nout = ctypes.c_int()
    assert lib.fv_host_mg_axis(0, 1, 0, ctypes.byref(nout), None, None, None) != 0
    assert lib.fv_host_mg_axis(8, 7, 0, ctypes.byref(nout), None, None, None) != 0
    assert lib.fv_host_mg_levels(0, 4, 4) == -1


def test_bench_hierarchy_matches_library(lib):
    """bench.py counts the multigrid's algorithmic bytes over the same
    hierarchy the library builds."""
    import bench
    for n in (4, 5, 13, 64, 100, 150, 256):
        lv = bench.mg_levels(n)
        assert len(lv) == lib.fv_host_mg_levels(n, n, n)
        for level, cells in enumerate(lv):
            nout = ctypes.c_int()
            assert lib.fv_host_mg_axis(n, 1, level, ctypes.byref(nout), None, None, None) == 0
            assert cells == nout.value ** 3
