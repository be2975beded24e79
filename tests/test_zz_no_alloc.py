"""The allocation-free pressure solve (fv_pressure_solve_noalloc) against the
grid-based entry point fv_pressure_solve in the same float32 arithmetic.

It exists for callers that cannot allocate device memory (inside a memory
pool they do not own, or without an allocator); its scratch lives in a fixed
device array of the library.  Besides matching the grid solve on two calls
in a row, a call after the first one on the device must leave the device's
free memory unchanged.  This file is collected last so a failure here never
hides the other tests; it passes alone and after them."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def _rhs(shape, seed):
    # a compatible right-hand side: divergence of a seeded velocity field
    r = synth.gaussian_cells(shape, seed)
    return r - r.mean()


@pytest.mark.parametrize("shape,kind", [((20, 24, 18), "cosine"), ((100, 100, 100), "cosine"),
                                        ((7, 9, 5), "sine0975")])
def test_noalloc_matches_grid_solve_twice(fv, shape, kind):
    nz, ny, nx = shape
    g = fv.Grid(nx, ny, nz, kind, alpha=0.0, re=100.0)
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((3, 4)):                     # two calls in a row
        r = torch.tensor(_rhs(shape, seed), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(r)
        fv.fv_pressure_solve(g, r, ref, "mixed")
        out = torch.full_like(r, float("nan"))
        st = fv.lib.fv_pressure_solve_noalloc(nx, ny, nz, fv.MAPS[kind], ctypes.c_void_p(r.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0, fv.lib.fv_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), call
    # once the first call on the device has reserved the array, a call takes
    # no device memory: the driver's free-memory figure does not move
    r = torch.tensor(_rhs(shape, 5), dtype=torch.float64, device="cuda")
    out = torch.empty_like(r)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = fv.lib.fv_pressure_solve_noalloc(nx, ny, nz, fv.MAPS[kind], ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    assert st == 0
    assert torch.cuda.mem_get_info()[0] == free0
    g.close()


def test_noalloc_rejects_sizes_beyond_limit(fv):
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = fv.lib.fv_pressure_solve_noalloc(129, 8, 8, 1, ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(r.data_ptr()), None)
    assert st == 1 and b"[4, 128]" in fv.lib.fv_last_error()
    st = fv.lib.fv_pressure_solve_noalloc(128, 128, 128, 1, ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(r.data_ptr()), None)
    assert st == 1 and b"1048576" in fv.lib.fv_last_error()
