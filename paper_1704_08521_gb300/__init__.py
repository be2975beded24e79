"""Python binding of libfvns (the C ABI in include/fvns.h).

Argument marshalling only: every computation runs in the CUDA kernels of
libfvns.so.  Device buffers are torch tensors (float64, CUDA, contiguous);
their data pointers and the current torch stream are passed through.  There
is no CPU fallback: importing this package fails loudly when the library is
missing (build it with ``__graft_entry__.build()``).

Storage layout (cell-indexed MAC, see include/fvns.h): a velocity vector of
an nx x ny x nz grid holds 3 * nz * ny * nx values [u | v | w], each block
C-ordered [k][j][i]; u[k][j][0], v[k][0][i], w[0][j][i] are walls (zero).
"""
import ctypes
import math
import os

from ._lib import lib, FvError, check, STATUS_NAMES  # noqa: F401

FV_MAP_SINE0975, FV_MAP_COSINE, FV_MAP_UNIFORM = 0, 1, 2
MAPS = {"sine0975": FV_MAP_SINE0975, "cosine": FV_MAP_COSINE, "uniform": FV_MAP_UNIFORM}
FV_FP64, FV_MIXED, FV_FF = 0, 1, 2
PRECS = {"fp64": FV_FP64, "mixed": FV_MIXED, "ff": FV_FF}


class fv_grid_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("n_cell", ctypes.c_int64), ("n_vel", ctypes.c_int64),
                ("n_unknown_vel", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]


class fv_simple_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_pass", ctypes.c_int), ("prec", ctypes.c_int),
                ("omega", ctypes.c_double), ("sigma", ctypes.c_double), ("async_", ctypes.c_int),
                ("pressure", ctypes.c_int), ("pressure_rtol", ctypes.c_double)]


class fv_simple_stats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("phi_first", ctypes.c_double),
                ("phi_last", ctypes.c_double), ("div_max", ctypes.c_double)]


class fv_newton_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_newton", ctypes.c_int), ("gmres_m", ctypes.c_int),
                ("gmres_max_it", ctypes.c_int), ("gmres_rtol", ctypes.c_double),
                ("prec", ctypes.c_int), ("sigma", ctypes.c_double),
                ("simple_eps", ctypes.c_double), ("linear", ctypes.c_int),
                ("gmres_sat", ctypes.c_double), ("precond", ctypes.c_int),
                ("precond_sigma", ctypes.c_double), ("forcing", ctypes.c_int),
                ("gmres_aug", ctypes.c_int), ("tau", ctypes.c_double)]


class fv_newton_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("gmres_total", ctypes.c_int),
                ("res_hist", ctypes.c_double * 64), ("res_final", ctypes.c_double),
                ("bicgstab_total", ctypes.c_int), ("lin_hist", ctypes.c_double * 64)]


LINEAR = {"gmres+bicgstab": 0, "gmres": 1, "bicgstab": 2}


class fv_arnoldi_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_restarts", ctypes.c_int), ("prec", ctypes.c_int),
                ("sigma", ctypes.c_double), ("simple_eps", ctypes.c_double)]


class fv_arnoldi_stats(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("ritz_resid", ctypes.c_double * 64)]


def _ptr(t):
    """Device pointer of a CUDA float64 contiguous tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f64(t, n, name):
    import torch
    if t.dtype != torch.float64 or t.numel() != n:
        raise ValueError(f"{name}: expected {n} float64 values, got {t.numel()} {t.dtype}")
    return _ptr(t)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Grid:
    """Owner of an fv_grid handle (Section 2-3: grid size, map, lid angle, Re)."""

    def __init__(self, nx, ny, nz, map="cosine", alpha=0.0, re=1000.0, stream=None):
        h = ctypes.c_void_p()
        st = _stream() if stream is None else ctypes.c_void_p(stream)
        check(lib.fv_grid_create(nx, ny, nz, MAPS[map] if isinstance(map, str) else int(map),
                                 ctypes.c_double(alpha), ctypes.c_double(re), st,
                                 ctypes.byref(h)), "fv_grid_create")
        self.handle = h
        self.shape = (nz, ny, nx)
        self.n_cell = nx * ny * nz
        self.n_vel = 3 * self.n_cell
        self.alpha, self.re, self.map = alpha, re, map

    def set_re(self, re):
        check(lib.fv_grid_set_re(self.handle, ctypes.c_double(re)), "fv_grid_set_re")
        self.re = re

    def set_stream(self, stream):
        check(lib.fv_grid_set_stream(self.handle, ctypes.c_void_p(stream)), "fv_grid_set_stream")

    def set_base(self, U):
        """Register U as the base flow (fv_grid_set_base); evaluations with
        U=None then use it."""
        check(lib.fv_grid_set_base(self.handle, _f64(U, self.n_vel, "U")), "fv_grid_set_base")

    def info(self):
        i = fv_grid_info()
        check(lib.fv_grid_get_info(self.handle, ctypes.byref(i)), "fv_grid_get_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib.fv_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_grid_create(nx, ny, nz, map="cosine", alpha=0.0, re=1000.0, stream=None):
    return Grid(nx, ny, nz, map, alpha, re, stream)


def ns_residual(g, U, P, F_mom, F_div):
    check(lib.ns_residual(g.handle, _f64(U, g.n_vel, "U"), _f64(P, g.n_cell, "P"),
                          _f64(F_mom, g.n_vel, "F_mom"), _f64(F_div, g.n_cell, "F_div")),
          "ns_residual")


def ns_jacvec(g, U, v, Jv, prec="fp64"):
    check(lib.ns_jacvec(g.handle, _f64(U, g.n_vel, "U"), _f64(v, g.n_vel, "v"),
                        _f64(Jv, g.n_vel, "Jv"), PRECS.get(prec, prec)), "ns_jacvec")


PRESSURE = {"tpf": 0, "mg": 1}


def simple_krylov_solve(g, U, v_in, v_out, p_out=None, eps=1e-8, max_pass=200, prec="fp64",
                        omega=1.0, sigma=0.0, async_=False, pressure="tpf", pressure_rtol=0.0):
    o = fv_simple_opts(eps, max_pass, PRECS.get(prec, prec), omega, sigma, 1 if async_ else 0,
                       PRESSURE.get(pressure, pressure), pressure_rtol)
    s = fv_simple_stats()
    check(lib.simple_krylov_solve(g.handle, None if U is None else _f64(U, g.n_vel, "U"),
                                  _f64(v_in, g.n_vel, "v_in"),
                                  _f64(v_out, g.n_vel, "v_out"),
                                  None if p_out is None else _f64(p_out, g.n_cell, "p_out"),
                                  ctypes.byref(o), ctypes.byref(s)), "simple_krylov_solve")
    return {"passes": s.passes, "phi_first": s.phi_first, "phi_last": s.phi_last,
            "div_max": s.div_max}


def newton_steady(g, U, P, tol=1e-10, max_newton=30, gmres_m=100, gmres_max_it=20000,
                  gmres_rtol=1e-8, prec="fp64", sigma=10.0, simple_eps=1e-10, raise_on_fail=True,
                  linear="gmres+bicgstab", gmres_sat=0.5, precond=0, precond_sigma=0.0, forcing=0,
                  gmres_aug=0, tau=0.0):
    o = fv_newton_opts(tol, max_newton, gmres_m, gmres_max_it, gmres_rtol, PRECS.get(prec, prec),
                       sigma, simple_eps, LINEAR.get(linear, linear), gmres_sat, int(precond),
                       precond_sigma, int(forcing), int(gmres_aug), float(tau))
    s = fv_newton_stats()
    st = lib.newton_steady(g.handle, _f64(U, g.n_vel, "U"), _f64(P, g.n_cell, "P"),
                           ctypes.byref(o), ctypes.byref(s))
    out = {"status": st, "iterations": s.iterations, "gmres_total": s.gmres_total,
           "bicgstab_total": s.bicgstab_total,
           "res_hist": list(s.res_hist[:min(s.iterations + 1, 64)]), "res_final": s.res_final,
           "lin_hist": list(s.lin_hist[:min(s.iterations, 64)])}
    if raise_on_fail:
        check(st, "newton_steady")
    return out


def arnoldi_leading(g, U, v0, m=30, nev=5, evec=None, tol=1e-10, max_restarts=5000,
                    prec="fp64", sigma=10.0, simple_eps=1e-10):
    lr = (ctypes.c_double * nev)()
    li = (ctypes.c_double * nev)()
    o = fv_arnoldi_opts(tol, max_restarts, PRECS.get(prec, prec), sigma, simple_eps)
    s = fv_arnoldi_stats()
    check(lib.arnoldi_leading(g.handle, _f64(U, g.n_vel, "U"), _f64(v0, g.n_vel, "v0"), m, nev,
                              lr, li, None if evec is None else _f64(evec, 2 * g.n_vel, "evec"),
                              ctypes.byref(o), ctypes.byref(s)), "arnoldi_leading")
    lam = [complex(lr[i], li[i]) for i in range(nev)]
    return lam, {"restarts": s.restarts, "matvecs": s.matvecs,
                 "ritz_resid": list(s.ritz_resid[:nev])}


class fv_critical_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("m", ctypes.c_int),
                ("nev", ctypes.c_int), ("prec", ctypes.c_int), ("newton_tol", ctypes.c_double),
                ("arnoldi_tol", ctypes.c_double), ("precond", ctypes.c_int),
                ("precond_sigma", ctypes.c_double), ("forcing", ctypes.c_int),
                ("max_restarts", ctypes.c_int), ("tau", ctypes.c_double), ("max_newton", ctypes.c_int)]


class fv_critical_stats(ctypes.Structure):
    _fields_ = [("evaluations", ctypes.c_int), ("re_hist", ctypes.c_double * 64),
                ("sigma_hist", ctypes.c_double * 64), ("omega_hist", ctypes.c_double * 64)]


def fv_critical_re(g, U, P, v0, re0, re1, rtol=1e-8, max_iter=30, m=30, nev=4, prec="fp64",
                   newton_tol=1e-10, arnoldi_tol=1e-10, precond=0, precond_sigma=0.0, forcing=0,
                   max_restarts=0, tau=0.0, max_newton=0):
    """Secant search of Re_cr (Section 3); returns (re_cr, omega_cr, history)."""
    o = fv_critical_opts(rtol, max_iter, m, nev, PRECS.get(prec, prec), newton_tol, arnoldi_tol,
                         int(precond), precond_sigma, int(forcing), int(max_restarts), float(tau),
                         int(max_newton))
    s = fv_critical_stats()
    rc, om = ctypes.c_double(), ctypes.c_double()
    check(lib.fv_critical_re(g.handle, _f64(U, g.n_vel, "U"), _f64(P, g.n_cell, "P"),
                             _f64(v0, g.n_vel, "v0"), ctypes.c_double(re0), ctypes.c_double(re1),
                             ctypes.byref(o), ctypes.byref(rc), ctypes.byref(om), ctypes.byref(s)),
          "fv_critical_re")
    k = min(s.evaluations, 64)
    return rc.value, om.value, [(s.re_hist[i], s.sigma_hist[i], s.omega_hist[i]) for i in range(k)]


PLANES = {"xz": 0, "yz": 1, "xy": 2}


def fv_plane_projection(g, v, plane, vp, psi=None):
    """Divergence-free projection of v onto the coordinate planes `plane`
    ('xz', 'yz', 'xy') and its vector potential (Section 4, Eqs. 11-17)."""
    nz, ny, nx = g.shape
    pl = PLANES.get(plane, plane)
    if psi is not None:
        dims = [nx, ny, nz]
        a, c = {0: (0, 2), 1: (1, 2), 2: (0, 1)}[pl]
        dims[a] += 1
        dims[c] += 1
        npsi = dims[0] * dims[1] * dims[2]
    check(lib.fv_plane_projection(g.handle, _f64(v, g.n_vel, "v"), pl, _f64(vp, g.n_vel, "vp"),
                                  None if psi is None else _f64(psi, npsi, "psi")),
          "fv_plane_projection")


def fv_dot_w(g, a, b):
    out = ctypes.c_double()
    check(lib.fv_dot_w(g.handle, _f64(a, g.n_vel, "a"), _f64(b, g.n_vel, "b"), ctypes.byref(out)),
          "fv_dot_w")
    return out.value


def fv_pressure_solve(g, r, phi, prec="fp64"):
    check(lib.fv_pressure_solve(g.handle, _f64(r, g.n_cell, "r"), _f64(phi, g.n_cell, "phi"),
                                PRECS.get(prec, prec)), "fv_pressure_solve")


class fv_mg_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("nu", ctypes.c_int),
                ("omega", ctypes.c_double)]


class fv_mg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("levels", ctypes.c_int), ("rel_res", ctypes.c_double)]


def fv_pressure_solve_mg(g, r, phi, guess=None, rtol=1e-10, max_iter=100, nu=1, omega=1.0,
                         raise_on_fail=True):
    """Multigrid-preconditioned CG pressure-correction solve (see include/fvns.h).
    Returns the stats as a dict (status included)."""
    o = fv_mg_opts(rtol, max_iter, nu, omega)
    st = fv_mg_stats()
    s = lib.fv_pressure_solve_mg(g.handle, _f64(r, g.n_cell, "r"), _f64(phi, g.n_cell, "phi"),
                                 None if guess is None else _f64(guess, g.n_cell, "guess"),
                                 ctypes.byref(o), ctypes.byref(st))
    if raise_on_fail:
        check(s, "fv_pressure_solve_mg")
    return {"status": s, "iterations": st.iterations, "levels": st.levels, "rel_res": st.rel_res}


def fv_pressure_solve_noalloc(shape, map, r, phi, stream=None):
    """Allocation-free float32 pressure-correction solve (see include/fvns.h)."""
    nz, ny, nx = shape
    n = nx * ny * nz
    st = _stream() if stream is None else ctypes.c_void_p(stream)
    check(lib.fv_pressure_solve_noalloc(nx, ny, nz, MAPS[map] if isinstance(map, str) else int(map),
                                        _f64(r, n, "r"), _f64(phi, n, "phi"), st),
          "fv_pressure_solve_noalloc")


KERNEL_KINDS = ["momentum", "divergence", "correct", "tpf_x", "tpf_yz", "dots", "vector", "tpf_xinv",
                "mg_smooth", "mg_other"]


def fv_profile_enable(g, on=True):
    check(lib.fv_profile_enable(g.handle, 1 if on else 0), "fv_profile_enable")


def fv_profile_read(g):
    ms = (ctypes.c_double * len(KERNEL_KINDS))()
    n = (ctypes.c_int64 * len(KERNEL_KINDS))()
    check(lib.fv_profile_read(g.handle, ms, n), "fv_profile_read")
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}


def fv_launch_count():
    return int(lib.fv_launch_count())


def fv_debug_inject_status(g, status):
    """Set the grid's device timeout word as an expired tensor-core wait does."""
    check(lib.fv_debug_inject_status(g.handle, int(status)), "fv_debug_inject_status")


def fv_bench_kernel(g, kind, reps=50):
    """Mean device time (ms) of one launch of a mixed-path kernel class."""
    ms = ctypes.c_double()
    check(lib.fv_bench_kernel(g.handle, KERNEL_KINDS.index(kind), reps, ctypes.byref(ms)),
          "fv_bench_kernel")
    return ms.value


class Batch:
    """Several grids advancing one Krylov-vector evaluation each per graph
    launch (fv_batch_* in include/fvns.h)."""

    def __init__(self, grids, stream=None):
        arr = (ctypes.c_void_p * len(grids))(*[g.handle.value for g in grids])
        h = ctypes.c_void_p()
        st = _stream() if stream is None else ctypes.c_void_p(stream)
        check(lib.fv_batch_create(len(grids), arr, st, ctypes.byref(h)), "fv_batch_create")
        self.handle, self.grids = h, list(grids)

    def krylov(self, U, x, out, eps=1e-8, sigma=0.0, sync=True):
        n = len(self.grids)
        pu = (ctypes.c_void_p * n)(*[_f64(U[i], self.grids[i].n_vel, "U").value for i in range(n)])
        px = (ctypes.c_void_p * n)(*[_f64(x[i], self.grids[i].n_vel, "x").value for i in range(n)])
        po = (ctypes.c_void_p * n)(*[_f64(out[i], self.grids[i].n_vel, "out").value for i in range(n)])
        passes = (ctypes.c_int * n)() if sync else None
        check(lib.fv_batch_krylov(self.handle, pu, px, po, ctypes.c_double(eps), ctypes.c_double(sigma),
                                  passes), "fv_batch_krylov")
        return list(passes) if sync else None

    def autotune(self, cache=None):
        """Pick the z-planes per work item of the batched momentum kernel:
        from the JSON cache when this batch shape was tuned before, else by
        timing the candidates (fv_batch_autotune) and recording the winner."""
        import json
        path = cache or os.environ.get("FVNS_AUTOTUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "fvns_autotune.json")
        key = "k_batch_jv|" + ";".join(f"{g.shape}|{g.re}" for g in self.grids)
        try:
            table = json.load(open(path))
        except (OSError, ValueError):
            table = {}
        if key in table:
            check(lib.fv_batch_set_tile(self.handle, int(table[key]["planes"])), "fv_batch_set_tile")
            return table[key]
        best = ctypes.c_int()
        ms = (ctypes.c_double * 4)()
        check(lib.fv_batch_autotune(self.handle, ctypes.byref(best), ms), "fv_batch_autotune")
        entry = {"planes": best.value, "ms": {str(p): ms[i] for i, p in enumerate((1, 2, 4, 8))}}
        table[key] = entry
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(table, open(path, "w"), indent=1)
        except OSError:
            pass
        return entry

    def close(self):
        if getattr(self, "handle", None):
            lib.fv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ns_divergence(g, v, r):
    """r = D v (Section 3 step 1), float64 device tensors."""
    check(lib.ns_divergence(g.handle, _f64(v, g.n_vel, "v"), _f64(r, g.n_cell, "r")),
          "ns_divergence")


def _f32(t, n, name):
    import torch
    if t.dtype != torch.float32 or t.numel() != n:
        raise ValueError(f"{name}: expected {n} float32 values, got {t.numel()} {t.dtype}")
    return _ptr(t)


class UNet:
    """Owner of an fv_unet handle: the learned guess of the pressure
    correction (3-D conv U-Net, BF16 tensor-core kernels)."""

    def __init__(self, seed=0, stream=None):
        h = ctypes.c_void_p()
        st = _stream() if stream is None else ctypes.c_void_p(stream)
        check(lib.fv_unet_create(seed, st, ctypes.byref(h)), "fv_unet_create")
        self.handle = h
        self.n_param = lib.fv_unet_param_count(h)

    def set_stream(self, stream):
        check(lib.fv_unet_set_stream(self.handle, ctypes.c_void_p(stream)), "fv_unet_set_stream")

    def set_params(self, params):
        check(lib.fv_unet_set_params(self.handle, _f32(params, self.n_param, "params")),
              "fv_unet_set_params")

    def get_params(self, params=None, grads=None):
        check(lib.fv_unet_get_params(
            self.handle, None if params is None else _f32(params, self.n_param, "params"),
            None if grads is None else _f32(grads, self.n_param, "grads")), "fv_unet_get_params")

    def forward(self, shape, planes, out):
        nx, ny, nz = shape
        n = nx * ny * nz
        check(lib.fv_unet_forward(self.handle, nx, ny, nz, _f32(planes, 4 * n, "planes"),
                                  _f32(out, n, "out")), "fv_unet_forward")

    def backward(self, target):
        loss = ctypes.c_double()
        check(lib.fv_unet_backward(self.handle, _f32(target, target.numel(), "target"),
                                   ctypes.byref(loss)), "fv_unet_backward")
        return loss.value

    def adam(self, lr):
        check(lib.fv_unet_adam(self.handle, lr), "fv_unet_adam")

    def guess(self, g, r, phi):
        check(lib.fv_unet_guess(self.handle, g.handle, _f64(r, g.n_cell, "r"),
                                _f64(phi, g.n_cell, "phi")), "fv_unet_guess")

    def train_step(self, g, r, phi, lr):
        loss = ctypes.c_double()
        check(lib.fv_unet_train_step(self.handle, g.handle, _f64(r, g.n_cell, "r"),
                                     _f64(phi, g.n_cell, "phi"), lr, ctypes.byref(loss)),
              "fv_unet_train_step")
        return loss.value

    def close(self):
        if getattr(self, "handle", None):
            lib.fv_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simple_krylov_solve_guess(g, net, U, v_in, v_out, p_out=None, eps=1e-8, max_pass=200,
                              prec="mixed", omega=1.0, sigma=0.0):
    """simple_krylov_solve whose first pass takes phi from the network."""
    o = fv_simple_opts(eps, max_pass, PRECS.get(prec, prec), omega, sigma, 0)
    s = fv_simple_stats()
    check(lib.simple_krylov_solve_guess(g.handle, net.handle, _f64(U, g.n_vel, "U"),
                                        _f64(v_in, g.n_vel, "v_in"), _f64(v_out, g.n_vel, "v_out"),
                                        None if p_out is None else _f64(p_out, g.n_cell, "p_out"),
                                        ctypes.byref(o), ctypes.byref(s)),
          "simple_krylov_solve_guess")
    return {"passes": s.passes, "phi_first": s.phi_first, "phi_last": s.phi_last,
            "div_max": s.div_max}
