"""GPU parity of the learned pressure guess (3-D conv U-Net on the BF16
tensor cores) against the float64 oracle with BF16 storage emulated at the
same points, plus its use as the first pass of the SIMPLE loop.

Tolerances (relative L2 norm of the difference).  BF16 storage makes the
network sensitive to rounding decisions: perturbing every convolution sum
of the emulating oracle by a relative 3e-7 (float32 accumulation) flips a
few BF16 roundings and ReLU decisions and moves its output by 1.3e-5,
2.4e-3 and 2.8e-3 on the three grids below and single layer gradients by
up to 8e-2 (1e-6: up to 0.17); one such draw reproduces the device's 8^3
loss to 7 digits.  A wrong tap, index, sign or missing term moves them by
0.3 to 1.  So:
  forward output              5e-3
  gradients, per layer        0.2,  all parameters together 5e-2
  Krylov vector with guess    2e-6 of the plain mixed-precision vector:
                              both loops stop at eps = 1e-8 relative to the
                              exact correction and run the same float32
                              exact passes; the difference is the stop
                              point (the mixed form's parity tolerance
                              against the oracle is 2e-5)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import unet as ou  # noqa: E402


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def _params(seed):
    rng = np.random.default_rng(seed)
    p = ou.init_params(seed)
    wo, bo, hw, hb, n = ou.layout()
    for c, (_, _, co) in enumerate(ou.CONVS):
        p[bo[c]:bo[c] + co] = 0.05 * rng.standard_normal(co)
    p[hb] = 0.1
    return p.astype(np.float32).astype(np.float64)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _net(fv, p):
    net = fv.UNet(seed=0)
    net.set_params(torch.tensor(p, dtype=torch.float32, device="cuda"))
    return net


SHAPES = [(8, 8, 8), (24, 16, 8), (16, 32, 24)]   # (nx, ny, nz)
FWD_TOL = 5e-3
GRAD_TOL = 0.2
GRAD_TOL_ALL = 5e-2


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(fv, shape):
    nx, ny, nz = shape
    p = _params(3)
    planes = np.random.default_rng(4).standard_normal((4, nz, ny, nx)).astype(np.float32).astype(np.float64)
    net = _net(fv, p)
    out = torch.empty(nx * ny * nz, dtype=torch.float32, device="cuda")
    net.forward(shape, torch.tensor(planes.ravel(), dtype=torch.float32, device="cuda"), out)
    torch.cuda.synchronize()
    ref, _ = ou.forward(p, planes, emulate=True)
    exact, _ = ou.forward(p, planes, emulate=False)
    got = out.cpu().numpy().reshape(nz, ny, nx)
    e_emu, e_exact = _rel(got, ref), _rel(got, exact)
    print(f"\nforward {shape}: vs emulated {e_emu:.2e}, vs float64 {e_exact:.2e}, "
          f"emulated vs float64 {_rel(ref, exact):.2e}")
    assert e_emu <= FWD_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_gradients_match_oracle(fv, shape):
    nx, ny, nz = shape
    p = _params(5)
    rng = np.random.default_rng(6)
    planes = rng.standard_normal((4, nz, ny, nx)).astype(np.float32).astype(np.float64)
    target = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
    net = _net(fv, p)
    n = nx * ny * nz
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    net.forward(shape, torch.tensor(planes.ravel(), dtype=torch.float32, device="cuda"), out)
    loss = net.backward(torch.tensor(target.ravel(), dtype=torch.float32, device="cuda"))
    grads = torch.empty(net.n_param, dtype=torch.float32, device="cuda")
    net.get_params(grads=grads)
    torch.cuda.synchronize()
    g = grads.cpu().numpy().astype(np.float64)
    ref_loss, ref_g, _ = ou.loss_and_grad(p, planes, target, emulate=True)
    _, exact_g, _ = ou.loss_and_grad(p, planes, target, emulate=False)
    wo, bo, hw, hb, npar = ou.layout()
    errs = {"head": _rel(g[hw:hw + 16], ref_g[hw:hw + 16])}
    for c, (_, ci, co) in enumerate(ou.CONVS):
        errs[f"W{c}"] = _rel(g[wo[c]:wo[c] + 27 * ci * co], ref_g[wo[c]:wo[c] + 27 * ci * co])
        errs[f"b{c}"] = _rel(g[bo[c]:bo[c] + co], ref_g[bo[c]:bo[c] + co])
    e_ex = max(_rel(g[wo[c]:wo[c] + 27 * ci * co], exact_g[wo[c]:wo[c] + 27 * ci * co])
               for c, (_, ci, co) in enumerate(ou.CONVS))
    print(f"\ngradients {shape}: loss {loss:.6e} vs {ref_loss:.6e}; worst vs emulated "
          f"{max(errs.values()):.2e} ({max(errs, key=errs.get)}); worst W vs float64 {e_ex:.2e}")
    total = _rel(g, ref_g)
    print(f"gradients {shape}: all parameters {total:.2e}")
    assert abs(loss - ref_loss) <= FWD_TOL * ref_loss
    assert total <= GRAD_TOL_ALL
    for k, e in errs.items():
        assert e <= GRAD_TOL, (k, e)


def test_adam_step_matches_definition(fv):
    p = _params(7)
    net = _net(fv, p)
    shape = (8, 8, 8)
    planes = torch.randn(4 * 512, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    out = torch.empty(512, dtype=torch.float32, device="cuda")
    net.forward(shape, planes, out)
    net.backward(torch.zeros(512, dtype=torch.float32, device="cuda"))
    g = torch.empty(net.n_param, dtype=torch.float32, device="cuda")
    net.get_params(grads=g)
    net.adam(1e-3)
    q = torch.empty(net.n_param, dtype=torch.float32, device="cuda")
    net.get_params(params=q)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    # first Adam step: m_hat = g, v_hat = g^2 -> p - lr g / (|g| + 1e-8)
    expect = p - 1e-3 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(q.cpu().numpy(), expect, rtol=0, atol=2e-6)


def test_invalid_arguments(fv):
    net = fv.UNet(seed=0)
    x = torch.zeros(4 * 12 * 8 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(12 * 8 * 8, dtype=torch.float32, device="cuda")
    with pytest.raises(fv.FvError):
        net.forward((12, 8, 8), x, out)          # 12 is not a multiple of 8
    with pytest.raises(fv.FvError):
        net.adam(0.0)
    net2 = fv.UNet(seed=0)
    with pytest.raises(fv.FvError):
        net2.backward(out)                        # no forward pass yet


def _pair(fv, g, U, seed):
    """(r, phi) of one Gaussian Krylov direction: w = L_U v, r = D w, phi = (DG)^+ r."""
    v = torch.tensor(synth.gaussian_velocity(g.shape, seed), device="cuda")
    w = torch.empty_like(v)
    fv.ns_jacvec(g, U, v, w, prec="fp64")
    r = torch.empty(g.n_cell, dtype=torch.float64, device="cuda")
    fv.ns_divergence(g, w, r)
    phi = torch.empty_like(r)
    fv.fv_pressure_solve(g, r, phi, prec="fp64")
    return v, r, phi


def test_training_reduces_loss_and_guess_keeps_the_krylov_vector(fv):
    shape = (32, 32, 32)
    g = fv.Grid(*shape, map="cosine", alpha=0.0, re=1900.0)
    U = torch.tensor(synth.vortex_base_flow(shape[::-1], "cosine", 0.0), device="cuda")
    net = fv.UNet(seed=11)
    pairs = [_pair(fv, g, U, 100 + s) for s in range(8)]
    losses = []
    for step in range(240):
        _, r, phi = pairs[step % len(pairs)]
        losses.append(net.train_step(g, r, phi, 2e-3 if step < 160 else 5e-4))
    first, last = np.mean(losses[:8]), np.mean(losses[-8:])
    assert last < 0.5 * first, (first, last)

    # a held-out direction: the guess is an approximation of phi ...
    v, r, phi = _pair(fv, g, U, 999)
    guess = torch.empty_like(phi)
    net.guess(g, r, guess)
    torch.cuda.synchronize()
    gs, ph = guess.cpu().numpy(), phi.cpu().numpy()
    err = _rel(gs - gs.mean(), ph - ph.mean())
    assert np.isfinite(err)
    # ... and the loop started from it reaches the same Krylov vector
    out_plain = torch.empty_like(v)
    out_guess = torch.empty_like(v)
    st_plain = fv.simple_krylov_solve(g, U, v, out_plain, eps=1e-8, prec="mixed")
    st_guess = fv.simple_krylov_solve_guess(g, net, U, v, out_guess, eps=1e-8, prec="mixed")
    a, b = out_guess.cpu().numpy(), out_plain.cpu().numpy()
    assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max()
    assert st_guess["passes"] >= 2
    # FV_FF form as well
    st_ff = fv.simple_krylov_solve_guess(g, net, U, v, out_guess, eps=1e-8, prec="ff")
    fv.simple_krylov_solve(g, U, v, out_plain, eps=1e-8, prec="ff")
    a, b = out_guess.cpu().numpy(), out_plain.cpu().numpy()
    assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max()
    print(f"\nU-Net 32^3: loss {first:.3e} -> {last:.3e}; held-out guess error {err:.3f}; "
          f"passes plain {st_plain['passes']} / guess {st_guess['passes']} (ff {st_ff['passes']})")
