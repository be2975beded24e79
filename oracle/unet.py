"""3-D convolutional U-Net of the learned pressure guess -- oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.

The learned guess has no counterpart in the paper: Section 3's loop starts
every Krylov-vector evaluation from phi = 0 and an exact pressure solve.
The network maps the right-hand side r = D w of the pressure equation
(Section 3 step 1) plus three metric channels to a guess of phi; the loop
then continues with exact passes, so the fixed point is the paper's.

This module is the plain float64 definition of that network: forward pass,
mean-free square loss and its gradient by the chain rule, written out layer
by layer with numpy.  Arrays are (nz, ny, nx, channels), cells x fastest,
the layout of the device activations.  With ``emulate=True`` every value the
device stores in BF16 (input, weights, activations, activation gradients)
is rounded to BF16 at the same points, so that a device result can be
compared with a tolerance set by float32 accumulation, not by BF16 storage.

Pins (tests/test_oracle_unet.py): the convolution against brute-force loops
and against scipy.signal.correlate; pooling / upsampling against their
adjoint identities; the whole gradient against central finite differences.
"""
import numpy as np

# (level, cin, cout) of the 14 convolutions: encoder 0a 0b 1a 1b 2a 2b,
# bottom a b, decoder 2a 2b 1a 1b 0a 0b (decoder a-inputs: [up, skip])
CONVS = [(0, 16, 16), (0, 16, 16), (1, 16, 32), (1, 32, 32), (2, 32, 48), (2, 48, 48),
         (3, 48, 64), (3, 64, 64), (2, 112, 48), (2, 48, 48), (1, 80, 32), (1, 32, 32),
         (0, 48, 16), (0, 16, 16)]


def layout():
    """Offsets of (W_c, b_c) per convolution, of the output weights and bias,
    and the total parameter count (float32 vector of the device)."""
    off = 0
    w, b = [], []
    for _, cin, cout in CONVS:
        w.append(off)
        off += 27 * cin * cout
        b.append(off)
        off += cout
    head_w = off
    head_b = off + 16
    return w, b, head_w, head_b, off + 17


def unpack(params):
    """Flat parameter vector -> ([W_c (27, cout, cin)], [b_c], w_head (16,), b_head)."""
    wo, bo, hw, hb, n = layout()
    p = np.asarray(params, dtype=np.float64)
    assert p.size == n
    Ws = [p[wo[c]:wo[c] + 27 * ci * co].reshape(27, co, ci) for c, (_, ci, co) in enumerate(CONVS)]
    bs = [p[bo[c]:bo[c] + co] for c, (_, _, co) in enumerate(CONVS)]
    return Ws, bs, p[hw:hw + 16], p[hb]


def bf16(x):
    """Round to the nearest BF16 value (ties to even), through float32."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def _shift(Xp, t, shape):
    """Neighbour values at tap t = 9(dz+1) + 3(dy+1) + (dx+1) from the
    zero-padded array Xp: out[k, j, i] = X[k+dz, j+dy, i+dx] (0 outside)."""
    dx, dy, dz = t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1
    nz, ny, nx = shape
    return Xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]


def conv3(X, W, b=None):
    """3x3x3 convolution with zero padding:
    Y[c, co] = b[co] + sum_t sum_ci X[nb(c, t), ci] W[t, co, ci]."""
    shape = X.shape[:3]
    Xp = np.pad(X, ((1, 1), (1, 1), (1, 1), (0, 0)))
    Y = np.zeros(shape + (W.shape[1],))
    for t in range(27):
        Y += _shift(Xp, t, shape) @ W[t].T
    if b is not None:
        Y += b
    return Y


def conv3_back(X, W, dY):
    """Gradients of conv3 for the output gradient dY: (dX, dW, db), dX by
    scattering each tap's contribution back to the neighbour it came from."""
    shape = X.shape[:3]
    Xp = np.pad(X, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dXp = np.zeros_like(Xp)
    dW = np.zeros_like(W)
    for t in range(27):
        dW[t] = np.einsum("zyxo,zyxi->oi", dY, _shift(Xp, t, shape))
        _shift(dXp, t, shape)[...] += dY @ W[t]
    return dXp[1:-1, 1:-1, 1:-1], dW, dY.sum(axis=(0, 1, 2))


def pool(X):
    """2x2x2 mean pooling."""
    nz, ny, nx, c = X.shape
    return X.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def up(X):
    """Nearest (piecewise-constant) upsampling by 2 along every axis."""
    return X.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def up_adjoint(dY):
    """Adjoint of up: the sum over each 2x2x2 block."""
    return 8.0 * pool(dY)


def forward(params, planes, emulate=False):
    """planes: (4, nz, ny, nx) input channels.  Returns (out (nz, ny, nx), cache)."""
    Ws, bs, hw, hb = unpack(params)
    r = bf16 if emulate else (lambda a: a)
    if emulate:
        Ws = [bf16(W) for W in Ws]
    nz, ny, nx = planes.shape[1:]
    X0 = np.zeros((nz, ny, nx, 16))
    X0[..., :4] = np.moveaxis(planes, 0, -1)
    X0 = r(X0)
    act, inputs, cats = [None] * 14, [None] * 14, [None] * 3
    X = X0
    for lev in range(4):
        for c in (2 * lev, 2 * lev + 1):
            inputs[c] = X
            act[c] = r(np.maximum(conv3(X, Ws[c], bs[c]), 0.0))
            X = act[c]
        if lev < 3:
            X = r(pool(X))
    low = act[7]
    for q in range(3):
        lev = 2 - q
        cats[q] = np.concatenate([up(low), act[2 * lev + 1]], axis=-1)
        X = cats[q]
        for c in (8 + 2 * q, 9 + 2 * q):
            inputs[c] = X
            act[c] = r(np.maximum(conv3(X, Ws[c], bs[c]), 0.0))
            X = act[c]
        low = X
    out = act[13] @ hw + hb
    return out, {"Ws": Ws, "hw": hw, "act": act, "inputs": inputs, "emulate": emulate}


def loss_and_grad(params, planes, target, emulate=False):
    """Mean-free square loss L = mean((e - mean e)^2), e = out - target, and
    dL/dparams (flat, the layout of ``layout``) by the chain rule."""
    out, cache = forward(params, planes, emulate)
    r = bf16 if emulate else (lambda a: a)
    Ws, hw, act, inputs = cache["Ws"], cache["hw"], cache["act"], cache["inputs"]
    n = out.size
    e = out - target
    e = e - e.mean()
    loss = float(np.mean(e * e))
    go = 2.0 * e / n
    wo, bo, hwo, hbo, npar = layout()
    grad = np.zeros(npar)
    grad[hwo:hwo + 16] = np.einsum("zyx,zyxk->k", go, act[13])
    grad[hbo] = go.sum()

    def layer_back(c, g):
        """g = dL/d act[c] -> dL/d input of layer c (and the parameter grads)."""
        g = g * (act[c] > 0)
        dX, dW, db = conv3_back(inputs[c], Ws[c], g)
        grad[wo[c]:wo[c] + dW.size] = dW.ravel()
        grad[bo[c]:bo[c] + db.size] = db
        return r(dX)

    g = r(go[..., None] * hw)
    skip_grads = [None] * 3
    for q in (2, 1, 0):
        lev = 2 - q
        g = layer_back(9 + 2 * q, g)
        dcat = layer_back(8 + 2 * q, g)
        lowc = CONVS[8 + 2 * q][1] - CONVS[2 * lev + 1][2]
        skip_grads[lev] = dcat[..., lowc:]
        g = r(up_adjoint(dcat[..., :lowc]))
    for lev in (3, 2, 1, 0):
        if lev < 3:
            g = r(skip_grads[lev] + up(g) / 8.0)
        g = layer_back(2 * lev + 1, g)
        g = layer_back(2 * lev, g)
    return loss, grad, out


def init_params(seed):
    """He-normal weights, zero biases, output weights N(0, 1/16) (seeded)."""
    rng = np.random.default_rng(seed)
    wo, bo, hw, hb, n = layout()
    p = np.zeros(n)
    for c, (_, cin, cout) in enumerate(CONVS):
        p[wo[c]:wo[c] + 27 * cin * cout] = rng.standard_normal(27 * cin * cout) * np.sqrt(2.0 / (27 * cin))
    p[hw:hw + 16] = 0.25 * rng.standard_normal(16)
    return p
