"""FP64 reference of the convolutional post-correction of the sweep (oracle; test infrastructure only).

The paper has no learned component.  This restates the small network the
GPU path uses as a flexible-GMRES post-correction of the sweep output
x = M_alpha r:  z = x + s N(x / s):

* s = rms(x) = sqrt(mean over points of |x|^2) per right-hand side (N sees a
  unit-scale input, and scaling r scales the correction: the preconditioner
  stays positively homogeneous);
* the input image has two channels (Re x / s, Im x / s) on the n x n grid,
  rows x2, columns x1;
* N = conv3x3(2 -> 32) + bias, ReLU, conv3x3(32 -> 32) + bias, ReLU,
  conv3x3(32 -> 2) + bias; "same" size with zero padding; the output's two
  channels are the real and imaginary parts of the correction;
* the training loss of pairs (x_k, e_k), e_k = A^{-1} r_k - M_alpha r_k the
  error of the sweep, is the mean over points and right-hand sides of
  |N(x_k/s_k) - e_k/s_k|^2;
* Adam (Kingma & Ba 2015) with bias correction updates the parameters.

Parameter vector (float, this order): W1[3][3][2][32], b1[32],
W2[3][3][32][32], b2[32], W3[3][3][32][2], b3[2]; W[dy+1][dx+1][ci][co]
multiplies input channel ci at offset (dy, dx) (rows, columns) for output
channel co (cross-correlation, as in every deep-learning convolution).

Everything is plain NumPy in float64.  ``bf16=True`` rounds the weights and
each layer's stored activations to bfloat16 (round to nearest even), the
storage precision of the GPU kernels, so that the two can be compared
element by element; the arithmetic stays float64.

A second loss, the one the solver's judge measures, fits the correction in
the residual norm: for rho = v - A x, mean over pairs of |A c - rho|^2 / |rho|^2.

Pins: the convolution against ``scipy.signal.correlate2d``, both gradients
against central finite differences (FP64), the first Adam step against its
closed form (every parameter moves by lr in the direction -sign(g)).
"""
import numpy as np

CH = 32
SHAPES = [("W1", (3, 3, 2, CH)), ("b1", (CH,)), ("W2", (3, 3, CH, CH)), ("b2", (CH,)),
          ("W3", (3, 3, CH, 2)), ("b3", (2,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Split the flat parameter vector into a dict of arrays (views)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def to_bf16(x):
    """Round float64 values to bfloat16 (via float32, round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, W, b):
    """y[i, j, co] = b[co] + sum_{dy, dx, ci} W[dy+1, dx+1, ci, co] x[i+dy, j+dx, ci], zero padding.

    x: (H, Wd, Cin), W: (3, 3, Cin, Cout), b: (Cout,)."""
    H, Wd, _ = x.shape
    xp = np.zeros((H + 2, Wd + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    y = np.broadcast_to(b, (H, Wd, W.shape[3])).copy()
    for dy in range(3):
        for dx in range(3):
            y += xp[dy:dy + H, dx:dx + Wd] @ W[dy, dx]
    return y


def conv3x3_backward(x, W, dy_):
    """Gradients of sum(dy_ * conv3x3(x, W, b)) w.r.t. x, W and b."""
    H, Wd, _ = x.shape
    xp = np.zeros((H + 2, Wd + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            win = xp[ky:ky + H, kx:kx + Wd]
            dW[ky, kx] = np.tensordot(win, dy_, axes=([0, 1], [0, 1]))
            dxp[ky:ky + H, kx:kx + Wd] += dy_ @ W[ky, kx].T
    return dxp[1:-1, 1:-1], dW, dy_.sum(axis=(0, 1))


def rms(r):
    r = np.asarray(r)
    return float(np.sqrt(np.mean(np.abs(r) ** 2)))


def image(r, s):
    """Two-channel unit-scale image of one complex field (n2, n1)."""
    return np.stack([r.real / s, r.imag / s], axis=-1)


def forward(theta, x, bf16=False):
    """Network output (H, W, 2) and the stored activations."""
    p = unpack(theta)
    q = (lambda a: to_bf16(a)) if bf16 else (lambda a: a)
    W1, W2, W3 = q(p["W1"]), q(p["W2"]), q(p["W3"])
    x = q(x)
    a1 = conv3x3(x, W1, p["b1"])
    h1 = q(np.maximum(a1, 0.0))
    a2 = conv3x3(h1, W2, p["b2"])
    h2 = q(np.maximum(a2, 0.0))
    o = conv3x3(h2, W3, p["b3"])
    return o, dict(x=x, h1=h1, h2=h2, W1=W1, W2=W2, W3=W3)


def correction(theta, r, bf16=False):
    """s N(r / s), s = rms(r), as a complex field (zero when r = 0); r is the sweep output."""
    s = rms(r)
    if s == 0.0:
        return np.zeros_like(np.asarray(r, dtype=np.complex128))
    o, _ = forward(theta, image(np.asarray(r, dtype=np.complex128), s), bf16)
    return s * (o[..., 0] + 1j * o[..., 1])


def loss_and_grad(theta, rs, es, bf16=False):
    """Mean squared error of N(r/s) against e/s over all points and pairs, and its gradient."""
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    L, npts = 0.0, 0
    for r, e in zip(rs, es):
        s = rms(r)
        o, c = forward(theta, image(r, s), bf16)
        t = image(e, s)
        d = o - t
        L += float(np.sum(d * d))
        npts += d.shape[0] * d.shape[1]
        do = 2.0 * d
        dh2, gW3, gb3 = conv3x3_backward(c["h2"], c["W3"], do)
        da2 = dh2 * (c["h2"] > 0)
        dh1, gW2, gb2 = conv3x3_backward(c["h1"], c["W2"], da2)
        da1 = dh1 * (c["h1"] > 0)
        _, gW1, gb1 = conv3x3_backward(c["x"], c["W1"], da1)
        for name, v in (("W1", gW1), ("b1", gb1), ("W2", gW2), ("b2", gb2), ("W3", gW3), ("b3", gb3)):
            g[name] += v
    return L / npts, pack(g) / npts


def residual_loss_and_grad(theta, xs, rhos, apply_A, bf16=False):
    """L = mean over pairs of |A c - rho|^2 / |rho|^2 with c = s N(x/s),
    s = rms(x), and its gradient (A complex symmetric: dL/dc = 2 conj(A conj(d))
    / (|rho|^2 R) for d = A c - rho; dL/do = s (Re, Im) of that)."""
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    L, R = 0.0, len(xs)
    for x, rho in zip(xs, rhos):
        s = rms(x)
        o, c = forward(theta, image(x, s), bf16)
        corr = s * (o[..., 0] + 1j * o[..., 1])
        d = apply_A(corr) - rho
        nr = float(np.sum(np.abs(rho) ** 2))
        L += float(np.sum(np.abs(d) ** 2)) / nr / R
        G = 2.0 * np.conj(apply_A(np.conj(d))) / (nr * R)
        do = s * np.stack([G.real, G.imag], axis=-1)
        dh2, gW3, gb3 = conv3x3_backward(c["h2"], c["W3"], do)
        da2 = dh2 * (c["h2"] > 0)
        dh1, gW2, gb2 = conv3x3_backward(c["h1"], c["W2"], da2)
        da1 = dh1 * (c["h1"] > 0)
        _, gW1, gb1 = conv3x3_backward(c["x"], c["W1"], da1)
        for name, v in (("W1", gW1), ("b1", gb1), ("W2", gW2), ("b2", gb2), ("W3", gW3), ("b3", gb3)):
            g[name] += v
    return L, pack(g)


class Adam:
    """Adam with bias correction (Kingma & Ba 2015, Algorithm 1)."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
