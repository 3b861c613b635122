"""FP64 CPU reference of the bed surrogate's network (TEST INFRASTRUCTURE ONLY).

A plain numpy restatement of the 6-layer 3x3 convolutional network that the
tensor-core kernels run: conv3x3 with zero padding 1 written as im2col + a
matrix product, ReLU on hidden layers, a linear last convolution whose output
corrects the input's linear extrapolation inside the input's activity mask,
and the backward pass of the mean squared or absolute error loss by the chain rule.  Only tests may import this
module; it shares no code with the CUDA library.

Layout: images [H][W][C]; weights W[nout][9*cin] with k = tap*cin + c and
tap = (dy+1)*3 + (dx+1); the output pixel (y, x) reads input (y+dy, x+dx).
"""
import numpy as np

CINS = (8, 32, 32, 32, 32, 32)
NOUTS = (32, 32, 32, 32, 32, 1)


def im2col(X):
    """[H][W][C] -> [H*W][9*C] with the 9 zero-padded shifts (tap-major)."""
    H, W, C = X.shape
    P = np.zeros((H + 2, W + 2, C), dtype=np.float64)
    P[1:-1, 1:-1] = X
    cols = []
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        cols.append(P[1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :])
    return np.concatenate(cols, axis=2).reshape(H * W, 9 * C)


def conv3x3(X, Wm, b):
    H, W, _ = X.shape
    return (im2col(X) @ Wm.T + b).reshape(H, W, -1)


def forward(X, params, round_fn=None):
    """Returns the list of layer outputs (post-activation for hidden layers)
    and the output [H][W] = m (z + p), z the last convolution, p and m input
    channels 6 and 7 (the linear extrapolation and the activity mask).
    round_fn (optional) is applied to every stored activation, e.g. to
    emulate BF16 storage."""
    r = round_fn or (lambda a: a)
    acts = [r(X)]
    h = acts[0]
    for i, (Wm, b) in enumerate(params):
        z = conv3x3(h, Wm, b)
        if i < 5:
            h = r(np.maximum(z, 0.0))
            acts.append(h)
        else:
            out = acts[0][:, :, 7] * (z[:, :, 0] + acts[0][:, :, 6])
    return acts, out


def loss_and_grads(X, target, params, round_fn=None, loss="mse"):
    """Mean squared (loss="mse") or absolute ("l1", subgradient 0 at a zero
    residual) error over pixels and the gradients (dW, db) of every layer by
    back-propagation; dgrad of conv3x3 is the correlation of the output
    gradient with the spatially flipped, transposed kernel, here via im2col
    of the output gradient."""
    r = round_fn or (lambda a: a)
    acts, out = forward(X, params, round_fn)
    H, W = out.shape
    d = out - target
    if loss == "l1":
        value = float(np.mean(np.abs(d)))
        dl = np.sign(d) / (H * W)
    else:
        value = float(np.mean(d * d))
        dl = (2.0 / (H * W)) * d
    g = r(dl * acts[0][:, :, 7])[:, :, None]             # dL/dz through out = m (z + p)
    grads = [None] * 6
    for i in range(5, -1, -1):
        Wm, b = params[i]
        xin = acts[i]
        cols = im2col(xin)
        dW = g.reshape(H * W, -1).T @ cols                   # [nout][9*cin]
        db = g.reshape(H * W, -1).sum(axis=0)
        grads[i] = (dW, db)
        if i == 0:
            break
        cin = xin.shape[2]
        # dX[y][x][c] = sum_{tap,n} g[y-dy][x-dx][n] W[n][tap*cin + c]
        Wf = Wm.reshape(-1, 9, cin)[:, ::-1, :]              # flipped taps
        Wd = Wf.transpose(2, 1, 0).reshape(cin, -1)           # [cin][9*nout], k = tap*nout + n
        dX = (im2col(g) @ Wd.T).reshape(H, W, cin)
        g = r(dX * (xin > 0))                                 # through the ReLU of layer i-1
    return value, grads, out


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    ps = []
    for i, (cin, nout) in enumerate(zip(CINS, NOUTS)):
        fan = 9 * cin
        Wm = rng.normal(0, scale * np.sqrt(2.0 / fan), (nout, 9 * cin))
        b = rng.normal(0, 0.1, nout)
        ps.append((Wm, b))
    return ps
