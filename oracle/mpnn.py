"""FP64 reference of the warm-start network -- TEST INFRASTRUCTURE ONLY.

Plain torch FP64 CPU tensors, the same architecture and parameter layout as the library's
gn_mpnn_* kernels (include/gn.h): features [log w, log(1+deg), mean and max of log w over the
neighbours], three layers h' = relu(W_s h + W_n mean_{N(i)} h + b), a sigmoid head, the mean
BCE-with-logits loss.  Gradients by torch autograd.  `bf16=True` rounds the weights to bf16
first, as the GPU kernels do.  Pinned by central finite differences (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

F, H, L = 4, 64, 3


def layer_shapes():
    shapes = []
    din = F
    for _ in range(L):
        shapes += [(H, din), (H, din), (H,)]
        din = H
    shapes += [(H,), (1,)]
    return shapes


def num_params():
    return int(sum(np.prod(s) for s in layer_shapes()))


def unpack(theta):
    out, o = [], 0
    for s in layer_shapes():
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def features(row_ptr, col_idx, w):
    rp = np.asarray(row_ptr, np.int64)
    n = len(rp) - 1
    lw = np.log(np.asarray(w, np.float64))
    deg = np.diff(rp)
    f = np.zeros((n, F))
    f[:, 0] = lw
    f[:, 1] = np.log1p(deg)
    for i in range(n):
        nb = col_idx[rp[i]:rp[i + 1]]
        if len(nb):
            f[i, 2] = lw[nb].mean()
            f[i, 3] = lw[nb].max()
    return f


def forward(row_ptr, col_idx, w, theta, target=None, bf16=True):
    """Returns (p, loss or None, grad of the loss w.r.t. theta or None)."""
    import torch
    rp = np.asarray(row_ptr, np.int64)
    n = len(rp) - 1
    deg = torch.tensor(np.diff(rp), dtype=torch.float64)
    rows = torch.from_numpy(np.repeat(np.arange(n), np.diff(rp)))
    cols = torch.from_numpy(np.asarray(col_idx, np.int64))
    th = torch.tensor(np.asarray(theta, np.float32))
    if bf16:
        th = th.to(torch.bfloat16)
    th = th.to(torch.float64).requires_grad_(target is not None)
    o = 0
    params = []
    for s in layer_shapes():
        k = int(np.prod(s))
        params.append(th[o:o + k].reshape(s))
        o += k
    h = torch.tensor(features(row_ptr, col_idx, w))
    for l in range(L):
        Ws, Wn, b = params[3 * l: 3 * l + 3]
        msum = torch.zeros_like(h).index_add(0, rows, h[cols])
        m = torch.where(deg[:, None] > 0, msum / torch.clamp(deg, min=1)[:, None], torch.zeros_like(msum))
        h = torch.relu(h @ Ws.T + m @ Wn.T + b)
    q = h @ params[-2] + params[-1]
    p = torch.sigmoid(q)
    if target is None:
        return p.detach().numpy(), None, None
    t = torch.tensor(np.asarray(target, np.float64))
    loss = torch.nn.functional.binary_cross_entropy_with_logits(q, t)
    loss.backward()
    return p.detach().numpy(), float(loss.item()), th.grad.numpy().copy()
