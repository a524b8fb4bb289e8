"""FP64 reference gradients of unrolled GN -- TEST INFRASTRUCTURE ONLY.

The forward is Def. WRGN written in the paper's x-space with torch FP64 CPU tensors:
    x_i <- x_i / (x_i + gamma_t * sum_{j in N(i)} (v_j / v_i) x_j),  v = sqrt(w),
with the appendix module's safe division (x_i = 1/2 where (B y)_i = v_i * denominator <= 1e-9)
and the gamma schedule of Sec. 6.  Gradients come from torch autograd (a library primitive).
Pinned against central finite differences in FP64 (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np


def gammas(T, k0=0, mode=0, gamma0=0.9, gamma1=1.5, ramp=1000):
    out = []
    for k in range(k0, k0 + T):
        if mode == 1 or ramp <= 1:
            out.append(gamma1)
        else:
            t = min(k, ramp - 1) / (ramp - 1)
            out.append(t * gamma1 + (1.0 - t) * gamma0)
    return out


def unrolled(row_ptr, col_idx, w, x0, gam):
    """x_T of len(gam) WRGN steps (torch FP64 tensors; w and x0 may require grad)."""
    import torch
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    rows = torch.from_numpy(np.repeat(np.arange(n), np.diff(rp)))
    cols = torch.from_numpy(np.asarray(col_idx, dtype=np.int64))
    v = torch.sqrt(w)
    x = x0
    for g in gam:
        nb = torch.zeros(n, dtype=torch.float64).index_add(0, rows, (v[cols] / v[rows]) * x[cols])
        d = x + g * nb
        ok = v * d > 1e-9
        x = torch.where(ok, x / torch.where(ok, d, torch.ones_like(d)), torch.full_like(d, 0.5))
    return x


def loss_and_grads(row_ptr, col_idx, w, x0, gvec, gam):
    """L = g . x_T and (dL/dw, dL/dx0) in FP64."""
    import torch
    wt = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    xt = torch.tensor(np.asarray(x0, dtype=np.float64), requires_grad=True)
    xT = unrolled(row_ptr, col_idx, wt, xt, gam)
    L = torch.dot(torch.tensor(np.asarray(gvec, dtype=np.float64)), xT)
    L.backward()
    return float(L.item()), wt.grad.numpy().copy(), xt.grad.numpy().copy(), xT.detach().numpy().copy()
