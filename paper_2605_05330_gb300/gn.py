"""Thin Python binding of libgn.so (include/gn.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream when tensors are passed; numpy arrays use the host I/O
mode of the C ABI.  Loading fails loudly when the library has not been built: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgn.so")

OK = 0
WARN_NOT_CONVERGED = 1
WARN_NOT_BINARY = 2
WARN_NOT_MAXIMAL = 3
STATUS = {0: "OK", 1: "WARN_NOT_CONVERGED", 2: "WARN_NOT_BINARY", 3: "WARN_NOT_MAXIMAL",
          -1: "ERR_ARG", -2: "ERR_NOT_SIMPLE", -3: "ERR_WEIGHT", -4: "ERR_NOT_NORMALIZABLE",
          -5: "ERR_CUDA", -6: "ERR_TIMEOUT", -7: "ERR_NOT_INDEPENDENT", -8: "ERR_NO_RECORD",
          -9: "ERR_TOO_LARGE"}
HOST, DEVICE = 0, 1
GAMMA_PURSUIT, GAMMA_FIXED = 0, 1
REORDER_NONE, REORDER_RCM, REORDER_DEGREE = 0, 1, 2
KERNEL_AUTO, KERNEL_PERSISTENT, KERNEL_CTA = 0, 1, 2
SYNC_AUTO, SYNC_GRID, SYNC_NEIGHBOUR, SYNC_TAGGED = 0, 1, 2, 3
GATHER_AUTO, GATHER_GLOBAL, GATHER_SMEM_CSR, GATHER_HALO = 0, 1, 2, 3
GATHER_HALO_PULL, GATHER_HALO_PUSH = 4, 5
EXCHANGE_NAMES = {0: "none", 1: "pull", 2: "push"}
GATHER_NAMES = {1: "global", 2: "smem_csr", 3: "halo"}


class GNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = STATUS.get(status, status)


class Params(ctypes.Structure):
    _fields_ = [("gamma_mode", ctypes.c_int), ("gamma0", ctypes.c_double), ("gamma1", ctypes.c_double),
                ("ramp_iters", ctypes.c_int), ("check_every", ctypes.c_int),
                ("theta_bin", ctypes.c_double), ("kernel", ctypes.c_int), ("record", ctypes.c_int),
                ("spin_limit", ctypes.c_longlong), ("debug_unreachable_barrier", ctypes.c_int),
                ("resume", ctypes.c_int), ("sync", ctypes.c_int)]


class CreateOpts(ctypes.Structure):
    _fields_ = [("reorder", ctypes.c_int), ("gather", ctypes.c_int)]


class RunInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("binary", ctypes.c_int),
                ("status", ctypes.c_int), ("resid_inf", ctypes.c_double), ("resid_l1", ctypes.c_double),
                ("objective", ctypes.c_double), ("energy", ctypes.c_double),
                ("safe_div_hits", ctypes.c_longlong), ("device_ms", ctypes.c_float),
                ("kernel", ctypes.c_int)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["status"] = STATUS.get(d["status"], d["status"])
        return d


_lib = None
P = ctypes.c_void_p


def lib():
    """Loads libgn.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2605_05330_gb300/build.py "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        L.gn_default_params.argtypes = [ctypes.POINTER(Params)]
        L.gn_default_params.restype = None
        L.gn_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, P, P, P, ctypes.c_int, ctypes.c_int, P]
        L.gn_create.restype = ctypes.c_int
        L.gn_create_ex.argtypes = [ctypes.POINTER(P), ctypes.c_int32, P, P, P, ctypes.c_int,
                                   ctypes.POINTER(CreateOpts), P]
        L.gn_create_ex.restype = ctypes.c_int
        L.gn_gather_mode.argtypes = [P]
        L.gn_gather_mode.restype = ctypes.c_int
        L.gn_halo_exchange.argtypes = [P]
        L.gn_halo_exchange.restype = ctypes.c_int
        L.gn_kernel_launches.argtypes = []
        L.gn_kernel_launches.restype = ctypes.c_int64
        L.gn_destroy.argtypes = [P]
        L.gn_destroy.restype = None
        L.gn_set_io.argtypes = [P, ctypes.c_int]
        L.gn_set_io.restype = ctypes.c_int
        L.gn_set_weights.argtypes = [P, P]
        L.gn_set_weights.restype = ctypes.c_int
        L.gn_num_vertices.argtypes = [P]
        L.gn_num_vertices.restype = ctypes.c_int32
        L.gn_num_entries.argtypes = [P]
        L.gn_num_entries.restype = ctypes.c_int64
        L.gn_vertex_order.argtypes = [P, P]
        L.gn_vertex_order.restype = ctypes.c_int
        L.gn_vertex_order_source.argtypes = [P]
        L.gn_vertex_order_source.restype = ctypes.c_int
        L.gn_run.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Params), ctypes.c_int, P,
                             ctypes.POINTER(RunInfo)]
        L.gn_run.restype = ctypes.c_int
        L.gn_extract_is.argtypes = [P, P, P, P, P, P]
        L.gn_extract_is.restype = ctypes.c_int
        L.gn_objective.argtypes = [P, P, ctypes.c_double, P, P]
        L.gn_objective.restype = ctypes.c_int
        L.gn_backward.argtypes = [P, P, P, P]
        L.gn_backward.restype = ctypes.c_int
        L.gn_last_error.argtypes = []
        L.gn_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def default_params(**kw) -> Params:
    p = Params()
    lib().gn_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _check(st, allow_warn=True):
    if st < 0 or (st > 0 and not allow_warn):
        raise GNError(st, lib().gn_last_error().decode())
    return STATUS[st]


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_of(t):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


class Graph:
    """A graph resident on the GPU (gn_create).  Pass numpy arrays (host I/O mode) or CUDA
    tensors (device I/O mode, current stream)."""

    def __init__(self, row_ptr, col_idx, w, reorder=REORDER_NONE, stream=None, gather=GATHER_AUTO):
        self._h = P()
        self.device_io = _is_torch(row_ptr) and row_ptr.is_cuda
        if self.device_io:
            import torch
            row_ptr = row_ptr.to(torch.int32).contiguous()
            col_idx = col_idx.to(torch.int32).contiguous()
            w = w.to(torch.float32).contiguous()
            st_ptr = stream if stream is not None else _stream_of(row_ptr)
            self.device = row_ptr.device
        else:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
            w = np.ascontiguousarray(w, dtype=np.float32)
            st_ptr = stream
            self.device = None
        self.n = int(row_ptr.shape[0]) - 1
        ci = col_idx if col_idx.shape[0] > 0 else None
        opts = CreateOpts(int(reorder), int(gather))
        st = lib().gn_create_ex(ctypes.byref(self._h), self.n, _ptr(row_ptr), _ptr(ci), _ptr(w),
                                DEVICE if self.device_io else HOST, ctypes.byref(opts), st_ptr)
        _check(st)
        self.nnz = int(lib().gn_num_entries(self._h))
        self.gather = GATHER_NAMES.get(int(lib().gn_gather_mode(self._h)), "none")
        self.exchange = EXCHANGE_NAMES[int(lib().gn_halo_exchange(self._h))]

    def close(self):
        if self._h:
            lib().gn_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vertex_order(self) -> np.ndarray:
        """The internal vertex order: entry r is the caller's id of internal vertex r."""
        order = np.empty(max(self.n, 1), dtype=np.int32)
        _check(lib().gn_vertex_order(self._h, order.ctypes.data_as(P)))
        return order[: self.n]

    def vertex_order_source(self) -> str:
        """Where the internal order was computed: "host", "device", or "none" (no reordering)."""
        return {0: "none", 1: "host", 2: "device"}[int(lib().gn_vertex_order_source(self._h))]

    def set_io(self, device: bool):
        _check(lib().gn_set_io(self._h, DEVICE if device else HOST))
        self.device_io = device

    def set_weights(self, w):
        """New vertex weights on the same graph (gn_set_weights)."""
        if not self.device_io:
            w = np.ascontiguousarray(w, dtype=np.float32)
        _check(lib().gn_set_weights(self._h, _ptr(w)))

    def _alloc(self, dtype, n):
        if self.device_io:
            import torch
            tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.int32: torch.int32}[dtype]
            return torch.empty(max(n, 1), dtype=tdt, device=self.device)
        return np.empty(max(n, 1), dtype=dtype)

    def run(self, x0=None, max_iters=2000, tol=1e-7, params: Params | None = None, start_iter=0,
            out=True, raise_on_warn=False):
        """Iterated WRGN (gn_run).  Returns (x, info dict); x is None when out=False."""
        p = params if params is not None else default_params()
        x = self._alloc(np.float32, self.n) if out else None
        if x0 is not None and not self.device_io:
            x0 = np.ascontiguousarray(x0, dtype=np.float32)
        info = RunInfo()
        st = lib().gn_run(self._h, _ptr(x0), int(max_iters), float(tol), ctypes.byref(p), int(start_iter),
                          _ptr(x), ctypes.byref(info))
        _check(st, allow_warn=not raise_on_warn)
        d = info.as_dict()
        d["status"] = STATUS[st]
        return (x[: self.n] if x is not None else None), d

    def extract_is(self, x=None):
        """Rounded set of x (or of the last run's state): (status, mask, members, count, W)."""
        mask = self._alloc(np.uint8, self.n)
        members = self._alloc(np.int32, self.n)
        cnt = ctypes.c_int32(0)
        wt = ctypes.c_double(0.0)
        if x is not None and not self.device_io:
            x = np.ascontiguousarray(x, dtype=np.float32)
        st = lib().gn_extract_is(self._h, _ptr(x), _ptr(mask), _ptr(members),
                                 ctypes.cast(ctypes.pointer(cnt), P), ctypes.cast(ctypes.pointer(wt), P))
        if st < 0 and st != -7:
            _check(st)
        return STATUS[st], mask[: self.n], members[: cnt.value], cnt.value, wt.value

    def objective(self, x=None, gamma=1.5):
        """FP64 (sum w x, E~(v x)) of x (or of the last run's state)."""
        o = ctypes.c_double(0.0)
        e = ctypes.c_double(0.0)
        if x is not None and not self.device_io:
            x = np.ascontiguousarray(x, dtype=np.float32)
        _check(lib().gn_objective(self._h, _ptr(x), float(gamma), ctypes.cast(ctypes.pointer(o), P),
                                  ctypes.cast(ctypes.pointer(e), P)))
        return o.value, e.value

    def backward(self, dL_dxT, want_w=True, want_x0=True):
        """Reverse mode of the last recorded run (gn_backward): (dL/dw, dL/dx0)."""
        gw = self._alloc(np.float32, self.n) if want_w else None
        gx = self._alloc(np.float32, self.n) if want_x0 else None
        if not self.device_io:
            dL_dxT = np.ascontiguousarray(dL_dxT, dtype=np.float32)
        _check(lib().gn_backward(self._h, _ptr(dL_dxT), _ptr(gw), _ptr(gx)))
        return (gw[: self.n] if gw is not None else None), (gx[: self.n] if gx is not None else None)


# ------------------------------------------------------------------------------------------
# batched GN

INSTANCE_CSR, INSTANCE_ASSIGNMENT = 0, 1


class BatchInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("converged", ctypes.c_int),
                ("binary", ctypes.c_int), ("resid_inf", ctypes.c_double), ("objective", ctypes.c_double),
                ("safe_div_hits", ctypes.c_longlong), ("resid_l1", ctypes.c_double), ("energy", ctypes.c_double)]


def _batch_lib():
    L = lib()
    if not hasattr(L, "_batch_ready"):
        L.gn_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, P, P, P, P, P, P, ctypes.c_int, P]
        L.gn_batch_create.restype = ctypes.c_int
        L.gn_batch_destroy.argtypes = [P]
        L.gn_batch_destroy.restype = None
        L.gn_batch_run.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Params), P, P]
        L.gn_batch_run.restype = ctypes.c_int
        L.gn_batch_last_ms.argtypes = [P]
        L.gn_batch_last_ms.restype = ctypes.c_float
        L.gn_batch_set_threads.argtypes = [P, ctypes.c_int]
        L.gn_batch_set_threads.restype = ctypes.c_int
        L.gn_batch_tune.argtypes = [P, ctypes.POINTER(Params), ctypes.c_int, P]
        L.gn_batch_tune.restype = ctypes.c_int
        L.gn_batch_extract.argtypes = [P, P, P, P, P]
        L.gn_batch_extract.restype = ctypes.c_int
        L.gn_batch_set_packing.argtypes = [P, ctypes.c_int]
        L.gn_batch_set_packing.restype = ctypes.c_int
        L.gn_batch_packing.argtypes = [P, P, P]
        L.gn_batch_packing.restype = ctypes.c_int
        L._batch_ready = True
    return L


def pack_batch(instances):
    """Concatenates instances for gn_batch_create.  Each item is either a CSR instance (an
    object with row_ptr, col_idx, w) or ("assignment", k, w) with w of length k*k."""
    count = len(instances)
    vtx = np.zeros(count + 1, np.int64)
    ent = np.zeros(count + 1, np.int64)
    kinds = np.zeros(max(count, 1), np.int32)
    rps, cis, ws = [], [], []
    for i, it in enumerate(instances):
        if isinstance(it, tuple) and it[0] == "assignment":
            k, w = it[1], np.asarray(it[2], np.float32)
            n = k * k
            kinds[i] = INSTANCE_ASSIGNMENT
            rps.append(np.zeros(n + 1, np.int32))
            ws.append(w)
            e = 0
        else:
            n = len(it.row_ptr) - 1
            rps.append(np.asarray(it.row_ptr, np.int32))
            cis.append(np.asarray(it.col_idx, np.int32))
            ws.append(np.asarray(it.w, np.float32))
            e = int(it.row_ptr[-1])
        vtx[i + 1] = vtx[i] + n
        ent[i + 1] = ent[i] + e
    rp = np.concatenate(rps) if rps else np.zeros(1, np.int32)
    ci = np.concatenate(cis) if cis else np.zeros(1, np.int32)
    w = np.concatenate(ws) if ws else np.zeros(1, np.float32)
    return vtx, ent, rp, ci, w, kinds


class Batch:
    """Many instances in one persistent launch (gn_batch_*).  device=True keeps every array of
    the calls on the GPU (torch tensors); otherwise numpy arrays (host I/O mode)."""

    def __init__(self, instances, device=False):
        L = _batch_lib()
        self._h = P()
        self.count = len(instances)
        vtx, ent, rp, ci, w, kinds = pack_batch(instances)
        self.vtx_off = vtx
        self.device_io = device
        if device:
            import torch
            self._keep = [torch.from_numpy(a).cuda() for a in (vtx, ent, rp, ci, w, kinds)]
            args = [ctypes.c_void_p(t.data_ptr()) for t in self._keep]
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        else:
            self._keep = [vtx, ent, rp, ci, w, kinds]
            args = [a.ctypes.data_as(P) for a in self._keep]
            stream = None
        _check(L.gn_batch_create(ctypes.byref(self._h), self.count, *args, DEVICE if device else HOST, stream))
        self.ntot = int(vtx[-1])

    def close(self):
        if self._h:
            _batch_lib().gn_batch_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _alloc(self, dtype, n):
        if self.device_io:
            import torch
            tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.int32: torch.int32,
                   np.float64: torch.float64}[dtype]
            return torch.empty(max(n, 1), dtype=tdt, device="cuda")
        return np.empty(max(n, 1), dtype=dtype)

    def run(self, x0=None, max_iters=2000, tol=1e-7, params: Params | None = None, out=True):
        p = params if params is not None else default_params()
        x = self._alloc(np.float32, self.ntot) if out else None
        info = (BatchInfo * max(self.count, 1))()
        if x0 is not None and not self.device_io:
            x0 = np.ascontiguousarray(x0, dtype=np.float32)
        st = _batch_lib().gn_batch_run(self._h, _ptr(x0), int(max_iters), float(tol), ctypes.byref(p), _ptr(x),
                                       ctypes.cast(info, P))
        _check(st)
        infos = [{f: getattr(info[i], f) for f, _ in BatchInfo._fields_} for i in range(self.count)]
        for d in infos:
            d["status"] = STATUS[d["status"]]
        return (x[: self.ntot] if x is not None else None), infos

    @property
    def last_ms(self):
        return float(_batch_lib().gn_batch_last_ms(self._h))

    def set_threads(self, t):
        _check(_batch_lib().gn_batch_set_threads(self._h, int(t)))

    def set_packing(self, warp_max_vertices):
        """Instances of at most this many vertices run a warp each (gn_batch_set_packing)."""
        _check(_batch_lib().gn_batch_set_packing(self._h, int(warp_max_vertices)))

    def packing(self):
        """(threshold, number of instances in warp mode) (gn_batch_packing)."""
        a, c = ctypes.c_int(0), ctypes.c_int(0)
        _check(_batch_lib().gn_batch_packing(self._h, ctypes.cast(ctypes.pointer(a), P),
                                             ctypes.cast(ctypes.pointer(c), P)))
        return a.value, c.value

    def tune(self, params: Params | None = None, max_iters=200):
        p = params if params is not None else default_params()
        t = ctypes.c_int(0)
        _check(_batch_lib().gn_batch_tune(self._h, ctypes.byref(p), int(max_iters), ctypes.cast(ctypes.pointer(t), P)))
        return t.value

    def extract(self):
        mask = self._alloc(np.uint8, self.ntot)
        counts = self._alloc(np.int32, self.count)
        weights = self._alloc(np.float64, self.count)
        statuses = self._alloc(np.int32, self.count)
        st = _batch_lib().gn_batch_extract(self._h, _ptr(mask), _ptr(counts), _ptr(weights), _ptr(statuses))
        if st < 0 and st != -7:
            _check(st)
        return STATUS[st], mask[: self.ntot], counts[: self.count], weights[: self.count], statuses[: self.count]


def random_start(u):
    """The appendix module's random simplex start from uniform draws u (CUDA tensor, any shape,
    values in (0, 1]); returns x0 of the same shape (gn_random_start)."""
    import torch
    L = lib()
    if not hasattr(L, "_start_ready"):
        L.gn_random_start.argtypes = [ctypes.c_int64, P, P, P]
        L.gn_random_start.restype = ctypes.c_int
        L._start_ready = True
    u = u.to(torch.float32).contiguous()
    x0 = torch.empty_like(u)
    _check(L.gn_random_start(u.numel(), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(x0.data_ptr()),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return x0


def multi_start(graph_inst, starts, seed, max_iters=2000, tol=1e-7, params: Params | None = None):
    """The paper's random-start protocol on one graph: `starts` random simplex starts run as
    one batch (copies of the graph as instances); returns the best start's (W(S), mask, info)
    and the per-start weights."""
    import torch
    from . import inputs
    n = graph_inst.n
    u = torch.from_numpy(inputs.uniforms(starts * n, seed)).cuda()
    x0 = random_start(u)
    b = Batch([graph_inst] * starts, device=True)
    x, infos = b.run(x0=x0, max_iters=max_iters, tol=tol, params=params)
    st, mask, counts, weights, statuses = b.extract()
    w = weights.cpu().numpy()
    best = int(np.argmax(w))
    m = mask.cpu().numpy()[best * n:(best + 1) * n]
    b.close()
    return float(w[best]), m, infos[best], w


# ------------------------------------------------------------------------------------------
# differentiable GN

def _grad_function():
    import torch

    class UnrolledGN(torch.autograd.Function):
        """x_T of `iters` unrolled WRGN steps from x0 (gamma schedule of the params); the
        backward is the library's adjoint (gn_backward) with sqrt(T) checkpointing."""

        @staticmethod
        def forward(ctx, row_ptr, col_idx, w, x0, iters, params, start_iter, graph):
            p = params if params is not None else default_params()
            p = default_params(**{f: getattr(p, f) for f, _ in Params._fields_})
            p.record = 1
            if graph is None:
                g, own = Graph(row_ptr, col_idx, w.detach()), True
            else:
                g, own = graph, False
                g.set_weights(w.detach().contiguous())
            x, info = g.run(x0=x0.detach().contiguous(), max_iters=start_iter + iters, tol=-1.0, params=p,
                            start_iter=start_iter)
            ctx.graph, ctx.own = g, own
            ctx.info = info
            return x

        @staticmethod
        def backward(ctx, gx):
            g = ctx.graph
            dw, dx0 = g.backward(gx.contiguous().to(torch.float32))
            if ctx.own:
                g.close()
            ctx.graph = None
            return None, None, dw, dx0, None, None, None, None

    return UnrolledGN


_unrolled = None


def unrolled_gn(row_ptr, col_idx, w, x0, iters, params: Params | None = None, start_iter=0, graph=None):
    """Differentiable GN on CUDA tensors: returns x_T (float32[n]); gradients flow to w and x0.

    graph: an existing device-I/O Graph of the same CSR to run on (its weights are replaced by w
    with gn_set_weights, so the CSR is neither validated nor laid out again); it holds the
    recorded run until backward, so one graph serves one forward/backward pair at a time.
    Without it each forward builds and frees a handle of its own."""
    global _unrolled
    if _unrolled is None:
        _unrolled = _grad_function()
    return _unrolled.apply(row_ptr, col_idx, w, x0, int(iters), params, int(start_iter), graph)
