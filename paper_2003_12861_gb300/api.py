"""Python face of the C ABI: models, datasets, NLL and gradient, fits, toys.

Argument marshalling only -- every step of the computation runs in
librfgpu.so.  PyTorch supplies device memory and streams where a caller
wants device-resident buffers (Data.from_torch, nll_grad_async)."""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from . import _lib as L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def make_nodes(nodes) -> "C.Array":
    arr = (L.rf_node * len(nodes))()
    for i, nd in enumerate(nodes):
        r = arr[i]
        r.kind = L.KIND[nd.kind]
        r.n_in = len(nd.inputs)
        for j, v in enumerate(nd.inputs):
            r.in_[j] = v
        r.value, r.lo, r.hi = float(nd.value), float(nd.lo), float(nd.hi)
        r.is_free = 1 if nd.free else 0
    return arr


class Model:
    """A compiled model (rf_model_create)."""

    def __init__(self, nodes, root: int):
        lib = L.load()
        arr = make_nodes(nodes)
        h = C.c_void_p()
        exprs = [(i, nd) for i, nd in enumerate(nodes) if nd.kind == "expr"]
        if exprs:
            keep = []
            ex = (L.rf_expr * len(exprs))()
            for j, (i, nd) in enumerate(exprs):
                ops = (C.c_int32 * max(1, len(nd.prog)))(*nd.prog)
                cst = (C.c_double * max(1, len(nd.consts)))(*nd.consts)
                keep += [ops, cst]
                ex[j].node, ex[j].n_ops, ex[j].ops = i, len(nd.prog), ops
                ex[j].n_consts, ex[j].consts = len(nd.consts), cst
            L.check(lib.rf_model_create_expr(arr, len(nodes), root, ex, len(exprs), C.byref(h)))
        else:
            L.check(lib.rf_model_create(arr, len(nodes), root, C.byref(h)))
        self._h = h
        self.nodes = list(nodes)
        self.root = root
        self.n_free = lib.rf_model_n_free(h)
        self.n_obs = lib.rf_model_n_obs(h)

    @classmethod
    def from_spec(cls, spec):
        return cls(spec.nodes, spec.root)

    def describe(self) -> str:
        buf = C.create_string_buffer(512)
        L.check(L.load().rf_model_describe(self._h, buf, 512))
        return buf.value.decode()

    def set_fp64(self, on: bool = True):
        """Run every event through the FP64 graph interpreter (rf_model_set_fp64)."""
        L.check(L.load().rf_model_set_fp64(self._h, 1 if on else 0))

    def set_launch(self, threads_per_block: int = 0, blocks_per_sm: int = 0):
        L.check(L.load().rf_set_launch(self._h, threads_per_block, blocks_per_sm))

    def close(self):
        if getattr(self, "_h", None):
            L.load().rf_model_destroy(self._h)
            self._h = None

    __del__ = close


class Data:
    """Event columns on the device (rf_data_upload / rf_generate_toys)."""

    def __init__(self, handle, model: Model, keep=None):
        self._h = handle
        self.model = model
        self._keep = keep  # borrowed device buffers must outlive the handle
        lib = L.load()
        self.n_events = lib.rf_data_n_events(handle)
        self.n_sets = lib.rf_data_n_sets(handle)

    @classmethod
    def upload(cls, model: Model, cols: Sequence[np.ndarray], offsets=None, f32: Sequence[bool] | None = None):
        lib = L.load()
        n_obs = model.n_obs
        if len(cols) != n_obs:
            raise ValueError(f"expected {n_obs} columns")
        f32 = f32 or [c.dtype == np.float32 for c in cols]
        conv = [np.ascontiguousarray(c, dtype=np.float32 if f else np.float64) for c, f in zip(cols, f32)]
        n = len(conv[0]) if conv else 0
        ptrs = (C.c_void_p * max(1, n_obs))(*[c.ctypes.data for c in conv])
        dt = (C.c_int32 * max(1, n_obs))(*[L.RF_F32 if f else L.RF_F64 for f in f32])
        if offsets is None:
            off_p, n_sets = None, 1
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            off_p, n_sets = off.ctypes.data_as(C.POINTER(C.c_int64)), len(off) - 1
        h = C.c_void_p()
        L.check(lib.rf_data_upload(model._h, ptrs, dt, n, off_p, n_sets, 0, C.byref(h)))
        return cls(h, model)

    @classmethod
    def from_torch(cls, model: Model, cols, offsets=None):
        """Borrow CUDA tensors (float32/float64, contiguous) as columns."""
        import torch

        lib = L.load()
        cols = [c.contiguous() for c in cols]
        for c in cols:
            if not c.is_cuda or c.dtype not in (torch.float32, torch.float64):
                raise ValueError("columns must be CUDA float32/float64 tensors")
        ptrs = (C.c_void_p * max(1, len(cols)))(*[c.data_ptr() for c in cols])
        dt = (C.c_int32 * max(1, len(cols)))(*[L.RF_F32 if c.dtype == torch.float32 else L.RF_F64 for c in cols])
        n = cols[0].numel() if cols else 0
        if offsets is None:
            off_p, n_sets, off = None, 1, None
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            off_p, n_sets = off.ctypes.data_as(C.POINTER(C.c_int64)), len(off) - 1
        h = C.c_void_p()
        L.check(lib.rf_data_upload(model._h, ptrs, dt, n, off_p, n_sets, 1, C.byref(h)))
        return cls(h, model, keep=cols)

    def read(self, col: int, i0: int = 0, i1: int | None = None) -> np.ndarray:
        i1 = self.n_events if i1 is None else i1
        out = np.zeros(i1 - i0)
        L.check(L.load().rf_data_read(self._h, col, i0, i1, _dp(out)))
        return out

    def offsets(self) -> np.ndarray:
        out = np.zeros(self.n_sets + 1, dtype=np.int64)
        L.check(L.load().rf_data_offsets(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def close(self):
        if getattr(self, "_h", None):
            L.load().rf_data_destroy(self._h)
            self._h = None

    __del__ = close


def _theta(model: Model, data: Data, theta):
    th = _f64(theta).reshape(-1)
    if th.size == model.n_free and data.n_sets > 1:
        th = np.tile(th, data.n_sets)
    if th.size != model.n_free * data.n_sets:
        raise ValueError("theta must hold n_sets x n_free values")
    return th


def autotune(model: Model, data: Data, passes: int = 5):
    """Pick the fastest launch shape for (model, data); returns (threads, blocks_per_sm, ms)."""
    t, b, ms = C.c_int32(), C.c_int32(), C.c_double()
    L.check(L.load().rf_autotune(model._h, data._h, passes, C.byref(t), C.byref(b), C.byref(ms)))
    return t.value, b.value, ms.value


def autotune_scan(model: Model, data: Data, passes: int = 3):
    """The autotuner's whole grid: [(blocks_per_sm, mean pass ms), ...]; the
    winner is kept on the model."""
    bps = (C.c_int32 * 16)()
    ms = (C.c_double * 16)()
    n = C.c_int32()
    L.check(L.load().rf_autotune_scan(model._h, data._h, passes, 16, bps, ms, C.byref(n)))
    return [(bps[i], ms[i]) for i in range(n.value)]


def nll(model: Model, data: Data, theta, stream=None, allow_domain=False):
    th = _theta(model, data, theta)
    out = np.zeros(data.n_sets)
    allow = (L.RF_OK, L.RF_E_DOMAIN) if allow_domain else (L.RF_OK,)
    L.check(L.load().rf_nll(model._h, data._h, _dp(th), _dp(out), _stream(stream)), allow)
    return out if data.n_sets > 1 else out[0]


def nll_grad(model: Model, data: Data, theta, stream=None, allow_domain=False):
    th = _theta(model, data, theta)
    out = np.zeros(data.n_sets)
    g = np.zeros(data.n_sets * max(1, model.n_free))
    allow = (L.RF_OK, L.RF_E_DOMAIN) if allow_domain else (L.RF_OK,)
    L.check(L.load().rf_nll_grad(model._h, data._h, _dp(th), _dp(out), _dp(g), _stream(stream)), allow)
    g = g[: data.n_sets * model.n_free].reshape(data.n_sets, model.n_free)
    return (out, g) if data.n_sets > 1 else (out[0], g[0])


def nll_grad_async(model: Model, data: Data, d_theta, d_out, d_flags, stream=None):
    """Device-resident pass: torch tensors (float64 theta, float64 out of
    n_sets x (1 + n_free), int32 flags); launches only."""
    L.check(L.load().rf_nll_grad_async(model._h, data._h, C.c_void_p(d_theta.data_ptr()),
                                       C.c_void_p(d_out.data_ptr()), C.c_void_p(d_flags.data_ptr()),
                                       _stream(stream)))


def nll_grad_stream(model: Model, data: Data, host_cols, theta, stream=None, allow_domain=False):
    """rf_nll_grad with the events in host memory (pinned torch tensors or
    numpy arrays, the dataset's layout and dtypes): copies overlap the pass.
    Returns (nll, grad) like nll_grad."""
    th = _theta(model, data, theta)
    S, P = data.n_sets, model.n_free
    ptrs = (C.c_void_p * len(host_cols))(*[C.c_void_p(c.data_ptr() if hasattr(c, "data_ptr") else
                                                        c.ctypes.data) for c in host_cols])
    nll = np.zeros(S)
    g = np.zeros(S * max(P, 1))
    allow = (L.RF_OK, L.RF_E_DOMAIN) if allow_domain else (L.RF_OK,)
    L.check(L.load().rf_nll_grad_stream(model._h, data._h, ptrs, _dp(th), _dp(nll), _dp(g), _stream(stream)), allow)
    g = g[: S * P].reshape(S, P)
    return (nll, g) if S > 1 else (nll[0], g[0])


# ------------------------------------------------------- sharded evaluation

def shard(n: int, align: int, rank: int, world: int):
    """Rank `rank`'s contiguous range [lo, hi) of n items split over `world`
    ranks at multiples of `align` (4096 for events, 1 for sets)."""
    lo, hi = C.c_int64(), C.c_int64()
    L.check(L.load().rf_shard(int(n), int(align), int(rank), int(world), C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def nll_grad_partial(model: Model, data: Data, d_theta, d_pairs, d_flags, stream=None):
    """One shard's compensated partial sums: torch tensors (float64 theta,
    float64 pairs of n_sets x (1 + n_free) x 2, int32 flags); launches only."""
    L.check(L.load().rf_nll_grad_partial(model._h, data._h, C.c_void_p(d_theta.data_ptr()),
                                         C.c_void_p(d_pairs.data_ptr()), C.c_void_p(d_flags.data_ptr()),
                                         _stream(stream)))


def combine_partials(pairs, flags):
    """The exchange step: pairs (world, n_sets, 1 + n_free, 2) and flags
    (world, n_sets) from every shard, merged in rank order.  Returns (out of
    n_sets x (1 + n_free): NLL then gradient, flags)."""
    pairs = np.ascontiguousarray(pairs, dtype=np.float64)
    flags = np.ascontiguousarray(flags, dtype=np.int32)
    world, S, Q, two = pairs.shape
    assert two == 2 and flags.shape == (world, S)
    out = np.zeros((S, Q))
    fo = np.zeros(S, dtype=np.int32)
    L.check(L.load().rf_combine_partials(_dp(pairs), flags.ctypes.data_as(C.POINTER(C.c_int32)), world, S, Q - 1,
                                         _dp(out), fo.ctypes.data_as(C.POINTER(C.c_int32))),
            (L.RF_OK, L.RF_E_DOMAIN))
    return out, fo


def gather_partials(pairs, flags, group=None):
    """all_gather of every rank's (pairs, flags) over torch.distributed, in
    rank order (the exchange's one collective)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    p = torch.as_tensor(np.ascontiguousarray(pairs, dtype=np.float64)).to(dev)
    f = torch.as_tensor(np.ascontiguousarray(flags, dtype=np.int32)).to(dev)
    ps = [torch.empty_like(p) for _ in range(world)]
    fs = [torch.empty_like(f) for _ in range(world)]
    dist.all_gather(ps, p, group=group)
    dist.all_gather(fs, f, group=group)
    return np.stack([t.cpu().numpy() for t in ps]), np.stack([t.cpu().numpy() for t in fs])


def nll_grad_sharded(model: Model, shard_data: Data, theta, group=None):
    """NLL and gradient of a dataset split over the ranks of `group`: this
    rank evaluates its shard (shard_data) on its GPU, the ranks exchange
    their compensated partial sums once, and every rank merges them in rank
    order.  theta: n_sets x n_free (the same on every rank).  Returns
    (nll, grad, flags) of the whole dataset."""
    import torch

    S, P = shard_data.n_sets, model.n_free
    th = torch.as_tensor(_theta(model, shard_data, theta).reshape(S, max(P, 1)), dtype=torch.float64).cuda()
    pairs = torch.zeros((S, 1 + P, 2), dtype=torch.float64, device="cuda")
    flags = torch.zeros(S, dtype=torch.int32, device="cuda")
    nll_grad_partial(model, shard_data, th, pairs, flags)
    torch.cuda.synchronize()
    allp, allf = gather_partials(pairs.cpu().numpy(), flags.cpu().numpy(), group)
    out, fo = combine_partials(allp, allf)
    return out[:, 0], out[:, 1:], fo


def nll_chunks(model: Model, data: Data, theta, set_index: int = 0, max_chunks: int = 1 << 16):
    """Per-chunk (sum log p, sum dlog p/dtheta) of one set: array (chunks, 1 + n_free)."""
    th = _theta(model, data, theta)
    P = model.n_free
    out = np.zeros(max_chunks * (1 + P))
    n = C.c_int32()
    L.check(L.load().rf_nll_chunks(model._h, data._h, _dp(th), set_index, _dp(out), max_chunks, C.byref(n)),
            (L.RF_OK, L.RF_E_DOMAIN))
    return out[: min(n.value, max_chunks) * (1 + P)].reshape(-1, 1 + P)


def fit(model: Model, data: Data, theta0=None, tol_edm: float = 1e-7, max_evals: int = 1000, want_cov=True,
        graph: bool = True, device_steps: bool = True):
    """rf_fit.  graph=False launches every evaluation directly (and steps on
    the host); device_steps=False keeps every quasi-Newton step on the host
    (the results are bitwise the same either way)."""
    S, P = data.n_sets, model.n_free
    th0 = None if theta0 is None else _theta(model, data, theta0)
    opts = L.rf_fit_opts(tol_edm, max_evals, 1 if want_cov else 0, 0 if graph else 1, 0 if device_steps else 1)
    th = np.zeros(S * P)
    nl = np.zeros(S)
    cov = np.zeros(S * P * P) if want_cov else None
    ne = np.zeros(S, dtype=np.int32)
    fs = np.zeros(S, dtype=np.int32)
    ip = C.POINTER(C.c_int32)
    L.check(L.load().rf_fit(model._h, data._h, _dp(th0) if th0 is not None else None, C.byref(opts), _dp(th),
                            _dp(nl), _dp(cov) if want_cov else None, ne.ctypes.data_as(ip), fs.ctypes.data_as(ip)))
    return dict(theta=th.reshape(S, P), nll=nl, cov=None if cov is None else cov.reshape(S, P, P), n_evals=ne,
                status=fs)


def fit_sets(model: Model, data: Data, sets, theta0=None, tol_edm: float = 1e-7, max_evals: int = 1000,
             want_cov=False, device_steps: bool = True):
    """rf_fit_sets: fit only the listed sets of a batch (results in the
    list's order), the events staying where they are."""
    idx = np.ascontiguousarray(sets, dtype=np.int32)
    n, P = len(idx), model.n_free
    th0 = None if theta0 is None else np.ascontiguousarray(theta0, dtype=np.float64).reshape(-1)
    if th0 is not None and th0.size != n * P:
        raise ValueError("theta0 must hold len(sets) x n_free values")
    opts = L.rf_fit_opts(tol_edm, max_evals, 1 if want_cov else 0, 0, 0 if device_steps else 1)
    th = np.zeros(max(1, n * P))
    nl = np.zeros(max(1, n))
    cov = np.zeros(max(1, n * P * P)) if want_cov else None
    ne = np.zeros(max(1, n), dtype=np.int32)
    fs = np.zeros(max(1, n), dtype=np.int32)
    ip = C.POINTER(C.c_int32)
    L.check(L.load().rf_fit_sets(model._h, data._h, idx.ctypes.data_as(ip), n, _dp(th0) if th0 is not None else None,
                                 C.byref(opts), _dp(th), _dp(nl), _dp(cov) if want_cov else None,
                                 ne.ctypes.data_as(ip), fs.ctypes.data_as(ip)))
    return dict(theta=th[: n * P].reshape(n, P), nll=nl[:n],
                cov=None if cov is None else cov[: n * P * P].reshape(n, P, P), n_evals=ne[:n], status=fs[:n])


def generate_toys(model: Model, theta, seed: int, mean_n, poisson: bool = True, f32: Sequence[bool] | None = None):
    mean_n = _f64(np.atleast_1d(mean_n))
    S = len(mean_n)
    th = None if theta is None else _f64(theta).reshape(-1)
    per_set = 1 if (th is not None and th.size == S * model.n_free and S > 1) else 0
    dt = None
    if f32 is not None:
        dt = (C.c_int32 * model.n_obs)(*[L.RF_F32 if f else L.RF_F64 for f in f32])
    h = C.c_void_p()
    L.check(L.load().rf_generate_toys(model._h, _dp(th) if th is not None else None, per_set, seed, S,
                                      _dp(mean_n), 1 if poisson else 0, dt, C.byref(h)))
    return Data(h, model)


def hist64(model: Model, data: Data, col: int, d_out, stream=None):
    L.check(L.load().rf_hist64(model._h, data._h, col, C.c_void_p(d_out.data_ptr()), _stream(stream)))


# ------------------------------------------------------------- measurement

def refill(data: Data, cols, stream=None):
    """Copy the next batch of host columns (same layout) into `data`.
    Columns may be numpy arrays or pinned CPU torch tensors."""
    ptrs = (C.c_void_p * max(1, len(cols)))(*[c.data_ptr() if hasattr(c, "data_ptr") else c.ctypes.data
                                              for c in cols])
    L.check(L.load().rf_data_refill(data._h, ptrs, _stream(stream)))


def kernel_timing(enable: bool):
    L.check(L.load().rf_kernel_timing(1 if enable else 0))


def kernel_time(reset: bool = True):
    ms = C.c_double()
    n = C.c_int64()
    L.check(L.load().rf_kernel_time(C.byref(ms), C.byref(n), 1 if reset else 0))
    return ms.value, n.value


def launch_count() -> int:
    """The library's kernel launches so far in this process (rf_launch_count)."""
    n = C.c_int64()
    L.check(L.load().rf_launch_count(C.byref(n)))
    return n.value


def slow_events(data: Data) -> int:
    n = C.c_int64()
    L.check(L.load().rf_slow_events(data._h, C.byref(n)))
    return n.value


def probe(kind: int, n_exp: int = 0, n_erfc: int = 0, n_log: int = 0, n_rcp: int = 0) -> float:
    r = C.c_double()
    L.check(L.load().rf_probe(kind, n_exp, n_erfc, n_log, n_rcp, C.byref(r)))
    return r.value


def _check_noalloc_args(model: Model, cols, d_theta, d_out, d_flags):
    """Argument checks of nll_grad_noalloc, before anything reaches the
    library: every buffer the pass reads or writes must be a contiguous CUDA
    tensor of the type and size the C entry point assumes, because it only
    receives their addresses."""
    import torch

    if len(cols) != model.n_obs:
        raise ValueError(f"expected {model.n_obs} columns, got {len(cols)}")
    n = None
    for c in cols:
        if not getattr(c, "is_cuda", False) or not c.is_contiguous():
            raise ValueError("columns must be contiguous CUDA tensors")
        if c.dtype not in (torch.float32, torch.float64):
            raise ValueError("columns must be float32 or float64")
        if n is None:
            n = c.numel()
        elif c.numel() != n:
            raise ValueError("columns must hold the same number of events")
    for name, t, dt, need in (("d_theta", d_theta, torch.float64, model.n_free),
                              ("d_out", d_out, torch.float64, 1 + model.n_free),
                              ("d_flags", d_flags, torch.int32, 1)):
        if not getattr(t, "is_cuda", False) or not t.is_contiguous() or t.dtype != dt:
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor")
        if t.numel() < need or (name == "d_theta" and t.numel() != need):
            raise ValueError(f"{name} must hold {'exactly' if name == 'd_theta' else 'at least'} {need} values")
    return n or 0


def noalloc_max_events(model: Model) -> int:
    """Largest dataset nll_grad_noalloc accepts for this model (host only)."""
    n = C.c_int64()
    L.check(L.load().rf_nll_grad_noalloc_max_events(model._h, C.byref(n)))
    return n.value


def nll_grad_noalloc(model: Model, cols, d_theta, d_out, d_flags, stream=None):
    """NLL + gradient of one dataset held in caller-owned CUDA tensors, with no
    device allocation by the library (its scratch is a static device array).
    For callers that cannot allocate device memory while they run.  Launches
    only, on `stream` (default: torch's current stream, so that the pass is
    ordered after the producers of the tensors); overlapping calls on one GPU
    must be serialised by the caller."""
    import torch

    n = _check_noalloc_args(model, cols, d_theta, d_out, d_flags)
    if stream is None:
        stream = torch.cuda.current_stream(cols[0].device if cols else d_out.device)
    ptrs = (C.c_void_p * max(1, len(cols)))(*[c.data_ptr() for c in cols])
    dt = (C.c_int32 * max(1, len(cols)))(*[L.RF_F32 if c.dtype == torch.float32 else L.RF_F64 for c in cols])
    L.check(L.load().rf_nll_grad_noalloc(model._h, ptrs, dt, n, C.c_void_p(d_theta.data_ptr()),
                                         C.c_void_p(d_out.data_ptr()), C.c_void_p(d_flags.data_ptr()),
                                         _stream(stream)))


# ----------------------------------------------------------- learned start

class MLP:
    """The learned-start network (rf_mlp_*): histogram -> fit start."""

    def __init__(self, n_in=64, n_hidden=128, n_hidden_layers=3, n_out=6, seed=0, _handle=None):
        lib = L.load()
        if _handle is None:
            h = C.c_void_p()
            L.check(lib.rf_mlp_create(n_in, n_hidden, n_hidden_layers, n_out, seed, C.byref(h)))
            _handle = h
        self._h = _handle
        self.n_params = lib.rf_mlp_n_params(self._h)

    @classmethod
    def load(cls, path: str):
        h = C.c_void_p()
        L.check(L.load().rf_mlp_load(path.encode(), C.byref(h)))
        return cls(_handle=h)

    def save(self, path: str):
        L.check(L.load().rf_mlp_save(self._h, path.encode()))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        L.check(L.load().rf_mlp_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        L.check(L.load().rf_mlp_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def forward(self, d_x, d_y, stream=None):
        L.check(L.load().rf_mlp_forward(self._h, C.c_void_p(d_x.data_ptr()), d_x.shape[0],
                                        C.c_void_p(d_y.data_ptr()), _stream(stream)))

    def predict(self, model: Model, data: Data, col: int = 0) -> np.ndarray:
        """Learned fit starts (rf_mlp_predict): n_sets x n_free, host."""
        out = np.zeros(data.n_sets * model.n_free)
        L.check(L.load().rf_mlp_predict(self._h, model._h, data._h, col, _dp(out)))
        return out.reshape(data.n_sets, model.n_free)

    def grad(self, d_x, d_t, d_grad=None, stream=None):
        loss = C.c_float()
        L.check(L.load().rf_mlp_grad(self._h, C.c_void_p(d_x.data_ptr()), C.c_void_p(d_t.data_ptr()),
                                     d_x.shape[0], C.byref(loss),
                                     C.c_void_p(d_grad.data_ptr()) if d_grad is not None else None,
                                     _stream(stream)))
        return loss.value

    def adam(self, lr: float, stream=None):
        L.check(L.load().rf_mlp_adam(self._h, lr, _stream(stream)))

    def train(self, d_x, d_t, batch=1024, epochs=10, lr=1e-3, seed=0, standardise=True):
        loss = C.c_float()
        L.check(L.load().rf_mlp_train(self._h, C.c_void_p(d_x.data_ptr()), C.c_void_p(d_t.data_ptr()),
                                      d_x.shape[0], batch, epochs, lr, seed, 1 if standardise else 0,
                                      C.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "_h", None):
            L.load().rf_mlp_destroy(self._h)
            self._h = None

    __del__ = close


def math_eval(fn: int, d_x, d_y, stream=None):
    """Library float-float functions (0 exp, 1 log, 2 rcp, 3 erfcx) or CUDA's
    FP64 ones (10-13) elementwise on CUDA float64 tensors."""
    L.check(L.load().rf_math_eval(fn, C.c_void_p(d_x.data_ptr()), C.c_void_p(d_y.data_ptr()), d_x.numel(),
                                  _stream(stream)))


# ------------------------------------------------------ binned likelihood

class BinnedModel:
    """A HistFactory-style binned model (rf_binned_*), built from the plain
    data of workloads.binned_model: n_bins, bin0, nominal, constrained,
    modifiers = (sample, kind, param, k_lo, k_hi, h_lo, h_hi)."""

    def __init__(self, spec):
        lib = L.load()
        nom = [np.ascontiguousarray(h, dtype=np.float64) for h in spec["nominal"]]
        bin0 = np.ascontiguousarray(spec["bin0"], dtype=np.int32)
        nb = np.array([len(h) for h in nom], dtype=np.int32)
        nominal = np.concatenate(nom)
        con = np.ascontiguousarray([1 if c else 0 for c in spec["constrained"]], dtype=np.int32)
        mods = spec["modifiers"]
        arr = (L.rf_modifier * max(1, len(mods)))()
        hd = []
        for j, (smp, kind, par, klo, khi, lo, hi) in enumerate(mods):
            arr[j] = L.rf_modifier(int(smp), int(kind), int(par), float(klo), float(khi))
            if kind == 2:
                hd += [np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)]
        hdata = np.concatenate(hd) if hd else np.zeros(1)
        ip = C.POINTER(C.c_int32)
        h = C.c_void_p()
        L.check(lib.rf_binned_create(int(spec["n_bins"]), len(nom), bin0.ctypes.data_as(ip), nb.ctypes.data_as(ip),
                                     _dp(nominal), len(con), con.ctypes.data_as(ip), len(mods), C.cast(arr, C.c_void_p),
                                     _dp(hdata), C.byref(h)))
        self._h = h
        self.n_bins = int(spec["n_bins"])
        self.n_params = lib.rf_binned_n_params(h)

    def __del__(self):
        if getattr(self, "_h", None):
            L.load().rf_binned_destroy(self._h)
            self._h = None

    def nll_grad(self, counts, theta, allow_domain=False):
        """counts (n_sets, n_bins), theta (n_sets, n_params) -> (nll, grad)."""
        counts = np.ascontiguousarray(np.atleast_2d(counts), dtype=np.float64)
        theta = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
        S = counts.shape[0]
        nll = np.zeros(S)
        g = np.zeros((S, self.n_params))
        allow = (L.RF_OK, L.RF_E_DOMAIN) if allow_domain else (L.RF_OK,)
        L.check(L.load().rf_binned_nll_grad(self._h, S, _dp(counts), _dp(theta), _dp(nll), _dp(g)), allow)
        return nll, g

    def nll_grad_async(self, d_counts, d_theta, d_out, d_flags, stream=None):
        """Device tensors: counts (S, n_bins), theta (S, P), out (S, 1 + P), flags (S,) int32."""
        L.check(L.load().rf_binned_nll_grad_async(self._h, d_counts.shape[0], C.c_void_p(d_counts.data_ptr()),
                                                  C.c_void_p(d_theta.data_ptr()), C.c_void_p(d_out.data_ptr()),
                                                  C.c_void_p(d_flags.data_ptr()), _stream(stream)))

    def fit(self, counts, theta0, lo, hi, tol_edm: float = 1e-7, max_evals: int = 1000, want_cov=True):
        """Batched fits of the datasets (rows of counts) from theta0; bounds
        lo/hi per parameter.  Returns dict(theta, nll, cov, n_evals, status)."""
        counts = np.ascontiguousarray(np.atleast_2d(counts), dtype=np.float64)
        S, P = counts.shape[0], self.n_params
        th0 = np.ascontiguousarray(np.broadcast_to(np.asarray(theta0, dtype=np.float64), (S, P)))
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        th = np.zeros((S, P))
        nl = np.zeros(S)
        cov = np.zeros((S, P, P)) if want_cov else None
        ne = np.zeros(S, dtype=np.int32)
        fs = np.zeros(S, dtype=np.int32)
        opts = L.rf_fit_opts(tol_edm, max_evals, 1 if want_cov else 0, 0, 0)
        ip = C.POINTER(C.c_int32)
        L.check(L.load().rf_binned_fit(self._h, S, _dp(counts), _dp(th0), _dp(lo), _dp(hi),
                                       C.cast(C.byref(opts), C.c_void_p), _dp(th), _dp(nl),
                                       _dp(cov) if want_cov else None, ne.ctypes.data_as(ip), fs.ctypes.data_as(ip)))
        return dict(theta=th, nll=nl, cov=cov, n_evals=ne, status=fs)

    def expected(self, d_theta, d_nu, stream=None):
        L.check(L.load().rf_binned_expected(self._h, d_theta.shape[0], C.c_void_p(d_theta.data_ptr()),
                                            C.c_void_p(d_nu.data_ptr()), _stream(stream)))


# --------------------------------------------------------------- autograd

_RFNLL = None


def _rfnll():
    global _RFNLL
    if _RFNLL is None:
        import torch

        class RfNLL(torch.autograd.Function):
            """NLL(theta) as a torch function.  forward runs one device-resident
            pass (rf_nll_grad_async) on the current stream and saves the
            gradient; backward returns grad_out * grad without a second pass.
            theta: (n_free,) for one set or shared by all sets, or
            (n_sets, n_free); the result is a scalar or (n_sets,) NLLs."""

            @staticmethod
            def forward(ctx, theta, model, data):
                S, P = data.n_sets, model.n_free
                th = theta.detach().to(device="cuda", dtype=torch.float64).contiguous().reshape(-1)
                shared = theta.dim() == 1 and S > 1
                if shared:
                    th = th.repeat(S)
                if th.numel() != S * P:
                    raise ValueError("theta must hold n_free or n_sets x n_free values")
                out = torch.empty(S * (1 + P), dtype=torch.float64, device="cuda")
                flags = torch.zeros(S, dtype=torch.int32, device="cuda")
                nll_grad_async(model, data, th, out, flags, stream=torch.cuda.current_stream())
                o = out.view(S, 1 + P)
                ctx.save_for_backward(o[:, 1:].clone())
                ctx.shared = shared
                ctx.single = theta.dim() == 1 and S == 1
                ctx.dtype = theta.dtype
                nll = o[:, 0].clone()
                return nll.reshape(()) if ctx.single else nll

            @staticmethod
            def backward(ctx, grad_out):
                (g,) = ctx.saved_tensors
                if ctx.single:
                    d = grad_out * g[0]
                elif ctx.shared:
                    d = (grad_out[:, None] * g).sum(0)
                else:
                    d = grad_out[:, None] * g
                return d.to(ctx.dtype), None, None

        _RFNLL = RfNLL
    return _RFNLL


def __getattr__(name):
    if name == "RfNLL":  # torch is imported on first use only
        return _rfnll()
    raise AttributeError(name)
