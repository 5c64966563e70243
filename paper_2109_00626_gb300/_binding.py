"""ctypes binding of libttc.so (include/ttc.h).

Argument marshalling only: every step of a contraction runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  There
is no CPU fallback: if the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_int, c_int32, c_size_t, c_uint8, c_uint64, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttc.so")

TT_F64, TT_F32, TT_BF16 = 0, 1, 2
TT_P_NATIVE, TT_P_TF32X3, TT_P_BF16, TT_P_BF16X3, TT_P_TF32 = 0, 1, 2, 3, 4
TT_LAYOUT_CHAIN, TT_LAYOUT_MERGED = 0, 1
TT_OP_FULL, TT_OP_PARTIAL, TT_OP_BACKWARD = 0, 1, 2
TT_STATUS_NONFINITE, TT_STATUS_OVERFLOW, TT_STATUS_TIMEOUT = 1, 2, 4
TT_MAX_ORDER = 64

PREC = {"native": TT_P_NATIVE, "tf32x3": TT_P_TF32X3, "bf16": TT_P_BF16, "bf16x3": TT_P_BF16X3, "tf32": TT_P_TF32}
LAYOUT = {"chain": TT_LAYOUT_CHAIN, "merged": TT_LAYOUT_MERGED}

# Every symbol include/ttc.h declares (checked by the CPU test-suite).
EXPORTS = [
    "tt_workspace_bytes",
    "tt_contract_full",
    "tt_partial_shape",
    "tt_contract_partial",
    "tt_contract_partial_k",
    "tt_batch_plan",
    "tt_batch_pack",
    "tt_contract_batched",
    "tt_contract_batched_noalloc",
    "tt_plan_info",
    "tt_plan_free",
    "tt_autotune",
    "tt_contract_backward",
    "tt_contract_backward_k",
    "tt_error_string",
    "tt_launch_count",
    "tt_selftest_wait",
    "tt_pairs_shape",
    "tt_contract_pairs",
    "tt_svd_workspace",
    "tt_svd",
    "tt_dense_permute",
    "tt_factored_shape",
    "tt_contract_factored",
    "tt_round_workspace",
    "tt_round",
]


class TTFactored(ctypes.Structure):
    """tt_factored: free positions, run-matrix shapes and arena offsets."""

    _fields_ = [
        ("n_free", c_int32),
        ("free_pos", c_int32 * 64),
        ("rows", c_int32 * 65),
        ("cols", c_int32 * 65),
        ("off_t", c_size_t * 65),
        ("off_log2", c_size_t * 65),
        ("bytes", c_size_t),
        ("ws_bytes", c_size_t),
    ]


class TTDesc(ctypes.Structure):
    _fields_ = [
        ("order", c_int32),
        ("modes", POINTER(c_int32)),
        ("ranks", POINTER(c_int32)),
        ("cores", POINTER(c_void_p)),
        ("dtype", c_int32),
    ]


class TTBatch(ctypes.Structure):
    _fields_ = [
        ("n_pairs", c_int32),
        ("x", POINTER(TTDesc)),
        ("y", POINTER(TTDesc)),
        ("mask", POINTER(POINTER(c_uint8))),
        ("z", POINTER(TTDesc)),
        ("prec", c_int32),
    ]


class TTError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (code {code})")


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libttc.so is not built; run paper_2109_00626_gb300.build.build() (needs nvcc)"
        )
    L = ctypes.CDLL(LIB_PATH)
    D = POINTER(TTDesc)
    U8 = POINTER(c_uint8)
    I32 = POINTER(c_int32)
    L.tt_workspace_bytes.argtypes = [c_int, D, D, U8, c_int, c_int, POINTER(c_size_t)]
    L.tt_contract_full.argtypes = [D, D, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    L.tt_partial_shape.argtypes = [D, D, U8, c_int, I32, I32, I32, I32]
    L.tt_contract_partial.argtypes = [D, D, U8, c_int, c_int, D, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    L.tt_batch_plan.argtypes = [POINTER(TTBatch), POINTER(c_void_p), POINTER(c_size_t), POINTER(c_size_t)]
    L.tt_batch_pack.argtypes = [c_void_p, c_void_p, c_size_t]
    L.tt_contract_batched.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    L.tt_contract_batched_noalloc.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.tt_plan_info.argtypes = [c_void_p, c_int32, I32, I32]
    L.tt_plan_free.argtypes = [c_void_p]
    L.tt_plan_free.restype = None
    L.tt_contract_backward.argtypes = [
        D, D, U8, c_int, c_int, c_void_p, D, D, D, c_int32, c_void_p, c_void_p, c_size_t, c_void_p
    ]
    L.tt_contract_partial_k.argtypes = [D, D, U8, c_int, D, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    L.tt_contract_backward_k.argtypes = [D, D, U8, c_int, D, D, D, c_void_p, c_void_p, c_size_t, c_void_p]
    L.tt_autotune.argtypes = [c_int, ctypes.c_char_p]
    L.tt_error_string.argtypes = [c_int]
    L.tt_error_string.restype = ctypes.c_char_p
    L.tt_launch_count.argtypes = []
    L.tt_selftest_wait.argtypes = [c_int, ctypes.c_int64, c_void_p, c_void_p]
    L.tt_pairs_shape.argtypes = [D, D, c_int, I32, I32, I32, I32, I32, I32]
    L.tt_contract_pairs.argtypes = [D, D, c_int, I32, I32, c_int, D, c_void_p, c_void_p, c_void_p]
    L.tt_svd_workspace.argtypes = [c_int, I32, c_int, c_int32, I32, POINTER(c_size_t)]
    L.tt_svd.argtypes = [c_void_p, c_int, I32, c_int, ctypes.c_double, c_int32, POINTER(c_void_p), c_void_p, c_void_p,
                         c_void_p, c_size_t, c_void_p]
    L.tt_dense_permute.argtypes = [c_void_p, c_int, I32, I32, c_int, c_void_p, c_void_p]
    L.tt_round_workspace.argtypes = [D, c_int32, POINTER(c_size_t)]
    L.tt_round.argtypes = [D, ctypes.c_double, c_int32, POINTER(c_void_p), c_void_p, c_void_p, c_void_p, c_size_t,
                           c_void_p]
    L.tt_factored_shape.argtypes = [D, D, U8, POINTER(TTFactored)]
    L.tt_contract_factored.argtypes = [D, D, U8, POINTER(TTFactored), c_void_p, c_void_p, c_void_p, c_size_t,
                                       c_void_p]
    L.tt_launch_count.restype = c_uint64
    _lib = L
    return L


def error_string(code: int) -> str:
    try:
        return lib().tt_error_string(int(code)).decode()
    except RuntimeError:
        return "library not loaded"


def launch_count() -> int:
    return int(lib().tt_launch_count())


def check(rc, where):
    if rc != 0:
        raise TTError(rc, where)


def _dtype_code(t):
    import torch

    if t.dtype == torch.float64:
        return TT_F64
    if t.dtype == torch.float32:
        return TT_F32
    if t.dtype == torch.bfloat16:
        return TT_BF16
    raise TypeError(f"unsupported core dtype {t.dtype}")


class Desc:
    """A tt_desc over a list of device tensors (kept alive by this object)."""

    def __init__(self, cores, modes=None, ranks=None, dtype=None):
        n = len(cores)
        if n < 1 or n > TT_MAX_ORDER:
            raise ValueError("TT order must be in [1, 64]")
        self.tensors = list(cores)
        if modes is None:
            for c in cores:
                if c.dim() != 3:
                    raise ValueError("cores must be 3-D (R, I, R')")
            modes = [int(c.shape[1]) for c in cores]
            ranks = [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]
        for c in cores:
            if not c.is_cuda or not c.is_contiguous():
                raise ValueError("cores must be contiguous CUDA tensors")
        self.modes = list(modes)
        self.ranks = list(ranks)
        self.dtype = _dtype_code(cores[0]) if dtype is None else dtype
        self._modes = (c_int32 * n)(*self.modes)
        self._ranks = (c_int32 * (n + 1))(*self.ranks)
        self._cores = (c_void_p * n)(*[c.data_ptr() for c in cores])
        self.desc = TTDesc(n, self._modes, self._ranks, self._cores, self.dtype)

    @property
    def ref(self):
        return ctypes.byref(self.desc)


def _mask_arr(mask):
    return (c_uint8 * len(mask))(*[1 if v else 0 for v in mask])


def _stream_ptr(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


_ws_cache = {}


def _shape_key(d):
    """(order, modes, ranks, dtype) of a descriptor, read from its C struct."""
    t = d.desc
    n = int(t.order)
    return (n, tuple(t.modes[k] for k in range(n)), tuple(t.ranks[k] for k in range(n + 1)), int(t.dtype))


def workspace_bytes(op, xd, yd, mask=None, layout="chain", prec="native"):
    """tt_workspace_bytes; the answer depends on shapes, dtype, mask, layout and
    precision only, so it is remembered per such key (the autograd functions
    ask on every call)."""
    key = (op, _shape_key(xd), _shape_key(yd), None if mask is None else tuple(int(bool(v)) for v in mask),
           layout, prec)
    hit = _ws_cache.get(key)
    if hit is not None:
        return hit
    nb = c_size_t(0)
    m = _mask_arr(mask) if mask is not None else None
    check(
        lib().tt_workspace_bytes(op, xd.ref, yd.ref, m, LAYOUT[layout], PREC[prec], ctypes.byref(nb)),
        "tt_workspace_bytes",
    )
    if len(_ws_cache) < 4096:
        _ws_cache[key] = int(nb.value)
    return int(nb.value)


_shape_cache = {}


def partial_shape(xd, yd, mask, layout="chain"):
    """tt_partial_shape: (modes, ranks, perm) of the result; remembered per
    (shapes, dtype, mask, layout) like the workspace sizes."""
    key = (_shape_key(xd), _shape_key(yd), tuple(int(bool(v)) for v in mask), layout)
    hit = _shape_cache.get(key)
    if hit is not None:
        return list(hit[0]), list(hit[1]), list(hit[2])
    res = _partial_shape(xd, yd, mask, layout)
    if len(_shape_cache) < 4096:
        _shape_cache[key] = res
    return list(res[0]), list(res[1]), list(res[2])


def _partial_shape(xd, yd, mask, layout):
    n = xd.desc.order
    order = c_int32(0)
    modes = (c_int32 * (2 * n))()
    ranks = (c_int32 * (2 * n + 1))()
    perm = (c_int32 * (2 * n))()
    check(
        lib().tt_partial_shape(xd.ref, yd.ref, _mask_arr(mask), LAYOUT[layout], ctypes.byref(order), modes, ranks, perm),
        "tt_partial_shape",
    )
    o = order.value
    nfree = sum(1 for v in mask if not v)
    return list(modes[:o]), list(ranks[: o + 1]), list(perm[: 2 * nfree])


def status_tensor(device=None):
    import torch

    return torch.zeros(1, dtype=torch.int32, device=device or "cuda")


class FullContraction:
    """Pre-marshalled full contraction <X, Y> (re-usable, graph-capturable)."""

    def __init__(self, x, y, prec="native", split=False):
        import torch

        self.xd, self.yd = Desc(x), Desc(y)
        dev = x[0].device
        self.out = torch.empty(1, dtype=torch.float64, device=dev)  # every path writes it
        self.log2 = torch.zeros(1, dtype=torch.int64, device=dev) if split else None
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.prec = PREC[prec]
        nb = workspace_bytes(TT_OP_FULL, self.xd, self.yd, None, "chain", prec)
        self.ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
        self.ws_bytes = nb

    def __call__(self, stream=None):
        rc = lib().tt_contract_full(
            self.xd.ref,
            self.yd.ref,
            self.prec,
            c_void_p(self.out.data_ptr()),
            c_void_p(self.log2.data_ptr()) if self.log2 is not None else None,
            c_void_p(self.status.data_ptr()),
            c_void_p(self.ws.data_ptr()),
            c_size_t(self.ws_bytes),
            _stream_ptr(stream),
        )
        check(rc, "tt_contract_full")
        return self.out


class PartialContraction:
    """Pre-marshalled partial contraction; output cores allocated once."""

    def __init__(self, x, y, mask, layout="chain", prec="native", split=False, out=None):
        import torch

        self.xd, self.yd = Desc(x), Desc(y)
        self.mask = list(mask)
        self._mask = _mask_arr(mask)
        self.layout = LAYOUT[layout]
        self.prec = PREC[prec]
        dev = x[0].device
        modes, ranks, perm = partial_shape(self.xd, self.yd, mask, layout)
        self.perm = perm
        if out is None:
            out = [
                torch.empty((ranks[t], modes[t], ranks[t + 1]), dtype=x[0].dtype, device=dev)
                for t in range(len(modes))
            ]
        self.z = out
        self.zd = Desc(out)
        self.log2 = torch.zeros(1, dtype=torch.int64, device=dev) if split else None
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        nb = workspace_bytes(TT_OP_PARTIAL, self.xd, self.yd, mask, layout, prec)
        self.ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
        self.ws_bytes = nb

    def __call__(self, stream=None):
        rc = lib().tt_contract_partial(
            self.xd.ref,
            self.yd.ref,
            self._mask,
            self.layout,
            self.prec,
            self.zd.ref,
            c_void_p(self.log2.data_ptr()) if self.log2 is not None else None,
            c_void_p(self.status.data_ptr()),
            c_void_p(self.ws.data_ptr()),
            c_size_t(self.ws_bytes),
            _stream_ptr(stream),
        )
        check(rc, "tt_contract_partial")
        return self.z


def pairs_shape(xd, yd, pairs):
    """tt_pairs_shape: (modes, ranks, perm) of the chain-layout result of
    contracting mode pairs[t][0] of X with mode pairs[t][1] of Y."""
    n = xd.desc.order + yd.desc.order
    s = len(pairs)
    xm = (c_int32 * max(s, 1))(*[int(a) for a, _ in pairs])
    ym = (c_int32 * max(s, 1))(*[int(b) for _, b in pairs])
    order = c_int32(0)
    modes = (c_int32 * n)()
    ranks = (c_int32 * (n + 1))()
    perm = (c_int32 * n)()
    check(lib().tt_pairs_shape(xd.ref, yd.ref, s, xm, ym, ctypes.byref(order), modes, ranks, perm), "tt_pairs_shape")
    o = order.value
    return list(modes[:o]), list(ranks[: o + 1]), list(perm[:o])


class PairsContraction:
    """Pre-marshalled contraction of TTs of (possibly) different orders over
    end-block mode pairs (tt_contract_pairs); output cores allocated once."""

    def __init__(self, x, y, pairs, prec="native", split=False):
        import torch

        self.xd, self.yd = Desc(x), Desc(y)
        self.pairs = [(int(a), int(b)) for a, b in pairs]
        s = len(self.pairs)
        self._xm = (c_int32 * max(s, 1))(*[a for a, _ in self.pairs])
        self._ym = (c_int32 * max(s, 1))(*[b for _, b in self.pairs])
        self.prec = PREC[prec]
        dev = x[0].device
        modes, ranks, perm = pairs_shape(self.xd, self.yd, self.pairs)
        self.perm = perm
        self.z = [torch.empty((ranks[t], modes[t], ranks[t + 1]), dtype=x[0].dtype, device=dev) for t in range(len(modes))]
        self.zd = Desc(self.z)
        self.log2 = torch.zeros(1, dtype=torch.int64, device=dev) if split else None
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def __call__(self, stream=None):
        rc = lib().tt_contract_pairs(
            self.xd.ref,
            self.yd.ref,
            len(self.pairs),
            self._xm,
            self._ym,
            self.prec,
            self.zd.ref,
            c_void_p(self.log2.data_ptr()) if self.log2 is not None else None,
            c_void_p(self.status.data_ptr()),
            _stream_ptr(stream),
        )
        check(rc, "tt_contract_pairs")
        return self.z


def contract_pairs(x, y, pairs, prec="native", stream=None):
    """Contract mode pairs[t][0] of X with pairs[t][1] of Y (end blocks, any
    orders); returns (cores, perm) of the chain-layout result."""
    op = PairsContraction(x, y, pairs, prec)
    op(stream)
    return op.z, op.perm


class FactoredContraction:
    """Pre-marshalled partial contraction over any S in factored form
    (tt_contract_factored): the output arena allocated once.  After a call,
    ``runs()`` gives, for t = 0 .. m, None for an empty run (the identity) or
    (T_t, log2_t): the run matrix's mantissas (rows x cols) and its int64 row
    scales, views into the arena."""

    def __init__(self, x, y, mask):
        import torch

        self.xd, self.yd = Desc(x), Desc(y)
        self.mask = [int(v) for v in mask]
        self._mask = (c_uint8 * len(self.mask))(*self.mask)
        self.f = TTFactored()
        check(lib().tt_factored_shape(self.xd.ref, self.yd.ref, self._mask, ctypes.byref(self.f)), "tt_factored_shape")
        dev = x[0].device
        self.dtype = x[0].dtype
        self.arena = torch.empty(self.f.bytes, dtype=torch.uint8, device=dev)
        self.ws = torch.empty(max(self.f.ws_bytes, 1), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.free_pos = list(self.f.free_pos[: self.f.n_free])

    def __call__(self, stream=None):
        rc = lib().tt_contract_factored(self.xd.ref, self.yd.ref, self._mask, ctypes.byref(self.f),
                                        c_void_p(self.arena.data_ptr()), c_void_p(self.status.data_ptr()),
                                        c_void_p(self.ws.data_ptr()), self.f.ws_bytes, _stream_ptr(stream))
        check(rc, "tt_contract_factored")

    def runs(self):
        import torch

        eb = torch.finfo(self.dtype).bits // 8
        out = []
        for t in range(self.f.n_free + 1):
            r, c = self.f.rows[t], self.f.cols[t]
            if r == 0:
                out.append(None)
                continue
            o, ol = self.f.off_t[t], self.f.off_log2[t]
            tm = self.arena[o: o + r * c * eb].view(self.dtype).view(r, c)
            lg = self.arena[ol: ol + r * 8].view(torch.int64)
            out.append((tm, lg))
        return out


def contract_factored(x, y, mask, stream=None):
    """Partial contraction over S = {k: mask[k]} in factored form; returns
    (free positions, runs) as FactoredContraction.runs()."""
    op = FactoredContraction(x, y, mask)
    op(stream)
    return op.free_pos, op.runs()


def svd_workspace(modes, dtype, max_rank=0):
    """tt_svd_workspace: (cap_ranks, ws_bytes) of decomposing a dense tensor of
    the given modes."""
    n = len(modes)
    md = (c_int32 * n)(*[int(v) for v in modes])
    cap = (c_int32 * (n + 1))()
    ws = c_size_t(0)
    check(lib().tt_svd_workspace(n, md, int(dtype), int(max_rank), cap, ctypes.byref(ws)), "tt_svd_workspace")
    return list(cap), ws.value


class Decomposition:
    """Pre-marshalled TT-SVD of dense tensors of one shape and dtype
    (tt_svd): workspace, core buffers at their largest ranks and the rank and
    status words allocated once.  ``__call__(x)`` enqueues the decomposition;
    ``cores()`` reads the chosen ranks (a device-to-host copy: it waits for the
    call) and returns views of the cores at those ranks."""

    def __init__(self, modes, dtype, eps, max_rank=0, device=None):
        import torch

        self.modes = [int(v) for v in modes]
        self.tdtype = dtype
        self.code = TT_F64 if dtype == torch.float64 else TT_F32
        if dtype not in (torch.float64, torch.float32):
            raise TypeError(f"unsupported dtype {dtype}")
        self.eps = float(eps)
        self.max_rank = int(max_rank)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.cap, nbytes = svd_workspace(self.modes, self.code, self.max_rank)
        self.ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
        n = len(self.modes)
        self.buf = [torch.empty(self.cap[k] * self.modes[k] * self.cap[k + 1], dtype=dtype, device=dev) for k in range(n)]
        self._ptrs = (c_void_p * n)(*[b.data_ptr() for b in self.buf])
        self._modes = (c_int32 * n)(*self.modes)
        self.ranks = torch.zeros(n + 1, dtype=torch.int32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def __call__(self, x, stream=None):
        if list(x.shape) != self.modes or x.dtype != self.tdtype or not x.is_contiguous():
            raise ValueError("tensor does not match the decomposition's modes / dtype, or is not contiguous")
        rc = lib().tt_svd(c_void_p(x.data_ptr()), len(self.modes), self._modes, self.code, self.eps, self.max_rank,
                          self._ptrs, c_void_p(self.ranks.data_ptr()), c_void_p(self.status.data_ptr()),
                          c_void_p(self.ws.data_ptr()), self.ws.numel(), _stream_ptr(stream))
        check(rc, "tt_svd")

    def cores(self):
        r = [int(v) for v in self.ranks.cpu().tolist()]
        return [self.buf[k][: r[k] * self.modes[k] * r[k + 1]].view(r[k], self.modes[k], r[k + 1])
                for k in range(len(self.modes))]


class Rounding:
    """Pre-marshalled TT rounding (tt_round) of TTs of one shape: workspace,
    output buffers (at the input's ranks) and rank / status words allocated
    once.  ``__call__()`` enqueues; ``cores()`` reads the new ranks (waits for
    the call) and returns views of the rounded cores."""

    def __init__(self, cores, eps, max_rank=0):
        import torch

        self.xd = Desc(cores)
        self.eps = float(eps)
        self.max_rank = int(max_rank)
        ws = c_size_t(0)
        check(lib().tt_round_workspace(self.xd.ref, self.max_rank, ctypes.byref(ws)), "tt_round_workspace")
        dev = cores[0].device
        self.modes = [int(c.shape[1]) for c in cores]
        self.ws = torch.empty(max(ws.value, 1), dtype=torch.uint8, device=dev)
        self.buf = [torch.empty(c.numel(), dtype=c.dtype, device=dev) for c in cores]
        self._ptrs = (c_void_p * len(cores))(*[b.data_ptr() for b in self.buf])
        self.ranks = torch.zeros(len(cores) + 1, dtype=torch.int32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def __call__(self, stream=None):
        rc = lib().tt_round(self.xd.ref, self.eps, self.max_rank, self._ptrs, c_void_p(self.ranks.data_ptr()),
                            c_void_p(self.status.data_ptr()), c_void_p(self.ws.data_ptr()), self.ws.numel(),
                            _stream_ptr(stream))
        check(rc, "tt_round")

    def cores(self):
        r = [int(v) for v in self.ranks.cpu().tolist()]
        return [self.buf[k][: r[k] * self.modes[k] * r[k + 1]].view(r[k], self.modes[k], r[k + 1])
                for k in range(len(self.modes))]


def tt_round(cores, eps, max_rank=0, stream=None):
    """TT rounding of the CUDA cores within eps ||X||_F (tt_round; waits for
    the call to read the new ranks)."""
    op = Rounding([c.contiguous() for c in cores], eps, max_rank)
    op(stream)
    out = op.cores()
    if int(op.status.item()) != 0:
        raise ValueError("tt_round: the TT holds a non-finite value (TT_STATUS_NONFINITE)")
    return out


def round_merged(cores, eps, max_rank=0, stream=None):
    """TT rounding of merged-layout cores, (r, I J, r') as the library writes
    them or (r, I, J, r'): rounded as a TT of modes I J, returned in the
    shape given."""
    flat = [c if c.dim() == 3 else c.reshape(c.shape[0], c.shape[1] * c.shape[2], c.shape[3]) for c in cores]
    out = tt_round(flat, eps, max_rank, stream)
    return [o if c.dim() == 3 else o.view(o.shape[0], c.shape[1], c.shape[2], o.shape[2]) for o, c in zip(out, cores)]


_side_streams = {}


def _side_stream(device):
    """A second stream per device for independent work of one call."""
    import torch

    key = torch.device(device).index
    if key not in _side_streams:
        with torch.cuda.device(key):
            _side_streams[key] = torch.cuda.Stream()
    return _side_streams[key]


def tt_decompose(x, eps, max_rank=0, stream=None):
    """TT cores of the dense CUDA tensor x with ||x - TT||_F <= eps ||x||_F
    (tt_svd; waits for the call to read the ranks)."""
    op = Decomposition(list(x.shape), x.dtype, eps, max_rank, x.device)
    op(x.contiguous(), stream)
    cores = op.cores()
    if int(op.status.item()) != 0:
        raise ValueError("tt_svd: the tensor holds a non-finite value (TT_STATUS_NONFINITE)")
    return cores


def dense_permute(x, axes, out=None, stream=None):
    """out = x with axis t = axis axes[t] of x (tt_dense_permute)."""
    import torch

    n = x.dim()
    axes = [int(a) for a in axes]
    if out is None:
        out = torch.empty([x.shape[a] for a in axes], dtype=x.dtype, device=x.device)
    md = (c_int32 * n)(*[int(v) for v in x.shape])
    ax = (c_int32 * n)(*axes)
    check(lib().tt_dense_permute(c_void_p(x.data_ptr()), n, md, ax, _dtype_code(x), c_void_p(out.data_ptr()),
                                 _stream_ptr(stream)), "tt_dense_permute")
    return out


def contract_dense_pairs(x, y, pairs, eps, prec="native", max_rank=0, stream=None):
    """Eq. 8 over mode pairs of two dense CUDA tensors by way of TTs (Alg. 2):
    each operand's paired modes are brought to the front in pair order
    (tt_dense_permute), both are decomposed with accuracy eps (tt_svd), and
    the leading blocks are contracted (tt_contract_pairs).  Returns (cores,
    perm) of the chain-layout result; its represented tensor is within
    (eps_x + eps_y + eps_x eps_y) ||x|| ||y|| of Eq. 8's Z in Frobenius norm,
    plus rounding."""
    pairs = [(int(a), int(b)) for a, b in pairs]
    s = len(pairs)
    ax = [a for a, _ in pairs] + [k for k in range(x.dim()) if k not in {a for a, _ in pairs}]
    ay = [b for _, b in pairs] + [k for k in range(y.dim()) if k not in {b for _, b in pairs}]
    import torch

    cur = torch.cuda.current_stream(x.device) if stream is None else stream
    xp = x.contiguous() if ax == list(range(x.dim())) else dense_permute(x.contiguous(), ax, stream=cur)
    yp = y.contiguous() if ay == list(range(y.dim())) else dense_permute(y.contiguous(), ay, stream=cur)
    # the two decompositions are independent: Y's runs on a second stream,
    # forked from and joined back into the caller's
    dx = Decomposition(list(xp.shape), xp.dtype, eps, max_rank, xp.device)
    dy = Decomposition(list(yp.shape), yp.dtype, eps, max_rank, yp.device)
    side = _side_stream(x.device)
    side.wait_stream(cur)
    dx(xp, cur)
    dy(yp, side)
    cur.wait_stream(side)
    cur.synchronize()  # the chosen ranks size the contraction
    xc, yc = dx.cores(), dy.cores()
    if int(dx.status.item()) != 0 or int(dy.status.item()) != 0:
        raise ValueError("tt_svd: the tensor holds a non-finite value (TT_STATUS_NONFINITE)")
    op = PairsContraction(xc, yc, [(t, t) for t in range(s)], prec)
    op(stream)
    return op.z, op.perm


def contract_full(x, y, prec="native", split=False, stream=None):
    """<X, Y> on the device.  Returns a float64 CUDA tensor of shape (1,), or
    (mantissa, log2) tensors with split=True.  Raises on argument errors; for
    the device status bits (TT_STATUS_*) use :class:`FullContraction`, whose
    ``status`` tensor they land in."""
    op = FullContraction(x, y, prec, split)
    op(stream)
    if split:
        return op.out, op.log2
    return op.out


def contract_partial(x, y, mask, layout="chain", prec="native", split=False, stream=None):
    """Partial contraction over S = {k: mask[k]}.  Returns (cores, perm) or
    (cores, perm, log2) with split=True."""
    op = PartialContraction(x, y, mask, layout, prec, split)
    op(stream)
    if split:
        return op.z, op.perm, op.log2
    return op.z, op.perm


class BatchedContraction:
    """Many independent contractions in one persistent launch.

    ``pairs`` is a list of (x_cores, y_cores, mask) with mask None for a full
    contraction or a 0/1 list selecting an end block (chain layout).  Output
    cores of partial pairs are allocated here (``self.z[p]``); ``self.out``
    holds the value of every full pair.  The plan (tile per pair, LPT order) is
    built once; ``__call__`` only enqueues a memset and one kernel, so it can
    be captured with :meth:`graph`.
    """

    def __init__(self, pairs, prec="native", split=False):
        import torch

        n = len(pairs)
        if n < 1:
            raise ValueError("empty batch")
        dev = pairs[0][0][0].device
        self.xd = [Desc(p[0]) for p in pairs]
        self.yd = [Desc(p[1]) for p in pairs]
        self.masks = [None if p[2] is None else list(p[2]) for p in pairs]
        self.z = []
        self.zd = []
        self.perm = []
        for i, (x, y, mask) in enumerate(pairs):
            if mask is None:
                self.z.append(None)
                self.zd.append(None)
                self.perm.append(None)
                continue
            modes, ranks, perm = partial_shape(self.xd[i], self.yd[i], mask, "chain")
            z = [torch.empty((ranks[t], modes[t], ranks[t + 1]), dtype=x[0].dtype, device=dev) for t in range(len(modes))]
            self.z.append(z)
            self.zd.append(Desc(z))
            self.perm.append(perm)
        self._xarr = (TTDesc * n)(*[d.desc for d in self.xd])
        self._yarr = (TTDesc * n)(*[d.desc for d in self.yd])
        dummy = self.xd[0].desc
        self._zarr = (TTDesc * n)(*[(d.desc if d is not None else dummy) for d in self.zd])
        self._mask_bufs = [(_mask_arr(m) if m is not None else None) for m in self.masks]
        mp = (POINTER(c_uint8) * n)(
            *[(ctypes.cast(b, POINTER(c_uint8)) if b is not None else POINTER(c_uint8)()) for b in self._mask_bufs]
        )
        self._mp = mp
        batch = TTBatch(n, self._xarr, self._yarr, mp, self._zarr, PREC[prec])
        plan = c_void_p()
        pb = c_size_t(0)
        wb = c_size_t(0)
        check(lib().tt_batch_plan(ctypes.byref(batch), ctypes.byref(plan), ctypes.byref(pb), ctypes.byref(wb)), "tt_batch_plan")
        self.plan = plan
        host = torch.empty(pb.value, dtype=torch.uint8).pin_memory()
        check(lib().tt_batch_pack(plan, c_void_p(host.data_ptr()), pb), "tt_batch_pack")
        self.packed = host.to(dev)
        self.ws = torch.zeros(max(wb.value, 256), dtype=torch.uint8, device=dev)
        self.ws_bytes = self.ws.numel()
        self.n = n
        self.out = torch.zeros(n, dtype=torch.float64, device=dev)
        self.log2 = torch.zeros(n, dtype=torch.int64, device=dev) if split else None
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def tiles(self):
        t = c_int32(0)
        out = []
        for p in range(self.n):
            check(lib().tt_plan_info(self.plan, p, None, ctypes.byref(t)), "tt_plan_info")
            out.append(int(t.value))
        return out

    def __call__(self, stream=None):
        rc = lib().tt_contract_batched(
            self.plan,
            c_void_p(self.packed.data_ptr()),
            c_void_p(self.out.data_ptr()),
            c_void_p(self.log2.data_ptr()) if self.log2 is not None else None,
            c_void_p(self.status.data_ptr()),
            c_void_p(self.ws.data_ptr()),
            c_size_t(self.ws_bytes),
            _stream_ptr(stream),
        )
        check(rc, "tt_contract_batched")
        return self.out

    def call_noalloc(self, stream=None):
        """The same launch through tt_contract_batched_noalloc: no workspace,
        the work-queue counter lives in the library's static device array."""
        rc = lib().tt_contract_batched_noalloc(
            self.plan,
            c_void_p(self.packed.data_ptr()),
            c_void_p(self.out.data_ptr()),
            c_void_p(self.log2.data_ptr()) if self.log2 is not None else None,
            c_void_p(self.status.data_ptr()),
            _stream_ptr(stream),
        )
        check(rc, "tt_contract_batched_noalloc")
        return self.out

    def graph(self):
        """Capture one launch in a CUDA graph; returns the torch CUDAGraph."""
        import torch

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self()  # warm-up outside capture (sets kernel attributes)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self()
        return g

    def __del__(self):
        try:
            if getattr(self, "plan", None) is not None and self.plan.value:
                lib().tt_plan_free(self.plan)
                self.plan = None
        except Exception:
            pass


def autotune(dtype="f32", cache_path=None):
    """Run the batched-tile autotuner and write its cache file (see tt_autotune)."""
    code = {"f32": TT_F32, "f64": TT_F64}[dtype]
    path = cache_path or os.path.join(_HERE, f"autotune_{dtype}.txt")
    check(lib().tt_autotune(code, path.encode()), "tt_autotune")
    return path


def partial_k(x, y, mask, z, stream=None):
    """Chain-layout partial contraction into the output cores ``z`` that also
    fills a backward workspace (K and, for a leading block, every left
    environment of the block; tt_contract_partial_k).  Returns (ws, status); pass ``ws`` to
    :func:`backward` as ``fwd_ws``."""
    import torch

    xd, yd, zd = Desc(x), Desc(y), Desc(z)
    dev = x[0].device
    nb = workspace_bytes(TT_OP_BACKWARD, xd, yd, mask, "chain")
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = lib().tt_contract_partial_k(
        xd.ref, yd.ref, _mask_arr(mask), TT_P_NATIVE, zd.ref, None, c_void_p(status.data_ptr()),
        c_void_p(ws.data_ptr()), c_size_t(ws.numel()), _stream_ptr(stream),
    )
    check(rc, "tt_contract_partial_k")
    return ws, status


def backward(x, y, mask=None, cot=None, dz=None, ckpt_stride=0, stream=None, layout="chain", fwd_ws=None):
    """Gradients of a full (mask None; ``cot`` = float64 device scalar) or a
    chain-layout partial contraction (``dz`` = cotangents of the output cores)
    with respect to every core of x and y.  Returns (gx, gy, status).
    ``fwd_ws``: the workspace :func:`partial_k` filled in the forward pass
    (tt_contract_backward_k: K and the left environments are not computed
    again).  ``ckpt_stride`` is passed through (>= 0; every environment is
    kept whatever its value)."""
    import torch

    xd, yd = Desc(x), Desc(y)
    gx = [torch.empty_like(c) for c in x]
    gy = [torch.empty_like(c) for c in y]
    gxd, gyd = Desc(gx), Desc(gy)
    dev = x[0].device
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    nb = workspace_bytes(TT_OP_BACKWARD, xd, yd, mask, layout)
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
    m = _mask_arr(mask) if mask is not None else None
    dzd = Desc(dz) if dz is not None else None
    if cot is not None:
        cot = cot.detach().to(device=dev, dtype=torch.float64).reshape(1).contiguous()
    if fwd_ws is not None:
        rc = lib().tt_contract_backward_k(
            xd.ref, yd.ref, m, TT_P_NATIVE, dzd.ref, gxd.ref, gyd.ref, c_void_p(status.data_ptr()),
            c_void_p(fwd_ws.data_ptr()), c_size_t(fwd_ws.numel()), _stream_ptr(stream),
        )
        check(rc, "tt_contract_backward_k")
        return gx, gy, status
    rc = lib().tt_contract_backward(
        xd.ref,
        yd.ref,
        m,
        LAYOUT[layout],
        TT_P_NATIVE,
        c_void_p(cot.data_ptr()) if cot is not None else None,
        dzd.ref if dzd is not None else None,
        gxd.ref,
        gyd.ref,
        int(ckpt_stride),
        c_void_p(status.data_ptr()),
        c_void_p(ws.data_ptr()),
        c_size_t(ws.numel()),
        _stream_ptr(stream),
    )
    check(rc, "tt_contract_backward")
    return gx, gy, status


def _autograd():
    import torch

    class TTFull(torch.autograd.Function):
        """z = <X, Y> with a hand-written adjoint (tt_contract_backward)."""

        @staticmethod
        def forward(ctx, nx, *cores):
            x = [c.contiguous() for c in cores[:nx]]
            y = [c.contiguous() for c in cores[nx:]]
            op = FullContraction(x, y)
            op()
            ctx.nx = nx
            ctx.save_for_backward(*x, *y)
            return op.out.reshape(())

        @staticmethod
        def backward(ctx, g):
            saved = ctx.saved_tensors
            x, y = list(saved[: ctx.nx]), list(saved[ctx.nx :])
            gx, gy, _ = backward(x, y, None, cot=g)
            return (None, *gx, *gy)

    class TTPartial(torch.autograd.Function):
        """Chain-layout partial contraction with a hand-written adjoint."""

        @staticmethod
        def forward(ctx, nx, mask, *cores):
            x = [c.contiguous() for c in cores[:nx]]
            y = [c.contiguous() for c in cores[nx:]]
            modes, ranks, _ = partial_shape(Desc(x), Desc(y), mask, "chain")
            z = [torch.empty((ranks[t], modes[t], ranks[t + 1]), dtype=x[0].dtype, device=x[0].device)
                 for t in range(len(modes))]
            fws, _ = partial_k(x, y, mask, z)  # K and the left environments kept for the backward pass
            ctx.nx = nx
            ctx.mask = list(mask)
            ctx.save_for_backward(*x, *y, fws)
            return tuple(z)

        @staticmethod
        def backward(ctx, *gz):
            saved = ctx.saved_tensors
            x, y = list(saved[: ctx.nx]), list(saved[ctx.nx : -1])
            fws = saved[-1]
            xd, yd = Desc(x), Desc(y)
            modes, ranks, _ = partial_shape(xd, yd, ctx.mask, "chain")
            dz = []
            for t, g in enumerate(gz):
                if g is None:
                    g = torch.zeros((ranks[t], modes[t], ranks[t + 1]), dtype=x[0].dtype, device=x[0].device)
                dz.append(g.contiguous())
            gx, gy, _ = backward(x, y, ctx.mask, dz=dz, fwd_ws=fws)
            return (None, None, *gx, *gy)

    return TTFull, TTPartial


_fns = None


def tt_full(x, y):
    """Differentiable <X, Y> (float64 scalar)."""
    global _fns
    if _fns is None:
        _fns = _autograd()
    return _fns[0].apply(len(x), *x, *y)


def tt_partial(x, y, mask):
    """Differentiable chain-layout partial contraction; returns the output cores."""
    global _fns
    if _fns is None:
        _fns = _autograd()
    return list(_fns[1].apply(len(x), list(mask), *x, *y))


_ones_cache = {}


def tt_sum(cores):
    """Sum of all entries of a TT (= <Z, all-ones rank-1 TT>), differentiable.
    The all-ones TT is a constant, built once per (mode sizes, dtype, device)."""
    import torch

    key = (tuple(int(c.shape[1]) for c in cores), cores[0].dtype, cores[0].device)
    ones = _ones_cache.get(key)
    if ones is None:
        ones = [torch.ones((1, int(c.shape[1]), 1), dtype=c.dtype, device=c.device) for c in cores]
        if len(_ones_cache) < 256:
            _ones_cache[key] = ones
    return tt_full(list(cores), list(ones))
