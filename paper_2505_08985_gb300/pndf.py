"""Python binding of libpndf.so: the C ABI entry points under the same names.

Argument marshalling only: every step runs in the library's CUDA kernels.
Torch tensors provide device memory and the current CUDA stream.  Importing
this module loads the library and raises if it is missing; there is no
fallback path.
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import _build

PNDF_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA runtime error",
                4: "device wait timed out", 5: "device buffer capacity exceeded", 6: "unsupported request",
                7: "kernel recorded a device-side error"}

PNDF_TEXEL_F32X2 = 0
PNDF_TEXEL_F16X2 = 1
PNDF_BOUNDS_F32 = 0
PNDF_BOUNDS_F16_OUTWARD = 1
PNDF_MODE_HIERARCHY = 0
PNDF_MODE_FLAT = 1
PNDF_QF_FP64 = 1
PNDF_QF_INVALID = 4
PNDF_QF_OVERFLOW = 8

# pndf_query_stats, one int32 per field in this order
STATS_NAMES = ("nodes", "leaf_blocks", "tri_tests", "hits", "hit_hash", "fp64_tris", "degenerate", "quads",
               "cluster_checks", "clusters")
STATS_FIELDS = len(STATS_NAMES)


PNDF_KERNEL_GAUSS = 0  # footprint kernels (pndf_kernel): Gaussian cut at 4 sigma,
PNDF_KERNEL_DISK = 1   # disk and box of the (3 sigma)^2 footprint
PNDF_KERNEL_BOX = 2


class PndfError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn}: {STATUS_NAMES.get(code, code)} (status {code})")
        self.code = code


class _BuildParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("texel_fmt", ctypes.c_int32), ("bounds_fmt", ctypes.c_int32),
                ("leaf_level", ctypes.c_int32), ("clusters", ctypes.c_int32)]


class _EvalConfig(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("sort", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("tau", ctypes.c_float), ("kernel", ctypes.c_int32),
                ("jac_eps", ctypes.c_float), ("split", ctypes.c_int32),
                ("ev_begin", ctypes.c_void_p), ("ev_end", ctypes.c_void_p)]


class _Segment(ctypes.Structure):
    _fields_ = [("q", ctypes.c_void_p), ("order", ctypes.c_void_p), ("D", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("map", ctypes.c_int32), ("first", ctypes.c_int32),
                ("count", ctypes.c_int32), ("kind", ctypes.c_int32), ("omega", ctypes.c_void_p)]


PNDF_SEGMENT_PNDF = 0
PNDF_SEGMENT_PROJECTED_AREA = 1


class _ServerConfig(ctypes.Structure):
    _fields_ = [("max_segments", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("slots", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("tau", ctypes.c_float), ("jac_eps", ctypes.c_float), ("max_area_requests", ctypes.c_int32)]


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libpndf.so is not built ({path}); run __graft_entry__.build() or "
                          f"python -m paper_2505_08985_gb300._build")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "pndf_build_hierarchy": ([vp, ctypes.POINTER(_BuildParams), vp, ctypes.POINTER(vp)], i32),
        "pndf_free_hierarchy": ([vp], None),
        "pndf_update_hierarchy": ([vp, vp, vp], i32),
        "pndf_hierarchy_bytes": ([vp], ctypes.c_size_t),
        "pndf_cluster_level": ([vp, i32, vp, vp, vp], i32),
        "pndf_sample_normals": ([vp, vp, vp, i64, i32, ctypes.c_float, vp, vp, vp, vp], i32),
        "pndf_ggx_create": ([vp, vp, ctypes.POINTER(vp)], i32),
        "pndf_ggx_free": ([vp], None),
        "pndf_ggx_lambda": ([vp, vp, vp, i64, vp, vp], i32),
        "pndf_shadow_masking": ([vp, vp, vp, vp, i64, vp, vp], i32),
        "pndf_ggx_level": ([vp, i32, vp, vp], i32),
        "pndf_eval_batch": ([vp, vp, i64, vp, vp, vp, vp], i32),
        "pndf_eval_batch_ex": ([vp, vp, i64, vp, vp, vp, ctypes.POINTER(_EvalConfig), vp], i32),
        "pndf_eval_batch_host": ([vp, vp, i64, vp, vp], i32),
        "pndf_eval_batch_noalloc": ([vp, vp, i64, vp, vp, vp], i32),
        "pndf_eval_noalloc_max_queries": ([], i64),
        "pndf_diffuse_projected_area": ([vp, vp, vp, i64, vp, vp], i32),
        "pndf_device_status": ([vp, ctypes.POINTER(ctypes.c_uint32)], i32),
        "pndf_last_device_status": ([vp, vp, ctypes.POINTER(ctypes.c_uint32)], i32),
        "pndf_status_string": ([i32], ctypes.c_char_p),
        "pndf_version": ([], i32),
        "pndf_launch_count": ([], i64),
        "pndf_sort_queries": ([vp, vp, i64, vp, vp], i32),
        "pndf_shard_work": ([vp, vp, i64, i32, vp, vp], i32),
        "pndf_gather_queries": ([vp, vp, i64, i64, vp, vp], i32),
        "pndf_scatter_results": ([vp, vp, i64, i64, vp, vp], i32),
        "pndf_server_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(_ServerConfig), ctypes.POINTER(vp)], i32),
        "pndf_server_step": ([vp, ctypes.POINTER(_Segment), i32, vp, vp], i32),
        "pndf_server_sync": ([vp], i32),
        "pndf_server_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()


def _check(fn: str, code: int):
    if code != PNDF_OK:
        raise PndfError(fn, code)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _need(t: torch.Tensor, name: str, dtype=None, device=True, shape_last=None, rows=None, numel=None, on=None):
    """Check a tensor argument before any call into the library: its type,
    dtype, contiguity and shape (rows: the first dimension; numel: the total
    element count; shape_last: the last dimension), then its placement (a
    CUDA tensor, on device `on` when given).  The C ABI takes bare pointers,
    so a short buffer or one on another GPU would otherwise be written past
    its end or in another device's memory."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_last is not None and (t.dim() < 1 or t.shape[-1] != shape_last):
        raise ValueError(f"{name} must have last dimension {shape_last}, got shape {tuple(t.shape)}")
    if rows is not None and (t.dim() < 1 or t.shape[0] != rows):
        raise ValueError(f"{name} must have {rows} rows, got shape {tuple(t.shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got shape {tuple(t.shape)}")
    if device and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if on is not None and t.device != torch.device(on):
        raise ValueError(f"{name} must be on {on}, got {t.device}")


def _same_device(h, queries: torch.Tensor):
    if queries.device != h.device:
        raise ValueError(f"queries are on {queries.device} but the hierarchy is on {h.device}")


class Hierarchy:
    """A built pyramid (library-owned device memory) plus the map's size/format."""

    def __init__(self, handle: int, n: int, texel_fmt: int, bounds_fmt: int, device: torch.device,
                 clusters: bool = False):
        self.handle = handle
        self.n = n
        self.texel_fmt = texel_fmt
        self.bounds_fmt = bounds_fmt
        self.device = device
        self.clusters = clusters

    @property
    def nbytes(self) -> int:
        return int(LIB.pndf_hierarchy_bytes(self.handle)) if self.handle else 0

    def free(self):
        if self.handle:
            LIB.pndf_free_hierarchy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _texels(texels: torch.Tensor, device=None) -> torch.device:
    """Check a texel tensor: a CUDA tensor, or a page-locked CPU tensor that the
    build kernel reads directly (on `device`, default the current one).
    Returns the device the build runs on."""
    _need(texels, "texels", device=False, shape_last=2)
    if texels.is_cuda:
        return texels.device
    if not texels.is_pinned():
        raise ValueError("texels must be a CUDA tensor or a page-locked (pinned) CPU tensor")
    return torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)


def pndf_build_hierarchy(texels: torch.Tensor, bounds_fmt: int = PNDF_BOUNDS_F32, stream=None,
                         clusters: bool = False) -> Hierarchy:
    """texels: (N, N, 2) float32 or float16 CUDA tensor, or a pinned CPU tensor
    read directly by the build kernel; texel (i, j) at [j, i].
    clusters: also build the cluster hierarchy (Sec. 4.2, Eq. 7-8) for tau > 0."""
    dev = _texels(texels)
    if texels.dim() != 3 or texels.shape[0] != texels.shape[1]:
        raise ValueError("texels must be (N, N, 2)")
    if texels.dtype == torch.float32:
        tf = PNDF_TEXEL_F32X2
    elif texels.dtype == torch.float16:
        tf = PNDF_TEXEL_F16X2
    else:
        raise ValueError("texels must be float32 or float16")
    p = _BuildParams(int(texels.shape[0]), tf, int(bounds_fmt), 0, int(bool(clusters)))
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        _check("pndf_build_hierarchy", LIB.pndf_build_hierarchy(_ptr(texels), ctypes.byref(p), _stream(stream),
                                                                ctypes.byref(h)))
    return Hierarchy(h.value, int(texels.shape[0]), tf, int(bounds_fmt), dev, bool(clusters))


def pndf_update_hierarchy(h: Hierarchy, texels: torch.Tensor, stream=None) -> Hierarchy:
    """Rebuild h in place from new texels of the same size and dtype (a CUDA
    tensor, or a pinned CPU tensor read directly by the build kernel)."""
    dev = _texels(texels, h.device)
    tf = PNDF_TEXEL_F32X2 if texels.dtype == torch.float32 else PNDF_TEXEL_F16X2
    if texels.shape[0] != h.n or tf != h.texel_fmt:
        raise ValueError("texels must match the hierarchy's size and format")
    with torch.cuda.device(dev):
        _check("pndf_update_hierarchy", LIB.pndf_update_hierarchy(h.handle, _ptr(texels), _stream(stream)))
    return h


def pndf_free_hierarchy(h: Hierarchy):
    h.free()


def top_level(n: int) -> int:
    """Pyramid height L: the smallest L >= 2 with 2^L >= n - 1 quads per side."""
    L = 0
    while (1 << L) < n - 1:
        L += 1
    return max(L, 2)


PNDF_SF_INVALID = 1
PNDF_SF_OUTSIDE = 2


def pndf_sample_normals(h: Hierarchy, queries: torch.Tensor, uniforms: torch.Tensor, kernel: int = PNDF_KERNEL_GAUSS,
                        jac_eps: float = 0.0, stream=None):
    """Eq. 6 sampling: one normal per query record from its two uniforms
    (uniforms: (n, 2) float32 CUDA tensor in [0, 1]).  Returns m (n, 2)
    float32, triangle ids (n,) int32 (-1 where none) and flags (n,) int32."""
    n = _queries(queries)
    _same_device(h, queries)
    _need(uniforms, "uniforms", dtype=torch.float32, shape_last=2, rows=n, on=queries.device)
    m = torch.empty(n, 2, dtype=torch.float32, device=queries.device)
    tri = torch.empty(n, dtype=torch.int32, device=queries.device)
    flags = torch.empty(n, dtype=torch.int32, device=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_sample_normals", LIB.pndf_sample_normals(h.handle, _ptr(queries), _ptr(uniforms), n, int(kernel),
                                                              float(jac_eps), _ptr(m), _ptr(tri), _ptr(flags),
                                                              _stream(stream)))
    return m, tri, flags


class GGX:
    """The GGX projected-area fit of every mip node of a hierarchy (Eq. 12)."""

    def __init__(self, handle: int, n: int, device: torch.device):
        self.handle = handle
        self.n = n
        self.device = device

    def free(self):
        if self.handle:
            LIB.pndf_ggx_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def pndf_ggx_create(h: Hierarchy, stream=None) -> GGX:
    out = ctypes.c_void_p()
    with torch.cuda.device(h.device):
        _check("pndf_ggx_create", LIB.pndf_ggx_create(h.handle, _stream(stream), ctypes.byref(out)))
    return GGX(out.value, h.n, h.device)


def pndf_ggx_lambda(g: GGX, queries: torch.Tensor, omega: torch.Tensor, stream=None) -> torch.Tensor:
    """Lambda'(omega) per query footprint; omega (n, 3) float32 unit directions."""
    n = _queries(queries)
    _same_device(g, queries)
    _need(omega, "omega", dtype=torch.float32, shape_last=3, rows=n, on=queries.device)
    out = torch.empty(n, dtype=torch.float32, device=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_ggx_lambda", LIB.pndf_ggx_lambda(g.handle, _ptr(queries), _ptr(omega), n, _ptr(out),
                                                      _stream(stream)))
    return out


def pndf_shadow_masking(g: GGX, queries: torch.Tensor, wi: torch.Tensor, wo: torch.Tensor, stream=None):
    """Height-correlated G(wi, wo, m) per query (m = the query normal)."""
    n = _queries(queries)
    _same_device(g, queries)
    _need(wi, "wi", dtype=torch.float32, shape_last=3, rows=n, on=queries.device)
    _need(wo, "wo", dtype=torch.float32, shape_last=3, rows=n, on=queries.device)
    out = torch.empty(n, dtype=torch.float32, device=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_shadow_masking", LIB.pndf_shadow_masking(g.handle, _ptr(queries), _ptr(wi), _ptr(wo), n,
                                                              _ptr(out), _stream(stream)))
    return out


def pndf_ggx_level(g: GGX, level: int, stream=None) -> torch.Tensor:
    """Level `level` of the fit: (S, S, 3) float32 (O_xx, O_xy, O_yy), indexed [J, I]."""
    S = 1 << (top_level(g.n) - level)
    out = torch.empty(S, S, 3, dtype=torch.float32, device=g.device)
    with torch.cuda.device(g.device):
        _check("pndf_ggx_level", LIB.pndf_ggx_level(g.handle, int(level), _ptr(out), _stream(stream)))
    return out


def pndf_cluster_level(h: Hierarchy, level: int, stream=None):
    """Level `level` of the cluster hierarchy: records (S, S, 8) float32 as
    (c00, d10, d01, d11) pairs with corners c = c00 + d, and residuals (S, S),
    indexed [J, I] (S = 2^(L - level))."""
    S = 1 << (top_level(h.n) - level)
    rec = torch.empty(S, S, 8, dtype=torch.float32, device=h.device)
    e = torch.empty(S, S, dtype=torch.float32, device=h.device)
    with torch.cuda.device(h.device):
        _check("pndf_cluster_level", LIB.pndf_cluster_level(h.handle, int(level), _ptr(rec), _ptr(e),
                                                            _stream(stream)))
    return rec, e


def _queries(q: torch.Tensor):
    _need(q, "queries", dtype=torch.float32, shape_last=8)
    return q.shape[0]


def pndf_eval_batch(h: Hierarchy, queries: torch.Tensor, out: torch.Tensor | None = None,
                    flags: torch.Tensor | None = None, stats: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """queries: (nq, 8) float32 CUDA tensor (x, y, sxx, sxy, syy, ms, mt, pad).
    Returns D (nq,) float32.  flags: optional (nq,) int32; stats: optional (nq, STATS_FIELDS) int32."""
    return pndf_eval_batch_ex(h, queries, out=out, flags=flags, stats=stats, stream=stream)


def _event_handle(ev):
    """Raw cudaEvent_t of a torch.cuda.Event (created on first use)."""
    if ev is None:
        return None
    if not ev.cuda_event:
        ev.record()
    return int(ev.cuda_event)


PNDF_SORT_NONE = 0
PNDF_SORT_LEVEL_TILE = 1
PNDF_SORT_LEVEL_NORMAL = 2
PNDF_SORT_LEVEL_TILE_NORMAL = 3
PNDF_SORT_LEVEL_NORMAL_TILE = 4
PNDF_SORT_DEFAULT = PNDF_SORT_LEVEL_TILE


def pndf_eval_batch_ex(h: Hierarchy, queries: torch.Tensor, out=None, flags=None, stats=None, mode: int = 0,
                       sort: int = PNDF_SORT_DEFAULT, warps_per_cta: int = 0, ctas_per_sm: int = 0, stream=None,
                       ev_begin=None, ev_end=None, tau: float = 0.0, kernel: int = PNDF_KERNEL_GAUSS,
                       jac_eps: float = 0.0, split: bool = True) -> torch.Tensor:
    """ev_begin / ev_end: optional torch.cuda.Event recorded around the traversal kernel.
    tau > 0: the cluster cut of Sec. 4.2 (the hierarchy must be built with clusters=True).
    kernel: footprint kernel (PNDF_KERNEL_GAUSS, _DISK, _BOX).
    jac_eps > 0: the Jacobian clamp of Eq. 6 (e.g. 1e-6).
    split=False: one warp per query (large footprints are not divided among
    warps; the results are the same bits)."""
    nq = _queries(queries)
    _same_device(h, queries)
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    _need(out, "out", dtype=torch.float32, numel=nq, on=queries.device)
    if flags is not None:
        _need(flags, "flags", dtype=torch.int32, numel=nq, on=queries.device)
    if stats is not None:
        _need(stats, "stats", dtype=torch.int32, shape_last=STATS_FIELDS, rows=nq, on=queries.device)
    cfg = _EvalConfig(int(mode), int(sort), int(warps_per_cta), int(ctas_per_sm), float(tau), int(kernel),
                      float(jac_eps), 0 if split else -1,
                      _event_handle(ev_begin), _event_handle(ev_end))
    with torch.cuda.device(queries.device):
        _check("pndf_eval_batch_ex", LIB.pndf_eval_batch_ex(h.handle, _ptr(queries), nq, _ptr(out), _ptr(flags),
                                                            _ptr(stats), ctypes.byref(cfg), _stream(stream)))
    return out


def pndf_eval_batch_noalloc(h: Hierarchy, queries: torch.Tensor, out: torch.Tensor | None = None,
                            flags: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """pndf_eval_batch without any device allocation inside the library (the
    sort scratch is a fixed device array of the library; see pndf.h).  The
    caller supplies `out` if it must not allocate either."""
    nq = _queries(queries)
    _same_device(h, queries)
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    _need(out, "out", dtype=torch.float32, numel=nq, on=queries.device)
    if flags is not None:
        _need(flags, "flags", dtype=torch.int32, numel=nq, on=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_eval_batch_noalloc", LIB.pndf_eval_batch_noalloc(h.handle, _ptr(queries), nq, _ptr(out),
                                                                      _ptr(flags), _stream(stream)))
    return out


def pndf_eval_noalloc_max_queries() -> int:
    return int(LIB.pndf_eval_noalloc_max_queries())


def pndf_eval_batch_host(h: Hierarchy, queries_host: torch.Tensor, out_host: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """Host-buffer variant: queries_host (nq, 8) float32 CPU (pinned for full speed)."""
    _need(queries_host, "queries_host", dtype=torch.float32, device=False, shape_last=8)
    if queries_host.is_cuda:
        raise ValueError("queries_host must be a CPU tensor")
    nq = queries_host.shape[0]
    if out_host is None:
        out_host = torch.empty(nq, dtype=torch.float32, pin_memory=queries_host.is_pinned())
    _need(out_host, "out_host", dtype=torch.float32, device=False, numel=nq)
    if out_host.is_cuda:
        raise ValueError("out_host must be a CPU tensor")
    with torch.cuda.device(h.device):
        _check("pndf_eval_batch_host", LIB.pndf_eval_batch_host(h.handle, _ptr(queries_host), nq, _ptr(out_host),
                                                                _stream(stream)))
    return out_host


def pndf_diffuse_projected_area(h: Hierarchy, queries: torch.Tensor, omega: torch.Tensor,
                                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """omega: (nq, 3) float32 CUDA unit directions with w_z > 0.  Returns P (nq,)."""
    nq = _queries(queries)
    _same_device(h, queries)
    _need(omega, "omega", dtype=torch.float32, shape_last=3, rows=nq, on=queries.device)
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    _need(out, "out", dtype=torch.float32, numel=nq, on=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_diffuse_projected_area", LIB.pndf_diffuse_projected_area(h.handle, _ptr(queries), _ptr(omega), nq,
                                                                              _ptr(out), _stream(stream)))
    return out


def pndf_device_status(stream=None) -> int:
    """Read and clear the device status word; returns the PNDF_QF_* bits (0 if clean)."""
    bits = ctypes.c_uint32(0)
    code = LIB.pndf_device_status(_stream(stream), ctypes.byref(bits))
    if code not in (PNDF_OK, 7):
        raise PndfError("pndf_device_status", code)
    return int(bits.value)


def pndf_last_device_status(h: Hierarchy, stream=None) -> int:
    """Read and clear hierarchy h's status word; returns the PNDF_QF_* bits
    that kernels recorded on h (0 if none)."""
    bits = ctypes.c_uint32(0)
    with torch.cuda.device(h.device):
        code = LIB.pndf_last_device_status(h.handle, _stream(stream), ctypes.byref(bits))
    if code not in (PNDF_OK, 7):
        raise PndfError("pndf_last_device_status", code)
    return int(bits.value)


def pndf_status_string(code: int) -> str:
    return LIB.pndf_status_string(int(code)).decode()


def pndf_version() -> int:
    return int(LIB.pndf_version())


def pndf_launch_count() -> int:
    return int(LIB.pndf_launch_count())


def pndf_sort_queries(h: Hierarchy, queries: torch.Tensor, order: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Evaluation order of a batch (int32 permutation, largest footprints first)."""
    nq = _queries(queries)
    _same_device(h, queries)
    if order is None:
        order = torch.empty(nq, dtype=torch.int32, device=queries.device)
    _need(order, "order", dtype=torch.int32, numel=nq, on=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_sort_queries", LIB.pndf_sort_queries(h.handle, _ptr(queries), nq, _ptr(order), _stream(stream)))
    return order


def pndf_shard_work(queries: torch.Tensor, order: torch.Tensor, block: int = 4096, stream=None) -> torch.Tensor:
    """Estimated work per block of `block` positions of the evaluation order
    (float64, ceil(nq / block) entries); see pndf.h."""
    nq = _queries(queries)
    _need(order, "order", dtype=torch.int32, numel=nq, on=queries.device)
    out = torch.empty((nq + block - 1) // block, dtype=torch.float64, device=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_shard_work", LIB.pndf_shard_work(_ptr(queries), _ptr(order), nq, int(block), _ptr(out),
                                                      _stream(stream)))
    return out


def pndf_gather_queries(queries: torch.Tensor, order: torch.Tensor, first: int, count: int, out=None,
                        stream=None) -> torch.Tensor:
    """queries[order[first:first + count]] as a contiguous (count, 8) batch."""
    nq = _queries(queries)
    _need(order, "order", dtype=torch.int32, numel=nq, on=queries.device)
    if first < 0 or count < 0 or first + count > nq:
        raise ValueError(f"range [{first}, {first + count}) outside the {nq}-query order")
    if out is None:
        out = torch.empty(count, 8, dtype=torch.float32, device=queries.device)
    _need(out, "out", dtype=torch.float32, shape_last=8, rows=count, on=queries.device)
    with torch.cuda.device(queries.device):
        _check("pndf_gather_queries", LIB.pndf_gather_queries(_ptr(queries), _ptr(order), int(first), int(count),
                                                              _ptr(out), _stream(stream)))
    return out


def pndf_scatter_results(D_shard: torch.Tensor, order: torch.Tensor, first: int, out: torch.Tensor, stream=None):
    """out[order[first + k]] = D_shard[k] for every k of the shard."""
    count = D_shard.numel()
    _need(out, "out", dtype=torch.float32)
    _need(order, "order", dtype=torch.int32, numel=out.numel(), on=out.device)
    _need(D_shard, "D_shard", dtype=torch.float32, on=out.device)
    if first < 0 or first + count > out.numel():
        raise ValueError(f"range [{first}, {first + count}) outside the {out.numel()}-query order")
    with torch.cuda.device(out.device):
        _check("pndf_scatter_results", LIB.pndf_scatter_results(_ptr(D_shard), _ptr(order), int(first), int(count),
                                                                _ptr(out), _stream(stream)))
    return out


class Server:
    """A serving table of resident hierarchies (see pndf_server_create)."""

    def __init__(self, handle: int, maps: list, max_segments: int, slots: int = 4):
        self.handle = handle
        self.maps = list(maps)
        self.max_segments = max_segments
        self.slots = slots
        self._segs = (_Segment * max_segments)()

    def destroy(self):
        if self.handle:
            LIB.pndf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pndf_server_create(maps: list, max_segments: int = 1024, warps_per_cta: int = 0, ctas_per_sm: int = 0,
                       slots: int = 0, kernel: int = PNDF_KERNEL_GAUSS, tau: float = 0.0,
                       jac_eps: float = 0.0, max_area_requests: int = 0) -> Server:
    """kernel / tau / jac_eps: what every served query evaluates, as in
    pndf_eval_batch_ex (tau > 0 needs maps built with clusters=True).
    max_area_requests: projected-area requests a step can hold (0: none)."""
    arr = (ctypes.c_void_p * len(maps))(*[m.handle for m in maps])
    cfg = _ServerConfig(int(max_segments), int(warps_per_cta), int(ctas_per_sm), int(slots), int(kernel),
                        float(tau), float(jac_eps), int(max_area_requests))
    h = ctypes.c_void_p()
    with torch.cuda.device(maps[0].device):
        _check("pndf_server_create", LIB.pndf_server_create(arr, len(maps), ctypes.byref(cfg), ctypes.byref(h)))
    return Server(h.value, maps, int(max_segments), int(slots) or 4)


def pndf_server_step(srv: Server, segments: list, stream=None, ev_done=None):
    """segments: list of (map_index, queries, order_or_None, D, flags_or_None,
    first, count) for P-NDF slices, or with two more items (kind, omega) where
    kind = PNDF_SEGMENT_PROJECTED_AREA and omega is the requests' (n, 3)
    directions (D then receives P); tensors must stay alive until the step
    completes."""
    n = len(segments)
    if n > srv.max_segments:
        raise ValueError("too many segments for this server")
    segs = srv._segs
    for i, seg in enumerate(segments):
        mi, q, order, D, flags, first, count = seg[:7]
        kind, omega = (seg[7], seg[8]) if len(seg) > 7 else (PNDF_SEGMENT_PNDF, None)
        # (a map index out of range is the library's to reject)
        dev = srv.maps[int(mi)].device if 0 <= int(mi) < len(srv.maps) else None
        _need(q, f"segment {i} queries", dtype=torch.float32, shape_last=8, on=dev)
        nq = q.shape[0]
        _need(D, f"segment {i} D", dtype=torch.float32, numel=nq, on=dev)
        if flags is not None:
            _need(flags, f"segment {i} flags", dtype=torch.int32, numel=nq, on=dev)
        if kind == PNDF_SEGMENT_PROJECTED_AREA:
            if order is not None or flags is not None:
                raise ValueError(f"segment {i}: projected-area segments take no order or flags")
            _need(omega, f"segment {i} omega", dtype=torch.float32, shape_last=3, rows=nq, on=dev)
        span = nq
        if order is not None:
            _need(order, f"segment {i} order", dtype=torch.int32, on=dev)
            span = order.numel()
        if first < 0 or count < 0 or first + count > span:
            raise ValueError(f"segment {i}: slice [{first}, {first + count}) outside its {span} entries")
        sg = segs[i]
        sg.q = _ptr(q)
        sg.order = _ptr(order)
        sg.D = _ptr(D)
        sg.flags = _ptr(flags)
        sg.map = int(mi)
        sg.first = int(first)
        sg.count = int(count)
        sg.kind = int(kind)
        sg.omega = _ptr(omega)
    _check("pndf_server_step", LIB.pndf_server_step(srv.handle, segs, n, _stream(stream), _event_handle(ev_done)))


def pndf_server_sync(srv: Server):
    _check("pndf_server_sync", LIB.pndf_server_sync(srv.handle))


def pndf_server_destroy(srv: Server):
    srv.destroy()
