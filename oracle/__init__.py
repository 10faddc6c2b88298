"""FP64 CPU oracle: Python entry points over ``pndf_oracle.c``.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package.  It imports nothing from the
CUDA package and the CUDA package imports nothing from it.

Functions
---------
pndf(st, queries, kernel=0, jac_eps=0) -> D (float64), flags (uint32), hits (int64), hit_hash (uint32);
                              kernel 0 Gaussian (4-sigma cut), 1 disk, 2 box (1.5 sigma);
                              jac_eps > 0: the Jacobian clamp of Eq. 6 (equilateral replacements)
sample(st, queries, U, kernel=0, jac_eps=0) -> m (n, 2), triangle ids, flags: Eq. 6 sampling
cluster_fits(st)           -> ClusterFits: corner normals and residual of every node, Eq. 7-8
cluster_fit(st, l, I, J)   -> (c (4, 2), e) for one node, or None outside the map
pndf_cluster(st, queries, tau, fits=None) -> as pndf, with the cluster cut e <= r_x r_y tau
projarea(st, queries, w)   -> P (float64)
ggx_fits(st)               -> Omega per mip node (Eq. 12 fit; box filter per node)
ggx_lambda(Omega, N, q, w) -> GGX Smith Lambda'(w) at each footprint
shadow_masking(Omega, N, q, wi, wo) -> height-correlated G (Sec. 4.3)
tri_integral(n0, n1, n2, w) -> integral of max(m~.w, 0)/m~_z over one normal triangle

``st`` is an (N, N, 2) array (texel (i, j) at ``st[j, i]``); ``queries`` an
(n, >=7) array of (x, y, sxx, sxy, syy, ms, mt).  Inputs are converted to
float64 exactly.  Work is split over host threads by query range (ctypes
releases the GIL during each call).

Flag bits (per query): 1 near an edge (1e-6 in normal space), 2 a hit within
1e-4 of the q = 16 cut, 4 near a zero-area triangle, 8 a hit on a triangle of
normal-space area < 1e-10, 16 invalid covariance, 32 (cluster cut only) a
node whose normal hull holds m has a residual within 1e-5 (relative) of
r_x r_y tau, or the entry radius is within 3e-5 of a power of two: FP32
and FP64 may then take the cut differently.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pndf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

F_NEAR_EDGE = 1
F_NEAR_CUT = 2
F_DEGENERATE = 4
F_TINY = 8
F_INVALID = 16
F_NEAR_TAU = 32
F_OUTSIDE = 64  # (sampling) the sampled uv point lies outside the map
F_EXCLUDE = F_NEAR_EDGE | F_NEAR_CUT | F_DEGENERATE | F_INVALID | F_NEAR_TAU
KERNEL_GAUSS, KERNEL_DISK, KERNEL_BOX = 0, 1, 2  # footprint kernels (see pndf_oracle.c)
GL_POINTS = 16

_lock = threading.Lock()
_default = None


def build(force: bool = False, src: str = _SRC, out: str = _SO) -> str:
    """Compile the oracle with gcc (no FP contraction, so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
                        "-shared", "-fPIC", "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, out)
    return out


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _as_map(st) -> np.ndarray:
    st = np.asarray(st.cpu() if hasattr(st, "cpu") else st)
    assert st.ndim == 3 and st.shape[0] == st.shape[1] and st.shape[2] == 2, st.shape
    return np.ascontiguousarray(st, dtype=np.float64)


def _as_queries(q) -> np.ndarray:
    q = np.asarray(q.cpu() if hasattr(q, "cpu") else q)
    return np.ascontiguousarray(q[:, :7], dtype=np.float64)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def top_level(N: int) -> int:
    """Pyramid height: the smallest L >= 2 with 2^L >= N - 1 quads per side."""
    L = 0
    while (1 << L) < N - 1:
        L += 1
    return max(L, 2)


class ClusterFits:
    """Corner normals c (n_nodes, 8) and residuals e (n_nodes,) of every node
    at levels 2..L, level by level, row-major (J, I) within a level; e = inf
    where the node has no cluster (not entirely inside the map).  hull
    (n_nodes, 4): box of the normals of the node's texels, its cluster corners
    and its children's hulls."""

    def __init__(self, N: int):
        self.N = N
        self.L = top_level(N)
        self.offsets = {}
        off = 0
        for l in range(2, self.L + 1):
            self.offsets[l] = off
            off += (1 << (self.L - l)) ** 2
        self.c = np.zeros((off, 8), np.float64)
        self.e = np.full(off, np.inf, np.float64)
        self.hull = np.zeros((off, 4), np.float64)  # normal hull of each node's pieces

    def level(self, l: int):
        S = 1 << (self.L - l)
        o = self.offsets[l]
        return self.c[o:o + S * S].reshape(S, S, 4, 2), self.e[o:o + S * S].reshape(S, S)


GGX_DIRECTIONS = 16
GGX_WZ = 0.3


def ggx_dirs(K: int = GGX_DIRECTIONS, wz: float = GGX_WZ) -> np.ndarray:
    """The fit directions: K azimuths 2 pi k / K at height w_z (grazing-ish)."""
    phi = 2.0 * np.pi * np.arange(K) / K
    r = math.sqrt(1.0 - wz * wz)
    return np.stack([r * np.cos(phi), r * np.sin(phi), np.full(K, wz)], 1)


def _chunks(n, threads, min_chunk=16):
    nchunks = max(1, min(threads * 8, (n + min_chunk - 1) // min_chunk))
    edges = np.linspace(0, n, nchunks + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


class Oracle:
    """The oracle bound to one compiled library (the default build, or a
    deliberately altered copy in the mutation tests)."""

    F_NEAR_EDGE = F_NEAR_EDGE
    F_NEAR_CUT = F_NEAR_CUT
    F_DEGENERATE = F_DEGENERATE
    F_TINY = F_TINY
    F_INVALID = F_INVALID
    F_NEAR_TAU = F_NEAR_TAU
    F_OUTSIDE = F_OUTSIDE
    F_EXCLUDE = F_EXCLUDE
    ggx_dirs = staticmethod(ggx_dirs)

    def __init__(self, so_path: str):
        lib = ctypes.CDLL(so_path)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_pndf.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                    dp, u32p, i64p, u32p]
        lib.oracle_sample.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_double, dp, i64p, u32p]
        lib.oracle_sample.restype = None
        lib.oracle_pndf.restype = None
        lib.oracle_projarea.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                                        ctypes.c_int]
        lib.oracle_projarea.restype = None
        lib.oracle_tri_integral.argtypes = [ctypes.c_double] * 9
        lib.oracle_tri_integral.restype = ctypes.c_double
        lib.oracle_ggx_node_P.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                          dp, dp, ctypes.c_int, dp]
        lib.oracle_ggx_node_P.restype = ctypes.c_int
        lib.oracle_ggx_fit.argtypes = [dp, dp, ctypes.c_int, dp]
        lib.oracle_ggx_fit.restype = ctypes.c_int
        lib.oracle_ggx_build.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                         dp, dp, ctypes.c_int, dp]
        lib.oracle_ggx_build.restype = None
        lib.oracle_ggx_lambda.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int64, ctypes.c_int64, dp]
        lib.oracle_ggx_lambda.restype = None
        lib.oracle_shadow_masking.argtypes = [dp, ctypes.c_int, dp, dp, dp, ctypes.c_int64, ctypes.c_int64, dp]
        lib.oracle_shadow_masking.restype = None
        lib.oracle_cluster_fit.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_cluster_fit.restype = ctypes.c_int
        lib.oracle_cluster_build.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_cluster_build.restype = None
        lib.oracle_cluster_hulls.argtypes = [dp, ctypes.c_int, dp, dp, dp]
        lib.oracle_cluster_hulls.restype = None
        lib.oracle_pndf_cluster.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_double, dp, dp, dp, dp, u32p, i64p, u32p]
        lib.oracle_pndf_cluster.restype = None
        self.lib = lib

    def pndf(self, st, queries, threads: int | None = None, kernel: int = 0, jac_eps: float = 0.0):
        lib = self.lib
        stm = _as_map(st)
        q = _as_queries(queries)
        n = q.shape[0]
        D = np.zeros(n, np.float64)
        flags = np.zeros(n, np.uint32)
        hits = np.zeros(n, np.int64)
        hh = np.zeros(n, np.uint32)
        N = stm.shape[0]

        def run(r):
            lib.oracle_pndf(_ptr(stm, ctypes.c_double), N, _ptr(q, ctypes.c_double), r[0], r[1], int(kernel),
                            float(jac_eps), _ptr(D, ctypes.c_double), _ptr(flags, ctypes.c_uint32),
                            _ptr(hits, ctypes.c_int64), _ptr(hh, ctypes.c_uint32))

        threads = threads or default_threads()
        if n:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                list(ex.map(run, _chunks(n, threads)))
        return D, flags, hits, hh

    def sample(self, st, queries, uniforms, kernel: int = 0, jac_eps: float = 0.0, threads: int | None = None):
        """Eq. 6 sampling: one normal per query record from its two uniforms.
        Returns m (n, 2), triangle ids (n,) (-1 where none) and flags (n,)."""
        lib = self.lib
        stm = _as_map(st)
        q = _as_queries(queries)
        U = np.ascontiguousarray(np.asarray(uniforms.cpu() if hasattr(uniforms, "cpu") else uniforms)[:, :2],
                                 dtype=np.float64)
        n = q.shape[0]
        assert U.shape[0] == n
        m = np.zeros((n, 2), np.float64)
        tri = np.zeros(n, np.int64)
        flags = np.zeros(n, np.uint32)
        N = stm.shape[0]

        def run(r):
            lib.oracle_sample(_ptr(stm, ctypes.c_double), N, _ptr(q, ctypes.c_double), _ptr(U, ctypes.c_double),
                              r[0], r[1], int(kernel), float(jac_eps), _ptr(m, ctypes.c_double),
                              _ptr(tri, ctypes.c_int64), _ptr(flags, ctypes.c_uint32))

        threads = threads or default_threads()
        if n:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                list(ex.map(run, _chunks(n, threads, 1024)))
        return m, tri, flags

    def cluster_fit(self, st, l: int, I: int, J: int):
        stm = _as_map(st)
        c = np.zeros(8, np.float64)
        e = np.zeros(1, np.float64)
        ok = self.lib.oracle_cluster_fit(_ptr(stm, ctypes.c_double), stm.shape[0], l, I, J,
                                         _ptr(c, ctypes.c_double), _ptr(e, ctypes.c_double))
        return (c.reshape(4, 2), float(e[0])) if ok else None

    def cluster_fits(self, st, threads: int | None = None) -> ClusterFits:
        stm = _as_map(st)
        N = stm.shape[0]
        fits = ClusterFits(N)
        jobs = []
        for l in range(2, fits.L + 1):
            S = 1 << (fits.L - l)
            jobs += [(l, a, b) for a, b in _chunks(S, threads or default_threads(), 1)]
        jobs.sort(key=lambda j: -j[0])  # the costly top levels first

        def run(j):
            self.lib.oracle_cluster_build(_ptr(stm, ctypes.c_double), N, j[0], j[1], j[2],
                                          _ptr(fits.c, ctypes.c_double), _ptr(fits.e, ctypes.c_double))

        with ThreadPoolExecutor(max_workers=threads or default_threads()) as ex:
            list(ex.map(run, jobs))
        self.lib.oracle_cluster_hulls(_ptr(stm, ctypes.c_double), N, _ptr(fits.c, ctypes.c_double),
                                      _ptr(fits.e, ctypes.c_double), _ptr(fits.hull, ctypes.c_double))
        return fits

    def pndf_cluster(self, st, queries, tau: float, fits: ClusterFits | None = None, threads: int | None = None,
                     kernel: int = 0):
        lib = self.lib
        stm = _as_map(st)
        q = _as_queries(queries)
        n = q.shape[0]
        N = stm.shape[0]
        fits = fits if fits is not None else self.cluster_fits(stm, threads)
        assert fits.N == N
        D = np.zeros(n, np.float64)
        flags = np.zeros(n, np.uint32)
        hits = np.zeros(n, np.int64)
        hh = np.zeros(n, np.uint32)

        def run(r):
            lib.oracle_pndf_cluster(_ptr(stm, ctypes.c_double), N, _ptr(q, ctypes.c_double), r[0], r[1],
                                    int(kernel), float(tau), _ptr(fits.c, ctypes.c_double), _ptr(fits.e, ctypes.c_double),
                                    _ptr(fits.hull, ctypes.c_double), _ptr(D, ctypes.c_double), _ptr(flags, ctypes.c_uint32),
                                    _ptr(hits, ctypes.c_int64), _ptr(hh, ctypes.c_uint32))

        threads = threads or default_threads()
        if n:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                list(ex.map(run, _chunks(n, threads)))
        return D, flags, hits, hh

    # -- GGX projected-area fit per mip node (Eq. 12) and shadow-masking --

    def ggx_node_P(self, st, l: int, I: int, J: int, dirs=None):
        stm = _as_map(st)
        dirs = np.ascontiguousarray(ggx_dirs() if dirs is None else dirs, dtype=np.float64)
        glx, glw = (np.ascontiguousarray(a) for a in np.polynomial.legendre.leggauss(GL_POINTS))
        P = np.zeros(dirs.shape[0], np.float64)
        ok = self.lib.oracle_ggx_node_P(_ptr(stm, ctypes.c_double), stm.shape[0], l, I, J, _ptr(dirs, ctypes.c_double),
                                        dirs.shape[0], _ptr(glx, ctypes.c_double), _ptr(glw, ctypes.c_double),
                                        GL_POINTS, _ptr(P, ctypes.c_double))
        return P if ok else None

    def ggx_fit(self, P, dirs=None):
        dirs = np.ascontiguousarray(ggx_dirs() if dirs is None else dirs, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        O = np.zeros(3, np.float64)
        ok = self.lib.oracle_ggx_fit(_ptr(P, ctypes.c_double), _ptr(dirs, ctypes.c_double), dirs.shape[0],
                                     _ptr(O, ctypes.c_double))
        return O if ok else None

    def ggx_fits(self, st, dirs=None, threads: int | None = None):
        """Omega (n_nodes, 3) = (O_xx, O_xy, O_yy) of every node of levels 2..L
        (the ClusterFits layout; NaN without a fit)."""
        stm = _as_map(st)
        N = stm.shape[0]
        dirs = np.ascontiguousarray(ggx_dirs() if dirs is None else dirs, dtype=np.float64)
        glx, glw = (np.ascontiguousarray(a) for a in np.polynomial.legendre.leggauss(GL_POINTS))
        lay = ClusterFits(N)
        O = np.full((lay.c.shape[0], 3), np.nan, np.float64)
        jobs = []
        for l in range(2, lay.L + 1):
            S = 1 << (lay.L - l)
            jobs += [(l, a, b) for a, b in _chunks(S, threads or default_threads(), 1)]
        jobs.sort(key=lambda j: -j[0])

        def run(j):
            self.lib.oracle_ggx_build(_ptr(stm, ctypes.c_double), N, j[0], j[1], j[2], _ptr(dirs, ctypes.c_double),
                                      dirs.shape[0], _ptr(glx, ctypes.c_double), _ptr(glw, ctypes.c_double),
                                      GL_POINTS, _ptr(O, ctypes.c_double))

        with ThreadPoolExecutor(max_workers=threads or default_threads()) as ex:
            list(ex.map(run, jobs))
        return O

    def ggx_lambda(self, Omega, N: int, queries, omega):
        q = _as_queries(queries)
        w = np.ascontiguousarray(np.asarray(omega.cpu() if hasattr(omega, "cpu") else omega)[:, :3], dtype=np.float64)
        O = np.ascontiguousarray(Omega, dtype=np.float64)
        out = np.zeros(q.shape[0], np.float64)
        if q.shape[0]:
            self.lib.oracle_ggx_lambda(_ptr(O, ctypes.c_double), N, _ptr(q, ctypes.c_double), _ptr(w, ctypes.c_double),
                                       0, q.shape[0], _ptr(out, ctypes.c_double))
        return out

    def shadow_masking(self, Omega, N: int, queries, wi, wo):
        q = _as_queries(queries)
        a = np.ascontiguousarray(np.asarray(wi.cpu() if hasattr(wi, "cpu") else wi)[:, :3], dtype=np.float64)
        b = np.ascontiguousarray(np.asarray(wo.cpu() if hasattr(wo, "cpu") else wo)[:, :3], dtype=np.float64)
        O = np.ascontiguousarray(Omega, dtype=np.float64)
        out = np.zeros(q.shape[0], np.float64)
        if q.shape[0]:
            self.lib.oracle_shadow_masking(_ptr(O, ctypes.c_double), N, _ptr(q, ctypes.c_double),
                                           _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double), 0, q.shape[0],
                                           _ptr(out, ctypes.c_double))
        return out

    def projarea(self, st, queries, omega, threads: int | None = None):
        lib = self.lib
        stm = _as_map(st)
        q = _as_queries(queries)
        w = np.ascontiguousarray(np.asarray(omega.cpu() if hasattr(omega, "cpu") else omega)[:, :3],
                                 dtype=np.float64)
        n = q.shape[0]
        assert w.shape[0] == n
        P = np.zeros(n, np.float64)
        N = stm.shape[0]
        # Gauss-Legendre nodes for the collapsed-triangle uv form (numpy's leggauss)
        glx, glw = (np.ascontiguousarray(a) for a in np.polynomial.legendre.leggauss(GL_POINTS))

        def run(r):
            lib.oracle_projarea(_ptr(stm, ctypes.c_double), N, _ptr(q, ctypes.c_double),
                                _ptr(w, ctypes.c_double), r[0], r[1], _ptr(P, ctypes.c_double),
                                _ptr(glx, ctypes.c_double), _ptr(glw, ctypes.c_double), GL_POINTS)

        threads = threads or default_threads()
        if n:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                list(ex.map(run, _chunks(n, threads, 4)))
        return P

    def tri_integral(self, n0, n1, n2, w) -> float:
        return float(self.lib.oracle_tri_integral(float(n0[0]), float(n0[1]), float(n1[0]), float(n1[1]),
                                                  float(n2[0]), float(n2[1]),
                                                  float(w[0]), float(w[1]), float(w[2])))


def _get() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def pndf(st, queries, threads: int | None = None, kernel: int = 0, jac_eps: float = 0.0):
    return _get().pndf(st, queries, threads, kernel, jac_eps)


def sample(st, queries, uniforms, kernel: int = 0, jac_eps: float = 0.0, threads: int | None = None):
    return _get().sample(st, queries, uniforms, kernel, jac_eps, threads)


def projarea(st, queries, omega, threads: int | None = None):
    return _get().projarea(st, queries, omega, threads)


def tri_integral(n0, n1, n2, w) -> float:
    return _get().tri_integral(n0, n1, n2, w)


def cluster_fit(st, l: int, I: int, J: int):
    return _get().cluster_fit(st, l, I, J)


def cluster_fits(st, threads: int | None = None) -> ClusterFits:
    return _get().cluster_fits(st, threads)


def pndf_cluster(st, queries, tau: float, fits: ClusterFits | None = None, threads: int | None = None,
                 kernel: int = 0):
    return _get().pndf_cluster(st, queries, tau, fits, threads, kernel)


def ggx_node_P(st, l, I, J, dirs=None):
    return _get().ggx_node_P(st, l, I, J, dirs)


def ggx_fit(P, dirs=None):
    return _get().ggx_fit(P, dirs)


def ggx_fits(st, dirs=None, threads: int | None = None):
    return _get().ggx_fits(st, dirs, threads)


def ggx_lambda(Omega, N, queries, omega):
    return _get().ggx_lambda(Omega, N, queries, omega)


def shadow_masking(Omega, N, queries, wi, wo):
    return _get().shadow_masking(Omega, N, queries, wi, wo)
