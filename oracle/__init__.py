"""CPU oracle for findpts / findpts_eval -- TEST INFRASTRUCTURE ONLY.

Plain brute-force FP64 C (``findpts_oracle.c``) behind ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the library in ``paper_1811_04891_gb300`` never does.

Parity pins (tests/test_oracle_*.py): GLL nodes/weights against closed forms
and quadrature exactness; the map against an independent Vandermonde
evaluation; find against forward-mapped known (e, r) and affine closed forms;
eval against exactly reproduced Q_N polynomials; ownership against tiny
overlapping boxes with closed-form delta; the default distance field against
closed forms on undeformed boxes, annular cylinders (rotated too) and rings;
ownership with that field on curved overlaps (a cylinder or ring crossing a
box face, both owners present) against the exact boundary distances, away
from ties.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "findpts_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

INSIDE, BORDER, NOT_FOUND = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("tol_accept", ctypes.c_double), ("tol_border", ctypes.c_double),
                ("tie_band", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("n_restarts", ctypes.c_int), ("prefilter", ctypes.c_int)]


@dataclass
class Params:
    tol_accept: float = 1e-12
    tol_border: float = 1e-6
    tie_band: float = 1e-10
    max_newton: int = 50
    n_restarts: int = 0
    prefilter: bool = True


def lib():
    global _lib
    if _lib is None:
        # FINDPTS_ORACLE_LIB: a separately built copy (the mutation tests load
        # deliberately broken builds this way to show that the pins catch them)
        _lib = ctypes.CDLL(os.environ.get("FINDPTS_ORACLE_LIB") or build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.c_int64
        _lib.or_gll.argtypes = [ctypes.c_int, dp, dp]
        _lib.or_lagrange.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp]
        _lib.or_map.argtypes = [ctypes.c_int, dp, i64, i64, i64, dp, dp, dp]
        _lib.or_find.argtypes = [ctypes.c_int, i64, dp, ip, dp, i64, dp, ip,
                                 ctypes.POINTER(_Params), ip, ip, ip, dp, dp]
        _lib.or_find.restype = i64
        _lib.or_eval.argtypes = [ctypes.c_int, i64, i64, ip, ip, dp, ctypes.c_int, dp, dp]
        _lib.or_dist_default.argtypes = [ctypes.c_int, i64, dp, ip, dp]
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib.or_set_threads.restype = None
        i8p = ctypes.POINTER(ctypes.c_int8)
        _lib.or_bfaces.argtypes = [ctypes.c_int, i64, dp, i8p, dp, dp, dp, i8p]
        _lib.or_bfaces.restype = i64
        _lib.or_flux_correct.argtypes = [i64, dp, dp, dp, i8p, dp, dp, dp]
        _lib.or_find_d.argtypes = [ctypes.c_int] + list(_lib.or_find.argtypes)
        _lib.or_find_d.restype = i64
        _lib.or_eval_d.argtypes = [ctypes.c_int] + list(_lib.or_eval.argtypes)
        _lib.or_map_d.argtypes = [ctypes.c_int] + list(_lib.or_map.argtypes)
        _lib.or_dist_default_2d.argtypes = [ctypes.c_int, i64, dp, ip, dp]
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int):
    """Threads of the oracle's later OpenMP loops (n >= 1)."""
    lib().or_set_threads(int(n))


def gll(N: int):
    """GLL points and weights of order N."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().or_gll(N, _d(x), _d(w)) != 0:
        raise ValueError("N out of range")
    return x, w


def lagrange(N: int, r: float):
    """Lagrange basis values h_i(r) and derivatives on the GLL points."""
    x, _ = gll(N)
    h = np.zeros(N + 1)
    dh = np.zeros(N + 1)
    lib().or_lagrange(N, _d(x), float(r), _d(h), _d(dh))
    return h, dh


def map_points(coords, N: int, e: int, r):
    """x^e(r) and J for reference points r [d][M] on a d-dimensional mesh
    (coords [d][E][n^d], d = 2 or 3); returns ([d][M], [d*d][M])."""
    coords = _f64(coords)
    d = coords.shape[0]
    r = _f64(r)
    M = r.shape[1]
    x = np.zeros((d, M))
    J = np.zeros((d * d, M))
    lib().or_map_d(d, N, _d(coords), coords.shape[1], int(e), M, _d(r), _d(x), _d(J))
    return x, J


def find(coords, N: int, sub, pts, qsess=None, dist=None, params: Params | None = None):
    """Brute-force findpts on a hex (coords [3][E][n^3], pts [3][P]) or quad
    (coords [2][E][n^2], pts [2][P]) mesh.  Returns dict(code, sub, elem,
    rst [d][P], dist2)."""
    prm = params or Params()
    coords = _f64(coords)
    dim = coords.shape[0]
    E = coords.shape[1]
    sub = _i32(sub)
    pts = _f64(pts)
    P = pts.shape[1]
    qs = None if qsess is None else _i32(qsess)
    dist = None if dist is None else _f64(dist)
    code = np.zeros(P, np.int32)
    osub = np.zeros(P, np.int32)
    oel = np.zeros(P, np.int32)
    rst = np.zeros((dim, P))
    d2 = np.zeros(P)
    cp = _Params(prm.tol_accept, prm.tol_border, prm.tie_band, prm.max_newton,
                 prm.n_restarts, int(prm.prefilter))
    if pts.shape[0] != dim:
        raise ValueError("pts must have as many rows as the mesh has dimensions")
    bad = lib().or_find_d(dim, N, E, _d(coords), _i(sub), None if dist is None else _d(dist), P,
                        _d(pts), None if qs is None else _i(qs), ctypes.byref(cp),
                        _i(code), _i(osub), _i(oel), _d(rst), _d(d2))
    if bad < 0:
        raise ValueError("oracle find: bad arguments")
    return {"code": code, "sub": osub, "elem": oel, "rst": rst, "dist2": d2}


def evaluate(N: int, code, elem, rst, fields):
    """findpts_eval by full triple (2D: double) sums; fields [F][E][n^d],
    rst [d][P] -> out [F][P]."""
    fields = _f64(fields)
    if fields.ndim == 2:
        fields = fields[None]
    F, E = fields.shape[0], fields.shape[1]
    code = _i32(code)
    elem = _i32(elem)
    rst = _f64(rst)
    P = code.shape[0]
    out = np.zeros((F, P))
    dim = rst.shape[0]
    if fields.shape[2] != (N + 1) ** dim:
        raise ValueError("fields must be [F][E][(N+1)^d] with d = rst rows")
    lib().or_eval_d(dim, N, E, P, _i(code), _i(elem), _d(rst), F, _d(fields), _d(out))
    return out


def bfaces(coords, N: int, kind):
    """Boundary-face quadrature of the faces marked in kind [E][6] (1 =
    prescribed data, 2 = interface): node positions [3][M], outward unit
    normals [3][M], weights dA [M], node kinds [M]."""
    coords = _f64(coords)
    E = coords.shape[1]
    kind = np.ascontiguousarray(kind, dtype=np.int8).reshape(-1)
    cap = int((kind != 0).sum()) * (N + 1) ** 2
    x = np.zeros((max(cap, 1), 3))
    nr = np.zeros((max(cap, 1), 3))
    dA = np.zeros(max(cap, 1))
    nk = np.zeros(max(cap, 1), np.int8)
    i8 = ctypes.POINTER(ctypes.c_int8)
    M = lib().or_bfaces(N, E, _d(coords), kind.ctypes.data_as(i8), _d(x), _d(nr), _d(dA), nk.ctypes.data_as(i8))
    return x[:M].T.copy(), nr[:M].T.copy(), dA[:M].copy(), nk[:M].copy()


def flux_correct(u, nrm, dA, nkind):
    """Eq. consv2 / corr on listed face nodes: u, nrm [3][M] -> (u_out [3][M], gamma, flux)."""
    M = dA.shape[0]
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).T)
    nn = np.ascontiguousarray(np.asarray(nrm, dtype=np.float64).T)
    out = np.zeros_like(uu)
    g = ctypes.c_double()
    fl = ctypes.c_double()
    nk = np.ascontiguousarray(nkind, dtype=np.int8)
    lib().or_flux_correct(M, _d(uu), _d(nn), _d(_f64(dA)), nk.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                          _d(out), ctypes.byref(g), ctypes.byref(fl))
    return out.T.copy(), g.value, fl.value


def extrapolate(hist):
    """Order-m extrapolation in time over equal steps from the m newest
    values (newest first): the polynomial of degree m-1 through
    (t_{n}, h_0), (t_{n-1}, h_1), ... evaluated at t_{n+1}, written out as
    Lagrange weights on the equally spaced abscissae."""
    m = len(hist)
    ts = [-float(j) for j in range(m)]          # t_n = 0, t_{n-1} = -1, ...
    out = np.zeros_like(np.asarray(hist[0], dtype=np.float64))
    for j in range(m):
        w = 1.0
        for k in range(m):
            if k != j:
                w *= (1.0 - ts[k]) / (ts[j] - ts[k])
        out = out + w * np.asarray(hist[j], dtype=np.float64)
    return out


def dist_default(coords, N: int, sub):
    """Default nodal distance field D^k [E][n^d] (brute force), d = 2 or 3."""
    coords = _f64(coords)
    E = coords.shape[1]
    if coords.shape[0] == 2:
        D = np.zeros((E, (N + 1) ** 2))
        lib().or_dist_default_2d(N, E, _d(coords), _i(_i32(sub)), _d(D))
        return D
    D = np.zeros((E, (N + 1) ** 3))
    lib().or_dist_default(N, E, _d(coords), _i(_i32(sub)), _d(D))
    return D
