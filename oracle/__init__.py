"""CPU oracle for the support-graph preconditioned CG path (FP64).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2410_04512_gb300``) and never imports it.

The arithmetic lives in ``sgp_oracle.c`` (plain sequential C, compiled with
``-ffp-contract=off``); this module compiles it on first use and wraps it
with numpy.  Each wrapper names the passage of arXiv 2410.04512 it follows.
Blocks are (m, 3, 3) float64 arrays; vectors are (n, 3) float64 arrays.

Parity pins: every function here is checked in ``tests/test_oracle_pins.py``
against closed forms, dense LAPACK, brute force or the paper's bounds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgp_oracle.c")
_LIB = os.path.join(_HERE, "_sgp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_OOM, ERR_DEGENERATE, ERR_NOT_SPD, ERR_NO_CONVERGENCE = 0, 1, 3, 4, 5, 6


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_PAR_SRC = os.path.join(_HERE, "cpu_parallel.c")
_PAR_LIB = os.path.join(_HERE, "_sgp_parallel.so")
_par = None


def build_parallel(force: bool = False) -> str:
    """Compile the all-cores CPU baseline (cpu_parallel.c together with the
    oracle's sources, OpenMP when the compiler has it).  Baseline
    infrastructure: only the benchmark's CPU leg and the tests use it."""
    srcs = [_SRC, _PAR_SRC]
    if force or not os.path.exists(_PAR_LIB) or any(os.path.getmtime(_PAR_LIB) < os.path.getmtime(f) for f in srcs):
        tmp = _PAR_LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
        try:
            subprocess.check_call(base + ["-fopenmp"] + srcs + ["-o", tmp, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + srcs + ["-o", tmp, "-lm"])
        os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


def _get_parallel():
    global _par
    with _lock:
        if _par is None:
            lib = ctypes.CDLL(build_parallel())
            P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
            lib.orc_omp_threads.argtypes = []
            lib.orc_omp_threads.restype = ctypes.c_int
            lib.orc_omp_pcg_tree.argtypes = [I64, I64, P, P, D, P, P, P, P, P, P, D, I64,
                                             ctypes.POINTER(I64), ctypes.POINTER(D)]
            lib.orc_omp_pcg_tree.restype = ctypes.c_int
            _par = lib
    return _par


def parallel_threads() -> int:
    """Threads the all-cores baseline runs with (1 without OpenMP)."""
    return int(_get_parallel().orc_omp_threads())


def pcg_parallel(n: int, ij, blocks, gamma0: float, F, factor: "TreeFactor", tol: float = 1e-8,
                 maxit: int = 100000) -> "PcgResult":
    """The same PCG with the tree preconditioner (Section 1.1), the Appendix
    B.2 product row by row and the vector operations over all cores, the
    tree solve (Appendix B.1) sequential.  Baseline timing only: the oracle
    proper is ``pcg``."""
    ij, blocks, F = _i32(ij), _f64(blocks), _f64(F)
    x = np.zeros((n, 3))
    it = ctypes.c_int64(0)
    rel = ctypes.c_double(0.0)
    f = factor.forest
    rc = _get_parallel().orc_omp_pcg_tree(n, ij.shape[0], _p(ij), _p(blocks), gamma0, _p(f.order),
                                          _p(f.parent), _p(factor.L), _p(factor.Dinv), _p(F), _p(x), tol,
                                          maxit, ctypes.byref(it), ctypes.byref(rel))
    if rc not in (OK, ERR_NO_CONVERGENCE):
        raise OracleError(rc, "pcg_parallel")
    return PcgResult(x, int(it.value), float(rel.value), rc)


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            lib.orc_contacts.argtypes = [I64, P, P, P, I64]
            lib.orc_contacts.restype = I64
            lib.orc_contacts_of_rows.argtypes = [I64, P, P, P, I64, P, I64]
            lib.orc_contacts_of_rows.restype = I64
            lib.orc_friction_blocks.argtypes = [I64, P, P, P, P, P, P]
            lib.orc_friction_blocks.restype = ctypes.c_int
            lib.orc_dense_laplacian.argtypes = [I64, I64, P, P, D, P]
            lib.orc_dense_laplacian.restype = None
            lib.orc_matvec.argtypes = [I64, I64, P, P, D, P, P]
            lib.orc_matvec.restype = None
            lib.orc_prim_msf.argtypes = [I64, I64, P, P, P, P, P, P]
            lib.orc_prim_msf.restype = I64
            lib.orc_tree_ldlt.argtypes = [I64, P, P, P, P, D, P, P, P]
            lib.orc_tree_ldlt.restype = ctypes.c_int
            lib.orc_tree_solve.argtypes = [I64, P, P, P, P, P, P]
            lib.orc_tree_solve.restype = ctypes.c_int
            lib.orc_block_jacobi.argtypes = [I64, I64, P, P, D, P]
            lib.orc_block_jacobi.restype = ctypes.c_int
            lib.orc_pcg.argtypes = [I64, I64, P, P, D, ctypes.c_int, P, P, P, P, P, P, D,
                                    I64, I64, ctypes.POINTER(I64), ctypes.POINTER(D)]
            lib.orc_pcg.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------------------
# Section 2 Steps 1-2: collision graph (brute force over all pairs)
# ---------------------------------------------------------------------------
def contacts(pos, radii) -> np.ndarray:
    """All pairs i < j with |r_j - r_i| < R_i + R_j, sorted; (m, 2) int32."""
    pos, radii = _f64(pos), _f64(radii)
    n = pos.shape[0]
    lib = _get()
    cap = max(16, 8 * n)
    while True:
        ij = np.empty((cap, 2), dtype=np.int32)
        m = lib.orc_contacts(n, _p(pos), _p(radii), _p(ij), cap)
        if m <= cap:
            return ij[:m].copy()
        cap = m


def contacts_kdtree(pos, radii) -> np.ndarray:
    """The contact set of ``contacts`` at sizes where the O(N^2) scan is too
    slow: candidate pairs within 2 max(R) from a k-d tree (scipy), each decided
    by the same FP64 expression as the C scan, sqrt((dx*dx + dy*dy) + dz*dz)
    < R_i + R_j with dx = x_j - x_i (numpy evaluates it element-wise with
    round-to-nearest and no fused multiply-add).  Sorted (m, 2) int32."""
    from scipy.spatial import cKDTree
    pos, radii = _f64(pos), _f64(radii)
    n = pos.shape[0]
    if n < 2:
        return np.zeros((0, 2), dtype=np.int32)
    cand = cKDTree(pos).query_pairs(2.0 * radii.max() * (1.0 + 1e-12), output_type="ndarray")
    if cand.size == 0:
        return np.zeros((0, 2), dtype=np.int32)
    cand = np.sort(cand, axis=1)
    i, j = cand[:, 0], cand[:, 1]
    dx = pos[j, 0] - pos[i, 0]
    dy = pos[j, 1] - pos[i, 1]
    dz = pos[j, 2] - pos[i, 2]
    s = dx * dx
    s = s + dy * dy
    s = s + dz * dz
    keep = np.sqrt(s) < radii[i] + radii[j]
    ij = cand[keep]
    ij = ij[np.lexsort((ij[:, 1], ij[:, 0]))]
    return np.ascontiguousarray(ij.astype(np.int32))


def contacts_of_rows(pos, radii, rows) -> np.ndarray:
    """Brute-force contacts (i, j > i) for the listed rows i only."""
    pos, radii = _f64(pos), _f64(radii)
    rows = np.ascontiguousarray(np.sort(np.asarray(rows, dtype=np.int64)))
    n = pos.shape[0]
    lib = _get()
    cap = max(16, 16 * len(rows))
    while True:
        ij = np.empty((cap, 2), dtype=np.int32)
        m = lib.orc_contacts_of_rows(n, _p(pos), _p(radii), _p(rows), len(rows), _p(ij), cap)
        if m <= cap:
            return ij[:m].copy()
        cap = m


# ---------------------------------------------------------------------------
# Section 2 Step 3, eq. (1); Section 3.1 tree weight (Lemma 2.1)
# ---------------------------------------------------------------------------
def friction_blocks(ij, pos, g_par, g_perp):
    """Upsilon_e = g_par u u^T + g_perp (I - u u^T) per edge and the tree
    weight min(g_par, g_perp).  Returns ((m,3,3) blocks, (m,) weights)."""
    ij, pos = _i32(ij), _f64(pos)
    g_par, g_perp = _f64(g_par), _f64(g_perp)
    m = ij.shape[0]
    blocks = np.empty((m, 3, 3), dtype=np.float64)
    w = np.empty(m, dtype=np.float64)
    rc = _get().orc_friction_blocks(m, _p(ij), _p(pos), _p(g_par), _p(g_perp), _p(blocks), _p(w))
    if rc:
        raise OracleError(rc, "friction_blocks")
    return blocks, w


def dense_laplacian(n: int, ij, blocks, gamma0: float) -> np.ndarray:
    """Dense block Laplacian (Definition in Section 2) with self-loops gamma0 I."""
    ij, blocks = _i32(ij), _f64(blocks)
    out = np.empty((3 * n, 3 * n), dtype=np.float64)
    _get().orc_dense_laplacian(n, ij.shape[0], _p(ij), _p(blocks), gamma0, _p(out))
    return out


def matvec(n: int, ij, blocks, gamma0: float, v) -> np.ndarray:
    """Appendix B.2 MatVec: x_i = gamma0 v_i + sum_j Upsilon_ij (v_i - v_j)."""
    ij, blocks, v = _i32(ij), _f64(blocks), _f64(v)
    x = np.empty((n, 3), dtype=np.float64)
    _get().orc_matvec(n, ij.shape[0], _p(ij), _p(blocks), gamma0, _p(v), _p(x))
    return x


# ---------------------------------------------------------------------------
# Section 3.1: maximum spanning forest (Prim, strict order w desc, id asc)
# ---------------------------------------------------------------------------
@dataclass
class Forest:
    tree_edges: np.ndarray   # edge ids in Prim insertion order
    order: np.ndarray        # vertices in Prim insertion order
    parent: np.ndarray       # parent vertex, -1 at each component's start vertex
    parent_edge: np.ndarray  # edge to the parent, -1 at the start vertex


def prim_msf(n: int, ij, w) -> Forest:
    ij, w = _i32(ij), _f64(w)
    m = ij.shape[0]
    te = np.empty(max(n, 1), dtype=np.int32)
    order = np.empty(max(n, 1), dtype=np.int32)
    parent = np.empty(max(n, 1), dtype=np.int32)
    pedge = np.empty(max(n, 1), dtype=np.int32)
    nt = _get().orc_prim_msf(n, m, _p(ij), _p(w), _p(te), _p(order), _p(parent), _p(pedge))
    if nt < 0:
        raise OracleError(ERR_OOM, "prim_msf")
    return Forest(te[:nt].copy(), order[:n].copy(), parent[:n].copy(), pedge[:n].copy())


# ---------------------------------------------------------------------------
# Section 3.3 Algorithm 2 (TreeLDLT) and Appendix B.1 (tree solve)
# ---------------------------------------------------------------------------
@dataclass
class TreeFactor:
    forest: Forest
    L: np.ndarray      # (n,3,3): block linking each vertex to its parent
    D: np.ndarray      # (n,3,3): pivot blocks
    Dinv: np.ndarray   # (n,3,3)


def tree_ldlt(forest: Forest, blocks, gamma0: float) -> TreeFactor:
    blocks = _f64(blocks)
    n = forest.order.shape[0]
    L = np.zeros((n, 3, 3))
    D = np.zeros((n, 3, 3))
    Dinv = np.zeros((n, 3, 3))
    rc = _get().orc_tree_ldlt(n, _p(forest.order), _p(forest.parent), _p(forest.parent_edge),
                              _p(blocks), gamma0, _p(L), _p(D), _p(Dinv))
    if rc:
        raise OracleError(rc, "tree_ldlt")
    return TreeFactor(forest, L, D, Dinv)


def tree_solve(fac: TreeFactor, b) -> np.ndarray:
    b = _f64(b)
    n = fac.forest.order.shape[0]
    x = np.empty((n, 3), dtype=np.float64)
    rc = _get().orc_tree_solve(n, _p(fac.forest.order), _p(fac.forest.parent), _p(fac.L),
                               _p(fac.Dinv), _p(b), _p(x))
    if rc:
        raise OracleError(rc, "tree_solve")
    return x


def block_jacobi(n: int, ij, blocks, gamma0: float) -> np.ndarray:
    """Inverses of the diagonal blocks of Gamma (Section 5, preconditioner (2))."""
    ij, blocks = _i32(ij), _f64(blocks)
    Dinv = np.empty((n, 3, 3), dtype=np.float64)
    rc = _get().orc_block_jacobi(n, ij.shape[0], _p(ij), _p(blocks), gamma0, _p(Dinv))
    if rc:
        raise OracleError(rc, "block_jacobi")
    return Dinv


PRECOND_NONE, PRECOND_TREE, PRECOND_JACOBI = 0, 1, 2


@dataclass
class PcgResult:
    x: np.ndarray
    iters: int
    relres: float   # recursive |r|/|F|
    status: int


def pcg(n: int, ij, blocks, gamma0: float, F, precond=PRECOND_TREE, factor: TreeFactor | None = None,
        jacobi_dinv=None, x0=None, tol: float = 1e-8, maxit: int = 100000,
        fixed_iters: int = 0) -> PcgResult:
    """Section 1.1 preconditioned conjugate gradients on Gamma v = F."""
    ij, blocks, F = _i32(ij), _f64(blocks), _f64(F)
    x = np.zeros((n, 3)) if x0 is None else _f64(x0).copy()
    order = parent = L = Dinv = None
    if precond == PRECOND_TREE:
        order, parent, L, Dinv = factor.forest.order, factor.forest.parent, factor.L, factor.Dinv
    elif precond == PRECOND_JACOBI:
        Dinv = _f64(jacobi_dinv)
    it = ctypes.c_int64(0)
    rel = ctypes.c_double(0.0)
    rc = _get().orc_pcg(n, ij.shape[0], _p(ij), _p(blocks), gamma0, precond, _p(order),
                        _p(parent), _p(L), _p(Dinv), _p(F), _p(x), tol, maxit, fixed_iters,
                        ctypes.byref(it), ctypes.byref(rel))
    if rc not in (OK, ERR_NO_CONVERGENCE):
        raise OracleError(rc, "pcg")
    return PcgResult(x, int(it.value), float(rel.value), rc)


# ---------------------------------------------------------------------------
# The whole path for one configuration (Section 2 Steps 1-4)
# ---------------------------------------------------------------------------
@dataclass
class System:
    n: int
    ij: np.ndarray
    g_par: np.ndarray
    g_perp: np.ndarray
    blocks: np.ndarray
    w: np.ndarray
    gamma0: float


def build_system(pos, radii, gammas_fn, gamma0: float, ij=None) -> System:
    """Contacts (brute force unless ``ij`` is given), per-pair coefficients
    from ``gammas_fn(ij)`` and the friction blocks."""
    if ij is None:
        ij = contacts(pos, radii)
    gp, gq = gammas_fn(ij)
    blocks, w = friction_blocks(ij, pos, gp, gq)
    return System(pos.shape[0], ij, _f64(gp), _f64(gq), blocks, w, gamma0)


def solve_system(sys: System, F, tol: float, precond=PRECOND_TREE, x0=None, maxit=100000,
                 fixed_iters=0):
    """Preconditioner set-up (Prim + TreeLDLT or block Jacobi) and PCG."""
    fac = None
    jd = None
    if precond == PRECOND_TREE:
        forest = prim_msf(sys.n, sys.ij, sys.w)
        fac = tree_ldlt(forest, sys.blocks, sys.gamma0)
    elif precond == PRECOND_JACOBI:
        jd = block_jacobi(sys.n, sys.ij, sys.blocks, sys.gamma0)
    res = pcg(sys.n, sys.ij, sys.blocks, sys.gamma0, F, precond, fac, jd, x0, tol, maxit,
              fixed_iters)
    return res, fac
