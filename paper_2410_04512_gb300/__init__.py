"""Python binding of libsgp.so, the sm_103a support-graph PCG library.

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  Device memory comes from torch tensors (contiguous, on the
context's device); work is ordered on the torch stream given at context
creation.  Names follow the C ABI in include/sgp.h.

There is no CPU fallback: if libsgp.so is missing or a CUDA device is not
available, creating a context raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgp.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_DEGENERATE, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_TIMEOUT = range(8)
PREC_F64, PREC_MIXED = 0, 1
PRECOND_TREE, PRECOND_BLOCK_JACOBI, PRECOND_NONE = 0, 1, 2
KT_SPMV, KT_TREE_SOLVE, KT_PCG_VECTOR, KT_WARM_BASIS, KT_WARM_LAYERS, KT_WARM_CHECK = 0, 1, 2, 3, 4, 5
STOP_RESIDUAL, STOP_ERROR = 0, 1
MPNN_PARAMS = 25539
MPNN_LOSS_L2, MPNN_LOSS_ENERGY = 0, 1
WARM_MR_SCALE = 1

_STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "DEGENERATE", 5: "NOT_SPD",
                 6: "NO_CONVERGENCE", 7: "TIMEOUT"}


class SgpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sgp error {_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int64), ("precond", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("x0_given", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("stop", ctypes.c_int32),
                ("mu", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("spmv_lpr", ctypes.c_int32), ("tail_cap", ctypes.c_int32), ("batch_chunk", ctypes.c_int32),
                ("spmv_ilp", ctypes.c_int32), ("bin_cap", ctypes.c_int32), ("ms_per_iteration", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("outer_iterations", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("err_bound", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsgp.so (building it first if it is absent and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "sgp_create": ([PP, ctypes.c_int, P], I32),
        "sgp_destroy": ([P], None),
        "sgp_last_error": ([P], ctypes.c_char_p),
        "sgp_version": ([], ctypes.c_char_p),
        "sgp_copy": ([P, P, P, I64], I32),
        "sgp_collision_graph": ([P, I64, P, P, PP], I32),
        "sgp_collision_graph_batched": ([P, I64, P, P, P, PP], I32),
        "sgp_pcg_solve_batched": ([P, P, P, I64, P, P, P, ctypes.POINTER(SolveOpts), P], I32),
        "sgp_graph_info": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64), PP], I32),
        "sgp_graph_destroy": ([P], None),
        "sgp_friction_assemble": ([P, P, P, P, P, D, I32, PP], I32),
        "sgp_spmv": ([P, P, P, P], I32),
        "sgp_spmv_dot_noalloc": ([P, P, P, P, P], I32),
        "sgp_matrix_edge_blocks": ([P, P, P, P], I32),
        "sgp_matrix_destroy": ([P], None),
        "sgp_max_spanning_tree": ([P, P, PP], I32),
        "sgp_grid_leaves": ([P, I64, P, D, P], I32),
        "sgp_local_spanning_forest": ([P, P, P, PP], I32),
        "sgp_tree_info": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64), PP], I32),
        "sgp_tree_destroy": ([P], None),
        "sgp_tree_factor": ([P, P, P, PP], I32),
        "sgp_tree_apply": ([P, P, P, P], I32),
        "sgp_factor_info": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I64),
                             ctypes.POINTER(I64)], I32),
        "sgp_factor_destroy": ([P], None),
        "sgp_pcg_solve": ([P, P, P, P, P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)], I32),
        "sgp_set_kernel_timing": ([P, I32], I32),
        "sgp_kernel_time": ([P, I32, ctypes.POINTER(D), ctypes.POINTER(I64), I32], I32),
        "sgp_launch_count": ([P, ctypes.POINTER(I64), I32], I32),
        "sgp_factor_layout": ([P] + [ctypes.POINTER(I32)] * 6, I32),
        "sgp_get_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "sgp_set_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "sgp_autotune": ([P, P, P, PP, I64, P, P, ctypes.POINTER(SolveOpts), I32, ctypes.POINTER(Tuning)], I32),
        "sgp_mpnn_create": ([P, P, I64, PP], I32),
        "sgp_mpnn_destroy": ([P], None),
        "sgp_mpnn_params": ([P, P, P, P], I32),
        "sgp_mpnn_forward": ([P, P, P, P, P, P, P], I32),
        "sgp_mpnn_backward": ([P, P, P, I32, ctypes.POINTER(D)], I32),
        "sgp_mpnn_step": ([P, P, ctypes.c_float], I32),
        "sgp_warm_start": ([P, P, P, P, P, P, P, I32, ctypes.POINTER(I32)], I32),
        "sgp_augment_tree": ([P, P, P, I32, PP], I32),
        "sgp_aug_info": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                          ctypes.POINTER(I64), ctypes.POINTER(I64)], I32),
        "sgp_aug_pieces": ([P, P, P], I32),
        "sgp_aug_edges": ([P, P, P], I32),
        "sgp_aug_matrix": ([P], P),
        "sgp_aug_destroy": ([P], None),
        "sgp_fcg_solve": ([P, P, P, P, P, P, ctypes.POINTER(SolveOpts), I64, ctypes.POINTER(SolveInfo)], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C ABI entry points this binding expects."""
    import re
    with open(os.path.join(os.path.dirname(_HERE), "include", "sgp.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:sgp_status|void|const \w+ \*)\s*\*?(sgp_\w+)\s*\(", txt, re.M)))


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_vec(t: torch.Tensor, n: int, dtype=torch.float64, cols: int = 3, name: str = "tensor"):
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    want = (n, cols) if cols else (n,)
    if tuple(t.shape) != want:
        raise ValueError(f"{name} must have shape {want}, got {tuple(t.shape)}")


class _Handle:
    _destroy = None

    def __init__(self, ctx: "Context"):
        self.ctx = ctx
        self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        if self.ptr and self.ptr.value and self._destroy and _lib is not None:
            getattr(_lib, self._destroy)(self.ptr)
            self.ptr = ctypes.c_void_p(None)


class Graph(_Handle):
    _destroy = "sgp_graph_destroy"

    def info(self):
        n, m, ij = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_void_p()
        self.ctx._ok(_lib.sgp_graph_info(self.ptr, ctypes.byref(n), ctypes.byref(m), ctypes.byref(ij)))
        return n.value, m.value, ij.value

    @property
    def n(self):
        return self.info()[0]

    @property
    def m(self):
        return self.info()[1]

    def edges(self) -> torch.Tensor:
        n, m, ij = self.info()
        out = torch.empty((m, 2), dtype=torch.int32, device=self.ctx.device)
        if m:
            self.ctx._ok(_lib.sgp_copy(self.ctx.ptr, _ptr(out), ctypes.c_void_p(ij), 8 * m))
        return out


class Matrix(_Handle):
    _destroy = "sgp_matrix_destroy"

    def __init__(self, ctx, n, m, precision):
        super().__init__(ctx)
        self.n, self.m, self.precision = n, m, precision

    def edge_blocks(self):
        blocks = torch.empty((self.m, 3, 3), dtype=torch.float64, device=self.ctx.device)
        w = torch.empty((self.m,), dtype=torch.float64, device=self.ctx.device)
        self.ctx._ok(_lib.sgp_matrix_edge_blocks(self.ctx.ptr, self.ptr, _ptr(blocks), _ptr(w)))
        return blocks, w


class _BorrowedMatrix(Matrix):
    _destroy = None


class Tree(_Handle):
    _destroy = "sgp_tree_destroy"

    def info(self):
        ne, nc, ids = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_void_p()
        self.ctx._ok(_lib.sgp_tree_info(self.ptr, ctypes.byref(ne), ctypes.byref(nc), ctypes.byref(ids)))
        return ne.value, nc.value, ids.value

    def edge_ids(self) -> torch.Tensor:
        ne, nc, ids = self.info()
        out = torch.empty((ne,), dtype=torch.int32, device=self.ctx.device)
        if ne:
            self.ctx._ok(_lib.sgp_copy(self.ctx.ptr, _ptr(out), ctypes.c_void_p(ids), 4 * ne))
        return out


class Factor(_Handle):
    _destroy = "sgp_factor_destroy"

    def info(self):
        """(rounds, levels) of the contraction schedule."""
        return self.stats()[:2]

    def stats(self):
        """(rounds, levels, L blocks, receiver entries)."""
        r, l = ctypes.c_int32(), ctypes.c_int32()
        nb, nr = ctypes.c_int64(), ctypes.c_int64()
        self.ctx._ok(_lib.sgp_factor_info(self.ptr, ctypes.byref(r), ctypes.byref(l), ctypes.byref(nb),
                                          ctypes.byref(nr)))
        return r.value, l.value, nb.value, nr.value

    def layout(self) -> dict:
        """The binned solve's layout: bins, top vertices, subtree bound, and
        whether the FP32 / FP64 applications use it."""
        v = [ctypes.c_int32() for _ in range(6)]
        self.ctx._ok(_lib.sgp_factor_layout(self.ptr, *[ctypes.byref(x) for x in v]))
        return dict(zip(("bins", "top", "leaks", "bin_cap", "fp32", "fp64"), (x.value for x in v)))


class Augmented(_Handle):
    """The augmented spanning forest T' and P' (Section 3.1)."""
    _destroy = "sgp_aug_destroy"

    def info(self) -> dict:
        t, k, cap = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ne, na = ctypes.c_int64(), ctypes.c_int64()
        self.ctx._ok(_lib.sgp_aug_info(self.ptr, ctypes.byref(t), ctypes.byref(k), ctypes.byref(cap),
                                       ctypes.byref(ne), ctypes.byref(na)))
        return {"t": t.value, "pieces": k.value, "piece_cap": cap.value, "edges": ne.value, "added": na.value}

    def pieces(self, n: int) -> torch.Tensor:
        out = torch.empty((n,), dtype=torch.int32, device=self.ctx.device)
        self.ctx._ok(_lib.sgp_aug_pieces(self.ctx.ptr, self.ptr, _ptr(out)))
        return out

    def edges(self) -> torch.Tensor:
        out = torch.empty((self.info()["edges"],), dtype=torch.int32, device=self.ctx.device)
        self.ctx._ok(_lib.sgp_aug_edges(self.ctx.ptr, self.ptr, _ptr(out)))
        return out

    def matrix(self, n: int) -> "Matrix":
        """P' as a matrix handle owned by this object (not destroyed with
        the returned wrapper)."""
        m = _BorrowedMatrix(self.ctx, n, self.info()["edges"], PREC_F64)
        m.ptr = ctypes.c_void_p(_lib.sgp_aug_matrix(self.ptr))
        m.owner = self
        return m


class Mpnn(_Handle):
    """The warm-start network (FP32 master weights and BF16 copies on the
    device, Adam state, activations of the last forward pass)."""
    _destroy = "sgp_mpnn_destroy"

    def params(self):
        """(master parameters, last gradient) as float32 numpy arrays."""
        import numpy as np
        p = np.empty(MPNN_PARAMS, dtype=np.float32)
        g = np.empty(MPNN_PARAMS, dtype=np.float32)
        self.ctx._ok(_lib.sgp_mpnn_params(self.ctx.ptr, self.ptr, p.ctypes.data_as(ctypes.c_void_p),
                                          g.ctypes.data_as(ctypes.c_void_p)))
        return p, g


@dataclass
class Info:
    iterations: int
    outer_iterations: int
    status: int
    rel_residual: float
    true_rel_residual: float
    err_bound: float = 0.0


class Context:
    """An sgp context on one CUDA device, ordered on a torch stream."""

    def __init__(self, device: int | torch.device = 0, stream: torch.cuda.Stream | None = None):
        lib = load_library()
        if not torch.cuda.is_available():
            raise SgpError(ERR_CUDA, "no CUDA device: this library has no CPU path")
        dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ptr = ctypes.c_void_p()
        rc = lib.sgp_create(ctypes.byref(self.ptr), dev.index or 0, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            raise SgpError(rc, "sgp_create failed")

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.sgp_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def _ok(self, rc: int):
        if rc != OK:
            raise SgpError(rc, _lib.sgp_last_error(self.ptr).decode())

    # -- calls of include/sgp.h ------------------------------------------
    def collision_graph(self, pos: torch.Tensor, radii: torch.Tensor, graph: Graph | None = None) -> Graph:
        n = pos.shape[0]
        _check_vec(pos, n, name="pos")
        _check_vec(radii, n, cols=0, name="radii")
        g = graph if graph is not None else Graph(self)
        self._ok(_lib.sgp_collision_graph(self.ptr, n, _ptr(pos), _ptr(radii), ctypes.byref(g.ptr)))
        return g

    def friction_assemble(self, graph: Graph, pos, gamma_par, gamma_perp, gamma0: float,
                          precision: int = PREC_F64, matrix: Matrix | None = None) -> Matrix:
        n, m, _ = graph.info()
        _check_vec(pos, n, name="pos")
        _check_vec(gamma_par, m, cols=0, name="gamma_par")
        _check_vec(gamma_perp, m, cols=0, name="gamma_perp")
        M = matrix if matrix is not None else Matrix(self, n, m, precision)
        M.n, M.m, M.precision = n, m, precision
        self._ok(_lib.sgp_friction_assemble(self.ptr, graph.ptr, _ptr(pos), _ptr(gamma_par),
                                            _ptr(gamma_perp), float(gamma0), precision,
                                            ctypes.byref(M.ptr)))
        return M

    def spmv(self, M: Matrix, v: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        _check_vec(v, M.n, name="v")
        y = torch.empty_like(v) if y is None else y
        self._ok(_lib.sgp_spmv(self.ptr, M.ptr, _ptr(v), _ptr(y)))
        return y

    def max_spanning_tree(self, M: Matrix, tree: Tree | None = None) -> Tree:
        T = tree if tree is not None else Tree(self)
        self._ok(_lib.sgp_max_spanning_tree(self.ptr, M.ptr, ctypes.byref(T.ptr)))
        return T

    # -- partitioned spanning forest (Section 6) --------------------------
    def grid_leaves(self, pos: torch.Tensor, h: float, leaf: torch.Tensor | None = None) -> torch.Tensor:
        """Leaf label of every cell in the uniform grid of side h (int32)."""
        n = pos.shape[0]
        _check_vec(pos, n, name="pos")
        leaf = torch.empty(n, dtype=torch.int32, device=pos.device) if leaf is None else leaf
        if leaf.dtype != torch.int32 or leaf.shape != (n,) or not leaf.is_contiguous() or not leaf.is_cuda:
            raise ValueError("leaf must be a contiguous CUDA int32 tensor of n entries")
        self._ok(_lib.sgp_grid_leaves(self.ptr, n, _ptr(pos), float(h), _ptr(leaf)))
        return leaf

    def local_spanning_forest(self, M: Matrix, leaf: torch.Tensor, tree: Tree | None = None) -> Tree:
        """Union of the leaves' maximum spanning forests (contacts between
        leaves dropped)."""
        if leaf.dtype != torch.int32 or leaf.shape != (M.n,) or not leaf.is_contiguous() or not leaf.is_cuda:
            raise ValueError("leaf must be a contiguous CUDA int32 tensor of n entries")
        T = tree if tree is not None else Tree(self)
        self._ok(_lib.sgp_local_spanning_forest(self.ptr, M.ptr, _ptr(leaf), ctypes.byref(T.ptr)))
        return T

    def tree_factor(self, M: Matrix, T: Tree, factor: Factor | None = None) -> Factor:
        Fh = factor if factor is not None else Factor(self)
        self._ok(_lib.sgp_tree_factor(self.ptr, M.ptr, T.ptr, ctypes.byref(Fh.ptr)))
        return Fh

    def tree_apply(self, Fh: Factor, b: torch.Tensor, x: torch.Tensor | None = None) -> torch.Tensor:
        x = torch.empty_like(b) if x is None else x
        self._ok(_lib.sgp_tree_apply(self.ptr, Fh.ptr, _ptr(b), _ptr(x)))
        return x

    def pcg_solve(self, M: Matrix, Fh: Factor | None, F: torch.Tensor, v: torch.Tensor | None = None,
                  tol: float = 1e-8, maxit: int = 100000, precond: int = PRECOND_TREE,
                  precision: int = PREC_F64, x0_given: bool = False, max_outer: int = 0,
                  inner_tol: float = 0.0, raise_on_error: bool = True, stop: int = 0, mu: float = 0.0):
        """PCG (Section 1.1); stop=STOP_ERROR stops on the Gauss-Radau bound
        of the Gamma-norm error (FP64), mu its lower eigenvalue bound."""
        _check_vec(F, M.n, name="F")
        v = torch.zeros_like(F) if v is None else v
        _check_vec(v, M.n, name="v")
        o = SolveOpts(tol, maxit, precond, precision, int(x0_given), max_outer, inner_tol, stop, mu)
        inf = SolveInfo()
        rc = _lib.sgp_pcg_solve(self.ptr, M.ptr, Fh.ptr if Fh is not None else None, _ptr(F), _ptr(v),
                                ctypes.byref(o), ctypes.byref(inf))
        info = Info(inf.iterations, inf.outer_iterations, inf.status, inf.rel_residual,
                    inf.true_rel_residual, inf.err_bound)
        if rc != OK and (raise_on_error or rc not in (ERR_NO_CONVERGENCE,)):
            self._ok(rc)
        return v, info

    # -- augmented spanning forest and flexible CG (Sections 3.1, 5) ---------
    def augment_tree(self, M: Matrix, T: Tree, t: int = 0, aug: "Augmented | None" = None) -> "Augmented":
        A = aug if aug is not None else Augmented(self)
        self._ok(_lib.sgp_augment_tree(self.ptr, M.ptr, T.ptr, t, ctypes.byref(A.ptr)))
        return A

    def fcg_solve(self, M: Matrix, A: "Augmented", Fh: Factor, F: torch.Tensor, v: torch.Tensor | None = None,
                  tol: float = 1e-8, maxit: int = 100000, inner_tol: float = 0.1, inner_maxit: int = 1000,
                  x0_given: bool = False, raise_on_error: bool = True):
        """Flexible CG with the augmented preconditioner applied by an inner
        PCG (Section 5); returns (v, Info) with Info.outer_iterations the
        flexible steps and Info.iterations the inner iterations."""
        _check_vec(F, M.n, name="F")
        v = torch.zeros_like(F) if v is None else v
        _check_vec(v, M.n, name="v")
        o = SolveOpts(tol, maxit, PRECOND_TREE, PREC_F64, int(x0_given), 0, inner_tol)
        inf = SolveInfo()
        rc = _lib.sgp_fcg_solve(self.ptr, M.ptr, A.ptr, Fh.ptr, _ptr(F), _ptr(v), ctypes.byref(o), inner_maxit,
                                ctypes.byref(inf))
        info = Info(inf.iterations, inf.outer_iterations, inf.status, inf.rel_residual, inf.true_rel_residual,
                    inf.err_bound)
        if rc != OK and (raise_on_error or rc not in (ERR_NO_CONVERGENCE,)):
            self._ok(rc)
        return v, info

    # -- batches of independent configurations ------------------------------
    def collision_graph_batched(self, offsets, pos: torch.Tensor, radii: torch.Tensor,
                                graph: Graph | None = None) -> Graph:
        import numpy as np
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        n = int(off[-1])
        _check_vec(pos, n, name="pos")
        _check_vec(radii, n, cols=0, name="radii")
        g = graph if graph is not None else Graph(self)
        self._ok(_lib.sgp_collision_graph_batched(self.ptr, len(off) - 1, off.ctypes.data_as(ctypes.c_void_p),
                                                  _ptr(pos), _ptr(radii), ctypes.byref(g.ptr)))
        return g

    def pcg_solve_batched(self, M: Matrix, Fh: Factor | None, offsets, F: torch.Tensor,
                          v: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 100000,
                          precond: int = PRECOND_TREE, precision: int = PREC_F64, x0_given: bool = False,
                          max_outer: int = 0, inner_tol: float = 0.0, raise_on_error: bool = True):
        """Solve every instance of a batch; returns (v, [Info per instance])."""
        import numpy as np
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        k = len(off) - 1
        _check_vec(F, M.n, name="F")
        v = torch.zeros_like(F) if v is None else v
        _check_vec(v, M.n, name="v")
        o = SolveOpts(tol, maxit, precond, precision, int(x0_given), max_outer, inner_tol)
        infos = (SolveInfo * k)()
        rc = _lib.sgp_pcg_solve_batched(self.ptr, M.ptr, Fh.ptr if Fh is not None else None, k,
                                        off.ctypes.data_as(ctypes.c_void_p), _ptr(F), _ptr(v), ctypes.byref(o),
                                        ctypes.cast(infos, ctypes.c_void_p))
        out = [Info(i.iterations, i.outer_iterations, i.status, i.rel_residual, i.true_rel_residual)
               for i in infos]
        if rc != OK and (raise_on_error or rc not in (ERR_NO_CONVERGENCE,)):
            self._ok(rc)
        return v, out

    # -- learned warm start ---------------------------------------------------
    def mpnn_create(self, params) -> Mpnn:
        import numpy as np
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        net = Mpnn(self)
        self._ok(_lib.sgp_mpnn_create(self.ptr, p.ctypes.data_as(ctypes.c_void_p), p.size,
                                      ctypes.byref(net.ptr)))
        return net

    def mpnn_forward(self, net: Mpnn, M: Matrix, Fh: Factor, F: torch.Tensor, v_prev: torch.Tensor | None = None,
                     v0: torch.Tensor | None = None) -> torch.Tensor:
        _check_vec(F, M.n, name="F")
        if v_prev is not None:
            _check_vec(v_prev, M.n, name="v_prev")
        v0 = torch.empty_like(F) if v0 is None else v0
        _check_vec(v0, M.n, name="v0")
        net._M = M  # the activations refer to the matrix's neighbour lists
        self._ok(_lib.sgp_mpnn_forward(self.ptr, net.ptr, M.ptr, Fh.ptr, _ptr(F), _ptr(v_prev), _ptr(v0)))
        return v0

    def mpnn_backward(self, net: Mpnn, v_target: torch.Tensor, loss: int = MPNN_LOSS_L2) -> float:
        _check_vec(v_target, net._M.n, name="v_target")
        L = ctypes.c_double()
        self._ok(_lib.sgp_mpnn_backward(self.ptr, net.ptr, _ptr(v_target), loss, ctypes.byref(L)))
        return L.value

    def mpnn_step(self, net: Mpnn, lr: float):
        self._ok(_lib.sgp_mpnn_step(self.ptr, net.ptr, float(lr)))

    def warm_start(self, net: Mpnn, M: Matrix, Fh: Factor, F: torch.Tensor, v_prev: torch.Tensor | None = None,
                   v0: torch.Tensor | None = None, mr_scale: bool = False):
        """(v0, used): the network's guess, or zeros when it does not beat
        the zero guess on the residual."""
        _check_vec(F, M.n, name="F")
        if v_prev is not None:
            _check_vec(v_prev, M.n, name="v_prev")
        v0 = torch.empty_like(F) if v0 is None else v0
        _check_vec(v0, M.n, name="v0")
        used = ctypes.c_int32()
        net._M = M
        self._ok(_lib.sgp_warm_start(self.ptr, net.ptr, M.ptr, Fh.ptr, _ptr(F), _ptr(v_prev), _ptr(v0),
                                     WARM_MR_SCALE if mr_scale else 0, ctypes.byref(used)))
        return v0, bool(used.value)

    # -- tuning ------------------------------------------------------------------
    def get_tuning(self) -> dict:
        t = Tuning()
        self._ok(_lib.sgp_get_tuning(self.ptr, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, spmv_lpr: int = 0, tail_cap: int = 1024, batch_chunk: int = 0, spmv_ilp: int = 0,
                   bin_cap: int = 0):
        """Set the launch-shape knobs (the defaults are the library's)."""
        t = Tuning(spmv_lpr, tail_cap, batch_chunk, spmv_ilp, bin_cap, 0.0)
        self._ok(_lib.sgp_set_tuning(self.ptr, ctypes.byref(t)))

    def autotune(self, M: Matrix, T: Tree | None, Fh: Factor | None, F: torch.Tensor, offsets=None,
                 precond: int = PRECOND_TREE, precision: int = PREC_F64, iterations: int = 30,
                 tol: float = 1e-8, maxit: int = 100000) -> dict:
        """Pick the launch-shape knobs: per candidate, `iterations` PCG
        iterations, or (iterations=0) a whole solve to `tol` plus the factor
        build.  Fh is rebuilt in place for each factor-shape candidate."""
        import numpy as np
        _check_vec(F, M.n, name="F")
        o = SolveOpts(tol, maxit if iterations == 0 else iterations, precond, precision, 0, 0, 0.0)
        t = Tuning()
        if offsets is not None:
            off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
            k, offp = len(off) - 1, off.ctypes.data_as(ctypes.c_void_p)
        else:
            k, offp = 0, None
        self._ok(_lib.sgp_autotune(self.ptr, M.ptr, T.ptr if T is not None else None,
                                   ctypes.byref(Fh.ptr) if Fh is not None else None, k, offp, _ptr(F),
                                   ctypes.byref(o), iterations, ctypes.byref(t)))
        return t.as_dict()

    # -- instrumentation ---------------------------------------------------
    def set_kernel_timing(self, enable: bool):
        self._ok(_lib.sgp_set_kernel_timing(self.ptr, int(enable)))

    def kernel_time(self, kclass: int, reset: bool = False):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._ok(_lib.sgp_kernel_time(self.ptr, kclass, ctypes.byref(ms), ctypes.byref(n), int(reset)))
        return ms.value, n.value

    def launch_count(self, reset: bool = False) -> int:
        c = ctypes.c_int64()
        self._ok(_lib.sgp_launch_count(self.ptr, ctypes.byref(c), int(reset)))
        return c.value


def version() -> str:
    return load_library().sgp_version().decode()
