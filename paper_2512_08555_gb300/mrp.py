"""Python binding of libmrp (ctypes): argument marshalling only.

Every step of the solve runs in the CUDA library; PyTorch supplies device
memory and the current stream.  There is no CPU fallback: if the library
is missing or cannot be loaded, constructing a solver raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmrp.so")

MRP_OK = 0
MRP_ERR_NOT_CONVERGED = 5
MRP_LAUNCH_NOSTAGE = 4096      # flag of the launch option (include/mrp.h)
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid forest", 3: "CUDA error", 4: "out of memory",
          5: "not converged", 6: "timeout", 7: "numerical", 9: "unsupported",
          10: "too large for the fixed scratch"}
FIELDS = {"U": 0, "F": 1, "R": 2, "UHAT": 3, "FRAW": 4}
STEPS = {"prepare_rhs": 0, "ghost_u": 1, "smooth": 2, "residual": 3, "restrict": 4,
         "coarse_solve": 5, "prolong": 6, "vcycle": 7, "coarse_solve_f32": 8}
EXPORTED = ["mrp_create", "mrp_solve", "mrp_solve_adjoint", "mrp_destroy", "mrp_error_string",
            "mrp_level_count", "mrp_level_info", "mrp_field_copy", "mrp_step", "mrp_lgf_extent",
            "mrp_lgf_copy", "mrp_fft_shape", "mrp_profile_enable", "mrp_profile_read",
            "mrp_coarse_solve_noalloc", "mrp_adjoint_len", "mrp_adjoint_op", "mrp_solve_graph",
            "mrp_solve_host", "mrp_fma_peak", "mrp_convert_check", "mrp_fixed_check"]
ADJ_OPS = {"cycle_T": 0, "res_T": 1, "out_T": 2, "rhs_T": 3}
PHASES = ["ghost", "smooth", "residual", "restrict", "coarse_fft", "prolong", "norm", "other"]
PHASES16 = [p + "_f64" for p in PHASES] + [p + "_f32" for p in PHASES]


class MrpError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")


class _Forest(C.Structure):
    _fields_ = [("nb0", C.c_int32 * 3), ("n", C.c_int32), ("origin", C.c_double * 3), ("h0", C.c_double),
                ("n_leaves", C.c_int32), ("leaf_level", C.POINTER(C.c_int32)),
                ("leaf_ijk", C.POINTER(C.c_int32)), ("ncomp", C.c_int32)]


class _Options(C.Structure):
    _fields_ = [("order", C.c_int32), ("tol", C.c_double), ("stop_rule", C.c_int32), ("max_cycles", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("precision", C.c_int32), ("inner_cycles", C.c_int32),
                ("max_outer", C.c_int32), ("launch", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("ir_steps", C.c_int32), ("residual", C.c_double), ("cauchy", C.c_double),
                ("fstar_max", C.c_double), ("leaf_nodes", C.c_int64), ("total_nodes", C.c_int64),
                ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path=LIB_PATH):
    """Load libmrp.so (built by ``paper_2512_08555_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.mrp_create.argtypes = [C.POINTER(P), C.POINTER(_Forest), I32, C.POINTER(_Options)]
    lib.mrp_solve.argtypes = [P, P, P, P, C.POINTER(Stats)]
    lib.mrp_solve_adjoint.argtypes = [P, P, P, P, C.POINTER(Stats)]
    lib.mrp_destroy.argtypes = [P]
    lib.mrp_error_string.argtypes = [C.c_int]
    lib.mrp_error_string.restype = C.c_char_p
    lib.mrp_level_count.argtypes = [P, C.POINTER(I32)]
    lib.mrp_level_info.argtypes = [P, I32, C.POINTER(I32), P, P]
    lib.mrp_field_copy.argtypes = [P, I32, I32, P, I32, P]
    lib.mrp_step.argtypes = [P, I32, I32, P, P]
    lib.mrp_lgf_extent.argtypes = [P, C.POINTER(I32)]
    lib.mrp_lgf_copy.argtypes = [P, I32, P]
    lib.mrp_fft_shape.argtypes = [P, P]
    lib.mrp_profile_enable.argtypes = [P, I32]
    lib.mrp_profile_read.argtypes = [P, I32, P, P, P, I32]
    lib.mrp_coarse_solve_noalloc.argtypes = [P, P, P, P]
    lib.mrp_adjoint_len.argtypes = [P, C.POINTER(I64)]
    lib.mrp_adjoint_op.argtypes = [P, I32, P, P, P]
    lib.mrp_solve_graph.argtypes = [P, P, P, P, C.POINTER(Stats)]
    lib.mrp_solve_host.argtypes = [P, P, P, P, C.POINTER(Stats)]
    lib.mrp_fma_peak.argtypes = [I32, C.POINTER(D), P]
    lib.mrp_convert_check.argtypes = [P, P, P, P, I64, P]
    lib.mrp_fixed_check.argtypes = [P, I32, P, P, P, I64, P]
    for name in EXPORTED:
        getattr(lib, name).restype = getattr(lib, name).restype or C.c_int
    lib.mrp_error_string.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc, where, allow=()):
    if rc != MRP_OK and rc not in allow:
        raise MrpError(rc, where)
    return rc


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Solver:
    """Solver for one forest, or a batch of forests (``mrp_create`` / ``mrp_solve``).

    ``forest``: a forest, or a list of forests solved together.  ``ncomp``:
    right-hand sides per forest (an int for all, or one per forest).  The
    caller layout of f and u is [forest][component][leaf][n][n][n], float64.
    """

    def __init__(self, forest, order=4, tol=1e-10, max_cycles=50, nu1=3, nu2=3, precision="fp64",
                 inner_cycles=0, max_outer=0, ncomp=1, stop="residual", launch=0):
        import torch  # noqa: F401  (CUDA context and memory come from torch)
        self.lib = load_library()
        forests = list(forest) if isinstance(forest, (list, tuple)) else [forest]
        comps = list(ncomp) if isinstance(ncomp, (list, tuple)) else [int(ncomp)] * len(forests)
        if len(comps) != len(forests):
            raise ValueError("ncomp needs one entry per forest")
        self.forests = forests
        self.forest = forests[0]
        self.ncomp = comps
        self.n = int(forests[0].n)
        self.n_leaves = int(forests[0].n_leaves)
        self.elems = sum(int(c) * int(f.n_leaves) * int(f.n) ** 3 for f, c in zip(forests, comps))
        self._keep = []
        arr = (_Forest * len(forests))()
        for i, (f, c) in enumerate(zip(forests, comps)):
            lev = np.ascontiguousarray(f.leaf_level, dtype=np.int32)
            ijk = np.ascontiguousarray(f.leaf_ijk, dtype=np.int32).reshape(-1, 3)
            self._keep += [lev, ijk]
            fd = arr[i]
            fd.nb0[:] = [int(v) for v in f.nb0]
            fd.n = int(f.n)
            fd.origin[:] = [float(v) for v in f.origin]
            fd.h0 = float(f.h0)
            fd.n_leaves = int(f.n_leaves)
            fd.leaf_level = lev.ctypes.data_as(C.POINTER(C.c_int32))
            fd.leaf_ijk = ijk.ctypes.data_as(C.POINTER(C.c_int32))
            fd.ncomp = int(c)
        op = _Options()
        op.order, op.tol, op.max_cycles = int(order), float(tol), int(max_cycles)
        op.stop_rule = {"residual": 0, "cauchy": 1}[stop]
        op.nu1, op.nu2 = int(nu1), int(nu2)
        op.precision = {"fp64": 0, "mixed": 1}[precision]
        op.inner_cycles, op.max_outer = int(inner_cycles), int(max_outer)
        op.launch = int(launch)
        self.h = C.c_void_p()
        _check(self.lib.mrp_create(C.byref(self.h), arr, len(forests), C.byref(op)), "mrp_create")

    def slices(self):
        """(start, stop) element ranges of every (forest, component) in the caller layout."""
        out, off = [], 0
        for f, c in zip(self.forests, self.ncomp):
            m = int(f.n_leaves) * int(f.n) ** 3
            for _ in range(int(c)):
                out.append((off, off + m))
                off += m
        return out

    def close(self):
        if self.h:
            self.lib.mrp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ solve
    def solve(self, f, u=None, stream=None, allow_not_converged=False):
        """u = solve(f); f, u: CUDA float64 tensors [n_leaves, n, n, n]."""
        import torch
        if f.dtype != torch.float64 or not f.is_cuda or not f.is_contiguous() or f.numel() != self.elems:
            raise ValueError("f must be a contiguous CUDA float64 tensor in the caller layout")
        if u is None:
            u = torch.empty_like(f)
        st = Stats()
        allow = (MRP_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        rc = self.lib.mrp_solve(self.h, C.c_void_p(f.data_ptr()), C.c_void_p(u.data_ptr()), _stream_ptr(stream),
                                C.byref(st))
        _check(rc, "mrp_solve", allow)
        return u, st

    def solve_graph(self, f, u=None, stream=None, allow_not_converged=False):
        """Same as ``solve``, as one CUDA graph launch (built on first use and when f or u change)."""
        import torch
        if f.dtype != torch.float64 or not f.is_cuda or not f.is_contiguous() or f.numel() != self.elems:
            raise ValueError("f must be a contiguous CUDA float64 tensor in the caller layout")
        if u is None:
            u = torch.empty_like(f)
        st = Stats()
        allow = (MRP_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        rc = self.lib.mrp_solve_graph(self.h, C.c_void_p(f.data_ptr()), C.c_void_p(u.data_ptr()), _stream_ptr(stream),
                                      C.byref(st))
        _check(rc, "mrp_solve_graph", allow)
        return u, st

    def solve_adjoint(self, w, fbar=None, stream=None, allow_not_converged=False):
        """fbar = S^T w, the gradient of <w, u> with respect to f for the converged solve.

        w, fbar: CUDA float64 tensors [n_leaves, n, n, n] (leaf layout of solve).
        """
        import torch
        if w.dtype != torch.float64 or not w.is_cuda or not w.is_contiguous() or w.numel() != self.elems:
            raise ValueError("w must be a contiguous CUDA float64 tensor in the caller layout")
        if fbar is None:
            fbar = torch.empty_like(w)
        st = Stats()
        allow = (MRP_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        rc = self.lib.mrp_solve_adjoint(self.h, C.c_void_p(w.data_ptr()), C.c_void_p(fbar.data_ptr()),
                                        _stream_ptr(stream), C.byref(st))
        _check(rc, "mrp_solve_adjoint", allow)
        return fbar, st

    def adjoint_len(self):
        v = C.c_int64()
        _check(self.lib.mrp_adjoint_len(self.h, C.byref(v)), "mrp_adjoint_len")
        return v.value

    def adjoint_op(self, name, x, stream=None):
        """One factor of the gradient (``ADJ_OPS``); see mrp_adjoint_op for the vector layouts."""
        import torch
        L = self.adjoint_len()
        out_len = {"cycle_T": L, "res_T": 2 * L, "out_T": 2 * L, "rhs_T": self.elems}[name]
        x = x.contiguous()
        out = torch.zeros(out_len, dtype=torch.float64, device="cuda")
        _check(self.lib.mrp_adjoint_op(self.h, ADJ_OPS[name], C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream)), f"mrp_adjoint_op({name})")
        return out

    # ------------------------------------------------------------------ step API
    def level_count(self):
        v = C.c_int32()
        _check(self.lib.mrp_level_count(self.h, C.byref(v)), "mrp_level_count")
        return v.value

    def level_info(self, k):
        nb = C.c_int32()
        _check(self.lib.mrp_level_info(self.h, k, C.byref(nb), None, None), "mrp_level_info")
        coords = np.zeros((nb.value, 3), np.int32)
        leaf = np.zeros(nb.value, np.uint8)
        _check(self.lib.mrp_level_info(self.h, k, C.byref(nb), coords.ctypes.data_as(C.c_void_p),
                                       leaf.ctypes.data_as(C.c_void_p)), "mrp_level_info")
        return coords, leaf.astype(bool)

    def field_shape(self, name, k):
        nb = len(self.level_info(k)[0])
        g = {"U": 1, "FRAW": 2}.get(name, 0)
        s = self.n + 2 * g
        return (nb, s, s, s)

    def field_get(self, name, k, stream=None):
        import torch
        buf = torch.empty(self.field_shape(name, k), dtype=torch.float64, device="cuda")
        _check(self.lib.mrp_field_copy(self.h, FIELDS[name], k, C.c_void_p(buf.data_ptr()), 0, _stream_ptr(stream)),
               "mrp_field_copy")
        torch.cuda.current_stream().synchronize()
        return buf

    def field_set(self, name, k, value, stream=None):
        import torch
        buf = torch.as_tensor(np.ascontiguousarray(value), dtype=torch.float64).cuda().contiguous()
        if tuple(buf.shape) != self.field_shape(name, k):
            raise ValueError("shape mismatch")
        _check(self.lib.mrp_field_copy(self.h, FIELDS[name], k, C.c_void_p(buf.data_ptr()), 1, _stream_ptr(stream)),
               "mrp_field_copy")
        torch.cuda.current_stream().synchronize()

    def step(self, name, level=0, f=None, stream=None):
        import torch
        ptr = C.c_void_p(f.data_ptr()) if f is not None else None
        _check(self.lib.mrp_step(self.h, STEPS[name], level, ptr, _stream_ptr(stream)), f"mrp_step({name})")
        torch.cuda.current_stream().synchronize()

    def lgf_table(self, nmax=None):
        ext = C.c_int32()
        _check(self.lib.mrp_lgf_extent(self.h, C.byref(ext)), "mrp_lgf_extent")
        nmax = ext.value if nmax is None else nmax
        out = np.zeros((nmax + 1,) * 3)
        _check(self.lib.mrp_lgf_copy(self.h, nmax, out.ctypes.data_as(C.c_void_p)), "mrp_lgf_copy")
        return out

    def profile(self, enable=True):
        _check(self.lib.mrp_profile_enable(self.h, 1 if enable else 0), "mrp_profile_enable")

    def profile_read(self, reset=True):
        ms = np.zeros(16)
        cnt = np.zeros(16, np.int64)
        nodes = np.zeros(16, np.int64)
        _check(self.lib.mrp_profile_read(self.h, 16, ms.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p),
                                         nodes.ctypes.data_as(C.c_void_p), 1 if reset else 0), "mrp_profile_read")
        return {p: {"ms": float(ms[i]), "launches": int(cnt[i]), "nodes": int(nodes[i])}
                for i, p in enumerate(PHASES16) if cnt[i] > 0}

    def solve_host(self, f_host, u_host=None, stream=None, allow_not_converged=False):
        """End to end from host memory through ``mrp_solve_host``: f in, solve graph, u out.

        ``f_host``/``u_host``: contiguous CPU float64 tensors in the caller
        layout (pinned for asynchronous copies at full bandwidth).
        """
        import torch
        if f_host.dtype != torch.float64 or f_host.is_cuda or not f_host.is_contiguous() or f_host.numel() != self.elems:
            raise ValueError("f_host must be a contiguous CPU float64 tensor in the caller layout")
        if u_host is None:
            u_host = torch.empty(f_host.shape, dtype=torch.float64, pin_memory=True)
        st = Stats()
        allow = (MRP_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        rc = self.lib.mrp_solve_host(self.h, C.c_void_p(f_host.data_ptr()), C.c_void_p(u_host.data_ptr()),
                                     _stream_ptr(stream), C.byref(st))
        _check(rc, "mrp_solve_host", allow)
        return u_host, st

    def fft_shape(self):
        P = np.zeros(3, np.int32)
        _check(self.lib.mrp_fft_shape(self.h, P.ctypes.data_as(C.c_void_p)), "mrp_fft_shape")
        return tuple(int(v) for v in P)


def fma_peak_tflops(precision="fp64", stream=None):
    """Measured FMA throughput of the current device (``mrp_fma_peak``), TFLOP/s."""
    lib = load_library()
    v = C.c_double()
    _check(lib.mrp_fma_peak({"fp64": 0, "fp32": 1}[precision], C.byref(v), _stream_ptr(stream)), "mrp_fma_peak")
    return v.value


def convert_check(d_in, f_in, stream=None):
    """The library's float/double conversions (``mrp_convert_check``): (float32 of d_in, float64 of f_in)."""
    import torch
    lib = load_library()
    f_out = torch.empty_like(d_in, dtype=torch.float32)
    d_out = torch.empty_like(f_in, dtype=torch.float64)
    _check(lib.mrp_convert_check(C.c_void_p(d_in.data_ptr()), C.c_void_p(f_out.data_ptr()), C.c_void_p(f_in.data_ptr()),
                                 C.c_void_p(d_out.data_ptr()), d_in.numel(), _stream_ptr(stream)), "mrp_convert_check")
    torch.cuda.current_stream().synchronize()
    return f_out, d_out


def fixed_check(u_in, shb, i_in, stream=None):
    """The leaf residual's fixed-point conversions (``mrp_fixed_check``): (int64 trunc(u_in 2^(shb+1075)),
    float64 of i_in)."""
    import torch
    lib = load_library()
    fx_out = torch.empty_like(u_in, dtype=torch.int64)
    d_out = torch.empty_like(i_in, dtype=torch.float64)
    _check(lib.mrp_fixed_check(C.c_void_p(u_in.data_ptr()), int(shb), C.c_void_p(fx_out.data_ptr()),
                               C.c_void_p(i_in.data_ptr()), C.c_void_p(d_out.data_ptr()), u_in.numel(),
                               _stream_ptr(stream)), "mrp_fixed_check")
    torch.cuda.current_stream().synchronize()
    return fx_out, d_out


def poisson_solve(solver, f):
    """u = S f with a gradient: differentiable wrapper of ``Solver.solve``.

    The backward pass is ``Solver.solve_adjoint`` (the transposed solve on the
    device), so d<w, u>/df = S^T w for the converged composite solution.
    """
    import torch

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, f_in):
            u, _ = solver.solve(f_in.contiguous())
            return u

        @staticmethod
        def backward(ctx, u_bar):
            f_bar, _ = solver.solve_adjoint(u_bar.contiguous())
            return f_bar

    return _Solve.apply(f)
