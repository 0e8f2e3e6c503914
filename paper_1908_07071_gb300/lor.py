"""ctypes binding of the C ABI in include/lor.h (argument marshalling only).

Every numerical step runs in the CUDA library ``liblor.so``; this module only
checks tensor dtypes/sizes and passes raw device pointers and the current CUDA
stream.  Importing it raises if the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblor.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lor.h")

LOR_OK, LOR_EINVAL, LOR_ENOMEM, LOR_ECUDA, LOR_EBREAKDOWN, LOR_ENAN, LOR_ENOCONV, LOR_ETIMEOUT, LOR_ESTATE = range(9)
LOR_CG, LOR_DG_IP, LOR_DG_BR2 = 0, 1, 2
LOR_FP64, LOR_FP32, LOR_MIXED = 0, 1, 2
ORDER_LEX, ORDER_RCM, ORDER_MDF = 0, 1, 2
STATUS_NAMES = {0: "LOR_OK", 1: "LOR_EINVAL", 2: "LOR_ENOMEM", 3: "LOR_ECUDA", 4: "LOR_EBREAKDOWN",
                5: "LOR_ENAN", 6: "LOR_ENOCONV", 7: "LOR_ETIMEOUT", 8: "LOR_ESTATE"}


class LorError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def measure_fp64_peak():
    """FP64 FMA throughput of the current CUDA device in TFLOP/s (lor_measure_fp64_peak)."""
    v = ctypes.c_double(0.0)
    st = load().lor_measure_fp64_peak(ctypes.byref(v))
    if st != LOR_OK:
        raise LorError(st, "FP64 peak probe failed")
    return v.value


def box_ordering(dims, ordering, a27=None):
    """ILU(0) ordering of a box of dims = (A, B[, C]) nodes (lor_box_ordering, host only):
    box indices in elimination order.  a27: (nodes, 3^d) stencil values, needed for MDF."""
    dim = len(dims)
    A, B = int(dims[0]), int(dims[1])
    C = int(dims[2]) if dim == 3 else 1
    n = A * B * C
    perm = np.zeros(n, dtype=np.int32)
    buf = None
    if a27 is not None:
        buf = np.ascontiguousarray(a27, dtype=np.float64)
        if buf.shape != (n, 27 if dim == 3 else 9):
            raise ValueError("a27 must have shape (nodes, 3^d)")
    st = load().lor_box_ordering(dim, A, B, C, int(ordering), None if buf is None else buf.ctypes.data_as(ctypes.c_void_p),
                                 perm.ctypes.data_as(ctypes.c_void_p))
    if st != LOR_OK:
        raise LorError(st, "lor_box_ordering failed")
    return perm.astype(np.int64)


def box_ilu0(dims, a27, perm):
    """ILU(0) of a box matrix in the order perm (lor_box_ilu0, host only): the factors in
    the stencil layout of a27 (lower multipliers at earlier neighbours, u_ii at the centre,
    upper entries at later ones) and the dependency level of every node."""
    dim = len(dims)
    A, B = int(dims[0]), int(dims[1])
    C = int(dims[2]) if dim == 3 else 1
    n = A * B * C
    buf = np.ascontiguousarray(a27, dtype=np.float64)
    if buf.shape != (n, 27 if dim == 3 else 9):
        raise ValueError("a27 must have shape (nodes, 3^d)")
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    if pm.shape != (n,):
        raise ValueError("perm must have one entry per node")
    lu = np.zeros_like(buf)
    level = np.zeros(n, dtype=np.int32)
    vp = ctypes.c_void_p
    st = load().lor_box_ilu0(dim, A, B, C, buf.ctypes.data_as(vp), pm.ctypes.data_as(vp), lu.ctypes.data_as(vp),
                             level.ctypes.data_as(vp))
    if st != LOR_OK:
        raise LorError(st, "lor_box_ilu0 failed")
    return lu, level


class Options(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("disc", ctypes.c_int), ("eta", ctypes.c_double),
                ("mg_levels", ctypes.c_int), ("prec", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_it", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("factor_bf16", ctypes.c_int),
                ("weighting", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("nvec", ctypes.c_longlong), ("ndof", ctypes.c_longlong), ("npatch", ctypes.c_longlong),
                ("ncoarse", ctypes.c_longlong), ("levels", ctypes.c_int), ("coarse_levels", ctypes.c_int),
                ("factor_rows", ctypes.c_longlong), ("device_bytes", ctypes.c_size_t)]


_lib = None


def load():
    """Loads liblor.so (raises FileNotFoundError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pi, pd = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.lor_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.lor_default_options.restype = None
    lib.lor_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options), vp, vp, vp]
    lib.lor_setup.argtypes = [vp]
    lib.lor_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.lor_rhs.argtypes = [vp, i, vp]
    lib.lor_rhs_f.argtypes = [vp, vp, vp]
    lib.lor_measure_fp64_peak.argtypes = [pd]
    lib.lor_quadrature_points.argtypes = [vp, vp]
    lib.lor_apply_A.argtypes = [vp, vp, vp, i]
    lib.lor_apply_P.argtypes = [vp, vp, vp, i]
    lib.lor_pcg_solve.argtypes = [vp, vp, vp, pi, pd]
    lib.lor_pcg_solve_host.argtypes = [vp, vp, vp, pi, pd]
    lib.lor_residual_history.argtypes = [vp, pd, i, pi]
    lib.lor_last_error.argtypes = [vp]
    lib.lor_last_error.restype = ctypes.c_char_p
    lib.lor_destroy.argtypes = [vp]
    lib.lor_destroy.restype = None
    lib.lor_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), vp]
    lib.lor_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), pi, pd]
    lib.lor_batch_stats.argtypes = [vp, pd, pi]
    lib.lor_batch_destroy.argtypes = [vp]
    lib.lor_batch_destroy.restype = None
    for name in ("lor_batch_create", "lor_batch_solve", "lor_batch_stats"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lor_learned_params.argtypes = [vp, vp, vp, i]
    lib.lor_learned_enable.argtypes = [vp, i]
    lib.lor_learned_variant.argtypes = [vp, i]
    lib.lor_learned_train.argtypes = [vp, i, i, ctypes.c_float, ctypes.c_ulonglong, vp]
    lib.lor_learned_eval.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    for name in ("lor_learned_params", "lor_learned_enable", "lor_learned_variant", "lor_learned_train",
                 "lor_learned_eval"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lor_rhs_static.argtypes = [i, i, i, i, i, vp, i, vp, vp]
    lib.lor_rhs_static.restype = ctypes.c_int
    lib.lor_device_status.argtypes = [vp]
    lib.lor_selftest_wait.argtypes = [vp, i]
    lib.lor_set_prec.argtypes = [vp, i]
    lib.lor_set_weighting.argtypes = [vp, i]
    lib.lor_set_schwarz.argtypes = [vp, i]
    lib.lor_set_ordering.argtypes = [vp, i]
    lib.lor_set_patch_spans.argtypes = [vp, vp]
    lib.lor_box_ordering.argtypes = [i, i, i, i, i, vp, vp]
    lib.lor_box_ilu0.argtypes = [i, i, i, i, vp, vp, vp, vp]
    lib.lor_patch_ordering.argtypes = [vp, i, ctypes.c_longlong, vp, i, ctypes.POINTER(i)]
    lib.lor_coefficient_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.lor_coefficient_points.argtypes = [vp, vp, vp]
    lib.lor_set_coefficient.argtypes = [vp, vp, vp]
    lib.lor_set_node_coordinates.argtypes = [vp, vp]
    lib.lor_pcg_state_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.lor_pcg_state_save.argtypes = [vp, vp, vp, ctypes.c_size_t]
    lib.lor_pcg_resume.argtypes = [vp, vp, ctypes.c_size_t, vp, vp, ctypes.POINTER(i), pd]
    lib.lor_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.lor_profile.argtypes = [vp, i]
    lib.lor_profile_read.argtypes = [vp, i, pd, ctypes.POINTER(ctypes.c_longlong)]
    for name in ("lor_coefficient_sizes", "lor_coefficient_points", "lor_set_coefficient", "lor_set_node_coordinates",
                 "lor_pcg_state_size", "lor_pcg_state_save", "lor_pcg_resume",
                 "lor_device_status", "lor_selftest_wait", "lor_set_prec", "lor_set_weighting", "lor_set_schwarz", "lor_set_ordering", "lor_set_patch_spans", "lor_box_ordering", "lor_box_ilu0", "lor_patch_ordering", "lor_launch_count", "lor_profile", "lor_profile_read", "lor_create", "lor_setup", "lor_get_info", "lor_rhs", "lor_rhs_f", "lor_measure_fp64_peak", "lor_quadrature_points", "lor_apply_A", "lor_apply_P",
                 "lor_pcg_solve", "lor_pcg_solve_host", "lor_residual_history"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def header_functions():
    """Names of the functions declared in include/lor.h."""
    txt = open(HEADER).read()
    decl = r"^\s*(?:lor_status|void|const\s+char\s*\*)\s*(lor_\w+)\s*\("
    return sorted(set(re.findall(decl, txt, re.M)))


def _ptr(t, dtype, n, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def coefficient_points(lib, ctx, dim):
    """Host coordinates of the coefficient sample points of a created context: the K_p
    Gauss points (nq, dim) and the LOR sub-cell Gauss points (nh, dim)."""
    nq, nh = ctypes.c_longlong(0), ctypes.c_longlong(0)
    st = lib.lor_coefficient_sizes(ctx, ctypes.byref(nq), ctypes.byref(nh))
    if st != LOR_OK:
        raise LorError(st, "lor_coefficient_sizes")
    xq = np.empty((nq.value, dim))
    xh = np.empty((nh.value, dim))
    st = lib.lor_coefficient_points(ctx, xq.ctypes.data_as(ctypes.c_void_p), xh.ctypes.data_as(ctypes.c_void_p))
    if st != LOR_OK:
        raise LorError(st, "lor_coefficient_points")
    return xq, xh


class Solver:
    """One LOR-preconditioned problem on the current CUDA device and stream."""

    def __init__(self, vertices, kappa, p, *, mg_levels=0, prec=LOR_FP64, rtol=1e-8, max_it=1000,
                 inner_rtol=1e-3, factor_bf16=False, disc=LOR_CG, eta=1.0, weighting=0, coefficient=None,
                 node_coordinates=None, ordering=0, patch_spans=None, stream=None):
        """vertices (dim, nz+1, ny+1, nx+1) and kappa (nz, ny, nx): numpy arrays or torch tensors, on the
        host or on the device (lor_create copies them either way).
        coefficient: optional callable b(X) of physical points X (n, dim) -> (n,) replacing the
        per-element kappa (CG only); it is evaluated at the points lor_coefficient_points lists.
        node_coordinates: optional (ntot, dim) physical coordinates of the level-0 GLL nodes in
        L-vector order, for curved (isoparametric) elements (CG only).
        ordering: ILU(0) ordering of the patch levels, 0 lexicographic, 1 RCM, 2 MDF
        (ORDER_LEX / ORDER_RCM / ORDER_MDF).
        patch_spans: optional int array (npatch, dim, 2): elements (lo, hi) each patch takes on
        either side of its vertex along each axis (1, 1 = the vertex patch); CG only."""
        import torch
        self.lib = load()

        def mesh_array(a):
            # torch CUDA tensors go to lor_create as device pointers, anything else as host arrays
            if isinstance(a, torch.Tensor) and a.is_cuda:
                a = a.detach().to(torch.float64).contiguous()
                return a, ctypes.c_void_p(a.data_ptr())
            a = np.ascontiguousarray(a, dtype=np.float64)
            return a, a.ctypes.data_as(ctypes.c_void_p)

        vertices, vptr = mesh_array(vertices)
        kappa, kptr = mesh_array(kappa)
        dim = vertices.shape[0]
        n = list(reversed(kappa.shape))
        opt = Options()
        self.lib.lor_default_options(ctypes.byref(opt))
        opt.dim, opt.p = dim, p
        opt.nx, opt.ny = n[0], n[1]
        opt.nz = n[2] if dim == 3 else 1
        opt.mg_levels, opt.prec, opt.rtol, opt.max_it = mg_levels, prec, rtol, max_it
        opt.inner_rtol, opt.factor_bf16 = inner_rtol, int(bool(factor_bf16))
        opt.disc, opt.eta = disc, eta
        opt.weighting = int(weighting)
        self.opt = opt
        self.dim, self.p, self.n = dim, p, tuple(n)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        ctx = ctypes.c_void_p()
        st = self.lib.lor_create(ctypes.byref(ctx), ctypes.byref(opt), vptr, kptr, ctypes.c_void_p(stream))
        if st != LOR_OK:
            raise LorError(st, "lor_create rejected the input")
        self.ctx = ctx
        if ordering:
            self._check(self.lib.lor_set_ordering(ctx, int(ordering)))
        if patch_spans is not None:
            sp = np.ascontiguousarray(patch_spans, dtype=np.int32)
            if sp.shape != (int(np.prod([v + 1 for v in n])), dim, 2):
                raise ValueError("patch_spans must have shape (npatch, dim, 2)")
            self._check(self.lib.lor_set_patch_spans(ctx, sp.ctypes.data_as(ctypes.c_void_p)))
        if node_coordinates is not None:
            Xn = np.ascontiguousarray(np.asarray(node_coordinates, dtype=np.float64).T)
            ntot = int(np.prod([v * p + 1 for v in n]))
            if Xn.shape != (dim, ntot):
                raise ValueError(f"node_coordinates must have shape ({ntot}, {dim})")
            self._check(self.lib.lor_set_node_coordinates(ctx, Xn.ctypes.data_as(ctypes.c_void_p)))
        if coefficient is not None:
            xq, xh = coefficient_points(self.lib, ctx, dim)
            bq = np.ascontiguousarray(coefficient(xq), dtype=np.float64)
            bh = np.ascontiguousarray(coefficient(xh), dtype=np.float64)
            if bq.shape != (len(xq),) or bh.shape != (len(xh),):
                raise ValueError("coefficient must map (n, dim) points to n values")
            self._check(self.lib.lor_set_coefficient(ctx, bq.ctypes.data_as(ctypes.c_void_p),
                                                     bh.ctypes.data_as(ctypes.c_void_p)))
        self._check(self.lib.lor_setup(ctx))
        self.info = Info()
        self._check(self.lib.lor_get_info(ctx, ctypes.byref(self.info)))
        self.nvec = self.info.nvec
        self.shape = tuple(reversed([v * p + 1 for v in n]))

    def _check(self, st):
        if st != LOR_OK:
            raise LorError(st, self.lib.lor_last_error(self.ctx).decode())

    def close(self):
        """Frees the context (lor_destroy); later calls on this Solver fail."""
        if getattr(self, "ctx", None):
            self.lib.lor_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dt(self, prec):
        import torch
        return torch.float64 if prec == LOR_FP64 else torch.float32

    def rhs(self, b, kind=0):
        """b = M f into the float64 CUDA tensor b: kind 0 is f = 1, kind 1 the manufactured d pi^2 prod sin(pi x_a)."""
        import torch
        self._check(self.lib.lor_rhs(self.ctx, kind, _ptr(b, torch.float64, self.nvec, "b")))

    def quadrature_points(self):
        """Physical coordinates (nel (p+1)^d, dim) of the Gauss points at which rhs_f takes f."""
        Q = self.p + 1
        nq = int(np.prod(self.n)) * Q ** self.dim
        xq = np.empty(nq * self.dim)
        self._check(self.lib.lor_quadrature_points(self.ctx, xq.ctypes.data_as(ctypes.c_void_p)))
        return xq.reshape(nq, self.dim)

    def rhs_f(self, fq, b):
        """b = M f from f at quadrature_points() (float64 CUDA tensor fq) into the float64 CUDA tensor b."""
        import torch
        Q = self.p + 1
        nq = int(np.prod(self.n)) * Q ** self.dim
        self._check(self.lib.lor_rhs_f(self.ctx, _ptr(fq, torch.float64, nq, "fq"), _ptr(b, torch.float64, self.nvec, "b")))

    def apply_A(self, x, y, prec=LOR_FP64):
        """y = A x (matrix-free operator) in FP64 (float64 tensors) or FP32 (float32 tensors)."""
        dt = self._dt(prec)
        self._check(self.lib.lor_apply_A(self.ctx, _ptr(x, dt, self.nvec, "x"), _ptr(y, dt, self.nvec, "y"), prec))

    def apply_P(self, r, z, prec=LOR_FP64):
        """z = B r (LOR additive-Schwarz preconditioner) in FP64 or FP32."""
        dt = self._dt(prec)
        self._check(self.lib.lor_apply_P(self.ctx, _ptr(r, dt, self.nvec, "r"), _ptr(z, dt, self.nvec, "z"), prec))

    def solve(self, b, x):
        """PCG (FP64, or mixed precision per prec) of A x = b on CUDA tensors; returns (iterations, rel_res)."""
        import torch
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.lib.lor_pcg_solve(self.ctx, _ptr(b, torch.float64, self.nvec, "b"),
                                           _ptr(x, torch.float64, self.nvec, "x"), ctypes.byref(it),
                                           ctypes.byref(rr)))
        return it.value, rr.value

    def solve_host(self, b: np.ndarray, x: np.ndarray):
        """The same solve from host float64 arrays (copies inside the call)."""
        if b.dtype != np.float64 or x.dtype != np.float64 or b.size != self.nvec or x.size != self.nvec:
            raise ValueError("host vectors must be float64 of length nvec")
        if not (b.flags.c_contiguous and x.flags.c_contiguous):
            raise ValueError("host vectors must be contiguous")
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.lib.lor_pcg_solve_host(self.ctx, b.ctypes.data_as(ctypes.c_void_p),
                                                x.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it),
                                                ctypes.byref(rr)))
        return it.value, rr.value

    def state_save(self, x):
        """The FP64 PCG state of the last solve (x its solution) as a host byte array."""
        import torch
        nb = ctypes.c_size_t(0)
        self._check(self.lib.lor_pcg_state_size(self.ctx, ctypes.byref(nb)))
        buf = np.empty(nb.value, dtype=np.uint8)
        self._check(self.lib.lor_pcg_state_save(self.ctx, _ptr(x, torch.float64, self.nvec, "x"),
                                                buf.ctypes.data_as(ctypes.c_void_p), nb.value))
        return buf

    def resume(self, state, b, x):
        """Continues PCG from `state` (state_save of the same problem); returns (iterations, rel_res)."""
        import torch
        state = np.ascontiguousarray(state, dtype=np.uint8)
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.lib.lor_pcg_resume(self.ctx, state.ctypes.data_as(ctypes.c_void_p), state.size,
                                            _ptr(b, torch.float64, self.nvec, "b"),
                                            _ptr(x, torch.float64, self.nvec, "x"), ctypes.byref(it),
                                            ctypes.byref(rr)))
        return it.value, rr.value

    def device_status(self):
        """Synchronizes and checks for a bounded device wait that ran out (raises LorError LOR_ETIMEOUT)."""
        self._check(self.lib.lor_device_status(self.ctx))

    def selftest_wait(self, polls=1 << 12):
        """Runs the bounded-wait self-test; returns the library status (LOR_ETIMEOUT expected)."""
        return self.lib.lor_selftest_wait(self.ctx, polls)

    def patch_ordering(self, level, patch):
        """ILU(0) order of one patch level: box indices of its rows in elimination order."""
        cnt = ctypes.c_int(0)
        self._check(self.lib.lor_patch_ordering(self.ctx, int(level), int(patch), None, 0, ctypes.byref(cnt)))
        out = np.zeros(max(cnt.value, 1), dtype=np.int32)
        self._check(self.lib.lor_patch_ordering(self.ctx, int(level), int(patch), out.ctypes.data_as(ctypes.c_void_p),
                                                cnt.value, ctypes.byref(cnt)))
        return out[:cnt.value].astype(np.int64)

    def set_schwarz(self, mode):
        """0: additive coarse space (Eq. (as)); 1: hybrid, coarse correction multiplicative."""
        self._check(self.lib.lor_set_schwarz(self.ctx, int(mode)))

    def set_weighting(self, weighting):
        """0: unit patch weights (the paper's method); 1: counting-matrix weights;
        2: partition-of-unity weights (square root of each patch's vertex function)."""
        self._check(self.lib.lor_set_weighting(self.ctx, int(weighting)))

    def set_prec(self, prec):
        """LOR_FP64 or LOR_MIXED for later solves."""
        self._check(self.lib.lor_set_prec(self.ctx, prec))

    def launches(self):
        """Number of kernels this context has launched so far."""
        n = ctypes.c_longlong(0)
        self._check(self.lib.lor_launch_count(self.ctx, ctypes.byref(n)))
        return n.value

    def profile(self, on):
        """Starts (clearing earlier records) or stops CUDA-event timing of the hot kernel classes."""
        self._check(self.lib.lor_profile(self.ctx, int(on)))

    def profile_read(self, kernel):
        """(total ms, launches) of one kernel class since profile(True)."""
        ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
        self._check(self.lib.lor_profile_read(self.ctx, kernel, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # ---- learned per-patch correction
    NPARAM = 8241

    def learned_params(self, params=None):
        """Sets (if given) and returns the FP32 parameter vector."""
        out = np.zeros(self.NPARAM, dtype=np.float32)
        pin = None
        if params is not None:
            pin = np.ascontiguousarray(params, dtype=np.float32)
            assert pin.size == self.NPARAM
        self._check(self.lib.lor_learned_params(self.ctx, None if pin is None else pin.ctypes.data_as(ctypes.c_void_p),
                                                out.ctypes.data_as(ctypes.c_void_p), self.NPARAM))
        return out

    def learned_enable(self, on=True):
        """Switches the learned per-patch correction (flexible CG) on or off."""
        self._check(self.lib.lor_learned_enable(self.ctx, int(bool(on))))

    def learned_variant(self, variant):
        """0: correction added after the V(1,1) cycle; 1: it replaces the level-0 post-smoothing."""
        self._check(self.lib.lor_learned_variant(self.ctx, int(variant)))

    def learned_train(self, steps, batch=64, lr=1e-3, seed=0):
        """Trains the network on the GPU (Adam); returns the loss of every step."""
        hist = np.zeros(max(steps, 1), dtype=np.float32)
        self._check(self.lib.lor_learned_train(self.ctx, steps, batch, ctypes.c_float(lr), seed,
                                               hist.ctypes.data_as(ctypes.c_void_p)))
        return hist[:steps]

    def learned_eval(self, ids, t, delta=None):
        """ids: int32 CUDA tensor of interior patch ids; t, delta: float32 (npatch, V).
        Returns (correction, per-patch loss or None, summed gradient or None)."""
        import torch
        n = ids.numel()
        c = torch.empty_like(t)
        loss = torch.empty(n, dtype=torch.float32, device="cuda") if delta is not None else None
        grad = np.zeros(self.NPARAM, dtype=np.float32) if delta is not None else None
        self._check(self.lib.lor_learned_eval(
            self.ctx, n, ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(t.data_ptr()),
            None if delta is None else ctypes.c_void_p(delta.data_ptr()), ctypes.c_void_p(c.data_ptr()),
            None if loss is None else ctypes.c_void_p(loss.data_ptr()),
            None if grad is None else grad.ctypes.data_as(ctypes.c_void_p)))
        return c, loss, grad

    def history(self):
        """Residual 2-norms of the last solve, one per iteration."""
        cnt = ctypes.c_int(0)
        self.lib.lor_residual_history(self.ctx, None, 0, ctypes.byref(cnt))
        out = (ctypes.c_double * max(cnt.value, 1))()
        self.lib.lor_residual_history(self.ctx, out, cnt.value, ctypes.byref(cnt))
        return np.array(out[:cnt.value])


class Batch:
    """Batched flexible-CG solves of several Solver contexts (one CUDA graph per iteration)."""

    def __init__(self, solvers, stream=None):
        import torch
        self.lib = load()
        self.solvers = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.ctx for s in self.solvers])
        b = ctypes.c_void_p()
        st = self.lib.lor_batch_create(ctypes.byref(b), len(self.solvers), arr, ctypes.c_void_p(stream))
        if st != LOR_OK:
            raise LorError(st, "lor_batch_create failed")
        self.b = b

    def solve(self, bs, xs):
        """Solves every context's problem (lists of float64 CUDA tensors); returns (iterations, rel_res) lists."""
        import torch
        n = len(self.solvers)
        pb = (ctypes.c_void_p * n)(*[_ptr(b, torch.float64, s.nvec, "b").value for b, s in zip(bs, self.solvers)])
        px = (ctypes.c_void_p * n)(*[_ptr(x, torch.float64, s.nvec, "x").value for x, s in zip(xs, self.solvers)])
        its = (ctypes.c_int * n)()
        rel = (ctypes.c_double * n)()
        st = self.lib.lor_batch_solve(self.b, pb, px, its, rel)
        if st != LOR_OK:
            raise LorError(st, "lor_batch_solve failed")
        return list(its), list(rel)

    def stats(self):
        """(milliseconds of the graph-launch loop of the last solve, nodes of the captured graph)."""
        ms, nodes = ctypes.c_double(0.0), ctypes.c_int(0)
        self.lib.lor_batch_stats(self.b, ctypes.byref(ms), ctypes.byref(nodes))
        return ms.value, nodes.value

    def close(self):
        """Frees the batch (the contexts stay)."""
        if getattr(self, "b", None):
            self.lib.lor_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
