"""Thin ctypes binding of libbddc (argument marshalling only).

Names follow the C ABI in ``include/bddc.h``.  Device buffers are torch CUDA
tensors (PyTorch provides memory and streams); every step of setup and solve
runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbddc.so")

OK, NOT_CONVERGED = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
PREC_FP64, PREC_MIXED, PREC_BF16 = 0, 1, 2
EDGE_NONE, EDGE_NEW, EDGE_OLD = 0, 1, 2
ELEM_Q1, ELEM_P1 = 0, 1


class Mesh(ct.Structure):
    _fields_ = [("lo", ct.c_double * 3), ("hi", ct.c_double * 3)]


class Partition(ct.Structure):
    _fields_ = [("nsub", ct.c_int * 3), ("elems_per_slab", ct.POINTER(ct.c_int) * 3)]


class Coeffs(ct.Structure):
    _fields_ = [("nu_elem", ct.c_void_p), ("beta_node", ct.c_void_p), ("beta_const", ct.c_double * 3),
                ("c", ct.c_double), ("f_node", ct.c_void_p), ("divb_node", ct.c_void_p), ("mem", ct.c_int),
                ("g_node", ct.c_void_p)]


class Opts(ct.Structure):
    _fields_ = [("theta_E", ct.c_double), ("theta_F", ct.c_double), ("tau", ct.c_double),
                ("precision", ct.c_int), ("restart", ct.c_int), ("max_iter", ct.c_int),
                ("rtol", ct.c_double), ("edge_gep", ct.c_int), ("face_gep", ct.c_int),
                ("all_primal", ct.c_int), ("inner_rtol", ct.c_double), ("max_refine", ct.c_int),
                ("learned_skip_p", ct.c_double), ("mlp_params", ct.c_void_p), ("tensor_cores", ct.c_int),
                ("coarse_elim", ct.c_int), ("apply_launch", ct.c_int), ("cond_est", ct.c_int),
                ("element", ct.c_int), ("local_nd", ct.c_int)]


class Stats(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("refine_steps", ct.c_int), ("converged", ct.c_int),
                ("relres", ct.c_double), ("relres_global", ct.c_double), ("pnumF", ct.c_int),
                ("pnumE", ct.c_int), ("n_pi", ct.c_int), ("n_gamma", ct.c_int), ("ndof", ct.c_int),
                ("nsub", ct.c_int), ("edges_skipped", ct.c_int), ("setup_ms", ct.c_double),
                ("solve_ms", ct.c_double), ("t_assemble_ms", ct.c_double), ("t_factor_ms", ct.c_double),
                ("t_face_ms", ct.c_double), ("t_edge_ms", ct.c_double), ("t_coarse_ms", ct.c_double),
                ("jacobi_sweeps_max", ct.c_int), ("t_mesh_ms", ct.c_double), ("t_basis_ms", ct.c_double),
                ("coarse_path", ct.c_int), ("coarse_fronts", ct.c_int), ("coarse_levels", ct.c_int),
                ("coarse_factor_gflop", ct.c_double), ("kappa_est", ct.c_double),
                ("gemv_rows", ct.c_int), ("gemv_tune_us", ct.c_double), ("nd_children", ct.c_int),
                ("factor_gflop", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libbddc.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libbddc.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ct.CDLL(LIB_PATH)
    vp, ip, dp = ct.c_void_p, ct.POINTER(ct.c_int), ct.POINTER(ct.c_double)
    L.bddc_default_opts.argtypes = [ct.POINTER(Opts)]
    L.bddc_setup.argtypes = [ct.POINTER(Mesh), ct.POINTER(Coeffs), ct.POINTER(Partition), ct.c_double,
                             ct.POINTER(Opts), vp, ct.POINTER(vp)]
    L.bddc_apply.argtypes = [vp, vp, vp, ct.c_int]
    L.bddc_apply_static.argtypes = [vp, vp, vp, ct.c_int]
    L.bddc_schur_apply.argtypes = [vp, vp, vp, ct.c_int]
    L.bddc_gmres_solve.argtypes = [vp, vp, vp, ct.c_int, ct.c_int, ct.POINTER(Stats)]
    L.bddc_get_stats.argtypes = [vp, ct.POINTER(Stats)]
    L.bddc_destroy.argtypes = [vp]
    L.bddc_strerror.argtypes = [ct.c_int]
    L.bddc_strerror.restype = ct.c_char_p
    L.bddc_last_error.restype = ct.c_char_p
    L.bddc_last_error.argtypes = []
    L.bddc_get_numbering.argtypes = [vp, ip]
    L.bddc_get_schur.argtypes = [vp, ct.c_int, dp, ip]
    L.bddc_get_entity_count.argtypes = [vp, ct.c_int]
    L.bddc_get_entity.argtypes = [vp, ct.c_int, ct.c_int, ip, ip, ip, ip, dp, dp, ip]
    L.bddc_get_edge_features.argtypes = [vp, ct.POINTER(ct.c_float), ip]
    fp = ct.POINTER(ct.c_float)
    L.bddc_mlp_forward.argtypes = [fp, vp, ct.c_int, vp, vp]
    L.bddc_mlp_loss_grad.argtypes = [fp, vp, vp, ct.c_int, fp, fp, vp]
    L.bddc_mlp_train.argtypes = [fp, vp, vp, ct.c_int, ct.c_int, ct.c_float, fp, vp]
    L.bddc_tc_selftest.argtypes = [fp, fp, fp, ct.c_int, ct.c_int, ct.c_int]
    L.bddc_wait_selftest.argtypes = [ct.c_int]
    L.bddc_kernel_timer.argtypes = [ct.c_int]
    L.bddc_kernel_timer_read.argtypes = [dp, ct.POINTER(ct.c_longlong), dp, dp]
    L.bddc_kernel_launches.argtypes = []
    L.bddc_kernel_launches.restype = ct.c_ulonglong
    _lib = L
    return L


EXPORTED = ["bddc_default_opts", "bddc_setup", "bddc_apply", "bddc_schur_apply", "bddc_gmres_solve",
            "bddc_get_stats", "bddc_destroy", "bddc_strerror", "bddc_last_error", "bddc_get_numbering", "bddc_get_schur",
            "bddc_get_entity_count", "bddc_get_entity", "bddc_get_edge_features", "bddc_kernel_launches",
            "bddc_apply_static", "bddc_kernel_timer", "bddc_kernel_timer_read", "bddc_mlp_forward",
            "bddc_mlp_loss_grad", "bddc_mlp_train", "bddc_tc_selftest", "bddc_wait_selftest"]


def tc_selftest(A, B, C, nr=128, nc=128, K=32):
    """C - A @ B on one 128 x 128 tile through the tensor-core path (host arrays)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    Cc = np.ascontiguousarray(C, dtype=np.float32).copy()
    check(lib().bddc_tc_selftest(_fptr(A), _fptr(B), _fptr(Cc), nr, nc, K), "bddc_tc_selftest")
    return Cc

MLP_FEATURES, MLP_CLASSES, MLP_PARAMS = 11, 8, 9608
MLP_PARAMS_FILE = os.path.join(HERE, "edge_mlp_params.npy")


def _fptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_float))


def _stream_ptr(stream):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(st.cuda_stream)


def mlp_forward(params, X, stream=None):
    """Class probabilities of feature rows X (torch CUDA float32, rows x 10)."""
    import torch
    th = np.ascontiguousarray(params, dtype=np.float32)
    X = X.contiguous()
    P = torch.empty((X.shape[0], MLP_CLASSES), dtype=torch.float32, device="cuda")
    check(lib().bddc_mlp_forward(_fptr(th), _ptr(X), X.shape[0], _ptr(P), _stream_ptr(stream)), "bddc_mlp_forward")
    return P


def mlp_loss_grad(params, X, y, stream=None):
    th = np.ascontiguousarray(params, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    y = y.to(dtype=__import__("torch").int32).contiguous()
    check(lib().bddc_mlp_loss_grad(_fptr(th), _ptr(X.contiguous()), _ptr(y), X.shape[0], _fptr(g), _fptr(loss),
                                   _stream_ptr(stream)), "bddc_mlp_loss_grad")
    return float(loss[0]), g


def mlp_train(params, X, y, epochs, lr=3e-3, stream=None):
    """Adam on the GPU; returns (new params, loss history of epochs + 1 values)."""
    th = np.ascontiguousarray(params, dtype=np.float32).copy()
    hist = np.zeros(epochs + 1, dtype=np.float32)
    y = y.to(dtype=__import__("torch").int32).contiguous()
    check(lib().bddc_mlp_train(_fptr(th), _ptr(X.contiguous()), _ptr(y), X.shape[0], epochs, lr, _fptr(hist),
                               _stream_ptr(stream)), "bddc_mlp_train")
    return th, hist


def load_mlp_params():
    """The trained parameters shipped with the package, or None."""
    if not os.path.exists(MLP_PARAMS_FILE):
        return None
    return np.ascontiguousarray(np.load(MLP_PARAMS_FILE), dtype=np.float32)

(KT_NONE, KT_ENGINE_UPDATE, KT_ENGINE_PANEL, KT_GEMV, KT_FACE, KT_EDGE, KT_ASSEMBLE, KT_TRANSFORM, KT_TRI,
 KT_COARSE, KT_ENGINE_TASKS, KT_APPLY_TASKS) = range(12)


def kernel_timer(kind):
    check(lib().bddc_kernel_timer(kind), "bddc_kernel_timer")


def kernel_timer_read():
    ms, n, fl, by = ct.c_double(), ct.c_longlong(), ct.c_double(), ct.c_double()
    check(lib().bddc_kernel_timer_read(ct.byref(ms), ct.byref(n), ct.byref(fl), ct.byref(by)),
          "bddc_kernel_timer_read")
    return dict(ms=ms.value, launches=n.value, flops=fl.value, bytes=by.value)


def kernel_launches():
    return int(lib().bddc_kernel_launches())


class BDDCError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().bddc_strerror(code).decode()
        detail = lib().bddc_last_error().decode()
        super().__init__(f"{where}: {msg} (code {code})" + (f": {detail}" if detail and detail != msg else ""))
        self.code = code


def check(code, where):
    if code < 0:
        raise BDDCError(code, where)
    return code


def default_opts(**kw):
    o = Opts()
    lib().bddc_default_opts(ct.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    return ct.c_void_p(t.data_ptr())


def resident_arrays(problem, pinned_host=False):
    """Coefficient arrays of `problem` as torch tensors: on the device, or in
    pinned host memory (for end-to-end timing through host pointers)."""
    import torch
    out = {}
    for name, attr in (("nu_elem", "nu_elem"), ("beta_node", "beta_node"), ("f_node", "f_node"),
                       ("g_node", "dirichlet_node")):
        arr = getattr(problem, attr, None)
        if arr is None:
            out[name] = None
            continue
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64).ravel())
        out[name] = t.pin_memory() if pinned_host else t.cuda()
    return out


class Solver:
    """One setup of the adaptive BDDC solver on the current CUDA device.

    problem: a ``workloads.Problem``; host=True passes the coefficient arrays
    from host memory, otherwise they are first placed on the device.
    """

    def __init__(self, problem, host=False, stream=None, arrays=None, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libbddc needs a CUDA GPU")
        L = lib()
        self.torch = torch
        self.problem = problem
        o = default_opts(theta_E=problem.theta_E, restart=problem.restart, rtol=problem.rtol,
                         max_iter=problem.max_iter)
        if problem.theta_F is not None:
            o.theta_F = problem.theta_F
        o.element = ELEM_P1 if getattr(problem, "element", "q1") == "p1" else ELEM_Q1
        self._mlp = None
        for k, v in opts.items():
            if k == "mlp_params":
                self._mlp = None if v is None else np.ascontiguousarray(v, dtype=np.float32)
                o.mlp_params = None if v is None else self._mlp.ctypes.data
                continue
            setattr(o, k, v)
        self.opts = o
        part = Partition()
        self._slabs = []
        for d in range(3):
            arr = (ct.c_int * len(problem.slabs[d]))(*[int(v) for v in problem.slabs[d]])
            self._slabs.append(arr)
            part.nsub[d] = len(problem.slabs[d])
            part.elems_per_slab[d] = ct.cast(arr, ct.POINTER(ct.c_int))
        mesh = Mesh()
        co = Coeffs()
        self._keep = []
        fields = {"nu_elem": problem.nu_elem, "beta_node": problem.beta_node, "f_node": problem.f_node,
                  "g_node": getattr(problem, "dirichlet_node", None)}
        for name, arr in fields.items():
            if arrays is not None:
                t = arrays.get(name)
                setattr(co, name, None if t is None else t.data_ptr())
                continue
            if arr is None:
                setattr(co, name, None)
                continue
            a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
            if host:
                self._keep.append(a)
                setattr(co, name, a.ctypes.data)
            else:
                t = torch.from_numpy(a).cuda()
                self._keep.append(t)
                setattr(co, name, t.data_ptr())
        co.c = float(problem.c)
        co.mem = MEM_HOST if host else MEM_DEVICE
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ct.c_void_p()
        check(L.bddc_setup(ct.byref(mesh), ct.byref(co), ct.byref(part), 0.0, ct.byref(o),
                           ct.c_void_p(self.stream.cuda_stream), ct.byref(ctx)), "bddc_setup")
        self.ctx = ctx
        self._keep = []
        st = Stats()
        L.bddc_get_stats(ctx, ct.byref(st))
        self.n_gamma = st.n_gamma
        self.ndof = st.ndof
        self.nsub = st.nsub
        self.setup_stats = st.as_dict()

    def close(self):
        if getattr(self, "ctx", None):
            lib().bddc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self):
        st = Stats()
        check(lib().bddc_get_stats(self.ctx, ct.byref(st)), "bddc_get_stats")
        return st.as_dict()

    def schur_apply(self, x):
        y = self.torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        xx = x if x.dim() == 1 else x.t().contiguous()
        yy = self.torch.empty_like(xx)
        check(lib().bddc_schur_apply(self.ctx, _ptr(xx), _ptr(yy), nrhs), "bddc_schur_apply")
        return yy if x.dim() == 1 else yy.t().contiguous()

    def apply(self, r):
        nrhs = 1 if r.dim() == 1 else r.shape[1]
        rr = r if r.dim() == 1 else r.t().contiguous()
        zz = self.torch.empty_like(rr)
        check(lib().bddc_apply(self.ctx, _ptr(rr), _ptr(zz), nrhs), "bddc_apply")
        return zz if r.dim() == 1 else zz.t().contiguous()

    def apply_static(self, r):
        """z = M^-1 r through bddc_apply_static (work vectors in the library's
        static device array; nothing is allocated by the library)."""
        nrhs = 1 if r.dim() == 1 else r.shape[1]
        rr = r if r.dim() == 1 else r.t().contiguous()
        zz = self.torch.empty_like(rr)
        check(lib().bddc_apply_static(self.ctx, _ptr(rr), _ptr(zz), nrhs), "bddc_apply_static")
        return zz if r.dim() == 1 else zz.t().contiguous()

    def solve(self, load=None, host=False):
        """Full solve; returns (u, stats).  load: (ndof,) or (ndof, nrhs) array/tensor or None."""
        torch = self.torch
        st = Stats()
        if host:
            nrhs = 1 if load is None or np.ndim(load) == 1 else load.shape[1]
            u = np.zeros((nrhs, self.ndof))
            lp = None
            if load is not None:
                lh = np.ascontiguousarray(np.asarray(load, dtype=np.float64).reshape(self.ndof, nrhs).T)
                lp = lh.ctypes.data
            rc = lib().bddc_gmres_solve(self.ctx, lp, u.ctypes.data, nrhs, MEM_HOST, ct.byref(st))
            check(rc, "bddc_gmres_solve")
            out = st.as_dict()
            out["rc"] = rc
            return (u[0] if nrhs == 1 else u.T), out
        if load is None:
            u = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
            rc = lib().bddc_gmres_solve(self.ctx, None, _ptr(u), 1, MEM_DEVICE, ct.byref(st))
        else:
            lt = load if isinstance(load, torch.Tensor) else torch.from_numpy(np.asarray(load, dtype=np.float64))
            lt = lt.to("cuda", torch.float64)
            nrhs = 1 if lt.dim() == 1 else lt.shape[1]
            lc = lt if lt.dim() == 1 else lt.t().contiguous()
            u = torch.empty_like(lc)
            rc = lib().bddc_gmres_solve(self.ctx, _ptr(lc), _ptr(u), nrhs, MEM_DEVICE, ct.byref(st))
            if nrhs > 1:
                u = u.t().contiguous()
        check(rc, "bddc_gmres_solve")
        out = st.as_dict()
        out["rc"] = rc
        return u, out

    # ---- introspection -------------------------------------------------
    def edge_features(self):
        """(features (n_edges x 10) float32, constraint counts (-1: skipped))."""
        ne = check(lib().bddc_get_entity_count(self.ctx, 1), "bddc_get_entity_count")
        F = np.zeros((max(ne, 1), MLP_FEATURES), dtype=np.float32)
        cnt = np.zeros(max(ne, 1), dtype=np.int32)
        check(lib().bddc_get_edge_features(self.ctx, _fptr(F), cnt.ctypes.data_as(ct.POINTER(ct.c_int))),
              "bddc_get_edge_features")
        return F[:ne], cnt[:ne]

    def numbering(self):
        out = (ct.c_int * self.n_gamma)()
        check(lib().bddc_get_numbering(self.ctx, out), "bddc_get_numbering")
        return np.frombuffer(out, dtype=np.int32).copy()

    def schur(self, s):
        nb = ct.c_int()
        check(lib().bddc_get_schur(self.ctx, s, None, ct.byref(nb)), "bddc_get_schur")
        out = np.zeros((nb.value, nb.value))
        check(lib().bddc_get_schur(self.ctx, s, out.ctypes.data_as(ct.POINTER(ct.c_double)), ct.byref(nb)),
              "bddc_get_schur")
        return out

    def entities(self, kind):
        L = lib()
        cnt = check(L.bddc_get_entity_count(self.ctx, kind), "bddc_get_entity_count")
        out = []
        for i in range(cnt):
            subs = (ct.c_int * 8)()
            n, k, ne = ct.c_int(), ct.c_int(), ct.c_int()
            check(L.bddc_get_entity(self.ctx, kind, i, subs, None, ct.byref(n), ct.byref(k), None, None,
                                    ct.byref(ne)), "bddc_get_entity")
            dofs = (ct.c_int * n.value)()
            Q = np.zeros(max(n.value * k.value, 1))
            lam = np.zeros(max(3 * n.value, 1))
            check(L.bddc_get_entity(self.ctx, kind, i, subs, dofs, ct.byref(n), ct.byref(k),
                                    Q.ctypes.data_as(ct.POINTER(ct.c_double)),
                                    lam.ctypes.data_as(ct.POINTER(ct.c_double)), ct.byref(ne)),
                  "bddc_get_entity")
            out.append(dict(subs=tuple(s for s in subs if s >= 0), dofs=np.array(dofs[:], dtype=int),
                            k=k.value, Q=Q[:n.value * k.value].reshape(k.value, n.value).T,
                            lam=lam[:ne.value].copy()))
        return out


def wait_selftest(limit):
    """bddc_wait_selftest: the bounded wait on a counter nothing increments;
    returns the library's code (BDDC_ETIMEOUT = -5 expected)."""
    return int(lib().bddc_wait_selftest(int(limit)))
