"""ctypes binding of libkl.so (include/kl.h).  Argument marshalling only."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))

KL_GEOM_BOX, KL_GEOM_NURBS = 0, 1
KL_K_EXP, KL_K_GAUSS, KL_K_EXP_SEPARABLE, KL_K_POLY_TEST = 0, 1, 2, 3
KL_P_FP64, KL_P_FP32, KL_P_DF64, KL_P_TC32, KL_P_TC64 = 0, 1, 2, 3, 4
KERNEL_KINDS = {"exp": KL_K_EXP, "gauss": KL_K_GAUSS, "exp_sep": KL_K_EXP_SEPARABLE, "poly": KL_K_POLY_TEST}
STATUS = {0: "KL_OK", 1: "KL_ERR_INVALID_ARG", 2: "KL_ERR_CUDA", 3: "KL_ERR_OOM",
          4: "KL_ERR_NOT_CONVERGED", 5: "KL_ERR_TIMEOUT", 6: "KL_ERR_NUMERIC"}

# every entry point declared in include/kl.h, with (restype, argtypes)
_c_int64 = ctypes.c_int64
_vp = ctypes.c_void_p


class KLGeometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kind", ctypes.c_int), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("deg", ctypes.c_int * 3), ("nctrl", ctypes.c_int * 3),
                ("knots", _vp * 3), ("ctrl", _vp)]


class KLSpace(ctypes.Structure):
    _fields_ = [("deg", ctypes.c_int * 3), ("elems", ctypes.c_int * 3), ("interp_deg", ctypes.c_int * 3),
                ("interp_elems", ctypes.c_int * 3), ("n_interfaces", ctypes.c_int * 3),
                ("interfaces", ctypes.c_void_p * 3)]


class KLKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma", ctypes.c_double), ("L", ctypes.c_double)]


class KLEigOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("block", ctypes.c_int), ("ncv", ctypes.c_int),
                ("maxiter", ctypes.c_int), ("seed", ctypes.c_uint64), ("start_dev", _vp),
                ("tol_low", ctypes.c_double), ("verify", ctypes.c_int), ("precision", ctypes.c_int),
                ("polish_block", ctypes.c_int), ("polish_ncv", ctypes.c_int), ("low_precision", ctypes.c_int),
                ("nstart", ctypes.c_int), ("polish_accurate", ctypes.c_int)]


class KLEigInfo(ctypes.Structure):
    _fields_ = [("applies", ctypes.c_int), ("applies_fp64", ctypes.c_int), ("block_applies", ctypes.c_int),
                ("restarts", ctypes.c_int), ("converged", ctypes.c_int), ("resid", ctypes.c_double * 64),
                ("ms_total", ctypes.c_double), ("ms_fp32_phase", ctypes.c_double),
                ("stage5_calls_fp64", ctypes.c_int), ("stage5_calls_fp32", ctypes.c_int),
                ("stage5_calls_df64", ctypes.c_int),
                ("ms_stage5_fp64", ctypes.c_double), ("ms_stage5_fp32", ctypes.c_double),
                ("ms_stage5_df64", ctypes.c_double),
                ("pairs_fp64", ctypes.c_double), ("pairs_fp32", ctypes.c_double), ("pairs_df64", ctypes.c_double),
                ("applies_df64", ctypes.c_int),
                ("stage5_calls_tc64", ctypes.c_int), ("ms_stage5_tc64", ctypes.c_double),
                ("pairs_tc64", ctypes.c_double), ("applies_tc64", ctypes.c_int),
                ("stage5_calls_tc32", ctypes.c_int), ("ms_stage5_tc32", ctypes.c_double),
                ("pairs_tc32", ctypes.c_double), ("applies_tc32", ctypes.c_int)]


class KLBatchInfo(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("cols_per_split", ctypes.c_int), ("ms_total", ctypes.c_double),
                ("ms_stage5", ctypes.c_double), ("requests", ctypes.c_longlong)]


SIGNATURES = {
    "kl_create": (ctypes.c_int, [ctypes.POINTER(KLGeometry), ctypes.POINTER(KLSpace), ctypes.POINTER(KLKernel),
                                 ctypes.POINTER(_vp)]),
    "kl_size": (ctypes.c_int, [_vp, ctypes.POINTER(_c_int64), ctypes.POINTER(_c_int64)]),
    "kl_dims": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "kl_apply": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _c_int64, _vp]),
    "kl_apply_prec": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _c_int64, _vp]),
    "kl_forward": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, _c_int64, ctypes.c_int, _vp]),
    "kl_covmv": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _c_int64, _vp, _c_int64, ctypes.c_int, _vp]),
    "kl_covmv_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _c_int64, _vp, _c_int64, ctypes.c_int, _vp]),
    "kl_backward": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, _c_int64, ctypes.c_int, _vp]),
    "kl_get_factor": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "kl_get_points": (ctypes.c_int, [_vp, _vp, _vp]),
    "kl_eigs": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(KLEigOpts), _vp, _vp, _c_int64,
                               ctypes.POINTER(KLEigInfo), _vp]),
    "kl_to_bspline": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _c_int64, _vp]),
    "kl_apply_batched": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp),
                                        ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_c_int64),
                                        _vp]),
    "kl_eigs_batched": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(KLEigOpts), _vp, ctypes.POINTER(_vp), ctypes.POINTER(_c_int64),
                                       ctypes.POINTER(KLEigInfo), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(KLBatchInfo)]),
    "kl_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.POINTER(_vp)]),
    "kl_mlp_num_params": (ctypes.c_int, [_vp, ctypes.POINTER(_c_int64)]),
    "kl_mlp_params": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "kl_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "kl_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    "kl_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _vp, _vp]),
    "kl_mlp_destroy": (None, [_vp]),
    "kl_prolong": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "kl_direction_factors": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            _vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _vp,
                                            _vp, _vp, _vp]),
    "kl_mapped_points": (ctypes.c_int, [ctypes.POINTER(KLGeometry), ctypes.POINTER(KLSpace),
                                        ctypes.POINTER(_c_int64), _vp, _vp]),
    "kl_prolongation_factor": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), _vp]),
    "kl_wait_selftest": (ctypes.c_int, [ctypes.c_double, _vp]),
    "kl_df2_selftest": (ctypes.c_int, [_c_int64, ctypes.c_uint64, _vp, _vp]),
    "kl_pipe_rates": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "kl_set_sym_slot_limit": (ctypes.c_int, [_c_int64]),
    "kl_set_tc_symmetric": (ctypes.c_int, [ctypes.c_int]),
    "kl_kernel_launches": (ctypes.c_uint64, []),
    "kl_last_error": (ctypes.c_char_p, []),
    "kl_destroy": (None, [_vp]),
}

_LIB = None


class KLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def library_path():
    return os.path.join(HERE, "libkl.so")


def load(path=None):
    """Load libkl.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError("libkl.so not found at %s; build it with `python -m paper_2011_13861_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_symbols(path=None):
    """Names from SIGNATURES that the shared object exports (no CUDA call is made)."""
    lib = ctypes.CDLL(path or library_path())
    return [n for n in SIGNATURES if hasattr(lib, n)]


def kernel_launches():
    """Kernels launched by libkl since it was loaded."""
    return int(load().kl_kernel_launches())


def _info_dict(info, k, st):
    return {"applies": info.applies, "applies_fp64": info.applies_fp64, "block_applies": info.block_applies,
            "restarts": info.restarts, "converged": info.converged, "resid": list(info.resid[:k]),
            "ms_total": info.ms_total, "ms_fp32_phase": info.ms_fp32_phase, "status": st,
            "stage5_calls_fp64": info.stage5_calls_fp64, "stage5_calls_fp32": info.stage5_calls_fp32,
            "ms_stage5_fp64": info.ms_stage5_fp64, "ms_stage5_fp32": info.ms_stage5_fp32,
            "pairs_fp64": info.pairs_fp64, "pairs_fp32": info.pairs_fp32,
            "stage5_calls_df64": info.stage5_calls_df64, "ms_stage5_df64": info.ms_stage5_df64,
            "pairs_df64": info.pairs_df64, "applies_df64": info.applies_df64,
            "stage5_calls_tc64": info.stage5_calls_tc64, "ms_stage5_tc64": info.ms_stage5_tc64,
            "pairs_tc64": info.pairs_tc64, "applies_tc64": info.applies_tc64,
            "stage5_calls_tc32": info.stage5_calls_tc32, "ms_stage5_tc32": info.ms_stage5_tc32,
            "pairs_tc32": info.pairs_tc32, "applies_tc32": info.applies_tc32}


def _check(status):
    if status != 0:
        raise KLError(status, load().kl_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _per_dir(v, dim, default=0):
    if v is None:
        return [default] * 3
    if isinstance(v, (int, float)):
        v = [v] * dim
    v = list(v) + [default] * (3 - len(v))
    return v[:3]


def _geometry_and_space(dim, p, ne, pt=None, net=None, lo=None, hi=None, nurbs=None, interfaces=None):
    """kl_geometry and kl_space structs for the arguments of KLProblem, and the host arrays
    they point into (keep them alive while the structs are used)."""
    g = KLGeometry(dim, KL_GEOM_BOX, (ctypes.c_double * 3)(*_per_dir(lo, dim, 0.0)),
                   (ctypes.c_double * 3)(*_per_dir(hi, dim, 1.0)))
    keep = []
    if nurbs is not None:
        import numpy as np
        # nurbs: dict(deg=[...], knots=[...], ctrl=array (n_d, ..., n_1, dim), weights=array (n_d, ..., n_1))
        g.kind = KL_GEOM_NURBS
        deg = [int(x) for x in nurbs["deg"]]
        knots = [np.ascontiguousarray(t, dtype=np.float64) for t in nurbs["knots"]]
        ctrl = np.asarray(nurbs["ctrl"], dtype=np.float64)
        wts = np.asarray(nurbs["weights"], dtype=np.float64)
        rec = np.zeros(wts.shape + (4,))
        rec[..., :ctrl.shape[-1]] = ctrl
        rec[..., 3] = wts
        rec = np.ascontiguousarray(rec.reshape(-1, 4))
        keep += knots + [rec]
        for k in range(dim):
            g.deg[k] = deg[k]
            g.nctrl[k] = len(knots[k]) - deg[k] - 1
            g.knots[k] = knots[k].ctypes.data
        g.ctrl = rec.ctypes.data
    sp = KLSpace((ctypes.c_int * 3)(*_per_dir(p, dim)), (ctypes.c_int * 3)(*_per_dir(ne, dim)),
                 (ctypes.c_int * 3)(*_per_dir(pt, dim)), (ctypes.c_int * 3)(*_per_dir(net, dim)))
    if interfaces is not None:
        # interfaces: per direction a sequence of patch-interface parameters (Sec. 3.6)
        for k in range(dim):
            vals = [float(x) for x in interfaces[k]] if k < len(interfaces) else []
            if vals:
                arr = (ctypes.c_double * len(vals))(*vals)
                keep.append(arr)
                sp.n_interfaces[k] = len(vals)
                sp.interfaces[k] = ctypes.cast(arr, ctypes.c_void_p).value
    return g, sp, keep


class KLProblem:
    """One discretised KL problem on the GPU (a kl_handle).

    dim, p, ne: spatial dimension, trial degree and element count per direction;
    kernel: 'exp' | 'gauss' | 'exp_sep' | 'poly';  pt, net: interpolation space (default = trial);
    lo, hi: box map; nurbs: NURBS map; interfaces: per direction, patch-interface parameters of a
    multipatch domain (C^0 trial and C^{-1} interpolation space there).  All vectors are float64 CUDA tensors of shape (N,) or (N, nvec)
    (column-major blocks are handled by passing the transposed storage, see _block).
    """

    def __init__(self, dim, p, ne, kernel="exp", sigma=1.0, L=1.0, pt=None, net=None, lo=None, hi=None,
                 nurbs=None, interfaces=None):
        lib = load()
        g, sp, keep = _geometry_and_space(dim, p, ne, pt, net, lo, hi, nurbs, interfaces)
        kk = KLKernel(KERNEL_KINDS[kernel] if isinstance(kernel, str) else int(kernel), float(sigma), float(L))
        h = ctypes.c_void_p()
        _check(lib.kl_create(ctypes.byref(g), ctypes.byref(sp), ctypes.byref(kk), ctypes.byref(h)))
        self._h = h
        self.dim = dim
        N, Nt = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.kl_size(h, ctypes.byref(N), ctypes.byref(Nt)))
        self.N, self.Nt = N.value, Nt.value
        n3, nt3 = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
        _check(lib.kl_dims(h, n3, nt3))
        self.n, self.nt = list(n3)[:dim], list(nt3)[:dim]

    def close(self):
        if getattr(self, "_h", None):
            load().kl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers: a block of nvec column vectors of length n is stored as a (nvec, n)
    #    row-major torch tensor, i.e. column-major (n x nvec) with leading dimension n.
    @staticmethod
    def _block(x, n):
        import torch
        if x.dtype != torch.float64 or not x.is_cuda:
            raise TypeError("expected a float64 CUDA tensor")
        if x.dim() == 1:
            x = x.reshape(1, -1)
        if x.shape[-1] != n or not x.is_contiguous():
            raise ValueError("expected a contiguous (nvec, %d) tensor" % n)
        return x

    def apply(self, v, precision=KL_P_FP64, out=None, stream=None):
        """y = A~' v (all nine stages of Algorithm 1).  v: (N,) or (nvec, N)."""
        import torch
        vb = self._block(v, self.N)
        y = out if out is not None else torch.empty_like(vb)
        _check(load().kl_apply_prec(self._h, int(precision), _ptr(vb), _ptr(y), vb.shape[0], self.N, _stream(stream)))
        return y.reshape(v.shape)

    def forward(self, v, stream=None):
        import torch
        vb = self._block(v, self.N)
        u = torch.empty((vb.shape[0], self.Nt), dtype=torch.float64, device=vb.device)
        _check(load().kl_forward(self._h, _ptr(vb), self.N, _ptr(u), self.Nt, vb.shape[0], _stream(stream)))
        return u if v.dim() == 2 else u[0]

    def covmv(self, u, precision=KL_P_FP64, stream=None):
        import torch
        ub = self._block(u, self.Nt)
        z = torch.empty_like(ub)
        _check(load().kl_covmv(self._h, int(precision), _ptr(ub), self.Nt, _ptr(z), self.Nt, ub.shape[0],
                               _stream(stream)))
        return z.reshape(u.shape)

    def covmv_noalloc(self, u, out, stream=None):
        """Stage 5 into the caller's `out` through kl_covmv_noalloc (no device allocation)."""
        ub = self._block(u, self.Nt)
        zb = self._block(out, self.Nt)
        _check(load().kl_covmv_noalloc(self._h, KL_P_FP64, _ptr(ub), self.Nt, _ptr(zb), self.Nt, ub.shape[0],
                                       _stream(stream)))
        return out

    def backward(self, z, stream=None):
        import torch
        zb = self._block(z, self.Nt)
        y = torch.empty((zb.shape[0], self.N), dtype=torch.float64, device=zb.device)
        _check(load().kl_backward(self._h, _ptr(zb), self.Nt, _ptr(y), self.N, zb.shape[0], _stream(stream)))
        return y if z.dim() == 2 else y[0]

    def to_bspline(self, vp, stream=None):
        import torch
        vb = self._block(vp, self.N)
        out = torch.empty_like(vb)
        _check(load().kl_to_bspline(self._h, _ptr(vb), _ptr(out), vb.shape[0], self.N, _stream(stream)))
        return out.reshape(vp.shape)

    def factor(self, k):
        """C_k = B~_k^{-T} M_k L_k^{-T} of direction k (n~_k x n_k numpy array)."""
        import numpy as np
        C = np.zeros((self.nt[k], self.n[k]))
        _check(load().kl_get_factor(self._h, k, C.ctypes.data_as(ctypes.c_void_p)))
        return C

    def points(self):
        import numpy as np
        X = np.zeros((self.Nt, 3))
        J = np.zeros(self.Nt)
        _check(load().kl_get_points(self._h, X.ctypes.data_as(ctypes.c_void_p), J.ctypes.data_as(ctypes.c_void_p)))
        return X[:, :self.dim].copy(), J

    def eigs(self, k, tol=1e-8, method=0, block=1, ncv=0, maxiter=0, seed=1, start=None, tol_low=0.0,
             verify=True, want_vectors=True, stream=None, raise_on_nonconv=True, precision=KL_P_FP64,
             polish_block=0, polish_ncv=0, low_precision=KL_P_FP32, polish_accurate=False):
        """The k largest eigenpairs (descending).  Returns (evals numpy, evecs (k, N) tensor or None, info dict)."""
        import numpy as np
        import torch
        # start: (nstart, N) float64 CUDA tensor; more rows than `block` are compressed by
        # Rayleigh-Ritz to the block leading Ritz vectors (kl_eig_opts.nstart)
        nstart = int(start.shape[0]) if (start is not None and start.dim() == 2) else 0
        if start is not None and max(nstart, 1) < int(block):
            raise ValueError("start must hold at least `block` vectors")
        if start is not None and (not start.is_contiguous() or start.dtype != torch.float64 or
                                  start.numel() != max(nstart, 1) * self.N):
            raise ValueError("start must be a contiguous float64 (nstart, N) tensor")
        opts = KLEigOpts(int(method), int(block), int(ncv), int(maxiter), int(seed) & (2 ** 64 - 1),
                         _ptr(start) if start is not None else None, float(tol_low), 1 if verify else 0,
                         int(precision), int(polish_block), int(polish_ncv), int(low_precision),
                         nstart if nstart > int(block) else 0, 1 if polish_accurate else 0)
        ev = np.zeros(k)
        vecs = None
        dev = torch.device("cuda", torch.cuda.current_device())
        if want_vectors:
            vecs = torch.empty((k, self.N), dtype=torch.float64, device=dev)
        info = KLEigInfo()
        st = load().kl_eigs(self._h, int(k), float(tol), ctypes.byref(opts), ev.ctypes.data_as(ctypes.c_void_p),
                            _ptr(vecs), self.N, ctypes.byref(info), _stream(stream))
        if st != 0 and (raise_on_nonconv or st != 4):
            _check(st)
        return ev, vecs, _info_dict(info, k, st)


def apply_batched(problems, vs, precision=KL_P_DF64, stream=None):
    """y_i = A~'_i v_i for every problem with one batched stage-5 launch (kl_apply_batched).
    vs: float64 CUDA tensors of shape (nvec_i, N_i) (or (N_i,)); returns the outputs alike."""
    import torch
    n = len(problems)
    hs = (_vp * n)(*[p._h.value for p in problems])
    blocks = [KLProblem._block(v, p.N) for v, p in zip(vs, problems)]
    outs = [torch.empty_like(b) for b in blocks]
    vp = (_vp * n)(*[_ptr(b) for b in blocks])
    yp = (_vp * n)(*[_ptr(o) for o in outs])
    nv = (ctypes.c_int * n)(*[b.shape[0] for b in blocks])
    ld = (_c_int64 * n)(*[p.N for p in problems])
    _check(load().kl_apply_batched(hs, n, int(precision), vp, yp, nv, ld, _stream(stream)))
    return [o.reshape(v.shape) for o, v in zip(outs, vs)]


def eigs_batched(problems, k, tol=1e-8, method=0, block=4, ncv=0, maxiter=0, seed=1, tol_low=0.0, verify=True,
                 want_vectors=True, precision=KL_P_DF64, polish_block=0, polish_ncv=0, low_precision=KL_P_FP32,
                 polish_accurate=False):
    """kl_eigs_batched: the k largest eigenpairs of every problem, solved together.  Returns
    (evals (count, k) numpy, list of (k, N_i) tensors or None, list of info dicts, statuses, batch info)."""
    import numpy as np
    import torch
    n = len(problems)
    opts = KLEigOpts(int(method), int(block), int(ncv), int(maxiter), int(seed) & (2 ** 64 - 1), None,
                     float(tol_low), 1 if verify else 0, int(precision), int(polish_block), int(polish_ncv),
                     int(low_precision), 0, 1 if polish_accurate else 0)
    ev = np.zeros((n, k))
    dev = torch.device("cuda", torch.cuda.current_device())
    vecs = [torch.empty((k, p.N), dtype=torch.float64, device=dev) for p in problems] if want_vectors else None
    hs = (_vp * n)(*[p._h.value for p in problems])
    vp = (_vp * n)(*[_ptr(v) for v in vecs]) if vecs else None
    ld = (_c_int64 * n)(*[p.N for p in problems])
    infos = (KLEigInfo * n)()
    sts = (ctypes.c_int * n)()
    bi = KLBatchInfo()
    st = load().kl_eigs_batched(hs, n, int(k), float(tol), ctypes.byref(opts), ev.ctypes.data_as(ctypes.c_void_p),
                                vp, ld, infos, sts, ctypes.byref(bi))
    if st != 0 and st != 4:
        _check(st)
    return (ev, vecs, [_info_dict(infos[i], k, sts[i]) for i in range(n)], list(sts),
            {"rounds": bi.rounds, "cols_per_split": bi.cols_per_split, "ms_total": bi.ms_total,
             "ms_stage5": bi.ms_stage5, "requests": bi.requests})


class MLP:
    """The warm-start network (kl_mlp_*): n_in -> depth x width (tanh) -> n_out, bfloat16 weights and
    layer inputs, float32 sums.  Inputs, targets and outputs are float32 CUDA tensors."""

    def __init__(self, n_in, width, depth, n_out, seed=0):
        h = ctypes.c_void_p()
        _check(load().kl_mlp_create(int(n_in), int(width), int(depth), int(n_out), int(seed) & (2 ** 64 - 1),
                                    ctypes.byref(h)))
        self._h = h
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out
        n = _c_int64()
        _check(load().kl_mlp_num_params(h, ctypes.byref(n)))
        self.nparam = n.value

    def layer_shapes(self):
        dims = [self.n_in] + [self.width] * self.depth + [self.n_out]
        return list(zip(dims[:-1], dims[1:]))

    def get_params(self):
        """Float32 parameters as lists (Ws, bs) of numpy arrays (W: in x out)."""
        import numpy as np
        flat = np.zeros(self.nparam, dtype=np.float32)
        _check(load().kl_mlp_params(self._h, flat.ctypes.data_as(ctypes.c_void_p), 0))
        return self._split(flat)

    def set_params(self, Ws, bs):
        import numpy as np
        flat = np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32)])
                               for W, b in zip(Ws, bs)])
        _check(load().kl_mlp_params(self._h, flat.ctypes.data_as(ctypes.c_void_p), 1))

    def _split(self, flat):
        Ws, bs, o = [], [], 0
        for a, b in self.layer_shapes():
            Ws.append(flat[o:o + a * b].reshape(a, b))
            o += a * b
            bs.append(flat[o:o + b])
            o += b
        return Ws, bs

    def forward(self, x, stream=None):
        import torch
        out = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        _check(load().kl_mlp_forward(self._h, _ptr(x), int(x.shape[0]), _ptr(out), _stream(stream)))
        return out

    def loss_grad(self, x, tgt, k, n, stream=None):
        """Per-sample losses (tensor) and the gradient of the batch-mean loss as (dWs, dbs)."""
        import numpy as np
        import torch
        loss = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        g = np.zeros(self.nparam, dtype=np.float32)
        _check(load().kl_mlp_loss_grad(self._h, _ptr(x), _ptr(tgt), int(x.shape[0]), int(k), int(n), _ptr(loss),
                                       g.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return loss, self._split(g)

    def train(self, x, tgt, k, n, epochs, batch, lr, seed=0, stream=None):
        """Adam epochs over the rows of x / tgt; returns the per-epoch mean losses."""
        import numpy as np
        hist = np.zeros(max(int(epochs), 1))
        _check(load().kl_mlp_train(self._h, _ptr(x), _ptr(tgt), int(x.shape[0]), int(k), int(n), int(epochs),
                                   int(batch), float(lr), int(seed) & (2 ** 64 - 1),
                                   hist.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return hist[:int(epochs)]

    def close(self):
        if getattr(self, "_h", None):
            load().kl_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prolong(coarse, fine, v, stream=None):
    """Standard-form vectors of `coarse`'s trial space carried exactly to `fine`'s (kl_prolong):
    v (nvec, N_c) float64 CUDA tensor -> (nvec, N_f)."""
    import torch
    vb = KLProblem._block(v, coarse.N)
    out = torch.empty((vb.shape[0], fine.N), dtype=torch.float64, device=vb.device)
    _check(load().kl_prolong(coarse._h, fine._h, _ptr(vb), _ptr(out), int(vb.shape[0]), _stream(stream)))
    return out if v.dim() > 1 else out.reshape(-1)


def direction_factors(deg, elems, interp_deg=0, interp_elems=0, interfaces=()):
    """kl_direction_factors (host only, no GPU): the set-up of one direction as kl_create builds
    it -- Greville abscissae and sides of the interpolation space, the Cholesky factor L_k of
    Z_k, and the folded factor C_k = B~_k^-T M_k L_k^-T -- as NumPy arrays."""
    import numpy as np
    lib = load()
    itf = np.ascontiguousarray(np.asarray(interfaces, dtype=np.float64).reshape(-1))
    itf_p = ctypes.c_void_p(itf.ctypes.data) if itf.size else None
    n, nt = ctypes.c_int(0), ctypes.c_int(0)
    args = (int(deg), int(elems), int(interp_deg), int(interp_elems), int(itf.size), itf_p)
    _check(lib.kl_direction_factors(*args, ctypes.byref(n), ctypes.byref(nt), None, None, None, None))
    xi = np.zeros(nt.value)
    side = np.zeros(nt.value, dtype=np.int32)
    L = np.zeros((n.value, n.value))
    C = np.zeros((nt.value, n.value))
    _check(lib.kl_direction_factors(*args, ctypes.byref(n), ctypes.byref(nt),
                                    ctypes.c_void_p(xi.ctypes.data), ctypes.c_void_p(side.ctypes.data),
                                    ctypes.c_void_p(L.ctypes.data), ctypes.c_void_p(C.ctypes.data)))
    return {"n": n.value, "nt": nt.value, "greville": xi, "side": side, "L": L, "C": C}


def prolongation_factor(deg, elems_coarse, elems_fine):
    """kl_prolongation_factor (host only, no GPU): Q_k = L_f^T P_k L_c^{-T} of one direction,
    (n_fine x n_coarse), the factor kl_prolong applies."""
    import numpy as np
    lib = load()
    nc, nf = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.kl_prolongation_factor(int(deg), int(elems_coarse), int(elems_fine), ctypes.byref(nc),
                                      ctypes.byref(nf), None))
    Q = np.zeros((nf.value, nc.value))
    _check(lib.kl_prolongation_factor(int(deg), int(elems_coarse), int(elems_fine), ctypes.byref(nc),
                                      ctypes.byref(nf), ctypes.c_void_p(Q.ctypes.data)))
    return Q


def mapped_points(dim, p, ne, pt=None, net=None, lo=None, hi=None, nurbs=None, interfaces=None):
    """kl_mapped_points (host only, no GPU): the mapped Greville grid X (Ntilde x 3, direction 1
    fastest) and J = sqrt(det DF) that KLProblem(dim, p, ne, ...) would upload."""
    import numpy as np
    lib = load()
    g, sp, keep = _geometry_and_space(dim, p, ne, pt, net, lo, hi, nurbs, interfaces)
    Nt = ctypes.c_int64(0)
    _check(lib.kl_mapped_points(ctypes.byref(g), ctypes.byref(sp), ctypes.byref(Nt), None, None))
    X = np.zeros((Nt.value, 3))
    J = np.zeros(Nt.value)
    _check(lib.kl_mapped_points(ctypes.byref(g), ctypes.byref(sp), ctypes.byref(Nt),
                                ctypes.c_void_p(X.ctypes.data), ctypes.c_void_p(J.ctypes.data)))
    del keep
    return X, J


def df2_selftest(n, seed=1, stream=None):
    """kl_df2_selftest: float words in which the packed-pair double-float kernel values, slices
    and sums differ from the scalar ones over n random column pairs (0 = bit-identical)."""
    out = _c_int64(0)
    _check(load().kl_df2_selftest(int(n), int(seed) & (2 ** 64 - 1), ctypes.byref(out), _stream(stream)))
    return out.value


def wait_selftest(seconds=0.05, stream=None):
    """kl_wait_selftest: status code of a bounded wait that nothing completes (KL_ERR_TIMEOUT
    expected) and the library's message."""
    st = load().kl_wait_selftest(float(seconds), _stream(stream))
    return st, load().kl_last_error().decode()


def pipe_rates(stream=None):
    """kl_pipe_rates: measured operations per second of the float64 FMA, float32 FMA, MUFU ex2
    and MUFU rsqrt pipes of the current GPU, the packed float32 pair FMA (FMAs per second), and
    the SM clock each launch ran at (dict)."""
    out = (ctypes.c_double * 10)()
    _check(load().kl_pipe_rates(ctypes.cast(out, ctypes.c_void_p), 10, _stream(stream)))
    return {"dfma_per_s": out[0], "ffma_per_s": out[1], "ex2_per_s": out[2], "rsqrt_per_s": out[3],
            "ffma2_per_s": out[8],
            "sm_mhz": {"dfma": out[4], "ffma": out[5], "ex2": out[6], "rsqrt": out[7], "ffma2": out[9]}}


def set_sym_slot_limit(nbytes):
    """kl_set_sym_slot_limit: largest partial-slot workspace (bytes) of the one-launch symmetric
    stage-5 schedule; above it the banded schedule with a fixed slot count runs."""
    _check(load().kl_set_sym_slot_limit(int(nbytes)))


def set_tc_symmetric(enable):
    """kl_set_tc_symmetric: the tensor-core float64-class stage 5 evaluates each kernel value once
    for both pairs (True) or all Ntilde^2 values (False, the default)."""
    _check(load().kl_set_tc_symmetric(1 if enable else 0))
