"""Thin ctypes binding of libregnk.so (the C ABI declared in include/reg.h).

Argument marshalling only: every step of the registration path runs in the
library's CUDA kernels. Field arguments are torch tensors on the CUDA device
(float32, contiguous); the binding passes their device pointers and the
current torch stream. There is no CPU fallback: if the library is missing or
the CUDA runtime is unavailable, the calls raise.
"""

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libregnk.so")

REG_OK, REG_EINVAL, REG_ENOMEM, REG_ECUDA, REG_ESTATE = 0, 1, 2, 3, 4
REG_ENOTCONV, REG_ELINESEARCH, REG_ENEGCURV, REG_ENONFINITE, REG_ETIMEOUT = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "REG_OK", 1: "REG_EINVAL", 2: "REG_ENOMEM", 3: "REG_ECUDA", 4: "REG_ESTATE",
                5: "REG_ENOTCONV", 6: "REG_ELINESEARCH", 7: "REG_ENEGCURV",
                8: "REG_ENONFINITE", 9: "REG_ETIMEOUT"}
REG_H1, REG_H2, REG_H3 = 1, 2, 3
REG_INTERP_SPLINE, REG_INTERP_LAGRANGE = 0, 1
REG_PC_REG, REG_PC_2L = 0, 1
REG_PCSOLVER_CHEB, REG_PCSOLVER_PCG = 0, 1
REG_HESSIAN_GN, REG_HESSIAN_FULL = 0, 1
REG_PRECISION_FP64, REG_PRECISION_FP32 = 0, 1
REG_SPEC_GRAD, REG_SPEC_DIV, REG_SPEC_REG, REG_SPEC_REGPOW = 0, 1, 2, 3
REG_SPEC_LOWPASS, REG_SPEC_HIGHPASS, REG_SPEC_PREFILTER, REG_SPEC_LERAY = 4, 5, 6, 7
REG_SPEC_REGOP, REG_SPEC_K = 8, 9
KERNEL_CLASSES = ["fft_rows", "fft_cols", "prefilter", "departure", "gather",
                  "adjoint_step", "incstate_step", "reduce", "vector", "matvec"]


class RegError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class reg_grid(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int)]


class reg_options(ctypes.Structure):
    _fields_ = [("reg_norm", ctypes.c_int), ("interp", ctypes.c_int), ("precond", ctypes.c_int),
                ("pc_solver", ctypes.c_int), ("cheb_iters", ctypes.c_int),
                ("pc_eps", ctypes.c_double), ("gabs", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("max_pcg", ctypes.c_int),
                ("lanczos_steps", ctypes.c_int), ("emax_safety", ctypes.c_double),
                ("lanczos_seed", ctypes.c_ulonglong), ("max_backtracks", ctypes.c_int),
                ("armijo_c1", ctypes.c_double), ("persistent_matvec", ctypes.c_int),
                ("inject_barrier_timeout", ctypes.c_int), ("programmatic_launch", ctypes.c_int),
                ("fused_transport", ctypes.c_int), ("coarse_nt", ctypes.c_int),
                ("coarse_interp", ctypes.c_int), ("step_tile", ctypes.c_int), ("incompressible", ctypes.c_int),
                ("hessian", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("flow_matvec", ctypes.c_int),
                ("beta_w", ctypes.c_double), ("graph_pdl", ctypes.c_int)]


class reg_info(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int),
                ("matvecs", ctypes.c_int), ("coarse_matvecs", ctypes.c_int),
                ("line_search_steps", ctypes.c_int), ("J0", ctypes.c_double),
                ("J", ctypes.c_double), ("gnorm_rel", ctypes.c_double),
                ("gnorm_inf", ctypes.c_double), ("gref_inf", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGNATURES = {
    "reg_default_options": [ctypes.POINTER(reg_options)],
    "reg_create": [reg_grid, _I, _D, ctypes.POINTER(reg_options), ctypes.POINTER(_P)],
    "reg_destroy": [_P],
    "reg_set_stream": [_P, _P],
    "reg_set_images": [_P, _P, _P],
    "reg_set_beta": [_P, _D],
    "reg_transport": [_P, _P, _P, _P],
    "reg_departure_points": [_P, _P, _P, _P],
    "reg_transport_rk2a": [_P, _P, _P, _P, _I],
    "reg_deformation_map": [_P, _P, _P, _P],
    "reg_adjoint_rk2a": [_P, _P, _P, _P, _I],
    "reg_interpolate": [_P, _P, _P, _P],
    "reg_spectral": [_P, _I, _D, _P, _P],
    "reg_restrict": [_P, _P, _P],
    "reg_prolong": [_P, _P, _P],
    "reg_objective_gradient": [_P, _P, ctypes.POINTER(_D), _P],
    "reg_objective": [_P, _P, ctypes.POINTER(_D)],
    "reg_hessian_matvec": [_P, _P, _P, _P],
    "reg_precond_apply": [_P, _P, _P],
    "reg_kkt_solve": [_P, _P, _P, _D, _I, _P, ctypes.POINTER(reg_info)],
    "reg_eigen_bounds": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "reg_solve": [_P, _P, _D, ctypes.POINTER(reg_info)],
    "reg_dot": [_P, _P, _P, ctypes.c_longlong, ctypes.POINTER(_D)],
    "reg_last_error": [_P],
    "reg_profile_enable": [_P, _I],
    "reg_profile_read": [_P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                         ctypes.POINTER(_D)],
    "reg_launch_count": [],
    "reg_step_tiles": [_P, ctypes.POINTER(_I)],
    "reg_interpolate_static": [_I, _I, _P, _P, _P, _P],
    "reg_batch_create": [ctypes.POINTER(reg_grid), _I, _I, ctypes.POINTER(_D),
                         ctypes.POINTER(reg_options), ctypes.POINTER(_P)],
    "reg_batch_destroy": [_P],
    "reg_batch_set_images": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "reg_batch_set_beta": [_P, ctypes.POINTER(_D)],
    "reg_batch_solve": [_P, ctypes.POINTER(_P), _D, _I, ctypes.POINTER(reg_info)],
    "reg_batch_hessian_matvec": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "reg_batch_last_error": [_P],
    "reg3_create": [_I, _I, _I, _I, _D, ctypes.POINTER(reg_options), ctypes.POINTER(_P)],
    "reg3_destroy": [_P],
    "reg3_set_stream": [_P, _P],
    "reg3_set_images": [_P, _P, _P],
    "reg3_transport": [_P, _P, _P, _P],
    "reg3_spectral": [_P, _I, _D, _P, _P],
    "reg3_deformation_map": [_P, _P, _P, _P],
    "reg3_precond_apply": [_P, _P, _P, _P],
    "reg3_eigen_bounds": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "reg3_objective_gradient": [_P, _P, ctypes.POINTER(_D), _P],
    "reg3_hessian_matvec": [_P, _P, _P, _P],
    "reg3_solve": [_P, _P, _D, ctypes.POINTER(reg_info)],
    "reg3_last_error": [_P],
    "reg_lockstep_create": [ctypes.POINTER(reg_grid), _I, _I, ctypes.POINTER(_D),
                            ctypes.POINTER(reg_options), ctypes.POINTER(_P)],
    "reg_lockstep_destroy": [_P],
    "reg_lockstep_set_stream": [_P, _P],
    "reg_lockstep_set_images": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "reg_lockstep_objective_gradient": [_P, ctypes.POINTER(_P), ctypes.POINTER(_D),
                                        ctypes.POINTER(_P)],
    "reg_lockstep_hessian_matvec": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                    ctypes.POINTER(_P)],
    "reg_lockstep_solve": [_P, ctypes.POINTER(_P), _D, ctypes.POINTER(reg_info)],
    "reg_lockstep_matvec_time": [_P, _I, ctypes.POINTER(_D)],
    "reg_lockstep_info": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_I),
                          ctypes.POINTER(_I)],
    "reg_lockstep_last_error": [_P],
    "reg_unet_param_count": [],
    "reg_unet_create": [_I, _I, ctypes.POINTER(_P)],
    "reg_unet_destroy": [_P],
    "reg_unet_size": [_P],
    "reg_unet_set_stream": [_P, _P],
    "reg_unet_set_params": [_P, _P],
    "reg_unet_get_params": [_P, _P],
    "reg_unet_forward": [_P, _I, _P, _P, _P, _P],
    "reg_unet_gradients": [_P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(_D)],
    "reg_unet_train_step": [_P, _I, _P, _P, _P, _P, ctypes.c_float, ctypes.POINTER(_D)],
    "reg_unet_set_conv_path": [_P, _I],
    "reg_unet_last_error": [_P],
    "reg_warm_start": [_P, _P, _P, ctypes.POINTER(_I)],
}

_lib = None


def load(path=LIB_PATH):
    """Load libregnk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1604_02153_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = {"reg_last_error": ctypes.c_char_p, "reg_batch_last_error": ctypes.c_char_p,
                      "reg_lockstep_last_error": ctypes.c_char_p,
                      "reg3_last_error": ctypes.c_char_p,
                      "reg_unet_last_error": ctypes.c_char_p, "reg_launch_count": ctypes.c_longlong,
                      "reg_unet_param_count": ctypes.c_longlong}.get(name, ctypes.c_int)
    _lib = lib
    return lib


def _ptr(t, numel=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def default_options(**overrides):
    o = reg_options()
    load().reg_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Registration:
    """One registration problem: a reg_ctx handle plus argument checking.

    Methods carry the C names without the ``reg_`` prefix; each passes the
    tensors' device pointers and the current torch CUDA stream.
    """

    def __init__(self, n1, n2, nt, beta, **options):
        import torch
        self.lib = load()
        self.n1, self.n2, self.nt = int(n1), int(n2), int(nt)
        self.N = self.n1 * self.n2
        self.options = default_options(**options)
        self.device = torch.cuda.current_device()
        h = ctypes.c_void_p()
        s = self.lib.reg_create(reg_grid(self.n1, self.n2), self.nt, float(beta),
                                ctypes.byref(self.options), ctypes.byref(h))
        if s != REG_OK:
            raise RegError(s, "reg_create failed")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.reg_destroy(h)
            self.h = None

    def close(self):
        self.__del__()

    def _call(self, name, *args):
        import torch
        self.lib.reg_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        s = getattr(self.lib, name)(self.h, *args)
        if s not in (REG_OK,):
            raise RegError(s, self.lib.reg_last_error(self.h).decode())
        return s

    # -- calls of include/reg.h ---------------------------------------------
    def set_images(self, m_R, m_T):
        self._call("reg_set_images", _ptr(m_R, self.N, "m_R"), _ptr(m_T, self.N, "m_T"))

    def set_beta(self, beta):
        self._call("reg_set_beta", float(beta))

    def transport(self, v, m0, m1):
        self._call("reg_transport", _ptr(v, 2 * self.N, "v"), _ptr(m0, self.N, "m0"),
                   _ptr(m1, self.N, "m1"))

    def deformation_map(self, v, u, det=None):
        self._call("reg_deformation_map", _ptr(v, 2 * self.N, "v"), _ptr(u, 2 * self.N, "u"),
                   _ptr(det, self.N, "det"))

    def transport_rk2a(self, v, m0, m1, nt):
        self._call("reg_transport_rk2a", _ptr(v, 2 * self.N, "v"), _ptr(m0, self.N, "m0"),
                   _ptr(m1, self.N, "m1"), int(nt))

    def adjoint_rk2a(self, v, lam1, lam0, nt):
        self._call("reg_adjoint_rk2a", _ptr(v, 2 * self.N, "v"), _ptr(lam1, self.N, "lam1"),
                   _ptr(lam0, self.N, "lam0"), int(nt))

    def departure_points(self, v, dX=None, dY=None):
        self._call("reg_departure_points", _ptr(v, 2 * self.N, "v"),
                   _ptr(dX, 2 * self.N, "dX"), _ptr(dY, 2 * self.N, "dY"))

    def interpolate(self, u, disp, out):
        self._call("reg_interpolate", _ptr(u, self.N, "u"), _ptr(disp, 2 * self.N, "disp"),
                   _ptr(out, self.N, "out"))

    def spectral(self, op, inp, out, s=0.0):
        # fields in and out per op (include/reg.h): grad scalar -> vector,
        # div vector -> scalar, prefilter scalar -> scalar, the rest vector -> vector
        nin = {REG_SPEC_GRAD: 1, REG_SPEC_PREFILTER: 1}.get(op, 2)
        nout = {REG_SPEC_DIV: 1, REG_SPEC_PREFILTER: 1}.get(op, 2)
        self._call("reg_spectral", int(op), float(s), _ptr(inp, nin * self.N, "in"),
                   _ptr(out, nout * self.N, "out"))

    def restrict(self, fine, coarse):
        self._call("reg_restrict", _ptr(fine, 2 * self.N, "fine"), _ptr(coarse, self.N // 2, "coarse"))

    def prolong(self, coarse, fine):
        self._call("reg_prolong", _ptr(coarse, self.N // 2, "coarse"), _ptr(fine, 2 * self.N, "fine"))

    def objective_gradient(self, v, g=None):
        J = ctypes.c_double()
        self._call("reg_objective_gradient", _ptr(v, 2 * self.N, "v"), ctypes.byref(J),
                   _ptr(g, 2 * self.N, "g"))
        return J.value

    def objective(self, v):
        J = ctypes.c_double()
        self._call("reg_objective", _ptr(v, 2 * self.N, "v"), ctypes.byref(J))
        return J.value

    def hessian_matvec(self, v, vt, Hvt):
        self._call("reg_hessian_matvec", _ptr(v, 2 * self.N, "v"), _ptr(vt, 2 * self.N, "vt"),
                   _ptr(Hvt, 2 * self.N, "Hvt"))

    def precond_apply(self, r, z):
        self._call("reg_precond_apply", _ptr(r, 2 * self.N, "r"), _ptr(z, 2 * self.N, "z"))

    def kkt_solve(self, v, rhs, rtol, maxit, x):
        info = reg_info()
        self._call("reg_kkt_solve", _ptr(v, 2 * self.N, "v"), _ptr(rhs, 2 * self.N, "rhs"),
                   float(rtol), int(maxit), _ptr(x, 2 * self.N, "x"), ctypes.byref(info))
        return info.as_dict()

    def eigen_bounds(self):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        self._call("reg_eigen_bounds", ctypes.byref(lo), ctypes.byref(hi))
        return lo.value, hi.value

    def warm_start(self, net, v):
        """reg_warm_start: v <- net(m_R, m_T) prolonged to this grid if it lowers
        J below J(0), else 0. Returns True if the network's velocity was kept."""
        acc = ctypes.c_int(0)
        self._call("reg_warm_start", net.h, _ptr(v, 2 * self.N, "v"), ctypes.byref(acc))
        return bool(acc.value)

    def solve(self, v, gtol, allow=(REG_OK,)):
        import torch
        info = reg_info()
        self.lib.reg_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        s = self.lib.reg_solve(self.h, _ptr(v, 2 * self.N, "v"), float(gtol), ctypes.byref(info))
        if s not in allow:
            raise RegError(s, self.lib.reg_last_error(self.h).decode())
        d = info.as_dict()
        d["status_name"] = STATUS_NAMES.get(s, str(s))
        return d

    def step_tiles(self):
        """Tile shapes of the step kernels, {(level, kernel): (threads, points)}
        for levels "fine" and "coarse" (when P_2L has one) and kernels
        "adjoint", "incstate" (reg_step_tiles)."""
        t = (ctypes.c_int * 4)()
        self._call("reg_step_tiles", t)
        out = {}
        for i, (lvl, ker) in enumerate((("fine", "adjoint"), ("fine", "incstate"),
                                        ("coarse", "adjoint"), ("coarse", "incstate"))):
            if t[i] > 0:
                out[(lvl, ker)] = (128 << ((t[i] - 1) // 3), 1 << ((t[i] - 1) % 3))
        return out

    def profile_enable(self, enable=True):
        self._call("reg_profile_enable", 1 if enable else 0)

    def profile_read(self):
        """{(level, class name): (ms, launches, algorithmic bytes)} since
        profile_enable; level "fine" is the problem grid, "coarse" the coarse
        grid of the two-level preconditioner."""
        out = {}
        for lvl, lname in enumerate(("fine", "coarse")):
            for k, name in enumerate(KERNEL_CLASSES):
                ms, n, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
                self._call("reg_profile_read", lvl, k, ctypes.byref(ms), ctypes.byref(n),
                           ctypes.byref(by))
                out[(lname, name)] = (ms.value, n.value, by.value)
        return out

    def dot(self, a, b):
        out = ctypes.c_double()
        self._call("reg_dot", _ptr(a, name="a"), _ptr(b, b.numel() if a is None else a.numel(), "b"),
                   ctypes.c_longlong(a.numel()), ctypes.byref(out))
        return out.value


class Batch:
    """reg_batch: independent problems solved concurrently (own context and
    stream each, a pool of host threads). Methods take lists of tensors."""

    def __init__(self, grids, nt, betas, **options):
        self.lib = load()
        self.grids = [(int(a), int(b)) for a, b in grids]
        self.B = len(self.grids)
        G = (reg_grid * self.B)(*[reg_grid(a, b) for a, b in self.grids])
        Bt = (ctypes.c_double * self.B)(*[float(x) for x in betas])
        self.options = default_options(**options)
        h = ctypes.c_void_p()
        s = self.lib.reg_batch_create(G, self.B, int(nt), Bt, ctypes.byref(self.options),
                                      ctypes.byref(h))
        if s != REG_OK:
            raise RegError(s, "reg_batch_create failed")
        self.h = h

    def _ptrs(self, ts, per_point, name):
        arr = (ctypes.c_void_p * self.B)()
        for i, (t, (a, b)) in enumerate(zip(ts, self.grids)):
            arr[i] = _ptr(t, per_point * a * b, f"{name}[{i}]").value
        return arr

    def _check(self, s):
        if s != REG_OK:
            raise RegError(s, self.lib.reg_batch_last_error(self.h).decode())

    def set_images(self, m_R, m_T):
        import torch
        torch.cuda.synchronize()
        self._check(self.lib.reg_batch_set_images(self.h, self._ptrs(m_R, 1, "m_R"),
                                                  self._ptrs(m_T, 1, "m_T")))

    def set_beta(self, betas):
        self._check(self.lib.reg_batch_set_beta(self.h, (ctypes.c_double * self.B)(*betas)))

    def solve(self, vs, gtol, threads=0, allow=(REG_OK, REG_ENOTCONV, REG_ELINESEARCH)):
        import torch
        torch.cuda.synchronize()
        infos = (reg_info * self.B)()
        s = self.lib.reg_batch_solve(self.h, self._ptrs(vs, 2, "v"), float(gtol), int(threads),
                                     infos)
        if s not in allow:
            self._check(s)
        out = []
        for i in range(self.B):
            d = infos[i].as_dict()
            d["status_name"] = STATUS_NAMES.get(d["status"], str(d["status"]))
            out.append(d)
        return out

    def hessian_matvec(self, vs, vts, Hs):
        import torch
        torch.cuda.synchronize()
        self._check(self.lib.reg_batch_hessian_matvec(self.h, self._ptrs(vs, 2, "v"),
                                                      self._ptrs(vts, 2, "vt"),
                                                      self._ptrs(Hs, 2, "Hvt")))

    def close(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.reg_batch_destroy(h)
            self.h = None

    __del__ = close


class Registration3:
    """reg3_ctx: the registration problem on an n1 x n2 x n3 periodic grid.
    Fields are contiguous float32 CUDA tensors (x_1 fastest), vector fields
    their three components back to back. Options as reg_options; precond
    defaults to P_REG here (REG_PC_2L, the two-level preconditioner with
    CHEB(k) or nested PCG(eps) coarse solves, needs every n_i / 2 to be a
    supported size). Methods carry the C names without the reg3_ prefix."""

    def __init__(self, n1, n2, n3, nt, beta, **options):
        self.lib = load()
        self.n1, self.n2, self.n3, self.nt = int(n1), int(n2), int(n3), int(nt)
        self.N = self.n1 * self.n2 * self.n3
        options.setdefault("precond", REG_PC_REG)
        self.options = default_options(**options)
        h = ctypes.c_void_p()
        s = self.lib.reg3_create(self.n1, self.n2, self.n3, self.nt, float(beta),
                                 ctypes.byref(self.options), ctypes.byref(h))
        if s != REG_OK:
            raise RegError(s, "reg3_create failed")
        self.h = h

    def _call(self, name, *args):
        import torch
        self.lib.reg3_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        s = getattr(self.lib, name)(self.h, *args)
        if s != REG_OK:
            raise RegError(s, self.lib.reg3_last_error(self.h).decode())
        return s

    def set_images(self, m_R, m_T):
        self._call("reg3_set_images", _ptr(m_R, self.N, "m_R"), _ptr(m_T, self.N, "m_T"))

    def transport(self, v, m0, m1):
        self._call("reg3_transport", _ptr(v, 3 * self.N, "v"), _ptr(m0, self.N, "m0"),
                   _ptr(m1, self.N, "m1"))

    def precond_apply(self, v, r, z):
        self._call("reg3_precond_apply", _ptr(v, 3 * self.N, "v"), _ptr(r, 3 * self.N, "r"),
                   _ptr(z, 3 * self.N, "z"))

    def eigen_bounds(self):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        self._call("reg3_eigen_bounds", ctypes.byref(lo), ctypes.byref(hi))
        return lo.value, hi.value

    def deformation_map(self, v, u, det=None):
        self._call("reg3_deformation_map", _ptr(v, 3 * self.N, "v"), _ptr(u, 3 * self.N, "u"),
                   _ptr(det, self.N, "det"))

    def spectral(self, op, x, out, s=1.0):
        nin = self.N if op == REG_SPEC_GRAD else 3 * self.N
        nout = self.N if op == REG_SPEC_DIV else 3 * self.N
        self._call("reg3_spectral", int(op), float(s), _ptr(x, nin, "in"), _ptr(out, nout, "out"))

    def objective_gradient(self, v, g=None):
        J = ctypes.c_double()
        self._call("reg3_objective_gradient", _ptr(v, 3 * self.N, "v"), ctypes.byref(J),
                   _ptr(g, 3 * self.N, "g") if g is not None else None)
        return J.value

    def hessian_matvec(self, v, vt, out):
        self._call("reg3_hessian_matvec", _ptr(v, 3 * self.N, "v"), _ptr(vt, 3 * self.N, "vt"),
                   _ptr(out, 3 * self.N, "Hvt"))

    def solve(self, v, gtol, allow=(REG_OK,)):
        import torch
        info = reg_info()
        self.lib.reg3_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        s = self.lib.reg3_solve(self.h, _ptr(v, 3 * self.N, "v"), float(gtol), ctypes.byref(info))
        if s not in allow:
            raise RegError(s, self.lib.reg3_last_error(self.h).decode())
        d = info.as_dict()
        d["status_name"] = STATUS_NAMES.get(s, str(s))
        return d

    def close(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.reg3_destroy(h)
            self.h = None

    __del__ = close


class Lockstep:
    """reg_lockstep: independent problems of uneven size advanced in lockstep
    (one launch per transport step over all problems, one CUDA graph for the
    matvec). Options as reg_options; precond defaults to P_REG here, the form
    the lockstep batch requires. Methods take lists of tensors."""

    def __init__(self, grids, nt, betas, **options):
        self.lib = load()
        self.grids = [(int(a), int(b)) for a, b in grids]
        self.B = len(self.grids)
        G = (reg_grid * self.B)(*[reg_grid(a, b) for a, b in self.grids])
        Bt = (ctypes.c_double * self.B)(*[float(x) for x in betas])
        options.setdefault("precond", REG_PC_REG)
        self.options = default_options(**options)
        h = ctypes.c_void_p()
        s = self.lib.reg_lockstep_create(G, self.B, int(nt), Bt, ctypes.byref(self.options),
                                         ctypes.byref(h))
        if s != REG_OK:
            raise RegError(s, "reg_lockstep_create failed")
        self.h = h

    def _ptrs(self, ts, per_point, name):
        arr = (ctypes.c_void_p * self.B)()
        for i, (t, (a, b)) in enumerate(zip(ts, self.grids)):
            arr[i] = _ptr(t, per_point * a * b, f"{name}[{i}]").value
        return arr

    def _check(self, s):
        if s != REG_OK:
            raise RegError(s, self.lib.reg_lockstep_last_error(self.h).decode())

    def _order(self):
        import torch
        s = torch.cuda.current_stream().cuda_stream
        self._check(self.lib.reg_lockstep_set_stream(self.h, ctypes.c_void_p(s)))

    def set_images(self, m_R, m_T):
        self._order()
        self._check(self.lib.reg_lockstep_set_images(self.h, self._ptrs(m_R, 1, "m_R"),
                                                     self._ptrs(m_T, 1, "m_T")))

    def objective_gradient(self, vs, gs=None):
        self._order()
        J = (ctypes.c_double * self.B)()
        g = self._ptrs(gs, 2, "g") if gs is not None else None
        self._check(self.lib.reg_lockstep_objective_gradient(self.h, self._ptrs(vs, 2, "v"), J, g))
        return list(J)

    def hessian_matvec(self, vs, vts, Hs):
        self._order()
        self._check(self.lib.reg_lockstep_hessian_matvec(self.h, self._ptrs(vs, 2, "v"),
                                                         self._ptrs(vts, 2, "vt"),
                                                         self._ptrs(Hs, 2, "Hvt")))

    def solve(self, vs, gtol, allow=(REG_OK, REG_ENOTCONV, REG_ELINESEARCH)):
        self._order()
        infos = (reg_info * self.B)()
        s = self.lib.reg_lockstep_solve(self.h, self._ptrs(vs, 2, "v"), float(gtol), infos)
        if s not in allow:
            self._check(s)
        out = []
        for i in range(self.B):
            d = infos[i].as_dict()
            d["status_name"] = STATUS_NAMES.get(d["status"], str(d["status"]))
            out.append(d)
        return out

    def matvec_time(self, reps=20):
        """Mean device time (ms) of one replay of the matvec graph of the last
        hessian_matvec (call it twice first)."""
        ms = ctypes.c_double()
        self._check(self.lib.reg_lockstep_matvec_time(self.h, int(reps), ctypes.byref(ms)))
        return ms.value

    def info(self):
        pts, tiles, launches = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.reg_lockstep_info(self.h, ctypes.byref(pts), ctypes.byref(tiles),
                                               ctypes.byref(launches)))
        return {"points": pts.value, "tiles": tiles.value, "matvec_graph_kernels": launches.value}

    def close(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.reg_lockstep_destroy(h)
            self.h = None

    __del__ = close


REG_STATIC_MAX_POINTS = 1024 * 1024


class UNet:
    """reg_unet: the warm-start U-Net (S x S grid, batches up to batch_max).

    Parameters move as flat float32 numpy arrays in the layout of
    include/reg.h; images and velocities are contiguous float32 CUDA tensors
    of B*S*S and B*2*S*S values; idx (optional) is an int32 CUDA tensor of
    problem indices into larger arrays."""

    def __init__(self, size, batch_max):
        self.lib = load()
        self.S, self.bmax = int(size), int(batch_max)
        h = ctypes.c_void_p()
        s = self.lib.reg_unet_create(self.S, self.bmax, ctypes.byref(h))
        if s != REG_OK:
            raise RegError(s, "reg_unet_create failed")
        self.h = h

    @staticmethod
    def param_count():
        return int(load().reg_unet_param_count())

    def _call(self, name, *args):
        import torch
        self.lib.reg_unet_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        s = getattr(self.lib, name)(self.h, *args)
        if s != REG_OK:
            raise RegError(s, self.lib.reg_unet_last_error(self.h).decode())

    def _idx(self, idx, B, *arrays):
        """idx as a pointer after checking the image-pair arrays it selects
        from: without idx each array holds B pairs' worth of S x S fields,
        with idx a whole number of them and every index below that count
        (a read of the indices, one synchronisation)."""
        import torch
        S2 = self.S * self.S
        for a, per in arrays:
            if a is None:
                continue
            _ptr(a, None, "images")
            if idx is None and a.numel() != B * per * S2:
                raise ValueError(f"{a.numel()} elements, expected {B * per * S2}")
            if a.numel() % (per * S2):
                raise ValueError(f"{a.numel()} elements: not whole {per} x {self.S}^2 fields")
        if idx is None:
            return None
        if not (isinstance(idx, torch.Tensor) and idx.is_cuda and idx.dtype == torch.int32
                and idx.is_contiguous() and idx.numel() == B):
            raise TypeError("idx must be a contiguous int32 CUDA tensor of B entries")
        count = min(a.numel() // (per * S2) for a, per in arrays if a is not None)
        if B and (int(idx.min()) < 0 or int(idx.max()) >= count):
            raise ValueError(f"idx outside the {count} pairs of the arrays")
        return ctypes.c_void_p(idx.data_ptr())

    def set_params(self, theta):
        import numpy as np
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.param_count():
            raise ValueError(f"{a.size} parameters, expected {self.param_count()}")
        self._call("reg_unet_set_params", a.ctypes.data_as(ctypes.c_void_p))

    def get_params(self):
        import numpy as np
        a = np.empty(self.param_count(), dtype=np.float32)
        self._call("reg_unet_get_params", a.ctypes.data_as(ctypes.c_void_p))
        return a

    def set_conv_path(self, path):
        """0: mma.sync convolutions; 1: tcgen05 convolutions (tensor memory)."""
        self._call("reg_unet_set_conv_path", int(path))

    def forward(self, B, m_R, m_T, v, idx=None):
        self._call("reg_unet_forward", int(B), self._idx(idx, B, (m_R, 1), (m_T, 1)), _ptr(m_R, name="m_R"),
                   _ptr(m_T, name="m_T"), _ptr(v, 2 * B * self.S * self.S, "v"))

    def gradients(self, B, m_R, m_T, v_target, idx=None):
        """(loss, dL/dparams as a float32 numpy array)."""
        import numpy as np
        g = np.empty(self.param_count(), dtype=np.float32)
        loss = ctypes.c_double()
        self._call("reg_unet_gradients", int(B), self._idx(idx, B, (m_R, 1), (m_T, 1), (v_target, 2)),
                   _ptr(m_R, name="m_R"),
                   _ptr(m_T, name="m_T"), _ptr(v_target, name="v_target"),
                   g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss))
        return loss.value, g

    def train_step(self, B, m_R, m_T, v_target, lr, idx=None):
        loss = ctypes.c_double()
        self._call("reg_unet_train_step", int(B), self._idx(idx, B, (m_R, 1), (m_T, 1), (v_target, 2)),
                   _ptr(m_R, name="m_R"),
                   _ptr(m_T, name="m_T"), _ptr(v_target, name="v_target"), ctypes.c_float(lr),
                   ctypes.byref(loss))
        return loss.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.reg_unet_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def interpolate_static(n1, n2, u, disp, out):
    """reg_interpolate_static: spline interpolation that allocates nothing.

    For callers that may not allocate device memory while running (memory
    owned by another framework's caching allocator, latency-bound loops);
    the coefficient scratch is a fixed 4 MiB device array inside the
    library, shared by all calls: calls overlapping on the GPU race on it.
    Raises RegError on a non-zero status.
    """
    import torch
    N = int(n1) * int(n2)
    s = load().reg_interpolate_static(int(n1), int(n2), _ptr(u, N, "u"), _ptr(disp, 2 * N, "disp"),
                                      _ptr(out, N, "out"),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if s != REG_OK:
        raise RegError(s, "reg_interpolate_static failed")


def launch_count():
    """Kernels launched by libregnk in this process so far."""
    return int(load().reg_launch_count())


def reg_create(n1, n2, nt, beta, **options):
    """Python spelling of reg_create: returns a Registration handle."""
    return Registration(n1, n2, nt, beta, **options)
