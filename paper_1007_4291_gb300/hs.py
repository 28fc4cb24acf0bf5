"""Thin ctypes binding of libhs (include/hs.h): argument marshalling only.

Every call goes through the C ABI of ``libhs.so``; there is no fallback.  If
the library is missing or fails to load, ``load()`` raises.  Functions keep
the C names: ``hs_setup``, ``hs_apply``, ``hs_matvec``, ``hs_solve``,
``hs_destroy``.  Vector arguments may be torch CUDA tensors (their
``data_ptr()`` is passed) or raw integer device pointers.
"""
import ctypes
import os

import numpy as np

_LIB = None
HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libhs.so")

HS_OK, HS_EINVAL, HS_ENOMEM, HS_EBREAKDOWN, HS_ETIMEOUT, HS_ENOCONV, HS_ECUDA, HS_EUNSUPPORTED = range(8)
HS_C64, HS_C128 = 64, 128

EXPORTED = ["hs_default_options", "hs_setup", "hs_setup_batched", "hs_setup_batched_opts", "hs_apply", "hs_apply_batched",
            "hs_apply_noalloc", "hs_autotune", "hs_matvec", "hs_solve", "hs_sync", "hs_last_device_status",
            "hs_plan_bytes", "hs_setup_flops", "hs_release_workspace", "hs_kernel_launches", "hs_destroy", "hs_strerror",
            "hs_cnn_create", "hs_cnn_get_params", "hs_cnn_set_mode", "hs_cnn_apply", "hs_cnn_gradient",
            "hs_cnn_train_step", "hs_cnn_train_step_residual", "hs_cnn_sync", "hs_cnn_destroy", "hs_attach_cnn"]
HS_CNN_NPARAM = 10434


class HsOptions(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("pml_C", ctypes.c_double), ("moving_pml_C", ctypes.c_double),
                ("layers_per_step", ctypes.c_int),
                ("factor_prec", ctypes.c_int), ("chunk", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("restart", ctypes.c_int), ("reorth", ctypes.c_int), ("spin_budget", ctypes.c_longlong),
                ("graphs", ctypes.c_int), ("krylov_basis", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("frontal_gemm", ctypes.c_int), ("tune_cache", ctypes.c_char_p), ("sep_rhs_per_cta", ctypes.c_int),
                ("two_front", ctypes.c_int), ("buffer_rows", ctypes.c_int), ("async_setup", ctypes.c_int)]


class HsSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("applies", ctypes.c_int),
                ("max_relres", ctypes.c_double), ("t_apply_ms", ctypes.c_double),
                ("t_matvec_ms", ctypes.c_double), ("t_orth_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double),
                ("cnn_applies", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, strerror(code), code))


def load(path=None):
    """Load libhs.so (raises if it is missing: the CUDA path has no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIBPATH
    if not os.path.exists(p):
        raise RuntimeError("libhs.so not built (%s); run paper_1007_4291_gb300.build.build()" % p)
    lib = ctypes.CDLL(p)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.hs_default_options.argtypes = [ctypes.POINTER(HsOptions)]
    lib.hs_setup.argtypes = [vp, d, i, i, i, i, ctypes.POINTER(HsOptions), vp, ctypes.POINTER(vp)]
    lib.hs_apply.argtypes = [vp, vp, vp, i, i, vp]
    lib.hs_setup_batched.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(d), ctypes.POINTER(i), i, i, i,
                                     ctypes.POINTER(HsOptions), vp, ctypes.POINTER(vp)]
    lib.hs_setup_batched_opts.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(d), ctypes.POINTER(i), i, i, i,
                                          ctypes.POINTER(HsOptions), vp, ctypes.POINTER(vp)]
    lib.hs_apply_batched.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(i), i, vp]
    lib.hs_autotune.argtypes = [vp, d, i, i, i, i, ctypes.POINTER(HsOptions), i, vp, ctypes.POINTER(i),
                                ctypes.POINTER(d), ctypes.POINTER(i)]
    lib.hs_matvec.argtypes = [vp, vp, vp, i, i, vp]
    lib.hs_apply_noalloc.argtypes = [vp, vp, vp, i, i, vp]
    lib.hs_apply_noalloc.restype = i
    lib.hs_solve.argtypes = [vp, vp, vp, i, d, i, ctypes.POINTER(HsSolveInfo), vp]
    lib.hs_sync.argtypes = [vp, vp]
    lib.hs_last_device_status.argtypes = [vp]
    lib.hs_setup_flops.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.hs_plan_bytes.argtypes = [vp]
    lib.hs_plan_bytes.restype = ll
    lib.hs_destroy.argtypes = [vp]
    lib.hs_strerror.argtypes = [i]
    lib.hs_strerror.restype = ctypes.c_char_p
    lib.hs_release_workspace.argtypes = []
    lib.hs_cnn_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.hs_cnn_get_params.argtypes = [vp, vp]
    lib.hs_cnn_set_mode.argtypes = [vp, i]
    lib.hs_cnn_apply.argtypes = [vp, vp, vp, i, i, i, vp]
    lib.hs_cnn_gradient.argtypes = [vp, vp, vp, i, i, i, ctypes.POINTER(d), vp, vp]
    lib.hs_cnn_train_step.argtypes = [vp, vp, vp, i, i, i, d, ctypes.POINTER(d), vp]
    lib.hs_cnn_destroy.argtypes = [vp]
    lib.hs_cnn_sync.argtypes = [vp, vp]
    lib.hs_cnn_train_step_residual.argtypes = [vp, vp, vp, vp, i, d, ctypes.POINTER(d), vp]
    lib.hs_attach_cnn.argtypes = [vp, vp]
    lib.hs_kernel_launches.argtypes = []
    lib.hs_kernel_launches.restype = ll
    for name in EXPORTED:
        if name not in ("hs_plan_bytes", "hs_strerror", "hs_kernel_launches"):
            getattr(lib, name).restype = i
    _LIB = lib
    return lib


def strerror(code):
    if _LIB is None:
        return "status %d" % code
    return _LIB.hs_strerror(int(code)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("unsupported pointer argument %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _check(code, where):
    if code != HS_OK:
        raise HsError(code, where)
    return code


def hs_default_options(**kw):
    lib = load()
    o = HsOptions()
    _check(lib.hs_default_options(ctypes.byref(o)), "hs_default_options")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def hs_setup(c, omega, n, dim, pml_width, moving_pml_width, opt=None, stream=None):
    """Build a plan from host velocities ``c`` (float64, n*n, x1 fastest)."""
    lib = load()
    c = np.ascontiguousarray(c, dtype=np.float64)
    if c.size != n ** dim:
        raise ValueError("c must hold n**dim values")
    plan = ctypes.c_void_p()
    o = opt if opt is not None else hs_default_options()
    _check(lib.hs_setup(c.ctypes.data, float(omega), int(n), int(dim), int(pml_width), int(moving_pml_width),
                        ctypes.byref(o), _stream(stream), ctypes.byref(plan)), "hs_setup")
    return plan


def hs_setup_batched(cs, omegas, ns, dim, pml_width, moving_pml_width, opt=None, stream=None):
    """Plans of several problems (host velocities cs[k] of ns[k]**dim points),
    all factored in one launch.  Returns the list of plans."""
    lib = load()
    k = len(cs)
    arrs = [np.ascontiguousarray(c, dtype=np.float64) for c in cs]
    for a, n in zip(arrs, ns):
        if a.size != n ** dim:
            raise ValueError("c must hold n**dim values")
    cp = (ctypes.c_void_p * k)(*[a.ctypes.data for a in arrs])
    om = (ctypes.c_double * k)(*[float(w) for w in omegas])
    nn = (ctypes.c_int * k)(*[int(n) for n in ns])
    out = (ctypes.c_void_p * k)()
    if isinstance(opt, (list, tuple)):      # one options struct per problem
        if len(opt) != k:
            raise ValueError("one options struct per problem")
        oa = (HsOptions * k)(*opt)
        _check(lib.hs_setup_batched_opts(k, cp, om, nn, int(dim), int(pml_width), int(moving_pml_width), oa,
                                         _stream(stream), out), "hs_setup_batched_opts")
    else:
        o = opt if opt is not None else hs_default_options()
        _check(lib.hs_setup_batched(k, cp, om, nn, int(dim), int(pml_width), int(moving_pml_width), ctypes.byref(o),
                                    _stream(stream), out), "hs_setup_batched")
    return [ctypes.c_void_p(out[q]) for q in range(k)]


def hs_apply_batched(plans, rs, zs, nrhs, dtype, stream=None):
    """z[k] = M_alpha^(k) r[k] for all plans in one (cached) CUDA graph."""
    k = len(plans)
    pp = (ctypes.c_void_p * k)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    rp = (ctypes.c_void_p * k)(*[_ptr(r) for r in rs])
    zp = (ctypes.c_void_p * k)(*[_ptr(z) for z in zs])
    nr = (ctypes.c_int * k)(*[int(q) for q in nrhs])
    return _check(load().hs_apply_batched(k, pp, rp, zp, nr, int(dtype), _stream(stream)), "hs_apply_batched")


def hs_autotune(c, omega, n, dim, pml_width, moving_pml_width, nrhs, opt=None, stream=None):
    """Time the candidate chunk lengths and separator groupings; returns
    (best chunk, ms per application, RHS per separator-solve CTA)."""
    lib = load()
    c = np.ascontiguousarray(c, dtype=np.float64)
    o = opt if opt is not None else hs_default_options()
    best, ms, sep = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    _check(lib.hs_autotune(c.ctypes.data, float(omega), int(n), int(dim), int(pml_width), int(moving_pml_width),
                           ctypes.byref(o), int(nrhs), _stream(stream), ctypes.byref(best), ctypes.byref(ms),
                           ctypes.byref(sep)), "hs_autotune")
    return best.value, ms.value, sep.value


def hs_cnn_create(params):
    """Network from a host parameter vector (HS_CNN_NPARAM values)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != HS_CNN_NPARAM:
        raise ValueError("expected %d parameters" % HS_CNN_NPARAM)
    net = ctypes.c_void_p()
    _check(load().hs_cnn_create(p.ctypes.data, ctypes.byref(net)), "hs_cnn_create")
    return net


def hs_cnn_get_params(net):
    out = np.empty(HS_CNN_NPARAM, dtype=np.float32)
    _check(load().hs_cnn_get_params(net, out.ctypes.data), "hs_cnn_get_params")
    return out


def hs_cnn_set_mode(net, tensor_cores):
    return _check(load().hs_cnn_set_mode(net, int(bool(tensor_cores))), "hs_cnn_set_mode")


def hs_cnn_apply(net, r, z, nrhs, n, dtype, stream=None):
    return _check(load().hs_cnn_apply(net, _ptr(r), _ptr(z), int(nrhs), int(n), int(dtype), _stream(stream)),
                  "hs_cnn_apply")


def hs_cnn_gradient(net, r, e, nrhs, n, dtype, stream=None):
    """Returns (loss, gradient as a float32 host array)."""
    loss = ctypes.c_double()
    g = np.empty(HS_CNN_NPARAM, dtype=np.float32)
    _check(load().hs_cnn_gradient(net, _ptr(r), _ptr(e), int(nrhs), int(n), int(dtype), ctypes.byref(loss),
                                  g.ctypes.data, _stream(stream)), "hs_cnn_gradient")
    return loss.value, g


def hs_cnn_train_step(net, r, e, nrhs, n, dtype, lr, stream=None):
    loss = ctypes.c_double()
    _check(load().hs_cnn_train_step(net, _ptr(r), _ptr(e), int(nrhs), int(n), int(dtype), float(lr),
                                    ctypes.byref(loss), _stream(stream)), "hs_cnn_train_step")
    return loss.value


def hs_cnn_train_step_residual(net, plan, x, rho, nrhs, lr, stream=None):
    loss = ctypes.c_double()
    _check(load().hs_cnn_train_step_residual(net, plan, _ptr(x), _ptr(rho), int(nrhs), float(lr), ctypes.byref(loss),
                                             _stream(stream)), "hs_cnn_train_step_residual")
    return loss.value


def hs_cnn_sync(net, stream=None):
    return load().hs_cnn_sync(net, _stream(stream))


def hs_cnn_destroy(net):
    return load().hs_cnn_destroy(net)


def hs_attach_cnn(plan, net):
    return _check(load().hs_attach_cnn(plan, net), "hs_attach_cnn")


def hs_kernel_launches():
    return load().hs_kernel_launches()


def hs_release_workspace():
    return load().hs_release_workspace()


def hs_apply(plan, r, z, nrhs, dtype, stream=None):
    return _check(load().hs_apply(plan, _ptr(r), _ptr(z), int(nrhs), int(dtype), _stream(stream)), "hs_apply")


def hs_apply_noalloc(plan, r, z, nrhs, dtype, stream=None):
    """hs_apply with all temporaries in the library's static device scratch."""
    return _check(load().hs_apply_noalloc(plan, _ptr(r), _ptr(z), int(nrhs), int(dtype), _stream(stream)),
                  "hs_apply_noalloc")


def hs_matvec(plan, x, y, nrhs, dtype, stream=None):
    return _check(load().hs_matvec(plan, _ptr(x), _ptr(y), int(nrhs), int(dtype), _stream(stream)), "hs_matvec")


def hs_solve(plan, f, u, nrhs, tol, maxit, stream=None, check=True):
    """Returns (status, info dict).  Raises on errors other than HS_ENOCONV
    unless ``check`` is False."""
    info = HsSolveInfo()
    code = load().hs_solve(plan, _ptr(f), _ptr(u), int(nrhs), float(tol), int(maxit), ctypes.byref(info),
                           _stream(stream))
    if check and code not in (HS_OK, HS_ENOCONV):
        raise HsError(code, "hs_solve")
    return code, info.as_dict()


def hs_sync(plan, stream=None):
    return load().hs_sync(plan, _stream(stream))


def hs_last_device_status(plan):
    return load().hs_last_device_status(plan)


def hs_plan_bytes(plan):
    return load().hs_plan_bytes(plan)


def hs_setup_flops(plan):
    """(frontal GEMM flops, pivot-block inversion flops) of a 3D plan's setup."""
    g, v = ctypes.c_double(), ctypes.c_double()
    _check(load().hs_setup_flops(plan, ctypes.byref(g), ctypes.byref(v)), "hs_setup_flops")
    return g.value, v.value


def hs_destroy(plan):
    return load().hs_destroy(plan)
