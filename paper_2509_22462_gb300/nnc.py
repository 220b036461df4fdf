"""ctypes binding of libnnc (include/nnc.h), with the same names as the C ABI.

The binding only marshals arguments: every step of the computation runs in the CUDA library.
If the library is missing or has no usable sm_103a device, calls raise; there is no fallback.
Host calls take and return numpy float64 arrays; the *_dev calls take CUDA torch tensors
(float64, contiguous) and queue work on the current torch stream.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnnc.so")

FP64, FP32, BF16, BF16X3, FP8 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "bf16x3": BF16X3, "fp8": FP8}
ACTS = {"identity": 0, "tanh": 1, "sigmoid": 2, "softplus": 3, "gelu": 4, "softmax": 5}
WANT_Y, WANT_J, WANT_H, WANT_G = 1, 2, 4, 8
STATUS = {0: "NNC_OK", -1: "NNC_ERR_ARG", -2: "NNC_ERR_CUDA", -3: "NNC_ERR_NONFINITE",
          -4: "NNC_ERR_TIMEOUT", -5: "NNC_ERR_OOM", -6: "NNC_ERR_UNSUPPORTED"}

# Every symbol that include/nnc.h declares.
EXPORTS = ["nnc_load_weights", "nnc_eval", "nnc_residual", "nnc_jacobian", "nnc_hessian_lag",
           "nnc_eval_batched", "nnc_eval_dev", "nnc_residual_dev", "nnc_jacobian_dev",
           "nnc_hessian_lag_dev", "nnc_eval_all_dev", "nnc_eval_kkt_dev", "nnc_eval_kkt", "nnc_free", "nnc_last_error",
           "nnc_net_info", "nnc_launch_count", "nnc_profile", "nnc_profile_read",
           "nnc_ipm_default_options", "nnc_ipm_adversarial", "nnc_ipm_adversarial_l1",
           "nnc_ipm_adversarial_l1_fullspace", "nnc_layer_weights", "nnc_selftest_bounded_wait", "nnc_selftest_net_wait",
           "nnc_kkt_solve", "nnc_stage_kkt_solve",
           "nnc_residual_noalloc", "nnc_batch_create", "nnc_batch_free", "nnc_batch_info",
           "nnc_batch_set_bias", "nnc_batch_use_graph", "nnc_batch_tune_set", "nnc_batch_tuning", "nnc_batch_autotune", "nnc_batch_eval_dev", "nnc_batch_residual_dev", "nnc_batch_eval_kkt_dev",
           "nnc_batch_eval", "nnc_batch_residual", "nnc_batch_eval_kkt", "nnc_ipm_scopf", "nnc_ws_create", "nnc_ws_free",
           "nnc_ws_set_scaling", "nnc_ws_loss_grad", "nnc_ws_adam_step", "nnc_ws_train",
           "nnc_ws_predict", "nnc_ws_get_params", "nnc_ipm_scopf_warm", "nnc_autotune", "nnc_tuning", "nnc_tune_set"]
IPM_STATUS = {0: "optimal", 1: "max_iter", 2: "linesearch_failed", 3: "nonfinite",
              4: "inertia_failed", 5: "eval_error"}


class IpmOptions(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mu0", ctypes.c_double),
                ("kappa_mu", ctypes.c_double), ("theta_mu", ctypes.c_double),
                ("kappa_eps", ctypes.c_double), ("tau_min", ctypes.c_double),
                ("kappa1", ctypes.c_double), ("kappa2", ctypes.c_double), ("s_max", ctypes.c_double),
                ("eta", ctypes.c_double), ("delta_w0", ctypes.c_double),
                ("delta_w_min", ctypes.c_double), ("delta_w_max", ctypes.c_double),
                ("kappa_w_plus", ctypes.c_double), ("kappa_w_plus_bar", ctypes.c_double),
                ("kappa_w_minus", ctypes.c_double), ("kappa_sigma", ctypes.c_double),
                ("max_backtracks", ctypes.c_int), ("max_ls_failures", ctypes.c_int),
                ("verbose", ctypes.c_int), ("warm_mu0", ctypes.c_double),
                ("kkt_on_device", ctypes.c_int)]


class IpmResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("obj", ctypes.c_double),
                ("kkt_error", ctypes.c_double), ("solve_seconds", ctypes.c_double),
                ("t_function", ctypes.c_double), ("t_jacobian", ctypes.c_double),
                ("t_hessian", ctypes.c_double), ("t_solver", ctypes.c_double),
                ("n_function", ctypes.c_int), ("n_jacobian", ctypes.c_int),
                ("n_hessian", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = IPM_STATUS.get(self.status, str(self.status))
        return d
PROFILE_KINDS = ["tangent_gemm", "syrk", "forward", "reverse", "other", "tangent_chain",
                 "value_pass"]


class NNCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def load_library(path: str = LIB_PATH):
    """Load libnnc.so (raise if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it first (python -m paper_2509_22462_gb300.build)")
    lib = ctypes.CDLL(path)
    for name in EXPORTS:
        getattr(lib, name)
    lib.nnc_load_weights.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_DP),
                                     ctypes.POINTER(_DP), ctypes.c_int, _P]
    lib.nnc_eval.argtypes = [_P, _DP, _DP, ctypes.c_int]
    lib.nnc_residual.argtypes = [_P, _DP, _DP, _DP]
    lib.nnc_jacobian.argtypes = [_P, _DP, _DP]
    lib.nnc_hessian_lag.argtypes = [_P, _DP, _DP, _DP, _DP]
    lib.nnc_eval_batched.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_DP),
                                     ctypes.POINTER(_DP), ctypes.POINTER(_DP), ctypes.POINTER(_DP),
                                     ctypes.POINTER(_DP), ctypes.c_uint]
    lib.nnc_eval_dev.argtypes = [_P, _P, _P, ctypes.c_int, _P]
    lib.nnc_residual_dev.argtypes = [_P, _P, _P, _P, _P]
    lib.nnc_jacobian_dev.argtypes = [_P, _P, _P, _P]
    lib.nnc_hessian_lag_dev.argtypes = [_P, _P, _P, _P, _P, _P]
    lib.nnc_eval_all_dev.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P]
    lib.nnc_eval_kkt_dev.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P]
    # host arrays passed as raw addresses (the per-call IPM path; data_as costs ~3 us a pointer)
    lib.nnc_eval_kkt.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P]
    lib.nnc_free.argtypes = [_P]
    lib.nnc_free.restype = None
    lib.nnc_ipm_default_options.restype = None
    lib.nnc_last_error.restype = ctypes.c_char_p
    lib.nnc_net_info.argtypes = [_P] + [ctypes.POINTER(ctypes.c_int)] * 4
    lib.nnc_launch_count.restype = ctypes.c_longlong
    lib.nnc_profile.argtypes = [_P, ctypes.c_int]
    lib.nnc_ipm_default_options.argtypes = [ctypes.POINTER(IpmOptions)]
    lib.nnc_batch_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int, _P]
    lib.nnc_batch_free.argtypes = [_P]
    lib.nnc_batch_free.restype = None
    lib.nnc_batch_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
    lib.nnc_batch_set_bias.argtypes = [_P, ctypes.c_int, _DP]
    lib.nnc_batch_use_graph.argtypes = [_P, ctypes.c_int]
    lib.nnc_batch_tune_set.argtypes = [_P, ctypes.c_int]
    lib.nnc_batch_tuning.argtypes = [_P, ctypes.POINTER(ctypes.c_int)]
    lib.nnc_batch_autotune.argtypes = [_P, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]
    lib.nnc_batch_eval_dev.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P]
    lib.nnc_batch_residual_dev.argtypes = [_P, _P, _P, _P, _P]
    lib.nnc_batch_eval_kkt_dev.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P]
    lib.nnc_batch_eval.argtypes = [_P, _DP, _DP, _DP, _DP, _DP, _DP]
    lib.nnc_batch_residual.argtypes = [_P, _DP, _DP, _DP]
    lib.nnc_batch_eval_kkt.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P]
    lib.nnc_ipm_scopf.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), _DP, ctypes.c_double, _DP,
                                  ctypes.POINTER(IpmOptions), _DP, _DP, ctypes.POINTER(IpmResult)]
    lib.nnc_autotune.argtypes = [_P, ctypes.c_char_p, ctypes.c_int]
    lib.nnc_tuning.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.nnc_tune_set.argtypes = [_P, ctypes.c_int, ctypes.c_int]
    lib.nnc_ipm_scopf_warm.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), _DP, ctypes.c_double, _DP, _DP, _DP,
                                       ctypes.POINTER(IpmOptions), _DP, _DP, ctypes.POINTER(IpmResult)]
    lib.nnc_ws_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(_DP), ctypes.c_int, _P]
    lib.nnc_ws_free.argtypes = [_P]
    lib.nnc_ws_free.restype = None
    lib.nnc_ws_set_scaling.argtypes = [_P, _DP, _DP, _DP, _DP]
    lib.nnc_ws_loss_grad.argtypes = [_P, _DP, _DP, ctypes.c_int, _DP, ctypes.POINTER(_DP)]
    lib.nnc_ws_adam_step.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.nnc_ws_train.argtypes = [_P, _DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_ulonglong, _DP]
    lib.nnc_ws_predict.argtypes = [_P, _DP, ctypes.c_int, _DP]
    lib.nnc_ws_get_params.argtypes = [_P, ctypes.POINTER(_DP)]
    lib.nnc_residual_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_P),
                                         ctypes.POINTER(_P), _P, _P, _P, _P]
    lib.nnc_kkt_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP, _DP, _DP, _DP, _DP,
                                  ctypes.c_double, ctypes.c_double, _DP, ctypes.POINTER(ctypes.c_int)]
    lib.nnc_stage_kkt_solve.argtypes = [ctypes.c_int, ctypes.c_int, _IP, _IP, ctypes.c_int, _IP, _IP, _DP,
                                        ctypes.c_int, _IP, _IP, _DP, _DP, ctypes.c_double,
                                        ctypes.c_double, _DP, _IP]
    lib.nnc_ipm_adversarial.argtypes = [_P, _DP, ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(IpmOptions), _DP, _DP,
                                        ctypes.POINTER(IpmResult)]
    lib.nnc_ipm_adversarial_l1.argtypes = [_P, _DP, ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(IpmOptions), _DP, _DP,
                                           ctypes.POINTER(IpmResult)]
    lib.nnc_ipm_adversarial_l1_fullspace.argtypes = [_P, _DP, ctypes.c_int, ctypes.c_double,
                                                     ctypes.POINTER(IpmOptions), _DP, _DP,
                                                     ctypes.POINTER(IpmResult)]
    lib.nnc_layer_weights.argtypes = [_P, ctypes.c_int, _DP, _DP, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.nnc_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
    lib.nnc_selftest_net_wait.argtypes = [_P, ctypes.c_int, ctypes.c_longlong]
    lib.nnc_profile_read.argtypes = [_P, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    for name in EXPORTS:
        if name not in ("nnc_free", "nnc_last_error", "nnc_launch_count", "nnc_ipm_default_options",
                        "nnc_batch_free", "nnc_ws_free"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code):
    if code != 0:
        raise NNCError(code, _lib.nnc_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ad(a):
    """Address of a C-contiguous numpy array, for c_void_p arguments."""
    return a.ctypes.data


def launch_count() -> int:
    return int(load_library().nnc_launch_count())


def _stream_ptr():
    """torch's current stream as a cudaStream_t.  torch reports the legacy default stream as 0,
    which the C ABI reads as "the net's own stream", so it is passed as cudaStreamLegacy (1)."""
    import torch
    h = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(h if h else 1)


def _tp(t):
    """Device pointer of a CUDA float64 tensor (None -> NULL)."""
    if t is None:
        return None
    assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


class Net:
    """An MLP y = NN(x) (Eq. 3) loaded into libnnc on the current CUDA device."""

    def __init__(self, widths, acts, W, b=None, precision="fp64", stream=None):
        lib = load_library()
        self.widths = [int(w) for w in widths]
        self.acts = list(acts)
        L = len(self.widths) - 1
        self.n_in, self.n_out = self.widths[0], self.widths[-1]
        self.precision = precision if isinstance(precision, str) else \
            {v: k for k, v in PRECISIONS.items()}[precision]
        Wc = [_f64(w) for w in W]
        bc = [_f64(x) for x in b] if b is not None else None
        for l in range(L):
            assert Wc[l].shape == (self.widths[l + 1], self.widths[l]), (l, Wc[l].shape)
        wid = (ctypes.c_int * (L + 1))(*self.widths)
        act = (ctypes.c_int * L)(*[ACTS[a] if isinstance(a, str) else int(a) for a in self.acts])
        Wp = (_DP * L)(*[_dp(w) for w in Wc])
        bp = (_DP * L)(*[_dp(x) for x in bc]) if bc is not None else None
        h = _P()
        _check(lib.nnc_load_weights(ctypes.byref(h), L, wid, act, Wp, bp,
                                    PRECISIONS[self.precision], stream))
        self._h = h

    @classmethod
    def from_mlp(cls, mlp, precision="fp64", stream=None):
        return cls(mlp.spec.widths, mlp.spec.acts, mlp.W, mlp.b, precision, stream)

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.nnc_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # ---------------------------------------------------------------- host calls
    def eval(self, x, fp64_residual=False):
        x = _f64(x)
        y = np.empty(self.n_out)
        _check(_lib.nnc_eval(self._h, _dp(x), _dp(y), int(bool(fp64_residual))))
        return y

    def residual(self, x, y):
        x, y = _f64(x), _f64(y)
        r = np.empty(self.n_out)
        _check(_lib.nnc_residual(self._h, _dp(x), _dp(y), _dp(r)))
        return r

    def jacobian(self, x):
        x = _f64(x)
        J = np.empty((self.n_out, self.n_in))
        _check(_lib.nnc_jacobian(self._h, _dp(x), _dp(J)))
        return J

    def hessian_lag(self, x, lam, want_grad=False):
        x, lam = _f64(x), _f64(lam)
        H = np.empty((self.n_in, self.n_in))
        g = np.empty(self.n_in) if want_grad else None
        _check(_lib.nnc_hessian_lag(self._h, _dp(x), _dp(lam), _dp(H),
                                    _dp(g) if want_grad else None))
        return (H, g) if want_grad else H

    def eval_kkt(self, x, y, lam, out=None):
        """nnc_eval_kkt: (r = y - NN(x), J, H, grad = lambda^T J) at one iterate, one value pass.
        out: optional (r, J, H, grad) float64 C-contiguous arrays to fill (for example views of
        pinned host memory), else new arrays."""
        x, y, lam = _f64(x), _f64(y), _f64(lam)
        if out is None:
            out = (np.empty(self.n_out), np.empty((self.n_out, self.n_in)),
                   np.empty((self.n_in, self.n_in)), np.empty(self.n_in))
        r, J, H, g = out
        for a, shape in zip(out, ((self.n_out,), (self.n_out, self.n_in), (self.n_in, self.n_in),
                                  (self.n_in,))):
            if a.dtype != np.float64 or a.shape != shape or not a.flags.c_contiguous:
                raise ValueError("eval_kkt: out arrays must be C-contiguous float64 of shapes "
                                 "(n_out,), (n_out, n_in), (n_in, n_in), (n_in,)")
        _check(_lib.nnc_eval_kkt(self._h, _ad(x), _ad(y), _ad(lam), _ad(r), _ad(J), _ad(H), _ad(g)))
        return r, J, H, g

    def autotune(self, cache_path=None, retune=False):
        """nnc_autotune: time the tile / split candidates and keep the fastest (JSON cache optional)."""
        _check(_lib.nnc_autotune(self._h, cache_path.encode() if cache_path else None, int(bool(retune))))

    def tune_set(self, tangent_bn=0, syrk_splits=0):
        """nnc_tune_set: pin the tangent N tile and / or the symmetric-product splits."""
        _check(_lib.nnc_tune_set(self._h, int(tangent_bn), int(syrk_splits)))

    def selftest_wait(self, which, cycles):
        """nnc_selftest_net_wait: queue a bounded wait that runs out into this net's error word."""
        _check(_lib.nnc_selftest_net_wait(self._h, int(which), int(cycles)))

    def tuning(self, layer):
        bn, sp = ctypes.c_int(), ctypes.c_int()
        _check(_lib.nnc_tuning(self._h, int(layer), ctypes.byref(bn), ctypes.byref(sp)))
        return bn.value, sp.value

    def profile(self, enable=True, kinds=None):
        """Start (or stop) event timing of the library's launches; `kinds` (names of
        PROFILE_KINDS) limits it to those kernel kinds."""
        if enable and kinds:
            mask = sum(1 << (PROFILE_KINDS.index(k) + 1) for k in kinds)
            _check(_lib.nnc_profile(self._h, mask))
        else:
            _check(_lib.nnc_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """{kind: (total ms, launches)} recorded since profile(True) (and clears the record)."""
        n = len(PROFILE_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        _check(_lib.nnc_profile_read(self._h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(PROFILE_KINDS)}

    # ---------------------------------------------------------------- device calls
    def eval_dev(self, x, y, fp64_residual=False, stream=None):
        _check(_lib.nnc_eval_dev(self._h, _tp(x), _tp(y), int(bool(fp64_residual)),
                                 stream or _stream_ptr()))

    def residual_dev(self, x, y, r, stream=None):
        _check(_lib.nnc_residual_dev(self._h, _tp(x), _tp(y), _tp(r), stream or _stream_ptr()))

    def jacobian_dev(self, x, J, stream=None):
        _check(_lib.nnc_jacobian_dev(self._h, _tp(x), _tp(J), stream or _stream_ptr()))

    def hessian_lag_dev(self, x, lam, H, grad=None, stream=None):
        _check(_lib.nnc_hessian_lag_dev(self._h, _tp(x), _tp(lam), _tp(H), _tp(grad),
                                        stream or _stream_ptr()))

    def eval_all_dev(self, x, lam=None, y=None, J=None, H=None, grad=None, stream=None):
        _check(_lib.nnc_eval_all_dev(self._h, _tp(x), _tp(lam), _tp(y), _tp(J), _tp(H), _tp(grad),
                                     stream or _stream_ptr()))

    def eval_kkt_dev(self, x, y=None, lam=None, r=None, J=None, H=None, grad=None, stream=None):
        """nnc_eval_kkt_dev: r = y - NN(x), J, H, grad at one iterate from a single value pass."""
        _check(_lib.nnc_eval_kkt_dev(self._h, _tp(x), _tp(y), _tp(lam), _tp(r), _tp(J), _tp(H),
                                     _tp(grad), stream or _stream_ptr()))


def eval_batched(nets, xs, lams=None, what=WANT_Y | WANT_J | WANT_H):
    """nnc_eval_batched over host arrays: returns (ys, Js, Hs) lists (None where not asked)."""
    lib = load_library()
    K = len(nets)
    xs = [_f64(x) for x in xs]
    lams = [_f64(l) for l in lams] if lams is not None else None
    ys = [np.empty(n.n_out) for n in nets] if what & WANT_Y else None
    Js = [np.empty((n.n_out, n.n_in)) for n in nets] if what & WANT_J else None
    Hs = [np.empty((n.n_in, n.n_in)) for n in nets] if what & WANT_H else None
    arr = lambda lst: (_DP * K)(*[_dp(a) for a in lst]) if lst is not None else None  # noqa: E731
    hs = (_P * K)(*[n.handle for n in nets])
    _check(lib.nnc_eval_batched(hs, K, arr(xs), arr(lams), arr(ys), arr(Js), arr(Hs), what))
    return ys, Js, Hs


def ipm_options(**kw) -> IpmOptions:
    o = IpmOptions()
    load_library().nnc_ipm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ipm_adversarial(net, x0, target=3, margin=0.1, **options):
    """Solve the adversarial problem with the host interior-point driver (include/nnc_ipm.h).
    Returns (result dict, v = (x, y, s), lambda)."""
    lib = load_library()
    x0 = _f64(x0)
    o = ipm_options(**options)
    nv = net.n_in + 2 * net.n_out - 1
    v = np.empty(nv)
    lam = np.empty(2 * net.n_out - 1)
    res = IpmResult()
    _check(lib.nnc_ipm_adversarial(net.handle, _dp(x0), int(target), float(margin), ctypes.byref(o),
                                   _dp(v), _dp(lam), ctypes.byref(res)))
    return res.as_dict(), v, lam


def ipm_adversarial_l1(net, x_ref, target, conf=0.6, **options):
    """Eq. 7 (L1 objective by split variables, y_t >= conf) with the host interior-point driver.
    Returns (result dict, v = (x, p, q, y), lambda)."""
    lib = load_library()
    x_ref = _f64(x_ref)
    o = ipm_options(**options)
    v = np.empty(3 * net.n_in + net.n_out)
    lam = np.empty(net.n_in + net.n_out)
    res = IpmResult()
    _check(lib.nnc_ipm_adversarial_l1(net.handle, _dp(x_ref), int(target), float(conf), ctypes.byref(o),
                                      _dp(v), _dp(lam), ctypes.byref(res)))
    return res.as_dict(), v, lam


def ipm_adversarial_l1_fullspace(net, x_ref, target, conf=0.6, **options):
    """Eq. 7 with the network in the full space (Eq. 4), host functions, sparse derivatives and the
    stage-by-stage KKT factorization.  Returns (result dict, v = (x, p, q, z_1, y_1, ..., z_L, y_L),
    lambda)."""
    lib = load_library()
    x_ref = _f64(x_ref)
    o = ipm_options(**options)
    hidden = sum(net.widths[1:])
    v = np.empty(3 * net.n_in + 2 * hidden)
    lam = np.empty(net.n_in + 2 * hidden)
    res = IpmResult()
    _check(lib.nnc_ipm_adversarial_l1_fullspace(net.handle, _dp(x_ref), int(target), float(conf),
                                                ctypes.byref(o), _dp(v), _dp(lam), ctypes.byref(res)))
    return res.as_dict(), v, lam


def layer_weights(net, layer):
    """(W, b, activation code) of layer `layer` as loaded (FP64 master copy)."""
    lib = load_library()
    act, rows, cols = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.nnc_layer_weights(net.handle, int(layer), None, None, ctypes.byref(act),
                                 ctypes.byref(rows), ctypes.byref(cols)))
    W = np.empty((rows.value, cols.value))
    b = np.empty(rows.value)
    _check(lib.nnc_layer_weights(net.handle, int(layer), _dp(W), _dp(b), None, None, None))
    return W, b, act.value


def selftest_bounded_wait(which, cycles):
    """Runs the bounded-wait self-test; returns (status, recorded wait code)."""
    lib = load_library()
    code = ctypes.c_int()
    st = lib.nnc_selftest_bounded_wait(int(which), int(cycles), ctypes.byref(code))
    return st, code.value


def kkt_solve(WDD, WSS, sigma, AD, AS, rhs, delta_w=0.0, delta_c=0.0):
    """nnc_kkt_solve (host FP64, no device work): returns (solution, (npos, nneg, nzero, full))."""
    lib = load_library()
    nd = WDD.shape[0]
    ns = len(WSS)
    m = AD.shape[0] if AD is not None and AD.size else (AS.shape[0] if AS is not None else 0)
    WDD, WSS, sigma = _f64(WDD), _f64(WSS), _f64(sigma)
    AD = _f64(AD if AD is not None else np.zeros((m, nd)))
    AS = _f64(AS if AS is not None else np.zeros((m, ns)))
    x = _f64(rhs).copy()
    inert = (ctypes.c_int * 4)()
    _check(lib.nnc_kkt_solve(nd, ns, m, _dp(WDD), _dp(WSS), _dp(sigma), _dp(AD), _dp(AS),
                             float(delta_w), float(delta_c), _dp(x), inert))
    return x, tuple(inert)


def stage_kkt_solve(n, m, var_stage, con_stage, W_trip, A_trip, sigma, rhs, delta_w=0.0,
                    delta_c=0.0):
    """nnc_stage_kkt_solve (host FP64): W_trip = (rows, cols, values) of W's lower triangle,
    A_trip = (constraint rows, variable columns, values); returns (solution or None, (npos, nneg,
    nzero))."""
    lib = load_library()
    iv = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    vs, cs = iv(var_stage), iv(con_stage)
    wr, wc, wv = iv(W_trip[0]), iv(W_trip[1]), _f64(W_trip[2])
    jr, jc, jv = iv(A_trip[0]), iv(A_trip[1]), _f64(A_trip[2])
    ip = lambda a: a.ctypes.data_as(_IP)
    x = _f64(rhs).copy()
    inert = (ctypes.c_int * 3)()
    _check(lib.nnc_stage_kkt_solve(int(n), int(m), ip(vs), ip(cs), len(wv), ip(wr), ip(wc), _dp(wv),
                                   len(jv), ip(jr), ip(jc), _dp(jv), _dp(_f64(sigma)),
                                   float(delta_w), float(delta_c), _dp(x), inert))
    return (x if inert[2] == 0 else None), tuple(inert)


def residual_noalloc(widths, acts, W_dev, b_dev, x, y, r, stream=None):
    """nnc_residual_noalloc: r = y - NN(x) in FP64 with caller-owned CUDA float64 tensors only
    (W_dev[l] of shape (d_{l+1}, d_l), b_dev[l] or None); the library allocates nothing."""
    lib = load_library()
    L = len(widths) - 1
    wid = (ctypes.c_int * (L + 1))(*[int(w) for w in widths])
    act = (ctypes.c_int * L)(*[ACTS[a] if isinstance(a, str) else int(a) for a in acts])
    Wp = (_P * L)(*[_tp(w) for w in W_dev])
    bp = (_P * L)(*[_tp(v) for v in b_dev]) if b_dev is not None else None
    _check(lib.nnc_residual_noalloc(L, wid, act, Wp, bp, _tp(x), _tp(y), _tp(r),
                                    stream or _stream_ptr()))


class Batch:
    """nnc_batch: K nets of equal hidden widths (different n_in) evaluated by grouped launches."""

    def __init__(self, nets, stream=None):
        lib = load_library()
        self.nets = list(nets)
        K = len(self.nets)
        hs = (_P * K)(*[n.handle for n in self.nets])
        h = _P()
        _check(lib.nnc_batch_create(ctypes.byref(h), hs, K, stream))
        self._h = h
        k, no, ns, hsum = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _check(lib.nnc_batch_info(h, ctypes.byref(k), ctypes.byref(no), ctypes.byref(ns), ctypes.byref(hsum)))
        self.K, self.n_out, self.n_sum, self.h_sum = k.value, no.value, ns.value, hsum.value
        self.n_in = [n.n_in for n in self.nets]
        self.off = np.concatenate([[0], np.cumsum(self.n_in)[:-1]]).astype(np.int64)
        self.hoff = np.concatenate([[0], np.cumsum(np.square(self.n_in))[:-1]]).astype(np.int64)

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.nnc_batch_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def use_graph(self, enable=True):
        _check(_lib.nnc_batch_use_graph(self._h, int(bool(enable))))

    def tune_set(self, syrk_splits):
        """nnc_batch_tune_set: pin the symmetric product's split-K count."""
        _check(_lib.nnc_batch_tune_set(self._h, int(syrk_splits)))

    def autotune(self, cache_path=None, retune=False):
        """nnc_batch_autotune: (grouped-tangent N tile, symmetric-product splits) chosen by timing."""
        bn, sp = ctypes.c_int(), ctypes.c_int()
        cp = cache_path.encode() if cache_path else None
        _check(_lib.nnc_batch_autotune(self._h, cp, int(bool(retune)), ctypes.byref(bn), ctypes.byref(sp)))
        return bn.value, sp.value

    def tuning(self):
        """nnc_batch_tuning: the symmetric product's split-K count in use."""
        v = ctypes.c_int()
        _check(_lib.nnc_batch_tuning(self._h, ctypes.byref(v)))
        return v.value

    def set_bias(self, layer, bias):
        bias = _f64(bias)
        _check(_lib.nnc_batch_set_bias(self._h, int(layer), _dp(bias)))

    def concat(self, xs):
        return np.concatenate([_f64(x) for x in xs])

    def split_outputs(self, y, J, H, g):
        ys = [y[k * self.n_out:(k + 1) * self.n_out] for k in range(self.K)] if y is not None else None
        Js = [J[self.off[k] * self.n_out:(self.off[k] + self.n_in[k]) * self.n_out].reshape(self.n_out, self.n_in[k])
              for k in range(self.K)] if J is not None else None
        Hs = [H[self.hoff[k]:self.hoff[k] + self.n_in[k] ** 2].reshape(self.n_in[k], self.n_in[k])
              for k in range(self.K)] if H is not None else None
        gs = [g[self.off[k]:self.off[k] + self.n_in[k]] for k in range(self.K)] if g is not None else None
        return ys, Js, Hs, gs

    def eval(self, xs, lams=None, want=("y", "J", "H", "g")):
        x = self.concat(xs)
        lam = self.concat(lams) if lams is not None else None
        y = np.empty(self.K * self.n_out) if "y" in want else None
        J = np.empty(self.n_sum * self.n_out) if "J" in want else None
        H = np.empty(self.h_sum) if ("H" in want and lam is not None) else None
        g = np.empty(self.n_sum) if ("g" in want and lam is not None) else None
        p = lambda a: _dp(a) if a is not None else None  # noqa: E731
        _check(_lib.nnc_batch_eval(self._h, _dp(x), p(lam), p(y), p(J), p(H), p(g)))
        return self.split_outputs(y, J, H, g)

    def residual(self, xs, ys):
        x, y = self.concat(xs), self.concat(ys)
        r = np.empty(self.K * self.n_out)
        _check(_lib.nnc_batch_residual(self._h, _dp(x), _dp(y), _dp(r)))
        return [r[k * self.n_out:(k + 1) * self.n_out] for k in range(self.K)]

    def eval_kkt(self, xs, ys, lams, out=None):
        """nnc_batch_eval_kkt (host arrays): per net the residual y - NN(x), J, H and the gradient
        lambda^T J from one value pass; returns concatenated (r, J, H, g).  xs, ys, lams: lists
        per net, or arrays already concatenated; out: optional concatenated (r, J, H, g) float64
        arrays to fill (for example in pinned host memory)."""
        cat = lambda v: v if isinstance(v, np.ndarray) and v.dtype == np.float64 and v.flags.c_contiguous \
            else self.concat(v)  # noqa: E731
        x, y, lam = cat(xs), cat(ys), cat(lams)
        sizes = (self.K * self.n_out, self.n_sum * self.n_out, self.h_sum, self.n_sum)
        if x.size != self.n_sum or y.size != self.K * self.n_out or lam.size != self.K * self.n_out:
            raise ValueError("eval_kkt: concatenated inputs of the wrong size")
        if out is None:
            out = tuple(np.empty(k) for k in sizes)
        for a, k in zip(out, sizes):
            if a.dtype != np.float64 or a.size != k or not a.flags.c_contiguous:
                raise ValueError("eval_kkt: out arrays must be C-contiguous float64 of the concatenated sizes")
        r, J, H, g = out
        _check(_lib.nnc_batch_eval_kkt(self._h, _ad(x), _ad(y), _ad(lam), _ad(r), _ad(J), _ad(H), _ad(g)))
        return r, J, H, g

    def eval_dev(self, x, lam=None, y=None, J=None, H=None, g=None, stream=None):
        _check(_lib.nnc_batch_eval_dev(self._h, _tp(x), _tp(lam), _tp(y), _tp(J), _tp(H), _tp(g),
                                       stream or _stream_ptr()))

    def residual_dev(self, x, y, r, stream=None):
        _check(_lib.nnc_batch_residual_dev(self._h, _tp(x), _tp(y), _tp(r), stream or _stream_ptr()))

    def eval_kkt_dev(self, x, y, lam, r=None, J=None, H=None, g=None, stream=None):
        """Residual y - NN(x), J, H and gradient of every net from one value pass."""
        _check(_lib.nnc_batch_eval_kkt_dev(self._h, _tp(x), _tp(y), _tp(lam), _tp(r), _tp(J), _tp(H),
                                           _tp(g), stream or _stream_ptr()))


def ipm_scopf(batch, G, subsets, cost, demand, delta, v_start=None, lam_start=None, **options):
    """The SCOPF-shaped problem with the host interior-point driver (include/nnc_ipm.h), cold or
    (with v_start, lam_start) warm-started.  subsets: list of K index arrays S_k.
    Returns (result dict, v = (x, y), lambda)."""
    lib = load_library()
    K = batch.K
    n_in = (ctypes.c_int * K)(*[len(s) for s in subsets])
    sub = np.concatenate([np.asarray(s, dtype=np.int32) for s in subsets]).astype(np.int32)
    subp = sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    cost, delta = _f64(cost), _f64(delta)
    o = ipm_options(**options)
    v = np.empty(G + K)
    lam = np.empty(K + 1)
    res = IpmResult()
    if v_start is None:
        _check(lib.nnc_ipm_scopf(batch.handle, int(G), n_in, subp, _dp(cost), float(demand), _dp(delta),
                                 ctypes.byref(o), _dp(v), _dp(lam), ctypes.byref(res)))
    else:
        vs, ls = _f64(v_start), _f64(lam_start)
        _check(lib.nnc_ipm_scopf_warm(batch.handle, int(G), n_in, subp, _dp(cost), float(demand), _dp(delta),
                                      _dp(vs), _dp(ls), ctypes.byref(o), _dp(v), _dp(lam), ctypes.byref(res)))
    return res.as_dict(), v, lam


class WarmStart:
    """nnc_ws: the warm-start MLP n_in -> h1 -> h2 -> n_out (GELU) trained by the library's kernels."""

    def __init__(self, params, precision="bf16", stream=None):
        lib = load_library()
        self.params0 = [_f64(p) for p in params]
        W1, _, W2, _, W3, _ = self.params0
        self.h1, self.n_in = W1.shape
        self.h2 = W2.shape[0]
        self.n_out = W3.shape[0]
        pp = (_DP * 6)(*[_dp(p) for p in self.params0])
        h = _P()
        _check(lib.nnc_ws_create(ctypes.byref(h), self.n_in, self.h1, self.h2, self.n_out, pp,
                                 PRECISIONS[precision], stream))
        self._h = h

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.nnc_ws_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _shapes(self):
        return [(self.h1, self.n_in), (self.h1,), (self.h2, self.h1), (self.h2,), (self.n_out, self.h2), (self.n_out,)]

    def set_scaling(self, in_mean, in_std, out_mean, out_std):
        a = [_f64(x) for x in (in_mean, in_std, out_mean, out_std)]
        _check(_lib.nnc_ws_set_scaling(self._h, *[_dp(x) for x in a]))

    def loss_grad(self, U, T):
        U, T = _f64(U), _f64(T)
        grads = [np.empty(s) for s in self._shapes()]
        loss = ctypes.c_double()
        gp = (_DP * 6)(*[_dp(g) for g in grads])
        _check(_lib.nnc_ws_loss_grad(self._h, _dp(U), _dp(T), U.shape[0], ctypes.byref(loss), gp))
        return loss.value, grads

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(_lib.nnc_ws_adam_step(self._h, lr, beta1, beta2, eps))

    def train(self, U, T, epochs, batch=64, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0):
        U, T = _f64(U), _f64(T)
        loss = ctypes.c_double()
        _check(_lib.nnc_ws_train(self._h, _dp(U), _dp(T), U.shape[0], int(epochs), int(batch), lr, beta1,
                                 beta2, eps, int(seed), ctypes.byref(loss)))
        return loss.value

    def predict(self, U):
        U = _f64(U)
        P = np.empty((U.shape[0], self.n_out))
        _check(_lib.nnc_ws_predict(self._h, _dp(U), U.shape[0], _dp(P)))
        return P

    def params(self):
        out = [np.empty(s) for s in self._shapes()]
        _check(_lib.nnc_ws_get_params(self._h, (_DP * 6)(*[_dp(o) for o in out])))
        return out
