"""Thin ctypes binding of the C ABI in include/speedup.h (same names).

Argument marshalling only: every step of the estimator runs inside
libspeedup_gb300.so.  Device buffers may be given as torch CUDA tensors or as
raw integer addresses; streams as torch.cuda.Stream, a raw cudaStream_t
integer, or None (the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SU_OK, SU_EINVAL, SU_ENOMEM, SU_ECUDA, SU_ETIMEOUT, SU_ENONFINITE, SU_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
MODELS = {"ho": 0, "aho": 1, "dw": 2, "mpt": 3, "poly": 4, "general": 5}
GENERAL_MAX_P = 18
PRECISIONS = {"fp64": 0, "fp32": 1}
MAX_P, MAX_S = 144, 10

EXPORTS = [
    "su_options_default", "su_last_error", "su_version", "speedup_amplitude",
    "speedup_generate_coeffs", "su_plan_create", "su_plan_destroy", "su_plan_sizes",
    "su_plan_execute", "su_plan_finalize", "speedup_logweights", "speedup_philox_words",
    "su_fma_peak", "speedup_normals", "speedup_amplitude_batch", "su_batch_plan_create",
    "su_batch_plan_destroy", "su_batch_plan_sizes", "su_batch_plan_execute", "su_batch_plan_finalize",
    "speedup_amplitude_noalloc", "su_proposal_create", "su_proposal_destroy", "su_mlp_forward",
    "speedup_amplitude_proposal", "speedup_proposal_logweights", "su_train_options_default",
    "su_mlp_loss_grad", "speedup_train_proposal", "su_autotune", "su_autotune_clear", "su_plan_shape",
    "speedup_evolution_matrix", "su_fault_inject", "su_plan_execute_timed", "su_plan_execute_range",
    "su_plan_create_nd", "speedup_amplitude_nd", "speedup_logweights_nd", "speedup_generate_nd",
    "su_fit_continuum", "speedup_wp", "speedup_wp_nd", "su_batch_plan_shape", "su_batch_autotune",
    "speedup_amplitude_judged", "su_evolution_band_size", "speedup_evolution_band", "speedup_evolution_spectrum",
    "su_plan_kernel", "su_fixed_shape", "su_batch_plan_kernel",
]
JUDGE_REASONS = {0: "plain faster", 1: "proposal faster", 2: "proposal unusable", 3: "plain unusable",
                 4: "pilots disagree"}
MAX_D = 4
MLP_PARAMS = 34178


class SpeedupError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"speedup error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("n_blocks", ctypes.c_int), ("hierarchy", ctypes.c_int),
                ("instance", ctypes.c_uint32), ("width_factor", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("sample0", ctypes.c_int64), ("seg_log2", ctypes.c_int),
                ("rounds", ctypes.c_int), ("kernel", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("seg_log2", ctypes.c_int), ("rounds", ctypes.c_int), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrainOptions(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_int64), ("steps", ctypes.c_int), ("batch_paths", ctypes.c_int),
                ("lr", ctypes.c_double), ("clip_quantile", ctypes.c_double), ("seed", ctypes.c_uint64)]


class Instance(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("T", ctypes.c_double), ("s", ctypes.c_int),
                ("p", ctypes.c_int), ("n_mc", ctypes.c_int64), ("hierarchy", ctypes.c_int),
                ("reserved", ctypes.c_int)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("s", ctypes.c_int), ("hierarchy", ctypes.c_int), ("seg_log2", ctypes.c_int),
                ("ns_per_slice", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Judge(ctypes.Structure):
    _fields_ = [("chosen", ctypes.c_int), ("reason", ctypes.c_int), ("target_rel_err", ctypes.c_double),
                ("pilot_amp", ctypes.c_double * 2), ("pilot_err", ctypes.c_double * 2),
                ("pilot_ess", ctypes.c_double * 2), ("pilot_relvar", ctypes.c_double * 2),
                ("pilot_s", ctypes.c_double * 2), ("t_target", ctypes.c_double * 2), ("z", ctypes.c_double),
                ("run_s", ctypes.c_double)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        d["chosen"] = "proposal" if self.chosen else "plain"
        d["reason"] = JUDGE_REASONS.get(self.reason, str(self.reason))
        return d


class SpectrumInfo(ctypes.Structure):
    _fields_ = [("half_width", ctypes.c_int), ("block", ctypes.c_int), ("iterations", ctypes.c_int),
                ("converged", ctypes.c_int), ("band_bytes", ctypes.c_int64), ("matvecs", ctypes.c_int64),
                ("lower", ctypes.c_double), ("upper", ctypes.c_double), ("band_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("block_matvecs", ctypes.c_int), ("block_matvec_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LevelResult(ctypes.Structure):
    _fields_ = [("amp", ctypes.c_double), ("log_amp", ctypes.c_double), ("err", ctypes.c_double),
                ("rel_err", ctypes.c_double), ("err_naive", ctypes.c_double), ("ess", ctypes.c_double),
                ("max_share", ctypes.c_double), ("n", ctypes.c_int64)]

    def as_dict(self, level):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["level"] = level
        return d


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libspeedup_gb300.so (building it first if asked); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libspeedup_gb300.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    i32, i64, u32, u64, d, vp = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.c_double, ctypes.c_void_p)
    pd = ctypes.POINTER(ctypes.c_double)
    pi = ctypes.POINTER(ctypes.c_int)
    L.su_options_default.argtypes = [ctypes.POINTER(Options)]
    L.su_options_default.restype = None
    L.su_last_error.restype = ctypes.c_char_p
    L.su_version.argtypes = [ctypes.c_char_p, i32]
    L.speedup_amplitude.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                                    ctypes.POINTER(LevelResult)]
    L.speedup_generate_coeffs.argtypes = [i32, pd, i32, i32, d, pd, i32, pi, pi]
    L.su_plan_create.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                                 ctypes.POINTER(vp)]
    L.su_plan_destroy.argtypes = [vp]
    L.su_plan_sizes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), pi, ctypes.POINTER(i64)]
    L.su_plan_execute.argtypes = [vp, vp, vp, vp, pi]
    L.su_plan_finalize.argtypes = [vp, pd, vp, ctypes.POINTER(LevelResult)]
    L.su_plan_shape.argtypes = [vp, pi, pi]
    L.su_plan_kernel.argtypes = [vp, pi]
    L.su_batch_plan_kernel.argtypes = [vp, pi]
    L.su_fixed_shape.argtypes = [i32, pd, i32, i32, pi]
    L.su_autotune.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                              ctypes.POINTER(Tuning), ctypes.POINTER(Tuning), i32, pi]
    L.su_autotune_clear.argtypes = []
    L.speedup_evolution_matrix.argtypes = [i32, pd, i32, i32, d, d, i32, i32, vp, vp]
    L.su_evolution_band_size.argtypes = [d, d, i32, pi, ctypes.POINTER(i64)]
    L.speedup_evolution_band.argtypes = [i32, pd, i32, i32, d, d, i32, i32, vp, i64, vp]
    L.speedup_evolution_spectrum.argtypes = [i32, pd, i32, i32, d, d, i32, i32, i32, pd, pd, vp,
                                             ctypes.POINTER(SpectrumInfo), vp]
    L.su_fault_inject.argtypes = [i32, i64]
    L.su_plan_execute_timed.argtypes = [vp, vp, vp, vp, pi, ctypes.POINTER(ctypes.c_float)]
    L.su_plan_execute_range.argtypes = [vp, i64, i64, vp, vp, vp, pi]
    L.speedup_logweights.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, i64, u64,
                                     ctypes.POINTER(Options), vp]
    L.speedup_philox_words.argtypes = [u64, u32, i64, i64, i32, vp, vp]
    L.su_plan_create_nd.argtypes = [i32, pi, pd, i32, pd, pd, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                                    ctypes.POINTER(vp)]
    L.speedup_amplitude_nd.argtypes = [i32, pi, pd, i32, pd, pd, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                                       ctypes.POINTER(LevelResult)]
    L.speedup_logweights_nd.argtypes = [i32, pi, pd, i32, pd, pd, d, i32, i32, i64, i64, u64,
                                        ctypes.POINTER(Options), vp]
    L.speedup_generate_nd.argtypes = [i32, pi, pd, i32, i32, d, pi, pd, i32, pi]
    L.speedup_wp.argtypes = [i32, pd, i32, i32, d, pd, pd, i64, pd]
    L.speedup_wp_nd.argtypes = [i32, pi, pd, i32, i32, d, pd, pd, i64, pd]
    L.su_fit_continuum.argtypes = [ctypes.POINTER(LevelResult), i32, i32, i32, i32, pd, pd, pd]
    L.su_fma_peak.argtypes = [i32, pd]
    pf = ctypes.POINTER(ctypes.c_float)
    L.su_proposal_create.argtypes = [pf, i32, ctypes.POINTER(vp)]
    L.su_proposal_destroy.argtypes = [vp]
    L.su_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    L.speedup_amplitude_proposal.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                                             vp, ctypes.POINTER(LevelResult)]
    L.speedup_amplitude_judged.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, u64, ctypes.POINTER(Options),
                                           vp, i64, d, ctypes.POINTER(LevelResult), ctypes.POINTER(Judge)]
    L.speedup_proposal_logweights.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, i64, u64,
                                              ctypes.POINTER(Options), vp, vp, vp]
    L.speedup_amplitude_noalloc.argtypes = [i32, pd, i32, d, d, d, i32, i32, i64, u64,
                                            ctypes.POINTER(Options), ctypes.POINTER(LevelResult)]
    L.speedup_normals.argtypes = [u64, u32, i64, i64, i32, i32, vp, vp]
    L.su_train_options_default.argtypes = [ctypes.POINTER(TrainOptions)]
    L.su_train_options_default.restype = None
    L.su_mlp_loss_grad.argtypes = [pf, vp, vp, vp, i64, pd, pf]
    L.speedup_train_proposal.argtypes = [i32, pd, i32, d, d, d, i32, i32, u64, ctypes.POINTER(TrainOptions), pf,
                                         pd]
    pinst = ctypes.POINTER(Instance)
    L.speedup_amplitude_batch.argtypes = [i32, pd, i32, i32, pinst, i64, i64, u64, ctypes.POINTER(Options),
                                          ctypes.POINTER(LevelResult)]
    L.su_batch_plan_create.argtypes = [i32, pd, i32, i32, pinst, i64, i64, u64, ctypes.POINTER(Options),
                                       ctypes.POINTER(vp)]
    L.su_batch_plan_destroy.argtypes = [vp]
    L.su_batch_plan_sizes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64)]
    L.su_batch_plan_shape.argtypes = [vp, i64, pi, pi, pi]
    L.su_batch_autotune.argtypes = [i32, pd, i32, i32, pinst, i64, i64, u64, ctypes.POINTER(Options), i32,
                                    ctypes.POINTER(BatchTuning), i32, pi]
    L.su_batch_plan_execute.argtypes = [vp, vp, vp, vp, pi]
    L.su_batch_plan_finalize.argtypes = [vp, pd, vp, ctypes.POINTER(LevelResult)]
    for name in EXPORTS:
        if name not in ("su_options_default", "su_last_error", "su_train_options_default"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc):
    if rc != SU_OK:
        raise SpeedupError(rc, load().su_last_error().decode())


def general_params(poly=(), gauss=(), sech=(), expo=()):
    """The parameters of the general potential (model "general"):
    poly = (a_0, .., a_d), d <= 8; gauss = up to four (A, beta, c) for
    A e^{-beta (q - c)^2}; sech = up to four (B, alpha, d) for
    B sech^2(alpha (q - d)); expo = up to four (E, kappa, x0) for
    E e^{-kappa (q - x0)}.  33 values without exponential terms, else 45."""
    if len(poly) > 9 or len(gauss) > 4 or len(sech) > 4 or len(expo) > 4:
        raise ValueError("degree <= 8, at most four Gaussian, sech^2 and exponential terms")
    out = [float(v) for v in poly] + [0.0] * (9 - len(poly))
    for terms in ((gauss, sech, expo) if expo else (gauss, sech)):
        for t in terms:
            if len(t) != 3:
                raise ValueError("each Gaussian or sech^2 term has three parameters")
            out += [float(v) for v in t]
        out += [0.0] * (3 * (4 - len(terms)))
    return tuple(out)


def _model(m):
    return MODELS[m] if isinstance(m, str) else int(m)


def _params(params):
    arr = (ctypes.c_double * max(len(params), 1))(*[float(v) for v in params])
    return arr, len(params)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("device buffer must be a tensor or an integer address")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError("stream must be torch.cuda.Stream, int or None")


def options(precision="fp64", n_blocks=64, hierarchy=True, instance=0, width_factor=1.0, stream=None,
            sample0=0, seg_log2=0, rounds=0, kernel="auto"):
    o = Options()
    load().su_options_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.n_blocks = int(n_blocks)
    o.hierarchy = 1 if hierarchy else 0
    o.instance = int(instance)
    o.width_factor = float(width_factor)
    o.stream = _stream(stream)
    o.sample0 = int(sample0)
    o.seg_log2 = int(seg_log2)
    o.rounds = int(rounds)
    o.kernel = {"auto": 0, "generic": 1}[kernel] if isinstance(kernel, str) else int(kernel)
    return o


def su_autotune(model, params, a, b, T, p, s, n_probe, seed, **kw):
    """Time every launch shape on n_probe samples, store the fastest for
    (precision, model, p, s); returns (best, all) as dicts."""
    pr, npar = _params(params)
    o = options(**kw)
    best = Tuning()
    cap = 64
    arr = (Tuning * cap)()
    n = ctypes.c_int(0)
    _check(load().su_autotune(_model(model), pr, npar, a, b, T, p, s, int(n_probe), int(seed), ctypes.byref(o),
                              ctypes.byref(best), arr, cap, ctypes.byref(n)))
    return best.as_dict(), [arr[i].as_dict() for i in range(min(n.value, cap))]


def su_autotune_clear():
    _check(load().su_autotune_clear())


def speedup_evolution_matrix(model, params, p, t, L, n, out, precision="fp64", stream=None):
    """U_ij = Delta A_1^(p)(x_i, x_j; t) on x_i = -L + i Delta into the device
    buffer out (n x n doubles)."""
    pr, npar = _params(params)
    _check(load().speedup_evolution_matrix(_model(model), pr, npar, int(p), float(t), float(L), int(n),
                                           PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                                           _ptr(out), _stream(stream)))


FAULTS = {"clear": 0, "alloc": 1, "table_nan": 2, "queue_stop": 3, "withhold_mma": 4}


def su_evolution_band_size(t, L, n):
    """(half width w, row pitch) of the evolution operator's band storage."""
    w, pitch = ctypes.c_int(0), ctypes.c_int64(0)
    _check(load().su_evolution_band_size(float(t), float(L), int(n), ctypes.byref(w), ctypes.byref(pitch)))
    return w.value, pitch.value


def speedup_evolution_band(model, params, p, t, L, n, out, precision="fp64", stream=None):
    """Upper band of U, diagonal-major, into out (a CUDA tensor of at least
    (w + 1) * pitch doubles): out[k * pitch + i] = U[i, i + k]."""
    pr, npar = _params(params)
    cap = out.numel() * out.element_size() if hasattr(out, "numel") else 1 << 62
    _check(load().speedup_evolution_band(_model(model), pr, npar, p, float(t), float(L), int(n),
                                         PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                                         _ptr(out), int(cap), _stream(stream)))


def speedup_evolution_spectrum(model, params, p, t, L, n, nev, vectors=None, precision="fp64", stream=None):
    """The nev lowest energies of the evolution operator (band eigensolver);
    returns (energies, residuals, info dict); vectors: optional CUDA tensor of
    nev * n doubles for the eigenfunctions."""
    pr, npar = _params(params)
    E = (ctypes.c_double * nev)()
    R = (ctypes.c_double * nev)()
    info = SpectrumInfo()
    _check(load().speedup_evolution_spectrum(_model(model), pr, npar, p, float(t), float(L), int(n),
                                             PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                                             int(nev), E, R, _ptr(vectors), ctypes.byref(info), _stream(stream)))
    return list(E), list(R), info.as_dict()


def su_fault_inject(kind, arg=0):
    """Test support: arm one of the library's fault hooks (see speedup.h)."""
    _check(load().su_fault_inject(FAULTS[kind] if isinstance(kind, str) else int(kind), int(arg)))


def su_version():
    buf = ctypes.create_string_buffer(512)
    _check(load().su_version(buf, 512))
    return buf.value.decode()


def su_last_error():
    return load().su_last_error().decode()


def speedup_amplitude(model, params, a, b, T, p, s, n_mc, seed, **kw):
    """Amplitude and errors for every level n = 0..s (list of dicts)."""
    pr, npar = _params(params)
    out = (LevelResult * (s + 1))()
    o = options(**kw)
    _check(load().speedup_amplitude(_model(model), pr, npar, a, b, T, p, s, int(n_mc), int(seed),
                                    ctypes.byref(o), out))
    return [out[n].as_dict(n) for n in range(s + 1)]


def speedup_amplitude_noalloc(model, params, a, b, T, p, s, n_mc, seed, **kw):
    """speedup_amplitude without device allocation (library-owned static scratch)."""
    pr, npar = _params(params)
    out = (LevelResult * (s + 1))()
    o = options(**kw)
    _check(load().speedup_amplitude_noalloc(_model(model), pr, npar, a, b, T, p, s, int(n_mc), int(seed),
                                            ctypes.byref(o), out))
    return [out[n].as_dict(n) for n in range(s + 1)]


def speedup_generate_coeffs(model, params, p, eps):
    """(P, ncol, ring, lens): W_p = sum_j xb^(2j) sum_i P_ij z^i (see speedup.h)."""
    pr, npar = _params(params)
    cap = 1 << 14
    tab = (ctypes.c_double * cap)()
    shape = (ctypes.c_int * (MAX_P + 2))()
    nt = ctypes.c_int(0)
    _check(load().speedup_generate_coeffs(_model(model), pr, npar, p, eps, tab, cap, shape,
                                          ctypes.byref(nt)))
    ncol = shape[0]
    lens = [shape[2 + j] for j in range(ncol)]
    return np.array(tab[:nt.value]), ncol, shape[1], lens


def su_fixed_shape(model, params, p):
    """Index of the compiled table shape of (model, p), or -1 (host only)."""
    pr, npar = _params(params)
    k = ctypes.c_int(0)
    _check(load().su_fixed_shape(_model(model), pr, npar, int(p), ctypes.byref(k)))
    return k.value


def speedup_logweights(model, params, a, b, T, p, s, sample0, n_samples, seed, out, **kw):
    """Per-sample log-weights into the device buffer out (n_samples x s doubles)."""
    pr, npar = _params(params)
    o = options(**kw)
    _check(load().speedup_logweights(_model(model), pr, npar, a, b, T, p, s, int(sample0), int(n_samples),
                                     int(seed), ctypes.byref(o), _ptr(out)))


def _nd_potential(V):
    """{exponent tuple: coefficient} -> (d, exps, coefs, n_terms) as ctypes arrays."""
    items = [(tuple(int(e) for e in k), float(v)) for k, v in dict(V).items()]
    if not items:
        raise ValueError("the potential needs at least one term")
    d = len(items[0][0])
    if any(len(k) != d for k, _ in items):
        raise ValueError("every exponent tuple needs the same length d")
    exps = (ctypes.c_int * (d * len(items)))(*[e for k, _ in items for e in k])
    coefs = (ctypes.c_double * len(items))(*[v for _, v in items])
    return d, exps, coefs, len(items)


def _vec(x, d):
    x = [float(v) for v in x]
    if len(x) != d:
        raise ValueError(f"endpoints need {d} coordinates")
    return (ctypes.c_double * d)(*x)


def speedup_generate_nd(V, p, eps):
    """W(x, xb; eps) of a system of d coordinates: {(e_x..., e_xb...): coefficient}."""
    d, ex, co, n = _nd_potential(V)
    cap = 1 << 14
    oe = (ctypes.c_int * (cap * 2 * d))()
    ow = (ctypes.c_double * cap)()
    nn = ctypes.c_int(0)
    _check(load().speedup_generate_nd(d, ex, co, n, int(p), float(eps), oe, ow, cap, ctypes.byref(nn)))
    return {tuple(oe[t * 2 * d:(t + 1) * 2 * d]): ow[t] for t in range(nn.value)}


def _points(x, xb, shape_tail=()):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    xb = np.ascontiguousarray(np.asarray(xb, dtype=np.float64))
    if x.shape != xb.shape or x.shape[x.ndim - len(shape_tail):] != shape_tail:
        raise ValueError("x and xb must have the same shape (points x coordinates)")
    return x, xb


def speedup_wp(model, params, p, eps, x, xb):
    """W_p(x, xb; eps) of a one-dimensional model at the points x, xb (host, no device)."""
    pr, npar = _params(params)
    x, xb = _points(x, xb)
    w = np.empty(x.shape)
    pd = ctypes.POINTER(ctypes.c_double)
    _check(load().speedup_wp(_model(model), pr, npar, int(p), float(eps), x.ctypes.data_as(pd),
                             xb.ctypes.data_as(pd), int(x.size), w.ctypes.data_as(pd)))
    return w


def speedup_wp_nd(V, p, eps, x, xb):
    """W(x, xb; eps) of a system of d coordinates at the points x, xb (shape (..., d); host, no device)."""
    d, ex, co, n = _nd_potential(V)
    x, xb = _points(x, xb, (d,))
    w = np.empty(x.shape[:-1])
    pd = ctypes.POINTER(ctypes.c_double)
    _check(load().speedup_wp_nd(d, ex, co, n, int(p), float(eps), x.ctypes.data_as(pd), xb.ctypes.data_as(pd),
                                int(w.size), w.ctypes.data_as(pd)))
    return w


def speedup_amplitude_nd(V, a, b, T, p, s, n_mc, seed, **kw):
    """Amplitude and errors of a system of d coordinates for every level n = 0..s."""
    d, ex, co, n = _nd_potential(V)
    out = (LevelResult * (s + 1))()
    o = options(**kw)
    _check(load().speedup_amplitude_nd(d, ex, co, n, _vec(a, d), _vec(b, d), T, p, s, int(n_mc), int(seed),
                                       ctypes.byref(o), out))
    return [out[k].as_dict(k) for k in range(s + 1)]


def speedup_logweights_nd(V, a, b, T, p, s, sample0, n_samples, seed, out, **kw):
    """Per-sample log-weights of a system of d coordinates into the device buffer out (n_samples x s)."""
    d, ex, co, n = _nd_potential(V)
    o = options(**kw)
    _check(load().speedup_logweights_nd(d, ex, co, n, _vec(a, d), _vec(b, d), T, p, s, int(sample0),
                                        int(n_samples), int(seed), ctypes.byref(o), _ptr(out)))


def su_fit_continuum(levels, p, n_min=1, n_terms=3):
    """(A, A_err, chi2) of Eq. fit from a list of level results (dicts as
    speedup_amplitude returns them, levels 0..s)."""
    s = len(levels) - 1
    arr = (LevelResult * (s + 1))()
    for n, r in enumerate(levels):
        for k, _ in LevelResult._fields_:
            if k in r:
                setattr(arr[n], k, r[k])
    a, da, c2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().su_fit_continuum(arr, s, int(p), int(n_min), int(n_terms), ctypes.byref(a), ctypes.byref(da),
                                   ctypes.byref(c2)))
    return a.value, da.value, c2.value


def speedup_normals(seed, instance, sample0, n_samples, n_normals, out, precision="fp64", stream=None):
    """The sampler's normals into the device buffer out (n_samples x n_normals doubles)."""
    _check(load().speedup_normals(int(seed), int(instance), int(sample0), int(n_samples), int(n_normals),
                                  PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                                  _ptr(out), _stream(stream)))


def speedup_philox_words(seed, instance, sample0, n_samples, n_calls, out, stream=None):
    _check(load().speedup_philox_words(int(seed), int(instance), int(sample0), int(n_samples),
                                       int(n_calls), _ptr(out), _stream(stream)))


def su_fma_peak(precision="fp64"):
    """Measured multiply-adds per second of the current device."""
    v = ctypes.c_double(0)
    _check(load().su_fma_peak(PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                              ctypes.byref(v)))
    return v.value


def _instances(instances):
    """Instances as tuples (a, b, T, s[, p[, n_mc[, hierarchy]]]) or dicts with
    those keys; p = 0 and n_mc = 0 take the batch's values."""
    n = len(instances)
    arr = (Instance * max(n, 1))()
    for i, x in enumerate(instances):
        if isinstance(x, dict):
            x = (x["a"], x["b"], x["T"], x["s"], x.get("p", 0), x.get("n_mc", 0), x.get("hierarchy", 0))
        x = tuple(x) + (0,) * (7 - len(x))
        a, b, T, s, p, n_mc, hier = x
        arr[i].a, arr[i].b, arr[i].T, arr[i].s = float(a), float(b), float(T), int(s)
        arr[i].p, arr[i].n_mc, arr[i].hierarchy = int(p), int(n_mc), 1 if hier else 0
    return arr, n


def _batch_results(out, arr, n):
    """Per instance: its top-level result (a dict), or with hierarchy the list
    of its s + 1 levels."""
    res, k = [], 0
    for i in range(n):
        s = arr[i].s
        if arr[i].hierarchy:
            res.append([out[k + lev].as_dict(lev) for lev in range(s + 1)])
            k += s + 1
        else:
            res.append(out[k].as_dict(s))
            k += 1
    return res


def speedup_amplitude_batch(model, params, p, instances, n_mc, seed, **kw):
    """Amplitude of every instance (see _instances): a dict of its top level,
    or the list of its levels where the instance asks for the hierarchy."""
    pr, npar = _params(params)
    arr, n = _instances(instances)
    n_out = sum(arr[i].s + 1 if arr[i].hierarchy else 1 for i in range(n))
    out = (LevelResult * max(n_out, 1))()
    o = options(**kw)
    _check(load().speedup_amplitude_batch(_model(model), pr, npar, p, arr, n, int(n_mc), int(seed),
                                          ctypes.byref(o), out))
    return _batch_results(out, arr, n)


def su_batch_autotune(model, params, p, instances, n_mc, seed, max_probe=64, **kw):
    """Time every register segment per (p, s, hierarchy) class of the batch on
    its first max_probe instances and store the fastest; returns the chosen
    shapes (list of dicts)."""
    pr, npar = _params(params)
    arr, n = _instances(instances)
    cap = 256
    best = (BatchTuning * cap)()
    nb = ctypes.c_int(0)
    o = options(**kw)
    _check(load().su_batch_autotune(_model(model), pr, npar, p, arr, n, int(n_mc), int(seed), ctypes.byref(o),
                                    int(max_probe), best, cap, ctypes.byref(nb)))
    return [best[i].as_dict() for i in range(min(nb.value, cap))]


class BatchPlan:
    """su_batch_plan_create / _execute / _finalize / _destroy."""

    def __init__(self, model, params, p, instances, n_mc, seed, **kw):
        pr, npar = _params(params)
        arr, n = _instances(instances)
        self._arr = arr
        self.n_inst = n
        o = options(**kw)
        h = ctypes.c_void_p()
        _check(load().su_batch_plan_create(_model(model), pr, npar, p, arr, n, int(n_mc), int(seed),
                                           ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        tb, sb, sa, nr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().su_batch_plan_sizes(h, ctypes.byref(tb), ctypes.byref(sb), ctypes.byref(sa),
                                          ctypes.byref(nr)))
        self.tuple_bytes, self.scratch_bytes, self.slice_actions = tb.value, sb.value, sa.value
        self.n_results = nr.value

    def su_batch_plan_shape(self, i):
        """(seg_log2, chunks per block, 1 if from su_batch_autotune else 0) of instance i."""
        f, k, fr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(load().su_batch_plan_shape(self._h, int(i), ctypes.byref(f), ctypes.byref(k), ctypes.byref(fr)))
        return f.value, k.value, fr.value

    def su_batch_plan_kernel(self):
        """Index of the table shape compiled into the batched kernel, or -1."""
        k = ctypes.c_int(0)
        _check(load().su_batch_plan_kernel(self._h, ctypes.byref(k)))
        return k.value

    def su_batch_plan_execute(self, d_tuples, d_scratch, stream=None):
        n = ctypes.c_int(0)
        _check(load().su_batch_plan_execute(self._h, _ptr(d_tuples), _ptr(d_scratch), _stream(stream),
                                            ctypes.byref(n)))
        return n.value

    def su_batch_plan_finalize(self, h_tuples, d_scratch=None):
        out = (LevelResult * max(self.n_results, 1))()
        arr = np.ascontiguousarray(h_tuples, dtype=np.float64)
        _check(load().su_batch_plan_finalize(self._h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             _ptr(d_scratch), out))
        return _batch_results(out, self._arr, self.n_inst)

    def close(self):
        if getattr(self, "_h", None):
            load().su_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Proposal:
    """A network uploaded for the learned proposal (su_proposal_create)."""

    def __init__(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != MLP_PARAMS:
            raise ValueError(f"the network has {MLP_PARAMS} parameters")
        h = ctypes.c_void_p()
        _check(load().su_proposal_create(th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), th.size,
                                         ctypes.byref(h)))
        self._h = h

    def su_mlp_forward(self, X, Y, stream=None):
        n = X.shape[0] if hasattr(X, "shape") else None
        _check(load().su_mlp_forward(self._h, _ptr(X), int(n), _ptr(Y), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().su_proposal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def speedup_amplitude_proposal(model, params, a, b, T, p, s, n_mc, seed, proposal, **kw):
    pr, npar = _params(params)
    out = (LevelResult * (s + 1))()
    kw.setdefault("precision", "fp32")
    o = options(**kw)
    _check(load().speedup_amplitude_proposal(_model(model), pr, npar, a, b, T, p, s, int(n_mc), int(seed),
                                             ctypes.byref(o), proposal._h, out))
    return [out[n].as_dict(n) for n in range(s + 1)]


def speedup_amplitude_judged(model, params, a, b, T, p, s, n_mc, seed, proposal, n_pilot=200_000,
                             target_rel_err=1e-4, **kw):
    """The proposal judged against the plain sampler on two pilots and used
    only where confirmed and faster; returns (levels, judge dict)."""
    pr, npar = _params(params)
    out = (LevelResult * (s + 1))()
    j = Judge()
    kw.setdefault("precision", "fp32")
    o = options(**kw)
    _check(load().speedup_amplitude_judged(_model(model), pr, npar, a, b, T, p, s, int(n_mc), int(seed),
                                           ctypes.byref(o), proposal._h, int(n_pilot), float(target_rel_err), out,
                                           ctypes.byref(j)))
    return [out[n].as_dict(n) for n in range(s + 1)], j.as_dict()


def speedup_proposal_logweights(model, params, a, b, T, p, s, sample0, n_samples, seed, proposal, out,
                                outs=None, **kw):
    pr, npar = _params(params)
    kw.setdefault("precision", "fp32")
    o = options(**kw)
    _check(load().speedup_proposal_logweights(_model(model), pr, npar, a, b, T, p, s, int(sample0),
                                              int(n_samples), int(seed), ctypes.byref(o), proposal._h,
                                              _ptr(out), _ptr(outs)))


def su_mlp_loss_grad(theta, X, u, rw):
    """(loss, flat gradient) of the rows X (n x 6), u, rw given as CUDA tensors."""
    th = np.ascontiguousarray(theta, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_double(0)
    pf = ctypes.POINTER(ctypes.c_float)
    _check(load().su_mlp_loss_grad(th.ctypes.data_as(pf), _ptr(X), _ptr(u), _ptr(rw), int(X.shape[0]),
                                   ctypes.byref(loss), g.ctypes.data_as(pf)))
    return loss.value, g


def speedup_train_proposal(model, params, a, b, T, p, s, seed, theta, n_train=None, steps=None, batch_paths=None,
                           lr=None, clip_quantile=None, train_seed=None):
    """Train the proposal network; returns (trained theta, per-step losses)."""
    to = TrainOptions()
    load().su_train_options_default(ctypes.byref(to))
    for k, v in (("n_train", n_train), ("steps", steps), ("batch_paths", batch_paths), ("lr", lr),
                 ("clip_quantile", clip_quantile), ("seed", train_seed)):
        if v is not None:
            setattr(to, k, v)
    th = np.array(theta, dtype=np.float32, copy=True)
    losses = np.zeros(to.steps, dtype=np.float64)
    pr, npar = _params(params)
    pf = ctypes.POINTER(ctypes.c_float)
    _check(load().speedup_train_proposal(_model(model), pr, npar, a, b, T, p, s, int(seed), ctypes.byref(to),
                                         th.ctypes.data_as(pf), losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return th, losses


class Plan:
    """su_plan_create / su_plan_execute / su_plan_finalize / su_plan_destroy."""

    def __init__(self, model, params, a, b, T, p, s, n_mc, seed, **kw):
        self.s = s
        pr, npar = _params(params)
        o = options(**kw)
        h = ctypes.c_void_p()
        _check(load().su_plan_create(_model(model), pr, npar, a, b, T, p, s, int(n_mc), int(seed),
                                     ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        tb, sb, lv, sa = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        _check(load().su_plan_sizes(h, ctypes.byref(tb), ctypes.byref(sb), ctypes.byref(lv),
                                    ctypes.byref(sa)))
        self.tuple_bytes, self.scratch_bytes = tb.value, sb.value
        self.levels, self.slice_actions = lv.value, sa.value

    def su_plan_shape(self):
        """(seg_log2, rounds) of this plan's launch."""
        f, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().su_plan_shape(self._h, ctypes.byref(f), ctypes.byref(r)))
        return f.value, r.value

    def su_plan_kernel(self):
        """Index of the table shape compiled into the sampler this plan
        launches, or -1 for the generic sampler."""
        k = ctypes.c_int(0)
        _check(load().su_plan_kernel(self._h, ctypes.byref(k)))
        return k.value

    def su_plan_execute_range(self, b0, b1, d_tuples, d_scratch, stream=None):
        """Sample error blocks [b0, b1) only (checkpoint / resume); returns launches."""
        n = ctypes.c_int(0)
        _check(load().su_plan_execute_range(self._h, int(b0), int(b1), _ptr(d_tuples), _ptr(d_scratch),
                                            _stream(stream), ctypes.byref(n)))
        return n.value

    def su_plan_execute_timed(self, d_tuples, d_scratch, stream=None):
        """Launch and time on the device; returns (launches, milliseconds)."""
        n, ms = ctypes.c_int(0), ctypes.c_float(0)
        _check(load().su_plan_execute_timed(self._h, _ptr(d_tuples), _ptr(d_scratch), _stream(stream),
                                            ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def su_plan_execute(self, d_tuples, d_scratch, stream=None):
        """Launch; returns the number of kernel launches made."""
        n = ctypes.c_int(0)
        _check(load().su_plan_execute(self._h, _ptr(d_tuples), _ptr(d_scratch), _stream(stream),
                                      ctypes.byref(n)))
        return n.value

    def su_plan_finalize(self, h_tuples, d_scratch=None):
        out = (LevelResult * (self.s + 1))()
        arr = np.ascontiguousarray(h_tuples, dtype=np.float64)
        _check(load().su_plan_finalize(self._h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       _ptr(d_scratch), out))
        return [out[n].as_dict(n) for n in range(self.s + 1)]

    def close(self):
        if getattr(self, "_h", None):
            load().su_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlanND(Plan):
    """su_plan_create_nd: a plan for a system of d coordinates (potential
    {exponent tuple: coefficient}, endpoint vectors a and b); executed and
    finalized like Plan."""

    def __init__(self, V, a, b, T, p, s, n_mc, seed, **kw):
        self.s = s
        d, ex, co, n = _nd_potential(V)
        o = options(**kw)
        h = ctypes.c_void_p()
        _check(load().su_plan_create_nd(d, ex, co, n, _vec(a, d), _vec(b, d), T, p, s, int(n_mc), int(seed),
                                        ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        tb, sb, lv, sa = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        _check(load().su_plan_sizes(h, ctypes.byref(tb), ctypes.byref(sb), ctypes.byref(lv),
                                    ctypes.byref(sa)))
        self.tuple_bytes, self.scratch_bytes = tb.value, sb.value
        self.levels, self.slice_actions = lv.value, sa.value
