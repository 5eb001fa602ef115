"""Python binding of libgbk.so (the C ABI in include/gbk.h).

Argument marshalling only: every step of the forward model runs in the
library's CUDA kernels.  Device buffers are torch tensors; the stream is
torch's current stream unless one is given.  If the shared library has not
been built this module raises -- there is no CPU fallback.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbk.so")

NPAR = 10
GBK_OK, GBK_EINVAL, GBK_ECUDA, GBK_EWORKSPACE, GBK_EUNSUPPORTED = 0, 1, 2, 3, 4
PATH_AUTO, PATH_FUSED, PATH_STAGED, PATH_SPLIT = 0, 1, 2, 3
MODEL_CUBE, MODEL_VFIELD_ARCTAN, MODEL_VFIELD_EPINAT = 0, 1, 2
JAC_FD_FORWARD, JAC_FD_CENTRAL, JAC_TANGENT = 0, 1, 2
LM_BATCHED, LM_PLAIN = 0, 1
FIT_STATUS = {0: "running", 1: "ftol", 2: "xtol", 3: "maxiter", 4: "lambda", 5: "nonfinite"}


class GbkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gbk status %d: %s" % (status, msg))
        self.status = status


class CGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("upsample", ctypes.c_int32), ("dv", ctypes.c_double), ("vc", ctypes.c_double),
                ("psf_fwhm", ctypes.c_double), ("lsf_fwhm", ctypes.c_double),
                ("lsf_mode", ctypes.c_int32), ("model", ctypes.c_int32),
                ("halo_sigmas", ctypes.c_double)]


class CTuning(ctypes.Structure):
    _fields_ = [("cluster_ctas", ctypes.c_int32), ("threads", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("ms", ctypes.c_float), ("candidates", ctypes.c_int32)]


class CLmOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("jacobian", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("free_mask", ctypes.c_uint32), ("ftol", ctypes.c_double), ("xtol", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("fd_step", ctypes.c_double * 10), ("path", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class CNsOpts(ctypes.Structure):
    _fields_ = [("n_live", ctypes.c_int32), ("batch", ctypes.c_int32), ("tol", ctypes.c_double),
                ("efr", ctypes.c_double), ("seed", ctypes.c_uint64), ("max_iter", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class CNsTrace(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("n_iter", ctypes.c_int32), ("live0", ctypes.c_void_p),
                ("live0_chi2", ctypes.c_void_p), ("n_props", ctypes.c_void_p), ("props", ctypes.c_void_p),
                ("chi2", ctypes.c_void_p), ("replaced", ctypes.c_void_p)]


class CObs(ctypes.Structure):
    _fields_ = [("v_obs", ctypes.c_void_p), ("s_obs", ctypes.c_void_p), ("w_v", ctypes.c_void_p),
                ("w_s", ctypes.c_void_p), ("mask", ctypes.c_void_p)]


_lib = None


def lib():
    """The loaded libgbk.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgbk.so is not built (run paper_1510_01815_gb300/build.py or "
                               "__graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t
        gp, op = ctypes.POINTER(CGeom), ctypes.POINTER(CObs)
        sig = {
            "gbk_workspace_bytes": (sz, [gp, i32, u32]),
            "gbk_eval_cubes": (i32, [gp, i32, vp, vp, vp, vp, sz, vp]),
            "gbk_chi2": (i32, [gp, i32, vp, op, vp, vp, u32, vp, sz, vp]),
            "gbk_chi2_from_maps": (i32, [i32, i32, i32, vp, op, vp, vp, vp]),
            "gbk_chi2_stage_times": (i32, [gp, i32, vp, op, vp, vp, sz, ctypes.POINTER(ctypes.c_float), vp]),
            "gbk_split_stage_times": (i32, [gp, i32, vp, op, vp, vp, sz, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_int32), vp]),
            "gbk_chi2_noalloc": (i32, [gp, i32, vp, op, vp, vp, vp]),
            "gbk_chi2_host_workspace_bytes": (sz, [gp, i32]),
            "gbk_chi2_host": (i32, [gp, i32, vp, op, vp, vp, sz, vp]),
            "gbk_measure_alu_peak": (i32, [ctypes.POINTER(ctypes.c_double)] * 3 + [vp]),
            "gbk_autotune": (i32, [gp, i32, vp, op, vp, ctypes.POINTER(CTuning), vp]),
            "gbk_get_tuning": (i32, [gp, ctypes.POINTER(CTuning)]),
            "gbk_set_tuning": (i32, [gp, ctypes.POINTER(CTuning)]),
            "gbk_fit_lm_workspace_bytes": (sz, [gp, i32, ctypes.POINTER(CLmOpts)]),
            "gbk_fit_lm": (i32, [gp, i32, vp, vp, vp, vp, ctypes.POINTER(CLmOpts), vp, vp, vp, vp, sz, vp]),
            "gbk_fit_lm_fallback_workspace_bytes": (sz, [gp, i32, ctypes.POINTER(CLmOpts)]),
            "gbk_wait_selfcheck": (i32, [ctypes.c_int64, i32, ctypes.POINTER(ctypes.c_int64), vp]),
            "gbk_fit_lm_fallback": (i32, [gp, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(CLmOpts), vp, vp, vp, vp,
                                          vp, sz, vp]),
            "gbk_jacobian": (i32, [gp, i32, vp, op, u32, vp, vp, vp, vp, vp, vp]),
            "gbk_jacobian_workspace_bytes": (sz, [gp, i32, u32]),
            "gbk_jacobian_ws": (i32, [gp, i32, vp, op, u32, vp, vp, vp, vp, vp, sz, vp]),
            "gbk_grid_workspace_bytes": (sz, [gp, ctypes.POINTER(ctypes.c_int32), i32]),
            "gbk_grid": (i32, [gp, op, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), i32, i32,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_double), vp, sz, vp]),
            "gbk_nested_sample_workspace_bytes": (sz, [gp, ctypes.POINTER(CNsOpts)]),
            "gbk_nested_sample": (i32, [gp, op, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(CNsOpts), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), vp, sz, vp]),
            "gbk_nested_sample_traced": (i32, [gp, op, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(CNsOpts),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_int32), vp, sz, vp,
                                               ctypes.POINTER(CNsTrace)]),
            "gbk_survey_workspace_bytes": (sz, [gp, i32, ctypes.POINTER(CLmOpts)]),
            "gbk_survey_eval": (i32, [gp, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
            "gbk_survey_fit_lm": (i32, [gp, i32, vp, vp, vp, vp, ctypes.POINTER(CLmOpts), vp, vp, vp, vp, sz,
                                        vp]),
            "gbk_survey_jacobian_workspace_bytes": (sz, [gp, i32, u32]),
            "gbk_survey_jacobian": (i32, [gp, i32, vp, vp, u32, vp, vp, vp, vp, sz, vp]),
            "gbk_initial_guess": (i32, [gp, i32, vp, vp, vp, vp, vp]),
            "gbk_survey_autotune": (i32, [gp, i32, vp, vp, vp, vp, sz, ctypes.POINTER(CTuning), vp]),
            "gbk_survey_get_tuning": (i32, [gp, i32, ctypes.POINTER(CTuning)]),
            "gbk_survey_set_tuning": (i32, [gp, i32, ctypes.POINTER(CTuning)]),
            "gbk_device_status": (i32, [ctypes.POINTER(ctypes.c_int32)]),
            "gbk_cnn_param_count": (sz, []),
            "gbk_cnn_workspace_bytes": (sz, [i32]),
            "gbk_cnn_init": (i32, [vp, ctypes.c_uint64, vp]),
            "gbk_cnn_targets": (i32, [i32, vp, vp, vp]),
            "gbk_cnn_decode": (i32, [i32, vp, vp, vp]),
            "gbk_cnn_synth_obs": (i32, [i32, vp, ctypes.c_uint64, ctypes.c_float, ctypes.c_float, vp, vp, vp, vp]),
            "gbk_cnn_forward": (i32, [vp, i32, vp, vp, vp, vp, vp, sz, vp]),
            "gbk_cnn_grad": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
            "gbk_cnn_train_step": (i32, [vp, vp, vp, i32, ctypes.c_float, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
            "gbk_gemm_bf16": (i32, [i32, i32, i32, vp, i32, vp, i32, vp, i32, vp, i32, ctypes.c_float, vp, vp, i32,
                                    vp]),
            "gbk_last_error": (ctypes.c_char_p, []),
            "gbk_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return ["gbk_workspace_bytes", "gbk_eval_cubes", "gbk_chi2", "gbk_chi2_from_maps", "gbk_chi2_stage_times", "gbk_split_stage_times",
            "gbk_chi2_noalloc", "gbk_chi2_host_workspace_bytes", "gbk_chi2_host",
            "gbk_measure_alu_peak", "gbk_autotune", "gbk_get_tuning", "gbk_set_tuning",
            "gbk_fit_lm_workspace_bytes", "gbk_fit_lm", "gbk_fit_lm_fallback_workspace_bytes", "gbk_fit_lm_fallback",
            "gbk_wait_selfcheck",
            "gbk_jacobian", "gbk_jacobian_workspace_bytes", "gbk_jacobian_ws", "gbk_grid_workspace_bytes",
            "gbk_grid",
            "gbk_nested_sample_workspace_bytes", "gbk_nested_sample", "gbk_nested_sample_traced",
            "gbk_survey_workspace_bytes",
            "gbk_survey_eval", "gbk_survey_fit_lm", "gbk_survey_jacobian_workspace_bytes", "gbk_survey_jacobian",
            "gbk_initial_guess", "gbk_survey_autotune", "gbk_survey_get_tuning",
            "gbk_survey_set_tuning", "gbk_device_status", "gbk_gemm_bf16", "gbk_cnn_param_count",
            "gbk_cnn_workspace_bytes", "gbk_cnn_init", "gbk_cnn_targets", "gbk_cnn_decode", "gbk_cnn_synth_obs",
            "gbk_cnn_forward", "gbk_cnn_grad", "gbk_cnn_train_step",
            "gbk_last_error", "gbk_version"]


def cgeom(g):
    """A gbk_geom from any object with the Geometry attributes."""
    return CGeom(int(g.nx), int(g.ny), int(g.nz), int(getattr(g, "upsample", 1)), float(g.dv),
                 float(getattr(g, "vc", 0.0)), float(getattr(g, "psf_fwhm", 0.0)),
                 float(getattr(g, "lsf_fwhm", 0.0)), int(getattr(g, "lsf_mode", 0)), int(getattr(g, "model", 0)),
                 float(getattr(g, "halo_sigmas", 4.0)))


def _check(status):
    if status != GBK_OK:
        raise GbkError(status, lib().gbk_last_error().decode())


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Obs:
    """Observed maps of one galaxy as device tensors ([ny][nx]; mask uint8)."""

    def __init__(self, v_obs, s_obs, w_v, w_s, mask):
        self.v_obs, self.s_obs, self.w_v, self.w_s, self.mask = v_obs, s_obs, w_v, w_s, mask
        self._c = CObs(_ptr(v_obs, torch.float32, "v_obs"), _ptr(s_obs, torch.float32, "s_obs"),
                       _ptr(w_v, torch.float32, "w_v"), _ptr(w_s, torch.float32, "w_s"),
                       _ptr(mask, torch.uint8, "mask"))

    @classmethod
    def from_numpy(cls, v, s, w_v, w_s, mask, device="cuda"):
        f = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        return cls(f(v), f(s), f(w_v), f(w_s),
                   torch.as_tensor(mask, dtype=torch.uint8).contiguous().to(device))

    def c(self):
        return self._c


def gbk_workspace_bytes(geom, n_models, flags=PATH_AUTO):
    g = cgeom(geom)
    n = lib().gbk_workspace_bytes(ctypes.byref(g), int(n_models), int(flags))
    err = lib().gbk_last_error().decode()
    if n == 0 and err:
        raise GbkError(GBK_EINVAL, err)
    return int(n)


def gbk_eval_cubes(geom, params, cubes=None, maps=None, workspace=None, stream=None):
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_eval_cubes(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"),
                                _ptr(cubes, torch.float32, "cubes"), _ptr(maps, torch.float32, "maps"),
                                _ptr(workspace, None, "workspace"), ws_bytes, _stream(stream)))


def gbk_chi2(geom, params, obs, chi2, resid=None, flags=PATH_AUTO, workspace=None, stream=None):
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_chi2(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"),
                          ctypes.byref(obs.c()), _ptr(chi2, torch.float64, "chi2"),
                          _ptr(resid, torch.float32, "resid"), int(flags),
                          _ptr(workspace, None, "workspace"), ws_bytes, _stream(stream)))


def gbk_split_stage_times(geom, params, obs, chi2, workspace, stream=None):
    """gbk_chi2 on the split path, timed per stage; returns ([set-up, line
    stage, PSF/moments stage] milliseconds, kernel launches)."""
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ms = (ctypes.c_float * 3)()
    nl = ctypes.c_int32()
    _check(lib().gbk_split_stage_times(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"),
                                       ctypes.byref(obs.c()), _ptr(chi2, torch.float64, "chi2"),
                                       _ptr(workspace, None, "workspace"), ws_bytes, ms, ctypes.byref(nl),
                                       _stream(stream)))
    return [float(v) for v in ms], nl.value


def gbk_chi2_stage_times(geom, params, obs, chi2, workspace, stream=None):
    """gbk_chi2 on the staged path, timed per stage; returns the
    milliseconds of (model cube, convolution, down-sampling, moments + chi2)."""
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ms = (ctypes.c_float * 4)()
    _check(lib().gbk_chi2_stage_times(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"),
                                      ctypes.byref(obs.c()), _ptr(chi2, torch.float64, "chi2"),
                                      _ptr(workspace, None, "workspace"), ws_bytes, ms, _stream(stream)))
    return [float(v) for v in ms]


def gbk_chi2_noalloc(geom, params, obs, chi2, resid=None, stream=None):
    """gbk_chi2 on the staged path using the library's built-in scratch
    instead of a caller workspace (for callers that cannot allocate)."""
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    _check(lib().gbk_chi2_noalloc(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"),
                                  ctypes.byref(obs.c()), _ptr(chi2, torch.float64, "chi2"),
                                  _ptr(resid, torch.float32, "resid"), _stream(stream)))


def gbk_chi2_host_workspace_bytes(geom, n_models):
    g = cgeom(geom)
    n = lib().gbk_chi2_host_workspace_bytes(ctypes.byref(g), int(n_models))
    err = lib().gbk_last_error().decode()
    if n == 0 and err:
        raise GbkError(GBK_EUNSUPPORTED if "serve" in err else GBK_EINVAL, err)
    return int(n)


def gbk_chi2_host(geom, params, obs, chi2, workspace, stream=None):
    """chi2 with parameters, maps (an Obs of host tensors) and result in host
    memory; the copies run inside the call (gbk_chi2_host)."""
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().gbk_chi2_host(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"), ctypes.byref(obs.c()),
                               _ptr(chi2, torch.float64, "chi2"), _ptr(workspace, None, "workspace"), ws_bytes,
                               _stream(stream)))


def gbk_chi2_from_maps(maps, obs, chi2, resid=None, stream=None):
    n, three, ny, nx = maps.shape
    _check(lib().gbk_chi2_from_maps(int(nx), int(ny), int(n), _ptr(maps, torch.float32, "maps"),
                                    ctypes.byref(obs.c()), _ptr(chi2, torch.float64, "chi2"),
                                    _ptr(resid, torch.float32, "resid"), _stream(stream)))


def gbk_measure_alu_peak(stream=None):
    """(scalar FFMA, packed f32x2 FMA, MUFU ex2) lane operations per second
    on the current device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().gbk_measure_alu_peak(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream(stream)))
    return a.value, b.value, c.value


def gbk_autotune(geom, params, obs, chi2_scratch, stream=None):
    """Times the fused-path tunings on this batch and keeps the fastest for
    the geometry; returns a dict of the choice."""
    g = cgeom(geom)
    n = params.shape[0] if params.dim() == 2 else params.numel() // NPAR
    t = CTuning()
    _check(lib().gbk_autotune(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"),
                              ctypes.byref(obs.c()), _ptr(chi2_scratch, torch.float64, "chi2_scratch"),
                              ctypes.byref(t), _stream(stream)))
    return {"cluster_ctas": t.cluster_ctas, "threads": t.threads, "persistent": t.persistent, "ms": t.ms,
            "candidates": t.candidates}


def gbk_get_tuning(geom):
    g = cgeom(geom)
    t = CTuning()
    _check(lib().gbk_get_tuning(ctypes.byref(g), ctypes.byref(t)))
    return {"cluster_ctas": t.cluster_ctas, "threads": t.threads, "persistent": t.persistent}


def gbk_set_tuning(geom, cluster_ctas=None, threads=None, persistent=0):
    """Forces a tuning for the geometry (None forgets it)."""
    g = cgeom(geom)
    if cluster_ctas is None:
        _check(lib().gbk_set_tuning(ctypes.byref(g), None))
        return
    t = CTuning(int(cluster_ctas), int(threads), int(persistent), 0.0, 0)
    _check(lib().gbk_set_tuning(ctypes.byref(g), ctypes.byref(t)))


def lm_opts(max_iter=200, jacobian=JAC_FD_FORWARD, mode=LM_BATCHED, free=(0, 1, 2, 3, 4, 5, 6, 7),
            ftol=1e-10, xtol=1e-10, lambda0=1e-3, fd_step=0.1, path=PATH_AUTO):
    """Options of gbk_fit_lm; fd_step is a scalar or ten values; path picks
    the batched mode's kernels (PATH_AUTO, PATH_SPLIT or PATH_FUSED)."""
    steps = [float(fd_step)] * NPAR if the_scalar(fd_step) else [float(v) for v in fd_step]
    mask = 0
    for k in free:
        mask |= 1 << int(k)
    return CLmOpts(int(max_iter), int(jacobian), int(mode), mask, float(ftol), float(xtol), float(lambda0),
                   (ctypes.c_double * 10)(*steps), int(path), 0)


def the_scalar(v):
    return not hasattr(v, "__len__")


def obs_array(obs_list, device="cuda"):
    """Device array of gbk_obs structs for gbk_fit_lm (keeps the tensors alive
    through the returned tuple)."""
    arr = (CObs * len(obs_list))(*[o.c() for o in obs_list])
    raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(device)
    return raw, obs_list


def gbk_fit_lm_workspace_bytes(geom, n_gal, opts):
    g = cgeom(geom)
    n = lib().gbk_fit_lm_workspace_bytes(ctypes.byref(g), int(n_gal), ctypes.byref(opts))
    err = lib().gbk_last_error().decode()
    if n == 0 and err:
        raise GbkError(GBK_EINVAL, err)
    return int(n)


def gbk_fit_lm(geom, obs_dev, lo, hi, params, opts, chi2_out, iters_out, status_out, workspace, stream=None):
    g = cgeom(geom)
    n = params.shape[0]
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_fit_lm(ctypes.byref(g), int(n), _ptr(obs_dev, torch.uint8, "obs"),
                            _ptr(lo, torch.float64, "lo"), _ptr(hi, torch.float64, "hi"),
                            _ptr(params, torch.float64, "params"), ctypes.byref(opts),
                            _ptr(chi2_out, torch.float64, "chi2_out"), _ptr(iters_out, torch.int32, "iters_out"),
                            _ptr(status_out, torch.int32, "status_out"), _ptr(workspace, None, "workspace"),
                            ws_bytes, _stream(stream)))


def fit_lm(geom, obs_list, p0, lo, hi, opts, device="cuda", stream=None):
    """Convenience: fits len(obs_list) galaxies sharing `geom`; returns
    (params, chi2, iters, status) as numpy arrays."""
    import numpy as np
    n = len(obs_list)
    obs_dev, _keep = obs_array(obs_list, device)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(n, NPAR)).to(device)
    p, dlo, dhi = t(p0), t(lo), t(hi)
    chi2 = torch.empty(n, dtype=torch.float64, device=device)
    iters = torch.empty(n, dtype=torch.int32, device=device)
    status = torch.empty(n, dtype=torch.int32, device=device)
    nb = gbk_fit_lm_workspace_bytes(geom, n, opts)
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=device)
    gbk_fit_lm(geom, obs_dev, dlo, dhi, p, opts, chi2, iters, status, ws, stream)
    return p.cpu().numpy(), chi2.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy()


def gbk_fit_lm_fallback_workspace_bytes(geom, n_gal, opts):
    g = cgeom(geom)
    n = lib().gbk_fit_lm_fallback_workspace_bytes(ctypes.byref(g), int(n_gal), ctypes.byref(opts))
    err = lib().gbk_last_error().decode()
    if n == 0 and err:
        raise GbkError(GBK_EINVAL, err)
    return int(n)


def gbk_fit_lm_fallback(geom, obs_dev, lo, hi, params, fallback_start, chi2_accept, opts, chi2_out, iters_out,
                        status_out, used_fallback, workspace, stream=None):
    g = cgeom(geom)
    n = params.shape[0]
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_fit_lm_fallback(ctypes.byref(g), int(n), _ptr(obs_dev, torch.uint8, "obs"),
                                     _ptr(lo, torch.float64, "lo"), _ptr(hi, torch.float64, "hi"),
                                     _ptr(params, torch.float64, "params"),
                                     _ptr(fallback_start, torch.float64, "fallback_start"),
                                     _ptr(chi2_accept, torch.float64, "chi2_accept"), ctypes.byref(opts),
                                     _ptr(chi2_out, torch.float64, "chi2_out"),
                                     _ptr(iters_out, torch.int32, "iters_out"),
                                     _ptr(status_out, torch.int32, "status_out"),
                                     _ptr(used_fallback, torch.int32, "used_fallback"),
                                     _ptr(workspace, None, "workspace"), ws_bytes, _stream(stream)))


def fit_lm_fallback(geom, obs_list, seed, fallback, lo, hi, opts, chi2_accept=None, device="cuda", stream=None):
    """Convenience: LM from `seed` with the fit from `fallback` as fallback
    (gbk_fit_lm_fallback); returns (params, chi2, iters, status,
    used_fallback) as numpy arrays."""
    import numpy as np
    n = len(obs_list)
    obs_dev, _keep = obs_array(obs_list, device)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(n, NPAR)).to(device)
    p, fb, dlo, dhi = t(seed), t(fallback), t(lo), t(hi)
    acc = None
    if chi2_accept is not None:
        acc = torch.as_tensor(np.ascontiguousarray(chi2_accept, dtype=np.float64).reshape(n)).to(device)
    chi2 = torch.empty(n, dtype=torch.float64, device=device)
    iters = torch.empty(n, dtype=torch.int32, device=device)
    status = torch.empty(n, dtype=torch.int32, device=device)
    used = torch.empty(n, dtype=torch.int32, device=device)
    nb = gbk_fit_lm_fallback_workspace_bytes(geom, n, opts)
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=device)
    gbk_fit_lm_fallback(geom, obs_dev, dlo, dhi, p, fb, acc, opts, chi2, iters, status, used, ws, stream)
    return (p.cpu().numpy(), chi2.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy(),
            used.cpu().numpy())


def cgeoms(geoms):
    """A host array of gbk_geom structs, one per galaxy (an array built
    earlier is passed through, so that repeated calls skip the marshalling)."""
    if isinstance(geoms, ctypes.Array):
        return geoms
    return (CGeom * len(geoms))(*[cgeom(g) for g in geoms])


def survey_pix_offsets(geoms):
    """Packed pixel offsets P_i = sum_{j<i} nx_j ny_j (length n + 1)."""
    off = [0]
    for g in geoms:
        off.append(off[-1] + int(g.nx) * int(g.ny))
    return off


def gbk_survey_workspace_bytes(geoms, opts=None):
    arr = cgeoms(geoms)
    nb = lib().gbk_survey_workspace_bytes(arr, len(geoms), ctypes.byref(opts) if opts is not None else None)
    if nb == 0 and len(geoms) > 0:
        err = lib().gbk_last_error().decode()
        if err:
            raise GbkError(GBK_EINVAL, err)
    return nb


def gbk_survey_eval(geoms, params, obs_dev=None, maps=None, chi2=None, resid=None, workspace=None, stream=None):
    arr = cgeoms(geoms)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_survey_eval(arr, len(geoms), _ptr(params, torch.float64, "params"),
                                 _ptr(obs_dev, torch.uint8, "obs"), _ptr(maps, torch.float32, "maps"),
                                 _ptr(chi2, torch.float64, "chi2"), _ptr(resid, torch.float32, "resid"),
                                 _ptr(workspace, None, "workspace"), ws_bytes, _stream(stream)))


def gbk_survey_fit_lm(geoms, obs_dev, lo, hi, params, opts, chi2_out, iters_out, status_out, workspace,
                      stream=None):
    arr = cgeoms(geoms)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_survey_fit_lm(arr, len(geoms), _ptr(obs_dev, torch.uint8, "obs"),
                                   _ptr(lo, torch.float64, "lo"), _ptr(hi, torch.float64, "hi"),
                                   _ptr(params, torch.float64, "params"), ctypes.byref(opts),
                                   _ptr(chi2_out, torch.float64, "chi2_out"),
                                   _ptr(iters_out, torch.int32, "iters_out"),
                                   _ptr(status_out, torch.int32, "status_out"), _ptr(workspace, None, "workspace"),
                                   ws_bytes, _stream(stream)))


def _tuning_dict(t, timed=False):
    d = {"cluster_ctas": t.cluster_ctas, "threads": t.threads, "persistent": t.persistent}
    if timed:
        d.update(ms=t.ms, candidates=t.candidates)
    return d


def gbk_survey_autotune(geoms, params, obs_dev, chi2_scratch, workspace, stream=None):
    """Times the survey launch shapes on gbk_survey_eval of this batch and
    keeps the fastest for the survey; returns a dict of the choice."""
    arr = cgeoms(geoms)
    ws_bytes = workspace.numel() * workspace.element_size()
    t = CTuning()
    _check(lib().gbk_survey_autotune(arr, len(geoms), _ptr(params, torch.float64, "params"),
                                     _ptr(obs_dev, torch.uint8, "obs"), _ptr(chi2_scratch, torch.float64, "chi2"),
                                     _ptr(workspace, None, "workspace"), ws_bytes, ctypes.byref(t), _stream(stream)))
    return _tuning_dict(t, True)


def gbk_survey_get_tuning(geoms):
    t = CTuning()
    _check(lib().gbk_survey_get_tuning(cgeoms(geoms), len(geoms), ctypes.byref(t)))
    return _tuning_dict(t)


def gbk_survey_set_tuning(geoms, persistent=None, cluster_ctas=0, threads=0):
    """Forces the survey's launch shape (persistent None forgets it)."""
    arr = cgeoms(geoms)
    if persistent is None:
        _check(lib().gbk_survey_set_tuning(arr, len(geoms), None))
        return
    t = CTuning(int(cluster_ctas), int(threads), int(persistent), 0.0, 0)
    _check(lib().gbk_survey_set_tuning(arr, len(geoms), ctypes.byref(t)))


def survey_eval(geoms, params, obs_list=None, want_maps=True, want_resid=False, device="cuda", stream=None):
    """Convenience: (maps per galaxy [3][ny][nx] or None, chi2 [n] or None,
    resid per galaxy [2][ny][nx] or None) for a ragged batch."""
    params = torch.as_tensor(params, dtype=torch.float64).reshape(len(geoms), NPAR).to(device).contiguous()
    off = survey_pix_offsets(geoms)
    maps = torch.empty(3 * off[-1], dtype=torch.float32, device=device) if want_maps else None
    obs_dev, _keep = obs_array(obs_list, device) if obs_list is not None else (None, None)
    c2 = torch.empty(len(geoms), dtype=torch.float64, device=device) if obs_list is not None else None
    res = torch.empty(2 * off[-1], dtype=torch.float32, device=device) if want_resid else None
    ws = torch.empty(max(gbk_survey_workspace_bytes(geoms), 1), dtype=torch.uint8, device=device)
    gbk_survey_eval(geoms, params, obs_dev, maps, c2, res, ws, stream)
    split = lambda t, k: [t[k * off[i]:k * off[i + 1]].view(k, g.ny, g.nx) for i, g in enumerate(geoms)]
    return (split(maps, 3) if maps is not None else None, c2, split(res, 2) if res is not None else None)


def survey_fit_lm(geoms, obs_list, p0, lo, hi, opts, device="cuda", stream=None):
    """Convenience: fits a ragged batch; returns (params, chi2, iters,
    status) as numpy arrays."""
    import numpy as np
    n = len(geoms)
    obs_dev, _keep = obs_array(obs_list, device)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(n, NPAR)).to(device)
    p, dlo, dhi = t(p0), t(lo), t(hi)
    chi2 = torch.empty(n, dtype=torch.float64, device=device)
    iters = torch.empty(n, dtype=torch.int32, device=device)
    status = torch.empty(n, dtype=torch.int32, device=device)
    ws = torch.empty(max(gbk_survey_workspace_bytes(geoms, opts), 1), dtype=torch.uint8, device=device)
    gbk_survey_fit_lm(geoms, obs_dev, dlo, dhi, p, opts, chi2, iters, status, ws, stream)
    return p.cpu().numpy(), chi2.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy()


def gbk_gemm_bf16(A, B, out_bf16=None, out_f32=None, bias=None, relu=False, mask=None, alpha=1.0, stream=None):
    """D = alpha A B^T (+ bias) (ReLU) (masked) on the tensor cores; A [M][K],
    B [N][K] BF16 (row strides may exceed K); outputs [M][ldo]."""
    M, K = A.shape
    N = B.shape[0]
    out = out_bf16 if out_bf16 is not None else out_f32
    ldo = out.stride(0)
    _check(lib().gbk_gemm_bf16(int(M), int(N), int(K), _strided(A, torch.bfloat16, "A"), int(A.stride(0)),
                               _strided(B, torch.bfloat16, "B"), int(B.stride(0)), _ptr(bias, torch.float32, "bias"),
                               int(bool(relu)), _strided(mask, torch.bfloat16, "mask"),
                               int(mask.stride(0)) if mask is not None else 0, float(alpha),
                               _strided(out_bf16, torch.bfloat16, "out_bf16"), _strided(out_f32, torch.float32, "out_f32"),
                               int(ldo), _stream(stream)))


def gbk_cnn_param_count():
    return int(lib().gbk_cnn_param_count())


def gbk_cnn_workspace_bytes(batch):
    nb = lib().gbk_cnn_workspace_bytes(int(batch))
    if nb == 0:
        raise GbkError(GBK_EINVAL, lib().gbk_last_error().decode())
    return nb


def gbk_cnn_init(params, seed, stream=None):
    _check(lib().gbk_cnn_init(_ptr(params, torch.float32, "params"), int(seed) & ((1 << 64) - 1), _stream(stream)))


def gbk_cnn_targets(params, targets, stream=None):
    _check(lib().gbk_cnn_targets(int(params.shape[0]), _ptr(params, torch.float64, "params"),
                                 _ptr(targets, torch.float32, "targets"), _stream(stream)))


def gbk_cnn_decode(out, params, stream=None):
    _check(lib().gbk_cnn_decode(int(out.shape[0]), _ptr(out, torch.float32, "out"),
                                _ptr(params, torch.float64, "params"), _stream(stream)))


def gbk_cnn_synth_obs(maps, seed, noise_v, dead_frac, v, sigma, mask, stream=None):
    _check(lib().gbk_cnn_synth_obs(int(maps.shape[0]), _ptr(maps, torch.float32, "maps"),
                                   int(seed) & ((1 << 64) - 1), float(noise_v), float(dead_frac),
                                   _ptr(v, torch.float32, "v"), _ptr(sigma, torch.float32, "sigma"),
                                   _ptr(mask, torch.uint8, "mask"), _stream(stream)))


def gbk_cnn_forward(params, v, sigma, mask, out, workspace, stream=None):
    _check(lib().gbk_cnn_forward(_ptr(params, torch.float32, "params"), int(v.shape[0]), _ptr(v, torch.float32, "v"),
                                 _ptr(sigma, torch.float32, "sigma"), _ptr(mask, torch.uint8, "mask"),
                                 _ptr(out, torch.float32, "out"), _ptr(workspace, None, "workspace"),
                                 workspace.numel() * workspace.element_size(), _stream(stream)))


def gbk_cnn_grad(params, v, sigma, mask, targets, grad, loss, workspace, stream=None):
    _check(lib().gbk_cnn_grad(_ptr(params, torch.float32, "params"), int(v.shape[0]), _ptr(v, torch.float32, "v"),
                              _ptr(sigma, torch.float32, "sigma"), _ptr(mask, torch.uint8, "mask"),
                              _ptr(targets, torch.float32, "targets"), _ptr(grad, torch.float32, "grad"),
                              _ptr(loss, torch.float32, "loss"), _ptr(workspace, None, "workspace"),
                              workspace.numel() * workspace.element_size(), _stream(stream)))


def gbk_cnn_train_step(params, adam_m, adam_v, step, lr, v, sigma, mask, targets, loss, workspace, stream=None):
    _check(lib().gbk_cnn_train_step(_ptr(params, torch.float32, "params"), _ptr(adam_m, torch.float32, "adam_m"),
                                    _ptr(adam_v, torch.float32, "adam_v"), int(step), float(lr), int(v.shape[0]),
                                    _ptr(v, torch.float32, "v"), _ptr(sigma, torch.float32, "sigma"),
                                    _ptr(mask, torch.uint8, "mask"), _ptr(targets, torch.float32, "targets"),
                                    _ptr(loss, torch.float32, "loss"), _ptr(workspace, None, "workspace"),
                                    workspace.numel() * workspace.element_size(), _stream(stream)))


class CnnSeed:
    """Convenience owner of the network's parameters, Adam state and
    workspace; every computation runs in the library's kernels."""

    def __init__(self, batch, seed=1, device="cuda"):
        self.batch, self.device = batch, device
        n = gbk_cnn_param_count()
        self.params = torch.empty(n, dtype=torch.float32, device=device)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.ws = torch.empty(gbk_cnn_workspace_bytes(batch), dtype=torch.uint8, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        gbk_cnn_init(self.params, seed)

    def train_step(self, v, sigma, mask, targets, lr):
        self.step += 1
        gbk_cnn_train_step(self.params, self.m, self.v, self.step, lr, v, sigma, mask, targets, self.loss, self.ws)

    def predict(self, v, sigma, mask):
        """Parameter vectors [n][10] (FP64, device) for n maps, in batches."""
        n = v.shape[0]
        B = self.batch
        out = torch.empty((B, 16), dtype=torch.float32, device=self.device)
        res = torch.empty((n, NPAR), dtype=torch.float64, device=self.device)
        for i in range(0, n, B):
            j = min(n, i + B)
            if j - i == B:
                gbk_cnn_forward(self.params, v[i:j], sigma[i:j], mask[i:j], out, self.ws)
            else:  # pad the last batch
                pv, ps = torch.zeros_like(v[:B]), torch.zeros_like(sigma[:B])
                pm = torch.zeros_like(mask[:B])
                pv[:j - i], ps[:j - i], pm[:j - i] = v[i:j], sigma[i:j], mask[i:j]
                gbk_cnn_forward(self.params, pv, ps, pm, out, self.ws)
            gbk_cnn_decode(out[:j - i].contiguous(), res[i:j])
        return res


def _strided(t, dtype, name):
    """Pointer of a row-major 2-D tensor whose rows may be padded."""
    if t is None:
        return None
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("%s must be 2-D with unit column stride" % name)
    return ctypes.c_void_p(t.data_ptr())


def gbk_jacobian(geom, params, obs, free=(0, 1, 2, 3, 4, 5, 6, 7), cot=None, jtj=None, jtv=None, chi2=None,
                 jac=None, stream=None):
    g = cgeom(geom)
    n = params.shape[0]
    mask = 0
    for k in free:
        mask |= 1 << int(k)
    _check(lib().gbk_jacobian(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"), ctypes.byref(obs.c()),
                              mask, _ptr(cot, torch.float32, "cot"), _ptr(jtj, torch.float64, "jtj"),
                              _ptr(jtv, torch.float64, "jtv"), _ptr(chi2, torch.float64, "chi2"),
                              _ptr(jac, torch.float32, "jac"), _stream(stream)))


def gbk_jacobian_workspace_bytes(geom, n_models, free=(0, 1, 2, 3, 4, 5, 6, 7)):
    g = cgeom(geom)
    mask = 0
    for k in free:
        mask |= 1 << int(k)
    n = lib().gbk_jacobian_workspace_bytes(ctypes.byref(g), int(n_models), mask)
    err = lib().gbk_last_error().decode()
    if n == 0 and err:
        raise GbkError(GBK_EUNSUPPORTED if "serves" in err else GBK_EINVAL, err)
    return n


def gbk_jacobian_ws(geom, params, obs, free=(0, 1, 2, 3, 4, 5, 6, 7), cot=None, jtj=None, jtv=None, chi2=None,
                    workspace=None, stream=None):
    """The split-shape analytic Jacobian reductions (J^T J, J^T v, sum r^2)."""
    g = cgeom(geom)
    n = params.shape[0]
    mask = 0
    for k in free:
        mask |= 1 << int(k)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_jacobian_ws(ctypes.byref(g), int(n), _ptr(params, torch.float64, "params"), ctypes.byref(obs.c()),
                                 mask, _ptr(cot, torch.float32, "cot"), _ptr(jtj, torch.float64, "jtj"),
                                 _ptr(jtv, torch.float64, "jtv"), _ptr(chi2, torch.float64, "chi2"),
                                 _ptr(workspace, None, "workspace"), ws_bytes, _stream(stream)))


def gbk_survey_jacobian_workspace_bytes(geoms, free=(0, 1, 2, 3, 4, 5, 6, 7)):
    mask = 0
    for k in free:
        mask |= 1 << int(k)
    nb = lib().gbk_survey_jacobian_workspace_bytes(cgeoms(geoms), len(geoms), mask)
    if nb == 0 and len(geoms) > 0:
        err = lib().gbk_last_error().decode()
        raise GbkError(GBK_EUNSUPPORTED if "serve" in err else GBK_EINVAL, err)
    return nb


def gbk_survey_jacobian(geoms, params, obs_dev, free=(0, 1, 2, 3, 4, 5, 6, 7), jtj=None, jtv=None, chi2=None,
                        workspace=None, stream=None):
    """The ragged split-shape Jacobian reductions of a survey batch (one model
    per galaxy; obs_dev a device array of gbk_obs, obs_array)."""
    mask = 0
    for k in free:
        mask |= 1 << int(k)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbk_survey_jacobian(cgeoms(geoms), len(geoms), _ptr(params, torch.float64, "params"),
                                     _ptr(obs_dev, torch.uint8, "obs"), mask, _ptr(jtj, torch.float64, "jtj"),
                                     _ptr(jtv, torch.float64, "jtv"), _ptr(chi2, torch.float64, "chi2"),
                                     _ptr(workspace, None, "workspace"), ws_bytes, _stream(stream)))


def survey_jacobian(geoms, params, obs_list, free=(0, 1, 2, 3, 4, 5, 6, 7), device="cuda"):
    """Convenience: (J^T J, J^T r, chi2) of a survey batch on the ragged split Jacobian."""
    params = torch.as_tensor(params, dtype=torch.float64).reshape(len(geoms), NPAR).to(device).contiguous()
    n, nf = len(geoms), len(free)
    jtj = torch.empty((n, nf, nf), dtype=torch.float64, device=device)
    jtv = torch.empty((n, nf), dtype=torch.float64, device=device)
    c2 = torch.empty(n, dtype=torch.float64, device=device)
    obs_dev, _keep = obs_array(obs_list, device)
    ws = torch.empty(max(1, gbk_survey_jacobian_workspace_bytes(geoms, free)), dtype=torch.uint8, device=device)
    gbk_survey_jacobian(geoms, params, obs_dev, free, jtj, jtv, c2, ws)
    return jtj, jtv, c2


def jacobian_split(geom, params, obs, free=(0, 1, 2, 3, 4, 5, 6, 7), device="cuda"):
    """Convenience: (J^T J, J^T r, chi2) from the split-shape Jacobian."""
    params = params.to(device=device, dtype=torch.float64).contiguous()
    n, nf = params.shape[0], len(free)
    jtj = torch.empty((n, nf, nf), dtype=torch.float64, device=device)
    jtv = torch.empty((n, nf), dtype=torch.float64, device=device)
    c2 = torch.empty(n, dtype=torch.float64, device=device)
    ws = torch.empty(max(1, gbk_jacobian_workspace_bytes(geom, n, free)), dtype=torch.uint8, device=device)
    gbk_jacobian_ws(geom, params, obs, free, None, jtj, jtv, c2, ws)
    return jtj, jtv, c2


def jacobian(geom, params, obs, free=(0, 1, 2, 3, 4, 5, 6, 7), device="cuda"):
    """Convenience: (J [n][10][2][ny][nx], J^T J, J^T r, chi2) as torch tensors."""
    params = params.to(device=device, dtype=torch.float64).contiguous()
    n, nf = params.shape[0], len(free)
    jac = torch.empty((n, NPAR, 2, geom.ny, geom.nx), dtype=torch.float32, device=device)
    jtj = torch.empty((n, nf, nf), dtype=torch.float64, device=device)
    jtv = torch.empty((n, nf), dtype=torch.float64, device=device)
    c2 = torch.empty(n, dtype=torch.float64, device=device)
    gbk_jacobian(geom, params, obs, free, None, jtj, jtv, c2, jac)
    return jac, jtj, jtv, c2


class ResidualMaps(torch.autograd.Function):
    """Weighted residual maps [n][2][ny][nx] of a batch of parameter sets
    against one galaxy, differentiable with respect to the parameters: the
    forward pass is the fused kernel (gbk_chi2 with residuals), the backward
    pass the analytic Jacobian kernel (gbk_jacobian with the incoming
    gradient as cotangent), so grad_params = J^T grad_resid for all ten
    parameters."""

    @staticmethod
    def forward(ctx, params, geom, obs):
        params = params.contiguous()
        n = params.shape[0]
        out = torch.empty(n, dtype=torch.float64, device=params.device)
        resid = torch.empty((n, 2, geom.ny, geom.nx), dtype=torch.float32, device=params.device)
        gbk_chi2(geom, params.detach(), obs, out, resid, PATH_FUSED)
        ctx.save_for_backward(params.detach())
        ctx.geom, ctx.obs = geom, obs
        return resid

    @staticmethod
    def backward(ctx, grad_resid):
        (params,) = ctx.saved_tensors
        n = params.shape[0]
        g = torch.empty((n, NPAR), dtype=torch.float64, device=params.device)
        cot = grad_resid.to(torch.float32).contiguous()
        gbk_jacobian(ctx.geom, params, ctx.obs, tuple(range(NPAR)), cot, None, g, None, None)
        return g.to(params.dtype), None, None


def residual_maps(params, geom, obs):
    """Differentiable residual maps (see ResidualMaps)."""
    return ResidualMaps.apply(params, geom, obs)


def gbk_grid(geom, obs, lo, hi, nodes, fixed, levels=3, chunk=16384, device="cuda", stream=None):
    """Nested-grid search; returns (best_params, best_index per level,
    best_chi2 per level) as numpy arrays."""
    import numpy as np
    g = cgeom(geom)
    D = ctypes.c_double * NPAR
    I = ctypes.c_int32 * NPAR
    nd = I(*[int(v) for v in nodes])
    nb = lib().gbk_grid_workspace_bytes(ctypes.byref(g), nd, int(chunk))
    if nb == 0:
        raise GbkError(GBK_EINVAL, lib().gbk_last_error().decode())
    ws = torch.empty(nb, dtype=torch.uint8, device=device)
    bp = D()
    bi = (ctypes.c_int64 * levels)()
    bc = (ctypes.c_double * levels)()
    _check(lib().gbk_grid(ctypes.byref(g), ctypes.byref(obs.c()), D(*[float(v) for v in lo]),
                          D(*[float(v) for v in hi]), nd, D(*[float(v) for v in fixed]), int(levels), int(chunk),
                          bp, bi, bc, _ptr(ws, None, "workspace"), nb, _stream(stream)))
    return np.array(bp[:]), np.array(bi[:]), np.array(bc[:])


def gbk_nested_sample(geom, obs, lo, hi, n_live=400, batch=None, tol=0.5, efr=1.0, seed=1, max_iter=100000,
                      device="cuda", stream=None):
    """Nested sampling; returns dict(mean, std, log_z, n_eval, n_iter)."""
    import numpy as np
    g = cgeom(geom)
    o = CNsOpts(int(n_live), int(batch if batch else max(1, n_live // 4)), float(tol), float(efr), int(seed),
                int(max_iter), 0)
    nb = lib().gbk_nested_sample_workspace_bytes(ctypes.byref(g), ctypes.byref(o))
    if nb == 0:
        raise GbkError(GBK_EINVAL, lib().gbk_last_error().decode())
    ws = torch.empty(nb, dtype=torch.uint8, device=device)
    D = ctypes.c_double * NPAR
    mean, std, lz = D(), D(), ctypes.c_double()
    ne, ni = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().gbk_nested_sample(ctypes.byref(g), ctypes.byref(obs.c()), D(*[float(v) for v in lo]),
                                   D(*[float(v) for v in hi]), ctypes.byref(o), mean, std, ctypes.byref(lz),
                                   ctypes.byref(ne), ctypes.byref(ni), _ptr(ws, None, "workspace"), nb,
                                   _stream(stream)))
    return {"mean": np.array(mean[:]), "std": np.array(std[:]), "log_z": lz.value, "n_eval": ne.value,
            "n_iter": ni.value}


def gbk_nested_sample_traced(geom, obs, lo, hi, n_live=400, batch=None, tol=0.5, efr=1.0, seed=1, max_iter=100000,
                             trace_iters=0, device="cuda", stream=None):
    """gbk_nested_sample with its first trace_iters iterations recorded:
    returns the result dict plus "trace" = dict(live0 [n_live][NPAR],
    live0_chi2 [n_live], n_props [T], props [T][batch][NPAR], chi2
    [T][batch], replaced [T][batch]) for the T <= trace_iters iterations run."""
    import numpy as np
    K = int(batch if batch else max(1, n_live // 4))
    g = cgeom(geom)
    o = CNsOpts(int(n_live), K, float(tol), float(efr), int(seed), int(max_iter), 0)
    nb = lib().gbk_nested_sample_workspace_bytes(ctypes.byref(g), ctypes.byref(o))
    if nb == 0:
        raise GbkError(GBK_EINVAL, lib().gbk_last_error().decode())
    ws = torch.empty(nb, dtype=torch.uint8, device=device)
    T = int(trace_iters)
    live0 = np.zeros((n_live, NPAR))
    live0_c = np.zeros(n_live)
    n_props = np.zeros(max(T, 1), np.int32)
    props = np.zeros((max(T, 1), K, NPAR))
    chi2 = np.zeros((max(T, 1), K))
    repl = np.zeros((max(T, 1), K), np.int32)
    tr = CNsTrace(T, 0, live0.ctypes.data, live0_c.ctypes.data, n_props.ctypes.data, props.ctypes.data,
                  chi2.ctypes.data, repl.ctypes.data)
    D = ctypes.c_double * NPAR
    mean, std, lz = D(), D(), ctypes.c_double()
    ne, ni = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().gbk_nested_sample_traced(ctypes.byref(g), ctypes.byref(obs.c()), D(*[float(v) for v in lo]),
                                          D(*[float(v) for v in hi]), ctypes.byref(o), mean, std, ctypes.byref(lz),
                                          ctypes.byref(ne), ctypes.byref(ni), _ptr(ws, None, "workspace"), nb,
                                          _stream(stream), ctypes.byref(tr)))
    n = tr.n_iter
    return {"mean": np.array(mean[:]), "std": np.array(std[:]), "log_z": lz.value, "n_eval": ne.value,
            "n_iter": ni.value,
            "trace": {"live0": live0, "live0_chi2": live0_c, "n_props": n_props[:n], "props": props[:n],
                      "chi2": chi2[:n], "replaced": repl[:n]}}


def gbk_initial_guess(geom, obs_dev, fixed, params_out, continuum=None, stream=None):
    """Initial parameter values (Sec. 2.1.9) of n galaxies sharing `geom`:
    obs_dev a device array of gbk_obs (obs_array), fixed / params_out
    [n][NPAR] FP64 device tensors, continuum [n][ny][nx] FP32 or None."""
    g = cgeom(geom)
    n = params_out.shape[0]
    _check(lib().gbk_initial_guess(ctypes.byref(g), int(n), _ptr(continuum, torch.float32, "continuum"),
                                   _ptr(obs_dev, torch.uint8, "obs"), _ptr(fixed, torch.float64, "fixed"),
                                   _ptr(params_out, torch.float64, "params_out"), _stream(stream)))


def initial_guess(geom, obs_list, fixed, continuum=None, device="cuda", stream=None):
    """Convenience: initial parameter values as a numpy array [n][NPAR]."""
    import numpy as np
    n = len(obs_list)
    obs_dev, _keep = obs_array(obs_list, device)
    f = torch.as_tensor(np.ascontiguousarray(fixed, dtype=np.float64).reshape(n, NPAR)).to(device)
    out = torch.empty((n, NPAR), dtype=torch.float64, device=device)
    c = None
    if continuum is not None:
        c = torch.as_tensor(continuum, dtype=torch.float32).reshape(n, geom.ny, geom.nx).to(device).contiguous()
    gbk_initial_guess(geom, obs_dev, f, out, c, stream)
    return out.cpu().numpy()


def gbk_wait_selfcheck(limit, complete, stream=None):
    """Runs the bounded device wait on a barrier that nothing completes
    (complete=False) or that one arrival completes; returns the wait's
    duration in ns.  A wait that runs out sets bit 2 of gbk_device_status()."""
    ns = ctypes.c_int64()
    _check(lib().gbk_wait_selfcheck(int(limit), 1 if complete else 0, ctypes.byref(ns), _stream(stream)))
    return ns.value


def gbk_device_status():
    """Reads and clears the device status word (0 = all bounded waits completed)."""
    v = ctypes.c_int32()
    _check(lib().gbk_device_status(ctypes.byref(v)))
    return v.value


def gbk_version():
    return lib().gbk_version().decode()


# ----------------------------------------------------------------------------
# Convenience wrappers that allocate outputs with torch (device memory is the
# caller's; these only size and allocate the tensors the C calls fill).

def workspace_for(geom, n_models, flags=PATH_AUTO, device="cuda"):
    nb = gbk_workspace_bytes(geom, n_models, flags)
    return torch.empty(max(nb, 1), dtype=torch.uint8, device=device) if nb else None


def eval_maps(geom, params, device="cuda", stream=None, split=False):
    """Maps of a batch: from the fused path (split=False; the staged path
    where the fused one does not serve) or from the split path (split=True)."""
    params = params.to(device=device, dtype=torch.float64).contiguous()
    n = params.shape[0]
    maps = torch.empty((n, 3, geom.ny, geom.nx), dtype=torch.float32, device=device)
    if split:
        ws = workspace_for(geom, n, PATH_SPLIT, device)
        if ws is None:
            raise GbkError(GBK_EUNSUPPORTED, "the split path does not serve this geometry")
    else:
        ws = workspace_for(geom, n, PATH_AUTO, device) if getattr(geom, "upsample", 1) > 1 else None
    gbk_eval_cubes(geom, params, maps=maps, workspace=ws, stream=stream)
    return maps


def eval_cubes(geom, params, device="cuda", stream=None):
    params = params.to(device=device, dtype=torch.float64).contiguous()
    n = params.shape[0]
    cubes = torch.empty((n, geom.nz, geom.ny, geom.nx), dtype=torch.float32, device=device)
    maps = torch.empty((n, 3, geom.ny, geom.nx), dtype=torch.float32, device=device)
    ws = workspace_for(geom, n, PATH_STAGED, device)
    gbk_eval_cubes(geom, params, cubes=cubes, maps=maps, workspace=ws, stream=stream)
    return cubes, maps


def chi2(geom, params, obs, flags=PATH_AUTO, want_resid=False, device="cuda", stream=None):
    params = params.to(device=device, dtype=torch.float64).contiguous()
    n = params.shape[0]
    out = torch.empty(n, dtype=torch.float64, device=device)
    resid = torch.empty((n, 2, geom.ny, geom.nx), dtype=torch.float32, device=device) if want_resid else None
    ws = workspace_for(geom, n, flags, device)
    gbk_chi2(geom, params, obs, out, resid, flags, ws, stream)
    return (out, resid) if want_resid else out
