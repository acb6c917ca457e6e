"""Python binding of the MRIP engine's C ABI (include/mrip.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``_build/libmrip.so``.  Device buffers are PyTorch CUDA tensors
(their ``data_ptr()`` is passed through); host buffers are numpy arrays.  The
functions keep the C names.  A missing library raises ``MripLibraryMissing``
-- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from ._abi import (MRIP_MAP_AUTO, MRIP_MAP_CTA, MRIP_MAP_PERSISTENT, MRIP_MAP_THREAD,  # noqa: F401
                   MRIP_MAP_WARP_1LANE, MRIP_MAP_WARP_COOP, MRIP_MM1, MRIP_TANDEM3,
                   MRIP_FOREST_FIRE, MRIP_WALK_L1_EXIT, STATUS_NAMES, MripError,
                   MripLibraryMissing, mrip_cv_params, mrip_cv_report, mrip_cv_stat,
                   mrip_forest_fire_params,
                   mrip_mm1_params, mrip_stat, mrip_tandem3_params, mrip_train_params,
                   mrip_walk_params, lib, library_path, load_library, using_library)
from ._abi import check as _check

__all__ = [n for n in dir() if n.startswith("mrip_") or n.startswith("MRIP_")] + [
    "MripError", "MripLibraryMissing", "lib", "library_path", "load_library", "using_library", "Model"]


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _dev(t, dtype=None, name="tensor", allow_none=False):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s must not be None" % name)
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype, name="array"):
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _t():
    import torch
    return torch


# ---------------------------------------------------------------------------
# stage entry points
# ---------------------------------------------------------------------------
def mrip_philox(ctr, key, out, stream=None):
    t = _t()
    n = ctr.shape[0]
    _check(lib().mrip_philox(_dev(ctr, t.int32, "ctr"), _dev(key, t.int32, "key"), n,
                             _dev(out, t.int32, "out"), _stream(stream)))


def mrip_expo(lo, hi, rate, u_out, e_out, stream=None):
    t = _t()
    _check(lib().mrip_expo(_dev(lo, t.int32), _dev(hi, t.int32), _dev(rate, t.float64),
                           lo.numel(), _dev(u_out, t.float64, allow_none=True),
                           _dev(e_out, t.float64, allow_none=True), _stream(stream)))


def mrip_mm1_simulate(dps, n_reps, n_clients, seed, mapping, wait, idle=None, system=None,
                      stream=None, rep0=0):
    t = _t()
    _check(lib().mrip_mm1_simulate(_dev(dps, t.float64, "dps"), dps.shape[0], int(rep0), int(n_reps),
                                   int(n_clients), int(seed), int(mapping),
                                   _dev(wait, t.float64, allow_none=True),
                                   _dev(idle, t.float64, allow_none=True),
                                   _dev(system, t.float64, allow_none=True), _stream(stream)))


def mrip_tandem3_simulate(dps, rep0, n_reps, n_clients, window, seed, tag, mapping, y, feat=None,
                          stream=None):
    t = _t()
    _check(lib().mrip_tandem3_simulate(_dev(dps, t.float64, "dps"), dps.shape[0], int(rep0),
                                       int(n_reps), int(n_clients), int(window), int(seed),
                                       int(tag), int(mapping), _dev(y, t.float64, "y"),
                                       _dev(feat, t.float64, allow_none=True), _stream(stream)))


def mrip_forest_fire_simulate(dps, n_reps, L, n_steps, density, seed, init=None, counts=None,
                              scalar=None, final=None, stream=None, rep0=0):
    t = _t()
    _check(lib().mrip_forest_fire_simulate(
        _dev(dps, t.float64, "dps"), dps.shape[0], int(rep0), int(n_reps), int(L), int(n_steps),
        float(density), int(seed), _dev(init, t.uint8, allow_none=True),
        _dev(counts, t.int32, allow_none=True), _dev(scalar, t.float64, allow_none=True),
        _dev(final, t.uint8, allow_none=True), _stream(stream)))


def mrip_forest_fire_skip_simulate(dps, n_reps, L, n_steps, density, seed, init=None, counts=None,
                                   scalar=None, final=None, stream=None, rep0=0):
    t = _t()
    _check(lib().mrip_forest_fire_skip_simulate(
        _dev(dps, t.float64, "dps"), dps.shape[0], int(rep0), int(n_reps), int(L), int(n_steps),
        float(density), int(seed), _dev(init, t.uint8, allow_none=True),
        _dev(counts, t.int32, allow_none=True), _dev(scalar, t.float64, allow_none=True),
        _dev(final, t.uint8, allow_none=True), _stream(stream)))


def mrip_walk_simulate(radii, n_reps, seed, max_steps, mapping, tau, warps_per_cta=0,
                       ctas_per_sm=0, chunk=0, stream=None, rep0=0):
    t = _t()
    r, rp = _host(radii, np.float64)
    _check(lib().mrip_walk_simulate(rp, r.size, int(rep0), int(n_reps), int(seed), int(max_steps),
                                    int(mapping), int(warps_per_cta), int(ctas_per_sm),
                                    int(chunk), _dev(tau, t.int64, "tau"), _stream(stream)))


def mrip_walk_simulate_noalloc(radii, n_reps, seed, max_steps, mapping, tau, warps_per_cta=0,
                               ctas_per_sm=0, chunk=0, stream=None, rep0=0):
    """mrip_walk_simulate for callers that cannot allocate device memory: its
    scratch is a fixed array inside the library (at most 1024 radii); calls
    must not overlap on the GPU."""
    t = _t()
    r, rp = _host(radii, np.float64)
    _check(lib().mrip_walk_simulate_noalloc(rp, r.size, int(rep0), int(n_reps), int(seed), int(max_steps),
                                            int(mapping), int(warps_per_cta), int(ctas_per_sm),
                                            int(chunk), _dev(tau, t.int64, "tau"),
                                            _stream(stream)))


def mrip_area_walk_simulate(n_reps, n_steps, seed, mapping, final_area, visits=None, stream=None,
                            rep0=0):
    t = _t()
    _check(lib().mrip_area_walk_simulate(int(rep0), int(n_reps), int(n_steps), int(seed), int(mapping),
                                         _dev(final_area, t.int32, "final_area"),
                                         _dev(visits, t.int32, allow_none=True), _stream(stream)))


def mrip_pi_simulate(n_reps, n_draws, seed, hits, stream=None, rep0=0):
    t = _t()
    _check(lib().mrip_pi_simulate(int(rep0), int(n_reps), int(n_draws), int(seed), _dev(hits, t.int64, "hits"),
                                  _stream(stream)))


def mrip_check_device_flags():
    _check(lib().mrip_check_device_flags())


def mrip_probe_mul_wide(stream=None):
    """Measured warp-wide widening multiplies per second (32 products each)."""
    v = ctypes.c_double(0.0)
    _check(lib().mrip_probe_mul_wide(ctypes.byref(v), _stream(stream)))
    return v.value


def mrip_debug_checks(library=None):
    """(enabled, first) of the bounds checks of a debug build: enabled is
    False for a release library; first is None or (site, index) of the first
    failed check since the last call (the records are cleared)."""
    L = library if library is not None else lib()
    en = ctypes.c_int32(0)
    first = ctypes.c_uint64(0)
    _check(L.mrip_debug_checks(ctypes.byref(en), ctypes.byref(first)))
    rec = first.value
    return bool(en.value), (None if rec == 0 else (rec >> 40, rec & ((1 << 40) - 1)))


def mrip_stats_reduce(x, out, stream=None):
    t = _t()
    _check(lib().mrip_stats_reduce(_dev(x, t.float64, "x"), x.shape[0], x.shape[1],
                                   _dev(out, t.float64, "out"), _stream(stream)))


def mrip_stats_reduce_i64(x, out, stream=None):
    t = _t()
    _check(lib().mrip_stats_reduce_i64(_dev(x, t.int64, "x"), x.shape[0], x.shape[1],
                                       _dev(out, t.float64, "out"), _stream(stream)))


def mrip_stats_finalize(nmm2, conf=0.95):
    a, p = _host(nmm2, np.float64)
    n_dp = a.size // 3
    out = (mrip_stat * max(n_dp, 1))()
    _check(lib().mrip_stats_finalize(p, n_dp, float(conf), out))
    return [_stat_dict(out[i]) for i in range(n_dp)]


def mrip_stats_merge(parts):
    """Merge (n_parts, n_dp, 3) host triples into (n_dp, 3), parts in order."""
    a, p = _host(parts, np.float64)
    a = a.reshape(a.shape[0], -1, 3)
    out = np.empty((a.shape[1], 3))
    _check(lib().mrip_stats_merge(p, a.shape[0], a.shape[1], out.ctypes.data_as(ctypes.c_void_p)))
    return out


def mrip_t_crit(conf, df):
    v = ctypes.c_double()
    _check(lib().mrip_t_crit(float(conf), int(df), ctypes.byref(v)))
    return v.value


def mrip_mlp_param_count(d_in):
    return int(lib().mrip_mlp_param_count(int(d_in)))


def mrip_mlp_init(d_in, seed, theta, stream=None):
    t = _t()
    _check(lib().mrip_mlp_init(int(d_in), int(seed), _dev(theta, t.float32, "theta"),
                               _stream(stream)))


def mrip_mlp_forward(theta, d_in, x, yhat, stream=None):
    t = _t()
    n = x.shape[1]
    _check(lib().mrip_mlp_forward(_dev(theta, t.float32, "theta"), int(d_in),
                                  _dev(x, t.float32, "x"), n, _dev(yhat, t.float32, "yhat"),
                                  _stream(stream)))


def mrip_mlp_loss_grad(theta, d_in, x, y, idx, B, grad, loss=None, stream=None):
    t = _t()
    n = x.shape[1]
    _check(lib().mrip_mlp_loss_grad(_dev(theta, t.float32, "theta"), int(d_in),
                                    _dev(x, t.float32, "x"), _dev(y, t.float32, "y"), n,
                                    _dev(idx, t.int64, allow_none=True), int(B),
                                    _dev(grad, t.float32, "grad"),
                                    _dev(loss, t.float32, allow_none=True), _stream(stream)))


def mrip_adam_step(theta, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   stream=None):
    t = _t()
    _check(lib().mrip_adam_step(_dev(theta, t.float32), _dev(m, t.float32), _dev(v, t.float32),
                                _dev(grad, t.float32), theta.numel(), int(step), float(lr),
                                float(beta1), float(beta2), float(eps), _stream(stream)))


def mrip_mlp_train(d_in, x, y, theta, batch, epochs, order_seed, lr=1e-3, beta1=0.9, beta2=0.999,
                   eps=1e-8, max_steps=0, patience=0, xv=None, yv=None, losses=None, grad=None,
                   m=None, v=None, val_losses=None, epoch0=0, m_in=None, v_in=None, stream=None):
    """Tensor-core training (synchronous).  x: float (d_in, n) planes; xv, yv
    the optional validation set; epoch0, m_in, v_in resume a run.  Returns
    (epochs run, epoch kept, steps run)."""
    t = _t()
    n = x.shape[1]
    n_val = 0 if xv is None else xv.shape[1]
    prm = mrip_train_params(batch=int(batch), epochs=int(epochs), patience=int(patience),
                            max_steps=int(max_steps), lr=lr, beta1=beta1, beta2=beta2, eps=eps,
                            order_seed=int(order_seed), epoch0=int(epoch0))
    info = (ctypes.c_int32 * 3)()
    _check(lib().mrip_mlp_train(int(d_in), _dev(x, t.float32, "x"), _dev(y, t.float32, "y"), n,
                                _dev(xv, t.float32, allow_none=True),
                                _dev(yv, t.float32, allow_none=True), n_val, ctypes.byref(prm),
                                _dev(theta, t.float32, "theta"),
                                _dev(m_in, t.float32, allow_none=True),
                                _dev(v_in, t.float32, allow_none=True),
                                _dev(losses, t.float32, allow_none=True),
                                _dev(grad, t.float32, allow_none=True),
                                _dev(m, t.float32, allow_none=True),
                                _dev(v, t.float32, allow_none=True),
                                _dev(val_losses, t.float32, allow_none=True), info,
                                _stream(stream)))
    return int(info[0]), int(info[1]), int(info[2])


def mrip_cv_reduce(y, g, gc, out, stream=None):
    t = _t()
    _check(lib().mrip_cv_reduce(_dev(y, t.float64), _dev(g, t.float64), y.shape[1],
                                _dev(gc, t.float64), gc.shape[1], y.shape[0],
                                _dev(out, t.float64), _stream(stream)))


def mrip_last_error():
    return lib().mrip_last_error().decode()


def _stat_dict(s):
    return dict(n=int(s.n), mean=s.mean, var=s.var, half_width=s.half_width, t_crit=s.t_crit)


def _cv_dict(s):
    return dict(n=int(s.n), m=int(s.m), beta=s.beta, mean=s.mean, var=s.var,
                half_width=s.half_width, t_crit=s.t_crit)


# ---------------------------------------------------------------------------
# model handles
# ---------------------------------------------------------------------------
_PARAMS = {MRIP_MM1: mrip_mm1_params, MRIP_TANDEM3: mrip_tandem3_params,
           MRIP_FOREST_FIRE: mrip_forest_fire_params, MRIP_WALK_L1_EXIT: mrip_walk_params}


def mrip_create_model(kind, **params):
    """Create a model handle; params are the fields of the kind's struct."""
    cls = _PARAMS.get(kind)
    if cls is None:
        raise MripError(1, "unknown model kind %r" % (kind,))
    p = cls(**params)
    h = ctypes.c_void_p()
    _check(lib().mrip_create_model(int(kind), ctypes.byref(p), ctypes.sizeof(p), ctypes.byref(h)))
    return h


def mrip_set_stream(model, stream):
    _check(lib().mrip_set_stream(model, _stream(stream)))


def mrip_run(model, design_points, n_reps, seed):
    a, p = _host(design_points, np.float64)
    n_dp = a.shape[0] if a.ndim > 1 else a.size
    _check(lib().mrip_run(model, p, n_dp, int(n_reps), int(seed)))


def mrip_run_range(model, design_points, rep_lo, rep_hi, seed):
    a, p = _host(design_points, np.float64)
    n_dp = a.shape[0] if a.ndim > 1 else a.size
    _check(lib().mrip_run_range(model, p, n_dp, int(rep_lo), int(rep_hi), int(seed)))


def mrip_moments(model, n_dp):
    out = np.empty((n_dp, 3))
    _check(lib().mrip_moments(model, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def mrip_run_device(model, d_design_points, n_reps, seed):
    t = _t()
    _check(lib().mrip_run_device(model, _dev(d_design_points, t.float64), d_design_points.shape[0],
                                 int(n_reps), int(seed)))


def mrip_stats(model, n_dp, conf=0.95):
    out = (mrip_stat * n_dp)()
    _check(lib().mrip_stats(model, float(conf), out))
    return [_stat_dict(out[i]) for i in range(n_dp)]


def mrip_output_bytes(model, which):
    b = ctypes.c_size_t()
    _check(lib().mrip_output_bytes(model, int(which), ctypes.byref(b)))
    return b.value


def mrip_outputs(model, which, dst):
    """Copy output plane `which` into dst (numpy array or CUDA tensor)."""
    if isinstance(dst, np.ndarray):
        if not dst.flags.c_contiguous:
            raise ValueError("dst must be contiguous")
        _check(lib().mrip_outputs(model, int(which), dst.ctypes.data_as(ctypes.c_void_p),
                                  dst.nbytes, 0))
    else:
        _check(lib().mrip_outputs(model, int(which), _dev(dst), dst.numel() * dst.element_size(),
                                  1))
    return dst


def mrip_set_plan(model, plan_json):
    _check(lib().mrip_set_plan(model, plan_json.encode()))


def mrip_get_plan(model):
    buf = ctypes.create_string_buffer(256)
    _check(lib().mrip_get_plan(model, buf, 256))
    return buf.value.decode()


def mrip_autotune(model, design_points, n_reps, seed, trials=3, cache_path=None):
    a, p = _host(design_points, np.float64)
    n_dp = a.shape[0] if a.ndim > 1 else a.size
    _check(lib().mrip_autotune(model, p, n_dp, int(n_reps), int(seed), int(trials),
                               cache_path.encode() if cache_path else None))


def mrip_run_cv(model, design_points, n_reps, seed, train_frac=0.1, val_frac=0.1, epochs=20,
                patience=3, batch=1024, gate=True, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                m_ctrl=0, conf=0.95, net_seed=None):
    """Returns (plain intervals, control-variate intervals, report dict);
    m_ctrl = 0 lets the library size the control runs; report["declined"] is
    0 (kept), 1 (declined after training) or 2 (declined by the screen)."""
    a, p = _host(design_points, np.float64)
    n_dp = a.shape[0]
    prm = mrip_cv_params(train_frac=train_frac, val_frac=val_frac, epochs=epochs, patience=patience,
                         batch=batch, gate=1 if gate else 0, lr=lr, beta1=beta1, beta2=beta2,
                         eps=eps, m_ctrl=int(m_ctrl or 0), conf=conf,
                         net_seed=int(seed if net_seed is None else net_seed))
    plain = (mrip_stat * n_dp)()
    cv = (mrip_cv_stat * n_dp)()
    rep = mrip_cv_report()
    _check(lib().mrip_run_cv(model, p, n_dp, int(n_reps), int(seed), ctypes.byref(prm), plain,
                             cv, ctypes.byref(rep)))
    report = {name: getattr(rep, name) for name, _ in mrip_cv_report._fields_}
    return [_stat_dict(plain[i]) for i in range(n_dp)], [_cv_dict(cv[i]) for i in range(n_dp)], \
        report


def mrip_cv_network(model, d_in):
    """(parameters float32[P], standardisation float64[d_in + 1][2]) of the
    handle's last control-variate run."""
    th = np.empty(mrip_mlp_param_count(d_in), dtype=np.float32)
    norm = np.empty(2 * (d_in + 1))
    _check(lib().mrip_cv_network(model, th.ctypes.data_as(ctypes.c_void_p),
                                 norm.ctypes.data_as(ctypes.c_void_p)))
    return th, norm.reshape(d_in + 1, 2)


def mrip_destroy(model):
    lib().mrip_destroy(model)


class Model:
    """Owning wrapper of a model handle."""

    def __init__(self, kind, **params):
        self.kind = kind
        self.h = mrip_create_model(kind, **params)
        self.n_dp = 0

    def set_stream(self, stream):
        mrip_set_stream(self.h, stream)

    def run(self, design_points, n_reps, seed):
        dp = np.asarray(design_points, dtype=np.float64)
        self.n_dp = dp.shape[0] if dp.ndim > 1 else dp.size
        mrip_run(self.h, dp, n_reps, seed)

    def run_range(self, design_points, rep_lo, rep_hi, seed):
        dp = np.asarray(design_points, dtype=np.float64)
        self.n_dp = dp.shape[0] if dp.ndim > 1 else dp.size
        mrip_run_range(self.h, dp, rep_lo, rep_hi, seed)

    def moments(self):
        return mrip_moments(self.h, self.n_dp)

    def run_device(self, d_design_points, n_reps, seed):
        self.n_dp = d_design_points.shape[0]
        mrip_run_device(self.h, d_design_points, n_reps, seed)

    def stats(self, conf=0.95):
        return mrip_stats(self.h, self.n_dp, conf)

    def outputs(self, which=0, dtype=np.float64, shape=None):
        nbytes = mrip_output_bytes(self.h, which)
        dst = np.empty(nbytes // np.dtype(dtype).itemsize, dtype=dtype)
        mrip_outputs(self.h, which, dst)
        return dst if shape is None else dst.reshape(shape)

    def set_plan(self, plan_json):
        mrip_set_plan(self.h, plan_json)

    def get_plan(self):
        return mrip_get_plan(self.h)

    def autotune(self, design_points, n_reps, seed, trials=3, cache_path=None):
        mrip_autotune(self.h, design_points, n_reps, seed, trials, cache_path)

    def run_cv(self, design_points, n_reps, seed, **kw):
        return mrip_run_cv(self.h, design_points, n_reps, seed, **kw)

    def cv_network(self):
        return mrip_cv_network(self.h, 8 if self.kind == MRIP_TANDEM3 else 6)

    def close(self):
        if self.h is not None:
            mrip_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_dir():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
