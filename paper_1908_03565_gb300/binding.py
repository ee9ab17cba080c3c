"""Thin ctypes binding of libjxlrecon (include/jxl_recon.h).

Only argument marshalling lives here: every step of the reconstruction runs
in the library's CUDA kernels.  Device buffers come from PyTorch (``torch``
is used for device memory and nothing else); host buffers are numpy arrays.
There is no fallback: if the shared library is missing or fails to load,
``load()`` raises.
"""
import ctypes
import threading
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjxlrecon.so")

JXLR_OK, JXLR_EAGAIN, JXLR_EINVAL, JXLR_ENOMEM = 0, 1, -1, -2
JXLR_EBUSY, JXLR_ECUDA, JXLR_ETIMEDOUT, JXLR_ECANCELLED = -3, -4, -5, -6
OUT_F32_LINEAR, OUT_F16_LINEAR, OUT_U8_SRGB, OUT_F32_XYB = 0, 1, 2, 3
PREC_FP32, PREC_TC_F16X3 = 0, 1
OUT_BYTES = {OUT_F32_LINEAR: 12, OUT_F16_LINEAR: 6, OUT_U8_SRGB: 3, OUT_F32_XYB: 12}

EXPORTS = ("jxl_recon_filter_defaults", "jxl_recon_create", "jxl_recon_submit",
           "jxl_recon_submit_xyb", "jxl_recon_poll", "jxl_recon_stage_ms",
           "jxl_recon_launch_count", "jxl_recon_device_bytes", "jxl_recon_destroy",
           "jxl_recon_last_error", "jxl_recon_run_noalloc", "jxl_recon_serve",
           "jxl_recon_batch_create", "jxl_recon_batch_launch", "jxl_recon_batch_query",
           "jxl_recon_batch_status",
           "jxl_recon_batch_destroy", "jxl_recon_submit_jpeg", "jxl_recon_epf_stats",
           "jxl_recon_server_start", "jxl_recon_server_enqueue", "jxl_recon_server_wait",
           "jxl_recon_server_stop")


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_cap_bytes", ctypes.c_size_t),
                ("max_slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("timing", ctypes.c_int), ("cuda_stream", ctypes.c_void_p)]


class Coeffs(ctypes.Structure):
    _fields_ = [("xsize", ctypes.c_uint32), ("ysize", ctypes.c_uint32),
                ("plane", ctypes.c_void_p * 3), ("row_stride_elems", ctypes.c_size_t),
                ("on_device", ctypes.c_int)]


class Cfl(ctypes.Structure):
    _fields_ = [("k", ctypes.c_void_p), ("kx_dc", ctypes.c_float), ("kb_dc", ctypes.c_float)]


class FilterParams(ctypes.Structure):
    _fields_ = [("gab", ctypes.c_int), ("gab_w1", ctypes.c_float * 3),
                ("gab_w2", ctypes.c_float * 3), ("epf", ctypes.c_int),
                ("epf_weight_min", ctypes.c_float), ("epf_scale", ctypes.c_float * 3),
                ("epf_sharp_lut", ctypes.c_float * 8), ("epf_range_max", ctypes.c_float),
                ("epf_range_mul", ctypes.c_float), ("epf_quant_mul", ctypes.c_float),
                ("epf_sigma_max", ctypes.c_uint32), ("sharpness", ctypes.c_void_p),
                ("m_dc", ctypes.c_float * 3), ("inv_opsin", ctypes.c_float * 9),
                ("opsin_bias", ctypes.c_float * 3), ("target_nits_div50", ctypes.c_uint32),
                ("dequant", ctypes.c_void_p), ("dc_smooth", ctypes.c_int),
                ("lf_predict", ctypes.c_int), ("qco", ctypes.c_int),
                ("qco_interval_mul", ctypes.c_float), ("noise", ctypes.c_int),
                ("noise_lut", ctypes.c_float * 16)]


class JpegComponent(ctypes.Structure):
    _fields_ = [("width_in_blocks", ctypes.c_uint32), ("height_in_blocks", ctypes.c_uint32),
                ("h_samp", ctypes.c_uint32), ("v_samp", ctypes.c_uint32),
                ("coeffs", ctypes.c_void_p), ("quant", ctypes.c_void_p), ("gab", ctypes.c_int),
                ("gab_w1", ctypes.c_float), ("gab_w2", ctypes.c_float),
                ("gab_threshold", ctypes.c_float), ("gab_limit", ctypes.c_int),
                ("cond", ctypes.c_int), ("cond_max_gap", ctypes.c_float),
                ("cond_min_step", ctypes.c_float)]


class JpegStream(ctypes.Structure):
    _fields_ = [("xsize", ctypes.c_uint32), ("ysize", ctypes.c_uint32),
                ("num_components", ctypes.c_uint32), ("comp", JpegComponent * 3),
                ("on_device", ctypes.c_int)]


class Output(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("row_stride_bytes", ctypes.c_size_t),
                ("dtype", ctypes.c_int), ("on_device", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("coeffs", ctypes.c_void_p), ("varblock_map", ctypes.c_void_p),
                ("quant_field", ctypes.c_void_p), ("cfl_map", ctypes.c_void_p),
                ("filter_params", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class ServeStats(ctypes.Structure):
    _fields_ = [("makespan_s", ctypes.c_double), ("busy_refusals", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("max_in_flight", ctypes.c_uint32),
                ("bypassed", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("age_bound_ms", ctypes.c_double), ("bypass", ctypes.c_int),
                ("exclusive_mpx", ctypes.c_double)]


def _stats_dict(stats):
    return {"makespan_s": stats.makespan_s, "busy_refusals": stats.busy_refusals,
            "completed": stats.completed, "max_in_flight": stats.max_in_flight,
            "bypassed": stats.bypassed}


class BatchInfo(ctypes.Structure):
    _fields_ = [("images", ctypes.c_uint32), ("pixels", ctypes.c_uint64),
                ("recon_items", ctypes.c_uint32), ("epf_items", ctypes.c_uint32),
                ("filter_items", ctypes.c_uint32), ("recon_grid", ctypes.c_int),
                ("epf_grid", ctypes.c_int), ("filter_grid", ctypes.c_int),
                ("kernels_per_launch", ctypes.c_int), ("autotuned", ctypes.c_int),
                ("filter_tma", ctypes.c_int), ("kind_ms", ctypes.c_float * 3),
                ("mix", ctypes.c_uint32)]


BATCH_AUTOTUNE = 1
BATCH_PLAIN_LOADS = 2
_lib = None


def load(path=LIB_PATH):
    """Loads the shared library (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libjxlrecon.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.jxl_recon_filter_defaults.argtypes = [P(FilterParams)]
    lib.jxl_recon_filter_defaults.restype = None
    lib.jxl_recon_create.argtypes = [P(Config), P(ctypes.c_void_p)]
    lib.jxl_recon_create.restype = ctypes.c_int
    lib.jxl_recon_submit.argtypes = [ctypes.c_void_p, P(Coeffs), ctypes.c_void_p,
                                     ctypes.c_void_p, P(Cfl), P(FilterParams), P(Output),
                                     P(ctypes.c_uint64)]
    lib.jxl_recon_submit.restype = ctypes.c_int
    lib.jxl_recon_submit_xyb.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.c_void_p, P(FilterParams), P(Output),
                                         P(ctypes.c_uint64)]
    lib.jxl_recon_submit_xyb.restype = ctypes.c_int
    lib.jxl_recon_submit_jpeg.argtypes = [ctypes.c_void_p, P(JpegStream), P(Output),
                                          P(ctypes.c_uint64)]
    lib.jxl_recon_submit_jpeg.restype = ctypes.c_int
    lib.jxl_recon_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64,
                                   P(ctypes.c_double)]
    lib.jxl_recon_poll.restype = ctypes.c_int
    lib.jxl_recon_stage_ms.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_float)]
    lib.jxl_recon_stage_ms.restype = ctypes.c_int
    lib.jxl_recon_epf_stats.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_float),
                                        P(ctypes.c_uint32)]
    lib.jxl_recon_epf_stats.restype = ctypes.c_int
    lib.jxl_recon_launch_count.argtypes = [ctypes.c_void_p]
    lib.jxl_recon_launch_count.restype = ctypes.c_uint64
    lib.jxl_recon_device_bytes.argtypes = [ctypes.c_void_p]
    lib.jxl_recon_device_bytes.restype = ctypes.c_size_t
    lib.jxl_recon_destroy.argtypes = [ctypes.c_void_p]
    lib.jxl_recon_destroy.restype = ctypes.c_int
    lib.jxl_recon_last_error.argtypes = [ctypes.c_void_p]
    lib.jxl_recon_last_error.restype = ctypes.c_char_p
    lib.jxl_recon_serve.argtypes = [ctypes.c_void_p, P(Request), ctypes.c_size_t,
                                    P(ctypes.c_double), P(ctypes.c_double), P(ServeStats)]
    lib.jxl_recon_serve.restype = ctypes.c_int
    lib.jxl_recon_batch_create.argtypes = [ctypes.c_void_p, P(Request), ctypes.c_size_t,
                                           ctypes.c_int, P(ctypes.c_void_p)]
    lib.jxl_recon_batch_create.restype = ctypes.c_int
    lib.jxl_recon_batch_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.jxl_recon_batch_launch.restype = ctypes.c_int
    lib.jxl_recon_batch_query.argtypes = [ctypes.c_void_p, P(BatchInfo)]
    lib.jxl_recon_batch_query.restype = ctypes.c_int
    lib.jxl_recon_batch_status.argtypes = [ctypes.c_void_p, P(ctypes.c_uint32)]
    lib.jxl_recon_batch_status.restype = ctypes.c_int
    lib.jxl_recon_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.jxl_recon_batch_destroy.restype = ctypes.c_int
    _lib = lib
    return lib


class JxlrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def filter_defaults(lib=None, **overrides):
    lib = lib or load()
    p = FilterParams()
    lib.jxl_recon_filter_defaults(ctypes.byref(p))
    for k, v in overrides.items():
        cur = getattr(p, k)
        if isinstance(cur, ctypes.Array):
            for i, x in enumerate(v):
                cur[i] = x
        else:
            setattr(p, k, v)
    return p


def _ptr(a):
    """Address of a numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags['C_CONTIGUOUS']
        return a.ctypes.data
    return a.data_ptr()


class Context:
    """One jxl_recon_ctx.  Methods mirror the C entry points."""

    def __init__(self, device=0, max_slots=1, hbm_cap_bytes=0, timing=False, stream=None,
                 precision=PREC_FP32):
        """stream: optional raw cudaStream_t (int) every request runs on;
        precision: PREC_FP32 or PREC_TC_F16X3."""
        self.lib = load()
        cfg = Config(device, hbm_cap_bytes, max_slots, precision, int(timing), stream)
        h = ctypes.c_void_p()
        st = self.lib.jxl_recon_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        self.h = h
        self._keep = {}

    def last_error(self):
        return self.lib.jxl_recon_last_error(None).decode()

    def close(self):
        if self.h:
            self.lib.jxl_recon_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, img, params, out, out_dtype, on_device, out_on_device=True,
               out_stride=None, kx_dc=0.0, kb_dc=0.0):
        """img: dict with coeffs (3, Hp, Wp) int16, vmap, acmul, cfl, sharpness
        as numpy arrays (on_device False) or torch CUDA tensors (True)."""
        xs, ys = img['xsize'], img['ysize']
        co = img['coeffs']
        stride = co.shape[2]
        planes = (ctypes.c_void_p * 3)(*[_ptr(co[c]) for c in range(3)])
        c = Coeffs(xs, ys, planes, stride, int(on_device))
        cfl = Cfl(_ptr(img['cfl']), kx_dc, kb_dc)
        if params.epf:
            params.sharpness = _ptr(img['sharpness'])
        if out_stride is None:
            out_stride = OUT_BYTES[out_dtype] * xs
        o = Output(_ptr(out), out_stride, out_dtype, int(out_on_device))
        t = ctypes.c_uint64()
        st = self.lib.jxl_recon_submit(self.h, ctypes.byref(c), _ptr(img['vmap']),
                                       _ptr(img['acmul']), ctypes.byref(cfl),
                                       ctypes.byref(params), ctypes.byref(o), ctypes.byref(t))
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        self._keep[t.value] = (img, params, out, c, cfl, o)
        return t.value

    def submit_xyb(self, xyb, xs, ys, vmap, acmul, sharpness, params, out, out_dtype,
                   out_stride=None):
        """xyb: (3, ys, stride) float32 CUDA tensor; others CUDA tensors."""
        if params.epf:
            params.sharpness = _ptr(sharpness)
        if out_stride is None:
            out_stride = OUT_BYTES[out_dtype] * xs
        o = Output(_ptr(out), out_stride, out_dtype, 1)
        t = ctypes.c_uint64()
        st = self.lib.jxl_recon_submit_xyb(self.h, _ptr(xyb), xs, ys, xyb.shape[2],
                                           _ptr(vmap), _ptr(acmul), ctypes.byref(params),
                                           ctypes.byref(o), ctypes.byref(t))
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        self._keep[t.value] = (xyb, vmap, acmul, sharpness, params, out, o)
        return t.value

    def submit_jpeg(self, stream, out, out_dtype, on_device=True, out_on_device=True,
                    out_stride=None):
        """stream: a synth.make_jpeg dict (coeffs as CUDA tensors when
        on_device, numpy arrays otherwise; quant always numpy)."""
        xs, ys = stream['xsize'], stream['ysize']
        st = JpegStream()
        st.xsize, st.ysize = xs, ys
        comps = stream['components']
        st.num_components = len(comps)
        keep = [stream]
        for i, c in enumerate(comps):
            k = st.comp[i]
            bh, bw = c['coeffs'].shape[:2]
            k.width_in_blocks, k.height_in_blocks = bw, bh
            k.h_samp, k.v_samp = c['h_samp'], c['v_samp']
            k.coeffs = _ptr(c['coeffs'])
            q = np.ascontiguousarray(c['quant'], dtype=np.uint16)
            keep.append(q)
            k.quant = q.ctypes.data
            if c.get('gab') is not None:
                k.gab = 1
                k.gab_w1, k.gab_w2, k.gab_threshold, k.gab_limit = c['gab']
            if c.get('cond') is not None:
                k.cond = 1
                k.cond_max_gap, k.cond_min_step = c['cond']
        st.on_device = 1 if on_device else 0
        if out_stride is None:
            out_stride = OUT_BYTES[out_dtype] * xs
        o = Output(_ptr(out), out_stride, out_dtype, 1 if out_on_device else 0)
        t = ctypes.c_uint64()
        r = self.lib.jxl_recon_submit_jpeg(self.h, ctypes.byref(st), ctypes.byref(o),
                                           ctypes.byref(t))
        if r != JXLR_OK:
            raise JxlrError(r, self.last_error())
        self._keep[t.value] = (keep, st, out, o)
        return t.value

    def poll(self, ticket, timeout_us=-1):
        """Returns (status, latency_ms); raises on errors other than
        EAGAIN/ETIMEDOUT."""
        lat = ctypes.c_double()
        st = self.lib.jxl_recon_poll(self.h, ticket, timeout_us, ctypes.byref(lat))
        if st in (JXLR_EAGAIN, JXLR_ETIMEDOUT):
            return st, None
        self._keep.pop(ticket, None)
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        return st, lat.value

    def serve(self, jobs, arrival_s):
        """jobs: list of (img, params, out, out_dtype) with device-resident
        arrays (torch CUDA tensors).  Replays the arrival schedule through the
        native request loop; returns (latency_ms array, stats dict)."""
        n = len(jobs)
        reqs, keep = requests(jobs)
        arr = (ctypes.c_double * n)(*arrival_s)
        lat = (ctypes.c_double * n)()
        stats = ServeStats()
        st = self.lib.jxl_recon_serve(self.h, reqs, n, arr, lat, ctypes.byref(stats))
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        return np.array(lat[:]), _stats_dict(stats)

    def server(self, age_bound_ms=5.0, bypass=True, exclusive_mpx=0.0):
        """A request server on this context (a native thread that admits
        enqueued requests as slots and HBM free up)."""
        return Server(self, age_bound_ms, bypass, exclusive_mpx)

    def batch(self, jobs, autotune=True, plain_loads=False):
        """A multi-image batch (CUDA graph) over device-resident jobs;
        plain_loads: the filter's tiles by ordinary loads instead of TMA."""
        return Batch(self, jobs, autotune, plain_loads)

    def stage_ms(self, ticket):
        ms = (ctypes.c_float * 4)()
        st = self.lib.jxl_recon_stage_ms(self.h, ticket, ms)
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        return list(ms)

    def epf_stats(self, ticket):
        """(device ms of the J.2 kernel, 8x8 blocks it filtered) of a finished
        request of a timing context."""
        ms, n = ctypes.c_float(), ctypes.c_uint32()
        st = self.lib.jxl_recon_epf_stats(self.h, ticket, ctypes.byref(ms), ctypes.byref(n))
        if st != JXLR_OK:
            raise JxlrError(st, self.last_error())
        return float(ms.value), int(n.value)

    def launch_count(self):
        return self.lib.jxl_recon_launch_count(self.h)

    def device_bytes(self):
        return self.lib.jxl_recon_device_bytes(self.h)


def requests(jobs):
    """Request array for (img, params, out, out_dtype) device jobs, plus the
    ctypes objects that must stay alive with it."""
    n = len(jobs)
    keep = []
    reqs = (Request * n)()
    for i, (img, params, out, dtype) in enumerate(jobs):
        co = img['coeffs']
        planes = (ctypes.c_void_p * 3)(*[_ptr(co[c]) for c in range(3)])
        c = Coeffs(img['xsize'], img['ysize'], planes, co.shape[2], 1)
        cfl = Cfl(_ptr(img['cfl']), 0.0, 0.0)
        p = FilterParams()
        ctypes.pointer(p)[0] = params
        if p.epf:
            p.sharpness = _ptr(img['sharpness'])
        o = Output(_ptr(out), OUT_BYTES[dtype] * img['xsize'], dtype, 1)
        keep += [planes, c, cfl, p, o, img, out]
        reqs[i] = Request(ctypes.addressof(c), _ptr(img['vmap']), _ptr(img['acmul']),
                          ctypes.addressof(cfl), ctypes.addressof(p), ctypes.addressof(o))
    return reqs, keep


class Server:
    """jxl_recon_server_*: enqueue from any thread, wait per request."""

    def __init__(self, ctx, age_bound_ms=5.0, bypass=True, exclusive_mpx=0.0):
        self.lib = ctx.lib
        self.ctx = ctx
        h = ctypes.c_void_p()
        cfg = ServerConfig(age_bound_ms, int(bypass), exclusive_mpx)
        self.lib.jxl_recon_server_start.argtypes = [ctypes.c_void_p, ctypes.POINTER(ServerConfig),
                                                    ctypes.POINTER(ctypes.c_void_p)]
        self.lib.jxl_recon_server_enqueue.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request),
                                                      ctypes.POINTER(ctypes.c_uint64)]
        self.lib.jxl_recon_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
        self.lib.jxl_recon_server_stop.argtypes = [ctypes.c_void_p, ctypes.POINTER(ServeStats)]
        st = self.lib.jxl_recon_server_start(ctx.h, ctypes.byref(cfg), ctypes.byref(h))
        if st != JXLR_OK:
            raise JxlrError(st, ctx.last_error())
        self.h = h
        self.keep = {}
        self._lock = threading.Lock()

    def enqueue(self, job):
        """job: (img, params, out, out_dtype), device-resident; returns an id."""
        reqs, keep = requests([job])
        rid = ctypes.c_uint64()
        st = self.lib.jxl_recon_server_enqueue(self.h, reqs, ctypes.byref(rid))
        if st != JXLR_OK:
            raise JxlrError(st, self.ctx.last_error())
        with self._lock:
            self.keep[rid.value] = (reqs, keep)
        return rid.value

    def wait(self, rid, timeout_us=-1):
        """Latency in ms of request rid (completion - enqueue)."""
        lat = ctypes.c_double()
        st = self.lib.jxl_recon_server_wait(self.h, rid, timeout_us, ctypes.byref(lat))
        with self._lock:
            self.keep.pop(rid, None)
        if st != JXLR_OK:
            raise JxlrError(st, self.ctx.last_error())
        return lat.value

    def stop(self):
        stats = ServeStats()
        self.lib.jxl_recon_server_stop(self.h, ctypes.byref(stats))
        self.h = None
        return _stats_dict(stats)


class Batch:
    """jxl_recon_batch: create once, launch (graph replay) many times."""

    def __init__(self, ctx, jobs, autotune=True, plain_loads=False):
        self.ctx = ctx
        self.lib = ctx.lib
        self.reqs, self.keep = requests(jobs)
        h = ctypes.c_void_p()
        st = self.lib.jxl_recon_batch_create(ctx.h, self.reqs, len(jobs),
                                             (BATCH_AUTOTUNE if autotune else 0) |
                                             (BATCH_PLAIN_LOADS if plain_loads else 0),
                                             ctypes.byref(h))
        if st != JXLR_OK:
            raise JxlrError(st, ctx.last_error())
        self.h = h

    def launch(self, stream=0):
        st = self.lib.jxl_recon_batch_launch(self.h, stream or None)
        if st != JXLR_OK:
            raise JxlrError(st, self.ctx.last_error())

    def info(self):
        i = BatchInfo()
        self.lib.jxl_recon_batch_query(self.h, ctypes.byref(i))
        d = {k: getattr(i, k) for k, _ in BatchInfo._fields_}
        d["kind_ms"] = [round(float(v), 4) for v in i.kind_ms]
        return d

    def status(self):
        """Error flags of the launches so far (bit 8: a filter tile-load wait
        expired); call after the launch's stream completed."""
        f = ctypes.c_uint32()
        st = self.lib.jxl_recon_batch_status(self.h, ctypes.byref(f))
        if st != JXLR_OK:
            raise JxlrError(st, self.ctx.last_error())
        return f.value

    def close(self):
        if self.h:
            self.lib.jxl_recon_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_device(img, torch_module, device="cuda"):
    """Copies a synthetic image's arrays to device tensors (torch memory)."""
    t = torch_module
    out = dict(img)
    for k in ('coeffs', 'vmap', 'acmul', 'cfl', 'sharpness'):
        out[k] = t.from_numpy(np.ascontiguousarray(img[k])).to(device)
    return out


def jpeg_to_device(stream, torch_module, device="cuda"):
    """Copies a JPEG1 stream's coefficient arrays to device tensors."""
    out = dict(stream)
    out['components'] = []
    for c in stream['components']:
        d = dict(c)
        d['coeffs'] = torch_module.from_numpy(np.ascontiguousarray(c['coeffs'])).to(device)
        out['components'].append(d)
    return out


def out_shape(img, dtype):
    """(ysize, xsize, 3) output array shape and numpy dtype."""
    npd = {OUT_F32_LINEAR: np.float32, OUT_F16_LINEAR: np.float16,
           OUT_U8_SRGB: np.uint8, OUT_F32_XYB: np.float32}[dtype]
    return (img['ysize'], img['xsize'], 3), npd


def decode(ctx, img, params, dtype=OUT_F32_LINEAR, device_io=True):
    """Synchronous convenience: one image through submit + poll.  Returns a
    numpy array (ysize, xsize, 3)."""
    import torch
    shape, npd = out_shape(img, dtype)
    if device_io:
        dimg = to_device(img, torch)
        tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
        out = torch.empty(shape, dtype=tdt, device="cuda")
        t = ctx.submit(dimg, params, out, dtype, on_device=True)
        ctx.poll(t)
        return out.cpu().numpy()
    out = np.empty(shape, dtype=npd)
    t = ctx.submit(img, params, out, dtype, on_device=False, out_on_device=False)
    ctx.poll(t)
    return out


def run_noalloc(img, params, out, out_dtype, stream=0, kx_dc=0.0, kb_dc=0.0, out_stride=None):
    """jxl_recon_run_noalloc: for callers that cannot allocate device memory.
    Everything (img's arrays as torch CUDA tensors, out) is on the device;
    the work is enqueued on ``stream`` (raw cudaStream_t, 0 = legacy default
    stream) and this returns without waiting.  The library's fixed scratch
    is shared by every call: order overlapping calls on one stream."""
    lib = load()
    fn = lib.jxl_recon_run_noalloc
    P = ctypes.POINTER
    fn.argtypes = [P(Coeffs), ctypes.c_void_p, ctypes.c_void_p, P(Cfl), P(FilterParams),
                   P(Output), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    xs, ys = img['xsize'], img['ysize']
    co = img['coeffs']
    planes = (ctypes.c_void_p * 3)(*[_ptr(co[c]) for c in range(3)])
    c = Coeffs(xs, ys, planes, co.shape[2], 1)
    cfl = Cfl(_ptr(img['cfl']), kx_dc, kb_dc)
    if params.epf:
        params.sharpness = _ptr(img['sharpness'])
    if out_stride is None:
        out_stride = OUT_BYTES[out_dtype] * xs
    o = Output(_ptr(out), out_stride, out_dtype, 1)
    st = fn(ctypes.byref(c), _ptr(img['vmap']), _ptr(img['acmul']), ctypes.byref(cfl),
            ctypes.byref(params), ctypes.byref(o), stream or None)
    if st != JXLR_OK:
        lib.jxl_recon_last_error.restype = ctypes.c_char_p
        raise JxlrError(st, lib.jxl_recon_last_error(None).decode())
