"""Python binding of libosiris.so, the GB300 backward ray tracer for null
geodesics in Kerr space-time (Velasquez-Cadavid et al., "OSIRIS",
arXiv:2202.00086).

Argument marshalling only: every step of the path (initial data, Hamilton's
equations, Cash-Karp steps, stopping surfaces, observables) runs in the CUDA
kernels of the library. PyTorch provides device memory and streams. There is
no CPU fallback: if the library is missing the calls raise.

The names follow the C interface in include/osiris.h.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libosiris.so")

OK, EINVAL, ECUDA, ENOMEM, ETIMEOUT = 0, -1, -2, -3, -4
STATUS_NONE, STATUS_CAPTURED, STATUS_ESCAPED, STATUS_DISK, STATUS_MAXSTEP, STATUS_ERROR = range(6)
FP64, MIXED, DF64 = 0, 1, 2
RKCK45, RKDP45 = 0, 1
DISK_NONE, DISK_KEPLERIAN, DISK_CONSTANT_L = 0, 1, 2
SPACETIME_KERR, SPACETIME_QMETRIC = 0, 1
STATS_LEN = 16
STAT_NAMES = ["rays", "accepted", "rejected", "root_steps", "rhs_evals", "status_none",
              "status_captured", "status_escaped", "status_disk", "status_maxstep",
              "status_error", "max_abs_H_bits", "fp64_steps"]

_P = ctypes.POINTER
_d = ctypes.c_double
_vp = ctypes.c_void_p


class TraceOpts(ctypes.Structure):
    _fields_ = [("tol", _d), ("max_steps", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("r_cap_factor", _d), ("r_esc_factor", _d),
                ("cell_deg", _d), ("cell_phase_deg", _d), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("stats", _vp), ("workspace", _vp),
                ("workspace_bytes", ctypes.c_size_t), ("integrator", ctypes.c_int32),
                ("rays_per_lane", ctypes.c_int32), ("refill_lanes", ctypes.c_int32)]


OUTPUT_FIELDS = [("status", torch.uint8), ("r", torch.float64), ("theta", torch.float64),
                 ("phi", torch.float64), ("max_abs_H", torch.float64), ("steps", torch.int32),
                 ("cell_i", torch.int16), ("cell_j", torch.int16), ("parity", torch.uint8),
                 ("g", torch.float64), ("intensity", torch.float64), ("r_hit", torch.float64)]
SHADOW_FIELDS = ["status", "r", "theta", "phi", "max_abs_H", "steps", "cell_i", "cell_j",
                 "parity"]
DISK_FIELDS = SHADOW_FIELDS + ["g", "intensity", "r_hit"]


class Outputs(ctypes.Structure):
    _fields_ = [(name, _vp) for name, _ in OUTPUT_FIELDS]


class Request(ctypes.Structure):
    _fields_ = [("camera", _vp), ("disk", ctypes.c_int32), ("r_in", _d), ("r_out", _d),
                ("tol", _d), ("out", Outputs), ("first_ray", ctypes.c_int64),
                ("n_rays", ctypes.c_int64), ("l0", _d)]


LIB_CHECKED_PATH = os.path.join(_HERE, "_build", "libosiris_checked.so")

_lib = None


def lib():
    """The loaded libosiris.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        _lib = load(LIB_PATH)
    return _lib


def load(path):
    """Load one build of the library (libosiris.so, or its bounds-checked twin
    libosiris_checked.so) with the argument types of every entry point."""
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = ctypes.CDLL(path)
    L.osiris_default_opts.argtypes = [_P(TraceOpts)]
    L.osiris_init_camera.argtypes = [_P(_vp), _d, _d, _d, _d, _d, _d, _d, ctypes.c_int32,
                                     ctypes.c_int32]
    L.osiris_init_camera_q.argtypes = [_P(_vp), _d, _d, _d, _d, _d, _d, _d, ctypes.c_int32,
                                       ctypes.c_int32]
    L.osiris_trace_states_ex.argtypes = [ctypes.c_int32, _d, _d, _d, _vp, _vp, _vp,
                                         ctypes.c_int64, ctypes.c_int32, _d, _d,
                                         _P(TraceOpts), _P(Outputs), _vp]
    L.osiris_destroy_camera.argtypes = [_vp]
    L.osiris_camera_rays.argtypes = [_vp]
    L.osiris_camera_rays.restype = ctypes.c_int64
    L.osiris_trace.argtypes = [_vp, _P(TraceOpts), _P(Outputs), _vp]
    L.osiris_render_disk.argtypes = [_vp, _d, _d, _P(TraceOpts), _P(Outputs), _vp]
    L.osiris_render_disk_l0.argtypes = [_vp, _d, _d, _d, _P(TraceOpts), _P(Outputs), _vp]
    L.osiris_workspace_bytes.argtypes = [ctypes.c_int32]
    L.osiris_workspace_bytes.restype = ctypes.c_size_t
    L.osiris_trace_batch.argtypes = [_P(Request), ctypes.c_int32, _P(TraceOpts), _vp]
    L.osiris_batch_plan_create.argtypes = [_P(_vp), ctypes.c_int32, ctypes.c_int32,
                                           _P(TraceOpts)]
    L.osiris_batch_plan_launch.argtypes = [_vp, _P(Request), ctypes.c_int32, _vp]
    L.osiris_batch_plan_destroy.argtypes = [_vp]
    L.osiris_trace_states.argtypes = [_d, _d, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32,
                                      _d, _d, _P(TraceOpts), _P(Outputs), _vp]
    L.osiris_copy_outputs_to_host.argtypes = [_P(Outputs), _P(Outputs), ctypes.c_int64, _vp]
    L.osiris_isco.argtypes = [_d]
    L.osiris_isco.restype = _d
    L.osiris_horizon.argtypes = [_d]
    L.osiris_horizon.restype = _d
    L.osiris_fma_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _vp,
                                   _P(_d), _vp]
    L.osiris_pipe_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_int32, _vp, _P(_d), _vp]
    L.osiris_pipe_probe_threads.argtypes = [ctypes.c_int32, ctypes.c_int32]
    L.osiris_pipe_probe_threads.restype = ctypes.c_int64
    L.osiris_strerror.argtypes = [ctypes.c_int]
    L.osiris_strerror.restype = ctypes.c_char_p
    L.osiris_stream_wait.argtypes = [_vp, _d]
    return L


class using_library:
    """Context manager: route every call of this module through another
    loaded build (e.g. load(LIB_CHECKED_PATH)) and restore the default after.
    Cameras must be created inside the block (their handles belong to the
    build that made them)."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        global _lib
        self.prev = lib()
        _lib = self.L
        return self.L

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev
        return False


class OsirisError(RuntimeError):
    def __init__(self, code, what):
        msg = lib().osiris_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (what, msg, code))
        self.code = code


def _check(code, what):
    if code != OK:
        raise OsirisError(code, what)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream)


class Camera:
    """Observer at (r_obs, incl_deg), image plane extent (x_min, x_max, y_min,
    y_max) with nx x ny pixels (osiris_init_camera)."""

    def __init__(self, a, r_obs, incl_deg, extent, nx, ny, q=None):
        """Kerr camera with spin a; with q given, a q-metric camera
        (osiris_init_camera_q, a is ignored)."""
        h = _vp()
        x0, x1, y0, y1 = (float(v) for v in extent)
        if q is None:
            _check(lib().osiris_init_camera(ctypes.byref(h), float(a), float(r_obs),
                                            float(incl_deg), x0, x1, y0, y1, int(nx), int(ny)),
                   "osiris_init_camera")
        else:
            _check(lib().osiris_init_camera_q(ctypes.byref(h), float(q), float(r_obs),
                                              float(incl_deg), x0, x1, y0, y1, int(nx),
                                              int(ny)), "osiris_init_camera_q")
        self.q = q
        self._h = h
        self.a, self.r_obs, self.incl_deg = float(a), float(r_obs), float(incl_deg)
        self.extent, self.nx, self.ny = (x0, x1, y0, y1), int(nx), int(ny)

    @property
    def handle(self):
        return self._h

    @property
    def n_rays(self):
        return self.nx * self.ny

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.osiris_destroy_camera(h)
            self._h = None

    @classmethod
    def from_render(cls, rd):
        return cls(rd["a"], rd["r_obs"], rd["incl_deg"], rd["extent"], rd["nx"], rd["ny"],
                   q=rd.get("q"))


def workspace_bytes(n_requests=1):
    return int(lib().osiris_workspace_bytes(int(n_requests)))


def make_opts(tol=1e-10, max_steps=1_000_000, precision=FP64, persistent=False,
              r_cap_factor=1.01, r_esc_factor=1.1, cell_deg=10.0, cell_phase_deg=0.0,
              block_size=0, blocks_per_sm=0, stats=None, workspace=None, integrator=RKCK45,
              rays_per_lane=0, refill_lanes=0):
    o = TraceOpts()
    lib().osiris_default_opts(ctypes.byref(o))
    o.tol, o.max_steps = float(tol), int(max_steps)
    o.precision = int(precision)
    o.persistent = 1 if persistent else 0
    o.r_cap_factor, o.r_esc_factor = float(r_cap_factor), float(r_esc_factor)
    o.cell_deg, o.cell_phase_deg = float(cell_deg), float(cell_phase_deg)
    o.block_size, o.blocks_per_sm = int(block_size), int(blocks_per_sm)
    o.integrator = int(integrator)
    o.rays_per_lane, o.refill_lanes = int(rays_per_lane), int(refill_lanes)
    o.stats = stats.data_ptr() if stats is not None else None
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def alloc_outputs(n, device="cuda", fields=SHADOW_FIELDS, pin_memory=False):
    """Dict of output tensors (one entry per ray) for the given fields."""
    dt = dict(OUTPUT_FIELDS)
    if str(device) == "cpu":
        return {f: torch.empty(n, dtype=dt[f], pin_memory=pin_memory) for f in fields}
    return {f: torch.empty(n, dtype=dt[f], device=device) for f in fields}


def outputs_struct(d):
    o = Outputs()
    for name, _ in OUTPUT_FIELDS:
        t = d.get(name) if d else None
        setattr(o, name, t.data_ptr() if t is not None else None)
    return o


def new_stats(device="cuda"):
    return torch.zeros(STATS_LEN, dtype=torch.int64, device=device)


def trace(camera, out=None, stream=None, **opts):
    """Shadow / lensing render of every pixel (osiris_trace)."""
    if out is None:
        out = alloc_outputs(camera.n_rays)
    o = make_opts(**opts)
    os_ = outputs_struct(out)
    _check(lib().osiris_trace(camera.handle, ctypes.byref(o), ctypes.byref(os_),
                              _stream_handle(stream)), "osiris_trace")
    return out


def render_disk(camera, r_in, r_out, out=None, stream=None, l0=None, **opts):
    """Thin-disk render: Keplerian (osiris_render_disk) or, with l0, a disk of
    constant specific angular momentum (osiris_render_disk_l0)."""
    if out is None:
        out = alloc_outputs(camera.n_rays, fields=DISK_FIELDS)
    o = make_opts(**opts)
    os_ = outputs_struct(out)
    if l0 is None:
        _check(lib().osiris_render_disk(camera.handle, float(r_in), float(r_out),
                                        ctypes.byref(o), ctypes.byref(os_),
                                        _stream_handle(stream)), "osiris_render_disk")
    else:
        _check(lib().osiris_render_disk_l0(camera.handle, float(r_in), float(r_out), float(l0),
                                           ctypes.byref(o), ctypes.byref(os_),
                                           _stream_handle(stream)), "osiris_render_disk_l0")
    return out


def request_array(requests):
    """ctypes array of osiris_request from dicts with keys camera, disk (bool),
    r_in, r_out, tol (<= 0: the opts tol), out (dict of device tensors of the
    whole render) and optionally first_ray / n_rays (a pixel range)."""
    n = len(requests)
    arr = (Request * max(1, n))()
    for k, q in enumerate(requests):
        arr[k].camera = q["camera"].handle
        dk = q.get("disk")
        arr[k].disk = (DISK_NONE if not dk else
                       DISK_CONSTANT_L if q.get("l0") is not None else DISK_KEPLERIAN)
        arr[k].l0 = float(q.get("l0") or 0.0)
        arr[k].r_in = float(q.get("r_in") or 0.0)
        arr[k].r_out = float(q.get("r_out") or 0.0)
        arr[k].tol = float(q.get("tol") or 0.0)
        arr[k].out = outputs_struct(q["out"])
        arr[k].first_ray = int(q.get("first_ray") or 0)
        arr[k].n_rays = int(q.get("n_rays") or 0)
    return arr


def trace_batch(requests, stream=None, **opts):
    """One persistent launch over many renders (osiris_trace_batch).

    requests: see request_array. opts must include a workspace tensor of at
    least workspace_bytes(len(requests)) bytes."""
    n = len(requests)
    arr = request_array(requests)
    o = make_opts(**opts)
    _check(lib().osiris_trace_batch(arr, n, ctypes.byref(o), _stream_handle(stream)),
           "osiris_trace_batch")
    return requests


class BatchPlan:
    """A batched persistent launch recorded as a CUDA graph and replayed per
    batch (osiris_batch_plan_*): create once with the plan's fixed options
    (workspace of workspace_bytes(max_requests) bytes, precision, integrator,
    launch shape, ...), then launch(requests) for each round. The plan keeps
    the workspace tensor alive; launches of one plan must go to one stream."""

    def __init__(self, max_requests, spacetime=None, **opts):
        if spacetime is None:
            spacetime = SPACETIME_KERR
        self._opts = make_opts(**opts)
        self._keep = opts.get("workspace"), opts.get("stats")
        self.max_requests = int(max_requests)
        h = _vp()
        _check(lib().osiris_batch_plan_create(ctypes.byref(h), self.max_requests, int(spacetime),
                                              ctypes.byref(self._opts)),
               "osiris_batch_plan_create")
        self._h = h

    def launch(self, requests, stream=None):
        """Trace the requests (see request_array) in one graph launch."""
        arr = request_array(requests)
        _check(lib().osiris_batch_plan_launch(self._h, arr, len(requests),
                                              _stream_handle(stream)),
               "osiris_batch_plan_launch")
        return requests

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.osiris_batch_plan_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


def trace_batch_static(requests, stream=None, **opts):
    """osiris_trace_batch_static: like trace_batch, but the queue and request
    table live in the library's fixed device array, so no workspace tensor
    is needed (any `workspace` option is ignored). At most
    OSIRIS_STATIC_MAX_REQUESTS (256) requests per call."""
    L = lib()
    fn = L.osiris_trace_batch_static
    fn.argtypes = [_P(Request), ctypes.c_int32, _P(TraceOpts), _vp]
    n = len(requests)
    arr = request_array(requests)
    o = make_opts(**opts)
    _check(fn(arr, n, ctypes.byref(o), _stream_handle(stream)), "osiris_trace_batch_static")
    return requests


def trace_states(a, r_obs, states, E, L, out=None, disk=False, r_in=0.0, r_out=0.0,
                 stream=None, q=None, mass2=0.0, **opts):
    """Trace rays from explicit device initial data (osiris_trace_states_ex):
    Kerr with spin a, or the q-metric when q is given; mass2 = 0 for light,
    1 for unit-mass particles (H = -1/2)."""
    n = int(E.numel())
    assert states.is_cuda and states.dtype == torch.float64 and states.is_contiguous()
    assert E.is_cuda and L.is_cuda and E.dtype == torch.float64 and L.dtype == torch.float64
    if out is None:
        out = alloc_outputs(n, fields=DISK_FIELDS if disk else SHADOW_FIELDS)
    o = make_opts(**opts)
    os_ = outputs_struct(out)
    sp, param = (SPACETIME_QMETRIC, float(q)) if q is not None else (SPACETIME_KERR, float(a))
    _check(lib().osiris_trace_states_ex(sp, param, float(r_obs), float(mass2),
                                        states.data_ptr(), E.data_ptr(), L.data_ptr(), n,
                                        1 if disk else 0, float(r_in), float(r_out),
                                        ctypes.byref(o), ctypes.byref(os_),
                                        _stream_handle(stream)), "osiris_trace_states_ex")
    return out


def stream_wait(timeout_s, stream=None):
    """Bounded wait for the work queued on the stream (osiris_stream_wait):
    returns OK when it is complete or ETIMEOUT when timeout_s ran out first;
    raises on a stream error."""
    rc = lib().osiris_stream_wait(_stream_handle(stream), float(timeout_s))
    if rc not in (OK, ETIMEOUT):
        _check(rc, "osiris_stream_wait")
    return rc


def copy_outputs_to_host(dev, host, n, stream=None):
    """Asynchronous device-to-host copy of every field present in both dicts."""
    d = outputs_struct(dev)
    h = outputs_struct(host)
    _check(lib().osiris_copy_outputs_to_host(ctypes.byref(d), ctypes.byref(h), int(n),
                                             _stream_handle(stream)),
           "osiris_copy_outputs_to_host")
    return host


def isco(a):
    return float(lib().osiris_isco(float(a)))


def horizon(a):
    return float(lib().osiris_horizon(float(a)))


PROBE_FMA, PROBE_MUL, PROBE_ADD, PROBE_MUL_AS_FMA, PROBE_ADD_AS_FMA = 0, 1, 2, 3, 4


def pipe_probe_threads(precision, op=PROBE_FMA):
    """Threads that fill every SM of the current device with resident probe
    blocks (osiris_pipe_probe_threads)."""
    n = int(lib().osiris_pipe_probe_threads(int(precision), int(op)))
    _check(min(n, 0), "osiris_pipe_probe_threads")
    return n


def pipe_probe(precision, op, n_threads, iters, out, stream=None):
    """Launch one pipe probe (osiris_pipe_probe); returns the launch's
    floating-point operation count."""
    fl = _d()
    _check(lib().osiris_pipe_probe(int(precision), int(op), int(n_threads), int(iters),
                                   out.data_ptr(), ctypes.byref(fl), _stream_handle(stream)),
           "osiris_pipe_probe")
    return fl.value


def fma_probe(precision, n_threads, iters, out, stream=None):
    """Launch the FMA throughput probe; returns the launch's flop count."""
    fl = _d()
    _check(lib().osiris_fma_probe(int(precision), int(n_threads), int(iters), out.data_ptr(),
                                  ctypes.byref(fl), _stream_handle(stream)), "osiris_fma_probe")
    return fl.value


def decode_stats(stats):
    """Counters of a stats tensor as a dict (max |H| decoded from its bits)."""
    v = stats.detach().cpu().tolist()
    out = {name: int(v[k]) for k, name in enumerate(STAT_NAMES)}
    out["max_abs_H"] = ctypes.cast(ctypes.pointer(ctypes.c_int64(v[11])),
                                   _P(_d)).contents.value
    return out


def resolve_r_in(render_dict):
    """r_in of a workload render, with the ISCO marker resolved by the library."""
    r_in = render_dict.get("r_in")
    if r_in == "isco":
        return isco(render_dict["a"])
    return r_in
