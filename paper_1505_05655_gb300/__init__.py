"""lutc: detector LUT generation and LUT-based image correction on GB300 (sm_103a).

Python face of the C ABI declared in ``include/lutc.h``.  Each function
mirrors one entry point of the same name (without the ``lutc_`` prefix) and
only marshals arguments: rasters are CUDA ``torch.uint16`` tensors
``[bands, height, width]`` (rows contiguous, bands stacked at height * row
pitch), coefficients are CUDA ``torch.int32`` tensors ``[bands, width]``,
tables are CUDA tensors of the dtypes the header states.  Work is enqueued
on ``stream`` (default: torch's current stream).
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import (LUTC_MAX_BANDS, LUTC_STRETCH, Coeffs, LutcError, Raster, check, lib)
from . import net  # noqa: E402,F401  (the TCP transport's client side)

__all__ = ["LutcError", "lib", "version", "lutgen", "apply_u16", "hist", "stretch", "compose", "apply_u8",
           "correct_image_workspace", "correct_image_tables", "correct_image", "apply_stretch", "trace_enable",
           "trace_read", "raster_desc", "coeff_descs", "set_tuning", "reset_tuning", "get_tuning", "Batch",
           "batch_autotune", "Server", "submit", "fit", "demosaic", "correct_image_host", "correct_frames_host",
           "net",
           "device_info"]


def _stream(stream, dev):
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _need(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
        raise TypeError("%s must be a CUDA %s tensor" % (name, dtype))


def version() -> int:
    return lib().lutc_version()


def raster_desc(raw: torch.Tensor, bits: int) -> Raster:
    """lutc_raster of a ``[bands, H, W]`` (or ``[H, W]``) uint16 CUDA tensor."""
    _need(raw, torch.uint16, "raw")
    if raw.dim() == 2:
        raw = raw.unsqueeze(0)
    if raw.dim() != 3:
        raise ValueError("raw must be [bands, height, width]")
    bands, h, w = raw.shape
    if raw.numel() == 0:
        return Raster(raw.data_ptr(), 2 * w, w, h, bands, bits)
    if raw.stride(2) != 1:
        raise ValueError("raw must be [bands, height, width] with contiguous rows")
    if bands > 1 and h > 0 and raw.stride(0) != h * raw.stride(1):
        raise ValueError("bands must be stacked at height * row pitch")
    return Raster(raw.data_ptr(), raw.stride(1) * 2, w, h, bands, bits)


def coeff_descs(A: torch.Tensor, G: torch.Tensor, O: torch.Tensor):
    """Host array of lutc_coeffs, one per band, for ``[bands, W]`` int32 CUDA tensors."""
    for t, n in ((A, "A"), (G, "G"), (O, "O")):
        _need(t, torch.int32, n)
    if A.dim() == 1:
        A, G, O = A.unsqueeze(0), G.unsqueeze(0), O.unsqueeze(0)
    bands, w = A.shape
    arr = (Coeffs * bands)()
    for b in range(bands):
        for t in (A[b], G[b], O[b]):
            if not t.is_contiguous():
                raise ValueError("coefficient rows must be contiguous")
        arr[b] = Coeffs(A[b].data_ptr(), G[b].data_ptr(), O[b].data_ptr(), w)
    return arr


def lutgen(A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int, out: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """Detector LUT ``[ncols, 2^bits]`` uint16 of one band."""
    desc = coeff_descs(A, G, O)
    if out is None:
        out = torch.empty((desc[0].ncols, 1 << bits), dtype=torch.uint16, device=A.device)
    _need(out, torch.uint16, "out")
    check(lib().lutc_lutgen(ctypes.byref(desc[0]), bits, out.data_ptr(), _stream(stream, A.device)), "lutc_lutgen")
    return out


def _out_like(raw: torch.Tensor, dtype, out):
    shape = raw.shape if raw.dim() == 3 else (1, *raw.shape)
    if out is None:
        out = torch.empty(shape, dtype=dtype, device=raw.device)
    _need(out, dtype, "out")
    o3 = out if out.dim() == 3 else out.unsqueeze(0)
    if out.numel() == 0:
        return out, o3.shape[2] * out.element_size()
    if o3.stride(2) != 1 or (o3.shape[0] > 1 and o3.shape[1] > 0 and o3.stride(0) != o3.shape[1] * o3.stride(1)):
        raise ValueError("out must be [bands, height, width] with contiguous rows stacked at height * pitch")
    return out, o3.stride(1) * out.element_size()


def apply_u16(raw: torch.Tensor, lut: torch.Tensor, bits: int, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """out = lut[b][c][min(raw, M)] with a materialised ``[bands, W, 2^bits]`` uint16 LUT."""
    desc = raster_desc(raw, bits)
    _need(lut, torch.uint16, "lut")
    out, pitch = _out_like(raw, torch.uint16, out)
    check(lib().lutc_apply_u16(ctypes.byref(desc), lut.data_ptr(), out.data_ptr(), pitch,
                               _stream(stream, raw.device)), "lutc_apply_u16")
    return out


def hist(raw: torch.Tensor, A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int,
         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per-band histogram ``[bands, 2^bits]`` uint64 of the detector-corrected raster."""
    desc = raster_desc(raw, bits)
    cd = coeff_descs(A, G, O)
    if out is None:
        out = torch.empty((desc.bands, 1 << bits), dtype=torch.uint64, device=raw.device)
    _need(out, torch.uint64, "out")
    check(lib().lutc_hist(ctypes.byref(desc), cd, out.data_ptr(), _stream(stream, raw.device)), "lutc_hist")
    return out


def stretch(hist_: torch.Tensor, bits: int, S: torch.Tensor | None = None, lohi: torch.Tensor | None = None,
            stream=None):
    """(S ``[bands, 2^bits]`` uint8, lohi ``[bands, 2]`` int32) of per-band histograms."""
    _need(hist_, torch.uint64, "hist")
    h2 = hist_ if hist_.dim() == 2 else hist_.unsqueeze(0)
    bands = h2.shape[0]
    if S is None:
        S = torch.empty((bands, 1 << bits), dtype=torch.uint8, device=hist_.device)
    if lohi is None:
        lohi = torch.empty((bands, 2), dtype=torch.int32, device=hist_.device)
    check(lib().lutc_stretch(hist_.data_ptr(), bands, bits, S.data_ptr(), lohi.data_ptr(),
                             _stream(stream, hist_.device)), "lutc_stretch")
    return S, lohi


def compose(lut: torch.Tensor, S: torch.Tensor, bits: int, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """Composed per-column LUT ``[ncols, 2^bits]`` uint8 of one band."""
    _need(lut, torch.uint16, "lut")
    _need(S, torch.uint8, "S")
    ncols = lut.shape[0]
    if out is None:
        out = torch.empty((ncols, 1 << bits), dtype=torch.uint8, device=lut.device)
    check(lib().lutc_compose(lut.data_ptr(), S.data_ptr(), ncols, bits, out.data_ptr(),
                             _stream(stream, lut.device)), "lutc_compose")
    return out


def apply_u8(raw: torch.Tensor, clut: torch.Tensor, bits: int, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """out8 = clut[b][c][min(raw, M)] with a materialised ``[bands, W, 2^bits]`` uint8 table."""
    desc = raster_desc(raw, bits)
    _need(clut, torch.uint8, "clut")
    out, pitch = _out_like(raw, torch.uint8, out)
    check(lib().lutc_apply_u8(ctypes.byref(desc), clut.data_ptr(), out.data_ptr(), pitch,
                              _stream(stream, raw.device)), "lutc_apply_u8")
    return out


def correct_image_workspace(desc: Raster) -> int:
    return int(lib().lutc_correct_image_workspace(ctypes.byref(desc)))


def correct_image_tables(desc: Raster):
    h, s, l = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    check(lib().lutc_correct_image_tables(ctypes.byref(desc), ctypes.byref(h), ctypes.byref(s), ctypes.byref(l)),
          "lutc_correct_image_tables")
    return h.value, s.value, l.value


def correct_image(raw: torch.Tensor, A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int,
                  stretch: bool = True, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                  stream=None, with_tables: bool = False):
    """The fused correction (uint8 with ``stretch``, else uint16).

    With ``with_tables`` also returns ``(hist [bands, 2^bits] uint64, S [bands, 2^bits] uint8,
    lohi [bands, 2] int32)`` as views into the workspace.
    """
    desc = raster_desc(raw, bits)
    cd = coeff_descs(A, G, O)
    out, pitch = _out_like(raw, torch.uint8 if stretch else torch.uint16, out)
    need = correct_image_workspace(desc)
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=raw.device)
    _need(workspace, torch.uint8, "workspace")
    check(lib().lutc_correct_image(ctypes.byref(desc), cd, LUTC_STRETCH if stretch else 0, out.data_ptr(), pitch,
                                   workspace.data_ptr(), workspace.numel(), _stream(stream, raw.device)),
          "lutc_correct_image")
    if not with_tables:
        return out
    ho, so, lo = correct_image_tables(desc)
    L = 1 << bits
    bands = desc.bands
    hist_ = workspace[ho:ho + bands * L * 8].view(torch.uint64).view(bands, L)
    S = workspace[so:so + bands * L].view(bands, L)
    lohi = workspace[lo:lo + bands * 8].view(torch.int32).view(bands, 2)
    return out, (hist_, S, lohi)


def apply_stretch(raw: torch.Tensor, A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int,
                  S: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Pass 2 alone: out8 = S[b][D[b][c][raw]] for a given ``[bands, 2^bits]`` uint8 S."""
    desc = raster_desc(raw, bits)
    cd = coeff_descs(A, G, O)
    _need(S, torch.uint8, "S")
    out, pitch = _out_like(raw, torch.uint8, out)
    check(lib().lutc_apply_stretch(ctypes.byref(desc), cd, S.data_ptr(), out.data_ptr(), pitch,
                                   _stream(stream, raw.device)), "lutc_apply_stretch")
    return out


def trace_enable(capacity: int) -> None:
    """Record per-phase CUDA events in the next ``capacity`` fused corrections (0 disables)."""
    check(lib().lutc_trace_enable(int(capacity)), "lutc_trace_enable")


def trace_read(max_calls: int):
    """Per-call phase durations in ms, ``[[pass1, scan, pass2], ...]``; starts a new trace."""
    buf = (ctypes.c_float * (3 * max(1, max_calls)))()
    n = lib().lutc_trace_read(buf, int(max_calls))
    if n < 0:
        check(n, "lutc_trace_read")
    return [[buf[3 * i + p] for p in range(3)] for i in range(n)]


def set_tuning(bits: int, path: int = 0, column_threads: int = 0, blocks_per_sm: int = 0) -> None:
    """Process-wide launch configuration for ``bits`` (all zeros = automatic)."""
    from ._lib import Tuning
    t = Tuning(path, column_threads, blocks_per_sm)
    check(lib().lutc_set_tuning(bits, ctypes.byref(t)), "lutc_set_tuning")


def reset_tuning(bits: int) -> None:
    check(lib().lutc_set_tuning(bits, None), "lutc_set_tuning")


def get_tuning(bits: int):
    from ._lib import Tuning
    t = Tuning()
    check(lib().lutc_get_tuning(bits, ctypes.byref(t)), "lutc_get_tuning")
    return (t.path, t.column_threads, t.blocks_per_sm)


def last_path() -> int:
    """Kernel family (LUTC_PATH_TMA or LUTC_PATH_STRIP) of this thread's last pass-kernel call, 0 before any."""
    p = ctypes.c_int(-1)
    check(lib().lutc_last_path(ctypes.byref(p)), "lutc_last_path")
    return p.value


class Batch:
    """A prepared batch of independent corrections (``lutc_batch_*``).

    ``images`` is a list of ``(raw, A, G, O, bits, out, stretch)`` with CUDA
    tensors as for :func:`correct_image`.  The tensors must outlive the batch.
    The workspace is allocated here (torch) and passed to the library.
    """

    def __init__(self, images, column_threads: int = 0, blocks_per_sm: int = 0, use_graph: bool = True,
                 stream=None, config=None):
        from ._lib import BatchConfig
        self.jobs, self._keep, self.device = _batch_jobs(images)
        n = self.n = len(images)
        self.workspace = _batch_workspace(self.jobs, n, self.device)
        if config is None:
            config = BatchConfig(column_threads, blocks_per_sm, 1 if use_graph else 0)
        self.config = config
        self._h = ctypes.c_void_p()
        check(lib().lutc_batch_create(self.jobs, n, ctypes.byref(config), self.workspace.data_ptr(),
                                      self.workspace.numel(), _stream(stream, self.device), ctypes.byref(self._h)),
              "lutc_batch_create")

    def run(self, stream=None) -> None:
        check(lib().lutc_batch_run(self._h, _stream(stream, self.device)), "lutc_batch_run")

    def outputs(self):
        return [k[5] for k in self._keep]

    def tables(self, i: int, bands: int, bits: int):
        """(hist [bands, 2^bits] uint64, S [bands, 2^bits] uint8, lohi [bands, 2] int32) of image i, as host arrays."""
        import numpy as np
        h, s, l = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        check(lib().lutc_batch_tables(self._h, i, ctypes.byref(h), ctypes.byref(s), ctypes.byref(l)),
              "lutc_batch_tables")
        L = 1 << bits
        base = self.workspace.data_ptr()
        ws = self.workspace
        hist_ = ws[h.value - base:h.value - base + bands * L * 8].view(torch.uint64).view(bands, L)
        S = ws[s.value - base:s.value - base + bands * L].view(bands, L)
        lohi = ws[l.value - base:l.value - base + bands * 8].view(torch.int32).view(bands, 2)
        return hist_.cpu().numpy(), S.cpu().numpy(), lohi.cpu().numpy()

    def close(self) -> None:
        if self._h:
            lib().lutc_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_jobs(images):
    """(lutc_job array, the objects it points into, device) for ``(raw, A, G, O, bits, out, stretch)`` tuples."""
    from ._lib import Job
    keep = []
    jobs = (Job * max(1, len(images)))()
    dev = None
    for i, (raw, A, G, O, bits, out, stretch) in enumerate(images):
        desc = raster_desc(raw, bits)
        cd = coeff_descs(A, G, O)
        out_t, pitch = _out_like(raw, torch.uint8 if stretch else torch.uint16, out)
        keep.append((cd, raw, A, G, O, out_t))
        jobs[i] = Job(desc, ctypes.cast(cd, ctypes.POINTER(Coeffs)), out_t.data_ptr(), pitch,
                      LUTC_STRETCH if stretch else 0)
        dev = raw.device
    return jobs, keep, dev if dev is not None else torch.device("cuda")


def _batch_workspace(jobs, n: int, device) -> torch.Tensor:
    need = int(lib().lutc_batch_workspace(jobs, n))
    if need == 0 and n > 0:
        raise LutcError(-1, "lutc_batch_workspace")
    return torch.empty(max(need, 256), dtype=torch.uint8, device=device)


def batch_correct(images, config=None, workspace: torch.Tensor | None = None, stream=None):
    """The whole batch in one call (``lutc_batch_correct``); returns the outputs.  ``images`` as for
    :class:`Batch`; ``config`` a ``BatchConfig`` (for instance from :func:`batch_autotune`) or None."""
    jobs, keep, dev = _batch_jobs(images)
    n = len(images)
    if workspace is None:
        workspace = _batch_workspace(jobs, n, dev)
    check(lib().lutc_batch_correct(jobs, n, ctypes.byref(config) if config is not None else None,
                                   workspace.data_ptr(), workspace.numel(), _stream(stream, dev)),
          "lutc_batch_correct")
    return [k[5] for k in keep]


def batch_autotune(images, reps: int = 3, stream=None):
    """Times every batch launch configuration on these images; returns (BatchConfig, ms)."""
    from ._lib import BatchConfig
    b = Batch(images, use_graph=False, stream=stream)
    best = BatchConfig()
    ms = ctypes.c_float()
    try:
        check(lib().lutc_batch_autotune(b.jobs, b.n, b.workspace.data_ptr(), b.workspace.numel(),
                                        _stream(stream, b.device), reps, ctypes.byref(best), ctypes.byref(ms)),
              "lutc_batch_autotune")
    finally:
        b.close()
    return best, ms.value


class Server:
    """The in-process request loop (``lutc_server_*``).

    ``submit`` takes a sensor id, a raster (CUDA uint16 tensor, or a host
    numpy/pinned tensor with ``host=True``) of ``[bands, H, W]`` and an output
    of ``[bands, H, W]`` uint8, and returns a ticket; ``wait`` returns the
    request's :class:`RequestInfo`.  Buffers must stay alive until then.
    """

    def __init__(self, budget_bytes: int = 0, max_batch: int = 0, max_wait_us: int = 0, streams: int = 0,
                 max_queue: int = 0, fake_device: bool = False, fake_latency_us: int = 0, fail_every: int = 0,
                 hold_when_idle: bool = False):
        from ._lib import ServerConfig
        self.cfg = ServerConfig(budget_bytes, max_batch, max_wait_us, streams, max_queue, int(fake_device),
                                fake_latency_us, fail_every, int(hold_when_idle))
        self._h = ctypes.c_void_p()
        self._keep = {}
        check(lib().lutc_server_create(ctypes.byref(self.cfg), ctypes.byref(self._h)), "lutc_server_create")

    def register_sensor(self, sensor_id: int, width: int, bands: int, bits: int, A, G, O) -> None:
        import numpy as np
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(bands, width)) for a in (A, G, O)]
        check(lib().lutc_server_register_sensor(self._h, sensor_id, width, bands, bits, arrs[0].ctypes.data,
                                                arrs[1].ctypes.data, arrs[2].ctypes.data),
              "lutc_server_register_sensor")

    @staticmethod
    def _addr_pitch(t, elem):
        """(address, row pitch in bytes) of a [bands, H, W] buffer whose bands are stacked at H x pitch."""
        import numpy as np
        if isinstance(t, np.ndarray):
            if t.ndim == 3 and t.shape[0] > 1 and t.strides[0] != t.shape[1] * t.strides[1]:
                raise ValueError("bands must be stacked at rows x pitch")
            return t.ctypes.data, t.strides[-2] if t.ndim >= 2 else t.shape[-1] * elem
        if t.dim() == 3 and t.numel() > 0:
            if t.shape[0] > 1 and t.stride(0) != t.shape[1] * t.stride(1):
                raise ValueError("bands must be stacked at rows x pitch")
            return t.data_ptr(), t.stride(1) * elem
        return t.data_ptr(), t.shape[-1] * elem

    def submit(self, sensor_id: int, raw, out, host: bool = False, keep=None) -> int:
        """Queues a request; returns its ticket (raises LutcError on refusal, e.g. LUTC_EBUSY)."""
        from ._lib import LUTC_REQ_HOST
        ip, pitch = self._addr_pitch(raw, 2)
        op, opitch = self._addr_pitch(out, 1)
        h = raw.shape[-2]
        t = ctypes.c_uint64()
        rc = lib().lutc_server_submit(self._h, sensor_id, ip, h, pitch, op, opitch, LUTC_REQ_HOST if host else 0,
                                      ctypes.byref(t))
        check(rc, "lutc_server_submit")
        self._keep[t.value] = (raw, out, keep)
        return t.value

    def try_submit(self, sensor_id: int, raw, out, host: bool = False):
        """Like submit, but returns (status, ticket) instead of raising."""
        from ._lib import LUTC_REQ_HOST
        ip, pitch = self._addr_pitch(raw, 2)
        op, opitch = self._addr_pitch(out, 1)
        t = ctypes.c_uint64()
        rc = lib().lutc_server_submit(self._h, sensor_id, ip, raw.shape[-2], pitch, op, opitch,
                                      LUTC_REQ_HOST if host else 0, ctypes.byref(t))
        if rc == 0:
            self._keep[t.value] = (raw, out, None)
        return rc, t.value

    def replay(self, schedule):
        """Open-loop replay (``lutc_server_replay``): ``schedule`` lists ``(at_s, sensor_id, raw, out, host)``
        with non-decreasing arrival times in seconds.  A native thread submits each request when it is
        due and this call collects them all; returns a dict of numpy arrays (``scheduled_s``,
        ``submit_s``, ``start_s``, ``launched_s``, ``done_s``, ``batch_size``, ``status``, ``cache_miss``)."""
        import numpy as np
        from ._lib import LUTC_REQ_HOST, ReplayRequest, RequestInfo
        n = len(schedule)
        reqs = (ReplayRequest * max(1, n))()
        for i, (at, sid, raw, out, host) in enumerate(schedule):
            ip, pitch = self._addr_pitch(raw, 2)
            op, opitch = self._addr_pitch(out, 1)
            reqs[i] = ReplayRequest(float(at), ip, op, pitch, opitch, sid, raw.shape[-2], LUTC_REQ_HOST if host else 0, 0)
        infos = (RequestInfo * max(1, n))()
        sched = (ctypes.c_double * max(1, n))()
        check(lib().lutc_server_replay(self._h, reqs, n, infos, sched), "lutc_server_replay")
        res = {k: np.array([getattr(infos[i], k) for i in range(n)])
               for k in ("submit_s", "start_s", "launched_s", "done_s", "batch_size", "status", "cache_miss")}
        res["scheduled_s"] = np.array(sched[:n])
        return res

    def wait(self, ticket: int, timeout_us: int = -1):
        """The request's RequestInfo, or None if it is still running after timeout_us."""
        from ._lib import LUTC_ETIMEOUT, RequestInfo
        info = RequestInfo()
        rc = lib().lutc_server_wait(self._h, ticket, timeout_us, ctypes.byref(info))
        if rc == LUTC_ETIMEOUT:
            return None
        check(rc, "lutc_server_wait")
        self._keep.pop(ticket, None)
        return info

    def cancel(self, ticket: int) -> bool:
        """Withdraws a queued request (it completes with LUTC_ECANCELED); False if it is already in a
        batch or done (it then completes normally)."""
        from ._lib import LUTC_EBUSY
        rc = lib().lutc_server_cancel(self._h, ticket)
        if rc == LUTC_EBUSY:
            return False
        check(rc, "lutc_server_cancel")
        return True

    def stats(self):
        c, b, u, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t(), ctypes.c_int32()
        check(lib().lutc_server_stats(self._h, ctypes.byref(c), ctypes.byref(b), ctypes.byref(u), ctypes.byref(m)),
              "lutc_server_stats")
        return dict(completed=c.value, batches=b.value, budget_in_use=u.value, largest_batch=m.value)

    def close(self) -> None:
        if self._h:
            lib().lutc_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def submit(task: int, params: str, inputs, outputs, workspace: torch.Tensor | None = None, stream=None) -> None:
    """The paper's task call: a task flag, a "key=value,..." parameter string, data and outputs."""
    ins = (ctypes.c_void_p * max(1, len(inputs)))(*[t.data_ptr() for t in inputs])
    outs = (ctypes.c_void_p * max(1, len(outputs)))(*[t.data_ptr() for t in outputs])
    dev = (inputs or outputs)[0].device
    ws = workspace.data_ptr() if workspace is not None else None
    nws = workspace.numel() if workspace is not None else 0
    check(lib().lutc_submit(task, params.encode(), ins, len(inputs), outs, len(outputs), ws, nws,
                            _stream(stream, dev)), "lutc_submit")


def device_info() -> str:
    """XML listing of the visible GPUs (the paper's GPU-information utility)."""
    need = ctypes.c_size_t()
    lib().lutc_device_info(None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(need.value)
    check(lib().lutc_device_info(buf, need.value, ctypes.byref(need)), "lutc_device_info")
    return buf.value.decode()


def fit(x: torch.Tensor, y: torch.Tensor, order: int, q16: bool = False, coef: torch.Tensor | None = None,
        status: torch.Tensor | None = None, codes: torch.Tensor | None = None, stream=None):
    """Per-column least-squares polynomial fit of order 1-3 (Section III.B).

    x: ``[n, ncols]`` uint16 on the device (rows may be padded); y: ``[n]`` (one target per
    line) or ``[n, ncols]`` float64.  Returns ``(coef [ncols, order+1] float64, status [ncols]
    int32)`` and, with ``q16``, the ``[3, ncols]`` int32 rows A, G, O for :func:`lutgen`.
    """
    _need(x, torch.uint16, "x")
    _need(y, torch.float64, "y")
    if x.dim() != 2 or (x.numel() and x.stride(1) != 1):
        raise ValueError("x must be [n, ncols] with contiguous rows")
    n, ncols = x.shape
    if y.dim() == 1:
        if y.shape[0] != n or (n and y.stride(0) != 1):
            raise ValueError("y must hold one contiguous target per line")
        y_pitch = 0
    else:
        if tuple(y.shape) != (n, ncols) or (y.numel() and y.stride(1) != 1):
            raise ValueError("y must be [n, ncols] with contiguous rows")
        y_pitch = y.stride(0) * 8
    dev = x.device
    if coef is None:
        coef = torch.empty((ncols, order + 1), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(ncols, dtype=torch.int32, device=dev)
    if q16 and codes is None:
        codes = torch.empty((3, ncols), dtype=torch.int32, device=dev)
    check(lib().lutc_fit(x.data_ptr(), x.stride(0) * 2, y.data_ptr(), y_pitch, n, ncols, order, coef.data_ptr(),
                         status.data_ptr(), codes.data_ptr() if q16 else None, _stream(stream, dev)), "lutc_fit")
    return (coef, status, codes) if q16 else (coef, status)


def demosaic(raw: torch.Tensor, pattern: str = "rggb", bits: int = 16, A: torch.Tensor | None = None,
             G: torch.Tensor | None = None, O: torch.Tensor | None = None, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """Bilinear Bayer demosaic of a ``[H, W]`` uint16 CFA raster into ``[3, H, W]`` uint16 R, G, B planes
    (Section III.A); with per-column coefficients ``A, G, O`` (``[W]`` int32) every photosite is
    detector-corrected first."""
    from ._lib import LUTC_BAYER
    desc = raster_desc(raw, bits)
    if desc.bands != 1:
        raise ValueError("demosaic takes one CFA band")
    cd = coeff_descs(A, G, O)[0] if A is not None else None
    H, W = raw.shape[-2], raw.shape[-1]
    if out is None:
        out = torch.empty((3, H, W), dtype=torch.uint16, device=raw.device)
    _need(out, torch.uint16, "out")
    if out.dim() != 3 or out.shape[0] != 3 or (out.numel() and (out.stride(2) != 1 or
                                                                 (H > 0 and out.stride(0) != H * out.stride(1)))):
        raise ValueError("out must be [3, H, W] with contiguous rows stacked at H * pitch")
    pitch = out.stride(1) * 2 if out.numel() else 2 * W
    check(lib().lutc_demosaic(ctypes.byref(desc), ctypes.byref(cd) if cd is not None else None,
                              LUTC_BAYER[pattern], out.data_ptr(), pitch, _stream(stream, raw.device)),
          "lutc_demosaic")
    return out


def correct_image_host(raw: torch.Tensor, A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int,
                       stretch: bool = True, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                       stream=None, device=None) -> torch.Tensor:
    """:func:`correct_image` for a raster in host memory (CPU tensor, ideally pinned), output in host
    memory; copies and both passes are pipelined in the library.  Synchronises nothing: synchronise
    ``stream`` (or the device) before reading ``out``."""
    if raw.device.type != "cpu" or raw.dtype != torch.uint16:
        raise TypeError("raw must be a host (CPU) torch.uint16 tensor")
    r3 = raw if raw.dim() == 3 else raw.unsqueeze(0)
    bands, h, w = r3.shape
    if r3.numel() and (r3.stride(2) != 1 or (bands > 1 and h > 0 and r3.stride(0) != h * r3.stride(1))):
        raise ValueError("raw must be [bands, height, width] with contiguous rows stacked at height * pitch")
    desc = Raster(r3.data_ptr(), (r3.stride(1) if r3.numel() else w) * 2, w, h, bands, bits)
    cd = coeff_descs(A, G, O)
    dev = A.device if device is None else torch.device(device)
    odt = torch.uint8 if stretch else torch.uint16
    if out is None:
        out = torch.empty(r3.shape, dtype=odt, pin_memory=raw.is_pinned())
    if out.device.type != "cpu" or out.dtype != odt:
        raise TypeError("out must be a host (CPU) %s tensor" % odt)
    o3 = out if out.dim() == 3 else out.unsqueeze(0)
    if o3.numel() and (o3.stride(2) != 1 or (bands > 1 and h > 0 and o3.stride(0) != h * o3.stride(1))):
        raise ValueError("out must be [bands, height, width] with contiguous rows stacked at height * pitch")
    opitch = (o3.stride(1) if o3.numel() else w) * out.element_size()
    flags = LUTC_STRETCH if stretch else 0
    need = int(lib().lutc_correct_image_host_workspace(ctypes.byref(desc), flags))
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    check(lib().lutc_correct_image_host(ctypes.byref(desc), cd, flags, out.data_ptr(), opitch, workspace.data_ptr(),
                                        workspace.numel(), _stream(stream, dev)), "lutc_correct_image_host")
    return out


def correct_frames_host(frames, A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int, stretch: bool = True,
                        outs=None, workspace: torch.Tensor | None = None, stream=None):
    """:func:`correct_image_host` over a sequence of same-shape host frames of one sensor, pipelined
    (a frame's copies in overlap the previous frame's drain).  Synchronises nothing."""
    if not frames:
        return []
    f0 = frames[0]
    for f in frames:
        if f.device.type != "cpu" or f.dtype != torch.uint16 or f.shape != f0.shape or f.stride() != f0.stride():
            raise TypeError("frames must be host (CPU) torch.uint16 tensors of one shape and layout")
    r3 = f0 if f0.dim() == 3 else f0.unsqueeze(0)
    bands, h, w = r3.shape
    if r3.numel() and (r3.stride(2) != 1 or (bands > 1 and h > 0 and r3.stride(0) != h * r3.stride(1))):
        raise ValueError("frames must be [bands, height, width] with contiguous rows stacked at height * pitch")
    desc = Raster(r3.data_ptr(), (r3.stride(1) if r3.numel() else w) * 2, w, h, bands, bits)
    cd = coeff_descs(A, G, O)
    dev = A.device
    odt = torch.uint8 if stretch else torch.uint16
    if outs is None:
        outs = [torch.empty(r3.shape, dtype=odt, pin_memory=f0.is_pinned()) for _ in frames]
    o0 = outs[0] if outs[0].dim() == 3 else outs[0].unsqueeze(0)
    for o in outs:
        if o.device.type != "cpu" or o.dtype != odt or o.stride() != outs[0].stride() or o.shape != outs[0].shape:
            raise TypeError("outs must be host (CPU) %s tensors of one shape and layout" % odt)
    opitch = (o0.stride(1) if o0.numel() else w) * outs[0].element_size()
    flags = LUTC_STRETCH if stretch else 0
    n = len(frames)
    need = int(lib().lutc_correct_frames_host_workspace(ctypes.byref(desc), flags, n))
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    fin = (ctypes.c_void_p * n)(*[f.data_ptr() for f in frames])
    fout = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    check(lib().lutc_correct_frames_host(ctypes.byref(desc), fin, n, cd, flags, fout, opitch, workspace.data_ptr(),
                                         workspace.numel(), _stream(stream, dev)), "lutc_correct_frames_host")
    return outs
