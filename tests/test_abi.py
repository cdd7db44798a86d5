"""The C-ABI library loads and exports every entry point include/lutc.h declares (CPU only).

Only host-side behaviour is exercised here: symbol export, the status text,
the workspace size query and argument checks that return before anything
reaches the GPU.  Nothing here launches a kernel.
"""
import ctypes
import os
import re

import pytest

from paper_1505_05655_gb300 import _lib
from paper_1505_05655_gb300._lib import Coeffs, Raster

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lutc.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^LUTC_API\s+[\w\s\*]+?\b(lutc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("lutc_lutgen", "lutc_apply_u16", "lutc_hist", "lutc_stretch", "lutc_compose", "lutc_apply_u8",
              "lutc_correct_image"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, "binding lacks " + name


def test_version_and_strerror():
    lib = _lib.lib()
    assert lib.lutc_version() >= 10000
    assert lib.lutc_strerror(0) == b"ok"
    assert lib.lutc_strerror(-1) == b"invalid argument"
    assert lib.lutc_strerror(12345) == b"unknown status"


def _raster(**kw):
    r = dict(data=0x10000, pitch_bytes=2 * 100, width=100, height=10, bands=1, bits=12)
    r.update(kw)
    return Raster(r["data"], r["pitch_bytes"], r["width"], r["height"], r["bands"], r["bits"])


def test_workspace_size_query():
    lib = _lib.lib()
    r = _raster(bands=4, bits=12)
    ws = lib.lutc_correct_image_workspace(ctypes.byref(r))
    # uint64 histogram + uint8 stretch table per band + lo/hi, 256-byte aligned blocks
    assert ws >= 4 * 4096 * 8 + 4 * 4096 + 4 * 8 and ws % 256 == 0
    assert lib.lutc_correct_image_workspace(ctypes.byref(_raster(bits=17))) == 0
    h, s, l = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.lutc_correct_image_tables(ctypes.byref(r), ctypes.byref(h), ctypes.byref(s), ctypes.byref(l)) == 0
    assert h.value == 0 and s.value >= 4 * 4096 * 8 and l.value >= s.value + 4 * 4096


@pytest.mark.parametrize("kw", [dict(bits=7), dict(bits=17), dict(bands=0), dict(bands=65), dict(width=-1),
                                dict(pitch_bytes=198), dict(data=0), dict(data=0x10001), dict(pitch_bytes=201)])
def test_bad_raster_is_rejected_before_launch(kw):
    lib = _lib.lib()
    r = _raster(**kw)
    c = (Coeffs * max(1, r.bands))()
    for i in range(len(c)):
        c[i] = Coeffs(0x20000, 0x30000, 0x40000, r.width)
    assert lib.lutc_correct_image(ctypes.byref(r), c, 1, ctypes.c_void_p(0x50000), 100, ctypes.c_void_p(0x60000),
                                  1 << 20, None) == _lib.LUTC_EINVAL
    assert lib.lutc_hist(ctypes.byref(r), c, ctypes.c_void_p(0x70000), None) == _lib.LUTC_EINVAL


def test_bad_arguments_are_rejected_before_launch():
    lib = _lib.lib()
    r = _raster()
    good = (Coeffs * 1)(Coeffs(0x20000, 0x30000, 0x40000, 100))
    wrong_cols = (Coeffs * 1)(Coeffs(0x20000, 0x30000, 0x40000, 99))
    null_coef = (Coeffs * 1)(Coeffs(0, 0x30000, 0x40000, 100))
    E = _lib.LUTC_EINVAL
    assert lib.lutc_correct_image(ctypes.byref(r), wrong_cols, 1, ctypes.c_void_p(0x50000), 100, ctypes.c_void_p(0x60000), 1 << 20, None) == E
    assert lib.lutc_correct_image(ctypes.byref(r), null_coef, 1, ctypes.c_void_p(0x50000), 100, ctypes.c_void_p(0x60000), 1 << 20, None) == E
    assert lib.lutc_correct_image(ctypes.byref(r), good, 4, ctypes.c_void_p(0x50000), 100, ctypes.c_void_p(0x60000), 1 << 20, None) == E
    assert lib.lutc_correct_image(ctypes.byref(r), good, 1, None, 100, ctypes.c_void_p(0x60000), 1 << 20, None) == E
    assert lib.lutc_correct_image(ctypes.byref(r), good, 1, ctypes.c_void_p(0x50000), 99, ctypes.c_void_p(0x60000), 1 << 20, None) == E
    assert lib.lutc_correct_image(ctypes.byref(r), good, 0, ctypes.c_void_p(0x50000), 199, None, 0, None) == E
    # too small a workspace is reported as such
    assert lib.lutc_correct_image(ctypes.byref(r), good, 1, ctypes.c_void_p(0x50000), 100, ctypes.c_void_p(0x60000), 64, None) == _lib.LUTC_ENOMEM
    assert lib.lutc_correct_image(ctypes.byref(r), None, 1, ctypes.c_void_p(0x50000), 100, ctypes.c_void_p(0x60000), 1 << 20, None) == E
    one = (Coeffs * 1)(Coeffs(0x20000, 0x30000, 0x40000, 10))
    assert lib.lutc_lutgen(None, 12, ctypes.c_void_p(0x50000), None) == E
    assert lib.lutc_lutgen(one, 20, ctypes.c_void_p(0x50000), None) == E
    assert lib.lutc_lutgen(one, 12, ctypes.c_void_p(0x50008), None) == E  # table must be 16-byte aligned
    assert lib.lutc_stretch(None, 1, 12, ctypes.c_void_p(0x50000), ctypes.c_void_p(0x60000), None) == E
    assert lib.lutc_stretch(ctypes.c_void_p(0x40000), 0, 12, ctypes.c_void_p(0x50000), ctypes.c_void_p(0x60000), None) == E
    assert lib.lutc_compose(ctypes.c_void_p(0x40000), None, 10, 12, ctypes.c_void_p(0x60000), None) == E
    assert lib.lutc_apply_u8(ctypes.byref(r), None, ctypes.c_void_p(0x60000), 100, None) == E
    assert lib.lutc_apply_u16(ctypes.byref(r), ctypes.c_void_p(0x40000), ctypes.c_void_p(0x60000), 199, None) == E


def test_empty_inputs_need_no_device_work():
    lib = _lib.lib()
    zero = (Coeffs * 1)(Coeffs(0, 0, 0, 0))
    assert lib.lutc_lutgen(zero, 12, None, None) == 0
    assert lib.lutc_compose(None, None, 0, 12, None, None) == 0
    r = _raster(width=0, data=0)
    assert lib.lutc_apply_u8(ctypes.byref(r), ctypes.c_void_p(0x40000), ctypes.c_void_p(0x60000), 0, None) == 0
    assert lib.lutc_correct_image(ctypes.byref(r), zero, 0, None, 0, None, 0, None) == 0


@pytest.mark.parametrize("params", ["width=10,bits=12,colour=3", "width=10,bits=", "width=-1,bits=12", "width=10;bits=12",
                                    "width=10,bits=12," + "x" * 200, "width=10,bits=99", "table=u32,width=1,bits=12",
                                    "width=10"])
def test_submit_rejects_bad_parameter_strings(params):
    lib = _lib.lib()
    bufs = (ctypes.c_void_p * 4)(0x1000, 0x2000, 0x3000, 0x4000)
    assert lib.lutc_submit(_lib.LUTC_TASK_LUTGEN, params.encode(), bufs, 3, bufs, 1, None, 0, None) == _lib.LUTC_EINVAL


def test_submit_rejects_unknown_task_and_missing_buffers():
    lib = _lib.lib()
    bufs = (ctypes.c_void_p * 4)(0x1000, 0x2000, 0x3000, 0x4000)
    assert lib.lutc_submit(42, b"width=10,bits=12", bufs, 3, bufs, 1, None, 0, None) == _lib.LUTC_EINVAL
    assert lib.lutc_submit(_lib.LUTC_TASK_LUTGEN, b"width=10,bits=12", bufs, 2, bufs, 1, None, 0, None) == _lib.LUTC_EINVAL
    assert lib.lutc_submit(_lib.LUTC_TASK_CORRECT_IMAGE, b"width=10,height=4,bits=12", bufs, 4, bufs, 0, None, 0,
                           None) == _lib.LUTC_EINVAL
    # a zero-sized task is valid and needs no device
    assert lib.lutc_submit(_lib.LUTC_TASK_LUTGEN, b"width=0,bits=12", bufs, 3, bufs, 1, None, 0, None) == 0


def test_device_info_document_is_well_formed():
    import xml.etree.ElementTree as ET
    lib = _lib.lib()
    need = ctypes.c_size_t()
    assert lib.lutc_device_info(None, 0, ctypes.byref(need)) == _lib.LUTC_ENOMEM and need.value > 10
    buf = ctypes.create_string_buffer(need.value)
    assert lib.lutc_device_info(buf, need.value, None) == 0
    root = ET.fromstring(buf.value.decode())
    assert root.tag == "gpus" and int(root.get("count")) == len(root.findall("gpu"))
    small = ctypes.create_string_buffer(8)
    assert lib.lutc_device_info(small, 8, None) == _lib.LUTC_ENOMEM and small.value == b""


def test_fit_arguments_are_rejected_before_launch():
    lib = _lib.lib()
    E = _lib.LUTC_EINVAL
    x, y, coef, st, q = 0x10000, 0x20000, 0x30000, 0x40000, 0x50000
    ok = lambda **kw: dict(dict(x=x, xp=200, y=y, yp=0, n=6, ncols=100, order=2, coef=coef, st=st, q=q), **kw)
    call = lambda a: lib.lutc_fit(a["x"], a["xp"], a["y"], a["yp"], a["n"], a["ncols"], a["order"], a["coef"],
                                  a["st"], a["q"], None)
    for bad in (dict(order=0), dict(order=4), dict(n=2), dict(n=65537), dict(order=3, n=6), dict(xp=198), dict(xp=201),
                dict(yp=792), dict(yp=804), dict(x=0), dict(y=0), dict(coef=0), dict(st=0), dict(x=0x10001),
                dict(y=0x20004), dict(ncols=-1)):
        assert call(ok(**bad)) == E, bad
    assert call(ok(ncols=0)) == 0  # nothing to fit, nothing launched


def test_demosaic_arguments_are_rejected_before_launch():
    lib = _lib.lib()
    E = _lib.LUTC_EINVAL
    r = _raster()
    good = Coeffs(0x20000, 0x30000, 0x40000, 100)
    out = ctypes.c_void_p(0x50000)
    assert lib.lutc_demosaic(ctypes.byref(r), None, 4, out, 200, None) == E
    assert lib.lutc_demosaic(ctypes.byref(r), None, -1, out, 200, None) == E
    assert lib.lutc_demosaic(ctypes.byref(r), None, 0, out, 198, None) == E
    assert lib.lutc_demosaic(ctypes.byref(r), None, 0, None, 200, None) == E
    assert lib.lutc_demosaic(ctypes.byref(r), None, 0, ctypes.c_void_p(0x50001), 200, None) == E
    assert lib.lutc_demosaic(ctypes.byref(_raster(bands=2)), None, 0, out, 200, None) == E
    assert lib.lutc_demosaic(ctypes.byref(r), ctypes.byref(Coeffs(0x20000, 0x30000, 0x40000, 99)), 0, out, 200,
                             None) == E
    assert lib.lutc_demosaic(ctypes.byref(r), ctypes.byref(Coeffs(0, 0x30000, 0x40000, 100)), 0, out, 200, None) == E
    assert lib.lutc_demosaic(ctypes.byref(_raster(width=0, data=0)), ctypes.byref(good), 0, out, 0, None) == 0
    bufs = (ctypes.c_void_p * 4)(0x1000, 0x2000, 0x3000, 0x4000)
    for p in (b"width=100,height=10,bits=12,pattern=rgbg", b"width=100,height=10,bits=12",
              b"width=100,height=10,bits=12,bands=2,pattern=rggb"):
        assert lib.lutc_submit(_lib.LUTC_TASK_DEMOSAIC, p, bufs, 1, bufs, 1, None, 0, None) == E


def test_host_path_workspace_and_rejections():
    lib = _lib.lib()
    r = _raster(bands=3, width=1000, height=500, pitch_bytes=2002)
    ws = lib.lutc_correct_image_host_workspace(ctypes.byref(r), 1)
    # tables + device raster (rows padded to 16 B) + uint8 staging (rows padded to 16 B)
    assert ws >= lib.lutc_correct_image_workspace(ctypes.byref(r)) + 3 * 500 * 2000 + 3 * 500 * 1008
    wd = lib.lutc_correct_image_host_workspace(ctypes.byref(r), 0)
    assert wd >= 3 * 500 * 2000 + 3 * 500 * 2000 and wd < ws + 3 * 500 * 1008
    assert lib.lutc_correct_image_host_workspace(ctypes.byref(r), 4) == 0
    assert lib.lutc_correct_image_host_workspace(ctypes.byref(_raster(bits=17)), 1) == 0
    c = (Coeffs * 3)(*[Coeffs(0x20000, 0x30000, 0x40000, 1000)] * 3)
    E = _lib.LUTC_EINVAL
    out, dws = ctypes.c_void_p(0x60000), ctypes.c_void_p(0x100000)
    assert lib.lutc_correct_image_host(ctypes.byref(r), c, 1, out, 999, dws, ws, None) == E
    assert lib.lutc_correct_image_host(ctypes.byref(r), c, 1, None, 1000, dws, ws, None) == E
    assert lib.lutc_correct_image_host(ctypes.byref(r), c, 0, out, 1001, dws, wd, None) == E  # odd uint16 pitch
    assert lib.lutc_correct_image_host(ctypes.byref(r), c, 1, out, 1000, dws, ws - 1, None) == _lib.LUTC_ENOMEM
    assert lib.lutc_correct_image_host(ctypes.byref(r), c, 1, out, 1000, ctypes.c_void_p(0x100010), ws, None) == E
    assert lib.lutc_correct_image_host(ctypes.byref(r), c, 2, out, 1000, dws, ws, None) == E


def test_selftest_limit_is_checked_on_the_host():
    lib = _lib.lib()
    assert lib.lutc_selftest_wait_timeout(0, None) == _lib.LUTC_EINVAL
    assert lib.lutc_selftest_wait_timeout((1 << 31) + 1, None) == _lib.LUTC_EINVAL


def test_frames_host_rejections():
    lib = _lib.lib()
    r = _raster(bands=2, width=1000, height=50, pitch_bytes=2000)
    one = lib.lutc_correct_image_host_workspace(ctypes.byref(r), 1)
    assert lib.lutc_correct_frames_host_workspace(ctypes.byref(r), 1, 1) == one
    assert lib.lutc_correct_frames_host_workspace(ctypes.byref(r), 1, 7) == 2 * one
    assert lib.lutc_correct_frames_host_workspace(ctypes.byref(r), 1, 0) == 0
    c = (Coeffs * 2)(*[Coeffs(0x20000, 0x30000, 0x40000, 1000)] * 2)
    fr = (ctypes.c_void_p * 3)(0x100000, 0x200000, 0x300000)
    outs = (ctypes.c_void_p * 3)(0x400000, 0x500000, 0x600000)
    E = _lib.LUTC_EINVAL
    ws = ctypes.c_void_p(0x1000000)
    assert lib.lutc_correct_frames_host(ctypes.byref(r), fr, -1, c, 1, outs, 1000, ws, 2 * one, None) == E
    assert lib.lutc_correct_frames_host(ctypes.byref(r), None, 3, c, 1, outs, 1000, ws, 2 * one, None) == E
    bad = (ctypes.c_void_p * 3)(0x100000, 0, 0x300000)
    assert lib.lutc_correct_frames_host(ctypes.byref(r), bad, 3, c, 1, outs, 1000, ws, 2 * one, None) == E
    assert lib.lutc_correct_frames_host(ctypes.byref(r), fr, 3, c, 1, outs, 1000, ws, one, None) == _lib.LUTC_ENOMEM
    assert lib.lutc_correct_frames_host(ctypes.byref(r), fr, 0, c, 1, outs, 1000, ws, 0, None) == 0


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of the header has the size and field offsets of its ctypes twin (compiled with the
    host C compiler against the header itself)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    twins = {"lutc_coeffs": _lib.Coeffs, "lutc_raster": _lib.Raster, "lutc_job": _lib.Job,
             "lutc_batch_config": _lib.BatchConfig, "lutc_server_config": _lib.ServerConfig,
             "lutc_request_info": _lib.RequestInfo, "lutc_tuning": _lib.Tuning,
             "lutc_replay_request": _lib.ReplayRequest}
    text = open(HEADER).read()
    assert set(re.findall(r"^\}\s*(lutc_\w+)\s*;", text, flags=re.M)) == set(twins), "a struct has no ctypes twin"
    c_name = {"in_": "in"}
    # field names in declaration order (padding would hide a missing trailing field from sizeof)
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(lutc_\w+)\s*;", text, flags=re.S):
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)\s*;", body)
        assert fields == [c_name.get(f, f) for f, _ in twins[name]._fields_], name
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lutc.h"', "int main(void) {"]
    for name, py in twins.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in py._fields_:
            cf = c_name.get(f, f)
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, cf))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for name, py in twins.items():
        assert int(got[name]) == ctypes.sizeof(py), name
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(py, f).offset, (name, f)


def test_batch_correct_rejects_bad_jobs_before_launch():
    lib = _lib.lib()
    E = _lib.LUTC_EINVAL
    assert lib.lutc_batch_correct(None, 1, None, None, 0, None) == E
    assert lib.lutc_batch_correct(None, -1, None, None, 0, None) == E
    jobs = (_lib.Job * 1)()
    jobs[0] = _lib.Job(Raster(0x100000, 2048, 1024, 16, 1, 20), None, 0x200000, 1024, 1)  # 20-bit DN
    assert lib.lutc_batch_correct(jobs, 1, None, ctypes.c_void_p(0x300000), 1 << 20, None) == E


# most bands whose fused-path tables fit the 1 MiB array of lutc_correct_image_static, per bit depth
STATIC_BAND_LIMIT = {16: 1, 15: 3, 14: 7, 13: 14, 12: 28, 11: 56, 10: 64, 9: 64, 8: 64}


@pytest.mark.parametrize("bits", sorted(STATIC_BAND_LIMIT))
def test_static_scratch_limit_per_bit_depth(bits):
    # the limit the header states (9 * 2^bits bytes per band plus rounding, in 1 MiB) is exactly
    # where the workspace query crosses the array's size
    lib = _lib.lib()
    fits = lambda bands: lib.lutc_correct_image_workspace(ctypes.byref(_raster(bands=bands, bits=bits))) \
        <= _lib.LUTC_STATIC_SCRATCH_BYTES
    n = STATIC_BAND_LIMIT[bits]
    assert fits(n)
    assert n == _lib.LUTC_MAX_BANDS or not fits(n + 1)


def test_static_entry_checks_arguments_before_the_size_limit():
    # on an oversized raster: malformed calls are LUTC_EINVAL, a well-formed one LUTC_ENOMEM; all of
    # it on the host, before anything reaches a device
    lib = _lib.lib()
    r = _raster(bands=2, bits=16)
    c = (Coeffs * 2)(*[Coeffs(0x20000, 0x30000, 0x40000, 100)] * 2)
    out = ctypes.c_void_p(0x50000)
    assert lib.lutc_correct_image_static(ctypes.byref(r), c, _lib.LUTC_STRETCH, out, 100, None) == _lib.LUTC_ENOMEM
    assert lib.lutc_correct_image_static(ctypes.byref(r), c, _lib.LUTC_STRETCH | 0x100, out, 100, None) == _lib.LUTC_EINVAL
    assert lib.lutc_correct_image_static(ctypes.byref(r), None, _lib.LUTC_STRETCH, out, 100, None) == _lib.LUTC_EINVAL
    assert lib.lutc_correct_image_static(ctypes.byref(r), c, _lib.LUTC_STRETCH, None, 100, None) == _lib.LUTC_EINVAL
    assert lib.lutc_correct_image_static(ctypes.byref(r), c, _lib.LUTC_STRETCH, out, 99, None) == _lib.LUTC_EINVAL
    assert lib.lutc_correct_image_static(ctypes.byref(_raster(bits=17)), c, 0, out, 200, None) == _lib.LUTC_EINVAL


def test_last_path_contract():
    # per host thread: 0 before any call with pixels; calls rejected by their checks leave it alone
    import threading
    lib = _lib.lib()
    seen = []

    def fresh_thread():
        p = ctypes.c_int(-1)
        seen.append((lib.lutc_last_path(ctypes.byref(p)), p.value))
        r = _raster()
        good = (Coeffs * 1)(Coeffs(0x20000, 0x30000, 0x40000, 100))
        assert lib.lutc_correct_image(ctypes.byref(r), good, 4, ctypes.c_void_p(0x50000), 100,
                                      ctypes.c_void_p(0x60000), 1 << 20, None) == _lib.LUTC_EINVAL
        assert lib.lutc_hist(ctypes.byref(_raster(bits=7)), good, ctypes.c_void_p(0x70000), None) == _lib.LUTC_EINVAL
        seen.append((lib.lutc_last_path(ctypes.byref(p)), p.value))

    t = threading.Thread(target=fresh_thread)
    t.start()
    t.join()
    assert seen == [(0, _lib.LUTC_PATH_AUTO), (0, _lib.LUTC_PATH_AUTO)]
    assert lib.lutc_last_path(None) == _lib.LUTC_EINVAL


def test_fp64_probe_rejects_bad_arguments_before_launch():
    lib = _lib.lib()
    E = _lib.LUTC_EINVAL
    assert lib.lutc_probe_fp64_fma(0, 10, ctypes.c_void_p(0x50000), None, None) == E
    assert lib.lutc_probe_fp64_fma(4, 0, ctypes.c_void_p(0x50000), None, None) == E
    assert lib.lutc_probe_fp64_fma(4, (1 << 24) + 1, ctypes.c_void_p(0x50000), None, None) == E
    assert lib.lutc_probe_fp64_fma(4, 10, None, None, None) == E
