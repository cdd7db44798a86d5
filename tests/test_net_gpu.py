"""Tasks submitted over the TCP transport give what the direct calls give (GPU).

Integer tasks are compared byte for byte with the local library call and,
for the correction and the demosaic, with the oracle; the fit with the local
call (same kernel, same inputs: identical bits).
"""
import xml.etree.ElementTree as ET

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import net  # noqa: E402


@pytest.fixture(scope="module")
def conn():
    srv = net.NetServer()
    s = srv.connect()
    yield s
    s.close()
    srv.close()


def test_correct_image_over_the_socket(conn):
    bands, h, w, bits = 3, 301, 777, 12
    raw = synth.raster(31, bands, h, w, bits)
    A, G, O = synth.coeff_set(31, bands, w)
    st, name, data = net.request(conn, "correct_image", "width=%d,height=%d,bands=%d,bits=%d" % (w, h, bands, bits),
                                 [raw, A, G, O], out_name="scene.u8")
    assert st == 0 and name == "scene.u8"
    out = np.frombuffer(data, np.uint8).reshape(bands, h, w)
    np.testing.assert_array_equal(out, oracle.correct_image(raw, A, G, O, bits))
    st, _, data = net.request(conn, "correct_image", "width=%d,height=%d,bands=%d,bits=%d,stretch=0" %
                              (w, h, bands, bits), [raw, A, G, O])
    d = [torch.from_numpy(a).cuda() for a in (raw, A, G, O)]
    ref = lutc.correct_image(*d, bits, stretch=False).cpu().numpy()
    assert st == 0 and np.array_equal(np.frombuffer(data, np.uint16).reshape(bands, h, w), ref)


def test_tables_over_the_socket(conn):
    w, bits = 300, 10
    A, G, O = synth.coeffs(5, 0, w)
    st, _, lut = net.request(conn, "lutgen", "width=%d,bits=%d" % (w, bits), [A, G, O])
    assert st == 0
    np.testing.assert_array_equal(np.frombuffer(lut, np.uint16).reshape(w, 1 << bits), oracle.lutgen(A, G, O, bits))
    raw = synth.raster(5, 1, 40, w, bits)
    st, _, h = net.request(conn, "hist", "width=%d,height=40,bits=%d" % (w, bits), [raw, A, G, O])
    hist = np.frombuffer(h, np.uint64)
    assert st == 0 and int(hist.sum()) == 40 * w
    st, _, sl = net.request(conn, "stretch", "bits=%d" % bits, [hist])
    assert st == 0 and len(sl) == (1 << bits) + 8


def test_demosaic_and_fit_over_the_socket(conn):
    h, w = 64, 200
    img = synth.raster(6, 1, h, w, 16)[0]
    st, _, data = net.request(conn, "demosaic", "width=%d,height=%d,bits=16,pattern=grbg" % (w, h), [img])
    assert st == 0
    np.testing.assert_array_equal(np.frombuffer(data, np.uint16).reshape(3, h, w), oracle.demosaic(img, "grbg"))
    A, G, O = synth.coeffs(6, 0, w)
    img12 = synth.raster(7, 1, h, w, 12)[0]
    st, _, data = net.request(conn, "demosaic", "width=%d,height=%d,bits=12,pattern=rggb" % (w, h), [img12, A, G, O])
    assert st == 0
    np.testing.assert_array_equal(np.frombuffer(data, np.uint16).reshape(3, h, w),
                                  oracle.demosaic(img12, "rggb", lut=oracle.lutgen(A, G, O, 12), bits=12))
    x, y = synth.calib(synth.CALIB_SEED, 6, 6000, 12, dead_frac=0.01)
    st, _, data = net.request(conn, "fit", "width=6000,height=6,order=2,targets=line", [x, y])
    assert st == 0
    coef = np.frombuffer(data[:6000 * 3 * 8], np.float64).reshape(6000, 3)
    status = np.frombuffer(data[6000 * 3 * 8:], np.int32)
    c_ref, s_ref = lutc.fit(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 2)
    assert np.array_equal(status, s_ref.cpu().numpy())
    np.testing.assert_array_equal(coef, c_ref.cpu().numpy())


def test_device_info_over_the_socket(conn):
    st, _, data = net.request(conn, "device_info", "")
    root = ET.fromstring(data.decode())
    assert st == 0 and int(root.get("count")) == torch.cuda.device_count()
    assert int(root.find("gpu/multiprocessor_count").text) == torch.cuda.get_device_properties(0).multi_processor_count
