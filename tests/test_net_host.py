"""The TCP transport's framing and host logic (CPU only, no kernel launched).

The server runs tasks through lutc_submit; without a GPU only device_info can
succeed, which is enough to exercise the header, the payload-length checks,
error replies on a connection that stays usable, concurrent connections and
shutdown.
"""
import struct
import threading
import time
import xml.etree.ElementTree as ET

import pytest
import torch

from paper_1505_05655_gb300 import _lib
from paper_1505_05655_gb300 import net

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="host-only checks (tasks would run on the GPU)")


def test_device_info_round_trip_and_bad_requests_on_one_connection():
    with net.NetServer() as srv:
        s = srv.connect()
        st, name, data = net.request(s, "device_info", "", out_name="gpus.xml")
        assert st == 0 and name == "gpus.xml"
        root = ET.fromstring(data.decode())
        assert root.tag == "gpus" and int(root.get("count")) == 0
        # a header without the '+' separator
        bad = bytearray(net.header("device_info", ""))
        bad[29] = ord("-")
        assert net.request(s, "", "", raw_header=bytes(bad))[0] == _lib.LUTC_EINVAL
        # unknown task, malformed parameters, payload length that does not match the parameters
        assert net.request(s, "sharpen", "width=4")[0] == _lib.LUTC_EINVAL
        assert net.request(s, "lutgen", "width=4;bits=12")[0] == _lib.LUTC_EINVAL
        assert net.request(s, "lutgen", "width=4,bits=12", payload=b"\0" * 47)[0] == _lib.LUTC_EINVAL
        # a well-formed task needs the GPU: refused with LUTC_ECUDA, not a dropped connection
        st, _, data = net.request(s, "lutgen", "width=4,bits=12", payload=b"\0" * 48)
        assert st == _lib.LUTC_ECUDA and data == b""
        # the connection still serves
        assert net.request(s, "device_info", "")[0] == 0
        s.close()
        deadline = time.time() + 5
        while srv.stats()["requests"] < 7 and time.time() < deadline:
            time.sleep(0.01)
        assert srv.stats() == {"requests": 7, "failures": 5}


def test_header_fields_are_fixed_width():
    h = net.header("correct_image", "width=10,height=2,bits=12", "out.raw")
    assert len(h) == net.HEADER_BYTES == 260
    assert h[:13] == b"correct_image" and h[29:30] == b"+" and h[30:55] == b"width=10,height=2,bits=12"
    assert h[230:237] == b"out.raw"
    with pytest.raises(ValueError):
        net.header("x" * 30, "")
    with pytest.raises(ValueError):
        net.header("fit", "p" * 201)


def test_concurrent_clients():
    with net.NetServer() as srv:
        errors = []

        def client():
            try:
                s = srv.connect()
                for _ in range(20):
                    assert net.request(s, "device_info", "")[0] == 0
                s.close()
            except Exception as e:  # reported below
                errors.append(e)

        ts = [threading.Thread(target=client) for _ in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errors


def test_shutdown_with_idle_connections_does_not_hang():
    srv = net.NetServer()
    conns = [srv.connect() for _ in range(3)]
    net.request(conns[0], "device_info", "")
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 5
    for c in conns:
        c.close()


def test_absurd_payload_length_drops_the_connection():
    with net.NetServer() as srv:
        s = srv.connect(timeout=10)
        s.sendall(net.header("lutgen", "width=4,bits=12") + struct.pack("<Q", 1 << 62))
        assert s.recv(16) == b""  # closed by the server
        s.close()
        s2 = srv.connect()
        assert net.request(s2, "device_info", "")[0] == 0  # the server itself is fine
        s2.close()


def test_port_in_use_is_refused():
    with net.NetServer() as srv:
        with pytest.raises(_lib.LutcError) as e:
            net.NetServer(port=srv.port)
        assert e.value.status == _lib.LUTC_EBUSY
