"""Client side of the library's TCP transport (the paper's Fig. 3 header), and the server handle.

The server is native (``lutc_net_server_*``); this module only frames requests and replies.
"""
from __future__ import annotations

import ctypes
import socket
import struct

import numpy as np

from ._lib import LutcError, check, lib

HEADER_BYTES = 260
FLAG_BYTES, PARAM_BYTES, NAME_BYTES = 29, 200, 30


def header(task: str, params: str, out_name: str = "") -> bytes:
    """The 260-byte request header: task flag, '+', parameter list, output name (NUL-padded fields)."""
    t, p, n = task.encode(), params.encode(), out_name.encode()
    if len(t) > FLAG_BYTES or len(p) > PARAM_BYTES or len(n) > NAME_BYTES:
        raise ValueError("header field too long")
    return t.ljust(FLAG_BYTES, b"\0") + b"+" + p.ljust(PARAM_BYTES, b"\0") + n.ljust(NAME_BYTES, b"\0")


def _recv(sock: socket.socket, n: int) -> bytes:
    buf = bytearray()
    while len(buf) < n:
        chunk = sock.recv(min(n - len(buf), 1 << 22))
        if not chunk:
            raise ConnectionError("connection closed")
        buf += chunk
    return bytes(buf)


def request(sock: socket.socket, task: str, params: str, inputs=(), out_name: str = "", raw_header: bytes | None = None,
            payload: bytes | None = None):
    """Sends one task and returns ``(status, output name, result bytes)``."""
    if payload is None:
        payload = b"".join(np.ascontiguousarray(a).tobytes() for a in inputs)
    hdr = raw_header if raw_header is not None else header(task, params, out_name)
    sock.sendall(hdr + struct.pack("<Q", len(payload)) + payload)
    status = struct.unpack("<i", _recv(sock, 4))[0]
    name = _recv(sock, NAME_BYTES).rstrip(b"\0").decode()
    n = struct.unpack("<Q", _recv(sock, 8))[0]
    return status, name, _recv(sock, n)


class NetServer:
    """A running TCP server on ``address:port`` (port 0 picks a free one) serving GPU ``device``."""

    def __init__(self, address: str = "127.0.0.1", port: int = 0, device: int = 0):
        self._h = ctypes.c_void_p()
        check(lib().lutc_net_server_create(address.encode(), port, device, ctypes.byref(self._h)),
              "lutc_net_server_create")
        self.address = address
        self.port = int(lib().lutc_net_server_port(self._h))

    def connect(self, timeout: float = 60.0) -> socket.socket:
        return socket.create_connection((self.address, self.port), timeout=timeout)

    def stats(self):
        r, f = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().lutc_net_server_stats(self._h, ctypes.byref(r), ctypes.byref(f)), "lutc_net_server_stats")
        return {"requests": r.value, "failures": f.value}

    def close(self) -> None:
        if self._h:
            lib().lutc_net_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["HEADER_BYTES", "header", "request", "NetServer", "LutcError"]
