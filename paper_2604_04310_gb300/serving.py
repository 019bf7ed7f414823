"""Python binding of the serving C ABI (frax_server_*): argument marshalling
only. Host arrays are float32 numpy arrays in SoA layout (rows, B)."""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .frax import FraxError, Model, lib

OPS = {"rnea": 0, "crba": 1, "aba": 2, "rnea_grad": 3}
EBUSY, ETIMEOUT = 5, 4


class ServerInfo(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("device_status", ctypes.c_int32),
                ("resident_ctas", ctypes.c_int32)]


def op_rows(op: str, nq: int, nv: int):
    """(input rows, output rows) of an op, as in include/frax.h."""
    return {
        "rnea": ([nq, nv, nv], [nv]),
        "crba": ([nq], [nv * nv]),
        "aba": ([nq, nv, nv], [nv]),
        "rnea_grad": ([nq, nv, nv, nv], [nq, nv, nv]),
    }[op]


class Server:
    def __init__(self, budget_bytes: int = 1 << 30, idle_exit_ms: float = 50.0):
        h = ctypes.c_void_p()
        self._st(lib().frax_server_create(int(budget_bytes), float(idle_exit_ms), ctypes.byref(h)))
        self.handle = h
        self.models = {}

    @staticmethod
    def _st(status):
        if status != 0:
            raise FraxError(status, lib().frax_last_error().decode())

    def add_model(self, model: Model) -> int:
        mid = ctypes.c_int()
        self._st(lib().frax_server_add_model(self.handle, model.handle, ctypes.byref(mid)))
        self.models[mid.value] = model
        return mid.value

    def submit(self, model_id: int, op: str, inputs, B: int | None = None):
        """Returns the request id, or None if the server is busy (budget or
        ring full: collect something and retry). Raises on other errors."""
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in inputs]
        B = arrs[0].shape[1] if B is None else B
        ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        req = ctypes.c_int64()
        st = lib().frax_server_submit(self.handle, model_id, OPS[op], int(B), ptrs, ctypes.byref(req))
        if st == EBUSY:
            return None
        self._st(st)
        return req.value

    def poll(self, req: int) -> bool:
        done = ctypes.c_int()
        self._st(lib().frax_server_poll(self.handle, req, ctypes.byref(done)))
        return bool(done.value)

    def wait_any(self, timeout_ms: float):
        """The id of a completed request, or None on timeout."""
        req = ctypes.c_int64()
        st = lib().frax_server_wait_any(self.handle, float(timeout_ms), ctypes.byref(req))
        if st == ETIMEOUT:
            return None
        self._st(st)
        return req.value

    def collect(self, req: int, model_id: int, op: str, B: int):
        """Outputs (list of (rows, B) float32 arrays) and latency in us."""
        m = self.models[model_id]
        _, out_rows = op_rows(op, m.nq, m.nv)
        outs = [np.empty((r, B), dtype=np.float32) for r in out_rows]
        ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
        lat = ctypes.c_double()
        self._st(lib().frax_server_collect(self.handle, req, ptrs, ctypes.byref(lat)))
        return outs, lat.value

    def replay(self, trace, arrival_us, keep_outputs=False, timeout_ms=120000.0):
        """Replays [(model_id, op, inputs)] with arrival times (us from now)
        natively; returns (latency_us array, outputs or None). keep_outputs:
        False (no outputs copied back), True (all), or a set of trace
        positions whose outputs are copied back (None elsewhere)."""
        n = len(trace)
        mids = (ctypes.c_int * n)(*[t[0] for t in trace])
        ops = (ctypes.c_int * n)(*[OPS[t[1]] for t in trace])
        arrs = [[np.ascontiguousarray(a, dtype=np.float32) for a in t[2]] for t in trace]
        Bs = (ctypes.c_int64 * n)(*[a[0].shape[1] for a in arrs])
        inp = (ctypes.c_void_p * (4 * n))()
        for k, a in enumerate(arrs):
            for j, x in enumerate(a):
                inp[4 * k + j] = x.ctypes.data
        arr = (ctypes.c_double * n)(*[float(x) for x in arrival_us])
        lat = (ctypes.c_double * n)()
        outs, outp = None, None
        if keep_outputs:
            outs = []
            outp = (ctypes.c_void_p * (3 * n))()
            for k, t in enumerate(trace):
                if keep_outputs is not True and k not in keep_outputs:
                    outs.append(None)
                    continue
                m = self.models[t[0]]
                _, rows = op_rows(t[1], m.nq, m.nv)
                o = [np.empty((r, Bs[k]), dtype=np.float32) for r in rows]
                outs.append(o)
                for j, x in enumerate(o):
                    outp[3 * k + j] = x.ctypes.data
        self._st(lib().frax_server_replay(self.handle, n, mids, ops, Bs, inp, arr, outp, lat, float(timeout_ms)))
        return np.frombuffer(lat, dtype=np.float64).copy(), outs

    def info(self) -> dict:
        inf = ServerInfo()
        self._st(lib().frax_server_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in ServerInfo._fields_}

    def close(self, force: bool = False, timeout_ms: float = 5000.0):
        if self.handle is not None and self.handle.value:
            self._st(lib().frax_server_destroy(self.handle, int(force), float(timeout_ms)))
            self.handle = None

    def __del__(self):
        try:
            self.close(force=True)
        except Exception:
            pass
