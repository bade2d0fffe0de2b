"""Python binding of the request server (include/cellmap_serve.h): argument
marshalling only. Requests carry page-locked host tensors (torch
pin_memory) so that the server's copies are asynchronous."""
import ctypes

import numpy as np
import torch

from . import _lib as L
from .api import make_box

TASKS = {"energy": 0, "forces": 1, "hist": 2}


class cl_request(ctypes.Structure):
    _fields_ = [("pos_host", ctypes.c_void_p), ("n", ctypes.c_longlong), ("box", L.cl_box), ("task", ctypes.c_int),
                ("nbins", ctypes.c_int), ("rmax", ctypes.c_double), ("energy_host", ctypes.c_void_p),
                ("forces_host", ctypes.c_void_p), ("virial_host", ctypes.c_void_p), ("hist_host", ctypes.c_void_p)]


def _declare(lib):
    if getattr(lib, "_serve_declared", False):
        return lib
    P, ll, i32, dbl = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_double
    lib.cl_serve_create.argtypes = [ll, i32, i32, ctypes.POINTER(P)]
    lib.cl_serve_submit.argtypes = [P, ctypes.POINTER(cl_request), ctypes.POINTER(ll)]
    lib.cl_serve_poll.argtypes = [P, ll]
    lib.cl_serve_wait.argtypes = [P, ll, dbl]
    lib.cl_serve_times.argtypes = [P, ll, P]
    lib.cl_serve_stats.argtypes = [P, P]
    lib.cl_serve_release.argtypes = [P, ll]
    lib.cl_serve_clock.argtypes = [P]
    lib.cl_serve_clock.restype = dbl
    lib.cl_serve_free.argtypes = [P]
    lib.cl_serve_free.restype = None
    for f in ("cl_serve_create", "cl_serve_submit", "cl_serve_poll", "cl_serve_wait", "cl_serve_times",
              "cl_serve_stats", "cl_serve_release"):
        getattr(lib, f).restype = i32
    lib._serve_declared = True
    return lib


class Request:
    """One request with its page-locked input and output buffers."""

    def __init__(self, x, h, cutoff, task, lcell=2, nbins=100, rmax=0.0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        self.pos = torch.from_numpy(x).pin_memory()
        self.n, self.dim = x.shape
        self.task = task
        self.c = cl_request()
        self.c.pos_host = self.pos.data_ptr() if self.n else None
        self.c.n = self.n
        self.c.box = make_box(h, cutoff, lcell)
        self.c.task = TASKS[task]
        self.c.nbins = int(nbins)
        self.c.rmax = float(rmax)
        self.energy = torch.zeros(1, dtype=torch.float64).pin_memory()
        self.c.energy_host = self.energy.data_ptr()
        self.forces = self.virial = self.hist = None
        if task == "forces":
            self.forces = torch.zeros((self.n, self.dim), dtype=torch.float32).pin_memory()
            self.virial = torch.zeros((self.dim, self.dim), dtype=torch.float64).pin_memory()
            self.c.forces_host = self.forces.data_ptr()
            self.c.virial_host = self.virial.data_ptr()
        if task == "hist":
            self.hist = torch.zeros(int(nbins), dtype=torch.int64).pin_memory()
            self.c.hist_host = self.hist.data_ptr()
        self.ticket = None


class Server:
    def __init__(self, arena_bytes=4 << 30, max_inflight=256, device=0):
        self.lib = _declare(L.lib())
        self.h = ctypes.c_void_p()
        L.check(self.lib.cl_serve_create(int(arena_bytes), int(max_inflight), int(device), ctypes.byref(self.h)),
                "cl_serve_create")

    def submit(self, req):
        t = ctypes.c_longlong(0)
        L.check(self.lib.cl_serve_submit(self.h, ctypes.byref(req.c), ctypes.byref(t)), "cl_serve_submit")
        req.ticket = t.value
        return t.value

    def poll(self, ticket):
        return int(self.lib.cl_serve_poll(self.h, ticket))

    def wait(self, ticket, timeout=60.0):
        return int(self.lib.cl_serve_wait(self.h, ticket, float(timeout)))

    def times(self, ticket):
        t = (ctypes.c_double * 4)()
        L.check(self.lib.cl_serve_times(self.h, ticket, t), "cl_serve_times")
        return list(t)

    def release(self, ticket):
        """Forget a finished ticket (0); 1 when it is still pending."""
        code = int(self.lib.cl_serve_release(self.h, ticket))
        if code < 0:
            L.check(code, "cl_serve_release")
        return code

    def stats(self):
        s = (ctypes.c_longlong * 6)()
        L.check(self.lib.cl_serve_stats(self.h, s), "cl_serve_stats")
        keys = ("batches", "completed", "failed", "largest_batch", "arena_used", "arena_bytes")
        return dict(zip(keys, list(s)))

    def clock(self):
        return float(self.lib.cl_serve_clock(self.h))

    def close(self):
        if self.h:
            self.lib.cl_serve_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
