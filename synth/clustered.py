"""ctypes front end of clustered.c (clustered 3D particle sets); built on demand."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "clustered.c")
LIB = os.path.join(HERE, "_libsynth.so")
_lib = None


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, SRC, "-lm"],
                   check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_clustered.argtypes = [ctypes.c_longlong, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_ulonglong, P, P]
        lib.synth_clustered.restype = ctypes.c_int
        _lib = lib
    return _lib


def generate(n, L, n_clusters, sigma, frac_clustered, size_range, min_sep, seed, max_tries=64):
    x = np.zeros((n, 3), dtype=np.float64)
    stats = np.zeros(4, dtype=np.int64)
    rc = _load().synth_clustered(n, L, n_clusters, sigma, frac_clustered, size_range[0], size_range[1],
                                 min_sep, max_tries, seed, x.ctypes.data_as(ctypes.c_void_p),
                                 stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise RuntimeError("synth_clustered failed: %d" % rc)
    return x, {"clustered": int(stats[0]), "background": int(stats[1]), "redirected": int(stats[2]),
               "largest_cluster": int(stats[3])}
