"""Python binding of the C ABI (include/cellmap.h), same names, argument
marshalling only: torch tensors supply device memory, torch streams supply the
CUDA stream, and every step of the computation runs in libcellmap's kernels.

Positions are (n, dim) float64 CUDA tensors; the box ``h`` is a (dim, dim)
matrix whose ROWS are the lattice vectors (orthorhombic: a diagonal matrix).
"""
import ctypes

import numpy as np
import torch

from . import _lib as L
from ._lib import (CL_RED_COUNT, CL_RED_HIST, CL_RED_PAIRLIST, CL_RED_SF_ENERGY, CL_RED_SF_ENERGY_FORCES_VIRIAL,
                   CL_RED_SUM_INV_R, CellMapError)

REDUCTIONS = {"count": CL_RED_COUNT, "sum_inv_r": CL_RED_SUM_INV_R, "energy": CL_RED_SF_ENERGY,
              "energy_forces_virial": CL_RED_SF_ENERGY_FORCES_VIRIAL, "hist": CL_RED_HIST,
              "pairlist": CL_RED_PAIRLIST}


def make_box(h, cutoff, lcell=2):
    h = np.asarray(h, dtype=np.float64)
    dim = h.shape[0]
    if h.shape != (dim, dim) or dim not in (2, 3):
        raise ValueError("box must be a 2x2 or 3x3 matrix")
    b = L.cl_box()
    b.dim = dim
    flat = h.reshape(-1)
    for k in range(dim * dim):
        b.h[k] = float(flat[k])
    b.cutoff = float(cutoff)
    b.lcell = int(lcell)
    return b


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_pos(pos, dim=None):
    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dtype == torch.float64 and pos.dim() == 2
            and pos.is_contiguous()):
        raise ValueError("positions must be a contiguous (n, dim) float64 CUDA tensor")
    if dim is not None and pos.shape[1] != dim:
        raise ValueError("positions have %d columns, box has dim %d" % (pos.shape[1], dim))


class CellList:
    """Owner of a cl_list handle; keeps the positions tensor alive because the
    library reads it again in cl_backward."""

    def __init__(self, handle, pos, h, cutoff, lcell):
        self._h = handle
        self.pos = pos
        self.n, self.dim = pos.shape
        self.h = np.asarray(h, dtype=np.float64).copy()
        self.cutoff = float(cutoff)
        self.lcell = int(lcell)
        self.device = pos.device

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("cell list was freed")
        return self._h

    def __del__(self):
        try:
            cl_free(self)
        except Exception:
            pass


def cl_build(pos, h, cutoff, lcell=2, stream=None):
    box = make_box(h, cutoff, lcell)
    _check_pos(pos, box.dim)
    out = ctypes.c_void_p()
    with torch.cuda.device(pos.device):
        L.check(L.lib().cl_build(_ptr(pos), pos.shape[0], ctypes.byref(box), _stream(stream), ctypes.byref(out)),
                "cl_build")
    return CellList(out, pos, h, cutoff, lcell)


def cl_update(cl, pos, h=None, cutoff=None, lcell=None, stream=None):
    _check_pos(pos, cl.dim)
    if pos.shape[0] != cl.n:
        raise ValueError("cl_update keeps the particle count")
    boxp = None
    if h is not None or cutoff is not None or lcell is not None:
        nh = cl.h if h is None else np.asarray(h, dtype=np.float64)
        nc = cl.cutoff if cutoff is None else cutoff
        nl = cl.lcell if lcell is None else lcell
        boxp = ctypes.byref(make_box(nh, nc, nl))
    with torch.cuda.device(pos.device):
        L.check(L.lib().cl_update(cl.handle, _ptr(pos), boxp, _stream(stream)), "cl_update")
    cl.pos = pos
    if boxp is not None:
        cl.h, cl.cutoff, cl.lcell = np.array(nh, dtype=np.float64), float(nc), int(nl)


def cl_map(cl, reduction, nbins=0, rmax=0.0, capacity=None, stream=None, out=None):
    """Run one built-in reduction; returns a dict of device tensors. For the
    pair list, out may hold preallocated (i, j, d) tensors (int32, int32,
    float32) whose common length is the capacity."""
    red = REDUCTIONS[reduction] if isinstance(reduction, str) else int(reduction)
    if red == CL_RED_PAIRLIST:
        return _pairlist(cl, capacity, stream, out)
    dev = cl.device
    res = L.cl_result()
    out = {}
    f64 = dict(dtype=torch.float64, device=dev)
    if red == CL_RED_COUNT:
        out["count"] = torch.zeros(1, dtype=torch.int64, device=dev)
        res.count = out["count"].data_ptr()
    elif red == CL_RED_SUM_INV_R:
        out["sum_inv_r"] = torch.zeros(1, **f64)
        res.sum_inv_r = out["sum_inv_r"].data_ptr()
    elif red == CL_RED_SF_ENERGY:
        out["energy"] = torch.zeros(1, **f64)
        res.energy = out["energy"].data_ptr()
    elif red == CL_RED_SF_ENERGY_FORCES_VIRIAL:
        out["energy"] = torch.zeros(1, **f64)
        out["forces"] = torch.empty((cl.n, cl.dim), dtype=torch.float32, device=dev)
        out["virial"] = torch.zeros((cl.dim, cl.dim), **f64)
        res.energy, res.forces, res.virial = (out[k].data_ptr() for k in ("energy", "forces", "virial"))
    elif red == CL_RED_HIST:
        out["hist"] = torch.zeros(int(nbins), dtype=torch.int64, device=dev)
        res.hist = out["hist"].data_ptr()
    params = L.cl_params()
    params.nbins = int(nbins)
    params.rmax = float(rmax)
    with torch.cuda.device(dev):
        L.check(L.lib().cl_map(cl.handle, red, ctypes.byref(params), ctypes.byref(res), _stream(stream)), "cl_map")
    return out


def _pairlist(cl, capacity, stream, bufs=None):
    dev = cl.device
    if bufs is not None:
        pi, pj, pd = bufs
        if not (pi.dtype == pj.dtype == torch.int32 and pd.dtype == torch.float32 and
                pi.is_contiguous() and pj.is_contiguous() and pd.is_contiguous() and
                pi.numel() == pj.numel() == pd.numel() and pi.device == pj.device == pd.device == dev):
            raise ValueError("out: contiguous (int32, int32, float32) tensors of one length on the list's device")
        capacity = pi.numel()
    cap = int(capacity) if capacity is not None else max(1024, cl.n * 8)
    lib = L.lib()
    while True:
        if bufs is None:
            pi = torch.empty(cap, dtype=torch.int32, device=dev)
            pj = torch.empty(cap, dtype=torch.int32, device=dev)
            pd = torch.empty(cap, dtype=torch.float32, device=dev)
        npairs = ctypes.c_longlong(0)
        res = L.cl_result()
        res.pair_i, res.pair_j, res.pair_d = pi.data_ptr(), pj.data_ptr(), pd.data_ptr()
        res.capacity = cap
        res.npairs = ctypes.pointer(npairs)
        with torch.cuda.device(dev):
            code = lib.cl_map(cl.handle, CL_RED_PAIRLIST, None, ctypes.byref(res), _stream(stream))
        if code == -6 and capacity is None:
            cap = int(npairs.value)
            continue
        L.check(code, "cl_map(pairlist)")
        k = int(npairs.value)
        return {"i": pi[:k], "j": pj[:k], "d": pd[:k], "npairs": k}


def cl_backward(cl, grad_energy, want_box=True, want_virial=True, stream=None):
    """dL/dx (n, dim) float64, dL/dH (dim, dim) float64 or None, virial or None."""
    dev = cl.device
    g = grad_energy.to(device=dev, dtype=torch.float64).reshape(1).contiguous()
    gp = torch.empty((cl.n, cl.dim), dtype=torch.float64, device=dev)
    gb = torch.empty((cl.dim, cl.dim), dtype=torch.float64, device=dev) if want_box else None
    vir = torch.empty((cl.dim, cl.dim), dtype=torch.float64, device=dev) if want_virial else None
    with torch.cuda.device(dev):
        L.check(L.lib().cl_backward(cl.handle, _ptr(g), _ptr(gp), _ptr(gb), _ptr(vir), _stream(stream)),
                "cl_backward")
    return gp, gb, vir


def cl_energy_grad(cl, scale=None, want_box=True, want_virial=False, stream=None, out=None):
    """Energy and scale * (dE/dx, dE/dH) in one sweep: (energy (1,), dE/dx (n, dim),
    dE/dH (dim, dim) or None, virial or None), float64 on the list's device.
    scale: 1-element tensor (default 1). out: optional tuple of preallocated
    (energy, dE/dx, dE/dH or None, virial or None) tensors to write into."""
    dev = cl.device
    if scale is None:
        g = torch.ones(1, dtype=torch.float64, device=dev)
    else:
        g = scale.to(device=dev, dtype=torch.float64).reshape(1).contiguous()
    if out is not None:
        e, gp, gb, vir = out
    else:
        e = torch.empty(1, dtype=torch.float64, device=dev)
        gp = torch.empty((cl.n, cl.dim), dtype=torch.float64, device=dev)
        gb = torch.empty((cl.dim, cl.dim), dtype=torch.float64, device=dev) if want_box else None
        vir = torch.empty((cl.dim, cl.dim), dtype=torch.float64, device=dev) if want_virial else None
    with torch.cuda.device(dev):
        L.check(L.lib().cl_energy_grad(cl.handle, _ptr(g), _ptr(e), _ptr(gp), _ptr(gb), _ptr(vir), _stream(stream)),
                "cl_energy_grad")
    return e, gp, gb, vir


def cl_scale(scale, x, out=None, stream=None):
    """out = scale * x for float64 CUDA tensors (scale: 1 element); returns out."""
    if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous float64 CUDA tensor")
    g = scale.to(device=x.device, dtype=torch.float64).reshape(1).contiguous()
    if out is None:
        out = torch.empty_like(x)
    with torch.cuda.device(x.device):
        L.check(L.lib().cl_scale(_ptr(g), _ptr(x), _ptr(out), x.numel(), _stream(stream)), "cl_scale")
    return out


def _per_particle(cl, a, cols, name):
    a = torch.as_tensor(a, device=cl.device, dtype=torch.float32)
    if cols:
        a = a.reshape(cl.n, cols)
    else:
        a = a.reshape(cl.n)
    if not a.is_contiguous():
        a = a.contiguous()
    return a


def cl_map_mass(cl, mass, stream=None):
    """Code 5 (second example): sum over the pair-images within the cutoff of
    m_i m_j / r; mass: n values (cast to float32). Returns a (1,) float64 tensor."""
    m = _per_particle(cl, mass, 0, "mass")
    out = torch.empty(1, dtype=torch.float64, device=cl.device)
    with torch.cuda.device(cl.device):
        L.check(L.lib().cl_map_mass(cl.handle, _ptr(m), _ptr(out), _stream(stream)), "cl_map_mass")
    return out


def cl_map_lj(cl, eps, sigma, forces=True, stream=None):
    """Code 6 and 7: Lennard-Jones energy 4 eps ((sigma/r)^12 - (sigma/r)^6) over
    the pair-images within the cutoff (not shifted) and, with forces=True, the
    forces -dE/dx (float32, (n, dim)). Returns (energy (1,) float64, forces or None)."""
    e = torch.empty(1, dtype=torch.float64, device=cl.device)
    f = torch.empty((cl.n, cl.dim), dtype=torch.float32, device=cl.device) if forces else None
    with torch.cuda.device(cl.device):
        L.check(L.lib().cl_map_lj(cl.handle, float(eps), float(sigma), _ptr(e), _ptr(f), _stream(stream)),
                "cl_map_lj")
    return e, f


def cl_map_velocity_hist(cl, vel, binstep, nbins, stream=None):
    """Code 10: pair counts and summed |v_i - v_j| per distance bin, bin
    k = ceil(r / binstep) (1-based, closed on the right), k <= nbins.
    vel: (n, dim) velocities (cast to float32). Returns (counts int64, vsum float64)."""
    v = _per_particle(cl, vel, cl.dim, "vel")
    counts = torch.empty(int(nbins), dtype=torch.int64, device=cl.device)
    vsum = torch.empty(int(nbins), dtype=torch.float64, device=cl.device)
    with torch.cuda.device(cl.device):
        L.check(L.lib().cl_map_velocity_hist(cl.handle, _ptr(v), float(binstep), int(nbins), _ptr(counts),
                                             _ptr(vsum), _stream(stream)), "cl_map_velocity_hist")
    return counts, vsum


def box_nonperiodic(pos, cutoff, lcell=2, pos2=None, stream=None):
    """Box for particles without periodic boundaries (Sec. 4.1): orthorhombic,
    each side larger than the extent of pos (and pos2) plus the cutoff, so that
    cl_build with it maps the pairs of the open system. Returns h (dim, dim)."""
    _check_pos(pos, pos.shape[1])
    n2 = 0
    if pos2 is not None:
        _check_pos(pos2, pos.shape[1])
        n2 = pos2.shape[0]
    box = L.cl_box()
    with torch.cuda.device(pos.device):
        L.check(L.lib().cl_box_nonperiodic(_ptr(pos), pos.shape[0], _ptr(pos2) if n2 else None, n2, pos.shape[1],
                                           float(cutoff), int(lcell), _stream(stream), ctypes.byref(box)),
                "cl_box_nonperiodic")
    d = box.dim
    return np.array([[box.h[a * d + b] for b in range(d)] for a in range(d)])


def cl_build_open(pos, cutoff, lcell=2, pos2=None, stream=None):
    """Cell list of particles without periodic boundaries (see box_nonperiodic)."""
    return cl_build(pos, box_nonperiodic(pos, cutoff, lcell, pos2, stream), cutoff, lcell, stream)


def cl_cross_count(cl, posb, stream=None):
    """Number of pair-images between set A (the cell list) and the points posb
    within the cutoff (Code 8). Returns an int."""
    _check_pos(posb, cl.dim)
    out = torch.empty(1, dtype=torch.int64, device=cl.device)
    with torch.cuda.device(cl.device):
        L.check(L.lib().cl_cross_count(cl.handle, _ptr(posb), posb.shape[0], _ptr(out), _stream(stream)),
                "cl_cross_count")
    return int(out.item())


def cl_cross_pairlist(cl, posb, capacity=None, stream=None):
    """Cross pairs (a, b) within the cutoff sorted by (b, a), with their
    distances: dict of int32 tensors a, b and float32 d."""
    _check_pos(posb, cl.dim)
    dev = cl.device
    cap = int(capacity) if capacity is not None else 0
    while True:
        pa = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        pb = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        pd = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
        n = ctypes.c_longlong(0)
        with torch.cuda.device(dev):
            code = L.lib().cl_cross_pairlist(cl.handle, _ptr(posb), posb.shape[0], cap, _ptr(pa), _ptr(pb), _ptr(pd),
                                             ctypes.byref(n), _stream(stream))
        if code == L.CL_ERR_CAPACITY and capacity is None:
            cap = n.value
            continue
        L.check(code, "cl_cross_pairlist")
        k = n.value
        return {"a": pa[:k], "b": pb[:k], "d": pd[:k], "npairs": k}


def cl_cross_knn(cl, posb, k, stream=None):
    """For each point of posb its k nearest points of set A within the cutoff:
    (a (nb, k) int32, -1 when missing; d (nb, k) float32, inf when missing)."""
    _check_pos(posb, cl.dim)
    nb = posb.shape[0]
    a = torch.empty((nb, int(k)), dtype=torch.int32, device=cl.device)
    d = torch.empty((nb, int(k)), dtype=torch.float32, device=cl.device)
    with torch.cuda.device(cl.device):
        L.check(L.lib().cl_cross_knn(cl.handle, _ptr(posb), nb, int(k), _ptr(a), _ptr(d), _stream(stream)),
                "cl_cross_knn")
    return a, d


def cl_cross_topk(cl, posb, k, stream=None):
    """Code 8: the k pairs (a in A, b in posb) of smallest distance within the
    cutoff, ascending: dict a, b (int32), d (float32), n (how many exist)."""
    _check_pos(posb, cl.dim)
    dev = cl.device
    a = torch.empty(int(k), dtype=torch.int32, device=dev)
    b = torch.empty(int(k), dtype=torch.int32, device=dev)
    d = torch.empty(int(k), dtype=torch.float32, device=dev)
    n = ctypes.c_longlong(0)
    with torch.cuda.device(dev):
        L.check(L.lib().cl_cross_topk(cl.handle, _ptr(posb), posb.shape[0], int(k), _ptr(a), _ptr(b), _ptr(d),
                                      ctypes.byref(n), _stream(stream)), "cl_cross_topk")
    return {"a": a, "b": b, "d": d, "n": n.value}


def cl_query(cl, what, stream=None):
    v = ctypes.c_longlong(0)
    key = L.INFO[what] if isinstance(what, str) else int(what)
    with torch.cuda.device(cl.device):
        L.check(L.lib().cl_query(cl.handle, key, ctypes.byref(v), _stream(stream)), "cl_query")
    return int(v.value)


def cl_box_info(h, cutoff, lcell=2):
    """Host-only: grid, face distances and stencil sizes (no GPU needed)."""
    box = make_box(h, cutoff, lcell)
    grid = (ctypes.c_longlong * 3)()
    widths = (ctypes.c_double * 3)()
    st = (ctypes.c_longlong * 2)()
    L.check(L.lib().cl_box_info(ctypes.byref(box), grid, widths, st), "cl_box_info")
    d = box.dim
    return {"grid": list(grid)[:d], "widths": list(widths)[:d], "stencil_half": st[0], "stencil_full": st[1]}


def cl_status(cl, stream=None):
    """Synchronizes and returns the latched device error code (0 = ok)."""
    with torch.cuda.device(cl.device):
        return int(L.lib().cl_status(cl.handle, _stream(stream)))


def cl_free(cl):
    if getattr(cl, "_h", None) is not None:
        L.lib().cl_free(cl._h)
        cl._h = None


def cl_energy_noalloc(pos, h, cutoff, lcell=2, out=None, stream=None):
    """Shifted-force energy without any device allocation inside the library
    (for callers that may not call cudaMalloc); n <= 65536. ``out`` is a
    1-element float64 CUDA tensor the caller supplies (allocated here when
    omitted, by torch, not by the library)."""
    box = make_box(h, cutoff, lcell)
    _check_pos(pos, box.dim)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=pos.device)
    with torch.cuda.device(pos.device):
        L.check(L.lib().cl_energy_noalloc(_ptr(pos), pos.shape[0], ctypes.byref(box), _ptr(out), _stream(stream)),
                "cl_energy_noalloc")
    return out


def cl_error_string(code):
    return L.lib().cl_error_string(int(code)).decode()
