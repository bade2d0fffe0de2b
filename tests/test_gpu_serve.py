"""Request server (continuous batching): each result is the same alone and in
the mix, matches the oracle, and failures stay with their request."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import BAND, TOL_E, TOL_F, TOL_W, check_count, check_energy, check_forces, check_hist, check_matrix

pytestmark = pytest.mark.gpu


def _S():
    from paper_2202_06427_gb300 import serve
    return serve


def _requests(k, n_max, seed):
    S = _S()
    out = []
    for spec in synth.serve_stream(n_requests=k, seed=seed, n_max=n_max):
        x = synth.request_positions(spec)
        out.append((spec, S.Request(x, spec["h"], spec["rc"], spec["task"], lcell=2, nbins=spec["nbins"])))
    return out


def _run(server, reqs):
    for _, r in reqs:
        server.submit(r)
    for _, r in reqs:
        assert server.wait(r.ticket, 120.0) == 0


def _same(a, b):
    """Alone (a) against mix (b): same kernels and reduction order, so equal
    up to FP32 summation order within a cell."""
    if a.task == "hist":
        np.testing.assert_array_equal(a.hist.numpy(), b.hist.numpy())
        return
    ea, eb = a.energy.item(), b.energy.item()
    assert abs(ea - eb) <= TOL_E * abs(ea) + 1e-12
    if a.task == "forces":
        fa, fb = a.forces.numpy().astype(np.float64), b.forces.numpy().astype(np.float64)
        assert np.abs(fa - fb).max() <= TOL_F * max(np.abs(fa).max(), 1e-30)
        va, vb = a.virial.numpy(), b.virial.numpy()
        assert np.abs(va - vb).max() <= TOL_W * np.abs(va).max()


def test_results_alone_equal_results_in_the_mix(cuda_ok):
    S = _S()
    mix = _requests(40, 30_000, 9001)
    alone = _requests(40, 30_000, 9001)
    srv = S.Server(arena_bytes=2 << 30, max_inflight=64)
    try:
        _run(srv, mix)
        st = srv.stats()
        assert st["largest_batch"] > 1, st  # the mix really was batched
    finally:
        srv.close()
    one = S.Server(arena_bytes=2 << 30, max_inflight=1)
    try:
        for spec_r in alone:
            _run(one, [spec_r])
        assert one.stats()["largest_batch"] == 1
    finally:
        one.close()
    for (spec, a), (_, b) in zip(alone, mix):
        _same(a, b)


def test_served_results_match_oracle(cuda_ok):
    S = _S()
    reqs = _requests(12, 20_000, 9002)
    srv = S.Server(arena_bytes=1 << 30, max_inflight=16)
    try:
        _run(srv, reqs)
    finally:
        srv.close()
    for spec, r in reqs:
        x = r.pos.numpy()
        ref = oracle.pair_map(x, spec["h"], spec["rc"], band=BAND, nbins=spec["nbins"] if spec["task"] == "hist" else 0)
        if spec["task"] == "hist":
            check_hist(r.hist.numpy(), ref)
        else:
            check_energy(r.energy.item(), ref["energy"])
        if spec["task"] == "forces":
            check_forces(r.forces.numpy(), ref["forces"])
            check_matrix(r.virial.numpy(), ref["virial"], TOL_W)


def test_failures_stay_with_their_request(cuda_ok):
    S = _S()
    good = _requests(4, 5_000, 9003)
    bad_nan = _requests(1, 3_000, 9004)[0][1]
    bad_nan.pos[7, 0] = float("nan")
    big_spec = synth.serve_stream(n_requests=1, seed=9005, n_min=150_000, n_max=150_000)[0]
    big = S.Request(synth.request_positions(big_spec), big_spec["h"], big_spec["rc"], "energy")
    empty = S.Request(np.zeros((0, 3)), np.eye(3) * 30.0, 5.0, "energy")
    srv = S.Server(arena_bytes=8 << 20, max_inflight=8)  # 8 MB: the 150k request cannot fit
    try:
        tickets = [srv.submit(r) for _, r in good[:2]]
        t_nan = srv.submit(bad_nan)
        t_big = srv.submit(big)
        t_empty = srv.submit(empty)
        tickets += [srv.submit(r) for _, r in good[2:]]
        from paper_2202_06427_gb300 import CellMapError
        with pytest.raises(CellMapError) as e:  # invalid box: refused at submission
            srv.submit(S.Request(np.zeros((4, 3)), np.zeros((3, 3)), 1.0, "energy"))
        assert e.value.code == -2
        assert srv.wait(t_nan, 60) == -4
        assert srv.wait(t_big, 60) == -5
        assert srv.wait(t_empty, 60) == 0 and empty.energy.item() == 0.0
        for t in tickets:
            assert srv.wait(t, 60) == 0
        st = srv.stats()
        assert st["failed"] == 2 and st["arena_used"] == 0
        # finished tickets are released; a released ticket is unknown afterwards
        for t in tickets + [t_nan, t_big, t_empty]:
            assert srv.release(t) == 0
        assert srv.poll(t_nan) == -1
        with pytest.raises(CellMapError) as e:
            srv.release(t_nan)
        assert e.value.code == -1
    finally:
        srv.close()
    for spec, r in good:
        x = r.pos.numpy()
        ref = oracle.pair_map(x, spec["h"], spec["rc"], band=BAND, nbins=spec["nbins"] if spec["task"] == "hist" else 0)
        if spec["task"] == "hist":
            check_hist(r.hist.numpy(), ref)
        else:
            check_energy(r.energy.item(), ref["energy"])


def _oracle_request(spec):
    """Oracle result of one request of the stream, its positions drawn again
    from the request's own seed (spawned worker)."""
    import oracle as O
    import synth as Sy
    x = Sy.request_positions(spec)
    nb = spec["nbins"] if spec["task"] == "hist" else 0
    ref = O.pair_map(x, spec["h"], spec["rc"], band=BAND, nbins=nb, forces=spec["task"] == "forces")
    keep = ("energy", "virial", "forces", "hist_core", "hist_maybe")
    return {k: ref[k] for k in keep if k in ref}


@pytest.mark.slow
def test_whole_served_stream_matches_oracle(cuda_ok):
    """All 512 requests of the served stream (2D and 3D, orthorhombic and
    triclinic, N from 1,000 to 200,000, energy / forces / 100-bin histogram),
    served together with continuous batching, each result checked against the
    oracle (a spawn pool runs one request per task)."""
    import multiprocessing as mp
    S = _S()
    specs = synth.serve_stream()
    reqs = [S.Request(synth.request_positions(sp), sp["h"], sp["rc"], sp["task"], lcell=2, nbins=sp["nbins"])
            for sp in specs]
    srv = S.Server(arena_bytes=4 << 30, max_inflight=256)
    try:
        for r in reqs:
            srv.submit(r)
        for r in reqs:
            assert srv.wait(r.ticket, 300.0) == 0
        assert srv.stats()["largest_batch"] > 1
    finally:
        srv.close()
    order = sorted(range(len(specs)), key=lambda k: -specs[k]["n"])  # largest first
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        refs = dict(zip(order, pool.map(_oracle_request, [specs[k] for k in order], chunksize=1)))
    for k, (spec, r) in enumerate(zip(specs, reqs)):
        ref = refs[k]
        if spec["task"] == "hist":
            check_hist(r.hist.numpy(), ref)
        else:
            check_energy(r.energy.item(), ref["energy"])
        if spec["task"] == "forces":
            check_forces(r.forces.numpy(), ref["forces"])
            check_matrix(r.virial.numpy(), ref["virial"], TOL_W)
