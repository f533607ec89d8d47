"""The z-slab split's halo exchange on CPU ranks over gloo (no GPU): each rank holds one slab of a
global ghost-inclusive array, takes its place and neighbours from the library's
osbli_domain_plan (host code of libosbli.so), and exchanges ghost planes with point-to-point
sends into its own ghost buffers -- 3 planes of the state, 2 of the z viscous fluxes, the depths
the split uses.  Afterwards every ghost plane holds the global array's plane across the face
(wrapped on periodic grids) and ghosts on physical faces are untouched, for 2 and 3 ranks,
periodic and not, and uneven slab lengths."""
import socket

import numpy as np
import pytest

mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange(dist, torch, L, nz_own, lo, hi, depth):
    """Ghost planes of L ([nz_own + 6][...]; interior planes 3 .. 3 + nz_own - 1) from the
    neighbours: my low ghosts (planes 3 - depth .. 2) receive the low neighbour's top planes,
    my high ghosts (3 + nz_own ..) its bottom ones.  Tag 0: bound for the receiver's low ghosts,
    tag 1: for its high ghosts."""
    reqs = []
    if hi >= 0:    # my top interior planes feed the high neighbour's low ghosts
        reqs.append(dist.isend(L[3 + nz_own - depth:3 + nz_own].contiguous(), hi, tag=0))
    if lo >= 0:    # my bottom interior planes feed the low neighbour's high ghosts
        reqs.append(dist.isend(L[3:3 + depth].contiguous(), lo, tag=1))
    bufs = {}
    if lo >= 0:
        bufs["lo"] = torch.empty_like(L[:depth])
        reqs.append(dist.irecv(bufs["lo"], lo, tag=0))
    if hi >= 0:
        bufs["hi"] = torch.empty_like(L[:depth])
        reqs.append(dist.irecv(bufs["hi"], hi, tag=1))
    for r in reqs:
        r.wait()
    if "lo" in bufs:
        L[3 - depth:3] = bufs["lo"]
    if "hi" in bufs:
        L[3 + nz_own:3 + nz_own + depth] = bufs["hi"]


def _rank(rank, world, port, nz, periodic, q):
    import torch
    import torch.distributed as dist

    from paper_2007_14933_b300 import osbli
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    k0, nzs, lo, hi = osbli.osbli_domain_plan(nz, world, periodic)
    G = torch.from_numpy(np.random.default_rng(5).random((nz, 4, 7)))    # global interior planes
    ok = []
    for depth in (3, 2):
        L = torch.full((nzs[rank] + 6, 4, 7), float("nan"), dtype=torch.float64)
        L[3:3 + nzs[rank]] = G[k0[rank]:k0[rank] + nzs[rank]]
        _exchange(dist, torch, L, nzs[rank], lo[rank], hi[rank], depth)
        for g in range(1, depth + 1):
            klo, khi = k0[rank] - g, k0[rank] + nzs[rank] - 1 + g
            for k, plane in ((klo, L[3 - g]), (khi, L[2 + nzs[rank] + g])):
                if 0 <= k < nz or periodic:
                    ok.append(bool(torch.equal(plane, G[k % nz])))
                else:
                    ok.append(bool(torch.isnan(plane).all()))       # physical face: untouched
        ok.append(bool(torch.isnan(L[:3 - depth]).all()) if depth < 3 else True)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, all(ok), sum(nzs), k0, nzs))


@pytest.mark.parametrize("world,nz,periodic", [(2, 13, True), (2, 11, False), (3, 14, True), (3, 16, False)])
def test_slab_halo_exchange_over_gloo(world, nz, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, nz, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, total, k0, nzs in out:
        assert ok, rank
        assert total == nz and k0[0] == 0 and all(k0[i + 1] == k0[i] + nzs[i] for i in range(world - 1))
        assert max(nzs) - min(nzs) <= 1


def test_plan_rejects_impossible_splits():
    from paper_2007_14933_b300 import osbli
    with pytest.raises(osbli.OsbliError):
        osbli.osbli_domain_plan(4, 5, True)
    with pytest.raises(osbli.OsbliError):
        osbli.osbli_domain_plan(100, 65, True)
    k0, nzs, lo, hi = osbli.osbli_domain_plan(10, 1, True)
    assert (k0, nzs, lo, hi) == ([0], [10], [0], [0])
    k0, nzs, lo, hi = osbli.osbli_domain_plan(10, 3, False)
    assert nzs == [4, 3, 3] and lo == [-1, 0, 1] and hi == [1, 2, -1]
