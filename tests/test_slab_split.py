"""Domain split across ranks (slabs of tile layers, one ghost tile layer per
neighbour): the host plan, and two gloo ranks on the CPU that step their
boxes with the FP64 oracle and exchange ghost layers after every step, as
the GPU ranks do over NCCL.  Their interiors must equal the undivided run bit
for bit: every node then gathers what it gathers in the whole domain."""
import os
import socket

import numpy as np
import pytest

from paper_1703_08015_gb300 import geometry as geo
from paper_1703_08015_gb300 import lbm
from paper_1703_08015_gb300 import slab

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.mark.parametrize("n_layers,world,periodic", [(6, 2, False), (6, 2, True), (7, 3, False), (7, 3, True),
                                                     (5, 5, True), (9, 1, True), (64, 8, False)])
def test_plan_covers_every_layer_once(n_layers, world, periodic):
    P = slab.plan(n_layers, world, periodic)
    owned = sorted(layer for p in P for layer in range(p["lo"], p["hi"]))
    assert owned == list(range(n_layers))
    for r, p in enumerate(P):
        b, e = p["interior"]
        assert p["box"][b:e] == list(range(p["lo"], p["hi"]))
        # every ghost layer is some rank's interior layer, received from that rank
        for peer, local, g in p["recv"]:
            assert p["box"][local] == g and P[peer]["lo"] <= g < P[peer]["hi"]
            assert (r, P[peer]["box"].index(g, *P[peer]["interior"]), g) in P[peer]["send"]
        for peer, local, g in p["send"]:
            assert b <= local < e and p["box"][local] == g
        if world == 1:
            assert p["send"] == [] and p["recv"] == [] and p["box"] == list(range(n_layers))
        if not periodic and world > 1:
            assert (p["ghost_lo"] is None) == (r == 0) and (p["ghost_hi"] is None) == (r == world - 1)
    # sends and receives of one pair of ranks are posted in the same order
    for r, p in enumerate(P):
        for q in range(world):
            mine = [g for peer, _, g in p["send"] if peer == q]
            theirs = [g for peer, _, g in P[q]["recv"] if peer == r]
            assert mine == theirs


def test_plan_needs_a_layer_per_rank():
    with pytest.raises(ValueError):
        slab.plan(3, 4, False)


def test_box_mask_stacks_the_box_layers():
    m = np.arange(2 * 3 * 18, dtype=np.int64).reshape(18, 3, 2) % 2
    P = slab.plan(5, 2, True)  # 18 nodes -> 5 layers of 4 (the last one 2 nodes)
    box = slab.box_mask(m.astype(np.uint8), lbm.LBM_D3Q19, 4, P[1])
    want = np.concatenate([m[8:12], m[12:16], m[16:18], m[0:4]])  # ghost 2, interior 3..4, ghost 0
    assert P[1]["box"] == [2, 3, 4, 0]
    assert np.array_equal(box, want)


def _rows(part, local_layer, a, n_box):
    lo = local_layer * a
    return lo, min(lo + a, n_box)


def _rank(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        mask, lat, a, per, tau, F, steps = case
        ax = 2 if lat == 19 else 1
        n = slab.split_axis_len(mask, lat)
        P = slab.plan(-(-n // a), world, bool(per[ax]))
        part = P[rank]
        box = slab.box_mask(mask, lat, a, part)
        per_box = list(per)
        per_box[ax] = 0
        n_box = box.shape[0] if lat == 19 else box.shape[1]

        def take(f, lo, hi):
            return f[:, lo:hi] if lat == 19 else f[:, :, lo:hi]

        f = oracle.init(lat, box)
        g = np.empty_like(f)
        for _ in range(steps):
            oracle.step(lat, box, per_box, tau, F, f, out=g, nthreads=1)
            f, g = g, f
            reqs, bufs = [], []
            for peer, layer, gl in part["send"]:
                t = torch.from_numpy(np.ascontiguousarray(take(f, *_rows(part, layer, a, n_box))))
                reqs.append(dist.isend(t, peer, tag=gl))
                bufs.append(t)
            recvd = []
            for peer, layer, gl in part["recv"]:
                lo, hi = _rows(part, layer, a, n_box)
                t = torch.empty(take(f, lo, hi).shape, dtype=torch.float64)
                reqs.append(dist.irecv(t, peer, tag=gl))
                recvd.append((lo, hi, t))
            for q in reqs:
                q.wait()
            for lo, hi, t in recvd:
                if lat == 19:
                    f[:, lo:hi] = t.numpy()
                else:
                    f[:, :, lo:hi] = t.numpy()
        lo, hi = slab.node_rows(part, a, n)
        out[rank] = take(f, lo, hi).copy()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    m3, _ = geo.sphere_pack_3d(shape=(16, 12, 22), seed=71, r_min=2, r_max=4, target_fluid=0.5)
    m3p, _ = geo.sphere_pack_3d(shape=(12, 16, 24), seed=72, r_min=2, r_max=4, target_fluid=0.5)
    m2, _ = geo.circles_2d(32, 40, seed=73, r_min=2, r_max=4, max_attempts=500)
    return [
        ("d3q19_walls_z", m3, 19, 4, (1, 0, 0), 0.6, (1e-5, 0, 2e-6), 25),
        ("d3q19_periodic_z", m3p, 19, 4, (1, 0, 1), 0.7, (1e-5, 0, 3e-6), 25),
        ("d2q9_split_y", m2, 9, 8, (1, 0, 0), 0.8, (1e-5, 2e-6, 0), 30),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_two_gloo_ranks_match_the_single_domain_bit_for_bit(oracle, case):
    name, mask, lat, a, per, tau, F, steps = case
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), (mask, lat, a, per, tau, F, steps), out), nprocs=world,
                       start_method="spawn", join=True)
    whole = oracle.run(lat, mask, per, tau, F, oracle.init(lat, mask), steps)
    got = np.concatenate([out[r] for r in range(world)], axis=1 if lat == 19 else 2)
    fl = np.broadcast_to(mask.astype(bool), whole.shape)
    assert got.shape == whole.shape
    assert np.array_equal(got[fl].view(np.uint64), whole[fl].view(np.uint64))
