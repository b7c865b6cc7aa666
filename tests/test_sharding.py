"""Multi-rank decomposition on CPU (gloo, world size 2).

Each rank filters its row band of one image (input window = band + halo)
with the FP64 checker; rank 0 gathers the bands and checks them against the
unsplit image bit for bit.  The image gradient of each band (window band +
2W, cotangent band + W) is gathered the same way, and the per-band sigma_r
gradients are all-reduced and compared with the unsplit sum."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1603_08109_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H, W, r, ss, sr, N = 37, 29, 3, 1.0, 30.0, 20
        img = synth.blocks_image(H, W, 6, 20.0, seed=3)
        g = synth.random_like((H, W), seed=4).astype(np.float64)
        w = oracle.spatial_kernel(1, r, ss)
        band = shard.row_bands(H, world, r)[rank]
        win = img[band.in0:band.in1]
        out = oracle.gpa_alg2(win, w, sr, N)[band.y0 - band.in0:band.y1 - band.in0]
        gb = shard.row_bands(H, world, r, grad=True)[rank]
        gwin = img[gb.in0:gb.in1]
        gcot = np.zeros_like(gwin, dtype=np.float64)
        gcot[gb.g0 - gb.in0:gb.g1 - gb.in0] = g[gb.g0:gb.g1]
        gin, _ = oracle.gpa_grad(gwin, w, sr, N, gcot)
        gin = gin[gb.y0 - gb.in0:gb.y1 - gb.in0]
        own = np.zeros_like(gwin, dtype=np.float64)
        own[gb.y0 - gb.in0:gb.y1 - gb.in0] = g[gb.y0:gb.y1]
        _, gs = oracle.gpa_grad(gwin, w, sr, N, own)
        gs_t = torch.tensor([gs], dtype=torch.float64)
        dist.all_reduce(gs_t)
        rows = [None] * world
        dist.all_gather_object(rows, (band.y0, out, gin))
        if rank == 0:
            full = oracle.gpa_alg2(img, w, sr, N)
            full_gin, full_gs = oracle.gpa_grad(img, w, sr, N, g)
            ok_out = all(np.array_equal(o, full[y0:y0 + o.shape[0]]) for y0, o, _ in rows)
            err_gin = max(float(np.abs(gi - full_gin[y0:y0 + gi.shape[0]]).max()) for y0, _, gi in rows)
            covered = sorted((y0, y0 + o.shape[0]) for y0, o, _ in rows)
            result_q.put((ok_out, err_gin, float(gs_t.item()), full_gs, covered))
    finally:
        dist.destroy_process_group()


def test_row_bands_cover_image():
    for H, world, r in ((37, 2, 3), (1, 1, 5), (100, 7, 9), (5, 4, 2)):
        bands = shard.row_bands(H, world, r)
        assert bands[0].y0 == 0 and bands[-1].y1 == H
        assert all(b.y1 == c.y0 for b, c in zip(bands, bands[1:]))
        assert max(b.rows for b in bands) - min(b.rows for b in bands) <= 1
        for b in bands:
            assert b.in0 == max(0, b.y0 - r) and b.in1 == min(H, b.y1 + r)


def test_assign_images_balances_costs():
    costs = [9, 7, 6, 5, 4, 3, 2, 1]
    parts = shard.assign_images(costs, 2)
    assert sorted(sum(parts, [])) == list(range(len(costs)))
    loads = [sum(costs[k] for k in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= 1


def test_two_rank_band_decomposition_matches_unsplit_image():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    ok_out, err_gin, gs_sum, gs_full, covered = q.get(timeout=10)
    assert ok_out
    assert err_gin <= 1e-12
    assert gs_sum == pytest.approx(gs_full, rel=1e-12, abs=1e-14)
    assert covered[0][0] == 0 and covered[-1][1] == 37
