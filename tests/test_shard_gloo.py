"""The multi-rank path on CPU: two gloo ranks each evaluate their own block
of events (with the oracle standing in for the per-rank CUDA pass), the pass
sums are all-reduced and rescaled by paper_2105_10529_gb300.shard, and the
result must equal one pass over all events; both ranks refine to the same
grid."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from paper_2105_10529_gb300 import shard

torch = pytest.importorskip("torch")

PROC = IN.GG_TT
N_PER_RANK = 120
ITERATION = 2


def _grid():
    rng = np.random.default_rng(5)
    dim, nb = IN.DIM[PROC], 50
    g = np.empty((dim, nb + 1))
    for d in range(dim):
        e = np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 1.8, nb))])
        g[d] = e / e[-1]
    return g


def _rank_sums(rank, grid, pdf, phys):
    """This rank's pass sums [2 + D nb], normalised by its own event count."""
    first, n = shard.event_range(N_PER_RANK, rank)
    dim, nb = grid.shape[0], grid.shape[1] - 1
    s = np.zeros(2 + dim * nb)
    for e in range(first, first + n):
        o = O.event(PROC, phys, pdf, grid, e, ITERATION)
        wn = o.w / n
        s[0] += wn
        s[1] += wn * wn
        for d in range(dim):
            s[2 + d * nb + o.bins[d]] += wn * wn
    return s


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        phys = IN.Physics(seed=1)
        pdf = O.Pdf(IN.make_pdf_grid())
        grid = _grid()
        t = torch.tensor(_rank_sums(rank, grid, pdf, phys), dtype=torch.float64)
        shard.allreduce_pass_sums(t, world)
        s = t.numpy()
        dim, nb = grid.shape[0], grid.shape[1] - 1
        new_grid = O.vegas_refine(s[2:].reshape(dim, nb), grid, phys.alpha)
        np.save(os.path.join(outdir, f"sums_{rank}.npy"), s)
        np.save(os.path.join(outdir, f"grid_{rank}.npy"), new_grid)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_equal_one_pass():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), d), nprocs=world, join=True)
        sums = [np.load(os.path.join(d, f"sums_{r}.npy")) for r in range(world)]
        grids = [np.load(os.path.join(d, f"grid_{r}.npy")) for r in range(world)]
    # every rank holds the same reduced sums and refines to the same grid, bit for bit
    assert np.array_equal(sums[0], sums[1])
    assert np.array_equal(grids[0], grids[1])
    # and they are the sums of one pass over both ranks' events
    phys = IN.Physics(seed=1)
    pdf = O.Pdf(IN.make_pdf_grid())
    grid = _grid()
    ref = O.vegas_pass(PROC, phys, pdf, grid, world * N_PER_RANK, iteration=ITERATION)
    assert sums[0][0] == pytest.approx(ref["sum_w"], rel=1e-12)
    assert sums[0][1] == pytest.approx(ref["sum_w2"], rel=1e-12)
    np.testing.assert_allclose(sums[0][2:], ref["hist"].ravel(), rtol=1e-12, atol=1e-300)
    ref_grid = O.vegas_refine(ref["hist"], grid, phys.alpha)
    np.testing.assert_allclose(grids[0], ref_grid, rtol=0, atol=1e-13)


def test_event_ranges_and_rescale():
    assert shard.event_range(1000, 0) == (0, 1000)
    assert shard.event_range(1000, 3) == (3000, 1000)
    with pytest.raises(ValueError):
        shard.event_range(0, 1)
    # three ranks of weights: the rescaled reduced sums equal the one-pass sums
    rng = np.random.default_rng(9)
    w = rng.exponential(size=3 * 50)
    per = [w[50 * r:50 * (r + 1)] / 50 for r in range(3)]
    red = np.array([sum(p.sum() for p in per), sum((p * p).sum() for p in per)])
    shard.rescale_reduced_sums(red, 3)
    assert red[0] == pytest.approx((w / 150).sum(), rel=1e-14)
    assert red[1] == pytest.approx(((w / 150) ** 2).sum(), rel=1e-14)
