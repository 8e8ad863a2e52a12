"""The row-partitioned solve across processes: two ranks, each a process of
its own on cuda:0, solve one graph together through solve_rows with a gloo
RowExchange (host-staged all-gather of w, all-reduce of the fixed-point
sums).  The ranks' kernels never wait on one another (every exchange is on
the host between launches), so they may share a GPU.  The FP64 result
equals pagerank_solve's bit for bit, as does the iteration count; FP32
equals the one-process solve over the same two ranges."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    try:
        import torch.distributed as dist
        import ffg_inputs as fi
        import paper_2210_01465_gb300 as ffg
        from paper_2210_01465_gb300.multi import RowExchange, solve_rows, split_rows
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        ffg.load()
        spec = fi.single_large()
        fd = torch.from_numpy(fi.runtimes(spec, seed=4)).cuda()
        g = ffg.build_graph(ffg.Space.from_spec(spec), fd, ffg.ADJACENT)
        bounds = split_rows(g.in_ptr.cpu().numpy(), world)
        out = {}
        for prec in (ffg.F64, ffg.F32):
            ex = RowExchange(bounds, ffg.pagerank_rows_w_bytes(prec), host=True)
            x, it, res, conv = solve_rows(g, [bounds[rank]], 0.85, 1e-12, prec=prec, exchange=ex)
            out[prec] = (x.cpu().numpy(), it, conv)
        dist.destroy_process_group()
        q.put((rank, out, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, f"{type(e).__name__}: {e}"))


@pytest.mark.timeout(600)
def test_row_partitioned_solve_two_processes_matches_single_launch():
    import ffg_inputs as fi
    import paper_2210_01465_gb300 as ffg
    from paper_2210_01465_gb300.multi import solve_rows, split_rows
    ffg.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, out, err = q.get(timeout=500)
        assert err is None, err
        res[rank] = out
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ffg.load()
    spec = fi.single_large()
    fd = torch.from_numpy(fi.runtimes(spec, seed=4)).cuda()
    g = ffg.build_graph(ffg.Space.from_spec(spec), fd, ffg.ADJACENT)
    x64, it64, _, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    assert conv
    bounds = split_rows(g.in_ptr.cpu().numpy(), world)
    x32, it32, _, _ = solve_rows(g, bounds, 0.85, 1e-12, prec=ffg.F32)
    for rank in range(world):
        xr, it, conv = res[rank][ffg.F64]
        assert conv and it == it64
        np.testing.assert_array_equal(xr, x64.cpu().numpy())
        xr, it, conv = res[rank][ffg.F32]
        assert conv and it == it32
        np.testing.assert_array_equal(xr, x32.cpu().numpy())
