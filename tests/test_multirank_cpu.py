"""Host logic of the multi-GPU form on CPU ranks (gloo, world size 2, 127.0.0.1).

The K build shards by partitions of each class's quartet list (hfx_build_K_part); the
bench runs one replica per rank and reports the maximum time over ranks.  Here two CPU
ranks check that the partitions the C library hands out (hfx_part_range, host-only) tile
every list exactly once across ranks, and that the bench's max-over-ranks reduction and
rank bookkeeping behave on gloo.  No GPU is touched."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

COUNTS = [0, 1, 2, 7, 1000, 105136264, 3 * 10 ** 9 + 7]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2009_03559_gb300 import hfx
    import bench
    ranges = torch.tensor([hfx.part_range(c, rank, world) for c in COUNTS], dtype=torch.int64)
    allr = [torch.zeros_like(ranges) for _ in range(world)]
    dist.all_gather(allr, ranges)
    ok = True
    for i, c in enumerate(COUNTS):
        cuts = sorted((int(r[i][0]), int(r[i][1])) for r in allr)
        ok &= cuts[0][0] == 0 and cuts[-1][1] == c
        ok &= all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
        ok &= all(hi - lo in (c // world, c // world + 1) for lo, hi in cuts)
    mx = bench.max_over_ranks(10.0 + rank, dist)
    ws, rk, local = bench.dist_info()
    ok &= mx == 10.0 + world - 1 and ws == world and rk == rank and local == rank
    with open(os.path.join(out_dir, f"rank{rank}"), "w") as f:
        f.write("ok" if ok else "bad")
    dist.barrier()
    dist.destroy_process_group()


def test_partitions_tile_lists_across_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        assert (tmp_path / f"rank{r}").read_text() == "ok"


def test_part_range_rejects_bad_arguments():
    from paper_2009_03559_gb300 import hfx
    for args in ((10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)):
        with pytest.raises(hfx.HFXError):
            hfx.part_range(*args)
