"""Host-side logic of the benchmark: the multi-rank reductions (gloo, two
ranks on the CPU) and the reference arm's JSON line."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max(1.5 + rank, world)
    v = bench.reduce_sum(10.0 * (rank + 1), world)
    bench.barrier(world)
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_rank_reductions_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time and the whole job's visits
    assert res[0] == res[1] == (2.5, 30.0)


def test_reference_arm_line(capsys):
    import bench
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--sources", "20"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0


def test_parse_tiles():
    import bench
    assert bench.parse_tiles("128,256,0,0") == [128, 256, 0, 0]
    for bad in ("128,256,0", "a,b,c,d", "1,2,3,-4", ""):
        with pytest.raises(SystemExit):
            bench.parse_tiles(bad)
