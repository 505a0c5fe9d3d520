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


def test_derivs_traffic_is_keyed_to_the_kernel_source(tmp_path):
    """The committed DRAM-traffic summary is keyed to the derivative kernel's
    source and flags, independent of where the checkout lives: the bench
    reports it only while the kernel is the one it was measured on."""
    import json
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = os.path.join(root, "paper_1803_00113_gb300", "csrc", "pixel.cu")
    d = json.load(open(os.path.join(root, "profiles", "derivs_kernel_dram.json")))
    h = bench.derivs_source_hash(src)
    if d["derivs_source_sha256_16"] == h:
        assert bench.traffic_per_launch(1000.0) == d["dram_bytes_per_visit"] * 1000.0
    else:
        assert bench.traffic_per_launch(1000.0) is None
    text = open(src, "rb").read()
    # a changed kernel source no longer matches; a changed comment does
    moved = tmp_path / "pixel.cu"
    moved.write_bytes(text.replace(b"kHalfLog2e", b"kHalfLog2E"))
    assert bench.derivs_source_hash(str(moved)) != h
    moved.write_bytes(text.replace(b"// Pixel kernels:", b"// Pixel kernels, reworded:\n//"))
    assert bench.derivs_source_hash(str(moved)) == h
