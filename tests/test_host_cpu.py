"""Host-side checks that need no GPU: the C ABI library and its exports, the
input generators, and the multi-rank aggregation of bench.py (gloo ranks)."""
import ctypes
import os
import re
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "bfgpu.h")).read()
    return sorted(set(re.findall(r"BF_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)))


def test_library_loads_and_exports_every_declared_function():
    from paper_2001_06231_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding lists the same functions
    import paper_2001_06231_gb300 as bf
    assert sorted(bf.EXPORTED) == names


def test_workload_generators_are_deterministic():
    from paper_2001_06231_gb300 import workloads as wl
    a, b = wl.unicycle3d(n=(40, 30, 16)), wl.unicycle3d(n=(40, 30, 16))
    assert np.array_equal(a.avoid, b.avoid) and np.array_equal(a.target, b.target)
    assert np.array_equal(a.G, b.G)
    c = wl.unicycle3d(n=(40, 30, 16), seed=99)
    assert not np.array_equal(a.avoid, c.avoid)
    d = wl.di2d()
    assert d.target.sum() == 36 and d.ncells == 4096
    f = wl.fire4d(n=(20, 20, 12, 4), target=((0, 400), (0, 400), (-1.0, 1.0), (10, 15)))
    assert f.G.min() < 0 < f.G.max()          # negative costs over fire


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    units = 1000.0 * (rank + 1)          # ranks solve different amounts of work
    seconds = 0.5 + 0.25 * rank          # and take different times
    v, u, t = bench.whole_job(units, seconds, dist, "cpu")
    out.put((rank, v, u, t))
    dist.destroy_process_group()


def test_bench_whole_job_aggregation_over_gloo_ranks():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, u, t in res:
        assert u == 3000.0 and t == 0.75 and abs(v - 4000.0) < 1e-9


def test_grid_division_by_multiply_high_is_exact():
    """Cell coordinates divide by the grid extents with a multiply-high and a
    shift (division by invariant integers, Granlund & Montgomery 1994):
    l = ceil(log2 n), m = floor(2^32 (2^l - n) / n) + 1, x // n = (mulhi(m, x) + x) >> l
    for every extent 1..16383 and every cell index below 2^31."""
    import numpy as np
    rng = np.random.default_rng(7)
    xs = np.concatenate([np.arange(0, 70000, dtype=np.uint64),
                         np.array([2**31 - 1, 2**31 - 2, 2**30, 2**31 - 64], dtype=np.uint64),
                         rng.integers(0, 2**31, 20000, dtype=np.uint64)])
    for n in range(1, 16384):
        l = (n - 1).bit_length()
        m = ((1 << 32) * ((1 << l) - n)) // n + 1
        assert 0 < m < (1 << 32)
        q = (((xs * np.uint64(m)) >> np.uint64(32)) + xs) >> np.uint64(l)
        assert np.array_equal(q, xs // np.uint64(n)), n
        # near multiples of n, where an off-by-one would show
        k = np.arange(1, 2**31 // n, max(1, (2**31 // n) // 500), dtype=np.uint64) * np.uint64(n)
        for x in (k - np.uint64(1), k):
            q = (((x * np.uint64(m)) >> np.uint64(32)) + x) >> np.uint64(l)
            assert np.array_equal(q, x // np.uint64(n)), n


def test_box_extent_division_by_multiply_high_is_exact():
    """Gather and marking split a lookup or row index t by box extents d with
    m = ceil(2^31 / d) and t // d = mulhi(2t, m) for 1 <= d <= 255 and
    t < 2^23: checked for every d on every t near a multiple of d (where an
    off-by-one would show) up to 2^23, and on every t below 2^16."""
    import numpy as np
    top = np.uint64(1 << 23)
    small = np.arange(0, 1 << 16, dtype=np.uint64)
    for d in range(1, 256):
        m = np.uint64(((1 << 31) + d - 1) // d)
        k = np.arange(1, (1 << 23) // d + 2, dtype=np.uint64) * np.uint64(d)
        ts = np.concatenate([small, k - np.uint64(1), k, top - np.uint64(1 + np.arange(4, dtype=np.uint64))])
        ts = ts[ts < top]
        q = ((ts << np.uint64(1)) * m) >> np.uint64(32)
        assert np.array_equal(q, ts // np.uint64(d)), d


def test_bench_kernel_hash_ignores_comments_and_profiles_parse(tmp_path, monkeypatch):
    """bench.py matches a committed ncu summary to the relax code it was taken
    on by a hash of the sources without comments: a comment edit keeps the
    hash, a code edit changes it; every summary bench.py names carries the
    keys it reads (kernel hash, relax form)."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cuh"
    src.write_text("// header\nint f(int x) { return x + 1; }  /* note */\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [str(src)])
    h0 = bench.kernel_hash()
    src.write_text("// another header\n\nint f(int x) {   return x + 1; }\n")
    assert bench.kernel_hash() == h0
    src.write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_hash() != h0
    for path in bench.PROFILES.values():
        kv = {k.strip(): v.strip() for k, v in (l.split(":", 1) for l in open(path)
                                                  if ":" in l and not l.startswith("#"))}
        assert re.fullmatch(r"[0-9a-f]{16}", kv["kernel_hash"]), path
        form = dict(x.split("=") for x in kv["relax_form"].split())
        assert {"plane_lists", "cell_masks", "input_frontier"} <= set(form), path
