"""The batched autotuner's persistent cache (host logic, on the CPU): keys, round trip,
and robustness to missing, corrupt or foreign files."""
import json

from paper_2001_04886_gb300 import _binding as B

CFG = dict(threads=256, ctas_per_sm=2, largest_first=1, cluster=4, coop_min_n=16384)


def test_key_depends_on_device_shape_and_method():
    shapes = [(32, 32), (200, 200), (57, 57)]
    k = B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300")
    assert k == B.tune_cache_key([list(sh) for sh in shapes], 4, 20, "NVIDIA GB300")   # stable
    assert k != B.tune_cache_key(shapes[::-1], 4, 20, "NVIDIA GB300")                # batch order matters
    assert k != B.tune_cache_key(shapes, 8, 40, "NVIDIA GB300")
    assert k != B.tune_cache_key(shapes, 4, 20, "another device")
    assert k != B.tune_cache_key(shapes[:2], 4, 20, "NVIDIA GB300")
    # the stopping test, sigma, the x0 guard and the library build change what was timed
    assert k != B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", tol=1e-10)
    assert k != B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", sigma=0.25)
    assert k != B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", x0_guard=True)
    assert k != B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", build="0" * 16)
    assert k != B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", precision="fp32")
    assert k == B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", precision="fp64")
    assert k == B.tune_cache_key(shapes, 4, 20, "NVIDIA GB300", build=B.library_build_id())


def test_concurrent_writers_keep_each_others_entries(tmp_path):
    """Writers in separate processes serialise their read-modify-write on a lock file."""
    import multiprocessing as mp

    p = str(tmp_path / "tune.json")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_put_many, args=(p, i)) for i in range(4)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(60)
        assert pr.exitcode == 0
    data = json.load(open(p))
    assert sorted(data) == sorted(f"w{i}-{j}" for i in range(4) for j in range(25))


def _put_many(path, i):
    for j in range(25):
        B.tune_cache_put(path, f"w{i}-{j}", CFG)


def test_round_trip_and_replacement(tmp_path):
    p = str(tmp_path / "tune.json")
    assert B.tune_cache_get(p, "k") is None                       # no file
    B.tune_cache_put(p, "k", CFG)
    assert B.tune_cache_get(p, "k") == CFG
    B.tune_cache_put(p, "k2", dict(CFG, cluster=2))
    assert B.tune_cache_get(p, "k") == CFG and B.tune_cache_get(p, "k2")["cluster"] == 2
    B.tune_cache_put(p, "k", dict(CFG, threads=128))
    assert B.tune_cache_get(p, "k")["threads"] == 128
    assert sorted(json.load(open(p))) == ["k", "k2"]
    assert not list(tmp_path.glob("*.tmp"))


def test_corrupt_or_partial_files_are_ignored(tmp_path):
    p = tmp_path / "tune.json"
    p.write_text("{not json")
    assert B.tune_cache_get(str(p), "k") is None
    B.tune_cache_put(str(p), "k", CFG)                            # rewrites a corrupt file
    assert B.tune_cache_get(str(p), "k") == CFG
    p.write_text(json.dumps({"k": {"threads": 256}}))              # missing fields
    assert B.tune_cache_get(str(p), "k") is None
    p.write_text(json.dumps([1, 2, 3]))                            # not a mapping
    assert B.tune_cache_get(str(p), "k") is None
