"""Host logic of the solve-queue autotuner (no GPU): the workload key, the
candidate set, the choice rule, the strided sample and the cache."""
import json

from paper_1902_00090_gb300 import autotune


class Op:
    def __init__(self, nx, ny):
        self.nx, self.ny, self.D = nx, ny, nx * ny


def test_workload_key_counts_the_size_mix():
    A = [Op(128, 128), Op(256, 256), Op(128, 128)]
    assert autotune.workload_key(A, 8, "c64", "f16") == "c64|f16|k8|128x128:2,256x256:1"


def test_candidates_respect_the_sample_size():
    assert autotune.candidates(40, widths=(16, 32, 64), lanes=(1, 2)) == [(16, 1), (16, 2), (32, 1), (32, 2)]
    # one group of 64: a second lane would have nothing to do
    assert autotune.candidates(64, widths=(64,), lanes=(1, 2)) == [(64, 1)]
    assert autotune.candidates(5, widths=(16,), lanes=(1, 2)) == [(5, 1)]


def test_choice_prefers_fewer_lanes_then_wider_groups_within_one_percent():
    t = [(16, 1, 100.0), (32, 1, 99.5), (32, 2, 100.5), (64, 2, 80.0)]
    assert autotune.choose(t) == (32, 1, 99.5)
    assert autotune.choose([(16, 1, 50.0), (16, 2, 60.0)]) == (16, 2, 60.0)


def test_sample_keeps_the_size_mix_whatever_the_order():
    sizes = [(128, 128), (192, 192), (256, 256), (384, 256)]
    cyclic = [Op(*sizes[i % 4]) for i in range(1024)]       # sizes interleaved
    blocks = [Op(*sizes[i // 256]) for i in range(1024)]     # sizes in blocks
    for A in (cyclic, blocks):
        idx = autotune.sample_indices(A, 64)
        assert len(idx) == 64 and idx == sorted(idx) and len(set(idx)) == 64
        mix = sorted((A[i].nx, A[i].ny) for i in idx)
        assert all(mix.count(s) == 16 for s in sizes)
    assert autotune.sample_indices(cyclic[:10], 64) == list(range(10))


def test_tune_times_every_candidate_once_and_caches(tmp_path):
    A = [Op(128, 128)] * 48 + [Op(192, 192)] * 16
    b = list(range(64))
    calls = []

    def run(lanes, As, bs, Us, w, nl, tol, restart, maxit, prec):
        calls.append((w, nl, len(As)))
        return {(16, 1): 10.0, (16, 2): 12.0, (32, 1): 11.0, (32, 2): 11.5, (64, 1): 9.0}[(w, nl)]

    cache = str(tmp_path / "tune.json")
    r = autotune.tune_queue(["c0", "c1"], A, b, sample=64, widths=(16, 32, 64), cache_path=cache, run=run,
                            repeats=1)
    assert (r["width"], r["lanes"], r["cached"]) == (16, 2, False)
    assert sorted(c[:2] for c in calls) == [(16, 1), (16, 2), (32, 1), (32, 2), (64, 1)]
    assert all(c[2] == 64 for c in calls)
    stored = json.load(open(cache))
    assert r["key"] in stored and stored[r["key"]]["width"] == 16
    r2 = autotune.tune_queue(["c0", "c1"], A, b, sample=64, widths=(16, 32, 64), cache_path=cache, run=run,
                             repeats=1)
    assert r2["cached"] and (r2["width"], r2["lanes"]) == (16, 2) and len(calls) == 5


def test_tune_repeats_each_candidate_and_keeps_its_best_rate():
    A = [Op(128, 128)] * 32
    b = list(range(32))
    noisy = {(16, 1): iter([10.0, 13.0]), (16, 2): iter([12.0, 12.1]), (32, 1): iter([12.5, 9.0])}
    calls = []

    def run(lanes, As, bs, Us, w, nl, tol, m, maxit, prec):
        calls.append((w, nl))
        return next(noisy[(w, nl)])

    r = autotune.tune_queue(["c0", "c1"], A, b, sample=32, widths=(16, 32), run=run, repeats=2)
    assert len(calls) == 6 and sorted(set(calls)) == [(16, 1), (16, 2), (32, 1)]
    # best of two: (16, 1) reaches 13.0, above the others' best by more than 1 %
    assert (r["width"], r["lanes"], r["solves_per_s"]) == (16, 1, 13.0)


def test_cache_key_separates_restart_lengths_and_tolerances(tmp_path):
    A = [Op(128, 128)] * 16
    b = list(range(16))
    seen = []

    def run(lanes, As, bs, Us, w, nl, tol, m, maxit, prec):
        seen.append((m, tol))
        return 10.0

    cache = str(tmp_path / "t.json")
    r200 = autotune.tune_queue(["c0"], A, b, sample=16, widths=(16,), lane_counts=(1,), restart=200, run=run,
                               cache_path=cache, repeats=1)
    r100 = autotune.tune_queue(["c0"], A, b, sample=16, widths=(16,), lane_counts=(1,), restart=100, run=run,
                               cache_path=cache, repeats=1)
    assert not r100["cached"] and r100["restart"] == 100 and r200["restart"] == 200
    assert r100["key"] != r200["key"] and seen == [(200, 1e-6), (100, 1e-6)]
    r4 = autotune.tune_queue(["c0"], A, b, sample=16, widths=(16,), lane_counts=(1,), restart=100, tol=1e-4,
                             run=run, cache_path=cache, repeats=1)
    assert not r4["cached"] and r4["key"] != r100["key"]
    assert autotune.tune_queue(["c0"], A, b, sample=16, widths=(16,), lane_counts=(1,), restart=100, run=run,
                               cache_path=cache, repeats=1)["cached"]


def test_tune_restart_lengths_too(tmp_path):
    A = [Op(128, 128)] * 32
    b = list(range(32))
    seen = []

    def run(lanes, As, bs, Us, w, nl, tol, m, maxit, prec):
        seen.append((w, nl, m))
        return {100: 10.0, 150: 12.0, 200: 11.0}[m] + (0.5 if (w, nl) == (16, 2) else 0.0)

    r = autotune.tune_queue(["c0", "c1"], A, b, sample=32, widths=(16, 32), restarts=(100, 150, 200, 300),
                            restart=200, run=run, cache_path=str(tmp_path / "t.json"))
    # 300 is above the restart asked for: not tried
    assert sorted({m for _, _, m in seen}) == [100, 150, 200]
    assert (r["width"], r["lanes"], r["restart"]) == (16, 2, 150)
    assert all(len(t) == 4 for t in r["timings"]) and "|m100,150,200" in r["key"]
    # without restart candidates the timings keep their three fields and the given restart
    r2 = autotune.tune_queue(["c0", "c1"], A, b, sample=32, widths=(16,), restart=150, run=run)
    assert all(len(t) == 3 for t in r2["timings"]) and r2["restart"] == 150
