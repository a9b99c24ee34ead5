"""Autotuner for the solve queue (`gmres_solve_queue`): how many solves one
batched launch covers (the group width) and how many lanes run groups at once.

Wide groups fill the GPU with fewer, larger launches, but a group holds its
lane until its slowest solve has converged; a second lane lets the next group
run beside those last solves.  Optionally the restart length is tuned too (no
longer than the one asked for): a shorter cycle costs less per step (the
basis grows quadratically per cycle) but may take more steps.  Which balance is best depends on the grid-size
mix, the subspace size and the precision, so it is measured: every candidate
(width, lanes) solves the same sample of the workload (drawn from every grid
size in proportion, so the size mix is kept), the fastest in converged solves
per second wins, and the choice is cached in a JSON file keyed by the
workload.  Widths above the sample size are not tried.
"""
from __future__ import annotations

import collections
import json
import os
import time


def workload_key(A, k: int, precision: str, basis: str) -> str:
    """Cache key: precision, basis storage, subspace size and the grid-size mix."""
    mix = sorted(collections.Counter((a.nx, a.ny) for a in A).items())
    return f"{precision}|{basis}|k{k}|" + ",".join(f"{nx}x{ny}:{c}" for (nx, ny), c in mix)


def candidates(n: int, widths=(16, 32, 64, 128, 256), lanes=(1, 2)):
    """(width, lanes) pairs worth timing on a sample of n solves: a width no
    larger than the sample, and more lanes only when there are that many groups."""
    out = []
    for w in widths:
        if w > n:
            continue
        for nl in lanes:
            if nl == 1 or (n + w - 1) // w >= nl:
                out.append((w, nl))
    if not out:
        out.append((n, 1))
    return out


def choose(timings):
    """timings: list of (width, lanes, solves_per_s[, restart]).  The fastest
    wins; within 1 % of it, fewer lanes, then the wider group (less host work),
    then the longer restart."""
    best = max(t[2] for t in timings)
    near = [t for t in timings if t[2] >= 0.99 * best]
    near.sort(key=lambda t: (t[1], -t[0], -(t[3] if len(t) > 3 else 0)))
    return near[0]


def sample_indices(A, m: int):
    """About m solves of the queue A with its grid-size mix: each size class
    contributes in proportion to its count, its solves spread evenly over the
    class in queue order; returned in queue order."""
    n = len(A)
    if m >= n:
        return list(range(n))
    classes = collections.defaultdict(list)
    for i, a in enumerate(A):
        classes[(a.nx, a.ny)].append(i)
    out = []
    for members in classes.values():
        c = max(1, round(m * len(members) / n))
        out += [members[int(j * len(members) / c)] for j in range(c)]
    return sorted(out)


def _run_queue(lanes, A, b, U, width, nl, tol, restart, maxit, precision):
    """Default runner: solves the sample through the library; converged solves per second."""
    import torch
    from . import binding
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, infos, _ = binding.gmres_solve_queue(lanes[:nl], A, b, U=U, width=width, tol=tol, restart=restart,
                                            maxit=maxit, precision=precision)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return sum(1 for i in infos if i["converged"]) / dt


def tune_queue(lanes, A, b, U=None, sample: int = 64, widths=(16, 32, 64, 128, 256), lane_counts=(1, 2),
               tol=1e-6, restart=200, maxit=5000, precision="c64", basis="f16", cache_path=None, run=None,
               restarts=None, repeats=2):
    """Returns {"width", "lanes", "restart", "solves_per_s", "timings", "key", "cached"}.

    lanes: pre-configured Contexts (at least max(lane_counts)); the first nl of
    them serve a candidate with nl lanes.  restarts: restart lengths to try as
    well (each at most `restart`); None keeps `restart`.  run(lanes, A, b, U,
    width, nl, tol, restart, maxit, precision) -> converged solves/s may
    replace the default runner (the library itself).  Every candidate is timed
    `repeats` times and keeps its best rate, so that the 1 % choice rule is
    not decided by one run's noise (about 2 % from run to run).
    """
    k = 0 if U is None else int(U[0].shape[0])
    ms = sorted({int(m) for m in restarts if 1 <= int(m) <= restart}) if restarts else [int(restart)]
    if not ms:
        raise ValueError(f"no restart length in {restarts} is within [1, {restart}]")
    if repeats < 1:
        raise ValueError(f"repeats={repeats} < 1")
    # the tolerance and the restart lengths tried are always part of the key: a
    # choice made for GMRES(200) must not answer a call that asks for GMRES(100)
    key = workload_key(A, k, precision, basis) + f"|tol{tol:g}|m" + ",".join(str(m) for m in ms)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key], key=key, cached=True)
    if len(lanes) < max(lane_counts):
        raise ValueError(f"{len(lanes)} contexts for up to {max(lane_counts)} lanes")
    idx = sample_indices(A, sample)
    As = [A[i] for i in idx]
    bs = [b[i] for i in idx]
    Us = None if U is None else [U[i] for i in idx]
    run = run or _run_queue
    timings = []
    for m in ms:
        for w, nl in candidates(len(idx), widths, lane_counts):
            t = (w, nl, max(float(run(lanes, As, bs, Us, w, nl, tol, m, maxit, precision))
                            for _ in range(repeats)))
            # (width, lanes, solves/s), with the restart length appended when it is tuned
            timings.append(t + (m,) if restarts else t)
    best = choose(timings)
    w, nl, v = best[:3]
    res = {"width": w, "lanes": nl, "restart": best[3] if restarts else int(restart), "solves_per_s": v,
           "timings": timings}
    if cache_path:
        cache[key] = res
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(res, key=key, cached=False)
