"""Shifts sharded across ranks (world_size 2, gloo on CPU): the counts gathered from both ranks,
and the bracket they give, equal the single-process Algorithm 1' with the same shifts; each rank
evaluates only its share; a rank that fails before the exchange ends the other's collective with
an error instead of a hang.

nu comes from the closed form of a diagonal pencil (nu = #{a_ii / b_ii < sigma}), so the test needs
no GPU; on a GPU the same code takes ``problem.factor(sigma).neg``."""
import os
import socket
import traceback
from datetime import timedelta

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import three_stage as ts
from paper_1710_05134_gb300 import multishift as ms

N, K, NSHIFT, MMAX = 4000, 1717, 8, 20


def _pencil():
    rng = np.random.default_rng(5)
    a = rng.normal(size=N)
    b = rng.uniform(0.5, 2.0, size=N)
    return np.sort(a / b)


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=20))
        lam = _pencil()
        calls = []

        def count(s):
            calls.append(s)
            return int(np.searchsorted(lam, s, side="left"))

        if mode == "fail" and rank == 1:
            raise RuntimeError("rank 1 fails before the exchange")
        br = ms.Bracket(-10.0, 10.0, 0, N)
        res = ms.multisection(count, K, br, m_max=MMAX, nshift=NSHIFT, rank=rank, world=world, dist=dist)
        out.put((rank, "ok", (res.lower, res.upper, res.nu_lower, res.nu_upper, res.history, calls)))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as exc:       # reported to the parent, which decides
        out.put((rank, "error", f"{type(exc).__name__}: {exc}\n{traceback.format_exc(limit=2)}"))


def _run(mode, world=2, wait=60):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, kind, val = q.get(timeout=wait)
        res[r] = (kind, val)
    for p in procs:
        p.join(timeout=wait)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank did not exit")
    return res


class _Ops:
    def __init__(self, lam):
        self.lam = lam

    def nu(self, s):
        return int(np.searchsorted(self.lam, s, side="left"))


def test_shard_positions():
    assert ms.shard(range(8), 0, 3) == [0, 3, 6]
    assert ms.shard(range(8), 2, 3) == [2, 5]
    assert sorted(sum((ms.shard(range(11), r, 4) for r in range(4)), [])) == list(range(11))
    with pytest.raises(ValueError):
        ms.shard(range(3), 3, 3)


def test_single_rank_matches_oracle_multisection():
    lam = _pencil()
    ops = _Ops(lam)
    ref = ts.multisect_mmax(ops, K, ts.Interval(-10.0, 10.0, 0, N, []), m_max=MMAX, nshift=NSHIFT)
    got = ms.multisection(ops.nu, K, ms.Bracket(-10.0, 10.0, 0, N), m_max=MMAX, nshift=NSHIFT)
    assert (got.lower, got.upper, got.nu_lower, got.nu_upper) == (ref.lower, ref.upper, ref.nu_lower, ref.nu_upper)
    assert got.nu_lower < K <= got.nu_upper and got.nu_upper - got.nu_lower <= MMAX
    # the bracket holds lambda_k: lambda_k in [lower, upper)
    assert got.lower <= lam[K - 1] < got.upper


def test_two_ranks_gloo():
    res = _run("ok")
    assert all(kind == "ok" for kind, _ in res.values()), res
    (lo0, hi0, nl0, nu0, h0, c0), (lo1, hi1, nl1, nu1, h1, c1) = res[0][1], res[1][1]
    single = ms.multisection(_Ops(_pencil()).nu, K, ms.Bracket(-10.0, 10.0, 0, N), m_max=MMAX, nshift=NSHIFT)
    assert (lo0, hi0, nl0, nu0) == (lo1, hi1, nl1, nu1) == (single.lower, single.upper, single.nu_lower, single.nu_upper)
    assert h0 == h1 == single.history
    steps = len(single.history) // NSHIFT
    assert len(c0) == len(c1) == steps * NSHIFT // 2        # each rank evaluated half the shifts
    assert not set(c0) & set(c1)


def test_rank_failure_is_reported():
    res = _run("fail")
    assert res[1][0] == "error" and "fails before the exchange" in res[1][1]
    assert res[0][0] == "error"                             # the peer's collective errored, no hang


def test_concurrent_counter_keeps_shift_order():
    """Several contexts evaluating one step's shifts from their own threads give the counts in
    shift order, no context used by two threads at once, and the same bracket as one context."""
    import threading
    import time
    lam = _pencil()
    lock = threading.Lock()
    active, peak, calls = {}, {}, {}

    def make(j):
        def count(s):
            with lock:
                active[j] = active.get(j, 0) + 1
                peak[j] = max(peak.get(j, 0), active[j])
                calls[j] = calls.get(j, 0) + 1
            time.sleep(0.001)
            with lock:
                active[j] -= 1
            return int(np.searchsorted(lam, s, side="left"))
        return count

    cc = ms.ConcurrentCounter([make(0), make(1)])
    try:
        sig = list(np.linspace(-2.0, 2.0, 9))
        assert cc.count_many(sig) == [int(np.searchsorted(lam, s, side="left")) for s in sig]
        got = ms.multisection(None, K, ms.Bracket(-10.0, 10.0, 0, N), m_max=MMAX, nshift=NSHIFT,
                              count_many=cc.count_many)
    finally:
        cc.close()
    single = ms.multisection(_Ops(lam).nu, K, ms.Bracket(-10.0, 10.0, 0, N), m_max=MMAX, nshift=NSHIFT)
    assert (got.lower, got.upper, got.nu_lower, got.nu_upper) == (single.lower, single.upper, single.nu_lower,
                                                                   single.nu_upper)
    # every context served, none by two threads at once
    assert set(calls) == {0, 1} and max(peak.values()) == 1


def test_bisection_to_width_matches_oracle():
    """Straight bisection to a relative width (the comparison run of Section 4.3.2) gives the
    oracle's lambda_k and iteration count, and lambda_k of the closed-form diagonal pencil within
    the width; multisection reaches the same width in fewer steps."""
    lam = _pencil()
    ops = _Ops(lam)
    lo, hi = -10.0, 10.0
    ref, it_ref = ts.bisect_straight(ops, K, lo, hi, rel_tol=1e-10)
    got, br, steps = ms.bisect_to_width(ops.nu, K, ms.Bracket(lo, hi, 0, N), rel_tol=1e-10)
    assert got == ref and steps == it_ref
    assert abs(got - lam[K - 1]) <= 1e-10 * max(abs(br.lower), abs(br.upper))
    assert br.nu_lower < K <= br.nu_upper
    got8, br8, steps8 = ms.bisect_to_width(ops.nu, K, ms.Bracket(lo, hi, 0, N), rel_tol=1e-10, nshift=8)
    assert abs(got8 - lam[K - 1]) <= 1e-10 * max(abs(br8.lower), abs(br8.upper))
    assert steps8 < steps / 2
    with pytest.raises(ValueError):
        ms.bisect_to_width(ops.nu, K, ms.Bracket(lo, hi, K, N))
