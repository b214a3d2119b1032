"""Independent shifts across ranks (one process per GPU).

The evaluations of one multisection step of Algorithm 1' (Section 2.1: nu_sigma(A, B) from the
inertia of A - sigma B, Sylvester's law) are independent factorizations.  They are partitioned
across ranks round-robin; the only exchange is an all-gather of one int64 count per shift, after
which every rank holds the same counts and takes the same sub-interval, so the ranks stay in step
without any other communication.

The shifts of a step and the bracket update are the library's (kep_multisection_points and
kep_multisection_update, the same code Algorithm 4 runs); this module only shards the shifts and
gathers the counts.

``count`` is any callable sigma -> nu (on a GPU: ``lambda s: problem.factor(s).neg``).  ``dist``
is ``torch.distributed`` (initialised) or None for a single process."""
from __future__ import annotations

from dataclasses import dataclass, field


def shard(items, rank: int, world: int) -> list:
    """The items rank ``rank`` of ``world`` evaluates: positions rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(items)[rank::world]


def gather_counts(local: list[int], total: int, rank: int, world: int, dist=None) -> list[int]:
    """Counts of all ``total`` shifts in shift order, from each rank's ``shard`` of them."""
    if dist is None or world == 1:
        if len(local) != total:
            raise ValueError("a single rank must evaluate every shift")
        return list(local)
    import torch
    per = (total + world - 1) // world
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    buf = torch.full((per,), -1, dtype=torch.int64, device=dev)
    if local:
        buf[:len(local)] = torch.tensor(local, dtype=torch.int64, device=dev)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = [0] * total
    for r in range(world):
        vals = parts[r].cpu().tolist()
        for j, q in enumerate(range(r, total, world)):
            if vals[j] < 0:
                raise RuntimeError(f"rank {r} sent no count for shift {q}")
            out[q] = int(vals[j])
    return out


@dataclass
class Bracket:
    """[lower, upper) with nu(lower) = nu_lower < k <= nu_upper = nu(upper)."""
    lower: float
    upper: float
    nu_lower: int
    nu_upper: int
    history: list = field(default_factory=list)   # (sigma, nu) of every evaluated shift


def multisection_step(count, k: int, br: Bracket, nshift: int, rank: int = 0, world: int = 1,
                      dist=None, count_many=None) -> Bracket:
    """One step: [lower, upper) cut into nshift + 1 equal parts at sigma_q = lower + q (upper -
    lower) / (nshift + 1), q = 1..nshift (the midpoint (lower + upper) / 2 for nshift = 1); keep the
    part whose ends bracket k.  count_many (a list
    of shifts -> their counts, e.g. ConcurrentCounter.count_many) replaces one-at-a-time count."""
    if nshift < 1:
        raise ValueError("nshift >= 1")
    from . import kep
    sig = kep.multisection_points(br.lower, br.upper, nshift)      # the library's Algorithm 1' step
    mine = shard(range(nshift), rank, world)
    local = count_many([sig[q] for q in mine]) if count_many else [int(count(sig[q])) for q in mine]
    nus = gather_counts([int(v) for v in local], nshift, rank, world, dist)
    try:
        lo, hi, nl, nh = kep.multisection_update(k, sig, nus, br.lower, br.upper, br.nu_lower, br.nu_upper)
    except kep.KepError as exc:
        raise RuntimeError("inertia counts are not monotone in sigma (or do not bracket k)") from exc
    return Bracket(lo, hi, nl, nh, br.history + list(zip(sig, nus)))


def multisection(count, k: int, br: Bracket, m_max: int = 20, nshift: int = 8, rank: int = 0,
                 world: int = 1, dist=None, max_steps: int = 200, count_many=None) -> Bracket:
    """Algorithm 1' with nshift shifts per step, until nu_upper - nu_lower <= m_max."""
    if not br.nu_lower < k <= br.nu_upper:
        raise ValueError("the bracket must hold k: nu_lower < k <= nu_upper")
    for _ in range(max_steps):
        if br.nu_upper - br.nu_lower <= m_max:
            return br
        br = multisection_step(count, k, br, nshift, rank, world, dist, count_many)
    raise RuntimeError("multisection did not narrow the bracket (a cluster of eigenvalues?)")


def bisect_to_width(count, k: int, br: Bracket, rel_tol: float = 1e-10, nshift: int = 1, rank: int = 0,
                    world: int = 1, dist=None, max_steps: int = 400, count_many=None):
    """Algorithm 1 run to a width instead of to m_max: narrow [lower, upper) (nu(lower) < k <=
    nu(upper)) until (upper - lower) / max(|lower|, |upper|) < rel_tol, the stop of the straight-
    bisection comparison in Section 4.3.2; lambda_k is taken as the midpoint.  nshift > 1 cuts each
    step into nshift + 1 parts.  Returns (lambda_hat, bracket, steps)."""
    if not br.nu_lower < k <= br.nu_upper:
        raise ValueError("the bracket must hold k: nu_lower < k <= nu_upper")
    steps = 0
    while (br.upper - br.lower) / max(abs(br.lower), abs(br.upper)) >= rel_tol:
        if steps >= max_steps:
            raise RuntimeError("bisection did not reach the width")
        nxt = multisection_step(count, k, br, nshift, rank, world, dist, count_many)
        if (nxt.lower, nxt.upper) == (br.lower, br.upper):
            break                                  # the shifts no longer separate (rounding)
        br = nxt
        steps += 1
    return 0.5 * (br.lower + br.upper), br, steps


class ConcurrentCounter:
    """Several shifts in flight on one device: one context (``Problem``) per in-flight shift, each
    on its own stream and driven from its own host thread (the library calls release the GIL), so
    that one factorization's latency-bound pivot steps overlap another's tensor-core updates.
    ``counters`` are callables sigma -> nu, one per context.  ``count_many`` evaluates a list of
    shifts and returns their counts in order."""

    def __init__(self, counters):
        from concurrent.futures import ThreadPoolExecutor
        if not counters:
            raise ValueError("at least one counter")
        self.counters = list(counters)
        self.pool = ThreadPoolExecutor(max_workers=len(self.counters))

    def count_many(self, sigmas) -> list[int]:
        sigmas = list(sigmas)
        k = len(self.counters)
        # context j evaluates shifts j, j + k, ... in order (each context is used by one thread)
        def run(j):
            return [(q, int(self.counters[j](sigmas[q]))) for q in range(j, len(sigmas), k)]
        out = [0] * len(sigmas)
        for fut in [self.pool.submit(run, j) for j in range(k)]:
            for q, nu in fut.result():
                out[q] = nu
        return out

    def close(self):
        self.pool.shutdown(wait=True)
