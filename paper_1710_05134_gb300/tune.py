"""Choice of the front order from which the Schur update runs on the tensor cores, and of the tile
edge of the other fronts' updates, by timing.

The exact-splitting tensor-core update pays a fixed cost per pivot window (digit slicing, a
persistent launch, pipeline fill) that small fronts cannot amortise, while the FP64 FMA update is
1/20 of its rate on large ones; the best crossover depends on the pattern's front sizes.  This
times complete factorizations at a few candidate thresholds on the caller's pattern and keeps the
fastest (ties to the larger threshold, which keeps more fronts on the FP64 path).  Inertia counts
do not depend on the threshold (Sylvester's law of inertia, Section 2.1); they are checked to be
equal across the candidates."""
from __future__ import annotations

import time


def tune_min_front(problem, sigmas, candidates=(256, 512, 768, 1024, 1536), reps: int = 1, sync=None,
                   clock=time.perf_counter) -> dict:
    """Time ``reps`` rounds of factorizations at ``sigmas`` for each candidate threshold, set the
    fastest on ``problem`` (``set_schur_mode(True, best)``) and return
    {"best": best, "seconds": {candidate: seconds per factorization}, "nu": counts}.
    ``sync`` (e.g. torch.cuda.synchronize) is called around each timed region."""
    sigmas = list(sigmas)
    if not sigmas or not candidates or reps < 1:
        raise ValueError("need shifts, candidates and reps >= 1")
    sync = sync or (lambda: None)
    secs, counts = {}, None
    for mf in candidates:
        problem.set_schur_mode(True, int(mf))
        problem.factor(sigmas[0])                    # workspace planning for this threshold, untimed
        sync()
        t0 = clock()
        nus = [problem.factor(s).neg for _ in range(reps) for s in sigmas]
        sync()
        secs[int(mf)] = (clock() - t0) / (reps * len(sigmas))
        if counts is None:
            counts = nus
        elif nus != counts:
            raise RuntimeError(f"inertia counts changed with the threshold {mf}: {nus} != {counts}")
    best = min(secs, key=lambda m: (secs[m], -m))
    problem.set_schur_mode(True, best)
    return {"best": best, "seconds": secs, "nu": counts}


def tune_schur(problem, sigmas, thresholds=(256, 512, 1024), tiles=(32, 64), reps: int = 1, sync=None,
               clock=time.perf_counter) -> dict:
    """Time ``reps`` rounds of factorizations at ``sigmas`` for every (tensor-core threshold, tile
    edge) pair, set the fastest pair on ``problem`` and return {"best": (threshold, tile),
    "seconds": {(threshold, tile): seconds per factorization}, "nu": counts}.  Ties go to the larger
    threshold, then the larger tile.  Counts must be equal for every pair (Sylvester's law)."""
    sigmas = list(sigmas)
    if not sigmas or not thresholds or not tiles or reps < 1:
        raise ValueError("need shifts, thresholds, tiles and reps >= 1")
    sync = sync or (lambda: None)
    secs, counts = {}, None
    for mf in thresholds:
        for tile in tiles:
            problem.set_schur_mode(True, int(mf))
            problem.set_schur_tile(int(tile))
            problem.factor(sigmas[0])                # workspace planning, graph capture: untimed
            sync()
            t0 = clock()
            nus = [problem.factor(s).neg for _ in range(reps) for s in sigmas]
            sync()
            secs[(int(mf), int(tile))] = (clock() - t0) / (reps * len(sigmas))
            if counts is None:
                counts = nus
            elif nus != counts:
                raise RuntimeError(f"inertia counts changed with (threshold, tile) = ({mf}, {tile}): {nus} != {counts}")
    best = min(secs, key=lambda k: (secs[k], -k[0], -k[1]))
    problem.set_schur_mode(True, best[0])
    problem.set_schur_tile(best[1])
    return {"best": best, "seconds": secs, "nu": counts}
