"""Autotuner for the library's launch shapes.

Every knob of the library's tuning table (``nacc_tune_set``) selects among
launch shapes that produce identical results; only the speed differs, and it
depends on the workload (ray lengths, how much is pruned, grid occupancy). The
tuner measures each candidate value on the caller's own buffers with CUDA
events on the launching stream and keeps the fastest, one knob at a time.
"""
from __future__ import annotations

import statistics
from typing import Callable, Dict, Iterable

import torch

from . import _lib

# Candidate values per knob (all valid for every input).
CANDIDATES = {
    "march_tile_rays": (2, 4, 8, 16, 32),
    "march_occupancy": (0, 1),
    "march_unroll": (0, 1),
    "prune_tile_rays": (2, 4, 8, 16, 32),
    "prune_occupancy": (0, 1, 2),
    "prune_interleave": (2, 4),
    "render_fwd_prefetch": (0, 1),
    "render_fwd_occupancy": (0, 1, 2),
    "render_bwd_occupancy": (0, 1, 2),
    "render_bwd_prefetch": (0, 1),
}


def time_ms(fn: Callable[[], None], reps: int = 5, warmup: int = 1, before: Callable[[], None] = None) -> float:
    """Median device time of ``fn`` (CUDA events on the current stream)."""
    for _ in range(warmup):
        if before:
            before()
        fn()
    out = []
    for _ in range(reps):
        if before:
            before()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def tune_knob(knob: str, fn: Callable[[], None], candidates: Iterable[int] = None, reps: int = 7,
              before: Callable[[], None] = None, margin: float = 0.03) -> Dict[str, object]:
    """Time ``fn`` under each candidate value of ``knob`` and set the fastest.

    Candidates are timed round-robin inside each repetition (so slow drifts of
    clock or temperature hit all of them alike) and compared by their median.
    The value the knob held before (the library default, or an earlier choice)
    stays unless the fastest candidate beats it by more than ``margin``: a win
    inside the run-to-run noise is not worth changing the launch shape for.
    """
    cands = tuple(CANDIDATES[knob] if candidates is None else candidates)
    incumbent = _lib.tune_get(knob)
    if incumbent not in cands:
        cands = (incumbent,) + cands
    samples = {v: [] for v in cands}
    for v in cands:  # one untimed run each (module loading, first-touch)
        _lib.tune_set(knob, v)
        if before:
            before()
        fn()
    for _ in range(reps):
        for v in cands:
            _lib.tune_set(knob, v)
            if before:
                before()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            samples[v].append(e0.elapsed_time(e1))
    times = {v: statistics.median(t) for v, t in samples.items()}
    best = min(times, key=times.get)
    if times[best] > (1.0 - margin) * times[incumbent]:
        best = incumbent
    _lib.tune_set(knob, best)
    return {"knob": knob, "best": best, "ms": {str(k): round(t, 4) for k, t in times.items()}}


def tune_hot_path(hp, sc, batch: int = 0, reps: int = 7, flush: Callable[[], None] = None):
    """Tune the knobs of one ``pipeline.HotPath`` on one batch of a ``scenarios.Scenario``
    (leaves its buffers holding that batch). ``flush`` runs before every timed
    repetition (e.g. a write larger than L2, as in the measured step)."""
    bt = sc.batches[batch]
    rec = []

    def tk(knob, fn):
        return tune_knob(knob, fn, reps=reps, before=flush)

    march = lambda: hp.march(bt["o"], bt["d"], bt["time"], bt["slot"])
    rec.append(tk("march_tile_rays", march))
    rec.append(tk("march_occupancy", march))
    rec.append(tk("march_unroll", march))
    march()
    M = int(hp.n_m.item())
    sc.field_marched(hp, batch, M)
    prune = lambda: hp.prune(M)
    rec.append(tk("prune_tile_rays", prune))
    rec.append(tk("prune_occupancy", prune))
    rec.append(tk("prune_interleave", prune))
    hp.prune(M)
    S = int(hp.n_k.item())
    sc.field_kept(hp, batch, S)
    fwd = lambda: hp.render_fwd(S)
    rec.append(tk("render_fwd_prefetch", fwd))
    rec.append(tk("render_fwd_occupancy", fwd))
    hp.render_fwd(S)
    hp.g_color.uniform_(-1e-6, 1e-6)
    rec.append(tk("render_bwd_occupancy", lambda: hp.render_bwd(S)))
    rec.append(tk("render_bwd_prefetch", lambda: hp.render_bwd(S)))
    # forward + backward with the optical depth recomputed, or saved by the forward
    times = {}
    for saved in (False, True):
        hp.save_optical_depth = saved
        times[int(saved)] = time_ms(lambda: (hp.render_fwd(S), hp.render_bwd(S)), reps=reps, before=flush)
    hp.save_optical_depth = times[1] < times[0]
    rec.append({"knob": "save_optical_depth", "best": int(hp.save_optical_depth),
                "ms": {str(k): round(v, 4) for k, v in times.items()}})
    torch.cuda.synchronize()
    hp.check_status("autotune")
    return {r["knob"]: r for r in rec}
