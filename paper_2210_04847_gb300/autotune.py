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
    "march_tile_rays": (1, 2, 4, 8, 16, 32),
    "march_occupancy": (0, 1),
    "march_unroll": (0, 1),
    "march_coarse": (0, 1),
    "march_box_tile": (0, 1, 2, 3),
    "prune_tile_rays": (2, 4, 6, 8, 12, 16, 24, 32),
    "prune_occupancy": (0, 1, 2),
    "prune_interleave": (2, 4),
    "render_fwd_prefetch": (0, 1),
    "render_fwd_occupancy": (0, 1, 2),
    "render_bwd_occupancy": (0, 1, 2),
    "render_bwd_prefetch": (0, 1),
    "render_fwd_stages": (0, 2, 3, 4),
    "render_bwd_stages": (0, 2, 3, 4),
    "render_mse_occupancy": (0, 1, 2),
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


def tune_configs(name: str, configs, fn: Callable[[], None], reps: int = 7, before: Callable[[], None] = None,
                 margin: float = 0.03) -> Dict[str, object]:
    """Time ``fn`` under each configuration (a dict knob -> value) and set the
    fastest. Configurations are timed round-robin inside each repetition (so
    slow drifts of clock or temperature hit all of them alike) and compared by
    their median. The first configuration is the incumbent: it stays unless
    another beats it by more than ``margin`` (a win inside the run-to-run noise
    is not worth changing the launch shape for)."""
    configs = [dict(c) for c in configs]

    def apply(c):
        for k, v in c.items():
            _lib.tune_set(k, v)

    samples = [[] for _ in configs]
    for c in configs:  # one untimed run each (module loading, first-touch)
        apply(c)
        if before:
            before()
        fn()
    for _ in range(reps):
        for i, c in enumerate(configs):
            apply(c)
            if before:
                before()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            samples[i].append(e0.elapsed_time(e1))
    times = [statistics.median(t) for t in samples]
    best = min(range(len(configs)), key=lambda i: times[i])
    if times[best] > (1.0 - margin) * times[0]:
        best = 0
    apply(configs[best])
    label = lambda c: ",".join("%s=%d" % kv for kv in c.items())
    return {"knob": name, "best": configs[best], "ms": {label(c): round(t, 4) for c, t in zip(configs, times)},
            "best_ms": times[best]}


def tune_knob(knob: str, fn: Callable[[], None], candidates: Iterable[int] = None, reps: int = 7,
              before: Callable[[], None] = None, margin: float = 0.03) -> Dict[str, object]:
    """Time ``fn`` under each candidate value of ``knob`` and set the fastest;
    the value the knob held before is the incumbent (see ``tune_configs``)."""
    cands = tuple(CANDIDATES[knob] if candidates is None else candidates)
    incumbent = _lib.tune_get(knob)
    order = (incumbent,) + tuple(v for v in cands if v != incumbent)
    r = tune_configs(knob, [{knob: v} for v in order], fn, reps=reps, before=before, margin=margin)
    return {"knob": knob, "best": r["best"][knob], "ms": {str(v): r["ms"]["%s=%d" % (knob, v)] for v in order},
            "best_ms": r["best_ms"]}


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
    rec.append(tk("march_coarse", march))
    if hp.sat_ok:  # the box walk (summed-area table) against the walks above
        # the table is rebuilt at every grid update, once per step: charge that to the box walk
        build = hp.sat_rebuild_call()
        times = {}
        for use in (True, False):
            hp.use_sat = use
            times[int(use)] = time_ms((lambda: (march(), build())) if use else march, reps=reps, before=flush)
        hp.use_sat = times[1] <= times[0]
        rec.append({"knob": "march_sat", "best": int(hp.use_sat), "ms": {str(k): round(v, 4) for k, v in times.items()},
                    "note": "1: march plus the table's rebuild; 0: march"})
        if hp.use_sat:
            rec.append(tk("march_box_tile", march))
            rec.append(tk("march_tile_rays", march))  # the box walks favour other tile sizes
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
    rec.append(tk("render_fwd_stages", fwd))
    hp.render_fwd(S)
    hp.g_color.uniform_(-1e-6, 1e-6)
    rec.append(tk("render_bwd_occupancy", lambda: hp.render_bwd(S)))
    rec.append(tk("render_bwd_prefetch", lambda: hp.render_bwd(S)))
    # the staged backward reads the optical depth the forward saved
    saved0 = hp.save_optical_depth
    hp.save_optical_depth = True
    hp.render_fwd(S)
    rec.append(tk("render_bwd_stages", lambda: hp.render_bwd(S)))
    hp.save_optical_depth = saved0
    # forward + loss gradient + backward in one call (the fused alternative)
    if bt.get("tgt") is not None:
        rec.append(tk("render_mse_occupancy", lambda: hp.render_mse(S, bt["tgt"])))
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
