"""Launch-shape selection for the fused step kernel.

The paper tunes two knobs by hand -- the virtual vector length VVL (sites
per thread) and the threads per block TPB (targetDP Sec. III.C and Sec. IV:
VVL = 8 on the CPU, VVL = 2 on the K40).  Here the knobs of the fused kernel
are the CTA tile (block_x x block_y sites of an x-y plane) and the number of
z planes a CTA marches (z_chunk).  ``autotune`` times candidate shapes on the
GPU through the C ABI and keeps the fastest in an on-disk cache keyed by GPU
name, lattice extents and precision; ``bench_config`` returns the cached
choice, or the library default when nothing was tuned.
"""
from __future__ import annotations

import json
import os
import time

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

# (kernel, block_x, block_y, z_chunk); 0 = library default
DEFAULT = ("auto", 0, 0, 0)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "none"


def _key(dims, precision) -> str:
    return f"{_gpu_name()}|{dims[0]}x{dims[1]}x{dims[2]}|{precision}"


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def bench_config(dims, precision):
    """Launch configuration used for lattice ``dims`` in ``precision``."""
    hit = _load().get(_key(dims, precision))
    return tuple(hit["config"]) if hit else DEFAULT


def candidates(precision):
    maxt = 256 if precision == "fp64" else 512
    out = []
    for bx in (32, 64, 128):
        for by in (1, 2, 4, 8, 16):
            if bx * by > maxt or bx * by < 64:
                continue
            for zc in (8, 16, 32, 64):
                out.append(("fused", bx, by, zc))
    return out


def time_config(lat, config, steps=5, warmup=2):
    """Mean seconds per step of ``config`` on an initialised Lattice."""
    import torch
    lat.set_kernel(*config)
    lat.step(warmup)
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    lat.step(steps)
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / 1e3 / steps


def autotune(dims, precision, params, phi0, configs=None, steps=5, save=True, log=None):
    """Time every candidate shape on ``dims``; returns (best_config, table)."""
    from .lattice import Lattice
    configs = configs or candidates(precision)
    table = []
    with Lattice.from_params(dims, params, precision=precision) as lat:
        lat.init(phi0)
        for cfg in configs:
            try:
                t = time_config(lat, cfg, steps=steps)
            except Exception as exc:  # an invalid shape for this build
                if log:
                    log(f"skip {cfg}: {exc}")
                continue
            table.append((cfg, t))
            if log:
                log(f"{cfg} {t * 1e3:.3f} ms")
    best = min(table, key=lambda r: r[1])
    if save:
        db = _load()
        db[_key(dims, precision)] = {"config": list(best[0]), "seconds_per_step": best[1],
                                     "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as fh:
            json.dump(db, fh, indent=1)
    return best[0], table


def _batch_key(batch) -> str:
    import hashlib
    h = hashlib.sha256(repr([sorted(d.items()) for d in batch.specs]).encode()).hexdigest()[:12]
    return f"{_gpu_name()}|batch{len(batch)}:{h}|{batch.precision}|{getattr(batch, 'form', 'general')}|v3"


def batch_candidates(precision):
    """(threads per CTA, CTAs per SM, CTA plan) shapes to time."""
    threads = (128, 256)
    return [(t, c, p) for p in ("lattice", "grid", 4, 8, 16) for t in threads for c in (0, 1, 2, 3)]


def apply_batch_config(batch, config):
    """Set a (threads, ctas_per_sm, plan) launch shape on an ensemble."""
    t, c, p = config
    batch.set_plan(p)
    batch.set_launch(t, c)


def autotune_batch(batch, steps=20, candidates=None, save=True, log=None):
    """Time every (threads, ctas_per_sm, plan) launch shape of an
    initialised ensemble for ``steps`` steps, keep the fastest on the
    ensemble and in the on-disk cache; returns (best, table).  Running the
    ensemble advances its lattices: re-initialise them afterwards if their
    state matters."""
    import torch
    table = []
    seen = set()
    for t, c, p in candidates or batch_candidates(batch.precision):
        try:
            apply_batch_config(batch, (t, c, p))
        except Exception as exc:
            if log:
                log(f"skip {(t, c, p)}: {exc}")
            continue
        info = batch.info()
        if (t, info[2], p) in seen:       # same grid as a shape already timed
            continue
        seen.add((t, info[2], p))
        batch.run(steps)                   # warm-up (captures the graph)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        batch.run(steps)
        e.record()
        e.synchronize()
        dt = s.elapsed_time(e) / 1e3 / steps
        table.append(((t, c, p), dt, info[2]))
        if log:
            log(f"threads={t} ctas/SM={c} plan={p} grid={info[2]}: {dt * 1e3:.3f} ms/step")
    best = min(table, key=lambda r: r[1])
    apply_batch_config(batch, best[0])
    batch.sync()
    if save:
        db = _load()
        db[_batch_key(batch)] = {"config": list(best[0]), "seconds_per_step": best[1],
                                 "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as fh:
            json.dump(db, fh, indent=1)
    return best[0], [(r[0], r[1]) for r in table]


def batch_config(batch):
    """Cached (threads, ctas_per_sm, plan) of this ensemble, or None."""
    hit = _load().get(_batch_key(batch))
    return tuple(hit["config"]) if hit else None
