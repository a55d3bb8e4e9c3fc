"""Kernel and launch-shape selection (autotuning) for one lattice and for
ensembles.

The paper tunes two knobs by hand -- the virtual vector length VVL (sites
per thread) and the threads per block TPB (targetDP Sec. III.C and Sec. IV:
VVL = 8 on the CPU, VVL = 2 on the K40).  Here the tuner chooses, for one
lattice, among the step kernels themselves and their launch shapes:

* ``two_pass``: threads per CTA of both passes and sites per thread of the
  phi pass (the VVL axis), ``("two_pass", tpb, vvl, 0)``;
* ``bulk``: shared-memory plane slots of g, CTAs per y-cluster and planes per
  CTA of the bulk-copy single pass, ``("bulk", slots, cluster, z_chunk)``;
* ``fused``: CTA tile and z run of the shared-memory fused kernel;
* ``taug1``: the tau_g = 1 reduced form, only when tau_g = 1 and asked for
  (it keeps a different state, so it is a separate family): y rows per warp,
  warps per CTA and z run of its phi pass, ``("taug1", rows, warps, z_run)``.

``autotune`` times every candidate on the GPU through the C ABI and keeps the
fastest in an on-disk cache keyed by GPU name, lattice extents, precision
and family set; ``bench_config`` returns the cached choice (or the library
default), ``ensure_tuned`` tunes on first use.  ``autotune_batch`` does the
same for an ensemble's (threads, CTAs per SM, CTA plan).
"""
from __future__ import annotations

import json
import os
import time

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

# (kernel, block_x, block_y, z_chunk); 0 = library default
DEFAULT = ("auto", 0, 0, 0)
# kernels of the general step (any tau_g), the families the benchmark's
# headline is tuned over
GENERAL = ("two_pass", "bulk", "fused")


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "none"


def _key(dims, precision, families=GENERAL) -> str:
    return f"{_gpu_name()}|{dims[0]}x{dims[1]}x{dims[2]}|{precision}|{'+'.join(families)}|v4"


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(key, entry):
    db = _load()
    db[key] = entry
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1)
    os.replace(tmp, CACHE)


def bench_config(dims, precision, families=GENERAL):
    """Launch configuration cached for lattice ``dims`` in ``precision``
    over ``families``, else the library default."""
    hit = _load().get(_key(dims, precision, families))
    return tuple(hit["config"]) if hit else DEFAULT


def cached_table(dims, precision, families=GENERAL):
    """The timed table behind a cached choice (None if not tuned)."""
    return _load().get(_key(dims, precision, families))


def _bulk_ok(dims, precision):
    es = 8 if precision == "fp64" else 4
    return precision in ("fp64", "fp32_shifted") and dims[0] <= 256 and (dims[0] * es) % 16 == 0


def candidates(precision, dims=None, families=GENERAL, tau_g=None):
    """Configurations to time for ``dims`` in ``precision``."""
    out = []
    if "two_pass" in families:
        for tpb in (128, 256):
            for vvl in (1, 2, 4):
                out.append(("two_pass", tpb, vvl, 0))
    if "bulk" in families and (dims is None or _bulk_ok(dims, precision)):
        slots = (3, 4) if precision == "fp64" else (2, 3, 4)
        for ng in slots:
            for cy in (1, 2, 4, 8):
                if dims is not None and (dims[1] % cy or cy > dims[1]):
                    continue
                # planes per CTA: also 20 and 24, whose CTA counts fill the
                # last wave better at 256^3 (measured: 20 is 0.7 % faster
                # than 16 there)
                for zc in (16, 20, 24, 32, 64):
                    out.append(("bulk", ng, cy, zc))
    if "fused" in families and precision != "fp64_df":
        for bx, by, zc in ((32, 4, 32), (64, 2, 32), (32, 8, 64), (64, 4, 16)):
            out.append(("fused", bx, by, zc))
    if "taug1" in families and tau_g == 1.0:
        # the phi pass's y rows per warp, warps per CTA and z run
        for ky in (1, 2) if precision == "fp64_df" else (1, 2, 4):
            for warps in (4, 8):
                for zc in (0, 32, 64):
                    out.append(("taug1", ky, warps, zc))
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
    lat.sync()
    return s.elapsed_time(e) / 1e3 / steps


def autotune(dims, precision, params, phi0, configs=None, families=GENERAL, steps=5, save=True, log=None):
    """Time every candidate on ``dims``; returns (best_config, table).  The
    table's rows are (config, seconds per step); configurations the library
    refuses for this lattice are skipped."""
    from .lattice import Lattice
    configs = configs or candidates(precision, dims, families, params.get("tau_g"))
    table = []
    with Lattice.from_params(dims, params, precision=precision) as lat:
        lat.init(phi0)
        for cfg in configs:
            try:
                t = time_config(lat, cfg, steps=steps)
            except Exception as exc:  # a shape this lattice or build refuses
                if log:
                    log(f"skip {cfg}: {exc}")
                continue
            table.append((tuple(cfg), t))
            if log:
                log(f"{cfg} {t * 1e3:.3f} ms")
    best = min(table, key=lambda r: r[1])
    if save:
        _save(_key(dims, precision, families),
              {"config": list(best[0]), "seconds_per_step": best[1], "steps": steps,
               "table": [[list(c), t] for c, t in table], "when": time.strftime("%Y-%m-%dT%H:%M:%S")})
    return best[0], table


def ensure_tuned(dims, precision, params, phi0, families=GENERAL, log=None):
    """The cached choice for ``dims``/``precision``/``families``, tuning on
    first use (the cache lives beside the built library)."""
    hit = _load().get(_key(dims, precision, families))
    if hit:
        return tuple(hit["config"])
    best, _ = autotune(dims, precision, params, phi0, families=families, log=log)
    return tuple(best)


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
