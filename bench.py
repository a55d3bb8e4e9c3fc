"""Benchmark of the binary-fluid D3Q19 lattice Boltzmann step on GB300.

A "step" is one timestep of the whole path (phi, 7-point stencil, fused f/g
collision, pull streaming) over a 256^3 periodic lattice, FP32-shifted
storage -- the fused-step-at-256^3 workload.  The same line also carries the
FP64 form's MLUPS on the same lattice, the per-field error of both forms
against the CPU oracle on a small sample, the roofline of the dominant
kernel, an end-to-end number through the C ABI with host buffers, and the
CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the lattice
(the step has no cross-lattice exchange): weak scaling, max time over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lb_inputs as LI  # noqa: E402

DIMS = (256, 256, 256)
BYTES_PER_SITE = {"fp32_shifted": 4 * 19 * 4, "fp64": 4 * 19 * 8}   # read+write f and g once
# tau_g = 1 reduced form: collide reads f (19) + phi, writes f (19) + (gmh, u) (4);
# the phi pass reads phi + (gmh, u) and writes phi -- 49 words per site
BYTES_PER_SITE_TAUG1 = {"fp32_shifted": 49 * 4, "fp64": 49 * 8}
METRIC = "MLUPS and % of HBM roofline (fused step), FP32-shifted vs FP64 at stated error"
ORACLE_SAMPLE = (64, 64, 64)
ORACLE_STEPS = 30
E2E_STEPS = 50
MRT_RATES = (1.3, 0.6)      # tau_bulk, tau_ghost of the MRT measurement
MASK_DENSITY = 0.1          # fraction of sites selected in the masked-moments measurement
FALLBACK_HBM = 6800.0
# kernels one timestep launches, per lb_set_kernel choice
STEP_KERNELS = {"auto": "timestep = k_phi_pull + k_collide_pull (two launches)",
                "two_pass": "timestep = k_phi_pull + k_collide_pull (two launches)",
                "fused": "k_fused", "staged": "k_staged", "slab": "k_slab", "lag": "k_lag", "bulk": "k_bulk",
                "taug1": "timestep = k_t1_collide + k_t1_phi (two launches)"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v, ws, device="cuda"):
    """The maximum of v over the ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM, "fallback"


# sources the default timestep's kernels are compiled from
TIMING_NOTE = ("launch duration = the timed region's steps run back to back, CUDA events around them, "
               "divided by their number; frac_single_launches: single steps each between two events")
STEP_SOURCES = ("d3q19.cuh", "lb_site.cuh", "lb_coll.cuh", "lb_pdl.cuh", "lb_kernels.cu")


def _kernel_sha(sources=STEP_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1405_6162_gb300", "csrc")
    for name in sources:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def _profile_value(name, key, need_current=True):
    """A number recorded in a committed ncu summary (profiles/<name>.md, a
    line "key: value"); None if absent or, when ``need_current``, if the
    summary was taken on other kernel sources than the current ones (the
    summary's "(sources: ...)" line, else the default timestep's)."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", txt)
    m_src = re.search(r"\(sources:\s*([^)]*)\)", txt)
    sources = tuple(x.strip() for x in m_src.group(1).split(",")) if m_src else STEP_SOURCES
    m_v = re.search(rf"^{re.escape(key)}:\s*([0-9.eE+-]+)", txt, re.M)
    if not m_v or (need_current and (not m_sha or m_sha.group(1) != _kernel_sha(sources))):
        return None
    return float(m_v.group(1))


class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml):
    SM clock, its maximum and the active clock-event reasons.  Nothing is
    set."""
    SM = 1                                                     # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index):
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        got = False
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            got = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) == 0
        except Exception:
            got = False
        if not got and self.lib.nvmlDeviceGetHandleByIndex_v2(device_index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.v = ctypes.c_uint()
        self.r = ctypes.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(self.v))
        self.max_mhz = float(self.v.value)

    def sample(self):
        self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, ctypes.byref(self.v))
        mhz = float(self.v.value)
        self.reasons_fn(self.h, ctypes.byref(self.r))
        return mhz, self.max_mhz, [name for bit, name in self.REASONS.items() if self.r.value & bit]


class Clocks:
    """SM clocks and throttle reasons sampled during a timed region: NVML
    back to back from a thread (~1 ms a sample; nvidia-smi at 100 ms as a
    fallback)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.rows = []
        self.src = None

    def __enter__(self):
        import threading
        try:
            nv = _Nvml(self.dev)
            self.stop = threading.Event()

            def run():
                while not self.stop.is_set():
                    self.rows.append(nv.sample())
                self.rows.append(nv.sample())

            self.rows.append(nv.sample())
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            self.src = "nvml"
            return self
        except (OSError, AttributeError):
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.src = "nvidia-smi"
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.src == "nvml":
            self.stop.set()
            self.thread.join(timeout=5)
        elif self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out = ""
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in (out or "").strip().splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    self.rows.append((float(parts[0]), float(parts[1]),
                                      [names[k] for k, v in enumerate(parts[3:7]) if v.lower() == "active"]))
                except ValueError:
                    continue
        return False

    def summary(self):
        if not self.src:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"]}
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "source": self.src}
        reasons = sorted({r for _, _, rs in self.rows for r in rs})
        sm = sorted(r[0] for r in self.rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_min_mhz": sm[0], "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": reasons, "samples": len(self.rows), "source": self.src}


def _time_steps(lat, steps, torch):
    """Per-launch CUDA-event times (s) of ``steps`` single-step launches."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s, e in ev:
        s.record()
        lat.step(1)
        e.record()
    torch.cuda.synchronize()
    return [s.elapsed_time(e) / 1e3 for s, e in ev]


def _fp64_peak(torch, reps=5):
    """FP64 FMA throughput (TFLOP/s) of this GPU, measured now: the best of
    ``reps`` timed launches of liblb's FMA-only probe kernel (8 CTAs of 256
    threads per SM, 16 independent chains per thread)."""
    from paper_1405_6162_gb300 import _lib as LL
    lib = LL.lib()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 8 * sms
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    fl = ctypes.c_double()
    best = 0.0
    for it in range(reps + 2):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        LL.check(lib.lb_probe_fp64_fma(blocks, 4096, sink.data_ptr(), ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.byref(fl)), "lb_probe_fp64_fma")
        e.record(stream)
        e.synchronize()
        if it >= 2:                                   # two warm-up launches
            best = max(best, fl.value / (s.elapsed_time(e) / 1e3) / 1e12)
    return {"tflops": best, "blocks": blocks, "threads": 256, "fmas_per_thread": 16 * 4096,
            "how": "lb_probe_fp64_fma (FMA-only kernel), CUDA events, best of %d launches" % reps}


def _oracle_errors(torch, params):
    """Per-field error of both GPU forms against the oracle on the sample,
    plus the oracle's own timing (the CPU baseline)."""
    import oracle
    from paper_1405_6162_gb300 import Lattice
    oracle.build()
    dims = ORACLE_SAMPLE
    phi0 = LI.spinodal_phi0(*dims, seed=1)
    f0, g0 = oracle.init(dims, params, phi0)
    t0 = time.perf_counter()
    f, g = oracle.step(dims, params, f0, g0, ORACLE_STEPS)
    t_or = time.perf_counter() - t0
    # the OpenMP build of the same loops (z planes over the host cores)
    t0 = time.perf_counter()
    f_omp, _ = oracle.step(dims, params, f0, g0, ORACLE_STEPS, kind="omp")
    t_omp = time.perf_counter() - t0
    assert np.array_equal(f_omp, f)       # same loops, same order per site
    want = oracle.moments(dims, f, g)
    c, _ = oracle.velocity_set()
    us = float(((np.abs(f).T @ np.abs(c).astype(float)) / f.sum(0)[:, None]).max())
    errs = {}
    for prec, kernel in (("fp64", "auto"), ("fp32_shifted", "auto"), ("fp64_df", "auto"), ("fp32_shifted", "taug1")):
        with Lattice.from_params(dims, params, precision=prec) as lat:
            lat.set_kernel(kernel)
            lat.init(phi0)
            lat.step(ORACLE_STEPS)
            got = lat.moments()
        key = prec if kernel == "auto" else f"{prec}_{kernel}"
        errs[key] = {k: float(np.abs(a - b).max() / max(np.abs(b).max(), us if k == "u" else 0.0))
                     for k, a, b in zip(("rho", "u", "phi"), got, want)}
    n = int(np.prod(dims))
    nt = oracle.threads("omp")
    base = {"value": n * ORACLE_STEPS / t_omp / 1e6, "unit": "MLUPS", "cores": nt, "kind": "oracle",
            "sample": f"{dims[0]}^3 spinodal (seed 1) x {ORACLE_STEPS} steps, FP64 C oracle, OpenMP over z "
                      f"planes on {nt} threads",
            "single_thread": {"value": n * ORACLE_STEPS / t_or / 1e6, "unit": "MLUPS", "cores": 1}}
    return errs, base


def _ensemble(torch, with_oracle=True):
    """The 64-lattice ensemble (sides U{16..64}, per-lattice tau and kappa,
    FP32-shifted), 500 steps in one graph replay of one persistent launch;
    with_oracle: the reduced form's three smallest lattices against the
    oracle after the 500 steps."""
    from paper_1405_6162_gb300 import Batch, tuning
    specs = LI.ensemble(3, 64)

    def init(b):
        for k, d in enumerate(specs):
            b[k].init(LI.spinodal_phi0(d["nx"], d["ny"], d["nz"], seed=1000 + k))

    with Batch(specs, precision="fp32_shifted") as b:
        init(b)
        cfg = tuning.batch_config(b)
        if cfg is None:
            cfg, _ = tuning.autotune_batch(b, steps=10)
            init(b)
        tuning.apply_batch_config(b, cfg)
        b.run(500)                    # captures the graph
        b.sync()
        init(b)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        b.run(500)
        e.record()
        e.synchronize()
        b.sync()
        t = s.elapsed_time(e) / 1e3
        info = b.info()
        out = {"lattices": len(specs), "sites": b.sites, "steps": 500, "seconds": t,
               "MLUPS": b.sites * 500 / t / 1e6, "precision": "fp32_shifted",
               "hbm_frac": b.sites * 500 * BYTES_PER_SITE["fp32_shifted"] / t / 1e9 / _peaks()[0],
               "launch": {"threads": info[3], "ctas": info[2], "work_items": info[1], "plan": b.plan,
                          "groups": b.groups()},
               "graph_replays": 1}
        # every lattice has tau_g = 1: the same ensemble in the reduced form
        b.set_form("taug1")
        init(b)
        cfg1 = tuning.batch_config(b)
        if cfg1 is None:
            cfg1, _ = tuning.autotune_batch(b, steps=10)
            init(b)
        tuning.apply_batch_config(b, cfg1)
        b.run(500)
        b.sync()
        init(b)
        s.record()
        b.run(500)
        e.record()
        e.synchronize()
        b.sync()
        t1 = s.elapsed_time(e) / 1e3
        info1 = b.info()
        # per-lattice error of the three smallest lattices against the oracle
        errs = []
        if with_oracle:
            import oracle
            oracle.build()
            small = sorted(range(len(specs)), key=lambda k: specs[k]["nx"] * specs[k]["ny"] * specs[k]["nz"])[:3]
            for k in small:
                d = specs[k]
                dd = (d["nx"], d["ny"], d["nz"])
                phi0k = LI.spinodal_phi0(*dd, seed=1000 + k)
                fo, go = oracle.step(dd, d, *oracle.init(dd, d, phi0k), 500, kind="omp")
                want = oracle.moments(dd, fo, go)
                got = b[k].moments()
                errs.append({"lattice": list(dd), **{nm: float(np.abs(a - w).max() / np.abs(w).max())
                                                     for nm, a, w in zip(("rho", "u", "phi"), got, want)}})
        out["taug1"] = {"seconds": t1, "MLUPS": b.sites * 500 / t1 / 1e6, "error_vs_oracle_500_steps": errs,
                        "launch": {"threads": info1[3], "ctas": info1[2], "work_items": info1[1],
                                   "plan": b.plan, "groups": b.groups()},
                        "hbm_frac": b.sites * 500 * BYTES_PER_SITE_TAUG1["fp32_shifted"] / t1 / 1e9 / _peaks()[0],
                        "what": "lb_batch_set_form(taug1): the tau_g = 1 reduced form for every lattice"}
        return out


def _reverse_steps(torch, dims, nsteps, warmup=3):
    """Seconds per reverse step (lb_adjoint_step through the C ABI, CUDA
    events around nsteps calls after warmup ones) on the FP64 lattice dims
    advanced 3 steps from a spinodal start, with seeded adjoint inputs."""
    from paper_1405_6162_gb300 import Lattice, _lib as LL
    params = dict(LI.DEFAULT_PARAMS)
    n = int(np.prod(dims))
    lib = LL.lib()
    with Lattice.from_params(dims, params, precision="fp64") as lat:
        lat.init(LI.spinodal_phi0(*dims, seed=6))
        lat.step(3)
        f, g = lat.get_state(device=True)
        cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        a_in = [cu(LI.uniform(7 + k, 19 * n, -1.0, 1.0)) for k in range(2)]
        a_out = [torch.empty(19 * n, dtype=torch.float64, device="cuda") for _ in range(2)]
        dk = torch.zeros(1, dtype=torch.float64, device="cuda")

        def call():
            rc = lib.lb_adjoint_step(lat.handle, f.data_ptr(), g.data_ptr(), a_in[0].data_ptr(), a_in[1].data_ptr(),
                                     a_out[0].data_ptr(), a_out[1].data_ptr(), dk.data_ptr())
            assert rc == 0, rc
        for _ in range(warmup):
            call()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(nsteps):
            call()
        e.record()
        e.synchronize()
        return s.elapsed_time(e) / 1e3 / nsteps


def _reduce_seconds(torch, lat, reps=10, warmup=3):
    """Median seconds of one lb_reduce call on ``lat`` (CUDA events around
    each call; a call is the per-block kernel, the final kernel, the 40-byte
    read-back and the return to the host)."""
    out = []
    for k in range(warmup + reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        lat.reduce()
        e.record()
        e.synchronize()
        if k >= warmup:
            out.append(s.elapsed_time(e) / 1e3)
    return float(np.median(out))


def _adjoint(torch):
    """Gradient of sum (phi_T - phi_target)^2 wrt phi0 and kappa, 64^3,
    T = 200, FP64, sqrt(T) checkpoints; forward-only time for reference."""
    import time as _t
    from paper_1405_6162_gb300.adjoint import trajectory
    dims, T = (64, 64, 64), 200
    params = dict(LI.DEFAULT_PARAMS)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    phi0 = cu(LI.spinodal_phi0(*dims, seed=4))
    xi = LI.interface_width(params["A"], params["kappa"])
    tgt = cu(LI.droplet_target(*dims, radius=16.0, xi=xi, seed=5))
    with torch.no_grad():
        trajectory(phi0, params["kappa"], dims, params, T)       # warm-up
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    with torch.no_grad():
        trajectory(phi0, params["kappa"], dims, params, T)
    torch.cuda.synchronize()
    t_fwd = _t.perf_counter() - t0
    def forward_backward(segment=None):
        x = phi0.clone().requires_grad_(True)
        kap = torch.tensor(params["kappa"], dtype=torch.float64, device="cuda", requires_grad=True)
        J = ((trajectory(x, kap, dims, params, T, segment) - tgt) ** 2).sum()
        J.backward()
        return kap

    def timed_fb(segment=None):
        forward_backward(segment)       # warm-up: first-call allocations of the reverse sweep
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        k = forward_backward(segment)
        torch.cuda.synchronize()
        return k, _t.perf_counter() - t0

    kap, t_all = timed_fb()
    # every state kept (one checkpoint per step, 2 x 19 N doubles each): no
    # recomputation; the difference is what sqrt(T) checkpointing costs
    kap_all, t_store = timed_fb(1)
    # dJ/dkappa against central differences of the forward alone, Richardson
    # extrapolated (J'' is large at these sizes, so plain O(h^2) differences
    # at h = 1e-5 still differ at ~1e-5)
    def phi_t(k):
        with torch.no_grad():
            return trajectory(phi0, k, dims, params, T)

    def central(h):
        # J(+) - J(-) summed site by site: J is ~2.6e5 while dJ/dkappa is O(1),
        # so differencing two rounded totals would lose ~4e-6
        pp, pm = phi_t(k0 + h), phi_t(k0 - h)
        return float(((pp - pm) * (pp + pm - 2 * tgt)).sum()) / (2 * h)

    k0 = params["kappa"]
    fd = [central(h) for h in (2e-5, 1e-5)]
    fd_rich = (4 * fd[1] - fd[0]) / 3
    g = kap.grad.item()
    # the reverse step against the FP64 pipe: flops per site from ncu counters
    # (profiles/adjoint_reverse_step_64cubed.md), time of 50 steps here
    t_rev = _reverse_steps(torch, dims, 50)
    fl = _profile_value("adjoint_reverse_step_64cubed", "fp64_flops_per_site", True)
    ins = _profile_value("adjoint_reverse_step_64cubed", "fp64_instr_per_site", True)
    pk = _fp64_peak(torch)["tflops"]
    n = int(np.prod(dims))
    rev = {"seconds_per_step": t_rev,
           "roofline": {"bound": "alu (FP64 pipe)", "kernels": "k_phi_local + k_adj_collide + k_adj_stencil + k_adj_kappa",
                        "achieved": fl * n / t_rev / 1e12 if fl else None, "peak": pk, "unit": "TFLOP/s",
                        "frac": fl * n / t_rev / 1e12 / pk if (fl and pk) else None, "flops_per_site": fl,
                        "pipe_frac": ins * n / t_rev / (pk * 1e12 / 2) if (ins and pk) else None,
                        "peak_kind": "measured in this run: FP64 FMA throughput of lb_probe_fp64_fma",
                        "note": "64^3 FP64 state (80 MB) is L2-resident; the bound is the FP64 pipe"}}
    return {"lattice": list(dims), "steps": T, "precision": "fp64", "checkpoints": "every 14 steps (~sqrt T)",
            "reverse_step": rev,
            "forward_s": t_fwd, "forward_backward_s": t_all, "ratio": t_all / t_fwd,
            "forward_backward_every_state_kept_s": t_store,
            "recompute_overhead": (t_all - t_store) / t_store,
            "same_gradient_every_state_kept": bool(kap.grad.item() == kap_all.grad.item()),
            "dJ_dkappa": g, "dJ_dkappa_fd_richardson": fd_rich, "rel_diff_vs_fd": abs(g - fd_rich) / abs(fd_rich)}


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import Lattice, tuning
    lbpkg.build()
    params = dict(LI.DEFAULT_PARAMS)
    n = int(np.prod(DIMS))
    phi0 = LI.spinodal_phi0(*DIMS, seed=1)
    peak, peak_kind = _peaks()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    fp64_peak = _fp64_peak(torch)
    # the step kernel and launch shape of each precision: the autotuner's
    # choice over the general-step kernels, tuned here on first use
    tuned = {}
    for prec in ("fp32_shifted", "fp64"):
        t0 = time.perf_counter()
        cached = tuning.cached_table(DIMS, prec) is not None
        cfg = tuning.ensure_tuned(DIMS, prec, params, phi0)
        tuned[prec] = {"config": list(cfg), "tuned_now": not cached, "seconds": time.perf_counter() - t0,
                       "table": (tuning.cached_table(DIMS, prec) or {}).get("table")}
    results = {}
    for prec in ("fp32_shifted", "fp64"):
        cfg = tuple(tuned[prec]["config"])
        with Lattice.from_params(DIMS, params, precision=prec) as lat:
            lat.set_kernel(*cfg)
            lat.init(phi0)
            lat.step(args.warmup)
            barrier()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            # clocks sampled over the timed steps and the per-launch timing
            # that follows them (a ~1 ms sampler needs the longer window)
            with Clocks(local) as clk:
                start.record()
                lat.step(args.steps)
                stop.record()
                barrier()
                # per-launch durations of the same kernel for the roofline
                per = _time_steps(lat, max(20, min(args.steps, 40)), torch)
            wall = max_over_ranks(start.elapsed_time(stop) / 1e3, ws)
            r = lat.reduce()
            t_reduce = _reduce_seconds(torch, lat)
        t_launch = float(np.mean(per))
        # the roofline's launch duration: the timed region's steps back to
        # back (CUDA events around them) over their number; t_launch, single
        # steps each bracketed by events, is reported beside it
        results[prec] = dict(cfg=cfg, wall=wall, t_step=wall / args.steps, t_launch=t_launch,
                             clocks=clk.summary(), mass=float(r[0]), t_reduce=t_reduce)

    def timed(prec, kernel, npts, mrt=None):
        """Whole-run and per-step times of `kernel` (a name or a full launch
        configuration) with the npts-point stencil (and the MRT collision with
        (tau_bulk, tau_ghost) = mrt)."""
        with Lattice.from_params(DIMS, params, precision=prec) as lat:
            lat.set_kernel(*((kernel,) if isinstance(kernel, str) else kernel))
            lat.set_stencil(npts)
            if mrt:
                lat.set_collision("mrt", *mrt)
            lat.init(phi0)
            lat.step(args.warmup)
            barrier()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            k = args.steps if prec == "fp32_shifted" else max(1, args.steps // 4)
            with Clocks(local) as clk:
                start.record()
                lat.step(k)
                stop.record()
                barrier()
            wall = max_over_ranks(start.elapsed_time(stop) / 1e3, ws)
            per = _time_steps(lat, max(5, min(k, 20)), torch)
        return dict(wall=wall, steps=k, t_step=wall / k, t_launch=float(np.mean(per)), clocks=clk.summary())

    # the tau_g = 1 reduced form on the same workload (the workload has tau_g = 1)
    # (its phi pass's launch shape tuned here on first use)
    tuned_t1 = {}
    for prec in ("fp32_shifted", "fp64"):
        t0 = time.perf_counter()
        cached = tuning.cached_table(DIMS, prec, ("taug1",)) is not None
        cfg = tuning.ensure_tuned(DIMS, prec, params, phi0, families=("taug1",))
        tuned_t1[prec] = {"config": list(cfg), "tuned_now": not cached, "seconds": time.perf_counter() - t0,
                          "table": (tuning.cached_table(DIMS, prec, ("taug1",)) or {}).get("table")}
    reduced = {prec: timed(prec, tuple(tuned_t1[prec]["config"]), 7) for prec in ("fp32_shifted", "fp64")}
    # masked moments (stream compaction) of a seeded 10 % site mask on the
    # benchmark lattice after the warm-up steps
    with Lattice.from_params(DIMS, params, precision="fp32_shifted") as lat:
        lat.init(phi0)
        lat.step(args.warmup)
        mask = torch.from_numpy((LI.uniform(77, n, 0.0, 1.0) < MASK_DENSITY).astype(np.uint8)).cuda()
        k_sel = lat.count_masked(mask)
        outs = [torch.empty(m * k_sel, dtype=torch.float64, device="cuda") for m in (1, 3, 1)]
        from paper_1405_6162_gb300 import _lib as LL
        lib = LL.lib()
        cnt = ctypes.c_longlong(0)

        def masked_call():
            rc = lib.lb_moments_masked(lat.handle, mask.data_ptr(), outs[0].data_ptr(), outs[1].data_ptr(),
                                       outs[2].data_ptr(), ctypes.byref(cnt), LL.LB_DEVICE)
            assert rc == 0
        for _ in range(3):
            masked_call()
        barrier()
        reps = 20
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(reps):
            masked_call()
        ev1.record()
        ev1.synchronize()
        t_mask = ev0.elapsed_time(ev1) / 1e3 / reps
    masked = {"density": MASK_DENSITY, "selected": k_sel, "ms_per_call": t_mask * 1e3,
              "selected_sites_per_s": k_sel / t_mask,
              # mask read twice (count, gather) + per selected site: 19 f + 19 g pulled (float) + 5 doubles out
              "algorithmic_bytes": 2 * n + k_sel * (38 * 4 + 5 * 8)}
    masked["achieved_gbs"] = masked["algorithmic_bytes"] / t_mask / 1e9
    masked["hbm_frac"] = masked["achieved_gbs"] / peak

    # the 128^3 lattice of the 1000-step spinodal workload, both precisions
    l128 = {}
    for prec, k in (("fp32_shifted", 400), ("fp64", 50)):
        d128 = (128, 128, 128)
        with Lattice.from_params(d128, params, precision=prec) as lat:
            lat.init(LI.spinodal_phi0(*d128, seed=1))
            lat.step(args.warmup)
            barrier()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record()
            lat.step(k)
            stop.record()
            barrier()
            w = max_over_ranks(start.elapsed_time(stop) / 1e3, ws)
        l128[prec] = {"MLUPS": ws * 128 ** 3 * k / w / 1e6, "steps": k,
                      "l2": "state 0.6 / 1.3 GB, larger than L2"}

    # double-float (FP64-class accuracy on the FP32 units) on the default step
    df = timed("fp64_df", "auto", 7)

    # the MRT collision of f on the default step
    mrt = {prec: timed(prec, "auto", 7, MRT_RATES) for prec in ("fp32_shifted", "fp64")}
    # the isotropic stencils on the default step
    stencils = {(npts, prec): timed(prec, "auto", npts) for npts in (19, 27) for prec in ("fp32_shifted", "fp64")}

    # end to end through the C ABI with host buffers (pinned), copies timed
    prec = "fp32_shifted"
    phi_host = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    phi_host[:] = phi0
    out_host = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    e2e_iters = 6
    with Lattice.from_params(DIMS, params, precision=prec) as lat:
        lat.set_kernel(*tuned[prec]["config"])
        lbl = lat.handle
        from paper_1405_6162_gb300 import _lib as LL
        lib = LL.lib()
        # one untimed round (the first host read-back allocates its staging buffer)
        lat.init(phi_host)
        lat.step(2)
        assert lib.lb_moments(lbl, None, None, out_host.ctypes.data, 0) == 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_iters):
            lat.init(phi_host)                       # H2D of the inputs
            lat.step(E2E_STEPS)
            rc = lib.lb_moments(lbl, None, None, out_host.ctypes.data, 0)   # D2H of the result
            assert rc == 0
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": ws * n * E2E_STEPS * e2e_iters / t_e2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": n * 8 / E2E_STEPS, "d2h_bytes_per_step": n * 8 / E2E_STEPS,
           "steps_per_transfer": E2E_STEPS}

    ens = _ensemble(torch, with_oracle=(rank == 0 and ws == 1))
    adj = _adjoint(torch)
    if rank != 0:
        return
    errs, cpu = (None, None)
    if ws == 1:
        errs, cpu = _oracle_errors(torch, params)

    def line_for(prec):
        r = results[prec]
        mlups = ws * n * args.steps / r["wall"] / 1e6
        kernel = STEP_KERNELS.get(r["cfg"][0], r["cfg"][0])
        # ncu summary of the kernel that ran (bulk: its own, with its sources listed)
        prof = f"step_bulk_{prec}_256cubed" if r["cfg"][0] == "bulk" else f"step_{prec}_256cubed"
        if prec == "fp32_shifted":
            achieved = BYTES_PER_SITE[prec] * n / r["t_step"] / 1e9
            roof = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": _profile_value(prof, "dram_bytes_per_step"),
                    "peak_kind": f"{peak_kind} (copy bandwidth)",
                    "algorithmic_bytes_per_launch": BYTES_PER_SITE[prec] * n,
                    "launch_seconds": r["t_step"], "timing": TIMING_NOTE,
                    "frac_single_launches": BYTES_PER_SITE[prec] * n / r["t_launch"] / 1e9 / peak}
        else:
            # FP64 is bound by the FP64 pipe: flops per site from ncu counters
            fl = _profile_value(prof, "fp64_flops_per_site")
            pk = fp64_peak["tflops"]
            achieved = fl * n / r["t_step"] / 1e12 if fl else None
            ins = _profile_value(prof, "fp64_instr_per_site")
            roof = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                    "frac": (achieved / pk) if (achieved and pk) else None,
                    # FP64 adds and multiplies occupy the pipe like an FMA: the
                    # instruction rate against the FMA-instruction peak (peak / 2)
                    "pipe_frac": (ins * n / r["t_step"] / (pk * 1e12 / 2)) if (ins and pk) else None,
                    "traffic": _profile_value(prof, "dram_bytes_per_step"),
                    "peak_kind": "measured in this run: FP64 FMA throughput of lb_probe_fp64_fma",
                    "peak_probe": fp64_peak,
                    "hbm_frac": BYTES_PER_SITE[prec] * n / r["t_step"] / 1e9 / peak}
        return mlups, roof

    def reduced_for(prec):
        r = reduced[prec]
        bpl = BYTES_PER_SITE_TAUG1[prec] * n
        achieved = bpl / r["t_step"] / 1e9
        return {"value": ws * n * r["steps"] / r["wall"] / 1e6, "unit": "MLUPS", "steps": r["steps"],
                "ms_per_step": r["wall"] / r["steps"] * 1e3, "clocks": r["clocks"],
                "roofline": {"bound": "hbm" if prec == "fp32_shifted" else "alu (FP64 pipe)",
                             "kernel": STEP_KERNELS["taug1"], "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak,
                             "traffic": _profile_value("step_taug1_256cubed", f"dram_bytes_per_step_{prec}"),
                             "peak_kind": f"{peak_kind} (copy bandwidth)",
                             "algorithmic_bytes_per_launch": bpl, "launch_seconds": r["t_step"],
                             "timing": TIMING_NOTE, "frac_single_launches": bpl / r["t_launch"] / 1e9 / peak},
                "launch": tuned_t1[prec]["config"], "tuned_now": tuned_t1[prec]["tuned_now"],
                "tuning_seconds": tuned_t1[prec]["seconds"],
                "tuning_table": tuned_t1[prec]["table"]}

    def stencil_for(npts, prec):
        r = stencils[(npts, prec)]
        achieved = BYTES_PER_SITE[prec] * n / r["t_step"] / 1e9
        out = {"value": ws * n * r["steps"] / r["wall"] / 1e6, "unit": "MLUPS", "steps": r["steps"],
               "ms_per_step": r["wall"] / r["steps"] * 1e3, "clocks": r["clocks"],
               "hbm_frac": achieved / peak, "achieved_gbs": achieved}
        if prec == "fp64":
            fl = _profile_value("step_isotropic_stencils_256cubed", f"fp64_flops_per_site_{npts}")
            pk = fp64_peak["tflops"]
            if fl and pk:
                out["alu"] = {"achieved_tflops": fl * n / r["t_step"] / 1e12, "peak_tflops": pk,
                              "frac": fl * n / r["t_step"] / 1e12 / pk, "flops_per_site": fl}
        return out

    def mrt_for(prec):
        r = mrt[prec]
        achieved = BYTES_PER_SITE[prec] * n / r["t_step"] / 1e9
        out = {"value": ws * n * r["steps"] / r["wall"] / 1e6, "unit": "MLUPS", "steps": r["steps"],
               "ms_per_step": r["wall"] / r["steps"] * 1e3, "clocks": r["clocks"],
               "hbm_frac": achieved / peak, "achieved_gbs": achieved}
        if prec == "fp64":
            fl = _profile_value("step_mrt_256cubed", "fp64_flops_per_site")
            pk = fp64_peak["tflops"]
            if fl and pk:
                out["alu"] = {"achieved_tflops": fl * n / r["t_step"] / 1e12, "peak_tflops": pk,
                              "frac": fl * n / r["t_step"] / 1e12 / pk, "flops_per_site": fl}
        return out

    def reduce_for(prec):
        # lb_reduce is bound by the FP64 pipe: FP64 additions per site from
        # ncu counters against the measured FP64 FMA-instruction rate (the
        # probe's TFLOP/s over 2); the HBM fraction of its 38 stored words
        # a site is given beside it
        t = results[prec]["t_reduce"]
        adds = _profile_value("reduce_128cubed", f"fp64_adds_per_site_{prec}")
        pk = fp64_peak["tflops"]
        gbs = 38 * (4 if prec == "fp32_shifted" else 8) * n / t / 1e9
        ach = adds * n / t / 1e12 if adds else None
        tr = _profile_value("reduce_128cubed", f"dram_bytes_per_site_{prec}")
        return {"ms_per_call": t * 1e3, "sites_per_s": n / t,
                "roofline": {"bound": "alu (FP64 pipe)", "kernel": "k_reduce_partial", "achieved": ach,
                             "peak": pk / 2 if pk else None, "unit": "T FP64 instructions/s",
                             "frac": ach / (pk / 2) if (ach and pk) else None, "fp64_adds_per_site": adds,
                             "peak_kind": "measured in this run: FMA instructions/s of lb_probe_fp64_fma",
                             "achieved_gbs": gbs, "hbm_frac": gbs / peak,
                             "traffic": tr * n if tr else None,
                             "timing": "median of 10 calls, CUDA events around each (both kernels, the "
                                       "40-byte read-back and the return)"}}

    def df_line():
        r = df
        achieved = BYTES_PER_SITE["fp64"] * n / r["t_step"] / 1e9
        return {"value": ws * n * r["steps"] / r["wall"] / 1e6, "unit": "MLUPS", "steps": r["steps"],
                "ms_per_step": r["wall"] / r["steps"] * 1e3, "clocks": r["clocks"],
                "speedup_vs_fp64": (r["steps"] / r["wall"]) / (args.steps / results["fp64"]["wall"]),
                "roofline": {"bound": "alu (FP32 pipe) / hbm", "kernel": STEP_KERNELS["two_pass"],
                             "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "traffic": _profile_value("step_fp64_df_256cubed", "dram_bytes_per_step"),
                             "peak_kind": f"{peak_kind} (copy bandwidth)",
                             "algorithmic_bytes_per_launch": BYTES_PER_SITE["fp64"] * n}}

    v32, roof32 = line_for("fp32_shifted")
    v64, roof64 = line_for("fp64")
    r32 = results["fp32_shifted"]
    out = {
        "metric": METRIC, "value": v32, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["wall"] / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "256^3 periodic D3Q19 binary fluid, spinodal phi0 ~ U[-0.01,0.01] seed 1, "
                               "tau=1, tau_g=1, rho0=1, Gamma=0.5, A=-0.0625, B=0.0625, kappa=0.04; "
                               "FP32-shifted fused step",
                   "lattice": list(DIMS), "precision": "fp32_shifted",
                   "launch": list(r32["cfg"]),
                   "l2": "inputs larger than L2 (5.1 GB state vs 129 MB L2): no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roof32,
        "fp64": {"value": v64, "unit": "MLUPS", "ms_per_step": results["fp64"]["wall"] / args.steps * 1e3,
                 "roofline": roof64, "launch": list(results["fp64"]["cfg"]),
                 "clocks": results["fp64"]["clocks"]},
        "error_vs_oracle": ({"sample": f"{ORACLE_SAMPLE[0]}^3 spinodal seed 1, {ORACLE_STEPS} steps, "
                                       "max|gpu-oracle| / max|oracle| per field (u: / max sum_i|f_i c_i|/rho)", **errs} if errs else None),
        "clocks": r32["clocks"],
        "taug1": {"what": "tau_g = 1 reduced form (LB_KERNEL_TAUG1): g kept as phi and (gmh, u), "
                          "same results as the general step to rounding; valid only at tau_g = 1",
                  "fp32_shifted": reduced_for("fp32_shifted"), "fp64": reduced_for("fp64")},
        "fp64_df": {"what": "double-float precision (LB_FP64_DF): every value an unevaluated sum of two floats "
                            "(~48 bits), arithmetic on the FP32 units; errors in error_vs_oracle.fp64_df",
                    **df_line()},
        "lattice_128": {"what": "the 128^3 spinodal lattice (seed 1), default step", **l128},
        "mrt": {"what": f"multiple-relaxation-time collision of f (lb_set_collision), tau = 1, "
                        f"tau_bulk = {MRT_RATES[0]}, tau_ghost = {MRT_RATES[1]}, on the default two-pass step",
                "fp32_shifted": mrt_for("fp32_shifted"), "fp64": mrt_for("fp64")},
        "reductions": {"what": "lb_reduce: FP64 totals of rho, rho u and phi over the 256^3 lattice of each "
                               "precision after the timed steps",
                       "fp32_shifted": reduce_for("fp32_shifted"), "fp64": reduce_for("fp64")},
        "masked_moments": {"what": "lb_moments_masked (stream compaction: count, scan, gather) of a seeded "
                                   "random site mask on the 256^3 FP32 lattice, device outputs, one call "
                                   "includes the read-back of the count",
                           **masked},
        "stencils": {"what": "isotropic 19- / 27-point phi stencils (lb_set_stencil) on the default "
                             "two-pass step; hbm_frac over the same 76-word algorithmic bytes",
                     **{f"{npts}pt": {prec: stencil_for(npts, prec) for prec in ("fp32_shifted", "fp64")}
                        for npts in (19, 27)}},
        "autotune": {"what": "kernel and launch shape of the headline (fp32_shifted) and of the fp64 line, "
                             "chosen by tuning.autotune over the general-step kernels (two_pass: threads per CTA, "
                             "phi sites per thread; bulk: g slots, CTAs per y-cluster, planes per CTA; fused: "
                             "tile and z run); table rows are [config, seconds per step]",
                     **tuned},
        "ensemble": ens,
        "adjoint": adj,
        "e2e": e2e,
        "gpu_launches": args.steps * (2 if r32["cfg"][0] in ("auto", "two_pass", "taug1") else 1),
        "cpu_baseline": cpu,
    }
    print(json.dumps(out))


def run_reference(args):
    """The CPU oracle timed as the reference arm, on a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    params = dict(LI.DEFAULT_PARAMS)
    dims = ORACLE_SAMPLE
    f, g = oracle.init(dims, params, LI.spinodal_phi0(*dims, seed=1))
    f, g = oracle.step(dims, params, f, g, args.warmup, kind="omp")
    t0 = time.perf_counter()
    f, g = oracle.step(dims, params, f, g, args.steps, kind="omp")   # the K steps in one call
    t = time.perf_counter() - t0
    n = int(np.prod(dims))
    v = n * args.steps / t / 1e6
    nt = oracle.threads("omp")
    sample = (f"{dims[0]}^3 spinodal (seed 1), the timed steps in one oracle call, FP64 C oracle, OpenMP over z "
              f"planes on {nt} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "256^3 periodic D3Q19 binary fluid (oracle timed on a 64^3 sample)",
                   "lattice": list(dims), "precision": "fp64"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": nt, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ensemble_only(args):
    """The 64-lattice ensemble, ``--steps`` steps in one launch in each form
    (a profiling case)."""
    import torch
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import Batch
    lbpkg.build()
    specs = LI.ensemble(3, 64)
    with Batch(specs, precision="fp32_shifted") as b:
        b.set_launch(128, 0)
        for form in ("general", "taug1"):
            b.set_form(form)
            for k, d in enumerate(specs):
                b[k].init(LI.spinodal_phi0(d["nx"], d["ny"], d["nz"], seed=1000 + k))
            b.run(args.steps)
            b.sync()
        torch.cuda.synchronize()
        print(json.dumps({"only": "ensemble", "lattices": len(specs), "sites": b.sites, "steps": args.steps}))


def run_adjoint_only(args):
    """``--steps`` reverse steps (lb_adjoint_step) of the --lattice FP64
    lattice after 3 warm-up calls (a profiling case)."""
    import torch
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    dims = tuple(args.lattice) * 3 if len(args.lattice) == 1 else tuple(args.lattice)
    t = _reverse_steps(torch, dims, args.steps)
    print(json.dumps({"only": "adjoint", "lattice": list(dims), "steps": args.steps, "seconds_per_step": t}))


def run_reduce_only(args):
    """``--steps`` lb_reduce calls on the --lattice lattice of --precision
    after a spinodal start and --warmup timesteps (a profiling case)."""
    import torch
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import Lattice
    lbpkg.build()
    dims = tuple(args.lattice) * 3 if len(args.lattice) == 1 else tuple(args.lattice)
    with Lattice.from_params(dims, dict(LI.DEFAULT_PARAMS), precision=args.precision) as lat:
        lat.init(LI.spinodal_phi0(*dims, seed=1))
        lat.step(args.warmup)
        t = _reduce_seconds(torch, lat, reps=args.steps)
        tot = lat.reduce()
    print(json.dumps({"only": "reduce", "lattice": list(dims), "precision": args.precision, "calls": args.steps,
                      "seconds_per_call": t, "totals": [float(x) for x in tot]}))


def run_fp64_peak_only(args):
    """The FP64 FMA-throughput probe alone (the FP64 roofline's peak)."""
    import torch
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    torch.cuda.set_device(_dist()[2])
    print(json.dumps({"only": "fp64-peak", **_fp64_peak(torch, reps=max(3, args.steps))}))


def run_step_only(args):
    """Just ``--steps`` timesteps of one lattice (a small case for profilers)."""
    import torch
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import Lattice, tuning
    lbpkg.build()
    dims = tuple(args.lattice) * 3 if len(args.lattice) == 1 else tuple(args.lattice)
    params = dict(LI.DEFAULT_PARAMS)
    cfg = tuning.bench_config(dims, args.precision)
    if args.kernel:
        cfg = (args.kernel, *args.block)
    with Lattice.from_params(dims, params, precision=args.precision) as lat:
        lat.set_kernel(*cfg)
        lat.set_stencil(args.stencil)
        if args.mrt:
            lat.set_collision("mrt", *args.mrt)
        lat.init(LI.spinodal_phi0(*dims, seed=1))
        lat.step(args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(args.steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if args.masked is not None:
            n = math.prod(dims)
            mask = torch.from_numpy((LI.uniform(77, n, 0.0, 1.0) < args.masked).astype(np.uint8)).cuda()
            for _ in range(3):
                lat.moments_masked(mask)
            torch.cuda.synchronize()
    print(json.dumps({"only": "step", "lattice": list(dims), "precision": args.precision, "launch": list(cfg),
                      "stencil": args.stencil,
                      "steps": args.steps, "MLUPS": math.prod(dims) * args.steps / dt / 1e6}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--only", choices=["step", "ensemble", "fp64-peak", "adjoint", "reduce"], default=None,
                    help="run only timesteps of one lattice, or of the 64-lattice ensemble in both forms "
                         "(profiling cases), the FP64 FMA-throughput probe, reverse steps of the adjoint, "
                         "or lattice totals (lb_reduce) of one lattice")
    ap.add_argument("--lattice", type=int, nargs="+", default=[128],
                    help="edge of the --only lattice, or its three extents")
    ap.add_argument("--precision", choices=["fp32_shifted", "fp64", "fp64_df"], default="fp32_shifted")
    ap.add_argument("--kernel", choices=["two_pass", "fused", "staged", "slab", "lag", "taug1", "bulk"], default=None,
                    help="override the tuned launch of the --only lattice")
    ap.add_argument("--block", type=int, nargs=3, default=(0, 0, 0), metavar=("BX", "BY", "ZC"))
    ap.add_argument("--stencil", type=int, choices=[7, 19, 27], default=7,
                    help="points of the phi stencil of the --only lattice")
    ap.add_argument("--mrt", type=float, nargs=2, default=None, metavar=("TAU_BULK", "TAU_GHOST"),
                    help="MRT collision of the --only lattice")
    ap.add_argument("--masked", type=float, default=None, metavar="DENSITY",
                    help="after the steps, three masked-moment copies of a random mask of this density")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only == "ensemble":
        return run_ensemble_only(args)
    if args.only == "adjoint":
        return run_adjoint_only(args)
    if args.only == "fp64-peak":
        return run_fp64_peak_only(args)
    if args.only == "reduce":
        return run_reduce_only(args)
    if args.only == "step":
        run_step_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
