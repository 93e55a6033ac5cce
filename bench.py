"""Benchmark of the SHCI variational hot path on one GB300 (or N replicas).

A step is one pass of the whole hot path over the heat-bath-selected
workload (24 orbitals, 6 alpha + 6 beta electrons, |V| = 1,000,000 selected by
the oracle's heat-bath selection, Sec. II.A Eq. 2; two roots, stored H):
helper lists, connectivity and H_ij for every connected pair, the cached
diagonal, then diagonally preconditioned Davidson to convergence (tol 1e-10,
residual 1e-6) with sigma = H c applied from the stored matrix.

Metric: full-matrix sigma nonzeros processed per second over the whole step
(sum over sigma launches of (2 * nnz_upper + n_det) * vectors, divided by the
step time, build included).  Time-to-E -- from the Davidson call's entry until
every root is within 1e-9 Ha of the oracle's energy of the same V (stored
beside the space) -- and the build time are reported beside it, plus the
dominant kernel's roofline.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--gpus N]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import shci_synth as S  # noqa: E402

WORKLOAD = "sel_24o_6a6b_1m"
TOL = 1e-10
MAX_ITER = 400
NOMINAL_FP64_TFLOPS = 1.25     # GB300 dense FP64, nominal at the maximum SM clock


def metric_name():
    return "sigma H·c nonzeros/s and Davidson time-to-E (|ΔE|<1e-9 Ha) vs roofline, 1 GB300"


def workload_desc(cfg, n_det=None):
    n = n_det if n_det is not None else cfg.n_det
    if not cfg.n_det:
        kind = "full-CI"
    elif cfg.space == "heat-bath":
        meta = S.selected_space_meta(cfg.stored_as or cfg.name)
        kind = ("heat-bath-selected (Sec. II.A Eq. 2, eps1 from %.0e by x%.1f, selected by the CPU oracle; "
                "SHA-256 %s...)" % (meta["selection"]["eps1_start"], meta["selection"]["eps1_factor"],
                                    meta["sha256"][:16]))
    else:
        kind = "score-and-noise stand-in"
    return ("%s: %d orbitals, %da+%db electrons, |V|=%d %s determinants, %d roots, stored H, FP64"
            % (cfg.name, cfg.n_orb, cfg.n_alpha, cfg.n_beta, n, kind, cfg.roots))


def oracle_energies(cfg, n_det):
    """The CPU oracle's lowest roots of H on the full stored space (written by
    tests/golden/make_selected_spaces.py), or None."""
    if cfg.space != "heat-bath" or n_det != cfg.n_det:
        return None
    meta = S.selected_space_meta(cfg.stored_as or cfg.name)
    orc = meta.get("oracle")
    return None if orc is None else np.array(orc["energies"][:cfg.roots])


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


PEAK_KINDS = ("dfma", "dadd", "imad", "xor_popc", "atomic_add_f64_l2", "gather_8b_l2")


def measure_peaks(device=0, which=PEAK_KINDS):
    """Operations per second of the project's peak-rate microbenchmarks
    (paper_1809_04600_gb300/measure/peaks.cu) on this GPU, now: the best over
    2, 4 and 8 CTAs per SM (and 8 or 16 chains per thread for FP64)."""
    import ctypes
    from paper_1809_04600_gb300 import build_lib
    lib = ctypes.CDLL(build_lib.build_peaks())
    lib.shci_peak_rate.restype = ctypes.c_int
    lib.shci_peak_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name in which:
        w = PEAK_KINDS.index(name)
        best = 0.0
        for ctas in (2, 4, 8):
            for chains in ((8, 16) if w <= 1 else (8,)):
                rate, ms = ctypes.c_double(), ctypes.c_double()
                rc = lib.shci_peak_rate(device, w, ctas, chains, ctypes.byref(rate), ctypes.byref(ms))
                if rc != 0:
                    raise RuntimeError("peak microbenchmark %s failed with CUDA error %d" % (name, rc))
                best = max(best, rate.value)
        out[name] = best
    return out


def replica_totals(dist, seconds, units, device="cpu"):
    """Whole-job figures of N independent replicas: the slowest rank's time and
    the units all ranks processed (value = units / time).  ``dist`` is
    torch.distributed (any backend) or None for one process."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


# the stored-sigma kernel's source region in csrc/sigma.cu: its shape macros,
# k_sigma_stored and its launch (edits elsewhere in the file leave it alone)
STORED_SIGMA_REGION = ("#ifndef SHCI_SIGMA_R2", "template <bool INTER>\nstatic void dispatch_stored")


def kernel_source_digest(path, region=None):
    """First 16 hex digits of the SHA-256 of a source file, or of the text
    between two markers of it (the first marker included)."""
    import hashlib
    text = open(path, "rb").read()
    if region is not None:
        a = text.index(region[0].encode())
        b = text.index(region[1].encode(), a)
        text = text[a:b]
    return hashlib.sha256(text).hexdigest()[:16]


def sigma_traffic(workload, stored_nnz):
    """DRAM bytes per sigma launch from the committed ncu summary, scaled to this
    workload's stored nonzeros; None if the summary is missing or was taken on
    a different version of the kernel source."""
    tpath = os.path.join(ROOT, "profiles", "sigma_stored_traffic.json")
    src = os.path.join(ROOT, "paper_1809_04600_gb300", "csrc", "sigma.cu")
    if not os.path.exists(tpath):
        return None
    try:
        tj = json.load(open(tpath))
        if tj.get("kernel_source_sha256_16") != kernel_source_digest(src, STORED_SIGMA_REGION):
            return None
        return float(tj["dram_bytes_per_stored_nnz"]) * stored_nnz
    except Exception:
        return None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import paper_1809_04600_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    P.build()
    P.load_library()

    cfg = S.config(args.config)
    h, eri, ec, dets = S.make_system(cfg)
    n = dets.shape[0]
    stream = torch.cuda.current_stream()
    d_h = torch.from_numpy(h).cuda()
    d_eri = torch.from_numpy(eri).cuda()
    d_dets = torch.from_numpy(dets.view(np.int64)).cuda()
    vecs = torch.empty((cfg.roots, n), dtype=torch.float64, device="cuda")
    ctx = P.Context(local, stream)
    H = ctx.handle

    def step():
        P.shci_load_integrals(H, cfg.n_orb, ec, d_h, d_eri)
        nnz = P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, d_dets, P.SHCI_STORED)
        t0 = time.perf_counter()
        e, it, rc = P.shci_davidson(H, cfg.roots, TOL, MAX_ITER, vecs=vecs)
        t_dav = time.perf_counter() - t0
        if rc != 0:
            raise RuntimeError("Davidson did not converge")
        return nnz, e, it, t_dav

    for _ in range(args.warmup):
        step()
    peaks = measure_peaks(local, ("dfma",))
    # timed region: device-timed with CUDA events on the library's stream
    P.shci_set_timing(H, True)
    launches0 = P.shci_get_stats(H)["kernel_launches"]
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t_wall = time.perf_counter()
    dav_times, builds, iters, energies, hists = [], [], [], None, []
    for _ in range(args.steps):
        nnz, e, it, t_dav = step()
        dav_times.append(t_dav)
        th, _, ts = P.shci_davidson_history(H, cfg.roots)
        hists.append((th, ts))
        builds.append(P.shci_get_stats(H)["build_ms"] / 1e3)
        iters.append(it)
        energies = e
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    st = P.shci_get_stats(H)
    # time-to-E: the first iteration with every root within 1e-9 Ha of the
    # oracle's energies of the same V (the stored space's record); without
    # them, of a tight (tol 1e-13) solve of the same H after the timed region
    e_tight, _, _ = P.shci_davidson(H, cfg.roots, 1e-13, 4 * MAX_ITER)
    e_orc = oracle_energies(cfg, n)
    e_ref = e_orc if e_orc is not None else e_tight
    tte, it_e = [], []
    for th, ts in hists:
        ok = np.nonzero(np.max(np.abs(th - e_ref[None, :]), axis=1) < 1e-9)[0]
        tte.append(float(ts[ok[0]]) if ok.size else float("nan"))
        it_e.append(int(ok[0]) + 1 if ok.size else -1)
    launches = st["kernel_launches"] - launches0
    nnz_full = 2 * st["nnz_upper"] + n
    vec_mults = st["sigma_vectors"]             # vectors multiplied in the timed region
    sigma_ms = st["sigma_ms_total"]
    units = float(nnz_full) * vec_mults         # full-matrix nonzeros processed
    ms, units = replica_totals(dist, ms, units, device="cuda")
    value = units / (ms / 1e3)

    # roofline of the dominant kernel (stored sigma): one FP64 FMA per stored
    # nonzero per vector; bytes: 12 per stored nonzero + diag + vectors
    per_launch_ms = sigma_ms / max(1, st["sigma_launches"])
    kbar = vec_mults / max(1, st["sigma_launches"])
    flops = 2.0 * nnz_full * kbar
    bytes_alg = 12.0 * (nnz_full - n) + n * (8.0 + 16.0 * kbar)
    achieved_tf = flops / (per_launch_ms / 1e3) / 1e12
    hbm_peak, peak_kind = load_peaks()
    fp64_peak_tf = 2.0 * peaks["dfma"] / 1e12
    achieved_gbs = bytes_alg / (per_launch_ms / 1e3) / 1e9
    traffic = sigma_traffic(cfg.name, nnz_full - n)

    # end-to-end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(P, H, cfg, h, eri, ec, dets, nnz_full, args)
        # whole job: units of all replicas over the slowest replica's time
        t_e2e, u_e2e = replica_totals(dist, e2e["s_per_step"], e2e["value"] * e2e["s_per_step"], device="cuda")
        e2e["value"] = u_e2e / t_e2e
        e2e["s_per_step"] = t_e2e

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, h, eri, ec, dets, args)

    large = None
    if rank == 0 and args.large_iters > 0:
        # free the bench workload's matrix first: the 5e7 space needs its own room
        ctx.close()
        ctx = None
        torch.cuda.empty_cache()
        large = large_section(P, args)

    out = {
        "metric": metric_name(),
        "value": value,
        "unit": "nnz/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(cfg), "n_det": n, "nnz_upper": st["nnz_upper"],
                   "roots": cfg.roots, "tol": TOL, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: the stored H (%.1f GB) is rebuilt and streamed every step"
                         % (12.0 * (nnz_full - n) / 1e9)},
        "time_to_E_s": float(np.mean(tte)),
        "time_to_E_def": ("from shci_davidson entry until every root's Ritz value is within 1e-9 Ha of the CPU "
                          "oracle's energies of the same V (per-iteration history of the library)"
                          if e_orc is not None else
                          "from shci_davidson entry until every root's Ritz value is within 1e-9 Ha of a tight "
                          "(tol 1e-13) solve of the same H (per-iteration history of the library)"),
        "energies_oracle": None if e_orc is None else [float(x) for x in e_orc],
        "abs_dE_vs_oracle": None if e_orc is None else float(np.max(np.abs(np.asarray(energies) - e_orc))),
        "iters_to_E": int(np.max(it_e)),
        "davidson_s": float(np.mean(dav_times)),
        "build_s": float(np.mean(builds)),
        "davidson_iters": int(np.mean(iters)),
        "energies": [float(x) for x in energies],
        "sigma_kernel_ms": per_launch_ms,
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp64_peak_tf, "traffic": traffic,
                     "kernel": "k_sigma_stored (FP64 FMA per stored nonzero per vector)",
                     "peak_kind": "measured: independent FP64 FMAs of the project microbenchmark "
                                  "(paper_1809_04600_gb300/measure/peaks.cu) in this run, 2 flops each",
                     "nominal_peak": NOMINAL_FP64_TFLOPS, "frac_of_nominal": achieved_tf / NOMINAL_FP64_TFLOPS},
        "roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak, "peak_kind": peak_kind},
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "large": large,
    }
    if ctx is not None:
        ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def large_section(P, args):
    """The largest configuration (76 orbitals, 14a14b, |V| = 5e7, on-the-fly
    sigma, lowest root), bounded so that the default bench stays short: the
    build (count pass), sigma per product over two products, the first
    `large_iters` Davidson iterations (time per iteration), and the oracle's
    brute-force sigma on sampled rows.  The full solve is
    `bench.py --workload large --large-davidson`."""
    import torch
    import oracle
    cfg = S.config("sel_76o_14a14b_50m")
    t = time.perf_counter()
    h, eri, ec, dets = S.make_system(cfg)
    t_gen = time.perf_counter() - t
    n = dets.shape[0]
    c = P.Context(0, torch.cuda.current_stream())
    H = c.handle
    P.shci_load_integrals(H, cfg.n_orb, ec, _dev(torch, h), _dev(torch, eri))
    nnz = P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, _dev(torch, dets), P.SHCI_ON_THE_FLY)
    build_ms = P.shci_get_stats(H)["build_ms"]
    cand = P.shci_get_stats(H)["candidates"]
    x = torch.from_numpy(S.random_vectors(n, 1, 3)).cuda()
    y = torch.empty_like(x)
    P.shci_set_timing(H, True)
    for _ in range(2):
        P.shci_sigma(H, x, y)
    st = P.shci_get_stats(H)
    sig_ms = st["sigma_ms_total"] / max(1, st["sigma_launches"])
    rows = np.concatenate([[0], np.random.default_rng(7).choice(n, 3, replace=False)])
    O = oracle.System(h, eri, ec)
    err = float(np.max(np.abs(y.cpu().numpy()[:, rows] - O.sigma_rows(dets, x.cpu().numpy(), rows))))
    P.shci_set_timing(H, False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    e, it, rc = P.shci_davidson(H, 1, TOL, args.large_iters, check=False)
    torch.cuda.synchronize()
    t_dav = time.perf_counter() - t
    th, rn, ts = P.shci_davidson_history(H, 1)
    c.close()
    nnz_full = 2 * nnz + n
    return {"workload": "%s: 76 orbitals, 14a+14b electrons, 12-orbital near-degenerate band, |V|=%d "
                        "score-and-noise stand-in determinants, lowest root, on-the-fly sigma, FP64" % (cfg.name, n),
            "n_det": n, "nnz_upper": nnz, "gen_s": t_gen, "build_count_ms": build_ms,
            "candidates_per_product": cand, "sigma_ms_per_product": sig_ms,
            "full_nnz_per_s": nnz_full / (sig_ms / 1e3), "candidates_per_s": cand / (sig_ms / 1e3),
            "oracle_sampled_rows": int(rows.size), "oracle_max_abs_err": err,
            "davidson_iterations_run": int(it), "davidson_s": t_dav, "s_per_iteration": t_dav / max(1, it),
            "ritz_value_last": float(th[-1, 0]), "residual_norm_last": float(rn[-1, 0]),
            "note": "bounded: the full lowest-root solve (tol 1e-10) is bench.py --workload large --large-davidson"}


def run_e2e(P, H, cfg, h, eri, ec, dets, nnz_full, args):
    """Same metric through the C ABI with host buffers: integrals and
    determinants copied host->device, energies and Ritz vectors copied back,
    all inside the timed region."""
    import torch
    n = dets.shape[0]
    hp = torch.from_numpy(h).pin_memory()
    ep = torch.from_numpy(eri).pin_memory()
    dp = torch.from_numpy(dets.view(np.int64)).pin_memory()
    vout = torch.empty((cfg.roots, n), dtype=torch.float64).pin_memory()
    steps = max(1, min(args.steps, 3))
    P.shci_set_timing(H, False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    vecs_total = 0
    for _ in range(steps):
        s0 = P.shci_get_stats(H)["sigma_vectors"]
        P.shci_load_integrals(H, cfg.n_orb, ec, hp, ep)
        P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, dp, P.SHCI_STORED)
        e, it, rc = P.shci_davidson(H, cfg.roots, TOL, MAX_ITER, vecs=vout)
        vecs_total += P.shci_get_stats(H)["sigma_vectors"] - s0
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / steps
    h2d = h.nbytes + eri.nbytes + dets.nbytes
    d2h = 8 * cfg.roots + vout.numel() * 8
    return {"value": float(nnz_full) * (vecs_total / steps) / dt, "unit": "nnz/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "s_per_step": dt}


# ------------------------------------------------------------------ CPU oracle arm

def cpu_baseline(cfg, h, eri, ec, dets, args, n_rows=None):
    """The oracle as it stands on the host cores: sigma = H c for a bounded
    sample of rows of the same workload (each row by brute force over all of V,
    k = roots vectors).  Returns throughput in full-matrix nonzeros/s."""
    import oracle
    oracle.build()
    O = oracle.System(h, eri, ec)
    n = dets.shape[0]
    rng = np.random.default_rng(2024)
    n_rows = n_rows or args.cpu_rows
    rows = np.sort(rng.choice(n, n_rows, replace=False))
    c = S.random_vectors(n, cfg.roots, 7)
    t = time.perf_counter()
    O.sigma_rows(dets, c, rows)
    dt = time.perf_counter() - t
    nnz_rows = sum(O.row(dets, int(i))[0].size + 1 for i in rows[:min(40, n_rows)])
    nnz_per_row = nnz_rows / min(40, n_rows)
    value = nnz_per_row * n_rows * cfg.roots / dt
    return {"value": value, "unit": "nnz/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d uniformly sampled rows of the %d-determinant space, %d vectors, each row by brute force "
                      "over all determinants (%.1f s); nonzeros/row estimated from 40 rows" %
                      (n_rows, n, cfg.roots, dt), "seconds": dt}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = S.config(args.config)
    h, eri, ec, dets = S.make_system(cfg)
    for _ in range(args.warmup):
        cpu_baseline(cfg, h, eri, ec, dets, args, n_rows=max(8, args.cpu_rows // 10))
    vals, secs = [], []
    res = None
    for _ in range(args.steps):
        res = cpu_baseline(cfg, h, eri, ec, dets, args, n_rows=max(8, args.cpu_rows // 4))
        vals.append(res["value"])
        secs.append(res["seconds"])
    value = float(np.mean(vals))
    out = {
        "impl": "reference",
        "metric": metric_name(),
        "value": value,
        "unit": "nnz/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(cfg), "n_det": dets.shape[0], "roots": cfg.roots},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"]},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_sigma_only(args):
    """Profiling driver: build the stored H of the workload (or a smaller space
    of the same shape with --n-det) and launch the sigma kernel repeatedly with
    `roots` vectors.  Prints the mean kernel time; not a bench line."""
    import torch
    import paper_1809_04600_gb300 as P
    P.build()
    P.load_library()
    cfg = S.config(args.config)
    h, eri, ec, dets = S.make_system(cfg, n_det=args.n_det)
    n = dets.shape[0]
    ctx = P.Context(0, torch.cuda.current_stream())
    P.shci_load_integrals(ctx.handle, cfg.n_orb, ec, torch.from_numpy(h).cuda(), torch.from_numpy(eri).cuda())
    P.shci_build_connectivity(ctx.handle, cfg.n_alpha, cfg.n_beta, torch.from_numpy(dets.view(np.int64)).cuda())
    x = torch.randn((cfg.roots, n), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    P.shci_set_timing(ctx.handle, True)
    for _ in range(args.sigma_only):
        P.shci_sigma(ctx.handle, x, y)
    st = P.shci_get_stats(ctx.handle)
    print(json.dumps({"n_det": n, "nnz_upper": st["nnz_upper"], "k": cfg.roots,
                      "sigma_ms": st["sigma_ms_total"] / max(1, st["sigma_launches"])}))
    ctx.close()


# ------------------------------------------------------------------ other workloads
# Each prints one JSON measurement line (not the default bench line).

def _gpu_setup():
    import torch
    import paper_1809_04600_gb300 as P
    P.build()
    P.load_library()
    return torch, P


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def run_fci(args):
    """Full-CI space, 10 orbitals, 4a4b (44,100 determinants): build + Davidson
    (1 root, tol 1e-10) per step; energy against the oracle's."""
    torch, P = _gpu_setup()
    import oracle
    cfg = S.config("fci_10o_4a4b")
    h, eri, ec, dets = S.make_system(cfg)
    n = dets.shape[0]
    ctx = P.Context(0, torch.cuda.current_stream())
    H = ctx.handle
    dh, de, dd = _dev(torch, h), _dev(torch, eri), _dev(torch, dets)

    def step():
        P.shci_load_integrals(H, cfg.n_orb, ec, dh, de)
        P.shci_build_connectivity(H, 4, 4, dd, P.SHCI_STORED)
        return P.shci_davidson(H, 1, TOL, MAX_ITER)

    for _ in range(max(3, args.warmup)):
        step()
    P.shci_set_timing(H, True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        e, it, rc = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / args.steps
    st = P.shci_get_stats(H)
    nnz_full = 2 * st["nnz_upper"] + n
    O = oracle.System(h, eri, ec)
    e_ref, _ = O.lowest_eigenpairs(dets, 1, tol=1e-12)
    print(json.dumps({"workload": workload_desc(cfg, n),
                      "metric": "sigma nnz/s over the step; time-to-E", "value": nnz_full * st["sigma_vectors"] /
                      args.steps / dt, "unit": "nnz/s", "s_per_step": dt, "build_ms": st["build_ms"],
                      "davidson_iters": it, "energy": float(e[0]), "energy_oracle": float(e_ref[0]),
                      "abs_dE": abs(float(e[0]) - float(e_ref[0])), "nnz_upper": st["nnz_upper"],
                      "sigma_kernel_ms": st["sigma_ms_total"] / max(1, st["sigma_launches"])}))
    ctx.close()


def run_large(args):
    """76 orbitals, 14a14b, 12-orbital band, |V| = 5e7 (or --n-det): on-the-fly
    sigma (no stored H).  Times the build (count pass) and sigma launches;
    checks sampled rows against the oracle's brute-force rows."""
    torch, P = _gpu_setup()
    import oracle
    cfg = S.config(args.config if args.config != WORKLOAD else "sel_76o_14a14b_50m")
    t = time.perf_counter()
    h, eri, ec, dets = S.make_system(cfg, n_det=args.n_det)
    t_gen = time.perf_counter() - t
    n = dets.shape[0]
    ctx = P.Context(0, torch.cuda.current_stream())
    H = ctx.handle
    P.shci_load_integrals(H, cfg.n_orb, ec, _dev(torch, h), _dev(torch, eri))
    nnz = P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, _dev(torch, dets), P.SHCI_ON_THE_FLY)
    st = P.shci_get_stats(H)
    x = torch.from_numpy(S.random_vectors(n, 1, 3)).cuda()
    y = torch.empty_like(x)
    P.shci_sigma(H, x, y)                       # warm-up
    P.shci_set_timing(H, True)
    reps = max(1, min(args.steps, 3))
    for _ in range(reps):
        P.shci_sigma(H, x, y)
    st2 = P.shci_get_stats(H)
    ms = st2["sigma_ms_total"] / st2["sigma_launches"]
    nnz_full = 2 * nnz + n
    # algorithmic HBM bytes per product: determinants (32 B), x, y and diag (8 B each)
    # per determinant, plus the helper lists read once (member strings and indices)
    bytes_alg = n * (16.0 * S.n_words(cfg.n_orb) * 2 + 24.0) + n * (8.0 + 4.0) * 2
    hbm_peak, kind = load_peaks()
    O = oracle.System(h, eri, ec)
    rng = np.random.default_rng(7)
    rows = np.concatenate([[0], rng.choice(n, 7, replace=False)])
    xr = x.cpu().numpy()
    yr = y.cpu().numpy()
    ref = O.sigma_rows(dets, xr, rows)
    err = float(np.max(np.abs(yr[:, rows] - ref)))
    out = {"workload": workload_desc(cfg).replace("stored H", "on-the-fly sigma"),
           "n_det": n, "nnz_upper": nnz, "gen_s": t_gen, "build_count_ms": st["build_ms"],
           "candidates_per_pass": st["candidates"], "sigma_ms": ms,
           "value": nnz_full / (ms / 1e3), "unit": "full-matrix nnz/s (one vector)",
           "roofline": {"bound": "alu", "hbm_achieved_gbs": bytes_alg / (ms / 1e3) / 1e9,
                        "hbm_peak_gbs": hbm_peak, "hbm_frac": bytes_alg / (ms / 1e3) / 1e9 / hbm_peak,
                        "candidates_per_s": st["candidates"] / (ms / 1e3)},
           "sampled_rows": int(rows.size), "max_abs_err_sampled_rows": err}
    if args.large_davidson:
        out["davidson"] = large_davidson(P, H, O, dets, cfg, rows)
    print(json.dumps(out))
    ctx.close()


def large_davidson(P, H, O, dets, cfg, rows):
    """The lowest root by Davidson with the on-the-fly product (the paper's
    direct method, Sec. VIII): iterations, wall time, sigma time per product,
    and the oracle's check of the eigen-residual (H c - E c) on sampled rows.
    No oracle energy exists at this size (its pair build is O(N^2))."""
    import torch
    n = dets.shape[0]
    v = torch.empty((1, n), dtype=torch.float64, device="cuda")
    P.shci_set_timing(H, True)
    s0 = P.shci_get_stats(H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e, it, rc = P.shci_davidson(H, 1, TOL, MAX_ITER, vecs=v, check=False)
    torch.cuda.synchronize()
    t_dav = time.perf_counter() - t0
    s1 = P.shci_get_stats(H)
    th, rn, ts = P.shci_davidson_history(H, 1)
    launches = s1["sigma_launches"] - s0["sigma_launches"]
    sig_ms = (s1["sigma_ms_total"] - s0["sigma_ms_total"]) / max(1, launches)
    vr = v.cpu().numpy()
    hv = O.sigma_rows(dets, vr, rows)
    res = hv[0] - e[0] * vr[0, rows]
    return {"roots": 1, "tol": TOL, "status": int(rc), "iterations": int(it), "energy": float(e[0]),
            "wall_s": t_dav, "sigma_launches": int(launches), "sigma_ms_per_product": sig_ms,
            "sigma_share": launches * sig_ms / 1e3 / t_dav, "final_residual_norm": float(rn[-1, 0]),
            "energy_change_last_iteration": float(abs(th[-1, 0] - th[-2, 0])) if th.shape[0] > 1 else None,
            "oracle_residual_sampled_rows_max": float(np.max(np.abs(res))),
            "oracle_residual_rows": int(rows.size),
            "start": "lowest eigenvector of H on the 64 determinants of lowest H_ii"}


def run_adjoint(args):
    """20 orbitals, 5a5b, |V| = 1e6: energy + hand-written backward; central
    differences along 16 seeded directions at full size (steps 1e-5 and 2e-5,
    combined by Richardson extrapolation; the plain step-1e-5 error is reported
    beside it)."""
    torch, P = _gpu_setup()
    cfg = S.config("sel_20o_5a5b_1m")
    h, eri, ec, dets = S.make_system(cfg, n_det=args.n_det)
    n = dets.shape[0]
    ctx = P.Context(0, torch.cuda.current_stream())
    H = ctx.handle
    dd = _dev(torch, dets)

    def energy(hh, ee, tol=1e-13):
        P.shci_load_integrals(H, cfg.n_orb, ec, _dev(torch, hh), _dev(torch, ee))
        P.shci_build_connectivity(H, 5, 5, dd, P.SHCI_STORED)
        v = torch.empty((1, n), dtype=torch.float64, device="cuda")
        e, it, rc = P.shci_davidson(H, 1, tol, 800, vecs=v)
        return float(e[0]), v

    e0, v = energy(h, eri, tol=1e-14)        # the gradient is first-order in the vector's error
    gh = torch.empty((cfg.n_orb, cfg.n_orb), dtype=torch.float64, device="cuda")
    ge = torch.empty(eri.size, dtype=torch.float64, device="cuda")
    P.shci_energy_backward(H, v[0], 1.0, gh, ge)      # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    reps = 3
    for _ in range(reps):
        P.shci_energy_backward(H, v[0], 1.0, gh, ge)
    torch.cuda.synchronize()
    t_bwd = (time.perf_counter() - t) / reps
    ghn, gen = gh.cpu().numpy(), ge.cpu().numpy()
    rng = np.random.default_rng(4004)
    step = 1e-5
    rel, rel_plain = [], []
    ndir = 16
    for _ in range(ndir):
        dh = rng.normal(size=h.shape)
        dh = 0.5 * (dh + dh.T)
        de = rng.normal(size=eri.size)
        fd = {}
        for st_ in (step, 2 * step):
            ep, _ = energy(h + st_ * dh, eri + st_ * de)
            em, _ = energy(h - st_ * dh, eri - st_ * de)
            fd[st_] = (ep - em) / (2 * st_)
        rich = (4.0 * fd[step] - fd[2 * step]) / 3.0      # Richardson: the h^2 term cancels
        an = float(np.sum(ghn * dh) + np.dot(gen, de))
        rel.append(abs(rich - an) / max(1.0, abs(an)))
        rel_plain.append(abs(fd[step] - an) / max(1.0, abs(an)))
    e_lin = ec + float(np.sum(h * ghn) + np.dot(eri, gen))
    print(json.dumps({"workload": workload_desc(cfg), "n_det": n, "energy": e0,
                      "backward_s": t_bwd, "fd_directions": ndir, "fd_step": step,
                      "fd_reference": "Richardson (4 D(h) - D(2h)) / 3 of central differences at h = 1e-5, 2e-5; "
                                      "gradient from the eigenvector solved to tol 1e-14",
                      "fd_max_rel_err": max(rel), "fd_rel_errs": rel,
                      "fd_plain_step_max_rel_err": max(rel_plain), "trace_gamma": float(np.trace(ghn)),
                      "energy_linear_identity_err": abs(e_lin - e0)}))
    ctx.close()


def run_select(args):
    """Heat-bath selection (Sec. II.A, Eq. 2) from the bench's 1e6-determinant
    space with its converged 2-root coefficients: GPU time per selection, the
    candidates and new determinants, and the oracle's brute force on a sample
    of determinants of V on the host cores."""
    torch, P = _gpu_setup()
    import oracle as O
    cfg = S.config(args.config)
    h, eri, ec, dets = S.make_system(cfg)
    ctx = P.Context(0, torch.cuda.current_stream())
    H = ctx.handle
    P.shci_load_integrals(H, cfg.n_orb, ec, _dev(torch, h), _dev(torch, eri))
    P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, _dev(torch, dets), P.SHCI_STORED)
    vecs = torch.empty((cfg.roots, dets.shape[0]), dtype=torch.float64, device="cuda")
    P.shci_davidson(H, cfg.roots, TOL, MAX_ITER, vecs=vecs)
    lines = []
    for eps1 in (args.eps1 or [1e-4, 3e-5]):
        t = time.perf_counter()
        new = P.shci_select(H, vecs, eps1)
        torch.cuda.synchronize()
        first = time.perf_counter() - t
        cap = int(new.shape[0])                 # one call per selection from here on
        times = []
        for _ in range(max(1, args.steps)):
            t = time.perf_counter()
            new = P.shci_select(H, vecs, eps1, cap=cap)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
        st = P.shci_get_stats(H)
        # the oracle on a sample of V (same coefficients), timed on the host cores
        rng = np.random.default_rng(0)
        samp = np.sort(rng.choice(dets.shape[0], args.select_sample, replace=False))
        c_h = vecs.cpu().numpy()
        osys = O.System(h, eri, ec)
        t = time.perf_counter()
        osys.select(dets[samp], c_h[:, samp], eps1)
        t_or = time.perf_counter() - t
        lines.append({"eps1": eps1, "n_det": int(dets.shape[0]), "new_dets": int(new.shape[0]),
                      "candidates": st["select_candidates"], "first_call_s": first,
                      "select_s": float(np.median(times)), "select_device_ms": st["select_ms"],
                      "dets_screened_per_s": dets.shape[0] / float(np.median(times)),
                      "oracle": {"sample_dets": int(samp.size), "seconds": t_or,
                                 "dets_screened_per_s": samp.size / t_or, "cores": 1,
                                 "kind": "brute force over every single and double excitation"}})
    # screened second-order Epstein-Nesbet energy of the ground state (Sec. II.B, Eq. 7)
    e0, _, _ = P.shci_davidson(H, 1, TOL, MAX_ITER, vecs=vecs[:1])
    pt = []
    for eps2 in (args.eps2 or [1e-5]):
        t = time.perf_counter()
        e2, npert = P.shci_pt2(H, vecs[0].contiguous(), float(e0[0]), eps2)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        st = P.shci_get_stats(H)
        pt.append({"eps2": eps2, "e_var": float(e0[0]), "dE2": e2, "n_pert": npert, "terms": st["pt2_terms"],
                   "batches": st["pt2_batches"], "seconds": dt, "device_ms": st["pt2_ms"]})
    # semistochastic (Eq. 8): deterministic at eps2_d plus sampled eps2 - eps2_d, beside the deterministic eps2
    semi = None
    if args.semi_eps2:
        eps2, eps2_d = args.semi_eps2, (args.eps2 or [1e-5])[0]
        t = time.perf_counter()
        est, err = P.shci_pt2_semistochastic(H, vecs[0].contiguous(), float(e0[0]), eps2, eps2_d, args.semi_nd,
                                             args.semi_samples, 2024)
        torch.cuda.synchronize()
        t_semi = time.perf_counter() - t
        t = time.perf_counter()
        ref, npert = P.shci_pt2(H, vecs[0].contiguous(), float(e0[0]), eps2)
        torch.cuda.synchronize()
        t_det = time.perf_counter() - t
        st = P.shci_get_stats(H)
        semi = {"eps2": eps2, "eps2_d": eps2_d, "n_d": args.semi_nd, "n_samples": args.semi_samples,
                "dE2_semistochastic": est, "std_error": err, "seconds": t_semi,
                "dE2_deterministic": ref, "deterministic_seconds": t_det, "deterministic_batches": st["pt2_batches"],
                "deterministic_terms": st["pt2_terms"], "n_pert": npert}
        # the 3-step scheme (Sec. IV, Eq. 11) for the same eps2
        t = time.perf_counter()
        r3 = P.shci_pt2_3step(H, vecs[0].contiguous(), float(e0[0]), eps2, 3 * eps2, eps2_d, 1e-4, 16, 32,
                              args.semi_nd, args.semi_samples, 2025)
        torch.cuda.synchronize()
        r3["seconds"] = time.perf_counter() - t
        r3.update({"eps2": eps2, "eps2_psto": 3 * eps2, "eps2_dtm": eps2_d, "target_error": 1e-4,
                   "batches_psto": 16, "batches_sto": 32})
        semi["three_step"] = r3
    # the same screened energy on a 600-determinant space of the same shape: GPU and oracle side by side
    h6, eri6, ec6, d6 = S.make_system(cfg, 600)
    c6 = P.Context(0, torch.cuda.current_stream())
    P.shci_load_integrals(c6.handle, cfg.n_orb, ec6, _dev(torch, h6), _dev(torch, eri6))
    P.shci_build_connectivity(c6.handle, cfg.n_alpha, cfg.n_beta, _dev(torch, d6), P.SHCI_STORED)
    v6 = torch.empty((1, d6.shape[0]), dtype=torch.float64, device="cuda")
    e6, _, _ = P.shci_davidson(c6.handle, 1, TOL, MAX_ITER, vecs=v6)
    P.shci_pt2(c6.handle, v6[0].contiguous(), float(e6[0]), 1e-5)     # lists built
    torch.cuda.synchronize()
    t = time.perf_counter()
    g6, _ = P.shci_pt2(c6.handle, v6[0].contiguous(), float(e6[0]), 1e-5)
    torch.cuda.synchronize()
    t_g6 = time.perf_counter() - t
    t = time.perf_counter()
    o6, _ = O.System(h6, eri6, ec6).pt2(d6, v6[0].cpu().numpy(), float(e6[0]), 1e-5)
    t_o6 = time.perf_counter() - t
    c6.close()
    print(json.dumps({"workload": workload_desc(cfg) + ", heat-bath selection with the converged 2-root "
                                                       "coefficients; screened PT2 of the ground state",
                      "lines": lines, "pt2": pt, "semistochastic": semi,
                      "pt2_600_dets": {"gpu_s": t_g6, "oracle_s": t_o6, "oracle_cores": 1, "dE2_gpu": g6,
                                       "dE2_oracle": o6, "eps2": 1e-5}}))
    ctx.close()


def run_extend(args):
    """Incremental Hamiltonian update (Sec. III, Algorithms 1 and 2) on the
    bench's 1e6-determinant space, which is in generation order: V_old = the
    first (1 - f) n determinants (built, stored H), then the last f n appended.
    Per fraction f, the device time of the incremental update against a full
    build of the grown space (the same call with the switch forced); the grown
    matrix's pair count against a direct build's and sampled rows against the
    oracle's brute force.  Then one variational iteration: select with eps1
    from the converged coefficients, grow V with the selected determinants,
    and solve again."""
    torch, P = _gpu_setup()
    import oracle
    cfg = S.config(args.config)
    h, eri, ec, dets = S.make_system(cfg)
    n = dets.shape[0]
    ctx = P.Context(0, torch.cuda.current_stream())
    H = ctx.handle
    P.shci_load_integrals(H, cfg.n_orb, ec, _dev(torch, h), _dev(torch, eri))
    dd = _dev(torch, dets)
    nnz_direct = 0
    for _ in range(2):
        nnz_direct = P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, dd, P.SHCI_STORED)
    build_ms = P.shci_get_stats(H)["build_ms"]
    O = oracle.System(h, eri, ec)
    lines = []
    for f in (args.extend_frac or [0.02, 0.05, 0.1, 0.2, 0.4]):
        n_old = n - int(round(f * n))
        line = {"fraction_new": f, "n_old": n_old, "n_new": n - n_old}
        for arm, ff in (("rebuild", 1e-9), ("incremental", 1.0)):
            ms = []
            for _ in range(max(1, args.steps)):
                P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, dd[:n_old], P.SHCI_STORED)
                nnz = P.shci_extend_connectivity(H, dd[n_old:], ff)
                st = P.shci_get_stats(H)
                if nnz != nnz_direct or st["extend_incremental"] != (arm == "incremental"):
                    raise RuntimeError("extend: %s arm gave %d pairs, a direct build %d" % (arm, nnz, nnz_direct))
                ms.append(st["extend_ms"])
            line[arm + "_ms"] = float(np.median(ms))
            line[arm + "_candidates"] = st["candidates"]
            if arm == "incremental":
                line["incremental_phase_ms"] = dict(zip(("lists", "count", "alloc_copy", "fill_release"),
                                                        st["extend_phase_ms"]))
        line["speedup"] = line["rebuild_ms"] / line["incremental_ms"]
        # rows of the incrementally grown matrix (old and new) against the oracle
        rng = np.random.default_rng(int(f * 1000))
        rows = np.concatenate([rng.choice(n_old, 3, replace=False), n_old + rng.choice(n - n_old, 3, replace=False)])
        err, same = 0.0, True
        for i in rows:
            gc, gv = P.shci_get_row(H, int(i))          # ascending columns
            oc, ov = O.row(dets, int(i))
            same &= bool(np.array_equal(gc, np.asarray(oc)))
            if same and len(oc):
                err = max(err, float(np.max(np.abs(gv - np.asarray(ov)))))
        line["oracle_rows"] = int(rows.size)
        line["oracle_rows_same_columns"] = same
        line["oracle_rows_max_abs_err"] = err
        lines.append(line)
    # one variational iteration from the full space: solve, select, grow, solve
    P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, dd, P.SHCI_STORED)
    vecs = torch.empty((cfg.roots, n), dtype=torch.float64, device="cuda")
    e0, _, _ = P.shci_davidson(H, cfg.roots, TOL, MAX_ITER, vecs=vecs)
    it = {"eps1": args.extend_eps1, "n_det": n, "energies": [float(x) for x in e0]}
    new = P.shci_select(H, vecs, args.extend_eps1)
    torch.cuda.synchronize()
    it["new_dets"] = int(new.shape[0])
    if new.shape[0]:
        t = time.perf_counter()
        nnz = P.shci_extend_connectivity(H, new, 1.0)
        torch.cuda.synchronize()
        st = P.shci_get_stats(H)
        it.update({"incremental_ms": st["extend_ms"], "incremental_wall_s": time.perf_counter() - t,
                   "nnz_upper": nnz})
        grown = torch.cat([dd, new])
        for _ in range(2):
            nnz2 = P.shci_build_connectivity(H, cfg.n_alpha, cfg.n_beta, grown, P.SHCI_STORED)
        it["rebuild_ms"] = P.shci_get_stats(H)["build_ms"]
        it["direct_build_same_nnz"] = nnz2 == nnz
        guess = torch.zeros((cfg.roots, grown.shape[0]), dtype=torch.float64, device="cuda")
        guess[:, :n] = vecs
        v2 = torch.empty_like(guess)
        t = time.perf_counter()
        e1, iters, _ = P.shci_davidson(H, cfg.roots, TOL, MAX_ITER, guess=guess, vecs=v2)
        torch.cuda.synchronize()
        it.update({"n_det_grown": int(grown.shape[0]), "energies_grown": [float(x) for x in e1],
                   "davidson_s": time.perf_counter() - t, "davidson_iters": iters})
    print(json.dumps({"workload": workload_desc(cfg) + ", in generation order; the last f n determinants "
                                                       "appended to the first (1 - f) n",
                      "direct_build_ms": build_ms, "nnz_upper": nnz_direct, "lines": lines,
                      "variational_iteration": it}))
    ctx.close()


BATCH_PHASES = ("start", "sigma_stored_and_alpha_items", "sigma_beta_items", "gram_columns", "eigensolver",
                "ritz_residuals", "convergence_restart", "basis_rotation", "second_pass_coef", "second_projection",
                "cholqr1_coef", "cholqr_apply", "cholqr2_coef", "next_block", "bookkeeping")


def run_batch(args):
    """64 uneven systems x 4 roots: one batched persistent launch vs 64
    sequential shci_davidson calls (same builds, same tolerance)."""
    torch, P = _gpu_setup()
    cfgs = S.batch_configs()
    if args.n_det:
        cfgs = [S.Config(c.name, c.n_orb, c.n_alpha, c.n_beta, c.rank, c.seed, min(c.n_det, args.n_det), c.roots)
                for c in cfgs]
    t = time.perf_counter()
    systems = []
    for c in cfgs:
        h, eri, ec, dets = S.make_system(c)
        systems.append(dict(n_orb=c.n_orb, n_alpha=c.n_alpha, n_beta=c.n_beta, h=_dev(torch, h),
                            eri=_dev(torch, eri), e_core=ec, dets=_dev(torch, dets)))
    t_gen = time.perf_counter() - t
    ctx = P.Context(0, torch.cuda.current_stream())
    budget = args.batch_budget_gb * 1e9
    t = time.perf_counter()
    b = P.shci_batch_create(ctx.handle, systems, stored_budget_bytes=budget)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t
    k = 4
    e, it, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), k, tol=TOL, max_iter=MAX_ITER)
    st0 = P.shci_batch_get_stats(b)
    torch.cuda.synchronize()
    t = time.perf_counter()
    e, it, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), k, tol=TOL, max_iter=MAX_ITER)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t
    st = P.shci_batch_get_stats(b)
    modes = P.shci_batch_get_modes(b, len(systems))
    P.shci_batch_destroy(b)
    # sequential: one context per system, the batch's storage decisions, Davidson timed alone
    seq_time, seq_e, seq_it = 0.0, [], []
    seq_parts = np.zeros(7)
    seq_sigma_by_mode = {}
    for d, mode in zip(systems, modes):
        c2 = P.Context(0, torch.cuda.current_stream())
        P.shci_load_integrals(c2.handle, d["n_orb"], d["e_core"], d["h"], d["eri"])
        P.shci_build_connectivity(c2.handle, d["n_alpha"], d["n_beta"], d["dets"], int(mode))
        P.shci_set_timing(c2.handle, False, davidson_phases=True)   # per-part device times, events only
        torch.cuda.synchronize()
        t = time.perf_counter()
        es, its, rcs = P.shci_davidson(c2.handle, k, TOL, MAX_ITER, check=False)
        torch.cuda.synchronize()
        seq_time += time.perf_counter() - t
        parts = np.array(P.shci_get_stats(c2.handle)["davidson_phase_ms"][:7])
        seq_parts += parts
        seq_sigma_by_mode[int(mode)] = seq_sigma_by_mode.get(int(mode), 0.0) + parts[5]
        seq_e.append(es)
        seq_it.append(its)
        c2.close()
    seq_e = np.array(seq_e)
    print(json.dumps({"workload": "64 systems: n_orb U{12..30}, 3-8 electrons per spin, |V| log-uniform "
                                  "1e4..2e6 (capped at half the full-CI size), 4 roots each, FP64",
                      "total_det": st["total_det"], "total_nnz_upper": st["total_nnz_upper"],
                      "n_stored": st["n_stored"], "n_stored_upper": st["n_stored_upper"],
                      "n_on_the_fly": st["n_on_the_fly"], "gen_s": t_gen,
                      "create_s": t_create, "batched_s": t_batch, "batched_device_ms": st["solve_ms"],
                      "sequential_s": seq_time, "speedup": seq_time / t_batch,
                      "max_abs_dE_vs_sequential": float(np.max(np.abs(e - seq_e))),
                      "graph": st["graph"], "grid_ctas": st["grid_ctas"],
                      "tuned": {"rows_per_item": st["tuned_rows_per_item"], "ctas_per_sm": st["tuned_ctas_per_sm"],
                                "lanes_per_row": st["tuned_lanes_per_row"], "vector_slice": st["tuned_vslice"],
                                "trial_ms": st0["tune_ms"]},
                      "max_iters": st["max_iters"], "all_converged": bool(conv.all()),
                      "iters_sum_batched": int(np.sum(it)), "iters_sum_sequential": int(np.sum(seq_it)),
                      "phase_ms": {name: round(v, 3) for name, v in zip(BATCH_PHASES, st["phase_ms"])},
                      "sequential_part_ms": {name: round(float(v), 3) for name, v in zip(
                          ("start", "eigensolver", "ritz_residuals", "restarts", "orthonormalisation", "sigma",
                           "gram_columns"), seq_parts)},
                      "sequential_sigma_ms_by_mode": {{0: "stored", 1: "on_the_fly", 3: "stored_upper"}[m]:
                                                      round(v, 3) for m, v in seq_sigma_by_mode.items()}}))
    ctx.close()


def run_upper(args):
    """The two stored forms of H on the bench space: sigma per launch for 1, 2
    and 4 vectors with both triangles stored (a pure gather) and with the
    upper triangle alone (the transposed half added by FP64 atomic adds), and
    the memory each takes."""
    torch, P = _gpu_setup()
    cfg = S.config(args.config)
    h, eri, ec, dets = S.make_system(cfg, n_det=args.n_det)
    n = dets.shape[0]
    out = {"workload": workload_desc(cfg, n).replace("stored H", "stored H in both forms"), "n_det": n,
           "forms": {}}
    for mode, name in ((P.SHCI_STORED, "both_triangles"), (P.SHCI_STORED_UPPER, "upper_triangle")):
        ctx = P.Context(0, torch.cuda.current_stream())
        P.shci_load_integrals(ctx.handle, cfg.n_orb, ec, _dev(torch, h), _dev(torch, eri))
        nnz = P.shci_build_connectivity(ctx.handle, cfg.n_alpha, cfg.n_beta, _dev(torch, dets), mode)
        held = nnz * (2 if mode == P.SHCI_STORED else 1)
        rec = {"stored_nonzeros": held, "stored_gb": 12.0 * held / 1e9, "sigma_ms": {}}
        for k in (1, 2, 4):
            x = torch.randn(k, n, dtype=torch.float64, device="cuda")
            y = torch.empty_like(x)
            for _ in range(3):
                P.shci_sigma(ctx.handle, x, y)
            P.shci_set_timing(ctx.handle, True)      # CUDA events around every sigma launch
            for _ in range(10):
                P.shci_sigma(ctx.handle, x, y)
            st = P.shci_get_stats(ctx.handle)
            P.shci_set_timing(ctx.handle, False)
            rec["sigma_ms"][str(k)] = st["sigma_ms_total"] / max(st["sigma_launches"], 1)
        rec["upper_pairs_per_s_k1"] = nnz / (rec["sigma_ms"]["1"] * 1e-3)
        out["forms"][name] = rec
        out["nnz_upper"] = nnz
        ctx.close()
    print(json.dumps(out))


def run_peaks(args):
    """The peak-rate microbenchmarks (FP64 FMA and add, INT32 multiply-add,
    XOR + popcount, FP64 atomics and random gathers in L2), with the clocks
    sampled while they run."""
    import torch
    torch.cuda.init()
    sampler = ClockSampler(0)
    sampler.start()
    best = measure_peaks(0)
    clocks = sampler.stop()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    print(json.dumps({"workload": "peak-rate microbenchmarks (measure/peaks.cu), best of 2/4/8 CTAs x 256 threads "
                                  "per SM",
                      "ops_per_s": best, "fp64_fma_tflops": 2.0 * best["dfma"] / 1e12,
                      "per_sm_per_clock": {k: v / sms / (mhz * 1e6) for k, v in best.items()},
                      "sms": sms, "clocks": clocks}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--cpu-rows", type=int, default=120000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-det", type=int, default=None,
                    help="profiling only: a smaller space of the same shape (not a bench line)")
    ap.add_argument("--sigma-only", type=int, default=0,
                    help="profiling only: build once, then launch the sigma kernel this many times")
    ap.add_argument("--workload", default="main",
                    choices=["main", "fci", "large", "adjoint", "batch", "select", "extend", "peaks", "upper"],
                    help="main: the bench line; others print the measurement line of another workload")
    ap.add_argument("--batch-budget-gb", type=float, default=240.0,
                    help="batch workload: device memory the stored matrices may take (capped at 0.8 x free)")
    ap.add_argument("--large-iters", type=int, default=3,
                    help="main bench line: Davidson iterations of the bounded 5e7 section (0: skip it)")
    ap.add_argument("--large-davidson", action="store_true",
                    help="large workload: also solve for the lowest root with the on-the-fly product")
    ap.add_argument("--eps1", type=float, action="append", help="selection thresholds (select workload)")
    ap.add_argument("--select-sample", type=int, default=200, help="determinants of V the oracle screens")
    ap.add_argument("--eps2", type=float, action="append", help="PT2 screening thresholds (select workload)")
    ap.add_argument("--semi-eps2", type=float, default=1e-6, help="semistochastic eps2 (0: skip)")
    ap.add_argument("--semi-nd", type=int, default=20000, help="draws per semistochastic sample")
    ap.add_argument("--semi-samples", type=int, default=16, help="semistochastic samples")
    ap.add_argument("--extend-frac", type=float, action="append",
                    help="fractions of new determinants (extend workload)")
    ap.add_argument("--extend-eps1", type=float, default=1e-3, help="selection threshold (extend workload)")
    args = ap.parse_args()
    if args.workload != "main":
        {"fci": run_fci, "large": run_large, "adjoint": run_adjoint, "batch": run_batch, "upper": run_upper,
         "select": run_select, "extend": run_extend, "peaks": run_peaks}[args.workload](args)
    elif args.sigma_only:
        run_sigma_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
