#!/usr/bin/env python
"""Benchmark of the SQD hot path (arXiv 2601.16169) on GB300.

Default line: the 4.0e8-determinant workload (scale36: 36 orbitals, 15+15
electrons, 20000 shared sampled strings), the paper's 1e8-1e9 scale
(Section VI).  One step is one sigma = H C of one FP64 vector over every
determinant (sqd_sigma, the product that takes 96.5% of a Davidson iteration),
on excitation tables built before the timed region; the headline `value` is
H.C applications per second.  Beside it, in the same run:

* time_to_converged_E: one ground-state Davidson solve on the same tables
  (|dE| <= 1e-8 Ha, |r| <= 1e-5), timed with CUDA events from the call to
  its return, with the Davidson's own classes (Ritz/residual, Gram-Schmidt,
  Rayleigh-Ritz) booked with their algorithmic flops and bytes;
* e2e: the same sigma steps through the C ABI from pinned host buffers, the
  vector copied in and sigma copied out inside the timed region;
* roofline of the dominant kernel (the alpha-beta paired singles) against
  the FP64 ALU peak, and the HBM fraction of the whole sigma;
* cpu_baseline: the oracle's sigma on 1e5 seeded rows, extrapolated;
* sub-records: the h2o29 8-root solve (whole path per step), the
  double-float sigma, the 64-subspace batched solver against 64 sequential
  solves, the adjoint (RDMs + orbital gradient) at adjoint29, the stored-H
  product, each with its oracle baseline where one is defined.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica of the sigma steps
(the path does not shard: replicas only) and rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sqd_inputs as si  # noqa: E402

METRIC = "Davidson sigma H·C/s and time-to-converged E (FP64) vs HBM roofline, 1×GB300"
UNIT = "H·C/s"

# Davidson settings per workload (convergence readings of the build)
SOLVE = {
    "scale36": dict(nroots=1, tol_residual=1e-5, tol_energy=1e-8, max_iter=400),
    "h2o29": dict(nroots=8, tol_residual=1e-8, tol_energy=1e-8, max_iter=200),
    "adjoint29": dict(nroots=1, tol_residual=1e-5, tol_energy=1e-8, max_iter=200),
    "full8": dict(nroots=1, tol_residual=1e-8, tol_energy=1e-10, max_iter=200),
}
DESCR = {
    "scale36": "scale36: norb=36, 15+15 electrons, 20000 shared sampled strings "
               "(P(k) ~ 1/(1+exp((k-15)/2.5))), 4.0e8 determinants, rank-72 integrals, "
               "ground state (|dE| <= 1e-8, ||r|| <= 1e-5)",
    "h2o29": "h2o29: norb=29, 5+5 electrons, 2000 shared sampled strings (P(k) ~ exp(-k/6)), "
             "4.0e6 determinants, rank-58 integrals, 8 roots to ||r|| <= 1e-8",
    "adjoint29": "adjoint29: norb=29, 5+5 electrons, 5000 shared strings, 2.5e7 determinants",
    "full8": "full8: norb=8, 4+4 electrons, full space, 4900 determinants",
}
SUBRECORDS = ("h2o29", "full8", "df", "spin_flip", "batched", "adjoint", "stored")

# FP64 peak for the ALU roofline: 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM
# (the nominal 1.25 TFLOP/s FP64 of GB300 at its maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
SIGMA_CLASSES = ("same_spin_alpha", "same_spin_beta", "alpha_beta")
DAVIDSON_CLASSES = ("davidson", "ortho", "ortho_block", "gcols", "eigh")
KERNEL_OF = {"same_spin_alpha": "k_same_spin", "same_spin_beta": "k_same_spin",
             "alpha_beta": "k_alpha_beta"}


def _args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10,
                   help="timed steps (one sigma of one vector each)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="scale36", choices=sorted(SOLVE))
    p.add_argument("--mode", default="headline",
                   choices=["headline", "solve", "sigma", "batched", "adjoint"],
                   help="headline: sigma steps + one converged solve + sub-records; "
                        "solve: the whole path (strings, tables, Davidson) per step; "
                        "sigma: one sigma per step on prebuilt tables (kernel-only line); "
                        "batched: the 64-subspace workload in one batched solve vs one "
                        "solve per subspace; adjoint: the backward pass (RDMs + orbital "
                        "gradient) of a converged state against one sigma")
    p.add_argument("--no-solve", action="store_true",
                   help="headline: skip the converged solve")
    p.add_argument("--sub", default=",".join(SUBRECORDS),
                   help="headline: comma-separated sub-records to add ('none' to skip): "
                        + ", ".join(SUBRECORDS))
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--cpu-rows", type=int, default=None,
                   help="rows of sigma in the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--nbatch", type=int, default=64)
    p.add_argument("--tol-residual", type=float, default=1e-6,
                   help="batched mode: residual tolerance of both solvers")
    p.add_argument("--sigma-mode", type=int, default=0, choices=[0, 1],
                   help="0: native FP64 sigma (headline); 1: double-float on the FP32 pipe")
    p.add_argument("--spin-flip", type=int, default=0, choices=[-1, 0, 1],
                   help="sigma/solve modes: vectors of one spin-flip sector (C^T = s C, "
                        "shared string sets only); 0: general vectors")
    p.add_argument("--correction", default="davidson", choices=["davidson", "olsen"],
                   help="Davidson correction vector (olsen: orthogonal to the Ritz vector)")
    p.add_argument("--max-iter", type=int, default=None,
                   help="stop Davidson after this many iterations (short profiling runs; "
                        "the line then reports an unconverged solve)")
    p.add_argument("--nroots", type=int, default=None,
                   help="solve mode: number of roots (default: the workload's)")
    p.add_argument("--max-subspace", type=int, default=None,
                   help="Davidson subspace limit (default max(6 nroots, 16))")
    p.add_argument("--stored", action="store_true",
                   help="sigma mode: apply the stored H (sparse matrix) instead")
    return p.parse_args(argv)


# ----------------------------------------------------------- clocks ------

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clocks(out)


def parse_clocks(text):
    """Median SM clock, maximum clock and the throttle reasons seen in the
    nvidia-smi samples (csv, no header, no units)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------ CPU baselines -----

def _cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


_VECTORS = {}


def _input_vector(N):
    """The seeded input vector of N determinants (drawn once per size: at
    4e8 determinants it is 3.2 GB of normal draws)."""
    if N not in _VECTORS:
        _VECTORS.clear()
        _VECTORS[N] = si.random_vectors(1, N, 13)[0]
    return _VECTORS[N]


def oracle_sigma_rate(w, rows_n, seed=0):
    """The oracle's sigma (as it stands) on rows_n seeded rows of one sigma
    of workload w on the host cores: (rows per second, seconds, rows)."""
    import oracle
    oracle.lib()
    N = w.ndet
    C = _input_vector(N)
    rows = np.sort(np.random.default_rng(seed).choice(N, size=min(rows_n, N), replace=False))
    t0 = time.perf_counter()
    oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, C, rows=rows)
    dt = time.perf_counter() - t0
    return len(rows) / dt, dt, len(rows)


def cpu_baseline(w, rows_n):
    """The oracle timed on the host cores on a bounded sample: rows_n seeded
    rows of one sigma.  H.C/s = rows/s divided by the determinant count (an
    extrapolation when the sample is smaller than the space)."""
    rate, dt, nr = oracle_sigma_rate(w, rows_n)
    N = w.ndet
    return {"value": rate / N, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": "%d seeded rows of one sigma of %s (%.1f s incl. neighbour lists); "
                      "H.C/s = rows/s / %d determinants%s"
                      % (nr, w.name, dt, N, " (extrapolated)" if nr < N else ""),
            "extrapolated": nr < N, "seconds": dt}


def cpu_baseline_one_thread(name, rows_n):
    """The same oracle sample on one host thread (a child process started
    with OMP_NUM_THREADS=1, so this process's OpenMP pool is untouched)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench, sqd_inputs as si; "
            "print(json.dumps(bench.cpu_baseline(si.workload(%r), %d)))" % (ROOT, name, rows_n))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                             text=True, timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as exc:  # reported, not fatal: the bench line stays valid
        return {"error": str(exc)[:200]}


def default_cpu_rows(name):
    return {"scale36": 100000, "h2o29": 4000000, "adjoint29": 100000, "full8": 4900}[name]


def cpu_baseline_batched(subs, iters, nsample=8, rows_each=20000):
    """The oracle's sigma on `rows_each` seeded rows of `nsample` seeded
    subspaces of the batch, extrapolated to the batched workload: sum over
    subspaces of (iterations + 1) sigma applications of N_b rows each."""
    pick = np.random.default_rng(5).choice(len(subs), size=min(nsample, len(subs)),
                                           replace=False)
    rows = secs = 0.0
    for b in sorted(pick):
        r, dt, nr = oracle_sigma_rate(subs[b], rows_each, seed=int(b))
        rows += nr
        secs += dt
    rate = rows / secs
    total_rows = float(sum(w.ndet * (int(i) + 1) for w, i in zip(subs, iters)))
    return {"value": rate, "unit": "det rows of sigma/s", "cores": _cores(), "kind": "oracle",
            "sample": "%d seeded rows of each of %d seeded subspaces (%.1f s); extrapolated "
                      "to the %.3g sigma rows of the 64 solves" % (rows_each, len(pick), secs,
                                                                   total_rows),
            "extrapolated": True, "solve_seconds_extrapolated": total_rows / rate}


def cpu_baseline_adjoint(w, iters, nentries=20):
    """The oracle on the adjoint workload, extrapolated: the solve as
    (iterations + 1) sigma products at the rate of 1e5 seeded rows, the RDMs
    as norb^4 2-RDM entries plus norb^2 1-RDM entries at the rate of
    `nentries` seeded entries (each a pass over every determinant)."""
    import oracle
    rate, dt_s, nr = oracle_sigma_rate(w, 100000)
    C = si.random_vectors(1, w.ndet, 13)[0]
    C /= np.linalg.norm(C)
    rng = np.random.default_rng(9)
    quads = [tuple(int(x) for x in rng.integers(0, w.norb, 4)) for _ in range(nentries)]
    t0 = time.perf_counter()
    oracle.rdm2(w.norb, w.strings_a, w.strings_b, C, entries=quads)
    dt2 = (time.perf_counter() - t0) / nentries
    pairs = [tuple(int(x) for x in rng.integers(0, w.norb, 2)) for _ in range(nentries)]
    t0 = time.perf_counter()
    oracle.rdm1(w.norb, w.strings_a, w.strings_b, C, entries=pairs)
    dt1 = (time.perf_counter() - t0) / nentries
    solve_s = (iters + 1) * w.ndet / rate
    rdm_s = dt2 * w.norb ** 4 + dt1 * w.norb ** 2
    return {"value": 1.0 / rdm_s, "unit": "backward passes/s", "cores": _cores(),
            "kind": "oracle",
            "sample": "%d seeded sigma rows (%.1f s), %d seeded 2-RDM and 1-RDM entries; "
                      "extrapolated to the %d-iteration solve and the full RDMs"
                      % (nr, dt_s, nentries, iters),
            "extrapolated": True, "solve_seconds_extrapolated": solve_s,
            "rdm_seconds_extrapolated": rdm_s}


# ------------------------------------------------------ replica timing ---

def aggregate_replicas(dev_ms, e2e_s, work, world, device=None):
    """Replicas-only multi-GPU: every rank runs its own copy of the
    workload.  Returns (max device ms, max e2e seconds, total work over
    ranks); with world == 1 the inputs unchanged."""
    if world <= 1:
        return dev_ms, e2e_s, work
    import torch
    import torch.distributed as dist
    tt = torch.tensor([dev_ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cnt = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(cnt)
    return float(tt[0]), float(tt[1]), float(cnt[0])


# ------------------------------------------------------- traffic record ---

def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_sigma.cu", "sigma_body.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2601_16169_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload="h2o29"):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/traffic_<workload>.txt), if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic_%s.txt" % workload)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if "=" in line and not line.lstrip().startswith("#"):
            k, v = line.split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != kernel_source_hash():
        return None
    v = vals.get("%s.bytes_per_launch" % kernel)
    return float(v) if v else None


def _hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except Exception:
        return 6800.0


def _hbm_peak_source():
    return ("measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json"))
            else "fallback 6800 GB/s")


# ------------------------------------------------------ library access ---

class Env:
    """The library, torch and one context on this rank's device."""

    def __init__(self, local_rank):
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2601_16169_gb300 as sqd
        torch.cuda.set_device(local_rank)
        self.torch, self.sqd, self.local_rank = torch, sqd, local_rank
        self.dev = torch.device("cuda", local_rank)
        self.ctx = sqd.Context(local_rank)
        self.stream = torch.cuda.current_stream(self.dev)

    def tensor(self, a, dtype=None):
        t = self.torch.from_numpy(np.ascontiguousarray(a))
        return t.to(self.dev)

    def tables(self, w, raw=None, h=None, V=None):
        """Strings filtered on the device, then the excitation tables."""
        raw = raw if raw is not None else self.tensor(w.raw_a.view(np.int64))
        h = h if h is not None else self.tensor(w.h)
        V = V if V is not None else self.tensor(w.V)
        s = self.sqd.build_strings(self.ctx, raw, w.norb, w.nelec_a)
        return self.sqd.excitation_tables(self.ctx, w.norb, s, w.nelec_a, s, w.nelec_b,
                                          h, V, 0.0)

    def events(self):
        E = self.torch.cuda.Event
        return E(enable_timing=True), E(enable_timing=True)

    def sync(self):
        self.torch.cuda.synchronize(self.dev)

    def close(self):
        self.ctx.close()


def class_record(prof, names):
    """Per profile class: ms, regions, algorithmic flops and bytes and the
    fractions of the FP64 peak and the HBM copy bandwidth they reach."""
    out = {}
    for k in names:
        v = prof[k]
        ms = v["ms"]
        tf = v["flops"] / (ms / 1e3) / 1e12 if ms else 0.0
        gbs = v["bytes"] / (ms / 1e3) / 1e9 if ms else 0.0
        out[k] = {"ms": round(ms, 3), "regions": v["regions"], "flops": v["flops"],
                  "bytes": v["bytes"], "tflops": tf, "frac_fp64_peak": tf / FP64_PEAK_TFLOPS,
                  "gbs": gbs, "frac_hbm": gbs / _hbm_peak()}
    return out


def sigma_roofline(prof, workload):
    """Roofline of the dominant sigma kernel (largest event time) against the
    FP64 ALU peak; achieved = its algorithmic flops per launch / mean launch
    time (library CUDA events on the context's stream)."""
    sig = {k: prof[k] for k in SIGMA_CLASSES}
    dom = max(sig, key=lambda k: sig[k]["ms"])
    d = sig[dom]
    achieved = (d["flops"] / d["regions"]) / (d["ms"] / d["regions"] / 1e3) / 1e12
    return {"bound": "alu", "kernel": "%s (%s)" % (KERNEL_OF[dom], dom),
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": recorded_traffic(dom, workload),
            "peak_source": "derived FP64: 152 SMs x 2070 MHz x 4 flop/clk/SM (of derived; "
                           "the FMA-chain probe in fp64_measured is its measured check)",
            "launch_ms": d["ms"] / d["regions"], "flops_per_launch": d["flops"] / d["regions"],
            "compulsory_bytes_per_launch": d["bytes"] / d["regions"],
            "traffic_note": "DRAM bytes per launch from one ncu capture of this kernel on this "
                            "workload (profiles/traffic_<workload>.txt); FP64-bound, so DRAM "
                            "runs at a few percent of its bandwidth whatever the re-reads"}


def sigma_summary(prof):
    """Whole-sigma numbers from the profile classes: time, FP64 rate, the
    bound max(compulsory bytes / HBM, flops / FP64 peak) over the measured
    time, and the HBM fraction of the compulsory bytes."""
    ms = sum(prof[k]["ms"] for k in SIGMA_CLASSES) + prof["transpose"]["ms"]
    fl = sum(prof[k]["flops"] for k in SIGMA_CLASSES)
    by = sum(prof[k]["bytes"] for k in SIGMA_CLASSES + ("transpose",))
    t_f, t_b = fl / (FP64_PEAK_TFLOPS * 1e12), by / (_hbm_peak() * 1e9)
    return {"ms": ms, "fp64_tflops": fl / (ms / 1e3) / 1e12 if ms else None,
            "bound": {"t_flops_ms": t_f * 1e3, "t_bytes_ms": t_b * 1e3, "t_measured_ms": ms,
                      "frac": max(t_f, t_b) / (ms / 1e3) if ms else None},
            "hbm_roofline": {"bound": "hbm", "achieved": by / (ms / 1e3) / 1e9 if ms else None,
                             "peak": _hbm_peak(), "unit": "GB/s",
                             "frac": (by / (ms / 1e3) / 1e9) / _hbm_peak() if ms else None,
                             "note": "compulsory sigma bytes (read C, read/write sigma, "
                                     "diagonal, transposes) / sigma time, of measured copy "
                                     "bandwidth"}}


# ------------------------------------------------------------ records ----

def _barrier():
    """Barrier over the replicas (nothing with one process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def sigma_steps(env, t, C, S, steps, warmup):
    """Warm-up, then `steps` sigma products timed with CUDA events on the
    context's stream, the library's per-kernel events on, clocks sampled."""
    sqd, ctx = env.sqd, env.ctx
    for _ in range(warmup):
        sqd.sigma(ctx, t, C, S)
    env.sync()
    _barrier()
    ctx.profile(True)
    clk = ClockSampler(env.local_rank).start()
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    for _ in range(steps):
        sqd.sigma(ctx, t, C, S)
    ev1.record(env.stream)
    env.sync()
    _barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    launches = ctx.launch_count()
    ctx.profile(False)
    return ms, prof, launches, clocks


def solve_record(env, t, opts, workload):
    """One converged Davidson solve on prebuilt tables, timed from the call
    to its return (CUDA events), with the per-class kernel times."""
    sqd, ctx = env.sqd, env.ctx
    env.sync()
    ctx.profile(True)
    clk = ClockSampler(env.local_rank).start()
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    e, X, it, res, rc = sqd.davidson(ctx, t, **opts)
    ev1.record(env.stream)
    env.sync()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    ctx.profile(False)
    del X
    sig = sigma_summary(prof)
    dav_ms = sum(prof[k]["ms"] for k in DAVIDSON_CLASSES)
    return {"time_to_converged_E_s": ms / 1e3, "iterations": int(it),
            "energies": [float(x) for x in e], "residuals": [float(x) for x in res],
            "status": int(rc), "sigma_applications": prof["same_spin_alpha"]["regions"],
            "settings": opts, "workload": DESCR[workload],
            "sigma_ms": sig["ms"], "sigma_share": sig["ms"] / ms,
            "davidson_vector_ms": dav_ms, "davidson_share": dav_ms / ms,
            "davidson_classes": class_record(prof, DAVIDSON_CLASSES),
            "sigma_classes": class_record(prof, SIGMA_CLASSES),
            "roofline": sigma_roofline(prof, workload), "clocks": clocks}


def e2e_sigma_pipelined(env, t, C, S, Cp, Sp, n):
    """n sigma steps through the public API from pinned host buffers, wall
    seconds.  Every step copies its input vector host -> device and its
    sigma device -> host; the copies run on two copy streams and overlap the
    neighbouring steps' sigma (two device buffer pairs, ordered by events),
    as a pipeline of host-resident work would."""
    torch, sqd, ctx = env.torch, env.sqd, env.ctx
    main = env.stream
    s_in, s_out = torch.cuda.Stream(env.dev), torch.cuda.Stream(env.dev)
    bufs = [(C, S), (torch.empty_like(C), torch.empty_like(S))]
    E = torch.cuda.Event
    ev_in, ev_done, ev_out = [E(), E()], [E(), E()], [E(), E()]
    env.sync()
    t0 = time.perf_counter()
    with torch.cuda.stream(s_in):
        bufs[0][0].copy_(Cp, non_blocking=True)
        ev_in[0].record(s_in)
    for k in range(n):
        c, sg = bufs[k % 2]
        main.wait_event(ev_in[k % 2])
        if k >= 2:
            main.wait_event(ev_out[k % 2])  # the copy-out of step k-2 left sg
        sqd.sigma(ctx, t, c, sg)
        ev_done[k % 2].record(main)
        if k + 1 < n:
            with torch.cuda.stream(s_in):
                if k >= 1:
                    s_in.wait_event(ev_done[(k + 1) % 2])  # step k-1 has read it
                bufs[(k + 1) % 2][0].copy_(Cp, non_blocking=True)
                ev_in[(k + 1) % 2].record(s_in)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[k % 2])
            Sp.copy_(sg, non_blocking=True)
            ev_out[k % 2].record(s_out)
    env.sync()
    dt = time.perf_counter() - t0
    del bufs
    return dt


def headline(args, rank, world, local_rank):
    """The default line: sigma steps on the 4.0e8-determinant workload, e2e
    through host buffers, one converged solve, then the sub-records."""
    env = Env(local_rank)
    torch, sqd, ctx = env.torch, env.sqd, env.ctx
    w = si.workload(args.workload)
    N = w.ndet
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    t = env.tables(w)
    ev1.record(env.stream)
    env.sync()
    tables_ms = ev0.elapsed_time(ev1)
    shape = (w.strings_a.size, w.strings_b.size)
    C_h = torch.from_numpy(si.random_vectors(1, N, 13).reshape(shape))
    C = C_h.to(env.dev)
    S = torch.empty_like(C)
    if args.sigma_mode:
        t.set_sigma_mode(args.sigma_mode)
    dev_ms, prof, launches, clocks = sigma_steps(env, t, C, S, args.steps, args.warmup)
    # measured FP64 rates of this GPU (the derived peak is the roofline's)
    fp64_dfma, fp64_dmma = ctx.measure_fp64_peaks()

    # e2e: the vector from pinned host memory, sigma back to it, per step
    n_e2e = args.e2e_steps if args.e2e_steps is not None else max(1, min(args.steps, 10))
    e2e_s = 0.0
    if n_e2e:
        Cp = C_h.pin_memory()
        Sp = torch.empty_like(Cp).pin_memory()
        sqd.sigma(ctx, t, C, S)
        env.sync()
        if world > 1:
            torch.distributed.barrier()
        e2e_s = e2e_sigma_pipelined(env, t, C, S, Cp, Sp, n_e2e)
        del Cp, Sp
    del C_h

    t_max, e2e_max, hc_tot = aggregate_replicas(dev_ms, e2e_s, args.steps, world, env.dev)
    sig = sigma_summary(prof)
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": hc_tot / (t_max / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded integrals and sampled strings shaped like the paper's "
                    "H2O/N2 sets (no dataset available)",
            "config": {"workload": DESCR[args.workload],
                       "step": "one sigma = H C of one vector over all %d determinants on "
                               "tables built before the timed region" % N,
                       "l2": "inputs larger than L2 (%.1f GB vectors)" % (8 * N / 1e9)
                       if 8 * N > 129e6 else "vectors may fit in L2",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "sigma_mode": "double-float (FP32 pipe)" if args.sigma_mode
                       else "fp64"},
            "det_per_s": hc_tot / (t_max / 1e3) * N,
            "tables_s": tables_ms / 1e3, "tables": t.info(),
            "sigma_fp64_tflops": sig["fp64_tflops"], "sigma_bound": sig["bound"],
            "roofline": sigma_roofline(prof, args.workload),
            "hbm_roofline": sig["hbm_roofline"],
            "kernels": class_record(prof, SIGMA_CLASSES),
            "transpose_ms_per_step": prof["transpose"]["ms"] / args.steps,
            "fp64_measured": {"dfma_tflops": fp64_dfma, "dmma_tflops": fp64_dmma,
                              "note": "probe grids of independent FP64 FMA chains and of "
                                      "FP64 tensor MMAs (m8n8k4) at the SM clock in clocks"},
            "e2e": {"value": n_e2e * world / e2e_max if n_e2e else None, "unit": UNIT,
                    "steps": n_e2e, "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N,
                    "path": "pinned host C -> device, sqd_sigma, device -> pinned host sigma; "
                            "the copies on two copy streams overlap the neighbouring steps' "
                            "sigma (wall clock from the first copy-in to the last copy-out)"}
            if n_e2e else None,
            "clocks": clocks, "gpu_launches": launches,
        }
    # the same sigma with the double-float products (opt-in mode 1)
    subs = [] if args.sub == "none" else [s for s in args.sub.split(",") if s]
    if world == 1 and "df" in subs and not args.sigma_mode:
        t.set_sigma_mode(1)
        ms_df, prof_df, _, clk_df = sigma_steps(env, t, C, S, 3, 2)
        t.set_sigma_mode(0)
        line["sigma_df32"] = {"ms_per_step": ms_df / 3, "value": 3 / (ms_df / 1e3),
                              "unit": UNIT, "speedup_vs_fp64": (dev_ms / args.steps) / (ms_df / 3),
                              "kernels": {k: round(prof_df[k]["ms"] / 3, 3)
                                          for k in SIGMA_CLASSES},
                              "clocks": clk_df,
                              "note": "double-float multiply-adds on the FP32 pipe, 48-bit "
                                      "operands; not the FP64 headline"}
    del C, S
    torch.cuda.empty_cache()
    if world == 1 and not args.no_solve:
        opts = dict(SOLVE[args.workload])
        if args.max_subspace:
            opts["max_subspace"] = args.max_subspace
        if args.max_iter is not None:
            opts["max_iter"] = args.max_iter
            opts["raise_on_nonconvergence"] = False
        if args.correction != "davidson":
            opts["correction"] = args.correction
        sr = solve_record(env, t, opts, args.workload)
        line["time_to_converged_E_s"] = sr["time_to_converged_E_s"]
        line["davidson_iterations"] = sr["iterations"]
        line["energy"] = sr["energies"][0]
        line["solve"] = sr
    t.close()
    env.close()
    torch.cuda.empty_cache()
    if rank != 0:
        return None
    if world == 1:
        for name in subs:
            if name == "df":
                continue
            fn = {"h2o29": sub_h2o29, "full8": sub_full8, "batched": sub_batched,
                  "adjoint": sub_adjoint, "stored": sub_stored}.get(name)
            if name == "spin_flip":
                fn = lambda a, lr: sub_spin_flip(a, lr, line.get("energy"))  # noqa: E731
            try:
                line[name] = fn(args, local_rank)
            except Exception as exc:  # a failed sub-record is reported, not fatal
                line[name] = {"error": "%s: %s" % (type(exc).__name__, str(exc)[:300])}
            torch.cuda.empty_cache()
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_rows or default_cpu_rows(args.workload))
        if "solve" in line:  # the same number of sigma products at the oracle's rate
            line["cpu_baseline"]["solve_seconds_extrapolated"] = \
                line["solve"]["sigma_applications"] / line["cpu_baseline"]["value"]
        line["cpu_baseline_1thread"] = cpu_baseline_one_thread(args.workload, 2000)
    return line


def run_solve(args, rank, world, local_rank, steps=None, warmup=None, e2e_steps=None,
              with_cpu=True):
    """The whole path per step on one workload: filter the raw strings,
    build the tables, Davidson to convergence.  Value: H.C applications per
    second over whole steps; e2e from pinned host buffers (raw strings and
    integrals in, energies out)."""
    env = Env(local_rank)
    torch, sqd, ctx = env.torch, env.sqd, env.ctx
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    w = si.workload(args.workload)
    opts = dict(SOLVE[args.workload])
    if getattr(args, "nroots", None):
        opts["nroots"] = args.nroots
    if args.max_subspace:
        opts["max_subspace"] = args.max_subspace
    if args.max_iter is not None:
        opts["max_iter"] = args.max_iter
        opts["raise_on_nonconvergence"] = False
    if args.correction != "davidson":
        opts["correction"] = args.correction
    raw_h = torch.from_numpy(w.raw_a.view(np.int64).copy()).pin_memory()
    h_h = torch.from_numpy(w.h.copy()).pin_memory()
    V_h = torch.from_numpy(w.V.copy()).pin_memory()
    raw_d, h_d, V_d = raw_h.to(env.dev), h_h.to(env.dev), V_h.to(env.dev)
    bytes_in = raw_h.numel() * 8 + h_h.numel() * 8 + V_h.numel() * 8

    def step(raw, h, V):
        t = env.tables(w, raw, h, V)
        if args.sigma_mode:
            t.set_sigma_mode(args.sigma_mode)
        if getattr(args, "spin_flip", 0):
            t.set_spin_flip(args.spin_flip)
        e, C, it, res, rc = sqd.davidson(ctx, t, **opts)
        t.close()
        del C
        return e, it, res

    for _ in range(warmup):
        step(raw_d, h_d, V_d)
    if world > 1:
        torch.distributed.barrier()
    env.sync()
    ctx.profile(True)
    clk = ClockSampler(local_rank).start()
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    results = [step(raw_d, h_d, V_d) for _ in range(steps)]
    ev1.record(env.stream)
    env.sync()
    _barrier()
    clocks = clk.stop()
    dev_ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    launches = ctx.launch_count()
    ctx.profile(False)
    hc = prof["same_spin_alpha"]["regions"]  # one region per sigma of one vector
    n_e2e = e2e_steps if e2e_steps is not None else (
        args.e2e_steps if args.e2e_steps is not None else max(1, min(steps, 2)))
    e2e_s = 0.0
    if n_e2e:
        env.sync()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            step(raw_h.to(env.dev, non_blocking=True), h_h.to(env.dev, non_blocking=True),
                 V_h.to(env.dev, non_blocking=True))  # energies come back to the host
        env.sync()
        e2e_s = time.perf_counter() - t0
    t_max, e2e_max, hc_tot = aggregate_replicas(dev_ms, e2e_s, hc, world, env.dev)
    env.close()
    if rank != 0:
        return None
    sig = sigma_summary(prof)
    value = hc_tot / (t_max / 1e3)
    out = {
        "mode": "solve", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": t_max / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "config": {"workload": DESCR[args.workload], "davidson": opts,
                   "step": "build_strings + excitation_tables + davidson",
                   "l2": "vectors may fit in L2" if w.ndet * 8 < 129e6 else
                   "inputs larger than L2",
                   "sigma_mode": "double-float (FP32 pipe)" if args.sigma_mode else "fp64"},
        "time_to_converged_E_s": t_max / 1e3 / steps,
        "davidson_iterations": int(results[-1][1]), "energy": float(results[-1][0][0]),
        "sigma_per_step": hc / steps, "det_per_s": value * w.ndet,
        "sigma_fp64_tflops": sig["fp64_tflops"], "sigma_share_of_step": sig["ms"] / dev_ms,
        "sigma_bound": sig["bound"], "hbm_roofline": sig["hbm_roofline"],
        "roofline": sigma_roofline(prof, args.workload),
        "tables_ms_per_step": (prof["tables"]["ms"] + prof["strings"]["ms"]) / steps,
        "davidson_classes": class_record(prof, DAVIDSON_CLASSES),
        "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
        "e2e": {"value": hc / steps * n_e2e * world / e2e_max, "unit": UNIT, "steps": n_e2e,
                "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": 8 * opts["nroots"]}
        if n_e2e else None,
        "clocks": clocks, "gpu_launches": launches}
    if with_cpu and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_rows or default_cpu_rows(args.workload))
        # the oracle's Davidson is its sigma products plus O(N m) vector work:
        # the same number of products at the oracle's rate
        out["cpu_baseline"]["solve_seconds_extrapolated"] = (hc / steps) / \
            out["cpu_baseline"]["value"]
        rows_1t = max(1000, (args.cpu_rows or default_cpu_rows(args.workload)) // 100)
        out["cpu_baseline_1thread"] = cpu_baseline_one_thread(
            args.workload, w.ndet if w.ndet <= 10000 else rows_1t)
    return out


def run_sigma_only(args, rank, world, local_rank):
    """One sigma = H C per step on tables built before the timed region (the
    kernel-only line; --stored applies the stored matrix instead)."""
    env = Env(local_rank)
    torch, sqd, ctx = env.torch, env.sqd, env.ctx
    w = si.workload(args.workload)
    t = env.tables(w)
    C = env.tensor(si.random_vectors(1, w.ndet, 13).reshape(w.strings_a.size, w.strings_b.size))
    sflip = getattr(args, "spin_flip", 0)
    if sflip:  # a vector of the sector
        C = C + sflip * C.T
        t.set_spin_flip(sflip)
    S = torch.empty_like(C)
    if getattr(args, "sigma_mode", 0):
        t.set_sigma_mode(args.sigma_mode)
    apply = sqd.sigma
    if getattr(args, "stored", False):
        sqd.stored_h_build(ctx, t)
        apply = sqd.sigma_stored
    for _ in range(args.warmup):
        apply(ctx, t, C, S)
    env.sync()
    _barrier()
    ctx.profile(True)
    clk = ClockSampler(local_rank).start()
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    for _ in range(args.steps):
        apply(ctx, t, C, S)
    ev1.record(env.stream)
    env.sync()
    _barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    launches = ctx.launch_count()
    info = t.info()
    t.close()
    env.close()
    if rank != 0:
        return None
    out = {"mode": "sigma", "sigma_mode": getattr(args, "sigma_mode", 0),
           "spin_flip": getattr(args, "spin_flip", 0), "metric": METRIC,
           "value": args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "dtype": "f64",
           "config": {"workload": DESCR[args.workload]}, "tables": info,
           "kernels": class_record(prof, SIGMA_CLASSES),
           "transpose_ms": prof["transpose"]["ms"] / max(1, args.steps),
           "clocks": clocks, "gpu_launches": launches}
    if getattr(args, "stored", False):
        st = prof["stored"]
        gbs = st["bytes"] / (st["ms"] / 1e3) / 1e9
        out["stored"] = {"ms_per_launch": st["ms"] / max(1, st["regions"]),
                         "bytes_per_launch": st["bytes"] / max(1, st["regions"]),
                         "achieved_gbs": gbs, "frac_hbm_peak": gbs / _hbm_peak(),
                         "peak_source": _hbm_peak_source(),
                         "tflops": st["flops"] / (st["ms"] / 1e3) / 1e12}
    return out


def run_batched(args, rank, world, local_rank, with_cpu=True):
    """Many independent subspaces (29 orbitals, 5+5 electrons, 200-3000
    strings each, one Hamiltonian): a step builds every subspace's tables and
    solves all ground states with sqd_davidson_batched; the comparison is one
    sqd_davidson per subspace on the same tables."""
    env = Env(local_rank)
    torch, sqd, ctx = env.torch, env.sqd, env.ctx
    subs = si.batched_workload(nbatch=args.nbatch)
    h = env.tensor(subs[0].h)
    V = env.tensor(subs[0].V)
    raws = [env.tensor(w.raw_a.view(np.int64)) for w in subs]
    tol_r = getattr(args, "tol_residual", 1e-6)
    opts = dict(tol_residual=tol_r, tol_energy=1e-8, max_iter=400)

    def tables():
        return [env.tables(w, r, h, V) for w, r in zip(subs, raws)]

    def step():
        tabs = tables()
        e, Cs, it, st, rc = sqd.davidson_batched(ctx, tabs, want_vectors=False, **opts)
        for t in tabs:
            t.close()
        return e, it

    for _ in range(args.warmup):
        step()
    env.sync()
    ctx.profile(True)
    clk = ClockSampler(local_rank).start()
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    for _ in range(args.steps):
        e_b, it_b = step()
    ev1.record(env.stream)
    env.sync()
    clocks = clk.stop()
    ms_b = ev0.elapsed_time(ev1) / args.steps
    prof = ctx.profile_read()
    launches = ctx.launch_count()
    ctx.profile(False)
    scale, device_loop = sqd.batched_tuning(ctx, with_loop=True)
    buckets = sqd.batched_tuning_buckets(ctx)
    # the same work as one solve per subspace
    env.sync()
    ev0.record(env.stream)
    tabs = tables()
    e_s, it_s = [], []
    for t in tabs:
        e, C, it, res, rc = sqd.davidson(ctx, t, nroots=1, **opts)
        e_s.append(e[0])
        it_s.append(it)
        t.close()
    ev1.record(env.stream)
    env.sync()
    ms_s = ev0.elapsed_time(ev1)
    env.close()
    ndet = np.array([w.ndet for w in subs], dtype=np.float64)
    rows = float(np.sum(ndet * (np.asarray(it_b) + 1)))
    out = {"mode": "batched", "metric": "sigma determinant rows per second over the batched "
                                        "solve (sum over subspaces of N_b x sigma applications)",
           "value": rows / (ms_b / 1e3), "unit": "det rows of sigma/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
           "higher_is_better": True, "dtype": "f64",
           "config": {"workload": "%d subspaces, norb=29, 5+5 electrons, 200-3000 strings each "
                                  "(%.3g determinants in total), ground states, ||r|| <= %g, "
                                  "|dE| <= 1e-8; step = tables + batched solve"
                                  % (len(subs), float(np.sum(ndet)), tol_r)},
           "sequential_ms": ms_s, "speedup_vs_sequential": ms_s / ms_b,
           "max_abs_energy_diff_vs_sequential": float(np.max(np.abs(np.asarray(e_b) - e_s))),
           "iterations_batched_max": int(np.max(it_b)), "iterations_sequential_max": int(max(it_s)),
           "iterations_batched_sum": int(np.sum(it_b)), "iterations_sequential_sum": int(sum(it_s)),
           "max_rel_energy_diff_vs_sequential":
               float(np.max(np.abs(np.asarray(e_b) - e_s) / np.abs(e_s))),
           "autotuned_group_scale": scale, "autotuned_buckets": buckets,
           "det_total": float(np.sum(ndet)),
           "loop_in_one_graph": device_loop,
           "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items() if v["ms"]},
           "classes": class_record(prof, [k for k in ("batched", "batched_sigma",
                                                      "batched_sigma_ab", "batched_vector",
                                                      "batched_eigh")
                                          if k in prof]),
           "roofline": batched_roofline(prof),
           "clocks": clocks, "gpu_launches": launches}
    if with_cpu and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batched(subs, it_b)
    return out


def batched_roofline(prof):
    """The batched loop against its two roofs: the sigma stage's algorithmic
    flops over its device-timed stage time against the FP64 peak, the vector
    stages' algorithmic bytes against the HBM copy bandwidth, and the loop
    as a whole: (sigma flops / FP64 peak + vector bytes / HBM) over the time
    of the three stages."""
    if "batched_sigma" not in prof or not prof["batched_sigma"]["ms"]:
        return None
    sg, vc, eg = prof["batched_sigma"], prof["batched_vector"], prof["batched_eigh"]
    t_roof = sg["flops"] / (FP64_PEAK_TFLOPS * 1e12) + vc["bytes"] / (_hbm_peak() * 1e9)
    t_loop = (sg["ms"] + vc["ms"] + eg["ms"]) / 1e3
    return {"sigma_frac_fp64": sg["flops"] / (sg["ms"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
            "vector_frac_hbm": vc["bytes"] / (vc["ms"] / 1e3) / 1e9 / _hbm_peak()
            if vc["ms"] else None,
            "loop_frac": t_roof / t_loop if t_loop else None,
            "loop_ms": t_loop * 1e3, "eigh_ms": eg["ms"],
            "note": "sigma of measured-derived FP64 peak; vector of measured HBM copy "
                    "bandwidth; loop = roof time / stage time"}


def run_adjoint(args, rank, world, local_rank, with_cpu=True):
    """Backward pass of E(h, V) on a converged ground state: one step is the
    spin-summed 1-RDM and 2-RDM of C (dE/dh, 2 dE/dV) plus the orbital
    gradient, timed against one sigma = H C on the same tables."""
    env = Env(local_rank)
    torch, sqd, ctx = env.torch, env.sqd, env.ctx
    name = args.workload if args.workload in ("adjoint29",) else "adjoint29"
    w = si.workload(name)
    t = env.tables(w)
    ev0, ev1 = env.events()
    ev0.record(env.stream)
    e, X, iters, res, rc = sqd.davidson(ctx, t, **SOLVE[name])
    ev1.record(env.stream)
    env.sync()
    solve_ms = ev0.elapsed_time(ev1)
    C = X[0].contiguous()
    S = torch.empty_like(C)

    def backward():
        g1, g2 = sqd.rdm(ctx, t, C)
        return sqd.orbital_gradient(ctx, t, g1, g2)

    def timed(fn, profile=False):
        for _ in range(args.warmup):
            fn()
        env.sync()
        if profile:
            ctx.profile(True)
        ev0.record(env.stream)
        for _ in range(args.steps):
            fn()
        ev1.record(env.stream)
        env.sync()
        return ev0.elapsed_time(ev1) / args.steps

    clk = ClockSampler(local_rank).start()
    sigma_ms = timed(lambda: sqd.sigma(ctx, t, C, S))
    back_ms = timed(backward, profile=True)
    prof = ctx.profile_read()
    clocks = clk.stop()
    launches = ctx.launch_count()
    info = t.info()
    t.close()
    env.close()
    if rank != 0:
        return None
    out = {"mode": "adjoint", "metric": METRIC,
           "value": 1e3 / back_ms, "unit": "backward passes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": back_ms,
           "higher_is_better": True, "dtype": "f64",
           "config": {"workload": DESCR[name] + "; backward = 1-RDM + 2-RDM + orbital gradient"},
           "tables": info, "backward_ms": back_ms, "sigma_ms": sigma_ms,
           "backward_over_sigma": back_ms / sigma_ms, "target_backward_over_sigma": 3.0,
           "forward_solve_ms": solve_ms, "forward_iterations": int(iters),
           "energy": float(e[0]), "rdm_kernel_ms": prof["rdm"]["ms"] / max(1, args.steps),
           "clocks": clocks, "gpu_launches": launches}
    if with_cpu and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_adjoint(w, int(iters))
    return out


# --------------------------------------------- sub-records of the headline --

def _sub_args(args, **kw):
    a = argparse.Namespace(**vars(args))
    a.sigma_mode, a.stored, a.max_iter, a.max_subspace = 0, False, None, None
    a.correction, a.cpu_rows, a.e2e_steps, a.nroots = "davidson", None, None, None
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def sub_h2o29(args, local_rank):
    """The 8-root h2o29 solve, whole path per step, with its oracle baselines."""
    a = _sub_args(args, workload="h2o29", steps=2, warmup=1)
    r = run_solve(a, 0, 1, local_rank, e2e_steps=1)
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "time_to_converged_E_s",
            "davidson_iterations", "energy", "det_per_s", "sigma_fp64_tflops",
            "sigma_share_of_step", "sigma_bound", "roofline", "davidson_classes", "kernel_ms",
            "e2e", "clocks", "cpu_baseline", "cpu_baseline_1thread", "config")
    return {k: r[k] for k in keep if k in r}


def oracle_solve(name):
    """The whole oracle solve of a small workload on the host cores: the
    diagonal, then the oracle's Davidson with its matrix-free sigma, under
    the same options as the device solve."""
    import oracle
    w = si.workload(name)
    o = SOLVE[name]
    t0 = time.perf_counter()
    hd = oracle.diag(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b)
    th, _, it, _, conv = oracle.davidson(
        lambda X: oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, X.T).T, hd,
        nroots=o["nroots"], tol_residual=o["tol_residual"], tol_energy=o["tol_energy"],
        max_iter=o["max_iter"])
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": _cores(), "kind": "oracle",
            "sample": "the whole oracle solve of %s (diagonal + Davidson, %d iterations), "
                      "not extrapolated" % (name, int(it)),
            "seconds": dt, "energies": [float(x) for x in th], "converged": bool(conv)}


def oracle_solve_one_thread(name):
    """oracle_solve on one host thread (a child process with OMP_NUM_THREADS=1)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_solve(%r)))" % (ROOT, name))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                             text=True, timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as exc:  # reported, not fatal
        return {"error": str(exc)[:200]}


def sub_full8(args, local_rank):
    """The 4900-determinant full space (8 orbitals, 4+4 electrons): the whole
    device path per step against the whole oracle solve, on all host cores
    and on one thread."""
    a = _sub_args(args, workload="full8", steps=20, warmup=3)
    r = run_solve(a, 0, 1, local_rank, e2e_steps=5)
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "time_to_converged_E_s",
            "davidson_iterations", "energy", "e2e", "clocks", "cpu_baseline",
            "cpu_baseline_1thread", "config")
    out = {k: r[k] for k in keep if k in r}
    if not args.no_cpu_baseline:
        so = oracle_solve("full8")
        out["cpu_baseline_solve"] = so
        out["cpu_baseline_solve_1thread"] = oracle_solve_one_thread("full8")
        out["abs_energy_diff_vs_oracle"] = abs(float(r["energy"]) - so["energies"][0])
        out["solve_speedup_vs_oracle"] = so["seconds"] / (r["ms_per_step"] / 1e3)
    return out


# spin-flip sector of the singlets: with the alpha-first determinant
# ordering a state of total spin S has C^T = (-1)^S C
SINGLET_SECTOR = 1


def sub_spin_flip(args, local_rank, e_general=None):
    """The default workload in the singlet spin-flip sector (C^T = C, one
    same-spin pass per sigma): sigma steps on a vector of the sector, then
    the lowest singlet-sector state, its energy beside the general solve's
    (equal when the ground state is a singlet)."""
    env = Env(local_rank)
    torch = env.torch
    w = si.workload(args.workload)
    sector = SINGLET_SECTOR
    t = env.tables(w)
    t.set_spin_flip(sector)
    n = w.strings_a.size
    C = env.tensor(si.random_vectors(1, w.ndet, 13).reshape(n, n))
    C = C + sector * C.T
    S = torch.empty_like(C)
    steps = max(3, min(args.steps, 10))
    dev_ms, prof, launches, clocks = sigma_steps(env, t, C, S, steps, 2)
    del C, S
    torch.cuda.empty_cache()
    sig = sigma_summary(prof)
    out = {"sector": sector, "value": steps / (dev_ms / 1e3), "unit": UNIT,
           "ms_per_step": dev_ms / steps, "steps": steps,
           "note": "sigma = T + s T^T + H_II C + sigma_ab on vectors with C^T = s C: one "
                   "same-spin pass; the general line forms both",
           "sigma_bound": sig["bound"], "roofline": sigma_roofline(prof, args.workload),
           "kernels": class_record(prof, SIGMA_CLASSES), "clocks": clocks,
           "gpu_launches": launches}
    # the recorded DRAM traffic is that of the general kernels, not of these
    out["roofline"]["traffic"] = None
    if not args.no_solve:
        sr = solve_record(env, t, dict(SOLVE[args.workload]), args.workload)
        out["time_to_converged_E_s"] = sr["time_to_converged_E_s"]
        out["davidson_iterations"] = sr["iterations"]
        out["energy"] = sr["energies"][0]
        out["residual"] = sr["residuals"][0]
        out["solve"] = sr
        if e_general is not None:
            out["abs_energy_diff_vs_general_solve"] = abs(sr["energies"][0] - e_general)
    t.close()
    env.close()
    return out


def sub_batched(args, local_rank):
    a = _sub_args(args, steps=1, warmup=0, nbatch=64)
    r = run_batched(a, 0, 1, local_rank)
    r.pop("metric", None)
    return r


def sub_adjoint(args, local_rank):
    a = _sub_args(args, workload="adjoint29", steps=3, warmup=1)
    r = run_adjoint(a, 0, 1, local_rank)
    r.pop("metric", None)
    return r


def sub_stored(args, local_rank):
    a = _sub_args(args, workload="h2o29", steps=5, warmup=2, stored=True)
    r = run_sigma_only(a, 0, 1, local_rank)
    return {"workload": DESCR["h2o29"], "stored": r["stored"],
            "ms_per_step": r["ms_per_step"], "clocks": r["clocks"]}


# ------------------------------------------------------- reference -------

def run_reference(args, rank, world):
    """The oracle as it stands on the host cores: each step one bounded
    sample of sigma rows of the same workload, H.C/s extrapolated."""
    if rank != 0:
        return None
    w = si.workload(args.workload)
    rows_n = args.cpu_rows or max(1000, default_cpu_rows(args.workload) // 4)
    for _ in range(args.warmup):
        cpu_baseline(w, max(1000, rows_n // 10))
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_baseline(w, rows_n)
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = float(np.mean(vals))
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": DESCR[args.workload],
                                            "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = _args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.mode == "sigma":
        line = run_sigma_only(args, rank, world, local_rank)
    elif args.mode == "solve":
        line = run_solve(args, rank, world, local_rank)
    elif args.mode == "batched":
        line = run_batched(args, rank, world, local_rank)
    elif args.mode == "adjoint":
        line = run_adjoint(args, rank, world, local_rank)
    else:
        line = headline(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
