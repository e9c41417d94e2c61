#!/usr/bin/env python
"""Throughput of the FWI hot path on GB300: one step = one full misfit-gradient
evaluation (forward sweep with receiver sampling, checkpoint encodes, L2 misfit,
checkpointed reverse sweep with recomputation, adjoint steps with zero-lag imaging,
FP64 gradient fold and finish) of a 3-D shot, through the library's C ABI.

Metric: Gpts/s fwd+adjoint = computed grid points x time steps x shots / step time.
Default workload: the 512^3 salt model (h 12.5 m, dt 0.6 ms, 4000 steps, 16th order,
20-cell sponge, 256 x 256 receivers, FP16 checkpoints).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

With N > 1 (torchrun) every rank runs an independent replica of the workload (shots
are independent units; the library has no multi-GPU path) and rank 0 prints one JSON
line with the whole-job rate.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload (rank 0 only).

Besides the contract's keys the line carries: ``roofline.kernels`` (each 3-D step
instantiation's launches, average CUDA-event time, algorithmic bytes per point, achieved
GB/s, fraction of the measured peak and recorded DRAM traffic per launch; ``roofline``
itself is the one with the most device time, with ``min_frac`` (the slowest kernel) and
``time_weighted_frac`` (all step kernels' algorithmic bytes over their device time)
beside it), ``layered_3d_256`` (the 256^3 layered model at 8th order with BF16
checkpoints: gradient rate, each step kernel's GB/s, and the forward step's cost per
point and step at order 8 against the headline workload's order 16), ``onchip_2d``
(one-shot 2-D forward runs of the serving mix's kind at 128^2..384^2, single steps against
temporal blocking on chip), ``serving`` (a Poisson stream of mixed 2-D/3-D forward/gradient requests
through the continuous-batching loop against one request at a time: shots/s, p50/p99
latency) and ``batched_2d`` (64 shots of the 400 x 1024 faulted model in one gradient
call against 64 one-shot calls, with the step kernels' times, and the forward-only rate
with single steps and with two steps per pass).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
BYTES_FWD = 16     # read u^n, u^{n-1}, W; write u^{n+1} (per point)
BYTES_STORE = 18   # the forward step that also writes the FP16/BF16 checkpoint of u^n
BYTES_ADJ = 26     # reverse step + imaging: read mu^{m+1}, mu^{m+2}, W, g and u^m (as the
                   # 2-byte checkpoint code, read in place); write mu^m, g.  (28 with an
                   # FP32 u^m.)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="salt_3d_512",
                    choices=["salt_3d_512", "layered_3d_256"])
    ap.add_argument("--nt", type=int, default=0, help="override the step count (short runs)")
    ap.add_argument("--n", type=int, default=0,
                    help="grid size of a scaled twin of the workload (profiling runs)")
    ap.add_argument("--snap-budget-gb", type=float, default=224.0)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-layered", action="store_true")
    ap.add_argument("--layered-nt", type=int, default=2000,
                    help="time steps of the 256^3 layered section (shorter for profiling)")
    ap.add_argument("--serving-requests", type=int, default=32)
    ap.add_argument("--serving-rates", default="0.8",
                    help="comma-separated fractions of the batched capacity for Poisson arrivals")
    ap.add_argument("--batched-nt", type=int, default=3000,
                    help="time steps of the batched 2-D section (shorter for profiling)")
    return ap.parse_args()


def gpts_per_s(points, steps, seconds):
    """Grid points updated per second, in billions: the Gcells/s of the paper's Table 1
    (cells x steps / time)."""
    return points * steps / seconds / 1e9


def workload(name, nt_override, n=0):
    from paper_1912_08063_gb300 import synth
    if name == "salt_3d_512":
        w = synth.salt_3d(n or 512)
    else:
        w = synth.layered_3d(n or 256)
    if nt_override:
        w.nt = nt_override
    return w


STEP3D_SOURCES = ["k_step3d.cuh", "k_step3d_m8.cu", "k_step3d_m4.cu", "k_step3d.cu", "step3d.h",
                  "code16.cuh", "k_step3d_tm.cuh", "k_step3d_tm8.cu", "k_step3d_tm4.cu", "tmap.cpp"]


def kernel_source_hash():
    """Hash of the 3-D step kernel's sources: a recorded DRAM traffic figure is reported
    only while these are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1912_08063_gb300", "csrc")
    for f in STEP3D_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def recorded_traffic(kernel):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current
    kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        e = d[kernel]
        if e.get("source_hash") == kernel_source_hash():
            return float(e["bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, sample_n=320, sample_nt=30):
    """The FP64 oracle, as it stands, on a bounded sample: a centred sample_n^3 crop of
    the model (same spacing, order, sponge, dt), one misfit-gradient evaluation of
    sample_nt steps.  Returns (Gpts/s, seconds, description, threads)."""
    import oracle
    n = w.shape[0]
    sample_n = min(sample_n, n)
    sample_nt = min(sample_nt, w.nt)
    c0 = (n - sample_n) // 2
    sl = slice(c0, c0 + sample_n)
    v = np.ascontiguousarray(w.v[sl, sl, sl], dtype=np.float64)
    src = np.array([[10, sample_n // 2, sample_n // 2]], dtype=np.int32)
    rec = np.array([[5, j, i] for j in range(0, sample_n, 8) for i in range(0, sample_n, 8)],
                   dtype=np.int32)
    wav = w.wavelets()[:1, :sample_nt]
    p = oracle.Problem(v, w.h, w.dt, sample_nt, order=w.order, nb=w.nb, src=src, rec=rec,
                       wavelet=wav)
    dobs = np.zeros((1, sample_nt, rec.shape[0]))
    oracle.build()
    t0 = time.perf_counter()
    p.gradient(dobs, seg=max(1, int(round(np.sqrt(sample_nt)))))
    t = time.perf_counter() - t0
    pts = 1
    for s in p.computed_shape():
        pts *= s
    desc = (f"oracle misfit gradient on a centred {sample_n}^3 crop of the {n}^3 model "
            f"({pts / 1e6:.1f} M computed points incl. sponge, order {w.order}, "
            f"{sample_nt} steps); Gpts/s = points x steps / wall time")
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return pts * sample_nt / t / 1e9, t, desc, threads


def cpu_baseline_one_core(args, sample_n=160, sample_nt=10):
    """The oracle on one host core (OMP_NUM_THREADS=1, in a child process so the
    OpenMP runtime of this one is untouched), on a smaller crop.  Returns a dict or
    None."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "w = bench.workload(%r, %d, %d); "
            "g, t, desc, thr = bench.cpu_baseline(w, %d, %d); "
            "print(json.dumps({'value': g, 'seconds': t, 'sample': desc, 'cores': thr}))"
            % (ROOT, args.workload, args.nt, args.n, sample_n, sample_nt))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                             text=True, timeout=300, check=True).stdout
        d = json.loads(out.strip().splitlines()[-1])
        return {"value": d["value"], "unit": "Gpts/s", "cores": d["cores"],
                "sample": d["sample"], "seconds": round(d["seconds"], 2)}
    except Exception:
        return None


def serving_section(dev, n_req, seed=4, rates=(0.8,)):
    """Serving workload (Poisson stream of forward/gradient requests, 75 % 2-D / 25 % 3-D,
    sides 128..1024 / 64..192, nt 500..3000): closed-loop capacity with continuous batching
    and one request at a time, then Poisson arrivals at 0.8 x the batched capacity (both
    ways), and at each further fraction in `rates` (batched only)."""
    import math

    import torch

    from paper_1912_08063_gb300 import fwi, synth

    def dt_for(ndim, h):
        lim = 1.0 / fwi.fwi_cfl_number(ndim, 8, (h, h, h), 4500.0, 1.0)
        return math.floor(0.8 * lim * 1e4) / 1e4

    reqs = synth.serving_requests(n_req, dt_for, seed=seed)
    for r in reqs:   # observed traces of gradient requests, before any timing
        if r["kind"] == "gradient":
            m = fwi.FwiModel(torch.from_numpy(r["v_obs"]).to(dev), r["h"], r["dt"], r["nt"])
            acq = fwi.Acquisition([r["src"]], r["rec"])
            r["d_obs"] = m.forward(acq, torch.from_numpy(r["wavelet"][None]).to(dev))[0].cpu().numpy()
            m.close()
    torch.cuda.synchronize()

    def run(max_active, arrivals, shared=True):
        for r, a in zip(reqs, arrivals):
            r["arrival"] = float(a)
        t0 = time.perf_counter()
        res, _ = fwi.fwi_serve(reqs, max_active=max_active, steps_per_turn=16, snap_slots=64,
                               shared_launch=shared)
        wall = time.perf_counter() - t0
        lat = np.array([x["t_done"] - a for x, a in zip(res, arrivals)])
        ok = sum(1 for x in res if x["status"] == 0)
        run.shared = (sum(1 for x in res if x["shared_launch"] == 1),
                      sum(1 for x in res if x["shared_launch"] == 2))
        return ok / wall, lat, ok

    zero = np.zeros(n_req)
    cap_ns, _, _ = run(16, zero, shared=False)
    cap_b, _, ok_b = run(16, zero)
    n_shared = run.shared
    cap_1, _, ok_1 = run(1, zero)
    lam = 0.8 * cap_b
    rng = np.random.default_rng(seed)
    arr = np.cumsum(rng.exponential(1.0 / lam, n_req))
    _, lat_b, _ = run(16, arr)
    _, lat_1, _ = run(1, arr)
    sweep = []
    for f in rates:
        if abs(f - 0.8) < 1e-9:
            lat, ok = lat_b, ok_b
        else:
            arr_f = np.cumsum(np.random.default_rng(seed).exponential(1.0 / (f * cap_b), n_req))
            _, lat, ok = run(16, arr_f)
        sweep.append({"rate_fraction": f, "rate_per_s": round(f * cap_b, 3), "completed": ok,
                      "p50_s": round(float(np.percentile(lat, 50)), 3),
                      "p99_s": round(float(np.percentile(lat, 99)), 3)})
    return {"requests": n_req, "completed": [ok_b, ok_1], "load_sweep": sweep,
            "shots_per_s": round(cap_b, 3), "shots_per_s_one_at_a_time": round(cap_1, 3),
            "shots_per_s_without_shared_launch": round(cap_ns, 3),
            "requests_in_shared_launch": {"multi_request_steps": n_shared[0],
                                          "cluster_on_chip": n_shared[1]},
            "poisson_rate_per_s": round(lam, 3),
            "p50_s": round(float(np.percentile(lat_b, 50)), 3),
            "p99_s": round(float(np.percentile(lat_b, 99)), 3),
            "p50_s_one_at_a_time": round(float(np.percentile(lat_1, 50)), 3),
            "p99_s_one_at_a_time": round(float(np.percentile(lat_1, 99)), 3),
            "workload": "serving mix: 75 % 2-D (128..1024)^2, 25 % 3-D (64..192)^3, nt 500..3000, "
                        "half forward / half gradient (BF16 checkpoints), 8th order"}


def batched_section(dev, nt=3000, budget_gb=224.0):
    """64 shots of the 400 x 1024 faulted 2-D model: one batched gradient call (shots on
    the grid's z launch dimension, FP64 gradient sum over shots) against 64 one-shot
    calls of the same kernels.  With the default checkpoint budget every step's u^n fits
    (BF16 checkpoints of 60 MB, 180 GB for 3000 steps), so the forward recursion runs
    once."""
    import torch

    from paper_1912_08063_gb300 import fwi, synth

    w = synth.faulted_2d(nt=nt)
    acq = fwi.Acquisition(w.src, w.rec)
    wav = torch.from_numpy(w.wavelets()).to(dev)
    obs = fwi.FwiModel(torch.from_numpy(w.v_obs).to(dev), w.h, w.dt, w.nt, order=w.order,
                       sponge_vref=4500.0)
    dobs = obs.forward(acq, wav)
    obs.close()
    m = fwi.FwiModel(torch.from_numpy(w.v).to(dev), w.h, w.dt, w.nt, order=w.order,
                     snap_dtype=w.snap_dtype, snap_budget_bytes=int(budget_gb * 2 ** 30),
                     sponge_vref=4500.0,
                     timing=True)
    m.gradient(acq, wav, dobs)   # warm-up
    torch.cuda.synchronize()
    i0 = m.info()
    t0 = time.perf_counter()
    phi, g = m.gradient(acq, wav, dobs)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    i1 = m.info()
    nf = i1["fwd_step_launches"] - i0["fwd_step_launches"]
    nst = i1["store_step_launches"] - i0["store_step_launches"]
    na = i1["adj_step_launches"] - i0["adj_step_launches"]
    fms = (i1["fwd_step_ms"] - i0["fwd_step_ms"]) / max(nf, 1)
    sms = (i1["store_step_ms"] - i0["store_step_ms"]) / max(nst, 1)
    ams = (i1["adj_step_ms"] - i0["adj_step_ms"]) / max(na, 1)
    # W is one field shared by all shots: per point and step the forward step moves
    # 12 + 4 / shots bytes, with a checkpoint store 2 more (u^n alone as a 16-bit code),
    # the reverse step 22 + 4 / shots (u^m as a 2-byte code)
    bf = 12.0 + 4.0 / w.nshots
    bs = bf + 2.0
    ba = BYTES_ADJ - 4.0 + 4.0 / w.nshots
    npts = i1["points"] * w.nshots
    kern = {"fwd_step_avg_ms": round(fms, 4), "fwd_step_launches": nf,
            "fwd_bytes_per_point": round(bf, 3),
            "fwd_step_GB/s": round(bf * npts / (fms * 1e-3) / 1e9, 1),
            "store_step_avg_ms": round(sms, 4), "store_step_launches": nst,
            "store_bytes_per_point": round(bs, 3),
            "store_step_GB/s": round(bs * npts / (sms * 1e-3) / 1e9, 1) if nst else None,
            "adj_step_avg_ms": round(ams, 4), "adj_step_launches": na,
            "adj_bytes_per_point": round(ba, 3),
            "adj_step_GB/s": round(ba * npts / (ams * 1e-3) / 1e9, 1),
            "kernel_seconds": round((nf * fms + nst * sms + na * ams) / 1e3, 3)}
    singles = [fwi.Acquisition(w.src[i:i + 1], w.rec) for i in range(w.nshots)]
    t0 = time.perf_counter()
    for i, a in enumerate(singles):
        m.gradient(a, wav[i:i + 1], dobs[i:i + 1])
    torch.cuda.synchronize()
    t1 = time.perf_counter() - t0
    pts = m.info()["points"]
    m.close()
    # forward only, the same 64 shots: single steps against two steps per pass (temporal
    # blocking, fwi_opts.temporal_blocking)
    fwd = {}
    for tbk in (False, True):
        mf = fwi.FwiModel(torch.from_numpy(w.v).to(dev), w.h, w.dt, w.nt, order=w.order,
                          sponge_vref=4500.0, temporal_blocking=tbk)
        mf.forward(acq, wav)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mf.forward(acq, wav)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        mf.close()
        key = "two_step_pass" if tbk else "single_step"
        fwd[key] = {"seconds": round(tf, 4),
                    "gpts_per_s": round(gpts_per_s(pts * w.nshots, w.nt, tf), 2)}
    return {"workload": w.name, "shots": w.nshots, "nt": w.nt, "forward_only": fwd,
            "checkpoint_slots": i1["snap_slots"],
            "forward_steps_per_gradient": i1["last_forward_steps"],
            "shots_per_s": round(w.nshots / tb, 3),
            "shots_per_s_per_shot_calls": round(w.nshots / t1, 3),
            "gpts_per_s": round(gpts_per_s(pts * w.nshots, w.nt, tb), 2),
            "seconds": round(tb, 3), "seconds_per_shot_calls": round(t1, 3), "kernels": kern}


def kernel_stats(info0, info1, npts, peak, traffic=True):
    """Per 3-D step instantiation between two fwi_model_info snapshots: launches, average
    CUDA-event time, algorithmic bytes per point, achieved GB/s and its fraction of the
    peak; plus the minimum fraction and the time-weighted one (all kernels' algorithmic
    bytes over their summed device time)."""
    kern = {}
    tot_bytes = tot_s = 0.0
    for key, nkey, mkey, bpp in (("fwd_step_3d", "fwd_step_launches", "fwd_step_ms", BYTES_FWD),
                                 ("store_step_3d", "store_step_launches", "store_step_ms", BYTES_STORE),
                                 ("adj_step_3d", "adj_step_launches", "adj_step_ms", BYTES_ADJ)):
        n = info1[nkey] - info0[nkey]
        tot = info1[mkey] - info0[mkey]
        avg = tot / n if n else 0.0
        gbs = bpp * npts / (avg * 1e-3) / 1e9 if n else None
        kern[key] = {"launches": n, "total_ms": tot, "avg_ms": avg, "bytes_per_point": bpp,
                     "GB/s": gbs, "frac": round(gbs / peak, 4) if n else None,
                     "traffic": recorded_traffic(key) if traffic else None}
        if n:
            tot_bytes += bpp * npts * n
            tot_s += tot * 1e-3
    fr = [k["frac"] for k in kern.values() if k["frac"] is not None]
    summary = {"min_frac": min(fr) if fr else None,
               "time_weighted_frac": round(tot_bytes / tot_s / 1e9 / peak, 4) if tot_s else None}
    return kern, summary


def layered_section(dev, nt=2000, budget_gb=224.0, peak=None, k1_order16=None):
    """The 256^3 layered model with Gaussian random perturbations (8th order, dt 0.8 ms,
    BF16 checkpoints, 128 x 128 receivers): one misfit gradient, timed after a warm-up,
    with each step kernel's achieved bandwidth; then the forward step alone, whose cost
    per point and step sets, against the 16th-order step of the headline workload, the
    GPU side of the order trade-off (Sec. 4, Fig. 6)."""
    import torch

    from paper_1912_08063_gb300 import fwi

    w = workload("layered_3d_256", nt)
    acq = fwi.Acquisition(w.src, w.rec)
    wav = torch.from_numpy(w.wavelets()).to(dev)
    obs = fwi.FwiModel(torch.from_numpy(w.v_obs).to(dev), w.h, w.dt, w.nt, order=w.order,
                       nb=w.nb, sponge_vref=4500.0)
    dobs = obs.forward(acq, wav)
    obs.close()
    m = fwi.FwiModel(torch.from_numpy(w.v).to(dev), w.h, w.dt, w.nt, order=w.order, nb=w.nb,
                     snap_dtype=w.snap_dtype, snap_budget_bytes=int(budget_gb * 2 ** 30),
                     sponge_vref=4500.0, timing=True)
    m.gradient(acq, wav, dobs)   # warm-up
    torch.cuda.synchronize()
    i0 = m.info()
    t0 = time.perf_counter()
    m.gradient(acq, wav, dobs)
    torch.cuda.synchronize()
    tg = time.perf_counter() - t0
    i1 = m.info()
    pts = i1["points"]
    kern, summ = kernel_stats(i0, i1, pts * w.nshots, peak, traffic=False)
    # forward only: the plain step's cost per point and step at order 8
    i2 = m.info()
    m.forward(acq, wav)
    torch.cuda.synchronize()
    i3 = m.info()
    m.close()
    nf = i3["fwd_step_launches"] - i2["fwd_step_launches"]
    f_ms = (i3["fwd_step_ms"] - i2["fwd_step_ms"]) / max(nf, 1)
    ps8 = f_ms * 1e9 / (pts * w.nshots)
    trade = {"fwd_ps_per_point_step_order8": round(ps8, 4)}
    if k1_order16:
        ms16, pts16 = k1_order16
        ps16 = ms16 * 1e9 / pts16
        trade.update({"fwd_ps_per_point_step_order16": round(ps16, 4),
                      "order16_over_order8": round(ps16 / ps8, 4)})
    return {"workload": w.name, "grid": list(w.shape), "computed_points": pts,
            "order": w.order, "nt": w.nt, "checkpoints": w.snap_dtype,
            "checkpoint_slots": i1["snap_slots"],
            "forward_steps_per_gradient": i1["last_forward_steps"],
            "step_ctas_fwd_adj_store": i1["step_ctas"],
            "seconds": round(tg, 4), "gpts_per_s": round(gpts_per_s(pts * w.nshots, w.nt, tg), 2),
            "kernels": kern, **summ, "order_tradeoff": trade}


def onchip_section(dev, sizes=(128, 256, 384), nt=1500):
    """One-shot 2-D forward runs of the serving mix's kind (smooth model 1500..4500 m/s,
    h 10 m, dt at 0.8 of the stability limit, source and receivers on surface row 2),
    timed with single steps and with temporal blocking on chip (fwi_opts.temporal_blocking
    = 2: up to 64 steps per launch, both states in the shared memory of one cluster of
    CTAs).  Best of three runs each."""
    import math

    import torch

    from paper_1912_08063_gb300 import fwi, synth

    rng = np.random.default_rng(3)
    out = {}
    for n in sizes:
        v = synth.smooth_random(rng, (n, n), 10.0, ell=300.0)
        v = (1500.0 + 3000.0 * (v - v.min()) / (v.max() - v.min())).astype(np.float32)
        h = 10.0
        dt = math.floor(0.8 / fwi.fwi_cfl_number(2, 8, (h, h, h), 4500.0, 1.0) * 1e4) / 1e4
        acq = fwi.Acquisition(np.array([[2, 0, n // 2]], dtype=np.int32),
                              np.array([[2, 0, x] for x in range(n)], dtype=np.int32))
        wav = torch.from_numpy(synth.ricker(15.0, dt, nt)[None].astype(np.float32)).to(dev)
        res = {}
        for tb in (0, 2):
            m = fwi.FwiModel(torch.from_numpy(v).to(dev), h, dt, nt, temporal_blocking=tb)
            m.forward(acq, wav)
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                m.forward(acq, wav)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            res["single_step_ms" if tb == 0 else "on_chip_ms"] = round(min(ts) * 1e3, 3)
            m.close()
        res["speedup"] = round(res["single_step_ms"] / res["on_chip_ms"], 2)
        out[f"{n}x{n}"] = res
    return {"nt": nt, "runs": out}


def replica_rate(ms_local, units_local, world, dist=None, device="cpu"):
    """Whole-job timing of N independent replicas: the step time is the maximum over
    ranks, the rate the units all ranks processed per second of that time.  Returns
    (ms, units per second); without a process group (world 1) the local values."""
    import torch
    t = torch.tensor([float(ms_local), float(units_local)], dtype=torch.float64, device=device)
    if world > 1:
        tmax = t[:1].clone()
        tsum = t[1:].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        t = torch.cat([tmax, tsum])
    ms, units = float(t[0].item()), float(t[1].item())
    return ms, units / (ms * 1e-3)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload, args.nt, args.n)
    vals = []
    for i in range(args.warmup + args.steps):
        g, t, desc, threads = cpu_baseline(w)
        if i >= args.warmup:
            vals.append((g, t))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(t for _, t in vals) * 1e3
    line = {"impl": "reference", "metric": "Gpts/s fwd+adjoint", "value": value,
            "unit": "Gpts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "note": "bounded CPU sample, see cpu_baseline"},
            "cpu_baseline": {"value": value, "unit": "Gpts/s", "cores": threads,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from paper_1912_08063_gb300 import fwi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload(args.workload, args.nt, args.n)
    dev = torch.device("cuda", local)
    budget = int(args.snap_budget_gb * (1 << 30))
    model = fwi.FwiModel(torch.from_numpy(w.v).to(dev), w.h, w.dt, w.nt, order=w.order,
                         nb=w.nb, snap_dtype=w.snap_dtype, snap_budget_bytes=budget,
                         sponge_vref=4500.0, timing=True)
    acq = fwi.Acquisition(w.src, w.rec)
    wav = torch.from_numpy(w.wavelets()).to(dev)
    # observed data from the perturbed model (input synthesis, untimed)
    obs_model = fwi.FwiModel(torch.from_numpy(w.v_obs).to(dev), w.h, w.dt, w.nt,
                             order=w.order, nb=w.nb, sponge_vref=4500.0)
    dobs = obs_model.forward(acq, wav)
    obs_model.close()
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        phi, g = model.gradient(acq, wav, dobs)
    torch.cuda.synchronize()
    info0 = model.info()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        phi, g = model.gradient(acq, wav, dobs)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms_local = e0.elapsed_time(e1) / args.steps
    info1 = model.info()

    pts = info1["points"]
    units = pts * w.nt * w.nshots
    ms, rate = replica_rate(ms_local, units, world, dist, dev)
    value = rate / 1e9   # Gpts/s over all ranks
    peak, peak_kind = measured_hbm()
    kern, summ = kernel_stats(info0, info1, pts * w.nshots, peak)
    launches = (info1["kernel_launches"] - info0["kernel_launches"])
    # the dominant kernel: the largest share of the step's device time; the slowest
    # kernel's fraction and the time-weighted one stand beside it
    kname = max(kern, key=lambda k: kern[k]["total_ms"])
    kd = kern[kname]
    achieved = kd["GB/s"] or 0.0
    roof = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": kd["traffic"],
            "algorithmic_bytes_per_launch": kd["bytes_per_point"] * pts * w.nshots,
            **summ, "kernels": kern}

    # end to end through the C ABI with pinned host buffers, copies inside the timing
    e2e = None
    if not args.no_e2e:
        v_h = torch.from_numpy(w.v).pin_memory()
        wav_h = torch.from_numpy(w.wavelets()).pin_memory()
        dobs_h = dobs.cpu().pin_memory()
        grad_h = torch.empty(w.shape, dtype=torch.float32).pin_memory()
        phi_h = np.zeros(1, dtype=np.float64)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fwi.fwi_update_velocity(model.handle, v_h)
            fwi.fwi_adjoint_gradient(model.handle, acq.c, wav_h, dobs_h, phi_h, grad_h)
        te_ms, e2e_rate = replica_rate((time.perf_counter() - t0) / args.e2e_steps * 1e3, units,
                                       world, dist, dev)
        te = te_ms * 1e-3
        h2d = v_h.numel() * 4 + wav_h.numel() * 4 + dobs_h.numel() * 4
        d2h = grad_h.numel() * 4 + 8
        e2e = {"value": e2e_rate / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": te * 1e3, "misfit": float(phi_h[0])}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        g, tsec, desc, threads = cpu_baseline(w)
        cpu = {"value": g, "unit": "Gpts/s", "cores": threads, "kind": "oracle",
               "sample": desc, "seconds": round(tsec, 2),
               "one_core": cpu_baseline_one_core(args)}

    # the other two workloads of the metric, measured after the timed region
    model.close()
    serving = batched = layered = onchip = None
    if rank == 0 and not args.no_layered and args.workload == "salt_3d_512":
        k1 = kern["fwd_step_3d"]
        layered = layered_section(dev, args.layered_nt, args.snap_budget_gb, peak,
                                  (k1["avg_ms"], pts * w.nshots) if k1["launches"] else None)
    if rank == 0 and not args.no_serving:
        onchip = onchip_section(dev)
    if rank == 0 and not args.no_serving:
        serving = serving_section(dev, args.serving_requests,
                                  rates=tuple(float(x) for x in args.serving_rates.split(",")))
    if rank == 0 and not args.no_batched:
        batched = batched_section(dev, args.batched_nt, args.snap_budget_gb)

    if rank == 0:
        line = {"metric": "Gpts/s fwd+adjoint", "value": round(value, 3), "unit": "Gpts/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "grid": list(w.shape), "computed_points": pts,
                           "order": w.order, "nt": w.nt, "shots": w.nshots,
                           "receivers": w.nrec, "checkpoints": w.snap_dtype,
                           "checkpoint_slots": info1["snap_slots"],
                           "forward_steps_per_gradient": info1["last_forward_steps"],
                           "adjoint_steps_per_gradient": info1["last_adjoint_steps"],
                           "step_ctas_fwd_adj_store": info1["step_ctas"],
                           "l2": "inputs larger than L2 (each field >= 100 MB)",
                           "parallelism": f"replicas x{world}"},
                "clocks": ck, "e2e": e2e, "gpu_launches": launches,
                "roofline": roof, "cpu_baseline": cpu, "misfit": float(phi.item()),
                "layered_3d_256": layered, "serving": serving, "onchip_2d": onchip,
                "batched_2d": batched}
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
