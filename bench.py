#!/usr/bin/env python
"""MSFT benchmark: diffraction patterns per second on one or more GB300s.

Workload (default): real spherical-harmonics shapes, l <= 8, R0 = 48 voxels,
a_lm ~ N(0, 0.05/l), random orientation, on a 128^3 grid, wavelength 10 voxels,
flat 512x512 detector to 60 deg, delta = 0.01, beta = 0.001; tensor-core
contraction with BF16 operands, split hi/lo phases and FP32 accumulation.
A step is one batch of `--batch` such patterns (each: voxelise + transmission
scan + contraction + intensity).  Inputs are synthetic and seeded.

Contract: W untimed warm-up steps, then K timed steps between a barrier and a
device synchronisation; rank 0 prints one JSON line.  Under torchrun each rank
simulates its own batch (independent patterns, no collective on the data path)
and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MSFT patterns/sec (128^3 harmonics shape, 512^2 detector to 60 deg)"
UNIT = "patterns/s"
WORKLOAD = "sh_l8_R48_grid128_det512_60deg"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tc_bf16_split")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--cpu-sample-pixels", type=int, default=32768)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=0,
                    help="run the serving mix with this many requests and print its own JSON line")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-device-time", type=int, default=0,
                    help="time this many requests of the serving mix one at a time on one stream and print a JSON line")
    ap.add_argument("--fit-step", type=int, default=0,
                    help="time this many forward+gradient fit steps of the 96^3 l<=6 workload and print a JSON line")
    ap.add_argument("--short-serving", type=int, default=2000,
                    help="requests of the serving study folded into the default line (0: skip)")
    ap.add_argument("--fig8b-case", type=float, nargs=2, metavar=("RADIUS_LAMBDA", "DETECTOR"),
                    help="time one Fig. 8b case (uniform-q detector) in --precision and print a JSON line; "
                         "for profiler runs")
    ap.add_argument("--main-only", action="store_true",
                    help="time the main step only (no comparator, fit step, plain configs, timing study, "
                         "CPU baseline or serving); for profiler runs")
    return ap.parse_args()


def serving_targets(reqs, precision):
    """Fit targets: the intensity of each request's perturbed shape, computed by
    the library with one handle per distinct geometry (untimed set-up)."""
    import torch
    import paper_2202_03411_gb300 as sm
    handles, out = {}, []
    for r in reqs:
        g = r.geometry
        key = (g.nx, g.det_nx)
        if key not in handles:
            handles[key] = sm.scatman_create(g, precision, soft=True, soft_width=0.5)
        h = handles[key]
        I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
        sm.scatman_voxelise(h, r.target)
        sm.scatman_forward(h, I)
        out.append(I)
    for h in handles.values():
        sm.scatman_sync(h)
    res = [t.cpu().numpy() for t in out]
    for h in handles.values():
        h.close()
    return res


def _stream_stats(lat, status, wall, n):
    import numpy as np
    return {"requests_per_s": n / wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "failed": int(sum(1 for x in status if x)),
            "wall_s": wall}


def serving_oracle_check(srv, reqs, targets, picks, n_sample=512, width=0.5):
    """A few requests served again with their intensity returned; each is
    compared with the FP64 oracle (soft occupancy of the server's width) on a
    pixel sample.  Returns the relative L2 errors."""
    import numpy as np

    import oracle
    out = []
    for i in picks:
        r = reqs[i]
        t, res = srv.submit(r.geometry, r.shape, targets[i], want_gradient=True, want_I=True)
        st, _ = srv.wait(t, timeout_s=120.0)
        g = r.geometry
        sample = np.sort(np.random.default_rng(i).choice(g.n_pix, size=min(n_sample, g.n_pix), replace=False))
        chi, _ = oracle.voxelise(r.shape, g, True, width)
        rho = oracle.slices(chi, g, r.shape.delta, r.shape.beta)
        Iref = np.abs(oracle.msft(rho, oracle.detector_q(g)[sample], g.voxel)) ** 2
        out.append({"request": int(i), "grid": g.nx, "detector": g.det_nx, "kind": int(r.shape.kind),
                    "status": int(st), "rel_l2_I": oracle.relative_l2(res["I"][sample].astype(np.float64), Iref),
                    "sample_pixels": int(len(sample))})
    return out


def serving_run(n_requests, slots, precision, fractions=(0.5, 0.8, 0.95), seed=0, oracle_picks=3):
    """Serving mix: forward + gradient fit requests over grids {48,64,96,128}^3 and
    detectors {128,256,512}^2, admitted under a 120 GB budget.  Runs, each on
    the same request stream:
      cold        a fresh server, every request arriving at once (handles are
                  created as requests need them, device allocations included);
      saturation  a warmed server (one handle per geometry created first), all
                  requests at once: the saturation throughput;
      poisson     Poisson arrivals at the given fractions of that throughput;
      one_slot    a warmed single-slot server at saturation (no overlap on the
                  device: the baseline the slots' concurrency is measured against).
    Latency is submit-to-result.  With oracle_picks > 0 a few requests are
    served once more with their intensity and checked against the FP64 oracle
    (on the CPU, after the timed runs)."""
    import numpy as np
    from paper_2202_03411_gb300.serving import Server, run_stream
    from workloads import serving_mix
    reqs = serving_mix(n_requests, rate_per_s=1.0, seed=seed)     # arrival times rescaled below
    targets = serving_targets(reqs, precision)
    budget = 120 * (1 << 30)
    out = {"requests": len(reqs), "slots": slots, "budget_bytes": budget}

    srv = Server(budget, slots=slots, precision=precision)
    _, lat, status, wall = run_stream(srv, reqs, targets, time_scale=0.0)
    out["cold"] = _stream_stats(lat, status, wall, len(reqs))
    out["cold"]["note"] = "fresh server: handles created on demand inside the run"
    srv.close()

    def warm(server):
        first = {}
        for r, t in zip(reqs, targets):
            first.setdefault((r.geometry.nx, r.geometry.det_nx), (r, t))
        run_stream(server, [r for r, _ in first.values()], [t for _, t in first.values()], time_scale=0.0)

    srv = Server(budget, slots=slots, precision=precision)
    warm(srv)
    _, lat, status, wall = run_stream(srv, reqs, targets, time_scale=0.0)
    sat = len(reqs) / wall
    out["saturation"] = _stream_stats(lat, status, wall, len(reqs))
    out["saturation_patterns_per_s"] = sat
    runs = []
    mean_gap = reqs[-1].arrival_s / len(reqs)
    for f in fractions:
        scale = 1.0 / (f * sat * mean_gap)          # arrival rate = f * saturation
        _, lat, status, wall = run_stream(srv, reqs, targets, time_scale=scale)
        row = _stream_stats(lat, status, wall, len(reqs))
        row.update({"load": f, "offered_per_s": f * sat})
        runs.append(row)
    out["poisson"] = runs
    out["stats"] = srv.stats()
    if oracle_picks > 0:
        picks = np.linspace(0, len(reqs) - 1, oracle_picks).astype(int).tolist()
        out["served_vs_fp64_oracle"] = serving_oracle_check(srv, reqs, targets, picks)
    srv.close()

    one = Server(budget, slots=1, precision=precision)
    warm(one)
    _, lat, status, wall = run_stream(one, reqs, targets, time_scale=0.0)
    out["one_slot"] = _stream_stats(lat, status, wall, len(reqs))
    one.close()
    out["slots_over_one_slot"] = sat / out["one_slot"]["requests_per_s"]
    return out



def serving_device_time(n_requests, precision, seed=0):
    """Device time of the serving mix's requests run one at a time on one
    stream (no overlap): voxelise + forward, then residual + backward, CUDA
    events around each part; one handle per geometry, created before timing,
    each request timed on its second run.  The served rate over 1 / (mean of
    these) says how much the server's slots overlap requests on the device."""
    import numpy as np
    import torch
    import paper_2202_03411_gb300 as sm
    from workloads import serving_mix
    reqs = serving_mix(n_requests, rate_per_s=1.0, seed=seed)
    targets = serving_targets(reqs, precision)
    stream = torch.cuda.current_stream()
    handles, rows = {}, {}
    for r, t in zip(reqs, targets):
        g = r.geometry
        key = (g.nx, g.det_nx)
        if key not in handles:
            handles[key] = sm.scatman_create(g, precision, soft=True, soft_width=0.5)
        h = handles[key]
        I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
        tt = torch.as_tensor(t, device="cuda")
        for rep in range(2):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            sm.scatman_voxelise(h, r.shape)
            sm.scatman_forward(h, I)
            ev[1].record(stream)
            sm.scatman_backward(h, 2.0 * (I - tt))
            ev[2].record(stream)
            torch.cuda.synchronize()
        rows.setdefault(key, []).append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
    for h in handles.values():
        h.close()
    per = {}
    tot = []
    for key in sorted(rows):
        a = np.array(rows[key])
        per["grid%d_det%d" % key] = {"requests": len(a), "forward_ms": float(a[:, 0].mean()),
                                     "backward_ms": float(a[:, 1].mean())}
        tot.extend(a.sum(1).tolist())
    mean = float(np.mean(tot))
    return {"requests": len(tot), "mean_ms": mean, "requests_per_s_if_serial": 1e3 / mean, "per_geometry": per}

def fit_step_run(n_shapes, precision, warm=2):
    """Forward + gradient fit steps on the 96^3 / 256^2 l<=6 harmonics workload
    (soft occupancy, loss sum (I - I_target)^2).  Per step: voxelise,
    contraction, residual, adjoint (scatman_backward, which synchronises)."""
    import numpy as np
    import torch
    import paper_2202_03411_gb300 as sm
    from workloads import perturbed, sh_grad_96
    g, shapes = sh_grad_96(n_shapes=n_shapes)
    h = sm.scatman_create(g, precision, soft=True, soft_width=0.5)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    targets = []
    for k, s in enumerate(shapes):
        sm.scatman_voxelise(h, perturbed(s, np.random.default_rng(k)))
        sm.scatman_forward(h, I)
        targets.append(I.clone())
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    rows = []
    for it, (s, t) in enumerate(list(zip(shapes, targets))[:warm] + list(zip(shapes, targets))):
        ev[0].record(stream)
        sm.scatman_voxelise(h, s)
        ev[1].record(stream)
        sm.scatman_forward(h, I)
        ev[2].record(stream)
        w = 2.0 * (I - t)
        ev[3].record(stream)
        sm.scatman_backward(h, w)
        ev[4].record(stream)
        torch.cuda.synchronize()
        if it >= warm:
            rows.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    h.close()
    a = np.array(rows)
    tot = a.sum(1)
    return {"workload": "sh_l6_R36_grid96_det256_45deg_soft", "precision": precision, "steps": len(rows),
            "fit_steps_per_s": 1e3 / tot.mean(), "p50_ms": float(np.percentile(tot, 50)),
            "p99_ms": float(np.percentile(tot, 99)),
            "stage_ms": {"voxelise": float(a[:, 0].mean()), "forward": float(a[:, 1].mean()),
                         "residual": float(a[:, 2].mean()), "backward": float(a[:, 3].mean())}}


def time_mode(g, shapes, precision, reps=1):
    """Mean ms per pattern (voxelise + forward) and the intensity of shapes[0]."""
    import torch
    import paper_2202_03411_gb300 as sm
    h = sm.scatman_create(g, precision)
    f64 = precision == "fp64"
    I = torch.empty(g.n_pix, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    sm.scatman_voxelise(h, shapes[0])
    sm.scatman_forward(h, I)
    sm.scatman_sync(h)
    I0 = I.double().cpu().numpy()
    stream = torch.cuda.current_stream()
    n = reps * len(shapes)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    ev[0].record(stream)
    k = 0
    for _ in range(reps):
        for s_ in shapes:
            sm.scatman_voxelise(h, s_)
            sm.scatman_forward(h, I)
            k += 1
            ev[k].record(stream)
    sm.scatman_sync(h)
    h.close()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(n))
    ms = ev[0].elapsed_time(ev[n]) / n
    time_mode.last_p50_p99 = (per[len(per) // 2], per[min(len(per) - 1, int(math.ceil(0.99 * len(per))) - 1)])
    return ms, I0


def plain_configs():
    """The FP64 sphere (32^3, 64^2 to 30 deg) and the FP32-vs-FP64 ellipsoids
    (96^3, 256^2 to 45 deg); errors against the oracle are added by the CPU leg."""
    from workloads import ellipsoid_96, sphere_32
    g1, s1 = sphere_32()
    ms1, I1 = time_mode(g1, s1, "fp64", reps=20)
    lat1 = time_mode.last_p50_p99
    g2, s2 = ellipsoid_96(n_shapes=64)
    ms32, I2_32 = time_mode(g2, s2[:16], "fp32")
    lat32 = time_mode.last_p50_p99
    ms64, I2_64 = time_mode(g2, s2[:4], "fp64")
    lat64 = time_mode.last_p50_p99
    out = {"sphere_32_fp64": {"patterns_per_s": 1e3 / ms1, "ms_per_pattern": ms1, "p50_p99_ms": lat1},
           "ellipsoid_96": {"fp32": {"patterns_per_s": 1e3 / ms32, "ms_per_pattern": ms32, "shapes_timed": 16,
                                     "p50_p99_ms": lat32},
                            "fp64": {"patterns_per_s": 1e3 / ms64, "ms_per_pattern": ms64, "shapes_timed": 4,
                                     "p50_p99_ms": lat64}}}
    return out, (g1, s1[0], I1), (g2, s2[0], I2_32, I2_64)


def plain_config_errors(c1, c2, n_sample=1024):
    """CPU leg: the oracle's answers for the two plain configurations (the
    sphere on the full detector, the ellipsoid on a pixel sample)."""
    import numpy as np

    import oracle
    g1, s1, I1 = c1
    Iref1, _ = oracle.forward(s1, g1)
    g2, s2, I32, I64 = c2
    sample = np.sort(np.random.default_rng(0).choice(g2.n_pix, size=n_sample, replace=False))
    chi, _ = oracle.voxelise(s2, g2)
    rho = oracle.slices(chi, g2, s2.delta, s2.beta)
    Iref2 = np.abs(oracle.msft(rho, oracle.detector_q(g2)[sample], g2.voxel)) ** 2
    return {"sphere_32_fp64_rel_l2": oracle.relative_l2(I1, Iref1),
            "ellipsoid_96_fp32_rel_l2": oracle.relative_l2(I32[sample], Iref2),
            "ellipsoid_96_fp64_rel_l2": oracle.relative_l2(I64[sample], Iref2),
            "ellipsoid_sample_pixels": n_sample}


def map_configs(precision):
    """Map shapes of Sec. 5.2 on the 96^3 / 256^2 / 45 deg geometry: radii maps
    (96 x 192 samples) and two-material volume maps (40^3 cells of 1.7 voxels,
    per-cell delta and beta).  Errors against the oracle are added by the CPU leg."""
    from workloads import radialmap_96, volumemap_96
    out, refs = {}, {}
    for name, maker in (("radialmap_96", radialmap_96), ("volumemap_index_96", volumemap_96)):
        g, shapes = maker(n_shapes=4)
        ms, I0 = time_mode(g, shapes, precision, reps=2)
        out[name] = {"precision": precision, "patterns_per_s": 1e3 / ms, "ms_per_pattern": ms,
                     "shapes_timed": len(shapes), "p50_p99_ms": time_mode.last_p50_p99}
        refs[name] = (g, shapes[0], I0)
    return out, refs


def map_config_errors(refs, n_sample=1024):
    """CPU leg: the oracle on a pixel sample of each map workload's first shape."""
    import numpy as np

    import oracle
    errs = {}
    for name, (g, s, I) in refs.items():
        sample = np.sort(np.random.default_rng(1).choice(g.n_pix, size=n_sample, replace=False))
        chi, _ = oracle.voxelise(s, g)
        rho = oracle.slices_n(chi, g, *oracle.voxel_index(s, g)) if s.varying_index() else \
            oracle.slices(chi, g, s.delta, s.beta)
        Iref = np.abs(oracle.msft(rho, oracle.detector_q(g)[sample], g.voxel)) ** 2
        errs[name + "_rel_l2"] = oracle.relative_l2(I[sample], Iref)
    errs["sample_pixels"] = n_sample
    return errs


def detector_run(g, I, reps=20, photon_density=1e3):
    """Ideal detector (Sec. 5.2, photon statistics) on the bench pattern: the
    launch that turns I into expected photons and Poisson counts."""
    import torch
    import paper_2202_03411_gb300 as sm
    h = sm.scatman_create(g, "tc_bf16_split")
    lam, cnt = sm.scatman_photon_counts(h, photon_density, 0, I)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(reps):
        sm.scatman_photon_counts(h, photon_density, k, I)
    e1.record(stream)
    sm.scatman_sync(h)
    ms = e0.elapsed_time(e1) / reps
    out = {"photon_density_per_length2": photon_density, "us_per_pattern": 1e3 * ms,
           "expected_photons": float(lam.sum().item()), "counted_photons": int(cnt.sum().item()),
           "note": "expected photons per pixel from the pixel solid angle and the cross-section; Poisson counts "
                   "from Philox-4x32-10 (FP64)"}
    h.close()
    return out


def fig8b_run(radii=(3.0, 5.0, 10.0, 20.0), dets=(256, 512, 1024, 2048), precisions=("fp32", "tc_bf16_split"),
              reps=5):
    """Sec. 6 timing study (Fig. 8b): the Listing-2 harmonics shape scaled to a mean
    radius of 3/5/10/20 wavelengths on the paper's uniform-q virtual detector of
    256^2 ... 2048^2 pixels at 30 deg (voxel = lambda / (2 sin 30 deg) = lambda).
    Each precision's ms per pattern (voxelise + forward, p50 of the runs); the
    tensor-core rows add their rel. L2 difference from the FP32 intensities."""
    import numpy as np
    from workloads import fig8b_case
    table = []
    for R in radii:
        for det in dets:
            g, shape = fig8b_case(R, det)
            row = {"radius_lambda": R, "grid": g.nx, "detector": det}
            I32 = None
            for prec in precisions:
                ms, I = time_mode(g, [shape], prec, reps=reps)
                row[prec] = {"ms_per_pattern": ms, "p50_ms": time_mode.last_p50_p99[0], "patterns_per_s": 1e3 / ms}
                if prec == "fp32":
                    I32 = I
                elif I32 is not None:
                    row[prec]["rel_l2_vs_fp32"] = float(np.linalg.norm(I - I32) / np.linalg.norm(I32))
            table.append(row)
    return {"precisions": list(precisions), "detector": "uniform-q (the paper's virtual detector), separable sums; "
            "tensor-core modes run the x/z sum as one tcgen05 GEMM over all detector rows", "cases": table}


def mode_comparator(g, shapes, precision, n=3):
    """Another precision mode on the same patterns: patterns/s, ms per pattern
    (voxelise + forward), the contraction flops it executes (each mode skips
    the empty parts of every slice) and the intensity of pattern 0."""
    import torch
    import paper_2202_03411_gb300 as sm
    h = sm.scatman_create(g, precision)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, shapes[0])
    sm.scatman_forward(h, I)
    sm.scatman_sync(h)
    issued = []
    for s in shapes[:n]:
        sm.scatman_voxelise(h, s)
        issued.append(sm.scatman_contraction_flops(h)[0])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for s in shapes[:n]:
        sm.scatman_voxelise(h, s)
        sm.scatman_forward(h, I)
    e1.record(stream)
    sm.scatman_sync(h)
    ms = e0.elapsed_time(e1) / n
    sm.scatman_voxelise(h, shapes[0])
    sm.scatman_forward(h, I)
    sm.scatman_sync(h)
    I0 = I.double().cpu().numpy()
    h.close()
    return {"precision": precision, "patterns_per_s": 1e3 / ms, "ms_per_pattern": ms, "patterns_timed": n,
            "executed_flops_per_pattern": statistics.mean(issued)}, I0


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def rank_batch(rank: int, batch: int):
    """The independent patterns rank `rank` simulates: its own seeds, no overlap."""
    from workloads import sh_128
    return sh_128(n_shapes=batch, seed0=rank * batch)


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time is the slowest rank's (all_reduce MAX); identity for one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def recorded_traffic(kernel: str, source: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source is unchanged since that capture (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, source), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
        return rec["dram_bytes_per_launch"] if h.startswith(rec["sha256_prefix"]) else None
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"scatman_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(shapes, g, I_gpu, n_sample, seed=0, threads=None):
    """The oracle, as it stands, on a bounded sample of the same workload: one
    pattern's full voxelisation and transmission plus the field at n_sample
    pixels, scaled to patterns/s.  Also returns the GPU result's relative L2
    error against the oracle on that sample.  threads: OpenMP threads (None:
    all host cores)."""
    import numpy as np

    import oracle
    all_threads = oracle.num_threads()
    if threads is not None:
        oracle.set_threads(threads)
    shape = shapes[0]
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(g.n_pix, size=min(n_sample, g.n_pix), replace=False))
    q = oracle.detector_q(g)[sample]
    t0 = time.perf_counter()
    chi, _ = oracle.voxelise(shape, g)
    rho = oracle.slices(chi, g, shape.delta, shape.beta)
    t1 = time.perf_counter()
    A = oracle.msft(rho, q, g.voxel)
    t2 = time.perf_counter()
    per_pattern = (t1 - t0) + (t2 - t1) * g.n_pix / len(sample)
    Iref = np.abs(A) ** 2
    err = oracle.relative_l2(I_gpu[sample], Iref) if I_gpu is not None else None
    cores = oracle.num_threads()
    oracle.set_threads(all_threads)
    return {"value": 1.0 / per_pattern, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 pattern: full 128^3 voxelisation + transmission, field at {len(sample)} of "
                      f"{g.n_pix} pixels, time scaled to the whole detector ({t2 - t0:.1f} s of CPU work)"}, err


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from workloads import sh_128
    g, shapes = sh_128(n_shapes=1)
    shape = shapes[0]
    rng = np.random.default_rng(0)
    n_s = max(1, args.cpu_sample_pixels // 4)
    q_all = oracle.detector_q(g)
    times, walls = [], []
    for k in range(args.warmup + args.steps):
        sample = rng.choice(g.n_pix, size=n_s, replace=False)
        t0 = time.perf_counter()
        chi, _ = oracle.voxelise(shape, g)
        rho = oracle.slices(chi, g, shape.delta, shape.beta)
        t1 = time.perf_counter()
        oracle.msft(rho, q_all[sample], g.voxel)
        t2 = time.perf_counter()
        if k >= args.warmup:
            times.append((t1 - t0) + (t2 - t1) * g.n_pix / n_s)
            walls.append(t2 - t0)
    per = statistics.mean(times)
    value = 1.0 / per
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
        "ms_per_pattern_scaled": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": 1, "precision": "fp64 oracle (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"per step (ms_per_step is its measured wall time): 1 pattern's full "
                                   f"voxelisation + transmission and the field at {n_s} random pixels; the "
                                   f"field time is scaled by {g.n_pix}/{n_s} to the whole detector for value"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def launches_per_pattern(precision: str, n_pix: int, sm_count: int) -> int:
    """Kernels one voxelise + forward launches: tensor-core modes reset the
    slice boxes, voxelise with the scan, pack the occupied-slice list and run
    the contraction, plus the sum of the cut tiles' partial fields when the
    last wave of 128-pixel tiles is cut into slice ranges; the CUDA-core modes
    voxelise and run the contraction with its fixed-order partial-sum
    reduction."""
    if not precision.startswith("tc_"):
        return 3
    tiles = (n_pix + 127) // 128
    rem = tiles % sm_count if tiles > sm_count else tiles
    parts = min(4, max(1, (sm_count + rem // 2) // rem)) if rem else 1
    return 5 if parts > 1 else 4


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.fit_step > 0:
        import __graft_entry__
        __graft_entry__.build()
        res = fit_step_run(args.fit_step, args.precision)
        print(json.dumps({"metric": "MSFT forward+gradient fit steps/s (96^3 harmonics, 256^2 detector)",
                          "value": res["fit_steps_per_s"], "unit": "fit steps/s", "n_gpus": 1,
                          "higher_is_better": True, "data": "synthetic", "fit_step": res}), flush=True)
        return
    if args.fig8b_case:
        import __graft_entry__
        __graft_entry__.build()
        res = fig8b_run(radii=(args.fig8b_case[0],), dets=(int(args.fig8b_case[1]),), precisions=(args.precision,),
                        reps=3)
        print(json.dumps({"metric": "MSFT ms per pattern (Fig. 8b case, uniform-q detector)", "unit": "ms",
                          "higher_is_better": False, "data": "synthetic", "fig8b": res}), flush=True)
        return
    if args.serving_device_time > 0:
        import __graft_entry__
        __graft_entry__.build()
        res = serving_device_time(args.serving_device_time, args.precision)
        print(json.dumps({"metric": "MSFT serving mix, device ms per request run alone", "value": res["mean_ms"],
                          "unit": "ms", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
                          "serving_device_time": res}), flush=True)
        return
    if args.serving > 0:
        import __graft_entry__
        __graft_entry__.build()
        res = serving_run(args.serving, args.serving_slots, args.precision)
        line = {"metric": "MSFT forward+gradient fit requests/s (serving mix, 120 GB budget)",
                "value": res["saturation_patterns_per_s"], "unit": "requests/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "bf16" if "bf16" in args.precision else "f16",
                "data": "synthetic", "config": {"workload": "serving_mix_grids48-128_det128-512",
                                                "precision": args.precision}, "serving": res}
        print(json.dumps(line), flush=True)
        return
    rank, world, local_rank = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    import paper_2202_03411_gb300 as sm
    g, shapes = rank_batch(rank, args.batch)
    B = len(shapes)
    stream = torch.cuda.current_stream()
    h = sm.scatman_create(g, args.precision)
    # a second handle on its own stream: the timed step alternates patterns
    # between the two, so one pattern's voxeliser runs on the SMs the other's
    # contraction has finished with (separate handles are independent)
    s_alt = torch.cuda.Stream()
    h_alt = sm.scatman_create(g, args.precision, stream=s_alt.cuda_stream)
    I_all = torch.empty((B, g.n_pix), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(B)]

    def step():
        # one handle, one stream: per-pattern events give the stage times
        for b, s in enumerate(shapes):
            ev[b][0].record(stream)
            sm.scatman_voxelise(h, s)
            ev[b][1].record(stream)
            sm.scatman_forward(h, I_all[b])
            ev[b][2].record(stream)

    ev2 = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(), torch.cuda.Event(enable_timing=True)]

    def step2():
        # the timed step: patterns alternate between the two handles' streams
        ev2[0].record(stream)
        s_alt.wait_event(ev2[0])
        for b, s in enumerate(shapes):
            hh = h_alt if b % 2 else h
            sm.scatman_voxelise(hh, s)
            sm.scatman_forward(hh, I_all[b])
        ev2[1].record(s_alt)
        stream.wait_event(ev2[1])
        ev2[2].record(stream)

    # real flops each pattern's contraction issues (occupied boxes), the dense
    # count, and the method's own work: 8 flop per (pixel, occupied voxel) pair
    # and phase product
    issued, dense, occupied = [], [], []
    for s_ in shapes:
        sm.scatman_voxelise(h, s_)
        a, d = sm.scatman_contraction_flops(h)
        issued.append(a)
        dense.append(d)
        occupied.append(int((sm.scatman_get_occupancy(h, (g.nz, g.nx, g.ny)) > 0).sum()))

    for _ in range(args.warmup):
        step2()
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local_rank)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1)                       # evict L2 between timed steps (not timed)
        step2()
        torch.cuda.synchronize()
        step_ms.append(ev2[0].elapsed_time(ev2[2]))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = world * B * args.steps / (total_ms / 1e3)
    # the same steps on one handle and one stream: stage times per pattern (the
    # roofline's contraction duration) and the rate without the overlap
    pat_ms, fwd_ms, vox_ms, step1_ms = [], [], [], []
    for _ in range(args.steps):
        flush.fill_(1)
        step()
        torch.cuda.synchronize()
        pat_ms += [ev[b][0].elapsed_time(ev[b][2]) for b in range(B)]
        fwd_ms += [ev[b][1].elapsed_time(ev[b][2]) for b in range(B)]
        vox_ms += [ev[b][0].elapsed_time(ev[b][1]) for b in range(B)]
        step1_ms.append(ev[0][0].elapsed_time(ev[B - 1][2]))
    clocks = sampler.stop()
    single_stream = world * B * args.steps / (max_over_ranks(sum(step1_ms), dist, "cuda") / 1e3)

    # roofline of the contraction kernel (the dominant launch)
    peaks, peak_kind = measured_peaks()
    n_vox = g.nx * g.ny * g.nz
    products = 2 if "split" in args.precision else 1
    executed = statistics.mean(issued)                 # real flops the contraction executes per pattern
    method = 8.0 * g.n_pix * statistics.mean(occupied) * products    # the method's own work per pattern
    fwd_avg_s = statistics.mean(fwd_ms) / 1e3
    achieved = method / fwd_avg_s / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": recorded_traffic("msft_tc_kernel", "paper_2202_03411_gb300/csrc/msft_tc.cu"),
                "kernel": "msft_tc_kernel",
                "peak_source": f"{peak_kind} bf16_tflops_sustained (cuBLAS bf16; f16 has the same nominal rate)",
                "flops_per_launch": method,
                "flops_basis": "the method's work: 8 flop x pixels x occupied voxels x phase products "
                               f"({statistics.mean(occupied):.0f} occupied voxels of {n_vox} on average)",
                "executed_flops_per_launch": executed,
                "executed_tflops": executed / fwd_avg_s / 1e12,
                "executed_frac": executed / fwd_avg_s / 1e12 / peak,
                "executed_over_method": executed / method,
                "dense_flops_per_launch": statistics.mean(dense),
                "dense_equivalent_tflops": statistics.mean(dense) / fwd_avg_s / 1e12,
                "frac_of_burst_peak": achieved / float(peaks.get("bf16_tflops", peak)),
                "useful_single_product_tflops": achieved / products}

    # the voxeliser + scan: ALU-bound (the harmonic radius per voxel); its HBM
    # writes are the slice operand and the occupancy
    tc = args.precision.startswith("tc_")
    nxp, nyp = (g.nx + 15) // 16 * 16, (g.ny + 15) // 16 * 16
    s_bytes = g.nz * 3 * nxp * nyp * 2 if tc else n_vox * (16 if args.precision == "fp64" else 8)
    vox_bytes = s_bytes + n_vox * 4
    vox_s = statistics.mean(vox_ms) / 1e3
    voxelise = {"bound": "alu", "bytes_written_per_launch": vox_bytes, "achieved_gbs": vox_bytes / vox_s / 1e9,
                "hbm_peak_gbs": float(peaks.get("hbm_gbs", 0.0)),
                "frac_of_hbm": vox_bytes / vox_s / 1e9 / float(peaks.get("hbm_gbs", 1.0)),
                "note": "one spherical-harmonics radius (l <= 8) per voxel; the writes are far below HBM speed"}

    # end to end through the C ABI with host memory: voxelise + forward + D2H per pattern
    # (the pipelined batch call: pattern i computes while pattern i - 1 downloads),
    # the patterns split between the two handles, each called from its own host
    # thread so the two batches overlap on the device like the timed step
    I_host = torch.empty((B, g.n_pix), dtype=torch.float32, pin_memory=True)
    halves = [(hh, [shapes[i] for i in range(k, B, 2)], [I_host[i] for i in range(k, B, 2)])
              for k, hh in ((0, h), (1, h_alt))]

    def acquire_both():
        errs = []

        def run(hh, ss, rows):
            try:
                sm.scatman_acquire_batch(hh, ss, rows)
            except Exception as exc:          # re-raised on the calling thread
                errs.append(exc)
        t = threading.Thread(target=run, args=halves[1])
        t.start()
        run(*halves[0])
        t.join()
        if errs:
            raise errs[0]

    acquire_both()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        acquire_both()
    e_el = max_over_ranks(time.perf_counter() - e0, dist, "cuda")
    h2d = B * (8 * (shapes[0].lmax + 1) ** 2 + 160)      # shape struct + coefficients handed over
    d2h = B * g.n_pix * 4
    e2e = {"value": world * B * args.steps / e_el, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    I0 = I_all[0].double().cpu().numpy()
    extras = world == 1 and not args.main_only
    fp32, I0_fp32 = mode_comparator(g, shapes, "fp32") if not args.main_only else (None, None)
    other_tc = "tc_f16_split" if args.precision != "tc_f16_split" else "tc_bf16_split"
    tc2, I0_tc2 = mode_comparator(g, shapes, other_tc, n=B) if extras else (None, None)
    fit = fit_step_run(32, args.precision) if extras else None
    plain, c1, c2 = plain_configs() if extras else (None, None, None)
    fig8b = fig8b_run() if extras else None
    maps, map_refs = map_configs(args.precision) if extras else (None, None)
    detector = detector_run(g, I_all[0]) if extras else None
    cpu = None
    err = None
    err_fp32 = None
    if rank == 0 and extras and not args.no_cpu_baseline:
        cpu, err = cpu_baseline(shapes, g, I0, args.cpu_sample_pixels)
        cpu["one_core"], _ = cpu_baseline(shapes, g, None, max(256, args.cpu_sample_pixels // 32), threads=1)
        _, err_fp32 = cpu_baseline(shapes, g, I0_fp32, 512)
        if tc2 is not None:
            _, tc2["rel_l2_I_vs_fp64_oracle"] = cpu_baseline(shapes, g, I0_tc2, 4096)
        if plain is not None:
            plain["errors_vs_fp64_oracle"] = plain_config_errors(c1, c2)
        if maps is not None:
            maps["errors_vs_fp64_oracle"] = map_config_errors(map_refs)
    tc_ms = statistics.mean(pat_ms)
    if fp32 is not None:
        fp32["rel_l2_I_vs_fp64_oracle"] = err_fp32
        # both modes skip the empty parts of each slice, so this ratio compares
        # the arithmetic (tensor cores vs FP32 CUDA cores) at nearly equal work
        fp32["tc_speedup_per_pattern"] = fp32["ms_per_pattern"] / tc_ms
        fp32["executed_flops_ratio_fp32_over_tc"] = fp32["executed_flops_per_pattern"] / (executed / products)
    if tc2 is not None:
        tc2["note"] = (f"{args.precision} is the headline because the benchmarked configuration specifies BF16 "
                       "operands; FP16 has the same tensor rate and a finer mantissa (|s| <= 1 and the phases fit "
                       "its range)")
    serving = None
    if args.short_serving > 0 and extras:
        try:
            serving = serving_run(args.short_serving, args.serving_slots, args.precision)
        except Exception as e:          # the main line is still printed
            serving = {"error": f"{type(e).__name__}: {e}"}

    pat_sorted = sorted(pat_ms)
    p50 = pat_sorted[len(pat_sorted) // 2]
    p99 = pat_sorted[min(len(pat_sorted) - 1, int(math.ceil(0.99 * len(pat_sorted))) - 1)]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if "bf16" in args.precision else "f16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_gpu": B, "grid": [g.nx, g.ny, g.nz],
                   "detector": [g.det_nx, g.det_ny], "theta_max_deg": g.theta_max_deg,
                   "wavelength_voxels": g.wavelength, "precision": args.precision, "parallelism": "replicas",
                   "streams": "2 handles on 2 streams per GPU, patterns alternating between them",
                   "l2": "flushed between timed steps (256 MB write, outside the timed events)"},
        "single_stream_patterns_per_s": single_stream,
        "latency_ms": {"p50": p50, "p99": p99, "unit": "ms per pattern (voxelise + contraction), one stream"},
        "stage_ms": {"voxelise_scan": statistics.mean(vox_ms), "contraction": statistics.mean(fwd_ms),
                     "note": "one handle on one stream, the same steps after the timed ones"},
        "error_vs_fp64_oracle": {"rel_l2_I": err, "on": "cpu_baseline sample of pattern 0"},
        "roofline": roofline,
        "voxelise_scan": voxelise,
        "fp32_cuda_core_comparator": fp32,
        "other_tensor_core_mode": tc2,
        "fit_step_96": fit,
        "plain_configs": plain,
        "fig8b_uniform_q": fig8b,
        "map_shapes_96": maps,
        "ideal_detector": detector,
        "serving": serving,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_pattern(args.precision, g.n_pix,
                                             torch.cuda.get_device_properties(local_rank).multi_processor_count)
                        * B * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    h.close()
    h_alt.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
