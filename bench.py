"""Benchmark: milliseconds per 50-aperture column-generation DAO plan on one GB300.

Workload (default): the H&N-shaped phantom (5 beams x 30x30 beamlets, 192x160x80
grid of 2.5 mm voxels, two nested PTVs, unspecified tissue down-sampled 2x2x2),
seeded and synthetic, with D and D^T stored as FP16 values and a per-beamlet
FP32 scale (FP32 accumulation, FP64 objective and reduced costs).  The same plan
with FP32 storage is timed beside it.  A step is one whole plan from an empty
pool: 50 rounds of D^T SpMV pricing, aperture column and projected-Newton master
solve.  Inputs are resident in HBM when the timed region starts; L2 is flushed
(a 256 MiB write) before every step and the flush is outside the per-step
events.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import phantom  # noqa: E402

K_PLAN = 50
WORKLOADS = {
    "hn": "H&N-shaped {prec}: 5 beams x 30x30 beamlets, 192x160x80 grid @2.5 mm, two PTVs, {k} apertures",
    "prostate": "prostate-shaped {prec}: 9 beams x 20x20 beamlets, 200x120x60 grid @2.5 mm, {k} apertures",
    "tiny": "small box {prec}: 5 beams x 10x10 beamlets, 40x40x12 grid @2.5 mm, {k} apertures",
}
PREC_NAMES = {"fp32": "FP32", "fp16": "FP16 values + per-beamlet FP32 scale", "bf16": "BF16 values + per-beamlet FP32 scale"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", choices=["prostate", "tiny", "hn"], default="hn")
    p.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default=None,
                   help="storage of D and D^T (default: fp16 for hn, fp32 otherwise)")
    p.add_argument("--apertures", type=int, default=K_PLAN)
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--skip-e2e", action="store_true")
    p.add_argument("--skip-spmv", action="store_true")
    p.add_argument("--skip-strip", action="store_true", help="no SpMV leg on the strip-profile matrix")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--skip-batch", action="store_true")
    p.add_argument("--skip-serve", action="store_true")
    p.add_argument("--serve-requests", type=int, default=600,
                   help="requests of the serving leg's Poisson stream (4 per second)")
    p.add_argument("--serve-burst", type=int, default=64,
                   help="requests of the serving leg's burst (200 per second: the server under load)")
    p.add_argument("--serve-solve-slots", type=int, default=0,
                   help="plans whose rounds the server puts on the GPU at once (0: every admitted plan)")
    p.add_argument("--serve-fp32-single", type=int, default=300,
                   help="requests of the same Poisson stream served by the plain form (FP32, one plan at a time); "
                        "0: skip")
    p.add_argument("--batch", type=int, default=16, help="instances per workload in the batched re-plan leg")
    a = p.parse_args()
    if a.precision is None:
        a.precision = "fp16" if a.config == "hn" else "fp32"
    return a


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _case(name):
    return phantom.make_case(phantom.CONFIGS[name]())


def _workload_config(case, name, apertures=K_PLAN, extra=None, prec="fp32"):
    cfg = {"workload": WORKLOADS[name].format(prec=PREC_NAMES[prec], k=int(apertures)), "voxels": case.n_voxels,
           "beamlets": case.n_beamlets, "beams": case.n_beams, "nnz": case.nnz, "apertures": int(apertures),
           "storage": prec, "seed": case.spec.seed, "l2": "flushed before each step (256 MiB write)",
           "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons every 50 ms, from
    before the warm-up to the end of the timed region.  ``timed()`` brackets the
    timed region on the host clock; ``stop()`` summarises the samples taken
    inside it, or, when the region is shorter than the sampling period, the
    samples of the warm-up and the timed region together (both under load), and
    says which.  The CSV goes to $DAO_BENCH_CLOCKS_DIR (default: the temp dir)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")
    PERIOD_MS = 50
    TS_FORMAT = "%Y/%m/%d %H:%M:%S.%f"

    def __init__(self, index: int, enabled: bool = True):
        import tempfile
        self.index = index
        self.proc = None
        self.tw = self.t0 = self.t1 = None
        folder = os.environ.get("DAO_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"dao_bench_clocks_rank{index}.csv")
        if enabled:
            self.f = None
            try:
                os.makedirs(folder, exist_ok=True)
                self.f = open(self.path, "w")
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.QUERY}",
                                              "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                             stdout=self.f, stderr=subprocess.DEVNULL)
            except Exception:
                self.proc = None
                if self.f is not None:
                    self.f.close()

    def wait_first_sample(self, limit_s: float = 3.0):
        """Block until nvidia-smi has written its first sample (at most
        limit_s), then mark the start of the loaded part of the run."""
        import datetime
        t_end = time.perf_counter() + limit_s
        while self.proc is not None and time.perf_counter() < t_end:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.01)
        self.tw = datetime.datetime.now()

    def timed(self, begin: bool):
        import datetime
        if begin:
            self.t0 = datetime.datetime.now()
        else:
            self.t1 = datetime.datetime.now()

    def stop(self):
        import datetime
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 10:
                continue
            try:
                sm, mx = float(f[1]), float(f[2])
            except ValueError:
                continue
            try:
                ts = datetime.datetime.strptime(f[9], self.TS_FORMAT)
            except ValueError:
                ts = None
            rows.append((ts, sm, mx, {nm for nm, v in zip(names, f[5:9]) if v.lower().startswith("active")}))
        if not rows:
            return None

        def between(a, b):
            return [r for r in rows if a is not None and b is not None and r[0] is not None and a <= r[0] <= b]
        inside, scope = between(self.t0, self.t1), "timed region"
        if not inside:
            inside = between(self.tw, self.t1)
            scope = "warm-up and timed region (the timed region is shorter than the sampling period)"
        if not inside and self.t0 is not None:
            inside = [r for r in rows if r[0] is not None and r[0] >= self.t0][:1]
            scope = "first sample after the timed region began"
        if not inside and all(r[0] is None for r in rows):
            inside, scope = rows, "every sample of the run (timestamps unreadable)"
        if not inside:
            return None
        reasons = set().union(*(r[3] for r in inside))
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "samples": len(inside), "period_ms": self.PERIOD_MS, "scope": scope, "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic bytes per kernel class (what the method must move)
# ---------------------------------------------------------------------------

def algorithmic_bytes(case, plan, kc, launches, prec="fp32"):
    V, N, B, nnz = case.n_voxels, case.n_beamlets, case.n_beams, case.nnz
    wide = prec == "fp32"
    if kc == "dt":        # a2: D^T values + voxel indices (4+4 or 2+4 B), row pointers, pi once, w out (+ scale)
        return launches * (nnz * (8 if wide else 6) + (N + 1) * 4 + V * 4 + N * 4 + (0 if wide else N * 4))
    if kc == "dose":      # a1: D values + column indices (4+4 or 2+2 B), row pointers, x once, z out, labels
        return launches * (nnz * (8 if wide else 4) + (V + 1) * 4 + N * 4 + V * 4 + V + (0 if wide else N * 4))
    if kc == "column":    # a4: beam b's entries (nnz/B on average), two segment bounds per row, column out
        return launches * (nnz / B * (8 if wide else 4) + V * 8 + V * 4)
    if kc == "master_pass":  # a5: slab columns read once per pass + labels; final passes also write z, pi
        ev, _, _ = plan.master_stats()
        total = V * 9.0                                  # the pass at K = 0 after reset
        for k, e in enumerate(ev):                       # pool size k + 1
            total += (e + 1) * (V * 4.0 * (k + 1) + V) + 8.0 * V
        return total
    return None


def _traffic(kernel: str, source: str, bytes_per_launch: float):
    """DRAM bytes per launch from the committed ncu capture of ``kernel``, scaled
    from the captured launch to ``bytes_per_launch`` (the capture's basis: the
    algorithmic bytes, or the slab bytes for the persistent solve) by the
    captured ratio; None if the kernel's source changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")))[kernel]
        sha = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()[:16]
        if sha != rec["source_sha256_16"]:
            return None
        return round(float(rec["ratio"]) * bytes_per_launch)
    except Exception:
        return None


def _l2_record(ms_solve, ev_p, b_solve):
    """Per-evaluation time of the persistent master solve and the rate at which
    its slab passes stream (from L2 after a launch's first pass), with the L2
    bytes of the committed ncu capture of the K = 50 launch (lts__t_bytes)."""
    n_ev = float(sum(ev_p))
    if n_ev <= 0:
        return None
    rec = {"us_per_evaluation": round(1e3 * ms_solve / n_ev, 3),
           "slab_bytes_per_evaluation": round(b_solve / n_ev),
           "slab_gbs": round(b_solve / (ms_solve * 1e-3) / 1e9, 1)}
    try:
        cap = json.load(open(os.path.join(ROOT, "profiles", "k_master_persist_traffic.json")))["k_master_persist"]
        rec["lts_bytes_per_launch_k50_capture"] = cap.get("lts_bytes_per_launch")
        rec["evaluations_in_capture"] = cap.get("evaluations_in_captured_launch")
    except Exception:
        pass
    return rec


def _peaks():
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------

def oracle_plan_seconds(case, k, split=None):
    """Seconds of the oracle's k-round plan; with ``split`` also the seconds of
    its first ``split`` rounds (from the per-round callback)."""
    import oracle
    marks = {}
    t = time.perf_counter()
    cb = None if split is None else (lambda r, pr, m: marks.setdefault(r, time.perf_counter()))
    oracle.column_generation(case, k, callback=cb)
    total = time.perf_counter() - t
    if split is None:
        return total
    return total, (marks[split - 1] - t) if split - 1 in marks else None


ONE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                  "NUMEXPR_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")


def oracle_plan_seconds_one_thread(config: str, k: int, timeout_s: float = 600.0):
    """The oracle's k-round plan on one host thread: a child interpreter with
    every BLAS / OpenMP thread count set to 1 (numpy reads them at import, so
    the parent's pools are untouched).  Seconds, or None if the child failed."""
    code = ("import bench, json; case = bench._case(%r); "
            "print(json.dumps(bench.oracle_plan_seconds(case, %d)))" % (config, int(k)))
    env = dict(os.environ)
    env.update({v: "1" for v in ONE_THREAD_ENV})
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=timeout_s)
        return float(json.loads(r.stdout.strip().splitlines()[-1])) if r.returncode == 0 else None
    except Exception:
        return None


ORACLE_PARALLEL = ("numpy BLAS threads on the dense master products (S^T diag(h) S, S y); the scipy sparse "
                   "products D x and D^T pi run on one thread; FP64 on the original D whatever the GPU storage")


def _cpu_threads():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


def run_reference(a):
    ws, rank, local = _dist()
    if rank != 0:
        return
    case = _case(a.config)
    cores = _cpu_threads()
    # a step is the full plan when the whole run fits in about four minutes, else
    # the first k CG rounds scaled by 50/k (this under-states the oracle's time:
    # later rounds have larger master problems)
    probe = oracle_plan_seconds(case, 5)
    est_full = probe * 50.0          # the 50-round plan costs about 50x its first 5 rounds (measured)
    k_s = a.apertures if est_full * (a.steps + 1) <= 240 else max(2, int(a.apertures * 240 / (est_full * (a.steps + 1))))
    for _ in range(a.warmup):
        oracle_plan_seconds(case, 2)
    times = [oracle_plan_seconds(case, k_s) * (a.apertures / k_s) for _ in range(a.steps)]
    ms = 1e3 * float(np.mean(times))
    sample = (f"full {a.apertures}-aperture plan per step" if k_s == a.apertures else
              f"first {k_s} of {a.apertures} CG rounds per step, scaled x{a.apertures / k_s:.2f}")
    out = {"impl": "reference", "metric": f"ms per {a.apertures}-aperture plan", "value": ms, "unit": "ms",
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _workload_config(case, a.config, a.apertures, prec=a.precision),
           "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample,
                            "parallel": ORACLE_PARALLEL},
           "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def strip_case(case):
    """The case's anatomy with D from the strip lateral profile, generated on
    the device by the library's pencil-beam model (dao_pencil_generate)."""
    import dataclasses
    from paper_1003_5402_gb300 import binding
    spec = dataclasses.replace(case.spec, profile="strip")
    args = dict(xyz=case.voxel_xyz, iso=case.iso, n_beams=spec.n_beams, rows=spec.rows, cols=spec.cols,
                beamlet_mm=spec.beamlet_mm, sigma_mm=spec.sigma_mm, mu_per_mm=spec.mu_per_mm, cutoff=spec.cutoff,
                profile="strip", body_kind=spec.body.kind, body_center=spec.body.center[:2],
                body_size=spec.body.size[:2], jitter=spec.jitter,
                jitter_stream=(spec.seed * 0x100000001 + 0x5EED) & 0xFFFFFFFFFFFFFFFF)
    rp, col, val = binding.pencil_generate(args)
    return dataclasses.replace(case, spec=spec, indptr=rp, indices=col, data=val)


def _make_case_spec(spec):
    return phantom.make_case(spec)


def batch_instances(n_each):
    """Re-plan instances: n_each prostate-shaped and n_each H&N-shaped phantoms,
    targets shifted and OARs scaled per instance (seeds 4000 + i), generated in
    a spawn process pool."""
    import multiprocessing as mp
    specs = [phantom.perturb(phantom.spec_prostate(), 4000 + i) for i in range(n_each)]
    specs += [phantom.perturb(phantom.spec_hn(), 4000 + n_each + i) for i in range(n_each)]
    workers = max(1, min(len(specs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_make_case_spec, specs)


def run_batch(torch, dev, flush, cases, n_each, apertures):
    """Batched re-plans in two forms, against the same plans one after another:
      - per-stream: dao_batch_solve, each instance's rounds as its own CUDA
        graphs on its own stream, master problems by the per-kernel path (its
        small kernels from many instances overlap on the GPU);
      - fused: dao_batch_solve_persistent, every round's master solves of all
        instances in one cooperative launch, a group of blocks per instance.
    H&N instances use FP16 storage; launch shapes come from the autotuner."""
    import tempfile
    from paper_1003_5402_gb300 import Plan, binding
    cache = os.path.join(tempfile.gettempdir(), "dao_autotune.txt")
    plans = []
    try:
        for i, c in enumerate(cases):
            prec = binding.DAO_PREC_FP16 if i >= n_each else binding.DAO_PREC_FP32
            p = Plan(c, device=dev, precision=prec, master_persistent=0)
            p.autotune(cache)
            plans.append(p)

        def timed(fn, reps=2):
            best, res = float("inf"), None
            for _ in range(reps):
                for p in plans:
                    p.reset()
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = fn()
                best = min(best, time.perf_counter() - t0)
            return best, res
        binding.batch_solve(plans, apertures)                    # warm: builds every round graph
        t_stream, res_s = timed(lambda: binding.batch_solve(plans, apertures))
        binding.batch_solve(plans, apertures, persistent=True)   # warm: captures the fused graph
        t_fused, res_f = timed(lambda: binding.batch_solve(plans, apertures, persistent=True))
        t_seq, _ = timed(lambda: [p.solve(apertures) for p in plans])
        n = len(plans)
        forms = {"per-stream": t_stream, "fused": t_fused}
        best_form = min(forms, key=forms.get)
        best = forms[best_form]
        return {"instances": n, "workloads": f"{n_each} prostate-shaped FP32 + {n_each} H&N-shaped FP16, "
                                             f"perturbed (seeds 4000+i), {apertures} apertures each",
                "form": best_form,
                "plans_per_s_batched": round(n / best, 2),
                "plans_per_s_fused": round(n / t_fused, 2), "plans_per_s_per_stream": round(n / t_stream, 2),
                "plans_per_s_sequential": round(n / t_seq, 2), "speedup": round(t_seq / best, 3),
                "fused_blocks_per_plan": int(binding.load().dao_batch_group_size(n, dev)),
                "apertures_done": sorted({r[1] for r in res_f} | {r[1] for r in res_s}),
                "timing": "host wall clock around the synchronous calls, L2 flushed before each, best of 2"}
    finally:
        for p in plans:
            p.close()


def serve_pool(n_each):
    """Distinct re-plan instances the serving leg draws its requests from: n_each
    perturbed small (19,200-voxel) and n_each perturbed prostate-shaped phantoms
    (seeds 9000 + i), generated in a spawn process pool."""
    import multiprocessing as mp
    specs = [phantom.perturb(phantom.spec_tiny(), 9000 + i) for i in range(n_each)]
    specs += [phantom.perturb(phantom.spec_prostate(), 9000 + n_each + i) for i in range(n_each)]
    workers = max(1, min(len(specs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_make_case_spec, specs)


def run_serve(dev, pool, n_requests, apertures, rate_per_s=4.0, seed=9000, max_slots=8, solve_slots=0, **plan_opt):
    """Poisson arrivals (rate 4 per second, seeded exponential gaps) of re-plan
    requests drawn from the pool; each request uploads its D and plans
    ``apertures`` apertures.  Latency is submission to results on the host.
    ``plan_opt``: dao_options of every plan (storage precision, master blocks);
    ``max_slots`` 1 serves one plan at a time in arrival order; ``solve_slots``
    1 lets admitted requests create their plans alongside the running one but
    queue their rounds one plan at a time."""
    from paper_1003_5402_gb300 import Server
    # gaps and pool draws from their own streams: the first n requests are the
    # same whatever the stream's length
    gaps = np.random.default_rng(seed).exponential(1.0 / rate_per_s, size=n_requests)
    which = np.random.default_rng(seed + 1).integers(0, len(pool), size=n_requests)
    with Server(max_slots=max_slots, device=dev, solve_slots=solve_slots, **plan_opt) as srv:
        # warm-up, as a long-running server is: one request of each size at
        # once, so that the library's memory pool already holds two concurrent
        # plans of the larger size (its one-time growth, tens of ms, is not a
        # request's latency)
        warm = [srv.submit(pool[0], apertures), srv.submit(pool[len(pool) // 2], apertures)]
        for w in warm:
            srv.wait(w)
        t0 = time.perf_counter()
        t_next = t0
        ids = []
        for g, w in zip(gaps, which):
            t_next += g
            d = t_next - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids.append(srv.submit(pool[int(w)], apertures))
        res = [srv.wait(i) for i in ids]
        makespan = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array([r["latency_ms"] for r in res])
    qms = np.array([r["queue_ms"] for r in res])
    ok = sum(r["status"] in (0, 1, 2) for r in res)
    phases = {k: {"p50": round(float(np.percentile([r[k] for r in res], 50)), 3),
                  "p99": round(float(np.percentile([r[k] for r in res], 99)), 3)}
              for k in ("queue_ms", "create_ms", "gpu_wait_ms", "solve_ms", "finish_ms")}
    errors = sorted({f'{r["status"]}: {r["error"]}' for r in res if r["status"] not in (0, 1, 2)})
    return {"requests": n_requests, "rate_per_s": rate_per_s, "max_slots": max_slots, "solve_slots": solve_slots,
            "completed_ok": int(ok),
            "errors": errors[:4],
            "plan_options": {k: v for k, v in plan_opt.items()},
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_ms": round(float(np.max(lat)), 3), "phases": phases,
            "queue_p99_ms": round(float(np.percentile(qms, 99)), 3), "max_active": st["max_active"],
            "plans_per_s": round(ok / makespan, 3), "makespan_s": round(makespan, 3),
            "workload": f"{len(pool) // 2} perturbed 19,200-voxel + {len(pool) // 2} perturbed prostate-shaped "
                        f"instances, {apertures} apertures, D uploaded per request",
            "latency": "submission to results in host memory (dao_create + column generation + dose D2H)"}


HBM_NOMINAL_GBS = 7900.0   # GB300 HBM3e, nominal


def pinned_inputs(torch, case):
    """The case's host arrays copied once, outside any timed region, into
    page-locked memory (torch pin_memory), with the dtypes dao_create takes, so
    that its uploads are DMA from pinned host memory.  The tensors stay alive
    with the returned object."""
    import types
    keep = []

    def pin(a, dtype):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).pin_memory()
        keep.append(t)
        return t.numpy()
    c = types.SimpleNamespace(
        indptr=pin(case.indptr, np.int64), indices=pin(case.indices, np.int32), data=pin(case.data, np.float32),
        rows=pin(case.rows, np.int32), cols=pin(case.cols, np.int32),
        voxel_struct=pin(case.voxel_struct, np.int32), is_target=pin(case.is_target, np.uint8),
        under_w=pin(case.under_w, np.float64), under_t=pin(case.under_t, np.float64),
        over_w=pin(case.over_w, np.float64), over_t=pin(case.over_t, np.float64),
        n_voxels=case.n_voxels, n_beamlets=case.n_beamlets)
    c.pinned_tensors = keep
    return c


def spmv_bandwidth(torch, plan, case, prec, flush, hbm_peak, tuning=None):
    """Cold-L2 a1 and a2 alone: median of 20 runs, each timed with CUDA events;
    the fraction of the measured copy peak and of the nominal 7.9 TB/s, and the
    kernel form the plan runs (the autotuner's choice when ``tuning`` is given)."""
    out = {}
    if tuning is not None:
        out["form"] = {"dose": tuning["dose_form"], "dose_lanes": tuning["dose_lanes"], "dt_map": tuning["dt_map"],
                       "dt_threads": tuning["dt_threads"]}
    x = torch.rand(case.n_beamlets, device="cuda")
    z = torch.empty(case.n_voxels, device="cuda")
    g = torch.empty_like(z)
    pi = torch.randn(case.n_voxels, device="cuda")
    w = torch.empty(case.n_beamlets, device="cuda")
    plan.k_dose(x, z, g, objective=False)       # the dose kernel times on this fluence
    plan.k_beamlet_prices(pi, w)
    for kc in ("dose", "dt"):
        us = plan.k_time_cold(kc, flush, reps=20)   # graph: [flush, event, kernel, event] x 20, median
        byt = algorithmic_bytes(case, plan, kc, 1, prec)
        gbs = byt / (us * 1e-6) / 1e9
        out[kc] = {"us": round(us, 2), "gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_peak, 4),
                   "frac_of_nominal": round(gbs / HBM_NOMINAL_GBS, 4), "bytes": int(byt)}
    return out


def max_over_ranks(value: float, ws: int, device) -> float:
    """The largest value over the ranks (every rank gets it); the value itself
    when there is one rank.  The timed region of a multi-GPU run is the slowest
    rank's."""
    if ws <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms_per_plan(total_ms: float, steps: int, ws: int) -> float:
    """ws replicas each plan ``steps`` times within total_ms (the slowest rank's
    time): the job's time per plan is total_ms / (steps * ws)."""
    return total_ms / (steps * ws)


def run_ours(a):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_1003_5402_gb300 import Plan, build
    build.build()
    case = _case(a.config)
    batch_cases = batch_instances(a.batch) if (not a.skip_batch and rank == 0) else None
    serve_cases = serve_pool(8) if (not a.skip_serve and rank == 0) else None
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    from paper_1003_5402_gb300 import binding
    PREC = {"fp32": binding.DAO_PREC_FP32, "fp16": binding.DAO_PREC_FP16, "bf16": binding.DAO_PREC_BF16}
    plan = Plan(case, device=dev, stream=stream.cuda_stream, precision=PREC[a.precision])
    # SpMV launch shapes chosen on a cold cache, outside the timed region
    import tempfile
    tuning = plan.autotune(os.path.join(tempfile.gettempdir(), "dao_autotune.txt"))
    sampler = ClockSampler(dev, enabled=not a.no_clocks)
    sampler.wait_first_sample()
    for _ in range(a.warmup):
        plan.reset()
        plan.solve(a.apertures)
    barrier()
    l0 = plan.launch_count()
    evs = []
    sampler.timed(True)
    t_host = time.perf_counter()
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.reset()
        st, n, trace = plan.solve(a.apertures)
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    t_host = time.perf_counter() - t_host
    sampler.timed(False)
    clocks = sampler.stop()
    launches = plan.launch_count() - l0
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = max_over_ranks(float(sum(step_ms)), ws, "cuda")
    F_final = float(trace[n - 1]) if n > 0 else None
    ev, stt, kkt = plan.master_stats()

    # kernel-class breakdown: one more plan with host-driven launches bracketed by events
    plan.profile_enable(True)
    plan.reset()
    plan.solve(a.apertures)
    prof = {kc: plan.profile_read(kc) for kc in ("dose", "dt", "price", "column", "master_solve", "master_pass",
                                                 "master_hess", "master_step")}
    ev_p, _, _ = plan.master_stats()
    plan.profile_enable(False)
    kernel_ms = {kc: round(ms, 4) for kc, (nl, ms) in prof.items()}
    kernel_launches = {kc: nl for kc, (nl, ms) in prof.items()}

    # roofline of the dominant kernel.  With the persistent master (default) that
    # is k_master_persist, one launch per round: its CUDA-event time per launch
    # from the profiled plan, its algorithmic bytes the slab columns and labels
    # read once per evaluation, V (4K + 1), times the evaluations of that solve.
    # The per-kernel master's k_master_eval is reported beside it
    # (roofline_eval_kernel): every launch re-timed back to back at its own pool
    # size, weighted by the evaluations.
    hbm_peak, peak_kind = _peaks()
    V = case.n_voxels
    roof = None
    nl_solve, ms_solve = prof["master_solve"]
    if nl_solve > 0:
        b_solve = sum(float(ev_p[k - 1]) * V * (4.0 * k + 1.0) for k in range(1, len(ev_p) + 1))
        us_launch = 1e3 * ms_solve / nl_solve
        achieved = b_solve / (ms_solve * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "k_master_persist", "achieved": round(achieved, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "peak_kind": peak_kind,
                # DRAM traffic: one slab read per launch (the evaluations re-read it from L2)
                "traffic": _traffic("k_master_persist", "paper_1003_5402_gb300/csrc/master.cu",
                                    sum(V * (4.0 * k + 1.0) for k in range(1, len(ev_p) + 1)) / max(len(ev_p), 1)),
                "bytes_per_launch": round(b_solve / nl_solve), "us_per_launch": round(us_launch, 2),
                "launches_per_plan": int(nl_solve), "evaluations_per_plan": int(sum(ev_p)),
                "timing": "CUDA events around each launch of the host-driven profiled plan (one launch per round)",
                "note": "latency-bound: each evaluation is a few dependent global round trips and a one-block "
                        "Newton step; the slab pass alone streams at the L2/HBM rate",
                # the survey's terms for this pass (L2/latency-bound): time per evaluation and the
                # rate of the slab re-read from L2 (every evaluation after a launch's first)
                "l2": _l2_record(ms_solve, ev_p, b_solve)}
    w_sum = t_sum = b_sum = 0.0
    for k in range(1, n + 1):
        cnt = int(ev[k - 1]) + 1                          # evaluations + the final pass
        us = plan.k_time("master_pass", k, 10)
        w_sum += cnt
        t_sum += cnt * us
        b_sum += cnt * (V * 4.0 * k + V)
    us_avg = t_sum / w_sum
    bytes_avg = b_sum / w_sum
    achieved = bytes_avg / (us_avg * 1e-6) / 1e9
    roof_eval = {"bound": "hbm", "kernel": "k_master_eval", "achieved": round(achieved, 1), "peak": hbm_peak,
                 "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "peak_kind": peak_kind,
                 "traffic": _traffic("k_master_eval", "paper_1003_5402_gb300/csrc/master.cu", bytes_avg),
                 "bytes_per_launch": round(bytes_avg),
                 "us_per_launch": round(us_avg, 3), "launches_per_plan": int(w_sum),
                 "timing": "CUDA events around back-to-back launches at each pool size of the timed plan"}
    if roof is None:
        roof = roof_eval

    # SpMV bandwidth, L2 cold: a1 and a2 alone, 20 runs each, FP32 storage and
    # 16-bit storage (FP16 values + per-beamlet scale, same workload); and the
    # same plan in the other storage (FP32 beside an FP16 headline, else FP16)
    spmv = mixed = None
    if not a.skip_spmv:
        other = "fp32" if a.precision != "fp32" else "fp16"
        spmv = {a.precision: spmv_bandwidth(torch, plan, case, a.precision, flush, hbm_peak, tuning)}
        with Plan(case, device=dev, stream=stream.cuda_stream, precision=PREC[other]) as p2:
            t_other = p2.autotune(os.path.join(tempfile.gettempdir(), "dao_autotune.txt"))
            spmv[other] = spmv_bandwidth(torch, p2, case, other, flush, hbm_peak, t_other)
            for _ in range(2):
                p2.reset()
                p2.solve(a.apertures)
            t2 = []
            for _ in range(3):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                p2.reset()
                _, n2, tr2 = p2.solve(a.apertures)
                e1.record(stream)
                torch.cuda.synchronize()
                t2.append(e0.elapsed_time(e1))
        mixed = {"headline_storage": PREC_NAMES[a.precision], "other_storage": PREC_NAMES[other],
                 "other_ms_per_plan": round(statistics.median(t2), 4),
                 "other_objective_final": float(tr2[n2 - 1]) if n2 else None,
                 "objective_rel_diff": (abs(float(tr2[n2 - 1]) - F_final) / F_final if n2 and F_final else None)}

    # SpMV bandwidth on the same anatomy with the strip lateral profile (a 5 mm
    # strip blurred by the Gaussian, closer to a finite-size pencil beam): more
    # entries per row; D generated on the device from the model, then planned
    spmv_strip = None
    if not a.skip_spmv and not a.skip_strip:
        spmv_strip = {}
        scase = strip_case(case)
        spmv_strip["nnz"] = int(scase.nnz)
        spmv_strip["nnz_gauss"] = int(case.nnz)
        for prec in (a.precision, "fp32" if a.precision != "fp32" else "fp16"):
            with Plan(scase, device=dev, stream=stream.cuda_stream, precision=PREC[prec]) as ps:
                ts = ps.autotune(os.path.join(tempfile.gettempdir(), "dao_autotune.txt"))
                spmv_strip[prec] = spmv_bandwidth(torch, ps, scase, prec, flush, hbm_peak, ts)

    # end to end through the public API from host buffers
    e2e = None
    if not a.skip_e2e:
        n_e2e = max(1, min(a.steps, 3))
        h2d = (case.indptr.nbytes + case.indices.nbytes + case.data.nbytes + case.rows.nbytes + case.cols.nbytes
               + case.voxel_struct.nbytes + case.is_target.nbytes + 4 * case.under_w.nbytes)
        d2h = case.n_voxels * 4 + 8 + a.apertures * 8
        try:
            e2e_case, inputs = pinned_inputs(torch, case), "page-locked host arrays"
        except Exception as exc:   # no page-locked memory to be had: ordinary host arrays
            e2e_case, inputs = case, f"pageable host arrays ({type(exc).__name__})"
        times = []
        for _ in range(n_e2e + 1):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            with Plan(e2e_case, device=dev, stream=stream.cuda_stream, precision=PREC[a.precision]) as p2:
                p2.solve(a.apertures)
                dose, F = p2.dose()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        times = times[1:]
        e2e_ms = max_over_ranks(1e3 * float(np.mean(times)), ws, "cuda")
        e2e = {"value": round(whole_job_ms_per_plan(e2e_ms, 1, ws), 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e, "inputs": inputs,
               "includes": "dao_create (validation, D^T build, upload) + dao_solve + dao_dose to host"}

    batch = None
    if batch_cases is not None:
        batch = run_batch(torch, dev, flush, batch_cases, a.batch, a.apertures)
    serve = None
    if serve_cases is not None:
        # requests arrive in page-locked host buffers, as a serving process keeps
        # them (their uploads are DMA transfers)
        try:
            serve_cases = [pinned_inputs(torch, c) for c in serve_cases]
            serve_inputs = "page-locked host arrays"
        except Exception as exc:   # no page-locked memory: ordinary host arrays
            serve_inputs = f"pageable host arrays ({type(exc).__name__})"
        # FP16 storage (the mixed-precision form), every request its own plan,
        # up to 8 admitted at once (--serve-solve-slots 1: their rounds on the
        # GPU one plan at a time in admission order)
        serve = run_serve(dev, serve_cases, a.serve_requests, a.apertures, solve_slots=a.serve_solve_slots,
                          precision=PREC["fp16"])
        serve["inputs"] = serve_inputs
        if a.serve_burst > 0:
            burst = run_serve(dev, serve_cases, a.serve_burst, a.apertures, rate_per_s=200.0, seed=9100,
                              solve_slots=a.serve_solve_slots, precision=PREC["fp16"])
            serve["burst"] = {k: burst[k] for k in ("requests", "rate_per_s", "solve_slots", "completed_ok", "errors",
                                                    "p50_ms", "p99_ms", "max_ms", "max_active", "plans_per_s",
                                                    "phases")}
        if a.serve_fp32_single > 0:
            # the plain form on the same Poisson stream: FP32 storage, one plan
            # at a time in arrival order (a request that arrives while a plan
            # runs waits for it)
            single = run_serve(dev, serve_cases, a.serve_fp32_single, a.apertures, max_slots=1,
                               precision=PREC["fp32"])
            serve["fp32_single_slot"] = {k: single[k] for k in ("requests", "rate_per_s", "max_slots", "completed_ok",
                                                                "errors", "p50_ms", "p99_ms", "max_ms", "plans_per_s",
                                                                "phases", "queue_p99_ms")}

    cpu = None
    if rank == 0 and ws == 1 and not a.skip_cpu:
        # the full plan when the oracle's first rounds predict at most about a
        # minute, else its first k rounds scaled by K / k (an under-estimate:
        # later rounds have larger master problems); one host thread on its first
        # 10 rounds, beside the same 10 rounds with the BLAS threads
        probe = oracle_plan_seconds(case, 3)
        k_s = a.apertures if probe / 3 * a.apertures * 1.5 <= 60 else max(5, int(60 / (probe / 3 * 1.5)))
        secs, secs10 = oracle_plan_seconds(case, k_s, split=10)
        secs1 = oracle_plan_seconds_one_thread(a.config, 10)
        cpu = {"value": round(secs * 1e3 * a.apertures / k_s, 1), "unit": "ms", "cores": _cpu_threads(),
               "kind": "oracle", "parallel": ORACLE_PARALLEL,
               "sample": (f"one full {a.apertures}-aperture plan of the same workload" if k_s == a.apertures else
                          f"the first {k_s} of {a.apertures} rounds of the same workload, scaled x{a.apertures / k_s:.2f}")
               + " (FP64 numpy/scipy on the original D)",
               "first_10_rounds_ms": None if secs10 is None else round(secs10 * 1e3, 1),
               "first_10_rounds_ms_1_thread": None if secs1 is None else round(secs1 * 1e3, 1)}

    plan.close()
    if rank == 0:
        ms_per_step = total_ms / a.steps
        lat = sorted(step_ms)
        out = {
            "metric": f"ms per {a.apertures}-aperture plan", "value": round(whole_job_ms_per_plan(total_ms, a.steps, ws), 4),
            "unit": "ms", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _workload_config(case, a.config, a.apertures, prec=a.precision),
            "roofline": roof, "roofline_eval_kernel": roof_eval, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                           "p99": round(float(np.percentile(lat, 99)), 4)},
            "spmv": spmv, "spmv_strip_profile": spmv_strip, "mixed_precision": mixed, "batch": batch, "serve": serve, "kernel_ms_host_driven_plan": kernel_ms, "kernel_launches_host_driven_plan": kernel_launches,
            "spmv_launch_shapes": tuning,
            "objective_final": F_final, "apertures_done": int(n), "master_evals": int(np.sum(ev)),
            "host_wall_s": round(t_host, 3), "device": torch.cuda.get_device_name(dev),
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
