#!/usr/bin/env python3
"""Exact reverse k-MIPS throughput and latency at |Q|=1M, |P|=500k, d=50, k=10.

One step = one batch of ``--nq`` queries (bit copies of random items, k=10)
through the whole online path (block filter, per-user filter, exact recheck /
verification, emit) via ``rmips_query_batch`` with device-resident inputs and
outputs.  The index (Algorithm 1) is built once before timing.  Prints one JSON
line on rank 0.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2110_07131_gb300 import datagen  # noqa: E402

METRIC = "exact reverse k-MIPS queries/s and p50/p99 ms at |Q|=1M |P|=500k d=50 k=10"
SEED = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=500_000)
    ap.add_argument("--d", type=int, default=50)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--k-max", type=int, default=25)
    ap.add_argument("--nq", type=int, default=10000, help="queries per step")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--p-prime", type=int, default=0, help="0 = bounds over all of P")
    ap.add_argument("--block-size", type=int, default=32)
    ap.add_argument("--no-blocks", action="store_true", help="Lemma 3 off (the paper's without-blocks ablation)")
    ap.add_argument("--batch-kernel", default="tc", choices=["tc", "cuda"],
                    help="batched filter on tensor cores (TF32 tiles) or CUDA cores (FP32 FMA)")
    ap.add_argument("--plain-queries", type=int, default=400)
    ap.add_argument("--e2e-threads", type=int, default=3,
                    help="caller threads of the end-to-end figure, each on its own stream")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU baseline time")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=100000,
                    help="largest number of requests of a serving run (0: skip)")
    ap.add_argument("--single-queries", type=int, default=2000,
                    help="device-resident single queries launched back to back (0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the variants, the precision workload, the error report and the CPU Simpfer")
    return ap.parse_args()


def workload(a):
    return {"workload": f"reverse k-MIPS |Q|={a.n} |P|={a.m} d={a.d} k={a.k} (k_max={a.k_max}), "
                        f"MF-like lognormal-norm synthetic vectors, queries = random items of P",
            "n_users": a.n, "n_items": a.m, "d": a.d, "k": a.k, "k_max": a.k_max,
            "queries_per_step": a.nq, "index": "full-P" if a.p_prime == 0 else f"P'={a.p_prime}",
            "block_size": a.block_size, "block_filter": not a.no_blocks, "filter_precision": a.precision,
            "batch_filter": (f"tcgen05 {dict(fp32='TF32', fp16='FP16', bf16='BF16')[a.precision]} tiles"
                             if a.batch_kernel == "tc" else "CUDA-core FP32 FMA tiles"),
            "l2": "inputs larger than L2 (Q 200 MB fp32 + bounds 200 MB); no flush between steps"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples (every 100 ms) around a timed region.

    Started before the warm-up so that sampling is running when the timed
    region begins; stop(t0, t1) keeps the samples stamped inside [t0, t1]
    (host wall clock) widened by one sampling period, or, for a region shorter
    than a period, the samples adjacent to it."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD = 0.1

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(int(self.PERIOD * 1000))],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def _rows(self):
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            rows.append((ts, parts[1:]))
        return rows

    def stop(self, t0: float = None, t1: float = None) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        deadline = time.time() + 1.0                  # let one sample land after the region
        while t1 is not None and time.time() < deadline and not any(ts > t1 for ts, _ in self._rows()):
            time.sleep(0.02)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self._rows()
        os.unlink(self.path)
        window = "timed region"
        if t0 is not None and t1 is not None:
            sel = [r for ts, r in rows if t0 - self.PERIOD <= ts <= t1 + self.PERIOD]
            if not sel:
                before = [r for ts, r in rows if ts < t0][-1:]
                after = [r for ts, r in rows if ts > t1][:1]
                sel, window = before + after, "samples adjacent to a region shorter than the sampling period"
            rows = sel
        else:
            rows = [r for _, r in rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window}


# --------------------------------------------------------------------------- CPU oracle timing
def oracle_sample(Q, P, q, k, seconds, rng):
    """Time the CPU oracle deciding a random user sample for one query.

    Returns (queries/s equivalent, users sampled, seconds, cores)."""
    from oracle import rmips_oracle as O
    n = Q.shape[0]
    users = rng.choice(n, 256, replace=False)
    t0 = time.perf_counter()
    O.decide_users(Q, P, q, k, users)
    t = time.perf_counter() - t0
    s = int(min(n, max(256, 256 * seconds / max(t, 1e-3))))
    users = rng.choice(n, s, replace=False)
    t0 = time.perf_counter()
    O.decide_users(Q, P, q, k, users)
    t = time.perf_counter() - t0
    return (s / n) / t, s, t, os.cpu_count()


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    Q, P = datagen.make_problem(a.n, a.m, a.d, SEED)
    qs, _ = datagen.queries_from_items(P, a.steps + a.warmup, SEED)
    rng = np.random.default_rng(0)
    from oracle import rmips_oracle as O
    per_step = max(64, int(a.n * 0.0005))
    for w in range(a.warmup):
        O.decide_users(Q, P, qs[w], a.k, rng.choice(a.n, 64, replace=False))
    times = []
    for s in range(a.steps):
        users = rng.choice(a.n, per_step, replace=False)
        t0 = time.perf_counter()
        O.decide_users(Q, P, qs[a.warmup + s], a.k, users)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    qps = a.steps * (per_step / a.n) / tot
    sample = (f"each step: the oracle decides {per_step} random users of one query (fraction "
              f"{per_step / a.n:.2e} of a query) over all {a.m} items in float64 numpy")
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(a),
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def result_sizes(offs):
    """Distribution of the per-query result sizes of one batch (CSR offsets)."""
    if offs is None or len(offs) < 2:
        return None
    sz = np.diff(np.asarray(offs, dtype=np.int64))
    out = {"queries": int(len(sz)), "total": int(sz.sum()), "max": int(sz.max())}
    for p in (50, 90, 99, 99.9):
        out[f"p{p}"] = float(np.percentile(sz, p))
    for lo, hi in ((0, 0), (1, 32), (33, 8192), (8193, None)):
        m = (sz >= lo) if hi is None else ((sz >= lo) & (sz <= hi))
        key = f"{lo}+" if hi is None else f"{lo}-{hi}"
        out[f"n_{key}"] = int(m.sum())
        out[f"ids_{key}"] = int(sz[m].sum())
    return out


# --------------------------------------------------------------------------- ranks
def reduce_over_ranks(ms: float, units: float, dist=None, device=None):
    """Max of the timed milliseconds and sum of the processed units over ranks.

    Every rank runs an independent replica (the path shards by users with no
    exchange step), so whole-job throughput is total units / slowest rank."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(units)
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_u, op=dist.ReduceOp.SUM)
    return float(t_ms.item()), float(t_u.item())


# --------------------------------------------------------------------------- serving
def serving_requests(P, n, d, n_req, seed):
    """The serving workload's requests: q a random item of P or a random
    N(0, I/d) vector (half each), k uniform in 1..25, and a user segment: none
    (a third), a contiguous id range of log-uniform size in 1e3..1e6 (a third)
    or one of 8 random id subsets of log-uniform size in 1e3..1e6 (a third).
    Returns (qs, ks, segs, subsets); segs[i] is None, (lo, hi) or ("subset", j)."""
    rng = np.random.default_rng(seed)
    qi, _ = datagen.queries_from_items(P, n_req, seed)
    qr = datagen.random_queries(n_req, d, seed)
    pick = rng.random(n_req) < 0.5
    qs = np.where(pick[:, None], qi, qr).astype(np.float32)
    ks = rng.integers(1, 26, n_req).astype(np.int32)
    hi_size = min(n, 1_000_000)
    subsets = [np.sort(rng.choice(n, int(min(hi_size, 10 ** rng.uniform(3, 6))), replace=False)) for _ in range(8)]
    segs = []
    for i in range(n_req):
        r = i % 3
        if r == 0:
            segs.append(None)
        elif r == 1:
            size = int(min(hi_size, 10 ** rng.uniform(3, 6)))
            lo = int(rng.integers(0, max(1, n - size + 1)))
            segs.append((lo, lo + size))
        else:
            segs.append(("subset", int(rng.integers(0, 8))))
    return qs, ks, segs, subsets


def serve_rates(rmips, index, qs, ks, segs, subsets, rates, n_serve, n_plain, opts):
    """Served and plain latency at each offered Poisson rate (see run_serving)."""
    import threading
    out = []
    for rate in rates:
        nr = min(len(qs), n_serve[rate])
        rng = np.random.default_rng(int(rate))
        arrive = np.cumsum(rng.exponential(1.0 / rate, nr))
        srv = rmips.Server(index, **opts)
        handles = [srv.add_segment(x) for x in subsets]
        sseg = [(("registered", handles[sg[1]]) if isinstance(sg, tuple) and sg[0] == "subset" else sg)
                for sg in segs[:nr]]
        groups, lags = [], np.zeros(nr)
        done_groups = []

        def collect():
            i = 0
            while True:
                if i < len(groups):
                    g0, g1, tk = groups[i]
                    if tk is None:
                        break
                    _, _, lat = srv.wait_many(tk)
                    done_groups.append((g0, g1, lat))
                    i += 1
                else:
                    time.sleep(0.0001)

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        i = 0
        while i < nr:
            now = time.perf_counter() - t0
            if arrive[i] > now:
                continue
            j = i
            while j < nr and arrive[j] <= now and j - i < 1024:
                j += 1
            tk = srv.submit_many(qs[i:j], ks[i:j], sseg[i:j])
            lags[i:j] = (time.perf_counter() - t0) - arrive[i:j]
            groups.append((i, j, tk))
            i = j
        groups.append((nr, nr, None))
        th.join()
        el = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat_s = np.zeros(nr)
        for g0, g1, lat in done_groups:
            lat_s[g0:g1] = lat + 1e3 * lags[g0:g1]
        served = {"offered_qps": rate, "requests": nr, "achieved_qps": nr / el,
                  "p50_ms": float(np.percentile(lat_s, 50)), "p99_ms": float(np.percentile(lat_s, 99)),
                  "max_ms": float(lat_s.max()), "mean_batch": st["mean_batch"], "batches": st["batches"],
                  "mean_submit_lag_ms": float(1e3 * lags.mean())}
        npl = min(nr, n_plain[rate])
        plat = np.zeros(npl)
        t0 = time.perf_counter()
        for i in range(npl):
            while time.perf_counter() - t0 < arrive[i]:
                pass
            sg = segs[i]
            if isinstance(sg, tuple) and sg[0] == "subset":
                sg = subsets[sg[1]]
            rmips.rmips_query(index, qs[i], int(ks[i]), segment=sg)
            plat[i] = (time.perf_counter() - t0) - arrive[i]
        pel = time.perf_counter() - t0
        plain = {"offered_qps": rate, "requests": npl, "achieved_qps": npl / pel,
                 "p50_ms": float(1e3 * np.percentile(plat, 50)), "p99_ms": float(1e3 * np.percentile(plat, 99)),
                 "max_ms": float(1e3 * plat.max())}
        out.append({"served": served, "plain": plain})
    return out


def run_serving(rmips, index, P, a):
    """Served (rmips_server_*) against plain (one rmips_query per request)
    latency at the same offered loads.  Arrivals follow a Poisson process at
    each rate; a request's latency runs from its scheduled arrival to the
    moment its result is available to the caller (for the server: the
    library's submit-to-completion time plus the submitter's lag behind the
    schedule).  The plain path takes the requests in arrival order on one
    host thread, so at a rate above what it can carry its queue, and its
    latency, grow for as long as the run lasts.  Two workloads: the serving
    workload with segments, and the same requests without segments (which the
    plain path can carry at 20k requests/s)."""
    n_req = min(a.serve_requests, 100_000)
    qs, ks, segs, subsets = serving_requests(P, a.n, a.d, max(n_req, 1), 41)
    opts = dict(max_batch=4096, max_wait_us=0, streams=2, max_pending=1 << 21, spin_us=200)
    warm = rmips.Server(index, **opts)
    warm.wait_many(warm.submit_many(qs[:4096], ks[:4096]))
    warm.close()
    out = {"workload": "Poisson arrivals; q = random item of P or random N(0, I/d) (half each); k uniform in "
                       "1..25; segment: none / contiguous id range / registered random id subset (a third each), "
                       "segment sizes log-uniform in 1e3..1e6",
           "server": "rmips_server: max_batch 4096, max_wait_us 0 (a batch closes as soon as one of the 2 "
                     "stream slots is free; requests queue while both are busy), spin_us 200 (server threads "
                     "and the waiting caller poll before blocking), batches of up to 4 requests as one-launch "
                     "single queries; admission by device result memory",
           "plain": "rmips_query per request on one host thread, host q and ids, segments as id ranges / id lists"}
    out["with_segments"] = serve_rates(rmips, index, qs, ks, segs, subsets, [20_000.0, 200_000.0, 1_000_000.0],
                                       {20_000.0: 10_000, 200_000.0: 40_000, 1_000_000.0: n_req},
                                       {20_000.0: 3_000, 200_000.0: 3_000, 1_000_000.0: 3_000}, opts)
    none = [None] * len(qs)
    out["without_segments"] = serve_rates(rmips, index, qs, ks, none, [], [5_000.0, 20_000.0, 200_000.0],
                                          {5_000.0: 5_000, 20_000.0: 10_000, 200_000.0: 40_000},
                                          {5_000.0: 5_000, 20_000.0: 10_000, 200_000.0: 4_000}, opts)
    return out


# --------------------------------------------------------------------------- extras
def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def simpfer_cpu_baseline(Q, P, qs, k, k_max, seconds=10.0):
    """The CPU Simpfer (Algorithms 1-3 in float64 with exact ties, OpenMP over
    blocks, |P'| = 4 k_max) on all host cores and on one core: queries/s."""
    from oracle import simpfer_cpu as S
    t0 = time.perf_counter()
    idx = S.SimpferCPU(Q, P, k_max=k_max, p_prime=4 * k_max, threads=0)
    build_s = time.perf_counter() - t0
    out = {"kind": "cpu simpfer (Algorithm 3 with Algorithm 2, float64, exact ties)", "p_prime": 4 * k_max,
           "index_build_s": build_s, "cpu_model": cpu_model(), "openmp": S.openmp()}
    for label, threads in (("all_cores", 0), ("one_core", 1)):
        n_done, t0 = 0, time.perf_counter()
        while n_done < len(qs) and (time.perf_counter() - t0 < seconds / 2 or n_done < 3):
            idx.query(qs[n_done], k, threads=threads)
            n_done += 1
        el = time.perf_counter() - t0
        out[label] = {"value": n_done / el, "unit": "queries/s", "queries": n_done,
                      "cores": S.max_threads() if threads == 0 else 1, "ms_per_query": 1e3 * el / n_done}
    idx.close()
    return out


def ip_error_report(Q, qs, d, rmips, torch, dev):
    """Largest error of the tensor-core inner products against float64 on
    tiles of the workload: the 128 largest-norm users and 128 random users
    against 64 of the queries, each padded to K = 64, per operand kind."""
    bound = {"tf32": 0.00198, "bf16": 0.00788, "fp16": 0.000995}
    un = np.linalg.norm(Q.astype(np.float64), axis=1)
    rng = np.random.default_rng(0)
    rep = {}
    for kind in ("tf32", "bf16", "fp16"):
        worst_rel, worst_abs = 0.0, 0.0
        for users in (np.argsort(-un)[:128], rng.choice(Q.shape[0], 128, replace=False)):
            for q0 in range(0, min(len(qs), 256), 64):
                A = np.zeros((128, 64), np.float32)
                B = np.zeros((64, 64), np.float32)
                A[:, :d] = Q[users]
                B[:min(64, len(qs) - q0), :d] = qs[q0:q0 + 64]
                dD = torch.zeros((128, 64), dtype=torch.float32, device=dev)
                rmips.rmips_debug_tc_tile(torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), dD, kind=kind)
                ref = A.astype(np.float64) @ B.astype(np.float64).T
                nrm = np.linalg.norm(A.astype(np.float64), axis=1)[:, None] * np.linalg.norm(B.astype(np.float64), axis=1)
                err = np.abs(dD.cpu().numpy().astype(np.float64) - ref)
                ok = nrm > 0
                worst_abs = max(worst_abs, float(err.max()))
                worst_rel = max(worst_rel, float((err[ok] / nrm[ok]).max()))
        rep[kind] = {"max_abs_ip_err": worst_abs, "max_rel_ip_err": worst_rel, "rel_bound": bound[kind],
                     "rel_err_over_bound": worst_rel / bound[kind]}
    rep["note"] = ("relative to ||u|| ||q||; the filter charges every product its bound and rechecks any "
                   "decision within it exactly, so the sets stay exact")
    return rep


def time_async_batches(rmips, torch, index, dqs, dks, nq, steps, dev, first=0):
    """Queries/s of `steps` asynchronous batches on two streams (after two warm-up batches)."""
    streams = [torch.cuda.current_stream(dev), torch.cuda.Stream(dev)]
    cap = max(1 << 20, nq * 2048)
    outs = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(2)]
    offs = torch.empty((steps + 2, nq + 1), dtype=torch.int64, device=dev)
    done = torch.full((steps + 2, 2), -1, dtype=torch.int64, device=dev)
    nb = dqs.shape[0] // nq

    def run(i0, cnt):
        for i in range(cnt):
            b = (first + i0 + i) % nb
            rmips.rmips_query_batch_async(index, dqs[b * nq:(b + 1) * nq], dks[:nq], outs[i & 1], offs[i0 + i],
                                          done[i0 + i], streams[i & 1])
    run(0, 2)
    torch.cuda.synchronize(dev)
    ev0, ev1, side = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), torch.cuda.Event()
    ev0.record(streams[0])
    streams[1].wait_event(ev0)
    run(2, steps)
    side.record(streams[1])
    streams[0].wait_event(side)
    ev1.record(streams[0])
    torch.cuda.synchronize(dev)
    d = done.cpu().numpy()
    if (d[:, 0] != 0).any():
        raise RuntimeError(f"batch status {d[:, 0].tolist()}")
    ms = ev0.elapsed_time(ev1)
    return steps * nq / (ms / 1e3), ms / steps, int(d[2:, 1].sum())


def variants_report(a, Q, P, qs, rmips, torch, dev):
    """The batched step on other indexes of the same workload: the paper's
    "without blocks" ablation, other block sizes and the BF16 / FP16 filter."""
    out = {}
    dqs = torch.from_numpy(qs).to(dev)
    dks = torch.full((a.nq,), a.k, dtype=torch.int32, device=dev)
    specs = [("blocks_32_tf32", dict()), ("no_blocks", dict(block_filter=False)),
             ("blocks_64", dict(block_size=64)), ("blocks_128", dict(block_size=128)),
             ("blocks_256", dict(block_size=256)), ("bf16_filter", dict(precision="bf16")),
             ("fp16_filter", dict(precision="fp16"))]
    for name, kw in specs:
        index = rmips.rmips_build_index(Q, P, k_max=a.k_max, **kw)
        rmips.rmips_profile_enable(index, True)
        qps, ms, ids = time_async_batches(rmips, torch, index, dqs, dks, a.nq, 4, dev)
        prof = rmips.rmips_profile_read(index)
        rmips.rmips_profile_enable(index, False)
        ml = max(1, prof["mfilter_launches"])
        out[name] = {"queries_per_s": qps, "ms_per_batch": ms, "filter_ms": prof["mfilter_ms"] / ml,
                     "pairs_kept_by_lemma3_per_query": prof["mfilter_pairs"] / (ml * a.nq),
                     "results_per_query": ids / (4 * a.nq)}
        index.close()
    base = out["blocks_32_tf32"]["queries_per_s"]
    out["blocks_speedup_over_no_blocks"] = base / out["no_blocks"]["queries_per_s"]
    out["config"] = (f"{a.nq} queries per batch, k = {a.k}, 4 timed batches after 2 warm-up batches on two "
                     "streams; the paper reports 1.1-3.8x for blocks on its CPU")
    return out


def precision_workload(rmips, torch, dev, steps=3):
    """The precision workload at its stated size: |Q| = 500k, |P| = 100k,
    d = 64, k = 10, 2,000 item + 2,000 random queries in one batch, per
    filter precision, with the tiles' inner-product error."""
    n, m, d, k, seed = 500_000, 100_000, 64, 10, 2
    Q, P = datagen.make_problem(n, m, d, seed)
    qi, _ = datagen.queries_from_items(P, 2000, seed)
    qs = np.concatenate([qi, datagen.random_queries(2000, d, seed)])
    dqs = torch.from_numpy(qs).to(dev)
    dks = torch.full((len(qs),), k, dtype=torch.int32, device=dev)
    out = {"workload": f"reverse k-MIPS |Q|={n} |P|={m} d={d} k={k}, 2,000 item + 2,000 random queries per batch"}
    for prec in ("fp32", "bf16", "fp16"):
        index = rmips.rmips_build_index(Q, P, k_max=25, precision=prec)
        qps, ms, ids = time_async_batches(rmips, torch, index, dqs, dks, len(qs), steps, dev)
        ids_h, offs = rmips.rmips_query_batch(index, qs, np.full(len(qs), k, np.int32))
        st = rmips.rmips_last_query_stats(index)
        out[prec] = {"queries_per_s": qps, "ms_per_batch": ms, "results": int(offs[-1]),
                     "pairs_rechecked": st["todo"], "exact_integer_decisions": st["exact_calls"]}
        index.close()
    out["ip_error"] = ip_error_report(Q, qs, d, rmips, torch, dev)
    return out


# --------------------------------------------------------------------------- GPU arm
def run_ours(a):
    import torch
    from paper_2110_07131_gb300 import rmips

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    Q, P = datagen.make_problem(a.n, a.m, a.d, SEED)
    t0 = time.perf_counter()
    index = rmips.rmips_build_index(Q, P, k_max=a.k_max, block_size=a.block_size, p_prime=a.p_prime,
                                    block_filter=not a.no_blocks,
                                    precision=a.precision, batch_tensor_cores=(a.batch_kernel == "tc"))
    build_s = time.perf_counter() - t0
    info = index.info()

    total_q = (a.warmup + 1 + a.steps) * a.nq
    qs, _ = datagen.queries_from_items(P, total_q, SEED + 7919 * rank)
    ks = np.full(a.nq, a.k, np.int32)
    dqs = torch.from_numpy(qs).to(dev)
    dks = torch.from_numpy(ks).to(dev)
    cap = max(1 << 20, a.nq * 2048)
    dout = torch.empty(cap, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    last_offs = [None]

    def step(i):
        sl = dqs[i * a.nq:(i + 1) * a.nq]
        _, offs = rmips.rmips_query_batch(index, sl, dks, out=dout, stream=stream)
        last_offs[0] = offs
        return int(offs[-1])

    # Batches are queued through the asynchronous call on two streams in
    # turn: consecutive batches are independent, so one batch's short
    # preparation kernels overlap the previous batch's recheck and emission
    # (each stream slot has its own workspace and output buffer).
    streams = [stream, torch.cuda.Stream(dev)]
    douts = [dout, torch.empty(cap, dtype=torch.int64, device=dev)]

    def run_async(first, count, offs, done):
        for i in range(count):
            j = first + i
            rmips.rmips_query_batch_async(index, dqs[j * a.nq:(j + 1) * a.nq], dks, douts[i & 1], offs[i], done[i],
                                          streams[i & 1])

    sampler = ClockSampler(local)
    sampler.start()                                  # sampling already runs when the timed region starts
    # warm-up: an even number of batches (at least W), so that each of the two
    # workspaces has seen the batch shape twice and replays captured graphs
    n_warm = a.warmup + (a.warmup & 1)
    w_offs = torch.empty((n_warm, a.nq + 1), dtype=torch.int64, device=dev)
    w_done = torch.full((n_warm, 2), -1, dtype=torch.int64, device=dev)
    run_async(0, n_warm, w_offs, w_done)
    torch.cuda.synchronize(dev)
    if (w_done[:, 0].cpu().numpy() != 0).any():
        raise RuntimeError("warm-up batch failed")
    if dist:
        dist.barrier()
    a_offs = torch.empty((a.steps, a.nq + 1), dtype=torch.int64, device=dev)
    a_done = torch.full((a.steps, 2), -1, dtype=torch.int64, device=dev)
    rmips.rmips_profile_enable(index, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_side = torch.cuda.Event()
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    ev0.record(streams[0])
    streams[1].wait_event(ev0)
    run_async(n_warm, a.steps, a_offs, a_done)
    ev_side.record(streams[1])
    streams[0].wait_event(ev_side)
    ev1.record(streams[0])
    torch.cuda.synchronize(dev)
    t_wall1 = time.time()
    done_h = a_done.cpu().numpy()
    if (done_h[:, 0] != 0).any():
        raise RuntimeError(f"batch status {done_h[:, 0].tolist()}")
    results = int(done_h[:, 1].sum())
    timed_offs = a_offs[-1].cpu().numpy()
    prof = rmips.rmips_profile_read(index)
    rmips.rmips_profile_enable(index, False)
    clocks = sampler.stop(t_wall0, t_wall1)
    # pipeline counters of the tensor-core filter, and the query statistics
    # (kept by the synchronous call only): the last timed batch once more,
    # outside the timed region, with the instrumented kernel
    rmips.rmips_profile_enable(index, 2)
    step(n_warm + a.steps - 1)
    torch.cuda.synchronize(dev)
    pprof = rmips.rmips_profile_read(index)
    rmips.rmips_profile_enable(index, False)
    qstats = rmips.rmips_last_query_stats(index)
    last_offs[0] = timed_offs
    ms = ev0.elapsed_time(ev1)
    ms_max, units = reduce_over_ranks(ms, a.steps * a.nq, dist, dev)
    value = units / (ms_max / 1e3)

    # end to end through the public API with host buffers (copies inside the
    # timed region): the queries and their k in pinned host memory (numpy
    # views of pinned tensors), the results returned as a new host array.
    # Caller threads (three by default) keep as many synchronous calls in
    # flight, each on its own CUDA stream (the library gives each call its own
    # workspace), so one call's copies and host work overlap another's kernels.
    import threading
    hq = torch.empty((a.nq, a.d), dtype=torch.float32, pin_memory=True).numpy()
    hq[:] = qs[:a.nq]
    hks = torch.empty(a.nq, dtype=torch.int32, pin_memory=True).numpy()
    hks[:] = ks
    e2e_threads = max(1, a.e2e_threads)
    e2e_steps = max(3, min(a.steps, 10))
    e2e_streams = [torch.cuda.Stream(dev) for _ in range(e2e_threads)]
    for s_ in e2e_streams:
        rmips.rmips_query_batch(index, hq, hks, stream=s_)
    d2h = [0] * e2e_threads
    e2e_err = []

    def e2e_worker(i):
        try:
            for _ in range(e2e_steps):
                ids, offs = rmips.rmips_query_batch(index, hq, hks, stream=e2e_streams[i])
                d2h[i] += ids.nbytes + offs.nbytes
        except Exception as ex:                          # surfaced below
            e2e_err.append(ex)
    workers = [threading.Thread(target=e2e_worker, args=(i,)) for i in range(e2e_threads)]
    t0 = time.perf_counter()
    for w in workers:
        w.start()
    for w in workers:
        w.join()
    e2e_s = (time.perf_counter() - t0) / (e2e_threads * e2e_steps)
    if e2e_err:
        raise e2e_err[0]
    e2e = {"value": a.nq / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": int(hq.nbytes + hks.nbytes),
           "d2h_bytes_per_step": int(sum(d2h) // (e2e_threads * e2e_steps)), "inputs": "pinned host memory",
           "api": f"rmips_query_batch (synchronous, host arrays in and out) from {e2e_threads} caller "
                  f"thread(s), each on its own CUDA stream, {e2e_threads} call(s) in flight"}

    # plain path: one query per call, host buffers, per-call latency
    lat, sizes = [], []
    for j in range(a.plain_queries):
        t1 = time.perf_counter()
        r = rmips.rmips_query(index, qs[j], a.k)
        lat.append((time.perf_counter() - t1) * 1e3)
        sizes.append(len(r))
    skip = 5 if len(lat) > 10 else 0
    lat_s = np.array(lat[skip:])
    slow = np.argsort(-lat_s)[:5]
    plain = {"qps": 1e3 / lat_s.mean(), "p50_ms": float(np.percentile(lat_s, 50)),
             "p99_ms": float(np.percentile(lat_s, 99)), "queries": int(len(lat_s)),
             "api": "rmips_query, host q and host ids, one query per call",
             "slowest": [[float(lat_s[i]), int(sizes[skip + i])] for i in slow],
             "largest_result": int(max(sizes))}

    serving = run_serving(rmips, index, P, a) if a.serve_requests > 0 else None

    # the top-k join over all users (Definition 1 for every user), device output
    join_s = None
    if a.p_prime == 0 and a.k <= a.k_max:
        jout = torch.empty((a.n, a.k), dtype=torch.int64, device=dev)
        rmips.rmips_topk_join(index, a.k, out=jout)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rmips.rmips_topk_join(index, a.k, out=jout)
        join_s = time.perf_counter() - t0
        del jout

    # single queries, one launch each, device-resident: bursts of 400
    # launches queued back to back on one stream behind a short device-side
    # sleep (torch.cuda._sleep, a bounded spin), so that the host has queued
    # the whole burst before the GPU reaches it and the timed region holds no
    # host gaps; CUDA events around each burst give the device time per
    # query, and the event pairs the library records around each launch give
    # the kernel's launch duration for the roofline
    single = None
    s_total_ms, ns1 = 0.0, 0
    sprof = {"filter_launches": 0, "filter_alg_bytes": 0.0, "filter_ms": 0.0, "users_tested": 0,
             "blocks_pruned": 0, "blocks_total": 1}
    if a.single_queries > 0:
        ns1 = min(a.single_queries, dqs.shape[0])
        burst = 400
        sout = torch.empty((2, max(1 << 16, a.n // 8)), dtype=torch.int64, device=dev)
        sdone = torch.full((ns1, 2), -1, dtype=torch.int64, device=dev)
        for j in range(20):                                    # warm-up (both workspaces)
            rmips.rmips_query_async(index, dqs[j], a.k, sout[j & 1], sdone[j], stream=stream)
        torch.cuda.synchronize(dev)
        def bursts():
            total = 0.0
            for b0 in range(0, ns1, burst):
                b1 = min(ns1, b0 + burst)
                torch.cuda._sleep(int(2e6 * 25))             # ~25 ms at 2 GHz
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for j in range(b0, b1):
                    rmips.rmips_query_async(index, dqs[j], a.k, sout[j & 1], sdone[j], stream=stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                total += e0.elapsed_time(e1)
            return total
        s_total_ms = bursts()                                  # throughput, profiling off
        rmips.rmips_profile_enable(index, True)                 # kernel launch times for the roofline
        bursts()
        sprof = rmips.rmips_profile_read(index)
        rmips.rmips_profile_enable(index, False)
        sd = sdone.cpu().numpy()
        if (sd[:, 0] != 0).any():
            raise RuntimeError(f"single query status {sorted(set(sd[:, 0].tolist()))}")
        single = {"qps": ns1 / (s_total_ms / 1e3), "us_per_query": 1e3 * s_total_ms / ns1, "queries": ns1,
                  "results_per_query": float(sd[:, 1].mean()),
                  "api": "rmips_query_async (one k_query1 launch per query), device q and ids, bursts of 400 "
                         "launches queued back to back on one stream"}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    sl = sprof["filter_launches"] or 1
    s_bytes = sprof["filter_alg_bytes"] / sl
    s_ms = sprof["filter_ms"] / sl                       # per launch, events around each launch (no overlap)
    # per launch in steady state: the unprofiled bursts' device time / launches
    # (consecutive launches overlap: the next query's CTAs start as SMs free up)
    s_ms_burst = s_total_ms / ns1 if ns1 else 0.0
    s_ach = s_bytes / (s_ms_burst / 1e3) / 1e9 if s_ms_burst > 0 else 0.0
    roof_single = {"bound": "hbm", "kernel": "k_query1 (one launch per query, one CTA per SM: a producer warp "
                                             "tests Lemma 3 for 32 spans at once and bulk-copies each run of kept "
                                             "32-user chunks; 10 consumer warps apply Lemmas 1/2 and recheck exactly; "
                                             "the last CTA emits)",
                   "achieved": s_ach, "peak": hbm, "unit": "GB/s", "frac": s_ach / hbm, "peak_source": peak_src,
                   "traffic": None, "alg_bytes_per_launch": s_bytes, "avg_launch_us": s_ms_burst * 1e3,
                   "avg_launch_us_isolated": s_ms * 1e3, "launches": sprof["filter_launches"],
                   "users_tested_per_query": sprof["users_tested"] / sl,
                   "alpha_blocks_pruned": sprof["blocks_pruned"] / max(1, sprof["blocks_total"]),
                   "timing": "back-to-back device-resident launches (rmips_query_async): CUDA events around bursts "
                             "of 400 launches on the launching stream give the time per launch (consecutive "
                             "launches overlap); avg_launch_us_isolated: the library's events around each launch, "
                             "which keep launches apart; bytes from the library's counters"}
    # FP32 FMA peak from unit counts and clock: SMs x 128 lanes x 2 flop x clock
    import torch as _t
    sms = _t.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0)
    alu_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    ml = prof["mfilter_launches"] or 1
    m_flops = prof["mfilter_alg_flops"] / ml
    m_ms = prof["mfilter_ms"] / ml
    m_ach = m_flops / (m_ms / 1e3) / 1e12 if m_ms > 0 else 0.0
    tc_path = a.batch_kernel == "tc" and a.d <= 64
    # DRAM bytes (read + write) of one k_mfilter_ws launch on the default
    # workload, from one ncu capture of the current kernel (241.1 MB + 4.1 MB)
    default_workload = (a.n, a.m, a.d, a.k, a.k_max, a.nq) == (1_000_000, 500_000, 50, 10, 25, 10_000)
    tc_traffic = 245.2e6 if (tc_path and default_workload and a.block_size == 32 and not a.no_blocks
                             and a.precision == "fp32") else None
    if tc_path:
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        if a.precision == "fp32":
            op, tc_peak = "TF32", bf16 * (1.1 / 2.25)
            peak_source = f"measured bf16 {bf16:.0f} TFLOP/s x nominal TF32/BF16 ratio 1.1/2.25"
        else:
            op, tc_peak = a.precision.upper(), bf16
            peak_source = f"measured bf16 {bf16:.0f} TFLOP/s (FP16 and BF16 share the rate)"
        roofline = {"bound": "tensor", "kernel": f"k_mfilter_ws (warp-specialized: TMA-fed tcgen05 {op} "
                                                  "128x128xK tiles into 4 TMEM stages + Lemmas 1/2 epilogue, "
                                                  "four MMA warps and two epilogue warp sets on alternate items)",
                    "achieved": m_ach, "peak": tc_peak, "unit": "TFLOP/s", "frac": m_ach / tc_peak,
                    "peak_source": peak_source,
                    "traffic": tc_traffic, "alg_flops_per_launch": m_flops, "avg_launch_ms": m_ms,
                    "pairs_per_launch": prof["mfilter_pairs"] / ml,
                    "tiles_per_launch": pprof["mfilter_tiles"] / max(1, pprof["mfilter_launches"]),
                    "filter_share_of_step": prof["mfilter_ms"] / ms if ms > 0 else None}
        cyc = pprof["mfilter_cycles"]
        waits = pprof["mfilter_wait"]
        names = ["loader_waits_free_slot", "feeder_waits_free_stage", "mma_waits_query_tile",
                 "mma_waits_free_accumulator", "epilogue_waits_accumulator", "mma_waits_user_tile",
                 "epilogue_reads_tmem", "mma_issues_mmas", "epilogue_per_pair_tests",
                 "epilogue_items_with_per_pair_tests", "epilogue_appends_pairs"]
        owner = [0, 1, 2, 2, 3, 2, 3, 2, 3, None, 3]
        roofline["active_tiles_per_launch"] = pprof["mfilter_active_tiles"] / max(1, pprof["mfilter_launches"])
        roofline["pipeline_wait_share"] = {n: (waits[i] if owner[i] is None else
                                               (waits[i] / cyc[owner[i]] if cyc[owner[i]] > 0 else None))
                                           for i, n in enumerate(names)}
    else:
        roofline = {"bound": "alu", "kernel": "k_mfilter (multi-query Lemma 3 prefixes + FP32 FFMA tiles + "
                                              "Lemmas 1/2 epilogue)",
                    "achieved": m_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": m_ach / alu_peak,
                    "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                    "traffic": None, "alg_flops_per_launch": m_flops, "avg_launch_ms": m_ms,
                    "pairs_per_launch": prof["mfilter_pairs"] / ml,
                    "filter_share_of_step": prof["mfilter_ms"] / ms if ms > 0 else None}

    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ({"fp32": "tf32", "fp16": "f16", "bf16": "bf16"}[a.precision] if tc_path
                      else ("f32" if a.precision == "fp32" else a.precision)) + "+f64 recheck",
            "data": "synthetic",
            "config": workload(a), "e2e": e2e, "roofline": roofline, "clocks": clocks,
            "gpu_launches": a.steps * ((16 if a.batch_kernel == "tc" and a.d <= 64 else 15) * ((a.nq + 16383) // 16384) + 1),
            "pipelining": f"each step one asynchronous batch call; batches queued on 2 CUDA streams in turn, "
                          f"each with its own workspace (independent batches overlap); {n_warm} untimed "
                          f"warm-up batches",
            "roofline_single_query_filter": roof_single, "single_query_device": single,
            "p50_ms": plain["p50_ms"], "p99_ms": plain["p99_ms"], "plain": plain, "serving": serving,
            "batch_latency_ms": ms_max / a.steps,
            "index_build_s": build_s, "index_device_bytes": info["device_bytes"],
            "topk_join_s": join_s,
            "index_incomplete_users": info["incomplete"],
            "users_returned_per_query": results / (a.steps * a.nq),
            "result_sizes_last_step": result_sizes(last_offs[0]),
            "pairs_kept_by_lemma3_per_query": prof["mfilter_pairs"] / (a.steps * a.nq),
            "last_step": {"pairs_decided_yes_in_o1": qstats["yes_fast"], "pairs_rechecked": qstats["todo"],
                          "exact_integer_decisions": qstats["exact_calls"], "results": qstats["result"]}}
    if rank == 0 and world == 1 and not a.no_extras:
        line["ip_error"] = ip_error_report(Q, qs[:256], a.d, rmips, torch, dev)
        index.close()
        index = None
        line["variants"] = variants_report(a, Q, P, qs[:4 * a.nq], rmips, torch, dev)
        line["precision_workload"] = precision_workload(rmips, torch, dev)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rng = np.random.default_rng(1)
        qps, s, t, cores = oracle_sample(Q, P, qs[0], a.k, a.cpu_seconds, rng)
        line["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                "sample": f"one query, {s} random users decided over all {a.m} items "
                                          f"in float64 numpy ({t:.1f} s), scaled to queries/s"}
        if not a.no_extras:
            line["cpu_baseline_simpfer"] = simpfer_cpu_baseline(Q, P, qs[:400], a.k, a.k_max)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if index is not None:
        index.close()
    if dist:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
