#!/usr/bin/env python
"""Exact RNG construction throughput (edges/s) on one GB300 per rank.

One step = the whole hot path over one synthetic workload: every pivot layer built
(assignment, radii, delta_max), every layer's GRNG linked (coarsest first), the
exemplar RNG built and its sorted edge list produced, all through the C ABI.

Workload: "lin96" -- 1,000,000 points in R^96 with intrinsic dimension 8
(x = A z + 0.01 eps, z ~ N(0, I_8), A_ij ~ N(0, 1/8)), L2, three nested random pivot
layers of 1,024 / 16,384 / 131,072 pivots.  The points (384 MB) exceed the 129 MB L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Under torchrun each rank builds its own replica (the build is not split across GPUs);
value = edges of all ranks / the slowest rank's time.
"""
import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact RNG edges/s at 1M pts: BF16+learned vs plain FP32, edges = oracle"
UNIT = "edges/s"
L2_BYTES = 129 * 1000 * 1000  # GB300 L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=None, help="points (default: the full 1,000,000)")
    ap.add_argument("--kind", default="lin96")
    ap.add_argument("--metric", default="l2", choices=["l2", "l1"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"],
                    help="distance tiles of the exemplar level: tensor cores (bf16) or CUDA cores (fp32)")
    ap.add_argument("--no-compare", action="store_true", help="skip the one-step plain FP32 comparison")
    ap.add_argument("--no-learned", action="store_true",
                    help="bf16 without the learned shortlist (by default the network is trained, untimed, on a "
                         "200,000-point build of the same generator and an 8-candidate shortlist is used)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=12000, help="points of the oracle's bounded sample")
    ap.add_argument("--check-rows", type=int, default=1000,
                    help="after timing, compare this many seeded points' RNG neighbourhoods with the FP64 oracle's "
                         "exact rows (0: skip)")
    ap.add_argument("--plain-steps", type=int, default=3,
                    help="timed steps of the plain FP32 comparison build (after one warm-up step)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="timed steps of the end-to-end measurement")
    ap.add_argument("--insert", type=int, default=0, metavar="B",
                    help="instead of the build benchmark: insert B batches of uneven size (log-uniform in "
                         "[1,000, 65,536] points, scaled to --n) into an index built on the rest, and print "
                         "points/s and per-batch latency")
    ap.add_argument("--skeleton", type=float, default=0.0, metavar="BETA",
                    help="instead of the build benchmark: the lune-based beta-skeleton (1 <= BETA <= 2) of the "
                         "workload, timed after the pivot layers")
    ap.add_argument("--search", type=int, default=0, metavar="B",
                    help="instead of the build benchmark: B batches of --search-m queries (RNG search)")
    ap.add_argument("--search-m", type=int, default=1000, help="queries per search batch")
    ap.add_argument("--no-search-leg", action="store_true",
                    help="build benchmark: skip the search of 5 x 1,000 queries on an index of the workload")
    ap.add_argument("--search-check", type=int, default=32,
                    help="queries of the first batch compared with the oracle (FP64 on the host)")
    ap.add_argument("--insert-verify", action="store_true",
                    help="with --insert: compare the final edges with a build from scratch on all points")
    return ap.parse_args()


def max_over_ranks(ms, pg, device):
    """The slowest rank's time (all ranks get it); `pg` is torch.distributed or None."""
    if pg is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(edges_per_rank, world, ms):
    """Whole-job throughput of replicas: every rank builds the same workload, so the job
    produced edges_per_rank x world edges in the slowest rank's time."""
    return edges_per_rank * world / (ms / 1000.0)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = list(csv.reader(io.StringIO(open(self.f.name).read())))
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_rooflines(stats, n, D, precision, peaks, sms):
    """Roofline entries of the exemplar tile sweep and of each level's tile sweeps and
    tier-3 kernel.  Algorithmic work per unit:
      exemplar Gram tiles (tcgen05): 2*D flops per unordered pair of points;
      FP32 tiles (CUDA cores): 2*D lane instructions (subtract + FMA) per unordered pair;
      tier 3: 2 distances (to both endpoints) x 2*D lane instructions per node tested;
      range-list tier: 8 bytes (node id and key) per list entry read, plus one padded row
      (4*Dp bytes) per listed node tested by distance -- a streaming bound against HBM;
      assignment: 2*D flops (tensor cores) or lane instructions (FP32 tiles) per (member, pivot).
    Peaks: bf16 sustained tensor rate from MEASURED_PEAKS.json (the kernels run inside a
    long step); FP32 lanes: SMs x 128 x the maximum SM clock (derived)."""
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    alu = sms * 128 * sm_max / 1000.0  # Gop/s
    bf = peaks.get("bf16_tflops_sustained")
    bf_src = "MEASURED_PEAKS bf16_tflops_sustained (of measured)" if bf else "fallback 1700 TFLOP/s sustained"
    bf = bf or 1700.0
    alu_src = f"derived: {sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (MEASURED_PEAKS sm_max_mhz)"
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS hbm_gbs (of measured)" if peaks.get("hbm_gbs") else "fallback 6800 GB/s"
    Dp = D if D <= 8 else (16 if D <= 16 else ((D + 31) // 32) * 32)
    out = []

    def add(kernel, bound, ms, work, unit, peak, src):
        if ms <= 0:
            return
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = work / (ms / 1000.0) / scale
        out.append({"kernel": kernel, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                    "frac": ach / peak, "traffic": None, "peak_source": src, "work_per_launch": work,
                    "launch_ms": ms})

    pairs = n * (n - 1) / 2
    km = stats["rng"].get("kernel_ms", {})
    if precision == "bf16":
        add("tc_sweep_kernel (exemplar Gram tiles, tcgen05 split-BF16)", "tensor", km.get("tiles", 0),
            pairs * 2 * D, "TFLOP/s", bf, bf_src)
    else:
        add("tile_pass_kernel (exemplar tiles, FP32 CUDA cores)", "alu", km.get("tiles", 0),
            pairs * 2 * D, "Gop/s", alu, alu_src)
    add("tier3_kernel (exemplar level)", "alu", km.get("tier3", 0),
        stats["rng"]["tier3_nodes_tested"] * 2 * 2 * D, "Gop/s", alu, alu_src)
    nmem = n
    for L in reversed(stats["layers"]):  # finest first: its members are the points
        m = L["m"]
        if L.get("assign_kernel_ms", 0) > 0:
            if L.get("assign_tensor_cores"):
                add(f"tc_assign_kernel (pivot layer m={m}, members {nmem})", "tensor", L["assign_kernel_ms"],
                    nmem * m * 2 * D, "TFLOP/s", bf, bf_src)
            else:
                add(f"assign_tile_kernel (pivot layer m={m}, members {nmem})", "alu", L["assign_kernel_ms"],
                    nmem * m * 2 * D, "Gop/s", alu, alu_src)
        nmem = m
    for L in stats["layers"]:
        m, G = L["m"], L["grng"]
        k = G.get("kernel_ms", {})
        add(f"tile_pass_kernel (pivot layer m={m}, two sweeps)", "alu", k.get("tiles", 0),
            m * (m - 1) / 2 * 2 * D, "Gop/s", alu, alu_src)
        add(f"tier3_kernel (pivot layer m={m})", "alu", k.get("tier3", 0),
            G["tier3_nodes_tested"] * 2 * 2 * D, "Gop/s", alu, alu_src)
        add(f"list_tier_kernel (pivot layer m={m})", "hbm", k.get("lists", 0),
            G.get("range_entries_read", 0) * 8 + G.get("range_nodes_tested", 0) * 4 * Dp, "GB/s", hbm, hbm_src)
    out.sort(key=lambda r: -r["launch_ms"])
    top = dict(out[0])
    top["traffic"] = measured_traffic(top["kernel"], n)
    top["others"] = [{k: r[k] for k in ("kernel", "bound", "achieved", "unit", "frac", "launch_ms")} for r in out[1:6]]
    return top


def train_shortlist(g, wl, kind, n_train=200000, k=8):
    """Untimed: record the exhaustive tier's candidate pools of one 200,000-point build of
    the same generator (other seeds), train the ranking network on the GPU, return it."""
    import numpy as np
    t0 = time.perf_counter()
    w = wl.make(kind, n=n_train, data_seed=7001, pivot_seed=7002)
    ix, _ = g.build_all(w.X, w.layers, flags=g.GRNG_FLAG_RECORD_MLP)
    F, y = ix.mlp_dataset()
    ix.close()
    pos = float(y.mean()) if y.size else 0.0
    if y.size == 0 or pos in (0.0, 1.0):
        return None
    wts = np.where(y > 0.5, 0.5 / pos, 0.5 / (1.0 - pos)).astype(np.float32)
    perm = np.random.default_rng(7003).permutation(F.shape[0])
    P, loss = g.mlp_train(g.mlp_init(7004), F[perm], y[perm], wts[perm], epochs=6, batch=4096, lr=1e-3)
    return {"params": P, "k": k, "train_points": n_train, "samples": int(F.shape[0]),
            "positives": int(y.sum()), "train_s": time.perf_counter() - t0, "final_loss": loss}


# Revision tags of the kernels whose DRAM traffic was captured with ncu (profiles/*traffic*.json);
# a kernel changed since its capture gets a new tag here, and its traffic reads as null.
KERNEL_REVS = {"tc_sweep_kernel": "chunk-bound"}  # the form captured at 1M


def measured_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` at n points from a committed ncu capture, or None."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "profiles", "*traffic*.json")):
        try:
            t = json.load(open(f))
        except ValueError:
            continue
        base = t.get("kernel", "").split(" ")[0]
        if t.get("kernel") == kernel and t.get("n") == n and KERNEL_REVS.get(base) == t.get("rev"):
            return t.get("dram_bytes_per_launch")
    return None


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(kind, n_sample, seed=3002, threads=None):
    """The FP64 oracle (brute force over all triples, Eq. 1) on a bounded sample, on all
    the host's cores or on `threads` of them."""
    import oracle
    from paper_2208_10022_gb300 import workloads as wl
    w = wl.make(kind, n=n_sample, data_seed=seed)
    prev = oracle.set_threads(threads) if threads else None
    try:
        t0 = time.perf_counter()
        E = oracle.rng_brute(w.X)
        dt = time.perf_counter() - t0
    finally:
        if prev:
            oracle.set_threads(prev)
    cores = threads or oracle.max_threads()
    return {"value": len(E) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"rng_brute on a seeded {n_sample}-point sample of the {kind} generator "
                      f"({len(E)} edges in {dt:.2f} s)", "seconds": dt, "edges": int(len(E))}


def cpu_model():
    """The host CPU's model name (lscpu), or the architecture when lscpu is absent."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def step_measures(stats, step_ms):
    """Work counters of one step, from the library's statistics (grng_stats):
    candidate lune tests are the candidate pairs every level decides (tier 1 to the FP64
    recheck), interceptor evaluations the exact tests of one interceptor against one pair
    outside the tile sweeps (tier 3, range-list distance tests, the learned shortlist), the
    recheck fraction the FP64 triples among those evaluations."""
    levels = [L["grng"] for L in stats["layers"]] + [stats["rng"]]
    cand = sum(L["candidate_pairs"] for L in levels)
    ev = sum(L["tier3_nodes_tested"] + L["range_nodes_tested"] + L["learned_tests"] for L in levels)
    fp64 = sum(L["fp64_triples"] for L in levels)
    s = step_ms / 1000.0
    n = stats["n"]
    # distance computations, the paper's cost measure (Sec. 1), by where they are made: tile
    # sweeps count every key of every tile (both orientations), the assignment every
    # member x pivot key, the exact tiers each tested interceptor (two distances in tier 3)
    ms = [L["m"] for L in stats["layers"]]
    blk = lambda k: ((k + 127) // 128) ** 2 * 128 * 128
    dist = {"exemplar_tiles": blk(n), "assignment": n * ms[-1] + sum(ms[i + 1] * ms[i] for i in range(len(ms) - 1)),
            "pivot_layer_tiles": sum(2 * blk(m) + (2 * blk(m) if L["grng"]["range_pairs"] else 0)
                                     for m, L in zip(ms, stats["layers"])),
            "node_ancestor_tables": sum(m * sum(ms[:i]) for i, m in enumerate(ms) if L_has_tier3(stats, i)),
            "exact_tiers": sum(2 * L["tier3_nodes_tested"] + L["range_nodes_tested"] + 2 * L["learned_tests"]
                               for L in levels)}
    dist["total"] = sum(dist.values())
    return {"candidate_pairs_per_step": cand, "candidate_lune_tests_per_s": cand / s,
            "exemplar_candidate_pairs": stats["rng"]["candidate_pairs"],
            "exemplar_pairs_of_all": stats["rng"]["candidate_pairs"] / max(1.0, n * (n - 1) / 2),
            "interceptor_evaluations_per_step": ev, "interceptor_evaluations_per_s": ev / s,
            "fp64_triples_per_step": fp64, "fp64_recheck_fraction": fp64 / max(1, ev),
            "distance_computations_per_step": dist,
            "distance_computations_over_all_pairs": dist["total"] / max(1.0, n * (n - 1) / 2)}


def L_has_tier3(stats, i):
    """Whether pivot layer i built its node x ancestor key table (a lower layer with pairs
    left for the exhaustive or range-list tiers)."""
    G = stats["layers"][i]["grng"]
    return i > 0 and (G["range_pairs"] > 0 or G["tier3_pairs"] > 0)


def tc_key_error(g, X, n=256, seed=3003):
    """Largest error of the tensor-core tile keys on a seeded 256-point sample of the
    workload against the FP64 keys, absolute and as a fraction of the stated bound."""
    import numpy as np
    rng = np.random.default_rng(seed)
    S = X[rng.choice(X.shape[0], size=min(n, X.shape[0]), replace=False)]
    try:
        got = g.tc_keys(S).astype(np.float64)
    except g.GrngError as ex:  # a diagnostic: report, never end the run
        return {"error": str(ex)}
    S64 = S.astype(np.float64)
    nrm = (S64 ** 2).sum(1)
    want = ((S64[:, None, :] - S64[None, :, :]) ** 2).sum(-1)
    Dp = ((S.shape[1] + 15) // 16) * 16
    bound = (2.0 ** -12 + (3 * Dp + 16) * 2.0 ** -24) * (nrm[:, None] + nrm[None, :])
    err = np.abs(got - want)
    return {"sample_points": int(S.shape[0]), "max_abs_err": float(err.max()),
            "max_err_over_bound": float((err / np.maximum(bound, 1e-300)).max()),
            "max_rel_err": float((err / np.maximum(want, 1e-30))[~np.eye(S.shape[0], dtype=bool)].max())}


def check_rows(X, E, count, seed=3004, metric=0):
    """The RNG neighbourhoods of `count` seeded points of the GPU edge list E against the
    FP64 oracle's exact rows (each row: every y tested against every z closer to x, Eq. 1),
    computed on the host's cores after the timed region."""
    import numpy as np
    import oracle
    n = X.shape[0]
    xs = np.sort(np.random.default_rng(seed).choice(n, size=min(count, n), replace=False))
    t0 = time.perf_counter()
    want = oracle.rng_rows(X, xs, metric)
    dt = time.perf_counter() - t0
    both = np.concatenate([E, E[:, ::-1]])
    order = np.argsort(both[:, 0], kind="stable")
    src, dst = both[order, 0], both[order, 1]
    lo = np.searchsorted(src, xs, "left")
    hi = np.searchsorted(src, xs, "right")
    bad = 0
    for t in range(len(xs)):
        if not np.array_equal(np.sort(dst[lo[t]:hi[t]]), want[t]):
            bad += 1
    return {"rows_checked": int(len(xs)), "row_mismatches": int(bad), "oracle_seconds": dt,
            "neighbours_checked": int(sum(len(r) for r in want))}


def workload_name(kind, n, D, sizes, metric="l2"):
    shape = {"lin96": "intrinsic dim 8", "lin128": "intrinsic dim 12", "mix16": "64-Gaussian mixture",
             "uniform8": "uniform in the unit cube"}.get(kind, kind)
    return (f"{kind}: {n:,} x {D} FP32, {shape}, {metric.upper()}, nested random pivot layers "
            f"{'/'.join(str(s) for s in sizes)}")


def run_reference(a, rank, world):
    if rank != 0:
        return 0
    from paper_2208_10022_gb300 import workloads as wl
    N0, D, sizes, _, _ = wl.SPECS[a.kind]
    n = a.n or N0
    last = None
    for _ in range(a.warmup):
        last = cpu_baseline(a.kind, a.cpu_sample)
    times, edges = [], 0
    for _ in range(a.steps):
        last = cpu_baseline(a.kind, a.cpu_sample)
        times.append(last["seconds"])
        edges += last["edges"]
    tot = sum(times)
    v = edges / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000 * tot / max(a.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a.kind, n, D, wl.scaled_layer_sizes(a.kind, n)),
                       "n": n, "dim": D, "metric": "L2",
                       "oracle_sample_points": a.cpu_sample,
                       "note": "each step times the FP64 oracle (brute force over all triples) on a seeded "
                               "sample of this workload's generator"},
            "cpu_baseline": {k: last[k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(a, rank, world, local):
    import numpy as np
    import torch

    import paper_2208_10022_gb300 as g
    from paper_2208_10022_gb300 import build as gb
    from paper_2208_10022_gb300 import workloads as wl

    gb.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    N0, D, sizes0, _, _ = wl.SPECS[a.kind]
    metric = wl.L1 if a.metric == "l1" else wl.L2
    w = wl.make(a.kind, n=a.n, metric=metric)
    n, L = w.n, len(w.layers)
    sizes = [len(l) for l in w.layers]
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(w.X).cuda()
    piv_d = [torch.from_numpy(l).cuda() for l in w.layers]

    prec = g.BF16 if a.precision == "bf16" else g.FP32
    learned = None
    if a.precision == "bf16" and not a.no_learned:
        learned = train_shortlist(g, wl, a.kind)
    mlp = {"mlp_params": learned["params"], "k_shortlist": learned["k"]} if learned else {}

    def step_device(plain=False):
        ix = g.Index(Xd, n_layers=L, stream=stream, precision=g.FP32 if plain else prec, metric=metric,
                     **({} if plain else mlp))
        for li in range(L - 1, -1, -1):
            ix.build_layer(li, piv_d[li], outputs=False)
        for li in range(L):
            ix.link_pivots(li, want_adjacency=False)
        ix.rng_build_exact()
        ne = ix.n_edges()
        out = torch.empty((max(ne, 1), 2), dtype=torch.int32, device="cuda")
        ix.rng_edges(out=out)
        st = ix.stats()
        ix.close()
        return ne, st, out[:ne]

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    wst = None
    for _ in range(a.warmup):
        _, wst, _ = step_device()
    barrier()
    if wst is not None:
        launches0 = wst["kernel_launches"]           # counter after the last warm-up step
    else:
        probe = g.Index(np.zeros((1, 1), np.float32))  # its creation launches one kernel
        launches0 = probe.stats()["kernel_launches"]
        probe.close()
    # inputs smaller than twice the L2 (129 MB) are flushed from it before every timed step:
    # a 512 MB write outside the step's events; larger inputs stream through it anyway
    flush = None
    if w.X.nbytes < 2 * L2_BYTES:
        flush = torch.empty(4 * L2_BYTES, dtype=torch.uint8, device="cuda")

    def timed_steps(fn, k):
        """k calls of fn, each bracketed by CUDA events on the launching stream (an L2 flush
        before each, outside its events, when the inputs would fit in L2); total ms, results."""
        tot, res = 0.0, []
        for _ in range(k):
            if flush is not None:
                flush.zero_()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            res.append(fn())
            t1.record(stream)
            t1.synchronize()
            tot += t0.elapsed_time(t1)
        return tot, res

    clk = Clocks(local)
    tms, outs = timed_steps(step_device, a.steps)
    torch.cuda.synchronize()
    clocks = clk.stop()
    edges = sum(o[0] for o in outs)
    _, stats, e_last = outs[-1]
    del outs
    launches1 = stats["kernel_launches"]  # counter after the last timed step
    barrier()
    ms = max_over_ranks(tms, pg, "cuda")
    value = aggregate_rate(edges, world, ms)

    # end to end through the C ABI with host buffers: H2D of points and pivots, D2H of edges
    e2e = None
    if not a.no_e2e:
        Xh = torch.from_numpy(w.X).pin_memory()
        pivh = [torch.from_numpy(l).pin_memory() for l in w.layers]
        eh = torch.empty((max(edges // max(a.steps, 1), 1) + 16, 2), dtype=torch.int32).pin_memory()
        barrier()
        e2e_steps = max(1, min(a.steps, a.e2e_steps))

        def step_host():
            nonlocal eh
            ix = g.Index(Xh, n_layers=L, stream=stream, precision=prec, metric=metric, **mlp)
            for li in range(L - 1, -1, -1):
                ix.build_layer(li, pivh[li], outputs=False)
            for li in range(L):
                ix.link_pivots(li, want_adjacency=False)
            ix.rng_build_exact()
            ne = ix.n_edges()
            if ne > eh.shape[0]:
                eh = torch.empty((ne, 2), dtype=torch.int32).pin_memory()
            ix.rng_edges(out=eh)
            ix.close()
            return ne

        etot, ens = timed_steps(step_host, e2e_steps)
        barrier()
        e_edges = sum(ens)
        ems = max_over_ranks(etot, pg, "cuda")
        e2e = {"value": aggregate_rate(e_edges, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(w.X.nbytes + sum(l.nbytes for l in w.layers)),
               "d2h_bytes_per_step": int(8 * (e_edges // e2e_steps)), "steps": e2e_steps,
               "ms_per_step": ems / e2e_steps}

    # rooflines of the main kernels, timed with CUDA events inside the library on the
    # launching stream; the line's "roofline" is the one with the largest time
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = kernel_rooflines(stats, n, D, a.precision, peaks, sms)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32" if a.precision == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": workload_name(a.kind, n, D, sizes, a.metric), "n": n, "dim": D, "layers": sizes,
                       "metric": a.metric.upper(), "precision": ("split-bf16 tcgen05 exemplar tiles" if a.precision == "bf16" else "fp32 tiles") + "; fp32 exact tiers; fp64 near-tie recheck",
                       "learned": ({k: learned[k] for k in ("k", "train_points", "samples", "positives", "train_s",
                                                            "final_loss")} if learned else None),
                       "l2_flush": ("inputs larger than L2 (points alone are %d MB)" % (w.X.nbytes >> 20)
                                    if flush is None else
                                    "L2 flushed before every timed step (a %d MB write outside the step's events; "
                                    "points are %d MB)" % (flush.numel() >> 20, w.X.nbytes >> 20)),
                       "parallelism": f"replicas x{world}"},
            "edges_per_step": edges // max(a.steps, 1), "roofline": roof, "clocks": clocks,
            "gpu_launches": launches1 - launches0, "e2e": e2e,
            "detail": {"rng": stats["rng"], "layers": stats["layers"],
                       "rng_ms": stats["rng_ms"], "rng_tile_ms": stats["rng_tile_ms"], "sort_ms": stats["sort_ms"]}}
    line["measures"] = step_measures(stats, ms / a.steps)
    if prec == g.BF16 and not a.no_compare:
        # the plain build: FP32 CUDA-core tiles everywhere, no learned shortlist, same workload;
        # one untimed warm-up step, then the timed steps; its edge list is compared with the
        # BF16 + learned build's element by element on the device
        step_device(plain=True)
        barrier()
        k32 = max(1, a.plain_steps)
        t32, o32 = timed_steps(lambda: step_device(plain=True), k32)
        ne32, st32, e32 = o32[-1]
        del o32
        ms32 = t32 / k32
        same = bool(ne32 == e_last.shape[0] and torch.equal(e32, e_last))
        line["compare"] = {"plain_fp32_value": ne32 / (ms32 / 1000.0), "plain_fp32_ms_per_step": ms32,
                           "plain_fp32_steps": k32, "plain_fp32_warmup": 1, "plain_fp32_edges": ne32,
                           "edge_set_equal": same, "speedup_vs_plain_fp32": (ms32 / (ms / a.steps)),
                           "plain_fp32_tile_ms": st32["rng_tile_ms"]}
        del e32
    if prec == g.BF16 and metric == wl.L2:
        line["tc_key_error"] = tc_key_error(g, w.X)
    if rank == 0 and not a.no_search_leg:
        try:
            line["search"] = search_leg(g, wl, a, w, Xd, piv_d, prec, metric, mlp, stream)
        except Exception as ex:  # a failed extra leg must not hide the build's line
            line["search"] = {"error": f"{type(ex).__name__}: {ex}"}
    if rank == 0 and a.check_rows > 0:
        line["rng_row_check"] = check_rows(w.X, e_last.cpu().numpy(), a.check_rows, metric=metric)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline(a.kind, a.cpu_sample)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        one = cpu_baseline(a.kind, max(1000, a.cpu_sample // 3), threads=1)
        line["cpu_baseline"]["one_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
        line["cpu_baseline"]["cpu_model"] = cpu_model()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def search_leg(g, wl, a, w, Xd, piv_d, prec, metric, mlp, stream, batches=5, m=1000, check=16):
    """RNG search on an index of the build's workload (built untimed): `batches` batches of m
    further points of the same generator, each timed with CUDA events; `check` queries of the
    first batch compared with the FP64 oracle."""
    import numpy as np
    import torch
    L = len(piv_d)
    ix = g.Index(Xd, n_layers=L, stream=stream, precision=prec, metric=metric, **mlp)
    for li in range(L - 1, -1, -1):
        ix.build_layer(li, piv_d[li], outputs=False)
    for li in range(L):
        ix.link_pivots(li, want_adjacency=False)
    ds = wl.SPECS[a.kind][3]
    Q = wl.gen_points(a.kind, w.n + batches * m, ds)[w.n:]
    Qd = torch.from_numpy(Q).cuda()
    ix.rng_search_batch(Qd[:64])  # the cached index rows and block keys
    lat, first = [], None
    for b in range(batches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.rng_search_batch(Qd[b * m:(b + 1) * m])
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
        if b == 0:
            first = ix.rng_search_result()
    st = ix.stats()["search"]
    ix.close()
    out = {"metric": "RNG search queries/s", "value": batches * m / (sum(lat) / 1000.0), "unit": "queries/s",
           "batches": batches, "queries_per_batch": m, "p50_ms": float(np.percentile(lat, 50)),
           "neighbours_per_query": st["neighbours"] / max(st["queries"], 1)}
    if check:  # the CPU baseline of the search: the FP64 oracle on the first queries, its answers compared
        import oracle
        off, nb = first
        t0 = time.perf_counter()
        want = oracle.rng_search(w.X, Q[:check], metric)
        cs = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": check / cs, "unit": "queries/s", "cores": oracle.max_threads(),
                               "kind": "oracle", "sample": f"{check} queries against all {w.n:,} index points"}
        out["oracle_check"] = {"queries": check, "mismatches": int(sum(
            0 if np.array_equal(nb[off[j]:off[j + 1]], want[j]) else 1 for j in range(check)))}
    return out


def run_insert(a, rank):
    """Batched insertion (rng_insert_batch): an index is built on n points of the workload,
    then the batches (sizes drawn log-uniformly in [1,000, 65,536], scaled by n / 2,000,000
    below 2M points) of further points of the same generator arrive in order; every batch is
    timed with CUDA events on the index's stream.  With --insert-verify the final edge list
    is compared element by element with a build from scratch on all points (same pivots)."""
    import numpy as np
    import torch

    import paper_2208_10022_gb300 as g
    from paper_2208_10022_gb300 import build as gb
    from paper_2208_10022_gb300 import workloads as wl
    gb.build()
    N0, D, _, ds, ps = wl.SPECS[a.kind]
    n = a.n or N0
    scale = min(1.0, n / 2_000_000)
    sizes = [max(1, int(b * scale)) for b in wl.insertion_batches(a.insert)]
    total = n + sum(sizes)
    X = wl.gen_points(a.kind, total, ds)
    layers = wl.nested_pivots(n, wl.scaled_layer_sizes(a.kind, n), ps)
    prec = g.BF16 if a.precision == "bf16" else g.FP32
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(X).cuda()
    t0 = time.perf_counter()
    ix, _ = g.build_all(Xd[:n], layers, precision=prec, stream=stream)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    edges0 = ix.n_edges()
    # an index smaller than twice the L2 is flushed from it before every batch (outside the
    # batch's events); a larger one does not fit in it anyway
    flush = torch.empty(4 * L2_BYTES, dtype=torch.uint8, device="cuda") if X.nbytes < 2 * L2_BYTES else None
    lat, at = [], n
    for b in sizes:
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.rng_insert_batch(Xd[at:at + b])
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
        at += b
    tot = sum(lat)
    ne = ix.n_edges()
    st = ix.stats()["insert"]
    verify = None
    if a.insert_verify:
        got = torch.empty((max(ne, 1), 2), dtype=torch.int32, device="cuda")
        ix.rng_edges(out=got)
        ix.close()
        ix2, _ = g.build_all(Xd, layers, precision=prec, stream=stream)
        ne2 = ix2.n_edges()
        want = torch.empty((max(ne2, 1), 2), dtype=torch.int32, device="cuda")
        ix2.rng_edges(out=want)
        verify = bool(ne2 == ne and torch.equal(got[:ne], want[:ne2]))
        ix2.close()
    small = [t for t, b in zip(lat, sizes) if b <= np.median(sizes)]
    large = [t for t, b in zip(lat, sizes) if b > np.median(sizes)]
    line = {"metric": "batched insertion points/s", "value": sum(sizes) / (tot / 1000.0), "unit": "points/s",
            "higher_is_better": True, "n_gpus": 1, "batches": len(sizes), "points": int(sum(sizes)),
            "base_points": int(n), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_small_half": float(np.percentile(small, 50)) if small else None,
            "p50_ms_large_half": float(np.percentile(large, 50)) if large else None,
            "edges_before": int(edges0), "edges_after": int(ne), "edge_set_equal_rebuild": verify,
            "base_build_s": build_s,
            "method": "incremental: batch points join their finest domains; pivot pairs whose radii grew are "
                      "re-tested; batch rows swept against all points for new edges; Stage VII removes old edges "
                      "a batch point enters",
            "work": st,
            "config": {"workload": f"{a.kind}: index of {n:,} x {D} FP32 + {len(sizes)} batches of the same "
                                   f"generator, L2, nested random pivot layers "
                                   f"{'/'.join(str(len(l)) for l in layers)}",
                       "batch_sizes": sizes, "precision": a.precision,
                       "l2_flush": ("L2 flushed before every batch (outside its events)" if flush is not None
                                    else "index larger than L2 (points alone are %d MB)" % (X.nbytes >> 20))}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_search(a, rank):
    """RNG search (rng_search_batch): an index is built on n points of the workload, then B
    batches of m queries of the same generator (points the index does not hold) are searched;
    each batch is timed with CUDA events on the index's stream, its queries resident on the
    device.  --search-check queries of the first batch are compared with the FP64 oracle
    (Eq. 1 over the index plus the query), whose time per query is the CPU baseline."""
    import numpy as np
    import torch

    import paper_2208_10022_gb300 as g
    from paper_2208_10022_gb300 import build as gb
    from paper_2208_10022_gb300 import workloads as wl
    gb.build()
    N0, D, _, ds, ps = wl.SPECS[a.kind]
    n = a.n or N0
    m, B = a.search_m, a.search
    X = wl.gen_points(a.kind, n + m * B, ds)
    layers = wl.nested_pivots(n, wl.scaled_layer_sizes(a.kind, n), ps)
    prec = g.BF16 if a.precision == "bf16" else g.FP32
    metric = g.L1 if a.metric == "l1" else g.L2
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(X).cuda()
    ix, _ = g.build_all(Xd[:n], layers, metric=metric, precision=prec, stream=stream)
    flush = torch.empty(4 * L2_BYTES, dtype=torch.uint8, device="cuda") if X.nbytes < 2 * L2_BYTES else None
    ix.rng_search_batch(Xd[n:n + min(m, 64)])  # warm-up: the cached index rows and block keys
    lat, counts, first = [], [], None
    for b in range(B):
        Q = Xd[n + b * m:n + (b + 1) * m]
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        counts.append(ix.rng_search_batch(Q))
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
        if b == 0:
            off, nb = ix.rng_search_result()
            first = (off.copy(), nb.copy())
    st = ix.stats()["search"]
    check = None
    cpu = None
    if a.search_check and rank == 0:
        import oracle
        k = min(a.search_check, m)
        t0 = time.perf_counter()
        want = oracle.rng_search(X[:n], X[n:n + k], metric)
        cpu_s = time.perf_counter() - t0
        off, nb = first
        bad = sum(0 if np.array_equal(nb[off[j]:off[j + 1]], want[j]) else 1 for j in range(k))
        check = {"queries": k, "mismatches": bad}
        cpu = {"value": k / cpu_s, "unit": "queries/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"{k} queries of the first batch against all {n:,} index points"}
    tot = sum(lat)
    line = {"metric": "RNG search queries/s", "value": m * B / (tot / 1000.0), "unit": "queries/s",
            "higher_is_better": True, "n_gpus": 1, "batches": B, "queries_per_batch": m,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "neighbours_per_query": float(np.sum(counts)) / (m * B),
            "candidate_pairs_per_query": st["candidate_pairs"] / max(st["queries"], 1),
            "tier1_survivors_per_query": st["tier1_survivors"] / max(st["queries"], 1),
            "outside_ball_fraction": st["outside_ball"] / max(st["queries"], 1),
            "oracle_check": check, "cpu_baseline": cpu, "work": st,
            "config": {"workload": f"{a.kind}: index of {n:,} x {D} FP32, L{1 if metric == g.L1 else 2}, nested "
                                   f"random pivot layers {'/'.join(str(len(l)) for l in layers)}; queries: further "
                                   f"points of the same generator",
                       "precision": a.precision,
                       "l2_flush": ("L2 flushed before every batch (outside its events)" if flush is not None
                                    else "index larger than L2 (points alone are %d MB)" % (X.nbytes >> 20))}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _canonical_keys_to(X64, i):
    """FP64 keys of every point to point i, the squared differences added in dimension order."""
    import numpy as np
    acc = np.zeros(X64.shape[0])
    for d in range(X64.shape[1]):
        t = X64[:, d] - X64[i, d]
        acc = acc + t * t
    return acc


def run_skeleton(a, rank):
    """Lune-based beta-skeleton (rng_build_skeleton): the pivot layers are built and linked,
    then the skeleton of all points is timed with CUDA events per step (no Theorem 1 below
    beta = 2: every pair is a candidate).  Sampled edges are checked to have no point inside
    their beta-lune, in canonical FP64 against every point; the FP64 oracle's brute force on a
    bounded sample is the CPU baseline."""
    import numpy as np
    import torch

    import paper_2208_10022_gb300 as g
    from paper_2208_10022_gb300 import build as gb
    from paper_2208_10022_gb300 import workloads as wl
    gb.build()
    beta = a.skeleton
    w = wl.make(a.kind, n=a.n)
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(w.X).cuda()
    ix, _ = g.build_all(Xd, w.layers, stream=stream)
    lat = []
    for it in range(a.warmup + a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.rng_build_skeleton(beta)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= a.warmup:
            lat.append(e0.elapsed_time(e1))
    E = ix.rng_edges()
    st = ix.stats()["rng"]
    X64 = w.X.astype(np.float64)
    lam, mu = beta / 2.0, 1.0 - beta / 2.0
    bad = 0
    sample = E[np.random.default_rng(7).choice(E.shape[0], size=min(100, E.shape[0]), replace=False)]
    for i, j in sample:
        ka, kb = _canonical_keys_to(X64, int(i)), _canonical_keys_to(X64, int(j))
        t = lam * ka[int(j)]
        inside = (mu * ka + lam * kb < t) & (lam * ka + mu * kb < t)
        inside[[int(i), int(j)]] = False
        bad += int(inside.any())
    cpu = None
    if rank == 0 and a.cpu_sample:
        import oracle
        k = min(a.cpu_sample, 2500, w.n)
        Xs = wl.subsample(w, k, 11).X
        t0 = time.perf_counter()
        Ec = oracle.beta_skeleton(Xs, beta)
        cs = time.perf_counter() - t0
        cpu = {"value": len(Ec) / cs, "unit": "edges/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"beta_skeleton brute force on a seeded {k}-point subsample ({len(Ec)} edges in {cs:.2f} s)"}
    ms = float(np.mean(lat))
    line = {"metric": f"beta-skeleton edges/s (beta={beta:g})", "value": E.shape[0] / (ms / 1000.0), "unit": "edges/s",
            "higher_is_better": True, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "edges": int(E.shape[0]), "sampled_edges_checked": int(sample.shape[0]), "sampled_edges_with_a_point_inside": bad,
            "cpu_baseline": cpu,
            "work": {k: st[k] for k in ("candidate_pairs", "tier1_survivors", "tier2a_links", "tier2a_blocked",
                                        "tier3_pairs", "fp64_triples", "edges")},
            "phase_ms": st["phase_ms"],
            "config": {"workload": f"{a.kind}: {w.n:,} x {w.dim} FP32, L2, nested random pivot layers "
                                   f"{'/'.join(str(len(l)) for l in w.layers)}", "beta": beta, "precision": "fp32"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    rank, world, local = dist_env()
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if a.insert:
        return run_insert(a, rank)
    if a.search:
        return run_search(a, rank)
    if a.skeleton:
        return run_skeleton(a, rank)
    return run_gpu(a, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
