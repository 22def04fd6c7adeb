"""HODLR2D matvec benchmark on GB300.

Workload (the headline configuration): N = 2^20 points i.i.d. uniform in
[-1,1]^2 (seed 0), multiquadric sqrt(r^2 + a^2) with a = 1/sqrt(N) = 2^-10,
leaf size 64 (kappa = 8 under the strict leaf rule), ACA eps = 1e-8, one
right-hand side x ~ N(0,1) (seed 1), FP64.  A step is one HODLR2D product
y = K_hat x (Alg. 2) on the built matrix; the build (Alg. 1) is timed once
and reported as t_build_ms.  The factors (GBs) exceed L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  The headline is the binary64 product (mode
f64); the float-float, binary32 and bfloat16 forms follow under "modes".
--impl reference times the CPU oracle's Alg. 2 product of the same workload
on one host core instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "N=2^20 HODLR2D matvec ms & %HBM roofline, FP64 vs mixed form at stated rel err"
N_FULL = 1 << 20
LEAF = 64
EPS = 1e-8
A_MQ = 1.0 / np.sqrt(N_FULL)
ROOT_BOX = (-1.0, -1.0, 2.0)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: 200, a timed region of about 2 s for the "
                        "binary64 product; 20 for the CPU reference arm)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--modes", default="f64,df32,f32,bf16",
                   help="product modes to time; the first is the headline")
    p.add_argument("--points", type=int, default=N_FULL, help="N (smaller for quick checks)")
    p.add_argument("--nrhs", type=int, default=1, help="right-hand sides per product")
    p.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    p.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    p.add_argument("--extras", default="all",
                   help="comma-separated secondary measurements to run (default: all)")
    p.add_argument("--batch-sets", type=int, default=256,
                   help="point sets of the batch measurement (smaller for profiling)")
    p.add_argument("--n-learned", type=int, default=1 << 22,
                   help="points of the learned-rank build (log r kernel)")
    args = p.parse_args()
    if args.steps is None:
        args.steps = 200 if args.impl == "ours" else 20
    return args


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    """(HBM GB/s, its source, binary64 TFLOP/s, its source).  HBM: the
    measured copy bandwidth of the GB300s.  Binary64: 152 SMs x 2
    binary64 FMA per clock x 2 flops x the maximum SM clock (2070 MHz), the
    unit counts behind the nominal 1.25 TFLOP/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        hbm, src = float(d["hbm_gbs"]), "measured"
        mhz = float(d.get("sm_max_mhz", 2070.0))
    except (OSError, KeyError, ValueError):
        hbm, src, mhz = 6800.0, "fallback", 2070.0
    return hbm, src, 152 * 2 * 2 * mhz * 1e6 / 1e12, "derived: 152 SM x 2 FMA/clk x 2 x %.0f MHz" % mhz


# ncu DRAM traffic (read + write bytes) per algorithmic byte of a kernel,
# keyed by (phase, mode), measured at N = 2^17: k_proj2 (DF32) 522.9 MB for
# 514.6 MB of factor values.  Traffic grows with the units processed, so a
# launch's traffic is this ratio times its algorithmic bytes.  Remove an entry
# when its kernel changes.
NCU_TRAFFIC_RATIO = {("proj", "df32"): 522.9 / 514.6,
                     # k_near64 at N = 2^17: 3.276 MB of DRAM traffic for 5.243 MB of
                     # algorithmic bytes (points and x, partly served by L2)
                     ("near", "f64"): 3.276 / 5.243}


def host_cpu():
    """(logical cores, CPU model) of the host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count(), model


def oracle_worker(conn, n, rows):
    """Child process (spawned before any CUDA call): the CPU oracle builds the
    benchmark workload (Alg. 1), reports, then on request times its Alg. 2
    product (median of 3, one core) and evaluates the direct product on the
    sampled rows.  Uses only oracle/ and the seeded inputs."""
    import oracle
    from paper_2204_05536_gb300 import inputs
    try:
        oracle.build()
        pts = inputs.uniform(n, seed=0)
        x = inputs.rhs(n, seed=1)
        ko = oracle.kernel("mq", 1.0 / np.sqrt(n))
        t0 = time.perf_counter()
        o = oracle.Oracle(pts, ko, LEAF, EPS, root=ROOT_BOX)
        conn.send({"build_s": time.perf_counter() - t0, "kappa": o.kappa})
        if conn.recv() != "time":
            return
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            o.matvec(x)
            ts.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        yd = oracle.direct_rows(pts, ko, x, rows)
        conn.send({"t_matvec_s": statistics.median(ts), "all_s": ts,
                   "t_rows_s": time.perf_counter() - t0, "y_direct_rows": yd})
    except Exception as e:  # reported, never raised into the benchmark
        conn.send({"error": repr(e)})


class OracleLeg:
    """The cpu_baseline leg: the oracle's build runs on one host core while
    the GPU is measured; its products are timed afterwards."""

    def __init__(self, n, rows):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=oracle_worker, args=(child, n, rows), daemon=True)
        self.proc.start()

    def result(self, timeout=900.0):
        out = {}
        if self.conn.poll(timeout):
            out.update(self.conn.recv())
        if "error" not in out and "build_s" in out:
            self.conn.send("time")
            if self.conn.poll(timeout):
                out.update(self.conn.recv())
        self.proc.join(timeout=30)
        if self.proc.is_alive():
            self.proc.terminate()
        return out


def workload_config(n, kappa, mode, nrhs=1):
    """The bench line's config (the same for both arms)."""
    fb = {"f64": 8, "df32": 8, "f32": 4, "bf16": 2}[mode]
    lg = int(np.log2(n))
    nn = "2^%d" % lg if n == 1 << lg else str(n)
    w = ("N=%s uniform [-1,1]^2 seed 0, MQ sqrt(r^2+a^2) a=1/sqrt(N), leaf 64 (kappa %d), "
         "ACA eps 1e-8, %d RHS N(0,1) seed 1" % (nn, kappa, nrhs))
    return {"workload": w,
            "n": n, "leaf": LEAF, "eps": EPS, "kernel": "mq", "a": 1.0 / np.sqrt(n), "nrhs": nrhs,
            "mode": mode, "kappa": kappa, "parallelism": "replicas",
            "l2": "no flush: factors (%d bytes per value) exceed the 129 MB L2" % fb}


def timed(g, x, y, mode, steps, warmup, stream):
    """steps products after warmup ones; ms per product (CUDA events)."""
    import torch
    for _ in range(warmup):
        g.matvec(x, mode=mode, out=y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.matvec(x, mode=mode, out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def events(stream):
    import torch
    return (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))


def extra_gmres_nrhs(pkg, inputs, n, stream):
    """RBF interpolation system of Eq. ker with the headline points and MQ
    kernel, beta = N on the diagonal (Sec. 5.1): GMRES(50) to a 1e-8 relative
    residual with the F64 product, and FP64 iterative refinement around
    binary32 / bfloat16 / float-float inner solves; then one product of 32
    right-hand sides per mode."""
    import torch
    g = pkg.HODLR2D(inputs.uniform(n, seed=0), pkg.kernel("mq", 1.0 / np.sqrt(n), diag=float(n)),
                    LEAF, EPS, root=ROOT_BOX)
    g.set_stream(stream)
    lam = torch.from_numpy(inputs.rhs(n, seed=2)).cuda()
    f = g.matvec(lam, mode="f64")
    gm = {}
    for mode in ("f64", "f32", "bf16", "df32"):
        if mode != "f64":
            g.prepare(mode)
        # one untimed solve per mode first: the Krylov workspace, the pinned
        # residual buffer and the first launch of every kernel on the path
        g.gmres(f, tol=1e-8, restart=50, maxit=2000, inner_mode=mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xs, it, rr, code = g.gmres(f, tol=1e-8, restart=50, maxit=2000, inner_mode=mode)
        torch.cuda.synchronize()
        r = f - g.matvec(xs, mode="f64")
        gm[mode] = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "products": it,
                    "relres_reported": rr, "relres_f64": float(torch.linalg.norm(r)
                                                               / torch.linalg.norm(f)),
                    "converged": code == 0,
                    "rel_err_lambda": float(torch.linalg.norm(xs - lam) / torch.linalg.norm(lam))}
    nr = 32
    Xc = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, nr, seed=3).T)).cuda()  # nrhs x n
    Yc = torch.empty_like(Xc)
    Y64 = torch.empty_like(Xc)
    g.matvec(Xc.t(), mode="f64", out=Y64)
    mr = {}
    for mode in ("f64", "df32", "f32", "bf16"):
        for _ in range(2):
            g.matvec(Xc.t(), mode=mode, out=Yc)
        torch.cuda.synchronize()
        e0, e1 = events(stream)
        e0.record(stream)
        for _ in range(3):
            g.matvec(Xc.t(), mode=mode, out=Yc)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        mr[mode] = {"ms": round(ms, 3), "products_per_s": round(nr / (ms * 1e-3), 1),
                    "rel2_vs_f64": float(torch.linalg.norm(Yc - Y64) / torch.linalg.norm(Y64))}
    g.close()
    return {"gmres_mq_beta_n": gm, "nrhs32": mr}


def extra_batch(pkg, inputs, stream, count=256):
    """Independent point sets (sizes log-uniform in [2048, 65536], rectangles of
    aspect ratio up to 4), IMQ a = 1/sqrt(n_i), binary32 factors, 1-8
    right-hand sides each, all products replayed as one CUDA graph, then as
    one persistent cooperative kernel (shapes autotuned).  The leaf
    size is tuned per size class (four log-spaced classes) on one member."""
    import torch
    sets = inputs.point_sets(count, seed=0)
    sizes = np.array([len(p) for p in sets])
    edges = np.exp(np.linspace(np.log(2048), np.log(65536), 5))
    cls = np.clip(np.searchsorted(edges, sizes, side="right") - 1, 0, 3)
    t0 = time.perf_counter()
    leaf_of = {}
    for c in range(4):
        members = np.nonzero(cls == c)[0]
        if len(members) == 0:
            continue
        i = int(members[len(members) // 2])
        best, _ = pkg.autotune_leaf(sets[i], pkg.kernel("imq", 1.0 / np.sqrt(sizes[i])), EPS,
                                    candidates=(32, 64, 128), nrhs=4, mode="f32", reps=3)
        leaf_of[c] = best
    t_tune = time.perf_counter() - t0
    rng = np.random.default_rng(5)
    mats, xs, ys = [], [], []
    t0 = time.perf_counter()
    for p, c in zip(sets, cls):
        m = pkg.HODLR2D(p, pkg.kernel("imq", 1.0 / np.sqrt(len(p))), leaf_of[int(c)], EPS)
        m.prepare("f32")
        mats.append(m)
        r = int(rng.integers(1, 9))
        xs.append(torch.from_numpy(rng.standard_normal((r, len(p)))).cuda())
        ys.append(torch.empty_like(xs[-1]))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    nprod = int(sum(x.shape[0] for x in xs))
    far_values = int(sum(m.stats()["far_values"] for m in mats))
    hbm_gbs = peaks()[0]
    b = pkg.Batch(mats, stream=stream, form="graph")
    b.matvec(xs, ys, mode="f32")  # records the graph
    torch.cuda.synchronize()
    e0, e1 = events(stream)
    e0.record(stream)
    for _ in range(5):
        b.matvec(xs, ys, mode="f32")
    e1.record(stream)
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / 5
    # one persistent cooperative kernel over all sets, shapes autotuned
    yp = [torch.empty_like(y) for y in ys]
    b.set_form("persistent")
    t0 = time.perf_counter()
    shapes, _ = b.autotune(xs, yp, mode="f32", reps=3)
    t_ptune = time.perf_counter() - t0
    table = {("graph" if a < 0 else "%d/%d/%d/%d" % (a, c, m, pl)): round(t, 3)
             for a, c, m, pl, t in b.tune_table()}
    b.set_form("auto")
    b.matvec(xs, yp, mode="f32")
    auto_form = b.last_form
    b.set_form("persistent")
    b.matvec(xs, yp, mode="f32")
    b.check()
    e0.record(stream)
    for _ in range(5):
        b.matvec(xs, yp, mode="f32")
    e1.record(stream)
    torch.cuda.synchronize()
    b.check()
    t_pers = e0.elapsed_time(e1) / 5
    phases = [round(v, 3) for v in b.phase_ms()]
    recorded = b.persistent_recorded
    pers_vs_graph = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c))
                        for a, c in zip(yp, ys))
    for m in mats:
        m.set_stream(stream)
    ys2 = [torch.empty_like(y) for y in ys]
    e0.record(stream)
    for _ in range(5):
        for m, x, y in zip(mats, xs, ys2):
            m.matvec(x.t(), mode="f32", out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 5
    same = all(bool(torch.equal(y, y2)) for y, y2 in zip(ys, ys2))
    y64 = [m.matvec(x.t(), mode="f64") for m, x in zip(mats[:8], xs[:8])]
    err = max(float(torch.linalg.norm(y.t() - z) / torch.linalg.norm(z))
              for y, z in zip(ys[:8], y64))
    b.close()
    for m in mats:
        m.close()
    return {"sets": count, "points": int(sizes.sum()), "products": nprod,
            "leaf_per_class": {str(int(round(edges[c]))): v for c, v in leaf_of.items()},
            "graph_ms": round(t_graph, 3), "sequential_launches_ms": round(t_seq, 3),
            "products_per_s_graph": round(nprod / (t_graph * 1e-3), 1),
            "factor_bytes_f32": 4 * far_values,
            "factor_read_once_ms_at_hbm_peak": round(4 * far_values / (hbm_gbs * 1e6), 3),
            "persistent_ms": round(t_pers, 3),
            "persistent_launch_in_cuda_graph": recorded,
            "products_per_s_persistent": round(nprod / (t_pers * 1e-3), 1),
            "persistent_shapes": {"pair_rows": shapes[0], "warp_rows": shapes[1]},
            "persistent_tune_s": round(t_ptune, 2),
            "persistent_tune_table_ms": table,
            "auto_form_after_tune": auto_form,
            "persistent_phase_ms": dict(zip(["gather", "pairs_proj_near", "chunk_sums",
                                             "expansions", "combine"], phases)),
            "rel2_persistent_vs_graph_max": pers_vs_graph,
            "graph_equals_sequential": same, "rel2_f32_vs_f64_first8": err,
            "tune_s": round(t_tune, 2), "build_s": round(t_build, 2)}


def extra_learned(pkg, inputs, stream, n_big):
    """Rank predictor trained on the GPU on the ACA ranks of log r builds at
    N = 2^16, 2^18, 2^20 (eps 1e-8), then used in an N = n_big build: build
    time, ACA workspace and fallbacks against the plain adaptive build; then
    a 16-RHS binary32 product of the result."""
    import torch
    feats, targets = [], []
    for nn in (1 << 16, 1 << 18, 1 << 20):
        gg = pkg.HODLR2D(inputs.uniform(nn, seed=nn), pkg.kernel("log"), LEAF, EPS, root=ROOT_BOX)
        f_, r_ = gg.pair_features()
        feats.append(f_)
        targets.append(r_)
        gg.close()
    F = np.concatenate(feats)
    T = np.concatenate(targets)
    perm = np.random.default_rng(0).permutation(len(T))
    model = pkg.RankModel(64, inputs.mlp_init(64, seed=1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = model.train(F[perm], T[perm], batch=1024, epochs=30, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pts = inputs.uniform(n_big, seed=0)
    res = {"train": {"pairs": int(len(T)), "final_mse_log2rank": loss,
                     "train_s": round(t_train, 2)}}
    Xc = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n_big, 16, seed=3).T)).cuda()
    ys = {}
    for name, mdl in (("plain", None), ("learned", model)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gg = pkg.HODLR2D(pts, pkg.kernel("log"), LEAF, EPS, root=ROOT_BOX, rank_model=mdl)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        st = gg.stats()
        gg.set_stream(stream)
        gg.prepare("f32")
        Y = torch.empty_like(Xc)
        for _ in range(2):
            gg.matvec(Xc.t(), mode="f32", out=Y)
        torch.cuda.synchronize()
        e0, e1 = events(stream)
        e0.record(stream)
        for _ in range(3):
            gg.matvec(Xc.t(), mode="f32", out=Y)
        e1.record(stream)
        torch.cuda.synchronize()
        ys[name] = Y
        res[name] = {"build_ms": round(t_b * 1e3, 1), "aca_ms": round(st["build_ms"][2], 1),
                     "aca_workspace_gb": round(st["aca_workspace_values"] * 8 / 1e9, 3),
                     "fallbacks": st["aca_fallbacks"], "npairs": st["npairs"],
                     "far_values": st["far_values"], "max_rank": st["max_rank"],
                     "f32_nrhs16_ms": round(e0.elapsed_time(e1) / 3, 3)}
        gg.close()
    res["products_identical"] = bool(torch.equal(ys["plain"], ys["learned"]))
    res["n"] = n_big
    model.close()
    return res


def direct_rows_gpu(pts, kind, a, diag, x, rows, chunk=1024):
    """Exact product rows (binary64, plain torch on the GPU) for the error
    checks of the paper replays: phi of Sec. 5.1 / Eq. ker, diagonal diag."""
    import torch
    P = torch.from_numpy(pts).cuda()
    X = torch.from_numpy(x).cuda()
    out = torch.empty(len(rows), dtype=torch.float64, device="cuda")
    rows_t = torch.from_numpy(np.asarray(rows)).cuda()
    for c0 in range(0, len(rows), chunk):
        ri = rows_t[c0:c0 + chunk]
        dx = P[ri, 0:1] - P[:, 0]
        dy = P[ri, 1:2] - P[:, 1]
        r = torch.sqrt(dx * dx + dy * dy)
        del dx, dy
        if kind == "inv_r":
            K = 1.0 / r
        elif kind == "phi1":
            K = torch.where(r >= a, torch.log(r) / np.log(a), (r * torch.log(r) - 1.0) /
                            (a * np.log(a) - 1.0))
        else:  # phi2
            K = torch.where(r >= a, a / r, r / a)
        K[torch.arange(len(ri), device="cuda"), ri] = diag
        out[c0:c0 + chunk] = K @ X
    return out.cpu().numpy()


def extra_panel_system(pkg, inputs, stream):
    """log r on the 512 x 512 jittered grid (N = 2^18, spacing h = 2/512),
    leaf 64, eps 1e-10, GMRES(50) to 1e-8 with b ~ N(0,1): the literal
    panel diagonal (h^2/2pi)(log h - 1.5), a first-kind system on which
    GMRES stalls (capped at 300 products), and the second-kind variant (the
    matrix scaled by 2pi/h^2: diagonal 2pi/h^2 + log h - 1.5)."""
    import torch
    pts, h = inputs.jittered_grid(512, seed=0)
    n = len(pts)
    b = torch.from_numpy(inputs.rhs(n, seed=1)).cuda()
    out = {}
    for name, diag, maxit in (
            ("literal", (h * h / (2 * np.pi)) * (np.log(h) - 1.5), 300),
            ("second_kind", 2 * np.pi / (h * h) + np.log(h) - 1.5, 2000)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = pkg.HODLR2D(pts, pkg.kernel("log", 0.0, diag), 64, 1e-10, root=ROOT_BOX)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        g.set_stream(stream)
        g.prepare("df32")
        g.prepare("f32")
        st = g.stats()
        res = {"kappa": st["kappa"], "r_m": st["max_rank"], "build_s": round(t_b, 3)}
        y = torch.empty_like(b)
        for mode in ("f64", "df32", "f32"):
            res["matvec_ms_" + mode] = round(timed(g, b, y, mode, 5, 2, stream), 3)
        for mode in ("f64", "df32", "f32"):
            g.gmres(b, tol=1e-8, restart=50, maxit=min(maxit, 60), inner_mode=mode)  # untimed
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xs, it, rr, code = g.gmres(b, tol=1e-8, restart=50, maxit=maxit, inner_mode=mode)
            torch.cuda.synchronize()
            res["gmres_" + mode] = {"ms": round((time.perf_counter() - t0) * 1e3, 1),
                                    "products": it, "relres": rr, "converged": code == 0}
        out[name] = res
        g.close()
    return out


def extra_paper_replay(pkg, inputs, stream):
    """The paper's own workloads on the GPU, next to its printed tables
    (context): Sec. 5.1 (1/r, Chebyshev grid, N_max 500, eps 1e-12; r_m,
    stored GB, build time, product time, max componentwise error over 2048
    sampled rows) and Sec. 5.2 (phi_1 and phi_2, a = 0.001, beta = N, GMRES
    to 1e-10; build, solve time, solution error)."""
    import torch
    out = {"sec51_inv_r": {}, "sec52_rbf": {}}
    rng = np.random.default_rng(11)
    for m in (100, 300, 500):
        n = m * m
        pts = inputs.chebyshev_grid(m)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = pkg.HODLR2D(pts, pkg.kernel("inv_r"), 500, 1e-12, root=ROOT_BOX)
        torch.cuda.synchronize()
        t_i = time.perf_counter() - t0
        g.set_stream(stream)
        g.prepare("df32")
        st = g.stats()
        psi = rng.uniform(0.0, 1.0, n)
        rows = np.sort(rng.choice(n, min(n, 2048), replace=False))
        b = direct_rows_gpu(pts, "inv_r", 0.0, 0.0, psi, rows)
        xd = torch.from_numpy(psi).cuda()
        res = {"kappa": st["kappa"], "r_m": st["max_rank"],
               "stored_gb": round((st["far_values"] + st["near_entries"]) * 8 / 1e9, 3),
               "factor_gb": round(st["far_values"] * 8 / 1e9, 3),
               "cr": round(st["compression_ratio"], 4), "t_i_s": round(t_i, 3)}
        for mode in ("f64", "df32"):
            y = torch.empty_like(xd)
            ms = timed(g, xd, y, mode, 5, 2, stream)
            yb = y.cpu().numpy()[rows]
            res[mode] = {"ms": round(ms, 3),
                         "eps_r": float(np.max(np.abs(yb - b) / np.abs(b)))}
        out["sec51_inv_r"][str(n)] = res
        g.close()
    m = 500
    n = m * m
    pts = inputs.chebyshev_grid(m)
    lam = rng.standard_normal(n)
    for kind in ("phi1", "phi2"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = pkg.HODLR2D(pts, pkg.kernel(kind, 0.001, diag=float(n)), 500, 1e-12, root=ROOT_BOX)
        torch.cuda.synchronize()
        t_i = time.perf_counter() - t0
        g.set_stream(stream)
        g.prepare("df32")
        st = g.stats()
        f = torch.from_numpy(direct_rows_gpu(pts, kind, 0.001, float(n), lam,
                                             np.arange(n))).cuda()
        res = {"kappa": st["kappa"], "r_m": st["max_rank"], "cr": round(st["compression_ratio"], 4),
               "t_i_s": round(t_i, 3)}
        for mode in ("f64", "df32"):
            g.gmres(f, tol=1e-10, restart=50, maxit=2000, inner_mode=mode)  # untimed
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xs, it, rr, code = g.gmres(f, tol=1e-10, restart=50, maxit=2000, inner_mode=mode)
            torch.cuda.synchronize()
            res[mode] = {"t_g_s": round(time.perf_counter() - t0, 4), "products": it,
                         "relres": rr, "converged": code == 0,
                         "rel_err_solution": float(np.linalg.norm(xs.cpu().numpy() - lam)
                                                   / np.linalg.norm(lam))}
        out["sec52_rbf"][kind + "_n" + str(n)] = res
        g.close()
    return out


def extras(pkg, inputs, n, n_learned, names="all", batch_sets=256):
    """Secondary measurements on one GPU (each section timed on its own);
    names: "all" or a comma-separated subset of the section names."""
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    pick = None if names == "all" else set(names.split(","))
    for name, fn in (("rbf_system", lambda: extra_gmres_nrhs(pkg, inputs, n, stream)),
                     ("paper_replay", lambda: extra_paper_replay(pkg, inputs, stream)),
                     ("panel_system_log", lambda: extra_panel_system(pkg, inputs, stream)),
                     ("batch_point_sets", lambda: extra_batch(pkg, inputs, stream, batch_sets)),
                     ("learned_rank_log", lambda: extra_learned(pkg, inputs, stream, n_learned))):
        if pick is not None and name not in pick:
            continue
        t0 = time.perf_counter()
        out[name] = fn()
        out[name]["section_s"] = round(time.perf_counter() - t0, 1)
    return out


def phase_roofline(prof, steps, mode, hbm, fp64):
    """Per phase of one product (serialised pass): ms, launches, algorithmic
    bytes and flops, and the fraction of the roofline that bounds it.  The
    binary64 kernels are bound by the binary64 pipe (GB300 issues 2 binary64
    FMAs per clock per SM against 128 binary32), so their roofline is the
    binary64 peak; the other modes' far field streams its factors, so theirs
    is the HBM peak."""
    out = {}
    for k, v in prof.items():
        if not v["launches"]:
            continue
        ms = v["ms"] / steps
        gbs = v["bytes"] / steps / (ms * 1e-3) / 1e9
        tfs = v["flops"] / steps / (ms * 1e-3) / 1e12
        alu = mode == "f64" and k not in ("gather", "combine")
        out[k] = {"ms": round(ms, 4), "launches": v["launches"] // steps,
                  "bytes": v["bytes"] // steps, "flops": v["flops"] // steps,
                  "GB_s": round(gbs, 1), "TFLOP_s": round(tfs, 4),
                  "bound": "alu" if alu else "hbm",
                  "frac": round(tfs / fp64 if alu else gbs / hbm, 4)}
    return out


def run_ours(args, ws, rank, local):
    n = args.points
    R = args.nrhs
    rows = np.random.default_rng(7).choice(n, 256, replace=False)
    # the oracle leg starts first, in a spawned process, before any CUDA call
    leg = OracleLeg(n, rows) if (rank == 0 and not args.no_cpu) else None

    import torch
    import paper_2204_05536_gb300 as pkg
    from paper_2204_05536_gb300 import inputs

    torch.cuda.set_device(local)
    pts = inputs.uniform(n, seed=0)
    a = 1.0 / np.sqrt(n)
    x_h = inputs.rhs(n, R, seed=1)  # (n,) or (n, R)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = pkg.HODLR2D(pts, pkg.kernel("mq", a), LEAF, EPS, root=ROOT_BOX)
    torch.cuda.synchronize()
    t_build = (time.perf_counter() - t0) * 1e3
    st = g.stats()
    modes = args.modes.split(",")
    stream = torch.cuda.current_stream()
    g.set_stream(stream)
    hbm, hbm_src, fp64, fp64_src = peaks()
    # device buffers: R x n (column-major n x R); the products take x.t()
    xc = torch.from_numpy(np.ascontiguousarray(x_h.T if R > 1 else x_h)).cuda()
    y = torch.empty_like(xc)
    x = xc.t() if R > 1 else xc
    per_mode = {}
    for mode in modes:
        if mode != "f64":
            g.prepare(mode)
        barrier(ws)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        ms = timed(g, x, y, mode, args.steps, args.warmup, stream)
        # second pass with per-phase events (kernels serialized); the clock
        # sampler keeps running through it, so that short timed regions still
        # get samples under the same load
        g.profile(True)
        for _ in range(args.steps):
            g.matvec(x, mode=mode, out=y)
        prof = g.get_profile()
        g.profile(False)
        torch.cuda.synchronize()
        clk = clocks.stop()
        barrier(ws)
        per_mode[mode] = {"ms": max_over_ranks(ms, ws), "prof": prof, "clocks": clk,
                          "y": y.clone()}
    mode = modes[0]
    ms_step = per_mode[mode]["ms"]
    prof = per_mode[mode]["prof"]
    clk = per_mode[mode]["clocks"]

    # end to end through the public API with pinned host buffers
    xp = torch.from_numpy(np.ascontiguousarray(x_h.T if R > 1 else x_h)).pin_memory()
    yp = torch.empty_like(xp).pin_memory()
    xnp, ynp = (xp.numpy().T if R > 1 else xp.numpy()), yp.numpy()
    g.set_stream(None)
    for _ in range(2):
        g.matvec(xnp, mode=mode, out=ynp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.matvec(xnp, mode=mode, out=ynp)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = max_over_ranks(e2e_ms, ws)
    g.set_stream(stream)

    # per-phase rooflines; the dominant kernel is the phase with the longest
    # time per launch
    phases = {m: phase_roofline(v["prof"], args.steps, m, hbm, fp64) for m, v in per_mode.items()}
    ph = phases[mode]
    dom = max(ph, key=lambda k: ph[k]["ms"] / ph[k]["launches"])
    d = ph[dom]
    per_launch_ms = d["ms"] / d["launches"]
    launches_per_step = sum(v["launches"] for v in ph.values())

    def product_fracs(m, ms):
        b = st["bytes_per_matvec"][m] + 16 * n * (R - 1)
        fl = sum(v["flops"] for v in phases[m].values())
        return {"hbm_frac": round(b / (ms * 1e-3) / 1e9 / hbm, 4), "bytes": b,
                "flops": fl, "fp64_frac": round(fl / (ms * 1e-3) / 1e12 / fp64, 4)
                if m == "f64" else None}

    if d["bound"] == "alu":
        roof = {"bound": "alu", "kernel": dom, "achieved": round(d["TFLOP_s"] * d["launches"], 4),
                "peak": round(fp64, 4), "unit": "TFLOP/s",
                "frac": round(d["TFLOP_s"] * d["launches"] / fp64, 4), "peak_source": fp64_src,
                "flops_per_launch": d["flops"] // d["launches"]}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(d["GB_s"] * d["launches"], 1),
                "peak": hbm, "unit": "GB/s", "frac": round(d["GB_s"] * d["launches"] / hbm, 4),
                "peak_source": hbm_src}
    roof.update({"bytes_per_launch": d["bytes"] // d["launches"],
                 "ms_per_launch": round(per_launch_ms, 4), "launches_per_product": d["launches"],
                 "traffic": (round(NCU_TRAFFIC_RATIO[(dom, mode)] * d["bytes"] / d["launches"])
                             if (dom, mode) in NCU_TRAFFIC_RATIO else None),
                 "product": product_fracs(mode, ms_step)})

    out = {
        "metric": METRIC,
        "value": round(ms_step, 4),
        "unit": "ms",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": mode,
        "data": "synthetic",
        "config": workload_config(n, st["kappa"], mode, R),
        "roofline": roof,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms",
                "h2d_bytes_per_step": 8 * n * R, "d2h_bytes_per_step": 8 * n * R},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk,
        "t_build_ms": round(t_build, 1),
        "build_phase_ms": [round(v, 1) for v in st["build_ms"]],
        "stats": {"far_values": st["far_values"], "near_entries": st["near_entries"],
                  "max_rank": st["max_rank"], "npairs": st["npairs"],
                  "unconverged": st["unconverged"],
                  "compression_ratio": st["compression_ratio"],
                  "max_rank_per_level": st["max_rank_per_level"],
                  "values_per_level": st["values_per_level"]},
        "modes": {m: {"ms": round(v["ms"], 4), **product_fracs(m, v["ms"]),
                      "clocks_sm_mhz": v["clocks"].get("sm_mhz"),
                      "phases_serialized": phases[m]}
                  for m, v in per_mode.items()},
    }
    if leg is not None:
        cb = leg.result()
        ncpu, model = host_cpu()
        if "t_matvec_s" in cb:
            out["cpu_baseline"] = {
                "value": round(cb["t_matvec_s"] * 1e3, 1), "unit": "ms", "cores": 1,
                "kind": "oracle",
                "sample": "the full workload: oracle Alg. 2 product at N=%d (kappa %d), median "
                          "of 3 on one host core (%s); oracle build %.1f s" % (
                              n, cb["kappa"], ", ".join("%.2f s" % t for t in cb["all_s"]),
                              cb["build_s"]),
                "host_cores": ncpu, "cpu_model": model}
            yd = cb["y_direct_rows"]
            errs = {}
            for m, v in per_mode.items():
                yr = (v["y"][0] if R > 1 else v["y"]).cpu().numpy()[rows]  # first RHS
                errs[m] = {"rel2_256_rows": float(np.linalg.norm(yr - yd) / np.linalg.norm(yd)),
                           "max_rel_256_rows": float(np.max(np.abs(yr - yd) / np.abs(yd)))}
            y64 = per_mode["f64"]["y"] if "f64" in per_mode else None
            if y64 is not None:
                for m, v in per_mode.items():
                    errs[m]["rel2_vs_f64_product"] = float(torch.linalg.norm(v["y"] - y64)
                                                           / torch.linalg.norm(y64))
            out["error_vs_direct"] = errs
        else:
            out["cpu_baseline"] = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle",
                                   "sample": "oracle leg failed: %s" % cb.get("error", "timeout"),
                                   "host_cores": ncpu, "cpu_model": model}
    for v in per_mode.values():
        del v["y"]
    g.close()
    if ws == 1 and not args.no_extras:
        out["extras"] = extras(pkg, inputs, n, args.n_learned, args.extras, args.batch_sets)
    return out


def run_reference(args, ws, rank):
    """The CPU oracle on one host core, on the same workload: its build
    (Alg. 1, untimed), then each step one oracle Alg. 2 product of the whole
    N = 2^20 problem.  Only rank 0 works; the other ranks return at once."""
    if rank != 0:
        return None
    import oracle
    from paper_2204_05536_gb300 import inputs
    oracle.build()
    n = args.points
    pts = inputs.uniform(n, seed=0)
    x = inputs.rhs(n, seed=1)
    t0 = time.perf_counter()
    o = oracle.Oracle(pts, oracle.kernel("mq", 1.0 / np.sqrt(n)), LEAF, EPS, root=ROOT_BOX)
    t_build = time.perf_counter() - t0
    for _ in range(args.warmup):
        o.matvec(x)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.matvec(x)
        ts.append(time.perf_counter() - t0)
    v = statistics.mean(ts) * 1e3
    ncpu, model = host_cpu()
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "ms",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 2),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(n, o.kappa, "f64"),
        "cpu_baseline": {"value": round(v, 2), "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": "the full workload: oracle Alg. 2 product at N=%d (kappa %d), "
                                   "mean of %d on one host core; oracle build %.1f s untimed"
                                   % (n, o.kappa, args.steps, t_build),
                         "host_cores": ncpu, "cpu_model": model},
        "e2e": {"value": round(v, 2), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
