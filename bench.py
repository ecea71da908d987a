"""Benchmark of the SPDE sampler on one node (one process per GPU).

Workload (the 128^3 headline case): embedding grid 128^3 on [0,1]^3,
kappa = 20, sigma = 1, nu = 1/2; target mesh = jittered 6-tet split of
96^3 cubes on the L-prism [0.05,0.95]^3 minus {x > 0.5, y > 0.5}
(3,981,312 tets); 64 samples per step, FP32 MINRES + V-cycle inside FP64
refinement to a relative FP64 residual of 1e-10; lognormal output
exp(theta_h) on the tets.  A step draws a fresh batch (its own Philox sample
indices), so every step solves new systems.  The per-step working set
(~21 GB of solver state) is far larger than L2, so no flush is needed.

Metric: samples/s of the batched mixed-precision path (whole job over all
ranks), with per-step (64-sample batch) latency p50/p99, next to the plain
FP64 GPU path measured on the same workload and the relative L2 difference
of their fields.  Ranks shard the samples (weak scaling, no collective on
the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "spde_sampler_128cube_lprism96", "grid_n": 128, "kappa": 20.0, "sigma": 1.0, "nu": 0.5,
            "mesh": "L-prism 96^3 cubes x 6 tets, jitter +-h/4 (seed 1)", "ntets": 3981312, "batch": 64,
            "tol": 1e-10, "seed": 1, "output": "lognormal f32 on tets",
            "l2_note": "inputs larger than L2 (solver state ~21 GB per step)"}
METRIC = "samples/s & p50/p99 latency at 1e-6 rel L2 vs plain FP64 GPU path, 128³ grid"

# serving stream: 4-level hierarchy (grid n, L-prism cubes m), requests as the MLMC driver would send them
SERVE_LEVELS = [(32, 24), (64, 48), (128, 96), (256, 192)]
SERVE_KAPPAS = (10.0, 20.0, 40.0)


# ---------------------------------------------------------------- host logic
_T0 = time.time()


def log(msg):
    sys.stderr.write("[bench %7.1fs] %s\n" % (time.time() - _T0, msg))
    sys.stderr.flush()


def first_sample(step, rank, world, batch):
    """Philox sample index of the first sample of (step, rank): disjoint batches."""
    return (step * world + rank) * batch


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(value, world):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(name):
    """DRAM bytes per launch per column from a committed ncu summary, if the
    kernel's sources are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(name)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    try:
        blob = b"".join(open(os.path.join(ROOT, s), "rb").read() for s in rec["sources"])
    except OSError:
        return None
    if hashlib.sha256(blob).hexdigest() != rec["sources_sha256"]:
        return None
    return rec


def serve_requests(nreq, rate, seed=7):
    """Poisson arrivals; level ~ U{0..3}; nsamples = floor(exp(U(0, ln 256))) in [1, 256];
    kappa in {10, 20, 40}; sigma ~ U(0.5, 2); an independent Philox seed per request."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    out = []
    for k in range(nreq):
        ns = int(min(256, max(1, np.floor(np.exp(rng.uniform(0.0, np.log(256.0)))))))
        out.append({"t": float(t[k]), "level": int(rng.integers(0, 4)), "nsamples": ns,
                    "kappa": float(SERVE_KAPPAS[int(rng.integers(0, 3))]), "sigma": float(rng.uniform(0.5, 2.0)),
                    "seed": int(rng.integers(1, 2 ** 62))})
    return out


def run_serving(pkg, smp, outbufs, reqs, poll_sleep=0.0005):
    """Open-loop submission at the requests' arrival times; latency = submit -> done (library clock)."""
    import numpy as np
    t0 = time.perf_counter()
    pending, lat, statuses = {}, [], []
    samples = 0

    def poll_all():
        for rid in list(pending):
            done, ms, st = pkg.spde_poll(smp.ctx, rid)
            if done:
                lat.append(ms)
                statuses.append(st)
                del pending[rid]

    for r in reqs:
        while time.perf_counter() - t0 < r["t"]:
            poll_all()
            time.sleep(poll_sleep)
        rid = pkg.spde_submit(smp.ctx, r["level"], r["nsamples"], r["kappa"], r["sigma"], r["seed"], 0,
                              pkg.SPDE_OUT_LOGNORMAL, outbufs[r["level"]])
        pending[rid] = r
        samples += r["nsamples"]
    while pending:
        poll_all()
        time.sleep(poll_sleep)
    span = time.perf_counter() - t0
    lat = np.sort(np.array(lat))
    return {"requests": len(reqs), "samples": samples, "makespan_s": span, "samples_per_s": samples / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "all_ok": all(st == pkg.SPDE_OK for st in statuses)}


_MESHES = {}


def lprism_cached(m):
    """The jittered L-prism of m^3 cubes (generated once per process)."""
    if m not in _MESHES:
        from synth import lprism_mesh
        _MESHES[m] = lprism_mesh(m)
    return _MESHES[m]


def serving_setup(pkg, local):
    """Sampler with the 4-level hierarchy and per-level shared output buffers (throughput runs
    overwrite them; serving correctness is covered by the tests)."""
    import torch
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-8, device=local)
    outbufs = {}
    for lvl, (n, m) in enumerate(SERVE_LEVELS):
        xyz, tets = lprism_cached(m)
        smp.add_level(lvl, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        smp.attach_mesh(lvl, xyz, tets)
        outbufs[lvl] = torch.empty((256, len(tets)), dtype=torch.float32, device="cuda")
    return smp, outbufs


MLMC_SAMPLES = (4096, 1024, 256, 64)


def timed_call(pkg, smp, stream, fn):
    """Device time (ms) of fn() on `stream`, CUDA events on that stream, outcome collected after."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    pkg.spde_wait(smp.ctx)
    return a.elapsed_time(b)


def run_mlmc_levels(pkg, local, stream, modes=(1, 0)):
    """The 4-level MLMC batch: 32^3/64^3/128^3/256^3 grids with L-prism 24^3/48^3/96^3/192^3 meshes,
    4096/1024/256/64 samples, kappa 20, tol 1e-8, lognormal FP32 out.  Each level has its own context
    (one level's workspace at a time) with the schedule the autotuner stored for (grid, batch); one call
    per level after a warm-up call, timed with CUDA events, through the graph-driven path (one graph
    launch per level and batch) and the synchronous host loop."""
    import torch
    rows, tot = [], {"graphs": 0.0, "host_loop": 0.0}
    for (n, m), S in zip(SERVE_LEVELS, MLMC_SAMPLES):
        xyz, tets = lprism_cached(m)
        row = {"grid": n, "mesh": "L-prism %d^3 cubes" % m, "ntets": int(len(tets)), "samples": S}
        out = torch.empty((S, len(tets)), dtype=torch.float32, device="cuda")
        tune = tuning_for(n, S)
        row["schedule"] = ({k: tune[k] for k in ("omega", "inner_tol", "flux_diag", "sweep_planes")}
                           if tune else "context defaults")
        for g in modes:
            key = "graphs" if g else "host_loop"
            smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-8, device=local, use_graphs=g)
            smp.add_level(0, n)
            smp.attach_mesh(0, xyz, tets)
            if tune:
                pkg.spde_level_set_tuning(smp.ctx, 0, tune)
            smp.sample(0, S, 20.0, 1.0, 3, 10 ** 7, pkg.SPDE_OUT_LOGNORMAL, out, stream)  # warm-up
            ms = timed_call(pkg, smp, stream, lambda: pkg.spde_sample(smp.ctx, 0, S, 20.0, 1.0, 3, 0,
                                                                       pkg.SPDE_OUT_LOGNORMAL, out, stream))
            st = smp.stats()
            row[key] = {"samples_per_s": S / (ms / 1000.0), "ms": ms, "outer_iters": st["outer_iters"],
                        "inner_iters": st["inner_iters"], "max_rel_residual": st["max_rel_residual"]}
            tot[key] += ms
            smp.close()
        del out
        rows.append(row)
    total = sum(MLMC_SAMPLES)
    return {"levels": rows, "kappa": 20.0, "sigma": 1.0, "tol": 1e-8, "output": "lognormal f32 on tets",
            "hierarchy_ms": tot, "hierarchy_samples": total,
            "hierarchy_samples_per_s": {k: total / (v / 1000.0) for k, v in tot.items() if v > 0}}


def run_fp16_coarse(pkg, local, stream):
    """Iterations and residual with the coarse kernel's levels stored in FP16 against FP32, on the
    headline grid (128^3, kappa 20, 64 samples, tol 1e-10) and the large level (512^3, kappa 40,
    2 samples, tol 1e-8); grid output, one timed call after a warm-up call per setting."""
    import torch
    res = {}
    for n, kappa, S, tol in ((128, 20.0, 64, 1e-10), (512, 40.0, 2, 1e-8)):
        out = torch.empty((S, n ** 3), dtype=torch.float32, device="cuda")
        row = {"kappa": kappa, "samples": S, "tol": tol}
        for fp16 in (0, 1):
            smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=tol, device=local, coarse_fp16=fp16)
            smp.add_level(0, n)
            smp.sample(0, S, kappa, 1.0, 3, 10 ** 7, pkg.SPDE_OUT_GRID_GAUSSIAN, out, stream)
            ms = timed_call(pkg, smp, stream, lambda: pkg.spde_sample(smp.ctx, 0, S, kappa, 1.0, 3, 0,
                                                                       pkg.SPDE_OUT_GRID_GAUSSIAN, out, stream))
            st = smp.stats()
            row["fp16" if fp16 else "fp32"] = {"ms": ms, "outer_iters": st["outer_iters"],
                                               "inner_iters": st["inner_iters"],
                                               "max_rel_residual": st["max_rel_residual"]}
            smp.close()
        del out
        res["%d^3" % n] = row
    res["levels_in_fp16"] = "those of the one-CTA coarse kernel (<= 4096 cells: 16^3 and below on a cube)"
    return res


def run_large(pkg, local, stream):
    """The large single level: 512^3 grid, kappa 40, batch of 2, tol 1e-8, L-prism 160^3 cubes
    (18.4 M tets), FP16 storage of the coarse kernel's levels, lognormal FP32 out; one timed call
    after a warm-up call."""
    import torch
    n, m, S, kappa = 512, 160, 2, 40.0
    xyz, tets = lprism_cached(m)
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-8, device=local, coarse_fp16=1)
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    setup = smp.stats()
    out = torch.empty((S, len(tets)), dtype=torch.float32, device="cuda")
    smp.sample(0, S, kappa, 1.0, 3, 10 ** 7, pkg.SPDE_OUT_LOGNORMAL, out, stream)
    ms = timed_call(pkg, smp, stream, lambda: pkg.spde_sample(smp.ctx, 0, S, kappa, 1.0, 3, 0,
                                                               pkg.SPDE_OUT_LOGNORMAL, out, stream))
    st = smp.stats()
    fp = pkg.spde_query_footprint(smp.ctx, 0, S)
    smp.close()
    del out
    return {"value": S / (ms / 1000.0), "unit": "samples/s", "ms_per_call": ms, "samples": S, "grid": "512^3",
            "kappa": kappa, "tol": 1e-8, "mesh": "L-prism %d^3 cubes" % m, "ntets": int(len(tets)),
            "nnz": setup["nnz"], "clip_ms": setup["setup_ms"], "solver_workspace_GB": fp / 1e9,
            "outer_iters": st["outer_iters"], "inner_iters": st["inner_iters"],
            "max_rel_residual": st["max_rel_residual"],
            "coarse_storage": "fp16 (levels of the one-CTA coarse kernel; FP32 arithmetic)"}


# ---------------------------------------------------------------- CPU oracle arm
class OracleSampler:
    """The FP64 oracle as it stands, timed whole on the host cores, on the headline workload.

    Set-up (once, reported apart, like the GPU's clipping): the L-prism mesh,
    G by the oracle's C clipping statement (half-space splitting, OpenMP over
    tets), Pi = W_h^{-1} G as a SciPy CSR matrix.  Per sample, measured end to
    end: Philox normals, the exact DCT solve on the full 128^3 grid, Pi theta
    (one sparse product over all 3,981,312 tets) and exp.
    """

    def __init__(self, xyz=None, tets=None):
        import numpy as np
        from oracle import clip_c, project
        from synth import lprism_mesh
        self.n = WORKLOAD["grid_n"]
        if xyz is None:
            xyz, tets = lprism_mesh(96)
        t0 = time.perf_counter()
        rp, col, val = clip_c.coupling_csr(xyz, tets, self.n)
        self.t_clip = time.perf_counter() - t0
        self.pi = project.projection_matrix(rp, col, val, project.tet_volumes(xyz, tets), self.n ** 3)
        self.ntets, self.nnz = len(tets), len(val)
        self.np = np

    def sample(self, sample_index):
        """Wall time (s) of one whole sample."""
        from oracle import mixed, philox, project
        t0 = time.perf_counter()
        xi = philox.normals(self.n ** 3, WORKLOAD["seed"], sample_index)
        th = mixed.solve_dct(self.n, WORKLOAD["kappa"], WORKLOAD["sigma"], xi)
        out = self.np.exp(project.project_csr(self.pi, th))
        assert out.shape == (self.ntets,)
        return time.perf_counter() - t0

    def describe(self, per_sample_s):
        return ("whole samples of the 128^3 / L-prism 96^3 workload: Philox normals + exact DCT solve (scipy.fft, "
                "all cores) + CSR projection of all %d tets (%d nonzeros) + exp, %.3f s per sample; Pi set-up "
                "(C clipping statement, all cores) %.1f s, excluded like the GPU's" % (self.ntets, self.nnz,
                                                                                      per_sample_s, self.t_clip))


def splu_baseline(n=16):
    """Factor-once SuperLU of the oracle's assembled mixed system and one solve (16^3)."""
    import scipy.sparse.linalg as spla
    from oracle import mixed, philox
    ms = mixed.MixedSystem(n)
    t0 = time.perf_counter()
    lu = spla.splu(ms.matrix(WORKLOAD["kappa"]))
    t_factor = time.perf_counter() - t0
    t0 = time.perf_counter()
    lu.solve(ms.rhs(WORKLOAD["kappa"], WORKLOAD["sigma"], philox.normals(n ** 3, 1, 0)))
    return {"grid": "%d^3" % n, "factor_s": t_factor, "solve_s": time.perf_counter() - t0}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    os_ = OracleSampler()
    for i in range(args.warmup):
        os_.sample(1000 + i)
    t0 = time.perf_counter()
    costs = [os_.sample(i) for i in range(args.steps)]
    wall = time.perf_counter() - t0
    value = args.steps / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism="samples sharded over 1 rank(s)"),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": os_.describe(statistics.mean(costs)), "setup_s": os_.t_clip},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

# ---------------------------------------------------------------- DCT comparison leg
def dct_ortho(x, dim):
    """Orthonormal DCT-II along `dim` through one complex FFT of the even/odd reordering (Makhoul)."""
    import torch
    n = x.shape[dim]
    x = x.movedim(dim, -1)
    v = torch.cat([x[..., ::2], x[..., 1::2].flip(-1)], dim=-1)
    k = torch.arange(n, device=x.device, dtype=x.dtype)
    tw = torch.polar(torch.ones_like(k), -math.pi * k / (2 * n))
    c = 2.0 * (torch.fft.fft(v, dim=-1) * tw).real
    sc = torch.full_like(k, math.sqrt(0.5 / n))
    sc[0] = math.sqrt(0.25 / n)
    return (c * sc).movedim(-1, dim).contiguous()


def idct_ortho(y, dim):
    """Inverse of dct_ortho along `dim` (the orthonormal DCT-III), one complex inverse FFT."""
    import torch
    n = y.shape[dim]
    y = y.movedim(dim, -1)
    k = torch.arange(n, device=y.device, dtype=y.dtype)
    sc = torch.full_like(k, math.sqrt(0.5 / n))
    sc[0] = math.sqrt(0.25 / n)
    c = y / sc
    cr = torch.cat([torch.zeros_like(c[..., :1]), c[..., 1:].flip(-1)], dim=-1)
    v = torch.fft.ifft(torch.polar(torch.ones_like(k), math.pi * k / (2 * n)) * torch.complex(c, -cr) / 2,
                       dim=-1).real
    x = torch.empty_like(v)
    x[..., ::2] = v[..., :(n + 1) // 2]
    x[..., 1::2] = v[..., (n + 1) // 2:].flip(-1)
    return x.movedim(-1, dim).contiguous()


def dct_field(xi, n, h, kappa, sigma):
    """Cell field g S^{-1} W^{1/2} xi for constant kappa on the n^3 box, by the DCT-II diagonalisation
    of the Schur complement (exact there, unlike for a varying kappa(x)); xi is [S][n^3], z slowest."""
    import torch
    k = torch.arange(n, device=xi.device, dtype=torch.float64)
    l1 = 12.0 * torch.sin(math.pi * k / (2 * n)) ** 2 / (2.0 + torch.cos(math.pi * k / n))
    lam = kappa ** 2 * h ** 3 + h * (l1[:, None, None] + l1[None, :, None] + l1[None, None, :])
    f = (h ** 1.5) * xi.reshape(-1, n, n, n)
    for d in (1, 2, 3):
        f = dct_ortho(f, d)
    f = f / lam
    for d in (1, 2, 3):
        f = idct_ortho(f, d)
    g = sigma * (4.0 * math.pi) ** 0.75 * math.sqrt(kappa) * math.sqrt(math.gamma(2.0) / math.gamma(0.5))
    return (g * f).reshape(xi.shape)


def fp64_peak_tflops():
    """FP64 roof of this GPU (the peaks file has none): a float64 4096^3 matmul, best of 5."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 2.0 * 4096 ** 3 / (best / 1000.0) / 1e12


# FP64 arithmetic per cell of the FP64 kernels (own count of the operations each performs)
FP64_FLOPS_PER_CELL = {
    "residual64": 10.0,       # cell row: 3 differences, 2 sums, kappa term (fma), F - Au, square-accumulate (fma)
    "flux_from_theta": 18.0,  # per axis: difference, fma, scale (forward), fma (back substitution)
}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1712_06758_gb300 as pkg
    from synth import lprism_mesh

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    W = dict(WORKLOAD)
    if args.batch:
        W["batch"] = args.batch
        W["workload"] += "_batch%d" % args.batch
    if args.grid:  # a smaller grid and its L-prism mesh (profiling runs)
        W.update(grid_n=args.grid, ntets=None, mesh="L-prism %d^3 cubes x 6 tets, jitter +-h/4 (seed 1)" % (3 * args.grid // 4))
        W["workload"] = "spde_sampler_%dcube_lprism%d" % (args.grid, 3 * args.grid // 4)
    S, n = W["batch"], W["grid_n"]
    log("mesh")
    xyz, tets = lprism_cached(3 * n // 4)
    log("attach")
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=W["tol"], device=local)
    smp.add_level(0, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    smp.attach_mesh(0, xyz, tets)
    setup = smp.stats()
    ntets = smp.ntets(0)
    out = torch.empty((S, ntets), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(i, dst):
        pkg.spde_sample(smp.ctx, 0, S, W["kappa"], W["sigma"], W["seed"], first_sample(i, rank, world, S),
                        pkg.SPDE_OUT_LOGNORMAL, dst, stream)

    log("warmup")
    for i in range(args.warmup):
        step(1000 + i, out)
        log("warmup step %d: %s" % (i, smp.stats()))
    iters = smp.stats()
    clocks = ClockSampler(local)
    pkg.spde_profile_enable(smp.ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    log("timed region")
    barrier(world)
    torch.cuda.synchronize()
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(i, out)
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    log("timed region done")
    clk = clocks.stop()
    prof = pkg.spde_profile(smp.ctx)
    pkg.spde_profile_enable(smp.ctx, False)
    elapsed_ms = reduce_max(t_start.elapsed_time(t_end), world)
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    value = world * args.steps * S / (elapsed_ms / 1000.0)

    # dominant kernel, live roofline
    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda p: p["ms"])
    achieved = dom["bytes"] / (dom["ms"] / 1000.0) / 1e9 if dom["ms"] > 0 else 0.0
    per_launch_bytes = dom["bytes"] / max(dom["launches"], 1)
    tr = kernel_traffic(dom["name"])
    traffic = None
    if tr:
        traffic = tr["dram_bytes_per_launch_per_column"] * per_launch_bytes / tr["algorithmic_bytes_per_launch_per_column"]
    roofline = {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic, "avg_launch_us": 1000.0 * dom["ms"] / max(dom["launches"], 1),
                "algorithmic_bytes_per_launch": per_launch_bytes, "share_of_step": dom["ms"] / elapsed_ms}
    kernels = {p["name"]: {"launches": p["launches"], "ms": round(p["ms"], 3),
                           "GBps": round(p["bytes"] / p["ms"] / 1e6, 1) if p["ms"] > 0 else None}
               for p in prof if p["launches"]}
    gpu_launches = int(sum(p["launches"] for p in prof))

    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
                              "config": W, "roofline": roofline, "kernels": kernels, "gpu_launches": gpu_launches,
                              "note": "reduced run (no plain path, e2e or CPU baseline)"}), flush=True)
        smp.close()
        return
    # e2e: same call with a pinned host output (the output crosses to host memory inside every call:
    # the output kernels write the mapped pinned buffer directly)
    log("e2e")
    host = torch.empty((S, ntets), dtype=torch.float32, pin_memory=True)
    host_np = host.numpy()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        pkg.spde_sample(smp.ctx, 0, S, W["kappa"], W["sigma"], W["seed"], first_sample(args.steps + i, rank, world, S),
                        pkg.SPDE_OUT_LOGNORMAL, host_np, stream)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e = {"value": world * args.steps * S / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": int(S * ntets * 4),
           "note": "spde_sample into pinned host memory; every call returns with the output in host memory"}

    # the same steps through the graph-driven path (per-kernel timing off): every call returns once
    # enqueued, convergence is decided on the device, the outcome is collected at the end
    log("graph path")
    step(2000, out)  # captures the graph
    torch.cuda.synchronize()
    pkg.spde_wait(smp.ctx)
    ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    ga.record(stream)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(3000 + i, out)
    host_enqueue_s = time.perf_counter() - t0
    gb.record(stream)
    torch.cuda.synchronize()
    pkg.spde_wait(smp.ctx)
    barrier(world)
    graph_ms = reduce_max(ga.elapsed_time(gb), world)
    gst = smp.stats()
    graphs = {"value": world * args.steps * S / (graph_ms / 1000.0), "unit": "samples/s",
              "ms_per_step": graph_ms / args.steps, "host_enqueue_ms_per_step": 1000.0 * host_enqueue_s / args.steps,
              "outer_iters": gst["outer_iters"], "inner_iters": gst["inner_iters"],
              "note": "spde_sample with use_graphs = 1: one graph launch per 64-sample call"}

    # serving: the open-loop stream on the 4-level hierarchy (tol 1e-8) swept over the request rates
    log("serving sweep")
    serving = serve_sweep(pkg, local, args.serve_requests)

    line = None
    if rank == 0:
        # plain FP64 path on the same workload (first samples of step 0), and the field difference
        log("plain path")
        nplain = args.plain_samples
        ref_out = torch.empty((S, ntets), dtype=torch.float32, device="cuda")
        step(0, ref_out)
        plain = pkg.Sampler(pkg.SPDE_PREC_FP64, tol=W["tol"], device=local)
        plain.add_level(0, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        plain.attach_mesh(0, xyz, tets)
        pout = torch.empty((nplain, ntets), dtype=torch.float32, device="cuda")
        plain.sample(0, 1, W["kappa"], W["sigma"], W["seed"], 0, pkg.SPDE_OUT_LOGNORMAL, pout[:1])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        plain.sample(0, nplain, W["kappa"], W["sigma"], W["seed"], first_sample(0, rank, world, S),
                     pkg.SPDE_OUT_LOGNORMAL, pout, stream)
        b.record(stream)
        torch.cuda.synchronize()
        plain_rate = nplain / (a.elapsed_time(b) / 1000.0)
        pst = plain.stats()
        d = (ref_out[:nplain].double() - pout.double()).norm(dim=1) / pout.double().norm(dim=1)
        plain.close()
        # the Schur-complement CG solver on the same workload and batch (same samples as step 0)
        log("schur-cg path")
        sch = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=W["tol"], device=local, solver=pkg.SPDE_SOLVER_SCHUR_CG)
        sch.add_level(0, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        sch.attach_mesh(0, xyz, tets)
        sout = torch.empty((S, ntets), dtype=torch.float32, device="cuda")
        sch.sample(0, S, W["kappa"], W["sigma"], W["seed"], first_sample(1000, rank, world, S),
                   pkg.SPDE_OUT_LOGNORMAL, sout, stream)
        torch.cuda.synchronize()
        a.record(stream)
        sch.sample(0, S, W["kappa"], W["sigma"], W["seed"], first_sample(0, rank, world, S),
                   pkg.SPDE_OUT_LOGNORMAL, sout, stream)
        b.record(stream)
        torch.cuda.synchronize()
        sch_rate = S / (a.elapsed_time(b) / 1000.0)
        sst = sch.stats()
        ds = (ref_out.double() - sout.double()).norm(dim=1) / sout.double().norm(dim=1)
        sch.close()
        del sout
        # direct DCT solve (torch.fft, FP64) between the same noise and projection kernels
        log("dct path")
        xi = torch.empty((S, n ** 3), dtype=torch.float64, device="cuda")
        dout = torch.empty((S, ntets), dtype=torch.float32, device="cuda")

        def dct_step():
            pkg.spde_noise(n ** 3, S, W["seed"], first_sample(0, rank, world, S), 1.0, xi, stream)
            th = dct_field(xi, n, 1.0 / n, W["kappa"], W["sigma"])
            pkg.spde_project(smp.ctx, 0, S, th, pkg.SPDE_OUT_LOGNORMAL, dout, stream)

        dct_step()
        torch.cuda.synchronize()
        a.record(stream)
        dct_step()
        b.record(stream)
        torch.cuda.synchronize()
        dct_rate = S / (a.elapsed_time(b) / 1000.0)
        dd = (ref_out.double() - dout.double()).norm(dim=1) / dout.double().norm(dim=1)
        del xi, dout
        # cell-wise kappa(x), sigma(x) on the same grid, mesh and batch
        log("fields path")
        cc = (np.arange(n) + 0.5) / n
        fz, fy, fx = np.meshgrid(cc, cc, cc, indexing="ij")
        kap_c = (20.0 * (1.0 + 0.5 * np.sin(2 * np.pi * fx) * np.cos(2 * np.pi * fz))).ravel()
        sig_c = (0.75 + 0.5 * fy).ravel()
        smp.set_fields(0, kap_c, sig_c)
        smp.sample_fields(0, S, W["seed"], first_sample(1000, rank, world, S), pkg.SPDE_OUT_LOGNORMAL, out, stream)
        torch.cuda.synchronize()
        a.record(stream)
        smp.sample_fields(0, S, W["seed"], first_sample(0, rank, world, S), pkg.SPDE_OUT_LOGNORMAL, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        fields_rate = S / (a.elapsed_time(b) / 1000.0)
        fst = smp.stats()
        # end to end: kappa and sigma uploaded from host arrays and the output read into pinned
        # host memory every step (new fields drop the level's captured graphs: each step recaptures)
        nfe = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(nfe):
            smp.set_fields(0, kap_c, sig_c)
            smp.sample_fields(0, S, W["seed"], first_sample(2000 + i, rank, world, S), pkg.SPDE_OUT_LOGNORMAL,
                              host_np, stream)
        torch.cuda.synchronize()
        fields_e2e = {"value": nfe * S / (time.perf_counter() - t0), "unit": "samples/s", "steps": nfe,
                      "h2d_bytes_per_step": int(2 * 8 * kap_c.size), "d2h_bytes_per_step": int(S * ntets * 4)}
        smp.set_fields(0, None, None)
        # the crooked-pipe stand-in: quarter cylinder (radius 2, height 7, elements graded toward the
        # r = 1 layer) in a cubic box of side 8 whose (0,3)^2 x (0,8) corner is the paper's embedding box
        log("quarter-cylinder workload")
        from synth import quarter_cylinder_mesh
        cxyz, ctets = quarter_cylinder_mesh(32, 48, 112)
        cyl = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=W["tol"], device=local)
        cyl.add_level(0, n, (0.0, 0.0, 0.0), (8.0, 8.0, 8.0))
        cyl.attach_mesh(0, cxyz, ctets)
        cset = cyl.stats()
        cout = torch.empty((S, len(ctets)), dtype=torch.float32, device="cuda")
        cyl.sample(0, S, 2.0, 1.0, W["seed"], first_sample(1000, rank, world, S), pkg.SPDE_OUT_LOGNORMAL, cout, stream)
        torch.cuda.synchronize()
        a.record(stream)
        cyl.sample(0, S, 2.0, 1.0, W["seed"], first_sample(0, rank, world, S), pkg.SPDE_OUT_LOGNORMAL, cout, stream)
        b.record(stream)
        torch.cuda.synchronize()
        cyl_rate = S / (a.elapsed_time(b) / 1000.0)
        cst = cyl.stats()
        cyl.close()
        # the same mesh with its axis along x ((x, y, z) -> (z, x, y)) on a 128 x 64 x 64 box grid of
        # the same spacing: [0,8] x [0,4] x [0,4], a quarter of the cube's cells
        bxyz = np.ascontiguousarray(cxyz[:, [2, 0, 1]])
        bdims = (128, 64, 64)
        cylb = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=W["tol"], device=local)
        cylb.add_level(0, bdims, (0.0, 0.0, 0.0), (8.0, 4.0, 4.0))
        cylb.attach_mesh(0, bxyz, ctets)
        cylb.sample(0, S, 2.0, 1.0, W["seed"], first_sample(1000, rank, world, S), pkg.SPDE_OUT_LOGNORMAL, cout, stream)
        torch.cuda.synchronize()
        a.record(stream)
        cylb.sample(0, S, 2.0, 1.0, W["seed"], first_sample(0, rank, world, S), pkg.SPDE_OUT_LOGNORMAL, cout, stream)
        b.record(stream)
        torch.cuda.synchronize()
        cylb_rate = S / (a.elapsed_time(b) / 1000.0)
        cbst = cylb.stats()
        cylb.close()
        del cout
        cylinder = {"value": cyl_rate, "unit": "samples/s", "samples": S, "ntets": int(len(ctets)),
                    "mesh": "quarter cylinder r = 2, height 7, 32 radial (graded to r = 1) x 48 x 112 cells",
                    "box": "[0,8]^3, n = %d" % n, "kappa": 2.0, "sigma": 1.0, "clip_ms": cset["setup_ms"],
                    "nnz": cset["nnz"], "outer_iters": cst["outer_iters"], "inner_iters": cst["inner_iters"],
                    "paper_box_fraction_of_grid": 3.0 * 3.0 * 8.0 / 8.0 ** 3,
                    "box_grid": {"value": cylb_rate, "unit": "samples/s", "grid": "128 x 64 x 64, h = 1/16",
                                 "axis": "x", "outer_iters": cbst["outer_iters"], "inner_iters": cbst["inner_iters"],
                                 "paper_box_fraction_of_grid": 3.0 * 3.0 * 8.0 / (8.0 * 4.0 * 4.0)}}
        # the SPE10-sized box (Sec. 7.2): 60 x 220 x 85 hexes of 20 x 10 x 2 ft, six tets each, centred
        # in the 1600 x 2420 x 240 ft bounding box, on a 256 x 256 x 32 box grid of 9.5 ft cells
        # (2432 x 2432 x 304 ft) whose corner is the bounding box's
        log("SPE10-box workload")
        from synth import spe10_mesh
        exyz, etets = spe10_mesh()
        edims, eh, es = (256, 256, 32), 9.5, 64
        spe = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=W["tol"], device=local)
        spe.add_level(0, edims, (0.0, 0.0, 0.0), tuple(eh * v for v in edims))
        spe.attach_mesh(0, exyz, etets)
        eset = spe.stats()
        eout = torch.empty((es, len(etets)), dtype=torch.float32, device="cuda")
        spe.sample(0, es, 0.02, 1.0, W["seed"], first_sample(1000, rank, world, es), pkg.SPDE_OUT_LOGNORMAL, eout, stream)
        torch.cuda.synchronize()
        a.record(stream)
        spe.sample(0, es, 0.02, 1.0, W["seed"], first_sample(0, rank, world, es), pkg.SPDE_OUT_LOGNORMAL, eout, stream)
        b.record(stream)
        torch.cuda.synchronize()
        spe_rate = es / (a.elapsed_time(b) / 1000.0)
        est = spe.stats()
        spe.close()
        del eout
        spe10 = {"value": spe_rate, "unit": "samples/s", "samples": es, "ntets": int(len(etets)),
                 "mesh": "SPE10 box 1200 x 2220 x 170 ft, 60 x 220 x 85 hexes of 20 x 10 x 2 ft, Kuhn-split",
                 "grid": "%d x %d x %d cells of %g ft from the origin" % (edims + (eh,)), "kappa": 0.02,
                 "correlation_length_ft": 50.0, "sigma": 1.0, "clip_ms": eset["setup_ms"], "nnz": eset["nnz"],
                 "outer_iters": est["outer_iters"], "inner_iters": est["inner_iters"],
                 "paper_box_fraction_of_grid": 1600.0 * 2420.0 * 240.0 / float(np.prod(edims) * eh ** 3)}
        # FP64 roof and the FP64 kernels against it
        log("fp64 roof")
        fp64_peak = fp64_peak_tflops()
        fp64 = {"peak_tflops": fp64_peak, "peak_source": "torch float64 matmul 4096^3, best of 5", "kernels": {}}
        for name, fl in FP64_FLOPS_PER_CELL.items():
            kk = kernels.get(name)
            if kk and kk["ms"] > 0:
                tf = fl * float(n) ** 3 * S * kk["launches"] / (kk["ms"] / 1000.0) / 1e12
                fp64["kernels"][name] = {"tflops": tf, "frac": tf / fp64_peak, "flops_per_cell": fl,
                                         "hbm_frac": kk["GBps"] / peak if kk["GBps"] else None}
        # the 4-level MLMC batch and the large single level
        log("mlmc levels")
        mlmc = run_mlmc_levels(pkg, local, stream)
        log("512^3 level")
        large = run_large(pkg, local, stream)
        log("fp16 coarse levels")
        fp16c = run_fp16_coarse(pkg, local, stream)
        # the oracle on the host cores: whole samples of the same workload
        log("cpu baseline")
        oc = OracleSampler(xyz, tets)
        oc.sample(1000)
        costs = [oc.sample(i) for i in range(3)]
        cost = statistics.mean(costs)
        desc = oc.describe(cost)
        splu = splu_baseline(16)
        line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": dict(W, parallelism="samples sharded over %d rank(s)" % world),
                "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                               "per": "one %d-sample batch call" % S},
                "serving": serving,
                "graphs": graphs,
                "mlmc_levels": mlmc,
                "large_512": large,
                "fp16_coarse": fp16c,
                "plain_fp64": {"value": plain_rate, "unit": "samples/s", "samples": nplain,
                               "ratio": value / world / plain_rate, "inner_iters": pst["inner_iters"],
                               "max_rel_l2_vs_mixed": float(d.max())},
                "schur_cg": {"value": sch_rate, "unit": "samples/s", "samples": S, "outer_iters": sst["outer_iters"],
                             "inner_iters": sst["inner_iters"], "max_rel_residual": sst["max_rel_residual"],
                             "max_rel_l2_vs_minres": float(ds.max())},
                "dct_direct": {"value": dct_rate, "unit": "samples/s", "samples": S,
                               "max_rel_l2_vs_minres": float(dd.max()),
                               "note": "constant kappa only; noise and projection kernels shared, FFTs torch.fft FP64"},
                "fields": {"value": fields_rate, "unit": "samples/s", "samples": S,
                           "kappa": "20 (1 + 0.5 sin(2 pi x) cos(2 pi z)) per cell", "sigma": "0.75 + 0.5 y per cell",
                           "outer_iters": fst["outer_iters"], "inner_iters": fst["inner_iters"],
                           "max_rel_residual": fst["max_rel_residual"], "e2e": fields_e2e},
                "fp64": fp64,
                "quarter_cylinder": cylinder,
                "spe10_box": spe10,
                "solver": {"outer_iters": iters["outer_iters"], "inner_iters": iters["inner_iters"],
                           "max_rel_residual": iters["max_rel_residual"]},
                "setup": {"clip_ms": setup["setup_ms"], "nnz": setup["nnz"]},
                "roofline": roofline, "kernels": kernels, "gpu_launches": gpu_launches, "e2e": e2e,
                "clocks": clk,
                "cpu_baseline": {"value": 1.0 / cost, "unit": "samples/s", "cores": os.cpu_count() or 1,
                                 "kind": "oracle", "sample": desc, "setup_s": oc.t_clip, "splu": splu}}
        print(json.dumps(line), flush=True)
    smp.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SERVE_RATES = (10.0, 30.0, 100.0, 300.0, 1000.0)


def serve_sweep(pkg, local, nreq):
    """The serving stream at 10, 30, 100, 300 and 1000 req/s, nreq requests per rate (open loop)."""
    smp, outbufs = serving_setup(pkg, local)
    rows = []
    for rate in SERVE_RATES:
        log("serving at %g req/s" % rate)
        r = run_serving(pkg, smp, outbufs, serve_requests(nreq, rate, seed=int(rate)))
        r["rate_req_per_s"] = rate
        rows.append(r)
    smp.close()
    sat = max(r["samples_per_s"] for r in rows)
    return {"rows": rows, "requests_per_rate": nreq, "levels": [n for n, _ in SERVE_LEVELS],
            "meshes": ["L-prism %d^3 cubes" % m for _, m in SERVE_LEVELS], "tol": 1e-8, "budget_GiB": 120,
            "saturation_samples_per_s": sat,
            "note": "open loop, Poisson arrivals; latency = submit to completion; request mix per rate seeded by the rate"}


TUNING_TABLE = os.path.join(ROOT, "paper_1712_06758_gb300", "tuning_table.json")
TUNE_CASES = [(128, 96, 64)] + [(n, m, s) for (n, m), s in zip(SERVE_LEVELS, MLMC_SAMPLES)]


def tuning_for(n, batch, kappa=20.0):
    """The stored schedule of (grid n^3, batch, kappa), or None."""
    try:
        with open(TUNING_TABLE) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    return table.get("entries", {}).get("%d^3/%d/%g" % (n, batch, kappa))


def run_autotune(args):
    """Runs the library's autotuner on the headline and MLMC workloads and writes the table."""
    import torch
    import paper_1712_06758_gb300 as pkg
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    entries = {}
    for n, m, S in TUNE_CASES:
        log("autotune %d^3 x %d" % (n, S))
        tol = WORKLOAD["tol"] if (n, S) == (128, 64) else 1e-8
        smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=tol, device=local)
        smp.add_level(0, n)
        t = pkg.spde_autotune(smp.ctx, 0, S, 20.0, 1.0)
        t.update({"tol": tol})
        entries["%d^3/%d/%g" % (n, S, 20.0)] = t
        smp.close()
    table = {"what": "schedules picked by spde_autotune (device time of one grid-output call per candidate)",
             "gpu": torch.cuda.get_device_name(local), "entries": entries}
    with open(TUNING_TABLE, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps(table), flush=True)


def run_serve_sweep(args):
    """The serving sweep: rates 10, 30, 100, 300, 1000 req/s, fixed request count per rate."""
    import torch
    import paper_1712_06758_gb300 as pkg
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    print(json.dumps(serve_sweep(pkg, local, args.serve_requests)), flush=True)


def main(argv=None):
    import faulthandler
    faulthandler.dump_traceback_later(120, repeat=True, file=sys.stderr)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--plain-samples", type=int, default=8)
    ap.add_argument("--batch", type=int, default=0, help="override the 64-sample batch (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="headline loop only (profiling runs)")
    ap.add_argument("--grid", type=int, default=0, help="another grid n^3 with an L-prism of (3n/4)^3 cubes (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests per rate of the serving sweep")
    ap.add_argument("--serve-sweep", action="store_true", help="only the serving sweep over 10..1000 req/s")
    ap.add_argument("--autotune", action="store_true", help="run the autotuner and write the tuning table")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.serve_sweep:
        run_serve_sweep(args)
    elif args.autotune:
        run_autotune(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
