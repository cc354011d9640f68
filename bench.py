"""Benchmark: directional H^2 compression of a dense Helmholtz collocation matrix.

Workload (default): n = 32768 Fibonacci-sphere points, kappa = 32, leaf 64,
eps = 1e-4, dense complex64 G (8 GiB) resident in HBM, mixed mode (leaf Gram
matrices from exact bf16 slice products on the tensor cores); the reported
relative error is measured against the complex128 matrix.  One step = one call
of dh2_compress: block norms + nearfield copy, the leaf factorisations of both
bases, the non-leaf level steps, the basis expansion and the projection.

Beside the headline the line carries (unless --skip-secondary) the plain FP64
GPU form and the FP32 form on the same problem with the rank deviations from
them, and the paper's parameter set (eta1 = 20, eta2 = 5) on the same points.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead on
a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

if "--impl" in sys.argv and "reference" in sys.argv:
    # the reference arm times the oracle on one core: BLAS and OpenMP threads are fixed to 1 before numpy
    # loads (the oracle itself is a serial loop over pairs)
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
MODE_LABEL = {"fp32": "FP32 complex64", "fp64": "FP64 complex128",
              "mixed": "mixed complex64 (tensor-core bf16x3 Gram, double-float pivoted Cholesky)"}

# FP32 ALU peak of the GB300 from its unit counts: 152 SMs x 128 FP32 lanes x
# 2 flops per FMA x 2.07 GHz maximum SM clock.
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# DRAM bytes (read + write) of the leaf launches of a kernel (all size classes
# together) at n=32768, kappa=32, leaf 64, from an ncu capture summarised under
# profiles/; valid only for the kernel sources it was measured on (sha1 of
# csrc/dh2_gram.cu + csrc/dh2_pair.cu).
KERNEL_TRAFFIC = {
    # gram_pipe_kernel<32>, <48> x2, gram_kernel<64>: one compression at n=32768 (ncu
    # dram__bytes_read.sum 5865124864 + dram__bytes_write.sum 1023523072)
    ("gram", "mixed"): {"sha1": "08165f8f3a8361e22036447170b4b073d3e7364a", "bytes": 6888647936},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(args):
    kind = ("helmholtz-collocation fibonacci-sphere" if args.kernel == "slp" else
            "helmholtz-double-layer-collocation ellipsoid-2:1:1")
    return {"workload": f"{kind} n={args.n} kappa={args.kappa:g} leaf={args.leaf} "
                        f"eps={args.eps:g} {MODE_LABEL[args.mode]}",
            "kernel": "1/2 I + double layer (Section 7, DLP)" if args.kernel == "dlp" else "single layer",
            "n": args.n, "kappa": args.kappa, "leaf": args.leaf, "eps": args.eps, "eta1": args.eta1,
            "eta2": args.eta2, "zeta": 2.0 / 3.0, "mode": args.mode,
            "nearfield": "copy" if args.nearfield == 0 else "view",
            "l2": "inputs larger than L2 (G is 8 GiB at n=32768)"}


def workload_points(args):
    """Points and (for the double-layer workload) normals of the workload."""
    from synth import ellipsoid_normals, fibonacci_sphere, random_ellipsoid

    if args.kernel == "dlp":
        pts = random_ellipsoid(args.n)
        return pts, ellipsoid_normals(pts)
    return fibonacci_sphere(args.n), None


def workload_matrix(args, P, Nrm, h, dtype, dev):
    """G in the tree's order as a column-major device view (what dh2_compress takes)."""
    from synth.inputs import dlp_matrix_torch, helmholtz_matrix_torch

    if args.kernel == "dlp":
        return dlp_matrix_torch(P, Nrm, args.kappa, dtype, dev)
    return helmholtz_matrix_torch(P, args.kappa, h, dtype, dev).t()  # symmetric: row-major == column-major


# --------------------------------------------------------------------------- oracle baseline

_ORACLE_SETUP = {}


def _oracle_setup(args):
    """The oracle's tree, column sets of both sides and per-pair work for the workload (built once per
    process, not timed)."""
    key = (args.n, args.kappa, args.leaf, args.eta1, args.eta2, args.eps, args.kernel)
    if key not in _ORACLE_SETUP:
        from oracle import dh2_oracle as O
        from synth import mean_nn_distance

        pts, nrm = workload_points(args)
        tp = O.TreeParams(leaf_size=args.leaf, kappa=args.kappa, eta1=args.eta1, eta2=args.eta2)
        cp = O.CompressParams(eps=args.eps)
        tr = O.build_tree(pts, tp)
        leaf_pairs, work = [], {}
        for side in ("row", "col"):
            F = O.column_sets(tr, side)
            for t in range(tr.nclusters()):
                if not tr.is_leaf(t):
                    continue
                for c, blocks in F[t].items():
                    N = sum(tr.size[tr.blocks[b][1] if side == "row" else tr.blocks[b][0]] for b in blocks)
                    leaf_pairs.append((side, t, c, tuple(blocks)))
                    work[(side, t, c)] = tr.size[t] ** 2 * N
        _ORACLE_SETUP[key] = dict(O=O, cp=cp, tr=tr, leaf_pairs=leaf_pairs, work=work, h=mean_nn_distance(pts),
                                  P=pts[tr.perm], Nrm=nrm[tr.perm] if nrm is not None else None, wcache={})
    return _ORACLE_SETUP[key]


def _kernel_block(S, args, r0, r1, c0, c1):
    """Entries G[r0:r1, c0:c1] of the workload matrix in the tree's order, complex128 (input generation,
    never inside a timed region)."""
    P, Nrm, h = S["P"], S["Nrm"], S["h"]
    d = P[r0:r1, None, :] - P[None, c0:c1, :]
    r = np.sqrt((d * d).sum(-1))
    k = args.kappa
    with np.errstate(divide="ignore", invalid="ignore"):
        if Nrm is None:
            g = np.exp(1j * k * r) / (4.0 * math.pi * r)
        else:
            dn = (d * Nrm[None, c0:c1, :]).sum(-1)
            g = (1.0 - 1j * k * r) * np.exp(1j * k * r) / (4.0 * math.pi * r ** 3) * dn
    ii, jj = np.nonzero(r == 0.0)
    g[ii, jj] = 1.0 / (4.0 * math.pi * h) if Nrm is None else 0.5
    return g


def _leaf_matrix(S, args, side, t, blocks):
    """G^omega_tc of one leaf pair (Section 6 leaf step, weights of Remark "Error control"), formed by the
    oracle's own block weights; generation only, not timed."""
    O, tr, cp, wc = S["O"], S["tr"], S["cp"], S["wcache"]
    parts = []
    for b in blocks:
        bt, bs, _, _ = tr.blocks[b]
        if b not in wc:  # omega_b needs the whole block's norm
            Gb = _kernel_block(S, args, tr.start[bt], tr.start[bt] + tr.size[bt], tr.start[bs],
                               tr.start[bs] + tr.size[bs])
            nb = math.sqrt(float(np.sum(Gb.real ** 2 + Gb.imag ** 2)))
            wc[b] = nb * cp.zeta ** (-tr.level[bt]) if nb > 0 else 1.0
        if side == "row":
            blk = _kernel_block(S, args, tr.start[t], tr.start[t] + tr.size[t], tr.start[bs], tr.start[bs] + tr.size[bs])
        else:
            blk = _kernel_block(S, args, tr.start[bt], tr.start[bt] + tr.size[bt], tr.start[t],
                                tr.start[t] + tr.size[t]).conj().T
        parts.append(blk / wc[b])
    return np.concatenate(parts, axis=1)


def oracle_leaf_sample(args, budget_s: float, seed: int = 0):
    """The FP64 oracle's complete leaf step -- numpy SVD of G^omega_tc, rank by the truncation rule,
    R = Q^* G^omega_tc -- timed on a seeded sample of the leaf pairs of BOTH bases of the workload, each
    leaf matrix formed (with the oracle's block weights) before its timer starts.  Returns the timed
    seconds, the sampled fraction of the leaf work (sum of m_t^2 #F_tc over both bases), the number of
    pairs and the wall time of the whole sample (generation included)."""
    S = _oracle_setup(args)
    O, tr, cp = S["O"], S["tr"], S["cp"]
    eps_l = [O.eps_hat(cp) * cp.zeta ** l for l in range(tr.depth + 1)]
    total_work = float(sum(S["work"].values()))
    order = np.random.default_rng(seed).permutation(len(S["leaf_pairs"]))
    w0 = time.perf_counter()
    done, t_used, cpu_used, npairs = 0.0, 0.0, 0.0, 0
    for idx in order:
        side, t, c, blocks = S["leaf_pairs"][idx]
        A = _leaf_matrix(S, args, side, t, blocks)
        t0, c0 = time.perf_counter(), time.process_time()
        Q, sig, k = O.leaf_pair_basis(A, eps_l[tr.level[t]])
        _ = Q.conj().T @ A
        t_used += time.perf_counter() - t0
        cpu_used += time.process_time() - c0
        done += S["work"][(side, t, c)]
        npairs += 1
        if t_used >= budget_s or time.perf_counter() - w0 >= 3.0 * budget_s:
            break
    # cores the timed work actually kept busy: process CPU time (all threads) over wall time
    return t_used, done / total_work, npairs, time.perf_counter() - w0, cpu_used / max(t_used, 1e-9)


_ANCHOR = {}


def oracle_full_anchor():
    """The whole oracle compression -- block weights, compress() of the row and of the column basis,
    project() -- timed end to end at n = 2048, kappa = 4, leaf 32, eps = 1e-4 on the Fibonacci sphere
    (the small configuration), G (complex128) and the tree built before the timer; plus the share of
    that time spent in leaf steps, measured by timing every leaf pair the same way as the sample."""
    if not _ANCHOR:
        from oracle import dh2_oracle as O
        from synth import fibonacci_sphere, helmholtz_matrix

        n, kappa = 2048, 4.0
        pts = fibonacci_sphere(n)
        tp = O.TreeParams(leaf_size=32, kappa=kappa)
        cp = O.CompressParams(eps=1e-4)
        tr = O.build_tree(pts, tp)
        G = helmholtz_matrix(pts, kappa)[np.ix_(tr.perm, tr.perm)]
        t0 = time.perf_counter()
        w = O.block_weights(tr, O.block_norms(tr, G), cp.zeta)
        t1 = time.perf_counter()
        V = O.compress(tr, G, cp, "row", w)
        t2 = time.perf_counter()
        W = O.compress(tr, G, cp, "col", w)
        t3 = time.perf_counter()
        O.project(tr, G, V, W)
        t4 = time.perf_counter()
        # the leaf steps alone, every leaf pair of both bases
        eps_l = [O.eps_hat(cp) * cp.zeta ** l for l in range(tr.depth + 1)]
        t_leaf = 0.0
        for side in ("row", "col"):
            F = O.column_sets(tr, side)
            for t in range(tr.nclusters()):
                if not tr.is_leaf(t):
                    continue
                for c, blocks in F[t].items():
                    A = np.concatenate([O._block_matrix(tr, G, side, b, t) / w[b] for b in blocks], axis=1)
                    a0 = time.perf_counter()
                    Q, sig, k = O.leaf_pair_basis(A, eps_l[tr.level[t]])
                    _ = Q.conj().T @ A
                    t_leaf += time.perf_counter() - a0
        total = t4 - t0
        _ANCHOR.update(n=n, kappa=kappa, leaf=32, weights_s=t1 - t0, row_s=t2 - t1, col_s=t3 - t2, project_s=t4 - t3,
                       total_s=total, gbs=16.0 * n * n / total / 1e9, leaf_step_s=t_leaf,
                       leaf_share=min(1.0, t_leaf / total))
    return dict(_ANCHOR)


def oracle_baseline(args, budget_s: float, seed: int = 0):
    """CPU baseline of the oracle on the workload: a measured leaf-step sample (oracle_leaf_sample),
    extrapolated to the whole compression by (1) the sampled share of the leaf work and (2) the share of
    the leaf steps in the whole oracle compression measured end to end at n = 2048 (oracle_full_anchor).
    Returns (estimated seconds of one whole compression, description dict, wall seconds of the sample)."""
    anchor = oracle_full_anchor()
    t_used, frac, npairs, wall, cores = oracle_leaf_sample(args, budget_s, seed)
    leaf_est = t_used / max(frac, 1e-300)
    est = leaf_est / anchor["leaf_share"]
    desc = {"timed": f"oracle leaf step (numpy SVD, truncation rule, R = Q^* A; complex128) on {npairs} seeded "
                     f"leaf pairs of both bases, {t_used:.2f} s of {wall:.1f} s wall (leaf matrices formed "
                     f"before each timer)",
            "sampled_leaf_work_fraction": frac,
            "extrapolated": True,
            "rule": "whole-compression seconds = timed seconds / sampled leaf-work fraction (work m_t^2 #F_tc) / "
                    "leaf-step share of the oracle's whole compression measured end to end at n=2048 "
                    f"({anchor['leaf_share']:.3f})",
            "anchor_n2048_end_to_end": anchor, "leaf_step_estimate_s": leaf_est, "whole_estimate_s": est,
            "effective_cores": cores}
    return est, desc, wall


# --------------------------------------------------------------------------- GPU arm

def _alg_flops(T, ranks):
    """Algorithmic flops of the leaf launches per basis pair (real flops, 8 per complex MAC):
    factor 4 m^2 N, R = Q^* A 8 k m N, summed with the computed ranks over both bases."""
    size = T.clusters()["size"].astype(np.float64)
    fac = rq = 0.0
    for sd in (0, 1):
        pr = T.pairs(sd)
        lf = pr["leaf"].astype(bool)
        m = size[pr["cluster"]][lf]
        N = pr["ncols"][lf].astype(np.float64)
        k = ranks[sd][lf].astype(np.float64)
        fac += float(np.sum(4.0 * m * m * N))
        rq += float(np.sum(8.0 * k * m * N))
    return fac, rq


def dist_init(world: int, backend: str | None = None) -> None:
    """Replicas under torchrun (one process per GPU, each compressing its own copy of the workload):
    a process group for the barriers around the timed regions and the maximum over ranks of their
    times; no collective on the data path (the problems are independent)."""
    import torch
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)


def _replicas() -> bool:
    import torch.distributed as dist

    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def barrier() -> None:
    """All ranks (a no-op on one process)."""
    if _replicas():
        import torch.distributed as dist

        dist.barrier()


def replica_max(ms: float) -> float:
    """The largest of the ranks' values (the timed region's milliseconds); the value itself on one
    process."""
    if not _replicas():
        return ms
    import torch
    import torch.distributed as dist

    on_gpu = dist.get_backend() == "nccl"
    t = torch.tensor([ms], dtype=torch.float64,
                     device=torch.device("cuda", torch.cuda.current_device()) if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_replica: float, world: int, ms: float) -> float:
    """Input GB/s of the whole job: every replica's bytes over the slowest replica's time."""
    return world * bytes_per_replica / (ms * 1e-3) / 1e9


def _timed_compress(D, T, G, mode, args, steps, warmup, clk=None, replicas=False):
    """Mean ms per dh2_compress over `steps` calls (CUDA events on the launching stream) and the
    per-phase and leaf-split means from the library's own events; returns the last matrix too.
    With `replicas` the timed region is bracketed by barriers of all ranks and the time is the
    largest over them."""
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        M = D.dh2_compress(T, G, eps=args.eps, mode=mode, nearfield=args.nearfield)
        del M
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phases = np.zeros(6)
    split = np.zeros(2)
    if clk is not None:
        clk.__enter__()
    try:
        torch.cuda.synchronize()
        if replicas:
            barrier()
        ev0.record(stream)
        for _ in range(steps):
            M = D.dh2_compress(T, G, eps=args.eps, mode=mode, nearfield=args.nearfield)
            phases += M.phase_ms()
            split += M.leaf_split_ms()
            del M
        ev1.record(stream)
        torch.cuda.synchronize()
        if replicas:
            barrier()
    finally:
        if clk is not None:
            clk.__exit__(None, None, None)
    ms = ev0.elapsed_time(ev1) / steps
    if replicas:
        ms = replica_max(ms)
    M = D.dh2_compress(T, G, eps=args.eps, mode=mode, nearfield=args.nearfield)
    return ms, phases / steps, split / steps, M


def _rank_hist(a, b):
    d = np.asarray(a, dtype=np.int64) - np.asarray(b, dtype=np.int64)
    vals, cnt = np.unique(d, return_counts=True)
    return {str(int(v)): int(c) for v, c in zip(vals, cnt)}


def run_gpu(args):
    import torch

    import paper_1510_07087_gb300 as D
    from synth import mean_nn_distance

    # one GPU per rank (replicas under torchrun); cuda:0 on one process
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    lead = int(os.environ.get("RANK", "0")) == 0
    pts, nrm = workload_points(args)
    h = mean_nn_distance(pts)
    T = D.dh2_tree_build(pts, args.leaf, args.kappa, args.eta1, args.eta2)
    perm = T.perm()
    st = T.stats()
    P = pts[perm]
    Nrm = nrm[perm] if nrm is not None else None
    cdt = torch.complex128 if args.mode == "fp64" else torch.complex64
    mode = MODE_CODE(D)[args.mode]
    Gd = workload_matrix(args, P, Nrm, h, cdt, dev)
    stream = torch.cuda.current_stream()
    elem = 16 if args.mode == "fp64" else 8
    in_bytes = elem * args.n * args.n

    # the library's autotuner picks its launch choices on this problem before anything is timed
    tuning = None
    if not args.no_autotune:
        table, log = D.autotune(T, Gd, eps=args.eps, mode=mode, nearfield=args.nearfield, reps=3)
        tuning = {"table": table, "candidates": log, "reps": 3,
                  "objective": "median device ms of the phase each knob acts on"}
    clk = ClockSampler(torch.cuda.current_device())
    ms, phases, split, M = _timed_compress(D, T, Gd, mode, args, args.steps, args.warmup, clk,
                                           replicas=world > 1)
    ranks = [M.ranks(0), M.ranks(1)]
    storage = M.storage()
    # matrix-vector product with the compressed matrix (Section 4), one right-hand side
    xv = torch.randn(args.n, dtype=cdt, device=dev)
    yv = torch.empty_like(xv)
    for _ in range(3):
        D.dh2_matvec(M, xv, yv)
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(10):
        D.dh2_matvec(M, xv, yv)
    m1.record(stream)
    torch.cuda.synchronize()
    matvec_ms = m0.elapsed_time(m1) / 10
    # error against the FP64 matrix (complex128, built the same way); with replicas on rank 0 only
    rel_err = None
    secondary = {}
    if args.mode != "fp64" and not args.skip_error and lead:
        G128 = workload_matrix(args, P, Nrm, h, torch.complex128, dev)
        rel_err = D.dh2_error(M, G128)
        if not args.skip_secondary:
            # the plain FP64 GPU form on the same problem (complex128 G), and the rank deviations of
            # this run's ranks from it (the FP64 form's ranks are the oracle's outside ties)
            ms64, ph64, _, M64 = _timed_compress(D, T, G128, D.MODE_FP64, args, 2, 1)
            r64 = [M64.ranks(0), M64.ranks(1)]
            secondary["fp64_form"] = {
                "ms_per_step": ms64, "value": 16 * args.n * args.n / (ms64 * 1e-3) / 1e9, "unit": "GB/s",
                "input": "complex128 G (16 B per entry)", "rel_err_vs_fp64": D.dh2_error(M64, G128),
                "phases_ms": [float(v) for v in ph64], "steps": 2, "warmup": 1,
                "speedup_of_headline": ms64 / ms}
            secondary["rank_deviation_vs_fp64_form"] = {
                "row": _rank_hist(ranks[0], r64[0]), "col": _rank_hist(ranks[1], r64[1])}
            del M64
            if args.mode == "mixed":
                ms32, _, _, M32 = _timed_compress(D, T, Gd, D.MODE_FP32, args, 2, 1)
                secondary["fp32_form"] = {"ms_per_step": ms32, "rel_err_vs_fp64": D.dh2_error(M32, G128)}
                secondary["rank_deviation_vs_fp32_form"] = {
                    "row": _rank_hist(ranks[0], M32.ranks(0)), "col": _rank_hist(ranks[1], M32.ranks(1))}
                del M32
        del G128
    elif not args.skip_error:
        rel_err = D.dh2_error(M, Gd)
    # end to end through the C ABI from pinned host memory, two ways, each with the ranks read back:
    # dh2_compress_host (the library copies G in column panels, overlapped with the column-basis
    # leaf work) and, for comparison, one H2D copy of G followed by dh2_compress
    e2e = None
    if not args.skip_e2e:
        Gh = torch.empty((args.n, args.n), dtype=cdt, pin_memory=True)
        Gh.copy_(Gd.t(), non_blocking=False)
        rk_h = [torch.empty(len(r), dtype=torch.int32, pin_memory=True) for r in ranks]
        d2h = sum(4 * len(r) for r in ranks)

        last_phases = {}

        def timed(step, tag):
            for it in range(args.warmup + args.steps):
                if it == args.warmup:
                    torch.cuda.synchronize()
                    if world > 1:
                        barrier()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                Me = step(it)
                for sd in (0, 1):
                    rk_h[sd].numpy()[:] = Me.ranks(sd)
                last_phases[tag] = [float(v) for v in Me.phase_ms()]
                del Me
            e1.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                barrier()
            return replica_max(e0.elapsed_time(e1) / args.steps) if world > 1 else e0.elapsed_time(e1) / args.steps

        seq = None
        if args.nearfield == 0:
            e2e_ms = timed(lambda it: D.dh2_compress_host(T, Gh.t(), eps=args.eps, mode=mode), "host")
        Gdev = torch.empty_like(Gh, device=dev)
        h2d_ev = []

        def copy_then_compress(it):
            if it >= args.warmup:
                eh = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                eh[0].record(stream)
            Gdev.copy_(Gh, non_blocking=True)
            if it >= args.warmup:
                eh[1].record(stream)
                h2d_ev.append(eh)
            return D.dh2_compress(T, Gdev.t(), eps=args.eps, mode=mode, nearfield=args.nearfield)

        seq_ms = timed(copy_then_compress, "seq")
        h2d_ms = sum(a.elapsed_time(b) for a, b in h2d_ev) / len(h2d_ev)
        seq = {"ms_per_step": seq_ms, "value": whole_job_gbs(in_bytes, world, seq_ms), "h2d_ms": h2d_ms,
               "h2d_gbs": in_bytes / (h2d_ms * 1e-3) / 1e9}
        if args.nearfield != 0:
            e2e_ms = seq_ms  # view mode: the host-input call copies into a buffer the matrix cannot keep
        e2e = {"value": whole_job_gbs(in_bytes, world, e2e_ms), "unit": "GB/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": d2h,
               "api": "dh2_compress_host" if args.nearfield == 0 else "H2D copy + dh2_compress",
               # host path phases: [panel copies with the leaf work overlapped, 0, 0, level steps,
               # expansion, projection]
               "phases_ms": last_phases.get("host"), "copy_then_compress": seq}
        del Gh, Gdev
    if not lead:
        return None  # replicas: the other ranks' part ends with the timed regions
    if not args.skip_secondary and args.kernel == "slp" and args.eta1 != 20.0:
        # the paper's parameter set (Section 7: eta1 = 20, eta2 = 5) on the same points: many coarse
        # admissible blocks, long column lists per pair
        del Gd
        Tp = D.dh2_tree_build(pts, args.leaf, args.kappa, 20.0, 5.0)
        Pp = pts[Tp.perm()]
        Gp = workload_matrix(args, Pp, None, h, cdt, dev)
        tuning_p = None
        headline_table = D.tuning()
        if not args.no_autotune:  # this problem's own launch choices (the level steps' segment width above all)
            tuning_p, _ = D.autotune(Tp, Gp, eps=args.eps, mode=mode, nearfield=args.nearfield, reps=1)
        msp, php, spp, Mp = _timed_compress(D, Tp, Gp, mode, args, 3, 2)
        D.set_tuning(headline_table)
        rp = [Mp.ranks(0), Mp.ranks(1)]
        errp = None
        if not args.skip_error:
            del Gp
            Gp128 = workload_matrix(args, Pp, None, h, torch.complex128, dev)
            errp = D.dh2_error(Mp, Gp128)
            del Gp128
        secondary["p_paper"] = {
            "eta1": 20.0, "eta2": 5.0, "ms_per_step": msp, "value": in_bytes / (msp * 1e-3) / 1e9, "unit": "GB/s",
            "adm_fraction": Tp.stats().adm_fraction, "rel_err_vs_fp64": errp,
            "k_max": int(max(rp[0].max(initial=0), rp[1].max(initial=0))),
            "phases_ms": [float(v) for v in php], "leaf_split_ms": [float(v) for v in spp], "steps": 3, "warmup": 2,
            "step_roofline_frac": in_bytes / (_peaks()[0]["hbm_gbs"] * 1e9) * 1e3 / msp, "tuning": tuning_p}
        del Mp
    peaks, src = _peaks()
    adm_bytes = elem * st.adm_fraction * args.n * args.n
    leaf_ms = float(phases[1])
    rq_ms = float(phases[2])
    fac_flops, rq_flops = _alg_flops(T, ranks)
    leaf_bytes = 2.0 * adm_bytes  # each basis reads every admissible entry once
    out_bytes = elem * (storage["V"] + storage["W"] + storage["E_V"] + storage["E_W"] + storage["S"])
    # the step roofline of the method: every entry of G read once, the representation written once;
    # the contractions at the measured dense bf16 tensor rate
    t_bytes = (in_bytes + out_bytes) / (peaks["hbm_gbs"] * 1e9) * 1e3
    t_flops = (fac_flops + rq_flops) / (peaks["bf16_tflops"] * 1e12) * 1e3
    t_roof_ms = max(t_bytes, t_flops)
    step_roof = {"bound": "hbm" if t_bytes >= t_flops else "tensor", "t_roof_ms": t_roof_ms, "frac": t_roof_ms / ms,
                 "achieved": (in_bytes + out_bytes) / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "peak_source": src, "alg_bytes": in_bytes + out_bytes, "t_hbm_ms": t_bytes,
                 "alg_flops": fac_flops + rq_flops, "t_tensor_ms": t_flops,
                 "note": "whole compression step: G read once plus V, W, E, S written once, at the measured copy "
                         "bandwidth; against max(that, leaf flops at the measured bf16 rate)"}
    mixed = args.mode == "mixed"
    gram_ms, fac_ms = float(split[0]), float(split[1])
    src_sha = _kernel_sha()
    if mixed:
        kern_ms = gram_ms
        roof = {"bound": "hbm", "kernel": "gram_kernel (leaf launches: tcgen05 bf16x3 sliced Gram of G^omega_tc, "
                                          "both bases)",
                "achieved": leaf_bytes / (kern_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": leaf_bytes / (kern_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "peak_source": src,
                "traffic": _traffic("gram", src_sha, args), "alg_bytes_per_launch": leaf_bytes,
                "launch_ms": kern_ms,
                "tensor_view": {"alg_flops": fac_flops, "achieved_tflops": fac_flops / (kern_ms * 1e-3) / 1e12,
                                "peak_tflops": peaks["bf16_tflops"],
                                "frac": fac_flops / (kern_ms * 1e-3) / 1e12 / peaks["bf16_tflops"],
                                "note": "4 m^2 N per pair; the bf16 slice products are not counted"},
                "factor_kernel": {"kernel": "pair_kernel<...,GRAM> (pivoted Cholesky, Jacobi, truncation, Q)",
                                  "ms": fac_ms}}
    else:
        kern_ms = leaf_ms
        roof = {"bound": "hbm", "kernel": "pair_kernel (leaf launches: LQ, pivoted truncation, Jacobi, Q)",
                "achieved": leaf_bytes / (kern_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": leaf_bytes / (kern_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "peak_source": src,
                "traffic": _traffic("pair", src_sha, args), "alg_bytes_per_launch": leaf_bytes,
                "launch_ms": kern_ms}
    roof["alu_view"] = {"alg_flops": fac_flops, "achieved_tflops": fac_flops / (leaf_ms * 1e-3) / 1e12,
                        "peak_tflops": FP32_ALU_TFLOPS, "frac": fac_flops / (leaf_ms * 1e-3) / 1e12 / FP32_ALU_TFLOPS,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz", "scope": "leaf phase"}
    roof["rq_kernel"] = {"ms": rq_ms, "alg_flops": rq_flops, "alg_bytes": leaf_bytes,
                         "achieved_gbs": leaf_bytes / (rq_ms * 1e-3) / 1e9,
                         "hbm_frac": leaf_bytes / (rq_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "achieved_tflops": rq_flops / (rq_ms * 1e-3) / 1e12}
    launches = M.launch_count()  # kernels the library launched for the last compression
    line = {
        "metric": "compression wall time & input GB/s at n=32768, kappa=32, eps=1e-4; rel. error vs FP64",
        "value": whole_job_gbs(in_bytes, world, ms), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "c64/f32 (f64 tail sums)", "fp64": "c128/f64",
                                       "mixed": "c64/bf16x3-tc/f32 (f64 tail sums)"}[args.mode],
        "data": "synthetic (Fibonacci sphere, Helmholtz collocation)", "config": workload(args),
        "rel_err_vs_fp64": rel_err, "step_roofline": step_roof, "roofline": roof,
        "phases_ms": {k: float(v) for k, v in zip(
            ["norms_nearfield", "leaf_factors", "leaf_R", "level_steps", "expansion", "projection"], phases)},
        "leaf_split_ms": {"gram": gram_ms, "factor": fac_ms} if mixed else None,
        "k_max": int(max(ranks[0].max(initial=0), ranks[1].max(initial=0))),
        "matvec_ms": matvec_ms,
        "mem_per_n_kib_c128": storage["total"] * 16 / 1024 / args.n,
        "adm_fraction": st.adm_fraction, "e2e": e2e, "secondary": secondary or None,
        "clocks": clk.summary(), "gpu_launches": launches * args.steps * world, "launches_per_step": launches,
        "tuning": tuning,
    }
    return line


def _storage_ratios(M, n, kappa, depth):
    """Stored entries against n k_max and n k_max + kappa^2 k_max^2 p (theorem on the complexity of
    DH^2 storage, Section 5: O(nk + kappa^2 k^2 log n)), with and without the nearfield."""
    st = M.storage()
    k_max = int(max(M.ranks(0).max(initial=0), M.ranks(1).max(initial=0)))
    far = st["total"] - st["near"]
    nk = max(1.0, float(n) * k_max)
    bound = nk + kappa * kappa * k_max * k_max * max(1, depth)
    return {"entries_total": st["total"], "entries_far": far, "entries_near": st["near"], "k_max": k_max,
            "total_over_nk": st["total"] / nk, "far_over_nk": far / nk, "total_over_bound": st["total"] / bound,
            "far_over_bound": far / bound, "mem_per_n_kib_c128": st["total"] * 16 / 1024 / n}


def sweep_cube(args):
    """The high-frequency sweep: unit-cube surface, uniform random points, n in {4096, 16384, 65536},
    kappa = 0.2 sqrt(n), eps in {1e-3, 1e-5}, leaf 64, both parameter sets.  n <= 16384: dense G in the
    mixed mode (complex64) and the FP64 mode (complex128); every n: matrix-free in FP32.  One JSON
    line per case."""
    import torch

    import paper_1510_07087_gb300 as D
    from synth import mean_nn_distance, random_cube_surface

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks, src = _peaks()
    for n in (4096, 16384, 65536):
        pts = random_cube_surface(n)
        h = mean_nn_distance(pts)
        kappa = 0.2 * math.sqrt(n)
        diag = 1.0 / (4.0 * math.pi * h)
        for eta1, eta2, pname in ((2.0 * math.sqrt(2.0), 1.0, "P-lit"), (20.0, 5.0, "P-paper")):
            T = D.dh2_tree_build(pts, 64, kappa, eta1, eta2)
            st = T.stats()
            P = pts[T.perm()]
            forms = []
            if n <= 16384:
                forms += [("mixed", D.MODE_MIXED_BF16X3, torch.complex64), ("fp64", D.MODE_FP64, torch.complex128)]
            forms.append(("fp32-matrix-free", D.MODE_FP32, None))
            G128 = None
            if n <= 16384:
                from synth.inputs import helmholtz_matrix_torch
                G128 = helmholtz_matrix_torch(P, kappa, h, torch.complex128, dev).t()
            for eps in (1e-3, 1e-5):
                for name, mode, cdt in forms:
                    sub = argparse.Namespace(**vars(args))
                    sub.eps, sub.n = eps, n
                    if cdt is not None:
                        G = G128 if cdt == torch.complex128 else G128.to(torch.complex64)
                        ms, ph, _, M = _timed_compress(D, T, G, mode, sub, 3, 2)
                        err = D.dh2_error(M, G128)
                        elem = 16 if cdt == torch.complex128 else 8
                    else:
                        def one():
                            return D.dh2_compress_kernel(T, pts, kappa, diag, eps=eps, mode=mode)
                        for _ in range(2):
                            del_ = one()
                            del del_
                        torch.cuda.synchronize()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(torch.cuda.current_stream())
                        for _ in range(3):
                            M = one()
                            ph = M.phase_ms()
                            del M
                        e1.record(torch.cuda.current_stream())
                        torch.cuda.synchronize()
                        ms = e0.elapsed_time(e1) / 3
                        M = one()
                        err = D.dh2_error(M, None)
                        elem = 8
                    line = {"sweep": "unit-cube high-frequency", "n": n, "kappa": kappa, "eps": eps, "params": pname,
                            "eta1": eta1, "eta2": eta2, "form": name, "ms_per_step": ms,
                            "input_gbs": elem * n * n / (ms * 1e-3) / 1e9 if cdt is not None else None,
                            "entries_per_s": n * n / (ms * 1e-3), "rel_err_vs_fp64": err,
                            "error_measure": "blockwise",
                            "adm_fraction": st.adm_fraction, "depth": st.depth,
                            "phases_ms": [float(v) for v in ph],
                            "storage": _storage_ratios(M, n, kappa, st.depth),
                            "step_roofline_frac": (elem * n * n / (peaks["hbm_gbs"] * 1e9) * 1e3 / ms
                                                   if cdt is not None else None)}
                    del M
                    print(json.dumps(line), flush=True)
            del G128


def sweep_small(args):
    """The two small configurations, median of 10 timed calls each after 3 warm-up calls:
    Fibonacci sphere n = 2048, kappa = 4, leaf 32, eps = 1e-4 in FP64 (complex128 G), and n = 8192,
    kappa = 16, leaf 32 at eps in {1e-4, 1e-6} in FP64, mixed and FP32, with the rank deviations of the
    reduced forms from the FP64 form.  One JSON line per case."""
    import torch

    import paper_1510_07087_gb300 as D
    from synth import fibonacci_sphere, mean_nn_distance
    from synth.inputs import helmholtz_matrix_torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    for n, kappa, eps_list, forms in ((2048, 4.0, (1e-4,), ("fp64",)),
                                      (8192, 16.0, (1e-4, 1e-6), ("fp64", "mixed", "fp32"))):
        pts = fibonacci_sphere(n)
        h = mean_nn_distance(pts)
        T = D.dh2_tree_build(pts, 32, kappa)
        st = T.stats()
        P = pts[T.perm()]
        G128 = helmholtz_matrix_torch(P, kappa, h, torch.complex128, dev).t()
        G64 = G128.to(torch.complex64)
        for eps in eps_list:
            r64 = None
            for form in forms:
                mode = MODE_CODE(D)[form]
                G = G128 if form == "fp64" else G64
                for _ in range(3):
                    M = D.dh2_compress(T, G, eps=eps, mode=mode)
                    del M
                times = []
                for _ in range(10):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    M = D.dh2_compress(T, G, eps=eps, mode=mode)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                    del M
                ms = statistics.median(times)
                M = D.dh2_compress(T, G, eps=eps, mode=mode)
                rk = [M.ranks(0), M.ranks(1)]
                if form == "fp64":
                    r64 = rk
                stg = M.storage()
                elem = 16 if form == "fp64" else 8
                line = {"sweep": "small configurations", "n": n, "kappa": kappa, "leaf": 32, "eps": eps,
                        "form": form, "ms_median_of_10": ms, "input_gbs": elem * n * n / (ms * 1e-3) / 1e9,
                        "rel_err_vs_fp64": D.dh2_error(M, G128), "adm_fraction": st.adm_fraction,
                        "k_max": int(max(rk[0].max(initial=0), rk[1].max(initial=0))),
                        "mem_per_n_kib_c128": stg["total"] * 16 / 1024 / n,
                        "rank_deviation_vs_fp64_form": (None if form == "fp64" or r64 is None else
                                                        {"row": _rank_hist(rk[0], r64[0]),
                                                         "col": _rank_hist(rk[1], r64[1])})}
                del M
                print(json.dumps(line), flush=True)
        del G128, G64


def _surface_problem(i):
    """Problem i of the 48-surface batch: 16 each of sphere, 2:1:1 ellipsoid and unit-cube surface,
    uniform random points with seed 151007087 + i, n ~ U{1024..12288}, kappa = U[8, 40] / diam."""
    from synth import random_cube_surface, random_ellipsoid, random_sphere

    seed = 151007087 + i
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1024, 12289))
    kind = ("sphere", "ellipsoid", "cube")[i // 16]
    diam = {"sphere": 2.0, "ellipsoid": 2.0, "cube": math.sqrt(3.0)}[kind]
    kappa = float(rng.uniform(8.0, 40.0)) / diam
    pts = {"sphere": random_sphere, "ellipsoid": random_ellipsoid, "cube": random_cube_surface}[kind](n, seed=seed)
    return kind, n, kappa, pts


def sweep_surfaces(args):
    """48 independent surfaces compressed by one dh2_compress_batched call (one launch per phase over
    all problems) against the same problems compressed one after the other; mixed mode, complex64."""
    import torch

    import paper_1510_07087_gb300 as D
    from synth import mean_nn_distance
    from synth.inputs import helmholtz_matrix_torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    trees, Gs, meta = [], [], []
    for i in range(48):
        kind, n, kappa, pts = _surface_problem(i)
        T = D.dh2_tree_build(pts, 64, kappa)
        h = mean_nn_distance(pts)
        G = helmholtz_matrix_torch(pts[T.perm()], kappa, h, torch.complex64, dev).t()
        trees.append(T)
        Gs.append(G)
        meta.append((kind, n, kappa, T.stats().adm_fraction))
    total_bytes = sum(8 * n * n for _, n, _, _ in meta)
    mode = D.MODE_MIXED_BF16X3
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            r = fn()
            del r
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            r = fn()
            del r
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    batched_ms = timed(lambda: D.dh2_compress_batched(trees, Gs, eps=args.eps, mode=mode), args.steps, args.warmup)
    seq_ms = timed(lambda: [D.dh2_compress(T, G, eps=args.eps, mode=mode) for T, G in zip(trees, Gs)],
                   max(1, args.steps // 2), 1)
    Ms = D.dh2_compress_batched(trees, Gs, eps=args.eps, mode=mode)
    errs = [D.dh2_error(M, G, which=D.ERR_FRO_CLOSED) for M, G in zip(Ms, Gs)]
    launches = Ms[0].launch_count()
    line = {"sweep": "48 surfaces, one batched call", "problems": 48, "mode": "mixed", "eps": args.eps,
            "bytes": total_bytes, "batched_ms": batched_ms, "batched_gbs": total_bytes / (batched_ms * 1e-3) / 1e9,
            "sequential_ms": seq_ms, "sequential_gbs": total_bytes / (seq_ms * 1e-3) / 1e9,
            "launches_batched": launches, "max_rel_err_closed_form_vs_c64": max(errs),
            "n_range": [min(m[1] for m in meta), max(m[1] for m in meta)],
            "adm_fraction_range": [min(m[3] for m in meta), max(m[3] for m in meta)],
            "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(line), flush=True)


def MODE_CODE(D):
    return {"fp32": D.MODE_FP32, "fp64": D.MODE_FP64, "mixed": D.MODE_MIXED_BF16X3}


def _kernel_sha():
    import hashlib

    h = hashlib.sha1()
    for f in ("dh2_gram.cu", "dh2_pair.cu"):
        h.update(open(os.path.join(ROOT, "paper_1510_07087_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _traffic(kernel, sha, args):
    """DRAM bytes (read + write) of the kernel's leaf launches from an ncu capture of this exact kernel
    source (KERNEL_TRAFFIC), scaled to the workload's admissible entries; None when the source has
    changed since the capture or the workload is another one."""
    rec = KERNEL_TRAFFIC.get((kernel, args.mode))
    if not rec or rec["sha1"] != sha or args.kernel != "slp" or args.leaf != 64 or args.kappa != 32.0:
        return None
    if args.eta1 != 2.0 * math.sqrt(2.0) or args.eta2 != 1.0 or args.n != 32768:
        return None
    return rec["bytes"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--kappa", type=float, default=32.0)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--eta1", type=float, default=2.0 * math.sqrt(2.0))
    ap.add_argument("--eta2", type=float, default=1.0)
    ap.add_argument("--mode", default="mixed", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--nearfield", type=int, default=0)
    ap.add_argument("--kernel", default="slp", choices=["slp", "dlp"],
                    help="slp: single-layer collocation on the Fibonacci sphere (the headline); "
                         "dlp: 1/2 I + double layer on a 2:1:1 ellipsoid")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch choices")
    ap.add_argument("--skip-error", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--sweep", default=None, choices=["small", "cube", "surfaces"],
                    help="instead of the headline: the small configurations, the unit-cube high-frequency sweep "
                         "or the 48-surface batch "
                         "(one JSON line per case)")
    ap.add_argument("--skip-secondary", action="store_true",
                    help="skip the FP64 / FP32 forms, the rank report and the eta1=20, eta2=5 run")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    elem = 16 if args.mode == "fp64" else 8
    in_bytes = elem * args.n * args.n
    if args.impl == "reference":
        if rank != 0:
            return
        vals, walls = [], []
        desc = {}
        # each step a bounded sample: the whole run stays within a few minutes for any K
        step_budget = max(0.5, min(args.cpu_budget, 90.0 / max(1, args.steps + args.warmup)))
        oracle_full_anchor()
        for _ in range(args.warmup):
            oracle_baseline(args, budget_s=step_budget, seed=1000 + _)
        for s_ in range(args.steps):
            est, desc, wall = oracle_baseline(args, budget_s=step_budget, seed=s_)
            vals.append(in_bytes / est / 1e9)
            walls.append(wall)
        v = statistics.median(vals)
        line = {"impl": "reference", "metric": "compression wall time & input GB/s at n=32768, kappa=32, "
                "eps=1e-4; rel. error vs FP64", "value": v, "unit": "GB/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                # the wall time of each bounded sample step; value is the extrapolated whole-compression rate
                "ms_per_step": 1e3 * statistics.mean(walls), "extrapolated": True,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128/f64",
                "data": "synthetic", "config": workload(args),
                "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": desc, "threads": "BLAS/OpenMP fixed to 1"},
                "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if args.sweep is not None:
        if rank == 0:
            {"small": sweep_small, "cube": sweep_cube, "surfaces": sweep_surfaces}[args.sweep](args)
        return
    dist_init(world)
    line = run_gpu(args)
    if line is None:
        return
    line["n_gpus"] = world
    if not args.skip_cpu and rank == 0:
        est, desc, _ = oracle_baseline(args, budget_s=args.cpu_budget)
        # cores: process CPU time over wall time of the timed oracle work (BLAS may use several threads)
        line["cpu_baseline"] = {"value": in_bytes / est / 1e9, "unit": "GB/s",
                                "cores": max(1, round(desc["effective_cores"], 1)), "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
