#!/usr/bin/env python
"""Throughput of the FFT Lippmann-Schwinger iteration on GB300 (voxel-iterations/s).

Workload (default): 512^3 periodised Boolean model of spheres (radius 8 voxels,
inclusion fraction 0.25, seed 1), matrix E = 1, nu = 0.3, inclusions E = 1000,
nu = 0.2, rotated-grid Green operator G^R with the accelerated scheme, FP32
bulk with FP64 reductions and FP64 refinement, stop at eta <= 1e-6.  One step
is one load case solved to tolerance; steps cycle through the six Mandel unit
loads of the full effective stiffness.  Inputs (3.2 GB of fields) are larger
than L2, so no flush is inserted between steps.

value    : total voxel-iterations of the timed steps / their device time
e2e      : the same metric through the public API with the phase image copied
           from pinned host memory and the result read back every step
roofline : the dominant kernel's algorithmic bytes per launch / its mean launch
           time (CUDA events on the solver stream) against the measured HBM peak
cpu_baseline: the FP64 CPU oracle on a bounded sample of the workload

--impl reference times the oracle itself (the reference arm of this repository).
Multi-GPU (torchrun): every rank solves its own load cases (replicas, no
collective on the data path); value = all ranks' voxel-iterations / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iters/s at 512^3 (AS, G^R, FP32 bulk + FP64 refinement, eta <= 1e-6)"
UNIT = "voxel-iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512, help="grid size per axis (512 = the workload)")
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--precision", default="fp32_refine64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the unfused cuFFT baseline")
    ap.add_argument("--cpu-n", type=int, default=128)
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 time-to-tolerance solve")
    ap.add_argument("--batched", type=int, default=0,
                    help="instead of the 512^3 workload, time COUNT batched Boolean samples of uneven sizes")
    ap.add_argument("--concurrency", type=int, default=8, help="worker streams of the batched solve")
    ap.add_argument("--batched-per-length", action="store_true",
                    help="with --batched: also time each grid length's samples alone (one worker) and one FP32 "
                         "iteration of a single sample per length")
    ap.add_argument("--warmstart", type=int, default=0,
                    help="instead of the 512^3 workload, train the warm-start network on COUNT solver-generated "
                         "64^3 samples and compare warm and plain starts on 256^3 samples")
    ap.add_argument("--warm-epochs", type=int, default=4)
    ap.add_argument("--warm-batch", type=int, default=1, help="samples per training step of the warm start")
    ap.add_argument("--warm-lr", type=float, default=5e-4, help="initial learning rate (decays 10x over training)")
    ap.add_argument("--warm-tc", action="store_true", help="train the warm start on the tensor cores")
    ap.add_argument("--warm-layers", type=int, default=0,
                    help="instead of the 512^3 workload, time each layer of the warm start's tensor-core inference "
                         "on an N^3 grid (random weights; CUDA events, best of 10)")
    ap.add_argument("--ncu-region", action="store_true",
                    help="for ncu --profile-from-start off: tune and warm up on the workload, then bracket two "
                         "FP32 iterations launched without graphs with the profiler start / stop calls")
    ap.add_argument("--warm-apply", type=int, default=4, help="256^3 samples of the warm-start comparison")
    ap.add_argument("--x1-sweep", action="store_true",
                    help="instead of the workload's timing, the forward x1 pass's time for every batch size and "
                         "load variant (imported schedules, the solver's profile mode)")
    ap.add_argument("--thin-grids", default="",
                    help="instead of the workload, per-kernel FP32 times on 512 x 512 x n3 grids for the listed n3 "
                         "(comma-separated), scaled to 512^3 voxels: does a pass speed up once its fields fit L2?")
    return ap.parse_args()


def workload(n):
    """Synthetic microstructure and phases of the benchmark (radius scales with n / 512)."""
    import numpy as np
    from paper_1412_8398_gb300 import microstructure as MS
    radius = 8.0 * n / 512.0
    ph, info = MS.boolean_spheres((n, n, n), radius, 0.25, seed=1)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)])
    return ph, lam, mu, info


def mandel_load(J):
    import numpy as np
    e = np.zeros(6)
    e[J] = 1.0 if J < 3 else 1.0 / math.sqrt(2.0)
    return e


def load_case(rank, i, world):
    """Mandel load index of step i on this rank: ranks interleave over the six loads."""
    return (rank + i * world) % 6


def replica_totals(ms, voxel_iters, world):
    """Whole-job figures of independent replicas: max time over ranks, summed work."""
    ms_max = allreduce([ms], _max_op(world), world)[0]
    vox_total = allreduce([float(voxel_iters)], _sum_op(world), world)[0]
    return ms_max, vox_total, vox_total / (ms_max / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, local, world


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(vals, op, world):
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return t.cpu().tolist()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# Algorithmic bytes per launch of each kernel (FP32 bulk; FP64 doubles the
# scalar size), for the path the workload takes (3D, G^R: eta from the
# real-space divergence stencil, so only tau is transformed).  Every field a
# pass must touch is counted once: eta_x reads eps (n_c scalars) and the phase
# (1 B) per voxel; fwd_x reads the same and writes n_c half-spectrum
# components; mid_y_fwd, fourier_z and mid_y_inv read and write n_c components;
# inv_x reads n_c components, eps and the phase and writes eps.  Halo re-reads
# are not counted.
def kernel_bytes(kind, n, nc=6):
    prec = 8 if kind.endswith("f64") else 4
    cplx = 2 * prec
    N = n ** 3
    half = n * n * (n // 2 + 1)
    k = kind.rsplit("_", 1)[0]
    if k == "eta_x":
        return N * (nc * prec + 1)
    if k == "fwd_x":
        return N * (nc * prec + 1) + nc * half * cplx
    if k in ("mid_y_fwd", "fourier_z", "mid_y_inv"):
        return 2 * nc * half * cplx
    if k == "inv_x":
        return nc * half * cplx + N * (2 * nc * prec + 1)
    return None


def source_hash():
    """Hash of the iteration's kernel sources (the FFT core and the kernel templates and their
    instantiation units): measured DRAM traffic stays valid while these are unchanged; host-side
    code (the solver driver, the warm-start network) does not change the bytes a pass moves."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1412_8398_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f == "fftls_fft.cuh" or f.startswith("fftls_kernels"):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kind, n):
    """dram bytes per launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = source_hash()
    for line in open(path):
        f = line.split()
        if len(f) == 5 and f[0] == "traffic" and f[1] == kind and int(f[2]) == n and f[4] == src:
            return float(f[3])
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_cores():
    """Cores this process may run on (sched_getaffinity where the platform has it)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample(n, index):
    """Sample `index` of the CPU baseline: an n^3 cut of the benchmark recipe that keeps its sphere
    radius (8 voxels), fraction (0.25) and phases; seed 1 + index, Mandel load index mod 6."""
    import numpy as np
    from paper_1412_8398_gb300 import microstructure as MS
    ph, info = MS.boolean_spheres((n, n, n), 8.0, 0.25, seed=1 + index)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)])
    return ph, lam, mu, mandel_load(index % 6)


def _oracle_worker(task):
    """One spawned worker: `iters` AS / G^R iterations of the oracle, as it stands, on sample `index`,
    continuing from eps_init when given.  Returns (index, voxels, iterations, seconds, strain)."""
    n, index, iters, eps_init = task
    import numpy as np
    from oracle import fftls_oracle as O
    ph, lam, mu, e = cpu_sample(n, index)
    eb = O.from_mandel(e, 3)
    t = time.perf_counter()
    r = O.solve(ph, lam, mu, eb, O.ROTATED, O.ACCELERATED, tol=0.0, max_iter=iters, eps_init=eps_init)
    dt = time.perf_counter() - t
    return index, int(ph.size), int(r["iterations"]), dt, r["strain"]


class OraclePool:
    """The CPU oracle on all host cores: one spawned single-threaded process per core (spawned, so
    that a parent holding a CUDA context forks nothing), each iterating its own sample."""

    def __init__(self, n, cores=None):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"  # inherited by the spawned workers: one thread each
        self.n = n
        self.cores = cores or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.state = [None] * self.cores

    def step(self, iters):
        """Every worker runs `iters` iterations of its sample (from its last iterate); returns the
        voxel-iterations done and the wall time of the whole group."""
        t = time.perf_counter()
        out = self.pool.map(_oracle_worker, [(self.n, i, iters, self.state[i]) for i in range(self.cores)])
        wall = time.perf_counter() - t
        vi = 0
        for index, vox, its, _, strain in out:
            self.state[index] = strain
            vi += vox * its
        return vi, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(n, iters):
    """The oracle (as it stands) on a bounded sample on every host core: aggregate voxel-iter/s."""
    try:
        pool = OraclePool(n)
        try:
            vi, wall = pool.step(iters)
        finally:
            pool.close()
    except Exception as e:  # the baseline is context, never a reason to lose the GPU line
        return {"error": repr(e)[:500]}
    return {"value": vi / wall, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{iters} AS/G^R iterations of the FP64 numpy oracle on each of {pool.cores} independent "
                      f"{n}^3 cuts of the recipe (sphere radius 8, fraction 0.25, chi 1000, seeds 1..{pool.cores}, "
                      f"Mandel loads cycled), one single-threaded process per host core, {wall:.1f} s wall"}


class CufftBaseline:
    """Unfused library baseline of one AS / G^R iteration in FP32: torch elementwise
    kernels for sigma = C(x):eps and tau = sigma - C0:eps, cuFFT (torch.fft) real-to-
    complex transforms of sigma (for eta) and tau, G' of G^R applied per mode on the
    half spectrum, the inverse transform and the accelerated update.  A timing baseline
    and a cross-check of the library's fused kernels, not part of the library."""

    IJ = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]

    def __init__(self, phase, lam, mu, lam0, mu0, eps_bar6):
        import numpy as np
        import torch
        self.t = torch
        dev = phase.device
        n3, n2, n1 = phase.shape
        self.N = n1 * n2 * n3
        lam_t = torch.tensor(np.asarray(lam, dtype=np.float32), device=dev)
        mu_t = torch.tensor(np.asarray(mu, dtype=np.float32), device=dev)
        ph = phase.long()
        self.lam, self.mu = lam_t[ph], mu_t[ph]
        kap = lam_t + 2.0 * mu_t / 3.0
        k0 = lam0 + 2.0 * mu0 / 3.0
        ak, am = (k0 / (kap + k0))[ph], (mu0 / (mu_t + mu0))[ph]
        self.am2, self.av = 2.0 * am, 2.0 * (ak - am) / 3.0
        self.lam0, self.mu0 = float(lam0), float(mu0)
        self.eb = torch.tensor(eps_bar6, dtype=torch.float32, device=dev)
        self.eps = self.eb.view(6, 1, 1, 1).expand(6, n3, n2, n1).contiguous()
        q = lambda n: 2.0 * np.pi * np.fft.fftfreq(n)
        q1 = 2.0 * np.pi * np.arange(n1 // 2 + 1) / n1
        s1, s2, s3 = np.sin(q1 / 2), np.sin(q(n2) / 2), np.sin(q(n3) / 2)
        c1, c2, c3 = np.cos(q1 / 2), np.cos(q(n2) / 2), np.cos(q(n3) / 2)
        # rotated-grid direction k^R / (phase * i): 2 sin(q_i/2) prod_{m != i} cos(q_m/2)
        k1 = 2 * s1[None, None, :] * c2[None, :, None] * c3[:, None, None]
        k2 = 2 * c1[None, None, :] * s2[None, :, None] * c3[:, None, None]
        k3 = 2 * c1[None, None, :] * c2[None, :, None] * s3[:, None, None]
        kr = np.stack([k1, k2, k3])
        kr[np.abs(kr) < 1e-12] = 0.0
        self.kr = torch.tensor(kr, dtype=torch.float32, device=dev)
        K2 = (self.kr ** 2).sum(0)
        self.zero = K2 == 0
        self.iK2 = torch.where(self.zero, torch.zeros_like(K2), 1.0 / torch.where(self.zero, torch.ones_like(K2), K2))
        w = np.full(n1 // 2 + 1, 2.0)
        w[0] = 1.0
        if n1 % 2 == 0:
            w[-1] = 1.0
        self.w = torch.tensor(w, dtype=torch.float32, device=dev)

    def stress(self, e):
        tr = e[0] + e[1] + e[2]
        s = 2.0 * self.mu * e
        s[:3] += self.lam * tr
        return s

    def step(self):
        """One iteration; returns eta of the current iterate (before the update)."""
        t = self.t
        e = self.eps
        sig = self.stress(e)
        tau = sig.clone()
        tr = e[0] + e[1] + e[2]
        tau -= 2.0 * self.mu0 * e
        tau[:3] -= self.lam0 * tr
        S = t.fft.rfftn(sig, dim=(1, 2, 3))
        T = t.fft.rfftn(tau, dim=(1, 2, 3))
        full = lambda X: [[X[[0, 5, 4][j] if i == 0 else ([5, 1, 3][j] if i == 1 else [4, 3, 2][j])]
                           for j in range(3)] for i in range(3)]
        Sm, Tm = full(S), full(T)
        div = [sum(self.kr[i] * Sm[i][j] for i in range(3)) for j in range(3)]
        num = sum((self.w * (d.real ** 2 + d.imag ** 2)).sum() for d in div)
        ms = sig.mean(dim=(1, 2, 3))
        den = float(t.sqrt((ms[:3] ** 2).sum() + 2.0 * (ms[3:] ** 2).sum())) * self.N
        eta = float(t.sqrt(num.double())) / den if den > 0 else 0.0
        V = [sum(self.kr[i] * Tm[i][j] for i in range(3)) for j in range(3)]
        Ssum = sum(self.kr[j] * V[j] for j in range(3))
        c0 = (self.lam0 + self.mu0) / (self.lam0 + 2.0 * self.mu0)
        f = -self.iK2 / self.mu0
        E = t.empty_like(T)
        for c, (i, j) in enumerate(self.IJ):
            E[c] = f * (0.5 * (self.kr[i] * V[j] + self.kr[j] * V[i]) - c0 * self.kr[i] * self.kr[j] * Ssum * self.iK2)
        E[:, self.zero] = 0
        E[:, 0, 0, 0] = self.eb * self.N
        en = t.fft.irfftn(E, s=e.shape[1:], dim=(1, 2, 3))
        d = en - e
        trd = d[0] + d[1] + d[2]
        upd = self.am2 * d
        upd[:3] += self.av * trd
        self.eps = e + upd
        return eta


def cufft_baseline(ph, lam, mu, iters, solver, warm=1):
    """Voxel-iterations / s of the unfused cuFFT pipeline (device-resident inputs), and
    its eta history over the first iterations against the library's FP32 path."""
    import numpy as np
    import torch
    from paper_1412_8398_gb300 import fftls
    l0, m0 = fftls.reference_medium(lam, mu, 3, "AS")
    dph = torch.from_numpy(ph).cuda()
    b = CufftBaseline(dph, lam, mu, l0, m0, [1.0, 0, 0, 0, 0, 0])
    etas = [b.step() for _ in range(3)]
    ours = solver.solve(dph, lam, mu, mandel_load(0), green="R", scheme="AS", tol=0.0, max_iter=3, precision="fp32",
                        want_strain=False, want_stress=False, device_outputs=True, raise_on_error=False)
    check = float(np.max(np.abs(np.array(etas) - ours.eta_history[:3]) / np.abs(ours.eta_history[:3])))
    for _ in range(warm):
        b.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        b.step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    out = {"value": ph.size / (ms / 1e3), "unit": UNIT, "ms_per_iteration": ms, "iterations_timed": iters,
           "what": "torch elementwise + cuFFT rfftn/irfftn (sigma and tau), FP32, AS / G^R, same workload",
           "crosscheck_eta_rel_diff_first_3_iterations": check}
    del b
    torch.cuda.empty_cache()
    return out


def bench_config(n, precision, fraction, world):
    """The `config` of the workload line (shared by both arms)."""
    return {"workload": f"boolean_spheres_{n}^3_R{8.0 * n / 512:g}_f0.25_chi1000_AS_R_{precision}_eta1e-6",
            "grid": [n, n, n], "realised_fraction": fraction, "load_cases": "Mandel unit loads, cycled",
            "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, as it stands, on every host core (rank 0 only), on the
    workload's config; each step is one oracle iteration of every core's cpu_n^3 sample (the recipe's
    sphere radius and fraction), continuing from the previous step's iterate."""
    if rank != 0:
        return
    config = bench_config(args.n, args.precision, workload(args.n)[3]["fraction"], world)
    pool = OraclePool(args.cpu_n)
    try:
        times, vis = [], []
        for i in range(args.warmup + args.steps):
            vi, wall = pool.step(1)
            if i >= args.warmup:
                times.append(wall)
                vis.append(vi)
    finally:
        pool.close()
    total = sum(times)
    value = sum(vis) / total
    sample = (f"one FP64 AS/G^R oracle iteration per step on each of {pool.cores} independent {args.cpu_n}^3 cuts of "
              f"the recipe (sphere radius 8, fraction 0.25), one single-threaded process per host core")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_batched(args, rank, local, world):
    """Batched workload: COUNT independent Boolean-sphere samples of uneven grid sizes
    ({32, 48, 64, 96, 128}^3, radius 3-8, fraction 0.1-0.4, contrast 10-1000, nu 0.3, eps_bar_11 = 1),
    AS with G^R to eta <= 1e-6.  Times the batched ladder (concurrent worker streams), the same
    ladder one sample at a time, and plain FP64 solves one at a time (the comparison of the
    metric).  Phase images are on the device before timing.  Ranks take every world-th sample."""
    import numpy as np
    import torch
    from paper_1412_8398_gb300 import build, fftls, microstructure as MS

    build.build()
    torch.cuda.set_device(local)
    specs = MS.batch_recipe(args.batched)[rank::world]
    samples = []
    for spec in specs:
        ph, lam, mu, info = MS.batch_sample(spec)
        samples.append({"phase": torch.from_numpy(ph).cuda(), "lam": lam, "mu": mu,
                        "eps_bar": np.diag([1.0, 0.0, 0.0])})
    vox = np.array([s["phase"].numel() for s in samples], dtype=np.float64)
    solver = fftls.Solver(local)
    kw = dict(green="R", scheme="AS", tol=1e-6, max_iter=args.max_iter)

    def timed(fn):
        torch.cuda.synchronize()
        barrier(world)
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        return out, dt

    # warm-up: tile schedules of every size and precision, worker buffers
    solver.solve_batched(samples, precision="fp32_refine64", concurrency=args.concurrency, **kw)
    k0, _ = solver.counters()
    (res, st), t_b = timed(lambda: solver.solve_batched(samples, precision="fp32_refine64",
                                                         concurrency=args.concurrency, **kw))
    k1, _ = solver.counters()
    (res1, _), t_s = timed(lambda: solver.solve_batched(samples, precision="fp32_refine64", concurrency=1, **kw))
    big = int(np.argmax(vox))
    solver.solve(samples[big]["phase"], samples[big]["lam"], samples[big]["mu"], samples[big]["eps_bar"],
                 precision="fp64", want_strain=False, want_stress=False, history=False, **dict(kw, max_iter=2),
                 raise_on_error=False)
    r64, t_64 = timed(lambda: [solver.solve(s["phase"], s["lam"], s["mu"], s["eps_bar"], precision="fp64",
                                            want_strain=False, want_stress=False, history=False, **kw)
                               for s in samples])
    per_length = None
    if args.batched_per_length:  # where the batch's time goes, one grid length at a time
        per_length = []
        for L in sorted({int(s["phase"].shape[0]) for s in samples}):
            grp = [s for s in samples if int(s["phase"].shape[0]) == L]
            solver.solve_batched(grp, precision="fp32_refine64", concurrency=1, **kw)
            (rg, _), tg = timed(lambda: solver.solve_batched(grp, precision="fp32_refine64", concurrency=1, **kw))
            s0 = grp[0]
            one = dict(kw, tol=0.0)
            solver.solve(s0["phase"], s0["lam"], s0["mu"], s0["eps_bar"], precision="fp32", want_strain=False,
                         want_stress=False, history=False, **dict(one, max_iter=5), raise_on_error=False)
            _, t1 = timed(lambda: solver.solve(s0["phase"], s0["lam"], s0["mu"], s0["eps_bar"], precision="fp32",
                                               want_strain=False, want_stress=False, history=False,
                                               **dict(one, max_iter=105), raise_on_error=False))
            # stragglers: the same samples as two groups split by contrast (similar iteration counts
            # within each), one after the other
            chi = [max(g["mu"]) / min(g["mu"]) for g in grp]
            order = sorted(range(len(grp)), key=lambda i: chi[i])
            t_split = 0.0
            for half in (order[:len(order) // 2], order[len(order) // 2:]):
                sub = [grp[i] for i in half]
                solver.solve_batched(sub, precision="fp32_refine64", concurrency=1, **kw)
                t_split += timed(lambda: solver.solve_batched(sub, precision="fp32_refine64", concurrency=1,
                                                              **kw))[1]
            its = [r.iterations for r in rg]
            per_length.append({"L": L, "samples": len(grp), "time_s": tg,
                               "voxel_iters_per_s": sum(L ** 3 * r.iterations for r in rg) / tg,
                               "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
                               "two_groups_by_contrast_s": t_split,
                               "single_fp32_ms_per_iteration": 1e3 * t1 / 105})
    its_b = np.array([r.iterations for r in res], dtype=np.float64)
    its_64 = np.array([r.iterations for r in r64], dtype=np.float64)
    rel = max(float(np.abs(a.mean_stress - b.mean_stress).max() / np.abs(b.mean_stress).max())
              for a, b in zip(res, r64))
    conv = sum(1 for r in res if r.converged)
    conv64 = sum(1 for r in r64 if r.converged)
    t_b_max = allreduce([t_b], _max_op(world), world)[0]
    t_s_max = allreduce([t_s], _max_op(world), world)[0]
    t_64_max = allreduce([t_64], _max_op(world), world)[0]
    vi_b = allreduce([float(np.dot(vox, its_b))], _sum_op(world), world)[0]
    vi_64 = allreduce([float(np.dot(vox, its_64))], _sum_op(world), world)[0]
    if rank == 0:
        out = {
            "metric": "time to eta <= 1e-6 over a batch of independent samples (AS, G^R)", "unit": "s",
            "value": t_b_max, "higher_is_better": False, "n_gpus": world, "impl": "ours",
            "data": "synthetic", "dtype": "f32+f64",
            "config": {"workload": f"batched_boolean_{args.batched}_samples_L32-128_R3-8_f0.1-0.4_chi10-1000",
                       "samples": args.batched, "voxels_total": int(allreduce([float(vox.sum())], _sum_op(world), world)[0]),
                       "concurrency": args.concurrency, "parallelism": "replicas" if world > 1 else "single GPU"},
            "batched_ladder": {"time_s": t_b_max, "voxel_iters_per_s": vi_b / t_b_max, "converged": conv,
                               "iterations_mean": float(its_b.mean()), "gpu_launches": k1 - k0},
            "sequential_ladder": {"time_s": t_s_max, "voxel_iters_per_s": vi_b / t_s_max},
            "fp64_sequential": {"time_s": t_64_max, "voxel_iters_per_s": vi_64 / t_64_max, "converged": conv64,
                                "iterations_mean": float(its_64.mean())},
            "speedup_vs_fp64": t_64_max / t_b_max,
            "max_rel_mean_stress_diff_vs_fp64": rel,
            "per_length": per_length,
            "tile_plans": solver.tile_plans(),
        }
        print(json.dumps(out))
    solver.close()


def run_warmstart(args, rank, local, world):
    """Learned warm start: train on COUNT solver-generated 64^3 Boolean samples (radius 3-8,
    fraction 0.1-0.4, contrast 10-1000, eps_bar_11 = 1, AS with G^R to eta <= 1e-6), then on
    --warm-apply 256^3 samples of the same recipe compare, each to eta <= 1e-6 with the same
    criterion: the ladder from eps_bar, the ladder from the network's eps^0 (inference timed in),
    and plain FP64 from eps_bar.  Rank 0 only (a single training run)."""
    import numpy as np
    import torch
    from paper_1412_8398_gb300 import build, fftls, microstructure as MS, warmstart as WS

    if rank != 0:
        return
    build.build()
    torch.cuda.set_device(local)
    solver = fftls.Solver(local)
    data, t_data = WS.make_dataset(solver, args.warmstart, 64, first_seed=20000, concurrency=args.concurrency)
    net = WS.WarmNet(device=local, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(data, epochs=args.warm_epochs, batch=args.warm_batch, lr=args.warm_lr,
                       lr_final=0.1 * args.warm_lr, tensor_cores=args.warm_tc)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del data
    specs = MS.batch_recipe(args.warm_apply, first_seed=30000, lengths=(256,))
    eb = np.diag([1.0, 0.0, 0.0])
    kw = dict(green="R", scheme="AS", tol=1e-6, max_iter=args.max_iter, want_strain=False, want_stress=False)
    rows = []
    first = True
    for spec in specs:
        ph, lam, mu, info = MS.batch_sample(spec)
        dph = torch.from_numpy(ph).cuda()
        if first:   # tile schedules and buffers of 256^3 outside the timed solves
            solver.solve(dph, lam, mu, eb, precision="fp32_refine64", **dict(kw, max_iter=3), raise_on_error=False)
            solver.solve(dph, lam, mu, eb, precision="fp64", **dict(kw, max_iter=3), raise_on_error=False)
            net.initial_strain(dph, spec["contrast"])
            first = False

        def timed(fn):
            torch.cuda.synchronize()
            t = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            return out, time.perf_counter() - t

        r0, t0_ = timed(lambda: solver.solve(dph, lam, mu, eb, precision="fp32_refine64", **kw))
        e0, t_inf = timed(lambda: net.initial_strain(dph, spec["contrast"]))
        r1, t1_ = timed(lambda: solver.solve(dph, lam, mu, eb, precision="fp32_refine64", eps_init=e0, **kw))
        r64, t64 = timed(lambda: solver.solve(dph, lam, mu, eb, precision="fp64", **kw))
        rows.append({"contrast": spec["contrast"], "fraction": info["fraction"], "radius": spec["radius"],
                     "zero": {"iterations": r0.iterations, "time_s": t0_, "converged": r0.converged},
                     "warm": {"iterations": r1.iterations, "time_s": t1_ + t_inf, "inference_s": t_inf,
                              "converged": r1.converged},
                     "fp64": {"iterations": r64.iterations, "time_s": t64, "converged": r64.converged},
                     "warm_vs_zero_rel_mean_stress": float(np.abs(r1.mean_stress - r0.mean_stress).max()
                                                           / np.abs(r0.mean_stress).max())})
        del e0, dph
    tot = lambda k, f: float(sum(r[k][f] for r in rows))
    out = {
        "metric": "time to eta <= 1e-6 with the learned warm start (AS, G^R, 256^3)", "unit": "s",
        "value": tot("warm", "time_s") / len(rows), "higher_is_better": False, "n_gpus": 1, "impl": "ours",
        "data": "synthetic", "dtype": "f32+f64 solve, bf16 inference",
        "config": {"workload": f"warmstart_train_{args.warmstart}x64^3_apply_{args.warm_apply}x256^3_boolean",
                   "train_samples": args.warmstart, "epochs": args.warm_epochs, "batch": args.warm_batch,
                   "lr": args.warm_lr, "training": "tensor cores (BF16)" if args.warm_tc else "FP32",
                   "parameters": WS.parameter_count()},
        "data_seconds": t_data, "train_seconds": t_train, "train_loss_per_epoch": losses,
        "iterations": {"zero_init": tot("zero", "iterations"), "warm": tot("warm", "iterations"),
                       "fp64_zero_init": tot("fp64", "iterations")},
        "time_s": {"zero_init_ladder": tot("zero", "time_s"), "warm_ladder_incl_inference": tot("warm", "time_s"),
                   "fp64_zero_init": tot("fp64", "time_s")},
        "samples": rows,
    }
    print(json.dumps(out))
    solver.close()


def run_x1_sweep(args, rank, local):
    """The forward x1 pass (k_fwd_x) on the workload (--n) for lines per batch 1..8 and the load variants
    (voxels per thread loaded together 1, 2, 4; 0 = the batch staged in shared memory by bulk copies),
    the other passes on the tuned schedule: CUDA-event ms per launch over 8 FP32 iterations (the
    solver's profile mode), best of two rounds.  Rank 0 only."""
    import numpy as np
    import torch
    from paper_1412_8398_gb300 import build, fftls

    if rank != 0:
        return
    build.build()
    torch.cuda.set_device(local)
    ph, lam, mu, _ = workload(args.n)
    dph = torch.from_numpy(ph).cuda()
    eb = np.diag([1.0, 0.0, 0.0])
    s = fftls.Solver(local)
    res = {}
    try:
        s.solve(dph, lam, mu, eb, "R", "AS", tol=0.0, max_iter=3, precision="fp32", want_strain=False,
                want_stress=False)
        base = [p for p in s.tile_plans() if p["precision"] == 0][0]
        for _ in range(2):
            for lines in range(1, 9):
                for vb in (1, 2, 4, 0):
                    try:
                        s.set_tile_plans([dict(base, x1_lines=lines, x1_vb=vb)])
                        s.solve(dph, lam, mu, eb, "R", "AS", tol=0.0, max_iter=8, precision="fp32",
                                want_strain=False, want_stress=False, profile=True)
                    except fftls.FftlsError:
                        continue  # does not fit shared memory
                    v = [t for k, t in s.profile().items() if k.startswith("fwd_x")][0]
                    key = f"{lines},{vb}"
                    res[key] = min(res.get(key, float("inf")), v[0] / v[1])
    finally:
        s.close()
    print(json.dumps({"metric": f"k_fwd_x ms per launch at {args.n}^3 FP32 by (lines per batch, voxels per load; "
                                "0 = staged by bulk copies)", "tuned": {k: base[k] for k in ("x1_lines", "x1_vb")},
                      "ms": res}), flush=True)


def run_thin_grids(args, rank, local):
    """Per-kernel CUDA-event times (the solver's profile mode: no graphs, events around every launch) of
    20 FP32 iterations of the workload's recipe on 512 x 512 x n3 grids, tuned schedules, each scaled to
    512^3 voxels.  The half spectrum takes 6.3 MB per x3-plane, so at n3 <= 16 every pass's fields fit
    the 129 MB L2: a pass bound by DRAM bandwidth would run faster per voxel there.  Rank 0 only."""
    import numpy as np
    import torch
    from paper_1412_8398_gb300 import build, fftls, microstructure as MS

    if rank != 0:
        return
    build.build()
    torch.cuda.set_device(local)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)])
    eb = np.diag([1.0, 0.0, 0.0])
    out = {"metric": "FP32 ms per launch scaled to 512^3 voxels, 512 x 512 x n3 grids", "unit": "ms", "rows": []}
    for n3 in [int(v) for v in args.thin_grids.split(",") if v]:
        ph, _ = MS.boolean_spheres((512, 512, n3), 8.0, 0.25, seed=1)
        dph = torch.from_numpy(ph).cuda()
        s = fftls.Solver(local)
        try:
            s.solve(dph, lam, mu, eb, "R", "AS", tol=0.0, max_iter=3, precision="fp32", want_strain=False,
                    want_stress=False)
            s.solve(dph, lam, mu, eb, "R", "AS", tol=0.0, max_iter=20, precision="fp32", want_strain=False,
                    want_stress=False, profile=True)
            prof = s.profile()
            plan = [p for p in s.tile_plans() if p["precision"] == 0][0]
        finally:
            s.close()
        scale = 512.0 ** 3 / (512 * 512 * n3)
        out["rows"].append({"n3": n3, "spectrum_mb": 512 * 512 * n3 * 6 * 8 * 257 / 256 / 2 / 1e6,
                            "ms_scaled": {k: v[0] / v[1] * scale for k, v in prof.items()},
                            "plan": {k: plan[k] for k in ("x1_lines", "x1_vb", "x5_lines", "y_w", "z_w", "e_planes")}})
    print(json.dumps(out), flush=True)


def run_warm_layers(args, rank, local, world):
    """Per-layer CUDA-event times of the warm start's tensor-core inference on an N^3 Boolean sample
    (random weights: the times do not depend on the values), the whole forward, the initial strain,
    and the FP32 forward for comparison.  Rank 0 only."""
    import ctypes
    import torch
    from paper_1412_8398_gb300 import build, microstructure as MS, warmstart as WS

    if rank != 0:
        return
    build.build()
    torch.cuda.set_device(local)
    L = args.warm_layers
    net = WS.WarmNet(device=local, seed=0)
    ph, _ = MS.boolean_spheres((L, L, L), 5.0, 0.2, seed=1)
    dph = torch.from_numpy(ph).cuda()
    n = (L, L, L)

    def ms(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    out = {"metric": "warm-start tensor-core inference, per layer", "unit": "ms", "grid": L, "layers": []}
    out["forward_tc_ms"] = ms(lambda: net.forward_tc(dph, 100.0))
    lib, t = net.lib, net.tc
    packed = net._tc_weights()
    layer = {l[0]: l for l in WS.LAYERS}
    _p = WS._p
    t_enc0 = ms(lambda: lib.fftls_nn_tc_conv_phase(_p(dph), net._w("enc0"), net._b("enc0"), _p(t["e0"]),
                                                   WS._I3(*n), 8, 0.0, 1, None))
    out["layers"].append({"layer": "enc0", "ms": t_enc0, "flop": 2.0 * L ** 3 * 27 * 2 * 8})
    cs = WS._stored
    for name, src, mode, skip in WS._TC_PLAN + [("out", "d0", 0, None)]:
        _, ci, co, k, lvl = layer[name]
        dst, planar, relu = (t["y"], 1, 0) if name == "out" else (t[WS._TC_OUT[name]], 0, 1)
        f = (lambda name=name, src=src, mode=mode, skip=skip, ci=ci, co=co, k=k, lvl=lvl, dst=dst, planar=planar,
             relu=relu: lib.fftls_nn_tc_conv3d(_p(t[src]), _p(packed[name]), net._b(name),
                                               _p(t[skip]) if skip else None, _p(dst), 1, ci, co,
                                               net._dims(n, lvl), k, mode, relu, planar, 0, None))
        vox = (L >> lvl) ** 3
        tl = ms(f)
        out["layers"].append({"layer": name, "ms": tl, "flop": 2.0 * vox * k ** 3 * cs(ci) * cs(co),
                              "tflops_padded": 2.0 * vox * k ** 3 * cs(ci) * cs(co) / tl / 1e9})
    y = net.forward_tc(dph, 100.0)
    eps = torch.empty((6, L, L, L), dtype=torch.float64, device="cuda")
    eb = (ctypes.c_double * 6)(1.0, 0, 0, 0, 0, 0)
    out["strain_init_ms"] = ms(lambda: lib.fftls_nn_strain_init(_p(y), _p(eps), WS._I3(*n), eb, 1.0,
                                                                _p(net.tc_mean_scratch), None))
    net._buffers(n, False)
    out["forward_fp32_ms"] = ms(lambda: (net.features(dph, 100.0), net.forward()))
    print(json.dumps(out))


def run_ncu_region(args, local):
    """A profiler region of two steady-state FP32 iterations of the workload (size --n)."""
    import torch
    from paper_1412_8398_gb300 import build, fftls

    build.build()
    torch.cuda.set_device(local)
    ph, lam, mu, info = workload(args.n)
    dph = torch.from_numpy(ph).cuda()
    s = fftls.Solver(local)
    kw = dict(green="R", scheme="AS", tol=1e-6, precision="fp32", want_strain=False, want_stress=False,
              history=False, device_outputs=True, raise_on_error=False)
    s.solve(dph, lam, mu, mandel_load(0), max_iter=3, **kw)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    s.solve(dph, lam, mu, mandel_load(0), max_iter=2, use_graphs=False, **kw)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_region": "2 FP32 iterations", "n": args.n, "tile_plans": s.tile_plans()}))
    s.close()


def main():
    args = parse()
    rank, local, world = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.batched > 0:
        run_batched(args, rank, local, world)
        return
    if args.warm_layers > 0:
        run_warm_layers(args, rank, local, world)
        return
    if args.thin_grids:
        run_thin_grids(args, rank, local)
        return
    if args.x1_sweep:
        run_x1_sweep(args, rank, local)
        return
    if args.warmstart > 0:
        run_warmstart(args, rank, local, world)
        return
    if args.ncu_region:
        run_ncu_region(args, local)
        return
    import numpy as np
    import torch
    from paper_1412_8398_gb300 import build, fftls

    build.build()
    torch.cuda.set_device(local)
    n = args.n
    ph, lam, mu, info = workload(n)
    N = ph.size
    dph = torch.from_numpy(ph).cuda()
    solver = fftls.Solver(local)
    stream = torch.cuda.Stream(device=local)
    kw = dict(green="R", scheme="AS", tol=1e-6, max_iter=args.max_iter, precision=args.precision,
              want_strain=False, want_stress=False, history=False, device_outputs=True, stream=stream)

    def step(i, **extra):
        J = load_case(rank, i, world)
        opts = dict(kw)
        opts.update(extra)
        r = solver.solve(dph, lam, mu, mandel_load(J), **opts)
        if r.status not in (fftls.OK,):
            raise RuntimeError(f"solve failed: {r.message}")
        return r

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    clk = ClockSampler(local)
    clk.start()
    k0, _ = solver.counters()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    iters = its32 = 0
    for i in range(args.steps):
        r = step(args.warmup + i)
        iters += r.iterations
        its32 += r.iterations_fp32
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    k1, _ = solver.counters()
    ms = ev0.elapsed_time(ev1)
    ms_max, vox_total, value = replica_totals(ms, float(N) * iters, world)

    # roofline: the same steps again with per-kernel CUDA events
    prof = {}
    for i in range(min(args.steps, 2)):
        step(args.warmup + i, profile=True, use_graphs=False)
        for kname, (kms, cnt) in solver.profile().items():
            a, b = prof.get(kname, (0.0, 0))
            prof[kname] = (a + kms, b + cnt)
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dname, (dms, dcnt) = dom
    peak, peak_kind = peaks()
    algo = kernel_bytes(dname, n)
    achieved = algo / (dms / dcnt / 1e3) / 1e9 if algo else None
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": measured_traffic(dname, n),
                "bytes_per_launch": algo, "launch_ms": dms / dcnt, "peak_source": f"hbm_gbs ({peak_kind})",
                "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                                "gbs": (kernel_bytes(k, n) / (v[0] / v[1] / 1e3) / 1e9) if kernel_bytes(k, n) else None}
                            for k, v in sorted(prof.items())}}

    # the unfused library pipeline (cuFFT + elementwise kernels) on the same workload
    cufft = None
    if not args.no_cufft and rank == 0:
        cufft = cufft_baseline(ph, lam, mu, 3, solver)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(ph.shape, dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[...] = ph
        hph = pinned.numpy()
        torch.cuda.synchronize()
        t = time.perf_counter()
        e_iters = 0
        for i in range(args.steps):
            J = load_case(rank, i, world)
            r = solver.solve(hph, lam, mu, mandel_load(J), green="R", scheme="AS", tol=1e-6,
                             max_iter=args.max_iter, precision=args.precision, want_strain=False,
                             want_stress=False, history=False, device_outputs=False)
            e_iters += r.iterations
        dt = time.perf_counter() - t
        _, _, e_value = replica_totals(dt * 1e3, float(N) * e_iters, world)
        e2e = {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": int(N),
               "d2h_bytes_per_step": 2 * 6 * 8,
               "outputs": "per load case the mean stress and mean strain (one column of the effective stiffness); "
                          "the strain and stress fields stay on the device"}

    # the metric's comparison: one load case solved with plain FP64 iterations, same tolerance
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        J = load_case(rank, 0, world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r64 = solver.solve(dph, lam, mu, mandel_load(J), **dict(kw, precision="fp64"))
        e1.record(stream)
        torch.cuda.synchronize()
        rl = solver.solve(dph, lam, mu, mandel_load(J), **kw)
        rel = float(np.abs(rl.mean_stress - r64.mean_stress).max() / np.abs(r64.mean_stress).max())
        fp64 = {"load": int(J), "fp64_time_to_tol_s": e0.elapsed_time(e1) / 1e3,
                "fp64_iterations": int(r64.iterations), "fp64_converged": bool(r64.converged),
                "fp64_voxel_iters_per_s": float(N) * r64.iterations / (e0.elapsed_time(e1) / 1e3),
                "ladder_vs_fp64_mean_stress_rel": rel}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_n, args.cpu_iters)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32_refine64" else args.precision,
            "data": "synthetic",
            "config": bench_config(n, args.precision, info["fraction"], world),
            "iterations_per_step": iters / args.steps, "fp32_iterations_per_step": its32 / args.steps,
            "time_to_tol_s": ms_max / 1e3 / args.steps,
            "vs_fp64": fp64,
            "gpu_launches": k1 - k0,
            "tile_plans": solver.tile_plans(),
            "clocks": clocks,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "cufft_baseline": cufft,
        }
        print(json.dumps(out))
    solver.close()


def _max_op(world):
    if world == 1:
        return None
    import torch.distributed as dist
    return dist.ReduceOp.MAX


def _sum_op(world):
    if world == 1:
        return None
    import torch.distributed as dist
    return dist.ReduceOp.SUM


if __name__ == "__main__":
    main()
