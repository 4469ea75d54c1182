#!/usr/bin/env python3
"""Benchmark of the NSF eigensolver hot path on one GB300 (or N, weak scaling).

A step is one complete eigensolve of the headline workload: 96^3 pseudochiral
cylinders, the 20 smallest positive eigenvalues by thick-restart invert
Lanczos on the HHPD-NFGEP with complex64 CG inside FP64 refinement and FP64
orthogonalisation (every row of the hot path: tables, assembly, twisted FFTs,
material product, projections, B_r, CG, Lanczos).  The printed `value` is
eigenpairs per second over all ranks.  Alongside: A_r matvecs/s in complex64
and complex128, CG iterations/s, the FP64 eigensolve for comparison, the
roofline of the dominant matvec pass, an end-to-end figure through the public
API with host inputs, and the CPU oracle's rate on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank solves its own k-point (independent problems; no
collective on the data path): weak scaling.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NFGEP matvecs/s & eigenpairs/s at 96^3, mixed vs FP64, % HBM roofline"
UNIT = "eigenpairs/s"
WORKLOAD = "pseudo96"
CONFIG = {"workload": "pseudo96: 96^3 pseudochiral (x-y) cylinders eps 13 r 0.1, gamma 0.4, k.a=(0.1,0.2,0.3)"
                      "+0.01*rank, nev 20",
          "l2": "eigensolve working set > L2; matvec timings flush L2",
          "grid": [96, 96, 96], "nev": 20}
NEV = 20
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden_values(name):
    """The oracle's stored eigenvalues of a workload and the A_r products and
    seconds its tier-O3 solve took (from the file header), or None."""
    path = os.path.join(GOLDEN, f"{name}_omega.txt")
    if not os.path.exists(path):
        return None
    vals, products, seconds = [], None, None
    for line in open(path):
        if line.startswith("#"):
            m = re.search(r"(\d+) A_r products, (\d+) s", line)
            if m:
                products, seconds = int(m.group(1)), float(m.group(2))
        elif line.strip():
            vals.append(float(line))
    return {"omega": vals, "products": products, "seconds": seconds}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--skip-fp64", action="store_true")
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--skip-e2e", action="store_true")
    p.add_argument("--skip-batch", action="store_true", help="skip the batched band-structure (bz48) leg")
    p.add_argument("--skip-grad", action="store_true", help="skip the eigenvalue-gradient (field64) leg")
    p.add_argument("--skip-bands", action="store_true", help="skip the band-structure (bands48) leg")
    p.add_argument("--skip-mesh", action="store_true", help="skip the mesh-convergence (8^3 .. 128^3) leg")
    p.add_argument("--skip-nfsep", action="store_true",
                   help="skip the leg for media outside the Assumption (NFSEP at 8^3, shift-and-invert Arnoldi)")
    p.add_argument("--skip-fields", action="store_true",
                   help="skip the eigenvector-fields leg (E, H of the headline eigenpairs and their GEP residuals)")
    p.add_argument("--cufft", action="store_true",
                   help="with --matvec-only: also time cuFFT (torch.fft) on the product's twelve transforms")
    p.add_argument("--skip-paper-ncv", action="store_true",
                   help="skip the headline solve with the paper's basis size ncv = 3 nev")
    p.add_argument("--skip-sphere64", action="store_true", help="skip the 64^3 FP64 sphere leg (config 2)")
    p.add_argument("--matvec-only", action="store_true",
                   help="time only the A_r products (profiling aid; prints a reduced line)")
    p.add_argument("--profile-grid", type=int, default=0,
                   help="profiling aid: only mixed eigensolves (nev 10) of the headline medium on an "
                        "N^3 grid, a few GB on the device; prints a reduced line")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(backend):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_kpoint(base, rank):
    # a distinct Bloch vector per rank (same grid and medium): independent problems
    return tuple(float(v) + 0.01 * rank for v in base)


KERNEL_SOURCES = ("matvec.h", "matvec_impl.cuh", "matvec_kernels.cuh", "matvec_pk.cuh", "fft_pk.cuh",
                  "fft_smem.cuh", "fft_reg.cuh", "nfs_complex.cuh", "cg_state.cuh", "tuning.h")
PASS_COUNTERS = os.path.join(ROOT, "profiles", "pseudo96_matvec_c64_counters.json")
PASS_KERNELS = ("k_pk_pass1", "k_pk_pass2", "k_pass3_fft_xy_project")


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        path = os.path.join(ROOT, "paper_1402_6297_gb300", "csrc", f)
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(pass_index):
    """DRAM bytes per launch of a pass from the committed ncu counters
    (profiles/pseudo96_matvec_c64_counters.json), or None when the kernel
    sources have changed since the counters were taken."""
    try:
        with open(PASS_COUNTERS) as f:
            d = json.load(f)
        if d.get("kernel_sources_sha256_16") != kernel_sources_hash():
            return None
        v = d["dram_bytes_per_launch"].get(PASS_KERNELS[pass_index])
        return int(v) if v is not None else None
    except (OSError, ValueError, KeyError):
        return None


def cg_iteration_roofline(n, product_bytes, info, hbm):
    vec = 4 * n * 8
    b = product_bytes + 2 * vec + 6 * vec
    us = 1e6 * info.seconds_cg / max(int(info.cg_iterations), 1)
    gbps = b / (us * 1e-6) / 1e9
    return {"bytes": b, "us": us, "GBps": gbps, "frac": gbps / hbm}


def bytes_per_pass(n, csize, kind):
    """Algorithmic HBM bytes of each pass of one A_r product (3-pass model):
    pass 1 reads u (4n) and writes six fields (6n); pass 2 reads and writes the
    six fields and reads the material (1/Phi per component and gamma); pass 3
    reads six fields and writes A_r u (4n)."""
    rsize = csize // 2
    mat_reals = 6 if kind == "chiral" else 4
    return [10 * n * csize, 12 * n * csize + mat_reals * n * rsize, 10 * n * csize]


# ---------------------------------------------------------------------------
# oracle (CPU) timing: the reference arm and the cpu_baseline field
# ---------------------------------------------------------------------------

def oracle_matvec_rate(w, seconds, max_calls=50, orc=None):
    import numpy as np

    import workloads as wl
    from oracle import nfgep
    if orc is None:
        orc = nfgep.NFGEP(w["grid"], w["kdota"], w["medium"])
    u = wl.random_complex(4 * orc.n, 3)
    orc.Ar(u)  # warm the FFT plans
    t0 = time.perf_counter()
    calls = 0
    while calls < max_calls:
        orc.Ar(u)
        calls += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    _ = np
    return calls / dt, calls, dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_products_per_solve():
    """A_r products of the oracle's own nev = 20 eigensolve of pseudo96 (from
    the stored tier-O3 solve), else of the 64^3 sphere's, else None."""
    for name in ("pseudo96", "sphere64"):
        gv = golden_values(name)
        if gv and gv["products"]:
            return gv["products"], name
    return None, None


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_eigensolve_sphere8():
    """A whole timed oracle eigensolve (tier O3: FFT NFGEP, ARPACK with CG at
    1e-13) of sphere8, nev 10, on the host cores."""
    import workloads as wl
    from oracle import nfgep
    w = wl.workload("sphere8")
    O = nfgep.NFGEP(w["grid"], w["kdota"], w["medium"])
    t0 = time.perf_counter()
    om, _ = O.eigs(w["nev"], tol=1e-12, cg_tol=1e-13)
    dt = time.perf_counter() - t0
    return {"workload": "sphere8, nev 10, tier O3 (FFT NFGEP, ARPACK invert Lanczos, CG 1e-13)",
            "seconds": dt, "eigenpairs_per_s": w["nev"] / dt, "products": O.nmatvec}


def run_reference(args):
    """The oracle as it stands on the host cores.  A whole oracle eigensolve of
    pseudo96 takes hours, so each step is a bounded sample of the workload
    (oracle FFT A_r products at 96^3), and `value` is a PROJECTION: the
    product rate times nev over the products of the oracle's own eigensolve
    (its stored tier-O3 solve).  `ms_per_step` is the time a step actually
    took.  A whole timed oracle eigensolve of the 8^3 workload rides along."""
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return 0
    import workloads as wl
    from oracle import nfgep
    w = wl.workload(WORKLOAD)
    orc = nfgep.NFGEP(w["grid"], w["kdota"], w["medium"])  # set-up outside the timed steps
    per, step_s = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, calls, dt = oracle_matvec_rate(w, seconds=max(2.0, args.cpu_seconds / max(args.steps, 1)), max_calls=4,
                                             orc=orc)
        if i >= args.warmup:
            per.append((rate, calls, dt))
            step_s.append(time.perf_counter() - t0)
    rate = sum(c for _, c, _ in per) / sum(d for _, _, d in per)
    products, src = oracle_products_per_solve()
    if products is None:
        products, src = 10533, "sphere64 (default)"
    value = rate * NEV / products
    sample = (f"PROJECTION: {sum(c for _, c, _ in per)} oracle FP64 FFT A_r products at 96^3 (pseudo96) over "
              f"{args.steps} steps at {rate:.3f}/s; eigenpairs/s = rate * {NEV} / {products} products of the "
              f"oracle's own eigensolve ({src}); ms_per_step is the sample's time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(step_s),
        "projected_ms_per_eigensolve": 1000.0 * products / rate, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "projection": True},
        "cpu_eigensolve": oracle_eigensolve_sphere8(),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# secondary legs (reported beside the headline): batching and the gradient
# ---------------------------------------------------------------------------

def batch_leg(nfs, wl, torch):
    """bz48: 48 k-points of G-X-M-R-G on mixed grids (16 each at 32^3, 48^3,
    64^3), chiral spheres, nev 10, mixed precision, solved as one batch (one
    class per grid size, run concurrently).  Compared with one problem per
    grid size solved alone, scaled to the whole set."""
    w = wl.workload("bz48")
    nev = w["nev"]
    probs = [(g, tuple(float(x) for x in k), m) for g, k, m in zip(w["grid"], w["kdota"], w["medium"])]
    opts = dict(cg_tol=1e-10, eig_tol=1e-10)
    b = nfs.Batch(probs, precision="mixed", **opts)
    b.eigs(nev, allow_noconv=True)  # warm-up: bases, graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    omega, infos = b.eigs(nev, allow_noconv=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    classes = b.num_classes
    b.close()
    seq, diffs = {}, {}
    for size in (32, 48, 64):
        i = next(j for j, (g, _, _) in enumerate(probs) if g[0] == size)
        g, k, m = probs[i]
        ctx = nfs.Context(g, k, m, precision="mixed", **opts)
        om1, _, _ = ctx.eigs(nev, vectors=False, allow_noconv=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        om1, _, _ = ctx.eigs(nev, vectors=False, allow_noconv=True)
        torch.cuda.synchronize()
        seq[size] = time.perf_counter() - t1
        ctx.close()
        diffs[str(size)] = float((abs(om1 - omega[i]) / om1).max())  # per eigenvalue
    seq_total = 16 * sum(seq.values())
    # the oracle's stored eigenvalues of one problem per grid size, where written
    vs_oracle = {}
    for i in (5, 21, 37):
        ref = golden_values(f"bz48_{i}")
        if ref is not None:
            vs_oracle[str(i)] = float(max(abs(a - b) / b for a, b in zip(omega[i], ref["omega"])))
    return {"workload": "bz48: 48 k-points on G-X-M-R-G, 16 each at 32^3/48^3/64^3, chiral spheres r 0.25, "
                        "gamma U[0.2,0.8], nev 10, mixed", "classes": classes, "seconds": dt,
            "eigenpairs_per_s": len(probs) * nev / dt,
            "nconv_min": int(min(i.nconv for i in infos)),
            "restarts_max": int(max(i.restarts for i in infos)),
            "lanczos_steps_max": int(max(i.lanczos_steps for i in infos)),
            "max_rel_diff_vs_single": diffs,  # max_i |omega_i(batch) - omega_i(alone)| / omega_i
            "sequential_estimate_s": seq_total, "speedup_vs_sequential": seq_total / dt,
            "sequential_sample_s": {str(k): v for k, v in seq.items()},
            "max_rel_err_vs_oracle": vs_oracle or None}  # problem index -> max_i |omega_i - oracle_i| / oracle_i


def grad_leg(nfs, wl, torch, np):
    """field64: d(sum of the 5 lowest omega)/d(per-voxel eps, gamma) through
    nfs_eig_grad (adjoint), after a mixed-precision eigensolve (nev 6)."""
    w = wl.workload("field64")
    g, k, med = w["grid"], w["kdota"], w["medium"]
    ctx = nfs.Context(g, k, med, precision="mixed", cg_tol=1e-10, eig_tol=1e-10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    omega, Y, info = ctx.eigs(6)
    torch.cuda.synchronize()
    t_eigs = time.perf_counter() - t0
    Y5 = Y[:5].contiguous()
    wts = np.ones(5)
    ctx.eig_grad(Y5, wts)  # warm
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_eps, d_gam = ctx.eig_grad(Y5, wts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.close()
    n = g[0] * g[1] * g[2]
    return {"workload": "field64: 64^3 smoothed chiral field (eps 1..13, gamma 0..0.8), k.a=(0.1,0.2,0.3), "
                        "gradient of the sum of the 5 lowest omega", "eigensolve_s": t_eigs,
            "grad_ms": statistics.median(ms), "voxels": n,
            "grad_norm_eps": float(d_eps.norm()), "grad_norm_gamma": float(d_gam.norm())}


def bands_leg(nfs, wl, torch):
    """bands48: the band-structure sweep of Section 5.3 on a 48^3 grid: the
    chiral sphere (eps_i, eps_o, gamma) = (13, 1, 0.5), 40 k-points along
    G-X-M-R-G (10 per segment), the 10 smallest positive omega at each
    (nfs_band_structure, mixed precision)."""
    g = (48, 48, 48)
    med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    ks, _ = nfs.kpath()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    omega, infos, chunks = nfs.band_structure(g, med, ks, 10, precision="mixed", cg_tol=1e-10, eig_tol=1e-10)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"workload": "bands48: 48^3 chiral sphere r=0.25 (13, 1, 0.5), 40 k-points G-X-M-R-G, nev 10",
            "seconds": dt, "eigenpairs_per_s": omega.size / dt, "kpoints_per_s": len(ks) / dt,
            "chunks": chunks, "lanczos_steps_mean": float(sum(i.lanczos_steps for i in infos) / len(infos)),
            "cg_iterations": int(sum(i.cg_iterations for i in infos)),
            "band1_range": [float(omega[:, 0].min()), float(omega[:, 0].max())]}


def mesh_leg(nfs, wl, torch):
    """mesh: the mesh-convergence study of Section 5.1 (Fig. diff_mesh): the
    three smallest omega of the chiral sphere (13, 1, 0.5) at k = (0.5, 0, 0)
    on n^3 grids, n = 2^3 ... 2^7 (mixed precision)."""
    out = []
    for n in (8, 16, 32, 64, 128):
        g = (n, n, n)
        med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
        ctx = nfs.Context(g, (0.5, 0.0, 0.0), med, precision="mixed")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        om, _, info = ctx.eigs(3, vectors=False)
        torch.cuda.synchronize()
        out.append({"n": n, "omega": [float(x) for x in om], "seconds": time.perf_counter() - t0,
                    "lanczos_steps": info.lanczos_steps})
        ctx.close()
    return {"workload": "mesh: chiral sphere r=0.25 (13, 1, 0.5), k=(0.5,0,0), nev 3, n^3 for n = 8..128",
            "grids": out}


def nfsep_leg(nfs, wl, torch):
    """nfsep8 / nfsep16: media outside the Assumption (eq. NFSEP_org,
    Algorithm 1's second branch): the four eigenvalues nearest 2 + 0.1i of a
    lossy bi-isotropic sphere on 8^3 and 16^3 by shift-and-invert Arnoldi with
    restarted GMRES(100) (complex128; the unpreconditioned inner solves
    dominate), against the oracle's stored eigenvalues where they exist.  A
    failure is reported in the line instead of ending the run."""
    import numpy as np
    out = {}
    for n in (8, 16):
        g = (n, n, n)
        med = wl.biisotropic_sphere(g, 0.25, 13.0 + 2.0j, 1.0, 0.5, 0.2)
        try:
            ctx = nfs.NFSEPContext(g, (0.1, 0.2, 0.3), med, eig_tol=1e-10, cg_tol=1e-12, cg_maxit=20000,
                                   max_restarts=20)
            ctx.eigs(4, 2.0 + 0.1j, vectors=False, allow_noconv=True)  # warm-up: graphs captured
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            om, _, info = ctx.eigs(4, 2.0 + 0.1j, vectors=False, allow_noconv=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            ctx.close()
        except Exception as e:  # noqa: BLE001 -- recorded, the other legs stand
            out[f"nfsep{n}"] = {"error": str(e)}
            continue
        err = None
        path = os.path.join(GOLDEN, f"nfsep{n}_omega.txt")
        if os.path.exists(path):
            ref = np.loadtxt(path)
            ref = ref[:, 0] + 1j * ref[:, 1]
            err = float(np.abs(om - ref).max() / np.abs(ref).max())
        out[f"nfsep{n}"] = {
            "workload": f"nfsep{n}: {n}^3 bi-isotropic sphere r=0.25 (eps 13+2i, gamma 0.5, chi 0.2), "
                        "k.a=(0.1,0.2,0.3), 4 eigenvalues nearest 2+0.1i, complex128",
            "seconds": dt, "omega": [[float(w.real), float(w.imag)] for w in om],
            "arnoldi_steps": info.arnoldi_steps, "restarts": info.restarts,
            "gmres_iterations": int(info.gmres_iterations), "nconv": info.nconv, "status": info.status,
            "products_per_s": int(info.gmres_iterations) / dt,
            "us_per_gmres_iteration": dt / max(1, int(info.gmres_iterations)) * 1e6,
            "max_rel_err_vs_oracle": err}
    return out


def cufft_comparison(torch, dev, grid, flush, stream, product_ms):
    """Context for the product's time: the twelve 3-D FFTs of one A_r product
    (six inverse, six forward, complex64) done by cuFFT through torch.fft on
    the six field arrays alone, L2 flushed before each, against the whole
    product (FFTs, spectral assembly, material and projections)."""
    n1, n2, n3 = grid
    x = torch.randn(6, n3, n2, n1, dtype=torch.complex64, device=dev)
    for _ in range(3):
        torch.fft.ifftn(x, dim=(1, 2, 3))
        torch.fft.fftn(x, dim=(1, 2, 3))
    out = {}
    for name, fn in (("ifftn_x6_ms", lambda: torch.fft.ifftn(x, dim=(1, 2, 3))),
                     ("fftn_x6_ms", lambda: torch.fft.fftn(x, dim=(1, 2, 3)))):
        ts = []
        for _ in range(20):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = statistics.median(ts)
    out["cufft_12_transforms_ms"] = out["ifftn_x6_ms"] + out["fftn_x6_ms"]
    out["product_c64_ms"] = product_ms
    out["product_vs_cufft_transforms"] = out["cufft_12_transforms_ms"] / product_ms
    return out


def sphere64_leg(nfs, wl, torch, np):
    """sphere64 (config 2): the 64^3 chiral sphere of seeded radius and
    chirality, the 20 smallest positive omega on the plain FP64 path, against
    the oracle's stored eigenvalues."""
    w = wl.workload("sphere64")
    ctx = nfs.Context(w["grid"], w["kdota"], w["medium"], precision="fp64")
    ctx.eigs(w["nev"], vectors=False, allow_noconv=True)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    om, _, info = ctx.eigs(w["nev"], vectors=False, allow_noconv=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.close()
    gv = golden_values("sphere64")
    err = float(np.max(np.abs(om - np.array(gv["omega"])) / np.array(gv["omega"]))) if gv else None
    return {"workload": "sphere64: 64^3 chiral sphere, radius U[0.2,0.3], gamma U[0.3,0.8] (seed 0), "
                        "k.a=(0.1,0.2,0.3), nev 20, FP64", "seconds": dt, "eigenpairs_per_s": w["nev"] / dt,
            "lanczos_steps": info.lanczos_steps, "cg_iterations": int(info.cg_iterations),
            "max_rel_err_vs_oracle": err}


def fields_leg(ctx, omega, Y, n, torch, hbm):
    """Algorithm 1's final step on the headline eigenpairs: the fields
    [E; H] = B^{-1} diag(P_r, Q_r) y of all NEV eigenvectors (nfs_eig_fields,
    FP64) and their residuals in the 6n GEP (nfs_gep_residual)."""
    stream = torch.cuda.current_stream()
    m = int(Y.shape[0])
    X = ctx.eig_fields(Y)  # warm
    ms = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.eig_fields(Y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    res = ctx.gep_residual(omega, X)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = ctx.gep_residual(omega, X)
    res_ms = 1000.0 * (time.perf_counter() - t0)
    per_vec = statistics.median(ms) / m
    # algorithmic bytes per vector (complex128): pass 1 reads y (4n) and
    # writes 6n fields; the z pass reads them with the material (3 reals of
    # 1/Phi, one gamma) and writes X (6n)
    fbytes = n * (4 * 16 + 6 * 16 + 6 * 16 + 4 * 8 + 6 * 16)
    return {"vectors": m, "fields_ms_per_vector": per_vec,
            "fields_GBps": fbytes / (per_vec / 1e3) / 1e9, "fields_frac": fbytes / (per_vec / 1e3) / 1e9 / hbm,
            "residual_ms_per_vector": res_ms / m, "max_gep_residual": float(max(res))}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import workloads as wl
    from paper_1402_6297_gb300 import nfs

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = wl.workload(WORKLOAD)
    grid, med = w["grid"], w["medium"]
    kd = rank_kpoint(w["kdota"], rank)
    n1, n2, n3 = grid
    n = n1 * n2 * n3
    hbm, peak_kind = peaks()
    stream = torch.cuda.current_stream()

    if args.profile_grid:
        g = (args.profile_grid,) * 3
        pc = nfs.Context(g, kd, wl.pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4, (0, 1), 0), precision="mixed",
                         cg_tol=1e-10, eig_tol=1e-10)
        for _ in range(args.warmup):
            pc.eigs(10, vectors=False, allow_noconv=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, _, pinfo = pc.eigs(10, vectors=False, allow_noconv=True)
        torch.cuda.synchronize()
        pc.close()
        if rank == 0:
            print(json.dumps({"mode": "profile-grid", "grid": list(g), "nev": 10,
                              "s_per_eigensolve": (time.perf_counter() - t0) / max(1, args.steps),
                              "lanczos_steps": pinfo.lanczos_steps, "seconds_orth": pinfo.seconds_orth}), flush=True)
        return 0

    ctx = nfs.Context(grid, kd, med, precision="mixed", cg_tol=1e-10, eig_tol=1e-10)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # ---- A_r products: whole product and each pass, CUDA events on the stream
    def time_matvec(dtype, reps=20):
        u = torch.from_numpy(wl.random_complex(4 * n, 5)).to(dev).to(dtype)
        out = torch.empty_like(u)
        for _ in range(3):
            ctx.matvec(u, out)
        whole, passes = [], [[], [], []]
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.matvec(u, out)
            e1.record(stream)
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            for i, mask in enumerate((1, 2, 4)):
                ctx.matvec_passes(mask, u, out)
                ev[i + 1].record(stream)
            torch.cuda.synchronize()
            whole.append(e0.elapsed_time(e1))
            for i in range(3):
                passes[i].append(ev[i].elapsed_time(ev[i + 1]))
        return statistics.median(whole), [statistics.mean(p) for p in passes]

    mv64_ms, pass64 = time_matvec(torch.complex64)
    mv128_ms, pass128 = time_matvec(torch.complex128)
    bpp = bytes_per_pass(n, 8, med.kind)
    dom = max(range(3), key=lambda i: pass64[i])
    achieved = bpp[dom] / (pass64[dom] / 1000.0) / 1e9
    whole_bytes = sum(bpp)
    roof = {"bound": "hbm", "kernel": PASS_KERNELS[dom],
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "traffic": profiled_traffic(dom),
            "traffic_note": "ncu dram read+write bytes per launch (cold cache; the fields a pass writes stay in L2)",
            "matvec_c64": {"bytes": whole_bytes, "ms": mv64_ms, "GBps": whole_bytes / (mv64_ms / 1e3) / 1e9,
                           "frac": whole_bytes / (mv64_ms / 1e3) / 1e9 / hbm},
            "pass_ms_c64": pass64, "pass_ms_c128": pass128,
            "pass_GBps_c64": [b / (t / 1e3) / 1e9 for b, t in zip(bpp, pass64)]}
    if args.matvec_only:
        if rank == 0:
            line = {"metric": "A_r products/s at 96^3 (pseudo96)", "mode": "matvec-only",
                    "matvecs_per_s": {"c64": 1000.0 / mv64_ms, "c128": 1000.0 / mv128_ms}, "roofline": roof}
            if args.cufft:
                line["cufft_comparison"] = cufft_comparison(torch, dev, grid, flush, stream, mv64_ms)
            print(json.dumps(line), flush=True)
        ctx.close()
        return 0

    # ---- the step: one mixed-precision eigensolve (nev = 20)
    for _ in range(args.warmup):
        ctx.eigs(NEV, vectors=True, allow_noconv=True)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    infos, step_ms, omega, Y = [], [], None, None
    t_host0 = time.perf_counter()
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("timed_steps")  # lets a profiler select the timed region
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        omega, Y, info = ctx.eigs(NEV, vectors=True, allow_noconv=True)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_pop()
    host_s = time.perf_counter() - t_host0
    barrier(world)
    clocks = sampler.stop() if sampler else None
    total_s = max_over_ranks(sum(step_ms) / 1000.0, world, dev)
    value = world * NEV * args.steps / total_s
    info = infos[-1]
    matvecs = info.matvecs_c64 + info.matvecs_c128
    cg_its = info.cg_iterations
    res = nfs.residuals(ctx, omega, Y)
    gv = golden_values(WORKLOAD) if rank == 0 and kd == tuple(w["kdota"]) else None
    oracle_err = float(np.max(np.abs(omega - np.array(gv["omega"])) / np.array(gv["omega"]))) if gv else None

    # ---- the paper's basis size (eigs with ncv = 3 nev = 60: thick restarts)
    paper_ncv = None
    if rank == 0 and not args.skip_paper_ncv:
        cp = nfs.Context(grid, kd, med, precision="mixed", cg_tol=1e-10, eig_tol=1e-10, ncv=3 * NEV)
        cp.eigs(NEV, vectors=False, allow_noconv=True)  # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        omp, _, infp = cp.eigs(NEV, vectors=False, allow_noconv=True)
        e1.record(stream)
        torch.cuda.synchronize()
        msp = e0.elapsed_time(e1)
        paper_ncv = {"ncv": 3 * NEV, "eigenpairs_per_s": NEV / (msp / 1000.0), "ms": msp,
                     "lanczos_steps": infp.lanczos_steps, "restarts": infp.restarts,
                     "cg_iterations": int(infp.cg_iterations),
                     "max_rel_diff_vs_default_ncv": float(np.max(np.abs(omp - omega) / omega)),
                     "max_rel_err_vs_oracle": (float(np.max(np.abs(omp - np.array(gv["omega"]))
                                                             / np.array(gv["omega"]))) if gv else None)}
        cp.close()

    # ---- FP64 eigensolve for comparison
    fp64 = None
    if not args.skip_fp64:
        ctx64 = nfs.Context(grid, kd, med, precision="fp64", cg_tol=1e-12, eig_tol=1e-10)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        om64, _, inf64 = ctx64.eigs(NEV, vectors=False, allow_noconv=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"eigenpairs_per_s": NEV / (ms64 / 1000.0), "ms": ms64,
                "lanczos_steps": inf64.lanczos_steps, "cg_iterations": int(inf64.cg_iterations),
                "max_rel_diff_mixed_vs_fp64": float(np.max(np.abs(omega - om64) / om64))}
        ctx64.close()

    # ---- end to end through the public API: host material in pinned memory
    # is copied by nfs_setup, the eigensolve runs, omega is read back.
    pin_eps = torch.from_numpy(np.ascontiguousarray(med.eps)).pin_memory()
    pin_gam = torch.from_numpy(np.ascontiguousarray(med.gamma)).pin_memory()
    med_pinned = wl.Medium(med.grid, med.kind, pin_eps.numpy(), pin_gam.numpy(), None, med.axes)
    e2e_ms = []
    for i in range(0 if args.skip_e2e else max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = nfs.Context(grid, kd, med_pinned, precision="mixed", cg_tol=1e-10, eig_tol=1e-10)
        om2, _, _ = c2.eigs(NEV, vectors=False, allow_noconv=True)
        c2.close()
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_total = max_over_ranks(sum(e2e_ms) / 1000.0, world, dev) if e2e_ms else 0.0
    e2e_value = world * NEV * len(e2e_ms) / e2e_total if e2e_ms else None
    h2d = pin_eps.numel() * 8 + pin_gam.numel() * 8
    d2h = NEV * 8

    fields = None if (args.skip_fields or rank != 0) else fields_leg(ctx, omega, Y, n, torch, hbm)
    sphere64 = None if (args.skip_sphere64 or rank != 0) else sphere64_leg(nfs, wl, torch, np)
    # the secondary legs get the device memory of the headline context
    ctx.close()
    batch = None if (args.skip_batch or rank != 0) else batch_leg(nfs, wl, torch)
    grad = None if (args.skip_grad or rank != 0) else grad_leg(nfs, wl, torch, np)
    bands = None if (args.skip_bands or rank != 0) else bands_leg(nfs, wl, torch)
    mesh = None if (args.skip_mesh or rank != 0) else mesh_leg(nfs, wl, torch)
    nfsep_r = None if (args.skip_nfsep or rank != 0) else nfsep_leg(nfs, wl, torch)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        rate, calls, dt = oracle_matvec_rate(w, args.cpu_seconds)
        products, src = oracle_products_per_solve()
        if products is None:
            products, src = matvecs, "this GPU eigensolve"
        cpu = {"value": rate * NEV / products, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "cpu_model": cpu_model(), "projection": True,
               "sample": f"PROJECTION: {calls} oracle FP64 FFT A_r products at 96^3 in {dt:.1f} s ({rate:.3f}/s); "
                         f"eigenpairs/s = rate * {NEV} / {products} products of the oracle's own eigensolve "
                         f"({src})",
               "eigensolve": oracle_eigensolve_sphere8()}
        gv = golden_values(WORKLOAD)
        if gv and gv["seconds"]:
            cpu["stored_oracle_eigensolve"] = {
                "workload": WORKLOAD, "seconds": gv["seconds"], "products": gv["products"],
                "eigenpairs_per_s": NEV / gv["seconds"],
                "note": "the tier-O3 solve that wrote tests/golden (one core of the build container, not this box)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s * 1000.0 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": CONFIG,
        "precision": "mixed: complex64 CG, double-single refinement residuals, FP64 Lanczos",
        "matvecs_per_s": {"c64": 1000.0 / mv64_ms, "c128": 1000.0 / mv128_ms},
        "cg_iters_per_s": cg_its / (statistics.mean(step_ms) / 1000.0),
        # one complex64 CG iteration, algorithmic bytes (64 n s + material):
        # the product (3-pass bytes) + pass 1 reading r and writing p + the
        # x/r step reading x, r, p, A p and writing x, r (vectors of 4n
        # complex64; the step runs fused into pass 3, which never stores A p)
        "cg_iteration": cg_iteration_roofline(n, sum(bpp), info, hbm),
        "eigensolve": {"lanczos_steps": info.lanczos_steps, "restarts": info.restarts,
                       "cg_iterations": int(cg_its), "matvecs_c64": int(info.matvecs_c64),
                       "matvecs_c128": int(info.matvecs_c128), "nconv": info.nconv,
                       "max_residual": max(res), "omega": [float(x) for x in omega],
                       "host_s": host_s,
                       "split_s": {"total": info.seconds_total, "cg": info.seconds_cg,
                                   "refine": info.seconds_refine, "ritz": info.seconds_ritz,
                                   "lanczos": info.seconds_total - info.seconds_cg - info.seconds_refine
                                   - info.seconds_ritz,
                                   "lanczos_recurrence": info.seconds_recurrence,
                                   "lanczos_orth": info.seconds_orth, "ritz_vectors": info.seconds_vectors},
                       "reorthogonalisations": info.reorthogonalisations,
                       "max_rel_err_vs_oracle": oracle_err},
        "paper_ncv": paper_ncv,
        "sphere64_fp64": sphere64,
        "fp64": fp64,
        "batch": batch,
        "gradient": grad,
        "fields": fields,
        "bands": bands,
        "mesh": mesh,
        "nfsep": nfsep_r,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # kernels the library launched inside the timed region (its own count,
        # CUDA graph nodes included)
        "gpu_launches": int(sum(i.kernel_launches for i in infos)),
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
