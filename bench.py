#!/usr/bin/env python3
"""Throughput benchmark of the stream-and-collide hot path on GB300.

Default workload (the headline metric): D3Q19 LBGK, FP32 arithmetic with
FP32 shifted storage (f - w), 256^3 periodic Taylor-Green vortex, tau 0.6,
u0 0.05.  One bench step = one lattice Boltzmann time step over all nodes
(one fused stream-collide launch); the K timed steps are replayed as one CUDA
graph (captured beforehand in an untimed run of K steps; --no-graph times K
direct launches).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tg256|duct|elbm|kida|ldc|batch] [--dtype f32s|f16s|bf16s|f32]

For N > 1 (torchrun) every rank runs an independent replica of the workload
(the domains do not exchange data; weak scaling) and rank 0 reports the
aggregate.  --impl reference times the FP64 CPU oracle on the host cores on a
bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

B_PER_NODE = {"f32s": 152, "f32": 152, "f16s": 76, "bf16s": 76, "f64": 304}   # D3Q19
ESIZE = {"f32s": 4, "f32": 4, "f16s": 2, "bf16s": 2, "f64": 8}
LATTICE_NAME = {0: "D2Q9", 1: "D3Q19", 2: "D3Q15", 3: "D3Q27"}
LATTICE_Q = {0: 9, 1: 19, 2: 15, 3: 27}
MODEL_NAME = {0: "LBGK", 1: "MRT", 2: "ELBM", 3: "REG", 4: "SMAG"}
# lbm_set_masked_kernel modes (LBM_MASKED_AUTO, _NODE, _ZRUN)
MASKED_KERNEL = {"auto": 0, "node": 1, "zrun": 2}


def bytes_per_node(dtype, lattice=1):
    """Algorithmic bytes of one node update: q values read and q written."""
    return 2 * LATTICE_Q[lattice] * ESIZE[dtype]


def algorithmic_bytes(nodes, fluid, fluid_bytes, solid_bytes):
    """Bytes a step must move: every fluid (updated) node its q values in and
    out plus its geometry word; a solid node only its geometry word (its
    populations are neither needed nor written)."""
    return fluid * fluid_bytes + (nodes - fluid) * solid_bytes
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tg256",
                    choices=["tg256", "duct", "elbm", "kida", "ldc", "batch", "mlp"])
    ap.add_argument("--alpha", default="newton", choices=["newton", "series", "mlp", "root"],
                    help="ELBM alpha solve for --workload elbm (root: the truncated-series "
                         "root guess)")
    ap.add_argument("--guard-steps", type=int, default=2,
                    help="ELBM guarded modes: evaluations that may end in early acceptance")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="N > 1 ranks: independent replicas (weak scaling), or one slab of the "
                         "workload per rank with the faces exchanged every step (Sec. 3.6; "
                         "strong scaling)")
    ap.add_argument("--dist-backend", default="",
                    help="torch.distributed backend of --decomp slab (default nccl; gloo "
                         "stages the faces through host memory)")
    ap.add_argument("--ndom", type=int, default=512, help="domains for --workload batch")
    ap.add_argument("--mlp-kernel", default="tc", choices=["tc", "fp32"],
                    help="--workload mlp (and the surrogate of --alpha mlp): BF16 "
                         "tensor-core or FP32 training kernel")
    ap.add_argument("--mlp-batch", type=int, default=16384, help="--workload mlp: minibatch")
    ap.add_argument("--batch-config", default="",
                    help="launch configuration for --workload batch instead of autotuning: "
                         "threads,ctas,tile_width,tile_rows,variant")
    ap.add_argument("--pattern", default="ab", choices=["ab", "aa"],
                    help="distribution access pattern (AA: one array)")
    ap.add_argument("--round", default="dither", choices=["dither", "nearest"],
                    help="rounding of FP16/BF16 stores")
    ap.add_argument("--dtype", default="f32s", choices=["f32s", "f32", "f16s", "bf16s"])
    ap.add_argument("--model", default="", choices=["", "bgk", "mrt", "reg", "smag"],
                    help="override the collision model of the tg256 / duct / kida workloads")
    ap.add_argument("--lattice", default="", choices=["", "q15", "q19", "q27"],
                    help="override the 3-D velocity set of the workload")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--shape", default="",
                    help="override the domain as NX,NY,NZ (e.g. the paper's duct 254,127,512)")
    ap.add_argument("--size", type=int, default=0,
                    help="override the cube edge of the 256^3 workloads (profiling runs)")
    ap.add_argument("--subdomains", type=int, default=0,
                    help="run the workload as S slabs with ghost-row exchange (one GPU)")
    ap.add_argument("--direct", action="store_true",
                    help="with --subdomains: store straight into the neighbour's ghost row")
    ap.add_argument("--no-overlap", action="store_true",
                    help="with --subdomains: exchange after whole slabs, no bulk/boundary split")
    ap.add_argument("--masked-kernel", default="auto", choices=["auto", "node", "zrun"],
                    help="kernel of masked 3-D AB steps (lbm_set_masked_kernel)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="time K direct launches instead of replaying the K steps as one CUDA "
                         "graph (captured in an untimed run of K steps after the warm-up)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# the sources of the headline kernel (LBGK stream-collide): its translation
# unit and the headers it includes
KERNEL_SOURCES = ("k_bgk.cu", "step_kernel.cuh", "collide.cuh", "lbm_device.cuh",
                  "fp_bits.cuh")
# the ELBM kernel's
ELBM_SOURCES = ("k_elbm.cu", "step_kernel.cuh", "collide.cuh", "lbm_device.cuh", "fp_bits.cuh")


def source_sha(names=KERNEL_SOURCES):
    """Hash of a kernel's sources; a recorded profiler figure is reported
    only while they are unchanged."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1311_2404_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fp64_inst_for(alpha, dtype, nodes):
    """FP64-pipe warp instructions per node of the ELBM kernel from the
    committed ncu record (profiles/fp64_elbm.json), if the ELBM sources are
    unchanged since that capture and the workload has the record's node
    count (the count per node depends on the field); else None."""
    path = os.path.join(ROOT, "profiles", "fp64_elbm.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(f"elbm:{alpha}:{dtype}")
    if not e or e.get("source_sha") != source_sha(ELBM_SOURCES) or e.get("nodes") != nodes:
        return None
    return float(e["fp64_warp_inst_per_node"])


def traffic_key(workload, dtype, model, lattice):
    """Key of a kernel's DRAM-traffic record: workload, storage, collision
    model and lattice (a record holds for that kernel only)."""
    return f"{workload}:{dtype}:{MODEL_NAME[model]}:{LATTICE_NAME[lattice]}"


def traffic_for(workload, dtype, model, lattice, nodes):
    """DRAM bytes per launch from the committed ncu summary for this kernel,
    if its sources are unchanged since that capture and the workload has the
    captured node count; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(traffic_key(workload, dtype, model, lattice))
    if not e or e.get("source_sha") != source_sha() or e.get("nodes") != nodes:
        return None
    return float(e["bytes_per_launch"])


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings: the slowest rank sets the
    job's time.  One all-reduce when world > 1."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_glups(nodes_per_rank, steps, world, ms_max):
    """Whole-job throughput: every rank's updates over the slowest rank's time."""
    return nodes_per_rank * steps * world / (ms_max * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload_spec(name, dtype, size=0, model="", lattice="", shape=""):
    spec = _workload_spec(name, dtype)
    if shape and name in ("duct", "tg256", "kida"):
        nxs, nys, nzs = (int(v) for v in shape.split(","))
        old = "x".join(str(v) for v in spec["n"]) if name == "duct" else f"{spec['n'][0]}^3"
        spec["n"] = (nxs, nys, nzs)
        spec["name"] = spec["name"].replace(old, f"{nxs}x{nys}x{nzs}")
    if lattice and name != "batch":
        from paper_1311_2404_gb300 import abi as lbm   # constants only: loads no library
        spec["lattice"] = {"q15": lbm.LBM_D3Q15, "q19": lbm.LBM_D3Q19,
                           "q27": lbm.LBM_D3Q27}[lattice]
        spec["name"] = spec["name"].replace("d3q19", "d3" + lattice)
    if model:
        spec["model"] = {"bgk": 0, "mrt": 1, "reg": 3, "smag": 4}[model]
        for m in ("lbgk", "mrt", "smag"):
            if f"_{m}_" in spec["name"]:
                spec["name"] = spec["name"].replace(f"_{m}_", f"_{model}_")
    if size and name in ("tg256", "elbm", "kida", "ldc"):
        spec["n"] = (size, size, size)
        for tag in ("256^3", "350^3", "254^3"):
            spec["name"] = spec["name"].replace(tag, f"{size}^3")
        if name == "ldc":
            from paper_1311_2404_gb300 import workloads as wl
            spec["tau"] = wl.ldc_tau(size)
    if size and name == "duct":
        spec["n"] = (2 * size, size, size)
        spec["name"] = spec["name"].replace("512x256x256", f"{2 * size}x{size}x{size}")
    return spec


def _workload_spec(name, dtype):
    # the ABI's constants only: the CPU reference arm must not load the CUDA library
    from paper_1311_2404_gb300 import abi as lbm
    dmap = {"f32s": lbm.LBM_F32S, "f32": lbm.LBM_F32, "f16s": lbm.LBM_F16S,
            "bf16s": lbm.LBM_BF16S}
    if name == "tg256":
        return dict(kind="tg", name="d3q19_lbgk_taylor_green_256^3", n=(256, 256, 256),
                    lattice=lbm.LBM_D3Q19,
                    model=lbm.LBM_BGK, tau=0.6, dtype=dmap[dtype], mask=None, force=(0, 0, 0))
    if name == "duct":
        return dict(kind="duct", name="d3q19_mrt_sphere_duct_512x256x256", n=(512, 256, 256),
                    lattice=lbm.LBM_D3Q19, model=lbm.LBM_MRT, tau=0.55, dtype=dmap[dtype],
                    mask="duct", force=(1e-5, 0, 0))
    if name == "elbm":
        return dict(kind="turb", name="d3q19_elbm_decaying_turbulence_256^3", n=(256, 256, 256),
                    lattice=lbm.LBM_D3Q19, model=lbm.LBM_ELBM, tau=0.5005, dtype=dmap[dtype],
                    mask=None, force=(0, 0, 0))
    if name == "ldc":
        # the paper's benchmark cavity, Re = 1000 with a lid at 0.05, regularized lid
        from paper_1311_2404_gb300 import workloads as wl
        return dict(kind="ldc", name="d3q19_lbgk_lid_driven_cavity_254^3", n=(254, 254, 254),
                    lattice=lbm.LBM_D3Q19, model=lbm.LBM_BGK, tau=wl.ldc_tau(254),
                    dtype=dmap[dtype], mask="ldc", force=(0, 0, 0),
                    bcs=[(0, lbm.LBM_BC_VELOCITY, lbm.LBM_BC_REGULARIZED, -2, [0.05, 0.0, 0.0])])
    if name == "kida":
        # Re = N u0 / nu = 4000 at N = 350, u0 = 0.05 (the paper's smaller Kida case)
        return dict(kind="kida", name="d3q19_smag_kida_vortex_350^3", n=(350, 350, 350),
                    lattice=lbm.LBM_D3Q19, model=lbm.LBM_SMAG, tau=0.5 + 3 * 350 * 0.05 / 4000,
                    dtype=dmap[dtype], mask=None, force=(0, 0, 0))
    raise ValueError(name)


def workload_inputs(spec):
    from paper_1311_2404_gb300 import workloads as wl
    nx, ny, nz = spec["n"]
    if spec["kind"] == "tg":
        rho, u = wl.taylor_green(nx, 0.05, nz=nz, D=3)
        mask = None
    elif spec["kind"] == "duct":
        mask, _ = wl.duct_with_spheres(nx, ny, nz)
        rho = np.ones((nz, ny, nx))
        u = np.zeros((3, nz, ny, nx))
    elif spec["kind"] == "kida":
        rho, u = wl.kida(nx, 0.05)
        mask = None
    elif spec["kind"] == "ldc":
        mask = wl.ldc_mask(nx)
        rho = np.ones((nz, ny, nx))
        u = np.zeros((3, nz, ny, nx))
    else:
        rho, u = wl.turbulence(nx)
        mask = None
    return rho.astype(np.float32), u.astype(np.float32), mask


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_multi(args):
    """The workload as S slabs exchanging ghost rows after every step."""
    import torch
    torch.cuda.set_device(0)
    from paper_1311_2404_gb300 import lbm
    spec = workload_spec(args.workload, args.dtype, args.size, args.model, args.lattice, args.shape)
    nx, ny, nz = spec["n"]
    nodes = nx * ny * nz
    rho, u, mask = workload_inputs(spec)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        m = lbm.lbm_multi_create(nx, ny, nz, spec["lattice"], spec["model"], spec["tau"],
                                 spec["dtype"], args.subdomains)
        lbm.lbm_multi_set_stream(m, stream.cuda_stream)
        lbm.lbm_multi_set_overlap(m, not args.no_overlap)
        lbm.lbm_multi_set_graph(m, True)
        if args.direct:
            lbm.lbm_multi_set_transfer(m, lbm.LBM_TRANSFER_DIRECT)
        for b in spec.get("bcs", ()):
            lbm.lbm_multi_set_boundary(m, *b)
        if mask is not None:
            lbm.lbm_multi_set_geometry(m, mask)
        if any(spec["force"]):
            lbm.lbm_multi_set_force(m, *spec["force"])
        lbm.lbm_multi_set_rounding(m, lbm.LBM_ROUND_NEAREST if args.round == "nearest"
                                   else lbm.LBM_ROUND_DITHER)
        lbm.lbm_multi_init_equilibrium(m, torch.from_numpy(rho).cuda(),
                                       torch.from_numpy(u).cuda())
        for _ in range(max(args.warmup, 3)):
            lbm.lbm_multi_step(m, 1)
        lbm.lbm_multi_step(m, args.steps)                 # capture the timed graph
        lbm.lbm_multi_sync(m)
        sampler = ClockSampler(0)
        sampler.start()
        torch.cuda.synchronize()
        l0 = lbm.lbm_multi_launch_count(m)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lbm.lbm_multi_step(m, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = lbm.lbm_multi_launch_count(m) - l0
        clocks = sampler.stop()
        lbm.lbm_multi_sync(m)
        hb = lbm.lbm_multi_halo_bytes(m)
        pin_r = torch.from_numpy(rho).pin_memory()
        pin_u = torch.from_numpy(u).pin_memory()
        out_r = torch.empty_like(pin_r).pin_memory()
        out_u = torch.empty_like(pin_u).pin_memory()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            lbm.lbm_multi_init_equilibrium(m, pin_r, pin_u)
            lbm.lbm_multi_step(m, 1)
            lbm.lbm_multi_get_macro(m, out_r, out_u)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / max(args.e2e_steps, 1)
        lbm.lbm_multi_destroy(m)
    glups = nodes * args.steps / (ms * 1e-3) / 1e9
    bpn = bytes_per_node(args.dtype, spec["lattice"]) + (4 if mask is not None else 0)
    fluid = int((mask != 1).sum()) if mask is not None else nodes
    alg = algorithmic_bytes(nodes, fluid, bpn, 4)
    per_launch_s = ms / 1e3 / args.steps
    achieved = alg / per_launch_s / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": "D3Q19 GLUPS & % HBM roofline; FP16/learned vs plain FP32 at fixed error",
        "value": round(glups, 4), "unit": "GLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms / args.steps, 6),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded analytic/random initial fields; no dataset)",
        "config": {"workload": spec["name"], "lattice": LATTICE_NAME[spec["lattice"]],
                   "model": {0: "LBGK", 1: "MRT", 2: "ELBM", 3: "REG", 4: "SMAG"}[spec["model"]],
                   "storage": args.dtype, "tau": spec["tau"], "nodes": nodes,
                   "subdomains": args.subdomains, "overlap": not args.no_overlap,
                   "transfer": "direct" if args.direct else "staged",
                   "halo_bytes_per_step": hb, "parallelism": "single (slabs emulated)",
                   "l2": "working set > 129 MB L2 (inputs larger than L2, no flush)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "bytes_per_node": round(alg / nodes, 2),
                     "note": "algorithmic bytes of the updates; the exchange adds "
                             "3 x halo bytes of copies per step"},
        "e2e": {"value": round(nodes / e2e_s / 1e9, 4), "unit": "GLUPS",
                "h2d_bytes_per_step": int(rho.nbytes + u.nbytes),
                "d2h_bytes_per_step": int(rho.nbytes + u.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_slabs(args):
    """The workload cut into one slab per rank (Sec. 3.6): every step each
    rank updates its slab and exchanges its two faces with its neighbours
    (NCCL point-to-point on the exchange stream, overlapped with the bulk
    rows).  The whole domain is fixed, so this is strong scaling."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    backend = args.dist_backend or "nccl"
    if world > 1:
        dist.init_process_group(backend)
    from paper_1311_2404_gb300 import lbm, slabs
    spec = workload_spec(args.workload, args.dtype, args.size, args.model, args.lattice, args.shape)
    nx, ny, nz = spec["n"]
    nodes = nx * ny * nz
    rho, u, mask = workload_inputs(spec)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sl = slabs.RankSlab(nx, ny, nz, spec["lattice"], spec["model"], spec["tau"],
                            spec["dtype"], rank, world, stream=stream.cuda_stream,
                            overlap=not args.no_overlap)
        for b in spec.get("bcs", ()):
            sl.set_boundary(*b)
        if mask is not None:
            sl.set_geometry(mask)
        if any(spec["force"]):
            sl.set_force(*spec["force"])
        sl.set_rounding(lbm.LBM_ROUND_NEAREST if args.round == "nearest"
                        else lbm.LBM_ROUND_DITHER)
        sl.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        sl.step(max(args.warmup, 3))
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if rank == 0 else None
        if sampler:
            sampler.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = lbm.lbm_multi_launch_count(sl.m)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sl.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        launches = lbm.lbm_multi_launch_count(sl.m) - l0
        clocks = sampler.stop() if sampler else None
        lo, hi = sl.rows
        local_nodes = nodes * (hi - lo) // (nz if spec["lattice"] != lbm.LBM_D2Q9 else ny)
        hb = sl.halo_bytes()
        # end to end: the rank's whole-domain inputs from pinned host memory,
        # one step, its rows back to pinned host memory
        pin_r = torch.from_numpy(rho).pin_memory()
        pin_u = torch.from_numpy(u).pin_memory()
        out_r = torch.zeros_like(pin_r).pin_memory()
        out_u = torch.zeros_like(pin_u).pin_memory()
        e2e_steps = max(1, min(args.e2e_steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            sl.init(pin_r, pin_u)
            sl.step(1)
            lbm.lbm_multi_get_macro(sl.m, out_r, out_u)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        sl.close()
    ms_max, e2e_ms = max_over_ranks([ms, e2e_s * 1e3], world, "cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    glups = nodes * args.steps / (ms_max * 1e-3) / 1e9
    bpn = bytes_per_node(args.dtype, spec["lattice"]) + (4 if mask is not None else 0)
    achieved = local_nodes * bpn / (ms / 1e3 / args.steps) / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": "D3Q19 GLUPS & % HBM roofline; FP16/learned vs plain FP32 at fixed error",
        "value": round(glups, 4), "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms_max / args.steps, 6),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded analytic/random initial fields; no dataset)",
        "config": {"workload": spec["name"], "lattice": LATTICE_NAME[spec["lattice"]],
                   "model": {0: "LBGK", 1: "MRT", 2: "ELBM", 3: "REG", 4: "SMAG"}[spec["model"]],
                   "storage": args.dtype, "tau": spec["tau"], "nodes": nodes,
                   "parallelism": f"slab{world}", "backend": backend if world > 1 else None,
                   "overlap": not args.no_overlap, "halo_bytes_per_step_per_rank": hb,
                   "l2": "working set > 129 MB L2 per rank (inputs larger than L2, no flush)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "bytes_per_node": bpn,
                     "note": "rank 0's slab updates per its own kernel time; the exchange "
                             "moves halo_bytes_per_step_per_rank more"},
        "e2e": {"value": round(nodes / (e2e_ms * 1e-3) / 1e9, 4), "unit": "GLUPS",
                "h2d_bytes_per_step": int(rho.nbytes + u.nbytes),
                "d2h_bytes_per_step": int((rho.nbytes + u.nbytes) * (hi - lo) //
                                          (nz if spec["lattice"] != lbm.LBM_D2Q9 else ny))},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def elbm_compare(lbm, sim, spec, rho, u, args, stream):
    """After the timed steps: kinetic energy of this run against a Newton run
    of the same steps from the same state, and the entropy-condition residual
    |g(alpha)| / a_2 over one more (untimed) step in diagnostic mode."""
    t = lbm.lbm_get_time(sim.h)
    E, _ = lbm.lbm_kinetic_energy_enstrophy(sim.h)
    out = {"t": int(t), "E": E}
    nx, ny, nz = spec["n"]
    if args.alpha != "newton":
        ref = lbm.Simulation(nx, ny, nz, spec["lattice"], spec["model"], spec["tau"],
                             spec["dtype"], stream=stream.cuda_stream)
        lbm.lbm_set_elbm(ref.h, lbm.LBM_ALPHA_NEWTON, 1e-12, 20, 1e-3)
        lbm.lbm_init_equilibrium(ref.h, torch_from(rho), torch_from(u))
        lbm.lbm_step(ref.h, int(t))
        Er, _ = lbm.lbm_kinetic_energy_enstrophy(ref.h)
        ref.close()
        out["E_rel_diff_vs_newton"] = abs(E - Er) / Er
    lbm.lbm_set_elbm_diagnostics(sim.h, 1)
    lbm.lbm_step(sim.h, 1)
    mean, mx, cnt = lbm.lbm_get_elbm_entropy_error(sim.h)
    lbm.lbm_set_elbm_diagnostics(sim.h, 0)
    out.update({"entropy_resid_mean": mean, "entropy_resid_max": mx, "entropy_resid_nodes": cnt})
    return out


def torch_from(a):
    import torch
    return torch.from_numpy(a).cuda()


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1311_2404_gb300 import lbm

    spec = workload_spec(args.workload, args.dtype, args.size, args.model, args.lattice, args.shape)
    nx, ny, nz = spec["n"]
    nodes = nx * ny * nz
    rho, u, mask = workload_inputs(spec)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = lbm.Simulation(nx, ny, nz, spec["lattice"], spec["model"], spec["tau"],
                             spec["dtype"], stream=stream.cuda_stream,
                             pattern=lbm.LBM_PATTERN_AA if args.pattern == "aa"
                             else lbm.LBM_PATTERN_AB)
        for b in spec.get("bcs", ()):
            lbm.lbm_set_boundary(sim.h, *b)
        if mask is not None:
            sim.set_geometry(mask)
        lbm.lbm_set_masked_kernel(sim.h, MASKED_KERNEL[args.masked_kernel])
        if any(spec["force"]):
            sim.set_force(*spec["force"])
        lbm.lbm_set_rounding(sim.h, lbm.LBM_ROUND_NEAREST if args.round == "nearest"
                             else lbm.LBM_ROUND_DITHER)
        if spec["model"] == lbm.LBM_ELBM:
            mode = {"newton": lbm.LBM_ALPHA_NEWTON, "series": lbm.LBM_ALPHA_SERIES_GUARDED,
                    "mlp": lbm.LBM_ALPHA_MLP_GUARDED,
                    "root": lbm.LBM_ALPHA_ROOT_GUARDED}[args.alpha]
            if args.alpha == "mlp":
                # the surrogate learns from Newton-solved steps of this very
                # workload (its field sets the distribution of the invariants)
                from paper_1311_2404_gb300 import alpha_training as at
                lbm.lbm_set_elbm(sim.h, lbm.LBM_ALPHA_NEWTON, 1e-12, 20, 1e-3)
                lbm.lbm_init_equilibrium(sim.h, torch.from_numpy(rho).cuda(),
                                         torch.from_numpy(u).cuda())
                Xp, yp = at.collect_pairs_from(sim, rounds=3, steps_between=2, stride=16)
                P, _ = at.train(Xp, yp, kernel=lbm.LBM_MLP_BF16_TC if args.mlp_kernel == "tc"
                                else lbm.LBM_MLP_FP32)
                lbm.lbm_load_alpha_mlp(sim.h, P)
            lbm.lbm_set_elbm(sim.h, mode, 1e-12, 20, 1e-3)
            lbm.lbm_set_elbm_guard(sim.h, args.guard_steps, 1e-6)
        rho_d = torch.from_numpy(rho).cuda()
        u_d = torch.from_numpy(u).cuda()
        lbm.lbm_init_equilibrium(sim.h, rho_d, u_d)      # inputs resident in HBM
        stream.synchronize()
        for _ in range(max(args.warmup, 3)):
            lbm.lbm_step(sim.h, 1)
        if args.graph:
            lbm.lbm_set_graph(sim.h, True)
            lbm.lbm_step(sim.h, args.steps)               # capture (untimed)
            if args.steps % 2:                            # the state back in the first array
                lbm.lbm_step(sim.h, 1)
        stream.synchronize()

        sampler = ClockSampler(local) if rank == 0 else None
        if sampler:
            sampler.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = lbm.lbm_launch_count(sim.h)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lbm.lbm_step(sim.h, args.steps)                   # K fused launches
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        launches = lbm.lbm_launch_count(sim.h) - l0
        clocks = sampler.stop() if sampler else None
        lbm.lbm_sync(sim.h)
        elbm_stats = None
        diag = None
        elbm_cmp = None
        if spec["kind"] == "kida":
            E, Om = lbm.lbm_kinetic_energy_enstrophy(sim.h)
            diag = {"t": int(lbm.lbm_get_time(sim.h)), "E": E, "Omega": Om,
                    "E_over_E0": round(E / (3 * 0.05 ** 2 / 8), 6)}
        if spec["model"] == lbm.LBM_ELBM:
            st = lbm.lbm_get_elbm_stats(sim.h)
            elbm_stats = {"g_evals_per_node": round(st[0] / max(st[5], 1), 4),
                          "skipped_frac": round(st[1] / max(st[5], 1), 4),
                          "guess_accepted_frac": round(st[4] / max(st[5], 1), 4),
                          "at_cap": int(st[3])}
            if spec["kind"] == "turb":
                elbm_cmp = elbm_compare(lbm, sim, spec, rho, u, args, stream)

        # end to end through the public API with host buffers
        pin_r = torch.from_numpy(rho).pin_memory()
        pin_u = torch.from_numpy(u).pin_memory()
        out_r = torch.empty_like(pin_r).pin_memory()
        out_u = torch.empty_like(pin_u).pin_memory()
        lbm.lbm_init_equilibrium(sim.h, pin_r, pin_u)
        lbm.lbm_step(sim.h, 1)
        lbm.lbm_get_macro(sim.h, out_r, out_u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            lbm.lbm_init_equilibrium(sim.h, pin_r, pin_u)
            lbm.lbm_step(sim.h, 1)
            lbm.lbm_get_macro(sim.h, out_r, out_u)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        sim.close()

    ms_max, e2e_ms = max_over_ranks([ms, e2e_s * 1e3], world, "cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    glups = job_glups(nodes, args.steps, world, ms_max)
    fluid = int((mask != 1).sum()) if mask is not None else nodes
    per_launch_s = ms / 1e3 / args.steps
    bpn = bytes_per_node(args.dtype, spec["lattice"]) + (4 if mask is not None else 0)
    alg = algorithmic_bytes(nodes, fluid, bpn, 4)
    achieved = alg / per_launch_s / 1e9
    peak, peak_kind = peaks()
    traffic = traffic_for(args.workload, args.dtype, spec["model"], spec["lattice"], nodes)
    line = {
        "metric": "D3Q19 GLUPS & % HBM roofline; FP16/learned vs plain FP32 at fixed error",
        "value": round(glups, 4),
        "unit": "GLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms_max / args.steps, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32s": "f32", "f32": "f32", "f16s": "f32", "bf16s": "f32"}[args.dtype],
        "data": "synthetic (seeded analytic/random initial fields; no dataset)",
        "config": {"workload": spec["name"], "lattice": LATTICE_NAME[spec["lattice"]],
                   "model": {0: "LBGK", 1: "MRT", 2: "ELBM", 3: "REG",
                             4: "SMAG"}[spec["model"]],
                   **({"smagorinsky_cs": 0.1} if spec["model"] == 4 else {}),
                   "storage": args.dtype, "tau": spec["tau"], "nodes": nodes,
                   **({"alpha": args.alpha} if spec["model"] == 2 else {}),
                   **({"mlp_training": args.mlp_kernel} if spec["model"] == 2
                      and args.alpha == "mlp" else {}),
                   **({"rounding": args.round} if args.dtype in ("f16s", "bf16s") else {}),
                   **({"pattern": "AA"} if args.pattern == "aa" else {}),
                   "launch": "cuda_graph" if args.graph else "direct",
                   **({"masked_kernel": args.masked_kernel} if mask is not None else {}),
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "AB working set %.2f GB > 129 MB L2 (inputs larger than L2, no flush)"
                         % (bytes_per_node(args.dtype, spec["lattice"]) * nodes / 1e9)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": peak_kind, "bytes_per_node": round(alg / nodes, 2),
                     **({"algorithmic": "%d fluid nodes x %d B + %d solid nodes x 4 B"
                                        % (fluid, bpn, nodes - fluid)}
                        if mask is not None else {})},
        "e2e": {"value": round(nodes * world / (e2e_ms * 1e-3) / 1e9, 4), "unit": "GLUPS",
                "h2d_bytes_per_step": int(rho.nbytes + u.nbytes),
                "d2h_bytes_per_step": int(rho.nbytes + u.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if mask is not None:
        line["config"]["fluid_nodes"] = fluid
        line["fluid_glups"] = round(job_glups(fluid, args.steps, world, ms_max), 4)
    if elbm_stats:
        line["elbm"] = elbm_stats
        if elbm_cmp:
            line["elbm"].update(elbm_cmp)
        # the entropic kernel is bound by the FP64 pipe (the alpha solve of
        # Eq. alpha_cond runs in FP64): its roofline is that pipe's measured
        # warp-instruction rate, its work the ncu count of FP64-pipe
        # instructions per node; the HBM figures stay beside it
        w_rate, f_rate = lbm.lbm_probe_fp64_rate(stream.cuda_stream)
        ipn = fp64_inst_for(args.alpha, args.dtype, nodes)
        hbm = line["roofline"]
        line["roofline"] = {
            "bound": "fp64", "unit": "G warp-inst/s",
            "achieved": round(ipn * nodes / per_launch_s / 1e9, 3) if ipn else None,
            "peak": round(w_rate / 1e9, 3),
            "frac": round(ipn * nodes / per_launch_s / w_rate, 4) if ipn else None,
            "peak_source": "measured (lbm_probe_fp64_rate: FP64 FMA chains, CUDA events, "
                           "this run)",
            "peak_fp64_tflops": round(f_rate / 1e12, 4),
            "fp64_warp_inst_per_node": ipn, "traffic": None,
            "hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "bytes_per_node")}}
    if diag:
        line["kida"] = diag
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, budget_s=12.0)
        line["cpu_baseline"]["single_thread"] = cpu_baseline(spec, budget_s=6.0, threads=1)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def _oracle_sample(spec, nz_s, ny_s=None):
    import oracle
    from paper_1311_2404_gb300 import workloads as wl
    nx, ny, nz = spec["n"]
    ny_s = ny_s or ny
    model = {0: oracle.BGK, 1: oracle.MRT, 2: oracle.ELBM, 3: oracle.REG,
             4: oracle.SMAG}[spec["model"]]
    p = oracle.make_params(nx, ny_s, nz_s, D={1: 3, 2: 15, 3: 27}[spec["lattice"]], model=model,
                           tau=spec["tau"], force=spec["force"])
    for b in spec.get("bcs", ()):
        oracle.set_bc(p, *b)
    if spec["kind"] == "tg":
        rho, u = wl.taylor_green(nx, 0.05, nz=nz_s, D=3)
        rho, u = rho[:, :ny_s].copy(), u[:, :, :ny_s].copy()
        mask = None
    elif spec["kind"] in ("duct", "ldc"):
        m = wl.duct_with_spheres(nx, ny, nz)[0] if spec["kind"] == "duct" else wl.ldc_mask(nx)
        # interior planes of the cavity (its first plane is a wall)
        z0 = 0 if spec["kind"] == "duct" else min(1, nz - nz_s)
        mask = np.ascontiguousarray(m[z0:z0 + nz_s, :ny_s])
        rho = np.ones((nz_s, ny_s, nx))
        u = np.zeros((3, nz_s, ny_s, nx))
    else:
        r, uu = wl.kida(nx, 0.05) if spec["kind"] == "kida" else wl.turbulence(nx)
        rho = np.ascontiguousarray(r[:nz_s, :ny_s])
        u = np.ascontiguousarray(uu[:, :nz_s, :ny_s])
        mask = None
    F = oracle.init(p, rho, u)
    return p, F, mask, nx * ny_s * nz_s


def cpu_baseline(spec, budget_s=12.0, steps=None, threads=0):
    import oracle
    oracle.build()
    cores = oracle.max_threads(threads)
    # pilot step on a slab deep enough to keep every thread busy (the oracle
    # parallelises over z), then as many steps as fit the budget
    nz_s = min(spec["n"][2], max(4 * cores, 32))
    p, F, mask, n = _oracle_sample(spec, nz_s)
    p.nthreads = threads
    t0 = time.perf_counter()
    oracle.run(p, F, 1, mask)
    dt1 = time.perf_counter() - t0
    p, F, mask, n = _oracle_sample(spec, nz_s)
    p.nthreads = threads
    nsteps = max(1, min(400, int(budget_s / max(dt1, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(p, F, nsteps, mask)
    dt = time.perf_counter() - t0
    return {"value": round(n * nsteps / dt / 1e9, 6), "unit": "GLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"{spec['n'][0]}x{spec['n'][1]}x{nz_s} slab of the workload, "
                      f"{nsteps} steps, FP64 C oracle, {dt:.1f} s"}


def batch_cpu_baseline(specs, budget_s=10.0):
    """The FP64 oracle on a sample of the ensemble's channels, one after the
    other, each for a few steps."""
    import oracle
    from paper_1311_2404_gb300 import workloads as wl
    oracle.build()
    cores = oracle.max_threads(0)
    done, t_used, nsamp = 0, 0.0, 0
    for sp in specs:
        p = oracle.make_params(sp["nx"], sp["ny"], 1, D=2, model=oracle.BGK, tau=sp["tau"],
                               force=(sp["gx"], 0.0, 0.0))
        rho = np.ones((1, sp["ny"], sp["nx"]))
        u = np.zeros((2, 1, sp["ny"], sp["nx"]))
        F = oracle.init(p, rho, u)
        t0 = time.perf_counter()
        oracle.run(p, F, 10, wl.batch_channel_mask(sp))
        t_used += time.perf_counter() - t0
        done += sp["nx"] * sp["ny"] * 10
        nsamp += 1
        if t_used > budget_s:
            break
    return {"value": round(done / t_used / 1e9, 6), "unit": "GLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"first {nsamp} of {len(specs)} channels, 10 steps each, FP64 C oracle, "
                      f"{t_used:.1f} s"}


def _blas_threads():
    """Threads numpy's BLAS uses (the oracle's matrix products), else the
    host's cores."""
    try:
        from threadpoolctl import threadpool_info
        n = sum(int(p.get("num_threads", 0)) for p in threadpool_info()
                if p.get("user_api") == "blas")
        if n > 0:
            return n
    except ImportError:
        pass
    return os.cpu_count() or 1


def run_reference_mlp(args):
    """The FP64 oracle's minibatch Adam (loss_and_grad, adam_step) on a
    sample of the synthetic pairs, timed on the host."""
    import oracle.mlp_oracle as mo
    from paper_1311_2404_gb300 import workloads as wl
    from paper_1311_2404_gb300.alpha_training import init_params, series2
    n = 1 << 16
    X, alpha = wl.mlp_pairs(n)
    Xr = X.astype(np.float64)
    scale = float(np.std(alpha - series2(Xr)))
    P = init_params(13, X.mean(0), 1.0 / (X.std(0) + 1e-12), scale).astype(np.float64)
    t = mo.target(P, Xr, alpha)
    B = min(args.mlp_batch, n)
    m = np.zeros(mo.NPARAM)
    v = np.zeros(mo.NPARAM)
    k = 0
    steps = max(args.steps, 1) + max(args.warmup, 0)
    t0 = time.perf_counter()
    for _ in range(steps):
        off = (k * B) % (n - B + 1)
        _, g = mo.loss_and_grad(P, Xr[off:off + B], t[off:off + B])
        k += 1
        P, m, v = mo.adam_step(P, g, m, v, k, lr=2e-3)
    el = time.perf_counter() - t0
    sps = steps * B / el
    print(json.dumps({
        "impl": "reference", "metric": "alpha-surrogate training throughput (minibatch Adam on the GPU)",
        "value": round(sps, 1), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(el / steps * 1e3, 3),
        "higher_is_better": True, "dtype": "f64", "data": "synthetic (seeded features and alpha)",
        "config": {"workload": "mlp_8_32_32_1_train_%d_pairs" % (1 << 20), "batch": B},
        "cpu_baseline": {"value": round(sps, 1), "unit": "samples/s", "cores": _blas_threads(),
                         "kind": "oracle", "sample": "%d minibatches of %d from %d pairs" % (steps, B, n)},
        "e2e": {"value": round(sps, 1), "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "mlp":
        run_reference_mlp(args)
        return
    spec = workload_spec(args.workload, args.dtype, args.size, args.model, args.lattice, args.shape)
    import oracle
    oracle.build()
    cores = oracle.max_threads(0)
    # per-step sample sized so warmup + steps finish in about two minutes; the
    # pilot slab keeps every oracle thread busy (it parallelises over z)
    nz_p = min(spec["n"][2], max(4 * cores, 32))
    p1, F1, m1, n1 = _oracle_sample(spec, nz_p)
    t0 = time.perf_counter()
    oracle.run(p1, F1, 1, m1)
    plane_s = (time.perf_counter() - t0) / nz_p
    total_steps = max(args.steps, 1) + max(args.warmup, 0)
    per_step_budget = 120.0 / total_steps
    if per_step_budget >= plane_s:
        nz_s, ny_s = max(1, min(spec["n"][2], int(per_step_budget / plane_s))), None
    else:
        nz_s, ny_s = 1, max(2, int(spec["n"][1] * per_step_budget / plane_s))
    p, F, mask, n = _oracle_sample(spec, nz_s, ny_s)
    if args.warmup > 0:
        oracle.run(p, F, args.warmup, mask)
    t0 = time.perf_counter()
    oracle.run(p, F, args.steps, mask)
    dt = time.perf_counter() - t0
    glups = n * args.steps / dt / 1e9
    sample = (f"{spec['n'][0]}x{ny_s or spec['n'][1]}x{nz_s} slab of the workload per step, "
              f"FP64 C oracle")
    line = {
        "impl": "reference",
        "metric": "D3Q19 GLUPS & % HBM roofline; FP16/learned vs plain FP32 at fixed error",
        "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded analytic/random initial fields; no dataset)",
        "config": {"workload": spec["name"], "lattice": LATTICE_NAME[spec["lattice"]],
                   "model": {0: "LBGK", 1: "MRT", 2: "ELBM", 3: "REG",
                             4: "SMAG"}[spec["model"]],
                   **({"smagorinsky_cs": 0.1} if spec["model"] == 4 else {}),
                   "storage": "f64 (oracle)", "tau": spec["tau"],
                   "nodes": spec["n"][0] * spec["n"][1] * spec["n"][2]},
        "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """512 uneven D2Q9 LBGK channels with a cylinder, one persistent
    cooperative launch per bench call of K steps (CUDA graph), autotuned."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1311_2404_gb300 import lbm
    from paper_1311_2404_gb300 import workloads as wl
    dt = {"f32s": lbm.LBM_F32S, "f16s": lbm.LBM_F16S}.get(args.dtype, lbm.LBM_F32S)
    specs = wl.batch_channel_specs(args.ndom)
    stream = torch.cuda.Stream()
    b = lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                             [s["tau"] for s in specs], dt)
    lbm.lbm_batch_set_stream(b, stream.cuda_stream)
    lbm.lbm_batch_set_rounding(b, lbm.LBM_ROUND_NEAREST if args.round == "nearest"
                               else lbm.LBM_ROUND_DITHER)
    rho_bytes = 0
    fluid = 0
    for d, sp in enumerate(specs):
        bm = wl.batch_channel_mask(sp)
        fluid += int((bm == 0).sum())
        lbm.lbm_batch_set_geometry(b, d, bm)
        lbm.lbm_batch_set_force(b, d, sp["gx"], 0.0)
        r = np.ones((1, sp["ny"], sp["nx"]), dtype=np.float32)
        u = np.zeros((2, 1, sp["ny"], sp["nx"]), dtype=np.float32)
        lbm.lbm_batch_init_equilibrium(b, d, r, u)
        rho_bytes += r.nbytes
    nodes = lbm.lbm_batch_nodes(b)
    if args.batch_config:
        lbm.lbm_batch_set_config(b, [int(v) for v in args.batch_config.split(",")])
    else:
        lbm.lbm_batch_autotune(b)
    cfg = lbm.lbm_batch_get_config(b)
    lbm.lbm_batch_step(b, max(args.warmup, 3))
    lbm.lbm_batch_sync(b)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = lbm.lbm_batch_launch_count(b)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lbm.lbm_batch_step(b, args.steps)                    # one persistent launch
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = lbm.lbm_batch_launch_count(b) - l0
    clocks = sampler.stop() if sampler else None
    lbm.lbm_batch_sync(b)
    # end to end: every domain's rho, u from pinned host memory, one step, every
    # domain's rho, v back to pinned host memory
    pins = []
    for sp in specs:
        r = torch.ones((1, sp["ny"], sp["nx"]), dtype=torch.float32).pin_memory()
        u = torch.zeros((2, 1, sp["ny"], sp["nx"]), dtype=torch.float32).pin_memory()
        pins.append((r, u, torch.empty_like(r).pin_memory(), torch.empty_like(u).pin_memory()))
    e2e_steps = max(1, min(args.e2e_steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for d, (r, u, _, _) in enumerate(pins):
            lbm.lbm_batch_init_equilibrium(b, d, r, u)
        lbm.lbm_batch_step(b, 1)
        for d, (_, _, ro, uo) in enumerate(pins):
            lbm.lbm_batch_get_macro(b, d, ro, uo)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    io_bytes = sum(int(r.numel() + u.numel()) * 4 for r, u, _, _ in pins)
    lbm.lbm_batch_destroy(b)
    ms_max, = max_over_ranks([ms], world, "cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    glups = job_glups(nodes, args.steps, world, ms_max)
    bpn = (72 if dt == lbm.LBM_F32S else 36) + 1
    alg = algorithmic_bytes(nodes, fluid, bpn, 1)
    achieved = alg / (ms / 1e3 / args.steps) / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": "D3Q19 GLUPS & % HBM roofline; FP16/learned vs plain FP32 at fixed error",
        "value": round(glups, 4), "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms_max / args.steps, 6),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded channel geometries; no dataset)",
        "config": {"workload": f"d2q9_lbgk_batched_channels_{args.ndom}", "lattice": "D2Q9",
                   "model": "LBGK", "storage": args.dtype if args.dtype in ("f32s", "f16s") else "f32s",
                   "domains": args.ndom, "nodes": nodes, "launch": [int(x) for x in cfg],
                   "parallelism": "single" if world == 1 else f"replicas{world}",
                   "l2": "working set %.1f GB > 129 MB L2" % (bpn * nodes / 1e9)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "bytes_per_node": round(alg / nodes, 2),
                     "algorithmic": "%d fluid nodes x %d B + %d solid nodes x 1 B"
                                    % (fluid, bpn, nodes - fluid)},
        "fluid_glups": round(job_glups(fluid, args.steps, world, ms_max), 4),
        "e2e": {"value": round(nodes * world / e2e_s / 1e9, 4), "unit": "GLUPS",
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    line["config"]["fluid_nodes"] = fluid
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(specs, budget_s=10.0)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# forward and backward multiply-adds of one sample through the 8-32-32-1
# surrogate: forward 8*32 + 32*32 + 32, backward D2 W2 (32*32), dW2
# (32*32), dW1 (32*8), dW3 (32)
MLP_FLOP_PER_SAMPLE = 2 * (8 * 32 + 32 * 32 + 32 + 32 * 32 + 32 * 32 + 32 * 8 + 32)


def run_mlp(args):
    """Training throughput of the alpha surrogate (minibatch Adam, all on the
    GPU) on 2^20 synthetic pairs: K epochs after W warm-up epochs, both
    kernels timed; the line reports the chosen one (--mlp-kernel)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1311_2404_gb300 import lbm
    from paper_1311_2404_gb300 import workloads as wl
    from paper_1311_2404_gb300.alpha_training import init_params, series2
    X, alpha = wl.mlp_pairs()
    n = len(alpha)
    Xd = torch.from_numpy(X).cuda()
    ad = torch.from_numpy(alpha).cuda()
    scale = float(np.std(alpha - series2(X.astype(np.float64))))
    P0 = init_params(13, X.mean(0), 1.0 / (X.std(0) + 1e-12), scale)
    kern = {"tc": lbm.LBM_MLP_BF16_TC, "fp32": lbm.LBM_MLP_FP32}
    res = {}
    steps, warm = max(1, args.steps), max(3, args.warmup)
    sampler = ClockSampler(0)
    for name in ("fp32", "tc") if args.mlp_kernel == "tc" else ("tc", "fp32"):
        P = P0.copy()
        loss = np.zeros(warm, dtype=np.float32)
        lbm.lbm_mlp_train_cfg(Xd, ad, n, warm, args.mlp_batch, 2e-3, 1, kern[name], P, loss)
        P = P0.copy()
        loss = np.zeros(steps, dtype=np.float32)
        if name == args.mlp_kernel:
            sampler.start()
        st = lbm.lbm_mlp_train_cfg(Xd, ad, n, steps, args.mlp_batch, 2e-3, 1, kern[name], P,
                                   loss)
        if name == args.mlp_kernel:
            clocks = sampler.stop()
        res[name] = (st, float(loss[-1]))
    # end to end: the pairs from pinned host memory, the trained parameters back
    Xh = torch.from_numpy(X).pin_memory()
    ah = torch.from_numpy(alpha).pin_memory()
    P = P0.copy()
    loss = np.zeros(1, dtype=np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xe = Xh.cuda(non_blocking=True)
    ae = ah.cuda(non_blocking=True)
    st_e = lbm.lbm_mlp_train_cfg(Xe, ae, n, 1, args.mlp_batch, 2e-3, 1, kern[args.mlp_kernel], P,
                                 loss)
    e2e_s = time.perf_counter() - t0
    st, final = res[args.mlp_kernel]
    sps = st["samples_per_s"]
    peak, _ = peaks()
    bf16_peak = None
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            bf16_peak = float(json.load(fh).get("bf16_tflops", 0.0)) or None
    achieved = sps * MLP_FLOP_PER_SAMPLE / 1e12
    line = {
        "metric": "alpha-surrogate training throughput (minibatch Adam on the GPU)",
        "value": round(sps, 1), "unit": "samples/s", "n_gpus": 1, "steps": steps,
        "warmup": warm, "ms_per_step": round(st["gpu_ms"] / st["steps"], 6),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if args.mlp_kernel == "tc" else "f32",
        "data": "synthetic (seeded features and alpha; no dataset)",
        "config": {"workload": "mlp_8_32_32_1_train_%d_pairs" % n, "batch": args.mlp_batch,
                   "epochs": steps, "kernel": args.mlp_kernel,
                   "l2": "pairs %.1f MB, resident" % ((X.nbytes + alpha.nbytes) / 1e6)},
        "roofline": {"bound": "tensor", "achieved": round(achieved, 3),
                     "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": round(achieved / bf16_peak, 6) if bf16_peak else None,
                     "traffic": None, "flop_per_sample": MLP_FLOP_PER_SAMPLE,
                     "peak_source": "measured bf16 (cuBLAS, burst)" if bf16_peak else None},
        "e2e": {"value": round(n / e2e_s, 1), "unit": "samples/s",
                "h2d_bytes_per_step": int(X.nbytes + alpha.nbytes),
                "d2h_bytes_per_step": int(P.nbytes)},
        "gpu_launches": int(st["steps"] * 3),
        "clocks": clocks,
        "final_loss": final,
        "compare": {k: {"samples_per_s": round(v[0]["samples_per_s"], 1), "final_loss": v[1]}
                    for k, v in res.items()},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.decomp == "slab":
        run_slabs(args)
    elif args.subdomains > 0:
        run_multi(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "mlp":
        run_mlp(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
