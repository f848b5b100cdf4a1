#!/usr/bin/env python
"""Benchmark of fast WQ/DWQ formation (arXiv 2211.06427) on one GB300 per rank.

Workload (default): the degree-4, 64^3-element gyroid mesh (sin6x cos6y + sin6y cos6z +
sin6z cos6x < 0.3 in [0,1]^3) with a log-normal B-spline coefficient field, Laplace
stiffness, octree depth 3.  One step = the whole hot path for that mesh: weight tables
(WQ and DWQ), classification and CSR pattern, coefficient at the quadrature points,
interior rows, cut-element matrices and cut rows.  Metric: nonzeros formed per second.

Multi-GPU: the path is formed per mesh, so N ranks run N independent replicas (weak
scaling, no collective on the data path); `value` = nnz of all replicas / max time.
`--impl reference` times the CPU oracle on a bounded row sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2211_06427_gb300 import synthetic  # noqa: E402

METRIC = "nonzeros formed/s vs plain FP64 GPU path, p=2..6, at stated error; % roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sfa", choices=["sfa", "reference"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--n-el", type=int, default=64)
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "fp32_m64", "tf32", "tf32x3"])
    ap.add_argument("--op", default="stiffness", choices=["mass", "stiffness"])
    ap.add_argument("--geometry", default="gyroid", choices=["gyroid", "full"])
    ap.add_argument("--batch-c5", action="store_true",
                    help="time the 64-mesh batch (one graph launch) against one FP64 call per mesh")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-ref", action="store_true", help="skip the FP64 GPU comparison steps")
    ap.add_argument("--sample-rows", type=int, default=12, help="rows per oracle sample")
    return ap.parse_args()


def workload(args):
    if args.geometry == "gyroid":
        return synthetic.c3_gyroid_64(args.p, n_el=args.n_el)
    return synthetic.c3_full_64(args.p, n_el=args.n_el)


def workload_name(args):
    g = "gyroid" if args.geometry == "gyroid" else "full cube"
    return f"{g} {args.n_el}^3, p={args.p}, {args.op}, log-normal B-spline c, octree depth 3"


# ------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------
def oracle_sample(desc, op, nrows, seed=0, om=None):
    """Time the CPU oracle (row-wise O2) on a bounded, mixed sample of rows.
    Returns (nnz formed, seconds, description)."""
    from oracle.formation import OracleMesh
    if om is None:
        om = OracleMesh(desc)
    g = om.geo
    rng = np.random.default_rng(seed)
    ints = np.nonzero(g.fclass == 1)[0]
    cuts = np.nonzero(g.fclass == 2)[0]
    frac_int = len(ints) / max(1, len(ints) + len(cuts))
    ni = int(round(nrows * frac_int))
    rows = list(rng.choice(ints, min(ni, len(ints)), replace=False)) + \
        list(rng.choice(cuts, min(nrows - ni, len(cuts)), replace=False))
    t0 = time.perf_counter()
    out = om.form_o2(op, rows)
    dt = time.perf_counter() - t0
    nnz = int(sum(len(v) for v in out.values()))
    return nnz, dt, om, f"oracle O2 rows: {len(rows)} sampled ({min(ni, len(ints))} interior, " \
                        f"{len(rows) - min(ni, len(ints))} cut, mesh proportions), oracle geometry built once, untimed"


def cpu_cores_used():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return 1


def run_reference(args):
    """The CPU oracle as it stands, timed on bounded row samples of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    desc = workload(args)
    om = None
    for w in range(max(1, args.warmup)):
        _, _, om, _ = oracle_sample(desc, args.op, max(2, args.sample_rows // 4), seed=100 + w, om=om)
    tot_nnz, tot_t, sample = 0, 0.0, ""
    for s in range(args.steps):
        nnz, dt, om, sample = oracle_sample(desc, args.op, args.sample_rows, seed=s, om=om)
        tot_nnz += nnz
        tot_t += dt
    value = tot_nnz / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "p": args.p, "n_el": args.n_el, "op": args.op},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": cpu_cores_used(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
def cpu_baseline_leg(args):
    """Oracle on this host in a child process pinned to one BLAS thread (bounded sample)."""
    code = ("import json,sys; sys.path.insert(0, %r); import bench, argparse; "
            "a=argparse.Namespace(**json.loads(sys.argv[1])); d=bench.workload(a); "
            "nnz,dt,om,s=bench.oracle_sample(d,a.op,a.sample_rows,seed=7); "
            "print(json.dumps({'nnz':nnz,'dt':dt,'sample':s}))") % ROOT
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, "-c", code, json.dumps(vars(args))], capture_output=True, text=True,
                           env=env, timeout=900)
        res = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": res["nnz"] / res["dt"], "unit": "nnz/s", "cores": 1, "kind": "oracle",
                "sample": res["sample"] + f"; {res['nnz']} nnz in {res['dt']:.1f} s"}
    except Exception as e:  # reported, never silently replaced
        return {"value": None, "unit": "nnz/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}


def algorithmic_interior_bytes(mesh, prec):
    return mesh.info["nnz_interior"] * (8 if prec == "fp64" else 4)


# DRAM bytes (read + write) per unit of work of a kernel, from one ncu capture of the same
# kernel build on a smaller case of the same workload (committed summaries under profiles/):
# kernel -> ((p, op, precision) it was taken on, bytes per unit, unit counter, source).
# Traffic grows with the units processed, so a full launch is the per-unit figure times its
# units.  Other shapes report null.
DRAM_PER_UNIT = {
    "k_cut_elemmat": ((4, "stiffness", "fp32"), (5.64e6 + 563.94e6) / 10681, "n_cut_elements",
                      "profiles/cut_kernels_gyroid48_p4_stiffness_fp32.md"),
    "k_cut_rows": ((4, "stiffness", "fp32"), (795.49e6 + 130.30e6) / 59801, "n_cut_rows",
                   "profiles/cut_kernels_gyroid48_p4_stiffness_fp32.md"),
    "k_interior_tc3": ((4, "stiffness", "tf32"), (10.79e6 + 299.73e6) / 89915392, "nnz_interior",
                       "profiles/interior_tc_full48_p4_stiffness_tf32.md"),
}


def nnz_interior(mesh):
    return mesh.info["nnz_interior"]


def dram_traffic(kernel, args, info, units):
    shape, per_unit, counter, _src = DRAM_PER_UNIT[kernel]
    if (args.p, args.op, args.prec) != shape:
        return None
    n = units if units is not None else info[counter]
    return per_unit * n


def elemmat_flops(p, stiff, n_pieces, n_cut, bspline_coef):
    """Algorithmic FLOPs of one cut-element-matrix launch: per octree piece the three
    sum-factorised moment stages NB Q^3 + NB^2 Q^2 + NB^3 Q MAC (plus 3 Q^4 MAC for a
    B-spline coefficient and 3 Q^3 multiplies for the weights), per cut element the E stage
    Q^2 NB^3 + Q^4 NB^2 + Q^6 NB MAC (mass) or 2 Q^2 NB^3 + 3 Q^4 NB^2 + 2 Q^6 NB (stiffness);
    Q = p + 1 Gauss points per direction, NB = 2p + 1 Bernstein moments per direction."""
    q, nb = p + 1, 2 * p + 1
    piece = nb * q ** 3 + nb * nb * q * q + nb ** 3 * q + (3 * q ** 4 if bspline_coef else 0)
    if stiff:
        elem = 2 * q * q * nb ** 3 + 3 * q ** 4 * nb * nb + 2 * q ** 6 * nb
    else:
        elem = q * q * nb ** 3 + q ** 4 * nb * nb + q ** 6 * nb
    return 2.0 * (n_pieces * piece + n_cut * elem) + 3.0 * q ** 3 * n_pieces


def cutrows_flops(p, stiff, info):
    """Algorithmic FLOPs of one cut-row launch from the classification's work counts: per
    (row, inside element outside the box) three sum-factorised Gauss stages, 7 Q^4 MAC for
    stiffness (3 Q^4 mass); per (row, cut element) Q^3 additions of an element-matrix row; per
    DWQ box NB NT m_f m_s m_t + NB^2 c2 m_s m_t + NB^3 c3 m_t MAC (NT = 2, c2 = 3, c3 = 2 for
    stiffness, 1 each for mass)."""
    q, nb = p + 1, 2 * p + 1
    nt, c2, c3 = (2, 3, 2) if stiff else (1, 1, 1)
    mac = ((7 if stiff else 3) * q ** 4 * info["cut_gauss_pairs"] + nb * nt * info["box_points_fst"] +
           nb * nb * c2 * info["box_points_st"] + nb ** 3 * c3 * info["box_points_t"])
    return 2.0 * mac + q ** 3 * info["cut_elem_pairs"]


# Non-tensor arithmetic peaks from unit counts and the maximum SM clock (2070 MHz):
# 152 SMs x 128 FP32 lanes x 2 FLOP per FMA; FP64 at the nominal 1.25 TFLOP/s.
SM_COUNT, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25


def run_c5(args):
    """64 independent meshes (n_el ~ U{8..48}, p ~ U{2..5}, 1-8 balls, analytic c): the whole
    batch formed by one graph launch (tiles autotuned per degree) against one call per mesh
    in FP64 and in the batch's precision.  Setup (tables, classification) is untimed."""
    import torch
    from paper_2211_06427_gb300 import sfa
    torch.cuda.set_device(0)
    descs = synthetic.c5_batch()
    meshes = [sfa.Mesh(d) for d in descs]
    nnz = sum(m.nnz for m in meshes)
    stream = torch.cuda.current_stream()
    prec = args.prec if args.prec != "fp64" else "fp32"
    tuned = {}
    for m, d in zip(meshes, descs):
        if (d["p"], prec) not in tuned:
            m.autotune(args.op, prec)
            tuned[(d["p"], prec)] = sfa.get_tuning(d["p"], args.op, prec)
    vdt = torch.float32
    outs = [torch.empty(max(m.nnz, 1), dtype=vdt, device="cuda") for m in meshes]
    outs64 = [torch.empty(max(m.nnz, 1), dtype=torch.float64, device="cuda") for m in meshes]

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))
    t_batch = timed(lambda: sfa.form_batched(meshes, args.op, prec, outs=outs), args.steps)
    t_single = timed(lambda: [m.form(args.op, prec, out=o) for m, o in zip(meshes, outs)], args.steps)
    t_fp64 = timed(lambda: [m.form(args.op, "fp64", out=o) for m, o in zip(meshes, outs64)], max(1, args.steps // 2))
    line = {"metric": "nonzeros formed/s, 64-mesh batch", "value": nnz / (t_batch / 1000.0), "unit": "nnz/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch,
            "higher_is_better": True, "dtype": {"fp32": "f32", "fp32_m64": "f32+f64", "tf32": "tf32",
                                               "tf32x3": "tf32x3"}[prec], "data": "synthetic",
            "config": {"workload": "C5: 64 meshes, n_el ~ U{8..48}, p ~ U{2..5}, 1-8 balls, analytic c, depth 3",
                       "op": args.op, "precision": prec, "nnz": nnz,
                       "tuning": {f"p={p}": list(v) for (p, _), v in sorted(tuned.items())}},
            "one_call_per_mesh_ms": t_single, "fp64_one_call_per_mesh_ms": t_fp64,
            "speedup_vs_fp64_per_mesh": t_fp64 / t_batch, "speedup_vs_same_precision_per_mesh": t_single / t_batch}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.batch_c5:
        run_c5(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2211_06427_gb300 import sfa

    desc = workload(args)
    stream = torch.cuda.current_stream()
    mesh = sfa.Mesh(desc, setup=False)

    # the weight tables and the classification are independent: the tables go on a second
    # stream while the classification (which synchronises its own stream) runs on the main one
    side = torch.cuda.Stream()

    def setup():
        side.wait_stream(stream)
        mesh.build_tables(stream=side)
        mesh.classify(stream=stream)
        stream.wait_stream(side)

    def step(vals):
        setup()
        return mesh.form(args.op, args.prec, out=vals)

    # first pass sizes the value buffer
    mesh.build_tables()
    mesh.classify()
    vdtype = torch.float64 if args.prec == "fp64" else torch.float32
    vals = torch.empty(max(1, mesh.nnz), dtype=vdtype, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    for _ in range(args.warmup):
        step(vals)
    torch.cuda.synchronize()
    nnz = mesh.nnz
    info = mesh.info

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_acc = np.zeros(7)
    launches0 = sfa.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between steps (untimed)
            ev[k][0].record(stream)
            step(vals)
            ev[k][1].record(stream)
            stage_acc += np.array(mesh.stage_ms())
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = (sfa.launch_count() - launches0) // args.steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    stages = (stage_acc / args.steps).tolist()
    value = world * nnz / (ms / 1000.0)

    # the plain FP64 GPU path on the same mesh (the metric's comparison), a few steps
    fp64_ref = None
    if args.prec != "fp64" and not args.no_fp64_ref:
        vals64 = torch.empty(max(1, nnz), dtype=torch.float64, device="cuda")

        def step64():
            setup()
            mesh.form(args.op, "fp64", out=vals64)
        step64()
        k64 = max(1, min(args.steps, 3))
        e64 = []
        for k in range(k64):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step64()
            b.record(stream)
            torch.cuda.synchronize()
            e64.append(a.elapsed_time(b))
        m64 = float(np.mean(e64))
        fp64_ref = {"ms_per_step": m64, "value": nnz / (m64 / 1000.0), "unit": "nnz/s", "steps": k64}
        del vals64

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        coef_h = torch.as_tensor(desc["coef_bspline"]).pin_memory() if desc["coef"] == "bspline" else None
        vals_h = torch.empty(nnz, dtype=vdtype).pin_memory()
        for _ in range(2):
            setup()
            mesh.form_host(args.op, args.prec, coef_h, vals_h)
        e_ms = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            setup()
            mesh.form_host(args.op, args.prec, coef_h, vals_h)
            b.record(stream)
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
        em = float(np.mean(e_ms))
        if dist:
            t = torch.tensor([em], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            em = float(t.item())
        e2e = {"value": world * nnz / (em / 1000.0), "unit": "nnz/s",
               "h2d_bytes_per_step": int(coef_h.numel() * 8) if coef_h is not None else 0,
               "d2h_bytes_per_step": int(nnz * vals_h.element_size()), "ms_per_step": em}

    # roofline of the interior-row kernel (the HBM-bound CSR value stream)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    stage_names = ["tables", "classification", "coefficient", "interior_rows", "cut_element_matrices", "cut_rows",
                   "backward"]
    stage_ms = {n: v for n, v in zip(stage_names, stages) if v >= 0}
    t_int = stage_ms.get("interior_rows", -1)
    roof_int = None
    if t_int and t_int > 0:
        byt = algorithmic_interior_bytes(mesh, args.prec)
        ach = byt / (t_int / 1000.0) / 1e9
        kern = ("k_interior_tc3" if args.prec in ("tf32", "tf32x3")
                else "k_interior_reg + k_interior")
        roof_int = {"bound": "hbm", "kernel": kern + " (interior-row stage)", "achieved": ach, "peak": hbm_peak,
                    "unit": "GB/s", "frac": ach / hbm_peak, "peak_source": peak_src + " hbm_gbs",
                    "traffic": dram_traffic("k_interior_tc3", args, info, nnz_interior(mesh))
                    if args.prec == "tf32" else None,
                    "algorithmic_bytes_per_launch": byt}
    # the dominant kernel of the step (one launch each per step): cut-element matrices or cut
    # rows (ALU-bound), else the interior-row stage (HBM)
    t_em = stage_ms.get("cut_element_matrices", -1)
    t_cr = stage_ms.get("cut_rows", -1)
    roof = roof_int
    stiff = args.op == "stiffness"
    fp32_src = "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    if t_em > 0 and t_em >= max(t_int, t_cr):
        flops = elemmat_flops(args.p, stiff, info["n_pieces"], info["n_cut_elements"], True)
        ach = flops / (t_em / 1000.0) / 1e12
        f64 = args.prec in ("fp64", "fp32_m64")  # moments accumulated in double
        peak = FP64_PEAK_TFLOPS if f64 else FP32_PEAK_TFLOPS
        roof = {"bound": "alu", "kernel": "k_cut_elemmat", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": "FP64 nominal 1.25 TFLOP/s" if f64 else fp32_src,
                "traffic": dram_traffic("k_cut_elemmat", args, info, None),
                "algorithmic_flops_per_launch": flops,
                "flop_model": "per-piece sum factorisation (the kernel groups pieces and does fewer)"}
    elif t_cr > 0 and t_cr >= t_int:
        flops = cutrows_flops(args.p, stiff, info)
        ach = flops / (t_cr / 1000.0) / 1e12
        peak = FP64_PEAK_TFLOPS if args.prec == "fp64" else FP32_PEAK_TFLOPS
        roof = {"bound": "alu", "kernel": "k_cut_rows", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": "FP64 nominal 1.25 TFLOP/s" if args.prec == "fp64" else fp32_src,
                "traffic": dram_traffic("k_cut_rows", args, info, None), "algorithmic_flops_per_launch": flops}

    clocks = clk.summary()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp32_m64": "f32+f64", "tf32": "tf32", "tf32x3": "tf32x3"}[args.prec],
            "data": "synthetic",
            "config": {"workload": workload_name(args), "p": args.p, "n_el": args.n_el, "op": args.op,
                       "precision": args.prec, "nnz": nnz, "interior_rows": info["n_interior_rows"],
                       "cut_rows": info["n_cut_rows"], "box_rows": info["n_box_rows"],
                       "cut_elements": info["n_cut_elements"], "pieces": info["n_pieces"],
                       "l2": "flushed between steps (256 MiB write, outside the timed events)",
                       "parallelism": f"replicas{world}",
                       "step": "tables (second stream) + classification + pattern + formation"},
            "stages_ms": stage_ms,
            "formation_nnz_per_s": nnz / (sum(stage_ms.get(k, 0) for k in
                                              ("coefficient", "interior_rows", "cut_element_matrices",
                                               "cut_rows")) / 1000.0),
            "fp64_gpu": fp64_ref,
            "speedup_vs_fp64_gpu": (value / world / fp64_ref["value"]) if fp64_ref else None,
            "roofline": roof, "roofline_interior": roof_int, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
