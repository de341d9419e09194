#!/usr/bin/env python
"""Benchmark: Lanczos-quadrature RPA correlation energy on the 64-atom Si-like cell.

Metric: probe-points per second (one probe-point = the Lanczos quadrature of d_j(i w) at one
coarse grid point and one frequency, run to completion), for the mixed form (FP32
stencil/COCG/projections with FP64 Lanczos, reorthogonalisation, tridiagonal eigen-solve,
refinement residuals and energy sums) next to the plain FP64 form, with the E_c error of the
mixed form against the FP64 form in mHa/atom.

Workload (default "si64"): periodic 2x2x2 diamond-Si-like cell, a = 20.52 bohr, 52^3 grid,
12th-order Laplacian, Gaussian wells plus 4 s/p projectors per atom, 128 occupied states,
10 mapped Gauss-Legendre frequencies, 40 Lanczos steps, coarse stride 2 (17,576 probes,
175,760 probe-points), tricubic interpolation.  Inputs are synthetic and seeded (synth/).

A step = one pass of the whole path over one batch: a seeded sample of probe-points spread
over all frequencies (u = nu^{1/2} q, Galerkin projection, COCG, density, nu^{1/2}, Lanczos
with reorthogonalisation, [f(T)]_11), then interpolation of the coarse array to the fine
grid and the E_c sum.  Inputs (~2 GB of COCG vectors per batch) exceed the 126 MB L2, so no
flush is needed between steps.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: system, frequencies, Lanczos steps, stride, interpolation, Sternheimer tol, atoms
    "si64": dict(system="si64", nw=10, nl=40, stride=(2, 2, 2), interp="cubic", tol=1e-4,
                 natom=64, desc="64-atom Si-like cell, 52^3 grid, 128 occupied states, 10 "
                 "frequencies, 40 Lanczos steps, coarse stride 2, tricubic"),
    "si8": dict(system="si8", nw=10, nl=40, stride=(2, 2, 2), interp="cubic", tol=1e-4, natom=8,
                desc="8-atom Si-like cell, 26^3 grid, 16 occupied states, 10 frequencies, "
                "40 Lanczos steps, coarse stride 2"),
    "si64p": dict(system="si64p", nw=8, nl=3, stride=(2, 2, 2), interp="cubic", tol=0.1,
                  natom=64, desc="64-atom Si-like cell on a 40^3 grid (h = 0.513 bohr), 128 "
                  "occupied states, 8 frequencies, 3 Lanczos steps, coarse stride 2, Sternheimer "
                  "tol 0.1: the settings of the paper's Si64 scaling run (64,000 probe-points)"),
    "lih32": dict(system="lih32", nw=8, nl=2, stride=(1, 1, 1), interp="none", tol=0.1,
                  natom=64, desc="(LiH)32-like rock-salt cell, 32^3 grid, 64 occupied states, "
                  "8 frequencies, 2 Lanczos steps, no interpolation, Sternheimer tol 0.1 (the "
                  "settings of the paper's LiH scaling runs)"),
    "toy": dict(system="toy", nw=8, nl=20, stride=(2, 2, 2), interp="cubic", tol=1e-4, natom=4,
                desc="toy periodic cube, 12^3 grid, 8 occupied states, 8 frequencies, "
                "20 Lanczos steps, coarse stride 2"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
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
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(smax)),
                    power_w_max=float(max(power)), samples=len(sm), reasons=sorted(reasons))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), src="measured")
    return dict(hbm_gbs=6800.0, src="fallback")


def make_system(name):
    import synth
    return synth.named_system(name)


def sample_probes(P, nw, per_freq, seed):
    rng = np.random.default_rng(seed)
    pr, fq = [], []
    for k in range(nw):
        ps = rng.choice(P, size=per_freq, replace=False)
        pr += list(ps)
        fq += [k] * per_freq
    return np.asarray(pr, dtype=np.int64), np.asarray(fq, dtype=np.int32)


# ------------------------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ------------------------------------------------------------------------------------------
def run_reference(args, wl):
    import oracle
    s = make_system(wl["system"])
    om, w = oracle.gl_frequencies(wl["nw"])
    P = int(np.prod([len(oracle.coarse_nodes(s.n[a], wl["stride"][a], s.bc[a])) for a in range(3)]))
    probes = oracle.coarse_probes(s.n, wl["stride"], s.bc)
    cores = os.cpu_count()
    osys = oracle.OracleSystem(s)
    # Bounded sample: one matrix-vector product (N_s Sternheimer solves) of one seeded coarse
    # point per step, the frequencies taken in turn so that K steps cover all of them
    # evenly; a probe-point costs N_l such products, so probe-pts/s = 1 / (N_l * t_step).
    times = []
    rng = np.random.default_rng(7)
    for it in range(args.warmup + args.steps):
        j = int(probes[rng.integers(P)])
        k = it % wl["nw"]
        t0 = time.perf_counter()
        oracle.lanczos(osys, np.array([j]), np.array([om[k]]), 1, tol=wl["tol"], maxit=20000,
                       nthreads=cores)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    tstep = float(np.mean(times))
    value = 1.0 / (wl["nl"] * tstep)
    sample = (f"per step: 1 Lanczos matrix-vector product ({s.ns} Sternheimer solves, tol "
              f"{wl['tol']}) of 1 seeded coarse point of the {wl['system']} workload, step i at "
              f"frequency i mod {wl['nw']}; probe-pts/s = 1/(N_l={wl['nl']} x mean step time)")
    line = dict(metric="probe-points/s", value=value, unit="probe-pts/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * tstep,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=wl["system"], desc=wl["desc"], l2="inputs > L2"),
                cpu_baseline=dict(value=value, unit="probe-pts/s", cores=cores, kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit="probe-pts/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def oracle_leg(s, wl, om, pidx, seed=11):
    """The oracle on the host cores, bounded sample: one Lanczos matrix-vector product (N_s
    Sternheimer solves at the workload's tolerance) for one seeded coarse point at every
    frequency.  Gives the CPU baseline (probe-pts/s = 1 / (N_l x mean time of a product)) and
    reference values d = [f(T_1)]_11 for the same (point, frequency) pairs."""
    import oracle
    cores = os.cpu_count()
    rng = np.random.default_rng(seed)
    sel = rng.choice(len(pidx), size=wl["nw"], replace=False)
    probes = np.asarray(pidx[sel], dtype=np.int64)
    osys = oracle.OracleSystem(s)
    times, d = [], []
    for k in range(wl["nw"]):
        t0 = time.perf_counter()
        r = oracle.lanczos(osys, probes[k:k + 1], np.array([om[k]]), 1, tol=wl["tol"],
                           maxit=20000, nthreads=cores)
        times.append(time.perf_counter() - t0)
        d.append(float(r["d"][0]))
    tm = float(np.mean(times))
    cpu = dict(value=1.0 / (wl["nl"] * tm), unit="probe-pts/s", cores=cores, kind="oracle",
               per_core=1.0 / (wl["nl"] * tm * cores),
               sample=(f"1 Lanczos matrix-vector product ({s.ns} Sternheimer solves, tol "
                       f"{wl['tol']}) for one seeded coarse point at each of the {wl['nw']} "
                       f"frequencies; probe-pts/s = 1/(N_l x mean product time {tm:.2f} s); "
                       f"per-frequency times {[round(t, 2) for t in times]} s"))
    return cpu, probes, np.asarray(d)


def oracle_error(R, context, wl, om, w, probes, d_ref, P, nd, natom):
    """The GPU forms on the oracle's (point, frequency) pairs with one Lanczos step each:
    max |d_gpu - d_oracle|, its relative size and the E_c error it implies (one point per
    frequency standing for all P coarse points, weighted, / 2 pi / atoms), in mHa/atom."""
    out = {}
    freqs = np.arange(wl["nw"], dtype=np.int32)
    for form in ("mixed", "fp64"):
        c = context(form, profile=0, nl=1)
        r = R.rpa_probe_density(c.ctx, probes, freqs, allow_nonconv=True)
        dd = np.asarray(r["d"]) - d_ref
        g3 = nd / P
        est = float(np.sum(w * P * dd)) * g3 / (2 * np.pi) / natom
        out[form] = dict(max_abs_dd=float(np.abs(dd).max()),
                         max_rel_dd=float(np.max(np.abs(dd) / np.abs(d_ref))),
                         ec_err_mha_per_atom_est=1e3 * abs(est), status=int(r["status"]))
        c.close()
    out["sample"] = (f"one seeded coarse point per frequency ({wl['nw']} probe-points), one "
                     f"Lanczos step, Sternheimer tol {wl['tol']} on both sides; the oracle is "
                     "the plain CPU FP64 restatement of Algorithm 1")
    return out


def run_ours(args, wl):
    import torch

    import paper_2609_16408_gb300 as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = make_system(wl["system"])
    om, w = R.rpa_gl_frequencies(wl["nw"])
    stream = torch.cuda.Stream(device=dev)
    nd = s.N_d
    nat = wl["natom"]

    mixed_form = "mixed_bf16" if args.proj == "bf16" else "mixed"

    def context(prec, profile=1, tile=-1, nl=None):
        c = R.Context(s.n, s.h, s.bc, s.fd_radius, stream=stream.cuda_stream)
        R.rpa_set_potential(c.ctx, s.vloc)
        R.rpa_set_projectors(c.ctx, [(g.idx, g.chi, g.gamma) for g in s.groups])
        R.rpa_set_occupied(c.ctx, s.psi, s.eps)
        R.rpa_set_frequencies(c.ctx, om, w)
        R.rpa_set_options(c.ctx, lanczos_max=nl or wl["nl"], stern_tol=wl["tol"],
                          stern_maxit=20000, precision=mixed_form if prec == "mixed" else prec,
                          stride=wl["stride"], interp=wl["interp"], refine=args.refine,
                          profile=profile, tile=tile if prec != "fp64" else -1,
                          graphs=args.graphs, inner_tol=args.inner_tol, lanes=args.lanes,
                          lanczos_block=args.lanczos_block if prec != "fp64" else 1)
        return c

    cm = context("mixed", tile=args.tile)
    P = R.rpa_num_probes(cm.ctx)
    probe_idx = torch.from_numpy(R.rpa_probe_indices(cm.ctx)).to(dev)
    dco = torch.zeros((wl["nw"], P), dtype=torch.float64, device=dev)
    statuses = []

    def sample(per_freq, seed):
        """This rank's probe-points of one step: a seeded global sample of world x per_freq
        points per frequency (the same on every rank), partitioned into contiguous blocks by
        the product's sharding rule."""
        from paper_2609_16408_gb300.shard import probe_point_shard
        gsel, gfq = sample_probes(P, wl["nw"], per_freq * world, seed)
        ids, _ = probe_point_shard(len(gsel), 1, rank, world)
        return gsel[ids], gfq[ids]

    def step(c, per_freq, seed, stats_acc=None):
        sel, fq = sample(per_freq, seed)
        pr = probe_idx[torch.from_numpy(sel).to(dev)]
        fqt = torch.from_numpy(fq).to(dev)
        out = R.rpa_probe_density(c.ctx, pr, fqt, allow_nonconv=True)
        statuses.append(int(out["status"]))
        dco[fqt.long(), torch.from_numpy(sel).to(dev)] = out["d"]
        dfi, ec = R.rpa_interpolate(c.ctx, dco, nd)
        if stats_acc is not None:
            stats_acc.append(out["stats"])
        return out, sel, fq

    per = args.probes_per_freq
    seed0 = 1000
    # warm-up
    for i in range(args.warmup):
        with torch.cuda.stream(stream):
            step(cm, per, seed0 + i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    l0 = R.rpa_kernel_launches()
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            step(cm, per, seed0 + 100 + i, stats)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = R.rpa_kernel_launches() - l0
    clk = clocks.stop()
    t = ev0.elapsed_time(ev1) * 1e-3
    if dist:
        tt = torch.tensor([t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    pts_per_rank = args.steps * per * wl["nw"]
    value = world * pts_per_rank / t

    # dominant kernel roofline (CUDA events on the launching stream, inside the timed region)
    ks = np.sum([st["kernel_seconds"] for st in stats], axis=0)
    kb = np.sum([st["kernel_bytes"] for st in stats], axis=0)
    kl = np.sum([st["kernel_launches"] for st in stats], axis=0)
    tile_rows = int(stats[-1].get("tile_rows", 0)) if stats else 0
    tile_tail = int(stats[-1].get("tile_rows_tail", 0)) if stats else 0

    def tiling(t):
        if t <= -101:
            return (f"bands of {-100 - t} full x rows, two x points per thread, 3-stage "
                    "cp.async pipeline")
        if t == -6:
            return "two-point kernel on packed full rows"
        if t in (-3, -4):
            return (f"64 x 8 tiles, two x points per thread, z window in a shared-memory ring, "
                    f"{1 if t == -3 else 2} centre-plane buffer(s)")
        return (f"{t} full x rows per block" if t > 0
                else ("64 x 8 tiles, two x points per thread" if t == -2 else "32 x 8 column tiles"))
    hname = ("k_dirmatvec_band" if tile_rows <= -101
             else "k_dirmatvec_rows" if tile_rows > 0
             else "k_dirmatvec_x2p" if tile_rows == -6
             else ("k_dirmatvec_x2" if tile_rows in (-2, -3, -4) else "k_dirmatvec"))
    names = ["proj_dots", hname, "k_scalars", "k_update_dots", "none"]
    dom = 1 if ks[1] >= ks[3] else 3
    pk = peaks()
    achieved = kb[dom] / ks[dom] / 1e9 if ks[dom] > 0 else 0.0
    # DRAM traffic per launch from the committed ncu capture (dram__bytes_read + write of one
    # launch, divided by the systems active in that launch), scaled to this run's average
    # number of active systems per launch; null once the kernel sources have changed.
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path) and kl[dom] > 0:
        tj = json.load(open(tr_path)).get(names[dom])
        if tj and tj.get("source_sha") == kernel_source_sha(names[dom]):
            alg_per_sys = {1: 4, 3: 6}[dom] * 2 * stats[0]["precision_bytes"] * nd
            sys_per_launch = kb[dom] / alg_per_sys / kl[dom]
            # per-system bytes of the captured grid, scaled to this grid's point count
            scale = nd / tj.get("grid_points", nd)
            traffic = tj["dram_bytes_per_system"] * scale * sys_per_launch
    roofline = dict(bound="hbm", kernel=names[dom], achieved=achieved, peak=pk["hbm_gbs"],
                    unit="GB/s", frac=achieved / pk["hbm_gbs"], traffic=traffic,
                    algorithmic_bytes_per_launch=float(kb[dom] / max(1, kl[dom])),
                    peak_src=pk["src"] + " (burst copy)",
                    launches=int(kl[dom]), seconds=float(ks[dom]),
                    algorithmic_bytes=float(kb[dom]),
                    # share of the sampled COCG kernel time (classes 0-4; slots 5 and 6
                    # split the same time into tail and bulk chunks)
                    cocg_share=float(ks[dom] / max(1e-30, sum(ks[:5]))))

    # FP64 form and mixed form timed on one and the same seeded sample, and the
    # mixed-vs-FP64 error on it
    fp64 = None
    if not args.no_fp64:
        c64 = context("fp64")
        sel, fq = sample(args.fp64_probes_per_freq, seed0 + 7)
        pr = probe_idx[torch.from_numpy(sel).to(dev)]
        fqt = torch.from_numpy(fq).to(dev)

        def timed(c):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                o = R.rpa_probe_density(c.ctx, pr, fqt, allow_nonconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            return o, e0.elapsed_time(e1) * 1e-3
        o64, t64 = timed(c64)
        omx, tmx = timed(cm)
        dd = (omx["d"] - o64["d"]).cpu().numpy()
        g3 = nd / P
        # E_c difference estimated from the sample: per frequency the sampled mean of d_mix -
        # d_fp64 times P (all coarse points), weighted and summed, with its standard error.
        # The interpolated fine sum weights each coarse point by N_d / P on average (exactly
        # g^3 when g divides every periodic axis).
        est, var = 0.0, 0.0
        for k in range(wl["nw"]):
            m = fq == k
            if m.any():
                est += w[k] * P * dd[m].mean()
                if m.sum() > 1:
                    var += (w[k] * P) ** 2 * dd[m].var(ddof=1) / m.sum()
        scale = g3 / (2 * np.pi) / nat
        fp64 = dict(value=world * len(sel) / t64, unit="probe-pts/s",
                    probe_points=int(len(sel)), seconds=t64,
                    mixed_value_same_sample=world * len(sel) / tmx, mixed_seconds=tmx,
                    mixed_speedup=t64 / tmx,
                    sample=(f"{args.fp64_probes_per_freq} seeded coarse points per frequency "
                            "per rank, both forms on the same points"),
                    nonconv_solves=dict(fp64=o64["stats"]["nonconv_solves"],
                                        mixed=omx["stats"]["nonconv_solves"]),
                    ec_diff_mha_per_atom_est=1e3 * abs(est) * scale,
                    ec_diff_mha_per_atom_stderr=(1e3 * np.sqrt(var) * scale
                                                 if args.fp64_probes_per_freq > 1 else None),
                    max_abs_dd=float(np.abs(dd).max()),
                    mean_abs_dd=float(np.abs(dd).mean()))
        c64.close()

    # end to end through the public API with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        vloc_h, psi_h, eps_h = pin(s.vloc), pin(s.psi), pin(s.eps)
        grp = [(pin(g.idx.astype(np.int32)), pin(g.chi), pin(g.gamma)) for g in s.groups]
        h2d = vloc_h.nbytes + psi_h.nbytes + eps_h.nbytes + sum(
            a.nbytes + b.nbytes + c.nbytes for a, b, c in grp)
        dco_h = np.zeros((wl["nw"], P))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            sel, fq = sample(per, seed0 + 500 + i)
            pr_h = R.rpa_probe_indices(cm.ctx)[sel]
            R.rpa_set_potential(cm.ctx, vloc_h)
            R.rpa_set_projectors(cm.ctx, grp)
            R.rpa_set_occupied(cm.ctx, psi_h, eps_h)
            out = R.rpa_probe_density(cm.ctx, pr_h, fq, allow_nonconv=True)
            dco_h[fq, sel] = out["d"]
            dfi_h, ec_h = R.rpa_interpolate(cm.ctx, dco_h, nd)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d_step = h2d + pr_h.nbytes + fq.nbytes + dco_h.nbytes
        d2h_step = out["d"].nbytes + dfi_h.nbytes + 8
        e2e = dict(value=world * args.e2e_steps * len(sel) / te, unit="probe-pts/s",
                   h2d_bytes_per_step=int(h2d_step), d2h_bytes_per_step=int(d2h_step))

    # the oracle on the host cores: CPU baseline and the error of both GPU forms against it
    cpu, oracle_err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, oprobes, d_ref = oracle_leg(s, wl, om, R.rpa_probe_indices(cm.ctx))
        with torch.cuda.stream(stream):
            oracle_err = oracle_error(R, context, wl, om, w, oprobes, d_ref, P, nd, nat)

    st0 = stats[0] if stats else {}
    tot_iters = sum(st["cocg_iters"] for st in stats)
    tot_solves = sum(st["solves"] for st in stats)
    full_pts = P * wl["nw"]
    line = dict(
        metric="probe-points/s", value=value, unit="probe-pts/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * t / args.steps,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32+f64",
        data="synthetic (seeded Si-like cell, synth/)",
        config=dict(workload=wl["system"], desc=wl["desc"], form=mixed_form,
                    projection=("bf16 tcgen05 kind::f16, 1 pass" if args.proj == "bf16"
                                else "tf32x3 tcgen05 kind::tf32"),
                    stride=list(wl["stride"]), interp=wl["interp"],
                    stern_tol=wl["tol"], refine=args.refine, inner_tol=args.inner_tol or "auto",
                    probe_points_per_step=per * wl["nw"] * world, l2="inputs > L2 (no flush)",
                    tile_rows=tile_rows, tile_rows_tail=tile_tail, cuda_graphs={0: "off", 1: "chunks of 4 iterations, host-checked",
                                 2: "whole COCG loops (conditional while nodes)"}[args.graphs],
                    h_apply_tiling=(f"{tiling(tile_rows)} (launches over > 32 systems), "
                                    f"{tiling(tile_tail)} (<= 32 systems)"
                                    + (" autotuned" if args.tile == -1 else " set by --tile")),
                    parallelism=f"probe-points sharded over {world} GPU(s)"),
        roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
        clocks=clk, fp64_form=fp64,
        ec_full_seconds_est=full_pts / value,
        cocg=dict(mean_iters=tot_iters / max(1, tot_solves), solves=tot_solves,
                  max_iters=max(st["max_cocg_iters"] for st in stats) if stats else 0,
                  refine_rounds=sum(st["refine_rounds"] for st in stats),
                  solves_per_s=world * tot_solves / t, iters_per_s=world * tot_iters / t,
                  nonconv_solves=sum(st["nonconv_solves"] for st in stats),
                  breakdown_solves=sum(st["breakdown_solves"] for st in stats),
                  step_statuses=sorted(set(statuses)),
                  # share of the sampled COCG kernel time in chunks whose launches covered
                  # at most 32 systems (the latency-bound tail of the slowest solves)
                  tail_time_fraction=(float(ks[5] / (ks[5] + ks[6]))
                                      if ks[5] + ks[6] > 0 else None),
                  tail_iteration_fraction=(float(kl[5] / (kl[5] + kl[6]))
                                           if kl[5] + kl[6] > 0 else None)),
        oracle_error=oracle_err,
        phases_s=list(np.sum([st["seconds_phase"] for st in stats], axis=0)) if stats else None,
    )
    if rank == 0:
        print(json.dumps(line), flush=True)
    cm.close()
    if dist:
        dist.destroy_process_group()


def run_uneven(args):
    """The uneven batch: Si-like cells of 8, 16 and 32 atoms (26^3, 26x26x52, 26x52x52) and
    the 12-atom Dirichlet cluster (40^3), mixed form, Lanczos early exit at 1e-6 relative
    change (up to 40 steps), Sternheimer tol 1e-4, each system's full E_c over a coarse set
    of three points per axis (trilinear interpolation) at four frequencies.  Times rpa_batch_energy (every system on its
    own stream and host thread, kernels of the different grids sharing the GPU) against the
    same contexts run one after the other, and prints one JSON line."""
    import time

    import torch

    import paper_2609_16408_gb300 as R
    import synth

    names = ["si8", "si16", "si32", "cluster12"]
    om, w = R.rpa_gl_frequencies(4)
    ctxs, pts = [], []
    for name in names:
        s = synth.named_system(name)
        stride = tuple(max(1, -(-n // 3)) for n in s.n)
        c = R.Context.from_system(s, om, w, precision="mixed", lanczos_max=40,
                                  lanczos_rtol=1e-6, stern_tol=1e-4, stern_maxit=20000,
                                  stride=stride, interp="linear", refine=args.refine,
                                  graphs=args.graphs)
        P = R.rpa_num_probes(c.ctx)
        ctxs.append((name, s, c, P))
        pts.append(P * len(om))
    # warm-up: autotuning, graph capture, workspaces
    for _ in range(max(1, args.warmup)):
        R.rpa_batch_energy([c.ctx for _, _, c, _ in ctxs])
    torch.cuda.synchronize()
    seq, per = 0.0, {}
    for name, s, c, P in ctxs:
        t = time.perf_counter()
        _, _, ec, st = R.rpa_energy_density(c.ctx, len(om), P, s.N_d, want_fine=False)
        dt = time.perf_counter() - t
        seq += dt
        per[name] = dict(grid=list(s.n), probe_points=P * len(om), seconds=dt, ec=ec,
                         mean_cocg_iters=st["cocg_iters"] / max(1, st["solves"]),
                         lanczos_steps_max=st["lanczos_steps_max"])
    t = time.perf_counter()
    ec_b, _ = R.rpa_batch_energy([c.ctx for _, _, c, _ in ctxs])
    bat = time.perf_counter() - t
    total = float(sum(pts))
    print(json.dumps(dict(
        metric="uneven batch: probe-points/s over four grids in one call", unit="probe-pts/s",
        value=total / bat, sequential_value=total / seq, batch_seconds=bat,
        sequential_seconds=seq, speedup=seq / bat,
        # mixed form: atomics in the projector sums make repeated runs differ by rounding
        ec_batch_vs_sequential_max_rel=float(np.max(np.abs(
            np.asarray(ec_b) - np.asarray([per[n]["ec"] for n in names])) /
            np.abs(np.asarray([per[n]["ec"] for n in names])))),
        systems=per, data="synthetic (seeded cells, synth/)",
        config=dict(workload="uneven batch (si8, si16, si32, cluster12)", form="mixed",
                    frequencies=len(om), lanczos_max=40, lanczos_rtol=1e-6, stern_tol=1e-4,
                    coarse="three points per axis", interp="linear"))), flush=True)


def run_interp_sweep(args, wl):
    """Interpolation study (Section 3.2 operators, Section 5.2 metrics) on the workload's cell:
    strides g = 2, 3 x {trilinear, tricubic} x {TF32x3, BF16} projection, against densities
    computed directly at a seeded sample of fine points that are not coarse points (FP64
    form, stride 1, Sternheimer tol 1e-8).  The interpolants are local, so d is computed only
    at the coarse points within 2g of a sample point (every 4-point stencil lies there) and
    the rest of the coarse array stays zero.  One frequency (the middle node) and N_l steps;
    Fourier interpolation needs the whole coarse array and is left out.  Prints one JSON line
    per variant with the wall time of its coarse probe-points and |dE|, L1 and ECR over the
    sample, plus the E_c error the sample implies for that frequency's term."""
    import torch

    import paper_2609_16408_gb300 as R
    torch.cuda.set_device(0)
    s = make_system(wl["system"])
    om, w = R.rpa_gl_frequencies(wl["nw"])
    km = wl["nw"] // 2
    nl = args.sweep_nl
    n = s.n
    nd = s.N_d
    rng = np.random.default_rng(2609)
    fine = []
    while len(fine) < args.sweep_points:
        x = rng.integers(0, n[0]), rng.integers(0, n[1]), rng.integers(0, n[2])
        if all(c % 6 != 0 for c in x):  # on no coarse node for g = 2 or 3
            fine.append(x)
    fine = np.array(fine)
    fidx = (fine[:, 0] + n[0] * (fine[:, 1] + n[1] * fine[:, 2])).astype(np.int64)

    def ctx(prec, g, interp="cubic", proj="tf32x3", tol=wl["tol"]):
        form = prec if prec == "fp64" else ("mixed_bf16" if proj == "bf16" else "mixed")
        return R.Context.from_system(s, om, w, lanczos_max=nl, stern_tol=tol,
                                     stern_maxit=20000, precision=form, stride=(g, g, g),
                                     interp=interp, refine=args.refine)
    c1 = ctx("fp64", 1, interp="none", tol=1e-8)
    ref = np.asarray(R.rpa_probe_density(c1.ctx, fidx, np.full(len(fidx), km, np.int32))["d"])
    c1.close()
    for g in (2, 3):
        for proj in ("tf32x3", "bf16"):
            c = ctx("mixed", g, proj=proj)
            P = R.rpa_num_probes(c.ctx)
            cidx = R.rpa_probe_indices(c.ctx)
            cc = np.stack([cidx % n[0], (cidx // n[0]) % n[1], cidx // (n[0] * n[1])], axis=1)
            near = np.zeros(P, dtype=bool)
            for f in fine:
                dist = np.abs(cc - f[None, :])
                dist = np.minimum(dist, np.asarray(n)[None, :] - dist)  # periodic distance
                near |= np.all(dist < 2 * g, axis=1)
            sel = np.nonzero(near)[0]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = R.rpa_probe_density(c.ctx, cidx[sel].astype(np.int64),
                                      np.full(len(sel), km, np.int32), allow_nonconv=True)
            tsec = time.perf_counter() - t0
            dco = np.zeros((wl["nw"], P))
            dco[km, sel] = out["d"]
            for kind in ("linear", "cubic"):
                R.rpa_set_options(c.ctx, c.opts, interp=kind)
                dfi, _ = R.rpa_interpolate(c.ctx, dco, nd)
                dd = np.asarray(dfi)[km, fidx] - ref
                s_ = abs(float(dd.sum()))
                l1 = float(np.abs(dd).sum())
                ec_est = (nd / len(fidx)) * float(dd.sum()) * w[km] / (2 * np.pi) / wl["natom"]
                line = dict(sweep="interpolation", workload=wl["system"], stride=g,
                            interp=kind, projection=proj, frequency=float(om[km]),
                            lanczos_steps=nl, stern_tol=wl["tol"],
                            coarse_probe_points=int(len(sel)), seconds=tsec,
                            probe_pts_per_s=len(sel) / tsec, full_coarse_points=int(P),
                            sample_points=int(len(fidx)), abs_err=s_, l1=l1,
                            ecr=s_ / l1 if l1 > 0 else 0.0,
                            max_rel_err=float(np.max(np.abs(dd) / np.abs(ref))),
                            ec_err_mha_per_atom_est=1e3 * abs(ec_est),
                            status=int(out["status"]))
                print(json.dumps(line), flush=True)
            c.close()


_KERNEL_FILES = {"k_dirmatvec": "cocg_fused.cu", "k_update_dots": "cocg_fused.cu",
                 "k_dirmatvec_x2": "cocg_x2.cu", "k_dirmatvec_rows": "cocg_rows.cu",
                 "k_dirmatvec_band": "cocg_band.cu", "k_dirmatvec_x2p": "cocg_x2p.cu"}


def kernel_source_sha(kernel="k_dirmatvec"):
    """Hash of the source file that defines `kernel` plus every CUDA header, to tell whether
    stored ncu counters still apply to the kernel being timed."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_16408_gb300", "csrc")
    files = [_KERNEL_FILES.get(kernel, "cocg_fused.cu")] + sorted(
        f for f in os.listdir(csrc) if f.endswith(".cuh"))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="si64", choices=sorted(WORKLOADS))
    ap.add_argument("--probes-per-freq", type=int, default=1)
    ap.add_argument("--fp64-probes-per-freq", type=int, default=2)
    ap.add_argument("--refine", type=int, default=4)
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="FP32 COCG tolerance of the mixed form per refinement round (0 = auto)")
    ap.add_argument("--nl", type=int, default=0,
                    help="override the Lanczos step count (profiling runs only)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--nw", type=int, default=0,
                    help="override the frequency count (small profiling cases only)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="H-apply tiling of the mixed form: -1 autotune, 0 32x8 column tiles, "
                         "-2 64x8 two-point tiles, h > 0 full-row tiles of height h, -100-h "
                         "bands of h full rows (asynchronous-copy pipeline)")
    ap.add_argument("--proj", default="tf32x3", choices=["tf32x3", "bf16"],
                    help="operand form of the mixed form's projection GEMMs")
    ap.add_argument("--stride", type=int, default=0,
                    help="override the coarse stride g on every axis (interpolation sweep)")
    ap.add_argument("--lanczos-block", type=int, default=1,
                    help="block Lanczos quadrature over blocks of this many probe-points of "
                         "one frequency (options.lanczos_block; mixed form); 1 = scalar")
    ap.add_argument("--lanes", type=int, default=1,
                    help="probe-point lanes run concurrently (options.lanes)")
    ap.add_argument("--graphs", type=int, default=2, choices=[0, 1, 2],
                    help="each COCG loop as one captured graph with device-side loop control "
                         "(2), COCG chunks as captured graphs replayed by the host (1), or "
                         "direct launches (0)")
    ap.add_argument("--sweep-interp", action="store_true",
                    help="interpolation study instead of the benchmark line (strides 2, 3 x "
                         "trilinear, tricubic x TF32x3, BF16 projection), one JSON line each")
    ap.add_argument("--uneven", action="store_true",
                    help="time the uneven batch (four grids in one rpa_batch_energy call) "
                         "against the same systems run one after the other")
    ap.add_argument("--sweep-nl", type=int, default=3, help="Lanczos steps of the sweep")
    ap.add_argument("--sweep-points", type=int, default=6, help="fine sample points")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.nl > 0:
        wl["nl"] = args.nl
        wl["desc"] += f" [profiling run: {args.nl} Lanczos steps]"
    if args.stride > 0:
        wl["stride"] = (args.stride,) * 3
        wl["desc"] += f" [stride {args.stride}]"
    if args.nw > 0:
        wl["nw"] = args.nw
        wl["desc"] += f" [profiling run: {args.nw} frequencies]"
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args, wl)
        return
    if args.sweep_interp:
        run_interp_sweep(args, wl)
        return
    if args.uneven:
        run_uneven(args)
        return
    run_ours(args, wl)


if __name__ == "__main__":
    main()
