"""Benchmark: Crank-Nicolson steps/s of the 3D time-dependent Dirac equation on one GB300.

Workload (default): the production-shaped hydrogen system -- R = 300 a.u., 1000 order-7
B-splines on a linear-then-geometric grid, |kappa| <= 30 with every mu (1860 channels,
n = 3.72 M complex unknowns), multipoles l <= 6, 3-cycle 800 nm sin^2 pulse at E0 = 0.1 a.u.,
dt = 0.005, BiCGSTAB to relative residual 1e-10.  Every step runs the whole hot path: pulse
factors, coupling assembly, A_- psi, BiCGSTAB (operator applies, preconditioner, updates).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--precision 0|1|2] [--t0 T] [--workload production|slice|small] [--no-fp64-compare]
Prints one JSON line (rank 0).  N > 1 (torchrun) runs N independent replicas, one per GPU,
with no data-path communication; the value is the total steps/s over all ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CN steps/s + SpMV HBM GB/s, 1 GB300: mixed/learned vs plain FP64 @ equal resid"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e3 / 1e6   # SMs x FP64 FMA/clk/SM x 2 flop x max clock (GHz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="production")
    ap.add_argument("--precision", type=int, default=2,
                    help="0 FP64, 1 c64 in FP64 refinement, 2 c64 in double-float refinement")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the plain FP64 solver on the same steps")
    ap.add_argument("--t0", type=float, default=None, help="start time (default: 0, the pulse start)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--batch-n", type=int, default=64, help="instances of --workload batch")
    ap.add_argument("--batch-lmax", type=int, default=2, help="multipole limit of the batch instances")
    ap.add_argument("--batch-kmax", type=int, default=20, help="|kappa| limit of the batch instances")
    ap.add_argument("--learned", action="store_true",
                    help="train the learned initial guess on production trajectories, then time guess=2 vs guess=1")
    ap.add_argument("--factorised", type=int, nargs="?", const=1, default=1,
                    help="complex64 apply of the inner solve in precision 2: 1 factorised, subgroup form "
                         "(default: radial band products x angular coefficients, coupling values not read), "
                         "2 factorised, per-channel form, 0 the stored coupling values (owner/gather passes)")
    ap.add_argument("--spectrum", action="store_true",
                    help="also time the photoelectron spectrum dP/dE of the final state (window (0, 2] a.u.)")
    ap.add_argument("--overlap", action="store_true",
                    help="precision 2: assemble the next step during the current solve (same arithmetic)")
    ap.add_argument("--host-loop", action="store_true",
                    help="time the headline on the host-driven loop (dirac_step) instead of the graph driver")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison legs (peak-field window, precision 1, learned guess, batch)")
    ap.add_argument("--no-batch-leg", action="store_true", help="skip the batch leg of the comparison")
    ap.add_argument("--train-n", type=int, default=12, help="training trajectories of the learned guess")
    ap.add_argument("--learned-eval", action="store_true",
                    help="wider training (--train-pulses x --train-windows windows of --train-steps steps), then "
                         "per-seed timing on --eval-seeds held-out pulses from seed --eval-seed0")
    ap.add_argument("--train-pulses", type=int, default=25)
    ap.add_argument("--train-windows", type=int, default=8)
    ap.add_argument("--eval-seeds", type=int, default=16)
    ap.add_argument("--eval-seed0", type=int, default=2000)
    ap.add_argument("--train-steps", type=int, default=10, help="steps per training trajectory")
    ap.add_argument("--guess-forward", type=int, default=0, metavar="M",
                    help="time only the learned-guess network forward on M seeded random positions (tcgen05 "
                         "kernel against the mma.sync kernel) and print one JSON line")
    return ap.parse_args()


def workload_desc(name, cfg):
    return ("%s: hydrogen Z=%g, R=%g a.u., N=%d order-%d B-splines (%s grid), |kappa|<=%d, %s, l<=%d, "
            "%g-cycle sin^2 pulse omega=%.6f a.u. E0=%g, dt=%g, tol=%g" %
            (name, cfg["Z"], cfg["R"], cfg["N"], cfg["order"], "linear" if cfg["grid"] == 0 else
             "linear-then-geometric", cfg["kappa_max"], "all mu" if cfg["two_mu_max"] <= 0 else
             "|mu|<=%g" % (cfg["two_mu_max"] / 2), cfg["l_max"], cfg["n_cycles"], cfg["omega"], cfg["E0"],
             cfg["dt"], cfg["tol"]))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def operator_counts(bas, cfg, kind):
    """Algorithmic bytes and flops of one operator apply A_+- x.

    kind 'f64': FP64 values and vectors; 'f32': FP32 values, complex64 vectors; 'df': double-float
    values (hi + lo floats, 8 B), split input vector (16 B per complex), complex128 output.
    Each stored coupling value (upper pairs only) is used twice (W x_b and W^T x_a), each use a real
    x complex multiply-add (4 flop); the radial blocks S and H0 add 8 flop per entry and channel."""
    n1, bd = cfg["N"] + 1, 2 * cfg["order"] - 1
    coup = bas.npairs * n1 * bd * 4
    diag = bas.nch * n1 * bd * 4
    nk2 = 2 * cfg["kappa_max"]
    flops = 8 * coup + 2 * 8 * diag
    vb, ib, ob = {"f64": (8, 16, 16), "f32": (4, 8, 8), "df": (8, 16, 16)}[kind]
    bytes_ = vb * coup + (ib + ob) * bas.n + 2 * vb * nk2 * n1 * bd * 4
    return coup, flops, bytes_


FP32_LANE_OPS = 152 * 128 * 2.070   # 10^9 lane operations/s: SMs x FP32 lanes x max clock (GHz)

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the owner passes from one ncu capture
# on the medium workload (6944 pairs x 601 radial slots), scaled to the production launch by the
# units processed (pairs x slots: x 9.817); the summaries under profiles/ give the commands and the
# raw counters.  Valid for the kernels as captured (a changed kernel needs a new capture).
TRAFFIC_MEDIUM = {"df": (1.768965e9 + 0.155458e9, "profiles/k_residual_own_df_medium.md"),
                  "df_owner": (1.768965e9 + 0.155458e9, "profiles/k_residual_own_df_medium.md"),
                  "f32": (0.887222e9 + 0.074195e9, "profiles/k_apply_own32_medium.md")}
MEDIUM_UNITS = 6944 * 601
DF_OPS_PER_FMA = 10                 # FP32 operations of one double-float multiply-add (df64.cuh df_fma)
DF_OPS_PER_FMA_OFF = 6              # ... in the fixed-binade form (df_fma_off), tolerances >= 1e-11
OFFSET_TOL = 1e-11                  # the library picks the fixed-binade form at tolerances >= this


def roofline_of(bas, cfg, phase, kind, ms, cnt, hbm_peak, fact=1):
    """Roofline of one operator-apply launch group, timed live by the library's event timers.

    kind 'f64': FP64 apply (FP64 ALU bound), 'f32': complex64 owner/gather apply (HBM bound),
    'df': double-float refinement residual pass (FP32 ALU/issue bound), 'df_owner': its owner pass.
    The owner pass's coupling products take DF_OPS_PER_FMA_OFF operations at tolerances >= 1e-11
    (the library's automatic choice), DF_OPS_PER_FMA below; the gather's diagonal blocks always ten."""
    cops = DF_OPS_PER_FMA_OFF if cfg["tol"] >= OFFSET_TOL else DF_OPS_PER_FMA
    coup, flops, bytes_ = operator_counts(bas, cfg, {"df_owner": "df", "fact32": "f32"}.get(kind, kind))
    t = ms / cnt / 1000.0
    gbs = bytes_ / t / 1e9
    traffic, tnote = None, None
    if kind in TRAFFIC_MEDIUM:
        units = bas.npairs * (cfg["N"] + 1)
        traffic = TRAFFIC_MEDIUM[kind][0] * units / MEDIUM_UNITS
        tnote = ("owner pass only, from %s (medium capture) scaled by pairs x radial slots (x%.3f)" %
                 (TRAFFIC_MEDIUM[kind][1], units / MEDIUM_UNITS))
    out = {"phase": phase, "apply_ms": t * 1000.0, "bytes_per_apply": bytes_, "gbs": gbs, "traffic": traffic}
    if tnote:
        out["traffic_note"] = tnote
    if kind == "f64":
        tf = flops / t / 1e12
        out.update({"kernel": "k_apply<double> (FP64 operator apply)", "flops_per_apply": flops, "bound": "alu",
                    "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"})
    elif kind == "fact32":
        # factorised complex64 apply: useful FMAs only (the radial band products of every channel and
        # multipole, the angular combination of each directed pair term, the diagonal blocks); it
        # reads no coupling values, so its HBM bytes are the vectors' and it is timed against the
        # FP32 FMA rate (one FMA per lane per clock)
        n1, bd = cfg["N"] + 1, 2 * cfg["order"] - 1
        L = cfg["l_max"] + 1
        fma_rad = bas.nch * L * n1 * 4 * 2 * bd * 2 * 2
        fma_ang = 2 * bas.nterms * n1 * 2 * 8
        fma_diag = bas.nch * n1 * 2 * bd * 2 * 4
        fma = fma_rad + fma_ang + fma_diag
        out["bytes_per_apply"] = (8 + 8) * bas.n
        out["gbs"] = out["bytes_per_apply"] / t / 1e9
        tf = 2 * fma / t / 1e12
        peak = 2 * FP32_LANE_OPS / 1e3
        out.update({"kernel": ("k_fact_tile32 (factorised complex64 inner-solve apply, subgroup form: radial pass "
                               "of tile t+1 beside the angular pass of tile t)" if fact == 1 else
                               "k_fact_radial32 + k_fact_angular32 (factorised complex64 inner-solve apply, "
                               "per-channel form)"),
                    "fma_per_apply": {"radial": fma_rad, "angular": fma_ang, "diagonal": fma_diag},
                    "bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                    "peak_source": "derived FP32 FMA rate: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"})
    elif kind == "f32":
        out.update({"kernel": "k_apply_own32 + k_apply_gather32 (complex64 inner-solve apply)",
                    "flops_per_apply": flops, "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak})
    elif kind == "df_owner":
        # the owner pass alone: it streams the hi and lo words of every stored coupling value once
        # (HBM), and forms each value's two uses (W u_b, W^T u_a) on re and im in double-float
        # (FP32 issue); against the two peaks it sits closer to the HBM one, which is reported as
        # the bound, with the FP32-issue view beside it
        dfma = 4 * coup
        ops = dfma * cops
        tops = ops / t / 1e12
        peak = FP32_LANE_OPS / 1e3
        out.update({"kernel": "k_residual_own_df (double-float refinement residual, owner pass)",
                    "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "alu_view": {"df_fma_per_apply": dfma, "ops_per_apply": ops, "achieved": tops, "peak": peak,
                                 "unit": "T FP32-lane-ops/s", "frac": tops / peak,
                                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (1 op per lane per "
                                                "clock); %d FP32 ops per double-float multiply-add (%s)" %
                                                (cops, "fixed-binade accumulators" if cops == DF_OPS_PER_FMA_OFF
                                                 else "Dot2 accumulators")}})
    else:
        # double-float multiply-adds: each stored value twice (W u_b, W^T u_a) on re and im, the
        # diagonal blocks S and tau H0 on both u and v (4 per entry and channel)
        n1, bd = cfg["N"] + 1, 2 * cfg["order"] - 1
        dfma = 4 * coup + 4 * bas.nch * n1 * bd * 4
        ops = 4 * coup * cops + 4 * bas.nch * n1 * bd * 4 * DF_OPS_PER_FMA
        tops = ops / t / 1e12
        peak = FP32_LANE_OPS / 1e3
        out.update({"kernel": "k_split_uv3 + k_residual_own_df + k_residual_gather_df (double-float refinement "
                              "residual)", "df_fma_per_apply": dfma, "ops_per_apply": ops, "bound": "alu",
                    "achieved": tops, "peak": peak, "unit": "T FP32-lane-ops/s", "frac": tops / peak,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (1 op per lane per clock); "
                                   "%d ops per coupling multiply-add, 10 per diagonal-block one" % cops})
    return out


def roofline(bas, cfg, phase_ms, phase_n, precision, hbm_peak, factorised=0):
    """The dominant kernel's roofline, plus the complex64 SpMV's when it ran.  In precision 2 the
    dominant kernel is the residual's owner pass, timed on its own (its phase lies inside 'apply');
    the whole residual pass (split, owner, gather) is reported beside it."""
    cands = []
    if phase_n.get("apply", 0):
        cands.append(("apply", "df" if precision == 2 else "f64", phase_ms["apply"], phase_n["apply"]))
    if phase_n.get("apply32", 0):
        cands.append(("apply32", "fact32" if factorised else "f32", phase_ms["apply32"], phase_n["apply32"]))
    outs = {c[0]: roofline_of(bas, cfg, c[0], c[1], c[2], c[3], hbm_peak, factorised) for c in cands}
    dom = max(cands, key=lambda c: c[2])[0]
    if dom == "apply" and precision == 2 and phase_n.get("owner", 0):
        whole = outs["apply"]
        own = roofline_of(bas, cfg, "owner", "df_owner", phase_ms["owner"], phase_n["owner"], hbm_peak)
        own["residual_pass"] = {k: whole[k] for k in ("kernel", "apply_ms", "achieved", "frac")}
        return own, outs.get("apply32")
    return outs[dom], outs.get("apply32")


def max_over_ranks(ms, dist=None, device=None):
    """The slowest rank's time (all ranks run the same replica workload; the job takes the longest)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(steps, ms, world):
    """(per-replica steps/s, whole-job steps/s): N independent replicas each advance `steps` steps
    in the slowest rank's time."""
    sps = steps / (ms / 1000.0)
    return sps, sps * world


# complex64 apply of the inner solve for every precision-2 operator the bench builds (--factorised)
INNER_FACT = 1


def inner_apply(op, precision):
    """Put a precision-2 operator on the inner-solve apply chosen by --factorised."""
    if precision == 2 and INNER_FACT:
        op.set_factorised(INNER_FACT)


def window_run(B, torch, bas, cfg, psi0_h, t0, warmup, steps, stream, dev, precision, guess=1, net=None,
               host_loop=False):
    """W warm-up steps (they fill the history and capture the graph) then K timed steps from psi0 at
    t0, on the graph driver (dirac_run) or the host loop (dirac_step); CUDA events on the op's stream.
    Returns (stats, final state, op)."""
    import numpy as np
    op = B.Operator(bas, cfg, stream=stream, tol=cfg["tol"], precision=precision, max_iter=1000, tol_inner=1e-5,
                    max_outer=20, guess=guess)
    inner_apply(op, precision)
    if net is not None:
        B.set_guess(op, net)
    with torch.cuda.stream(stream):
        psi = torch.from_numpy(psi0_h).to(dev)
        hist = torch.zeros((3 if guess == 2 else 2) * bas.n, dtype=torch.complex128, device=dev)
    run = (lambda n, t, nh: op.step(psi, n, t, hist=hist, n_hist=nh)) if host_loop else \
        (lambda n, t, nh: op.run(psi, n, t, hist, n_hist=nh))
    _, _, nh = run(warmup, t0, 0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    its, res, nh = run(steps, t0 + warmup * cfg["dt"], nh)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    out = {"value": steps / (ms / 1000.0), "unit": "steps/s", "ms_per_step": ms / steps,
           "iters_per_step": float(np.mean(its)), "max_resid": float(np.max(res)),
           "dtype": ["f64", "c64+f64", "c64+df64"][precision], "driver": "dirac_step" if host_loop else "dirac_run"}
    return out, psi, op


def state_errors(obs_op, ref, psi, ref_obs=None):
    """Per-result errors of a state against the plain FP64 state at the same time: wavefunction
    relative L2, and the absolute differences of the norm, <H0>, ground and bound populations."""
    import torch
    o_ref = ref_obs if ref_obs is not None else obs_op.observables(ref, bound=True)
    o = obs_op.observables(psi, bound=True)
    out = {"psi_rel_l2": (torch.linalg.norm(psi - ref) / torch.linalg.norm(ref)).item()}
    for k in ("norm", "energy", "p_ground", "p_bound"):
        out[k] = abs(o[k] - o_ref[k])
    return out, o_ref


def train_guess(B, torch, bas, cfg, precision, n_train, train_steps, per_step=65536, iters=1500):
    """Learned initial guess: trajectories of the method itself (extrapolated guess) for seeded pulses
    at seeded times on the workload's basis give (features, target) samples, drawn with probability
    proportional to s^2; the network is trained by the library's kernels.  Returns (net, note)."""
    from paper_2512_21697_gb300 import learned as L, workloads as W
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    X, Tg = [], []
    t_data = time.time()
    for pc in L.pulse_variants(cfg, range(1000, 1000 + n_train)):
        tr = L.Trajectory(bas, pc, train_steps, precision=precision, tol=cfg["tol"])
        x, t, sc = L.samples(tr)
        xs, ts = L.importance_subsample(x, t, sc, per_step * (train_steps - 4), g)
        X.append(xs)
        Tg.append(ts)
        del tr, x, t, sc
        torch.cuda.empty_cache()
    X, Tg = torch.cat(X), torch.cat(Tg)
    n_samples = int(X.shape[0])
    t_data = time.time() - t_data
    net = B.GuessNet(8192, W.guess_net_init(7))
    t_train = time.time()
    losses = L.train(net, X, Tg, iters, batch=8192, lr=1e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.time() - t_train
    del X, Tg
    note = ("%d seeded pulses (seeds 1000..%d) x %d steps (extrapolated guess), %d samples drawn with probability "
            "proportional to s^2, %d Adam steps of 8192; data %.1f s, training %.1f s; loss %.3g -> %.3g" %
            (n_train, 999 + n_train, train_steps, n_samples, iters, t_data, t_train, losses[0], losses[-1]))
    return net, note


def train_guess_windows(B, torch, bas, cfg, precision, pulses, windows, steps, per_step=65536, iters=3000,
                        seed0=1000):
    """Wider training set: `pulses` seeded pulses (seeds seed0..), each stepping `windows` windows of
    `steps` steps from the ground state at seeded start times, one operator per pulse; every window's
    samples are drawn at once (probability proportional to s^2) so the set streams into device
    memory.  Returns (net, note)."""
    import numpy as np
    from paper_2512_21697_gb300 import learned as L, workloads as W
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    X, Tg = [], []
    t_data = time.time()
    for pc in L.pulse_variants(cfg, range(seed0, seed0 + pulses)):
        op = B.Operator(bas, pc, tol=cfg["tol"], precision=precision, max_iter=1000, tol_inner=1e-5, max_outer=30,
                        guess=1)
        T = pc["n_cycles"] * 2 * math.pi / pc["omega"]
        rng = np.random.default_rng(int(round(pc["E0"] * 1e9)) % (2 ** 31))
        for t_s in rng.uniform(0.05, 0.95, windows) * T:
            tr = L.Trajectory(bas, pc, steps, precision=precision, tol=cfg["tol"], op=op, t_start=t_s)
            x, t, sc = L.samples(tr)
            xs, ts = L.importance_subsample(x, t, sc, per_step * (steps - 4), g)
            X.append(xs)
            Tg.append(ts)
            del tr, x, t, sc
        del op
        torch.cuda.empty_cache()
    X, Tg = torch.cat(X), torch.cat(Tg)
    n_samples = int(X.shape[0])
    t_data = time.time() - t_data
    net = B.GuessNet(8192, W.guess_net_init(7))
    t_train = time.time()
    losses = L.train(net, X, Tg, iters, batch=8192, lr=1e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.time() - t_train
    del X, Tg
    note = ("%d seeded pulses (seeds %d..%d) x %d windows of %d steps from seeded start times (%d windows, "
            "extrapolated guess), %d samples drawn with probability proportional to s^2, %d Adam steps of 8192; "
            "data %.1f s, training %.1f s; loss %.3g -> %.3g" %
            (pulses, seed0, seed0 + pulses - 1, windows, steps, pulses * windows, n_samples, iters, t_data, t_train,
             losses[0], losses[-1]))
    return net, note


def learned_eval(args, world, rank, local, dist):
    """--learned-eval: the wider training set (train_guess_windows), then every held-out seeded pulse
    (seeds --eval-seed0.., never trained on) from its own seeded start time: W warm-up steps and K
    timed steps on the graph driver with the extrapolated guess and with the learned one, to the
    workload's tolerance; per-seed iterations/step and steps/s."""
    import numpy as np
    import torch
    from paper_2512_21697_gb300 import binding as B, learned as L, workloads as W
    dev = torch.device("cuda", local)
    cfg = dict(W.WORKLOADS[args.workload])
    bas = B.Basis(cfg)
    net, note = train_guess_windows(B, torch, bas, cfg, args.precision, args.train_pulses, args.train_windows,
                                    args.train_steps)
    psi0, _ = bas.initial_state()
    rows = []
    clocks = ClockSampler(local)
    clocks.start()
    for seed, pc in zip(range(args.eval_seed0, args.eval_seed0 + args.eval_seeds),
                        L.pulse_variants(cfg, range(args.eval_seed0, args.eval_seed0 + args.eval_seeds))):
        row = {"seed": seed, "E0": pc["E0"], "wavelength_nm": W.NM_HARTREE / pc["omega"], "cycles": pc["n_cycles"],
               "t_start_over_T": pc["t_start"] / (pc["n_cycles"] * 2 * math.pi / pc["omega"])}
        for guess, key in ((1, "extrapolated"), (2, "learned")):
            stream = torch.cuda.Stream()
            r, _, op = window_run(B, torch, bas, pc, psi0, pc["t_start"], args.warmup, args.steps, stream, dev,
                                  args.precision, guess=guess, net=net if guess == 2 else None)
            row[key] = {k: r[k] for k in ("value", "ms_per_step", "iters_per_step", "max_resid")}
            del op
            torch.cuda.empty_cache()
        row["speedup"] = row["learned"]["value"] / row["extrapolated"]["value"]
        rows.append(row)
    ck = clocks.stop()
    agg = {k: float(np.mean([r[g][k] for r in rows])) for g in ("learned",) for k in ("value", "iters_per_step")}
    ext = {k: float(np.mean([r["extrapolated"][k] for r in rows])) for k in ("value", "iters_per_step")}
    line = {"metric": METRIC, "value": agg["value"] * world, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / agg["value"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ["f64", "c64+f64", "c64+df64"][args.precision], "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, cfg) + "; learned initial guess on %d held-out "
                                   "seeded pulses (seeds %d..%d), each from its own seeded start time" %
                                   (args.eval_seeds, args.eval_seed0, args.eval_seed0 + args.eval_seeds - 1),
                       "training": note},
            "mean_learned": agg, "mean_extrapolated": ext,
            "mean_speedup_vs_extrapolated": float(np.mean([r["speedup"] for r in rows])),
            "per_seed": rows, "clocks": ck}
    if rank == 0:
        print(json.dumps(line), flush=True)


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(cfg, its_per_step, seconds, seed=5):
    """The oracle, as it stands, on a bounded sample: rows of A_+ x at the full workload."""
    import numpy as np
    import oracle
    from paper_2512_21697_gb300 import workloads as W
    oracle.build()
    orc = oracle.Oracle(**W.oracle_params(cfg))
    x = W.random_state(orc.n, seed)
    x[~orc.active_mask()] = 0
    rng = np.random.default_rng(seed)
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    done, elapsed, batch = 0, 0.0, 256
    while elapsed < seconds:
        rows = rng.integers(0, orc.n, batch)
        t0 = time.perf_counter()
        orc.apply_rows(0.5 * T, +1, x, rows // orc.nb, rows % orc.nb)
        elapsed += time.perf_counter() - t0
        done += batch
    t_apply = elapsed / done * orc.n
    applies = 3 + 2 * its_per_step
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 1.0 / (t_apply * applies), "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d rows of A_+ x (of n=%d) at the full workload, %.1f s; step = %.1f operator "
                      "applies (3 + 2 x %.2f BiCGSTAB iterations/step)" % (done, orc.n, elapsed, applies,
                                                                         its_per_step)}


def reference_arm(args):
    """Oracle arm: the CPU oracle as it stands, same workload, metric and unit."""
    from paper_2512_21697_gb300 import workloads as W
    cfg = W.WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # iterations per step: the oracle's own BiCGSTAB on the slice system in the same window
    import oracle
    sl = oracle.Oracle(**W.oracle_params(W.SLICE))
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    t0 = args.t0 if args.t0 is not None else 0.0
    x, _ = sl.ground_state()
    its = []
    for s in range(2):
        x, it, _ = sl.step(x, t0 + s * cfg["dt"], tol=cfg["tol"])
        its.append(it)
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_baseline(cfg, sum(its) / len(its), max(2.0, args.cpu_seconds / 2))["value"])
    cb = cpu_baseline(cfg, sum(its) / len(its), 1.0)
    v = statistics.median(vals[args.warmup:])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, cfg), "t_start": t0},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def guess_forward_bench(args, reps=20):
    """The network forward alone (dirac_guess_forward) on M seeded random feature rows with the
    workload module's seeded initial weights: the tcgen05 kernel (tensor_cores=1) and the warp-level
    mma.sync kernel (tensor_cores=2), CUDA events around `reps` launches each, after a warm-up."""
    import torch
    from paper_2512_21697_gb300 import binding as B, workloads as W
    M = args.guess_forward
    net = B.GuessNet(8192, W.guess_net_init(7))
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn((M, 32), generator=g, device="cuda", dtype=torch.float32)
    out = torch.empty((M, 4), device="cuda", dtype=torch.float32)
    flop = 2.0 * M * (32 * 256 + 2 * 256 * 256 + 256 * 4)
    peak = 1906.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    res = {}
    for tc in (1, 2):
        net.forward(x, out, tensor_cores=tc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.forward(x, out, tensor_cores=tc)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[["", "tcgen05", "mma_sync"][tc]] = {"ms": ms, "tflops": flop / ms / 1e9, "frac_bf16_peak": flop / ms / 1e9 / peak}
    print(json.dumps({"guess_forward": {"positions": M, "flop_per_forward": flop, "bf16_peak_tflops": peak, **res}}),
          flush=True)


def learned_bench(args, world, rank, local, dist):
    """--learned: train the learned initial guess on trajectories of the workload's basis, then time
    the same K steps at peak field (or --t0) with the extrapolated guess and with the learned one
    (both on the graph driver, both solving to the same tolerance)."""
    import torch
    from paper_2512_21697_gb300 import binding as B, workloads as W
    dev = torch.device("cuda", local)
    cfg = dict(W.WORKLOADS[args.workload])
    bas = B.Basis(cfg)
    net, note = train_guess(B, torch, bas, cfg, args.precision, args.train_n, args.train_steps)
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    t0 = args.t0 if args.t0 is not None else 0.5 * T
    psi0, _ = bas.initial_state()
    res = {}
    for guess in (1, 2):
        stream = torch.cuda.Stream()
        clocks = ClockSampler(local)
        clocks.start()
        r, _, op = window_run(B, torch, bas, cfg, psi0, t0, args.warmup, args.steps, stream, dev, args.precision,
                              guess=guess, net=net if guess == 2 else None, host_loop=args.host_loop)
        r["clocks"] = clocks.stop()
        res[guess] = r
        del op
    line = {"metric": METRIC, "value": res[2]["value"] * world, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[2]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ["f64", "c64+f64", "c64+df64"][args.precision], "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, cfg) + "; learned initial guess, start at t=%.2f" % t0,
                       "training": note},
            "learned": res[2], "extrapolated": res[1], "speedup_vs_extrapolated": res[2]["value"] / res[1]["value"],
            "clocks": res[2]["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _batch_ops(B, torch, cfgs, bases, dev, precision, guess):
    """Operators for as many instances as the free device memory allows (1.5x the largest instance
    seen so far plus 24 GB must stay free), each on its own stream."""
    ops, used = [], []
    biggest = 0
    for cfg, bas in zip(cfgs, bases):
        free, _ = torch.cuda.mem_get_info(dev)
        if biggest and free < 1.5 * biggest + 24e9:
            break
        op = B.Operator(bas, cfg, stream=torch.cuda.Stream(), tol=cfg["tol"], precision=precision, max_iter=1000,
                        tol_inner=1e-5, max_outer=20, guess=guess)
        inner_apply(op, precision)
        biggest = max(biggest, op.device_bytes())
        ops.append(op)
        used.append((cfg, bas))
    return ops, used


def _batch_time(B, torch, ops, used, dev, args, t0s, window, hist_len):
    """Warm-up steps (they also fill the history), then the timed batch call: (wall seconds,
    iterations, residuals)."""
    psis = [torch.from_numpy(bas.initial_state()[0]).to(dev) for _, bas in used]
    hists = [torch.zeros(hist_len * bas.n, dtype=torch.complex128, device=dev) for _, bas in used]
    nh = [0] * len(ops)
    _, _, nh = B.solve_batch(ops, psis, hists, args.warmup, t0s, n_hist=nh, window=window)
    tcur = [t + args.warmup * c["dt"] for t, (c, _) in zip(t0s, used)]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    its, res, nh = B.solve_batch(ops, psis, hists, args.steps, tcur, n_hist=nh, window=window)
    torch.cuda.synchronize()
    return time.perf_counter() - w0, its, res


def batch_measure(args, world, local, n_req, learned, peak, fp64=True):
    """Batched workload: independent instances (own pulse and radial size) stepped concurrently by
    dirac_solve_batch with the window and preconditioner schedule picked by dirac_batch_tune.
    Returns ({"mixed", "mixed_learned", "fp64": instance-steps/s ...}, config, clocks).  With
    learned, the network is trained first on trajectories of the batch's own instances; with peak,
    the instances start at their peak field."""
    import concurrent.futures as cf
    import numpy as np
    import torch
    from paper_2512_21697_gb300 import binding as B, learned as L, workloads as W
    dev = torch.device("cuda", local)
    cfgs = W.batch_instances(n_req, seed0=0, kappa_max=args.batch_kmax, l_max=args.batch_lmax)
    t_setup = time.time()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        bases = list(ex.map(B.Basis, cfgs))
    ops, used = _batch_ops(B, torch, cfgs, bases, dev, args.precision, 2 if learned else 1)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    n_inst = len(ops)
    T = [c["n_cycles"] * 2 * math.pi / c["omega"] for c, _ in used]
    t0s = [0.5 * t for t in T] if peak else [0.0] * n_inst
    # schedule autotuner on the starting states
    psis = [torch.from_numpy(bas.initial_state()[0]).to(dev) for _, bas in used]
    hists = [torch.zeros(3 * bas.n, dtype=torch.complex128, device=dev) for _, bas in used]
    cand = [w for w in (1, 4, 8, 16, 0) if w <= n_inst]
    best, tune_ms = B.batch_tune(ops, psis, hists, t0s, cand)
    del psis, hists
    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    wall, its, res = _batch_time(B, torch, ops, used, dev, args, t0s, best, 3)
    ck = clocks.stop()
    out["mixed"] = {"value": n_inst * args.steps / wall * world, "iters_per_step": float(np.mean(its)),
                    "max_resid": float(np.max(res))}
    train_note = None
    if learned:
        # training data: trajectories of the first instances at seeded times inside their pulses
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        X, Tg = [], []
        t_train = time.time()
        for i in range(min(8, n_inst)):
            cfg, bas = used[i]
            u = float(np.random.default_rng(1000 + i).uniform(0.1, 0.9))
            pc = dict(cfg, t_start=u * T[i])   # the instance's own pulse, at a seeded time
            tr = L.Trajectory(bas, pc, 10, precision=args.precision, tol=cfg["tol"])
            x, t, sc = L.samples(tr)
            xs, ts = L.importance_subsample(x, t, sc, 262144, g)
            X.append(xs)
            Tg.append(ts)
            del tr, x, t, sc
        X, Tg = torch.cat(X), torch.cat(Tg)
        net = B.GuessNet(8192, W.guess_net_init(7))
        losses = L.train(net, X, Tg, 1500, batch=8192, lr=1e-3, seed=1)
        torch.cuda.synchronize()
        t_train = time.time() - t_train
        train_note = "8 instances x 10 steps at seeded times, %d samples (p ~ s^2), 1500 Adam steps; %.1f s; loss " \
                     "%.3g -> %.3g" % (X.shape[0], t_train, losses[0], losses[-1])
        del X, Tg
        for op in ops:
            B.set_guess(op, net)
        wall_l, its_l, res_l = _batch_time(B, torch, ops, used, dev, args, t0s, best, 3)
        out["mixed_learned"] = {"value": n_inst * args.steps / wall_l * world, "iters_per_step": float(np.mean(its_l)),
                                "max_resid": float(np.max(res_l))}
    del ops
    torch.cuda.empty_cache()
    if fp64:
        ops64, used64 = _batch_ops(B, torch, [c for c, _ in used], [b for _, b in used], dev, 0, 1)
        n64 = len(ops64)
        t064 = t0s[:n64]
        wall64, its64, res64 = _batch_time(B, torch, ops64, used64, dev, args, t064, best, 2)
        out["fp64"] = {"value": n64 * args.steps / wall64 * world, "instances": n64,
                       "iters_per_step": float(np.mean(its64)), "max_resid": float(np.max(res64))}
        del ops64
    head = out.get("mixed_learned", out["mixed"])
    if "fp64" in out:
        out["speedup_vs_fp64"] = head["value"] / out["fp64"]["value"]   # instance-steps/s against instance-steps/s
    config = {"workload": "batch: %d instances (of %d requested), E0 log-uniform [0.02, 0.2], wavelength "
                          "[400, 1600] nm, 2-6 cycles, N 400-1000, |kappa|<=%d, l<=%d, R=300, dt=0.005, "
                          "tol=1e-10, start %s" % (n_inst, n_req, args.batch_kmax, args.batch_lmax,
                                                   "at each instance's peak field" if peak else "at the pulse start"),
              "instances": n_inst, "unknowns": int(sum(b.n for _, b in used)), "window": best,
              "precond_schedule": "tuned (one lane per channel, or one warp per channel with rows fixed to lanes)",
              "tune_ms": {"windows": cand, "lanes": tune_ms[0].tolist(), "warps": tune_ms[1].tolist()},
              "setup_s": t_setup, "timing": "host wall clock around the batch call (many streams)",
              "steps": args.steps, "warmup": args.warmup}
    if train_note:
        config["training"] = train_note
    return out, config, ck


def batch_bench(args, world, rank, local, dist):
    """--workload batch: the batch measurement as the bench line (value: instance-steps/s of the
    mixed-precision batch, with --learned of the mixed + learned one)."""
    peak = args.learned or args.t0 is not None
    out, config, ck = batch_measure(args, world, local, args.batch_n, args.learned, peak,
                                    fp64=not args.no_fp64_compare)
    head = out.get("mixed_learned", out["mixed"])
    n_inst = config["instances"]
    config["parallelism"] = "replicas x%d" % world
    line = {
        "metric": METRIC, "value": head["value"], "unit": "instance-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": n_inst * 1000.0 / head["value"] * world, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ["f64", "c64+f64", "c64+df64"][args.precision],
        "data": "synthetic", "config": config, "batch": out, "clocks": ck,
    }
    if "speedup_vs_fp64" in out:
        line["speedup_vs_fp64"] = out["speedup_vs_fp64"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def spectrum_measure(op, bas, psi, e_hi=2.0, n_grid=2001, reps=5):
    """dP/dE (Eq. dPdE) of the state on [0, e_hi]: the first call's wall time (eigenpairs of the
    window, once per window) and the device time of later calls (projection, densities, grid)
    with CUDA events on the op's stream; the projection kernel's FP64 work against the FP64 peak."""
    import time
    import numpy as np
    import torch
    grid = np.linspace(0.0, e_hi, n_grid)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P, nl, nq = op.spectrum(psi, 0.0, e_hi, grid, counts=True)
    setup_s = time.perf_counter() - t0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(op.stream)
    for _ in range(reps):
        op.spectrum(psi, 0.0, e_hi, grid)
    ev1.record(op.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    ns = 2 * (bas.n // (2 * bas.nch))
    # per projection: a real eigenvector against complex S psi, 2 FMA = 4 flops per entry; plus S psi
    # per channel (2 n1 rows x 13 block-diagonals x 2 x 2 FMA)
    flops = 4.0 * nq * ns + bas.nch * ns * 13 * 2 * 4.0
    return {"window": [0.0, e_hi], "grid_points": n_grid, "levels": nl, "projections": nq,
            "eigen_setup_s": setup_s, "ms_per_call": ms, "calls_per_s": 1e3 / ms,
            "max_dpde": float(np.max(P)), "fp64_flops_per_call": flops,
            "fp64_tflops": flops / (ms * 1e-3) / 1e12,
            "note": "call time includes the grid copy in and the result copy out; eigenpairs kept"}


def main():
    global INNER_FACT
    args = parse()
    INNER_FACT = args.factorised
    if args.impl == "reference":
        reference_arm(args)
        return
    import numpy as np
    import torch
    from paper_2512_21697_gb300 import binding as B, workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.guess_forward:
        if rank == 0:
            guess_forward_bench(args)
        return
    if args.workload == "batch":
        batch_bench(args, world, rank, local, dist)
        return
    if args.learned_eval:
        learned_eval(args, world, rank, local, dist)
        return
    if args.learned:
        learned_bench(args, world, rank, local, dist)
        return
    cfg = dict(W.WORKLOADS[args.workload])
    T = cfg["n_cycles"] * 2 * math.pi / cfg["omega"]
    t0 = args.t0 if args.t0 is not None else 0.0
    dt = cfg["dt"]
    dev = torch.device("cuda", local)
    t_wall0 = time.time()

    bas = B.Basis(cfg)
    psi0_h, e0 = bas.initial_state()
    stream = torch.cuda.Stream()
    op = B.Operator(bas, cfg, stream=stream, tol=cfg["tol"], precision=args.precision, max_iter=1000,
                    tol_inner=1e-5, max_outer=20)
    if args.precision == 2 and args.overlap:
        op.set_overlap(True)   # next step's assembly overlaps the current solve (same arithmetic)
    inner_apply(op, args.precision)
    with torch.cuda.stream(stream):
        psi = torch.from_numpy(psi0_h).to(dev)
        hist = torch.zeros(2 * bas.n, dtype=torch.complex128, device=dev)
    graph = not args.host_loop and not args.overlap   # the graph driver does not overlap the assembly
    run = (lambda n, t, nh: op.run(psi, n, t, hist, n_hist=nh)) if graph else \
        (lambda n, t, nh: op.step(psi, n, t, hist=hist, n_hist=nh))
    # warm-up steps (the first one captures the graph)
    _, _, nh = run(args.warmup, t0, 0)
    tcur = t0 + args.warmup * dt
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    its, res, nh = run(args.steps, tcur, nh)
    ev1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    tcur += args.steps * dt
    ms = max_over_ranks(ms, dist, dev)
    sps, value = replica_rate(args.steps, ms, world)
    psi_head = psi.clone()          # the state after W + K steps from t0, for the per-result errors

    # the same kernels on the host-driven loop with the library's phase timers (CUDA events on the
    # op's stream around every launch group; event records are not allowed inside the graph's
    # conditional bodies): per-phase times, the dominant kernel's launch time for the roofline, and
    # the launch count per step
    op.profile(True)
    hl0, hl1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    hl0.record(stream)
    its_h, res_h, nh = op.step(psi, args.steps, tcur, hist=hist, n_hist=nh)
    hl1.record(stream)
    torch.cuda.synchronize()
    ms_host = hl0.elapsed_time(hl1)
    phase_ms, phase_n, launches = op.profile_read()
    op.profile(False)
    tcur += args.steps * dt

    # end to end through the C ABI with host buffers: per step, the state in from pinned host memory,
    # one dirac_run (or dirac_step) call, the state back out
    psi_h = torch.from_numpy(psi0_h).pin_memory()
    out_h = torch.empty_like(psi_h).pin_memory()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        psi_e = torch.empty_like(psi)
        hist_e = torch.zeros_like(hist)
    e2e_steps = max(2, min(args.steps, 5))
    st_e = {"nh": 0, "t": tcur}

    def e2e_step(first):
        with torch.cuda.stream(stream):
            psi_e.copy_(psi_h if first else out_h, non_blocking=True)
        if graph:
            _, _, st_e["nh"] = op.run(psi_e, 1, st_e["t"], hist_e, n_hist=st_e["nh"])
        else:
            _, _, st_e["nh"] = op.step(psi_e, 1, st_e["t"], hist=hist_e, n_hist=st_e["nh"])
        with torch.cuda.stream(stream):
            out_h.copy_(psi_e, non_blocking=True)
        st_e["t"] += dt

    for s_ in range(args.warmup):   # untimed, as for the device-resident value: fills the history
        e2e_step(s_ == 0)
    torch.cuda.synchronize()
    ee0.record(stream)
    for s_ in range(e2e_steps):
        e2e_step(False)
    ee1.record(stream)
    torch.cuda.synchronize()
    e2e_sps = e2e_steps / (ee0.elapsed_time(ee1) / 1000.0) * world

    peak_bw, peak_src = hbm_peak()
    roof, roof32 = roofline(bas, cfg, phase_ms, phase_n, args.precision, peak_bw,
                            args.factorised if args.precision == 2 else 0)
    for r in (roof, roof32):
        if r and r["bound"] == "hbm":
            r["peak_source"] = "%s copy bandwidth %.1f GB/s" % ("measured" if peak_src == "measured" else
                                                              "fallback", peak_bw)
    roof["timing"] = ("phase events around the kernel's launches during %d host-loop steps run right after the "
                      "headline's graph-driven steps (same kernels, same window)" % args.steps)
    coup = bas.npairs * (cfg["N"] + 1) * (2 * cfg["order"] - 1) * 4
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    obs = op.observables(psi)
    spec = spectrum_measure(op, bas, psi) if args.spectrum else None
    del op
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ["f64", "c64+f64", "c64+df64"][args.precision], "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, cfg), "n": bas.n, "channels": bas.nch,
                   "pairs": bas.npairs, "t_start": t0,
                   "precision": ["fp64", "mixed: c64 BiCGSTAB in FP64 refinement",
                                 "mixed: c64 BiCGSTAB in double-float refinement"][args.precision],
                   "driver": ("dirac_run: the time loop as one CUDA graph with conditional WHILE/IF nodes, one "
                              "graph launch and one status read-back per call" if graph else
                              "dirac_step: host-driven loop"),
                   "inner_apply": (["stored coupling values (owner/gather passes)",
                                    "factorised: radial band products x angular coefficients, subgroup form",
                                    "factorised: radial band products x angular coefficients, per-channel form"]
                                   [args.factorised] if args.precision == 2 else None),
                   "assembly": "overlapped with the previous step's solve" if (args.precision == 2 and
                                                                               args.overlap) else "in step",
                   "l2": "inputs larger than L2: %.1f GB of coupling values streamed per operator apply" %
                         (8 * coup / 1e9),
                   "parallelism": "replicas x%d (independent instances, no collective)" % world},
        "iters_per_step": float(np.mean(its)), "max_resid": float(np.max(res)),
        "host_loop": {"value": args.steps / (ms_host / 1000.0), "ms_per_step": ms_host / args.steps,
                      "iters_per_step": float(np.mean(its_h)), "max_resid": float(np.max(res_h)),
                      "launches_per_step": launches / args.steps,
                      "note": "dirac_step on the same op, the next K steps: the graph driver replaces these "
                              "launches and the per-step status read-back by one graph launch per call"},
        "phase_ms_per_step": {k: v / args.steps for k, v in phase_ms.items()},
        "spmv_gbs": (roof32 if roof32 and roof32.get("unit") == "GB/s" else roof)["gbs"],
        "roofline": roof,
        "e2e": {"value": e2e_sps, "unit": "steps/s", "h2d_bytes_per_step": bas.n * 16,
                "d2h_bytes_per_step": bas.n * 16},
        "gpu_launches": launches,
        "clocks": ck,
        "observables": obs,
    }
    if spec:
        line["spectrum"] = spec
    if roof32 and roof32 is not roof:
        line["roofline_apply32" if roof32.get("bound") == "alu" else "roofline_spmv32"] = roof32
    if args.precision != 0 and not args.no_fp64_compare:
        # plain FP64 on the same window and driver: the baseline of speedup_vs_fp64, and the per-result
        # errors of the mixed state against it (same start state, same W + K steps)
        fp64, psi64, op64 = window_run(B, torch, bas, cfg, psi0_h, t0, args.warmup, args.steps, stream, dev, 0,
                                       host_loop=not graph)
        errs, o64 = state_errors(op64, psi64, psi_head)
        fp64["errors_of_headline_vs_fp64"] = errs
        line["fp64_baseline"] = fp64
        line["speedup_vs_fp64"] = value / (fp64["value"] * world)
        if not args.no_compare:
            comp = {"pulse_start": {"t_start": t0, "fp64": fp64,
                                    "precision2": {"value": value, "ms_per_step": ms / args.steps,
                                                   "iters_per_step": float(np.mean(its)),
                                                   "max_resid": float(np.max(res)), "errors_vs_fp64": errs}}}
            # precision 1: the literal form (FP64 refinement residual) on the same window
            p1, psi1, op1 = window_run(B, torch, bas, cfg, psi0_h, t0, args.warmup, args.steps, stream, dev, 1,
                                       host_loop=not graph)
            del op1
            p1["errors_vs_fp64"], _ = state_errors(op64, psi64, psi1, ref_obs=o64)
            p1["speedup_vs_fp64"] = p1["value"] / fp64["value"]
            comp["pulse_start"]["precision1"] = p1
            del psi1, psi64
            # peak-field window: plain FP64, precision 1, precision 2, precision 2 + learned guess
            tp = 0.5 * T
            peak = {"t_start": tp}
            f64p, r64, _op = window_run(B, torch, bas, cfg, psi0_h, tp, args.warmup, args.steps, stream, dev, 0,
                                        host_loop=not graph)
            del _op
            peak["fp64"] = f64p
            o64p = op64.observables(r64, bound=True)
            for name, prec in (("precision1", 1), ("precision2", 2)):
                r, pp, _op = window_run(B, torch, bas, cfg, psi0_h, tp, args.warmup, args.steps, stream, dev, prec,
                                        host_loop=not graph)
                del _op
                r["errors_vs_fp64"], _ = state_errors(op64, r64, pp, ref_obs=o64p)
                r["speedup_vs_fp64"] = r["value"] / f64p["value"]
                peak[name] = r
                del pp
            try:
                net, note = train_guess(B, torch, bas, cfg, 2, args.train_n, args.train_steps)
                r, pp, _op = window_run(B, torch, bas, cfg, psi0_h, tp, args.warmup, args.steps, stream, dev, 2,
                                        guess=2, net=net, host_loop=not graph)
                del _op
                r["errors_vs_fp64"], _ = state_errors(op64, r64, pp, ref_obs=o64p)
                r["speedup_vs_fp64"] = r["value"] / f64p["value"]
                r["training"] = note
                peak["precision2_learned"] = r
                del pp, net
            except Exception as e:   # reported, never required
                peak["precision2_learned"] = {"error": str(e)}
            comp["peak_field"] = peak
            del r64
            if not args.no_batch_leg:
                del op64
                torch.cuda.empty_cache()
                try:
                    bout, bconf, bck = batch_measure(args, world, local, args.batch_n, True, True)
                    comp["batch_peak_field"] = {"result": bout, "config": bconf, "clocks": bck}
                except Exception as e:
                    comp["batch_peak_field"] = {"error": str(e)}
                op64 = None
            line["compare"] = comp
        del op64
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(cfg, float(np.mean(its)), args.cpu_seconds)
        except Exception as e:  # the baseline is reported, never required
            line["cpu_baseline"] = {"error": str(e)}
    line["bench_wall_s"] = time.time() - t_wall0
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
