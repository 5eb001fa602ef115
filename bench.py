"""Benchmark of the forward-model hot path (model cube -> PSF x LSF convolution
-> moments -> masked chi-squared) on the Fabry-Perot-like workload: one
192 x 192 x 48 galaxy (10 km/s channels, PSF FWHM 3 px, LSF FWHM 30 km/s,
S/N < 3 masked) and 400 parameter sets per step -- the live points of one
nested-sampling iteration, evaluated in one batched launch.

A step is one pass of the whole hot path over one batch of 400 models.
The line also carries `fits`: galaxy fits/s of the plain per-galaxy
finite-difference LM (the paper's arrangement) and of the batched forms on
one batch of noiseless mock galaxies, with the recovery they reach.  The
parameter sets are drawn from the uniform prior of the workload (a fresh batch
per step, resident in HBM before timing starts); L2 is flushed (a 256 MiB
write) between timed steps.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbk|reference]

Under torchrun each rank evaluates its own batches (independent models, no
data-path collective); value is the total over ranks divided by the slowest
rank's time.  `--impl reference` times the FP64 CPU oracle on the host cores
instead (a bounded sample of the same workload per step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1510_01815_gb300 import synth  # noqa: E402

METRIC = "model-cube evals/s and galaxy fits/s at matched chi2 (learned+batched vs plain)"
# Minimal lane operations of the line-sampling loop per extended voxel:
# u = fma(e, alpha dv, u0), w = u*u, s0 += g, s1 += g u, s2 += g w on the FMA
# pipe, and g = 2^-w on the MUFU.
FMA_OPS_PER_EXT_VOXEL = 5
MUFU_OPS_PER_EXT_VOXEL = 1
OPS_PER_EXT_VOXEL = FMA_OPS_PER_EXT_VOXEL + MUFU_OPS_PER_EXT_VOXEL
# Minimal FP32 operations of one PSF tap on a moment triplet re-centred
# exactly (s0 += w q0; s1 += w (q1 + D q0); s2 += w (q2 + 2 D q1 + D^2 q0)),
# and of the moments, residuals and chi2 of one data spaxel.
OPS_PER_PSF_TAP = 9
OPS_PER_DATA_SPAXEL = 10
# The split path's PSF passes: each thread's inputs are moved once to a
# reference velocity r (l1 = q1 + d q0, l2 = q2 + d (2 q1 + d q0), d = a - r:
# five FP32 operations per input, 4 + 2R inputs per four outputs), a tap is
# three FMAs (s0 += w q0, s1 += w l1, s2 += w l2), and each output moves its
# sums from r to its own centre once (five operations).
OPS_PER_PSF_TAP_SPLIT = 3
OPS_PER_PSF_INPUT_SPLIT = 5
OPS_PER_PSF_OUTPUT_SPLIT = 5


def split_pass_ops_per_output(taps):
    """FP32 operations of one output of a split-path PSF pass of `taps` taps."""
    return OPS_PER_PSF_TAP_SPLIT * taps + OPS_PER_PSF_INPUT_SPLIT * (3 + taps) / 4.0 + OPS_PER_PSF_OUTPUT_SPLIT
# Per-unit work of the unfolded method (cube + separable PSF x LSF
# convolution + moments) at the Fabry-Perot size, in FP32 instructions per
# data voxel: the line (an ex2 and 3 FP32 per extended voxel, 1.41 extended
# voxels per data voxel), the separable convolution's 13-tap passes on the
# shrinking cube (about 40) and the moments (3) -- about 47.
UNFOLDED_FP32_PER_DATA_VOXEL = 47.0
# DRAM bytes (read + write) of one fused launch of 400 Fabry-Perot models per
# tuning (CTAs per model, threads, persistent), as measured by one-pass ncu
# captures of `bench.py --quick --steps 5 --warmup 2 --tuning <T>` on a
# GB300 (dram__bytes_read.sum + dram__bytes_write.sum of the fused launch);
# reported only for a run at that tuning and with that kernel build.
FUSED_TRAFFIC_400 = {(12, 512, 0): 1433600.0, (12, 512, 1): 1318400.0}
# DRAM bytes (read + write) of one launch of the split path's line stage
# per step size (models per step -> bytes), from a one-pass ncu capture of
# `bench.py --quick --steps 5 --warmup 2` on a GB300 with the current kernel
# build (dram__bytes_read.sum + dram__bytes_write.sum, mean over launches);
# 36 975 B read + 9 604 B written per launch of 80 models, the mean of 60
# launches.
SPLIT_LINE_TRAFFIC = {400: 46579.0}
SPLIT_LINE_TRAFFIC_MODELS = 80  # models per line-stage launch of a 400-model step
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gbk", choices=["gbk", "reference"])
    ap.add_argument("--models", type=int, default=synth.FP_LIVE_POINTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fits", action="store_true", help="skip the galaxy-fit (LM) measurement")
    ap.add_argument("--fit-galaxies", type=int, default=2048)
    ap.add_argument("--fit-plain", type=int, default=256, help="galaxies of the plain LM form in the fits leg")
    ap.add_argument("--no-survey", action="store_true", help="skip the ragged survey-fit measurement")
    ap.add_argument("--survey-galaxies", type=int, default=2048)
    ap.add_argument("--survey-plain", type=int, default=64, help="galaxies the plain survey LM is timed on")
    ap.add_argument("--no-cnn", action="store_true", help="skip the learned-seed (CNN) measurement")
    ap.add_argument("--no-vfield", action="store_true", help="skip the velocity-field (Epinat) measurement")
    ap.add_argument("--no-degeneracy", action="store_true", help="skip the V_t - i degeneracy chi2 maps")
    ap.add_argument("--no-mock", action="store_true", help="skip the mock-dataset recovery study")
    ap.add_argument("--no-ns", action="store_true", help="skip nested sampling of Fabry-Perot galaxies")
    ap.add_argument("--no-jacobian", action="store_true", help="skip the analytic Jacobian kernel timing")
    ap.add_argument("--no-grid", action="store_true", help="skip the full-size nested-grid search")
    ap.add_argument("--mock-galaxies", type=int, default=1000, help="galaxies per noise level of the mock study")
    ap.add_argument("--no-gemm", action="store_true", help="skip the tensor-core GEMM measurement")
    ap.add_argument("--cnn-train", type=int, default=1048576, help="training galaxies of the CNN seed")
    ap.add_argument("--cnn-epochs", type=int, default=2)
    ap.add_argument("--cnn-batch", type=int, default=1024)
    ap.add_argument("--cnn-test", type=int, default=4096, help="held-out galaxies of the seed comparison")
    ap.add_argument("--path", default="split", choices=["fused", "staged", "split"],
                    help="split (default: line and PSF stages through an L2-resident buffer), fused (one "
                         "cluster of CTAs per model) or staged (cube materialised in HBM) evaluation")
    ap.add_argument("--quick", action="store_true", help="kernel timing only (for profiler runs)")
    ap.add_argument("--lm-only", default=None, choices=["survey", "single"],
                    help="run one batched analytic-Jacobian LM fit of the survey (2048 ragged galaxies) or of "
                         "the single-geometry batch (2048 C1 galaxies), print its fits/s and exit (for "
                         "profiler runs)")
    ap.add_argument("--tuning", default=None,
                    help="CTAS,THREADS,PERSISTENT: use this fused-kernel tuning instead of autotuning")
    return ap.parse_args()


def job_throughput(local_ms, units_per_rank, dist=None):
    """Whole-job throughput of a weak-scaling run: the units every rank
    processed, over the slowest rank's time.  Returns (units/s, max ms)."""
    import torch
    world, t = 1, float(local_ms)
    if dist is not None:
        world = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units_per_rank / (t * 1e-3), t


def rank_pool(rank, n, steps):
    """Each rank's own parameter sets (Fabry-Perot prior): disjoint seeds,
    so no two ranks evaluate the same models."""
    rng = np.random.default_rng(7000 + rank)
    return synth.draw_fp_params(rng, n * steps).reshape(steps, n, synth.NPAR)


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def ext_dims(g):
    """(ex, ey, ez) of the extended grid: data grid plus the kernel radii
    R = ceil(4 sigma) on each side (PSF in pixels, LSF in channels)."""
    import math
    s_xy = g.psf_fwhm / 2.3548200450309493
    s_z = g.lsf_fwhm / 2.3548200450309493 / g.dv
    R = math.ceil(g.halo_sigmas * s_xy) if s_xy > 0 else 0
    Rz = math.ceil(g.halo_sigmas * s_z) if (s_z > 0 and g.lsf_mode == 0) else 0
    return g.nx + 2 * R, g.ny + 2 * R, g.nz + 2 * Rz


# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "0x1"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
FIT_FREE = synth.FREE_DEFAULT


def fit_batch(gbk, torch, n, seed, device):
    """n noiseless single-galaxy mocks (32 x 32 x 64) with truths spread over a
    32-pixel frame, their maps from the library, and 20 %-perturbed starts
    clipped to the fit bounds (i in 1-89 deg, Sec. 3.1)."""
    g = synth.SINGLE_GEOM
    rng = np.random.default_rng(seed)
    truth = np.tile(synth.SINGLE_TRUTH, (n, 1))
    truth[:, synth.X0] = rng.uniform(13.0, 18.0, n)
    truth[:, synth.Y0] = rng.uniform(13.0, 18.0, n)
    truth[:, synth.PA] = rng.uniform(0.0, 180.0, n)
    truth[:, synth.INCL] = rng.uniform(30.0, 70.0, n)
    truth[:, synth.VMAX] = rng.uniform(100.0, 300.0, n)
    truth[:, synth.RT] = rng.uniform(2.0, 5.0, n)
    truth[:, synth.SIG0] = rng.uniform(20.0, 60.0, n)
    maps = gbk.eval_maps(g, torch.from_numpy(truth), device=device).cpu().numpy()
    shape = (g.ny, g.nx)
    wv, ws = synth.weights(shape, 5.0)
    ones = np.ones(shape, np.uint8)
    obs = [gbk.Obs.from_numpy(maps[i, 1], maps[i, 2], wv, ws, ones, device=device) for i in range(n)]
    lo = np.tile(truth[0], (n, 1))
    hi = lo.copy()
    lo[:, synth.X0], hi[:, synth.X0] = 0.0, 31.0
    lo[:, synth.Y0], hi[:, synth.Y0] = 0.0, 31.0
    lo[:, synth.PA], hi[:, synth.PA] = -360.0, 720.0
    lo[:, synth.INCL], hi[:, synth.INCL] = 1.0, 89.0
    lo[:, synth.VSYS], hi[:, synth.VSYS] = -200.0, 200.0
    lo[:, synth.VMAX], hi[:, synth.VMAX] = 1.0, 600.0
    lo[:, synth.RT], hi[:, synth.RT] = 0.05, 30.0
    lo[:, synth.SIG0], hi[:, synth.SIG0] = 1.0, 300.0
    lo[:, synth.I0] = hi[:, synth.I0] = truth[:, synth.I0]
    lo[:, synth.H] = hi[:, synth.H] = truth[:, synth.H]
    p0 = np.array([synth.perturb(rng, truth[i], FIT_FREE, 0.2, lo[i], hi[i]) for i in range(n)])
    return g, truth, obs, p0, lo, hi


def run_fits(gbk, torch, n, n_plain, device, forms):
    """Galaxy fits/s of the LM forms on the same noiseless batch (the plain
    one-galaxy-at-a-time form on its first n_plain galaxies), with the
    recovery the paper's thresholds ask for (|dV_t| < 2 km/s, |dPA| < 1 deg).
    forms: (name, mode, Jacobian, kernel path)."""
    g, truth, obs, p0, lo, hi = fit_batch(gbk, torch, n, 4242, device)
    out = {"workload": "%d noiseless 32x32x64 mock galaxies (the plain form: the first %d), 20%% perturbed "
                       "starts, %d free parameters" % (n, n_plain, len(FIT_FREE))}
    for name, mode, jac, path in forms:
        sub = n_plain if mode == gbk.LM_PLAIN else n
        opts = gbk.lm_opts(max_iter=200, jacobian=jac, mode=mode, free=FIT_FREE, path=path)
        gbk.fit_lm(g, obs[:4], p0[:4], lo[:4], hi[:4], opts, device=device)  # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        q, c, it, st = gbk.fit_lm(g, obs[:sub], p0[:sub], lo[:sub], hi[:sub], opts, device=device)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        dv = np.abs(q[:, synth.VMAX] - truth[:sub, synth.VMAX])
        dpa = np.abs((q[:, synth.PA] - truth[:sub, synth.PA] + 180.0) % 360.0 - 180.0)
        out[name] = {"galaxies": sub, "kernels": "two-stage where served" if path == gbk.PATH_AUTO else "cluster",
                     "fits_per_s": sub / dt, "seconds": dt, "p50_iters": float(np.percentile(it, 50)),
                     "p99_iters": float(np.percentile(it, 99)),
                     "recovered_frac": float(np.mean((dv < 2.0) & (dpa < 1.0))),
                     "median_dvmax": float(np.median(dv)), "median_dpa": float(np.median(dpa)),
                     "median_chi2": float(np.median(c))}
    if "plain_fd" in out:
        for name in out:
            if isinstance(out[name], dict) and name != "plain_fd":
                out[name]["speedup_vs_plain"] = out[name]["fits_per_s"] / out["plain_fd"]["fits_per_s"]
    return out


def survey_batch(gbk, torch, n, seed, device):
    """n survey galaxies of different geometry (24-96 spaxels square, 32-128
    channels, PSF 4 px, LSF 20-60 km/s, channel width keeping the line in
    the band), maps from the library at the true parameters, seeded noise
    (5 km/s on v, 5 sqrt(2) on sigma), 2 % dead fibres, 20 %-perturbed
    starts inside the fit bounds."""
    rng = np.random.default_rng(seed)
    gal = synth.draw_survey(rng, n)
    geoms = [g for g, _ in gal]
    truth = np.array([p for _, p in gal])
    maps, _, _ = gbk.survey_eval(geoms, truth, device=device)
    obs, lo, hi, p0 = [], [], [], []
    for i, g in enumerate(geoms):
        m = maps[i].cpu().numpy()
        shape = (g.ny, g.nx)
        v = (m[1] + synth.gaussian_noise(rng, shape, 5.0)).astype(np.float32)
        s = (m[2] + synth.gaussian_noise(rng, shape, 5.0 * np.sqrt(2.0))).astype(np.float32)
        wv, ws = synth.weights(shape, 5.0)
        mask = synth.dead_fibre_mask(rng, shape).astype(np.uint8)
        obs.append(gbk.Obs.from_numpy(v, s, wv, ws, mask, device=device))
        l, h = truth[i].copy(), truth[i].copy()
        l[synth.X0], h[synth.X0] = 0.0, g.nx - 1.0
        l[synth.Y0], h[synth.Y0] = 0.0, g.ny - 1.0
        l[synth.PA], h[synth.PA] = -360.0, 720.0
        l[synth.INCL], h[synth.INCL] = 1.0, 89.0
        l[synth.VSYS], h[synth.VSYS] = -200.0, 200.0
        l[synth.VMAX], h[synth.VMAX] = 1.0, 600.0
        l[synth.RT], h[synth.RT] = 0.05, 60.0
        l[synth.SIG0], h[synth.SIG0] = 1.0, 300.0
        lo.append(l)
        hi.append(h)
        p0.append(synth.perturb(rng, truth[i], FIT_FREE, 0.2, l, h))
    return geoms, truth, obs, np.array(p0), np.array(lo), np.array(hi)


def run_survey(gbk, torch, n, n_plain, device):
    """Survey-scale fitting: galaxy fits/s of the batched LM over a ragged
    batch against the plain one-galaxy-at-a-time LM, iterations p50/p99,
    recovery, and the ragged evaluator's throughput."""
    geoms, truth, obs, p0, lo, hi = survey_batch(gbk, torch, n, 4, device)
    pix = sum(g.nx * g.ny for g in geoms)
    vox = sum(g.nx * g.ny * g.nz for g in geoms)
    out = {"workload": "%d survey galaxies, 24-96 spaxels square x 32-128 channels (log-uniform), PSF 4 px, "
                       "LSF 20-60 km/s, noise 5 / 5 sqrt(2) km/s, 2%% dead fibres, 20%% perturbed starts, "
                       "%d free parameters" % (n, len(FIT_FREE)),
           "data_voxels": vox, "spaxels": pix}
    # ragged evaluator: one chi2 per galaxy
    obs_dev, _keep = gbk.obs_array(obs, device)
    d_p = torch.from_numpy(truth).to(device)
    d_c = torch.empty(n, dtype=torch.float64, device=device)
    ws = torch.empty(max(gbk.gbk_survey_workspace_bytes(geoms), 1), dtype=torch.uint8, device=device)
    cg = gbk.cgeoms(geoms)  # marshalled once; the library caches the plan

    def time_eval(reps=20):
        for _ in range(3):
            gbk.gbk_survey_eval(cg, d_p, obs_dev, None, d_c, None, ws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            gbk.gbk_survey_eval(cg, d_p, obs_dev, None, d_c, None, ws)
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    # launch shapes: one launch per cluster-size group, the default single
    # persistent launch, and the autotuner's choice (kept for the fits below)
    shapes = {}
    gbk.gbk_survey_set_tuning(geoms, 0)
    shapes["per_group_launches"] = time_eval()
    gbk.gbk_survey_set_tuning(geoms, None)
    t_def = gbk.gbk_survey_get_tuning(geoms)
    shapes["one_launch_%dx%d" % (t_def["cluster_ctas"], t_def["threads"])] = time_eval()
    best = gbk.gbk_survey_autotune(geoms, d_p, obs_dev, d_c, ws)
    ms = time_eval()
    out["eval"] = {"ms_per_survey": ms, "evals_per_s": n / (ms * 1e-3), "data_voxels_per_s": vox / (ms * 1e-3),
                   "tuning": best, "shapes_ms": shapes,
                   "note": "time per call: cached plan, geometry-table upload, counter reset and the fused "
                           "launch(es); tuning = the survey autotuner's choice, used by the fits below"}
    for name, mode, jac, sub, path in (("batched_tangent", gbk.LM_BATCHED, gbk.JAC_TANGENT, n, gbk.PATH_AUTO),
                                       ("batched_tangent_cluster_kernels", gbk.LM_BATCHED, gbk.JAC_TANGENT, n,
                                        gbk.PATH_FUSED),
                                       ("batched_fd", gbk.LM_BATCHED, gbk.JAC_FD_FORWARD, n, gbk.PATH_AUTO),
                                       ("plain_fd", gbk.LM_PLAIN, gbk.JAC_FD_FORWARD, n_plain, gbk.PATH_AUTO)):
        opts = gbk.lm_opts(max_iter=200, jacobian=jac, mode=mode, free=FIT_FREE, path=path)
        gbk.survey_fit_lm(geoms[:4], obs[:4], p0[:4], lo[:4], hi[:4], opts, device=device)  # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        q, c, it, st = gbk.survey_fit_lm(geoms[:sub], obs[:sub], p0[:sub], lo[:sub], hi[:sub], opts, device=device)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        tr = truth[:sub]
        dv = np.abs(q[:, synth.VMAX] - tr[:, synth.VMAX])
        dpa = np.abs((q[:, synth.PA] - tr[:, synth.PA] + 180.0) % 360.0 - 180.0)
        out[name] = {"galaxies": sub, "fits_per_s": sub / dt, "seconds": dt,
                     "p50_iters": float(np.percentile(it, 50)), "p99_iters": float(np.percentile(it, 99)),
                     "converged_frac": float(np.mean(np.isin(st, [1, 2]))),
                     "recovered_frac": float(np.mean((dv < 2.0) & (dpa < 1.0))),
                     "median_dvmax": float(np.median(dv)), "median_dpa": float(np.median(dpa))}
    for name in ("batched_tangent", "batched_tangent_cluster_kernels", "batched_fd"):
        out[name]["speedup_vs_plain"] = out[name]["fits_per_s"] / out["plain_fd"]["fits_per_s"]
    out["batched_tangent"]["note"] = ("every galaxy on the ragged two-stage analytic Jacobian; trial points on the "
                                      "survey's cluster evaluator")
    out["batched_tangent_cluster_kernels"]["note"] = ("cluster Jacobian kernel for the galaxies whose halo rows fit "
                                                      "a CTA's shared memory, finite differences for the wider ones")
    return out


CNN_LAYER_MNK = ((1024, 32, 16), (256, 64, 128), (64, 128, 256), (16, 256, 512), (1, 256, 4096), (1, 16, 256))


def cnn_flops_per_sample():
    """GEMM flops of one training sample: forward, weight gradient (with the
    bias column) and input gradient of every layer but the first."""
    f = 0
    for l, (rows, c, k) in enumerate(CNN_LAYER_MNK):
        f += 2 * rows * c * k            # forward
        f += 2 * rows * c * (k + 1)      # dW (and db)
        if l > 0:
            f += 2 * rows * c * k        # dX
    return f


def cnn_data(gbk, torch, n, seed, device, chunk=65536, continuum=False):
    """n synthetic galaxies of the CNN workload: parameters from the prior,
    maps from the library (64 x 64 x 64 cubes), observations with 5 km/s
    noise and 2 % dead fibres from the library's counter-based streams (and,
    on request, the continuum maps m0)."""
    rng = np.random.default_rng(seed)
    p = synth.draw_cnn_params(rng, n)
    dp = torch.from_numpy(p).to(device)
    v = torch.empty((n, 64, 64), dtype=torch.float32, device=device)
    s = torch.empty_like(v)
    m = torch.empty((n, 64, 64), dtype=torch.uint8, device=device)
    t = torch.empty((n, 10), dtype=torch.float32, device=device)
    c = torch.empty_like(v) if continuum else None
    for i in range(0, n, chunk):
        j = min(n, i + chunk)
        maps = gbk.eval_maps(synth.CNN_GEOM, dp[i:j], device=device)
        gbk.gbk_cnn_synth_obs(maps, seed * 1000003 + i, 5.0, 0.02, v[i:j], s[i:j], m[i:j])
        if continuum:
            c[i:j] = maps[:, 0]
        del maps
    gbk.gbk_cnn_targets(dp, t)
    return (p, v, s, m, t, c) if continuum else (p, v, s, m, t)


def run_cnn(gbk, torch, n_train, epochs, batch, n_test, n_plain, device, n_ns=8):
    """Learned seed: train the CNN on synthetic maps, then compare batched LM
    (analytic Jacobian) started from its predictions with batched LM started
    from the Sec. 2.1.9 values and from 20 %-perturbed truths, and with the
    plain finite-difference LM, on held-out galaxies (fits/s, iterations,
    recovery)."""
    out = {"workload": "%d training + %d held-out galaxies, 64x64 maps of 64x64x64 cubes (dv 20, PSF 2.5 px, "
                       "LSF 30 km/s), noise 5 / 5 sqrt(2) km/s, 2%% dead fibres" % (n_train, n_test)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, v, s, m, t = cnn_data(gbk, torch, n_train, 11, device)
    torch.cuda.synchronize()
    out["data_seconds"] = time.perf_counter() - t0
    net = gbk.CnnSeed(batch, seed=3, device=device)
    steps_per_epoch = n_train // batch
    lr0 = 1e-3
    for w in range(3):  # warm-up steps (not timed)
        net.train_step(v[:batch], s[:batch], m[:batch], t[:batch], lr0)
    first_loss = float(net.loss)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    total = epochs * steps_per_epoch
    for it in range(total):
        i = (it % steps_per_epoch) * batch
        lr = lr0 * (0.1 if it >= 0.8 * total else 1.0)
        net.train_step(v[i:i + batch], s[i:i + batch], m[i:i + batch], t[i:i + batch], lr)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    flops = cnn_flops_per_sample() * batch * total
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    out["train"] = {"steps": total, "batch": batch, "epochs": epochs, "ms": ms, "samples_per_s": batch * total / (ms * 1e-3),
                    "gemm_tflops": flops / (ms * 1e-3) / 1e12, "bf16_peak_tflops": peak,
                    "tensor_frac": flops / (ms * 1e-3) / 1e12 / peak, "first_loss": first_loss,
                    "final_loss": float(net.loss),
                    "note": "whole training step (encode, 6 forward, 6+5 backward GEMMs, split-K sums, Adam) per "
                            "launch sequence; flops count the GEMMs only; peak = measured cuBLAS bf16 sustained"}
    del v, s, m, t
    # held-out galaxies (seed 5)
    ptest, vt, st, mt, _, ct = cnn_data(gbk, torch, n_test, 5, device, continuum=True)
    torch.cuda.synchronize()
    a.record()
    pred = net.predict(vt, st, mt)
    b.record()
    b.synchronize()
    out["predict"] = {"galaxies": n_test, "ms": a.elapsed_time(b)}
    pred = pred.cpu().numpy()
    g = synth.CNN_GEOM
    wv, ws_ = synth.weights((64, 64), 5.0)
    dwv, dws = torch.from_numpy(wv).to(device), torch.from_numpy(ws_).to(device)
    obs = [gbk.Obs(vt[i], st[i], dwv, dws, mt[i]) for i in range(n_test)]
    lo = np.tile(ptest[0], (n_test, 1))
    hi = lo.copy()
    lo[:, synth.X0], hi[:, synth.X0] = 0.0, 63.0
    lo[:, synth.Y0], hi[:, synth.Y0] = 0.0, 63.0
    lo[:, synth.PA], hi[:, synth.PA] = -360.0, 720.0
    lo[:, synth.INCL], hi[:, synth.INCL] = 1.0, 89.0
    lo[:, synth.VSYS], hi[:, synth.VSYS] = -200.0, 200.0
    lo[:, synth.VMAX], hi[:, synth.VMAX] = 1.0, 600.0
    lo[:, synth.RT], hi[:, synth.RT] = 0.05, 30.0
    lo[:, synth.SIG0], hi[:, synth.SIG0] = 1.0, 300.0
    for k in (synth.I0, synth.H):  # fixed at the truth in every fit (Sec. 2.1.9)
        lo[:, k] = hi[:, k] = ptest[:, k]
    seed_p = np.clip(pred, lo, hi)
    seed_p[:, synth.I0], seed_p[:, synth.H] = ptest[:, synth.I0], ptest[:, synth.H]
    rng = np.random.default_rng(55)
    pert = np.array([synth.perturb(rng, ptest[i], FIT_FREE, 0.2, lo[i], hi[i]) for i in range(n_test)])
    # the paper's own starting point (Sec. 2.1.9), measured on the maps
    obs_dev, _keep = gbk.obs_array(obs, device)
    heur = torch.empty((n_test, synth.NPAR), dtype=torch.float64, device=device)
    gbk.gbk_initial_guess(g, obs_dev, torch.from_numpy(ptest).to(device), heur, ct)
    heur = np.clip(heur.cpu().numpy(), lo, hi)

    def err(q, tr):
        dv = np.abs(q[:, synth.VMAX] - tr[:, synth.VMAX])
        dpa = np.abs((q[:, synth.PA] - tr[:, synth.PA] + 180.0) % 360.0 - 180.0)
        return dv, dpa

    dv0, dpa0 = err(seed_p, ptest)
    out["seed_error"] = {"median_dvmax": float(np.median(dv0)), "median_dpa": float(np.median(dpa0)),
                         "p90_dvmax": float(np.percentile(dv0, 90)), "p90_dpa": float(np.percentile(dpa0, 90))}
    dvh, dpah = err(heur, ptest)
    out["heuristic_start_error"] = {"median_dvmax": float(np.median(dvh)), "median_dpa": float(np.median(dpah)),
                                    "p90_dvmax": float(np.percentile(dvh, 90)),
                                    "p90_dpa": float(np.percentile(dpah, 90))}
    fits = {}
    # batched forms: the analytic Jacobian; the plain form: the paper's
    # finite differences.  Each form is warmed up on a few galaxies first
    # (graph capture and launch configurations are set up once per form).
    for name, mode, start, sub in (("batched_cnn_seed", gbk.LM_BATCHED, seed_p, n_test),
                                   ("batched_heuristic", gbk.LM_BATCHED, heur, n_test),
                                   ("batched_perturbed", gbk.LM_BATCHED, pert, n_test),
                                   ("plain_perturbed", gbk.LM_PLAIN, pert, n_plain)):
        jac = gbk.JAC_TANGENT if mode == gbk.LM_BATCHED else gbk.JAC_FD_FORWARD
        opts = gbk.lm_opts(max_iter=200, jacobian=jac, mode=mode, free=FIT_FREE)
        gbk.fit_lm(g, obs[:4], start[:4], lo[:4], hi[:4], opts, device=device)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q, c, it, stt = gbk.fit_lm(g, obs[:sub], start[:sub], lo[:sub], hi[:sub], opts, device=device)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dv, dpa = err(q, ptest[:sub])
        fits[name] = q
        out[name] = {"galaxies": sub, "fits_per_s": sub / dt, "jacobian": "analytic" if jac == gbk.JAC_TANGENT else
                     "forward differences", "p50_iters": float(np.percentile(it, 50)),
                     "mean_iters": float(np.mean(it)), "max_iters": int(np.max(it)),
                     "p99_iters": float(np.percentile(it, 99)), "converged_frac": float(np.mean(np.isin(stt, [1, 2]))),
                     "recovered_frac": float(np.mean((dv < 2.0) & (dpa < 1.0))),
                     "median_dvmax": float(np.median(dv)), "median_dpa": float(np.median(dpa))}
    out["batched_cnn_seed"]["speedup_vs_plain"] = out["batched_cnn_seed"]["fits_per_s"] / out["plain_perturbed"]["fits_per_s"]
    # the seed with the plain fit as its fallback: galaxies whose seeded fit
    # does not converge or ends above 1.5 x the number of residuals are
    # refitted from the Sec. 2.1.9 start, and the lower chi2 is kept
    nres = 2.0 * (mt != 0).sum(dim=(1, 2)).double().cpu().numpy()
    opts = gbk.lm_opts(max_iter=200, jacobian=gbk.JAC_TANGENT, mode=gbk.LM_BATCHED, free=FIT_FREE)
    gbk.fit_lm_fallback(g, obs[:4], seed_p[:4], heur[:4], lo[:4], hi[:4], opts, chi2_accept=1.5 * nres[:4],
                        device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q, c, it, stt, used = gbk.fit_lm_fallback(g, obs, seed_p, heur, lo, hi, opts, chi2_accept=1.5 * nres,
                                              device=device)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dv, dpa = err(q, ptest)
    out["batched_cnn_seed_fallback"] = {
        "galaxies": n_test, "fits_per_s": n_test / dt, "refitted_frac": float(np.mean(used > 0)),
        "fallback_kept_frac": float(np.mean(used == 1)), "chi2_accept": "1.5 x unmasked residuals",
        "converged_frac": float(np.mean(np.isin(stt, [1, 2]))), "within_accept_frac": float(np.mean(c <= 1.5 * nres)),
        "recovered_frac": float(np.mean((dv < 2.0) & (dpa < 1.0))),
        "median_dvmax": float(np.median(dv)), "median_dpa": float(np.median(dpa))}
    # the plain fit as the judge of the seed's error (what real data allow):
    # the seed against the fit from the Sec. 2.1.9 start
    dvj, dpaj = err(seed_p, fits["batched_heuristic"])
    out["seed_error_vs_plain_fit"] = {"median_dvmax": float(np.median(dvj)), "median_dpa": float(np.median(dpaj)),
                                      "p90_dvmax": float(np.percentile(dvj, 90)),
                                      "p90_dpa": float(np.percentile(dpaj, 90))}
    out["nested_sampling"] = run_cnn_ns(gbk, torch, g, obs, ptest, pred, lo, hi, n_ns, device)
    return out


def run_cnn_ns(gbk, torch, g, obs, truth, pred, lo, hi, n_gal, device, n_live=200, batch=50):
    """Nested sampling (Sec. 2.3.2) of n_gal held-out galaxies over the
    full prior box against a box centred on the network's prediction with
    half-widths 3x the seed's 90th-percentile error on the other held-out
    galaxies: likelihood evaluations, wall time and recovery."""
    cal = slice(n_gal, None)
    err = np.abs(pred[cal] - truth[cal])
    err[:, synth.PA] = np.abs((pred[cal, synth.PA] - truth[cal, synth.PA] + 180.0) % 360.0 - 180.0)
    half = 3.0 * np.percentile(err, 90, axis=0)
    res = {"full_prior": [], "cnn_box": []}
    inside = 0
    for j in range(n_gal):
        flo, fhi = lo[j].copy(), hi[j].copy()
        for k, (a_, b_) in synth.CNN_RANGES.items():
            if k != synth.H:
                flo[k], fhi[k] = a_, b_
        slo, shi = flo.copy(), fhi.copy()
        for k in FIT_FREE:
            if k == synth.PA:
                slo[k], shi[k] = pred[j, k] - half[k], pred[j, k] + half[k]
            else:
                slo[k], shi[k] = max(flo[k], pred[j, k] - half[k]), min(fhi[k], pred[j, k] + half[k])
        dpa0 = abs((pred[j, synth.PA] - truth[j, synth.PA] + 180.0) % 360.0 - 180.0)
        inside += int(all(slo[k] <= truth[j, k] <= shi[k] for k in FIT_FREE if k != synth.PA)
                      and dpa0 <= half[synth.PA])
        for name, (blo, bhi) in (("full_prior", (flo, fhi)), ("cnn_box", (slo, shi))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = gbk.gbk_nested_sample(g, obs[j], blo, bhi, n_live=n_live, batch=batch, tol=0.5, seed=100 + j,
                                      device=device)
            dt = time.perf_counter() - t0
            dv = abs(r["mean"][synth.VMAX] - truth[j, synth.VMAX])
            dpa = abs((r["mean"][synth.PA] - truth[j, synth.PA] + 180.0) % 360.0 - 180.0)
            res[name].append((r["n_eval"], r["n_iter"], dt, dv, dpa))
    out = {"galaxies": n_gal, "n_live": n_live, "batch": batch, "truth_in_cnn_box_frac": inside / n_gal,
           "cnn_box_half_widths": {synth.PARAM_NAMES[k]: float(half[k]) for k in FIT_FREE}}
    for name, rows in res.items():
        a_ = np.array(rows)
        out[name] = {"mean_evals": float(a_[:, 0].mean()), "mean_iters": float(a_[:, 1].mean()),
                     "seconds_per_galaxy": float(a_[:, 2].mean()), "median_dvmax": float(np.median(a_[:, 3])),
                     "median_dpa": float(np.median(a_[:, 4])),
                     "recovered_frac": float(np.mean((a_[:, 3] < 2.0) & (a_[:, 4] < 1.0)))}
    out["eval_ratio"] = out["cnn_box"]["mean_evals"] / out["full_prior"]["mean_evals"]
    out["speedup"] = out["full_prior"]["seconds_per_galaxy"] / out["cnn_box"]["seconds_per_galaxy"]
    return out


def run_vfield(gbk, torch, n_models, n_fit, n_plain, device):
    """Velocity-field strategy with the Epinat curve (the GHASP setting,
    Sec. 4.2): 256 x 256 fields, evaluation throughput, and batched vs plain
    LM over the nine free parameters from 10 %-perturbed starts on fields
    with 5 km/s noise."""
    g = synth.Geometry(256, 256, 1, 10.0, model=2)
    rng = np.random.default_rng(21)

    def draw(n):
        p = np.zeros((n, synth.NPAR))
        p[:, 0] = rng.uniform(115, 140, n)
        p[:, 1] = rng.uniform(115, 140, n)
        p[:, 2] = rng.uniform(0, 360, n)
        p[:, 3] = rng.uniform(30, 70, n)
        p[:, 4] = rng.uniform(-50, 50, n)
        p[:, 5] = rng.uniform(100, 300, n)
        p[:, 6] = rng.uniform(5, 30, n)
        p[:, 7] = 30.0
        p[:, 8] = rng.uniform(0.6, 2.5, n)
        p[:, 9] = rng.uniform(0.5, 1.5, n)
        return p

    truth = draw(n_models)
    maps = gbk.eval_maps(g, torch.from_numpy(truth[:1]), device=device).cpu().numpy()[0]
    wv, ws_ = synth.weights((256, 256), 5.0)
    ws_[:] = 0.0  # velocity only: the nine-parameter problem has no dispersion model
    v = (maps[1] + synth.gaussian_noise(rng, (256, 256), 5.0)).astype(np.float32)
    obs = gbk.Obs.from_numpy(v, maps[2], wv, ws_, np.ones((256, 256), np.uint8), device=device)
    d_p = torch.from_numpy(truth).to(device)
    c2 = torch.empty(n_models, dtype=torch.float64, device=device)
    for _ in range(3):
        gbk.gbk_chi2(g, d_p, obs, c2, None, gbk.PATH_FUSED, None)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(20):
        gbk.gbk_chi2(g, d_p, obs, c2, None, gbk.PATH_FUSED, None)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / 20
    out = {"workload": "Epinat velocity fields 256x256 (nine free parameters), %d models per launch" % n_models,
           "eval": {"ms_per_launch": ms, "evals_per_s": n_models / (ms * 1e-3),
                    "pixels_per_s": n_models * 65536 / (ms * 1e-3)}}
    # fits: fields of n_fit galaxies with 5 km/s noise
    ft = draw(n_fit)
    fm = gbk.eval_maps(g, torch.from_numpy(ft), device=device)
    noise = rng.normal(0.0, 5.0, size=(n_fit, 256, 256)).astype(np.float32)
    fm[:, 1] += torch.from_numpy(noise).to(device)
    wz = torch.zeros((256, 256), dtype=torch.float32, device=device)
    dwv = torch.from_numpy(wv).to(device)
    ones = torch.ones((256, 256), dtype=torch.uint8, device=device)
    fobs = [gbk.Obs(fm[i, 1], fm[i, 2], dwv, wz, ones) for i in range(n_fit)]
    free = (0, 1, 2, 3, 4, 5, 6, 8, 9)
    lo, hi = ft.copy(), ft.copy()
    for k, (l, h) in {0: (0, 255), 1: (0, 255), 2: (-360, 720), 3: (1, 89), 4: (-200, 200), 5: (1, 600),
                      6: (0.05, 100), 8: (0.1, 5), 9: (0.05, 5)}.items():
        lo[:, k], hi[:, k] = l, h
    p0 = np.array([synth.perturb(rng, ft[i], free, 0.1, lo[i], hi[i]) for i in range(n_fit)])
    for name, mode, jac, sub in (("batched_tangent", gbk.LM_BATCHED, gbk.JAC_TANGENT, n_fit),
                                 ("batched_fd", gbk.LM_BATCHED, gbk.JAC_FD_FORWARD, n_fit),
                                 ("plain_fd", gbk.LM_PLAIN, gbk.JAC_FD_FORWARD, n_plain)):
        opts = gbk.lm_opts(max_iter=200, mode=mode, free=free, jacobian=jac)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q, c, it, st = gbk.fit_lm(g, fobs[:sub], p0[:sub], lo[:sub], hi[:sub], opts, device=device)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dv = np.abs(q[:, 5] - ft[:sub, 5])
        dpa = np.abs((q[:, 2] - ft[:sub, 2] + 180.0) % 360.0 - 180.0)
        out[name] = {"galaxies": sub, "fits_per_s": sub / dt, "p50_iters": float(np.percentile(it, 50)),
                     "p99_iters": float(np.percentile(it, 99)), "converged_frac": float(np.mean(np.isin(st, [1, 2]))),
                     "median_dpa": float(np.median(dpa)), "median_dvt": float(np.median(dv))}
    for name in ("batched_tangent", "batched_fd"):
        out[name]["speedup_vs_plain"] = out[name]["fits_per_s"] / out["plain_fd"]["fits_per_s"]
    return out


# Recovery thresholds of the clean mock dataset (Sec. 4.1): x0, y0 < 1 px,
# PA < 1 deg, i < 1 deg, r_t < 1 px, V_t < 5 km/s, sigma0 < 1 km/s.
MOCK_THRESHOLDS = {synth.X0: 1.0, synth.Y0: 1.0, synth.PA: 1.0, synth.INCL: 1.0, synth.RT: 1.0, synth.VMAX: 5.0,
                   synth.SIG0: 1.0}


def mock_study(gbk, torch, n, noise, seed, device):
    """The mock-dataset study of Sec. 3.1 / 4.1 at one noise level: n
    galaxies over the parameter space of the mock dataset (32 - 96 spaxels,
    PSF 4 px, LSF 20 - 60 km/s, V_sys = 0), maps from the library at the
    truth plus Gaussian noise (noise on v, sqrt(2) noise on sigma; weights
    for E = max(noise, 1)), 2 % dead fibres, batched LM with the analytic
    (ragged two-stage) Jacobian from 20 %-perturbed starts.  Returns the
    truths, fits, iterations, statuses and 1-sigma errors from the Fisher
    matrix J^T J of the analytic Jacobian at the fit (None at zero noise)."""
    rng = np.random.default_rng(seed)
    gal = synth.draw_survey(rng, n, nxy_range=(32, 96))
    geoms = [g for g, _ in gal]
    truth = np.array([p for _, p in gal])
    maps, _, _ = gbk.survey_eval(geoms, truth, device=device)
    e = max(noise, 1.0)
    obs, lo, hi, p0 = [], [], [], []
    for i, g in enumerate(geoms):
        m = maps[i].cpu().numpy()
        shape = (g.ny, g.nx)
        v = (m[1] + synth.gaussian_noise(rng, shape, noise)).astype(np.float32)
        s = (m[2] + synth.gaussian_noise(rng, shape, noise * np.sqrt(2.0))).astype(np.float32)
        wv, ws = synth.weights(shape, e)
        mask = synth.dead_fibre_mask(rng, shape).astype(np.uint8)
        obs.append(gbk.Obs.from_numpy(v, s, wv, ws, mask, device=device))
        l, h = truth[i].copy(), truth[i].copy()
        l[synth.X0], h[synth.X0] = 0.0, g.nx - 1.0
        l[synth.Y0], h[synth.Y0] = 0.0, g.ny - 1.0
        l[synth.PA], h[synth.PA] = -360.0, 720.0
        l[synth.INCL], h[synth.INCL] = 1.0, 89.0
        l[synth.VSYS], h[synth.VSYS] = -200.0, 200.0
        l[synth.VMAX], h[synth.VMAX] = 1.0, 600.0
        l[synth.RT], h[synth.RT] = 0.05, 60.0
        l[synth.SIG0], h[synth.SIG0] = 1.0, 300.0
        lo.append(l)
        hi.append(h)
        p0.append(synth.perturb(rng, truth[i], FIT_FREE, 0.2, l, h))
    opts = gbk.lm_opts(max_iter=200, jacobian=gbk.JAC_TANGENT, free=FIT_FREE)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q, c, it, st = gbk.survey_fit_lm(geoms, obs, np.array(p0), np.array(lo), np.array(hi), opts, device=device)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    err = None
    if noise > 0:
        nf = len(FIT_FREE)
        err = np.full((n, nf), np.nan)
        jtj = gbk.survey_jacobian(geoms, q, obs, FIT_FREE, device=device)[0].cpu().numpy()
        for i in range(n):
            try:
                err[i] = np.sqrt(np.maximum(np.diag(np.linalg.inv(jtj[i])), 0.0))
            except np.linalg.LinAlgError:
                pass
    return truth, q, it, st, err, dt


def mock_residuals(truth, q):
    """|fit - truth| per parameter, PA wrapped to (-180, 180]."""
    d = np.abs(q - truth)
    d[:, synth.PA] = np.abs((q[:, synth.PA] - truth[:, synth.PA] + 180.0) % 360.0 - 180.0)
    return d


def run_mock_study(gbk, torch, n, device):
    """Recovery statistics of the mock dataset (Sec. 4.1, the analogues of
    the paper's tables of recovered counts, median residuals and
    standardised residuals) at 0, 1, 5 and 20 km/s of velocity noise."""
    names = synth.PARAM_NAMES
    out = {"workload": "%d mock galaxies per noise level (Sec. 3.1 parameter space: 32-96 spaxels, 32-128 "
                       "channels, PSF 4 px, LSF 20-60 km/s, V_sys = 0), 2%% dead fibres, 20%% perturbed starts, "
                       "batched LM with the analytic Jacobian; 1-sigma errors from its J^T J at the fit" % n}
    for noise in (0.0, 1.0, 5.0, 20.0):
        truth, q, it, st, err, dt = mock_study(gbk, torch, n, noise, 31 + int(noise), device)
        d = mock_residuals(truth, q)
        r = {"fits_per_s": n / dt, "converged_frac": float(np.mean(np.isin(st, [1, 2]))),
             "p50_iters": float(np.median(it)), "p99_iters": float(np.percentile(it, 99)),
             "median_residual": {names[k]: float(np.median(d[:, k])) for k in FIT_FREE}}
        if noise == 0:
            r["within_thresholds"] = {names[k]: int(np.sum(d[:, k] < t)) for k, t in MOCK_THRESHOLDS.items()}
        else:
            z = np.abs(q[:, list(FIT_FREE)] - truth[:, list(FIT_FREE)])
            z[:, FIT_FREE.index(synth.PA)] = d[:, synth.PA]
            with np.errstate(divide="ignore", invalid="ignore"):
                z = z / err  # a zero error (a degenerate J^T J) gives inf: such fits are left out
            ok = np.isfinite(z).all(axis=1)
            r["standardised_within_1sigma"] = {names[k]: float(np.mean(z[ok, j] < 1.0)) for j, k in enumerate(FIT_FREE)}
            r["standardised_within_2sigma"] = {names[k]: float(np.mean(z[ok, j] < 2.0)) for j, k in enumerate(FIT_FREE)}
            r["errors_finite_frac"] = float(np.mean(ok))
        out["noise_%g" % noise] = r
    return out


def run_ns_fp(gbk, torch, device, n_gal=2, n_live=400, batch=100):
    """Nested sampling (Sec. 2.3.2) of Fabry-Perot galaxies (192 x 192 x 48,
    the workload of the headline number): n_live live points, `batch`
    proposals per iteration evaluated in one fused launch, uniform prior over
    the workload's ranges (x0, y0 in 0.35 - 0.65 N, V_sys +-30 km/s);
    observations with 5 / 5 sqrt(2) km/s noise, S/N < 3 and 2 % dead-fibre
    masks."""
    g = synth.FP_GEOM
    rng = np.random.default_rng(77)
    truth = synth.draw_fp_params(rng, n_gal)
    maps = gbk.eval_maps(g, torch.from_numpy(truth), device=device).cpu().numpy()
    shape = (g.ny, g.nx)
    wv, ws = synth.weights(shape, 5.0)
    rows = []
    for j in range(n_gal):
        m = maps[j]
        v = (m[1] + rng.normal(0.0, 5.0, shape)).astype(np.float32)
        s = (m[2] + rng.normal(0.0, 5.0 * np.sqrt(2.0), shape)).astype(np.float32)
        mask = (synth.sn_mask(m[0]) * synth.dead_fibre_mask(rng, shape)).astype(np.uint8)
        obs = gbk.Obs.from_numpy(v, s, wv, ws, mask, device=device)
        lo, hi = truth[j].copy(), truth[j].copy()
        lo[synth.X0], hi[synth.X0] = 0.35 * g.nx, 0.65 * g.nx
        lo[synth.Y0], hi[synth.Y0] = 0.35 * g.ny, 0.65 * g.ny
        lo[synth.VSYS], hi[synth.VSYS] = -30.0, 30.0
        for k, (a_, b_) in synth.FP_RANGES.items():
            lo[k], hi[k] = a_, b_
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = gbk.gbk_nested_sample(g, obs, lo, hi, n_live=n_live, batch=batch, tol=0.5, seed=11 + j, device=device)
        dt = time.perf_counter() - t0
        dpa = abs((r["mean"][synth.PA] - truth[j, synth.PA] + 180.0) % 360.0 - 180.0)
        rows.append({"seconds": dt, "n_eval": r["n_eval"], "n_iter": r["n_iter"], "evals_per_s": r["n_eval"] / dt,
                     "log_z": r["log_z"], "dvmax": float(abs(r["mean"][synth.VMAX] - truth[j, synth.VMAX])),
                     "dpa": float(dpa), "dincl": float(abs(r["mean"][synth.INCL] - truth[j, synth.INCL])),
                     "post_std_vmax": float(r["std"][synth.VMAX])})
    return {"workload": "Fabry-Perot 192x192x48 galaxies, %d live points, %d proposals per launch, 8 free "
                        "parameters" % (n_live, batch), "galaxies": rows,
            "mean_seconds_per_galaxy": float(np.mean([x["seconds"] for x in rows]))}


def run_jacobian(gbk, torch, device, n=2048, geom=None):
    """The analytic Jacobian (J^T J, J^T r and chi2 of the eight free
    parameters, J not written) on n models of one geometry (default the
    single-galaxy 32 x 32 x 64 cube), against the 1 + 8 evaluations a
    forward-difference Jacobian needs for the same models: the two-stage
    kernels (gbk_jacobian_ws, gbk_chi2 on the split path) as the headline,
    the one-cluster-per-model kernels beside them."""
    g = geom or synth.SINGLE_GEOM
    rng = np.random.default_rng(9)
    truth = synth.SINGLE_TRUTH.copy()
    ps = np.array([synth.perturb(rng, truth, FIT_FREE, 0.2) for _ in range(n)])
    m = gbk.eval_maps(g, torch.from_numpy(truth[None]), device=device)[0]
    shape = (g.ny, g.nx)
    wv, ws = synth.weights(shape, 5.0)
    v = m[1] + torch.from_numpy(rng.normal(0.0, 5.0, shape).astype(np.float32)).to(device)
    s = m[2] + torch.from_numpy(rng.normal(0.0, 5.0 * np.sqrt(2.0), shape).astype(np.float32)).to(device)
    obs = gbk.Obs(v.contiguous(), s.contiguous(), torch.from_numpy(wv).to(device), torch.from_numpy(ws).to(device),
                  torch.ones(shape, dtype=torch.uint8, device=device))
    dp = torch.from_numpy(ps).to(device)
    nf = len(FIT_FREE)
    jtj = torch.empty((n, nf, nf), dtype=torch.float64, device=device)
    jtv = torch.empty((n, nf), dtype=torch.float64, device=device)
    c2 = torch.empty(n, dtype=torch.float64, device=device)
    dfd = dp.repeat(1 + nf, 1).contiguous()
    cfd = torch.empty(dfd.shape[0], dtype=torch.float64, device=device)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    wsj = torch.empty(gbk.gbk_jacobian_workspace_bytes(g, n, FIT_FREE), dtype=torch.uint8, device=device)
    wse = gbk.workspace_for(g, dfd.shape[0], gbk.PATH_SPLIT)
    tj = timed(lambda: gbk.gbk_jacobian_ws(g, dp, obs, FIT_FREE, None, jtj, jtv, c2, wsj))
    tc = timed(lambda: gbk.gbk_jacobian(g, dp, obs, FIT_FREE, None, jtj, jtv, c2, None))
    tf = timed(lambda: gbk.gbk_chi2(g, dfd, obs, cfd, None, gbk.PATH_SPLIT, wse))
    tff = timed(lambda: gbk.gbk_chi2(g, dfd, obs, cfd, None, gbk.PATH_FUSED, None))
    return {"workload": "%d models of a %dx%dx%d cube, 8 free parameters" % (n, g.nx, g.ny, g.nz),
            "jacobian_ms": tj, "fd_evals_ms": tf, "jacobian_vs_fd_evals": tj / tf,
            "jacobians_per_s": n / (tj * 1e-3),
            "kernels": "two-stage Jacobian (gbk_jacobian_ws) against 1 + 8 two-stage evaluations",
            "cluster_jacobian_ms": tc, "cluster_fd_evals_ms": tff}


def run_grid(gbk, torch, device, chunk=1 << 17):
    """Nested grids (Sec. 2.3.3) at full size: a 64 x 64 x 64 cube, 10^5
    nodes per level over PA, i, V_max, r_t, sigma0 (10 each), 3 levels,
    evaluated `chunk` models per launch; x0, y0, V_sys, I0, h fixed at the
    truth; 5 / 5 sqrt(2) km/s noise."""
    g = synth.Geometry(64, 64, 64, 20.0, 0.0, 2.5, 30.0)
    rng = np.random.default_rng(3)
    truth = synth.params(31.5, 31.5, rng.uniform(0, 360), rng.uniform(20, 80), 0.0, rng.uniform(50, 300),
                         rng.uniform(1, 8), rng.uniform(10, 80), 1.0, 8.0)
    m = gbk.eval_maps(g, torch.from_numpy(truth[None]), device=device)[0].cpu().numpy()
    shape = (g.ny, g.nx)
    wv, ws = synth.weights(shape, 5.0)
    obs = gbk.Obs.from_numpy((m[1] + rng.normal(0, 5.0, shape)).astype(np.float32),
                             (m[2] + rng.normal(0, 5.0 * np.sqrt(2.0), shape)).astype(np.float32), wv, ws,
                             np.ones(shape, np.uint8), device=device)
    nodes = [1] * 10
    lo, hi = truth.copy(), truth.copy()
    for k, (a_, b_) in {synth.PA: (0.0, 360.0), synth.INCL: (20.0, 80.0), synth.VMAX: (50.0, 300.0),
                        synth.RT: (1.0, 8.0), synth.SIG0: (10.0, 80.0)}.items():
        nodes[k] = 10
        lo[k], hi[k] = a_, b_
    gbk.gbk_grid(g, obs, lo, hi, nodes, truth, levels=1, chunk=chunk, device=device)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bp, bi, bc = gbk.gbk_grid(g, obs, lo, hi, nodes, truth, levels=3, chunk=chunk, device=device)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"workload": "64x64x64 cube, 10^5 nodes per level x 3 levels (PA, i, V_max, r_t, sigma0), %d models "
                        "per launch" % min(chunk, 100000), "seconds": dt, "nodes_per_s": 3e5 / dt,
            "best": {synth.PARAM_NAMES[k]: float(bp[k]) for k in (synth.PA, synth.INCL, synth.VMAX, synth.RT,
                                                                   synth.SIG0)},
            "truth": {synth.PARAM_NAMES[k]: float(truth[k]) for k in (synth.PA, synth.INCL, synth.VMAX, synth.RT,
                                                                      synth.SIG0)},
            "best_chi2_per_level": [float(c) for c in bc]}


def run_degeneracy(gbk, torch, device):
    """The V_t - i degeneracy (Sec. 6.1): reduced chi-squared maps over
    (i, V_t) of single-galaxy 32 x 32 x 64 mocks with V_t = 200 km/s at i = 20, 40, 60, 70 deg and
    5 / 5 sqrt(2) km/s noise; every map is one gbk_chi2 launch over a
    0.25 deg x 1 km/s grid.  Reports the best node and the extents of the
    1 and 3 sigma regions (chi2 - min <= 2.30, 11.83)."""
    g = synth.SINGLE_GEOM
    inc_ax = np.arange(5.0, 85.0 + 1e-9, 0.25)
    vt_ax = np.arange(50.0, 600.0 + 1e-9, 1.0)
    ii, vv = np.meshgrid(inc_ax, vt_ax, indexing="ij")
    wv, ws = synth.weights((g.ny, g.nx), 5.0)
    dwv, dws = torch.from_numpy(wv).to(device), torch.from_numpy(ws).to(device)
    ones = torch.ones((g.ny, g.nx), dtype=torch.uint8, device=device)
    out = {"workload": "single-galaxy geometry (32x32x64), V_t = 200 km/s, noise 5 / 5 sqrt(2) km/s, %d x %d (i, V_t) nodes "
                       "per map, other parameters at the truth" % (len(inc_ax), len(vt_ax)), "maps": {}}
    total_ms, total_models = 0.0, 0
    for inc in (20.0, 40.0, 60.0, 70.0):
        p = synth.SINGLE_TRUTH.copy()
        p[synth.INCL], p[synth.VMAX] = inc, 200.0
        m = gbk.eval_maps(g, torch.from_numpy(p[None]), device=device)[0]
        rng = np.random.default_rng(100 + int(inc))
        v = m[1] + torch.from_numpy(rng.normal(0.0, 5.0, (g.ny, g.nx)).astype(np.float32)).to(device)
        s = m[2] + torch.from_numpy(rng.normal(0.0, 5.0 * np.sqrt(2.0), (g.ny, g.nx)).astype(np.float32)).to(device)
        obs = gbk.Obs(v.contiguous(), s.contiguous(), dwv, dws, ones)
        grid = np.repeat(p[None], ii.size, 0)
        grid[:, synth.INCL], grid[:, synth.VMAX] = ii.ravel(), vv.ravel()
        dg = torch.from_numpy(grid).to(device)
        gbk.chi2(g, dg, obs, device=device)  # warm-up (and the launch tuning)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        c = gbk.chi2(g, dg, obs, device=device)
        b.record()
        b.synchronize()
        total_ms += a.elapsed_time(b)
        total_models += ii.size
        c = c.cpu().numpy().reshape(ii.shape)
        d = c - c.min()
        k = np.unravel_index(np.argmin(c), c.shape)
        r1, r3 = d <= 2.30, d <= 11.83
        vs = vv[r3] * np.sin(np.radians(ii[r3]))
        out["maps"]["%g" % inc] = {
            "best_incl": float(inc_ax[k[0]]), "best_vt": float(vt_ax[k[1]]),
            "min_reduced_chi2": float(c.min() / (2 * g.nx * g.ny - 2)),
            "sigma1_incl": [float(ii[r1].min()), float(ii[r1].max())],
            "sigma1_vt": [float(vv[r1].min()), float(vv[r1].max())],
            "sigma3_incl": [float(ii[r3].min()), float(ii[r3].max())],
            "sigma3_vt": [float(vv[r3].min()), float(vv[r3].max())],
            "sigma3_vt_sini_rel_spread": float(np.ptp(vs) / np.mean(vs))}
    out["evals_per_s"] = total_models / (total_ms * 1e-3)
    return out


def run_gemm(gbk, torch, device, sizes=((8192, 8192, 8192), (32768, 256, 4096), (262144, 64, 48))):
    """The tcgen05 BF16 GEMM on large shapes against the measured bf16
    peak; cuBLAS (torch.matmul) on the same shapes is timed beside it for
    context only -- the library never calls it."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    out = {"peak_tflops": peak, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" if peaks else "fallback",
           "shapes": []}
    g = torch.Generator(device=device).manual_seed(3)
    for M, N, K in sizes:
        A = torch.randn((M, K), generator=g, device=device).to(torch.bfloat16)
        B = torch.randn((N, K), generator=g, device=device).to(torch.bfloat16)
        C = torch.empty((M, N), dtype=torch.bfloat16, device=device)
        reps = max(3, min(50, int(2e13 / (2.0 * M * N * K))))
        for _ in range(3):
            gbk.gbk_gemm_bf16(A, B, out_bf16=C)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            gbk.gbk_gemm_bf16(A, B, out_bf16=C)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        for _ in range(3):
            torch.matmul(A, B.T)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            torch.matmul(A, B.T)
        b.record()
        b.synchronize()
        ms_ref = a.elapsed_time(b) / reps
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out["shapes"].append({"M": M, "N": N, "K": K, "ms": ms, "tflops": tf, "frac": tf / peak,
                              "cublas_tflops": 2.0 * M * N * K / (ms_ref * 1e-3) / 1e12})
        del A, B, C
    return out


def make_galaxy(gbk, torch, g, seed, device):
    """One synthetic Fabry-Perot galaxy: true parameters from the prior, maps
    from the library at those parameters, seeded noise (5 km/s on v,
    5 sqrt(2) on sigma), S/N < 3 and 2% dead-fibre masks."""
    rng = np.random.default_rng(seed)
    p_true = synth.draw_fp_params(rng, 1)
    maps = gbk.eval_maps(g, torch.from_numpy(p_true), device=device).cpu().numpy()[0]
    shape = (g.ny, g.nx)
    v = (maps[1] + synth.gaussian_noise(rng, shape, 5.0)).astype(np.float32)
    s = (maps[2] + synth.gaussian_noise(rng, shape, 5.0 * np.sqrt(2.0))).astype(np.float32)
    wv, ws = synth.weights(shape, 5.0)
    mask = (synth.sn_mask(maps[0]) * synth.dead_fibre_mask(rng, shape)).astype(np.uint8)
    return p_true[0], (v, s, wv, ws, mask)


def cpu_baseline(g, obs_np, n_models, seed):
    """The FP64 oracle, as it stands, on all host cores: one batch of models
    evaluated with OpenMP (one model per core at a time)."""
    import oracle
    cores = oracle.max_threads()
    n = max(4, cores)
    rng = np.random.default_rng(seed + 99)
    ps = synth.draw_fp_params(rng, n)
    o = oracle.Obs(*obs_np)
    og = oracle.Geom(**g.asdict())
    t = time.perf_counter()
    oracle.chi2_batch(og, ps, o, nthreads=cores)
    dt = time.perf_counter() - t
    # and one core: two models, one after the other
    t = time.perf_counter()
    oracle.chi2_batch(og, ps[:2], o, nthreads=1)
    dt1 = time.perf_counter() - t
    return {"value": n / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": "%d of the %d models of one step (192x192x48, direct 3-D convolution, FP64), "
                      "OpenMP over models, %.1f s" % (n, n_models, dt),
            "single_core": {"value": 2 / dt1, "unit": "evals/s", "cores": 1,
                            "sample": "2 models on one thread, %.1f s" % dt1}}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    g = synth.FP_GEOM
    cores = oracle.max_threads()
    per_step = max(4, cores)
    rng = np.random.default_rng(2015)
    p_true = synth.draw_fp_params(rng, 1)[0]
    og = oracle.Geom(**g.asdict())
    m = oracle.evaluate(og, p_true)
    shape = (g.ny, g.nx)
    wv, wsig = synth.weights(shape, 5.0)
    obs = oracle.Obs((m[1] + rng.normal(0, 5, shape)).astype(np.float32),
                     (m[2] + rng.normal(0, 7.07, shape)).astype(np.float32), wv, wsig,
                     (synth.sn_mask(m[0]) * synth.dead_fibre_mask(rng, shape)).astype(np.uint8))
    # The oracle takes seconds per step, so the run is bounded in time: the
    # requested warm-up steps (stopped early only past a 90 s bound), then
    # timed steps until K are done or the budget is spent (at least one).
    # The value is a rate, models per second, so the bound does not bias it;
    # the steps actually run are reported.
    budget_s = float(os.environ.get("GBK_REFERENCE_BUDGET_S", "150"))
    warm_budget_s = float(os.environ.get("GBK_REFERENCE_WARM_BUDGET_S", "90"))
    pool = synth.draw_fp_params(rng, per_step * (args.warmup + args.steps))
    warm = 0
    tw = time.perf_counter()
    while warm < args.warmup:
        oracle.chi2_batch(og, pool[warm * per_step:(warm + 1) * per_step], obs, nthreads=cores)
        warm += 1
        if time.perf_counter() - tw > warm_budget_s:
            break
    t = time.perf_counter()
    done = 0
    for s in range(args.warmup, args.warmup + args.steps):
        oracle.chi2_batch(og, pool[s * per_step:(s + 1) * per_step], obs, nthreads=cores)
        done += 1
        if time.perf_counter() - t > budget_s:
            break
    dt = time.perf_counter() - t
    value = per_step * done / dt
    sample = ("%d of the %d models per step (192x192x48), FP64 oracle, OpenMP over models; %d of %d steps "
              "timed within a %.0f s budget, %d warm-up" % (per_step, args.models, done, args.steps, budget_s, warm))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": done, "warmup": warm, "steps_requested": args.steps, "warmup_requested": args.warmup,
        "ms_per_step": 1e3 * dt / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fabry-perot 192x192x48, 400 live points per step", "models_per_step": per_step,
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_lm_only(gbk, torch, which, device):
    """One batched LM fit with the analytic Jacobian of the survey leg's or
    the fits leg's batch (2048 galaxies each), timed from the host; one JSON
    line.  Meant for launch lists of the fit's kernels."""
    opts = gbk.lm_opts(max_iter=200, jacobian=gbk.JAC_TANGENT, free=FIT_FREE)
    if which == "survey":
        geoms, truth, obs, p0, lo, hi = survey_batch(gbk, torch, 2048, 4, device)
        fit = lambda: gbk.survey_fit_lm(geoms, obs, np.array(p0), np.array(lo), np.array(hi), opts, device=device)
    else:
        g, truth, obs, p0, lo, hi = fit_batch(gbk, torch, 2048, 4242, device)
        fit = lambda: gbk.fit_lm(g, obs, p0, lo, hi, opts, device=device)
    torch.cuda.synchronize()
    t = time.perf_counter()
    q, c, it, st = fit()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    print(json.dumps({"lm_only": which, "galaxies": 2048, "fits_per_s": 2048 / dt, "max_iters": int(np.max(it)),
                      "iters_sum": int(np.sum(it))}))


def run_gbk(args):
    import torch
    from paper_1510_01815_gb300 import build as gbuild
    gbuild.build()
    from paper_1510_01815_gb300 import gbk

    ws, rank, local = dist_info()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.lm_only:
        run_lm_only(gbk, torch, args.lm_only, dev)
        return
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    g = synth.FP_GEOM
    n = args.models
    K, W = args.steps, args.warmup
    p_true, obs_np = make_galaxy(gbk, torch, g, 2015, dev)
    obs = gbk.Obs.from_numpy(*obs_np, device=dev)
    pool_np = rank_pool(rank, n, K + W)
    pool = torch.from_numpy(pool_np).to(dev)
    chi2 = torch.empty((K + W, n), dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    staged = args.path == "staged"
    split = args.path == "split"
    ws_staged = gbk.workspace_for(g, n, gbk.PATH_STAGED, dev) if staged else None
    ws_split = gbk.workspace_for(g, n, gbk.PATH_SPLIT, dev) if split else None

    def step(s):
        if staged:
            gbk.gbk_chi2(g, pool[s], obs, chi2[s], None, gbk.PATH_STAGED, ws_staged, stream)
        elif split:
            gbk.gbk_chi2(g, pool[s], obs, chi2[s], None, gbk.PATH_SPLIT, ws_split, stream)
        else:
            gbk.gbk_chi2(g, pool[s], obs, chi2[s], None, gbk.PATH_FUSED, None, stream)

    if staged or split:
        tuning = {"cluster_ctas": 0, "threads": 0, "persistent": 0, "candidates": 0}
    elif args.tuning:
        cs_, nt_, pe_ = (int(v) for v in args.tuning.split(","))
        gbk.gbk_set_tuning(g, cs_, nt_, pe_)
        tuning = {"cluster_ctas": cs_, "threads": nt_, "persistent": pe_, "candidates": 0}
    else:
        tuning = gbk.gbk_autotune(g, pool[0], obs, chi2[0], stream)
    for s in range(W):
        step(s)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    if not args.quick:
        clocks.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        step(W + k)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if not args.quick else None
    times = [starts[k].elapsed_time(ends[k]) for k in range(K)]
    total_ms = float(sum(times))
    assert torch.isfinite(chi2[W:]).all(), "non-finite chi2 in the timed steps"
    value, total_ms = job_throughput(total_ms, n * K, dist)
    ms_step = total_ms / K

    out = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "fabry-perot 192x192x48 at 10 km/s, PSF 3 px, LSF 30 km/s, "
                                  "400 live points per step (one batched launch)",
                      "models_per_step": n, "path": args.path, "l2": "flushed between steps (256 MiB write)",
                      "tuning": {"cluster_ctas": tuning["cluster_ctas"], "threads": tuning["threads"],
                                 "persistent": tuning["persistent"], "candidates": tuning["candidates"]},
                      "parallelism": "replicas" if ws > 1 else "single"},
           "gpu_launches": K * (4 if staged else 1)}
    if split:
        # per-launch CUDA events (gbk_split_stage_times) over K further steps
        # of the same batches, L2 flushed before each: the kernels' times
        stage_reps, nl = [], 0
        for k in range(K):
            flush.fill_(k & 0xFF)
            st_ms, nl = gbk.gbk_split_stage_times(g, pool[W + k], obs, chi2[W + k], ws_split, stream)
            stage_reps.append(st_ms)
        stage_mean = np.mean(np.array(stage_reps), axis=0)
        out["gpu_launches"] = K * nl
        out["stages"] = [{"stage": name, "kernel": kern, "ms_per_step": float(t), "share": float(t / sum(stage_mean))}
                         for name, kern, t in zip(("set-up", "line sums + PSF along x", "PSF along y + moments + chi2"),
                                                  ("split_setup_kernel", "split_line_kernel", "split_psf_kernel"),
                                                  stage_mean)]
    if staged:
        out["config"]["path"] = "staged"
    if args.quick:
        if rank == 0:
            print(json.dumps(out))
        return

    ex, ey, ez = ext_dims(g)
    if staged:
        # HBM roofline of the staged chain: extended cube written and read
        # once, data cube written and read once (algorithmic bytes)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        per_model = 4.0 * (2 * ex * ey * ez + 2 * g.nx * g.ny * g.nz)
        ach = n * per_model / (ms_step * 1e-3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "kernel": "staged chain (model cube, conv, moments)",
                           "basis": "%.1f MB algorithmic traffic per model" % (per_model / 1e6),
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}
        # per-stage times (CUDA events between the stages, median of 5 calls
        # with L2 flushed before each) and each stage's algorithmic bytes
        reps = []
        for r in range(5):
            flush.fill_(r & 0xFF)
            reps.append(gbk.gbk_chi2_stage_times(g, pool[0], obs, chi2[0], ws_staged, stream))
        med = np.median(np.array(reps), axis=0)
        ext_b, data_b = 4.0 * ex * ey * ez * n, 4.0 * g.nx * g.ny * g.nz * n
        stage_bytes = (ext_b, ext_b + data_b, 0.0, data_b)
        out["stages"] = [{"stage": name, "ms": float(t), "algorithmic_bytes": b_,
                          "gbs": (b_ / (t * 1e-3) / 1e9) if t > 0 and b_ > 0 else None,
                          "frac": (b_ / (t * 1e-3) / 1e9 / hbm) if t > 0 and b_ > 0 else None}
                         for name, t, b_ in zip(("model cube (a1-a2)", "PSF x LSF convolution (a3)",
                                                 "down-sampling (a4)", "moments + chi2 (a5-a6)"), med, stage_bytes)]
        out["clocks"] = clk
        if rank == 0:
            print(json.dumps(out))
        return

    if split:
        # ---- roofline of the dominant kernel: the line stage, ALU bound ----
        # Algorithmic work per model: the line sampling (5 FP32 + 1 ex2 per
        # extended voxel) and the PSF pass along x of every extended row
        # (6 FP32 per tap per output, ey x nx outputs).
        taps = 2 * ((ex - g.nx) // 2) + 1
        fma_a = FMA_OPS_PER_EXT_VOXEL * ex * ey * ez + split_pass_ops_per_output(taps) * ey * g.nx
        mufu_a = MUFU_OPS_PER_EXT_VOXEL * ex * ey * ez
        r32, r32x2, rmu = gbk.gbk_measure_alu_peak(stream)
        rfma = max(r32, r32x2)
        t_min = max(fma_a / rfma, mufu_a / rmu)
        peak_ops = (fma_a + mufu_a) / t_min
        t_a = out["stages"][1]["ms_per_step"] * 1e-3
        achieved_ops = (fma_a + mufu_a) * n / t_a
        out["roofline"] = {
            "bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
            "frac": achieved_ops / peak_ops, "traffic": SPLIT_LINE_TRAFFIC.get(n),
            "traffic_note": ("DRAM bytes per launch (%d models) from one ncu capture of this kernel build: its "
                             "x-filtered planes stay in L2" % SPLIT_LINE_TRAFFIC_MODELS if n in SPLIT_LINE_TRAFFIC
                             else "no capture of this kernel build at this batch size"),
            "kernel": "split_line_kernel",
            "basis": "per model %.1f M FP32 + %.1f M ex2 lane ops: %d FP32 + %d ex2 per extended voxel (%d x %d x "
                     "%d), %.1f FP32 per output of the PSF pass along x (%d taps x %d FMAs, %d per input and %d per "
                     "output for the re-centring; %d x %d outputs); its time per step from CUDA events around each "
                     "launch (%.3f ms of %.3f); measured FP32 pipe %.1f T lane-ops/s (scalar %.1f, f32x2 %.1f), "
                     "ex2 %.1f T/s"
                     % (fma_a / 1e6, mufu_a / 1e6, FMA_OPS_PER_EXT_VOXEL, MUFU_OPS_PER_EXT_VOXEL, ex, ey, ez,
                        split_pass_ops_per_output(taps), taps, OPS_PER_PSF_TAP_SPLIT, OPS_PER_PSF_INPUT_SPLIT,
                        OPS_PER_PSF_OUTPUT_SPLIT, ey, g.nx, t_a * 1e3,
                        sum(st["ms_per_step"] for st in out["stages"]),
                        rfma / 1e12, r32 / 1e12, r32x2 / 1e12, rmu / 1e12),
            "peak_source": "measured on this device by gbk_measure_alu_peak"}
        # the whole step on the same basis (both stages, every launch)
        fma_all = fma_a + split_pass_ops_per_output(taps) * g.ny * g.nx + OPS_PER_DATA_SPAXEL * g.nx * g.ny
        out["roofline_whole_step"] = {
            "achieved": (fma_all + mufu_a) * n / (ms_step * 1e-3) / 1e12, "unit": "Tops/s",
            "frac": (fma_all + mufu_a) * n / (ms_step * 1e-3) / ((fma_all + mufu_a) / max(fma_all / rfma, mufu_a / rmu)),
            "basis": "both stages: %.1f M FP32 + %.1f M ex2 per model over the step time" % (fma_all / 1e6, mufu_a / 1e6)}
    if not split:
        # ---- roofline of the fused kernel: ALU (FP32 pipe + MUFU ex2) ----
        # Algorithmic work per model of the folded method: the line sampling
        # (5 FP32 + 1 ex2 per extended voxel), the two exact PSF passes on the
        # moment triplets (x over ey * nx, y over ny * nx outputs, 2R + 1 taps)
        # and the moments/residuals/chi2 of each data spaxel.
        taps = 2 * ((ex - g.nx) // 2) + 1
        fma_model = (FMA_OPS_PER_EXT_VOXEL * ex * ey * ez + OPS_PER_PSF_TAP * taps * (ey * g.nx + g.ny * g.nx)
                     + OPS_PER_DATA_SPAXEL * g.nx * g.ny)
        mufu_model = MUFU_OPS_PER_EXT_VOXEL * ex * ey * ez
        r32, r32x2, rmu = gbk.gbk_measure_alu_peak(stream)
        rfma = max(r32, r32x2)
        t_min = max(fma_model / rfma, mufu_model / rmu)
        peak_ops = (fma_model + mufu_model) / t_min
        achieved_ops = (fma_model + mufu_model) * n / (ms_step * 1e-3)
        tuned = (tuning["cluster_ctas"], tuning["threads"], tuning["persistent"])
        traffic = FUSED_TRAFFIC_400.get(tuned) if n == 400 else None
        out["roofline"] = {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12,
                           "unit": "Tops/s", "frac": achieved_ops / peak_ops, "traffic": traffic,
                           "traffic_note": "DRAM bytes per launch from one ncu capture at this tuning "
                                           "(algorithmic: 0.66 MB of parameters, observed maps and chi2)"
                                           if traffic else "no capture at this configuration",
                           "kernel": "fused_eval_kernel",
                           "basis": "per model %.1f M FP32 + %.1f M ex2 lane ops: %d FP32 + %d ex2 per extended voxel "
                                    "(%d x %d x %d), %d per PSF tap on the moment triplets (%d taps; x pass %d x %d, "
                                    "y pass %d x %d outputs), %d per data spaxel; measured FP32 pipe %.1f T lane-ops/s "
                                    "(scalar %.1f, f32x2 %.1f), ex2 %.1f T/s"
                                    % (fma_model / 1e6, mufu_model / 1e6, FMA_OPS_PER_EXT_VOXEL, MUFU_OPS_PER_EXT_VOXEL,
                                       ex, ey, ez, OPS_PER_PSF_TAP, taps, ey, g.nx, g.ny, g.nx, OPS_PER_DATA_SPAXEL,
                                       rfma / 1e12, r32 / 1e12, r32x2 / 1e12, rmu / 1e12),
                           "peak_source": "measured on this device by gbk_measure_alu_peak"}
    data_vox = g.nx * g.ny * g.nz
    sv = UNFOLDED_FP32_PER_DATA_VOXEL * data_vox * n / (ms_step * 1e-3)
    out["roofline_unfolded_basis"] = {
        "achieved": sv / 1e12, "peak": rfma / 1e12, "unit": "T FP32 instr/s", "frac": sv / rfma,
        "basis": "%.0f FP32 instructions per data voxel of the unfolded cube + separable convolution + moments "
                 "method; the fused kernel reaches the same result with far fewer operations (z convolution "
                 "folded into channel weights, PSF applied to moment triplets), so this is an effective rate"
                 % UNFOLDED_FP32_PER_DATA_VOXEL}
    out["clocks"] = clk

    # ---- end to end through the public API with host buffers ----
    pin_params = torch.from_numpy(pool_np).pin_memory()
    pin_chi2 = torch.empty((K + W, n), dtype=torch.float64).pin_memory()
    pin_obs = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in obs_np]
    d_params = torch.empty((n, synth.NPAR), dtype=torch.float64, device=dev)
    d_obs = [torch.empty(a.shape, dtype=a.dtype, device=dev) for a in pin_obs]
    e_obs = gbk.Obs(*d_obs)
    d_chi2 = torch.empty(n, dtype=torch.float64, device=dev)

    if split:
        # the host-buffer entry point: parameters, maps and chi2 in pinned
        # host memory, the copies inside the call (the maps' copy beside the
        # first line stage)
        h_obs = gbk.Obs(*pin_obs)
        ws_host = torch.empty(gbk.gbk_chi2_host_workspace_bytes(g, n), dtype=torch.uint8, device=dev)

    def e2e_step(s):
        if split:
            gbk.gbk_chi2_host(g, pin_params[s], h_obs, pin_chi2[s], ws_host, stream)
            return
        d_params.copy_(pin_params[s], non_blocking=True)
        for d, h in zip(d_obs, pin_obs):
            d.copy_(h, non_blocking=True)
        gbk.gbk_chi2(g, d_params, e_obs, d_chi2, None, gbk.PATH_AUTO, None, stream)
        pin_chi2[s].copy_(d_chi2, non_blocking=True)

    for s in range(W):
        e2e_step(s)
    torch.cuda.synchronize()
    e_ms = 0.0
    for k in range(K):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step(W + k)
        b.record(stream)
        b.synchronize()
        e_ms += a.elapsed_time(b)
    h2d = n * synth.NPAR * 8 + sum(int(h.numel() * h.element_size()) for h in pin_obs)
    e_value, e_ms = job_throughput(e_ms, n * K, dist)
    out["e2e"] = {"value": e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": n * 8}
    ok = np.allclose(pin_chi2[W:].numpy(), chi2[W:].cpu().numpy(), rtol=0, atol=0)
    out["e2e"]["matches_device_run"] = bool(ok)
    out["gpu_launches_e2e"] = out["gpu_launches"]

    # The single-GPU measurements below describe one GPU; a multi-GPU run
    # (weak scaling of the headline) skips them.
    if ws > 1:
        args.no_fits = args.no_survey = args.no_gemm = args.no_vfield = args.no_ns = True
        args.no_jacobian = args.no_grid = args.no_degeneracy = args.no_mock = args.no_cnn = True
    if not args.no_fits:
        out["fits"] = run_fits(gbk, torch, args.fit_galaxies, args.fit_plain, dev,
                               [("plain_fd", gbk.LM_PLAIN, gbk.JAC_FD_FORWARD, gbk.PATH_AUTO),
                                ("batched_fd", gbk.LM_BATCHED, gbk.JAC_FD_FORWARD, gbk.PATH_AUTO),
                                ("batched_tangent", gbk.LM_BATCHED, gbk.JAC_TANGENT, gbk.PATH_AUTO),
                                ("batched_tangent_cluster_kernels", gbk.LM_BATCHED, gbk.JAC_TANGENT,
                                 gbk.PATH_FUSED)])
    if not args.no_survey:
        out["survey"] = run_survey(gbk, torch, args.survey_galaxies, args.survey_plain, dev)
    if not args.no_gemm:
        out["gemm"] = run_gemm(gbk, torch, dev)
    if not args.no_vfield:
        out["vfield"] = run_vfield(gbk, torch, 1024, 512, 8, dev)
    if not args.no_ns:
        out["nested_sampling_fp"] = run_ns_fp(gbk, torch, dev)
    if not args.no_jacobian:
        out["jacobian"] = run_jacobian(gbk, torch, dev)
    if not args.no_grid:
        out["grid"] = run_grid(gbk, torch, dev)
    if not args.no_degeneracy:
        out["degeneracy"] = run_degeneracy(gbk, torch, dev)
    if not args.no_mock:
        out["mock_study"] = run_mock_study(gbk, torch, args.mock_galaxies, dev)
    if not args.no_cnn:
        out["cnn"] = run_cnn(gbk, torch, args.cnn_train, args.cnn_epochs, args.cnn_batch, args.cnn_test, 64, dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, obs_np, n, 2015)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gbk(args)


if __name__ == "__main__":
    main()
