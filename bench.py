"""Benchmark: source-ear samples/s of the sparse factorized HRIR renderer on one GB300.

Workload (the batched rendering configuration): 1024 sources x 480000 samples (10 s at
48 kHz) of seeded AR(1) noise, directions uniform over a 1250-direction grid, K = 16
non-negative reflection taps of 200 per (direction, ear), 32-tap resonance per ear, output
the full-length stereo mix.  One step = one hrir_render_batch call (sparse gather-FMA mix
kernel + fixed-order reduction/resonance kernel) over the whole batch, inputs resident in
HBM (1.97 GB, larger than the 129 MB L2, so no flush is needed).  The same batch is also
rendered by the dense-HRIR direct path, by overlap-save FFT convolution (P = 4096), and with
K = 8 and K = 32; those numbers are extra keys ("paths") of the same JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own independent batch (seed offset by rank; no
collective on the data path) and rank 0 prints one JSON line with the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

S_DEFAULT, L_DEFAULT, K_DEFAULT = 1024, 480000, 16
METRIC = "source-ear samples/s (sparse vs dense/FFT conv, same GB300); p99 block latency"
WORKLOAD = "batched: 1024 sources x 480000 samples AR(1), 1250 directions, K=16 of 200 taps, Lf=32"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
N_SM, FP32_LANES = 152, 128          # GB300: 152 SMs x 128 FP32 FMA lanes


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak: SMs x lanes x 2 flop x clock."""
    return N_SM * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region.  The sampler is live (its
    first sample read) before the caller's warm-up; mark() starts the region, and the summary
    holds the samples taken after it, including one taken at or after the region's end, so a
    region shorter than the sampling period is still sampled."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=200):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.first = 0

    def _wait_for_sample(self, n, limit_s):
        t0 = time.monotonic()
        while len(self.lines) <= n and time.monotonic() - t0 < limit_s and self.proc.poll() is None:
            time.sleep(0.005)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return self
        self._wait_for_sample(0, 5.0)
        self.mark()
        return self

    def mark(self):
        """The timed region starts: only samples read from now on are summarised."""
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            # one sample at or after the end of the region
            self._wait_for_sample(len(self.lines), 2.0 * self.period_ms / 1e3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.first:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def profiled_traffic(kernel_file, profile_file):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (the summary records the source's sha256); else None."""
    path = os.path.join(ROOT, "profiles", profile_file)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b:
        return None
    src = os.path.join(ROOT, "paper_1502_03162_gb300", "csrc", kernel_file)
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return float(m_b.group(1)) if cur == m_sha.group(1) else None


class Replicas:
    """One process per GPU (torchrun): RANK / WORLD_SIZE / LOCAL_RANK from the launcher's
    environment.  Each rank renders its own independent batch (seed offset by the rank), so
    there is no collective on the data path: a barrier brackets the timed region, the step
    time is the maximum over ranks, and the whole-job rate counts every rank's units."""

    def __init__(self, backend="nccl", device="cuda"):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def seed(self, base):
        return base + self.rank

    def whole_job(self, units_per_rank, ms_per_step):
        """Units of all ranks per second, at the slowest rank's step time."""
        return units_per_rank * self.world / (ms_per_step / 1e3)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def make_inputs(S, L, seed, torch):
    from paper_1502_03162_gb300 import synth
    ld = (L + 7) // 8 * 8
    host = torch.empty((S, ld), dtype=torch.float32, pin_memory=True)
    cfg = synth.batched_config(S=S, L=L, seed=seed, ld=ld, out=host.numpy())
    return cfg, host


def time_steps(fn, steps, warmup, torch, barrier):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    st = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        fn()
    b.record(st)
    torch.cuda.synchronize()
    barrier()
    return a.elapsed_time(b) / steps  # ms per step


def cpu_baseline(cfg, idx, w, nnz, res):
    """The oracle as it stands on the host cores, on bounded samples of the same batch (the
    first n sources over the full 480000 samples): the sparse cascade on all cores and on
    one core, and the dense-HRIR and FFT definitions on all cores.  Each worker process
    renders a contiguous slice of the sources; the slices' mixes are summed in FP64."""
    L = min(L_DEFAULT, cfg["y"].shape[1])
    S = cfg["y"].shape[0]
    cores = len(os.sched_getaffinity(0))
    legs = {"sparse": (min(S, 64 * cores), None), "one_core": (min(S, 128), 1),
            "dense": (min(S, 4 * cores), None), "fft": (min(S, 2 * cores), None)}
    n_max = max(n for n, _ in legs.values())
    from oracle.pool import SlicedRenderer
    tm = SlicedRenderer(cfg["y"][:n_max, :L], cfg["dirs"][:n_max], idx, w, nnz, 200, res, cores)
    res_legs = {}
    try:
        for name, (n, workers) in legs.items():
            mode = "sparse" if name == "one_core" else name
            dt, _ = tm.run(n, L, mode, workers)
            used = min(workers or cores, n)
            res_legs[name] = {
                "value": n * L * 2 / dt, "unit": "source-ear samples/s", "cores": used,
                "kind": "oracle",
                "sample": f"{n} of the {S} sources x {L} samples, {mode} definition, FP64, "
                          f"{used} process(es) over contiguous source slices ({dt:.1f} s)"}
    finally:
        tm.close()
    top = dict(res_legs["sparse"])
    top["one_core"] = res_legs["one_core"]
    top["dense"] = res_legs["dense"]
    top["fft"] = res_legs["fft"]
    return top


def run_reference(args):
    """The oracle timed on the host cores on the same workload (bounded sample per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1502_03162_gb300 import synth
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    # sources per step sized so that the whole run takes about a minute of the host's cores
    # (the oracle renders about 4e7 source-ear samples per second per core)
    per_step_s = 60.0 / max(1, args.steps + args.warmup)
    n_src = int(max(1, min(S_DEFAULT, round(per_step_s * 4e7 * cores / (2 * L_DEFAULT)))))
    cfg = synth.batched_config(S=n_src, L=L_DEFAULT, seed=2)
    idx, w, nnz = oracle.topk(cfg["G"], K_DEFAULT)
    from oracle.pool import SlicedRenderer
    tm = SlicedRenderer(cfg["y"], cfg["dirs"], idx, w, nnz, 200, cfg["res"], cores)
    try:
        for _ in range(args.warmup):
            tm.run(min(n_src, cores), L_DEFAULT, "sparse")
        dt = sum(tm.run(n_src, L_DEFAULT, "sparse")[0] for _ in range(args.steps)) / args.steps
    finally:
        tm.close()
    value = n_src * L_DEFAULT * 2 / dt
    used = min(cores, n_src)
    sample = (f"{n_src} sources x {L_DEFAULT} samples per step, sparse cascade, FP64, "
              f"{used} processes over contiguous source slices")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "source-ear samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle sample)"},
        "cpu_baseline": {"value": value, "unit": "source-ear samples/s", "cores": used,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "source-ear samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def bench_stream(rend, torch, block, warm_audio_s=10.0, audio_s=60.0, seed=12, rate=200.0,
                 fs=48000, max_slots=8192, pool_bytes=4 << 30):
    """Serving loop: Poisson arrivals (rate per second of audio), source lengths log-uniform in
    [0.1, 30] s, one session per source, admission bound by slots and the device pool.  The
    arrival clock is audio time (unpaced).  Returns latency percentiles of hrir_stream_step
    and throughput in source-ear samples per wall second."""
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(seed)
    noise = torch.empty(1 << 25, dtype=torch.float32, pin_memory=True)   # 128 MB of sources
    noise.numpy()[:] = rng.standard_normal(noise.numel(), dtype=np.float32)
    nz = noise.numpy()
    st = hrir.Stream(rend, block, max_slots, pool_bytes)
    n_dirs = 1250
    t_audio, next_arrival, req = 0.0, rng.exponential(1.0 / rate), 0
    queue = []
    lat, rows_hist, refused = [], [], 0
    samples = 0
    total_steps = int((warm_audio_s + audio_s) * fs / block)
    warm_steps = int(warm_audio_s * fs / block)
    t_wall0 = None
    for step in range(total_steps):
        t_audio += block / fs
        while next_arrival <= t_audio:
            n = int(round(np.exp(rng.uniform(np.log(0.1), np.log(30.0))) * fs))
            off = int(rng.integers(0, nz.size - n))
            queue.append((req, nz[off:off + n], int(rng.integers(0, n_dirs))))
            req += 1
            next_arrival += rng.exponential(1.0 / rate)
        while queue:
            rid, y, d = queue[0]
            rc = st.admit(rid, rid, y, d)
            if rc != hrir.HRIR_OK:
                refused += 1
                break
            queue.pop(0)
        if step == warm_steps:
            torch.cuda.synchronize()
            t_wall0 = time.perf_counter()
        t0 = time.perf_counter()
        blocks, sessions, done = st.step()
        t1 = time.perf_counter()
        if step >= warm_steps:
            lat.append(t1 - t0)
            rows_hist.append(len(sessions))
            samples += len(sessions) * block * 2
    wall = time.perf_counter() - t_wall0
    st.close()
    lat_ms = np.array(lat) * 1e3
    return {"block": block, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
            "value": samples / wall, "unit": "source-ear samples/s",
            "mean_active_sources": float(np.mean(rows_hist)), "max_active_sources": int(max(rows_hist)),
            "steps": len(lat), "audio_s": audio_s, "realtime_factor": audio_s / wall,
            "refused_admissions": refused, "pool_bytes": pool_bytes, "max_slots": max_slots,
            "arrivals_per_s": rate}


def bench_learned(rend, torch, seed=13, S=4096, L=96000, seg=256, k=16, train_steps=20):
    """Learned filters and moving sources (4096 sources x 2 s at 48 kHz, a direction every 256
    samples, random-initialised network of the trained architecture): network inference for
    every (source, segment, ear) row, top-k, and the crossfade render; plus the network's
    training step (forward + backward + Adam) on one HRIR set's 1250 directions x 2 ears."""
    from paper_1502_03162_gb300 import hrir, learned, synth
    rng = np.random.default_rng(seed)
    n_seg = (L + seg - 1) // seg
    az, el = synth.trajectories(rng, S, n_seg)
    rows = torch.from_numpy(learned.direction_rows(az, el)).cuda()
    params = torch.from_numpy(learned.init_params(200, seed, 0.02)).cuda()
    y = torch.from_numpy(synth.sources_ar1(rng, S, L)).cuda()
    n_rows = rows.shape[0]
    g = torch.empty((n_rows, 200), dtype=torch.float32, device="cuda")
    idx = torch.empty((S, n_seg, 2, k), dtype=torch.int16, device="cuda")
    w = torch.empty((S, n_seg, 2, k), dtype=torch.float32, device="cuda")
    nnz = torch.empty((S, n_seg, 2), dtype=torch.uint8, device="cuda")
    out = torch.empty((2, L + 230), dtype=torch.float32, device="cuda")
    infer32 = lambda: hrir.hrir_mlp_forward(rend.ctx, rows, params, 200, out=g)  # noqa: E731
    infer = lambda: hrir.hrir_mlp_forward_bf16(rend.ctx, rows, params, 200, out=g)  # noqa: E731
    pack = lambda: hrir.hrir_topk_pack(rend.ctx, g.view(S, n_seg, 2, 200), k, idx, w, nnz)  # noqa: E731
    render = lambda: hrir.hrir_render_moving(rend.ctx, y, idx, w, nnz, seg, out=out)  # noqa: E731
    nb = lambda: None  # noqa: E731
    t_inf32 = time_steps(infer32, 2, 1, torch, nb)
    t_inf = time_steps(infer, 3, 1, torch, nb)
    t_pack = time_steps(pack, 3, 1, torch, nb)
    t_ren = time_steps(render, 5, 2, torch, nb)
    assert rend.sync() == 0
    units = S * L * 2
    # training step on one synthetic HRIR set's reflection rows
    p = synth.hrir_set_params(4)
    gaz, gel = synth.az_el_grid()
    T = np.stack([synth.hrir_set_reflections(p, gaz, gel, np.full(gaz.size, e)) for e in range(2)],
                 1).reshape(-1, 200).astype(np.float32)
    trows = torch.from_numpy(learned.direction_rows(gaz, gel)).cuda()
    tT = torch.from_numpy(T).cuda()
    B = trows.shape[0]
    acts = torch.empty((B, hrir.hrir_mlp_act_stride(200)), dtype=torch.float32, device="cuda")
    tout = torch.empty((B, 200), dtype=torch.float32, device="cuda")
    grads = torch.empty_like(params)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    tp = params.clone()
    step_no = [0]

    def train_step():
        step_no[0] += 1
        hrir.hrir_mlp_forward(rend.ctx, trows, tp, 200, out=tout, acts=acts)
        hrir.hrir_mlp_backward(rend.ctx, trows, tp, acts, tout, tT, 200, grads=grads, loss=loss)
        hrir.hrir_mlp_adam(rend.ctx, tp, grads, m, v, step_no[0], 1e-3)
    t_train = time_steps(train_step, train_steps, 3, torch, nb)
    assert rend.sync() == 0
    flops_fwd_row = 2 * (5 * 256 + 2 * 256 * 256 + 256 * 200)
    return {"workload": f"moving: {S} sources x {L} samples, direction every {seg} samples, "
                        f"network filters top-{k}, linear crossfade",
            "render": {"value": units / (t_ren / 1e3), "unit": "source-ear samples/s",
                       "ms": t_ren, "fp32_tflops": 4.0 * k * units / (t_ren / 1e3) / 1e12},
            "filters": {"rows": n_rows, "precision": "bf16 tensor cores", "ms": t_inf,
                        "rows_per_s": n_rows / (t_inf / 1e3),
                        "tflops": flops_fwd_row * n_rows / (t_inf / 1e3) / 1e12,
                        "fp32_tc_split3_ms": t_inf32,
                        "fp32_tc_split3_tflops": flops_fwd_row * n_rows / (t_inf32 / 1e3) / 1e12,
                        "topk_ms": t_pack},
            "end_to_end": {"value": units / ((t_inf + t_pack + t_ren) / 1e3),
                           "unit": "source-ear samples/s", "ms": t_inf + t_pack + t_ren},
            "train_step": {"rows": B, "ms": t_train, "steps_per_s": 1e3 / t_train,
                           "fp32_tflops": 3 * flops_fwd_row * B / (t_train / 1e3) / 1e12}}


def bench_sparsified(rend, torch, src, dirs, L, steps, pk, pk_kind):
    """Variable-NNZE tables from the device's L1-NNLS fine-tune (Eq. 14) of synthetic HRIR set
    4 (1250 directions x 2 ears) with the set's own resonance, at the paper's lambda = 1e-3,
    with D = I and with the window transform D_W (sigma = 60 samples, Eq. 16); each table
    keeps every non-zero (top-K with K = the largest NNZE).  The batch is rendered with them:
    throughput per mean NNZE of the sources' directions.  Plus the time of Algorithm 1's 50
    rounds (hrir_factorize) on the same set."""
    from paper_1502_03162_gb300 import hrir, synth
    X, _, _, p = synth.hrir_set(4)
    f = (p["res"] / np.linalg.norm(p["res"], axis=1, keepdims=True)).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    fd = torch.from_numpy(f).cuda()
    S = src.shape[0]
    units = S * L * 2
    out = torch.empty((2, L + 230), dtype=torch.float32, device="cuda")
    nb = lambda: None  # noqa: E731
    dirs_h = dirs.cpu().numpy()
    res = {}
    for name, lam, sigma in (("lam1e-3_DI", 1e-3, 0.0), ("lam1e-3_DW60", 1e-3, 60.0)):
        G = torch.empty((X.shape[0], 2, 200), dtype=torch.float32, device="cuda")
        nnz = torch.empty((X.shape[0], 2), dtype=torch.int32, device="cuda")
        fine = lambda: hrir.hrir_sparsify(rend.ctx, Xd, fd, 200, lam, sigma, 1e-4, G=G, nnz=nnz)  # noqa: E731,B023
        t_fine = time_steps(fine, 2, 1, torch, nb)
        k = int(nnz.max().item())
        idx, w, nn = rend.topk_pack(G, k)
        idx_h = (idx.cpu().numpy().astype(np.int64) & 0xFFFF).astype(np.uint16)
        nn_h = nn.cpu().numpy()
        rend.load_filters(idx_h, w.cpu().numpy(), nn_h, 200, f)
        rend.set_timing(True)
        rend.kernel_times(reset=True)
        t = time_steps(lambda: rend.render(src, dirs, mode="sparse", length=L, out=out), steps, 2,
                       torch, nb)
        kt = rend.kernel_times(reset=True)
        rend.set_timing(False)
        assert rend.sync() == 0
        nnze = float(nn_h[dirs_h].mean())          # taps per source-ear sample, this batch
        kms = kt["mix_sparse"][0] / max(kt["mix_sparse"][1], 1)
        roof = roofline_of(2.0 * nnze * units, S * L * 4.0, kms, pk, pk_kind)
        res[name] = {"value": units / (t / 1e3), "unit": "source-ear samples/s", "ms_per_step": t,
                     "mean_nnze": nnze, "max_nnze": k, "fine_tune_ms": t_fine,
                     "fine_tune_rows": int(X.shape[0] * 2), "roofline": roof}
    # Algorithm 1 itself on the device: the paper's 50 rounds over the set's 1250 x 2 HRIRs
    # from a seeded random start (the same start every run)
    G0 = torch.from_numpy(np.random.default_rng(3).random((X.shape[0], 2, 200), dtype=np.float32)).cuda()
    Gf = torch.empty_like(G0)

    def factorize():
        Gf.copy_(G0)
        hrir.hrir_factorize(rend.ctx, Xd, Gf, 200, iters=50)
    t_fact = time_steps(factorize, 2, 1, torch, nb)
    assert rend.sync() == 0
    res["factorize_50_rounds"] = {"ms": t_fact, "rows": int(X.shape[0] * 2), "rounds": 50}
    return res


def bench_precision(rend, torch, src, dirs, L, steps):
    """BF16/FP16 source storage: the sparse mix (FP32 arithmetic) and the per-source resonance
    on the tensor cores (Toeplitz-block GEMM, y * f for every source and ear)."""
    from paper_1502_03162_gb300 import hrir
    S = src.shape[0]
    units = S * L * 2
    out = torch.empty((2, L + 230), dtype=torch.float32, device="cuda")
    nb = lambda: None  # noqa: E731
    res = {}
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        s16 = src.to(dt)
        t = time_steps(lambda: rend.render(s16, dirs, mode="sparse", length=L, out=out),
                       steps, 2, torch, nb)
        res[f"sparse_{name}"] = {"value": units / (t / 1e3), "ms_per_step": t}
        if name == "bf16":
            u = torch.empty((S, 2, (L + 31 + 3) // 4 * 4), dtype=torch.float32, device="cuda")
            rend.set_timing(True)
            rend.kernel_times(reset=True)
            t = time_steps(lambda: hrir.hrir_resonance_per_source(rend.ctx, s16, length=L, out=u),
                           max(3, steps // 3), 1, torch, nb)
            kt = rend.kernel_times(reset=True)
            rend.set_timing(False)
            kms = kt["resonance_gemm"][0] / max(kt["resonance_gemm"][1], 1)
            bytes_alg = S * L * 2 + S * 2 * (L + 31) * 4
            res["resonance_gemm_bf16"] = {
                "value": units / (t / 1e3), "unit": "source-ear samples/s", "ms": t,
                "kernel_ms": kms, "hbm_gbs": bytes_alg / (kms / 1e3) / 1e9,
                "tensor_tflops": 768.0 * S * L / (kms / 1e3) / 1e12,
                "useful_tflops": 128.0 * S * L / (kms / 1e3) / 1e12}
            # the order (y * f) * g: u rendered to 1 and 4 direction sets by the taps alone
            rng = np.random.default_rng(21)
            dsets = torch.from_numpy(np.stack([rng.integers(0, 1250, S).astype(np.int32)
                                               for _ in range(4)])).cuda()
            dsets[0].copy_(dirs)
            vout = torch.empty((4, 2, L + 230), dtype=torch.float32, device="cuda")
            views = {}
            for nv in (1, 4):
                t = time_steps(lambda: hrir.hrir_render_precomputed(rend.ctx, u, dsets[:nv], length=L + 31,  # noqa: B023
                                                                     out=vout[:nv]),
                               max(3, steps // 3), 1, torch, nb)
                views[f"views{nv}"] = {"ms": t, "ms_per_view": t / nv,
                                       "value": nv * units / (t / 1e3), "unit": "source-ear samples/s"}
            res["precomputed_views_bf16"] = views
            del u
        del s16
    assert rend.sync() == 0
    return res


def fft_flops_per_unit(n_src, P=4096, hrir_len=231):
    """Algorithmic FP32 flops per source-ear sample of the overlap-save FFT path as built
    (frame P, hop B = P - G with G = H - 1 rounded up to 8): one complex P-point FFT (counted
    5 P log2 P) per source pair and frame serves both sources and both ears; one complex
    multiply-add (8 flops) per bin, source and ear; one inverse FFT per ear and frame,
    shared by all sources."""
    guard = (hrir_len - 1 + 7) // 8 * 8
    B = P - guard
    fft = 5.0 * P * np.log2(P)
    bins = P // 2 + 1
    return fft / (4.0 * B) + 8.0 * bins / B + fft / (n_src * B)


def roofline_of(flops, nbytes, kernel_ms, pk, pk_kind):
    """Roofline of one kernel launch: the binding roof (FP32 pipe or HBM) for its
    algorithmic flops and bytes, achieved = that quantity / the launch's duration."""
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_peak_tflops(sm_max)
    hbm_peak = float(pk["hbm_gbs"])
    t_alu = flops / (fp32_peak * 1e12)
    t_hbm = nbytes / (hbm_peak * 1e9)
    sec = kernel_ms / 1e3
    if t_alu >= t_hbm:
        achieved = flops / sec / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak}
    else:
        achieved = nbytes / sec / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak}
    roof["peak_source"] = (f"FP32 FMA: {N_SM} SMs x {FP32_LANES} lanes x 2 x {sm_max:.0f} MHz "
                           f"(sm_max_mhz of {pk_kind} peaks); HBM {hbm_peak:.0f} GB/s {pk_kind}")
    roof["kernel_ms"] = kernel_ms
    roof["algorithmic"] = {"flop": flops, "bytes": nbytes}
    roof["hbm_frac"] = nbytes / sec / 1e9 / hbm_peak
    roof["alu_frac"] = flops / sec / 1e12 / fp32_peak
    return roof


# per mode: the dominant kernel family, its algorithmic flops per source-ear sample, the
# profile summary that records its DRAM traffic
MODE_KERNELS = {"sparse": ("mix_sparse", "mix_sparse_tmem.cu", "mix_sparse_batched_1024x480000_k16.md"),
                "dense": ("mix_dense", "mix_direct.cu", "mix_dense_batched_256x480000.md"),
                "fft": ("fft", "fft.cu", "fft_mix_batched_256x480000.md")}


def mode_flops_per_unit(mode, k, n_src):
    if mode == "sparse":
        return 2.0 * k                   # one FMA per tap
    if mode == "dense":
        return 2.0 * 231                 # one FMA per HRIR tap
    return fft_flops_per_unit(n_src)


def run_sharded(args):
    """--shard: the batch's sources split over the ranks (contiguous slices), each rank renders
    the reflection mix of its slice, the mixes are gathered in rank order (all_gather, the one
    exchange: 2 x (L + 199) FP32 per rank) and every rank applies the resonance once to their
    sum (Sec. II linearity).  Strong scaling: every step renders the whole batch."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Replicas("nccl", device="cuda")
    rank, world, local = ranks.rank, ranks.world, ranks.local
    from paper_1502_03162_gb300 import hrir
    from paper_1502_03162_gb300.shard import render_sharded, shard_range
    import __graft_entry__
    __graft_entry__.build()
    S, L = args.sources, args.length
    cfg, host = make_inputs(S, L, seed=2, torch=torch)      # the same batch on every rank
    s0, s1 = shard_range(S, rank, world)
    rend = hrir.Renderer(local)
    G = torch.from_numpy(cfg["G"]).cuda()
    idx, w, nnz = rend.topk_pack(G, K_DEFAULT)
    idx_h = (idx.cpu().numpy().astype(np.int64) & 0xFFFF).astype(np.uint16)
    rend.load_filters(idx_h, w.cpu().numpy(), nnz.cpu().numpy(), 200, cfg["res"])
    host_slice = host[s0:s1]
    src = host_slice.cuda()
    dirs_h = torch.from_numpy(cfg["dirs"][s0:s1].copy())
    dirs = dirs_h.cuda()
    step = lambda: render_sharded(rend, src, dirs, length=L)  # noqa: E731
    pk, pk_kind = peaks()
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        rend.kernel_times(reset=True)
        rend.set_timing(True)
        clk.mark()
        ms = time_steps(step, args.steps, 0, torch, ranks.barrier)
        rend.set_timing(False)
    kt = rend.kernel_times(reset=True)
    assert rend.sync() == 0
    ms = ranks.max_over_ranks(ms)
    units = S * L * 2                                        # the whole batch, every step
    kms, kn = kt.get("mix_sparse", (0.0, 0))
    roof = roofline_of(2.0 * K_DEFAULT * (s1 - s0) * L * 2, (s1 - s0) * L * 4.0, kms / max(kn, 1),
                       pk, pk_kind)
    roof["traffic"] = profiled_traffic(*MODE_KERNELS["sparse"][1:])
    roof["traffic"] = roof["traffic"] * (s1 - s0) / S if roof["traffic"] else None
    # end to end: this rank's slice from pinned host memory, the sharded render, the output back
    out_h = torch.empty((2, L + 230), dtype=torch.float32, pin_memory=True)

    def e2e_step():
        src.copy_(host_slice, non_blocking=True)
        out_h.copy_(render_sharded(rend, src, dirs, length=L))
    e2e_step()
    torch.cuda.synchronize()
    ranks.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(2, args.steps // 4)
    for _ in range(e2e_steps):
        e2e_step()
    e2e_ms = ranks.max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps)
    result = {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": "source-ear samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded AR(1) sources, synthetic 1250-direction filters)",
        "config": {"workload": WORKLOAD if (S, L) == (S_DEFAULT, L_DEFAULT)
                   else f"{S} sources x {L} samples AR(1), 1250 directions, K=16 of 200 taps, Lf=32",
                   "sources": S, "length": L, "k": K_DEFAULT, "refl_len": 200, "res_len": 32,
                   "mode": "sparse, sharded",
                   "l2": f"inputs larger than L2 ({S * L * 4 / 1e9:.2f} GB source batch), no flush",
                   "parallelism": f"source shards x{world} (reflection mixes gathered, resonance once)"},
        "roofline": roof,
        "gpu_launches": int(sum(n for _, n in kt.values())),
        "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in kt.items()},
        "clocks": clk.summary(),
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": "source-ear samples/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int((s1 - s0) * host.shape[1] * 4),
                "d2h_bytes_per_step": int(2 * (L + 230) * 4)},
    }
    if rank == 0:
        print(json.dumps(result))
    rend.close()
    ranks.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sources", type=int, default=S_DEFAULT)
    ap.add_argument("--length", type=int, default=L_DEFAULT)
    ap.add_argument("--mode", default="sparse", choices=["sparse", "dense", "fft"],
                    help="path of the headline step (dense and fft for profiling the baselines)")
    ap.add_argument("--no-extras", action="store_true", help="only the headline path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stream", action="store_true", help="skip the serving-loop benchmark")
    ap.add_argument("--shard", action="store_true",
                    help="split the batch's sources over the ranks (strong scaling) instead of "
                         "one independent batch per rank")
    ap.add_argument("--learned-sources", type=int, default=4096,
                    help="moving sources of the learned-filter workload (smaller for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.shard:
        run_sharded(args)
        return

    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Replicas("nccl", device="cuda")
    rank, world, local = ranks.rank, ranks.world, ranks.local
    barrier, max_over_ranks = ranks.barrier, ranks.max_over_ranks

    from paper_1502_03162_gb300 import hrir
    import __graft_entry__
    __graft_entry__.build()
    S, L = args.sources, args.length
    cfg, host = make_inputs(S, L, seed=ranks.seed(2), torch=torch)
    rend = hrir.Renderer(local)
    G = torch.from_numpy(cfg["G"]).cuda()
    src = host.cuda()
    dirs_h = torch.from_numpy(cfg["dirs"])
    dirs = dirs_h.cuda()
    out = torch.empty((2, L + 230), dtype=torch.float32, device="cuda")
    pk, pk_kind = peaks()
    units = S * L * 2
    src_bytes = S * L * 4.0

    def load(k):
        idx, w, nnz = rend.topk_pack(G, k)
        idx_h = (idx.cpu().numpy().astype(np.int64) & 0xFFFF).astype(np.uint16)
        rend.load_filters(idx_h, w.cpu().numpy(), nnz.cpu().numpy(), 200, cfg["res"])
        return idx_h, w.cpu().numpy(), nnz.cpu().numpy()

    def timed_path(mode, steps, warmup, k=K_DEFAULT):
        """ms per step of one path with its kernels timed by the library's CUDA events on
        the launching stream; returns (ms, roofline of the dominant kernel, launches)."""
        fn = lambda: rend.render(src, dirs, mode=mode, length=L, out=out)  # noqa: E731
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        rend.kernel_times(reset=True)
        rend.set_timing(True)
        t = time_steps(fn, steps, 0, torch, barrier)
        rend.set_timing(False)
        kt = rend.kernel_times(reset=True)
        assert rend.sync() == 0
        fam, kfile, prof = MODE_KERNELS[mode]
        kms, kn = kt.get(fam, (0.0, 0))
        roof = roofline_of(mode_flops_per_unit(mode, k, S) * units, src_bytes, kms / max(kn, 1),
                           pk, pk_kind)
        roof["traffic"] = profiled_traffic(kfile, prof)
        return max_over_ranks(t), roof, int(sum(n for _, n in kt.values())), kt

    tables16 = load(K_DEFAULT)
    mode = args.mode
    step = lambda: rend.render(src, dirs, mode=mode, length=L, out=out)  # noqa: E731
    # headline: kernel timing on, clocks sampled from before the warm-up
    rend.set_timing(False)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        rend.kernel_times(reset=True)
        rend.set_timing(True)
        clk.mark()
        ms = time_steps(step, args.steps, 0, torch, barrier)
        rend.set_timing(False)
    ktimes = rend.kernel_times(reset=True)
    assert rend.sync() == 0
    ms = max_over_ranks(ms)
    value = ranks.whole_job(units, ms)

    # kernel-level roofline of the dominant kernel
    fam, kfile, prof = MODE_KERNELS[mode]
    kms, kn = ktimes.get(fam, (0.0, 0))
    roof = roofline_of(mode_flops_per_unit(mode, K_DEFAULT, S) * units, src_bytes,
                       kms / max(kn, 1), pk, pk_kind)
    roof["traffic"] = profiled_traffic(kfile, prof)

    result = {
        "metric": METRIC, "value": value, "unit": "source-ear samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded AR(1) sources, synthetic 1250-direction filters)",
        "config": {"workload": WORKLOAD if (S, L, mode) == (S_DEFAULT, L_DEFAULT, "sparse")
                   else f"{S} sources x {L} samples AR(1), 1250 directions, K=16 of 200 taps, "
                        f"Lf=32, {mode} path",
                   "sources": S, "length": L, "k": K_DEFAULT,
                   "refl_len": 200, "res_len": 32, "mode": mode,
                   "l2": f"inputs larger than L2 ({src_bytes / 1e9:.2f} GB source batch), no flush",
                   "parallelism": f"replicas x{world} (independent batches)"},
        "roofline": roof,
        "gpu_launches": int(sum(n for _, n in ktimes.values())),
        "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in ktimes.items()},
        "clocks": clk.summary(),
    }

    if not args.no_extras:
        extras = {}
        # the plain methods on the same batch and filters: dense-HRIR direct convolution and
        # overlap-save FFT convolution (P = 4096)
        for m, steps in (("dense", max(2, args.steps // 5)), ("fft", max(3, args.steps // 5))):
            t, r_m, _, _ = timed_path(m, steps, 2)
            extras[f"{m}_k16" if m == "dense" else "fft_p4096"] = {
                "value": ranks.whole_job(units, t), "ms_per_step": t, "roofline": r_m}
        for k in (8, 32):
            load(k)
            t, r_k, _, _ = timed_path("sparse", max(3, args.steps // 2), 2, k=k)
            extras[f"sparse_k{k}"] = {"value": ranks.whole_job(units, t), "ms_per_step": t,
                                      "roofline": r_k}
        load(K_DEFAULT)
        if mode == "sparse":
            extras["sparse_k16"] = {"value": value, "ms_per_step": ms, "roofline": roof}
        result["paths"] = extras

    # end to end through the public host-buffer call: H2D of the pinned batch, render, D2H
    host_out = torch.empty((2, L + 230), dtype=torch.float32, pin_memory=True)
    e2e_step = lambda: rend.render_host(host, dirs_h, mode=mode, length=L, out=host_out)  # noqa: E731
    e2e_steps = max(2, args.steps // 4)
    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms)
    h2d = int(S * host.shape[1] * 4 + S * 4)
    # the host link's own rate: one plain copy of the same pinned batch, CUDA events
    copy_ms = time_steps(lambda: src.copy_(host, non_blocking=True), 3, 1, torch, barrier)
    link_gbs = S * host.shape[1] * 4 / (copy_ms / 1e3) / 1e9
    e2e_link = h2d / (e2e_ms / 1e3) / 1e9
    result["e2e"] = {"value": ranks.whole_job(units, e2e_ms), "unit": "source-ear samples/s",
                     "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": int(2 * (L + 230) * 4),
                     "host_link_gbs": e2e_link, "host_copy_gbs": link_gbs,
                     "host_link_frac": e2e_link / link_gbs}

    if not args.no_extras:
        result["sparsified"] = bench_sparsified(rend, torch, src, dirs, L, max(3, args.steps // 5),
                                                pk, pk_kind)
        load(K_DEFAULT)
        result["precision"] = bench_precision(rend, torch, src, dirs, L, max(3, args.steps // 5))
        result["learned"] = bench_learned(rend, torch, S=args.learned_sources)

    if not args.no_stream:
        load(K_DEFAULT)
        st = {f"B{b}": bench_stream(rend, torch, b) for b in (256, 128)}
        # admission bound by the device pool: 256 MiB holds about 1400 s of audio, below the
        # ~5200 s that the ~1000 concurrent sources of the unconstrained loop hold
        st["B256_pool256MiB"] = bench_stream(rend, torch, 256, pool_bytes=256 << 20)
        result["stream"] = st
        result["p99_block_latency_ms"] = {k: v["p99_ms"] for k, v in st.items()}

    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(cfg, *tables16, cfg["res"])
    if rank == 0:
        print(json.dumps(result))
    rend.close()
    ranks.close()


if __name__ == "__main__":
    main()
