"""Benchmark of the SEM Q-isosurface render path on GB300.

One step = one snapshot through the whole path, as one CUDA graph: Q on all elements with its
isosurfaces (sem_qcriterion_isosurface_async: the Q kernel also counts each element's
triangles), the other field's isosurfaces appended behind them (no host synchronisation, one
triangle buffer) and one sem_render_async of the frame.

Headline workload (the largest single-GPU configuration): the Rayleigh-Benard-like box of
64x64x64 elements, N = 7 (134M GLL nodes), velocity and temperature (2.15 GB of FP32), the
Q-isosurface at 0.1 max Q and the temperature isosurface T = 0.5, one 3840x2160 perspective
frame.  The 32^3-element channel (16.8M nodes, three Q isovalues, 1920x1080) is measured the
same way and reported under ``extra``.

Prints one JSON line (rank 0).  ``value`` is elements/s with the inputs already resident in
HBM; ``e2e`` is the same metric with every step's inputs copied from pinned host memory and the
frame read back inside the timed region.  ``roofline`` reports the dominant kernel against the
measured HBM bandwidth; ``cpu_baseline`` times the FP64 CPU oracle on bounded samples, on one
host thread and on all host cores.

``--impl reference`` times the CPU oracle alone (the reference arm) on the same workload.
Under torchrun each rank runs an independent replica on its own GPU (weak scaling).
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SEM elements/s through Q-isosurface render; frames/s; fraction of HBM roofline"
UNIT = "elements/s"
WORKLOADS = {
    "rb64": "RB-like 64x64x64 elements, N=7 (134M GLL nodes), velocity + temperature (2.15 GB FP32), "
            "Q-isosurface at 0.1 max Q + temperature isosurface T=0.5, one 3840x2160 perspective frame",
    "channel32": "channel 32x32x32 elements, N=7 (16.8M GLL nodes), 512 Fourier modes, 3 Q-isosurfaces, "
                 "1920x1080 perspective",
    # the headline's structure at 1/8 size (the small case for profiling)
    "rb32": "RB-like 32x32x32 elements, N=7 (16.8M GLL nodes), velocity + temperature (268 MB FP32), "
            "Q-isosurface at 0.1 max Q + temperature isosurface T=0.5, one 1920x1080 perspective frame",
}
HEADLINE = "rb64"
# segment colours of the two-field frame: Q red, temperature blue
RB_COLOURS = [[0.9, 0.3, 0.2], [0.2, 0.5, 0.9]]
KERNEL_SOURCES = {"k_sem_grad": "paper_2312_09888_gb300/csrc/sem_qcrit.cu",
                  "k_sem_qd": "paper_2312_09888_gb300/csrc/sem_qcrit.cu",
                  "k_sem_q8": "paper_2312_09888_gb300/csrc/sem_qcrit.cu",
                  "k_sem_q8_count": "paper_2312_09888_gb300/csrc/sem_qcrit.cu",
                  "k_iso_count_m": "paper_2312_09888_gb300/csrc/sem_iso.cu",
                  "k_iso_count_p": "paper_2312_09888_gb300/csrc/sem_iso.cu",
                  "k_iso_emit_m": "paper_2312_09888_gb300/csrc/sem_iso.cu",
                  "k_raster_small": "paper_2312_09888_gb300/csrc/sem_render.cu",
                  "k_resolve": "paper_2312_09888_gb300/csrc/sem_render.cu"}


def algorithmic_bytes_per_step(name, P):
    """Bytes a kernel must move per step at the least (each input read once, each output
    written once), summed over its launches in the step."""
    NP3 = (P.N + 1) ** 3
    surf = P.surface_stats
    table = {
        # one component read (4 B/node) + its three derivatives written (12 B/node)
        "k_sem_grad": 16 * P.npts,
        # u, v, w read (12 B/node) + Q written (4 B/node)
        "k_sem_qd": 16 * P.npts,
        "k_sem_q8": 16 * P.npts,
        # the same, the Q field's triangle counts written from the kernel (4 B per element and isovalue)
        "k_sem_q8_count": 16 * P.npts + 4 * P.E * P.surface_stats[0]["niso"],
        # per field counted by a separate pass (every field but Q, whose counts come from the fused
        # Q kernel): read once for all its isovalues + one int32 count per element and isovalue
        "k_iso_count_m": sum(4 * P.npts + 4 * P.E * s["niso"] for s in surf[1:]),
        "k_iso_count_p": sum(4 * P.npts + 4 * P.E * s["niso"] for s in surf[1:]),
        # per field: its active elements read + 36 B per triangle written + the offsets read
        "k_iso_emit_m": sum(4 * NP3 * s["active_elems"] + 36 * s["ntri"] + 8 * (s["niso"] * P.E + 1) for s in surf),
        # 36 B per triangle read (the 64-bit depth keys live in L2)
        # (a frame drawn in parts: Q's part one tile per block, the other fields' parts as ranges)
        "k_raster_small": 36 * (P.last_ntri if P.nseg == len(P.surfaces[0][1]) else P.surface_stats[0]["ntri"]),
        "k_raster_range": 36 * sum(st["ntri"] for st in P.surface_stats[1:]),
        # key read 8 B + RGBA 4 B + depth 4 B per pixel, and the winner's colour per covered pixel
        "k_resolve": 16 * P.W * P.H + 4 * P.covered,
    }
    return table.get(name)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(per_rank_elems, per_rank_seconds):
    """Whole-job throughput: all units processed / the slowest rank's time."""
    return float(sum(per_rank_elems)) / float(max(per_rank_seconds))


def max_over_ranks(x: float, device) -> float:
    """Largest value of x over the ranks of the default process group (x itself if none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _file_sha(path):
    """Hash of a source file's code: comments and whitespace removed, so that a counter capture
    stays matched to its kernel through comment edits and is dropped by any code change."""
    import re
    with open(os.path.join(ROOT, path)) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256(" ".join(src.split()).encode()).hexdigest()[:16]


def _traffic_for(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, or None if absent or stale."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(f"{workload}:{kernel}")
        if d and d.get("source_sha") == _file_sha(KERNEL_SOURCES[kernel]):
            return d.get("bytes_per_launch_full")
    except Exception:
        return None
    return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        """Start sampling every 20 ms; returns once the first sample is written, so that the
        samples that follow fall inside the region timed next."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t_end = time.time() + 10.0
            while time.time() < t_end and self.proc.poll() is None and not self._rows():
                time.sleep(0.01)
            self.skip = len(self._rows())
        except Exception:
            self.proc = None

    def _rows(self):
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 9:
                rows.append(f)
        return rows

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self._rows()
        os.unlink(self.path)
        # samples taken while the timed region ran (at least the last one before it ended)
        rows = rows[self.skip:] or rows[-1:]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------ workload

def make_workload(name, device):
    import sem_inputs as si
    if name == "rb64":
        return si.rb_box(device=device)
    if name == "rb32":
        return si.rb_box(nel=32, W=1920, H=1080, device=device)
    return si.channel(device=device)


class Pipeline:
    """Device buffers and the per-step call sequence through the C ABI.

    Inputs: the velocity (and, on the Rayleigh-Benard-like box, the temperature), FP32 on the
    device.  Surfaces: Q at the workload's fractions of max Q (fixed once at setup from the GPU's
    Q), then the temperature at its isovalue; their triangles share one buffer, one colour
    segment per (field, isovalue)."""

    def __init__(self, S, w, device_index=0, autotune=True):
        import numpy as np
        import torch
        self.S, self.w, self.torch = S, w, torch
        self.stream = torch.cuda.current_stream()
        self.sess = S.Session(device_index, self.stream)
        self.ctx = self.sess.ctx
        if not autotune:
            S.sem_autotune_set(self.ctx, False)
        xyz = w.mesh.xyz(w.fields.device).cpu().numpy()
        self.mesh = self.sess.mesh(w.mesh.N, xyz)
        del xyz
        self.N = w.mesh.N
        self.E = w.E
        self.npts = w.E * w.mesh.NP ** 3
        self.inputs = [w.fields[c].float().contiguous() for c in range(w.fields.shape[0])]
        w.fields = None  # the FP64 originals are not needed past this point
        torch.cuda.empty_cache()
        self.Q = torch.empty_like(self.inputs[0])
        S.sem_qcriterion(self.ctx, self.mesh, *self.inputs[:3], self.Q)
        qmax = S.sem_field_max(self.ctx, self.Q)
        self.surfaces = [("Q", [float(np.float32(f * qmax)) for f in w.iso_fracs])]
        if "t_iso" in w.extra:
            self.surfaces.append((3, [float(np.float32(w.extra["t_iso"]))]))
        self.colours = RB_COLOURS if len(self.surfaces) > 1 else None
        self.nseg = sum(len(isos) for _, isos in self.surfaces)
        counts = [S.sem_isosurface_multi(self.ctx, self.mesh, self.field(src), isos, None)
                  for src, isos in self.surfaces]
        total = sum(sum(c) for c in counts)
        self.cap = int(total * 1.05) + 1024
        self.tris = torch.empty(self.cap * 9, device="cuda")
        self.W, self.H = w.camera["W"], w.camera["H"]
        self.rgba = torch.empty(self.W * self.H * 4, dtype=torch.uint8, device="cuda")
        self.depth = torch.empty(self.W * self.H, device="cuda")
        self.counts_dev = torch.zeros(self.nseg + 1, dtype=torch.int64, device="cuda")
        self.graph = None
        # per field: isovalues, triangles, and the elements holding a triangle (the emit pass
        # reads only those)
        self.surface_stats = []
        te = torch.empty(self.cap, dtype=torch.int32, device="cuda")
        for (src, isos), c in zip(self.surfaces, counts):
            S.sem_isosurface_multi(self.ctx, self.mesh, self.field(src), isos, self.tris, tri_elem=te, cap=self.cap)
            n = sum(c)
            self.surface_stats.append({"field": "Q" if src == "Q" else "T", "niso": len(isos), "isovalues": isos,
                                       "ntri": n, "active_elems": int(torch.unique(te[:n]).numel()) if n else 0})
        del te
        self.covered = 0
        self.last_ntri = total

    def field(self, src, inputs=None):
        return self.Q if src == "Q" else (inputs or self.inputs)[src]

    def step_async(self, inputs=None, rgba=None, depth=None, events=None):
        """The step without host synchronisation, one library call: Q with its isosurfaces (the
        counting of Q's triangles runs inside the Q kernel), the other fields' isosurfaces on the
        library's auxiliary stream, overlapping Q's scan and emit, and the frame, each stream
        drawing the segments it has just emitted before one resolve.  `events` (4 CUDA events)
        bracket the call (events 1 and 2 both mark its start)."""
        S, ctx, m = self.S, self.ctx, self.mesh
        inputs = inputs or self.inputs
        if events is not None:
            for e in events[:3]:
                e.record(self.stream)
        (src0, q_isos), rest = self.surfaces[0], self.surfaces[1:]
        assert src0 == "Q"
        S.sem_frame_async(ctx, m, *inputs[:3], self.Q, q_isos, [self.field(src, inputs) for src, _ in rest],
                          [isos for _, isos in rest], self.tris, self.counts_dev, self.colours, self.w.camera,
                          self.W, self.H, self.rgba if rgba is None else rgba, self.depth if depth is None else depth,
                          cap=self.cap)
        if events is not None:
            events[3].record(self.stream)

    def capture(self):
        """One CUDA graph per step: Q -> isosurfaces -> frame."""
        self.graph = self.capture_with(self.inputs, self.rgba, self.depth)

    def capture_with(self, inputs, rgba, depth):
        """A graph of the step reading `inputs` and writing `rgba`, `depth` (Q, triangles and
        counts are shared: the steps run one after another on one stream)."""
        torch = self.torch
        self.step_async(inputs, rgba, depth)  # sizes the library scratch outside the capture
        self.S.sem_synchronize(self.ctx)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.S.sem_set_stream(self.ctx, torch.cuda.current_stream())
            self.step_async(inputs, rgba, depth)
        self.S.sem_set_stream(self.ctx, self.stream)
        return g

    def step(self):
        """The host-synchronised form of the step (exact triangle counts back on the host)."""
        S, ctx, m = self.S, self.ctx, self.mesh
        S.sem_qcriterion(ctx, m, *self.inputs[:3], self.Q)
        off, segs = 0, []
        for src, isos in self.surfaces:
            c = S.sem_isosurface_multi(ctx, m, self.field(src), isos, self.tris[off * 9:], cap=self.cap - off)
            segs += c
            off += sum(c)
        S.sem_render(ctx, self.tris, off, segs, self.colours, self.w.camera, self.W, self.H, self.rgba, self.depth)
        self.last_ntri = off
        return off


# GEMM shapes (M, N, K as executed, padded) of the autoencoder's training step at batch B
def _ae_gemm_shapes(B):
    return {"fwd1": (B, 512, 1536), "fwd2": (B, 64, 512), "fwd3": (B, 512, 64), "fwd4": (B, 1536, 512),
            "dx4": (B, 512, 1536), "dw4": (1536, 512, B), "dx3": (B, 64, 512), "dw3": (512, 64, B),
            "dx2": (B, 512, 64), "dw2": (128, 512, B), "dw1": (512, 1536, B)}


def measure_in_transit(S, ctx, ae, steps=50, warmup=4):
    """The in-transit use of the learned compression, end to end on the Taylor-Green snapshot of
    32^3 elements (N = 7): per step either the velocity (201 MB FP32) or its latent (3.1 MB BF16)
    comes from pinned host memory, the latent is decoded on the device, then Q, the isosurface at
    0.1 max Q and a 1920x1080 frame, read back to pinned host memory.  Both forms are one CUDA
    graph per step, pipelined over two device slots."""
    import math as _m
    import torch
    import sem_inputs as si
    f = si.ae_snapshot(203, nel=32, device="cuda")
    E = f.shape[1]
    mesh = si.uniform_box((32,) * 3, (0.0,) * 3, (2 * _m.pi,) * 3, 7)
    m = S.sem_load_mesh(ctx, 7, mesh.xyz().numpy())
    cam = si.box_camera_persp((0.0,) * 3, (2 * _m.pi,) * 3, 1920, 1080)
    W, H = 1920, 1080
    Q = torch.empty_like(f[0])
    S.sem_qcriterion(ctx, m, f[0].contiguous(), f[1].contiguous(), f[2].contiguous(), Q)
    iso = [float(0.1 * S.sem_field_max(ctx, Q))]
    n = S.sem_isosurface_multi(ctx, m, Q, iso, None)
    cap = int(sum(n) * 1.5) + 4096
    tris = torch.empty(cap * 9, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    lat_host = torch.empty(E * 48, dtype=torch.bfloat16)
    lat_dev = torch.empty(E * 48, dtype=torch.bfloat16, device="cuda")
    S.sem_ae_encode(ctx, ae, f[0].contiguous(), f[1].contiguous(), f[2].contiguous(), lat_dev)
    lat_host.copy_(lat_dev.cpu())
    lat_host = lat_host.pin_memory()
    vel_host = [f[c].cpu().pin_memory() for c in range(3)]

    def make_slot(from_latent):
        sl = dict(vel=[torch.empty_like(f[c]) for c in range(3)], rgba=torch.empty(W * H * 4, dtype=torch.uint8,
                                                                                     device="cuda"),
                  depth=torch.empty(W * H, device="cuda"), lat=torch.empty_like(lat_dev))
        if from_latent:
            sl["lat"].copy_(lat_dev)
        else:
            for c in range(3):
                sl["vel"][c].copy_(f[c])

        def step():
            if from_latent:
                S.sem_ae_decode(ctx, ae, sl["lat"], E, *sl["vel"])
            S.sem_qcriterion(ctx, m, *sl["vel"], Q)
            S.sem_isosurface_multi_async(ctx, m, Q, iso, tris, cnt, cap=cap)
            S.sem_render_async(ctx, tris, cap, cnt, 1, None, cam, W, H, sl["rgba"], sl["depth"])

        step()
        S.sem_synchronize(ctx)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            S.sem_set_stream(ctx, torch.cuda.current_stream())
            step()
        S.sem_set_stream(ctx, stream)
        sl["replay"] = g.replay
        sl["graph"] = g
        return sl

    img_host = torch.empty(W * H * 4, dtype=torch.uint8).pin_memory()
    dep_host = torch.empty(W * H, dtype=torch.float32).pin_memory()

    def timed(from_latent):
        slots = [make_slot(from_latent), make_slot(from_latent)]
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in, ev_done, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
        used = [False, False]

        def one(k):
            sl = slots[k % 2]
            i = k % 2
            with torch.cuda.stream(h2d):
                if used[i]:
                    h2d.wait_event(ev_out[i])
                if from_latent:
                    sl["lat"].copy_(lat_host, non_blocking=True)
                else:
                    for c in range(3):
                        sl["vel"][c].copy_(vel_host[c], non_blocking=True)
                ev_in[i].record(h2d)
            stream.wait_event(ev_in[i])
            sl["replay"]()
            ev_done[i].record(stream)
            with torch.cuda.stream(d2h):
                d2h.wait_event(ev_done[i])
                img_host.copy_(sl["rgba"], non_blocking=True)
                dep_host.copy_(sl["depth"], non_blocking=True)
                ev_out[i].record(d2h)
            used[i] = True

        for k in range(warmup):
            one(k)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(h2d)
        for k in range(steps):
            one(k)
        b.record(d2h)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    ms_plain, ms_lat = timed(False), timed(True)
    S.sem_synchronize(ctx)
    S.sem_mesh_free(m)
    eps = lambda ms: round(E / (ms * 1e-3), 1)  # noqa: E731
    return {"workload": "Taylor-Green 32^3 elements, N=7, Q-isosurface at 0.1 max Q, 1920x1080, end to end",
            "velocity_in": {"h2d_bytes_per_step": int(E * 1536 * 4), "ms_per_step": round(ms_plain, 4),
                            "elements_per_s": eps(ms_plain)},
            "latent_in": {"h2d_bytes_per_step": int(E * 96), "ms_per_step": round(ms_lat, 4),
                          "elements_per_s": eps(ms_lat)}}


def measure_learned(S, ctx, bf16_peak, peak_src, steps=100, warmup=20):
    """The learned per-element compression on the benchmark's scale: AdamW steps of the
    1536-512-48-512-1536 BF16 autoencoder at batch 8192 on samples of 8 Taylor-Green snapshots
    of 32^3 elements (not part of the timed frame step), and encode/decode of one snapshot."""
    import torch
    import sem_inputs as si
    B = 8192
    train = torch.cat([si.ae_samples(si.ae_snapshot(s, nel=32, device="cuda")) for s in range(0, 200, 25)])
    ae = S.sem_ae_create(ctx, B)
    stream = torch.cuda.current_stream()
    try:
        S.sem_ae_set_params(ctx, ae, si.ae_init_params())
        S.sem_ae_fit_normalization(ctx, ae, train[:32768])
        g = torch.Generator(device="cuda")
        g.manual_seed(si.seed_for(5, 2000))
        idx = torch.randint(0, train.shape[0], (steps + warmup, B), generator=g, device="cuda")
        for i in range(warmup):
            S.sem_ae_train_step(ctx, ae, train, idx[i], lr=1e-4)
        torch.cuda.synchronize()
        S.sem_trace_enable(ctx, True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(warmup, warmup + steps):
            S.sem_ae_train_step(ctx, ae, train, idx[i], lr=1e-4)
        b.record(stream)
        torch.cuda.synchronize()
        trace = S.sem_trace_collect(ctx)
        S.sem_trace_enable(ctx, False)
        step_ms = a.elapsed_time(b) / steps
        shapes = _ae_gemm_shapes(B)
        gemm = {}
        for name, (M, N, K) in shapes.items():
            ms, n = trace.get("k_gemm_bf16 " + name, (0.0, 0))
            if n:
                t = ms / n
                gemm[name] = {"ms": round(t, 5), "tflops": round(2.0 * M * N * K / (t * 1e-3) / 1e12, 1)}
        gemm_ms = sum(v["ms"] for v in gemm.values())
        gemm_flops = sum(2.0 * M * N * K for M, N, K in shapes.values())
        dims = [(1536, 512), (512, 48), (48, 512), (512, 1536)]
        model_flops = 2.0 * B * (2 * sum(i * o for i, o in dims) + sum(i * o for i, o in dims[1:]))
        best = max(gemm, key=lambda k: gemm[k]["tflops"])
        # encode + decode of one snapshot (32768 elements)
        f = si.ae_snapshot(201, nel=32, device="cuda")
        E = f.shape[1]
        lat = torch.empty(E * 48, dtype=torch.bfloat16, device="cuda")
        out = [torch.empty(E, 512, device="cuda") for _ in range(3)]
        uvw = [f[c].contiguous() for c in range(3)]
        for _ in range(3):
            S.sem_ae_encode(ctx, ae, *uvw, lat)
            S.sem_ae_decode(ctx, ae, lat, E, *out)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        for _ in range(10):
            S.sem_ae_encode(ctx, ae, *uvw, lat)
        e1.record(stream)
        for _ in range(10):
            S.sem_ae_decode(ctx, ae, lat, E, *out)
        e2.record(stream)
        torch.cuda.synchronize()
        enc_ms, dec_ms = e0.elapsed_time(e1) / 10, e1.elapsed_time(e2) / 10
        # a short training run so the decoded field looks like the data, then the in-transit form
        for i in range(3000):
            S.sem_ae_train_step(ctx, ae, train, idx[i % (steps + warmup)], lr=1e-3 * (1.0 - i / 3000.0) + 1e-5)
        in_transit = measure_in_transit(S, ctx, ae)
        return {"model": "per-element autoencoder 1536-512-48-512-1536, BF16 tensor cores, FP32 accumulation",
                "train_batch": B, "train_ms_per_step": round(step_ms, 4),
                "train_samples_per_s": round(B / (step_ms * 1e-3), 1),
                "train_model_tflops": round(model_flops / (step_ms * 1e-3) / 1e12, 1),
                "gemm_share_of_step": round(gemm_ms / step_ms, 3),
                "gemm_tflops_all": round(gemm_flops / (gemm_ms * 1e-3) / 1e12, 1),
                "roofline": {"kernel": "k_gemm_bf16 " + best, "bound": "tensor",
                             "achieved": gemm[best]["tflops"], "peak": bf16_peak, "peak_source": peak_src,
                             "unit": "TFLOP/s", "frac": round(gemm[best]["tflops"] / bf16_peak, 4)},
                "gemms": gemm,
                # the autotuner's choice per (M, N, K, epilogue): tile width, stages, K split, persistent
                "gemm_choices": [{"shape": [c[0], c[1], c[2]], "epilogue": c[3], "bn": c[4], "stages": c[5],
                                  "split": c[6], "persistent": c[7], "ms": round(c[8], 5)}
                                 for c in S.sem_autotune_choices(ctx)],
                "encode_elements_per_s": round(E / (enc_ms * 1e-3), 1),
                "decode_elements_per_s": round(E / (dec_ms * 1e-3), 1),
                "latent_bytes_per_element": 96, "in_transit": in_transit}
    finally:
        S.sem_ae_destroy(ae)
        del train
        torch.cuda.empty_cache()


def measure_curved(S, ctx, vel, box_mesh, steps=20, warmup=3):
    """sem_qcriterion on a general (curved) mesh of the benchmark's size: 32^3 elements, N = 7,
    interior element corners moved by up to 0.15 element sizes (sem_inputs.perturbed_box), the
    benchmark's velocity values; against the same call on the box mesh.  Algorithmic bytes:
    16 B per node (u, v, w in, Q out) plus 36 B per node of inverse Jacobian on the curved mesh."""
    import time
    import torch
    import sem_inputs as si
    xyz = si.perturbed_box((32, 32, 32), (0.0, -1.0, 0.0), (2 * 3.141592653589793, 1.0, 3.141592653589793), 7,
                           amp=0.15, seed=si.seed_for(2, 99))
    t0 = time.perf_counter()
    m = S.sem_load_mesh(ctx, 7, xyz)
    load_s = time.perf_counter() - t0
    Q = torch.empty_like(vel[0])
    nodes = vel[0].numel()
    out = {"mesh": "32^3 elements, N=7, interior corners moved up to 0.15 element sizes", "load_s": round(load_s, 2)}
    for name, mesh, per_node in (("curved", m, 52), ("box", box_mesh, 16)):
        for _ in range(warmup):
            S.sem_qcriterion(ctx, mesh, *vel, Q)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            S.sem_qcriterion(ctx, mesh, *vel, Q)
        b.record()
        torch.cuda.synchronize()
        us = a.elapsed_time(b) / steps * 1e3
        out[name] = {"us": round(us, 1), "gbs": round(per_node * nodes / (us * 1e-6) / 1e9, 1)}
    S.sem_mesh_free(m)
    return out


BATCH_FRACS = (0.05, 0.1, 0.2, 0.4)


def measure_batched(S, ctx, snapshots=64, steps=3):
    """The batching workload (one CUDA graph per time step): 64 snapshots of the Taylor-Green
    field with phase 2 pi s / 64 in x and y and 1e-3 noise, each over 16 partitions of uneven
    size and mixed order (batched_partitions); per snapshot Q of every partition
    (sem_qcriterion_batch: one persistent launch per order), the isosurfaces of Q and of u at
    {0.05, 0.1, 0.2, 0.4} of their maxima, every partition's appended behind the previous one's in
    one triangle buffer per field, and one 1024x1024 frame per (snapshot, field, isovalue), each
    drawing that isovalue's segments of all 16 partitions (sem_render_segments_async): 512 frames
    per graph.  The snapshots' velocities stay resident (as a solver's fields would be); when
    they do not fit in 60 % of the free memory, the graph cycles over as many distinct ones as
    fit (each still larger than L2).  Against the same calls issued eagerly with the host waiting
    for every snapshot (the plain path)."""
    import numpy as np
    import torch
    import sem_inputs as si
    t_setup = time.perf_counter()
    parts = si.batching_partitions()
    E_total = sum(p["E"] for p in parts)
    nodes = sum(p["E"] * (p["N"] + 1) ** 3 for p in parts)
    free, _ = torch.cuda.mem_get_info()
    distinct = int(max(1, min(snapshots, (0.6 * free) // (12 * nodes + 1))))
    phases = [2 * math.pi * s / 64 for s in range(distinct)]
    for p in parts:
        p["m"] = S.sem_load_mesh(ctx, p["N"], p["mesh"].xyz_range(0, p["E"]))
        p["snap"] = [v.contiguous() for v in si.taylor_green_snapshots(p["mesh"], p["E"], phases, 1e-3,
                                                                        si.seed_for(4, 1 + len(parts)), "cuda")]
        p["Q"] = torch.empty(p["E"] * (p["N"] + 1) ** 3, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_setup
    meshes = [p["m"] for p in parts]

    def comps(d):
        return [[p["snap"][d][c].view(-1) for p in parts] for c in range(3)]

    # isovalues from snapshot 0's maxima (setup, untimed)
    u0, v0, w0 = comps(0)
    S.sem_qcriterion_batch(ctx, meshes, u0, v0, w0, [p["Q"] for p in parts])
    qmax = max(S.sem_field_max(ctx, p["Q"]) for p in parts)
    umax = max(S.sem_field_max(ctx, u) for u in u0)
    isos = [[float(np.float32(f * qmax)) for f in BATCH_FRACS], [float(np.float32(f * umax)) for f in BATCH_FRACS]]
    # triangle buffers sized by the largest snapshot (counts of every snapshot, host-synchronised)
    need = [0, 0]
    for d in range(distinct):
        ud, vd, wd = comps(d)
        S.sem_qcriterion_batch(ctx, meshes, ud, vd, wd, [p["Q"] for p in parts])
        for f in range(2):
            tot = 0
            for k, p in enumerate(parts):
                tot += sum(S.sem_isosurface_multi(ctx, p["m"], p["Q"] if f == 0 else ud[k], isos[f], None))
            need[f] = max(need[f], tot)
    cap = [int(n * 1.02) + 4096 for n in need]
    tris = [torch.empty(c * 9, device="cuda") for c in cap]
    cnt = [torch.zeros(16 * 4 + 1, dtype=torch.int64, device="cuda") for _ in range(2)]
    frames = torch.empty((snapshots, 2, 4, 1024 * 1024 * 4), dtype=torch.uint8, device="cuda")
    cam = si.box_camera_persp((0.0,) * 3, (2 * math.pi,) * 3, 1024, 1024)
    colours = [[0.9, 0.35, 0.25], [0.25, 0.6, 0.9], [0.35, 0.85, 0.4], [0.95, 0.8, 0.25]] * 16
    masks = [sum(1 << (4 * k + q) for k in range(16)) for q in range(4)]

    def snapshot(s):
        ud, vd, wd = comps(s % distinct)
        S.sem_qcriterion_batch(ctx, meshes, ud, vd, wd, [p["Q"] for p in parts])
        for f in range(2):
            for k, p in enumerate(parts):
                fld = p["Q"] if f == 0 else ud[k]
                fn = S.sem_isosurface_multi_async if k == 0 else S.sem_isosurface_multi_append_async
                fn(ctx, p["m"], fld, isos[f], tris[f], cnt[f][4 * k:4 * k + 5], cap=cap[f])
            for q in range(4):
                S.sem_render_segments_async(ctx, tris[f], cap[f], cnt[f], 64, colours, masks[q], cam, 1024, 1024,
                                            frames[s, f, q], None)

    def step():
        for s in range(snapshots):
            snapshot(s)

    def plain():
        for s in range(snapshots):
            snapshot(s)
            S.sem_synchronize(ctx)

    stream = torch.cuda.current_stream()
    step()  # first call of each shape: scratch sized, launch widths tuned
    S.sem_synchronize(ctx)
    t0 = time.perf_counter()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(ctx, torch.cuda.current_stream())
        step()
    S.sem_set_stream(ctx, stream)
    g.replay()  # instantiation
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t0

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    ms_graph = timed(g.replay, steps)
    S.sem_synchronize(ctx)  # capacity or timeout flags raised inside the graph
    ms_plain = timed(plain, 1)
    # per-kernel device time of one snapshot, from the library's trace of its eager calls
    S.sem_trace_enable(ctx, True)
    S.sem_trace_collect(ctx)
    snapshot(0)
    S.sem_synchronize(ctx)
    per_snapshot = {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in S.sem_trace_collect(ctx).items()}
    S.sem_trace_enable(ctx, False)
    covered = float((frames[:, :, :, 3::4] > 0).float().mean())
    out = {"workload": f"{snapshots} snapshots x 16 partitions (E_p ~ U{{4096..40960}}, N_p in {{5,7,9}}, "
                       f"{E_total} elements, {nodes} nodes per snapshot) of the Taylor-Green field with 1e-3 noise; "
                       "Q and u isosurfaces at {0.05,0.1,0.2,0.4} of their maxima; one 1024x1024 frame per "
                       "snapshot, field and isovalue (512 per graph); one CUDA graph per time step",
           "snapshots": snapshots, "distinct_resident_snapshots": distinct,
           "resident_velocity_bytes": int(12 * nodes * distinct), "elements_per_snapshot": E_total,
           "orders": [p["N"] for p in parts], "partition_elements": [p["E"] for p in parts],
           "frames_per_graph": snapshots * 8, "graph_nodes_approx": None,
           "graph_ms": round(ms_graph, 3), "graph_frames_per_s": round(snapshots * 8 / (ms_graph * 1e-3), 1),
           "graph_elements_per_s": round(snapshots * E_total / (ms_graph * 1e-3), 1),
           "plain_ms": round(ms_plain, 3), "plain_frames_per_s": round(snapshots * 8 / (ms_plain * 1e-3), 1),
           "plain_elements_per_s": round(snapshots * E_total / (ms_plain * 1e-3), 1),
           "graph_speedup_vs_plain": round(ms_plain / ms_graph, 3),
           "max_triangles_per_snapshot": need, "frame_coverage": round(covered, 4),
           "setup_s": {"generate": round(gen_s, 1), "capture_and_instantiate": round(capture_s, 2)},
           "kernels_per_snapshot": per_snapshot,
           "autotune_widths": S.sem_autotune_width_choices(ctx)}
    del g, frames, tris
    for p in parts:
        S.sem_mesh_free(p["m"])
    parts.clear()
    torch.cuda.empty_cache()
    return out


def _peaks():
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(pp)) if os.path.exists(pp) else {}


def time_workload(S, P, K, warmup, local, barrier, use_graph=True):
    """Per-stage and per-kernel times from K eager traced steps, then the headline: K steps
    replayed as one CUDA graph each, between a barrier + synchronize on both sides, with the
    clocks sampled during the timed region."""
    import numpy as np
    import torch
    for _ in range(warmup):
        P.step_async()
    S.sem_synchronize(P.ctx)
    # the graph's calls, eager, with the library's per-launch trace and stage events
    stage_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    barrier()
    S.sem_trace_enable(P.ctx, True)
    for k in range(K):
        P.step_async(events=stage_ev[k])
    barrier()
    trace = S.sem_trace_collect(P.ctx)
    S.sem_trace_enable(P.ctx, False)
    S.sem_synchronize(P.ctx)
    P.last_ntri = int(P.counts_dev[-1])
    P.covered = int((P.rgba.view(-1, 4)[:, 3] > 0).sum())
    stage_ms = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(3)] for e in stage_ev])
    if use_graph:
        P.capture()
        for _ in range(warmup):
            P.graph.replay()
    run_step = P.graph.replay if use_graph else P.step
    clocks = Clocks(local)
    barrier()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(P.stream)
    for _ in range(K):
        run_step()
    t1.record(P.stream)
    barrier()
    clk = clocks.stop()
    P.S.sem_synchronize(P.ctx)  # raises if a capacity or timeout flag was set in the graph
    secs = max_over_ranks(t0.elapsed_time(t1) / 1e3, "cuda")
    total_elems = sum_over_ranks(P.E * K, "cuda")
    mean_stage = stage_ms.mean(axis=0)
    return {"value": aggregate([total_elems], [secs]), "secs": secs, "trace": trace, "clocks": clk,
            "stage_ms": {"frame_call": round(float(mean_stage[2]), 4),
                         "eager_step": round(float(stage_ms.sum(axis=1).mean()), 4)}}


def kernel_table(P, trace, K, hbm_peak, workload):
    """Per-kernel CUDA-event times (library trace) with algorithmic bytes and the fraction of
    the HBM peak, and the roofline object of the dominant kernel."""
    kernels = {}
    for name, (tot_ms, n) in trace.items():
        per_step = algorithmic_bytes_per_step(name, P)
        ent = {"ms_per_step": round(tot_ms / K, 5), "launches_per_step": n / K}
        if per_step is not None and n:
            per_launch = per_step * K / n
            gbs = per_launch / (tot_ms / n * 1e-3) / 1e9
            ent.update({"algorithmic_bytes_per_launch": int(per_launch), "achieved_gbs": round(gbs, 1),
                        "frac": round(gbs / hbm_peak, 4)})
        kernels[name] = ent
    dom = max(trace, key=lambda k: trace[k][0])
    dom_ms = trace[dom][0] / trace[dom][1]
    per_step = algorithmic_bytes_per_step(dom, P)
    dom_bytes = per_step * K / trace[dom][1] if per_step is not None else None
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_bytes else None
    return kernels, {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1) if achieved else None,
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4) if achieved else None,
                     "traffic": _traffic_for(dom, workload),
                     "algorithmic_bytes_per_launch": int(dom_bytes) if dom_bytes else None,
                     "launch_ms": round(dom_ms, 5)}


def measure_e2e(P, K, warmup, barrier):
    """End to end through the C ABI: every step's inputs (velocity, and temperature where the
    workload has it) from pinned host memory and its frame (RGBA + depth) back to pinned host
    memory, pipelined over two device slots: while step k computes (graph replay), a copy stream
    brings step k+1's inputs in and another reads step k-1's frame back."""
    import torch
    host_in = [v.cpu().pin_memory() for v in P.inputs]
    host_img = torch.empty(P.rgba.numel(), dtype=torch.uint8).pin_memory()
    host_dep = torch.empty(P.depth.numel(), dtype=torch.float32).pin_memory()
    slots = [(P.inputs, P.rgba, P.depth),
             ([v.clone() for v in P.inputs], torch.empty_like(P.rgba), torch.empty_like(P.depth))]
    runs = [P.graph.replay, P.capture_with(*slots[1]).replay]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in, ev_done, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
    issued = [False, False]

    def e2e_step(k):
        sl = k % 2
        ins, rgba, dep = slots[sl]
        with torch.cuda.stream(h2d):
            if issued[sl]:
                h2d.wait_event(ev_out[sl])  # the slot's previous frame has been read back
            for d, h in zip(ins, host_in):
                d.copy_(h, non_blocking=True)
            ev_in[sl].record(h2d)
        P.stream.wait_event(ev_in[sl])
        runs[sl]()
        ev_done[sl].record(P.stream)
        with torch.cuda.stream(d2h):
            d2h.wait_event(ev_done[sl])
            host_img.copy_(rgba, non_blocking=True)
            host_dep.copy_(dep, non_blocking=True)
            ev_out[sl].record(d2h)
        issued[sl] = True

    for k in range(max(2, warmup // 2)):
        e2e_step(k)
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(h2d)
    for k in range(K):
        e2e_step(k)
    b.record(d2h)
    barrier()
    es = max_over_ranks(a.elapsed_time(b) / 1e3, "cuda")
    h2d_bytes = int(sum(h.numel() * 4 for h in host_in))
    # the host link's ceiling: the same copy-in alone, back to back on the copy stream
    for _ in range(2):
        a.record(h2d)
        for _ in range(3):
            for d, h in zip(slots[1][0], host_in):
                d.copy_(h, non_blocking=True)
        b.record(h2d)
        b.synchronize()
    link = 3 * h2d_bytes / (a.elapsed_time(b) / 1e3) / 1e9
    step_gbs = h2d_bytes / (es / K) / 1e9
    total_elems = sum_over_ranks(P.E * K, "cuda")
    P.S.sem_synchronize(P.ctx)
    del slots
    return {"value": aggregate([total_elems], [es]), "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
            "d2h_bytes_per_step": int(host_img.numel() + host_dep.numel() * 4), "ms_per_step": es * 1e3 / K,
            "h2d_gbs": round(step_gbs, 1), "h2d_link_gbs": round(link, 1), "frac_of_link": round(step_gbs / link, 3),
            "pipelining": "two device slots; copy-in of step k+1 and read-back of step k-1 overlap step k"}


def run_ours(args):
    import torch
    import paper_2312_09888_gb300 as S

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    S.get_lib()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    peaks = _peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    K = args.steps
    w = make_workload(args.workload, "cuda")
    mesh_cpu = w.mesh
    camera = w.camera
    P = Pipeline(S, w, local, autotune=not args.no_autotune)
    del w
    head = time_workload(S, P, K, args.warmup, local, barrier, use_graph=not args.no_graph)
    kernels, roof = kernel_table(P, head["trace"], K, hbm_peak, args.workload)
    roof["peak_source"] = peak_src
    launches_per_step = sum(n for _, n in head["trace"].values()) / K
    e2e = None
    if not args.no_e2e and not args.no_graph:
        e2e = measure_e2e(P, K, args.warmup, barrier)

    qprec = None
    if args.q_precisions:
        # sem_qcriterion alone at each arithmetic (CUDA events, 20 launches after 3 warm-up)
        qprec = {}
        for name in ("FP32", "BF16", "FP16", "BF16X2", "TF32"):
            prec = getattr(S, "SEM_" + name)
            for _ in range(3):
                S.sem_qcriterion(P.ctx, P.mesh, *P.inputs[:3], P.Q, prec)
            qa, qb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            qa.record(P.stream)
            for _ in range(20):
                S.sem_qcriterion(P.ctx, P.mesh, *P.inputs[:3], P.Q, prec)
            qb.record(P.stream)
            torch.cuda.synchronize()
            us = qa.elapsed_time(qb) / 20 * 1e3
            qprec[name] = {"us": round(us, 2), "gbs": round(16 * P.npts / (us * 1e-6) / 1e9, 1)}
        S.sem_qcriterion(P.ctx, P.mesh, *P.inputs[:3], P.Q)

    mem_now, mem_peak = S.sem_memory(P.ctx)
    torch_peak = int(torch.cuda.max_memory_allocated())  # the caller's buffers (torch allocator)
    emit_units = [c for c in S.sem_autotune_emit_choices(P.ctx) if c[:2] == (P.N, P.E)]
    widths = S.sem_autotune_width_choices(P.ctx)
    surfaces = P.surface_stats
    W, H, ntri, npts, E, N = P.W, P.H, int(P.last_ntri), P.npts, P.E, P.N
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mesh_cpu, P, camera, budget_s=args.cpu_seconds)
    # the headline's buffers are released before the secondary measurements
    P.sess.close()
    del P
    torch.cuda.empty_cache()

    extra = {}
    if not args.no_extra and args.workload != "channel32":
        w2 = make_workload("channel32", "cuda")
        P2 = Pipeline(S, w2, local)
        del w2
        r2 = time_workload(S, P2, K, args.warmup, local, barrier, use_graph=not args.no_graph)
        k2, roof2 = kernel_table(P2, r2["trace"], K, hbm_peak, "channel32")
        extra["channel32"] = {"workload": WORKLOADS["channel32"], "value": round(r2["value"], 1), "unit": UNIT,
                              "ms_per_step": round(r2["secs"] * 1e3 / K, 4),
                              "frames_per_s": round(K * world / r2["secs"], 2), "triangles": int(P2.last_ntri),
                              "stage_ms": r2["stage_ms"], "kernels": k2, "roofline": roof2, "clocks": r2["clocks"]}
        if args.curved:
            extra["channel32"]["curved"] = measure_curved(S, P2.ctx, P2.inputs[:3], P2.mesh)
        P2.sess.close()
        del P2
        torch.cuda.empty_cache()

    ctx2 = S.sem_create(local, torch.cuda.current_stream())
    try:
        batched = None if args.no_batched else measure_batched(S, ctx2, snapshots=args.batched_snapshots)
        learned = None
        if not args.no_learned:
            bpk = peaks.get("bf16_tflops")
            learned = measure_learned(S, ctx2, bpk or 1900.0, "measured" if bpk else "fallback")
    finally:
        S.sem_destroy(ctx2)

    value, secs = head["value"], head["secs"]
    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": round(secs * 1e3 / K, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "frames_per_s": round(K * world / secs, 2),
           "config": {"workload": WORKLOADS[args.workload], "elements": E, "order": N, "nodes": npts,
                      "surfaces": surfaces, "image": [W, H], "triangles": ntri,
                      "l2": f"inputs {sum(4 * npts for _ in range(3 + (len(surfaces) > 1))) / 1e9:.2f} GB "
                            "> 129 MB L2 (no flush)",
                      "parallelism": f"replicas x{world}"},
           "step_mode": "eager" if args.no_graph else "cuda_graph",
           "stage_ms": head["stage_ms"], "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": head["clocks"],
           "kernels": kernels, "gpu_launches": int(round(launches_per_step * K)),
           "memory": {"library_bytes_in_use": mem_now, "library_bytes_peak": mem_peak,
                      "caller_buffers_bytes_peak": torch_peak},
           "autotune": {"emit_units_per_atomic": sorted({c[3] for c in emit_units}) or None,
                        "launch_widths": [{"kind": k, "N": n, "size": sz, "width": wd, "ms": round(ms, 4)}
                                          for k, n, sz, wd, ms in widths]},
           "extra": extra or None, "learned": learned}
    if qprec is not None:
        out["q_precisions"] = qprec
    if batched is not None:
        out["batched"] = batched
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------ CPU oracle

def _slab(mesh, inputs, e0, nelem):
    """Host FP64 copies of elements [e0, e0 + nelem): node coordinates and the FP32 inputs the
    GPU reads (velocity, and temperature where present), promoted exactly."""
    import torch
    idx = torch.arange(e0, e0 + nelem, device=inputs[0].device)
    return mesh.xyz_range(e0, e0 + nelem), [t.view(-1, (mesh.N + 1) ** 3)[idx].double().cpu().numpy()
                                            for t in inputs]


def _oracle_step(oracle, N, xyz, fields, surfaces, colours, cam):
    """One step of the oracle on a slab: Q from the velocity, every surface's isosurfaces, and
    one full-size frame of the slab's triangles."""
    import numpy as np
    Q = oracle.qcriterion(N, xyz, np.stack(fields[:3]))
    tris, seg = [], []
    for src, isos in surfaces:
        f = Q if src == "Q" else fields[src]
        for iso in isos:
            r = oracle.isosurface(N, xyz, f, iso)
            tris.append(r["tris"])
            seg.append(r["ntri"])
    allt = np.concatenate(tris) if tris else np.zeros((0, 3, 3))
    oracle.render(allt, seg, colours[:len(seg)], cam)


_PALETTE = [[0.9, 0.35, 0.25], [0.25, 0.6, 0.9], [0.35, 0.85, 0.4]]


def _oracle_run(slabs, N, surfaces, colours, cam, threads, budget_s=None, reps=None):
    """Runs the oracle step on every slab, one slab per thread, repeated until `budget_s` seconds
    (or `reps` times); the ctypes calls release the GIL, so the threads run on separate host
    cores.  Returns (elements processed, seconds)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle

    def worker(slab):
        xyz, fields = slab
        done, t0 = 0, time.perf_counter()
        while True:
            _oracle_step(oracle, N, xyz, fields, surfaces, colours, cam)
            done += xyz.shape[1]
            if (reps is not None and done >= reps * xyz.shape[1]) or \
                    (budget_s is not None and time.perf_counter() - t0 >= budget_s):
                return done

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        done = sum(ex.map(worker, slabs[:threads]))
    return done, time.perf_counter() - t0


def cpu_baseline(mesh, P, cam, budget_s=15.0):
    """Times the FP64 oracle on slabs of 1/64 of the elements (contiguous, spread over the mesh) of
    the same workload -- Q, every isosurface, and a full-size frame of the slab's triangles --
    once on one thread and once with one thread per host core, each for about `budget_s`
    seconds; elements/s = elements processed / wall seconds."""
    import oracle
    oracle.lib()
    cores = os.cpu_count() or 1
    nelem = max(64, P.E // 64)
    colours = P.colours or _PALETTE
    starts = [(t * (P.E // cores)) // nelem * nelem for t in range(cores)]
    slabs = [_slab(mesh, P.inputs, min(e0, P.E - nelem), nelem) for e0 in starts]
    _oracle_step(oracle, P.N, *slabs[0], P.surfaces, colours, cam)  # builds the oracle's case table once
    d1, s1 = _oracle_run(slabs, P.N, P.surfaces, colours, cam, 1, budget_s=budget_s)
    dn, sn = _oracle_run(slabs, P.N, P.surfaces, colours, cam, cores, budget_s=budget_s)
    what = (f"slabs of {nelem} contiguous elements (1/64 of the mesh) of the workload: Q + "
            f"{sum(len(i) for _, i in P.surfaces)} isosurfaces + a {P.W}x{P.H} frame of the slab's triangles")
    single = {"value": round(d1 / s1, 2), "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"{what}; one thread, {d1 // nelem} slab steps in {s1:.1f} s"}
    return {"value": round(dn / sn, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}; one thread per core on {cores} cores (nproc), each on its own slab, "
                      f"{dn // nelem} slab steps in {sn:.1f} s",
            "single_thread": single}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on all host cores (one thread per
    core, each on its own slab of the workload); each step is one slab per thread."""
    import numpy as np
    import torch
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.lib()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    w = make_workload(args.workload, dev)
    N, E = w.mesh.N, w.E
    inputs = [w.fields[c].float().contiguous() for c in range(w.fields.shape[0])]
    cam, mesh, fracs, extra = w.camera, w.mesh, w.iso_fracs, dict(w.extra)
    del w
    cores = os.cpu_count() or 1
    nelem = args.ref_elements if args.ref_elements else max(64, E // 64)
    starts = [(t * (E // cores)) // nelem * nelem for t in range(cores)]
    slabs = [_slab(mesh, inputs, min(e0, E - nelem), nelem) for e0 in starts]
    del inputs
    # isovalues from the oracle's own Q on the first slab (the full field's max would need the
    # oracle on every element)
    Q0 = oracle.qcriterion(N, slabs[0][0], np.stack(slabs[0][1][:3]))
    surfaces = [("Q", [float(np.float32(f * Q0.max())) for f in fracs])]
    if "t_iso" in extra:
        surfaces.append((3, [float(np.float32(extra["t_iso"]))]))
    colours = RB_COLOURS if len(surfaces) > 1 else _PALETTE
    _oracle_step(oracle, N, *slabs[0], surfaces, colours, cam)  # builds the oracle's case table once
    if args.warmup:
        _oracle_run(slabs, N, surfaces, colours, cam, cores, reps=args.warmup)
    done, el = _oracle_run(slabs, N, surfaces, colours, cam, cores, reps=args.steps)
    value = done / el
    sample = (f"each step: one slab of {nelem} contiguous elements per thread, {cores} threads on {cores} cores "
              f"(nproc), slabs spread over the mesh (Q + {sum(len(i) for _, i in surfaces)} isosurfaces + "
              f"a {cam['W']}x{cam['H']} frame of the slab's triangles); Q isovalue from the first slab's max Q")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload]},
           "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS),
                    help="rb64: the 64^3-element two-field 3840x2160 workload (headline); channel32: 32^3 channel")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager steps instead of the captured graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary 32^3 channel measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the autoencoder measurement")
    ap.add_argument("--curved", action="store_true",
                    help="also time sem_qcriterion on a general (curved) 32^3 mesh (extra.channel32.curved)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batching workload (64 snapshots x 16 partitions x 2 fields x 4 isovalues per graph)")
    ap.add_argument("--batched-snapshots", type=int, default=64)
    ap.add_argument("--q-precisions", action="store_true",
                    help="also time sem_qcriterion at FP32, BF16, FP16, split BF16 and TF32 (q_precisions)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="library defaults instead of the autotuner's choices (for profiling captures)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-elements", type=int, default=0,
                    help="reference arm: elements per slab (default 1/64 of the mesh)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
