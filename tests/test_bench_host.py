"""bench.py's host-side contract, on the CPU: the reference arm's JSON line (the FP64 oracle
timed on bounded samples of a benchmark workload, one thread per host core) and the source hash
that keeps a counter capture matched to its kernel."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "channel32", "--steps", "1",
                        "--warmup", "0", "--ref-elements", "4"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("channel 32x32x32")
    # one oracle thread per host core, each on its own slab
    assert d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)


def test_source_hash_ignores_comments_only(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(int *x) { x[0] = 1; /* one */ }\n")
    b = tmp_path / "b.cu"
    b.write_text("// another header\n\n__global__ void k(int *x)\n{\n    x[0] = 1;  // one\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("// header\n__global__ void k(int *x) { x[0] = 2; }\n")
    assert bench._file_sha(str(a)) == bench._file_sha(str(b))
    assert bench._file_sha(str(a)) != bench._file_sha(str(c))


def test_byte_model_of_the_frame_in_parts():
    """The algorithmic bytes the bench divides by: a two-field frame drawn in parts reads every
    triangle once over its two raster kernels (Q's part one tile per block, the temperature's
    as a range), and a one-field frame reads them all in the one-tile-per-block kernel."""
    sys.path.insert(0, ROOT)
    import bench
    from types import SimpleNamespace
    surf = [{"field": "Q", "niso": 1, "ntri": 4647976, "active_elems": 47017},
            {"field": "T", "niso": 1, "ntri": 1377188, "active_elems": 13965}]
    two = SimpleNamespace(N=7, E=262144, npts=262144 * 512, surface_stats=surf, last_ntri=6025164, nseg=2,
                          surfaces=[("Q", [0.1]), (3, [0.5])], W=3840, H=2160, covered=1000)
    small, rng = bench.algorithmic_bytes_per_step("k_raster_small", two), bench.algorithmic_bytes_per_step(
        "k_raster_range", two)
    assert small == 36 * 4647976 and rng == 36 * 1377188 and small + rng == 36 * two.last_ntri
    # the fused Q kernel: u, v, w read and Q written (16 B per node) + one count per element
    assert bench.algorithmic_bytes_per_step("k_sem_q8_count", two) == 16 * two.npts + 4 * two.E
    # Q of the other orders (u, v, w in, Q out) and the derivative kernel (u in, three derivatives
    # out) move 16 B per node each
    assert bench.algorithmic_bytes_per_step("k_sem_qd", two) == 16 * two.npts
    assert bench.algorithmic_bytes_per_step("k_sem_grad", two) == 16 * two.npts
    assert bench.KERNEL_SOURCES["k_sem_qd"] == bench.KERNEL_SOURCES["k_sem_q8"]
    one = SimpleNamespace(N=7, E=32768, npts=32768 * 512, surface_stats=surf[:1], last_ntri=4647976, nseg=3,
                          surfaces=[("Q", [0.1, 0.2, 0.3])], W=1920, H=1080, covered=10)
    assert bench.algorithmic_bytes_per_step("k_raster_small", one) == 36 * one.last_ntri
