"""The benchmark on the CPU: its reference arm (the FP64 oracle on the host)
prints one JSON line with the contract's keys, bounded in wall time whatever
--steps asks for; its roofline bookkeeping (algorithmic bytes, and ncu
traffic only for the kernel source it was captured on) holds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                       capture_output=True, text=True, timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line_and_time_bound():
    d = run_bench("--impl", "reference", "--steps", "100000", "--warmup", "50",
                  "--ref-seconds", "1.5")
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["higher_is_better"] is True and d["unit"] == "iters/s"
    assert 1 <= d["steps"] < 100000 and d["requested_steps"] == 100000 and d["warmup"] <= 3
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0 and not [l for l in r.stdout.splitlines() if l.startswith("{")]


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_match_the_committed_record():
    """Per-launch algorithmic bytes of the two iteration kernels at 256x256
    (m 66 060 rays, d 65 536 pixels, 15 017 956 nonzeros): the A or A^T
    stream at 6 B per nonzero in the sliced, packed layout (8 B for FP32
    values and 4-byte columns), its offsets, and each vector once, as the
    ncu record states."""
    b = _bench_module()
    m, d, nnz = 66060, 65536, 15017956
    fwd, pix = b.kernel_bytes(m, d, nnz, 6, True)
    # written out: matrix, offsets (one per slice of 8 rows), f, g, gamma, y_prev, y, w,
    # stencil vectors
    assert fwd == 6 * nnz + 4 * (m // 8 + 1) + 4 * d + (4 + 4 + 8 + 8 + 4) * m + 12 * d
    assert pix == 6 * nnz + 4 * (d // 8 + 1) + 4 * m + 20 * d
    assert b.kernel_bytes(m, d, nnz)[1] == 8 * nnz + 4 * (d + 1) + 4 * m + 20 * d
    # folded by the quarter-turn symmetry: half the stored entries and rows
    ffw, fpx = b.kernel_bytes(m, d, nnz, 6, True, True)
    assert ffw == 6 * (nnz // 2) + 4 * (m // 2 // 8 + 1) + 4 * d + 28 * m + 12 * d
    assert fpx == 6 * (nnz // 2) + 4 * (d // 8 + 1) + 4 * m + 20 * d
    # the record of the committed capture: algorithmic bytes in the plain
    # format, and the bytes its layout streams
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    cfw, cpx = b.kernel_bytes(m, d, nnz)
    for layout, ent in rec["layouts"].items():
        ks = ent["kernels"]
        assert cfw == ks["k_forward"]["algorithmic_bytes_per_launch"]
        assert cpx == ks["k_pixel"]["algorithmic_bytes_per_launch"]
        sfw, spx = b.kernel_bytes(m, d, nnz, rec["bytes_per_nnz"], True, layout == "folded")
        assert sfw == ks["k_forward"]["stored_bytes_per_launch"]
        assert spx == ks["k_pixel"]["stored_bytes_per_launch"]
        # the captured traffic is near the bytes the layout streams
        for k in ("k_forward", "k_pixel"):
            assert 1.0 <= ks[k]["dram_bytes_per_launch"] / ks[k]["stored_bytes_per_launch"] < 1.2
    # both streams dominate: 12 B per nonzero is 97-98 % of an iteration's bytes
    assert 0.97 < 12 * nnz / (fwd + pix) < 0.99
    # a batched iteration of 64 slices reads the matrix once: far below 64 iterations
    kb = b.batched_bytes(66060, 65536, 15017956, 64)
    assert 16 * 15017956 < kb < 3 * (fwd + pix)


def test_traffic_is_reported_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    """ncu traffic is attached to the roofline only while the loop kernels'
    sources are those the capture was taken on (their SHA-256 is in the
    record)."""
    import hashlib
    b = _bench_module()
    src = tmp_path / "paper_2409_13344_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    files = {name: f"// {name}\n".encode() for name in b.KERNEL_SOURCES}
    for name, code in files.items():
        (src / name).write_bytes(code)
    sha = hashlib.sha256(b"".join(files[n] for n in b.KERNEL_SOURCES)).hexdigest()
    rec = {"kernel_sources_sha256": sha,
           "layouts": {"unfolded": {"kernels": {"k_pixel": {"dram_bytes_per_launch": 123}}}}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.committed_traffic("k_pixel") == 123
    assert b.committed_traffic("k_pixel", "folded") is None
    assert b.committed_traffic("k_forward") is None
    for name in b.KERNEL_SOURCES:  # a change to any of them drops the figure
        (src / name).write_bytes(files[name] + b"// changed\n")
        assert b.committed_traffic("k_pixel") is None
        (src / name).write_bytes(files[name])
    assert b.committed_traffic("k_pixel") == 123


def test_main_leg_layout_keeps_timed_streams_above_l2():
    """The main single-slice leg folds only when the folded streams still
    exceed L2: at 256x256 (95 MB folded, L2 136 MB) it streams the whole
    matrices (185 MB), at 512x512 the folded halves (about 740 MB)."""
    b = _bench_module()
    l2 = 136314880
    for (m, d, nnz), folds in (((66060, 65536, 15017956), False),
                               ((263160, 262144, 120155712), True)):
        fold_stream = sum(b.kernel_bytes(m, d, nnz, 6, True, True))
        plain_stream = sum(b.kernel_bytes(m, d, nnz, 6, True, False))
        assert plain_stream > l2
        assert b.main_leg_folds("auto", fold_stream, l2) == folds
        streamed = fold_stream if folds else plain_stream
        assert streamed > l2
    assert b.main_leg_folds("on", 1, l2) and not b.main_leg_folds("off", 10 ** 12, l2)
