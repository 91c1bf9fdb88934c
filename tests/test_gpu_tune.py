"""Autotuner of the tensor-core band kernel (TCORR_TUNE) on the GPU."""
import json

import numpy as np
import pytest

import oracle
from paper_1708_08619_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_1708_08619_gb300 import build, tcorr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    tcorr.load()
    return tcorr


def test_tuner_times_candidates_once_and_persists(T, tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("TCORR_TUNE", "1")
    monkeypatch.setenv("TCORR_TUNE_CACHE", str(cache))
    x = synth.random_walk_positions(1500, 700, 0.01, 3.0, seed=31)
    xd = torch.from_numpy(x).cuda()
    m1 = T.tcorr_msd(xd, 500, 1, "fp16x3").cpu().numpy()
    lines = [json.loads(l) for l in cache.read_text().splitlines() if l.strip()]
    assert len(lines) == 1 and lines[0]["key"].startswith("m4.k0.")
    # the work-item length and the supertile of the claim order are tuned; sub_kb 0 keeps
    # the accuracy-chosen default
    assert lines[0]["kseg"] in (4096, 8192, 16384) and lines[0]["sub_kb"] == 0
    assert (lines[0]["super_rows"], lines[0]["super_cols"]) in ((16, 10), (32, 5), (8, 19))
    assert lines[0]["pair"] in (0, 1)               # the tile shape: one CTA or a CTA pair
    m2 = T.tcorr_msd(xd, 500, 1, "fp16x3").cpu().numpy()
    assert np.array_equal(m1, m2)                    # same tuned choice, no second tuning
    assert len(cache.read_text().splitlines()) == 1
    parity.check_tc_msd(m1, oracle.msd(x, 500, 1), what="tuned fp16x3 msd")
    assert T.tcorr_status_poll() == 0


def test_every_supertile_shape_gives_the_same_sums(T, monkeypatch):
    """The claim order only changes which CTA runs an item: the windows land at
    their canonical index and the lag reduction sums them in a fixed order, so
    the results are bit-identical for every supertile shape (edge cases: one
    tile at a time, whole rows, shapes that do not divide the grid)."""
    x = torch.from_numpy(synth.random_walk_positions(3000, 400, 0.01, 3.0, seed=33)).cuda()
    ref = {}
    for shape in ("16x10", "1x1", "1x4096", "4096x1", "7x3", "32x5"):
        monkeypatch.setenv("TCORR_SUPER", shape)
        for s in (1, 3):
            m = T.tcorr_msd(x, 1500, s, "fp16x3").cpu().numpy()
            ref.setdefault(s, m)
            assert np.array_equal(m, ref[s]), (shape, s)
    assert T.tcorr_status_poll() == 0


_CHILD = """
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1708_08619_gb300 import build, synth, tcorr
build.build(); tcorr.load()
x = torch.from_numpy(synth.random_walk_positions(1200, 300, 0.01, 3.0, seed=34)).cuda()
m = tcorr.tcorr_msd(x, 400, 1, "fp16x3").cpu().numpy()
print(float(m[-1]))
"""


def test_cache_lines_without_a_supertile_are_read(T, tmp_path):
    """A cache line written before the supertile was tuned (kseg and sub_kb only)
    is read at the first lookup of a fresh process and used: no tuning run
    follows, so nothing is appended to the file."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = _CHILD.format(root=root)
    new = tmp_path / "new.jsonl"
    env = dict(os.environ, TCORR_TUNE="1", TCORR_TUNE_CACHE=str(new))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    key = json.loads(new.read_text().splitlines()[0])["key"]
    old = tmp_path / "old.jsonl"
    old.write_text(json.dumps({"key": key, "kseg": 4096, "sub_kb": 0}) + "\n")
    env["TCORR_TUNE_CACHE"] = str(old)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert len(old.read_text().splitlines()) == 1          # the old line was used, no re-tuning
    assert np.isfinite(float(r.stdout.strip().splitlines()[-1]))


_CHILD_SHA = """
import sys, hashlib, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1708_08619_gb300 import build, synth, tcorr
build.build(); tcorr.load()
x = torch.from_numpy(synth.random_walk_positions(1200, 300, 0.01, 3.0, seed=34)).cuda()
m = tcorr.tcorr_msd(x, 400, 1, "fp16x3").cpu().numpy()
print(hashlib.sha256(m.tobytes()).hexdigest())
"""


def test_cached_tile_shape_selects_the_kernel(T, tmp_path):
    """A cache line that chooses the CTA-pair tile shape runs the pair kernel:
    its result is bit for bit that of TCORR_PAIR=1 with the same work-item
    length and supertile, and differs in rounding from the one-CTA tiling."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = _CHILD_SHA.format(root=root)

    def run(env_extra):
        env = dict(os.environ, **env_extra)
        for k in ("TCORR_PAIR", "TCORR_TUNE", "TCORR_TUNE_CACHE", "TCORR_KSEG", "TCORR_SUPER"):
            if k not in env_extra:
                env.pop(k, None)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return r.stdout.strip().splitlines()[-1]

    probe = tmp_path / "probe.jsonl"
    run({"TCORR_TUNE": "1", "TCORR_TUNE_CACHE": str(probe)})
    key = json.loads(probe.read_text().splitlines()[0])["key"]
    sha = {}
    for pair in (0, 1):
        cache = tmp_path / f"pair{pair}.jsonl"
        cache.write_text(json.dumps({"key": key, "kseg": 4096, "sub_kb": 0, "super_rows": 16, "super_cols": 10,
                                     "pair": pair}) + "\n")
        sha[pair] = run({"TCORR_TUNE": "1", "TCORR_TUNE_CACHE": str(cache)})
        assert len(cache.read_text().splitlines()) == 1      # the line was used, no re-tuning
    forced = run({"TCORR_PAIR": "1", "TCORR_KSEG": "4096", "TCORR_SUPER": "16x10"})
    assert sha[1] == forced
    assert sha[0] != sha[1]
