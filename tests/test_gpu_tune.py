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
    # only the work-item length is tuned; sub_kb 0 keeps the accuracy-chosen default
    assert lines[0]["kseg"] in (4096, 8192, 16384) and lines[0]["sub_kb"] == 0
    m2 = T.tcorr_msd(xd, 500, 1, "fp16x3").cpu().numpy()
    assert np.array_equal(m1, m2)                    # same tuned choice, no second tuning
    assert len(cache.read_text().splitlines()) == 1
    parity.check_tc_msd(m1, oracle.msd(x, 500, 1), what="tuned fp16x3 msd")
    assert T.tcorr_status_poll() == 0
