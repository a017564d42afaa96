"""Precision study (sph_precision_study): the tiered decision is never
wrong; the FP16 / FP32 absolute and FP16 cell-relative wrong-decision counts
equal, as integers, a CPU emulation of the same operation sequence with one
IEEE rounding per step (tests/study_emulation.py); FP16 absolute coordinates
fail first, as Tables 1-2 report (GPU required)."""
import numpy as np
import pytest

import oracle
import study_emulation
from paper_2401_08586_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_08586_gb300 import sph as _sph
    _sph.load()
    return _sph


EXACT = ("candidates", "neighbours", "wrong_fp16_abs", "wrong_fp32_abs", "wrong_fp16_rcll")


def test_table1_circle(sph):
    from paper_2401_08586_gb300 import study
    rows = study.table1(sph, torch)
    for r in rows:
        xyz = W.circle_pairs(1.0, r["dR"], 60, dim=2, seed=0, center=(0.0, 0.0))
        want = study_emulation.counts(xyz, 1.0, 0, 1)
        assert {k: r[k] for k in EXACT} == want, r["dR"]
    w16 = [r["wrong_fp16_abs"] for r in rows]
    w32 = [r["wrong_fp32_abs"] for r in rows]
    for r in rows:
        assert r["candidates"] == 60 and r["wrong_tiered"] == 0
    # with particles at kh (1 +- dR) the rounded distances collapse onto kh as
    # dR shrinks, so about one side (half the set) ends up wrong
    assert w16[0] == 0 and w16[1] == 0 and w16[-1] >= 20
    assert w32[:4] == [0, 0, 0, 0] and w32[-1] >= 10
    assert all(a <= b + 5 for a, b in zip(w16, w16[1:]))  # grows as dR shrinks


def test_table2_random(sph):
    from paper_2401_08586_gb300 import study
    rows = study.table2(sph, torch, ds_list=[0.01, 0.005, 0.002])
    for r in rows:
        assert r["wrong_tiered"] == 0
    for r in rows[:2]:
        xyz = W.random_uniform(r["n"], 2, 1)
        want = study_emulation.counts(xyz, 2 * 1.2 * r["ds"])
        assert {k: r[k] for k in EXACT} == want, r["ds"]
    p16 = [r["pct"]["wrong_fp16_abs"] for r in rows]
    prc = [r["pct"]["wrong_fp16_rcll"] for r in rows]
    assert p16[0] < p16[-1] and p16[-1] > 0.05
    assert prc[-1] < p16[-1]


def test_study_counts_pinned_to_oracle(sph):
    xyz = W.random_uniform(5000, 3, 4)
    kh = 0.08
    g = sph.Grid(torch.from_numpy(xyz).cuda(), kh / 2, kh)
    c = sph.sph_precision_study(g.handle)
    rp, col = oracle.cll(xyz, kh)
    assert c["neighbours"] == col.size and c["wrong_tiered"] == 0
    # candidates: every ordered pair in the 3^3 cells around each particle
    rows = sph.sph_precision_study(g.handle, 10, 20)
    assert rows["neighbours"] == int(rp[20] - rp[10])
    g.close()
