"""Host side of the Gauss-Newton checkpoint (save_gn_checkpoint / load_gn_checkpoint):
a round trip restores m, the fields and the step records exactly; a file of another kind or
of other shapes is refused before anything is overwritten; the write replaces the file
whole (no temporary file is left behind)."""
import os

import pytest
import torch

from paper_2209_02815_gb300 import h1w


def _state(seed=0):
    g = torch.Generator().manual_seed(seed)
    m = torch.randn(60, dtype=torch.float64, generator=g)
    U = torch.randn(4, 60, dtype=torch.float64, generator=g)
    hist = []
    for i in range(3):
        h = h1w.GnInfo()
        h.fwd_iters, h.gn_iters, h.misfit, h.rel_res_true, h.step_norm = 10 - i, 5 + i, 1.0 / (i + 1), 1e-9, 0.5 ** i
        hist.append(h)
    return m, U, hist


def test_round_trip(tmp_path):
    m, U, hist = _state()
    p = str(tmp_path / "gn.pt")
    h1w.save_gn_checkpoint(p, 3, m, U, hist)
    assert os.listdir(tmp_path) == ["gn.pt"]
    m2, U2 = torch.zeros_like(m), torch.zeros_like(U)
    step, hist2 = h1w.load_gn_checkpoint(p, m2, U2)
    assert step == 3 and torch.equal(m2, m) and torch.equal(U2, U)
    for a, b in zip(hist, hist2):
        for f, _ in h1w.GnInfo._fields_:
            assert getattr(a, f) == getattr(b, f)


def test_overwrite_keeps_latest(tmp_path):
    p = str(tmp_path / "gn.pt")
    m, U, hist = _state(0)
    h1w.save_gn_checkpoint(p, 1, m, U, hist[:1])
    m1, U1, hist1 = _state(1)
    h1w.save_gn_checkpoint(p, 2, m1, U1, hist1[:2])
    m2, U2 = torch.zeros_like(m), torch.zeros_like(U)
    step, h = h1w.load_gn_checkpoint(p, m2, U2)
    assert step == 2 and len(h) == 2 and torch.equal(m2, m1) and torch.equal(U2, U1)


def test_refuses_other_files_and_shapes(tmp_path):
    m, U, hist = _state()
    p = str(tmp_path / "gn.pt")
    h1w.save_gn_checkpoint(p, 1, m, U, hist)
    m_bad = torch.zeros(61, dtype=torch.float64)
    U_keep = torch.full_like(U, 7.0)
    with pytest.raises(ValueError, match="shapes"):
        h1w.load_gn_checkpoint(p, m_bad, U_keep)
    assert float(U_keep.min()) == 7.0                      # nothing was copied
    q = str(tmp_path / "other.pt")
    torch.save({"step": 1, "m": m, "U": U, "hist": []}, q)
    with pytest.raises(ValueError, match="not an h1w"):
        h1w.load_gn_checkpoint(q, torch.zeros_like(m), torch.zeros_like(U))
