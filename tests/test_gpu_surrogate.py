"""MLP surrogate with contour fallback: training runs, the weights file is
checked, and every output (surrogate or fallback) agrees with the CPU oracle
within 1e-4 on positions near caustics that the oracle itself placed; on
GPU-sampled positions the surrogate path agrees with pure contour integration
(all queries forced to fall back)."""
import os
import shutil

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2501_03322_gb300 as P  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-4


@pytest.fixture(scope="module")
def trained(tmp_path_factory):
    path = tmp_path_factory.mktemp("sur") / "weights.bin"
    stats = P.surrogate_train(path, nsamples=1 << 18, seed=11, epochs=3)
    return path, stats


def test_training_statistics(trained):
    path, st = trained
    assert os.path.getsize(path) > 4 * 199000
    assert st["drawn"] == 1 << 18 and 4096 <= st["rows"] <= st["labelled"] <= st["drawn"]
    assert np.isfinite(st["loss"]) and st["target_std"] > 0


def test_corrupted_weights_rejected(trained, tmp_path):
    path, _ = trained
    bad = tmp_path / "bad.bin"
    shutil.copy(path, bad)
    with open(bad, "r+b") as f:
        f.seek(100)
        b = f.read(1)
        f.seek(100)
        f.write(bytes([b[0] ^ 0xFF]))
    x = np.array([0.1])
    with pytest.raises(P.TwError):
        P.surrogate_mag(bad, x * 0 + 1.0, x * 0 + 1e-3, x * 0 + 1e-3, x, x)


def test_surrogate_with_fallback_matches_oracle(trained):
    path, _ = trained
    rows = [ln.split() for ln in open(os.path.join(GOLD, "surrogate_queries.txt")) if not ln.startswith("#")]
    a = np.array([[float(v) for v in r[:6]] for r in rows])
    ok = np.array([int(r[6]) == 0 for r in rows])
    for prec in (P.PREC_FP64, P.PREC_MIXED):
        out, nf = P.surrogate_mag(path, a[:, 0], a[:, 1], a[:, 2], a[:, 3], a[:, 4], rel_tol=TOL, precision=prec)
        assert 0 <= nf <= len(rows)
        err = np.abs(out[ok] / a[ok, 5] - 1)
        assert err.max() <= TOL, (err.max(), nf)


def test_surrogate_matches_pure_contour_on_sampled_queries(trained):
    path, _ = trained
    q = P.surrogate_sample(seed=7, n=1 << 20)
    out, cnt = P.surrogate_mag(path, *q, rel_tol=TOL, details=True)
    ref = P.mag_multi(*q, rel_tol=TOL)  # plain contour integration of every query
    torch.cuda.synchronize()
    assert cnt["fallback"] + cnt["network"] + cnt["expansion"] == 1 << 20
    r = (out / ref - 1).abs()
    i = int(torch.argmax(torch.nan_to_num(r, nan=1e30)).item())
    worst = [float(t[i]) for t in q] + [float(out[i]), float(ref[i])]
    assert torch.isfinite(out).all() and r.max().item() <= 2 * TOL, (r.max().item(), cnt, worst)
