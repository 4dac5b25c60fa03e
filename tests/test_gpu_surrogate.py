"""MLP surrogate with contour fallback: training runs, the weights file is
checked, and every output (surrogate or fallback) agrees with the CPU oracle
within 1e-4 on positions near caustics that the oracle itself placed; on
GPU-sampled positions the surrogate path agrees with pure contour integration
(all queries forced to fall back).  The network trained as the benchmark
trains it answers queries of its band, and every query it answers agrees with
the oracle within 1e-4."""
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
    stats = P.surrogate_train(path, nsamples=1 << 20, seed=11, epochs=3)
    return path, stats


@pytest.fixture(scope="module")
def trained_full(tmp_path_factory):
    """The benchmark's network: 1e7 draws (seed 0), 30 epochs."""
    path = tmp_path_factory.mktemp("sur_full") / "weights.bin"
    stats = P.surrogate_train(path, nsamples=10_000_000, seed=0, epochs=30)
    return path, stats


def load_queries(name):
    rows = [ln.split() for ln in open(os.path.join(GOLD, name)) if not ln.startswith("#") and ln.strip()]
    a = np.array([[float(v) for v in r[:6]] for r in rows])
    ok = np.array([int(r[6]) == 0 for r in rows])
    return a, ok


def test_training_statistics(trained):
    path, st = trained
    assert os.path.getsize(path) > 4 * 199000
    assert st["drawn"] == 1 << 20 and 4096 <= st["rows"] <= st["labelled"] <= st["drawn"]
    assert np.isfinite(st["loss"]) and st["target_std"] > 0
    assert 128 <= st["heldout"] and st["kappa_cal"] >= 3.0


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


def test_surrogate_matches_pure_contour_on_sampled_queries(trained_full):
    path, _ = trained_full
    q = P.surrogate_sample(seed=7, n=1 << 20)
    out, cnt = P.surrogate_mag(path, *q, rel_tol=TOL, details=True)
    ref = P.mag_multi(*q, rel_tol=TOL)  # plain contour integration of every query
    torch.cuda.synchronize()
    assert cnt["fallback"] + cnt["network"] + cnt["expansion"] == 1 << 20
    r = (out / ref - 1).abs()
    i = int(torch.argmax(torch.nan_to_num(r, nan=1e30)).item())
    worst = [float(t[i]) for t in q] + [float(out[i]), float(ref[i])]
    assert torch.isfinite(out).all() and r.max().item() <= 2 * TOL, (r.max().item(), cnt, worst)


def test_network_answers_within_tolerance_of_oracle(trained_full):
    """Oracle-placed queries near caustics and a few radii off them: the
    network answers some of them (TW_POS_NETWORK), and each of those, like
    every other output, is within 1e-4 of the oracle, in both precisions."""
    path, st = trained_full
    assert st["kappa_cal"] >= 3.0 and st["heldout_accepted"] > 0.1
    assert st["heldout_accepted_max_err"] <= 0.25 * TOL
    a1, ok1 = load_queries("surrogate_queries.txt")
    a2, ok2 = load_queries("surrogate_band.txt")
    a, ok = np.r_[a1, a2], np.r_[ok1, ok2]
    for prec in (P.PREC_FP64, P.PREC_MIXED):
        stat = np.zeros(len(a), np.int8)
        out, cnt = P.surrogate_mag(path, a[:, 0], a[:, 1], a[:, 2], a[:, 3], a[:, 4], rel_tol=TOL, precision=prec,
                                   details=True, status=stat)
        net = stat == P.POS_NETWORK
        assert cnt["network"] == int(net.sum()) >= 32, cnt
        assert cnt["expansion"] == int((stat == P.POS_EXPANSION).sum())
        err = np.abs(out / a[:, 5] - 1)
        assert err[net & ok].max() <= TOL, err[net & ok].max()
        assert err[ok].max() <= TOL, err[ok].max()


def test_network_answers_match_tight_contour_on_sampled_queries(trained_full):
    """2^20 GPU-sampled queries (device arrays, status on the device): every
    network answer against FP64 contour integration at rel_tol 1e-7."""
    path, _ = trained_full
    q = P.surrogate_sample(seed=7, n=1 << 20)
    stat = torch.zeros(1 << 20, dtype=torch.int8, device="cuda")
    out, cnt = P.surrogate_mag(path, *q, rel_tol=TOL, precision=P.PREC_MIXED, details=True, status=stat)
    idx = torch.nonzero(stat == P.POS_NETWORK).flatten()
    assert idx.numel() == cnt["network"] > 1000, cnt
    sub = [t[idx].contiguous() for t in q]
    ref = P.mag_multi(*sub, rel_tol=1e-7, precision=P.PREC_FP64)
    r = (out[idx] / ref - 1).abs()
    assert r.max().item() <= TOL, r.max().item()


def test_full_size_launch_with_oracle_queries(trained_full):
    """The benchmark's workload at full size: 10^7 queries of its stream
    (seed 1) in one call, with the oracle-placed golden queries written
    over its first entries; those outputs against the oracle, every output
    finite, the counts adding up."""
    path, _ = trained_full
    n = 10_000_000
    q = P.surrogate_sample(1, n)
    a1, ok1 = load_queries("surrogate_queries.txt")
    a2, ok2 = load_queries("surrogate_band.txt")
    a, ok = np.r_[a1, a2], np.r_[ok1, ok2]
    m = len(a)
    for k in range(5):
        q[k][:m] = torch.as_tensor(a[:, k], device="cuda")
    out, cnt = P.surrogate_mag(path, *q, rel_tol=TOL, precision=P.PREC_MIXED, details=True)
    assert cnt["fallback"] + cnt["network"] + cnt["expansion"] == n
    assert bool(torch.isfinite(out).all())
    got = out[:m].cpu().numpy()
    err = np.abs(got[ok] / a[ok, 5] - 1)
    assert err.max() <= TOL, err.max()
