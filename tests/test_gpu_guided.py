"""The surrogate-guided scan end to end at a small scale: what the trained
network gains over the plain Monte Carlo method without it.

On a 128 x 128 grid of (F, b) of the dichotomous model (400 averaged periods),
the guided map -- network predictions where the calibrated rule trusts them,
Monte Carlo re-runs elsewhere -- must reproduce plain Monte Carlo at a random
sample of grid points within |d<v>| <= 0.01, while spending fewer path-steps
(labels and re-runs together) than the plain map of the grid.
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_guided_scan_small_grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import guided
    r = guided.guided_dichot_scan(nx=128, ny=128, n_label=4096, label_paths=2048, rerun_paths=4096,
                                  transient=20, periods=400, n_valid=1024, steps=6000,
                                  log=lambda *a: None)
    assert r["validation_frac_within_0.01"] >= 0.995, r
    assert r["validation_max_abs_err"] <= 0.02, r
    assert r["flagged_fraction"] < 0.3, r
    assert r["ratio_plain_over_guided_total"] > 2.0, r


def test_box_surrogate_pipeline_small():
    """The Poisson-box surrogate end to end at a small size: labels from one
    scan, two networks trained on the device, held-out error below the label
    spread, timed inference."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import box_surrogate
    r = box_surrogate.run(n_label=2048, paths=256, steps=1500, n_infer=1 << 14, log=lambda *a: None)
    assert r["labels"] == 2048 + 256 and r["heldout"] == 256
    assert r["heldout_v_rmse"] < r["label_v_std"], r
    assert r["inference_points_per_s"] > 0
    # the guided screen of the 64 x 64 scan: flagged points are re-run exactly
    # (the plain map's own values there), so the guided map can only differ
    # where the calibrated rule trusted the network
    s = r["screen_scan_64x64"]
    assert s["grid"] == [64, 64] and 0 <= s["flagged"] <= 4096
    assert s["path_steps_reruns"] <= s["path_steps_plain_map"]
    if s["flagged"] == 4096:
        assert s["max_abs_err"] == 0.0



def test_poisson_slice_screen():
    """The 64 x 64 Poisson scan screened by networks of its (F, log Q) slice,
    at a small size: every grid point within 0.01 of the plain map (all 4096
    are compared), at fewer path-steps than the plain map, labels included."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import box_surrogate
    r = box_surrogate.slice_screen_64x64(n_label=512, n_hold=256, steps=3000)
    assert r["frac_within_0.01"] == 1.0, r
    assert r["ratio_plain_over_guided_total"] > 1.0, r


def test_concurrent_training_equals_sequential():
    """The guided scans train their two networks from two host threads at once;
    each network's parameters must be those of training it alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np
    from paper_1409_4923_gb300 import guided
    rng = np.random.default_rng(3)
    N = 4096
    X = np.stack([rng.uniform(0.5, 1.5, N), rng.uniform(2, 6, N), rng.uniform(3, 7, N), rng.uniform(-0.3, 0.3, N),
                  10.0 ** rng.uniform(-4, -1, N), rng.uniform(0.1, 5, N), rng.uniform(0.01, 0.5, N)], axis=1)
    T = np.stack([np.sin(3 * X[:, 3]) * X[:, 0], -3.0 + 0.1 * X[:, 1]], axis=1)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    shift, scale = guided.box_maps(X.min(0), X.max(0), 1 << 4)
    params = []
    for concurrent in (True, False):
        nets, hists = guided.train_ensemble(Xd, Td, shift, scale, 1 << 4, steps=300, batch=256,
                                            concurrent=concurrent)
        params.append([n.get_params() for n in nets])
        for n in nets:
            n.close()
    for a, b in zip(*params):
        assert np.array_equal(a, b)
