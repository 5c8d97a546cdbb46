"""The warm-start network's CUDA kernels against the FP64 reference
(oracle/net.py) on the same parameters and inputs, and the learned warm
start against the flat start, judged by DM.

Bounds: forward output relative L2 <= 1e-5 and parameter gradient relative
L2 <= 1e-4 (FP32 accumulation against FP64, with the same BF16-rounded
weights on both sides)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def test_forward_and_gradients_match_the_reference():
    import torch
    from oracle import net as onet
    from paper_1808_10375_gb300 import dm
    from synth import warmstart as ws
    net = dm.dm_net_create(max_batch=4, seed=5)
    rng = np.random.default_rng(6)
    p = (onet.he_params(rng) + 0.01 * rng.standard_normal(onet.param_count())).astype(np.float32)
    assert dm.dm_net_param_count(net) == p.size
    dm.dm_net_set_params(net, p)
    assert np.array_equal(dm.dm_net_get_params(net), p)
    x, t = ws.pairs(2, 7)
    y = dm.dm_net_forward(net, x)
    acts = onet.forward(p.astype(np.float64), x.cpu().numpy().astype(np.float64))
    err_y = _rel(y.cpu().numpy(), acts[-1])
    g, loss = dm.dm_net_gradients(net, x, t)
    ref_loss, ref_g = onet.loss_and_gradients(p.astype(np.float64), x.cpu().numpy().astype(np.float64),
                                              t.cpu().numpy().astype(np.float64))
    err_g = _rel(g, ref_g)
    print(f"forward rel L2 {err_y:.2e}, gradient rel L2 {err_g:.2e}, loss {loss:.6g} vs {ref_loss:.6g}")
    assert err_y <= 1e-5
    assert err_g <= 1e-4
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    dm.dm_net_free(net)


def test_gauge_loss_and_gradients_match_the_reference():
    """The phase-gauge-invariant loss through the network against the FP64
    reference; turning every target patch by its own constant phase leaves
    the loss unchanged."""
    import torch
    from oracle import net as onet
    from paper_1808_10375_gb300 import dm
    from synth import warmstart as ws
    net = dm.dm_net_create(max_batch=4, seed=5)
    dm.dm_net_set_loss(net, dm.DM_NET_LOSS_GAUGE)
    rng = np.random.default_rng(8)
    p = (onet.he_params(rng) + 0.01 * rng.standard_normal(onet.param_count())).astype(np.float32)
    dm.dm_net_set_params(net, p)
    x, t = ws.pairs(3, 9)
    g, loss = dm.dm_net_gradients(net, x, t)
    ref_loss, ref_g = onet.loss_and_gradients(p.astype(np.float64), x.cpu().numpy().astype(np.float64),
                                              t.cpu().numpy().astype(np.float64), loss="gauge")
    err_g = _rel(g, ref_g)
    print(f"gauge loss {loss:.6g} vs {ref_loss:.6g}, gradient rel L2 {err_g:.2e}")
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert err_g <= 1e-4
    t2 = t.clone()
    t2[:, 1] += torch.tensor([0.4, -2.0, 3.1], device=t.device)[:, None, None]
    _, loss2 = dm.dm_net_gradients(net, x, t2)
    assert abs(loss2 - loss) <= 1e-5 * loss
    with pytest.raises(dm.DMError):
        dm.dm_net_set_loss(net, 7)
    dm.dm_net_free(net)


def test_dm_refined_pairs():
    """One simulated 4-mode scan: every view gives an input frame, a target
    patch of the object after 20 DM iterations and the true patch; the
    refined targets are much closer to the truth (after the best phase per
    patch) than the flat object is."""
    import torch
    from paper_1808_10375_gb300 import warmstart
    x, t, g = warmstart.refined_pairs(1, 4242, dm_iters=20)
    assert x.shape == (2500, 1, 128, 128) and t.shape == (2500, 2, 64, 64) and g.shape == t.shape
    assert torch.isfinite(x).all() and torch.isfinite(t).all()
    flat = torch.zeros_like(g)
    flat[:, 0] = 1.0
    err_dm = warmstart.fit_of(t, g)["complex_rel_err_gauge_aligned"]
    err_flat = warmstart.fit_of(flat, g)["complex_rel_err_gauge_aligned"]
    print("DM-refined target error", err_dm, "flat", err_flat)
    assert err_dm < 0.5 * err_flat


def test_warm_start_is_trained_and_judged_by_dm():
    """The network trains on simulated pairs with the library's kernels, its
    stitched start is judged by DM's own Fourier error (the start with the
    lower error after the trial iterations is kept), and DM converges from
    both starts.  On these random-field objects the network gains nothing:
    its start error is the flat start's, and the trial's Fourier errors
    differ by a few per cent, so the judge's pick does not predict which
    start ends lower after 60 iterations.  The test records the comparison
    and checks the mechanism, not a gain."""
    from paper_1808_10375_gb300 import dm, warmstart
    from synth import make_scan
    from synth import warmstart as ws
    net = dm.dm_net_create(max_batch=64, seed=11)
    losses = warmstart.train(net, steps=1500, batch=64, lr=1e-3, seed=12, data_count=20000)
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1][1] < 0.5 * losses[0][1]
    cfg = dict(n=128, modes=4, grid=(12, 12), step=10, jitter=1, obj=(250, 250), probe="hg", fwhm=ws.FWHM,
               photons=ws.PHOTONS, seed=13)
    scan = make_scan(cfg, noise=False)
    o_warm = warmstart.predict_start(net, scan.intensities, scan.pos, scan.obj_shape)
    o0, pick, ef = warmstart.judged_start(scan, scan.probe, o_warm, trial_iters=10)
    res = warmstart.compare(scan, scan.probe, o_warm, iters=60)
    for name in ("flat", "warm"):
        e = dict(res[name]["errors"])
        print(name, "start error", round(e[0], 4), "after 20 / 60 iterations", round(e[20], 4), round(e[60], 4))
    print("judge:", pick, ef)
    assert pick == min(ef, key=ef.get)
    assert np.array_equal(o0, o_warm.detach().cpu().numpy().astype(np.complex64) if pick == "warm"
                          else np.ones(scan.obj_shape, np.complex64))
    for name in ("flat", "warm"):
        e = dict(res[name]["errors"])
        assert e[60] <= 0.25 * e[0], (name, e[0], e[60])
    dm.dm_net_free(net)


def test_training_is_reproducible():
    """Two networks from the same seed, trained with the gauge-invariant loss
    on the same seeded batches (gathered by torch right before each call, as
    warmstart.train does), end
    with bit-identical parameters: every network kernel is deterministic, and
    each call waits for its inputs and finishes before returning."""
    from paper_1808_10375_gb300 import dm, warmstart
    params = []
    for _ in range(2):
        net = dm.dm_net_create(max_batch=32, seed=3)
        dm.dm_net_set_loss(net, dm.DM_NET_LOSS_GAUGE)
        warmstart.train(net, steps=40, batch=32, lr=1e-3, seed=4, data_count=512)
        params.append(dm.dm_net_get_params(net))
        dm.dm_net_free(net)
    assert np.array_equal(params[0], params[1])
