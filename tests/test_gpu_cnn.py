"""The learned warm start on the GPU: forward and gradients against the FP64
reference network, GPU training, and what the trained network gains."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as orc  # noqa: E402
from paper_1601_03801_gb300 import sedi  # noqa: E402
from paper_1601_03801_gb300.workloads import small_case  # noqa: E402


def init_params(seed, last_zero=False):
    """He-style initialisation in the packed parameter order."""
    rng = np.random.default_rng(seed)
    p = []
    for li, (ci, co) in enumerate([(4, 32), (32, 32), (32, 4)]):
        std = np.sqrt(2.0 / (27 * ci))
        w = rng.normal(0, std, co * ci * 27)
        if last_zero and li == 2:
            w[:] = 0.0
        p += [w, np.zeros(co)]
    return np.concatenate(p)


@pytest.fixture(scope="module")
def small():
    return small_case(parity_addon=True)


def test_forward_matches_reference(small):
    prm, _ = small
    g = sedi.Sedi(dict(prm, precision_form="split"))
    p = init_params(1)
    g.cnn_set_params(p)
    C = int(np.prod(prm["ncell"]))
    x = np.random.default_rng(2).normal(0, 1, (4, C))
    y = g.cnn_forward(x)
    ref = orc.cnn_forward(p, x, prm["ncell"], prm["periodic"], round_bf16=True)
    scale = np.abs(ref).max()
    # bf16 storage at the same points; FP32 vs FP64 accumulation may flip a rounding
    assert np.abs(y - ref).max() <= 2e-2 * scale
    assert np.abs(y - ref).mean() <= 1e-3 * scale
    np.testing.assert_array_equal(g.cnn_get_params(), p.astype(np.float32).astype(np.float64))


def test_gradient_matches_reference(small):
    prm, _ = small
    g = sedi.Sedi(dict(prm, precision_form="split"))
    p = init_params(3)
    g.cnn_set_params(p)
    C = int(np.prod(prm["ncell"]))
    rng = np.random.default_rng(4)
    x = rng.normal(0, 1, (4, C))
    t = rng.normal(0, 1, (4, C))
    loss, grad = g.cnn_loss_grad(x, t)
    loss_ref, grad_ref = orc.cnn_loss_grad(p, x, t, prm["ncell"], prm["periodic"])
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    rel = np.linalg.norm(grad - grad_ref) / np.linalg.norm(grad_ref)
    cos = grad @ grad_ref / (np.linalg.norm(grad) * np.linalg.norm(grad_ref))
    assert rel < 5e-2 and cos > 0.998, (rel, cos)
    # every parameter block receives gradient
    for a, b in ((0, 3456), (3456, 3488), (3488, 31136), (31168, 34624), (34624, 34628)):
        assert np.abs(grad[a:b]).max() > 0


def one_step_pairs(prm, parts, snapshots, substeps=40):
    """(phi^m, phi^{m+1}) of (eps, F) for the four pseudo-steps, made by the method
    itself: deposition on the GPU, one backward-Euler pseudo-step per smoothing call
    (n_tau = 1 with half the bandwidth is one step of the 4-step operator)."""
    run = sedi.Sedi(dict(prm, precision_form="split"))
    run.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    one = sedi.Sedi(dict(prm, precision_form="split", n_tau=1,
                         bandwidth=tuple(b / np.sqrt(prm["n_tau"]) for b in prm["bandwidth"])))
    S = [prm["shift_eps"], prm["shift_force"]]
    out = []
    for _ in range(snapshots):
        run.step(substeps)
        q = run.deposit()
        phi = np.stack([np.ldexp(q[0].astype(float), -S[0])] +
                       [np.ldexp(q[4 + a].astype(float), -S[1]) for a in range(3)])
        for _m in range(prm["n_tau"]):
            nxt, _ = one.smooth(phi)
            out.append((phi, nxt))
            phi = nxt
    return out, run


def test_training_cuts_smoother_iterations(small):
    prm, parts = small
    pairs, run = one_step_pairs(prm, parts, snapshots=6)
    x0 = np.stack([p[0] for p in pairs])
    scale = np.maximum(np.abs(x0).max(axis=(0, 2)), 1e-30)
    xs = np.stack([p[0] / scale[:, None] for p in pairs])
    ts = np.stack([(p[1] - p[0]) / scale[:, None] for p in pairs])
    trainer = sedi.Sedi(dict(prm, precision_form="split"))
    trainer.cnn_set_params(init_params(5, last_zero=True))
    losses = trainer.cnn_train(xs[:-4], ts[:-4], steps=400, lr=2e-3)
    assert losses[-20:].mean() < 0.2 * losses[:5].mean(), (losses[:5], losses[-20:])
    params = trainer.cnn_get_params()
    # held-out snapshot: same state, smoothing from phi^m vs from the learned guess
    x, v, w, _ = run.get_particles()
    res = []
    for warm in (0, 1):
        h = sedi.Sedi(dict(prm, precision_form="split", use_cnn_guess=warm, cnn_scale=tuple(scale)))
        h.set_particles(x, v, w, parts["d"], parts["rho"])
        h.cnn_set_params(params)
        it0 = h.stats()["cg_iterations"]
        eps, Us, F = h.average()
        res.append((h.stats()["cg_iterations"] - it0, eps, F))
    (it_cold, e0, f0), (it_warm, e1, f1) = res
    assert it_warm < it_cold, (it_cold, it_warm)
    # the solve still meets the tolerance: results agree to the smoothing tolerance
    assert np.abs(e1 - e0).max() <= 1e-7 * np.abs(e0).max()
    assert np.abs(f1 - f0).max() <= 1e-7 * np.abs(f0).max()
