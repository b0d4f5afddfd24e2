"""Failure detection on the GPU without faulting it: a bounded device wait that runs
out is reported as SEDI_ETIMEOUT and leaves the handle usable, and non-finite input
is reported (SEDI_ENONFINITE from the device, SEDI_EINVAL at the boundary)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1601_03801_gb300 import sedi  # noqa: E402
from paper_1601_03801_gb300.workloads import default_params, random_fields, small_case  # noqa: E402

ETIMEOUT, ENONFINITE, EINVAL = -8, -7, -1


def test_grid_barrier_timeout_is_reported_and_handle_recovers(monkeypatch):
    """A 96 x 96 x 24 mesh is too large for a thread-block cluster, so its smoothing
    runs on the cooperative grid with a bounded grid barrier.  With the barrier's
    poll limit set to 1 the first wait runs out: every block returns, the call
    reports SEDI_ETIMEOUT, and the same handle then steps particles and smooths
    normally once the limit is back (a fresh handle reads the default)."""
    prm = default_params(hi=(96e-3, 96e-3, 24e-3), ncell=(96, 96, 24), wall_hi=(0, 0, 1),
                         bandwidth=(2e-3, 2e-3, 1.5e-3))
    phi = random_fields(prm["ncell"], 2, seed=61)
    monkeypatch.setenv("SEDI_BARRIER_SPIN_LIMIT", "1")
    g = sedi.Sedi(dict(prm, precision_form="split"))
    monkeypatch.delenv("SEDI_BARRIER_SPIN_LIMIT")
    with pytest.raises(sedi.SediError) as e:
        g.smooth(phi)
    assert e.value.code == ETIMEOUT
    # the context and the handle are still usable
    _, parts = small_case()
    n = 200
    x = parts["x"][:n] * np.array([96e-3 / 20e-3, 96e-3 / 20e-3, 24e-3 / 40e-3])
    x[:, 2] = np.clip(x[:, 2], 0.6e-3, 23e-3)
    g.set_particles(x, np.zeros((n, 3)), np.zeros((n, 3)), parts["d"][:n], parts["rho"][:n])
    g.step(10)
    g.sync()
    h = sedi.Sedi(dict(prm, precision_form="split"))
    out, it = h.smooth(phi)
    assert np.isfinite(out).all() and np.all(it > 0)
    assert abs(out[0].sum() / phi[0].sum() - 1) < 1e-9


def test_nonfinite_inputs_are_reported():
    prm, parts = small_case(parity_addon=True)
    # a NaN velocity reaches the forces: the device flags it and the next
    # synchronising call reports it
    v = parts["v"].copy()
    v[17, 2] = np.nan
    g = sedi.Sedi(dict(prm, precision_form="split"))
    g.set_particles(parts["x"], v, parts["w"], parts["d"], parts["rho"])
    g.step(2)
    with pytest.raises(sedi.SediError) as e:
        g.sync()
    assert e.value.code == ENONFINITE
    # a NaN in a prescribed fluid field: the drag of the spheres around that cell
    C = int(np.prod(prm["ncell"]))
    U = np.zeros((C, 3))
    U[C // 3, 0] = np.nan
    g = sedi.Sedi(dict(prm, precision_form="split"))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.set_fluid(U=U)
    g.step(2)
    with pytest.raises(sedi.SediError) as e:
        g.sync()
    assert e.value.code == ENONFINITE
    # a NaN position is refused at the boundary, before any kernel sees it
    x = parts["x"].copy()
    x[3, 0] = np.nan
    g = sedi.Sedi(dict(prm, precision_form="split"))
    with pytest.raises(sedi.SediError) as e:
        g.set_particles(x, parts["v"], parts["w"], parts["d"], parts["rho"])
    assert e.value.code == EINVAL
