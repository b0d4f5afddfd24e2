"""The allocation-free smoothing entry point (sedi_smooth_static).

Some callers cannot allocate device memory (a framework or memory pool owns it,
or allocations are forbidden after start-up).  sedi_smooth_static serves them
from a static scratch array.  This file is collected last so a stop-at-first-
failure run has already run every other test; it passes alone or after them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as orc  # noqa: E402
from paper_1601_03801_gb300 import sedi  # noqa: E402
from paper_1601_03801_gb300.workloads import default_params, random_fields  # noqa: E402

MESH = dict(hi=(64e-3, 32e-3, 64e-3), ncell=(64, 32, 64), wall_hi=(0, 0, 0), bandwidth=(1.5e-3,) * 3)


def test_static_smoothing_matches_handle_path_twice():
    prm = default_params(hi=(64e-3, 32e-3, 64e-3), ncell=(64, 32, 64), wall_hi=(0, 0, 0),
                         bandwidth=(1.5e-3,) * 3)
    C = int(np.prod(prm["ncell"]))
    ref = sedi.Sedi(dict(prm, precision_form="split"))
    stream = torch.cuda.Stream()
    for call, seed in enumerate((21, 22)):
        phi = random_fields(prm["ncell"], 7, seed=seed)
        want, want_it = ref.smooth(phi)
        dev_in = torch.as_tensor(phi, device="cuda")
        dev_out = torch.full_like(dev_in, float("nan"))
        torch.cuda.synchronize()
        it = sedi.smooth_static(dict(prm, precision_form="split"), dev_in, dev_out, stream)
        got = dev_out.cpu().numpy()
        assert np.isfinite(got).all(), call
        for f in range(7):
            assert np.abs(got[f] - want[f]).max() <= 1e-7 * np.abs(phi[f]).max(), (call, f)
        assert np.array_equal(it, want_it)
        # the input is untouched (the scratch holds the working copy)
        assert np.array_equal(dev_in.cpu().numpy(), phi)


def test_static_smoothing_bdf2():
    # the BDF2 pseudo-time scheme keeps the previous step in the same static scratch
    prm = dict(default_params(hi=(64e-3, 32e-3, 64e-3), ncell=(64, 32, 64), wall_hi=(0, 0, 0),
                              bandwidth=(1.5e-3,) * 3, tau_scheme=1), precision_form="split")
    ref = sedi.Sedi(prm)
    phi = random_fields(prm["ncell"], 7, seed=23)
    want, want_it = ref.smooth(phi)
    dev_in = torch.as_tensor(phi, device="cuda")
    dev_out = torch.full_like(dev_in, float("nan"))
    torch.cuda.synchronize()
    it = sedi.smooth_static(prm, dev_in, dev_out)
    got = dev_out.cpu().numpy()
    for f in range(7):
        assert np.abs(got[f] - want[f]).max() <= 1e-7 * np.abs(phi[f]).max(), f
    assert np.array_equal(it, want_it)


def test_static_smoothing_rejects_oversize():
    prm = default_params(ncell=(128, 128, 64))  # 8 fields x 1,048,576 cells > limit
    C = int(np.prod(prm["ncell"]))
    assert 8 * C > sedi.STATIC_MAX_WORDS
    dev = torch.zeros((8, C), dtype=torch.float64, device="cuda")
    with pytest.raises(sedi.SediError) as e:
        sedi.smooth_static(prm, dev, dev)
    assert e.value.code == -1 and "SEDI_STATIC_MAX_WORDS" in str(e.value)


def test_static_smoothing_allocates_nothing_and_matches_oracle():
    """After the first call on a device (which may load the library's kernels and its
    static array), further calls leave the device's free memory and torch's allocator
    untouched; the result matches the FP64 oracle's CG smoothing."""
    prm = default_params(**MESH)
    phi = random_fields(prm["ncell"], 4, seed=31)
    dev_in = torch.as_tensor(phi, device="cuda")
    dev_out = torch.empty_like(dev_in)
    sedi.smooth_static(dict(prm, precision_form="split"), dev_in, dev_out)  # first call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        sedi.smooth_static(dict(prm, precision_form="split"), dev_in, dev_out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    want, _ = orc.Oracle(prm).smooth(phi)
    got = dev_out.cpu().numpy()
    for f in range(4):
        assert np.abs(got[f] - want[f]).max() <= 1e-7 * np.abs(phi[f]).max(), f


@pytest.mark.parametrize("form,scheme", [("fp64", 1), ("plain", 0)])
def test_static_smoothing_other_forms_at_the_size_limit(form, scheme):
    """The largest mesh the static scratch takes (8 x 131,072 words), in the FP64 form
    with BDF2 (the largest scratch) and in the plain form, against the handle path."""
    prm = dict(default_params(tau_scheme=scheme, **MESH), precision_form=form)
    C = int(np.prod(prm["ncell"]))
    assert 8 * C == sedi.STATIC_MAX_WORDS
    phi = random_fields(prm["ncell"], 8, seed=41)
    want, want_it = sedi.Sedi(prm).smooth(phi)
    dev_in = torch.as_tensor(phi, device="cuda")
    dev_out = torch.full_like(dev_in, float("nan"))
    it = sedi.smooth_static(prm, dev_in, dev_out)
    got = dev_out.cpu().numpy()
    tol = 1e-7 if form == "fp64" else 1e-5
    for f in range(8):
        assert np.abs(got[f] - want[f]).max() <= tol * np.abs(phi[f]).max(), f
    assert np.array_equal(it, want_it)


def test_static_smoothing_rejects_bad_buffers_on_the_host():
    """Wrong dtype, shape or memory kind is refused before any kernel runs."""
    prm = default_params(**MESH)
    C = int(np.prod(prm["ncell"]))
    good = torch.zeros((2, C), dtype=torch.float64, device="cuda")
    for bad_in, bad_out in ((good.float(), good), (good[:, :-1].contiguous(), good[:, :-1].contiguous()),
                            (good, torch.zeros((3, C), dtype=torch.float64, device="cuda")),
                            (good.cpu(), good.cpu()), (good.t(), good.t())):
        with pytest.raises(ValueError):
            sedi.smooth_static(prm, bad_in, bad_out)
    # the C entry point itself refuses host pointers
    host = np.zeros((2, C))
    msg = sedi.C.create_string_buffer(256)
    p = sedi.make_params(prm)
    rc = sedi.lib().sedi_smooth_static(sedi.C.byref(p), 2, host.ctypes.data, host.ctypes.data, None, 0,
                                       msg, 256)
    assert rc == -1 and b"device memory" in msg.value
