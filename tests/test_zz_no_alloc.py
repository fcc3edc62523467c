"""lbm_totals_noalloc: the global sums of lbm_totals for callers that cannot
call cudaMalloc (an application whose device memory all belongs to its own
pool allocator, or monitoring code that must stay out of the CUDA allocator
while a time-stepping loop runs).  It needs no context and allocates nothing:
its work space is a fixed array inside the library.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _entry():
    import paper_1608_04658_gb300 as lbm
    fn = lbm.lib().lbm_totals_noalloc
    fn.argtypes = [C.POINTER(lbm.Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return lbm, fn


def _call(fn, lat, out, flags=True):
    import ctypes as C
    return fn(C.byref(lat.params), C.c_void_p(lat.f.data_ptr()),
              C.c_void_p(lat.flags.data_ptr()) if flags else None,
              C.c_void_p(out.data_ptr()), C.c_void_p(lat.stream.cuda_stream))


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
def test_noalloc_totals_match_the_context_totals(storage):
    """Two calls in a row (the shared work space keeps the previous call's
    partials) each equal lbm_totals on the same state, up to the addition
    order of FP64 sums."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm, fn = _entry()
    shape = (40, 36, 52)
    rho, u, xi = synth.parity_fields(shape, 9)
    lat = lbm.Lattice(shape, 0.03, storage=storage, faces=(1, 1, 1, 1, 0, 0))
    lat.set_geometry(lbm.sphere((19.3, 17.6, 25.2), 6.1, U=(0.0, 0.0, -0.02), free=True, g=(0.0, 0.0, -1e-4)))
    lat.init_state(rho, 0.3 * u, xi, 1e-3)
    out = torch.zeros(5, dtype=torch.float64, device=lat.device)
    for _ in range(2):
        lat.step(3)
        ref = lat.totals()
        assert _call(fn, lat, out) == 0
        lat.stream.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * ref[0])


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_noalloc_totals_on_a_large_bodiless_box(storage):
    """128^3 nodes give 128 block partials, so each lane of the final sum adds
    four of them; no body, so the call takes no flags (NULL) and the context
    sums every node too.  Two calls in a row, a step between them."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm, fn = _entry()
    shape = (128, 128, 128)
    wl = synth.tgv_periodic(128)
    rho, u = synth.taylor_green_fields(wl["shape"], wl["u0"])
    lat = lbm.Lattice(shape, wl["nu"], storage=storage)
    lat.init_state(rho, u)
    out = torch.zeros(5, dtype=torch.float64, device=lat.device)
    for _ in range(2):
        lat.step(1)
        ref = lat.totals()
        assert _call(fn, lat, out, flags=False) == 0
        lat.stream.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * ref[0])


def test_noalloc_rejects_buffers_not_on_the_current_device():
    """Host memory for the populations or the output is refused before
    anything is enqueued."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm, fn = _entry()
    shape = (8, 8, 8)
    lat = lbm.Lattice(shape, 0.05, storage="fp32")
    lat.init_state(*synth.uniform_fields(shape))
    host_f = np.zeros(27 * 8 * 8 * 8, dtype=np.float32)
    host_out = np.zeros(5)
    dev_out = torch.zeros(5, dtype=torch.float64, device=lat.device)
    assert fn(C.byref(lat.params), C.c_void_p(host_f.ctypes.data), None, C.c_void_p(dev_out.data_ptr()),
              C.c_void_p(lat.stream.cuda_stream)) == 1  # LBM_ERR_ARG
    assert fn(C.byref(lat.params), C.c_void_p(lat.f.data_ptr()), None, C.c_void_p(host_out.ctypes.data),
              C.c_void_p(lat.stream.cuda_stream)) == 1
    # a correct call afterwards still works
    assert _call(fn, lat, dev_out, flags=False) == 0
    lat.stream.synchronize()
    assert np.allclose(dev_out.cpu().numpy(), lat.totals(), rtol=1e-12, atol=1e-12 * 512)


def test_noalloc_rejects_lattices_beyond_its_work_space():
    lbm, fn = _entry()
    p = lbm.make_params((512, 512, 260), 0.1)  # 68,157,440 nodes > 67,108,864
    dummy = C.c_void_p(256)
    assert fn(C.byref(p), dummy, None, dummy, None) == 1  # LBM_ERR_ARG
    p = lbm.make_params((40, 36, 52), 0.1)
    assert fn(C.byref(p), None, None, dummy, None) == 1
