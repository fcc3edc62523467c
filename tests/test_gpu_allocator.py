"""The caller's device allocator (lbm_set_allocator): the library's scratch
taken from PyTorch's caching allocator gives the same bits as cudaMalloc'd
scratch, the blocks go back when the context lets them go, a refused
allocation is LBM_ERR_OOM, and the allocator cannot change under live
scratch.  Also lbm_init_equilibrium against lbm_init_state without noise."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_04658_gb300 as lbm
    lbm.build()
    lbm.lib()


def _counting_torch_allocator(lat):
    import torch
    dev = lat.device.index
    live = {}

    def alloc(n, stream):
        p = torch.cuda.caching_allocator_alloc(n, dev, stream)
        live[p] = n
        return p

    def release(p, stream):
        del live[p]
        torch.cuda.caching_allocator_delete(p)
    lat.use_allocator(alloc, release)
    return live


def _sphere_run(storage, torch_alloc):
    import paper_1608_04658_gb300 as lbm
    shape = (24, 20, 22)
    rho, u, xi = synth.parity_fields(shape, 4)
    lat = lbm.Lattice(shape, 0.02, storage=storage, faces=(1, 1, 1, 1, 0, 0))
    live = _counting_torch_allocator(lat) if torch_alloc else None
    lat.set_geometry(lbm.sphere((11.37, 9.61, 10.83), 4.3, U=(0.02, -0.01, 0.03), free=True, g=(0, 0, -1e-4)))
    lat.init_state(rho, 0.3 * u, xi, 1e-3)
    lat.step(8)
    F, M = lat.forces()
    J = lat.adjoint(6, w_force=(1.0, 0.0, 0.0))
    return lat, live, lat.populations(), F, J


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_torch_allocator_gives_the_same_bits(storage):
    lat0, _, f0, F0, J0 = _sphere_run(storage, False)
    lat1, live, f1, F1, J1 = _sphere_run(storage, True)
    assert np.array_equal(f0, f1)
    assert np.array_equal(F0, F1)
    # the adjoint's sums over the body's band slots take double atomics in
    # whatever order the warps reach them, so its last bits may vary
    assert J1["J"] == pytest.approx(J0["J"], rel=1e-9)
    assert np.allclose(J1["dJ_dtheta"], J0["dJ_dtheta"], rtol=1e-8, atol=1e-14)
    # the body's scratch is held; the adjoint's blocks were handed back
    assert len(live) > 0
    held = dict(live)
    lat1.close()
    assert len(live) == 0 and len(held) > 0
    lat0.close()


def test_allocator_refusal_and_state_rules():
    import paper_1608_04658_gb300 as lbm
    from paper_1608_04658_gb300 import binding
    lat = lbm.Lattice((24, 20, 22), 0.02, storage="fp32", faces=(1, 1, 1, 1, 0, 0))
    lat.use_allocator(lambda n, s: None, lambda p, s: None)
    with pytest.raises(lbm.LbmError) as e:
        lat.set_geometry(lbm.sphere((11.37, 9.61, 10.83), 4.3))
    assert e.value.status == binding.LBM_ERR_OOM
    # the context stays usable without a body
    lat.init_state(*synth.uniform_fields((24, 20, 22)))
    lat.step(2)
    # back to cudaMalloc, then a body: the allocator cannot change under it
    lat.use_torch_allocator()
    lat.set_geometry(lbm.sphere((11.37, 9.61, 10.83), 4.3))
    with pytest.raises(lbm.LbmError) as e:
        lat.use_torch_allocator()
    assert e.value.status == binding.LBM_ERR_STATE
    lat.close()


def test_misaligned_blocks_are_refused():
    """A block that is not 256-byte aligned goes straight back to the caller
    and the call fails with LBM_ERR_OOM, before any kernel could see it."""
    import torch

    import paper_1608_04658_gb300 as lbm
    from paper_1608_04658_gb300 import binding
    lat = lbm.Lattice((24, 20, 22), 0.02, storage="fp32", faces=(1, 1, 1, 1, 0, 0))
    dev = lat.device.index
    held, returned = [], []

    def alloc(n, stream):
        p = torch.cuda.caching_allocator_alloc(n + 256, dev, stream)
        held.append(p)
        return p + 16

    lat.use_allocator(alloc, lambda p, stream: returned.append(p))
    with pytest.raises(lbm.LbmError) as e:
        lat.set_geometry(lbm.sphere((11.37, 9.61, 10.83), 4.3))
    assert e.value.status == binding.LBM_ERR_OOM
    assert returned == [held[0] + 16]
    for p in held:
        torch.cuda.caching_allocator_delete(p)
    lat.close()


def test_refinement_scratch_from_the_coarse_allocator():
    import paper_1608_04658_gb300 as lbm
    from parity_util import random_fields
    shape, lo, hi = (24, 20, 18), (5, 4, 3), (16, 13, 12)
    out = []
    for torch_alloc in (False, True):
        rho, u, xi, amp = random_fields(shape, 3)
        lat = lbm.Lattice(shape, 0.02, storage="fp32")
        live = _counting_torch_allocator(lat) if torch_alloc else None
        ref = lbm.Refinement(lat, lo, hi)
        if torch_alloc:
            assert len(live) == 4  # t, t+1 and the half step's moments, the skipped box
        frho, fu, fxi, famp = random_fields(ref.fine.shape, 103)
        lat.init_state(rho, u, xi, amp)
        ref.fine.init_state(frho, fu, fxi, famp)
        ref.init()
        ref.step(3)
        out.append((lat.populations(), ref.fine.populations()))
        n = len(live) if torch_alloc else 0
        ref.close()
        if torch_alloc:
            assert len(live) == n - 4  # (the coarse plane buffer of populations() stays)
        ref.fine.close()
        lat.close()
    # the nodes the refined step defines (the block's deep inside and the fine
    # pad hold whatever their buffers held)
    vc = np.ones(out[0][0].shape[1:], dtype=bool)
    vc[lo[2] + 2:hi[2] - 1, lo[1] + 2:hi[1] - 1, lo[0] + 2:hi[0] - 1] = False
    assert np.array_equal(out[0][0][:, vc], out[1][0][:, vc])
    assert np.array_equal(out[0][1][:, :-1, :-1, :-1], out[1][1][:, :-1, :-1, :-1])


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_init_equilibrium_matches_init_state_without_noise(storage):
    import paper_1608_04658_gb300 as lbm
    shape = (16, 12, 10)
    rho, u, _ = synth.parity_fields(shape, 7)
    a = lbm.Lattice(shape, 0.02, storage=storage)
    b = lbm.Lattice(shape, 0.02, storage=storage)
    a.init_equilibrium(rho, u)
    b.init_state(rho, u)
    assert np.array_equal(a.populations(), b.populations())
