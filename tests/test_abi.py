"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point include/lbm.h declares, its structs have the layout the
binding assumes, and argument errors are reported before any CUDA call."""
import ctypes as C
import os
import subprocess
import tempfile

import pytest

import paper_1608_04658_gb300 as lbm
from paper_1608_04658_gb300 import binding


@pytest.fixture(scope="module")
def L():
    lbm.build()
    return lbm.lib()


def test_every_declared_symbol_is_exported(L):
    names = lbm.declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name


def _c_layout(struct, fields):
    src = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{binding.HEADER}"', "int main(void){",
           f'printf("%zu\\n", sizeof({struct}));']
    src += [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src += ["return 0;}"]
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write("\n".join(src))
        subprocess.check_call(["gcc", "-std=c99", "-o", exe, c])
        return [int(v) for v in subprocess.check_output([exe]).split()]


@pytest.mark.parametrize("cls,cname", [(binding.Params, "lbm_params"), (binding.Geometry, "lbm_geometry"),
                                       (binding.BodyState, "lbm_body_state"),
                                       (binding.AdjointSpec, "lbm_adjoint")])
def test_struct_layout_matches_header(cls, cname):
    fields = [f for f, _ in cls._fields_]
    got = _c_layout(cname, fields)
    assert got[0] == C.sizeof(cls)
    for f, off in zip(fields, got[1:]):
        assert getattr(cls, f).offset == off, f


def test_force_record_layout_matches_the_binding():
    """The binding reads force records as rows of RECORD_DOUBLES doubles in a
    ring of RECORD_DEPTH: F at 0..2, M at 3..5, the step time at 6."""
    got = _c_layout("lbm_force_record", ["F", "M", "t", "status", "reserved"])
    assert got == [8 * binding.RECORD_DOUBLES, 0, 24, 48, 56, 60]
    text = open(binding.HEADER).read()
    assert f"#define LBM_RECORD_DEPTH {binding.RECORD_DEPTH}" in text


def test_invalid_arguments_are_rejected_without_a_gpu(L):
    ctx = C.c_void_p()
    dummy = C.c_void_p(16)
    p = lbm.make_params((0, 4, 4), 0.1)
    assert L.lbm_create(C.byref(p), dummy, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    p = lbm.make_params((4, 4, 4), 0.1)
    assert L.lbm_create(C.byref(p), None, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    p = lbm.make_params((4, 4, 4), 0.1, faces=(0, 1, 0, 0, 0, 0))  # periodic on one side only
    assert L.lbm_create(C.byref(p), dummy, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    p = lbm.make_params((4, 4, 4), -1.0)
    assert L.lbm_create(C.byref(p), dummy, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    p = lbm.make_params((4, 4, 4), 0.1)
    p.storage = 9
    assert L.lbm_create(C.byref(p), dummy, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    p = lbm.make_params((4, 4, 4), 0.1)
    assert L.lbm_create(C.byref(p), C.c_void_p(24), dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    assert not ctx.value
    p = lbm.make_params((2048, 2048, 1024), 0.1)  # N >= 2^31
    assert L.lbm_create(C.byref(p), dummy, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    p = lbm.make_params((400, 400, 500), 0.1)  # 27 N = 2.16e9: plane offsets beyond 32 bits
    assert L.lbm_create(C.byref(p), dummy, dummy, dummy, None, C.byref(ctx)) == binding.LBM_ERR_ARG
    assert L.lbm_step(None, 1) == binding.LBM_ERR_ARG
    assert L.lbm_last_error(None) == b"null context"
    # the slab, two-phase step and force hand-over entry points, null context
    d6 = (C.c_double * 6)()
    for rc in (L.lbm_step_interior(None), L.lbm_step_edges(None), L.lbm_set_slab(None, 0, 8, 0, 8),
               L.lbm_pack_layers(None, 0, 1, dummy), L.lbm_unpack_layers(None, 0, 1, dummy),
               L.lbm_body_force_to_device(None, dummy), L.lbm_sum_body_force(None, dummy, 1),
               L.lbm_set_body_force(None, d6, d6), L.lbm_init_state(None, dummy, dummy, None, 0.0),
               L.lbm_init_state_f32(None, dummy, dummy, None, 0.0)):
        assert rc == binding.LBM_ERR_ARG
    # the allocator hook and the equilibrium initialisation, null context
    assert L.lbm_set_allocator(None, binding._ALLOC_FN(), binding._RELEASE_FN(), None) == binding.LBM_ERR_ARG
    assert L.lbm_init_equilibrium(None, dummy, dummy) == binding.LBM_ERR_ARG
    # the refinement entry points, null contexts and handles
    r = C.c_void_p(7)
    i3 = (C.c_int32 * 3)(1, 1, 1)
    assert L.lbm_refine_create(None, None, i3, i3, C.byref(r)) == binding.LBM_ERR_ARG
    assert not r.value
    assert L.lbm_refine_create(dummy, dummy, i3, i3, None) == binding.LBM_ERR_ARG
    assert L.lbm_refine_init(None) == binding.LBM_ERR_ARG
    assert L.lbm_refine_step(None, 1) == binding.LBM_ERR_ARG
    assert L.lbm_refine_save(None, b"x") == binding.LBM_ERR_ARG
    assert L.lbm_refine_load(None, b"x") == binding.LBM_ERR_ARG
    L.lbm_refine_destroy(None)


def test_product_package_does_not_import_the_oracle():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys, paper_1608_04658_gb300 as p; p.lib(); "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.check_output([sys.executable, "-c", code], cwd=root).decode().strip()
    assert out == "False"
    for dirpath, _, files in os.walk(os.path.join(root, "paper_1608_04658_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "kbc_oracle" not in text, f


def test_fine_shape_of_closed_and_spanning_blocks():
    """The binding sizes the fine lattice as lbm_refine_create requires: 2 (hi -
    lo) + 2 nodes along a closed axis, 2n along a spanned periodic one; a
    block reaching both ends of a non-periodic axis is not spanning."""
    from paper_1608_04658_gb300 import binding
    assert binding.fine_shape((24, 20, 18), (0,) * 6, (5, 4, 3), (16, 13, 12)) == \
        ((False, False, False), (24, 20, 20))
    assert binding.fine_shape((48, 32, 4), (2, 3, 2, 2, 0, 0), (12, 8, 0), (35, 23, 4)) == \
        ((False, False, True), (48, 32, 8))
    assert binding.fine_shape((16, 12, 10), (0, 0, 0, 0, 1, 1), (4, 3, 0), (11, 8, 10))[0] == (False, False, False)


def test_closing_a_lattice_first_closes_its_refinements(monkeypatch):
    """A refinement keeps pointers to both levels, so closing either Lattice
    destroys the refinement before the context (library calls recorded, not
    made)."""
    import weakref
    from paper_1608_04658_gb300 import binding
    calls = []

    class Rec:
        def lbm_destroy(self, ctx):
            calls.append(("destroy", ctx))

        def lbm_refine_destroy(self, r):
            calls.append(("refine_destroy", r))

    monkeypatch.setattr(binding, "lib", lambda: Rec())
    coarse = binding.Lattice.__new__(binding.Lattice)
    fine = binding.Lattice.__new__(binding.Lattice)
    coarse._ctx, fine._ctx, coarse._dependents, fine._dependents = "c", "f", [], []
    ref = binding.Refinement.__new__(binding.Refinement)
    ref._r, ref.coarse, ref.fine = "r", coarse, fine
    coarse._dependents.append(weakref.ref(ref))
    fine._dependents.append(weakref.ref(ref))
    coarse.close()
    fine.close()
    ref.close()
    assert calls == [("refine_destroy", "r"), ("destroy", "c"), ("destroy", "f")]


def test_a_refused_refinement_closes_the_fine_lattice_it_made(monkeypatch):
    """lbm_refine_create refusing the block raises LbmError with the coarse
    context's message, and the fine Lattice made for it is closed at once
    (library calls recorded, not made)."""
    import types

    from paper_1608_04658_gb300 import binding
    made = []

    class FakeLattice:
        def __init__(self, shape, nu, storage, **kw):
            self.shape, self.nu, self._ctx, self.closed = shape, nu, "f", False
            made.append(self)

        def close(self):
            self.closed = True

    class Rec:
        def lbm_refine_create(self, c, f, lo, hi, out):
            return binding.LBM_ERR_ARG

        def lbm_last_error(self, ctx):
            return b"block outside the coarse lattice"

    monkeypatch.setattr(binding, "lib", lambda: Rec())
    monkeypatch.setattr(binding, "Lattice", FakeLattice)
    coarse = types.SimpleNamespace(_ctx="c", shape=(24, 20, 18), storage="fp32", rho0=1.0, device=None,
                                   _dependents=[],
                                   params=types.SimpleNamespace(face=[0] * 6, nu=0.02, gamma_mode=0))
    with pytest.raises(binding.LbmError) as e:
        binding.Refinement(coarse, (5, 4, 3), (16, 13, 12))
    assert e.value.status == binding.LBM_ERR_ARG and "outside" in str(e.value)
    assert len(made) == 1 and made[0].closed and made[0].shape == (24, 20, 20)
    assert coarse._dependents == []
