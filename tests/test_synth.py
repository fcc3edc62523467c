"""The seeded input generator both sides draw from: splitmix64 (Steele, Lea,
Flood 2014) against the outputs of its published reference implementation
started from state 0, the 53-bit map to [0, 1), and the counter layout that
keeps (seed, stream) sequences apart."""
import numpy as np

import synth

# first outputs of the reference splitmix64 generator from state 0
REFERENCE = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]


def test_splitmix64_matches_the_reference_sequence():
    got = synth.splitmix64(np.arange(5, dtype=np.uint64))
    assert [int(v) for v in got] == REFERENCE


def test_uniform_takes_the_top_53_bits_of_the_counter_sequence():
    u = synth.uniform(0, 0, 5)
    assert list(u) == [(v >> 11) / 2.0 ** 53 for v in REFERENCE]
    assert ((u >= 0.0) & (u < 1.0)).all()


def test_seeds_and_streams_index_disjoint_counters():
    a = synth.uniform(3, 1, 4)
    base = (3 << 40) | (1 << 32)
    z = synth.splitmix64(np.arange(base, base + 4, dtype=np.uint64))
    assert list(a) == [(int(v) >> 11) / 2.0 ** 53 for v in z]
    assert not np.array_equal(synth.uniform(3, 0, 4), a)
    assert not np.array_equal(synth.uniform(4, 1, 4), a)


def test_refined_fields_agree_at_coincident_nodes():
    """The refined block workload's two levels carry one flow: the fine field
    at fine node j (coarse coordinate lo + j/2) equals the coarse field there
    at the coincident nodes (even j), so the initial state has no jump at the
    block's surface."""
    import numpy as np

    import synth
    wl = synth.refined_block(shape=(64, 32, 16), lo=(16, 8, 2), hi=(47, 23, 13))
    rc, uc = synth.refined_fields(wl, "coarse")
    rf, uf = synth.refined_fields(wl, "fine")
    (x0, y0, z0), (x1, y1, z1) = wl["lo"], wl["hi"]
    fz, fy, fx = rf.shape
    assert (fx, fy, fz) == wl["fine_shape"]
    sub_u = uc[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]
    assert np.allclose(uf[0:2 * (z1 - z0) + 1:2, 0:2 * (y1 - y0) + 1:2, 0:2 * (x1 - x0) + 1:2], sub_u,
                       rtol=0, atol=1e-15)
    assert np.array_equal(rf[:-1, :-1, :-1][::2, ::2, ::2], rc[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1])
