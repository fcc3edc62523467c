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
