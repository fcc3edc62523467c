"""Host logic of the run monitor: record cadence, JSON-lines output and the
fields it takes from the global sums and the body state (a stand-in lattice
with the binding's method names, so no GPU is needed)."""
import io
import json

import numpy as np

from paper_1608_04658_gb300 import monitor


class _Lattice:
    def __init__(self):
        self.n = 0

    def step(self, k):
        self.n += k

    def totals(self):
        return np.array([1000.0 + self.n, 0.1, 0.2, 0.3, 0.5])

    def body(self):
        z = np.zeros(3)
        return dict(X=np.array([1.0, 2.0, self.n]), U=z, F=np.array([0.0, 0.0, -self.n]), M=z, t=float(self.n),
                    n_boundary=7, n_links=11, n_uncovered=0, status=0)


def test_records_every_k_steps_and_after_the_last(tmp_path):
    lat = _Lattice()
    path = tmp_path / "run.jsonl"
    recs = monitor.run_logged(lat, 10, 3, path)
    assert [r["step"] for r in recs] == [3, 6, 9, 10]
    assert lat.n == 10
    lines = path.read_text().splitlines()
    assert [json.loads(s) for s in lines] == recs
    last = recs[-1]
    assert last["mass"] == 1010.0 and last["momentum"] == [0.1, 0.2, 0.3] and last["kinetic_energy"] == 0.5
    assert last["F"] == [0.0, 0.0, -10.0] and last["X"] == [1.0, 2.0, 10.0] and last["t"] == 10.0
    assert last["n_links"] == 11 and last["status"] == 0
    # appends to an existing log; a stream is left open
    monitor.run_logged(lat, 2, 5, path)
    assert len(path.read_text().splitlines()) == 5
    buf = io.StringIO()
    monitor.run_logged(lat, 1, 1, buf)
    assert json.loads(buf.getvalue())["step"] == 1


def test_rejects_a_zero_cadence():
    import pytest
    with pytest.raises(ValueError):
        monitor.run_logged(_Lattice(), 5, 0, io.StringIO())
