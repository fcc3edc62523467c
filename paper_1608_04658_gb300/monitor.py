"""Run monitoring: after every k steps, one JSON line with the FP64 global sums
(mass, momentum, kinetic energy; `lbm_totals`) and the body's force, torque,
pose, time, counters and status bits (`lbm_get_body`).  Both reads
synchronise with the context's stream, so k sets how often the host waits.
"""
from __future__ import annotations

import json


def record(lat, step: int) -> dict:
    """One monitoring record of lattice `lat` after `step` steps."""
    T = lat.totals()
    b = lat.body()

    def vec(v):
        return [float(x) for x in v]

    return {"step": int(step), "mass": float(T[0]), "momentum": vec(T[1:4]), "kinetic_energy": float(T[4]),
            "F": vec(b["F"]), "M": vec(b["M"]), "X": vec(b["X"]), "U": vec(b["U"]), "t": float(b["t"]),
            "n_boundary": int(b["n_boundary"]), "n_links": int(b["n_links"]),
            "n_uncovered": int(b["n_uncovered"]), "status": int(b["status"])}


def run_logged(lat, nsteps: int, every: int, out) -> list[dict]:
    """Advances `lat` by nsteps steps and writes a record after every `every`
    steps and after the last one, one JSON object per line, to `out` (a path,
    appended to, or a text stream).  Returns the records."""
    if every < 1 or nsteps < 0:
        raise ValueError("every must be >= 1 and nsteps >= 0")
    stream = open(out, "a") if isinstance(out, (str, bytes)) or hasattr(out, "__fspath__") else out
    recs = []
    try:
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            lat.step(k)
            done += k
            r = record(lat, done)
            stream.write(json.dumps(r) + "\n")
            stream.flush()
            recs.append(r)
    finally:
        if stream is not out:
            stream.close()
    return recs
