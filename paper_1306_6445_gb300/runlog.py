"""Chunked runs with a JSON-lines log: the per-chunk record of a long lattice run.

`run_logged` advances a lattice in chunks of time steps and after each chunk appends one
JSON object per line to a log file: the step count, the chunk's MLUPS (host wall time
around the synchronised chunk), the relative mass drift since the first record, max |v|
(both from the library's FP64 reduction, lb_reduce) and, for a droplet, the GPU Laplace
measurement (lb_measure_droplet: rho_in, rho_out, theta). All numbers come from the
library's kernels; this module only orders the calls and writes the records.
"""
from __future__ import annotations

import json
import time


def run_logged(lat, steps: int, chunk: int, path: str, radius: float | None = None,
               clock=time.perf_counter):
    """Advance `lat` (an lbm.Lattice, or anything with the same step / sync / reduce /
    measure_droplet / nx / ny / steps_done members) by `steps` time steps in chunks of at
    most `chunk`, appending one record per chunk to `path`. Returns the records.

    A record: {"step", "mlups", "mass", "mass_drift", "max_v"} plus, when `radius` is given,
    {"rho_in", "rho_out", "theta"} of the droplet centred on the lattice."""
    if steps < 0 or chunk < 1:
        raise ValueError("steps must be >= 0 and chunk >= 1")
    records = []
    mass0 = None
    done = 0
    with open(path, "a") as fh:
        while done < steps:
            n = min(chunk, steps - done)
            lat.sync()
            t0 = clock()
            lat.step(n)
            lat.sync()
            dt = clock() - t0
            done += n
            mass, _, _, vmax = (float(v) for v in lat.reduce())
            if mass0 is None:
                mass0 = mass
            rec = {"step": int(lat.steps_done),
                   "mlups": lat.nx * lat.ny * n / dt / 1e6 if dt > 0 else None,
                   "mass": mass, "mass_drift": (mass - mass0) / mass0, "max_v": vmax}
            if radius is not None:
                m = lat.measure_droplet(radius)
                rec.update(rho_in=m["rho_in"], rho_out=m["rho_out"], theta=m["theta"])
            fh.write(json.dumps(rec) + "\n")
            fh.flush()
            records.append(rec)
    return records
