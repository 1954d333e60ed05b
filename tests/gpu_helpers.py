"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the
same seeded workload and compare element by element."""
import numpy as np

import oracle
import paper_2609_25670_b300 as lbm

FIELDS = ("phi", "U", "T", "ux", "uy", "rho")


def active(p):
    out = ["phi"]
    if p.has_U:
        out.append("U")
    if p.has_T:
        out.append("T")
    if p.has_flow:
        out += ["ux", "uy", "rho"]
    return out


def run_gpu(p, fields, steps, precision="f64", graphs=True, chunks=None):
    sim = lbm.Simulation(p, precision=precision)
    sim.set_graphs(graphs)
    sim.init_fields(fields)
    for c in (chunks or [steps]):
        sim.advance(c)
    out = {k: sim.field(k) for k in active(p)}
    out["diag"] = sim.diagnostics()
    sim.close()
    return out


def run_oracle(p, fields, steps):
    o = oracle.Oracle(p, fields)
    o.advance(steps)
    out = {k: o.get(k) for k in active(p)}
    out["diag"] = o.diagnostics()
    o.close()
    return out


def max_err(a, b, keys):
    return {k: float(np.abs(a[k] - b[k]).max()) for k in keys}
