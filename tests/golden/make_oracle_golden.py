"""Writes oracle_events.json: per-event outputs of the FP64 oracle for a few
events of every process, as a frozen record that the tests compare the oracle
(regressions) and the CUDA path against.

Each event runs the whole pipeline of the paper's Sec. 2.1 in the oracle:
Philox uniforms, the VEGAS map at a fixed non-uniform grid, the parton map and
RAMBO phase space, the fiducial cuts, the PDFs and the spin- and colour-summed
|M|^2 of Sec. 2.2, and the event weight.  The paper prints no per-event values,
so every number here comes from the oracle through this script, which calls
nothing but oracle/ and the seeded input module.

    python -m tests.golden.make_oracle_golden
"""
import json
import os

import oracle as O
from paper_2105_10529_gb300 import inputs as IN

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "oracle_events.json")

PHYSICS = {
    IN.EE_MUMU: IN.Physics(sqrt_s=91.19, seed=11),
    IN.GG_TT: IN.Physics(seed=12),
    IN.UU_TT: IN.Physics(seed=13, channel=1),
    IN.GG_TTG: IN.Physics(seed=14),
    IN.UG_TTU: IN.Physics(seed=15, channel=3),
    IN.GG_TTGG: IN.Physics(seed=16),
    IN.GG_TTGGG: IN.Physics(seed=17),
}
ITERATION = 5
N_FIRST = {IN.EE_MUMU: 8, IN.GG_TT: 8, IN.UU_TT: 8, IN.GG_TTG: 8, IN.UG_TTU: 8, IN.GG_TTGG: 4, IN.GG_TTGGG: 6}
HIGH_EVENT = (1 << 32) + 3          # the Philox counter's second word in use
U_STORED = 4                        # uniforms stored per event (the first dimensions, at most D)


def grid_for(dim: int, nb: int = 50):
    """A fixed non-uniform VEGAS grid without random numbers: edges (b / nb)^a_d
    with a_d = 0.7 + 0.15 (d mod 5), so bins and widths differ per dimension."""
    g = []
    for d in range(dim):
        a = 0.7 + 0.15 * (d % 5)
        g.append([(b / nb) ** a for b in range(nb + 1)])
    return g


def events_of(proc: int):
    return list(range(N_FIRST[proc])) + [HIGH_EVENT]


def main():
    import numpy as np
    pdf = O.Pdf(IN.make_pdf_grid())
    out = {"note": "FP64 oracle outputs written by tests/golden/make_oracle_golden.py", "iteration": ITERATION,
           "u_stored": U_STORED, "processes": {}}
    for proc, phys in PHYSICS.items():
        dim = IN.DIM[proc]
        grid = np.array(grid_for(dim, phys.n_bins))
        evs = []
        for e in events_of(proc):
            o = O.event(proc, phys, pdf, grid, e, ITERATION)
            evs.append({"event": e, "u": [float(x) for x in o.u[:min(U_STORED, dim)]],
                        "bins": [int(b) for b in o.bins[:dim]], "mask": int(o.mask),
                        "me2": float(o.me2), "w": float(o.w)})
        out["processes"][str(proc)] = {"name": IN.PROCESS_NAMES[proc], "physics": phys.as_dict(), "events": evs}
    with open(PATH, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
