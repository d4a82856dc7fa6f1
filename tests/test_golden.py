"""The FP64 oracle against its frozen per-event record (tests/golden/): the
same uniforms, VEGAS bins and cut masks bit for bit, and |M|^2 and the weight
to 1e-12 relative (a later change to the oracle's arithmetic shows here)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2105_10529_gb300 import inputs as IN
from tests.golden import make_oracle_golden as G


@pytest.fixture(scope="module")
def golden():
    with open(G.PATH) as f:
        return json.load(f)


def test_golden_covers_every_process(golden):
    assert golden["iteration"] == G.ITERATION
    assert sorted(int(k) for k in golden["processes"]) == sorted(G.PHYSICS)
    for k, rec in golden["processes"].items():
        assert [e["event"] for e in rec["events"]] == G.events_of(int(k))
        assert any(e["mask"] == 1 and e["w"] != 0.0 for e in rec["events"])


@pytest.mark.parametrize("proc", sorted(G.PHYSICS))
def test_oracle_reproduces_golden(proc, golden):
    rec = golden["processes"][str(proc)]
    phys = IN.Physics(**rec["physics"])
    assert phys == G.PHYSICS[proc]
    dim = IN.DIM[proc]
    grid = np.array(G.grid_for(dim, phys.n_bins))
    pdf = O.Pdf(IN.make_pdf_grid())
    for e in rec["events"]:
        o = O.event(proc, phys, pdf, grid, e["event"], golden["iteration"])
        assert list(o.u[:len(e["u"])]) == e["u"], e["event"]
        assert [int(b) for b in o.bins[:dim]] == e["bins"], e["event"]
        assert int(o.mask) == e["mask"], e["event"]
        for key, val in (("me2", o.me2), ("w", o.w)):
            assert abs(val - e[key]) <= 1e-12 * abs(e[key]) + 1e-300, (e["event"], key, val, e[key])
