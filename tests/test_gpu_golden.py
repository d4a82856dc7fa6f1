"""The CUDA path through the C ABI against the oracle's frozen per-event
record (tests/golden/oracle_events.json): uniforms of the stored dimensions,
VEGAS bins and cut masks bit for bit; |M|^2 and the weight within 1e-12
(FP64 path) and 1e-5 (mixed path) relative."""
import json

import numpy as np
import pytest

from paper_2105_10529_gb300 import inputs as IN
from tests.golden import make_oracle_golden as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def golden():
    with open(G.PATH) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("proc", sorted(G.PHYSICS))
def test_cuda_path_matches_golden(proc, prec, golden):
    from paper_2105_10529_gb300.api import Context
    rec = golden["processes"][str(proc)]
    phys = IN.Physics(**rec["physics"])
    dim = IN.DIM[proc]
    grid = torch.tensor(np.array(G.grid_for(dim, phys.n_bins)), device="cuda")
    ctx = Context(phys, IN.make_pdf_grid(), precision=prec)
    evs = rec["events"]
    first = [e for e in evs if e["event"] < G.HIGH_EVENT]
    got = []
    for offset, n in ((0, len(first)), (G.HIGH_EVENT, 1)):
        _, ev = ctx.vegas_pass(proc, phys.sqrt_s, grid, n, ev_offset=offset, iteration=golden["iteration"],
                               want_events=True, fields=("u", "bins", "mask", "me2", "w"))
        got += [{k: ev[k][i].cpu().numpy() for k in ev} for i in range(n)]
    ctx.device_status()
    ctx.close()
    for e, g in zip(evs, got):
        assert list(g["u"][:len(e["u"])]) == e["u"], e["event"]
        assert [int(b) for b in g["bins"]] == e["bins"], e["event"]
        assert int(g["mask"]) == e["mask"], e["event"]
        for key in ("me2", "w"):
            val = float(g[key])
            assert abs(val - e[key]) <= TOL[prec] * abs(e[key]) + 1e-300, (e["event"], key, val, e[key])
