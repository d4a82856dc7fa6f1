"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module holds no arithmetic of the method: only the workload parameters
and the synthetic PDF grid (an input table of x f(x, Q^2) values).  The paper's
runs used a real PDF set through PDFFlow (Sec. 1, Sec. 3); none is available
here, so a smooth parametrised grid with seeded multiplicative noise stands
in for it.

Grid: 100 nodes in x, ln-uniform on [1e-6, 1], by 50 nodes in Q^2,
ln-uniform on [1, 1e8] GeV^2, for three flavours (0 gluon, 1 u, 2 ubar):

    x g(x, Q^2)    = A x^-0.3 (1-x)^5 (1 + 0.1 ln Q^2)
    x u(x, Q^2)    = B x^0.5  (1-x)^3
    x ubar(x, Q^2) = 0.2 B x^0.5 (1-x)^3

with A = 0.5 / Beta(0.7, 6) (momentum fraction 1/2 at Q^2 = 1) and
B = 2 / Beta(0.5, 4) (valence number 2), each node multiplied by
(1 + 0.01 z), z uniform in [-1, 1) from numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

PDF_NX = 100
PDF_NQ = 50
PDF_NFLAV = 3
PDF_X_MIN = 1e-6
PDF_Q2_MIN = 1.0
PDF_Q2_MAX = 1e8
PDF_NOISE_SEED = 0x5DF

# process ids (same numbering in the C ABI and in the oracle)
EE_MUMU, GG_TT, UU_TT, GG_TTG, UG_TTU, GG_TTGG, GG_TTGGG = 0, 1, 2, 3, 4, 5, 6
PROCESS_NAMES = {
    EE_MUMU: "e+e- -> mu+mu-",
    GG_TT: "g g -> t tbar",
    UU_TT: "u ubar -> t tbar",
    GG_TTG: "g g -> t tbar g",
    UG_TTU: "u g -> t tbar u",
    GG_TTGG: "g g -> t tbar g g",
    GG_TTGGG: "g g -> t tbar g g g",
}
N_EXT = {EE_MUMU: 4, GG_TT: 4, UU_TT: 4, GG_TTG: 5, UG_TTU: 5, GG_TTGG: 6, GG_TTGGG: 7}
DIM = {EE_MUMU: 2, GG_TT: 10, UU_TT: 10, GG_TTG: 14, UG_TTU: 14, GG_TTGG: 18, GG_TTGGG: 22}


def _beta(a: float, b: float) -> float:
    return math.gamma(a) * math.gamma(b) / math.gamma(a + b)


def make_pdf_grid(seed: int = PDF_NOISE_SEED, noise: float = 0.01) -> np.ndarray:
    """Synthetic x f(x, Q^2) grid, shape (3, 100, 50), float64, C order [flav][ix][iq]."""
    lx = np.linspace(math.log(PDF_X_MIN), 0.0, PDF_NX)
    lq = np.linspace(math.log(PDF_Q2_MIN), math.log(PDF_Q2_MAX), PDF_NQ)
    x = np.exp(lx)
    x[-1] = 1.0
    A = 0.5 / _beta(0.7, 6.0)
    B = 2.0 / _beta(0.5, 4.0)
    X, LQ = np.meshgrid(x, lq, indexing="ij")
    g = A * X ** -0.3 * (1.0 - X) ** 5 * (1.0 + 0.1 * LQ)
    u = B * X ** 0.5 * (1.0 - X) ** 3 * np.ones_like(LQ)
    ub = 0.2 * u
    grid = np.stack([g, u, ub]).astype(np.float64)
    if noise:
        rng = np.random.default_rng(seed)
        z = rng.uniform(-1.0, 1.0, size=grid.shape)
        grid = grid * (1.0 + noise * z)
    grid[:, -1, :] = 0.0          # x = 1
    return np.ascontiguousarray(grid)


@dataclass
class Physics:
    """Physical parameters of the synthetic workloads (all in GeV)."""
    sqrt_s: float = 13000.0
    mt: float = 173.0
    alpha_s: float = 0.118
    mz: float = 91.188
    wz: float = 2.441404
    alpha_em_inv: float = 132.507
    gf: float = 1.16639e-5
    pt_min: float = 30.0
    eta_max: float = 2.5
    dr_min: float = 0.4
    seed: int = 0
    channel: int = 0
    n_bins: int = 50
    alpha: float = 1.5

    def as_dict(self):
        return asdict(self)


@dataclass
class Workload:
    name: str
    process: int
    n_events: int
    n_iter: int
    physics: Physics = field(default_factory=Physics)


def workloads():
    """The five synthetic workloads: e+e- at the Z pole, gg -> tt, gg -> ttg,
    gg -> ttgg at 13 TeV, and the batched pp -> tt + jets channels."""
    return {
        "ee_mumu": Workload("e+e- -> mu+mu-, sqrt(s)=91.19 GeV, 1e5 x 5", EE_MUMU, 100_000, 5,
                            Physics(sqrt_s=91.19, seed=0)),
        "gg_tt": Workload("gg -> t tbar, 13 TeV, 1e7 x 10", GG_TT, 10_000_000, 10, Physics(seed=1)),
        "gg_ttg": Workload("gg -> t tbar g, 13 TeV, 1e7 x 10", GG_TTG, 10_000_000, 10, Physics(seed=2)),
        "gg_ttgg": Workload("gg -> t tbar g g, 13 TeV, 4e6 x 10", GG_TTGG, 4_000_000, 10, Physics(seed=3)),
        # the multi-leg extension: three final gluons (pT > 30 GeV, |eta| < 2.5 and Delta R > 0.4
        # between every pair, as for two)
        "gg_ttggg": Workload("gg -> t tbar g g g, 13 TeV, 1e6 x 10", GG_TTGGG, 1_000_000, 10, Physics(seed=6)),
    }


BATCH_CHANNELS = [(GG_TT, 4_000_000), (UU_TT, 1_000_000), (GG_TTG, 2_000_000),
                  (UG_TTU, 1_000_000), (GG_TTGG, 1_000_000)]
