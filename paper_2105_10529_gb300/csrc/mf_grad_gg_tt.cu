// Derivative kernels of the process gg_tt (the m_t derivative pass in forward mode, d|M|^2/dp
// by the reverse sweep), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_tt.cuh"
#include "generated/bg_gg_tt.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_tt>;
using G = GradOps<P, Me_gg_tt, true>;
// d|M|^2/dp by the reverse sweep of the Berends-Giele recursion (FP64 and mixed)
using E = BgEvalGrad<BgGen_gg_tt, 1>;
const GradOpsTable kGrad = { &G::grad, &E::launch, 2, true, true };
}  // namespace

const GradOpsTable* grad_gg_tt() { return &kGrad; }
}  // namespace mf
