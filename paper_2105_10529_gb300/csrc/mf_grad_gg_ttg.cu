// Derivative kernels of the process gg_ttg (forward mode), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_gg_ttg.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_gg_ttg>;
using G = GradOps<P, Me_gg_ttg, true>;
const GradOpsTable kGrad = { &G::grad, &G::evaluate_grad, 3, true };
}  // namespace

const GradOpsTable* grad_gg_ttg() { return &kGrad; }
}  // namespace mf
