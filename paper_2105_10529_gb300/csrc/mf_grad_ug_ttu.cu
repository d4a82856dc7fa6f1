// Derivative kernels of the process ug_ttu (forward mode), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_ug_ttu.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_ug_ttu, 1, 0>;
using G = GradOps<P, Me_ug_ttu, true>;
const GradOpsTable kGrad = { &G::grad, &G::evaluate_grad, 3, true, true };
}  // namespace

const GradOpsTable* grad_ug_ttu() { return &kGrad; }
}  // namespace mf
