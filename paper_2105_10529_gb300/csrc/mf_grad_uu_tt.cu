// Derivative kernels of the process uu_tt (forward mode), in a translation
// unit of their own so that they compile in parallel with the value kernels.
#include "mf_dispatch.cuh"
#include "generated/me_uu_tt.cuh"

namespace mf {
namespace {
using P = ProcTops<Me_uu_tt, 1, 2>;
using G = GradOps<P, Me_uu_tt, true>;
const GradOpsTable kGrad = { &G::grad, &G::evaluate_grad, 2, true, true };
}  // namespace

const GradOpsTable* grad_uu_tt() { return &kGrad; }
}  // namespace mf
