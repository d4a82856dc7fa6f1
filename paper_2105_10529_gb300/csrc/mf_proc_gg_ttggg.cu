// Kernels of g g -> t tbar g g g: the fused integrand (mixed and FP64) with the
// warp-level Berends-Giele matrix element, and its evaluate / helicity-profile
// kernel, instantiated in their own translation unit.
#include "mf_dispatch.cuh"
#include "mf_me_gg_ttggg.cuh"

namespace mf {
namespace {
using ME = Me_gg_ttggg;
using P = ProcTops<ME>;
// mixed precision: one 256-thread CTA per SM (8 warps, each with its 14 KB state); FP64:
// 128 threads (the state is twice as large)
constexpr int T32 = 256, T64 = 128;
using L32 = SmemLayout<P, float, T32>;
using L64 = SmemLayout<P, double, T64>;

const void* fn(int prec)
{
    // per-event outputs are a run-time choice of the same kernel (kp.ev_out)
    return prec ? (const void*)integrand_kernel<P, float, T32, false, false>
                : (const void*)integrand_kernel<P, double, T64, false, false>;
}

size_t smem(int prec, int nb, int npv, bool obs) { return prec ? L32::bytes(nb, npv, obs) : L64::bytes(nb, npv, obs); }

cudaError_t prepare(size_t sm32, size_t sm64)
{
    cudaError_t e = cudaFuncSetAttribute(fn(1), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn(0), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64);
    return e;
}

cudaError_t occupancy(int prec, size_t sm, int* b)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, fn(prec), prec ? T32 : T64, sm);
}

cudaError_t integrand(int prec, bool, int, int, const KParams& kp, int nblk, size_t sm, cudaStream_t s)
{
    // the matrix-element batches stage the events' momenta in the per-CTA record region
    if (kp.inv_rec == nullptr || nblk > kp.inv_ctas) return cudaErrorInvalidValue;
    KParams arg = kp;
    void* args[1] = { &arg };
    return cudaLaunchKernel(fn(prec), dim3(nblk), dim3(prec ? T32 : T64), args, sm, s);
}

const void* kernel(int prec, bool, int, int) { return fn(prec); }

// mf_evaluate (me2) and mf_helicity_profile (hel_out): one warp per point, 4 warps per CTA
cudaError_t launch_eval(int prec, const double* mom, long long n, double* me2, double* hel, double mt, double gs,
                        cudaStream_t s)
{
    const size_t s32 = ME::cta_bytes<float>(4), s64 = ME::cta_bytes<double>(4);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute((const void*)bg_evaluate_kernel<float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)bg_evaluate_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)s64);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long want = (n + 3) / 4;
    const int nblk = (int)(want < 4096 ? want : 4096);
    if (prec) bg_evaluate_kernel<float><<<nblk, 128, s32, s>>>(mom, n, me2, hel, mt, gs);
    else bg_evaluate_kernel<double><<<nblk, 128, s64, s>>>(mom, n, me2, hel, mt, gs);
    return cudaGetLastError();
}

cudaError_t evaluate(int prec, const double* mom, long long n, double* me2, double mt, double gs, const EwParams&, int,
                     cudaStream_t s)
{
    return launch_eval(prec, mom, n, me2, nullptr, mt, gs, s);
}

cudaError_t profile(int prec, const double* mom, long long n, double* out, double mt, double gs, const EwParams&, int,
                    cudaStream_t s)
{
    return launch_eval(prec, mom, n, nullptr, out, mt, gs, s);
}

const ProcOps kOps = { P::D, P::NEXT, P::NPDF, &smem, &prepare, &occupancy, &integrand, &evaluate, &kernel,
                       &profile, ME::NHEL, ME::NHEL / 2 };
}  // namespace

const ProcOps* ops_gg_ttggg() { return &kOps; }

namespace {
// d|M|^2/dp and the m_t derivative pass by the reverse sweep (FP64 and mixed)
const GradOpsTable kGrad = { &BgGradPass<P, BgGen_gg_ttggg, 6>::grad, &BgEvalGrad<BgGen_gg_ttggg, 6>::launch, 5, true,
                             true, true, 2 };
}  // namespace
const GradOpsTable* grad_gg_ttggg() { return &kGrad; }
}  // namespace mf
