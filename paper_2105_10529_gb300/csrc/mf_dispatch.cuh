// Per-process launch table shared by the process translation units and the
// C ABI (host side only).
#pragma once
#include <algorithm>
#include <cuda_runtime.h>
#include "mf_integrand.cuh"

namespace mf {

struct ProcOps {
    int D, NEXT, npdf;
    size_t (*smem)(int prec, int nb, int npv, bool obs);   // obs: room for the observable histogram
    cudaError_t (*prepare)(size_t smem_mixed, size_t smem_fp64);
    cudaError_t (*occupancy)(int prec, size_t smem, int* blocks_per_sm);
    // sched: 0 free-running warps, 1 CTA barrier between helicities (heavy processes),
    // 2 barrier and the colour sum on the tensor cores (processes with P::TC, mixed precision),
    // 3 warp-per-event schedule with the tensor-core colour sum (P::TC, mixed precision,
    // kp.inv_rec set for every CTA; otherwise as 2);
    // 4 the helicity-recycled recursion with one warp per event (matrix elements with
    // RcTraits; otherwise as 3);
    // hsplit: 1, or 2 lanes per event each summing half the helicities (heavy processes,
    // mixed precision, sched >= 1; otherwise 1).
    // write: per-event outputs.  Schedule 3 and the helicity split run the same kernel with
    // and without them (kp.ev_out selects the stores at run time); the other schedules have
    // a separately compiled kernel with the stores
    cudaError_t (*integrand)(int prec, bool write, int sched, int hsplit, const KParams& kp, int nblk, size_t smem,
                             cudaStream_t s);
    cudaError_t (*evaluate)(int prec, const double* mom, long long n, double* me2, double mt, double gs,
                            const EwParams& ew, int nblk, cudaStream_t s);
    // the integrand kernel (function) that integrand() launches with these settings
    const void* (*kernel)(int prec, bool write, int sched, int hsplit);
    // per-helicity |M_h|^2 of caller momenta, out [n][nhel] (helicity profile)
    cudaError_t (*profile)(int prec, const double* mom, long long n, double* out, double mt, double gs,
                           const EwParams& ew, int nblk, cudaStream_t s);
    int nhel;
    // helicity sampling in the integrand (mf_set_helicity_sampling): the size of the helicity sum
    // it samples from (the parity-halved configurations), 0 where the integrand does not sample
    int hel_sample_max;
    // CTAs per SM of the kernel that integrand() launches with these settings when it is not
    // the occupancy of the default kernel (null, or 0: the occupancy applies)
    int (*sched_ctas)(int prec, int sched, int hsplit) = nullptr;
};

// helicity-profile launch of a matrix element with a hel_profile member
template <class ME>
cudaError_t profile_launch(int prec, const double* mom, long long n, double* out, double mt, double gs, const EwParams&,
                           int nblk, cudaStream_t s)
{
    if (prec) helicity_profile_kernel<ME, float><<<nblk, 64, 0, s>>>(mom, n, out, mt, gs);
    else helicity_profile_kernel<ME, double><<<nblk, 64, 0, s>>>(mom, n, out, mt, gs);
    return cudaGetLastError();
}

// Derivative kernels of one process, built in their own translation units.
struct GradOpsTable {
    cudaError_t (*grad)(int prec, const KParams& kp, int nblk, double* partials, int k_as, double alpha_s,
                        cudaStream_t s);
    cudaError_t (*evaluate_grad)(int prec, const double* mom, long long n, double* me2, double* dme2, double mt,
                                 double gs, int nblk, cudaStream_t s);
    int k_as;          // power of alpha_s in |M|^2
    bool has_fp64;     // FP64 (Dual<double>) derivative pass built
    bool has_fp64_evaluate;   // FP64 d|M|^2/dp built (evaluate_grad)
    bool has_pass = true;     // the derivative pass of the integrand (grad) exists
    int ctas_per_sm = 8;      // the largest grid the derivative pass takes: this many CTAs per SM
};

// The derivative pass by forward mode through the recursion (gluon processes with its tables G):
// two 128-thread CTAs per SM at most (their staging shares the per-SM record regions)
template <class P, class G, int SYM_DEN>
struct BgGradPass {
    template <typename R>
    static cudaError_t run(const KParams& kp, int nblk, double* partials, int k_as, double alpha_s, cudaStream_t s)
    {
        constexpr int MW = bg_grad_pass_warps<P, G, R>();
        static bool attr = false;   // per precision
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute((const void*)bg_grad_kernel<P, G, R, SYM_DEN, MW>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)bg_grad_pass_smem<P, G, R>(MAX_BINS, MW));
            if (e != cudaSuccess) return e;
            attr = true;
        }
        bg_grad_kernel<P, G, R, SYM_DEN, MW><<<nblk, 128, bg_grad_pass_smem<P, G, R>(kp.nb, MW), s>>>(kp, partials, k_as,
                                                                                                      alpha_s);
        return cudaGetLastError();
    }
    static cudaError_t grad(int prec, const KParams& kp, int nblk, double* partials, int k_as, double alpha_s,
                            cudaStream_t s)
    {
        if (kp.inv_rec == nullptr || nblk > 2 * kp.inv_ctas) return cudaErrorInvalidValue;
        return prec ? run<float>(kp, nblk, partials, k_as, alpha_s, s) : run<double>(kp, nblk, partials, k_as, alpha_s, s);
    }
};

const GradOpsTable* grad_gg_tt();
const GradOpsTable* grad_gg_ttg();
const GradOpsTable* grad_gg_ttgg();
const GradOpsTable* grad_uu_tt();
const GradOpsTable* grad_ug_ttu();
const GradOpsTable* grad_gg_ttggg();

template <class P, class ME, bool FP64>
struct GradOps {
    static cudaError_t grad(int prec, const KParams& kp, int nblk, double* partials, int k_as, double alpha_s,
                            cudaStream_t s)
    {
        const size_t sm = sizeof(double) * (P::D * (kp.nb + 1) + 16);
        if (prec) grad_kernel<P, Dual<float>><<<nblk, 128, sm, s>>>(kp, partials, k_as, alpha_s);
        else if constexpr (FP64) grad_kernel<P, Dual<double>><<<nblk, 128, sm, s>>>(kp, partials, k_as, alpha_s);
        else return cudaErrorNotSupported;
        return cudaGetLastError();
    }
    static cudaError_t evaluate_grad(int prec, const double* mom, long long n, double* me2, double* dme2, double mt,
                                     double gs, int nblk, cudaStream_t s)
    {
        if (prec) evaluate_grad_kernel<ME, Dual<float>><<<nblk, 128, 0, s>>>(mom, n, me2, dme2, mt, gs);
        else if constexpr (FP64) evaluate_grad_kernel<ME, Dual<double>><<<nblk, 128, 0, s>>>(mom, n, me2, dme2, mt, gs);
        else return cudaErrorNotSupported;
        return cudaGetLastError();
    }
};

const ProcOps* ops_ee_mumu();
const ProcOps* ops_gg_tt();
const ProcOps* ops_gg_ttg();
const ProcOps* ops_gg_ttgg();
const ProcOps* ops_uu_tt();
const ProcOps* ops_ug_ttu();
const ProcOps* ops_gg_ttggg();

// whether a warp-per-event process (HL) has the helicity-recycled schedule
template <class P, bool HL> struct ProcHasRc : std::false_type {};
template <class P> struct ProcHasRc<P, true> : HasRc<typename P::Me> {};

// integrand launch helpers for a process trait P: T32 threads per CTA for the
// mixed-precision kernels, T64 for the FP64 ones
template <class P, int T32, int T64 = T32>
struct IntegrandOps {
    template <typename R> static constexpr int tpb() { return sizeof(R) == 4 ? T32 : T64; }
    static size_t smem(int prec, int nb, int npv, bool obs)
    {
        return prec ? SmemLayout<P, float, T32>::bytes(nb, npv, obs) : SmemLayout<P, double, T64>::bytes(nb, npv, obs);
    }
    static constexpr bool HS = P::HEAVY;   // the barrier variant exists for heavy processes only
    static constexpr bool HT = P::TC;      // and the tensor-core colour sum for P::TC processes
    template <typename R, bool W, bool S>
    static const void* fn() { return (const void*)integrand_kernel<P, R, tpb<R>(), W, S && HS>; }
    template <bool W>
    static const void* fn_tc() { return (const void*)integrand_kernel<P, float, T32, W, HT, HT>; }
    // helicity split variants (mixed precision, barrier schedule, no per-event outputs)
    static const void* fn_hs() { return (const void*)integrand_kernel<P, float, T32, false, HS, false, HS ? 2 : 1>; }
    static const void* fn_hs_tc() { return (const void*)integrand_kernel<P, float, T32, false, HT, HT, HT ? 2 : 1>; }
    // warp-per-event schedule (P::TC processes with LH_TPB-thread mixed-precision CTAs)
    static constexpr bool HL = HT && T32 == LH_TPB;
    static const void* fn_lh() { return (const void*)integrand_kernel<P, float, T32, false, HL, HL, 1, HL>; }
    static size_t smem_lh(int nb, int npv, bool obs) { return SmemLayout<P, float, T32, HL>::bytes(nb, npv, obs); }
    // the helicity-recycled warp-per-event schedule (matrix elements with RcTraits, mf_rc.cuh):
    // RC_CTAS CTAs of RC_TPB threads per SM (one of 256: two CTAs of 128, whose FP64
    // kinematics and matrix elements could overlap, ran 10% slower with twice as many batches)
    static constexpr bool HR = ProcHasRc<P, HL>::value;
    static constexpr int RC_TPB = 256, RC_CTAS = 1;
    static const void* fn_rc()
    {
        if constexpr (HR) return (const void*)integrand_kernel<P, float, RC_TPB, false, true, true, 1, 2>;
        else return fn_lh();
    }
    static size_t smem_rc(int nb, int npv, bool obs)
    {
        if constexpr (HR) return SmemLayout<P, float, RC_TPB, 2>::bytes(nb, npv, obs);
        else return smem_lh(nb, npv, obs);
    }
    static int sched_ctas(int prec, int sched, int hsplit)
    {
        return (HR && prec && sched == 4 && hsplit == 1) ? RC_CTAS : 0;
    }
    // the dynamic shared memory of every variant of one precision (sm32, sm64: bytes)
    static cudaError_t prepare(size_t sm32, size_t sm64)
    {
        const void* f32[8] = { fn<float, false, false>(), fn<float, true, false>(), fn<float, false, true>(),
                               fn<float, true, true>(), fn_tc<false>(), fn_tc<true>(), fn_hs(), fn_hs_tc() };
        const void* f64[4] = { fn<double, false, false>(), fn<double, true, false>(), fn<double, false, true>(),
                               fn<double, true, true>() };
        for (const void* f : f32) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
            if (e != cudaSuccess) return e;
        }
        for (const void* f : f64) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64);
            if (e != cudaSuccess) return e;
        }
        if constexpr (HL) {
            // the warp-per-event kernel needs far less shared memory: ask for the smallest
            // carveout that holds it, so that the rest of the SM's L1 serves its local memory
            int dev = 0, smem_sm = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            if (e != cudaSuccess) return e;
            const size_t need = smem_lh(MAX_BINS, 0, true) + 1024;
            int pct = smem_sm > 0 ? (int)((need * 100 + (size_t)smem_sm - 1) / (size_t)smem_sm) : 100;
            if (pct > 100) pct = 100;
            e = cudaFuncSetAttribute(fn_lh(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(fn_lh(), cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            if (e != cudaSuccess) return e;
        }
        if constexpr (HR) {
            // the recycled schedule keeps its store in shared memory: its own limit, and the
            // smallest carveout that holds its CTAs, so that L1 keeps the rest (the task tables,
            // the PDF grid and the records are read through it; a carveout of 100% left L1
            // 28 KB and cost 9%)
            int dev = 0, smem_sm = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            if (e != cudaSuccess) return e;
            const size_t need = smem_rc(MAX_BINS, 0, true);
            const size_t per_sm = (need + 1024) * RC_CTAS;
            int pct = smem_sm > 0 ? (int)((per_sm * 100 + (size_t)smem_sm - 1) / (size_t)smem_sm) : 100;
            if (pct > 100) pct = 100;
            e = cudaFuncSetAttribute(fn_rc(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(fn_rc(), cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    static cudaError_t occupancy(int prec, size_t sm, int* b)
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, prec ? fn<float, false, false>() : fn<double, false, false>(),
                                                             prec ? T32 : T64, sm);
    }
    // the kernel that a launch with these settings runs
    template <typename R, bool W>
    static const void* pick(int sched, int hsplit)
    {
        constexpr int TPB = tpb<R>();
        if constexpr (HS && sizeof(R) == 4) {
            if (hsplit == 2 && sched >= 1) {
                if constexpr (HT) {
                    if (sched >= 2) return (const void*)integrand_kernel<P, float, TPB, false, true, true, 2>;
                }
                return (const void*)integrand_kernel<P, float, TPB, false, true, false, 2>;
            }
        }
        if constexpr (HR && sizeof(R) == 4) {
            if (sched == 4 && hsplit == 1) return fn_rc();
        }
        if constexpr (HL && sizeof(R) == 4) {
            if (sched >= 3 && hsplit == 1) return fn_lh();
        }
        if constexpr (HT && sizeof(R) == 4) {
            if (sched >= 2) return (const void*)integrand_kernel<P, float, TPB, W, true, true>;
        }
        if (sched && HS) return (const void*)integrand_kernel<P, R, TPB, W, HS>;
        return (const void*)integrand_kernel<P, R, TPB, W, false>;
    }
    static const void* kernel(int prec, bool write, int sched, int hsplit)
    {
        if (prec) return write ? pick<float, true>(sched, hsplit) : pick<float, false>(sched, hsplit);
        return write ? pick<double, true>(sched, hsplit) : pick<double, false>(sched, hsplit);
    }
    static cudaError_t integrand(int prec, bool write, int sched, int hsplit, const KParams& kp, int nblk, size_t sm,
                                 cudaStream_t s)
    {
        KParams arg = kp;
        void* args[1] = { &arg };
        // no record region for every CTA: as schedule 2
        if (sched == 4 && sched_ctas(prec, sched, hsplit) > 0) {
            if (kp.inv_rec == nullptr || (long long)nblk * RC_TPB > (long long)kp.inv_ctas * LH_TPB) sched = 2;
        } else if (sched >= 3 && (kp.inv_rec == nullptr || nblk > kp.inv_ctas)) {
            sched = 2;
        }
        const void* f = kernel(prec, write, sched, hsplit);
        int threads = prec ? T32 : T64;
        if constexpr (HL) {
            // the warp-per-event kernel runs with its own, smaller dynamic shared memory
            if (f == fn_lh()) sm = smem_lh(kp.nb, kp.pdfg.nx * kp.pdfg.nq, kp.nobs > 0);
            if constexpr (HR) {
                if (f == fn_rc()) {
                    sm = smem_rc(kp.nb, kp.pdfg.nx * kp.pdfg.nq, kp.nobs > 0);
                    threads = RC_TPB;
                }
            }
        }
        return cudaLaunchKernel(f, dim3(nblk), dim3(threads), args, sm, s);
    }
};

}  // namespace mf
