// Colour sum on the 5th-generation tensor cores (tcgen05, sm_100 family).
//
// Per helicity, |M_h|^2 = sum_ij Re(conj(J_i) C_ij J_j) = Re(J)^T C Re(J) +
// Im(J)^T C Im(J) for the symmetric colour matrix C (Sec. 2.2: the colour
// sum of the colour-flow amplitudes).  With one event per thread, every
// group of 128 threads (warps 4g .. 4g+3) forms two dense (128 x 24) x
// (24 x 24) contractions D = J C per helicity, on 128 TMEM columns of its
// own (group g at column 128 g; CTAs of 128 or 256 threads):
//
//   A = J, one TMEM lane per event (the thread writes its own row with
//       tcgen05.st), split into two bf16 pieces J = J1 + J2 + r with
//       |r| <= 2^-16 |J|;
//   B = 54 C, integers in [-64, 512], exact in bf16, in shared memory
//       (K-major, no swizzle), zero-padded to 32 x 32;
//   D = (J1 + J2) (54 C) accumulated in FP32 in TMEM.
//
// Each thread then forms sum_i (2 J_i - J1_i - J2_i) D_i = J^T (54 C) J -
// r^T (54 C) r, i.e. the colour sum up to a relative 2^-32 (times the
// condition of C), read back with tcgen05.ld from its own lane.
//
// Waits on the MMA completion mbarrier are bounded: on expiry the thread
// raises the error flag and goes on (the result of that helicity is wrong
// and the host reports MF_ERR_TIMEOUT).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace mf {

// TMEM columns of one 128-thread group (lane = event/thread); a CTA of G
// groups allocates G x 128 columns (a power of two)
constexpr uint32_t TC_COLS = 128;
constexpr uint32_t TC_A_RE1 = 0, TC_A_RE2 = 16, TC_A_IM1 = 32, TC_A_IM2 = 48;   // 16 columns each (32 bf16)
constexpr uint32_t TC_D_RE = 64, TC_D_IM = 96;                                  // 32 FP32 columns each
constexpr int TC_N = 32, TC_K = 32;      // padded N (output columns) and K of the contraction
constexpr unsigned TC_WAIT_LIMIT = 1u << 20;

// Per-CTA state in shared memory (16-byte aligned)
struct TcCta {
    uint16_t B[TC_N * TC_K];             // 54 C as bf16 in the core-matrix layout below
    unsigned long long mbar;             // MMA-completion barrier
    uint32_t tmem;                       // TMEM base address of the allocation
    uint32_t phase;                      // parity of the next completion (same in every thread)
    unsigned* err;                       // device flag raised when a wait runs out
    uint32_t dead;                       // set after an expired wait: no further MMAs or waits
    uint32_t pad_;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of B element (n, k) in the K-major, no-swizzle canonical layout:
// core matrices of 8 rows (n) x 16 bytes (8 bf16 along k), 8-row groups
// 128 bytes apart (SBO), k-groups 512 bytes apart (LBO).
__host__ __device__ __forceinline__ uint32_t tc_b_offset(int n, int k)
{
    return (uint32_t)((k >> 3) * 512 + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 128-thread groups of this CTA (blockDim.x is 128 or 256)
__device__ __forceinline__ uint32_t tc_groups() { return blockDim.x >> 7; }

// one warp: allocate ncols columns, the address lands in *dst (shared memory)
__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
                 "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// two x16 loads and the wait in one statement, so that no use of the
// registers can be scheduled before the data has arrived
__device__ __forceinline__ void tc_ld16x2(uint32_t ta, uint32_t (&a)[16], uint32_t tb, uint32_t (&b)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%32];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
                 "%27, %28, %29, %30, %31}, [%33];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
                   "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]),
                   "=r"(a[15]), "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]),
                   "=r"(b[7]), "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]),
                   "=r"(b[14]), "=r"(b[15])
                 : "r"(ta), "r"(tb)
                 : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[tmem] B[smem desc]; accumulate = 0 overwrites D
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
                 : "memory");
}
// the mbarrier completes one phase when the MMAs issued so far by this thread are done
__device__ __forceinline__ void tc_commit(unsigned long long* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
// bounded wait for the completion of the phase with the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, uint32_t parity, unsigned limit = TC_WAIT_LIMIT)
{
    const uint32_t a = smem_u32(mbar);
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t bf16_bits(float x)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    return (uint32_t)__bfloat16_as_ushort(h);
}
// two floats rounded to bf16 and packed: x0 in the low half, x1 in the high half
__device__ __forceinline__ uint32_t bf16x2_bits(float x0, float x1)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_value(uint32_t bits)
{
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)bits));
}

// Set-up by the whole CTA (every thread calls), once per CTA: B = 54 C from
// c54 [ncol][ncol] (row-major, symmetric), the mbarrier and the TMEM
// allocation of cols columns per group (warp 0), after which the CTA
// relinquishes the allocation permit.
template <int NCOL>
__device__ __forceinline__ void tc_setup(TcCta* tc, const short* c54, unsigned* err, uint32_t cols = TC_COLS)
{
    static_assert(NCOL <= TC_N && NCOL <= TC_K, "colour basis larger than the padded contraction");
    for (int idx = threadIdx.x; idx < TC_N * TC_K; idx += blockDim.x) {
        const int n = idx / TC_K, k = idx % TC_K;
        const float v = (n < NCOL && k < NCOL) ? (float)c54[n * NCOL + k] : 0.0f;
        tc->B[tc_b_offset(n, k) / 2] = (uint16_t)bf16_bits(v);
    }
    if (threadIdx.x == 0) {
        mbar_init(&tc->mbar, 1);
        tc->phase = 0;
        tc->err = err;
        tc->dead = 0;
    }
    // generic-proxy writes of B become visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        tc_alloc(&tc->tmem, cols * tc_groups());
        // give up the right to allocate again: while a CTA holds it, no further
        // CTA of the kernel is placed on the SM
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Release by the whole CTA (every thread calls) once no thread uses TMEM any more.
__device__ __forceinline__ void tc_teardown(TcCta* tc, uint32_t cols = TC_COLS)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tc_dealloc(tc->tmem, cols * tc_groups());
}

// TMEM address of this thread's lane at column 0 of its group's columns: a
// warp reaches lanes 32 (w mod 4) .. +31, the group w / 4 its own columns
__device__ __forceinline__ uint32_t tc_lane(const TcCta* tc)
{
    const uint32_t warp = threadIdx.x >> 5;
    return tc->tmem + (((warp & 3u) * 32u) << 16) + (warp >> 2) * TC_COLS;
}

// Colour sum of this thread's colour-flow amplitudes (jamp: NCOL complex in
// shared memory, re/im interleaved), scaled by 54.  Every thread of the
// CTA (128 or 256 threads) calls it for the same helicity.  tc->err is set to
// 1 when a wait runs out.
template <int NCOL>
__device__ __forceinline__ float tc_colour_sum(TcCta* tc, const volatile float* jamp)
{
    const int tid = threadIdx.x;
    const uint32_t lane_base = tc_lane(tc);
    // parity of this call's completion, read by every thread before the barrier
    // after which thread 0 flips it
    const uint32_t parity = tc->phase & 1u;
    // A pieces: 32 bf16 per row (k >= NCOL zero), packed two per 32-bit column, low half = even k;
    // u = 2 J - (J1 + J2) stays in registers for the final contraction
    float u[2][TC_K];
#pragma unroll
    for (int part = 0; part < 2; ++part) {          // 0: real parts, 1: imaginary parts
        uint32_t p1[16], p2[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int k0 = 2 * c, k1 = 2 * c + 1;
            const float x0 = k0 < NCOL ? jamp[2 * k0 + part] : 0.0f;
            const float x1 = k1 < NCOL ? jamp[2 * k1 + part] : 0.0f;
            const uint32_t w1 = bf16x2_bits(x0, x1);
            const float h0 = __uint_as_float(w1 << 16), h1 = __uint_as_float(w1 & 0xFFFF0000u);
            const uint32_t w2 = bf16x2_bits(x0 - h0, x1 - h1);
            const float l0 = __uint_as_float(w2 << 16), l1 = __uint_as_float(w2 & 0xFFFF0000u);
            u[part][k0] = fmaf(2.0f, x0, -(h0 + l0));
            u[part][k1] = fmaf(2.0f, x1, -(h1 + l1));
            p1[c] = w1;
            p2[c] = w2;
        }
        tc_st16(lane_base + (part ? TC_A_IM1 : TC_A_RE1), p1);
        tc_st16(lane_base + (part ? TC_A_IM2 : TC_A_RE2), p2);
    }
    tc_wait_st();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // after an expired wait the CTA stops using the tensor cores (uniform: read after the barrier)
    if (tc->dead) {
        __syncthreads();
        return 0.0f;
    }
    if (tid == 0) {
        tc->phase = parity ^ 1u;
        constexpr uint32_t idesc = tc_idesc(128, TC_N);
        const uint32_t b0 = smem_u32(tc->B);
        // per group: D_re = (A_re1 + A_re2) B, D_im = (A_im1 + A_im2) B; K = 32 in two steps of 16
        const uint32_t groups = tc_groups();
        for (uint32_t g = 0; g < groups; ++g) {
            const uint32_t base = tc->tmem + g * TC_COLS;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const uint32_t d = base + (part ? TC_D_IM : TC_D_RE);
                const uint32_t a1 = base + (part ? TC_A_IM1 : TC_A_RE1);
                const uint32_t a2 = base + (part ? TC_A_IM2 : TC_A_RE2);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t bd = tc_smem_desc(b0 + (uint32_t)ks * 1024u, 512u, 128u);
                    tc_mma_ts(d, a1 + 8u * ks, bd, idesc, ks > 0 ? 1u : 0u);
                    tc_mma_ts(d, a2 + 8u * ks, bd, idesc, 1u);
                }
            }
        }
        tc_commit(&tc->mbar);   // one arrival once every MMA above has completed
    }
    if (!mbar_wait(&tc->mbar, parity)) {
        tc->dead = 1u;
        if (tc->err) atomicExch(tc->err, 1u);
    }
    tc_fence_after();
    uint32_t dre[16], dim[16];
    float acc = 0.0f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        tc_ld16x2(lane_base + TC_D_RE + 16 * half, dre, lane_base + TC_D_IM + 16 * half, dim);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int k = 16 * half + c;
            if (k < NCOL) {
                acc = fmaf(u[0][k], __uint_as_float(dre[c]), acc);
                acc = fmaf(u[1][k], __uint_as_float(dim[c]), acc);
            }
        }
    }
    // the flipped parity is visible to every thread, and every read of D is
    // done, before the next call writes A and issues the next MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return acc;
}

// ------------------------------------------------------------------ amplitudes produced in TMEM
//
// The helicity-recycled recursion (mf_rc.cuh) forms a configuration's colour-flow
// amplitudes two at a time and writes them straight into its TMEM lane, so no row of
// shared memory holds them: per group of 128 threads TC_RC_COLS columns, the A pieces
// and D as above and, from column TC_U, the FP32 u = 2 J - J1 - J2 of every flow
// (flows 2c, 2c + 1 at columns TC_U + 4c + 0..3 as re, re, im, im).
constexpr uint32_t TC_RC_COLS = 256;
constexpr uint32_t TC_U = 128;

__device__ __forceinline__ uint32_t tc_rc_lane(const TcCta* tc)
{
    const uint32_t warp = threadIdx.x >> 5;
    return tc->tmem + (((warp & 3u) * 32u) << 16) + (warp >> 2) * TC_RC_COLS;
}
__device__ __forceinline__ void tc_st1(uint32_t taddr, uint32_t v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tc_st4(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v0), "r"(v1),
                 "r"(v2), "r"(v3)
                 : "memory");
}

// Once per CTA after tc_setup (every thread calls): the A columns of the padding flows
// k = NCOL .. TC_K - 1 are zero (the amplitudes only ever write the first NCOL / 2 columns).
template <int NCOL>
__device__ __forceinline__ void tc_rc_zero_pad(const TcCta* tc)
{
    static_assert(NCOL % 2 == 0 && NCOL <= TC_K, "pairs of flows");
    const uint32_t lb = tc_rc_lane(tc);
#pragma unroll
    for (uint32_t c = NCOL / 2; c < TC_K / 2; ++c) {
        tc_st1(lb + TC_A_RE1 + c, 0u);
        tc_st1(lb + TC_A_RE2 + c, 0u);
        tc_st1(lb + TC_A_IM1 + c, 0u);
        tc_st1(lb + TC_A_IM2 + c, 0u);
    }
    tc_wait_st();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Flows 2c and 2c + 1 of this thread's configuration (warp-uniform call): their bf16
// pieces into column c of the four A regions, u into its four columns.
__device__ __forceinline__ void tc_rc_put_pair(uint32_t lane_base, int c, float re0, float im0, float re1, float im1)
{
    const uint32_t r1 = bf16x2_bits(re0, re1);
    const float rh0 = __uint_as_float(r1 << 16), rh1 = __uint_as_float(r1 & 0xFFFF0000u);
    const uint32_t r2 = bf16x2_bits(re0 - rh0, re1 - rh1);
    const float rl0 = __uint_as_float(r2 << 16), rl1 = __uint_as_float(r2 & 0xFFFF0000u);
    const uint32_t i1 = bf16x2_bits(im0, im1);
    const float ih0 = __uint_as_float(i1 << 16), ih1 = __uint_as_float(i1 & 0xFFFF0000u);
    const uint32_t i2 = bf16x2_bits(im0 - ih0, im1 - ih1);
    const float il0 = __uint_as_float(i2 << 16), il1 = __uint_as_float(i2 & 0xFFFF0000u);
    tc_st1(lane_base + TC_A_RE1 + c, r1);
    tc_st1(lane_base + TC_A_RE2 + c, r2);
    tc_st1(lane_base + TC_A_IM1 + c, i1);
    tc_st1(lane_base + TC_A_IM2 + c, i2);
    tc_st4(lane_base + TC_U + 4 * c, __float_as_uint(fmaf(2.0f, re0, -(rh0 + rl0))),
           __float_as_uint(fmaf(2.0f, re1, -(rh1 + rl1))), __float_as_uint(fmaf(2.0f, im0, -(ih0 + il0))),
           __float_as_uint(fmaf(2.0f, im1, -(ih1 + il1))));
}

// The colour sum of the amplitudes that tc_rc_put_pair left in every thread's lane,
// scaled by 54 (as tc_colour_sum; every thread of the CTA calls, once per round).
template <int NCOL>
__device__ __forceinline__ float tc_rc_colour_sum(TcCta* tc)
{
    static_assert(NCOL <= 32 && NCOL % 2 == 0, "one x16 load of u per 16 flows");
    const int tid = threadIdx.x;
    const uint32_t lane_base = tc_rc_lane(tc);
    const uint32_t parity = tc->phase & 1u;
    tc_wait_st();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tc->dead) {
        __syncthreads();
        return 0.0f;
    }
    if (tid == 0) {
        tc->phase = parity ^ 1u;
        constexpr uint32_t idesc = tc_idesc(128, TC_N);
        const uint32_t b0 = smem_u32(tc->B);
        const uint32_t groups = tc_groups();
        for (uint32_t g = 0; g < groups; ++g) {
            const uint32_t base = tc->tmem + g * TC_RC_COLS;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const uint32_t d = base + (part ? TC_D_IM : TC_D_RE);
                const uint32_t a1 = base + (part ? TC_A_IM1 : TC_A_RE1);
                const uint32_t a2 = base + (part ? TC_A_IM2 : TC_A_RE2);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t bd = tc_smem_desc(b0 + (uint32_t)ks * 1024u, 512u, 128u);
                    tc_mma_ts(d, a1 + 8u * ks, bd, idesc, ks > 0 ? 1u : 0u);
                    tc_mma_ts(d, a2 + 8u * ks, bd, idesc, 1u);
                }
            }
        }
        tc_commit(&tc->mbar);
    }
    if (!mbar_wait(&tc->mbar, parity)) {
        tc->dead = 1u;
        if (tc->err) atomicExch(tc->err, 1u);
    }
    tc_fence_after();
    float acc = 0.0f;
    // flows 16 h .. 16 h + 15: D (re, im) and the u columns of pairs 8 h .. 8 h + 7
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        if (16 * half >= NCOL) break;
        uint32_t dre[16], dim[16], uu[32];
        tc_ld16x2(lane_base + TC_D_RE + 16 * half, dre, lane_base + TC_D_IM + 16 * half, dim);
        uint32_t u0[16], u1[16];
        tc_ld16x2(lane_base + TC_U + 32 * half, u0, lane_base + TC_U + 32 * half + 16, u1);
#pragma unroll
        for (int i = 0; i < 16; ++i) { uu[i] = u0[i]; uu[16 + i] = u1[i]; }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int k = 16 * half + 2 * c + e;
                if (k < NCOL) {
                    acc = fmaf(__uint_as_float(uu[4 * c + e]), __uint_as_float(dre[2 * c + e]), acc);
                    acc = fmaf(__uint_as_float(uu[4 * c + 2 + e]), __uint_as_float(dim[2 * c + e]), acc);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return acc;
}

}  // namespace mf

