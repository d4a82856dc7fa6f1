// Fused per-event integrand, VEGAS pass reduction/refinement and the
// matrix-element evaluation kernel (Sec. 2.1 of arXiv:2105.10529: the
// event pipeline from random numbers through kinematics and matrix element
// to histogram filling, all resident on the GPU, Sec. 3.1).
//
// One thread evaluates one event at a time (grid-stride over the pass).  All
// per-event state (uniforms, momenta, wavefunctions) lives in registers; the
// only HBM traffic is the per-CTA partial sums at the end of the kernel.
// Reductions are deterministic: fixed warp-shuffle trees, per-warp shared
// histograms updated by one leader lane per distinct bin in lane order,
// warps combined in index order, CTAs combined in index order.
#pragma once
#include <cstddef>
#include <cstdint>
#include <type_traits>
#include "mf_bg.cuh"
#include "mf_device.cuh"
#include "mf_helas.cuh"
#include "mf_kin_df.cuh"
#include "mf_tc.cuh"

namespace mf {

constexpr double GEV2_TO_PB = 0.3893793721e9;   // (hbar c)^2 in pb GeV^2
constexpr int MAX_DIM = 22;
constexpr int KIN_NEXT_MAX = 7;      // largest process (2 -> 5) for the global kinematics store
constexpr int KIN_CAP_UNIT = 256;    // ring entries per region of the global kinematics store
constexpr int MAX_BINS = 64;
constexpr int MAX_OBS_BINS = 100;    // observable histogram: regular bins (plus under- and overflow)
constexpr int LH_INV_WORDS_MAX = 144;   // words of a warp-per-event record (g g -> t tbar g g: 134; recycled: 144)
constexpr int LH_TPB = 256;             // threads per CTA of the warp-per-event schedule

// The warp-per-event schedules (template argument LH of the heavy integrand): 1, the
// Feynman-diagram helicity body with one lane per configuration (schedule 3); 2, the
// helicity-recycled recursion of mf_rc.cuh (schedule 4), for the matrix elements that
// specialise RcTraits there: warp_bytes(), the shared memory of one warp's store, and
// extra_bytes(tpb), the tables of a CTA of tpb threads after the warps' regions.
template <class ME> struct RcTraits;
template <class ME> struct HasRc : std::false_type {};

struct EwParams { double e2, sw2, cw2, mz, wz; };

struct KParams {
    double sqrt_s, S, ln_tau0, mt, gs, vol_const;   // vol_const * shat^(n-2) = massless n-body volume
    double pt_min2, sinh_eta, dr_min2;              // <= 0 disables
    EwParams ew;
    uint2 key;
    uint32_t channel, iteration;
    int nb;
    long long n_events, ev_offset;
    double inv_n;
    PdfGeom pdfg;
    const double* grid;     // [D][nb+1]
    const double* pdf;      // [3][nx][nq]
    double ln_muf2_fixed;   // ln m_t^2, the fixed 2 -> 2 factorisation scale
    double* partials;       // [gridDim.x][2 + D nb]
    unsigned long long* counters;   // [0] events passing cuts, [1] non-finite weights zeroed
    unsigned* dev_err;      // raised when a bounded device wait runs out (nullable)
    // global storage of queued events' kinematics for heavy processes whose shared
    // memory has no room for it (nullable): kin_ctas regions of [NEXT_MAX 4 + 1]
    // [KIN_CAP_UNIT] doubles and [D_MAX][KIN_CAP_UNIT] bins; a CTA whose ring holds
    // u KIN_CAP_UNIT entries uses regions u b .. u b + u - 1 as one (CTA b)
    double* kin;
    uint8_t* kin_bins;
    int kin_ctas;
    const uint8_t* mask_in; // frozen cut masks (nullable)
    // helicity-independent records of the warp-per-event schedule (nullable): inv_ctas
    // regions of [LH_INV_WORDS_MAX][256] floats, field-major, one region per CTA
    float* inv_rec;
    int inv_ctas;
    // observable histogram (nobs = 0: off): transverse momentum of the first final-state
    // particle in nobs uniform bins from obs_lo, obs_inv_w = nobs / (hi - lo); per CTA
    // (blockIdx.x) a row of [nobs + 2][2] sums (sum w/N, sum (w/N)^2; bin 0 underflow,
    // nobs + 1 overflow) in obs_partials
    int nobs;
    double obs_lo, obs_inv_w;
    double* obs_partials;
    // per-event outputs (nullable).  ev_out != 0 asks every integrand kernel to write the
    // non-null ones: the kernels that a pass without outputs runs write them as well (a
    // run-time branch per event, outside the helicity body), so that the kernel a
    // benchmark times is the kernel whose events a parity test reads
    double* ev_u; double* ev_x; uint8_t* ev_bins; double* ev_w; uint8_t* ev_mask; double* ev_me2; double* ev_p;
    int ev_out;
    // helicity sampling of the warp-level matrix elements (0: the full helicity sum): configurations
    // per event, drawn from a Philox stream of its own (counter block 0xFF, key offset by hel_stream)
    int hel_samples;
    uint32_t hel_stream;
    // the mixed-precision path's kinematics in double-float: the constants above as double-floats
    // (fill_kin_df) and the PDF grid's double-float copy (nullable: then converted per node)
    KinDf kd;
    const Df* pdf_df;
};

// the four random words of an event's helicity draws: counter (event lo, event hi, iteration,
// channel << 8 | 0xFF), a block no VEGAS dimension uses, under the seed key offset by the stream
__device__ __forceinline__ uint4 helicity_draw_words(const KParams& kp, unsigned long long ev)
{
    const uint4 c = make_uint4((uint32_t)ev, (uint32_t)(ev >> 32), kp.iteration, (kp.channel << 8) | 0xFFu);
    return philox4x32_10(c, make_uint2(kp.key.x ^ 0x68656C69u ^ kp.hel_stream, kp.key.y));
}

// Observable bin of an event: 0 below obs_lo (and for a non-finite p_T), nobs + 1 at or
// above the upper edge, else 1 + floor((p_T - obs_lo) obs_inv_w).  p_T of particle 2
// (the first final-state particle; the top quark in the top-pair processes), in FP64.
__device__ __forceinline__ int obs_bin(const KParams& kp, double px, double py)
{
    const double pt = sqrt(px * px + py * py);
    if (!(pt >= kp.obs_lo)) return 0;
    const double t = (pt - kp.obs_lo) * kp.obs_inv_w;
    if (!(t < (double)kp.nobs)) return kp.nobs + 1;
    return 1 + (int)t;
}

// ------------------------------------------------------------------ e+ e- -> mu+ mu-

// Photon and Z exchange between chirality-split currents (massless
// fermions): M = -i e^2 sum_ij A_ij(s)/s J^e_i . J^mu_j with
// A_ij = Q_e Q_mu + g_i g_j s / (sW^2 cW^2 (s - MZ^2 + i MZ GZ)).
struct MeEeMumu {
    static constexpr int NEXT = 4, NHEL = 16;
    template <typename R>
    __device__ static double me2(const double (&p)[4][4], const EwParams& ew)
    {
        const double s = 2.0 * mdot(p[0], p[1]);
        const double gL = -0.5 + ew.sw2, gR = ew.sw2;     // T3 - Q sW^2, -Q sW^2 with Q = -1
        const double dre = s - ew.mz * ew.mz, dim = ew.mz * ew.wz;
        const double dd = dre * dre + dim * dim;
        const double chr = s * dre / dd / (ew.sw2 * ew.cw2), chi = -s * dim / dd / (ew.sw2 * ew.cw2);
        const double g[2] = { gL, gR };
        cx<R> A[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                A[i][j] = mkc(R(ew.e2 / s * (1.0 + g[i] * g[j] * chr)), R(ew.e2 / s * g[i] * g[j] * chi));
        const FermionBasis<R> f1 = fermion_basis<R>(p[0], 0.0), f2 = fermion_basis<R>(p[1], 0.0);
        const FermionBasis<R> f3 = fermion_basis<R>(p[2], 0.0), f4 = fermion_basis<R>(p[3], 0.0);
        R acc = R(0);
        // helicity filtering: the massless e- e+ (and mu- mu+) annihilate into (come from) a
        // vector current only with opposite helicity bits, 4 of the 16 configurations
#pragma unroll 1
        for (int j = 0; j < NHEL_NZ; ++j) acc += hel<R>(hel_nz(j), A, f1, f2, f3, f4);
        return 0.25 * double(acc);
    }
    static constexpr int NHEL_NZ = 4;
    __host__ __device__ static constexpr int hel_nz(int j)
    {
        return (j & 1) | ((~j & 1) << 1) | (((j >> 1) & 1) << 2) | ((~(j >> 1) & 1) << 3);
    }
    // one helicity configuration (ih bit i: helicity of particle i, set = +1), unaveraged
    template <typename R>
    __device__ static R hel(int ih, const cx<R> (&A)[2][2], const FermionBasis<R>& f1, const FermionBasis<R>& f2,
                            const FermionBasis<R>& f3, const FermionBasis<R>& f4)
    {
        const int h1 = (ih & 1) ? 1 : -1, h2 = (ih & 2) ? 1 : -1, h3 = (ih & 4) ? 1 : -1, h4 = (ih & 8) ? 1 : -1;
        W4<R> eL, eR, mL, mR;
        ffv_cur_lr(ext_vbar(f2, h2), ext_u(f1, h1), eL, eR);
        ffv_cur_lr(ext_ubar(f3, h3), ext_v(f4, h4), mL, mR);
        cx<R> amp = cmul(A[0][0], cdot(eL, mL));
        amp = cfma(A[0][1], cdot(eL, mR), amp);
        amp = cfma(A[1][0], cdot(eR, mL), amp);
        amp = cfma(A[1][1], cdot(eR, mR), amp);
        return amp.r * amp.r + amp.i * amp.i;
    }
    // averaged |M_h|^2 of all 16 configurations (diagnostic; the filtered ones come out zero)
    template <typename R>
    __device__ static void hel_profile(const double (&p)[4][4], const EwParams& ew, double* out)
    {
        const double s = 2.0 * mdot(p[0], p[1]);
        const double gL = -0.5 + ew.sw2, gR = ew.sw2;
        const double dre = s - ew.mz * ew.mz, dim = ew.mz * ew.wz;
        const double dd = dre * dre + dim * dim;
        const double chr = s * dre / dd / (ew.sw2 * ew.cw2), chi = -s * dim / dd / (ew.sw2 * ew.cw2);
        const double g[2] = { gL, gR };
        cx<R> A[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                A[i][j] = mkc(R(ew.e2 / s * (1.0 + g[i] * g[j] * chr)), R(ew.e2 / s * g[i] * g[j] * chi));
        const FermionBasis<R> f1 = fermion_basis<R>(p[0], 0.0), f2 = fermion_basis<R>(p[1], 0.0);
        const FermionBasis<R> f3 = fermion_basis<R>(p[2], 0.0), f4 = fermion_basis<R>(p[3], 0.0);
        for (int ih = 0; ih < NHEL; ++ih) out[ih] = 0.25 * double(hel<R>(ih, A, f1, f2, f3, f4));
    }
};

// ------------------------------------------------------------------ process traits

// matrix elements evaluated by a whole warp per event (the Berends-Giele recursion of
// mf_bg.cuh) declare BG = true
template <class ME, class = void> struct MeIsBg : std::false_type {};
template <class ME> struct MeIsBg<ME, std::void_t<decltype(ME::BG)>> : std::bool_constant<ME::BG> {};

struct ProcEe {
    static constexpr int NEXT = 4, NF = 2, D = 2, NPDF = 0;
    static constexpr bool HEAVY = false;
    static constexpr bool BG = false;
    static constexpr bool TC = false;
    static constexpr bool STORE_KIN = false;
    template <typename R> static constexpr size_t slot_bytes() { return 0; }
};

// F1, F2: PDF flavours of the two incoming partons (0 gluon, 1 u, 2 ubar)
template <class ME, int F1 = 0, int F2 = 0>
struct ProcTops {
    using Me = ME;
    static constexpr int NEXT = ME::NEXT;
    static constexpr int NF = NEXT - 2;        // t, tbar, light partons
    static constexpr int D = 2 + 4 * NF;
    static constexpr int NLIGHT = NF - 2;
    static constexpr int NPDF = 1;             // PDFs are read from the global grid (through L1)
    static constexpr int FLAV1 = F1, FLAV2 = F2;
    // warp-level matrix element (one warp per event, state in the warp's shared memory)
    static constexpr bool BG = MeIsBg<ME>::value;
    // heavy matrix elements (2 -> 3 and more with a per-thread invariant slot, or warp-level):
    // queue of the events that pass the cuts, one CTA-level histogram, shared-memory slots
    static constexpr bool HEAVY = NEXT >= 5 && (ME::template slot_bytes<float>() > 0 || BG);
    // the colour sum can run on the tensor cores (heavy processes with a 24-flow basis)
    static constexpr bool TC = HEAVY && ME::TC_COLOUR;
    // the kinematics of queued events are kept in shared memory (where it fits: 2 -> 3),
    // so that the matrix-element batch does not recompute them in FP64
    static constexpr bool STORE_KIN = HEAVY && NEXT == 5;
    template <typename R> static constexpr size_t slot_bytes() { return HEAVY ? ME::template slot_bytes<R>() : 0; }
};

// per-event result
template <int D>
struct EventOut {
    double u[D], x[D];
    uint8_t bins[D];
    double w, me2;
    int mask;
};

// ------------------------------------------------------------------ one event

template <typename R>
__device__ __forceinline__ void event_ee(const KParams& kp, const double* sgrid, unsigned long long ev,
                                         EventOut<2>& o, double (&p)[4][4])
{
    event_uniforms<2>(ev, kp.iteration, kp.channel, kp.key, o.u);
    const double jv = vegas_map<2>(sgrid, kp.nb, o.u, o.x, o.bins);
    const double E = 0.5 * kp.sqrt_s;
    const double c = 2.0 * o.x[0] - 1.0, sn = sqrt(1.0 - c * c);
    double sf, cf;
    sincospi(2.0 * o.x[1], &sf, &cf);
    const double pp[4][4] = { { E, 0, 0, E }, { E, 0, 0, -E }, { E, E * sn * cf, E * sn * sf, E * c },
                              { E, -E * sn * cf, -E * sn * sf, -E * c } };
    for (int i = 0; i < 4; ++i)
        for (int m = 0; m < 4; ++m) p[i][m] = pp[i][m];
    o.mask = kp.mask_in ? kp.mask_in[ev - kp.ev_offset] : 1;
    o.me2 = o.mask ? MeEeMumu::me2<R>(p, kp.ew) : 0.0;
    const double s = kp.S;
    o.w = o.mask ? o.me2 / (2.0 * s) * (1.0 / (8.0 * 3.14159265358979323846)) * jv * GEV2_TO_PB : 0.0;
}

// light-parton cuts in the lab frame: pT > pt_min, |pz| < pT sinh(eta_max),
// and Delta R between the two final gluons
template <class P>
__device__ __forceinline__ int cuts_tops(const KParams& kp, const double (&pl)[P::NEXT][4])
{
    int ok = 1;
    const double sh2 = kp.sinh_eta * kp.sinh_eta;
#pragma unroll
    for (int j = 0; j < P::NLIGHT; ++j) {
        const double* q = pl[4 + j];
        const double pt2 = q[1] * q[1] + q[2] * q[2];
        if (kp.pt_min2 > 0.0) ok &= (pt2 > kp.pt_min2);
        // |eta| < eta_max  <=>  p_z^2 < p_T^2 sinh^2(eta_max)
        if (kp.sinh_eta > 0.0) ok &= (q[3] * q[3] < pt2 * sh2);
    }
    // Delta R between every pair of final gluons (gluon processes with two or more)
    if (P::NLIGHT >= 2 && kp.dr_min2 > 0.0 && ok) {
#pragma unroll
        for (int ia = 0; ia < P::NLIGHT; ++ia)
#pragma unroll
            for (int ib = ia + 1; ib < P::NLIGHT; ++ib) {
                const double* a = pl[4 + ia];
                const double* b = pl[4 + ib];
                const double pta2 = a[1] * a[1] + a[2] * a[2], ptb2 = b[1] * b[1] + b[2] * b[2];
                const double pa = sqrt(pta2 + a[3] * a[3]), pb = sqrt(ptb2 + b[3] * b[3]);
                // eta = ln((|p| + p_z) / p_T), so eta_a - eta_b in one logarithm (|p| + p_z formed
                // as p_T^2 / (|p| - p_z) for p_z < 0, without cancellation); the azimuthal
                // difference in (-pi, pi] from one atan2 of the transverse cross and dot products
                const double ua = a[3] >= 0.0 ? pa + a[3] : pta2 / (pa - a[3]);
                const double ub = b[3] >= 0.0 ? pb + b[3] : ptb2 / (pb - b[3]);
                const double deta = log(ua * sqrt(ptb2) / (ub * sqrt(pta2)));
                const double dphi = atan2(a[1] * b[2] - a[2] * b[1], a[1] * b[1] + a[2] * b[2]);
                ok &= (deta * deta + dphi * dphi > kp.dr_min2);
            }
    }
    return ok;
}

// Everything of one event except the matrix element: uniforms, VEGAS map,
// parton map, RAMBO, lab boost, cuts, scale and PDFs.  pref receives the
// weight factor that multiplies |M|^2: f1 f2 / (2 shat) W J_parton J_VEGAS
// in pb GeV^2.  S is double, or Dual<double> carrying d/d m_t (then the cut
// decisions are taken on the values, i.e. at the base point).
template <class P, typename S>
__device__ __forceinline__ void kinematics_tops_t(const KParams& kp, const double* sgrid, const double* spdf,
                                                  unsigned long long ev, S mt, EventOut<P::D>& o,
                                                  S (&p)[P::NEXT][4], S& pref)
{
    constexpr int NF = P::NF, D = P::D;
    event_uniforms<D>(ev, kp.iteration, kp.channel, kp.key, o.u);
    const double jv = vegas_map<D>(sgrid, kp.nb, o.u, o.x, o.bins);
    S ln_tau0;
    if constexpr (is_dual<S>::value) ln_tau0 = log(4.0 * mt * mt / kp.S);
    else ln_tau0 = kp.ln_tau0;
    S tau, jp, lx1, lx2;
    parton_map(o.x[0], o.x[1], ln_tau0, tau, jp, lx1, lx2);
    const S shat = tau * kp.S;
    const S rs = sqrt(shat);
    S m[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) m[i] = i < 2 ? mt : S(0.0);
    S pf[NF][4];
    S vol = S(kp.vol_const);
#pragma unroll
    for (int i = 0; i < NF - 2; ++i) vol = vol * shat;
    const S wps = rambo<NF>(rs, m, o.x + 2, pf, vol);
    const S h = 0.5 * rs;
    p[0][0] = h; p[0][1] = S(0.0); p[0][2] = S(0.0); p[0][3] = h;
    p[1][0] = h; p[1][1] = S(0.0); p[1][2] = S(0.0); p[1][3] = -h;
#pragma unroll
    for (int i = 0; i < NF; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[2 + i][c] = pf[i][c];
    // longitudinal boost to the lab frame, rapidity y = ln(x1/x2)/2 (values only: it feeds the cuts)
    const double ey = exp(0.5 * (val(lx1) - val(lx2))), iey = 1.0 / ey;
    const double ch = 0.5 * (ey + iey), sh = 0.5 * (ey - iey);
    double pl[P::NEXT][4];
#pragma unroll
    for (int i = 0; i < P::NEXT; ++i) {
        pl[i][0] = ch * val(p[i][0]) + sh * val(p[i][3]);
        pl[i][1] = val(p[i][1]);
        pl[i][2] = val(p[i][2]);
        pl[i][3] = ch * val(p[i][3]) + sh * val(p[i][0]);
    }
    o.mask = kp.mask_in ? (int)kp.mask_in[ev - kp.ev_offset] : cuts_tops<P>(kp, pl);
    if (val(wps) <= 0.0) o.mask = 0;
    // factorisation scale: m_t for 2 -> 2, H_T / 2 otherwise (as ln mu_F^2)
    S lq;
    if constexpr (NF == 2) {
        if constexpr (is_dual<S>::value) lq = log(mt * mt);
        else lq = kp.ln_muf2_fixed;
    } else {
        S ht = S(0.0);
#pragma unroll
        for (int i = 2; i < P::NEXT; ++i) {
            const S mi = (i < 4) ? mt : S(0.0);
            ht = ht + sqrt(mi * mi + p[i][1] * p[i][1] + p[i][2] * p[i][2]);
        }
        lq = log(0.25 * ht * ht);
    }
    const int npv = kp.pdfg.nx * kp.pdfg.nq;
    // f1 f2 / (2 shat) with f = (x f) / x: one division, by 2 shat x1 x2
    const S xf1 = pdf_xf_log(spdf + P::FLAV1 * npv, kp.pdfg, lx1, lq);
    const S xf2 = pdf_xf_log(spdf + P::FLAV2 * npv, kp.pdfg, lx2, lq);
    pref = xf1 * xf2 / (2.0 * shat * tau) * wps * jp * jv * GEV2_TO_PB;
    o.me2 = 0.0;
    o.w = 0.0;
}

template <class P>
__device__ __forceinline__ void kinematics_tops(const KParams& kp, const double* sgrid, const double* spdf,
                                                unsigned long long ev, EventOut<P::D>& o, double (&p)[P::NEXT][4],
                                                double& pref)
{
    kinematics_tops_t<P, double>(kp, sgrid, spdf, ev, kp.mt, o, p, pref);
}

// The same kinematics in double-float (the mixed-precision path).  The VEGAS bins, the cut
// decisions and the PDF cells are those of the FP64 kinematics (bins exactly; the cuts on the
// lab-frame light-parton momenta converted to FP64); the momenta and the weight factor carry
// about 48 bits.  outs: also the FP64 uniforms and mapped points of the per-event outputs.
// sgdf: the VEGAS grid [D][nb+1] in double-float (null: sgrid's edges are converted).
template <class P>
__device__ __forceinline__ void kinematics_tops_df(const KParams& kp, const double* sgrid, const Df* sgdf,
                                                   unsigned long long ev, EventOut<P::D>& o, Df (&p)[P::NEXT][4],
                                                   Df& pref, bool outs)
{
    constexpr int NF = P::NF, D = P::D;
    const KinDf& K = kp.kd;
    unsigned long long kw[D];
    event_words<D>(ev, kp.iteration, kp.channel, kp.key, kw);
    Df x[D];
    const Df jv = vegas_map_df<D>(sgdf, sgrid, kp.nb, kw, x, o.bins);
    if (outs) {
        uint8_t b64[D];
        event_uniforms<D>(ev, kp.iteration, kp.channel, kp.key, o.u);
        (void)vegas_map<D>(sgrid, kp.nb, o.u, o.x, b64);
    }
    // parton map: tau = tau0^x0, ln x1 = x1' ln tau, ln x2 = (1 - x1') ln tau
    const Df lt = x[0] * K.ln_tau0;
    const Df lx1 = x[1] * lt, lx2 = df_add(-x[1], 1.0f) * lt;
    const Df tau = exp(lt);
    const Df jp = tau * (-lt) * (-K.ln_tau0);
    const Df shat = tau * K.S;
    const Df rs = sqrt(shat);
    Df vol = K.vol_const;
#pragma unroll
    for (int i = 0; i < NF - 2; ++i) vol = vol * shat;
    Df pf[NF][4];
    const Df wps = rambo_df<NF>(rs, K.mt, x + 2, pf, vol);
    const Df h = df_scale(rs, 0.5f), z(0.0f, 0.0f);
    p[0][0] = h; p[0][1] = z; p[0][2] = z; p[0][3] = h;
    p[1][0] = h; p[1][1] = z; p[1][2] = z; p[1][3] = -h;
#pragma unroll
    for (int i = 0; i < NF; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[2 + i][c] = pf[i][c];
    // the light partons in the lab frame (rapidity ln(x1/x2)/2), as doubles for the cuts
    double pl[P::NEXT][4];
#pragma unroll
    for (int i = 0; i < P::NEXT; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) pl[i][c] = 0.0;
    if constexpr (P::NLIGHT > 0) {
        const Df ey = exp(df_scale(lx1 - lx2, 0.5f)), iey = df_div(Df(1.0f, 0.0f), ey);
        const Df ch = df_scale(ey + iey, 0.5f), sh = df_scale(ey - iey, 0.5f);
#pragma unroll
        for (int i = 4; i < P::NEXT; ++i) {
            pl[i][0] = (double)(ch * p[i][0] + sh * p[i][3]);
            pl[i][1] = (double)p[i][1];
            pl[i][2] = (double)p[i][2];
            pl[i][3] = (double)(ch * p[i][3] + sh * p[i][0]);
        }
    }
    o.mask = kp.mask_in ? (int)kp.mask_in[ev - kp.ev_offset] : cuts_tops<P>(kp, pl);
    if (wps.hi <= 0.0f) o.mask = 0;
    // factorisation scale: m_t for 2 -> 2, H_T / 2 otherwise (as ln mu_F^2)
    Df lq;
    if constexpr (NF == 2) {
        lq = K.ln_muf2_fixed;
    } else {
        const Df mt2 = K.mt * K.mt;
        Df ht(0.0f, 0.0f);
#pragma unroll
        for (int i = 2; i < P::NEXT; ++i) {
            const Df pt2 = p[i][1] * p[i][1] + p[i][2] * p[i][2];
            ht = ht + sqrt(i < 4 ? mt2 + pt2 : pt2);
        }
        lq = log(df_scale(ht * ht, 0.25f));
    }
    const int npv = kp.pdfg.nx * kp.pdfg.nq;
    const Df* gdf = kp.pdf_df;
    const Df xf1 = pdf_xf_df(kp.pdf + P::FLAV1 * npv, gdf ? gdf + P::FLAV1 * npv : nullptr, kp.pdfg, K, lx1, lq);
    const Df xf2 = pdf_xf_df(kp.pdf + P::FLAV2 * npv, gdf ? gdf + P::FLAV2 * npv : nullptr, kp.pdfg, K, lx2, lq);
    // the PDFs enter last and apart, so that two small ones do not meet in a product below
    // the double-float range
    pref = wps * jp * jv * GEV2_TO_PB / (df_scale(shat, 2.0f) * tau) * xf1 * xf2;
    o.me2 = 0.0;
    o.w = 0.0;
}

// the same, out of line: the heavy processes' kernels call it, so that its register demand
// does not shape the allocation of their matrix-element loops (inlined, it left spills there)
template <class P>
__device__ __noinline__ void kinematics_tops_df_call(const KParams& kp, const double* sgrid, const Df* sgdf,
                                                     unsigned long long ev, EventOut<P::D>& o, Df (&p)[P::NEXT][4],
                                                     Df& pref, bool outs)
{
    kinematics_tops_df<P>(kp, sgrid, sgdf, ev, o, p, pref, outs);
}

// One event's kinematics in the arithmetic of its path: FP64 for the FP64 matrix elements,
// double-float for the mixed-precision ones.  M: the type of the momenta handed on (double, or
// Df for a matrix element that takes double-float momenta).  sgdf: the double-float VEGAS grid
// (mixed precision; null where the kernel keeps none).  outs: the per-event outputs' uniforms and points are wanted.
template <class P, typename R, typename M>
__device__ __forceinline__ void kinematics_path(const KParams& kp, const double* sgrid, const Df* sgdf,
                                                unsigned long long ev, EventOut<P::D>& o, M (&p)[P::NEXT][4],
                                                double& pref, bool outs)
{
    if constexpr (sizeof(R) == 4) {
        Df pd[P::NEXT][4], pr;
        if constexpr (P::HEAVY) kinematics_tops_df_call<P>(kp, sgrid, sgdf, ev, o, pd, pr, outs);
        else kinematics_tops_df<P>(kp, sgrid, sgdf, ev, o, pd, pr, outs);
        pref = (double)pr;
#pragma unroll
        for (int i = 0; i < P::NEXT; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) p[i][c] = M(pd[i][c]);
    } else {
        static_assert(std::is_same<M, double>::value, "the FP64 path hands on FP64 momenta");
        kinematics_tops<P>(kp, sgrid, kp.pdf, ev, o, p, pref);
    }
}

template <class P, typename R>
__device__ __forceinline__ void event_tops(const KParams& kp, const double* sgrid, const double* spdf,
                                           unsigned long long ev, EventOut<P::D>& o, double (&p)[P::NEXT][4],
                                           void* slot)
{
    double pref;
    kinematics_tops<P>(kp, sgrid, spdf, ev, o, p, pref);
    // matrix element only for events that pass; the warp skips it when no lane needs it
    if (__any_sync(__activemask(), o.mask)) {
        if (o.mask) o.me2 = P::Me::template me2<R>(p, kp.mt, kp.gs, slot);
    }
    if (o.mask) o.w = pref * o.me2;
}

// ------------------------------------------------------------------ shared-memory layout

// Byte offsets of the kernel's dynamic shared memory:
//   grid [D][nb+1] (FP64, or double-float for the mixed kinematics) | histograms | value buffer |
//   bins buffer (heavy) | event queue and counts (heavy) | block-sum scratch |
//   tensor-core colour-sum state (TC processes) | per-thread slots (heavy)
// Light processes keep one histogram per warp (updated by bin leaders);
// heavy ones keep one per CTA, filled by one thread per dimension in event
// order after every round.
// LH (warp-per-event schedule): dynamic shared memory starts with one colour-flow
// row per thread (2 NCOL + 2 words: 8-byte aligned, and for 8-byte accesses an
// even word stride of 2 mod 32 per half-warp is conflict-free), followed by one
// record per warp (16-byte aligned); both offsets are compile-time constants of the
// helicity body
template <class P, bool LH> struct LhRows { static constexpr int words() { return 0; } };
template <class P> struct LhRows<P, true> { static constexpr int words() { return 2 * P::Me::NCOL + 2; } };
// a warp's region (its record, or with LH = 2 its store) and the CTA's extra bytes after them
template <class P, typename R, int LH, int TPB> struct LhRegion {
    static constexpr size_t stride() { return (P::template slot_bytes<R>() + 15) & ~(size_t)15; }
    static constexpr size_t extra() { return 0; }
};
template <class P, typename R, int TPB> struct LhRegion<P, R, 2, TPB> {
    static constexpr size_t stride() { return (RcTraits<typename P::Me>::warp_bytes() + 15) & ~(size_t)15; }
    static constexpr size_t extra() { return RcTraits<typename P::Me>::extra_bytes(TPB); }
};

template <class P, typename R, int TPB, int LH = 0>
struct SmemLayout {
    static constexpr int WARPS = TPB / 32;
    static constexpr int D = P::D;
    static constexpr int NHIST = P::HEAVY ? 1 : WARPS;
    static constexpr __host__ __device__ size_t al(size_t x) { return (x + 15) & ~(size_t)15; }
    // LH: the rows [TPB][LH_JROW] words (LH = 1; with LH = 2 the rows live in tensor memory),
    // then the warps' regions [WARPS], LH_REC_STRIDE bytes apart, at LH_REC_OFF, then the
    // CTA's extra tables (LH = 2) at LH_EXTRA_OFF
    static constexpr int LH_JROW = LhRows<P, LH == 1>::words();
    static constexpr int LH_REC_OFF = TPB * LH_JROW * (int)sizeof(R);
    static constexpr int LH_REC_STRIDE = LH ? (int)LhRegion<P, R, LH, TPB>::stride() : 0;
    static constexpr int LH_EXTRA_OFF = LH_REC_OFF + WARPS * LH_REC_STRIDE;
    static constexpr size_t lh_bytes()
    {
        return LH ? al((size_t)LH_EXTRA_OFF + LhRegion<P, R, LH, TPB>::extra()) : 0;
    }
    // warp-level matrix elements: the colour matrix and one state per warp at the start
    static constexpr __host__ __device__ size_t bg_bytes()
    {
        if constexpr (P::BG) return al(P::Me::template cta_bytes<R>(WARPS));
        else return 0;
    }
    static __host__ __device__ size_t grid_off() { return lh_bytes() + bg_bytes(); }
    // the mixed-precision kinematics keep the grid in double-float in the FP64 grid's place (8
    // bytes an edge either way: the recycled kernel's shared memory stays below the 196 KB
    // carveout step, which leaves L1 60 KB instead of 28); their per-event outputs read the FP64
    // edges from global memory
    static constexpr bool GDF = sizeof(R) == 4 && P::NPDF > 0;
    static __host__ __device__ size_t gdf_off(int nb) { return grid_off(); }
    static __host__ __device__ size_t pdf_off(int nb) { return al(grid_off() + sizeof(double) * D * (nb + 1)); }
    static __host__ __device__ size_t hist_off(int nb, int npv) { return al(pdf_off(nb)); }
    static __host__ __device__ size_t vbuf_off(int nb, int npv) { return al(hist_off(nb, npv) + sizeof(double) * NHIST * D * nb); }
    static __host__ __device__ size_t bbuf_off(int nb, int npv) { return al(vbuf_off(nb, npv) + sizeof(double) * TPB); }
    static __host__ __device__ size_t queue_off(int nb, int npv) { return al(bbuf_off(nb, npv) + (P::HEAVY ? (size_t)TPB * D : 0)); }
    // ring of 2 TPB queued events; with KIN their momenta [NEXT 4][2 TPB],
    // weight factors [2 TPB] and bins [2 TPB][D] follow
    static constexpr int CAP = 2 * TPB;
    static constexpr bool KIN = P::STORE_KIN && sizeof(R) == 4;   // mixed precision only
    static __host__ __device__ size_t kin_off(int nb, int npv)
    {
        return al(queue_off(nb, npv) + (P::HEAVY ? sizeof(int) * CAP + sizeof(int) * (WARPS + 2) : 0));
    }
    static __host__ __device__ size_t kin_bytes()
    {
        return KIN ? sizeof(double) * (P::NEXT * 4 + 1) * CAP + (size_t)D * CAP : 0;
    }
    static __host__ __device__ size_t red_off(int nb, int npv) { return al(kin_off(nb, npv) + kin_bytes()); }
    static __host__ __device__ size_t tc_off(int nb, int npv)
    {
        return (red_off(nb, npv) + sizeof(double) * 2 * WARPS + 127) & ~(size_t)127;
    }
    static __host__ __device__ size_t slot_off(int nb, int npv)
    {
        return al(P::TC ? tc_off(nb, npv) + sizeof(TcCta) : red_off(nb, npv) + sizeof(double) * 2 * WARPS);
    }
    // observable histograms [NHIST][MAX_OBS_BINS + 2][2], then per-thread w/N and (heavy) bin buffers
    static constexpr size_t OBS_ROW = 2 * (MAX_OBS_BINS + 2);
    static __host__ __device__ size_t slot_region() { return LH ? 0 : (size_t)TPB * P::template slot_bytes<R>(); }
    static __host__ __device__ size_t obs_off(int nb, int npv) { return al(slot_off(nb, npv) + slot_region()); }
    static __host__ __device__ size_t obs_w_off(int nb, int npv) { return obs_off(nb, npv) + sizeof(double) * NHIST * OBS_ROW; }
    static __host__ __device__ size_t obs_b_off(int nb, int npv) { return obs_w_off(nb, npv) + sizeof(double) * TPB; }
    // obs: with the observable region (kernels touch it only when kp.nobs > 0)
    static __host__ __device__ size_t bytes(int nb, int npv, bool obs = false)
    {
        return obs ? al(obs_b_off(nb, npv) + sizeof(int16_t) * TPB) : obs_off(nb, npv);
    }
};

// end of the kernel: two sums per CTA (warp trees, then warps in order), the
// CTA histogram(s) summed in warp order, written to this CTA's partials
template <class P, int TPB, int NHIST>
__device__ __forceinline__ void write_partials(const KParams& kp, double sw, double sw2, unsigned long long npass,
                                               unsigned long long nnan, double* sred, const double* shist, double* out)
{
    constexpr int D = P::D, WARPS = TPB / 32;
    const int nb = kp.nb, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sw += __shfl_down_sync(0xffffffffu, sw, off);
        sw2 += __shfl_down_sync(0xffffffffu, sw2, off);
    }
    if (lane == 0) { sred[2 * warp] = sw; sred[2 * warp + 1] = sw2; }
    // counters: integer sums are order independent
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        npass += __shfl_down_sync(0xffffffffu, npass, off);
        nnan += __shfl_down_sync(0xffffffffu, nnan, off);
    }
    if (lane == 0 && (npass || nnan)) {
        atomicAdd(kp.counters + 0, npass);
        atomicAdd(kp.counters + 1, nnan);
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < WARPS; ++w) { a += sred[2 * w]; b += sred[2 * w + 1]; }
        out[0] = a; out[1] = b;
    }
    for (int i = tid; i < D * nb; i += TPB) {
        double s = 0.0;
        for (int w = 0; w < NHIST; ++w) s += shist[w * D * nb + i];
        out[2 + i] = s;
    }
}

// this CTA's observable row: the NHIST histograms summed in order
template <int NHIST, size_t OBS_ROW>
__device__ __forceinline__ void write_obs_partials(const KParams& kp, const double* sobs)
{
    if (kp.nobs <= 0) return;
    const int n2 = 2 * (kp.nobs + 2);
    double* row = kp.obs_partials + (size_t)blockIdx.x * n2;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < NHIST; ++w) s += sobs[w * OBS_ROW + i];
        row[i] = s;
    }
}

template <int D>
__device__ __forceinline__ void write_event(const KParams& kp, long long e, const EventOut<D>& o, bool kin)
{
    if (kin) {
        for (int d = 0; d < D; ++d) {
            if (kp.ev_u) kp.ev_u[e * D + d] = o.u[d];
            if (kp.ev_x) kp.ev_x[e * D + d] = o.x[d];
            if (kp.ev_bins) kp.ev_bins[e * D + d] = o.bins[d];
        }
        if (kp.ev_mask) kp.ev_mask[e] = (uint8_t)o.mask;
    }
    if (kp.ev_w) kp.ev_w[e] = o.w;
    if (kp.ev_me2) kp.ev_me2[e] = o.me2;
}

template <int NEXT, typename M>
__device__ __forceinline__ void write_momenta(const KParams& kp, long long e, const M (&pm)[NEXT][4])
{
    if (kp.ev_p)
        for (int i = 0; i < NEXT; ++i)
            for (int c = 0; c < 4; ++c) kp.ev_p[(e * NEXT + i) * 4 + c] = (double)pm[i][c];
}

// the VEGAS grid into shared memory (every thread of the CTA calls; the caller synchronises):
// its FP64 edges, or for the mixed-precision kinematics their double-float values
template <class L>
__device__ __forceinline__ void stage_grid(const KParams& kp, unsigned char* smem_raw, double* sgrid)
{
    const int n = L::D * (kp.nb + 1);
    if constexpr (L::GDF) {
        Df* sgdf = reinterpret_cast<Df*>(smem_raw + L::gdf_off(kp.nb));
        for (int i = threadIdx.x; i < n; i += blockDim.x) sgdf[i] = Df(kp.grid[i]);
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sgrid[i] = kp.grid[i];
    }
}
template <class L> __device__ __forceinline__ const Df* grid_df(const KParams& kp, const unsigned char* smem_raw)
{
    return L::GDF ? reinterpret_cast<const Df*>(smem_raw + L::gdf_off(kp.nb)) : nullptr;
}
// the FP64 edges the kinematics read: shared memory, or global memory where the shared copy is
// double-float (only the per-event outputs read them then)
template <class L> __device__ __forceinline__ const double* grid_fp64(const KParams& kp, const double* sgrid)
{
    return L::GDF ? kp.grid : sgrid;
}

// queued events' momenta: FP64 words, or a double-float's two floats in one 8-byte word
__device__ __forceinline__ void kin_st(double* a, int i, double v) { a[i] = v; }
__device__ __forceinline__ void kin_st(double* a, int i, const Df& v) { reinterpret_cast<Df*>(a)[i] = v; }
__device__ __forceinline__ void kin_ld(const double* a, int i, double& v) { v = a[i]; }
__device__ __forceinline__ void kin_ld(const double* a, int i, Df& v) { v = reinterpret_cast<const Df*>(a)[i]; }
// the top mass and the strong coupling in the scalar K of the momenta (double or Df)
template <typename K> __device__ __forceinline__ K kin_mt(const KParams& kp)
{
    if constexpr (std::is_same<K, Df>::value) return kp.kd.mt;
    else return kp.mt;
}
template <typename K> __device__ __forceinline__ K kin_gs(const KParams& kp)
{
    if constexpr (std::is_same<K, Df>::value) return kp.kd.gs;
    else return kp.gs;
}

// Light processes (cheap matrix elements): one event per thread per round,
// per-warp histograms updated by bin leaders.
// Events first + r * step + tid (r = 0, 1, ...) below end; the CTA's sums go to out.
template <class P, typename R, int TPB, bool WRITE>
__device__ __forceinline__ void integrand_light(const KParams& kp, unsigned char* smem_raw, long long first,
                                                long long step, long long end, double* out)
{
    constexpr int D = P::D;
    using L = SmemLayout<P, R, TPB>;
    const int nb = kp.nb;
    const int npv = kp.pdfg.nx * kp.pdfg.nq;
    double* sgrid = reinterpret_cast<double*>(smem_raw + L::grid_off());
    double* shist = reinterpret_cast<double*>(smem_raw + L::hist_off(nb, npv));
    double* svbuf = reinterpret_cast<double*>(smem_raw + L::vbuf_off(nb, npv));
    double* sred = reinterpret_cast<double*>(smem_raw + L::red_off(nb, npv));
    double* sobs = reinterpret_cast<double*>(smem_raw + L::obs_off(nb, npv));
    double* swbuf = reinterpret_cast<double*>(smem_raw + L::obs_w_off(nb, npv));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool obs = kp.nobs > 0;
    const Df* sgdf = grid_df<L>(kp, smem_raw);

    stage_grid<L>(kp, smem_raw, sgrid);
    for (int i = tid; i < L::NHIST * D * nb; i += TPB) shist[i] = 0.0;
    if (obs)
        for (int i = tid; i < L::NHIST * (int)L::OBS_ROW; i += TPB) sobs[i] = 0.0;
    __syncthreads();

    double* myhist = shist + warp * D * nb;
    double* myobs = sobs + warp * L::OBS_ROW;
    const bool wr = WRITE || kp.ev_out != 0;   // per-event outputs
    double sw = 0.0, sw2 = 0.0;
    unsigned long long npass = 0, nnan = 0;
    // the momenta: double-float from the mixed-precision kinematics, FP64 otherwise
    using KM = std::conditional_t<sizeof(R) == 4 && P::NPDF != 0, Df, double>;
    const long long rounds = end > first ? (end - first + step - 1) / step : 0;
    for (long long r = 0; r < rounds; ++r) {
        const long long e = first + r * step + tid;
        const bool valid = e < end;
        EventOut<D> o;
        KM pm[P::NEXT][4];
        o.w = 0.0; o.me2 = 0.0; o.mask = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) o.bins[d] = 0;
        if (valid) {
            const unsigned long long ev = (unsigned long long)(kp.ev_offset + e);
            if constexpr (P::NPDF == 0) {
                event_ee<R>(kp, sgrid, ev, o, pm);
            } else {
                double pref;
                kinematics_path<P, R>(kp, grid_fp64<L>(kp, sgrid), sgdf, ev, o, pm, pref, wr);
                // the per-event kinematics go out before the matrix element, so that the
                // uniforms and mapped points need not stay live across it (the same kernel
                // serves passes with and without outputs)
                if (wr) { write_event<D>(kp, e, o, true); write_momenta<P::NEXT>(kp, e, pm); }
                // matrix element only for events that pass; the warp skips it when no lane needs it
                if (__any_sync(__activemask(), o.mask)) {
                    if (o.mask) o.me2 = (double)P::Me::template me2<R>(pm, kin_mt<KM>(kp), kin_gs<KM>(kp), nullptr);
                }
                if (o.mask) o.w = pref * o.me2;
            }
            if (!isfinite(o.w)) { o.w = 0.0; ++nnan; }
            npass += o.mask ? 1 : 0;
            if (wr) {
                if constexpr (P::NPDF == 0) { write_event<D>(kp, e, o, true); write_momenta<P::NEXT>(kp, e, pm); }
                else write_event<D>(kp, e, o, false);
            }
        }
        const double wn = o.w * kp.inv_n;
        const double v = wn * wn;
        sw += wn;
        sw2 += v;
        // per-warp histogram: one leader per distinct bin sums its peers in lane order
        svbuf[tid] = v;
        __syncwarp();
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const unsigned peers = __match_any_sync(0xffffffffu, (unsigned)o.bins[d]);
            if (lane == __ffs(peers) - 1) {
                double s = 0.0;
                for (unsigned m = peers; m; m &= m - 1) s += svbuf[warp * 32 + __ffs(m) - 1];
                myhist[d * nb + o.bins[d]] += s;
            }
        }
        if (obs) {
            // observable: the same leader scheme on the event's p_T bin (sum w/N and sum (w/N)^2)
            swbuf[tid] = wn;
            __syncwarp();
            const int ob = valid ? obs_bin(kp, (double)pm[2][1], (double)pm[2][2]) : 0;
            const unsigned peers = __match_any_sync(0xffffffffu, (unsigned)ob);
            if (lane == __ffs(peers) - 1) {
                double s1 = 0.0, s2 = 0.0;
                for (unsigned m = peers; m; m &= m - 1) {
                    const int l = warp * 32 + __ffs(m) - 1;
                    s1 += swbuf[l];
                    s2 += svbuf[l];
                }
                myobs[2 * ob] += s1;
                myobs[2 * ob + 1] += s2;
            }
        }
        __syncwarp();
    }
    write_partials<P, TPB, L::NHIST>(kp, sw, sw2, npass, nnan, sred, shist, out);
    write_obs_partials<L::NHIST, L::OBS_ROW>(kp, sobs);
}

// |M|^2 of the batch's events under the warp-per-event schedule (every thread of
// the CTA calls it; see integrand_heavy).  smem_raw: the kernel's dynamic shared
// memory in the LH layout of SmemLayout, sme: [TPB] doubles of scratch, take:
// events in the batch, mine/pm: this thread's batch entry and its momenta.
// Returns this thread's event's |M|^2 (meaningful where mine).
template <class P, typename R, int TPB>
__device__ __forceinline__ double lh_batch_me2(const KParams& kp, unsigned char* smem_raw, TcCta* tc, double* sme,
                                               int take, bool mine, const double (&pm)[P::NEXT][4])
{
    using ME = typename P::Me;
    using Inv = typename ME::template Inv<R>;
    using L = SmemLayout<P, R, TPB, true>;
    constexpr int WARPS = TPB / 32, NW = ME::INV_WORDS, JROW = L::LH_JROW, REC_OFF = L::LH_REC_OFF;
    constexpr int REC_STRIDE = L::LH_REC_STRIDE;
    static_assert(ME::NHEL / 2 == 32, "one lane per helicity of the parity-halved sum");
    static_assert(NW <= LH_INV_WORDS_MAX && sizeof(R) == 4 && offsetof(Inv, jamp) == NW * sizeof(R),
                  "record layout: the helicity-independent words precede the colour flows");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // this CTA's records, field-major: word f of entry j at grec[f TPB + j]
    float* grec = kp.inv_rec + (size_t)blockIdx.x * LH_INV_WORDS_MAX * TPB;
    if (mine) {
        Inv rec;
        ME::template inv<R>(pm, kp.mt, rec);
        const float* wsrc = reinterpret_cast<const float*>(&rec);
#pragma unroll
        for (int f = 0; f < NW; ++f) grec[f * TPB + tid] = wsrc[f];
    }
    __syncthreads();
    float* wwords = reinterpret_cast<float*>(smem_raw + REC_OFF + (size_t)warp * REC_STRIDE);
    const volatile float* jrow = reinterpret_cast<const volatile float*>(smem_raw) + (size_t)tid * JROW;
    const int nsub = (take + WARPS - 1) / WARPS;
    for (int sub = 0; sub < nsub; ++sub) {
        const int j = sub * WARPS + warp;
        const int jj = j < take ? j : 0;          // a warp without an event repeats entry 0 and discards it
        for (int f = lane; f < NW; f += 32) wwords[f] = grec[f * TPB + jj];
        __syncwarp();
        ME::template hel_j<R, JROW, REC_OFF, REC_STRIDE>(1 + 2 * lane);
        float mh = tc_colour_sum<ME::NCOL>(tc, jrow);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mh += __shfl_xor_sync(0xffffffffu, mh, off);
        if (lane == 0 && j < take) sme[j] = (double)mh;
        __syncwarp();
    }
    __syncthreads();
    const float acc = 2.0f * (float)sme[tid < take ? tid : 0];
    double gk = 1.0;
    for (int i = 0; i < ME::NGLUON; ++i) gk = gk * (kp.gs * kp.gs);
    __syncthreads();   // sme is reused by the caller
    return (double)acc / ME::COLOUR_DEN * gk * ME::AVG * ME::SYM;
}

// |M|^2 of the batch's events for a warp-level matrix element (P::BG; every thread of the
// CTA calls it, see integrand_heavy): the queued events' FP64 momenta go to this CTA's
// region of kp.inv_rec (field-major), then warp w evaluates events w, w + WARPS, ...
// with its shared-memory state.  sme: [TPB] doubles of scratch; returns this thread's
// event's |M|^2 (meaningful where mine).
template <class P, typename R, int TPB>
__device__ __forceinline__ double bg_batch_me2(const KParams& kp, unsigned char* smem_raw, double* sme, int take,
                                               bool mine, const double (&pm)[P::NEXT][4], unsigned long long ev)
{
    using ME = typename P::Me;
    constexpr int WARPS = TPB / 32;
    static_assert((P::NEXT * 4 + 1) * TPB <= LH_INV_WORDS_MAX * LH_TPB / 2, "momenta fit the CTA's record region");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* grec = reinterpret_cast<double*>(kp.inv_rec + (size_t)blockIdx.x * LH_INV_WORDS_MAX * LH_TPB);
    if (mine) {
#pragma unroll
        for (int f = 0; f < P::NEXT * 4; ++f) grec[(size_t)f * TPB + tid] = pm[f >> 2][f & 3];
        grec[(size_t)P::NEXT * 4 * TPB + tid] = __longlong_as_double((long long)ev);   // the event number
    }
    __syncthreads();
    const float* cs = reinterpret_cast<const float*>(smem_raw);
    auto& w = *reinterpret_cast<typename ME::template Warp<R>*>(smem_raw + ME::colour_bytes() +
                                                                (size_t)warp * ME::template warp_bytes<R>());
    for (int j = warp; j < take; j += WARPS) {
        uint4 rnd = make_uint4(0u, 0u, 0u, 0u);
        if (kp.hel_samples > 0)
            rnd = helicity_draw_words(kp, (unsigned long long)__double_as_longlong(grec[(size_t)P::NEXT * 4 * TPB + j]));
        const double v = ME::template warp_me2<R>(w, cs, grec + j, TPB, kp.mt, false, nullptr, 0.0, kp.hel_samples, rnd);
        if (lane == 0) sme[j] = v;
    }
    __syncthreads();
    const double me = sme[tid < take ? tid : 0] * ME::norm(kp.gs);
    __syncthreads();   // sme is reused by the caller
    return me;
}

// the helicity-recycled schedule (LH = 2), defined in mf_rc.cuh: the CTA's set-up after
// tc_setup, and |M|^2 of a batch (as lh_batch_me2; the momenta in double-float)
template <class P, int TPB> __device__ void rc_cta_setup(unsigned char* smem_raw, TcCta* tc);
template <class P, int TPB>
__device__ double rc_batch_me2(const KParams& kp, unsigned char* smem_raw, TcCta* tc, double* sme, int take, bool mine,
                               const Df (&pm)[P::NEXT][4]);

// Heavy processes (expensive matrix elements): kinematics first, then the
// events that pass the cuts are queued in event order and their matrix
// elements are evaluated TPB at a time, so no lane idles through a matrix
// element for an event that the cuts reject.  Every thread of the CTA takes
// part in each batch (the final partial batch repeats the first queued
// event on the idle lanes and discards it), which allows an optional CTA
// barrier between helicities (SYNC) that keeps the warps on the same code.
// The histogram is filled by one thread per dimension in queue order.
// HS: helicity split (HS = 1 or 2).  With 2, thread t and thread t + TPB/2
// share one event and each sums every other helicity; a CTA then takes
// TPB / 2 events per round (step is a multiple of TPB / HS), a batch holds
// TPB / 2 events, and every warp still evaluates one helicity at a time (the
// halves live in different warps, so the helicity stays warp-uniform).
// LH: warp-per-event schedule (tensor-core processes, no per-event outputs).  A
// batch first computes every queued event's helicity-independent pieces, one
// event per thread, into this CTA's region of kp.inv_rec; then warp w takes
// the batch's events w, w + WARPS, ..., copies the event's record into its
// shared-memory record and lane l evaluates helicity 1 + 2 l of the
// parity-halved sum (32 helicities, 32 lanes), with the colour sum of all 256
// rows on the tensor cores and the event's sum over its lanes by a fixed
// shuffle tree.  The per-event record is shared by the warp, so shared memory
// holds 8 records instead of 256 per-thread slots and leaves the rest to L1.
template <class P, typename R, int TPB, bool WRITE, bool SYNC, bool TC = false, int HS = 1, int LH = 0>
__device__ __forceinline__ void integrand_heavy(const KParams& kp, unsigned char* smem_raw, long long first,
                                                long long step, long long end, double* out)
{
    static_assert(HS == 1 || (HS == 2 && SYNC && !WRITE), "helicity split: pairs of lanes, barrier schedule");
    static_assert(!TC || (P::TC && SYNC && (TPB == 128 || TPB == 256) && sizeof(R) == 4),
                  "tensor-core colour sum: float, barrier schedule, one TMEM lane per thread");
    static_assert(!LH || (TC && HS == 1 && !WRITE && (TPB == LH_TPB || (LH == 2 && TPB == 128))),
                  "warp-per-event: tensor cores, no split or outputs");
    constexpr int D = P::D, WARPS = TPB / 32;
    using L = SmemLayout<P, R, TPB, LH>;
    const int nb = kp.nb;
    const int npv = kp.pdfg.nx * kp.pdfg.nq;
    double* sgrid = reinterpret_cast<double*>(smem_raw + L::grid_off());
    double* shist = reinterpret_cast<double*>(smem_raw + L::hist_off(nb, npv));
    double* svbuf = reinterpret_cast<double*>(smem_raw + L::vbuf_off(nb, npv));
    uint8_t* sbins = smem_raw + L::bbuf_off(nb, npv);
    // events per round and per batch
    constexpr int EPB = TPB / HS;
    // ring of queued events as r EPB + tid (event first + r step + tid)
    constexpr int CAP = L::CAP;
    int* squeue = reinterpret_cast<int*>(smem_raw + L::queue_off(nb, npv));
    int* scount = squeue + CAP;                                  // [0] length, [1] head, [2 + w] warp counts
    double* kpm = reinterpret_cast<double*>(smem_raw + L::kin_off(nb, npv));   // [NEXT 4][CAP]
    double* kpref = kpm + P::NEXT * 4 * CAP;                                      // [CAP]
    uint8_t* kbins = reinterpret_cast<uint8_t*>(kpref + CAP);                     // [D][CAP]
    double* sred = reinterpret_cast<double*>(smem_raw + L::red_off(nb, npv));
    double* sobs = reinterpret_cast<double*>(smem_raw + L::obs_off(nb, npv));
    double* swbuf = reinterpret_cast<double*>(smem_raw + L::obs_w_off(nb, npv));
    int16_t* sobin = reinterpret_cast<int16_t*>(smem_raw + L::obs_b_off(nb, npv));
    const bool obs = kp.nobs > 0;
    const bool wr = WRITE || kp.ev_out != 0;   // per-event outputs
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    void* slot = (void*)(smem_raw + L::slot_off(nb, npv) + (size_t)tid * P::template slot_bytes<R>());
    const Df* sgdf = grid_df<L>(kp, smem_raw);
    // the momenta handed to the matrix element: double-float where the mixed-precision matrix
    // element takes them in that arithmetic (the recycled schedule's records, the generated
    // prologues of the per-thread schedules), else FP64
    using KM = std::conditional_t<LH == 2 || (sizeof(R) == 4 && LH == 0 && !P::BG), Df, double>;
    // batches read back the kinematics stored when the events were queued: in shared
    // memory (L::KIN), else for mixed precision in this CTA's global region (kp.kin)
    constexpr bool GKIN = !L::KIN && !WRITE && sizeof(R) == 4 && CAP <= KIN_CAP_UNIT * 2;
    constexpr bool MAYREUSE = (L::KIN && !WRITE) || GKIN;
    bool reuse = L::KIN && !WRITE;
    if constexpr (GKIN) {
        // kp.kin_ctas regions of KIN_CAP_UNIT entries; this CTA takes CAP / KIN_CAP_UNIT of them
        constexpr int UNITS = (CAP + KIN_CAP_UNIT - 1) / KIN_CAP_UNIT;
        if (kp.kin != nullptr && ((int)blockIdx.x + 1) * UNITS <= kp.kin_ctas) {
            reuse = true;
            kpm = kp.kin + (size_t)blockIdx.x * (KIN_NEXT_MAX * 4 + 1) * (UNITS * KIN_CAP_UNIT);
            kpref = kpm + P::NEXT * 4 * CAP;
            kbins = kp.kin_bins + (size_t)blockIdx.x * MAX_DIM * (UNITS * KIN_CAP_UNIT);
        }
    }

    stage_grid<L>(kp, smem_raw, sgrid);
    for (int i = tid; i < D * nb; i += TPB) shist[i] = 0.0;
    if (obs)
        for (int i = tid; i < (int)L::OBS_ROW; i += TPB) sobs[i] = 0.0;
    if (tid == 0) { scount[0] = 0; scount[1] = 0; }
    TcCta* tc = nullptr;
    if constexpr (TC) {
        tc = reinterpret_cast<TcCta*>(smem_raw + L::tc_off(nb, npv));
        if constexpr (LH == 2) {
            // the recursion orders its colour flows differently: its own copy of 54 C
            tc_setup<P::Me::NCOL>(tc, RcTraits<typename P::Me>::colour54(), kp.dev_err, TC_RC_COLS);
            rc_cta_setup<P, TPB>(smem_raw, tc);
        } else {
            tc_setup<P::Me::NCOL>(tc, P::Me::colour54(), kp.dev_err, TC_COLS);
        }
    }
    if constexpr (P::BG) P::Me::load_colour(reinterpret_cast<float*>(smem_raw));
    __syncthreads();

    double sw = 0.0, sw2 = 0.0;
    unsigned long long npass = 0, nnan = 0;
    const long long rounds = end > first ? (end - first + step - 1) / step : 0;
    for (long long r = 0; r <= rounds; ++r) {
        const bool flush = (r == rounds);
        if (!flush) {
            // kinematics of this round's events; queue the ones that pass, in event order
            const long long e = first + r * step + tid;
            int pass = 0;
            EventOut<D> o;
            KM pm[P::NEXT][4];
            double pref = 0.0;
            if (tid < EPB && e < end) {
                kinematics_path<P, R>(kp, grid_fp64<L>(kp, sgrid), sgdf, (unsigned long long)(kp.ev_offset + e), o, pm,
                                      pref, wr);
                pass = o.mask ? 1 : 0;
                npass += pass;
                if (wr) {
                    write_event<D>(kp, e, o, true);
                    if (!pass) write_momenta<P::NEXT>(kp, e, pm);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (lane == 0) scount[2 + warp] = __popc(bal);
            __syncthreads();
            const int cnt = scount[0], head = scount[1];
            int woff = 0, tot = 0;
            for (int w = 0; w < WARPS; ++w) { woff += (w < warp) ? scount[2 + w] : 0; tot += scount[2 + w]; }
            if (pass) {
                const int pos = (head + cnt + woff + __popc(bal & ((1u << lane) - 1u))) % CAP;
                squeue[pos] = (int)r * EPB + tid;
                if (MAYREUSE && reuse) {
#pragma unroll
                    for (int i = 0; i < P::NEXT; ++i)
#pragma unroll
                        for (int c = 0; c < 4; ++c) kin_st(kpm, (i * 4 + c) * CAP + pos, pm[i][c]);
                    kpref[pos] = pref;
#pragma unroll
                    for (int d = 0; d < D; ++d) kbins[d * CAP + pos] = o.bins[d];
                }
            }
            __syncthreads();
            if (tid == 0) scount[0] = cnt + tot;
            __syncthreads();
        }
        // evaluate full batches (and, at the end, whatever is left)
        for (;;) {
            const int cnt = scount[0], head = scount[1];
            if (cnt == 0 || (!flush && cnt < EPB)) break;
            const int take = cnt < EPB ? cnt : EPB;
            const int eidx = tid % EPB, hpart = tid / EPB;
            const bool mine = eidx < take;
            const bool owner = mine && hpart == 0;     // the lane that books the event
            const int pos = (head + (mine ? eidx : 0)) % CAP;
            const int li = squeue[pos];
            const long long e = first + (long long)(li / EPB) * step + (li % EPB);
            EventOut<D> o;
            KM pm[P::NEXT][4];
            double pref;
            if (MAYREUSE && reuse) {
#pragma unroll
                for (int i = 0; i < P::NEXT; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) kin_ld(kpm, (i * 4 + c) * CAP + pos, pm[i][c]);
                pref = kpref[pos];
#pragma unroll
                for (int d = 0; d < D; ++d) o.bins[d] = kbins[d * CAP + pos];
            } else {
                kinematics_path<P, R>(kp, grid_fp64<L>(kp, sgrid), sgdf, (unsigned long long)(kp.ev_offset + e), o, pm,
                                      pref, false);
            }
            double me;
            if constexpr (P::BG) {
                static_assert(HS == 1 && !LH && !TC, "warp-level matrix element: its own schedule");
                me = bg_batch_me2<P, R, TPB>(kp, smem_raw, svbuf, take, mine, pm,
                                             (unsigned long long)(kp.ev_offset + e));
            } else if constexpr (LH == 2) {
                me = rc_batch_me2<P, TPB>(kp, smem_raw, tc, svbuf, take, mine, pm);
            } else if constexpr (LH == 1) {
                me = lh_batch_me2<P, R, TPB>(kp, smem_raw, tc, svbuf, take, mine, pm);
            } else if constexpr (TC) {
                me = (double)P::Me::template me2<R, SYNC, true>(pm, kin_mt<KM>(kp), kin_gs<KM>(kp), slot, tc, hpart, HS);
            } else {
                me = (double)P::Me::template me2<R, SYNC>(pm, kin_mt<KM>(kp), kin_gs<KM>(kp), slot, nullptr, hpart, HS);
            }
            if constexpr (HS == 2) {
                // the owner adds the second half, evaluated in another warp
                svbuf[tid] = me;
                __syncthreads();
                if (hpart == 0) me += svbuf[tid + EPB];
                __syncthreads();
            }
            double w = owner ? pref * me : 0.0;
            if (!isfinite(w)) { w = 0.0; if (owner) ++nnan; }
            if (wr) {
                if (owner) {
                    o.me2 = me; o.w = w;
                    write_event<D>(kp, e, o, false);
                    write_momenta<P::NEXT>(kp, e, pm);
                }
            }
            const double wn = w * kp.inv_n;
            const double v = wn * wn;
            sw += wn;
            sw2 += v;
            svbuf[tid] = v;
#pragma unroll
            for (int d = 0; d < D; ++d) sbins[d * TPB + tid] = o.bins[d];
            if (obs) {
                swbuf[tid] = wn;
                sobin[tid] = (int16_t)(owner ? obs_bin(kp, (double)pm[2][1], (double)pm[2][2]) : 0);
            }
            __syncthreads();
            if (tid < D) {
                double* h = shist + tid * nb;
                const uint8_t* b = sbins + tid * TPB;
                for (int t = 0; t < take; ++t) h[b[t]] += svbuf[t];   // the owners, in queue order
            } else if (obs && tid == D) {
                for (int t = 0; t < take; ++t) {                     // the observable, in queue order
                    sobs[2 * sobin[t]] += swbuf[t];
                    sobs[2 * sobin[t] + 1] += svbuf[t];
                }
            }
            // the batch's entries leave the ring
            __syncthreads();
            if (tid == 0) { scount[1] = (head + take) % CAP; scount[0] = cnt - take; }
            __syncthreads();
        }
    }
    if constexpr (TC) tc_teardown(tc, LH == 2 ? TC_RC_COLS : TC_COLS);
    write_partials<P, TPB, 1>(kp, sw, sw2, npass, nnan, sred, shist, out);
    write_obs_partials<1, L::OBS_ROW>(kp, sobs);
}

// ------------------------------------------------------------------ the fused integrand kernel

// Light processes in mixed precision ask for two CTAs per SM (at most 128 registers a thread for
// 256-thread CTAs): their kernels are bound by the FP64 pipe's latency, which more warps hide.
template <class P, typename R> constexpr int integrand_min_ctas() { return (!P::HEAVY && sizeof(R) == 4) ? 2 : 1; }

template <class P, typename R, int TPB, bool WRITE, bool SYNC, bool TC = false, int HS = 1, int LH = 0>
__global__ void __launch_bounds__(TPB, integrand_min_ctas<P, R>()) integrand_kernel(KParams kp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double* out = kp.partials + (size_t)blockIdx.x * (2 + P::D * kp.nb);
    if constexpr (P::HEAVY) {
        constexpr int EPB = TPB / HS;   // events per CTA and round
        const long long first = (long long)blockIdx.x * EPB, step = (long long)gridDim.x * EPB;
        if constexpr (LH || P::BG) {
            // the host launches this schedule only with a record region for every CTA (the
            // recycled schedule's CTAs of TPB threads take TPB / LH_TPB of a region each)
            const bool room = LH == 2 ? (long long)blockIdx.x * TPB < (long long)kp.inv_ctas * LH_TPB
                                      : (int)blockIdx.x < kp.inv_ctas;
            if (kp.inv_rec == nullptr || !room) {
                if (threadIdx.x == 0 && kp.dev_err) atomicExch(kp.dev_err, 1u);
                for (int i = threadIdx.x; i < 2 + P::D * kp.nb; i += TPB) out[i] = 0.0;
                return;
            }
        }
        integrand_heavy<P, R, TPB, WRITE, SYNC, TC, HS, LH>(kp, smem_raw, first, step, kp.n_events, out);
    } else {
        const long long first = (long long)blockIdx.x * TPB, step = (long long)gridDim.x * TPB;
        integrand_light<P, R, TPB, WRITE>(kp, smem_raw, first, step, kp.n_events, out);
    }
}

// ------------------------------------------------------------------ evaluate

template <class ME, typename R>
__global__ void __launch_bounds__(128) evaluate_kernel(const double* __restrict__ mom, long long n, double* __restrict__ me2,
                                                       double mt, double gs)
{
    extern __shared__ __align__(16) unsigned char slots[];
    void* slot = slots + (size_t)threadIdx.x * ME::template slot_bytes<R>();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double p[ME::NEXT][4];
        for (int i = 0; i < ME::NEXT; ++i)
            for (int c = 0; c < 4; ++c) p[i][c] = mom[(e * ME::NEXT + i) * 4 + c];
        me2[e] = ME::template me2<R>(p, mt, gs, slot);
    }
}

template <typename R>
__global__ void __launch_bounds__(128) evaluate_ee_kernel(const double* __restrict__ mom, long long n, double* __restrict__ me2,
                                                          EwParams ew)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double p[4][4];
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 4; ++c) p[i][c] = mom[(e * 4 + i) * 4 + c];
        me2[e] = MeEeMumu::me2<R>(p, ew);
    }
}

// ------------------------------------------------------------------ helicity profile

// per-helicity averaged |M_h|^2 of caller momenta: out [n][ME::NHEL] (diagnostic of the
// helicity sum: its entries add up to evaluate's |M|^2)
template <class ME, typename R>
__global__ void __launch_bounds__(64) helicity_profile_kernel(const double* __restrict__ mom, long long n,
                                                              double* __restrict__ out, double mt, double gs)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double p[ME::NEXT][4];
        for (int i = 0; i < ME::NEXT; ++i)
            for (int c = 0; c < 4; ++c) p[i][c] = mom[(e * ME::NEXT + i) * 4 + c];
        ME::template hel_profile<R>(p, mt, gs, out + e * ME::NHEL);
    }
}

template <typename R>
__global__ void __launch_bounds__(64) helicity_profile_ee_kernel(const double* __restrict__ mom, long long n,
                                                                 double* __restrict__ out, EwParams ew)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double p[4][4];
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 4; ++c) p[i][c] = mom[(e * 4 + i) * 4 + c];
        MeEeMumu::hel_profile<R>(p, ew, out + e * MeEeMumu::NHEL);
    }
}

// ------------------------------------------------------------------ derivatives

// Derivative pass (forward mode): every event's weight and its derivative
// with respect to m_t in one evaluation (R = Dual<float> or Dual<double> in
// the matrix element, Dual<double> elsewhere), at the base-point cut masks
// and a fixed VEGAS grid.  Per CTA: sum w, sum dw/dm_t, sum (dw/dm_t)^2 and
// sum k w / alpha_s (|M|^2 is proportional to alpha_s^k), all with the
// estimator's 1/N, reduced deterministically.
template <class P, typename R>
__global__ void __launch_bounds__(128) grad_kernel(KParams kp, double* partials, int k_as, double alpha_s)
{
    using S = Dual<double>;
    constexpr int D = P::D, TPB = 128, WARPS = TPB / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sgrid = reinterpret_cast<double*>(smem_raw);
    double* sred = sgrid + D * (kp.nb + 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < D * (kp.nb + 1); i += TPB) sgrid[i] = kp.grid[i];
    __syncthreads();
    double acc[4] = { 0.0, 0.0, 0.0, 0.0 };
    const long long n = kp.n_events;
    const S mt(kp.mt, 1.0), gs(kp.gs, 0.0);
    for (long long e = (long long)blockIdx.x * TPB + tid; e < n; e += (long long)gridDim.x * TPB) {
        EventOut<D> o;
        S pm[P::NEXT][4], pref;
        kinematics_tops_t<P, S>(kp, sgrid, kp.pdf, (unsigned long long)(kp.ev_offset + e), mt, o, pm, pref);
        if (!o.mask) continue;
        const S me = P::Me::template me2<R>(pm, mt, gs, nullptr);
        S w = pref * me;
        if (!isfinite(w.v) || !isfinite(w.d)) continue;
        const double wn = w.v * kp.inv_n, dn = w.d * kp.inv_n;
        acc[0] += wn;
        acc[1] += dn;
        acc[2] += dn * dn;
        acc[3] += k_as * wn / alpha_s;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sred[4 * warp + k] = v;
    }
    __syncthreads();
    if (tid < 4) {
        double v = 0.0;
        for (int w = 0; w < WARPS; ++w) v += sred[4 * w + tid];
        partials[(size_t)blockIdx.x * 4 + tid] = v;
    }
}

// Derivative pass of a gluon process through the recursion (G: its tables, SYM_DEN the
// identical-gluon factor): each thread carries one event's kinematics with the m_t tangent
// (Dual<double>: the parton map, RAMBO's mass rescaling, the scale and the PDFs), the
// events that pass are staged with their momenta and tangents in this CTA's region of
// kp.inv_rec, and warp w < MW evaluates events w, w + MW, ... of the round: |M|^2 and its
// derivative along (dp/dm_t, dm_t = 1) in forward mode (bg_warp_me2_dir: one direction,
// so no reverse sweep).  Per CTA the same four sums as grad_kernel, reduced
// deterministically.
template <class P, class G, typename R, int SYM_DEN, int MW>
__global__ void __launch_bounds__(128) bg_grad_kernel(KParams kp, double* partials, int k_as, double alpha_s)
{
    // MW: the warps with a recursion state (as many as fit the shared memory); every warp
    // runs the kinematics, warps w < MW the matrix elements
    using S = Dual<double>;
    constexpr int D = P::D, NEXT = P::NEXT, NW = NEXT * 4, TPB = 128, WARPS = TPB / 32, CROW = G::NPERM + 1;
    static_assert((2 * NW + 2) * TPB <= LH_INV_WORDS_MAX * LH_TPB / 4, "staging fits half a record region");
    extern __shared__ __align__(128) unsigned char mf_bgp_smem[];
    const size_t cbytes = ((sizeof(float) * G::NPERM * CROW) + 127) & ~(size_t)127;
    const size_t wbytes = (sizeof(BgDirWarp<G, R>) + 15) & ~(size_t)15;
    float* cs = reinterpret_cast<float*>(mf_bgp_smem);
    double* sgrid = reinterpret_cast<double*>(mf_bgp_smem + cbytes + MW * wbytes);
    double* sres = sgrid + D * (kp.nb + 1);            // [TPB][2]: |M|^2 and its derivative
    double* sred = sres + 2 * TPB;                      // [WARPS][4]
    int* smask = reinterpret_cast<int*>(sred + 4 * WARPS);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (kp.inv_rec == nullptr || (int)(blockIdx.x >> 1) >= kp.inv_ctas) {
        // the host launches at most two CTAs per region; a larger grid is an error, not a skip
        if (tid == 0 && kp.dev_err) atomicExch(kp.dev_err, 1u);
        if (tid < 4) partials[(size_t)blockIdx.x * 4 + tid] = 0.0;
        return;
    }
    // two CTAs share one region of the record buffer, each taking half of it
    double* grec = reinterpret_cast<double*>(kp.inv_rec + (size_t)(blockIdx.x >> 1) * LH_INV_WORDS_MAX * LH_TPB) +
                   (blockIdx.x & 1) * (LH_INV_WORDS_MAX * LH_TPB / 4);
    for (int i = tid; i < G::NPERM * G::NPERM; i += TPB) cs[(i / G::NPERM) * CROW + i % G::NPERM] = __ldg(G::colour() + i);
    for (int i = tid; i < D * (kp.nb + 1); i += TPB) sgrid[i] = kp.grid[i];
    __syncthreads();
    auto& st = *reinterpret_cast<BgDirWarp<G, R>*>(mf_bgp_smem + cbytes + (warp < MW ? warp : 0) * wbytes);
    double norm = 1.0 / (256.0 * SYM_DEN);
    for (int i = 0; i < G::K; ++i) norm *= kp.gs * kp.gs;
    double acc[4] = { 0.0, 0.0, 0.0, 0.0 };
    const long long n = kp.n_events;
    const S mt(kp.mt, 1.0);
    for (long long base = (long long)blockIdx.x * TPB; base < n; base += (long long)gridDim.x * TPB) {
        const long long e = base + tid;
        int pass = 0;
        S pref = S(0.0);
        if (e < n) {
            EventOut<D> o;
            S pm[NEXT][4];
            kinematics_tops_t<P, S>(kp, sgrid, kp.pdf, (unsigned long long)(kp.ev_offset + e), mt, o, pm, pref);
            pass = o.mask;
            if (pass) {
#pragma unroll
                for (int f = 0; f < NW; ++f) {
                    grec[(size_t)f * TPB + tid] = pm[f >> 2][f & 3].v;
                    grec[(size_t)(NW + f) * TPB + tid] = pm[f >> 2][f & 3].d;
                }
            }
        }
        smask[tid] = pass;
        __syncthreads();
        for (int j = warp; warp < MW && j < TPB; j += MW) {
            if (!smask[j]) continue;                    // the same j for the whole warp
            // forward mode along (dp/dm_t, dm_t = 1): the staged momenta and their tangents
            double dme = 0.0;
            const double v = bg_warp_me2_dir<G, R>(st, cs, CROW, grec + j, grec + (size_t)NW * TPB + j, TPB, kp.mt, 1.0,
                                                   &dme);
            if (lane == 0) { sres[2 * j] = v * norm; sres[2 * j + 1] = dme * norm; }
            __syncwarp();
        }
        __syncthreads();
        if (pass) {
            const double me = sres[2 * tid], dme = sres[2 * tid + 1];
            const double w = pref.v * me, dw = pref.d * me + pref.v * dme;
            if (isfinite(w) && isfinite(dw)) {
                const double wn = w * kp.inv_n, dn = dw * kp.inv_n;
                acc[0] += wn;
                acc[1] += dn;
                acc[2] += dn * dn;
                acc[3] += k_as * wn / alpha_s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sred[4 * warp + k] = v;
    }
    __syncthreads();
    if (tid < 4) {
        double v = 0.0;
        for (int w = 0; w < WARPS; ++w) v += sred[4 * w + tid];
        partials[(size_t)blockIdx.x * 4 + tid] = v;
    }
}

template <class P, class G, typename R>
constexpr size_t bg_grad_pass_smem(int nb, int mw)
{
    return (((sizeof(float) * G::NPERM * (G::NPERM + 1)) + 127) & ~(size_t)127) +
           (size_t)mw * ((sizeof(BgDirWarp<G, R>) + 15) & ~(size_t)15) +
           sizeof(double) * (P::D * (nb + 1) + 2 * 128 + 16) + sizeof(int) * 128;
}
// recursion warps of the derivative pass: as many (1 .. 4) as fit 227 KB with a 64-bin grid
template <class P, class G, typename R>
constexpr int bg_grad_pass_warps()
{
    int w = 4;
    while (w > 1 && bg_grad_pass_smem<P, G, R>(MAX_BINS, w) > 227 * 1024) --w;
    return w;
}

// d|M|^2 / d p for every momentum component (the components treated as
// independent variables): one forward-mode evaluation per component.
template <class ME, typename R>
__global__ void __launch_bounds__(128) evaluate_grad_kernel(const double* __restrict__ mom, long long n,
                                                            double* __restrict__ me2, double* __restrict__ dme2,
                                                            double mt, double gs)
{
    using S = Dual<double>;
    constexpr int NC = 4 * ME::NEXT;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double p0[ME::NEXT][4];
        for (int i = 0; i < ME::NEXT; ++i)
            for (int c = 0; c < 4; ++c) p0[i][c] = mom[(e * ME::NEXT + i) * 4 + c];
        for (int j = 0; j < NC; ++j) {
            S p[ME::NEXT][4];
            for (int i = 0; i < ME::NEXT; ++i)
                for (int c = 0; c < 4; ++c) p[i][c] = S(p0[i][c], (4 * i + c) == j ? 1.0 : 0.0);
            const S m = ME::template me2<R>(p, S(mt, 0.0), S(gs, 0.0), nullptr);
            dme2[e * NC + j] = m.d;
            if (j == 0 && me2) me2[e] = m.v;
        }
    }
}

}  // namespace mf
