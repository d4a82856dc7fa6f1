// HELAS-style helicity wavefunctions and vertices for the matrix element
// (Sec. 2.2 of arXiv:2105.10529: external wavefunctions, vertices and
// propagators evaluated per helicity and summed into |M|^2).
//
// Conventions (own, written for this library):
//  * metric (+,-,-,-); chiral (Weyl) representation
//      gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]], sigma^mu = (1, s), sigmabar^mu = (1, -s);
//  * a spinor is (L0, L1, R0, R1); a row spinor (psibar) uses the same layout;
//  * helicity eigenspinors chi_+/-(p) of sigma.p/|p|; omega_+/- = sqrt(E +/- |p|);
//      u(p,l)    = (omega_-l chi_l ; omega_l chi_l)
//      v(p,l)    = (-l omega_l chi_-l ; l omega_-l chi_-l)
//      ubar(p,l) = (omega_l chi_l^+ , omega_-l chi_l^+)
//      vbar(p,l) = (l omega_-l chi_-l^+ , -l omega_l chi_-l^+)
//  * gluon polarisation eps(k,l) = (-l e1 - i e2)/sqrt(2), e1 = (0, cos th cos ph,
//    cos th sin ph, -sin th), e2 = (0, -sin ph, cos ph, 0); outgoing gluons use conj(eps);
//  * vertex routines return the Lorentz structure only: couplings g, the
//    factors of i and the colour weights are applied by the generated code.
//
// Every routine is templated on the real type R (float for the mixed path,
// double for the FP64 path).  Helicity-independent quantities (momenta,
// propagator denominators, the spinor normalisations omega) are computed
// per event in FP64 and passed in as R.
#pragma once
#include <cstdint>
#include "mf_dual.cuh"

namespace mf {

template <typename R> struct cx { R r, i; };

template <typename R> __device__ __forceinline__ cx<R> mkc(R r, R i) { cx<R> c; c.r = r; c.i = i; return c; }
template <typename R> __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return mkc(a.r + b.r, a.i + b.i); }
template <typename R> __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return mkc(a.r - b.r, a.i - b.i); }
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b)
{
    return mkc(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return mkc(a.r * s, a.i * s); }
// a*b + c
template <typename R> __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c)
{
    return mkc(fma(a.r, b.r, fma(-a.i, b.i, c.r)), fma(a.r, b.i, fma(a.i, b.r, c.i)));
}
// a*b - c*d
template <typename R> __device__ __forceinline__ cx<R> cmulsub(cx<R> a, cx<R> b, cx<R> c, cx<R> d)
{
    return csub(cmul(a, b), cmul(c, d));
}

// four complex components: a spinor (L0,L1,R0,R1) or a vector (mu = 0..3)
template <typename R> struct W4 { cx<R> c[4]; };

// Minkowski product of two complex vectors (no conjugation)
template <typename R> __device__ __forceinline__ cx<R> cdot(const W4<R>& a, const W4<R>& b)
{
    cx<R> s = cmul(a.c[0], b.c[0]);
    s = csub(s, cmul(a.c[1], b.c[1]));
    s = csub(s, cmul(a.c[2], b.c[2]));
    s = csub(s, cmul(a.c[3], b.c[3]));
    return s;
}
// Minkowski product of a real momentum with a complex vector
template <typename R> __device__ __forceinline__ cx<R> rdot(const R* k, const W4<R>& a)
{
    return mkc(k[0] * a.c[0].r - k[1] * a.c[1].r - k[2] * a.c[2].r - k[3] * a.c[3].r,
               k[0] * a.c[0].i - k[1] * a.c[1].i - k[2] * a.c[2].i - k[3] * a.c[3].i);
}

// ------------------------------------------------------------------ external states

// gluon: eps(k, l) for an incoming gluon, conj(eps) for an outgoing one.
// e1, e2: spatial parts of the transverse basis (R[3] each), already scaled by 1/sqrt(2).
template <typename R> __device__ __forceinline__ W4<R> ext_gluon(const R* e1, const R* e2, int hel, bool outgoing)
{
    W4<R> w;
    R l = hel > 0 ? R(1) : R(-1);
    R s = outgoing ? R(1) : R(-1);
    w.c[0] = mkc(R(0), R(0));
    for (int j = 0; j < 3; ++j) w.c[j + 1] = mkc(-l * e1[j], s * e2[j]);
    return w;
}

// Fermion external states from the per-event pieces: chi[0] = chi_+, chi[1] = chi_-
// (two components each), om[0] = omega_+, om[1] = omega_-.
template <typename R> struct FermionBasis { cx<R> chi[2][2]; R om[2]; };

template <typename R> __device__ __forceinline__ cx<R> conjc(cx<R> a) { return mkc(a.r, -a.i); }

// volatile read of a per-event invariant: re-read at every use instead of
// being held in a register across the helicity body
template <typename R> __device__ __forceinline__ R ldv(const R& x) { return *(const volatile R*)&x; }
template <typename T> __device__ __forceinline__ Dual<T> ldv(const Dual<T>& x) { return Dual<T>(ldv(x.v), ldv(x.d)); }

// reads and writes of the colour-flow accumulators kept in shared memory
template <typename R> __device__ __forceinline__ R vget(const volatile R& x) { return x; }
template <typename T> __device__ __forceinline__ Dual<T> vget(const volatile Dual<T>& x) { return Dual<T>(x.v, x.d); }
template <typename R> __device__ __forceinline__ void vset(volatile R& x, R a) { x = a; }
template <typename T> __device__ __forceinline__ void vset(volatile Dual<T>& x, Dual<T> a) { x.v = a.v; x.d = a.d; }
// jamp += c a for c = +1, -1, +i, -i, and a general complex c
template <typename R> __device__ __forceinline__ void jadd_p(volatile cx<R>& j, cx<R> a)
{
    vset(j.r, vget(j.r) + a.r); vset(j.i, vget(j.i) + a.i);
}
template <typename R> __device__ __forceinline__ void jadd_m(volatile cx<R>& j, cx<R> a)
{
    vset(j.r, vget(j.r) - a.r); vset(j.i, vget(j.i) - a.i);
}
template <typename R> __device__ __forceinline__ void jadd_pi(volatile cx<R>& j, cx<R> a)
{
    vset(j.r, vget(j.r) - a.i); vset(j.i, vget(j.i) + a.r);
}
template <typename R> __device__ __forceinline__ void jadd_mi(volatile cx<R>& j, cx<R> a)
{
    vset(j.r, vget(j.r) + a.i); vset(j.i, vget(j.i) - a.r);
}
template <typename R> __device__ __forceinline__ void jadd_c(volatile cx<R>& j, cx<R> a, R cr, R ci)
{
    vset(j.r, vget(j.r) + (cr * a.r - ci * a.i)); vset(j.i, vget(j.i) + (cr * a.i + ci * a.r));
}

// Wide shared-memory accesses of the warp-per-event helicity body (float only; the
// record's momenta 16-byte and the colour-flow accumulators 8-byte aligned): one
// instruction where the scalar forms above take four or two.  Like ldv they are
// issued at every use (volatile asm: never merged or hoisted), in program order.
__device__ __forceinline__ uint32_t smem_addr(const volatile void* p)
{
    return (uint32_t)__cvta_generic_to_shared((const void*)p);
}
// o = x (four floats)
__device__ __forceinline__ void ldv4(const float (&x)[4], float (&o)[4])
{
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]) : "r"(smem_addr(x)));
}
// o = x - y (four floats each)
__device__ __forceinline__ void ldv4_diff(const float (&x)[4], const float (&y)[4], float (&o)[4])
{
    float a[4], b[4];
    ldv4(x, a);
    ldv4(y, b);
    for (int m = 0; m < 4; ++m) o[m] = a[m] - b[m];
}
__device__ __forceinline__ void jzero64(volatile cx<float>& j)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %1};" :: "r"(smem_addr(&j)), "f"(0.0f));
}
// j += (dr, di) with one 64-bit load and one 64-bit store
__device__ __forceinline__ void jadd64(volatile cx<float>& j, float dr, float di)
{
    const uint32_t a = smem_addr(&j);
    float r, i;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r), "=f"(i) : "r"(a));
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" :: "r"(a), "f"(r + dr), "f"(i + di));
}
__device__ __forceinline__ void jadd64_p(volatile cx<float>& j, cx<float> a) { jadd64(j, a.r, a.i); }
__device__ __forceinline__ void jadd64_m(volatile cx<float>& j, cx<float> a) { jadd64(j, -a.r, -a.i); }
__device__ __forceinline__ void jadd64_pi(volatile cx<float>& j, cx<float> a) { jadd64(j, -a.i, a.r); }
__device__ __forceinline__ void jadd64_mi(volatile cx<float>& j, cx<float> a) { jadd64(j, a.i, -a.r); }

template <typename R> __device__ __forceinline__ FermionBasis<R> load_basis(const FermionBasis<R>& f)
{
    FermionBasis<R> o;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) o.chi[a][b] = mkc(ldv(f.chi[a][b].r), ldv(f.chi[a][b].i));
    o.om[0] = ldv(f.om[0]);
    o.om[1] = ldv(f.om[1]);
    return o;
}

template <typename R> __device__ __forceinline__ W4<R> ext_u(const FermionBasis<R>& f, int hel)
{
    int l = hel > 0 ? 0 : 1;          // chi_l
    R wl = f.om[l], wml = f.om[1 - l];
    W4<R> w;
    w.c[0] = cscale(f.chi[l][0], wml); w.c[1] = cscale(f.chi[l][1], wml);
    w.c[2] = cscale(f.chi[l][0], wl);  w.c[3] = cscale(f.chi[l][1], wl);
    return w;
}
template <typename R> __device__ __forceinline__ W4<R> ext_ubar(const FermionBasis<R>& f, int hel)
{
    int l = hel > 0 ? 0 : 1;
    R wl = f.om[l], wml = f.om[1 - l];
    W4<R> w;
    w.c[0] = cscale(conjc(f.chi[l][0]), wl);  w.c[1] = cscale(conjc(f.chi[l][1]), wl);
    w.c[2] = cscale(conjc(f.chi[l][0]), wml); w.c[3] = cscale(conjc(f.chi[l][1]), wml);
    return w;
}
template <typename R> __device__ __forceinline__ W4<R> ext_v(const FermionBasis<R>& f, int hel)
{
    int l = hel > 0 ? 0 : 1;          // omega_l, chi_-l
    R sl = hel > 0 ? R(1) : R(-1);
    R wl = f.om[l], wml = f.om[1 - l];
    W4<R> w;
    w.c[0] = cscale(f.chi[1 - l][0], -sl * wl); w.c[1] = cscale(f.chi[1 - l][1], -sl * wl);
    w.c[2] = cscale(f.chi[1 - l][0], sl * wml); w.c[3] = cscale(f.chi[1 - l][1], sl * wml);
    return w;
}
template <typename R> __device__ __forceinline__ W4<R> ext_vbar(const FermionBasis<R>& f, int hel)
{
    int l = hel > 0 ? 0 : 1;
    R sl = hel > 0 ? R(1) : R(-1);
    R wl = f.om[l], wml = f.om[1 - l];
    W4<R> w;
    w.c[0] = cscale(conjc(f.chi[1 - l][0]), sl * wml); w.c[1] = cscale(conjc(f.chi[1 - l][1]), sl * wml);
    w.c[2] = cscale(conjc(f.chi[1 - l][0]), -sl * wl); w.c[3] = cscale(conjc(f.chi[1 - l][1]), -sl * wl);
    return w;
}

// ------------------------------------------------------------------ slashed vectors

// Sigma(J) = J^0 - J.s and Sigmabar(J) = J^0 + J.s as 2x2 complex matrices
template <typename R> struct M2 { cx<R> m00, m01, m10, m11; };

template <typename R> __device__ __forceinline__ M2<R> sig(const W4<R>& J)
{
    M2<R> s;
    s.m00 = csub(J.c[0], J.c[3]);
    s.m11 = cadd(J.c[0], J.c[3]);
    // -(J1 - i J2), -(J1 + i J2)
    s.m01 = mkc(-J.c[1].r - J.c[2].i, -J.c[1].i + J.c[2].r);
    s.m10 = mkc(-J.c[1].r + J.c[2].i, -J.c[1].i - J.c[2].r);
    return s;
}
template <typename R> __device__ __forceinline__ M2<R> sigbar(const W4<R>& J)
{
    M2<R> s;
    s.m00 = cadd(J.c[0], J.c[3]);
    s.m11 = csub(J.c[0], J.c[3]);
    s.m01 = mkc(J.c[1].r + J.c[2].i, J.c[1].i - J.c[2].r);
    s.m10 = mkc(J.c[1].r - J.c[2].i, J.c[1].i + J.c[2].r);
    return s;
}
// row (x0,x1) times M
template <typename R> __device__ __forceinline__ void rowm(cx<R> x0, cx<R> x1, const M2<R>& m, cx<R>& y0, cx<R>& y1)
{
    y0 = cfma(x1, m.m10, cmul(x0, m.m00));
    y1 = cfma(x1, m.m11, cmul(x0, m.m01));
}
// M times column (x0,x1)
template <typename R> __device__ __forceinline__ void mcol(const M2<R>& m, cx<R> x0, cx<R> x1, cx<R>& y0, cx<R>& y1)
{
    y0 = cfma(m.m01, x1, cmul(m.m00, x0));
    y1 = cfma(m.m11, x1, cmul(m.m10, x0));
}
// real-momentum versions: Sigma(q) = q0 - q.s, Sigmabar(q) = q0 + q.s applied to spinor halves
template <typename R> __device__ __forceinline__ void rowq(cx<R> x0, cx<R> x1, const R* q, bool bar, cx<R>& y0, cx<R>& y1)
{
    R s = bar ? R(1) : R(-1);
    R a = q[0] + s * q[3], d = q[0] - s * q[3];
    // off-diagonal: m01 = s (q1 - i q2), m10 = s (q1 + i q2)
    R b = s * q[1], c = s * q[2];
    // y0 = x0 a + x1 m10 ; y1 = x0 m01 + x1 d
    y0 = mkc(x0.r * a + x1.r * b - x1.i * c, x0.i * a + x1.i * b + x1.r * c);
    y1 = mkc(x0.r * b + x0.i * c + x1.r * d, x0.i * b - x0.r * c + x1.i * d);
}
template <typename R> __device__ __forceinline__ void qcol(const R* q, bool bar, cx<R> x0, cx<R> x1, cx<R>& y0, cx<R>& y1)
{
    R s = bar ? R(1) : R(-1);
    R a = q[0] + s * q[3], d = q[0] - s * q[3];
    R b = s * q[1], c = s * q[2];
    // y0 = a x0 + m01 x1 ; y1 = m10 x0 + d x1
    y0 = mkc(a * x0.r + b * x1.r + c * x1.i, a * x0.i + b * x1.i - c * x1.r);
    y1 = mkc(b * x0.r - c * x0.i + d * x1.r, b * x0.i + c * x0.r + d * x1.i);
}

// ------------------------------------------------------------------ fermion vertices

// psibar Jslash psi
template <typename R> __device__ __forceinline__ cx<R> ffv_amp(const W4<R>& fb, const W4<R>& f, const W4<R>& J)
{
    // (a,b) [[0,S],[Sb,0]] (c;d) = a S d + b Sb c
    M2<R> S = sig(J), Sb = sigbar(J);
    cx<R> y0, y1;
    mcol(S, f.c[2], f.c[3], y0, y1);
    cx<R> r = cfma(fb.c[1], y1, cmul(fb.c[0], y0));
    mcol(Sb, f.c[0], f.c[1], y0, y1);
    r = cfma(fb.c[2], y0, r);
    r = cfma(fb.c[3], y1, r);
    return r;
}

// psibar gamma^mu psi, scaled by s
template <typename R> __device__ __forceinline__ W4<R> ffv_cur(const W4<R>& fb, const W4<R>& f, R s)
{
    // J^0 = a.d + b.c ; J^k = a s^k d - b s^k c
    cx<R> a0 = fb.c[0], a1 = fb.c[1], b0 = fb.c[2], b1 = fb.c[3];
    cx<R> c0 = f.c[0], c1 = f.c[1], d0 = f.c[2], d1 = f.c[3];
    W4<R> J;
    cx<R> ad00 = cmul(a0, d0), ad11 = cmul(a1, d1), ad01 = cmul(a0, d1), ad10 = cmul(a1, d0);
    cx<R> bc00 = cmul(b0, c0), bc11 = cmul(b1, c1), bc01 = cmul(b0, c1), bc10 = cmul(b1, c0);
    J.c[0] = cadd(cadd(ad00, ad11), cadd(bc00, bc11));
    J.c[1] = csub(cadd(ad01, ad10), cadd(bc01, bc10));
    // s^2: a s2 d = -i a0 d1 + i a1 d0 = i (a1 d0 - a0 d1)
    cx<R> x = csub(ad10, ad01), y = csub(bc10, bc01);
    cx<R> t = csub(x, y);
    J.c[2] = mkc(-t.i, t.r);
    J.c[3] = csub(csub(ad00, ad11), csub(bc00, bc11));
    for (int m = 0; m < 4; ++m) J.c[m] = cscale(J.c[m], s);
    return J;
}

// chirality-split currents psibar gamma^mu P_L psi and psibar gamma^mu P_R psi
// (P_L = diag(1,1,0,0) in the chiral basis): J_L = b sigmabar^mu c, J_R = a sigma^mu d
template <typename R> __device__ __forceinline__ void ffv_cur_lr(const W4<R>& fb, const W4<R>& f, W4<R>& JL, W4<R>& JR)
{
    cx<R> a0 = fb.c[0], a1 = fb.c[1], b0 = fb.c[2], b1 = fb.c[3];
    cx<R> c0 = f.c[0], c1 = f.c[1], d0 = f.c[2], d1 = f.c[3];
    cx<R> ad00 = cmul(a0, d0), ad11 = cmul(a1, d1), ad01 = cmul(a0, d1), ad10 = cmul(a1, d0);
    cx<R> bc00 = cmul(b0, c0), bc11 = cmul(b1, c1), bc01 = cmul(b0, c1), bc10 = cmul(b1, c0);
    JR.c[0] = cadd(ad00, ad11);
    JR.c[1] = cadd(ad01, ad10);
    cx<R> x = csub(ad10, ad01);
    JR.c[2] = mkc(-x.i, x.r);
    JR.c[3] = csub(ad00, ad11);
    JL.c[0] = cadd(bc00, bc11);
    JL.c[1] = mkc(-(bc01.r + bc10.r), -(bc01.i + bc10.i));
    cx<R> y = csub(bc10, bc01);
    JL.c[2] = mkc(y.i, -y.r);
    JL.c[3] = csub(bc11, bc00);
}

// off-shell row spinor: fb Jslash (qslash + m) * s
template <typename R> __device__ __forceinline__ W4<R> ffv_row(const W4<R>& fb, const W4<R>& J, const R* q, R m, R s)
{
    // (a,b) Jslash = (b Sb, a S)
    M2<R> S = sig(J), Sb = sigbar(J);
    cx<R> p0, p1, r0, r1;
    rowm(fb.c[2], fb.c[3], Sb, p0, p1);     // left half  a'
    rowm(fb.c[0], fb.c[1], S, r0, r1);      // right half b'
    // (a',b') (qslash + m) = (m a' + b' Sb_q, a' S_q + m b')
    cx<R> t0, t1, u0, u1;
    rowq(r0, r1, q, true, t0, t1);
    rowq(p0, p1, q, false, u0, u1);
    W4<R> o;
    o.c[0] = cscale(mkc(fma(m, p0.r, t0.r), fma(m, p0.i, t0.i)), s);
    o.c[1] = cscale(mkc(fma(m, p1.r, t1.r), fma(m, p1.i, t1.i)), s);
    o.c[2] = cscale(mkc(fma(m, r0.r, u0.r), fma(m, r0.i, u0.i)), s);
    o.c[3] = cscale(mkc(fma(m, r1.r, u1.r), fma(m, r1.i, u1.i)), s);
    return o;
}

// off-shell column spinor: (qslash + m) Jslash f * s
template <typename R> __device__ __forceinline__ W4<R> ffv_col(const W4<R>& J, const W4<R>& f, const R* q, R m, R s)
{
    // Jslash (c;d) = (S d ; Sb c)
    M2<R> S = sig(J), Sb = sigbar(J);
    cx<R> c0, c1, d0, d1;
    mcol(S, f.c[2], f.c[3], c0, c1);
    mcol(Sb, f.c[0], f.c[1], d0, d1);
    // (qslash + m)(c';d') = (m c' + S_q d' ; Sb_q c' + m d')
    cx<R> t0, t1, u0, u1;
    qcol(q, false, d0, d1, t0, t1);
    qcol(q, true, c0, c1, u0, u1);
    W4<R> o;
    o.c[0] = cscale(mkc(fma(m, c0.r, t0.r), fma(m, c0.i, t0.i)), s);
    o.c[1] = cscale(mkc(fma(m, c1.r, t1.r), fma(m, c1.i, t1.i)), s);
    o.c[2] = cscale(mkc(fma(m, d0.r, u0.r), fma(m, d0.i, u0.i)), s);
    o.c[3] = cscale(mkc(fma(m, d1.r, u1.r), fma(m, d1.i, u1.i)), s);
    return o;
}

// ------------------------------------------------------------------ gluon vertices

// three-gluon current (k3 = -(k1+k2), all incoming), scaled by s:
// V^rho = (J1.J2)(k1-k2)^rho + J2^rho (k2-k3).J1 + J1^rho (k3-k1).J2
template <typename R> __device__ __forceinline__ W4<R> vvv_cur(const W4<R>& J1, const W4<R>& J2, const R* k1, const R* k2, R s)
{
    R a[4], b[4], c[4];
    for (int m = 0; m < 4; ++m) {
        a[m] = k1[m] - k2[m];
        b[m] = k1[m] + R(2) * k2[m];          // k2 - k3
        c[m] = -(R(2) * k1[m] + k2[m]);       // k3 - k1
    }
    cx<R> j12 = cdot(J1, J2), bj1 = rdot(b, J1), cj2 = rdot(c, J2);
    W4<R> o;
    for (int m = 0; m < 4; ++m) {
        cx<R> t = cscale(j12, a[m]);
        t = cfma(J2.c[m], bj1, t);
        t = cfma(J1.c[m], cj2, t);
        o.c[m] = cscale(t, s);
    }
    return o;
}

// three-gluon vertex contracted with three currents
template <typename R> __device__ __forceinline__ cx<R> vvv_amp(const W4<R>& J1, const W4<R>& J2, const W4<R>& J3,
                                                               const R* k1, const R* k2, const R* k3)
{
    R a[4], b[4], c[4];
    for (int m = 0; m < 4; ++m) { a[m] = k1[m] - k2[m]; b[m] = k2[m] - k3[m]; c[m] = k3[m] - k1[m]; }
    cx<R> r = cmul(cdot(J1, J2), rdot(a, J3));
    r = cfma(cdot(J2, J3), rdot(b, J1), r);
    r = cfma(cdot(J3, J1), rdot(c, J2), r);
    return r;
}

// the three Lorentz structures of the four-gluon vertex as currents, scaled by s:
// L1 = (J1.J3) J2 - (J2.J3) J1, L2 = (J1.J2) J3 - (J2.J3) J1, L3 = (J1.J2) J3 - (J1.J3) J2
template <typename R> __device__ __forceinline__ void vvvv_cur(const W4<R>& J1, const W4<R>& J2, const W4<R>& J3, R s,
                                                               W4<R>& L1, W4<R>& L2, W4<R>& L3)
{
    cx<R> d12 = cscale(cdot(J1, J2), s), d13 = cscale(cdot(J1, J3), s), d23 = cscale(cdot(J2, J3), s);
    for (int m = 0; m < 4; ++m) {
        L1.c[m] = cmulsub(d13, J2.c[m], d23, J1.c[m]);
        L2.c[m] = cmulsub(d12, J3.c[m], d23, J1.c[m]);
        L3.c[m] = cmulsub(d12, J3.c[m], d13, J2.c[m]);
    }
}

// Jq . L_t for the three structures
template <typename R> __device__ __forceinline__ void vvvv_amp(const W4<R>& J1, const W4<R>& J2, const W4<R>& J3, const W4<R>& Jq,
                                                               cx<R>& a1, cx<R>& a2, cx<R>& a3)
{
    cx<R> d12 = cdot(J1, J2), d13 = cdot(J1, J3), d23 = cdot(J2, J3);
    cx<R> q1 = cdot(Jq, J1), q2 = cdot(Jq, J2), q3 = cdot(Jq, J3);
    a1 = cmulsub(d13, q2, d23, q1);
    a2 = cmulsub(d12, q3, d23, q1);
    a3 = cmulsub(d12, q3, d13, q2);
}

// ------------------------------------------------------------------ per-event external pieces (FP64)

template <typename S> __device__ __forceinline__ S mdot(const S* a, const S* b)
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

// Transverse basis of a massless momentum p (e1, e2 spatial parts, scaled by 1/sqrt 2).
// For a Dual momentum the values are those of the plain basis and the tangents those of
// the parallel-transported basis, de = -(e . dn) n with n = p/|p|: the helicity-summed
// |M|^2 does not depend on the choice of transverse basis, and the transported one is
// smooth where the plain one is not (a momentum along the z axis, whose azimuth is
// undefined).
template <typename S>
__device__ __forceinline__ void gluon_basis(const S* p, S* e1, S* e2);

template <typename T>
__device__ __forceinline__ void gluon_basis_dual(const Dual<T>* p, Dual<T>* e1, Dual<T>* e2)
{
    const T pv[4] = { p[0].v, p[1].v, p[2].v, p[3].v };
    T a[3], b[3];
    gluon_basis(pv, a, b);
    const T pa = sqrt(pv[1] * pv[1] + pv[2] * pv[2] + pv[3] * pv[3]);
    const T n[3] = { pv[1] / pa, pv[2] / pa, pv[3] / pa };
    const T ndp = n[0] * p[1].d + n[1] * p[2].d + n[2] * p[3].d;
    const T dn[3] = { (p[1].d - n[0] * ndp) / pa, (p[2].d - n[1] * ndp) / pa, (p[3].d - n[2] * ndp) / pa };
    const T ca = a[0] * dn[0] + a[1] * dn[1] + a[2] * dn[2];
    const T cb = b[0] * dn[0] + b[1] * dn[1] + b[2] * dn[2];
    for (int j = 0; j < 3; ++j) {
        e1[j] = Dual<T>(a[j], -ca * n[j]);
        e2[j] = Dual<T>(b[j], -cb * n[j]);
    }
}

template <typename S>
__device__ __forceinline__ void gluon_basis(const S* p, S* e1, S* e2)
{
    if constexpr (is_dual<S>::value) {
        gluon_basis_dual(p, e1, e2);
        return;
    }
    const double r2 = 0.70710678118654752440;
    const S pt2 = p[1] * p[1] + p[2] * p[2];
    const S pa = sqrt(pt2 + p[3] * p[3]);
    const S pt = sqrt(pt2);
    const S ct = p[3] / pa, st = pt / pa;
    const S cp = val(pt) > 0.0 ? p[1] / pt : S(1.0);
    const S sp = val(pt) > 0.0 ? p[2] / pt : S(0.0);
    e1[0] = r2 * ct * cp; e1[1] = r2 * ct * sp; e1[2] = -r2 * st;
    e2[0] = -r2 * sp;     e2[1] = r2 * cp;      e2[2] = S(0.0);
}

// Helicity eigenspinors and omega_+/- of a fermion of mass m (FP64);
// omega_- = m / omega_+ avoids the cancellation in E - |p|, and is exactly 0 for a
// massless fermion (E - |p| there is rounding), so that massless spinors have exact
// chirality and helicity-violating amplitudes vanish exactly.
template <typename R, typename S> __device__ __forceinline__ FermionBasis<R> fermion_basis(const S* p, S m)
{
    FermionBasis<R> f;
    const S pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    const S ppz = pa + p[3];
    const S omp = sqrt(p[0] + pa);
    const S omm = val(m) > 0.0 ? m / omp : S(0.0);
    f.om[0] = R(omp); f.om[1] = R(omm);
    if (val(ppz) > 1e-12 * (val(pa) + 1e-300)) {
        const S n = 1.0 / sqrt(2.0 * pa * ppz);
        f.chi[0][0] = mkc(R(ppz * n), R(0));
        f.chi[0][1] = mkc(R(p[1] * n), R(p[2] * n));
        f.chi[1][0] = mkc(R(-p[1] * n), R(p[2] * n));
        f.chi[1][1] = mkc(R(ppz * n), R(0));
    } else {
        f.chi[0][0] = mkc(R(0), R(0)); f.chi[0][1] = mkc(R(1), R(0));
        f.chi[1][0] = mkc(R(-1), R(0)); f.chi[1][1] = mkc(R(0), R(0));
    }
    return f;
}

}  // namespace mf
