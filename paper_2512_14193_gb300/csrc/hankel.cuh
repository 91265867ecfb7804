// Device evaluation of the Hankel functions H0^(1)(z), H1^(1)(z) for complex z, Re z > 0
// (principal branch), in FP64.  These build every kernel of section 2.2:
// G = (i/4) H0^(1)(k r) and its normal derivatives (H0' = -H1).
//
// Three zones by |z|, each accurate to about 1e-14 relative in |H|:
//  * |z| < 3    : ascending series of J0, J1, Y0, Y1, summed while (|z|^2/4)^m/(m!)^2 > 1e-17
//    (at most 14 terms).
//  * 3 <= |z| < 80 : Taylor expansion about the nearest anchor z0 of a grid with spacing 1/4
//    (|z - z0| <= 0.177).  The Taylor coefficients of H0 about z0 follow from Bessel's equation
//    z^2 y'' + z y' + z^2 y = 0 written in delta = z - z0:
//       z0^2 (k+1)(k+2) a_{k+2} = -[ z0 (k+1)(2k+1) a_{k+1} + (k^2 + z0^2) a_k
//                                    + 2 z0 a_{k-1} + a_{k-2} ],
//    a_0 = H0(z0), a_1 = -H1(z0); H1(z) = -H0'(z) is the differentiated series.  The host table
//    (hankel_table.cu: ODE integration in double-double) holds a_0 .. a_18 for every anchor, so
//    the device evaluates the polynomial and its derivative by Horner's scheme: 18 complex
//    multiply-adds each, the nine of a_8 .. a_0 in FP64 (72 FP64 FMAs), the rest in FP32.
//  * |z| >= 80  : Hankel's asymptotic expansion
//       H_nu(z) ~ sqrt(2/(pi z)) e^{i(z - nu pi/2 - pi/4)} sum_k i^k a_k(nu) / z^k,
//       a_k(nu) = prod_{j=1..k} (4nu^2 - (2j-1)^2) / (k! 8^k),
//    summed until the terms fall below 1e-17 (at most 40 terms; about 9 at |z| = 80).  A Horner
//    pass costs about a quarter of the FP64 work of this zone (two complex reciprocals, a complex
//    root, FP64 sincos and exp), which is why the Taylor table reaches out to |z| = 80.
// GB300 runs FP64 at 1/64 of its FP32 rate, and the series terms fall fast: past the first six
// terms of the asymptotic series (|a_7 / z^7| < 1e-8 for |z| >= 20), the first nine of the Taylor
// one (relative 3e-11 for H0, 2e-9 for the differentiated H1) and the first nine of the ascending
// one (|w|^10/(10!)^2 < 2.5e-10) the rest of the sum is below 1e-8 of it, so those terms are
// formed and summed in FP32 (their rounding errors stay near 1e-15 of the result) and added to
// the FP64 sum once.  The leading terms, log, exp, sincos and the roots stay FP64.
#pragma once
#include "common.cuh"

namespace hk {

constexpr double R_SERIES = 3.0;
constexpr double R_ASYM = 80.0;
constexpr double EULER_GAMMA = 0.57721566490153286060651209008240243;
constexpr double TWO_OVER_PI = 0.63661977236758134307553505349005745;
constexpr double ONE_OVER_PI = 0.31830988618379067153776752674502872;

__device__ __forceinline__ float2 f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 fscale(float2 v, float s) { return make_float2(v.x * s, v.y * s); }

__device__ __forceinline__ double2 clog(double2 z) {
    return make_double2(log(hypot(z.x, z.y)), atan2(z.y, z.x));
}

// principal square root
__device__ __forceinline__ double2 csqrt(double2 w) {
    double m = hypot(w.x, w.y);
    if (m == 0.0) return make_double2(0.0, 0.0);
    double s = sqrt(0.5 * (m + fabs(w.x)));
    if (w.x >= 0.0) return make_double2(s, w.y / (2.0 * s));
    return make_double2(fabs(w.y) / (2.0 * s), copysign(s, w.y));
}

__device__ __forceinline__ void series(double2 z, double2& h0, double2& h1) {
    // w = -z^2/4; t0_m = w^m/(m!)^2, t1_m = w^m/(m!(m+1)!)
    double2 w = cscale(cmul(z, z), -0.25);
    // |w|^m/(m!)^2 <= 1e-17 for |w| <= THR[m-1] (and the later terms are smaller still): the sums
    // stop at the first such m, taken from |w| in FP32 once rather than from FP64 tests of the
    // terms.  |w| < 2.25 in this zone, so at most 14 terms are summed (at |z| = 3), 9 for |z| <= 1.
    constexpr float THR[15] = {1e-17f,    6.32456e-9f, 7.11379e-6f, 2.75490e-4f, 2.70192e-3f,
                               1.31556e-2f, 4.25859e-2f, 0.106263f,  0.222133f,  0.409216f,
                               0.686394f, 1.07166f,    1.58169f,    2.23167f,    3.03529f};
    const float2 zf = f2(z);
    const float wa = 0.25f * (zf.x * zf.x + zf.y * zf.y);
    double2 t0 = make_double2(1.0, 0.0), t1 = make_double2(1.0, 0.0);
    double2 J0 = t0, J1 = t1;
    double2 S0 = make_double2(0.0, 0.0);                      // sum H_m t0_m
    double2 S1 = cscale(t1, -2.0 * EULER_GAMMA + 1.0);        // sum (psi(m+1)+psi(m+2)) t1_m, m = 0 term
    double Hm = 0.0;
    constexpr int M64 = 10;  // terms 1 .. 9 in FP64; from term 10 on |t_m| < 2.5e-10 |t_0|, so FP32
#pragma unroll
    for (int m = 1; m < M64; ++m) {
        if (wa <= THR[m - 1]) break;
        double dm = (double)m;
        t0 = cscale(cmul(t0, w), 1.0 / (dm * dm));
        t1 = cscale(cmul(t1, w), 1.0 / (dm * (dm + 1.0)));
        Hm += 1.0 / dm;
        J0 = cadd(J0, t0);
        J1 = cadd(J1, t1);
        S0 = cadd(S0, cscale(t0, Hm));
        S1 = cadd(S1, cscale(t1, -2.0 * EULER_GAMMA + 2.0 * Hm + 1.0 / (dm + 1.0)));
    }
    if (wa > THR[M64 - 1]) {
        // the same sums in FP32 from term 10 on, added to the FP64 sums once
        const float2 fw = f2(w);
        float2 ft0 = f2(t0), ft1 = f2(t1);
        float2 fJ0 = make_float2(0.f, 0.f), fJ1 = fJ0, fS0 = fJ0, fS1 = fJ0;
        float fH = (float)Hm;
#pragma unroll
        for (int m = M64; m < 16; ++m) {
            if (wa <= THR[m - 1]) break;
            const float dm = (float)m;
            ft0 = fscale(cmul(ft0, fw), 1.0f / (dm * dm));
            ft1 = fscale(cmul(ft1, fw), 1.0f / (dm * (dm + 1.0f)));
            fH += 1.0f / dm;
            fJ0 = cadd(fJ0, ft0);
            fJ1 = cadd(fJ1, ft1);
            fS0 = cadd(fS0, fscale(ft0, fH));
            fS1 = cadd(fS1, fscale(ft1, (float)(-2.0 * EULER_GAMMA) + 2.0f * fH + 1.0f / (dm + 1.0f)));
        }
        J0 = cadd(J0, make_double2(fJ0.x, fJ0.y));
        J1 = cadd(J1, make_double2(fJ1.x, fJ1.y));
        S0 = cadd(S0, make_double2(fS0.x, fS0.y));
        S1 = cadd(S1, make_double2(fS1.x, fS1.y));
    }
    double2 zh = cscale(z, 0.5);
    J1 = cmul(J1, zh);
    double2 L = clog(zh);
    // Y0 = (2/pi)(ln(z/2) + gamma) J0 - (2/pi) S0
    double2 Y0 = csub(cscale(cmul(make_double2(L.x + EULER_GAMMA, L.y), J0), TWO_OVER_PI), cscale(S0, TWO_OVER_PI));
    // Y1 = -2/(pi z) + (2/pi) ln(z/2) J1 - (1/pi)(z/2) S1
    double2 Y1 = cscale(cinv(z), -TWO_OVER_PI);
    Y1 = cadd(Y1, cscale(cmul(L, J1), TWO_OVER_PI));
    Y1 = csub(Y1, cscale(cmul(zh, S1), ONE_OVER_PI));
    h0 = make_double2(J0.x - Y0.y, J0.y + Y0.x);  // J0 + i Y0
    h1 = make_double2(J1.x - Y1.y, J1.y + Y1.x);
}

__device__ __forceinline__ void taylor(double2 z, const HankelTable& T, double2& h0, double2& h1) {
    int ix = __double2int_rn((z.x - T.re0) * T.inv_step);
    int iy = __double2int_rn((z.y - T.im0) * T.inv_step);
    ix = min(max(ix, 0), T.nx - 1);
    iy = min(max(iy, 0), T.ny - 1);
    const double2 z0 = make_double2(T.re0 + ix * T.step, T.im0 + iy * T.step);
    const double2* C = T.c + (long)HT_SLOTS * ((long)iy * T.nx + ix);
    const double2 d = csub(z, z0);
    // Horner's scheme for P(d) = sum a_k d^k and its derivative together (Q <- Q d + P before
    // P <- P d + a_k): a_18 .. a_9 in FP32, then a_8 .. a_0 in FP64.  H0 = P, H1 = -P'.
    const float4* C32 = reinterpret_cast<const float4*>(C + HT_K64);
    float2 c32[HT_K32];
#pragma unroll
    for (int j = 0; j < HT_K32 / 2; ++j) {
        const float4 v = __ldg(C32 + j);
        c32[2 * j] = make_float2(v.x, v.y);
        c32[2 * j + 1] = make_float2(v.z, v.w);
    }
    const float2 fd = f2(d);
    float2 fp = c32[HT_K32 - 1], fq = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = HT_K32 - 2; j >= 0; --j) {
        fq = cadd(cmul(fq, fd), fp);
        fp = cadd(cmul(fp, fd), c32[j]);
    }
    double2 P = make_double2(fp.x, fp.y), Q = make_double2(fq.x, fq.y);
#pragma unroll
    for (int k = HT_K64 - 1; k >= 0; --k) {
        const double2 ak = __ldg(C + k);
        Q = make_double2(fma(Q.x, d.x, fma(-Q.y, d.y, P.x)), fma(Q.x, d.y, fma(Q.y, d.x, P.y)));
        P = make_double2(fma(P.x, d.x, fma(-P.y, d.y, ak.x)), fma(P.x, d.y, fma(P.y, d.x, ak.y)));
    }
    h0 = P;
    h1 = cneg(Q);
}

__device__ __forceinline__ void asym(double2 z, double2& h0, double2& h1) {
    double2 w = cmuli(cinv(z));  // i/z
    double2 t0 = make_double2(1.0, 0.0), t1 = t0, s0 = t0, s1 = t0;
    constexpr int K64 = 6;  // terms 1 .. 6 in FP64, the rest in FP32
    bool done = false;
    for (int k = 1; k <= K64; ++k) {
        double o = (double)(2 * k - 1);
        t0 = cscale(cmul(t0, w), (0.0 - o * o) / (8.0 * k));
        t1 = cscale(cmul(t1, w), (4.0 - o * o) / (8.0 * k));
        s0 = cadd(s0, t0);
        s1 = cadd(s1, t1);
        if (cnorm1(t0) <= 1e-17 * cnorm1(s0) && cnorm1(t1) <= 1e-17 * cnorm1(s1)) {
            done = true;
            break;
        }
    }
    if (!done) {
        const float2 fw = f2(w);
        float2 ft0 = f2(t0), ft1 = f2(t1), f0 = make_float2(0.f, 0.f), f1 = f0;
        const float n0 = 1e-17f * (float)cnorm1(s0), n1 = 1e-17f * (float)cnorm1(s1);
        for (int k = K64 + 1; k < 40; ++k) {
            const float o = (float)(2 * k - 1);
            ft0 = fscale(cmul(ft0, fw), (0.f - o * o) / (8.f * (float)k));
            ft1 = fscale(cmul(ft1, fw), (4.f - o * o) / (8.f * (float)k));
            f0 = cadd(f0, ft0);
            f1 = cadd(f1, ft1);
            if (cnorm1(ft0) <= n0 && cnorm1(ft1) <= n1) break;
        }
        s0 = cadd(s0, make_double2(f0.x, f0.y));
        s1 = cadd(s1, make_double2(f1.x, f1.y));
    }
    // c = sqrt(2/(pi z)) * exp(i (z - pi/4)); the -pi/4 is applied as the exact rotation
    // (1 - i)/sqrt(2) after sincos(Re z): subtracting pi/4 from a large Re z in FP64 would lose
    // up to half an ulp of the argument (5e-14 of phase at |z| = 550).
    double2 c = csqrt(cscale(cinv(z), TWO_OVER_PI));
    double sn, cs;
    sincos(z.x, &sn, &cs);
    double e = exp(-z.y) * 0.70710678118654752440;
    c = cmul(c, make_double2(e * (cs + sn), e * (sn - cs)));
    h0 = cmul(c, s0);
    h1 = cneg(cmuli(cmul(c, s1)));  // -i c s1
}

__device__ __forceinline__ void hankel01(double2 z, const HankelTable& T, double2& h0, double2& h1) {
    const double r2 = z.x * z.x + z.y * z.y;
    if (r2 < R_SERIES * R_SERIES) series(z, h0, h1);
    else if (r2 < R_ASYM * R_ASYM) taylor(z, T, h0, h1);
    else asym(z, h0, h1);
}

}  // namespace hk
