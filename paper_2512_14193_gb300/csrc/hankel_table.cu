// Host construction of the Hankel anchor table used by the device Taylor zone (hankel.cuh).
//
// Anchors z0 = re0 + ix*step + i (im0 + iy*step), step = 1/4, cover Re z0 in [0, 81] and
// Im z0 in [-81, 81]; each stores (H0^(1)(z0), H1^(1)(z0)).  Values are produced without
// special-function libraries.  For 21 < |z0| <= 81, Hankel's asymptotic expansion is accurate to a
// few units of FP64 rounding and gives them directly.  Inside, along each grid row (fixed
// Im z0 = y) start at a point with |z| >= 21 and integrate Bessel's equation
// z^2 y'' + z y' + z^2 y = 0 leftwards in steps of -1/4 with Taylor series summed in
// double-double arithmetic (about 32 digits), down to |z| < 2.5 or Re z = 0.  Along a row the
// second solution H^(2) keeps a fixed size ratio e^{2y} to H^(1), so the start error neither
// grows nor is amplified; every anchor is accurate to about 1e-16 relative.  Only anchors with
// 2.5 <= |z0| <= 81 are filled (the Taylor zone uses 3 <= |z| < 80 and the nearest anchor is
// within 0.177).  Rows are built in parallel on the host's cores.
//
// For the device, every filled anchor also gets the Taylor coefficients a_0 .. a_18 of H0 about it
// (a_0 = H0(z0), a_1 = H0'(z0) = -H1(z0), the rest by the recurrence Bessel's equation gives in
// d = z - z0), computed in double-double from the double-double values of the integration and
// rounded once: the device then evaluates H0(z0 + d) and H1 = -H0' by Horner's scheme.  Relative to
// a_0, |a_k| 0.177^k < 3e-11 from k = 9 on (at |z0| = 2.8, and smaller further out; the derivative
// scales term k by k/0.177), so a_9 .. a_18 are kept in FP32, and at k = 19 the terms are below
// 1e-19 of the sum.  In the device's domain (arg z in [-70, 60] degrees) |H0| stays within
// [1e-31, 1e32], so the FP32 coefficients neither overflow nor lose more than terms below 1e-22.
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <string>
#include <thread>
#include <utility>
#include <vector>

namespace {

// ---- double-double ----------------------------------------------------------------------------
struct dd {
    double hi, lo;
};
inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
inline dd operator+(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd x) { return {-x.hi, -x.lo}; }
inline dd operator-(dd x, dd y) { return x + (-y); }
inline dd operator*(dd x, dd y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator*(dd x, double y) {
    dd p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return quick_two_sum(p.hi, p.lo);
}
inline dd ddiv(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * q1;
    double q2 = r.hi / b.hi;
    r = r - b * q2;
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return q + dd{q3, 0.0};
}
inline dd mkdd(double a) { return {a, 0.0}; }

struct cdd {
    dd re, im;
};
inline cdd operator+(cdd a, cdd b) { return {a.re + b.re, a.im + b.im}; }
inline cdd operator*(cdd a, cdd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cdd operator*(cdd a, double s) { return {a.re * s, a.im * s}; }
inline cdd cinv_dd(cdd a) {
    dd den = a.re * a.re + a.im * a.im;
    return {ddiv(a.re, den), ddiv(-a.im, den)};
}
inline double mag1(cdd a) { return std::fabs(a.re.hi) + std::fabs(a.im.hi); }

// ---- double complex helpers for the asymptotic start --------------------------------------------
struct cd {
    double re, im;
};
inline cd mul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cd inv(cd a) {
    double d = a.re * a.re + a.im * a.im;
    return {a.re / d, -a.im / d};
}

// H0, H1 by Hankel's asymptotic expansion (|z| >= 21: terms fall below 1e-17 before diverging)
void asym_start(double x, double y, cd& h0, cd& h1) {
    cd z{x, y};
    cd w = inv(z);
    w = {-w.im, w.re};  // i/z
    cd t0{1, 0}, t1{1, 0}, s0{1, 0}, s1{1, 0};
    double prev0 = 1.0, prev1 = 1.0;
    for (int k = 1; k < 80; ++k) {
        double o = 2.0 * k - 1.0;
        cd n0 = mul(t0, w), n1 = mul(t1, w);
        n0 = {n0.re * (-o * o) / (8.0 * k), n0.im * (-o * o) / (8.0 * k)};
        n1 = {n1.re * (4.0 - o * o) / (8.0 * k), n1.im * (4.0 - o * o) / (8.0 * k)};
        double m0 = std::fabs(n0.re) + std::fabs(n0.im), m1 = std::fabs(n1.re) + std::fabs(n1.im);
        if (m0 > prev0 || m1 > prev1) break;  // past the smallest term of the divergent series
        t0 = n0;
        t1 = n1;
        s0 = {s0.re + t0.re, s0.im + t0.im};
        s1 = {s1.re + t1.re, s1.im + t1.im};
        prev0 = m0;
        prev1 = m1;
        if (m0 < 1e-19 && m1 < 1e-19) break;
    }
    // sqrt(2/(pi z)) via polar form
    double r = std::hypot(x, y), th = std::atan2(y, x);
    double m = std::sqrt(2.0 / (M_PI * r));
    cd c{m * std::cos(-0.5 * th), m * std::sin(-0.5 * th)};
    double e = std::exp(-y);
    const double r2 = 0.70710678118654752440;  // e^{-i pi/4} applied exactly
    cd ph{e * r2 * (std::cos(x) + std::sin(x)), e * r2 * (std::sin(x) - std::cos(x))};
    c = mul(c, ph);
    h0 = mul(c, s0);
    cd cs1 = mul(c, s1);
    h1 = {cs1.im, -cs1.re};  // -i c s1
}

// One Taylor step of Bessel's equation (order 0) from z0 to z0 + d (d real) in double-double.
// In: y = H0(z0), yp = H0'(z0).  Out: values at z0 + d.
void taylor_step(cdd z0, double d, cdd& y, cdd& yp) {
    cdd z0sq = z0 * z0;
    cdd iz2 = cinv_dd(z0sq);
    cdd am2{mkdd(0), mkdd(0)}, am1 = am2;
    cdd ak = y, ak1 = yp;
    cdd s0 = y + ak1 * d;
    cdd s1 = ak1;
    double dpow = d;  // d^(k+1), exact for d = -1/4 up to large k
    for (int k = 0; k < 120; ++k) {
        double kk = (double)k;
        cdd br = (z0 * ak1) * ((kk + 1.0) * (2.0 * kk + 1.0));
        cdd c2 = {z0sq.re + mkdd(kk * kk), z0sq.im};
        br = br + c2 * ak;
        br = br + (z0 * am1) * 2.0;
        br = br + am2;
        // a_{k+2} = -br / (z0^2 (k+1)(k+2)); 1/((k+1)(k+2)) is inexact in binary, so divide in dd
        cdd t = br * iz2;
        dd den = mkdd((kk + 1.0) * (kk + 2.0));
        cdd an = {-ddiv(t.re, den), -ddiv(t.im, den)};
        cdd t1 = an * (dpow * (kk + 2.0));
        dpow *= d;
        cdd t0 = an * dpow;
        s0 = s0 + t0;
        s1 = s1 + t1;
        am2 = am1;
        am1 = ak;
        ak = ak1;
        ak1 = an;
        if (mag1(t0) < 1e-34 * mag1(s0) && mag1(t1) < 1e-34 * mag1(s1)) break;
    }
    y = s0;
    yp = s1;
}

// Taylor coefficients a_0 .. a_{n-1} of H0 about z0 from a_0 = y = H0(z0), a_1 = yp = H0'(z0), by the
// recurrence taylor_step sums: z0^2 (k+1)(k+2) a_{k+2} = -[z0 (k+1)(2k+1) a_{k+1} + (k^2 + z0^2) a_k
// + 2 z0 a_{k-1} + a_{k-2}].
void taylor_coefs(cdd z0, cdd y, cdd yp, cdd* a, int n) {
    const cdd z0sq = z0 * z0;
    const cdd iz2 = cinv_dd(z0sq);
    a[0] = y;
    a[1] = yp;
    for (int k = 0; k + 2 < n; ++k) {
        const double kk = (double)k;
        cdd br = (z0 * a[k + 1]) * ((kk + 1.0) * (2.0 * kk + 1.0));
        const cdd c2 = {z0sq.re + mkdd(kk * kk), z0sq.im};
        br = br + c2 * a[k];
        if (k >= 1) br = br + (z0 * a[k - 1]) * 2.0;
        if (k >= 2) br = br + a[k - 2];
        const cdd t = br * iz2;
        const dd den = mkdd((kk + 1.0) * (kk + 2.0));
        a[k + 2] = {-ddiv(t.re, den), -ddiv(t.im, den)};
    }
}

std::vector<double2> g_table;
std::vector<double2> g_coef;
int g_nx = 0, g_ny = 0;
constexpr double R_ODE = 21.0;  // anchors inside come from the ODE integration
constexpr double R_TAB = 81.0;  // table radius (the device Taylor zone ends at |z| = 80)
const double g_step = 0.25, g_re0 = 0.0, g_im0 = -R_TAB;
std::once_flag g_once;

// Fills anchor (ix, iy) at z0 = x + i y from y = H0(z0), yp = H0'(z0): the anchor pair and the
// Taylor coefficient block.
void store(int iy, int ix, double x, double y, cdd Y, cdd Yp) {
    size_t o = 2 * ((size_t)iy * g_nx + ix);
    g_table[o] = make_double2(Y.re.hi + Y.re.lo, Y.im.hi + Y.im.lo);
    g_table[o + 1] = make_double2(-(Yp.re.hi + Yp.re.lo), -(Yp.im.hi + Yp.im.lo));
    cdd a[HT_K64 + HT_K32];
    taylor_coefs(cdd{mkdd(x), mkdd(y)}, Y, Yp, a, HT_K64 + HT_K32);
    double2* blk = &g_coef[(size_t)HT_SLOTS * ((size_t)iy * g_nx + ix)];
    for (int k = 0; k < HT_K64; ++k) blk[k] = make_double2(a[k].re.hi + a[k].re.lo, a[k].im.hi + a[k].im.lo);
    float f[2 * HT_K32];
    for (int j = 0; j < HT_K32; ++j) {
        const cdd& v = a[HT_K64 + j];
        f[2 * j] = (float)(v.re.hi + v.re.lo);
        f[2 * j + 1] = (float)(v.im.hi + v.im.lo);
    }
    std::memcpy(blk + HT_K64, f, sizeof f);
}

// One grid row (fixed Im z0 = y): the anchors with R_ODE < |z0| <= R_TAB straight from Hankel's
// asymptotic expansion, then those with 2.5 <= |z0| <= R_ODE by integrating Bessel's equation
// leftwards from the first grid point with |z| >= R_ODE.
void build_row(int iy) {
    const double y = g_im0 + iy * g_step;
    for (int ix = 0; ix < g_nx; ++ix) {
        const double x = g_re0 + ix * g_step;
        const double r = std::hypot(x, y);
        if (r <= R_ODE + 1e-12 || r > R_TAB + 1e-12) continue;
        cd h0, h1;
        asym_start(x, y, h0, h1);
        store(iy, ix, x, y, cdd{mkdd(h0.re), mkdd(h0.im)}, cdd{mkdd(-h1.re), mkdd(-h1.im)});
    }
    double xs = std::ceil(std::sqrt(std::fmax(0.0, R_ODE * R_ODE - y * y)) / g_step) * g_step;
    cd h0, h1;
    asym_start(xs, y, h0, h1);
    cdd Y{mkdd(h0.re), mkdd(h0.im)};
    cdd Yp{mkdd(-h1.re), mkdd(-h1.im)};  // H0' = -H1
    double x = xs;
    while (true) {
        int ix = (int)std::lround((x - g_re0) / g_step);
        double r = std::hypot(x, y);
        if (ix < g_nx && r <= R_ODE + 1e-12) store(iy, ix, x, y, Y, Yp);
        if (x <= g_re0 + 1e-12 || r < 2.5) break;
        cdd z0{mkdd(x), mkdd(y)};
        taylor_step(z0, -g_step, Y, Yp);
        x -= g_step;
    }
}

void build() {
    g_nx = (int)std::lround((R_TAB - g_re0) / g_step) + 1;   // Re 0 .. R_TAB
    g_ny = (int)std::lround(-2.0 * g_im0 / g_step) + 1;      // Im -R_TAB .. R_TAB
    g_table.assign((size_t)g_nx * g_ny * 2, make_double2(0.0, 0.0));
    g_coef.assign((size_t)g_nx * g_ny * HT_SLOTS, make_double2(0.0, 0.0));
    // rows are independent and write disjoint parts of the tables
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = (int)std::max(1u, std::min(hw, 32u));
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([t, nt]() {
            for (int iy = t; iy < g_ny; iy += nt) build_row(iy);
        });
    for (auto& x : th) x.join();
}

}  // namespace

const std::vector<double2>& hankel_anchor_host(int& nx, int& ny, double& re0, double& im0, double& step) {
    std::call_once(g_once, build);
    nx = g_nx;
    ny = g_ny;
    re0 = g_re0;
    im0 = g_im0;
    step = g_step;
    return g_table;
}

const std::vector<double2>& hankel_coef_host() {
    std::call_once(g_once, build);
    return g_coef;
}

unsigned long long cuda_context_id() {
    using GetCurrent = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static const std::pair<GetCurrent, GetId> fns = []() {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        const bool ok =
            cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess;
        if (!ok) {
            cudaGetLastError();
            return std::pair<GetCurrent, GetId>(nullptr, nullptr);
        }
        return std::pair<GetCurrent, GetId>(reinterpret_cast<GetCurrent>(a), reinterpret_cast<GetId>(b));
    }();
    if (fns.first == nullptr || fns.second == nullptr) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (fns.first(&ctx) != 0 || ctx == nullptr || fns.second(ctx, &id) != 0) return 0;
    return id;
}

namespace {
constexpr int TAB_MAX_DEVICES = 64;
std::mutex g_dev_mu;
double2* g_dev_tab[TAB_MAX_DEVICES] = {};
unsigned long long g_dev_ctx[TAB_MAX_DEVICES] = {};  // the context each copy was uploaded in
}  // namespace

bm_status hankel_table_device(int dev, const double2** out) {
    *out = nullptr;
    if (dev < 0 || dev >= TAB_MAX_DEVICES) {
        bm_set_error("Hankel table: device index " + std::to_string(dev) + " out of range");
        return BM_EINVAL;
    }
    const std::vector<double2>& tab = hankel_coef_host();
    const unsigned long long ctx = cuda_context_id();
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (g_dev_tab[dev] == nullptr || ctx == 0 || ctx != g_dev_ctx[dev]) {
        // a copy from an earlier (reset) context is not freed: its memory went with that context
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, tab.size() * sizeof(double2));
        if (e == cudaSuccess) e = cudaMemcpy(p, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (p) cudaFree(p);
            cudaGetLastError();
            bm_set_error(std::string("Hankel table upload: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? BM_ENOMEM : BM_ECUDA;
        }
        g_dev_tab[dev] = static_cast<double2*>(p);
        g_dev_ctx[dev] = ctx;
    }
    *out = g_dev_tab[dev];
    return BM_OK;
}

extern "C" bm_status bm_hankel_anchor_table(double* out, int cap_anchors, int* nx, int* ny, double* re0,
                                            double* im0, double* step) {
    int a, b;
    double r0, i0, s;
    const std::vector<double2>& t = hankel_anchor_host(a, b, r0, i0, s);
    if (nx) *nx = a;
    if (ny) *ny = b;
    if (re0) *re0 = r0;
    if (im0) *im0 = i0;
    if (step) *step = s;
    if (out) {
        if (cap_anchors < a * b) return BM_EINVAL;
        for (size_t i = 0; i < t.size(); ++i) {
            out[2 * i] = t[i].x;
            out[2 * i + 1] = t[i].y;
        }
    }
    return BM_OK;
}

extern "C" bm_status bm_hankel_taylor_table(double* out, int cap_anchors, int* nterms) {
    int a, b;
    double r0, i0, st;
    hankel_anchor_host(a, b, r0, i0, st);
    const std::vector<double2>& t = hankel_coef_host();
    const int K = HT_K64 + HT_K32;
    if (nterms) *nterms = K;
    if (out) {
        if (cap_anchors < a * b) return BM_EINVAL;
        for (long q = 0; q < (long)a * b; ++q) {
            const double2* blk = t.data() + (size_t)HT_SLOTS * q;
            double* o = out + 2L * K * q;
            for (int k = 0; k < HT_K64; ++k) {
                o[2 * k] = blk[k].x;
                o[2 * k + 1] = blk[k].y;
            }
            float f[2 * HT_K32];
            std::memcpy(f, blk + HT_K64, sizeof f);
            for (int j = 0; j < 2 * HT_K32; ++j) o[2 * HT_K64 + j] = (double)f[j];
        }
    }
    return BM_OK;
}
