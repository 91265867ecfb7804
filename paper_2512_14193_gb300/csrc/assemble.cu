// Nystrom assembly of the direct-indirect (Eq. dis_mixedBM) and ordinary (Eq. dis_BM) systems,
// and the small O(N) / O(N M) kernels around it: node geometry, plane-wave right-hand sides,
// ||A||_inf, far field, the Hankel probe, and the FP32 operand packs for the tensor cores.
//
// Kernels of section 2.2 with d = x_i - y_j, r = |d|, w_j = h |x'(t_j)| (row i target, column j
// source):
//   S  = (i/4) H0(kr) w_j             D  = (ik/4) H1(kr) (d.nu_j)/r w_j
//   D* = -(ik/4) H1(kr) (d.nu_i)/r w_j
//   N  = (ik/4)[k H0 (d.nu_i)(d.nu_j)/r^2 - 2 H1 (d.nu_i)(d.nu_j)/r^3 + H1 (nu_i.nu_j)/r] w_j
// r is symmetric in (i, j), so one Hankel evaluation per wavenumber serves both (i, j) and
// (j, i): the swapped entry flips the sign of d and swaps which normal is the target's.
// Diagonal: the one-point zeta-corrected trapezoid rule of section 4 -
//   S_ii = w_i [i/4 - (ln(k/2) + gamma)/(2 pi) - ln(w_i/(2 pi))/(2 pi)]
//   D_ii = D*_ii = -kappa_i w_i/(4 pi)
//   N_ii = -pi/(6 h |x'_i|) - (k^2/(4 pi)) ln(h/(2 pi)) w_i
// Blocks (Theorem thm:LU): M13 = -S1, M23 = -(D*1 + I/2)/eps1, M31 = D0 - I/2 + beta N0,
// M32 = -eps0 (S0 + beta (D*0 + I/2)); ordinary (Eq. dis_BM, (2,2) block -eps1 S1):
// [M31, M32; D1 + I/2, -eps1 S1].
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "hankel.cuh"
#include "kernels.cuh"

namespace {

constexpr double PI = 3.14159265358979323846264338327950288;

__global__ void geom_kernel(int kind, double p0, double p1, double p2, int N, const double* __restrict__ user,
                            double* __restrict__ g) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double h = 2.0 * PI / N;
    double t = h * j;
    double x, y, dx, dy, ddx, ddy;
    if (kind == BM_CURVE_USER) {
        x = user[6 * j + 0];
        y = user[6 * j + 1];
        dx = user[6 * j + 2];
        dy = user[6 * j + 3];
        ddx = user[6 * j + 4];
        ddy = user[6 * j + 5];
    } else {
        double s, c;
        sincos(t, &s, &c);
        if (kind == BM_CURVE_CIRCLE) {
            x = p1 + p0 * c;
            y = p2 + p0 * s;
            dx = -p0 * s;
            dy = p0 * c;
            ddx = -p0 * c;
            ddy = -p0 * s;
        } else if (kind == BM_CURVE_ELLIPSE) {
            x = p0 * c;
            y = p1 * s;
            dx = -p0 * s;
            dy = p1 * c;
            ddx = -p0 * c;
            ddy = -p1 * s;
        } else if (kind == BM_CURVE_STAR) {
            double sm, cm;
            sincos(p2 * t, &sm, &cm);
            double r = p0 + p1 * cm, dr = -p1 * p2 * sm, ddr = -p1 * p2 * p2 * cm;
            x = r * c;
            y = r * s;
            dx = dr * c - r * s;
            dy = dr * s + r * c;
            ddx = ddr * c - 2.0 * dr * s - r * c;
            ddy = ddr * s + 2.0 * dr * c - r * s;
        } else {  // kite
            double s2, c2;
            sincos(2.0 * t, &s2, &c2);
            x = c + p0 * c2 - p0;
            y = p1 * s;
            dx = -s - 2.0 * p0 * s2;
            dy = p1 * c;
            ddx = -c - 4.0 * p0 * c2;
            ddy = -p1 * s;
        }
    }
    double sp = hypot(dx, dy);
    g[0 * N + j] = x;
    g[1 * N + j] = y;
    g[2 * N + j] = dy / sp;   // nu = (y', -x')/|x'|
    g[3 * N + j] = -dx / sp;
    g[4 * N + j] = sp;
    g[5 * N + j] = (dx * ddy - dy * ddx) / (sp * sp * sp);
    g[6 * N + j] = h * sp;
}

struct AsmArgs {
    int N;
    double h;
    double2 k0, k1, eps0, eps1, beta;
    HankelTable T;
    const double* g;
    double2* o[4];  // output quadrants (see header comment)
    long ld[4];
};

struct PairVals {
    // per wavenumber: cS = (i/4) H0, cD = (ik/4) H1 / r, B = N bracket (without weight)
    double2 cS0, cD0, B0, cS1, cD1;
};

__device__ __forceinline__ void pair_vals(const AsmArgs& a, double dx, double dy, double dni, double dnj, double ninj,
                                          PairVals& v) {
    double r = sqrt(dx * dx + dy * dy);
    double ir = 1.0 / r;
    double2 h0, h1;
    hk::hankel01(cscale(a.k0, r), a.T, h0, h1);
    double2 ik0 = cscale(cmuli(a.k0), 0.25);  // i k0 / 4
    v.cS0 = cscale(cmuli(h0), 0.25);
    v.cD0 = cscale(cmul(ik0, h1), ir);
    // N bracket: k H0 dni dnj / r^2 - 2 H1 dni dnj / r^3 + H1 ninj / r
    double pp = dni * dnj * ir * ir;
    double2 br = cscale(cmul(a.k0, h0), pp);
    br = cadd(br, cscale(h1, (ninj - 2.0 * pp) * ir));
    v.B0 = cmul(ik0, br);
    hk::hankel01(cscale(a.k1, r), a.T, h0, h1);
    double2 ik1 = cscale(cmuli(a.k1), 0.25);
    v.cS1 = cscale(cmuli(h0), 0.25);
    v.cD1 = cscale(cmul(ik1, h1), ir);
}

// Entries of the four output quadrants for an ordered pair with given target/source normal
// projections (dn_t = d.nu_target, dn_s = d.nu_source) and source weight ws.
template <int FORM>
__device__ __forceinline__ void outputs(const AsmArgs& a, const PairVals& v, double dn_t, double dn_s, double ws,
                                        double2 out[4]) {
    double2 S0 = cscale(v.cS0, ws);
    double2 D0 = cscale(v.cD0, dn_s * ws);
    double2 Ds0 = cscale(v.cD0, -dn_t * ws);
    double2 N0 = cscale(v.B0, ws);
    double2 S1 = cscale(v.cS1, ws);
    double2 M31 = cadd(D0, cmul(a.beta, N0));
    double2 M32 = cneg(cmul(a.eps0, cadd(S0, cmul(a.beta, Ds0))));
    if (FORM == BM_MIXED) {
        double2 Ds1 = cscale(v.cD1, -dn_t * ws);
        out[0] = cneg(S1);                      // M13
        out[1] = cneg(cdiv(Ds1, a.eps1));       // M23
        out[2] = M31;
        out[3] = M32;
    } else {
        double2 D1 = cscale(v.cD1, dn_s * ws);
        out[0] = M31;
        out[1] = M32;
        out[2] = D1;
        out[3] = cneg(cmul(a.eps1, S1));
    }
}

template <int FORM>
__device__ __forceinline__ void diag_outputs(const AsmArgs& a, int i, double2 out[4]) {
    const double* g = a.g;
    int N = a.N;
    double sp = g[4 * N + i], ka = g[5 * N + i], w = g[6 * N + i];
    const double g_e = hk::EULER_GAMMA;
    auto Sd = [&](double2 k) {
        double2 hk2 = cscale(k, 0.5);
        double2 L = hk::clog(hk2);
        double re = -(L.x + g_e) / (2.0 * PI) - log(w / (2.0 * PI)) / (2.0 * PI);
        double im = 0.25 - L.y / (2.0 * PI);
        return make_double2(w * re, w * im);
    };
    double Dd = -ka * w / (4.0 * PI);
    double lh = log(a.h / (2.0 * PI));
    double2 k0sq = cmul(a.k0, a.k0);
    double2 Nd = cadd(make_double2(-PI / (6.0 * a.h * sp), 0.0), cscale(k0sq, -lh * w / (4.0 * PI)));
    double2 S0 = Sd(a.k0), S1 = Sd(a.k1);
    double2 M31 = cadd(make_double2(Dd - 0.5, 0.0), cmul(a.beta, Nd));
    double2 M32 = cneg(cmul(a.eps0, cadd(S0, cmul(a.beta, make_double2(Dd + 0.5, 0.0)))));
    if (FORM == BM_MIXED) {
        out[0] = cneg(S1);
        out[1] = cneg(cdiv(make_double2(Dd + 0.5, 0.0), a.eps1));
        out[2] = M31;
        out[3] = M32;
    } else {
        out[0] = M31;
        out[1] = M32;
        out[2] = make_double2(Dd + 0.5, 0.0);
        out[3] = cneg(cmul(a.eps1, S1));
    }
}

constexpr int AT = 32;  // assembly tile
constexpr int AY = 8;   // threads in y

// One 32 x 32 tile pair (I <= J) of the assembled blocks, chosen by blockIdx.x.
template <int FORM>
__device__ __forceinline__ void assemble_tile(const AsmArgs& a) {
    extern __shared__ double2 st[];  // [4][AT][AT+1] staging of the transposed tile
    // decode the upper-triangular tile pair (I <= J) from the linear block index
    long idx = blockIdx.x;
    long J = (long)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (J * (J + 1) / 2 > idx) --J;
    while ((J + 1) * (J + 2) / 2 <= idx) ++J;
    long I = idx - J * (J + 1) / 2;
    const int N = a.N;
    const double* g = a.g;
    int tx = threadIdx.x, ty = threadIdx.y;
    int i = (int)I * AT + tx;
    bool diag_tile = (I == J);
    double xi = 0, yi = 0, nxi = 0, nyi = 0, wi = 0;
    if (i < N) {
        xi = g[i];
        yi = g[N + i];
        nxi = g[2 * N + i];
        nyi = g[3 * N + i];
        wi = g[6 * N + i];
    }
#pragma unroll 1
    for (int q = 0; q < AT / AY; ++q) {
        int jl = ty + AY * q;
        int j = (int)J * AT + jl;
        bool valid = (i < N) && (j < N);
        double2 o1[4], o2[4];
        if (valid) {
            if (i == j) {
                diag_outputs<FORM>(a, i, o1);
            } else {
                double xj = g[j], yj = g[N + j], nxj = g[2 * N + j], nyj = g[3 * N + j], wj = g[6 * N + j];
                double dx = xi - xj, dy = yi - yj;
                double dni = dx * nxi + dy * nyi, dnj = dx * nxj + dy * nyj, ninj = nxi * nxj + nyi * nyj;
                PairVals v;
                pair_vals(a, dx, dy, dni, dnj, ninj, v);
                // (i, j): target i, source j
                outputs<FORM>(a, v, dni, dnj, wj, o1);
                if (!diag_tile) {
                    // (j, i): d -> -d, target j (d.nu_j -> -dnj), source i (-dni)
                    outputs<FORM>(a, v, -dnj, -dni, wi, o2);
                }
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) a.o[b][(long)i + (long)j * a.ld[b]] = o1[b];
        }
        if (!diag_tile) {
#pragma unroll
            for (int b = 0; b < 4; ++b) st[(b * AT + jl) * (AT + 1) + tx] = valid ? o2[b] : make_double2(0, 0);
        }
    }
    if (diag_tile) return;
    __syncthreads();
    // write the transposed tile: entry (row j, col i); lanes run over j for coalescing
#pragma unroll 1
    for (int q = 0; q < AT / AY; ++q) {
        int il = ty + AY * q;
        int ii = (int)I * AT + il;
        int jj = (int)J * AT + tx;
        if (ii < N && jj < N) {
#pragma unroll
            for (int b = 0; b < 4; ++b) a.o[b][(long)jj + (long)ii * a.ld[b]] = st[(b * AT + tx) * (AT + 1) + il];
        }
    }
}

template <int FORM>
__global__ void __launch_bounds__(AT* AY) assemble_kernel(AsmArgs a) {
    assemble_tile<FORM>(a);
}

// Several systems of the same size at once (contour points of one curve): system blockIdx.z takes
// its wavenumbers, material constants and output blocks from args[blockIdx.z].
template <int FORM>
__global__ void __launch_bounds__(AT* AY) assemble_batch_kernel(const AsmArgs* __restrict__ args) {
    assemble_tile<FORM>(args[blockIdx.z]);
}

// row sums of |A| for ||A||_inf; rows of an m x ncols column-major block, plus `add` per row
__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}
// max over rows of (add + sum_j |A(i, j)|) into *out (an infinity-norm term of the backward error).
// CTA: 32 consecutive rows (lane = row, so every load instruction reads 32 consecutive entries),
// its 8 warps taking every 8th column, eight loads in flight per thread.  The moduli are formed in
// FP32 from the entries rounded to FP32 (by integer operations: the FP64 pipe is narrow) and each
// thread sums its columns in FP32, the eight warps' sums added in FP64: a relative error of a few
// 1e-6 at most, ample for a norm that only scales the backward error.
__global__ void __launch_bounds__(256) rownorm_kernel(const double2* __restrict__ A, long ld, int m, int ncols,
                                                      double add, double* out) {
    __shared__ double part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float sf = 0.f;
    if (i < m) {
        const double2* a = A + i;
        int j = warp;
        for (; j + 56 < ncols; j += 64) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = a[(long)(j + 8 * u) * ld];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float x = f32_rn(v[u].x), y = f32_rn(v[u].y);
                sf += sqrtf(fmaf(x, x, y * y));
            }
        }
        for (; j < ncols; j += 8) {
            const double2 v = a[(long)j * ld];
            const float x = f32_rn(v.x), y = f32_rn(v.y);
            sf += sqrtf(fmaf(x, x, y * y));
        }
    }
    // FP32 overflow (entries above ~1e19) falls back to the FP64 modulus for this thread's row
    double s = (double)sf;
    if (!isfinite(sf) && i < m) {
        s = 0.0;
        for (int j = warp; j < ncols; j += 8) {
            const double2 v = A[i + (long)j * ld];
            s += hypot(v.x, v.y);
        }
    }
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
        double t = 0.0;
        if (i < m) {
            t = add;
#pragma unroll
            for (int w = 0; w < 8; ++w) t += part[w][lane];
        }
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0 && t > 0) atomic_max_pos(out, t);
    }
}

__global__ void plane_wave_kernel(const double* __restrict__ g, int N, double2 k0, double2 beta,
                                  const double* __restrict__ ang, int nrhs, int form, double2* B, long ldb) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    int nsys = (form == BM_MIXED) ? 3 * N : 2 * N;
    if (r >= nsys || c >= nrhs) return;
    int off = (form == BM_MIXED) ? 2 * N : 0;
    double2 val = make_double2(0.0, 0.0);
    if (r >= off && r < off + N) {
        int j = r - off;
        double sa, ca;
        sincos(ang[c], &sa, &ca);
        double s = ca * g[j] + sa * g[N + j];
        double dn = ca * g[2 * N + j] + sa * g[3 * N + j];
        // u = exp(i k0 s), q = i k0 dn u
        double e = exp(-k0.y * s), sn, cs;
        sincos(k0.x * s, &sn, &cs);
        double2 u = make_double2(e * cs, e * sn);
        double2 q = cscale(cmul(cmuli(k0), u), dn);
        val = cneg(cadd(u, cmul(beta, q)));
    }
    B[r + (long)c * ldb] = val;
}

// Far field: U[m, c] = c0 sum_j w_j e^{-i k0 xhat_m . y_j} [(-i k0 xhat_m . nu_j) u_jc - eps0 q_jc],
// c0 = e^{i pi/4} / sqrt(8 pi k0).  A contraction over the nodes: with the weighted phases
// P_mj = w_j e^{-i k0 xhat_m . y_j}, U = c0 (Au X_u + Aq X_q), Au_mj = -i k0 (xhat_m . nu_j) P_mj,
// Aq_mj = -eps0 P_mj.  CTA: FF_MT = 8 angles x up to FF_CT = 128 right-hand sides x one of S node
// slices (S = the cluster size).  Per 32-node chunk the 8 x 32 phases (one FP64 exp and sincos
// each) are formed once, one per thread, and serve every column; each thread keeps the sums of one
// angle and columns oc, oc + 32, ...  The S slices' partial sums are added in rank order through
// distributed shared memory (deterministic, no workspace).
constexpr int FF_MT = 8, FF_JT = 32, FF_CT = 128, FF_THREADS = 256;
constexpr int FF_OUT = FF_MT * FF_CT / FF_THREADS;  // sums per thread

__device__ __forceinline__ double2 ld_cluster_d2(const double2* p, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(r) : "memory");
    return v;
}
__device__ __forceinline__ void ff_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(FF_THREADS) far_field_kernel(const double* __restrict__ g, int N, double2 k0,
                                                               double2 eps0, const double2* __restrict__ X, long ldx,
                                                               const double* __restrict__ ang, int M, int nrhs,
                                                               double2* U, long ldu) {
    extern __shared__ double2 ffs[];
    const int S = (int)gridDim.x, z = (int)blockIdx.x;  // node slice = rank in the cluster
    const int m0 = (int)blockIdx.y * FF_MT, c0 = (int)blockIdx.z * FF_CT;
    const int nc = min(FF_CT, nrhs - c0), ncp = nc + 1;  // padded row of the X chunk
    double2* sAu = ffs;                   // [FF_JT][FF_MT]
    double2* sAq = sAu + FF_JT * FF_MT;   // [FF_JT][FF_MT]
    double2* sXu = sAq + FF_JT * FF_MT;   // [FF_JT][ncp]
    double2* sXq = sXu + FF_JT * ncp;     // [FF_JT][ncp]
    const int t = (int)threadIdx.x;
    const int om = t % FF_MT, oc = t / FF_MT;  // this thread's angle (phases and sums) and first column
    const int pj = t / FF_MT;                  // this thread's node within a chunk (phases)
    const bool mok = m0 + om < M;
    double sa = 0.0, ca = 0.0;
    if (mok) sincos(ang[m0 + om], &sa, &ca);
    double2 acc[FF_OUT];
#pragma unroll
    for (int i = 0; i < FF_OUT; ++i) acc[i] = make_double2(0.0, 0.0);
    const int jb = (int)((long)z * N / S), je = (int)((long)(z + 1) * N / S);
    for (int jc = jb; jc < je; jc += FF_JT) {
        const int nj = min(FF_JT, je - jc);
        __syncthreads();  // the previous chunk has been read
        {
            double2 au = make_double2(0.0, 0.0), aq = au;
            if (mok && pj < nj) {
                const int j = jc + pj;
                const double sx = ca * g[j] + sa * g[N + j];
                const double xn = ca * g[2 * N + j] + sa * g[3 * N + j];
                const double e = exp(k0.y * sx) * g[6 * N + j];
                double sn, cs;
                sincos(-k0.x * sx, &sn, &cs);
                const double2 ph = make_double2(e * cs, e * sn);  // w_j e^{-i k0 s}
                au = cscale(cmul(cmuli(k0), ph), -xn);            // -i k0 (xhat . nu) w_j e^{-i k0 s}
                aq = cneg(cmul(eps0, ph));
            }
            sAu[pj * FF_MT + om] = au;
            sAq[pj * FF_MT + om] = aq;
        }
        for (int q = t; q < FF_JT * nc; q += FF_THREADS) {
            const int jj = q % FF_JT, cc = q / FF_JT;
            double2 u = make_double2(0.0, 0.0), v = u;
            if (jj < nj) {
                const double2* col = X + (long)(c0 + cc) * ldx + jc + jj;
                u = col[0];
                v = col[N];
            }
            sXu[jj * ncp + cc] = u;
            sXq[jj * ncp + cc] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < FF_JT; ++jj) {
            const double2 a = sAu[jj * FF_MT + om], b = sAq[jj * FF_MT + om];
#pragma unroll
            for (int i = 0; i < FF_OUT; ++i) {
                const int cc = oc + 32 * i;
                if (cc < nc) {
                    const double2 u = sXu[jj * ncp + cc], v = sXq[jj * ncp + cc];
                    acc[i].x = fma(a.x, u.x, fma(-a.y, u.y, fma(b.x, v.x, fma(-b.y, v.y, acc[i].x))));
                    acc[i].y = fma(a.x, u.y, fma(a.y, u.x, fma(b.x, v.y, fma(b.y, v.x, acc[i].y))));
                }
            }
        }
    }
    // this slice's partial sums into shared memory (o = column * 8 + angle), then rank z adds the
    // slices of its share of the outputs in rank order
    __syncthreads();
    double2* sP = sXu;
#pragma unroll
    for (int i = 0; i < FF_OUT; ++i) {
        const int cc = oc + 32 * i;
        if (cc < nc) sP[cc * FF_MT + om] = acc[i];
    }
    ff_cluster_sync();
    const double2 kk = hk::csqrt(cscale(k0, 8.0 * PI));
    const double2 cpre = cmul(make_double2(0.70710678118654752440, 0.70710678118654752440), cinv(kk));
    const int nout = FF_MT * nc;
    for (int o = z * FF_THREADS + t; o < nout; o += S * FF_THREADS) {
        double2 sum = make_double2(0.0, 0.0);
        for (int r = 0; r < S; ++r) sum = cadd(sum, ld_cluster_d2(sP + o, r));
        const int m = m0 + o % FF_MT, cc = c0 + o / FF_MT;
        if (m < M) U[m + (long)cc * ldu] = cmul(cpre, sum);
    }
    ff_cluster_sync();  // no CTA leaves while another still reads its shared memory
}

__global__ void hankel_probe_kernel(const double2* __restrict__ z, int n, HankelTable T, double2* h0, double2* h1) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a, b;
    hk::hankel01(z[i], T, a, b);
    h0[i] = a;
    h1[i] = b;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Schur A operand: Mbot (N x 2N col-major FP64) -> row-major [N][ldk] planar FP32, segments
// (3xTF32: [hi | hi | lo]); B operand: Mtop (2N x N) -> [N][ldk] with column n of Mtop as row n
// (3xTF32: [hi | lo | hi]).  Padding columns [nseg*K, ldk) are zeroed.
__global__ void pack_rowmajor_kernel(const double2* __restrict__ M, long ldm, int rows, int K, int split,
                                     float* __restrict__ Pr, float* __restrict__ Pi, long ldk) {
    __shared__ float2 t[32][33];
    int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int q = ty; q < 32; q += 8) {
        int r = r0 + tx, k = k0 + q;
        double2 v = (r < rows && k < K) ? M[r + (long)k * ldm] : make_double2(0, 0);
        t[q][tx] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        int r = r0 + q, k = k0 + tx;
        if (r >= rows || k >= K) continue;
        float2 v = t[tx][q];
        long o = (long)r * ldk + k;
        if (!split) {
            Pr[o] = v.x;
            Pi[o] = v.y;
        } else {
            float hr = tf32_rna(v.x), hi = tf32_rna(v.y);
            Pr[o] = hr;
            Pi[o] = hi;
            Pr[o + K] = hr;
            Pi[o + K] = hi;
            Pr[o + 2 * K] = v.x - hr;
            Pi[o + 2 * K] = v.y - hi;
        }
    }
}

__global__ void pack_colmajor_kernel(const double2* __restrict__ M, long ldm, int K, int cols, int split,
                                     float* __restrict__ Pr, float* __restrict__ Pi, long ldk) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long kext = split ? 3L * K : (long)K;
    long total = (long)cols * ldk;
    if (idx >= total) return;
    int n = (int)(idx / ldk);
    long kk = idx - (long)n * ldk;
    float vr = 0.f, vi = 0.f;
    if (kk < kext) {
        long k = kk % K;
        int seg = (int)(kk / K);
        double2 v = M[k + (long)n * ldm];
        float fr = (float)v.x, fi = (float)v.y;
        if (!split) {
            vr = fr;
            vi = fi;
        } else {
            float hr = tf32_rna(fr), hi = tf32_rna(fi);
            if (seg == 1) {
                vr = fr - hr;
                vi = fi - hi;
            } else {
                vr = hr;
                vi = hi;
            }
        }
    }
    Pr[idx] = vr;
    Pi[idx] = vi;
}

__global__ void pad_zero_rows_kernel(float* Pr, float* Pi, long ldk, int rows, long kext) {
    // zero the K padding [kext, ldk) of each row of a row-major pack
    long pad = ldk - kext;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pad <= 0 || idx >= (long)rows * pad) return;
    long r = idx / pad, c = kext + idx % pad;
    Pr[r * ldk + c] = 0.f;
    Pi[r * ldk + c] = 0.f;
}

__global__ void to_c32_kernel(const double2* __restrict__ A, long lda, int m, int n, float* Fr, float* Fi, long ldf) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    double2 v = A[i + (long)j * lda];
    Fr[i + (long)j * ldf] = (float)v.x;
    Fi[i + (long)j * ldf] = (float)v.y;
}


// ------------------------------------------------------------------------------------------------
// High-order zeta corrections (the "order 31" rule of section 5.3; order 2p + 3 for all four
// operators), added to the assembled blocks on the band |i - j| <= p + 1 around the diagonal.
//
// The punctured trapezoid sum of a kernel with an |x|^s singularity at the node x = 0 (x = s - t in
// the curve parameter, equispaced nodes x = jh) has the expansion
//     int |x|^s g dx = h sum_{j != 0} |jh|^s g(jh) - 2 sum_{k >= 0} zeta(-s-2k) h^(s+2k+1) g^(2k)(0) / (2k)!.
//  * log|x| (the derivative in s at s = 0; zeta(-2k) = 0 for k >= 1): the correction is
//    h ln(h/2pi) g(0) + 2 sum_{k>=1} zeta'(-2k) h^(2k+1) g^(2k)(0) / (2k)!, turned into weights
//    h tau_m on g(mh), |m| <= p, exact for even polynomials of degree <= 2p:
//        sum_{m=1..p} tau_m m^(2k) = zeta'(-2k), k = 1..p;  sigma_0 = -2 sum tau_m on the diagonal
//    (beyond the ln(h/2pi) of the one-point rule).  The kernels' log parts come from the
//    log(z/2) J_n(z) terms of Y_0, Y_1 (log r = log|x| + log(r/|x|), the second smooth):
//        S: -(1/2pi) J0(kr) w        D: -(k/2pi) J1(kr) (d.nu_s)/r w     D*: +(k/2pi) J1(kr) (d.nu_t)/r w
//        N: -(k/2pi) [k J0 (d.nu_t)(d.nu_s)/r^2 - 2 J1 (d.nu_t)(d.nu_s)/r^3 + J1 (nu_t.nu_s)/r] w
//  * x^-2 (N; zeta(0) = -1/2 and the series stops): -(pi^2/3h) g(0) (the one-point rule) plus
//    (h/2) g''(0), with g(x) = x^2 (N minus its log part) and g''(0) from the central stencil over
//    |m| <= p + 1; g(0) = 1 / (2 pi |x'(t)|).
// J_n(z) = (H_n(z) + conj(H_n(conj z))) / 2 reuses the Hankel evaluation (the conjugate argument
// stays in the supported sector).  One thread per (row, offset); every entry is touched by one
// thread.
constexpr int ZETA_PMAX = 20;

struct ZetaArgs {
    int p;
    double tau[ZETA_PMAX + 1];  // tau[0] = sigma_0, tau[m] for m = 1..p
    double c2[ZETA_PMAX + 2];   // second-derivative stencil weights c_0 .. c_{p+1}
};

__device__ __forceinline__ void bessel01(double2 z, const HankelTable& T, double2& j0, double2& j1) {
    double2 h0, h1, g0, g1;
    hk::hankel01(z, T, h0, h1);
    hk::hankel01(make_double2(z.x, -z.y), T, g0, g1);
    j0 = make_double2(0.5 * (h0.x + g0.x), 0.5 * (h0.y - g0.y));
    j1 = make_double2(0.5 * (h1.x + g1.x), 0.5 * (h1.y - g1.y));
}

template <int FORM>
__global__ void zeta_band_kernel(AsmArgs a, ZetaArgs zc) {
    const int W = 2 * zc.p + 3;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)a.N * W) return;
    const int N = a.N;
    const int i = (int)(idx / W);
    const int m = (int)(idx % W) - (zc.p + 1);
    const int j = ((i + m) % N + N) % N;
    const double* g = a.g;
    const double twopi = 2.0 * PI;
    double2 S0c = make_double2(0, 0), S1c = S0c, D0c = S0c, Ds0c = S0c, D1c = S0c, Ds1c = S0c, N0c = S0c;
    if (m == 0) {
        const double w = g[6 * N + i], sp = g[4 * N + i];
        S0c = make_double2(zc.tau[0] * (-w / twopi), 0.0);
        S1c = S0c;
        N0c = cscale(cmul(a.k0, a.k0), zc.tau[0] * (-w / (2.0 * twopi)));
        N0c.x += zc.c2[0] / (2.0 * a.h) / (twopi * sp);
    } else {
        const int am = m < 0 ? -m : m;
        const double logw = am <= zc.p ? zc.tau[am] : 0.0;
        const double xi = g[i], yi = g[N + i], nxi = g[2 * N + i], nyi = g[3 * N + i];
        const double xj = g[j], yj = g[N + j], nxj = g[2 * N + j], nyj = g[3 * N + j], wj = g[6 * N + j];
        const double dx = xi - xj, dy = yi - yj;
        const double r = sqrt(dx * dx + dy * dy), ir = 1.0 / r;
        const double dni = dx * nxi + dy * nyi, dnj = dx * nxj + dy * nyj, ninj = nxi * nxj + nyi * nyj;
        const double pp = dni * dnj * ir * ir;
        // wavenumber k0: log parts of S, D, D*, N and the full N entry
        double2 h0, h1, j0, j1;
        const double2 z0 = cscale(a.k0, r);
        hk::hankel01(z0, a.T, h0, h1);
        bessel01(z0, a.T, j0, j1);
        const double2 c0 = cscale(a.k0, 1.0 / twopi);  // k0 / 2pi
        const double2 AS0 = cscale(j0, -wj / twopi);
        const double2 AD0 = cscale(cmul(c0, j1), -dnj * ir * wj);
        const double2 ADs0 = cscale(cmul(c0, j1), dni * ir * wj);
        double2 brJ = cscale(cmul(a.k0, j0), pp);
        brJ = cadd(brJ, cscale(j1, (ninj - 2.0 * pp) * ir));
        const double2 AN0 = cscale(cmul(c0, brJ), -wj);
        double2 brH = cscale(cmul(a.k0, h0), pp);
        brH = cadd(brH, cscale(h1, (ninj - 2.0 * pp) * ir));
        const double2 Nfull = cscale(cmul(cscale(cmuli(a.k0), 0.25), brH), wj);
        const double2 Nnonlog = csub(Nfull, cscale(AN0, log(am * a.h)));
        S0c = cscale(AS0, logw);
        D0c = cscale(AD0, logw);
        Ds0c = cscale(ADs0, logw);
        N0c = cadd(cscale(AN0, logw), cscale(Nnonlog, 0.5 * zc.c2[am] * (double)am * (double)am));
        // wavenumber k1: log parts of S and D* (mixed) or D (ordinary)
        if (logw != 0.0) {
            bessel01(cscale(a.k1, r), a.T, j0, j1);
            const double2 c1 = cscale(a.k1, 1.0 / twopi);
            S1c = cscale(j0, -wj / twopi * logw);
            D1c = cscale(cmul(c1, j1), -dnj * ir * wj * logw);
            Ds1c = cscale(cmul(c1, j1), dni * ir * wj * logw);
        }
    }
    const double2 M31 = cadd(D0c, cmul(a.beta, N0c));
    const double2 M32 = cneg(cmul(a.eps0, cadd(S0c, cmul(a.beta, Ds0c))));
    double2 out[4];
    if (FORM == BM_MIXED) {
        out[0] = cneg(S1c);
        out[1] = cneg(cdiv(Ds1c, a.eps1));
        out[2] = M31;
        out[3] = M32;
    } else {
        out[0] = M31;
        out[1] = M32;
        out[2] = D1c;
        out[3] = cneg(cmul(a.eps1, S1c));
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        double2* e = a.o[b] + (long)i + (long)j * a.ld[b];
        *e = cadd(*e, out[b]);
    }
}

// zeta(s), s >= 3 odd, by Euler-Maclaurin summation with 11 terms and 7 Bernoulli corrections
double zeta_odd(int s) {
    const int M = 12;
    double sum = 0.0;
    for (int n = M - 1; n >= 1; --n) sum += std::pow((double)n, -s);
    const double Ms = std::pow((double)M, -s);
    sum += M * Ms / (s - 1) + 0.5 * Ms;
    const double B[7] = {1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66, -691.0 / 2730, 7.0 / 6};
    double fact = 1.0, rising = s, Mp = Ms / M;
    for (int j = 1; j <= 7; ++j) {
        fact *= (2.0 * j - 1) * (2.0 * j);
        sum += B[j - 1] / fact * rising * Mp;
        rising *= (s + 2.0 * j - 1) * (s + 2.0 * j);
        Mp /= (double)M * M;
    }
    return sum;
}

// Weights of the correction: tau_m solve sum_m (tau_m m^2) (m^2)^k = zeta'(-2(k+1)), k = 0..p-1,
// a Vandermonde system in the nodes m^2 solved by the Bjorck-Pereyra algorithm (accurate to
// rounding for positive increasing nodes); c_m is the closed form of the central second-derivative
// stencil of half-width q: c_m = 2 (-1)^(m+1) (q!)^2 / (m^2 (q-m)! (q+m)!), c_0 = -2 sum c_m.
ZetaArgs zeta_weights(int p) {
    ZetaArgs z{};
    z.p = p;
    std::vector<double> x(p), b(p);
    for (int m = 1; m <= p; ++m) x[m - 1] = (double)m * m;
    double f2k = 1.0, tp2k = 1.0;  // (2k)!, (2 pi)^(2k)
    for (int k = 1; k <= p; ++k) {
        f2k *= (2.0 * k - 1) * (2.0 * k);
        tp2k *= 4.0 * PI * PI;
        b[k - 1] = ((k % 2) ? -1.0 : 1.0) * f2k * zeta_odd(2 * k + 1) / (2.0 * tp2k);
    }
    const int n = p - 1;
    for (int k = 0; k < n; ++k)
        for (int i = n; i > k; --i) b[i] -= x[k] * b[i - 1];
    for (int k = n - 1; k >= 0; --k) {
        for (int i = k + 1; i <= n; ++i) b[i] /= (x[i] - x[i - k - 1]);
        for (int i = k; i < n; ++i) b[i] -= b[i + 1];
    }
    double sum = 0.0;
    for (int m = 1; m <= p; ++m) {
        z.tau[m] = b[m - 1] / x[m - 1];
        sum += z.tau[m];
    }
    z.tau[0] = -2.0 * sum;
    const int q = p + 1;
    double fq = 1.0;
    for (int t = 2; t <= q; ++t) fq *= t;
    double csum = 0.0;
    for (int m = 1; m <= q; ++m) {
        double den = (double)m * m;
        for (int t = 2; t <= q - m; ++t) den *= t;
        for (int t = 2; t <= q + m; ++t) den *= t;
        z.c2[m] = 2.0 * ((m % 2) ? 1.0 : -1.0) * fq * fq / den;
        csum += z.c2[m];
    }
    z.c2[0] = -2.0 * csum;
    return z;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
cudaError_t launch_geometry(cudaStream_t s, int kind, const double p[4], int N, const double* d_user, double* d_geom) {
    geom_kernel<<<ceil_div(N, 256), 256, 0, s>>>(kind, p[0], p[1], p[2], N, d_user, d_geom);
    return cudaGetLastError();
}

static AsmArgs asm_args(const bm_ctx* c) {
    AsmArgs a{};
    a.N = c->N;
    a.h = 2.0 * PI / c->N;
    a.k0 = c->k0;
    a.k1 = c->k1;
    a.eps0 = c->eps0;
    a.eps1 = c->eps1;
    a.beta = c->beta;
    a.T = c->htab;
    a.g = c->d_geom;
    long N = c->N;
    if (c->form == BM_MIXED) {
        a.o[0] = c->d_Mtop;
        a.o[1] = c->d_Mtop + N;
        a.o[2] = c->d_Mbot;
        a.o[3] = c->d_Mbot + N * c->ldbot;
        a.ld[0] = a.ld[1] = c->ldtop;
        a.ld[2] = a.ld[3] = c->ldbot;
    } else {
        a.o[0] = c->d_A;
        a.o[1] = c->d_A + N * c->ldA;
        a.o[2] = c->d_A + N;
        a.o[3] = c->d_A + N + N * c->ldA;
        a.ld[0] = a.ld[1] = a.ld[2] = a.ld[3] = c->ldA;
    }
    return a;
}

cudaError_t launch_assemble(cudaStream_t s, const bm_ctx* c) {
    const AsmArgs a = asm_args(c);
    long T = ceil_div(c->N, AT);
    long nblk = T * (T + 1) / 2;
    size_t smem = 4 * AT * (AT + 1) * sizeof(double2);
    dim3 blk(AT, AY);
    cudaError_t e;
    if (c->form == BM_MIXED) {
        e = cudaFuncSetAttribute(assemble_kernel<BM_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        assemble_kernel<BM_MIXED><<<(unsigned)nblk, blk, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(assemble_kernel<BM_ORDINARY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        assemble_kernel<BM_ORDINARY><<<(unsigned)nblk, blk, smem, s>>>(a);
    }
    return cudaGetLastError();
}

// One launch assembling the systems of B handles of equal N and formulation (grid.z = handle);
// d_args: device scratch of B * asm_args_bytes() bytes, filled here.
size_t asm_args_bytes() { return sizeof(AsmArgs); }
cudaError_t launch_assemble_batch(cudaStream_t s, bm_ctx* const* cs, int B, void* d_args) {
    if (B < 1) return cudaSuccess;
    std::vector<AsmArgs> h(B);
    for (int b = 0; b < B; ++b) h[b] = asm_args(cs[b]);
    cudaError_t e = cudaMemcpyAsync(d_args, h.data(), sizeof(AsmArgs) * B, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const int N = cs[0]->N;
    long T = ceil_div(N, AT);
    long nblk = T * (T + 1) / 2;
    size_t smem = 4 * AT * (AT + 1) * sizeof(double2);
    dim3 blk(AT, AY), grid((unsigned)nblk, 1, (unsigned)B);
    const AsmArgs* args = reinterpret_cast<const AsmArgs*>(d_args);
    if (cs[0]->form == BM_MIXED) {
        e = cudaFuncSetAttribute(assemble_batch_kernel<BM_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        assemble_batch_kernel<BM_MIXED><<<grid, blk, smem, s>>>(args);
    } else {
        e = cudaFuncSetAttribute(assemble_batch_kernel<BM_ORDINARY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        assemble_batch_kernel<BM_ORDINARY><<<grid, blk, smem, s>>>(args);
    }
    return cudaGetLastError();
}

cudaError_t launch_zeta_band(cudaStream_t s, const bm_ctx* c) {
    const int p = c->zeta_p;
    if (p <= 0) return cudaSuccess;
    AsmArgs a{};
    a.N = c->N;
    a.h = 2.0 * PI / c->N;
    a.k0 = c->k0;
    a.k1 = c->k1;
    a.eps0 = c->eps0;
    a.eps1 = c->eps1;
    a.beta = c->beta;
    a.T = c->htab;
    a.g = c->d_geom;
    long N = c->N;
    if (c->form == BM_MIXED) {
        a.o[0] = c->d_Mtop;
        a.o[1] = c->d_Mtop + N;
        a.o[2] = c->d_Mbot;
        a.o[3] = c->d_Mbot + N * c->ldbot;
        a.ld[0] = a.ld[1] = c->ldtop;
        a.ld[2] = a.ld[3] = c->ldbot;
    } else {
        a.o[0] = c->d_A;
        a.o[1] = c->d_A + N * c->ldA;
        a.o[2] = c->d_A + N;
        a.o[3] = c->d_A + N + N * c->ldA;
        a.ld[0] = a.ld[1] = a.ld[2] = a.ld[3] = c->ldA;
    }
    const ZetaArgs z = zeta_weights(p);
    const long total = N * (2L * p + 3);
    const unsigned grid = (unsigned)ceil_div(total, 128);
    if (c->form == BM_MIXED)
        zeta_band_kernel<BM_MIXED><<<grid, 128, 0, s>>>(a, z);
    else
        zeta_band_kernel<BM_ORDINARY><<<grid, 128, 0, s>>>(a, z);
    return cudaGetLastError();
}

// Host diagnostic: the correction weights the band kernel uses (no device work).
extern "C" bm_status bm_zeta_weights(int p, double* tau, double* c2) {
    if (p < 1 || p > ZETA_PMAX || tau == nullptr || c2 == nullptr) return BM_EINVAL;
    const ZetaArgs z = zeta_weights(p);
    for (int m = 0; m <= p; ++m) tau[m] = z.tau[m];
    for (int m = 0; m <= p + 1; ++m) c2[m] = z.c2[m];
    return BM_OK;
}

cudaError_t launch_normA(cudaStream_t s, const bm_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->d_normA, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (c->form == BM_MIXED) {
        rownorm_kernel<<<ceil_div(2 * c->N, 32), 256, 0, s>>>(c->d_Mtop, c->ldtop, 2 * c->N, c->N, 1.0, c->d_normA);
        rownorm_kernel<<<ceil_div(c->N, 32), 256, 0, s>>>(c->d_Mbot, c->ldbot, c->N, 2 * c->N, 0.0, c->d_normA);
    } else {
        rownorm_kernel<<<ceil_div(2 * c->N, 32), 256, 0, s>>>(c->d_A, c->ldA, 2 * c->N, 2 * c->N, 0.0, c->d_normA);
    }
    return cudaGetLastError();
}

cudaError_t launch_plane_wave(cudaStream_t s, const bm_ctx* c, const double* d_ang, int nrhs, double2* B, long ldb) {
    dim3 grid(ceil_div(c->nsys, 256), nrhs);
    plane_wave_kernel<<<grid, 256, 0, s>>>(c->d_geom, c->N, c->k0, c->beta, d_ang, nrhs, c->form, B, ldb);
    return cudaGetLastError();
}

cudaError_t launch_far_field(cudaStream_t s, const bm_ctx* c, const double2* X, long ldx, int nrhs, const double* d_ang,
                             int M, double2* U, long ldu) {
    const int at = ceil_div(M, FF_MT), ct = ceil_div(nrhs, FF_CT);
    // node slices per cluster: enough CTAs for about two per SM, at most 8 (portable clusters), at
    // least a chunk of nodes per slice
    int S = 1;
    while (S < 8 && (long)at * ct * S < 2L * c->num_sms && 2L * S * FF_JT <= c->N) S *= 2;
    const int cmax = std::min(nrhs, FF_CT);
    const size_t smem = (size_t)(2 * FF_JT * FF_MT + 2 * FF_JT * (cmax + 1)) * sizeof(double2);
    if (at > 65535) return cudaErrorInvalidConfiguration;  // more than 524280 angles in one call
    // the shared-memory limit is a per-device attribute of the kernel (idempotent, so a race between
    // host threads only sets it twice)
    static DeviceFlags attr;
    if (attr.pending()) {
        cudaError_t e = cudaFuncSetAttribute(far_field_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((2 * FF_JT * FF_MT + 2 * FF_JT * (FF_CT + 1)) * sizeof(double2)));
        if (e != cudaSuccess) return e;
        attr.done();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S, at, ct);
    cfg.blockDim = dim3(FF_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeClusterDimension;
    la[0].val.clusterDim.x = S;
    la[0].val.clusterDim.y = 1;
    la[0].val.clusterDim.z = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, far_field_kernel, c->d_geom, c->N, c->k0, c->eps0, X, ldx, d_ang, M, nrhs, U,
                              ldu);
}

__global__ void f32_convert_kernel(const double* __restrict__ x, int n, float* rn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rn[i] = f32_rn(x[i]);
}

cudaError_t launch_f32_convert(cudaStream_t s, const double* x, int n, float* rn) {
    f32_convert_kernel<<<ceil_div(n, 256), 256, 0, s>>>(x, n, rn);
    return cudaGetLastError();
}

cudaError_t launch_hankel_probe(cudaStream_t s, const bm_ctx* c, const double2* z, int n, double2* h0, double2* h1) {
    hankel_probe_kernel<<<ceil_div(n, 128), 128, 0, s>>>(z, n, c->htab, h0, h1);
    return cudaGetLastError();
}

// Operands of the Schur-complement product (part of the factorisation, like the FP32 copy of the
// ordinary matrix): A = [M31 M32] row-major, B = [M13; M23] column by column.
cudaError_t launch_pack_schur(cudaStream_t s, const bm_ctx* c, int split) {
    int N = c->N;
    int K = 2 * N;
    dim3 blk(32, 8);
    dim3 grid(ceil_div(K, 32), ceil_div(N, 32));
    pack_rowmajor_kernel<<<grid, blk, 0, s>>>(c->d_Mbot, c->ldbot, N, K, split, c->d_Ap_r, c->d_Ap_i, c->ldk_schur);
    long kext = split ? 3L * K : (long)K;
    long padn = (long)N * (c->ldk_schur - kext);
    if (padn > 0) pad_zero_rows_kernel<<<ceil_div(padn, 256), 256, 0, s>>>(c->d_Ap_r, c->d_Ap_i, c->ldk_schur, N, kext);
    long total = (long)N * c->ldk_schur;
    pack_colmajor_kernel<<<ceil_div(total, 256), 256, 0, s>>>(c->d_Mtop, c->ldtop, K, N, split, c->d_Bp_r, c->d_Bp_i,
                                                               c->ldk_schur);
    return cudaGetLastError();
}

// Rows of [M13; M23] (2N x N) for the skinny products [M13; M23] z of the solve (made once at
// assembly, like the split planes of the residual); only the tensor maps read this pack, which
// stop at K, so its padding columns stay unset.
cudaError_t launch_pack_solve(cudaStream_t s, const bm_ctx* c, int split) {
    int N = c->N;
    dim3 blk(32, 8);
    dim3 gridc(ceil_div(N, 32), ceil_div(2 * N, 32));
    pack_rowmajor_kernel<<<gridc, blk, 0, s>>>(c->d_Mtop, c->ldtop, 2 * N, N, split, c->d_Cp_r, c->d_Cp_i, c->ldk_c);
    return cudaGetLastError();
}

cudaError_t launch_to_c32(cudaStream_t s, const double2* A, long lda, int m, int n, float* Fr, float* Fi, long ldf) {
    long total = (long)m * n;
    to_c32_kernel<<<ceil_div(total, 256), 256, 0, s>>>(A, lda, m, n, Fr, Fi, ldf);
    return cudaGetLastError();
}
