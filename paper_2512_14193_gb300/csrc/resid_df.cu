// Refinement residual r = r + alpha A x in double-float arithmetic on the FP32 cores.
//
// GB300 runs FP64 at ~1.2 TFLOP/s but FP32 at ~73 TFLOP/s, so the residual of iterative
// refinement (the only step that needs more than FP32 accuracy) is computed with pairs of FP32
// numbers instead of FP64:
//   * the FP64 operator is split once after assembly into float4 planes (re_hi, re_lo, im_hi,
//     im_lo) with hi = fl32(a), lo = fl32(a - hi) (a = hi + lo to ~2^-48 relative), plus a
//     float2 plane of re + im split the same way; the iterate x is split the same way by a small
//     kernel before the product (so the product kernel itself does no FP64 work, which runs at
//     1/64 of the FP32 rate on this part);
//   * the complex product uses three real products (Karatsuba / Gauss):
//         P1 = re a re x,  P2 = im a im x,  P3 = (re a + im a)(re x + im x),
//         re(a x) = P1 - P2,  im(a x) = P3 - P1 - P2,
//     each summed over K as an unevaluated pair (s, c): the leading product hi_a * hi_x is formed
//     exactly as p + e with one FMA (TwoProd) and added to s with TwoSum (Knuth), whose rounding
//     error goes to c together with e and the cross terms hi_a lo_x + lo_a hi_x (all ~2^-24 of
//     the terms), so the long sum keeps ~46 bits; lo_a lo_x (2^-48) is dropped;
//   * the three sums combine in FP64 at the end; the cancellation in P3 - P1 - P2 costs at most
//     a factor ~4 on the ~1e-12 relative accuracy, far below what a backward error of 1e-9 needs.
// 36 FP32 operations per complex multiply-add (four real products would take 48).
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BM = 64, BN = 16, BK = 16;  // 4 rows x 1 column per thread

// s += a * b with exact product (TwoProd) and compensated sum (TwoSum); both rounding errors go
// to the plain FP32 sum c, which also takes the cross terms (all three are ~2^-24 of the terms
// they come from, so one FP32 sum carries them as well as two).  The _rn intrinsics keep the
// compiler from contracting these steps into FMAs, which would break their exactness.
__device__ __forceinline__ void acc2(float& s, float& c, float a, float b) {
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    float u = __fadd_rn(s, p);
    float bb = __fsub_rn(u, s);
    float err = __fadd_rn(__fsub_rn(s, __fsub_rn(u, bb)), __fsub_rn(p, bb));
    s = u;
    c += err;
    c += e;
}

// Three compensated sums (P1, P2, P3) side by side: leading parts s, FP32 error/cross-term sums c.
struct DfAcc {
    float s1, s2, s3;
    float c1, c2, c3;
};

// a = (re_hi, re_lo, im_hi, im_lo), as = (sum_hi, sum_lo); x and xs likewise
__device__ __forceinline__ void dfma(DfAcc& c, const float4& a, const float2& as, const float4& x, const float2& xs) {
    acc2(c.s1, c.c1, a.x, x.x);
    acc2(c.s2, c.c2, a.z, x.z);
    acc2(c.s3, c.c3, as.x, xs.x);
    c.c1 = fmaf(a.x, x.y, c.c1);
    c.c1 = fmaf(a.y, x.x, c.c1);
    c.c2 = fmaf(a.z, x.w, c.c2);
    c.c2 = fmaf(a.w, x.z, c.c2);
    c.c3 = fmaf(as.x, xs.y, c.c3);
    c.c3 = fmaf(as.y, xs.x, c.c3);
}

__device__ __forceinline__ float2 split1(double v) {
    float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// One launch runs every product of a residual as equal-length work units: a unit is one BM x BN
// output tile over one K split.  Products with S > 1 splits write each split's raw sum to the
// workspace W and a reduction adds alpha * (sum over splits, in order) to C afterwards, so the
// result does not depend on scheduling.  Units of a row tile are consecutive (column tile
// fastest), so the blocks that read the same A tile run at about the same time and share it
// through L2.
struct DfJob {
    int nprod, n;
    double alpha;
    DfProd p[2];
    int first_unit[3];  // units of product q: [first_unit[q], first_unit[q + 1])
};

__global__ void __launch_bounds__(256, 3) resid_df_kernel(const __grid_constant__ DfJob J) {
    constexpr int TM = BM / 16;
    __shared__ float4 As[BK][BM + 1];
    __shared__ float2 Qs[BK][BM + 1];
    __shared__ float4 Xs[BK][BN + 1];
    __shared__ float2 Ys[BK][BN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int q = (int)blockIdx.x >= J.first_unit[1] ? 1 : 0;
    const DfProd& P = J.p[q];
    const int n = J.n, m = P.m, k = P.k;
    const int tn = (n + BN - 1) / BN;
    int u = (int)blockIdx.x - J.first_unit[q];
    const int jt = u % tn;
    u /= tn;
    const int z = u % P.S, it = u / P.S;
    const int kb = (int)((long)z * k / P.S), ke = (int)((long)(z + 1) * k / P.S);
    const long i0 = (long)it * BM, j0 = (long)jt * BN;
    const bool active = j0 + ty < n;
    DfAcc acc[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) acc[a] = DfAcc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int e = t; e < BM * BK; e += 256) {
            int ii = e % BM, kk = e / BM;
            long gi = i0 + ii;
            int gk = k0 + kk;
            const bool in = gi < m && gk < ke;
            As[kk][ii] = in ? __ldg(P.A + gi + (long)gk * P.lda) : make_float4(0.f, 0.f, 0.f, 0.f);
            Qs[kk][ii] = in ? __ldg(P.Q + gi + (long)gk * P.lda) : make_float2(0.f, 0.f);
        }
        {
            int kk = t % BK, jj = t / BK;  // BN * BK == 256
            long gj = j0 + jj;
            int gk = k0 + kk;
            const bool in = gj < n && gk < ke;
            Xs[kk][jj] = in ? __ldg(P.XP + gk + gj * P.ldx) : make_float4(0.f, 0.f, 0.f, 0.f);
            Ys[kk][jj] = in ? __ldg(P.XQ + gk + gj * P.ldx) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // threads of columns past the last right-hand side (the ragged column tile: 65 = 4 x 16 + 1)
        // only help with the loads
        if (active) {
#pragma unroll 4
            for (int kk = 0; kk < BK; ++kk) {
                const float4 xv = Xs[kk][ty];
                const float2 yv = Ys[kk][ty];
#pragma unroll
                for (int a = 0; a < TM; ++a) dfma(acc[a], As[kk][tx + 16 * a], Qs[kk][tx + 16 * a], xv, yv);
            }
        }
        __syncthreads();
    }
    const long gj = j0 + ty;
    if (gj >= n) return;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        long gi = i0 + tx + 16 * a;
        if (gi >= m) continue;
        const DfAcc& r = acc[a];
        double p1 = (double)r.s1 + (double)r.c1;
        double p2 = (double)r.s2 + (double)r.c2;
        double p3 = (double)r.s3 + (double)r.c3;
        const double re = p1 - p2, im = (p3 - p1) - p2;
        if (P.S == 1) {
            double2& c = P.C[gi + gj * P.ldc];
            c.x += J.alpha * re;
            c.y += J.alpha * im;
        } else {
            P.W[(long)z * m * n + gi + gj * m] = make_double2(re, im);
        }
    }
}

// C += alpha * sum_z W[z] (z in order)
__global__ void df_reduce_kernel(const double2* __restrict__ W, int S, int m, int n, double alpha, double2* C,
                                 long ldc) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long zs = (long)m * n;
    if (idx >= zs) return;
    const int j = (int)(idx / m), i = (int)(idx % m);
    double re = 0.0, im = 0.0;
    for (int z = 0; z < S; ++z) {
        const double2 w = W[idx + z * zs];
        re += w.x;
        im += w.y;
    }
    double2& c = C[i + (long)j * ldc];
    c.x += alpha * re;
    c.y += alpha * im;
}

__global__ void split_planes_kernel(const double2* __restrict__ A, long lda, int m, int n, float4* __restrict__ P,
                                    float2* __restrict__ Q, long ldp) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    const double2 v = A[i + (long)j * lda];
    const float2 r = split1(v.x), im = split1(v.y);
    P[i + (long)j * ldp] = make_float4(r.x, r.y, im.x, im.y);
    Q[i + (long)j * ldp] = split1(v.x + v.y);
}

}  // namespace

// The products of one residual (at most two, sharing n and alpha) as one launch of equal-length
// work units; a product with S > 1 K splits takes S m n elements of the workspace W (products
// with S > 1 use disjoint parts of it: at most one product may have S > 1).  Adds the kernels it
// launched to *launched.
cudaError_t gemm_df(cudaStream_t s, const DfProd* prods, int nprod, int n, double alpha, int* launched) {
    if (nprod < 1 || nprod > 2 || n <= 0) return cudaSuccess;
    DfJob J{};
    J.nprod = nprod;
    J.n = n;
    J.alpha = alpha;
    const int tn = ceil_div(n, BN);
    int u = 0;
    for (int q = 0; q < 2; ++q) {
        J.first_unit[q] = u;
        if (q < nprod) {
            J.p[q] = prods[q];
            if (prods[q].m > 0 && prods[q].k > 0) u += ceil_div(prods[q].m, BM) * prods[q].S * tn;
        }
    }
    J.first_unit[2] = u;
    if (nprod == 1) J.first_unit[1] = u;
    if (u == 0) return cudaSuccess;
    resid_df_kernel<<<u, 256, 0, s>>>(J);
    *launched += 1;
    for (int q = 0; q < nprod; ++q) {
        const DfProd& P = prods[q];
        if (P.S > 1 && P.m > 0 && P.k > 0) {
            const long t = (long)P.m * n;
            df_reduce_kernel<<<ceil_div(t, 256), 256, 0, s>>>(P.W, P.S, P.m, n, alpha, P.C, P.ldc);
            *launched += 1;
        }
    }
    return cudaGetLastError();
}

// P = split(A): float4 (re_hi, re_lo, im_hi, im_lo) planes of an FP64 column-major matrix, and
// Q = split(re + im) (float2), both with leading dimension ldp
cudaError_t launch_split_planes(cudaStream_t s, const double2* A, long lda, int m, int n, float4* P, float2* Q,
                                long ldp) {
    long t = (long)m * n;
    if (t == 0) return cudaSuccess;
    split_planes_kernel<<<ceil_div(t, 256), 256, 0, s>>>(A, lda, m, n, P, Q, ldp);
    return cudaGetLastError();
}
