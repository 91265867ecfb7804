// Refinement residual r = beta r + alpha A x in double-float arithmetic on the FP32 cores.
//
// GB300 runs FP64 at ~1.2 TFLOP/s but FP32 at ~73 TFLOP/s, so the residual of iterative
// refinement (the only step that needs more than FP32 accuracy) is computed with pairs of FP32
// numbers instead of FP64:
//   * each FP64 operand is split once, when its tile is staged in shared memory, into
//     hi = fl32(a) and lo = fl32(a - hi) (a = hi + lo to ~2^-48 relative);
//   * the leading product hi_a * hi_x is formed exactly as p + e with one FMA (TwoProd) and
//     accumulated into an unevaluated pair (s, t) with TwoSum (Knuth), so the long sum of
//     K = N..2N products keeps ~46 bits;
//   * the cross terms hi_a lo_x + lo_a hi_x (2^-24 of the total) are summed in plain FP32 and
//     lo_a lo_x (2^-48) is dropped.
// The result is accurate to ~1e-12 of |A||x| - three orders below what certifying a backward
// error of 1e-9 needs - at ~50 FP32 operations per complex multiply-add.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BM = 64, BN = 16, BK = 16;

struct df4 {  // a complex FP64 value split into FP32 hi/lo parts
    float rh, rl, ih, il;
};

__device__ __forceinline__ df4 split(double2 v) {
    df4 s;
    s.rh = (float)v.x;
    s.rl = (float)(v.x - (double)s.rh);
    s.ih = (float)v.y;
    s.il = (float)(v.y - (double)s.ih);
    return s;
}

// (s, t) += a * b: exact product (TwoProd), compensated sum (TwoSum).  The _rn intrinsics keep
// the compiler from contracting these steps into FMAs, which would break their exactness.
__device__ __forceinline__ void acc2(float& s, float& t, float a, float b) {
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    float u = __fadd_rn(s, p);
    float bb = __fsub_rn(u, s);
    float err = __fadd_rn(__fsub_rn(s, __fsub_rn(u, bb)), __fsub_rn(p, bb));
    s = u;
    t += err + e;
}

struct DfAcc {
    float rs, rt, is, it, rc, ic;  // real (sum, compensation), imag (sum, compensation), cross terms
};

__device__ __forceinline__ void dfma(DfAcc& c, const df4& a, const df4& x) {
    // re += ar xr - ai xi ; im += ar xi + ai xr (hi parts exact, cross terms in FP32)
    acc2(c.rs, c.rt, a.rh, x.rh);
    acc2(c.rs, c.rt, -a.ih, x.ih);
    acc2(c.is, c.it, a.rh, x.ih);
    acc2(c.is, c.it, a.ih, x.rh);
    c.rc = fmaf(a.rh, x.rl, c.rc);
    c.rc = fmaf(a.rl, x.rh, c.rc);
    c.rc = fmaf(-a.ih, x.il, c.rc);
    c.rc = fmaf(-a.il, x.ih, c.rc);
    c.ic = fmaf(a.rh, x.il, c.ic);
    c.ic = fmaf(a.rl, x.ih, c.ic);
    c.ic = fmaf(a.ih, x.rl, c.ic);
    c.ic = fmaf(a.il, x.rh, c.ic);
}

// C (m x n) = C + alpha A (m x k) X (k x n); all FP64 interleaved column-major
__global__ void __launch_bounds__(256) resid_df_kernel(int m, int n, int k, const double2* __restrict__ A, long lda,
                                                       const double2* __restrict__ X, long ldx, double2* C, long ldc,
                                                       double alpha) {
    constexpr int TM = BM / 16;
    __shared__ df4 As[BK][BM + 1];
    __shared__ df4 Xs[BK][BN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const long i0 = (long)blockIdx.x * BM, j0 = (long)blockIdx.y * BN;
    DfAcc acc[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) acc[a] = DfAcc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
        for (int e = t; e < BM * BK; e += 256) {
            int ii = e % BM, kk = e / BM;
            long gi = i0 + ii;
            int gk = k0 + kk;
            double2 v = (gi < m && gk < k) ? A[gi + (long)gk * lda] : make_double2(0.0, 0.0);
            As[kk][ii] = split(v);
        }
        {
            int kk = t % BK, jj = t / BK;  // BN * BK == 256
            long gj = j0 + jj;
            int gk = k0 + kk;
            double2 v = (gj < n && gk < k) ? X[gk + gj * ldx] : make_double2(0.0, 0.0);
            Xs[kk][jj] = split(v);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            df4 xv = Xs[kk][ty];
#pragma unroll
            for (int a = 0; a < TM; ++a) dfma(acc[a], As[kk][tx + 16 * a], xv);
        }
        __syncthreads();
    }
    const long gj = j0 + ty;
    if (gj >= n) return;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        long gi = i0 + tx + 16 * a;
        if (gi >= m) continue;
        double re = (double)acc[a].rs + (double)acc[a].rt + (double)acc[a].rc;
        double im = (double)acc[a].is + (double)acc[a].it + (double)acc[a].ic;
        double2& c = C[gi + gj * ldc];
        c.x += alpha * re;
        c.y += alpha * im;
    }
}

}  // namespace

cudaError_t gemm_df(cudaStream_t s, int m, int n, int k, double alpha, const double2* A, long lda, const double2* X,
                    long ldx, double2* C, long ldc) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    dim3 grid(ceil_div(m, BM), ceil_div(n, BN));
    resid_df_kernel<<<grid, 256, 0, s>>>(m, n, k, A, lda, X, ldx, C, ldc, alpha);
    return cudaGetLastError();
}
