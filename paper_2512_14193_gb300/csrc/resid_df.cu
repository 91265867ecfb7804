// Refinement residual r = r + alpha A x in double-float arithmetic on the FP32 cores.
//
// GB300 runs FP64 at ~1.2 TFLOP/s but FP32 at ~73 TFLOP/s, so the residual of iterative
// refinement (the only step that needs more than FP32 accuracy) is computed with pairs of FP32
// numbers instead of FP64:
//   * the FP64 operator is split once after assembly into float4 planes (re_hi, re_lo, im_hi,
//     im_lo) with hi = fl32(a), lo = fl32(a - hi) (a = hi + lo to ~2^-48 relative); the iterate
//     x is split the same way when its tile is staged in shared memory;
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

constexpr int BM = 64, BN = 16, BK = 16;  // 4 rows x 1 column per thread

__device__ __forceinline__ float4 split(double2 v) {
    float4 s;
    s.x = (float)v.x;
    s.y = (float)(v.x - (double)s.x);
    s.z = (float)v.y;
    s.w = (float)(v.y - (double)s.z);
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

// Four compensated sums, one per real partial product, so their TwoSum chains run side by side.
struct DfAcc {
    float s1, t1, s2, t2, s3, t3, s4, t4;  // ar xr, -ai xi (real); ar xi, ai xr (imag)
    float rc, ic;                          // cross terms (FP32)
};

// a = (re_hi, re_lo, im_hi, im_lo), x likewise
__device__ __forceinline__ void dfma(DfAcc& c, const float4& a, const float4& x) {
    acc2(c.s1, c.t1, a.x, x.x);
    acc2(c.s2, c.t2, -a.z, x.z);
    acc2(c.s3, c.t3, a.x, x.z);
    acc2(c.s4, c.t4, a.z, x.x);
    c.rc = fmaf(a.x, x.y, c.rc);
    c.rc = fmaf(a.y, x.x, c.rc);
    c.rc = fmaf(-a.z, x.w, c.rc);
    c.rc = fmaf(-a.w, x.z, c.rc);
    c.ic = fmaf(a.x, x.w, c.ic);
    c.ic = fmaf(a.y, x.z, c.ic);
    c.ic = fmaf(a.z, x.y, c.ic);
    c.ic = fmaf(a.w, x.x, c.ic);
}

// C (m x n, FP64) += alpha A (m x k, split planes) X (k x n, FP64)
__global__ void __launch_bounds__(256) resid_df_kernel(int m, int n, int k, const float4* __restrict__ A, long lda,
                                                       const double2* __restrict__ X, long ldx, double2* C, long ldc,
                                                       double alpha) {
    constexpr int TM = BM / 16;
    __shared__ float4 As[BK][BM + 1];
    __shared__ float4 Xs[BK][BN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const long i0 = (long)blockIdx.x * BM, j0 = (long)blockIdx.y * BN;
    DfAcc acc[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) acc[a] = DfAcc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
        for (int e = t; e < BM * BK; e += 256) {
            int ii = e % BM, kk = e / BM;
            long gi = i0 + ii;
            int gk = k0 + kk;
            As[kk][ii] = (gi < m && gk < k) ? __ldg(A + gi + (long)gk * lda) : make_float4(0.f, 0.f, 0.f, 0.f);
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
            float4 xv = Xs[kk][ty];
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
        double re = ((double)acc[a].s1 + (double)acc[a].t1) + ((double)acc[a].s2 + (double)acc[a].t2) + (double)acc[a].rc;
        double im = ((double)acc[a].s3 + (double)acc[a].t3) + ((double)acc[a].s4 + (double)acc[a].t4) + (double)acc[a].ic;
        double2& c = C[gi + gj * ldc];
        c.x += alpha * re;
        c.y += alpha * im;
    }
}

__global__ void split_planes_kernel(const double2* __restrict__ A, long lda, int m, int n, float4* __restrict__ P,
                                    long ldp) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    P[i + (long)j * ldp] = split(A[i + (long)j * lda]);
}

}  // namespace

cudaError_t gemm_df(cudaStream_t s, int m, int n, int k, double alpha, const float4* A, long lda, const double2* X,
                    long ldx, double2* C, long ldc) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    dim3 grid(ceil_div(m, BM), ceil_div(n, BN));
    resid_df_kernel<<<grid, 256, 0, s>>>(m, n, k, A, lda, X, ldx, C, ldc, alpha);
    return cudaGetLastError();
}

// P = split(A): float4 (re_hi, re_lo, im_hi, im_lo) planes of an FP64 column-major matrix
cudaError_t launch_split_planes(cudaStream_t s, const double2* A, long lda, int m, int n, float4* P, long ldp) {
    long t = (long)m * n;
    if (t == 0) return cudaSuccess;
    split_planes_kernel<<<ceil_div(t, 256), 256, 0, s>>>(A, lda, m, n, P, ldp);
    return cudaGetLastError();
}
