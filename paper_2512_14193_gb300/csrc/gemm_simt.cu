// Complex GEMM on the CUDA cores: C = beta C + alpha op(A) B for column-major views.
//
// FP64 (Z64, interleaved double2): the engine of the FP64 path (Schur complement
// U33 = -[M31 M32][M13; M23] of Theorem thm:LU, LU trailing updates, FP64 residuals of
// refinement).  GB300 executes FP64 on the CUDA cores only, so this kernel is bound by the FP64
// pipe; it keeps a 64 x 64 (or 64 x 16 for few right-hand sides) tile per CTA with 4 x 4
// (4 x 1) complex accumulators per thread staged through shared memory.
// FP32 (C32, planar): skinny updates inside the LU panel and the FP32 correction solves.
//
// op(A) = A (m x k view) or, with a_trans, A is given as its transpose stored column-major
// (k x m view), i.e. row-major A - the layout of the tensor-core operand packs.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BK = 16;

template <class V, bool AT, int BM, int BN>
__global__ void __launch_bounds__(256) cgemm_simt_kernel(int m, int n, int k, V A, V B, V C,
                                                         typename V::real alpha, typename V::real beta) {
    using R = typename V::real;
    using CV = typename V::cv;
    constexpr int TM = BM / 16, TN = BN / 16;
    __shared__ CV As[BK][BM + 1];
    __shared__ CV Bs[BK][BN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const long i0 = (long)blockIdx.x * BM, j0 = (long)blockIdx.y * BN;
    CV acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = czero<R>();

    for (int k0 = 0; k0 < k; k0 += BK) {
        // A tile BM x BK
#pragma unroll
        for (int e = t; e < BM * BK; e += 256) {
            int ii, kk;
            if (AT) {
                kk = e % BK;
                ii = e / BK;
            } else {
                ii = e % BM;
                kk = e / BM;
            }
            long gi = i0 + ii;
            int gk = k0 + kk;
            CV v = czero<R>();
            if (gi < m && gk < k) v = AT ? A.get(gk, gi) : A.get(gi, gk);
            As[kk][ii] = v;
        }
        // B tile BK x BN
#pragma unroll
        for (int e = t; e < BN * BK; e += 256) {
            int kk = e % BK, jj = e / BK;
            long gj = j0 + jj;
            int gk = k0 + kk;
            CV v = czero<R>();
            if (gj < n && gk < k) v = B.get(gk, gj);
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            CV av[TM], bv[TN];
#pragma unroll
            for (int a = 0; a < TM; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) cfma(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        long gi = i0 + tx + 16 * a;
        if (gi >= m) continue;
#pragma unroll
        for (int b = 0; b < TN; ++b) {
            long gj = j0 + ty + 16 * b;
            if (gj >= n) continue;
            CV r;
            r.x = alpha * acc[a][b].x;
            r.y = alpha * acc[a][b].y;
            if (beta != (R)0) {
                CV c = C.get(gi, gj);
                r.x += beta * c.x;
                r.y += beta * c.y;
            }
            C.set(gi, gj, r);
        }
    }
}

template <class V, bool AT>
cudaError_t launch_impl(cudaStream_t s, int m, int n, int k, V A, V B, V C, typename V::real alpha,
                        typename V::real beta) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (n <= 16) {
        dim3 grid(ceil_div(m, 64), ceil_div(n, 16));
        cgemm_simt_kernel<V, AT, 64, 16><<<grid, 256, 0, s>>>(m, n, k, A, B, C, alpha, beta);
    } else {
        dim3 grid(ceil_div(m, 64), ceil_div(n, 64));
        cgemm_simt_kernel<V, AT, 64, 64><<<grid, 256, 0, s>>>(m, n, k, A, B, C, alpha, beta);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_z64(cudaStream_t s, int m, int n, int k, double alpha, Z64 A, bool a_trans, Z64 B, double beta,
                     Z64 C) {
    if (k <= 0) {
        if (beta == 1.0) return cudaSuccess;
    }
    return a_trans ? launch_impl<Z64, true>(s, m, n, k, A, B, C, alpha, beta)
                   : launch_impl<Z64, false>(s, m, n, k, A, B, C, alpha, beta);
}

cudaError_t gemm_c32(cudaStream_t s, int m, int n, int k, float alpha, C32 A, bool a_trans, C32 B, float beta,
                     C32 C) {
    if (k <= 0) {
        if (beta == 1.0f) return cudaSuccess;
    }
    return a_trans ? launch_impl<C32, true>(s, m, n, k, A, B, C, alpha, beta)
                   : launch_impl<C32, false>(s, m, n, k, A, B, C, alpha, beta);
}
