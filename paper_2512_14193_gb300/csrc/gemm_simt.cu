// Complex GEMM on the CUDA cores: C = beta C + alpha op(A) B for column-major views.
//
// FP64 (Z64, interleaved double2): the engine of the FP64 path (Schur complement
// U33 = -[M31 M32][M13; M23] of Theorem thm:LU, LU trailing updates, the FP64 residual of
// refinement).  GB300 executes FP64 on the CUDA cores only, so this kernel is bound by the FP64
// pipe; it keeps a 64 x BN tile per CTA (BN = 16, 32 or 64, whichever pads the column count
// least) with 4 x BN/16 complex accumulators per thread staged through shared memory.
// FP32 (C32, planar): skinny updates inside the LU panel and the FP32 correction solves.
// Mixed (A and C FP64 storage, B FP32, FP32 arithmetic): the refinement residual update
// r -= A d for a small correction d.
//
// op(A) = A (m x k view) or, with a_trans, A is given as its transpose stored column-major
// (k x m view), i.e. row-major A - the layout of the tensor-core operand packs.
#include "common.cuh"
#include "kernels.cuh"

#include <type_traits>

namespace {

constexpr int BK = 16;

template <class R> BM_HD cplx_t<R> conv(double2 v);
template <class R> BM_HD cplx_t<R> conv(float2 v);
template <> BM_HD double2 conv<double>(double2 v) { return v; }
template <> BM_HD float2 conv<float>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> BM_HD float2 conv<float>(float2 v) { return v; }

template <class VC> BM_HD typename VC::cv from_acc(double2 v) {
    typename VC::cv r;
    r.x = (typename VC::real)v.x;
    r.y = (typename VC::real)v.y;
    return r;
}
template <class VC> BM_HD typename VC::cv from_acc(float2 v) {
    typename VC::cv r;
    r.x = (typename VC::real)v.x;
    r.y = (typename VC::real)v.y;
    return r;
}

// VA, VB, VC: storage views of A, B, C; R: arithmetic precision
template <class VA, class VB, class VC, class R, bool AT, int BM, int BN>
__global__ void __launch_bounds__(256) cgemm_simt_kernel(int m, int n, int k, VA A, VB B, VC C, R alpha, R beta) {
    using CV = cplx_t<R>;
    constexpr int TM = BM / 16, TN = BN / 16;
    pdl_wait();
    pdl_trigger();
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
            if (gi < m && gk < k) v = conv<R>(AT ? A.get(gk, gi) : A.get(gi, gk));
            As[kk][ii] = v;
        }
#pragma unroll
        for (int e = t; e < BN * BK; e += 256) {
            int kk = e % BK, jj = e / BK;
            long gj = j0 + jj;
            int gk = k0 + kk;
            CV v = czero<R>();
            if (gj < n && gk < k) v = conv<R>(B.get(gk, gj));
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
    // all of this thread's C reads are issued before its first write (the compiler cannot move a
    // read of C past a write to C, so interleaving them would cost one memory latency each)
    using OCV = typename VC::cv;
    OCV cin[TM][TN];
    if (beta != (R)0) {
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) {
                const long gi = i0 + tx + 16 * a, gj = j0 + ty + 16 * b;
                if (gi < m && gj < n) cin[a][b] = C.get(gi, gj);
            }
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
            OCV out = from_acc<VC>(r);
            if (beta != (R)0) {
                out.x += (typename VC::real)beta * cin[a][b].x;
                out.y += (typename VC::real)beta * cin[a][b].y;
            }
            C.set(gi, gj, out);
        }
    }
}

template <class VA, class VB, class VC, class R, bool AT>
cudaError_t launch_impl(cudaStream_t s, int m, int n, int k, VA A, VB B, VC C, R alpha, R beta) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    // every launch may overlap the previous kernel's tail: the kernel waits (pdl_wait) before it
    // reads anything
    auto go = [&](auto kern, dim3 grid) { return launch_pdl(kern, grid, dim3(256), 0, s, m, n, k, A, B, C, alpha, beta); };
    // Few right-hand sides (n <= 80, e.g. 65): one column tile covers them all, so A is streamed
    // once; 32-row tiles when 64-row ones would leave SMs idle.
    if (n > 32 && n <= 80) {
        if ((long)ceil_div(m, 64) >= 2 * 152)
            return go(cgemm_simt_kernel<VA, VB, VC, R, AT, 64, 80>, dim3(ceil_div(m, 64), 1));
        return go(cgemm_simt_kernel<VA, VB, VC, R, AT, 32, 80>, dim3(ceil_div(m, 32), 1));
    }
    // FP64 products too small to fill the GPU with 64-row tiles (the FP64 pipe gives each SM only
    // ~8 GFLOP/s, so idle SMs cost directly): 32 x 16 tiles
    if constexpr (std::is_same<R, double>::value) {
        static int sms = 0;
        if (sms == 0) {
            int dev = 0, v = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
                sms = v;
            else
                sms = 1;
        }
        if ((long)ceil_div(m, 64) * ceil_div(n, 64) < sms)
            return go(cgemm_simt_kernel<VA, VB, VC, R, AT, 32, 16>, dim3(ceil_div(m, 32), ceil_div(n, 16)));
    }
    // otherwise the column tile with the least padding (ties go to the wider tile)
    int bn = 64;
    long best = (long)ceil_div(n, 64) * 64 - n;
    for (int cand : {32, 16}) {
        long waste = (long)ceil_div(n, cand) * cand - n;
        if (waste < best) {
            best = waste;
            bn = cand;
        }
    }
    if (bn == 16) return go(cgemm_simt_kernel<VA, VB, VC, R, AT, 64, 16>, dim3(ceil_div(m, 64), ceil_div(n, 16)));
    if (bn == 32) return go(cgemm_simt_kernel<VA, VB, VC, R, AT, 64, 32>, dim3(ceil_div(m, 64), ceil_div(n, 32)));
    return go(cgemm_simt_kernel<VA, VB, VC, R, AT, 64, 64>, dim3(ceil_div(m, 64), ceil_div(n, 64)));
}

}  // namespace

cudaError_t gemm_z64(cudaStream_t s, int m, int n, int k, double alpha, Z64 A, bool a_trans, Z64 B, double beta,
                     Z64 C) {
    if (k <= 0 && beta == 1.0) return cudaSuccess;
    return a_trans ? launch_impl<Z64, Z64, Z64, double, true>(s, m, n, k, A, B, C, alpha, beta)
                   : launch_impl<Z64, Z64, Z64, double, false>(s, m, n, k, A, B, C, alpha, beta);
}

cudaError_t gemm_c32(cudaStream_t s, int m, int n, int k, float alpha, C32 A, bool a_trans, C32 B, float beta,
                     C32 C) {
    if (k <= 0 && beta == 1.0f) return cudaSuccess;
    return a_trans ? launch_impl<C32, C32, C32, float, true>(s, m, n, k, A, B, C, alpha, beta)
                   : launch_impl<C32, C32, C32, float, false>(s, m, n, k, A, B, C, alpha, beta);
}

// C (FP64) += alpha A (FP64 storage) B (FP32 planar), products and sums in FP32
cudaError_t gemm_update_z64_c32(cudaStream_t s, int m, int n, int k, float alpha, Z64 A, C32 B, Z64 C) {
    if (k <= 0) return cudaSuccess;
    return launch_impl<Z64, C32, Z64, float, false>(s, m, n, k, A, B, C, alpha, 1.0f);
}

// C (FP64) += alpha A_hi (FP32 hi parts of split planes) B (FP32 planar), FP32 arithmetic
cudaError_t gemm_update_f4hi_c32(cudaStream_t s, int m, int n, int k, float alpha, F4Hi A, C32 B, Z64 C) {
    if (k <= 0) return cudaSuccess;
    return launch_impl<F4Hi, C32, Z64, float, false>(s, m, n, k, A, B, C, alpha, 1.0f);
}
