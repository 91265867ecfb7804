// Solves with the factored system, FP64 residuals and iterative refinement.
//
// Mixed system, arbitrary 3N right-hand sides (Corollary lem:for_ssm_RHS):
//     z3 = U33^{-1} (b3 - M31 b1 - M32 b2),  x1 = b1 - M13 z3,  x2 = b2 - M23 z3,  x3 = z3
// with [M31 M32] and [M13; M23] each applied as one product (K = 2N and M = 2N).
// Ordinary system: x = A^{-1} b by the LU of the 2N matrix.
//
// CF32 precisions: the correction solve above runs in FP32 with the FP32 factors and the FP32
// operand packs; the residual r = b - A x uses the FP64 assembled operator (structured for the
// mixed system: r1 = b1 - x1 - M13 x3, r2 = b2 - x2 - M23 x3, r3 = b3 - M31 x1 - M32 x2) and
// x += A32^{-1} r repeats until the normwise backward error
//     eta = max_c ||r_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf)
// is at most refine_tol.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace {

__global__ void resid_init_kernel(const double2* __restrict__ B, const double2* __restrict__ X, long ld, int nsys,
                                  int nsub, int nrhs, double2* __restrict__ R) {
    // R = B - X on rows [0, nsub) (identity blocks), R = B elsewhere
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nsys * nrhs) return;
    int c = (int)(idx / nsys), i = (int)(idx % nsys);
    long o = i + (long)c * ld;
    double2 v = B[o];
    if (i < nsub) v = csub(v, X[o]);
    R[o] = v;
}

__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// per column: eta_c = max|R| / (normA max|X| + max|B|); out[0] = max_c eta_c, out[1] = 1 if any
// non-finite value was seen in B (the input check)
__global__ void eta_kernel(const double2* __restrict__ R, const double2* __restrict__ X,
                           const double2* __restrict__ B, long ld, int nsys, const double* __restrict__ normA,
                           double* out) {
    int c = blockIdx.x;
    double r = 0, x = 0, b = 0;
    bool bad = false;
    // magnitudes in FP32 (the ratio needs a few digits; FP64 hypot would cost the FP64 pipe)
    float rf = 0.f, xf = 0.f, bf = 0.f;
#pragma unroll 4
    for (int i = threadIdx.x; i < nsys; i += blockDim.x) {
        long o = i + (long)c * ld;
        double2 bv = B[o];
        if (!isfinite(bv.x) || !isfinite(bv.y)) bad = true;
        double2 rv = R[o], xv = X[o];
        rf = fmaxf(rf, hypotf((float)rv.x, (float)rv.y));
        xf = fmaxf(xf, hypotf((float)xv.x, (float)xv.y));
        bf = fmaxf(bf, hypotf((float)bv.x, (float)bv.y));
    }
    r = rf;
    x = xf;
    b = bf;
    __shared__ double sr[32], sx[32], sb[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) sbad = 1;
    for (int o = 16; o > 0; o >>= 1) {
        r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sr[w] = r;
        sx[w] = x;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int q = 1; q < nw; ++q) {
            r = fmax(r, sr[q]);
            x = fmax(x, sx[q]);
            b = fmax(b, sb[q]);
        }
        r = fmax(r, sr[0]);
        x = fmax(x, sx[0]);
        b = fmax(b, sb[0]);
        double den = (*normA) * x + b;
        double eta = (den > 0) ? r / den : (r > 0 ? 1.0 : 0.0);
        if (!isfinite(eta)) eta = 1e300;
        atomic_max_pos(out, eta);
        if (sbad) out[1] = 1.0;
    }
}

__global__ void to_c32_kernel(const double2* __restrict__ A, long lda, int m, int n, float* __restrict__ Fr,
                              float* __restrict__ Fi, long ldf) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    double2 v = A[i + (long)j * lda];
    Fr[i + (long)j * ldf] = (float)v.x;
    Fi[i + (long)j * ldf] = (float)v.y;
}

// X[r0 + i, c] += D[i, c]
__global__ void add_c32_kernel(double2* __restrict__ X, long ldx, int r0, int m, int n, const float* __restrict__ Dr,
                               const float* __restrict__ Di, long ldd) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    double2& x = X[r0 + i + (long)j * ldx];
    x.x += (double)Dr[i + (long)j * ldd];
    x.y += (double)Di[i + (long)j * ldd];
}

// X[r0 + i, c] -= D[i, c]
__global__ void sub_c32_kernel(double2* __restrict__ X, long ldx, int r0, int m, int n, const float* __restrict__ Dr,
                               const float* __restrict__ Di, long ldd) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    double2& x = X[r0 + i + (long)j * ldx];
    x.x -= (double)Dr[i + (long)j * ldd];
    x.y -= (double)Di[i + (long)j * ldd];
}

__global__ void copy_z64_kernel(const double2* __restrict__ S, long lds, int m, int n, double2* __restrict__ D,
                                long ldd) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)m * n) return;
    int j = (int)(idx / m), i = (int)(idx % m);
    D[i + (long)j * ldd] = S[i + (long)j * lds];
}

#define SV_CUDA(expr)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            bm_set_error(std::string("solve: ") + #expr + ": " + cudaGetErrorString(_e));              \
            return BM_ECUDA;                                                                           \
        }                                                                                              \
    } while (0)

// K splits of a skinny tensor-core product, never more than the partial-sum workspace holds
int skinny_split(const bm_ctx* c, int m, int n, int kext) {
    int S = tc_split_k(m, n, kext, c->num_sms);
    while (S > 1 && (size_t)S * m * n > c->pk_elems) --S;
    return S;
}

cudaError_t copy_z64(cudaStream_t s, const double2* S, long lds, int m, int n, double2* D, long ldd) {
    long t = (long)m * n;
    if (t == 0) return cudaSuccess;
    copy_z64_kernel<<<ceil_div(t, 256), 256, 0, s>>>(S, lds, m, n, D, ldd);
    return cudaGetLastError();
}

}  // namespace

// Direct FP64 solve: X = A^{-1} B (B, X: nsys x nrhs with leading dimension ld, device).
bm_status solve_fp64(bm_ctx* c, const double2* B, double2* X, long ld, int nrhs) {
    cudaStream_t s = c->stream;
    const int N = c->N;
    const long ldy = c->n;
    if (c->form == BM_MIXED) {
        // t3 = b3 - [M31 M32] [b1; b2]
        {
            BM_PROF(c, "copy_z64_kernel");
            SV_CUDA(copy_z64(s, B + 2 * N, ld, N, nrhs, c->d_Y64b, ldy));
        }
        {
            BM_PROF(c, "cgemm_simt_kernel<Z64> (solve product)");
            SV_CUDA(gemm_z64(s, N, nrhs, 2 * N, -1.0, Z64{c->d_Mbot, c->ldbot}, false, Z64{const_cast<double2*>(B), ld},
                             1.0, Z64{c->d_Y64b, ldy}));
        }
        {
            BM_PROF(c, "gather_rows_kernel");
            SV_CUDA(launch_gather_rows_z64(s, c->d_perm, N, nrhs, c->d_Y64b, ldy, c->d_Y64, ldy));
        }
        BM_TRY(getrs_z64(c, c->d_Y64, ldy, nrhs));
        {
            BM_PROF(c, "copy_z64_kernel");
            SV_CUDA(copy_z64(s, c->d_Y64, ldy, N, nrhs, X + 2 * N, ld));
        }
        // [x1; x2] = [b1; b2] - [M13; M23] z3
        {
            BM_PROF(c, "copy_z64_kernel");
            SV_CUDA(copy_z64(s, B, ld, 2 * N, nrhs, X, ld));
        }
        {
            BM_PROF(c, "cgemm_simt_kernel<Z64> (solve product)");
            SV_CUDA(gemm_z64(s, 2 * N, nrhs, N, -1.0, Z64{c->d_Mtop, c->ldtop}, false, Z64{X + 2 * N, ld}, 1.0,
                             Z64{X, ld}));
        }
    } else {
        {
            BM_PROF(c, "gather_rows_kernel");
            SV_CUDA(launch_gather_rows_z64(s, c->d_perm, c->n, nrhs, B, ld, c->d_Y64, ldy));
        }
        BM_TRY(getrs_z64(c, c->d_Y64, ldy, nrhs));
        {
            BM_PROF(c, "copy_z64_kernel");
            SV_CUDA(copy_z64(s, c->d_Y64, ldy, c->n, nrhs, X, ld));
        }
    }
    return BM_OK;
}

// R = B - A X with the FP64 assembled operator.  Not captured in a graph: counts its own launches.
bm_status residual_fp64(bm_ctx* c, const double2* B, const double2* X, double2* R, long ld, int nrhs) {
    cudaStream_t s = c->stream;
    const int N = c->N;
    long t = (long)c->nsys * nrhs;
    int nsub = (c->form == BM_MIXED) ? 2 * N : 0;
    {
        BM_PROF(c, "resid_init_kernel");
        resid_init_kernel<<<ceil_div(t, 256), 256, 0, s>>>(B, X, ld, c->nsys, nsub, nrhs, R);
        SV_CUDA(cudaGetLastError());
    }
    BM_PROF(c, "cgemm_simt_kernel<Z64> (FP64 residual)");
    if (c->form == BM_MIXED) {
        SV_CUDA(gemm_z64(s, 2 * N, nrhs, N, -1.0, Z64{c->d_Mtop, c->ldtop}, false,
                         Z64{const_cast<double2*>(X) + 2 * N, ld}, 1.0, Z64{R, ld}));
        SV_CUDA(gemm_z64(s, N, nrhs, 2 * N, -1.0, Z64{c->d_Mbot, c->ldbot}, false, Z64{const_cast<double2*>(X), ld},
                         1.0, Z64{R + 2 * N, ld}));
    } else {
        SV_CUDA(gemm_z64(s, 2 * N, nrhs, 2 * N, -1.0, Z64{c->d_A, c->ldA}, false, Z64{const_cast<double2*>(X), ld},
                         1.0, Z64{R, ld}));
    }
    c->launches += (c->form == BM_MIXED) ? 3 : 2;
    return BM_OK;
}

// R = B - A X with the FP64 operator, products and sums in double-float on the FP32 cores.  Not
// captured in a graph: counts its own launches.
bm_status residual_df(bm_ctx* c, const double2* B, const double2* X, double2* R, long ld, int nrhs) {
    cudaStream_t s = c->stream;
    const int N = c->N;
    long t = (long)c->nsys * nrhs;
    int nsub = (c->form == BM_MIXED) ? 2 * N : 0;
    {
        BM_PROF(c, "resid_init_kernel");
        resid_init_kernel<<<ceil_div(t, 256), 256, 0, s>>>(B, X, ld, c->nsys, nsub, nrhs, R);
        SV_CUDA(cudaGetLastError());
    }
    const long ldp = c->nsys;
    {
        BM_PROF(c, "split_planes_kernel (iterate)");
        SV_CUDA(launch_split_planes(s, X, ld, c->nsys, nrhs, c->d_XP, c->d_XQ, ldp));
    }
    BM_PROF(c, "resid_df_kernel (+ split-K reduction)");
    // K splits chosen so every work unit spans K = N: the K = 2N products are split in two
    int nl = 0;
    if (c->form == BM_MIXED) {
        DfProd P[2] = {
            {c->d_Pbot, c->d_Qbot, c->ldbot, c->d_XP, c->d_XQ, ldp, R + 2 * N, ld, c->d_Wdf, N, 2 * N, 2},
            {c->d_Ptop, c->d_Qtop, c->ldtop, c->d_XP + 2 * N, c->d_XQ + 2 * N, ldp, R, ld, nullptr, 2 * N, N, 1}};
        SV_CUDA(gemm_df(s, P, 2, nrhs, -1.0, &nl));
    } else {
        DfProd P[1] = {{c->d_PA, c->d_QA, c->ldA, c->d_XP, c->d_XQ, ldp, R, ld, c->d_Wdf, 2 * N, 2 * N, 2}};
        SV_CUDA(gemm_df(s, P, 1, nrhs, -1.0, &nl));
    }
    c->launches += 2 + nl;
    return BM_OK;
}

// R = B - A X with the FP64 operator, from exact digit products on the tensor cores (resid_tc.cu).
// Not captured in a graph: counts its own launches.
bm_status residual_tc(bm_ctx* c, const double2* B, const double2* X, double2* R, long ld, int nrhs) {
    cudaStream_t s = c->stream;
    const int N = c->N;
    long t = (long)c->nsys * nrhs;
    int nsub = (c->form == BM_MIXED) ? 2 * N : 0;
    {
        BM_PROF(c, "resid_init_kernel");
        resid_init_kernel<<<ceil_div(t, 256), 256, 0, s>>>(B, X, ld, c->nsys, nsub, nrhs, R);
        SV_CUDA(cudaGetLastError());
    }
    const int nt = rt_col_tile(c->rt_nd), npad = (nrhs + nt - 1) / nt * nt;
    const int nprod = (c->form == BM_MIXED) ? 2 : 1;
    {
        BM_PROF(c, "digits_x (col_exponent/digits_x_kernel)");
        for (int q = 0; q < nprod; ++q) {
            const int r0 = (c->form == BM_MIXED && q == 0) ? 2 * N : 0;
            const int K = (c->form == BM_MIXED && q == 0) ? N : 2 * N;
            SV_CUDA(launch_digits_x(s, X, ld, r0, K, nrhs, npad, c->d_dxe[q], c->d_dx[q], c->dx_ldk[q], c->rt_nd));
        }
    }
    // mixed: Mbot (K = 2N, the longer units) first, then Mtop; ordinary: A
    RtArgs P[2];
    double* w = c->d_rtw;
    int np = 0;
    int S[2];
    {
        const long mq[2] = {c->form == BM_MIXED ? N : 2L * N, 2L * N};
        const long Kq[2] = {2L * N, c->form == BM_MIXED ? N : 2L * N};
        rt_plan_splits(nprod, mq, Kq, nrhs, c->rt_nd, c->num_sms, S);
    }
    auto add = [&](int dg, int dx, double2* Cout, int m, int K) {
        const int Sq = S[np];
        RtArgs a{c->tm_dg[dg], c->tm_dx[dx], c->d_dge[dg], c->d_dxe[dx], Cout, ld, nullptr, nullptr, m, K, Sq};
        if (Sq > 1) {
            a.Wr = w;
            a.Wi = w + (size_t)Sq * m * nrhs;
            w += 2 * (size_t)Sq * m * nrhs;
        }
        P[np++] = a;
    };
    if (c->form == BM_MIXED) {
        add(1, 1, R + 2 * N, N, 2 * N);
        add(0, 0, R, 2 * N, N);
    } else {
        add(0, 0, R, 2 * N, 2 * N);
    }
    if ((size_t)(w - c->d_rtw) > c->rtw_elems) {
        bm_set_error("residual_tc: split-K workspace too small");
        return BM_EINVAL;
    }
    int nl = 0;
    {
        BM_PROF(c, "resid_tc_kernel (+ split-K reduction)");
        SV_CUDA(gemm_rt(s, P, np, nrhs, -1.0, c->d_err, &nl, c->rt_nd));
    }
    c->launches += 1 + 2 * nprod + nl;
    return BM_OK;
}

// d_eta[0] = backward error (max over columns), d_eta[1] = non-finite flag of B
bm_status backward_error(bm_ctx* c, const double2* R, const double2* X, const double2* B, long ld, int nrhs,
                         double* d_eta) {
    SV_CUDA(cudaMemsetAsync(d_eta, 0, 2 * sizeof(double), c->stream));
    // one CTA of 1024 threads per column (few columns: the loads in flight per SM set the time)
    BM_PROF(c, "eta_kernel");
    eta_kernel<<<nrhs, 1024, 0, c->stream>>>(R, X, B, ld, c->nsys, c->d_normA, d_eta);
    SV_CUDA(cudaGetLastError());
    return BM_OK;
}

// X += A32^{-1} R (FP32 correction solve with the FP32 factors and packs).
bm_status correction_c32(bm_ctx* c, const double2* R, double2* X, long ld, int nrhs) {
    cudaStream_t s = c->stream;
    const int N = c->N;
    const long ldw = c->nsys;
    float* Wr = c->d_Wr;
    float* Wi = c->d_Wi;
    float* Vr = c->d_W2r;
    float* Vi = c->d_W2i;
    const long ldv = c->n;
    long t = (long)c->nsys * nrhs;
    {
        BM_PROF(c, "to_c32_kernel");
        to_c32_kernel<<<ceil_div(t, 256), 256, 0, s>>>(R, ld, c->nsys, nrhs, Wr, Wi, ldw);
        SV_CUDA(cudaGetLastError());
    }
    const bool split = (c->prec == BM_CF32_3XTF32_IR);
    if (c->form == BM_MIXED && c->tc_skinny) {
        // the two skinny products on the tensor cores, split over K (few output tiles)
        const int K = 2 * N;
        int nl = 0;
        // W3 -= [M31 M32] [W1; W2]
        const long k1 = split ? 3L * K : (long)K;
        {
            BM_PROF(c, "pack_b_kernel");
            SV_CUDA(launch_pack_b(s, Wr, Wi, ldw, K, nrhs, split, c->d_Bx1r, c->d_Bx1i, c->ldk_schur));
        }
        {
            BM_PROF(c, "cgemm_tc_kernel (skinny, + split-K reduction)");
            SV_CUDA(gemm_tc_split(s, c->tm_schur[0], c->tm_schur[1], c->tm_skinny[2], c->tm_skinny[3], N, nrhs, (int)k1,
                                  -1.f, 1.f, TcDest{Wr + 2 * N, Wi + 2 * N, nullptr, ldw},
                                  skinny_split(c, N, nrhs, (int)k1), c->d_Pkr, c->d_Pki, c->d_err, &nl));
        }
        {
            BM_PROF(c, "gather_rows_kernel");
            SV_CUDA(launch_gather_rows_c32(s, c->d_perm, N, nrhs, Wr + 2 * N, Wi + 2 * N, ldw, Vr, Vi, ldv));
        }
        BM_TRY(getrs_c32(c, Vr, Vi, ldv, nrhs));
        // [W1; W2] -= [M13; M23] z3; the pack of z3 stays for the next residual update
        const long k2 = split ? 3L * N : (long)N;
        {
            BM_PROF(c, "pack_b_kernel");
            SV_CUDA(launch_pack_b(s, Vr, Vi, ldv, N, nrhs, split, c->d_Bx2r, c->d_Bx2i, c->ldk_c));
        }
        {
            BM_PROF(c, "cgemm_tc_kernel (skinny, + split-K reduction)");
            SV_CUDA(gemm_tc_split(s, c->tm_skinny[0], c->tm_skinny[1], c->tm_skinny[4], c->tm_skinny[5], 2 * N, nrhs,
                                  (int)k2, -1.f, 1.f, TcDest{Wr, Wi, nullptr, ldw},
                                  skinny_split(c, 2 * N, nrhs, (int)k2), c->d_Pkr, c->d_Pki, c->d_err, &nl));
        }
        BM_PROF(c, "add_c32_kernel");
        long t2 = (long)K * nrhs;
        add_c32_kernel<<<ceil_div(t2, 256), 256, 0, s>>>(X, ld, 0, K, nrhs, Wr, Wi, ldw);
        long t3 = (long)N * nrhs;
        add_c32_kernel<<<ceil_div(t3, 256), 256, 0, s>>>(X, ld, 2 * N, N, nrhs, Vr, Vi, ldv);
        SV_CUDA(cudaGetLastError());
    } else if (c->form == BM_MIXED) {
        const int K = 2 * N;
        // W3 -= [M31 M32] [W1; W2]   (A operand pack is row-major: pass it as its transpose)
        C32 Ahi{c->d_Ap_r, c->d_Ap_i, c->ldk_schur};
        C32 W12{Wr, Wi, ldw};
        C32 W3{Wr + 2 * N, Wi + 2 * N, ldw};
        SV_CUDA(gemm_c32(s, N, nrhs, K, -1.0f, Ahi, true, W12, 1.0f, W3));
        if (split) {
            C32 Alo{c->d_Ap_r + 2 * K, c->d_Ap_i + 2 * K, c->ldk_schur};
            SV_CUDA(gemm_c32(s, N, nrhs, K, -1.0f, Alo, true, W12, 1.0f, W3));
        }
        SV_CUDA(launch_gather_rows_c32(s, c->d_perm, N, nrhs, Wr + 2 * N, Wi + 2 * N, ldw, Vr, Vi, ldv));
        BM_TRY(getrs_c32(c, Vr, Vi, ldv, nrhs));
        // [W1; W2] -= [M13; M23] z3 (B operand pack is column-major [M13; M23])
        C32 Bhi{c->d_Bp_r, c->d_Bp_i, c->ldk_schur};
        C32 Z{Vr, Vi, ldv};
        SV_CUDA(gemm_c32(s, K, nrhs, N, -1.0f, Bhi, false, Z, 1.0f, W12));
        if (split) {
            C32 Blo{c->d_Bp_r + K, c->d_Bp_i + K, c->ldk_schur};
            SV_CUDA(gemm_c32(s, K, nrhs, N, -1.0f, Blo, false, Z, 1.0f, W12));
        }
        long t2 = (long)K * nrhs;
        add_c32_kernel<<<ceil_div(t2, 256), 256, 0, s>>>(X, ld, 0, K, nrhs, Wr, Wi, ldw);
        long t3 = (long)N * nrhs;
        add_c32_kernel<<<ceil_div(t3, 256), 256, 0, s>>>(X, ld, 2 * N, N, nrhs, Vr, Vi, ldv);
        SV_CUDA(cudaGetLastError());
    } else {
        {
            BM_PROF(c, "gather_rows_kernel");
            SV_CUDA(launch_gather_rows_c32(s, c->d_perm, c->n, nrhs, Wr, Wi, ldw, Vr, Vi, ldv));
        }
        BM_TRY(getrs_c32(c, Vr, Vi, ldv, nrhs));
        BM_PROF(c, "add_c32_kernel");
        long t2 = (long)c->n * nrhs;
        add_c32_kernel<<<ceil_div(t2, 256), 256, 0, s>>>(X, ld, 0, c->n, nrhs, Vr, Vi, ldv);
        SV_CUDA(cudaGetLastError());
    }
    return BM_OK;
}

// R -= A d for the correction d of the last correction_c32 call (still in the FP32 work buffers),
// with the products in FP32.  d is small next to x after the first correction, so the FP32
// product error (~1e-6 |A| |d|) stays far below the backward-error target: this replaces the
// full FP64 residual b - A x from the second refinement step on.  Runs outside the captured
// graphs, so it adds its own kernel launches to the handle's count.
bm_status residual_update_c32(bm_ctx* c, double2* R, long ld, int nrhs) {
    cudaStream_t s = c->stream;
    const int N = c->N;
    BM_PROF(c, "residual update (FP32 products)");
    const long ldw = c->nsys, ldv = c->n;
    if (c->form == BM_MIXED && c->tc_skinny && c->prec == BM_CF32_3XTF32_IR) {
        // 3xTF32 products on the tensor cores (FP32-level accuracy, as the SIMT FP32 update):
        // rows [0, 2N): r -= d12 + [M13; M23] d3 with d3 still packed by the correction;
        // rows [2N, 3N): r -= [M31 M32] d12 with d12 packed here
        long t2 = (long)2 * N * nrhs;
        sub_c32_kernel<<<ceil_div(t2, 256), 256, 0, s>>>(R, ld, 0, 2 * N, nrhs, c->d_Wr, c->d_Wi, ldw);
        SV_CUDA(cudaGetLastError());
        int n1 = 0, n2 = 0;
        const long k2 = 3L * N, k1 = 6L * N;
        SV_CUDA(gemm_tc_split(s, c->tm_skinny[0], c->tm_skinny[1], c->tm_skinny[4], c->tm_skinny[5], 2 * N, nrhs,
                              (int)k2, -1.f, 1.f, TcDest{nullptr, nullptr, R, ld},
                              skinny_split(c, 2 * N, nrhs, (int)k2), c->d_Pkr, c->d_Pki, c->d_err, &n1));
        SV_CUDA(launch_pack_b(s, c->d_Wr, c->d_Wi, ldw, 2 * N, nrhs, 1, c->d_Bx1r, c->d_Bx1i, c->ldk_schur));
        SV_CUDA(gemm_tc_split(s, c->tm_schur[0], c->tm_schur[1], c->tm_skinny[2], c->tm_skinny[3], N, nrhs, (int)k1,
                              -1.f, 1.f, TcDest{nullptr, nullptr, R + 2 * N, ld},
                              skinny_split(c, N, nrhs, (int)k1), c->d_Pkr, c->d_Pki, c->d_err, &n2));
        c->launches += 2 + n1 + n2;
    } else if (c->form == BM_MIXED) {
        // rows [0, 2N): r -= d12 + [M13; M23] d3 ; rows [2N, 3N): r -= [M31 M32] d12
        long t2 = (long)2 * N * nrhs;
        sub_c32_kernel<<<ceil_div(t2, 256), 256, 0, s>>>(R, ld, 0, 2 * N, nrhs, c->d_Wr, c->d_Wi, ldw);
        SV_CUDA(cudaGetLastError());
        SV_CUDA(gemm_update_f4hi_c32(s, 2 * N, nrhs, N, -1.0f, F4Hi{c->d_Ptop, c->ldtop}, C32{c->d_W2r, c->d_W2i, ldv},
                                    Z64{R, ld}));
        SV_CUDA(gemm_update_f4hi_c32(s, N, nrhs, 2 * N, -1.0f, F4Hi{c->d_Pbot, c->ldbot}, C32{c->d_Wr, c->d_Wi, ldw},
                                    Z64{R + 2 * N, ld}));
        c->launches += 3;
    } else {
        SV_CUDA(gemm_update_f4hi_c32(s, 2 * N, nrhs, 2 * N, -1.0f, F4Hi{c->d_PA, c->ldA}, C32{c->d_W2r, c->d_W2i, ldv},
                                    Z64{R, ld}));
        c->launches += 1;
    }
    return BM_OK;
}

cudaError_t launch_copy_z64(cudaStream_t s, const double2* S, long lds, int m, int n, double2* D, long ldd) {
    return copy_z64(s, S, lds, m, n, D, ldd);
}
