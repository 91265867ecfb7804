// Launchers shared between the library's translation units (internal).
#pragma once
#include "common.cuh"

// assemble.cu
cudaError_t launch_geometry(cudaStream_t s, int kind, const double p[4], int N, const double* d_user, double* d_geom);
cudaError_t launch_assemble(cudaStream_t s, const bm_ctx* c);
size_t asm_args_bytes();
cudaError_t launch_assemble_batch(cudaStream_t s, bm_ctx* const* cs, int B, void* d_args);
cudaError_t launch_zeta_band(cudaStream_t s, const bm_ctx* c);  // high-order zeta corrections (zeta_p > 0)
cudaError_t launch_normA(cudaStream_t s, const bm_ctx* c);
cudaError_t launch_plane_wave(cudaStream_t s, const bm_ctx* c, const double* d_ang, int nrhs, double2* B, long ldb);
cudaError_t launch_far_field(cudaStream_t s, const bm_ctx* c, const double2* X, long ldx, int nrhs, const double* d_ang,
                             int M, double2* U, long ldu);
cudaError_t launch_hankel_probe(cudaStream_t s, const bm_ctx* c, const double2* z, int n, double2* h0, double2* h1);
cudaError_t launch_f32_convert(cudaStream_t s, const double* x, int n, float* rn);
cudaError_t launch_pack_schur(cudaStream_t s, const bm_ctx* c, int split);  // Schur operands (in bm_factor)
cudaError_t launch_pack_solve(cudaStream_t s, const bm_ctx* c, int split);  // [M13; M23] rows (assembly)
cudaError_t launch_to_c32(cudaStream_t s, const double2* A, long lda, int m, int n, float* Fr, float* Fi, long ldf);

// gemm_simt.cu
cudaError_t gemm_z64(cudaStream_t s, int m, int n, int k, double alpha, Z64 A, bool a_trans, Z64 B, double beta, Z64 C);
cudaError_t gemm_c32(cudaStream_t s, int m, int n, int k, float alpha, C32 A, bool a_trans, C32 B, float beta, C32 C);
cudaError_t gemm_update_z64_c32(cudaStream_t s, int m, int n, int k, float alpha, Z64 A, C32 B, Z64 C);

// gemm_tc.cu (tensor maps are CUtensorMap, passed as opaque 128-byte blobs)
bm_status tc_make_map(void* tmap, const float* base, long rows, long kext, long ldk, int box_rows);
cudaError_t gemm_tc(cudaStream_t s, const void* tAr, const void* tAi, const void* tBr, const void* tBi, float* Cr,
                    float* Ci, long ldc, int m, int n, int kext, float alpha, float beta, int* d_err);
constexpr int TC_BM = 128;
constexpr int TC_BN = 128;
// destination of a split-K product: FP32 planar (re, im) or, when z is set, FP64 interleaved
struct TcDest {
    float* re;
    float* im;
    double2* z;
    long ld;
};
int tc_split_k(int m, int n, int kext, int num_sms);
cudaError_t gemm_tc_split(cudaStream_t s, const void* tAr, const void* tAi, const void* tBr, const void* tBi, int m,
                          int n, int kext, float alpha, float beta, TcDest dst, int S, float* Pr, float* Pi,
                          int* d_err, int* launched);
cudaError_t launch_pack_b(cudaStream_t s, const float* Vr, const float* Vi, long ldv, int K, int nrhs, int split,
                          float* Br, float* Bi, long ldk);
size_t tc_batch_entry_bytes();
cudaError_t gemm_tc_batch(cudaStream_t s, int B, const void* const* maps, float* const* Cr, float* const* Ci,
                          const long* ldc, int m, int n, int kext, float alpha, void* d_entries, int* d_err);

// lu.cu
bm_status lu_setup(bm_ctx* c, int cluster_cap, int panel_kernel);
bm_status lu_factor_enqueue(bm_ctx* c);       // factor d_F64 / d_F32 in place (stream-ordered)
size_t swap_map_bytes();
bm_status getrs_z64(bm_ctx* c, double2* Y, long ldy, int nrhs);   // in place; Y holds P B (rows gathered by perm)
bm_status getrs_c32(bm_ctx* c, float* Yr, float* Yi, long ldy, int nrhs);
cudaError_t launch_gather_rows_z64(cudaStream_t s, const int* perm, int n, int nrhs, const double2* B, long ldb,
                                   double2* Y, long ldy);
cudaError_t launch_gather_rows_c32(cudaStream_t s, const int* perm, int n, int nrhs, const float* Br, const float* Bi,
                                   long ldb, float* Yr, float* Yi, long ldy);

// solve.cu
bm_status solve_fp64(bm_ctx* c, const double2* B, double2* X, long ld, int nrhs);
bm_status residual_fp64(bm_ctx* c, const double2* B, const double2* X, double2* R, long ld, int nrhs);
bm_status backward_error(bm_ctx* c, const double2* R, const double2* X, const double2* B, long ld, int nrhs,
                         double* d_eta);
bm_status correction_c32(bm_ctx* c, const double2* R, double2* X, long ld, int nrhs);
bm_status residual_update_c32(bm_ctx* c, double2* R, long ld, int nrhs);
bm_status residual_df(bm_ctx* c, const double2* B, const double2* X, double2* R, long ld, int nrhs);
bm_status residual_tc(bm_ctx* c, const double2* B, const double2* X, double2* R, long ld, int nrhs);

// resid_df.cu: C += alpha A X in double-float arithmetic (A as split planes, X and C FP64)
// one product C (m x n) += alpha A (m x k) X (k x n) of a double-float residual; S K splits (S > 1
// writes S m n raw partial sums to W, reduced in order afterwards)
struct DfProd {
    const float4* A;   // split planes of the operator (re_hi, re_lo, im_hi, im_lo)
    const float2* Q;   // split re + im
    long lda;
    const float4* XP;  // the iterate split the same way
    const float2* XQ;
    long ldx;
    double2* C;
    long ldc;
    double2* W;
    int m, k, S;
};
cudaError_t gemm_df(cudaStream_t s, const DfProd* prods, int nprod, int n, double alpha, int* launched);
cudaError_t launch_split_planes(cudaStream_t s, const double2* A, long lda, int m, int n, float4* P, float2* Q,
                                long ldp);
// gemm_simt.cu: C (FP64) += alpha A_hi B with A the hi parts of split planes, FP32 arithmetic
cudaError_t gemm_update_f4hi_c32(cudaStream_t s, int m, int n, int k, float alpha, F4Hi A, C32 B, Z64 C);
cudaError_t launch_copy_z64(cudaStream_t s, const double2* S, long lds, int m, int n, double2* D, long ldd);

// resid_tc.cu: r += alpha A x to FP64-level accuracy from exact bf16 digit products on the tensor
// cores (digit planes of A made once after assembly, of x per residual)
struct RtArgs {
    const void* tmA;   // host copies of the tensor maps (opaque 128-byte blobs)
    const void* tmX;
    const int* eA;     // row exponents of A (device)
    const int* fX;     // column exponents of x (device)
    double2* C;        // output, C += alpha A x
    long ldc;
    double* Wr;        // split-K workspace (S > 1): S m n doubles each
    double* Wi;
    int m, K, S;
};
long rt_ldk(long K);                 // leading dimension of a digit plane row (K rounded to 64)
int rt_digit_planes(int nd);         // planes per operand (nd digits x Re, Im)
int rt_col_tile(int nd);             // right-hand sides per CTA
// K splits S[q] of the nprod products (m[q] rows, K[q] columns) of one launch with n right-hand sides
void rt_plan_splits(int nprod, const long* m, const long* K, int n, int nd, int num_sms, int* S);
bm_status rt_make_map(void* tmap, const void* base, long rows, long K, long ldk, long plane_elems, int box_rows,
                      int nd);
cudaError_t launch_digits_a(cudaStream_t s, const double2* A, long lda, int rows, int K, int* e, void* D, long ldk,
                            void* rowmax, int nd);
cudaError_t launch_digits_x(cudaStream_t s, const double2* X, long ldx, int r0, int K, int n, int npad, int* f,
                            void* D, long ldk, int nd);
cudaError_t gemm_rt(cudaStream_t s, const RtArgs* prods, int nprod, int n, double alpha, int* d_err, int* launched,
                    int nd);

// api.cu: assembly in two halves (the batched contour solver assembles many handles at once)
bm_status assemble_impl(bm_ctx* c, const bm_curve* curve, int N, bm_c64 k_out, bm_c64 k_in, bm_formulation form,
                        const bm_opts* opts, bool defer_kernels);
bm_status assemble_post(bm_ctx* c, bool run_assembly_kernel, bool wait);  // wait: synchronise the stream
bm_status factor_lu_enqueue(bm_ctx* c);              // LU of the Schur complement in place (graph)
bm_status factor_result(bm_ctx* c, int* info);       // waits, reads info / timeout, sets the state
bm_status set_panel_cluster(bm_ctx* c, int cap);     // panel cluster cap of an assembled handle
