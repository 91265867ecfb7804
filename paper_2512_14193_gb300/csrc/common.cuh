// Shared internals of the GB300 Burton-Miller library: complex helpers, matrix accessors,
// launch helpers and the handle layout.  Not part of the public ABI (include/bm.h is).
#pragma once

#include <atomic>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <map>

#include "../../include/bm.h"

#ifndef BM_HD
#define BM_HD __host__ __device__ __forceinline__
#endif

// ---------------------------------------------------------------------------------------------
// Complex arithmetic on double2 / float2 (interleaved re, im)
// ---------------------------------------------------------------------------------------------
BM_HD double2 cmk(double a, double b) { return make_double2(a, b); }
BM_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
BM_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
BM_HD double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
BM_HD double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
BM_HD double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
BM_HD double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }  // i * a
BM_HD double cnorm1(double2 a) { return fabs(a.x) + fabs(a.y); }
BM_HD double2 cinv(double2 a) {
    // 1/a with scaling (Smith's method)
    if (fabs(a.x) >= fabs(a.y)) {
        double r = a.y / a.x, d = a.x + a.y * r;
        return make_double2(1.0 / d, -r / d);
    } else {
        double r = a.x / a.y, d = a.y + a.x * r;
        return make_double2(r / d, -1.0 / d);
    }
}
BM_HD double2 cdiv(double2 a, double2 b) { return cmul(a, cinv(b)); }
// a += b * c
BM_HD void cfma(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}

BM_HD float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
BM_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
BM_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
BM_HD float cnorm1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
BM_HD float2 cinv(float2 a) {
    if (fabsf(a.x) >= fabsf(a.y)) {
        float r = a.y / a.x, d = a.x + a.y * r;
        return make_float2(1.0f / d, -r / d);
    } else {
        float r = a.x / a.y, d = a.y + a.x * r;
        return make_float2(r / d, -1.0f / d);
    }
}
BM_HD void cfma(float2& a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}

// ---------------------------------------------------------------------------------------------
// f32_rn(x) = (float)x rounded to nearest even (IEEE 754 binary64 -> binary32), by integer
// arithmetic on the bit pattern, for kernels whose other work is FP32 and integer (the row norms);
// it falls back to the hardware conversion where the result would not be a normal FP32 number
// (zero, results below 2^-126 or from 2^127 on, infinities, NaN).  Measured: the packing kernels
// were not faster with it (nor with an integer double-float split) than with the hardware
// conversion, so they keep the latter.
#ifdef __CUDACC__
__device__ __forceinline__ float f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;  // binary32 biased exponent
    if (e < 1 || e > 253) return (float)x;
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 of the 52 mantissa bits
    const unsigned rest = lo & 0x1FFFFFFFu;                  // the 29 bits dropped
    unsigned f = ((unsigned)e << 23) | m;
    f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;  // a carry moves to the exponent
    return __uint_as_float(f | (hi & 0x80000000u));
}
#endif

// Kernel attributes set with cudaFuncSetAttribute belong to one device.  A launcher keeps one
// DeviceFlags (static storage, so zero-initialised) per attribute it sets: pending() stays true
// until done() for the calling thread's current device; for a device index past 63, or when the
// current device cannot be read, it is always true and the attribute is set on every launch.
struct DeviceFlags {
    std::atomic<bool> f[64];
    static int dev() {
        int d = -1;
        if (cudaGetDevice(&d) != cudaSuccess) {
            cudaGetLastError();
            d = -1;
        }
        return d;
    }
    bool pending() const {
        const int d = dev();
        return d < 0 || d >= 64 || !f[d].load(std::memory_order_acquire);
    }
    void done() {
        const int d = dev();
        if (d >= 0 && d < 64) f[d].store(true, std::memory_order_release);
    }
};

template <class R> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <class R> using cplx_t = typename cplx_of<R>::type;

template <class R> BM_HD cplx_t<R> czero();
template <> BM_HD double2 czero<double>() { return make_double2(0.0, 0.0); }
template <> BM_HD float2 czero<float>() { return make_float2(0.f, 0.f); }

// ---------------------------------------------------------------------------------------------
// Column-major complex matrix views.
//   Z64: FP64 interleaved (double2), element (i, j) at p[i + j*ld]
//   C32: FP32 planar, element (i, j) at re[i + j*ld], im[i + j*ld]
// Both expose get/set and a pointer offset to a sub-block.
// ---------------------------------------------------------------------------------------------
struct Z64 {
    using real = double;
    using cv = double2;
    double2* p;
    long ld;
    BM_HD cv get(long i, long j) const { return p[i + j * ld]; }
    BM_HD void set(long i, long j, cv v) const { p[i + j * ld] = v; }
    BM_HD Z64 sub(long i, long j) const { return Z64{p + i + j * ld, ld}; }
};
struct C32 {
    using real = float;
    using cv = float2;
    float* re;
    float* im;
    long ld;
    BM_HD cv get(long i, long j) const { return make_float2(re[i + j * ld], im[i + j * ld]); }
    BM_HD void set(long i, long j, cv v) const {
        re[i + j * ld] = v.x;
        im[i + j * ld] = v.y;
    }
    BM_HD C32 sub(long i, long j) const { return C32{re + i + j * ld, im + i + j * ld, ld}; }
};

// F4Hi: read-only view of the hi parts of split FP64 planes (float4 = re_hi, re_lo, im_hi, im_lo)
struct F4Hi {
    using real = float;
    using cv = float2;
    const float4* p;
    long ld;
    BM_HD cv get(long i, long j) const {
        float4 v = p[i + j * ld];
        return make_float2(v.x, v.z);
    }
    BM_HD void set(long, long, cv) const {}
    BM_HD F4Hi sub(long i, long j) const { return F4Hi{p + i + j * ld, ld}; }
};

// ---------------------------------------------------------------------------------------------
// Error handling
// ---------------------------------------------------------------------------------------------
void bm_set_error(const std::string& msg);
#define BM_CUDA_TRY(expr)                                                                        \
    do {                                                                                         \
        cudaError_t _e = (expr);                                                                 \
        if (_e != cudaSuccess) {                                                                 \
            bm_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                    \
            return BM_ECUDA;                                                                     \
        }                                                                                        \
    } while (0)
#define BM_TRY(expr)                                                                             \
    do {                                                                                         \
        bm_status _s = (expr);                                                                   \
        if (_s != BM_OK) return _s;                                                              \
    } while (0)

static inline long pad32(long n) { return (n + 31) / 32 * 32; }
static inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------------------------
// Hankel anchor table (built on the host in double-double, see hankel_table.cpp)
// ---------------------------------------------------------------------------------------------
// Taylor coefficients a_0 .. a_18 of H0^(1) about every anchor z0 (H0(z0 + d) = sum a_k d^k):
// a_0 .. a_8 as FP64 complex, a_9 .. a_18 as FP32 complex (two per 16-byte slot), 14 slots
// (224 bytes) per anchor at [(iy * nx + ix) * HT_SLOTS].
constexpr int HT_K64 = 9, HT_K32 = 10, HT_SLOTS = HT_K64 + HT_K32 / 2;
struct HankelTable {
    const double2* c;  // coefficient blocks, HT_SLOTS per anchor
    int nx, ny;
    double re0, im0, step, inv_step;
};
// Builds (once per process) the host copy of the anchor table: {H0(z0), H1(z0)} per anchor.
const std::vector<double2>& hankel_anchor_host(int& nx, int& ny, double& re0, double& im0, double& step);
// The coefficient blocks of the same anchors (built with the anchor table).
const std::vector<double2>& hankel_coef_host();
// The device copy of the coefficient blocks on `dev` (the current device): uploaded by the first
// call in each CUDA context of the device and shared by every handle there; it lives as long as
// the context (no handle owns it or counts it against its HBM budget).
bm_status hankel_table_device(int dev, const double2** out);
// Unique ID of the calling thread's current CUDA context (driver API through the runtime's
// entry-point query); 0 if there is none or the query is unavailable.  IDs are never reused within
// a process, so a context that replaced a reset one has a new ID.
unsigned long long cuda_context_id();

// ---------------------------------------------------------------------------------------------
// The handle
// ---------------------------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Sizes and leading dimensions of one assembled system (api.cu make_plan).
struct Plan {
    long ldtop = 0, ldbot = 0, ldA = 0, ldF = 0, ldk_schur = 0, ldk_lu = 0, ldk_c = 0;
    int n = 0, nsys = 0, nb = 0, kseg = 0, nblk = 0;
    size_t bytes = 0;
};

struct bm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    size_t held = 0;
    std::map<void*, size_t> allocs;

    HankelTable htab{};

    // problem
    bool assembled = false;
    bool factored = false;
    bool singular = false;
    int N = 0;
    int n = 0;          // system size factored by the dense LU: N (mixed, U33) or 2N (ordinary)
    int nsys = 0;       // rows of the full system: 3N or 2N
    int form = BM_MIXED;
    int prec = BM_FP64;
    double2 k0{}, k1{}, eps0{}, eps1{}, beta{};
    double refine_tol = 1e-9;
    int refine_maxit = 30;
    int resid_mode = BM_RESID_TC_UPDATE;
    int nb = 0;
    int zeta_p = 0;  // high-order zeta correction points (0: the one-point rule)

    // geometry (device, SoA of N each): x, y, nx, ny, speed, kappa, w
    double* d_geom = nullptr;

    // FP64 operator
    //  mixed:    Mtop = [M13; M23] (2N x N, ld ldtop), Mbot = [M31 M32] (N x 2N, ld ldbot)
    //  ordinary: A (2N x 2N, ld ldA)
    double2* d_Mtop = nullptr;
    double2* d_Mbot = nullptr;
    long ldtop = 0, ldbot = 0;
    double2* d_A = nullptr;
    long ldA = 0;
    double* d_normA = nullptr;  // ||A||_inf (device scalar)
    // the FP64 operator split into FP32 hi/lo planes (CF32 precisions; same layout and leading
    // dimensions as d_Mtop / d_Mbot / d_A) for the double-float residual
    float4* d_Ptop = nullptr;
    float4* d_Pbot = nullptr;
    float4* d_PA = nullptr;
    float2* d_Qtop = nullptr;  // re + im of the same entries, split hi/lo (3-product complex multiply)
    float2* d_Qbot = nullptr;
    float2* d_QA = nullptr;
    // the FP64 operator as base-128 digit planes for the tensor-core residual (CF32 precisions):
    // [0] Mtop (mixed) or A (ordinary), [1] Mbot (mixed); 14 bf16 planes [rows][ldk] each, with the
    // power-of-two exponent of every row
    void* d_dg[2] = {nullptr, nullptr};
    int* d_dge[2] = {nullptr, nullptr};
    long dg_ldk[2] = {0, 0};
    int rt_nd = 7;            // digits per operand (8 for BM_RESID_TC_ALL)
    alignas(64) unsigned char tm_dg[2][128];
    // x digit planes for the two products (K ranges [2N, 3N) and [0, 2N) mixed; [0, 2N) ordinary),
    // their column exponents, and the split-K workspace of the tensor-core residual
    void* d_dx[2] = {nullptr, nullptr};
    int* d_dxe[2] = {nullptr, nullptr};
    long dx_ldk[2] = {0, 0};
    alignas(64) unsigned char tm_dx[2][128];
    double* d_rtw = nullptr;
    size_t rtw_elems = 0;

    // factorisation storage
    double2* d_F64 = nullptr;  // FP64 LU (n x n, ld ldF)
    float* d_F32r = nullptr;   // FP32 planar LU
    float* d_F32i = nullptr;
    long ldF = 0;
    int* d_ipiv = nullptr;
    int* d_perm = nullptr;
    int* d_info = nullptr;
    int* d_err = nullptr;
    void* d_maps = nullptr;    // row-interchange maps used by the factorisation: big panel (even),
                               // sub-panel, big panel (odd)
    // look-ahead of the FP32 factorisation: the panel chain on la_hi (high priority), the rest of
    // each trailing update on la_lo; events start, fork, join, done
    cudaStream_t la_hi = nullptr, la_lo = nullptr;
    cudaEvent_t la_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // inverted diagonal blocks of L and U (getrs), bs x bs each, n/bs blocks
    void* d_dinvL = nullptr;
    void* d_dinvU = nullptr;
    int bs_solve = 64;

    // tensor-core operand packs (FP32 planar, K-major, segments for 3xTF32)
    float* d_Ap_r = nullptr;  // Schur A operand [M31 M32] (N rows x Kext)
    float* d_Ap_i = nullptr;
    float* d_Bp_r = nullptr;  // Schur B operand [M13; M23]^T rows (N rows x Kext)
    float* d_Bp_i = nullptr;
    long ldk_schur = 0;
    int kseg_schur = 0;       // K of one segment (2N)
    float* d_Lp_r = nullptr;  // LU trailing-update packs
    float* d_Lp_i = nullptr;
    float* d_Up_r = nullptr;
    float* d_Up_i = nullptr;
    long ldk_lu = 0;
    float* d_Cp_r = nullptr;  // [M13; M23] rows, K = N (2N rows x Kext): A operand of the skinny
    float* d_Cp_i = nullptr;  //   products [M13; M23] z of the mixed correction and residual update
    long ldk_c = 0;
    float* d_O32r = nullptr;  // ordinary: FP32 copy of A is the LU buffer (d_F32*)

    // solve workspace (sized for the largest nrhs seen)
    int ws_nrhs = 0;
    int last_nrhs = 0;        // nrhs of the last bm_solve (its B, X stay in the workspace)
    double2* d_X = nullptr;   // nsys x nrhs FP64 iterate
    double2* d_R = nullptr;   // nsys x nrhs FP64 residual
    double2* d_Bw = nullptr;  // nsys x nrhs FP64 copy of B
    float* d_Wr = nullptr;    // FP32 planar work (nsys x nrhs) x 2
    float* d_Wi = nullptr;
    float* d_W2r = nullptr;
    float* d_W2i = nullptr;
    double2* d_Y64 = nullptr; // FP64 work for the FP64 solve
    double2* d_Y64b = nullptr;
    double2* d_Zw64 = nullptr;  // n x nrhs work buffers of the blocked triangular solves
    int* d_flow = nullptr;  // readiness flags of the persistent triangular solve (FP32)
    long flow_len = 0;      // their count
    float* d_Zwr = nullptr;
    float* d_Zwi = nullptr;
    double* d_colred = nullptr;  // per-column reductions (4 x nrhs)
    // mixed CF32: B operand packs of the skinny tensor-core products (ws_nrhs rows, K-major) and
    // the split-K partial-sum workspace
    float* d_Bx1r = nullptr;  // [W1; W2] columns, K = 2N (ld ldk_schur)
    float* d_Bx1i = nullptr;
    float* d_Bx2r = nullptr;  // z3 columns, K = N (ld ldk_c)
    float* d_Bx2i = nullptr;
    float* d_Pkr = nullptr;
    float* d_Pki = nullptr;
    float4* d_XP = nullptr;   // CF32: the iterate split for the double-float residual (nsys x nrhs)
    float2* d_XQ = nullptr;
    double2* d_Wdf = nullptr; // split-K partial sums of the double-float residual (4N x nrhs)
    size_t pk_elems = 0;      // capacity of each partial-sum plane (floats)

    // cached graphs (with the number of kernel nodes each replay launches)
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        int kernels = 0;
    };
    GraphSlot g_factor;
    GraphSlot g_lu;                     // the LU of U33 alone (batched contour points)
    std::map<int, GraphSlot> g_solve;   // correction solve, keyed by nrhs
    std::map<int, GraphSlot> g_fp64;    // FP64 direct solve, keyed by nrhs
    unsigned long long launches = 0;    // kernels launched by this handle

    // tensor maps (opaque bytes, built on the host)
    alignas(64) unsigned char tm_schur[4][128];
    alignas(64) unsigned char tm_lu[6][128];  // L21 pack, U12 pack, U12 pack from row NB
    // skinny products: [0,1] [M13; M23] pack, [2,3] B pack of [W1; W2], [4,5] B pack of z3
    alignas(64) unsigned char tm_skinny[6][128];
    bool tm_ok = false;
    bool tc_skinny = false;  // mixed CF32: skinny products of the solve on the tensor cores
    int num_sms = 0;

    // panel launch configuration
    int panel_cluster_c32 = 0;   // max cluster size the device co-schedules for the FP32 / FP64
    int panel_cluster_z64 = 0;   //   panel kernels (queried once per handle)
    int panel_cluster = 0;       // cluster size used (the device's, capped by bm_opts.panel_cluster_max)
    bool panel_lane_col = true;  // FP32 panels on the lane-per-column kernel where it fits
    bool eager = false;          // bm_opts.eager: no CUDA graphs
    int opt_cluster_cap = 0;     // bm_opts.panel_cluster_max / panel_kernel of the assembled system
    int opt_panel_kernel = 0;
    int opt_test_wait = 0;       // bm_opts.test_wait_timeout
    Plan nd_plan;                // plan of the assembled system
    bool post_pending = false;   // assembled with its kernels deferred (assemble_post not yet run)

    // per-kernel timing (bm_profile): while set, every launch is bracketed by two events on the
    // handle's stream and recorded here (graphs are bypassed)
    struct ProfRec {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec>* prof = nullptr;
};

// Brackets the launches of its scope with events when the handle is profiling (else nothing).
struct ProfScope {
    bm_ctx* c;
    const char* name;
    cudaEvent_t a = nullptr;
    ProfScope(bm_ctx* c_, const char* n) : c(c_), name(n) {
        if (c->prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, c->stream);
    }
    ~ProfScope() {
        cudaEvent_t b = nullptr;
        if (c->prof && a && cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, c->stream);
            c->prof->push_back({name, a, b});
        }
    }
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
};
#define BM_PROF_CAT2(a, b) a##b
#define BM_PROF_CAT(a, b) BM_PROF_CAT2(a, b)
#define BM_PROF(ctx, name) ProfScope BM_PROF_CAT(bm_prof_, __LINE__)(ctx, name)

// allocation helpers (api.cu)
bm_status ctx_alloc(bm_ctx* c, void** p, size_t bytes);
void ctx_free(bm_ctx* c, void* p);
size_t request_bytes(int N, int form, int prec, int nb, int nrhs);  // api.cu
void ctx_release(bm_ctx* c);                                        // api.cu

// ---------------------------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with launch_pdl may start while the previous
// kernel of its stream is still running.  It calls pdl_wait() before it touches any memory the
// previous kernels may write or read (only data that stays fixed for the whole sequence, such as
// factors during a solve, may be read before), which returns once the previous grid has completed
// and its writes are visible; pdl_trigger() then lets the next kernel start launching.  In a
// kernel launched without the attribute both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Not for cluster launches: the panel kernels (clusters) keep plain stream ordering.
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
#endif
