// Refinement residual r = r + alpha A x to FP64-level accuracy on the tensor cores.
//
// Iterative refinement needs the residual b - A x of the FP32 iterate far more accurately than
// FP32 arithmetic gives (the backward-error target is 1e-9 and the iterate is already at ~1e-7),
// and GB300 runs FP64 at ~1.2 TFLOP/s.  The product is therefore formed from exact integer
// products on the bf16 tensor cores (a splitting in the manner of Ozaki et al.):
//   * every row i of A is scaled by a power of two, 2^-e_i, so that its entries (real and imaginary
//     parts) lie in (-1/2, 1/2), and written as seven base-128 digits
//         A_ij 2^-e_i = sum_{d=1..7} a_ij,d 128^-d,   a_ij,d integers in [-64, 64]
//     (exact to 2^-50 of the row's largest entry); every column c of x likewise with 2^-f_c;
//   * each digit is an integer of at most 7 bits, so bf16 holds it exactly and every product of
//     two digits is an exact integer below 2^12;
//   * the pairs (d, d') with d + d' <= 8 are grouped by level l = d + d' - 2 (weight 128^-l), one
//     FP32 accumulator per level in tensor memory.  Over a K chunk of 256 the level sums stay below
//     2^24 (at most 7 pairs x 2 real products per complex term x 256 x 2^12), so every partial sum
//     is an integer that FP32 represents exactly: nothing is rounded inside a chunk, whatever order
//     the hardware adds in;
//   * after each chunk the seven level sums are combined and added to a running double-float sum
//     (pairs of FP32) per output; the dropped pairs (d + d' > 8) weigh below 2^-56.
// The complex product uses four real products per digit pair with the A-negate bit of the
// instruction descriptor for -Im A Im x (as the TF32 kernel does).  The x digit tiles sit one after
// another in shared memory (digit d' at rows 32 d'), and level l's accumulator at tensor-memory
// column 32 l, so one MMA of width N = 32 (7 - d) multiplies A digit d by all the x digits it pairs
// with and lands each pair in its level: four MMAs per A digit and 16-wide K step.
//
// CTA: 128 output rows x up to 32 right-hand sides, K range [kbeg, kend) (split K, deterministic
// reduction afterwards when there is more than one split).  Warp 0 issues TMA loads (per 64-wide
// K block: the 14 digit planes of x, then the 7 digit pairs (Re, Im) of A one stage at a time),
// warp 1 issues the MMAs, warps 2-9 read the level sums from tensor memory after each chunk (warps
// 2-5 the real parts, 6-9 the imaginary parts, one output row per thread) and keep the running
// sums.  All waits are bounded (2 s); a timeout sets *err and the CTA drains what it issued.
#include "common.cuh"
#include "kernels.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

namespace {

constexpr int RT_BM = 128;   // output rows per CTA
constexpr int RT_BK = 64;    // K elements per stage: bf16 rows of 128 bytes (one swizzle span)
constexpr int RT_AST = 3;    // stages of A digit pairs
constexpr int RT_TILE_A = RT_BM * RT_BK * 2;  // one digit plane of A: 16 KB
constexpr int RT_A_STAGE = 2 * RT_TILE_A;     // Re and Im of one digit
constexpr int RT_THREADS = 320;
constexpr uint64_t RT_WAIT_NS = 2000000000ull;
// D digits per operand (7: pairs to level 6, 2^-50; 9: to level 8, 2^-64) and NT right-hand sides
// per CTA (32 for D = 7, 16 for D = 9).  Level sums over a chunk stay below 2^24: D pairs x 2
// products x 4096 x chunk K, so the chunk is 256 for D = 7 and 128 for D = 9.  Tensor memory:
// real parts of levels 0..D-1 at columns NT l, imaginary parts at NT (D + l).
template <int D>
struct RtCfg {
    static constexpr int NT = D <= 7 ? 32 : 16;         // right-hand sides per CTA
    static constexpr int TILE_X = NT * RT_BK * 2;       // one digit plane of x
    static constexpr int KB_CHUNK = D <= 7 ? 4 : 2;     // K blocks of 64 per exact chunk
    static constexpr int X_BUF = 2 * D * TILE_X;        // all digits of x, Re and Im
    static constexpr int SMEM = RT_AST * RT_A_STAGE + 2 * X_BUF + 1024 + 256;
    static_assert(2 * D * NT <= 512, "the level accumulators fit tensor memory");
    static_assert(D * NT <= 256, "the widest MMA (A digit 0 against all x digits) has N <= 256");
    static_assert(D * 2 * 4096L * 64 * KB_CHUNK <= (1L << 24), "chunk sums stay exact in FP32");
    static_assert(SMEM <= 232448, "shared memory");
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on timeout or when another thread already gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > RT_WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* tmap, uint32_t bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t ta, float* v) {
    uint32_t a[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]),
          "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
        : "r"(ta)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(a[i]);
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t neg_a, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (neg_a << 13) | ((n >> 3) << 17) | ((uint32_t)(RT_BM >> 4) << 24);
}
// s + t exactly as hi + lo (Knuth's TwoSum); the rn intrinsics keep the steps from being contracted
__device__ __forceinline__ void two_sum(float& hi, float& lo, float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
}

struct RtProd {
    CUtensorMap tmA;   // the A digit planes (3-D: K, rows, 14 planes)
    CUtensorMap tmX;   // the x digit planes (3-D: K, columns, 14 planes)
    const int* eA;     // row exponents of A
    const int* fX;     // column exponents of x
    double2* C;        // output (FP64 complex), C += alpha A x
    long ldc;
    double* Wr;        // split-K workspace (S > 1): S planes of m x n, Re and Im
    double* Wi;
    int m, K, S;       // rows, K, K splits
};
struct RtJob {
    RtProd p[2];
    int nprod, n, ntile_n;  // right-hand sides, column tiles
    double alpha;
    int first_unit[3];
};

template <int D>
__global__ void __launch_bounds__(RT_THREADS, 1) resid_tc_kernel(const __grid_constant__ RtJob J, int* __restrict__ err) {
    constexpr int RT_D = D, RT_KB_CHUNK = RtCfg<D>::KB_CHUNK, RT_X_BUF = RtCfg<D>::X_BUF;
    constexpr int RT_NT = RtCfg<D>::NT, RT_TILE_X = RtCfg<D>::TILE_X;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                               // RT_AST stages of (Re, Im) digit tiles of A
    uint8_t* sX = smem + RT_AST * RT_A_STAGE;         // 2 buffers of all 14 digit tiles of x
    uint64_t* bars = reinterpret_cast<uint64_t*>(sX + 2 * RT_X_BUF);
    // afull[3], aempty[3], xfull[2], xempty[2], accfull, accempty, drain
    const uint32_t afull = su32(bars), aempty = afull + 8 * RT_AST, xfull = aempty + 8 * RT_AST;
    const uint32_t xempty = xfull + 16, accfull = xempty + 16, accempty = accfull + 8, drain = accempty + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * RT_AST + 7);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    // ---- work unit: product q, row tile, K split z, column tile ----
    const int q = (int)blockIdx.x >= J.first_unit[1] ? 1 : 0;
    const RtProd& P = J.p[q];
    int u = (int)blockIdx.x - J.first_unit[q];
    const int tn = u % J.ntile_n;
    u /= J.ntile_n;
    const int z = u % P.S, it = u / P.S;
    const int nkb_all = (P.K + RT_BK - 1) / RT_BK;
    const int kb0 = (int)((long)z * nkb_all / P.S), kb1 = (int)((long)(z + 1) * nkb_all / P.S);
    const int nkb = kb1 - kb0;
    const int nchunks = (nkb + RT_KB_CHUNK - 1) / RT_KB_CHUNK;
    const int row0 = it * RT_BM, col0 = tn * RT_NT;
    const int ncols = min(RT_NT, J.n - col0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RT_AST; ++s) {
            mbar_init(afull + 8 * s, 1);
            mbar_init(aempty + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(xfull + 8 * s, 1);
            mbar_init(xempty + 8 * s, 1);
        }
        mbar_init(accfull, 1);
        mbar_init(accempty, 256);  // the eight reading warps
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int a_issued = 0, x_issued = 0;
        for (int kb = 0; kb < nkb && !*abort_flag; ++kb) {
            const int xb = kb & 1;
            if (kb >= 2 && !mbar_wait(xempty + 8 * xb, (uint32_t)((kb >> 1) - 1) & 1u, abort_flag)) break;
            const int kx = (kb0 + kb) * RT_BK;
            mbar_expect_tx(xfull + 8 * xb, RT_X_BUF);
            uint8_t* xbuf = sX + xb * RT_X_BUF;
            // shared layout: the seven real-part digit tiles, then the seven imaginary-part ones
            for (int pl = 0; pl < 2 * RT_D; ++pl)
                tma_load_3d(su32(xbuf + ((pl & 1) * RT_D + (pl >> 1)) * RT_TILE_X), &P.tmX, xfull + 8 * xb, kx, col0,
                            pl);
            x_issued = kb + 1;
            for (int d = 0; d < RT_D; ++d) {
                const int idx = kb * RT_D + d, s = idx % RT_AST;
                if (idx >= RT_AST && !mbar_wait(aempty + 8 * s, (uint32_t)(idx / RT_AST - 1) & 1u, abort_flag)) break;
                uint8_t* as = sA + s * RT_A_STAGE;
                mbar_expect_tx(afull + 8 * s, RT_A_STAGE);
                tma_load_3d(su32(as), &P.tmA, afull + 8 * s, kx, row0, 2 * d);
                tma_load_3d(su32(as + RT_TILE_A), &P.tmA, afull + 8 * s, kx, row0, 2 * d + 1);
                a_issued = idx + 1;
            }
        }
        if (*abort_flag) {
            // copies already in flight land before shared memory is released
            for (int idx = (a_issued > RT_AST ? a_issued - RT_AST : 0); idx < a_issued; ++idx) {
                const uint64_t t0 = gtimer();
                while (!mbar_try(afull + 8 * (idx % RT_AST), (uint32_t)(idx / RT_AST) & 1u) && gtimer() - t0 < RT_WAIT_NS) {
                }
            }
            for (int kb = (x_issued > 2 ? x_issued - 2 : 0); kb < x_issued; ++kb) {
                const uint64_t t0 = gtimer();
                while (!mbar_try(xfull + 8 * (kb & 1), (uint32_t)(kb >> 1) & 1u) && gtimer() - t0 < RT_WAIT_NS) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int ch = kb / RT_KB_CHUNK, first_of_chunk = (kb % RT_KB_CHUNK) == 0;
            // the readers have taken the previous chunk's level sums out of tensor memory
            if (first_of_chunk && ch > 0 && !mbar_wait(accempty, (uint32_t)(ch - 1) & 1u, abort_flag)) break;
            const int xb = kb & 1;
            if (!mbar_wait(xfull + 8 * xb, (uint32_t)(kb >> 1) & 1u, abort_flag)) break;
            fence_after();
            const uint32_t xbase = su32(sX + xb * RT_X_BUF);
            for (int d = 0; d < RT_D; ++d) {
                const int idx = kb * RT_D + d, s = idx % RT_AST;
                if (!mbar_wait(afull + 8 * s, (uint32_t)(idx / RT_AST) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t ar = su32(sA + s * RT_A_STAGE), ai = ar + RT_TILE_A;
                // x digits 0 .. 6 - d (rows 0 .. 32 (7 - d) of the stacked tiles) into levels d .. 6
                const uint32_t nw = (uint32_t)(RT_NT * (RT_D - d));
                const uint32_t idp = idesc_bf16(0, nw), idn = idesc_bf16(1, nw);
                const uint32_t Dr = tmem + (uint32_t)(d * RT_NT), Di = Dr + RT_D * RT_NT;
                const uint32_t xr = xbase, xi = xbase + RT_D * RT_TILE_X;
#pragma unroll
                for (int kk = 0; kk < RT_BK / 16; ++kk) {
                    const uint32_t off = kk * 32;  // 16 bf16 = 32 bytes along K inside the swizzle span
                    const uint64_t dar = desc_sw128(ar + off), dai = desc_sw128(ai + off);
                    const uint64_t dxr = desc_sw128(xr + off), dxi = desc_sw128(xi + off);
                    // digit 0 of A reaches every level: its first product of a chunk overwrites them
                    const uint32_t acc = (first_of_chunk && d == 0 && kk == 0) ? 0u : 1u;
                    mma_bf16(Dr, dar, dxr, idp, acc);
                    mma_bf16(Dr, dai, dxi, idn, 1u);
                    mma_bf16(Di, dar, dxi, idp, acc);
                    mma_bf16(Di, dai, dxr, idp, 1u);
                }
                mma_commit(aempty + 8 * s);
            }
            if (!ok) break;
            mma_commit(xempty + 8 * xb);
            if ((kb % RT_KB_CHUNK) == RT_KB_CHUNK - 1 || kb == nkb - 1) mma_commit(accfull);
        }
        if (*abort_flag) {
            // products already issued finish before tensor memory and shared memory are released
            mma_commit(drain);
            const uint64_t t0 = gtimer();
            while (!mbar_try(drain, 0u) && gtimer() - t0 < RT_WAIT_NS) {
            }
        }
    } else if (warp >= 2) {
        // ---------------- level-sum readers: warps 2-5 real parts, 6-9 imaginary parts ----------------
        const int qw = warp & 3;  // tensor-memory lane quarter this warp may read
        const int part = warp >= 6 ? 1 : 0;
        const uint32_t lane_off = (uint32_t)(qw * 32) << 16;
        float sh[RT_NT], sl[RT_NT];  // running double-float sums of this row's outputs
#pragma unroll
        for (int j = 0; j < RT_NT; ++j) sh[j] = sl[j] = 0.f;
        for (int ch = 0; ch < nchunks; ++ch) {
            if (!mbar_wait(accfull, (uint32_t)ch & 1u, abort_flag)) break;
            fence_after();
#pragma unroll
            for (int g = 0; g < RT_NT / 16; ++g) {
                float th[16], tl[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) th[j] = tl[j] = 0.f;
                // level sums are exact integers; scale by 128^-l (exact) and add in double-float
#pragma unroll 1
                for (int lev = 0; lev < RT_D; ++lev) {
                    float v[16];
                    tmem_ld16(tmem + lane_off + (uint32_t)(part * RT_D * RT_NT + lev * RT_NT + g * 16), v);
                    const float w = __int_as_float((127 - 7 * lev) << 23);  // 2^(-7 lev)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float hi, lo;
                        two_sum(hi, lo, th[j], v[j] * w);
                        th[j] = hi;
                        tl[j] = __fadd_rn(tl[j], lo);
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    // (sh, sl) += (th, tl)
                    float hi, lo;
                    two_sum(hi, lo, sh[g * 16 + j], th[j]);
                    lo = __fadd_rn(lo, __fadd_rn(sl[g * 16 + j], tl[j]));
                    const float s2 = __fadd_rn(hi, lo);
                    sl[g * 16 + j] = __fsub_rn(lo, __fsub_rn(s2, hi));
                    sh[g * 16 + j] = s2;
                }
            }
            fence_before();
            mbar_arrive(accempty);
        }
        if (!*abort_flag) {
            const int row = row0 + qw * 32 + lane;
            if (row < P.m) {
                // value = 128^-2 2^(e_row + f_col) sum  (digits carry 128^-d each)
                const int er = P.eA[row];
#pragma unroll
                for (int j = 0; j < RT_NT; ++j) {
                    if (j >= ncols) break;
                    const int col = col0 + j;
                    const double v = ldexp((double)sh[j] + (double)sl[j], er + P.fX[col] - 14);
                    if (P.S == 1) {
                        double* o = reinterpret_cast<double*>(P.C + row + (long)col * P.ldc) + part;
                        *o += J.alpha * v;
                    } else {
                        double* W = part ? P.Wi : P.Wr;
                        W[((long)z * J.n + col) * P.m + row] = v;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

// C += alpha sum_z W[z]  (z in order; W: S planes of n columns of m rows, Re and Im)
__global__ void rt_reduce_kernel(const double* __restrict__ Wr, const double* __restrict__ Wi, int S, int m, int n,
                                 double alpha, double2* __restrict__ C, long ldc) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long zs = (long)m * n;
    if (idx >= zs) return;
    const int j = (int)(idx / m), i = (int)(idx % m);
    double re = 0.0, im = 0.0;
    for (int z = 0; z < S; ++z) {
        re += Wr[idx + z * zs];
        im += Wi[idx + z * zs];
    }
    double2& c = C[i + (long)j * ldc];
    c.x += alpha * re;
    c.y += alpha * im;
}

// Row maxima of A (rows x K, column-major FP64 complex) over max(|Re|, |Im|): each thread a row and
// 256 columns, combined by an atomic maximum on the bit patterns (non-negative doubles order as
// their bits).  mx must start at zero.
__global__ void row_max_kernel(const double2* __restrict__ A, long lda, int rows, int K,
                               unsigned long long* __restrict__ mx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int j0 = blockIdx.y * 256, j1 = min(K, j0 + 256);
    // |Re|, |Im| as bit patterns with the sign cleared (integer maximum: FP64 compares run on the
    // narrow FP64 pipe).  NaN patterns (above that of infinity) count as zero, as fmax would skip them.
    constexpr unsigned long long MAG = 0x7FFFFFFFFFFFFFFFull, INF = 0x7FF0000000000000ull;
    auto mag = [](double d) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(d) & MAG;
        return b > INF ? 0ull : b;
    };
    unsigned long long m = 0;
    const double2* a = A + i;
    int j = j0;
    for (; j + 8 <= j1; j += 8) {
        double2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = a[(long)(j + u) * lda];
#pragma unroll
        for (int u = 0; u < 8; ++u) m = max(m, max(mag(v[u].x), mag(v[u].y)));
    }
    for (; j < j1; ++j) {
        const double2 v = a[(long)j * lda];
        m = max(m, max(mag(v.x), mag(v.y)));
    }
    atomicMax(mx + i, m);
}
// e_i with max_j max(|Re|, |Im|) < 2^(e_i - 1) (0 for a zero row)
__global__ void row_exponent_kernel(const unsigned long long* __restrict__ mx, int rows, int* __restrict__ e) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const double m = __longlong_as_double((long long)mx[i]);
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);  // m = f 2^ex, f in [1/2, 1)
    e[i] = m > 0.0 ? ex + 1 : 0;
}

// bf16 bit pattern of a small integer r, |r| <= 128 (exact: at most 8 significant bits)
__device__ __forceinline__ unsigned short bf16_of_int(int r) {
    if (r == 0) return 0;
    const unsigned a = (unsigned)abs(r);
    const int e = 31 - __clz(a);  // position of the leading bit, 0..7
    const unsigned mant = (a << (7 - e)) & 0x7Fu;
    return (unsigned short)((r < 0 ? 0x8000u : 0u) | ((unsigned)(127 + e) << 7) | mant);
}

// The nd base-128 digits of v 2^-ex (|v 2^-ex| < 1/2), most significant first, each an integer in
// [-64, 64]: v 2^(7 nd - ex) rounded to the nearest integer M (|M| <= 2^(7 nd - 1)), written as
// M = sum_d a_d 128^(nd - 1 - d) with balanced digits in [-64, 63] peeled off from the least
// significant end and the most significant digit the remainder (which may be +64).
// Integer arithmetic on the FP64 bit pattern only (FP64 arithmetic and conversions are slow here).
__device__ __forceinline__ void digits_of(double v, int ex, int nd, __nv_bfloat16* out, long stride) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((bits >> 52) & 0x7FF);
    long long M = 0;
    // zero and subnormals (below any row scale used here) give zero digits; so does a value that
    // does not fit its scale (only possible for non-finite data, which the backward error reports)
    if (E != 0 && E != 0x7FF) {
        const long long mant = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
        const int sh = E - 1075 + 7 * nd - ex;  // v 2^(7 nd - ex) = mant 2^sh, mant in [2^52, 2^53)
        if (sh > 7 * nd - 54)                   // |v 2^-ex| >= 1/2: does not fit the scale
            M = 0;
        else if (sh >= 0)
            M = mant << sh;
        else if (sh > -62)
            M = (mant + (1ll << (-sh - 1))) >> (-sh);  // round half up
        if (bits >> 63) M = -M;
    }
    for (int d = nd - 1; d >= 1; --d) {
        int r = (int)(M & 127);
        if (r >= 64) r -= 128;
        M = (M - r) >> 7;
        reinterpret_cast<unsigned short*>(out)[d * stride] = bf16_of_int(r);
    }
    reinterpret_cast<unsigned short*>(out)[0] = bf16_of_int((int)M);
}

// Digit planes of A: plane 2d + part holds digit d of the real (part 0) or imaginary (1) parts, K-major
// ([row][ldk]); written through a 32 x 32 shared tile so both sides are coalesced.
__global__ void digits_a_kernel(const double2* __restrict__ A, long lda, int rows, int K, const int* __restrict__ e,
                                __nv_bfloat16* __restrict__ D, long ldk, long plane, int nd) {
    __shared__ double2 t[32][33];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + tx, k = k0 + q;
        t[q][tx] = (r < rows && k < K) ? A[r + (long)k * lda] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, k = k0 + tx;
        if (r >= rows || k >= K) continue;
        const double2 v = t[tx][q];
        const int ex = e[r];
        __nv_bfloat16* o = D + (long)r * ldk + k;
        digits_of(v.x, ex, nd, o, 2 * plane);
        digits_of(v.y, ex, nd, o + plane, 2 * plane);
    }
}

// Column exponents of x over rows [r0, r0 + K) for the n columns (one block per column).
__global__ void col_exponent_kernel(const double2* __restrict__ X, long ldx, int r0, int K, int* __restrict__ f) {
    const int c = blockIdx.x;
    double mx = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const double2 v = X[r0 + i + (long)c * ldx];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sm[w]);
        int ex = 0;
        if (mx > 0.0 && isfinite(mx)) frexp(mx, &ex);
        f[c] = (mx > 0.0 && isfinite(mx)) ? ex + 1 : 0;
    }
}

// Digit planes of x rows [r0, r0 + K) (columns c < n; columns up to npad are zero): plane 2d + part,
// layout [col][ldk].
__global__ void digits_x_kernel(const double2* __restrict__ X, long ldx, int r0, int K, int n, int npad,
                                const int* __restrict__ f, __nv_bfloat16* __restrict__ D, long ldk, long plane,
                                int nd) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)npad * K) return;
    const int c = (int)(idx / K), k = (int)(idx % K);
    __nv_bfloat16* o = D + (long)c * ldk + k;
    if (c >= n) {
        for (int p = 0; p < 2 * nd; ++p) o[p * plane] = __float2bfloat16_rn(0.f);
        return;
    }
    const double2 v = X[r0 + k + (long)c * ldx];
    const int ex = f[c];
    digits_of(v.x, ex, nd, o, 2 * plane);
    digits_of(v.y, ex, nd, o + plane, 2 * plane);
}

PFN_cuTensorMapEncodeTiled_v12000 rt_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

// 3-D tensor map over 14 bf16 digit planes, each [rows][ldk] (K-major): dims {K, rows, 14},
// box {64, box_rows, 1}, 128-byte swizzle; reads outside {K, rows} return zeros.
bm_status rt_make_map(void* tmap, const void* base, long rows, long K, long ldk, long plane_elems, int box_rows,
                      int nd) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = rt_encode();
    if (enc == nullptr) {
        bm_set_error("cuTensorMapEncodeTiled is unavailable from the driver");
        return BM_ECUDA;
    }
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ldk * 2) % 16 != 0 || (plane_elems * 2) % 16 != 0) {
        bm_set_error("digit-plane tensor map: base or stride not 16-byte aligned");
        return BM_EINVAL;
    }
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)(2 * nd)};
    cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)plane_elems * 2};
    cuuint32_t box[3] = {(cuuint32_t)RT_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(tmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base),
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        bm_set_error("cuTensorMapEncodeTiled (digit planes) failed with code " + std::to_string((int)r));
        return BM_ECUDA;
    }
    return BM_OK;
}

long rt_ldk(long K) { return (K + RT_BK - 1) / RT_BK * RT_BK; }
int rt_digit_planes(int nd) { return 2 * nd; }
int rt_col_tile(int nd) { return nd <= 7 ? RtCfg<7>::NT : RtCfg<9>::NT; }

// Row exponents and digit planes of A; rowmax is scratch of `rows` 8-byte words.
cudaError_t launch_digits_a(cudaStream_t s, const double2* A, long lda, int rows, int K, int* e, void* D, long ldk,
                            void* rowmax, int nd) {
    if (rows <= 0 || K <= 0) return cudaSuccess;
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(rowmax);
    cudaError_t err = cudaMemsetAsync(mx, 0, (size_t)rows * 8, s);
    if (err != cudaSuccess) return err;
    row_max_kernel<<<dim3(ceil_div(rows, 128), ceil_div(K, 256)), 128, 0, s>>>(A, lda, rows, K, mx);
    row_exponent_kernel<<<ceil_div(rows, 128), 128, 0, s>>>(mx, rows, e);
    dim3 blk(32, 8), grid(ceil_div(K, 32), ceil_div(rows, 32));
    digits_a_kernel<<<grid, blk, 0, s>>>(A, lda, rows, K, e, reinterpret_cast<__nv_bfloat16*>(D), ldk,
                                         (long)rows * ldk, nd);
    return cudaGetLastError();
}

cudaError_t launch_digits_x(cudaStream_t s, const double2* X, long ldx, int r0, int K, int n, int npad, int* f,
                            void* D, long ldk, int nd) {
    if (n <= 0 || K <= 0) return cudaSuccess;
    col_exponent_kernel<<<n, 256, 0, s>>>(X, ldx, r0, K, f);
    const long t = (long)npad * K;
    digits_x_kernel<<<ceil_div(t, 256L), 256, 0, s>>>(X, ldx, r0, K, n, npad, f, reinterpret_cast<__nv_bfloat16*>(D),
                                                      ldk, (long)npad * ldk, nd);
    return cudaGetLastError();
}

// K splits of the products of one residual launch.  A CTA holds a whole SM (its shared memory
// and all 512 tensor-memory columns), so the launch aims at one CTA per SM: every CTA covers
// ceil(work / SMs) K blocks of 64, at least 4 (the set-up and the x digit loads amortised) and at
// most 32, where work counts the K blocks of every row and column tile of the launch.  Large
// systems land on 32 (N = 4096: two and four splits); small ones split further, so that, e.g., a
// 1024-point mixed system with 16 right-hand sides runs 128 CTAs instead of 24.  Every split keeps
// at least one K block (S <= K blocks).
void rt_plan_splits(int nprod, const long* m, const long* K, int n, int nd, int num_sms, int* S) {
    auto cdiv = [](long a, long b) { return (a + b - 1) / b; };
    const long ntn = cdiv(n, rt_col_tile(nd));
    long work = 0;
    for (int q = 0; q < nprod; ++q) work += cdiv(m[q], RT_BM) * ntn * cdiv(K[q], RT_BK);
    const long per = std::min(32L, std::max(4L, cdiv(work, std::max(num_sms, 1))));
    for (int q = 0; q < nprod; ++q) {
        const long kb = cdiv(K[q], RT_BK);
        S[q] = (int)std::max(1L, std::min(std::min(16L, kb), cdiv(kb, per)));
    }
}

// The products of one residual (at most two, sharing n and alpha): C += alpha A x each.  A product
// with S > 1 K splits writes S m n doubles (Re and Im) to its workspace, reduced in order afterwards.
cudaError_t gemm_rt(cudaStream_t s, const RtArgs* prods, int nprod, int n, double alpha, int* d_err, int* launched,
                    int nd) {
    if (nprod < 1 || nprod > 2 || n <= 0 || (nd != 7 && nd != 9)) return cudaSuccess;
    static DeviceFlags attr7, attr9;
    if (nd == 7 && attr7.pending()) {
        cudaError_t e = cudaFuncSetAttribute(resid_tc_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             RtCfg<7>::SMEM);
        if (e != cudaSuccess) return e;
        attr7.done();
    }
    if (nd == 9 && attr9.pending()) {
        cudaError_t e = cudaFuncSetAttribute(resid_tc_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             RtCfg<9>::SMEM);
        if (e != cudaSuccess) return e;
        attr9.done();
    }
    RtJob J{};
    J.nprod = nprod;
    J.n = n;
    J.ntile_n = ceil_div(n, rt_col_tile(nd));
    J.alpha = alpha;
    int u = 0;
    for (int q = 0; q < 2; ++q) {
        J.first_unit[q] = u;
        if (q < nprod) {
            const RtArgs& a = prods[q];
            RtProd& p = J.p[q];
            std::memcpy(&p.tmA, a.tmA, sizeof(CUtensorMap));
            std::memcpy(&p.tmX, a.tmX, sizeof(CUtensorMap));
            p.eA = a.eA;
            p.fX = a.fX;
            p.C = a.C;
            p.ldc = a.ldc;
            p.Wr = a.Wr;
            p.Wi = a.Wi;
            p.m = a.m;
            p.K = a.K;
            p.S = a.S;
            if (a.m > 0 && a.K > 0) u += ceil_div(a.m, RT_BM) * a.S * J.ntile_n;
        }
    }
    J.first_unit[2] = u;
    if (nprod == 1) J.first_unit[1] = u;
    if (u == 0) return cudaSuccess;
    if (nd == 7)
        resid_tc_kernel<7><<<u, RT_THREADS, RtCfg<7>::SMEM, s>>>(J, d_err);
    else
        resid_tc_kernel<9><<<u, RT_THREADS, RtCfg<9>::SMEM, s>>>(J, d_err);
    *launched += 1;
    for (int q = 0; q < nprod; ++q) {
        const RtArgs& a = prods[q];
        if (a.S > 1 && a.m > 0 && a.K > 0) {
            const long t = (long)a.m * n;
            rt_reduce_kernel<<<ceil_div(t, 256L), 256, 0, s>>>(a.Wr, a.Wi, a.S, a.m, n, alpha, a.C, a.ldc);
            *launched += 1;
        }
    }
    return cudaGetLastError();
}
