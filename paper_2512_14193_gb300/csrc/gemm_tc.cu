// Complex GEMM on the 5th-generation tensor cores (sm_103a): C = beta C + alpha A B^T with
// A (m x K) and B (n x K) given as K-major planar FP32 packs, computed in TF32 with FP32
// accumulation in tensor memory.  This is the contraction of Theorem thm:LU
// (U33 = -[M31 M32][M13; M23]) and of every LU trailing update A22 -= L21 U12.
//
// Complex product with four real products ("4M") on planar operands:
//     Dr = Ar Br^T - Ai Bi^T,  Di = Ar Bi^T + Ai Br^T
// Two TMEM accumulators (128 lanes x 128 columns each); the minus sign uses the A-negate bit of
// the instruction descriptor.  The 3xTF32 variant needs no kernel change: its packs repeat the
// K range as [A_hi | A_hi | A_lo] and [B_hi | B_lo | B_hi], so one K-extended product sums
// A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// CTA tile 128 x 128, K step 32 (128-byte rows), 3-stage TMA -> shared-memory pipeline with
// mbarriers.  Warp 0 lane 0 issues TMA loads, warp 1 lane 0 issues tcgen05.mma; all four warps
// then read the accumulators (tcgen05.ld 32x32b, warp w owns TMEM lanes 32(w mod 4) .. +31 = rows)
// and update C with coalesced column-major stores.  For C = C + alpha A B^T (the LU trailing
// updates) a six-warp form loads the C tile into the upper half of TMEM during the main loop, so
// the epilogue only stores.  Every mbarrier wait is bounded (2 s by the global timer); a timeout
// sets *err, skips the epilogue, waits for issued copies and products and frees TMEM.  err[1] is
// a test hook: when it is set the MMA warp first waits on a barrier that nothing completes, gives
// up after 1 ms and takes that timeout path without issuing any product.
#include "common.cuh"
#include "kernels.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <vector>

namespace {

constexpr int BM = TC_BM, BN = TC_BN;
constexpr int BKE = 32;  // K elements per stage (fp32: 128-byte rows, one swizzle span)
constexpr int STAGES = 3;
constexpr int TILE_A = BM * BKE * 4;
constexpr int TILE_B = BN * BKE * 4;
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 2 * BN;  // Dr, Di
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr uint64_t TEST_WAIT_NS = 1000000ull;  // the test hook's wait limit

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; returns false on timeout or when another thread already gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive fp32 accumulator columns of this thread's TMEM lane, of two accumulators (real
// and imaginary part), one wait for both
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
    uint32_t a[16], b[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
        "[%33];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]),
          "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(b[0]),
          "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]),
          "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        va[i] = __uint_as_float(a[i]);
        vb[i] = __uint_as_float(b[i]);
    }
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M = 128, N = BN.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t neg_a) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (neg_a << 13) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

// Output modes: OUT_C32 C (FP32 planar) = beta C + alpha D; OUT_Z64 C64 (FP64) = beta C64 + alpha D;
// OUT_PART the raw D of this K split to a workspace slice (split-K partial sums); OUT_C32_PRE as
// OUT_C32 for beta != 0, with six warps: warps 2-5 copy the C tile into TMEM columns 2BN..4BN while
// the MMAs run, so the epilogue reads D and C from TMEM and only stores (the C loads no longer
// follow the main loop; one CTA per SM leaves nothing else to overlap them with).
enum { OUT_C32 = 0, OUT_Z64 = 1, OUT_PART = 2, OUT_C32_PRE = 3 };

template <int OUT>
__host__ __device__ constexpr int tc_threads() { return OUT == OUT_C32_PRE ? 192 : 128; }
template <int OUT>
__host__ __device__ constexpr uint32_t tc_tmem_cols() { return OUT == OUT_C32_PRE ? 2 * TMEM_COLS : TMEM_COLS; }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The body of one CTA: tile (tm, tn) of C, K split z of S.  The four tensor maps are param-space
// copies (single product) or global-memory entries of a batch.
template <int OUT>
__device__ __forceinline__ void cgemm_tc_body(const CUtensorMap& tmAr, const CUtensorMap& tmAi, const CUtensorMap& tmBr,
                                              const CUtensorMap& tmBi, float* __restrict__ Cr, float* __restrict__ Ci,
                                              double2* __restrict__ C64, long ldc, long zstride, int m, int n, int kext,
                                              int S, int zsplit, float alpha, float beta, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // full[S], empty[S], done, never (the test hook's barrier: initialised, never arrived on)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tm = blockIdx.x, tn = blockIdx.y;
    // this CTA's K split: k-blocks [kb_begin, kb_begin + nkb)
    const int nkb_all = (kext + BKE - 1) / BKE;
    const int kb_begin = (int)((long)zsplit * nkb_all / S);
    const int nkb = (int)((long)(zsplit + 1) * nkb_all / S) - kb_begin;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
    const uint32_t never = smem_u32(bars + 2 * STAGES + 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        mbar_init(never, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), tc_tmem_cols<OUT>());
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t Dr = tmem, Di = tmem + BN;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag)) break;
            uint8_t* st = smem + s * STAGE_BYTES;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, STAGE_BYTES);
            const int kx = (kb_begin + kb) * BKE;
            tma_load_2d(smem_u32(st), &tmAr, fb, kx, tm * BM);
            tma_load_2d(smem_u32(st + TILE_A), &tmAi, fb, kx, tm * BM);
            tma_load_2d(smem_u32(st + 2 * TILE_A), &tmBr, fb, kx, tn * BN);
            tma_load_2d(smem_u32(st + 2 * TILE_A + TILE_B), &tmBi, fb, kx, tn * BN);
            issued = kb + 1;
        }
        if (*abort_flag) {
            // let copies already in flight land before shared memory is released
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb) {
                const uint64_t t0 = gtimer();
                while (!mbar_try(full0 + 8 * (kb % STAGES), (uint32_t)(kb / STAGES) & 1u) && gtimer() - t0 < WAIT_NS) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idp = idesc_tf32(0), idn = idesc_tf32(1);
        if (err[1] != 0) {
            // test hook: a wait that nothing ends, bounded like every other wait
            const uint64_t t0 = gtimer();
            while (!mbar_try(never, 0u) && gtimer() - t0 < TEST_WAIT_NS) {
            }
            *abort_flag = 1;
        }
        for (int kb = 0; kb < nkb && !*abort_flag; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (!mbar_wait(full0 + 8 * s, ph, abort_flag)) break;
            fence_after();
            const uint32_t ar = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t ai = ar + TILE_A, br = ar + 2 * TILE_A, bi = br + TILE_B;
#pragma unroll
            for (int kk = 0; kk < BKE / 8; ++kk) {
                const uint32_t off = kk * 32;  // 8 tf32 = 32 bytes along K inside the swizzle span
                const uint64_t dar = desc_sw128(ar + off), dai = desc_sw128(ai + off);
                const uint64_t dbr = desc_sw128(br + off), dbi = desc_sw128(bi + off);
                const uint32_t acc = (kb | kk) ? 1u : 0u;
                mma_tf32(Dr, dar, dbr, idp, acc);
                mma_tf32(Dr, dai, dbi, idn, 1u);
                mma_tf32(Di, dar, dbi, idp, acc);
                mma_tf32(Di, dai, dbr, idp, 1u);
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);
        if (*abort_flag) {
            // the products already issued finish (and the commit lands) before TMEM and shared
            // memory are released
            const uint64_t t0 = gtimer();
            while (!mbar_try(done, 0u) && gtimer() - t0 < WAIT_NS) {
            }
        }
    }
    __syncwarp();
    if (OUT == OUT_C32_PRE && warp >= 2) {
        // ---------------- C tile -> TMEM while the MMAs run (warps 2-5) ----------------
        const int qw = warp & 3;  // TMEM lane quarter this warp may access
        const long row = (long)tm * BM + qw * 32 + lane;
        const uint32_t lane_off = (uint32_t)(qw * 32) << 16;
        const long col0 = (long)tn * BN;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float cr[16], ci[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const long col = col0 + c0 + q;
                const bool in = row < m && col < n;
                cr[q] = in ? __ldg(Cr + row + col * ldc) : 0.f;
                ci[q] = in ? __ldg(Ci + row + col * ldc) : 0.f;
            }
            tmem_st16(Dr + 2 * BN + lane_off + c0, cr);
            tmem_st16(Di + 2 * BN + lane_off + c0, ci);
        }
        tmem_wait_st();
    }
    // ---------------- epilogue: all four warps (warps 2-5 in OUT_C32_PRE) ----------------
    mbar_wait(done, 0, abort_flag);
    fence_before();
    __syncthreads();  // the abort decision below must be uniform: tcgen05.ld is warp-synchronous
    fence_after();
    if (!*abort_flag && (OUT != OUT_C32_PRE || warp >= 2)) {
        const int qw = (OUT == OUT_C32_PRE) ? (warp & 3) : warp;
        const long row = (long)tm * BM + qw * 32 + lane;
        const uint32_t lane_off = (uint32_t)(qw * 32) << 16;
        const long col0 = (long)tn * BN;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float vr[16], vi[16];
            tmem_ld16x2(Dr + lane_off + c0, Di + lane_off + c0, vr, vi);
            if (OUT == OUT_C32_PRE) {
                float cr[16], ci[16];
                tmem_ld16x2(Dr + 2 * BN + lane_off + c0, Di + 2 * BN + lane_off + c0, cr, ci);
                if (row < m) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const long col = col0 + c0 + q;
                        if (col < n) {
                            const long o = row + col * ldc;
                            Cr[o] = fmaf(beta, cr[q], alpha * vr[q]);
                            Ci[o] = fmaf(beta, ci[q], alpha * vi[q]);
                        }
                    }
                }
            } else if (OUT == OUT_PART && row < m) {
                // slice z of the workspace: m x n column-major, leading dimension ldc (= m)
                float* Pr = Cr + (long)zsplit * zstride;
                float* Pi = Ci + (long)zsplit * zstride;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const long col = col0 + c0 + q;
                    if (col < n) {
                        Pr[row + col * ldc] = vr[q];
                        Pi[row + col * ldc] = vi[q];
                    }
                }
            } else if (OUT == OUT_Z64 && row < m) {
                double2 cz[16];
                if (beta != 0.f) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const long col = col0 + c0 + q;
                        cz[q] = (col < n) ? C64[row + col * ldc] : make_double2(0.0, 0.0);
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const long col = col0 + c0 + q;
                    if (col < n) {
                        double r = (double)alpha * (double)vr[q], im = (double)alpha * (double)vi[q];
                        if (beta != 0.f) {
                            r = fma((double)beta, cz[q].x, r);
                            im = fma((double)beta, cz[q].y, im);
                        }
                        C64[row + col * ldc] = make_double2(r, im);
                    }
                }
            } else if (OUT == OUT_C32 && row < m) {
                // issue every load of this 16-column chunk before any store, so the chunk costs
                // one memory round trip instead of sixteen
                float cr[16], ci[16];
                if (beta != 0.f) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const long col = col0 + c0 + q;
                        cr[q] = (col < n) ? __ldg(Cr + row + col * ldc) : 0.f;
                        ci[q] = (col < n) ? __ldg(Ci + row + col * ldc) : 0.f;
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const long col = col0 + c0 + q;
                    if (col < n) {
                        const long o = row + col * ldc;
                        float r = alpha * vr[q], im = alpha * vi[q];
                        if (beta != 0.f) {
                            r = fmaf(beta, cr[q], r);
                            im = fmaf(beta, ci[q], im);
                        }
                        Cr[o] = r;
                        Ci[o] = im;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, tc_tmem_cols<OUT>());
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

template <int OUT>
__global__ void __launch_bounds__(192, 1)
    cgemm_tc_kernel(const __grid_constant__ CUtensorMap tmAr, const __grid_constant__ CUtensorMap tmAi,
                    const __grid_constant__ CUtensorMap tmBr, const __grid_constant__ CUtensorMap tmBi,
                    float* __restrict__ Cr, float* __restrict__ Ci, double2* __restrict__ C64, long ldc, long zstride,
                    int m, int n, int kext, int S, float alpha, float beta, int* __restrict__ err) {
    cgemm_tc_body<OUT>(tmAr, tmAi, tmBr, tmBi, Cr, Ci, C64, ldc, zstride, m, n, kext, S, (int)blockIdx.z, alpha, beta,
                       err);
}

// One product per blockIdx.z: C_z = beta C_z + alpha A_z B_z^T for a batch of equal-shape products
// (the contour points' Schur complements), maps and outputs read from global memory.
struct alignas(64) TcBatchEntry {
    CUtensorMap map[4];  // A re, A im, B re, B im
    float* Cr;
    float* Ci;
    long ldc;
};
__global__ void __launch_bounds__(128, 1)
    cgemm_tc_batch_kernel(const TcBatchEntry* __restrict__ E, int m, int n, int kext, float alpha, int* __restrict__ err) {
    const TcBatchEntry& e = E[blockIdx.z];
    cgemm_tc_body<OUT_C32>(e.map[0], e.map[1], e.map[2], e.map[3], e.Cr, e.Ci, nullptr, e.ldc, 0, m, n, kext, 1, 0,
                           alpha, 0.f, err);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

// 2-D tensor map over a row-major [rows][ldk] FP32 pack: dims {kext, rows}, box {32, box_rows},
// 128-byte swizzle; reads outside {kext, rows} return zeros.
bm_status tc_make_map(void* tmap, const float* base, long rows, long kext, long ldk, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (enc == nullptr) {
        bm_set_error("cuTensorMapEncodeTiled is unavailable from the driver");
        return BM_ECUDA;
    }
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ldk * 4) % 16 != 0) {
        bm_set_error("tensor map: base or stride not 16-byte aligned");
        return BM_EINVAL;
    }
    cuuint64_t dims[2] = {(cuuint64_t)kext, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 4};
    cuuint32_t box[2] = {(cuuint32_t)BKE, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(tmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base),
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        bm_set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return BM_ECUDA;
    }
    return BM_OK;
}

namespace {

template <int OUT>
cudaError_t launch_tc(cudaStream_t s, dim3 grid, const void* tAr, const void* tAi, const void* tBr, const void* tBi,
                      float* Cr, float* Ci, double2* C64, long ldc, long zstride, int m, int n, int kext, int S,
                      float alpha, float beta, int* d_err) {
    static DeviceFlags attr_set;
    if (attr_set.pending()) {
        cudaError_t e =
            cudaFuncSetAttribute(cgemm_tc_kernel<OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set.done();
    }
    cgemm_tc_kernel<OUT><<<grid, tc_threads<OUT>(), SMEM_BYTES, s>>>(
        *reinterpret_cast<const CUtensorMap*>(tAr), *reinterpret_cast<const CUtensorMap*>(tAi),
        *reinterpret_cast<const CUtensorMap*>(tBr), *reinterpret_cast<const CUtensorMap*>(tBi), Cr, Ci, C64, ldc,
        zstride, m, n, kext, S, alpha, beta, d_err);
    return cudaGetLastError();
}

// C = beta C + alpha sum_z P[z]  (P: S slices of m x n column-major, leading dimension m)
__global__ void splitk_reduce_c32_kernel(const float* __restrict__ Pr, const float* __restrict__ Pi, int S, int m,
                                         int n, float alpha, float beta, float* __restrict__ Cr,
                                         float* __restrict__ Ci, long ldc) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long zs = (long)m * n;
    if (idx >= zs) return;
    const int j = (int)(idx / m), i = (int)(idx % m);
    float r = 0.f, im = 0.f;
    for (int z = 0; z < S; ++z) {
        r += __ldg(Pr + idx + z * zs);
        im += __ldg(Pi + idx + z * zs);
    }
    const long o = i + (long)j * ldc;
    float cr = alpha * r, ci = alpha * im;
    if (beta != 0.f) {
        cr = fmaf(beta, Cr[o], cr);
        ci = fmaf(beta, Ci[o], ci);
    }
    Cr[o] = cr;
    Ci[o] = ci;
}

// C64 = beta C64 + alpha sum_z P[z], the slice sum in FP32 (it is an FP32 product)
__global__ void splitk_reduce_z64_kernel(const float* __restrict__ Pr, const float* __restrict__ Pi, int S, int m,
                                         int n, float alpha, float beta, double2* __restrict__ C, long ldc) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long zs = (long)m * n;
    if (idx >= zs) return;
    const int j = (int)(idx / m), i = (int)(idx % m);
    float r = 0.f, im = 0.f;
    for (int z = 0; z < S; ++z) {
        r += __ldg(Pr + idx + z * zs);
        im += __ldg(Pi + idx + z * zs);
    }
    double2& c = C[i + (long)j * ldc];
    double cr = (double)alpha * (double)r, ci = (double)alpha * (double)im;
    if (beta != 0.f) {
        cr = fma((double)beta, c.x, cr);
        ci = fma((double)beta, c.y, ci);
    }
    c = make_double2(cr, ci);
}

// B operand of a skinny product: V (K x nrhs FP32 planar, column-major) -> row c of a [nrhs][ldk]
// K-major pack; 3xTF32 segments [hi | lo | hi] with hi = tf32(v), lo = v - hi.
__global__ void pack_b_kernel(const float* __restrict__ Vr, const float* __restrict__ Vi, long ldv, int K, int nrhs,
                              int split, float* __restrict__ Br, float* __restrict__ Bi, long ldk) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)K * nrhs) return;
    const int c = (int)(idx / K), k = (int)(idx % K);
    const float vr = __ldg(Vr + k + (long)c * ldv), vi = __ldg(Vi + k + (long)c * ldv);
    const long o = (long)c * ldk + k;
    if (!split) {
        Br[o] = vr;
        Bi[o] = vi;
        return;
    }
    uint32_t hr, hi;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hr) : "f"(vr));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(vi));
    const float fr = __uint_as_float(hr), fi = __uint_as_float(hi);
    Br[o] = fr;
    Bi[o] = fi;
    Br[o + K] = vr - fr;
    Bi[o + K] = vi - fi;
    Br[o + 2L * K] = fr;
    Bi[o + 2L * K] = fi;
}

}  // namespace

// C = beta C + alpha A B^T, C FP32 planar column-major (m x n, ld ldc); one K range per CTA.
cudaError_t gemm_tc(cudaStream_t s, const void* tAr, const void* tAi, const void* tBr, const void* tBi, float* Cr,
                    float* Ci, long ldc, int m, int n, int kext, float alpha, float beta, int* d_err) {
    if (m <= 0 || n <= 0 || kext <= 0) return cudaSuccess;
    dim3 grid(ceil_div(m, BM), ceil_div(n, BN), 1);
    if (beta != 0.f)
        return launch_tc<OUT_C32_PRE>(s, grid, tAr, tAi, tBr, tBi, Cr, Ci, nullptr, ldc, 0, m, n, kext, 1, alpha,
                                      beta, d_err);
    return launch_tc<OUT_C32>(s, grid, tAr, tAi, tBr, tBi, Cr, Ci, nullptr, ldc, 0, m, n, kext, 1, alpha, beta,
                              d_err);
}

// Number of K splits for a product with few output tiles: about three waves of CTAs over the
// SMs (one CTA per SM fits), at most 32 splits and at least one 32-wide K step per split.
int tc_split_k(int m, int n, int kext, int num_sms) {
    const long tiles = (long)ceil_div(m, BM) * ceil_div(n, BN);
    const int nkb = ceil_div(kext, BKE);
    long S = (3L * num_sms) / tiles;
    if (S > 32) S = 32;
    if (S > nkb) S = nkb;
    if (S < 1) S = 1;
    return (int)S;
}

// Split-K product into an FP32 planar (dst.re, dst.im) or FP64 (dst.z) destination:
// dst = beta dst + alpha A B^T.  With S > 1 splits, each writes its partial product to the
// workspace (Pr, Pi: S m n floats each) and one reduction kernel sums the slices in a fixed order
// (deterministic).  Returns the number of kernels launched in *launched.
cudaError_t gemm_tc_split(cudaStream_t s, const void* tAr, const void* tAi, const void* tBr, const void* tBi, int m,
                          int n, int kext, float alpha, float beta, TcDest dst, int S, float* Pr, float* Pi,
                          int* d_err, int* launched) {
    *launched = 0;
    if (m <= 0 || n <= 0 || kext <= 0) return cudaSuccess;
    const bool z64 = dst.z != nullptr;
    if (S <= 1) {
        dim3 grid(ceil_div(m, BM), ceil_div(n, BN), 1);
        *launched = 1;
        if (z64)
            return launch_tc<OUT_Z64>(s, grid, tAr, tAi, tBr, tBi, nullptr, nullptr, dst.z, dst.ld, 0, m, n, kext, 1,
                                      alpha, beta, d_err);
        return launch_tc<OUT_C32>(s, grid, tAr, tAi, tBr, tBi, dst.re, dst.im, nullptr, dst.ld, 0, m, n, kext, 1,
                                  alpha, beta, d_err);
    }
    dim3 grid(ceil_div(m, BM), ceil_div(n, BN), S);
    const long zs = (long)m * n;
    cudaError_t e = launch_tc<OUT_PART>(s, grid, tAr, tAi, tBr, tBi, Pr, Pi, nullptr, m, zs, m, n, kext, S, 1.f, 0.f,
                                        d_err);
    if (e != cudaSuccess) return e;
    const int nb = (int)ceil_div(zs, 256L);
    if (z64)
        splitk_reduce_z64_kernel<<<nb, 256, 0, s>>>(Pr, Pi, S, m, n, alpha, beta, dst.z, dst.ld);
    else
        splitk_reduce_c32_kernel<<<nb, 256, 0, s>>>(Pr, Pi, S, m, n, alpha, beta, dst.re, dst.im, dst.ld);
    *launched = 2;
    return cudaGetLastError();
}

cudaError_t launch_pack_b(cudaStream_t s, const float* Vr, const float* Vi, long ldv, int K, int nrhs, int split,
                          float* Br, float* Bi, long ldk) {
    const long t = (long)K * nrhs;
    if (t == 0) return cudaSuccess;
    pack_b_kernel<<<ceil_div(t, 256L), 256, 0, s>>>(Vr, Vi, ldv, K, nrhs, split, Br, Bi, ldk);
    return cudaGetLastError();
}

// Batched Schur-type product: for each of B entries (maps: 4 opaque 128-byte tensor maps, outputs)
// C = alpha A B^T (beta = 0), one launch with grid.z = B.  d_entries: device scratch of
// B * tc_batch_entry_bytes() bytes, filled here.
size_t tc_batch_entry_bytes() { return sizeof(TcBatchEntry); }
cudaError_t gemm_tc_batch(cudaStream_t s, int B, const void* const* maps, float* const* Cr, float* const* Ci,
                          const long* ldc, int m, int n, int kext, float alpha, void* d_entries, int* d_err) {
    if (B < 1 || m <= 0 || n <= 0 || kext <= 0) return cudaSuccess;
    static DeviceFlags attr;
    if (attr.pending()) {
        cudaError_t e = cudaFuncSetAttribute(cgemm_tc_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr.done();
    }
    std::vector<TcBatchEntry> h(B);
    for (int b = 0; b < B; ++b) {
        for (int q = 0; q < 4; ++q)
            std::memcpy(&h[b].map[q], static_cast<const unsigned char*>(maps[b]) + 128 * q, sizeof(CUtensorMap));
        h[b].Cr = Cr[b];
        h[b].Ci = Ci[b];
        h[b].ldc = ldc[b];
    }
    cudaError_t e = cudaMemcpyAsync(d_entries, h.data(), sizeof(TcBatchEntry) * B, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(m, BM), ceil_div(n, BN), B);
    cgemm_tc_batch_kernel<<<grid, 128, SMEM_BYTES, s>>>(reinterpret_cast<const TcBatchEntry*>(d_entries), m, n, kext,
                                                        alpha, d_err);
    return cudaGetLastError();
}
