// Dense complex LU with partial pivoting on the GPU (the N x N Schur complement U33 of
// Theorem thm:LU, or the 2N x 2N ordinary matrix of Eq. dis_BM), and the triangular solves.
//
// Right-looking blocked LU with two block sizes:
//   for each big panel of NB columns (C32: 256, Z64: 64):
//     for each sub-panel of nbp columns:
//        panel kernel      : unblocked LU with partial pivoting of rows [j, n) x nbp columns on a
//                            cluster of up to 16 CTAs.  C32 panels of at most 4096 rows use the
//                            lane-per-column kernel (panel_c32.cu: nbp = 32, lane k of every warp
//                            holds column k of 4-16 rows, about 64-256 rows per CTA); taller C32
//                            panels and all Z64 panels use the register-row kernel
//                            (lu_internal.cuh: one to four rows per thread, nbp = 32/16/8 for C32,
//                            16/8/4 for Z64).  Each column's pivot candidates (value, index, whole
//                            row) go to every CTA through distributed shared memory; CTA 0 also
//                            builds the row-interchange maps.
//        swap_trsm_kernel  : row interchanges + unit-lower solve for the rest of the big panel
//        gemm (SIMT)       : rank-nbp update of the rest of the big panel
//     swap_trsm_kernel     : interchanges for all other columns, U12 = L11^{-1} A12 (and its
//                            K-major pack for the tensor cores)
//     trailing update      : A22 -= L21 U12  (tensor-core TF32 / 3xTF32 for C32, SIMT for Z64)
// Pivot = first row index of max |Re| + |Im| (the LAPACK izamax rule).  An exactly zero pivot
// records the 1-based column in *info and skips the scaling, as LAPACK getrf does.
//
// Solves (getrs): Y = P B, then block forward substitution with the unit L and block back
// substitution with U; the bs x bs diagonal blocks are inverted once after the factorisation so
// that every step is a small matrix product.  For C32 the off-diagonal bs x bs tiles of each
// block column are then multiplied by that column's inverted diagonal block (the "G form"), so
// that a step is one product with no dependence on the inverse:
//   forward:  Y[below b] -= (L[below b, b] L_bb^{-1}) Y_b,  then Z_b = L_bb^{-1} Y_b for all b at once
//   backward: Z[above b] -= (U[above b, b] U_bb^{-1}) Z_b,  then X_b = U_bb^{-1} Z_b for all b at once
// (the same sums as L_bb^{-1} Y_b formed inside every step, without recomputing it in each CTA).
#include "lu_internal.cuh"

#include <map>
#include <mutex>

using namespace lu_detail;

namespace {

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Row interchanges (from a swap map) for columns in [a0, a1) u [b0, b1); for columns of the
// second range also X = L11^{-1} X on rows [t0, t0+tb) with the unit-lower L11 at (t0, t0),
// staged in shared memory: whole when it fits, else in chunks of ST_KC columns that the CTA's
// warps step through together.  Optionally writes the solved rows as a K-major tensor-core pack
// (column c -> row c - b0).  One warp per column.
// Asynchronous 4-byte global -> shared copies (cp.async, zero-filled when !full).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool full) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(full ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Strictly lower part of columns [k0, k0 + kc) of the tb x tb block at (t0, t0) of a planar FP32
// matrix into dst (interleaved complex, leading dimension tb), by cp.async (nthreads threads).
__device__ __forceinline__ void stage_lower_async(float2* dst, const C32& A, long t0, int tb, int k0, int kc,
                                                  int nthreads) {
    const int tot = tb * kc;
    for (int e = threadIdx.x; e < tot; e += nthreads) {
        const int i = e % tb, kk = e / tb;
        const bool in = i > k0 + kk;
        const long off = in ? (t0 + i) + (t0 + k0 + kk) * A.ld : 0;
        cp_async4(&dst[e].x, A.re + off, in);
        cp_async4(&dst[e].y, A.im + off, in);
    }
}

constexpr int ST_WARPS = 16, ST_COLS = 1;
constexpr int ST_KC = 32;  // L11 columns per shared-memory chunk when L11 does not fit whole
template <class V>
__global__ void __launch_bounds__(ST_WARPS * 32) swap_trsm_kernel(V A, const SwapMap* __restrict__ map, int a0, int a1,
                                                                   int b0, int b1, int t0, int tb, float* Upr,
                                                                   float* Upi, long ldk, int split, int l_in_smem) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    constexpr int QMAX = 8;  // rows per lane: tb <= 256
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    CV* Ls = reinterpret_cast<CV*>(smraw);  // tb x tb, column-major
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int na = a1 - a0, nbc = b1 - b0;
    const int ncols = na + nbc;
    const int cta_col0 = blockIdx.x * ST_WARPS * ST_COLS;
    const bool cta_has_b = (cta_col0 + ST_WARPS * ST_COLS > na) && tb > 0;
    // strictly lower part of L11 columns [k0, k0 + kc) into Ls (leading dimension tb), SB loads in
    // flight per thread at a time
    auto stage = [&](int k0, int kc) {
        constexpr int SB = 8;
        const int tot = tb * kc;
        for (int e0 = 0; e0 < tot; e0 += SB * ST_WARPS * 32) {
            CV v[SB];
#pragma unroll
            for (int m = 0; m < SB; ++m) {
                const int e = e0 + threadIdx.x + m * ST_WARPS * 32;
                const int i = e % tb, kk = e / tb;
                v[m] = (e < tot && i > k0 + kk) ? A.get((long)t0 + i, (long)t0 + k0 + kk) : czero<Rl>();
            }
#pragma unroll
            for (int m = 0; m < SB; ++m) {
                const int e = e0 + threadIdx.x + m * ST_WARPS * 32;
                if (e < tot) Ls[e] = v[m];
            }
        }
    };
    if (cta_has_b && l_in_smem == 1) {
        if constexpr (std::is_same<V, C32>::value) {
            stage_lower_async(Ls, A, t0, tb, 0, tb, ST_WARPS * 32);
            cp_async_commit();
            cp_async_wait<0>();
        } else {
            stage(0, tb);
        }
        __syncthreads();
    }
    static_assert(ST_COLS == 1, "one column per warp");
    const int cnt = map ? map->count : 0;
    const int gw = cta_col0 + warp;
    const bool valid = gw < ncols;
    const bool in_b = valid && gw >= na;
    const long col = in_b ? (long)b0 + (gw - na) : (long)a0 + gw;
    if (valid && cnt > 0) {
        CV v[MAP_MAX / 32];
#pragma unroll
        for (int q = 0; q < MAP_MAX / 32; ++q) {
            int t = lane + 32 * q;
            if (t < cnt) v[q] = A.get(map->src[t], col);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < MAP_MAX / 32; ++q) {
            int t = lane + 32 * q;
            if (t < cnt) A.set(map->dst[t], col, v[q]);
        }
        __syncwarp();
    }
    const bool do_trsm = in_b && tb > 0;
    CV x[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
        int i = lane + 32 * q;
        x[q] = (do_trsm && i < tb) ? A.get((long)t0 + i, col) : czero<Rl>();
    }
    // x -= L11 columns k in [kb, ke), all in one group of 32 (k = 32 QK + l); lk(i, k) reads
    // L(t0 + i, t0 + k) from wherever it is staged.  With the group a compile-time constant, the
    // value x_k comes straight from register x[QK] of lane l, and only rows of groups >= QK are
    // touched, without per-row predicates beyond the diagonal group.
    auto steps_q = [&](auto qc, int kb, int ke, auto lk) {
        constexpr int QK = decltype(qc)::value;
        for (int k = kb; k < ke; ++k) {
            const int l = k & 31;
            CV nx;
            nx.x = -__shfl_sync(0xffffffffu, x[QK].x, l);
            nx.y = -__shfl_sync(0xffffffffu, x[QK].y, l);
            if (lane > l && lane + 32 * QK < tb) cfma(x[QK], lk(lane + 32 * QK, k), nx);
#pragma unroll
            for (int q = QK + 1; q < QMAX; ++q) {
                if (32 * q >= tb) break;  // warp-uniform: groups past tb issue nothing
                const int i = lane + 32 * q;
                if (i < tb) cfma(x[q], lk(i, k), nx);
            }
        }
    };
    auto steps = [&](int kb, int ke, auto lk) {
        for (int g0 = kb; g0 < ke;) {
            const int g1 = min(ke, (g0 & ~31) + 32);
            switch (g0 >> 5) {
                case 0: steps_q(std::integral_constant<int, 0>{}, g0, g1, lk); break;
                case 1: steps_q(std::integral_constant<int, 1>{}, g0, g1, lk); break;
                case 2: steps_q(std::integral_constant<int, 2>{}, g0, g1, lk); break;
                case 3: steps_q(std::integral_constant<int, 3>{}, g0, g1, lk); break;
                case 4: steps_q(std::integral_constant<int, 4>{}, g0, g1, lk); break;
                case 5: steps_q(std::integral_constant<int, 5>{}, g0, g1, lk); break;
                case 6: steps_q(std::integral_constant<int, 6>{}, g0, g1, lk); break;
                default: steps_q(std::integral_constant<int, 7>{}, g0, g1, lk); break;
            }
            g0 = g1;
        }
    };
    static_assert(QMAX == 8, "one case per group of 32 rows");
    if (l_in_smem == 2) {
        // L11 larger than the shared-memory budget: stage it ST_KC columns at a time, the whole
        // CTA stepping through the chunks together (warps without a column to solve only help)
        if constexpr (!std::is_same<V, C32>::value) {  // FP64: L11 (NB <= 64) always fits whole
            if (cta_has_b)
                for (int k0 = 0; k0 < tb; k0 += ST_KC) {
                    const int kc = min(ST_KC, tb - k0);
                    __syncthreads();
                    stage(k0, kc);
                    __syncthreads();
                    if (do_trsm) steps(k0, k0 + kc, [&](int i, int kk) { return Ls[i + (kk - k0) * tb]; });
                }
        } else if (cta_has_b) {
            // two buffers of ST_KC / 2 columns: the next chunk's cp.async copies run while the
            // warps step through the current one
            constexpr int KC = ST_KC / 2;
            CV* const buf1 = Ls + tb * KC;
            stage_lower_async(Ls, A, t0, tb, 0, min(KC, tb), ST_WARPS * 32);
            cp_async_commit();
            for (int k0 = 0, c = 0; k0 < tb; k0 += KC, ++c) {
                const int kc = min(KC, tb - k0);
                if (k0 + KC < tb) {
                    stage_lower_async((c & 1) ? Ls : buf1, A, t0, tb, k0 + KC, min(KC, tb - k0 - KC), ST_WARPS * 32);
                    cp_async_commit();
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();  // chunk c is in shared memory for every warp
                const CV* cur = (c & 1) ? buf1 : Ls;
                if (do_trsm) steps(k0, k0 + kc, [&](int i, int kk) { return cur[i + (kk - k0) * tb]; });
                __syncthreads();  // every warp is done with chunk c before its buffer is refilled
            }
        }
    } else if (do_trsm) {
        if (l_in_smem)
            steps(0, tb, [&](int i, int kk) { return Ls[i + kk * tb]; });
        else
            steps(0, tb, [&](int i, int kk) { return A.get((long)t0 + i, (long)t0 + kk); });
    }
    if (do_trsm) {
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            int i = lane + 32 * q;
            if (i < tb) A.set((long)t0 + i, col, x[q]);
        }
        if (Upr != nullptr) {
            // K-major pack of this column (row index = col - b0); segments [hi | lo | hi] when split
            long rowp = col - b0;
            float* pr = Upr + rowp * ldk;
            float* pi = Upi + rowp * ldk;
#pragma unroll
            for (int q = 0; q < QMAX; ++q) {
                int i = lane + 32 * q;
                if (i < tb) {
                    float vr = (float)x[q].x, vi = (float)x[q].y;
                    if (!split) {
                        pr[i] = vr;
                        pi[i] = vi;
                    } else {
                        float hr = tf32_rna(vr), hi = tf32_rna(vi);
                        pr[i] = hr;
                        pi[i] = hi;
                        pr[tb + i] = vr - hr;
                        pi[tb + i] = vi - hi;
                        pr[2 * tb + i] = hr;
                        pi[2 * tb + i] = hi;
                    }
                }
            }
            long kext = split ? 3L * tb : (long)tb;
            long kpad = (kext + 31) / 32 * 32;
            for (long i = kext + lane; i < kpad; i += 32) {
                pr[i] = 0.f;
                pi[i] = 0.f;
            }
        }
    }
}

// L21 pack: rows [r0, r0+m) x columns [c0, c0+kb) of A -> row-major [m][ldk] planar, segments
// [hi | hi | lo] when split (K padded with zeros to a multiple of 32).
__global__ void pack_L_kernel(C32 A, long r0, long c0, int m, int kb, int split, float* Pr, float* Pi, long ldk) {
    __shared__ float2 t[32][33];
    int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int q = ty; q < 32; q += 8) {
        int i = i0 + tx, k = k0 + q;
        t[q][tx] = (i < m && k < kb) ? A.get(r0 + i, c0 + k) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    long kext = split ? 3L * kb : (long)kb;
    long kpad = (kext + 31) / 32 * 32;
    for (int q = ty; q < 32; q += 8) {
        int i = i0 + q, k = k0 + tx;
        if (i >= m) continue;
        float* pr = Pr + (long)i * ldk;
        float* pi = Pi + (long)i * ldk;
        if (k < kb) {
            float2 v = t[tx][q];
            if (!split) {
                pr[k] = v.x;
                pi[k] = v.y;
            } else {
                float hr = tf32_rna(v.x), hi = tf32_rna(v.y);
                pr[k] = hr;
                pi[k] = hi;
                pr[kb + k] = hr;
                pi[kb + k] = hi;
                pr[2 * kb + k] = v.x - hr;
                pi[2 * kb + k] = v.y - hi;
            }
        }
        if (blockIdx.x == 0)
            for (long kk = kext + tx; kk < kpad; kk += 32) {
                pr[kk] = 0.f;
                pi[kk] = 0.f;
            }
    }
}

__global__ void iota_kernel(int* p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// A ROWS x COLS tile of view A at (r0, c0) into shared memory (column-major, leading dimension
// ROWS), zero outside nr x nc.  Each thread issues all its global loads before its first shared
// store, so one memory latency covers the whole tile (256 threads).
template <int ROWS, int COLS, class V>
__device__ __forceinline__ void load_tile(typename V::cv* dst, const V& A, long r0, long c0, int nr, int nc) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    static_assert(ROWS * COLS % 256 == 0, "tile must split evenly over 256 threads");
    constexpr int PER = ROWS * COLS / 256;
    CV v[PER];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int i = e % ROWS, j = e / ROWS;
        v[m] = (i < nr && j < nc) ? A.get(r0 + i, c0 + j) : czero<Rl>();
    }
#pragma unroll
    for (int m = 0; m < PER; ++m) dst[threadIdx.x + 256 * m] = v[m];
}

// The same for a dense column-major B x B block (leading dimension B), zero outside n x n.
template <int B, class CV>
__device__ __forceinline__ void load_block(CV* dst, const CV* __restrict__ src, int nb) {
    static_assert(B * B % 256 == 0, "block must split evenly over 256 threads");
    constexpr int PER = B * B / 256;
    CV v[PER];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int e = threadIdx.x + 256 * m;
        const int i = e % B, j = e / B;
        v[m] = (i < nb && j < nb) ? src[e] : CV{};
    }
#pragma unroll
    for (int m = 0; m < PER; ++m) dst[threadIdx.x + 256 * m] = v[m];
}

// Inverse of each 64 x 64 diagonal block (unit lower L or upper U) of the LU factor, by a
// column sweep over X = I: for k in order (L: 0..rb-1; U: rb-1..0, row k first divided by U_kk),
// every later row i takes X_i -= T_ik X_k.  Thread t holds X[t % 64, t / 64 + 4 m] (m < 16) in
// registers; row k goes through a double-buffered shared row, so each step needs one barrier
// (the reciprocals 1 / U_kk are formed before the sweep).
// Entries outside the rb x rb leading block are zero.
constexpr int TI_B = 64;
template <class V, bool UPPER, int CG>
__global__ void __launch_bounds__(256) tri_inv_kernel(V F, int n, typename V::cv* __restrict__ out) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    // CG column groups (blockIdx.y): the columns of the inverse are independent, so the FP64
    // factors, whose pipe is slow on each SM, spread one block over CG CTAs
    constexpr int B = TI_B, M = B * B / 256 / CG;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* T = reinterpret_cast<CV*>(sm);  // [B][B] column-major
    CV* buf = T + B * B;                // [2][B]
    CV* dg = buf + 2 * B;               // [B] 1 / U_kk
    const int t = threadIdx.x, i = t % B, c0 = t / B;
    const int mg = (int)blockIdx.y * M;  // this CTA's columns: c0 + 4 (mg + m), m < M
    const long r0 = (long)blockIdx.x * B;
    const int rb = (int)min((long)B, n - r0);
    load_tile<B, B>(T, F, r0, r0, rb, rb);
    if (UPPER && t < rb) dg[t] = cinv(F.get(r0 + t, r0 + t));
    CV x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        x[m] = czero<Rl>();
        if (i == c0 + 4 * (mg + m) && i < rb) x[m].x = (Rl)1;
    }
    __syncthreads();
    for (int s = 0; s < rb; ++s) {
        const int k = UPPER ? rb - 1 - s : s;
        CV* bk = buf + (s & 1) * B;
        if (i == k) {
            if (UPPER) {
                const CV d = dg[k];
#pragma unroll
                for (int m = 0; m < M; ++m) x[m] = cmul(x[m], d);
            }
#pragma unroll
            for (int m = 0; m < M; ++m) bk[c0 + 4 * (mg + m)] = x[m];
        }
        __syncthreads();
        if (UPPER ? i < k : (i > k && i < rb)) {
            CV tik = T[i + k * B];
            tik.x = -tik.x;
            tik.y = -tik.y;
#pragma unroll
            for (int m = 0; m < M; ++m) cfma(x[m], tik, bk[c0 + 4 * (mg + m)]);
        }
    }
    CV* o = out + (long)blockIdx.x * B * B;
#pragma unroll
    for (int m = 0; m < M; ++m) o[i + (c0 + 4 * (mg + m)) * B] = x[m];
}

// One block step of a blocked triangular solve with inverted diagonal blocks (one launch per
// block, all right-hand sides):
//   Zb = Tinv Y[r0:r0+rb, :]                          (written to Z by the CTAs of row tile 0)
//   Y[rest0:rest0+nrest, :] -= F[rest0.., r0:r0+rb] Zb (each CTA one 64-row tile of the rest)
// Forward (unit L) and backward (U) passes use the same kernel with the rows below or above the
// block as the rest; Z is a second buffer, so no CTA reads a block that another one rewrites.
constexpr int TS_BM = 64;
template <class V, int BN>
__global__ void __launch_bounds__(256) trsv_step_kernel(V F, V Y, V Z, int r0, int rb, int rest0, int nrest, int nrhs,
                                                        int bs, const typename V::cv* __restrict__ Tinv) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* Ts = reinterpret_cast<CV*>(sm);  // [bs][bs] column-major
    CV* Yb = Ts + bs * bs;               // [BN][bs]
    CV* Zb = Yb + BN * bs;               // [BN][bs]
    CV* Ft = Zb + BN * bs;               // [bs][TS_BM] column-major tile of F
    const int t = threadIdx.x;
    const int j0 = blockIdx.y * BN;
    const int nc = min(BN, nrhs - j0);
    for (int e = t; e < bs * bs; e += 256) Ts[e] = Tinv[e];
    for (int e = t; e < bs * BN; e += 256) {
        int i = e % bs, jj = e / bs;
        Yb[jj * bs + i] = (i < rb && jj < nc) ? Y.get((long)r0 + i, (long)j0 + jj) : czero<Rl>();
    }
    const long tr0 = (long)rest0 + (long)blockIdx.x * TS_BM;
    const int tm = (int)min((long)TS_BM, (long)rest0 + nrest - tr0);
    if (nrest > 0)
        for (int e = t; e < TS_BM * bs; e += 256) {
            int i = e % TS_BM, k = e / TS_BM;
            Ft[k * TS_BM + i] = (i < tm && k < rb) ? F.get(tr0 + i, (long)r0 + k) : czero<Rl>();
        }
    __syncthreads();
    // register micro-tiles: thread (tx, ty) owns rows tx + 16a (a < bs/16) and columns ty + 16b
    constexpr int TN = BN / 16;
    const int tx = t % 16, ty = t / 16;
    const int TMb = bs / 16;  // bs is 64: 4 rows per thread
    {
        CV acc[4][TN];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) acc[a][b] = czero<Rl>();
        // threads whose columns all lie past the last right-hand side skip the products (with one
        // right-hand side, 15 of 16 column slots: the FP64 pipe is the bound of these small steps)
        const int kend = (ty < nc) ? rb : 0;
        for (int k = 0; k < kend; ++k) {
            CV tv[4], yv[TN];
#pragma unroll
            for (int a = 0; a < 4; ++a) tv[a] = (a < TMb) ? Ts[tx + 16 * a + k * bs] : czero<Rl>();
#pragma unroll
            for (int b = 0; b < TN; ++b) yv[b] = Yb[(ty + 16 * b) * bs + k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) cfma(acc[a][b], tv[a], yv[b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b)
                if (a < TMb) Zb[(ty + 16 * b) * bs + tx + 16 * a] = acc[a][b];
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int e = t; e < bs * BN; e += 256) {
            int i = e % bs, jj = e / bs;
            if (i < rb && jj < nc) Z.set((long)r0 + i, (long)j0 + jj, Zb[jj * bs + i]);
        }
    if (nrest <= 0) return;
    CV acc[4][TN];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = czero<Rl>();
    const int kend2 = (ty < nc) ? rb : 0;
    for (int k = 0; k < kend2; ++k) {
        CV fv[4], zv[TN];
#pragma unroll
        for (int a = 0; a < 4; ++a) fv[a] = Ft[k * TS_BM + tx + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) zv[b] = Zb[(ty + 16 * b) * bs + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) cfma(acc[a][b], fv[a], zv[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = tx + 16 * a;
        if (i >= tm) continue;
#pragma unroll
        for (int b = 0; b < TN; ++b) {
            const int jj = ty + 16 * b;
            if (jj >= nc) continue;
            CV y = Y.get(tr0 + i, (long)j0 + jj);
            y.x -= acc[a][b].x;
            y.y -= acc[a][b].y;
            Y.set(tr0 + i, (long)j0 + jj, y);
        }
    }
}

// G form of the factors (C32): every off-diagonal bs x bs tile F[it, b] (it != b) becomes
// F[it, b] T_b with T_b = L_bb^{-1} below the diagonal and U_bb^{-1} above it.  One CTA per tile,
// in place (each CTA reads its whole tile before writing it).  bs == TS_BM == 64.
template <class V>
__global__ void __launch_bounds__(256) g_form_kernel(V F, int n, const typename V::cv* __restrict__ dinvL,
                                                     const typename V::cv* __restrict__ dinvU) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    constexpr int B = TS_BM;
    const int it = blockIdx.x, b = blockIdx.y;
    if (it == b) return;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* Ft = reinterpret_cast<CV*>(sm);  // [B][B] column-major tile of F
    CV* Ts = Ft + B * B;                 // [B][B] column-major T_b
    const int t = threadIdx.x;
    const long r0 = (long)it * B, c0 = (long)b * B;
    const int tm = (int)min((long)B, n - r0), rb = (int)min((long)B, n - c0);
    const CV* T = (it > b ? dinvL : dinvU) + (long)b * B * B;
    load_tile<B, B>(Ft, F, r0, c0, tm, rb);
    load_block<B>(Ts, T, rb);
    __syncthreads();
    const int tx = t % 16, ty = t / 16;  // rows tx + 16 a, columns ty + 16 c
    CV acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = czero<Rl>();
    for (int k = 0; k < rb; ++k) {
        CV fv[4], tv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) fv[a] = Ft[k * B + tx + 16 * a];
#pragma unroll
        for (int c = 0; c < 4; ++c) tv[c] = Ts[k + (ty + 16 * c) * B];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) cfma(acc[a][c], fv[a], tv[c]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = tx + 16 * a;
        if (i >= tm) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = ty + 16 * c;
            if (j < rb) F.set(r0 + i, c0 + j, acc[a][c]);
        }
    }
}

// One step of a blocked triangular solve in G form (all right-hand sides):
//   Y[rest0:rest0+nrest, :] -= G[rest0.., r0:r0+rb] Y[r0:r0+rb, :]
// (each CTA one 64-row tile of the rest and BN columns; the rows it reads and writes are disjoint).
template <class V, int BN>
__global__ void __launch_bounds__(256) trsv_g_step_kernel(V F, V Y, int r0, int rb, int rest0, int nrest, int nrhs) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    constexpr int B = TS_BM;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* Yb = reinterpret_cast<CV*>(sm);  // [BN][B]
    CV* Ft = Yb + BN * B;                // [B][B] column-major tile of G
    const int t = threadIdx.x;
    const int j0 = blockIdx.y * BN;
    const int nc = min(BN, nrhs - j0);
    const long tr0 = (long)rest0 + (long)blockIdx.x * B;
    const int tm = (int)min((long)B, (long)rest0 + nrest - tr0);
    load_tile<B, B>(Ft, F, tr0, r0, tm, rb);
    pdl_wait();
    pdl_trigger();
    load_tile<B, BN>(Yb, Y, r0, j0, rb, nc);
    __syncthreads();
    constexpr int TN = BN / 16;
    const int tx = t % 16, ty = t / 16;
    CV acc[4][TN];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[a][c] = czero<Rl>();
    // threads whose columns all lie past the last right-hand side (the ragged column tile, e.g.
    // 65 = 4 x 16 + 1) skip the product, so their warps leave the SM early
    const int kend = (ty < nc) ? rb : 0;
    for (int k = 0; k < kend; ++k) {
        CV fv[4], yv[TN];
#pragma unroll
        for (int a = 0; a < 4; ++a) fv[a] = Ft[k * B + tx + 16 * a];
#pragma unroll
        for (int c = 0; c < TN; ++c) yv[c] = Yb[(ty + 16 * c) * B + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < TN; ++c) cfma(acc[a][c], fv[a], yv[c]);
    }
    // read all of this thread's outputs before writing any (the reads do not wait on the writes)
    CV yo[4][TN];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int i = tx + 16 * a, jj = ty + 16 * c;
            yo[a][c] = (i < tm && jj < nc) ? Y.get(tr0 + i, (long)j0 + jj) : czero<Rl>();
        }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int i = tx + 16 * a, jj = ty + 16 * c;
            if (i < tm && jj < nc) {
                CV y = yo[a][c];
                y.x -= acc[a][c].x;
                y.y -= acc[a][c].y;
                Y.set(tr0 + i, (long)j0 + jj, y);
            }
        }
}

// Z_b = T_b Y_b for every diagonal block b at once (grid: blocks x column tiles of BN).
template <class V, int BN>
__global__ void __launch_bounds__(256) trsv_diag_kernel(V Y, V Z, int n, int nrhs,
                                                        const typename V::cv* __restrict__ Tinv) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    constexpr int B = TS_BM;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* Ts = reinterpret_cast<CV*>(sm);  // [B][B] column-major
    CV* Yb = Ts + B * B;                 // [BN][B]
    const int t = threadIdx.x;
    const long r0 = (long)blockIdx.x * B;
    const int rb = (int)min((long)B, n - r0);
    const int j0 = blockIdx.y * BN;
    const int nc = min(BN, nrhs - j0);
    load_block<B>(Ts, Tinv + (long)blockIdx.x * B * B, rb);
    pdl_wait();
    pdl_trigger();
    load_tile<B, BN>(Yb, Y, r0, j0, rb, nc);
    __syncthreads();
    constexpr int TN = BN / 16;
    const int tx = t % 16, ty = t / 16;
    CV acc[4][TN];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[a][c] = czero<Rl>();
    for (int k = 0; k < rb; ++k) {
        CV tv[4], yv[TN];
#pragma unroll
        for (int a = 0; a < 4; ++a) tv[a] = Ts[tx + 16 * a + k * B];
#pragma unroll
        for (int c = 0; c < TN; ++c) yv[c] = Yb[(ty + 16 * c) * B + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < TN; ++c) cfma(acc[a][c], tv[a], yv[c]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = tx + 16 * a;
        if (i >= rb) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int jj = ty + 16 * c;
            if (jj < nc) Z.set(r0 + i, (long)j0 + jj, acc[a][c]);
        }
    }
}

// Persistent blocked triangular solve in G form (C32): the block steps and the diagonal blocks of
// one triangle (forward: lower, backward: upper) in a single cooperative launch.  Work item (i, j)
// is tile row i (64 rows) of column tile j (16 right-hand sides).  It accumulates
// sum_b G[i, b] Y[b, j] over the tile rows b before i (lower) or after i (upper), each as soon as
// item (b, j) has published its final rows through the flag ready[b, j]; then it writes
// Y[i, j] -= that sum (the rows later items read), publishes ready[i, j], and writes
// Z[i, j] = T_i Y[i, j] with T_i the inverted diagonal block.  CTA q takes items q, q + grid, ...
// in dependency order, so the earliest unfinished item never waits; with every CTA resident
// (cooperative launch) no wait can deadlock.  Waits are bounded (1 s by the global timer): a
// timeout raises *err and the item goes on with what it has.
constexpr int FL_BN = 8;
__device__ __forceinline__ void flow_wait(const int* flag, int* err) {
    if (*reinterpret_cast<volatile int*>(err) != 0) return;  // an earlier wait gave up: no more waiting
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0) return;
        if (it == 0) t0 = gtime();
        else if (gtime() - t0 > 1000000000ull) {
            atomicExch(err, 1);
            return;
        }
    }
}
// acc[c] += sum_k M[r, k] V[k, c] for k < kn: M column-major B x B, V row-major [k][BN]
__device__ __forceinline__ void flow_mac(float2 (&acc)[FL_BN], const float2* M, const float2* V, int r, int kn) {
    for (int k = 0; k < kn; ++k) {
        const float2 g = M[k * TS_BM + r];
        const float4* v4 = reinterpret_cast<const float4*>(V + k * FL_BN);
#pragma unroll
        for (int c2 = 0; c2 < FL_BN / 2; ++c2) {
            const float4 y = v4[c2];
            cfma(acc[2 * c2], g, make_float2(y.x, y.y));
            cfma(acc[2 * c2 + 1], g, make_float2(y.z, y.w));
        }
    }
}
template <bool UPPER>
__global__ void __launch_bounds__(256, 4) trsv_flow_kernel(C32 F, C32 Y, C32 Z, int n, int nrhs,
                                                           const float2* __restrict__ Tinv, int* ready, int* err,
                                                           const int* never, const int* hook) {
    constexpr int B = TS_BM, BN = FL_BN, RS = 256 / B;  // RS k-slices of the 64 rows
    extern __shared__ __align__(16) unsigned char sm[];
    float2* Gs = reinterpret_cast<float2*>(sm);     // [B][B] column-major: G[i, b], then T_i
    float2* Red = Gs;                               // [RS][B][BN] partial sums of the k-slices (over Gs)
    float2* Yb = Gs + B * B;                        // [B][BN] row-major: Y[b, j], then Y[i, j]
    float2* Yo = Yb + B * BN;                       // [B][BN] this item's own right-hand-side rows
    const int t = threadIdx.x;
    const int nblk = (n + B - 1) / B, ct = (nrhs + BN - 1) / BN;
    const int items = nblk * ct;
    const int r = t % B, ks = t / B;  // this thread: row r, k in [ks B / RS, (ks + 1) B / RS)
    const int kb0 = ks * (B / RS);
    pdl_wait();
    pdl_trigger();
    const bool hooked = never != nullptr && *hook != 0;  // test hook (set at assembly)
    for (int q = blockIdx.x; q < items; q += gridDim.x) {
        __syncthreads();  // the previous item is done with the shared buffers
        const int i = UPPER ? nblk - 1 - q / ct : q / ct, j = q % ct;
        const long r0 = (long)i * B;
        const int tm = (int)min((long)B, n - r0);
        const int j0 = j * BN, nc = min(BN, nrhs - j0);
        // this item's own right-hand-side rows (written only by it), fetched early
#pragma unroll
        for (int m = 0; m < B * BN / 256; ++m) {
            const int e = t + 256 * m;
            const int k = e / BN, c = e % BN;
            Yo[e] = (k < tm && c < nc) ? Y.get(r0 + k, (long)j0 + c) : make_float2(0.f, 0.f);
        }
        float2 acc[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) acc[c] = make_float2(0.f, 0.f);
        const int nsteps = UPPER ? nblk - 1 - i : i;
        for (int st = 0; st < nsteps; ++st) {
            const int b = UPPER ? nblk - 1 - st : st;
            const long c0 = (long)b * B;
            const int rb = (int)min((long)B, n - c0);
            __syncthreads();  // the buffers are free
            load_tile<B, B>(Gs, F, r0, c0, tm, rb);
            // (test hook: the last item's first wait is on a flag that nothing sets)
            const int* wf = (hooked && q == items - 1 && st == 0) ? never : ready + b * ct + j;
            if (t == 0) flow_wait(wf, err);
            __syncthreads();  // item (b, j) is final
#pragma unroll
            for (int m = 0; m < B * BN / 256; ++m) {
                const int e = t + 256 * m;
                const int k = e / BN, c = e % BN;
                float2 v = make_float2(0.f, 0.f);
                if (k < rb && c < nc) {
                    const long off = (c0 + k) + (long)(j0 + c) * Y.ld;
                    v = make_float2(__ldcg(Y.re + off), __ldcg(Y.im + off));
                }
                Yb[e] = v;
            }
            __syncthreads();
            flow_mac(acc, Gs + kb0 * B, Yb + kb0 * BN, r, min(B / RS, max(rb - kb0, 0)));
        }
        // combine the k-slices: the final rows of Y[i, j], published for the later items
        __syncthreads();  // Gs is free: Red lies over it
#pragma unroll
        for (int c = 0; c < BN; ++c) Red[(ks * B + r) * BN + c] = acc[c];
        __syncthreads();
        if (ks == 0) {
#pragma unroll
            for (int c = 0; c < BN; ++c) {
                float2 y = Yo[r * BN + c];
#pragma unroll
                for (int q2 = 0; q2 < RS; ++q2) {
                    const float2 p2 = Red[(q2 * B + r) * BN + c];
                    y.x -= p2.x;
                    y.y -= p2.y;
                }
                if (r < tm && c < nc) Y.set(r0 + r, (long)j0 + c, y);
                Yb[r * BN + c] = y;
            }
        }
        // the CTA barrier orders every thread's rows before thread 0's release (cumulative at gpu
        // scope), so a reader that acquires the flag sees them
        __syncthreads();
        if (t == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(ready + i * ct + j), "r"(1) : "memory");
        // Z[i, j] = T_i Y[i, j] (rows r, k-slice ks; the slices summed as above)
        load_block<B>(Gs, Tinv + (long)i * B * B, tm);
        __syncthreads();
        float2 z[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) z[c] = make_float2(0.f, 0.f);
        flow_mac(z, Gs + kb0 * B, Yb + kb0 * BN, r, min(B / RS, max(tm - kb0, 0)));
        __syncthreads();  // every slice has read Gs: Red may overwrite it
#pragma unroll
        for (int c = 0; c < BN; ++c) Red[(ks * B + r) * BN + c] = z[c];
        __syncthreads();
        if (ks == 0 && r < tm) {
#pragma unroll
            for (int c = 0; c < BN; ++c) {
                float2 sum = make_float2(0.f, 0.f);
#pragma unroll
                for (int q2 = 0; q2 < RS; ++q2) {
                    const float2 p2 = Red[(q2 * B + r) * BN + c];
                    sum.x += p2.x;
                    sum.y += p2.y;
                }
                if (c < nc) Z.set(r0 + r, (long)j0 + c, sum);
            }
        }
    }
}

__global__ void gather_rows_z64_kernel(const int* __restrict__ perm, int n, int nrhs, const double2* __restrict__ B,
                                       long ldb, double2* __restrict__ Y, long ldy) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)n * nrhs) return;
    int c = (int)(idx / n), i = (int)(idx % n);
    Y[i + (long)c * ldy] = B[perm[i] + (long)c * ldb];
}
__global__ void gather_rows_c32_kernel(const int* __restrict__ perm, int n, int nrhs, const float* __restrict__ Br,
                                       const float* __restrict__ Bi, long ldb, float* __restrict__ Yr,
                                       float* __restrict__ Yi, long ldy) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)n * nrhs) return;
    int c = (int)(idx / n), i = (int)(idx % n);
    Yr[i + (long)c * ldy] = Br[perm[i] + (long)c * ldb];
    Yi[i + (long)c * ldy] = Bi[perm[i] + (long)c * ldb];
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
#define LU_CUDA(expr)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            bm_set_error(std::string("lu: ") + #expr + ": " + cudaGetErrorString(_e));                 \
            return BM_ECUDA;                                                                           \
        }                                                                                              \
    } while (0)

template <class V>
cudaError_t launch_swap_trsm(cudaStream_t s, V A, const SwapMap* map, int a0, int a1, int b0, int b1, int t0, int tb,
                             float* Upr, float* Upi, long ldk, int split) {
    using CV = typename V::cv;
    long ncols = (long)(a1 - a0) + (b1 - b0);
    if (ncols <= 0) return cudaSuccess;
    // L11 staging: whole (1) when it fits 160 KB, else in ST_KC-column chunks (2)
    size_t lbytes = (size_t)tb * tb * sizeof(CV);
    int l_in_smem = tb <= 0 ? 0 : (lbytes <= 160 * 1024 ? 1 : 2);
    size_t smem = l_in_smem == 1 ? lbytes : (l_in_smem == 2 ? (size_t)tb * ST_KC * sizeof(CV) : 0);
    auto kern = swap_trsm_kernel<V>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int grid = ceil_div(ncols, ST_WARPS * ST_COLS);
    return launch_pdl(kern, dim3(grid), dim3(ST_WARPS * 32), smem, s, A, map, a0, a1, b0, b1, t0, tb, Upr, Upi, ldk,
                      split, l_in_smem);
}

cudaError_t gemm_any(cudaStream_t s, int m, int n, int k, Z64 A, Z64 B, Z64 C) {
    return gemm_z64(s, m, n, k, -1.0, A, false, B, 1.0, C);
}
cudaError_t gemm_any(cudaStream_t s, int m, int n, int k, C32 A, C32 B, C32 C) {
    return gemm_c32(s, m, n, k, -1.0f, A, false, B, 1.0f, C);
}

template <class V>
bm_status factor_t(bm_ctx* c, V F, bool tc, int split) {
    const int n = c->n;
    const int NB = c->nb;
    const int cl_max = c->panel_cluster;
    SwapMap* const maps = reinterpret_cast<SwapMap*>(c->d_maps);
    SwapMap* const d_map2 = maps + 1;  // sub-panel map (register-row panels)
    // Look-ahead (FP32 with tensor-core trailing updates): after big panel J, the interchanges,
    // U12 solve and trailing update of the next big panel's columns run first on the high-priority
    // stream, which then factors that panel while the low-priority stream finishes the rest of the
    // trailing update; the next block step waits for it.  Profiling keeps the serial order.
    const bool la = std::is_same<V, C32>::value && tc && !c->prof && n > 2 * NB && c->la_hi != nullptr;
    cudaStream_t s = la ? c->la_hi : c->stream;
    cudaStream_t s2 = c->la_lo;
    cudaEvent_t ev_start = c->la_ev[0], ev_fork = c->la_ev[1], ev_join = c->la_ev[2], ev_done = c->la_ev[3];
    if (la) {
        LU_CUDA(cudaEventRecord(ev_start, c->stream));
        LU_CUDA(cudaStreamWaitEvent(s, ev_start, 0));
        LU_CUDA(cudaStreamWaitEvent(s2, ev_start, 0));
    }
    {
        BM_PROF(c, "iota");
        iota_kernel<<<ceil_div(n, 256), 256, 0, s>>>(c->d_perm, n);
        LU_CUDA(cudaGetLastError());
    }
    for (int J = 0, blk = 0; J < n; J += NB, ++blk) {
        const int jb = std::min(NB, n - J);
        SwapMap* const d_map = (blk & 1) ? maps + 2 : maps;  // this big panel's map (two in flight)
        for (int j = J; j < J + jb;) {
            PanelShape ps;
            if (!panel_shape<V>(n - j, cl_max, c->panel_lane_col, ps)) {
                bm_set_error("lu: system too large for the panel kernel");
                return BM_EINVAL;
            }
            const int ib = std::min(ps.nbp, J + jb - j);
            // the lane-per-column kernel (FP32) also applies the sub-panel's interchanges to the
            // big panel's other columns and solves L11 against its columns on the right
            bool fused = false;
            if constexpr (std::is_same<V, C32>::value) {
                if (ps.RPW > 0) {
                    BM_PROF(c, "panel_lc_kernel");
                    LcParams lp{F, j, n - j, ib, J, jb, c->d_ipiv, c->d_info, c->d_info + 1, d_map, c->d_perm};
                    LU_CUDA(launch_panel_lc(s, ps, lp));
                    fused = true;
                }
            }
            if (!fused) {
                BM_PROF(c, "panel_kernel");
                LU_CUDA(launch_panel(s, F, ps, j, n - j, ib, c->d_ipiv, c->d_info, J, jb, d_map2, d_map, c->d_perm));
            }
            if (jb > ib) {
                if (!fused) {
                    BM_PROF(c, "swap_trsm_kernel (sub-panel)");
                    LU_CUDA(launch_swap_trsm<V>(s, F, d_map2, J, j, j + ib, J + jb, j, ib, nullptr, nullptr, 0, 0));
                }
                if (j + ib < J + jb) {
                    BM_PROF(c, "cgemm_simt_kernel (panel update)");
                    LU_CUDA(gemm_any(s, n - j - ib, J + jb - j - ib, ib, F.sub(j + ib, j), F.sub(j, j + ib),
                                     F.sub(j + ib, j + ib)));
                }
            }
            j += ib;
        }
        const bool pack = tc && (J + jb < n);
        const int mm = n - J - jb;          // trailing rows and columns
        const int nnext = la ? std::min(NB, mm) : mm;  // trailing columns updated on s
        // the rest of the previous trailing update (columns this block row touches) is done
        if (la && blk > 0) LU_CUDA(cudaStreamWaitEvent(s, ev_join, 0));
        {
            BM_PROF(c, "swap_trsm_kernel (block row)");
            // on s: the next big panel's columns (all trailing columns without look-ahead), and the
            // columns left of this panel unless the rest stream takes them
            LU_CUDA(launch_swap_trsm<V>(s, F, d_map, 0, la ? 0 : J, J + jb, J + jb + nnext, J, jb,
                                        pack ? c->d_Up_r : nullptr, pack ? c->d_Up_i : nullptr, c->ldk_lu, split));
        }
        if (mm > 0) {
            if (tc) {
                if constexpr (std::is_same<V, C32>::value) {
                    dim3 blk2(32, 8), grid(ceil_div(jb, 32), ceil_div(mm, 32));
                    {
                        BM_PROF(c, "pack_L_kernel");
                        pack_L_kernel<<<grid, blk2, 0, s>>>(F, J + jb, J, mm, jb, split, c->d_Lp_r, c->d_Lp_i,
                                                            c->ldk_lu);
                        LU_CUDA(cudaGetLastError());
                    }
                    const int kext = split ? 3 * jb : jb;
                    C32 Cv = F.sub(J + jb, J + jb);
                    {
                        BM_PROF(c, "cgemm_tc_kernel (trailing update)");
                        LU_CUDA(gemm_tc(s, c->tm_lu[0], c->tm_lu[1], c->tm_lu[2], c->tm_lu[3], Cv.re, Cv.im, Cv.ld, mm,
                                        nnext, kext, -1.0f, 1.0f, c->d_err));
                    }
                    if (la) {
                        // the rest on s2: interchanges of the columns left of this panel and right of
                        // the next one, their U12 rows (packed from pack row NB on) and their update
                        LU_CUDA(cudaEventRecord(ev_fork, s));
                        LU_CUDA(cudaStreamWaitEvent(s2, ev_fork, 0));
                        LU_CUDA(launch_swap_trsm<V>(s2, F, d_map, 0, J, J + jb + nnext, n, J, jb,
                                                    c->d_Up_r + (long)NB * c->ldk_lu, c->d_Up_i + (long)NB * c->ldk_lu,
                                                    c->ldk_lu, split));
                        if (mm > nnext) {
                            C32 Cr = F.sub(J + jb, J + jb + nnext);
                            LU_CUDA(gemm_tc(s2, c->tm_lu[0], c->tm_lu[1], c->tm_lu[4], c->tm_lu[5], Cr.re, Cr.im, Cr.ld,
                                            mm, mm - nnext, kext, -1.0f, 1.0f, c->d_err));
                        }
                        LU_CUDA(cudaEventRecord(ev_join, s2));
                    }
                }
            } else {
                BM_PROF(c, "cgemm_simt_kernel (trailing update)");
                LU_CUDA(gemm_any(s, mm, mm, jb, F.sub(J + jb, J), F.sub(J, J + jb), F.sub(J + jb, J + jb)));
            }
        }
    }
    if (la) LU_CUDA(cudaStreamWaitEvent(s, ev_join, 0));
    // inverted diagonal blocks for getrs
    const int bs = c->bs_solve;
    if (bs != TI_B || bs != TS_BM) {
        bm_set_error("lu: the solve block size must be 64");
        return BM_EINVAL;
    }
    const int nblk = ceil_div(n, bs);
    size_t smem = ((size_t)bs * bs + 3 * (size_t)bs) * sizeof(typename V::cv);
    using CV = typename V::cv;
    constexpr int CG = std::is_same<V, C32>::value ? 1 : 4;  // column groups per block (FP64: 4)
    LU_CUDA(cudaFuncSetAttribute(tri_inv_kernel<V, false, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    LU_CUDA(cudaFuncSetAttribute(tri_inv_kernel<V, true, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    {
        BM_PROF(c, "tri_inv_kernel");
        tri_inv_kernel<V, false, CG><<<dim3(nblk, CG), 256, smem, s>>>(F, n, reinterpret_cast<CV*>(c->d_dinvL));
        tri_inv_kernel<V, true, CG><<<dim3(nblk, CG), 256, smem, s>>>(F, n, reinterpret_cast<CV*>(c->d_dinvU));
        LU_CUDA(cudaGetLastError());
    }
    if constexpr (std::is_same<V, C32>::value) {
        if (nblk > 1) {
            BM_PROF(c, "g_form_kernel");
            const size_t gsm = 2 * (size_t)TS_BM * TS_BM * sizeof(CV);
            LU_CUDA(cudaFuncSetAttribute(g_form_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
            g_form_kernel<V><<<dim3(nblk, nblk), 256, gsm, s>>>(F, n, reinterpret_cast<const CV*>(c->d_dinvL),
                                                                reinterpret_cast<const CV*>(c->d_dinvU));
            LU_CUDA(cudaGetLastError());
        }
    }
    if (la) {  // join the handle's stream
        LU_CUDA(cudaEventRecord(ev_done, s));
        LU_CUDA(cudaStreamWaitEvent(c->stream, ev_done, 0));
    }
    return BM_OK;
}

template <class V, int BN>
cudaError_t launch_trsv_step(cudaStream_t s, V F, V Y, V Z, int r0, int rb, int rest0, int nrest, int nrhs, int bs,
                             const typename V::cv* Tinv) {
    size_t smem = ((size_t)bs * bs + 2 * (size_t)BN * bs + (size_t)bs * TS_BM) * sizeof(typename V::cv);
    auto kern = trsv_step_kernel<V, BN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(std::max(1, ceil_div(nrest, TS_BM)), ceil_div(nrhs, BN));
    kern<<<grid, 256, smem, s>>>(F, Y, Z, r0, rb, rest0, nrest, nrhs, bs, Tinv);
    return cudaGetLastError();
}

template <class V, int BN>
cudaError_t launch_trsv_g_step(cudaStream_t s, V F, V Y, int r0, int rb, int rest0, int nrest, int nrhs) {
    size_t smem = ((size_t)BN * TS_BM + (size_t)TS_BM * TS_BM) * sizeof(typename V::cv);
    dim3 grid(ceil_div(nrest, TS_BM), ceil_div(nrhs, BN));
    auto kern = trsv_g_step_kernel<V, BN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, grid, dim3(256), smem, s, F, Y, r0, rb, rest0, nrest, nrhs);
}

template <class V, int BN>
cudaError_t launch_trsv_diag(cudaStream_t s, V Y, V Z, int n, int nrhs, const typename V::cv* Tinv) {
    size_t smem = ((size_t)TS_BM * TS_BM + (size_t)BN * TS_BM) * sizeof(typename V::cv);
    dim3 grid(ceil_div(n, TS_BM), ceil_div(nrhs, BN));
    auto kern = trsv_diag_kernel<V, BN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, grid, dim3(256), smem, s, Y, Z, n, nrhs, Tinv);
}

// one cooperative launch of the persistent triangular solve: as many CTAs as the items, at most
// the number the device keeps resident (queried once per process and device)
template <bool UPPER>
cudaError_t launch_trsv_flow(cudaStream_t s, C32 F, C32 Y, C32 Z, int n, int nrhs, const float2* T, int* ready,
                             int* err, const int* never, const int* hook, int items, int num_sms) {
    auto kern = trsv_flow_kernel<UPPER>;
    const int smem = (TS_BM * TS_BM + 2 * FL_BN * TS_BM) * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<int, int> per_sm_cache;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = per_sm_cache.find(dev);
        if (it == per_sm_cache.end()) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
            if (e != cudaSuccess) return e;
            it = per_sm_cache.emplace(dev, per_sm).first;
        }
        per_sm = it->second;
    }
    const int grid = std::max(1, std::min(items, std::max(per_sm, 1) * std::max(num_sms, 1)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, F, Y, Z, n, nrhs, T, ready, err, never, hook);
}

// Solve L U X = Y in place (Y holds P B); Zw is an n x nrhs work buffer.
template <class V>
bm_status getrs_t(bm_ctx* c, V F, V Y, V Zw, int nrhs, const typename V::cv* dinvL, const typename V::cv* dinvU) {
    cudaStream_t s = c->stream;
    const int n = c->n, bs = c->bs_solve;
    const int nblk = ceil_div(n, bs);
    // Column tiles of 16 right-hand sides halve each CTA's work (the steps are latency-bound) as
    // long as the widest step still fits about one wave of resident CTAs (two per SM); beyond
    // that, 32-wide tiles (fewer, fatter CTAs) are faster.
    const long widest16 = (long)ceil_div(std::max(n - bs, 1), TS_BM) * ceil_div(nrhs, 16);
    const bool narrow = nrhs <= 16 || widest16 <= (long)(1.1 * 2 * std::max(c->num_sms, 1));
    if constexpr (std::is_same<V, C32>::value) {  // factors in G form
        const int ct = ceil_div(nrhs, FL_BN), items = nblk * ct;
        if (bs == TS_BM && c->d_flow != nullptr && 2L * items <= c->flow_len) {
            // one persistent launch per triangle (block steps and diagonal blocks)
            BM_PROF(c, "trsv_flow_kernel");
            // a timed-out wait raises the handle's device-wait word, which the refinement loop reads
            // back with every backward error (BM_ETIMEOUT)
            // (test hook: with d_info[3] set at assembly, one wait of the forward sweep is on the
            // never-set word after the flags)
            LU_CUDA(cudaMemsetAsync(c->d_flow, 0, (size_t)2 * items * sizeof(int), s));
            LU_CUDA(launch_trsv_flow<false>(s, F, Y, Zw, n, nrhs, dinvL, c->d_flow, c->d_err, c->d_flow + c->flow_len,
                                            c->d_info + 3, items, c->num_sms));
            LU_CUDA(launch_trsv_flow<true>(s, F, Zw, Y, n, nrhs, dinvU, c->d_flow + items, c->d_err, nullptr,
                                           c->d_info + 3, items, c->num_sms));
            return BM_OK;
        }
        auto gstep = [&](V Yv, int r0, int rb, int rest0, int nrest) {
            return narrow ? launch_trsv_g_step<V, 16>(s, F, Yv, r0, rb, rest0, nrest, nrhs)
                          : launch_trsv_g_step<V, 32>(s, F, Yv, r0, rb, rest0, nrest, nrhs);
        };
        auto diag = [&](V Yv, V Zv, const typename V::cv* T) {
            return narrow ? launch_trsv_diag<V, 16>(s, Yv, Zv, n, nrhs, T)
                          : launch_trsv_diag<V, 32>(s, Yv, Zv, n, nrhs, T);
        };
        for (int b = 0; b + 1 < nblk; ++b) {  // Y[below b] -= G_L Y_b
            int r0 = b * bs, rb = std::min(bs, n - r0);
            BM_PROF(c, "trsv_g_step_kernel");
            LU_CUDA(gstep(Y, r0, rb, r0 + rb, n - r0 - rb));
        }
        {
            BM_PROF(c, "trsv_diag_kernel");
            LU_CUDA(diag(Y, Zw, dinvL));  // Zw = L^{-1} P B
        }
        for (int b = nblk - 1; b > 0; --b) {  // Zw[above b] -= G_U Zw_b
            int r0 = b * bs, rb = std::min(bs, n - r0);
            BM_PROF(c, "trsv_g_step_kernel");
            LU_CUDA(gstep(Zw, r0, rb, 0, r0));
        }
        BM_PROF(c, "trsv_diag_kernel");
        LU_CUDA(diag(Zw, Y, dinvU));  // Y = U^{-1} Zw
    } else {
        auto step = [&](V Yv, V Zv, int r0, int rb, int rest0, int nrest, const typename V::cv* T) {
            return narrow ? launch_trsv_step<V, 16>(s, F, Yv, Zv, r0, rb, rest0, nrest, nrhs, bs, T)
                          : launch_trsv_step<V, 32>(s, F, Yv, Zv, r0, rb, rest0, nrest, nrhs, bs, T);
        };
        for (int b = 0; b < nblk; ++b) {  // Zw = L^{-1} Y
            int r0 = b * bs, rb = std::min(bs, n - r0);
            BM_PROF(c, "trsv_step_kernel");
            LU_CUDA(step(Y, Zw, r0, rb, r0 + rb, n - r0 - rb, dinvL + (long)b * bs * bs));
        }
        for (int b = nblk - 1; b >= 0; --b) {  // Y = U^{-1} Zw
            int r0 = b * bs, rb = std::min(bs, n - r0);
            BM_PROF(c, "trsv_step_kernel");
            LU_CUDA(step(Zw, Y, r0, rb, 0, r0, dinvU + (long)b * bs * bs));
        }
    }
    return BM_OK;
}

}  // namespace

// Panel launch configuration of the handle: the largest cluster the device co-schedules (queried
// once), capped by bm_opts.panel_cluster_max (fewer CTAs put more rows on each thread, which selects
// the narrower sub-panel variants), and the panel kernel bm_opts.panel_kernel selects.
bm_status lu_setup(bm_ctx* c, int cluster_cap, int panel_kernel) {
    // the occupancy query is a property of the device and kernel: asked once per process and device
    static std::mutex mu;
    static std::map<int, int> cache[2];
    int& dev_max = (c->prec == BM_FP64) ? c->panel_cluster_z64 : c->panel_cluster_c32;
    if (dev_max == 0) {
        const int kind = (c->prec == BM_FP64) ? 1 : 0;
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache[kind].find(c->device);
        if (it == cache[kind].end())
            it = cache[kind].emplace(c->device, kind ? query_cluster_max_z64() : query_cluster_max_c32()).first;
        dev_max = it->second;
    }
    c->panel_cluster = dev_max;
    if (cluster_cap >= 1 && cluster_cap <= MAX_CLUSTER) c->panel_cluster = std::min(c->panel_cluster, cluster_cap);
    c->panel_lane_col = panel_kernel == 0;
    // the look-ahead's streams (panel chain at the device's highest priority, the rest of the
    // trailing updates at its lowest) and events, created once per handle
    if (c->prec != BM_FP64 && c->la_hi == nullptr) {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->la_hi, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->la_lo, cudaStreamNonBlocking, least) != cudaSuccess) {
            bm_set_error("lu: cannot create the factorisation's streams");
            return BM_ECUDA;
        }
        for (cudaEvent_t& e : c->la_ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                bm_set_error("lu: cannot create the factorisation's events");
                return BM_ECUDA;
            }
    }
    return BM_OK;
}

bm_status lu_factor_enqueue(bm_ctx* c) {
    if (c->prec == BM_FP64) {
        Z64 F{c->d_F64, c->ldF};
        return factor_t<Z64>(c, F, false, 0);
    }
    C32 F{c->d_F32r, c->d_F32i, c->ldF};
    return factor_t<C32>(c, F, true, c->prec == BM_CF32_3XTF32_IR ? 1 : 0);
}

// Y holds P B already (rows gathered with d_perm); solves L U X = Y in place.
bm_status getrs_z64(bm_ctx* c, double2* Y, long ldy, int nrhs) {
    Z64 F{c->d_F64, c->ldF};
    Z64 Yv{Y, ldy};
    Z64 Zv{c->d_Zw64, (long)c->n};
    return getrs_t<Z64>(c, F, Yv, Zv, nrhs, reinterpret_cast<const double2*>(c->d_dinvL),
                        reinterpret_cast<const double2*>(c->d_dinvU));
}

bm_status getrs_c32(bm_ctx* c, float* Yr, float* Yi, long ldy, int nrhs) {
    C32 F{c->d_F32r, c->d_F32i, c->ldF};
    C32 Yv{Yr, Yi, ldy};
    C32 Zv{c->d_Zwr, c->d_Zwi, (long)c->n};
    return getrs_t<C32>(c, F, Yv, Zv, nrhs, reinterpret_cast<const float2*>(c->d_dinvL),
                        reinterpret_cast<const float2*>(c->d_dinvU));
}

cudaError_t launch_gather_rows_z64(cudaStream_t s, const int* perm, int n, int nrhs, const double2* B, long ldb,
                                   double2* Y, long ldy) {
    long total = (long)n * nrhs;
    gather_rows_z64_kernel<<<ceil_div(total, 256), 256, 0, s>>>(perm, n, nrhs, B, ldb, Y, ldy);
    return cudaGetLastError();
}
cudaError_t launch_gather_rows_c32(cudaStream_t s, const int* perm, int n, int nrhs, const float* Br, const float* Bi,
                                   long ldb, float* Yr, float* Yi, long ldy) {
    long total = (long)n * nrhs;
    gather_rows_c32_kernel<<<ceil_div(total, 256), 256, 0, s>>>(perm, n, nrhs, Br, Bi, ldb, Yr, Yi, ldy);
    return cudaGetLastError();
}

size_t swap_map_bytes() { return sizeof(SwapMap); }
