// Dense complex LU with partial pivoting on the GPU (the N x N Schur complement U33 of
// Theorem thm:LU, or the 2N x 2N ordinary matrix of Eq. dis_BM), and the triangular solves.
//
// Right-looking blocked LU with two block sizes:
//   for each big panel of NB columns (C32: 128, Z64: 64):
//     for each sub-panel of nbp columns (nbp = 32/16/8 for C32, 16/8/4 for Z64 - wider when the
//     rows below the diagonal are fewer):
//        panel_kernel      : unblocked LU with partial pivoting of rows [j, n) x nbp columns.
//                            Rows are spread over a cluster of up to 16 CTAs, one to four rows per
//                            thread, held in registers.  Each column's pivot candidates (value,
//                            index, whole row) are pushed to every CTA through distributed shared
//                            memory; the cluster barrier is split into arrive/wait so that the
//                            rank-1 update of all but the next column runs while it completes.
//                            The last CTA work also builds the row-interchange maps.
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
// that every step is a small matrix product.
#include "common.cuh"
#include "kernels.cuh"

#include <cooperative_groups.h>
#include <algorithm>
#include <climits>
#include <type_traits>

namespace cg = cooperative_groups;

namespace {

constexpr int PANEL_THREADS = 512;
constexpr int MAX_CLUSTER = 16;
constexpr int MAP_MAX = 512;  // 2 * max NB (NB <= 256)

struct SwapMap {  // new[dst[t]] = old[src[t]], t < count
    int count;
    int dst[MAP_MAX];
    int src[MAP_MAX];
};

template <class Rl>
__device__ __forceinline__ bool better(Rl v1, int i1, Rl v2, int i2) {
    return v1 > v2 || (v1 == v2 && i1 < i2);
}

// ------------------------------------------------------------------------------------------------
// swap maps: the net effect of ib sequential interchanges (j0+k <-> ipiv[j0+k]) on the rows they
// touch.  Run by one warp; s_* are shared scratch arrays of MAP_MAX/2 (pk, cidx, extra) and
// MAP_MAX (content) ints.
// ------------------------------------------------------------------------------------------------
__device__ void build_map_warp(const int* ipiv, int j0, int ib, SwapMap* out, int* pk, int* cidx, int* extra,
                               int* content) {
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < ib; k += 32) pk[k] = ipiv[j0 + k];
    for (int t = lane; t < 2 * ib; t += 32) content[t] = t;
    __syncwarp();
    int nextra = 0;
    for (int k = 0; k < ib; ++k) {
        int p = pk[k];
        int ci;
        if (p < j0 + ib) {
            ci = p - j0;
        } else {
            int found = INT_MAX;  // earlier interchange with the same row?
            for (int base = 0; base < k; base += 32) {
                int kk = base + lane;
                bool hit = (kk < k) && (pk[kk] == p);
                unsigned b = __ballot_sync(0xffffffffu, hit);
                if (b) {
                    found = base + __ffs(b) - 1;
                    break;
                }
            }
            if (found != INT_MAX) {
                ci = cidx[found];
            } else {
                ci = ib + nextra;
                if (lane == 0) extra[nextra] = p;
                ++nextra;
            }
        }
        if (lane == 0) {
            cidx[k] = ci;
            int t = content[k];
            content[k] = content[ci];
            content[ci] = t;
        }
        __syncwarp();
    }
    int cnt = ib + nextra;
    for (int t = lane; t < cnt; t += 32) {
        int d = (t < ib) ? j0 + t : extra[t - ib];
        int sidx = content[t];
        int sr = (sidx < ib) ? j0 + sidx : extra[sidx - ib];
        out->dst[t] = d;
        out->src[t] = sr;
    }
    if (lane == 0) out->count = cnt;
    __syncwarp();
}

// apply a map to an int vector (the row order of the factorisation), one warp
__device__ void apply_map_int_warp(const SwapMap* map, int* v) {
    const int lane = threadIdx.x & 31;
    const int cnt = map->count;
    int val[MAP_MAX / 32];
#pragma unroll
    for (int q = 0; q < MAP_MAX / 32; ++q) {
        int t = lane + 32 * q;
        if (t < cnt) val[q] = v[map->src[t]];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < MAP_MAX / 32; ++q) {
        int t = lane + 32 * q;
        if (t < cnt) v[map->dst[t]] = val[q];
    }
    __syncwarp();
}

// ------------------------------------------------------------------------------------------------
// panel factorisation
// ------------------------------------------------------------------------------------------------
template <class CV, int NBP>
__device__ __forceinline__ CV pick(const CV (&r)[NBP], int c) {
    CV v = r[0];
#pragma unroll
    for (int k = 1; k < NBP; ++k)
        if (k == c) v = r[k];
    return v;
}

template <class V, int NBP, int RPT>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
    panel_kernel(V A, int j0, int m, int ib, int R, int* __restrict__ ipiv, int* __restrict__ info, int J, int jb,
                 SwapMap* __restrict__ map_inner, SwapMap* __restrict__ map_big, int* __restrict__ perm) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    cg::cluster_group cluster = cg::this_cluster();
    const int cta = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    __shared__ CV cand_row[2][MAX_CLUSTER][NBP];
    __shared__ CV diag_row[2][NBP];
    __shared__ Rl cand_val[2][MAX_CLUSTER];
    __shared__ int cand_idx[2][MAX_CLUSTER];
    __shared__ CV ucur[2][NBP];   // local copies of the last two pivot rows
    __shared__ CV mycand[NBP];    // this CTA's candidate row, staged for publishing
    __shared__ CV mydiag[NBP];    // the diagonal row (if this CTA owns it), staged
    __shared__ Rl red_val[PANEL_THREADS / 32];
    __shared__ int red_idx[PANEL_THREADS / 32];
    __shared__ int s_map[MAP_MAX / 2 * 3 + MAP_MAX];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int rb = cta * R;
    const int nloc = max(0, min(R, m - rb));
    const CV zero = czero<Rl>();

    CV row[RPT][NBP];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int lr = tid + q * PANEL_THREADS;
#pragma unroll
        for (int k = 0; k < NBP; ++k)
            row[q][k] = (lr < nloc && k < ib) ? A.get((long)j0 + rb + lr, (long)j0 + k) : zero;
    }
    Rl bv = (Rl)-1;
    int bi = INT_MAX;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int lr = tid + q * PANEL_THREADS;
        if (lr < nloc) {
            Rl v = cnorm1(row[q][0]);
            if (v > bv) {
                bv = v;
                bi = rb + lr;
            }
        }
    }
    cluster.sync();  // every CTA of the cluster runs before remote shared-memory traffic

    for (int c = 0; c < ib; ++c) {
        const int par = c & 1;
        const CV* uprev = ucur[par ^ 1];  // pivot row of column c-1 (valid for c > 0)
        // ---- (1) CTA-wide argmax of column c: max |Re|+|Im|, then the smallest row ----
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Rl ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (better(ov, oi, bv, bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            red_val[warp] = bv;
            red_idx[warp] = bi;
        }
        __syncthreads();
        Rl cv = (lane < PANEL_THREADS / 32) ? red_val[lane] : (Rl)-1;
        int ci = (lane < PANEL_THREADS / 32) ? red_idx[lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {  // whole warp, so every lane ends with the CTA result
            Rl ov = __shfl_xor_sync(0xffffffffu, cv, o);
            int oi = __shfl_xor_sync(0xffffffffu, ci, o);
            if (better(ov, oi, cv, ci)) {
                cv = ov;
                ci = oi;
            }
        }
        // ---- (2) stage the candidate row and the diagonal row with pivot c-1's update applied ----
        const bool own_diag = (c >= rb && c < rb + nloc);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int gr = rb + tid + q * PANEL_THREADS;
            const bool is_cand = (gr == ci), is_diag = (gr == c);
            if (is_cand || is_diag) {
                CV lp = zero;
                if (c > 0) {
                    lp = pick<CV, NBP>(row[q], c - 1);
                    lp.x = -lp.x;
                    lp.y = -lp.y;
                }
#pragma unroll
                for (int k = 0; k < NBP; ++k) {
                    CV v = row[q][k];
                    if (c > 0 && k > c) cfma(v, lp, uprev[k]);
                    if (is_cand) mycand[k] = v;
                    if (is_diag) mydiag[k] = v;
                }
            }
        }
        __syncthreads();
        // ---- (3) publish to every CTA, arrive ----
        for (int e = tid; e < CL * NBP; e += PANEL_THREADS) {
            const int dst = e / NBP, col = e % NBP;
            CV* rr = cluster.map_shared_rank(&cand_row[par][cta][0], dst);
            rr[col] = (ci != INT_MAX) ? mycand[col] : zero;
            if (own_diag) {
                CV* rd = cluster.map_shared_rank(&diag_row[par][0], dst);
                rd[col] = mydiag[col];
            }
            if (col == 0) {
                *cluster.map_shared_rank(&cand_val[par][cta], dst) = (ci != INT_MAX) ? cv : (Rl)-1;
                *cluster.map_shared_rank(&cand_idx[par][cta], dst) = ci;
            }
        }
        cluster.barrier_arrive();
        // ---- (4) while the barrier completes: pivot c-1's update of columns c+1.. ----
        if (c > 0) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int lr = tid + q * PANEL_THREADS;
                if (lr < nloc && rb + lr > c - 1) {
                    CV lp = pick<CV, NBP>(row[q], c - 1);
                    lp.x = -lp.x;
                    lp.y = -lp.y;
#pragma unroll
                    for (int k = 0; k < NBP; ++k)
                        if (k > c) cfma(row[q][k], lp, uprev[k]);
                }
            }
        }
        cluster.barrier_wait();
        // ---- (5) pivot decision for column c (identical in every CTA) ----
        Rl pv = (Rl)-1;
        int pi = INT_MAX, pq = 0;
        for (int q = 0; q < CL; ++q) {
            Rl v = cand_val[par][q];
            int ix = cand_idx[par][q];
            if (better(v, ix, pv, pi)) {
                pv = v;
                pi = ix;
                pq = q;
            }
        }
        const CV* u = &cand_row[par][pq][0];
        const CV* drow = &diag_row[par][0];
        const bool sing = !(pv > (Rl)0);
        if (tid < NBP) ucur[par][tid] = u[tid];
        if (cta == 0 && tid == 0) {
            ipiv[j0 + c] = j0 + pi;
            if (sing && info != nullptr && *info == 0) *info = j0 + c + 1;
        }
        // ---- (6) interchange rows c and pi ----
        if (!sing && pi != c) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int gr = rb + tid + q * PANEL_THREADS;
                if (gr == c) {
#pragma unroll
                    for (int k = 0; k < NBP; ++k) row[q][k] = u[k];
                } else if (gr == pi) {
#pragma unroll
                    for (int k = 0; k < NBP; ++k) row[q][k] = drow[k];
                }
            }
        }
        // ---- (7) scale column c, update column c+1, argmax of column c+1 ----
        const CV uc = u[0 + c];
        const CV inv = sing ? zero : cinv(uc);
        const CV un = (c + 1 < NBP) ? u[c + 1] : zero;
        bv = (Rl)-1;
        bi = INT_MAX;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int lr = tid + q * PANEL_THREADS;
            const int gr = rb + lr;
            if (lr < nloc && gr > c) {
                CV l = pick<CV, NBP>(row[q], c);
                if (!sing) l = cmul(l, inv);
                CV nl;
                nl.x = -l.x;
                nl.y = -l.y;
#pragma unroll
                for (int k = 0; k < NBP; ++k) {
                    if (k == c) row[q][k] = l;
                    if (k == c + 1) {
                        cfma(row[q][k], nl, un);
                        Rl v = cnorm1(row[q][k]);
                        if (v > bv) {
                            bv = v;
                            bi = gr;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int lr = tid + q * PANEL_THREADS;
        if (lr < nloc)
#pragma unroll
            for (int k = 0; k < NBP; ++k)
                if (k < ib) A.set((long)j0 + rb + lr, (long)j0 + k, row[q][k]);
    }
    // ---- row-interchange maps (CTA 0, warp 0): this sub-panel's, and the big panel's at its end ----
    if (cta == 0) {
        __syncthreads();
        __threadfence_block();
        if (warp == 0) {
            int* pk = s_map;
            int* cidx = pk + MAP_MAX / 2;
            int* extra = cidx + MAP_MAX / 2;
            int* content = extra + MAP_MAX / 2;
            if (map_inner) build_map_warp(ipiv, j0, ib, map_inner, pk, cidx, extra, content);
            if (map_big && j0 + ib == J + jb) {
                build_map_warp(ipiv, J, jb, map_big, pk, cidx, extra, content);
                __threadfence_block();
                if (perm) apply_map_int_warp(map_big, perm);
            }
        }
    }
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Row interchanges (from a swap map) for columns in [a0, a1) u [b0, b1); for columns of the
// second range also X = L11^{-1} X on rows [t0, t0+tb) with the unit-lower L11 at (t0, t0),
// staged in shared memory when it fits.  Optionally writes the solved rows as a K-major
// tensor-core pack (column c -> row c - b0).  One warp per column, COLS columns per warp.
constexpr int ST_WARPS = 8, ST_COLS = 4;
template <class V>
__global__ void __launch_bounds__(ST_WARPS * 32) swap_trsm_kernel(V A, const SwapMap* __restrict__ map, int a0, int a1,
                                                                   int b0, int b1, int t0, int tb, float* Upr,
                                                                   float* Upi, long ldk, int split, int l_in_smem) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    constexpr int QMAX = 8;  // rows per lane: tb <= 256
    extern __shared__ __align__(16) unsigned char smraw[];
    CV* Ls = reinterpret_cast<CV*>(smraw);  // tb x tb, column-major
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int na = a1 - a0, nbc = b1 - b0;
    const int ncols = na + nbc;
    const int cta_col0 = blockIdx.x * ST_WARPS * ST_COLS;
    const bool cta_has_b = (cta_col0 + ST_WARPS * ST_COLS > na) && tb > 0;
    if (cta_has_b && l_in_smem) {
        for (int e = threadIdx.x; e < tb * tb; e += blockDim.x) {
            int i = e % tb, k = e / tb;
            Ls[e] = (i > k) ? A.get((long)t0 + i, (long)t0 + k) : czero<Rl>();
        }
        __syncthreads();
    }
    const int cnt = map ? map->count : 0;
    for (int cc = 0; cc < ST_COLS; ++cc) {
        const int gw = cta_col0 + warp * ST_COLS + cc;
        if (gw >= ncols) break;
        const bool in_b = gw >= na;
        const long col = in_b ? (long)b0 + (gw - na) : (long)a0 + gw;
        if (cnt > 0) {
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
        if (!in_b || tb <= 0) continue;
        CV x[QMAX];
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            int i = lane + 32 * q;
            x[q] = (i < tb) ? A.get((long)t0 + i, col) : czero<Rl>();
        }
        for (int k = 0; k < tb; ++k) {
            const int qk = k >> 5, lk = k & 31;
            CV xk = czero<Rl>();
#pragma unroll
            for (int q = 0; q < QMAX; ++q)
                if (q == qk) xk = x[q];
            xk.x = __shfl_sync(0xffffffffu, xk.x, lk);
            xk.y = __shfl_sync(0xffffffffu, xk.y, lk);
            CV nx;
            nx.x = -xk.x;
            nx.y = -xk.y;
#pragma unroll
            for (int q = 0; q < QMAX; ++q) {
                int i = lane + 32 * q;
                if (q >= qk && i > k && i < tb) {
                    CV l = l_in_smem ? Ls[i + k * tb] : A.get((long)t0 + i, (long)t0 + k);
                    cfma(x[q], l, nx);
                }
            }
        }
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

// Inverse of each bs x bs diagonal block (unit lower L or upper U) of the LU factor.
template <class V, bool UPPER>
__global__ void tri_inv_kernel(V F, int n, int bs, typename V::cv* __restrict__ out) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* T = reinterpret_cast<CV*>(sm);  // [bs][bs] column-major
    CV* X = T + bs * bs;
    const int b = blockIdx.x;
    const int r0 = b * bs;
    const int rb = min(bs, n - r0);
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        int i = e % bs, j = e / bs;
        T[e] = (i < rb && j < rb) ? F.get((long)r0 + i, (long)r0 + j) : czero<Rl>();
    }
    __syncthreads();
    const int c = threadIdx.x;  // one column of the inverse per thread
    if (c >= rb)
        for (int i = 0; i < bs; ++i) X[i + c * bs] = czero<Rl>();
    if (c < rb) {
        if (!UPPER) {
            for (int i = 0; i < rb; ++i) {
                CV s = czero<Rl>();
                if (i == c) s.x = (Rl)1;
                if (i > c) {
                    for (int k = c; k < i; ++k) {
                        CV nl = T[i + k * bs];
                        nl.x = -nl.x;
                        nl.y = -nl.y;
                        cfma(s, nl, X[k + c * bs]);
                    }
                }
                X[i + c * bs] = (i < c) ? czero<Rl>() : s;
            }
        } else {
            for (int i = rb - 1; i >= 0; --i) {
                CV s = czero<Rl>();
                if (i <= c) {
                    if (i == c) s.x = (Rl)1;
                    for (int k = i + 1; k <= c; ++k) {
                        CV nu = T[i + k * bs];
                        nu.x = -nu.x;
                        nu.y = -nu.y;
                        cfma(s, nu, X[k + c * bs]);
                    }
                    s = cmul(s, cinv(T[i + i * bs]));
                }
                X[i + c * bs] = s;
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) out[(long)b * bs * bs + e] = X[e];
}

// Y[r0:r0+rb, :] = Tinv * Y[r0:r0+rb, :] in place (one CTA per 32 right-hand sides)
template <class V>
__global__ void apply_inv_kernel(V Y, int r0, int rb, int nrhs, int bs, const typename V::cv* __restrict__ Tinv) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    extern __shared__ __align__(16) unsigned char sm[];
    CV* Ys = reinterpret_cast<CV*>(sm);  // [32][bs]
    const int c0 = blockIdx.x * 32;
    const int nc = min(32, nrhs - c0);
    for (int e = threadIdx.x; e < bs * 32; e += blockDim.x) {
        int i = e % bs, cc = e / bs;
        Ys[cc * bs + i] = (i < rb && cc < nc) ? Y.get((long)r0 + i, (long)c0 + cc) : czero<Rl>();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rb * nc; e += blockDim.x) {
        int i = e % rb, cc = e / rb;
        CV s = czero<Rl>();
        for (int k = 0; k < rb; ++k) cfma(s, Tinv[i + (long)k * bs], Ys[cc * bs + k]);
        Y.set((long)r0 + i, (long)c0 + cc, s);
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

struct PanelShape {
    int CL, R, RPT, nbp;
};

// cluster size, rows per CTA, rows per thread and sub-panel width for a panel of m rows
template <class V>
bool panel_shape(int m, int cl_max, PanelShape& ps) {
    constexpr int W = std::is_same<V, C32>::value ? 32 : 16;  // widest sub-panel (1 row per thread)
    int CL = std::min(cl_max, std::max(1, ceil_div(m, PANEL_THREADS)));
    int R = ceil_div(m, CL);
    int RPT = ceil_div(R, PANEL_THREADS);
    if (RPT > 4) return false;
    if (RPT == 3) RPT = 4;
    ps = PanelShape{CL, R, RPT, W / RPT};
    return true;
}

template <class V, int NBP, int RPT>
cudaError_t launch_panel_t(cudaStream_t s, V A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                           int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    auto kern = panel_kernel<V, NBP, RPT>;
    if (ps.CL > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ps.CL, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ps.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, A, j0, m, ib, ps.R, ipiv, info, J, jb, mi, mb, perm);
}

template <class V>
cudaError_t launch_panel(cudaStream_t s, V A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info, int J,
                         int jb, SwapMap* mi, SwapMap* mb, int* perm);
template <>
cudaError_t launch_panel<C32>(cudaStream_t s, C32 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                              int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    if (ps.RPT == 1) return launch_panel_t<C32, 32, 1>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    if (ps.RPT == 2) return launch_panel_t<C32, 16, 2>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    return launch_panel_t<C32, 8, 4>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
}
template <>
cudaError_t launch_panel<Z64>(cudaStream_t s, Z64 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                              int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    if (ps.RPT == 1) return launch_panel_t<Z64, 16, 1>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    if (ps.RPT == 2) return launch_panel_t<Z64, 8, 2>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    return launch_panel_t<Z64, 4, 4>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
}

template <class V>
int query_cluster_max() {
    // largest cluster size (16 or 8) the device will co-schedule for the panel kernel
    auto kern = panel_kernel<V, std::is_same<V, C32>::value ? 32 : 16, 1>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    return ncl >= 1 ? 16 : 8;
}

template <class V>
cudaError_t launch_swap_trsm(cudaStream_t s, V A, const SwapMap* map, int a0, int a1, int b0, int b1, int t0, int tb,
                             float* Upr, float* Upi, long ldk, int split) {
    using CV = typename V::cv;
    long ncols = (long)(a1 - a0) + (b1 - b0);
    if (ncols <= 0) return cudaSuccess;
    size_t lbytes = (size_t)tb * tb * sizeof(CV);
    int l_in_smem = (tb > 0 && lbytes <= 160 * 1024) ? 1 : 0;
    size_t smem = l_in_smem ? lbytes : 0;
    auto kern = swap_trsm_kernel<V>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int grid = ceil_div(ncols, ST_WARPS * ST_COLS);
    kern<<<grid, ST_WARPS * 32, smem, s>>>(A, map, a0, a1, b0, b1, t0, tb, Upr, Upi, ldk, split, l_in_smem);
    return cudaGetLastError();
}

cudaError_t gemm_any(cudaStream_t s, int m, int n, int k, Z64 A, Z64 B, Z64 C) {
    return gemm_z64(s, m, n, k, -1.0, A, false, B, 1.0, C);
}
cudaError_t gemm_any(cudaStream_t s, int m, int n, int k, C32 A, C32 B, C32 C) {
    return gemm_c32(s, m, n, k, -1.0f, A, false, B, 1.0f, C);
}

template <class V>
bm_status factor_t(bm_ctx* c, V F, bool tc, int split) {
    cudaStream_t s = c->stream;
    const int n = c->n;
    const int NB = c->nb;
    const int cl_max = c->panel_cluster;
    SwapMap* d_map = reinterpret_cast<SwapMap*>(c->d_maps);  // big-panel map
    SwapMap* d_map2 = d_map + 1;                              // sub-panel map
    iota_kernel<<<ceil_div(n, 256), 256, 0, s>>>(c->d_perm, n);
    LU_CUDA(cudaGetLastError());
    for (int J = 0; J < n; J += NB) {
        const int jb = std::min(NB, n - J);
        for (int j = J; j < J + jb;) {
            PanelShape ps;
            if (!panel_shape<V>(n - j, cl_max, ps)) {
                bm_set_error("lu: system too large for the panel kernel");
                return BM_EINVAL;
            }
            const int ib = std::min(ps.nbp, J + jb - j);
            LU_CUDA(launch_panel<V>(s, F, ps, j, n - j, ib, c->d_ipiv, c->d_info, J, jb, d_map2, d_map, c->d_perm));
            if (jb > ib) {
                LU_CUDA(launch_swap_trsm<V>(s, F, d_map2, J, j, j + ib, J + jb, j, ib, nullptr, nullptr, 0, 0));
                if (j + ib < J + jb)
                    LU_CUDA(gemm_any(s, n - j - ib, J + jb - j - ib, ib, F.sub(j + ib, j), F.sub(j, j + ib),
                                     F.sub(j + ib, j + ib)));
            }
            j += ib;
        }
        const bool pack = tc && (J + jb < n);
        LU_CUDA(launch_swap_trsm<V>(s, F, d_map, 0, J, J + jb, n, J, jb, pack ? c->d_Up_r : nullptr,
                                    pack ? c->d_Up_i : nullptr, c->ldk_lu, split));
        if (J + jb < n) {
            const int mm = n - J - jb;
            if (tc) {
                if constexpr (std::is_same<V, C32>::value) {
                    dim3 blk(32, 8), grid(ceil_div(jb, 32), ceil_div(mm, 32));
                    pack_L_kernel<<<grid, blk, 0, s>>>(F, J + jb, J, mm, jb, split, c->d_Lp_r, c->d_Lp_i, c->ldk_lu);
                    LU_CUDA(cudaGetLastError());
                    int kext = split ? 3 * jb : jb;
                    C32 Cv = F.sub(J + jb, J + jb);
                    LU_CUDA(gemm_tc(s, c->tm_lu[0], c->tm_lu[1], c->tm_lu[2], c->tm_lu[3], Cv.re, Cv.im, Cv.ld, mm, mm,
                                    kext, -1.0f, 1.0f, c->d_err));
                }
            } else {
                LU_CUDA(gemm_any(s, mm, mm, jb, F.sub(J + jb, J), F.sub(J, J + jb), F.sub(J + jb, J + jb)));
            }
        }
    }
    // inverted diagonal blocks for getrs
    const int bs = c->bs_solve;
    const int nblk = ceil_div(n, bs);
    size_t smem = 2 * (size_t)bs * bs * sizeof(typename V::cv);
    using CV = typename V::cv;
    LU_CUDA(cudaFuncSetAttribute(tri_inv_kernel<V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LU_CUDA(cudaFuncSetAttribute(tri_inv_kernel<V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tri_inv_kernel<V, false><<<nblk, bs, smem, s>>>(F, n, bs, reinterpret_cast<CV*>(c->d_dinvL));
    tri_inv_kernel<V, true><<<nblk, bs, smem, s>>>(F, n, bs, reinterpret_cast<CV*>(c->d_dinvU));
    LU_CUDA(cudaGetLastError());
    return BM_OK;
}

template <class V>
bm_status getrs_t(bm_ctx* c, V F, V Y, int nrhs, const typename V::cv* dinvL, const typename V::cv* dinvU) {
    cudaStream_t s = c->stream;
    const int n = c->n, bs = c->bs_solve;
    const int nblk = ceil_div(n, bs);
    size_t smem = (size_t)32 * bs * sizeof(typename V::cv);
    LU_CUDA(cudaFuncSetAttribute(apply_inv_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ncta = ceil_div(nrhs, 32);
    for (int b = 0; b < nblk; ++b) {
        int r0 = b * bs, rb = std::min(bs, n - r0);
        apply_inv_kernel<V><<<ncta, 256, smem, s>>>(Y, r0, rb, nrhs, bs, dinvL + (long)b * bs * bs);
        LU_CUDA(cudaGetLastError());
        if (r0 + rb < n) LU_CUDA(gemm_any(s, n - r0 - rb, nrhs, rb, F.sub(r0 + rb, r0), Y.sub(r0, 0), Y.sub(r0 + rb, 0)));
    }
    for (int b = nblk - 1; b >= 0; --b) {
        int r0 = b * bs, rb = std::min(bs, n - r0);
        apply_inv_kernel<V><<<ncta, 256, smem, s>>>(Y, r0, rb, nrhs, bs, dinvU + (long)b * bs * bs);
        LU_CUDA(cudaGetLastError());
        if (r0 > 0) LU_CUDA(gemm_any(s, r0, nrhs, rb, F.sub(0, r0), Y.sub(r0, 0), Y.sub(0, 0)));
    }
    return BM_OK;
}

}  // namespace

bm_status lu_setup(bm_ctx* c) {
    if (c->panel_cluster == 0) {
        c->panel_cluster = (c->prec == BM_FP64) ? query_cluster_max<Z64>() : query_cluster_max<C32>();
        // BM_PANEL_CLUSTER_MAX caps the panel cluster (1..16); fewer CTAs put more rows on
        // each thread, which selects the narrower sub-panel variants
        if (const char* e = getenv("BM_PANEL_CLUSTER_MAX")) {
            int v = atoi(e);
            if (v >= 1 && v <= 16) c->panel_cluster = std::min(c->panel_cluster, v);
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
    return getrs_t<Z64>(c, F, Yv, nrhs, reinterpret_cast<const double2*>(c->d_dinvL),
                        reinterpret_cast<const double2*>(c->d_dinvU));
}

bm_status getrs_c32(bm_ctx* c, float* Yr, float* Yi, long ldy, int nrhs) {
    C32 F{c->d_F32r, c->d_F32i, c->ldF};
    C32 Yv{Yr, Yi, ldy};
    return getrs_t<C32>(c, F, Yv, nrhs, reinterpret_cast<const float2*>(c->d_dinvL),
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
