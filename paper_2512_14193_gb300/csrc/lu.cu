// Dense complex LU with partial pivoting on the GPU (the N x N Schur complement U33 of
// Theorem thm:LU, or the 2N x 2N ordinary matrix of Eq. dis_BM), and the triangular solves.
//
// Right-looking blocked LU with two block sizes:
//   for each big panel of NB columns (C32: 128, Z64: 64):
//     for each sub-panel of nbp columns (<= 32):
//        panel_kernel      : unblocked LU with partial pivoting of rows [j, n) x nbp columns.
//                            Rows are spread over a cluster of up to 16 CTAs held in shared
//                            memory; each column's pivot candidates (value, index, whole row) are
//                            pushed to every CTA through distributed shared memory, so one
//                            cluster barrier per column decides the pivot everywhere.
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

// ------------------------------------------------------------------------------------------------
// panel factorisation
// ------------------------------------------------------------------------------------------------
constexpr int PANEL_THREADS = 512;
constexpr int MAX_CLUSTER = 16;

template <class CV> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };

template <class CV>
__host__ __device__ size_t panel_smem_bytes(int nbp, int R) {
    using Rl = typename real_of<CV>::type;
    size_t b = (size_t)nbp * R * sizeof(CV);                // slab
    b += (size_t)2 * MAX_CLUSTER * nbp * sizeof(CV);         // candidate rows
    b += (size_t)2 * nbp * sizeof(CV);                       // diagonal rows
    b += (size_t)2 * MAX_CLUSTER * sizeof(Rl) + 2 * MAX_CLUSTER * sizeof(int);
    b += 32 * (sizeof(Rl) + sizeof(int)) + 64;
    return b;
}

template <class Rl>
__device__ __forceinline__ bool better(Rl v1, int i1, Rl v2, int i2) {
    return v1 > v2 || (v1 == v2 && i1 < i2);
}

template <class V, int NBP>
__global__ void __launch_bounds__(PANEL_THREADS) panel_kernel(V A, int j0, int m, int ib, int R,
                                                              int* __restrict__ ipiv, int* __restrict__ info) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    cg::cluster_group cluster = cg::this_cluster();
    const int cta = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    extern __shared__ __align__(16) unsigned char sm[];
    CV* slab = reinterpret_cast<CV*>(sm);                     // [NBP][R]
    CV* cand_row = slab + (size_t)NBP * R;                     // [2][MAX_CLUSTER][NBP]
    CV* diag_row = cand_row + 2 * MAX_CLUSTER * NBP;           // [2][NBP]
    Rl* cand_val = reinterpret_cast<Rl*>(diag_row + 2 * NBP);  // [2][MAX_CLUSTER]
    int* cand_idx = reinterpret_cast<int*>(cand_val + 2 * MAX_CLUSTER);
    Rl* red_val = reinterpret_cast<Rl*>(cand_idx + 2 * MAX_CLUSTER);  // [32]
    int* red_idx = reinterpret_cast<int*>(red_val + 32);               // [32]

    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const int rb = cta * R;
    const int nloc = max(0, min(R, m - rb));

    for (int c = 0; c < ib; ++c)
        for (int r = tid; r < nloc; r += nth) slab[c * R + r] = A.get((long)j0 + rb + r, (long)j0 + c);

    Rl bv = (Rl)-1;
    int bi = INT_MAX;
    for (int r = tid; r < nloc; r += nth) {
        Rl v = cnorm1(slab[r]);
        if (v > bv) {
            bv = v;
            bi = rb + r;
        }
    }
    __syncthreads();
    cluster.sync();  // every CTA of the cluster is running before remote shared-memory traffic

    for (int c = 0; c < ib; ++c) {
        const int par = c & 1;
        // ---- CTA-wide argmax (max value, then smallest index) ----
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
        Rl cv = red_val[0];
        int ci = red_idx[0];
        for (int w = 1; w < nwarp; ++w) {
            if (better(red_val[w], red_idx[w], cv, ci)) {
                cv = red_val[w];
                ci = red_idx[w];
            }
        }
        // ---- publish candidate row (and the diagonal row if owned) to every CTA ----
        const bool own_diag = (c >= rb && c < rb + nloc);
        for (int e = tid; e < CL * NBP; e += nth) {
            int dst = e / NBP, col = e % NBP;
            CV val = czero<Rl>();
            if (ci != INT_MAX && col < ib) val = slab[col * R + (ci - rb)];
            CV* rr = cluster.map_shared_rank(cand_row + (par * MAX_CLUSTER + cta) * NBP, dst);
            rr[col] = val;
            if (own_diag) {
                CV* rd = cluster.map_shared_rank(diag_row + par * NBP, dst);
                rd[col] = (col < ib) ? slab[col * R + (c - rb)] : czero<Rl>();
            }
            if (col == 0) {
                Rl* rv = cluster.map_shared_rank(cand_val + par * MAX_CLUSTER + cta, dst);
                int* ri = cluster.map_shared_rank(cand_idx + par * MAX_CLUSTER + cta, dst);
                *rv = (ci != INT_MAX) ? cv : (Rl)-1;
                *ri = ci;
            }
        }
        cluster.sync();
        // ---- pivot decision (identical in every CTA) ----
        Rl pv = (Rl)-1;
        int pi = INT_MAX, pq = 0;
        for (int q = 0; q < CL; ++q) {
            Rl v = cand_val[par * MAX_CLUSTER + q];
            int ix = cand_idx[par * MAX_CLUSTER + q];
            if (better(v, ix, pv, pi)) {
                pv = v;
                pi = ix;
                pq = q;
            }
        }
        const CV* u = cand_row + (par * MAX_CLUSTER + pq) * NBP;
        const CV* drow = diag_row + par * NBP;
        const bool sing = !(pv > (Rl)0);
        if (cta == 0 && tid == 0) {
            ipiv[j0 + c] = j0 + pi;
            if (sing && info != nullptr && *info == 0) *info = j0 + c + 1;
        }
        if (!sing && pi != c) {
            if (own_diag)
                for (int col = tid; col < ib; col += nth) slab[col * R + (c - rb)] = u[col];
            if (pi >= rb && pi < rb + nloc)
                for (int col = tid; col < ib; col += nth) slab[col * R + (pi - rb)] = drow[col];
        }
        __syncthreads();
        // ---- scale column c and rank-1 update of the local rows below the pivot ----
        CV inv = sing ? czero<Rl>() : cinv(u[c]);
        bv = (Rl)-1;
        bi = INT_MAX;
        for (int r = tid; r < nloc; r += nth) {
            int gr = rb + r;
            if (gr <= c) continue;
            CV l = slab[c * R + r];
            if (!sing) {
                l = cmul(l, inv);
                slab[c * R + r] = l;
            }
            CV nl;
            nl.x = -l.x;
            nl.y = -l.y;
            for (int k2 = c + 1; k2 < ib; ++k2) {
                CV a = slab[k2 * R + r];
                cfma(a, nl, u[k2]);
                slab[k2 * R + r] = a;
            }
            if (c + 1 < ib) {
                Rl v = cnorm1(slab[(c + 1) * R + r]);
                if (v > bv) {
                    bv = v;
                    bi = gr;
                }
            }
        }
        __syncthreads();
    }
    for (int c = 0; c < ib; ++c)
        for (int r = tid; r < nloc; r += nth) A.set((long)j0 + rb + r, (long)j0 + c, slab[c * R + r]);
}

// ------------------------------------------------------------------------------------------------
// swap maps: the net effect of ib sequential interchanges (j0+k <-> ipiv[j0+k]) on the affected
// rows, as new[dst[t]] = old[src[t]] for t < count.  One warp.
// ------------------------------------------------------------------------------------------------
constexpr int MAP_MAX = 512;  // 2 * max NB (NB <= 256)
struct SwapMap {
    int count;
    int dst[MAP_MAX];
    int src[MAP_MAX];
};

__global__ void build_swap_map_kernel(const int* __restrict__ ipiv, int j0, int ib, SwapMap* __restrict__ out) {
    __shared__ int pk[MAP_MAX / 2];
    __shared__ int cidx[MAP_MAX / 2];
    __shared__ int extra[MAP_MAX / 2];
    __shared__ int content[MAP_MAX];
    const int lane = threadIdx.x;
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
            // earlier k' with the same pivot row?
            int found = INT_MAX;
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
        int s = (sidx < ib) ? j0 + sidx : extra[sidx - ib];
        out->dst[t] = d;
        out->src[t] = s;
    }
    if (lane == 0) out->count = cnt;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Row interchanges (from a swap map) for columns in [a0, a1) u [b0, b1); for columns of the
// second range also X = L11^{-1} X on rows [t0, t0+tb) with the unit-lower L11 at (t0, t0).
// Optionally writes the solved rows as a K-major tensor-core pack (column c -> row c - b0).
// One warp per column; also permutes `perm` (as one extra int column) when given.
template <class V>
__global__ void __launch_bounds__(256) swap_trsm_kernel(V A, const SwapMap* __restrict__ map, int a0, int a1,
                                                         int b0, int b1, int t0, int tb, float* Upr, float* Upi,
                                                         long ldk, int split, int* perm) {
    using CV = typename V::cv;
    using Rl = typename V::real;
    constexpr int QMAX = 8;  // rows per lane: tb <= 256
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int na = a1 - a0, nbc = b1 - b0;
    const int cnt = map ? map->count : 0;
    if (gw == na + nbc && perm != nullptr && map != nullptr) {
        // permute the row-order vector: perm_new[dst] = perm_old[src]
        int v[MAP_MAX / 32];
#pragma unroll
        for (int q = 0; q < MAP_MAX / 32; ++q) {
            int t = lane + 32 * q;
            if (t < cnt) v[q] = perm[map->src[t]];
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < MAP_MAX / 32; ++q) {
            int t = lane + 32 * q;
            if (t < cnt) perm[map->dst[t]] = v[q];
        }
        return;
    }
    if (gw >= na + nbc) return;
    const bool in_b = gw >= na;
    const long col = in_b ? (long)b0 + (gw - na) : (long)a0 + gw;
    // interchanges
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
    if (!in_b || tb <= 0) return;
    // forward substitution with the unit-lower block (lanes own rows lane + 32 q)
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
            if (q >= qk && i > k && i < tb) cfma(x[q], A.get((long)t0 + i, (long)t0 + k), nx);
        }
    }
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
        int i = lane + 32 * q;
        if (i < tb) A.set((long)t0 + i, col, x[q]);
    }
    if (Upr != nullptr) {
        // K-major pack of this column (row index = col - b0); segments [hi | lo | hi] when split
        long row = col - b0;
        float* pr = Upr + row * ldk;
        float* pi = Upi + row * ldk;
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
        // zero padding (done by the first column block)
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
struct PanelCfg {
    int nbp = 32;
    int cl_max = 8;
};

template <class V, int NBP>
cudaError_t launch_panel_t(cudaStream_t s, V A, int j0, int m, int ib, int cl_max, int* ipiv, int* info) {
    using CV = typename V::cv;
    const int rcap = (int)((200 * 1024 - 4096) / ((size_t)NBP * sizeof(CV)));
    int CL = ceil_div(m, rcap);
    if (CL < 1) CL = 1;
    if (CL > cl_max) return cudaErrorInvalidValue;
    int R = ceil_div(m, CL);
    size_t smem = panel_smem_bytes<CV>(NBP, R);
    auto kern = panel_kernel<V, NBP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, A, j0, m, ib, R, ipiv, info);
}

template <class V>
cudaError_t launch_panel(cudaStream_t s, V A, int nbp, int j0, int m, int ib, int cl_max, int* ipiv, int* info);
template <>
cudaError_t launch_panel<C32>(cudaStream_t s, C32 A, int nbp, int j0, int m, int ib, int cl_max, int* ipiv,
                              int* info) {
    if (nbp == 32) return launch_panel_t<C32, 32>(s, A, j0, m, ib, cl_max, ipiv, info);
    if (nbp == 16) return launch_panel_t<C32, 16>(s, A, j0, m, ib, cl_max, ipiv, info);
    return launch_panel_t<C32, 8>(s, A, j0, m, ib, cl_max, ipiv, info);
}
template <>
cudaError_t launch_panel<Z64>(cudaStream_t s, Z64 A, int nbp, int j0, int m, int ib, int cl_max, int* ipiv,
                              int* info) {
    if (nbp == 16) return launch_panel_t<Z64, 16>(s, A, j0, m, ib, cl_max, ipiv, info);
    if (nbp == 8) return launch_panel_t<Z64, 8>(s, A, j0, m, ib, cl_max, ipiv, info);
    return launch_panel_t<Z64, 4>(s, A, j0, m, ib, cl_max, ipiv, info);
}

template <class V>
int pick_nbp(int n, int cl_max, int nbp_max) {
    using CV = typename V::cv;
    for (int nbp = nbp_max; nbp >= 4; nbp /= 2) {
        int rcap = (int)((200 * 1024 - 4096) / ((size_t)nbp * sizeof(CV)));
        if ((long)rcap * cl_max >= n) return nbp;
    }
    return -1;
}

template <class V>
int query_cluster_max() {
    // largest cluster size (16 or 8) the device will co-schedule for the panel kernel
    using CV = typename V::cv;
    int nbp = 16;
    size_t smem = panel_smem_bytes<CV>(nbp, 512);
    auto kern = panel_kernel<V, 16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 8;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 8;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
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
                             float* Upr, float* Upi, long ldk, int split, int* perm) {
    long ncols = (long)(a1 - a0) + (b1 - b0) + (perm ? 1 : 0);
    if (ncols <= 0) return cudaSuccess;
    long threads = ncols * 32;
    swap_trsm_kernel<V><<<ceil_div(threads, 256), 256, 0, s>>>(A, map, a0, a1, b0, b1, t0, tb, Upr, Upi, ldk, split,
                                                                perm);
    return cudaGetLastError();
}

cudaError_t gemm_any(cudaStream_t s, int m, int n, int k, Z64 A, Z64 B, Z64 C) {
    return gemm_z64(s, m, n, k, -1.0, A, false, B, 1.0, C);
}
cudaError_t gemm_any(cudaStream_t s, int m, int n, int k, C32 A, C32 B, C32 C) {
    return gemm_c32(s, m, n, k, -1.0f, A, false, B, 1.0f, C);
}

#define LU_CUDA(expr)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            bm_set_error(std::string("lu: ") + #expr + ": " + cudaGetErrorString(_e));                 \
            return BM_ECUDA;                                                                           \
        }                                                                                              \
    } while (0)

template <class V>
bm_status factor_t(bm_ctx* c, V F, bool tc, int split) {
    cudaStream_t s = c->stream;
    const int n = c->n;
    const int NB = c->nb;
    const int cl_max = c->panel_cluster;
    const int nbp = pick_nbp<V>(n, cl_max, std::is_same<V, C32>::value ? 32 : 16);
    if (nbp < 0) {
        bm_set_error("lu: system too large for the panel kernel");
        return BM_EINVAL;
    }
    SwapMap* d_map = reinterpret_cast<SwapMap*>(c->d_maps);  // big-panel map
    SwapMap* d_map2 = d_map + 1;                              // sub-panel map
    iota_kernel<<<ceil_div(n, 256), 256, 0, s>>>(c->d_perm, n);
    LU_CUDA(cudaGetLastError());
    for (int J = 0; J < n; J += NB) {
        const int jb = std::min(NB, n - J);
        for (int j = J; j < J + jb; j += nbp) {
            const int ib = std::min(nbp, J + jb - j);
            LU_CUDA(launch_panel<V>(s, F, nbp, j, n - j, ib, cl_max, c->d_ipiv, c->d_info));
            if (jb > ib) {
                build_swap_map_kernel<<<1, 32, 0, s>>>(c->d_ipiv, j, ib, d_map2);
                LU_CUDA(cudaGetLastError());
                LU_CUDA(launch_swap_trsm<V>(s, F, d_map2, J, j, j + ib, J + jb, j, ib, nullptr, nullptr, 0, 0,
                                            nullptr));
                if (j + ib < J + jb)
                    LU_CUDA(gemm_any(s, n - j - ib, J + jb - j - ib, ib, F.sub(j + ib, j), F.sub(j, j + ib),
                                     F.sub(j + ib, j + ib)));
            }
        }
        build_swap_map_kernel<<<1, 32, 0, s>>>(c->d_ipiv, J, jb, d_map);
        LU_CUDA(cudaGetLastError());
        const bool pack = tc && (J + jb < n);
        LU_CUDA(launch_swap_trsm<V>(s, F, d_map, 0, J, J + jb, n, J, jb, pack ? c->d_Up_r : nullptr,
                                    pack ? c->d_Up_i : nullptr, c->ldk_lu, split, c->d_perm));
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
