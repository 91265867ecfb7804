// Internals of the LU panel factorisation shared by lu.cu and the per-precision panel
// translation units (panel_c32.cu, panel_z64.cu), which compile in parallel.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

#include <cooperative_groups.h>
#include <algorithm>
#include <climits>
#include <type_traits>

namespace lu_detail {
namespace cg = cooperative_groups;

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
// FP64: the values are magnitudes (>= 0) or -1 for "no candidate", whose bit patterns as signed
// 64-bit integers order like the values, so the comparison runs on the integer pipe instead of
// the FP64 pipe (1/64 of the FP32 rate on this part)
template <>
__device__ __forceinline__ bool better<double>(double v1, int i1, double v2, int i2) {
    const long long a = __double_as_longlong(v1), b = __double_as_longlong(v2);
    return a > b || (a == b && i1 < i2);
}

// ------------------------------------------------------------------------------------------------
// swap maps: the net effect of ib sequential interchanges (j0+k <-> ipiv[j0+k]) on the rows they
// touch.  Run by one warp; s_* are shared scratch arrays of MAP_MAX/2 (pk, cidx, extra) and
// MAP_MAX (content) ints.
// ------------------------------------------------------------------------------------------------
__device__ inline void build_map_warp(const int* ipiv, int j0, int ib, SwapMap* out, int* pk, int* cidx, int* extra,
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
__device__ inline void apply_map_int_warp(const SwapMap* map, int* v) {
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
// helpers of the cluster panel kernels: register-array access by a runtime index (a chain of
// selects, no local memory), distributed shared memory, bounded mbarrier waits, warp argmax
// ------------------------------------------------------------------------------------------------
template <class T, int N>
__device__ __forceinline__ T row_get(const T (&row)[N], int s) {
    T v = row[0];
#pragma unroll
    for (int r = 1; r < N; ++r)
        if (r == s) v = row[r];
    return v;
}
template <class T, int N>
__device__ __forceinline__ void row_set(T (&row)[N], int s, T v) {
#pragma unroll
    for (int r = 0; r < N; ++r)
        if (r == s) row[r] = v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t remote_addr(uint32_t local, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
// 8 bytes from registers into another CTA's shared memory, completing on that CTA's mbarrier
__device__ __forceinline__ void push8(uint32_t raddr, uint32_t x, uint32_t y, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "r"(x), "r"(y), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait (2 s by the global timer) for phase `parity` of a local mbarrier, with cluster-scope
// acquire of the data that completed it; false on a timeout
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok = 0;
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it == 0) t0 = gtime();
        else if (gtime() - t0 > 2000000000ull) return false;
    }
}
// best (value, row) over the warp: the largest value, then the smallest row.  Values are
// non-negative floats, whose bit patterns order like the values; "no candidate" is (0, INT_MAX).
__device__ __forceinline__ void warp_best(uint32_t& vbits, uint32_t& idx) {
    const uint32_t vm = __reduce_max_sync(0xffffffffu, vbits);
    idx = __reduce_min_sync(0xffffffffu, vbits == vm ? idx : 0xffffffffu);
    vbits = vm;
}
// 1 / a by Smith's scaling, with IEEE reciprocals instead of divisions
__device__ __forceinline__ float2 cinv_rcp(float2 a) {
    if (fabsf(a.x) >= fabsf(a.y)) {
        const float r = a.y * __frcp_rn(a.x), id = __frcp_rn(fmaf(a.y, r, a.x));
        return make_float2(id, -r * id);
    }
    const float r = a.x * __frcp_rn(a.y), id = __frcp_rn(fmaf(a.x, r, a.y));
    return make_float2(r * id, -id);
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

    // Fully unrolled: c is a compile-time constant in every copy of the body, so the register
    // rows are indexed directly (a runtime c would turn each access into a chain of selects).
#pragma unroll
    for (int c = 0; c < NBP; ++c) {
        if (c >= ib) break;
        const int par = c & 1;
        const CV* uprev = ucur[par ^ 1];  // pivot row of column c-1 (valid for c > 0)
        // ---- (1) CTA-wide argmax of column c: max |Re|+|Im|, then the smallest row (warps that
        //          hold no rows keep (-1, none)) ----
        if (RPT > 1 || warp * 32 < nloc) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                Rl ov = __shfl_xor_sync(0xffffffffu, bv, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (better(ov, oi, bv, bi)) {
                    bv = ov;
                    bi = oi;
                }
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
        bool sing = !(pv > (Rl)0);
        if (pi < c || pi >= m) {  // no usable candidate (a column of NaNs): keep row c, singular
            pi = c;
            pq = 0;
            sing = true;
        }
        const CV* u = &cand_row[par][pq][0];
        const CV* drow = &diag_row[par][0];
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
        // only warps that hold rows use 1/u_c (FP64 division is long on the FP64 pipe)
        CV inv = zero;
        if (!sing && (RPT > 1 || warp * 32 < nloc)) inv = cinv(uc);
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


struct PanelShape {
    int CL, R, RPT, nbp;
    int RPW;  // > 0: lane-per-column kernel with RPW register rows per warp (C32), else the register-row kernel
    int SRW;  // lane-per-column kernel: rows per warp held in shared memory (after the register rows)
};

// cluster size, rows per CTA, rows per thread and sub-panel width for a panel of m rows.  The
// lane-per-column kernel (lane_col, C32 only) spreads the rows over as many CTAs as give each about
// 64 rows (4 per warp: the per-column update shrinks with the rows per warp), up to the cluster
// limit; it holds up to 16 rows per warp in registers and, for panels taller than that, 16 more
// per warp in shared memory (512 rows per CTA).  Taller panels use the register-row kernel.
template <class V>
bool panel_shape(int m, int cl_max, bool lane_col, PanelShape& ps) {
    if (std::is_same<V, C32>::value && lane_col) {
        const int CL = std::min(cl_max, std::max(1, ceil_div(m, 64)));
        const int need = ceil_div(ceil_div(m, CL), PANEL_THREADS / 32);  // rows per warp
        int rpw = 2;
        while (rpw < need) rpw *= 2;
        if (rpw <= 16) {
            ps = PanelShape{CL, (PANEL_THREADS / 32) * rpw, 0, 32, rpw, 0};
            return true;
        }
        if (need <= 32) {
            ps = PanelShape{CL, (PANEL_THREADS / 32) * 32, 0, 32, 16, 16};
            return true;
        }
    }
    constexpr int W = std::is_same<V, C32>::value ? 32 : 16;  // widest sub-panel (1 row per thread)
    // about 64 rows per CTA while the cluster allows (FP64 issues slowly on each SM, so short panels
    // are spread rather than kept on one CTA), one row per thread up to 512 rows per CTA
    int CL = std::min(cl_max, std::max(1, ceil_div(m, 64)));
    int R = ceil_div(m, CL);
    int RPT = ceil_div(R, PANEL_THREADS);
    if (RPT > 4) return false;
    if (RPT == 3) RPT = 4;
    ps = PanelShape{CL, R, RPT, W / RPT, 0, 0};
    return true;
}

// Lane-per-column panel of an FP32 sub-panel, rows [j0, j0 + m) x columns [j0, j0 + ib) of its big
// panel [J, J + jb).  Besides the factorisation (pivots to ipiv) it applies the sub-panel's row
// interchanges to the other columns of the big panel and solves the unit-lower block against the
// big panel's columns right of the sub-panel (U12 = L11^{-1} A12), so no separate launch is needed
// for either.  The last sub-panel of a big panel also writes the big panel's interchange map and
// applies it to the row order perm.
struct LcParams {
    C32 A;
    int j0, m, ib;
    int J, jb;
    int* ipiv;
    int* info;  // first singular column (1-based) if still 0
    int* err;   // raised by a timed-out wait
    SwapMap* map_big;
    int* perm;
};
cudaError_t launch_panel_lc(cudaStream_t s, const PanelShape& ps, const LcParams& p);

cudaError_t launch_panel(cudaStream_t s, C32 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                         int J, int jb, SwapMap* mi, SwapMap* mb, int* perm);
cudaError_t launch_panel(cudaStream_t s, Z64 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                         int J, int jb, SwapMap* mi, SwapMap* mb, int* perm);
int query_cluster_max_c32();
int query_cluster_max_z64();

}  // namespace lu_detail
