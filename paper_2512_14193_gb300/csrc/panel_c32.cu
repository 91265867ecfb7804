// Panel factorisation kernels (C32 instantiations); see lu.cu for the algorithm.
#include "lu_internal.cuh"

namespace lu_detail {
namespace {

// ------------------------------------------------------------------------------------------------
// Lane-per-column panel kernel (FP32 complex).  A sub-panel of m rows x ib <= 32 columns is held
// in registers with lane k of every warp holding column k: warp w of cluster CTA r owns the RPW
// consecutive rows starting at r R + w RPW (R = 16 RPW rows per CTA).  The column loop is a
// compact runtime loop (the register-row kernel unrolls it 32 times, which overflows the
// instruction cache).  Per column c:
//   1. every lane tracks the best row of its own column (max |Re|+|Im|, then smallest row), so
//      lane c of each warp holds the warp's candidate; the CTA's best is two warp reductions
//      (redux.sync max of the value bits, then min of the row index among the maxima);
//   2. the warp owning each CTA's candidate row stages it (lane k its column k entry) with its
//      value and index in shared memory, the owner of row c stages row c; after one CTA barrier
//      warp d sends both to cluster CTA d with st.async (the CL destinations are served by CL warps
//      at once instead of one warp in turn).  Each receiver's mbarrier for this column completes
//      when all bytes have landed (no cluster barrier, no proxy fence);
//   3. every CTA picks the pivot from the CL candidates (the same two reductions);
//   4. rows c and pivot are interchanged in the registers of their owners;
//   5. lane c stages its column (the rows' column-c entries) in shared memory and every lane
//      reads it back as broadcasts; then on the rows below c, new = alpha row + a_c beta with
//      per-lane (alpha, beta) = (1, 0) left of c, (0, 1/u_c) at c (the multiplier) and
//      (1, -u_k / u_c) right of c (the rank-1 update): no divergent branches.
// Receive buffers and mbarriers are double-buffered by column parity.  A CTA sends column c + 2
// only after it received every CTA's column c + 1 data, and each CTA sends c + 1 only after it has
// read its column c buffers, so no buffer is overwritten while still in use.  Waits are bounded (2 s by the global timer): on a
// timeout the kernel raises *err and carries on without waiting, so every CTA still reaches the
// final cluster barrier.
// ------------------------------------------------------------------------------------------------
template <int RPW>
__device__ __forceinline__ float2 row_get(const float2 (&row)[RPW], int s) {
    float2 v = row[0];
#pragma unroll
    for (int r = 1; r < RPW; ++r)
        if (r == s) v = row[r];
    return v;
}
template <int RPW>
__device__ __forceinline__ void row_set(float2 (&row)[RPW], int s, float2 v) {
#pragma unroll
    for (int r = 0; r < RPW; ++r)
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
// bounded wait for phase `parity` of a local mbarrier, with cluster-scope acquire of the data
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

template <int RPW>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
    panel_lc_kernel(C32 A, int j0, int m, int ib, int* __restrict__ ipiv, int* __restrict__ info,
                    int* __restrict__ err, int J, int jb, SwapMap* __restrict__ map_inner,
                    SwapMap* __restrict__ map_big, int* __restrict__ perm) {
    constexpr int WARPS = PANEL_THREADS / 32;
    constexpr int R = WARPS * RPW;
    constexpr int CAND = 33;  // candidate record: 32 entries, then (value bits, row index)
    cg::cluster_group cluster = cg::this_cluster();
    const int cta = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    __shared__ alignas(16) float2 cand_buf[2][MAX_CLUSTER][CAND];  // received candidates
    __shared__ alignas(16) float2 diag_buf[2][32];                  // received row c
    __shared__ alignas(16) float2 colbuf[WARPS][RPW];               // column c of each warp's rows
    __shared__ alignas(16) float2 stage_cand[CAND];                 // this CTA's candidate, to send
    __shared__ alignas(16) float2 stage_diag[32];                   // row c if this CTA owns it
    __shared__ alignas(8) uint64_t bars[2];
    __shared__ uint2 red[2][WARPS];
    __shared__ int s_map[MAP_MAX / 2 * 3 + MAP_MAX];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = cta * R;          // first panel row of this CTA
    const int wb = rb + warp * RPW;  // first panel row of this warp
    const float2 zero = make_float2(0.f, 0.f);
    const uint32_t bytes = (uint32_t)CL * (CAND * 8) + 32 * 8;  // per column, at every receiver
    bool timed_out = false;

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    float2 row[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        const int g = wb + r;
        row[r] = (g < m && lane < ib) ? A.get((long)j0 + g, (long)j0 + lane) : zero;
    }
    // candidates of every column (lane k: column k) over all rows
    float bv = -1.f;
    int bi = INT_MAX;
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        const int g = wb + r;
        const float v = (g < m) ? cnorm1(row[r]) : -1.f;
        bi = (v > bv) ? g : bi;
        bv = fmaxf(v, bv);
    }
    cluster.sync();  // mbarriers initialised and every CTA running before the first copy

#pragma unroll 1
    for (int c = 0; c < ib; ++c) {
        const int par = c & 1;
        const uint32_t bar = smem_addr(&bars[par]);
        if (threadIdx.x == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        // ---- (1) CTA candidate of column c ----
        if (lane == c) red[par][warp] = (bi != INT_MAX) ? make_uint2(__float_as_uint(bv), (uint32_t)bi)
                                                         : make_uint2(0u, (uint32_t)INT_MAX);
        __syncthreads();
        uint32_t cvb = 0u, ciu = (uint32_t)INT_MAX;
        if (lane < WARPS) {
            const uint2 e = red[par][lane];
            cvb = e.x;
            ciu = e.y;
        }
        warp_best(cvb, ciu);
        const int ci = (int)ciu;
        // ---- (2) stage the candidate row (its owner warp, else warp 0 stages zeros) and row c,
        //          then warp d sends them to cluster CTA d ----
        const bool has = ci != INT_MAX;
        if (warp == (has ? (ci - rb) / RPW : 0)) {
            stage_cand[lane] = has ? row_get<RPW>(row, ci - wb) : zero;
            if (lane == 0) stage_cand[32] = make_float2(__uint_as_float(cvb), __uint_as_float(ciu));
        }
        const bool own_diag = c >= rb && c < rb + R;  // row c lies in this CTA
        if (c >= wb && c < wb + RPW) stage_diag[lane] = row_get<RPW>(row, c - wb);
        __syncthreads();
        if (warp < CL) {
            const int d = warp;
            const uint32_t rbar = remote_addr(bar, d);
            const float2 v = stage_cand[lane];
            push8(remote_addr(smem_addr(&cand_buf[par][cta][lane]), d), __float_as_uint(v.x), __float_as_uint(v.y),
                  rbar);
            if (lane == 0) push8(remote_addr(smem_addr(&cand_buf[par][cta][32]), d), cvb, ciu, rbar);
            if (own_diag) {
                const float2 g = stage_diag[lane];
                push8(remote_addr(smem_addr(&diag_buf[par][lane]), d), __float_as_uint(g.x), __float_as_uint(g.y),
                      rbar);
            }
        }
        // ---- (3) wait for this column's data, pick the pivot ----
        if (!timed_out && !bar_wait(bar, (uint32_t)(c >> 1) & 1u)) {
            timed_out = true;
            atomicExch(err, 1);
        }
        uint32_t pvb = 0u, piu = (uint32_t)INT_MAX;
        if (lane < CL) {
            const uint2 e = reinterpret_cast<const uint2*>(&cand_buf[par][lane][32])[0];
            pvb = e.x;
            piu = e.y;
        }
        warp_best(pvb, piu);
        int pi = (int)piu;
        bool sing = !(__uint_as_float(pvb) > 0.f);
        // no usable candidate (a column of NaNs, or data lost to a timed-out wait): keep row c and
        // report the column as singular, so every index stays inside the panel
        if (pi < c || pi >= m) {
            pi = c;
            sing = true;
        }
        const int pq = pi / R;  // the CTA that owns the pivot row
        const float2 u = cand_buf[par][pq][lane];
        const float2 dr = diag_buf[par][lane];
        if (cta == 0 && threadIdx.x == 0) {
            ipiv[j0 + c] = j0 + pi;
            if (sing && info != nullptr && *info == 0) *info = j0 + c + 1;
        }
        // ---- (4) interchange rows c and pi ----
        if (!sing && pi != c) {
            if (c >= wb && c < wb + RPW) row_set<RPW>(row, c - wb, u);
            if (pi >= wb && pi < wb + RPW) row_set<RPW>(row, pi - wb, dr);
        }
        // ---- (5) new = alpha row + a_c beta on the rows below c; candidates of the next columns ----
        const float2 ucc = make_float2(__shfl_sync(0xffffffffu, u.x, c), __shfl_sync(0xffffffffu, u.y, c));
        const float2 inv = sing ? make_float2(1.f, 0.f) : cinv_rcp(ucc);
        float alpha;
        float2 beta;
        if (lane < c) {
            alpha = 1.f;
            beta = zero;
        } else if (lane == c) {
            alpha = 0.f;
            beta = inv;
        } else {
            alpha = 1.f;
            beta = cmul(make_float2(-u.x, -u.y), inv);
        }
        if (lane == c) {
#pragma unroll
            for (int r = 0; r < RPW; r += 2)
                *reinterpret_cast<float4*>(&colbuf[warp][r]) = make_float4(row[r].x, row[r].y, row[r + 1].x,
                                                                           row[r + 1].y);
        }
        __syncwarp();
        bv = -1.f;
        bi = INT_MAX;
        const int r_lo = c + 1 - wb;  // rows r >= r_lo lie below c
        const int r_hi = m - wb;      // rows r < r_hi exist
        if (r_lo <= 0 && r_hi >= RPW) {
#pragma unroll
            for (int r = 0; r < RPW; r += 2) {
                const float4 a2 = *reinterpret_cast<const float4*>(&colbuf[warp][r]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float ax = h ? a2.z : a2.x, ay = h ? a2.w : a2.y;
                    float2 t;
                    t.x = fmaf(ax, beta.x, fmaf(-ay, beta.y, alpha * row[r + h].x));
                    t.y = fmaf(ax, beta.y, fmaf(ay, beta.x, alpha * row[r + h].y));
                    row[r + h] = t;
                    const float v = cnorm1(t);
                    bi = (v > bv) ? wb + r + h : bi;
                    bv = fmaxf(v, bv);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < RPW; r += 2) {
                const float4 a2 = *reinterpret_cast<const float4*>(&colbuf[warp][r]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (r + h >= r_lo && r + h < r_hi) {
                        const float ax = h ? a2.z : a2.x, ay = h ? a2.w : a2.y;
                        float2 t;
                        t.x = fmaf(ax, beta.x, fmaf(-ay, beta.y, alpha * row[r + h].x));
                        t.y = fmaf(ax, beta.y, fmaf(ay, beta.x, alpha * row[r + h].y));
                        row[r + h] = t;
                        const float v = cnorm1(t);
                        bi = (v > bv) ? wb + r + h : bi;
                        bv = fmaxf(v, bv);
                    }
                }
            }
        }
        __syncwarp();  // colbuf is rewritten by the next column
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        const int g = wb + r;
        if (g < m && lane < ib) A.set((long)j0 + g, (long)j0 + lane, row[r]);
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
    // no CTA leaves while a copy into its shared memory could still be on the way (only possible
    // after a timed-out wait)
    cluster.sync();
}

template <int RPW>
cudaError_t launch_panel_lc_t(cudaStream_t s, C32 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv,
                              int* info, int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    auto kern = panel_lc_kernel<RPW>;
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
    return cudaLaunchKernelEx(&cfg, kern, A, j0, m, ib, ipiv, info, info + 1, J, jb, mi, mb, perm);
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


}  // namespace

cudaError_t launch_panel(cudaStream_t s, C32 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                         int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    switch (ps.RPW) {
        case 2: return launch_panel_lc_t<2>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
        case 4: return launch_panel_lc_t<4>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
        case 8: return launch_panel_lc_t<8>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
        case 16: return launch_panel_lc_t<16>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
        default: break;
    }
    if (ps.RPT == 1) return launch_panel_t<C32, 32, 1>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    if (ps.RPT == 2) return launch_panel_t<C32, 16, 2>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    return launch_panel_t<C32, 8, 4>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
}

int query_cluster_max_c32() { return query_cluster_max<C32>(); }

}  // namespace lu_detail
