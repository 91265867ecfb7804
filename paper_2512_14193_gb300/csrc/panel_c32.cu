// Panel factorisation kernels (C32 instantiations); see lu.cu for the algorithm.
#include "lu_internal.cuh"

namespace lu_detail {
namespace {

// ------------------------------------------------------------------------------------------------
// Lane-per-column panel kernel (FP32 complex).  A sub-panel of m rows x ib <= 32 columns is held
// in registers with lane k of every warp holding column k: warp w of cluster CTA r owns the RPW
// consecutive rows starting at r R + w RPW (R = 16 RPW rows per CTA).  Column c of a row is then
// one warp shuffle away from every lane, so the column loop needs no per-column code copies (the
// register-row kernel unrolls it 32 times, which overflows the instruction cache) and no select
// chains over the row's registers.  Per column c:
//   1. every lane tracks the best row of its own column (max |Re|+|Im|, then smallest row), so
//      lane c of each warp holds the warp's candidate; the CTA's best comes from 16 shared entries;
//   2. each CTA pushes its candidate row with its value and index, and the owner of row c pushes
//      row c, into every CTA of the cluster with st.async; each receiver's mbarrier for this
//      column completes when all bytes have landed (no cluster barrier, no fence);
//   3. every CTA picks the pivot from the CL candidates;
//   4. rows c and pivot are interchanged in the registers of their owners;
//   5. rows below c: new = alpha row + a_c beta, with a_c the row's column-c entry (a shuffle) and
//      per-lane (alpha, beta) = (1, 0) left of c, (0, 1/u_c) at c (the multiplier), and
//      (1, -u_k / u_c) right of c (the rank-1 update): no divergent branches.
// Receive buffers and mbarriers are double-buffered by column parity.  A CTA pushes column c + 2
// only after it received every CTA's column c + 1 push, and each CTA pushes c + 1 only after it
// has read its column c buffers, so a buffer is never overwritten while still in use.  Waits are
// bounded (2 s by the global timer): on a timeout the kernel raises *err and carries on without
// waiting, so every CTA still reaches the final cluster barrier.
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
// 8 bytes into another CTA's shared memory, completing on that CTA's mbarrier
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
// bounded wait for phase `parity` of a local mbarrier, with cluster-scope acquire of the pushed data
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

template <int RPW>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
    panel_lc_kernel(C32 A, int j0, int m, int ib, int* __restrict__ ipiv, int* __restrict__ info,
                    int* __restrict__ err, int J, int jb, SwapMap* __restrict__ map_inner,
                    SwapMap* __restrict__ map_big, int* __restrict__ perm) {
    constexpr int WARPS = PANEL_THREADS / 32;
    constexpr int R = WARPS * RPW;
    cg::cluster_group cluster = cg::this_cluster();
    const int cta = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    __shared__ float2 cand_row[2][MAX_CLUSTER][32];
    __shared__ float2 diag_row[2][32];
    __shared__ uint2 cand_vi[2][MAX_CLUSTER];  // (value bits, row index)
    __shared__ alignas(8) uint64_t bars[2];
    __shared__ float red_val[2][WARPS];
    __shared__ int red_idx[2][WARPS];
    __shared__ int s_map[MAP_MAX / 2 * 3 + MAP_MAX];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = cta * R;          // first panel row of this CTA
    const int wb = rb + warp * RPW;  // first panel row of this warp
    const float2 zero = make_float2(0.f, 0.f);
    const uint32_t bytes = (uint32_t)CL * (32 * 8 + 8) + 32 * 8;  // per column, at every receiver
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
    cluster.sync();  // mbarriers initialised and every CTA running before the first push

#pragma unroll 1
    for (int c = 0; c < ib; ++c) {
        const int par = c & 1;
        const uint32_t bar = smem_addr(&bars[par]);
        if (threadIdx.x == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        // ---- (1) CTA candidate of column c ----
        if (lane == c) {
            red_val[par][warp] = bv;
            red_idx[par][warp] = bi;
        }
        __syncthreads();
        float cv = (lane < WARPS) ? red_val[par][lane] : -1.f;
        int ci = (lane < WARPS) ? red_idx[par][lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, cv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
            if (better(ov, oi, cv, ci)) {
                cv = ov;
                ci = oi;
            }
        }
        // ---- (2) push: candidate row (its owner warp, else warp 0 sends zeros) and row c ----
        const bool has = ci != INT_MAX;
        const int owner = has ? (ci - rb) / RPW : 0;
        if (warp == owner) {
            const float2 v = has ? row_get<RPW>(row, ci - wb) : zero;
            const uint32_t la = smem_addr(&cand_row[par][cta][lane]);
            for (int d = 0; d < CL; ++d)
                push8(remote_addr(la, d), __float_as_uint(v.x), __float_as_uint(v.y), remote_addr(bar, d));
            if (lane < CL)
                push8(remote_addr(smem_addr(&cand_vi[par][cta]), lane), __float_as_uint(has ? cv : -1.f), (uint32_t)ci,
                      remote_addr(bar, lane));
        }
        if (c >= wb && c < wb + RPW) {
            const float2 v = row_get<RPW>(row, c - wb);
            const uint32_t la = smem_addr(&diag_row[par][lane]);
            for (int d = 0; d < CL; ++d)
                push8(remote_addr(la, d), __float_as_uint(v.x), __float_as_uint(v.y), remote_addr(bar, d));
        }
        // ---- (3) wait for every push of this column, pick the pivot ----
        if (!timed_out && !bar_wait(bar, (uint32_t)(c >> 1) & 1u)) {
            timed_out = true;
            atomicExch(err, 1);
        }
        float pv = -1.f;
        int pi = INT_MAX;
        if (lane < CL) {
            const uint2 e = cand_vi[par][lane];
            pv = __uint_as_float(e.x);
            pi = (int)e.y;
        }
        int pq = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, pv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, pi, o);
            const int oq = __shfl_xor_sync(0xffffffffu, pq, o);
            if (better(ov, oi, pv, pi)) {
                pv = ov;
                pi = oi;
                pq = oq;
            }
        }
        const float2 u = cand_row[par][pq][lane];
        const float2 dr = diag_row[par][lane];
        const bool sing = !(pv > 0.f);
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
        const float2 inv = sing ? make_float2(1.f, 0.f) : cinv(ucc);
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
        bv = -1.f;
        bi = INT_MAX;
        const int r_lo = c + 1 - wb;  // rows r >= r_lo lie below c
        const int r_hi = m - wb;      // rows r < r_hi exist
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            if (r >= r_lo && r < r_hi) {  // uniform across the warp
                const float ax = __shfl_sync(0xffffffffu, row[r].x, c);
                const float ay = __shfl_sync(0xffffffffu, row[r].y, c);
                float2 t;
                t.x = fmaf(ax, beta.x, fmaf(-ay, beta.y, alpha * row[r].x));
                t.y = fmaf(ax, beta.y, fmaf(ay, beta.x, alpha * row[r].y));
                row[r] = t;
                const float v = cnorm1(t);
                bi = (v > bv) ? wb + r : bi;
                bv = fmaxf(v, bv);
            }
        }
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
    // no CTA leaves while a push into its shared memory could still be on the way (only possible
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
