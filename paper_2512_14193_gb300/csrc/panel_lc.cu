// Lane-per-column LU panel of the FP32 factorisation (partial pivoting, Thm thm:LU's LU of U33 and
// the ordinary system's LU), one thread-block cluster per sub-panel of m rows x ib <= 32 columns.
//
// Layout.  Lane k of every warp holds column k.  Warp w of cluster CTA r owns RPW consecutive rows
// in registers, starting at r R + w RPW (R = 16 (RPW + SRW) rows per CTA), and, for panels taller
// than 16 rows per warp, SRW more rows in shared memory after the CTA's register rows.  The CTA's
// rows are read and written through shared memory in coalesced column segments.
//
// Per column c:
//   1. every lane tracks the best row of its own column (max |Re|+|Im|, then the smallest row), so
//      lane c of each warp holds the warp's candidate; every warp stages its candidate row, the
//      owner of row c stages row c;
//   2. after one CTA barrier, warp d picks the CTA's best of the warps' candidates (two warp
//      reductions) and sends it with row c to cluster CTA d with st.async, which completes on the
//      receiver's mbarrier for this column (buffers double-buffered by column parity);
//   3. every CTA picks the pivot from the CL candidates with the same reductions;
//   4. rows c and pivot are interchanged where they live;
//   5. new = alpha row + a_c beta on the rows below c, with per-lane (alpha, beta) = (1, 0) left of
//      c, (0, 1/u_c) at c (the multiplier) and (1, -u_k / u_c) right of c (the rank-1 update), in
//      packed two-wide FP32 arithmetic, a_c broadcast from lane c by shuffles; the same pass finds
//      the candidates of the next column.
// A CTA sends column c + 2 only after it received every CTA's column c + 1 data, and each CTA sends
// c + 1 only after it has read its column c buffers, so no buffer is overwritten while in use.
// Waits are bounded (2 s): on a timeout the kernel raises *err and carries on without waiting.
//
// After the columns: the panel is stored, every CTA derives the sub-panel's net row interchange
// from the pivots it saw, and the cluster's warps apply it to the big panel's other columns and
// solve L11 against the columns right of the sub-panel.
#include "lu_internal.cuh"

namespace lu_detail {
namespace {

using u64 = unsigned long long;

// packed pairs of FP32 values (the f32x2 instructions of sm_100 and later)
__device__ __forceinline__ u64 pk2(float x, float y) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 up2(u64 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// 1 / a for a != 0: a is scaled by a power of two (exact) to |a|_inf in [1, 2), and
// conj(a) / |a|^2 uses one hardware reciprocal refined by a Newton step (a few ulps, no overflow or
// underflow for any finite a).
__device__ __forceinline__ float2 cinv_fast(float2 a) {
    const float s = fmaxf(fabsf(a.x), fabsf(a.y));
    const int eb = min(max((int)((__float_as_uint(s) >> 23) & 0xff), 1), 253);  // biased exponent
    const float sc = __uint_as_float((uint32_t)(254 - eb) << 23);                  // 2^-(eb - 127)
    const float x = a.x * sc, y = a.y * sc;
    const float d = fmaf(x, x, y * y);
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    r = r * fmaf(-d, r, 2.f);
    const float rs = r * sc;
    return make_float2(x * rs, -y * rs);
}

// ------------------------------------------------------------------------------------------------
// Net effect of the interchanges (a_k <-> p_k), k = 0 .. nk-1 in order, with a_k = base + k and
// p_k >= a_k: the map new[dst] = old[src] over the rows they touch.  Row a_k is never touched after
// step k, and row p_k before step k only by earlier steps with the same p, so with
//   prevA(k) = last k' < k with p_k' = a_k,   prevB(k) = last k' < k with p_k' = p_k,
//   val(k)   = content of row a_k just before step k = val(prevA(k)), or a_k if there is none,
// slot a_k ends with val(prevB(k)) (or p_k's own row if prevB(k) does not exist), and a row
// x >= base + nk that occurs as some p_k ends with val(k) of its last occurrence.  The chains of
// val are resolved by pointer jumping.  Entries 0 .. nk-1 of the map are the slots a_k in order,
// then the rows below them.
// ------------------------------------------------------------------------------------------------

// one warp, nk <= 32, rows relative to the sub-panel (base 0); dst/src hold up to 64 entries
__device__ __forceinline__ int submap_warp(const int* piv, int nk, int* dst, int* src) {
    const int lane = threadIdx.x & 31;
    const bool valid = lane < nk;
    const int a = lane, p = valid ? piv[lane] : -1;
    int prevA = -1, prevB = -1;
    bool last = true;
    for (int t = 0; t < nk; ++t) {
        const int q = __shfl_sync(0xffffffffu, p, t);
        if (t < lane) {
            prevA = (q == a) ? t : prevA;
            prevB = (q == p) ? t : prevB;
        } else if (t > lane && q == p) {
            last = false;
        }
    }
    int v = a, ptr = prevA;
#pragma unroll
    for (int r = 0; r < 6; ++r) {  // chains of at most 32 steps
        const int src_lane = ptr >= 0 ? ptr : lane;
        const int pv = __shfl_sync(0xffffffffu, v, src_lane);
        const int pp = __shfl_sync(0xffffffffu, ptr, src_lane);
        if (ptr >= 0) {
            v = pv;
            ptr = pp;
        }
    }
    const int fin = __shfl_sync(0xffffffffu, v, prevB >= 0 ? prevB : lane);
    if (valid) {
        dst[lane] = a;
        src[lane] = prevB >= 0 ? fin : p;
    }
    const bool extra = valid && p >= nk && last;
    const unsigned em = __ballot_sync(0xffffffffu, extra);
    if (extra) {
        const int e = nk + __popc(em & ((1u << lane) - 1u));
        dst[e] = p;
        src[e] = v;
    }
    return nk + __popc(em);
}

// the whole CTA (at least nk threads), nk <= 256, absolute rows (a_k = base + k); writes the map
// to global memory and returns its entry count to every thread.  Scratch: 7 * 256 ints.
__device__ int bigmap_cta(const int* piv, int base, int nk, SwapMap* out, int* scr) {
    int* P = scr;             // p_k
    int* V0 = scr + 256;      // val (pointer jumping, two buffers)
    int* V1 = scr + 512;
    int* Q0 = scr + 768;      // pointers
    int* Q1 = scr + 1024;
    int* wcnt = scr + 1280;   // extras per warp
    const int k = threadIdx.x;
    const bool valid = k < nk;
    int p = -1, prevA = -1, prevB = -1;
    bool last = true;
    if (valid) P[k] = p = piv[k];
    __syncthreads();
    if (valid) {
        const int a = base + k;
        for (int t = 0; t < nk; ++t) {
            const int q = P[t];
            if (t < k) {
                prevA = (q == a) ? t : prevA;
                prevB = (q == p) ? t : prevB;
            } else if (t > k && q == p) {
                last = false;
            }
        }
        V0[k] = a;
        Q0[k] = prevA;
    }
    __syncthreads();
    int* Vc = V0;
    int* Qc = Q0;
    int* Vn = V1;
    int* Qn = Q1;
    for (int r = 0; r < 9; ++r) {  // chains of at most 256 steps
        if (valid) {
            const int q = Qc[k];
            Vn[k] = q >= 0 ? Vc[q] : Vc[k];
            Qn[k] = q >= 0 ? Qc[q] : -1;
        }
        __syncthreads();
        int* t = Vc;
        Vc = Vn;
        Vn = t;
        t = Qc;
        Qc = Qn;
        Qn = t;
    }
    const bool extra = valid && p >= base + nk && last;
    const unsigned em = __ballot_sync(0xffffffffu, extra);
    const int lane = k & 31, w = k >> 5;
    if (lane == 0) wcnt[w] = __popc(em);
    if (valid) {
        out->dst[k] = base + k;
        out->src[k] = prevB >= 0 ? Vc[prevB] : p;
    }
    __syncthreads();
    int off = nk, tot = nk;
    const int nw = (int)(blockDim.x >> 5);
    for (int q = 0; q < nw; ++q) {
        if (q < w) off += wcnt[q];
        tot += wcnt[q];
    }
    if (extra) {
        const int e = off + __popc(em & ((1u << lane) - 1u));
        out->dst[e] = p;
        out->src[e] = Vc[k];
    }
    if (k == 0) out->count = tot;
    return tot;
}


constexpr int LDS = 33;  // row stride (complex entries) of the shared-memory staging of a CTA's rows

template <int RPW, int SRW>
__global__ void __launch_bounds__(PANEL_THREADS, 1) panel_lc_kernel(const __grid_constant__ LcParams P) {
    constexpr int WARPS = PANEL_THREADS / 32;
    constexpr int RR = WARPS * RPW;          // rows of a CTA in registers
    constexpr int R = WARPS * (RPW + SRW);   // rows of a CTA
    constexpr int CAND = 33;                 // candidate record: 32 entries, then (value bits, row index)
    extern __shared__ __align__(16) float2 stg[];  // R x LDS: staging of the CTA's rows; shared-memory rows
    __shared__ alignas(16) float2 cand_buf[2][MAX_CLUSTER][CAND];  // received candidates
    __shared__ alignas(16) float2 diag_buf[2][32];                  // received row c
    __shared__ alignas(16) float2 wst[2][WARPS][32];                // each warp's candidate row
    __shared__ alignas(16) float2 stage_diag[32];                   // row c if this CTA owns it
    __shared__ alignas(8) uint64_t bars[2];
    __shared__ uint2 red[2][WARPS];
    __shared__ int piv_s[32];         // pivot rows of the sub-panel, relative to j0
    __shared__ int sm_dst[64], sm_src[64], sm_cnt;
    __shared__ alignas(16) float2 L11s[32][LDS];
    __shared__ int scr[7 * 256];

    cg::cluster_group cluster = cg::this_cluster();
    const int cta = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const C32 A = P.A;
    const int j0 = P.j0, m = P.m, ib = P.ib;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = cta * R;          // first panel row of this CTA
    const int wb = rb + warp * RPW;  // first register row of this warp
    const int sb = RR + warp * SRW;  // first shared-memory row of this warp (CTA-local)
    const float2 zero = make_float2(0.f, 0.f);
    const uint32_t bytes = (uint32_t)CL * (CAND * 8) + 32 * 8;  // per column, at every receiver
    bool timed_out = false;

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the cluster barrier that guards the first remote copy is entered now and left after the
    // load, which hides the CTAs' different start times
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    // launched as a programmatic dependent: the previous kernel of the stream has finished and its
    // writes are visible after this wait; the next kernel may start launching (it waits likewise)
    pdl_wait();
    pdl_trigger();

    // ---- load the CTA's rows: column segments of R rows, coalesced, through shared memory ----
    {
        constexpr int PER = R * 32 / PANEL_THREADS;
        const long row0 = (long)j0 + rb;
#pragma unroll 8
        for (int q = 0; q < PER; ++q) {
            const int e = (int)threadIdx.x + q * PANEL_THREADS;
            const int lr = e % R, k = e / R;
            float2 v = zero;
            if (rb + lr < m && k < ib) {
                const long off = row0 + lr + (long)(j0 + k) * A.ld;
                v = make_float2(A.re[off], A.im[off]);
            }
            stg[lr * LDS + k] = v;
        }
    }
    __syncthreads();
    u64 row[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        const float2 v = stg[(warp * RPW + r) * LDS + lane];
        row[r] = pk2(v.x, v.y);
    }
    // candidates of every column (lane k: column k) over the warp's rows, in increasing row order
    float bv = -1.f;
    int bi = INT_MAX;
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        const float v = (wb + r < m) ? cnorm1(up2(row[r])) : -1.f;
        bi = (v > bv) ? wb + r : bi;
        bv = fmaxf(v, bv);
    }
#pragma unroll
    for (int s = 0; s < SRW; ++s) {
        const int g = rb + sb + s;
        const float v = (g < m) ? cnorm1(stg[(sb + s) * LDS + lane]) : -1.f;
        bi = (v > bv) ? g : bi;
        bv = fmaxf(v, bv);
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");

#pragma unroll 1
    for (int c = 0; c < ib; ++c) {
        const int par = c & 1;
        const uint32_t bar = smem_addr(&bars[par]);
        if (threadIdx.x == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        // ---- (1) every warp stages its candidate row of column c (lane c holds the warp's best;
        //          lane k writes the row's column-k entry) and row c's owner stages row c ----
        const uint32_t wvb = __shfl_sync(0xffffffffu, bi != INT_MAX ? __float_as_uint(bv) : 0u, c);
        const int wi = __shfl_sync(0xffffffffu, bi, c);
        {
            float2 v = zero;
            if (wi != INT_MAX) {
                const int lr = wi - rb;  // one of this warp's rows
                if (lr < RR) v = up2(row_get(row, lr - warp * RPW));
                else v = stg[lr * LDS + lane];
            }
            wst[par][warp][lane] = v;
            if (lane == 0) red[par][warp] = make_uint2(wvb, (uint32_t)wi);
        }
        const bool own_diag = cta == 0;  // row c < 32 <= RR lies in CTA 0's registers
        if (own_diag && warp == c / RPW) stage_diag[lane] = up2(row_get(row, c - warp * RPW));
        __syncthreads();
        // ---- (2) warp d picks the CTA's candidate among the warps' and sends it, with row c, to
        //          cluster CTA d ----
        if (warp < CL) {
            uint32_t cvb = 0u, ciu = (uint32_t)INT_MAX;
            if (lane < WARPS) {
                const uint2 e = red[par][lane];
                cvb = e.x;
                ciu = e.y;
            }
            warp_best(cvb, ciu);
            int ws = 0;  // the warp that staged it
            if (ciu != (uint32_t)INT_MAX) {
                const int lr = (int)ciu - rb;
                ws = lr < RR ? lr / RPW : (lr - RR) / (SRW > 0 ? SRW : 1);
            }
            const int d = warp;
            const uint32_t rbar = remote_addr(bar, d);
            const float2 v = wst[par][ws][lane];
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
            atomicExch(P.err, 1);
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
        if (threadIdx.x == 0) piv_s[c] = pi;
        if (cta == 0 && threadIdx.x == 0 && sing && P.info != nullptr && *P.info == 0) *P.info = j0 + c + 1;
        // ---- (4) interchange rows c and pi ----
        if (!sing && pi != c) {
            if (own_diag && warp == c / RPW) row_set(row, c - warp * RPW, pk2(u.x, u.y));
            if (pq == cta) {
                const int plr = pi - rb;
                if (plr < RR) {
                    if (warp == plr / RPW) row_set(row, plr - warp * RPW, pk2(dr.x, dr.y));
                } else if constexpr (SRW > 0) {
                    if (warp == (plr - RR) / SRW) stg[plr * LDS + lane] = dr;
                }
            }
        }
        // ---- (5) new = alpha row + a_c beta on the rows below c; candidates of the next columns ----
        const float2 ucc = make_float2(__shfl_sync(0xffffffffu, u.x, c), __shfl_sync(0xffffffffu, u.y, c));
        const float2 inv = sing ? make_float2(1.f, 0.f) : cinv_fast(ucc);
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
        const u64 al2 = pk2(alpha, alpha), b1 = pk2(beta.x, beta.y), b2 = pk2(-beta.y, beta.x);
        bv = -1.f;
        bi = INT_MAX;
        const int r_lo = c + 1 - wb;  // register rows r >= r_lo lie below c
        const int r_hi = m - wb;      // register rows r < r_hi exist
        if (r_lo <= 0 && r_hi >= RPW) {
#pragma unroll
            for (int r = 0; r < RPW; ++r) {
                const float2 a = up2(row[r]);  // the row's column-c entry, from lane c
                const float ax = __shfl_sync(0xffffffffu, a.x, c), ay = __shfl_sync(0xffffffffu, a.y, c);
                u64 t = mul2(al2, row[r]);
                t = fma2(pk2(ax, ax), b1, t);
                t = fma2(pk2(ay, ay), b2, t);
                row[r] = t;
                const float v = cnorm1(up2(t));
                bi = (v > bv) ? wb + r : bi;
                bv = fmaxf(v, bv);
            }
        } else {
#pragma unroll
            for (int r = 0; r < RPW; ++r) {
                if (r >= r_lo && r < r_hi) {
                    const float2 a = up2(row[r]);
                    const float ax = __shfl_sync(0xffffffffu, a.x, c), ay = __shfl_sync(0xffffffffu, a.y, c);
                    u64 t = mul2(al2, row[r]);
                    t = fma2(pk2(ax, ax), b1, t);
                    t = fma2(pk2(ay, ay), b2, t);
                    row[r] = t;
                    const float v = cnorm1(up2(t));
                    bi = (v > bv) ? wb + r : bi;
                    bv = fmaxf(v, bv);
                }
            }
        }
        if constexpr (SRW > 0) {
            // shared-memory rows: the column-c entry is read by every lane (a broadcast) before
            // lane c overwrites it with the multiplier
#pragma unroll 4
            for (int s = 0; s < SRW; ++s) {
                const int lr = sb + s, g = rb + lr;
                if (g > c && g < m) {
                    const float2 a = stg[lr * LDS + c];
                    const float2 x = stg[lr * LDS + lane];
                    u64 t = mul2(al2, pk2(x.x, x.y));
                    t = fma2(pk2(a.x, a.x), b1, t);
                    t = fma2(pk2(a.y, a.y), b2, t);
                    const float2 tv = up2(t);
                    __syncwarp();
                    stg[lr * LDS + lane] = tv;
                    const float v = cnorm1(tv);
                    bi = (v > bv) ? g : bi;
                    bv = fmaxf(v, bv);
                }
            }
        }
    }

    // ---- store the CTA's rows (coalesced, through shared memory) and the pivots ----
#pragma unroll
    for (int r = 0; r < RPW; ++r) stg[(warp * RPW + r) * LDS + lane] = up2(row[r]);
    __syncthreads();
    {
        constexpr int PER = R * 32 / PANEL_THREADS;
        const long row0 = (long)j0 + rb;
#pragma unroll 8
        for (int q = 0; q < PER; ++q) {
            const int e = (int)threadIdx.x + q * PANEL_THREADS;
            const int lr = e % R, k = e / R;
            if (rb + lr < m && k < ib) {
                const long off = row0 + lr + (long)(j0 + k) * A.ld;
                const float2 v = stg[lr * LDS + k];
                A.re[off] = v.x;
                A.im[off] = v.y;
            }
        }
    }
    if (cta == 0 && (int)threadIdx.x < ib) P.ipiv[j0 + threadIdx.x] = j0 + piv_s[threadIdx.x];
    // every CTA's stores are ordered before the cluster barrier's release; the tail reads L11
    // after its acquire.  No copy into this CTA's shared memory is on the way past this point.
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    const int nleft = j0 - P.J;                 // big-panel columns left of the sub-panel
    const int nright = P.J + P.jb - (j0 + ib);  // and right of it
    if (nleft + nright > 0 && warp == 0) sm_cnt = submap_warp(piv_s, ib, sm_dst, sm_src);
    if (cta == 0 && P.map_big != nullptr && nright == 0) {
        // the big panel's map from the pivots of its sub-panels (this one's from shared memory)
        __syncthreads();
        if ((int)threadIdx.x < P.jb)
            scr[1536 + threadIdx.x] = (int)threadIdx.x < nleft ? P.ipiv[P.J + threadIdx.x]
                                                              : j0 + piv_s[threadIdx.x - nleft];
        __syncthreads();
        const int cnt = bigmap_cta(scr + 1536, P.J, P.jb, P.map_big, scr);
        __syncthreads();
        if (P.perm != nullptr) {
            int v = 0;
            const int t = (int)threadIdx.x;
            if (t < cnt) v = P.perm[P.map_big->src[t]];
            __syncthreads();
            if (t < cnt) P.perm[P.map_big->dst[t]] = v;
        }
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (nleft + nright == 0) return;

    // ---- the sub-panel's interchanges on the big panel's other columns; L11^{-1} on the right ----
    if (nright > 0) {
        for (int e = threadIdx.x; e < 32 * 32; e += PANEL_THREADS) {
            const int i = e % 32, k = e / 32;
            L11s[i][k] = (i > k && i < ib) ? A.get((long)j0 + i, (long)j0 + k) : zero;
        }
    }
    __syncthreads();
    const int cnt = sm_cnt;
    const int sd0 = lane < cnt ? sm_dst[lane] : 0, ss0 = lane < cnt ? sm_src[lane] : 0;
    const int sd1 = lane + 32 < cnt ? sm_dst[lane + 32] : 0, ss1 = lane + 32 < cnt ? sm_src[lane + 32] : 0;
    for (int t = cta * WARPS + warp; t < nleft + nright; t += CL * WARPS) {
        const bool right = t >= nleft;
        const long col = right ? (long)j0 + ib + (t - nleft) : (long)P.J + t;
        float2 x0 = zero, x1 = zero;
        if (lane < cnt) x0 = A.get((long)j0 + ss0, col);
        if (lane + 32 < cnt) x1 = A.get((long)j0 + ss1, col);
        if (right) {  // entries 0 .. ib-1 are rows j0 + lane: x0 -= L11 x below the diagonal
            // (L11s is zero on and above the diagonal and beyond ib, so every lane takes every step)
#pragma unroll
            for (int k = 0; k < 31; ++k) {
                const float2 l = L11s[lane][k];
                const float2 xk = make_float2(__shfl_sync(0xffffffffu, x0.x, k), __shfl_sync(0xffffffffu, x0.y, k));
                x0.x = fmaf(-l.x, xk.x, fmaf(l.y, xk.y, x0.x));
                x0.y = fmaf(-l.x, xk.y, fmaf(-l.y, xk.x, x0.y));
            }
        }
        __syncwarp();  // every source is read before any destination is written
        if (lane < cnt) A.set((long)j0 + sd0, col, x0);
        if (lane + 32 < cnt) A.set((long)j0 + sd1, col, x1);
    }
}

template <int RPW, int SRW>
cudaError_t launch_lc_t(cudaStream_t s, const PanelShape& ps, const LcParams& p) {
    auto kern = panel_lc_kernel<RPW, SRW>;
    const int smem = (PANEL_THREADS / 32) * (RPW + SRW) * LDS * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && ps.CL > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ps.CL, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ps.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace

cudaError_t launch_panel_lc(cudaStream_t s, const PanelShape& ps, const LcParams& p) {
    if (p.ib < 1 || p.ib > 32 || p.m < p.ib || ps.CL < 1 || ps.CL > MAX_CLUSTER ||
        (long)ps.CL * PANEL_THREADS / 32 * (ps.RPW + ps.SRW) < p.m || p.jb > MAP_MAX / 2)
        return cudaErrorInvalidValue;
    if (ps.SRW == 16 && ps.RPW == 16) return launch_lc_t<16, 16>(s, ps, p);
    if (ps.SRW != 0) return cudaErrorInvalidValue;
    switch (ps.RPW) {
        case 2: return launch_lc_t<2, 0>(s, ps, p);
        case 4: return launch_lc_t<4, 0>(s, ps, p);
        case 8: return launch_lc_t<8, 0>(s, ps, p);
        case 16: return launch_lc_t<16, 0>(s, ps, p);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lu_detail
