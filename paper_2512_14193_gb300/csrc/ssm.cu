// Contour eigenvalue solver: block Sakurai-Sugiura projection (Hankel form) over the discretised
// boundary integral systems, section 5.3 (sec:ssm).  The steps and their notation are stated with
// bm_ssm in bm.h.  The contour points T(z_p) X = V are independent systems of one size; they run in
// batches, a handle per point, phase by phase: one batched launch assembles every point's system, one
// batched tensor-core launch forms every point's Schur complement (CF32 precisions), each point's
// LU replays its captured graph on its own stream (all at once; the panel cluster size is chosen on
// the first batch by timing the candidates), host threads run the refined solves, and one launch
// projects P_p = V^H X_p for every point.  Then, on the device: the moments and the two block
// Hankel matrices in one kernel (points summed in a fixed order, so the result does not depend on
// scheduling), the SVD of H and the eigenvalues of the r x r pencil with cuSOLVER (the matrices
// are at most 256 x 256), the pencil itself in two small kernels.
#include "common.cuh"
#include "kernels.cuh"

#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

// mu_k[a, b] = sum_p w_p zeta_p^k P_p[a, b] for k < 2M, written into H (k = i + j) and Hs
// (k = i + j + 1); H, Hs: LM x LM column-major.  One thread per (a, b, k).
__global__ void hankel_kernel(const double2* __restrict__ Pp, int P, int L, int M, double radius,
                              double2* __restrict__ H, double2* __restrict__ Hs) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long LL = (long)L * L;
    if (idx >= LL * 2 * M) return;
    const int k = (int)(idx / LL);
    const int e = (int)(idx % LL);
    const int a = e % L, b = e / L;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < P; ++p) {
        const double th = 2.0 * kPi * (p + 0.5) / P;
        double s1, c1, sk, ck;
        sincos(th, &s1, &c1);
        sincos((double)k * th, &sk, &ck);
        // w_p zeta_p^k = (radius / P) zeta_p^(k+1)
        const double wr = radius / P * (c1 * ck - s1 * sk), wi = radius / P * (c1 * sk + s1 * ck);
        const double2 v = Pp[(long)p * LL + e];
        re += wr * v.x - wi * v.y;
        im += wr * v.y + wi * v.x;
    }
    const double2 mu = make_double2(re, im);
    const long ld = (long)L * M;
    for (int i = 0; i < M; ++i) {
        const int j = k - i;
        if (j >= 0 && j < M) H[(i * L + a) + (j * L + b) * ld] = mu;
        const int j2 = k - 1 - i;
        if (j2 >= 0 && j2 < M) Hs[(i * L + a) + (j2 * L + b) * ld] = mu;
    }
}

// T[a, j] = sum_b Hs[a, b] conj(VT[j, b]) / S[j]   (m x r; VT = W2^H, so W2[b, j] = conj(VT[j, b]))
__global__ void pencil_right_kernel(const double2* __restrict__ Hs, const double2* __restrict__ VT,
                                    const double* __restrict__ S, int m, int r, double2* __restrict__ T) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * r) return;
    const int a = idx % m, j = idx / m;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < m; ++b) {
        const double2 h = Hs[a + (long)b * m], v = VT[j + (long)b * m];
        re += h.x * v.x + h.y * v.y;  // h * conj(v)
        im += h.y * v.x - h.x * v.y;
    }
    T[a + (long)j * m] = make_double2(re / S[j], im / S[j]);
}

// B[i, j] = sum_a conj(U[a, i]) T[a, j]   (r x r)
__global__ void pencil_left_kernel(const double2* __restrict__ U, const double2* __restrict__ T, int m, int r,
                                   double2* __restrict__ B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= r * r) return;
    const int i = idx % r, j = idx / r;
    double re = 0.0, im = 0.0;
    for (int a = 0; a < m; ++a) {
        const double2 u = U[a + (long)i * m], t = T[a + (long)j * m];
        re += u.x * t.x + u.y * t.y;  // conj(u) * t
        im += u.x * t.y - u.y * t.x;
    }
    B[i + (long)j * r] = make_double2(re, im);
}

// out_b[a + b' L] = sum_r conj(V[r, a]) X_b[r, b'] for every point b of a batch (blockIdx.z),
// written to slot p0 + b of Pp (one block per entry, fixed reduction order).
__global__ void proj_batch_kernel(const double2* __restrict__ V, long ldv, const double2* const* __restrict__ Xs,
                                  long ldx, int n, int L, int p0, double2* __restrict__ Pp) {
    const int a = blockIdx.x, b = blockIdx.y, pt = blockIdx.z;
    const double2* X = Xs[pt];
    double re = 0.0, im = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 v = V[r + (long)a * ldv], x = X[r + (long)b * ldx];
        re += v.x * x.x + v.y * x.y;
        im += v.x * x.y - v.y * x.x;
    }
    __shared__ double sr[32], si[32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sr[w] = re;
        si[w] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            tr += sr[q];
            ti += si[q];
        }
        Pp[(long)(p0 + pt) * L * L + a + (long)b * L] = make_double2(tr, ti);
    }
}

#define SSM_CUDA(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            bm_set_error(std::string("bm_ssm: ") + #expr + ": " + cudaGetErrorString(_e)); \
            return BM_ECUDA;                                                             \
        }                                                                                \
    } while (0)

struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = reinterpret_cast<T*>(q);
        return e;
    }
};

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t) { return std::chrono::duration<double, std::milli>(Clock::now() - t).count(); }

// The handles of one batch of contour points and the device scratch the batched launches share.
// A batch outlives its bm_ssm call: it waits in a per-process cache for the next call with the same
// system shape, so repeated contour solves assemble into buffers that already exist (allocating
// again costs more than the assembly itself).  bm_ssm_release frees the cache.
struct Batch {
    std::vector<bm_ctx*> h;      // one handle per point of the batch
    std::vector<double2*> X;     // per handle: nsys x L solutions
    double2** dXs = nullptr;     // device copy of X (projection)
    void* d_asm = nullptr;       // assembly arguments, one per point
    void* d_tc = nullptr;        // Schur-product entries, one per point
    cudaStream_t s0 = nullptr;   // the batched launches' stream (handle 0's)
    cudaEvent_t ev = nullptr;
    std::vector<long> key;       // shape: device, N, formulation, precision options, batch, L
    int cl_tuned = 0;            // panel cluster size the autotuner picked for this shape
    double tune[3] = {0.0, 0.0, 0.0};

    void destroy() {
        if (!h.empty() && h[0]) cudaSetDevice(h[0]->device);
        for (bm_ctx*& c : h) {
            if (c) bm_destroy(c);
            c = nullptr;
        }
        for (double2* x : X)
            if (x) cudaFree(x);
        X.clear();
        if (dXs) cudaFree(dXs);
        if (d_asm) cudaFree(d_asm);
        if (d_tc) cudaFree(d_tc);
        if (ev) cudaEventDestroy(ev);
        dXs = nullptr;
        d_asm = d_tc = nullptr;
        ev = nullptr;
    }
};

std::mutex g_cache_mu;
std::vector<Batch*> g_cache;  // idle batches

Batch* take_cached(const std::vector<long>& key) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (size_t i = 0; i < g_cache.size(); ++i)
        if (g_cache[i]->key == key) {
            Batch* b = g_cache[i];
            g_cache.erase(g_cache.begin() + i);
            return b;
        }
    return nullptr;
}

void give_cached(Batch* b) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (size_t i = 0; i < g_cache.size(); ++i)
        if (g_cache[i]->key == b->key) {  // keep the newer batch of a shape
            g_cache[i]->destroy();
            delete g_cache[i];
            g_cache.erase(g_cache.begin() + i);
            break;
        }
    g_cache.push_back(b);
}

// Factor phase of a batch: the Schur complements (batched tensor-core product for the CF32
// precisions, FP64 product per point otherwise), then every point's LU from its captured graph
// on its own stream, all at once.
bm_status factor_batch(Batch& bt, int B) {
    bm_ctx* c0 = bt.h[0];
    const int N = c0->N;
    // the pivot / timeout words of every point, cleared ahead of everything that may set them
    for (int b = 0; b < B; ++b) SSM_CUDA(cudaMemsetAsync(bt.h[b]->d_info, 0, 2 * sizeof(int), bt.s0));
    SSM_CUDA(cudaEventRecord(bt.ev, bt.s0));
    for (int b = 0; b < B; ++b) SSM_CUDA(cudaStreamWaitEvent(bt.h[b]->stream, bt.ev, 0));
    if (c0->form == BM_MIXED && c0->prec != BM_FP64) {
        std::vector<const void*> maps(B);
        std::vector<float*> Cr(B), Ci(B);
        std::vector<long> ld(B);
        for (int b = 0; b < B; ++b) {
            bm_ctx* c = bt.h[b];
            SSM_CUDA(launch_pack_schur(bt.s0, c, c->prec == BM_CF32_3XTF32_IR));
            maps[b] = c->tm_schur;
            Cr[b] = c->d_F32r;
            Ci[b] = c->d_F32i;
            ld[b] = c->ldF;
        }
        const long kext = (c0->prec == BM_CF32_3XTF32_IR) ? 3L * c0->kseg_schur : c0->kseg_schur;
        SSM_CUDA(gemm_tc_batch(bt.s0, B, maps.data(), Cr.data(), Ci.data(), ld.data(), N, N, (int)kext, -1.0f, bt.d_tc,
                               c0->d_err));
        c0->launches += 3 * B + 1;
        SSM_CUDA(cudaEventRecord(bt.ev, bt.s0));
        for (int b = 0; b < B; ++b) SSM_CUDA(cudaStreamWaitEvent(bt.h[b]->stream, bt.ev, 0));
    } else {
        for (int b = 0; b < B; ++b) {
            bm_ctx* c = bt.h[b];
            if (c->form == BM_MIXED) {
                SSM_CUDA(gemm_z64(c->stream, N, N, 2 * N, -1.0, Z64{c->d_Mbot, c->ldbot}, false, Z64{c->d_Mtop, c->ldtop},
                                  0.0, Z64{c->d_F64, c->ldF}));
            } else if (c->prec == BM_FP64) {
                SSM_CUDA(launch_copy_z64(c->stream, c->d_A, c->ldA, c->n, c->n, c->d_F64, c->ldF));
            } else {
                SSM_CUDA(launch_to_c32(c->stream, c->d_A, c->ldA, c->n, c->n, c->d_F32r, c->d_F32i, c->ldF));
            }
            c->launches += 1;
        }
    }
    for (int b = 0; b < B; ++b) BM_TRY(factor_lu_enqueue(bt.h[b]));
    for (int b = 0; b < B; ++b) {
        int info = 0;
        bm_status st = factor_result(bt.h[b], &info);
        if (st != BM_OK) return st;
    }
    return BM_OK;
}

}  // namespace

extern "C" bm_status bm_ssm(int device, const bm_curve* curve, int N, bm_formulation form, const bm_opts* opts,
                            const bm_ssm_opts* so_in, const bm_c64* V, int ldv, int L, bm_c64* omega, int cap,
                            double* sigma, bm_ssm_info* info) {
    const auto t0 = Clock::now();
    if (info) *info = bm_ssm_info{};
    if (curve == nullptr || so_in == nullptr || V == nullptr || omega == nullptr) return BM_EINVAL;
    bm_ssm_opts so = *so_in;
    if (so.rank_tol == 0.0) so.rank_tol = 1e-8;
    if (so.workers == 0) so.workers = 16;
    if (so.batch == 0) so.batch = std::min(so.npoints, 32);
    const int nsys = (form == BM_MIXED) ? 3 * N : 2 * N;
    const int M = so.nmoments;
    if (!(so.radius > 0) || so.npoints < 4 || so.npoints > 4096 || M < 1 || M > 16 || L < 1 || L * M > 256 ||
        so.workers < 1 || so.workers > 64 || so.batch < 1 || so.batch > 64 || so.panel_cluster < 0 ||
        so.panel_cluster > 16 || !(so.rank_tol > 0 && so.rank_tol < 1) || ldv < nsys || cap < L * M ||
        (form != BM_MIXED && form != BM_ORDINARY) || N < 8) {
        bm_set_error("bm_ssm: invalid argument (radius > 0, 4 <= npoints <= 4096, 1 <= M <= 16, "
                     "1 <= L, L M <= 256, 1 <= workers <= 64, 1 <= batch <= 64, 0 <= panel_cluster <= 16, "
                     "0 < rank_tol < 1, ldv >= system size, cap >= L M)");
        return BM_EINVAL;
    }
    if (opts && (opts->zeta_p < 0 || opts->zeta_p > 20 || (opts->zeta_p > 0 && N < 2 * opts->zeta_p + 3))) {
        bm_set_error("bm_ssm: zeta_p must be in [0, 20] with N >= 2 zeta_p + 3");
        return BM_EINVAL;
    }
    if (!std::isfinite(so.center.re) || !std::isfinite(so.center.im) || !std::isfinite(so.k_ratio.re) ||
        !std::isfinite(so.k_ratio.im))
        return BM_ENONFINITE;
    for (long c = 0; c < L; ++c)
        for (long r = 0; r < nsys; ++r) {
            const bm_c64 v = V[r + c * ldv];
            if (!std::isfinite(v.re) || !std::isfinite(v.im)) return BM_ENONFINITE;
        }
    SSM_CUDA(cudaSetDevice(device));
    const int B = std::min(so.batch, so.npoints);
    const int m = L * M;
    Scratch sc;
    double2 *dV = nullptr, *dPp = nullptr;
    SSM_CUDA(sc.alloc(&dV, (size_t)nsys * L * 16));
    SSM_CUDA(sc.alloc(&dPp, (size_t)so.npoints * L * L * 16));
    SSM_CUDA(cudaMemcpy2D(dV, (size_t)nsys * 16, V, (size_t)ldv * 16, (size_t)nsys * 16, L, cudaMemcpyHostToDevice));

    const bm_opts o0 = opts ? *opts : bm_opts{};
    const std::vector<long> key = {device, N, (long)form, (long)o0.prec, (long)o0.nb, (long)o0.zeta_p,
                                   (long)o0.refine_residual, (long)B, (long)L, (long)o0.eager, (long)o0.panel_kernel};
    Batch* bp = take_cached(key);
    bool fresh = bp == nullptr;
    if (fresh) {
        bp = new Batch();
        bp->key = key;
    }
    Batch& bt = *bp;
    auto cleanup = [&]() {
        bt.destroy();
        delete bp;
    };
    bm_status st = BM_OK;
    if (fresh) {
        bt.h.assign(B, nullptr);
        bt.X.assign(B, nullptr);
        for (int b = 0; b < B && st == BM_OK; ++b) {
            st = bm_create(&bt.h[b], device, nullptr, 0);
            if (st == BM_OK && cudaMalloc(&bt.X[b], (size_t)nsys * L * 16) != cudaSuccess) {
                bm_set_error("bm_ssm: cudaMalloc of a point's solution buffer failed");
                st = BM_ENOMEM;
            }
        }
        if (st == BM_OK && (cudaMalloc(&bt.dXs, (size_t)B * sizeof(double2*)) != cudaSuccess ||
                            cudaMalloc(&bt.d_asm, (size_t)B * asm_args_bytes()) != cudaSuccess ||
                            cudaMalloc(&bt.d_tc, (size_t)B * tc_batch_entry_bytes()) != cudaSuccess ||
                            cudaEventCreateWithFlags(&bt.ev, cudaEventDisableTiming) != cudaSuccess)) {
            bm_set_error("bm_ssm: batch scratch allocation failed");
            st = BM_ENOMEM;
        }
        if (st != BM_OK) {
            cudaGetLastError();
            cleanup();
            return st;
        }
        bt.s0 = bt.h[0]->stream;
        SSM_CUDA(cudaMemcpy(bt.dXs, bt.X.data(), (size_t)B * sizeof(double2*), cudaMemcpyHostToDevice));
    }

    double t_asm = 0.0, t_fac = 0.0, t_sol = 0.0, tune[3] = {0.0, 0.0, 0.0};
    // a cached batch remembers the autotuner's pick for its shape; the points are assembled with the
    // cluster size in their options, so a reused handle keeps its captured graphs
    int cl_used = so.panel_cluster != 0 ? so.panel_cluster : bt.cl_tuned;
    bm_opts po = o0;
    po.panel_cluster_max = cl_used;
    int max_it = 0;
    double max_eta = 0.0;
    for (int p0 = 0; p0 < so.npoints && st == BM_OK; p0 += B) {
        const int nb = std::min(B, so.npoints - p0);
        // ---- assembly: per point set-up, one batched launch, per point derived data ----
        auto ta = Clock::now();
        for (int b = 0; b < nb && st == BM_OK; ++b) {
            const int p = p0 + b;
            const double th = 2.0 * kPi * (p + 0.5) / so.npoints;
            const bm_c64 z{so.center.re + so.radius * std::cos(th), so.center.im + so.radius * std::sin(th)};
            const bm_c64 zin{so.k_ratio.re * z.re - so.k_ratio.im * z.im, so.k_ratio.re * z.im + so.k_ratio.im * z.re};
            st = assemble_impl(bt.h[b], curve, N, z, zin, form, &po, true);
            if (st != BM_OK) bm_set_error(std::string(bm_last_error()) + " (contour point " + std::to_string(p) + ")");
        }
        if (st != BM_OK) break;
        {
            cudaError_t e = launch_assemble_batch(bt.s0, bt.h.data(), nb, bt.d_asm);
            if (e == cudaSuccess) e = cudaStreamSynchronize(bt.s0);
            if (e != cudaSuccess) {
                bm_set_error(std::string("bm_ssm: batched assembly: ") + cudaGetErrorString(e));
                st = BM_ECUDA;
                break;
            }
            bt.h[0]->launches += 1;
        }
        // every point's derived data on its own stream at once, then one wait for them all
        for (int b = 0; b < nb && st == BM_OK; ++b) st = assemble_post(bt.h[b], false, false);
        for (int b = 0; b < nb && st == BM_OK; ++b)
            if (cudaStreamSynchronize(bt.h[b]->stream) != cudaSuccess) {
                bm_set_error("bm_ssm: assembly of a contour point failed");
                st = BM_ECUDA;
            }
        if (st != BM_OK) break;
        t_asm += ms_since(ta);
        // ---- factorisation (the first batch picks the panel cluster size when asked to) ----
        auto tf = Clock::now();
        if (cl_used == 0) {
            const int cands[3] = {16, 8, 4};
            double best = 1e300;
            for (int q = 0; q < 3 && st == BM_OK; ++q) {
                for (int b = 0; b < nb && st == BM_OK; ++b) st = set_panel_cluster(bt.h[b], cands[q]);
                if (st != BM_OK) break;
                // first run captures the graphs; the second is timed
                st = factor_batch(bt, nb);
                auto tq = Clock::now();
                if (st == BM_OK) st = factor_batch(bt, nb);
                tune[q] = ms_since(tq);
                if (tune[q] < best) {
                    best = tune[q];
                    cl_used = cands[q];
                }
            }
            if (st != BM_OK) break;
            for (int b = 0; b < nb && st == BM_OK; ++b) st = set_panel_cluster(bt.h[b], cl_used);
            bt.cl_tuned = cl_used;
            po.panel_cluster_max = cl_used;
            for (int q = 0; q < 3; ++q) bt.tune[q] = tune[q];
            tf = Clock::now();
        }
        if (st == BM_OK) st = factor_batch(bt, nb);
        if (st != BM_OK) {
            bm_set_error(std::string(bm_last_error()) + " (contour points " + std::to_string(p0) + ".." +
                         std::to_string(p0 + nb - 1) + ")");
            break;
        }
        t_fac += ms_since(tf);
        // ---- refined solves, `workers` host threads over the points ----
        auto ts = Clock::now();
        const int W = std::min(so.workers, nb);
        std::vector<bm_status> pst(nb, BM_OK);
        std::vector<bm_solve_info> pinfo(nb);
        std::vector<std::string> perr(nb);
        std::vector<std::thread> th;
        for (int w = 0; w < W; ++w)
            th.emplace_back([&, w]() {
                if (cudaSetDevice(device) != cudaSuccess) {
                    for (int b = w; b < nb; b += W) pst[b] = BM_ECUDA;
                    return;
                }
                for (int b = w; b < nb; b += W) {
                    pst[b] = bm_solve(bt.h[b], L, reinterpret_cast<const bm_c64*>(dV), nsys,
                                      reinterpret_cast<bm_c64*>(bt.X[b]), nsys, 1, &pinfo[b]);
                    if (pst[b] != BM_OK) perr[b] = bm_last_error();
                }
            });
        for (auto& t : th) t.join();
        for (int b = 0; b < nb; ++b) {
            if (pst[b] != BM_OK && st == BM_OK) {
                st = pst[b];
                bm_set_error(perr[b] + " (contour point " + std::to_string(p0 + b) + ")");
            }
            max_it = std::max(max_it, pinfo[b].iterations);
            max_eta = std::max(max_eta, pinfo[b].backward_error);
        }
        if (st != BM_OK) break;
        // ---- projection of every point of the batch, one launch ----
        proj_batch_kernel<<<dim3(L, L, nb), 256, 0, bt.s0>>>(dV, nsys, bt.dXs, nsys, nsys, L, p0, dPp);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(bt.s0);
        if (e != cudaSuccess) {
            bm_set_error(std::string("bm_ssm: projection: ") + cudaGetErrorString(e));
            st = BM_ECUDA;
            break;
        }
        bt.h[0]->launches += 1;
        t_sol += ms_since(ts);
    }
    const double t_points = ms_since(t0);
    if (st != BM_OK) {
        cleanup();
        return st;
    }
    give_cached(bp);

    // ---- moments, Hankel matrices, SVD, pencil, eigenvalues ----
    double2 *dH = nullptr, *dHs = nullptr, *dU = nullptr, *dVT = nullptr, *dT = nullptr, *dB = nullptr,
            *dW = nullptr;
    double *dS = nullptr, *dRw = nullptr;
    int* dInfo = nullptr;
    SSM_CUDA(sc.alloc(&dH, (size_t)m * m * 16));
    SSM_CUDA(sc.alloc(&dHs, (size_t)m * m * 16));
    SSM_CUDA(sc.alloc(&dU, (size_t)m * m * 16));
    SSM_CUDA(sc.alloc(&dVT, (size_t)m * m * 16));
    SSM_CUDA(sc.alloc(&dT, (size_t)m * m * 16));
    SSM_CUDA(sc.alloc(&dB, (size_t)m * m * 16));
    SSM_CUDA(sc.alloc(&dW, (size_t)m * 16));
    SSM_CUDA(sc.alloc(&dS, (size_t)m * 8));
    SSM_CUDA(sc.alloc(&dRw, (size_t)m * 8));
    SSM_CUDA(sc.alloc(&dInfo, sizeof(int)));
    const long nthr = (long)L * L * 2 * M;
    hankel_kernel<<<ceil_div(nthr, 128L), 128>>>(dPp, so.npoints, L, M, so.radius, dH, dHs);
    SSM_CUDA(cudaGetLastError());

    cusolverDnHandle_t hs = nullptr;
    cusolverDnParams_t prm = nullptr;
    auto solver_fail = [&](const char* what, int code) {
        if (prm) cusolverDnDestroyParams(prm);
        if (hs) cusolverDnDestroy(hs);
        bm_set_error(std::string("bm_ssm: ") + what + " returned " + std::to_string(code));
        return BM_ECUDA;
    };
    cusolverStatus_t cs = cusolverDnCreate(&hs);
    if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail("cusolverDnCreate", (int)cs);
    int lwork = 0;
    cs = cusolverDnZgesvd_bufferSize(hs, m, m, &lwork);
    if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail("cusolverDnZgesvd_bufferSize", (int)cs);
    cuDoubleComplex* dWork = nullptr;
    if (sc.alloc(&dWork, (size_t)std::max(lwork, 1) * 16) != cudaSuccess) return solver_fail("workspace", 0);
    cs = cusolverDnZgesvd(hs, 'A', 'A', m, m, reinterpret_cast<cuDoubleComplex*>(dH), m, dS,
                          reinterpret_cast<cuDoubleComplex*>(dU), m, reinterpret_cast<cuDoubleComplex*>(dVT), m, dWork,
                          lwork, dRw, dInfo);
    if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail("cusolverDnZgesvd", (int)cs);
    std::vector<double> S(m);
    int hinfo = 0;
    SSM_CUDA(cudaMemcpy(S.data(), dS, (size_t)m * 8, cudaMemcpyDeviceToHost));
    SSM_CUDA(cudaMemcpy(&hinfo, dInfo, sizeof(int), cudaMemcpyDeviceToHost));
    if (hinfo != 0) return solver_fail("cusolverDnZgesvd (info)", hinfo);
    int r = 0;
    while (r < m && S[r] > so.rank_tol * S[0]) ++r;
    if (sigma) std::copy(S.begin(), S.end(), sigma);
    std::vector<double2> zeta(r);
    if (r > 0) {
        pencil_right_kernel<<<ceil_div((long)m * r, 128L), 128>>>(dHs, dVT, dS, m, r, dT);
        pencil_left_kernel<<<ceil_div((long)r * r, 128L), 128>>>(dU, dT, m, r, dB);
        SSM_CUDA(cudaGetLastError());
        cs = cusolverDnCreateParams(&prm);
        if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail("cusolverDnCreateParams", (int)cs);
        size_t dws = 0, hws = 0;
        cs = cusolverDnXgeev_bufferSize(hs, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_NOVECTOR, r, CUDA_C_64F,
                                        dB, r, CUDA_C_64F, dW, CUDA_C_64F, nullptr, 1, CUDA_C_64F, nullptr, 1,
                                        CUDA_C_64F, &dws, &hws);
        if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail("cusolverDnXgeev_bufferSize", (int)cs);
        void* dGw = nullptr;
        if (sc.alloc(&dGw, std::max<size_t>(dws, 16)) != cudaSuccess) return solver_fail("workspace", 0);
        std::vector<unsigned char> hGw(std::max<size_t>(hws, 16));
        cs = cusolverDnXgeev(hs, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_NOVECTOR, r, CUDA_C_64F, dB, r,
                             CUDA_C_64F, dW, CUDA_C_64F, nullptr, 1, CUDA_C_64F, nullptr, 1, CUDA_C_64F, dGw, dws,
                             hGw.data(), hws, dInfo);
        if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail("cusolverDnXgeev", (int)cs);
        SSM_CUDA(cudaMemcpy(zeta.data(), dW, (size_t)r * 16, cudaMemcpyDeviceToHost));
        SSM_CUDA(cudaMemcpy(&hinfo, dInfo, sizeof(int), cudaMemcpyDeviceToHost));
        if (hinfo != 0) return solver_fail("cusolverDnXgeev (info)", hinfo);
    }
    if (prm) cusolverDnDestroyParams(prm);
    cusolverDnDestroy(hs);
    // omega = center + radius zeta: inside first, each group by real part
    std::vector<std::pair<int, bm_c64>> out;
    for (const double2& zv : zeta) {
        const bool in = std::hypot(zv.x, zv.y) < 1.0;
        out.push_back({in ? 0 : 1, bm_c64{so.center.re + so.radius * zv.x, so.center.im + so.radius * zv.y}});
    }
    std::sort(out.begin(), out.end(), [](const auto& a, const auto& b) {
        if (a.first != b.first) return a.first < b.first;
        if (a.second.re != b.second.re) return a.second.re < b.second.re;
        return a.second.im < b.second.im;
    });
    int nin = 0;
    for (int i = 0; i < r; ++i) {
        omega[i] = out[i].second;
        nin += out[i].first == 0;
    }
    if (info) {
        info->rank = r;
        info->n_inside = nin;
        info->max_iterations = max_it;
        info->max_backward_error = max_eta;
        info->t_points_ms = t_points;
        info->t_total_ms = ms_since(t0);
        info->t_assemble_ms = t_asm;
        info->t_factor_ms = t_fac;
        info->t_solve_ms = t_sol;
        info->batch = B;
        info->panel_cluster = cl_used;
        for (int q = 0; q < 3; ++q) info->tune_ms[q] = tune[q] != 0.0 ? tune[q] : bt.tune[q];
    }
    return BM_OK;
}

extern "C" bm_status bm_ssm_release(int device) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (size_t i = 0; i < g_cache.size();) {
        if (device < 0 || g_cache[i]->key[0] == device) {
            g_cache[i]->destroy();
            delete g_cache[i];
            g_cache.erase(g_cache.begin() + i);
        } else {
            ++i;
        }
    }
    return BM_OK;
}
