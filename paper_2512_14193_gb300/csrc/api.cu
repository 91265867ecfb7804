// C ABI of the library (include/bm.h): handle management, admission, and the orchestration of
// assembly -> factorisation -> solve -> far field on the handle's stream.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace {
thread_local std::string g_last_error;
}

void bm_set_error(const std::string& msg) { g_last_error = msg; }

extern "C" const char* bm_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* bm_strerror(bm_status s) {
    switch (s) {
        case BM_OK: return "BM_OK";
        case BM_EINVAL: return "BM_EINVAL: invalid argument";
        case BM_ENOMEM: return "BM_ENOMEM: HBM budget exceeded or allocation failed";
        case BM_ESINGULAR: return "BM_ESINGULAR: exactly zero pivot";
        case BM_ENOTCONV: return "BM_ENOTCONV: refinement did not converge";
        case BM_ENONFINITE: return "BM_ENONFINITE: non-finite input";
        case BM_ETIMEOUT: return "BM_ETIMEOUT: device wait timed out";
        case BM_ESTATE: return "BM_ESTATE: call order violated";
        case BM_ECUDA: return "BM_ECUDA: CUDA runtime error";
    }
    return "unknown bm_status";
}

// ------------------------------------------------------------------------------------------------
// allocation with budget accounting
// ------------------------------------------------------------------------------------------------
namespace {
// One stream-ordered memory pool per device for all handles of the process.  Freed blocks stay
// mapped in the pool (release threshold: unlimited), so handles that come and go - contour batches,
// serving requests - reuse memory instead of mapping it again on every allocation.  The handles'
// HBM budgets still bound what each holds.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool[dev] == nullptr) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}
}  // namespace

bm_status ctx_alloc(bm_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return BM_OK;
    if (c->held + bytes > c->budget) {
        bm_set_error("allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
        return BM_ENOMEM;
    }
    // stream-ordered allocation on the handle's stream: unlike cudaMalloc / cudaFree it never
    // waits for the rest of the device, so handles that come and go (a serving loop, contour
    // workers) do not stall each other's streams
    cudaMemPool_t pool = device_pool(c->device);
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, c->stream) : cudaMallocAsync(p, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        bm_set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        return BM_ENOMEM;
    }
    c->allocs[*p] = bytes;
    c->held += bytes;
    return BM_OK;
}

void ctx_free(bm_ctx* c, void* p) {
    if (p == nullptr) return;
    auto it = c->allocs.find(p);
    if (it != c->allocs.end()) {
        c->held -= it->second;
        c->allocs.erase(it);
    }
    cudaFreeAsync(p, c->stream);
}

namespace {

template <class T>
bm_status alloc_t(bm_ctx* c, T** p, size_t bytes) {
    void* q = nullptr;
    bm_status s = ctx_alloc(c, &q, bytes);
    *p = reinterpret_cast<T*>(q);
    return s;
}

#define FREE(ptr)              \
    do {                       \
        ctx_free(c, (ptr));    \
        (ptr) = nullptr;       \
    } while (0)

void drop_slot(bm_ctx::GraphSlot& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.kernels = 0;
}

void drop_solve_graphs(bm_ctx* c) {
    for (auto& kv : c->g_solve) drop_slot(kv.second);
    c->g_solve.clear();
    for (auto& kv : c->g_fp64) drop_slot(kv.second);
    c->g_fp64.clear();
}

void drop_graphs(bm_ctx* c) {
    drop_slot(c->g_factor);
    drop_slot(c->g_lu);
    drop_solve_graphs(c);
}

void free_solve_ws(bm_ctx* c) {
    FREE(c->d_X);
    FREE(c->d_R);
    FREE(c->d_Bw);
    FREE(c->d_Wr);
    FREE(c->d_Wi);
    FREE(c->d_W2r);
    FREE(c->d_W2i);
    FREE(c->d_Y64);
    FREE(c->d_Y64b);
    FREE(c->d_Zw64);
    FREE(c->d_Zwr);
    FREE(c->d_Zwi);
    FREE(c->d_Bx1r);
    FREE(c->d_Bx1i);
    FREE(c->d_Bx2r);
    FREE(c->d_Bx2i);
    FREE(c->d_Pkr);
    FREE(c->d_Pki);
    FREE(c->d_XP);
    FREE(c->d_XQ);
    FREE(c->d_Wdf);
    FREE(c->d_flow);
    c->flow_len = 0;
    for (int q = 0; q < 2; ++q) {
        FREE(c->d_dx[q]);
        FREE(c->d_dxe[q]);
    }
    FREE(c->d_rtw);
    c->rtw_elems = 0;
    c->pk_elems = 0;
    c->ws_nrhs = 0;
    c->last_nrhs = 0;
    drop_solve_graphs(c);
}

void free_problem(bm_ctx* c) {
    drop_graphs(c);
    free_solve_ws(c);
    FREE(c->d_geom);
    FREE(c->d_Mtop);
    FREE(c->d_Mbot);
    FREE(c->d_A);
    FREE(c->d_Ptop);
    FREE(c->d_Pbot);
    FREE(c->d_PA);
    FREE(c->d_Qtop);
    FREE(c->d_Qbot);
    FREE(c->d_QA);
    FREE(c->d_F64);
    FREE(c->d_F32r);
    FREE(c->d_F32i);
    FREE(c->d_ipiv);
    FREE(c->d_perm);
    FREE(c->d_dinvL);
    FREE(c->d_dinvU);
    FREE(c->d_Ap_r);
    FREE(c->d_Ap_i);
    FREE(c->d_Bp_r);
    FREE(c->d_Bp_i);
    FREE(c->d_Lp_r);
    FREE(c->d_Lp_i);
    FREE(c->d_Up_r);
    FREE(c->d_Up_i);
    FREE(c->d_Cp_r);
    FREE(c->d_Cp_i);
    for (int q = 0; q < 2; ++q) {
        FREE(c->d_dg[q]);
        FREE(c->d_dge[q]);
    }
    c->assembled = c->factored = c->singular = false;
    c->tm_ok = false;
    c->tc_skinny = false;
}

bool finite_c(bm_c64 z) { return std::isfinite(z.re) && std::isfinite(z.im); }
double2 d2(bm_c64 z) { return make_double2(z.re, z.im); }

long round_up(long a, long b) { return (a + b - 1) / b * b; }

Plan make_plan(int N, int form, int prec, int nb_user, int bs, int nd) {
    Plan p;
    const bool c32 = prec != BM_FP64;
    const bool split = prec == BM_CF32_3XTF32_IR;
    p.n = (form == BM_MIXED) ? N : 2 * N;
    p.nsys = (form == BM_MIXED) ? 3 * N : 2 * N;
    p.nb = nb_user > 0 ? nb_user : (c32 ? 256 : 64);
    p.ldF = pad32(p.n);
    size_t b = 7 * (size_t)N * 8;
    if (form == BM_MIXED) {
        p.ldtop = pad32(2L * N);
        p.ldbot = pad32(N);
        b += (size_t)p.ldtop * N * 16 + (size_t)p.ldbot * 2 * N * 16;
    } else {
        p.ldA = pad32(2L * N);
        b += (size_t)p.ldA * 2 * N * 16;
    }
    if (!c32) {
        b += (size_t)p.ldF * p.n * 16;
    } else {
        b += (size_t)p.ldF * p.n * 8;
        // split hi/lo planes of the FP64 operator (same size as the FP64 blocks) and of re + im
        b += (form == BM_MIXED) ? (size_t)p.ldtop * N * 24 + (size_t)p.ldbot * 2 * N * 24
                                : (size_t)p.ldA * 2 * N * 24;
        if (form == BM_MIXED) {
            p.kseg = 2 * N;
            long kext = split ? 3L * p.kseg : p.kseg;
            p.ldk_schur = round_up(kext, 32);
            b += 2 * (size_t)N * p.ldk_schur * 8;
            // [M13; M23] rows for the skinny products of the solve
            p.ldk_c = round_up(split ? 3L * N : (long)N, 32);
            b += 2 * (size_t)N * p.ldk_c * 8;
        }
        long kl = split ? 3L * p.nb : p.nb;
        p.ldk_lu = round_up(kl, 32);
        b += 2 * (size_t)p.n * p.ldk_lu * 8;
        // digit planes of the operator for the tensor-core residual, their row exponents, and the
        // row-maximum scratch of their construction
        const size_t planes = (size_t)rt_digit_planes(nd) * 2;
        if (form == BM_MIXED)
            b += planes * (2L * N * rt_ldk(N) + (size_t)N * rt_ldk(2L * N)) + 3L * N * 4 + 2L * N * 8;
        else
            b += planes * 2L * N * rt_ldk(2L * N) + 2L * N * 4 + 2L * N * 8;
    }
    p.nblk = ceil_div(p.n, bs);
    b += 2 * (size_t)p.n * 4;
    b += 2 * (size_t)p.nblk * bs * bs * (c32 ? 8 : 16);
    p.bytes = b;
    return p;
}

}  // namespace

// Device bytes one request needs: the assembled system and its factorisation, plus the solve
// workspace for nrhs right-hand sides (an estimate from the same sizes ensure_ws uses, with a
// margin for the split-K partial sums).
size_t request_bytes(int N, int form, int prec, int nb, int nrhs) {
    Plan p = make_plan(N, form, prec, nb, 64, 9);
    const size_t w = (size_t)std::max(nrhs, 8);
    size_t b = p.bytes + 7 * (size_t)N * 8 + (size_t)p.nsys * w * 16 * 3 + (size_t)p.n * w * 16 * 2;
    if (prec == BM_FP64) {
        b += (size_t)p.n * w * 16;
    } else {
        b += (size_t)p.nsys * w * 8 + (size_t)p.n * w * 16 + (size_t)p.nsys * w * 24 + 4 * (size_t)N * w * 16;
        if (form == BM_MIXED) b += 2 * w * (size_t)(p.ldk_schur + p.ldk_c) * 4 + ((size_t)64 << 20);
    }
    return b;
}

// Release the handle's system, factorisation and solve workspace (stream-ordered frees).
void ctx_release(bm_ctx* c) {
    cudaSetDevice(c->device);
    free_problem(c);
}


// ------------------------------------------------------------------------------------------------
extern "C" bm_status bm_create(bm_ctx** out, int device, void* cuda_stream, size_t hbm_budget_bytes) {
    if (out == nullptr) return BM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        bm_set_error("no CUDA device is available");
        return BM_ECUDA;
    }
    if (device < 0 || device >= ndev) return BM_EINVAL;
    BM_CUDA_TRY(cudaSetDevice(device));
    bm_ctx* c = new bm_ctx();
    c->device = device;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        c->num_sms < 1)
        c->num_sms = 1;
    if (cuda_stream) {
        c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            bm_set_error(cudaGetErrorString(e));
            return BM_ECUDA;
        }
        c->own_stream = true;
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
    int nx, ny;
    double re0, im0, step;
    hankel_anchor_host(nx, ny, re0, im0, step);
    const double2* tab = nullptr;
    bm_status s = hankel_table_device(device, &tab);
    if (s == BM_OK) s = alloc_t(c, &c->d_normA, 4 * sizeof(double));
    if (s == BM_OK) s = alloc_t(c, &c->d_info, 64 * sizeof(int));
    if (s == BM_OK) s = alloc_t(c, &c->d_maps, 3 * swap_map_bytes());
    if (s != BM_OK) {
        bm_destroy(c);
        return s;
    }
    c->d_err = c->d_info + 1;
    c->htab = HankelTable{tab, nx, ny, re0, im0, step, 1.0 / step};
    *out = c;
    return BM_OK;
}

extern "C" bm_status bm_destroy(bm_ctx* c) {
    if (c == nullptr) return BM_EINVAL;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_problem(c);
    FREE(c->d_normA);
    FREE(c->d_info);
    FREE(c->d_maps);
    if (c->la_hi) cudaStreamSynchronize(c->la_hi);
    if (c->la_lo) cudaStreamSynchronize(c->la_lo);
    for (cudaEvent_t& e : c->la_ev)
        if (e) cudaEventDestroy(e);
    if (c->la_hi) cudaStreamDestroy(c->la_hi);
    if (c->la_lo) cudaStreamDestroy(c->la_lo);
    for (auto& kv : c->allocs) cudaFreeAsync(kv.first, c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);  // the stream-ordered frees above complete
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return BM_OK;
}

extern "C" bm_status bm_enqueue_probe(bm_ctx* c, int which, int reps) {
    if (c == nullptr || reps < 1) return BM_EINVAL;
    if (!c->assembled) return BM_ESTATE;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    if (which == BM_PROBE_SCHUR) {
        if (c->form != BM_MIXED) return BM_EINVAL;
        c->factored = false;
        drop_slot(c->g_factor);
        for (int r = 0; r < reps; ++r) {
            if (c->prec == BM_FP64) {
                BM_CUDA_TRY(gemm_z64(s, c->N, c->N, 2 * c->N, -1.0, Z64{c->d_Mbot, c->ldbot}, false,
                                     Z64{c->d_Mtop, c->ldtop}, 0.0, Z64{c->d_F64, c->ldF}));
            } else {
                long kext = (c->prec == BM_CF32_3XTF32_IR) ? 3L * c->kseg_schur : c->kseg_schur;
                BM_CUDA_TRY(gemm_tc(s, c->tm_schur[0], c->tm_schur[1], c->tm_schur[2], c->tm_schur[3], c->d_F32r,
                                    c->d_F32i, c->ldF, c->N, c->N, (int)kext, -1.0f, 0.0f, c->d_err));
            }
            c->launches += 1;
        }
        return BM_OK;
    }
    if (which == BM_PROBE_RESIDUAL) {
        if (c->last_nrhs < 1) return BM_ESTATE;
        for (int r = 0; r < reps; ++r) {
            if (c->prec != BM_FP64 && c->resid_mode == BM_RESID_DF_UPDATE)
                BM_TRY(residual_df(c, c->d_Bw, c->d_X, c->d_R, c->nsys, c->last_nrhs));
            else if (c->prec != BM_FP64 && (c->resid_mode == BM_RESID_TC_UPDATE || c->resid_mode == BM_RESID_TC_ALL))
                BM_TRY(residual_tc(c, c->d_Bw, c->d_X, c->d_R, c->nsys, c->last_nrhs));
            else
                BM_TRY(residual_fp64(c, c->d_Bw, c->d_X, c->d_R, c->nsys, c->last_nrhs));
        }
        return BM_OK;
    }
    return BM_EINVAL;
}

extern "C" bm_status bm_kernel_launches(bm_ctx* c, unsigned long long* count) {
    if (c == nullptr || count == nullptr) return BM_EINVAL;
    *count = c->launches;
    return BM_OK;
}

extern "C" bm_status bm_memory(bm_ctx* c, size_t* held, size_t* budget) {
    if (c == nullptr) return BM_EINVAL;
    if (held) *held = c->held;
    if (budget) *budget = c->budget;
    return BM_OK;
}

// ------------------------------------------------------------------------------------------------
// Everything bm_assemble does; with defer_kernels the assembly kernel and what follows it (the
// zeta band, the norm, the derived packs and planes, the tensor maps) wait for assemble_post, so that
// a caller can assemble several handles' systems in one batched launch in between.
bm_status assemble_impl(bm_ctx* c, const bm_curve* curve, int N, bm_c64 k_out, bm_c64 k_in, bm_formulation form,
                        const bm_opts* opts, bool defer_kernels) {
    if (c == nullptr || curve == nullptr) return BM_EINVAL;
    if (N < 8 || N > 65536) {
        bm_set_error("N must be in [8, 65536]");
        return BM_EINVAL;
    }
    if (form != BM_MIXED && form != BM_ORDINARY) return BM_EINVAL;
    if (curve->kind < BM_CURVE_CIRCLE || curve->kind > BM_CURVE_USER) return BM_EINVAL;
    if (curve->kind == BM_CURVE_USER && curve->user == nullptr) return BM_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(curve->p[i])) return BM_ENONFINITE;
    if (!finite_c(k_out) || !finite_c(k_in)) return BM_ENONFINITE;
    const double deg = 180.0 / M_PI;
    for (bm_c64 k : {k_out, k_in}) {
        if (!(k.re > 0)) {
            bm_set_error("wavenumbers need Re k > 0");
            return BM_EINVAL;
        }
        if (std::fabs(std::atan2(k.im, k.re)) * deg > 60.0 + 1e-9 && k.im > 0) {
            bm_set_error("wavenumbers need arg k <= 60 degrees");
            return BM_EINVAL;
        }
        if (std::atan2(k.im, k.re) * deg < -89.0) {
            bm_set_error("wavenumbers need arg k > -89 degrees");
            return BM_EINVAL;
        }
    }
    if ((curve->kind == BM_CURVE_CIRCLE && !(curve->p[0] > 0)) ||
        (curve->kind == BM_CURVE_ELLIPSE && !(curve->p[0] > 0 && curve->p[1] > 0)) ||
        (curve->kind == BM_CURVE_STAR && !(curve->p[0] > std::fabs(curve->p[1]))) ||
        (curve->kind == BM_CURVE_KITE && !(curve->p[1] != 0))) {
        bm_set_error("curve parameters do not describe a simple closed curve");
        return BM_EINVAL;
    }
    int prec = opts ? opts->prec : BM_FP64;
    if (prec < BM_FP64 || prec > BM_CF32_3XTF32_IR) return BM_EINVAL;
    int nb = opts ? opts->nb : 0;
    if (opts && (opts->refine_residual < BM_RESID_TC_UPDATE || opts->refine_residual > BM_RESID_TC_ALL))
        return BM_EINVAL;
    if (opts && opts->refine_tol > 0 && opts->refine_tol < 1e-12 && opts->refine_residual != BM_RESID_FP64_ALL &&
        opts->refine_residual != BM_RESID_TC_ALL && prec != BM_FP64) {
        bm_set_error("refine_tol below 1e-12 needs refine_residual = BM_RESID_FP64_ALL or BM_RESID_TC_ALL (updated "
                     "residuals are reliable to about 1e-12)");
        return BM_EINVAL;
    }
    if (nb != 0 && (nb % 32 != 0 || nb < 32 || nb > 256)) {
        bm_set_error("nb must be a multiple of 32 in [32, 256]");
        return BM_EINVAL;
    }
    const int cl_cap = opts ? opts->panel_cluster_max : 0;
    const int pkern = opts ? opts->panel_kernel : 0;
    const bool eager = opts && opts->eager != 0;
    const int test_wait = opts ? opts->test_wait_timeout : 0;
    if (cl_cap < 0 || cl_cap > 16 || pkern < 0 || pkern > 1 || test_wait < 0 || test_wait > 2) {
        bm_set_error("panel_cluster_max must be in [0, 16], panel_kernel 0 or 1 and test_wait_timeout 0, 1 or 2");
        return BM_EINVAL;
    }
    const int zeta_p = opts ? opts->zeta_p : 0;
    if (zeta_p < 0 || zeta_p > 20 || (zeta_p > 0 && N < 2 * zeta_p + 3)) {
        bm_set_error("zeta_p must be in [0, 20] with N >= 2 zeta_p + 3");
        return BM_EINVAL;
    }
    if (zeta_p > 0) {
        // The corrections evaluate J0, J1 at k r on the stencil as (H(z) + conj H(conj z)) / 2; the
        // conjugate argument stays in the supported sector when |arg k| <= 60 degrees, or when
        // every |k r| on the stencil stays in the ascending-series zone (|z| < 3), for which any
        // argument is exact.  r is at most the arc length (zeta_p + 1) h max|x'|.
        double speed = 0.0;
        const double* q = curve->p;
        switch (curve->kind) {
            case BM_CURVE_CIRCLE: speed = std::fabs(q[0]); break;
            case BM_CURVE_ELLIPSE: speed = std::max(std::fabs(q[0]), std::fabs(q[1])); break;
            case BM_CURVE_STAR: speed = std::hypot(std::fabs(q[0]) + std::fabs(q[1]), std::fabs(q[1] * q[2])); break;
            case BM_CURVE_KITE: speed = std::hypot(1.0 + 2.0 * std::fabs(q[0]), q[1]); break;
            default:
                for (int j = 0; j < N; ++j) speed = std::max(speed, std::hypot(curve->user[6 * j + 2], curve->user[6 * j + 3]));
        }
        const double kmax = std::max(std::hypot(k_out.re, k_out.im), std::hypot(k_in.re, k_in.im));
        const double zmax = kmax * (zeta_p + 1) * (2.0 * M_PI / N) * speed;
        if (zmax >= 2.9)
            for (bm_c64 k : {k_out, k_in})
                if (std::fabs(std::atan2(k.im, k.re)) * deg > 60.0 + 1e-9) {
                    bm_set_error("the high-order zeta corrections need |arg k| <= 60 degrees here");
                    return BM_EINVAL;
                }
    }
    double eps0 = (opts && opts->eps0 != 0.0) ? opts->eps0 : 1.0;
    double2 k0 = d2(k_out), k1 = d2(k_in);
    double2 eps1, beta;
    if (opts && opts->eps_set) {
        if (!finite_c(opts->eps1)) return BM_ENONFINITE;
        eps1 = d2(opts->eps1);
    } else {
        double2 r = cdiv(k1, k0);
        eps1 = cscale(cmul(r, r), eps0);
    }
    if (opts && opts->beta_set) {
        if (!finite_c(opts->beta)) return BM_ENONFINITE;
        beta = d2(opts->beta);
    } else {
        beta = cmuli(cinv(k0));
    }

    BM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStreamSynchronize(c->stream);
    const int rmode = opts ? opts->refine_residual : BM_RESID_TC_UPDATE;
    const int nd = rmode == BM_RESID_TC_ALL ? 9 : 7;
    Plan p = make_plan(N, form, prec, nb, 64, nd);
    // Same shape as the assembled system: assemble again into the same buffers (no device
    // allocation or release - cudaFree would wait for every stream of the device - and the cached
    // graphs and tensor maps stay valid, as they depend only on these pointers and sizes).
    const bool reuse = c->assembled && c->N == N && c->form == form && c->prec == prec && c->nb == p.nb &&
                       c->rt_nd == nd && curve->kind != BM_CURVE_USER;
    if (!reuse) free_problem(c);
    // the captured factorisation depends on the launch settings: capture again when they change
    if (reuse && (eager != c->eager || cl_cap != c->opt_cluster_cap || pkern != c->opt_panel_kernel))
        drop_graphs(c);
    c->eager = eager;
    c->opt_cluster_cap = cl_cap;
    c->opt_panel_kernel = pkern;
    c->bs_solve = 64;
    if (!reuse && c->held + p.bytes > c->budget) {
        bm_set_error("admission: system needs " + std::to_string(p.bytes) + " bytes, budget leaves " +
                     std::to_string(c->budget - c->held));
        return BM_ENOMEM;
    }
    c->N = N;
    c->n = p.n;
    c->nsys = p.nsys;
    c->form = form;
    c->prec = prec;
    c->nb = p.nb;
    c->zeta_p = zeta_p;
    c->k0 = k0;
    c->k1 = k1;
    c->eps0 = make_double2(eps0, 0.0);
    c->eps1 = eps1;
    c->beta = beta;
    c->refine_tol = (opts && opts->refine_tol > 0) ? opts->refine_tol : 1e-9;
    c->refine_maxit = (opts && opts->refine_maxit > 0) ? opts->refine_maxit : 30;
    c->resid_mode = rmode;
    c->rt_nd = nd;
    c->ldtop = p.ldtop;
    c->ldbot = p.ldbot;
    c->ldA = p.ldA;
    c->ldF = p.ldF;
    c->ldk_schur = p.ldk_schur;
    c->kseg_schur = p.kseg;
    c->ldk_lu = p.ldk_lu;
    c->ldk_c = p.ldk_c;
    const bool c32 = prec != BM_FP64;
    c->assembled = c->factored = c->singular = false;
    bm_status s = BM_OK;
    if (!reuse) {
    s = alloc_t(c, &c->d_geom, 7 * (size_t)N * 8);
    if (s == BM_OK && form == BM_MIXED) {
        s = alloc_t(c, &c->d_Mtop, (size_t)p.ldtop * N * 16);
        if (s == BM_OK) s = alloc_t(c, &c->d_Mbot, (size_t)p.ldbot * 2 * N * 16);
    } else if (s == BM_OK) {
        s = alloc_t(c, &c->d_A, (size_t)p.ldA * 2 * N * 16);
    }
    if (s == BM_OK && !c32) s = alloc_t(c, &c->d_F64, (size_t)p.ldF * p.n * 16);
    if (s == BM_OK && c32) {
        if (form == BM_MIXED) {
            s = alloc_t(c, &c->d_Ptop, (size_t)p.ldtop * N * 16);
            if (s == BM_OK) s = alloc_t(c, &c->d_Pbot, (size_t)p.ldbot * 2 * N * 16);
            if (s == BM_OK) s = alloc_t(c, &c->d_Qtop, (size_t)p.ldtop * N * 8);
            if (s == BM_OK) s = alloc_t(c, &c->d_Qbot, (size_t)p.ldbot * 2 * N * 8);
        } else {
            s = alloc_t(c, &c->d_PA, (size_t)p.ldA * 2 * N * 16);
            if (s == BM_OK) s = alloc_t(c, &c->d_QA, (size_t)p.ldA * 2 * N * 8);
        }
    }
    if (s == BM_OK && c32) {
        s = alloc_t(c, &c->d_F32r, (size_t)p.ldF * p.n * 4);
        if (s == BM_OK) s = alloc_t(c, &c->d_F32i, (size_t)p.ldF * p.n * 4);
        if (s == BM_OK && form == BM_MIXED) {
            size_t pb = (size_t)N * p.ldk_schur * 4;
            if (s == BM_OK) s = alloc_t(c, &c->d_Ap_r, pb);
            if (s == BM_OK) s = alloc_t(c, &c->d_Ap_i, pb);
            if (s == BM_OK) s = alloc_t(c, &c->d_Bp_r, pb);
            if (s == BM_OK) s = alloc_t(c, &c->d_Bp_i, pb);
            size_t cb = (size_t)2 * N * p.ldk_c * 4;
            if (s == BM_OK) s = alloc_t(c, &c->d_Cp_r, cb);
            if (s == BM_OK) s = alloc_t(c, &c->d_Cp_i, cb);
        }
        size_t lb = (size_t)p.n * p.ldk_lu * 4;
        if (s == BM_OK) s = alloc_t(c, &c->d_Lp_r, lb);
        if (s == BM_OK) s = alloc_t(c, &c->d_Lp_i, lb);
        if (s == BM_OK) s = alloc_t(c, &c->d_Up_r, lb);
        if (s == BM_OK) s = alloc_t(c, &c->d_Up_i, lb);
    }
    if (s == BM_OK && c32) {
        // [0] Mtop (2N x N) or A (2N x 2N), [1] Mbot (N x 2N)
        const int np = rt_digit_planes(nd);
        const long rows0 = 2L * N, k0 = (form == BM_MIXED) ? N : 2L * N;
        c->dg_ldk[0] = rt_ldk(k0);
        s = alloc_t(c, &c->d_dg[0], (size_t)np * rows0 * c->dg_ldk[0] * 2);
        if (s == BM_OK) s = alloc_t(c, &c->d_dge[0], (size_t)rows0 * 4);
        if (s == BM_OK && form == BM_MIXED) {
            c->dg_ldk[1] = rt_ldk(2L * N);
            s = alloc_t(c, &c->d_dg[1], (size_t)np * N * c->dg_ldk[1] * 2);
            if (s == BM_OK) s = alloc_t(c, &c->d_dge[1], (size_t)N * 4);
        }
    }
    if (s == BM_OK) s = alloc_t(c, &c->d_ipiv, (size_t)p.n * 4);
    if (s == BM_OK) s = alloc_t(c, &c->d_perm, (size_t)p.n * 4);
    size_t dinv = (size_t)p.nblk * c->bs_solve * c->bs_solve * (c32 ? 8 : 16);
    if (s == BM_OK) s = alloc_t(c, &c->d_dinvL, dinv);
    if (s == BM_OK) s = alloc_t(c, &c->d_dinvU, dinv);
    if (s != BM_OK) {
        free_problem(c);
        return s;
    }
    }  // !reuse
    cudaStream_t st = c->stream;
    if (c32 && !reuse) {
        size_t lb = (size_t)p.n * p.ldk_lu * 4;
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Lp_r, 0, lb, st));
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Lp_i, 0, lb, st));
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Up_r, 0, lb, st));
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Up_i, 0, lb, st));
    }
    double* d_user = nullptr;
    if (curve->kind == BM_CURVE_USER) {
        for (long i = 0; i < 6L * N; ++i)
            if (!std::isfinite(curve->user[i])) {
                free_problem(c);
                return BM_ENONFINITE;
            }
        s = alloc_t(c, &d_user, 6 * (size_t)N * 8);
        if (s != BM_OK) {
            free_problem(c);
            return s;
        }
        BM_CUDA_TRY(cudaMemcpyAsync(d_user, curve->user, 6 * (size_t)N * 8, cudaMemcpyHostToDevice, st));
    }
    BM_CUDA_TRY(launch_geometry(st, curve->kind, curve->p, N, d_user, c->d_geom));
    c->opt_test_wait = test_wait;
    c->nd_plan = p;
    if (defer_kernels) {
        BM_CUDA_TRY(cudaStreamSynchronize(st));
        if (d_user) ctx_free(c, d_user);
        c->post_pending = true;
        return BM_OK;
    }
    bm_status sp = assemble_post(c, true, true);
    if (d_user) ctx_free(c, d_user);
    return sp;
}

extern "C" bm_status bm_assemble(bm_ctx* c, const bm_curve* curve, int N, bm_c64 k_out, bm_c64 k_in,
                                 bm_formulation form, const bm_opts* opts) {
    return assemble_impl(c, curve, N, k_out, k_in, form, opts, false);
}

// The second half of assembly: the assembly kernel (unless a batched launch already wrote the
// blocks), the zeta band, ||A||, the packs and planes the CF32 solves use, the panel set-up and the
// tensor maps.
bm_status assemble_post(bm_ctx* c, bool run_assembly_kernel, bool wait) {
    cudaStream_t st = c->stream;
    const int N = c->N, form = c->form, prec = c->prec, nd = c->rt_nd;
    const bool c32 = prec != BM_FP64;
    const Plan& p = c->nd_plan;
    bm_status s = BM_OK;
    c->post_pending = false;
    if (run_assembly_kernel) {
        BM_CUDA_TRY(launch_assemble(st, c));
        c->launches += 1;
    }
    BM_CUDA_TRY(launch_zeta_band(st, c));
    BM_CUDA_TRY(launch_normA(st, c));
    c->launches += ((form == BM_MIXED) ? 2 : 1) + (c->zeta_p > 0 ? 1 : 0);
    if (c32) {
        if (form == BM_MIXED) {
            BM_CUDA_TRY(launch_pack_solve(st, c, prec == BM_CF32_3XTF32_IR));
            BM_CUDA_TRY(launch_split_planes(st, c->d_Mtop, c->ldtop, 2 * N, N, c->d_Ptop, c->d_Qtop, c->ldtop));
            BM_CUDA_TRY(launch_split_planes(st, c->d_Mbot, c->ldbot, N, 2 * N, c->d_Pbot, c->d_Qbot, c->ldbot));
            c->launches += 3;
        } else {
            BM_CUDA_TRY(launch_split_planes(st, c->d_A, c->ldA, 2 * N, 2 * N, c->d_PA, c->d_QA, c->ldA));
            c->launches += 1;
        }
        // digit planes of the operator for the tensor-core residual
        void* rowmax = nullptr;
        s = ctx_alloc(c, &rowmax, 2L * N * 8);
        if (s != BM_OK) {
            free_problem(c);
            return s;
        }
        if (form == BM_MIXED) {
            BM_CUDA_TRY(launch_digits_a(st, c->d_Mtop, c->ldtop, 2 * N, N, c->d_dge[0], c->d_dg[0], c->dg_ldk[0], rowmax,
                                        nd));
            BM_CUDA_TRY(launch_digits_a(st, c->d_Mbot, c->ldbot, N, 2 * N, c->d_dge[1], c->d_dg[1], c->dg_ldk[1], rowmax,
                                        nd));
            c->launches += 6;
        } else {
            BM_CUDA_TRY(launch_digits_a(st, c->d_A, c->ldA, 2 * N, 2 * N, c->d_dge[0], c->d_dg[0], c->dg_ldk[0], rowmax,
                                        nd));
            c->launches += 3;
        }
        ctx_free(c, rowmax);  // stream-ordered: released once the digit kernels are done with it
    }
    BM_TRY(lu_setup(c, c->opt_cluster_cap, c->opt_panel_kernel));
    // test hook read by the tensor-core products (d_err[1], any nonzero value sets it); a memset keeps
    // the stream asynchronous (a copy from pageable memory would wait for the kernels above)
    BM_CUDA_TRY(cudaMemsetAsync(c->d_info + 2, c->opt_test_wait == 1 ? 1 : 0, sizeof(int), c->stream));
    BM_CUDA_TRY(cudaMemsetAsync(c->d_info + 3, c->opt_test_wait == 2 ? 1 : 0, sizeof(int), c->stream));
    if (wait) BM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c32) {
        const bool split = prec == BM_CF32_3XTF32_IR;
        if (form == BM_MIXED) {
            long kext = split ? 3L * p.kseg : p.kseg;
            BM_TRY(tc_make_map(c->tm_schur[0], c->d_Ap_r, N, kext, p.ldk_schur, TC_BM));
            BM_TRY(tc_make_map(c->tm_schur[1], c->d_Ap_i, N, kext, p.ldk_schur, TC_BM));
            BM_TRY(tc_make_map(c->tm_schur[2], c->d_Bp_r, N, kext, p.ldk_schur, TC_BN));
            BM_TRY(tc_make_map(c->tm_schur[3], c->d_Bp_i, N, kext, p.ldk_schur, TC_BN));
            long kext_c = split ? 3L * N : (long)N;
            BM_TRY(tc_make_map(c->tm_skinny[0], c->d_Cp_r, 2L * N, kext_c, p.ldk_c, TC_BM));
            BM_TRY(tc_make_map(c->tm_skinny[1], c->d_Cp_i, 2L * N, kext_c, p.ldk_c, TC_BM));
            c->tc_skinny = true;
        }
        {
            const long rows0 = 2L * N, k0 = (form == BM_MIXED) ? N : 2L * N;
            BM_TRY(rt_make_map(c->tm_dg[0], c->d_dg[0], rows0, k0, c->dg_ldk[0], rows0 * c->dg_ldk[0], 128, nd));
            if (form == BM_MIXED)
                BM_TRY(rt_make_map(c->tm_dg[1], c->d_dg[1], N, 2L * N, c->dg_ldk[1], (long)N * c->dg_ldk[1], 128, nd));
        }
        long klu = p.ldk_lu;
        BM_TRY(tc_make_map(c->tm_lu[0], c->d_Lp_r, p.n, klu, p.ldk_lu, TC_BM));
        BM_TRY(tc_make_map(c->tm_lu[1], c->d_Lp_i, p.n, klu, p.ldk_lu, TC_BM));
        BM_TRY(tc_make_map(c->tm_lu[2], c->d_Up_r, p.n, klu, p.ldk_lu, TC_BN));
        BM_TRY(tc_make_map(c->tm_lu[3], c->d_Up_i, p.n, klu, p.ldk_lu, TC_BN));
        if (p.n > p.nb) {  // the U12 pack from its row nb on (the look-ahead's rest of a trailing update)
            BM_TRY(tc_make_map(c->tm_lu[4], c->d_Up_r + (long)p.nb * p.ldk_lu, p.n - p.nb, klu, p.ldk_lu, TC_BN));
            BM_TRY(tc_make_map(c->tm_lu[5], c->d_Up_i + (long)p.nb * p.ldk_lu, p.n - p.nb, klu, p.ldk_lu, TC_BN));
        }
        c->tm_ok = true;
    }
    c->assembled = true;
    return BM_OK;
}

// ------------------------------------------------------------------------------------------------
namespace {

// Everything bm_factor enqueues: prepare the matrix to factor, then the LU.
bm_status factor_sequence(bm_ctx* c) {
    cudaStream_t s = c->stream;
    BM_CUDA_TRY(cudaMemsetAsync(c->d_info, 0, 2 * sizeof(int), s));
    if (c->prec == BM_FP64) {
        Z64 F{c->d_F64, c->ldF};
        if (c->form == BM_MIXED) {
            // U33 = -[M31 M32] [M13; M23]
            BM_PROF(c, "cgemm_simt_kernel<Z64> (Schur complement)");
            BM_CUDA_TRY(gemm_z64(s, c->N, c->N, 2 * c->N, -1.0, Z64{c->d_Mbot, c->ldbot}, false,
                                 Z64{c->d_Mtop, c->ldtop}, 0.0, F));
        } else {
            BM_PROF(c, "copy_z64_kernel");
            BM_CUDA_TRY(launch_copy_z64(s, c->d_A, c->ldA, c->n, c->n, c->d_F64, c->ldF));
        }
    } else {
        if (c->form == BM_MIXED) {
            // the FP32 operands of the Schur product, then U33 = -[M31 M32] [M13; M23]
            {
                BM_PROF(c, "pack_schur (pack_rowmajor/colmajor_kernel)");
                BM_CUDA_TRY(launch_pack_schur(s, c, c->prec == BM_CF32_3XTF32_IR));
            }
            long kext = (c->prec == BM_CF32_3XTF32_IR) ? 3L * c->kseg_schur : c->kseg_schur;
            BM_PROF(c, "cgemm_tc_kernel (Schur complement)");
            BM_CUDA_TRY(gemm_tc(s, c->tm_schur[0], c->tm_schur[1], c->tm_schur[2], c->tm_schur[3], c->d_F32r,
                                c->d_F32i, c->ldF, c->N, c->N, (int)kext, -1.0f, 0.0f, c->d_err));
        } else {
            BM_PROF(c, "to_c32_kernel");
            BM_CUDA_TRY(launch_to_c32(s, c->d_A, c->ldA, c->n, c->n, c->d_F32r, c->d_F32i, c->ldF));
        }
    }
    return lu_factor_enqueue(c);
}

int count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Run `fn` through a cached CUDA graph (captured on first use), or eagerly if graphs are off.
template <class Fn>
bm_status run_captured(bm_ctx* c, bm_ctx::GraphSlot* slot, Fn fn) {
    if (c->eager || c->prof) return fn();
    if (slot->exec == nullptr) {
        cudaGraph_t g = nullptr;
        BM_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        bm_status s = fn();
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (s != BM_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) {
            bm_set_error(std::string("stream capture: ") + cudaGetErrorString(e));
            return BM_ECUDA;
        }
        slot->kernels = count_kernel_nodes(g);
        // kernel nodes keep the priority of the stream they were captured from (the factorisation's
        // panel chain runs ahead of the trailing updates it overlaps)
        e = cudaGraphInstantiate(&slot->exec, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            slot->exec = nullptr;
            bm_set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
            return BM_ECUDA;
        }
    }
    BM_CUDA_TRY(cudaGraphLaunch(slot->exec, c->stream));
    c->launches += (unsigned long long)slot->kernels;
    return BM_OK;
}

}  // namespace

// The LU part of bm_factor alone (the Schur complement already in place, d_info cleared before it),
// replayed from its own graph; stream-ordered, no synchronisation.  factor_result reads the outcome.
bm_status factor_lu_enqueue(bm_ctx* c) {
    return run_captured(c, &c->g_lu, [&]() -> bm_status { return lu_factor_enqueue(c); });
}

bm_status factor_result(bm_ctx* c, int* info) {
    int h[2] = {0, 0};
    BM_CUDA_TRY(cudaMemcpyAsync(h, c->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (info) *info = h[0];
    if (h[1] != 0) {
        bm_set_error("factorisation: a bounded device-side wait timed out");
        c->factored = false;
        return BM_ETIMEOUT;
    }
    c->factored = true;
    c->singular = h[0] != 0;
    if (c->singular) {
        bm_set_error("zero pivot in column " + std::to_string(h[0]));
        return BM_ESINGULAR;
    }
    return BM_OK;
}

// Panel cluster size of an assembled handle (drops the captured factorisations).
bm_status set_panel_cluster(bm_ctx* c, int cap) {
    c->opt_cluster_cap = cap;
    drop_slot(c->g_factor);
    drop_slot(c->g_lu);
    return lu_setup(c, cap, c->opt_panel_kernel);
}

extern "C" bm_status bm_factor(bm_ctx* c, int* info) {
    if (c == nullptr) return BM_EINVAL;
    if (info) *info = 0;
    if (!c->assembled) {
        bm_set_error("bm_factor before bm_assemble");
        return BM_ESTATE;
    }
    BM_CUDA_TRY(cudaSetDevice(c->device));
    BM_TRY(run_captured(c, &c->g_factor, [&]() { return factor_sequence(c); }));
    int h[2] = {0, 0};
    BM_CUDA_TRY(cudaMemcpyAsync(h, c->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (h[1] != 0) {
        bm_set_error("factorisation: a bounded device-side wait timed out");
        c->factored = false;
        return BM_ETIMEOUT;
    }
    c->factored = true;
    c->singular = h[0] != 0;
    if (info) *info = h[0];
    if (c->singular) {
        bm_set_error("zero pivot in column " + std::to_string(h[0]));
        return BM_ESINGULAR;
    }
    return BM_OK;
}

// ------------------------------------------------------------------------------------------------
namespace {

bm_status ensure_ws(bm_ctx* c, int nrhs) {
    if (nrhs <= c->ws_nrhs) return BM_OK;
    free_solve_ws(c);
    int w = std::max(nrhs, 8);
    size_t zb = (size_t)c->nsys * w * 16;
    BM_TRY(alloc_t(c, &c->d_X, zb));
    BM_TRY(alloc_t(c, &c->d_R, zb));
    BM_TRY(alloc_t(c, &c->d_Bw, zb));
    size_t yb = (size_t)c->n * w * 16;
    BM_TRY(alloc_t(c, &c->d_Y64, yb));
    BM_TRY(alloc_t(c, &c->d_Y64b, yb));
    if (c->prec == BM_FP64) {
        BM_TRY(alloc_t(c, &c->d_Zw64, yb));
    } else {
        size_t fb = (size_t)c->nsys * w * 4;
        BM_TRY(alloc_t(c, &c->d_Wr, fb));
        BM_TRY(alloc_t(c, &c->d_Wi, fb));
        size_t vb = (size_t)c->n * w * 4;
        BM_TRY(alloc_t(c, &c->d_W2r, vb));
        BM_TRY(alloc_t(c, &c->d_W2i, vb));
        BM_TRY(alloc_t(c, &c->d_Zwr, vb));
        BM_TRY(alloc_t(c, &c->d_Zwi, vb));
        BM_TRY(alloc_t(c, &c->d_XP, (size_t)c->nsys * w * 16));
        BM_TRY(alloc_t(c, &c->d_XQ, (size_t)c->nsys * w * 8));
        BM_TRY(alloc_t(c, &c->d_Wdf, (size_t)4 * c->N * w * 16));
        // two triangles x (64-row tiles) x (8-column tiles)
        c->flow_len = 2L * ceil_div(c->n, 64) * ceil_div(w, 8);
        BM_TRY(alloc_t(c, &c->d_flow, (size_t)(c->flow_len + 1) * sizeof(int)));  // + a flag never set (test hook)
        BM_CUDA_TRY(cudaMemsetAsync(c->d_flow, 0, (size_t)(c->flow_len + 1) * sizeof(int), c->stream));
    }
    if (c->prec != BM_FP64) {
        // x digit planes and split-K workspace of the tensor-core residual
        const int N = c->N, np = rt_digit_planes(c->rt_nd);
        const int npad = (int)round_up(w, rt_col_tile(c->rt_nd));
        const int nprod = (c->form == BM_MIXED) ? 2 : 1;
        long mq[2], Kq[2];
        for (int q = 0; q < nprod; ++q) {
            // mixed: [0] rows [2N, 3N) for Mtop (K = N), [1] rows [0, 2N) for Mbot (K = 2N);
            // ordinary: [0] rows [0, 2N) for A (K = 2N)
            const long K = (c->form == BM_MIXED && q == 0) ? N : 2L * N;
            mq[q] = (c->form == BM_MIXED && q == 1) ? N : 2L * N;
            Kq[q] = K;
            c->dx_ldk[q] = rt_ldk(K);
            BM_TRY(alloc_t(c, &c->d_dx[q], (size_t)np * npad * c->dx_ldk[q] * 2));
            BM_TRY(alloc_t(c, &c->d_dxe[q], (size_t)npad * 4));
            BM_TRY(rt_make_map(c->tm_dx[q], c->d_dx[q], npad, K, c->dx_ldk[q], (long)npad * c->dx_ldk[q],
                               rt_col_tile(c->rt_nd), c->rt_nd));
        }
        // the split count depends on the number of right-hand sides: size for the largest need
        size_t wsz = 0;
        for (int r = 1; r <= w; ++r) {
            int S[2];
            rt_plan_splits(nprod, mq, Kq, r, c->rt_nd, c->num_sms, S);
            size_t t = 0;
            for (int q = 0; q < nprod; ++q)
                if (S[q] > 1) t += 2 * (size_t)S[q] * mq[q] * r;
            wsz = std::max(wsz, t);
        }
        if (wsz) BM_TRY(alloc_t(c, &c->d_rtw, wsz * 8));
        c->rtw_elems = wsz;
    }
    if (c->tc_skinny) {
        const int N = c->N;
        const bool split = c->prec == BM_CF32_3XTF32_IR;
        const long k1 = split ? 6L * N : 2L * N, k2 = split ? 3L * N : (long)N;
        BM_TRY(alloc_t(c, &c->d_Bx1r, (size_t)w * c->ldk_schur * 4));
        BM_TRY(alloc_t(c, &c->d_Bx1i, (size_t)w * c->ldk_schur * 4));
        BM_TRY(alloc_t(c, &c->d_Bx2r, (size_t)w * c->ldk_c * 4));
        BM_TRY(alloc_t(c, &c->d_Bx2i, (size_t)w * c->ldk_c * 4));
        // rows past a call's nrhs only feed output columns that are never stored; zero them anyway
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Bx1r, 0, (size_t)w * c->ldk_schur * 4, c->stream));
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Bx1i, 0, (size_t)w * c->ldk_schur * 4, c->stream));
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Bx2r, 0, (size_t)w * c->ldk_c * 4, c->stream));
        BM_CUDA_TRY(cudaMemsetAsync(c->d_Bx2i, 0, (size_t)w * c->ldk_c * 4, c->stream));
        // partial sums of the two product shapes (N x nrhs over 2N, 2N x nrhs over N) for every
        // nrhs up to w (the split count falls when nrhs crosses a tile boundary)
        size_t pe = 0;
        for (int q = 1; q <= w; ++q) {
            pe = std::max(pe, (size_t)tc_split_k(N, q, (int)k1, c->num_sms) * N * q);
            pe = std::max(pe, (size_t)tc_split_k(2 * N, q, (int)k2, c->num_sms) * 2 * N * q);
        }
        BM_TRY(alloc_t(c, &c->d_Pkr, pe * 4));
        BM_TRY(alloc_t(c, &c->d_Pki, pe * 4));
        c->pk_elems = pe;
        BM_TRY(tc_make_map(c->tm_skinny[2], c->d_Bx1r, w, k1, c->ldk_schur, TC_BN));
        BM_TRY(tc_make_map(c->tm_skinny[3], c->d_Bx1i, w, k1, c->ldk_schur, TC_BN));
        BM_TRY(tc_make_map(c->tm_skinny[4], c->d_Bx2r, w, k2, c->ldk_c, TC_BN));
        BM_TRY(tc_make_map(c->tm_skinny[5], c->d_Bx2i, w, k2, c->ldk_c, TC_BN));
    }
    c->ws_nrhs = w;
    return BM_OK;
}

bm_status read_eta(bm_ctx* c, double* eta, bool* nonfinite) {
    double h[2];
    int herr = 0;
    BM_CUDA_TRY(cudaMemcpyAsync(h, c->d_normA + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BM_CUDA_TRY(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (herr != 0) {
        bm_set_error("a bounded device wait timed out (tensor-core product or triangular solve)");
        return BM_ETIMEOUT;
    }
    *eta = h[0];
    if (nonfinite) *nonfinite = h[1] != 0.0;
    return BM_OK;
}

}  // namespace

extern "C" bm_status bm_solve(bm_ctx* c, int nrhs, const bm_c64* B, int ldb, bm_c64* X, int ldx, int on_device,
                              bm_solve_info* info) {
    if (c == nullptr) return BM_EINVAL;
    if (info) std::memset(info, 0, sizeof(*info));
    if (!c->factored || c->singular) {
        bm_set_error(c->singular ? "bm_solve on a singular factorisation" : "bm_solve before bm_factor");
        return BM_ESTATE;
    }
    if (nrhs < 1 || B == nullptr || X == nullptr || ldb < c->nsys || ldx < c->nsys) return BM_EINVAL;
    if ((const void*)B == (const void*)X) return BM_EINVAL;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    BM_TRY(ensure_ws(c, nrhs));
    c->last_nrhs = nrhs;
    cudaStream_t s = c->stream;
    const long ld = c->nsys;
    cudaEvent_t e0, e1, r0, r1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&r0);
    cudaEventCreate(&r1);
    auto cleanup = [&]() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(r0);
        cudaEventDestroy(r1);
    };
    cudaEventRecord(e0, s);
    cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t ce = cudaMemcpy2DAsync(c->d_Bw, ld * 16, B, (size_t)ldb * 16, (size_t)c->nsys * 16, nrhs, kin, s);
    if (ce != cudaSuccess) {
        cleanup();
        bm_set_error(std::string("copy of B: ") + cudaGetErrorString(ce));
        return BM_ECUDA;
    }
    double* d_eta = c->d_normA + 2;
    double eta = 0.0;
    bool nonfinite = false;
    int iters = 0;
    float t_res = 0.f;
    bm_status st = BM_OK;
    if (c->prec == BM_FP64) {
        st = run_captured(c, &c->g_fp64[nrhs], [&]() { return solve_fp64(c, c->d_Bw, c->d_X, ld, nrhs); });
        if (st == BM_OK && info) {
            cudaEventRecord(r0, s);
            st = residual_fp64(c, c->d_Bw, c->d_X, c->d_R, ld, nrhs);
            cudaEventRecord(r1, s);
            c->launches += 1;  // the backward error below (the residual counts its own)
            if (st == BM_OK) st = backward_error(c, c->d_R, c->d_X, c->d_Bw, ld, nrhs, d_eta);
            if (st == BM_OK) st = read_eta(c, &eta, &nonfinite);
            cudaEventElapsedTime(&t_res, r0, r1);
        }
    } else {
        // x0 = 0, r0 = b: the first correction is the plain FP32 solve
        cudaMemsetAsync(c->d_X, 0, (size_t)ld * nrhs * 16, s);
        cudaMemcpyAsync(c->d_R, c->d_Bw, (size_t)ld * nrhs * 16, cudaMemcpyDeviceToDevice, s);
        for (int it = 0;; ++it) {
            const bool fresh_all = c->resid_mode == BM_RESID_FP64_ALL || c->resid_mode == BM_RESID_TC_ALL;
            if (it == 1 || (it > 1 && fresh_all)) {
                // r = b - A x in FP64 or double-float (after the first correction x is the plain
                // FP32 solve)
                cudaEventRecord(r0, s);
                if (c->resid_mode == BM_RESID_DF_UPDATE)
                    st = residual_df(c, c->d_Bw, c->d_X, c->d_R, ld, nrhs);
                else if (c->resid_mode == BM_RESID_TC_UPDATE || c->resid_mode == BM_RESID_TC_ALL)
                    st = residual_tc(c, c->d_Bw, c->d_X, c->d_R, ld, nrhs);
                else
                    st = residual_fp64(c, c->d_Bw, c->d_X, c->d_R, ld, nrhs);
                cudaEventRecord(r1, s);
                if (st != BM_OK) break;
            } else if (it > 1) {
                // r -= A d for the last correction d (FP32 products; d is small by now)
                cudaEventRecord(r0, s);
                st = residual_update_c32(c, c->d_R, ld, nrhs);
                cudaEventRecord(r1, s);
                if (st != BM_OK) break;
            }
            st = backward_error(c, c->d_R, c->d_X, c->d_Bw, ld, nrhs, d_eta);
            c->launches += 1;
            if (st == BM_OK) st = read_eta(c, &eta, &nonfinite);
            if (st != BM_OK) break;
            if (it > 0) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, r0, r1);
                t_res += ms;
            }
            if (nonfinite) {
                st = BM_ENONFINITE;
                break;
            }
            if (eta <= c->refine_tol) break;
            if (it >= c->refine_maxit) {
                bm_set_error("refinement stopped at backward error " + std::to_string(eta));
                st = BM_ENOTCONV;
                break;
            }
            st = run_captured(c, &c->g_solve[nrhs], [&]() { return correction_c32(c, c->d_R, c->d_X, ld, nrhs); });
            if (st != BM_OK) break;
            ++iters;
        }
    }
    if (st == BM_OK || st == BM_ENOTCONV) {
        if (c->prec == BM_FP64 && nonfinite) st = BM_ENONFINITE;
        cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        ce = cudaMemcpy2DAsync(X, (size_t)ldx * 16, c->d_X, ld * 16, (size_t)c->nsys * 16, nrhs, kout, s);
        if (ce != cudaSuccess) {
            cleanup();
            bm_set_error(std::string("copy of X: ") + cudaGetErrorString(ce));
            return BM_ECUDA;
        }
    }
    cudaEventRecord(e1, s);
    cudaError_t se = cudaStreamSynchronize(s);
    float t_all = 0.f;
    cudaEventElapsedTime(&t_all, e0, e1);
    cleanup();
    if (se != cudaSuccess) {
        bm_set_error(std::string("solve: ") + cudaGetErrorString(se));
        return BM_ECUDA;
    }
    if (info) {
        info->iterations = iters;
        info->backward_error = eta;
        info->t_solve_ms = t_all;
        info->t_residual_ms = t_res;
    }
    return st;
}

// Corollary lem:block_LU: the block-diagonal right-hand side diag(B1, B2, B3) solved as its 3N
// columns by the Corollary lem:for_ssm_RHS path of bm_solve.
extern "C" bm_status bm_solve_block(bm_ctx* c, int c1, const bm_c64* B1, int ld1, int c2, const bm_c64* B2, int ld2,
                                    int c3, const bm_c64* B3, int ld3, bm_c64* X, int ldx, int on_device,
                                    bm_solve_info* info) {
    if (c == nullptr || X == nullptr) return BM_EINVAL;
    if (!c->assembled || c->form != BM_MIXED || !c->factored || c->singular) {
        bm_set_error("bm_solve_block needs a factored, non-singular mixed system");
        return BM_ESTATE;
    }
    const int N = c->N;
    const int cs[3] = {c1, c2, c3};
    const bm_c64* Bs[3] = {B1, B2, B3};
    const int lds[3] = {ld1, ld2, ld3};
    long C = 0;
    for (int b = 0; b < 3; ++b) {
        if (cs[b] < 0 || (cs[b] > 0 && (Bs[b] == nullptr || lds[b] < N))) return BM_EINVAL;
        C += cs[b];
    }
    if (C < 1 || C > (1 << 20) || ldx < 3 * N) return BM_EINVAL;
    const long ldb = 3L * N;
    if (!on_device) {
        std::vector<bm_c64> B((size_t)(ldb * C), bm_c64{0.0, 0.0});
        long col = 0;
        for (int b = 0; b < 3; ++b)
            for (int j = 0; j < cs[b]; ++j, ++col)
                std::memcpy(&B[(size_t)(col * ldb + (long)b * N)], Bs[b] + (size_t)j * lds[b], sizeof(bm_c64) * N);
        return bm_solve(c, (int)C, B.data(), (int)ldb, X, ldx, 0, info);
    }
    BM_CUDA_TRY(cudaSetDevice(c->device));
    bm_c64* dB = nullptr;
    bm_status s = alloc_t(c, &dB, sizeof(bm_c64) * (size_t)(ldb * C));
    if (s != BM_OK) return s;
    cudaStream_t st = c->stream;
    cudaError_t e = cudaMemsetAsync(dB, 0, sizeof(bm_c64) * (size_t)(ldb * C), st);
    long col = 0;
    for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
        if (cs[b] > 0)
            e = cudaMemcpy2DAsync(dB + col * ldb + (long)b * N, sizeof(bm_c64) * ldb, Bs[b], sizeof(bm_c64) * lds[b],
                                  sizeof(bm_c64) * N, cs[b], cudaMemcpyDeviceToDevice, st);
        col += cs[b];
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        ctx_free(c, dB);
        bm_set_error(std::string("bm_solve_block staging: ") + cudaGetErrorString(e));
        return BM_ECUDA;
    }
    s = bm_solve(c, (int)C, dB, (int)ldb, X, ldx, 1, info);
    cudaStreamSynchronize(st);
    ctx_free(c, dB);
    return s;
}

// ------------------------------------------------------------------------------------------------
extern "C" bm_status bm_rhs_plane_wave(bm_ctx* c, const double* angles, int nrhs, bm_c64* B, int ldb, int on_device) {
    if (c == nullptr || angles == nullptr || B == nullptr || nrhs < 1) return BM_EINVAL;
    if (!c->assembled) return BM_ESTATE;
    if (ldb < c->nsys) return BM_EINVAL;
    for (int i = 0; i < nrhs; ++i)
        if (!std::isfinite(angles[i])) return BM_ENONFINITE;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    double* d_ang = nullptr;
    BM_TRY(alloc_t(c, &d_ang, (size_t)nrhs * 8));
    double2* dB = nullptr;
    if (!on_device) {
        bm_status st = alloc_t(c, &dB, (size_t)c->nsys * nrhs * 16);
        if (st != BM_OK) {
            ctx_free(c, d_ang);
            return st;
        }
    }
    double2* out = on_device ? reinterpret_cast<double2*>(B) : dB;
    long ldo = on_device ? ldb : c->nsys;
    cudaMemcpyAsync(d_ang, angles, (size_t)nrhs * 8, cudaMemcpyHostToDevice, s);
    cudaError_t e = launch_plane_wave(s, c, d_ang, nrhs, out, ldo);
    c->launches += 1;
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpy2DAsync(B, (size_t)ldb * 16, dB, (size_t)c->nsys * 16, (size_t)c->nsys * 16, nrhs,
                              cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    ctx_free(c, d_ang);
    if (dB) ctx_free(c, dB);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        bm_set_error(std::string("plane wave: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return BM_ECUDA;
    }
    return BM_OK;
}

extern "C" bm_status bm_far_field(bm_ctx* c, const bm_c64* X, int ldx, int nrhs, const double* angles, int M,
                                  bm_c64* Uinf, int ldu, int on_device) {
    if (c == nullptr || X == nullptr || angles == nullptr || Uinf == nullptr || nrhs < 1 || M < 1) return BM_EINVAL;
    if (!c->assembled) return BM_ESTATE;
    if (ldx < c->nsys || ldu < M) return BM_EINVAL;
    for (int i = 0; i < M; ++i)
        if (!std::isfinite(angles[i])) {
            bm_set_error("bm_far_field: angle " + std::to_string(i) + " is not finite");
            return BM_ENONFINITE;
        }
    BM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    double* d_ang = nullptr;
    double2 *dX = nullptr, *dU = nullptr;
    bm_status st = alloc_t(c, &d_ang, (size_t)M * 8);
    if (st == BM_OK && !on_device) st = alloc_t(c, &dX, (size_t)2 * c->N * nrhs * 16);
    if (st == BM_OK && !on_device) st = alloc_t(c, &dU, (size_t)M * nrhs * 16);
    if (st != BM_OK) {
        ctx_free(c, d_ang);
        ctx_free(c, dX);
        return st;
    }
    const double2* xin = on_device ? reinterpret_cast<const double2*>(X) : dX;
    long ldxi = on_device ? ldx : 2L * c->N;
    double2* uo = on_device ? reinterpret_cast<double2*>(Uinf) : dU;
    long ldo = on_device ? ldu : M;
    cudaMemcpyAsync(d_ang, angles, (size_t)M * 8, cudaMemcpyHostToDevice, s);
    if (!on_device)
        cudaMemcpy2DAsync(dX, (size_t)2 * c->N * 16, X, (size_t)ldx * 16, (size_t)2 * c->N * 16, nrhs,
                          cudaMemcpyHostToDevice, s);
    cudaError_t e = launch_far_field(s, c, xin, ldxi, nrhs, d_ang, M, uo, ldo);
    c->launches += 1;
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpy2DAsync(Uinf, (size_t)ldu * 16, dU, (size_t)M * 16, (size_t)M * 16, nrhs,
                              cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    ctx_free(c, d_ang);
    ctx_free(c, dX);
    ctx_free(c, dU);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        bm_set_error(std::string("far field: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return BM_ECUDA;
    }
    return BM_OK;
}

extern "C" bm_status bm_copy_block(bm_ctx* c, int which, bm_c64* dst, int ldd, int on_device) {
    if (c == nullptr || dst == nullptr) return BM_EINVAL;
    if (!c->assembled) return BM_ESTATE;
    const double2* src;
    long lds;
    int rows, cols;
    const long N = c->N;
    if (c->form == BM_MIXED) {
        if (which < 0 || which > 3) return BM_EINVAL;
        rows = cols = (int)N;
        if (which == 0) {
            src = c->d_Mtop;
            lds = c->ldtop;
        } else if (which == 1) {
            src = c->d_Mtop + N;
            lds = c->ldtop;
        } else if (which == 2) {
            src = c->d_Mbot;
            lds = c->ldbot;
        } else {
            src = c->d_Mbot + N * c->ldbot;
            lds = c->ldbot;
        }
    } else {
        if (which != 0) return BM_EINVAL;
        rows = cols = (int)(2 * N);
        src = c->d_A;
        lds = c->ldA;
    }
    if (ldd < rows) return BM_EINVAL;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    BM_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)ldd * 16, src, (size_t)lds * 16, (size_t)rows * 16, cols,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    BM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BM_OK;
}

extern "C" bm_status bm_hankel01(bm_ctx* c, const bm_c64* z, int n, bm_c64* h0, bm_c64* h1, int on_device) {
    if (c == nullptr || z == nullptr || h0 == nullptr || h1 == nullptr || n < 1) return BM_EINVAL;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    double2 *dz = nullptr, *d0 = nullptr, *d1 = nullptr;
    if (!on_device) {
        bm_status st = alloc_t(c, &dz, (size_t)n * 16);
        if (st == BM_OK) st = alloc_t(c, &d0, (size_t)n * 16);
        if (st == BM_OK) st = alloc_t(c, &d1, (size_t)n * 16);
        if (st != BM_OK) {
            ctx_free(c, dz);
            ctx_free(c, d0);
            return st;
        }
        cudaMemcpyAsync(dz, z, (size_t)n * 16, cudaMemcpyHostToDevice, s);
    }
    const double2* zi = on_device ? reinterpret_cast<const double2*>(z) : dz;
    double2* o0 = on_device ? reinterpret_cast<double2*>(h0) : d0;
    double2* o1 = on_device ? reinterpret_cast<double2*>(h1) : d1;
    cudaError_t e = launch_hankel_probe(s, c, zi, n, o0, o1);
    c->launches += 1;
    if (e == cudaSuccess && !on_device) {
        cudaMemcpyAsync(h0, d0, (size_t)n * 16, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h1, d1, (size_t)n * 16, cudaMemcpyDeviceToHost, s);
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    ctx_free(c, dz);
    ctx_free(c, d0);
    ctx_free(c, d1);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        bm_set_error(std::string("hankel probe: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return BM_ECUDA;
    }
    return BM_OK;
}

extern "C" bm_status bm_f32_convert(bm_ctx* c, const double* x, int n, float* rn) {
    if (c == nullptr || x == nullptr || rn == nullptr || n < 1) return BM_EINVAL;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    double* dx = nullptr;
    float* df = nullptr;
    bm_status st = alloc_t(c, &dx, (size_t)n * 8);
    if (st == BM_OK) st = alloc_t(c, &df, (size_t)n * 4);
    if (st != BM_OK) {
        ctx_free(c, dx);
        return st;
    }
    cudaMemcpyAsync(dx, x, (size_t)n * 8, cudaMemcpyHostToDevice, s);
    cudaError_t e = launch_f32_convert(s, dx, n, df);
    c->launches += 1;
    if (e == cudaSuccess) cudaMemcpyAsync(rn, df, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    ctx_free(c, dx);
    ctx_free(c, df);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        bm_set_error(std::string("f32 convert probe: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return BM_ECUDA;
    }
    return BM_OK;
}

// ------------------------------------------------------------------------------------------------
extern "C" bm_status bm_profile(bm_ctx* c, int nrhs, const bm_c64* B, int ldb, bm_c64* X, int ldx, int on_device,
                                bm_kernel_time* out, int cap, int* count) {
    if (c == nullptr || count == nullptr || cap < 0) return BM_EINVAL;
    *count = 0;
    BM_CUDA_TRY(cudaSetDevice(c->device));
    std::vector<bm_ctx::ProfRec> recs;
    c->prof = &recs;
    int info = 0;
    bm_status st = bm_factor(c, &info);
    if (st == BM_OK) st = bm_solve(c, nrhs, B, ldb, X, ldx, on_device, nullptr);
    c->prof = nullptr;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    std::vector<std::pair<std::string, std::pair<int, double>>> groups;
    for (auto& r : recs) {
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, r.a, r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& g) { return g.first == r.name; });
        if (it == groups.end()) {
            groups.push_back({r.name, {1, (double)ms}});
        } else {
            it->second.first += 1;
            it->second.second += ms;
        }
    }
    if (st != BM_OK) return st;
    if (e != cudaSuccess) {
        bm_set_error(std::string("bm_profile: ") + cudaGetErrorString(e));
        return BM_ECUDA;
    }
    std::sort(groups.begin(), groups.end(), [](const auto& a, const auto& b) { return a.second.second > b.second.second; });
    *count = (int)groups.size();
    if (out)
        for (int i = 0; i < std::min(cap, (int)groups.size()); ++i) {
            std::memset(out[i].name, 0, sizeof(out[i].name));
            std::strncpy(out[i].name, groups[i].first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = groups[i].second.first;
            out[i].ms = groups[i].second.second;
        }
    return BM_OK;
}
