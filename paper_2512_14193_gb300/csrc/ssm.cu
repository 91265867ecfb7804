// Contour eigenvalue solver: block Sakurai-Sugiura projection (Hankel form) over the discretised
// boundary integral systems, section 5.3 (sec:ssm).  The steps and their notation are stated with
// bm_ssm in bm.h.  Per contour point a worker handle assembles, factors and solves T(z_p) X = V
// on its own stream and projects P_p = V^H X (L x L); the workers run concurrently from host
// threads (the systems are independent).  Then, on the device: the moments and the two block
// Hankel matrices in one kernel (points summed in a fixed order, so the result does not depend on
// scheduling), the SVD of H and the eigenvalues of the r x r pencil with cuSOLVER (the matrices
// are at most 256 x 256), the pencil itself in two small kernels.
#include "common.cuh"
#include "kernels.cuh"

#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

// out[a + b L] = sum_r conj(V[r, a]) X[r, b]   (one block per entry, fixed reduction order)
__global__ void proj_kernel(const double2* __restrict__ V, long ldv, const double2* __restrict__ X, long ldx, int n,
                            int L, double2* __restrict__ out) {
    const int a = blockIdx.x, b = blockIdx.y;
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
        out[a + (long)b * L] = make_double2(tr, ti);
    }
}

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

struct Worker {
    bm_ctx* h = nullptr;
    double2* X = nullptr;  // nsys x L solutions
    bm_status st = BM_OK;
    std::string err;
    int max_it = 0;
    double max_eta = 0.0;
};

#define SSM_CUDA(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            bm_set_error(std::string("bm_ssm: ") + #expr + ": " + cudaGetErrorString(_e)); \
            return BM_ECUDA;                                                             \
        }                                                                                \
    } while (0)

// One contour point on one worker: assemble, factor, solve, project into slot p.
bm_status run_point(Worker& w, int p, const bm_curve* curve, int N, bm_formulation form, const bm_opts* opts,
                    const bm_ssm_opts& so, const double2* dV, long ldv, int L, double2* dPp) {
    const double th = 2.0 * kPi * (p + 0.5) / so.npoints;
    const bm_c64 z{so.center.re + so.radius * std::cos(th), so.center.im + so.radius * std::sin(th)};
    const bm_c64 zin{so.k_ratio.re * z.re - so.k_ratio.im * z.im, so.k_ratio.re * z.im + so.k_ratio.im * z.re};
    const std::string where = " (contour point " + std::to_string(p) + ")";
    bm_status st = bm_assemble(w.h, curve, N, z, zin, form, opts);
    int info = 0;
    if (st == BM_OK) st = bm_factor(w.h, &info);
    bm_solve_info si{};
    if (st == BM_OK)
        st = bm_solve(w.h, L, reinterpret_cast<const bm_c64*>(dV), (int)ldv, reinterpret_cast<bm_c64*>(w.X),
                      (int)ldv, 1, &si);
    if (st != BM_OK) {
        w.err = std::string(bm_last_error()) + where;
        return st;
    }
    w.max_it = std::max(w.max_it, si.iterations);
    w.max_eta = std::max(w.max_eta, si.backward_error);
    cudaStream_t s = w.h->stream;
    proj_kernel<<<dim3(L, L), 256, 0, s>>>(dV, ldv, w.X, ldv, w.h->nsys, L, dPp + (long)p * L * L);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        w.err = std::string("projection: ") + cudaGetErrorString(e) + where;
        return BM_ECUDA;
    }
    w.h->launches += 1;
    return BM_OK;
}

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

}  // namespace

extern "C" bm_status bm_ssm(int device, const bm_curve* curve, int N, bm_formulation form, const bm_opts* opts,
                            const bm_ssm_opts* so_in, const bm_c64* V, int ldv, int L, bm_c64* omega, int cap,
                            double* sigma, bm_ssm_info* info) {
    const auto t0 = std::chrono::steady_clock::now();
    if (info) *info = bm_ssm_info{};
    if (curve == nullptr || so_in == nullptr || V == nullptr || omega == nullptr) return BM_EINVAL;
    bm_ssm_opts so = *so_in;
    if (so.rank_tol == 0.0) so.rank_tol = 1e-8;
    if (so.workers == 0) so.workers = 4;
    const int nsys = (form == BM_MIXED) ? 3 * N : 2 * N;
    const int M = so.nmoments;
    if (!(so.radius > 0) || so.npoints < 4 || so.npoints > 4096 || M < 1 || M > 16 || L < 1 || L * M > 256 ||
        so.workers < 1 || so.workers > 16 || !(so.rank_tol > 0 && so.rank_tol < 1) || ldv < nsys || cap < L * M ||
        (form != BM_MIXED && form != BM_ORDINARY) || N < 8) {
        bm_set_error("bm_ssm: invalid argument (radius > 0, 4 <= npoints <= 4096, 1 <= M <= 16, "
                     "1 <= L, L M <= 256, 1 <= workers <= 16, 0 < rank_tol < 1, ldv >= system size, "
                     "cap >= L M)");
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
    const int W = std::min(so.workers, so.npoints);
    const int m = L * M;
    Scratch sc;
    double2 *dV = nullptr, *dPp = nullptr;
    SSM_CUDA(sc.alloc(&dV, (size_t)nsys * L * 16));
    SSM_CUDA(sc.alloc(&dPp, (size_t)so.npoints * L * L * 16));
    SSM_CUDA(cudaMemcpy2D(dV, (size_t)nsys * 16, V, (size_t)ldv * 16, (size_t)nsys * 16, L, cudaMemcpyHostToDevice));

    std::vector<Worker> ws(W);
    auto cleanup = [&]() {
        for (Worker& w : ws) {
            if (w.h) bm_destroy(w.h);
            w.h = nullptr;
        }
    };
    bm_status st = BM_OK;
    for (int i = 0; i < W && st == BM_OK; ++i) {
        st = bm_create(&ws[i].h, device, nullptr, 0);
        if (st == BM_OK && sc.alloc(&ws[i].X, (size_t)nsys * L * 16) != cudaSuccess) {
            bm_set_error("bm_ssm: cudaMalloc of a worker's solution buffer failed");
            st = BM_ENOMEM;
        }
    }
    // The first point of every worker runs here, one after another: it allocates the worker's
    // buffers and captures its graphs, which then stay in place while the workers run together.
    for (int i = 0; i < W && st == BM_OK; ++i) {
        st = run_point(ws[i], i, curve, N, form, opts, so, dV, nsys, L, dPp);
        if (st != BM_OK) bm_set_error(ws[i].err);
    }
    if (st != BM_OK) {
        cleanup();
        return st;
    }
    std::vector<std::thread> th;
    for (int i = 0; i < W; ++i)
        th.emplace_back([&, i]() {
            Worker& w = ws[i];
            if (cudaSetDevice(device) != cudaSuccess) {
                w.st = BM_ECUDA;
                w.err = "cudaSetDevice failed in a worker thread";
                return;
            }
            for (int p = i + W; p < so.npoints && w.st == BM_OK; p += W)
                w.st = run_point(w, p, curve, N, form, opts, so, dV, nsys, L, dPp);
        });
    for (auto& t : th) t.join();
    const auto t1 = std::chrono::steady_clock::now();
    int max_it = 0;
    double max_eta = 0.0;
    for (Worker& w : ws) {
        if (w.st != BM_OK && st == BM_OK) {
            st = w.st;
            bm_set_error(w.err);
        }
        max_it = std::max(max_it, w.max_it);
        max_eta = std::max(max_eta, w.max_eta);
    }
    if (st != BM_OK) {
        cleanup();
        return st;
    }
    cleanup();

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
        info->t_points_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        info->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return BM_OK;
}
