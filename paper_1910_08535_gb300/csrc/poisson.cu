// Multi-D Poisson solve (Sec. 4.3 problem -Lap u = f, zero Dirichlet rows).
//
// The tested operator K = sum_a (-C_a) (x) A_others (rows off the boundary;
// identity rows on it) is not a Kronecker product, so the 1D banded
// factorisations of the mass solve do not invert it.  Its interior block is
// K_II = sum_a L_a (x) A_others with L = -C restricted to the unknowns, and
// every 1D pencil (L_a, A_a) has a real spectrum with well-conditioned
// eigenvectors (both for B-spline and for piece-wise constant tests):
//   A_a^{-1} L_a = V_a Lambda_a V_a^{-1}.
// With W_a = V_a^{-1} A_a^{-1},
//   K_II^{-1} = (V_x (x) V_y (x) V_z) diag(1 / (lx + ly + lz)) (W_x (x) W_y (x) W_z),
// i.e. d dense per-axis transforms, a diagonal scaling and d more transforms:
// dense GEMMs over the coefficient tensor -- by default the library's tcgen05
// tensor-core kernel in split TF32 (tcgemm.cuh), or cuBLAS FP32 / BF16x9 by
// flag -- with a fused diagonal kernel.  The transforms run in FP32; the operator P = diag(I, K_II^{-1}) they
// form is applied inside iterative refinement whose residual b - K u is taken
// by the contraction kernel in FP64 or double-float arithmetic: one correction
// for pair tensors (FP32 + refinement), `iters` corrections for FP64 tensors.
// Boundary rows: P copies the residual, so the boundary values and the
// coupling K_IB they induce are settled by the refinement itself.
//
// Set-up (once per context): the 1D pencils are factored and diagonalised in
// FP64 with cuSOLVER (LU, nonsymmetric eigensolver), then stored as FP32
// matrices embedded in the axis' full index range.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <list>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "contract.cuh"
#include "poisson.h"
#include "tcgemm.cuh"

namespace igapw {

// ---- contraction instantiations for K u and b - K u (2D and 3D) -------------
template <int DIM, int W>
static cudaError_t poisson_mode(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st) {
    if (mode == MODE_PK) {
        if (io == FMT_F64) return pick_tile<DIM, W, double, MODE_PK, FMT_F64>(a, st);
        return pick_tile<DIM, W, DF, MODE_PK, FMT_PAIR>(a, st);
    }
    if (io == FMT_F64) return pick_tile<DIM, W, double, MODE_PRES, FMT_F64>(a, st);
    if (cmp == FMT_F64) return pick_tile<DIM, W, double, MODE_PRES, FMT_PAIR>(a, st);
    return pick_tile<DIM, W, DF, MODE_PRES, FMT_PAIR>(a, st);
}

template <int DIM>
static cudaError_t poisson_w(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st) {
    switch (a.W) {
        case 3: return poisson_mode<DIM, 3>(a, mode, cmp, io, st);
        case 5: return poisson_mode<DIM, 5>(a, mode, cmp, io, st);
        case 7: return poisson_mode<DIM, 7>(a, mode, cmp, io, st);
        case 9: return poisson_mode<DIM, 9>(a, mode, cmp, io, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_poisson_contract(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st) {
    if (mode != MODE_PK && mode != MODE_PRES) return cudaErrorInvalidValue;
    if (a.dim == 2) return poisson_w<2>(a, mode, cmp, io, st);
    if (a.dim == 3) return poisson_w<3>(a, mode, cmp, io, st);
    return cudaErrorInvalidValue;
}

// ---- elementwise kernels ------------------------------------------------------
// Coefficient tensors are (n_z, n_y, n_x); the spectral-domain buffers of the
// transforms are (n_z, n_y, px) with the x pitch px padded to a multiple of 8
// (32-byte aligned GEMM leading dimensions), zero in the padding columns.
// Grid: (ceil(px / 256), n_y, n_z); one thread per (padded) coefficient.
struct Grid3 {
    int n[3];
    int px;
    long long ntot;
    const int* is_free[3];   // NULL beyond the problem's dimension
    const float* lam[3];     // padded eigenvalues; NULL beyond the problem's dimension
};

__device__ __forceinline__ bool grid_index(const Grid3& g, int& x, int& y, int& z, long long& i, long long& ip) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    if (x >= g.px) return false;
    const long long row = (long long)z * g.n[1] + y;
    i = row * g.n[0] + x;
    ip = row * g.px + x;
    return true;
}

__device__ __forceinline__ bool free_at(const Grid3& g, int x, int y, int z) {
    bool f = g.is_free[0][x] != 0;
    if (g.is_free[1]) f = f && g.is_free[1][y] != 0;
    if (g.is_free[2]) f = f && g.is_free[2][z] != 0;
    return f;
}

// t = r in the padded layout (FP32 input), zero padding
__global__ void fdm_pack_kernel(Grid3 g, const float* r, float* t) {
    int x, y, z;
    long long i, ip;
    if (!grid_index(g, x, y, z, i, ip)) return;
    t[ip] = x < g.n[0] ? r[i] : 0.f;
}

// rho = (float) b and t = rho in the padded layout (FP64 input)
__global__ void fdm_pack_f64_kernel(Grid3 g, const double* b, float* rho, float* t) {
    int x, y, z;
    long long i, ip;
    if (!grid_index(g, x, y, z, i, ip)) return;
    float v = 0.f;
    if (x < g.n[0]) {
        v = (float)b[i];
        rho[i] = v;
    }
    t[ip] = v;
}

// t /= lx + ly + lz  (spectral domain; boundary and padding entries are zero)
__global__ void fdm_diag_kernel(Grid3 g, float* t) {
    int x, y, z;
    long long i, ip;
    if (!grid_index(g, x, y, z, i, ip)) return;
    float s = g.lam[0][x];
    if (g.lam[1]) s += g.lam[1][y];
    if (g.lam[2]) s += g.lam[2][z];
    t[ip] = t[ip] / s;
}

// u0 = P r: the transformed value off the boundary, r itself on it
__global__ void fdm_first_kernel(Grid3 g, const float* t, const float* r, float* u0) {
    int x, y, z;
    long long i, ip;
    if (!grid_index(g, x, y, z, i, ip) || x >= g.n[0]) return;
    u0[i] = free_at(g, x, y, z) ? t[ip] : r[i];
}

// pair output (hi, lo) = u0 + P rho, rounded to nearest as a double-float
__global__ void fdm_final_pair_kernel(Grid3 g, const float* u0, const float* t, const float* rho, float* out) {
    int x, y, z;
    long long i, ip;
    if (!grid_index(g, x, y, z, i, ip) || x >= g.n[0]) return;
    const float d = free_at(g, x, y, z) ? t[ip] : rho[i];
    float s, e;
    two_sum(u0[i], d, s, e);
    out[i] = s;
    out[i + g.ntot] = e;
}

// u = (first ? 0 : u) + P rho in FP64
__global__ void fdm_update_f64_kernel(Grid3 g, const float* t, const float* rho, double* u, int first) {
    int x, y, z;
    long long i, ip;
    if (!grid_index(g, x, y, z, i, ip) || x >= g.n[0]) return;
    const double d = (double)(free_at(g, x, y, z) ? t[ip] : rho[i]);
    u[i] = first ? d : u[i] + d;
}

// ---- set-up ---------------------------------------------------------------------
namespace {

#define FDM_CUDA(x)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) {                                                            \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                          \
            return e_ == cudaErrorMemoryAllocation ? -3 : -4;                               \
        }                                                                                   \
    } while (0)
#define FDM_SOLVER(x)                                                                       \
    do {                                                                                    \
        cusolverStatus_t e_ = (x);                                                          \
        if (e_ != CUSOLVER_STATUS_SUCCESS) {                                                \
            err = std::string(#x) + ": cusolver status " + std::to_string((int)e_);         \
            return -4;                                                                      \
        }                                                                                   \
    } while (0)
#define FDM_BLAS(x)                                                                         \
    do {                                                                                    \
        cublasStatus_t e_ = (x);                                                            \
        if (e_ != CUBLAS_STATUS_SUCCESS) {                                                  \
            err = std::string(#x) + ": cublas status " + std::to_string((int)e_);           \
            return -4;                                                                      \
        }                                                                                   \
    } while (0)

int pad8(int n) { return (n + 7) & ~7; }

// Scoped device buffers, solver handle and private stream of one fdm_build
// call.  Buffers are stream-ordered (cudaMallocAsync / cudaFreeAsync) so that
// set-up never synchronises the device: other contexts keep running.
struct Scratch {
    cudaStream_t ss = nullptr;
    std::vector<void*> dev;
    cusolverDnHandle_t solver = nullptr;
    cusolverDnParams_t params = nullptr;
    ~Scratch() {
        for (void* p : dev) cudaFreeAsync(p, ss);
        if (ss) cudaStreamSynchronize(ss);
        if (params) cusolverDnDestroyParams(params);
        if (solver) cusolverDnDestroy(solver);
        if (ss) cudaStreamDestroy(ss);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        cudaError_t e = cudaMallocAsync((void**)p, (count ? count : 1) * sizeof(T), ss);
        if (e == cudaSuccess) dev.push_back(*p);
        return e;
    }
    cudaError_t h2d(void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ss);
    }
    cudaError_t d2h(void* dst, const void* src, size_t bytes) {
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ss);
        return e == cudaSuccess ? cudaStreamSynchronize(ss) : e;
    }
};

// LU factorisation (in place) followed by X <- A^{-1} X (n x nrhs, column-major).
int lu_solve(Scratch& S, int64_t n, double* A, int64_t* ipiv, double* X, int64_t nrhs, int* dinfo,
             std::string& err, const char* what) {
    size_t dws = 0, hws = 0;
    FDM_SOLVER(cusolverDnXgetrf_bufferSize(S.solver, S.params, n, n, CUDA_R_64F, A, n, CUDA_R_64F, &dws, &hws));
    void* dbuf = nullptr;
    FDM_CUDA(S.alloc((unsigned char**)&dbuf, dws));
    std::vector<unsigned char> hbuf(hws ? hws : 1);
    FDM_SOLVER(cusolverDnXgetrf(S.solver, S.params, n, n, CUDA_R_64F, A, n, ipiv, CUDA_R_64F, dbuf, dws,
                                hbuf.data(), hws, dinfo));
    int info = 0;
    FDM_CUDA(S.d2h(&info, dinfo, sizeof info));
    if (info != 0) {
        err = std::string(what) + ": singular 1D matrix (getrf info " + std::to_string(info) + ")";
        return -2;
    }
    FDM_SOLVER(cusolverDnXgetrs(S.solver, S.params, CUBLAS_OP_N, n, nrhs, CUDA_R_64F, A, n, ipiv, CUDA_R_64F, X,
                                n, dinfo));
    return 0;
}

int build_axis(FdmAxisData& out, int a, const FdmAxisInput& in, Scratch& S, cublasHandle_t blas, std::string& err) {
    const int n = in.n, W = in.W;
    std::vector<int> fr, pos(n, -1);
    for (int i = 0; i < n; ++i)
        if (in.is_free[i]) {
            pos[i] = (int)fr.size();
            fr.push_back(i);
        }
    const int64_t m = (int64_t)fr.size();
    if (m == 0) {
        err = "axis " + std::to_string(a) + " has no unknowns";
        return -1;
    }
    // dense interior blocks, column-major: A_I and L_I = -C_I
    std::vector<double> Ai((size_t)m * m, 0.0), Li((size_t)m * m, 0.0);
    for (int r = 0; r < m; ++r) {
        const int i = fr[r];
        for (int w = 0; w < W; ++w) {
            const int j = in.fstart[i] + w;
            if (j < 0 || j >= n || pos[j] < 0) continue;
            Ai[(size_t)r + (size_t)pos[j] * m] = in.A[(size_t)i * W + w];
            Li[(size_t)r + (size_t)pos[j] * m] = -in.C[(size_t)i * W + w];
        }
    }
    const size_t mm = (size_t)m * m;
    double *dLU, *dG, *dV, *dAI, *dB, *dX;
    int64_t* ipiv;
    int* dinfo;
    cuDoubleComplex* dw;
    FDM_CUDA(S.alloc(&dLU, mm));
    FDM_CUDA(S.alloc(&dG, mm));
    FDM_CUDA(S.alloc(&dV, mm));
    FDM_CUDA(S.alloc(&dAI, mm));
    FDM_CUDA(S.alloc(&dB, mm));
    FDM_CUDA(S.alloc(&dX, mm));
    FDM_CUDA(S.alloc(&ipiv, (size_t)m));
    FDM_CUDA(S.alloc(&dinfo, 1));
    FDM_CUDA(S.alloc(&dw, (size_t)m));
    FDM_CUDA(S.h2d(dLU, Ai.data(), mm * 8));
    FDM_CUDA(S.h2d(dAI, Ai.data(), mm * 8));
    FDM_CUDA(S.h2d(dG, Li.data(), mm * 8));
    // G = A_I^{-1} L_I
    int rc = lu_solve(S, m, dLU, ipiv, dG, m, dinfo, err, "mass block");
    if (rc) return rc;
    // G = V diag(lambda) V^{-1}
    size_t dws = 0, hws = 0;
    FDM_SOLVER(cusolverDnXgeev_bufferSize(S.solver, S.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR,
                                          m, CUDA_R_64F, dG, m, CUDA_C_64F, dw, CUDA_R_64F, nullptr, 1, CUDA_R_64F,
                                          dV, m, CUDA_R_64F, &dws, &hws));
    void* dbuf = nullptr;
    FDM_CUDA(S.alloc((unsigned char**)&dbuf, dws));
    std::vector<unsigned char> hbuf(hws ? hws : 1);
    FDM_SOLVER(cusolverDnXgeev(S.solver, S.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, m,
                               CUDA_R_64F, dG, m, CUDA_C_64F, dw, CUDA_R_64F, nullptr, 1, CUDA_R_64F, dV, m,
                               CUDA_R_64F, dbuf, dws, hbuf.data(), hws, dinfo));
    int info = 0;
    FDM_CUDA(S.d2h(&info, dinfo, sizeof info));
    if (info != 0) {
        err = "eigensolver did not converge (geev info " + std::to_string(info) + ")";
        return -4;
    }
    std::vector<cuDoubleComplex> lam_c((size_t)m);
    FDM_CUDA(S.d2h(lam_c.data(), dw, (size_t)m * sizeof(cuDoubleComplex)));
    double lmax = 0.0, imax = 0.0, lmin = INFINITY;
    for (auto z : lam_c) {
        lmax = std::fmax(lmax, std::fabs(z.x));
        lmin = std::fmin(lmin, z.x);
        imax = std::fmax(imax, std::fabs(z.y));
    }
    // a Neumann pencil annihilates the constants (one zero eigenvalue, up to
    // rounding); a Dirichlet axis elsewhere keeps every sum of eigenvalues positive
    const double lfloor = in.neumann ? -1e-9 * lmax : 0.0;
    if (imax > 1e-9 * lmax || !(lmin > lfloor)) {
        err = "1D pencil spectrum not real and positive (max |imag| " + std::to_string(imax) + ", min real " +
              std::to_string(lmin) + ")";
        return -1;
    }
    // W = (A_I V)^{-1} = V^{-1} A_I^{-1}
    const double one = 1.0, zero = 0.0;
    FDM_BLAS(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)m, (int)m, (int)m, &one, dAI, (int)m, dV, (int)m,
                         &zero, dB, (int)m));
    std::vector<double> I(mm, 0.0);
    for (int64_t k = 0; k < m; ++k) I[(size_t)k + (size_t)k * m] = 1.0;
    FDM_CUDA(S.h2d(dX, I.data(), mm * 8));
    rc = lu_solve(S, m, dB, ipiv, dX, m, dinfo, err, "eigenvector block");
    if (rc) return rc;
    std::vector<double> V(mm), X(mm);
    FDM_CUDA(S.d2h(V.data(), dV, mm * 8));
    FDM_CUDA(S.d2h(X.data(), dX, mm * 8));
    // check a few eigenpairs against the pencil: |L v - lambda A v| <= tol |L| |v|
    double lnorm = 0.0;
    for (double v : Li) lnorm = std::fmax(lnorm, std::fabs(v));
    for (int t = 0; t < 4; ++t) {
        const int64_t k = (t * (m - 1)) / 3;
        double worst = 0.0;
        for (int64_t r = 0; r < m; ++r) {
            double lv = 0.0, av = 0.0;
            for (int64_t c = 0; c < m; ++c) {
                lv += Li[(size_t)r + (size_t)c * m] * V[(size_t)c + (size_t)k * m];
                av += Ai[(size_t)r + (size_t)c * m] * V[(size_t)c + (size_t)k * m];
            }
            worst = std::fmax(worst, std::fabs(lv - lam_c[k].x * av));
        }
        if (!(worst <= 1e-8 * lnorm * (double)m)) {
            err = "inaccurate eigenpair " + std::to_string(k) + " (residual " + std::to_string(worst) + ")";
            return -4;
        }
    }
    // embed in the full index range as FP32, padded to np = a multiple of 8
    const int np = pad8(n);
    std::vector<float> Wf((size_t)np * np, 0.f), Vf((size_t)np * np, 0.f), lf(np, 1.f);
    for (int64_t k = 0; k < m; ++k) {
        lf[fr[k]] = (float)lam_c[k].x;
        for (int64_t r = 0; r < m; ++r) {
            Vf[(size_t)fr[r] + (size_t)fr[k] * np] = (float)V[(size_t)r + (size_t)k * m];
            Wf[(size_t)fr[k] + (size_t)fr[r] * np] = (float)X[(size_t)k + (size_t)r * m];
        }
    }
    out.n = n;
    out.np = np;
    FDM_CUDA(cudaGetDevice(&out.device));
    FDM_CUDA(cudaMalloc((void**)&out.Wm, (size_t)np * np * sizeof(float)));
    FDM_CUDA(cudaMalloc((void**)&out.Vm, (size_t)np * np * sizeof(float)));
    FDM_CUDA(cudaMalloc((void**)&out.lam, (size_t)np * sizeof(float)));
    FDM_CUDA(S.h2d(out.Wm, Wf.data(), Wf.size() * 4));
    FDM_CUDA(S.h2d(out.Vm, Vf.data(), Vf.size() * 4));
    FDM_CUDA(S.h2d(out.lam, lf.data(), lf.size() * 4));
    FDM_CUDA(cudaStreamSynchronize(S.ss));   // host vectors go out of scope
    return 0;
}

}  // namespace

FdmAxisData::~FdmAxisData() {
    if (Wm) cudaFree(Wm);
    if (Vm) cudaFree(Vm);
    if (lam) cudaFree(lam);
}

namespace {

// Process-wide cache of diagonalised pencils, keyed by the device and the
// exact bytes of the 1D tables (n, W, A, C, window starts, unknown flags).
// It keeps the most recently used entries alive up to kCacheBytes of device
// memory; contexts hold their own references, so an entry dropped from the
// cache lives on until its last context is destroyed.
constexpr size_t kCacheBytes = size_t(2) << 30;
std::mutex g_cache_mu;
std::list<std::pair<std::string, std::shared_ptr<FdmAxisData>>> g_lru;   // front = most recent
std::unordered_map<std::string, decltype(g_lru)::iterator> g_index;
size_t g_cache_bytes = 0;

size_t entry_bytes(const FdmAxisData& d) { return ((size_t)2 * d.np * d.np + d.np) * sizeof(float); }

std::string cache_key(int device, const FdmAxisInput& in) {
    std::string k;
    auto put = [&k](const void* p, size_t b) { k.append(reinterpret_cast<const char*>(p), b); };
    put(&device, sizeof device);
    put(&in.n, sizeof in.n);
    put(&in.W, sizeof in.W);
    put(in.A.data(), in.A.size() * sizeof(double));
    put(in.C.data(), in.C.size() * sizeof(double));
    put(in.fstart.data(), in.fstart.size() * sizeof(int));
    put(in.is_free.data(), in.is_free.size() * sizeof(int));
    const char nm = in.neumann ? 1 : 0;
    put(&nm, 1);
    return k;
}

std::shared_ptr<FdmAxisData> cache_get(const std::string& key) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_index.find(key);
    if (it == g_index.end()) return nullptr;
    g_lru.splice(g_lru.begin(), g_lru, it->second);
    return it->second->second;
}

void cache_put(const std::string& key, const std::shared_ptr<FdmAxisData>& d) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    if (g_index.count(key)) return;
    g_lru.emplace_front(key, d);
    g_index[key] = g_lru.begin();
    g_cache_bytes += entry_bytes(*d);
    while (g_cache_bytes > kCacheBytes && g_lru.size() > 1) {
        auto& last = g_lru.back();
        g_cache_bytes -= entry_bytes(*last.second);
        g_index.erase(last.first);
        g_lru.pop_back();
    }
}

}  // namespace

// D(m, n) = sum_k A(m, k) B(n, k) of the transform along axis a: M applied
// to the padded spectral tensor `in` (n_z, n_y, px), written to `out`.  With
// `pre` (the matrix' tc_presplit tiles) the matrix operand is read from
// them; without, from M (column-major, leading dimension np).
static TcGemmArgs tc_axis_args(const FdmState& s, int a, const float* M, const float* in, float* out, const float* pre) {
    const int px = s.px, ny = s.n[1], nz = s.n[2];
    const int ld = s.axis[a]->np;
    TcGemmArgs g{};
    g.status = s.status;
    g.batch = 1;
    g.sDm = 1;
    if (a == 0) {          // out(x, j) = sum_k M(x, k) in(k, j), j = (z, y)
        g.M = px; g.N = ny * nz; g.K = px;
        g.A = M; g.sAm = 1; g.sAk = ld;
        g.B = in; g.sBn = px; g.sBk = 1;
        g.D = out; g.sDn = px;
        if (pre) { g.A = pre; g.pre = 1; g.bn = s.pre_bn[a]; }
    } else if (a == 1) {   // per z: out(x, y) = sum_k in(x, k) M(y, k)
        g.M = px; g.N = ny; g.K = ny; g.batch = nz;
        g.A = in; g.sAm = 1; g.sAk = px; g.bA = (long long)px * ny;
        g.B = M; g.sBn = 1; g.sBk = ld; g.bB = 0;
        g.D = out; g.sDn = px; g.bD = (long long)px * ny;
        if (pre) { g.B = pre; g.pre = 2; g.bn = s.pre_bn[a]; }
    } else {               // out(xy, z) = sum_k in(xy, k) M(z, k)
        g.M = px * ny; g.N = nz; g.K = nz;
        g.A = in; g.sAm = 1; g.sAk = (long long)px * ny;
        g.B = M; g.sBn = 1; g.sBk = ld;
        g.D = out; g.sDn = (long long)px * ny;
        if (pre) { g.B = pre; g.pre = 2; g.bn = s.pre_bn[a]; }
    }
    // the planned split of K (its workspace and counters are the state's)
    if (pre && s.splits[a] > 1) {
        g.splits = s.splits[a];
        for (int i = 0; i < 5; ++i) g.kb[i] = s.kb[a][i];
        g.ws = s.tc_ws;
        g.cnt = s.tc_cnt;
    }
    // the live operand's tensor map, when one was made for this input buffer
    if (pre && s.tmaps) {
        const int buf = in == s.t[0] ? 0 : in == s.t[1] ? 1 : -1;
        if (buf >= 0 && s.tmap_ok[a][buf]) {
            g.tmap = static_cast<const CUtensorMap*>(s.tmaps) + (a * 2 + buf);
            g.tmap_rows = s.tmap_rows[a];
        }
    }
    return g;
}

void fdm_release(FdmState& s) {
    for (int k = 0; k < 2; ++k)
        if (s.t[k]) cudaFreeAsync(s.t[k], s.stream);
    s.t[0] = s.t[1] = nullptr;
    for (int a = 0; a < 3; ++a) {
        for (int h = 0; h < 2; ++h)
            if (s.pre[a][h]) cudaFreeAsync(s.pre[a][h], s.stream);
        s.pre[a][0] = s.pre[a][1] = nullptr;
        s.pre_role[a] = s.pre_bn[a] = s.tmap_rows[a] = 0;
        s.tmap_ok[a][0] = s.tmap_ok[a][1] = false;
    }
    if (s.tmaps) cudaFreeAsync(s.tmaps, s.stream);
    s.tmaps = nullptr;
    if (s.tc_ws) cudaFreeAsync(s.tc_ws, s.stream);
    if (s.tc_cnt) cudaFreeAsync(s.tc_cnt, s.stream);
    s.tc_ws = nullptr;
    s.tc_cnt = nullptr;
    for (int a = 0; a < 3; ++a) s.splits[a] = 1;
    if (s.blas) cublasDestroy(s.blas);
    s.blas = nullptr;
    for (int a = 0; a < 3; ++a) {
        s.axis[a].reset();
        s.Wm[a] = s.Vm[a] = s.lam[a] = nullptr;
    }
}

int fdm_build(FdmState& s, int dim, const FdmAxisInput* ax, const int* const* is_free_dev, int gemm,
              unsigned* status, cudaStream_t st, std::string& err) {
    fdm_release(s);
    s.dim = dim;
    s.gemm = gemm;
    s.status = status;
    s.stream = st;
    for (int a = 0; a < 3; ++a) {
        s.n[a] = a < dim ? ax[a].n : 1;
        s.is_free[a] = a < dim ? is_free_dev[a] : nullptr;
    }
    s.px = pad8(s.n[0]);
    const size_t tbytes = (size_t)s.px * s.n[1] * s.n[2] * sizeof(float);
    for (int k = 0; k < 2; ++k) FDM_CUDA(cudaMallocAsync((void**)&s.t[k], tbytes, st));
    int device = 0;
    FDM_CUDA(cudaGetDevice(&device));
    FDM_BLAS(cublasCreate(&s.blas));
    std::unique_ptr<Scratch> S;   // solver set-up only on a cache miss
    for (int a = 0; a < dim; ++a) {
        const std::string key = cache_key(device, ax[a]);
        std::shared_ptr<FdmAxisData> d = cache_get(key);
        if (!d) {
            if (!S) {
                S.reset(new Scratch());
                FDM_CUDA(cudaStreamSynchronize(st));   // the folded tables are final
                FDM_CUDA(cudaStreamCreateWithFlags(&S->ss, cudaStreamNonBlocking));
                FDM_SOLVER(cusolverDnCreate(&S->solver));
                FDM_SOLVER(cusolverDnCreateParams(&S->params));
                FDM_SOLVER(cusolverDnSetStream(S->solver, S->ss));
                FDM_BLAS(cublasSetStream(s.blas, S->ss));
            }
            d = std::make_shared<FdmAxisData>();
            int rc = build_axis(*d, a, ax[a], *S, s.blas, err);
            if (rc) return rc;
            cache_put(key, d);
        }
        s.axis[a] = d;
        s.Wm[a] = d->Wm;
        s.Vm[a] = d->Vm;
        s.lam[a] = d->lam;
    }
    if (S) FDM_CUDA(cudaStreamSynchronize(S->ss));
    FDM_BLAS(cublasSetStream(s.blas, st));
    if (gemm == FDM_GEMM_TC) {
        // the constant operand of every transform, split once (gemm_axis),
        // for the planned tile width; the split of K and its workspace
        long long ws_floats = 0, counters = 0;
        for (int a = 0; a < dim; ++a) {
            TcGemmArgs g = tc_axis_args(s, a, nullptr, nullptr, nullptr, nullptr);
            const int ld = s.axis[a]->np;
            const int role = a == 0 ? 1 : 2;
            const TcPlan plan = tc_plan(g, tc_sm_count(), 0, true);
            const int bn = plan.bn;
            s.splits[a] = plan.splits;
            for (int i = 0; i < 5; ++i) s.kb[a][i] = plan.kb[i];
            ws_floats = std::max(ws_floats, tc_split_ws_floats(g, plan));
            counters = std::max(counters, tc_split_counters(g, plan));
            const int R = role == 1 ? tc::BM : bn;
            const int rows = role == 1 ? g.M : g.N;
            const long long nf = tc_presplit_floats(rows, g.K, R, role == 2);
            for (int h = 0; h < 2; ++h) {
                const float* Mat = h == 0 ? s.Wm[a] : s.Vm[a];
                FDM_CUDA(cudaMallocAsync((void**)&s.pre[a][h], (size_t)nf * sizeof(float), st));
                // x axis: A(x', k) = M[x' + k ld]; y/z axes: B(n, k) = M[n + k ld]
                FDM_CUDA(launch_tc_presplit(Mat, 1, ld, rows, g.K, R, role == 2, s.pre[a][h], st));
            }
            s.pre_role[a] = role;
            s.pre_bn[a] = bn;
        }
        if (ws_floats > 0) {
            FDM_CUDA(cudaMallocAsync((void**)&s.tc_ws, (size_t)ws_floats * sizeof(float), st));
            FDM_CUDA(cudaMallocAsync((void**)&s.tc_cnt, (size_t)counters * sizeof(unsigned), st));
            FDM_CUDA(cudaMemsetAsync(s.tc_cnt, 0, (size_t)counters * sizeof(unsigned), st));
        }
        // tensor maps of the spectral operand for TMA loads: the live operand
        // is B (x axis, tiles of bn rows) or A (y/z axes, tiles of 128 rows),
        // read from t[0] or t[1] depending on the transform's position
        std::vector<CUtensorMap> maps(6);
        for (int a = 0; a < dim; ++a) {
            s.tmap_rows[a] = a == 0 ? s.pre_bn[a] : tc::BM;
            for (int buf = 0; buf < 2; ++buf) {
                const TcGemmArgs g = tc_axis_args(s, a, nullptr, s.t[buf], nullptr, nullptr);
                s.tmap_ok[a][buf] = a == 0 ? tc_make_tmap(&maps[a * 2 + buf], g.B, g.sBn, g.sBk, g.bB, g.N, g.K,
                                                         g.batch, s.tmap_rows[a])
                                           : tc_make_tmap(&maps[a * 2 + buf], g.A, g.sAm, g.sAk, g.bA, g.M, g.K,
                                                         g.batch, s.tmap_rows[a]);
            }
        }
        FDM_CUDA(cudaMallocAsync(&s.tmaps, maps.size() * sizeof(CUtensorMap), st));
        FDM_CUDA(cudaMemcpyAsync(s.tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
        FDM_CUDA(cudaStreamSynchronize(st));   // the host vector of maps goes out of scope
    }
    if (gemm == FDM_GEMM_BF16X9) {
        FDM_BLAS(cublasSetMathMode(s.blas, CUBLAS_FP32_EMULATED_BF16X9_MATH));
        FDM_BLAS(cublasSetEmulationStrategy(s.blas, CUBLAS_EMULATION_STRATEGY_EAGER));
    }
    return 0;
}

// ---- solve ---------------------------------------------------------------------
namespace {

// out = M applied along axis a of the padded spectral tensor `in` (n_z, n_y, px)
int gemm_axis(FdmState& s, int a, const float* M, const float* in, float* out, std::string& err) {
    const int px = s.px, ny = s.n[1], nz = s.n[2];
    const int ld = s.axis[a]->np;   // padded leading dimension of M
    if (s.gemm == FDM_GEMM_TC) {
        // the same products as the cuBLAS calls below, with the axis matrix
        // taken from its pre-split tiles
        TcGemmArgs g = tc_axis_args(s, a, M, in, out, s.pre[a][M == s.Wm[a] ? 0 : 1]);
        FDM_CUDA(launch_tc_gemm(g, s.stream_now));
        return 0;
    }
    const float one = 1.f, zero = 0.f;
    const cublasComputeType_t ct = s.gemm == FDM_GEMM_BF16X9 ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F;
    if (a == 0) {
        FDM_BLAS(cublasGemmEx(s.blas, CUBLAS_OP_N, CUBLAS_OP_N, px, ny * nz, px, &one, M, CUDA_R_32F, ld, in,
                              CUDA_R_32F, px, &zero, out, CUDA_R_32F, px, ct, CUBLAS_GEMM_DEFAULT));
    } else if (a == 1) {
        FDM_BLAS(cublasGemmStridedBatchedEx(s.blas, CUBLAS_OP_N, CUBLAS_OP_T, px, ny, ny, &one, in, CUDA_R_32F, px,
                                            (long long)px * ny, M, CUDA_R_32F, ld, 0, &zero, out, CUDA_R_32F, px,
                                            (long long)px * ny, nz, ct, CUBLAS_GEMM_DEFAULT));
    } else {
        FDM_BLAS(cublasGemmEx(s.blas, CUBLAS_OP_N, CUBLAS_OP_T, px * ny, nz, nz, &one, in, CUDA_R_32F, px * ny, M,
                              CUDA_R_32F, ld, &zero, out, CUDA_R_32F, px * ny, ct, CUBLAS_GEMM_DEFAULT));
    }
    return 0;
}

Grid3 grid_of(const FdmState& s, long long ntot) {
    Grid3 g{};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = s.n[a];
        g.is_free[a] = s.is_free[a];
        g.lam[a] = a < s.dim ? s.lam[a] : nullptr;
    }
    g.px = s.px;
    g.ntot = ntot;
    return g;
}

dim3 grid_dims(const Grid3& g) { return dim3((g.px + 255) / 256, g.n[1], g.n[2]); }

// Transforms the padded tensor in s.t[0] in place (result in s.t[0]): W's,
// 1/(sum lambda), V's -- 2 dim GEMMs ping-ponging between s.t[0] and s.t[1].
int apply_fdm(FdmState& s, const Grid3& g, cudaStream_t st, std::string& err) {
    float* buf[2] = {s.t[0], s.t[1]};
    int cur = 0;
    for (int a = 0; a < s.dim; ++a, cur ^= 1) {
        int rc = gemm_axis(s, a, s.Wm[a], buf[cur], buf[cur ^ 1], err);
        if (rc) return rc;
    }
    fdm_diag_kernel<<<grid_dims(g), 256, 0, st>>>(g, buf[cur]);
    FDM_CUDA(cudaGetLastError());
    for (int a = 0; a < s.dim; ++a, cur ^= 1) {
        int rc = gemm_axis(s, a, s.Vm[a], buf[cur], buf[cur ^ 1], err);
        if (rc) return rc;
    }
    return 0;
}

}  // namespace

int fdm_solve(FdmState& s, const ContractArgs& ca, const void* b, void* u, bool fp64, int iters, float* rho,
              float* u0, bool pair_fp64_residual, cudaStream_t st, std::string& err) {
    FDM_BLAS(cublasSetStream(s.blas, st));
    s.stream_now = st;
    const Grid3 g = grid_of(s, ca.ntot);
    const dim3 gd = grid_dims(g);
    const float* t = s.t[0];
    if (!fp64) {
        const float* bhi = (const float*)b;
        fdm_pack_kernel<<<gd, 256, 0, st>>>(g, bhi, s.t[0]);
        FDM_CUDA(cudaGetLastError());
        int rc = apply_fdm(s, g, st, err);
        if (rc) return rc;
        fdm_first_kernel<<<gd, 256, 0, st>>>(g, t, bhi, u0);
        FDM_CUDA(cudaGetLastError());
        ContractArgs a = ca;
        a.u = u0;
        a.r = b;
        a.out = rho;
        a.alpha = 0.0;
        a.beta = -1.0;
        FDM_CUDA(launch_poisson_contract(a, MODE_PRES, pair_fp64_residual ? FMT_F64 : FMT_PAIR, FMT_PAIR, st));
        fdm_pack_kernel<<<gd, 256, 0, st>>>(g, rho, s.t[0]);
        FDM_CUDA(cudaGetLastError());
        rc = apply_fdm(s, g, st, err);
        if (rc) return rc;
        fdm_final_pair_kernel<<<gd, 256, 0, st>>>(g, u0, t, rho, (float*)u);
        FDM_CUDA(cudaGetLastError());
        return 0;
    }
    fdm_pack_f64_kernel<<<gd, 256, 0, st>>>(g, (const double*)b, rho, s.t[0]);
    FDM_CUDA(cudaGetLastError());
    for (int it = 0; it <= iters; ++it) {
        int rc = apply_fdm(s, g, st, err);
        if (rc) return rc;
        fdm_update_f64_kernel<<<gd, 256, 0, st>>>(g, t, rho, (double*)u, it == 0);
        FDM_CUDA(cudaGetLastError());
        if (it == iters) break;
        ContractArgs a = ca;
        a.u = u;
        a.r = b;
        a.out = rho;
        a.alpha = 0.0;
        a.beta = -1.0;
        FDM_CUDA(launch_poisson_contract(a, MODE_PRES, FMT_F64, FMT_F64, st));
        fdm_pack_kernel<<<gd, 256, 0, st>>>(g, rho, s.t[0]);
        FDM_CUDA(cudaGetLastError());
    }
    return 0;
}

// The tensor-core GEMM on caller buffers (igapw_tc_gemm): synchronous; a
// pre-split operand (pre = 1: A, 2: B) is split into a temporary buffer
// first.  in.splits: 0 = tile width and split of K from tc_plan, 1 = no
// split, 2-4 = that many equal chunk ranges (temporary workspace and
// counters).  Returns a CUDA error, or cudaErrorLaunchTimeout when a
// pipeline wait of the kernel timed out.
static __device__ unsigned g_tc_entry_status;

cudaError_t tc_gemm_entry(const TcGemmArgs& in, cudaStream_t st) {
    TcGemmArgs g = in;
    if ((g.pre == 1 || g.pre == 2) && g.batch != 1 && (g.pre == 1 ? g.bA : g.bB) != 0) return cudaErrorInvalidValue;
    const int sms = tc_sm_count();
    const int nkc = (g.K + tc::BK - 1) / tc::BK;
    TcPlan plan;
    if (g.splits == 0) {
        plan = tc_plan(g, sms, g.bn, true);
    } else {
        if (g.splits < 0 || g.splits > kTcMaxSplits || g.splits > nkc) return cudaErrorInvalidValue;
        plan.bn = g.bn ? g.bn : tc_pick_width(&g, 1, sms);
        plan.splits = g.splits;
        for (int i = 0; i < 5; ++i) plan.kb[i] = i <= plan.splits ? (int)((long long)nkc * i / plan.splits) : nkc;
    }
    unsigned* status = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&status, g_tc_entry_status);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    g.status = status;
    float* ws = nullptr;
    unsigned* cnt = nullptr;
    if (plan.splits > 1) {
        e = cudaMallocAsync((void**)&ws, (size_t)tc_split_ws_floats(g, plan) * sizeof(float), st);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void**)&cnt, (size_t)tc_split_counters(g, plan) * sizeof(unsigned), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(cnt, 0, (size_t)tc_split_counters(g, plan) * sizeof(unsigned), st);
    }
    tc_apply_plan(g, plan, ws, cnt);
    float* tmp = nullptr;
    if (e == cudaSuccess && (g.pre == 1 || g.pre == 2)) {
        const int R = g.pre == 1 ? tc::BM : g.bn;
        const int rows = g.pre == 1 ? g.M : g.N;
        e = cudaMallocAsync((void**)&tmp, (size_t)tc_presplit_floats(rows, g.K, R, g.pre == 2) * sizeof(float), st);
        if (e != cudaSuccess) {
            tmp = nullptr;
        } else if (g.pre == 1) {
            e = launch_tc_presplit(g.A, g.sAm, g.sAk, rows, g.K, R, false, tmp, st);
            g.A = tmp;
        } else {
            e = launch_tc_presplit(g.B, g.sBn, g.sBk, rows, g.K, R, true, tmp, st);
            g.B = tmp;
        }
    }
    // the live operand by TMA where a tensor map can describe it
    void* dmap = nullptr;
    if (e == cudaSuccess && (g.pre == 1 || g.pre == 2)) {
        CUtensorMap hm;
        const int R = g.pre == 1 ? g.bn : tc::BM;
        const bool ok = g.pre == 1 ? tc_make_tmap(&hm, g.B, g.sBn, g.sBk, g.bB, g.N, g.K, g.batch, R)
                                   : tc_make_tmap(&hm, g.A, g.sAm, g.sAk, g.bA, g.M, g.K, g.batch, R);
        if (ok) {
            e = cudaMallocAsync(&dmap, sizeof(CUtensorMap), st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dmap, &hm, sizeof hm, cudaMemcpyHostToDevice, st);
            g.tmap = static_cast<const CUtensorMap*>(dmap);
            g.tmap_rows = R;
        }
    }
    if (e == cudaSuccess) e = launch_tc_gemm(g, st);
    if (tmp) cudaFreeAsync(tmp, st);
    if (dmap) cudaFreeAsync(dmap, st);
    if (ws) cudaFreeAsync(ws, st);
    if (cnt) cudaFreeAsync(cnt, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e;
    unsigned h = 0;
    e = cudaMemcpy(&h, status, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    return (h & STATUS_TC_TIMEOUT) ? cudaErrorLaunchTimeout : cudaSuccess;
}

}  // namespace igapw
