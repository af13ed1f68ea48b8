// Runs the chunked explicit-step kernel (chunkstep.cuh) and its table set-up
// kernel (chunktables.cuh) on the CPU, every CUDA thread a host thread, with
// every buffer allocated at its exact size so that AddressSanitizer reports
// any access outside it.  Input (binary, from tests/test_chunk_emu.py):
//   int dim, n[3], p, W, NL, nsteps; double dt; then per axis int fstart[n],
//   double A[n][W], C[n][W] (window format); then float u[2][ntot] (hi, lo).
// Output: float u[2][ntot] after nsteps steps.  The banded LU without
// pivoting of A is computed here (the library's factor kernel does the same).
#include "cuda_emu.h"

#include <cstdio>
#include <cstdlib>
#include <thread>
#include <vector>

#include "../../paper_1910_08535_gb300/csrc/chunkstep.cuh"
#include "../../paper_1910_08535_gb300/csrc/chunktables.cuh"

using namespace igapw;

template <class T>
static T* exact(size_t count) {
    T* p = static_cast<T*>(std::malloc(count * sizeof(T)));
    if (!p) std::abort();
    std::memset(p, 0, count * sizeof(T));
    return p;
}

struct AxisIn {
    int n;
    std::vector<int> fs;
    std::vector<double> A, C;
};

static ChunkDev build_tables(const AxisIn& ax, int p, int W) {
    const int n = ax.n;
    // banded LU without pivoting (Doolittle), KL = KU = p
    std::vector<double> M((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int w = 0; w < W; ++w) {
            const int j = ax.fs[i] + w;
            if (j < n) M[(size_t)i * n + j] = ax.A[(size_t)i * W + w];
        }
    for (int k = 0; k < n; ++k)
        for (int i = k + 1; i <= std::min(n - 1, k + p); ++i) {
            const double l = M[(size_t)i * n + k] / M[(size_t)k * n + k];
            M[(size_t)i * n + k] = l;
            for (int j = k + 1; j <= std::min(n - 1, k + p); ++j) M[(size_t)i * n + j] -= l * M[(size_t)k * n + j];
        }
    double* L = exact<double>((size_t)n * p);
    double* U = exact<double>((size_t)n * p);
    double* dinv = exact<double>(n);
    for (int i = 0; i < n; ++i) {
        for (int m = 1; m <= p; ++m) {
            L[i * p + m - 1] = i - m >= 0 ? M[(size_t)i * n + i - m] : 0.0;
            U[i * p + m - 1] = i + m < n ? M[(size_t)i * n + i + m] : 0.0;
        }
        dinv[i] = 1.0 / M[(size_t)i * n + i];
    }
    float2* Adf = exact<float2>((size_t)n * W);
    float2* Cdf = exact<float2>((size_t)n * W);
    for (size_t e = 0; e < (size_t)n * W; ++e) {
        split_double(ax.A[e], Adf[e].x, Adf[e].y);
        split_double(ax.C[e], Cdf[e].x, Cdf[e].y);
    }
    int* fs = exact<int>(n);
    for (int i = 0; i < n; ++i) fs[i] = ax.fs[i];
    const int RS = IGAPW_CHUNK_ROWS, P = (n + RS - 1) / RS, q4 = (2 * W + 4) / 4;
    const size_t np = (size_t)P * RS;   // padded line
    ChunkTableArgs ca{};
    ca.n = n; ca.p = p; ca.W = W; ca.RS = RS; ca.P = P;
    ca.L = L; ca.U = U; ca.dinv = dinv; ca.Adf = Adf; ca.Cdf = Cdf; ca.fstart = fs;
    ca.work = exact<double>(2 * np * p);
    ca.cw = exact<float4>(np * q4); ca.aw = exact<float4>(np * q4);
    ca.fl = exact<float4>(np); ca.fu = exact<float4>(np); ca.fg = exact<float4>(np); ca.fh = exact<float4>(np);
    ca.fd = exact<float>(np);
    ca.psf = exact<float>((size_t)P * P * p * p); ca.psb = exact<float>((size_t)P * P * p * p);
    ca.J = exact<int>(1);
    emu_threadIdx = {}; emu_blockIdx = {}; emu_blockDim = {1, 1, 1};
    chunk_tables_kernel(ca);
    ChunkDev d{};
    d.rows = RS; d.P = P;
    d.cw = ca.cw; d.aw = ca.aw; d.fl = ca.fl; d.fu = ca.fu; d.fd = ca.fd; d.fg = ca.fg; d.fh = ca.fh;
    d.psf = ca.psf; d.psb = ca.psb; d.J = ca.J;
    return d;
}

template <int KP, int W, int MODE>
static void run(const AxisStepArgs& a) {
    constexpr bool XL = (MODE == 0 || MODE == 3);
    const int n = a.ax.n, P = a.ax.ck.P, NL = a.lines_per_block;
    const long long nlines = XL ? (long long)a.n[1] * a.n[2]
                                : (a.axis == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
    const size_t sm = chunkstep::smem_bytes(XL, P * IGAPW_CHUNK_ROWS, W, NL, P, KP);
    const long long blocks = (nlines + NL - 1) / NL;
    const int threads = NL * P;
    for (long long b = 0; b < blocks; ++b) {
        unsigned char* smem = static_cast<unsigned char*>(std::malloc(sm));
        std::memset(smem, 0xff, sm);   // garbage, as on the device
        std::barrier<> bar(threads);
        std::vector<std::thread> ts;
        for (int t = 0; t < threads; ++t)
            ts.emplace_back([&, t] {
                emu_threadIdx = {(unsigned)t, 0, 0};
                emu_blockIdx = {(unsigned)b, 0, 0};
                emu_blockDim = {(unsigned)threads, 1, 1};
                emu_barrier = &bar;
                emu_smem_ptr = smem;
                chunk_step_kernel<KP, W, MODE, IGAPW_CHUNK_ROWS>(a);
            });
        for (auto& t : ts) t.join();
        std::free(smem);
    }
}

template <int KP, int W>
static void run_mode(const AxisStepArgs& a, int mode) {
    switch (mode) {
        case 0: run<KP, W, 0>(a); break;
        case 1: run<KP, W, 1>(a); break;
        case 2: run<KP, W, 2>(a); break;
        case 3: run<KP, W, 3>(a); break;
    }
}

template <int KP>
static void run_w(const AxisStepArgs& a, int mode) {
    switch (a.W) {
        case 3: run_mode<KP, 3>(a, mode); break;
        case 5: run_mode<KP, 5>(a, mode); break;
        case 7: run_mode<KP, 7>(a, mode); break;
        case 9: run_mode<KP, 9>(a, mode); break;
        default: std::fprintf(stderr, "bad W\n"); std::exit(2);
    }
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int hdr[8];
    double dt;
    if (std::fread(hdr, sizeof(int), 8, f) != 8 || std::fread(&dt, sizeof dt, 1, f) != 1) return 2;
    const int dim = hdr[0], p = hdr[4], W = hdr[5], NL = hdr[6], nsteps = hdr[7];
    int nn[3] = {hdr[1], hdr[2], hdr[3]};
    long long ntot = 1;
    for (int a = 0; a < 3; ++a) ntot *= nn[a];
    AxisIn ax[3];
    for (int a = 0; a < dim; ++a) {
        const int n = nn[a];
        ax[a].n = n;
        ax[a].fs.resize(n);
        ax[a].A.resize((size_t)n * W);
        ax[a].C.resize((size_t)n * W);
        if (std::fread(ax[a].fs.data(), sizeof(int), n, f) != (size_t)n ||
            std::fread(ax[a].A.data(), sizeof(double), (size_t)n * W, f) != (size_t)n * W ||
            std::fread(ax[a].C.data(), sizeof(double), (size_t)n * W, f) != (size_t)n * W)
            return 2;
    }
    float* u = exact<float>((size_t)2 * ntot);
    float* acc = exact<float>((size_t)2 * ntot);
    if (std::fread(u, sizeof(float), (size_t)2 * ntot, f) != (size_t)2 * ntot) return 2;
    std::fclose(f);
    ChunkDev ck[3];
    for (int a = 0; a < dim; ++a) ck[a] = build_tables(ax[a], p, W);
    unsigned* status = exact<unsigned>(1);
    for (int s = 0; s < nsteps; ++s)
        for (int axis = 0; axis < dim; ++axis) {
            AxisStepArgs a{};
            a.axis = axis;
            for (int k = 0; k < 3; ++k) a.n[k] = nn[k];
            a.W = W;
            a.lines_per_block = NL;
            a.cfg = 3;
            a.ntot = ntot;
            a.ax.n = nn[axis];
            a.ax.ck = ck[axis];
            a.u = u;
            a.u_out = u;
            a.acc = acc;
            a.dt = dt;
            a.status = status;
            const int mode = dim == 1 ? 3 : (axis == 0 ? 0 : (axis == dim - 1 ? 2 : 1));
            switch (p) {
                case 2: run_w<2>(a, mode); break;
                case 3: run_w<3>(a, mode); break;
                case 4: run_w<4>(a, mode); break;
                default: return 2;
            }
        }
    FILE* o = std::fopen(argv[2], "wb");
    if (!o) return 2;
    std::fwrite(u, sizeof(float), (size_t)2 * ntot, o);
    std::fclose(o);
    return *status ? 3 : 0;
}
