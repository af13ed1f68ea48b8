// Batched 2D Poisson solves over many uneven instances (Sec. 4.3 problem,
// -Lap u = f with zero Dirichlet rows, FP32 pairs with one refinement step).
//
// Every instance keeps its own context (1D tables, diagonalised pencils from
// the process-wide cache); the batch packs their tensors into shared device
// arrays and runs each stage of the solve for all instances at once:
//   source   one persistent kernel over (instance, tile) work items taken from
//            an atomic counter: the manufactured source amp sin(kx pi x)
//            sin(ky pi y) evaluated at each instance's quadrature points and
//            summed over the test supports (PW cells or B-spline supports)
//   P        grouped FP32 GEMMs (cuBLAS, one call per transform stage for all
//            instances) with a batched diagonal-scaling kernel in between
//   residual one persistent kernel per window width: rho = b - K u0 in
//            double-float (sum-factorised over a tile with its halo)
//   update   batched elementwise kernels
// The whole solve is captured once into a CUDA graph and replayed.  Tile
// shapes of the two persistent kernels are chosen at creation by timing the
// candidates on the batch itself.
#include <cublas_v2.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/igapw.h"
#include "common.cuh"
#include "kernels.h"
#include "poisson.h"
#include "tcgemm.cuh"

namespace igapw {
namespace {

struct BInst {
    int nx, ny, px, W;
    long long off;     // F32 tensors at off, pair tensors at 2 off (hi plane, then lo plane)
    long long poff;    // padded spectral buffers (ny x px)
    int qx, qy;        // quadrature points per axis
    AxisDev ax[2];
    const double* qpx;
    const double* qpy;
    const float* lamx;
    const float* lamy;
};

struct BSrc {
    float amp, kx, ky, pad;
};

// ---- persistent source kernel ----------------------------------------------
// b[i, j] = amp (sum_r TWy[j][r] sy(y_r)) (sum_q TWx[i][q] sx(x_q)) in
// double-float: the tensor-product quadrature sum of the separable source.
template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) batch_source_kernel(const BInst* insts, const BSrc* src, const int4* items,
                                                               int nitems, int* counter, float* bpair) {
    __shared__ int slot;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) slot = atomicAdd(counter, 1);
        __syncthreads();
        const int k = slot;
        if (k >= nitems) return;
        const int4 w = items[k];
        const BInst& I = insts[w.x];
        const BSrc S = src[w.x];
        const int i = w.y + (int)threadIdx.x % TX, j = w.z + (int)threadIdx.x / TX;
        if (i >= I.nx || j >= I.ny) continue;
        const AxisDev& X = I.ax[0];
        const AxisDev& Y = I.ax[1];
        DFAcc gx, gy;
        gx.init();
        gy.init();
        const int psx = X.pstart[i], psy = Y.pstart[j];
        for (int c = 0; c < X.wq; ++c) {
            const int q = psx + c;
            if (q >= I.qx) break;
            const float2 t = X.TW.df[i * X.wq + c];
            gx.add_prod_f(DF{t.x, t.y}, sinpif(S.kx * (float)I.qpx[q]));
        }
        for (int c = 0; c < Y.wq; ++c) {
            const int q = psy + c;
            if (q >= I.qy) break;
            const float2 t = Y.TW.df[j * Y.wq + c];
            gy.add_prod_f(DF{t.x, t.y}, sinpif(S.ky * (float)I.qpy[q]));
        }
        const DF r = df_mul(df_mul(gx.result(), gy.result()), DF{S.amp, 0.f});
        const long long e = (long long)j * I.nx + i;
        const long long nt = (long long)I.nx * I.ny;
        if (!IGAPW_IDX("batch source out", e, nt)) continue;
        bpair[2 * I.off + e] = r.hi;
        bpair[2 * I.off + nt + e] = r.lo;
    }
}

// ---- persistent residual kernel: rho = b - K u0 ------------------------------
// K u = -(C_x (x) A_y + A_x (x) C_y) u off the boundary, u on it.  A tile of
// TX x TY outputs stages u0 with the window halo, a y-pass forms ZA = A_y u,
// ZC = C_y u on the tile rows (all halo columns), an x-pass finishes
// rho = b + C_x ZA + A_x ZC.
template <int W, int TX, int TY>
__global__ void __launch_bounds__(256) batch_residual_kernel(const BInst* insts, const int4* items, int nitems,
                                                             int* counter, const float* u0, const float* bpair,
                                                             float* rho) {
    constexpr int XH = TX + W - 1, YH = TY + W - 1;
    __shared__ float us[YH][XH + 1];
    __shared__ float2 za[TY][XH + 1];
    __shared__ float2 zc[TY][XH + 1];
    __shared__ int slot;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) slot = atomicAdd(counter, 1);
        __syncthreads();
        const int k = slot;
        if (k >= nitems) return;
        const int4 w = items[k];
        const BInst& I = insts[w.x];
        const AxisDev& X = I.ax[0];
        const AxisDev& Y = I.ax[1];
        const int nx = I.nx, ny = I.ny;
        const int x0 = w.y, y0 = w.z;
        const int nxo = min(TX, nx - x0), nyo = min(TY, ny - y0);
        const int xl = X.fstart[x0], yl = Y.fstart[y0];
        const int nxh = X.fstart[x0 + nxo - 1] + W - xl;
        const int nyh = Y.fstart[y0 + nyo - 1] + W - yl;
        const float* u = u0 + I.off;
        for (int e = threadIdx.x; e < YH * XH; e += blockDim.x) {
            const int r = e / XH, c = e - r * XH;
            const int gy = yl + r, gx = xl + c;
            us[r][c] = (r < nyh && c < nxh && gy < ny && gx < nx &&
                        IGAPW_IDX("batch residual u", (long long)gy * nx + gx, (long long)nx * ny))
                           ? u[(long long)gy * nx + gx]
                           : 0.f;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TY * XH; e += blockDim.x) {
            const int yy = e / XH, c = e - yy * XH;
            if (yy >= nyo || c >= nxh) continue;
            const int j = y0 + yy;
            const int sy = Y.fstart[j] - yl;
            DFAcc a1, a2;
            a1.init();
            a2.init();
#pragma unroll
            for (int v = 0; v < W; ++v) {
                const float uv = us[sy + v][c];
                const float2 ta = Y.A.df[j * W + v];
                const float2 tc = Y.C.df[j * W + v];
                a1.add_prod_f(DF{ta.x, ta.y}, uv);
                a2.add_prod_f(DF{tc.x, tc.y}, uv);
            }
            const DF r1 = a1.result(), r2 = a2.result();
            za[yy][c] = make_float2(r1.hi, r1.lo);
            zc[yy][c] = make_float2(r2.hi, r2.lo);
        }
        __syncthreads();
        const long long nt = (long long)nx * ny;
        for (int e = threadIdx.x; e < TY * TX; e += blockDim.x) {
            const int yy = e / TX, xx = e - yy * TX;
            if (yy >= nyo || xx >= nxo) continue;
            const int i = x0 + xx, j = y0 + yy;
            const long long g = (long long)j * nx + i;
            if (!IGAPW_IDX("batch residual out", g, nt)) continue;
            DFAcc acc;
            acc.s = bpair[2 * I.off + g];
            acc.c = bpair[2 * I.off + nt + g];
            if (X.is_free[i] && Y.is_free[j]) {
                const int sx = X.fstart[i] - xl;
#pragma unroll
                for (int v = 0; v < W; ++v) {
                    const float2 tc = X.C.df[i * W + v];
                    const float2 ta = X.A.df[i * W + v];
                    const float2 a = za[yy][sx + v];
                    const float2 c = zc[yy][sx + v];
                    acc.add_prod(DF{tc.x, tc.y}, DF{a.x, a.y});
                    acc.add_prod(DF{ta.x, ta.y}, DF{c.x, c.y});
                }
            } else {
                acc.add(DF{-u[g], 0.f});
            }
            rho[I.off + g] = acc.result().hi;
        }
    }
}

// ---- batched elementwise kernels over (instance, row) -------------------------
enum { EL_PACK_HI = 0, EL_PACK_F32 = 1, EL_DIAG = 2, EL_FIRST = 3, EL_FINAL = 4 };

__global__ void __launch_bounds__(256) batch_elem_kernel(const BInst* insts, const int2* rows, int nrows, int mode,
                                                         const float* bpair, const float* f32in, float* t,
                                                         float* u0, float* upair) {
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int2 rw = rows[r];
        const BInst& I = insts[rw.x];
        const int y = rw.y, nx = I.nx;
        const long long nt = (long long)nx * I.ny;
        const bool fy = I.ax[1].is_free[y] != 0;
        for (int x = threadIdx.x; x < I.px; x += blockDim.x) {
            const long long tp = I.poff + (long long)y * I.px + x;
            const long long g = (long long)y * nx + x;
            if (!IGAPW_IDX("batch elem row", y, I.ny) || (x < nx && !IGAPW_IDX("batch elem", g, nt))) continue;
            switch (mode) {
                case EL_PACK_HI: t[tp] = x < nx ? bpair[2 * I.off + g] : 0.f; break;
                case EL_PACK_F32: t[tp] = x < nx ? f32in[I.off + g] : 0.f; break;
                case EL_DIAG: t[tp] = t[tp] / (I.lamx[x] + I.lamy[y]); break;
                case EL_FIRST:
                    if (x < nx) u0[I.off + g] = (fy && I.ax[0].is_free[x]) ? t[tp] : bpair[2 * I.off + g];
                    break;
                case EL_FINAL:
                    if (x < nx) {
                        const float d = (fy && I.ax[0].is_free[x]) ? t[tp] : f32in[I.off + g];
                        float s, e;
                        two_sum(u0[I.off + g], d, s, e);
                        upair[2 * I.off + g] = s;
                        upair[2 * I.off + nt + g] = e;
                    }
                    break;
            }
        }
    }
}

struct Tile {
    int tx, ty;
};
const Tile kTiles[3] = {{32, 8}, {64, 4}, {16, 16}};

}  // namespace
}  // namespace igapw

using namespace igapw;

struct igapw_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int count = 0;
    std::vector<igapw_ctx*> ctx;
    std::vector<BInst> hinst;
    std::vector<long long> off, ntot;
    long long total = 0, ptotal = 0;
    BInst* dinst = nullptr;
    BSrc* dsrc = nullptr;
    float *b = nullptr, *u = nullptr, *u0 = nullptr, *rho = nullptr, *t0 = nullptr, *t1 = nullptr;
    int* counter = nullptr;      // [8] work-queue counters
    int2* rows = nullptr;
    int nrows = 0;
    // work items per tile shape (source: all instances; residual: per window width)
    int4* items[3] = {nullptr, nullptr, nullptr};
    int nitems[3] = {0, 0, 0};
    std::vector<int> wclass;     // distinct window widths
    std::vector<int4*> ritems[3];
    std::vector<int> rnitems[3];
    int src_tile = 0, res_tile = 0;
    // grouped GEMMs on the tensor cores (tcgemm.cuh): per stage the GEMM
    // descriptions, the tile work list, the tile width and which operand is
    // pre-split (the instance's W / V matrix)
    bool tc = true;
    TcGemmArgs* tg[4] = {nullptr, nullptr, nullptr, nullptr};
    int4* titems[4] = {nullptr, nullptr, nullptr, nullptr};
    int tn[4] = {0, 0, 0, 0}, tbn[4] = {0, 0, 0, 0}, tpre[4] = {0, 0, 0, 0};
    unsigned* status = nullptr;  // device status word (tensor-core wait timeouts)
    // grouped GEMMs on cuBLAS (IGAPW_FLAG_FDM_CUBLAS)
    cublasHandle_t blas = nullptr;
    void* blas_ws = nullptr;
    std::vector<int> gm[4], gn[4], gk[4], glda[4], gldb[4], gldc[4], gsize;
    std::vector<cublasOperation_t> gta[4], gtb[4];
    std::vector<float> galpha, gbeta;
    const float** gA[4] = {nullptr, nullptr, nullptr, nullptr};
    const float** gB[4] = {nullptr, nullptr, nullptr, nullptr};
    float** gC[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<void*> allocs;
    cudaGraphExec_t graph = nullptr;
    int sms = 152;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(igapw_batch* b, int code, const std::string& m) {
    if (b) b->err = m;
    else g_batch_error = m;
    return code;
}

#define BCK(b, x)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess)                                                                   \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? IGAPW_ERR_OOM : IGAPW_ERR_CUDA,     \
                         std::string(#x) + ": " + cudaGetErrorString(e_));                       \
    } while (0)
#define BBL(b, x)                                                                                \
    do {                                                                                         \
        cublasStatus_t e_ = (x);                                                                 \
        if (e_ != CUBLAS_STATUS_SUCCESS)                                                         \
            return bfail(b, IGAPW_ERR_CUDA, std::string(#x) + ": cublas status " + std::to_string((int)e_)); \
    } while (0)

template <typename T>
cudaError_t balloc(igapw_batch* b, T** p, size_t count) {
    cudaError_t e = cudaMallocAsync((void**)p, (count ? count : 1) * sizeof(T), b->stream);
    if (e == cudaSuccess) b->allocs.push_back(*p);
    return e;
}

template <typename T>
cudaError_t bupload(igapw_batch* b, T** p, const std::vector<T>& h) {
    cudaError_t e = balloc(b, p, h.size());
    if (e == cudaSuccess && !h.empty())
        e = cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream);
    return e;
}

std::vector<int4> make_items(const igapw_batch* b, const std::vector<int>& which, int tx, int ty) {
    std::vector<int4> it;
    for (int i : which) {
        const BInst& I = b->hinst[i];
        for (int y0 = 0; y0 < I.ny; y0 += ty)
            for (int x0 = 0; x0 < I.nx; x0 += tx) it.push_back(make_int4(i, x0, y0, 0));
    }
    // largest instances first: the tail of the queue is made of small tiles
    std::stable_sort(it.begin(), it.end(), [&](const int4& a, const int4& c) {
        return b->ntot[a.x] > b->ntot[c.x];
    });
    return it;
}

cudaError_t launch_source(igapw_batch* b, int tile) {
    cudaError_t e = cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)b->sms * 4;
    switch (tile) {
        case 0: batch_source_kernel<32, 8><<<grid, 256, 0, b->stream>>>(b->dinst, b->dsrc, b->items[0], b->nitems[0], b->counter, b->b); break;
        case 1: batch_source_kernel<64, 4><<<grid, 256, 0, b->stream>>>(b->dinst, b->dsrc, b->items[1], b->nitems[1], b->counter, b->b); break;
        default: batch_source_kernel<16, 16><<<grid, 256, 0, b->stream>>>(b->dinst, b->dsrc, b->items[2], b->nitems[2], b->counter, b->b); break;
    }
    return cudaGetLastError();
}

template <int W>
cudaError_t residual_w(igapw_batch* b, int tile, const int4* items, int n, int* counter) {
    const unsigned grid = (unsigned)b->sms * 4;
    switch (tile) {
        case 0: batch_residual_kernel<W, 32, 8><<<grid, 256, 0, b->stream>>>(b->dinst, items, n, counter, b->u0, b->b, b->rho); break;
        case 1: batch_residual_kernel<W, 64, 4><<<grid, 256, 0, b->stream>>>(b->dinst, items, n, counter, b->u0, b->b, b->rho); break;
        default: batch_residual_kernel<W, 16, 16><<<grid, 256, 0, b->stream>>>(b->dinst, items, n, counter, b->u0, b->b, b->rho); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_residual(igapw_batch* b, int tile) {
    for (size_t c = 0; c < b->wclass.size(); ++c) {
        int* counter = b->counter + 1 + c;
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), b->stream);
        if (e != cudaSuccess) return e;
        const int4* it = b->ritems[tile][c];
        const int n = b->rnitems[tile][c];
        switch (b->wclass[c]) {
            case 3: e = residual_w<3>(b, tile, it, n, counter); break;
            case 5: e = residual_w<5>(b, tile, it, n, counter); break;
            case 7: e = residual_w<7>(b, tile, it, n, counter); break;
            case 9: e = residual_w<9>(b, tile, it, n, counter); break;
            default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t elem(igapw_batch* b, int mode, const float* f32in) {
    const unsigned grid = (unsigned)std::min(b->nrows, b->sms * 16);
    batch_elem_kernel<<<grid, 256, 0, b->stream>>>(b->dinst, b->rows, b->nrows, mode, b->b, f32in, b->t0, b->u0, b->u);
    return cudaGetLastError();
}

int gemm_stage(igapw_batch* b, int s) {
    if (b->tc) {
        BCK(b, launch_tc_gemm_grouped(b->tg[s], b->titems[s], b->tn[s], b->tbn[s], b->tpre[s], b->stream));
        return IGAPW_OK;
    }
    BBL(b, cublasSgemmGroupedBatched(b->blas, b->gta[s].data(), b->gtb[s].data(), b->gm[s].data(), b->gn[s].data(),
                                     b->gk[s].data(), b->galpha.data(), b->gA[s], b->glda[s].data(), b->gB[s],
                                     b->gldb[s].data(), b->gbeta.data(), b->gC[s], b->gldc[s].data(), b->count,
                                     b->gsize.data()));
    return IGAPW_OK;
}

// P applied to t0 (padded): t1 = Wx t0, t0 = t1 Wy^T, diag, t1 = Vx t0, t0 = t1 Vy^T
int apply_p(igapw_batch* b) {
    int rc = gemm_stage(b, 0);
    if (!rc) rc = gemm_stage(b, 1);
    if (rc) return rc;
    BCK(b, elem(b, EL_DIAG, nullptr));
    rc = gemm_stage(b, 2);
    if (!rc) rc = gemm_stage(b, 3);
    return rc;
}

int enqueue_solve(igapw_batch* b) {
    BCK(b, elem(b, EL_PACK_HI, nullptr));
    int rc = apply_p(b);
    if (rc) return rc;
    BCK(b, elem(b, EL_FIRST, nullptr));
    BCK(b, launch_residual(b, b->res_tile));
    BCK(b, elem(b, EL_PACK_F32, b->rho));
    rc = apply_p(b);
    if (rc) return rc;
    BCK(b, elem(b, EL_FINAL, b->rho));
    return IGAPW_OK;
}

float time_it(igapw_batch* b, cudaError_t (*fn)(igapw_batch*, int), int tile) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fn(b, tile);
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < 3; ++r) fn(b, tile);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

void release_batch(igapw_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (void* p : b->allocs) cudaFreeAsync(p, b->stream);
    b->allocs.clear();
    if (b->blas) cublasDestroy(b->blas);
    b->blas = nullptr;
    for (igapw_ctx* c : b->ctx) igapw_destroy(c);
    b->ctx.clear();
    if (b->cap) cudaStreamDestroy(b->cap);
    b->cap = nullptr;
}

int build(igapw_batch* b, const igapw_desc* descs) {
    int dev = 0;
    BCK(b, cudaGetDevice(&dev));
    BCK(b, cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    BCK(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    b->hinst.resize(b->count);
    b->off.resize(b->count);
    b->ntot.resize(b->count);
    std::vector<int2> rows;
    for (int i = 0; i < b->count; ++i) {
        const igapw_desc& d = descs[i];
        if (d.dim != 2 || d.op != IGAPW_OP_POISSON || d.bc != IGAPW_BC_DIRICHLET0 || d.precision != IGAPW_FP32_REFINE)
            return bfail(b, IGAPW_ERR_ARG, "instance " + std::to_string(i) +
                                               ": the batch takes 2D POISSON, DIRICHLET0, FP32_REFINE descriptors");
        igapw_ctx* c = nullptr;
        int rc = igapw_create(&c, &d, b->stream);
        if (rc) return bfail(b, rc, "instance " + std::to_string(i) + ": " + igapw_last_error(nullptr));
        b->ctx.push_back(c);
        CtxView v{};
        ctx_view(c, v);
        BInst& I = b->hinst[i];
        I.nx = v.n[0];
        I.ny = v.n[1];
        I.W = v.W;
        I.px = v.fdm->px;
        I.off = b->total;
        I.poff = b->ptotal;
        I.qx = v.q[0];
        I.qy = v.q[1];
        I.ax[0] = v.ax[0];
        I.ax[1] = v.ax[1];
        I.qpx = v.qx[0];
        I.qpy = v.qx[1];
        I.lamx = v.fdm->lam[0];
        I.lamy = v.fdm->lam[1];
        b->off[i] = b->total;
        b->ntot[i] = v.ntot;
        b->total += v.ntot;
        b->ptotal += (long long)I.px * I.ny;
        for (int y = 0; y < I.ny; ++y) rows.push_back(make_int2(i, y));
        if (std::find(b->wclass.begin(), b->wclass.end(), I.W) == b->wclass.end()) b->wclass.push_back(I.W);
    }
    if (b->wclass.size() > 7) return bfail(b, IGAPW_ERR_ARG, "too many window widths");
    BCK(b, balloc(b, &b->b, 2 * b->total));
    BCK(b, balloc(b, &b->u, 2 * b->total));
    BCK(b, balloc(b, &b->u0, b->total));
    BCK(b, balloc(b, &b->rho, b->total));
    BCK(b, balloc(b, &b->t0, b->ptotal));
    BCK(b, balloc(b, &b->t1, b->ptotal));
    BCK(b, balloc(b, &b->counter, 8));
    BCK(b, bupload(b, &b->dinst, b->hinst));
    std::vector<BSrc> zero(b->count, BSrc{0.f, 1.f, 1.f, 0.f});
    BCK(b, bupload(b, &b->dsrc, zero));
    b->nrows = (int)rows.size();
    BCK(b, bupload(b, &b->rows, rows));
    // work items for every tile shape: source over all instances, residual per window width
    std::vector<int> all(b->count);
    std::iota(all.begin(), all.end(), 0);
    for (int t = 0; t < 3; ++t) {
        const auto it = make_items(b, all, kTiles[t].tx, kTiles[t].ty);
        b->nitems[t] = (int)it.size();
        BCK(b, bupload(b, &b->items[t], it));
        for (int w : b->wclass) {
            std::vector<int> sel;
            for (int i = 0; i < b->count; ++i)
                if (b->hinst[i].W == w) sel.push_back(i);
            const auto ri = make_items(b, sel, kTiles[t].tx, kTiles[t].ty);
            int4* d = nullptr;
            BCK(b, bupload(b, &d, ri));
            b->ritems[t].push_back(d);
            b->rnitems[t].push_back((int)ri.size());
        }
    }
    // grouped GEMM descriptions (column-major views of the (ny, px) row-major buffers)
    BBL(b, cublasCreate(&b->blas));
    BCK(b, cudaMallocAsync(&b->blas_ws, 32u << 20, b->stream));
    b->allocs.push_back(b->blas_ws);
    BBL(b, cublasSetWorkspace(b->blas, b->blas_ws, 32u << 20));
    BBL(b, cublasSetStream(b->blas, b->stream));
    b->gsize.assign(b->count, 1);
    b->galpha.assign(b->count, 1.f);
    b->gbeta.assign(b->count, 0.f);
    std::vector<const float*> A[4], B[4];
    std::vector<float*> C[4];
    for (int i = 0; i < b->count; ++i) {
        CtxView v{};
        ctx_view(b->ctx[i], v);
        const BInst& I = b->hinst[i];
        const FdmState& F = *v.fdm;
        const int ldx = F.axis[0]->np, ldy = F.axis[1]->np;
        float* T0 = b->t0 + I.poff;
        float* T1 = b->t1 + I.poff;
        // stage 0: T1 = Wx T0 ; 1: T0 = T1 Wy^T ; 2: T1 = Vx T0 ; 3: T0 = T1 Vy^T
        const float* Mx[2] = {F.Wm[0], F.Vm[0]};
        const float* My[2] = {F.Wm[1], F.Vm[1]};
        for (int h = 0; h < 2; ++h) {
            const int sx = 2 * h, sy = 2 * h + 1;
            b->gta[sx].push_back(CUBLAS_OP_N); b->gtb[sx].push_back(CUBLAS_OP_N);
            b->gm[sx].push_back(I.px); b->gn[sx].push_back(I.ny); b->gk[sx].push_back(I.px);
            b->glda[sx].push_back(ldx); b->gldb[sx].push_back(I.px); b->gldc[sx].push_back(I.px);
            A[sx].push_back(Mx[h]); B[sx].push_back(T0); C[sx].push_back(T1);
            b->gta[sy].push_back(CUBLAS_OP_N); b->gtb[sy].push_back(CUBLAS_OP_T);
            b->gm[sy].push_back(I.px); b->gn[sy].push_back(I.ny); b->gk[sy].push_back(I.ny);
            b->glda[sy].push_back(I.px); b->gldb[sy].push_back(ldy); b->gldc[sy].push_back(I.px);
            A[sy].push_back(T1); B[sy].push_back(My[h]); C[sy].push_back(T0);
        }
    }
    for (int s = 0; s < 4; ++s) {
        BCK(b, bupload(b, &b->gA[s], A[s]));
        BCK(b, bupload(b, &b->gB[s], B[s]));
        BCK(b, bupload(b, &b->gC[s], C[s]));
    }
    // the same GEMMs on the tensor cores: x stages take the x matrix as A
    // (pre-split, tile rows 128), y stages the y matrix as B (pre-split with
    // the y stages' common tile width)
    b->tc = !(descs[0].flags & IGAPW_FLAG_FDM_CUBLAS);
    if (b->tc) {
        BCK(b, balloc(b, &b->status, 1));
        BCK(b, cudaMemsetAsync(b->status, 0, sizeof(unsigned), b->stream));
        std::vector<TcGemmArgs> G[4];
        for (int i = 0; i < b->count; ++i) {
            for (int s = 0; s < 4; ++s) {
                TcGemmArgs g{};
                g.M = b->gm[s][i]; g.N = b->gn[s][i]; g.K = b->gk[s][i]; g.batch = 1;
                g.A = A[s][i]; g.sAm = 1; g.sAk = b->glda[s][i];
                if (b->gtb[s][i] == CUBLAS_OP_N) { g.B = B[s][i]; g.sBn = b->gldb[s][i]; g.sBk = 1; }
                else { g.B = B[s][i]; g.sBn = 1; g.sBk = b->gldb[s][i]; }
                g.D = C[s][i]; g.sDm = 1; g.sDn = b->gldc[s][i];
                g.status = b->status;
                G[s].push_back(g);
            }
        }
        for (int s = 0; s < 4; ++s) {
            const bool xstage = (s % 2) == 0;
            b->tpre[s] = xstage ? 1 : 2;
            b->tbn[s] = tc_pick_width(G[s].data(), (int)G[s].size(), b->sms);
            std::vector<CUtensorMap> maps(G[s].size());
            std::vector<char> has_map(G[s].size(), 0);
            for (size_t gi = 0; gi < G[s].size(); ++gi) {
                TcGemmArgs& g = G[s][gi];
                // the live operand (spectral buffer) by TMA: B of the x stages
                // (tiles of the stage's width), A of the y stages (128 rows)
                has_map[gi] = xstage ? tc_make_tmap(&maps[gi], g.B, g.sBn, g.sBk, g.bB, g.N, g.K, 1, b->tbn[s])
                                     : tc_make_tmap(&maps[gi], g.A, g.sAm, g.sAk, g.bA, g.M, g.K, 1, tc::BM);
                const int R = xstage ? tc::BM : b->tbn[s];
                const int rows = xstage ? g.M : g.N;
                float* pre = nullptr;
                BCK(b, balloc(b, &pre, (size_t)tc_presplit_floats(rows, g.K, R, !xstage)));
                if (xstage) {
                    BCK(b, launch_tc_presplit(g.A, g.sAm, g.sAk, rows, g.K, R, false, pre, b->stream));
                    g.A = pre;
                } else {
                    BCK(b, launch_tc_presplit(g.B, g.sBn, g.sBk, rows, g.K, R, true, pre, b->stream));
                    g.B = pre;
                }
                g.pre = b->tpre[s];
                g.bn = b->tbn[s];
            }
            CUtensorMap* dmaps = nullptr;
            BCK(b, bupload(b, &dmaps, maps));
            for (size_t gi = 0; gi < G[s].size(); ++gi)
                if (has_map[gi]) {
                    G[s][gi].tmap = dmaps + gi;
                    G[s][gi].tmap_rows = xstage ? b->tbn[s] : tc::BM;
                }
            const std::vector<int4> items = tc_group_items(G[s], b->tbn[s]);
            b->tn[s] = (int)items.size();
            BCK(b, bupload(b, &b->tg[s], G[s]));
            BCK(b, bupload(b, &b->titems[s], items));
        }
    }
    // tile autotuning on the batch itself (zero inputs)
    BCK(b, cudaMemsetAsync(b->b, 0, 2 * b->total * sizeof(float), b->stream));
    BCK(b, cudaMemsetAsync(b->u0, 0, b->total * sizeof(float), b->stream));
    float best_s = 1e30f, best_r = 1e30f;
    for (int t = 0; t < 3; ++t) {
        const float ts = time_it(b, launch_source, t);
        const float tr = time_it(b, launch_residual, t);
        if (ts < best_s) { best_s = ts; b->src_tile = t; }
        if (tr < best_r) { best_r = tr; b->res_tile = t; }
    }
    BCK(b, cudaGetLastError());
    BCK(b, cudaStreamSynchronize(b->stream));
    return IGAPW_OK;
}

}  // namespace

extern "C" {

int igapw_batch_create(igapw_batch** out, const igapw_desc* descs, int count, void* cuda_stream) {
    if (!out) return bfail(nullptr, IGAPW_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || count <= 0) return bfail(nullptr, IGAPW_ERR_ARG, "need count >= 1 descriptors");
    igapw_batch* b = new (std::nothrow) igapw_batch();
    if (!b) return bfail(nullptr, IGAPW_ERR_OOM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->count = count;
    const int rc = build(b, descs);
    if (rc) {
        g_batch_error = b->err;
        release_batch(b);
        delete b;
        return rc;
    }
    *out = b;
    return IGAPW_OK;
}

int igapw_batch_source_sine(igapw_batch* b, const double* params) {
    if (!b) return bfail(nullptr, IGAPW_ERR_ARG, "batch is NULL");
    if (!params) return bfail(b, IGAPW_ERR_ARG, "params is NULL");
    std::vector<BSrc> s(b->count);
    for (int i = 0; i < b->count; ++i)
        s[i] = BSrc{(float)params[3 * i], (float)params[3 * i + 1], (float)params[3 * i + 2], 0.f};
    // the copy is stream-ordered; the host vector must live until it has run
    BCK(b, cudaMemcpyAsync(b->dsrc, s.data(), s.size() * sizeof(BSrc), cudaMemcpyHostToDevice, b->stream));
    BCK(b, launch_source(b, b->src_tile));
    BCK(b, cudaStreamSynchronize(b->stream));
    return IGAPW_OK;
}

int igapw_batch_solve(igapw_batch* b) {
    if (!b) return bfail(nullptr, IGAPW_ERR_ARG, "batch is NULL");
    if (!b->graph) {
        BBL(b, cublasSetStream(b->blas, b->cap));
        cudaStream_t keep = b->stream;
        b->stream = b->cap;
        BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
        const int rc = enqueue_solve(b);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        b->stream = keep;
        cublasSetStream(b->blas, b->stream);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        BCK(b, e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(b, e);
    }
    BCK(b, cudaGraphLaunch(b->graph, b->stream));
    return IGAPW_OK;
}

int igapw_batch_sync_status(igapw_batch* b) {
    if (!b) return bfail(nullptr, IGAPW_ERR_ARG, "batch is NULL");
    BCK(b, cudaStreamSynchronize(b->stream));
    if (!b->status) return IGAPW_OK;
    unsigned st = 0;
    BCK(b, cudaMemcpy(&st, b->status, sizeof st, cudaMemcpyDeviceToHost));
    if (st & STATUS_TC_TIMEOUT)
        return bfail(b, IGAPW_ERR_TIMEOUT, "a tensor-core GEMM of the batch solve timed out waiting for its pipeline");
    return IGAPW_OK;
}

int igapw_batch_tensor(igapw_batch* b, int i, int which, void** dev, long long* n_total) {
    if (!b) return bfail(nullptr, IGAPW_ERR_ARG, "batch is NULL");
    if (i < 0 || i >= b->count || (which != 0 && which != 1) || !dev)
        return bfail(b, IGAPW_ERR_ARG, "bad instance, tensor or output");
    *dev = (which == 0 ? b->b : b->u) + 2 * b->off[i];
    if (n_total) *n_total = b->ntot[i];
    return IGAPW_OK;
}

int igapw_batch_info(igapw_batch* b, int* tiles) {
    if (!b) return bfail(nullptr, IGAPW_ERR_ARG, "batch is NULL");
    if (tiles) {
        tiles[0] = kTiles[b->src_tile].tx;
        tiles[1] = kTiles[b->src_tile].ty;
        tiles[2] = kTiles[b->res_tile].tx;
        tiles[3] = kTiles[b->res_tile].ty;
    }
    return IGAPW_OK;
}

const char* igapw_batch_last_error(igapw_batch* b) {
    if (!b) return g_batch_error.c_str();
    return b->err.c_str();
}

int igapw_batch_destroy(igapw_batch* b) {
    if (!b) return IGAPW_OK;
    release_batch(b);
    delete b;
    return IGAPW_OK;
}

}  // extern "C"
