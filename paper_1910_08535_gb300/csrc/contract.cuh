#pragma once
// Kernel (b): sum-factorised per-axis contractions of the coefficient tensor
// with the folded quadrature tables.
//
// Operator action (MODE_OP).  The tested operator of u + beta Lap u with tests
// T = T_x T_y T_z (PW indicators or B-splines) factorises per axis into the
// folded tables A = int T_i B_j and C = int T_i B_j'':
//   r = A_x [ alpha A_y A_z u + beta (C_y A_z u + A_y C_z u) ] + beta C_x [ A_y A_z u ]
// computed as z-pass (ZA = A_z u, ZC = C_z u), y-pass (Q1 = A_y ZA,
// Q2 = alpha Q1 + beta (C_y ZA + A_y ZC)), x-pass (r = A_x Q2 + beta C_x Q1):
// 7 banded passes.  The quadrature itself lives in the tables: kernel (a)
// summed w_q B_j(x_q) over each cell (PW: the test is 1) or multiplied by the
// test B-spline (Galerkin).
//
// A block owns an x-tile x a y-tile of outputs for a chunk of z-planes.  It
// streams z: a ring of W input planes (with the x/y halo the windows need) is
// refilled one plane at a time, so every input plane is read once per block.
//
// MODE_SYS applies the factored system S_z S_y S_x; MODE_RES forms the
// refinement residual r - S u0 (FP64 or double-float arithmetic).
//
// MODE_PK / MODE_PRES: the multi-D Poisson operator K of Sec. 4.3,
// sum_a (-C_a) (x) A_others on rows off the boundary (the operator pass with
// alpha = 0, beta = -1; the 1D tables keep their true rows there, so columns on
// the boundary contribute), and the identity on boundary rows (any axis index
// a Dirichlet row).  PK writes K u, PRES the FP32 residual r - K u.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace igapw {

template <typename CT>
struct Acc;
template <>
struct Acc<double> {
    double s;
    __device__ __forceinline__ void init() { s = 0.0; }
    __device__ __forceinline__ void add_prod(double t, double v) { s = fma(t, v, s); }
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double result() const { return s; }
};
template <>
struct Acc<DF> : DFAcc {};

template <typename CT>
struct SBuf;
template <>
struct SBuf<double> {
    double* p;
    __device__ __forceinline__ double ld(int i) const { return p[i]; }
    __device__ __forceinline__ void st(int i, double v) const { p[i] = v; }
    static constexpr int bytes = 8;
    __device__ __forceinline__ void carve(unsigned char*& base, int count) {
        p = reinterpret_cast<double*>(base);
        base += (size_t)count * 8;
    }
};
template <>
struct SBuf<DF> {
    float2* p;   // (hi, lo) interleaved: one 8-byte access per value
    __device__ __forceinline__ DF ld(int i) const {
        const float2 v = p[i];
        return DF{v.x, v.y};
    }
    __device__ __forceinline__ void st(int i, DF v) const { p[i] = make_float2(v.hi, v.lo); }
    static constexpr int bytes = 8;
    __device__ __forceinline__ void carve(unsigned char*& base, int count) {
        p = reinterpret_cast<float2*>(base);
        base += (size_t)count * 8;
    }
};

template <typename CT>
__device__ __forceinline__ CT tab(const TableSet& t, int idx);
template <>
__device__ __forceinline__ double tab<double>(const TableSet& t, int idx) { return __ldg(t.d + idx); }
template <>
__device__ __forceinline__ DF tab<DF>(const TableSet& t, int idx) {
    const float2 v = __ldg(t.df + idx);
    return DF{v.x, v.y};
}

template <typename CT>
__device__ __forceinline__ CT zero_v();
template <>
__device__ __forceinline__ double zero_v<double>() { return 0.0; }
template <>
__device__ __forceinline__ DF zero_v<DF>() { return DF{0.f, 0.f}; }

template <typename CT>
__device__ __forceinline__ CT from_double(double v);
template <>
__device__ __forceinline__ double from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ DF from_double<DF>(double v) {
    DF r;
    split_double(v, r.hi, r.lo);
    return r;
}

template <int MODE>
constexpr bool op_tables() { return MODE == MODE_OP || MODE == MODE_PK || MODE == MODE_PRES; }

// coefficient input u (MODE_OP / SYS / PK), u0 (MODE_RES), u (MODE_PRES:
// F32 with pair r, F64 with F64 r)
template <typename CT, int MODE, int IO>
__device__ __forceinline__ CT load_u(const ContractArgs& a, long long g) {
    if (!IGAPW_IDX("contract load_u", g, a.ntot)) return CT{};
    if constexpr (MODE == MODE_RES || (MODE == MODE_PRES && IO == FMT_PAIR)) {
        const float v = ((const float*)a.u)[g];
        if constexpr (std::is_same<CT, double>::value) return (double)v;
        else return DF{v, 0.f};
    } else if constexpr (IO == FMT_F64) {
        return ((const double*)a.u)[g];
    } else {
        const float* u = (const float*)a.u;
        return DF{u[g], u[g + a.ntot]};
    }
}

template <typename CT, int MODE, int IO>
__device__ __forceinline__ void store_r(const ContractArgs& a, long long g, CT v) {
    if (!IGAPW_IDX("contract store_r", g, a.ntot)) return;
    if constexpr (MODE == MODE_PRES && IO == FMT_F64) {
        ((float*)a.out)[g] = (float)(((const double*)a.r)[g] - v);
    } else if constexpr (MODE == MODE_RES || MODE == MODE_PRES) {
        const float* r = (const float*)a.r;
        if constexpr (std::is_same<CT, DF>::value) {
            DFAcc acc;
            acc.s = r[g];
            acc.c = r[g + a.ntot];
            acc.add(DF{-v.hi, -v.lo});
            ((float*)a.out)[g] = acc.result().hi;
        } else {
            const double rr = (double)r[g] + (double)r[g + a.ntot];
            ((float*)a.out)[g] = (float)(rr - v);
        }
    } else if constexpr (IO == FMT_F64) {
        ((double*)a.out)[g] = v;
    } else {
        ((float*)a.out)[g] = v.hi;
        ((float*)a.out)[g + a.ntot] = v.lo;
    }
}

// Row/column iteration over a rows x cols tile with a fixed thread stride,
// without an integer division per element.
struct Iter2 {
    int r, c, dr, dc, cols;
    __device__ __forceinline__ Iter2(int cols_, int start, int stride) : cols(cols_) {
        r = start / cols;
        c = start - r * cols;
        dr = stride / cols;
        dc = stride - dr * cols;
    }
    __device__ __forceinline__ void next() {
        c += dc;
        r += dr;
        if (c >= cols) {
            c -= cols;
            ++r;
        }
    }
};

template <int DIM, int W, int TX, int TY, typename CT, int MODE, int IO>
__global__ void __launch_bounds__(256) contract_kernel(const ContractArgs a) {
    constexpr bool OP = op_tables<MODE>();
    constexpr int XH = TX + W - 1;
    constexpr int YH = DIM >= 2 ? TY + W - 1 : 1;
    constexpr int TYE = DIM >= 2 ? TY : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const AxisDev& AX = a.ax[0];
    const AxisDev& AY = a.ax[1];
    const AxisDev& AZ = a.ax[2];
    const int x0 = blockIdx.x * a.tx;
    const int y0 = DIM >= 2 ? blockIdx.y * a.ty : 0;
    const int nxo = min(a.tx, nx - x0);
    const int nyo = DIM >= 2 ? min(a.ty, ny - y0) : 1;
    const int xl = AX.fstart[x0];
    const int nxh = AX.fstart[x0 + nxo - 1] + W - xl;
    const int yl = DIM >= 2 ? AY.fstart[y0] : 0;
    const int nyh = DIM >= 2 ? AY.fstart[y0 + nyo - 1] + W - yl : 1;
    const long long plane = (long long)nx * ny;

    unsigned char* base = smem_raw;
    SBuf<CT> ring, ZA, ZC, Q1, Q2;
    if constexpr (DIM == 3) ring.carve(base, W * YH * XH);
    if constexpr (DIM >= 2) ZA.carve(base, YH * XH);
    if constexpr (DIM == 3 && OP) ZC.carve(base, YH * XH);
    Q1.carve(base, TYE * XH);
    if constexpr (OP) Q2.carve(base, TYE * XH);

    const CT alpha = from_double<CT>(a.alpha);
    const CT beta = from_double<CT>(a.beta);
    const TableSet& TYa = OP ? AY.A : AY.S;
    const TableSet& TZa = OP ? AZ.A : AZ.S;

    // x-pass over the y-rows of Q1/Q2 for output plane zo, then store
    auto x_pass = [&](int zo) {
        for (Iter2 it(nxo, threadIdx.x, blockDim.x); it.r < nyo; it.next()) {
            const int y = it.r, x = it.c;
            const int xc = x0 + x;
            const int sx = AX.fstart[xc] - xl;
            const int qb = y * XH + sx;
            Acc<CT> r1, r2;
            r1.init();
            r2.init();
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if constexpr (OP) {
                    r1.add_prod(tab<CT>(AX.A, xc * W + w), Q2.ld(qb + w));
                    r2.add_prod(tab<CT>(AX.C, xc * W + w), Q1.ld(qb + w));
                } else {
                    r1.add_prod(tab<CT>(AX.S, xc * W + w), Q1.ld(qb + w));
                }
            }
            CT v;
            if constexpr (OP) {
                Acc<CT> t;
                t.init();
                t.add(r1.result());
                t.add_prod(beta, r2.result());
                v = t.result();
            } else {
                v = r1.result();
            }
            const long long g = (long long)zo * plane + (long long)(y0 + y) * nx + xc;
            if constexpr (MODE == MODE_PK || MODE == MODE_PRES) {
                bool fr = AX.is_free[xc] != 0;
                if constexpr (DIM >= 2) fr = fr && AY.is_free[y0 + y] != 0;
                if constexpr (DIM == 3) fr = fr && AZ.is_free[zo] != 0;
                if (!fr) v = load_u<CT, MODE, IO>(a, g);
            }
            store_r<CT, MODE, IO>(a, g, v);
        }
    };

    // y-pass: ZA (and ZC) rows -> Q1 (and Q2)
    auto y_pass = [&]() {
        for (Iter2 it(nxh, threadIdx.x, blockDim.x); it.r < nyo; it.next()) {
            const int y = it.r, xx = it.c;
            const int yr = y0 + y;
            const int sy = AY.fstart[yr] - yl;
            Acc<CT> q1;
            q1.init();
            if constexpr (OP) {
                Acc<CT> t2;
                t2.init();
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const CT za = ZA.ld((sy + w) * XH + xx);
                    const CT ta = tab<CT>(AY.A, yr * W + w);
                    q1.add_prod(ta, za);
                    t2.add_prod(tab<CT>(AY.C, yr * W + w), za);
                    if constexpr (DIM == 3) t2.add_prod(ta, ZC.ld((sy + w) * XH + xx));
                }
                const CT v1 = q1.result();
                Acc<CT> q2;
                q2.init();
                q2.add_prod(alpha, v1);
                q2.add_prod(beta, t2.result());
                Q1.st(y * XH + xx, v1);
                Q2.st(y * XH + xx, q2.result());
            } else {
#pragma unroll
                for (int w = 0; w < W; ++w) q1.add_prod(tab<CT>(TYa, yr * W + w), ZA.ld((sy + w) * XH + xx));
                Q1.st(y * XH + xx, q1.result());
            }
        }
    };

    if constexpr (DIM == 1) {
        for (int e = threadIdx.x; e < nxh; e += blockDim.x) {
            const int gx = xl + e;
            const CT v = gx < nx ? load_u<CT, MODE, IO>(a, gx) : zero_v<CT>();
            Q1.st(e, v);
            if constexpr (OP) {
                Acc<CT> t;
                t.init();
                t.add_prod(alpha, v);
                Q2.st(e, t.result());
            }
        }
        __syncthreads();
        x_pass(0);
    } else if constexpr (DIM == 2) {
        for (Iter2 it(nxh, threadIdx.x, blockDim.x); it.r < nyh; it.next()) {
            const int gy = yl + it.r, gx = xl + it.c;
            ZA.st(it.r * XH + it.c, (gy < ny && gx < nx) ? load_u<CT, MODE, IO>(a, (long long)gy * nx + gx) : zero_v<CT>());
        }
        __syncthreads();
        y_pass();
        __syncthreads();
        x_pass(0);
    } else {
        const int z0 = blockIdx.z * a.zchunk;
        const int z1 = min(z0 + a.zchunk, nz);
        // this thread's elements of a halo plane: e = threadIdx.x + k * 256
        constexpr int PF = (YH * XH + 255) / 256;
        int poff[PF];        // ring offset (row * XH + col), -1 if none
        long long pg[PF];    // global offset within a z-plane, -1 if outside the tensor
        {
            Iter2 it(nxh, threadIdx.x, 256);
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const bool in = it.r < nyh;
                const int gy = yl + it.r, gx = xl + it.c;
                poff[k] = in ? it.r * XH + it.c : -1;
                pg[k] = (in && gy < ny && gx < nx) ? (long long)gy * nx + gx : -1;
                it.next();
            }
        }
        auto plane_val = [&](int z, int k) {
            CT v = zero_v<CT>();
            if (z < nz && pg[k] >= 0) v = load_u<CT, MODE, IO>(a, (long long)z * plane + pg[k]);
            return v;
        };
        // register prefetch of the plane the next output plane needs, issued
        // before this plane's z-pass and committed to the ring after it
        CT pf[PF];
        int rhi = AZ.fstart[z0];
        for (int zo = z0; zo < z1; ++zo) {
            const int zs = AZ.fstart[zo];
            while (rhi < zs + W) {          // fill (first plane of the chunk only)
                const int slot = (rhi % W) * (YH * XH);
#pragma unroll
                for (int k = 0; k < PF; ++k) pf[k] = plane_val(rhi, k);
#pragma unroll
                for (int k = 0; k < PF; ++k)
                    if (poff[k] >= 0) ring.st(slot + poff[k], pf[k]);
                ++rhi;
            }
            const bool pre = (zo + 1 < z1) && (AZ.fstart[zo + 1] + W > rhi);
            if (pre) {
#pragma unroll
                for (int k = 0; k < PF; ++k) pf[k] = plane_val(rhi, k);
            }
            // this plane's z tables, uniform over the block
            CT tza[W], tzc[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                tza[w] = tab<CT>(TZa, zo * W + w);
                if constexpr (OP) tzc[w] = tab<CT>(AZ.C, zo * W + w);
            }
            int slot_w[W];
#pragma unroll
            for (int w = 0; w < W; ++w) slot_w[w] = ((zs + w) % W) * (YH * XH);
            __syncthreads();
            // z-pass
            for (Iter2 it(nxh, threadIdx.x, blockDim.x); it.r < nyh; it.next()) {
                const int off = it.r * XH + it.c;
                Acc<CT> za, zc;
                za.init();
                zc.init();
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const CT v = ring.ld(slot_w[w] + off);
                    za.add_prod(tza[w], v);
                    if constexpr (OP) zc.add_prod(tzc[w], v);
                }
                ZA.st(off, za.result());
                if constexpr (OP) ZC.st(off, zc.result());
            }
            __syncthreads();
            if (pre) {                      // slot of plane zs is free now
                const int slot = (rhi % W) * (YH * XH);
#pragma unroll
                for (int k = 0; k < PF; ++k)
                    if (poff[k] >= 0) ring.st(slot + poff[k], pf[k]);
                ++rhi;
            }
            y_pass();
            __syncthreads();
            x_pass(zo);
            __syncthreads();
        }
    }
}

template <int DIM, int W, int TX, int TY, typename CT, int MODE, int IO>
static cudaError_t run_contract(const ContractArgs& a, cudaStream_t st) {
    constexpr bool OP = op_tables<MODE>();
    constexpr int XH = TX + W - 1;
    constexpr int YH = DIM >= 2 ? TY + W - 1 : 1;
    constexpr int TYE = DIM >= 2 ? TY : 1;
    size_t elems = 0;
    if (DIM == 3) elems += (size_t)W * YH * XH;
    if (DIM >= 2) elems += (size_t)YH * XH;
    if (DIM == 3 && OP) elems += (size_t)YH * XH;
    elems += (size_t)TYE * XH * (OP ? 2 : 1);
    const size_t sm = elems * 8;
    auto k = contract_kernel<DIM, W, TX, TY, CT, MODE, IO>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    // balanced runtime tiles: the fewest tiles of at most TX (TY), evenly sized
    ContractArgs b = a;
    const int ntx = (a.n[0] + TX - 1) / TX;
    b.tx = (a.n[0] + ntx - 1) / ntx;
    const int nty = DIM >= 2 ? (a.n[1] + TY - 1) / TY : 1;
    b.ty = DIM >= 2 ? (a.n[1] + nty - 1) / nty : 1;
    int nz_blocks = 1;
    if (DIM == 3) {
        // z-chunks: about 4 resident blocks per SM over the grid
        const long long want = 4LL * 152;
        long long chunks = (want + (long long)ntx * nty - 1) / ((long long)ntx * nty);
        if (chunks < 1) chunks = 1;
        b.zchunk = (int)((a.n[2] + chunks - 1) / chunks);
        if (b.zchunk < 4) b.zchunk = 4;
        nz_blocks = (a.n[2] + b.zchunk - 1) / b.zchunk;
    }
    dim3 grid((a.n[0] + b.tx - 1) / b.tx, DIM >= 2 ? (a.n[1] + b.ty - 1) / b.ty : 1, nz_blocks);
    k<<<grid, 256, sm, st>>>(b);
    return cudaGetLastError();
}

template <int DIM, int W, typename CT, int MODE, int IO>
static cudaError_t pick_tile(const ContractArgs& a, cudaStream_t st) {
    if constexpr (DIM == 1) return run_contract<1, W, 256, 1, CT, MODE, IO>(a, st);
    else if constexpr (DIM == 2) return run_contract<2, W, 64, 8, CT, MODE, IO>(a, st);
    else return run_contract<3, W, 48, 8, CT, MODE, IO>(a, st);
}


}  // namespace igapw
