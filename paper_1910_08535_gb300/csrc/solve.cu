// Kernel (c2): batched banded line solves along one axis of the coefficient
// tensor (one batch of 1D systems with many right-hand sides per axis, the
// alternating-directions solve of Sec. 4.1).
//
// A line is split into P contiguous chunks (P a power of two <= 32, chunks of
// about 16 rows), one per lane of a lane group; a warp holds 32/P groups and
// every group solves NB lines at once (independent recurrences interleaved).
// Forward substitution L y = r: each lane solves its chunk with the previous
// chunk's tail taken as zero, the true tails follow from a Hillis-Steele scan
// over the group's lanes (p x p operators precomputed per lane and level), and
// a rank-p spike correction finishes the chunk (fused into the backward sweep).
// Backward substitution U x = y mirrors it with heads and a reverse scan.
// Lines are staged in shared memory with coalesced loads (x-lines row by row,
// y- and z-lines as 32-wide column blocks); the tables are staged once per
// block.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "linesolve.cuh"

namespace igapw {

template <typename T, int IN>
__device__ __forceinline__ T load_in(const void* p, long long g) {
    if constexpr (IN == FMT_F64) return (T)((const double*)p)[g];
    else return (T)((const float*)p)[g];   // FMT_F32, or the hi plane of FMT_PAIR
}

template <typename T, int OUT>
__device__ __forceinline__ void store_out(const SolveArgs& s, long long g, T v, unsigned& bad) {
    if constexpr (OUT == FMT_F64) {
        ((double*)s.out)[g] = (double)v;
        if (!isfinite((double)v)) bad = 1;
    } else if constexpr (OUT == FMT_F32) {
        ((float*)s.out)[g] = (float)v;
    } else {
        // finish: state = u0 + correction as a normalized pair
        float hi, lo;
        two_sum(s.u0[g], (float)v, hi, lo);
        ((float*)s.out)[g] = hi;
        ((float*)s.out)[g + s.ntot] = lo;
        if (!isfinite(hi)) bad = 1;
    }
}

// x-lines (contiguous): a block stages lpb consecutive lines, odd pitch.
template <typename T, int KP, int IN, int OUT, int NB>
__global__ void __launch_bounds__(256) solve_x_kernel(SolveArgs s, LineSys<T> S, int lpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tabs = reinterpret_cast<T*>(smem_raw);
    const int nx = s.n[0];
    T* buf = tabs + table_elems<T, KP>(nx, S.P);
    __shared__ int bnd[33];
    const int pitch = nx | 1;   // odd pitch: lanes on different lines hit different banks
    const long long nlines = (long long)s.n[1] * s.n[2];
    const long long l0 = (long long)blockIdx.x * lpb;
    const int nl = (int)min((long long)lpb, nlines - l0);
    const SolveSmem<T> st = stage_tables<T, KP>(S, tabs);
    for (int e = threadIdx.x; e < 33; e += blockDim.x) bnd[e] = S.b[e];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    // warp per line, lane per row: coalesced, no index division
    for (int l = warp; l < nl; l += nw) {
        const T* src = nullptr;
        const long long g0 = (l0 + l) * nx;
        T v[8];
        for (int i0 = 0; i0 < nx; i0 += 256) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * 32 + lane;
                if (i < nx) v[u] = load_in<T, IN>(s.in, g0 + i);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * 32 + lane;
                if (i < nx) buf[l * pitch + i] = v[u];
            }
        }
        (void)src;
    }
    cp_async_wait_all();
    __syncthreads();
    const int P = S.P;
    const int groups = 32 / P;
    const int grp = lane / P, k = lane - grp * P;
    const int per_warp = groups * NB;
    // warp w takes line sets w, w + nw, ... of per_warp lines; group g the NB after g*NB
    for (int base = warp * per_warp; base < nl; base += nw * per_warp) {
        const int first = base + grp * NB;
        const int nb = max(0, min(NB, nl - first));
        line_solve<T, KP, NB>(buf + (size_t)min(first, nl) * pitch, 1, pitch, nb, st, P, bnd, k, nx);
    }
    __syncthreads();
    unsigned bad = 0;
    for (int l = warp; l < nl; l += nw) {
        const long long g0 = (l0 + l) * nx;
        for (int i = lane; i < nx; i += 32) store_out<T, OUT>(s, g0 + i, buf[l * pitch + i], bad);
    }
    if (bad && s.status) atomicOr(s.status, STATUS_NONFINITE);
}

// Lines along y (os = n_y n_x, rs = n_x, outer = z) or z (os = n_x,
// rs = n_x n_y, outer = y); element (outer o, row i, column x) at
// o*os + i*rs + x.  A block stages 32 consecutive x for NO outer indices and
// all rows: line (o, c) is column o*32 + c of a [row][NO*32 + 1] buffer.
template <typename T, int KP, int IN, int OUT, int NB>
__global__ void __launch_bounds__(256) solve_strided_kernel(SolveArgs s, LineSys<T> S, int nline, int outer,
                                                            int NO, int lgNO, long long os, long long rs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tabs = reinterpret_cast<T*>(smem_raw);
    T* buf = tabs + table_elems<T, KP>(nline, S.P);
    __shared__ int bnd[33];
    const int nx = s.n[0];
    const int x0 = blockIdx.x * 32;
    const int nc = min(32, nx - x0);
    const int o0 = blockIdx.y * NO;
    const int no = min(NO, outer - o0);
    const int pitch = NO * 32 + 1;
    const SolveSmem<T> st = stage_tables<T, KP>(S, tabs);
    for (int e = threadIdx.x; e < 33; e += blockDim.x) bnd[e] = S.b[e];
    const int cols = NO * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    // warp per (row, outer) segment of 32 columns, lane per column
    const int tot = nline * NO;
    const bool colok = lane < nc;
    const long long gbase = (long long)o0 * os + x0 + lane;
    for (int b0 = warp; b0 < tot; b0 += nw * 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = b0 + u * nw;
            const int i = idx >> lgNO, o = idx & (NO - 1);
            v[u] = (idx < tot && colok && o < no) ? load_in<T, IN>(s.in, gbase + o * os + (long long)i * rs) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = b0 + u * nw;
            if (idx < tot) buf[(idx >> lgNO) * pitch + (idx & (NO - 1)) * 32 + lane] = v[u];
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int P = S.P;
    const int groups = 32 / P;
    const int grp = lane / P, k = lane - grp * P;
    const int per_warp = groups * NB;
    for (int base = warp * per_warp; base < cols; base += nw * per_warp) {
        const int first = base + grp * NB;
        const int nb = max(0, min(NB, cols - first));
        line_solve<T, KP, NB>(buf + min(first, cols), pitch, 1, nb, st, P, bnd, k, nline);
    }
    __syncthreads();
    unsigned bad = 0;
    for (int idx = warp; idx < tot; idx += nw) {
        const int i = idx >> lgNO, o = idx & (NO - 1);
        if (colok && o < no) store_out<T, OUT>(s, gbase + o * os + (long long)i * rs, buf[i * pitch + o * 32 + lane], bad);
    }
    if (bad && s.status) atomicOr(s.status, STATUS_NONFINITE);
}

// Long y/z-lines (the 32-column block of solve_strided_kernel does not fit):
// CW columns (a power of two <= 32) of one outer index per block, lane ->
// (column lane % CW, row offset lane / CW); the tables are read from global
// memory (all lanes of a lane group read the same row: broadcast L1 accesses).
template <typename T, int KP, int IN, int OUT>
__global__ void __launch_bounds__(256) solve_cols_kernel(SolveArgs s, LineSys<T> S, int nline, int CW, int lgCW,
                                                         long long os, long long rs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);
    __shared__ int bnd[33];
    const int nx = s.n[0];
    const int x0 = blockIdx.x * CW;
    const int nc = min(CW, nx - x0);
    const int pitch = CW + 1;
    const SolveSmem<T> st{S.L, S.U, S.dinv, S.G, S.H, S.PhiF, S.PhiB, 32};
    for (int e = threadIdx.x; e < 33; e += blockDim.x) bnd[e] = S.b[e];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = lane & (CW - 1), r0 = lane >> lgCW, rpw = 32 >> lgCW;
    const long long gbase = (long long)blockIdx.y * os + x0 + c;
    for (int i = warp * rpw + r0; i < nline; i += nw * rpw) {
        if (!IGAPW_IDX("cols smem", i * pitch + c, nline * pitch)) continue;
        if (c < nc && !IGAPW_IDX("cols g", gbase + (long long)i * rs, s.ntot)) continue;
        buf[i * pitch + c] = c < nc ? load_in<T, IN>(s.in, gbase + (long long)i * rs) : T(0);
    }
    __syncthreads();
    const int P = S.P;
    const int groups = 32 / P;
    const int grp = lane / P, k = lane - grp * P;
    for (int base = warp * groups; base < CW; base += nw * groups) {
        const int first = base + grp;
        line_solve<T, KP, 1>(buf + min(first, CW), pitch, 1, first < CW ? 1 : 0, st, P, bnd, k, nline);
    }
    __syncthreads();
    unsigned bad = 0;
    for (int i = warp * rpw + r0; i < nline; i += nw * rpw)
        if (c < nc && IGAPW_IDX("cols store", gbase + (long long)i * rs, s.ntot))
            store_out<T, OUT>(s, gbase + (long long)i * rs, buf[i * pitch + c], bad);
    if (bad && s.status) atomicOr(s.status, STATUS_NONFINITE);
}

static int smem_limit() {
    static int lim = -1;
    if (lim < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return lim;
}

template <typename T, int KP, int IN, int OUT>
static cudaError_t run_solve(const SolveArgs& s, const LineSys<T>& S, cudaStream_t st) {
    constexpr int NB = 1;
    const int groups = 32 / S.P;
    const int lines_per_warp = groups * NB;
    if (s.axis == 0) {
        const int nx = s.n[0];
        const long long nlines = (long long)s.n[1] * s.n[2];
        const size_t tb = table_elems<T, KP>(nx, S.P) * sizeof(T);
        int warps = 8;
        while (warps > 1 && tb + (size_t)warps * lines_per_warp * (nx | 1) * sizeof(T) > 100 * 1024) warps >>= 1;
        const int lpb = warps * lines_per_warp;
        const size_t sm = tb + (size_t)lpb * (nx | 1) * sizeof(T);
        if ((int)sm > smem_limit()) return cudaErrorInvalidValue;
        auto k = solve_x_kernel<T, KP, IN, OUT, NB>;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        const long long blocks = (nlines + lpb - 1) / lpb;
        k<<<(unsigned)blocks, warps * 32, sm, st>>>(s, S, lpb);
    } else {
        const int nx = s.n[0], ny = s.n[1], nz = s.n[2];
        const int nline = s.axis == 1 ? ny : nz;
        const long long os = s.axis == 1 ? (long long)ny * nx : (long long)nx;
        const long long rs = s.axis == 1 ? (long long)nx : (long long)nx * ny;
        const int outer = s.axis == 1 ? nz : ny;
        // NO outer indices x 32 columns per block; one warp per lines_per_warp lines
        int NO = 1;
        while (NO * 32 < 8 * lines_per_warp && NO < outer) NO *= 2;
        const size_t tb = table_elems<T, KP>(nline, S.P) * sizeof(T);
        while (NO > 1 && tb + (size_t)nline * (NO * 32 + 1) * sizeof(T) > 100 * 1024) NO >>= 1;
        const int warps = std::min(8, (NO * 32 + lines_per_warp - 1) / lines_per_warp);
        const size_t sm = tb + (size_t)nline * (NO * 32 + 1) * sizeof(T);
        if ((int)sm > smem_limit()) {
            // long lines: fewer columns per block, tables from global memory
            int CW = 32;
            while (CW > 1 && (size_t)nline * (CW + 1) * sizeof(T) > (size_t)smem_limit()) CW >>= 1;
            const size_t sc = (size_t)nline * (CW + 1) * sizeof(T);
            if (sc > (size_t)smem_limit()) return cudaErrorInvalidValue;
            int lg = 0;
            while ((1 << lg) < CW) ++lg;
            auto kc = solve_cols_kernel<T, KP, IN, OUT>;
            if (sc > 48 * 1024) cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
            dim3 grid((nx + CW - 1) / CW, outer);
            kc<<<grid, 256, sc, st>>>(s, S, nline, CW, lg, os, rs);
            return cudaGetLastError();
        }
        auto k = solve_strided_kernel<T, KP, IN, OUT, NB>;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid((nx + 31) / 32, (outer + NO - 1) / NO);
        int lg = 0;
        while ((1 << lg) < NO) ++lg;
        k<<<grid, warps * 32, sm, st>>>(s, S, nline, outer, NO, lg, os, rs);
    }
    return cudaGetLastError();
}

template <typename T, int KP>
static cudaError_t dispatch_fmt(const SolveArgs& s, const LineSys<T>& S, int in_fmt, int out_fmt,
                                cudaStream_t st) {
    if (in_fmt == FMT_F64 && out_fmt == FMT_F64) return run_solve<T, KP, FMT_F64, FMT_F64>(s, S, st);
    if (in_fmt == FMT_F32 && out_fmt == FMT_F32) return run_solve<T, KP, FMT_F32, FMT_F32>(s, S, st);
    if (in_fmt == FMT_PAIR && out_fmt == FMT_F32) return run_solve<T, KP, FMT_PAIR, FMT_F32>(s, S, st);
    if (in_fmt == FMT_F32 && out_fmt == FMT_PAIR) return run_solve<T, KP, FMT_F32, FMT_PAIR>(s, S, st);
    if (in_fmt == FMT_PAIR && out_fmt == FMT_PAIR) return run_solve<T, KP, FMT_PAIR, FMT_PAIR>(s, S, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_solve(const SolveArgs& s, const AxisDev& ax, int p, int in_fmt, int out_fmt,
                         bool fp64, cudaStream_t st) {
    if (fp64) {
        if (in_fmt != FMT_F64 || out_fmt != FMT_F64) return cudaErrorInvalidValue;
        switch (p) {
            case 2: return run_solve<double, 2, FMT_F64, FMT_F64>(s, ax.ls64, st);
            case 3: return run_solve<double, 3, FMT_F64, FMT_F64>(s, ax.ls64, st);
            case 4: return run_solve<double, 4, FMT_F64, FMT_F64>(s, ax.ls64, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (p) {
        case 2: return dispatch_fmt<float, 2>(s, ax.ls32, in_fmt, out_fmt, st);
        case 3: return dispatch_fmt<float, 3>(s, ax.ls32, in_fmt, out_fmt, st);
        case 4: return dispatch_fmt<float, 4>(s, ax.ls32, in_fmt, out_fmt, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace igapw
