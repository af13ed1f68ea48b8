// Kernel (c2): batched banded line solves along one axis of the coefficient
// tensor (one batch of 1D systems with many right-hand sides per axis, the
// alternating-directions solve of Sec. 4.1).
//
// Each warp solves one line.  The line is split into P <= 32 chunks, one per
// lane.  Forward substitution L y = r: every lane solves its chunk with the
// previous chunk's tail taken as zero, the true tails follow from a
// Hillis-Steele scan over the lanes (p x p operators precomputed per lane and
// level), and a rank-p spike correction finishes the chunk.  Backward
// substitution U x = y mirrors it with heads and a reverse scan.  Lines are
// staged in shared memory with coalesced loads: x-lines row by row, y- and
// z-lines as 32-wide column blocks.
#include "common.cuh"
#include "kernels.h"

namespace igapw {

template <typename T, int KP>
__device__ __forceinline__ void warp_solve(T* x, const int st, const LineSys<T>& S, const int lane) {
    const unsigned FULL = 0xffffffffu;
    const int P = S.P;
    const bool act = lane < P;
    const int lo = act ? S.b[lane] : 0;
    const int hi = act ? S.b[lane + 1] : 0;
    const T* __restrict__ L = S.L;
    const T* __restrict__ U = S.U;
    const T* __restrict__ G = S.G;
    const T* __restrict__ H = S.H;
    const T* __restrict__ dinv = S.dinv;

    // ---- forward: local chunk solve with a zero incoming tail ------------
    for (int i = lo; i < hi; ++i) {
        T acc = x[i * st];
#pragma unroll
        for (int m = 1; m <= KP; ++m)
            if (i - m >= lo) acc -= L[i * KP + m - 1] * x[(i - m) * st];
        x[i * st] = acc;
    }
    T a[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) a[c] = act ? x[(hi - KP + c) * st] : T(0);
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const int d = 1 << l;
        T ap[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) ap[c] = __shfl_up_sync(FULL, a[c], d);
        if (act && lane >= d) {
            const T* __restrict__ Ph = S.PhiF + (l * 32 + lane) * KP * KP;
            T na[KP];
#pragma unroll
            for (int r = 0; r < KP; ++r) {
                T s = a[r];
#pragma unroll
                for (int c = 0; c < KP; ++c) s += Ph[r * KP + c] * ap[c];
                na[r] = s;
            }
#pragma unroll
            for (int r = 0; r < KP; ++r) a[r] = na[r];
        }
    }
    T tp[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) {
        tp[c] = __shfl_up_sync(FULL, a[c], 1);
        if (lane == 0) tp[c] = T(0);
    }
    if (act && lane > 0) {
        for (int i = lo; i < hi; ++i) {
            T acc = x[i * st];
#pragma unroll
            for (int c = 0; c < KP; ++c) acc -= G[i * KP + c] * tp[c];
            x[i * st] = acc;
        }
    }
    // ---- backward: local chunk solve with a zero incoming head -----------
    for (int i = hi - 1; i >= lo; --i) {
        T acc = x[i * st];
#pragma unroll
        for (int m = 1; m <= KP; ++m)
            if (i + m < hi) acc -= U[i * KP + m - 1] * x[(i + m) * st];
        x[i * st] = acc * dinv[i];
    }
    T h[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) h[c] = act ? x[(lo + c) * st] : T(0);
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const int d = 1 << l;
        T hp[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) hp[c] = __shfl_down_sync(FULL, h[c], d);
        if (act && lane + d < P) {
            const T* __restrict__ Ph = S.PhiB + (l * 32 + lane) * KP * KP;
            T nh[KP];
#pragma unroll
            for (int r = 0; r < KP; ++r) {
                T s = h[r];
#pragma unroll
                for (int c = 0; c < KP; ++c) s += Ph[r * KP + c] * hp[c];
                nh[r] = s;
            }
#pragma unroll
            for (int r = 0; r < KP; ++r) h[r] = nh[r];
        }
    }
    T sn[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) {
        sn[c] = __shfl_down_sync(FULL, h[c], 1);
        if (lane + 1 >= P) sn[c] = T(0);
    }
    if (act && lane + 1 < P) {
        for (int i = lo; i < hi; ++i) {
            T acc = x[i * st];
#pragma unroll
            for (int c = 0; c < KP; ++c) acc -= H[i * KP + c] * sn[c];
            x[i * st] = acc;
        }
    }
}

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

template <typename T, int KP, int IN, int OUT>
__global__ void __launch_bounds__(256) solve_x_kernel(SolveArgs s, LineSys<T> S, int lpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);
    const int nx = s.n[0];
    const int pitch = nx + 1;
    const long long nlines = (long long)s.n[1] * s.n[2];
    const long long l0 = (long long)blockIdx.x * lpb;
    const int nl = (int)min((long long)lpb, nlines - l0);
    for (int e = threadIdx.x; e < nl * nx; e += blockDim.x) {
        const int l = e / nx, i = e - l * nx;
        buf[l * pitch + i] = load_in<T, IN>(s.in, (l0 + l) * nx + i);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = warp; l < nl; l += nw) warp_solve<T, KP>(buf + l * pitch, 1, S, lane);
    __syncthreads();
    unsigned bad = 0;
    for (int e = threadIdx.x; e < nl * nx; e += blockDim.x) {
        const int l = e / nx, i = e - l * nx;
        store_out<T, OUT>(s, (l0 + l) * nx + i, buf[l * pitch + i], bad);
    }
    if (bad && s.status) atomicOr(s.status, STATUS_NONFINITE);
}

// Lines along y (os = n_y n_x, rs = n_x, outer = z) or z (os = n_x,
// rs = n_x n_y, outer = y); element (outer o, row i, column x) at
// o*os + i*rs + x.  A block stages COLS consecutive x for all rows.
template <typename T, int KP, int IN, int OUT, int COLS>
__global__ void __launch_bounds__(256) solve_strided_kernel(SolveArgs s, LineSys<T> S, int nline,
                                                            long long os, long long rs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);
    const int nx = s.n[0];
    const int x0 = blockIdx.x * COLS;
    const int nc = min(COLS, nx - x0);
    const long long base = (long long)blockIdx.y * os + x0;
    constexpr int pitch = COLS + 1;
    for (int e = threadIdx.x; e < nline * COLS; e += blockDim.x) {
        const int i = e / COLS, c = e - i * COLS;
        if (c < nc) buf[i * pitch + c] = load_in<T, IN>(s.in, base + i * rs + c);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < nc; c += nw) warp_solve<T, KP>(buf + c, pitch, S, lane);
    __syncthreads();
    unsigned bad = 0;
    for (int e = threadIdx.x; e < nline * COLS; e += blockDim.x) {
        const int i = e / COLS, c = e - i * COLS;
        if (c < nc) store_out<T, OUT>(s, base + i * rs + c, buf[i * pitch + c], bad);
    }
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
    const int threads = 256;
    if (s.axis == 0) {
        const int nx = s.n[0];
        const long long nlines = (long long)s.n[1] * s.n[2];
        int lpb = 8;
        while (lpb > 1 && (size_t)lpb * (nx + 1) * sizeof(T) > 96 * 1024) lpb >>= 1;
        const size_t sm = (size_t)lpb * (nx + 1) * sizeof(T);
        if ((int)sm > smem_limit()) return cudaErrorInvalidValue;
        auto k = solve_x_kernel<T, KP, IN, OUT>;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        const long long blocks = (nlines + lpb - 1) / lpb;
        k<<<(unsigned)blocks, threads, sm, st>>>(s, S, lpb);
    } else {
        constexpr int COLS = sizeof(T) == 8 ? 16 : 32;
        const int nx = s.n[0], ny = s.n[1], nz = s.n[2];
        const int nline = s.axis == 1 ? ny : nz;
        const long long os = s.axis == 1 ? (long long)ny * nx : (long long)nx;
        const long long rs = s.axis == 1 ? (long long)nx : (long long)nx * ny;
        const int outer = s.axis == 1 ? nz : ny;
        const size_t sm = (size_t)nline * (COLS + 1) * sizeof(T);
        if ((int)sm > smem_limit()) return cudaErrorInvalidValue;
        auto k = solve_strided_kernel<T, KP, IN, OUT, COLS>;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid((nx + COLS - 1) / COLS, outer);
        k<<<grid, threads, sm, st>>>(s, S, nline, os, rs);
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
