// Shared device definitions: double-float (FP32 pair) arithmetic, per-axis
// device descriptors, and the status word.
#pragma once
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>
#include <stdint.h>

namespace igapw {

// ---------------------------------------------------------------------------
// Double-float arithmetic.  A value is hi + lo with |lo| <= ulp(hi)/2.
// Error-free transforms: the product of two floats is p + e exactly with
// p = a*b, e = fma(a, b, -p) (the FMA is exact up to its final rounding);
// the sum of two floats is s + e exactly with Knuth's branch-free two-sum.
// Built without fast-math, so these expressions are evaluated as written.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ DF df_make(float hi, float lo) {
    DF r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}

// Accumulator of a compensated dot product: running sum s with the exact
// rounding errors of every addition and product collected in c.
struct DFAcc {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
    // s + c += t * v with t, v double-float: the hi*hi product is split exactly,
    // the cross terms hi*lo + lo*hi enter c directly (lo*lo is below 2^-48).
    __device__ __forceinline__ void add_prod(DF t, DF v) {
        float p = t.hi * v.hi;
        float e = fmaf(t.hi, v.hi, -p);
        e = fmaf(t.hi, v.lo, e);
        e = fmaf(t.lo, v.hi, e);
        float s2, err;
        two_sum(s, p, s2, err);
        s = s2;
        c += err + e;
    }
    // s + c += t * v with v a plain float (its low part is zero)
    __device__ __forceinline__ void add_prod_f(DF t, float v) {
        float p = t.hi * v;
        float e = fmaf(t.hi, v, -p);
        e = fmaf(t.lo, v, e);
        float s2, err;
        two_sum(s, p, s2, err);
        s = s2;
        c += err + e;
    }
    // s + c += v
    __device__ __forceinline__ void add(DF v) {
        float s2, err;
        two_sum(s, v.hi, s2, err);
        s = s2;
        c += err + v.lo;
    }
    __device__ __forceinline__ DF result() const { return df_make(s, c); }
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return df_make(s, e);
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_make(p, e);
}

__host__ __device__ inline void split_double(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// ---------------------------------------------------------------------------
// Per-axis device tables.  Window format: row i couples to columns
// [fstart[i], fstart[i] + W) with W the padded kernel width of the context.
// ---------------------------------------------------------------------------
struct TableSet {
    const double* d;    // FP64 [n * W]
    const float2* df;   // double-float (hi, lo) interleaved [n * W]
};

// Precomputed data of the partitioned banded solve of one 1D system
// (banded LU without pivoting, KL = KU = p).  Rows are split into P <= 32
// chunks b[k] .. b[k+1]-1, one per lane of a warp.
template <typename T>
struct LineSys {
    int n, P;
    int b[33];
    const T* L;      // [n * p]   L[i*p + m-1] = l_{i, i-m}
    const T* U;      // [n * p]   U[i*p + m-1] = u_{i, i+m}
    const T* dinv;   // [n]       1 / u_{i,i}
    const T* G;      // [n * p]   forward spike: y_i -= sum_c G[i*p+c] * tail_{k-1}[c]
    const T* H;      // [n * p]   backward spike: x_i -= sum_c H[i*p+c] * head_{k+1}[c]
    const T* PhiF;   // [5 * 32 * p * p] forward scan operators per level and lane
    const T* PhiB;   // [5 * 32 * p * p] backward scan operators
};

// Packed FP32 tables of the chunked explicit step (chunkstep.cuh), built once
// per axis by launch_chunk_tables from the FP64 factors.  A line of n rows is
// padded to P * rows rows (decoupled identity rows) and cut into P chunks of
// `rows` rows; chunk k's
// partitioned solve takes the true tail of chunk k-1 as the local tail plus
// the composed spike operators of up to J-1 earlier chunks (J = P unless the
// operators decay below 1e-16 sooner).
struct ChunkDev {
    int rows;             // rows per chunk (the kernel's compile-time chunk length)
    int P;                // chunks per line
    const float4* cw;     // [np][nq4]: C window as (hi, lo) pairs, then fstart (int bits)
    const float4* aw;     // [np][nq4]: A window, same layout
    const float4* fl;     // [np]: l_{i,i-1} .. l_{i,i-p}
    const float4* fu;     // [np]: u_{i,i+1} .. u_{i,i+p} times 1/u_ii; 1/u_ii in .w when p <= 3
    const float* fd;      // [np]: 1 / u_{i,i}
    const float4* fg;     // [np]: forward spike of row i times 1/u_ii (columns: the previous chunk's last p rows)
    const float4* fh;     // [np]: backward spike (columns: the next chunk's first p rows)
    const float* psf;     // [P][P][p][p]: psf[k][d] = Phi_{k-1} ... Phi_{k-d} (forward tails)
    const float* psb;     // [P][P][p][p]: psb[k][d] = Theta_{k+1} ... Theta_{k+d} (backward heads)
    const int* J;         // chunks that enter a composed tail or head (device scalar)
};

struct AxisDev {
    int n;          // coefficients on this axis
    int nq;         // quadrature points on this axis
    int wq;         // point-window width (padded)
    const int* fstart;   // [n]
    const int* pstart;   // [n]
    const int* pcount;   // [n] points of each row's window actually carrying its test
    const int* is_free;  // [n]
    TableSet A;     // int T_i B_j        (Dirichlet rows: identity)
    TableSet C;     // int T_i B_j''      (Dirichlet rows: zero)
    TableSet S;     // system matrix factored for the solve
    TableSet TW;    // test weights over the point window [n * wq]
    LineSys<double> ls64;
    LineSys<float> ls32;
    ChunkDev ck;    // chunked-step tables (ck.P == 0: not built)
};

// Bounds-check record of one translation unit (debug builds).
struct BoundsReport {
    unsigned count;
    long long index, limit, line;
    const char* file;
};
using BoundsReader = BoundsReport (*)();
void register_bounds_reader(BoundsReader r);   // api.cu

// Status bits written by kernels (read back by igapw_sync_status).
enum : unsigned { STATUS_NONFINITE = 1u, STATUS_SINGULAR = 2u, STATUS_TC_TIMEOUT = 4u };

// Debug builds (-DIGAPW_BOUNDS_CHECK): index checks that skip an out-of-range
// access and record it in a per-translation-unit counter together with the
// first offender's index, limit and source line; igapw_sync_status reads the
// counters of every unit and fails with IGAPW_ERR_DEVICE_STATUS.  Release
// builds compile the checks away.
#ifdef IGAPW_BOUNDS_CHECK
static __device__ unsigned g_igapw_nbad;
static __device__ long long g_igapw_first[3];
__device__ __forceinline__ bool igapw_check_idx(int line, long long i, long long lim) {
    if (i >= 0 && i < lim) return true;
    if (atomicAdd(&g_igapw_nbad, 1u) == 0) {
        g_igapw_first[0] = i;
        g_igapw_first[1] = lim;
        g_igapw_first[2] = line;
    }
    return false;
}
#define IGAPW_IDX(site, i, lim) igapw_check_idx(__LINE__, (long long)(i), (long long)(lim))
#else
#define IGAPW_IDX(site, i, lim) true
#endif

}  // namespace igapw

namespace igapw {

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes per copy):
// many copies stay in flight without holding registers; cp_async_wait_all()
// followed by __syncthreads() makes them visible to the block.
// ---------------------------------------------------------------------------
#ifndef IGAPW_HOST_EMU
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// the dynamic shared memory of a kernel
#define IGAPW_DYNAMIC_SMEM(name) extern __shared__ __align__(16) unsigned char name[]
#else
// Host emulation of kernels (tests/c/cuda_emu.h): plain copies, and the
// block's shared memory from the emulator.
inline void cp_async4(void* smem, const void* gmem) { std::memcpy(smem, gmem, 4); }
inline void cp_async8(void* smem, const void* gmem) { std::memcpy(smem, gmem, 8); }
inline void cp_async_wait_all() {}
#define IGAPW_DYNAMIC_SMEM(name) unsigned char* name = igapw_emu_smem()
#endif

}  // namespace igapw

#if defined(IGAPW_BOUNDS_CHECK) && !defined(IGAPW_HOST_EMU)
namespace igapw {
// Reads and clears this translation unit's bounds-check record (host side).
static BoundsReport igapw_read_bounds_tu() {
    BoundsReport r{};
    r.file = __BASE_FILE__;
    long long f[3] = {0, 0, 0};
    if (cudaMemcpyFromSymbol(&r.count, g_igapw_nbad, sizeof(unsigned)) != cudaSuccess) return r;
    if (r.count) {
        cudaMemcpyFromSymbol(f, g_igapw_first, sizeof f);
        const unsigned zero = 0;
        cudaMemcpyToSymbol(g_igapw_nbad, &zero, sizeof zero);
    }
    r.index = f[0];
    r.limit = f[1];
    r.line = f[2];
    return r;
}
static const int igapw_bounds_registered = (register_bounds_reader(&igapw_read_bounds_tu), 0);
}  // namespace igapw
#endif
