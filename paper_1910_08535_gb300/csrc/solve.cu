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

namespace igapw {

// Solve tables of one axis staged in shared memory (read in the recurrences).
template <typename T>
struct SolveSmem {
    const T* L;
    const T* U;
    const T* dinv;
    const T* G;
    const T* H;
    const T* PhiF;
    const T* PhiB;
};

// Copies count elements with UNR independent loads in flight per thread
// (a plain strided loop would wait one memory latency per iteration).
template <int UNR, typename Ld, typename St>
__device__ __forceinline__ void batched_copy(int count, Ld&& ld, St&& st) {
    const int step = blockDim.x * UNR;
    for (int base = threadIdx.x; base < count; base += step) {
        decltype(ld(0)) v[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int e = base + k * blockDim.x;
            if (e < count) v[k] = ld(e);
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int e = base + k * blockDim.x;
            if (e < count) st(e, v[k]);
        }
    }
}

template <typename T, int KP>
__host__ __device__ constexpr size_t table_elems(int n) {
    return (size_t)4 * n * KP + n + 2 * 5 * 32 * KP * KP;
}

// Copies the LineSys tables into shared memory at `base`; returns the views.
template <typename T, int KP>
__device__ SolveSmem<T> stage_tables(const LineSys<T>& S, T* base) {
    const int n = S.n;
    T* L = base;
    T* U = L + n * KP;
    T* G = U + n * KP;
    T* H = G + n * KP;
    T* dinv = H + n * KP;
    T* PhiF = dinv + n;
    T* PhiB = PhiF + 5 * 32 * KP * KP;
    const int nk = n * KP, nphi = 5 * 32 * KP * KP;
    batched_copy<4>(nk, [&](int e) { return S.L[e]; }, [&](int e, T v) { L[e] = v; });
    batched_copy<4>(nk, [&](int e) { return S.U[e]; }, [&](int e, T v) { U[e] = v; });
    batched_copy<4>(nk, [&](int e) { return S.G[e]; }, [&](int e, T v) { G[e] = v; });
    batched_copy<4>(nk, [&](int e) { return S.H[e]; }, [&](int e, T v) { H[e] = v; });
    batched_copy<4>(n, [&](int e) { return S.dinv[e]; }, [&](int e, T v) { dinv[e] = v; });
    batched_copy<8>(nphi, [&](int e) { return S.PhiF[e]; }, [&](int e, T v) { PhiF[e] = v; });
    batched_copy<8>(nphi, [&](int e) { return S.PhiB[e]; }, [&](int e, T v) { PhiB[e] = v; });
    return SolveSmem<T>{L, U, dinv, G, H, PhiF, PhiB};
}

// One lane group (P lanes, chunk k = lane index in the group) solves nb <= NB
// lines: line b, row i at x[i*st + b*lst].
template <typename T, int KP, int NB>
__device__ __forceinline__ void group_solve(T* x, const int st, const int lst, const int nb,
                                            const SolveSmem<T>& S, const int P, const int* bnd,
                                            const int k) {
    const unsigned FULL = 0xffffffffu;
    const int lo = bnd[k];
    const int hi = bnd[k + 1];

    // ---- forward local solve (zero incoming tail), sliding window --------
    T win[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int m = 0; m < KP; ++m) win[b][m] = T(0);
    for (int i = lo; i < hi; ++i) {
        T l[KP];
#pragma unroll
        for (int m = 0; m < KP; ++m) l[m] = S.L[i * KP + m];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T acc = (b < nb) ? x[i * st + b * lst] : T(0);
#pragma unroll
            for (int m = 0; m < KP; ++m) acc -= l[m] * win[b][m];
            if (b < nb) x[i * st + b * lst] = acc;
#pragma unroll
            for (int m = KP - 1; m > 0; --m) win[b][m] = win[b][m - 1];
            win[b][0] = acc;
        }
    }
    // tails a[c] = y_{hi-KP+c} = win[KP-1-c]
    T a[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) a[b][c] = win[b][KP - 1 - c];
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int d = 1 << lv;
        if (d >= P) break;   // uniform over the warp
        const bool upd = k >= d;
        const T* Ph = S.PhiF + (lv * 32 + k) * KP * KP;
        T ph[KP * KP];
#pragma unroll
        for (int e = 0; e < KP * KP; ++e) ph[e] = upd ? Ph[e] : T(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T ap[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) ap[c] = __shfl_up_sync(FULL, a[b][c], d, P);
            T na[KP];
#pragma unroll
            for (int r = 0; r < KP; ++r) {
                T s = a[b][r];
#pragma unroll
                for (int c = 0; c < KP; ++c) s += ph[r * KP + c] * ap[c];
                na[r] = s;
            }
#pragma unroll
            for (int r = 0; r < KP; ++r) a[b][r] = na[r];
        }
    }
    T tp[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            tp[b][c] = __shfl_up_sync(FULL, a[b][c], 1, P);
            if (k == 0) tp[b][c] = T(0);
        }

    // ---- backward local solve with the forward spike correction fused -----
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int m = 0; m < KP; ++m) win[b][m] = T(0);
    for (int i = hi - 1; i >= lo; --i) {
        T u[KP], g[KP];
#pragma unroll
        for (int m = 0; m < KP; ++m) { u[m] = S.U[i * KP + m]; g[m] = S.G[i * KP + m]; }
        const T di = S.dinv[i];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T acc = (b < nb) ? x[i * st + b * lst] : T(0);
#pragma unroll
            for (int c = 0; c < KP; ++c) acc -= g[c] * tp[b][c];
#pragma unroll
            for (int m = 0; m < KP; ++m) acc -= u[m] * win[b][m];
            acc *= di;
            if (b < nb) x[i * st + b * lst] = acc;
#pragma unroll
            for (int m = KP - 1; m > 0; --m) win[b][m] = win[b][m - 1];
            win[b][0] = acc;
        }
    }
    // heads h[c] = x_{lo+c} = win[c]
    T h[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) h[b][c] = win[b][c];
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int d = 1 << lv;
        if (d >= P) break;
        const bool upd = k + d < P;
        const T* Ph = S.PhiB + (lv * 32 + k) * KP * KP;
        T ph[KP * KP];
#pragma unroll
        for (int e = 0; e < KP * KP; ++e) ph[e] = upd ? Ph[e] : T(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T hp[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) hp[c] = __shfl_down_sync(FULL, h[b][c], d, P);
            T nh[KP];
#pragma unroll
            for (int r = 0; r < KP; ++r) {
                T s = h[b][r];
#pragma unroll
                for (int c = 0; c < KP; ++c) s += ph[r * KP + c] * hp[c];
                nh[r] = s;
            }
#pragma unroll
            for (int r = 0; r < KP; ++r) h[b][r] = nh[r];
        }
    }
    T sn[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            sn[b][c] = __shfl_down_sync(FULL, h[b][c], 1, P);
            if (k + 1 >= P) sn[b][c] = T(0);
        }
    if (k + 1 < P) {
        for (int i = lo; i < hi; ++i) {
            T hh[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) hh[c] = S.H[i * KP + c];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (b < nb) {
                    T acc = x[i * st + b * lst];
#pragma unroll
                    for (int c = 0; c < KP; ++c) acc -= hh[c] * sn[b][c];
                    x[i * st + b * lst] = acc;
                }
            }
        }
    }
}

// Register-resident variant: the lane's chunk (at most CH rows) is copied
// from shared memory into registers, solved there (all loops unrolled over
// CH with the runtime length as a predicate, so no load sits on the
// recurrence), and written back.  The farthest band entries are applied
// first so each row waits on its predecessor for a single FMA.
template <typename T, int KP, int NB, int CH>
__device__ __forceinline__ void group_solve_reg(T* x, const int st, const int lst, const int nb,
                                                const SolveSmem<T>& S, const int P, const int* bnd,
                                                const int k) {
    const unsigned FULL = 0xffffffffu;
    const int lo = bnd[k];
    const int len = bnd[k + 1] - lo;
    T v[NB][CH];
#pragma unroll
    for (int t = 0; t < CH; ++t)
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b][t] = (t < len && b < nb) ? x[(lo + t) * st + b * lst] : T(0);

    // ---- forward local solve (zero incoming tail) -------------------------
    T a[NB][KP];   // tail: a[c] = y_{hi-KP+c}
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) a[b][c] = T(0);
#pragma unroll
    for (int t = 0; t < CH; ++t) {
        if (t < len) {
            const T* Lr = S.L + (lo + t) * KP;
            T l[KP];
#pragma unroll
            for (int m = 0; m < KP; ++m) l[m] = Lr[m];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                T acc = v[b][t];
#pragma unroll
                for (int m = KP; m >= 1; --m)
                    if (t - m >= 0) acc -= l[m - 1] * v[b][t - m];
                v[b][t] = acc;
#pragma unroll
                for (int c = 0; c < KP - 1; ++c) a[b][c] = a[b][c + 1];
                a[b][KP - 1] = acc;
            }
        }
    }
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int d = 1 << lv;
        if (d >= P) break;
        const bool upd = k >= d;
        const T* Ph = S.PhiF + (lv * 32 + k) * KP * KP;
        T ph[KP * KP];
#pragma unroll
        for (int e = 0; e < KP * KP; ++e) ph[e] = upd ? Ph[e] : T(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T ap[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) ap[c] = __shfl_up_sync(FULL, a[b][c], d, P);
            T na[KP];
#pragma unroll
            for (int r = 0; r < KP; ++r) {
                T s = a[b][r];
#pragma unroll
                for (int c = 0; c < KP; ++c) s += ph[r * KP + c] * ap[c];
                na[r] = s;
            }
#pragma unroll
            for (int r = 0; r < KP; ++r) a[b][r] = na[r];
        }
    }
    T tp[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            tp[b][c] = __shfl_up_sync(FULL, a[b][c], 1, P);
            if (k == 0) tp[b][c] = T(0);
        }

    // ---- backward local solve, forward spike correction fused -------------
#pragma unroll
    for (int t = CH - 1; t >= 0; --t) {
        if (t < len) {
            const int i = lo + t;
            T u[KP], g[KP];
#pragma unroll
            for (int m = 0; m < KP; ++m) { u[m] = S.U[i * KP + m]; g[m] = S.G[i * KP + m]; }
            const T di = S.dinv[i];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                T acc = v[b][t];
#pragma unroll
                for (int c = 0; c < KP; ++c) acc -= g[c] * tp[b][c];
#pragma unroll
                for (int m = KP; m >= 1; --m)
                    if (t + m < CH && t + m < len) acc -= u[m - 1] * v[b][(t + m < CH) ? t + m : 0];
                v[b][t] = acc * di;
            }
        }
    }
    T h[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) h[b][c] = v[b][c];
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int d = 1 << lv;
        if (d >= P) break;
        const bool upd = k + d < P;
        const T* Ph = S.PhiB + (lv * 32 + k) * KP * KP;
        T ph[KP * KP];
#pragma unroll
        for (int e = 0; e < KP * KP; ++e) ph[e] = upd ? Ph[e] : T(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T hp[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) hp[c] = __shfl_down_sync(FULL, h[b][c], d, P);
            T nh[KP];
#pragma unroll
            for (int r = 0; r < KP; ++r) {
                T s = h[b][r];
#pragma unroll
                for (int c = 0; c < KP; ++c) s += ph[r * KP + c] * hp[c];
                nh[r] = s;
            }
#pragma unroll
            for (int r = 0; r < KP; ++r) h[b][r] = nh[r];
        }
    }
    T sn[NB][KP];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            sn[b][c] = __shfl_down_sync(FULL, h[b][c], 1, P);
            if (k + 1 >= P) sn[b][c] = T(0);
        }
#pragma unroll
    for (int t = 0; t < CH; ++t) {
        if (t < len) {
            T hh[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) hh[c] = S.H[(lo + t) * KP + c];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                T acc = v[b][t];
#pragma unroll
                for (int c = 0; c < KP; ++c) acc -= hh[c] * sn[b][c];
                if (b < nb) x[(lo + t) * st + b * lst] = acc;
            }
        }
    }
}

// Dispatch between the register-resident and the shared-memory solve.
template <typename T, int KP, int NB>
__device__ __forceinline__ void line_solve(T* x, const int st, const int lst, const int nb,
                                           const SolveSmem<T>& S, const int P, const int* bnd,
                                           const int k, const int n) {
    if ((n + P - 1) / P <= 20) group_solve_reg<T, KP, NB, 20>(x, st, lst, nb, S, P, bnd, k);
    else group_solve<T, KP, NB>(x, st, lst, nb, S, P, bnd, k);
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

// x-lines (contiguous): a block stages lpb consecutive lines, odd pitch.
template <typename T, int KP, int IN, int OUT, int NB>
__global__ void __launch_bounds__(256) solve_x_kernel(SolveArgs s, LineSys<T> S, int lpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tabs = reinterpret_cast<T*>(smem_raw);
    const int nx = s.n[0];
    T* buf = tabs + table_elems<T, KP>(nx);
    __shared__ int bnd[33];
    const int pitch = nx | 1;   // odd pitch: lanes on different lines hit different banks
    const long long nlines = (long long)s.n[1] * s.n[2];
    const long long l0 = (long long)blockIdx.x * lpb;
    const int nl = (int)min((long long)lpb, nlines - l0);
    const SolveSmem<T> st = stage_tables<T, KP>(S, tabs);
    if (threadIdx.x < 33) bnd[threadIdx.x] = S.b[threadIdx.x];
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
    T* buf = tabs + table_elems<T, KP>(nline);
    __shared__ int bnd[33];
    const int nx = s.n[0];
    const int x0 = blockIdx.x * 32;
    const int nc = min(32, nx - x0);
    const int o0 = blockIdx.y * NO;
    const int no = min(NO, outer - o0);
    const int pitch = NO * 32 + 1;
    const SolveSmem<T> st = stage_tables<T, KP>(S, tabs);
    if (threadIdx.x < 33) bnd[threadIdx.x] = S.b[threadIdx.x];
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
        const size_t tb = table_elems<T, KP>(nx) * sizeof(T);
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
        const size_t tb = table_elems<T, KP>(nline) * sizeof(T);
        while (NO > 1 && tb + (size_t)nline * (NO * 32 + 1) * sizeof(T) > 100 * 1024) NO >>= 1;
        const int warps = std::min(8, (NO * 32 + lines_per_warp - 1) / lines_per_warp);
        const size_t sm = tb + (size_t)nline * (NO * 32 + 1) * sizeof(T);
        if ((int)sm > smem_limit()) return cudaErrorInvalidValue;
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
