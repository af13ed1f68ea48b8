// Device-side building blocks of the partitioned banded line solve, shared
// by the batched solve kernels (solve.cu) and the split explicit step (step.cu).
//
// A line is split into P contiguous chunks (P a power of two <= 32), one per
// lane of a lane group; a warp holds 32/P groups and every group solves NB
// lines at once.  Forward substitution L y = r: each lane solves its chunk
// with the previous chunk's tail taken as zero, the true tails follow from a
// Hillis-Steele scan over the group's lanes (p x p operators precomputed per
// lane and level), and a rank-p spike correction finishes the chunk (fused
// into the backward sweep).  Backward substitution U x = y mirrors it with
// heads and a reverse scan.
#pragma once
#include "common.cuh"

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
    int lanes;          // lane stride of the scan operators: 32 in global memory, P when staged
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

// Scan levels of a P-chunk partition (levels 0 .. log2(P) - 1 are used).
__host__ __device__ constexpr int scan_levels(int P) { return P <= 1 ? 0 : (P <= 2 ? 1 : (P <= 4 ? 2 : (P <= 8 ? 3 : (P <= 16 ? 4 : 5)))); }

// Shared-memory elements of one axis' staged tables: LU rows and spikes, and
// the scan operators of the P lanes and log2(P) levels actually used.
template <typename T, int KP>
__host__ __device__ constexpr size_t table_elems(int n, int P) {
    return (size_t)4 * n * KP + n + (size_t)2 * scan_levels(P) * P * KP * KP;
}

// Copies the LineSys tables into shared memory at `base` with asynchronous
// copies (the caller waits: cp_async_wait_all + __syncthreads); returns the views.
template <typename T, int KP>
__device__ SolveSmem<T> stage_tables(const LineSys<T>& S, T* base) {
    const int n = S.n, P = S.P;
    const int nlev = scan_levels(P);
    T* L = base;
    T* U = L + n * KP;
    T* G = U + n * KP;
    T* H = G + n * KP;
    T* dinv = H + n * KP;
    T* PhiF = dinv + n;
    T* PhiB = PhiF + nlev * P * KP * KP;
    const int nk = n * KP, pp = KP * KP, nphi = nlev * P * pp;
    auto cp = [](T* d, const T* s) {
        if constexpr (sizeof(T) == 8) cp_async8(d, s);
        else cp_async4(d, s);
    };
    for (int e = threadIdx.x; e < nk; e += blockDim.x) {
        cp(L + e, S.L + e);
        cp(U + e, S.U + e);
        cp(G + e, S.G + e);
        cp(H + e, S.H + e);
    }
    for (int e = threadIdx.x; e < n; e += blockDim.x) cp(dinv + e, S.dinv + e);
    // scan operators: entry (level lv, lane k) moves from lane stride 32 to P
    for (int e = threadIdx.x; e < nphi; e += blockDim.x) {
        const int blk = e / pp, r = e - blk * pp;
        const int lv = blk / P, k = blk - lv * P;
        cp(PhiF + e, S.PhiF + (lv * 32 + k) * pp + r);
        cp(PhiB + e, S.PhiB + (lv * 32 + k) * pp + r);
    }
    return SolveSmem<T>{L, U, dinv, G, H, PhiF, PhiB, P};
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
        const T* Ph = S.PhiF + (lv * S.lanes + k) * KP * KP;
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
        const T* Ph = S.PhiB + (lv * S.lanes + k) * KP * KP;
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
        const T* Ph = S.PhiF + (lv * S.lanes + k) * KP * KP;
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
        const T* Ph = S.PhiB + (lv * S.lanes + k) * KP * KP;
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

// Sequential solve of one whole line by one lane (P = 1), for short lines
// (at most 20 rows, or too few rows for two chunks of p).  Values stream through a register prefetch ring of D rows so no
// shared-memory load sits on the recurrence; the farthest band entries are
// applied first so each row waits on its predecessor for one FMA.
template <typename T, int KP, int D>
__device__ __forceinline__ void seq_solve(T* x, const int st, const int n, const SolveSmem<T>& S) {
    T w[KP];
#pragma unroll
    for (int m = 0; m < KP; ++m) w[m] = T(0);
    T pf[D];
#pragma unroll
    for (int k = 0; k < D; ++k) pf[k] = k < n ? x[k * st] : T(0);
    for (int i0 = 0; i0 < n; i0 += D) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int i = i0 + k;
            if (i < n) {
                const T xi = pf[k];
                pf[k] = (i + D < n) ? x[(i + D) * st] : T(0);
                T acc = xi;
#pragma unroll
                for (int m = KP - 1; m >= 0; --m) acc -= S.L[i * KP + m] * w[m];
                x[i * st] = acc;
#pragma unroll
                for (int m = KP - 1; m > 0; --m) w[m] = w[m - 1];
                w[0] = acc;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < KP; ++m) w[m] = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) pf[k] = (n - 1 - k >= 0) ? x[(n - 1 - k) * st] : T(0);
    for (int i0 = n - 1; i0 >= 0; i0 -= D) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int i = i0 - k;
            if (i >= 0) {
                const T xi = pf[k];
                pf[k] = (i - D >= 0) ? x[(i - D) * st] : T(0);
                T acc = xi;
#pragma unroll
                for (int m = KP - 1; m >= 0; --m) acc -= S.U[i * KP + m] * w[m];
                acc *= S.dinv[i];
                x[i * st] = acc;
#pragma unroll
                for (int m = KP - 1; m > 0; --m) w[m] = w[m - 1];
                w[0] = acc;
            }
        }
    }
}

// Dispatch: sequential (P = 1), register-resident chunks, or shared-memory chunks.
template <typename T, int KP, int NB>
__device__ __forceinline__ void line_solve(T* x, const int st, const int lst, const int nb,
                                           const SolveSmem<T>& S, const int P, const int* bnd,
                                           const int k, const int n) {
#ifdef IGAPW_BOUNDS_CHECK
    // report only: skipping one lane would desynchronise the group's shuffles
    (void)IGAPW_IDX("solve bnd hi", bnd[P], n + 1);
    (void)IGAPW_IDX("solve bnd lo", bnd[k], bnd[k + 1] + 1);
#endif
    if (P == 1) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < nb) seq_solve<T, KP, 4>(x + b * lst, st, n, S);
    } else if ((n + P - 1) / P <= 20) {
        group_solve_reg<T, KP, NB, 20>(x, st, lst, nb, S, P, bnd, k);
    } else {
        group_solve<T, KP, NB>(x, st, lst, nb, S, P, bnd, k);
    }
}

}  // namespace igapw
