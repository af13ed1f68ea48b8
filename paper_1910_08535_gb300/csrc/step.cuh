#pragma once
// The explicit heat step in split form (one kernel launch per axis): kernel
// template and launch helpers, instantiated per value type and degree by
// step_f64_p*.cu / step_df_p*.cu.
//
// Each step of Sec. 4.2, Eq. (6) solves (Mz (x) My (x) Mx) u' = T(u + dt Lap u)
// with M = T B the tested mass and the tested Laplacian
//   T Lap u = (C_x (x) A_y (x) A_z + A_x (x) C_y (x) A_z + A_x (x) A_y (x) C_z) u,
// A = int T_i B_j, C = int T_i B_j'' per axis (PW cells or B-spline tests).
// Because the mass is the Kronecker product of the per-axis A, the factors of
// the other axes cancel against their inverses:
//   u' = u + dt * sum_a (A_a^{-1} C_a applied along axis a) u.
// So one step is, for every axis a and every line along a:
//   g = C_a u (tested Laplacian along the line), w = A_a^{-1} g (banded solve),
//   accumulated as u' = u + dt (w_x + w_y + w_z).
// This is the same discrete scheme as RHS-then-solve (the same M and T); only
// the rounding order differs.  The line never leaves the block: contraction,
// solve, residual and correction run on a shared-memory copy of the line.
//
// FP32-pair mode: g in double-float; w0 = A^{-1} g_hi in FP32; residual
// rho = g - A w0 in double-float; delta = A^{-1} rho in FP32; w = w0 + delta.
// FP64 mode: g and the solve in FP64.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "linesolve.cuh"

namespace igapw {

namespace {

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename VT>
struct StepTypes;
template <>
struct StepTypes<double> {
    using S = double;   // solve type
};
template <>
struct StepTypes<DF> {
    using S = float;
};

__device__ __forceinline__ DF ld_tab(const TableSet& t, int idx, DF) {
    const float2 v = t.df[idx];
    return DF{v.x, v.y};
}
__device__ __forceinline__ double ld_tab(const TableSet& t, int idx, double) { return t.d[idx]; }

// Global value of the state / accumulator tensor.
__device__ __forceinline__ DF ld_state(const void* p, long long g, long long ntot, DF) {
    const float* f = (const float*)p;
    return DF{f[g], f[g + ntot]};
}
__device__ __forceinline__ double ld_state(const void* p, long long g, long long, double) {
    return ((const double*)p)[g];
}
__device__ __forceinline__ void st_state(void* p, long long g, long long ntot, DF v) {
    ((float*)p)[g] = v.hi;
    ((float*)p)[g + ntot] = v.lo;
}
__device__ __forceinline__ void st_state(void* p, long long g, long long, double v) { ((double*)p)[g] = v; }

}  // namespace

// MODE: 0 FIRST (acc = u + dt w), 1 MID (acc += dt w), 2 LAST (u = acc + dt w),
// 3 ONLY (u = u + dt w).  XL: lines along x (contiguous) or along y/z.
// CFG: 0 = tables staged, 32 columns per y/z block (or x-lines); 1 = tables
// read from global memory (long lines), runtime lines/columns; 2 = tables
// staged, 16 columns per y/z block (less shared memory per block: more
// resident blocks per SM).
template <typename VT, int KP, int W, int MODE, bool XL, int CFG>
__global__ void __launch_bounds__(256) axis_step_kernel(const AxisStepArgs a) {
    constexpr bool TG = (CFG == 1);
    using TS = typename StepTypes<VT>::S;
    constexpr bool DFM = std::is_same<VT, DF>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int bnd[33];
    const AxisDev& AX = a.ax;
    const LineSys<TS>& LS = *(DFM ? (const LineSys<TS>*)&AX.ls32 : (const LineSys<TS>*)&AX.ls64);
    const int n = AX.n;
    const int nx = a.n[0], ny = a.n[1];
    const int NL = a.lines_per_block;   // XL: lines; else columns, a power of two <= 32

    // ---- shared memory carve-up ------------------------------------------
    // every segment starts on a 16-byte boundary (8-byte cp.async targets).
    // TG (long lines): the tables are read from global memory (every lane of
    // a warp reads the same row: one broadcast L1 access) to leave room for
    // lines.  A compile-time switch, so that staged tables keep shared-memory
    // loads.
    unsigned char* p = smem_raw;
    SolveSmem<TS> S;
    const VT* Ct;
    const VT* At;
    const int* fs;
    if constexpr (TG) {
        S = SolveSmem<TS>{LS.L, LS.U, LS.dinv, LS.G, LS.H, LS.PhiF, LS.PhiB, 32};
        if constexpr (DFM) {
            Ct = reinterpret_cast<const VT*>(AX.C.df);
            At = reinterpret_cast<const VT*>(AX.A.df);
        } else {
            Ct = reinterpret_cast<const VT*>(AX.C.d);
            At = reinterpret_cast<const VT*>(AX.A.d);
        }
        fs = AX.fstart;
    } else {
        TS* tabs = reinterpret_cast<TS*>(p);
        p += align16(table_elems<TS, KP>(n, LS.P) * sizeof(TS));
        VT* ct = reinterpret_cast<VT*>(p);
        VT* at = ct + n * W;
        p += align16((size_t)2 * n * W * sizeof(VT));
        int* f = reinterpret_cast<int*>(p);
        p += align16((size_t)n * sizeof(int));
        S = stage_tables<TS, KP>(LS, tabs);
        for (int e = threadIdx.x; e < n * W; e += blockDim.x) {
            if constexpr (DFM) {
                cp_async8(ct + e, AX.C.df + e);
                cp_async8(at + e, AX.A.df + e);
            } else {
                cp_async8(ct + e, AX.C.d + e);
                cp_async8(at + e, AX.A.d + e);
            }
        }
        for (int e = threadIdx.x; e < n; e += blockDim.x) cp_async4(f + e, AX.fstart + e);
        Ct = ct;
        At = at;
        fs = f;
    }
    // lines carry W zero rows past n, so the contraction windows need no guards
    const int nr = n + W;
    // staged y/z blocks always hold 32 columns: a compile-time pitch of 33 turns
    // the row offsets of the banded windows into immediate offsets; a single
    // column (lines too long for more) needs no padding against bank conflicts
    const int pitch = XL ? (nr | 1) : (TG ? (NL == 1 ? 1 : NL + 1) : (CFG == 2 ? 17 : 33));
    const int st = XL ? 1 : pitch;      // row stride within a line
    const int lst = XL ? pitch : 1;     // line stride
    const int cap = XL ? NL * pitch : nr * pitch;
    VT* G = reinterpret_cast<VT*>(p);               // g (and, FP64, the solve buffer)
    VT* Ub = G + cap;                               // u during the contraction
    TS* X = reinterpret_cast<TS*>(Ub);              // FP32 pair mode: w0 ...
    TS* R = X + cap;                                //  ... and the residual / correction
    for (int e = threadIdx.x; e < 33; e += blockDim.x) bnd[e] = LS.b[e];

    // ---- which lines: global index of (line l, row i) ---------------------
    // launched with 256 threads (8 warps) always
    constexpr int nw = 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // y/z-lines: lane -> column cl of the block's NL columns, row offset ro of
    // the RPW rows a warp covers per pass
    // (staged tables come with 32 or 16 columns, fixed at compile time)
    const int lgNL = (XL || CFG == 0) ? 0 : (CFG == 2 ? 4 : __ffs(NL) - 1);
    const int cl = XL ? 0 : (CFG == 0 ? lane : (lane & ((1 << lgNL) - 1)));
    const int ro = (XL || CFG == 0) ? 0 : (lane >> lgNL);
    const int RPW = (XL || CFG == 0) ? 1 : (32 >> lgNL);
    long long l0 = 0, os = 0, rs = 0;
    int nl, x0 = 0;
    if (XL) {
        const long long nlines = (long long)a.n[1] * a.n[2];
        l0 = (long long)blockIdx.x * NL;
        nl = (int)min((long long)NL, nlines - l0);
    } else {
        x0 = blockIdx.x * NL;
        nl = min(NL, nx - x0);
        if (a.axis == 1) { os = (long long)ny * nx; rs = nx; }
        else { os = nx; rs = (long long)nx * ny; }
    }
    auto gidx = [&](int l, int i) -> long long {
        if (XL) return (l0 + l) * n + i;
        return (long long)blockIdx.y * os + (long long)i * rs + x0 + l;
    };

    // asynchronous copy of a state / accumulator tensor's lines into buf
    auto stage = [&](VT* buf, const void* src) {
        if (XL) {
            for (int l = warp; l < nl; l += nw)
                for (int i = lane; i < n; i += 32) {
                    const long long g = gidx(l, i);
                    VT* d = buf + l * pitch + i;
                    if (!IGAPW_IDX("step stage x smem", l * pitch + i, cap) || !IGAPW_IDX("step stage x g", g, a.ntot))
                        continue;
                    if constexpr (DFM) {
                        cp_async4(&d->hi, (const float*)src + g);
                        cp_async4(&d->lo, (const float*)src + g + a.ntot);
                    } else {
                        cp_async8(d, (const double*)src + g);
                    }
                }
        } else {
            for (int i = warp * RPW + ro; i < n; i += nw * RPW) {
                VT* d = buf + i * pitch + cl;
                if (!IGAPW_IDX("step stage c smem", i * pitch + cl, cap)) continue;
                if (cl < nl) {
                    const long long g = gidx(cl, i);
                    if (!IGAPW_IDX("step stage c g", g, a.ntot)) continue;
                    if constexpr (DFM) {
                        cp_async4(&d->hi, (const float*)src + g);
                        cp_async4(&d->lo, (const float*)src + g + a.ntot);
                    } else {
                        cp_async8(d, (const double*)src + g);
                    }
                } else {
                    *d = VT{};
                }
            }
        }
    };

    // visits every staged (line, row) of the block, rows [r0, r1), without divisions
    auto for_each = [&](int r0, int r1, auto&& f) {
        if (XL) {
            for (int l = warp; l < nl; l += nw)
                for (int i = r0 + lane; i < r1; i += 32) f(l, i);
        } else {
            for (int i = r0 + warp * RPW + ro; i < r1; i += nw * RPW) f(cl, i);
        }
    };

    // ---- P0: stage u ---------------------------------------------------------
    stage(Ub, a.u);
    for_each(n, nr, [&](int l, int i) {
        if (IGAPW_IDX("step pad", i * st + l * lst, cap)) Ub[i * st + l * lst] = VT{};
    });
    cp_async_wait_all();
    __syncthreads();

    // ---- P1: g = C u along the line (compensated in pair mode) --------------
    for_each(0, n, [&](int l, int i) {
        if (!IGAPW_IDX("step P1 ub", fs[i] * st + l * lst + (W - 1) * st, cap) || !IGAPW_IDX("step P1 g", i * st + l * lst, cap))
            return;
        const VT* ub = Ub + fs[i] * st + l * lst;
        const VT* ct = Ct + i * W;
        if constexpr (DFM) {
            DFAcc acc;
            acc.init();
#pragma unroll
            for (int w = 0; w < W; ++w) acc.add_prod(ct[w], ub[w * st]);
            G[i * st + l * lst] = acc.result();
        } else {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) s = fma(ct[w], ub[w * st], s);
            G[i * st + l * lst] = s;
        }
    });
    __syncthreads();

    const int P = LS.P;
    const int groups = 32 / P;
    const int grp = lane / P, k = lane - grp * P;
    const int nlines_b = XL ? nl : NL;   // lines per group set: groups = 32 / P
    if constexpr (DFM) {
        // ---- P2: w0 = A^{-1} g_hi (FP32) ------------------------------------
        for_each(0, nr, [&](int l, int i) { X[i * st + l * lst] = i < n ? G[i * st + l * lst].hi : 0.f; });
        __syncthreads();
        for (int base = warp * groups; base < nlines_b; base += nw * groups) {
            const int first = base + grp;
            line_solve<TS, KP, 1>(X + min(first, nlines_b) * lst, st, lst, first < nlines_b ? 1 : 0, S, P, bnd,
                                  k, n);
        }
        __syncthreads();
        // ---- P3: rho = g - A w0 (double-float) ------------------------------
        for_each(0, n, [&](int l, int i) {
            const TS* xw = X + fs[i] * st + l * lst;
            const VT* at = At + i * W;
            DFAcc acc;
            const DF g = G[i * st + l * lst];
            acc.s = g.hi;
            acc.c = g.lo;
#pragma unroll
            for (int w = 0; w < W; ++w) acc.add_prod_f(DF{-at[w].hi, -at[w].lo}, xw[w * st]);
            R[i * st + l * lst] = acc.result().hi;
        });
        __syncthreads();
        // g is dead: prefetch the tensor the update adds to into G meanwhile
        stage(G, (MODE == 0 || MODE == 3) ? a.u : a.acc);
        // ---- P4: delta = A^{-1} rho (FP32) ----------------------------------
        for (int base = warp * groups; base < nlines_b; base += nw * groups) {
            const int first = base + grp;
            line_solve<TS, KP, 1>(R + min(first, nlines_b) * lst, st, lst, first < nlines_b ? 1 : 0, S, P, bnd,
                                  k, n);
        }
        cp_async_wait_all();
        __syncthreads();
    } else {
        // u is dead: prefetch the tensor the update adds to into Ub meanwhile
        stage(Ub, (MODE == 0 || MODE == 3) ? a.u : a.acc);
        for (int base = warp * groups; base < nlines_b; base += nw * groups) {
            const int first = base + grp;
            if (first < nlines_b && !IGAPW_IDX("step solve extent", first * lst + (n - 1) * st, cap)) continue;
            line_solve<TS, KP, 1>(reinterpret_cast<TS*>(G) + min(first, nlines_b) * lst, st, lst,
                                  first < nlines_b ? 1 : 0, S, P, bnd, k, n);
        }
        cp_async_wait_all();
        __syncthreads();
    }

    // ---- P5: accumulate dt * w ---------------------------------------------
    const VT dtv = [&] {
        if constexpr (DFM) {
            DF d;
            split_double(a.dt, d.hi, d.lo);
            return d;
        } else {
            return a.dt;
        }
    }();
    unsigned bad = 0;
    auto finish = [&](int l, int i) {
        const long long g = gidx(l, i);
        if (!IGAPW_IDX("step finish smem", i * st + l * lst, cap) || !IGAPW_IDX("step finish g", g, a.ntot)) return;
        VT w;
        if constexpr (DFM) {
            float hi, lo;
            two_sum(X[i * st + l * lst], R[i * st + l * lst], hi, lo);
            w = DF{hi, lo};
        } else {
            w = G[i * st + l * lst];
        }
        const VT base = DFM ? G[i * st + l * lst] : Ub[i * st + l * lst];
        VT r;
        if constexpr (DFM) {
            DFAcc acc;
            acc.s = base.hi;
            acc.c = base.lo;
            acc.add_prod(dtv, w);
            r = acc.result();
            if (!isfinite(r.hi)) bad = 1;
        } else {
            r = fma(dtv, w, base);
            if (!isfinite(r)) bad = 1;
        }
        if (MODE == 0 || MODE == 1) st_state(a.acc, g, a.ntot, r);
        else st_state(a.u_out, g, a.ntot, r);
    };
    if (XL) {
        for (int l = warp; l < nl; l += nw)
            for (int i = lane; i < n; i += 32) finish(l, i);
    } else {
        for (int i = warp * RPW + ro; i < n; i += nw * RPW)
            if (cl < nl) finish(cl, i);
    }
    if (bad && a.status) atomicOr(a.status, STATUS_NONFINITE);
}

template <typename VT, int KP, int W, int MODE>
static cudaError_t run_axis_step(const AxisStepArgs& a0, cudaStream_t st) {
    using TS = typename StepTypes<VT>::S;
    AxisStepArgs a = a0;
    const int n = a.ax.n;
    const bool xl = a.axis == 0;
    const long long nlines = (long long)a.n[1] * a.n[2];
    int lim = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // bytes of shared memory for nl lines (XL) or nl columns, with or without
    // the tables staged
    auto smem_for = [&](int nl, bool tg) {
        const size_t cap = xl ? (size_t)nl * ((n + W) | 1) : (size_t)(n + W) * (tg && nl == 1 ? 1 : nl + 1);
        size_t b = (size_t)2 * cap * sizeof(VT);
        if (!tg)
            b += align16(table_elems<TS, KP>(n, a.ax.ls64.P) * sizeof(TS)) + align16((size_t)2 * n * W * sizeof(VT)) +
                 align16((size_t)n * sizeof(int));
        return b;
    };
    // Staged tables while enough lines share them (>= 8 x-lines, or all 32
    // columns); long lines read them from global memory instead, with as many
    // lines (a power of two for columns) as fit.
    const int nl_max = xl ? (int)std::min<long long>(32, nlines) : 32;
    int NL = nl_max;
    int cfg = 0;
    while (xl && NL > 8 && smem_for(NL, false) > (size_t)lim) NL = (NL + 1) / 2;
    if (smem_for(NL, false) > (size_t)lim) {
        cfg = 1;
        NL = nl_max;
        while (NL > 1 && smem_for(NL, true) > (size_t)lim) NL = xl ? (NL + 1) / 2 : NL / 2;
    }
    if (!xl && cfg == 0) {
        // 16 staged columns when that keeps more blocks resident per SM (the
        // step is latency-bound: 3 blocks of 16 columns beat 2 of 32 on 131-row
        // lines, 174 vs 190 us per heat3d step; 8 columns lose again)
        int smsm = 0;
        cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        auto resident = [&](size_t b) { return std::min<long long>(8, (long long)smsm / (long long)(b + 1024)); };
        if (resident(smem_for(16, false)) > resident(smem_for(32, false))) {
            cfg = 2;
            NL = 16;
        }
    }
    if (a0.cfg >= 0) {   // forced (autotuner): validate the shape
        cfg = a0.cfg;
        NL = cfg == 2 ? 16 : a0.lines_per_block;
        if (NL < 1 || NL > nl_max || (cfg == 2 && xl) || cfg > 2) return cudaErrorInvalidValue;
        if (!xl && (NL & (NL - 1))) return cudaErrorInvalidValue;
        if (!xl && cfg == 0 && NL != 32) return cudaErrorInvalidValue;
    }
    a.lines_per_block = NL;
    const size_t sm = smem_for(NL, cfg == 1);
    if (sm > (size_t)lim) return cudaErrorInvalidValue;
    // modes 0 (first of several axes) and 3 (1D) run along x, modes 1 and 2 across
    constexpr bool XL = (MODE == 0 || MODE == 3);
    if (xl != XL) return cudaErrorInvalidValue;
    void (*k)(const AxisStepArgs) = nullptr;
    if constexpr (XL) {
        k = cfg == 1 ? axis_step_kernel<VT, KP, W, MODE, XL, 1> : axis_step_kernel<VT, KP, W, MODE, XL, 0>;
    } else {
        k = cfg == 1   ? axis_step_kernel<VT, KP, W, MODE, XL, 1>
            : cfg == 2 ? axis_step_kernel<VT, KP, W, MODE, XL, 2>
                       : axis_step_kernel<VT, KP, W, MODE, XL, 0>;
    }
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if constexpr (XL) {
        k<<<(unsigned)((nlines + NL - 1) / NL), 256, sm, st>>>(a);
    } else {
        const int outer = a.axis == 1 ? a.n[2] : a.n[1];
        dim3 grid((a.n[0] + NL - 1) / NL, outer);
        k<<<grid, 256, sm, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename VT, int KP, int W>
static cudaError_t pick_mode(const AxisStepArgs& a, int mode, cudaStream_t st) {
    switch (mode) {
        case 0: return run_axis_step<VT, KP, W, 0>(a, st);
        case 1: return run_axis_step<VT, KP, W, 1>(a, st);
        case 2: return run_axis_step<VT, KP, W, 2>(a, st);
        case 3: return run_axis_step<VT, KP, W, 3>(a, st);
    }
    return cudaErrorInvalidValue;
}

template <typename VT, int KP>
static cudaError_t pick_w(const AxisStepArgs& a, int mode, cudaStream_t st) {
    switch (a.W) {
        case 3: return pick_mode<VT, KP, 3>(a, mode, st);
        case 5: return pick_mode<VT, KP, 5>(a, mode, st);
        case 7: return pick_mode<VT, KP, 7>(a, mode, st);
        case 9: return pick_mode<VT, KP, 9>(a, mode, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace igapw
