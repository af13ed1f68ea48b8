#pragma once
// The explicit heat step in split form, FP32-pair mode, with every line held
// in registers chunk by chunk (one kernel launch per axis).
//
// Each step of Sec. 4.2, Eq. (6) solves (Mz (x) My (x) Mx) u' = T(u + dt Lap u)
// with the tested mass M = A_z (x) A_y (x) A_x, A = int T_i B_j, and the tested
// Laplacian sum_a C_a (x) A_others, C = int T_i B_j''.  The other axes' mass
// factors cancel against their inverses, so one step is
//   u' = u + dt * sum_a (A_a^{-1} C_a along axis a) u,
// and the launch for axis a computes, for every line along a,
//   g   = C u                    (double-float: exact products, two-sum)
//   w0  = A^{-1} g_hi            (FP32 banded LU solve)
//   rho = g - A w0               (double-float residual)
//   d   = A^{-1} rho             (FP32)
//   out = base + dt (w0 + d)     (double-float)
// with base = u (first axis) or the accumulator of the earlier axes.
//
// Work layout.  A block holds NL lines (a power of two: lane l of a line
// group) and P chunks per line; thread (l, k) owns rows [k R, k R + R) of
// line l (R = the compile-time chunk length; lines are padded to P R rows
// with decoupled identity rows, so every chunk is full and the unrolled row
// loops carry no guards), keeps g, the forward and the backward iterates of
// those rows in registers,
// and exchanges only p chunk-boundary values per solve direction through
// shared memory.  The partitioned solve: each chunk solves with a zero tail,
// the true tail of the previous chunk is the sum of the local tails of the
// earlier chunks mapped by precomputed products of the p x p spike operators
// (they decay geometrically; products below 1e-16 are dropped), and the
// rank-p spike corrections are fused into the backward sweep and the final
// pass.  The state tile (u, hi and lo interleaved) and w0 live in shared
// memory so that the banded windows of rows near a chunk edge can reach the
// neighbouring chunk's rows.  Tables are read through the read-only cache
// (every lane of a line group reads the same row: one broadcast load).
#include "common.cuh"
#include "kernels.h"

namespace igapw {

namespace chunkstep {

__host__ __device__ constexpr int nq4(int W) { return (2 * W + 4) / 4; }

// shared memory of one block (bytes), shared by kernel and launcher; np = the
// padded line length P * rows
__host__ __device__ inline size_t smem_bytes(bool xl, int np, int W, int NL, int P, int KP) {
    const int nr = np + W;
    // must match the carve-up in chunk_step_kernel: y/z tiles use a row stride of 32
    const size_t cap = xl ? (size_t)NL * (nr | 1) : (size_t)nr * 32;
    return cap * 8 + cap * 8 + cap * 4 + (size_t)2 * P * KP * NL * 4;
}

// Read-only table loads that ask L1 to keep the line (evict_last): the
// tables (a few tens of KB, read by every block) would otherwise be evicted
// by the streaming state tiles that pass through L1 on their way to shared
// memory, and every row's table reads would go to L2.
__device__ __forceinline__ float4 ld_keep(const float4* p) {
#ifdef IGAPW_HOST_EMU
    return *p;
#else
    float4 v;
    asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
#endif
}

// Programmatic dependent launch (the three per-axis launches of a step run
// back to back on one stream): wait() blocks until the previous kernel of the
// stream has completed and its writes are visible; launch_dependents() lets
// the next kernel's blocks start once every block of this one has started.
// Both are no-ops for a launch without the programmatic-serialization
// attribute.
__device__ __forceinline__ void griddep_wait() {
#ifndef IGAPW_HOST_EMU
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void griddep_launch_dependents() {
#ifndef IGAPW_HOST_EMU
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Loads v[0..KP) of a float4 table row.
template <int KP>
__device__ __forceinline__ void ld4(const float4* t, int i, float (&v)[4]) {
    const float4 q = ld_keep(t + i);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}

}  // namespace chunkstep

// MODE: 0 FIRST (acc = u + dt w, lines along x), 1 MID (acc += dt w),
// 2 LAST (u_out = acc + dt w), 3 ONLY (u_out = u + dt w, 1D, along x).
template <int KP, int W, int MODE, int RS>
__global__ void __launch_bounds__(512) chunk_step_kernel(const AxisStepArgs a) {
    constexpr bool XL = (MODE == 0 || MODE == 3);
    constexpr int NQ4 = chunkstep::nq4(W);
    IGAPW_DYNAMIC_SMEM(smem_raw);
    const ChunkDev& T = a.ax.ck;
    const int n = a.ax.n;
    const int P = T.P;
    const int np = P * RS;              // padded line length
    const int NL = a.lines_per_block;
    const int lgNL = __ffs(NL) - 1;
    const int l = threadIdx.x & (NL - 1);
    const int k = threadIdx.x >> lgNL;
    const int nr = np + W;
    // staged tiles: x-lines [line][row] with an odd pitch (conflict-free per
    // lane), y/z-lines [row][32 lines] (a compile-time row stride)
    const int pitch = XL ? (nr | 1) : 32;
    constexpr int ust = XL ? 1 : 32;    // row stride within a staged line
    const int lst = XL ? pitch : 1;     // line stride
    const int cap = XL ? NL * pitch : nr * 32;
    float2* U2 = reinterpret_cast<float2*>(smem_raw);     // u (hi, lo); later the update's base / output
    float2* G2 = U2 + cap;                                // g = C u (hi, lo), own rows
    float* W0 = reinterpret_cast<float*>(G2 + cap);       // w0
    float* TF = W0 + cap;                                 // [P][KP][NL] forward tails
    float* TB = TF + P * KP * NL;                         // [P][KP][NL] backward heads
    const long long ntot = a.ntot;
    const int nx = a.n[0], ny = a.n[1];
    const long long nlines = XL ? (long long)a.n[1] * a.n[2] : (a.axis == 1 ? (long long)nx * a.n[2] : (long long)nx * ny);
    const long long L0 = (long long)blockIdx.x * NL;
    const int nl = (int)min((long long)NL, nlines - L0);
    const long long rs = XL ? 1 : (a.axis == 1 ? (long long)nx : (long long)nx * ny);   // row stride in memory
    // first element of line L0 + ll
    auto line_base = [&](int ll) -> long long {
        const long long L = L0 + ll;
        if (XL) return L * n;
        if (a.axis == 1) {
            const long long z = L / nx;
            return z * nx * ny + (L - z * nx);
        }
        return L;
    };
    const float* uh = static_cast<const float*>(a.u);

    // Dependencies within a step (x, y, z launches): the x launch reads u as
    // the previous step's z launch left it, so it waits for that launch before
    // anything and only then lets the y launch start; the y and z launches
    // read u (final for the step) right away and wait for their predecessor
    // only before they read its accumulator (z also before it writes u).
    if constexpr (XL) {
        chunkstep::griddep_wait();
        chunkstep::griddep_launch_dependents();
    } else {
        chunkstep::griddep_launch_dependents();
    }

    // ---- stage u (all rows of the block's lines) and zero the pad rows --------
    // x-lines are copied line by line, TPL consecutive threads per line
    // (coalesced); a block may have fewer than 32 threads
    const int TPL = min(32, (int)blockDim.x);
    const int tl = threadIdx.x % TPL, tg = threadIdx.x / TPL, ntg = blockDim.x / TPL;
    if (XL) {
        for (int ll = tg; ll < NL; ll += ntg) {
            float2* d = U2 + ll * pitch;
            if (ll < nl) {
                const long long g0 = line_base(ll);
                for (int i = tl; i < n; i += TPL) {
                    if (!IGAPW_IDX("chunk stage x", g0 + i, ntot)) continue;
                    cp_async4(&d[i].x, uh + g0 + i);
                    cp_async4(&d[i].y, uh + g0 + i + ntot);
                }
            } else {
                for (int i = tl; i < n; i += TPL) d[i] = make_float2(0.f, 0.f);
            }
            // padded rows and the window overhang: zero
            for (int i = n + tl; i < pitch; i += TPL) d[i] = make_float2(0.f, 0.f);
            for (int i = np + tl; i < pitch; i += TPL) W0[ll * pitch + i] = 0.f;
        }
    } else {
        const long long g0 = l < nl ? line_base(l) : 0;
        const float* sh = uh + g0;
        const float* sl = sh + ntot;
        const int rsi = (int)rs;
        for (int i = k; i < n; i += P) {
            float2* d = U2 + i * ust + l;
            if (l < nl) {
                if (!IGAPW_IDX("chunk stage c", g0 + (long long)i * rs, ntot)) continue;
                cp_async4(&d->x, sh + i * rsi);
                cp_async4(&d->y, sl + i * rsi);
            } else {
                *d = make_float2(0.f, 0.f);
            }
        }
        for (int i = n + k; i < nr; i += P) U2[i * ust + l] = make_float2(0.f, 0.f);
        for (int i = np + k; i < nr; i += P) W0[i * ust + l] = 0.f;
    }
    cp_async_wait_all();
    __syncthreads();

    const int r0 = k * RS;
    const float2* ul = U2 + l * lst;
    float* wl = W0 + l * lst;
    const int J = __ldg(T.J);

    float y[RS];
    float2* gown = G2 + l * lst + r0 * ust;   // this thread's rows of g
#pragma unroll
    for (int j = 0; j < RS; ++j) y[j] = 0.f;

    // forward local substitution step for row j of the chunk (zero incoming tail)
    auto fwd = [&](int j, int i, float v) {
        float lv[4];
        chunkstep::ld4<KP>(T.fl, i, lv);
        // the p-th neighbour first: only the last FMA waits on y[j-1]
#pragma unroll
        for (int m = KP; m >= 1; --m)
            if (j - m >= 0) v = fmaf(-lv[m - 1], y[j - m], v);
        y[j] = v;
    };
    // composed incoming tail (forward) of chunk k from the exported local tails
    auto tail_in = [&](float (&t)[KP]) {
#pragma unroll
        for (int c = 0; c < KP; ++c) t[c] = 0.f;
        if (k == 0) return;
#pragma unroll
        for (int c = 0; c < KP; ++c) t[c] = TF[((k - 1) * KP + c) * NL + l];
        for (int d = 1; d < J && k - 1 - d >= 0; ++d) {
            const float* ps = T.psf + ((size_t)k * P + d) * KP * KP;
            float s[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) s[c] = TF[((k - 1 - d) * KP + c) * NL + l];
#pragma unroll
            for (int r = 0; r < KP; ++r)
#pragma unroll
                for (int c = 0; c < KP; ++c) t[r] = fmaf(__ldg(ps + r * KP + c), s[c], t[r]);
        }
    };
    auto head_in = [&](float (&h)[KP]) {
#pragma unroll
        for (int c = 0; c < KP; ++c) h[c] = 0.f;
        if (k == P - 1) return;
#pragma unroll
        for (int c = 0; c < KP; ++c) h[c] = TB[((k + 1) * KP + c) * NL + l];
        for (int d = 1; d < J && k + 1 + d <= P - 1; ++d) {
            const float* ps = T.psb + ((size_t)k * P + d) * KP * KP;
            float s[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) s[c] = TB[((k + 1 + d) * KP + c) * NL + l];
#pragma unroll
            for (int r = 0; r < KP; ++r)
#pragma unroll
                for (int c = 0; c < KP; ++c) h[r] = fmaf(__ldg(ps + r * KP + c), s[c], h[r]);
        }
    };
    // backward sweep with the forward spike fused; exports the local head
    auto backward = [&]() {
        float t[KP];
        tail_in(t);
#pragma unroll
        for (int j = RS - 1; j >= 0; --j) {
            const int i = r0 + j;
            float gv[4], uv[4];
            chunkstep::ld4<KP>(T.fg, i, gv);
            chunkstep::ld4<KP>(T.fu, i, uv);
            const float di = (KP <= 3) ? uv[3] : __ldg(T.fd + i);
            // rows scaled by 1 / u_ii: only the last FMA waits on y[j+1]
            float z = y[j] * di;
#pragma unroll
            for (int c = 0; c < KP; ++c) z = fmaf(-gv[c], t[c], z);
#pragma unroll
            for (int m = KP; m >= 1; --m)
                if (j + m < RS) z = fmaf(-uv[m - 1], y[j + m], z);
            y[j] = z;
        }
        if (k > 0) {
#pragma unroll
            for (int c = 0; c < KP; ++c) TB[(k * KP + c) * NL + l] = y[c];
        }
    };
    // final backward spike: y = x_hat - H h
    auto finish_solve = [&]() {
        float h[KP];
        head_in(h);
        if (k == P - 1) return;
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            float hv[4];
            chunkstep::ld4<KP>(T.fh, r0 + j, hv);
            float v = y[j];
#pragma unroll
            for (int c = 0; c < KP; ++c) v = fmaf(-hv[c], h[c], v);
            y[j] = v;
        }
    };

    // ---- P1: g = C u (double-float) fused with the forward sweep of w0 --------
#pragma unroll
    for (int j = 0; j < RS; ++j) {
        const int i = r0 + j;
        float cv[NQ4 * 4];
#pragma unroll
        for (int q = 0; q < NQ4; ++q) {
            const float4 c4 = chunkstep::ld_keep(T.cw + (size_t)i * NQ4 + q);
            cv[4 * q] = c4.x;
            cv[4 * q + 1] = c4.y;
            cv[4 * q + 2] = c4.z;
            cv[4 * q + 3] = c4.w;
        }
        const int fs = __float_as_int(cv[2 * W]);
        if (!IGAPW_IDX("chunk P1 window", fs + W - 1, nr)) continue;
        const float2* uu = ul + fs * ust;
        float s, cc;
        {
            const float2 v = uu[0];
            s = cv[0] * v.x;
            cc = fmaf(cv[0], v.x, -s);
            cc = fmaf(cv[0], v.y, cc);
            cc = fmaf(cv[1], v.x, cc);
        }
#pragma unroll
        for (int w = 1; w < W; ++w) {
            const float2 v = uu[w * ust];
            const float ch = cv[2 * w], cl = cv[2 * w + 1];
            const float pr = ch * v.x;
            float e = fmaf(ch, v.x, -pr);
            e = fmaf(ch, v.y, e);
            e = fmaf(cl, v.x, e);
            float s2, er;
            two_sum(s, pr, s2, er);
            s = s2;
            cc += er + e;
        }
        float gh, gl;
        fast_two_sum(s, cc, gh, gl);
        gown[j * ust] = make_float2(gh, gl);
        fwd(j, i, gh);
    }
    if (k < P - 1) {
#pragma unroll
        for (int c = 0; c < KP; ++c) TF[(k * KP + c) * NL + l] = y[RS - KP + c];
    }
    __syncthreads();
    backward();
    __syncthreads();
    finish_solve();
    // publish w0 for the residual windows of the neighbouring rows
#pragma unroll
    for (int j = 0; j < RS; ++j) wl[(r0 + j) * ust] = y[j];
    __syncthreads();

    // the base of the update: the accumulator of the earlier axes (y/z lines),
    // staged into the dead u tile while the residual and the correction run
    if constexpr (!XL) {
        chunkstep::griddep_wait();   // the previous axis' accumulator is complete
        if (l < nl) {
            // 32-bit row offsets from per-line pointers (a line spans < 2^31 elements)
            const long long g0 = line_base(l) + (long long)r0 * rs;
            const float* ah = static_cast<const float*>(a.acc) + g0;
            const float* al = ah + ntot;
            const int rsi = (int)rs;
            const int R = min(RS, n - r0);   // rows of the chunk inside the line
            for (int j = 0; j < R; ++j) {
                if (!IGAPW_IDX("chunk base", g0 + (long long)j * rs, ntot)) continue;
                float2* d = U2 + (r0 + j) * ust + l;
                cp_async4(&d->x, ah + j * rsi);
                cp_async4(&d->y, al + j * rsi);
            }
        }
    }

    // ---- P3: rho = g - A w0 (double-float) fused with the forward sweep -------
#pragma unroll
    for (int j = 0; j < RS; ++j) {
        const int i = r0 + j;
        float av[NQ4 * 4];
#pragma unroll
        for (int q = 0; q < NQ4; ++q) {
            const float4 a4 = chunkstep::ld_keep(T.aw + (size_t)i * NQ4 + q);
            av[4 * q] = a4.x;
            av[4 * q + 1] = a4.y;
            av[4 * q + 2] = a4.z;
            av[4 * q + 3] = a4.w;
        }
        const int fs = __float_as_int(av[2 * W]);
        if (!IGAPW_IDX("chunk P3 window", fs + W - 1, nr)) continue;
        const float* ww = wl + fs * ust;
        const float2 g = gown[j * ust];
        float s = g.x, cc = g.y;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float x = ww[w * ust];
            const float ah = -av[2 * w], al = -av[2 * w + 1];
            const float pr = ah * x;
            float e = fmaf(ah, x, -pr);
            e = fmaf(al, x, e);
            float s2, er;
            two_sum(s, pr, s2, er);
            s = s2;
            cc += er + e;
        }
        fwd(j, i, s + cc);
    }
    if (k < P - 1) {
#pragma unroll
        for (int c = 0; c < KP; ++c) TF[(k * KP + c) * NL + l] = y[RS - KP + c];
    }
    __syncthreads();
    backward();
    __syncthreads();
    finish_solve();

    // ---- P5: out = base + dt (w0 + d) ------------------------------------------
    float dth, dtl;
    split_double(a.dt, dth, dtl);
    if constexpr (!XL) cp_async_wait_all();   // own rows only: no barrier needed
    unsigned bad = 0;
    float* oh = static_cast<float*>((MODE == 0 || MODE == 1) ? a.acc : a.u_out);
    const long long gl0 = (!XL && l < nl) ? line_base(l) : 0;
    // this thread's first row of the line (y/z lines), advanced row by row
    float* oq = oh + gl0 + (long long)r0 * rs;
    const long long rsl = rs;
#pragma unroll
    for (int j = 0; j < RS; ++j) {
        const int i = r0 + j;
        const float w0 = wl[i * ust];
        const float ph = dth * w0;
        float pe = fmaf(dth, w0, -ph);
        pe = fmaf(dtl, w0, pe);
        pe = fmaf(dth, y[j], pe);
        float2* bp = U2 + l * lst + i * ust;
        const float2 b = *bp;
        float s, e;
        two_sum(b.x, ph, s, e);
        float hi, lo;
        fast_two_sum(s, b.y + (pe + e), hi, lo);
        if (!isfinite(hi)) bad = 1;
        if (XL) {
            *bp = make_float2(hi, lo);
        } else {
            if (l < nl && i < n && IGAPW_IDX("chunk out", gl0 + (long long)i * rs, ntot)) {
                oq[0] = hi;
                oq[ntot] = lo;
            }
            oq += rsl;
        }
    }
    if constexpr (XL) {
        __syncthreads();
        for (int ll = tg; ll < nl; ll += ntg) {
            const long long g0 = line_base(ll);
            const float2* s = U2 + ll * pitch;
            for (int i = tl; i < n; i += TPL) {
                if (!IGAPW_IDX("chunk out x", g0 + i, ntot)) continue;
                const float2 v = s[i];
                oh[g0 + i] = v.x;
                oh[g0 + i + ntot] = v.y;
            }
        }
    }
    if (bad && a.status) atomicOr(a.status, STATUS_NONFINITE);
}

#ifndef IGAPW_HOST_EMU
// Launch: lines_per_block = NL (32, 16 or 8); P chunks per line from the tables.
template <int KP, int W, int MODE, int RS>
static cudaError_t run_chunk_step(const AxisStepArgs& a, cudaStream_t st) {
    constexpr bool XL = (MODE == 0 || MODE == 3);
    const int n = a.ax.n, P = a.ax.ck.P, NL = a.lines_per_block;
    if (P <= 0 || a.ax.ck.rows != RS || (NL != 8 && NL != 16 && NL != 32) || NL * P > 512 ||
        (long long)(P - 1) * RS >= n || (long long)P * RS < n)
        return cudaErrorInvalidValue;
    const int np = P * RS;
    if ((a.axis == 0) != XL) return cudaErrorInvalidValue;
    const long long nlines = XL ? (long long)a.n[1] * a.n[2]
                                : (a.axis == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
    const size_t sm = chunkstep::smem_bytes(XL, np, W, NL, P, KP);
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sm > (size_t)lim) return cudaErrorInvalidValue;
    auto kern = chunk_step_kernel<KP, W, MODE, RS>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const long long blocks = (nlines + NL - 1) / NL;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)(NL * P));
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

#endif  // IGAPW_HOST_EMU

}  // namespace igapw
