// Kernel (b): contraction launch dispatch (operator, system and residual
// modes; the kernel template is in contract.cuh) and the source RHS kernels.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "contract.cuh"

namespace igapw {

template <int DIM, int W>
static cudaError_t dispatch_mode(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st) {
    if (mode == MODE_RES) {
        if (cmp == FMT_F64) return pick_tile<DIM, W, double, MODE_RES, FMT_PAIR>(a, st);
        return pick_tile<DIM, W, DF, MODE_RES, FMT_PAIR>(a, st);
    }
    if (io == FMT_F64) {
        if (mode == MODE_OP) return pick_tile<DIM, W, double, MODE_OP, FMT_F64>(a, st);
        return pick_tile<DIM, W, double, MODE_SYS, FMT_F64>(a, st);
    }
    if (mode == MODE_OP) return pick_tile<DIM, W, DF, MODE_OP, FMT_PAIR>(a, st);
    return pick_tile<DIM, W, DF, MODE_SYS, FMT_PAIR>(a, st);
}

template <int DIM>
static cudaError_t dispatch_w(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st) {
    switch (a.W) {
        case 3: return dispatch_mode<DIM, 3>(a, mode, cmp, io, st);
        case 5: return dispatch_mode<DIM, 5>(a, mode, cmp, io, st);
        case 7: return dispatch_mode<DIM, 7>(a, mode, cmp, io, st);
        case 9: return dispatch_mode<DIM, 9>(a, mode, cmp, io, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_contract(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st) {
    switch (a.dim) {
        case 1: return dispatch_w<1>(a, mode, cmp, io, st);
        case 2: return dispatch_w<2>(a, mode, cmp, io, st);
        case 3: return dispatch_w<3>(a, mode, cmp, io, st);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Kernel (b-src): source right-hand side b = (TW_z TW_y TW_x) f, one pass per
// axis.  A pass maps in[(o*Qa + q)*Ni + x] to out[(o*na + i)*Ni + x] with
// out = sum_w TW[i][w] in[.. pstart[i] + w ..]: PW sums the weights of the
// cell's points (test 1), Galerkin multiplies by the test B-spline.
// ---------------------------------------------------------------------------
template <typename CT, int IN_F32, int OUT_PLANES>
__global__ void __launch_bounds__(256) source_pass_kernel(const void* in, void* out, long long nout_total,
                                                          int Qa, int na, long long Ni, long long No,
                                                          int wq, const int* __restrict__ pstart,
                                                          TableSet tw, long long plane_out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = No * na * Ni;
    if (e >= total) return;
    const long long x = e % Ni;
    const long long t = e / Ni;
    const int i = (int)(t % na);
    const long long o = t / na;
    const int ps = pstart[i];
    Acc<CT> acc;
    acc.init();
    for (int w = 0; w < wq; ++w) {
        const int q = ps + w;
        if (q >= Qa) break;
        const long long gi = (o * Qa + q) * Ni + x;
        if (!IGAPW_IDX("source pass in", gi, No * (long long)Qa * Ni)) continue;
        CT v;
        if constexpr (std::is_same<CT, double>::value) {
            v = IN_F32 ? (double)((const float*)in)[gi] : ((const double*)in)[gi];
        } else {
            if constexpr (IN_F32) v = DF{((const float*)in)[gi], 0.f};
            else v = ((const DF*)in)[gi];
        }
        acc.add_prod(tab<CT>(tw, i * wq + w), v);
    }
    const CT r = acc.result();
    if constexpr (std::is_same<CT, double>::value) {
        ((double*)out)[e] = r;
    } else {
        if constexpr (OUT_PLANES) {
            ((float*)out)[e] = r.hi;
            ((float*)out)[e + plane_out] = r.lo;
        } else {
            ((DF*)out)[e] = r;
        }
    }
    (void)nout_total;
}

// ---------------------------------------------------------------------------
// Kernel (b-src), PW tests: every quadrature point lies in exactly one test
// cell per axis, so b[k][j][i] is the weighted sum of the samples of the cell
// (k, j, i) alone (Sec. 4.1 PW loop: weight times 1.0) -- one thread per
// coefficient, each sample read once, x-neighbouring threads reading
// neighbouring cells (coalesced).  Pair mode: x sums in double-float, the
// y/z weight products exact (df_mul), accumulation compensated.
// ---------------------------------------------------------------------------
template <typename CT, int IN_F32>
__global__ void __launch_bounds__(256) source_pw_kernel(const SourceArgs a) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    if (e >= (long long)nx * ny * nz) return;
    const int i = (int)(e % nx);
    const long long t = e / nx;
    const int j = (int)(t % ny);
    const int k = (int)(t / ny);
    const int Qx = a.q[0], Qy = a.q[1], Qz = a.q[2];
    const AxisDev& X = a.ax[0];
    const int wx = X.wq, psx = X.pstart[i];
    const int wy = a.dim >= 2 ? a.ax[1].wq : 1, psy = a.dim >= 2 ? a.ax[1].pstart[j] : 0;
    const int wz = a.dim >= 3 ? a.ax[2].wq : 1, psz = a.dim >= 3 ? a.ax[2].pstart[k] : 0;
    Acc<CT> acc;
    acc.init();
    for (int az = 0; az < wz; ++az) {
        const int qz = psz + az;
        if (qz >= Qz) break;
        const CT tz = a.dim >= 3 ? tab<CT>(a.ax[2].TW, k * wz + az) : from_double<CT>(1.0);
        for (int by = 0; by < wy; ++by) {
            const int qy = psy + by;
            if (qy >= Qy) break;
            const CT ty = a.dim >= 2 ? tab<CT>(a.ax[1].TW, j * wy + by) : from_double<CT>(1.0);
            const long long row = ((long long)qz * Qy + qy) * Qx;
            Acc<CT> sx;
            sx.init();
            for (int c = 0; c < wx; ++c) {
                const int qx = psx + c;
                if (qx >= Qx) break;
                if (!IGAPW_IDX("source pw f", row + qx, (long long)Qx * Qy * a.q[2])) continue;
                const CT tw = tab<CT>(X.TW, i * wx + c);
                if constexpr (std::is_same<CT, double>::value) {
                    const double fv = IN_F32 ? (double)((const float*)a.f)[row + qx] : ((const double*)a.f)[row + qx];
                    sx.add_prod(tw, fv);
                } else {
                    sx.add_prod_f(tw, ((const float*)a.f)[row + qx]);
                }
            }
            if constexpr (std::is_same<CT, double>::value) acc.add_prod(tz * ty, sx.result());
            else acc.add_prod(df_mul(tz, ty), sx.result());
        }
    }
    const CT r = acc.result();
    if (!IGAPW_IDX("source out", e, a.ntot)) return;
    if constexpr (std::is_same<CT, double>::value) {
        ((double*)a.out)[e] = r;
    } else {
        ((float*)a.out)[e] = r.hi;
        ((float*)a.out)[e + a.ntot] = r.lo;
    }
}

// ---------------------------------------------------------------------------
// Neumann face term (Sec. 4.3): for every coefficient of the end face of a
// Neumann axis, the tests of the other axes (their point windows, PW or
// B-spline) applied to the face data g, added to the end row (the only test
// that is non-zero at the end).  One thread per face coefficient.
// ---------------------------------------------------------------------------
template <typename CT, int IN_F32>
__global__ void __launch_bounds__(256) neumann_face_kernel(const NeumannArgs a) {
    int o[2] = {0, 0};
    int no = 0;
    for (int k = 0; k < a.dim; ++k)
        if (k != a.axis) o[no++] = k;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n0 = a.n[o[0]], n1 = no > 1 ? a.n[o[1]] : 1;
    if (e >= (long long)n0 * n1) return;
    const int i0 = (int)(e % n0), i1 = (int)(e / n0);
    const AxisDev& A0 = a.ax[o[0]];
    const int w0 = A0.wq, ps0 = A0.pstart[i0], Q0 = a.q[o[0]];
    const int w1 = no > 1 ? a.ax[o[1]].wq : 1, ps1 = no > 1 ? a.ax[o[1]].pstart[i1] : 0;
    const int Q1 = no > 1 ? a.q[o[1]] : 1;
    Acc<CT> acc;
    acc.init();
    for (int c1 = 0; c1 < w1; ++c1) {
        const int q1 = ps1 + c1;
        if (q1 >= Q1) break;
        const CT t1 = no > 1 ? tab<CT>(a.ax[o[1]].TW, i1 * w1 + c1) : from_double<CT>(1.0);
        Acc<CT> s0;
        s0.init();
        for (int c0 = 0; c0 < w0; ++c0) {
            const int q0 = ps0 + c0;
            if (q0 >= Q0) break;
            const CT tw = tab<CT>(A0.TW, i0 * w0 + c0);
            const long long gi = (long long)q1 * Q0 + q0;
            if constexpr (std::is_same<CT, double>::value) {
                s0.add_prod(tw, IN_F32 ? (double)((const float*)a.g)[gi] : ((const double*)a.g)[gi]);
            } else {
                s0.add_prod_f(tw, ((const float*)a.g)[gi]);
            }
        }
        acc.add_prod(t1, s0.result());
    }
    int idx[3] = {0, 0, 0};
    idx[o[0]] = i0;
    if (no > 1) idx[o[1]] = i1;
    idx[a.axis] = a.side ? a.n[a.axis] - 1 : 0;
    const long long g = ((long long)idx[2] * a.n[1] + idx[1]) * a.n[0] + idx[0];
    const CT r = acc.result();
    if constexpr (std::is_same<CT, double>::value) {
        ((double*)a.b)[g] += r;
    } else {
        float* b = (float*)a.b;
        DFAcc t;
        t.s = b[g];
        t.c = b[g + a.ntot];
        t.add(r);
        const DF v = t.result();
        b[g] = v.hi;
        b[g + a.ntot] = v.lo;
    }
}

// The first term of a compensated sum: the exact product split (double-float)
// or the product (FP64) starts the accumulator, which saves the two-sum of
// adding it to zero.
__device__ __forceinline__ void acc_first_prod_f(Acc<DF>& a, DF t, float v) {
    a.s = t.hi * v;
    float e = fmaf(t.hi, v, -a.s);
    a.c = fmaf(t.lo, v, e);
}
__device__ __forceinline__ void acc_first_prod_f(Acc<double>& a, double t, double v) { a.s = t * v; }
__device__ __forceinline__ void acc_first_prod(Acc<DF>& a, DF t, DF v) {
    a.s = t.hi * v.hi;
    float e = fmaf(t.hi, v.hi, -a.s);
    e = fmaf(t.hi, v.lo, e);
    a.c = fmaf(t.lo, v.hi, e);
}
__device__ __forceinline__ void acc_first_prod(Acc<double>& a, double t, double v) { a.s = t * v; }

// PW source, loads batched: for every z point of the cell, the whole y-by-x
// slab of the cell's samples (its own point counts, at most MAXW per axis) is
// loaded before it is summed, so a thread keeps up to MAXW^2 loads in flight.
// MAXW is the largest point count per cell over the axes (2, 3 or 4): the slab
// loops are unrolled and predicated, so a MAXW above the real counts would
// issue the masked-off compensated products all the same.  One thread per
// coefficient (i, j) of a z-plane (32-bit index; the host keeps nx * ny below
// 2^31 - 256); the grid's y dimension walks the planes, and the x and y test
// weights are loaded once per thread.
template <typename CT, int IN_F32, int MAXW>
__global__ void __launch_bounds__(256) source_pw_rows_kernel(const SourceArgs a) {
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int plane = nx * ny;
    const int pe = blockIdx.x * blockDim.x + threadIdx.x;
    if (pe >= plane) return;
    const int j = pe / nx;
    const int i = pe - j * nx;
    const int Qx = a.q[0], Qy = a.q[1];
    const AxisDev& X = a.ax[0];
    const int wx = X.wq, psx = X.pstart[i], cx = X.pcount[i];
    const int wy = a.dim >= 2 ? a.ax[1].wq : 1, psy = a.dim >= 2 ? a.ax[1].pstart[j] : 0;
    const int cy = a.dim >= 2 ? a.ax[1].pcount[j] : 1;
    using FT = typename std::conditional<IN_F32 != 0, float, double>::type;
    CT tx[MAXW], ty[MAXW];
#pragma unroll
    for (int c = 0; c < MAXW; ++c) {
        tx[c] = c < cx ? tab<CT>(X.TW, i * wx + c) : zero_v<CT>();
        ty[c] = (a.dim < 2) ? (c == 0 ? from_double<CT>(1.0) : zero_v<CT>())
                            : (c < cy ? tab<CT>(a.ax[1].TW, j * wy + c) : zero_v<CT>());
    }
    // the products of the x and y test weights, once for all the thread's planes
    CT txy[MAXW][MAXW];
#pragma unroll
    for (int by = 0; by < MAXW; ++by)
#pragma unroll
        for (int c = 0; c < MAXW; ++c) {
            if constexpr (std::is_same<CT, double>::value) txy[by][c] = ty[by] * tx[c];
            else txy[by][c] = df_mul(ty[by], tx[c]);
        }
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const long long e = (long long)k * plane + pe;
        const int wz = a.dim >= 3 ? a.ax[2].wq : 1, psz = a.dim >= 3 ? a.ax[2].pstart[k] : 0;
        const int cz = a.dim >= 3 ? a.ax[2].pcount[k] : 1;
        // b = sum_z tz (sum_{y,x} (ty tx) f): per z point of the cell one
        // compensated sum over its y-by-x samples, weighted by tz into b
        Acc<CT> acc;
        acc.init();
        for (int az = 0; az < cz; ++az) {
            const int qz = psz + az;
            const CT tz = a.dim >= 3 ? tab<CT>(a.ax[2].TW, k * wz + az) : from_double<CT>(1.0);
            FT fv[MAXW][MAXW];
#pragma unroll
            for (int by = 0; by < MAXW; ++by) {
                const long long row = ((long long)qz * Qy + (psy + by)) * Qx + psx;
                if constexpr (MAXW == 2 && IN_F32 != 0) {
                    // a 2-point cell row as one 8-byte load where it is aligned
                    fv[by][0] = fv[by][1] = FT(0);
                    if (by < cy) {
                        if (cx == 2 && (row & 1) == 0 &&
                            IGAPW_IDX("source rows f", row + 1, (long long)Qx * Qy * a.q[2])) {
                            const float2 v = __ldg(reinterpret_cast<const float2*>((const float*)a.f + row));
                            fv[by][0] = v.x;
                            fv[by][1] = v.y;
                        } else {
#pragma unroll
                            for (int c = 0; c < 2; ++c)
                                if (c < cx && IGAPW_IDX("source rows f", row + c, (long long)Qx * Qy * a.q[2]))
                                    fv[by][c] = ((const FT*)a.f)[row + c];
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < MAXW; ++c)
                        fv[by][c] = (by < cy && c < cx &&
                                     IGAPW_IDX("source rows f", row + c, (long long)Qx * Qy * a.q[2]))
                                        ? ((const FT*)a.f)[row + c]
                                        : FT(0);
                }
            }
            // every sum starts from its first product (the windows hold at
            // least one point unless the row is a Dirichlet row)
            Acc<CT> sxy;
            if (cx > 0 && cy > 0) acc_first_prod_f(sxy, txy[0][0], fv[0][0]);
            else sxy.init();
#pragma unroll
            for (int by = 0; by < MAXW; ++by)
#pragma unroll
                for (int c = 0; c < MAXW; ++c) {
                    if ((by > 0 || c > 0) && by < cy && c < cx) {
                        if constexpr (std::is_same<CT, double>::value) sxy.add_prod(txy[by][c], (double)fv[by][c]);
                        else sxy.add_prod_f(txy[by][c], (float)fv[by][c]);
                    }
                }
            if (az == 0) acc_first_prod(acc, tz, sxy.result());
            else acc.add_prod(tz, sxy.result());
        }
        const CT r = acc.result();
        if (!IGAPW_IDX("source rows out", e, a.ntot)) continue;
        if constexpr (std::is_same<CT, double>::value) {
            ((double*)a.out)[e] = r;
        } else {
            ((float*)a.out)[e] = r.hi;
            ((float*)a.out)[e + a.ntot] = r.lo;
        }
    }
}

// PW source with the x-window of every sample row loaded before it is summed
// (up to MAXW points per cell and axis, predicated): the loads of a row are in
// flight together instead of one per dependent compensated product.
template <typename CT, int IN_F32, int MAXW>
__global__ void __launch_bounds__(256) source_pw_xrow_kernel(const SourceArgs a) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    if (e >= (long long)nx * ny * nz) return;
    const int i = (int)(e % nx);
    const long long t = e / nx;
    const int j = (int)(t % ny);
    const int k = (int)(t / ny);
    const int Qx = a.q[0], Qy = a.q[1], Qz = a.q[2];
    const AxisDev& X = a.ax[0];
    const int wx = X.wq, psx = X.pstart[i];
    const int wy = a.dim >= 2 ? a.ax[1].wq : 1, psy = a.dim >= 2 ? a.ax[1].pstart[j] : 0;
    const int wz = a.dim >= 3 ? a.ax[2].wq : 1, psz = a.dim >= 3 ? a.ax[2].pstart[k] : 0;
    CT tx[MAXW];
#pragma unroll
    for (int c = 0; c < MAXW; ++c) tx[c] = c < wx ? tab<CT>(X.TW, i * wx + c) : zero_v<CT>();
    Acc<CT> acc;
    acc.init();
    for (int az = 0; az < wz; ++az) {
        const int qz = psz + az;
        if (qz >= Qz) break;
        const CT tz = a.dim >= 3 ? tab<CT>(a.ax[2].TW, k * wz + az) : from_double<CT>(1.0);
        for (int by = 0; by < wy; ++by) {
            const int qy = psy + by;
            if (qy >= Qy) break;
            const CT ty = a.dim >= 2 ? tab<CT>(a.ax[1].TW, j * wy + by) : from_double<CT>(1.0);
            const long long row = ((long long)qz * Qy + qy) * Qx;
            float fv[MAXW];
            double dv[MAXW];
#pragma unroll
            for (int c = 0; c < MAXW; ++c) {
                const int qx = psx + c;
                const bool in = c < wx && qx < Qx && IGAPW_IDX("source xrow f", row + qx, (long long)Qx * Qy * Qz);
                if constexpr (IN_F32) fv[c] = in ? ((const float*)a.f)[row + qx] : 0.f;
                else dv[c] = in ? ((const double*)a.f)[row + qx] : 0.0;
            }
            Acc<CT> sx;
            sx.init();
#pragma unroll
            for (int c = 0; c < MAXW; ++c) {
                if (c < wx) {
                    if constexpr (std::is_same<CT, double>::value) sx.add_prod(tx[c], IN_F32 ? (double)fv[c] : dv[c]);
                    else sx.add_prod_f(tx[c], fv[c]);
                }
            }
            if constexpr (std::is_same<CT, double>::value) acc.add_prod(tz * ty, sx.result());
            else acc.add_prod(df_mul(tz, ty), sx.result());
        }
    }
    const CT r = acc.result();
    if (!IGAPW_IDX("source out", e, a.ntot)) return;
    if constexpr (std::is_same<CT, double>::value) {
        ((double*)a.out)[e] = r;
    } else {
        ((float*)a.out)[e] = r.hi;
        ((float*)a.out)[e + a.ntot] = r.lo;
    }
}

// ---------------------------------------------------------------------------
// Source RHS of a separable source f = amp prod_a sin(k_a pi x_a): because the
// tests are tensor products, b = amp (x)_a v_a with the 1D factors
// v_a[i] = sum_w TW_a[i][w] sin(k_a pi x_{pstart[i] + w}) (the same sums the
// axis passes of the general source RHS form), in FP64.
// ---------------------------------------------------------------------------
__global__ void sine_factor_kernel(int n, int wq, int Q, const int* __restrict__ pstart,
                                   const double* __restrict__ tw, const double* __restrict__ qx, double k,
                                   double* __restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int w = 0; w < wq; ++w) {
        const int q = pstart[i] + w;
        const double t = tw[(size_t)i * wq + w];
        if (q >= Q || t == 0.0) continue;
        s = fma(t, sinpi(k * qx[q]), s);
    }
    v[i] = s;
}

template <bool PAIR>
__global__ void __launch_bounds__(256) sine_outer_kernel(long long ntot, int nx, int ny, double amp,
                                                         const double* __restrict__ vx, const double* __restrict__ vy,
                                                         const double* __restrict__ vz, void* out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ntot) return;
    const long long nxy = (long long)nx * ny;
    const int z = (int)(e / nxy);
    const long long r = e - (long long)z * nxy;
    const int y = (int)(r / nx), x = (int)(r - (long long)y * nx);
    const double b = amp * vz[z] * vy[y] * vx[x];
    if constexpr (PAIR) {
        float h, l;
        split_double(b, h, l);
        static_cast<float*>(out)[e] = h;
        static_cast<float*>(out)[e + ntot] = l;
    } else {
        static_cast<double*>(out)[e] = b;
    }
}

cudaError_t launch_source_sine(const SineSourceArgs& a, int fp64, cudaStream_t st) {
    for (int d = 0; d < a.dim; ++d) {
        const AxisDev& X = a.ax[d];
        sine_factor_kernel<<<(X.n + 127) / 128, 128, 0, st>>>(X.n, X.wq, a.q[d], X.pstart, X.TW.d, a.qx[d], a.k[d],
                                                              a.v[d]);
    }
    const long long blocks = (a.ntot + 255) / 256;
    if (fp64)
        sine_outer_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(a.ntot, a.n[0], a.n[1], a.amp, a.v[0], a.v[1],
                                                                  a.v[2], a.out);
    else
        sine_outer_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(a.ntot, a.n[0], a.n[1], a.amp, a.v[0], a.v[1],
                                                                 a.v[2], a.out);
    return cudaGetLastError();
}

cudaError_t launch_neumann(const NeumannArgs& a, int fp64, cudaStream_t st) {
    long long face = 1;
    for (int k = 0; k < a.dim; ++k)
        if (k != a.axis) face *= a.n[k];
    const unsigned blocks = (unsigned)((face + 255) / 256);
    if (fp64) neumann_face_kernel<double, 0><<<blocks, 256, 0, st>>>(a);
    else neumann_face_kernel<DF, 1><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_source(const SourceArgs& a, int fp64, cudaStream_t st) {
    if (a.pw) {
        const long long total = (long long)a.n[0] * a.n[1] * a.n[2];
        const unsigned blocks = (unsigned)((total + 255) / 256);
        int wmax = a.ax[0].wq;
        for (int k = 1; k < a.dim; ++k) wmax = std::max(wmax, a.ax[k].wq);
        const long long plane = (long long)a.n[0] * a.n[1];
        if (wmax <= 4 && plane <= INT_MAX - 256) {
            // z planes per thread: enough blocks for 16 per SM, the rest of the
            // planes walked by each thread, which loads its x and y test weights
            // and windows once for all of them
            const long long xb = (plane + 255) / 256;
            int sms = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const long long zb = std::max<long long>(1, (16LL * std::max(sms, 1) + xb - 1) / xb);
            const dim3 grid((unsigned)xb, (unsigned)std::min<long long>(std::min<long long>(a.n[2], zb), 65535));
            if (wmax <= 2) {
                if (fp64) source_pw_rows_kernel<double, 0, 2><<<grid, 256, 0, st>>>(a);
                else source_pw_rows_kernel<DF, 1, 2><<<grid, 256, 0, st>>>(a);
            } else if (wmax == 3) {
                if (fp64) source_pw_rows_kernel<double, 0, 3><<<grid, 256, 0, st>>>(a);
                else source_pw_rows_kernel<DF, 1, 3><<<grid, 256, 0, st>>>(a);
            } else {
                if (fp64) source_pw_rows_kernel<double, 0, 4><<<grid, 256, 0, st>>>(a);
                else source_pw_rows_kernel<DF, 1, 4><<<grid, 256, 0, st>>>(a);
            }
        } else if (a.ax[0].wq <= 8) {
            if (fp64) source_pw_xrow_kernel<double, 0, 8><<<blocks, 256, 0, st>>>(a);
            else source_pw_xrow_kernel<DF, 1, 8><<<blocks, 256, 0, st>>>(a);
        } else if (a.ax[0].wq <= 16) {
            if (fp64) source_pw_xrow_kernel<double, 0, 16><<<blocks, 256, 0, st>>>(a);
            else source_pw_xrow_kernel<DF, 1, 16><<<blocks, 256, 0, st>>>(a);
        } else {
            if (fp64) source_pw_kernel<double, 0><<<blocks, 256, 0, st>>>(a);
            else source_pw_kernel<DF, 1><<<blocks, 256, 0, st>>>(a);
        }
        return cudaGetLastError();
    }
    // Galerkin: passes x (Ni = 1), then y (Ni = n_x), then z (Ni = n_x n_y)
    const int d = a.dim;
    long long dims_in[3] = {a.q[0], d >= 2 ? a.q[1] : 1, d >= 3 ? a.q[2] : 1};
    const void* src = a.f;
    void* bufs[2] = {a.work0, a.work1};
    for (int ax = 0; ax < d; ++ax) {
        long long Ni = 1, No = 1;
        for (int k = 0; k < ax; ++k) Ni *= dims_in[k];
        for (int k = ax + 1; k < 3; ++k) No *= dims_in[k];
        const int Qa = (int)dims_in[ax], na = a.n[ax];
        const bool last = (ax == d - 1);
        void* dst = last ? a.out : bufs[ax & 1];
        const long long total = No * na * Ni;
        const unsigned blocks = (unsigned)((total + 255) / 256);
        const AxisDev& A = a.ax[ax];
        if (fp64) {
            source_pass_kernel<double, 0, 0><<<blocks, 256, 0, st>>>(src, dst, total, Qa, na, Ni, No, A.wq,
                                                                      A.pstart, A.TW, a.ntot);
        } else if (ax == 0) {
            if (last) source_pass_kernel<DF, 1, 1><<<blocks, 256, 0, st>>>(src, dst, total, Qa, na, Ni, No, A.wq, A.pstart, A.TW, a.ntot);
            else source_pass_kernel<DF, 1, 0><<<blocks, 256, 0, st>>>(src, dst, total, Qa, na, Ni, No, A.wq, A.pstart, A.TW, a.ntot);
        } else {
            if (last) source_pass_kernel<DF, 0, 1><<<blocks, 256, 0, st>>>(src, dst, total, Qa, na, Ni, No, A.wq, A.pstart, A.TW, a.ntot);
            else source_pass_kernel<DF, 0, 0><<<blocks, 256, 0, st>>>(src, dst, total, Qa, na, Ni, No, A.wq, A.pstart, A.TW, a.ntot);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dims_in[ax] = na;
        src = dst;
    }
    return cudaSuccess;
}

}  // namespace igapw
