#pragma once
// Set-up kernel of the chunked explicit step's tables (launched by
// launch_chunk_tables in tables.cu; also compiled for the host emulator of
// the tests).
#include "common.cuh"
#include "kernels.h"

namespace igapw {

// ---------------------------------------------------------------------------
// Packed tables of the chunked explicit step (chunkstep.cuh), from the FP64
// factors of factor_kernel.  One thread (set-up, O(n p^2 + P^2 p^3)).
// The line is padded to np = P RS rows (rows n .. np-1: identity rows of the
// factors, zero C and A windows, so they decouple and stay zero) and cut into
// P chunks of exactly RS rows.
// Spikes (the same algebra as factor_kernel, for this partition):
//   forward  y_i = yhat_i - sum_c G[i][c] t_{k-1}[c],  t_{k-1} = last p rows of chunk k-1
//   backward x_i = xhat_i - sum_c H[i][c] h_{k+1}[c],  h_{k+1} = first p rows of chunk k+1
// Chunk operators: t_k = tail(yhat_k) + Phi_k t_{k-1}, Phi_k[r][c] = -G[b_{k+1}-p+r][c];
// h_k = head(xhat_k) + Theta_k h_{k+1}, Theta_k[r][c] = -H[b_k+r][c].  Their products
//   psf[k][d] = Phi_{k-1} ... Phi_{k-d},  psb[k][d] = Theta_{k+1} ... Theta_{k+d}
// map the local tails (heads) of earlier (later) chunks to the incoming one;
// J - 1 is the largest d whose product has an entry above 1e-16.
// ---------------------------------------------------------------------------
__global__ void chunk_tables_kernel(ChunkTableArgs a) {
    if (blockIdx.x * blockDim.x + threadIdx.x != 0) return;
    const int n = a.n, p = a.p, W = a.W, RS = a.RS, P = a.P;
    const int np = P * RS;
    const int nq4 = (2 * W + 4) / 4;
    double* G = a.work;           // [np][p]
    double* H = a.work + np * p;  // [np][p]
    auto bnd = [&](int k) { return k * RS; };
    // factors of the padded line
    auto Lf = [&](int i, int m) { return i < n ? a.L[i * p + m - 1] : 0.0; };
    auto Uf = [&](int i, int m) { return i < n ? a.U[i * p + m - 1] : 0.0; };
    auto Df = [&](int i) { return i < n ? a.dinv[i] : 1.0; };
    for (int k = 0; k < P; ++k) {
        const int b0 = bnd(k), b1 = bnd(k + 1);
        for (int i = b0; i < b1; ++i) {
            for (int c = 0; c < p; ++c) G[i * p + c] = 0.0;
            if (k == 0) continue;
            for (int m = 1; m <= p; ++m) {
                const double l = Lf(i, m);
                const int j = i - m;
                if (j < b0) {
                    if (!IGAPW_IDX("chunk G", j - b0 + p, p)) continue;
                    G[i * p + (j - b0 + p)] += l;
                } else {
                    for (int c = 0; c < p; ++c) G[i * p + c] -= l * G[j * p + c];
                }
            }
        }
    }
    for (int k = 0; k < P; ++k) {
        const int b0 = bnd(k), b1 = bnd(k + 1);
        for (int i = b1 - 1; i >= b0; --i) {
            for (int c = 0; c < p; ++c) H[i * p + c] = 0.0;
            if (k == P - 1) continue;
            for (int m = 1; m <= p; ++m) {
                const double u = Uf(i, m);
                const int j = i + m;
                if (j >= np) continue;
                if (j >= b1) {
                    if (!IGAPW_IDX("chunk H", j - b1, p)) continue;
                    H[i * p + (j - b1)] += u;
                } else {
                    for (int c = 0; c < p; ++c) H[i * p + c] -= u * H[j * p + c];
                }
            }
            for (int c = 0; c < p; ++c) H[i * p + c] *= Df(i);
        }
    }
    // packed rows (padded rows: zero windows starting at the row itself)
    for (int i = 0; i < np; ++i) {
        float* cw = reinterpret_cast<float*>(a.cw + (size_t)i * nq4);
        float* aw = reinterpret_cast<float*>(a.aw + (size_t)i * nq4);
        for (int e = 0; e < 4 * nq4; ++e) { cw[e] = 0.f; aw[e] = 0.f; }
        if (i < n) {
            for (int w = 0; w < W; ++w) {
                cw[2 * w] = a.Cdf[i * W + w].x;
                cw[2 * w + 1] = a.Cdf[i * W + w].y;
                aw[2 * w] = a.Adf[i * W + w].x;
                aw[2 * w + 1] = a.Adf[i * W + w].y;
            }
        }
        const int fs = i < n ? a.fstart[i] : i;
        cw[2 * W] = __int_as_float(fs);
        aw[2 * W] = __int_as_float(fs);
        float fl[4] = {0.f, 0.f, 0.f, 0.f}, fu[4] = {0.f, 0.f, 0.f, 0.f};
        float fg[4] = {0.f, 0.f, 0.f, 0.f}, fh[4] = {0.f, 0.f, 0.f, 0.f};
        // the backward rows are stored scaled by 1 / u_ii, so that the
        // recurrence x_i = dinv_i yhat_i - sum (G dinv)_i t - sum (u dinv)_{i,m} x_{i+m}
        // has one FMA per row on its dependency chain
        for (int m = 0; m < p; ++m) {
            fl[m] = (float)Lf(i, m + 1);
            fu[m] = (float)(Uf(i, m + 1) * Df(i));
            fg[m] = (float)(G[i * p + m] * Df(i));
            fh[m] = (float)H[i * p + m];
        }
        if (p <= 3) fu[3] = (float)Df(i);
        a.fl[i] = make_float4(fl[0], fl[1], fl[2], fl[3]);
        a.fu[i] = make_float4(fu[0], fu[1], fu[2], fu[3]);
        a.fg[i] = make_float4(fg[0], fg[1], fg[2], fg[3]);
        a.fh[i] = make_float4(fh[0], fh[1], fh[2], fh[3]);
        a.fd[i] = (float)Df(i);
    }
    // chunk operator products
    const int pp = p * p;
    for (int e = 0; e < P * P * pp; ++e) { a.psf[e] = 0.f; a.psb[e] = 0.f; }
    int J = 1;
    double run[IGAPW_MAXP * IGAPW_MAXP], tmp[IGAPW_MAXP * IGAPW_MAXP], op[IGAPW_MAXP * IGAPW_MAXP];
    for (int dir = 0; dir < 2; ++dir) {
        for (int k = 0; k < P; ++k) {
            for (int d = 1; d < P; ++d) {
                // next factor: Phi_{k-d} (forward, k-d >= 1) or Theta_{k+d} (backward, k+d <= P-2)
                const int q = dir == 0 ? k - d : k + d;
                if (dir == 0 ? q < 1 : q > P - 2) break;
                for (int r = 0; r < p; ++r)
                    for (int c = 0; c < p; ++c)
                        op[r * p + c] = dir == 0 ? -G[(bnd(q + 1) - p + r) * p + c] : -H[(bnd(q) + r) * p + c];
                if (d == 1) {
                    for (int e = 0; e < pp; ++e) run[e] = op[e];
                } else {
                    for (int r = 0; r < p; ++r)
                        for (int c = 0; c < p; ++c) {
                            double s = 0.0;
                            for (int m = 0; m < p; ++m) s += run[r * p + m] * op[m * p + c];
                            tmp[r * p + c] = s;
                        }
                    for (int e = 0; e < pp; ++e) run[e] = tmp[e];
                }
                double mx = 0.0;
                for (int e = 0; e < pp; ++e) mx = fmax(mx, fabs(run[e]));
                float* dst = (dir == 0 ? a.psf : a.psb) + ((size_t)k * P + d) * pp;
                for (int e = 0; e < pp; ++e) dst[e] = (float)run[e];
                if (mx > 1e-16 && d + 1 > J) J = d + 1;
                if (mx <= 1e-16) break;
            }
        }
    }
    *a.J = J;
}

}  // namespace igapw
