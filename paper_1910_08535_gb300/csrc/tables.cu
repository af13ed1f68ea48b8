// Kernel (a): Cox--de Boor basis / derivative tables at the quadrature points
// and their fold into banded per-axis tables; kernel (c1): FP64 banded LU of
// the per-axis system matrices plus the data of the partitioned line solve.
#include "common.cuh"
#include "kernels.h"
#include "chunktables.cuh"

namespace igapw {

// ---------------------------------------------------------------------------
// (a1) basis table.  One thread per quadrature point x_q lying in the knot span
// [t_s, t_{s+1}), s = first + p.  The p+1 non-zero B-splines B_{s-p..s, p} are
// built degree by degree with the Cox--de Boor recursion
//   B_{j,k} = (x - t_j)/(t_{j+k} - t_j) B_{j,k-1} + (t_{j+k+1} - x)/(t_{j+k+1} - t_{j+1}) B_{j+1,k-1}
// (0/0 := 0), and differentiated with
//   B'_{j,k} = k [ B_{j,k-1}/(t_{j+k} - t_j) - B_{j+1,k-1}/(t_{j+k+1} - t_{j+1}) ].
// vals[(q*(p+1) + a)*3 + d] = d^d B_{first+a}(x_q).
// ---------------------------------------------------------------------------
__global__ void basis_table_kernel(const double* __restrict__ t, int p, int Q,
                                   const double* __restrict__ qx, const int* __restrict__ qfirst,
                                   double* __restrict__ vals) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const double x = qx[q];
    const int s = qfirst[q] + p;
    double N[IGAPW_MAXP + 1][IGAPW_MAXP + 1];   // N[k][a] = B_{s-k+a, k}(x)
    N[0][0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        for (int a = 0; a <= k; ++a) {
            const int j = s - k + a;
            double v = 0.0;
            if (a >= 1) {
                double den = t[j + k] - t[j];
                if (den != 0.0) v += (x - t[j]) / den * N[k - 1][a - 1];
            }
            if (a <= k - 1) {
                double den = t[j + k + 1] - t[j + 1];
                if (den != 0.0) v += (t[j + k + 1] - x) / den * N[k - 1][a];
            }
            N[k][a] = v;
        }
    }
    // first derivatives of degree p-1 functions B_{m,p-1}, m = s-p+1..s (index m-(s-p+1))
    double D1[IGAPW_MAXP + 1];
    for (int b = 0; b < p; ++b) {
        const int m = s - p + 1 + b;
        const int k = p - 1;
        double v = 0.0;
        // B_{m,k-1} has level index m - (s-k+1) = b - 1; B_{m+1,k-1} has index b
        if (b >= 1) {
            double den = t[m + k] - t[m];
            if (den != 0.0) v += k * N[k - 1][b - 1] / den;
        }
        if (b <= k - 1) {
            double den = t[m + k + 1] - t[m + 1];
            if (den != 0.0) v -= k * N[k - 1][b] / den;
        }
        D1[b] = v;
    }
    for (int a = 0; a <= p; ++a) {
        const int j = s - p + a;
        double d1 = 0.0, d2 = 0.0;
        // B_{j,p-1} = N[p-1][a-1], B_{j+1,p-1} = N[p-1][a]; same indices for D1
        if (a >= 1) {
            double den = t[j + p] - t[j];
            if (den != 0.0) { d1 += p * N[p - 1][a - 1] / den; d2 += p * D1[a - 1] / den; }
        }
        if (a <= p - 1) {
            double den = t[j + p + 1] - t[j + 1];
            if (den != 0.0) { d1 -= p * N[p - 1][a] / den; d2 -= p * D1[a] / den; }
        }
        double* o = vals + ((size_t)q * (p + 1) + a) * 3;
        o[0] = N[p][a];
        o[1] = d1;
        o[2] = d2;
    }
}

// ---------------------------------------------------------------------------
// (a2) fold.  One thread per (row i, window slot w).  With the test weight
//   tw(i,q) = w_q            (PW: point q lies in cell i; the test is 1)
//   tw(i,q) = w_q B_i(x_q)   (Galerkin)
// A[i][w] = sum_q tw(i,q) B_j(x_q), C[i][w] = sum_q tw(i,q) B_j''(x_q),
// j = fstart[i] + w, summed over the points of row i in increasing x.
// Dirichlet rows: A = identity row, C = 0.  S = A, or -C (identity on
// Dirichlet rows) for the 1D Poisson system.  TW[i][w] = tw(i, pstart[i]+w).
// ---------------------------------------------------------------------------
__global__ void fold_kernel(FoldArgs f) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nA = f.n * f.W;
    const int nT = f.n * f.WQ;
    if (tid < nA) {
        const int i = tid / f.W, w = tid % f.W;
        const int j = f.fstart[i] + w;
        double sa = 0.0, sc = 0.0;
        if (!f.is_free[i]) {
            sa = (j == i) ? 1.0 : 0.0;
        } else if (j < f.n) {
            const int q0 = f.pstart[i], q1 = q0 + f.pcount[i];
            for (int q = q0; q < q1; ++q) {
                const int first = f.qfirst[q];
                const int a = j - first;
                if (a < 0 || a > f.p) continue;
                double tw = f.qw[q];
                if (f.test == 0) {
                    const int ai = i - first;
                    tw *= (ai >= 0 && ai <= f.p) ? f.vals[((size_t)q * (f.p + 1) + ai) * 3] : 0.0;
                } else if (f.test == 2) {
                    tw = f.twr[(size_t)i * f.WQ + (q - q0)];
                }
                sa += tw * f.vals[((size_t)q * (f.p + 1) + a) * 3 + 0];
                sc += tw * f.vals[((size_t)q * (f.p + 1) + a) * 3 + 2];
            }
        }
        // Neumann axis (Sec. 4.3): the operator row is -C + E with
        // E_ij = T_i(b) B_j'(b) - T_i(a) B_j'(a); the end rows hold the tests
        // that are 1 at the ends, so C_ij -= E_ij on rows 0 and n-1
        if (f.neumann && j < f.n) {
            if (i == f.n - 1) sc -= f.dright[j];
            if (i == 0) sc += f.dleft[j];
        }
        double ss = sa;
        if (f.poisson) ss = f.is_free[i] ? -sc : sa;
        f.A[tid] = sa;
        f.C[tid] = sc;
        f.S[tid] = ss;
        float h, l;
        split_double(sa, h, l);
        f.Adf[tid] = make_float2(h, l);
        split_double(sc, h, l);
        f.Cdf[tid] = make_float2(h, l);
        split_double(ss, h, l);
        f.Sdf[tid] = make_float2(h, l);
    } else if (tid < nA + nT) {
        const int k = tid - nA;
        const int i = k / f.WQ, w = k % f.WQ;
        double tw = 0.0;
        if (f.is_free[i] && w < f.pcount[i]) {
            const int q = f.pstart[i] + w;
            tw = f.qw[q];
            if (f.test == 0) {
                const int ai = i - f.qfirst[q];
                tw *= (ai >= 0 && ai <= f.p) ? f.vals[((size_t)q * (f.p + 1) + ai) * 3] : 0.0;
            } else if (f.test == 2) {
                tw = f.twr[(size_t)i * f.WQ + w];
            }
        }
        f.TW[k] = tw;
        float h, l;
        split_double(tw, h, l);
        f.TWdf[k] = make_float2(h, l);
    }
}

// ---------------------------------------------------------------------------
// (c1) factor.  One thread per axis (the work is O(n p^2)).  The system matrix
// S (window format) is copied into a band of half-width p, factored by
// Doolittle elimination without pivoting (no fill outside the band), and the
// partitioned-solve data are derived:
//  forward  (L y = r):  chunk k, row i: y_i = y~_i - sum_c G[i][c] y_{b_k - p + c}
//           G_i = sum_{m: i-m < b_k} l_{i,m} e_{i-m-b_k+p} - sum_{m: i-m >= b_k} l_{i,m} G_{i-m}
//  backward (U x = y):  x_i = x~_i - sum_c H[i][c] x_{b_{k+1} + c}
//           H_i = dinv_i ( sum_{m: i+m >= b_{k+1}} u_{i,m} e_{i+m-b_{k+1}} - sum_{in} u_{i,m} H_{i+m} )
//  scan operators: tails t_k = a_k + F_k t_{k-1}, F_k = -G[last p rows of chunk k];
//  heads s_k = a'_k + F'_k s_{k+1}, F'_k = -H[first p rows of chunk k];
//  Hillis-Steele level l combines with the lane 2^l away:
//  Phi^{(0)} = F, Phi^{(l+1)}_k = Phi^{(l)}_k Phi^{(l)}_{k -/+ 2^l}.
// ---------------------------------------------------------------------------
__global__ void factor_kernel(FactorArgs a) {
    if (blockIdx.x * blockDim.x + threadIdx.x != 0) return;
    const int n = a.n, p = a.p, W = a.W, bw = 2 * p + 1;
    double* band = a.work;   // [n * bw], band[i*bw + (j - i + p)]
    for (int i = 0; i < n * bw; ++i) band[i] = 0.0;
    double scale = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int w = 0; w < W; ++w) {
            const int j = a.fstart[i] + w;
            const double v = a.S[i * W + w];
            if (j >= n || v == 0.0) continue;
            const int m = j - i;
            if (m < -p || m > p) { atomicOr(a.status, STATUS_SINGULAR); return; }
            band[i * bw + m + p] = v;
            scale = fmax(scale, fabs(v));
        }
    }
    for (int k = 0; k < n; ++k) {
        const double piv = band[k * bw + p];
        if (!(fabs(piv) > 1e-13 * scale)) { atomicOr(a.status, STATUS_SINGULAR); return; }
        const int iend = min(n - 1, k + p);
        for (int i = k + 1; i <= iend; ++i) {
            const double l = band[i * bw + (k - i + p)] / piv;
            band[i * bw + (k - i + p)] = l;
            if (l == 0.0) continue;
            for (int j = k + 1; j <= iend; ++j) band[i * bw + (j - i + p)] -= l * band[k * bw + (j - k + p)];
        }
    }
    for (int i = 0; i < n; ++i) {
        for (int m = 1; m <= p; ++m) {
            a.L[i * p + m - 1] = (i - m >= 0) ? band[i * bw + (p - m)] : 0.0;
            a.U[i * p + m - 1] = (i + m < n) ? band[i * bw + (p + m)] : 0.0;
        }
        a.dinv[i] = 1.0 / band[i * bw + p];
    }
    const int P = a.P;
    // forward spikes
    for (int k = 0; k < P; ++k) {
        const int b0 = a.b[k], b1 = a.b[k + 1];
        for (int i = b0; i < b1; ++i) {
            for (int c = 0; c < p; ++c) a.G[i * p + c] = 0.0;
            if (k == 0) continue;
            for (int m = 1; m <= p; ++m) {
                const double l = a.L[i * p + m - 1];
                const int j = i - m;
                if (j < b0) {
                    if (!IGAPW_IDX("factor G", j - b0 + p, p)) continue;
                    a.G[i * p + (j - b0 + p)] += l;
                } else {
                    for (int c = 0; c < p; ++c) a.G[i * p + c] -= l * a.G[j * p + c];
                }
            }
        }
    }
    // backward spikes
    for (int k = 0; k < P; ++k) {
        const int b0 = a.b[k], b1 = a.b[k + 1];
        for (int i = b1 - 1; i >= b0; --i) {
            for (int c = 0; c < p; ++c) a.H[i * p + c] = 0.0;
            if (k == P - 1) continue;
            for (int m = 1; m <= p; ++m) {
                const double u = a.U[i * p + m - 1];
                const int j = i + m;
                if (j >= b1) {
                    if (!IGAPW_IDX("factor H", j - b1, p)) continue;
                    a.H[i * p + (j - b1)] += u;
                } else {
                    for (int c = 0; c < p; ++c) a.H[i * p + c] -= u * a.H[j * p + c];
                }
            }
            for (int c = 0; c < p; ++c) a.H[i * p + c] *= a.dinv[i];
        }
    }
    // scan operators
    const int pp = p * p;
    double tmp[IGAPW_MAXP * IGAPW_MAXP];
    for (int l = 0; l < 5; ++l)
        for (int k = 0; k < 32; ++k)
            for (int e = 0; e < pp; ++e) { a.PhiF[(l * 32 + k) * pp + e] = 0.0; a.PhiB[(l * 32 + k) * pp + e] = 0.0; }
    for (int k = 0; k < P; ++k) {
        const int b0 = a.b[k], b1 = a.b[k + 1];
        if (!IGAPW_IDX("factor chunk", b1 - p, n) || !IGAPW_IDX("factor chunk lo", b0, b1 - p + 1)) continue;
        for (int r = 0; r < p; ++r)
            for (int c = 0; c < p; ++c) {
                a.PhiF[k * pp + r * p + c] = -a.G[(b1 - p + r) * p + c];
                a.PhiB[k * pp + r * p + c] = -a.H[(b0 + r) * p + c];
            }
    }
    for (int l = 0; l < 4; ++l) {
        const int d = 1 << l;
        for (int k = 0; k < P; ++k) {
            // forward: Phi^{l+1}_k = Phi^l_k Phi^l_{k-d}
            if (k - d >= 0) {
                const double* X = a.PhiF + (l * 32 + k) * pp;
                const double* Y = a.PhiF + (l * 32 + k - d) * pp;
                for (int r = 0; r < p; ++r)
                    for (int c = 0; c < p; ++c) {
                        double s = 0.0;
                        for (int m = 0; m < p; ++m) s += X[r * p + m] * Y[m * p + c];
                        tmp[r * p + c] = s;
                    }
                for (int e = 0; e < pp; ++e) a.PhiF[((l + 1) * 32 + k) * pp + e] = tmp[e];
            }
            // backward: Phi'^{l+1}_k = Phi'^l_k Phi'^l_{k+d}
            if (k + d < P) {
                const double* X = a.PhiB + (l * 32 + k) * pp;
                const double* Y = a.PhiB + (l * 32 + k + d) * pp;
                for (int r = 0; r < p; ++r)
                    for (int c = 0; c < p; ++c) {
                        double s = 0.0;
                        for (int m = 0; m < p; ++m) s += X[r * p + m] * Y[m * p + c];
                        tmp[r * p + c] = s;
                    }
                for (int e = 0; e < pp; ++e) a.PhiB[((l + 1) * 32 + k) * pp + e] = tmp[e];
            }
        }
    }
    // FP32 copies
    for (int i = 0; i < n * p; ++i) {
        a.L32[i] = (float)a.L[i];
        a.U32[i] = (float)a.U[i];
        a.G32[i] = (float)a.G[i];
        a.H32[i] = (float)a.H[i];
    }
    for (int i = 0; i < n; ++i) a.dinv32[i] = (float)a.dinv[i];
    for (int i = 0; i < 5 * 32 * pp; ++i) { a.PhiF32[i] = (float)a.PhiF[i]; a.PhiB32[i] = (float)a.PhiB[i]; }
}

void launch_chunk_tables(const ChunkTableArgs& a, cudaStream_t st) { chunk_tables_kernel<<<1, 1, 0, st>>>(a); }

void launch_basis_table(const double* t, int p, int Q, const double* qx, const int* qfirst,
                        double* vals, cudaStream_t st) {
    if (Q <= 0) return;
    basis_table_kernel<<<(Q + 127) / 128, 128, 0, st>>>(t, p, Q, qx, qfirst, vals);
}

void launch_fold(const FoldArgs& f, cudaStream_t st) {
    const int total = f.n * f.W + f.n * f.WQ;
    fold_kernel<<<(total + 127) / 128, 128, 0, st>>>(f);
}

void launch_factor(const FactorArgs& a, cudaStream_t st) { factor_kernel<<<1, 1, 0, st>>>(a); }

}  // namespace igapw
