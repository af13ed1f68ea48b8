// Host-side set-up of one axis (knots, Gauss rule, PW cells, quadrature points,
// banded windows).  O(n) work; everything heavier runs on the device.
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace igapw {

static void legendre(int nq, double t, double& pn, double& pn1) {
    // P_nq(t) and P_{nq-1}(t) by (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}
    double p0 = 1.0, p1 = t;
    if (nq == 0) { pn = 1.0; pn1 = 0.0; return; }
    for (int k = 1; k < nq; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    pn = p1;
    pn1 = p0;
}

void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w) {
    // Newton iteration on P_nq; P'_nq(t) = nq (t P_nq - P_{nq-1}) / (t^2 - 1);
    // weights 2 / ((1 - t^2) P'_nq(t)^2).  Start: t_i ~ cos(pi (i + 3/4) / (nq + 1/2)).
    x.assign(nq, 0.0);
    w.assign(nq, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < nq; ++i) {
        double t = std::cos(pi * (i + 0.75) / (nq + 0.5));
        double pn, pn1, dp;
        for (int it = 0; it < 100; ++it) {
            legendre(nq, t, pn, pn1);
            dp = nq * (t * pn - pn1) / (t * t - 1.0);
            double step = pn / dp;
            t -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        legendre(nq, t, pn, pn1);
        dp = nq * (t * pn - pn1) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
    std::vector<int> idx(nq);
    for (int i = 0; i < nq; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int l, int r) { return x[l] < x[r]; });
    std::vector<double> xs(nq), ws(nq);
    for (int i = 0; i < nq; ++i) { xs[i] = x[idx[i]]; ws[i] = w[idx[i]]; }
    x.swap(xs);
    w.swap(ws);
}

static std::string fmt(const char* f, int a, int b = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

// Values of the k+1 degree-k B-splines that are non-zero on knot span s
// (t[s] <= x <= t[s+1]) at x: N[r] = B_{s-k+r,k}(x), r = 0..k (the standard
// triangular Cox--de Boor evaluation).
static void span_values(const std::vector<double>& t, int s, int k, double x, double* N) {
    double left[8], right[8];
    N[0] = 1.0;
    for (int j = 1; j <= k; ++j) {
        left[j] = x - t[s + 1 - j];
        right[j] = t[s + j] - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            const double den = right[r + 1] + left[j - r];
            const double tmp = den != 0.0 ? N[r] / den : 0.0;
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
    }
}

// B_j'(x) for all j at an end of the axis: B'_{j,p} = p (B_{j,p-1} / (t_{j+p} - t_j)
// - B_{j+1,p-1} / (t_{j+p+1} - t_{j+1})) with the degree p-1 values of span s.
static void end_derivs(const AxisSetup& ax, int s, double x, std::vector<double>& d) {
    const int p = ax.p, n = ax.n;
    const std::vector<double>& t = ax.knots;
    double N[8];
    span_values(t, s, p - 1, x, N);
    auto lower = [&](int j) {   // B_{j,p-1}(x)
        const int r = j - (s - (p - 1));
        return (r >= 0 && r <= p - 1) ? N[r] : 0.0;
    };
    d.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        double v = 0.0;
        const double d1 = t[j + p] - t[j], d2 = t[j + p + 1] - t[j + 1];
        if (d1 > 0.0) v += lower(j) / d1;
        if (d2 > 0.0) v -= lower(j + 1) / d2;
        d[j] = p * v;
    }
}

std::string build_axis(AxisSetup& ax, int n_elem, int p, int nq, int test, int bc,
                       const std::vector<double>& knots_in, int refine) {
    ax = AxisSetup();
    if (p < 2 || p > 4) return fmt("degree %d unsupported (2..4: C^1 or smoother)", p);
    if (n_elem < 1) return fmt("n_elem %d < 1", n_elem);
    if (nq < 1 || nq > 16) return fmt("nq %d out of range 1..16", nq);
    if (test != 0 && test != 1 && test != 2) return fmt("test %d unknown", test);
    if (test == 2 && (refine < 2 || refine > 64)) return fmt("refine %d out of range 2..64", refine);
    if (bc != 0 && bc != 1) return fmt("bc %d unknown", bc);
    ax.n_elem = n_elem; ax.p = p; ax.nq = nq; ax.test = test; ax.bc = bc;
    ax.n = n_elem + p;
    const int n = ax.n;
    const int nk = n + p + 1;

    // ---- knots (Sec. 2: open knot vector, n = N_e + p functions) ---------
    if (knots_in.empty()) {
        ax.knots.assign(nk, 0.0);
        for (int k = 0; k < nk; ++k) {
            int i = k - p;
            ax.knots[k] = i <= 0 ? 0.0 : (i >= n_elem ? 1.0 : (double)i / n_elem);
        }
    } else {
        if ((int)knots_in.size() != nk)
            return fmt("knot vector length %d, expected %d", (int)knots_in.size(), nk);
        ax.knots = knots_in;
        for (int k = 1; k < nk; ++k)
            if (!(ax.knots[k] >= ax.knots[k - 1])) return "knot vector not non-decreasing";
        for (int k = 1; k <= p; ++k)
            if (ax.knots[k] != ax.knots[0] || ax.knots[nk - 1 - k] != ax.knots[nk - 1])
                return "knot vector must repeat each end point p+1 times";
        if (!(ax.knots[nk - 1] > ax.knots[0])) return "empty knot interval";
        int mult = 0;
        for (int k = p + 1; k < nk - p - 1; ++k) {
            mult = (k > p + 1 && ax.knots[k] == ax.knots[k - 1]) ? mult + 1 : 1;
            if (mult > p - 1) return "interior knot multiplicity > p-1 breaks C^1 continuity";
            if (ax.knots[k] == ax.knots[0] || ax.knots[k] == ax.knots[nk - 1])
                return "interior knot equals an end point";
        }
    }
    const double a = ax.knots[0], b = ax.knots[nk - 1];
    const double tol = 1e-12 * (b - a);
    ax.brk.clear();
    for (int k = 0; k < nk; ++k)
        if (ax.brk.empty() || ax.knots[k] > ax.brk.back()) ax.brk.push_back(ax.knots[k]);
    const int ne = (int)ax.brk.size() - 1;

    // first non-zero function on element e: s - p with t_s <= brk[e] < t_{s+1}
    std::vector<int> efirst(ne);
    for (int e = 0; e < ne; ++e) {
        int s = 0;
        for (int k = 0; k < nk - 1; ++k)
            if (ax.knots[k] <= ax.brk[e] && ax.knots[k + 1] > ax.brk[e]) s = k;
        efirst[e] = s - p;
    }
    auto element_of = [&](double x) {
        int e = (int)(std::upper_bound(ax.brk.begin(), ax.brk.end(), x) - ax.brk.begin()) - 1;
        return std::min(std::max(e, 0), ne - 1);
    };

    // ---- unknowns (Sec. 4.3: Dirichlet rows are replaced) -----------------
    ax.is_free.assign(n, 1);
    if (bc == 1) { ax.is_free[0] = 0; ax.is_free[n - 1] = 0; }
    std::vector<int> unk;
    for (int i = 0; i < n; ++i) if (ax.is_free[i]) unk.push_back(i);
    if (unk.empty()) return "no unknowns on an axis";

    std::vector<double> gx, gw;
    gauss_legendre(nq, gx, gw);
    auto add_piece = [&](double lo, double hi, int row) {
        double jac = 0.5 * (hi - lo);
        int e = element_of(0.5 * (lo + hi));
        for (int q = 0; q < nq; ++q) {
            ax.qx.push_back(lo + jac * (gx[q] + 1.0));
            ax.qw.push_back(jac * gw[q]);
            ax.qfirst.push_back(efirst[e]);
            ax.qrow.push_back(row);
        }
    };

    ax.pstart.assign(n, 0);
    ax.pcount.assign(n, 0);
    // PW cells (also the groups of the refined test space): midpoints of
    // consecutive Greville abscissae of the unknowns, domain ends outside
    auto make_cells = [&]() -> std::string {
        std::vector<double> xi(n);
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = j + 1; k <= j + p; ++k) s += ax.knots[k];
            xi[j] = s / p;
        }
        ax.cells.push_back(a);
        for (size_t k = 0; k + 1 < unk.size(); ++k) {
            double c = 0.5 * (xi[unk[k]] + xi[unk[k + 1]]);
            for (double kn : ax.brk)
                if (std::fabs(kn - c) < tol) c = kn;   // snap a knot-coincident midpoint
            ax.cells.push_back(c);
        }
        ax.cells.push_back(b);
        for (size_t k = 0; k + 1 < ax.cells.size(); ++k)
            if (!(ax.cells[k + 1] > ax.cells[k])) return "degenerate PW cell";
        return "";
    };
    if (test == 1) {
        std::string err = make_cells();
        if (!err.empty()) return err;
        for (size_t k = 0; k < unk.size(); ++k) {
            int row = unk[k];
            double lo = ax.cells[k], hi = ax.cells[k + 1];
            ax.pstart[row] = (int)ax.qx.size();
            double cur = lo;
            for (double kn : ax.brk) {
                if (kn > lo && kn < hi) { add_piece(cur, kn, row); cur = kn; }
            }
            add_piece(cur, hi, row);
            ax.pcount[row] = (int)ax.qx.size() - ax.pstart[row];
        }
    } else if (test == 2) {
        // ---- refined test space (Sec. 2): every element split into `refine`
        // parts; test k = sum of the refined B-splines whose Greville abscissa
        // lies in PW cell k (a contiguous range J_k = [mlo, mhi])
        std::string err = make_cells();
        if (!err.empty()) return err;
        std::vector<double> tr(p, a);
        for (int e = 0; e < ne; ++e)
            for (int k = 0; k < refine; ++k) tr.push_back(ax.brk[e] + (ax.brk[e + 1] - ax.brk[e]) * k / refine);
        for (int k = 0; k <= p; ++k) tr.push_back(b);
        const int nr = (int)tr.size() - p - 1;     // refined functions
        const int ner = ne * refine;               // refined elements
        std::vector<int> mlo(unk.size(), nr), mhi(unk.size(), -1);
        for (int m = 0; m < nr; ++m) {
            double g = 0.0;
            for (int k = m + 1; k <= m + p; ++k) g += tr[k];
            g /= p;
            size_t k = 0;
            while (k + 1 < unk.size() && !(g < ax.cells[k + 1])) ++k;   // cell k: [c_k, c_{k+1}), last closed
            mlo[k] = std::min(mlo[k], m);
            mhi[k] = std::max(mhi[k], m);
        }
        std::vector<int> er_first_pt(ner);
        for (int er = 0; er < ner; ++er) {
            er_first_pt[er] = (int)ax.qx.size();
            add_piece(tr[p + er], tr[p + er + 1], -1);
        }
        // test values at the points of each row's support
        std::vector<std::vector<double>> rowvals(n);
        for (size_t k = 0; k < unk.size(); ++k) {
            const int row = unk[k];
            if (mhi[k] < mlo[k]) return "refined test without functions (refine too small)";
            const int e0 = std::max(0, mlo[k] - p), e1 = std::min(ner - 1, mhi[k]);
            ax.pstart[row] = er_first_pt[e0];
            ax.pcount[row] = (e1 - e0 + 1) * nq;
            for (int er = e0; er <= e1; ++er) {
                for (int q = 0; q < nq; ++q) {
                    const int pt = er_first_pt[er] + q;
                    double N[8];
                    span_values(tr, p + er, p, ax.qx[pt], N);
                    double t = 0.0;
                    for (int r = 0; r <= p; ++r)
                        if (er + r >= mlo[k] && er + r <= mhi[k]) t += N[r];
                    rowvals[row].push_back(ax.qw[pt] * t);
                }
            }
        }
        int wq = 0;
        for (int i = 0; i < n; ++i) wq = std::max(wq, ax.pcount[i]);
        ax.tw_refined.assign((size_t)n * std::max(wq, 1), 0.0);
        for (int i = 0; i < n; ++i)
            for (size_t c = 0; c < rowvals[i].size(); ++c) ax.tw_refined[(size_t)i * wq + c] = rowvals[i][c];
    } else {
        // ---- Galerkin: nq Gauss points per element -------------------------
        std::vector<int> efirst_pt(ne);
        for (int e = 0; e < ne; ++e) {
            efirst_pt[e] = (int)ax.qx.size();
            add_piece(ax.brk[e], ax.brk[e + 1], -1);
        }
        for (int i = 0; i < n; ++i) {
            if (!ax.is_free[i]) continue;
            // elements where B_i is non-zero: efirst[e] <= i <= efirst[e] + p
            int e0 = -1, e1 = -1;
            for (int e = 0; e < ne; ++e)
                if (efirst[e] <= i && i <= efirst[e] + p) { if (e0 < 0) e0 = e; e1 = e; }
            if (e0 < 0) return "basis function without support";
            ax.pstart[i] = efirst_pt[e0];
            ax.pcount[i] = (e1 - e0 + 1) * nq;
        }
    }
    ax.wq = 0;
    for (int i = 0; i < n; ++i) ax.wq = std::max(ax.wq, ax.pcount[i]);

    // ---- function windows -----------------------------------------------
    std::vector<int> lo(n), hi(n);
    for (int i = 0; i < n; ++i) {
        if (!ax.is_free[i]) { lo[i] = hi[i] = i; continue; }
        lo[i] = n; hi[i] = -1;
        for (int q = ax.pstart[i]; q < ax.pstart[i] + ax.pcount[i]; ++q) {
            lo[i] = std::min(lo[i], ax.qfirst[q]);
            hi[i] = std::max(hi[i], ax.qfirst[q] + p);
        }
    }
    ax.w = 0;
    for (int i = 0; i < n; ++i) ax.w = std::max(ax.w, hi[i] - lo[i] + 1);
    ax.flo = lo;
    ax.fhi = hi;
    for (int i = 0; i < n; ++i) {
        // the band of the factored system must stay within +-p of the diagonal
        if (hi[i] - i > p || i - lo[i] > p) return "row couples beyond the +-p band";
    }
    if (ax.w > 2 * p + 1) return "window wider than 2p+1";
    // the narrowest window width the kernels are built for (3, 5, 7 or 9)
    const int wpad = ax.w <= 3 ? 3 : ax.w <= 5 ? 5 : ax.w <= 7 ? 7 : 9;
    if (ax.w > 9 || !set_window(ax, wpad))
        return "knot vector too irregular for the banded layout (row windows must step by 0 or 1 within a "
               "window of 9 columns)";

    // ---- chunks of the partitioned line solve: P <= 32, length >= p -------
    set_chunks(ax, 1);
    // end derivatives: left end on the first non-empty span (s = p), right end
    // on the last (s = n - 1), evaluated at the end point itself
    end_derivs(ax, p, ax.knots[0], ax.dleft);
    end_derivs(ax, n - 1, ax.knots[n + p], ax.dright);
    return "";
}

void set_chunks(AxisSetup& ax, long long lines) {
    // P a power of two <= 32 (the lane group of a warp that shares a line):
    // the smallest P whose chunks fit the register-resident solve
    // (ceil(n / P) <= 20 rows), never with chunks shorter than p rows.  The
    // split step solves the few lines a block holds, so one lane per whole line
    // (P = 1) would leave most of its threads idle in the solve phases however
    // many lines the batch has (`lines` is kept for the interface).
    (void)lines;
    const int n = ax.n, p = ax.p;
    ax.P = 1;
    while (ax.P < 32 && (n + ax.P - 1) / ax.P > 20 && n / (2 * ax.P) >= p) ax.P *= 2;
    for (int k = 0; k <= ax.P; ++k) ax.chunk_b[k] = (int)((long long)k * n / ax.P);
}

bool set_window(AxisSetup& ax, int wk) {
    // Row i's window [fstart[i], fstart[i] + wk) must hold its non-zero
    // columns [flo[i], fhi[i]], and consecutive windows step by 0 or 1 (the
    // staged kernels load the union of a block's row windows).  Where the
    // padded width leaves room, a window may start below its row's first
    // non-zero column: each row takes the highest start the previous row
    // allows, which keeps the most room for the rows after it.
    ax.fstart.assign(ax.n, 0);
    for (int i = 0; i < ax.n; ++i) {
        int hi = std::min(ax.flo[i], std::max(0, ax.n - wk));   // a window wider than the axis starts at 0
        int lo = std::max(0, ax.fhi[i] - wk + 1);
        if (i > 0) {
            hi = std::min(hi, ax.fstart[i - 1] + 1);
            lo = std::max(lo, ax.fstart[i - 1]);
        }
        if (hi < lo) return false;
        ax.fstart[i] = hi;
    }
    return true;
}

}  // namespace igapw
