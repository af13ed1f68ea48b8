// Host-side set-up of one axis: knots, Gauss rules, PW test cells, quadrature
// points and the banded "window" layout used by every device table.
//
// Window layout.  Row i of a 1D table couples to the W consecutive columns
// [start[i], start[i] + W); W is fixed per axis, start[] is non-decreasing and
// steps by at most one from row to row.  The same start[] serves the tested
// mass table int T_i B_j and the tested Laplacian table int T_i B_j'' (they
// share their sparsity), and the system matrix that is factored.
#pragma once
#include <string>
#include <vector>

namespace igapw {

struct AxisSetup {
    int n_elem = 0, p = 0, nq = 0, test = 0, bc = 0;
    int n = 0;                       // number of basis functions n_elem + p
    std::vector<double> knots;       // open knot vector, n + p + 1 values
    std::vector<double> brk;         // distinct break points, n_elem + 1 values

    // quadrature points in increasing x (all elements, or all PW pieces)
    std::vector<double> qx, qw;
    std::vector<int> qfirst;         // first non-zero function at each point: B_{qfirst..qfirst+p}
    std::vector<int> qrow;           // PW: row (unknown) whose cell holds the point; -1 Galerkin

    // rows: which coefficients are unknowns (Dirichlet rows are not)
    std::vector<int> is_free;        // n entries, 1 = unknown, 0 = Dirichlet row

    // point window per row: points [pstart[i], pstart[i] + pcount[i]) carry its test
    std::vector<int> pstart, pcount;
    int wq = 0;                      // max pcount (point window width)

    // function window per row (operator tables and system matrix)
    std::vector<int> fstart;
    int w = 0;                       // window width (unpadded)
    std::vector<int> flo, fhi;       // first/last non-zero column of each row

    // partitioned line solve: P chunks with bounds chunk_b[0..P]
    int P = 0;
    int chunk_b[33] = {0};

    // PW cell break points (empty for Galerkin)
    std::vector<double> cells;

    // refined test space: w_q T_i(x_q) over each row's point window, [n][wq]
    // (rows of width wq; B-spline and PW tests compute theirs on the device)
    std::vector<double> tw_refined;

    // first derivatives of every basis function at the two ends of the axis
    // (the Neumann boundary term of Sec. 4.3 uses them)
    std::vector<double> dleft, dright;
};

// Builds everything for one axis from (n_elem, p, nq, test, bc) and optional
// caller knots (empty = open uniform on [0,1]).  Returns "" or an error text.
// test: 0 B-splines, 1 PW cells, 2 refined test space (`refine` parts per
// element, Sec. 2).
std::string build_axis(AxisSetup& ax, int n_elem, int p, int nq, int test, int bc,
                       const std::vector<double>& knots_in, int refine = 0);

// Re-centres the function windows for a padded kernel width wk >= ax.w:
// fstart[i] = max(0, min(flo[i], n - wk)).  False if the starts do not step by
// 0 or 1 from row to row or a row's columns do not fit its window.
bool set_window(AxisSetup& ax, int wk);

// Chooses the chunking of the partitioned line solve for an axis whose batch
// holds `lines` independent lines (P chunks, bounds chunk_b).
void set_chunks(AxisSetup& ax, long long lines);

// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_nq.
void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w);

}  // namespace igapw
