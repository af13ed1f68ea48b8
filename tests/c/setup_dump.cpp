// Test harness: builds one axis with the library's host set-up (setup.cpp)
// and prints its quadrature points, weights, PW cells, point windows and
// refined test weights, one field per line ("name v0 v1 ..."), so the tests
// can compare them with the oracle on a machine without a GPU.
//   setup_dump n_elem p nq test bc refine [knot ...]
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "setup.h"

template <typename T>
static void put(const char* name, const std::vector<T>& v) {
    std::printf("%s", name);
    for (const T& x : v) std::printf(" %.17g", (double)x);
    std::printf("\n");
}

int main(int argc, char** argv) {
    if (argc < 7) {
        std::fprintf(stderr, "usage: setup_dump n_elem p nq test bc refine [knot ...]\n");
        return 2;
    }
    const int ne = std::atoi(argv[1]), p = std::atoi(argv[2]), nq = std::atoi(argv[3]);
    const int test = std::atoi(argv[4]), bc = std::atoi(argv[5]), refine = std::atoi(argv[6]);
    std::vector<double> knots;
    for (int i = 7; i < argc; ++i) knots.push_back(std::strtod(argv[i], nullptr));
    igapw::AxisSetup ax;
    const std::string err = igapw::build_axis(ax, ne, p, nq, test, bc, knots, refine);
    if (!err.empty()) {
        std::printf("error %s\n", err.c_str());
        return 0;
    }
    std::printf("n %d\nwq %d\nP %d\n", ax.n, ax.wq, ax.P);
    put("knots", ax.knots);
    put("qx", ax.qx);
    put("qw", ax.qw);
    put("qrow", ax.qrow);
    put("is_free", ax.is_free);
    put("pstart", ax.pstart);
    put("pcount", ax.pcount);
    put("cells", ax.cells);
    put("tw_refined", ax.tw_refined);
    put("dleft", ax.dleft);
    put("dright", ax.dright);
    return 0;
}
