// Host check of the tensor-core GEMM's launch planner (csrc/tcgemm.cuh:
// tc_plan, tc_makespan, the split workspace sizes), compiled for the CPU.
// Reads lines "M N K batch sms fixed_bn allow_split" from stdin and prints,
// per line, "bn splits kb0 kb1 kb2 kb3 kb4 makespan ws_floats counters
// tiles per_chunk block_overhead split_overhead".
#include "cuda_emu.h"

#include <cstdio>

#include "../../paper_1910_08535_gb300/csrc/tcgemm.cuh"

int main() {
    int M, N, K, batch, sms, fixed_bn, allow;
    while (std::scanf("%d %d %d %d %d %d %d", &M, &N, &K, &batch, &sms, &fixed_bn, &allow) == 7) {
        igapw::TcGemmArgs g{};
        g.M = M;
        g.N = N;
        g.K = K;
        g.batch = batch;
        const igapw::TcPlan p = igapw::tc_plan(g, sms, fixed_bn, allow != 0);
        const double t = igapw::tc_makespan(igapw::tc_tiles(g, p.bn), p.splits, p.kb,
                                            igapw::tc_cost(1, p.bn, 1, 1), sms);
        std::printf("%d %d %d %d %d %d %d %.6f %lld %lld %lld %.6f %.6f %.6f\n", p.bn, p.splits, p.kb[0], p.kb[1],
                    p.kb[2], p.kb[3], p.kb[4], t, igapw::tc_split_ws_floats(g, p), igapw::tc_split_counters(g, p),
                    igapw::tc_tiles(g, p.bn), igapw::tc_cost(1, p.bn, 1, 1), igapw::kTcBlockOverhead,
                    igapw::kTcSplitOverhead);
    }
    return 0;
}
