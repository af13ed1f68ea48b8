#pragma once
// FP32-accurate dense GEMM on the 5th-generation tensor cores (tcgen05,
// sm_100a / sm_103a) for the fast-diagonalisation transforms of the 2D/3D
// Poisson solve:  D(m, n) = sum_k A(m, k) B(n, k)  with arbitrary strides.
//
// Precision: split TF32 ("3xTF32").  Each FP32 operand x is split into two
// TF32 values, x_hi = x rounded to TF32 and x_lo = (x - x_hi) rounded to TF32
// (|x_lo| <= 2^-11 |x|, x_hi + x_lo within 2^-23 |x| of x), and D
// accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 in tensor memory.
// The dropped A_lo B_lo term (<= 2^-22 |a b|) and the split remainders leave
// a relative error of about 2^-21 per product, a few units of FP32 rounding;
// the Poisson solve's refinement with a double-float residual removes it.
//
// Work layout.  One CTA computes a BM x BN tile of D (BM = 128: the tensor
// memory lanes; BN = 64, 96 or 128 columns, chosen per launch by a cost
// model).  K is walked in chunks of 32 through 2-4 shared-memory stages
// in a producer/consumer pipeline:
//   - warps 0-7 ("loaders") read the chunk of a live operand from global
//     memory (each warp its own rows, coalesced along whichever of the rows or
//     K has unit stride), split it into hi and lo parts and store them in the
//     canonical K-major layout without swizzle (8-row x 16-byte core matrices,
//     spaced so that the stores are free of bank conflicts);
//   - an operand that is a constant matrix (the transforms' eigenvector
//     matrices) can be split once, ahead of time, into exactly that layout
//     (tc_presplit); warp 9 then streams its chunks with bulk asynchronous
//     copies (cp.async.bulk) that complete on a per-stage mbarrier, and the
//     loaders handle the other operand only; given a tensor map of that live
//     operand, warp 9 also brings its raw FP32 chunk into the stage by TMA
//     (cp.async.bulk.tensor) and the loaders split it from shared memory;
//   - warp 8 waits until the stage is complete (the loaders' `full` barrier
//     and the copy's), issues the chunk's 8 MMAs (4 K-steps, each
//     A_hi [B_hi; B_lo] with N = 2 BN into adjacent accumulators and A_lo
//     B_hi with N = BN) and commits them to the stage's `empty` mbarrier, which the loaders and
//     warp 9 wait on before they refill the stage; the MMAs of a group of
//     two chunks write fresh partial sums into one of two tensor-memory
//     buffers;
//   - the loaders add each group's partial sums (tcgen05.ld, one row per
//     thread, half the columns per warp) into FP32 registers, which frees
//     the buffer for the group after next, and finally store D.
// When the tiles alone would leave SMs idle, the host plan (tc_plan) splits
// the K chunks of every tile over up to 4 CTAs; each writes its partial tile
// to a workspace and the last to finish adds them in split order (no CTA
// waits on another).
// Summing the groups in registers matters for accuracy: the tensor core
// truncates when it accumulates (measured: a drift toward zero of about
// 2^-25 per accumulation step), which over all of K would cost the solver's
// one-step refinement two orders of magnitude in backward error.  Every wait is bounded: on a timeout the kernel
// records STATUS_TC_TIMEOUT in the status word, lets its MMAs drain, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <vector>

#include "common.cuh"

namespace igapw {

struct TcGemmArgs {
    int M, N, K;                  // D is M x N
    int batch;                    // independent GEMMs (grid z)
    const float* A;               // A(m, k) = A[bA * b + m * sAm + k * sAk]
    long long sAm, sAk, bA;
    const float* B;               // B(n, k) = B[bB * b + n * sBn + k * sBk]
    long long sBn, sBk, bB;
    float* D;                     // D(m, n) = D[bD * b + m * sDm + n * sDn]
    long long sDm, sDn, bD;
    unsigned* status;             // timeout flag (may be null)
    // pre = 1: A points to tc_presplit tiles of A (rows M, tile rows BM);
    // pre = 2: B points to tc_presplit tiles of B (rows N, tile rows bn).
    // The strides of a pre-split operand are unused; its batch stride (bA /
    // bB, in floats of the tile buffer) may be 0 (one matrix for all).
    int pre;
    int bn;                       // tile width (0: chosen at launch; required with pre = 2)
    // With a pre-split operand: a tensor map (device memory, 64-byte aligned)
    // of the other, live operand made by tc_make_tmap for tiles of tmap_rows
    // rows; its chunks then arrive by TMA instead of per-thread loads.  The
    // kernel uses it only when tmap_rows is its live tile's row count (BN
    // for a live B, 128 for a live A).  Null: per-thread loads.
    const CUtensorMap* tmap;
    int tmap_rows;
    // Split of K over several CTAs per tile (splits <= 1: none; at most
    // kTcMaxSplits; single launches only, not grouped ones).  CTA z =
    // s * batch + b sums the K chunks kb[s] .. kb[s+1]-1 (kb[0] = 0,
    // kb[splits] = ceil(K / 32), every range non-empty) of tile (m, n, b) and
    // writes the FP32 partial tile to ws (splits x tiles x 128 x bn floats);
    // the last of the tile's CTAs to finish (counted in cnt[tile], zero before
    // the launch and again after it) adds the partials in split order, so the
    // result does not depend on which CTA finishes last, and stores D.
    int splits;
    int kb[5];
    float* ws;
    unsigned* cnt;
};
constexpr int kTcMaxSplits = 4;

namespace tc {
constexpr int BM = 128;
constexpr int BK = 32;
}  // namespace tc

// ---- shared-memory operand tiles ---------------------------------------------
// An R-row tile of BK = 32 K values (hi or lo part) in the canonical K-major
// layout without swizzle: the core matrix (k group kq, row group rg) at
// kq * LBO + rg * SBO bytes, row r & 7 of it at 16 (r & 7).  SBO = 144 and
// LBO = R/8 * 144 + 16 (not the dense 128 and R * 16): with these spacings
// the 8 core matrices of one row lie in 8 different bank groups, and so do
// the 8 rows r & 7 across the row groups, so a row written as 8 x 16 bytes,
// or one K column of 32 rows written as 32 x 4 bytes, is conflict-free.
constexpr unsigned kTcSbo = 144u;
__host__ __device__ constexpr unsigned tc_lbo(int rows) { return (unsigned)(rows / 8) * kTcSbo + 16u; }
__host__ __device__ constexpr unsigned tc_tile_bytes(int rows) { return 8u * tc_lbo(rows); }
__host__ __device__ constexpr unsigned tc_tile_offset(int rows, int r, int k) {
    return (unsigned)(k >> 2) * tc_lbo(rows) + (unsigned)(r >> 3) * kTcSbo + (unsigned)(r & 7) * 16u +
           (unsigned)(k & 3) * 4u;
}
// Rows of the live operand's raw tile (the operand that is not pre-split;
// both live: no raw tile, the loaders read global memory themselves).
template <int BN, int PRE>
__host__ __device__ constexpr int tc_raw_rows() { return PRE == 1 ? BN : PRE == 2 ? tc::BM : 0; }
// A stage: the hi and lo tiles of A, one tile of 2 BN rows holding B's hi
// rows then its lo rows (so that one MMA with N = 2 BN takes A_hi B_hi and
// A_hi B_lo together), then the live operand's raw FP32 chunk as TMA writes
// it (rows x 32 floats, or 32 x rows).
template <int BN, int PRE>
__host__ __device__ constexpr unsigned tc_stage_bytes() {
    return 2u * tc_tile_bytes(tc::BM) + tc_tile_bytes(2 * BN) + (unsigned)tc_raw_rows<BN, PRE>() * tc::BK * 4u;
}

// Tensor-memory columns allocated for the accumulators of a BN-wide tile:
// two chunk buffers x (hi x hi, cross terms) x BN columns, as a power of two
// (at most the 512 columns of an SM).
__host__ __device__ constexpr unsigned tmem_cols(int bn) { return 4 * bn <= 256 ? 256u : 512u; }

// K chunks in flight through shared memory: as many stages as fit in 227 KB
// next to the barriers (at most 4).
template <int BN, int PRE>
__host__ __device__ constexpr int tc_stages() {
    const int fit = (int)((227u * 1024u - 256u) / tc_stage_bytes<BN, PRE>());
    return fit < 4 ? fit : 4;
}

// Shared memory of one CTA: the stages, then the mbarriers (full, empty and
// bulk-copy per stage, two chunk-accumulator pairs, done), the
// tensor-memory address and the abort flag (256 bytes).
template <int BN, int PRE>
__host__ __device__ constexpr size_t tc_smem_bytes() {
    return (size_t)tc_stages<BN, PRE>() * tc_stage_bytes<BN, PRE>() + 256;
}

// Bytes of one block of a pre-split operand with tiles of R rows: the hi
// tile then the lo tile (an A operand), or one tile of 2 R rows with the hi
// rows first (a B operand, `comb`), the layouts of a stage.
__host__ __device__ constexpr unsigned tc_presplit_block_bytes(int R, bool comb) {
    return comb ? tc_tile_bytes(2 * R) : 2u * tc_tile_bytes(R);
}

// Floats of the pre-split form of a rows x K operand with tiles of R rows:
// ceil(rows / R) x ceil(K / 32) blocks.
inline long long tc_presplit_floats(int rows, int K, int R, bool comb) {
    return (long long)((rows + R - 1) / R) * ((K + tc::BK - 1) / tc::BK) * (tc_presplit_block_bytes(R, comb) / 4);
}

// ---- launch planning (host code) ----------------------------------------------
// Tile widths the kernels are built for (multiples of 32: the loaders read
// 16 columns per tensor-memory load, per half of the warps; at most 128: the
// four accumulator halves fill the 512 tensor-memory columns of an SM).
constexpr int kTcWidths[3] = {64, 96, 128};

// Estimated time (arbitrary units) of tiles of width bn over `sms` SMs: the
// split-TF32 MMAs with N <= 256 are bound by shared-memory bandwidth (about
// 128 bytes per clock on an SM), so a K chunk of one tile costs its shared
// traffic: per K step the two MMAs read A_hi and A_lo (BM x 8 each) and B
// (2 bn x 8 and bn x 8) 4-byte values, and the hi and lo parts of both
// operands are written once.  Tiles are
// spread over the SMs, so the busiest SM holds ceil(tiles / sms) of them.
inline double tc_cost(long long tiles, int bn, long long chunks, int sms) {
    const double per_chunk = (4.0 * (2 * tc::BM + 3 * bn) * 8 * 4 + 2.0 * (tc::BM + bn) * tc::BK * 4) / 128.0;
    return (double)((tiles + sms - 1) / sms) * per_chunk * (double)chunks;
}

inline long long tc_tiles(const TcGemmArgs& g, int bn) {
    return (long long)((g.M + tc::BM - 1) / tc::BM) * ((g.N + bn - 1) / bn) * g.batch;
}

// Tile width of the fastest estimated cover of a set of GEMMs (one launch).
inline int tc_pick_width(const TcGemmArgs* gs, int count, int sms) {
    int best = 64;
    double best_t = 1e300;
    for (int bn : kTcWidths) {
        long long tiles = 0, chunks = 0;
        for (int i = 0; i < count; ++i) {
            tiles += tc_tiles(gs[i], bn);
            chunks = std::max<long long>(chunks, (gs[i].K + tc::BK - 1) / tc::BK);
        }
        const double t = tc_cost(tiles, bn, chunks, sms);
        if (t < best_t * 0.999) { best_t = t; best = bn; }
    }
    return best;
}

// A split of K for one launch: tile width, number of splits and the chunk
// boundaries kb[0] = 0 < kb[1] < ... < kb[splits] = ceil(K / 32).
struct TcPlan {
    int bn = 64;
    int splits = 1;
    int kb[5] = {0, 0, 0, 0, 0};
};

// Start-up and end of a CTA (barrier and tensor-memory set-up, filling the
// pipeline, draining the last chunk groups, storing the tile), and the extra
// end of a CTA of a split product (its partial tile out, the partials in),
// in K chunks of pipeline time: a CTA's first MMA comes about two chunk
// intervals after it starts.
constexpr double kTcBlockOverhead = 3.0, kTcSplitOverhead = 0.75;

// Estimated time of `tiles` tiles whose K chunks are split at kb: the CTAs
// start in launch order (every tile of split 0, then of split 1, ...), each on
// the first SM to free up, and a CTA costs its chunks plus the overheads.
inline double tc_makespan(long long tiles, int splits, const int* kb, double per_chunk, int sms) {
    const double extra = kTcBlockOverhead + (splits > 1 ? kTcSplitOverhead : 0.0);
    if (splits == 1) return (double)((tiles + sms - 1) / sms) * per_chunk * (kb[1] + extra);
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    const long long n = std::min<long long>(sms, tiles * splits);
    for (long long i = 0; i < n; ++i) free_at.push(0.0);
    double end = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
        const double cost = per_chunk * ((kb[sp + 1] - kb[sp]) + extra);
        for (long long t = 0; t < tiles; ++t) {
            const double t0 = free_at.top();
            free_at.pop();
            free_at.push(t0 + cost);
            end = std::max(end, t0 + cost);
        }
    }
    return end;
}

// Fastest estimated tile width and split of K for one GEMM on `sms` SMs
// (bn fixed when a pre-split B operand was tiled for it; splits only with
// allow_split: the caller then provides the workspace and counters).  A
// split is taken only when it is estimated 5% faster than none.
inline TcPlan tc_plan(const TcGemmArgs& g, int sms, int fixed_bn, bool allow_split) {
    const int nkc = (g.K + tc::BK - 1) / tc::BK;
    TcPlan best;
    double best_t = 1e300;
    for (int bn : kTcWidths) {
        if (fixed_bn && bn != fixed_bn) continue;
        const long long tiles = tc_tiles(g, bn);
        const double per_chunk = tc_cost(1, bn, 1, 1);
        // candidate boundaries: no split; two parts (the first the larger, so
        // that the second parts fill the SMs the first leaves idle); three
        // and four equal parts
        std::vector<std::vector<int>> cands;
        cands.push_back({0, nkc});
        if (allow_split && tiles < 2LL * sms) {
            for (int f : {50, 60, 67, 75, 80}) {
                const int c1 = (nkc * f + 50) / 100;
                if (c1 >= 1 && c1 < nkc) cands.push_back({0, c1, nkc});
            }
            for (int S = 3; S <= kTcMaxSplits; ++S) {
                if (nkc < 2 * S) break;
                std::vector<int> kb(S + 1);
                for (int i = 0; i <= S; ++i) kb[i] = (int)((long long)nkc * i / S);
                cands.push_back(kb);
            }
        }
        for (const std::vector<int>& kb : cands) {
            const int S = (int)kb.size() - 1;
            const double t = tc_makespan(tiles, S, kb.data(), per_chunk, sms) * (S > 1 ? 1.05 : 1.0);
            if (t < best_t * 0.999) {
                best_t = t;
                best.bn = bn;
                best.splits = S;
                for (int i = 0; i < 5; ++i) best.kb[i] = i <= S ? kb[i] : nkc;
            }
        }
    }
    return best;
}

// Floats of the workspace and counters of a split plan for GEMM g.
inline long long tc_split_ws_floats(const TcGemmArgs& g, const TcPlan& p) {
    return p.splits > 1 ? (long long)p.splits * tc_tiles(g, p.bn) * tc::BM * p.bn : 0;
}
inline long long tc_split_counters(const TcGemmArgs& g, const TcPlan& p) {
    return p.splits > 1 ? tc_tiles(g, p.bn) : 0;
}

// Sets g's tile width and split from plan p (workspace ws and zeroed
// counters cnt sized by tc_split_ws_floats and tc_split_counters).
inline void tc_apply_plan(TcGemmArgs& g, const TcPlan& p, float* ws, unsigned* cnt) {
    g.bn = p.bn;
    g.splits = p.splits > 1 ? p.splits : 0;
    for (int i = 0; i < 5; ++i) g.kb[i] = p.kb[i];
    g.ws = p.splits > 1 ? ws : nullptr;
    g.cnt = p.splits > 1 ? cnt : nullptr;
}

#ifndef IGAPW_HOST_EMU
namespace tc {

constexpr unsigned kSpinLimit = 1u << 26;   // mbarrier polls before giving up
#ifndef TC_GROUP
#define TC_GROUP 2
#endif
constexpr int kGroup = TC_GROUP;             // K chunks summed in tensor memory before the register sum
#ifndef TC_PREFETCH
#define TC_PREFETCH 1                         // K chunks whose loads are in flight in registers
#endif
constexpr int kLoadWarps = 8;                // warps 0-7 load and split; 8 issues the MMAs; 9 streams pre-split tiles
constexpr int kThreads = 32 * (kLoadWarps + 2);
// (10 warps: three share one of the SM's four register-file quarters of 16K
// registers, so a thread gets at most 168)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Non-blocking test of the phase (cheaper than a try_wait on a phase that
// completed long ago)
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the mbarrier phase `parity` to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    for (unsigned it = 0; it < kSpinLimit; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Bounded wait that also gives up when another warp has aborted; false on
// timeout or abort (a timeout raises the abort flag).
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned long long* bar, unsigned parity, volatile int* abort_flag) {
    if (mbar_test(bar, parity)) return true;
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

// arrive and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// bulk asynchronous copy global -> shared (16-byte aligned, size a multiple
// of 16), completing `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// TMA tile load (3D tensor map in global memory) into shared memory,
// completing its bytes on the mbarrier; the innermost coordinate must be a
// multiple of 4 floats (16 bytes).
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): canonical K-major layout without
// swizzle; start address, leading-dimension byte offset (K direction) and
// stride byte offset (M/N direction), all in 16-byte units; descriptor
// version 1 (bits 46-47); layout type 0 = no swizzle (bits 61-63).
__device__ __forceinline__ unsigned long long smem_desc(const void* p, unsigned lbo, unsigned sbo) {
    unsigned long long d = 0;
    d |= (unsigned long long)((smem_u32(p) & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor: kind::tf32, D in FP32, A and B TF32 and K-major,
// M = 128, N = BN.
template <int BN>
__device__ __forceinline__ unsigned instr_desc() {
    unsigned d = 0;
    d |= 1u << 4;                 // D format: F32
    d |= 2u << 7;                 // A format: TF32
    d |= 2u << 10;                // B format: TF32
    d |= (unsigned)(BN >> 3) << 17;
    d |= (unsigned)(BM >> 4) << 24;
    return d;
}

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// x = x_hi + x_lo + e: x_hi is x rounded to TF32 (10 fraction bits, ties
// away from zero, by adding half of the dropped range to the bit pattern
// before clearing it), so |x_lo| <= 2^-11 |x| and x - x_hi is exact in FP32;
// x_lo is that difference rounded to TF32 in the same way (|e| <= 2^-23 |x|),
// so the tensor core reads both parts exactly.
__device__ __forceinline__ float round_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = round_tf32(x);
    lo = round_tf32(x - hi);
}

// How a live operand is read from global memory (uniform per operand):
//   KVEC: unit stride along K, 16-byte aligned rows: a warp reads 4 rows x 32 K
//         values (float4 per thread, 4 full 128-byte lines);
//   MVEC: unit stride along the rows, 16-byte aligned K columns: a warp reads
//         32 rows x 4 K values (float4 of 4 rows per thread, 4 full lines);
//   SCALAR: any other strides (4 scalar loads per item, KVEC item order).
enum { KVEC = 0, MVEC = 1, SCALAR = 2 };

__device__ __forceinline__ int operand_mode(const float* src, long long sR, long long sK) {
    const bool al = (reinterpret_cast<unsigned long long>(src) & 15) == 0;
    if (al && sK == 1 && (sR & 3) == 0) return KVEC;
    if (al && sR == 1 && (sK & 3) == 0) return MVEC;
    return SCALAR;
}

// Loader of one live operand of R rows (rows r0.. of Rmax, K values k0.. of
// K): item j of a thread is warp item w = warp + 8 j (R / 32 items per
// thread).  KVEC/SCALAR: row 4 w + lane / 8, K group lane % 8.  MVEC: rows
// 32 (w % (R/32)) + 4 (lane % 8) .. + 3, K value 4 (w / (R/32)) + lane / 8.
// The shared tiles it writes have LR rows (R for A; 2 R for B, whose lo rows
// follow its hi rows in the same tile).
template <int R, int LR = R>
struct Loader {
    static constexpr int N = R / 32;
    const float* src;
    long long sR, sK;
    int mode, Rmax, r0, K, warp, lane;

    __device__ __forceinline__ void fetch(int k0, float4 (&dst)[N]) const {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int w = warp + kLoadWarps * j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mode == MVEC) {
                const int gr = r0 + 32 * (w % (R / 32)) + 4 * (lane & 7);
                const int gk = k0 + 4 * (w / (R / 32)) + (lane >> 3);
                if (gk < K) {
                    const float* q = src + gr + (long long)gk * sK;
                    if (gr + 3 < Rmax) {
                        v = __ldg(reinterpret_cast<const float4*>(q));
                    } else {
                        if (gr < Rmax) v.x = __ldg(q);
                        if (gr + 1 < Rmax) v.y = __ldg(q + 1);
                        if (gr + 2 < Rmax) v.z = __ldg(q + 2);
                    }
                }
            } else {
                const int gr = r0 + 4 * w + (lane >> 3);
                const int gk = k0 + 4 * (lane & 7);
                if (gr < Rmax) {
                    const float* q = src + (long long)gr * sR + (long long)gk * sK;
                    if (mode == KVEC && gk + 3 < K) {
                        v = __ldg(reinterpret_cast<const float4*>(q));
                    } else {
                        if (gk < K) v.x = __ldg(q);
                        if (gk + 1 < K) v.y = __ldg(q + sK);
                        if (gk + 2 < K) v.z = __ldg(q + 2 * sK);
                        if (gk + 3 < K) v.w = __ldg(q + 3 * sK);
                    }
                }
            }
            dst[j] = v;
        }
    }

    // the same items from the chunk's raw tile in shared memory as TMA wrote
    // it: [R][32] (unit stride along K) or [32][R] (unit stride along rows)
    __device__ __forceinline__ void fetch_raw(const float* raw, float4 (&dst)[N]) const {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int w = warp + kLoadWarps * j;
            if (mode == MVEC) {
                const int r = 32 * (w % (R / 32)) + 4 * (lane & 7);
                const int k = 4 * (w / (R / 32)) + (lane >> 3);
                dst[j] = *reinterpret_cast<const float4*>(raw + k * R + r);
            } else {
                const int r = 4 * w + (lane >> 3);
                dst[j] = *reinterpret_cast<const float4*>(raw + r * BK + 4 * (lane & 7));
            }
        }
    }

    __device__ __forceinline__ void store(const float4 (&v)[N], unsigned char* thi, unsigned char* tlo) const {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int w = warp + kLoadWarps * j;
            float4 h, l;
            split_tf32(v[j].x, h.x, l.x);
            split_tf32(v[j].y, h.y, l.y);
            split_tf32(v[j].z, h.z, l.z);
            split_tf32(v[j].w, h.w, l.w);
            if (mode == MVEC) {
                // four rows, one K value: four scalar stores
                const int r = 32 * (w % (R / 32)) + 4 * (lane & 7);
                const int k = 4 * (w / (R / 32)) + (lane >> 3);
                const unsigned o0 = tc_tile_offset(LR, r, k);
                const unsigned d1 = tc_tile_offset(LR, r + 1, k) - o0, d2 = tc_tile_offset(LR, r + 2, k) - o0,
                               d3 = tc_tile_offset(LR, r + 3, k) - o0;
                *reinterpret_cast<float*>(thi + o0) = h.x;
                *reinterpret_cast<float*>(thi + o0 + d1) = h.y;
                *reinterpret_cast<float*>(thi + o0 + d2) = h.z;
                *reinterpret_cast<float*>(thi + o0 + d3) = h.w;
                *reinterpret_cast<float*>(tlo + o0) = l.x;
                *reinterpret_cast<float*>(tlo + o0 + d1) = l.y;
                *reinterpret_cast<float*>(tlo + o0 + d2) = l.z;
                *reinterpret_cast<float*>(tlo + o0 + d3) = l.w;
            } else {
                const int r = 4 * w + (lane >> 3);
                const unsigned off = tc_tile_offset(LR, r, 4 * (lane & 7));
                *reinterpret_cast<float4*>(thi + off) = h;
                *reinterpret_cast<float4*>(tlo + off) = l;
            }
        }
    }
};

}  // namespace tc

// One BM x BN tile of D (rows m0.., columns n0.., batch entry b; the K
// chunks of split sp when K is split) by one CTA of 320 threads (roles in the
// header comment).  PRE = 0: both operands live; 1: A pre-split; 2: B
// pre-split.  SPLIT = false compiles the split of K out (grouped launches).
template <int BN, int PRE, bool SPLIT>
__device__ __forceinline__ void tc_tile(const TcGemmArgs& g, const int m0, const int n0, const int b, const int sp) {
    using namespace tc;
    constexpr int NS = tc_stages<BN, PRE>();
    constexpr unsigned STAGE = tc_stage_bytes<BN, PRE>();
    constexpr unsigned RAW = 2u * tc_tile_bytes(BM) + tc_tile_bytes(2 * BN);   // raw tile offset in a stage
    constexpr int RR = tc_raw_rows<BN, PRE>();
    constexpr unsigned TA = tc_tile_bytes(BM), TB2 = tc_tile_bytes(2 * BN);
    constexpr unsigned LBOA = tc_lbo(BM), LBOB2 = tc_lbo(2 * BN);
    constexpr unsigned BLO = (unsigned)(BN / 8) * kTcSbo;   // B's lo rows after its hi rows
    static_assert(NS >= 2 && (3 * NS + 5) * 8 + 12 <= 256, "stage count");
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    unsigned long long* full = reinterpret_cast<unsigned long long*>(tsm_raw + NS * STAGE);
    unsigned long long* empty = full + NS;
    unsigned long long* txb = empty + NS;   // bulk copies of the pre-split operand
    unsigned long long* accf = txb + NS;    // [2] a chunk group's partial sums are in tensor memory
    unsigned long long* acce = accf + 2;    // [2] the loaders have added them up (buffer free)
    unsigned long long* done = acce + 2;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* last_flag = abort_flag + 1;   // this CTA adds up the tile's partials
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkc = (g.K + BK - 1) / BK;        // K chunks of the whole product
    const bool split = SPLIT && g.splits > 1;
    const int kc0 = split ? g.kb[sp] : 0;       // this CTA's chunks: kc0 .. kc0 + nchunks - 1
    const int nchunks = split ? g.kb[sp + 1] - kc0 : nkc;

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 32 * kLoadWarps);   // every loader thread
            mbar_init(&empty[i], 1);                // the MMA commit
            mbar_init(&txb[i], 1);                  // expect_tx + the copy's bytes
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);                 // the MMA commit
            mbar_init(&acce[i], 32 * kLoadWarps);   // every loader thread
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    constexpr unsigned TCOLS = tmem_cols(BN);
    if (warp == 0) {
        // tensor memory for the tile's FP32 chunk accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp < kLoadWarps) {
        // ---- loader warps ------------------------------------------------------
        const float* A = g.A + (long long)b * g.bA;
        const float* Bm = g.B + (long long)b * g.bB;
        const Loader<BM> la{A, g.sAm, g.sAk, operand_mode(A, g.sAm, g.sAk), g.M, m0, g.K, warp, lane};
        const Loader<BN, 2 * BN> lb{Bm, g.sBn, g.sBk, operand_mode(Bm, g.sBn, g.sBk), g.N, n0, g.K, warp, lane};
        // The live operands of the next PD chunks wait in registers (PD sets
        // used in turn); a chunk's loads are issued after the previous
        // chunk's stores are fenced and published, so the fence never waits
        // for loads in flight.
        constexpr int PD = TC_PREFETCH;
        // the live operand by TMA (a pre-split operand and a tensor map)
        const bool tma = PRE != 0 && g.tmap != nullptr && g.tmap_rows == RR;
        float4 ra[PD][BM / 32], rb[PD][BN / 32];
#pragma unroll
        for (int j = 0; j < PD; ++j)
            if (j < nchunks && !tma) {
                if (PRE != 1) la.fetch((kc0 + j) * BK, ra[j]);
                if (PRE != 2) lb.fetch((kc0 + j) * BK, rb[j]);
            }
        // Accumulation: the MMAs of a group of kGroup K chunks write fresh
        // partial sums into tensor-memory buffer (group % 2) (hi x hi products
        // and cross products in separate halves), and every loader thread adds
        // its row's partials into FP32 registers (round to nearest) once the
        // group's MMAs are done.  The tensor core truncates when it
        // accumulates, so a sum over all of K in tensor memory would drift
        // toward zero by about 2^-25 per accumulation step; here at most
        // 4 kGroup steps accumulate in tensor memory and the group sums round
        // to nearest.
        constexpr int HC = BN / 2;                       // columns of this warp's half
        const int lq = warp & 3, half = warp >> 2;
        float acc[HC];
#pragma unroll
        for (int j = 0; j < HC; ++j) acc[j] = 0.f;
        bool ok = true;
        // warp-uniform bounded wait (lane 0 polls): the tensor-memory loads
        // below are warp-collective
        auto wait_u = [&](unsigned long long* bar, unsigned parity) {
            const bool r = lane == 0 ? mbar_wait_or_abort(bar, parity, abort_flag) : true;
            return __shfl_sync(0xffffffffu, r, 0);
        };
        auto drain = [&](int q) {   // chunk group q
            const int buf = q & 1;
            if (!wait_u(&accf[buf], (unsigned)(q >> 1) & 1u)) {
                ok = false;
                return;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                unsigned v[HC];
#pragma unroll
                for (int cc = 0; cc < HC; cc += 16) {
                    const unsigned col = (unsigned)((buf * 2 + part) * BN + half * HC + cc);
                    const unsigned taddr = tmem + ((unsigned)(lq * 32) << 16) + col;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15}, [%16];"
                        : "=r"(v[cc + 0]), "=r"(v[cc + 1]), "=r"(v[cc + 2]), "=r"(v[cc + 3]), "=r"(v[cc + 4]),
                          "=r"(v[cc + 5]), "=r"(v[cc + 6]), "=r"(v[cc + 7]), "=r"(v[cc + 8]), "=r"(v[cc + 9]),
                          "=r"(v[cc + 10]), "=r"(v[cc + 11]), "=r"(v[cc + 12]), "=r"(v[cc + 13]), "=r"(v[cc + 14]),
                          "=r"(v[cc + 15])
                        : "r"(taddr));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] += __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acce[buf]);
        };
        auto chunk = [&](int c, float4 (&xa)[BM / 32], float4 (&xb)[BN / 32]) {
            const int s = c % NS;
            unsigned char* st = tsm_raw + s * STAGE;
            if (tma) {
                // the chunk's raw tile (and the pre-split tiles) have landed;
                // warp 9 waited for the stage to be free before it issued them
                if (!wait_u(&txb[s], (unsigned)(c / NS) & 1u)) {
                    ok = false;
                    return;
                }
                const float* raw = reinterpret_cast<const float*>(st + RAW);
                if (PRE == 1) lb.fetch_raw(raw, xb);
                if (PRE == 2) la.fetch_raw(raw, xa);
            } else if (c >= NS && !wait_u(&empty[s], (unsigned)((c / NS) - 1) & 1u)) {
                ok = false;
                return;
            }
            if (PRE != 1) la.store(xa, st, st + TA);
            if (PRE != 2) lb.store(xb, st + 2 * TA, st + 2 * TA + BLO);
            // generic-proxy stores -> visible to the tensor core (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
            if (!tma && c + PD < nchunks) {
                if (PRE != 1) la.fetch((kc0 + c + PD) * BK, xa);
                if (PRE != 2) lb.fetch((kc0 + c + PD) * BK, xb);
            }
            // the group before last, at the end of a group: its MMAs finished
            // a whole group ago, and its buffer is free again before the next
            // group's first MMA needs it
            if (c % kGroup == kGroup - 1 && c >= 2 * kGroup - 1) drain(c / kGroup - 1);
        };
        for (int c = 0; c < nchunks && ok; c += PD) {
#pragma unroll
            for (int j = 0; j < PD; ++j)
                if (ok && c + j < nchunks) chunk(c + j, ra[j], rb[j]);
        }
        // the groups not yet added: the last one or two
        for (int q = (nchunks - 1) / kGroup - 1; q <= (nchunks - 1) / kGroup; ++q) {
            const bool done_in_loop = q >= 0 && (q + 2) * kGroup - 1 <= nchunks - 1;
            if (ok && q >= 0 && !done_in_loop) drain(q);
        }

        // ---- epilogue: warp w holds rows 32 (w % 4) + lane of the tile and
        // the column half w / 4
        bool store = ok;
        if (split) {
            // this split's partial tile, column-major (a warp writes 128
            // contiguous bytes per column), then the CTA is counted in; the
            // last of the tile's CTAs adds the partials in split order
            const int mtc = (g.M + BM - 1) / BM, ntc = (g.N + BN - 1) / BN;
            const long long tiles = (long long)mtc * ntc * g.batch;
            const long long tile = ((long long)b * mtc + m0 / BM) * ntc + n0 / BN;
            const long long tsz = (long long)BM * BN;
            float* w0 = g.ws + tile * tsz + lq * 32 + lane + half * HC * BM;
            float* wp = w0 + (long long)sp * tiles * tsz;
#pragma unroll
            for (int j = 0; j < HC; ++j) wp[j * BM] = acc[j];
            __threadfence();
            asm volatile("bar.sync 1, 256;" ::: "memory");   // the loader warps
            if (tid == 0) {
                __threadfence();
                const unsigned prev = atomicAdd(g.cnt + tile, 1u);
                const int last = prev == (unsigned)(g.splits - 1);
                if (last) g.cnt[tile] = 0u;   // all splits counted: zero for the next launch
                __threadfence();
                *last_flag = last;
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");
            store = ok && *last_flag;
            if (store) {
                // every partial from the workspace (this CTA's own included),
                // bypassing L1, in split order
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] = __ldcg(w0 + j * BM);
                for (int t = 1; t < g.splits; ++t) {
                    const float* wt = w0 + (long long)t * tiles * tsz;
#pragma unroll
                    for (int j = 0; j < HC; ++j) acc[j] += __ldcg(wt + j * BM);
                }
            }
        }
        if (store) {
            const int row = m0 + lq * 32 + lane;
            float* Dp = g.D + (long long)b * g.bD;
            if (row < g.M) {
#pragma unroll
                for (int j = 0; j < HC; ++j) {
                    const int n = n0 + half * HC + j;
                    if (n < g.N) Dp[row * g.sDm + n * g.sDn] = acc[j];
                }
            }
        }
    } else if (warp == kLoadWarps) {
        // ---- MMA warp: lane 0 issues, the warp follows --------------------------
        const unsigned idesc = instr_desc<BN>(), idesc2 = instr_desc<2 * BN>();
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % NS, q = c / kGroup, buf = q & 1;
            const bool first = c % kGroup == 0, last = c % kGroup == kGroup - 1 || c == nchunks - 1;
            bool okc = true;
            if (lane == 0) {
                okc = mbar_wait_or_abort(&full[s], (unsigned)(c / NS) & 1u, abort_flag);
                if (PRE && okc) okc = mbar_wait_or_abort(&txb[s], (unsigned)(c / NS) & 1u, abort_flag);
                // the loaders have added up group q - 2, which used this buffer
                if (first && q >= 2 && okc)
                    okc = mbar_wait_or_abort(&acce[buf], (unsigned)((q >> 1) - 1) & 1u, abort_flag);
            }
            if (!__shfl_sync(0xffffffffu, okc, 0)) break;
            if (lane == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned char* st = tsm_raw + s * STAGE;
                const unsigned dhh = tmem + (unsigned)(buf * 2 * BN), dx = dhh + (unsigned)BN;
#pragma unroll
                for (int ks = 0; ks < BK / 8; ++ks) {
                    // K = 8 step ks: core-matrix columns 2 ks, 2 ks + 1
                    const unsigned long long dah = smem_desc(st + 2 * ks * LBOA, LBOA, kTcSbo);
                    const unsigned long long dal = smem_desc(st + TA + 2 * ks * LBOA, LBOA, kTcSbo);
                    const unsigned long long db = smem_desc(st + 2 * TA + 2 * ks * LBOB2, LBOB2, kTcSbo);
                    const unsigned acc = (first && ks == 0) ? 0u : 1u;
                    // A_hi [B_hi; B_lo] into the adjacent (hi x hi, cross)
                    // accumulators with N = 2 BN, then A_lo B_hi (the first BN
                    // rows of the B tile) into the cross one
                    mma_tf32(dhh, dah, db, idesc2, acc);
                    mma_tf32(dx, dal, db, idesc, 1u);
                }
                mma_commit(&empty[s]);
                if (last) mma_commit(&accf[buf]);
            }
            __syncwarp();
        }
        // all MMAs issued so far complete -> done (also after an abort, so that
        // no MMA is in flight when the tensor memory is freed)
        if (lane == 0) {
            mma_commit(done);
            mbar_wait(done, 0u);
        }
        __syncwarp();
    } else if (PRE != 0 && lane == 0) {
        // ---- bulk-copy thread: the pre-split operand's chunks -------------------
        const int rt = PRE == 1 ? m0 / BM : n0 / BN;
        const unsigned blk = PRE == 1 ? 2u * TA : TB2;   // bytes of one pre-split block
        const long long bstride = PRE == 1 ? g.bA : g.bB;
        const float* base = (PRE == 1 ? g.A : g.B) + (long long)b * bstride +
                            ((long long)rt * nkc + kc0) * (blk / 4);
        unsigned char* dst0 = tsm_raw + (PRE == 1 ? 0u : 2u * TA);
        // the live operand's raw chunk by TMA: rows r0.. of the live operand,
        // coordinates (k, row, batch) or (row, k, batch) after its unit stride
        const bool tma = g.tmap != nullptr && g.tmap_rows == RR;
        const float* lsrc = PRE == 1 ? g.B + (long long)b * g.bB : g.A + (long long)b * g.bA;
        const int lmode = PRE == 1 ? operand_mode(lsrc, g.sBn, g.sBk) : operand_mode(lsrc, g.sAm, g.sAk);
        const int lr0 = PRE == 1 ? n0 : m0;
        const int lz = g.batch > 1 ? b : 0;
        constexpr unsigned RAWB = (unsigned)RR * BK * 4u;
        int issued = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % NS;
            if (c >= NS && !mbar_wait_or_abort(&empty[s], (unsigned)((c / NS) - 1) & 1u, abort_flag)) break;
            mbar_arrive_expect_tx(&txb[s], blk + (tma ? RAWB : 0u));
            bulk_copy(dst0 + s * STAGE, base + (long long)c * (blk / 4), blk, &txb[s]);
            if (tma) {
                unsigned char* rdst = tsm_raw + s * STAGE + RAW;
                if (lmode == MVEC) tma_load3(rdst, g.tmap, lr0, (kc0 + c) * BK, lz, &txb[s]);
                else tma_load3(rdst, g.tmap, (kc0 + c) * BK, lr0, lz, &txb[s]);
            }
            issued = c + 1;
        }
        // after an abort, let the copies in flight land before the CTA exits
        // (the phase of a copy's barrier completes when its bytes arrived)
        if (*abort_flag) {
            for (int c = issued - NS < 0 ? 0 : issued - NS; c < issued; ++c)
                (void)mbar_wait(&txb[c % NS], (unsigned)(c / NS) & 1u);
        }
    }

    if (tid == 0 && *abort_flag && g.status) atomicOr(g.status, STATUS_TC_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

template <int BN, int PRE>
__global__ void __launch_bounds__(tc::kThreads, 1) tc_gemm_kernel(const TcGemmArgs g) {
    const int z = (int)blockIdx.z;
    const int s = g.splits > 1 ? z / g.batch : 0;   // z = s * batch + b
    tc_tile<BN, PRE, true>(g, blockIdx.x * tc::BM, blockIdx.y * BN, z - s * g.batch, s);
}

// Grouped form: independent GEMMs of different shapes in one launch; CTA i
// computes the tile items[i] = (GEMM, m tile, n tile, batch entry).
template <int BN, int PRE>
__global__ void __launch_bounds__(tc::kThreads, 1) tc_gemm_grouped_kernel(const TcGemmArgs* gs, const int4* items) {
    const int4 it = items[blockIdx.x];
    tc_tile<BN, PRE, false>(gs[it.x], it.y * tc::BM, it.z * BN, it.w, 0);
}

// Pre-split form of a rows x K operand X(r, k) = X[r * sR + k * sK] with
// tiles of R rows (tc_presplit_floats floats at `out`; zero outside X and in
// the layout's gaps): per block the hi tile then the lo tile (A), or one tile
// of 2 R rows, hi rows first (B, `comb`).
static __global__ void tc_presplit_kernel(const float* X, long long sR, long long sK, int rows, int K, int R, bool comb,
                                          float* out) {
    const int nkc = (K + tc::BK - 1) / tc::BK;
    const long long per_block = (long long)(tc_presplit_block_bytes(R, comb) / 4);
    const long long total = (long long)((rows + R - 1) / R) * nkc * R * tc::BK;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(i % tc::BK);
        const long long t = i / tc::BK;
        const int rr = (int)(t % R);
        const long long blk = t / R;             // rt * nkc + kc
        const int kc = (int)(blk % nkc), rt = (int)(blk / nkc);
        const int r = rt * R + rr, k = kc * tc::BK + kk;
        const float x = (r < rows && k < K) ? X[(long long)r * sR + (long long)k * sK] : 0.f;
        float hi, lo;
        tc::split_tf32(x, hi, lo);
        float* dst = out + blk * per_block;
        if (comb) {
            dst[tc_tile_offset(2 * R, rr, kk) / 4] = hi;
            dst[tc_tile_offset(2 * R, R + rr, kk) / 4] = lo;
        } else {
            const unsigned o = tc_tile_offset(R, rr, kk) / 4;
            dst[o] = hi;
            dst[tc_tile_bytes(R) / 4 + o] = lo;
        }
    }
}

inline cudaError_t launch_tc_presplit(const float* X, long long sR, long long sK, int rows, int K, int R, bool comb,
                                      float* out, cudaStream_t st) {
    if (rows <= 0 || K <= 0 || (R % 32) != 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)tc_presplit_floats(rows, K, R, comb) * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const long long total = (long long)((rows + R - 1) / R) * ((K + tc::BK - 1) / tc::BK) * R * tc::BK;
    const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 4096);
    tc_presplit_kernel<<<grid, 256, 0, st>>>(X, sR, sK, rows, K, R, comb, out);
    return cudaGetLastError();
}

// Tensor map (host copy) of a live operand X(r, k) = X[b bX + r sR + k sK]
// (rows x K, `batch` entries) for TMA loads of its chunks: R x 32 values
// ([R][32] in shared memory when K has unit stride, [32][R] when the rows
// do), zero outside the operand.  False when the strides or the alignment
// allow no tensor map (the kernel then loads the operand per thread).
inline bool tc_make_tmap(CUtensorMap* m, const float* X, long long sR, long long sK, long long bX, int rows, int K,
                         int batch, int R) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if ((reinterpret_cast<unsigned long long>(X) & 15) != 0 || rows <= 0 || K <= 0 || R <= 0 || R > 256) return false;
    if (batch > 1 && (bX <= 0 || (bX * 4) % 16 != 0)) return false;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3], es[3] = {1, 1, 1};
    if (sK == 1 && sR >= K && (sR * 4) % 16 == 0) {
        dims[0] = (cuuint64_t)K;
        dims[1] = (cuuint64_t)rows;
        strides[0] = (cuuint64_t)(sR * 4);
        box[0] = tc::BK;
        box[1] = (cuuint32_t)R;
    } else if (sR == 1 && sK >= rows && (sK * 4) % 16 == 0) {
        dims[0] = (cuuint64_t)rows;
        dims[1] = (cuuint64_t)K;
        strides[0] = (cuuint64_t)(sK * 4);
        box[0] = (cuuint32_t)R;
        box[1] = tc::BK;
    } else {
        return false;
    }
    dims[2] = batch > 1 ? (cuuint64_t)batch : 1;
    strides[1] = batch > 1 ? (cuuint64_t)(bX * 4) : strides[0] * dims[1];
    box[2] = 1;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline int tc_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            sms = n;
        if (sms <= 0) sms = 148;
    }
    return sms;
}

template <int BN, int PRE>
inline cudaError_t launch_tc_gemm_w(const TcGemmArgs& g, cudaStream_t st) {
    const size_t sm = tc_smem_bytes<BN, PRE>();
    cudaFuncSetAttribute(tc_gemm_kernel<BN, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned zs = (unsigned)(g.splits > 1 ? g.splits : 1);
    const dim3 grid((unsigned)((g.M + tc::BM - 1) / tc::BM), (unsigned)((g.N + BN - 1) / BN), (unsigned)g.batch * zs);
    tc_gemm_kernel<BN, PRE><<<grid, tc::kThreads, sm, st>>>(g);
    return cudaGetLastError();
}

template <int PRE>
inline cudaError_t launch_tc_gemm_p(const TcGemmArgs& g, int bn, cudaStream_t st) {
    switch (bn) {
        case 64: return launch_tc_gemm_w<64, PRE>(g, st);
        case 96: return launch_tc_gemm_w<96, PRE>(g, st);
        case 128: return launch_tc_gemm_w<128, PRE>(g, st);
        default: return cudaErrorInvalidValue;
    }
}

// Launches D = A B^T (strided, batched) on the tensor cores with tile width
// g.bn (0: tc_pick_width).  A pre-split B needs g.bn = the R it was split for.
inline cudaError_t launch_tc_gemm(const TcGemmArgs& g, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0 || g.pre < 0 || g.pre > 2) return cudaErrorInvalidValue;
    if (g.pre == 2 && g.bn == 0) return cudaErrorInvalidValue;
    if (g.splits > 1) {
        // a split needs its width fixed (the workspace is sized for it), the
        // workspace and counters, and non-empty chunk ranges covering K
        const int nkc = (g.K + tc::BK - 1) / tc::BK;
        if (g.splits > kTcMaxSplits || g.bn == 0 || !g.ws || !g.cnt || g.kb[0] != 0 || g.kb[g.splits] != nkc ||
            (long long)g.batch * g.splits > 65535)
            return cudaErrorInvalidValue;
        for (int i = 0; i < g.splits; ++i)
            if (g.kb[i + 1] <= g.kb[i]) return cudaErrorInvalidValue;
    }
    const int bn = g.bn ? g.bn : tc_pick_width(&g, 1, tc_sm_count());
    if (g.pre == 1) return launch_tc_gemm_p<1>(g, bn, st);
    if (g.pre == 2) return launch_tc_gemm_p<2>(g, bn, st);
    return launch_tc_gemm_p<0>(g, bn, st);
}

// Work items (GEMM, m tile, n tile, batch entry) of a grouped launch with
// n tiles of width bn.
inline std::vector<int4> tc_group_items(const std::vector<TcGemmArgs>& gs, int bn) {
    std::vector<int4> items;
    for (size_t i = 0; i < gs.size(); ++i)
        for (int b = 0; b < gs[i].batch; ++b)
            for (int mt = 0; mt < (gs[i].M + tc::BM - 1) / tc::BM; ++mt)
                for (int nt = 0; nt < (gs[i].N + bn - 1) / bn; ++nt) items.push_back(make_int4((int)i, mt, nt, b));
    return items;
}

template <int BN, int PRE>
inline cudaError_t launch_tc_grouped_w(const TcGemmArgs* gs, const int4* items, int n_items, cudaStream_t st) {
    const size_t sm = tc_smem_bytes<BN, PRE>();
    cudaFuncSetAttribute(tc_gemm_grouped_kernel<BN, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    tc_gemm_grouped_kernel<BN, PRE><<<(unsigned)n_items, tc::kThreads, sm, st>>>(gs, items);
    return cudaGetLastError();
}

template <int PRE>
inline cudaError_t launch_tc_grouped_p(const TcGemmArgs* gs, const int4* items, int n_items, int bn, cudaStream_t st) {
    switch (bn) {
        case 64: return launch_tc_grouped_w<64, PRE>(gs, items, n_items, st);
        case 96: return launch_tc_grouped_w<96, PRE>(gs, items, n_items, st);
        case 128: return launch_tc_grouped_w<128, PRE>(gs, items, n_items, st);
        default: return cudaErrorInvalidValue;
    }
}

// Grouped launch of n_items tiles of width bn (gs and items in device memory,
// items from tc_group_items with the same bn; every GEMM of the group has
// the same `pre`).
inline cudaError_t launch_tc_gemm_grouped(const TcGemmArgs* gs, const int4* items, int n_items, int bn, int pre,
                                          cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (pre == 1) return launch_tc_grouped_p<1>(gs, items, n_items, bn, st);
    if (pre == 2) return launch_tc_grouped_p<2>(gs, items, n_items, bn, st);
    return launch_tc_grouped_p<0>(gs, items, n_items, bn, st);
}
#endif  // IGAPW_HOST_EMU

}  // namespace igapw
