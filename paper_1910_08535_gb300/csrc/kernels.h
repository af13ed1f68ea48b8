// Internal launch interface between the C ABI (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <string>

struct igapw_ctx;

#include "common.cuh"

#define IGAPW_MAXP 4
// rows per chunk of the chunked explicit step (the kernels' compile-time chunk length)
#ifndef IGAPW_CHUNK_ROWS
#define IGAPW_CHUNK_ROWS 17
#endif

namespace igapw {

struct FoldArgs {
    int n, p, W, WQ, test, poisson;
    int neumann;                 // add the Neumann boundary term to C (rows 0 and n-1)
    const double* dleft;         // [n] B_j'(a)
    const double* dright;        // [n] B_j'(b)
    const double* twr;           // refined test space: w_q T_i(x_q), [n][WQ] (test == 2)
    const int* fstart;
    const int* pstart;
    const int* pcount;
    const int* is_free;
    const int* qfirst;
    const double* qw;
    const double* vals;
    double *A, *C, *S, *TW;
    float2 *Adf, *Cdf, *Sdf, *TWdf;
};

struct FactorArgs {
    int n, p, W, P;
    int b[33];
    const int* fstart;
    const double* S;
    double* work;
    double *L, *U, *dinv, *G, *H, *PhiF, *PhiB;
    float *L32, *U32, *dinv32, *G32, *H32, *PhiF32, *PhiB32;
    unsigned* status;
};

// Packed tables of the chunked step (chunkstep.cuh) from the FP64 factors.
struct ChunkTableArgs {
    int n, p, W, RS, P;           // lines padded to P * RS rows
    const double *L, *U, *dinv;   // factor_kernel output, [n][p] / [n]
    const float2 *Adf, *Cdf;      // [n][W] double-float windows
    const int* fstart;
    double* work;                 // [2 P RS p]
    float4 *cw, *aw;              // [P RS][nq4]
    float4 *fl, *fu, *fg, *fh;    // [P RS]
    float *fd, *psf, *psb;        // [P RS], [P][P][p][p]
    int* J;
};
void launch_chunk_tables(const ChunkTableArgs& a, cudaStream_t st);

void launch_basis_table(const double* t, int p, int Q, const double* qx, const int* qfirst,
                        double* vals, cudaStream_t st);
void launch_fold(const FoldArgs& f, cudaStream_t st);
void launch_factor(const FactorArgs& a, cudaStream_t st);

// ---- sum-factorised contractions (rhs.cu) ----------------------------------
// MODE_OP:  r = T(alpha u + beta Lap u) with the folded A / C tables
// MODE_SYS: r = (S_z (x) S_y (x) S_x) u with the system tables
// MODE_RES: rho = r - (S_z (x) S_y (x) S_x) u0   (refinement residual)
// MODE_PK:  r = K u, the multi-D Poisson operator: MODE_OP with alpha = 0,
//           beta = -1 on rows off the boundary, u itself on boundary rows
// MODE_PRES: rho = r - K u (F32 out; u F32 with pair r, or F64 with F64 r)
enum { MODE_OP = 0, MODE_SYS = 1, MODE_RES = 2, MODE_PK = 3, MODE_PRES = 4 };
// compute / storage formats
enum { FMT_F64 = 0, FMT_PAIR = 1, FMT_F32 = 2 };

struct ContractArgs {
    int dim, W;
    int n[3];               // n_x, n_y, n_z
    int zchunk;
    int tx, ty;             // runtime tile widths (<= the kernel's compile-time tile)
    AxisDev ax[3];
    const void* u;          // MODE_OP/SYS/PK: F64 or PAIR; MODE_RES: F32 u0; MODE_PRES: F32 or F64
    const void* r;          // MODE_RES/PRES: right-hand side (PAIR, or F64 for PRES)
    void* out;              // F64 / PAIR / F32 (MODE_RES)
    long long ntot;         // elements per plane of a pair tensor
    double alpha, beta;
};

// cmp: FMT_F64 (double arithmetic) or FMT_PAIR (double-float arithmetic);
// io: FMT_F64 (double tensors) or FMT_PAIR (pair tensors; MODE_RES reads
// F32 u0 + PAIR r and writes F32).  Returns a CUDA error code.
cudaError_t launch_contract(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st);

// ---- source right-hand side (rhs.cu) ----------------------------------------
// b = (TW_z (x) TW_y (x) TW_x) f over the quadrature grid: PW tests in one
// fused pass (every point belongs to one cell), Galerkin one axis per pass.
struct SourceArgs {
    int dim;
    int pw;                 // PW tests: one fused pass, no intermediates
    int n[3];               // coefficients per axis
    int q[3];               // points per axis
    AxisDev ax[3];
    const void* f;          // F64 or F32 samples, x fastest
    void* out;              // F64 or PAIR
    void* work0;            // scratch, >= max intermediate size (doubles or pairs)
    void* work1;
    long long ntot;
};
cudaError_t launch_source(const SourceArgs& a, int fp64, cudaStream_t st);

// b = amp (x)_a v_a, v_a = TW_a sin(k_a pi x_a) at the axis' points (separable
// sine source); v: three device buffers of n_a doubles (the context sets
// v[d] = 1.0 once for the absent axes).
struct SineSourceArgs {
    int dim;
    int n[3];
    int q[3];
    AxisDev ax[3];
    const double* qx[3];
    double k[3];
    double amp;
    double* v[3];
    void* out;
    long long ntot;
};
cudaError_t launch_source_sine(const SineSourceArgs& a, int fp64, cudaStream_t st);

// b += face term of a Neumann axis: sum over the other axes' point windows of
// their test weights times g, added to the rows at the axis end.
struct NeumannArgs {
    int dim, axis, side;
    int n[3];
    int q[3];
    AxisDev ax[3];
    const void* g;          // F64 or F32 samples on the other axes' point grid
    void* b;                // F64 or PAIR
    long long ntot;
};
cudaError_t launch_neumann(const NeumannArgs& a, int fp64, cudaStream_t st);

// ---- line solves (solve.cu) -------------------------------------------------
// Solves along one axis of a (n_z, n_y, n_x) tensor with the axis' LU.
//   in_fmt  FMT_F64 | FMT_F32 | FMT_PAIR (hi plane read as FP32)
//   out_fmt FMT_F64 | FMT_F32 | FMT_PAIR (finish: out = u0 + x as a pair, u0 F32)
struct SolveArgs {
    int axis;
    int n[3];
    const void* in;
    void* out;
    const float* u0;        // finish epilogue only
    long long ntot;
    unsigned* status;
};
cudaError_t launch_solve(const SolveArgs& s, const AxisDev& ax, int p, int in_fmt, int out_fmt,
                         bool fp64, cudaStream_t st);

// ---- split explicit step (step.cu) -------------------------------------------
// One launch per axis: for every line along `axis`, g = C u, w = A^{-1} g (with
// one double-float refinement in pair mode), and
//   mode 0: acc = u + dt w; 1: acc += dt w; 2: u_out = acc + dt w; 3: u_out = u + dt w.
struct AxisStepArgs {
    int axis;
    int n[3];
    int W;
    int lines_per_block;    // lines staged per block: x-lines, or columns (a power of
                            // two <= 32) of y/z-lines (set by the launcher, or forced)
    int cfg;                // -1: the launcher's own choice; else forced with lines_per_block:
                            // 0 staged tables, 1 tables in global memory, 2 staged 16 columns,
                            // 3 the chunked register kernel (FP32 pairs; 32, 16 or 8 lines)
    int pdl;                // chunked kernel: launch with programmatic stream serialization
                            // (the step's launches overlap; see chunkstep.cuh)
    long long ntot;
    AxisDev ax;
    const void* u;
    void* u_out;
    void* acc;
    double dt;
    unsigned* status;
};
cudaError_t launch_axis_step(const AxisStepArgs& a, int mode, bool fp64, int p, cudaStream_t st);

// ---- allocation-free source entry point (noalloc.cu <-> api.cu) ------------
// Fills the source launch arguments of a context (work buffers left NULL) and
// the bytes each of the two intermediates needs; records errors on the context.
// Device address of the static scratch array of the allocation-free source
// entry point on the current device (loads the module holding it if needed).
cudaError_t noalloc_scratch_address(void** out);
// Current-device scope for entry points, and the device a context belongs to.
struct DeviceGuard {
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;

private:
    int prev_ = -1;
    bool switched_ = false;
};
int ctx_device(const ::igapw_ctx* c);
int source_setup(::igapw_ctx* c, const void* f_dev, void* b_dev, SourceArgs& a, size_t& need,
                 cudaStream_t& st, bool& f64);
int record_error(::igapw_ctx* c, int code, const std::string& msg);

// ---- read-only view of a context for the batched entry points (batch.cu) ----
struct FdmState;
struct CtxView {
    int dim, W, p, precision, op, test;
    int n[3];
    int q[3];                 // quadrature points per axis
    long long ntot;
    AxisDev ax[3];
    const double* qx[3];      // device quadrature-point coordinates per axis
    const FdmState* fdm;      // 2D/3D Poisson contexts: spectral data
};
int ctx_view(::igapw_ctx* c, CtxView& v);

}  // namespace igapw
