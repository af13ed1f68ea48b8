// Multi-D Poisson solve by fast diagonalisation (poisson.cu <-> api.cu).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "kernels.h"

typedef struct cublasContext* cublasHandle_t;

namespace igapw {

// Host view of one axis' folded 1D tables (window layout, n x W).
struct FdmAxisInput {
    int n = 0, W = 0;
    std::vector<double> A, C;        // int T_i B_j, int T_i B_j'' (Dirichlet rows: A identity, C 0)
    std::vector<int> fstart, is_free;
    bool neumann = false;            // Neumann axis: the pencil has the constants as a zero mode
};

// Spectral data of one 1D pencil, embedded in the full index range [0, n):
// unknown k of the axis' free set sits at index free[k]; boundary rows and
// columns of W and V are zero and the boundary eigenvalues are 1 (never
// divided into a non-zero value).  Shared by every axis and context with the
// same 1D tables (a process-wide cache, see poisson.cu); freed with the last
// reference.
struct FdmAxisData {
    int device = 0, n = 0;
    int np = 0;             // n padded to a multiple of 8 (leading dimension)
    float* Wm = nullptr;    // np x np column-major, V^{-1} A_I^{-1} (zero padding)
    float* Vm = nullptr;    // np x np column-major, V (zero padding)
    float* lam = nullptr;   // np eigenvalues of A_I^{-1} L_I (1 on boundary and padding)
    ~FdmAxisData();
};

struct FdmState {
    int dim = 0;
    int n[3] = {1, 1, 1};
    std::shared_ptr<FdmAxisData> axis[3];
    float* Wm[3] = {nullptr, nullptr, nullptr};
    float* Vm[3] = {nullptr, nullptr, nullptr};
    float* lam[3] = {nullptr, nullptr, nullptr};
    const int* is_free[3] = {nullptr, nullptr, nullptr};
    int px = 1;                                    // padded x pitch of the spectral buffers
    float* t[2] = {nullptr, nullptr};              // spectral buffers, (n_z, n_y, px) floats each
    cudaStream_t stream = nullptr;                 // stream of the buffers' allocation
    cublasHandle_t blas = nullptr;
    int gemm = 0;                                  // transforms: FDM_GEMM_TC, _CUBLAS or _BF16X9
    unsigned* status = nullptr;                    // device status word (tensor-core wait timeouts)
    cudaStream_t stream_now = nullptr;             // stream of the solve in progress
    // tensor-core engine: W and V of every axis split once into hi/lo
    // shared-memory tiles (tcgemm.cuh), as the GEMM's A operand (x axis,
    // pre_role 1) or B operand (y and z axes, pre_role 2, tile width pre_bn)
    float* pre[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    int pre_role[3] = {0, 0, 0};
    int pre_bn[3] = {0, 0, 0};
    // device tensor maps of the live (spectral) operand per axis and input
    // buffer t[0] / t[1] (null entries: per-thread loads), their tile rows
    void* tmaps = nullptr;
    bool tmap_ok[3][2] = {{false, false}, {false, false}, {false, false}};
    int tmap_rows[3] = {0, 0, 0};
    // split of K per axis (tcgemm.cuh's tc_plan: splits, chunk boundaries;
    // the tile width is pre_bn), the split products' partial tiles and
    // per-tile counters (zero between launches)
    int splits[3] = {1, 1, 1};
    int kb[3][5] = {};
    float* tc_ws = nullptr;
    unsigned* tc_cnt = nullptr;
};

// Engines of the dense per-axis transforms: the library's tcgen05 split-TF32
// kernel (tcgemm.cuh), cuBLAS FP32 GEMMs, cuBLAS BF16x9 emulation.
enum { FDM_GEMM_TC = 0, FDM_GEMM_CUBLAS = 1, FDM_GEMM_BF16X9 = 2 };

// Builds the spectral data of every axis (FP64 LU and eigendecomposition on
// the device, then FP32 copies).  Returns 0, or a message in err.
int fdm_build(FdmState& s, int dim, const FdmAxisInput* ax, const int* const* is_free_dev, int gemm,
              unsigned* status, cudaStream_t st, std::string& err);
void fdm_release(FdmState& s);

// Poisson solve K u = b.  Scratch: rho (ntot floats) and, for pair tensors,
// u0 (ntot floats); the spectral buffers are the state's own.  b and u are
// pair tensors (fp64 == false) or double tensors (fp64 == true; `iters`
// refinement steps).
int fdm_solve(FdmState& s, const ContractArgs& ca, const void* b, void* u, bool fp64, int iters, float* rho,
              float* u0, bool pair_fp64_residual, cudaStream_t st, std::string& err);

// The tensor-core GEMM of the transforms on caller buffers (tcgemm.cuh;
// synchronous; cudaErrorLaunchTimeout when a pipeline wait timed out).
struct TcGemmArgs;
cudaError_t tc_gemm_entry(const TcGemmArgs& g, cudaStream_t st);

// r = K u (MODE_PK) or rho = r - K u (MODE_PRES) through the contraction kernel.
cudaError_t launch_poisson_contract(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st);

}  // namespace igapw
