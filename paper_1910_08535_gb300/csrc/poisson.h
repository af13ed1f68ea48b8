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
    bool tensor = false;                           // FP32 GEMMs emulated on the bf16 tensor pipe
};

// Builds the spectral data of every axis (FP64 LU and eigendecomposition on
// the device, then FP32 copies).  Returns 0, or a message in err.
int fdm_build(FdmState& s, int dim, const FdmAxisInput* ax, const int* const* is_free_dev, bool tensor,
              cudaStream_t st, std::string& err);
void fdm_release(FdmState& s);

// Poisson solve K u = b.  Scratch: rho (ntot floats) and, for pair tensors,
// u0 (ntot floats); the spectral buffers are the state's own.  b and u are
// pair tensors (fp64 == false) or double tensors (fp64 == true; `iters`
// refinement steps).
int fdm_solve(FdmState& s, const ContractArgs& ca, const void* b, void* u, bool fp64, int iters, float* rho,
              float* u0, bool pair_fp64_residual, cudaStream_t st, std::string& err);

// r = K u (MODE_PK) or rho = r - K u (MODE_PRES) through the contraction kernel.
cudaError_t launch_poisson_contract(const ContractArgs& a, int mode, int cmp, int io, cudaStream_t st);

}  // namespace igapw
