/*
 * igapw.h -- C ABI of the GB300 (sm_103a) library for isogeometric analysis with
 * piece-wise constant test functions (arXiv 1910.08535).
 *
 * What the library computes (paper section in brackets):
 *   - trial space: tensor-product B-splines of degree p on open knot vectors,
 *     n = N_e + p functions per axis                           [Sec. 2, Eq. (2)]
 *   - tests: B-splines (Galerkin, the comparator) or piece-wise constant
 *     indicators I_i of N_x linearly independent cells (PW)  [Sec. 2, Sec. 3]
 *   - operator action / right-hand side by Gauss quadrature, not integrated
 *     by parts                                                [Sec. 2, Sec. 4.1]
 *   - Kronecker-factored mass solve Mx (x) My (x) Mz as three batches of 1D
 *     banded systems (alternating directions)                 [Sec. 4.1]
 *   - explicit Euler steps, one L2 projection each            [Sec. 4.2, Eq. (6)]
 *   - zero Dirichlet rows by row replacement (Poisson)        [Sec. 4.3]
 *   - 2D/3D Poisson -Lap u = f: the tested operator is a sum of Kronecker
 *     products, solved by fast diagonalisation of the 1D pencils plus
 *     iterative refinement (the paper uses a sparse direct solver) [Sec. 4.3]
 *
 * PW test cells.  The paper leaves the choice of the N_x intervals open and only
 * requires them to be linearly independent (Sec. 2).  This library bounds cell k
 * by the midpoints between consecutive Greville abscissae of the unknowns (the
 * domain ends close the first and last cell) and pairs cell k with unknown k.
 * Every cell is split at the knots into polynomial pieces with their own
 * nq-point Gauss rule.
 *
 * Conventions for every call
 *   - Return 0 on success, a negative IGAPW_ERR_* code on failure; the message
 *     is then available from igapw_last_error(ctx).  No C++ exception crosses
 *     the ABI.
 *   - Tensors are dense, C-ordered, x fastest: shape (n_z, n_y, n_x) in 3D,
 *     (n_y, n_x) in 2D, (n_x) in 1D, with n_a = N_{e,a} + p.  Device pointers
 *     must be 16-byte aligned and are owned by the caller; the library never
 *     frees or reallocates them.  The library's own device buffers are
 *     stream-ordered allocations on the context stream (cudaMallocAsync), so
 *     creating or destroying a context does not synchronise the device.
 *   - Precision IGAPW_FP64: coefficient and RHS tensors are double.
 *     Precision IGAPW_FP32_REFINE: coefficient and RHS tensors are double-float
 *     pairs stored as two consecutive float planes, hi then lo: a float buffer
 *     of 2 * n_total elements whose value is hi + lo.  Contractions run in FP32
 *     with error-free products and two-sum accumulation; line solves run in
 *     FP32 with one step of iterative refinement whose residual is formed in
 *     double-float (or in FP64 with IGAPW_FLAG_FP64_RESIDUAL; GB300 runs FP64
 *     at 1/58 of its FP32 rate, so double-float is the default).  Quadrature-point
 *     samples f passed to igapw_rhs_source are plain float in this mode.
 *   - Work is enqueued on the CUDA stream given at create time and is
 *     asynchronous; calls do not synchronize unless stated.
 *   - The context owns all device tables, factors and scratch buffers.
 */
#ifndef IGAPW_H
#define IGAPW_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define IGAPW_OK                 0
#define IGAPW_ERR_ARG           -1  /* invalid argument or unsupported combination */
#define IGAPW_ERR_SINGULAR      -2  /* zero pivot in a 1D banded factorization      */
#define IGAPW_ERR_OOM           -3  /* device or host allocation failed             */
#define IGAPW_ERR_CUDA          -4  /* a CUDA runtime call failed                   */
#define IGAPW_ERR_DEVICE_STATUS -5  /* a kernel reported a bad value (NaN / Inf)    */
#define IGAPW_ERR_TIMEOUT       -6  /* a bounded device wait gave up                */

/* ---- descriptor enums --------------------------------------------------- */
#define IGAPW_GALERKIN      0  /* B-spline tests (comparator)                       */
#define IGAPW_PWCONST       1  /* piece-wise constant tests                         */
#define IGAPW_REFINED       2  /* refined test space (Sec. 2): test k is the sum of
                                  the B-splines of the test space refined `refine`
                                  times whose Greville abscissae lie in PW cell k;
                                  tends to the PW test as refine grows           */

#define IGAPW_BC_NONE       0  /* all n coefficients free                           */
#define IGAPW_BC_DIRICHLET0 1  /* first/last coefficient per axis held at 0 (1D; in
                                  2D/3D for the POISSON system only)                */

#define IGAPW_FP64          0
#define IGAPW_FP32_REFINE   1

#define IGAPW_OP_MASS       0  /* F u = u         (L2 projection, Sec. 4.1)         */
#define IGAPW_OP_LAPLACE    1  /* F u = Lap u     (apply only)                      */
#define IGAPW_OP_HEAT       2  /* F u = u + dt Lap u (explicit step, Sec. 4.2)      */
#define IGAPW_OP_POISSON    3  /* F u = -Lap u    (Poisson system, Sec. 4.3)        */

#define IGAPW_FLAG_FP64_RESIDUAL 1  /* FP32_REFINE: form the refinement residual of
                                       igapw_solve (and of RHS-then-solve steps) in
                                       FP64 instead of double-float (FP32 pairs)      */
#define IGAPW_FLAG_STEP_RHS_SOLVE 2 /* igapw_step runs the literal sequence of Sec. 4.2:
                                       tested RHS T(u + dt Lap u), then the Kronecker
                                       mass solve; default is the split form (see
                                       igapw_step)                                    */
#define IGAPW_FLAG_FDM_BF16X9 4     /* 2D/3D POISSON: run the transforms of the solve
                                       as cuBLAS FP32 GEMMs emulated with bf16 terms
                                       on the tensor pipe (BF16x9) instead of the
                                       library's tcgen05 split-TF32 kernel            */
#define IGAPW_FLAG_FDM_CUBLAS 8     /* 2D/3D POISSON: run the transforms as plain
                                       cuBLAS FP32 GEMMs (CUDA cores) instead of the
                                       library's tcgen05 split-TF32 kernel            */

#define IGAPW_MAX_DIM    3
#define IGAPW_MAX_DEGREE 4

typedef struct igapw_ctx igapw_ctx;

/* Problem descriptor.  dim in {1,2,3}; n_elem[a] >= 1 elements on axis a
 * (entries beyond dim ignored); degree p in {2,3,4} (C^{p-1}, at least C^1 as
 * the method requires, Sec. 2); nq >= 1 Gauss points per element (Galerkin) or
 * per polynomial piece of a cell (PW) or per refined element (REFINED);
 * test = IGAPW_GALERKIN | IGAPW_PWCONST | IGAPW_REFINED;
 * bc = IGAPW_BC_*; precision = IGAPW_FP64 | IGAPW_FP32_REFINE; op = IGAPW_OP_*
 * selects the matrix igapw_solve inverts (POISSON: -Lap u with bc = DIRICHLET0
 * required -- in 1D the banded 1D operator, in 2D/3D the multi-D operator;
 * anything else: the tensor-product mass matrix); flags = IGAPW_FLAG_*.
 * With neumann_axes, the operator rows of a Neumann axis get the boundary
 * term [T du/dn] of Sec. 4.3 (-int T B'' + T(b) B'(b) - T(a) B'(a) along that
 * axis) and every coefficient on it is an unknown.
 * A 2D/3D POISSON context also diagonalises every 1D pencil (L_a, A_a) at
 * creation (FP64 LU and nonsymmetric eigensolver through cuSOLVER, O(n_a^3));
 * creation fails with IGAPW_ERR_ARG if a pencil's spectrum is not real and
 * positive (non-negative on a Neumann axis). */
typedef struct {
    int dim;
    int n_elem[3];
    int degree;
    int nq;
    int test;
    int bc;
    int precision;
    int op;
    int flags;
    int neumann_axes;   /* POISSON, 2D/3D: bit a set = axis a carries Neumann data on both
                           of its end faces instead of zero Dirichlet rows (Sec. 4.3 mixed
                           boundary conditions); at least one axis must stay Dirichlet */
    int refine;         /* IGAPW_REFINED: parts per element of the test space (2..64);
                           its quadrature has nq points per refined element */
} igapw_desc;

/* Builds knots, Gauss rules and PW cells on the host, evaluates the basis by
 * Cox--de Boor at every quadrature point and folds it into per-axis banded
 * tables on the device (int T_i B_j and int T_i B_j''), then factors the 1D
 * system bands in FP64 on the device (banded LU, no pivoting) [Sec. 2, Sec. 4.1].
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out owns device memory until igapw_destroy.  Blocks until the
 * set-up kernels finish so that a singular factorization (IGAPW_ERR_SINGULAR,
 * linearly dependent tests, Sec. 2) is reported here.
 * The context belongs to the CUDA device current at this call: every later
 * call on it makes that device current for its duration and restores the
 * caller's device before returning (cuda_stream must belong to that device). */
int igapw_create(igapw_ctx** out, const igapw_desc* desc, void* cuda_stream);

/* Replaces the knot vector of one axis by a caller-given open knot vector
 * (len = n_elem[axis] + 2p + 1 non-decreasing values, first and last repeated
 * p+1 times, no interior knot repeated more than p-1 times so C^1 holds) and
 * rebuilds that axis' tables and factors.  Host pointer, copied. Synchronous.
 * Layout limit: every row of the 1D tables is stored as a window of W
 * consecutive columns whose start advances by 0 or 1 from row to row.  With
 * PW or refined tests, a knot vector whose element sizes change abruptly (a
 * cell spanning several small elements next to large ones: most random knot
 * vectors, or geometric grading above a ratio of about 1.5 per element) breaks
 * that rule and is rejected with IGAPW_ERR_ARG and a message; B-spline tests
 * accept any open knot vector. */
int igapw_set_knots(igapw_ctx* ctx, int axis, const double* knots, int len);

/* The 1D quadrature point set of one axis in increasing x: every element
 * (Galerkin) or every polynomial piece of every cell (PW) with its nq Gauss
 * points.  igapw_rhs_source expects f sampled on the tensor product of these
 * sets (x fastest).  If x and w are NULL only *count is written; otherwise they
 * must hold *count doubles (host memory).  Synchronous, host only. */
int igapw_quad_points(igapw_ctx* ctx, int axis, double* x, double* w, int* count);

/* Exports the basis table of kernel (a) for one axis to host memory:
 * vals[(q * (p+1) + a) * 3 + k] = d^k B_{s_q + a}(x_q), k = 0,1,2, where
 * s_q = first_fn[q] is the first non-zero function at point q.  vals holds
 * count*(p+1)*3 doubles, first_fn holds count ints (either may be NULL).
 * Synchronous (test aid). */
int igapw_basis_table(igapw_ctx* ctx, int axis, double* vals, int* first_fn);

/* Source right-hand side b = int T_i f over the tensor grid of quadrature
 * points: PW sums the quadrature weights times f over each cell (the test is
 * 1; one fused pass, every sample read once), Galerkin multiplies by the test
 * B-splines (one pass per axis through intermediates allocated on the first
 * call) [Sec. 4.1 generation loops].
 * f_dev: device, FP64 (FP64 mode) or float (FP32_REFINE) samples on the
 * igapw_quad_points grid.  b_dev: device coefficient-shaped tensor (double, or
 * float hi/lo pair planes).  Dirichlet rows get b = 0. Asynchronous. */
int igapw_rhs_source(igapw_ctx* ctx, const void* f_dev, void* b_dev);

/* Source RHS of the separable source f(x) = amp * prod_a sin(k[a] pi x_a)
 * [Sec. 4.1 generation of the right-hand side, for a source known in closed
 * form]: b = T f over the context's quadrature points, with the source
 * evaluated on the device (FP64 sinpi) instead of sampled by the caller.
 * Because the tests are tensor products, b = amp (x)_a v_a with the 1D sums
 * v_a[i] = sum_q T_a,i(x_q) w_q sin(k[a] pi x_q) over the axis' points
 * (v in FP64, b written as FP64 or FP32 pairs per precision; Dirichlet rows
 * b = 0).  With amp = pi^2 sum_a k[a]^2 it is the source of the manufactured
 * solution u = prod_a sin(k[a] pi x_a) of -Lap u = f.  k: host array of dim
 * doubles.  b_dev: caller-owned device tensor.  Asynchronous; allocates
 * nothing (the context holds the 1D factors). */
int igapw_rhs_source_sine(igapw_ctx* ctx, double amp, const double* k, void* b_dev);

/* Allocation-free variant of igapw_rhs_source (the paper has no counterpart:
 * this is a deployment aid).  igapw_rhs_source allocates the two intermediate
 * tensors of its axis-by-axis passes on its first call for a context (a
 * stream-ordered allocation after a wait for the context stream); callers
 * that cannot let the library allocate there (hosts that reserve all device
 * memory up front, schedulers admitting work against a fixed device-memory
 * budget, latency-critical loops that cannot take that wait) call this
 * instead.  It computes the
 * same b into the caller's b_dev, taking its intermediates from one static
 * device array of IGAPW_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until exit; it calls no allocating routine.
 *   - Sizes: with B-spline tests each intermediate needs
 *     8 * max(q_z q_y n_x, q_z n_y n_x) bytes (q_a = igapw_quad_points count);
 *     PW tests (one fused pass) and 1D need none.  Above half the array the
 *     call returns IGAPW_ERR_ARG with the sizes in igapw_last_error.
 *   - The array lives in a module of its own, which CUDA may load lazily (and
 *     only then reserve the array): igapw_create looks its address up on the
 *     context's device, so the array is in place before the first call, and
 *     this entry point itself never causes that load.  Each call looks the
 *     address up again on the context's device (a lookup, no allocation).
 *   - All calls on a device share the array and leave their intermediates in
 *     it; calls whose work overlaps on the GPU (different streams or contexts
 *     without ordering between them) race on it and must be serialised.
 * Asynchronous on the context stream, like igapw_rhs_source. */
#define IGAPW_NOALLOC_SCRATCH_BYTES (8u << 20)
int igapw_rhs_source_noalloc(igapw_ctx* ctx, const void* f_dev, void* b_dev);

/* Operator action r = T(F u) with F chosen by op (IGAPW_OP_MASS, LAPLACE,
 * HEAT with time step dt, POISSON), tests T of the context, computed by
 * sum-factorised per-axis contractions of the folded quadrature tables
 * [Sec. 2 / Sec. 3 systems; Sec. 4.2 RHS].  u_dev, r_dev: device tensors of
 * the context precision; they must not overlap.  For a Dirichlet context the
 * Dirichlet rows return r_i = u_i (row replacement, Sec. 4.3); in 2D/3D a row
 * is a Dirichlet row when any of its axis indices is, and POISSON applies
 * sum_a (-int T B'' along a) (x) (int T B along the other axes) on the
 * others. Asynchronous. */
int igapw_apply(igapw_ctx* ctx, int op, double dt, const void* u_dev, void* r_dev);

/* Neumann data term of Sec. 4.3: b += int over the end face (side 0: x_a = 0
 * end, 1: the far end) of a Neumann axis of T G, for G sampled on the tensor
 * grid of the other axes' quadrature points (igapw_quad_points; x fastest among
 * them; FP64 samples, or FP32 in FP32_REFINE contexts).  With the tests' end
 * values T_i(end) = 1 for the end row only (PW end cells and open-knot
 * B-splines alike), this adds the face's 1D-tested data to the rows whose
 * index on `axis` is the end.  Dirichlet rows stay untouched.  b_dev is a
 * context tensor (accumulated in place).  Asynchronous. */
int igapw_rhs_neumann(igapw_ctx* ctx, int axis, int side, const void* g_dev, void* b_dev);

/* Exports one 1D matrix of an axis as a dense row-major n x n double array in
 * host memory: which = IGAPW_OP_MASS (int T_i B_j), IGAPW_OP_LAPLACE
 * (int T_i B_j''), or IGAPW_OP_POISSON (the factored 1D Poisson system with
 * Dirichlet rows).  Synchronous (test aid). */
int igapw_assemble_1d(igapw_ctx* ctx, int axis, int which, double* dense_host);

/* Solves S u = r with S the tensor product of the per-axis system matrices
 * (mass, or the 1D Poisson operator): one batch of banded line solves per
 * axis with the precomputed FP64 LU factors [Sec. 4.1 ADS].  FP32_REFINE: an
 * FP32 solve, the residual r - S u0 (double-float or FP64), a second FP32
 * solve, u = u0 + correction stored as a hi/lo pair.  r_dev == u_dev is
 * allowed.
 * 2D/3D POISSON contexts solve K u = r for the multi-D operator instead: with
 * A_a^{-1} L_a = V_a Lambda_a V_a^{-1} per axis (unknown rows and columns),
 * P = diag(I on Dirichlet rows, (V_x V_y V_z) diag(1/(lx+ly+lz)) (W_x W_y W_z)),
 * W_a = V_a^{-1} A_a^{-1}, applied as FP32 GEMMs along each axis, inside
 * iterative refinement whose residual r - K u is taken by the contraction
 * kernel: one correction in FP32_REFINE (residual in double-float, or FP64
 * with IGAPW_FLAG_FP64_RESIDUAL), three corrections in FP64 (FP64 residual).
 * r_dev and u_dev must differ.  Asynchronous. */
int igapw_solve(igapw_ctx* ctx, const void* r_dev, void* u_dev);

/* nsteps explicit Euler steps of u_t = Lap u in place on u_dev [Sec. 4.2,
 * Eq. (6)]: every step solves M u' = T(u + dt Lap u) with the tested mass
 * M = A_z (x) A_y (x) A_x and the tested Laplacian, A = int T_i B_j and
 * C = int T_i B_j'' per axis.  Default (split form): the other axes' mass
 * factors cancel against the solve, so each step runs one kernel per axis that
 * forms g = C u along every line of that axis, solves A w = g along the same
 * line and accumulates u' = u + dt (w_x + w_y + w_z) -- the same discrete
 * scheme with a different rounding order.  With IGAPW_FLAG_STEP_RHS_SOLVE the
 * step forms the RHS with igapw_apply(HEAT) and solves with igapw_solve.
 * Needs a mass-matrix context (op != POISSON).  The step sequence is captured
 * once per (dt, nsteps, u_dev) into a CUDA graph and replayed. Asynchronous,
 * except the first split-form call on a context: it times the launch shapes of
 * the per-axis kernel (staged or global tables, lines or columns per block) on
 * scratch tensors and waits for the context stream, so that call must not be
 * made inside a stream capture. */
int igapw_step(igapw_ctx* ctx, double dt, int nsteps, void* u_dev);

/* Launch shape of the split-form step kernel along one axis (a tuning
 * control; no counterpart in the paper, which fixes no implementation).
 * kind: 0 lines staged with the tables in shared memory (lines = x-lines or
 * y/z columns per block, 32/16/8), 1 tables read from global memory (long
 * lines), 2 staged tables with 16 columns, 3 the chunked kernel that keeps
 * every line in registers in chunks of 17 rows (FP32_REFINE contexts whose
 * lines have at most 544 rows; lines = 32, 16 or 8 lines per block).
 * igapw_set_step_shape pins axis `axis` to (kind, lines); kind = -1 hands the
 * axis back to the autotuner of the first igapw_step call.  A shape that
 * cannot run on the context makes the next igapw_step fail with
 * IGAPW_ERR_CUDA.  Pinning drops the captured step graphs.
 * igapw_get_step_shape reports the shape in use (kind = -1: not tuned yet). */
int igapw_set_step_shape(igapw_ctx* ctx, int axis, int kind, int lines);
int igapw_get_step_shape(igapw_ctx* ctx, int axis, int* kind, int* lines);

/* Same as igapw_step with HOST buffers: copies u_host (pinned memory gives an
 * asynchronous copy) into a context-owned device state, runs nsteps, copies
 * the result back to u_host and synchronizes the stream before returning.
 * u_host holds n_total doubles (FP64) or 2*n_total floats (FP32_REFINE). */
int igapw_step_host(igapw_ctx* ctx, double dt, int nsteps, void* u_host);

/* Waits for the context stream, then returns IGAPW_OK, IGAPW_ERR_CUDA if an
 * asynchronous CUDA error occurred, or IGAPW_ERR_DEVICE_STATUS if a kernel
 * flagged a non-finite value in a solve.  Clears the device status word. */
int igapw_sync_status(igapw_ctx* ctx);

/* Message for the last failure on this context (or on create, when ctx is
 * NULL: the thread's last create error).  Never NULL. */
const char* igapw_last_error(igapw_ctx* ctx);

/* Number of coefficients n_total = prod_a n_a, and n_a per axis (dims may be
 * NULL). */
long long igapw_size(igapw_ctx* ctx, int* dims);

/* Frees everything the context owns.  Synchronizes its stream first. */
int igapw_destroy(igapw_ctx* ctx);

/* ---- the dense transform kernel -------------------------------------------
 * D(m, n) = sum_k A(m, k) B(n, k) for batch entries b = 0 .. batch-1, with
 * A(m, k) = A[b bA + m sAm + k sAk], B(n, k) = B[b bB + n sBn + k sBk],
 * D(m, n) = D[b bD + m sDm + n sDn] (device pointers, FP32, strides in
 * elements): the split-TF32 tcgen05 GEMM that runs the fast-diagonalisation
 * transforms of the POISSON solve (each FP32 operand split into a TF32 high
 * part and an FP32 low part, three tensor-core products summed in FP32;
 * relative error about 2^-21 per product; each 32-wide K chunk summed in
 * tensor memory, the chunks summed in FP32 registers).  pre = 1 (2): A (B) is split once
 * into shared-memory tiles before the product and streamed by bulk copies,
 * the path the solver takes for its constant matrices; a pre-split operand
 * must have batch stride 0 when batch > 1.  bn: tile width (0, 64, 96 or
 * 128; 0 lets the cost model choose).  splits: K split over several CTAs
 * per tile when the tiles alone leave SMs idle (0: the cost model chooses
 * the split together with the width; 1: none; 2-4: that many equal ranges of
 * 32-wide K chunks, at most ceil(K / 32)); each CTA writes its FP32 partial
 * tile to a workspace and the tile's last CTA adds the partials in a fixed
 * order, so the result does not depend on the CTAs' timing.  Synchronous on
 * cuda_stream (NULL: the legacy default stream).  IGAPW_ERR_TIMEOUT if a
 * pipeline wait of the kernel timed out; the message is in
 * igapw_last_error(NULL).  Allocates temporary buffers when pre != 0 or K
 * is split. */
int igapw_tc_gemm(int M, int N, int K, int batch, const float* A, long long sAm, long long sAk, long long bA,
                  const float* B, long long sBn, long long sBk, long long bB, float* D, long long sDm, long long sDn,
                  long long bD, int pre, int bn, int splits, void* cuda_stream);

/* ---- batched 2D Poisson over many uneven instances ----------------------
 * The problem of Sec. 4.3 (-Lap u = f, zero Dirichlet rows, Eq. (7) tested
 * with PW cells or B-splines) for `count` independent 2D instances of
 * different sizes and degrees, FP32 pairs with one refinement step (as
 * igapw_solve on a 2D POISSON context).  Each stage runs for all instances
 * in one launch: the source RHS (a persistent kernel over a work queue of
 * instance tiles), the fast-diagonalisation transforms (grouped GEMMs on the
 * library's tensor-core kernel, each instance's x and y matrices split once
 * into hi/lo tiles at creation; plain cuBLAS grouped FP32 GEMMs instead when
 * descs[0].flags has IGAPW_FLAG_FDM_CUBLAS), the
 * double-float residual (persistent kernels, one per window width) and the
 * elementwise updates; the solve is captured once into a CUDA graph.  The
 * batch owns the instances' RHS and solution tensors (pair layout, see
 * igapw_batch_tensor). */
typedef struct igapw_batch igapw_batch;

/* descs[count]: each dim = 2, op = POISSON, bc = DIRICHLET0, precision =
 * FP32_REFINE (else IGAPW_ERR_ARG).  Builds one context per instance (tables,
 * diagonalised pencils), packs their tensors, and times the candidate tile
 * shapes of the two persistent kernels on the batch, keeping the fastest.
 * Synchronous. */
int igapw_batch_create(igapw_batch** out, const igapw_desc* descs, int count, void* cuda_stream);

/* RHS of every instance for the manufactured source
 * f_i(x, y) = amp_i sin(kx_i pi x) sin(ky_i pi y), evaluated in the kernel at
 * each instance's quadrature points (FP32, like igapw_rhs_source samples) and
 * summed over the test supports in double-float.  params: host array of
 * count x 3 doubles (amp, kx, ky).  Synchronous. */
int igapw_batch_source_sine(igapw_batch* b, const double* params);

/* u_i = K_i^{-1} b_i for every instance (the batch's RHS tensors, e.g. from
 * igapw_batch_source_sine or written through igapw_batch_tensor).
 * Asynchronous on the batch stream (one graph launch). */
int igapw_batch_solve(igapw_batch* b);

/* Synchronizes the batch stream and reads the batch's device status word:
 * IGAPW_ERR_TIMEOUT if a tensor-core GEMM gave up waiting for its pipeline
 * (its results are then invalid), else IGAPW_OK (or the CUDA error of the
 * stream). */
int igapw_batch_sync_status(igapw_batch* b);

/* Device pointer of instance i's RHS (which = 0) or solution (which = 1):
 * a pair tensor of 2 * n_total floats owned by the batch. */
int igapw_batch_tensor(igapw_batch* b, int i, int which, void** dev, long long* n_total);

/* Tile shapes picked by the autotuner: tiles[0..1] source (x, y), tiles[2..3]
 * residual (x, y). */
int igapw_batch_info(igapw_batch* b, int* tiles);

/* Message of the last failure on the batch (NULL: the thread's last create
 * error).  Never NULL. */
const char* igapw_batch_last_error(igapw_batch* b);

/* Frees the batch and its instances' contexts (synchronizes the stream). */
int igapw_batch_destroy(igapw_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* IGAPW_H */
