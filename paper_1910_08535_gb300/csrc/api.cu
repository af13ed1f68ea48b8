// C ABI (include/igapw.h): context set-up, operator action, solves, explicit
// steps captured as CUDA graphs.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/igapw.h"
#include "kernels.h"
#include "poisson.h"
#include "tcgemm.cuh"
#include "setup.h"

using namespace igapw;

namespace {

thread_local std::string g_create_error;

struct AxisMem {
    double *knots = nullptr, *qx = nullptr, *qw = nullptr, *vals = nullptr;
    int *qfirst = nullptr, *fstart = nullptr, *pstart = nullptr, *pcount = nullptr, *is_free = nullptr;
    double *A = nullptr, *C = nullptr, *S = nullptr, *TW = nullptr;
    double *dleft = nullptr, *dright = nullptr, *twr = nullptr;
    float2 *Adf = nullptr, *Cdf = nullptr, *Sdf = nullptr, *TWdf = nullptr;
    double *band = nullptr, *L = nullptr, *U = nullptr, *dinv = nullptr, *G = nullptr, *H = nullptr,
           *PhiF = nullptr, *PhiB = nullptr;
    float *L32 = nullptr, *U32 = nullptr, *dinv32 = nullptr, *G32 = nullptr, *H32 = nullptr,
          *PhiF32 = nullptr, *PhiB32 = nullptr;
    // chunked-step tables
    double* ck_work = nullptr;
    float4 *ck_cw = nullptr, *ck_aw = nullptr, *ck_fl = nullptr, *ck_fu = nullptr, *ck_fg = nullptr, *ck_fh = nullptr;
    float *ck_fd = nullptr, *ck_psf = nullptr, *ck_psb = nullptr;
    int* ck_J = nullptr;
};

struct GraphEntry {
    double dt;
    int nsteps;
    void* u;
    cudaGraphExec_t exec;
};

}  // namespace

struct igapw_ctx {
    igapw_desc d{};
    int device = 0;          // the CUDA device current at igapw_create; every call runs on it
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int dim = 1, p = 2, W = 3, WQ = 1;
    int n[3] = {1, 1, 1};
    long long ntot = 1;
    AxisSetup ax[3];
    AxisMem mem[3];
    AxisDev dev[3];
    std::vector<void*> allocs;
    // scratch
    void* r = nullptr;       // RHS: double [ntot] or pair [2 ntot]
    void* w = nullptr;       // line-solve intermediate: double or float [ntot]
    float* u0 = nullptr;     // FP32 first solve [ntot]
    float* rho = nullptr;    // FP32 residual [ntot]
    void* state = nullptr;   // igapw_step_host device state
    double* sine_v[3] = {nullptr, nullptr, nullptr};   // rhs_source_sine 1D factors
    void* src0 = nullptr;    // rhs_source intermediates
    void* src1 = nullptr;
    size_t src_bytes = 0;
    unsigned* status = nullptr;
    std::string err;
    std::vector<GraphEntry> graphs;
    FdmState* fdm = nullptr;  // multi-D Poisson contexts: spectral data of the 1D pencils
    // split-step launch shapes per axis picked by timing (-1: not tuned yet)
    int step_cfg[3] = {-1, -1, -1};
    int step_nl[3] = {0, 0, 0};
    bool step_pinned[3] = {false, false, false};
};

namespace {

// FP64 multi-D Poisson: refinement corrections after the first FP32 solve
constexpr int kPoissonRefineF64 = 3;
// chunked explicit step: rows per chunk (the kernels' compile-time length) and
// the most chunks a line may have (512 threads at 16 lines per block)
constexpr int kChunkRows = IGAPW_CHUNK_ROWS;
constexpr int kChunkMaxP = 32;

int fail(igapw_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

}  // namespace

namespace igapw {

// Makes `dev` the current device for the scope of an entry point and restores
// the caller's device on return (a context's memory, streams and graphs
// belong to the device it was created on).
DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) == cudaSuccess && prev_ != dev) switched_ = cudaSetDevice(dev) == cudaSuccess;
}
DeviceGuard::~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
}

int ctx_device(const ::igapw_ctx* c) { return c->device; }

// Bounds-check readers of the translation units (debug builds register one each).
static std::vector<BoundsReader>& bounds_readers() {
    static std::vector<BoundsReader> r;
    return r;
}
void register_bounds_reader(BoundsReader r) { bounds_readers().push_back(r); }

}  // namespace igapw

namespace {

#define CKC(c, x)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (x);                                                                       \
        if (e_ != cudaSuccess)                                                                      \
            return fail(c, e_ == cudaErrorMemoryAllocation ? IGAPW_ERR_OOM : IGAPW_ERR_CUDA,        \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

// Device buffers are stream-ordered allocations on the context stream, so
// creating and destroying contexts never synchronises the whole device (other
// contexts keep running, e.g. while a request server evicts one).
template <typename T>
cudaError_t dalloc(igapw_ctx* c, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), c->stream);
    if (e == cudaSuccess) c->allocs.push_back(*p);
    return e;
}

template <typename T>
cudaError_t upload(igapw_ctx* c, T** p, const std::vector<T>& h) {
    cudaError_t e = dalloc(c, p, h.size());
    if (e != cudaSuccess) return e;
    if (!h.empty()) e = cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
    return e;
}

int pad_width(int w) {
    if (w <= 3) return 3;
    if (w <= 5) return 5;
    if (w <= 7) return 7;
    if (w <= 9) return 9;
    return -1;
}

void free_graphs(igapw_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

bool fp64(const igapw_ctx* c);

// (Re)builds the device tables and factors of axis a from c->ax[a].
int build_axis_device(igapw_ctx* c, int a) {
    AxisSetup& s = c->ax[a];
    AxisMem& m = c->mem[a];
    const int n = s.n, p = s.p, W = c->W, WQ = c->WQ;
    const int Q = (int)s.qx.size();
    CKC(c, upload(c, &m.knots, s.knots));
    CKC(c, upload(c, &m.qx, s.qx));
    CKC(c, upload(c, &m.qw, s.qw));
    CKC(c, upload(c, &m.qfirst, s.qfirst));
    CKC(c, upload(c, &m.fstart, s.fstart));
    CKC(c, upload(c, &m.pstart, s.pstart));
    CKC(c, upload(c, &m.pcount, s.pcount));
    CKC(c, upload(c, &m.is_free, s.is_free));
    if (s.test == 2) {   // refined tests: host table re-laid with the context's point-window stride
        std::vector<double> twr((size_t)n * WQ, 0.0);
        for (int i = 0; i < n; ++i)
            for (int w = 0; w < s.pcount[i]; ++w) twr[(size_t)i * WQ + w] = s.tw_refined[(size_t)i * s.wq + w];
        CKC(c, upload(c, &m.twr, twr));
    }
    CKC(c, upload(c, &m.dleft, s.dleft));
    CKC(c, upload(c, &m.dright, s.dright));
    const int neumann = (c->d.neumann_axes >> a) & 1;
    if (neumann) {
        // the end rows' windows must hold every column with a non-zero end derivative
        for (int j = 0; j < n; ++j) {
            if (s.dleft[j] != 0.0 && (j < s.fstart[0] || j >= s.fstart[0] + W))
                return fail(c, IGAPW_ERR_ARG, "Neumann term outside the first row's window");
            if (s.dright[j] != 0.0 && (j < s.fstart[n - 1] || j >= s.fstart[n - 1] + W))
                return fail(c, IGAPW_ERR_ARG, "Neumann term outside the last row's window");
        }
    }
    CKC(c, dalloc(c, &m.vals, (size_t)Q * (p + 1) * 3));
    const size_t nw = (size_t)n * W, nt = (size_t)n * WQ;
    CKC(c, dalloc(c, &m.A, nw)); CKC(c, dalloc(c, &m.C, nw)); CKC(c, dalloc(c, &m.S, nw));
    CKC(c, dalloc(c, &m.TW, nt));
    CKC(c, dalloc(c, &m.Adf, nw)); CKC(c, dalloc(c, &m.Cdf, nw)); CKC(c, dalloc(c, &m.Sdf, nw));
    CKC(c, dalloc(c, &m.TWdf, nt));
    const size_t np = (size_t)n * p, nphi = (size_t)5 * 32 * p * p;
    CKC(c, dalloc(c, &m.band, (size_t)n * (2 * p + 1)));
    CKC(c, dalloc(c, &m.L, np)); CKC(c, dalloc(c, &m.U, np)); CKC(c, dalloc(c, &m.dinv, (size_t)n));
    CKC(c, dalloc(c, &m.G, np)); CKC(c, dalloc(c, &m.H, np));
    CKC(c, dalloc(c, &m.PhiF, nphi)); CKC(c, dalloc(c, &m.PhiB, nphi));
    CKC(c, dalloc(c, &m.L32, np)); CKC(c, dalloc(c, &m.U32, np)); CKC(c, dalloc(c, &m.dinv32, (size_t)n));
    CKC(c, dalloc(c, &m.G32, np)); CKC(c, dalloc(c, &m.H32, np));
    CKC(c, dalloc(c, &m.PhiF32, nphi)); CKC(c, dalloc(c, &m.PhiB32, nphi));

    // kernel (a): basis table, then fold into the banded tables
    launch_basis_table(m.knots, p, Q, m.qx, m.qfirst, m.vals, c->stream);
    FoldArgs f{};
    f.n = n; f.p = p; f.W = W; f.WQ = WQ; f.test = s.test; f.poisson = (c->d.op == IGAPW_OP_POISSON && c->dim == 1);
    f.neumann = neumann; f.dleft = m.dleft; f.dright = m.dright; f.twr = m.twr;
    f.fstart = m.fstart; f.pstart = m.pstart; f.pcount = m.pcount; f.is_free = m.is_free;
    f.qfirst = m.qfirst; f.qw = m.qw; f.vals = m.vals;
    f.A = m.A; f.C = m.C; f.S = m.S; f.TW = m.TW;
    f.Adf = m.Adf; f.Cdf = m.Cdf; f.Sdf = m.Sdf; f.TWdf = m.TWdf;
    launch_fold(f, c->stream);
    // kernel (c1): FP64 banded LU + partitioned-solve data
    FactorArgs fa{};
    fa.n = n; fa.p = p; fa.W = W; fa.P = s.P;
    for (int k = 0; k <= s.P; ++k) fa.b[k] = s.chunk_b[k];
    fa.fstart = m.fstart; fa.S = m.S; fa.work = m.band;
    fa.L = m.L; fa.U = m.U; fa.dinv = m.dinv; fa.G = m.G; fa.H = m.H; fa.PhiF = m.PhiF; fa.PhiB = m.PhiB;
    fa.L32 = m.L32; fa.U32 = m.U32; fa.dinv32 = m.dinv32; fa.G32 = m.G32; fa.H32 = m.H32;
    fa.PhiF32 = m.PhiF32; fa.PhiB32 = m.PhiB32;
    fa.status = c->status;
    // 2D/3D Poisson contexts solve by fast diagonalisation: no banded LU
    const bool banded = !(c->d.op == IGAPW_OP_POISSON && c->dim >= 2);
    if (banded) launch_factor(fa, c->stream);
    CKC(c, cudaGetLastError());
    // tables of the chunked explicit step (FP32-pair contexts with a mass matrix,
    // lines of at most kChunkMaxP chunks)
    int ckP = 0;
    if (banded && !fp64(c) && c->d.op != IGAPW_OP_POISSON && p <= 4) {
        ckP = (n + kChunkRows - 1) / kChunkRows;
        if (ckP > kChunkMaxP) ckP = 0;
    }
    if (ckP > 0) {
        const int q4 = (2 * W + 4) / 4;
        const size_t np = (size_t)ckP * kChunkRows;   // padded line
        CKC(c, dalloc(c, &m.ck_work, 2 * np * p));
        CKC(c, dalloc(c, &m.ck_cw, np * q4)); CKC(c, dalloc(c, &m.ck_aw, np * q4));
        CKC(c, dalloc(c, &m.ck_fl, np)); CKC(c, dalloc(c, &m.ck_fu, np));
        CKC(c, dalloc(c, &m.ck_fg, np)); CKC(c, dalloc(c, &m.ck_fh, np));
        CKC(c, dalloc(c, &m.ck_fd, np));
        CKC(c, dalloc(c, &m.ck_psf, (size_t)ckP * ckP * p * p)); CKC(c, dalloc(c, &m.ck_psb, (size_t)ckP * ckP * p * p));
        CKC(c, dalloc(c, &m.ck_J, (size_t)1));
        ChunkTableArgs ca{};
        ca.n = n; ca.p = p; ca.W = W; ca.RS = kChunkRows; ca.P = ckP;
        ca.L = m.L; ca.U = m.U; ca.dinv = m.dinv; ca.Adf = m.Adf; ca.Cdf = m.Cdf; ca.fstart = m.fstart;
        ca.work = m.ck_work;
        ca.cw = m.ck_cw; ca.aw = m.ck_aw; ca.fl = m.ck_fl; ca.fu = m.ck_fu; ca.fg = m.ck_fg; ca.fh = m.ck_fh;
        ca.fd = m.ck_fd; ca.psf = m.ck_psf; ca.psb = m.ck_psb; ca.J = m.ck_J;
        launch_chunk_tables(ca, c->stream);
        CKC(c, cudaGetLastError());
    }

    AxisDev& D = c->dev[a];
    D.n = n; D.nq = Q; D.wq = WQ;
    D.fstart = m.fstart; D.pstart = m.pstart; D.pcount = m.pcount; D.is_free = m.is_free;
    D.A = {m.A, m.Adf};
    D.C = {m.C, m.Cdf};
    D.S = {m.S, m.Sdf};
    D.TW = {m.TW, m.TWdf};
    D.ls64.n = n; D.ls64.P = s.P;
    D.ls32.n = n; D.ls32.P = s.P;
    for (int k = 0; k < 33; ++k) { D.ls64.b[k] = s.chunk_b[k]; D.ls32.b[k] = s.chunk_b[k]; }
    D.ls64.L = m.L; D.ls64.U = m.U; D.ls64.dinv = m.dinv; D.ls64.G = m.G; D.ls64.H = m.H;
    D.ls64.PhiF = m.PhiF; D.ls64.PhiB = m.PhiB;
    D.ls32.L = m.L32; D.ls32.U = m.U32; D.ls32.dinv = m.dinv32; D.ls32.G = m.G32; D.ls32.H = m.H32;
    D.ls32.PhiF = m.PhiF32; D.ls32.PhiB = m.PhiB32;
    D.ck = ChunkDev{};
    if (ckP > 0) {
        D.ck.rows = kChunkRows; D.ck.P = ckP;
        D.ck.cw = m.ck_cw; D.ck.aw = m.ck_aw; D.ck.fl = m.ck_fl; D.ck.fu = m.ck_fu;
        D.ck.fd = m.ck_fd; D.ck.fg = m.ck_fg; D.ck.fh = m.ck_fh;
        D.ck.psf = m.ck_psf; D.ck.psb = m.ck_psb; D.ck.J = m.ck_J;
    }
    return IGAPW_OK;
}

int check_setup_status(igapw_ctx* c) {
    CKC(c, cudaStreamSynchronize(c->stream));
    unsigned st = 0;
    CKC(c, cudaMemcpy(&st, c->status, sizeof st, cudaMemcpyDeviceToHost));
    if (st & STATUS_SINGULAR) {
        unsigned z = 0;
        cudaMemcpy(c->status, &z, sizeof z, cudaMemcpyHostToDevice);
        return fail(c, IGAPW_ERR_SINGULAR, "zero pivot in a 1D banded factorization (linearly dependent tests)");
    }
    return IGAPW_OK;
}

bool fp64(const igapw_ctx* c) { return c->d.precision == IGAPW_FP64; }

ContractArgs contract_args(igapw_ctx* c) {
    ContractArgs a{};
    a.dim = c->dim;
    a.W = c->W;
    for (int k = 0; k < 3; ++k) { a.n[k] = c->n[k]; a.ax[k] = c->dev[k]; }
    // z-chunk: aim at >= 2 blocks per SM over the whole grid
    a.zchunk = c->n[2];
    if (c->dim == 3) {
        const long long xy_tiles = (long long)((c->n[0] + 31) / 32) * ((c->n[1] + 7) / 8);
        const long long want = 2 * 152;
        long long chunks = (want + xy_tiles - 1) / xy_tiles;
        if (chunks < 1) chunks = 1;
        a.zchunk = (int)((c->n[2] + chunks - 1) / chunks);
        if (a.zchunk < 4) a.zchunk = 4;
    }
    a.ntot = c->ntot;
    return a;
}

// The solve chain: axis 0 reads `in`, the last axis writes `out`.
int solve_chain(igapw_ctx* c, const void* in, int in_fmt, void* out, int out_fmt, const float* u0,
                cudaStream_t st) {
    const bool f64 = fp64(c);
    for (int a = 0; a < c->dim; ++a) {
        SolveArgs s{};
        s.axis = a;
        for (int k = 0; k < 3; ++k) s.n[k] = c->n[k];
        s.ntot = c->ntot;
        s.status = c->status;
        s.u0 = u0;
        s.in = a == 0 ? in : c->w;
        s.out = a == c->dim - 1 ? out : c->w;
        const int fi = a == 0 ? in_fmt : (f64 ? FMT_F64 : FMT_F32);
        const int fo = a == c->dim - 1 ? out_fmt : (f64 ? FMT_F64 : FMT_F32);
        cudaError_t e = launch_solve(s, c->dev[a], c->p, fi, fo, f64, st);
        if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("line solve: ") + cudaGetErrorString(e));
    }
    return IGAPW_OK;
}

// Full solve S u = r (with refinement in FP32_REFINE mode).
int enqueue_solve(igapw_ctx* c, const void* r, void* u, cudaStream_t st) {
    if (fp64(c)) return solve_chain(c, r, FMT_F64, u, FMT_F64, nullptr, st);
    int rc = solve_chain(c, r, FMT_PAIR, c->u0, FMT_F32, nullptr, st);
    if (rc) return rc;
    ContractArgs a = contract_args(c);
    a.u = c->u0;
    a.r = r;
    a.out = c->rho;
    const int cmp = (c->d.flags & IGAPW_FLAG_FP64_RESIDUAL) ? FMT_F64 : FMT_PAIR;
    cudaError_t e = launch_contract(a, MODE_RES, cmp, FMT_PAIR, st);
    if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
    return solve_chain(c, c->rho, FMT_F32, u, FMT_PAIR, c->u0, st);
}

int enqueue_apply(igapw_ctx* c, int mode, double alpha, double beta, const void* u, void* r, cudaStream_t st) {
    ContractArgs a = contract_args(c);
    a.u = u;
    a.out = r;
    a.alpha = alpha;
    a.beta = beta;
    const int f = fp64(c) ? FMT_F64 : FMT_PAIR;
    cudaError_t e = launch_contract(a, mode, f, f, st);
    if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("contract: ") + cudaGetErrorString(e));
    return IGAPW_OK;
}

int enqueue_steps(igapw_ctx* c, double dt, int nsteps, void* u, cudaStream_t st) {
    if (!(c->d.flags & IGAPW_FLAG_STEP_RHS_SOLVE)) {
        // split form: one kernel per axis and step (step.cu)
        for (int s = 0; s < nsteps; ++s) {
            for (int ax = 0; ax < c->dim; ++ax) {
                AxisStepArgs a{};
                a.axis = ax;
                for (int k = 0; k < 3; ++k) a.n[k] = c->n[k];
                a.W = c->W;
                a.ntot = c->ntot;
                a.ax = c->dev[ax];
                a.u = u;
                a.u_out = u;
                a.acc = c->r;
                a.dt = dt;
                a.status = c->status;
                a.cfg = c->step_cfg[ax];
                a.lines_per_block = c->step_nl[ax];
                // chunked launches overlap their predecessor (programmatic dependent
                // launch): each waits on the device before it reads what the
                // previous launch writes (chunkstep.cuh)
                a.pdl = a.cfg == 3 ? 1 : 0;
                const int mode = c->dim == 1 ? 3 : (ax == 0 ? 0 : (ax == c->dim - 1 ? 2 : 1));
                cudaError_t e = launch_axis_step(a, mode, fp64(c), c->p, st);
                if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("axis step: ") + cudaGetErrorString(e));
            }
        }
        return IGAPW_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
        int rc = enqueue_apply(c, MODE_OP, 1.0, dt, u, c->r, st);
        if (rc) return rc;
        rc = enqueue_solve(c, c->r, u, st);
        if (rc) return rc;
    }
    return IGAPW_OK;
}

// Split-step autotuner: per axis, times every launch shape of the step kernels
// (chunked with 32 / 16 / 8 lines; staged tables with 32 / 16 / 8 lines or
// columns; tables in global memory with 32 down to 1, the narrow shapes for
// lines of several thousand rows) on zeroed scratch tensors
// and keeps the first valid shape unless a later one is 10% faster.  Runs once
// per context, before the first step is captured.
int tune_step(igapw_ctx* c, double dt) {
    static const int cand[][2] = {{3, 32}, {3, 16}, {3, 8}, {0, 32}, {0, 16}, {0, 8}, {2, 16},
                                  {1, 32}, {1, 16}, {1, 8}, {1, 4}, {1, 2}, {1, 1}};
    const size_t bytes = (size_t)c->ntot * 8;   // one pair or FP64 tensor
    unsigned char *tu = nullptr, *tacc = nullptr;
    CKC(c, cudaMallocAsync((void**)&tu, bytes, c->stream));
    CKC(c, cudaMallocAsync((void**)&tacc, bytes, c->stream));
    CKC(c, cudaMemsetAsync(tu, 0, bytes, c->stream));
    CKC(c, cudaMemsetAsync(tacc, 0, bytes, c->stream));
    cudaEvent_t e0, e1;
    CKC(c, cudaEventCreate(&e0));
    CKC(c, cudaEventCreate(&e1));
    int rc = IGAPW_OK;
    for (int ax = 0; ax < c->dim && !rc; ++ax) {
        if (c->step_pinned[ax]) continue;
        const int mode = c->dim == 1 ? 3 : (ax == 0 ? 0 : (ax == c->dim - 1 ? 2 : 1));
        float best = 1e30f;
        for (const auto& cd : cand) {
            AxisStepArgs a{};
            a.axis = ax;
            for (int k = 0; k < 3; ++k) a.n[k] = c->n[k];
            a.W = c->W;
            a.ntot = c->ntot;
            a.ax = c->dev[ax];
            a.u = tu;
            a.u_out = tu;
            a.acc = tacc;
            a.dt = dt;
            a.status = c->status;
            a.cfg = cd[0];
            a.lines_per_block = cd[1];
            if (launch_axis_step(a, mode, fp64(c), c->p, c->stream) != cudaSuccess) {
                cudaGetLastError();   // shape not valid for this axis: skip
                continue;
            }
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 3; ++r) launch_axis_step(a, mode, fp64(c), c->p, c->stream);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = fail(c, IGAPW_ERR_CUDA, "step autotuning failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            // candidates come in order of preference: a later one must be 10%
            // faster to replace the current choice (timing noise, or a profiler
            // serialising every launch, does not flip it)
            if (best > 1e29f || ms < 0.9f * best) {
                best = ms;
                c->step_cfg[ax] = cd[0];
                c->step_nl[ax] = cd[1];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(tu, c->stream);
    cudaFreeAsync(tacc, c->stream);
    CKC(c, cudaStreamSynchronize(c->stream));
    return rc;
}

int valid_desc(const igapw_desc* d, std::string& why) {
    if (!d) { why = "desc is NULL"; return 0; }
    if (d->dim < 1 || d->dim > 3) { why = "dim must be 1, 2 or 3"; return 0; }
    for (int a = 0; a < d->dim; ++a)
        if (d->n_elem[a] < 1) { why = "n_elem must be >= 1"; return 0; }
    if (d->degree < 2 || d->degree > IGAPW_MAX_DEGREE) { why = "degree must be 2..4 (C^1 or smoother)"; return 0; }
    if (d->nq < 1 || d->nq > 16) { why = "nq must be 1..16"; return 0; }
    if (d->test != IGAPW_GALERKIN && d->test != IGAPW_PWCONST && d->test != IGAPW_REFINED) {
        why = "unknown test";
        return 0;
    }
    if (d->test == IGAPW_REFINED && (d->refine < 2 || d->refine > 64)) {
        why = "the refined test space needs refine in 2..64";
        return 0;
    }
    if (d->bc != IGAPW_BC_NONE && d->bc != IGAPW_BC_DIRICHLET0) { why = "unknown bc"; return 0; }
    if (d->bc == IGAPW_BC_DIRICHLET0 && d->dim != 1 && d->op != IGAPW_OP_POISSON) {
        why = "Dirichlet rows in 2D/3D are supported for the POISSON system only";
        return 0;
    }
    if (d->precision != IGAPW_FP64 && d->precision != IGAPW_FP32_REFINE) { why = "unknown precision"; return 0; }
    if (d->op < IGAPW_OP_MASS || d->op > IGAPW_OP_POISSON) { why = "unknown op"; return 0; }
    if (d->op == IGAPW_OP_POISSON && d->bc != IGAPW_BC_DIRICHLET0) {
        why = "the POISSON system needs Dirichlet rows";
        return 0;
    }
    if (d->neumann_axes) {
        const int all = (1 << d->dim) - 1;
        if (d->op != IGAPW_OP_POISSON || d->dim < 2) {
            why = "Neumann axes are supported for the 2D/3D POISSON system";
            return 0;
        }
        if ((d->neumann_axes & ~all) || (d->neumann_axes & all) == all) {
            why = "neumann_axes must name axes of the problem and leave at least one Dirichlet axis";
            return 0;
        }
    }
    return 1;
}

int alloc_scratch(igapw_ctx* c) {
    const size_t nt = (size_t)c->ntot;
    for (int a = 0; a < 3; ++a) {
        if (a < c->dim) {
            CKC(c, dalloc(c, &c->sine_v[a], (size_t)c->n[a]));
        } else {   // an absent axis enters the separable source as the factor 1
            CKC(c, upload(c, &c->sine_v[a], std::vector<double>{1.0}));
        }
    }
    if (fp64(c)) {
        CKC(c, dalloc(c, (double**)&c->r, nt));
        CKC(c, dalloc(c, (double**)&c->w, nt));
    } else {
        CKC(c, dalloc(c, (float**)&c->r, 2 * nt));
        CKC(c, dalloc(c, (float**)&c->w, nt));
        CKC(c, dalloc(c, &c->u0, nt));
        CKC(c, dalloc(c, &c->rho, nt));
    }
    return IGAPW_OK;
}

// Boundary rows of axis a: a Neumann axis has none (every coefficient is free).
int axis_bc(const igapw_desc& d, int a) {
    return ((d.neumann_axes >> a) & 1) ? IGAPW_BC_NONE : d.bc;
}

// Multi-D Poisson contexts: diagonalise the 1D pencils of every axis (poisson.cu).
int build_fdm(igapw_ctx* c) {
    if (c->d.op != IGAPW_OP_POISSON || c->dim < 2) return IGAPW_OK;
    CKC(c, cudaStreamSynchronize(c->stream));
    FdmAxisInput in[3];
    const int* fr[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < c->dim; ++a) {
        const AxisSetup& s = c->ax[a];
        in[a].n = s.n;
        in[a].W = c->W;
        in[a].A.resize((size_t)s.n * c->W);
        in[a].C.resize((size_t)s.n * c->W);
        CKC(c, cudaMemcpy(in[a].A.data(), c->mem[a].A, in[a].A.size() * 8, cudaMemcpyDeviceToHost));
        CKC(c, cudaMemcpy(in[a].C.data(), c->mem[a].C, in[a].C.size() * 8, cudaMemcpyDeviceToHost));
        in[a].fstart = s.fstart;
        in[a].is_free = s.is_free;
        in[a].neumann = (c->d.neumann_axes >> a) & 1;
        fr[a] = c->mem[a].is_free;
    }
    c->fdm = new (std::nothrow) FdmState();
    if (!c->fdm) return fail(c, IGAPW_ERR_OOM, "host allocation failed");
    std::string err;
    const int gemm = (c->d.flags & IGAPW_FLAG_FDM_BF16X9)   ? FDM_GEMM_BF16X9
                     : (c->d.flags & IGAPW_FLAG_FDM_CUBLAS) ? FDM_GEMM_CUBLAS
                                                            : FDM_GEMM_TC;
    const int rc = fdm_build(*c->fdm, c->dim, in, fr, gemm, c->status, c->stream, err);
    if (rc) return fail(c, rc, "Poisson set-up: " + err);
    return IGAPW_OK;
}

int setup_all(igapw_ctx* c, const std::vector<double>* knots_override, int override_axis) {
    const igapw_desc& d = c->d;
    int wmax = 0, wqmax = 0;
    for (int a = 0; a < c->dim; ++a) {
        std::vector<double> kn;
        if (knots_override && a == override_axis) kn = *knots_override;
        else if (!c->ax[a].knots.empty() && c->ax[a].n_elem == d.n_elem[a] && knots_override) kn = c->ax[a].knots;
        std::string e = build_axis(c->ax[a], d.n_elem[a], d.degree, d.nq, d.test, axis_bc(d, a), kn, d.refine);
        if (!e.empty()) return fail(c, IGAPW_ERR_ARG, "axis " + std::to_string(a) + ": " + e);
        wmax = std::max(wmax, c->ax[a].w);
        wqmax = std::max(wqmax, c->ax[a].wq);
    }
    c->W = pad_width(wmax);
    c->WQ = std::max(wqmax, 1);
    if (c->W < 0) return fail(c, IGAPW_ERR_ARG, "window too wide");
    for (int a = 0; a < c->dim; ++a)
        if (!set_window(c->ax[a], c->W)) return fail(c, IGAPW_ERR_ARG, "banded window layout failed");
    for (int a = 0; a < c->dim; ++a) set_chunks(c->ax[a], c->ntot / c->n[a]);
    for (int a = 0; a < c->dim; ++a) {
        int rc = build_axis_device(c, a);
        if (rc) return rc;
    }
    int rc = check_setup_status(c);
    if (rc) return rc;
    return build_fdm(c);
}

void release(igapw_ctx* c) {
    free_graphs(c);
    if (c->fdm) {
        fdm_release(*c->fdm);
        delete c->fdm;
        c->fdm = nullptr;
    }
    for (void* p : c->allocs) cudaFreeAsync(p, c->stream);
    c->allocs.clear();
}

}  // namespace

extern "C" {

int igapw_create(igapw_ctx** out, const igapw_desc* desc, void* cuda_stream) {
    if (!out) return fail(nullptr, IGAPW_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!valid_desc(desc, why)) return fail(nullptr, IGAPW_ERR_ARG, why);
    igapw_ctx* c = new (std::nothrow) igapw_ctx();
    if (!c) return fail(nullptr, IGAPW_ERR_OOM, "host allocation failed");
    c->d = *desc;
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)cuda_stream;
    c->dim = desc->dim;
    c->p = desc->degree;
    c->ntot = 1;
    for (int a = 0; a < 3; ++a) {
        c->n[a] = a < c->dim ? desc->n_elem[a] + desc->degree : 1;
        c->ntot *= c->n[a];
    }
    int rc = IGAPW_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = fail(c, IGAPW_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    if (!rc) {
        e = dalloc(c, &c->status, 1);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream);
        if (e != cudaSuccess) rc = fail(c, IGAPW_ERR_CUDA, std::string("status: ") + cudaGetErrorString(e));
    }
    if (!rc) rc = setup_all(c, nullptr, -1);
    if (!rc) rc = alloc_scratch(c);
    if (!rc) {
        // place the static scratch of igapw_rhs_source_noalloc on this device now
        // (its module is loaded on first use), so that entry point never has to
        void* p = nullptr;
        e = noalloc_scratch_address(&p);
        if (e != cudaSuccess) rc = fail(c, IGAPW_ERR_CUDA, std::string("static scratch: ") + cudaGetErrorString(e));
    }
    if (rc) {
        g_create_error = c->err;
        release(c);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        delete c;
        return rc;
    }
    *out = c;
    return IGAPW_OK;
}

int igapw_set_knots(igapw_ctx* c, int axis, const double* knots, int len) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (axis < 0 || axis >= c->dim || !knots || len <= 0) return fail(c, IGAPW_ERR_ARG, "bad axis or knots");
    CKC(c, cudaStreamSynchronize(c->stream));
    std::vector<double> kn(knots, knots + len);
    AxisSetup trial;
    std::string e = build_axis(trial, c->d.n_elem[axis], c->d.degree, c->d.nq, c->d.test, axis_bc(c->d, axis), kn,
                               c->d.refine);
    if (!e.empty()) return fail(c, IGAPW_ERR_ARG, e);
    // rebuild every axis (the padded window width is shared); keep other axes' knots
    std::vector<std::vector<double>> keep(3);
    for (int a = 0; a < c->dim; ++a) keep[a] = c->ax[a].knots;
    keep[axis] = kn;
    free_graphs(c);
    release(c);
    for (int a = 0; a < 3; ++a) {   // launch shapes are re-tuned
        c->step_cfg[a] = -1;
        c->step_pinned[a] = false;
    }
    CKC(c, dalloc(c, &c->status, 1));
    CKC(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    int wmax = 0, wqmax = 0;
    for (int a = 0; a < c->dim; ++a) {
        std::string err = build_axis(c->ax[a], c->d.n_elem[a], c->d.degree, c->d.nq, c->d.test, axis_bc(c->d, a), keep[a],
                                     c->d.refine);
        if (!err.empty()) return fail(c, IGAPW_ERR_ARG, err);
        wmax = std::max(wmax, c->ax[a].w);
        wqmax = std::max(wqmax, c->ax[a].wq);
    }
    c->W = pad_width(wmax);
    c->WQ = std::max(wqmax, 1);
    if (c->W < 0) return fail(c, IGAPW_ERR_ARG, "window too wide");
    for (int a = 0; a < c->dim; ++a)
        if (!set_window(c->ax[a], c->W)) return fail(c, IGAPW_ERR_ARG, "banded window layout failed");
    for (int a = 0; a < c->dim; ++a) set_chunks(c->ax[a], c->ntot / c->n[a]);
    for (int a = 0; a < c->dim; ++a) {
        int rc = build_axis_device(c, a);
        if (rc) return rc;
    }
    c->r = c->w = c->state = c->src0 = c->src1 = nullptr;
    c->u0 = c->rho = nullptr;
    c->src_bytes = 0;
    int rc = check_setup_status(c);
    if (rc) return rc;
    rc = build_fdm(c);
    if (rc) return rc;
    return alloc_scratch(c);
}

int igapw_quad_points(igapw_ctx* c, int axis, double* x, double* w, int* count) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (axis < 0 || axis >= c->dim || !count) return fail(c, IGAPW_ERR_ARG, "bad axis or count");
    const AxisSetup& s = c->ax[axis];
    *count = (int)s.qx.size();
    if (x) std::memcpy(x, s.qx.data(), s.qx.size() * sizeof(double));
    if (w) std::memcpy(w, s.qw.data(), s.qw.size() * sizeof(double));
    return IGAPW_OK;
}

int igapw_basis_table(igapw_ctx* c, int axis, double* vals, int* first_fn) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (axis < 0 || axis >= c->dim) return fail(c, IGAPW_ERR_ARG, "bad axis");
    const AxisSetup& s = c->ax[axis];
    if (vals) {
        CKC(c, cudaStreamSynchronize(c->stream));
        CKC(c, cudaMemcpy(vals, c->mem[axis].vals, s.qx.size() * (s.p + 1) * 3 * sizeof(double),
                          cudaMemcpyDeviceToHost));
    }
    if (first_fn) std::memcpy(first_fn, s.qfirst.data(), s.qfirst.size() * sizeof(int));
    return IGAPW_OK;
}

int igapw_rhs_source(igapw_ctx* c, const void* f_dev, void* b_dev) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!f_dev || !b_dev) return fail(c, IGAPW_ERR_ARG, "NULL tensor");
    SourceArgs a{};
    a.dim = c->dim;
    long long q[3] = {1, 1, 1};
    for (int k = 0; k < 3; ++k) {
        a.n[k] = c->n[k];
        a.q[k] = k < c->dim ? (int)c->ax[k].qx.size() : 1;
        q[k] = a.q[k];
        a.ax[k] = c->dev[k];
    }
    a.pw = c->d.test == IGAPW_PWCONST;
    // Galerkin intermediates: after the x pass (q_z q_y n_x), after the y pass (q_z n_y n_x)
    const size_t need = 8 * (size_t)std::max(q[2] * q[1] * c->n[0], q[2] * c->n[1] * c->n[0]);
    if (!a.pw && c->dim > 1 && c->src_bytes < need) {
        CKC(c, cudaStreamSynchronize(c->stream));
        unsigned char *b0 = nullptr, *b1 = nullptr;
        CKC(c, dalloc(c, &b0, need));
        CKC(c, dalloc(c, &b1, need));
        c->src0 = b0;
        c->src1 = b1;
        c->src_bytes = need;
    }
    a.f = f_dev;
    a.out = b_dev;
    a.work0 = c->src0;
    a.work1 = c->src1;
    a.ntot = c->ntot;
    cudaError_t e = launch_source(a, fp64(c), c->stream);
    if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("source: ") + cudaGetErrorString(e));
    return IGAPW_OK;
}

int igapw_rhs_source_sine(igapw_ctx* c, double amp, const double* k, void* b_dev) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!k || !b_dev) return fail(c, IGAPW_ERR_ARG, "NULL argument");
    SineSourceArgs a{};
    a.dim = c->dim;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = c->n[d];
        a.q[d] = d < c->dim ? (int)c->ax[d].qx.size() : 1;
        a.ax[d] = c->dev[d];
        a.qx[d] = d < c->dim ? c->mem[d].qx : nullptr;
        a.k[d] = d < c->dim ? k[d] : 0.0;
        a.v[d] = c->sine_v[d];
    }
    a.amp = amp;
    a.out = b_dev;
    a.ntot = c->ntot;
    cudaError_t e = launch_source_sine(a, fp64(c), c->stream);
    if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("sine source: ") + cudaGetErrorString(e));
    return IGAPW_OK;
}

int igapw_rhs_neumann(igapw_ctx* c, int axis, int side, const void* g_dev, void* b_dev) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!g_dev || !b_dev) return fail(c, IGAPW_ERR_ARG, "NULL tensor");
    if (axis < 0 || axis >= c->dim || !((c->d.neumann_axes >> axis) & 1))
        return fail(c, IGAPW_ERR_ARG, "axis is not a Neumann axis of this context");
    if (side != 0 && side != 1) return fail(c, IGAPW_ERR_ARG, "side must be 0 or 1");
    NeumannArgs a{};
    a.dim = c->dim;
    a.axis = axis;
    a.side = side;
    for (int k = 0; k < 3; ++k) {
        a.n[k] = c->n[k];
        a.q[k] = k < c->dim ? (int)c->ax[k].qx.size() : 1;
        a.ax[k] = c->dev[k];
    }
    a.g = g_dev;
    a.b = b_dev;
    a.ntot = c->ntot;
    cudaError_t e = launch_neumann(a, fp64(c), c->stream);
    if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("Neumann term: ") + cudaGetErrorString(e));
    return IGAPW_OK;
}

int igapw_apply(igapw_ctx* c, int op, double dt, const void* u_dev, void* r_dev) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!u_dev || !r_dev) return fail(c, IGAPW_ERR_ARG, "NULL tensor");
    if (u_dev == r_dev) return fail(c, IGAPW_ERR_ARG, "u and r must not overlap");
    switch (op) {
        case IGAPW_OP_MASS: return enqueue_apply(c, MODE_OP, 1.0, 0.0, u_dev, r_dev, c->stream);
        case IGAPW_OP_LAPLACE: return enqueue_apply(c, MODE_OP, 0.0, 1.0, u_dev, r_dev, c->stream);
        case IGAPW_OP_HEAT: return enqueue_apply(c, MODE_OP, 1.0, dt, u_dev, r_dev, c->stream);
        case IGAPW_OP_POISSON:
            if (c->d.op != IGAPW_OP_POISSON) return fail(c, IGAPW_ERR_ARG, "POISSON apply needs a POISSON context");
            if (c->fdm) {
                ContractArgs a = contract_args(c);
                a.u = u_dev;
                a.out = r_dev;
                a.alpha = 0.0;
                a.beta = -1.0;
                const int f = fp64(c) ? FMT_F64 : FMT_PAIR;
                cudaError_t e = launch_poisson_contract(a, MODE_PK, f, f, c->stream);
                if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("Poisson apply: ") + cudaGetErrorString(e));
                return IGAPW_OK;
            }
            return enqueue_apply(c, MODE_SYS, 1.0, 0.0, u_dev, r_dev, c->stream);
    }
    return fail(c, IGAPW_ERR_ARG, "unknown op");
}

int igapw_assemble_1d(igapw_ctx* c, int axis, int which, double* dense) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (axis < 0 || axis >= c->dim || !dense) return fail(c, IGAPW_ERR_ARG, "bad axis or output");
    const double* src = nullptr;
    if (which == IGAPW_OP_MASS) src = c->mem[axis].A;
    else if (which == IGAPW_OP_LAPLACE) src = c->mem[axis].C;
    else if (which == IGAPW_OP_POISSON && c->d.op == IGAPW_OP_POISSON) src = c->mem[axis].S;
    else return fail(c, IGAPW_ERR_ARG, "which must be MASS, LAPLACE or (POISSON context) POISSON");
    const int n = c->ax[axis].n, W = c->W;
    std::vector<double> win((size_t)n * W);
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemcpy(win.data(), src, win.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::memset(dense, 0, (size_t)n * n * sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int w = 0; w < W; ++w) {
            const int j = c->ax[axis].fstart[i] + w;
            if (j < n) dense[(size_t)i * n + j] = win[(size_t)i * W + w];
        }
    return IGAPW_OK;
}

int igapw_solve(igapw_ctx* c, const void* r_dev, void* u_dev) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!r_dev || !u_dev) return fail(c, IGAPW_ERR_ARG, "NULL tensor");
    if (c->fdm) {
        if (r_dev == u_dev) return fail(c, IGAPW_ERR_ARG, "the multi-D Poisson solve needs distinct r and u");
        float* rho = fp64(c) ? (float*)c->w : c->rho;
        std::string err;
        const int rc = fdm_solve(*c->fdm, contract_args(c), r_dev, u_dev, fp64(c), kPoissonRefineF64, rho, c->u0,
                                 (c->d.flags & IGAPW_FLAG_FP64_RESIDUAL) != 0, c->stream, err);
        if (rc) return fail(c, rc, "Poisson solve: " + err);
        return IGAPW_OK;
    }
    return enqueue_solve(c, r_dev, u_dev, c->stream);
}

int igapw_step(igapw_ctx* c, double dt, int nsteps, void* u_dev) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!u_dev || nsteps < 0) return fail(c, IGAPW_ERR_ARG, "bad arguments");
    if (c->d.op == IGAPW_OP_POISSON) return fail(c, IGAPW_ERR_ARG, "explicit steps need a mass-matrix context (op != POISSON)");
    if (nsteps == 0) return IGAPW_OK;
    bool untuned = false;
    for (int a = 0; a < c->dim; ++a) untuned = untuned || c->step_cfg[a] < 0;
    if (!(c->d.flags & IGAPW_FLAG_STEP_RHS_SOLVE) && untuned) {
        const int rc = tune_step(c, dt);
        if (rc) return rc;
    }
    // graphs of up to CHUNK steps, replayed
    const int CHUNK = 50;
    int left = nsteps;
    while (left > 0) {
        const int k = left < CHUNK ? left : CHUNK;
        cudaGraphExec_t exec = nullptr;
        for (auto& g : c->graphs)
            if (g.dt == dt && g.nsteps == k && g.u == u_dev) exec = g.exec;
        if (!exec) {
            CKC(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
            int rc = enqueue_steps(c, dt, k, u_dev, c->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
            if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
            CKC(c, e);
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CKC(c, e);
            if (c->graphs.size() >= 16) free_graphs(c);
            c->graphs.push_back({dt, k, u_dev, exec});
        }
        CKC(c, cudaGraphLaunch(exec, c->stream));
        left -= k;
    }
    return IGAPW_OK;
}

int igapw_set_step_shape(igapw_ctx* c, int axis, int kind, int lines) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (axis < 0 || axis >= c->dim) return fail(c, IGAPW_ERR_ARG, "axis out of range");
    if (kind < -1 || kind > 3) return fail(c, IGAPW_ERR_ARG, "unknown step kernel kind");
    if (kind >= 0 && (lines < 1 || lines > 32)) return fail(c, IGAPW_ERR_ARG, "lines per block must be 1..32");
    free_graphs(c);
    c->step_cfg[axis] = kind;
    c->step_nl[axis] = kind >= 0 ? lines : 0;
    c->step_pinned[axis] = kind >= 0;
    return IGAPW_OK;
}

int igapw_get_step_shape(igapw_ctx* c, int axis, int* kind, int* lines) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (axis < 0 || axis >= c->dim || !kind || !lines) return fail(c, IGAPW_ERR_ARG, "bad arguments");
    *kind = c->step_cfg[axis];
    *lines = c->step_nl[axis];
    return IGAPW_OK;
}

int igapw_step_host(igapw_ctx* c, double dt, int nsteps, void* u_host) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    if (!u_host) return fail(c, IGAPW_ERR_ARG, "NULL host buffer");
    const size_t bytes = fp64(c) ? (size_t)c->ntot * 8 : (size_t)c->ntot * 8;
    if (!c->state) {
        unsigned char* s = nullptr;
        CKC(c, dalloc(c, &s, bytes));
        c->state = s;
    }
    CKC(c, cudaMemcpyAsync(c->state, u_host, bytes, cudaMemcpyHostToDevice, c->stream));
    int rc = igapw_step(c, dt, nsteps, c->state);
    if (rc) return rc;
    CKC(c, cudaMemcpyAsync(u_host, c->state, bytes, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaStreamSynchronize(c->stream));
    return IGAPW_OK;
}

int igapw_sync_status(igapw_ctx* c) {
    if (!c) return fail(nullptr, IGAPW_ERR_ARG, "ctx is NULL");
    DeviceGuard dg_(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, IGAPW_ERR_CUDA, std::string("async error: ") + cudaGetErrorString(e));
    // debug builds: out-of-range accesses the kernels skipped
    unsigned nbad = 0;
    std::string first;
    for (BoundsReader rd : bounds_readers()) {
        const BoundsReport b = rd();
        if (b.count && first.empty())
            first = std::string(b.file) + ":" + std::to_string(b.line) + " index " + std::to_string(b.index) +
                    " limit " + std::to_string(b.limit);
        nbad += b.count;
    }
    if (nbad) return fail(c, IGAPW_ERR_DEVICE_STATUS, "bounds check: " + std::to_string(nbad) +
                                                          " out-of-range accesses skipped, first at " + first);
    unsigned st = 0;
    CKC(c, cudaMemcpy(&st, c->status, sizeof st, cudaMemcpyDeviceToHost));
    if (st) {
        unsigned z = 0;
        CKC(c, cudaMemcpy(c->status, &z, sizeof z, cudaMemcpyHostToDevice));
        if (st & STATUS_NONFINITE) return fail(c, IGAPW_ERR_DEVICE_STATUS, "a solve produced a non-finite value");
        if (st & STATUS_TC_TIMEOUT)
            return fail(c, IGAPW_ERR_TIMEOUT, "a tensor-core transform gave up waiting for its MMAs");
        return fail(c, IGAPW_ERR_DEVICE_STATUS, "device status " + std::to_string(st));
    }
    return IGAPW_OK;
}

int igapw_tc_gemm(int M, int N, int K, int batch, const float* A, long long sAm, long long sAk, long long bA,
                  const float* B, long long sBn, long long sBk, long long bB, float* D, long long sDm, long long sDn,
                  long long bD, int pre, int bn, int splits, void* cuda_stream) {
    g_create_error.clear();
    if (M <= 0 || N <= 0 || K <= 0 || batch <= 0 || !A || !B || !D || pre < 0 || pre > 2 ||
        (bn != 0 && bn != 64 && bn != 96 && bn != 128) || splits < 0 || splits > kTcMaxSplits ||
        splits > (K + 31) / 32 || (long long)batch * (splits > 1 ? splits : 1) > 65535) {
        g_create_error = "igapw_tc_gemm: need M, N, K, batch >= 1, non-NULL A, B, D, pre in {0, 1, 2}, bn in {0, 64, 96, "
                         "128}, splits in 0 .. min(4, ceil(K / 32)), batch x splits <= 65535";
        return IGAPW_ERR_ARG;
    }
    if (pre != 0 && batch != 1 && (pre == 1 ? bA : bB) != 0) {
        g_create_error = "igapw_tc_gemm: a pre-split operand is one matrix for every batch entry (its batch stride 0)";
        return IGAPW_ERR_ARG;
    }
    TcGemmArgs g{};
    g.M = M; g.N = N; g.K = K; g.batch = batch;
    g.A = A; g.sAm = sAm; g.sAk = sAk; g.bA = bA;
    g.B = B; g.sBn = sBn; g.sBk = sBk; g.bB = bB;
    g.D = D; g.sDm = sDm; g.sDn = sDn; g.bD = bD;
    g.pre = pre;
    g.bn = bn;
    g.splits = splits;
    const cudaError_t e = tc_gemm_entry(g, (cudaStream_t)cuda_stream);
    if (e == cudaErrorLaunchTimeout) {
        g_create_error = "igapw_tc_gemm: a pipeline wait of the kernel timed out";
        return IGAPW_ERR_TIMEOUT;
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("igapw_tc_gemm: ") + cudaGetErrorString(e);
        return e == cudaErrorInvalidValue ? IGAPW_ERR_ARG : IGAPW_ERR_CUDA;
    }
    return IGAPW_OK;
}

const char* igapw_last_error(igapw_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

long long igapw_size(igapw_ctx* c, int* dims) {
    if (!c) return -1;
    if (dims)
        for (int a = 0; a < 3; ++a) dims[a] = c->n[a];
    return c->ntot;
}

int igapw_destroy(igapw_ctx* c) {
    if (!c) return IGAPW_OK;
    DeviceGuard dg_(c->device);
    cudaStreamSynchronize(c->stream);
    release(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return IGAPW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Helpers for the allocation-free source entry point (noalloc.cu).  They fill
// the same launch arguments igapw_rhs_source uses, without touching the
// context's lazily allocated intermediates.
// ---------------------------------------------------------------------------
namespace igapw {

int source_setup(igapw_ctx* c, const void* f_dev, void* b_dev, SourceArgs& a, size_t& need,
                 cudaStream_t& st, bool& f64) {
    a = SourceArgs{};
    a.dim = c->dim;
    long long q[3] = {1, 1, 1};
    for (int k = 0; k < 3; ++k) {
        a.n[k] = c->n[k];
        a.q[k] = k < c->dim ? (int)c->ax[k].qx.size() : 1;
        q[k] = a.q[k];
        a.ax[k] = c->dev[k];
    }
    a.pw = c->d.test == IGAPW_PWCONST;
    need = (c->dim > 1 && !a.pw) ? 8 * (size_t)std::max(q[2] * q[1] * c->n[0], q[2] * c->n[1] * c->n[0]) : 0;
    a.f = f_dev;
    a.out = b_dev;
    a.ntot = c->ntot;
    st = c->stream;
    f64 = fp64(c);
    return IGAPW_OK;
}

int record_error(igapw_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }

int ctx_view(igapw_ctx* c, CtxView& v) {
    if (!c) return IGAPW_ERR_ARG;
    v.dim = c->dim;
    v.W = c->W;
    v.p = c->p;
    v.precision = c->d.precision;
    v.op = c->d.op;
    v.test = c->d.test;
    v.ntot = c->ntot;
    for (int a = 0; a < 3; ++a) {
        v.n[a] = c->n[a];
        v.ax[a] = c->dev[a];
        v.qx[a] = a < c->dim ? c->mem[a].qx : nullptr;
        v.q[a] = a < c->dim ? (int)c->ax[a].qx.size() : 1;
    }
    v.fdm = c->fdm;
    return IGAPW_OK;
}

}  // namespace igapw
