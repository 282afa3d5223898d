// Host orchestration and C-ABI of the GB300 HDG IMEX stage solver (include/hdg.h).
//
// Every step of the path runs in the kernels of hdg_kernels.cuh; the host only sequences
// launches on the context's stream and reads back solver scalars between chunks of Krylov
// iterations (convergence tests).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <exception>
#include <mutex>
#include <algorithm>
#include <chrono>
#include <thread>
#include <new>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hdg.h"
#include "hdg_kernels.cuh"
#include "hdg_mg_kernels.cuh"
#include "hdg_mg32.cuh"
#include "hdg_gs32.cuh"
#include "hdg_stage32.cuh"
#include "hdg_stage_f2.cuh"
#include "hdg_tracer.cuh"
#include "mesh.h"
#include "refelem.h"

using namespace hdg;

namespace {
thread_local std::string g_last_error;

struct CudaError : std::runtime_error {
    explicit CudaError(const std::string &s) : std::runtime_error(s) {}
};
struct OomError : std::runtime_error {
    explicit OomError(const std::string &s) : std::runtime_error(s) {}
};
struct TimeoutError : std::runtime_error {
    explicit TimeoutError(const std::string &s) : std::runtime_error(s) {}
};

#define CK(x)                                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) {                                                               \
            if (e_ == cudaErrorMemoryAllocation) throw OomError(cudaGetErrorString(e_));       \
            throw CudaError(std::string(#x) + ": " + cudaGetErrorString(e_));                  \
        }                                                                                      \
    } while (0)
#define CKL() CK(cudaGetLastError())

// IMEX tableaus (Alg. 1 form: stage 0 explicit, a_im[i][0] = b_im[0] = 0; the SSP tableaus of
// App. A have an implicit stage 0, see imex_step_body).
struct Tab {
    int s = 0;
    double Ae[4][4] = {}, Ai[4][4] = {}, be[4] = {}, bi[4] = {}, c[4] = {};
};

Tab make_tableau(int which) {
    Tab T;
    if (which == HDG_ARS222) {              // Ascher, Ruuth & Spiteri (1997), (2,2,2)
        double g = 1.0 - 1.0 / std::sqrt(2.0), d = 1.0 - 1.0 / (2.0 * g);
        T.s = 3;
        T.Ai[1][1] = g; T.Ai[2][1] = 1 - g; T.Ai[2][2] = g;
        T.Ae[1][0] = g; T.Ae[2][0] = d; T.Ae[2][1] = 1 - d;
        T.bi[1] = 1 - g; T.bi[2] = g;
        T.be[0] = d; T.be[1] = 1 - d;
        T.c[1] = g; T.c[2] = 1.0;
    } else if (which == HDG_ARS343) {       // ARS (3,4,3); gamma: root of 6g^3-18g^2+9g-1 in (0,1)
        double g = 0.4358665215;
        for (int it = 0; it < 8; ++it) g -= (6 * g * g * g - 18 * g * g + 9 * g - 1) / (18 * g * g - 36 * g + 9);
        double b1 = -1.5 * g * g + 4 * g - 0.25, b2 = 1.5 * g * g - 5 * g + 1.25;
        T.s = 4;
        T.Ai[1][1] = g;
        T.Ai[2][1] = (1 - g) / 2; T.Ai[2][2] = g;
        T.Ai[3][1] = b1; T.Ai[3][2] = b2; T.Ai[3][3] = g;
        T.Ae[1][0] = g;
        T.Ae[2][0] = 0.3212788860; T.Ae[2][1] = 0.3966543747;
        T.Ae[3][0] = -0.105858296; T.Ae[3][1] = 0.5529291479; T.Ae[3][2] = 0.5529291479;
        T.bi[1] = b1; T.bi[2] = b2; T.bi[3] = g;
        T.be[1] = b1; T.be[2] = b2; T.be[3] = g;
        T.c[1] = g; T.c[2] = (1 + g) / 2; T.c[3] = 1.0;
    } else if (which == HDG_IMEX_EULER) {   // App. A, IMEX Euler
        T.s = 2;
        T.Ai[1][1] = 1.0; T.Ae[1][0] = 1.0;
        T.bi[1] = 1.0; T.be[0] = 1.0;
        T.c[1] = 1.0;
    } else if (which == HDG_SSP2_332) {     // App. A, SSP2(3,3,2); explicit abscissae (0, 1/2, 1)
        T.s = 3;
        T.Ai[0][0] = 0.25; T.Ai[1][1] = 0.25;
        T.Ai[2][0] = T.Ai[2][1] = T.Ai[2][2] = 1.0 / 3.0;
        T.Ae[1][0] = 0.5; T.Ae[2][0] = 0.5; T.Ae[2][1] = 0.5;
        for (int i = 0; i < 3; ++i) T.bi[i] = T.be[i] = 1.0 / 3.0;
        T.c[1] = 0.5; T.c[2] = 1.0;
    } else if (which == HDG_SSP3_433) {     // App. A, SSP3(4,3,3)
        const double al = 0.24169426078821, be = 0.06042356519705, et = 0.12915286960590;
        const double de = 0.5 - al - be - et;
        T.s = 4;
        T.Ai[0][0] = al;
        T.Ai[1][0] = -al; T.Ai[1][1] = al;
        T.Ai[2][1] = 1.0 - al; T.Ai[2][2] = al;
        T.Ai[3][0] = be; T.Ai[3][1] = et; T.Ai[3][2] = de; T.Ai[3][3] = al;
        T.Ae[2][1] = 1.0; T.Ae[3][1] = 0.25; T.Ae[3][2] = 0.25;
        T.bi[1] = T.be[1] = 1.0 / 6.0; T.bi[2] = T.be[2] = 1.0 / 6.0; T.bi[3] = T.be[3] = 2.0 / 3.0;
        T.c[2] = 1.0; T.c[3] = 0.5;
    } else {
        throw std::invalid_argument("unknown tableau");
    }
    return T;
}

struct MGLevel {               // a P1 level of the trace multigrid (operator for one c)
    P1Grid G{};
    double *A = nullptr, *dinv = nullptr;
    double invth = 0, c1 = 0, c2 = 0;
};

struct CondCache {
    double c = 0;
    double *Scell = nullptr, *Zc = nullptr, *Ac = nullptr, *Sell = nullptr, *Dinv = nullptr;
    int *tcol = nullptr;
    // multigrid (empty: facet block-Jacobi CG)
    bool mg = false;
    cudaGraphExec_t g_setup = nullptr, g_chunk = nullptr;   // captured MG-CG setup / 8 iterations
    cudaGraphExec_t g_stage = nullptr;                      // whole stage solve, device-side loops
    int stage_kernels = 0;                                  // its kernels outside the loops
    double t_invth = 0, t_c1 = 0, t_c2 = 0;   // trace-level Chebyshev
    std::vector<MGLevel> lv;                  // lv[0] = level 1 (P1 on the mesh), ...
    double *Minv = nullptr;
    int Nc = 0;
    float *Lrhs32 = nullptr, *Lbs32 = nullptr;             // preconditioner Step-II maps (FP32)
    // FP32 copy of the multigrid for the preconditioner's one-V-cycle Step II (hdg_mg32.cuh)
    bool mg32 = false;
    float *Sell32 = nullptr, *Dinv32 = nullptr, *Minv32 = nullptr;
    std::vector<float *> A32, dinv32;
    size_t tail32_smem = 0;
    float *tail_img = nullptr;                // the tail's shared-memory image (dinv, stencils)
    int first32 = 0;                          // P1 levels >= first32 run in the one-block tail
};

struct MGWork {                // per-level work vectors (shared by all coefficients)
    double *b = nullptr, *xa = nullptr, *xb = nullptr, *d = nullptr, *t = nullptr;
};
struct MGWork32 {              // the same for the FP32 V-cycle
    float *b = nullptr, *xa = nullptr, *xb = nullptr, *d = nullptr, *t = nullptr;
};

void cheb_coefs(double lmax, double &invth, double &c1, double &c2) {
    // degree-2 Chebyshev on [lmax / 10, lmax]
    double lmin = lmax / 10.0, th = 0.5 * (lmax + lmin), de = 0.5 * (lmax - lmin);
    double sg = th / de, r0 = 1.0 / sg, r1 = 1.0 / (2.0 * sg - r0);
    invth = 1.0 / th;
    c1 = r0 * r1;
    c2 = 2.0 * r1 / de;
}
}  // namespace

struct hdg_ctx {
    hdg_params P{};
    hdg_mesh_desc D{};
    cudaStream_t st = nullptr;
    int device = 0;                                          // CUDA device current at setup
    RefTables T;
    HostMesh H;
    int K = 0, MU = 0, NU = 0, NP = 0, NT = 0, NL = 0;
    long long ncells = 0, nfacets = 0, nQ = 0, nPv = 0, nL = 0;
    double area = 1.0;
    Tab tab;
    // device allocations (freed in hdg_destroy)
    std::vector<void *> allocs;
    double *dref = nullptr;
    RefDev R{};
    MeshDev M{};
    CellGeo *geo = nullptr;
    // state (modal)
    double *Q = nullptr, *p = nullptr, *lam = nullptr;
    double t = 0.0;
    // IMEX stages
    std::vector<double *> Qs, rs, ps, ls;
    // initial guesses of the stage solves (stage_guesses): the last step's stage solutions (HQs,
    // Hps, Hls), the pressure and trace ones of the step before (H2ps, H2ls), the velocity at the
    // last step's start (Qprev) and end (Qlast), and a device count of the steps kept (0..2)
    std::vector<double *> HQs, Hps, Hls, H2ps, H2ls;
    double *Qprev = nullptr, *Qlast = nullptr;
    int *dhist = nullptr;
    unsigned long long *dcheck = nullptr;                    // max |Q - Qlast|, max |Qlast| (bits)
    // forcing
    double *Fload = nullptr;
    bool has_forcing = false;
    // time factors of the forcing for one step (stage sums 1..s-1, final sum s, reconstruction 7):
    // device copy read by the step graph, pinned host staging refreshed before each launch
    double *dfv = nullptr, *hfv = nullptr;
    double (*phi)(double, void *) = nullptr;
    void *phi_user = nullptr;
    // passive tracer (App. B): state (modal DG_k), stage values / derivatives, advecting velocity
    bool has_tracer = false;
    double *qtr = nullptr, *tr_q = nullptr, *tr_dq[4] = {}, *tr_U = nullptr;
    // continuous space CG_{k+1} for P_CG: numbering, Jacobi diagonal, Krylov vectors ([d][point])
    CGMap cgm{};
    double *cg_b = nullptr, *cg_u = nullptr, *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_Ap = nullptr,
           *cg_w = nullptr;
    // Step I
    double *Dblk = nullptr, *Binv = nullptr, *wq = nullptr, *utr = nullptr;
    double *pen = nullptr;                                   // -c alpha fw_q of the assembled operator
    int inv_ok = 0;                                          // inverses of the assembly: INV64 | INV32
    int trace_vcycles = 0;                                   // > 0: trace solves are that many V-cycles
    // FP32 copies for the loose (inner) Step-I solves: tables, block inverses, weights, GMRES work
    float *ephi32 = nullptr, *pen32 = nullptr, *Binv32 = nullptr, *wq32 = nullptr, *utr32 = nullptr;
    float *nrm32 = nullptr;                                  // cell normals in FP32 [6 cell + 2 e + d]
    // relaxed (FP32) stage-operator products: diagonal blocks, geometry, reference tables
    float *Dblk32 = nullptr, *geo32 = nullptr, *Dhat32 = nullptr, *Ehat32 = nullptr;
    float *Tadv2 = nullptr;                                  // advection tensor: FP32 hi plane, lo plane
    float2 *ephi2a = nullptr, *Sfac2 = nullptr;              // facet values, facet masses as pairs
    float2 *fw2 = nullptr, *leg2 = nullptr, *Iv2 = nullptr, *bdminv2 = nullptr;   // BDM tables as pairs
    // pair-arithmetic stage operator (HDG_MIXED, k_stage_apply_f2): the blocks' rest after their
    // FP32 rounding, the reference tables as pairs; blk32_ok: Dblk32 / Dblk32lo hold the
    // operator last assembled
    float *Dblk32lo = nullptr;
    float2 *ephi2 = nullptr, *Ehat2 = nullptr, *Dhat2 = nullptr;
    bool blk32_ok = false;
    bool gs_ok = false;                                      // cells 2-coloured by index parity (hdg_gs32.cuh)
    float *gV32 = nullptr, *gw32 = nullptr, *gu32 = nullptr;
    cudaGraphExec_t g_stepI32 = nullptr;                     // one loose Step-I solve (host-driven mode)
    int stepI32_kernels = 0;
    int *dstatus = nullptr;
    // Step II
    double *vK = nullptr, *wK = nullptr, *tb = nullptr, *tx = nullptr, *tr = nullptr, *tz = nullptr,
           *tp[2] = {nullptr, nullptr}, *tAp = nullptr;
    // GMRES (Step I)
    double *gV = nullptr, *gw = nullptr, *gz = nullptr, *gu = nullptr;
    GmresState *gs = nullptr, *hgs = nullptr;
    // flexible GMRES on the stage system (vectors of nQ + np + nlambda)
    double *fV = nullptr, *fZ = nullptr, *fx = nullptr, *fb = nullptr, *fw = nullptr, *fr = nullptr, *fu = nullptr;
    float *fV32 = nullptr, *fw32 = nullptr;                  // FP32 shadows of the basis and of w
    double *fv = nullptr, *fz = nullptr;                     // preconditioner input / output (fixed)
    GmresState *fgs = nullptr, *hfgs = nullptr;
    // temporaries
    double *q[8] = {};
    double *pp[3] = {};
    double *ll[3] = {};
    // multigrid work
    std::vector<MGWork> mgw;
    std::vector<MGWork32> mgw32;
    double *txa = nullptr, *td = nullptr, *tt = nullptr, *cellA = nullptr, *mgB = nullptr;
    float *tb32 = nullptr, *tr32 = nullptr, *tx32 = nullptr, *txa32 = nullptr, *td32 = nullptr;
    double *tzold = nullptr;                                 // flexible CG: the previous z
    unsigned long long *dlmax = nullptr;
    // reductions
    double *partials = nullptr;
    unsigned *counter = nullptr;
    Scalars *sc = nullptr;
    Scalars *hsc = nullptr;     // pinned host mirror
    std::deque<CondCache> cache;
    cudaEvent_t e0 = nullptr, e1 = nullptr, te0 = nullptr, te1 = nullptr;
    cudaStream_t cap = nullptr;                              // capture stream for CUDA graphs
    static constexpr int CAP_LEVELS = 8;
    cudaStream_t capst[CAP_LEVELS] = {};                     // capture streams of nested loop bodies
    int cap_level = 0;                                       // nesting depth of the current capture
    bool capturing = false;
    int *dguard = nullptr;                                   // loop guards, one per nesting level
    static constexpr int MAX_LOOPS = 512;
    int *dnk = nullptr;                                      // kernels per pass of each recorded loop
    int nloops = 0;
    std::vector<int> nk_host;                                // host copy of dnk
    DevCount *dcnt = nullptr, *hcnt = nullptr;               // device-side counters (+ pinned mirror)
    cudaGraphExec_t g_step = nullptr;                        // one IMEX step (device-side loops)
    int step_kernels = 0;                                    // kernels of g_step outside its loops
    cudaGraphExec_t gm_first = nullptr, gm_restart = nullptr;   // captured GMRES(30) cycles
    double *gb = nullptr, *gx = nullptr;                     // their fixed right-hand side / solution
    // hdg_params.timeout_ms: the host's wait for a step graph is bounded; a step whose wait ran out
    // is still queued on the stream, and its bookkeeping (time, counters) is applied by the next call
    double deadline = 0;                                     // steady-clock ms; 0: no limit on this wait
    bool pending = false;                                    // a timed-out step is still on the stream
    double pending_t = 0;
    cudaEvent_t ewait = nullptr;                             // marks the end of the step being waited for
    int *hstat = nullptr;                                    // pinned copy of dstatus
    // running stats of the current call
    hdg_stats S{};

    template <class T_>
    T_ *alloc(size_t n) {
        void *p_ = nullptr;
        const size_t b_ = n * sizeof(T_) > 0 ? n * sizeof(T_) : 16;
        CK(cudaMalloc(&p_, b_));
        allocs.push_back(p_);
        bytes += b_;
        return (T_ *)p_;
    }
    size_t bytes = 0;                                        // device bytes allocated by alloc()
    RedBuf rb() const { return RedBuf{partials, counter}; }
};

namespace {

// HDG_TRACE_CG=1 in the environment: print the trace CG's scalars after every iteration (stderr)
bool trace_cg_enabled() {
    static int on = -1;
    if (on < 0) {
        const char *e = std::getenv("HDG_TRACE_CG");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on == 1;
}

// ------------------------------------------------------------------ helpers
void read_scalars(hdg_ctx *c) {
    CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
}

int grid_for(long long n) { return red_grid(n); }

// Kernel launch with programmatic stream serialisation (programmatic dependent launch): the
// kernel may start while its predecessor on the stream drains; the kernel's first statement
// (wait_prior_kernel) waits for the predecessor's completion. Works on plain streams and under
// stream capture (graph edges become programmatic).
template <class... KArgs, class... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Krylov orthogonalisation kernels: at most four blocks per SM, several rows per thread
int g_num_sms = 0;
int grid_orth(long long n) {
    if (!g_num_sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            g_num_sms = v;
        if (g_num_sms <= 0) g_num_sms = 152;
    }
    const int g = red_grid(n);
    return g < 4 * g_num_sms ? g : 4 * g_num_sms;
}

// per-cell team kernels: 128 threads = TEAMS_PER_BLOCK teams of TEAM_LANES lanes
constexpr int TEAMS_PER_BLOCK = 128 / TEAM_LANES;
inline unsigned cell_blocks(const hdg_ctx *c) { return (unsigned)((c->ncells + TEAMS_PER_BLOCK - 1) / TEAMS_PER_BLOCK); }

// thread-per-facet trace kernels use small blocks so that a few thousand facets still spread
// over all SMs
constexpr int FACET_THREADS = 64;
inline int grid_facets(long long nf) { return (int)((nf + FACET_THREADS - 1) / FACET_THREADS); }

// Component timer: events around one component on the context's stream; the elapsed time is
// added to a hdg_stats bucket when the component ends (each component ends with a host sync).
// Inside a graph capture the timer does nothing.
struct CompTimer {
    hdg_ctx *c;
    double *bucket;
    CompTimer(hdg_ctx *c_, double *b) : c(c_), bucket(b) {
        if (c->capturing) bucket = nullptr;
        else CK(cudaEventRecord(c->te0, c->st));
    }
    ~CompTimer() noexcept(false) {
        if (!bucket || std::uncaught_exceptions()) return;
        CK(cudaEventRecord(c->te1, c->st));
        CK(cudaEventSynchronize(c->te1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, c->te0, c->te1));
        *bucket += ms;
    }
};

// Record the launches issued by f (on c->st, temporarily the capture stream) into a graph.
// kernel nodes of a graph, not counting the bodies of its conditional nodes
int count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    CK(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) CK(cudaGraphGetNodes(g, nodes.data(), &n));
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

template <class F>
cudaGraphExec_t capture_graph(hdg_ctx *c, F &&f, int *nkernels = nullptr) {
    cudaStream_t user = c->st;
    c->st = c->cap;
    c->capturing = true;
    c->cap_level = 0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        try {
            f();
        } catch (...) {
            cudaStreamEndCapture(c->cap, &g);
            if (g) cudaGraphDestroy(g);
            c->st = user;
            c->capturing = false;
            throw;
        }
        e = cudaStreamEndCapture(c->cap, &g);
    }
    c->st = user;
    c->capturing = false;
    CK(e);
    if (nkernels) *nkernels = count_kernel_nodes(g);
    // kernels per pass of the loops recorded in this capture
    CK(cudaMemcpy(c->dnk, c->nk_host.data(), sizeof(int) * c->nloops, cudaMemcpyHostToDevice));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return ex;
}

// Inside a capture on c->st: append a device-side while loop (a conditional graph node).
// init(L) launches, on c->st, the kernel that sets the loop's first condition; the body is
// recorded from body(L) on the next nesting level's stream into the node's body graph and must
// end with a kernel that sets the condition for the next pass (k_loop_ctl or k_gm_loop_ctl).
template <class Init, class Body>
void capture_while(hdg_ctx *c, Init &&init, Body &&body) {
    if (!c->capturing) throw std::logic_error("capture_while outside a graph capture");
    const int lev = c->cap_level + 1;
    if (lev >= hdg_ctx::CAP_LEVELS) throw std::logic_error("device loops nested too deeply");
    if (c->nloops >= hdg_ctx::MAX_LOOPS) throw std::logic_error("too many device loops recorded");
    const int id = c->nloops++;
    c->nk_host.resize(c->nloops, 0);
    cudaStream_t s = c->st;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    LoopCtl L{};
    CK(cudaGraphConditionalHandleCreate(&L.h, g, 0, 0));
    L.guard = c->dguard + lev;
    L.nk = c->dnk + id;
    L.launches = &c->dcnt->launches;
    init(L);
    CKL();
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = L.h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    if (!c->capst[lev]) CK(cudaStreamCreateWithFlags(&c->capst[lev], cudaStreamNonBlocking));
    cudaStream_t bs = c->capst[lev];
    CK(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->st = bs;
    c->cap_level = lev;
    cudaGraph_t outg = nullptr;
    try {
        body(L);
        CKL();
    } catch (...) {
        cudaStreamEndCapture(bs, &outg);
        c->st = s;
        c->cap_level = lev - 1;
        throw;
    }
    c->st = s;
    c->cap_level = lev - 1;
    CK(cudaStreamEndCapture(bs, &outg));
    c->nk_host[id] = count_kernel_nodes(bodyg);
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
}

inline LinComb lincomb() {
    LinComb L{};
    L.fterm = -1;
    return L;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Wait for the work queued on the context's stream; with a deadline, poll an event until it has
// passed and then throw TimeoutError (the work stays queued and completes on the stream).
void wait_stream(hdg_ctx *c) {
    if (!(c->deadline > 0)) {
        CK(cudaStreamSynchronize(c->st));
        return;
    }
    CK(cudaEventRecord(c->ewait, c->st));
    for (;;) {
        cudaError_t e = cudaEventQuery(c->ewait);
        if (e == cudaSuccess) return;
        if (e != cudaErrorNotReady) CK(e);
        if (now_ms() > c->deadline) {
            char msg[160];
            snprintf(msg, sizeof msg, "the step's GPU work did not finish within timeout_ms = %.3f; it completes on "
                                      "the context's stream", c->P.timeout_ms);
            throw TimeoutError(msg);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// The continuous space of P_CG (App. B), set up on first use (outside graph captures)
void ensure_cg(hdg_ctx *c) {
    if (c->cg_b) return;
    if (c->capturing) throw std::logic_error("continuous space set up inside a graph capture");
    const CGNumbering N = build_cg_numbering(c->H, c->K + 1);
    const int nl = N.nl;
    std::vector<double> dinv(N.npts, 0.0);
    for (int pt = 0; pt < N.npts; ++pt) {
        double dsum = 0.0;
        for (int e = N.node_ptr[pt]; e < N.node_ptr[pt + 1]; ++e) {
            const int ent = N.node_list[e], cell = ent / nl, l = ent % nl;
            double s = 0.0;
            for (int a = 0; a < nl; ++a) s += c->T.nod_u[a * nl + l] * c->T.nod_u[a * nl + l];
            dsum += c->H.geo[cell].detJ * s;
        }
        dinv[pt] = 1.0 / dsum;
    }
    int *gid = c->alloc<int>(N.cell_gid.size()), *ptr = c->alloc<int>(N.node_ptr.size()),
        *lst = c->alloc<int>(N.node_list.size());
    double *dv = c->alloc<double>(N.npts);
    CK(cudaMemcpy(gid, N.cell_gid.data(), N.cell_gid.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ptr, N.node_ptr.data(), N.node_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(lst, N.node_list.data(), N.node_list.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dv, dinv.data(), dinv.size() * sizeof(double), cudaMemcpyHostToDevice));
    c->cgm = CGMap{gid, ptr, lst, dv, N.npts, nl, (int)c->ncells};
    const size_t n2 = 2 * (size_t)N.npts;
    c->cg_u = c->alloc<double>(n2); c->cg_r = c->alloc<double>(n2); c->cg_z = c->alloc<double>(n2);
    c->cg_p = c->alloc<double>(n2); c->cg_Ap = c->alloc<double>(n2);
    c->cg_w = c->alloc<double>((size_t)c->ncells * 2 * nl);
    c->cg_b = c->alloc<double>(n2);
    CK(cudaMemset(c->cg_p, 0, n2 * sizeof(double)));
}

// Buffers of the tracer (one DG_k field and its stage values)
void ensure_tracer_buffers(hdg_ctx *c) {
    ensure_cg(c);
    if (c->qtr) return;
    c->qtr = c->alloc<double>(c->nPv);
    c->tr_q = c->alloc<double>(c->nPv);
    for (auto &x : c->tr_dq) x = c->alloc<double>(c->nPv);
    c->tr_U = c->alloc<double>(c->nQ);
}

template <int K>
struct Impl {
    typedef Dims<K> Dm;
    static constexpr int MU = Dm::MU, NU = Dm::NU, NP = Dm::NP, NT = Dm::NT, NL = Dm::NL, K_ = K;

    static void to_modal(hdg_ctx *c, const double *nodal, double *modal, int kind) {
        // kind 0: velocity, 1: pressure, 2: trace
        const double *Tm = kind == 0 ? c->R.nod_u : kind == 1 ? c->R.nod_p : c->R.nod_t;
        int n = kind == 0 ? MU : kind == 1 ? NP : NT;
        long long nvec = kind == 0 ? 2 * c->ncells : kind == 1 ? c->ncells : c->nfacets;
        launch_k(k_basis_change, grid_for(nvec * n), VEC_THREADS, 0, c->st, Tm, n, nodal, modal, nvec);
        CKL();
    }
    static void to_nodal(hdg_ctx *c, const double *modal, double *nodal, int kind) {
        const double *Tm = kind == 0 ? c->R.mod_u : kind == 1 ? c->R.mod_p : c->R.mod_t;
        int n = kind == 0 ? MU : kind == 1 ? NP : NT;
        long long nvec = kind == 0 ? 2 * c->ncells : kind == 1 ? c->ncells : c->nfacets;
        launch_k(k_basis_change, grid_for(nvec * n), VEC_THREADS, 0, c->st, Tm, n, modal, nodal, nvec);
        CKL();
    }
    static void mass(hdg_ctx *c, const double *in, double *out, int mode) {
        launch_k(k_mass_scale, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, NU, in, out, c->ncells, mode);
        CKL();
    }

    // ---------------------------------------------------------------- condensation cache
    static CondCache &condense(hdg_ctx *c, double cc) {
        for (auto &e : c->cache)
            if (e.c == cc) return e;
        if (c->capturing) throw std::logic_error("condensation for a new coefficient inside a graph capture");
        CondCache E;
        E.c = cc;
        E.Scell = c->alloc<double>((size_t)c->ncells * NL * NL);
        E.Zc = c->alloc<double>((size_t)c->ncells * NP * NL);
        E.Ac = c->alloc<double>((size_t)c->ncells * NP * NP);
        E.Sell = c->alloc<double>((size_t)5 * NT * c->nL);
        E.tcol = c->alloc<int>((size_t)5 * c->nfacets);
        E.Dinv = c->alloc<double>((size_t)NT * c->nL);
        size_t smem = sizeof(double) * (NP * NU + NL * NU + 2 * NP * NP + 2 * NP * NL + NL * NL);
        CK(cudaFuncSetAttribute(k_condense<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch_k(k_condense<K>, (unsigned)c->ncells, 128, smem, c->st, c->R, c->M, cc, c->P.tau, E.Scell, E.Zc, E.Ac);
        CKL();
        launch_k(k_assemble_trace<NT>, grid_for(c->nfacets), VEC_THREADS, 0, c->st, c->M, E.Scell, E.Sell, E.tcol, E.Dinv);
        CKL();
        if (c->P.trace_mg && c->H.p1_ok) build_mg(c, E);
        if (E.mg && (c->P.inner_trace_fp32 || c->P.trace_fp32_vcycle)) build_mg32(c, E);
        c->cache.push_back(E);
        return c->cache.back();
    }

    // multigrid hierarchy of the trace operator for one coefficient (hdg_mg.cuh)
    static void build_mg(hdg_ctx *c, CondCache &E) {
        std::vector<P1Grid> grids;
        int nl = c->H.n;
        grids.push_back(make_p1grid(nl, c->H.px, c->H.py));
        while (nl % 2 == 0 && nl / 2 >= 4) {
            nl /= 2;
            grids.push_back(make_p1grid(nl, c->H.px, c->H.py));
        }
        const int Nc = grids.back().nverts;
        if (Nc > 1024) return;                                   // coarsest too large: block-Jacobi CG
        const int L = (int)grids.size();
        if (c->mgw.empty()) {
            for (int l = 0; l < L; ++l) {
                MGWork w;
                size_t n = grids[l].nverts;
                w.b = c->alloc<double>(n); w.xa = c->alloc<double>(n); w.xb = c->alloc<double>(n);
                w.d = c->alloc<double>(n); w.t = c->alloc<double>(n);
                c->mgw.push_back(w);
            }
            c->txa = c->alloc<double>(c->nL); c->td = c->alloc<double>(c->nL); c->tt = c->alloc<double>(c->nL);
            c->cellA = c->alloc<double>((size_t)9 * c->ncells);
            c->mgB = c->alloc<double>((size_t)Nc * Nc);
            c->dlmax = c->alloc<unsigned long long>(16);
        }
        E.lv.resize(L);
        for (int l = 0; l < L; ++l) {
            E.lv[l].G = grids[l];
            E.lv[l].A = c->alloc<double>((size_t)P1_NS * grids[l].nverts);
            E.lv[l].dinv = c->alloc<double>(grids[l].nverts);
        }
        E.Minv = c->alloc<double>((size_t)Nc * Nc);
        E.Nc = Nc;
        CK(cudaMemsetAsync(c->dlmax, 0, 16 * sizeof(unsigned long long), c->st));
        launch_k(k_p1_cellop<NT>, grid_for(c->ncells), VEC_THREADS, 0, c->st, E.Scell, c->M.cell_flip, (int)c->ncells, c->cellA);
        launch_k(k_p1_assemble, grid_for(grids[0].nverts), VEC_THREADS, 0, c->st, grids[0], c->cellA, c->M.vert_cell,
                                                                         c->M.cell_vert, E.lv[0].A, E.lv[0].dinv,
                                                                         c->dlmax + 1);
        for (int l = 1; l < L; ++l)
            launch_k(k_p1_coarsen, grid_for(grids[l].nverts), VEC_THREADS, 0, c->st, grids[l], grids[l - 1], E.lv[l - 1].A,
                                                                             E.lv[l].A, E.lv[l].dinv, c->dlmax + 1 + l);
        launch_k(k_trace_bound<NT>, grid_for(c->nfacets), VEC_THREADS, 0, c->st, E.Sell, E.tcol, E.Dinv, (int)c->nfacets,
                                                                          c->dlmax);
        CK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->st));
        launch_k(k_coarse_inverse, 1, 1024, 0, c->st, grids[L - 1], E.lv[L - 1].A, c->mgB, E.Minv, c->dstatus);
        CKL();
        unsigned long long bits[16];
        int st = 0;
        CK(cudaMemcpyAsync(bits, c->dlmax, sizeof bits, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(&st, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (st) throw std::domain_error("multigrid: singular coarsest operator");
        double lm;
        std::memcpy(&lm, &bits[0], sizeof lm);
        cheb_coefs(lm, E.t_invth, E.t_c1, E.t_c2);
        for (int l = 0; l < L; ++l) {
            std::memcpy(&lm, &bits[1 + l], sizeof lm);
            cheb_coefs(lm, E.lv[l].invth, E.lv[l].c1, E.lv[l].c2);
        }
        E.mg = true;
    }

    // Parameters of the fused coarse part of the V-cycle, from level `first` down
    static MGTail tail_params(hdg_ctx *c, const CondCache &E, int first, const double *tres, double *z) {
        MGTail T{};
        T.first = first;
        T.L = (int)E.lv.size();
        T.Nc = E.Nc;
        T.nfacets = (int)c->nfacets;
        for (int l = 0; l < T.L; ++l) {
            T.G[l] = E.lv[l].G; T.A[l] = E.lv[l].A; T.dinv[l] = E.lv[l].dinv;
            T.invth[l] = E.lv[l].invth; T.c1[l] = E.lv[l].c1; T.c2[l] = E.lv[l].c2;
            T.b[l] = c->mgw[l].b; T.xa[l] = c->mgw[l].xa; T.xb[l] = c->mgw[l].xb; T.d[l] = c->mgw[l].d; T.t[l] = c->mgw[l].t;
        }
        T.Minv = E.Minv;
        T.vert_facet = c->M.vert_facet; T.vert_fsign = c->M.vert_fsign; T.facet_vert = c->M.facet_vert;
        T.tres = tres;
        T.z = z;
        return T;
    }

    // P1 levels with more vertices than this run as separate grid-wide kernels; the smaller ones
    // share one block (HDG_MG_FUSE_MAX overrides the default)
    static int mg_fuse_max() {
        static int v = -1;
        if (v < 0) {
            const char *e = std::getenv("HDG_MG_FUSE_MAX");
            v = e ? std::atoi(e) : 300;
            if (v < 0) v = 0;
        }
        return v;
    }

    // Middle of the V-cycle: from the trace residual tt, correct z0 through the P1 hierarchy
    static void vcycle_p1(hdg_ctx *c, const CondCache &E, double *z0) {
        const int nf = (int)c->nfacets, L = (int)E.lv.size();
        Scalars *sc = c->sc;
        int first = 0;
        while (first < L - 1 && E.lv[first].G.nverts > mg_fuse_max()) ++first;
        if (first > 0)
            launch_k(k_restrict_t<NT>, grid_for(E.lv[0].G.nverts), VEC_THREADS, 0, c->st, E.lv[0].G.nverts, c->tt,
                                                                                  c->M.vert_facet, c->M.vert_fsign,
                                                                                  c->mgw[0].b, sc);
        for (int l = 0; l < first; ++l) {
            const MGLevel &V = E.lv[l];
            const MGWork &W = c->mgw[l];
            const int g = grid_for(V.G.nverts);
            launch_k(k_pcheb0, g, VEC_THREADS, 0, c->st, V.dinv, W.b, W.xa, W.d, V.invth, V.G.nverts, sc);
            launch_k(k_pcheb, g, VEC_THREADS, 0, c->st, V.G, V.A, V.dinv, W.b, W.xa, W.xb, W.d, V.c1, V.c2, sc);
            launch_k(k_presid, g, VEC_THREADS, 0, c->st, V.G, V.A, W.b, W.xb, W.t, sc);
            launch_k(k_prestrict, grid_for(E.lv[l + 1].G.nverts), VEC_THREADS, 0, c->st, E.lv[l + 1].G, V.G, W.t,
                                                                                   c->mgw[l + 1].b, sc);
        }
        launch_k(k_mg_tail<NT>, 1, 1024, 0, c->st, tail_params(c, E, first, c->tt, z0), sc);
        for (int l = first - 1; l >= 0; --l) {
            const MGLevel &V = E.lv[l];
            const MGWork &W = c->mgw[l];
            const int g = grid_for(V.G.nverts);
            launch_k(k_pprolong, g, VEC_THREADS, 0, c->st, V.G, E.lv[l + 1].G, c->mgw[l + 1].xb, W.xb, sc);
            launch_k(k_pcheb, g, VEC_THREADS, 0, c->st, V.G, V.A, V.dinv, W.b, W.xb, W.xa, W.d, 0.0, V.invth, sc);
            launch_k(k_pcheb, g, VEC_THREADS, 0, c->st, V.G, V.A, V.dinv, W.b, W.xa, W.xb, W.d, V.c1, V.c2, sc);
        }
        if (first > 0)
            launch_k(k_prolong_t<NT>, grid_for(nf), VEC_THREADS, 0, c->st, c->M.facet_vert, c->mgw[0].xb, z0, nf, sc);
    }

    // z0 = V-cycle(r0); with fused_start the first Chebyshev step (txa = d = Dinv r0 / theta) has
    // already been done by the CG update kernel; with rz_first >= 0 the last smoothing step also
    // performs the CG reduction (k_tcheb_rz).
    static void vcycle(hdg_ctx *c, const CondCache &E, const double *r0, double *z0, bool fused_start = false,
                       int rz_first = -1) {
        const int nf = (int)c->nfacets;
        const int gf = grid_facets(nf), gr = grid_for(c->nL);
        Scalars *sc = c->sc;
        if (!fused_start) launch_k(k_tcheb0<NT>, gf, FACET_THREADS, 0, c->st, E.Dinv, r0, c->txa, c->td, E.t_invth, nf, sc);
        launch_k(k_tcheb<NT>, gf, FACET_THREADS, 0, c->st, E.Sell, E.tcol, E.Dinv, r0, c->txa, z0, c->td, E.t_c1, E.t_c2, nf, sc);
        launch_k(k_tresid<NT>, gr, VEC_THREADS, 0, c->st, E.Sell, E.tcol, r0, z0, c->tt, nf, sc);
        vcycle_p1(c, E, z0);
        launch_k(k_tcheb<NT>, gf, FACET_THREADS, 0, c->st, E.Sell, E.tcol, E.Dinv, r0, z0, c->txa, c->td, 0.0, E.t_invth, nf, sc);
        if (rz_first < 0)
            launch_k(k_tcheb<NT>, gf, FACET_THREADS, 0, c->st, E.Sell, E.tcol, E.Dinv, r0, c->txa, z0, c->td, E.t_c1, E.t_c2, nf, sc);
        else
            launch_k(k_tcheb_rz<NT>, gf, FACET_THREADS, 0, c->st, E.Sell, E.tcol, E.Dinv, r0, c->txa, z0, c->td, E.t_c1, E.t_c2, nf,
                                                           rz_first, c->rb(), sc);
    }

    // ---------------------------------------------------------------- trace CG: S x = b
    static void trace_solve(hdg_ctx *c, CondCache &E, const double *b, double *x, double rtol) {
        const int nf = (int)c->nfacets;
        if (E.mg) { trace_solve_mg(c, E, b, x, rtol); return; }
        launch_k(k_trace_mean<NT>, grid_for(nf), VEC_THREADS, 0, c->st, b, nf, c->rb(), c->sc);
        CKL();
        launch_k(k_cg_setup<NT>, grid_for(nf), VEC_THREADS, 0, c->st, b, E.Dinv, x, c->tr, c->tz, c->tp[0], nf, c->rb(),
                                                               c->sc, rtol, c->P.max_iters);
        CKL();
        const int gr = grid_for(c->nL), gf = grid_for(nf);
        if (c->capturing) {             // device-side loop, two iterations per pass
            capture_while(
                c, [&](LoopCtl L) { launch_k(k_loop_init, 1, 1, 0, c->st, L, &c->sc->done); },
                [&](LoopCtl L) {
                    for (int m = 0; m < 2; ++m) {
                        double *pold = c->tp[m & 1], *pnew = c->tp[(m + 1) & 1];
                        launch_k(k_cg_apply<NT>, cg_apply_grid<NT>(nf), 128, 0, c->st, E.Sell, E.tcol, c->tz, pold, pnew, c->tAp, nf,
                                                                     c->rb(), c->sc);
                        launch_k(k_cg_update<NT>, gf, VEC_THREADS, 0, c->st, E.Dinv, pnew, c->tAp, x, c->tr, c->tz, nf,
                                                                      c->rb(), c->sc);
                    }
                    launch_k(k_loop_ctl, 1, 1, 0, c->st, L, c->P.max_iters / 2 + 2, &c->sc->done);
                });
            launch_k(k_count_solve, 1, 1, 0, c->st, c->dcnt, nullptr, c->sc);
            CKL();
            return;
        }
        const int chunk = trace_cg_enabled() ? 2 : 16;
        for (long long launched = 0;; launched += chunk) {
            if (launched > (long long)c->P.max_iters + 2 * chunk)
                throw std::length_error("trace CG: no convergence flag from the device");
            for (int m = 0; m < chunk; ++m) {
                double *pold = c->tp[m & 1], *pnew = c->tp[(m + 1) & 1];
                launch_k(k_cg_apply<NT>, cg_apply_grid<NT>(nf), 128, 0, c->st, E.Sell, E.tcol, c->tz, pold, pnew, c->tAp, nf, c->rb(), c->sc);
                launch_k(k_cg_update<NT>, gf, VEC_THREADS, 0, c->st, E.Dinv, pnew, c->tAp, x, c->tr, c->tz, nf, c->rb(), c->sc);
            }
            CKL();
            read_scalars(c);
            if (trace_cg_enabled())
                fprintf(stderr, "trace CG it %d rz %.6e pAp %.6e alpha %.3e beta %.3e zmean %.3e relres %.3e done %d bd %d\n",
                        c->hsc->iters, c->hsc->rz, c->hsc->pAp, c->hsc->alpha, c->hsc->beta, c->hsc->zmean,
                        c->hsc->relres, c->hsc->done, c->hsc->breakdown);
            if (c->hsc->done) break;
        }
        c->S.trace_solves += 1;
        c->S.trace_iters += c->hsc->iters;
        c->S.last_trace_relres = c->hsc->relres;
        if (c->hsc->breakdown == 2) throw std::domain_error("trace CG: non-finite residual");
        if (c->hsc->relres > rtol) {
            char msg[256];
            snprintf(msg, sizeof msg, "trace CG: stopped at iteration %d (%s), relres %.3e", c->hsc->iters,
                     c->hsc->breakdown ? "p^T S p <= 0" : "iteration cap", c->hsc->relres);
            throw std::length_error(msg);
        }
    }

    // CG preconditioned by one multigrid V-cycle per iteration. The setup and chunks of 8
    // iterations are CUDA graphs captured once per operator (input c->tb, solution c->tx); kernels
    // of a chunk return at once after convergence.
    static void trace_solve_mg(hdg_ctx *c, CondCache &E, const double *b, double *x, double rtol) {
        const int nf = (int)c->nfacets;
        const int gr = grid_for(c->nL);
        if (b != c->tb) CK(cudaMemcpyAsync(c->tb, b, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
        launch_k(k_set_tol, 1, 1, 0, c->st, c->sc, rtol, c->P.max_iters);
        CKL();
        if (c->trace_vcycles > 0) {     // a fixed number of V-cycles in place of the CG (inner solves)
            launch_k(k_trace_mean<NT>, grid_for(nf), VEC_THREADS, 0, c->st, c->tb, nf, c->rb(), c->sc);
            launch_k(k_cg_setup_mg<NT>, gr, VEC_THREADS, 0, c->st, c->tb, c->tx, c->tr, c->tp[0], nf, c->sc);
            for (int v = 0; v < c->trace_vcycles; ++v) {
                if (v > 0) {            // r = b - mean - S x
                    launch_k(k_trace_resid<NT>, gr, VEC_THREADS, 0, c->st, E.Sell, E.tcol, c->tb, c->tx, c->tr, nf, c->sc);
                }
                vcycle(c, E, c->tr, c->tz, false, -1);
                launch_k(k_axpy_done, gr, VEC_THREADS, 0, c->st, c->tz, c->tx, c->nL, c->sc);
            }
            CKL();
            if (x != c->tx) CK(cudaMemcpyAsync(x, c->tx, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
            if (c->capturing) launch_k(k_count_solve, 1, 1, 0, c->st, c->dcnt, nullptr, c->sc);
            else c->S.trace_solves += 1;
            CKL();
            return;
        }
        if (c->capturing) {             // device-side loop, two iterations per pass
            const bool f32 = fcg32(c, E);
            launch_k(k_trace_mean<NT>, grid_for(nf), VEC_THREADS, 0, c->st, c->tb, nf, c->rb(), c->sc);
            launch_k(k_cg_setup_mg<NT>, gr, VEC_THREADS, 0, c->st, c->tb, c->tx, c->tr, c->tp[0], nf, c->sc);
            if (f32) cg_vcycle32(c, E, 1);
            else vcycle(c, E, c->tr, c->tz, false, 1);
            capture_while(
                c, [&](LoopCtl L) { launch_k(k_loop_init, 1, 1, 0, c->st, L, &c->sc->done); },
                [&](LoopCtl L) {
                    for (int m = 0; m < 2; ++m) {
                        double *pold = c->tp[m & 1], *pnew = c->tp[(m + 1) & 1];
                        launch_k(k_cg_apply<NT>, cg_apply_grid<NT>(nf), 128, 0, c->st, E.Sell, E.tcol, c->tz, pold, pnew, c->tAp, nf,
                                                                     c->rb(), c->sc);
                        if (f32) {
                            launch_k(k_cg_update_xr<NT>, gr, VEC_THREADS, 0, c->st, (const double *)pnew,
                                     (const double *)c->tAp, c->tx, c->tr, nf, (const Scalars *)c->sc);
                            cg_vcycle32(c, E, 0);
                            continue;
                        }
                        launch_k(k_cg_update_cheb0<NT>, grid_facets(nf), FACET_THREADS, 0, c->st, 
                            pnew, c->tAp, c->tx, c->tr, E.Dinv, c->txa, c->td, E.t_invth, nf, c->sc);
                        vcycle(c, E, c->tr, c->tz, true, 0);
                    }
                    launch_k(k_loop_ctl, 1, 1, 0, c->st, L, c->P.max_iters / 2 + 2, &c->sc->done);
                });
            if (x != c->tx) CK(cudaMemcpyAsync(x, c->tx, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
            launch_k(k_count_solve, 1, 1, 0, c->st, c->dcnt, nullptr, c->sc);
            CKL();
            return;
        }
        const int chunk = trace_cg_enabled() ? 1 : 8;
        if (!E.g_setup) {
            const bool f32 = fcg32(c, E);
            E.g_setup = capture_graph(c, [&]() {
                launch_k(k_trace_mean<NT>, grid_for(nf), VEC_THREADS, 0, c->st, c->tb, nf, c->rb(), c->sc);
                launch_k(k_cg_setup_mg<NT>, gr, VEC_THREADS, 0, c->st, c->tb, c->tx, c->tr, c->tp[0], nf, c->sc);
                if (f32) cg_vcycle32(c, E, 1);
                else vcycle(c, E, c->tr, c->tz, false, 1);
                CKL();
            });
            E.g_chunk = capture_graph(c, [&]() {
                for (int m = 0; m < chunk; ++m) {
                    double *pold = c->tp[m & 1], *pnew = c->tp[(m + 1) & 1];
                    launch_k(k_cg_apply<NT>, cg_apply_grid<NT>(nf), 128, 0, c->st, E.Sell, E.tcol, c->tz, pold, pnew, c->tAp, nf,
                                                                 c->rb(), c->sc);
                    if (f32) {
                        launch_k(k_cg_update_xr<NT>, gr, VEC_THREADS, 0, c->st, (const double *)pnew, (const double *)c->tAp,
                                 c->tx, c->tr, nf, (const Scalars *)c->sc);
                        cg_vcycle32(c, E, 0);
                        continue;
                    }
                    launch_k(k_cg_update_cheb0<NT>, grid_facets(nf), FACET_THREADS, 0, c->st, pnew, c->tAp, c->tx, c->tr, E.Dinv,
                                                                                        c->txa, c->td, E.t_invth, nf, c->sc);
                    vcycle(c, E, c->tr, c->tz, true, 0);
                }
                CKL();
            });
        }
        CK(cudaGraphLaunch(E.g_setup, c->st));
        for (long long launched = 0;; launched += chunk) {
            if (launched > (long long)c->P.max_iters + 2 * chunk)
                throw std::length_error("trace CG: no convergence flag from the device");
            CK(cudaGraphLaunch(E.g_chunk, c->st));
            read_scalars(c);
            if (trace_cg_enabled())
                fprintf(stderr, "mg CG it %d rz %.6e pAp %.6e alpha %.3e beta %.3e zmean %.3e relres %.3e done %d bd %d\n",
                        c->hsc->iters, c->hsc->rz, c->hsc->pAp, c->hsc->alpha, c->hsc->beta, c->hsc->zmean,
                        c->hsc->relres, c->hsc->done, c->hsc->breakdown);
            if (c->hsc->done) break;
        }
        if (x != c->tx) CK(cudaMemcpyAsync(x, c->tx, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
        c->S.trace_solves += 1;
        c->S.trace_iters += c->hsc->iters;
        c->S.last_trace_relres = c->hsc->relres;
        if (c->hsc->breakdown == 2) throw std::domain_error("trace CG: non-finite residual");
        if (c->hsc->relres > rtol) {
            char msg[256];
            snprintf(msg, sizeof msg, "trace CG (multigrid): stopped at iteration %d (%s), relres %.3e", c->hsc->iters,
                     c->hsc->breakdown ? "p^T S p <= 0" : "iteration cap", c->hsc->relres);
            throw std::length_error(msg);
        }
    }

    // Mixed solve: [[M, -cG], [B, C]] (U, dp, dl) = (Ru, -Gamma(X, p, lam)) ; outputs U, dp, dl
    // (no mean shift). Ru: dual (modal) or null; X, p, lam: or null.
    static void mixed_solve(hdg_ctx *c, double cc, const double *Ru, const double *X, const double *p,
                            const double *lam, double *U, double *dp, double *dl, const double *Rp_add = nullptr,
                            const double *Rl_add = nullptr, double rtol = -1.0) {
        CondCache &E = condense(c, cc);
        CompTimer tm_(c, &c->S.ms_trace);
        size_t smem_rhs = sizeof(double) * TEAMS_PER_BLOCK * (NL + 4 * MU + NP + NL);
        unsigned nb = cell_blocks(c);
        launch_k(k_mixed_rhs<K>, nb, 128, smem_rhs, c->st, c->R, c->M, c->P.tau, Ru, X, p, lam, Rp_add, E.Zc, c->vK, c->wK);
        CKL();
        launch_k(k_facet_gather<NT>, grid_for(c->nL), VEC_THREADS, 0, c->st, c->M, c->vK, Rl_add, c->tb, (float *)nullptr);
        CKL();
        trace_solve(c, E, c->tb, dl, rtol > 0 ? rtol : c->P.trace_rtol);
        size_t smem_bs = sizeof(double) * TEAMS_PER_BLOCK * (NL + NP);
        launch_k(k_mixed_backsub<K>, nb, 128, smem_bs, c->st, c->R, c->M, cc, Ru, c->wK, dl, E.Zc, E.Ac, U, dp);
        CKL();
    }

    // FP32 cell maps of the preconditioner's Step II for coefficient cc (formed once, outside
    // graph captures)
    // FP32 copy of the trace multigrid of coefficient E.c for the one-V-cycle inner Step II; left
    // out (FP64 V-cycle) when the P1 hierarchy's vectors do not fit one block's shared memory
    // The levels from first32 down run in one block (k_tv_tail, everything in shared memory); the
    // larger ones above as grid-wide kernels. first32: the first level whose sub-hierarchy fits the
    // block (<= 200 KiB, rows of at most 1024 points) and has at most HDG_MG32_TAIL_MAX (default
    // 1200) vertices: one block serves the small levels, the large ones keep all SMs busy.
    static int mg32_tail_max() {
        static int v = -1;
        if (v < 0) {
            const char *e = std::getenv("HDG_MG32_TAIL_MAX");
            v = e ? std::atoi(e) : 1200;
            if (v < 1) v = 1;
        }
        return v;
    }
    static size_t tail32_bytes(const CondCache &E, int first) {
        P1Grid G[MG_MAX_LEVELS];
        const int L = (int)E.lv.size();
        for (int l = first; l < L; ++l) G[l - first] = E.lv[l].G;
        return sizeof(float) * tail32_floats(G, L - first);
    }
    static bool tail32_fits(const CondCache &E, int first) {
        const int L = (int)E.lv.size();
        if (tail32_bytes(E, first) > (size_t)200 * 1024) return false;
        for (int l = first; l < L; ++l)
            if (E.lv[l].G.nvx > 1024) return false;
        return E.lv[first].G.nverts <= mg32_tail_max() || first == L - 1;
    }
    static void build_mg32(hdg_ctx *c, CondCache &E) {
        const int L = (int)E.lv.size();
        if (L < 1 || L > MG_MAX_LEVELS) return;
        int first = 0;
        while (first < L - 1 && !tail32_fits(E, first)) ++first;
        if (!tail32_fits(E, first)) return;
        const size_t smem = tail32_bytes(E, first);
        auto f32 = [&](const double *a, long long n) {
            float *b = c->alloc<float>((size_t)n);
            launch_k(k_f64_to_f32, grid_for(n), VEC_THREADS, 0, c->st, a, b, n);
            return b;
        };
        E.Sell32 = f32(E.Sell, 5LL * NT * c->nL);
        E.Dinv32 = f32(E.Dinv, (long long)NT * c->nL);
        E.A32.resize(L);
        E.dinv32.resize(L);
        for (int l = 0; l < L; ++l) {
            E.A32[l] = f32(E.lv[l].A, (long long)P1_NS * E.lv[l].G.nverts);
            E.dinv32[l] = f32(E.lv[l].dinv, E.lv[l].G.nverts);
        }
        E.Minv32 = f32(E.Minv, (long long)E.Nc * E.Nc);
        CKL();
        if (!c->tb32) {
            c->tb32 = c->alloc<float>(c->nL); c->tr32 = c->alloc<float>(c->nL); c->tx32 = c->alloc<float>(c->nL);
            c->txa32 = c->alloc<float>(c->nL); c->td32 = c->alloc<float>(c->nL);
            c->tzold = c->alloc<double>(c->nL);
        }
        if (c->mgw32.empty())               // the hierarchy depends on the mesh only
            for (int l = 0; l < L; ++l) {
                const size_t nv = (size_t)E.lv[l].G.nverts;
                MGWork32 w;
                w.b = c->alloc<float>(nv); w.xa = c->alloc<float>(nv); w.xb = c->alloc<float>(nv);
                w.d = c->alloc<float>(nv); w.t = c->alloc<float>(nv);
                c->mgw32.push_back(w);
            }
        {   // the tail's shared-memory image: dinv and the stencil of each level at their offsets
            E.tail_img = c->alloc<float>(smem / sizeof(float));
            CK(cudaMemsetAsync(E.tail_img, 0, smem, c->st));
            size_t off = 0;
            for (int l = first; l < L; ++l) {
                const size_t nv = (size_t)E.lv[l].G.nverts;
                CK(cudaMemcpyAsync(E.tail_img + off + 4 * nv, E.dinv32[l], nv * sizeof(float), cudaMemcpyDeviceToDevice,
                                   c->st));
                CK(cudaMemcpyAsync(E.tail_img + off + 5 * nv, E.A32[l], P1_NS * nv * sizeof(float),
                                   cudaMemcpyDeviceToDevice, c->st));
                off += 12 * nv;
            }
        }
        E.first32 = first;
        CK(cudaFuncSetAttribute(k_tv_tail<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        E.tail32_smem = smem;
        E.mg32 = true;
    }

    static Tail32 tail32_params(hdg_ctx *c, const CondCache &E) {
        Tail32 T{};
        const int f0 = E.first32;
        T.L = (int)E.lv.size() - f0;
        T.Nc = E.Nc;
        T.nfacets = (int)c->nfacets;
        int off = 0;
        for (int l = 0; l < T.L; ++l) {
            const MGLevel &V = E.lv[f0 + l];
            T.G[l] = V.G; T.A[l] = E.A32[f0 + l]; T.dinv[l] = E.dinv32[f0 + l];
            T.invth[l] = (float)V.invth; T.c1[l] = (float)V.c1; T.c2[l] = (float)V.c2;
            T.off[l] = off;
            off += 12 * V.G.nverts;
        }
        T.Minv = E.Minv32;
        T.b1 = c->mgw32[f0].b;
        T.e1 = c->mgw32[f0].xb;
        T.img = reinterpret_cast<const float4 *>(E.tail_img);
        T.nimg4 = (int)(E.tail32_smem / sizeof(float4));
        return T;
    }

    // The P1 part of the FP32 V-cycle: from the right-hand side on the mesh vertices (mgw32[0].b)
    // to the correction there (mgw32[0].xb); the levels above first32 as grid-wide kernels around
    // the one-block tail
    static void p1_cycle32(hdg_ctx *c, const CondCache &E) {
        const int f0 = E.first32;
        for (int l = 0; l < f0; ++l) {
            const MGLevel &V = E.lv[l];
            const MGWork32 &W = c->mgw32[l];
            const int nv = V.G.nverts, g = grid_for(nv);
            launch_k(k_p32_cheb0, g, VEC_THREADS, 0, c->st, (const float *)E.dinv32[l], (const float *)W.b, W.xa, W.d,
                     (float)V.invth, nv);
            launch_k(k_p32_cheb, g, VEC_THREADS, 0, c->st, V.G, (const float *)E.A32[l], (const float *)E.dinv32[l],
                     (const float *)W.b, (const float *)W.xa, W.xb, W.d, (float)V.c1, (float)V.c2);
            launch_k(k_p32_resid, g, VEC_THREADS, 0, c->st, V.G, (const float *)E.A32[l], (const float *)W.b,
                     (const float *)W.xb, W.t);
            launch_k(k_p32_restrict, grid_for(E.lv[l + 1].G.nverts), VEC_THREADS, 0, c->st, E.lv[l + 1].G, V.G,
                     (const float *)W.t, c->mgw32[l + 1].b);
        }
        launch_k(k_tv_tail<NT>, 1, 1024, E.tail32_smem, c->st, tail32_params(c, E));
        for (int l = f0 - 1; l >= 0; --l) {
            const MGLevel &V = E.lv[l];
            const MGWork32 &W = c->mgw32[l];
            const int g = grid_for(V.G.nverts);
            launch_k(k_p32_prolong, g, VEC_THREADS, 0, c->st, V.G, E.lv[l + 1].G, (const float *)c->mgw32[l + 1].xb, W.xb);
            launch_k(k_p32_cheb, g, VEC_THREADS, 0, c->st, V.G, (const float *)E.A32[l], (const float *)E.dinv32[l],
                     (const float *)W.b, (const float *)W.xb, W.xa, W.d, 0.f, (float)V.invth);
            launch_k(k_p32_cheb, g, VEC_THREADS, 0, c->st, V.G, (const float *)E.A32[l], (const float *)E.dinv32[l],
                     (const float *)W.b, (const float *)W.xa, W.xb, W.d, (float)V.c1, (float)V.c2);
        }
    }

    // Inner Step II's trace solve as one FP32 V-cycle: right-hand side gathered from the cells'
    // lambda rows (c->vK) minus sub, result (FP64) in out
    static void trace_vcycle32(hdg_ctx *c, const CondCache &E, const double *sub, double *out) {
        const int nf = (int)c->nfacets;
        const unsigned gb = tv_blocks(nf, TGrp<NT>::G);
        const TraceOp32 T{E.Sell32, E.Dinv32, E.tcol, nf};
        const float invth = (float)E.t_invth, c1 = (float)E.t_c1, c2 = (float)E.t_c2;
        launch_k(k_tv_gather<NT>, grid_for(c->nL), VEC_THREADS, 0, c->st, c->M, c->vK, sub, c->tb32, c->rb(), c->sc,
                                                                  c->capturing ? c->dcnt : nullptr);
        launch_k(k_tv_cheb01<NT>, gb, 128, 0, c->st, T, (const float *)c->tb32, (const double *)nullptr, (const Scalars *)c->sc,
                 invth, c1, c2, c->tr32, c->tx32, c->td32);
        const int nv0 = E.lv[0].G.nverts;
        float *b1 = c->mgw32[0].b, *e1 = c->mgw32[0].xb;
        launch_k(k_tv_restrict<NT>, (unsigned)((16LL * nv0 + 127) / 128), 128, 0, c->st, T, c->tr32, c->tx32,
                                                                   c->M.vert_facet, c->M.vert_fsign, nv0, b1);
        p1_cycle32(c, E);
        launch_k(k_tv_cheb<NT>, gb, 128, 0, c->st, T, c->tr32, c->tx32, e1, c->M.facet_vert, c->txa32, c->td32, 0.f, invth,
                                                           (double *)nullptr);
        launch_k(k_tv_cheb<NT>, gb, 128, 0, c->st, T, c->tr32, c->txa32, (const float *)nullptr, c->M.facet_vert,
                                                           (float *)nullptr, c->td32, c1, c2, out);
        CKL();
        if (!c->capturing) c->S.trace_solves += 1;
    }

    // The trace CG's preconditioner as the FP32 V-cycle (flexible CG): z = V(r) for r = c->tr
    // (FP64, off the constant mode), then the flexible CG reduction (first: rz0).
    static bool fcg32(const hdg_ctx *c, const CondCache &E) { return E.mg32 && c->P.trace_fp32_vcycle; }
    static void cg_vcycle32(hdg_ctx *c, const CondCache &E, int first) {
        const int nf = (int)c->nfacets;
        const unsigned gb = tv_blocks(nf, TGrp<NT>::G);
        const TraceOp32 T{E.Sell32, E.Dinv32, E.tcol, nf};
        const float invth = (float)E.t_invth, c1 = (float)E.t_c1, c2 = (float)E.t_c2;
        const int nv0 = E.lv[0].G.nverts;
        float *b1 = c->mgw32[0].b, *e1 = c->mgw32[0].xb;
        launch_k(k_tv_cheb01<NT>, gb, 128, 0, c->st, T, (const float *)nullptr, (const double *)c->tr,
                 (const Scalars *)nullptr, invth, c1, c2, c->tr32, c->tx32, c->td32);
        launch_k(k_tv_restrict<NT>, (unsigned)((16LL * nv0 + 127) / 128), 128, 0, c->st, T, c->tr32, c->tx32,
                                                                   c->M.vert_facet, c->M.vert_fsign, nv0, b1);
        p1_cycle32(c, E);
        launch_k(k_tv_cheb<NT>, gb, 128, 0, c->st, T, c->tr32, c->tx32, e1, c->M.facet_vert, c->txa32, c->td32, 0.f, invth,
                                                           (double *)nullptr);
        launch_k(k_tv_cheb<NT>, gb, 128, 0, c->st, T, c->tr32, c->txa32, (const float *)nullptr, c->M.facet_vert,
                                                           (float *)nullptr, c->td32, c1, c2, c->tz);
        launch_k(k_fcg_rz<NT>, grid_for(c->nL), VEC_THREADS, 0, c->st, (const double *)c->tr, (const double *)c->tz,
                 c->tzold, nf, first, c->rb(), c->sc);
    }

    static void ensure_pre_maps(hdg_ctx *c, double cc) {
        CondCache &E = condense(c, cc);
        if (c->capturing || c->P.precision != HDG_MIXED) return;
        if (c->P.inner_trace_fp32 && E.mg && !E.mg32) build_mg32(c, E);
        if (E.Lrhs32) return;
        E.Lrhs32 = c->alloc<float>((size_t)c->ncells * (NU + NP) * (NL + NP));
        E.Lbs32 = c->alloc<float>((size_t)c->ncells * (NP + NL) * (NU + NP));
        constexpr int SCR = NU + NP + NL + NP + (NL + 4 * MU + NP + NL) + NU + NP + (NL + NP);
        const size_t smem = sizeof(double) * TEAMS_PER_BLOCK * SCR;
        CK(cudaFuncSetAttribute(k_build_pre_maps<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch_k(k_build_pre_maps<K>, cell_blocks(c), 128, smem, c->st, c->R, c->M, cc, c->P.tau, E.Zc, E.Ac, E.Lrhs32,
                                                                 E.Lbs32);
        CKL();
    }

    static void mean_shift(hdg_ctx *c, double *p, double *lam) {
        launch_k(k_p_integral<K>, grid_for(c->ncells), VEC_THREADS, 0, c->st, c->M, p, c->rb(), c->sc);
        CKL();
        launch_k(k_p_shift<K>, grid_for(c->ncells > c->nfacets ? c->ncells : c->nfacets), VEC_THREADS, 0, c->st, 
            c->M, c->area, p, lam, c->sc);
        CKL();
    }

    // ---------------------------------------------------------------- Step I operator
    // Step-I solves to loose tolerances (the inner solves of the stage preconditioner) run in FP32;
    // tight ones in FP64. The assembly forms the block inverses the coming solves need.
    static constexpr int INV64 = 1, INV32 = 2, BLK32 = 4;     // BLK32: FP32 copy of the blocks (Dblk32)
    static bool loose(const hdg_ctx *c, double rtol) { return rtol >= 1e-4 && c->P.precision == HDG_MIXED; }
    static int inv_for(const hdg_ctx *c, double rtol) { return loose(c, rtol) ? INV32 : INV64; }

    // Step-I operator M - cc F(Qs): diagonal blocks, neighbour and penalty weights, and the
    // block-Jacobi inverses named by inv (INV64 | INV32; with BLK32 also the blocks in FP32)
    // the assembly's tables as pairs (HDG_MIXED: the block formed in pair arithmetic)
    static AsmF2 tadv2(const hdg_ctx *c) {
        return c->P.precision == HDG_MIXED ? AsmF2{c->Tadv2, c->ephi2a, c->Sfac2} : AsmF2{};
    }
    static void assemble_stepI(hdg_ctx *c, const double *Qs, double cc, int inv) {
        CompTimer tm_(c, &c->S.ms_assembly);
        const size_t smem = sizeof(double) * ((inv & INV64) ? fimpl_smem_doubles<K>() : fimpl_smem_noinv_doubles<K>());
        CK(cudaFuncSetAttribute(k_fimpl_assemble<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * fimpl_smem_doubles<K>())));
        if (!c->capturing) CK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->st));   // (graphs: once per launch)
        launch_k(k_fimpl_assemble<K>, (unsigned)c->ncells, 128, smem, c->st, 
            c->R, c->M, Qs, cc, c->P.alpha, c->P.delta_up, c->Dblk, c->wq, c->wq32, c->pen, c->pen32,
            (inv & INV64) ? c->Binv : nullptr, c->dstatus, tadv2(c));
        CKL();
        float *blk32 = (inv & BLK32) ? c->Dblk32 : nullptr;
        c->blk32_ok = blk32 && c->Dblk32lo;
        if (inv & INV32) {              // FP32 inverses: a warp per cell, the block in registers
            launch_k(k_block_inv32<K>, (unsigned)((c->ncells * 32 + 127) / 128), 128, 0, c->st, (const double *)c->Dblk,
                     c->Binv32, blk32, c->ncells, use_gs(c) ? 1 : 0, c->dstatus);
            CKL();
        } else if (blk32) {
            launch_k(k_blocks_to_f32<K>, grid_for((long long)GsBlk<K>::SIZE * c->ncells), VEC_THREADS, 0, c->st,
                     (const double *)c->Dblk, blk32, (long long)c->ncells);
            CKL();
        }
        if (c->blk32_ok) {              // the rest of each block after its FP32 rounding (pair products)
            launch_k(k_blocks_lo<K>, grid_for((long long)GsBlk<K>::SIZE * c->ncells), VEC_THREADS, 0, c->st,
                     (const double *)c->Dblk, c->Dblk32lo, (long long)c->ncells);
            CKL();
        }
        c->inv_ok = inv;
    }

    static void cell_apply(hdg_ctx *c, const double *x, double *y) {
        launch_k(k_cell_apply_mf<K>, cell_blocks(c), 128, sizeof(double) * TEAMS_PER_BLOCK * 6 * Dm::NFQ, c->st, 
            EdgeTab<double>{c->R.ephi, c->pen}, c->M, c->Dblk, c->wq, x, y);
        CKL();
    }

    // one Arnoldi step of the Step-I GMRES in precision T: V_j, z = Binv V_j (edge values only),
    // w = B z, dots, orthogonalisation. FP64 (tight solves): classical Gram-Schmidt twice, in two
    // more kernels. FP32 (inner solves): one pass folded into the two kernels (the norm by
    // Pythagoras in the product kernel, the subtraction in the next step's preconditioner kernel).
    template <class T>
    static void gmres_arnoldi(hdg_ctx *c, const EdgeTab<T> &E, const T *Binv, const T *wq, T *utr, T *w, T *V) {
        const long long n = c->nQ;
        const unsigned cb = cell_blocks(c), ab = cb < (unsigned)MAX_RED_BLOCKS ? cb : (unsigned)MAX_RED_BLOCKS;
        const int go = grid_orth(n);
        constexpr bool F = sizeof(T) == sizeof(float);
        launch_k(k_gm_precond_mf<K, T, F>, cb, 128, sizeof(T) * TEAMS_PER_BLOCK * 2 * NU, c->st, E, c->M, Binv, w, V,
                 utr, c->gs);
        launch_k(k_gm_apply_mf<K, T, F>, ab, 128, sizeof(T) * TEAMS_PER_BLOCK * 6 * Dm::NFQ, c->st, E, c->M, wq, utr, w,
                 V, c->rb(), c->gs);
        if (!F) {
            launch_k(k_gm_orth1<T>, go, VEC_THREADS, 0, c->st, w, V, n, c->rb(), c->gs);
            launch_k(k_gm_orth2<T>, go, VEC_THREADS, 0, c->st, w, V, n, c->rb(), c->gs);
        }
    }
    static void gmres_arnoldi64(hdg_ctx *c) {
        gmres_arnoldi<double>(c, EdgeTab<double>{c->R.ephi, c->pen}, c->Binv, c->wq, c->utr, c->gw, c->gV);
    }

    // Arnoldi steps per pass of the inner FP32 loop (HDG_INNER_UNROLL overrides the default)
    static int inner_unroll() {
        static int v = -1;
        if (v < 0) {
            const char *e = std::getenv("HDG_INNER_UNROLL");
            v = e ? std::atoi(e) : 4;
            if (v < 1) v = 1;
            if (v > 8) v = 8;
        }
        return v;
    }

    static bool use_gs(const hdg_ctx *c) { return c->gs_ok && c->P.inner_gs; }
    // the colour kernels run a warp per cell, four warps per 128-thread block
    static constexpr int GS_WARPS = 4;
    static unsigned gs_blocks(const hdg_ctx *c) {
        return (unsigned)(((c->ncells + 1) / 2 + GS_WARPS - 1) / GS_WARPS);
    }

    // One Arnoldi step of the inner FP32 solve: the preconditioner (block Jacobi, or red-black block
    // Gauss-Seidel, hdg_gs32.cuh), the product with the block partials of its dots, and the
    // finishing kernel (ctl: it also keeps the loop L's state; limit: the loop's pass guard)
    static void inner_step32(hdg_ctx *c, LoopCtl L, int limit, int ctl) {
        const EdgeTab<float> E{c->ephi32, c->pen32, c->nrm32};
        const unsigned cb = cell_blocks(c), ab = cb < (unsigned)MAX_RED_BLOCKS ? cb : (unsigned)MAX_RED_BLOCKS;
        if (use_gs(c)) {
            const size_t smg = sizeof(float) * GS_WARPS * (2 * NU + 6 * Dm::NFQ);
            for (int col = 0; col < 2; ++col)
                launch_k(k_gs_diag<K>, gs_blocks(c), 128, smg, c->st, E, c->M, (const float *)c->Binv32, (const float *)c->gw32,
                         c->gV32, c->utr32, (const float *)c->wq32, (const GmresState *)c->gs, col);
            launch_k(k_gs_apply<K>, ab, 128, sizeof(float) * TEAMS_PER_BLOCK * 6 * Dm::NFQ, c->st, E, c->M,
                     (const float *)c->wq32, (const float *)c->utr32, c->gw32, (const float *)c->gV32, c->rb(), c->gs);
        } else {
            gmres_arnoldi<float>(c, E, c->Binv32, c->wq32, c->utr32, c->gw32, c->gV32);
        }
        launch_k(k_gm_finish_ctl, 1, 256, 0, c->st, L, limit, c->rb(), (int)ab, c->gs, ctl);
    }

    // A loose Step-I solve in FP32, recorded into the current capture: one GMRES(GM_M) cycle from
    // x = 0 with its Arnoldi steps as a device-side loop, stopping at the tolerance or after GM_M
    // steps (an inexact solve is what the flexible outer iteration expects). b, x: FP64.
    static void stepI32_record(hdg_ctx *c, const double *b, double *x) {
        const long long n = c->nQ;
        const int g = grid_for(n);
        const EdgeTab<float> E{c->ephi32, c->pen32, c->nrm32};
        launch_k(k_gm_start<float>, g, VEC_THREADS, 0, c->st, n, b, nullptr, c->gw32, 1, c->rb(), c->gs, -1.0, 0, GM_M);
        capture_while(
            c, [&](LoopCtl L) { launch_k(k_loop_init, 1, 1, 0, c->st, L, &c->gs->cycle_end); },
            [&](LoopCtl L) {
                const int U = inner_unroll();
                for (int u = 0; u < U; ++u) inner_step32(c, L, GM_M / U + 2, u == U - 1 ? 1 : 0);
            });
        launch_k(k_gm_solve32, 1, 256, 0, c->st, c->gs);
        if (use_gs(c)) {
            const EdgeTab<float> E32{c->ephi32, c->pen32, c->nrm32};
            for (int col = 0; col < 2; ++col)
                launch_k(k_gs_combine<K>, gs_blocks(c), 128, sizeof(float) * GS_WARPS * (2 * NU + 6 * Dm::NFQ), c->st,
                         E32, c->M, (const float *)c->gV32, (const float *)c->Binv32, (const float *)c->wq32, c->utr32, x,
                         (const GmresState *)c->gs, col == 1 ? c->dcnt : (DevCount *)nullptr, col);
        } else {
            launch_k(k_gm_combine_update<K, float>, cell_blocks(c), 128, sizeof(float) * TEAMS_PER_BLOCK * NU, c->st, c->gV32,
                     c->Binv32, x, c->M, (const GmresState *)c->gs, c->dcnt);
        }
        CKL();
    }

    // cycle start: w = b - B x (x = 0 on the first cycle)
    static void gmres_start(hdg_ctx *c, int first) {
        if (!first) cell_apply(c, c->gx, c->gz);
        launch_k(k_gm_start<double>, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->nQ, c->gb, first ? nullptr : c->gz, c->gw,
                                                                      first, c->rb(), c->gs, -1.0, 0, 0);
    }

    // Restarted GMRES(GM_M) on the assembled Step-I operator with right block-Jacobi
    // preconditioning: B x = b, x0 = 0, stop at ||b - B x|| <= rtol ||b||. One restart cycle is a
    // CUDA graph (right-hand side c->gb, solution c->gx; kernels return at once after convergence).
    static void gmres_cycle(hdg_ctx *c, int first, int m) {
        const long long n = c->nQ;
        const int g = grid_for(n);
        gmres_start(c, first);
        launch_k(k_gm_set_cycle, 1, 1, 0, c->st, c->gs, m);
        for (int j = 0; j < m; ++j) gmres_arnoldi64(c);
        launch_k(k_gm_solve, 1, 256, 0, c->st, c->gs, nullptr);
        launch_k(k_gm_combine<double>, g, VEC_THREADS, 0, c->st, c->gV, c->gu, n, c->gs);
        launch_k(k_gm_update_x<K, double>, g, VEC_THREADS, 0, c->st, c->Binv, c->gu, c->gx, c->ncells, first);
        CKL();
    }

    // The same cycle with its Arnoldi steps as a device-side loop (inside a graph capture).
    static void gmres_cycle_dev(hdg_ctx *c, int first, int m) {
        const long long n = c->nQ;
        const int g = grid_for(n);
        gmres_start(c, first);
        launch_k(k_gm_set_cycle, 1, 1, 0, c->st, c->gs, m);
        capture_while(
            c, [&](LoopCtl L) { launch_k(k_loop_init, 1, 1, 0, c->st, L, &c->gs->cycle_end); },
            [&](LoopCtl L) {
                gmres_arnoldi64(c);
                launch_k(k_loop_ctl, 1, 1, 0, c->st, L, m + 1, &c->gs->cycle_end);
            });
        launch_k(k_gm_solve, 1, 256, 0, c->st, c->gs, nullptr);
        launch_k(k_gm_combine<double>, g, VEC_THREADS, 0, c->st, c->gV, c->gu, n, c->gs);
        launch_k(k_gm_update_x<K, double>, g, VEC_THREADS, 0, c->st, c->Binv, c->gu, c->gx, c->ncells, first);
        CKL();
    }

    static void stepI_solve(hdg_ctx *c, const double *b, double *x, double rtol = -1.0) {
        if (!(rtol > 0)) rtol = c->P.stepI_rtol;
        CompTimer tm_(c, &c->S.ms_stepI);
        if (!(c->inv_ok & inv_for(c, rtol))) throw std::logic_error("Step-I solve without the block inverses it needs");
        launch_k(k_gm_set_tol, 1, 1, 0, c->st, c->gs, rtol, c->P.max_iters);
        CKL();
        if (loose(c, rtol)) {           // FP32, one cycle of at most GM_M steps
            if (c->capturing) {
                stepI32_record(c, b, x);
                return;
            }
            if (b != c->gb) CK(cudaMemcpyAsync(c->gb, b, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
            if (!c->g_stepI32)
                c->g_stepI32 = capture_graph(c, [&]() { stepI32_record(c, c->gb, c->gx); }, &c->stepI32_kernels);
            launch_counted(c, c->g_stepI32);
            CK(cudaStreamSynchronize(c->st));
            graph_stats(c, c->stepI32_kernels);
            if (x != c->gx) CK(cudaMemcpyAsync(x, c->gx, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
            return;
        }
        if (b != c->gb) CK(cudaMemcpyAsync(c->gb, b, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
        const int m = GM_M;
        if (c->capturing) {             // restarts as a device-side loop
            gmres_cycle_dev(c, 1, m);
            const int limit = c->P.max_iters + 2;
            capture_while(
                c, [&](LoopCtl L) { launch_k(k_gm_loop_ctl, 1, 1, 0, c->st, L, limit, c->gs, 1); },
                [&](LoopCtl L) {
                    gmres_cycle_dev(c, 0, m);
                    launch_k(k_gm_loop_ctl, 1, 1, 0, c->st, L, limit, c->gs, 0);
                });
            if (x != c->gx) CK(cudaMemcpyAsync(x, c->gx, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
            launch_k(k_count_solve, 1, 1, 0, c->st, c->dcnt, c->gs, nullptr);
            CKL();
            return;
        }
        cudaGraphExec_t &gf = c->gm_first, &gr = c->gm_restart;
        if (!gf) {
            gf = capture_graph(c, [&]() { gmres_cycle(c, 1, m); });
            gr = capture_graph(c, [&]() { gmres_cycle(c, 0, m); });
        }
        for (int cyc = 0;; ++cyc) {
            if (cyc > c->P.max_iters / m + 2) throw std::length_error("GMRES: no convergence flag from the device");
            CK(cudaGraphLaunch(cyc == 0 ? gf : gr, c->st));
            CK(cudaMemcpyAsync(c->hgs, c->gs, sizeof(GmresState), cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            const GmresState &G = *c->hgs;
            if (G.breakdown == 2) throw std::domain_error("GMRES: non-finite residual");
            if (G.converged) break;
            if (G.total >= c->P.max_iters) {
                char msg[256];
                snprintf(msg, sizeof msg, "GMRES: iteration cap %d reached, relres %.3e", G.total,
                         G.bnorm > 0 ? G.resid / G.bnorm : 0.0);
                throw std::length_error(msg);
            }
        }
        if (x != c->gx) CK(cudaMemcpyAsync(x, c->gx, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
        c->S.stepI_solves += 1;
        c->S.stepI_iters += c->hgs->total;
    }

    // ---------------------------------------------------------------- Alg. 2
    // r: dual (modal); Qs: advecting velocity (modal); Q, p, lam: in/out (modal)
    static int richardson(hdg_ctx *c, double cc, const double *r, const double *Qsv, double *Q, double *p,
                          double *lam) {
        assemble_stepI(c, Qsv, cc, inv_for(c, c->P.stepI_rtol));
        int hstat = 0;
        CK(cudaMemcpyAsync(&hstat, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        condense(c, cc);
        CK(cudaStreamSynchronize(c->st));
        if (hstat) throw std::domain_error("singular tentative-velocity block");
        const bool fixed = c->P.n_richardson > 0;
        const int nmax = fixed ? c->P.n_richardson : c->P.richardson_max;
        double *BQ = c->q[0], *dr = c->q[1], *Qbar = c->q[2], *X = c->q[3], *U = c->q[4];
        double *dp = c->pp[0], *dl = c->ll[0];
        size_t smem_res = sizeof(double) * TEAMS_PER_BLOCK * NL;
        unsigned nb = cell_blocks(c);
        int it = 0;
        for (it = 0; it < nmax; ++it) {
            cell_apply(c, Q, BQ);
            launch_k(k_rich_residual<K>, nb, 128, smem_res, c->st, c->R, c->M, cc, r, BQ, p, lam, dr, 1.0);
            CKL();
            stepI_solve(c, dr, Qbar);                                            // Step I
            LinComb L = lincomb();
            L.nterms = 2; L.coef[0] = 1; L.vec[0] = Q; L.coef[1] = 1; L.vec[1] = Qbar;
            launch_k(k_lincomb, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, NU, L, X, c->ncells);
            CKL();
            mixed_solve(c, cc, nullptr, X, p, lam, U, dp, dl);                  // Step II
            launch_k(k_rich_update<K>, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->M, Q, Qbar, U, p, dp, lam, dl, c->rb(), c->sc);
            CKL();                                                               // Step III
            mean_shift(c, p, lam);
            read_scalars(c);
            double dq = std::sqrt(std::fmax(c->hsc->red0, 0.0)), qn = std::sqrt(std::fmax(c->hsc->red1, 0.0));
            c->S.last_update_norm = dq;
            if (!std::isfinite(dq)) throw std::domain_error("Richardson: non-finite update");
            if (!fixed && dq <= c->P.richardson_rtol * qn) { ++it; break; }
        }
        c->S.richardson_iters += it;
        c->S.stage_solves += 1;
        if (!fixed && !(c->S.last_update_norm <= c->P.richardson_rtol * std::sqrt(std::fmax(c->hsc->red1, 0.0))))
            return 1;
        return 0;
    }

    // Stage operator y = A(c) x, x = (Q | p | lam) contiguous:
    //   yQ = (M - cF) Q - c G (p, lam),  (yp | ylam) = B Q + C (p, lam)   (one fused cell pass)
    // y32 (optional): an FP32 copy of y
    // relaxed products in use: HDG_MIXED, relax_eta > 0 and the FP32 blocks allocated
    static bool relax_on(const hdg_ctx *c) {
        return c->P.precision == HDG_MIXED && c->P.relax_eta > 0 && c->Dblk32 != nullptr;
    }
    static double relax_of(const hdg_ctx *c) { return relax_on(c) ? c->P.relax_eta : 0.0; }

    // the FP32 stage-operator kernel (runs when gs->lowprec is set)
    static void stage_apply32(hdg_ctx *c, double cc, const double *Q, const double *p, const double *lam, double *yQ,
                              double *yp, float *yQ32, float *yp32, double *zslot, const int *zslot_j,
                              GmresState *gs, DevCount *acc) {
        launch_k(k_stage_apply32<K>, (unsigned)((c->ncells + STAGE32_WARPS - 1) / STAGE32_WARPS), 32 * STAGE32_WARPS,
                 sizeof(double) * STAGE32_WARPS * ((stage32_scratch_floats<K>() + 1) / 2), c->st, c->R,
                 Ref32{c->Dhat32, c->Ehat32}, EdgeTab<float>{c->ephi32, c->pen32, c->nrm32}, c->M,
                 (const float *)c->geo32, (const float *)c->Dblk32, (const float *)c->wq32, (float)cc, (float)c->P.tau, Q,
                 p, lam, yQ, yp, c->vK, yQ32, yp32, zslot, zslot_j, gs, acc);
    }

    static f2 pair_of(double x) {
        const float h = (float)x;
        return f2{h, (float)(x - (double)h)};
    }
    // HDG_MIXED with the FP32 copy of the blocks current: the FP64-accurate products in pairs,
    // for stage tolerances of PAIR_MIN_RTOL and above (pairs carry about 2^-46 = 1.4e-14 of the
    // terms' magnitudes; at 1e-12 that already cost 8 % more outer iterations on a 16 x 16 walled
    // channel, k = 4, so tighter tolerances take the FP64 kernel, whose products are 2^7 finer)
    static constexpr double PAIR_MIN_RTOL = 5e-11;
    static bool use_f2(const hdg_ctx *c) {
        return c->P.precision == HDG_MIXED && c->blk32_ok && c->P.richardson_rtol >= PAIR_MIN_RTOL;
    }
    static void stage_apply_f2(hdg_ctx *c, double cc, const double *Q, const double *p, const double *lam, double *yQ,
                               double *yp, float *yQ32, float *yp32, double *zslot, const int *zslot_j,
                               const int *skip) {
        const size_t smem = sizeof(f2) * STAGE32_WARPS * stage_f2_scratch<K>();
        launch_k(k_stage_apply_f2<K>, (unsigned)((c->ncells + STAGE32_WARPS - 1) / STAGE32_WARPS), 32 * STAGE32_WARPS, smem,
                 c->st, RefF2{c->ephi2, c->Ehat2, c->Dhat2}, (const double *)c->pen, c->M, (const float *)c->Dblk32,
                 (const float *)c->Dblk32lo, (const double *)c->wq, pair_of(cc), pair_of(c->P.tau), Q, p, lam, yQ, yp,
                 c->vK, yQ32, yp32,
                 zslot, zslot_j, skip);
    }

    // y = A(c) x (the stage operator). relax_gs (optional, with relaxed products in use): the
    // product is taken by the FP32 kernel when relax_gs->lowprec is set, else by the FP64 one
    // (both are launched; the other returns at once).
    static void stage_apply(hdg_ctx *c, double cc, const double *x, double *y, float *y32 = nullptr,
                            double *zslot = nullptr, const GmresState *zgs = nullptr,
                            GmresState *relax_gs = nullptr) {
        const double *Q = x, *p = x + c->nQ, *lam = x + c->nQ + c->nPv;
        double *yQ = y, *yp = y + c->nQ, *yl = y + c->nQ + c->nPv;
        float *yQ32 = y32, *yp32 = y32 ? y32 + c->nQ : nullptr, *yl32 = y32 ? y32 + c->nQ + c->nPv : nullptr;
        const int *lowprec = relax_gs && relax_on(c) ? &relax_gs->lowprec : nullptr;
        const int *zj = zgs ? &zgs->j : (const int *)nullptr;
        if (use_f2(c)) {
            stage_apply_f2(c, cc, Q, p, lam, yQ, yp, yQ32, yp32, zslot, zj, lowprec);
        } else {
            unsigned nb = cell_blocks(c);
            launch_k(k_stage_apply<K>, nb, 128, sizeof(double) * TEAMS_PER_BLOCK * (6 * Dm::NFQ + NL + 2 * MU), c->st,
                c->R, EdgeTab<double>{c->R.ephi, c->pen}, c->M, c->Dblk, c->wq, cc, c->P.tau, Q, p, lam, yQ, yp, c->vK,
                yQ32, yp32, zslot, zj, lowprec);
        }
        CKL();
        if (lowprec) {
            stage_apply32(c, cc, Q, p, lam, yQ, yp, yQ32, yp32, zslot, zj, relax_gs, c->capturing ? c->dcnt : nullptr);
            CKL();
        }
        launch_k(k_facet_gather<NT>, grid_for(c->nL), VEC_THREADS, 0, c->st, c->M, c->vK, nullptr, yl, yl32);
        CKL();
    }

    // Step II of the stage preconditioner: from the Step-I velocity X and the constraint rows
    // (vp, vl) of the input, the velocity correction U and (zp, zl)
    // With Qbar and zQ set and the FP32 cell maps in use, zQ receives Qbar + U directly (U is not
    // written) and the function returns true.
    static bool pre_step2(hdg_ctx *c, double cc, const double *X, const double *vp, const double *vl, double *U,
                          double *zp, double *zl, const double *Qbar = nullptr, double *zQ = nullptr) {
        bool fused = false;
        c->trace_vcycles = c->P.inner_trace_vcycles;
        try {
            CondCache &E = condense(c, cc);
            if (E.Lrhs32) {             // Step II from the precomputed FP32 cell maps
                CompTimer tm_(c, &c->S.ms_trace);
                const unsigned nb = cell_blocks(c);
                launch_k(k_pre_rhs<K>, nb, 128, sizeof(double) * TEAMS_PER_BLOCK * (NU + NP), c->st, c->M, E.Lrhs32, X, vp,
                                                                                            c->vK, c->wK);
                if (E.mg32 && c->P.inner_trace_fp32 && c->trace_vcycles == 1) {
                    trace_vcycle32(c, E, vl, zl);
                } else {
                    launch_k(k_facet_gather<NT>, grid_for(c->nL), VEC_THREADS, 0, c->st, c->M, c->vK, vl, c->tb, (float *)nullptr);
                    CKL();
                    trace_solve(c, E, c->tb, zl, c->P.inner_trace_rtol);
                }
                fused = Qbar && zQ;
                launch_k(k_pre_backsub<K>, nb, 128, sizeof(double) * TEAMS_PER_BLOCK * (NP + NL), c->st, c->M, E.Lbs32, c->wK,
                                                                                                zl, fused ? zQ : U, zp,
                                                                                                fused ? Qbar : nullptr);
                CKL();
            } else {
                mixed_solve(c, cc, nullptr, X, nullptr, nullptr, U, zp, zl, vp, vl, c->P.inner_trace_rtol);
            }
        } catch (...) {
            c->trace_vcycles = 0;
            throw;
        }
        c->trace_vcycles = 0;
        return fused;
    }

    // Chorin split as a preconditioner: z = P^{-1} v (Step I, then Step II on the constraint rows)
    static void chorin_precond(hdg_ctx *c, double cc, const double *v, double *z) {
        const double *vQ = v, *vp = v + c->nQ, *vl = v + c->nQ + c->nPv;
        double *zQ = z, *zp = z + c->nQ, *zl = z + c->nQ + c->nPv;
        double *Qbar = c->q[2], *U = c->q[4];
        stepI_solve(c, vQ, Qbar, c->P.inner_stepI_rtol);
        if (pre_step2(c, cc, Qbar, vp, vl, U, zp, zl, Qbar, zQ)) return;    // zQ = Qbar + U written there
        LinComb L = lincomb();
        L.nterms = 2; L.coef[0] = 1; L.vec[0] = Qbar; L.coef[1] = 1; L.vec[1] = U;
        launch_k(k_lincomb, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, NU, L, zQ, c->ncells);
        CKL();
    }

    // Orthogonalise w against the stage FGMRES basis: classical Gram-Schmidt, two passes (a
    // selective second pass was tried: the first pass cancels most of w at every step here).
    // The second pass's norm comes from Pythagoras with its own dots, so the last kernel only
    // forms v_{j+1} = (w' - V h2) / hn in V (and in vfix when set): no reduction there, and the
    // next Arnoldi step starts from V_{j+1} without a normalisation kernel.
    // The first pass's dots run in FP32 on the shadows (c->fw32 = FP32 w from the stage operator).
    static float *fV32(const hdg_ctx *c) { return c->P.precision == HDG_MIXED ? c->fV32 : nullptr; }
    static float *fw32(const hdg_ctx *c) { return c->P.precision == HDG_MIXED ? c->fw32 : nullptr; }
    static void fgmres_orth(hdg_ctx *c, double *w, long long N, GmresState *fgs, double *vfix) {
        const int go = grid_orth(N);
        if (c->P.precision == HDG_MIXED)
            launch_k(k_vec_dot<float>, go, VEC_THREADS, 0, c->st, (const float *)c->fw32, (const float *)c->fV32, N,
                     c->rb(), fgs);
        else
            launch_k(k_vec_dot<double>, go, VEC_THREADS, 0, c->st, (const double *)w, (const double *)c->fV, N, c->rb(), fgs);
        launch_k(k_fgm_orth1, go, VEC_THREADS, 0, c->st, w, c->fV, N, c->rb(), fgs);
        launch_k(k_fgm_orth2n, grid_for(N), VEC_THREADS, 0, c->st, (const double *)w, c->fV, vfix, N,
                 (const GmresState *)fgs, fV32(c));
        CKL();
    }

    // The flexible GMRES of a stage solve recorded into the current graph capture (x = c->fx,
    // b = c->fb): restart cycles, Arnoldi steps, and the inner Step-I GMRES and trace CG are
    // device-side while loops (conditional graph nodes), so a stage solve needs no host round trip.
    static void stage_fgmres_capture(hdg_ctx *c, double cc) {
        const long long N = c->nQ + c->nPv + c->nL;
        const int g = grid_for(N);
        double *x = c->fx, *b = c->fb, *w = c->fw, *res = c->fr, *u = c->fu;
        GmresState *fgs = c->fgs;
        const double rtol = c->P.richardson_rtol;
        const int maxit = c->P.richardson_max;
        auto residual = [&](int first) {            // res = b - A x; cycle start
            stage_apply(c, cc, x, w);
            CK(cudaMemcpyAsync(res, b, 8 * N, cudaMemcpyDeviceToDevice, c->st));
            launch_k(k_axpby, g, VEC_THREADS, 0, c->st, -1.0, w, 1.0, res, N);
            launch_k(k_vec_start, g, VEC_THREADS, 0, c->st, res, N, first, c->rb(), fgs, rtol, maxit, relax_of(c));
            launch_k(k_gm_set_cycle, 1, 1, 0, c->st, fgs, GM_M);
            CKL();
        };
        launch_k(k_vec_norm_into, g, VEC_THREADS, 0, c->st, b, N, c->rb(), fgs);
        residual(2);
        capture_while(
            c, [&](LoopCtl L) { launch_k(k_gm_loop_ctl, 1, 1, 0, c->st, L, maxit + 2, fgs, 1); },
            [&](LoopCtl L) {
                launch_k(k_vec_normalize, g, VEC_THREADS, 0, c->st, res, w, c->fV, c->fv, N, fgs, fV32(c));   // V_0
                CKL();
                capture_while(
                    c, [&](LoopCtl L2) { launch_k(k_loop_init, 1, 1, 0, c->st, L2, &fgs->cycle_end); },
                    [&](LoopCtl L2) {
                        chorin_precond(c, cc, c->fv, c->fz);
                        stage_apply(c, cc, c->fz, w, fw32(c), c->fZ, fgs, fgs);   // also Z_j = fz
                        fgmres_orth(c, w, N, fgs, c->fv);
                        launch_k(k_loop_ctl, 1, 1, 0, c->st, L2, GM_M + 1, &fgs->cycle_end);
                        CKL();
                    });
                launch_k(k_gm_solve, 1, 256, 0, c->st, fgs, nullptr);
                launch_k(k_gm_combine<double>, g, VEC_THREADS, 0, c->st, c->fZ, u, N, fgs);
                launch_k(k_vec_add, g, VEC_THREADS, 0, c->st, u, x, N);
                residual(0);
                launch_k(k_gm_loop_ctl, 1, 1, 0, c->st, L, maxit + 2, fgs, 0);
                CKL();
            });
        launch_k(k_count_stage, 1, 1, 0, c->st, c->dcnt, fgs);
        CKL();
    }

    // device counters of a graph launch -> stats; errors the device recorded
    static void graph_stats(hdg_ctx *c, int static_kernels) {
        const DevCount &D = *c->hcnt;
        c->S.stepI_iters += (int)D.stepI_iters;
        c->S.stepI_solves += (int)D.stepI_solves;
        c->S.trace_iters += (int)D.trace_iters;
        c->S.trace_solves += (int)D.trace_solves;
        c->S.richardson_iters += (int)D.outer_iters;
        c->S.stage_solves += (int)D.stage_solves;
        c->S.graph_kernels += (long long)static_kernels + (long long)D.launches;
        c->S.stage_products32 += D.products32;
        if (D.breakdowns) throw std::domain_error("device-side solve: non-finite residual");
    }

    static void launch_counted(hdg_ctx *c, cudaGraphExec_t ex) {
        CK(cudaMemsetAsync(c->dcnt, 0, sizeof(DevCount), c->st));
        CK(cudaGraphLaunch(ex, c->st));
        CK(cudaMemcpyAsync(c->hcnt, c->dcnt, sizeof(DevCount), cudaMemcpyDeviceToHost, c->st));
    }

    // Stage solve to tolerance: flexible GMRES(GM_M) on A(c) x = (r, 0, 0) right-preconditioned by
    // the Chorin split (Alg. 2's preconditioner; plain Alg. 2 is its Richardson iteration).
    static int stage_fgmres(hdg_ctx *c, double cc, const double *r, const double *Qsv, double *Q, double *p,
                            double *lam) {
        assemble_stepI(c, Qsv, cc, inv_for(c, c->P.inner_stepI_rtol) | (relax_on(c) ? BLK32 : 0));
        ensure_pre_maps(c, cc);
        CondCache &E = condense(c, cc);
        if (!c->capturing) {
            int hstat = 0;
            CK(cudaMemcpyAsync(&hstat, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            if (hstat) throw std::domain_error("singular tentative-velocity block");
        }
        const long long N = c->nQ + c->nPv + c->nL;
        const int g = grid_for(N);
        double *x = c->fx, *b = c->fb, *w = c->fw, *res = c->fr, *u = c->fu;
        // x = (Q, p, lam), b = (r, 0, 0)
        CK(cudaMemcpyAsync(x, Q, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(x + c->nQ, p, 8 * c->nPv, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(x + c->nQ + c->nPv, lam, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(b, r, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemsetAsync(b + c->nQ, 0, 8 * (c->nPv + c->nL), c->st));
        if (c->capturing || c->P.device_loops) {
            if (c->capturing) {
                stage_fgmres_capture(c, cc);
            } else {
                if (!E.g_stage) E.g_stage = capture_graph(c, [&]() { stage_fgmres_capture(c, cc); }, &E.stage_kernels);
                launch_counted(c, E.g_stage);
                CK(cudaMemcpyAsync(c->hfgs, c->fgs, sizeof(GmresState), cudaMemcpyDeviceToHost, c->st));
                CK(cudaStreamSynchronize(c->st));
                graph_stats(c, E.stage_kernels);
                c->S.last_update_norm = c->hfgs->bnorm > 0 ? c->hfgs->resid / c->hfgs->bnorm : 0.0;
            }
            CK(cudaMemcpyAsync(Q, x, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
            CK(cudaMemcpyAsync(p, x + c->nQ, 8 * c->nPv, cudaMemcpyDeviceToDevice, c->st));
            CK(cudaMemcpyAsync(lam, x + c->nQ + c->nPv, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
            mean_shift(c, p, lam);
            return c->capturing ? 0 : (c->hfgs->converged ? 0 : 1);
        }
        launch_k(k_vec_norm_into, g, VEC_THREADS, 0, c->st, b, N, c->rb(), c->fgs);
        CKL();
        int outer = 0, converged = 0;
        for (int cyc = 0; cyc < 1000; ++cyc) {
            stage_apply(c, cc, x, w);                                            // res = b - A x
            CK(cudaMemcpyAsync(res, b, 8 * N, cudaMemcpyDeviceToDevice, c->st));
            launch_k(k_axpby, g, VEC_THREADS, 0, c->st, -1.0, w, 1.0, res, N);
            launch_k(k_vec_start, g, VEC_THREADS, 0, c->st, res, N, cyc == 0 ? 2 : 0, c->rb(), c->fgs,
                                                     c->P.richardson_rtol, c->P.richardson_max, relax_of(c));
            launch_k(k_gm_set_cycle, 1, 1, 0, c->st, c->fgs, GM_M);
            CKL();
            CK(cudaMemcpyAsync(c->hfgs, c->fgs, sizeof(GmresState), cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            if (c->hfgs->breakdown == 2) throw std::domain_error("stage FGMRES: non-finite residual");
            if (c->hfgs->converged) { converged = 1; break; }
            launch_k(k_vec_normalize, g, VEC_THREADS, 0, c->st, res, w, c->fV, nullptr, N, c->fgs, fV32(c));   // V_0
            CKL();
            for (int j = 0; j < GM_M; ++j) {
                double *Vj = c->fV + (size_t)j * N, *Zj = c->fZ + (size_t)j * N;
                chorin_precond(c, cc, Vj, Zj);
                if (relax_on(c) && c->hfgs->lowprec) c->S.stage_products32 += 1;    // the state read last
                stage_apply(c, cc, Zj, w, fw32(c), nullptr, nullptr, c->fgs);
                fgmres_orth(c, w, N, c->fgs, nullptr);
                CKL();
                CK(cudaMemcpyAsync(c->hfgs, c->fgs, sizeof(GmresState), cudaMemcpyDeviceToHost, c->st));
                CK(cudaStreamSynchronize(c->st));
                ++outer;
                if (c->hfgs->breakdown == 2) throw std::domain_error("stage FGMRES: non-finite residual");
                if (c->hfgs->cycle_end) break;
            }
            launch_k(k_gm_solve, 1, 256, 0, c->st, c->fgs, nullptr);
            launch_k(k_gm_combine<double>, g, VEC_THREADS, 0, c->st, c->fZ, u, N, c->fgs);
            launch_k(k_vec_add, g, VEC_THREADS, 0, c->st, u, x, N);
            CKL();
            // the next pass forms the residual in FP64 and decides convergence on it
            if (outer >= c->P.richardson_max) break;
        }
        CK(cudaMemcpyAsync(Q, x, 8 * c->nQ, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(p, x + c->nQ, 8 * c->nPv, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(lam, x + c->nQ + c->nPv, 8 * c->nL, cudaMemcpyDeviceToDevice, c->st));
        mean_shift(c, p, lam);
        c->S.richardson_iters += outer;
        c->S.stage_solves += 1;
        c->S.last_update_norm = c->hfgs->bnorm > 0 ? c->hfgs->resid / c->hfgs->bnorm : 0.0;
        return converged ? 0 : 1;
    }

    // A stage solve in the configured mode: fixed n_R (Alg. 2 as printed), Alg. 2 to tolerance,
    // or Alg. 2's preconditioner inside flexible GMRES to tolerance.
    static int stage_solve(hdg_ctx *c, double cc, const double *r, const double *Qsv, double *Q, double *p,
                           double *lam) {
        if (c->P.n_richardson <= 0 && c->P.stage_krylov) return stage_fgmres(c, cc, r, Qsv, Q, p, lam);
        return richardson(c, cc, r, Qsv, Q, p, lam);
    }

    static void bdm(hdg_ctx *c, const double *Q, double *Qs) {
        CompTimer tm_(c, &c->S.ms_bdm);
        bdm_launch(c, Q, Qs);
    }
    // the BDM kernel: in pairs under HDG_MIXED (k_bdm_f2), FP64 otherwise
    static void bdm_launch(hdg_ctx *c, const double *Q, double *Qs) {
        unsigned nb = cell_blocks(c);
        if (c->P.precision == HDG_MIXED)
            launch_k(k_bdm_f2<K>, nb, 128, sizeof(f2) * TEAMS_PER_BLOCK * bdm_f2_scratch<K_>(), c->st,
                     BdmF2{c->ephi2a, c->fw2, c->leg2, c->Iv2, c->bdminv2}, c->M, Q, Qs);
        else
            launch_k(k_bdm<K>, nb, 128, sizeof(double) * TEAMS_PER_BLOCK * bdm_scratch<K_>(), c->st, c->R, c->M, Q, Qs);
        CKL();
    }

    // f^impl(w, Q, P(Q)) + phi(t) (w.F) as a dual vector, using the Step-I buffers (c = 1)
    static void fimpl_dual(hdg_ctx *c, const double *Q, const double *Qs, double tt, double *out) {
        assemble_stepI(c, Qs, 1.0, 0);
        cell_apply(c, Q, c->q[6]);
        LinComb L = lincomb();
        L.nterms = 2;
        L.coef[0] = 1.0; L.vec[0] = Q; L.mass[0] = 1;
        L.coef[1] = -1.0; L.vec[1] = c->q[6];
        if (c->has_forcing) {
            L.nterms = 3;
            L.vec[2] = c->Fload;
            if (c->capturing) {         // phi(t) from the step's device values
                L.coef[2] = 1.0; L.fterm = 2; L.fscale = c->dfv + 7;
            } else {
                L.coef[2] = c->phi ? c->phi(tt, c->phi_user) : 1.0;
            }
        }
        launch_k(k_lincomb, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, NU, L, out, c->ncells);
        CKL();
    }

    // Sec. 2.7: (U.w) - g(w,p,l) = f^impl(w,Q,P(Q)) + (w.f(t)), Gamma(U,p,l) = 0
    static void reconstruct(hdg_ctx *c, const double *Q, double tt, double *p, double *lam) {
        double *Qs = c->q[5], *Ru = c->q[7];
        bdm(c, Q, Qs);
        fimpl_dual(c, Q, Qs, tt, Ru);
        mixed_solve(c, 1.0, Ru, nullptr, nullptr, nullptr, c->q[4], p, lam);
        mean_shift(c, p, lam);
    }

    // ---------------------------------------------------------------- tracer (App. B)
    // U = P_CG(Q) in each cell's modal basis (Q modal): Jacobi-preconditioned CG to 1e-13 on the
    // continuous space, a device-side loop when recording a graph
    static void cg_project(hdg_ctx *c, const double *Qm, double *Um) {
        const CGMap &C = c->cgm;
        const long long n2 = 2LL * C.npts;
        const int g = grid_for(n2);
        const unsigned cb = cell_blocks(c);
        const size_t smem = sizeof(double) * TEAMS_PER_BLOCK * 4 * MU;
        launch_k(k_cgp_rhs, grid_for(n2), VEC_THREADS, 0, c->st, c->geo, c->R.nod_u, C, Qm, c->cg_b);
        launch_k(k_cgp_start, g, VEC_THREADS, 0, c->st, C, (const double *)c->cg_b, c->cg_u, c->cg_r, c->cg_z, c->rb(),
                 c->sc, 1e-13, 400);
        auto iteration = [&]() {
            launch_k(k_cgp_cell<K>, cb, 128, smem, c->st, c->M, c->R.nod_u, C, (const double *)c->cg_z,
                     (const double *)c->cg_p, c->cg_w, (const Scalars *)c->sc);
            launch_k(k_cgp_gather, g, VEC_THREADS, 0, c->st, C, (const double *)c->cg_w, (const double *)c->cg_z, c->cg_p,
                     c->cg_Ap, c->rb(), c->sc);
            launch_k(k_cgp_update, g, VEC_THREADS, 0, c->st, C, (const double *)c->cg_p, (const double *)c->cg_Ap,
                     c->cg_u, c->cg_r, c->cg_z, c->rb(), c->sc);
        };
        if (c->capturing) {
            capture_while(
                c, [&](LoopCtl L) { launch_k(k_loop_init, 1, 1, 0, c->st, L, &c->sc->done); },
                [&](LoopCtl L) {
                    iteration();
                    iteration();
                    launch_k(k_loop_ctl, 1, 1, 0, c->st, L, 400 / 2 + 2, &c->sc->done);
                });
        } else {
            for (int chunk = 0;; ++chunk) {
                if (chunk > 400 / 8 + 2) throw std::length_error("P_CG: no convergence flag from the device");
                for (int it = 0; it < 8; ++it) iteration();
                CKL();
                read_scalars(c);
                if (c->hsc->done) break;
            }
            if (c->hsc->breakdown == 2) throw std::domain_error("P_CG: non-finite residual");
        }
        launch_k(k_cgp_to_modal<K>, grid_for((long long)c->ncells * 2 * MU), VEC_THREADS, 0, c->st, c->R.nod_u, C,
                 (const double *)c->cg_u, Um);
        CKL();
    }

    static void tracer_rhs(hdg_ctx *c, const double *q, const double *Um, double *out) {
        launch_k(k_tracer_rhs<K>, cell_blocks(c), 128, sizeof(double) * TEAMS_PER_BLOCK * (3 * Dm::NQ + 3 * Dm::NFQ),
                 c->st, c->R, c->M, q, Um, out);
        CKL();
    }

    // eq. advection_update_stages / eq. advection_update_final with the explicit tableau, advected
    // by P_CG of the step's stage velocities (Q_0 = Q^n for an explicit first stage); the final sum
    // includes i = 0 (see hdg.h)
    static void tracer_step(hdg_ctx *c) {
        const Tab &T = c->tab;
        const double dt = c->P.dt;
        const int s = T.s;
        for (int i = 0; i < s; ++i) {
            bool need = T.be[i] != 0.0;
            for (int r = i + 1; r < s; ++r) need = need || T.Ae[r][i] != 0.0;
            const double *qi = c->qtr;
            LinComb L = lincomb();
            int n = 0;
            L.coef[n] = 1.0; L.vec[n] = c->qtr; L.mass[n] = 0; ++n;
            for (int j = 0; j < i; ++j)
                if (T.Ae[i][j] != 0.0) { L.coef[n] = dt * T.Ae[i][j]; L.vec[n] = c->tr_dq[j]; L.mass[n] = 0; ++n; }
            if (n > 1 && need) {
                L.nterms = n;
                launch_k(k_lincomb, grid_for(c->nPv), VEC_THREADS, 0, c->st, c->geo, NP, L, c->tr_q, c->ncells);
                CKL();
                qi = c->tr_q;
            }
            if (!need) continue;
            cg_project(c, c->Qs[i], c->tr_U);
            tracer_rhs(c, qi, c->tr_U, c->tr_dq[i]);
        }
        LinComb L = lincomb();
        int n = 0;
        L.coef[n] = 1.0; L.vec[n] = c->qtr; L.mass[n] = 0; ++n;
        for (int i = 0; i < s; ++i)
            if (T.be[i] != 0.0) { L.coef[n] = dt * T.be[i]; L.vec[n] = c->tr_dq[i]; L.mass[n] = 0; ++n; }
        L.nterms = n;
        launch_k(k_lincomb, grid_for(c->nPv), VEC_THREADS, 0, c->st, c->geo, NP, L, c->qtr, c->ncells);
        CKL();
    }

    // Time factors of the forcing f(t) = phi(t) F for the step from t0: out[i] = dt sum_j a^ex_ij
    // phi(t0 + c_j dt) for stage i (eq. imex_residual), out[s] = dt sum_i b^ex_i phi(t0 + c_i dt)
    // (eq. final_residual), out[7] = phi(t0 + dt) (the reconstruction at the new time).
    static void forcing_values(const hdg_ctx *c, double t0, double out[8]) {
        const Tab &T = c->tab;
        const double dt = c->P.dt;
        for (int i = 0; i < 8; ++i) out[i] = 0.0;
        if (!c->has_forcing) return;
        auto phi = [&](double t) { return c->phi ? c->phi(t, c->phi_user) : 1.0; };
        double ph[4] = {0, 0, 0, 0};
        for (int j = 0; j < T.s; ++j) ph[j] = phi(t0 + T.c[j] * dt);
        for (int i = 1; i < T.s; ++i)
            for (int j = 0; j < i; ++j) out[i] += dt * T.Ae[i][j] * ph[j];
        for (int i = 0; i < T.s; ++i) out[T.s] += dt * T.be[i] * ph[i];
        out[7] = phi(t0 + dt);
    }

    // ---------------------------------------------------------------- Alg. 1
    // One step from t0 (c->t is not advanced here). Inside a graph capture every solve is recorded
    // with device-side loops and the return value is 0 (non-convergence is counted on the device).
    // Stage initial guesses across steps (stages solved to a tolerance only: a fixed number of
    // Richardson sweeps, Alg. 2 as printed with n_richardson > 0, starts from the previous stage's
    // solution, and its result depends on that start). keep = false (step start): with history,
    // the velocity guess of each implicit stage i >= i0 is its solution in the previous step plus
    // the state's change over that step (k_stage_guess); its pressure and trace guesses extrapolate
    // the stage's own solutions of the last two steps linearly (k_stage_guess_self; after one kept
    // step, the last solution). Without history each stage starts from the previous stage's
    // solution (k_copy_unless in the stage loop). keep = true (after the stage solves): the
    // solutions are kept and the count of kept steps raised. The count is a device value, so the
    // recorded step graph takes every form; an entry point that sets the state from outside a
    // step clears it unless the state is the one the last step left.
    static void stage_guesses(hdg_ctx *c, int i0, bool keep) {
        if (c->P.n_richardson > 0) return;          // the count stays zero
        const int s = c->tab.s;
        StageVecs SQ{}, SP{}, SL{};
        for (int i = i0; i < s; ++i) {
            const int k = SQ.n++;
            SP.n++; SL.n++;
            SP.aux[k] = c->H2ps[i]; SL.aux[k] = c->H2ls[i];
            if (keep) {
                SQ.dst[k] = c->HQs[i]; SQ.src[k] = c->Qs[i];
                SP.dst[k] = c->Hps[i]; SP.src[k] = c->ps[i];
                SL.dst[k] = c->Hls[i]; SL.src[k] = c->ls[i];
            } else {
                SQ.dst[k] = c->Qs[i]; SQ.src[k] = c->HQs[i];
                SP.dst[k] = c->ps[i]; SP.src[k] = c->Hps[i];
                SL.dst[k] = c->ls[i]; SL.src[k] = c->Hls[i];
            }
        }
        if (keep) {
            launch_k(k_stage_keep, grid_for(c->nQ), VEC_THREADS, 0, c->st, SQ, c->nQ, c->dhist, 0);
            launch_k(k_stage_keep, grid_for(c->nPv), VEC_THREADS, 0, c->st, SP, c->nPv, c->dhist, 0);
            launch_k(k_stage_keep, grid_for(c->nL), VEC_THREADS, 0, c->st, SL, c->nL, c->dhist, 1);
        } else {
            launch_k(k_stage_guess, grid_for(c->nQ), VEC_THREADS, 0, c->st, (const int *)c->dhist, (const double *)c->Q,
                     c->Qprev, SQ, c->nQ);
            launch_k(k_stage_guess_self, grid_for(c->nPv), VEC_THREADS, 0, c->st, (const int *)c->dhist, SP, c->nPv);
            launch_k(k_stage_guess_self, grid_for(c->nL), VEC_THREADS, 0, c->st, (const int *)c->dhist, SL, c->nL);
        }
        CKL();
    }

    static int imex_step_body(hdg_ctx *c, double t0) {
        const Tab &T = c->tab;
        const double dt = c->P.dt;
        const int s = T.s;
        double fv[8];
        forcing_values(c, t0, fv);
        size_t bq = sizeof(double) * c->nQ;
        CK(cudaMemcpyAsync(c->Qs[0], c->Q, bq, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(c->ps[0], c->p, sizeof(double) * c->nPv, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(c->ls[0], c->lam, sizeof(double) * c->nL, cudaMemcpyDeviceToDevice, c->st));
        int nc = 0;
        // stages with a_ii != 0 are solved; the first stage is explicit (Q_0 = Q^n, Alg. 1) unless
        // the tableau has a_00 != 0 (SSP2(3,3,2), SSP3(4,3,3)): then it is solved too, advected by
        // P(Q^n), and every sum below runs over all implicit stages. M Q^n is read from the state,
        // which the step overwrites only in the final update.
        const int i0 = T.Ai[0][0] != 0.0 ? 0 : 1;
        stage_guesses(c, i0, false);                // from the previous step, when it left them
        for (int i = i0; i < s; ++i) {
            // eq. imex_residual: r_i = M Q^n + sum_j (a_ij/a_jj)(M Q_j - r_j) + dt sum_j aex_ij (w.f_j)
            LinComb L = lincomb();
            int n = 0;
            L.coef[n] = 1.0; L.vec[n] = c->Q; L.mass[n] = 1; ++n;
            for (int j = i0; j < i; ++j) {
                double w = T.Ai[i][j] / T.Ai[j][j];
                if (w == 0.0) continue;
                L.coef[n] = w; L.vec[n] = c->Qs[j]; L.mass[n] = 1; ++n;
                L.coef[n] = -w; L.vec[n] = c->rs[j]; L.mass[n] = 0; ++n;
            }
            if (c->has_forcing && c->capturing) {
                L.coef[n] = 1.0; L.vec[n] = c->Fload; L.mass[n] = 0; L.fterm = n; L.fscale = c->dfv + i; ++n;
            } else if (c->has_forcing && fv[i] != 0.0) {
                L.coef[n] = fv[i]; L.vec[n] = c->Fload; L.mass[n] = 0; ++n;
            }
            L.nterms = n;
            launch_k(k_lincomb, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, NU, L, c->rs[i], c->ncells);
            CKL();
            if (i > 0) {
                bdm(c, c->Qs[i - 1], c->q[5]);                                   // Q*_{i-1}
                // without history the stage starts from the previous stage's solution
                launch_k(k_copy_unless, grid_for(c->nQ), VEC_THREADS, 0, c->st, (const int *)c->dhist,
                         (const double *)c->Qs[i - 1], c->Qs[i], c->nQ);
                launch_k(k_copy_unless, grid_for(c->nPv), VEC_THREADS, 0, c->st, (const int *)c->dhist,
                         (const double *)c->ps[i - 1], c->ps[i], c->nPv);
                launch_k(k_copy_unless, grid_for(c->nL), VEC_THREADS, 0, c->st, (const int *)c->dhist,
                         (const double *)c->ls[i - 1], c->ls[i], c->nL);
                CKL();
            } else {
                bdm(c, c->Q, c->q[5]);                                           // P(Q^n); Q_0 starts at Q^n
            }
            nc |= stage_solve(c, T.Ai[i][i] * dt, c->rs[i], c->q[5], c->Qs[i], c->ps[i], c->ls[i]);
        }
        stage_guesses(c, i0, true);                 // this step's stage solutions kept
        // eq. final_residual and eq. final_update (coefficient b_{s-1}^im dt)
        LinComb L = lincomb();
        int n = 0;
        L.coef[n] = 1.0; L.vec[n] = c->Q; L.mass[n] = 1; ++n;
        for (int i = i0; i < s; ++i) {
            double w = T.bi[i] / T.Ai[i][i];
            if (w == 0.0) continue;
            L.coef[n] = w; L.vec[n] = c->Qs[i]; L.mass[n] = 1; ++n;
            L.coef[n] = -w; L.vec[n] = c->rs[i]; L.mass[n] = 0; ++n;
        }
        if (c->has_forcing && c->capturing) {
            L.coef[n] = 1.0; L.vec[n] = c->Fload; L.mass[n] = 0; L.fterm = n; L.fscale = c->dfv + s; ++n;
        } else if (c->has_forcing && fv[s] != 0.0) {
            L.coef[n] = fv[s]; L.vec[n] = c->Fload; L.mass[n] = 0; ++n;
        }
        L.nterms = n;
        double *rn = c->q[7];
        launch_k(k_lincomb, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, NU, L, rn, c->ncells);
        CKL();
        mixed_solve(c, dt * T.bi[s - 1], rn, nullptr, nullptr, nullptr, c->Q, c->pp[1], c->ll[1]);
        reconstruct(c, c->Q, t0 + dt, c->p, c->lam);                            // Sec. 2.7
        if (c->has_tracer) tracer_step(c);                                       // App. B
        if (c->P.n_richardson <= 0)                 // the state this step leaves (see hdg_set_state)
            CK(cudaMemcpyAsync(c->Qlast, c->Q, sizeof(double) * c->nQ, cudaMemcpyDeviceToDevice, c->st));
        return nc;
    }

    // The step as one CUDA graph: stages solved by flexible GMRES with device-side loops; the
    // forcing's time factors are device values refreshed before each launch.
    static bool step_graph_ok(const hdg_ctx *c) {
        return c->P.device_loops && c->P.n_richardson <= 0 && c->P.stage_krylov;
    }

    // One step as the graph: prepare (first call: condensations and capture) and enqueue it on the
    // context's stream without waiting; step_finish waits for it and does the bookkeeping.
    static void step_enqueue(hdg_ctx *c) {
        const double t0 = c->t, dt = c->P.dt;
        if (!c->g_step) {
            const Tab &T = c->tab;                      // condensations the step uses, built first
            for (int i = 0; i < T.s; ++i)
                if (T.Ai[i][i] != 0.0) ensure_pre_maps(c, T.Ai[i][i] * dt);
            condense(c, dt * T.bi[T.s - 1]);
            condense(c, 1.0);
            c->g_step = capture_graph(c, [&]() { imex_step_body(c, t0); }, &c->step_kernels);
        }
        if (c->has_forcing) {                           // this step's forcing time factors
            forcing_values(c, t0, c->hfv);
            CK(cudaMemcpyAsync(c->dfv, c->hfv, 8 * sizeof(double), cudaMemcpyHostToDevice, c->st));
        }
        CK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->st));
        c->deadline = c->P.timeout_ms > 0 ? now_ms() + c->P.timeout_ms : 0;   // counted from the launch
        launch_counted(c, c->g_step);
        CK(cudaMemcpyAsync(c->hstat, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        c->pending = true;
        c->pending_t = t0 + dt;
    }

    static int step_finish(hdg_ctx *c) {
        wait_stream(c);
        c->pending = false;
        c->deadline = 0;
        const int hstat = *c->hstat;
        if (hstat) throw std::domain_error("singular tentative-velocity block");
        graph_stats(c, c->step_kernels);
        c->t = c->pending_t;
        return c->hcnt->stage_unconverged ? 1 : 0;
    }

    static int imex_step(hdg_ctx *c) {
        const double t0 = c->t, dt = c->P.dt;
        if (!step_graph_ok(c)) {
            int nc = imex_step_body(c, t0);
            c->t = t0 + dt;
            return nc;
        }
        step_enqueue(c);
        return step_finish(c);
    }
};

// A step that timed out in an earlier call: wait for it without a limit, then apply its bookkeeping.
void settle_pending(hdg_ctx *c) {
    if (!c->pending) return;
    CK(cudaStreamSynchronize(c->st));
    c->pending = false;
    c->t = c->pending_t;
}

hdg_status map_exception() {
    try {
        throw;
    } catch (const OomError &e) {
        g_last_error = e.what();
        return HDG_ERR_OOM;
    } catch (const CudaError &e) {
        g_last_error = e.what();
        return HDG_ERR_CUDA;
    } catch (const TimeoutError &e) {
        g_last_error = e.what();
        return HDG_ERR_TIMEOUT;
    } catch (const std::length_error &e) {
        g_last_error = e.what();
        return HDG_ERR_NOT_CONVERGED;
    } catch (const std::domain_error &e) {
        g_last_error = e.what();
        return HDG_ERR_NUMERIC;
    } catch (const std::invalid_argument &e) {
        g_last_error = e.what();
        return HDG_ERR_INVALID_ARG;
    } catch (const std::bad_alloc &e) {
        g_last_error = e.what();
        return HDG_ERR_OOM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return HDG_ERR_INVALID_ARG;
    }
}

#define DISPATCH(ctx, ...)                                                     \
    switch ((ctx)->K) {                                                        \
        case 1: { typedef Impl<1> I; __VA_ARGS__; } break;                     \
        case 2: { typedef Impl<2> I; __VA_ARGS__; } break;                     \
        case 3: { typedef Impl<3> I; __VA_ARGS__; } break;                     \
        case 4: { typedef Impl<4> I; __VA_ARGS__; } break;                     \
        default: throw std::invalid_argument("unsupported degree");            \
    }

void begin_call(hdg_ctx *c) {
    g_last_error.clear();
    settle_pending(c);
    c->S = hdg_stats{};
    CK(cudaEventRecord(c->e0, c->st));
}
// HDG_ERR_NOT_CONVERGED with its message (the state keeps the last iterate)
hdg_status not_converged(const char *where) {
    g_last_error = std::string(where) + ": a stage solve did not reach richardson_rtol within richardson_max iterations";
    return HDG_ERR_NOT_CONVERGED;
}
void end_call(hdg_ctx *c, hdg_stats *out) {
    CK(cudaEventRecord(c->e1, c->st));
    CK(cudaEventSynchronize(c->e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->e0, c->e1));
    c->S.ms_total = ms;
    if (out) *out = c->S;
}


}  // namespace

// =========================================================================== C-ABI
extern "C" {

void hdg_default_params(hdg_params *p) {
    if (!p) return;
    p->k = 2;
    p->alpha = 1.0;
    p->tau = 1.0;
    p->delta_up = 1.0;
    p->tableau = HDG_ARS222;
    p->dt = 0.01;
    p->n_richardson = 2;
    p->richardson_rtol = 1e-10;
    p->richardson_max = 50;
    p->trace_rtol = 1e-12;
    p->stepI_rtol = 1e-10;
    p->max_iters = 5000;
    p->stage_krylov = 1;
    p->inner_stepI_rtol = 2e-2;
    p->inner_trace_rtol = 1e-1;
    p->trace_mg = 1;
    p->device_loops = 1;
    p->inner_trace_vcycles = 1;
    p->precision = HDG_MIXED;
    p->timeout_ms = 0.0;
    p->relax_eta = 1e-5;
    p->inner_trace_fp32 = 1;
    p->trace_fp32_vcycle = 1;
    p->inner_gs = 1;
}

const char *hdg_status_string(hdg_status s) {
    switch (s) {
        case HDG_OK: return "ok";
        case HDG_ERR_INVALID_ARG: return "invalid argument";
        case HDG_ERR_CUDA: return "CUDA error";
        case HDG_ERR_OOM: return "out of device memory";
        case HDG_ERR_NOT_CONVERGED: return "iteration did not converge";
        case HDG_ERR_NUMERIC: return "non-finite value";
        case HDG_ERR_UNSUPPORTED: return "unsupported";
        case HDG_ERR_TIMEOUT: return "timed out";
    }
    return "unknown status";
}

const char *hdg_last_error(void) { return g_last_error.c_str(); }

hdg_status hdg_mesh_counts(const hdg_mesh_desc *mesh, int k, int64_t *ncells, int64_t *nfacets) {
    if (!mesh || mesh->n < 1 || k < 1 || k > 4) return HDG_ERR_INVALID_ARG;
    if (ncells) *ncells = 2LL * mesh->n * mesh->n;
    if (nfacets) *nfacets = mesh_facet_count(mesh->n, mesh->periodic_x != 0, mesh->periodic_y != 0);
    return HDG_OK;
}

hdg_status hdg_reference_rule(int k, int which, double *pts, double *wts, int *npts) {
    if (k < 1 || k > 4 || !npts || (which != 0 && which != 1)) return HDG_ERR_INVALID_ARG;
    try {
        if (which == 0) {
            std::vector<double> x, y, w;
            int n = triangle_rule(volume_points_1d(k), x, y, w);
            if (pts && wts) {
                if (*npts < n) return HDG_ERR_INVALID_ARG;
                for (int i = 0; i < n; ++i) { pts[2 * i] = x[i]; pts[2 * i + 1] = y[i]; wts[i] = w[i]; }
            }
            *npts = n;
        } else {
            int n = facet_points(k);
            if (pts && wts) {
                if (*npts < n) return HDG_ERR_INVALID_ARG;
                gauss_legendre01(n, pts, wts);
            }
            *npts = n;
        }
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_reference_basis(int m, int npts, const double *pts, double *vals) {
    if (m < 0 || m > 8 || npts < 0 || (npts > 0 && (!pts || !vals))) return HDG_ERR_INVALID_ARG;
    int d = dim_P(m);
    for (int i = 0; i < npts; ++i) dubiner(m, pts[2 * i], pts[2 * i + 1], vals + (size_t)i * d, nullptr);
    return HDG_OK;
}

hdg_status hdg_setup_mesh(hdg_ctx **out, const hdg_mesh_desc *mesh, const hdg_params *params,
                          void *cuda_stream) {
    if (!out || !mesh || !params) return HDG_ERR_INVALID_ARG;
    *out = nullptr;
    if (mesh->n < 1 || mesh->n > 4096 || !(mesh->Lx > 0) || !(mesh->Ly > 0)) return HDG_ERR_INVALID_ARG;
    if (params->k < 1 || params->k > 4 || !(params->dt > 0) || !(params->tau > 0) || params->alpha < 0 ||
        params->delta_up < 0 || params->max_iters < 1 || !(params->trace_rtol > 0) || !(params->stepI_rtol > 0))
        return HDG_ERR_INVALID_ARG;
    if (params->n_richardson <= 0 && (!(params->richardson_rtol > 0) || params->richardson_max < 1))
        return HDG_ERR_INVALID_ARG;
    if (params->n_richardson <= 0 && params->stage_krylov &&
        (!(params->inner_stepI_rtol > 0) || !(params->inner_trace_rtol > 0)))
        return HDG_ERR_INVALID_ARG;
    if (params->tableau < HDG_ARS222 || params->tableau > HDG_SSP3_433) return HDG_ERR_INVALID_ARG;
    if (params->precision != HDG_FP64 && params->precision != HDG_MIXED) return HDG_ERR_INVALID_ARG;
    if (!(params->timeout_ms >= 0)) return HDG_ERR_INVALID_ARG;
    if (!(params->relax_eta >= 0) || !std::isfinite(params->relax_eta)) return HDG_ERR_INVALID_ARG;
    hdg_ctx *c = new (std::nothrow) hdg_ctx();
    if (!c) return HDG_ERR_OOM;
    try {
        c->P = *params;
        c->D = *mesh;
        c->st = (cudaStream_t)cuda_stream;
        CK(cudaGetDevice(&c->device));
        if (c->P.precision == HDG_FP64) {        // every part of the path in FP64
            c->P.inner_trace_fp32 = 0;
            c->P.trace_fp32_vcycle = 0;
        }
        c->tab = make_tableau(params->tableau);
        c->T = build_tables(params->k);
        c->H = build_mesh(mesh->n, mesh->Lx, mesh->Ly, mesh->periodic_x != 0, mesh->periodic_y != 0);
        // every neighbour of the other parity? (and cells in fours, so that the two teams of a warp in
        // the colour kernels are both in range or both out: their team syncs are whole-warp)
        c->gs_ok = c->H.ncells % 4 == 0;
        for (int k = 0; k < c->H.ncells && c->gs_ok; ++k)
            for (int e = 0; e < 3; ++e) {
                const int o = c->H.cell_nbr[3 * k + e];
                if (o >= 0 && (o & 1) == (k & 1)) { c->gs_ok = false; break; }
            }
        c->K = params->k;
        c->MU = c->T.mu; c->NU = 2 * c->T.mu; c->NP = c->T.np; c->NT = c->T.nt; c->NL = 3 * c->T.nt;
        c->ncells = c->H.ncells;
        c->nfacets = c->H.nfacets;
        c->nQ = c->ncells * c->NU;
        c->nPv = c->ncells * c->NP;
        c->nL = c->nfacets * c->NT;
        c->area = mesh->Lx * mesh->Ly;
        // reference tables: one allocation
        const RefTables &T = c->T;
        std::vector<const std::vector<double> *> tabs = {&T.qw, &T.phi, &T.dphi, &T.fw, &T.ephi, &T.leg,
                                                         &T.Dhat, &T.Ehat, &T.Tpp, &T.bdm_inv, &T.Iv, &T.nod_u,
                                                         &T.nod_p, &T.mod_u, &T.mod_p, &T.nod_t, &T.mod_t,
                                                         &T.Sfac, &T.Tadv};
        size_t tot = 0;
        for (auto *v : tabs) tot += v->size();
        std::vector<double> hbuf;
        hbuf.reserve(tot);
        std::vector<size_t> offs;
        for (auto *v : tabs) { offs.push_back(hbuf.size()); hbuf.insert(hbuf.end(), v->begin(), v->end()); }
        c->dref = c->alloc<double>(tot);
        CK(cudaMemcpy(c->dref, hbuf.data(), tot * sizeof(double), cudaMemcpyHostToDevice));
        const double **dst[] = {&c->R.qw, &c->R.phi, &c->R.dphi, &c->R.fw, &c->R.ephi, &c->R.leg, &c->R.Dhat,
                                &c->R.Ehat, &c->R.Tpp, &c->R.bdm_inv, &c->R.Iv, &c->R.nod_u, &c->R.nod_p,
                                &c->R.mod_u, &c->R.mod_p, &c->R.nod_t, &c->R.mod_t, &c->R.Sfac, &c->R.Tadv};
        for (size_t i = 0; i < tabs.size(); ++i) *dst[i] = c->dref + offs[i];
        {
            const size_t n = T.Tadv.size();
            std::vector<float> t2(2 * n);
            for (size_t i = 0; i < n; ++i) {
                const float h = (float)T.Tadv[i];
                t2[i] = h;
                t2[n + i] = (float)(T.Tadv[i] - (double)h);
            }
            c->Tadv2 = c->alloc<float>(2 * n);
            CK(cudaMemcpy(c->Tadv2, t2.data(), 2 * n * sizeof(float), cudaMemcpyHostToDevice));
            auto pairs = [&](const std::vector<double> &v) {
                std::vector<float2> f(v.size());
                for (size_t i = 0; i < v.size(); ++i) {
                    const float h = (float)v[i];
                    f[i] = make_float2(h, (float)(v[i] - (double)h));
                }
                float2 *d = c->alloc<float2>(f.size());
                CK(cudaMemcpy(d, f.data(), f.size() * sizeof(float2), cudaMemcpyHostToDevice));
                return d;
            };
            c->ephi2a = pairs(T.ephi);
            c->Sfac2 = pairs(T.Sfac);
            c->fw2 = pairs(T.fw);
            c->leg2 = pairs(T.leg);
            c->Iv2 = pairs(T.Iv);
            c->bdminv2 = pairs(T.bdm_inv);
        }
        // mesh
        c->geo = c->alloc<CellGeo>(c->ncells);
        CK(cudaMemcpy(c->geo, c->H.geo.data(), sizeof(CellGeo) * c->ncells, cudaMemcpyHostToDevice));
        auto up = [&](const std::vector<int> &v) {
            int *d = c->alloc<int>(v.size());
            CK(cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
            return (const int *)d;
        };
        c->M.geo = c->geo;
        c->M.cell_facet = up(c->H.cell_facet);
        c->M.cell_flip = up(c->H.cell_flip);
        c->M.cell_nbr = up(c->H.cell_nbr);
        c->M.cell_nbr_edge = up(c->H.cell_nbr_edge);
        c->M.facet_cell = up(c->H.facet_cell);
        c->M.facet_edge = up(c->H.facet_edge);
        c->M.ncells = (int)c->ncells;
        c->M.nfacets = (int)c->nfacets;
        if (c->H.p1_ok) {
            c->M.cell_vert = up(c->H.cell_vert);
            c->M.facet_vert = up(c->H.facet_vert);
            c->M.vert_facet = up(c->H.vert_facet);
            c->M.vert_fsign = up(c->H.vert_fsign);
            c->M.vert_cell = up(c->H.vert_cell);
            c->M.nverts = c->H.nverts;
        }
        // state and work buffers
        const size_t nQ = c->nQ, nP = c->nPv, nL = c->nL;
        c->Q = c->alloc<double>(nQ); c->p = c->alloc<double>(nP); c->lam = c->alloc<double>(nL);
        CK(cudaMemset(c->Q, 0, nQ * 8)); CK(cudaMemset(c->p, 0, nP * 8)); CK(cudaMemset(c->lam, 0, nL * 8));
        for (int i = 0; i < c->tab.s; ++i) {
            c->Qs.push_back(c->alloc<double>(nQ)); c->rs.push_back(c->alloc<double>(nQ));
            c->ps.push_back(c->alloc<double>(nP)); c->ls.push_back(c->alloc<double>(nL));
            c->HQs.push_back(c->alloc<double>(nQ)); c->Hps.push_back(c->alloc<double>(nP));
            c->Hls.push_back(c->alloc<double>(nL));
            c->H2ps.push_back(c->alloc<double>(nP)); c->H2ls.push_back(c->alloc<double>(nL));
        }
        c->Qprev = c->alloc<double>(nQ); c->Qlast = c->alloc<double>(nQ);
        c->dhist = c->alloc<int>(1);
        CK(cudaMemset(c->dhist, 0, sizeof(int)));
        c->dcheck = c->alloc<unsigned long long>(2);
        c->Fload = c->alloc<double>(nQ);
        c->dfv = c->alloc<double>(8);
        CK(cudaMallocHost(&c->hfv, 8 * sizeof(double)));
        const int nfq = (3 * c->K + 5) / 2;                      // facet points (Dims<K>::NFQ)
        c->Dblk = c->alloc<double>((size_t)c->NU * nQ);
        c->wq = c->alloc<double>((size_t)c->ncells * 3 * nfq);
        c->utr = c->alloc<double>((size_t)c->ncells * 3 * nfq * 2);
        c->pen = c->alloc<double>(nfq);
        c->pen32 = c->alloc<float>(nfq);
        {
            // the column-slice layout (block Jacobi) or the per-cell blocks of the red-black passes
            const size_t nup = (size_t)(c->NU + 3) / 4 * 4, blk = ((size_t)c->NU * nup + 31) / 32 * 32;
            c->Binv32 = c->alloc<float>(std::max((size_t)c->NU * nQ, blk * (size_t)c->ncells));
        }
        c->wq32 = c->alloc<float>((size_t)c->ncells * 3 * nfq);
        c->utr32 = c->alloc<float>((size_t)c->ncells * 3 * nfq * 2);
        c->gV32 = c->alloc<float>((size_t)(GM_M + 1) * nQ);
        c->gw32 = c->alloc<float>(nQ);
        c->gu32 = c->alloc<float>(nQ);
        {
            std::vector<float> e32(c->T.ephi.begin(), c->T.ephi.end());
            c->ephi32 = c->alloc<float>(e32.size());
            CK(cudaMemcpy(c->ephi32, e32.data(), e32.size() * sizeof(float), cudaMemcpyHostToDevice));
            std::vector<float> n32((size_t)6 * c->ncells);
            for (long long k = 0; k < c->ncells; ++k)
                for (int e = 0; e < 3; ++e) {
                    n32[6 * k + 2 * e] = (float)c->H.geo[k].nx[e];
                    n32[6 * k + 2 * e + 1] = (float)c->H.geo[k].ny[e];
                }
            c->nrm32 = c->alloc<float>(n32.size());
            CK(cudaMemcpy(c->nrm32, n32.data(), n32.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
        c->Binv = c->alloc<double>((size_t)c->NU * nQ);
        c->dstatus = c->alloc<int>(1);
        c->vK = c->alloc<double>((size_t)c->ncells * c->NL);
        c->wK = c->alloc<double>(nP);
        c->tb = c->alloc<double>(nL); c->tx = c->alloc<double>(nL); c->tr = c->alloc<double>(nL);
        c->tz = c->alloc<double>(nL); c->tp[0] = c->alloc<double>(nL); c->tp[1] = c->alloc<double>(nL);
        c->tAp = c->alloc<double>(nL);
        c->gV = c->alloc<double>((size_t)(GM_M + 1) * nQ);
        c->gw = c->alloc<double>(nQ); c->gz = c->alloc<double>(nQ); c->gu = c->alloc<double>(nQ);
        c->gb = c->alloc<double>(nQ); c->gx = c->alloc<double>(nQ);
        c->gs = c->alloc<GmresState>(1);
        CK(cudaMemset(c->gs, 0, sizeof(GmresState)));
        CK(cudaMallocHost(&c->hgs, sizeof(GmresState)));
        if (params->n_richardson <= 0 && params->stage_krylov) {
            const size_t N = nQ + nP + nL;
            c->fV = c->alloc<double>((size_t)(GM_M + 1) * N);
            c->fV32 = c->alloc<float>((size_t)(GM_M + 1) * N);
            c->fw32 = c->alloc<float>(N);
            c->fZ = c->alloc<double>((size_t)GM_M * N);
            c->fx = c->alloc<double>(N); c->fb = c->alloc<double>(N); c->fw = c->alloc<double>(N);
            c->fr = c->alloc<double>(N); c->fu = c->alloc<double>(N);
            c->fv = c->alloc<double>(N); c->fz = c->alloc<double>(N);
            c->fgs = c->alloc<GmresState>(1);
            CK(cudaMemset(c->fgs, 0, sizeof(GmresState)));
            CK(cudaMallocHost(&c->hfgs, sizeof(GmresState)));
            if (params->precision == HDG_MIXED && params->relax_eta > 0) {
                const size_t nup = (size_t)(c->NU + 3) / 4 * 4;       // the per-cell layout GsBlk
                c->Dblk32 = c->alloc<float>(((size_t)c->NU * nup + 31) / 32 * 32 * (size_t)c->ncells);
                std::vector<float> g32((size_t)GEO32 * c->ncells);
                for (long long k = 0; k < c->ncells; ++k) {
                    const CellGeo &G = c->H.geo[k];
                    float *o = &g32[(size_t)GEO32 * k];
                    for (int i = 0; i < 4; ++i) o[i] = (float)G.Jinv[i];
                    o[4] = (float)G.detJ;
                    for (int e = 0; e < 3; ++e) o[5 + e] = (float)G.h[e];
                }
                auto up32 = [&](const std::vector<double> &v) {
                    std::vector<float> f(v.begin(), v.end());
                    float *d = c->alloc<float>(f.size());
                    CK(cudaMemcpy(d, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
                    return d;
                };
                c->geo32 = c->alloc<float>(g32.size());
                CK(cudaMemcpy(c->geo32, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice));
                c->Dhat32 = up32(c->T.Dhat);
                c->Ehat32 = up32(c->T.Ehat);
                c->Dblk32lo = c->alloc<float>(((size_t)c->NU * nup + 31) / 32 * 32 * (size_t)c->ncells);
                auto up2 = [&](const std::vector<double> &v) {
                    std::vector<float2> f(v.size());
                    for (size_t i = 0; i < v.size(); ++i) {
                        const float h = (float)v[i];
                        f[i] = make_float2(h, (float)(v[i] - (double)h));
                    }
                    float2 *d = c->alloc<float2>(f.size());
                    CK(cudaMemcpy(d, f.data(), f.size() * sizeof(float2), cudaMemcpyHostToDevice));
                    return d;
                };
                c->ephi2 = up2(c->T.ephi);
                c->Ehat2 = up2(c->T.Ehat);
                c->Dhat2 = up2(c->T.Dhat);
            }
        }
        for (auto &x : c->q) x = c->alloc<double>(nQ);
        for (auto &x : c->pp) x = c->alloc<double>(nP);
        for (auto &x : c->ll) x = c->alloc<double>(nL);
        c->partials = c->alloc<double>((size_t)MAX_RED_BLOCKS * (GM_M + 2));
        c->counter = c->alloc<unsigned>(1);
        CK(cudaMemset(c->counter, 0, sizeof(unsigned)));
        c->sc = c->alloc<Scalars>(1);
        CK(cudaMemset(c->sc, 0, sizeof(Scalars)));
        CK(cudaMallocHost(&c->hsc, sizeof(Scalars)));
        CK(cudaEventCreate(&c->e0));
        CK(cudaEventCreate(&c->e1));
        CK(cudaEventCreate(&c->te0));
        CK(cudaEventCreate(&c->te1));
        CK(cudaEventCreateWithFlags(&c->ewait, cudaEventDisableTiming));
        CK(cudaMallocHost(&c->hstat, sizeof(int)));
        CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        c->dguard = c->alloc<int>(hdg_ctx::CAP_LEVELS);
        c->dnk = c->alloc<int>(hdg_ctx::MAX_LOOPS);
        c->dcnt = c->alloc<DevCount>(1);
        CK(cudaMemset(c->dguard, 0, hdg_ctx::CAP_LEVELS * sizeof(int)));
        CK(cudaMemset(c->dnk, 0, hdg_ctx::MAX_LOOPS * sizeof(int)));
        CK(cudaMemset(c->dcnt, 0, sizeof(DevCount)));
        CK(cudaMallocHost(&c->hcnt, sizeof(DevCount)));
        CK(cudaDeviceSynchronize());
    } catch (...) {
        hdg_status s = map_exception();
        hdg_destroy(c);
        return s;
    }
    *out = c;
    return HDG_OK;
}

void hdg_destroy(hdg_ctx *c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    for (auto &E : c->cache) {
        if (E.g_setup) cudaGraphExecDestroy(E.g_setup);
        if (E.g_chunk) cudaGraphExecDestroy(E.g_chunk);
        if (E.g_stage) cudaGraphExecDestroy(E.g_stage);
    }
    if (c->gm_first) cudaGraphExecDestroy(c->gm_first);
    if (c->gm_restart) cudaGraphExecDestroy(c->gm_restart);
    if (c->g_stepI32) cudaGraphExecDestroy(c->g_stepI32);
    if (c->g_step) cudaGraphExecDestroy(c->g_step);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaStream_t s : c->capst)
        if (s) cudaStreamDestroy(s);
    for (void *p : c->allocs) cudaFree(p);
    if (c->hstat) cudaFreeHost(c->hstat);
    if (c->hfv) cudaFreeHost(c->hfv);
    if (c->ewait) cudaEventDestroy(c->ewait);
    if (c->hsc) cudaFreeHost(c->hsc);
    if (c->hgs) cudaFreeHost(c->hgs);
    if (c->hfgs) cudaFreeHost(c->hfgs);
    if (c->hcnt) cudaFreeHost(c->hcnt);
    if (c->e0) cudaEventDestroy(c->e0);
    if (c->e1) cudaEventDestroy(c->e1);
    if (c->te0) cudaEventDestroy(c->te0);
    if (c->te1) cudaEventDestroy(c->te1);
    delete c;
}

hdg_status hdg_dof_sizes(const hdg_ctx *c, int64_t *nQ, int64_t *np, int64_t *nlambda) {
    if (!c) return HDG_ERR_INVALID_ARG;
    if (nQ) *nQ = c->nQ;
    if (np) *np = c->nPv;
    if (nlambda) *nlambda = c->nL;
    return HDG_OK;
}

hdg_status hdg_set_state(hdg_ctx *c, const double *Q, const double *p, const double *lam, double t) {
    if (!c || !Q) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        DISPATCH(c, {
            I::to_modal(c, Q, c->Q, 0);
            if (p) I::to_modal(c, p, c->p, 1); else CK(cudaMemsetAsync(c->p, 0, c->nPv * 8, c->st));
            if (lam) I::to_modal(c, lam, c->lam, 2); else CK(cudaMemsetAsync(c->lam, 0, c->nL * 8, c->st));
        });
        // the stage history stays only if the velocity is the one the last step left (up to the
        // rounding of a round trip through get_state): max |Q - Qlast| <= 1e-9 max |Qlast|
        CK(cudaMemsetAsync(c->dcheck, 0, 2 * sizeof(unsigned long long), c->st));
        launch_k(k_max_diff, grid_for(c->nQ), VEC_THREADS, 0, c->st, (const double *)c->Q, (const double *)c->Qlast,
                 c->nQ, c->dcheck);
        launch_k(k_keep_if_close, 1, 1, 0, c->st, (const unsigned long long *)c->dcheck, 1e-9, c->dhist);
        CKL();
        c->t = t;
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_get_state(hdg_ctx *c, double *Q, double *p, double *lam, double *t) {
    if (!c) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        DISPATCH(c, {
            if (Q) I::to_nodal(c, c->Q, Q, 0);
            if (p) I::to_nodal(c, c->p, p, 1);
            if (lam) I::to_nodal(c, c->lam, lam, 2);
        });
        if (t) *t = c->t;
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_project(hdg_ctx *c, int field, const double *values_at_qp, double *dofs) {
    if (!c || !values_at_qp || !dofs || (field != 0 && field != 1)) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        const int nq = c->T.nq, mu = c->MU;
        const int n = field == 0 ? c->MU : c->NP;
        const long long nvec = field == 0 ? 2 * c->ncells : c->ncells;
        double *modal = field == 0 ? c->q[6] : c->pp[2];
        launch_k(k_project_qp, grid_for(nvec * n), VEC_THREADS, 0, c->st, c->R.qw, c->R.phi, nq, mu, n, values_at_qp, modal,
                 nvec);
        CKL();
        DISPATCH(c, I::to_nodal(c, modal, dofs, field));
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_set_tracer(hdg_ctx *c, const double *q) {
    if (!c) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        if (c->g_step) {                      // the recorded step depends on the tracer
            CK(cudaStreamSynchronize(c->st));
            CK(cudaGraphExecDestroy(c->g_step));
            c->g_step = nullptr;
        }
        if (!q) {
            c->has_tracer = false;
            return HDG_OK;
        }
        ensure_tracer_buffers(c);
        DISPATCH(c, I::to_modal(c, q, c->qtr, 1));
        c->has_tracer = true;
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_get_tracer(hdg_ctx *c, double *q) {
    if (!c || !q) return HDG_ERR_INVALID_ARG;
    if (!c->has_tracer) {
        g_last_error = "hdg_get_tracer: no tracer set";
        return HDG_ERR_INVALID_ARG;
    }
    try {
        settle_pending(c);
        DISPATCH(c, I::to_nodal(c, c->qtr, q, 1));
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_cg_project(hdg_ctx *c, const double *Q, double *Qcg) {
    if (!c || !Q || !Qcg) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        ensure_tracer_buffers(c);
        DISPATCH(c, {
            I::to_modal(c, Q, c->q[0], 0);
            I::cg_project(c, c->q[0], c->q[1]);
            I::to_nodal(c, c->q[1], Qcg, 0);
        });
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_tracer_rhs(hdg_ctx *c, const double *q, const double *U, double *dq) {
    if (!c || !q || !U || !dq) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        DISPATCH(c, {
            I::to_modal(c, q, c->pp[0], 1);
            I::to_modal(c, U, c->q[0], 0);
            I::tracer_rhs(c, c->pp[0], c->q[0], c->pp[1]);
            I::to_nodal(c, c->pp[1], dq, 1);
        });
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_set_forcing(hdg_ctx *c, const double *F, double (*phi)(double, void *), void *user) {
    if (!c) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        if (c->g_step) {                      // the recorded step depends on the forcing terms
            CK(cudaStreamSynchronize(c->st));
            CK(cudaGraphExecDestroy(c->g_step));
            c->g_step = nullptr;
        }
        if (!F) {
            c->has_forcing = false;
            c->phi = nullptr;
            return HDG_OK;
        }
        DISPATCH(c, {
            I::to_modal(c, F, c->q[0], 0);
            I::mass(c, c->q[0], c->Fload, 0);
        });
        c->has_forcing = true;
        c->phi = phi;
        c->phi_user = user;
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_imex_step(hdg_ctx *c, int nsteps, hdg_stats *stats) {
    if (!c || nsteps < 0) return HDG_ERR_INVALID_ARG;
    int nc = 0;
    try {
        begin_call(c);
        for (int s = 0; s < nsteps; ++s) DISPATCH(c, nc |= I::imex_step(c));
        end_call(c, stats);
    } catch (...) {
        hdg_status s = map_exception();
        if (stats) *stats = c->S;
        return s;
    }
    return nc ? not_converged("hdg_imex_step") : HDG_OK;
}

hdg_status hdg_batch_step(hdg_ctx *const *ctxs, int n, int nsteps, hdg_stats *stats) {
    if (!ctxs || n < 0 || nsteps < 0) return HDG_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return HDG_ERR_INVALID_ARG;
    std::vector<int> nc(n, 0), graph(n, 0);
    hdg_status first_err = HDG_OK;
    auto fail = [&](int i) {
        hdg_status s = map_exception();
        if (stats) stats[i] = ctxs[i]->S;
        if (first_err == HDG_OK) first_err = s;
    };
    for (int i = 0; i < n; ++i) {
        try {
            begin_call(ctxs[i]);
            DISPATCH(ctxs[i], graph[i] = I::step_graph_ok(ctxs[i]) ? 1 : 0);
        } catch (...) {
            fail(i);
            return first_err;
        }
    }
    for (int s = 0; s < nsteps && first_err == HDG_OK; ++s) {
        // enqueue every context's step graph (each on its own stream), then wait for them in turn;
        // contexts whose steps cannot be one graph run their step synchronously here
        for (int i = 0; i < n && first_err == HDG_OK; ++i) {
            try {
                if (graph[i]) {
                    DISPATCH(ctxs[i], I::step_enqueue(ctxs[i]));
                } else {
                    DISPATCH(ctxs[i], nc[i] |= I::imex_step(ctxs[i]));
                }
            } catch (...) {
                fail(i);
            }
        }
        for (int i = 0; i < n; ++i) {
            if (!graph[i] || !ctxs[i]->pending) continue;
            try {
                DISPATCH(ctxs[i], nc[i] |= I::step_finish(ctxs[i]));
            } catch (...) {
                fail(i);
            }
        }
    }
    if (first_err != HDG_OK) return first_err;
    int any = 0;
    for (int i = 0; i < n; ++i) {
        try {
            end_call(ctxs[i], stats ? &stats[i] : nullptr);
        } catch (...) {
            fail(i);
            return first_err;
        }
        any |= nc[i];
    }
    return any ? not_converged("hdg_batch_step") : HDG_OK;
}

size_t hdg_ctx_bytes(const hdg_ctx *c) { return c ? c->bytes : 0; }

// Upper estimate of a context's device memory once it has taken IMEX steps: the buffers allocated
// at set-up plus the per-coefficient operators (one condensation per distinct implicit diagonal,
// the final update and the reconstruction; FP32 cell maps and multigrid copies for the stage
// coefficients), with 15 % for the small tables and work vectors not counted term by term.
double hdg_estimate_bytes(const hdg_mesh_desc *mesh, const hdg_params *params) {
    if (!mesh || !params || mesh->n < 1 || params->k < 1 || params->k > 4) return 0.0;
    const double k = params->k, n = mesh->n;
    const double MU = (k + 2) * (k + 3) / 2, NU = 2 * MU, NP = (k + 1) * (k + 2) / 2, NT = k + 1, NL = 3 * NT;
    const double nc = 2 * n * n, nf = (double)mesh_facet_count(mesh->n, mesh->periodic_x != 0, mesh->periodic_y != 0);
    const double nQ = nc * NU, nP = nc * NP, nL = nf * NT, N = nQ + nP + nL;
    const double nfq = std::floor((3 * k + 5) / 2);
    Tab T;
    try {
        T = make_tableau(params->tableau);
    } catch (...) {
        return 0.0;
    }
    std::vector<double> cs;
    for (int i = 0; i < T.s; ++i)
        if (T.Ai[i][i] != 0.0 && std::find(cs.begin(), cs.end(), T.Ai[i][i]) == cs.end()) cs.push_back(T.Ai[i][i]);
    const double nstage_c = (double)cs.size(), ncond = nstage_c + 2;
    double b = 0;
    b += 8 * ((T.s + 1) * (nQ + nP + nL) + T.s * nQ + nQ);                 // state, stages, forcing
    b += 8 * (T.s * (nQ + 2 * (nP + nL)) + 2 * nQ);                       // stage history (guesses)
    b += 8 * 2 * NU * nQ + 4 * nc * std::ceil(NU * 4 * std::ceil(NU / 4) / 32) * 32;   // Dblk, Binv, Binv32
    b += 8 * 3 * nc * 3 * nfq * 2 + 4 * 3 * nc * 3 * nfq * 2;             // weights, edge values
    b += 4 * (32 + 2) * nQ + 8 * (32 + 5) * nQ;                            // Step-I Krylov (FP32, FP64)
    if (params->n_richardson <= 0 && params->stage_krylov) {
        b += 8 * (31 + 30 + 7) * N + 4 * 32 * N;                           // stage FGMRES
        if (params->precision == HDG_MIXED && params->relax_eta > 0)
            b += 2 * 4 * nc * std::ceil(NU * 4 * std::ceil(NU / 4) / 32) * 32 + 4 * 8 * nc;   // FP32 blocks + rest, geometry
    }
    b += 8 * (8 * nQ + 3 * nP + 3 * nL + nc * NL + 10 * nL);               // temporaries, trace work
    b += ncond * 8 * (nc * (NL * NL + NP * NL + NP * NP) + 6 * NT * nL) + ncond * 4 * 5 * nf;
    if (params->precision == HDG_MIXED)
        b += nstage_c * 4 * (2 * nc * (NU + NP) * (NL + NP) + 6 * NT * nL);
    b += 8 * 40 * (n + 1) * (n + 1);                                       // P1 multigrid
    return 1.15 * b + (1 << 20);
}

hdg_status hdg_solve_stage(hdg_ctx *c, double cc, const double *R, const double *Qstar, double *Q,
                           double *p, double *lam, hdg_stats *stats) {
    if (!c || !(cc > 0) || !R || !Qstar || !Q || !p || !lam) return HDG_ERR_INVALID_ARG;
    int nc = 0;
    try {
        begin_call(c);
        DISPATCH(c, {
            double *r = c->Qs[0], *Qs = c->Qs[1 % c->tab.s], *Qm = c->rs[0];
            I::to_modal(c, R, c->q[0], 0);
            I::mass(c, c->q[0], r, 0);
            I::to_modal(c, Qstar, Qs, 0);
            I::to_modal(c, Q, Qm, 0);
            I::to_modal(c, p, c->ps[0], 1);
            I::to_modal(c, lam, c->ls[0], 2);
            nc = I::stage_solve(c, cc, r, Qs, Qm, c->ps[0], c->ls[0]);
            I::to_nodal(c, Qm, Q, 0);
            I::to_nodal(c, c->ps[0], p, 1);
            I::to_nodal(c, c->ls[0], lam, 2);
        });
        end_call(c, stats);
    } catch (...) {
        hdg_status s = map_exception();
        if (stats) *stats = c->S;
        return s;
    }
    return nc ? not_converged("hdg_solve_stage") : HDG_OK;
}

hdg_status hdg_bdm_project(hdg_ctx *c, const double *Q, double *Qstar) {
    if (!c || !Q || !Qstar) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        DISPATCH(c, {
            I::to_modal(c, Q, c->q[0], 0);
            I::bdm(c, c->q[0], c->q[1]);
            I::to_nodal(c, c->q[1], Qstar, 0);
        });
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_fimpl_apply(hdg_ctx *c, const double *Qstar, const double *Q, double *out) {
    if (!c || !Qstar || !Q || !out) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        DISPATCH(c, {
            I::to_modal(c, Qstar, c->q[1], 0);
            I::to_modal(c, Q, c->q[2], 0);
            bool hf = c->has_forcing;
            c->has_forcing = false;
            I::fimpl_dual(c, c->q[2], c->q[1], 0.0, c->q[3]);
            c->has_forcing = hf;
            I::mass(c, c->q[3], c->q[4], 1);
            I::to_nodal(c, c->q[4], out, 0);
        });
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_tentative_solve(hdg_ctx *c, double cc, const double *Qstar, const double *R, double *Qbar,
                               hdg_stats *stats) {
    if (!c || !(cc > 0) || !Qstar || !R || !Qbar) return HDG_ERR_INVALID_ARG;
    try {
        begin_call(c);
        DISPATCH(c, {
            I::to_modal(c, Qstar, c->q[1], 0);
            I::to_modal(c, R, c->q[2], 0);
            I::mass(c, c->q[2], c->q[3], 0);
            I::assemble_stepI(c, c->q[1], cc, I::inv_for(c, c->P.stepI_rtol));
            I::stepI_solve(c, c->q[3], c->q[4], c->P.stepI_rtol);
            I::to_nodal(c, c->q[4], Qbar, 0);
        });
        end_call(c, stats);
    } catch (...) {
        hdg_status s = map_exception();
        if (stats) *stats = c->S;
        return s;
    }
    return HDG_OK;
}

hdg_status hdg_mixed_solve(hdg_ctx *c, double cc, const double *R, const double *X, double *U, double *p,
                           double *lam, hdg_stats *stats) {
    if (!c || !(cc > 0) || !U || !p || !lam) return HDG_ERR_INVALID_ARG;
    try {
        begin_call(c);
        DISPATCH(c, {
            double *Ru = nullptr, *Xm = nullptr;
            if (R) { I::to_modal(c, R, c->q[0], 0); I::mass(c, c->q[0], c->q[1], 0); Ru = c->q[1]; }
            if (X) { I::to_modal(c, X, c->q[2], 0); Xm = c->q[2]; }
            I::mixed_solve(c, cc, Ru, Xm, nullptr, nullptr, c->q[3], c->pp[0], c->ll[0]);
            I::mean_shift(c, c->pp[0], c->ll[0]);
            I::to_nodal(c, c->q[3], U, 0);
            I::to_nodal(c, c->pp[0], p, 1);
            I::to_nodal(c, c->ll[0], lam, 2);
        });
        end_call(c, stats);
    } catch (...) {
        hdg_status s = map_exception();
        if (stats) *stats = c->S;
        return s;
    }
    return HDG_OK;
}

hdg_status hdg_trace_apply(hdg_ctx *c, double cc, const double *lam, double *out) {
    if (!c || !(cc > 0) || !lam || !out) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        DISPATCH(c, {
            CondCache &E = I::condense(c, cc);
            I::to_modal(c, lam, c->ll[0], 2);
            launch_k(k_trace_apply<I::NT>, grid_for(c->nL), VEC_THREADS, 0, c->st, E.Sell, E.tcol, c->ll[0], c->ll[1], (int)c->nfacets);
            CKL();
            launch_k(k_trace_riesz, grid_for(c->nL), VEC_THREADS, 0, c->st, c->geo, c->M.facet_cell, c->M.facet_edge, I::NT,
                                                                      c->ll[1], c->ll[2], c->nfacets);
            CKL();
            I::to_nodal(c, c->ll[2], out, 2);
        });
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

hdg_status hdg_div_free_project(hdg_ctx *c, hdg_stats *stats) {
    if (!c) return HDG_ERR_INVALID_ARG;
    try {
        begin_call(c);
        CK(cudaMemsetAsync(c->dhist, 0, sizeof(int), c->st));     // the state changes outside a step
        DISPATCH(c, {
            I::mixed_solve(c, 1.0, nullptr, c->Q, nullptr, nullptr, c->q[0], c->pp[0], c->ll[0]);
            LinComb L = lincomb();
            L.nterms = 2; L.coef[0] = 1; L.vec[0] = c->Q; L.coef[1] = 1; L.vec[1] = c->q[0];
            launch_k(k_lincomb, grid_for(c->nQ), VEC_THREADS, 0, c->st, c->geo, I::NU, L, c->Q, c->ncells);
            CKL();
            I::reconstruct(c, c->Q, c->t, c->p, c->lam);
        });
        end_call(c, stats);
    } catch (...) {
        hdg_status s = map_exception();
        if (stats) *stats = c->S;
        return s;
    }
    return HDG_OK;
}

hdg_status hdg_reconstruct_pressure(hdg_ctx *c, hdg_stats *stats) {
    if (!c) return HDG_ERR_INVALID_ARG;
    try {
        begin_call(c);
        CK(cudaMemsetAsync(c->dhist, 0, sizeof(int), c->st));     // the state changes outside a step
        DISPATCH(c, I::reconstruct(c, c->Q, c->t, c->p, c->lam));
        end_call(c, stats);
    } catch (...) {
        hdg_status s = map_exception();
        if (stats) *stats = c->S;
        return s;
    }
    return HDG_OK;
}

hdg_status hdg_time_kernel(hdg_ctx *c, int which, double cc, int reps, double *ms, double *bytes) {
    if (!c || reps < 1 || !ms || !bytes || which < 0 || which > 16 || (which != 1 && !(cc > 0)))
        return HDG_ERR_INVALID_ARG;
    if (which == 12 && !(c->Dblk32 && c->P.precision == HDG_MIXED && c->P.relax_eta > 0)) return HDG_ERR_INVALID_ARG;
    if (which >= 2 && which != 8 && which != 11 && which != 12 && !c->fv) return HDG_ERR_INVALID_ARG;
    try {
        settle_pending(c);
        if (which == 10) {
            double t10 = 0.0;
            DISPATCH(c, {
                // S inner FP32 Arnoldi steps (preconditioner pass, product, finishing kernel) launched
                // back to back after a cycle start, minus the cycle start alone, per step
                constexpr int S = 20;
                I::bdm(c, c->Q, c->q[5]);
                I::assemble_stepI(c, c->q[5], cc, I::INV32);
                I::mass(c, c->Q, c->fv, 0);
                const long long n = c->nQ;
                auto start = [&]() {
                    launch_k(k_gm_start<float>, grid_for(n), VEC_THREADS, 0, c->st, n, (const double *)c->fv,
                             (const double *)nullptr, c->gw32, 1, c->rb(), c->gs, 1e-30, 1000, GM_M);
                };
                auto steps = [&]() {
                    start();
                    for (int k = 0; k < S; ++k) I::inner_step32(c, LoopCtl{}, 0, 0);
                };
                steps();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) start();
                CK(cudaEventRecord(c->e1, c->st));
                CK(cudaEventSynchronize(c->e1));
                float t_start = 0;
                CK(cudaEventElapsedTime(&t_start, c->e0, c->e1));
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) steps();
                CK(cudaEventRecord(c->e1, c->st));
                CK(cudaEventSynchronize(c->e1));
                float t_all = 0;
                CK(cudaEventElapsedTime(&t_all, c->e0, c->e1));
                t10 = (double)(t_all - t_start) / reps / S;
                *bytes = 0;
            });
            *ms = t10;
            return HDG_OK;
        }
        if (which == 6 || which == 9 || which == 13 || which == 14) {
            double t6_ms = 0.0;
            DISPATCH(c, {
                if (which >= 13 && !I::use_gs(c)) throw std::invalid_argument("hdg_time_kernel: modes 13, 14 time the "
                                                                              "red-black Gauss-Seidel inner kernels (inner_gs)");
                // one FP32 inner Step-I solve fills the basis and edge values; then the Arnoldi
                // product of step j = 4 is launched alone
                constexpr int J = 4;
                I::bdm(c, c->Q, c->q[5]);
                I::assemble_stepI(c, c->q[5], cc, I::INV32);
                I::mass(c, c->Q, c->fv, 0);
                launch_k(k_gm_set_tol, 1, 1, 0, c->st, c->gs, 1e-30, J + 1);   // runs J + 1 steps
                CKL();
                cudaGraphExec_t ex = capture_graph(c, [&]() { I::stepI32_record(c, c->fv, c->q[2]); });
                CK(cudaGraphLaunch(ex, c->st));
                const EdgeTab<float> E{c->ephi32, c->pen32, c->nrm32};
                const unsigned cb = cell_blocks(c), ab = cb < (unsigned)MAX_RED_BLOCKS ? cb : (unsigned)MAX_RED_BLOCKS;
                const size_t sm = sizeof(float) * TEAMS_PER_BLOCK * 6 * I::Dm::NFQ;
                // the kernel as the solve runs it at step J: each launch follows a one-thread
                // kernel that puts step J back (the solve above ended its cycle); that kernel's own
                // time, measured alone, is subtracted
                auto reset = [&]() { launch_k(k_gm_set_step, 1, 1, 0, c->st, c->gs, J); };
                const size_t smg = sizeof(float) * I::GS_WARPS * (2 * I::NU + 6 * I::Dm::NFQ);
                auto launch = [&]() {
                    reset();
                    if (which == 6)
                        launch_k(k_gm_apply_mf<I::K_, float, true>, ab, 128, sm, c->st, E, c->M, c->wq32, c->utr32,
                                 c->gw32, c->gV32, c->rb(), c->gs);
                    else if (which == 9)
                        launch_k(k_gm_precond_mf<I::K_, float, true>, cb, 128, sizeof(float) * TEAMS_PER_BLOCK * 2 * I::NU,
                                 c->st, E, c->M, c->Binv32, c->gw32, c->gV32, c->utr32, c->gs);
                    else if (which == 13)       // both colours (the time per launch is half the pair's)
                        for (int col = 0; col < 2; ++col)
                            launch_k(k_gs_diag<I::K_>, I::gs_blocks(c), 128, smg, c->st, E, c->M, (const float *)c->Binv32,
                                     (const float *)c->gw32, c->gV32, c->utr32, (const float *)c->wq32,
                                     (const GmresState *)c->gs, col);
                    else
                        launch_k(k_gs_apply<I::K_>, ab, 128, sm, c->st, E, c->M, (const float *)c->wq32,
                                 (const float *)c->utr32, c->gw32, (const float *)c->gV32, c->rb(), c->gs);
                };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) reset();
                CK(cudaEventRecord(c->e1, c->st));
                CK(cudaEventSynchronize(c->e1));
                float t_reset = 0;
                CK(cudaEventElapsedTime(&t_reset, c->e0, c->e1));
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
                CK(cudaEventSynchronize(c->e1));
                float t_pair = 0;
                CK(cudaEventElapsedTime(&t_pair, c->e0, c->e1));
                t6_ms = (double)(t_pair - t_reset) / reps;
                cudaGraphExecDestroy(ex);
                const int nfq = I::Dm::NFQ;
                const double nc = (double)c->ncells;
                if (which == 6)   // neighbour edge values (2 floats per point) + weights + v_j read + w
                                  // written + the J + 1 basis vectors of the dots
                    *bytes = 4.0 * (nc * 3 * nfq * 3 + 2.0 * c->nQ + (J + 1.0) * c->nQ);
                else if (which == 9)   // block inverses + w read + V_0..V_{J-1} read (projections) + V_J
                                       // written + edge values written (2 floats per point)
                    *bytes = 4.0 * (nc * I::NU * I::NU + (J + 2.0) * c->nQ + nc * 3 * nfq * 2);
                else if (which == 13) {   // per launch (one colour, half the cells): the colour's block
                                          // inverses, w, V_0..V_{J-1} read, V_J and edge values written;
                                          // black also reads its red neighbours' edge values and weights
                    *bytes = 0.5 * 4.0 * (nc * GsBlk<I::K_>::SIZE + (J + 2.0) * c->nQ + nc * 3 * nfq * 2 +
                                          0.5 * nc * 3 * nfq * 3);
                    t6_ms *= 0.5;
                } else                // red cells' neighbour edge values and weights, v_j read, w written,
                                      // the J + 1 basis vectors of the dots
                    *bytes = 4.0 * (0.5 * nc * 3 * nfq * 3 + 2.0 * c->nQ + (J + 1.0) * c->nQ);
            });
            *ms = t6_ms;
            return HDG_OK;
        }
        if (which >= 2 && which != 8 && which != 11 && which != 12 && which != 13 && which != 14 && which != 15 &&
            which != 16) {
            DISPATCH(c, {
                // operator of a stage at coefficient cc around the current state; v = (M Q, 0, 0)
                I::bdm(c, c->Q, c->q[5]);
                I::assemble_stepI(c, c->q[5], cc, I::inv_for(c, c->P.inner_stepI_rtol));
                I::condense(c, cc);
                I::ensure_pre_maps(c, cc);
                I::mass(c, c->Q, c->fv, 0);
                const long long N = c->nQ + c->nPv + c->nL;
                CK(cudaMemsetAsync(c->fv + c->nQ, 0, 8 * (N - c->nQ), c->st));
                cudaGraphExec_t ex = capture_graph(c, [&]() {
                    if (which == 2) I::stepI_solve(c, c->fv, c->q[2], c->P.inner_stepI_rtol);
                    else if (which == 3)
                        I::mixed_solve(c, cc, nullptr, c->fv, nullptr, nullptr, c->q[4], c->fz + c->nQ,
                                       c->fz + c->nQ + c->nPv, nullptr, nullptr, c->P.inner_trace_rtol);
                    else if (which == 4) I::chorin_precond(c, cc, c->fv, c->fz);
                    else if (which == 7)
                        I::pre_step2(c, cc, c->fv, c->fv + c->nQ, c->fv + c->nQ + c->nPv, c->q[4], c->fz + c->nQ,
                                     c->fz + c->nQ + c->nPv);
                    else I::stage_apply(c, cc, c->fv, c->fw);
                });
                CK(cudaGraphLaunch(ex, c->st));
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) CK(cudaGraphLaunch(ex, c->st));
                CK(cudaEventRecord(c->e1, c->st));
                CK(cudaEventSynchronize(c->e1));
                cudaGraphExecDestroy(ex);
            });
            float t = 0;
            CK(cudaEventElapsedTime(&t, c->e0, c->e1));
            *ms = t / reps;
            *bytes = 0;
            return HDG_OK;
        }
        DISPATCH(c, {
            const int NT = I::NT, NU = I::NU;
            double b = 0;
            std::vector<int> hc;
            if (which == 0) {
                CondCache &E = I::condense(c, cc);
                // operator blocks actually read (wall facets have 3 of 5) + block-column indices
                long long nblk = 0;
                for (long long f = 0; f < c->nfacets; ++f) nblk += 1 + 2 * (c->H.facet_cell[2 * f + 1] >= 0 ? 2 : 1);
                b = 8.0 * nblk * NT * NT + 4.0 * 5 * c->nfacets + 8.0 * 4 * c->nL;   // + z, pold read; pnew, Ap written
                Scalars h{};
                h.done = 0; h.beta = 0.5; h.rz = 1.0; h.zmean = 0.0;
                CK(cudaMemcpyAsync(c->sc, &h, sizeof(Scalars), cudaMemcpyHostToDevice, c->st));
                const int nf = (int)c->nfacets;
                auto launch = [&]() {
                    launch_k(k_cg_apply<I::NT>, cg_apply_grid<I::NT>(nf), 128, 0, c->st, E.Sell, E.tcol, c->tz, c->tp[0], c->tp[1], c->tAp, nf,
                                                                    c->rb(), c->sc);
                };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
            } else if (which == 15 || which == 16) {
                // 15: k_fimpl_assemble alone (the stage solves' form: block, weights, no FP64
                // inverse) for coefficient cc around the current state's P(Q); bytes: Q* of the cell
                // and its neighbours read, the block and weights written (FP64 and FP32 weights).
                // 16: k_bdm alone on the current state; bytes: Q read, P(Q) written
                const int nfq = (3 * c->K + 5) / 2;
                I::bdm(c, c->Q, c->q[5]);
                const size_t smem = sizeof(double) * fimpl_smem_noinv_doubles<I::K_>();
                if (which == 15)
                    b = (double)c->ncells * (8.0 * 4 * NU + 8.0 * NU * NU + 12.0 * 3 * nfq + 4.0 * 6);
                else
                    b = 16.0 * c->nQ;
                auto launch = [&]() {
                    if (which == 15)
                        launch_k(k_fimpl_assemble<I::K_>, (unsigned)c->ncells, 128, smem, c->st, c->R, c->M,
                                 (const double *)c->q[5], cc, c->P.alpha, c->P.delta_up, c->Dblk, c->wq, c->wq32, c->pen,
                                 c->pen32, (double *)nullptr, c->dstatus, I::tadv2(c));
                    else
                        I::bdm_launch(c, (const double *)c->Q, c->q[5]);
                };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
            } else if (which == 11) {
                // k_condense alone for coefficient cc (rewrites the cached factors with the same
                // values); bytes: geometry and flip read + S_K, Z_K, A_K^-1 written
                CondCache &E = I::condense(c, cc);
                const int NP = I::NP, NL = I::NL;
                const size_t smem = sizeof(double) * (NP * NU + NL * NU + 2 * NP * NP + 2 * NP * NL + NL * NL);
                b = (double)c->ncells * (sizeof(CellGeo) + 3 * sizeof(int) + 8.0 * (NL * NL + NP * NL + NP * NP));
                auto launch = [&]() {
                    launch_k(k_condense<I::K_>, (unsigned)c->ncells, 128, smem, c->st, c->R, c->M, cc, c->P.tau, E.Scell,
                             E.Zc, E.Ac);
                };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
            } else if (which == 12) {
                // k_stage_apply32 alone (its flag forced on), like 8; bytes: FP32 diagonal blocks,
                // weights, geometry and normals + neighbour maps + Q, p, lambda read + yQ, yp, v written
                const int nfq = (3 * c->K + 5) / 2;
                b = 4.0 * c->ncells * ((double)GsBlk<I::K_>::SIZE + 3 * nfq + GEO32 + 6) + 4.0 * 6 * c->ncells +
                    8.0 * (2.0 * c->nQ + 2.0 * c->nPv + c->nL + (double)c->ncells * 3 * NT);
                const int one = 1;
                CK(cudaMemcpyAsync(&c->fgs->lowprec, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
                auto launch = [&]() {
                    I::stage_apply32(c, cc, c->Q, c->p, c->lam, c->q[6], c->pp[1], (float *)nullptr, (float *)nullptr,
                                     (double *)nullptr, (const int *)nullptr, c->fgs, (DevCount *)nullptr);
                };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
            } else if (which == 8) {
                // k_stage_apply alone on the operator last assembled (c scales the pressure and trace
                // coupling), input the current state (Q, p, lambda); bytes: diagonal blocks +
                // neighbour weights + neighbour maps + Q, p, lambda read + yQ, yp, v written
                // (HDG_MIXED with relaxed products: the pair-arithmetic kernel k_stage_apply_f2, which
                // the stage solves take, on the FP32 block copy and its rest: the same bytes)
                const int nfq = (3 * c->K + 5) / 2;
                const bool f2k = c->P.precision == HDG_MIXED && c->Dblk32lo && c->P.richardson_rtol >= I::PAIR_MIN_RTOL;
                b = (f2k ? 8.0 * c->ncells * GsBlk<I::K_>::SIZE : 8.0 * c->ncells * (double)NU * NU) +
                    8.0 * c->ncells * 3 * nfq + 4.0 * 6 * c->ncells +
                    8.0 * (2.0 * c->nQ + 2.0 * c->nPv + c->nL + (double)c->ncells * 3 * NT);
                const unsigned nb = cell_blocks(c);
                const size_t sm = sizeof(double) * TEAMS_PER_BLOCK * (6 * nfq + 3 * NT + 2 * I::MU);
                auto launch = [&]() {
                    if (f2k)
                        I::stage_apply_f2(c, cc, c->Q, c->p, c->lam, c->q[6], c->pp[1], (float *)nullptr,
                                          (float *)nullptr, (double *)nullptr, (const int *)nullptr, (const int *)nullptr);
                    else
                        launch_k(k_stage_apply<I::K_>, nb, 128, sm, c->st, c->R, EdgeTab<double>{c->R.ephi, c->pen}, c->M,
                                 c->Dblk, c->wq, cc, c->P.tau, c->Q, c->p, c->lam, c->q[6], c->pp[1], c->vK,
                                 (float *)nullptr, (float *)nullptr, (double *)nullptr, (const int *)nullptr,
                                 (const int *)nullptr);
                };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
            } else {
                // diagonal blocks + neighbour weights + neighbour maps (2 ints x 3) + x read, y written
                const int nfq = (3 * c->K + 5) / 2;
                b = 8.0 * c->ncells * ((double)NU * NU + 3 * nfq) + 4.0 * 6 * c->ncells + 8.0 * 2 * c->nQ;
                auto launch = [&]() { I::cell_apply(c, c->gz, c->gw); };
                launch();
                CKL();
                CK(cudaEventRecord(c->e0, c->st));
                for (int r = 0; r < reps; ++r) launch();
                CK(cudaEventRecord(c->e1, c->st));
            }
            CK(cudaEventSynchronize(c->e1));
            float t = 0;
            CK(cudaEventElapsedTime(&t, c->e0, c->e1));
            *ms = t / reps;
            *bytes = b;
        });
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}

}  // extern "C"

// =========================================================================== no-allocation variant
// hdg_trace_apply_noalloc: the trace-operator apply without the context's per-coefficient operator
// cache (whose first use for a new c calls cudaMalloc). Its scratch is this file-scope device
// array, reached from host code only through the address cudaGetSymbolAddress returns (taken once
// per device, on the first call made on that device).
namespace {
constexpr long long NOALLOC_MAX_DOUBLES = 1LL << 20;          // 8 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_DOUBLES];
constexpr int NOALLOC_MAX_DEVICES = 64;
static double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mutex;                                   // guards g_noalloc_ptr

// per cell: condense S_K in shared memory (cell_condense) and write z_K = S_K l_K (canonical rows)
template <int K>
__global__ void k_condense_apply_cell(RefDev R, MeshDev M, double c, double tau, const double *__restrict__ lam,
                                      double *z) {
    wait_prior_kernel();
    typedef Dims<K> Dm;
    constexpr int NP = Dm::NP, NT = Dm::NT, NL = Dm::NL, NU = Dm::NU;
    extern __shared__ double sm[];
    const int cell = blockIdx.x;
    if (cell >= M.ncells) return;
    Team tm{(int)threadIdx.x, (int)blockDim.x};
    CellGeo g = M.geo[cell];
    int flip[3] = {M.cell_flip[3 * cell], M.cell_flip[3 * cell + 1], M.cell_flip[3 * cell + 2]};
    double *work = sm;
    double *S = work + NP * NU + NL * NU + 2 * NP * NP + 2 * NP * NL + NL * NL;
    double *Zs = S + NL * NL, *As = Zs + NP * NL, *lK = As + NP * NP;
    cell_condense<K>(tm, R, g, flip, c, tau, work, S, Zs, As);
    TFOR(i, NL) {
        int e = i / NT, j = i % NT;
        lK[i] = lam[(size_t)M.cell_facet[3 * cell + e] * NT + j];             // canonical orientation
    }
    tm.sync();
    TFOR(r, NL) {
        double s = 0;
        for (int q = 0; q < NL; ++q) s += S[r * NL + q] * lK[q];
        z[(size_t)cell * NL + r] = s;
    }
}

template <int K>
void trace_apply_noalloc_impl(hdg_ctx *c, double cc, const double *lam_nodal, double *out_nodal, double *scr) {
    typedef Dims<K> Dm;
    constexpr int NP = Dm::NP, NT = Dm::NT, NL = Dm::NL, NU = Dm::NU;
    double *lm = scr, *ym = lm + c->nL, *yr = ym + c->nL, *z = yr + c->nL;
    launch_k(k_basis_change, red_grid(c->nL), VEC_THREADS, 0, c->st, c->R.nod_t, NT, lam_nodal, lm, c->nfacets);
    CKL();
    size_t smem = sizeof(double) * (NP * NU + NL * NU + 2 * NP * NP + 2 * NP * NL + NL * NL + NL * NL + NP * NL +
                                    NP * NP + NL);
    launch_k(k_condense_apply_cell<K>, (unsigned)c->ncells, 128, smem, c->st, c->R, c->M, cc, c->P.tau, lm, z);
    CKL();
    launch_k(k_facet_gather<NT>, red_grid(c->nL), VEC_THREADS, 0, c->st, c->M, z, nullptr, ym, (float *)nullptr);
    CKL();
    launch_k(k_trace_riesz, red_grid(c->nL), VEC_THREADS, 0, c->st, c->geo, c->M.facet_cell, c->M.facet_edge, NT, ym, yr,
                                                              c->nfacets);
    CKL();
    launch_k(k_basis_change, red_grid(c->nL), VEC_THREADS, 0, c->st, c->R.mod_t, NT, yr, out_nodal, c->nfacets);
    CKL();
}
}  // namespace

extern "C" hdg_status hdg_trace_apply_noalloc(hdg_ctx *c, double cc, const double *lam, double *out) {
    if (!c || !(cc > 0) || !lam || !out) return HDG_ERR_INVALID_ARG;
    const long long need = 3 * c->nL + c->ncells * c->NL;
    if (need > NOALLOC_MAX_DOUBLES) {
        g_last_error = "hdg_trace_apply_noalloc: mesh too large for the static scratch (needs " +
                       std::to_string(need) + " doubles, maximum " + std::to_string(NOALLOC_MAX_DOUBLES) + ")";
        return HDG_ERR_INVALID_ARG;
    }
    // the scratch address belongs to the context's device, which must be the current one (the
    // kernels run on the context's stream, and the address is looked up with that device current)
    const int dev = c->device;
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) {
        g_last_error = std::string("hdg_trace_apply_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
        return HDG_ERR_CUDA;
    }
    if (cur != dev) {
        g_last_error = "hdg_trace_apply_noalloc: current device " + std::to_string(cur) +
                       " is not the context's device " + std::to_string(dev);
        return HDG_ERR_INVALID_ARG;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        g_last_error = "hdg_trace_apply_noalloc: device index " + std::to_string(dev) +
                       " is beyond the library's table of " + std::to_string(NOALLOC_MAX_DEVICES) + " devices";
        return HDG_ERR_UNSUPPORTED;
    }
    double *scr = nullptr;
    {
        // once per device, with that device current; concurrent first calls from several host
        // threads are serialised here
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            double *ptr = nullptr;
            e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                g_last_error = std::string("hdg_trace_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return HDG_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = ptr;
        }
        scr = g_noalloc_ptr[dev];
    }
    try {
        switch (c->K) {
            case 1: trace_apply_noalloc_impl<1>(c, cc, lam, out, scr); break;
            case 2: trace_apply_noalloc_impl<2>(c, cc, lam, out, scr); break;
            case 3: trace_apply_noalloc_impl<3>(c, cc, lam, out, scr); break;
            case 4: trace_apply_noalloc_impl<4>(c, cc, lam, out, scr); break;
            default: return HDG_ERR_INVALID_ARG;
        }
        CK(cudaStreamSynchronize(c->st));
    } catch (...) {
        return map_exception();
    }
    return HDG_OK;
}
