/*
 * hdg.h — C-ABI of the GB300 hybridised DG IMEX stage solver for the incompressible Euler
 * equations (Mueller, "A Higher-order Hybridisable Discontinuous Galerkin IMEX method for the
 * incompressible Euler equations", arXiv 2410.09790).
 *
 * Discretisation (Sec. 2.2-2.4): on a structured triangulation of [0,Lx]x[0,Ly] (Sec. 3.2),
 * velocity Q in [DG_{k+1}]^2, pressure p in DG_k with (p)_Omega = 0, trace lambda in P_k on
 * every facet. Time stepping: the s-stage IMEX scheme of Alg. 1, each implicit stage solved
 * either by the Chorin-split Richardson iteration of Alg. 2 (a fixed number of iterations, as
 * printed, or to a tolerance) or to a tolerance by flexible GMRES preconditioned by that split;
 * Step II is condensed onto the trace (Sec. 2.8) and solved by multigrid-preconditioned CG.
 *
 * Exchange format. Every array crossing this interface holds NODAL VALUES on the canonical
 * mesh (independent of the library's internal modal basis):
 *   cells: n x n rectangles, rectangle (i,j) split along its (i,j)-(i+1,j+1) diagonal into
 *          cell 2(jn+i) = (A,B,C) and cell 2(jn+i)+1 = (A,C,D) with A=(i,j), B=(i+1,j),
 *          C=(i+1,j+1), D=(i,j+1) (in units Lx/n, Ly/n), vertices v0,v1,v2 in that order;
 *   a degree-m cell field: values at v0 + (i/m)(v1-v0) + (j/m)(v2-v0), i+j <= m, j outer,
 *          i inner;  Q: double[ncells][2][(k+2)(k+3)/2];  p: double[ncells][(k+1)(k+2)/2];
 *   facets: horizontal H(i,j) from (i,j) to (i+1,j), then vertical V(i,j) from (i,j) to
 *          (i,j+1), then diagonals D(i,j) from (i,j) to (i+1,j+1), each j-major; periodic
 *          directions omit the duplicate edges; lambda: double[nfacets][k+1] at the points
 *          t = i/k along the facet from its first to its second end point.
 *   dual vectors (one-forms on V_Q, e.g. the stage residual r_i of eq. imex_residual) are
 *          passed by their L2 Riesz representer R (r(w) = (R, w)_Omega), as a velocity field.
 *
 * Memory. Array arguments are DEVICE pointers (e.g. torch CUDA tensors) unless the name says
 * host; the library copies in/out on the context's stream and keeps no caller pointer. All
 * arrays are contiguous float64 in the layouts above. The context owns every internal buffer
 * (allocated in hdg_setup_mesh and on first use of a new coefficient c; freed by hdg_destroy).
 *
 * Errors. Every call returns an hdg_status; nothing aborts or traps. HDG_ERR_NOT_CONVERGED still
 * leaves the last iterate in place and fills the stats. Iteration counts are bounded by
 * hdg_params.max_iters. Calls on one context must not overlap (one host thread at a time).
 */
#ifndef HDG_GB300_H
#define HDG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_ctx hdg_ctx;

typedef enum {
    HDG_OK = 0,
    HDG_ERR_INVALID_ARG = 1,   /* bad size, degree, pointer or parameter                   */
    HDG_ERR_CUDA = 2,          /* a CUDA runtime call failed (message: hdg_last_error)      */
    HDG_ERR_OOM = 3,           /* device allocation failed                                  */
    HDG_ERR_NOT_CONVERGED = 4, /* an iteration hit its cap; best iterate kept               */
    HDG_ERR_NUMERIC = 5,       /* NaN / Inf in a residual norm                              */
    HDG_ERR_UNSUPPORTED = 6,   /* valid request this build does not handle                  */
    HDG_ERR_TIMEOUT = 7        /* hdg_params.timeout_ms ran out before the GPU work finished */
} hdg_status;

/* IMEX tableaus: ARS(2,2,2) and ARS(3,4,3) (Ascher, Ruuth and Spiteri 1997), and App. A's IMEX
 * Euler, SSP2(3,3,2) (explicit abscissae read as (0, 1/2, 1)) and SSP3(4,3,3). The SSP tableaus
 * have an implicit first stage (a_00 != 0), outside Alg. 1's assumed form: every stage with
 * a_ii != 0 is solved (the first advected by P(Q^n)) and the sums of eq. imex_residual and
 * eq. final_residual run over all implicit stages. */
typedef enum { HDG_ARS222 = 0, HDG_ARS343 = 1, HDG_IMEX_EULER = 2, HDG_SSP2_332 = 3, HDG_SSP3_433 = 4 } hdg_tableau;

typedef enum { HDG_FP64 = 0, HDG_MIXED = 1 } hdg_precision;

/* Mesh (Sec. 3.2): n x n rectangles over [0,Lx]x[0,Ly]; walls (n.Q = 0, weakly) on every
 * non-periodic side. */
typedef struct {
    int n;
    double Lx, Ly;
    int periodic_x, periodic_y;
} hdg_mesh_desc;

/* Method parameters. Defaults (hdg_default_params): alpha = tau = delta_up = 1 (Sec. 3.2),
 * n_richardson = 2 (Sec. 3.2), trace_rtol = 1e-12, stepI_rtol = 1e-10 (Sec. 3.4.2). */
typedef struct {
    int k;                    /* pressure degree, 1..4 (velocity k+1, trace k)             */
    double alpha;             /* normal-jump penalty of eq. f_impl                         */
    double tau;               /* HDG stabilisation of eq. flux_hdg                         */
    double delta_up;          /* upwind switch/weight of eq. f_impl                        */
    int tableau;              /* hdg_tableau                                               */
    double dt;                /* time step                                                 */
    int n_richardson;         /* > 0: fixed number of Alg. 2 iterations                    */
    double richardson_rtol;   /* used when n_richardson <= 0: stop at ||dQ||_M <= rtol ||Q||_M */
    int richardson_max;       /* cap for the tolerance mode                                */
    double trace_rtol;        /* CG on the trace system: preconditioned residual           */
    double stepI_rtol;        /* GMRES(30) on the tentative velocity system (residual)     */
    int max_iters;            /* cap for each Krylov solve                                 */
    /* Stage solves to tolerance (n_richardson <= 0): stage_krylov = 0 iterates Alg. 2 until
     * ||dQ||_M <= richardson_rtol ||Q||_M; stage_krylov = 1 (default) runs flexible GMRES(30) on
     * the monolithic stage system with Alg. 2's Chorin split as the preconditioner (Step I and
     * Step II solved to inner_stepI_rtol / inner_trace_rtol, defaults 2e-2 / 1e-1) until the
     * stage residual is <= richardson_rtol times the right-hand side; richardson_max caps the
     * outer iterations. Both reach the same fixed point, the monolithic stage solution. */
    int stage_krylov;
    double inner_stepI_rtol;
    double inner_trace_rtol;
    /* Trace CG preconditioner: 1 (default) = one V-cycle of the non-nested multigrid of Sec. 2.8
     * (degree-2 Chebyshev on facet block-Jacobi; P1 coarse space on the vertices with the Galerkin
     * operator; geometric P1 hierarchy n -> n/2 while n stays even and >= 4; dense pseudo-inverse
     * on the coarsest grid, which must have <= 1024 vertices, else block-Jacobi is used);
     * 0 = facet block-Jacobi. */
    int trace_mg;
    /* Stage solves with stage_krylov = 1: 1 (default) records the whole flexible GMRES, with its
     * inner Step-I GMRES and trace CG, as one CUDA graph whose loops run on the device
     * (conditional graph nodes, each with an iteration guard) and replays it per stage: no host
     * round trip inside a stage solve; inner solves that stop at their iteration cap do not raise
     * an error there (the outer residual test decides). 0 = loops driven from the host (per-
     * component timings in hdg_stats are only filled in this mode). */
    int device_loops;
    /* Step II inside the stage preconditioner (stage_krylov = 1, multigrid on): n > 0 (default 1)
     * = exactly n V-cycles of the trace multigrid (a fixed linear preconditioner; the flexible
     * outer iteration decides the accuracy); 0 = trace CG to inner_trace_rtol. */
    int inner_trace_vcycles;
    /* Arithmetic of the stage preconditioner (stage_krylov = 1; hdg_precision). HDG_MIXED
     * (default): the inner Step-I GMRES, the preconditioner's Step-II cell maps and V-cycle, the
     * tight trace CG's V-cycle and the first orthogonalisation pass of the stage FGMRES run in FP32;
     * the stage residual, its Krylov basis, the trace operator and the CG's iterates stay FP64, so
     * the result meets the same FP64 stage tolerance. Under HDG_MIXED the FP64-bound contractions
     * run on the FP32 pipes at FP64-class accuracy, as unevaluated pairs of FP32 numbers (about
     * 2^-46 of the terms' magnitudes): the Step-I block (advection contraction, weighted facet
     * masses, entries), the BDM projection and, with relax_eta > 0 and richardson_rtol >= 5e-11,
     * the stage FGMRES's FP64-accurate products.
     * HDG_FP64: every kernel of the path computes in FP64 instructions (inner Step I by FP64 GMRES
     * with block Jacobi; inner_trace_fp32 and trace_fp32_vcycle are forced to 0). */
    int precision;
    /* The one-V-cycle Step II inside the stage preconditioner (inner_trace_vcycles = 1): 1
     * (default) = the V-cycle in FP32 (operators rounded once per stage coefficient; the large P1
     * levels as grid-wide kernels, the small ones — from the first level with at most 1200
     * vertices whose sub-hierarchy fits 200 KiB of shared memory — in one thread block);
     * 0 = the FP64 V-cycle. The outer iteration's tolerance is unchanged: this only alters the
     * preconditioner. */
    int inner_trace_fp32;
    /* Trace CG with the multigrid (tight solves: final update, pressure reconstruction, mixed
     * solves): 1 (default) = preconditioned by the same V-cycle in FP32 (when the hierarchy fits
     * one block, as for inner_trace_fp32), with the flexible (Polak-Ribiere) CG update since the
     * FP32 V-cycle is not exactly one fixed symmetric map; everything else of the CG (operator,
     * residual, iterate, dot products, the tolerance on sqrt(r.z / r0.z0)) stays FP64. 0 = the
     * FP64 V-cycle with plain preconditioned CG. */
    int trace_fp32_vcycle;
    /* Right preconditioner of the inner FP32 Step-I GMRES: 1 (default) = red-black block
     * Gauss-Seidel on the cells' diagonal blocks (the structured triangulation's cells are
     * two-coloured by index parity; checked at setup, else block Jacobi): about half the Arnoldi
     * steps for one more kernel per step; 0 = block Jacobi. */
    int inner_gs;
    /* > 0: bound, in milliseconds counted from the step's launch, on the host's wait for the GPU
     * work of each step of hdg_imex_step when the step runs as one CUDA graph (device_loops = 1,
     * stage_krylov = 1). When it runs out the call returns HDG_ERR_TIMEOUT at
     * once; the step stays queued on the context's stream and completes there (nothing is
     * cancelled), and the next call on the context waits for it without a limit and then advances
     * the context's time. Set-up work before a context's first step graph (condensations, graph
     * capture) is not bounded. 0 (default): no limit. */
    double timeout_ms;
    /* Relaxed stage-operator products (HDG_MIXED with stage_krylov only). The stage FGMRES takes
     * an Arnoldi product A(c) z_j in FP32 once its residual estimate r_j satisfies
     * r_j * relax_eta <= richardson_rtol * ||b||: by the inexact-Krylov bound (Simoncini and
     * Szyld 2003) a product error of relative size relax_eta then moves the final residual by
     * about the tolerance at most, and every restart (and the final check) forms b - A x in FP64,
     * so the stage tolerance holds regardless. relax_eta is the relative error assumed for an
     * FP32 product. 0: every product in FP64. Default 1e-5. */
    double relax_eta;
} hdg_params;

typedef struct {
    int richardson_iters;     /* Alg. 2 (or outer Krylov) iterations, summed over the call  */
    int trace_solves;         /* trace (Step II type) solves in the last call               */
    int trace_iters;          /* CG iterations summed over those solves                    */
    int stepI_solves;
    int stepI_iters;          /* GMRES iterations summed                                   */
    int stage_solves;         /* Alg. 2 solves in the last call                            */
    double last_update_norm;  /* ||Q^(m) - Q^(m-1)||_M of the last Richardson iteration     */
    double last_trace_relres; /* final relative (preconditioned) residual of the last CG    */
    double ms_total;          /* device time of the call (CUDA events)                     */
    /* per-component device time of the call (CUDA events; Sec. 3.4.1's buckets): trace
     * solves (pressure / Step II, incl. their condensed right-hand sides and back-substitution),
     * tentative-velocity solves (Step I), assembly of the Step-I operator, BDM projections */
    double ms_trace;
    double ms_stepI;
    double ms_assembly;
    double ms_bdm;
    /* kernels run by the call's CUDA graphs (device_loops = 1): the graphs' kernel nodes plus
     * every pass of their device-side loops, counted exactly on the device; in that mode an IMEX
     * step (stage_krylov = 1) is one graph, so this counts all of its kernels */
    long long graph_kernels;
    /* stage-operator products the stage FGMRES took in FP32 (relax_eta), summed over the call */
    long long stage_products32;
} hdg_stats;

void hdg_default_params(hdg_params *p);
const char *hdg_status_string(hdg_status s);
/* Message of the last call on this thread that failed (a CUDA error's text, the reason for
 * HDG_ERR_INVALID_ARG where one is known, the solve that did not converge). Calls that run solver
 * work on a context clear it when they start. Host string, valid until the next call. */
const char *hdg_last_error(void);

/* Host-only queries (no GPU needed). Sizes of the exchange arrays for a mesh and degree. */
hdg_status hdg_mesh_counts(const hdg_mesh_desc *mesh, int k, int64_t *ncells, int64_t *nfacets);

/* Host-only: the library's reference element, for tests.
 * which = 0: volume rule on the reference triangle (0,0),(1,0),(0,1) used for degree k forms;
 * which = 1: facet rule on [0,1] (Gauss-Legendre, (3k+5)/2 points, shared with eq. f_impl's
 *            upwind term). pts (host) gets 2 (which=0) or 1 (which=1) coordinates per point.
 * Call with pts = wts = NULL to get *npts. */
hdg_status hdg_reference_rule(int k, int which, double *pts, double *wts, int *npts);
/* Host-only: values of the library's orthonormal basis of P_m on the reference triangle at
 * npts points (host, x/y interleaved) -> vals[npts][dim P_m] (host). */
hdg_status hdg_reference_basis(int m, int npts, const double *pts, double *vals);

/* Create a context: build the mesh and reference tables, upload them, allocate state. The
 * stream (cudaStream_t, may be NULL for the legacy default stream) orders all work of the
 * context. Uses the current CUDA device. */
hdg_status hdg_setup_mesh(hdg_ctx **out, const hdg_mesh_desc *mesh, const hdg_params *params,
                          void *cuda_stream);
void hdg_destroy(hdg_ctx *ctx);

/* Sizes (doubles) of the nodal Q, p and lambda arrays. */
hdg_status hdg_dof_sizes(const hdg_ctx *ctx, int64_t *nQ, int64_t *np, int64_t *nlambda);

/* State (device pointers, nodal). p and lam may be NULL (taken as zero). Setting a velocity
 * other than the one the last step left (beyond 1e-9 of its largest coefficient) drops the
 * stage history that hdg_imex_step starts its stage solves from; setting that same state again
 * (a get/set round trip) keeps it. */
hdg_status hdg_set_state(hdg_ctx *ctx, const double *Q, const double *p, const double *lam, double t);
hdg_status hdg_get_state(hdg_ctx *ctx, double *Q, double *p, double *lam, double *t_host);

/* L2 projection of sampled data onto a cell space (Sec. 2.2: the initial velocity and the forcing
 * enter the method as elements of V_Q; non-polynomial data is projected with a fixed rule).
 * values_at_qp (device) samples the data at the library's volume quadrature points, whose
 * reference coordinates (xi, eta) hdg_reference_rule(k, 0, ...) returns: the point of a cell is
 * v0 + xi (v1 - v0) + eta (v2 - v0) (vertex order of the exchange format). The rule integrates
 * polynomials of degree 2 floor((3k+4)/2) - 1 exactly, so data of degree up to that minus the
 * space's degree is projected exactly (it reproduces every polynomial of the space).
 *   field 0: values_at_qp double[ncells][2][nq] (x and y components) -> dofs = Q (nodal, device)
 *   field 1: values_at_qp double[ncells][nq]                          -> dofs = p (nodal, device)
 * The projection is cell-local: dofs_K = argmin over the space of ||u - f||_{L2(K)} with the
 * integral replaced by the rule. HDG_ERR_INVALID_ARG for another field or a NULL pointer. */
hdg_status hdg_project(hdg_ctx *ctx, int field, const double *values_at_qp, double *dofs);

/* Forcing f(x, t) = phi(t) F(x) with F a velocity field (nodal, device): f^ex(w, t) =
 * (w . f(t)) (eq. f_expl). phi is called on the host, once per stage time of each step (for a
 * step recorded as a CUDA graph, before the graph's launch: the graph reads the values from device
 * memory); NULL phi means phi = 1. F = NULL removes the forcing. */
hdg_status hdg_set_forcing(hdg_ctx *ctx, const double *F, double (*phi)(double t, void *user), void *user);

/* Several contexts advanced together: nsteps steps of Alg. 1 for each context. Per step, every
 * context's step (recorded as one CUDA graph, see device_loops) is enqueued on its own stream
 * before any is waited for, so independent instances of different mesh sizes and degrees run on
 * the GPU at the same time; contexts whose steps cannot be one graph take theirs synchronously in
 * turn. Each result is the one hdg_imex_step gives for that context alone (bitwise: the kernels
 * are deterministic and the contexts share no buffers). Contexts should have distinct streams
 * (shared streams serialise their work). stats: n entries or NULL. The paper has no counterpart
 * (it times one run at a time). Returns the first error met; HDG_ERR_NOT_CONVERGED if any context's
 * stage solves stopped at their cap. */
hdg_status hdg_batch_step(hdg_ctx *const *ctxs, int n, int nsteps, hdg_stats *stats);
/* Device bytes the context has allocated so far (host query). */
size_t hdg_ctx_bytes(const hdg_ctx *ctx);
/* Upper estimate (bytes) of the device memory of a context with this mesh and these parameters
 * once it has taken IMEX steps (host-only; 0 for invalid arguments). */
double hdg_estimate_bytes(const hdg_mesh_desc *mesh, const hdg_params *params);

/* Serving runtime: independent Euler runs ("requests": a mesh, parameters, an initial velocity
 * and a number of IMEX steps) of different sizes and degrees, admitted in arrival order while the
 * device-memory budget (hdg_estimate_bytes of the request's configuration, plus the bytes every
 * context holds) and the slot limit allow, and advanced together with continuous batching: each
 * call of hdg_server_progress admits what fits, takes one step of every active request at once
 * (hdg_batch_step) and retires the requests that have taken their steps. Contexts stay resident
 * on the device with their condensed operators and recorded step graphs: a retired request's
 * context is kept idle and reused by the next request with the same configuration (mesh and
 * parameters), and idle contexts are released, least recently used first, when an admission
 * needs their memory. Each request's result equals the result of running it alone. One host
 * thread at a time per server. The paper has no counterpart. */
typedef struct hdg_server hdg_server;
typedef struct {
    int submitted, admitted, completed, active, queued;
    int contexts_created, contexts_reused, contexts_released;
    double bytes_in_use;        /* device bytes held by the server's contexts (active and idle) */
    long long steps;            /* IMEX steps taken over all requests */
    long long stage_solves;     /* stage solves over all requests */
} hdg_server_stats;
hdg_status hdg_server_create(hdg_server **out, int device, double mem_budget_bytes, int max_active);
/* Q0_host: the request's initial velocity (host, nodal, the Q layout); it is copied. The initial
 * state is (Q0, p = 0, lambda = 0) projected to be divergence-free with its pressure reconstructed
 * (hdg_div_free_project) before the first step. id: the request's number. */
hdg_status hdg_server_submit(hdg_server *srv, const hdg_mesh_desc *mesh, const hdg_params *params,
                             const double *Q0_host, int nsteps, long long *id);
hdg_status hdg_server_progress(hdg_server *srv, hdg_server_stats *stats);
/* A completed request's result (host arrays in the exchange layouts, any may be NULL) and its
 * latency from submission to completion in ms (host clock); releases the result. HDG_ERR_INVALID_ARG
 * if the request is unknown or not complete. */
hdg_status hdg_server_result(hdg_server *srv, long long id, double *Q_host, double *p_host, double *lam_host,
                             double *latency_ms);
void hdg_server_destroy(hdg_server *srv);

/* Passive tracer (App. B): q in DG_k (nodal, device, the pressure layout double[ncells][(k+1)(k+2)/2])
 * advected explicitly by every hdg_imex_step with the explicit tableau of the IMEX method:
 *   q_i = q^n + dt sum_{j<i} a^ex_ij d_j,  q^{n+1} = q^n + dt sum_i b^ex_i d_i,
 *   d_i = M^-1 a(., q_i, P_CG(Q_i)),  a(chi, q, U) = (q, div(chi U)) - sum over interior facets
 *   <q^up [[chi U.n]]>  (q^up: the upwind value; U.n at a facet point averaged over its sides)
 * (eq. advection_update_stages, eq. advection_update_final; the printed final sum starts at i = 1,
 * which would leave IMEX Euler's tracer (b^ex = (1, 0)) unchanged: it is read from i = 0). Q_i are
 * the step's stage velocities (Q_0 = Q^n for an explicit first stage). P_CG is the L2 projection
 * onto the continuous space CG_{k+1} (Jacobi-preconditioned CG on the device, to 1e-13). Walls
 * carry no tracer flux. q = NULL removes the tracer. */
hdg_status hdg_set_tracer(hdg_ctx *ctx, const double *q);
hdg_status hdg_get_tracer(hdg_ctx *ctx, double *q);
/* Component entry points of the tracer: Qcg = P_CG(Q) (nodal DG velocities in and out; the output
 * takes one value per lattice point shared by several cells), and dq = M^-1 a(., q, U) (nodal DG_k
 * in and out) for a continuous velocity U (e.g. the output of hdg_cg_project). */
hdg_status hdg_cg_project(hdg_ctx *ctx, const double *Q, double *Qcg);
hdg_status hdg_tracer_rhs(hdg_ctx *ctx, const double *q, const double *U, double *dq);

/* Alg. 1 x nsteps: s-1 stage solves (Alg. 2), final update (eq. final_update) and pressure
 * reconstruction (Sec. 2.7) per step, on the context's state. Stages solved to a tolerance
 * (n_richardson = 0) start, once a step has been taken, from their own solutions in the
 * previous steps (velocity shifted by the state's change over the last step, pressure and trace
 * extrapolated from the last two); otherwise, and with a fixed number of Richardson sweeps, from
 * the previous stage's values. hdg_div_free_project and hdg_reconstruct_pressure drop that
 * history. */
hdg_status hdg_imex_step(hdg_ctx *ctx, int nsteps, hdg_stats *stats);

/* One stage solve (Alg. 2): find (Q, p, lambda) with
 *   (Q.w) - c (f^impl(w, Q, Q*) + g(w, p, lambda)) = (R, w),  Gamma(psi, mu, Q, p, lambda) = 0
 * (eq. imex_implicit_solve + constraint). R: Riesz representer of the right-hand side; Qstar:
 * the advecting velocity (used as given; pass P(Q_{i-1}) for the paper's scheme). Q, p, lam:
 * initial iterate in, result out (nodal, device). */
hdg_status hdg_solve_stage(hdg_ctx *ctx, double c, const double *R, const double *Qstar,
                           double *Q, double *p, double *lam, hdg_stats *stats);

/* Component entry points (each one row of the hot path, for verification):
 * BDM^0_{k+1} projection Q* = P(Q) (Sec. 2.3). */
hdg_status hdg_bdm_project(hdg_ctx *ctx, const double *Q, double *Qstar);
/* Riesz representer of w -> f^impl(w, Q, Q*) (eq. f_impl). */
hdg_status hdg_fimpl_apply(hdg_ctx *ctx, const double *Qstar, const double *Q, double *out);
/* Tentative velocity (Alg. 2 Step I): (Qbar.w) - c f^impl(w, Qbar, Q*) = (R, w). */
hdg_status hdg_tentative_solve(hdg_ctx *ctx, double c, const double *Qstar, const double *R,
                               double *Qbar, hdg_stats *stats);
/* Mixed solve (the operator of Step II, eq. final_update and Sec. 2.7):
 *   (U.w) - c g(w, p, lambda) = (R, w),   Gamma(psi, mu, U, p, lambda) = -Gamma(psi, mu, X, 0, 0)
 * with (p)_Omega = 0. R or X may be NULL (zero). Outputs nodal, device. */
hdg_status hdg_mixed_solve(hdg_ctx *ctx, double c, const double *R, const double *X,
                           double *U, double *p, double *lam, hdg_stats *stats);
/* Riesz representer (on the trace space) of the condensed trace operator applied to lam:
 * mu -> sum_K <S_K lam, mu> for coefficient c (Sec. 2.8, the operator the CG solves with). */
hdg_status hdg_trace_apply(hdg_ctx *ctx, double c, const double *lam, double *out);
/* Replace the state's Q by its discretely divergence-free part (Step II with c = 1), and set
 * (p, lambda) to the pressure reconstruction of the result (Sec. 2.7). */
hdg_status hdg_div_free_project(hdg_ctx *ctx, hdg_stats *stats);
/* Pressure reconstruction (Sec. 2.7) of the state's Q at the state's time. */
hdg_status hdg_reconstruct_pressure(hdg_ctx *ctx, hdg_stats *stats);

/* Instrumentation: launch one kernel of the path `reps` times on the context's stream between
 * CUDA events (after one untimed launch) and report the mean device time per launch and the
 * algorithmic bytes one launch moves (operator entries it must read + vectors read/written
 * once). which = 0: trace operator apply fused with the CG direction update and dot product
 * (the kernel the trace CG runs every iteration) for coefficient c; which = 1: tentative-velocity
 * operator apply (dense diagonal blocks, matrix-free neighbour coupling) for the operator last
 * assembled (call hdg_tentative_solve or hdg_imex_step first). Operands are the context's
 * current buffers.
 * which = 2..5 (stage solves to tolerance only; bytes = 0) time one component of the stage
 * preconditioner, recorded as a CUDA graph with device-side loops, for the stage operator at
 * coefficient c around the current state and v = (M Q, 0, 0): 2 = Step-I solve to
 * inner_stepI_rtol, 3 = Step-II (mixed) solve to inner_trace_rtol, 4 = the whole Chorin-split
 * preconditioner, 5 = the stage operator apply. which = 6: the FP32 Arnoldi product of the inner
 * Step-I GMRES (neighbour coupling of B^-1 v_j, the dots with the basis and ||w||, the Givens
 * step) at step j = 4, launched alone after one inner solve has filled the basis (each launch
 * after a one-thread kernel that resets the step, whose time is subtracted); bytes = its
 * algorithmic bytes. which = 7 (bytes = 0): the preconditioner's Step II as the stage solves run it
 * (FP32 cell maps, then the inner trace solve: one V-cycle, in FP32 when inner_trace_fp32 is on),
 * recorded and replayed like 2..5. which = 8: the fused stage-operator kernel the stage solves
 * take for their FP64-accurate products, alone (the FGMRES matrix-vector product without the
 * facet gather: FP64, or under HDG_MIXED with relax_eta > 0 and a stage tolerance of 5e-11 or
 * more the pair-arithmetic kernel reading the block as its FP32 copy and rest), on the operator
 * last assembled, input the current state; bytes = its algorithmic bytes. which = 9: the FP32
 * preconditioner pass of the inner Step-I GMRES (v_j formed from w and the projections, z = B^-1 v_j, z's edge values) at
 * step j = 4, launched like 6; bytes = its algorithmic bytes. which = 10 (bytes = 0): one inner FP32
 * Arnoldi step as the solve runs it (preconditioner passes, product, finishing kernel), from 20 steps
 * launched back to back after a cycle start, less the cycle start alone. which = 11: the per-cell
 * condensation (k_condense, Sec. 2.8) for coefficient c alone; bytes = geometry read + S_K, Z_K and
 * A_K^-1 written. which = 12: the FP32 stage-operator kernel (the relaxed FGMRES product, see
 * relax_eta) alone, like 8, on the FP32 copy of the diagonal blocks of the last stage assembly
 * (needs HDG_MIXED with stage_krylov and relax_eta > 0, and a stage solve run first); bytes =
 * its algorithmic bytes. which = 13, 14 (inner_gs on): the red-black Gauss-Seidel kernels of the
 * inner FP32 Step-I GMRES at step j = 4, launched like 6: 13 = the colour pass (k_gs_diag; both
 * colours launched, time and bytes per launch), 14 = the Arnoldi product with its dots
 * (k_gs_apply); bytes = their algorithmic bytes. which = 15: the Step-I assembly kernel alone
 * (k_fimpl_assemble in the stage solves' form: block and weights, no FP64 inverse) for coefficient
 * c around the current state's BDM projection (the context's Step-I operator is overwritten; the
 * next stage solve assembles its own); which = 16: the BDM projection kernel alone on the current
 * state (in pairs under HDG_MIXED, as the stage solves take it); bytes = their algorithmic bytes. */
hdg_status hdg_time_kernel(hdg_ctx *ctx, int which, double c, int reps, double *ms_per_launch,
                           double *bytes_per_launch);

/* The trace-operator apply of hdg_trace_apply (same operator, same output) without any device
 * allocation. The paper has no counterpart. It serves callers that must not call cudaMalloc once
 * they run: hosts that hand all device memory to their own pool allocator at start-up (a library
 * allocation would then fail or break the pool's accounting), and time-critical loops for which
 * cudaMalloc is off limits because it may synchronise the whole device. hdg_trace_apply may
 * allocate: it caches the condensed operator of every new coefficient c. This variant condenses
 * the cells again on every call and keeps its intermediate vectors in one static device array of
 * 2^20 doubles (8 MiB) inside the library, which every GPU that loads the library holds until the
 * process exits.
 *   Limit: 3 * nlambda + ncells * 3(k+1) <= 2^20 doubles (e.g. 64 x 64 meshes with k <= 4,
 *   128 x 128 with k <= 3); larger meshes return HDG_ERR_INVALID_ARG with the sizes in
 *   hdg_last_error().
 *   The context's device must be the current device (else HDG_ERR_INVALID_ARG). The first call on
 *   each device looks up the array's device address (cudaGetSymbolAddress, once per device, under a
 *   lock); make that first call before any stream capture begins.
 *   Every call on a device shares the array, which keeps the last call's contents (nothing in it
 *   needs to start at zero: every element a call reads it has written first). Calls whose work
 *   overlaps on the GPU (other streams, other contexts, other host threads) race on the array and
 *   must be ordered by the caller. The context's own buffers are not touched. lam and out hold
 *   nlambda doubles each (device). Synchronises the context's stream before returning. */
hdg_status hdg_trace_apply_noalloc(hdg_ctx *ctx, double c, const double *lam, double *out);

#ifdef __cplusplus
}
#endif
#endif
