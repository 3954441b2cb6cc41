/*
 * emd_gb300.h -- C ABI of the GB300 (sm_103a) dynamic-formulation EMD misfit library.
 *
 * The library computes the earth mover's distance between an observed and a predicted
 * seismic gather on an nr x nt grid (receivers x time), as defined in Sec. 2.1-2.2 of
 * arXiv 1808.07284: the gathers are compared through the Mainini recombination
 * mu = Pcal+ + Pobs-, nu = Pobs+ + Pcal- (Sec. 2.1), and the distance is
 *     min_u ||u||_{1,1} + eps/2 ||u||_2^2   s.t.  div u + Pcal - Pobs = 0,  zero boundary flux
 * times dx*dt, solved by PDHG with linesearch (Algorithm 1).  The solver returns the
 * distance, the dual potential phi (the adjoint source, Sec. 2.3) and the flux m = u.
 *
 * Conventions shared by every entry point:
 *  - Grids are row-major [nr][nt]: element (i, j) sits at i*nt + j; i = receiver
 *    (spacing dx), j = time sample (spacing dt, contiguous).  The flux m is [2][nr][nt]:
 *    the x (receiver) component plane first, then the t (time) plane.
 *  - Every array argument is a DEVICE pointer owned by the caller, FP32, unless stated
 *    otherwise.  The library never allocates device memory: scratch space is the
 *    caller's `workspace` (device, 256-byte aligned, size from the *_workspace_size
 *    queries) and is only valid for the duration of the call.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default stream).
 *    Calls that return host results (emd_result, masses) synchronise that stream
 *    before returning.
 *  - Every call validates its arguments and returns EMD_ERR_ARG without launching
 *    anything when they are invalid (nt >= 2, nr >= 1, dt > 0, dx > 0 and finite,
 *    0 < xi < 1, 0 < zeta < 1, delta > 0, eps >= 0, max_iter >= 1, non-null pointers).
 *    Device-side failures (non-finite iterates, a linesearch that never passes) come
 *    back as a status, never as a trap; a CUDA error is EMD_ERR_CUDA.
 *  - No entry point is reentrant on the same workspace: calls that share a workspace
 *    must be ordered (same stream, or synchronised).
 */
#ifndef EMD_GB300_H
#define EMD_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without requiring the CUDA headers. */
typedef struct CUstream_st *emd_stream_t;

typedef enum {
  EMD_OK = 0,
  EMD_ERR_ARG = 1,        /* invalid argument; nothing was launched                      */
  EMD_ERR_CUDA = 2,       /* a CUDA runtime call failed (launch, copy, sync)             */
  EMD_ERR_NONFINITE = 3,  /* an inner product became NaN/Inf (e.g. NaN in the inputs)    */
  EMD_ERR_LINESEARCH = 4, /* Algorithm 1's backtracking did not pass in ls_max_trials    */
  EMD_ERR_TIMEOUT = 5,    /* a bounded device-side wait (4 s) of a persistent solve ran out;
                             the kernel winds down instead of hanging                    */
  EMD_ERR_WORKSPACE = 6   /* workspace NULL, too small or not 256-byte aligned           */
} emd_status;

typedef enum {
  EMD_BAL_NONE = 0, /* solve with f = Pcal - Pobs as printed (infeasible if sum f != 0)   */
  EMD_BAL_MEAN = 1  /* remove the mean of f first, so that the zero-flux problem is feasible */
} emd_balance;

/* Ground cost of the flux norm.  The paper's Phi uses ||u||_{1,1} = sum |u^x| + |u^t|
 * (Sec. 2.2); the isotropic ||u||_{1,2} = sum sqrt((u^x)^2 + (u^t)^2), with u^x and u^t of
 * one grid index paired, is the formulation of the work the paper builds on (its prox is
 * the vector shrink max(1 - alpha/||v||, 0) v).  dist and dist_l1 use the chosen norm. */
typedef enum {
  EMD_NORM_ANISO = 1, /* ||u||_{1,1} (default, as printed)                                */
  EMD_NORM_ISO = 2    /* ||u||_{1,2}                                                     */
} emd_norm;

/*
 * Solver parameters (Sec. 2.2 and Algorithm 1).  emd_default_params() fills the paper's
 * constants: eps = 1e-4, xi = 0.5, zeta = 0.99, delta = 1e5, plus max_iter = 2000,
 * tol = 0, check_every = 10, ls_max_trials = 40, linesearch = 1, ls_norm = 2,
 * balance = EMD_BAL_MEAN, no warm start, tile = 0, launch_mode = 0, no trace,
 * norm = EMD_NORM_ANISO.
 */
typedef struct {
  double eps;        /* regularisation epsilon of Phi = ||u||_{1,1} + eps/2 ||u||^2      */
  double xi;         /* backtracking factor of the linesearch, in (0, 1)                 */
  double zeta;       /* linesearch test constant, in (0, 1)                              */
  double delta;      /* dual/primal step ratio: beta = delta * alpha                     */
  double alpha0;     /* first primal step; <= 0 selects 1/sqrt(delta*lambda) with the
                        bound lambda = 4/dx^2 + 4/dt^2 (4/dt^2 when nr == 1); with
                        linesearch == 0 it selects alpha = beta = 1/sqrt(lambda)         */
  double tol;        /* stop when max(||div u + f|| / ||f||, ||u^{k+1}-u^k|| / ||u^{k+1}||)
                        <= tol, tested every check_every iterations; 0 = run max_iter    */
  int max_iter;      /* cap on accepted PDHG iterations (>= 1)                           */
  int check_every;   /* iterations between stopping tests (>= 1)                         */
  int ls_max_trials; /* backtracking trials per iteration before EMD_ERR_LINESEARCH       */
  int linesearch;    /* 1: Algorithm 1; 0: fixed-step PDHG with ubar = 2u^{k+1} - u^k    */
  int ls_norm;       /* norm of the linesearch test; only 2 (Euclidean) is implemented   */
  int balance;       /* emd_balance                                                      */
  const float *phi_init; /* optional warm start for phi, device [nr][nt]; NULL = zeros   */
  const float *m_init;   /* optional warm start for u, device [2][nr][nt]; NULL = zeros  */
  int tile;          /* stencil tile-shape id (emd_tile_count() of them); 0 = automatic:
                        gathers of <= 7168 cells are solved in shared memory (one CTA
                        each, launch_mode 0), thin ones (<= 8 receivers) by the plain
                        pass, the rest by the TMA pass in the tile shape an autotuner
                        picks on the first solve of each (device, sizes) configuration
                        (a few short timed trial solves, then cached per process)       */
  int launch_mode;   /* 0: automatic -- every pass in one persistent cooperative launch when
                        the TMA pass serves the gathers, else graph replays of the pass;
                        1: one plain launch per pass; 2: one launch per pass, replayed
                        from a captured CUDA graph                                       */
  int debug_fault;   /* fault injection for tests, never set in production: 0 = off;
                        1 = every linesearch trial fails (exercises EMD_ERR_LINESEARCH);
                        2 = the persistent solve never publishes a decision, so its
                        bounded waits run out after 4 s and it winds down (exercises
                        EMD_ERR_TIMEOUT; the resident and per-pass paths ignore it)    */
  double *trace;     /* optional per-iteration history, device, B x max_iter x 4 doubles
                        (gather-major): for iteration k, alpha_{k+1}, theta_{k+1}, the
                        linesearch trials it took, and ||div u^{k+1} + f|| / ||f||.
                        Entries past a gather's last iteration are left untouched.
                        NULL = no history.                                                */
  int norm;          /* emd_norm: EMD_NORM_ANISO (default) or EMD_NORM_ISO                */
} emd_params;

/* Host-side result of one solve.  Distances are in the units of dx*dt*|u|. */
typedef struct {
  double dist;        /* dx*dt*Phi(u): the EMD misfit as defined in Sec. 2.2             */
  double dist_l1;     /* dx*dt*||u||_{1,1}: the same without the eps term                */
  double mass_mu;     /* dx*dt*sum(mu), mu = Pcal+ + Pobs-                               */
  double mass_nu;     /* dx*dt*sum(nu), nu = Pobs+ + Pcal-                               */
  double imbalance;   /* mass_mu - mass_nu = dx*dt*sum(Pcal - Pobs)                     */
  double residual;    /* max(r_feas, r_step) after the last iteration                    */
  double r_feas;      /* ||div u + f||_2 / ||f||_2                                       */
  double r_step;      /* ||u^{k+1} - u^k||_2 / ||u^{k+1}||_2                             */
  double duality_gap; /* dx*dt*(Phi(u) - <phi,f> + sum h*(grad phi)), h* the conjugate of
                         |v| + eps/2 v^2; tends to 0 at the saddle point                 */
  double alpha;       /* last accepted primal step alpha_k                               */
  double theta;       /* last theta_k                                                    */
  int iters;          /* accepted PDHG iterations                                        */
  int ls_trials;      /* linesearch trials in total (>= iters)                           */
  int status;         /* emd_status of this solve                                        */
  int launches;       /* kernel launches this solve made (a graph's nodes count one each) */
  int tile;           /* tile-shape id the solve ran (1..emd_tile_count(); the autotuner's
                         choice when params->tile was 0); 0 for the shared-memory solve     */
} emd_result;

/* Fills *p with the defaults listed above.  p must not be NULL. */
void emd_default_params(emd_params *p);

/* Number of stencil tile shapes compiled into the library (valid ids: 1..count).  Ids 1-6
 * are the plain-staging pass (16/8/32 x 120, 8/16 x 248, 1 x 248 tiles), 7-9 the
 * TMA-staged tile pass (13, 8 and 21 x 120 tiles), 10-11 the marching pass (a warp walks
 * 120-sample strips down the receivers with 6 or 4 rows in flight). */
int emd_tile_count(void);

/* Bytes of device workspace emd_dyn_solve needs for one nr x nt gather (0 if invalid). */
size_t emd_workspace_size(int nt, int nr);

/*
 * Mainini decomposition and recombination (Sec. 2.1).
 * Inputs f_obs, f_pred: device [nr][nt].  Outputs (each nullable): mu, nu device
 * [nr][nt] with mu = Pcal+ + Pobs-, nu = Pobs+ + Pcal-; masses (HOST, 2 doubles)
 * = {dx*dt*sum(mu), dx*dt*sum(nu)} accumulated in FP64 (dt alone when nr == 1).
 * Needs emd_workspace_size(nt, nr) bytes of workspace (only a few KB are touched).
 * Synchronises `stream` when masses != NULL.
 */
emd_status emd_decompose(const float *f_obs, const float *f_pred, int nt, int nr, double dt,
                         double dx, float *mu, float *nu, double *masses, void *workspace,
                         size_t ws_bytes, emd_stream_t stream);

/*
 * One EMD solve: Algorithm 1 (PDHG with linesearch) on f = Pcal - Pobs (Sec. 2.2).
 * Inputs f_obs (Pobs), f_pred (Pcal): device [nr][nt].  params: host pointer (NULL =
 * defaults).  Outputs: phi device [nr][nt] (the dual potential after the last
 * iteration), m device [2][nr][nt] (the flux u), result HOST (required).
 * Iterates are FP32; the linesearch inner products, the stopping residual, the mass
 * sums and the distance accumulate in FP64.  Algorithm 1 lets alpha_{k+1} be chosen in
 * [alpha_k, alpha_k sqrt(1 + theta_k)]: the solver takes the upper end, except for
 * identical gathers (the balanced f identically zero, and with it the dual move for every
 * step size), where it keeps alpha_k; such a solve returns phi = 0, m = 0 and distance 0
 * with status EMD_OK at any iteration count.  Returns the solve's status (also in
 * result->status).  Synchronises `stream`.
 */
emd_status emd_dyn_solve(const float *f_obs, const float *f_pred, int nt, int nr, double dt,
                         double dx, const emd_params *params, float *phi, float *m,
                         emd_result *result, void *workspace, size_t ws_bytes,
                         emd_stream_t stream);

/* Bytes of workspace for emd_dyn_solve_batched over B gathers of sizes nt[b] x nr[b]
 * (host arrays).  0 if any size is invalid. */
size_t emd_batched_workspace_size(int B, const int *nt, const int *nr);

/*
 * B independent solves (the paper solves one EMD per shot), each gather with its own
 * linesearch state; gathers that meet tol stop while the rest go on.  How the passes are
 * launched follows params->launch_mode as for emd_dyn_solve: by default (0) one persistent
 * cooperative launch runs every PDHG iteration of every gather (gathers of at most 7168
 * cells each get one shared-memory-resident CTA instead); 1 issues one launch per
 * iteration over all gathers, 2 replays those launches from a captured CUDA graph.  All arrays of pointers and sizes are HOST
 * arrays of length B; the pointers they hold are device pointers with the layouts of
 * emd_dyn_solve.  params apply to every gather (its warm-start pointers must be NULL).
 * results: HOST array of B.  Returns EMD_OK if every gather succeeded, else the first
 * non-OK status (each gather's own status is in results[b].status).
 */
emd_status emd_dyn_solve_batched(int B, const float *const *f_obs, const float *const *f_pred,
                                 const int *nt, const int *nr, const double *dt,
                                 const double *dx, const emd_params *params,
                                 float *const *phi, float *const *m, emd_result *results,
                                 void *workspace, size_t ws_bytes, emd_stream_t stream);

/*
 * Adjoint source of the returned distance (Sec. 2.3: d f_OT / d Pcal = phi).
 * With dist = dx*dt*Phi, d dist / d Pcal = g * dx*dt * (phi - mean(phi)) when
 * balance == EMD_BAL_MEAN (phi - 0 otherwise), g = *grad_out (device FP32 scalar; NULL
 * means 1).  grad_pred receives it, grad_obs (nullable) its negative; both device
 * [nr][nt].  Needs emd_workspace_size(nt, nr) bytes of workspace.  Does not synchronise.
 */
emd_status emd_adjoint(const float *phi, int nt, int nr, double dt, double dx, int balance,
                       const float *grad_out, float *grad_pred, float *grad_obs,
                       void *workspace, size_t ws_bytes, emd_stream_t stream);

/* Bytes of workspace emd_adjoint_batched needs for B gathers (0 if B < 1). */
size_t emd_batched_adjoint_workspace_size(int B);

/*
 * Adjoint sources of B gathers at once (Sec. 2.3, as emd_adjoint for each gather): one
 * launch sums every gather's phi (balance == EMD_BAL_MEAN), one launch scales them.
 * phi, grad_pred: HOST arrays of B device pointers ([nr[b]][nt[b]] each, FP32); grad_obs:
 * HOST array of B device pointers or NULL (entries may be NULL); nt, nr, dt, dx: HOST
 * arrays of B.  grad_out: device array of B FP32 upstream gradients, NULL meaning 1 for
 * every gather.  Workspace: emd_batched_adjoint_workspace_size(B) bytes (device, 256-byte
 * aligned).  Does not synchronise.
 */
emd_status emd_adjoint_batched(int B, const float *const *phi, const int *nt, const int *nr,
                               const double *dt, const double *dx, int balance,
                               const float *grad_out, float *const *grad_pred,
                               float *const *grad_obs, void *workspace, size_t ws_bytes,
                               emd_stream_t stream);

/* Bytes of workspace for emd_misfit_batched_host over B gathers of sizes nt[b] x nr[b]
 * (host arrays): the batched solve's and the batched adjoint's workspaces, then device
 * staging for each gather's inputs, phi and m.  0 if any size is invalid. */
size_t emd_misfit_batched_host_workspace_size(int B, const int *nt, const int *nr);

/*
 * The misfit step of a full-waveform inversion for gathers held in HOST memory: the B
 * distances (Sec. 2.1-2.2, Algorithm 1; as emd_dyn_solve_batched) and their adjoint
 * sources d dist_b / d Pcal_b (Sec. 2.3; as emd_adjoint_batched with params->balance and
 * upstream gradient 1), host buffers in and out.
 *  - f_obs, f_pred: HOST arrays of B HOST pointers, each [nr[b]][nt[b]] FP32 row-major.
 *  - grad_pred: HOST array of B HOST pointers that receive the adjoint sources (same
 *    layout), or NULL for the distances only; entries may be NULL.
 *  - nt, nr, dt, dx, results: HOST arrays of B.  params as for emd_dyn_solve_batched; the
 *    warm-start pointers must be NULL (trace, if set, is a device array as documented).
 *  - workspace: emd_misfit_batched_host_workspace_size(B, nt, nr) bytes, device, 256-byte
 *    aligned; phi and m of the solve are kept there and not returned.
 * The inputs are copied into the workspace gather by gather on a stream the call creates
 * (ordered after the caller's earlier work on `stream`); each gather's preparation (f, the
 * mass sums, zeroed iterates) is launched on `stream` behind an event on its own copy, so
 * it overlaps the copies still in flight.  One batched solve, one batched adjoint and the
 * copies of the adjoint sources back to grad_pred follow on `stream`, which the call
 * synchronises: on return the host buffers hold the results.  Page-locked host memory
 * (cudaHostAlloc, cudaHostRegister) gives the copies the host link's full rate and the
 * overlap; pageable memory also works, staged by the CUDA driver.  The call allocates no
 * device memory; it creates and destroys one stream and B + 1 events.
 * Returns as emd_dyn_solve_batched (adjoint sources are still computed for gathers with a
 * non-OK status); EMD_ERR_ARG, without copying or launching anything, for an invalid
 * argument, B > 65535 included; EMD_ERR_WORKSPACE for a NULL, short or misaligned
 * workspace.
 */
emd_status emd_misfit_batched_host(int B, const float *const *f_obs, const float *const *f_pred,
                                   const int *nt, const int *nr, const double *dt,
                                   const double *dx, const emd_params *params,
                                   float *const *grad_pred, emd_result *results, void *workspace,
                                   size_t ws_bytes, emd_stream_t stream);

/*
 * emd_dyn_solve without a workspace argument, for callers that cannot allocate device
 * memory: code whose host framework owns every device allocation (a custom allocator or
 * a fixed memory budget), real-time loops that must never block on an allocation, or
 * plug-ins that are handed only input and output buffers.  The paper has no counterpart;
 * this is a deployment convenience.
 *
 * Scratch space is a 16 MiB array compiled into the library (every GPU that loads the
 * library holds it until the process exits), so the gather must satisfy
 * emd_workspace_size(nt, nr) <= 16 MiB (about 450k cells, e.g. 1024 x 400); larger
 * gathers return EMD_ERR_WORKSPACE without launching anything.  Arguments, outputs and
 * results are those of emd_dyn_solve, with two differences: tile = 0 takes the library's
 * default tile shape without the autotuner's timed trial solves, and no CUDA graph is
 * captured (launch_mode 0 runs the shared-memory or the persistent cooperative solve and,
 * where neither can be launched, one plain launch per pass; launch_mode 2 is run as 1).
 * Nothing calls cudaMalloc or cudaFree.  Like emd_dyn_solve the call copies small host
 * tables to the device and synchronises `stream` to read the result back.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress with that device
 * current).  Every call on a device shares the one array, which keeps the last call's
 * contents (each call re-initialises what it needs): calls that overlap on the GPU
 * (different streams, or different host threads without ordering) race and give wrong
 * results.
 */
emd_status emd_dyn_solve_noalloc(const float *f_obs, const float *f_pred, int nt, int nr,
                                 double dt, double dx, const emd_params *params, float *phi,
                                 float *m, emd_result *result, emd_stream_t stream);

/*
 * Two-grid solve (Sec. 2.2, closing paragraph; Sec. 3.3).  The paper speeds up large
 * gathers by solving the EMD on a resampled, coarser gather, building the primal variable
 * on the original grid by sinc interpolation and running the primal-dual method on the
 * fine grid from there (Sec. 3.3: time resampled 3000 -> 301 samples, 150 coarse
 * iterations).  Readings fixed here:
 *  - the coarse grid coarsens the time axis only, by the integer `factor` r: coarse
 *    sample J of a row is the mean of fine samples rJ .. rJ + r - 1 (record padded with
 *    zeros to a multiple of r, so the mass is kept), coarse spacing r*dt, same dx;
 *  - sinc interpolation is the Whittaker-Shannon sum over every coarse sample of the
 *    record, at fine positions (j - (r-1)/2)/r (cell-centred: phi, x flux) or j/r (time
 *    flux, which sits on the faces between time cells), in coarse-sample units; the
 *    outer faces (x flux of receiver 0, time flux of sample 0) are zero;
 *  - phi is interpolated along with u unless interpolate_phi = 0 (then the fine solve
 *    starts from phi = 0, the paper's sentence read literally).
 */
typedef struct {
  int factor;          /* time coarsening r >= 1 (1 = a coarse solve on the fine grid)    */
  int coarse_max_iter; /* cap on the coarse solve's accepted iterations (>= 1)            */
  double coarse_tol;   /* the coarse solve's stopping residual; 0 = run coarse_max_iter   */
  int interpolate_phi; /* 1: phi is interpolated too (default); 0: fine phi starts at 0  */
} emd_mg_params;

/* Fills *p: factor = 10, coarse_max_iter = 150, coarse_tol = 0 (the Sec. 3.3 setting),
 * interpolate_phi = 1.  p must not be NULL. */
void emd_default_mg_params(emd_mg_params *p);

/* Bytes of workspace emd_dyn_solve_mg needs (0 if invalid, e.g. ceil(nt/factor) < 2).
 * Never less than emd_workspace_size(nt, nr). */
size_t emd_mg_workspace_size(int nt, int nr, int factor);

/* The same for emd_dyn_solve_batched_mg over B gathers (host size arrays). */
size_t emd_batched_mg_workspace_size(int B, const int *nt, const int *nr, int factor);

/*
 * Time restriction, the first step of the two-grid solve: out[i][J] = (1/r) *
 * sum_{j = rJ}^{min(rJ + r, nt) - 1} in[i][j] for J < ceil(nt / r).  in: device [nr][nt],
 * out: device [nr][ceil(nt / r)], FP32 (summed in FP32, in order of j).  r >= 1.
 * Does not synchronise.
 */
emd_status emd_restrict_time(const float *in, int nt, int nr, int factor, float *out,
                             emd_stream_t stream);

/*
 * Sinc interpolation, the third step of the two-grid solve: out[i][j] = sum_J in[i][J]
 * sinc(x_j - J), J < nc, j < nt, with x_j = j / r when staggered = 1 (time faces) and
 * (j - (r - 1)/2) / r when staggered = 0 (cell centres).  zero_row0 / zero_col0 = 1 write
 * 0 to row 0 / column 0 (outer faces).  in: device [nr][nc], out: device [nr][nt], FP32
 * accumulation.  Does not synchronise.
 */
emd_status emd_prolong_time(const float *in, int nc, int nr, int factor, int nt, int staggered,
                            int zero_row0, int zero_col0, float *out, emd_stream_t stream);

/*
 * Two-grid EMD solve: restriction of f_obs and f_pred, a coarse Algorithm 1 solve (params
 * with max_iter = coarse_max_iter and tol = coarse_tol, no trace), sinc interpolation of
 * its phi and u into the output arrays phi and m, and the fine Algorithm 1 solve with
 * params, warm-started from there.  Arguments are those of emd_dyn_solve, plus mg (host,
 * NULL = defaults) and coarse (HOST, nullable: the coarse solve's result, on the coarse
 * grid).  params->phi_init and params->m_init must be NULL (the warm start is the coarse
 * solution).  result describes the fine solve; result->launches counts every launch of
 * the call.  Workspace: emd_mg_workspace_size(nt, nr, mg->factor) bytes.  A coarse solve
 * that fails returns its status without the fine solve.  Synchronises `stream`.
 */
emd_status emd_dyn_solve_mg(const float *f_obs, const float *f_pred, int nt, int nr, double dt,
                            double dx, const emd_params *params, const emd_mg_params *mg,
                            float *phi, float *m, emd_result *result, emd_result *coarse,
                            void *workspace, size_t ws_bytes, emd_stream_t stream);

/*
 * Batched two-grid solve: both stages of every gather run as one batched solve each (one
 * restriction and one interpolation launch for all gathers).  Arguments are those of
 * emd_dyn_solve_batched plus mg and coarse (HOST array of B, nullable).  Workspace:
 * emd_batched_mg_workspace_size(B, nt, nr, mg->factor) bytes.
 */
emd_status emd_dyn_solve_batched_mg(int B, const float *const *f_obs,
                                    const float *const *f_pred, const int *nt, const int *nr,
                                    const double *dt, const double *dx,
                                    const emd_params *params, const emd_mg_params *mg,
                                    float *const *phi, float *const *m, emd_result *results,
                                    emd_result *coarse, void *workspace, size_t ws_bytes,
                                    emd_stream_t stream);

/*
 * The conventional least-squares misfit the paper compares the EMD with (Sec. 2.1:
 * f_L2 = 1/2 integral (Pcal - Pobs)^2 dx dt) and its adjoint source (Sec. 2.3:
 * d f_L2 / d Pcal = Pcal - Pobs), discretised with the cell area A = dx*dt (dt when
 * nr == 1): value (HOST, nullable) = A/2 * sum (Pcal - Pobs)^2, summed in FP64;
 * grad_pred (device [nr][nt], nullable) = A (Pcal - Pobs); grad_obs (nullable) its
 * negative.  Differences are taken in FP32.  Needs 256 bytes of workspace (any
 * emd_workspace_size buffer will do).  Synchronises `stream` when value != NULL.
 */
emd_status emd_lsd(const float *f_obs, const float *f_pred, int nt, int nr, double dt, double dx,
                   double *value, float *grad_pred, float *grad_obs, void *workspace,
                   size_t ws_bytes, emd_stream_t stream);

/* Static, human-readable name of a status code. */
const char *emd_status_string(emd_status s);

#ifdef __cplusplus
}
#endif

#endif /* EMD_GB300_H */
