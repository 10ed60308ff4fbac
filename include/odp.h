/*
 * odp.h -- C ABI of libodp, the GB300 (sm_103a) solver for the time-dependent
 * Hamilton-Jacobi level-set update of OptimizedDP (arXiv 2204.05520).
 *
 * What it computes (paper, Section 2.1, Algorithm 1): starting from a target
 * function l(z) sampled on a dense N-D grid, phi(z, 0) = l(z), the value
 * function is advanced in look-back time tau.  Each time step computes, at
 * every grid node, one-sided spatial derivatives p-, p+ (first-order upwind or
 * second-order ENO, Section 3.1.4), their mean pbar, the optimal control and
 * disturbance of the Hamiltonian and H = pbar . f(z, u*, d*), a
 * Lax-Friedrichs dissipation with per-dimension coefficients alpha taken as a
 * grid-wide maximum (Section 2.1, global-alpha approximation), a CFL-limited
 * step dt (Algorithm 1), a forward-Euler or TVD-RK2 update (Section 3.1.3) and,
 * for a backward reachable tube, the min with l (the HJ variational
 * inequality of Section 2.1, method "minVWithV0" of Section 4.3).
 *
 * Conventions for every function:
 *  - Return value: an odp_status, ODP_OK (0) on success, a negative code
 *    otherwise.  No C++ exception crosses the ABI.  odp_last_error() returns a
 *    message for the calling thread's last failure.
 *  - Grids are dense C-order arrays (last dimension fastest, as NumPy lays
 *    them out; paper Section 5.2), float32 values, at most ODP_MAX_DIMS
 *    dimensions and fewer than 2^31 nodes.
 *  - Node i of an axis sits at lo + i*h, h = (hi - lo)/(n - 1) on a
 *    non-periodic axis and (hi - lo)/n on a periodic one (Section 3.1.1).
 *    Ghost nodes outside a non-periodic axis are extrapolated so that they
 *    keep the sign of the boundary node:  g_k = phi_b + k*sign(phi_b)*
 *    |phi_b - phi_inner| for the k-th ghost, sign(0) = +1.
 *  - Work is asynchronous on the CUDA stream given to odp_grid_create
 *    (a cudaStream_t passed as void*, NULL = the legacy default stream).
 *    Functions that return data to the host or report device-side errors
 *    synchronise that stream; each says so.
 *  - Pointers marked "device" are CUDA device pointers (for example a torch
 *    tensor's data_ptr()); "host" pointers may be pageable or pinned.  The
 *    library copies what it is given and never keeps a caller pointer.
 *  - A grid object is not thread-safe: calls on one grid must not overlap.
 */
#ifndef ODP_H
#define ODP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ODP_MAX_DIMS 6

typedef int odp_status;
#define ODP_OK 0
#define ODP_EINVAL (-1)   /* invalid argument (sizes, ranges, NULL pointers)        */
#define ODP_ENOMEM (-2)   /* device allocation failed or a memory budget is exceeded */
#define ODP_ECUDA (-3)    /* a CUDA runtime call failed (message in odp_last_error)  */
#define ODP_ESTATE (-4)   /* call out of order: dynamics or target missing, no solve */
#define ODP_ETIMEOUT (-5) /* the solve reached its step limit before the horizon     */
#define ODP_ENUMERIC (-6) /* a non-finite value appeared in the value function       */
#define ODP_EBUSY (-7)    /* the object is in use                                   */

typedef struct odp_grid odp_grid;

/* Closed set of hand-coded dynamics (paper Section 4.2 plug-ins, Appendix).
 * params per model, all bounds >= 0:
 *  ODP_DYN_SINGLE_INT  any ndim: z' = u, |u_i| <= params[0]
 *  ODP_DYN_DUBINS3D    z = (x, y, th): x' = v cos th, y' = v sin th, th' = w,
 *                      |w| <= w_max; params (v, w_max)            (Appendix, 3D Dubins)
 *  ODP_DYN_DUBINSCAR4D z = (x, y, v, th): x' = v cos th, y' = v sin th, v' = a,
 *                      th' = w; params (a_max, w_max)             (Appendix, 4D Dubins)
 *  ODP_DYN_REL6D       z = (x, y, th, v_p, w_p, v_e): relative pursuit-evasion
 *                      x' = -v_p + v_e cos th + w_p y, y' = v_e sin th - w_p x,
 *                      th' = w_e - w_p, v_p' = a_p, w_p' = alpha_p, v_e' = a_e;
 *                      control (a_p, alpha_p), disturbance (a_e, w_e);
 *                      params (a_p max, alpha_p max, a_e max, w_e max)
 *                      (the 3D pursuit-evasion model of Section 4.2 extended
 *                      with speed and turn-rate states as in the 5D Dubins car)
 *  ODP_DYN_ADVECTION   any ndim: z' = c, params c_0 .. c_{ndim-1} (no inputs)
 *  ODP_DYN_DUBINS_CAPTURE z = (x, y, th): pursuit-evasion of two Dubins cars in
 *                      relative coordinates (Section 4.2): x' = -v + v cos th + a y,
 *                      y' = v sin th - a x, th' = b - a; control a (evader turn,
 *                      |a| <= A), disturbance b (pursuer turn, |b| <= B);
 *                      params (v, A, B); every alpha component is reduced per
 *                      stage (interval bounds of the coupled switching
 *                      function y p_x - x p_y - p_th over each node's box)
 * Angles (th) must lie on a periodic axis. */
typedef enum {
    ODP_DYN_SINGLE_INT = 0,
    ODP_DYN_DUBINS3D = 1,
    ODP_DYN_DUBINSCAR4D = 2,
    ODP_DYN_REL6D = 3,
    ODP_DYN_ADVECTION = 4,
    ODP_DYN_DUBINS_CAPTURE = 5
} odp_dyn;

/* Role of an input in the Hamiltonian (Algorithm 1, optimal control and
 * disturbance step; Section 4.2 uMode/dMode).  ODP_MAX takes +bound when its
 * switching function is >= 0, ODP_MIN takes -bound when it is >= 0. */
typedef enum { ODP_MIN = 0, ODP_MAX = 1 } odp_mode;

/* Backward reachable set (plain PDE, method "None") or tube (phi <- min(phi,
 * l) after every full step, method "minVWithV0"); Section 4.3. */
typedef enum { ODP_BRS = 0, ODP_BRT = 1 } odp_set;

typedef struct {
    int64_t steps;     /* full time steps over all tau segments                 */
    double last_dt;    /* dt of the last step                                   */
    double t_final;    /* look-back time reached (tau[n_tau-1] on success)      */
    float alpha[8];    /* dissipation coefficients alpha_d of the last stage    */
    double device_ms;  /* device time of the time loop (CUDA events)            */
    double bytes;      /* algorithmic HBM bytes of the time loop                */
    int64_t launches;  /* kernels launched by the time loop                     */
} odp_solve_stats;

/* Message describing the calling thread's last failure ("" if none). */
const char *odp_last_error(void);

/* Library version string. */
const char *odp_version(void);

/* Create a grid (Section 3.1.1).  n, lo, hi, periodic: ndim entries each
 * (host).  n[d] >= 2 on a non-periodic axis, >= 1 on a periodic one;
 * hi[d] > lo[d].  cuda_stream: the stream all work on this grid is issued on.
 * Allocates the value buffers on the current device.  *out receives the
 * grid; release it with odp_grid_destroy.
 * Errors: ODP_EINVAL, ODP_ENOMEM, ODP_ECUDA. */
odp_status odp_grid_create(int ndim, const int32_t *n, const double *lo, const double *hi,
                           const uint8_t *periodic, void *cuda_stream, odp_grid **out);

/* Launch geometry the library would use for a grid of this shape (host only,
 * no CUDA call; no paper counterpart).  out[0..13] = padded last axis, rows
 * per thread of the row-blocked pass, its row groups, its planes, its threads,
 * plane-streaming pass used (0/1), stream-axis length, stream-axis chunk per
 * CTA, CTAs, threads per CTA, shared bytes for stencil radius 1 and 2, rows
 * per band, bands.  n_out >= 14.
 * Errors: ODP_EINVAL. */
odp_status odp_plan_geometry(int ndim, const int32_t *n, int64_t *out, int n_out);

/* Free a grid and all device memory it owns (synchronises its stream).
 * NULL is accepted. */
odp_status odp_grid_destroy(odp_grid *g);

/* Number of nodes of a grid (product of n). */
int64_t odp_grid_points(const odp_grid *g);

/* Choose the dynamics (Section 4.2 plug-ins, Appendix models; see odp_dyn).
 * params: n_params doubles (host), copied.  u_mode / d_mode: roles of the
 * control and the disturbance.  On the grid's device the call also sizes the
 * launches of the stage kernels for this model (it queries their occupancy;
 * no allocation).  Errors: ODP_EINVAL (unknown model, wrong dimension count,
 * missing parameters, negative bound, angle axis not periodic), ODP_ECUDA (a
 * failed CUDA query). */
odp_status odp_set_dynamics(odp_grid *g, odp_dyn kind, const double *params, int n_params,
                            odp_mode u_mode, odp_mode d_mode);

/* Set the target function l(z) (initial value phi(z, 0) = l(z); Section 2.1),
 * n_elems = odp_grid_points(g) float32 values in C order.  on_device: 1 if l
 * is a device pointer, 0 for host memory.  The values are copied
 * (asynchronously for device and pinned host memory).  Errors: ODP_EINVAL. */
odp_status odp_set_target(odp_grid *g, const float *l, int64_t n_elems, int on_device);

/* Reach-avoid obstacle (Section 4.3, the target and obstacle computation
 * methods): g(z) at every node in C order, positive inside the obstacle.
 * After each full time step of later solves phi <- max(phi, g), taken after
 * the tube's min with l.  g is copied like the target (on_device as there);
 * g == NULL removes the obstacle.  Grids with an obstacle are refused by
 * odp_batch_solve.  Errors: ODP_EINVAL, ODP_ENOMEM. */
odp_status odp_set_obstacle(odp_grid *g, const float *gv, int64_t n_elems, int on_device);

/* Time-varying target (Section 2.1's time-varying variants; the target and
 * obstacle computation methods of Section 4.3): n_sets = n_tau arrays of
 * n_elems = odp_grid_points(g) floats, l_seq[k] the target at tau[k], dense C
 * order one after the other (on_device as for odp_set_target).  A solve then
 * starts from l_seq[0] and every step of segment (tau[k], tau[k+1]] takes its
 * BRT min with l_seq[k+1], the set at the end of the segment it lands in.
 * The schedule replaces the grid's target (odp_set_target replaces the
 * schedule again); l_seq == NULL removes it.  Solves whose n_tau differs from
 * n_sets are refused, and so are batched solves and the time-to-reach sweep
 * on a grid with a schedule.  Errors: ODP_EINVAL, ODP_ENOMEM, ODP_ECUDA. */
odp_status odp_set_target_schedule(odp_grid *g, const float *l_seq, int n_sets, int64_t n_elems, int on_device);

/* Time-varying obstacle: as odp_set_target_schedule, g_seq[k] the obstacle
 * at tau[k]; the steps of segment (tau[k], tau[k+1]] take their max with
 * g_seq[k+1].  It replaces the grid's obstacle (odp_set_obstacle replaces it
 * again); g_seq == NULL removes the obstacle.  Errors: as above. */
odp_status odp_set_obstacle_schedule(odp_grid *g, const float *g_seq, int n_sets, int64_t n_elems, int on_device);

/* Lax-Friedrichs dissipation of later solves (no change to the CFL step):
 * per_node = 0 (default) uses the grid alpha, the largest rate over the grid
 * per component (Section 2.1); per_node = 1 uses each node's own alpha_i, the
 * largest rate over the input extremes its derivative box admits (Algorithm
 * 1's second loop).  Per-node solves run the generic stage kernels; for the
 * capture model, whose bounds come from interval arithmetic over the box,
 * the per-stage alpha pass writes each node's coefficients to a buffer of 12
 * bytes per node that the solve allocates on first use.  Grids with
 * per_node = 1 are refused by odp_batch_solve.  Errors: ODP_EINVAL. */
odp_status odp_set_dissipation(odp_grid *g, int per_node);

/* Limit the number of full time steps of one solve (default 10,000,000).  A
 * solve that reaches the limit stops and reports ODP_ETIMEOUT. */
odp_status odp_set_step_limit(odp_grid *g, int64_t max_steps);

/* Choose how odp_solve_hjb runs the time loop (no paper counterpart):
 * host_stepped = 0 (default) launches one CUDA graph whose device-side WHILE
 * node runs every step; host_stepped = 1 launches the same kernels, in the
 * same order, one step at a time from the host and reads the loop condition
 * back after each step (one synchronisation per step).  Results are
 * identical; the host-stepped loop exists for profilers and debuggers that do
 * not follow kernels inside conditional graph nodes.  Errors: ODP_EINVAL. */
odp_status odp_set_loop_mode(odp_grid *g, int host_stepped);

/* Choose the kernel that runs the stage pass of Algorithm 1 (derivatives,
 * Hamiltonian, Lax-Friedrichs update and set operations) for grids of 3 or
 * more dimensions; no paper counterpart, both compute the same per-node
 * arithmetic, so results are identical.  The bulk-staged pass (Dubins3D,
 * DubinsCar4D and Rel6D grids whose last axis is a multiple of 4 nodes, with
 * grid-wide dissipation) has a producer thread per CTA stage every neighbour
 * tile with bulk async copies into shared-memory rings; the plane-streaming
 * pass has the compute threads load their own neighbours.  pass = 0
 * (default) picks the one that measured faster (bulk-staged on grids of 4 or
 * more dimensions, plane-streaming on 3-D grids); pass = 1 forces the
 * plane-streaming pass; pass = 2 the bulk-staged pass.  The choice holds for later solves of the grid; batched
 * and served solves always use the plane-streaming pass.  Errors: ODP_EINVAL
 * (pass out of range, or 2 on a grid whose shape the bulk-staged pass does
 * not take: last axis not a multiple of 4, fewer than 4 rows or stream
 * planes, or rings beyond 200 KB of shared memory). */
odp_status odp_set_stage_pass(odp_grid *g, int pass);

/* Solve the HJ PDE (Algorithm 1) from tau[0] = 0 to tau[n_tau-1].
 *  tau          n_tau >= 2 strictly increasing look-back times (host), tau[0] = 0;
 *               each segment is integrated separately, the last CFL step of a
 *               segment clipped to its end (HJSolver's tau schedule, Section 4.3)
 *  set          ODP_BRS or ODP_BRT
 *  space_order  1 (upwind) or 2 (ENO2)
 *  time_order   1 (forward Euler) or 2 (TVD-RK2)
 *  cfl          (0, 1]: dt = cfl / sum_d(alpha_d / h_d)
 *  keep_snapshots  1 keeps phi at every tau (readable with odp_value_readback)
 *  stats        NULL: the solve is only enqueued and returns at once; device-side
 *               errors then surface in odp_value_readback or odp_solve_status.
 *               Non-NULL: the call synchronises the stream and fills *stats.
 * The whole time loop runs as one CUDA graph with a device-side while loop;
 * dt and t are kept in float64 on the device.
 * Errors: ODP_ESTATE (no dynamics or target), ODP_EINVAL, ODP_ENOMEM,
 * ODP_ECUDA, and with stats != NULL also ODP_ETIMEOUT, ODP_ENUMERIC. */
odp_status odp_solve_hjb(odp_grid *g, const double *tau, int n_tau, odp_set set,
                         int space_order, int time_order, double cfl, int keep_snapshots,
                         odp_solve_stats *stats);

/* Wait for the grid's last solve and return its device-side status
 * (ODP_OK, ODP_ETIMEOUT or ODP_ENUMERIC); synchronises the stream.  Fills
 * *stats when non-NULL (device_ms and bytes only if the solve was timed). */
odp_status odp_solve_status(odp_grid *g, odp_solve_stats *stats);

/* Copy the value function out: tau_index -1 (or n_tau-1) = the final value,
 * 0..n_tau-2 need keep_snapshots.  dst: n_elems = odp_grid_points(g) floats,
 * device memory if on_device else host memory.  Synchronises the stream and
 * reports the solve's device-side status (ODP_ETIMEOUT, ODP_ENUMERIC).
 * Errors: ODP_ESTATE (no solve yet), ODP_EINVAL, ODP_ECUDA. */
odp_status odp_value_readback(odp_grid *g, int tau_index, float *dst, int64_t n_elems,
                              int on_device);

/* ------------------------------------------------------------------------
 * Batched solves (no paper counterpart: many independent Algorithm 1 solves
 * advanced together).
 * ------------------------------------------------------------------------ */
typedef struct {
    double device_ms;      /* device time of the batch's launches             */
    int64_t rounds;        /* lockstep rounds (the largest step count)        */
    int32_t ctas_per_sm;   /* launch shape chosen by the autotuner (0: the
                              plane-streaming rounds, occupancy by hardware)  */
    int32_t rows_per_thread;
    double point_updates;  /* sum over grids of nodes x steps                  */
    double bytes;          /* algorithmic HBM bytes                            */
    int32_t plane_chunk;   /* plane path: stream planes per CTA, chosen by the
                              autotuner (0: row-blocked path)                 */
    int32_t graph;         /* plane path: 1 the batch graph was captured by
                              this call, 2 a cached graph was replayed        */
    int64_t launches;      /* plane path: kernel launches in the batch graph   */
    int32_t tuned;         /* 1: this call ran the autotuner                   */
    int32_t reserved;
} odp_batch_stats;

/* Solve n independent grids over [0, T[i]] together.  Every grid must have
 * its dynamics and target set and live on the same device; work is issued on
 * grids[0]'s stream and the call synchronises it.  Each grid takes exactly
 * the step sequence of a single odp_solve_hjb over tau = {0, T[i]} (same
 * float64 step schedule, same per-node kernel arithmetic) and its final value
 * is read back with odp_value_readback(g, -1).  When every grid is a Dubins3D
 * or DubinsCar4D grid that the plane-streaming pass takes, each round (step
 * index) and RK phase is one launch over every grid still running, all of
 * them one CUDA graph captured once per batch signature (model, orders,
 * grid count, rounds, launch shapes) and replayed by later calls; the
 * stream-chunk cap of the plane items (8, 16, 32 or 64 planes per CTA) is
 * autotuned on the first rounds and cached per signature; other
 * batches run one persistent cooperative launch of the row-blocked pass, its
 * shape (CTAs per SM) autotuned on the first rounds and cached per batch
 * signature.  Supported models: Dubins3D, DubinsCar4D, and the 2-3D single
 * integrator (Rel6D needs a per-stage alpha pass and is refused; so are grids
 * with an obstacle or per-node dissipation).  stats may be NULL.
 * Errors: ODP_EINVAL, ODP_ESTATE, ODP_ENOMEM, ODP_ECUDA. */
odp_status odp_batch_solve(odp_grid *const *grids, int n, const double *T, odp_set set, int space_order,
                           int time_order, double cfl, odp_batch_stats *stats);

/* Turn the batched solve's autotuner on (1, default) or off (0: the
 * occupancy limit is used). */
odp_status odp_batch_set_autotune(int enabled);

/* ------------------------------------------------------------------------
 * Serving loop (no paper counterpart): continuous batching of solves under an
 * HBM budget.
 * ------------------------------------------------------------------------ */
typedef struct odp_server odp_server;

/* One solve request: a grid, a model, a target and a horizon T
 * (tau = {0, T}).  The server runs Dubins3D (3-D) and DubinsCar4D (4-D)
 * requests whose second-last axis has at least 4 nodes and whose angle axis
 * (the last one) is periodic. */
typedef struct {
    int32_t ndim;
    int32_t n[ODP_MAX_DIMS];
    double lo[ODP_MAX_DIMS];
    double hi[ODP_MAX_DIMS];
    uint8_t periodic[ODP_MAX_DIMS];
    odp_dyn kind;
    int32_t n_params;
    double params[8];
    odp_mode u_mode, d_mode;
    const float *target;      /* host, C order; copied by odp_server_submit */
    double T;
    odp_set set;
    int32_t space_order, time_order;
    double cfl;
} odp_request;

#define ODP_REQ_QUEUED 0      /* waiting for HBM                            */
#define ODP_REQ_RESIDENT 1    /* admitted, advancing with the batch         */
#define ODP_REQ_DONE 2        /* horizon reached; value resident in HBM     */
#define ODP_REQ_FAILED 3      /* a non-finite value appeared                */

typedef struct {
    int32_t state;            /* ODP_REQ_*                                   */
    int32_t reserved;
    int64_t steps;            /* time steps of the solve (known once admitted) */
    int64_t steps_done;
    double queue_s;           /* submit -> admission                         */
    double latency_s;         /* submit -> done                              */
    double t_submit, t_done;  /* host monotonic clock, seconds               */
    double bytes;             /* HBM held by the request                     */
} odp_request_stats;

typedef struct {
    double budget_bytes, used_bytes;
    int64_t queued, resident, launches;
} odp_server_stats;

/* Create a server whose resident solves may hold hbm_budget_bytes of device
 * memory (allocated once, here, as one arena).  Work runs on cuda_stream.
 * Errors: ODP_EINVAL, ODP_ENOMEM, ODP_ECUDA. */
odp_status odp_server_create(size_t hbm_budget_bytes, void *cuda_stream, odp_server **out);

/* Free the server and every request's memory (synchronises its stream). */
odp_status odp_server_destroy(odp_server *s);

/* Queue a request (the target is copied; the call returns at once).
 * Errors: ODP_EINVAL (unsupported model or shape), ODP_ENOMEM (the request
 * alone exceeds the budget). */
odp_status odp_server_submit(odp_server *s, const odp_request *req, uint64_t *req_id);

/* Cap the work in flight: admission stops while the resident (admitted,
 * unfinished) solves hold max_nodes grid nodes or more, and a request that
 * would take them past the cap waits (unless nothing is resident).
 * max_nodes = 0 (the default) admits whatever fits the HBM budget.  Above
 * saturation a cap keeps queued requests waiting in arrival order instead of
 * slowing every resident solve.  Errors: ODP_EINVAL (negative cap). */
odp_status odp_server_set_max_resident(odp_server *s, int64_t max_nodes);

/* One scheduling step: admit queued requests in arrival order while their
 * arrays fit the budget (and the resident-node cap), advance every resident
 * solve by up to `rounds` of its own time steps (one plane-streaming launch
 * per round and class of solves, or one persistent launch of the row-blocked
 * pass when a resident grid cannot take the plane pass), retire the solves
 * that reached their horizon (their values stay in HBM).  *n_done (may be
 * NULL) counts the requests finished by this step.  Synchronises the stream.
 * Errors: ODP_EINVAL, ODP_ECUDA. */
odp_status odp_server_step(odp_server *s, int rounds, int *n_done);

/* State and timings of a request.  Returns ODP_ENUMERIC for a failed one. */
odp_status odp_server_poll(odp_server *s, uint64_t req_id, odp_request_stats *out);

/* Copy a finished request's value (odp C order, n_elems floats) to host or
 * device memory.  Errors: ODP_ESTATE (not done), ODP_EINVAL. */
odp_status odp_server_readback(odp_server *s, uint64_t req_id, float *dst, int64_t n_elems, int on_device);

/* Forget a request and return its HBM to the budget (ODP_EBUSY while it is
 * resident and unfinished). */
odp_status odp_server_release(odp_server *s, uint64_t req_id);

/* Budget, memory in use, queue and resident counts, launches so far. */
odp_status odp_server_info(odp_server *s, odp_server_stats *out);

/* Allocation-free single solve.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a solve -- code running inside a memory pool or arena it does not own (a
 * framework's caching allocator, a serving process that partitioned its HBM
 * up front) or code that must not call cudaMalloc/cudaFree because those
 * calls synchronise the device.  It solves one grid over tau = {0, T} exactly
 * as odp_grid_create + odp_set_dynamics + odp_set_target + odp_solve_hjb +
 * odp_value_readback would (same step schedule, same kernel arithmetic), but
 * calls no allocating routine: everything besides the caller's buffers lives
 * in one file-scope device array of 16 MiB that every GPU loading the library
 * holds until the process exits.
 *  l, out       device pointers, odp_grid_points floats each, dense C order
 *               (l: the target; out: the final value); the caller owns both
 *  other args   as odp_grid_create / odp_set_dynamics / odp_solve_hjb; models:
 *               Dubins3D, DubinsCar4D, 2-3D single integrator
 *  cuda_stream  stream the work runs on (NULL: legacy default stream); the
 *               call synchronises it before returning
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  The call copies its small records
 * from host memory and synchronises its stream before returning, so it
 * cannot be recorded into a CUDA graph: on a capturing stream it returns
 * ODP_EINVAL.  All calls share the array and it keeps the last call's
 * contents: each call clears what must start at zero.  Calls whose GPU work
 * overlapped would race on the array; the library prevents that within a
 * process by holding a per-device lock for the whole call (calls on one
 * device run one after another; calls on different devices do not wait for
 * each other).  The caller's current device is restored before returning.
 * Errors: ODP_EINVAL (arguments, a capturing stream, or a grid needing more
 * than the array holds: about 1.3 million nodes), ODP_ENUMERIC, ODP_ECUDA. */
odp_status odp_solve_noalloc(int ndim, const int32_t *n, const double *lo, const double *hi,
                             const uint8_t *periodic, odp_dyn kind, const double *params, int n_params,
                             odp_mode u_mode, odp_mode d_mode, const float *l, double T, odp_set set,
                             int space_order, int time_order, double cfl, float *out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Time-to-reach function (Section 2.2, Algorithm 2): the static HJ equation
 * -min_u max_d grad(phi) . f(z, u, d) = 1 outside the target set {l <= 0},
 * phi = 0 on it, solved by Lax-Friedrichs sweeping.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t sweeps;       /* sweeps taken                                        */
    double change;        /* largest |phi - phi_old| of the last sweep            */
    double device_ms;     /* device time of the sweep loop (CUDA events)          */
    double bytes;         /* algorithmic HBM bytes: one read and one write of
                             every node per sweep                                */
    int64_t launches;     /* kernels launched by the sweep loop                   */
    int64_t tile_planes;  /* tile hyperplanes (launches of the interior pass) per
                             sweep                                               */
} odp_ttr_stats;

/* Time-to-reach function of the grid's dynamics and target (Algorithm 2).
 * phi starts at 0 on the target nodes (l <= 0, decided in float32 on the
 * values given to odp_set_target) and at `big` elsewhere (the paper uses a
 * large value such as 10000 for infinity).  Each sweep visits the interior
 * nodes (those not first or last on a non-periodic axis) in the nested C-order
 * loops of Algorithm 2, axis d descending when bit d of the sweep index mod
 * 2^ndim is set (alternating directions, Section 5.3), and updates in place
 *   phi_i <- min(phi_i, (1 + pbar . f(z, u*, d*)
 *                        + sum_d sigma_d (phi(i+e_d) + phi(i-e_d)) / (2 h_d))
 *                       / sum_d(sigma_d / h_d))
 * with pbar the central difference of the current values, u* minimising and
 * d* maximising pbar . f, sigma_d = |f_d(z, u*, d*)| (a node with
 * sum_d sigma_d / h_d = 0 keeps its value).  The library evaluates the
 * equal form (1 + sum_d w_d phi(i + sign(f_d) e_d)) / sum_d w_d, w_d =
 * |f_d| / h_d (the smaller neighbour on an input axis), which has no
 * cancellation in float32.  Then each non-periodic axis in
 * turn sets its first and last nodes to min(max(2 phi_1 - phi_2, phi_2),
 * phi_b) along that axis.  Sweeps repeat while max|phi - phi_old| > eps, at
 * most max_sweeps times.  The GPU visits the nodes hyperplane by hyperplane,
 * which gives every node the same neighbour values as the sequential order.
 * The result is the grid's value: read it with odp_value_readback(g, -1, ...).
 * Models: single integrator (1-4 dimensions), Dubins3D, DubinsCar4D, with
 * u_mode ODP_MIN and d_mode ODP_MAX; every axis needs at least 4 nodes.
 * The loop runs as one CUDA graph with a device-side while node
 * (odp_set_loop_mode(g, 1): one sweep at a time from the host).
 * stats: NULL enqueues the work and returns; non-NULL synchronises the stream
 * and fills *stats.
 * Errors: ODP_ESTATE (no dynamics or target), ODP_EINVAL (model, modes,
 * dimensions, eps < 0, big not a positive finite float, max_sweeps < 1),
 * ODP_ENOMEM, ODP_ECUDA; with stats != NULL also ODP_ETIMEOUT (max_sweeps
 * reached first) and ODP_ENUMERIC. */
odp_status odp_solve_ttr(odp_grid *g, double eps, double big, int64_t max_sweeps, odp_ttr_stats *stats);

/* Measurement helper (no paper counterpart): launch the fused stage kernel of
 * the grid's last solve `reps` times on its stream, outside the graph, and
 * return the mean device time of one launch in *ms_out (CUDA events; the call
 * synchronises).  stage: 0 = Euler, 1 = RK2 stage 1, 2 = RK2 stage 2 (must
 * match the last solve's time order).  The launches overwrite the value
 * buffers: solve again before reading values back.
 * Errors: ODP_ESTATE (no solve yet), ODP_EINVAL, ODP_ECUDA. */
odp_status odp_time_stage(odp_grid *g, int stage, int reps, double *ms_out);

#ifdef __cplusplus
}
#endif

#endif /* ODP_H */
