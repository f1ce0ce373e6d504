/*
 * cgks.h -- C ABI of libcgks: the GB300 (sm_103a) implementation of the
 * p-multigrid compact gas-kinetic scheme of Ji, Shyy & Xu,
 * "A p-multigrid compact gas-kinetic scheme for steady-state acceleration"
 * (arXiv:2109.09965), for 2-D hybrid (triangle / quadrilateral) meshes.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns CGKS_OK (0) or a negative CGKS_E* status.
 *    cgks_strerror() names a status.  Nothing aborts the process.
 *  - Host arrays are owned by the caller and only read or written during
 *    the call; the library copies what it keeps.  Device memory is owned
 *    by the library (allocated through the optional allocator callback of
 *    cgks_params, else cudaMalloc) and released by *_destroy.
 *  - State arrays at the ABI are in the caller's cell order, array of
 *    structs: W[c*4 + v] with v = (rho, rho*u, rho*v, rho*E) and
 *    Wx[(c*2 + d)*4 + v] = cell-averaged d(W_v)/dx_d.  Internally the
 *    library stores structure-of-arrays in its own cell order (reverse
 *    Cuthill-McKee within graph colours, see cgks_mesh_ordering).
 *  - All device work runs on the stream given in cgks_params (NULL = the
 *    legacy default stream).  Calls that return host results synchronise
 *    that stream.  A solver is not thread safe; use one per host thread.
 *  - A device-side status word records non-finite or non-positive
 *    density / pressure; once set, stepping calls return CGKS_EDIVERGED
 *    until cgks_set_state() loads a new state.
 *  - There is no CPU fallback: without a usable CUDA device the solver
 *    constructor returns CGKS_ECUDA.
 */
#ifndef CGKS_H
#define CGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CGKS_OK = 0,
  CGKS_EINVAL = -1,     /* bad argument (NULL pointer, size, parameter) */
  CGKS_ENOMEM = -2,     /* host or device allocation failed */
  CGKS_EMESH = -3,      /* mesh rejected at creation */
  CGKS_ECUDA = -4,      /* CUDA runtime error or no device */
  CGKS_EDIVERGED = -5,  /* non-finite or non-positive rho / p on the device */
  CGKS_ETIMEOUT = -6,   /* a bounded wait expired */
  CGKS_EBUDGET = -7     /* request does not fit the memory budget */
};

/* cell types (node order counter-clockwise, as VTK) */
/* cell types: 2-D triangle / quadrilateral; 3-D tetrahedron, prism,
 * pyramid, hexahedron.  Node order: 2-D counter-clockwise; 3-D "positive"
 * (the first face counter-clockwise seen from the rest of the cell):
 *   tet 0 1 2 | 3;  prism 0 1 2 | 3 4 5 (node k+3 above node k);
 *   pyramid 0 1 2 3 | 4;  hex 0 1 2 3 | 4 5 6 7 (node k+4 above node k). */
enum { CGKS_TRI = 0, CGKS_QUAD = 1, CGKS_TET = 2, CGKS_PRISM = 3, CGKS_PYRAMID = 4, CGKS_HEX = 5 };

/* boundary conditions, Section 4 of the paper: reflective (slip) wall,
 * non-slip adiabatic wall (optionally moving tangentially), far field with
 * 1-D Riemann invariants against a free stream, Dirichlet (the given state,
 * uniform outside) and supersonic outflow (the inside continued: state and
 * gradient copied), the last two for the shock reflection problem (2-D
 * only).  Only walls enter the reconstruction stencils. */
enum { CGKS_BC_SLIP = 0, CGKS_BC_NOSLIP = 1, CGKS_BC_FARFIELD = 2, CGKS_BC_DIRICHLET = 3, CGKS_BC_OUTFLOW = 4 };

/* explicit time schemes: S1O2 (Section 2.4) and the two-stage fourth-order
 * S2O4 named in Section 1 (Li & Du 2016) */
enum { CGKS_S1O2 = 0, CGKS_S2O4 = 1 };

/* arithmetic of the hot path */
enum { CGKS_FP64 = 0, CGKS_MIXED = 1 };

/* First-order flux of the low-order level (Section 3: KFVS by default; the
 * paper also runs a Lax-Friedrichs solver there and finds the convergence
 * nearly unchanged).  L-F: (F_n(U_l) + F_n(U_r)) / 2 - lambda_p (U_r - U_l) / 2
 * with lambda_p the spectral radius of the implicit operator, max of the
 * two sides. */
enum { CGKS_FLUX_KFVS = 0, CGKS_FLUX_LF = 1 };

/* Order of the point relaxation (Algorithm 1), 2-D.
 *   COLOUR:      colour classes over the whole mesh, colours ascending then
 *                descending in every sweep (the index order of Algorithm 1
 *                replaced by a distance-1 colouring; default).
 *   PARTITIONED: the paper's threaded sweep (Section 3 and the parallel
 *                cylinder runs of Section 4), made deterministic: the
 *                reverse Cuthill-McKee order of each mesh is cut into
 *                P = ceil(n_cells / sweep_part_cells) partitions (the cell
 *                at RCM position k is in partition floor(k P / n_cells));
 *                within a partition the colour classes relax in order,
 *                and a neighbour in another partition is read as it was at
 *                the start of the sweep (forward and backward pass
 *                together).  One launch per sweep, one thread-block
 *                cluster per partition. */
enum { CGKS_SWEEP_COLOUR = 0, CGKS_SWEEP_PARTITIONED = 1 };

/* Gas-kinetic flux of the high-order level (Section 2.3; Section 4 uses the
 * smooth one for subsonic flow, the full one with WENO weights for
 * transonic and supersonic flow).
 *   SMOOTH: Eq. (2nd-smooth-flux).
 *   FULL:   Eq. (2nd-flux), with numerical collision time
 *           tau_n = mu/p + tau_c1 dt + tau_c2 dt |p_l - p_r| / (p_l + p_r)
 *           in the exponentials; its time dependence enters the time
 *           schemes through the integrals over [0, dt] and [0, dt/2].
 * 3-D takes FULL and conservative WENO weights; characteristic WENO and the
 * Dirichlet / outflow boundaries are 2-D only. */
enum { CGKS_FLUX_SMOOTH = 0, CGKS_FLUX_FULL = 1 };

/* Variables the compact WENO weights act on (Section 4: conservative by
 * default, characteristic for the shock reflection problem).
 *   CONSERVATIVE:   per cell, per conservative component.
 *   CHARACTERISTIC: per face side, per characteristic field of the Euler
 *                   flux Jacobian along the face normal at the mean of the
 *                   two cell averages. */
enum { CGKS_WENO_CONSERVATIVE = 0, CGKS_WENO_CHARACTERISTIC = 1 };

#define CGKS_MAX_BC 16

typedef struct {
  int32_t kind;          /* CGKS_BC_* */
  int32_t pad_;
  double u_wall[3];      /* no-slip wall velocity (tangential; 2-D uses x, y) */
  double rho, u[3], p;   /* far-field free stream or Dirichlet state (primitive variables; 2-D uses x, y) */
} cgks_bc;

typedef void *(*cgks_alloc_fn)(size_t bytes, void *ctx);
typedef void (*cgks_free_fn)(void *ptr, void *ctx);

typedef struct {
  double gamma;          /* ratio of specific heats (1.4) */
  double mu;             /* constant dynamic viscosity; 0 = Euler */
  double alpha;          /* jump coefficient of the equilibrium normal slope (1/2) */
  double cfl_hi;         /* explicit CFL of the high-order level (0.3-0.5, Section 4) */
  double cfl_lo;         /* local CFL of the low-order level (1000, Section 4) */
  int32_t n_implicit;    /* backward-Euler steps per V-cycle (6, Section 3) */
  int32_t n_sweeps;      /* forward+backward relaxation pairs per step (2) */
  int32_t time_scheme;   /* CGKS_S1O2 or CGKS_S2O4 */
  int32_t precision;     /* CGKS_FP64 or CGKS_MIXED */
  int32_t n_bc;          /* entries used in bc[] (boundary tags index it) */
  int32_t use_graph;     /* 1: capture each V-cycle in a CUDA graph */
  int32_t low_order_fused; /* 1: the low-order level as one persistent cooperative launch (2-D);
                            0 (default): one graph-replayed kernel per phase, faster on GB300 */
  int32_t autotune;      /* 1 (default): the block-size autotuner picks the launch shapes (see
                            cgks_get_tuning); 0: the fixed default shapes */
  int32_t programmatic_launch; /* 1 (default): each kernel of a cycle may be scheduled while its
                            predecessor runs and waits on the device for it (programmatic
                            dependent launch, sm_90+); 0: plain stream order.  Same results. */
  int32_t flux_lo;       /* CGKS_FLUX_KFVS (default) or CGKS_FLUX_LF */
  int32_t flux_hi;       /* CGKS_FLUX_SMOOTH (default) or CGKS_FLUX_FULL */
  int32_t weno_vars;     /* CGKS_WENO_CONSERVATIVE (default) or CGKS_WENO_CHARACTERISTIC */
  int32_t sweep_order;   /* CGKS_SWEEP_COLOUR (default) or CGKS_SWEEP_PARTITIONED (2-D only;
                            not with low_order_fused) */
  int32_t sweep_part_cells; /* cells per partition of the partitioned sweep, >= 64
                            (0: 2048; smaller partitions lag more couplings and
                            converge more slowly) */
  int32_t lo_viscous;    /* 1: the low-order residual carries a first-order viscous flux
                            (reading of Section 3's first-order finite volume scheme for
                            viscous flow): normal gradients from the two cell states over
                            their centre distance along the face normal, Stokes'
                            hypothesis, Pr = 1 heat flux.  Needed on wall cells thinner
                            than the viscous length mu / (rho c), where the inviscid
                            correction overshoots; 0 (default): inviscid KFVS / L-F.
                            Not with low_order_fused. */
  int32_t pad2_;
  double tau_c1, tau_c2; /* numerical collision time constants of the full flux (0.01, 1) */
  double weno_eps;       /* > 0: compact WENO nonlinear weights with this epsilon (Section 4 uses
                            1e-2 and 1e-6); 0 (default): linear weights */
  double weno_g0;        /* linear weight of the quadratic candidate of the WENO step (0.95) */
  cgks_bc bc[CGKS_MAX_BC];
  void *stream;          /* cudaStream_t for all device work (NULL = default) */
  cgks_alloc_fn alloc;   /* optional device allocator (NULL = cudaMalloc) */
  cgks_free_fn free;     /* matching free */
  void *alloc_ctx;       /* passed to alloc / free */
} cgks_params;

typedef struct {
  int64_t n_cells, n_faces, n_bfaces;
  int32_t n_colours;     /* colours of the sweep order */
  int32_t dim;
  int64_t device_bytes;  /* device memory a solver on this mesh holds */
} cgks_mesh_info_t;

typedef struct cgks_mesh cgks_mesh;
typedef struct cgks_solver cgks_solver;

/* Fill p with the defaults above (gamma 1.4, Euler, CFL 0.4 / 1000,
 * 6 implicit steps, 2 sweeps, S1O2, FP64, graphs on, autotune on,
 * programmatic launch on, per-phase low-order launches, no boundaries). */
void cgks_default_params(cgks_params *p);

/* Build a mesh from nodes, cells and tagged boundary faces (the finite-
 * volume setting of Section 2.1).
 *   dim           2 or 3
 *   xyz           [n_nodes*dim] node coordinates
 *   cell_type     [n_cells] CGKS_TRI / CGKS_QUAD (2-D), CGKS_TET /
 *                 CGKS_PRISM / CGKS_PYRAMID / CGKS_HEX (3-D)
 *   cell_ptr      [n_cells+1] offsets into cell_nodes
 *   cell_nodes    node indices in the order given with the cell types
 *   bface_ptr     [n_bfaces+1] offsets into bface_nodes (2 nodes per edge
 *                 in 2-D; 3 or 4 per face in 3-D, any order)
 *   bface_tag     [n_bfaces] index into cgks_params.bc[]
 * Builds faces, areas / volumes, centroids, Gauss quadrature per face (2
 * points per edge; 3 per triangle, 4 per quadrilateral in 3-D), the reverse
 * Cuthill-McKee order and the greedy colouring.  Returns CGKS_EMESH for
 * negatively ordered or degenerate cells, faces shared by more than two
 * cells, or boundary faces without a tag.  Host only.
 * State layouts at the ABI, caller cell order: W [n_cells][dim+2],
 * Wx [n_cells][dim][dim+2]. */
int cgks_mesh_create(int dim, int64_t n_nodes, const double *xyz, int64_t n_cells,
                     const uint8_t *cell_type, const int64_t *cell_ptr, const int64_t *cell_nodes,
                     int64_t n_bfaces, const int64_t *bface_ptr, const int64_t *bface_nodes,
                     const int32_t *bface_tag, cgks_mesh **out);

int cgks_mesh_info(const cgks_mesh *m, cgks_mesh_info_t *out);

/* Sweep order of the coloured point relaxation (the index order of
 * Algorithm 1 replaced by colour classes): rcm[k] = caller cell at position
 * k of the reverse Cuthill-McKee order, colour[c] = colour of caller cell c. */
int cgks_mesh_ordering(const cgks_mesh *m, int64_t *rcm, int32_t *colour);

int cgks_mesh_destroy(cgks_mesh *m);

/* Create a solver on a mesh: uploads geometry and operators to the device
 * and allocates the state.  The mesh may be destroyed afterwards. */
int cgks_solver_create(const cgks_mesh *m, const cgks_params *p, cgks_solver **out);
int cgks_solver_destroy(cgks_solver *s);

/* Load cell averages W and cell-averaged gradients Wx (NULL = zero) from
 * host memory (layouts above).  Clears the status word. */
int cgks_set_state(cgks_solver *s, const double *W, const double *Wx);
/* Same from device memory (same layouts, caller order). */
int cgks_set_state_device(cgks_solver *s, const double *W_dev, const double *Wx_dev);
/* Copy the state to host memory (either pointer may be NULL). */
int cgks_get_state(cgks_solver *s, double *W, double *Wx);
int cgks_get_state_device(cgks_solver *s, double *W_dev, double *Wx_dev);

/* One explicit high-order step (Sections 2.2-2.4): compact reconstruction,
 * gas-kinetic smooth flux and interface state at every Gauss point,
 * S1O2 or S2O4 update of W and Gauss-Green update of Wx.
 *   dt <= 0: global time step from cfl_hi.  *dt_used (may be NULL) gets it. */
int cgks_highorder_step(cgks_solver *s, double dt, double *dt_used);

/* n explicit high-order steps without host synchronisation in between;
 * res_hist (host, may be NULL) receives the density residual of each. */
int cgks_explicit_steps(cgks_solver *s, int n, double *res_hist);

/* Low-order level alone (Section 3, steps 3-5) on the current state, with
 * R_p0 of the last high-order evaluation: forcing, n_implicit backward-
 * Euler steps by coloured point relaxation, prolongation of the correction. */
int cgks_loworder_smooth(cgks_solver *s);

/* n two-level V-cycles (Section 3, steps 1-5): high-order step, residual
 * R_p0 re-evaluated at W^{n+1}, low-order implicit solve, correction.
 * res_hist (host, may be NULL) receives Res of each cycle. */
int cgks_pmg_cycle(cgks_solver *s, int n_cycles, double *res_hist);

/* Density residual Res = sum|rho^{n+1} - rho^n| / sum rho^n of the last
 * update (Section 4), and optionally the L2 norm of each component of the
 * last high-order residual R_p0 (r_l2[dim+2], may be NULL). */
int cgks_residual(cgks_solver *s, double *res, double *r_l2);

/* Test access to intermediate results of the last high-order evaluation in
 * the caller's cell order: R_p0 [n_cells*(dim+2)] (may be NULL). */
int cgks_get_rp0(cgks_solver *s, double *Rp0);

const char *cgks_strerror(int status);

/* ---- serving: many steady solves advanced together (no counterpart in
 * the paper; the per-solve arithmetic is the V-cycle above) ----
 * A server keeps every admitted solve's state on the device and advances
 * all of them with one batched V-cycle per cgks_server_step: their cells
 * and faces are concatenated into one index space (each solve's cells
 * padded to a multiple of 256), so every kernel of the cycle runs once for
 * the whole batch.  Requests are admitted first-come-first-served while the
 * sum of their device footprints stays within hbm_budget and fewer than
 * max_active are running; a solve retires when its density residual Res
 * (Section 4) has dropped by res_drop relative to its first cycle, when it
 * reaches max_cycles, or when it diverges.  Each solve's arithmetic is
 * identical to running it alone with cgks_pmg_cycle. */
typedef struct cgks_server cgks_server;

typedef struct {
  int32_t precision;     /* CGKS_FP64 or CGKS_MIXED for every solve */
  int32_t time_scheme;   /* CGKS_S1O2 or CGKS_S2O4 */
  double cfl_hi, cfl_lo; /* shared by all solves */
  int32_t n_implicit, n_sweeps;
  int32_t max_active;    /* solves per batch */
  int32_t max_cycles;    /* retire unconverged solves after this many cycles */
  int32_t use_graph;
  int32_t low_order_fused; /* 1: persistent cooperative low-order level */
  int32_t autotune;      /* 1 (default): autotuned launch shapes for the batch */
  int32_t programmatic_launch; /* 1 (default): programmatic dependent launch (see cgks_params) */
  int32_t flux_lo;       /* CGKS_FLUX_KFVS (default) or CGKS_FLUX_LF for every solve */
  int32_t lo_viscous;    /* 1: first-order viscous flux on the low-order level (see cgks_params) */
  void *stream;          /* cudaStream_t (NULL = default) */
  cgks_alloc_fn alloc;
  cgks_free_fn free;
  void *alloc_ctx;
} cgks_server_opts;

enum { CGKS_REQ_QUEUED = 0, CGKS_REQ_ACTIVE = 1, CGKS_REQ_CONVERGED = 2, CGKS_REQ_STOPPED = 3,
       CGKS_REQ_DIVERGED = 4, CGKS_REQ_REJECTED = 5 };

typedef struct {
  int32_t state;         /* CGKS_REQ_* */
  int32_t cycles;        /* V-cycles run */
  double res_first, res_last;
  double t_submit, t_admit, t_done;  /* seconds on the server's steady clock */
  int64_t n_cells;
} cgks_req_status;

/* Fill opts with defaults (FP64, S1O2, CFL 0.4 / 1000, 6 x 2, 64 active,
 * 20000 cycles, graphs on, autotune on, programmatic launch on). */
void cgks_server_default_opts(cgks_server_opts *o);
int cgks_server_create(size_t hbm_budget, const cgks_server_opts *opts, cgks_server **out);
/* Queue a request.  The mesh and W0 ([n_cells*4], caller order, host) are
 * copied; p supplies gamma, mu, alpha, the boundary conditions and the
 * flux class (the batch-wide fields come from the server options).  Each
 * request picks one of two flux classes, which share a batch: smooth
 * (CGKS_FLUX_SMOOTH, weno_eps 0: Section 4's subsonic setting) or limited
 * (CGKS_FLUX_FULL with weno_eps > 0 on conservative variables: its
 * transonic and supersonic setting); every limited request of a server
 * must carry the same weno_eps, weno_g0, tau_c1 and tau_c2 (CGKS_EINVAL
 * otherwise, and for any other flux setting).  max_cycles > 0 caps
 * this request's cycles below the server's max_cycles.  A request whose
 * footprint alone exceeds the budget is rejected (CGKS_EBUDGET); so are
 * the requests of a batch the server fails to allocate (the step that
 * tried returns the error). */
int cgks_server_submit(cgks_server *srv, const cgks_mesh *m, const cgks_params *p, const double *W0,
                       double res_drop, int32_t max_cycles, int64_t *req_id);
/* Retire finished solves, admit queued ones, run one batched V-cycle.
 * *n_active (may be NULL) receives the number of solves that ran. */
int cgks_server_step(cgks_server *srv, int32_t *n_active);
/* Status of a request; W_out (host [n_cells*4], may be NULL) receives the
 * final state once the request is done.  timeout_ms > 0: keep stepping the
 * server until the request is done or the time is up (CGKS_ETIMEOUT). */
int cgks_server_poll(cgks_server *srv, int64_t req_id, cgks_req_status *st, double *W_out, int timeout_ms);
/* Device bytes a request on mesh m counts against the budget: its share of
 * a batch's arena, its residual history and the stash that carries its
 * state across batch rebuilds. */
int cgks_server_footprint(const cgks_server *srv, const cgks_mesh *m, int64_t *bytes);
/* Bytes of device memory the active batch holds, and queued / active counts. */
int cgks_server_info(cgks_server *srv, int64_t *device_bytes, int32_t *n_queued, int32_t *n_active);
int cgks_server_destroy(cgks_server *srv);

/* ---- instrumentation (no counterpart in the paper) ----
 * Per-kernel timers: while on, every kernel launch of this solver is
 * bracketed by CUDA events on the library's stream and CUDA graphs are
 * bypassed.  cgks_get_timing fills up to max entries (kernel name, total
 * milliseconds, launch count) and returns the number of entries. */
int cgks_set_timing(cgks_solver *s, int on);
int cgks_get_timing(cgks_solver *s, int max, const char **names, double *total_ms, int64_t *count);
int cgks_reset_timing(cgks_solver *s);
/* Polls a grid-barrier wait of the persistent low-order launch
 * (low_order_fused, 2-D) makes before it gives up.  Past the limit the
 * launch ends early, every slot's status word gets the timeout bit, and the
 * call that ran it returns CGKS_ETIMEOUT; cgks_set_state clears the status
 * and the next launch starts from a cleared barrier.  polls = 0 restores
 * the default of 4,194,304 polls (seconds, far beyond any phase); a small
 * value makes the wait run out on purpose (tests of the timeout path).
 * CGKS_EINVAL for polls < 0 or a 3-D solver. */
int cgks_set_barrier_spin_limit(cgks_solver *s, int64_t polls);
/* Kernels launched by this solver so far, and kernels per V-cycle (cycle=1)
 * or per explicit step (cycle=0). */
int64_t cgks_launch_count(const cgks_solver *s);
int cgks_launches_per_call(const cgks_solver *s, int cycle);

/* ---- wall loads (post-processing of a converged field) ----
 * The momentum flux through every boundary face of one tag, evaluated by
 * the high-order level at the current state: the gas-kinetic flux F0 of
 * Section 2.2 (the smooth flux at t = 0, or with CGKS_FLUX_FULL the
 * constant term of its fit over one step of the current CFL time step;
 * pressure and viscous stress together), averaged over
 * the face's Gauss points, in the global frame, per unit length (2-D) or
 * area (3-D), in the direction of the face normal out of the fluid.  On a
 * wall it is the traction the fluid exerts: the body force is
 * sum(S * traction), and its normal and tangential parts give the surface
 * pressure and shear (Cd, Cl, Cp, Cf and the separation angle of Section
 * 4's cylinder and sphere tables).  At a steady state the boundary
 * tractions of all tags balance to the residual level.
 *   tag          boundary tag (index into cgks_params.bc[])
 *   max_faces    capacity of the output arrays (0: count only)
 *   n_faces      receives the number of faces with this tag
 *   x, n         [max_faces * dim] face centre and unit normal
 *   S            [max_faces] face length / area
 *   traction     [max_faces * dim] momentum flux per unit length / area
 * Host arrays, caller-owned, in the library's face order.  Runs a
 * reconstruction and face-flux evaluation on the solver's stream and
 * synchronises.  Returns CGKS_EINVAL (after setting n_faces) when
 * max_faces is too small. */
int cgks_wall_loads(cgks_solver *s, int32_t tag, int64_t max_faces, int64_t *n_faces, double *x, double *n,
                    double *S, double *traction);

/* ---- launch-shape autotuner (no counterpart in the paper) ----
 * Four kernels take a launch shape: the compact reconstruction, the
 * gas-kinetic face flux, the low-order (KFVS) face flux and the colour
 * sweep, in that order (CGKS_TUNE_KERNELS).  A shape (CGKS_TUNE_SHAPES of
 * them, index 0..4) is a block size, a number of items (cells or faces;
 * cells per lane group for the sweep) per thread and a minimum number of
 * resident blocks per SM (a register cap); cgks_tune_shape describes one.
 * Each item is computed by the same arithmetic under every shape, so the
 * shape never changes a result, only the time.
 * With autotune on, the first 3 x CGKS_TUNE_SHAPES V-cycles (or explicit
 * steps) that launch a kernel run without CUDA graphs, each with the next
 * shape in turn for that kernel; the first round only warms up (module
 * loading), the other rounds time every launch with CUDA events.  Then
 * each kernel keeps the shape of least mean launch time and the graphs are
 * captured with it.  The tuning cycles are ordinary cycles: the state
 * advances exactly as with fixed shapes. */
#define CGKS_TUNE_KERNELS 4
#define CGKS_TUNE_SHAPES 5
typedef struct {
  int32_t shape[CGKS_TUNE_KERNELS];  /* the shape in use (while tuning: the next one to try) */
  int32_t done[CGKS_TUNE_KERNELS];   /* 1 once the kernel's shape is final */
  double ms[CGKS_TUNE_KERNELS][CGKS_TUNE_SHAPES];  /* mean timed launch per shape (ms); 0 = not timed */
} cgks_tuning;
/* block size, items per thread, minimum resident blocks per SM of shape
 * index 0 .. CGKS_TUNE_SHAPES-1 (CGKS_EINVAL otherwise) */
int cgks_tune_shape(int32_t shape, int32_t *block, int32_t *per_thread, int32_t *min_blocks);
int cgks_get_tuning(cgks_solver *s, cgks_tuning *t);
/* Fix the shapes (each 0 .. CGKS_TUNE_SHAPES-1) and end any tuning. */
int cgks_set_tuning(cgks_solver *s, const int32_t shape[CGKS_TUNE_KERNELS]);
int cgks_server_get_tuning(cgks_server *srv, cgks_tuning *t);

/* ---- allocation-free residual (the paper has no counterpart) ----
 * Some callers cannot allocate device memory when they call into the
 * library: serving processes that fix their device memory at start-up and
 * keep cudaMalloc off the request path (it can block, synchronise the
 * device or fail under the budget), and host frameworks that own all device
 * memory and forbid libraries from allocating.  This entry point computes
 * the density residual Res = sum|rho_new - rho_old| / sum rho_old of two
 * device states without allocating anything.
 * 2-D states only: the states are read with the 2-D stride of 4 doubles per
 * cell; a 3-D state ([n_cells*5]) gives a wrong number.
 *   W_new_dev, W_old_dev  device arrays [n_cells*4], the 2-D ABI state
 *                         layout (only component 0, rho, is read)
 *   n_cells               1 .. 1,048,576; larger returns CGKS_EINVAL
 *   res_dev               device pointer receiving one double
 *   stream                cudaStream_t the two kernels run on (NULL = default)
 * Its scratch is a fixed 64 KiB __device__ array inside libcgks that every
 * GPU loading the library holds until the process exits.  The first call
 * in a CUDA context looks up that array's address in the context
 * (cudaGetSymbolAddress) and caches it per context handle; make that first
 * call before any stream capture.  (A context destroyed and a new one
 * created under the same handle would reuse a stale address: call from
 * contexts that live as long as the calls do.)  All calls share the one
 * array and it keeps the last call's partial sums; every call overwrites
 * the slots it reads, so nothing needs clearing, but calls that overlap on
 * the GPU (different streams, contexts or host threads) race on it and
 * must be serialised by the caller.  Returns CGKS_OK, CGKS_EINVAL or
 * CGKS_ECUDA. */
int cgks_density_residual_noalloc(const double *W_new_dev, const double *W_old_dev, int64_t n_cells,
                                  double *res_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif
