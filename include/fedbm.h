/*
 * fedbm.h -- C ABI of the GB300 finite element discrete Boltzmann library.
 *
 * The library advances the discrete-velocity BGK equation
 *     d f_i/dt + e_i . grad f_i = -(f_i - f_i^eq)/tau           (Sec. II.A, eq. DBE)
 * discretised by nodal DG on straight-sided triangles (Sec. II.B.1, eq. byparts)
 * with an upwind (or central) numerical flux, diffuse-scattering walls
 * (Sec. II.A.4, eq. FullBC / eq. UsedBC), the Hermite equilibrium of eq. feq
 * (optionally with the third Hermite term of eq. Herm3a), tau from eq. KnTau, and
 * explicit five-stage fourth-order low-storage Runge-Kutta time marching (the
 * paper's Sec. IV allows explicit RK of any order).  Every stage is one fused
 * CUDA kernel on sm_103a.
 *
 * Conventions shared by every entry point:
 *  - Return value: FEDBM_OK (0) on success, a negative FEDBM_E* code on error;
 *    fedbm_last_error() then returns a message (thread-local storage, valid
 *    until the next failing call on the same thread).  No C++ exception crosses
 *    the ABI.
 *  - Canonical state layout: double f[K][Np][Q], velocity index fastest.
 *    Structured meshes: element k = 2*(iy*nx + ix) + t of square (ix, iy);
 *    t = 0 is the triangle (A, B, C), t = 1 is (A, C, D), where A, B, C, D are
 *    the square's corners (x0,y0), (x1,y0), (x1,y1), (x0,y1); unstructured
 *    meshes: element k is the caller's triangle k.  Nodes are the warp & blend nodes
 *    (alpha = 0) numbered row by row in the reference s direction; velocity
 *    i = ix*n + iy of the n x n tensor set.  Node moments use [K][Np].
 *  - Ownership: the caller owns every buffer it passes; the library never keeps
 *    a caller pointer after a call returns.  The library owns its device state
 *    (allocated in fedbm_create, freed in fedbm_destroy) on the device that is
 *    current when fedbm_create is called.
 *  - Streams: all device work of a solver is ordered on the stream given to
 *    fedbm_create (NULL = legacy default stream).  Calls marked "synchronous"
 *    wait for that stream before returning.
 *  - on_device = 1 means the pointer is device memory of the solver's device;
 *    0 means host memory (pinned or pageable).
 */
#ifndef FEDBM_H
#define FEDBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FEDBM_OK          0
#define FEDBM_EINVAL     -1   /* bad argument or descriptor                   */
#define FEDBM_ENOMEM     -2   /* device or host allocation failed             */
#define FEDBM_ECUDA      -3   /* a CUDA runtime call failed                   */
#define FEDBM_ENONFINITE -4   /* NaN/Inf in the state or rho <= 0 at a node   */
#define FEDBM_ETIMEOUT   -5   /* a bounded device-side wait gave up           */
#define FEDBM_ENOTSUP    -6   /* configuration not compiled into the library  */
#define FEDBM_ENOCONV    -7   /* an implicit step's Newton iteration did not
                                 reach its tolerance                          */

/* ---- enumerations ------------------------------------------------------- */
enum fedbm_bc_kind {
  FEDBM_BC_PERIODIC     = 0,  /* pairs with the opposite side                 */
  FEDBM_BC_WALL_DIFFUSE = 1,  /* eq. FullBC, zero net mass flux               */
  FEDBM_BC_WALL_EQ      = 2   /* eq. UsedBC with rho_b = 1                    */
};
enum fedbm_velset_kind { FEDBM_VELSET_GH = 0, FEDBM_VELSET_NC = 1 };
enum fedbm_precision {
  FEDBM_FP64     = 0,         /* state, residual and arithmetic in FP64       */
  FEDBM_FP32     = 1,         /* state, residual and arithmetic in FP32       */
  FEDBM_BF16_DEV = 2,         /* state: BF16 per-element-scaled deviation from
                                 the rest equilibrium; FP32 residual and math */
  FEDBM_FP16_DEV = 3          /* same with FP16 deviation codes               */
};
enum fedbm_reduction {
  FEDBM_RED_DEFAULT   = 0,    /* the compute precision (FP64 in FP64 mode,
                                 FP32 otherwise)                              */
  FEDBM_RED_FP64      = 1,    /* velocity moments accumulated in FP64          */
  FEDBM_RED_COMP_FP32 = 2     /* compensated (Neumaier) FP32 accumulation      */
};

enum fedbm_tau_model {
  FEDBM_TAU_KN         = 0,   /* eq. KnTau: tau = Kn L / (sqrt(3) c_s)        */
  FEDBM_TAU_KIM_PITSCH = 1,   /* Kim & Pitsch mean free path: Kn carries a
                                 factor sqrt(pi/6), tau = Kn L / (sqrt(pi/2) c_s) */
  FEDBM_TAU_PSI        = 2    /* eq. KnTau times psi(Kn) =
                                 (2/pi) arctan(sqrt(2) Kn^(-3/4)) (Zhang)      */
};

/* ---- descriptors -------------------------------------------------------- */
/* Mesh of straight-sided triangles on the rectangle [0, lx] x [0, ly].
 * Sides: 0 -> y = 0, 1 -> x = lx, 2 -> y = ly, 3 -> x = 0.  Periodic sides must
 * come in opposite pairs.  Wall velocities are tangential (the component
 * normal to the wall must be 0).
 *
 * Structured (ntri = 0, Sec. III.A): nx x ny Cartesian cells, each split along
 * its lower-left/upper-right diagonal into two triangles; K = 2 nx ny.
 *
 * Unstructured (ntri > 0, the cavity meshes of Sec. III.B): a conforming
 * triangulation given by nvert vertices vert_xy[nvert][2] and ntri triangles
 * tri[ntri][3] (vertex indices, counter-clockwise); element k is triangle k,
 * face f joins its vertices f and f+1 mod 3.  The vertices must span
 * [0, lx] x [0, ly] (lx, ly are taken from them; the lx, ly fields and nx, ny
 * are ignored); every edge that only one triangle has must lie on a side of
 * that rectangle, and periodic sides must carry edges with the same end-point
 * coordinates along the side.  Both arrays are host memory, read during the
 * call that takes the descriptor (create, or a host-only query) and not kept.
 * Errors (EINVAL): indices out of range, a clockwise or degenerate triangle,
 * an edge shared by more than two triangles, a boundary edge inside the
 * rectangle, unmatched periodic edges. */
typedef struct fedbm_mesh_desc {
  int32_t nx, ny;        /* structured: cells in x and y; K = 2 nx ny          */
  int32_t order;         /* polynomial degree p, 0..6                         */
  int32_t bc[4];         /* enum fedbm_bc_kind per side                        */
  double  wall_ux[4];    /* wall velocity per side, units of sqrt(RT)          */
  double  wall_uy[4];
  double  lx, ly;        /* structured: domain size; 0 means 1                 */
  int32_t nvert, ntri;   /* unstructured: vertex and triangle counts (0: structured) */
  const double*  vert_xy; /* unstructured: [nvert][2] vertex coordinates       */
  const int32_t* tri;     /* unstructured: [ntri][3] counter-clockwise triangles */
} fedbm_mesh_desc;

/* Velocity set (Sec. II.A.3, Table 1; Newton-Cotes grid of Sec. III.B).
 * Velocities are in units of sqrt(RT) (theta = RT = c_s^2 = 1); Q = n * n. */
typedef struct fedbm_velset_desc {
  int32_t kind;          /* enum fedbm_velset_kind                              */
  int32_t n;             /* 1-D points (GH: 1..40, NC: 2..64)                   */
  double  nc_extent;     /* NC nodes on [-extent, extent] (0 means 4)           */
  int32_t nc_sqrt2;      /* NC grid unit: 0 -> sqrt(RT), 1 -> sqrt(2RT)         */
  int32_t eq_order;      /* Hermite order of f^eq: 2 (eq. feq) or 3 (eq. Herm3a) */
} fedbm_velset_desc;

typedef struct fedbm_params {
  double  kn;            /* Knudsen number; tau from it by tau_model below       */
  double  length;        /* characteristic length L (0 means 1)                 */
  double  beta;          /* flux parameter: 1 upwind, 0.5 central (Sec. II.B.1) */
  double  cfl;           /* dt = cfl*r_in,min/(max|e|*(p+1)^2) when dt <= 0     */
  double  dt;            /* explicit time step (> 0 overrides cfl)              */
  int32_t precision;     /* enum fedbm_precision                                */
  int32_t reduction;     /* enum fedbm_reduction                                */
  int32_t collision;     /* 1: BGK collision on; 0: pure advection              */
  int32_t elems_per_cta; /* stage-kernel tile: elements per CTA (0 = auto)      */
  int32_t threads_per_cta; /* stage-kernel tile: threads per CTA, multiple of 32,
                            <= 256 (0 = auto)                                  */
  int32_t pipeline_stages; /* stage-kernel tile buffers per CTA: 1, or 2 to load
                              the next tile while computing one (0 = auto: 3
                              where that form measured faster, i.e. 256 padded
                              velocities with FP32 state at degree 1-4 or BF16
                              at degree 3-5, when the tile arguments are 0
                              too; else 1);
                              3 = the warp-specialised form: a producer warp
                              keeps a ring of three one-element tiles filled
                              (bulk copies) for eight consumer warps, one
                              velocity per thread, 288 threads per CTA (tile
                              arguments ignored); FP32 or BF16 state with 256
                              padded velocities at degree <= 5, else EINVAL.
                              The autotuner times it where it exists      */
  int32_t tensor_cores;  /* stage-kernel form: 0 = the FMA kernel (the
                            faster form on every measured shape), with the
                            tensor-core form as one of the autotuner's
                            candidates; 1 = tensor cores (tcgen05 TF32 MMAs
                            for the Dr, Ds, LIFT contractions) required
                            (EINVAL where the form has none); -1 = FMA
                            kernel only, also for the autotuner.  The tensor-core
                            form exists at degree <= 5 for FP32, BF16 and FP16
                            state with 128, 256 or 1024 padded velocities,
                            and for FP32 and BF16 state with 16 (eight
                            elements stacked per MMA tile)                   */
  int32_t test_wait_timeout; /* test hook, keep 0: when 1, every stage kernel
                              waits for 16 bytes that never arrive, so its
                              bounded wait (about 2 s) runs out, the kernel
                              returns and the next synchronous read-out
                              (fedbm_mass, or get_moments / get_state to
                              host memory) reports FEDBM_ETIMEOUT            */
  int32_t tau_model;     /* enum fedbm_tau_model (Sec. II.A.4); 0 = eq. KnTau   */
  int32_t velocity_split; /* velocity-split stage kernel, a thread-block cluster
                             of CTAs sharing each element (FP64, FP32, BF16
                             state): 0 = automatic (used when one CTA cannot
                             hold all velocities of an element, e.g. D2Q1089
                             at degree 5 and 6), 1 = never, 2, 4 or 8 = that
                             cluster size (EINVAL where it does not divide
                             the padded velocity count into multiples of 8) */
  int32_t rounding;      /* encode of the new BF16 deviation state: 0 = round to
                            nearest even; 1 = stochastic rounding (BF16 only:
                            a counter-based draw per value, stage and step, so
                            that stage increments below half a BF16 unit are
                            kept in expectation instead of being rounded away;
                            the draws restart with each state load)       */
} fedbm_params;

typedef struct fedbm_info_t {
  int64_t K, Np, Nfp, Q, Q_padded;
  double  dt, tau, time;
  int64_t steps;                 /* completed RK steps                           */
  int32_t precision, reduction, order, eq_order;
  int32_t elems_per_cta, threads_per_cta;
  int32_t pipeline_stages, grid; /* stage-kernel buffers per CTA (3: the warp-
                                    specialised form); persistent grid          */
  int32_t group, ngroups;        /* batches: kernel group of this case; group count */
  int32_t tensor_cores;          /* 1 if the group's stage kernel is the tensor-core form */
  int32_t velocity_split;        /* CTAs per element tile: 1, or the cluster size of the
                                    velocity-split form                          */
  int64_t state_bytes;           /* device bytes of one state buffer             */
  int64_t residual_bytes;        /* device bytes of the RK residual              */
} fedbm_info_t;

typedef struct fedbm_solver fedbm_solver;   /* opaque, library-owned */

/* ---- host-only queries (no GPU needed) ---------------------------------- */

/* 2-D velocity set of a descriptor (Sec. II.A.3, Table 1).  Writes Q values to
 * each of ex, ey, w (any may be NULL) and Q to *q.  Pass ex = ey = w = NULL to
 * query Q first.  Errors: EINVAL for an unsupported descriptor. */
int fedbm_velset(const fedbm_velset_desc* vs, double* ex, double* ey, double* w, int32_t* q);

/* Reference-element operators of degree p (Sec. II.B.1): nodes r, s [Np];
 * derivative matrices Dr, Ds [Np][Np] row-major; LIFT [Np][3*Nfp] (inverse
 * mass matrix times the face mass matrices, faces 0: s=-1, 1: r+s=0, 2: r=-1,
 * face nodes in increasing r, s, s); mass matrix M [Np][Np]; fmask [3][Nfp].
 * Any output may be NULL.  Errors: EINVAL if p is outside 0..6. */
int fedbm_ref_operators(int32_t p, double* r, double* s, double* Dr, double* Ds,
                        double* LIFT, double* M, int32_t* fmask);

/* Physical node coordinates x, y [K][Np] of a mesh descriptor, and the time
 * step the given velocity set / params would use (*dt, may be NULL). */
int fedbm_mesh_nodes(const fedbm_mesh_desc* mesh, const fedbm_velset_desc* vs,
                     const fedbm_params* prm, double* x, double* y, double* dt);

/* Face connectivity of a mesh descriptor: nbr[K][3].  For face f of element k
 * (face f joins vertices f and f+1 mod 3 of the counter-clockwise triangle),
 * nbr = (kn << 3) | (fn << 1) | rev with kn the neighbour element, fn its face
 * and rev = 1 when the two faces list their shared nodes in opposite order; a
 * wall face stores -(side + 1).  Periodic sides wrap to the opposite side. */
int fedbm_mesh_connectivity(const fedbm_mesh_desc* mesh, int32_t* nbr);

/* ---- solver lifecycle ---------------------------------------------------- */

/* Build the velocity set, mesh, operators and wall data on the host in FP64,
 * upload them, and allocate the device state (two state buffers and one
 * residual).  cuda_stream is a cudaStream_t (NULL = default stream).  The
 * state is left zero; call fedbm_set_state or fedbm_set_equilibrium before
 * stepping.  Errors: EINVAL, ENOMEM, ECUDA, ENOTSUP. */
int fedbm_create(const fedbm_mesh_desc* mesh, const fedbm_velset_desc* vs,
                 const fedbm_params* prm, void* cuda_stream, fedbm_solver** out);

/* Free every device and host resource of the solver (NULL is allowed). */
void fedbm_destroy(fedbm_solver* s);

/* Load a canonical FP64 state f[K][Np][Q] (host or device) and encode it into
 * the storage precision.  Resets time and step count to 0.  Asynchronous for
 * device input; host input is copied before the call returns. */
int fedbm_set_state(fedbm_solver* s, const double* f, int32_t on_device);

/* The same from a canonical FP32 state float f[K][Np][Q] (host or device):
 * for FP32 storage each value is stored as given, so a caller whose data are
 * FP32 moves half the bytes of the FP64 call; the deviation forms encode from
 * the FP32 values in FP64 as fedbm_set_state does. */
int fedbm_set_state_f32(fedbm_solver* s, const float* f, int32_t on_device);

/* f_i = f_i^eq(rho0, u0) * (1 + amp * u), u in [-1, 1) drawn by SplitMix64 at
 * canonical index (k*Np + j)*Q + i of seed (a seeded perturbation of an
 * equilibrium, computed on the device).  Resets time and step count. */
int fedbm_set_equilibrium(fedbm_solver* s, double rho0, double ux0, double uy0,
                          double amp, uint64_t seed);

/* Advance nsteps full LSRK(5,4) steps (5 fused stage kernels each), replayed
 * from a CUDA graph captured on first use.  Asynchronous. */
int fedbm_rk_step(fedbm_solver* s, int32_t nsteps);

/* Run one LSRK(5,4) stage (0..4) with the same kernel rk_step uses; stage 0
 * ignores the residual's previous contents (its A coefficient is 0).  For
 * testing single stages.  Asynchronous. */
int fedbm_rk_stage(fedbm_solver* s, int32_t stage);

/* ---- implicit time marching (Sec. II.B.3) ---------------------------------
 * The paper marches eq. byparts with singly diagonally implicit Runge-Kutta
 * methods: a four-stage fourth-order scheme for the Couette order study and the
 * one-stage first-order scheme (backward Euler) for the cavities, each stage
 * linearised by Newton's method and solved by GMRES.  The paper prints no
 * tableau for its fourth-order scheme; the library offers two published
 * fourth-order SDIRK tableaux and a caller-given one:
 *   FEDBM_IMPLICIT_BE         backward Euler (1 stage, order 1, L-stable)
 *   FEDBM_IMPLICIT_SDIRK3_O4  Crouzeix/Norsett (3 stages, order 4, A-stable,
 *                             gamma = 1/2 + cos(pi/18)/sqrt(3))
 *   FEDBM_IMPLICIT_SDIRK5_O4  Hairer & Wanner (5 stages, order 4, L-stable,
 *                             gamma = 1/4, stiffly accurate)
 *   FEDBM_IMPLICIT_CUSTOM     stages 1..6, A (row-major 6 x 6, lower
 *                             triangular, every diagonal entry A[0][0] > 0), b
 * Stage i solves Y_i = u_n + dt sum_{j<i} a_ij k_j + dt gamma R(Y_i) by
 * Newton's method, k_i = (Y_i - base_i)/(dt gamma), u_{n+1} = u_n + dt sum b_i k_i.
 * Each Newton correction solves (I - dt gamma J) d = -G with restarted
 * GMRES(m) (classical Gram-Schmidt with re-orthogonalisation, optionally right
 * preconditioned by element-and-velocity block Jacobi), J v =
 * (R(Y + e v) - R(Y)) / e matrix-free; every R is one
 * launch of the fused stage kernel.  Vectors are FP64 in the device layout;
 * R runs in the solver's precision (FP64 or FP32 state only). */
enum fedbm_implicit_scheme {
  FEDBM_IMPLICIT_BE = 0,
  FEDBM_IMPLICIT_SDIRK3_O4 = 1,
  FEDBM_IMPLICIT_SDIRK5_O4 = 2,
  FEDBM_IMPLICIT_CUSTOM = 3
};
typedef struct fedbm_implicit_params {
  int32_t scheme;          /* enum fedbm_implicit_scheme                          */
  int32_t stages;          /* FEDBM_IMPLICIT_CUSTOM only: 1..6                    */
  double  A[36];           /* FEDBM_IMPLICIT_CUSTOM only: row-major 6 x 6 tableau */
  double  b[6];            /* FEDBM_IMPLICIT_CUSTOM only: weights                 */
  double  dt;              /* time step (not limited by the CFL condition), > 0   */
  double  newton_rtol;     /* stage converged when |G|_2 <= max(rtol |G_0|_2, atol);
                              0 means 1e-10                                        */
  double  newton_atol;     /* absolute 2-norm tolerance; 0 means none            */
  int32_t newton_max_iter; /* per stage; 0 means 20                               */
  int32_t gmres_restart;   /* m (1..200); 0 means 30                              */
  int32_t gmres_max_iter;  /* per Newton correction; 0 means 1000                 */
  double  gmres_rtol;      /* forcing term: |J d + G| <= rtol |G|; 0 means 1e-4   */
  int32_t preconditioner;  /* 0: none; 1: element-and-velocity block Jacobi (right
                              preconditioning by the inverse of each element's
                              own-node block of I - dt gamma J at each velocity:
                              transport within the element, the element's own
                              upwind face traces and the 1/tau relaxation;
                              built once per dt gamma, K Np^2 Qp doubles) */
} fedbm_implicit_params;
typedef struct fedbm_implicit_stats {
  int32_t newton_iters;    /* Newton corrections over all stages and steps        */
  int32_t gmres_iters;     /* GMRES iterations (Jacobian-vector products)         */
  int32_t rhs_evals;       /* stage-kernel launches evaluating R                  */
  int32_t converged;       /* 1 if every stage met its Newton tolerance           */
  double  residual;        /* |G|_2 of the last stage                             */
} fedbm_implicit_stats;

/* Advance nsteps implicit steps of size ip->dt from the current state
 * (synchronous).  The time reported by fedbm_info grows by dt per step.
 * stats may be NULL.  Errors: EINVAL (batches, BF16/FP16 state, bad
 * parameters), ENOCONV (a stage's Newton iteration reached newton_max_iter;
 * the state is then the last step's result), ENONFINITE, ECUDA, ENOMEM. */
int fedbm_implicit_step(fedbm_solver* s, const fedbm_implicit_params* ip, int32_t nsteps,
                        fedbm_implicit_stats* stats);

/* Node moments rho, u_x, u_y [K][Np] in FP64 of the current state.
 * Synchronous for host outputs; with host outputs it also returns ETIMEOUT if
 * a stage kernel since the last state load gave up a bounded wait (the state
 * is then only partly updated).  That timeout word stays set until the next
 * fedbm_set_state / fedbm_set_equilibrium; fedbm_rk_step is asynchronous and
 * cannot report it itself. */
int fedbm_get_moments(fedbm_solver* s, double* rho, double* ux, double* uy, int32_t on_device);

/* Decode the current state into canonical FP64 f[K][Np][Q].  Synchronous for
 * host output, and then reports ETIMEOUT as fedbm_get_moments does. */
int fedbm_get_state(fedbm_solver* s, double* f, int32_t on_device);

/* Decode the LSRK residual register into canonical FP64 [K][Np][Q]. */
int fedbm_get_residual(fedbm_solver* s, double* res, int32_t on_device);

/* Global mass sum_k J_k 1^T M rho_k (synchronous), every stored value decoded
 * and summed in FP64 (the velocity sum of each node too, whatever the storage
 * precision).  Returns ENONFINITE if any node has a non-finite value or
 * rho <= 0, and ETIMEOUT if a stage kernel since the last state load reported
 * a bounded wait that gave up. */
int fedbm_mass(fedbm_solver* s, double* total_mass);

int fedbm_info(const fedbm_solver* s, fedbm_info_t* info);

/* ---- batched form -------------------------------------------------------- */
/* Many independent cases (each its own mesh, Kn, wall speeds, time step) that
 * advance together (for example sweeps over the paper's Couette and cavity
 * cases of Sec. III).  Cases with the same degree, velocity set, precision,
 * reduction, collision switch, beta and tile parameters form one group: their
 * element lists are concatenated and one stage-kernel launch per RK stage
 * covers them all (per-element time step and 1/tau, per-case wall slots);
 * groups are independent branches of one CUDA graph per RK step.  Every case
 * takes one step of its own dt per fedbm_batch_rk_step step.  Case indices
 * follow the order of `cases`. */
typedef struct fedbm_case_desc {
  fedbm_mesh_desc   mesh;
  fedbm_velset_desc velset;
  fedbm_params      params;
} fedbm_case_desc;

typedef struct fedbm_batch fedbm_batch;     /* opaque, library-owned */

/* Set up every case (as fedbm_create does for one).  Errors: EINVAL, ENOMEM,
 * ECUDA. */
int fedbm_batch_create(const fedbm_case_desc* cases, int32_t ncases, void* cuda_stream,
                       fedbm_batch** out);
void fedbm_batch_destroy(fedbm_batch* b);
/* Per-case counterparts of the solver calls (case c, 0 <= c < ncases). */
int fedbm_batch_set_state(fedbm_batch* b, int32_t c, const double* f, int32_t on_device);
int fedbm_batch_set_state_f32(fedbm_batch* b, int32_t c, const float* f, int32_t on_device);
int fedbm_batch_set_equilibrium(fedbm_batch* b, int32_t c, double rho0, double ux0, double uy0,
                                double amp, uint64_t seed);
int fedbm_batch_get_state(fedbm_batch* b, int32_t c, double* f, int32_t on_device);
int fedbm_batch_get_moments(fedbm_batch* b, int32_t c, double* rho, double* ux, double* uy,
                            int32_t on_device);
int fedbm_batch_mass(fedbm_batch* b, int32_t c, double* total_mass);
int fedbm_batch_info(const fedbm_batch* b, int32_t c, fedbm_info_t* info);
/* Advance every case nsteps LSRK(5,4) steps (one graph launch per step). */
int fedbm_batch_rk_step(fedbm_batch* b, int32_t nsteps);
/* Re-tile one group's stage kernel as the FMA form (0 = automatic for each
 * argument; pipeline_stages = 3 selects the warp-specialised form, whose tile
 * is fixed); used by the tile autotuner.  Takes effect from the next step.
 * On EINVAL (a tile that is not valid or does not fit shared memory) the group
 * keeps its current form and tile. */
int fedbm_batch_set_tiles(fedbm_batch* b, int32_t group, int32_t elems_per_cta,
                          int32_t threads_per_cta, int32_t pipeline_stages);
/* Switch one group's stage kernel to the tensor-core form (on = 1; EINVAL if
 * the group's form has none, or if it was created with tensor_cores = -1) or
 * back to the default FMA form with automatic tiles (on = 0; the
 * warp-specialised form where pipeline_stages = 0 would choose it).  Next step
 * onwards. */
int fedbm_batch_set_tensor_cores(fedbm_batch* b, int32_t group, int32_t on);

/* Tile autotuner: for every kernel group, time each candidate stage-kernel
 * tile (elements per CTA 1..32, threads per CTA 64/128/256, one or two
 * pipeline stages, the tensor-core form where the group has it and was not
 * created with tensor_cores = -1, and from 256 padded velocities up the
 * velocity-split form with clusters of 2 and 4 CTAs unless velocity_split = 1)
 * on `trials` launches (0 means 5) and keep the fastest.  Groups that use the
 * velocity-split form because no FMA tile fits keep it.
 * The current state is left unchanged.  With a cache_path (NULL or "" for
 * none), results are read from and written to a JSON object keyed by device
 * name, degree, padded velocity count, precision, reduction and element
 * count.  Synchronous.  Errors: ECUDA if no candidate runs. */
int fedbm_batch_autotune(fedbm_batch* b, const char* cache_path, int32_t trials);
int fedbm_autotune(fedbm_solver* s, const char* cache_path, int32_t trials);

/* Allocation-free mass diagnostic.  The paper has no counterpart; this entry
 * point serves callers that must not allocate device memory once they are
 * running -- an application whose device memory belongs to another allocator
 * (a framework's caching allocator or a fixed pre-reserved pool), or a
 * real-time loop that cannot pay for cudaMalloc's latency and implicit device
 * synchronisation.  It computes the same FP64 sum as fedbm_mass,
 *     total = sum_k jac[k] * sum_n mass_colsum[n] * sum_i f[k][n][i],
 * from caller-owned device buffers: f canonical FP64 [K][Np][Q], jac [K]
 * (element Jacobians, area / 2), mass_colsum [Np] (column sums 1^T M of the
 * reference mass matrix, see fedbm_ref_operators), and writes total[0] and
 * status[0] (0 = fine, 1 = a node has a non-finite value or rho <= 0) to
 * device memory, asynchronously on cuda_stream (NULL = default stream).
 * It calls no cudaMalloc/cudaFree: its scratch (one FP64 partial sum per 256
 * nodes plus a status word, 65,792 bytes) is a fixed __device__ array that
 * every GPU loading the library holds until the process exits.  Capacity:
 * K * Np <= 2,097,152 nodes; larger inputs return FEDBM_EINVAL with a message
 * and launch nothing.  The scratch's device address belongs to the CUDA
 * context that is current at the call (a context loads its own copy of the
 * array): the first call in each context (the device's primary context, a
 * driver-API context of the caller's, or the new primary context after
 * cudaDeviceReset) looks the address up with cudaGetSymbolAddress and caches it
 * under the context's unique ID, so make that first call before any stream
 * capture.  All calls in one context share the one scratch array; every call
 * clears the status word before use, but calls that may overlap on the GPU
 * (different streams without ordering) race and give wrong results.
 * Errors: EINVAL (null pointer, sizes), ECUDA. */
int fedbm_mass_noalloc(const double* f, const double* jac, const double* mass_colsum,
                       int64_t K, int32_t Np, int32_t Q, double* total, int32_t* status,
                       void* cuda_stream);

const char* fedbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FEDBM_H */
