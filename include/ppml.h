/*
 * ppml.h -- C ABI of libppml.so, a GB300 (sm_103a) implementation of one timestep of
 * the PPML operator-splitting Godunov scheme of Kulikov & Vorobyov (arXiv:1607.01105)
 * for the ideal-gas Euler equations with total and internal energy on a uniform grid.
 *
 * What a step computes (paper Sec. 1 "NUMERICAL SCHEME" and the Appendix):
 *   Eulerian stage (Sec. 1.1/1.2, eqs. SCHdensEulerian..SCHintenEulerian,
 *     lowriemannvelocity, lowriemannpressure): PPML parabolas of v and p per cell and
 *     axis (Appendix Steps 1-3), the acoustic Riemann solution (V, P) at every face with
 *     the modified Roe averages, and the update rho v -= tau dP/dx, rho E -= tau d(PV)/dx,
 *     rho eps -= tau (gamma-1) rho eps dV/dx summed over the three axes;
 *   Lagrangian stage (Sec. 1.3, eqs. genlagrange, fluxonlagrangestage,
 *     modspaceaveragevelocitylagrange, veltemplate): the 9-point transverse velocity
 *     template, Roe-weighted face velocity, upwind parabola-average fluxes of rho, rho v,
 *     rho E, rho eps, unsplit update;
 *   energy consistency (Sec. 1.4), the CFL step of the new state (Sec. 1.1) and FP64
 *     conservation sums.
 *
 * Conventions shared by every call:
 *   - State: six device arrays (rho, m_x, m_y, m_z, rho E, rho eps), each nx*ny*nz
 *     interior cells, x fastest, contiguous, element type per ppml_grid_desc.dtype,
 *     16-byte aligned.  No ghost cells: the boundary conditions are applied when the
 *     kernels read neighbours (outflow = zero-gradient, periodic = wrap, reflecting =
 *     mirror with the normal momentum negated; edges and corners as if ghosts were
 *     filled along x, then y, then z).
 *   - The caller owns every state array and the stream; the library owns its handle,
 *     the intermediate state U* and its reduction scratch (allocated by ppml_init_grid
 *     with cudaMalloc, freed by ppml_free_grid).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous
 *     on that stream unless they return a host value (documented per call).
 *   - Return value: PPML_OK (0) or an error code; ppml_last_error() gives a message for
 *     the calling thread.  No call aborts, prints or exits.
 *   - Not thread-safe per handle: one handle must not be used from two host threads at
 *     once.  Different handles are independent.
 */
#ifndef PPML_H
#define PPML_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PPML_OK = 0,
  PPML_E_INVAL = 1,       /* bad argument: sizes, gamma, cfl, null or misaligned pointers */
  PPML_E_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
  PPML_E_NONPHYSICAL = 3, /* reported by ppml_read_diag: rho <= 0, rho eps <= 0 or NaN seen */
  PPML_E_TIMEOUT = 4,     /* reserved: no call waits on another kernel */
  PPML_E_NOMEM = 5        /* device or host allocation failed */
} ppml_status;

typedef enum {
  PPML_F32 = 0, /* state in float; dt, conservation sums and the energy correction in double */
  PPML_F64 = 1  /* everything in double */
} ppml_dtype;

typedef enum {
  PPML_BC_OUTFLOW = 0,
  PPML_BC_PERIODIC = 1,
  PPML_BC_REFLECT = 2,
  PPML_BC_HALO = 3, /* z faces only: a slab of a z-decomposed grid (see "z-slab decomposition") */
  PPML_BC_INFLOW = 4 /* the face's ghost cells hold a prescribed state (ppml_grid_desc.inflow);
                        at an edge or corner of two ghost regions the later axis (x, y, z order)
                        decides; not on a grid with a reflecting face */
} ppml_bc;

/* scheme variants (ppml_grid_desc.flags) */
#define PPML_FIRST_ORDER 1u /* piecewise-constant states in both stages (Sec. 1.1, the first-order
                               scheme the paper compares against) */
#define PPML_VHAT_1PT 2u    /* face velocity of the Lagrangian stage from the line only, without
                               the 9-point template (the 1-point variant of Sec. 1.3) */

/* flag bits accumulated on the device (ppml_diag.flags) */
#define PPML_FLAG_NONPHYSICAL 1u /* an output cell had rho <= 0, rho eps <= 0 or a NaN/Inf */
#define PPML_FLAG_DT_ZERO 2u     /* the CFL step underflowed to 0 (or t_end reached) */

/* Problem statement (paper Sec. 1 and Sec. 1.1: grid, gamma, CFL number, boundaries). */
typedef struct {
  int nx, ny, nz;     /* interior cells per axis, >= 1; an axis with one cell is inactive */
  double h[3];        /* cell size per axis (> 0); cell volume h[0]*h[1]*h[2] */
  double gamma;       /* ratio of specific heats, > 1 */
  double cfl;         /* Courant number, 0 < cfl < 1 (paper: 0.2) */
  int bc[6];          /* ppml_bc per face: -x, +x, -y, +y, -z, +z; periodic faces come in
                         pairs; an inactive axis may not be reflecting */
  int dtype;          /* ppml_dtype */
  double vacuum_frac; /* vacuum threshold of the energy correction relative to the mean
                         initial density (paper Sec. 1.4: five orders of magnitude, 1e-5);
                         <= 0 selects 1e-5 */
  double t_end;       /* > 0: the device-side CFL step is clipped so t lands on t_end */
  int flags;          /* PPML_FIRST_ORDER | PPML_VHAT_1PT variants; 0 = the PPML scheme */
  double rho_ref;     /* > 0: reference density of the vacuum threshold (a slab passes the
                         whole grid's mean); 0: the mean of the initial state */
  double inflow[6][6]; /* per face, for PPML_BC_INFLOW faces: the conserved state of its ghost
                          cells (rho > 0, m_x, m_y, m_z, rho E, rho eps > 0; finite); other
                          faces' entries are not read */
} ppml_grid_desc;

/* Six device pointers: rho, m_x, m_y, m_z, rho E, rho eps (see conventions), and for FP32
 * states optionally the low parts of the first five.  lo all NULL: a plain float state.
 * lo all set (FP32 only): a double-float state, field f = f[f] + lo[f] with |lo| at most
 * half an ulp of f[f], about 48 significant bits.  The stencil arithmetic reads the high
 * parts; every update of rho, m and rho E is added in double-float and the energy
 * consistency of Sec. 1.4 takes rho E - |m|^2 / (2 rho) from both parts, so the internal
 * energy of cold, fast flow (a small difference of large totals) keeps FP64-class
 * accuracy.  Mixing NULL and non-NULL lo pointers, or lo with PPML_F64, is PPML_E_INVAL;
 * a step's input and output states carry low parts both or neither. */
typedef struct {
  void* f[6];
  void* lo[5];
} ppml_state;

/* Host copy of the device-resident diagnostics after the last step or dt call. */
typedef struct {
  double t;          /* simulated time reached */
  double dt_next;    /* CFL step of the last output state, clipped to t_end */
  double vmax, cmax; /* max |v| and max sound speed of that state */
  double sums[6];    /* sum over cells of each field times the cell volume (FP64) */
  long long steps;   /* steps taken since init */
  long long n_vacuum;/* cells that took the vacuum branch of the energy correction, last step */
  long long n_bad;   /* cells flagged non-physical in the last diagnosed state */
  unsigned flags;    /* PPML_FLAG_* bits raised since init */
} ppml_diag;

typedef struct ppml_grid ppml_grid;

/* Create a handle for the grid in *d and allocate its scratch (U*: five fields of the
 * state's type, in FP32 also the four low parts of U*'s m and rho E; reduction partials).
 * Reads u0 once on `stream` to fix the mean initial density (the vacuum threshold
 * reference, Sec. 1.4) and the first CFL step; synchronizes the stream.  u0 is not
 * modified.  On error *out is NULL. */
int ppml_init_grid(const ppml_grid_desc* d, const ppml_state* u0, void* stream, ppml_grid** out);

/* Free the handle and its scratch (synchronizes the device first).  NULL is a no-op. */
int ppml_free_grid(ppml_grid* g);

/* CFL step of state u (Sec. 1.1: tau = cfl * min_a h_a / (max|v| + max c), the maxima
 * taken separately, |v| Euclidean, inactive axes excluded), clipped to t_end - t.  The
 * result is stored on the device (ppml_dt_device) for the next ppml_step with dt <= 0;
 * if dt_host is non-NULL the stream is synchronized and the value copied there. */
int ppml_cfl_dt(ppml_grid* g, const ppml_state* u, double* dt_host, void* stream);

/* One full step U^n -> U^{n+1} (Eulerian stage, Lagrangian stage, energy correction),
 * with the CFL step and the FP64 sums of U^{n+1} computed in the same pass.
 * dt > 0: use it; dt <= 0: use the device-resident step from ppml_cfl_dt or from the
 * previous ppml_step (no host synchronization, so steps can be captured in a CUDA graph).
 * u_in and u_out must not alias; u_in is not modified.  Asynchronous. */
int ppml_step(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out, double dt, void* stream);

/* ppml_step with a gravitational potential (paper eqs. for rho v and rho E: the source
 * terms -rho grad Phi and -rho v . grad Phi).  phi: device array of nx*ny*nz cells of the
 * state's type, or NULL (then identical to ppml_step).  The Eulerian stage adds
 * m -= tau rho grad Phi and rho E -= tau m . grad Phi from U^n with cell-centred central
 * differences of Phi (boundary values of Phi: zero-gradient at outflow and reflecting
 * faces, wrapped at periodic ones). */
int ppml_step_phi(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out, const void* phi,
                  double dt, void* stream);

/* Periodic solve of the 27-point discretisation of Delta Phi = 4 pi G rho (paper Sec. "The
 * Poisson solver", eq. stencil27point and the harmonic-space formula of its Stages 2-3):
 * Phi = IFFT( -(2/3) pi G h^2 FFT(rho) / (1 - prod_a (1 - (2/3) sin^2(pi k_a/N_a))) ), the
 * k = 0 mode set to zero (the potential of rho minus its mean).  The printed formula lacks
 * the minus sign that the stencil's symbol carries.  Requires h[0] = h[1] = h[2] on active
 * axes.  rho, phi: device arrays of nx*ny*nz cells of the grid's type (may not alias).
 * Uses cuFFT plans and a spectrum buffer created on the first call and kept in the handle.
 * Asynchronous. */
int ppml_poisson_periodic(ppml_grid* g, const void* rho, void* phi, double G, void* stream);

/* Global Fourier amplitudes of a disk (paper, section on the gravitationally unstable
 * disks, eq. of A_m(t)): A_m = |sum Sigma e^{i m phi}| / sum Sigma over the columns whose
 * centre is within r_f of the z axis, Sigma the column density (sum over z of rho h_z) and
 * phi = atan2(y, x) of the column centre, for m = 1..m_max (1 <= m_max <=
 * PPML_FOURIER_MAX_MODES).  Column (i, j) is centred at ((i + 1/2 - nx/2) h_x,
 * (j + 1/2 - ny/2) h_y): the grid is centred on the axis.  rho: device array of the grid's
 * type.  Sums in FP64 in a fixed order.  Writes a_out[m_max] on the host; synchronizes the
 * stream.  PPML_E_INVAL for bad arguments or no mass within r_f.  Buffers of about 0.3 MB
 * are created on the first call and kept in the handle. */
#define PPML_FOURIER_MAX_MODES 16
int ppml_fourier_amplitudes(ppml_grid* g, const void* rho, double r_f, int m_max, double* a_out,
                            void* stream);

/* Right-hand side exactly as printed (4 pi G h^2 rho; second-order accurate). */
#define PPML_POISSON_PRINTED_RHS 1u

/* Isolated-boundary Poisson solve (paper Sec. "The Poisson solver", Stages 1-3, with the
 * 27-point stencil eq. stencil27point), for a mass distribution that vanishes outside the
 * grid.  Stage 1: the monopole and quadrupole moments of the cell masses rho h^3 about the
 * grid centre give the potential on the shell of cells just outside the grid,
 *   Phi_b = -G M / r - (G/2) (I_x + I_y + I_z - 3 I_0) / r^3
 * (MacCullagh's formula; the paper prints the quadrupole term without the 1/2), and the shell
 * values in the stencil of a boundary cell move to the right-hand side.  Stages 2-3: the
 * Dirichlet problem is diagonal in the sine basis, so the transform is a type-I sine
 * transform along each axis and the paper's harmonic formula is used with pi j / N replaced
 * by pi j / (2 (N + 1)), j = 1..N.  Right-hand side 4 pi G h^2 (rho + D7 rho / 12) (D7 the
 * 7-point second difference, rho = 0 outside the grid), which gives the fourth order the
 * paper reports in its Table 1; flags = PPML_POISSON_PRINTED_RHS uses 4 pi G h^2 rho.
 * Geometry: cell (i, j, k) is centred at ((i + 1/2 - nx/2) h, (j + 1/2 - ny/2) h,
 * (k + 1/2 - nz/2) h); the grid is centred on the origin of the expansion.  Requires
 * h[0] = h[1] = h[2].  rho, phi: device arrays of nx*ny*nz cells of the grid's type (may
 * not alias; phi is also the work array).  Moments and shell values are formed in FP64; the
 * transforms run in the grid's type.  The first call creates cuFFT plans and buffers of
 * about 2 (N+1)/N x 3 states' worth of the grid's type, kept in the handle.  Asynchronous.
 * PPML_E_INVAL for bad arguments or unknown flags. */
int ppml_poisson_isolated(ppml_grid* g, const void* rho, void* phi, double G, unsigned flags,
                          void* stream);

/* Launch shape of the stage kernels (the paper has no counterpart: a systems choice).  A
 * step runs one CTA per 16^3 tile; the tiles are launched in one of PPML_TILE_ORDERS
 * orders, which decide which tiles run at the same time and hence which halos and template
 * boxes the L2 cache still holds: 0 x-major (ppml_init_grid's choice), 1 z-major, 2 in
 * blocks of 2^3 tiles, 3 in blocks of 4^3 tiles (x-major within and over the blocks).
 * Results do not depend on the order (every tile computes the same values, and the CFL and
 * sum partials are reduced in tile order).  ppml_grid_set_order fixes it (PPML_E_INVAL for
 * another value).  ppml_grid_tune times each order for trial_steps (>= 1) steps, the faster
 * of two runs, on scratch copies of u's six fields with the handle's step scalars saved
 * and restored (u and the handle's time are unchanged), keeps the fastest and returns it
 * in *order_out (may be NULL) and the times in ms_out (may be NULL).  It allocates and
 * frees two scratch states and synchronizes the stream; do not capture it in a graph. */
#define PPML_TILE_ORDERS 4
int ppml_grid_set_order(ppml_grid* g, int order);
int ppml_grid_tune(ppml_grid* g, const ppml_state* u, int trial_steps, int* order_out,
                   double ms_out[PPML_TILE_ORDERS], void* stream);

/* ------------------------------------------------------------ z-slab decomposition
 * A grid split along z into slabs, one per GPU (the paper runs on one node and has no
 * decomposition; this is the timestep spread over devices).  A slab's grid is the grid with
 * nz = the slab's planes and PPML_BC_HALO on each z face it shares with another slab (the
 * whole grid's own z boundaries stay on the outer slabs' other faces; a periodic z axis
 * makes both faces of every slab halo faces).  Behind a halo face the caller's arrays hold
 * PPML_HALO_PLANES planes of the neighbour's cells: the caller allocates them before
 * (after) the interior planes and passes pointers to the first interior plane.  That holds
 * for the state and for the U* arrays given to the stage calls; low parts of double-float
 * states need no halo planes.  One step of every slab, ranks in lockstep:
 *   fill U^n's halo planes from the neighbours; ppml_eulerian_stage(g, u, u_star, dt);
 *   fill u_star's halo planes from the neighbours;
 *   ppml_lagrangian_stage(g, u_star, u_out, dt, red);
 *   all-reduce red over the slabs (max of red[0..1], sum of red[2..9]);
 *   ppml_apply_reduced(g, red, 1, dt).
 * Before the first step: ppml_local_reduce(g, u0, red), the all-reduce, and
 * ppml_apply_reduced(g, red, 0, 0) set the first CFL step.  dt > 0: that step for every
 * call of the step; dt <= 0: the device-resident step.  The states then equal a single grid's
 * bit for bit (every cell takes the same operations on the same values; the CFL step comes
 * from the same maxima); the sums differ only in the order of addition.  Grids with halo
 * faces are refused by ppml_step, ppml_step_phi, ppml_step_noalloc, the Poisson solves and
 * ppml_grid_tune, which step through the handle's own U* (it has no halo planes).
 * red: PPML_REDUCE_LEN device doubles, caller-owned: max|v|, max c, the six FP64 sums
 * (times the cell volume), the counts of vacuum-branch and of non-physical cells.
 *   ppml_local_reduce      red of the state u's cells (this slab's), asynchronous
 *   ppml_lagrangian_stage  S5-S8 from the caller's U* (rho in u_star->f[0], as
 *                          ppml_eulerian_stage writes it) into u_out, and red of u_out;
 *                          does not advance the handle's time; asynchronous
 *   ppml_apply_reduced     the handle's scalars (t, steps, maxima, sums, flags, next CFL
 *                          step) from an all-reduced red; advance != 0 adds the step of
 *                          size dt (dt <= 0: the device-resident step); asynchronous */
#define PPML_HALO_PLANES 3
#define PPML_REDUCE_LEN 10
int ppml_local_reduce(ppml_grid* g, const ppml_state* u, double* red, void* stream);
int ppml_lagrangian_stage(ppml_grid* g, const ppml_state* u_star, ppml_state* u_out, double dt,
                          double* red, void* stream);
int ppml_apply_reduced(ppml_grid* g, const double* red, int advance, double dt, void* stream);

/* Only the Eulerian stage (S0-S3): writes U* (rho copied, m, rho E, rho eps updated; with
 * their low parts for double-float states) into u_star.  The stage does not change rho:
 * u_star->f[0] (and lo[0]) may be u_in's, and is then left as it is.  Used for stage-level
 * checks and by the z-slab decomposition; same dt convention as ppml_step; does not
 * advance t. */
int ppml_eulerian_stage(ppml_grid* g, const ppml_state* u_in, ppml_state* u_star, double dt,
                        void* stream);

/* FP64 sums of each field of u times the cell volume.  Synchronizes the stream. */
int ppml_conserved_sums(ppml_grid* g, const ppml_state* u, double out[6], void* stream);

/* Copy the device-resident diagnostics to the host.  Synchronizes the stream.  Returns
 * PPML_E_NONPHYSICAL (with *out filled) if PPML_FLAG_NONPHYSICAL is set. */
int ppml_read_diag(ppml_grid* g, ppml_diag* out, void* stream);

/* Device address of the handle's current step size (one double). */
const double* ppml_dt_device(const ppml_grid* g);

/* Measurement hook (not part of the paper's method).  enable != 0: every following
 * ppml_step records CUDA events on its stream around each of its kernels (Eulerian,
 * Lagrangian, finalize) and accumulates their durations; enable == 0 stops recording.
 * Do not enable while capturing a CUDA graph.  Resets the accumulated times. */
int ppml_profile(ppml_grid* g, int enable);

/* Accumulated kernel durations in milliseconds (ms[0] Eulerian, ms[1] Lagrangian,
 * ms[2] finalize) and the number of profiled steps.  Synchronizes the device. */
int ppml_kernel_times(ppml_grid* g, double ms[3], long long* steps);

/* ------------------------------------------------------------ step without allocation
 * The paper has no counterpart to this call: it exists for callers that cannot call
 * cudaMalloc -- code running while another part of the process captures a CUDA graph
 * (allocation is not permitted then), plugins whose host application owns the device
 * memory budget, real-time loops that must not allocate.  It performs the same step as
 * ppml_step (same kernels) without a handle: U*, the reduction partials and the step
 * scalars live in a fixed device buffer inside libppml.so sized for grids of at most
 * PPML_NOALLOC_MAX_CELLS cells (about 12 MB, held on every GPU that loads the library
 * until the process exits).  Nothing is allocated by the call (no cudaMalloc/cudaFree).
 *   d         the problem statement (as for ppml_init_grid); nx*ny*nz above the limit
 *             returns PPML_E_INVAL; d->t_end must be 0 (the call keeps no simulated time,
 *             so there is nothing to clip the step against)
 *   u_in      input state, not modified; u_out output state (no aliasing); plain float
 *             or double states only (low parts are PPML_E_INVAL here); grids with
 *             PPML_BC_INFLOW faces are PPML_E_INVAL (their states live in a grid handle)
 *   dt        step size, > 0 (there is no device-resident step here)
 *   rho_mean  mean initial density, > 0 (reference of the vacuum threshold)
 *   out       NULL, or nine doubles receiving the CFL step of u_out, max|v|, max c and the
 *             six FP64 sums of u_out; non-NULL synchronizes the stream, and only then are
 *             non-physical output cells reported (PPML_E_NONPHYSICAL, out still filled)
 * The first call on a device looks up the buffer's device address (cudaGetSymbolAddress)
 * and sets the kernels' shared-memory limits; make it before any stream capture.  Every
 * call shares the one buffer, which keeps the last call's contents: calls that overlap on
 * the GPU (unordered streams or host threads) race on it. */
#define PPML_NOALLOC_MAX_CELLS 262144
int ppml_step_noalloc(const ppml_grid_desc* d, const ppml_state* u_in, ppml_state* u_out,
                      double dt, double rho_mean, double out[9], void* stream);

/* ---------------------------------------------------------------- batched 1D problems
 * Many independent 1D problems of uneven lengths (outflow boundaries, gamma shared),
 * advanced by one persistent launch per call.  Each instance keeps its own time, CFL
 * step and end time.  Packed layout: four device arrays (rho, m, rho E, rho eps) of
 * sum(ncells) elements of the batch's type, instance i at [offset_i, offset_i + n_i).
 * An FP32 batch stepped with low-part arrays holds rho, m and rho E as double-float pairs
 * (the stencils read the high parts; updates and the Sec. 1.4 difference use both; the
 * low parts live in three more caller arrays between calls).  An instance
 * whose state has a cell with rho <= 0, rho eps <= 0 or a non-finite value stops there
 * (no further step) and is flagged PPML_FLAG_NONPHYSICAL. */
typedef struct ppml_batch ppml_batch;

/* ncells[n_inst] (each >= 4), h[n_inst] (> 0), t_end[n_inst] (> 0) are host arrays;
 * they are copied.  vacuum_frac <= 0 selects 1e-5 (reference: each instance's own mean
 * initial density, computed at the first ppml_batch_step).  Every instance must fit in
 * one CTA's shared memory: a one-CTA instance of n cells needs 4 (n + 6) + 4 (n + 1) floats
 * in FP32 (7 (n + 6) + 4 (n + 1) with low parts), 4 (n + 6) + 2 (n + 1) doubles in FP64,
 * plus 1 KB, within the device's opt-in limit (on GB300 up to 7228 FP32, 5255 FP32 with
 * low parts, or 4817 FP64 cells); a paired instance (see ppml_batch_set_split) needs the
 * same for m = ceil(n / 2) with 4 (m + 12) + 4 (m + 8) floats (7 (m + 12) + 4 (m + 8) with
 * low parts) or 4 (m + 12) + 2 (m + 8) doubles; else PPML_E_INVAL (for the low parts, at
 * the ppml_batch_step that passes them). */
int ppml_batch_init(int n_inst, const int* ncells, const double* h, const double* t_end,
                    double gamma, double cfl, double vacuum_frac, int dtype, ppml_batch** out);

/* Advance every unfinished instance by up to max_steps steps (each instance stops at its
 * t_end) in one launch.  state: four device pointers (see layout), updated in place.
 * lo: NULL (plain float or double state), or (FP32 only) three device arrays of the state's
 * layout with the low parts of rho, m, rho E: a double-float state, read at the start and
 * written at the end of the call (zero them, or set them to x - (float)x of an FP64 x,
 * before the first call).  If done_host is non-NULL the stream is synchronized, the
 * number of instances that reached their t_end is written there, and PPML_E_NONPHYSICAL is
 * returned if some instance stopped on a non-physical state (ppml_batch_status names them);
 * with done_host NULL the call is asynchronous and reports nothing about the states. */
int ppml_batch_step(ppml_batch* b, void* const state[4], void* const lo[3], int max_steps,
                    int* done_host, void* stream);

/* Launch shape of the batch (the paper has no counterpart: a systems choice).  Each
 * instance is one CTA of 256, 512 or 1024 threads; ppml_batch_init selects 512.
 * ppml_batch_set_threads fixes the size (PPML_E_INVAL for any other value).
 * ppml_batch_tune times each size for trial_steps steps (>= 1) of the given state, the
 * fastest of two runs each, on scratch copies of the state and of the instances' times
 * (the caller's state and the batch's progress are unchanged), keeps the fastest and
 * returns it in *threads_out (may be NULL) and the three times in ms_out[3] (may be NULL).
 * Allocates and frees scratch of one state; synchronizes the stream.  Results of a step
 * do not depend on the size in FP64 (the same operations per cell in the same order). */
int ppml_batch_set_threads(ppml_batch* b, int threads);
int ppml_batch_tune(ppml_batch* b, void* const state[4], int trial_steps, int* threads_out,
                    double ms_out[3], void* stream);

/* Instances of at least min_cells cells (min_cells >= 64) are each split over the two CTAs
 * of one thread-block cluster, half of the cells each; the two exchange a 6-cell halo and
 * their CFL maxima through distributed shared memory once per step, so the longest runs
 * use two SMs.  The launch is then one grid of two-CTA clusters, each taking a split
 * instance or two whole instances of neighbouring sizes (one per CTA), largest first.
 * min_cells = 0: no split (one CTA per instance).  ppml_batch_init selects
 * max(1024, ceil(7 largest / 8)).  Results do not depend on the split (the same operations
 * per cell, in the same order).  The new work plan goes to new device buffers (host to
 * device copy) and applies to later ppml_batch_step calls; launches already queued and
 * CUDA graphs captured before keep the plan they were launched with (its buffers live until
 * ppml_batch_free).  PPML_E_INVAL for 0 < min_cells < 64 or if an instance would not fit
 * (the previous split is kept). */
int ppml_batch_set_split(ppml_batch* b, int min_cells);

/* The work plan of a batch of n_inst instances of ncells[i] cells for a split threshold
 * split_min (0, or >= 64), as ppml_batch_init / ppml_batch_set_split build it; host only,
 * no device call.  If some instance has at least split_min cells, *n_items work items of
 * two ints are written to items (room for 2 n_inst ints), largest first by the size of the
 * item's largest instance: (a, -2) is instance a split over a CTA pair, (a, b) runs
 * instances a and b on the two CTAs of a cluster (b = -1: none), whole instances paired in
 * order of size.  Otherwise *n_items = 0 and, if order is non-NULL, order (n_inst ints)
 * receives the instances largest first (one CTA each).  Ties keep the instances' order. */
int ppml_batch_plan(int n_inst, const int* ncells, int split_min, int* items, int* n_items,
                    int* order);

/* Per-instance time reached, steps taken and flags (PPML_FLAG_NONPHYSICAL for an instance
 * stopped on a non-physical state); host arrays of n_inst, each may be NULL.  Synchronizes.
 * Returns PPML_E_NONPHYSICAL (arrays still filled) if some instance is flagged. */
int ppml_batch_status(ppml_batch* b, double* t_host, int* steps_host, unsigned* flags_host,
                      void* stream);

int ppml_batch_free(ppml_batch* b);

/* ---------------------------------------------------------------- measurement aid
 * Fused multiply-add throughput of the current device for dtype PPML_F32 or PPML_F64
 * (the paper has no counterpart: the denominator of the arithmetic rooflines).  Launches a
 * kernel of 8 CTAs of 256 threads per SM, each thread running 8 independent FMA chains for
 * `iters` (>= 1) iterations without memory traffic, once untimed and once timed with CUDA
 * events on `stream`; writes the FMAs per second of the timed launch (an FMA counted once)
 * to *fma_per_s.  Allocates and frees one scratch array; synchronizes the stream. */
int ppml_fma_peak(int dtype, int iters, double* fma_per_s, void* stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* ppml_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PPML_H */
