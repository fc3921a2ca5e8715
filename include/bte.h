/*
 * bte.h -- C ABI of libbte, a GB300 (sm_103a) solver for the hot path of the
 * non-gray phonon Boltzmann transport equation of arXiv:2305.19400, Sec. 3.
 *
 * What one call of bte_step computes (Sec. 3.1, Eq. 4-6, and the temperature
 * update of Sec. 2.2/3.2): for every cell P, direction d and band-polarisation b
 * the finite-volume update of the intensity I[P][d][b] -- upwind face fluxes
 * plus relaxation toward the band equilibrium intensity I0_b(T) -- with wall
 * ghosts from Eq. 6, then the per-cell reduction over (d, b) to an energy, the
 * nonlinear temperature solve and the I0 refresh.  Every step runs as CUDA
 * kernels on the caller's stream; nothing runs on the host between launches.
 *
 * Conventions for every entry point:
 *  - Return value: BTE_OK (0) or a negative BTE_E_* code; BTE_W_FALLBACK (+1)
 *    is success with at least one bisection fallback in a temperature solve.
 *    The library never exits, aborts or traps the device.  bte_last_error()
 *    gives a one-line message for the last failing call on that handle.
 *  - Pointers documented as "host" are read (or written) during the call and
 *    stay owned by the caller.  Pointers documented as "device" are CUDA
 *    device pointers on the device that was current at bte_init_mesh.
 *  - Call order: bte_init_mesh -> bte_set_bands -> [bte_bind_workspace] ->
 *    bte_set_bc (every side of every geometry) -> bte_set_initial (every
 *    geometry) -> bte_step / bte_get_* any number of times -> bte_destroy.
 *    Anything else returns BTE_E_STATE.
 *  - Handles are not thread-safe; use one handle per host thread.
 */
#ifndef BTE_H
#define BTE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define BTE_OK 0
#define BTE_E_ARG (-1)       /* bad argument (null pointer, size, index, value) */
#define BTE_E_STATE (-2)     /* call out of order */
#define BTE_E_CUDA (-3)      /* a CUDA runtime call failed (message names it) */
#define BTE_E_NOMEM (-4)     /* workspace too small or device allocation failed */
#define BTE_E_NONFINITE (-5) /* a cell energy or temperature became NaN/Inf */
#define BTE_E_TIMEOUT (-6)   /* reserved for a bounded device-side wait that gave up; no kernel of this
                              * library waits on another, so no call returns it */
#define BTE_E_EXCHANGE (-7)  /* the band-range exchange callback returned non-zero */
#define BTE_W_FALLBACK 1     /* success; some temperature solves fell back to bisection */

/* ---- enumerations ---- */
enum { BTE_DIRS_INPLANE = 0, BTE_DIRS_POLAR_AZIM = 1 };
enum { BTE_FP64 = 0, BTE_FP32 = 1, BTE_BF16 = 2 };
enum { BTE_BC_ISOTHERMAL = 0, BTE_BC_SPECULAR = 1, BTE_BC_DIFFUSE = 2, BTE_BC_PARTIAL = 3,
       BTE_BC_ROTATIONAL = 4 /* unstructured meshes only (bte_umesh.h) */ };
enum { BTE_IMPLICIT_JACOBI = 0, BTE_EXPLICIT = 1, BTE_IMPLICIT_GS = 2 };
enum { BTE_T_PSEUDO = 0, BTE_T_LATTICE = 1, BTE_E_LATTICE = 2 };

typedef struct bte_ctx* bte_handle;

/* One structured Cartesian geometry.  dim = 2 (nz must be 1) or 3.  Cell sizes
 * in metres.  Cell (i,j,k) has local index i + nx*(j + ny*k). */
typedef struct {
  int dim, nx, ny, nz;
  double dx, dy, dz;
} bte_geom;

/* Solver options (bte_default_opts fills the defaults shown).
 *  dir_kind   BTE_DIRS_INPLANE: n_inplane directions in the x-y plane
 *             (phi_d = (d+1/2) 2 pi/n, n % 4 == 0; Sec. 3.1 uses 16-20);
 *             BTE_DIRS_POLAR_AZIM: n_polar x n_azim control angles
 *             (n_polar even, n_azim % 4 == 0; 20 x 20 = 400 in Sec. 3.1).
 *             At most 2048 directions (the sweep keeps the direction table
 *             in shared memory); more return BTE_E_ARG.
 *  precision  storage of I and the sweep arithmetic: BTE_FP64 (default),
 *             BTE_FP32 or BTE_BF16 (FP32 arithmetic); the reduction, the
 *             temperature solve and I0 are FP64 in every mode.
 *  learned    0 (default): cells the cached-model solve cannot settle start
 *             their exact solve from the model root, or from their previous
 *             T_p when the model has no root in [1, 5000] K; 1: in the second
 *             case they start from the trained networks' guess instead (net
 *             A: E_p -> T, then surrogate Newton steps on net B: T -> I0_b)
 *             before the exact FP64 refinement (a model root is the closer
 *             start whenever there is one).  bte_solve_T takes the networks'
 *             guess for every energy.  Requires bte_train_mlp before the
 *             first bte_step.
 *  n_gauss    Gauss-Legendre points per band for I0_b(T) (default 16, <= 32).
 *  newton_rtol target relative accuracy of the temperature solve (1e-14).
 *  newton_maxit iteration cap before the bisection fallback (50).
 *  cuda_stream cudaStream_t every launch and copy uses (NULL: legacy default stream).
 *  T_ref      reference temperature of the FP32/BF16 modes, which store the
 *             deviation I - I0_b(T_ref), and of beta_T_exp (default 300 K).
 *  use_graph  1: each time step's ninner sweep launches are captured once in a
 *             CUDA graph (per scheme, ninner and buffer rotation) and replayed
 *             on cuda_stream; 0 (default): launched one by one.
 *  autotune   1: the first bte_step runs bte_autotune (default 0).
 *  beta_T_exp temperature dependence of the relaxation rates (Sec. 2.2: tau
 *             depends on T; the paper gives no law): beta_b(T) = beta_b
 *             (T_p / T_ref)^beta_T_exp per cell, T_p the cell's current
 *             pseudo-temperature, beta_b the table value (at T_ref).  0
 *             (default) keeps tau fixed; |beta_T_exp| <= 16.  The factor is
 *             common to all bands, so the T_p equation keeps its root.
 *  fp64_strict BTE_FP64 only.  0 (default): the implicit point-Jacobi sweep
 *             (any ninner) of a handle with fixed relaxation rates and
 *             isothermal or mirror walls keeps the intensity in double-float
 *             form (two floats, 48-bit significand) and computes the update on
 *             the FP32 pipe with error-free transformations; the reduction,
 *             the temperature solve and I0 stay IEEE FP64.  Between such steps
 *             the intensity stays in that form; every call that reads or
 *             writes intensities (bte_get_intensity, bte_set_intensity,
 *             bte_get_flux, bte_get_wall_flux_noalloc, bte_set_initial) or
 *             steps another way converts it to FP64 in place first (one
 *             kernel).  The update rounds to about 2^-48 relative instead of
 *             2^-53, for |I| in [2^-74, 2^127) (smaller values keep a float's
 *             24 bits).  1: every update in IEEE FP64 arithmetic (DFMA). */
typedef struct {
  int dir_kind;
  int n_inplane, n_polar, n_azim;
  int precision;
  int learned;
  int n_gauss;
  double newton_rtol;
  int newton_maxit;
  void* cuda_stream;
  double T_ref;
  int use_graph;
  int autotune;
  double beta_T_exp;
  int fp64_strict;
} bte_opts;

/* Per-call statistics of bte_step (filled only when a non-NULL pointer is
 * passed; that makes the call wait for the stream to finish). */
typedef struct {
  long long updates;          /* cell*dir*band updates performed */
  long long solve_evals;      /* band-quadrature evaluations in temperature solves */
  long long solves;           /* temperature solves (cells x inner iterations) */
  long long fallbacks;        /* bisection fallbacks */
  long long nonfinite;        /* cells whose energy or temperature was not finite */
  int launches;               /* kernels launched by the call */
  double gpu_ms;              /* device time between the first and last launch */
} bte_stats;

/* Fills *opts with the defaults listed above (the discretisation choices of
 * Sec. 3.1: direction set, band quadrature, precision).  Returns BTE_E_ARG on
 * NULL. */
int bte_default_opts(bte_opts* opts);

/* Creates a solver for n_geom >= 1 independent geometries sharing one
 * direction set and band table (Sec. 3.1 discretisation); all of them 2-D or
 * all 3-D (a mixture returns BTE_E_ARG).  geoms: host array
 * of n_geom.  opts: host, may be NULL for defaults.  *out receives the handle
 * (NULL on failure).  No device memory is allocated yet. */
int bte_init_mesh(bte_handle* out, int n_geom, const bte_geom* geoms, const bte_opts* opts);

/* Band-polarisation table (Sec. 3.1: 40 bands -> 55 band-polarisations).
 * Host arrays of nb values: band edges omega_lo < omega_hi [rad/s], group
 * velocity vg > 0 [m/s], scattering rate beta = 1/tau >= 0 [1/s], degeneracy
 * > 0.  I0_b(T) = g_b hbar/(8 pi^3 v_b^2) int w^3/(exp(hbar w/kB T)-1) dw over
 * the band (Debye-type band, Bose-Einstein occupation).  1 <= nb <= 256. */
int bte_set_bands(bte_handle h, int nb, const double* omega_lo, const double* omega_hi, const double* vg,
                  const double* beta, const double* degeneracy);

/* Band partition (Sec. 3.3: the bands couple only through the temperature
 * update, which needs a per-cell sum over bands).  After bte_set_bands and
 * before any call that needs device memory (bte_bind_workspace,
 * bte_workspace_bytes, bte_set_bc, bte_set_initial), bte_set_band_range makes
 * this handle store and sweep only bands [band_lo, band_hi) of the table; the
 * temperature solve still uses every band.  Each inner iteration then runs
 * sweep -> exchange -> cell solve -> fix-up: the sweep writes this handle's
 * per-cell partial sums (E_L, E_p) over its bands, and the callback given to
 * bte_set_exchange must replace them by their sum over all ranks' band ranges
 * (an all-reduce), after which every rank solves the same T_p for every cell.
 * The ranges of the ranks must tile [0, nb) and every rank must use the same
 * mesh, directions, table, walls, initial state, dt and options.
 *   fn(buf, count, cuda_stream, user): buf is a device array of count
 *   (= 2 * total cells) doubles, [cell][E_L, E_p]: the caller's dev_buf when
 *   that is not NULL (device memory of at least 2 * total cells doubles that
 *   stays alive while the handle steps), else an array inside the library's
 *   workspace.  The partials are complete in stream order on cuda_stream (a
 *   cudaStream_t) when fn is called, and fn must leave the sums in buf in that
 *   stream's order (it may synchronize the stream).  fn returns 0 on success;
 *   any other value makes bte_step return BTE_E_EXCHANGE.  `user` is passed
 *   through.  The library calls fn from the thread that called bte_step.
 * A band-range handle steps without CUDA graphs (opts.use_graph is ignored),
 * bte_step returns BTE_E_STATE until an exchange is set, bte_get_flux and
 * bte_get_wall_flux_noalloc return the partial sums over this handle's bands,
 * bte_get_intensity / bte_set_intensity cover [cell][dir][band_lo..band_hi),
 * and bte_set_intensity needs Tp_cells (E_L comes from the next step's sums).
 * bte_set_band_range returns BTE_E_ARG unless 0 <= band_lo < band_hi <= nb. */
typedef int (*bte_allreduce_fn)(double* dev_buf, long long count, void* cuda_stream, void* user);
int bte_set_band_range(bte_handle h, int band_lo, int band_hi);
int bte_set_exchange(bte_handle h, bte_allreduce_fn fn, void* user, double* dev_buf);

/* Device bytes the solver needs (valid after bte_set_bands), and binding of a
 * caller-owned device buffer of at least that size (e.g. a torch.empty
 * uint8 tensor).  The buffer holds the discretised state of Sec. 3.1-3.2:
 * the intensity I_{d,b} of every cell (the unknown of Eq. 4-5, three
 * buffers for I^n, the iterate and the next iterate), the per-cell mutable
 * variables I0_b and T of Sec. 3.2, the wall ghosts of Eq. 6 and the
 * coefficient tables of Eq. 5's volume and surface terms.  The buffer must stay alive until bte_destroy; the library
 * never frees it.  Without a bound buffer the library cudaMallocs its own at
 * the first call that needs device memory and frees it in bte_destroy.
 * bte_bind_workspace returns BTE_E_NOMEM if bytes is too small, BTE_E_STATE
 * after device memory is already in use. */
size_t bte_workspace_bytes(bte_handle h);
int bte_bind_workspace(bte_handle h, void* dev_ptr, size_t bytes);

/* Wall condition of one side (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z) of geometry
 * `geom` (Eq. 6).  BTE_BC_ISOTHERMAL: ghost intensity I0_b(T_face); T_faces is
 * a host array with one temperature per face on that side (x sides: j+ny*k,
 * y sides: i+nx*k, z sides: i+nx*j) or NULL to use T_uniform for all.
 * BTE_BC_SPECULAR (symmetry): ghost = same cell, mirrored direction.
 * BTE_BC_DIFFUSE (a rough wall; an extension beyond Eq. 6): every incoming
 * direction of band b gets sum_out |S_d.n| I_d,b / sum_in |S_d.n| of the wall
 * cell's current iterate (out: moving into the wall), so the wall returns
 * each band's whole energy flux isotropically.  T_faces and T_uniform are
 * ignored for it. */
int bte_set_bc(bte_handle h, int geom, int side, int type, const double* T_faces, double T_uniform);

/* Makes one side partially specular (BTE_BC_PARTIAL; an extension beyond
 * Eq. 6): every incoming direction d of band b gets
 *   p x I_{mirror(d),b} + (1 - p) x sum_out |S.n| I_b / sum_in |S.n|
 * of the wall cell's current iterate, i.e. a fraction p of the energy
 * reflected as by a mirror and the rest as by a diffuse wall; p = 1 is
 * BTE_BC_SPECULAR, p = 0 BTE_BC_DIFFUSE.  0 <= p <= 1, else BTE_E_ARG.  The
 * side's ghost rows (faces x directions x bands in the storage type) are
 * allocated with cudaMalloc outside any bound workspace (BTE_E_NOMEM on
 * failure) and refreshed by one kernel before every sweep. */
int bte_set_specularity(bte_handle h, int geom, int side, double p);

/* Equilibrium initial state (Sec. 3.2): I[P][d][b] = I0_b(T_P) for all d and
 * T_p = T_L = T_P.  T_cells: host array of the geometry's cells, or NULL for
 * T_uniform everywhere.  Temperatures must lie in [1, 5000] K. */
int bte_set_initial(bte_handle h, int geom, const double* T_cells, double T_uniform);

/* Advances every geometry by nsteps time steps of size dt [s].
 * scheme BTE_IMPLICIT_JACOBI: backward Euler, each step solved by ninner
 *   point-Jacobi inner iterations; each inner iteration is one sweep
 *   I^{k+1} = [I^n/dt + beta I0^k + v sum_ax c_ax I_up^k]/[1/dt + beta + v sum_ax c_ax]
 *   (c_ax = |S_ax|/(w_d Delta_ax)), then reduction, T_p solve, I0 refresh.
 * scheme BTE_EXPLICIT: forward Euler (Eq. 3 with Eq. 5), ninner ignored.
 * scheme BTE_IMPLICIT_GS (every storage precision): backward Euler
 *   with sweep-ordered (Gauss-Seidel) inner iterations, an extension beyond
 *   the paper's point-Jacobi form: each (d, b) visits the cells in its upwind
 *   order, so an interior upwind neighbour holds its value of the current
 *   inner iteration; mirror and diffuse wall ghosts and I0 stay at I^k.  The
 *   fixed point is the same backward-Euler solution; fewer inner iterations
 *   reach a given residual.  Two kernels per inner iteration (the pass, then
 *   the per-cell reduction and T_p step), plus one with beta_T_exp != 0.
 * stats: host, may be NULL (then the call only queues work and returns). */
int bte_step(bte_handle h, double dt, int nsteps, int ninner, int scheme, bte_stats* stats);

/* Times the sweep over candidate launch shapes (directions per team step:
 * the default and half of it; cells per CTA; grid size, persistent grids of
 * 2/4 CTAs per SM or one CTA per work item; 2 or 3 CTAs per SM) with the
 * current state and keeps the fastest for this handle.  With scheme
 * BTE_IMPLICIT_GS it times the sweep-ordered pass instead, over directions
 * per CTA and the column-tile size.  The timing launches write only a spare
 * intensity buffer (no solver state changes).  `report` (host, may be NULL)
 * receives a CSV table of the candidates. */
int bte_autotune(bte_handle h, double dt, int scheme, char* report, size_t report_len);

/* Cell temperatures of one geometry (Sec. 3.1: temperature is derived from
 * the intensity summed over all directions and bands; Sec. 2.2 and 3.2: the
 * per-cell temperature update after each step, which sets I0_b and tau_b):
 * BTE_T_PSEUDO (T_p, the temperature whose equilibrium I0_b(T_p) the
 * relaxation term of Eq. 4 drives toward: sum_b W beta_b I0_b(T_p)/v_b =
 * sum_b beta_b G_b/v_b) or BTE_T_LATTICE (T_L, the energy-equivalent
 * temperature: sum_b W I0_b(T_L)/v_b = sum_b G_b/v_b), G_b = sum_d w_d I_{d,b};
 * or, with which = BTE_E_LATTICE, the right-hand side of the T_L equation
 * itself, E_L = sum_b G_b/v_b, the cell's energy density (J/m^3) after the
 * last inner iteration (what Sec. 2.2's first-law temperature update works
 * from; cell volume times E_L summed over cells is the stored energy).  out: ncells doubles, host or device
 * (out_on_device != 0).  Waits for the stream. */
int bte_get_T(bte_handle h, int geom, int which, double* out, int out_on_device);

/* Heat flux of one geometry: the energy flux carried by the intensity, i.e.
 * the surface term of Eq. 5 (|v_g|_b times the integral of I_{d,b} s_d . n
 * over the cell boundary, summed over d and b) evaluated per cell and per
 * wall.  q_cells: ncells*dim doubles, q(P) = sum_b sum_d
 * S_d I[P][d][b] (W/m^2), or NULL.  q_walls: 2*dim doubles, per side the mean
 * over its faces of sum_b sum_d (S_d . n_out) I_face (upwind face value,
 * ghost for incoming directions; positive = leaving), or NULL.  Host or
 * device per out_on_device.  Waits for the stream. */
int bte_get_flux(bte_handle h, int geom, double* q_cells, double* q_walls, int out_on_device);

/* Copies the intensity I_{d,b} of one geometry (the unknown of Eq. 4-5,
 * indexed as in Sec. 3.1) out as FP64 [cell][dir][band]
 * (ncells*nd*nb doubles, unpadded), host or device. */
int bte_get_intensity(bte_handle h, int geom, double* out, int out_on_device);

/* Replaces the intensity of one geometry with `in` (FP64 [cell][dir][band],
 * host or device per in_on_device) and sets T_p to Tp_cells (host/device,
 * ncells) -- a checkpoint restore, i.e. an arbitrary initial condition in
 * place of the equilibrium one of Sec. 3.2.  I0 is recomputed from T_p (the
 * per-cell variable of Sec. 3.2 that depends on temperature). */
int bte_set_intensity(bte_handle h, int geom, const double* in, const double* Tp_cells, int in_on_device);

/* Direction table the solver uses (the discrete direction vectors s_d of
 * Sec. 3.1 and the reflection index r of Eq. 6): S (nd*3, control-angle
 * integrals of the unit vector), w (nd, solid angles), refl (3*nd, mirror direction across an
 * x, y, z wall).  Host arrays; any may be NULL.  Returns nd (>0) or an error. */
int bte_get_directions(bte_handle h, double* S, double* w, int* refl);

/* Per-side mean outgoing wall flux of one geometry (the q_walls of
 * bte_get_flux), computed without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * -- processes with a fixed device-memory budget or whose device memory is
 * owned by another allocator, and latency-critical loops where an allocation
 * would synchronize the device.  Its per-face scratch is a static device array
 * inside libbte.so (65536 doubles + 8, about 512 KB, held by every GPU that
 * loads the library until the process exits), so a wall may have at most
 * 65536 faces (larger walls return BTE_E_ARG).  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, once per
 * device); make that first call before any stream capture.  All calls share
 * the array, which keeps the last call's contents; every face slot is written
 * before it is read, so nothing needs clearing, but calls that overlap on the
 * GPU (other streams, other host threads) race on it.  q_walls: 2*dim doubles,
 * host or device per out_on_device.  Waits for the handle's stream. */
int bte_get_wall_flux_noalloc(bte_handle h, int geom, double* q_walls, int out_on_device);
/* (FP64-mode handles only; other precisions return BTE_E_ARG.) */

/* Learned temperature / equilibrium guess (the path's pattern (4)): trains
 * two 1-64-64-k tanh networks with FP32 weights on the device -- net A maps
 * the normalised scattering-weighted energy E_p to T, net B maps T to the 55
 * (nb) normalised ratios I0_b(T)/I0_b(T_ref) -- on n_pairs samples of T
 * uniform in [T_lo, T_hi] K labelled by the library's FP64 band quadrature;
 * `epochs` passes of Adam (minibatch 1024, learning rate 2e-3 decaying to
 * 2e-4).  Forward, backward and update run in the library's kernels; training
 * allocates its sample and activation buffers stream-ordered on cuda_stream
 * and frees them before returning.  loss (host, may be NULL): 2 doubles, the
 * final mean squared error of nets A and B in normalised units.
 * 1024 <= n_pairs <= 2^26, 1 <= T_lo < T_hi <= 5000, epochs >= 1. */
int bte_train_mlp(bte_handle h, long long n_pairs, double T_lo, double T_hi, int epochs, unsigned long long seed,
                  double* loss);

/* Parameters of net 0 (A) or 1 (B) as FP32 host arrays in the layout
 * W1[64], b1[64], W2[64][64], b2[64], W3[k][64], b3[k] (k = 1 or nb).
 * bte_mlp_params returns the parameter count (out may be NULL to query it). */
int bte_mlp_params(bte_handle h, int net, float* out, int n);
int bte_mlp_set_params(bte_handle h, int net, const float* in, int n);

/* Mean squared error and its gradient for net 0/1 on n samples (host arrays):
 * x[n] inputs, y[k][n] targets (sample index fastest), grad in the parameter
 * layout, loss (may be NULL).  Uses the same device kernels as training. */
int bte_mlp_grad(bte_handle h, int net, const float* x, const float* y, int n, float* grad, double* loss);

/* Solves sum_b W beta_b I0_b(T)/v_b = Ep[i] for n energies (host arrays),
 * starting from T0[i] (or 300 K when T0 is NULL) or, with learned = 1, from
 * the trained networks' guess; exact FP64 Halley refinement to the solve
 * tolerance, bisection fallback.  T_out[i] (NaN when no root lies in
 * [1, 5000] K) and evals[i] (exact quadrature evaluations; may be NULL). */
int bte_solve_T(bte_handle h, const double* Ep, const double* T0, int n, int learned, double* T_out, int* evals);

/* Per-launch device time of the sweeps (the paper has no counterpart; it
 * serves the roofline of the sweep kernel).  bte_set_sweep_timing(h, 1) makes
 * every later bte_step record a CUDA event before and after each inner
 * iteration's sweep launch (for BTE_IMPLICIT_GS: the pass and its per-cell
 * step) on the solver's stream; with use_graph the events are recorded by
 * nodes of the step's graph.  Switching it drops the handle's graphs.
 * bte_sweep_times waits for the last event and writes the durations (ms) of
 * the sweeps of the most recent time step, in inner-iteration order, to
 * ms[0 .. n); it returns how many sweeps that step had (ms may be NULL when
 * n = 0), or BTE_E_STATE when no step ran since timing was switched on. */
int bte_set_sweep_timing(bte_handle h, int on);
int bte_sweep_times(bte_handle h, float* ms, int n);

/* Measured arithmetic peak of the current device (the roofline denominators of
 * the sweeps; the paper has no counterpart).  kind BTE_PEAK_FP64_FMA: FP64
 * fused multiply-adds (the FP64 sweep's pipe); BTE_PEAK_FP32X2_FMA: packed
 * two-float FMAs (the pipe of the double-float sweep and the reduced modes).
 * Loop kernels of independent FMA chains on 8 CTAs of 256 threads per SM,
 * about 30 ms each, timed with CUDA events on a stream of their own; the best
 * of three timed launches after one warm-up.  *flops receives flop/s (2 per
 * FMA), *ms (may be NULL) that launch's time.  The figure scales with the SM
 * clock of the moment; the caller samples it.  Allocates no memory on the
 * device; runs on the current device and waits for its own stream.  Returns
 * BTE_E_ARG for an unknown kind or NULL flops, BTE_E_CUDA on a CUDA error. */
enum { BTE_PEAK_FP64_FMA = 0, BTE_PEAK_FP32X2_FMA = 1 };
int bte_measure_peak(int kind, double* flops, double* ms);

/* Frees everything the library allocated (not a bound workspace).  The
 * paper has no counterpart (resource release of this library's handle). */
int bte_destroy(bte_handle h);

/* Last error message of the handle ("" if none); h may be NULL for errors
 * from bte_init_mesh.  The paper has no counterpart (error reporting of this
 * library).  The string lives until the next call on the handle. */
const char* bte_last_error(bte_handle h);

#ifdef __cplusplus
}
#endif
#endif /* BTE_H */
