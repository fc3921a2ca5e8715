// bte_internal.h -- definitions shared by the library's own translation units.
//
// Device data layout (all in one workspace, see bte_capi.cu):
//   I buffers      3 x [cell][dir][nbp]      storage type per precision mode
//                                            (FP32/BF16 store I - I0_b(T_ref))
//   I0cell         [cell][nbp]  double        I0_b(T_p) of every cell
//   J, Teval       [cell][3][nbp], [cell]     cached quadrature model per cell
//   Tp, TL, EL     [cell]       double        temperatures, lattice energy
//   I0wall         [wall face][nbp] double    Eq. 6 ghost for isothermal faces
//   coef           [class][5][dir][nbp] double  sweep coefficients (A_n, A_x, A_y, A_z, A_s)
//   node_c, node_C [nbp][ng]    double        Gauss nodes: hbar*omega/kB and weights
//   per-band / per-direction / per-geometry tables, work list, counters.
// nbp is nb rounded up to a multiple of 8, so one (cell, dir) row is a whole
// number of 16-byte vectors in every precision.  Padding bands carry zero
// coefficients and stay zero.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

struct bte_ctx;

namespace bte {

constexpr double kHbar = 1.054571817e-34;  // J s (CODATA 2018)
constexpr double kBoltz = 1.380649e-23;    // J/K (CODATA 2018, exact)
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxGauss = 32;
constexpr int kMaxBands = 256;
constexpr double kTmin = 1.0, kTmax = 5000.0;  // bracket of the temperature solves

enum Side { XLO = 0, XHI = 1, YLO = 2, YHI = 3, ZLO = 4, ZHI = 5 };

// One geometry as the kernels see it.
struct DevGeom {
  int nx, ny, nz, dim;
  long long cell0;        // global index of the first cell
  long long face0[6];     // first global wall-face row of each side (isothermal sides)
  int bc[6];              // 0 ghost row (isothermal, diffuse), 1 mirror, 3 per-direction ghost rows
  int cls;                // coefficient-table class (cells with equal dx, dy, dz)
  int pad;
  const void* gdir[6];    // bc 3 (partially specular): [side face][dir][nbo] ghosts, storage type
};

// A run of consecutive cells of one geometry processed by one CTA.
struct WorkItem {
  int geom;
  int cell_begin;  // local cell index
  int cell_count;
  int pad;
};

// Sweep-ordered (Gauss-Seidel) pass: one unit = the directions dir0 .. dir0+ndc-1
// of the octant list (all with the same upwind sides) over one geometry.
struct GsUnit {
  int geom;
  int dir0;  // first entry in SweepArgs::gs_dirs
  int ndc;   // directions in this unit (<= SweepArgs::gs_ndc)
  int pad;
};

// Per direction: bit a of `up` set when S_{d,a} > 0 (upwind neighbour on the low
// side along axis a); mirror directions across x, y, z walls.
struct DirInfo {
  int up;
  int rx, ry, rz;
};

// A cell whose temperature the sweep could not settle on its cached model.
struct FixItem {
  long long P;  // global cell
  double Ep;    // right-hand side of the T_p equation: sum_b beta_b G_b / v_b
  double T0;    // start temperature of the exact solve
  int model;    // 1: T0 is the cached model's root (a warm start); 0: the previous T_p
  int pad;
};

// Counters written by the kernels (atomics), read back for bte_stats.
struct DevCounters {
  unsigned long long evals;
  unsigned long long solves;
  unsigned long long fallbacks;
  unsigned long long nonfinite;
};

struct ThermoTables {
  const double* node_c;   // [nbp][ng] hbar*omega_i/kB (K)
  const double* node_C;   // [nbp][ng] I0_b(T) = sum_i node_C / expm1(node_c / T)
  const double* a_p;      // [nbp] W beta_b / v_b  (T_p equation weights)
  const double* a_L;      // [nbp] W / v_b         (T_L equation weights)
  const double* inv_v;    // [nbo] 1/v_b of the stored bands (0 on padding)
  const double* beta;     // [nbo] beta_b of the stored bands (0 on padding)
  int ng;
  int nbp;    // all bands, padded: width of node tables, J, a_p and a_L
  int nb;     // all bands
  int nbo;    // bands this handle stores (padded): width of I rows, I0cell, wall ghosts
  int nbr;    // bands this handle stores (real): stored band b < nbr is global band band0 + b
  int band0;  // global index of the first stored band (0 unless the handle owns a band range)
};

struct SweepArgs {
  const void* In;           // I^n   (storage type; deviation from I0ref in the reduced modes)
  const void* Ik;           // I^k   (== In for the explicit scheme)
  void* Iout;               // I^{k+1}
  void* Bout;               // FP64, bmode 1: receives B = A_n I^n (the inner-iteration invariant term)
  int bmode;                // FP64 implicit: 0 In is I^n; 1 In is I^n and B is written; 2 In holds B
  double* I0cell;           // [cell][nbp] in: I0^k, out: I0^{k+1}
  double* Tp;               // [cell] in/out
  double* Teval;            // [cell] evaluation point of the cached quadrature model
  double* J;                // [cell][3][nbp] I0, dI0/dT, d2I0/dT2 at Teval
  double* Msum;             // [cell][3] sum_b a_p,b J_k,b: the T_p model's sums, kept with J
  double* EL;               // [cell] out
  const double* I0wall;     // [face][nbp] FP64 ghosts
  const float* I0wall_dev;  // [face][nbp] FP32 ghosts minus I0ref (reduced modes)
  const double* I0ref;      // [nbp] I0_b(T_ref) (reduced modes)
  int ff;                   // FP64: 0 DFMA arithmetic (sweep_kernel); else the double-float sweep
                            // (sweep_ff_kernel; bit 0: In and I^k are ff pairs, bit 1: I^{k+1} and B
                            // are written as ff; B is always ff)
  // FP64 double-float sweep with factored coefficients (bte_sweep_ff.cuh), tables
  // in the double-float pair layout of bte_ff.cuh (h_b, h_b+1, l_b, l_b+1 per two bands):
  const void* coef_R;       // [cls][nd][nbp] R = 1/(1/(v_b dt) + beta_b/v_b + sum_ax c_ax,d)
  const float* band_ff;     // [2][nbp] 1/(v_b dt), beta_b/v_b of the stored bands (0 on padding)
  const float* dirc_ff;     // [cls][nd][3][2] c_ax,d as (h, l)
  const void* coef;         // FP64: [cls][5][nd][nbp] A_n, A_x, A_y, A_z, A_s;
                            // reduced: [cls][2][nd][nbp] float P, Q with
                            // I' = P I^n + Q (v_b sum_ax c_ax I_up + beta_b dI0)
  const float4* dirc;       // reduced: [cls][nd] (c_x, c_y, c_z, sum), c_ax = |S_d,ax|/(w_d Delta_ax)
  const float* vb32;        // [nbp] v_b (reduced)
  const float* bb32;        // [nbp] beta_b (reduced)
  FixItem* fix;             // cells handed to the fix-up kernel
  unsigned* fix_count;
  const DirInfo* dirs;
  const double* wdir;       // [nd]
  const float* wdir32;      // [nd]
  const DevGeom* geoms;
  const WorkItem* items;
  int nitems;
  int nd;
  int lpc;                  // lanes per direction row = nbp / values per lane
  int dteam;                // directions one cell team covers per step (team = lpc * dteam lanes)
  int solve_tp;             // 0 when every beta_b == 0 (T_p then unused)
  double trust_rel;         // cached model accepted when |T - T_e| <= trust_rel * T
  int maxit;
  double Wtot;              // sum of direction weights
  int dry;                  // 1: timing run, the epilogue writes no solver state
  int partial;              // 1: band-range handle; the epilogue writes per-cell partial (E_L, E_p)
  double* Epart;            //    to Epart[cell][2] and the solve runs after the caller's all-reduce
  double beta_exp;          // beta_b(T) = beta_b (T_p / beta_Tref)^beta_exp per cell (0: fixed tau)
  double beta_Tref;
  int explicit_scheme;      // reduced modes compute P, Q on the fly from these:
  float dt32, rdt32;        // dt and 1/dt
  DevCounters* counters;
  // sweep-ordered pass (scheme BTE_IMPLICIT_GS, FP64)
  const GsUnit* gs_units;
  const int* gs_dirs;       // direction indices grouped by octant
  int gs_nunits;
  int gs_ndc;               // directions per unit (the CTA layout)
  int gs_tx, gs_ty;         // cross-section of a column tile (2-D: gs_tx cells along x)
  const double* bscale;     // [cell] beta_b(T_p)/beta_b (beta_exp != 0), written before each pass
  ThermoTables th;
};

// Launchers (bte_kernels.cu).  precision: BTE_FP64 = 0, BTE_FP32 = 1, BTE_BF16 = 2.
int values_per_lane(int precision);
// Raises the dynamic shared memory limit of kernel func on the current device
// to at least bytes (no call below 48 KB).  The limit only grows, under a
// lock: handles on several host threads launch the same kernel with different
// needs, and a per-launch setting could lower another thread's limit between
// its own setting and its launch.
cudaError_t raise_dynamic_smem(const void* func, size_t bytes);
cudaError_t launch_sweep(int precision, int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s);
cudaError_t launch_sweep_fp64(int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s);
cudaError_t launch_sweep_fp32(int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s);
cudaError_t launch_sweep_bf16(int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s);
struct MLPView;
cudaError_t launch_fixup(const SweepArgs& a, const MLPView* mlp, cudaStream_t s);
cudaError_t launch_solve_cells(const SweepArgs& a, long long ncells, cudaStream_t s);
// sweep-ordered pass (bte_gs.cu) and its per-cell step (bte_kernels.cu): the
// pass writes Iout; the reduction writes E_L, E_p of the stored bands to Epart
// (partial) or solves T_p and refreshes I0 at once (whole handle)
cudaError_t launch_gs_sweep(int precision, const SweepArgs& a, int dim, int threads, cudaStream_t s);
cudaError_t launch_gs_reduce(int precision, const SweepArgs& a, long long ncells, cudaStream_t s);
cudaError_t launch_beta_scale(double* out, const double* Tp, double Tref, double p, long long ncells, cudaStream_t s);
cudaError_t launch_diffuse_ghosts(int precision, const void* I, const double* I0ref, double* I0wall, float* I0wall_dev,
                                  const DevGeom* geoms, int geom, int side, const double* S, int nd, int nbp,
                                  int nfaces, cudaStream_t s);
// Partially specular side: per face, direction and band, p x the cell's mirrored
// value + (1 - p) x the diffuse value, into out [face][dir][nbp] (storage type).
cudaError_t launch_partial_ghosts(int precision, const void* I, const double* I0ref, const DevGeom* geoms, int geom,
                                  int side, const double* S, const DirInfo* dirs, int nd, int nbp, int nfaces,
                                  double p, void* out, cudaStream_t s);
// learned guess (bte_mlp.cu)
int mlp_param_total(int nb);
cudaError_t launch_mlp_norm(ThermoTables th, double T_lo, double T_hi, const double* I0ref, double* r_lo, double* r_hi,
                            double* E_lohi, cudaStream_t s);
cudaError_t launch_mlp_pairs(ThermoTables th, double T_lo, double T_hi, const double* I0ref, const double* r_lo,
                             const double* r_hi, const double* E_lohi, unsigned long long seed, int n, float* xA,
                             float* yA, float* yB, cudaStream_t s);
cudaError_t mlp_forward_backward(const float* p, int k, const float* X, int ldx, const float* Tg, int ldt, int B,
                                 float* grad, float* act, float* part, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s);
cudaError_t launch_solve_batch(ThermoTables th, const double* Ep, const double* T0, int n, double trust_rel, int maxit,
                               const MLPView* mlp, double* Tout, int* evals, cudaStream_t s);
cudaError_t launch_init_cells(int precision, void* I, double* I0cell, double* J, double* Msum, double* Tp, double* Te,
                              double* TL, double* EL, const double* Tcells, const double* I0ref, long long cell0,
                              int ncells, int nd, ThermoTables th, cudaStream_t s);
cudaError_t launch_state_from_Tp(double* I0cell, double* J, double* Msum, const double* Tp, double* Te, long long ncells,
                                 ThermoTables th, cudaStream_t s);
cudaError_t launch_wall_I0(double* I0wall, const double* Tfaces, long long nfaces, ThermoTables th, cudaStream_t s);
cudaError_t launch_wall_dev(float* out, const double* I0wall, const double* I0ref, long long nfaces, int nbp,
                            cudaStream_t s);
cudaError_t launch_solve_TL(double* TL, const double* EL, const double* Tguess, const double* J, const double* Teval,
                            long long ncells, ThermoTables th, double trust_rel, int maxit, DevCounters* counters,
                            cudaStream_t s);
cudaError_t launch_flux_cells(int precision, const void* I, const double* I0ref, double* q, const double* S,
                              long long cell0, int ncells, int nd, int nbp, int dim, cudaStream_t s);
cudaError_t launch_flux_faces(int precision, const void* I, const double* I0ref, const double* I0wall,
                              const DevGeom* geoms, int geom, int side, const DirInfo* dirs, const double* S, int nd,
                              int nbp, double* face_out, int nfaces, cudaStream_t s);
cudaError_t launch_mean(const double* v, int n, double* out, cudaStream_t s);
// In place: npairs 16-byte ff pairs of two bands (bte_ff.cuh layout) -> two doubles each.
cudaError_t launch_ff_to_doubles(void* buf, long long npairs, cudaStream_t s);
cudaError_t launch_pack(int precision, const double* src, double* dst_out, const void* Isrc, void* Idst,
                        const double* I0ref, long long ncells, int nd, int nb, int nbp, int to_padded, cudaStream_t s);
cudaError_t launch_energy_L(int precision, const void* I, const double* I0ref, double* EL, const double* wdir,
                            long long ncells, int nd, ThermoTables th, cudaStream_t s);

// Read-only view of one geometry's device state, for entry points that live
// outside bte_capi.cu (bte_noalloc.cu).  flux_view returns BTE_E_* codes.
struct FluxView {
  int precision;          // storage of I (BTE_FP64 = 0, BTE_FP32 = 1, BTE_BF16 = 2)
  const double* I;        // current intensity buffer (padded rows; FP64 only when precision == 0)
  const double* I0wall;
  const DevGeom* geoms;
  const DirInfo* dirs;
  const double* S;        // [nd][3]
  int nd, nbp, dim;
  int nfaces[6];          // faces per side (0 for sides beyond 2*dim)
  cudaStream_t stream;
  int dev;                // device that holds the handle's memory and stream
};
int flux_view(bte_ctx* h, int geom, FluxView* out);
int handle_device(bte_ctx* h);  // device that was current at bte_init_mesh
int set_handle_error(bte_ctx* h, int code, const char* fmt, ...);

}  // namespace bte
