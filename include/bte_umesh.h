/* bte_umesh.h -- the phonon BTE hot path on unstructured meshes.
 *
 * The paper's discretisation (Sec. 3.1, Eq. 5) integrates the BTE over a
 * control volume and turns the advection into a sum over the cell's faces;
 * its meshes come from Gmsh or MEDIT files or an internal generator (Sec.
 * 3.3).  This interface takes such a mesh as a face list and runs the same
 * per-iteration update as bte.h on it:
 *   for every cell P, direction d, band b and face f of P, with
 *   g_f = (S_d . n_f A_f) / (w_d V_P) (n_f pointing out of P),
 *   outflow faces (g_f > 0) use the cell's own value and inflow faces
 *   (g_f < 0) the upwind value: the neighbour's, or the boundary ghost.
 *   Implicit (one point-Jacobi sweep per inner iteration):
 *     I^{k+1} = [I^n/dt + beta_b I0_b + v_b sum_{g<0} |g| I_up^k]
 *               / [1/dt + beta_b + v_b sum_{g>0} g]
 *   Explicit (Eq. 3): I^{n+1} = I^n + dt [beta_b (I0_b - I^n) - v_b sum_f g_f I_f^n].
 * followed by the per-cell reduction, the T_p solve and the I0 refresh of
 * bte.h (all FP64).  Storage: FP64, or as in bte.h the deviation
 * I - I0_b(T_ref) in FP32 or BF16 with the update in FP32.
 *
 * Boundary faces carry an integer tag; each tag gets one condition:
 *   BTE_BC_ISOTHERMAL  ghost I0_b(T_face) (Eq. 6);
 *   BTE_BC_SPECULAR    ghost = the cell's own value in the direction mirrored
 *                      across the face (Eq. 6); every face of the tag must be
 *                      normal to a coordinate axis (the direction sets are
 *                      mirror-symmetric only across the axis planes);
 *   BTE_BC_DIFFUSE     every incoming direction gets
 *                      sum_out (S.n) I / sum_in |S.n| of the cell (zero net flux).
 *
 * Call order: bte_umesh_create -> bte_umesh_set_bands -> bte_umesh_set_bc
 * (every boundary tag) -> bte_umesh_set_initial -> bte_umesh_step / getters.
 * Every function returns a BTE_* status of bte.h (0 on success) and leaves a
 * message for bte_umesh_last_error.  Device memory is allocated by the
 * handle (cudaMalloc) and freed by bte_umesh_destroy.
 */
#ifndef BTE_UMESH_H
#define BTE_UMESH_H

#include "bte.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bte_umesh_ctx* bte_umesh;

/* A mesh as a face list (host arrays, copied by bte_umesh_create).
 *  dim        2 (areas and edge lengths per unit depth, nA[f][2] = 0) or 3.
 *  volume     [ncells] cell volumes (> 0).
 *  owner      [nfaces] cell that owns the face (0 <= owner < ncells).
 *  neighbor   [nfaces] the other cell, or -1 on the boundary.
 *  nA         [nfaces][3] area vector, pointing out of the owner.
 *  tag        [nfaces] boundary tag (>= 0) of boundary faces; ignored on
 *             interior faces.
 *  fc         [nfaces][3] face centres, or NULL; needed only by faces that
 *             take BTE_BC_ROTATIONAL.
 * A cell may have at most 64 faces. */
typedef struct {
  int dim;
  long long ncells, nfaces;
  const double* volume;
  const long long* owner;
  const long long* neighbor;
  const double* nA;
  const int* tag;
  const double* fc;
} bte_umesh_desc;

/* Creates a handle.  opts: as in bte.h (precision BTE_FP64, BTE_FP32 or
 * BTE_BF16; beta_T_exp as in bte.h, |beta_T_exp| <= 16, the relaxation rates
 * beta_b (T_p / T_ref)^beta_T_exp per cell, refreshed before every sweep;
 * learned must be 0; use_graph and autotune are not used by this handle,
 * which launches each kernel directly with a fixed shape); may be NULL for
 * the defaults.  *out receives the handle, NULL on failure (message in
 * bte_umesh_last_error(NULL)). */
int bte_umesh_create(const bte_umesh_desc* mesh, const bte_opts* opts, bte_umesh* out);

/* Band table, as bte_set_bands (Sec. 3.1: 40 bands -> 55 band-polarisations). */
int bte_umesh_set_bands(bte_umesh u, int nb, const double* omega_lo, const double* omega_hi, const double* vg,
                        const double* beta, const double* degeneracy);

/* Condition of every boundary face with tag `tag`.  type: BTE_BC_ISOTHERMAL
 * (T_faces: host [nfaces] temperatures indexed by face id, read on this
 * tag's faces, or NULL for T_uniform), BTE_BC_SPECULAR or BTE_BC_DIFFUSE
 * (T ignored), BTE_BC_PARTIAL (an extension beyond the paper's walls, as
 * bte_set_specularity: every incoming direction gets p x the mirrored value
 * + (1 - p) x the diffuse value; p from T_faces indexed by face id, or
 * T_uniform when T_faces is NULL, each in [0, 1]), or BTE_BC_ROTATIONAL (the
 * axisymmetric problems of Sec. 3.1: the mesh is one wedge of angle alpha =
 * T_uniform radians of a body of revolution about the z axis, and these are
 * its two side faces, planes through the axis; across a side face lies the
 * wedge itself rotated by alpha, so the ghost of direction s is the owner's
 * own intensity in s rotated back by alpha, which sends the flux through the
 * side faces from one azimuthal direction to the next (the discrete angular
 * redistribution); the sense per face follows from its outward normal against
 * e_theta at its centre (the mesh needs fc); alpha must map the direction set
 * onto itself (polar x azimuthal sets: a multiple of the azimuthal bin width;
 * in-plane sets: of 2 pi / n), and every rotational tag takes the same
 * alpha).  Specular and partial faces must be normal to an axis.  A tag no boundary face carries, an
 * unknown type or a value out of range returns BTE_E_ARG and changes
 * nothing.  May be called again after bte_umesh_set_initial to change a
 * tag's condition for the following steps. */
int bte_umesh_set_bc(bte_umesh u, int tag, int type, const double* T_faces, double T_uniform);

/* Equilibrium initial state at T_cells (host [ncells], or NULL for T_uniform):
 * I_{d,b} = I0_b(T_P) for every direction, the initial condition of Sec. 3.2. */
int bte_umesh_set_initial(bte_umesh u, const double* T_cells, double T_uniform);

/* nsteps time steps of dt [s] of the face-sum update of Eq. 5 (with Eq. 6
 * ghosts on tagged faces); scheme BTE_IMPLICIT_JACOBI (ninner inner
 * iterations) or BTE_EXPLICIT (ninner ignored).  Each inner iteration is a
 * sweep kernel, the per-cell step and the fix-up (plus one kernel for the
 * diffuse and partially specular faces, and one for the per-cell relaxation
 * scale when beta_T_exp != 0).  stats: as bte_step, may be NULL. */
int bte_umesh_step(bte_umesh u, double dt, int nsteps, int ninner, int scheme, bte_stats* stats);

/* Cell temperatures (BTE_T_PSEUDO or BTE_T_LATTICE, defined as in bte_get_T:
 * the temperature update of Sec. 2.2 and 3.2) into out: ncells doubles,
 * host (on_device = 0) or device memory (1). */
int bte_umesh_get_T(bte_umesh u, int which, double* out, int on_device);

/* Intensities I_{d,b} (the unknown of Eq. 4-5) into host out[ncells][nd][nb]. */
int bte_umesh_get_intensity(bte_umesh u, double* out);

/* Checkpoint restore: replaces the intensities with host in[ncells][nd][nb]
 * (FP64; stored as deviations in the reduced modes) and T_p with host
 * Tp_cells[ncells]; I0 and the cached temperature models are recomputed from
 * T_p and E_L from the intensities.  Needs bte_umesh_set_initial first. */
int bte_umesh_set_intensity(bte_umesh u, const double* in, const double* Tp_cells);

/* Heat flux, the surface term of Eq. 5 summed over directions and bands:
 * q (host [ncells][3], may be NULL) = sum_b sum_d S_d I_{d,b} per
 * cell; Q (host [nfaces], may be NULL) = the net heat flow out through each
 * boundary face, sum_b sum_d (S_d . n_f A_f) I_face (own value leaving,
 * ghost entering), 0 on interior faces. */
int bte_umesh_get_flux(bte_umesh u, double* q, double* Q);

/* Last error message and release of the handle; the paper has no
 * counterpart (error reporting and resource release of this library). */
const char* bte_umesh_last_error(bte_umesh u);
void bte_umesh_destroy(bte_umesh u);

#ifdef __cplusplus
}
#endif

#endif /* BTE_UMESH_H */
