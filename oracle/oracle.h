/*
 * oracle.h -- plain FP64 CPU oracle of the immersed boundary - lattice
 * Boltzmann (IB-LB) wetting time step of Bellantoni et al., "Immersed
 * boundary - lattice Boltzmann method for wetting problems" (arXiv 2503.20605).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and never calls it.
 *
 * Every array is a plain C array owned by the caller unless stated otherwise.
 * Lattice arrays cover the fluid cells only, in the layout
 *     a[k][z'][y][x]   (x fastest),  z' = Z - 1 when walls are on, Z otherwise,
 * where (X, Y, Z) are the integer lattice-node coordinates of the full box
 * nx * ny * nz (solid layers Z = 0 and Z = nz - 1 when walls are on).
 * Membrane node positions q_j are (x, y, z) triples in the same coordinates.
 *
 * Parity status: every function here is pinned by a test in tests/ against a
 * closed form, an invariant, a brute-force evaluation or a number printed in
 * the paper, except where its comment says "parity unpinned".
 */
#ifndef IBLB_ORACLE_H
#define IBLB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;          /* full box, lattice nodes                        */
    int walls;               /* 1: solid layers Z=0, Z=nz-1, halfway bounce-back;
                                0: periodic in z as well                        */
    double tau_out, tau_in;  /* BGK relaxation times outside / inside           */
    double rho0;             /* initial (reference) density                     */
    double body_force[3];    /* uniform force density added on every fluid cell */
    double sigma;            /* surface tension                                 */
    int wetting;             /* 1: wall interaction Pi(h) on, 0: off            */
    double A, xi;            /* Pi(h) = A[(xi/h)^n - (xi/h)^m]                 */
    int n, m;
    double h_min_frac;       /* near-wall guard h_eff = max(h, h_min_frac*xi)   */
    int volume_correction;   /* 1: rescale the mesh about its centroid to V0    */
    double shear_modulus;    /* Skalak membrane moduli k_s, k_alpha added to the */
    double area_modulus;     /* surface tension (0, 0: the paper's droplet)     */
} orc_params;

typedef struct orc_sim orc_sim;

/* --- D3Q19 lattice (Tab. I) --------------------------------------------- */
void   orc_d3q19(int *c /* 19*3 */, double *w /* 19 */, int *opp /* 19 */);
void   orc_feq(double rho, const double *u, double *feq /* 19 */);
void   orc_guo_source(double tau, const double *u, const double *F, double *S /* 19 */);
void   orc_collide_cell(double tau, const double *F, double *f /* 19, in: pulled f, out: f* */,
                        double *rho, double *u);

/* --- IB coupling (Sec. II A) --------------------------------------------- */
double orc_psi(double r);
void   orc_spread(const orc_params *p, const double *xyz, const double *phi, int n_nodes,
                  double *F /* 3*cells, accumulated into */);
void   orc_interp(const orc_params *p, const double *xyz, int n_nodes, const double *U,
                  double *qdot /* 3*n */);

/* --- membrane forces (Sec. II B, II C) ----------------------------------- */
double orc_wetting_A(double sigma, double theta_eq_rad, double xi, int n, int m);
double orc_Pi(double h, double A, double xi, int n, int m);
int    orc_membrane_forces(const orc_params *p, const double *xyz, int n_nodes,
                           const int *tri, int n_tri, double *phi /* 3*n */,
                           double *phi_sigma /* 3*n or NULL */, double *phi_pi /* 3*n or NULL */);
void   orc_membrane_elastic(const orc_params *p, const double *xyz_ref, const double *xyz, int n_nodes,
                            const int *tri, int n_tri, double *phi /* 3*n, added to */);
double orc_mesh_area(const double *xyz, const int *tri, int n_tri);
double orc_mesh_volume(const double *xyz, const int *tri, int n_tri);

/* --- in/out classification for tau(x) (Sec. II A, "ray tracing") -------- */
void   orc_inside(const orc_params *p, const double *xyz, const int *tri, int n_tri,
                  unsigned char *inside /* cells */);

/* --- observables (Sec. III, App. C) --------------------------------------- */
enum { ORC_OBS_MASS = 0, ORC_OBS_VOLUME, ORC_OBS_AREA, ORC_OBS_CX, ORC_OBS_CY, ORC_OBS_CZ,
       ORC_OBS_ZMIN, ORC_OBS_ZMAX, ORC_OBS_THETA_R0, ORC_OBS_THETA_RV, ORC_OBS_RC_CUT,
       ORC_OBS_RC_FLAT, ORC_OBS_N_CUT, ORC_OBS_CHI_FLAT, ORC_OBS_N };
double orc_theta_from_height(double ell, double R);
void   orc_mesh_observe(const double *xyz, int n_nodes, const int *tri, int n_tri, double R0,
                        double z_wall, double zcut_frac, double eps_flat, double *out);

/* --- full time step -------------------------------------------------------- */
orc_sim *orc_create(const orc_params *p);
void   orc_destroy(orc_sim *s);
int    orc_set_membrane(orc_sim *s, const double *xyz, int n_nodes, const int *tri, int n_tri);
void   orc_set_nodes(orc_sim *s, const double *xyz);
void   orc_get_nodes(const orc_sim *s, double *xyz);
void   orc_set_populations(orc_sim *s, const double *f);
void   orc_get_populations(const orc_sim *s, double *f);
void   orc_step(orc_sim *s, int nsteps);
void   orc_set_threads(int n);   /* threads of the stream-collide loop (OpenMP builds) */
int    orc_get_threads(void);
void   orc_get_macros(const orc_sim *s, double *rho, double *u);
void   orc_get_force_density(const orc_sim *s, double *F);
void   orc_get_node_forces(const orc_sim *s, double *phi);
void   orc_get_tau(const orc_sim *s, double *tau);
void   orc_observe(const orc_sim *s, double zcut_frac, double eps_flat, double *out);
long   orc_clamped_nodes(const orc_sim *s);
long   orc_cells(const orc_sim *s);

#ifdef __cplusplus
}
#endif
#endif
