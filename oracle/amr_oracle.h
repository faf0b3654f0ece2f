/*
 * amr_oracle.h -- plain FP64 CPU oracle for the per-patch finite-volume update
 * of block-structured AMR compressible Euler / GLM-MHD
 * (Wang, Abel & Kaehler, "Adaptive Mesh Fluid Simulations on GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: its own geometry, ghost fill, reconstruction, Riemann
 * solver, time integrator, refluxing and restriction are written here from the
 * paper (Sec. 3, Sec. 4 Eqs. for U, F, EOS, MOL, RK2, PLM, minmod, HLL;
 * Sec. 5.1 three-line RK2 form; Sec. 7.1 GLM-MHD).
 *
 * Conventions of every state array that crosses this interface:
 *   interior cells only, FP64, layout [var][z][y][x] (x fastest).
 * Hydro variables (nvar = 5):  U = (rho, rho vx, rho vy, rho vz, rho E),
 *                              W = (rho, vx, vy, vz, p)
 * GLM-MHD (nvar = 9):          U = (rho, rho v, rho E + B^2/2, Bx, By, Bz, psi),
 *                              W = (rho, vx, vy, vz, p, Bx, By, Bz, psi)
 */
#ifndef AMR_ORACLE_H
#define AMR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_HLL = 0, ORC_LLF = 1, ORC_FLUXREC = 2 };
enum { ORC_PLM = 0, ORC_WENO3 = 1 };
enum { ORC_BC_OUTFLOW = 0, ORC_BC_PERIODIC = 1 };

typedef struct {
  int nvar;           /* 5 (Euler) or 9 (GLM-MHD) */
  int riemann;        /* ORC_HLL (two-wave HLL), ORC_LLF (the printed Sec. 4 flux) or
                         ORC_FLUXREC (direct flux reconstruction, Euler only) */
  int plm_literal;    /* 1: add the full limited slope at faces (printed PLM), 0: half slope */
  double gamma;
  double theta;       /* generalised-minmod parameter, 0 <= theta <= 2 */
  double cfl;
  int base_n[3];      /* level-0 cells per axis */
  double domain_lo[3], domain_hi[3];
  int bc[6];          /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */
  int max_level;
  double ch;          /* GLM cleaning speed; <= 0: max signal speed at the start of each coarse step */
  double p_floor;     /* pressure floor of the reconstructed variables (0 = off): e >= p_floor / ((gamma-1) rho) */
  double glm_alpha;   /* GLM damping: psi *= exp(-glm_alpha c_h dt_l / min_d dx_l) after every level step (0 = off) */
  int nthreads;       /* OpenMP threads over patches; <= 0: library default */
  int recon;          /* face states: ORC_PLM (Sec. 4) or ORC_WENO3 (third-order WENO on the same
                         three-cell stencils, a higher-order scheme in the sense of the abstract);
                         ORC_WENO3 with ORC_HLL or ORC_LLF only */
} orc_config;

typedef struct { int level; int lo[3]; int n[3]; } orc_patch;

typedef struct orc_sim orc_sim;

/* Create a simulation; returns NULL on invalid input (message in orc_error()). */
orc_sim* orc_create(const orc_config* cfg, int npatch, const orc_patch* patches);
const char* orc_error(void);
void orc_destroy(orc_sim* s);

/* Set one patch from primitive W or conserved U (interior, [nvar][z][y][x]). */
int orc_set_prim(orc_sim* s, int patch, const double* w);
int orc_set_cons(orc_sim* s, int patch, const double* u);
int orc_get_cons(const orc_sim* s, int patch, double* u);

/* CFL step size of the current state (max over all cells of all levels). */
double orc_cfl_dt(orc_sim* s);
/* One coarse step of size dt (dt <= 0: CFL step).  Returns 0 or -1. */
int orc_step(orc_sim* s, double dt, double* dt_used);
/* Sum of U * cell volume over leaf (uncovered) cells, nvar values. */
void orc_totals(const orc_sim* s, double* out);
/* Cleaning speed used by the last step (MHD). */
double orc_last_ch(const orc_sim* s);
/* GLM-MHD only (-1 otherwise): refill the face ghosts of every level at the
 * current time, then over leaf cells, with D = sum_d (B_d(i+e_d) - B_d(i-e_d)) / (2 dx_d)
 * and b = |B| / min_d dx_d of the cell's level:
 *   out[0] = sum |D| dV,  out[1] = max |D|,  out[2] = sum b dV,  out[3] = max b.
 * out[0]/out[2] and out[1]/out[3] are dimensionless divergence errors. */
int orc_divb(orc_sim* s, double* out);

/* ---- test hooks: fill the face ghosts of one level (state 0: U, 1: U1) at
 * parent-time fraction alpha, and read a patch's full ghosted array
 * [nvar][n2+4][n1+4][n0+4] (edge/corner ghosts are never filled: NaN) ---- */
int orc_fill_ghosts(orc_sim* s, int level, int which, double alpha);
int orc_get_ghosted(const orc_sim* s, int patch, int which, double* out);
/* Save the current state of a level as the "old" time level used by
 * prolongation (done automatically at the start of every coarse-level step). */
int orc_save_old(orc_sim* s, int level);

/* ---- regridding ----
 * orc_flags: after filling every level's face ghosts at the current time, one
 * byte per interior cell of every patch (patch order, [z][y][x]): 1 where
 * max_d |rho(i+e_d) - rho(i-e_d)| / (2 rho(i)) > threshold.
 * orc_regrid_fill: a new simulation on `patches`, whose levels <= keep_level are
 * the old ones unchanged; a cell of a finer level takes the old same-level
 * value where an old patch holds it, else the conservative prolongation of the
 * (new) parent level.  Returns NULL on error. */
int orc_flags(orc_sim* s, double threshold, unsigned char* out);
orc_sim* orc_regrid_fill(orc_sim* old, int npatch, const orc_patch* patches, int keep_level);

/* ---- regrid in the middle of a coarse step (Sec. 3: after each step of a level,
 * the finer levels are rebuilt) ----
 * orc_set_regrid_hook: during orc_step, after every completed step of a level
 * l <= max_level (its own children advanced, restricted and refluxed) call
 * hook(ctx, l, alpha) with alpha the time fraction of l's parent step reached
 * (0.5 or 1; 1 for level 0); a non-zero return aborts the step.  hook NULL
 * removes it.
 * orc_flags_at: the flags of orc_flags at that moment: face ghosts of level l
 * from its parent at fraction alpha, of the finer levels at fraction 1, without
 * touching the saved old-time states; only levels >= l are meaningful.
 * orc_regrid_inplace: replace the hierarchy of `s` by `patches` (levels <= keep
 * unchanged, finer levels filled as by orc_regrid_fill), keeping the old-time
 * states and flux registers of the kept levels so the step can continue.
 * Returns 0 or -1. */
typedef int (*orc_regrid_hook)(void* ctx, int level, double alpha);
void orc_set_regrid_hook(orc_sim* s, int max_level, orc_regrid_hook hook, void* ctx);
int orc_flags_at(orc_sim* s, double threshold, int level, double alpha, unsigned char* out);
int orc_regrid_inplace(orc_sim* s, int npatch, const orc_patch* patches, int keep_level);

/* ---- point functions, exposed for unit pins ---- */
double orc_minmod3(double a, double b, double c);
double orc_minmod2(double a, double b);
/* PLM left/right states at face i-1/2 from four cell values u[0..3] = u_{i-2..i+1}. */
void orc_plm_face(const orc_config* cfg, const double* u4, double* ul, double* ur);
/* Physical flux of primitive state w along dir (0,1,2); ch used for MHD psi/B_d entries. */
void orc_phys_flux(const orc_config* cfg, const double* w, int dir, double ch, double* f);
void orc_prim_to_cons(const orc_config* cfg, const double* w, double* u);
void orc_cons_to_prim(const orc_config* cfg, const double* u, double* w);
/* Interface flux from primitive left/right states along dir. */
void orc_riemann(const orc_config* cfg, const double* wl, const double* wr, int dir, double ch, double* f);
/* Third-order WENO face states of face i-1/2 from u4 = (u_{i-2}, u_{i-1}, u_i, u_{i+1}). */
void orc_weno3_face(const double* u, double* ul, double* ur);
/* Direct flux reconstruction at the face between cells 1 and 2 of four conserved
 * states u4[4][nvar] along dir (Euler): Lax-Friedrichs split fluxes, each
 * reconstructed by PLM from its upwind side. */
void orc_fluxrec_face(const orc_config* cfg, const double* u4, int dir, double* f);

#ifdef __cplusplus
}
#endif
#endif
