/*
 * amrfd_oracle.h -- the CPU oracle's own interface.
 *
 * TEST INFRASTRUCTURE ONLY. This header and amrfd_oracle.c form a plain,
 * single-threaded FP64 CPU restatement of the conservative finite-difference
 * update of Porth et al. (MPI-AMRVAC, ApJS 2014), Sec. 2.1-2.3: Lax-Friedrichs
 * flux splitting, MP5 reconstruction (Suresh & Huynh 1997, cited in Sec. 2.2),
 * SSPRK time stepping and the CFL time step. Only the test suite, the bench's
 * CPU-baseline leg and the smoke check may call it. It shares no code, header,
 * table or constant with the CUDA library under paper_1407_2052_gb300/.
 *
 * Parity unpinned (these follow stated readings of the paper; no check against
 * anything but this code fixes them): the value eps = 1e-10 of the MP5 acceptance
 * test, the scope of the splitting speed (per direction, per RK stage, over active
 * cells), the unsplit multi-D time step, the GLM damping length c_r = 0.18 and the
 * GLM speed frozen over a step, and LIMO3's switch radius r and blend width.
 *
 * State layout: one domain is an interior-only array U[v][z][y][x], x fastest,
 * with n[0]*n[1]*n[2] cells per variable (unused dimensions have n = 1).
 *   Euler  (nv = 2 + ndim): rho, m_1..m_ndim, E
 *   MHD+GLM (nv = 9):       rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi
 */
#ifndef AMRFD_ORACLE_H
#define AMRFD_ORACLE_H
#include <stdint.h>

#define ORC_EULER 0
#define ORC_MHD_GLM 1
#define ORC_SSPRK3 0
#define ORC_SSPRK54 1
#define ORC_SSPRK43 2
#define ORC_MP5 0
#define ORC_LIMO3 1
#define ORC_BC_PERIODIC 0
#define ORC_BC_OUTFLOW 1
#define ORC_BC_SYMMETRIC 2 /* mirror ghosts; variables flagged in asym[d][f] change sign */

/* flags reported by orc_step / orc_speeds */
#define ORC_FLAG_NONPHYSICAL 1

typedef struct orc_cfg {
  int physics;    /* ORC_EULER | ORC_MHD_GLM */
  int ndim;       /* 1..3 */
  int integrator; /* ORC_SSPRK3 | ORC_SSPRK54 | ORC_SSPRK43 */
  int recon;      /* ORC_MP5 | ORC_LIMO3 */
  double gamma;
  double glm_cr;  /* psi damping length c_r = c_p^2/c_h; <= 0 disables damping */
  double limo3_r; /* LIMO3: radius r of the asymptotic region (eta uses r dx) */
} orc_cfg;

typedef struct orc_dom {
  int n[3];       /* interior cells per dimension */
  int nb[3];      /* blocks per dimension (block edge = n[d]/nb[d]) */
  double dx[3];
  int bc[3][2];   /* ORC_BC_* for the low and high face of each dimension */
  unsigned asym[3][2]; /* ORC_BC_SYMMETRIC: bit v set = variable v is odd across the face */
} orc_dom;

int orc_nvar(const orc_cfg *c);

/* point-wise pieces (exposed so tests can pin each against closed forms) */
int orc_cons2prim(const orc_cfg *c, const double *u, double *w /* rho,vx,vy,vz,p,Bx,By,Bz,psi */);
double orc_char_speed(const orc_cfg *c, const double *w, int d);
void orc_flux(const orc_cfg *c, const double *u, const double *w, int d, double ch, double *f);
double orc_mp5(double a, double b, double cc, double d, double e);
double orc_limo3(double um, double u0, double up, double rdx);
double orc_minmod(double a, double b);
double orc_minmod4(double w, double x, double y, double z);

/* SSPRK tables in Shu-Osher form; returns the number of stages s and fills
   alpha[i][k], beta[i][k] for i = 1..s (row i-1 of the 5x5 arrays). */
int orc_ssprk_table(int integrator, double alpha[5][5], double beta[5][5]);

/* per-direction maximal characteristic speed over active interior cells,
   and max over active cells of sum_d c_d/dx_d. Returns flags. */
int orc_speeds(const orc_cfg *c, const orc_dom *dm, const double *U, const uint8_t *block_active,
               double alpha_raw[3], double *rate_max);

/* L(U) for one domain with given splitting speeds alpha[3] and GLM speed ch. */
int orc_residual(const orc_cfg *c, const orc_dom *dm, const double *U, const double alpha[3],
                 double ch, double *L);

/* one full SSPRK step in place. block_active may be NULL (all active).
   alpha_stage (may be NULL) receives the splitting speeds of every stage,
   [s][3]; ch_out (may be NULL) the frozen GLM speed. Returns flags. */
int orc_step(const orc_cfg *c, const orc_dom *dm, double *U, double dt, const uint8_t *block_active,
             double *alpha_stage, double *ch_out);

/* The same step with the splitting speeds of every stage (alpha_in, [s][3], as
   returned in alpha_stage by orc_step) and the GLM speed ch_in held fixed: the
   map whose derivative the discrete adjoint transposes. */
int orc_step_frozen(const orc_cfg *c, const orc_dom *dm, double *U, double dt, const uint8_t *block_active,
                    const double *alpha_in, double ch_in);

/* CFL time step of one domain; returns flags. */
int orc_dt(const orc_cfg *c, const orc_dom *dm, const double *U, const uint8_t *block_active,
           double cfl, double t, double t_end, double *dt_out);

/* Dynamic grid activation (App. C). Step 1, a criterion: flag[b] = 1 when every
   cell and variable of block b lies within tol (absolute) of the reference state
   Uref (the block is a candidate for de-activation), else 0. */
void orc_flag_steady(const orc_cfg *c, const orc_dom *dm, const double *U, const double *Uref, double tol,
                     uint8_t *flag);

/* Steps 2 and 3: blocks not flagged are active; then, `belt` times, every
   candidate block with an active neighbour (face, edge or corner; across periodic
   faces) becomes active, all candidates tested against the previous round's
   flags. Writes the final active flags. */
void orc_activate(const orc_dom *dm, const uint8_t *flag, int belt, uint8_t *active);

#endif
