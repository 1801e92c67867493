/*
 * hydro_oracle.h -- plain FP64 CPU oracle for the WENO5 / Lax-Friedrichs / SSP-RK3 update of the
 * 2D Euler equations with a level-set scalar (Leung, Chu & Lin 2015, Sec. 2.1 "Hydrodynamics",
 * Eq. euler2D, and Sec. 2.2 "Level-set method").
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA library against a slow, obviously
 * correct restatement of the method. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may call it; the product path never does.
 *
 * Layout: every state array is structure-of-arrays, U[f][j][i] (i = x index, contiguous), doubles,
 * f = 0 rho, 1 rho*u (m_x, or rho*v_r), 2 rho*v (m_y, or rho*v_z), 3 total energy density tau,
 * 4 level-set phi (only when nfields == 5). Values are point values at cell centres
 * x_i = x0 + (i + 1/2) dx, y_j = y0 + (j + 1/2) dy.
 */
#ifndef HYDRO_ORACLE_H
#define HYDRO_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_TRANSMISSIVE = 1, ORC_REFLECT = 2, ORC_AXIS = 3 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENONPHYSICAL = -3 };

typedef struct {
  int nx, ny;
  double x0, x1, y0, y1;
  double gamma;        /* ideal-gas ratio of specific heats, p = (gamma-1) rho eps           */
  double cfl;          /* Courant number c_cfl                                                */
  int geometry;        /* 0: Cartesian (x, y); 1: axisymmetric (r, z) with x = r            */
  double gravity;      /* constant acceleration along y (= z); source (0, 0, rho g, m_y g)    */
  int bc[4];           /* x-lo, x-hi, y-lo, y-hi, values ORC_*                                */
  int nfields;         /* 4 (hydro) or 5 (hydro + level set phi)                              */
  double flame_speed;  /* burning speed s_f of the level-set front                            */
  int scheme;          /* 0 component-wise WENO5; 1 characteristic-wise with Roe-averaged       *
                        * eigenvectors (the adjoint covers scheme 0 only)                       */
  int rk_stages;       /* 3 (or 0): three-stage SSP-RK3; 5: the five-stage third-order scheme    *
                        * (the adjoint is of the 3-stage one)                                   */
} orc_config;

int orc_validate(const orc_config* c);
void orc_set_threads(int n);
int orc_get_threads(void);

/* WENO5-JS reconstruction at the right face of c from the left-biased list (a,b,c,d,e). */
double orc_weno5(double a, double b, double c, double d, double e);
void orc_weno5_weights(double a, double b, double c, double d, double e, double w[3]);
/* Gradient of orc_weno5 with respect to its five arguments. */
void orc_weno5_grad(double a, double b, double c, double d, double e, double g[5]);

/* Global Lax-Friedrichs speeds of a state: max |u|+c and max |v|+c over interior cells. */
int orc_alpha(const orc_config* c, const double* U, double* ax, double* ay);
/* CFL signal speed max(c + |u| + |v|) and the time step c_cfl * min(dx,dy) / that maximum. */
int orc_max_speed(const orc_config* c, const double* U, double* smax);
int orc_dt(const orc_config* c, const double* U, double* dt);

/* Spatial operator L(U) (flux divergence plus sources, plus the level-set right-hand side). */
int orc_rhs(const orc_config* c, const double* U, double ax, double ay, double* L);

/* nsteps steps (SSP-RK3, or the five-stage scheme with rk_stages = 5), in place. t accumulates dt. If
 * dt_log / alpha_log are non-NULL they receive per step dt (nsteps doubles) and per stage (alpha_x,
 * alpha_y) (2 * stages * nsteps doubles). */
int orc_step(const orc_config* c, double* U, int nsteps, double* t, double* dt_last,
             double* dt_log, double* alpha_log);
/* Same map with dt and the per-stage alphas frozen at the given logged values. */
int orc_step_frozen(const orc_config* c, double* U, int nsteps, const double* dt_log,
                    const double* alpha_log);

/* Roe average of the conserved states a, b (rho, m_x, m_y, tau) and the eigen-system of the flux
 * Jacobian along dir (0 x, 1 y) there, in the rotated frame (rho, m_n, m_t, tau): R[4*c + k] is component c
 * of right eigenvector k, Lm[4*k + c] the left eigenvectors (rows), lam the wave speeds v_n - c, v_n, v_n,
 * v_n + c. ORC_ENONPHYSICAL if the averaged sound speed is not real. */
int orc_roe_eigen(double gamma, int dir, const double a[4], const double b[4], double R[16], double Lm[16],
                  double lam[4]);

/* Conserved totals sum U_f dV, f = 0..4 (phi total is 0 when nfields == 4). */
int orc_totals(const orc_config* c, const double* U, double out[5]);

/* Discrete adjoint of one frozen SSP-RK3 step: lambda holds dJ/dU^{n+1} on entry and dJ/dU^n on exit.
 * alpha holds (alpha_x, alpha_y) for the three stages. */
int orc_adjoint_step(const orc_config* c, const double* Un, double* lambda, double dt,
                     const double alpha[6]);
/* Level-set reinitialisation of phi (field 4) in place (Sec. 2.2); *npoints receives the number of
 * front points. orc_reinit_blend is the blending weight H(d) for grid size delta. */
int orc_reinit(const orc_config* c, double* U, int* npoints);
double orc_reinit_blend(double d, double delta);

/* Self-gravity potential of rho [ny][nx] on an (r,z) grid by red-black SOR (Sec. 2.1); mass is the
 * grid's mass (sum of rho 2 pi r dr dz); phi holds the initial guess on entry and the result on exit;
 * *iters receives the sweeps done. */
int orc_poisson(const orc_config* c, const double* rho, double grav_const, double mass, double omega, double tol,
                int max_iters, double* phi, int* iters);

/* Adjoint of the spatial operator: out = (dL/dU)^T mu (alpha frozen). */
int orc_rhs_adjoint(const orc_config* c, const double* U, double ax, double ay, const double* mu,
                    double* out);

#ifdef __cplusplus
}
#endif
#endif
