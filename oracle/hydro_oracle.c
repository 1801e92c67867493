/*
 * hydro_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see hydro_oracle.h).
 *
 * What it computes, in the order of the paper's method:
 *   - Euler equations in conservative form with right-hand-side sources (Sec. 2.1, Eq. euler2D):
 *     state (rho, rho v_r, rho v_z, tau); in (r,z) the geometric terms -(1/r)(rho v_r, rho v_r^2,
 *     rho v_r v_z, (tau+p) v_r) and the gravity terms -rho dPhi/dz, -rho v_z dPhi/dz are sources.
 *   - ideal-gas closure p = rho eps (gamma - 1) (Sec. 5.1, one-dimensional code tests).
 *   - finite-difference WENO on fluxes split by a global Lax-Friedrichs splitting; the positive and
 *     negative parts are reconstructed by upwinding and summed (Sec. 2.1). WENO5-JS constants
 *     (eps = 1e-6, power 2, linear weights 1/10, 6/10, 3/10) follow Jiang & Shu (1996), which the
 *     paper cites for the scheme.
 *   - three-stage third-order SSP Runge-Kutta, the "original prescription" the paper names (Sec. 2.1).
 *   - CFL time step dt = c_cfl * Delta / max(c_s + |v_r| + |v_z|) (Sec. 5.4, PTD code test).
 *   - level set dS/dt = -(v + v_flame) . grad S with the flame moving along the front normal into
 *     the fuel (S > 0 ash, S < 0 fuel) (Sec. 2.2), advected with WENO (Hamilton-Jacobi WENO5 of
 *     Jiang & Peng 2000 with a local Lax-Friedrichs Hamiltonian).
 * Every loop is written for clarity: ghost cells are filled into padded copies, split fluxes are
 * formed point by point, each face calls the textbook WENO5 function twice, and the stages combine
 * whole arrays. Rows are distributed over OpenMP threads when compiled with -fopenmp; every output
 * element is computed by exactly one thread, so results do not depend on the thread count.
 */
#include "hydro_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 3 /* ghost layers: the WENO5 stencil reaches three cells across a face */

static const double WENO_EPS = 1e-6;

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_validate(const orc_config* c) {
  if (!c) return ORC_EINVAL;
  if (c->nx < 3 || c->ny < 3) return ORC_EINVAL;
  if (c->nfields != 4 && c->nfields != 5) return ORC_EINVAL;
  if (!(c->x1 > c->x0) || !(c->y1 > c->y0) || !(c->gamma > 1.0) || !(c->cfl > 0.0)) return ORC_EINVAL;
  if (c->geometry != 0 && c->geometry != 1) return ORC_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (c->bc[k] < ORC_PERIODIC || c->bc[k] > ORC_AXIS) return ORC_EINVAL;
  /* periodic faces come in pairs */
  if ((c->bc[0] == ORC_PERIODIC) != (c->bc[1] == ORC_PERIODIC)) return ORC_EINVAL;
  if ((c->bc[2] == ORC_PERIODIC) != (c->bc[3] == ORC_PERIODIC)) return ORC_EINVAL;
  /* the symmetry axis is the r = 0 face of an (r,z) grid */
  if (c->bc[1] == ORC_AXIS || c->bc[2] == ORC_AXIS || c->bc[3] == ORC_AXIS) return ORC_EINVAL;
  if (c->bc[0] == ORC_AXIS && (c->geometry != 1 || c->x0 != 0.0)) return ORC_EINVAL;
  if (c->geometry == 1 && c->x0 < 0.0) return ORC_EINVAL;
  if (c->scheme != 0 && c->scheme != 1) return ORC_EINVAL;
  if (c->rk_stages != 0 && c->rk_stages != 3 && c->rk_stages != 5) return ORC_EINVAL;
  return ORC_OK;
}

/* ---------------------------------------------------------------- WENO5-JS (Jiang & Shu 1996) */

/* Candidate values, smoothness indicators and nonlinear weights of the fifth-order reconstruction of
 * the value at the right face of c from the cell list (a, b, c, d, e). */
static void weno5_parts(double a, double b, double c, double d, double e, double q[3], double w[3]) {
  q[0] = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  q[1] = (-b + 5.0 * c + 2.0 * d) / 6.0;
  q[2] = (2.0 * c + 5.0 * d - e) / 6.0;
  double beta0 = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c) +
                 0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
  double beta1 = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d) + 0.25 * (b - d) * (b - d);
  double beta2 = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e) +
                 0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
  double a0 = 0.1 / ((WENO_EPS + beta0) * (WENO_EPS + beta0));
  double a1 = 0.6 / ((WENO_EPS + beta1) * (WENO_EPS + beta1));
  double a2 = 0.3 / ((WENO_EPS + beta2) * (WENO_EPS + beta2));
  double s = a0 + a1 + a2;
  w[0] = a0 / s;
  w[1] = a1 / s;
  w[2] = a2 / s;
}

double orc_weno5(double a, double b, double c, double d, double e) {
  double q[3], w[3];
  weno5_parts(a, b, c, d, e, q, w);
  return w[0] * q[0] + w[1] * q[1] + w[2] * q[2];
}

void orc_weno5_weights(double a, double b, double c, double d, double e, double w[3]) {
  double q[3];
  weno5_parts(a, b, c, d, e, q, w);
}

/* ------------------------------------------------------------------------------ ghost cells */

/* Source cell and normal-momentum sign of ghost layer k (0 nearest) of a face of a line of n cells. */
static void ghost_source(int bc, int hi_side, int k, int n, int* src, int* flip) {
  *flip = 0;
  switch (bc) {
    case ORC_PERIODIC: *src = hi_side ? k : n - 1 - k; break;
    case ORC_TRANSMISSIVE: *src = hi_side ? n - 1 : 0; break;
    default: /* reflecting wall or symmetry axis: mirror image, normal momentum reversed */
      *src = hi_side ? n - 1 - k : k;
      *flip = 1;
      break;
  }
}

/* Padded copy P[f][(j+G)*(nx+2G) + (i+G)] of U with x ghosts on interior rows and y ghosts on interior
 * columns. Corner ghosts are never read (the scheme works one direction at a time) and stay zero. */
static double* make_padded(const orc_config* c, const double* U) {
  const int nx = c->nx, ny = c->ny, nf = c->nfields;
  const int px = nx + 2 * G, py = ny + 2 * G;
  double* P = (double*)calloc((size_t)nf * px * py, sizeof(double));
  if (!P) return NULL;
  for (int f = 0; f < nf; ++f) {
    const double* Uf = U + (size_t)f * nx * ny;
    double* Pf = P + (size_t)f * px * py;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) Pf[(size_t)(j + G) * px + (i + G)] = Uf[(size_t)j * nx + i];
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < G; ++k) {
        int src, flip;
        ghost_source(c->bc[0], 0, k, nx, &src, &flip);
        double v = Uf[(size_t)j * nx + src];
        Pf[(size_t)(j + G) * px + (G - 1 - k)] = (flip && f == 1) ? -v : v;
        ghost_source(c->bc[1], 1, k, nx, &src, &flip);
        v = Uf[(size_t)j * nx + src];
        Pf[(size_t)(j + G) * px + (G + nx + k)] = (flip && f == 1) ? -v : v;
      }
    for (int i = 0; i < nx; ++i)
      for (int k = 0; k < G; ++k) {
        int src, flip;
        ghost_source(c->bc[2], 0, k, ny, &src, &flip);
        double v = Uf[(size_t)src * nx + i];
        Pf[(size_t)(G - 1 - k) * px + (i + G)] = (flip && f == 2) ? -v : v;
        ghost_source(c->bc[3], 1, k, ny, &src, &flip);
        v = Uf[(size_t)src * nx + i];
        Pf[(size_t)(G + ny + k) * px + (i + G)] = (flip && f == 2) ? -v : v;
      }
  }
  return P;
}

/* --------------------------------------------------------------------------- point physics */

static double pressure(double gamma, double rho, double mx, double my, double E) {
  double u = mx / rho, v = my / rho;
  return (gamma - 1.0) * (E - 0.5 * (mx * u + my * v));
}

static int cell_ok(double rho, double p) { return isfinite(rho) && isfinite(p) && rho > 0.0 && p > 0.0; }

int orc_alpha(const orc_config* c, const double* U, double* ax, double* ay) {
  if (orc_validate(c)) return ORC_EINVAL;
  const size_t n = (size_t)c->nx * c->ny;
  double mx_ = 0.0, my_ = 0.0;
  int bad = 0;
  for (size_t k = 0; k < n; ++k) {
    double rho = U[k], mx = U[n + k], my = U[2 * n + k], E = U[3 * n + k];
    double p = pressure(c->gamma, rho, mx, my, E);
    if (!cell_ok(rho, p)) { bad = 1; continue; }
    double cs = sqrt(c->gamma * p / rho);
    double sx = fabs(mx / rho) + cs, sy = fabs(my / rho) + cs;
    if (sx > mx_) mx_ = sx;
    if (sy > my_) my_ = sy;
  }
  *ax = mx_;
  *ay = my_;
  return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

int orc_max_speed(const orc_config* c, const double* U, double* smax) {
  if (orc_validate(c)) return ORC_EINVAL;
  const size_t n = (size_t)c->nx * c->ny;
  double m = 0.0;
  int bad = 0;
  for (size_t k = 0; k < n; ++k) {
    double rho = U[k], mx = U[n + k], my = U[2 * n + k], E = U[3 * n + k];
    double p = pressure(c->gamma, rho, mx, my, E);
    if (!cell_ok(rho, p)) { bad = 1; continue; }
    double s = sqrt(c->gamma * p / rho) + fabs(mx / rho) + fabs(my / rho);
    if (s > m) m = s;
  }
  *smax = m;
  return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

int orc_dt(const orc_config* c, const double* U, double* dt) {
  double s;
  int rc = orc_max_speed(c, U, &s);
  if (rc) return rc;
  const double dx = (c->x1 - c->x0) / c->nx, dy = (c->y1 - c->y0) / c->ny;
  *dt = c->cfl * (dx < dy ? dx : dy) / s;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ spatial operator */

/* Physical flux of the 4 hydro components along direction dir (0 x, 1 y) at one point. */
static void euler_flux(int dir, double gamma, const double Uc[4], double F[4]) {
  double rho = Uc[0], mx = Uc[1], my = Uc[2], E = Uc[3];
  double u = mx / rho, v = my / rho;
  double p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v));
  if (dir == 0) {
    F[0] = mx;
    F[1] = mx * u + p;
    F[2] = my * u;
    F[3] = (E + p) * u;
  } else {
    F[0] = my;
    F[1] = mx * v;
    F[2] = my * v + p;
    F[3] = (E + p) * v;
  }
}

#include "hydro_oracle_char.inc"

/* Flux difference (fhat_{m+1/2} - fhat_{m-1/2}) / h along one line of n cells for the 4 hydro
 * components. line[c][k] holds component c at line index k - G (k = 0 .. n + 2G - 1). */
static void line_divergence(int dir, double gamma, double alpha, double h, int n, double* const line[4],
                            double* const out[4], double* work, int scheme) {
  const int m = n + 2 * G;
  if (scheme == 1) { /* characteristic-wise: face fluxes from the Roe-averaged eigen-system */
    double* fh = work + 8 * m;
    for (int f = 0; f <= n; ++f) {
      double o[4];
      char_face_flux(dir, gamma, alpha, line, f - 1 + G, o);
      for (int cc = 0; cc < 4; ++cc) fh[cc * (n + 1) + f] = o[cc];
    }
    for (int cc = 0; cc < 4; ++cc)
      for (int i = 0; i < n; ++i) out[cc][i] = (fh[cc * (n + 1) + i + 1] - fh[cc * (n + 1) + i]) / h;
    return;
  }
  double* fp = work;          /* [4][m] positive split flux */
  double* fm = work + 4 * m;  /* [4][m] negative split flux */
  double* fh = work + 8 * m;  /* [4][n+1] numerical flux at faces -1/2 .. n-1/2 */
  for (int k = 0; k < m; ++k) {
    double Uc[4] = {line[0][k], line[1][k], line[2][k], line[3][k]}, F[4];
    euler_flux(dir, gamma, Uc, F);
    for (int cc = 0; cc < 4; ++cc) {
      fp[cc * m + k] = 0.5 * (F[cc] + alpha * Uc[cc]);
      fm[cc * m + k] = 0.5 * (F[cc] - alpha * Uc[cc]);
    }
  }
  for (int cc = 0; cc < 4; ++cc) {
    const double* p = fp + cc * m;
    const double* q = fm + cc * m;
    for (int f = 0; f <= n; ++f) {
      int l = f - 1 + G; /* padded index of the cell left of face f - 1/2 */
      double plus = orc_weno5(p[l - 2], p[l - 1], p[l], p[l + 1], p[l + 2]);
      double minus = orc_weno5(q[l + 3], q[l + 2], q[l + 1], q[l], q[l - 1]);
      fh[cc * (n + 1) + f] = plus + minus;
    }
    for (int i = 0; i < n; ++i) out[cc][i] = (fh[cc * (n + 1) + i + 1] - fh[cc * (n + 1) + i]) / h;
  }
}

/* One-sided HJ-WENO5 derivatives of phi along one line (Jiang & Peng 2000): dm = left-biased,
 * dp = right-biased, from the undivided differences of the padded line. */
static void line_phi_derivatives(double h, int n, const double* phi, double* dm, double* dp, double* work) {
  const int m = n + 2 * G;
  double* D = work; /* D[k] = (phi[k+1] - phi[k]) / h, k = 0 .. m-2 (padded indices) */
  for (int k = 0; k + 1 < m; ++k) D[k] = (phi[k + 1] - phi[k]) / h;
  for (int i = 0; i < n; ++i) {
    int k = i + G; /* padded index of the cell */
    dm[i] = orc_weno5(D[k - 3], D[k - 2], D[k - 1], D[k], D[k + 1]);
    dp[i] = orc_weno5(D[k + 2], D[k + 1], D[k], D[k - 1], D[k - 2]);
  }
}

int orc_rhs(const orc_config* c, const double* U, double ax, double ay, double* L) {
  if (orc_validate(c)) return ORC_EINVAL;
  const int nx = c->nx, ny = c->ny, nf = c->nfields;
  const int px = nx + 2 * G, py = ny + 2 * G;
  const size_t n = (size_t)nx * ny, pn = (size_t)px * py;
  const double dx = (c->x1 - c->x0) / nx, dy = (c->y1 - c->y0) / ny;
  double* P = make_padded(c, U);
  double* dF = (double*)malloc(sizeof(double) * 4 * n);
  double* dG = (double*)malloc(sizeof(double) * 4 * n);
  double* phd = (double*)malloc(sizeof(double) * 4 * n); /* phi_x-, phi_x+, phi_y-, phi_y+ */
  if (!P || !dF || !dG || !phd) {
    free(P); free(dF); free(dG); free(phd);
    return ORC_EINVAL;
  }

  /* x sweep: one row at a time */
#pragma omp parallel
  {
    const int m = px;
    double* line = (double*)malloc(sizeof(double) * 5 * m);
    double* out = (double*)malloc(sizeof(double) * 4 * nx);
    double* work = (double*)malloc(sizeof(double) * (8 * m + 4 * (nx + 1) + m));
#pragma omp for schedule(static)
    for (int j = 0; j < ny; ++j) {
      double* lp[4];
      double* op[4];
      for (int cc = 0; cc < 4; ++cc) {
        lp[cc] = line + cc * m;
        op[cc] = out + cc * nx;
        memcpy(lp[cc], P + cc * pn + (size_t)(j + G) * px, sizeof(double) * m);
      }
      line_divergence(0, c->gamma, ax, dx, nx, lp, op, work, c->scheme);
      for (int cc = 0; cc < 4; ++cc) memcpy(dF + cc * n + (size_t)j * nx, op[cc], sizeof(double) * nx);
      if (nf == 5) {
        double* ph = line + 4 * m;
        memcpy(ph, P + 4 * pn + (size_t)(j + G) * px, sizeof(double) * m);
        line_phi_derivatives(dx, nx, ph, phd + 0 * n + (size_t)j * nx, phd + 1 * n + (size_t)j * nx, work);
      }
    }
    free(line); free(out); free(work);
  }

  /* y sweep: one column at a time */
#pragma omp parallel
  {
    const int m = py;
    double* line = (double*)malloc(sizeof(double) * 5 * m);
    double* out = (double*)malloc(sizeof(double) * 4 * ny);
    double* work = (double*)malloc(sizeof(double) * (8 * m + 4 * (ny + 1) + m));
    double* dm = (double*)malloc(sizeof(double) * ny);
    double* dp = (double*)malloc(sizeof(double) * ny);
#pragma omp for schedule(static)
    for (int i = 0; i < nx; ++i) {
      double* lp[4];
      double* op[4];
      for (int cc = 0; cc < 4; ++cc) {
        lp[cc] = line + cc * m;
        op[cc] = out + cc * ny;
        for (int k = 0; k < m; ++k) lp[cc][k] = P[cc * pn + (size_t)k * px + (i + G)];
      }
      line_divergence(1, c->gamma, ay, dy, ny, lp, op, work, c->scheme);
      for (int cc = 0; cc < 4; ++cc)
        for (int j = 0; j < ny; ++j) dG[cc * n + (size_t)j * nx + i] = op[cc][j];
      if (nf == 5) {
        double* ph = line + 4 * m;
        for (int k = 0; k < m; ++k) ph[k] = P[4 * pn + (size_t)k * px + (i + G)];
        line_phi_derivatives(dy, ny, ph, dm, dp, work);
        for (int j = 0; j < ny; ++j) {
          phd[2 * n + (size_t)j * nx + i] = dm[j];
          phd[3 * n + (size_t)j * nx + i] = dp[j];
        }
      }
    }
    free(line); free(out); free(work); free(dm); free(dp);
  }

  /* combine: L = -(dF/dx + dG/dy) + S ; level set L_phi = -H_hat */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)j * nx + i;
      double rho = U[k], mx = U[n + k], my = U[2 * n + k], E = U[3 * n + k];
      double u = mx / rho, v = my / rho;
      double p = (c->gamma - 1.0) * (E - 0.5 * (mx * u + my * v));
      double S[4] = {0.0, 0.0, 0.0, 0.0};
      if (c->geometry == 1) { /* (r,z): -(1/r)(rho v_r, rho v_r^2, rho v_r v_z, (tau + p) v_r) */
        double r = c->x0 + (i + 0.5) * dx;
        S[0] = -mx / r;
        S[1] = -(mx * u) / r;
        S[2] = -(mx * v) / r;
        S[3] = -((E + p) * u) / r;
      }
      if (c->gravity != 0.0) { /* -rho dPhi/dz and -rho v_z dPhi/dz with dPhi/dz = -g */
        S[2] += rho * c->gravity;
        S[3] += my * c->gravity;
      }
      for (int cc = 0; cc < 4; ++cc) L[cc * n + k] = -(dF[cc * n + k] + dG[cc * n + k]) + S[cc];
      if (nf == 5) {
        double xm = phd[k], xp = phd[n + k], ym = phd[2 * n + k], yp = phd[3 * n + k];
        double sf = c->flame_speed;
        double gx = 0.5 * (xm + xp), gy = 0.5 * (ym + yp);
        double H = (u * gx + v * gy) - sf * sqrt(gx * gx + gy * gy);
        double axl = fabs(u) + sf, ayl = fabs(v) + sf;
        double Hhat = H - (0.5 * axl * (xp - xm) + 0.5 * ayl * (yp - ym));
        L[4 * n + k] = -Hhat;
      }
    }

  free(P); free(dF); free(dG); free(phd);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------ time stepping */

static int state_ok(const orc_config* c, const double* U) {
  const size_t n = (size_t)c->nx * c->ny;
  for (size_t k = 0; k < n; ++k) {
    double p = pressure(c->gamma, U[k], U[n + k], U[2 * n + k], U[3 * n + k]);
    if (!cell_ok(U[k], p)) return 0;
    if (c->nfields == 5 && !isfinite(U[4 * n + k])) return 0;
  }
  return 1;
}

/* One SSP-RK3 step with the given dt; alphas are taken from the stage inputs unless frozen != NULL. */
static int rk3_step(const orc_config* c, double* U, double dt, const double* frozen, double* alpha_out) {
  const size_t total = (size_t)c->nfields * c->nx * c->ny;
  double* L = (double*)malloc(sizeof(double) * total);
  double* U1 = (double*)malloc(sizeof(double) * total);
  double* U2 = (double*)malloc(sizeof(double) * total);
  int rc = ORC_OK;
  double a[6];
  if (!L || !U1 || !U2) { rc = ORC_EINVAL; goto done; }

  /* stage 1: U1 = U + dt L(U) */
  if (frozen) { a[0] = frozen[0]; a[1] = frozen[1]; }
  else if ((rc = orc_alpha(c, U, &a[0], &a[1]))) goto done;
  if ((rc = orc_rhs(c, U, a[0], a[1], L))) goto done;
  for (size_t k = 0; k < total; ++k) U1[k] = U[k] + dt * L[k];
  if (!state_ok(c, U1)) { rc = ORC_ENONPHYSICAL; goto done; }

  /* stage 2: U2 = 3/4 U + 1/4 (U1 + dt L(U1)) */
  if (frozen) { a[2] = frozen[2]; a[3] = frozen[3]; }
  else if ((rc = orc_alpha(c, U1, &a[2], &a[3]))) goto done;
  if ((rc = orc_rhs(c, U1, a[2], a[3], L))) goto done;
  for (size_t k = 0; k < total; ++k) U2[k] = 0.75 * U[k] + 0.25 * (U1[k] + dt * L[k]);
  if (!state_ok(c, U2)) { rc = ORC_ENONPHYSICAL; goto done; }

  /* stage 3: U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2)) */
  if (frozen) { a[4] = frozen[4]; a[5] = frozen[5]; }
  else if ((rc = orc_alpha(c, U2, &a[4], &a[5]))) goto done;
  if ((rc = orc_rhs(c, U2, a[4], a[5], L))) goto done;
  for (size_t k = 0; k < total; ++k) U[k] = (1.0 / 3.0) * U[k] + (2.0 / 3.0) * (U2[k] + dt * L[k]);
  if (!state_ok(c, U)) { rc = ORC_ENONPHYSICAL; goto done; }
  if (alpha_out) memcpy(alpha_out, a, sizeof a);

done:
  free(L); free(U1); free(U2);
  return rc;
}

/* The paper's five-stage, third-order Runge-Kutta scheme (Sec. 2.1). Its coefficients are in a cited
 * reference, not in the paper; the reading taken is Spiteri & Ruuth's five-stage third-order scheme SSP(5,3)
 * (SIAM J. Numer. Anal. 40, 2002; the coefficients as tabulated by Ruuth, Math. Comp. 75, 2006), in
 * Shu-Osher form: u(0) = U^n, u(i) = sum_{k<i} RK5_A[i-1][k] u(k) + dt sum_{k<i} RK5_B[i-1][k] L(u(k)),
 * U^{n+1} = u(5), every L taken with the Lax-Friedrichs speeds of the state it acts on. */
static const double RK5_A[5][5] = {
    {1.0, 0.0, 0.0, 0.0, 0.0},
    {0.0, 1.0, 0.0, 0.0, 0.0},
    {0.56656131914033, 0.0, 0.43343868085967, 0.0, 0.0},
    {0.09299483444413, 0.00002090369620, 0.0, 0.90698426185967, 0.0},
    {0.00736132260920, 0.20127980325145, 0.00182955389682, 0.0, 0.78952932024253}};
static const double RK5_B[5][5] = {
    {0.37726891511710, 0.0, 0.0, 0.0, 0.0},
    {0.0, 0.37726891511710, 0.0, 0.0, 0.0},
    {0.0, 0.0, 0.16352294089771, 0.0, 0.0},
    {0.00071997378654, 0.0, 0.0, 0.34217696850008, 0.0},
    {0.00277719819460, 0.00001567934613, 0.0, 0.0, 0.29786487010104}};

/* One step of the five-stage scheme with the given dt; alphas from the stage states unless frozen != NULL
 * (frozen[2 k], frozen[2 k + 1] for L(u(k))); alpha_out (may be NULL) receives the 10 alphas used. */
static int rk5_step(const orc_config* c, double* U, double dt, const double* frozen, double* alpha_out) {
  const size_t total = (size_t)c->nfields * c->nx * c->ny;
  double* u[5] = {NULL, NULL, NULL, NULL, NULL};  /* u(0) .. u(4) */
  double* L[5] = {NULL, NULL, NULL, NULL, NULL};  /* L(u(0)) .. L(u(4)) */
  int rc = ORC_OK;
  for (int k = 0; k < 5; ++k) {
    u[k] = (double*)malloc(sizeof(double) * total);
    L[k] = (double*)malloc(sizeof(double) * total);
    if (!u[k] || !L[k]) { rc = ORC_EINVAL; goto done; }
  }
  memcpy(u[0], U, sizeof(double) * total);
  for (int i = 1; i <= 5; ++i) {
    double ax, ay;
    if (frozen) { ax = frozen[2 * (i - 1)]; ay = frozen[2 * (i - 1) + 1]; }
    else if ((rc = orc_alpha(c, u[i - 1], &ax, &ay))) goto done;
    if (alpha_out) { alpha_out[2 * (i - 1)] = ax; alpha_out[2 * (i - 1) + 1] = ay; }
    if ((rc = orc_rhs(c, u[i - 1], ax, ay, L[i - 1]))) goto done;
    double* out = i < 5 ? u[i] : U;
    for (size_t q = 0; q < total; ++q) {
      double v = 0.0, w = 0.0;
      for (int k = 0; k < i; ++k) {
        v += RK5_A[i - 1][k] * u[k][q];
        w += RK5_B[i - 1][k] * L[k][q];
      }
      out[q] = v + dt * w;
    }
    if (!state_ok(c, out)) { rc = ORC_ENONPHYSICAL; goto done; }
  }
done:
  for (int k = 0; k < 5; ++k) { free(u[k]); free(L[k]); }
  return rc;
}

int orc_step(const orc_config* c, double* U, int nsteps, double* t, double* dt_last, double* dt_log,
             double* alpha_log) {
  if (orc_validate(c) || !U || nsteps < 0) return ORC_EINVAL;
  for (int s = 0; s < nsteps; ++s) {
    double dt;
    int rc = orc_dt(c, U, &dt);
    if (rc) return rc;
    rc = c->rk_stages == 5 ? rk5_step(c, U, dt, NULL, alpha_log ? alpha_log + 10 * s : NULL)
                           : rk3_step(c, U, dt, NULL, alpha_log ? alpha_log + 6 * s : NULL);
    if (rc) return rc;
    if (dt_log) dt_log[s] = dt;
    if (t) *t += dt;
    if (dt_last) *dt_last = dt;
  }
  return ORC_OK;
}

int orc_step_frozen(const orc_config* c, double* U, int nsteps, const double* dt_log,
                    const double* alpha_log) {
  if (orc_validate(c) || !U || nsteps < 0 || !dt_log || !alpha_log) return ORC_EINVAL;
  for (int s = 0; s < nsteps; ++s) {
    int rc = c->rk_stages == 5 ? rk5_step(c, U, dt_log[s], alpha_log + 10 * s, NULL)
                               : rk3_step(c, U, dt_log[s], alpha_log + 6 * s, NULL);
    if (rc) return rc;
  }
  return ORC_OK;
}

int orc_totals(const orc_config* c, const double* U, double out[5]) {
  if (orc_validate(c)) return ORC_EINVAL;
  const int nx = c->nx, ny = c->ny;
  const size_t n = (size_t)nx * ny;
  const double dx = (c->x1 - c->x0) / nx, dy = (c->y1 - c->y0) / ny;
  const double two_pi = 6.283185307179586476925286766559;
  for (int f = 0; f < 5; ++f) {
    double s = 0.0;
    if (f < c->nfields)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double dV = c->geometry == 1 ? two_pi * (c->x0 + (i + 0.5) * dx) * dx * dy : dx * dy;
          s += U[f * n + (size_t)j * nx + i] * dV;
        }
    out[f] = s;
  }
  return ORC_OK;
}

#include "hydro_oracle_adjoint.inc"
#include "hydro_oracle_reinit.inc"
#include "hydro_oracle_poisson.inc"
