// adjoint_kernel.cuh -- discrete adjoint of one SSP-RK3 stage of the WENO5 / Lax-Friedrichs update
// with the level set (Leung, Chu & Lin 2015, Sec. 2.1-2.2), dt and the Lax-Friedrichs speeds frozen.
//
// A stage maps its input W to V = a U^n + b (W + dt L(W)). Given nu = dJ/dV the adjoint is
//   dJ/dW = b (nu + dt J_L(W)^T nu),   dJ/dU^n += a nu.
// J_L^T nu is assembled in three launches:
//   adj_point_kernel   per interior cell: the point terms -- (r,z) and gravity sources, and the level
//                      set's local Lax-Friedrichs Hamiltonian, whose adjoint w.r.t. its four one-sided
//                      derivatives (hb) is stored for the line pass and w.r.t. u, v goes to the cell;
//   adj_line_kernel    tiles over the padded grid INCLUDING its ghost frame: for every point, the
//                      face adjoints (nu_f - nu_{f-1}) / h of the six faces whose WENO5 stencils contain
//                      it, times the WENO5 gradients, through the Lax-Friedrichs split and the Euler
//                      flux Jacobian; and the level-set adjoint through the HJ-WENO5 gradients;
//   adj_blend_kernel   per interior cell: folds the ghost-frame adjoints back onto the cells they are
//                      images of (the adjoint of the boundary fill) and applies the RK blend.
// nu and hb are zero outside the interior, so faces outside the grid contribute nothing; such faces
// are skipped (their stencils may reach unfilled corner points).
#pragma once
#include "stage_kernel.cuh"

namespace hydro {

// gbar * dW/dv of the WENO5-JS value W(a, b, c, d, e) (Jiang & Shu weights), added to g[0..4].
// With D_k = eps + beta_k, alpha_k = d_k / D_k^2, w_k = alpha_k / sum alpha:
//   dW/dv = sum_k w_k dq_k/dv + sum_k (q_k - W) / sum alpha * dalpha_k/dbeta_k * dbeta_k/dv,
//   dalpha_k/dbeta_k = -2 alpha_k / D_k,  dbeta_k/dv = 13/6 s_k ds_k/dv + 1/2 t_k dt_k/dv.
// FP32 forms the four reciprocals 1/D_k and 1/sum alpha with approximate reciprocals and folds the 1/6 of
// the candidate values into their coefficients; FP64 keeps true divisions.
template <typename real>
__device__ __forceinline__ void weno5_grad_acc(real a, real b, real c, real d, real e, real gbar, real& ga,
                                               real& gb, real& gc, real& gd, real& ge) {
  const real s0 = a - real(2) * b + c, t0 = a - real(4) * b + real(3) * c;
  const real s1 = b - real(2) * c + d, t1 = b - d;
  const real s2 = c - real(2) * d + e, t2 = real(3) * c - real(4) * d + e;
  const real D0 = real(1e-6) + real(13.0 / 12.0) * s0 * s0 + real(0.25) * t0 * t0;
  const real D1 = real(1e-6) + real(13.0 / 12.0) * s1 * s1 + real(0.25) * t1 * t1;
  const real D2 = real(1e-6) + real(13.0 / 12.0) * s2 * s2 + real(0.25) * t2 * t2;
  real q0, q1, q2, a0, a1, a2, rS, n0, n1, n2;  // n_k = -2 alpha_k / D_k
  if constexpr (sizeof(real) == 4) {
    using T = RT<float>;
    q0 = T::fma_(real(1.0 / 3.0), a, T::fma_(real(-7.0 / 6.0), b, real(11.0 / 6.0) * c));
    q1 = T::fma_(real(-1.0 / 6.0), b, T::fma_(real(5.0 / 6.0), c, real(1.0 / 3.0) * d));
    q2 = T::fma_(real(1.0 / 3.0), c, T::fma_(real(5.0 / 6.0), d, real(-1.0 / 6.0) * e));
    const real r0 = T::rcp(D0), r1 = T::rcp(D1), r2 = T::rcp(D2);
    a0 = real(0.1) * r0 * r0;
    a1 = real(0.6) * r1 * r1;
    a2 = real(0.3) * r2 * r2;
    rS = T::rcp(a0 + a1 + a2);
    n0 = real(-2) * a0 * r0;
    n1 = real(-2) * a1 * r1;
    n2 = real(-2) * a2 * r2;
  } else {
    q0 = (real(2) * a - real(7) * b + real(11) * c) / real(6);
    q1 = (-b + real(5) * c + real(2) * d) / real(6);
    q2 = (real(2) * c + real(5) * d - e) / real(6);
    a0 = real(0.1) / (D0 * D0);
    a1 = real(0.6) / (D1 * D1);
    a2 = real(0.3) / (D2 * D2);
    rS = real(1) / (a0 + a1 + a2);
    n0 = real(-2) * a0 / D0;
    n1 = real(-2) * a1 / D1;
    n2 = real(-2) * a2 / D2;
  }
  const real w0 = a0 * rS, w1 = a1 * rS, w2 = a2 * rS;
  const real W = w0 * q0 + w1 * q1 + w2 * q2;
  const real c0 = (q0 - W) * rS * n0;
  const real c1 = (q1 - W) * rS * n1;
  const real c2 = (q2 - W) * rS * n2;
  const real A0 = c0 * real(13.0 / 6.0) * s0, B0 = c0 * real(0.5) * t0;
  const real A1 = c1 * real(13.0 / 6.0) * s1, B1 = c1 * real(0.5) * t1;
  const real A2 = c2 * real(13.0 / 6.0) * s2, B2 = c2 * real(0.5) * t2;
  const real k6 = real(1) / real(6);
  ga += gbar * (w0 * (real(2) * k6) + A0 + B0);
  gb += gbar * (w0 * (real(-7) * k6) + w1 * (-k6) - real(2) * A0 - real(4) * B0 + A1 + B1);
  gc += gbar * (w0 * (real(11) * k6) + w1 * (real(5) * k6) + w2 * (real(2) * k6) + A0 + real(3) * B0 -
                real(2) * A1 + A2 + real(3) * B2);
  gd += gbar * (w1 * (real(2) * k6) + w2 * (real(5) * k6) + A1 - B1 - real(2) * A2 - real(4) * B2);
  ge += gbar * (w2 * (-k6) + A2 + B2);
}

template <typename real>
__device__ __forceinline__ real weno5_plain(real a, real b, real c, real d, real e) {
  if constexpr (sizeof(real) == 4) {  // FP32: shared smoothness data (the stage kernel's weights up to rounding)
    return weno_side(a, b, c, d, e, betas(a, b, c).m, betas(b, c, d).t, betas(c, d, e).p);
  } else {
    const real q0 = (real(2) * a - real(7) * b + real(11) * c) / real(6);
    const real q1 = (-b + real(5) * c + real(2) * d) / real(6);
    const real q2 = (real(2) * c + real(5) * d - e) / real(6);
    const real s0 = a - real(2) * b + c, t0 = a - real(4) * b + real(3) * c;
    const real s1 = b - real(2) * c + d, t1 = b - d;
    const real s2 = c - real(2) * d + e, t2 = real(3) * c - real(4) * d + e;
    const real D0 = real(1e-6) + real(13.0 / 12.0) * s0 * s0 + real(0.25) * t0 * t0;
    const real D1 = real(1e-6) + real(13.0 / 12.0) * s1 * s1 + real(0.25) * t1 * t1;
    const real D2 = real(1e-6) + real(13.0 / 12.0) * s2 * s2 + real(0.25) * t2 * t2;
    const real a0 = real(0.1) / (D0 * D0), a1 = real(0.6) / (D1 * D1), a2 = real(0.3) / (D2 * D2);
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
  }
}

// dF_r/dU_s of the Euler flux along x (dir 0) or y (dir 1) at one state.
template <typename real>
__device__ __forceinline__ void flux_jacobian(int dir, real gamma, real rho, real mx, real my, real E,
                                              real J[4][4]) {
  real rr;  // 1 / rho
  if constexpr (sizeof(real) == 4)
    rr = RT<float>::rcp(rho);
  else
    rr = real(1) / rho;
  const real u = sizeof(real) == 4 ? mx * rr : mx / rho, v = sizeof(real) == 4 ? my * rr : my / rho;
  const real gm1 = gamma - real(1);
  const real p = gm1 * (E - real(0.5) * (mx * u + my * v));
  const real dp[4] = {gm1 * real(0.5) * (u * u + v * v), -gm1 * u, -gm1 * v, gm1};
  const real du[4] = {sizeof(real) == 4 ? -u * rr : -u / rho, rr, real(0), real(0)};
  const real dv[4] = {sizeof(real) == 4 ? -v * rr : -v / rho, real(0), rr, real(0)};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const real dmx = (s == 1) ? real(1) : real(0), dmy = (s == 2) ? real(1) : real(0);
    const real dE = (s == 3) ? real(1) : real(0);
    if (dir == 0) {
      J[0][s] = dmx;
      J[1][s] = dmx * u + mx * du[s] + dp[s];
      J[2][s] = dmy * u + my * du[s];
      J[3][s] = (dE + dp[s]) * u + (E + p) * du[s];
    } else {
      J[0][s] = dmy;
      J[1][s] = dmx * v + mx * dv[s];
      J[2][s] = dmy * v + my * dv[s] + dp[s];
      J[3][s] = (dE + dp[s]) * v + (E + p) * dv[s];
    }
  }
}

template <typename real>
struct AdjParams {
  const real* W;     // stage input state (padded, ghosts filled)
  const real* nu;    // dJ/dV (padded, zero outside the interior)
  real* mu;          // J_L^T nu on the padded grid including the ghost frame
  real* hb;          // [4] level-set Hamiltonian adjoints w.r.t. phi_x^-, phi_x^+, phi_y^-, phi_y^+ (padded)
  real* out;         // dJ/dW = b (nu + dt mu_folded) (padded, interior written)
  real* acc;         // dJ/dU^n accumulator (padded, interior)
  long long fstride;
  int nx, ny, pitch, rows;
  int bc[4];
  int geometry;
  real gamma, gravity, flame_speed, ax, ay;
  double dx, dy, x0, dt, a, b;
  // the same in the working precision, formed on the host (no FP64 arithmetic in the FP32 kernels)
  real rdx_r, rdy_r, dx_r, x0_r, dt_r, a_r, b_r;
  int acc_mode;      // 0: acc = a nu ; 1: acc += a nu ; 2: acc += out (final stage), write out too
  int tile_rows;     // line-adjoint tile rows: 16, 32 (FP32 only), or 0 for the size rule
};

// ---------------------------------------------------------------------------- point terms

// FP32 one-sided derivatives of one cell from its six differences d[0..5] (d[3] is the cell's right
// difference): phi^- = W(d0 .. d4), phi^+ = W(d5 .. d1), the four difference triplets formed once.
__device__ __forceinline__ void phi_derivs_f32(const float (&d)[6], float& dm, float& dp) {
  constexpr float EPS = 1e-6f * TRI_EPS_SCALE;
  TriD32 t[5];
  Tri32 l[5], r[5];
#pragma unroll
  for (int j = 1; j <= 4; ++j) {
    t[j] = tri_data(d[j - 1], d[j], d[j + 1], EPS);
    l[j] = tri_roles(t[j], true);
    r[j] = tri_roles(t[j], false);
  }
  dm = tri_face(l[1].up, l[2].mid, l[3].down);
  dp = tri_face(r[4].up, r[3].mid, r[2].down);
}

template <typename real, int NF>
__global__ void __launch_bounds__(256) adj_point_kernel(AdjParams<real> P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= P.nx) return;
  const long long fs = P.fstride;
  const long long k = static_cast<long long>(j + GY) * P.pitch + i + GX;
  const real rho = P.W[k], mx = P.W[fs + k], my = P.W[2 * fs + k], E = P.W[3 * fs + k];
  // 1 / rho: an approximate reciprocal in FP32, a true division in FP64
  const real rr = sizeof(real) == 4 ? static_cast<real>(RT<float>::rcp(static_cast<float>(rho))) : real(1) / rho;
  const real u = sizeof(real) == 4 ? mx * rr : mx / rho, v = sizeof(real) == 4 ? my * rr : my / rho;
  const real p = (P.gamma - real(1)) * (E - real(0.5) * (mx * u + my * v));
  real nu[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) nu[f] = P.nu[f * fs + k];
  real g[4] = {real(0), real(0), real(0), real(0)};
  if (P.geometry == 1) {  // sources -(1/r)(m_r, m_r u, m_r v, (E + p) u)
    const real r = sizeof(real) == 4 ? P.x0_r + (static_cast<real>(i) + real(0.5)) * P.dx_r
                                     : static_cast<real>(P.x0 + (i + 0.5) * P.dx);
    real J[4][4];
    flux_jacobian<real>(0, P.gamma, rho, mx, my, E, J);
    real JS[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      JS[0][s] = -((s == 1) ? real(1) : real(0)) / r;
      JS[1][s] = -(((s == 1) ? u : real(0)) + mx * ((s == 0) ? -u / rho : (s == 1) ? real(1) / rho : real(0))) / r;
      JS[2][s] = -(((s == 1) ? v : real(0)) + mx * ((s == 0) ? -v / rho : (s == 2) ? real(1) / rho : real(0))) / r;
      JS[3][s] = -J[3][s] / r;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) g[s] += JS[q][s] * nu[q];
  }
  if (P.gravity != real(0)) {
    g[0] += P.gravity * nu[2];
    g[2] += P.gravity * nu[3];
  }
  (void)p;
  if constexpr (NF == 5) {
    const real* ph = P.W + 4 * fs + k;
    const real rdx = P.rdx_r, rdy = P.rdy_r;
    real dxs[6], dys[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      dxs[q] = (ph[q - 2] - ph[q - 3]) * rdx;                          // D_{i-3+q}
      dys[q] = (ph[(q - 2) * P.pitch] - ph[(q - 3) * P.pitch]) * rdy;  // D_{j-3+q}
    }
    real xm, xq, ym, yq, Hgx, Hgy;
    const real sf = P.flame_speed;
    if constexpr (sizeof(real) == 4) {  // the stage kernel's FP32 one-sided derivatives (triplet form)
      phi_derivs_f32(dxs, xm, xq);
      phi_derivs_f32(dys, ym, yq);
      const real gx = real(0.5) * (xm + xq), gy = real(0.5) * (ym + yq);
      const real n2 = gx * gx + gy * gy;
      const real rn = n2 > real(0) ? RT<float>::rcp(RT<float>::sqrt_(n2)) : real(0);
      Hgx = u - sf * gx * rn;
      Hgy = v - sf * gy * rn;
    } else {
      xm = weno5_plain(dxs[0], dxs[1], dxs[2], dxs[3], dxs[4]);
      xq = weno5_plain(dxs[5], dxs[4], dxs[3], dxs[2], dxs[1]);
      ym = weno5_plain(dys[0], dys[1], dys[2], dys[3], dys[4]);
      yq = weno5_plain(dys[5], dys[4], dys[3], dys[2], dys[1]);
      const real gx = real(0.5) * (xm + xq), gy = real(0.5) * (ym + yq);
      const real nrm = sqrt(gx * gx + gy * gy);
      Hgx = u - (nrm > real(0) ? sf * gx / nrm : real(0));
      Hgy = v - (nrm > real(0) ? sf * gy / nrm : real(0));
    }
    const real gx = real(0.5) * (xm + xq), gy = real(0.5) * (ym + yq);
    const real axl = fabs(u) + sf, ayl = fabs(v) + sf;
    const real hbar = -nu[4];  // L_phi = -H_hat
    P.hb[0 * fs + k] = hbar * (real(0.5) * Hgx + real(0.5) * axl);
    P.hb[1 * fs + k] = hbar * (real(0.5) * Hgx - real(0.5) * axl);
    P.hb[2 * fs + k] = hbar * (real(0.5) * Hgy + real(0.5) * ayl);
    P.hb[3 * fs + k] = hbar * (real(0.5) * Hgy - real(0.5) * ayl);
    const real su = u > real(0) ? real(1) : (u < real(0) ? real(-1) : real(0));
    const real sv = v > real(0) ? real(1) : (v < real(0) ? real(-1) : real(0));
    const real ub = hbar * (gx - su * real(0.5) * (xq - xm));
    const real vb = hbar * (gy - sv * real(0.5) * (yq - ym));
    if constexpr (sizeof(real) == 4) {
      g[0] -= (ub * u + vb * v) * rr;
      g[1] += ub * rr;
      g[2] += vb * rr;
    } else {
      g[0] += ub * (-u / rho) + vb * (-v / rho);
      g[1] += ub / rho;
      g[2] += vb / rho;
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) P.mu[s * fs + k] = g[s];
  if constexpr (NF == 5) P.mu[4 * fs + k] = real(0);
}

// ---------------------------------------------------------------------------- line adjoints

constexpr int ATX = 32, ARUN = 8;   // output columns per tile, points per line item
// output rows per tile TY: 16 (two CTAs of NF x 64 threads per SM in FP32), or 32 for FP32 grids with at
// least one such tile per SM (one CTA of NF x 128 threads per SM, every warp in the same phase of the tile, a
// box of 45 x 44 points for 32 x 32 outputs); FP64 16 rows, 256 threads
// threads per CTA: one line item each in both passes (NF x 4 TY items) for FP32
template <typename real, int NF, int TY>
__host__ __device__ constexpr int adj_threads() { return sizeof(real) == 4 ? NF * 4 * TY : 256; }
constexpr int AHX = 6;                        // box halo (hydro needs 5, level set 6)
// box rows of odd length and output rows of ATX + 1: the rows of an x-pass warp (32 rows of one run, or 16
// rows x 2 runs 16 columns apart) fall on 32 distinct banks, and so do the run outputs the lanes write
constexpr int ABW = ATX + 2 * AHX + 1, AOS = ATX + 1;

template <typename real, int NF, int TY>
struct ATile {
  static constexpr int ATY = TY, ABH = ATY + 2 * AHX;
  static constexpr int BOX = ABW * ABH;
  static constexpr int OFF_W = 0;                        // [NF][ABH][ABW] state
  static constexpr int OFF_P = OFF_W + NF * BOX;         // [3][ABH][ABW]  u, v, p
  static constexpr int OFF_N = OFF_P + 3 * BOX;          // [NF][ABH][ABW] nu
  static constexpr int OFF_H = OFF_N + NF * BOX;         // [4][ABH][ABW]  hb (level set)
  static constexpr int OFF_PB = OFF_H + (NF == 5 ? 4 * BOX : 0);  // [4][ATY][AOS] f+bar + f-bar
  static constexpr int OFF_MB = OFF_PB + 4 * ATY * AOS;  // [4][ATY][AOS] f+bar - f-bar
  static constexpr int OFF_MU = OFF_MB + 4 * ATY * AOS;  // [NF][ATY][AOS] accumulated mu
  static constexpr int ELEMS = OFF_MU + NF * ATY * AOS;
  static constexpr size_t BYTES = ELEMS * sizeof(real);
};

// ---- FP32 line adjoints in triplet form. A point triplet (L, C, R) serves three faces of one
// reconstruction direction, as their upwind-most, central and downwind-most stencil ("up", "mid", "dn").
// With s = (L + R) - 2C, t = L - R and h_r the role's t_r / 2 (s - t/2, t/2, s + t/2 from the left; s + t/2,
// -t/2, s - t/2 from the right), the role's candidate value is q_r, its indicator D_r = eps + 13/12 s^2
// + h_r^2, its weight a_r = d_r / D_r^2 (linear weights 1, 6, 3) and n_r = a_r / D_r. These are formed
// once per triplet. A face with cotangent gbar then needs W = sum a_r q_r / sum a_r and, per role,
//   gbar dW/d(a', b', c') = WG dq_r + A (1, -2, 1) + B dt_r,
//   WG = gbar a_r / sum a,  cg = -2 gbar (q_r - W) n_r / sum a,  A = 13/6 s cg,  B = h_r cg,
// on the role's three points in reconstruction order, with dq_r = (2, -7, 11)/6, (-1, 5, 2)/6, (2, 5, -1)/6
// and dt_r = (1, -4, 3), (1, 0, -1), (3, -4, 1) for up, mid, dn (Jiang & Shu's candidate values and
// smoothness indicators differentiated). q_r - W is not formed as a difference of the two (close on
// smooth data, so its FP32 rounding would be amplified): with w_r = a_r / sum a, the candidate
// differences q_up - q_mid = (s_up - s_mid) / 3 and q_mid - q_dn = (s_dn - s_mid) / 6 (exact identities of
// the candidate values) give q_up - W = w_mid D01 + w_dn D02, q_mid - W = w_dn D12 - w_up D01,
// q_dn - W = -(w_up D02 + w_mid D12), from the triplets' second differences s.
struct ARole {
  float a, nr, h;  // weight, weight / D, the role's half-difference h_r
};
struct ATri {
  ARole up, mid, dn;
  float s13;  // 13/6 s
};
struct ATriData {
  float s, th, mm, pp, rm, rt, rp;
};
__device__ __forceinline__ ATriData adj_tri_data(float L, float C, float R) {
  using T = RT<float>;
  ATriData d;
  d.s = T::fma_(-2.0f, C, L + R);
  d.th = 0.5f * (L - R);
  const float bs = T::fma_((13.0f / 12.0f) * d.s, d.s, 1e-6f);
  d.mm = d.s - d.th;
  d.pp = d.s + d.th;
  d.rm = T::rcp(T::fma_(d.mm, d.mm, bs));
  d.rt = T::rcp(T::fma_(d.th, d.th, bs));
  d.rp = T::rcp(T::fma_(d.pp, d.pp, bs));
  return d;
}
__device__ __forceinline__ ATri adj_tri_roles(const ATriData& d, bool left_to_right) {
  const float at = 6.0f * d.rt * d.rt;
  ATri r;
  r.s13 = (13.0f / 6.0f) * d.s;
  if (left_to_right) {
    r.up = {d.rm * d.rm, 0.0f, d.mm};
    r.up.nr = r.up.a * d.rm;
    r.mid = {at, at * d.rt, d.th};
    r.dn = {3.0f * d.rp * d.rp, 0.0f, d.pp};
    r.dn.nr = r.dn.a * d.rp;
  } else {
    r.up = {d.rp * d.rp, 0.0f, d.pp};
    r.up.nr = r.up.a * d.rp;
    r.mid = {at, at * d.rt, -d.th};
    r.dn = {3.0f * d.rm * d.rm, 0.0f, d.mm};
    r.dn.nr = r.dn.a * d.rm;
  }
  return r;
}
// One role's share of a face's gradient onto its points (reconstruction order a', b', c').
template <int ROLE>
__device__ __forceinline__ void adj_role(const ARole& r, float s13, float qmw, float g, float m2g, float& ga,
                                         float& gb, float& gc) {
  using T = RT<float>;
  constexpr float q0 = ROLE == 0 ? 2.0f / 6.0f : ROLE == 1 ? -1.0f / 6.0f : 2.0f / 6.0f;
  constexpr float q1 = ROLE == 0 ? -7.0f / 6.0f : 5.0f / 6.0f;
  constexpr float q2 = ROLE == 0 ? 11.0f / 6.0f : ROLE == 1 ? 2.0f / 6.0f : -1.0f / 6.0f;
  constexpr float t0 = ROLE == 2 ? 3.0f : 1.0f;
  constexpr float t1 = ROLE == 1 ? 0.0f : -4.0f;
  constexpr float t2 = ROLE == 0 ? 3.0f : ROLE == 1 ? -1.0f : 1.0f;
  const float WG = r.a * g;
  const float cg = qmw * r.nr * m2g;  // qmw = q_r - W
  const float A = s13 * cg, B = r.h * cg;
  ga += T::fma_(WG, q0, T::fma_(B, t0, A));
  gb += (ROLE == 1) ? T::fma_(WG, q1, -2.0f * A) : T::fma_(WG, q1, T::fma_(B, t1, -2.0f * A));
  gc += T::fma_(WG, q2, T::fma_(B, t2, A));
}
// A face's q_r - W for its three roles (from the triplets' 13/6 s values, see above), and the gradient
// factors gbar / sum a and -2 gbar / sum a.
__device__ __forceinline__ void adj_face_w(const ARole& u, const ARole& m, const ARole& d, float su13, float sm13,
                                           float sd13, float gbar, float& eu, float& em, float& ed, float& g,
                                           float& m2g) {
  using T = RT<float>;
  const float rS = T::rcp((u.a + m.a) + d.a);
  const float wu = u.a * rS, wm = m.a * rS, wd = d.a * rS;
  const float D01 = (su13 - sm13) * (2.0f / 13.0f);  // q_up - q_mid = (s_up - s_mid) / 3
  const float D12 = (sd13 - sm13) * (1.0f / 13.0f);  // q_mid - q_dn = (s_dn - s_mid) / 6
  const float D02 = D01 + D12;
  eu = T::fma_(wm, D01, wd * D02);
  em = T::fma_(wd, D12, -(wu * D01));
  ed = -T::fma_(wu, D02, wm * D12);
  g = gbar * rS;
  m2g = -2.0f * g;
}

// FP32 hydro line adjoint (same faces, points and outputs as adj_hydro_line below).
__device__ __forceinline__ void adj_hydro_line_f32(const float* __restrict__ Uc, const float* __restrict__ Xc,
                                                   const float* __restrict__ vel, const float* __restrict__ pr,
                                                   const float* __restrict__ nuc, int S, int kind, float alpha,
                                                   float rd, float* __restrict__ pb, float* __restrict__ mb, int DS) {
  constexpr int NP = ARUN + 10;  // points, index m + 5
  float fp[NP], fm[NP], ap[NP], am[NP];
  ATri tp[NP], tm[NP];  // triplets by centre point
  auto point = [&](int q) {
    const int m = q - 5;
    const float uu = Uc[m * S];
    float F;
    if (kind == 0) F = Xc[m * S];
    else {
      const float vn = vel[m * S], p = pr[m * S];
      F = kind == 1 ? uu * vn + p : kind == 2 ? uu * vn : (uu + p) * vn;
    }
    fp[q] = 0.5f * (F + alpha * uu);
    fm[q] = 0.5f * (F - alpha * uu);
    ap[q] = 0.0f;
    am[q] = 0.0f;
  };
#pragma unroll
  for (int q = 0; q < 5; ++q) point(q);  // points -5 .. -1
  tp[1] = adj_tri_roles(adj_tri_data(fp[0], fp[1], fp[2]), true);
  tp[2] = adj_tri_roles(adj_tri_data(fp[1], fp[2], fp[3]), true);
  tm[2] = adj_tri_roles(adj_tri_data(fm[1], fm[2], fm[3]), false);
  tm[3] = adj_tri_roles(adj_tri_data(fm[2], fm[3], fm[4]), false);
#pragma unroll
  for (int f = -2; f <= ARUN + 2; ++f) {
    // face f lies between points f-1 and f; its left-biased stencil is points f-3 .. f+1 (triplets centred
    // at f-2, f-1, f) and its right-biased one f+2 .. f-2 (triplets centred at f+1, f, f-1)
    const int q = f + 5;
    if (q + 2 < NP) point(q + 2);
    tp[q] = adj_tri_roles(adj_tri_data(fp[q - 1], fp[q], fp[q + 1]), true);
    tm[q + 1] = adj_tri_roles(adj_tri_data(fm[q], fm[q + 1], fm[q + 2]), false);
    const float fb = (nuc[f * S] - nuc[(f - 1) * S]) * rd;
    if (fb != 0.0f) {
      float eu, em, ed, g, m2g;
      adj_face_w(tp[q - 2].up, tp[q - 1].mid, tp[q].dn, tp[q - 2].s13, tp[q - 1].s13, tp[q].s13, fb, eu, em, ed, g,
                 m2g);
      adj_role<0>(tp[q - 2].up, tp[q - 2].s13, eu, g, m2g, ap[q - 3], ap[q - 2], ap[q - 1]);
      adj_role<1>(tp[q - 1].mid, tp[q - 1].s13, em, g, m2g, ap[q - 2], ap[q - 1], ap[q]);
      adj_role<2>(tp[q].dn, tp[q].s13, ed, g, m2g, ap[q - 1], ap[q], ap[q + 1]);
      adj_face_w(tm[q + 1].up, tm[q].mid, tm[q - 1].dn, tm[q + 1].s13, tm[q].s13, tm[q - 1].s13, fb, eu, em, ed, g,
                 m2g);
      adj_role<0>(tm[q + 1].up, tm[q + 1].s13, eu, g, m2g, am[q + 2], am[q + 1], am[q]);
      adj_role<1>(tm[q].mid, tm[q].s13, em, g, m2g, am[q + 1], am[q], am[q - 1]);
      adj_role<2>(tm[q - 1].dn, tm[q - 1].s13, ed, g, m2g, am[q], am[q - 1], am[q - 2]);
    }
    const int k = f - 3;  // output point completed by this face
    if (k >= 0 && k < ARUN) {
      pb[k * DS] = ap[k + 5] + am[k + 5];
      mb[k * DS] = ap[k + 5] - am[k + 5];
    }
  }
}

// FP32 level-set line adjoint (same cells and outputs as adj_phi_line below): both one-sided
// derivatives of a cell reconstruct the same differences, so each triplet's data serve both directions.
__device__ __forceinline__ void adj_phi_line_f32(const float* __restrict__ ph, const float* __restrict__ hm,
                                                 const float* __restrict__ hp, int S, float rd, float* __restrict__ dst,
                                                 int DS) {
  constexpr int ND = ARUN + 11;  // differences D_n, n = -6 .. ARUN+4, index n + 6
  float D[ND], Db[ND];
  ATri tl[ND], tr[ND];
  auto diff = [&](int q) {
    const int n = q - 6;
    D[q] = (ph[(n + 1) * S] - ph[n * S]) * rd;
    Db[q] = 0.0f;
  };
  auto tri = [&](int q) {
    const ATriData d = adj_tri_data(D[q - 1], D[q], D[q + 1]);
    tl[q] = adj_tri_roles(d, true);
    tr[q] = adj_tri_roles(d, false);
  };
#pragma unroll
  for (int q = 0; q < 5; ++q) diff(q);
  tri(1);
  tri(2);
  tri(3);
#pragma unroll
  for (int i = -3; i <= ARUN + 2; ++i) {
    const int q = i + 6;
    if (q + 2 < ND) diff(q + 2);
    if (q + 1 < ND - 1) tri(q + 1);
    const float bm = hm[i * S], bp = hp[i * S];
    float eu, em, ed, g, m2g;
    if (bm != 0.0f) {
      adj_face_w(tl[q - 2].up, tl[q - 1].mid, tl[q].dn, tl[q - 2].s13, tl[q - 1].s13, tl[q].s13, bm, eu, em, ed, g,
                 m2g);
      adj_role<0>(tl[q - 2].up, tl[q - 2].s13, eu, g, m2g, Db[q - 3], Db[q - 2], Db[q - 1]);
      adj_role<1>(tl[q - 1].mid, tl[q - 1].s13, em, g, m2g, Db[q - 2], Db[q - 1], Db[q]);
      adj_role<2>(tl[q].dn, tl[q].s13, ed, g, m2g, Db[q - 1], Db[q], Db[q + 1]);
    }
    if (bp != 0.0f) {
      adj_face_w(tr[q + 1].up, tr[q].mid, tr[q - 1].dn, tr[q + 1].s13, tr[q].s13, tr[q - 1].s13, bp, eu, em, ed, g,
                 m2g);
      adj_role<0>(tr[q + 1].up, tr[q + 1].s13, eu, g, m2g, Db[q + 2], Db[q + 1], Db[q]);
      adj_role<1>(tr[q].mid, tr[q].s13, em, g, m2g, Db[q + 1], Db[q], Db[q - 1]);
      adj_role<2>(tr[q - 1].dn, tr[q - 1].s13, ed, g, m2g, Db[q], Db[q - 1], Db[q - 2]);
    }
    const int k = i - 3;  // output whose two differences are complete
    if (k >= 0 && k < ARUN) dst[k * DS] += (Db[k - 1 + 6] - Db[k + 6]) * rd;
  }
}

// One hydro line of ARUN output points: faces f = -2 .. ARUN+2 relative to the first output point,
// points m = -5 .. ARUN+4. Writes (f+bar + f-bar) and (f+bar - f-bar) of the outputs. The faces advance
// left to right; a point's split fluxes are formed just before the first face that reads them (face m-1)
// and its output is written after the last face that adds to it (face m+3), so only a six-point window
// of values is live at a time.
template <typename real>
__device__ __forceinline__ void adj_hydro_line(const real* __restrict__ Uc, const real* __restrict__ Xc,
                                               const real* __restrict__ vel, const real* __restrict__ pr,
                                               const real* __restrict__ nuc, int S, int kind, real alpha, real rd,
                                               real* __restrict__ pb, real* __restrict__ mb, int DS) {
  constexpr int NP = ARUN + 10;  // points, index m + 5
  real fp[NP], fm[NP], ap[NP], am[NP];
  auto point = [&](int q) {
    const int m = q - 5;
    const real uu = Uc[m * S];
    real F;
    if (kind == 0) F = Xc[m * S];
    else {
      const real vn = vel[m * S], p = pr[m * S];
      F = kind == 1 ? uu * vn + p : kind == 2 ? uu * vn : (uu + p) * vn;
    }
    fp[q] = real(0.5) * (F + alpha * uu);
    fm[q] = real(0.5) * (F - alpha * uu);
    ap[q] = real(0);
    am[q] = real(0);
  };
#pragma unroll
  for (int q = 0; q < 5; ++q) point(q);  // points -5 .. -1
#pragma unroll
  for (int f = -2; f <= ARUN + 2; ++f) {
    // face f lies between points f-1 and f; its left-biased stencil is points f-3 .. f+1 and its
    // right-biased one f+2 .. f-2: point f+2 is new
    const int q = f + 5;
    if (q + 2 < NP) point(q + 2);
    const real fb = (nuc[f * S] - nuc[(f - 1) * S]) * rd;
    if (fb != real(0)) {
      weno5_grad_acc(fp[q - 3], fp[q - 2], fp[q - 1], fp[q], fp[q + 1], fb, ap[q - 3], ap[q - 2], ap[q - 1], ap[q],
                     ap[q + 1]);
      weno5_grad_acc(fm[q + 2], fm[q + 1], fm[q], fm[q - 1], fm[q - 2], fb, am[q + 2], am[q + 1], am[q], am[q - 1],
                     am[q - 2]);
    }
    const int k = f - 3;  // output point completed by this face
    if (k >= 0 && k < ARUN) {
      pb[k * DS] = ap[k + 5] + am[k + 5];
      mb[k * DS] = ap[k + 5] - am[k + 5];
    }
  }
}

// Level-set line: output points k = 0 .. ARUN-1 receive phibar_k = (Dbar_{k-1} - Dbar_k) / h, where
// D_n = (phi_{n+1} - phi_n) / h and Dbar collects hb^- dW/dD over phi^-_i = W(D_{i-3..i+1}) and hb^+
// over phi^+_i = W(D_{i+2..i-2}) for the cells i = -3 .. ARUN+2 of the line.
template <typename real>
__device__ __forceinline__ void adj_phi_line(const real* __restrict__ ph, const real* __restrict__ hm,
                                                   const real* __restrict__ hp, int S, real rd, real* __restrict__ dst,
                                                   int DS) {
  constexpr int ND = ARUN + 11;  // differences D_n, n = -6 .. ARUN+4, index n + 6
  real D[ND], Db[ND];
  // D_n formed just before the first cell that reads it, outputs written after the last cell that adds
  // to the differences they need (a six-value window is live at a time)
  auto diff = [&](int q) {
    const int n = q - 6;
    D[q] = (ph[(n + 1) * S] - ph[n * S]) * rd;
    Db[q] = real(0);
  };
#pragma unroll
  for (int q = 0; q < 5; ++q) diff(q);
#pragma unroll
  for (int i = -3; i <= ARUN + 2; ++i) {
    const int q = i + 6;
    if (q + 2 < ND) diff(q + 2);
    const real bm = hm[i * S], bp = hp[i * S];
    if (bm != real(0))
      weno5_grad_acc(D[q - 3], D[q - 2], D[q - 1], D[q], D[q + 1], bm, Db[q - 3], Db[q - 2], Db[q - 1], Db[q],
                     Db[q + 1]);
    if (bp != real(0))
      weno5_grad_acc(D[q + 2], D[q + 1], D[q], D[q - 1], D[q - 2], bp, Db[q + 2], Db[q + 1], Db[q], Db[q - 1],
                     Db[q - 2]);
    const int k = i - 3;  // output whose two differences are complete
    if (k >= 0 && k < ARUN) dst[k * DS] += (Db[k - 1 + 6] - Db[k + 6]) * rd;
  }
}

template <typename real, int NF, int TY>
__global__ void __launch_bounds__(adj_threads<real, NF, TY>(), (sizeof(real) == 4 && TY == 16) ? 2 : 1)
    adj_line_kernel(AdjParams<real> P, int tiles_x) {
  using TL = ATile<real, NF, TY>;
  constexpr int ATY = TL::ATY;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* sm = reinterpret_cast<real*>(smem_raw);
  real* sW = sm + TL::OFF_W;
  real* sP = sm + TL::OFF_P;
  real* sN = sm + TL::OFF_N;
  real* sH = sm + TL::OFF_H;
  real* sPB = sm + TL::OFF_PB;
  real* sMB = sm + TL::OFF_MB;
  real* sMU = sm + TL::OFF_MU;
  const int tid = threadIdx.x;
  constexpr int NT = adj_threads<real, NF, TY>();
  const long long fs = P.fstride;
  // output points are padded-grid points: columns 1 .. nx+6 (cells -3 .. nx+2), rows 0 .. ny+5
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int c0 = 1 + tx * ATX, r0 = ty * ATY;  // padded coordinates of the tile's first output point
  const int bc0 = c0 - AHX, br0 = r0 - AHX;    // padded coordinates of box point (0, 0)
  const real gamma = P.gamma;

  // ---- load the boxes (zero outside the allocation), primitive variables
  for (int idx = tid; idx < TL::BOX; idx += NT) {
    const int r = idx / ABW, c = idx - r * ABW;
    const int gr = br0 + r, gc = bc0 + c;
    const bool in = gr >= 0 && gr < P.rows && gc >= 0 && gc < P.pitch;
    const long long k = static_cast<long long>(gr) * P.pitch + gc;
    real wv[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      wv[f] = in ? P.W[f * fs + k] : real(0);
      sW[f * TL::BOX + idx] = wv[f];
      sN[f * TL::BOX + idx] = in ? P.nu[f * fs + k] : real(0);
    }
    if constexpr (NF == 5) {
#pragma unroll
      for (int q = 0; q < 4; ++q) sH[q * TL::BOX + idx] = in ? P.hb[q * fs + k] : real(0);
    }
    real u, v;
    if constexpr (sizeof(real) == 4) {
      const real rr = RT<float>::rcp(wv[0]);
      u = wv[1] * rr;
      v = wv[2] * rr;
    } else {
      u = wv[1] / wv[0];
      v = wv[2] / wv[0];
    }
    sP[0 * TL::BOX + idx] = u;
    sP[1 * TL::BOX + idx] = v;
    sP[2 * TL::BOX + idx] = (gamma - real(1)) * (wv[3] - real(0.5) * (wv[1] * u + wv[2] * v));
  }
  for (int idx = tid; idx < NF * ATY * AOS; idx += NT) sMU[idx] = real(0);
  __syncthreads();

#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const bool xp = pass == 0;
    const real alpha = xp ? P.ax : P.ay;
    const real rd = xp ? P.rdx_r : P.rdy_r;
    const int S = xp ? 1 : ABW;
    const int DS = xp ? 1 : AOS;
    // items: (field, line, run); x: ATY rows x 4 runs; y: ATX columns x 2 runs
    const int per_c = xp ? ATY * (ATX / ARUN) : ATX * (ATY / ARUN);
    for (int it = tid; it < NF * per_c; it += NT) {
      const int c = it / per_c, rem = it - c * per_c;
      int orow, ocol;  // first output point of the run, tile coordinates
      if (xp) {
        orow = rem % ATY;
        // a warp holds 32 rows of one run (ATY 32) or 16 rows of two runs 16 columns apart (ATY 16)
        ocol = (((rem / ATY) & 1) * 2 + (rem / (2 * ATY))) * ARUN;
      } else {
        ocol = rem % ATX;
        orow = (rem / ATX) * ARUN;
      }
      const int bidx = (orow + AHX) * ABW + (ocol + AHX);
      if (c < 4) {
        const int kind = (c == 0) ? 0 : (c == 3) ? 3 : ((c == 1) == xp) ? 1 : 2;
        if constexpr (sizeof(real) == 4)
          adj_hydro_line_f32(sW + c * TL::BOX + bidx, sW + (xp ? 1 : 2) * TL::BOX + bidx,
                             sP + (xp ? 0 : 1) * TL::BOX + bidx, sP + 2 * TL::BOX + bidx, sN + c * TL::BOX + bidx, S,
                             kind, alpha, rd, sPB + (c * ATY + orow) * AOS + ocol, sMB + (c * ATY + orow) * AOS + ocol,
                             DS);
        else
          adj_hydro_line<real>(sW + c * TL::BOX + bidx, sW + (xp ? 1 : 2) * TL::BOX + bidx,
                               sP + (xp ? 0 : 1) * TL::BOX + bidx, sP + 2 * TL::BOX + bidx, sN + c * TL::BOX + bidx,
                               S, kind, alpha, rd, sPB + (c * ATY + orow) * AOS + ocol,
                               sMB + (c * ATY + orow) * AOS + ocol, DS);
      } else if constexpr (NF == 5) {
        if constexpr (sizeof(real) == 4)
          adj_phi_line_f32(sW + 4 * TL::BOX + bidx, sH + (xp ? 0 : 2) * TL::BOX + bidx,
                           sH + (xp ? 1 : 3) * TL::BOX + bidx, S, rd, sMU + (4 * ATY + orow) * AOS + ocol, DS);
        else
          adj_phi_line<real>(sW + 4 * TL::BOX + bidx, sH + (xp ? 0 : 2) * TL::BOX + bidx,
                             sH + (xp ? 1 : 3) * TL::BOX + bidx, S, rd, sMU + (4 * ATY + orow) * AOS + ocol, DS);
      }
    }
    __syncthreads();
    // split and flux-Jacobian adjoint at every output point of the tile
    for (int idx = tid; idx < ATY * ATX; idx += NT) {
      const int orow = idx / ATX, ocol = idx - orow * ATX;
      const int b = (orow + AHX) * ABW + (ocol + AHX);
      const real rho = sW[b], mx = sW[TL::BOX + b], my = sW[2 * TL::BOX + b], E = sW[3 * TL::BOX + b];
      real pb[4], mb[4];
      bool any = false;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        pb[r] = sPB[(r * ATY + orow) * AOS + ocol];
        mb[r] = sMB[(r * ATY + orow) * AOS + ocol];
        any = any || pb[r] != real(0) || mb[r] != real(0);
      }
      if (!any) continue;  // also skips unfilled corner points
      real J[4][4];
      flux_jacobian<real>(xp ? 0 : 1, gamma, rho, mx, my, E, J);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        real acc = real(0.5) * alpha * mb[s];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc += real(0.5) * J[r][s] * pb[r];
        sMU[(s * ATY + orow) * AOS + ocol] += acc;
      }
    }
    __syncthreads();
  }
  // ---- write mu: interior points add to the point terms already there; frame points are set
  for (int idx = tid; idx < ATY * ATX; idx += NT) {
    const int orow = idx / ATX, ocol = idx - orow * ATX;
    const int gr = r0 + orow, gc = c0 + ocol;
    const int i = gc - GX, j = gr - GY;
    if (gr >= P.ny + 2 * GY || gc >= P.nx + GX + 3) continue;
    const bool ix = i >= 0 && i < P.nx, iy = j >= 0 && j < P.ny;
    if (!ix && !iy) continue;  // corner: not part of the scheme
    const long long k = static_cast<long long>(gr) * P.pitch + gc;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const real v = sMU[(f * ATY + orow) * AOS + ocol];
      P.mu[f * fs + k] = (ix && iy) ? P.mu[f * fs + k] + v : v;
    }
  }
}

// ---------------------------------------------------------------------------- fold and blend

template <typename real, int NF>
__global__ void __launch_bounds__(256) adj_blend_kernel(AdjParams<real> P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= P.nx) return;
  const long long fs = P.fstride;
  const int nx = P.nx, ny = P.ny;
  const long long k = static_cast<long long>(j + GY) * P.pitch + i + GX;
  real m[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) m[f] = P.mu[f * fs + k];
  // adjoint of the ghost fill: every ghost point that is an image of (i, j) hands its adjoint back
  auto take = [&](int gi, int gj, bool fx, bool fy) {
    const long long g = static_cast<long long>(gj + GY) * P.pitch + gi + GX;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      real v = P.mu[f * fs + g];
      if ((f == 1 && fx) || (f == 2 && fy)) v = -v;
      m[f] += v;
    }
  };
  if (i < 3 || i >= nx - 3) {
    const int bl = P.bc[0], bh = P.bc[1];
    if (bl == BC_PERIODIC) {
      if (i >= nx - 3) take(i - nx, j, false, false);
    } else if (bl == BC_TRANSMISSIVE) {
      if (i == 0) { take(-1, j, false, false); take(-2, j, false, false); take(-3, j, false, false); }
    } else if (i < 3) {
      take(-1 - i, j, true, false);
    }
    if (bh == BC_PERIODIC) {
      if (i < 3) take(nx + i, j, false, false);
    } else if (bh == BC_TRANSMISSIVE) {
      if (i == nx - 1) { take(nx, j, false, false); take(nx + 1, j, false, false); take(nx + 2, j, false, false); }
    } else if (i >= nx - 3) {
      take(2 * nx - 1 - i, j, true, false);
    }
  }
  if (j < 3 || j >= ny - 3) {
    const int bl = P.bc[2], bh = P.bc[3];
    if (bl == BC_PERIODIC) {
      if (j >= ny - 3) take(i, j - ny, false, false);
    } else if (bl == BC_TRANSMISSIVE) {
      if (j == 0) { take(i, -1, false, false); take(i, -2, false, false); take(i, -3, false, false); }
    } else if (j < 3) {
      take(i, -1 - j, false, true);
    }
    if (bh == BC_PERIODIC) {
      if (j < 3) take(i, ny + j, false, false);
    } else if (bh == BC_TRANSMISSIVE) {
      if (j == ny - 1) { take(i, ny, false, false); take(i, ny + 1, false, false); take(i, ny + 2, false, false); }
    } else if (j >= ny - 3) {
      take(i, 2 * ny - 1 - j, false, true);
    }
  }
  const real dt = P.dt_r, a = P.a_r, b = P.b_r;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const real nu = P.nu[f * fs + k];
    const real o = b * (nu + dt * m[f]);
    P.out[f * fs + k] = o;
    if (P.acc_mode == 0) P.acc[f * fs + k] = a * nu;
    else if (P.acc_mode == 1) P.acc[f * fs + k] += a * nu;
    else P.acc[f * fs + k] += o;
  }
}

}  // namespace hydro
