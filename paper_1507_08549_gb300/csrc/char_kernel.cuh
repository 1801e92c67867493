// char_kernel.cuh -- characteristic-wise WENO5 flux divergence (Leung, Chu & Lin 2015, Sec. 2.1: the
// "WENO-Roe" construction of Jiang & Shu 1996).
//
// At every face the Lax-Friedrichs split fluxes f+- = (F +- alpha U) / 2 of the six stencil cells are
// projected on the left eigenvectors of the flux Jacobian at the Roe average of the face's two cells,
// each characteristic field is reconstructed with WENO5 (f+ left-biased, f- right-biased), and the sum
// is projected back with the right eigenvectors. The eigen-system is written in the rotated frame
// (rho, m_n, m_t, tau) so that x and y faces run the same instructions:
//   R = [1, 1, 0, 1; u_n - c, u_n, 0, u_n + c; u_t, u_t, 1, u_t; H - u_n c, q^2/2, u_t, H + u_n c]
//   L = R^-1 = [(b2 + u_n/c)/2, -(b1 u_n + 1/c)/2, -b1 u_t/2, b1/2;  1 - b2, b1 u_n, b1 u_t, -b1;
//               -u_t, 0, 1, 0;  (b2 - u_n/c)/2, -(b1 u_n - 1/c)/2, -b1 u_t/2, b1/2],
//   b1 = (gamma - 1)/c^2, b2 = b1 q^2/2, from s = sqrt(rho): v~ = (s_l v_l + s_r v_r)/(s_l + s_r) for u_n,
//   u_t and H = (tau + p)/rho, c^2 = (gamma - 1)(H - q^2/2).
//
// char_div_kernel writes D = dF/dx + dG/dy of the four hydro components for one stage input into a
// padded buffer laid out like the states; the stage kernel then takes D from there instead of its own
// component-wise passes (the level set, sources, RK blend and reductions are unchanged). Persistent CTAs
// of 256 threads walk 32 x 16 (FP32) or 32 x 8 (FP64) tiles; each tile's box with its 3-cell halo arrives
// by one TMA tensor copy into one of two staging buffers (the next tile's copy is in flight while the
// current one is computed); one thread per face computes the face flux (x faces, then y faces), then one
// thread per cell differences them.
//
// FP64: every operation the plain definition writes, in its order, rounded once (products by the 0 and 1
// entries of R and L included), so D is reproducible bit for bit by a sequential implementation.
// FP32: fused operations, the shared-smoothness WENO of the stage kernel, and the projections written with
// the zero, unit and repeated entries of L and R folded out.
#pragma once
#include "stage_kernel.cuh"

namespace hydro {

constexpr int CX = 32, CBW = CX + 6;          // tile columns, halo box columns
constexpr int CHAR_THREADS = 256;
// tile rows: 16 in FP32 (the 3-row halo then costs 1.38 loaded rows per tile row instead of 1.75), 8 in
// FP64 (the shared-memory tile stays under the 48 KB static limit)
template <typename real>
struct CharTile {
  static constexpr int CY = sizeof(real) == 4 ? 16 : 8;
  static constexpr int CBH = CY + 6;
};

// The staging box of a tile: CHAR_BOX_W = 40 padded columns from 32 bx (cells 32 bx - 4 .. 32 bx + 35; a TMA
// box starts on a 16-byte boundary), CBH rows from CY by, the 4 hydro fields.
constexpr int CHAR_BOX_W = 40;

template <typename real>
struct CharSmem {
  static constexpr int CY = CharTile<real>::CY, CBH = CharTile<real>::CBH;
  real U[4][CBH][CBW];
  real u[CBH][CBW], v[CBH][CBW], p[CBH][CBW];
  real FX[4][CY][CX + 1];   // x-face fluxes, face f left of tile column f
  real FY[4][CY + 1][CX];   // y-face fluxes, face f below tile row f
};

// dynamic shared memory: CharSmem | staging box 0 | staging box 1 | 2 mbarriers (128-byte aligned parts)
template <typename real>
struct CharLayout {
  static constexpr int CBH = CharTile<real>::CBH;
  static constexpr unsigned BOX_BYTES = 4u * CBH * CHAR_BOX_W * sizeof(real);
  static constexpr size_t STAGE_OFF = ((sizeof(CharSmem<real>) + 127) / 128) * 128;
  static constexpr size_t STAGE_STRIDE = ((BOX_BYTES + 127) / 128) * 128;
  static constexpr size_t BAR_OFF = STAGE_OFF + 2 * STAGE_STRIDE;
  static constexpr size_t BYTES = BAR_OFF + 16;
};

// operation policy: FP64 rounds each written operation once; FP32 lets the compiler fuse
template <typename real>
struct CO;

template <>
struct CO<double> {
  static __device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sq(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double rc(double a) { return __ddiv_rn(1.0, a); }
  static __device__ __forceinline__ double weno(double a, double b, double c, double d, double e) {
    return Ar<double>::weno5(a, b, c, d, e);
  }
};

template <>
struct CO<float> {
  static __device__ __forceinline__ float ad(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sb(float a, float b) { return a - b; }
  static __device__ __forceinline__ float ml(float a, float b) { return a * b; }
  static __device__ __forceinline__ float dv(float a, float b) { return a * RT<float>::rcp(b); }
  static __device__ __forceinline__ float sq(float a) { return RT<float>::sqrt_(a); }
  static __device__ __forceinline__ float rc(float a) { return RT<float>::rcp(a); }
  static __device__ __forceinline__ float weno(float a, float b, float c, float d, float e) {
    return weno_side(a, b, c, d, e, betas(a, b, c).m, betas(b, c, d).t, betas(c, d, e).p);
  }
};

// Face flux between box cells (r, c) and its right (dir 0) or upper (dir 1) neighbour. out[] in the frame
// (rho, m_x, m_y, tau). Returns false when the averaged sound speed is not real.
template <typename real>
__device__ __forceinline__ bool char_face(const CharSmem<real>& S, int dir, int r, int c, real alpha, real gm1,
                                          real out[4]) {
  using O = CO<real>;
  const int n = dir == 0 ? 1 : 2, t = dir == 0 ? 2 : 1;
  const int dr = dir == 0 ? 0 : 1, dc = dir == 0 ? 1 : 0;
  // Roe average of the cells l = (r, c) and l + 1
  real s[2], vn[2], vt[2], H[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int rr = r + k * dr, cc = c + k * dc;
    const real rho = S.U[0][rr][cc];
    s[k] = O::sq(rho);
    vn[k] = dir == 0 ? S.u[rr][cc] : S.v[rr][cc];
    vt[k] = dir == 0 ? S.v[rr][cc] : S.u[rr][cc];
    H[k] = O::dv(O::ad(S.U[3][rr][cc], S.p[rr][cc]), rho);
  }
  const real den = O::ad(s[0], s[1]);
  const real un = O::dv(O::ad(O::ml(s[0], vn[0]), O::ml(s[1], vn[1])), den);
  const real ut = O::dv(O::ad(O::ml(s[0], vt[0]), O::ml(s[1], vt[1])), den);
  const real h = O::dv(O::ad(O::ml(s[0], H[0]), O::ml(s[1], H[1])), den);
  const real q2 = O::ad(O::ml(un, un), O::ml(ut, ut));
  const real c2 = O::ml(gm1, O::sb(h, O::ml(real(0.5), q2)));
  if (!(c2 > real(0)) || !isfinite(c2)) return false;
  const real cs = O::sq(c2), rcs = O::rc(cs);
  const real b1 = O::dv(gm1, c2), b2 = O::ml(real(0.5), O::ml(b1, q2));
  const real Lm[4][4] = {
      {O::ml(real(0.5), O::ad(b2, O::ml(un, rcs))), O::ml(real(-0.5), O::ad(O::ml(b1, un), rcs)),
       O::ml(real(-0.5), O::ml(b1, ut)), O::ml(real(0.5), b1)},
      {O::sb(real(1), b2), O::ml(b1, un), O::ml(b1, ut), -b1},
      {-ut, real(0), real(1), real(0)},
      {O::ml(real(0.5), O::sb(b2, O::ml(un, rcs))), O::ml(real(-0.5), O::sb(O::ml(b1, un), rcs)),
       O::ml(real(-0.5), O::ml(b1, ut)), O::ml(real(0.5), b1)}};
  // projected split fluxes of the six stencil cells l-2 .. l+3. FP32 uses the structure of L:
  // with K = f3 - u_n f1 - u_t f2, P = (b2 f0 + b1 K)/2 and Q = (u_n f0 - f1)/(2c),
  //   w0 = P + Q, w1 = f0 - 2P, w2 = f2 - u_t f0, w3 = P - Q;
  // FP64 keeps the plain matrix-vector products (bitwise against the oracle).
  real wp[4][6], wm[4][6];
  const real hb1 = real(0.5) * b1, hb2 = real(0.5) * b2, hrc = real(0.5) * rcs;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int rr = r + (k - 2) * dr, cc = c + (k - 2) * dc;
    const real Ur[4] = {S.U[0][rr][cc], S.U[n][rr][cc], S.U[t][rr][cc], S.U[3][rr][cc]};
    const real vnk = dir == 0 ? S.u[rr][cc] : S.v[rr][cc];
    const real pk = S.p[rr][cc];
    // rotated flux (m_n, m_n v_n + p, m_t v_n, (tau + p) v_n), as the frame flux's components
    const real Fr[4] = {Ur[1], O::ad(O::ml(Ur[1], vnk), pk), O::ml(Ur[2], vnk), O::ml(O::ad(Ur[3], pk), vnk)};
    real fp[4], fm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Ar<real>::split(Fr[q], Ur[q], alpha, fp[q], fm[q]);
    if constexpr (sizeof(real) == 4) {
      auto project = [&](const real (&f)[4], real (&w)[4][6]) {
        const real K = f[3] - un * f[1] - ut * f[2];
        const real P = hb2 * f[0] + hb1 * K;
        const real Q = hrc * (un * f[0] - f[1]);
        w[0][k] = P + Q;
        w[1][k] = f[0] - real(2) * P;
        w[2][k] = f[2] - ut * f[0];
        w[3][k] = P - Q;
      };
      project(fp, wp);
      project(fm, wm);
    } else {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        wp[w][k] = O::ad(O::ad(O::ad(O::ml(Lm[w][0], fp[0]), O::ml(Lm[w][1], fp[1])), O::ml(Lm[w][2], fp[2])),
                         O::ml(Lm[w][3], fp[3]));
        wm[w][k] = O::ad(O::ad(O::ad(O::ml(Lm[w][0], fm[0]), O::ml(Lm[w][1], fm[1])), O::ml(Lm[w][2], fm[2])),
                         O::ml(Lm[w][3], fm[3]));
      }
    }
  }
  real wh[4];
#pragma unroll
  for (int w = 0; w < 4; ++w)
    wh[w] = O::ad(O::weno(wp[w][0], wp[w][1], wp[w][2], wp[w][3], wp[w][4]),
                  O::weno(wm[w][5], wm[w][4], wm[w][3], wm[w][2], wm[w][1]));
  real fr[4];
  if constexpr (sizeof(real) == 4) {  // R w^ with R's structure: S = w0 + w3, D = w3 - w0
    const real Sm = wh[0] + wh[3], Dd = wh[3] - wh[0];
    fr[0] = Sm + wh[1];
    fr[1] = un * fr[0] + cs * Dd;
    fr[2] = ut * fr[0] + wh[2];
    fr[3] = h * Sm + un * cs * Dd + real(0.5) * q2 * wh[1] + ut * wh[2];
  } else {
    const real Rm[4][4] = {{real(1), real(1), real(0), real(1)},
                           {O::sb(un, cs), un, real(0), O::ad(un, cs)},
                           {ut, ut, real(1), ut},
                           {O::sb(h, O::ml(un, cs)), O::ml(real(0.5), q2), ut, O::ad(h, O::ml(un, cs))}};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      fr[q] = O::ad(O::ad(O::ad(O::ml(Rm[q][0], wh[0]), O::ml(Rm[q][1], wh[1])), O::ml(Rm[q][2], wh[2])),
                    O::ml(Rm[q][3], wh[3]));
  }
  out[0] = fr[0];
  out[n] = fr[1];
  out[t] = fr[2];
  out[3] = fr[3];
  return true;
}

// D = dF/dx + dG/dy of the hydro components of the stage input p->win into p->ext_div (padded layout), over
// tiles w = blockIdx.x, blockIdx.x + gridDim.x, ... of the tiles_x-wide tile grid.
template <typename real>
__device__ __forceinline__ void char_issue_box(const GridParams<real>& g, int w, int tiles_x, real* dst, uint64_t* bar) {
  constexpr int CY = CharTile<real>::CY;
  mbar_arrive_expect_tx(bar, CharLayout<real>::BOX_BYTES);
  tma_load_3d(dst, g.tmap_char, (w % tiles_x) * CX, (w / tiles_x) * CY, 0, bar);
}

template <typename real>
__global__ void __launch_bounds__(CHAR_THREADS) char_div_kernel(const GridParams<real>* __restrict__ pp, int tiles_x,
                                                               int ntiles) {
  using L = CharLayout<real>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  CharSmem<real>& S = *reinterpret_cast<CharSmem<real>*>(smem_raw);
  real* stage = reinterpret_cast<real*>(smem_raw + L::STAGE_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + L::BAR_OFF);
  __shared__ int s_abort;
  const GridParams<real>& g = *pp;
  const int nx = g.nx, ny = g.ny, pitch = g.pitch;
  const long long fs = g.fstride;
  constexpr int CY = CharTile<real>::CY, CBH = CharTile<real>::CBH;
  constexpr int SSTR = static_cast<int>(L::STAGE_STRIDE / sizeof(real));
  const int tid = threadIdx.x;
  const real gm1 = g.gm1;
  // the tensor copies write 128-byte aligned buffers (the same address for every thread)
  if ((smem_u32(smem_raw) & 127u) != 0u) {
    if (tid == 0 && static_cast<int>(blockIdx.x) < ntiles) atomicOr(g.err, ERR_LAYOUT);
    return;
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_abort = 0;
  }
  __syncthreads();
  if (tid == 0 && static_cast<int>(blockIdx.x) < ntiles) char_issue_box(g, blockIdx.x, tiles_x, stage, &bar[0]);
  const real ax = g.alpha_in[0], ay = g.alpha_in[1];
  unsigned parity[2] = {0u, 0u};
  int it = 0;
  for (int w = blockIdx.x; w < ntiles; w += gridDim.x, ++it) {
    const int b = it & 1;
    const real* box = stage + b * SSTR;
    // the next tile's box into the other buffer, whose reads (the previous tile's primitives) ended at a
    // barrier: the issuing thread's proxy fence orders them before the copy
    const int wn = w + gridDim.x;
    if (tid == 0 && wn < ntiles) {
      fence_proxy_async_smem();
      char_issue_box(g, wn, tiles_x, stage + (b ^ 1) * SSTR, &bar[b ^ 1]);
    }
    const int x0 = (w % tiles_x) * CX, y0 = (w / tiles_x) * CY;
    if (!mbar_wait_bounded(&bar[b], parity[b])) {
      atomicOr(g.err, ERR_TIMEOUT);
      s_abort = 1;
    }
    parity[b] ^= 1u;
    // box cell (r, c) is grid cell (x0 - 3 + c, y0 - 3 + r): staging column c + 1 (outside the allocation
    // the copy reads zeros, and such points get no primitives)
    for (int idx = tid; idx < CBH * CBW; idx += CHAR_THREADS) {
      const int r = idx / CBW, c = idx - r * CBW;
      real U[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        U[f] = box[(f * CBH + r) * CHAR_BOX_W + c + 1];
        S.U[f][r][c] = U[f];
      }
      real u = real(0), v = real(0), p = real(0);
      if (U[0] != real(0)) Ar<real>::prims(U[0], U[1], U[2], U[3], gm1, u, v, p);
      S.u[r][c] = u;
      S.v[r][c] = v;
      S.p[r][c] = p;
    }
    __syncthreads();
    if (s_abort) {
      // a copy did not complete: wait (with a limit) for the copies in flight -- this box and the next --
      // before the CTA leaves
      if (tid == 0) {
        mbar_wait_limit(&bar[b], parity[b] ^ 1u, TILE_WAIT_POLLS, TILE_WAIT_NS);
        if (wn < ntiles) mbar_wait_limit(&bar[b ^ 1], parity[b ^ 1], TILE_WAIT_POLLS, TILE_WAIT_NS);
      }
      break;
    }
    bool bad = false;
    // x faces: tile row fr, face fc (left of tile column fc); needed for rows < ny and faces <= nx - x0
    for (int it2 = tid; it2 < CY * (CX + 1); it2 += CHAR_THREADS) {
      const int fr = it2 / (CX + 1), fc = it2 - fr * (CX + 1);
      real o[4] = {real(0), real(0), real(0), real(0)};
      if (y0 + fr < ny && x0 + fc <= nx) bad |= !char_face(S, 0, fr + 3, fc + 2, ax, gm1, o);
#pragma unroll
      for (int f = 0; f < 4; ++f) S.FX[f][fr][fc] = o[f];
    }
    // y faces: face fr below tile row fr, tile column fc
    for (int it2 = tid; it2 < (CY + 1) * CX; it2 += CHAR_THREADS) {
      const int fr = it2 / CX, fc = it2 - fr * CX;
      real o[4] = {real(0), real(0), real(0), real(0)};
      if (x0 + fc < nx && y0 + fr <= ny) bad |= !char_face(S, 1, fr + 2, fc + 3, ay, gm1, o);
#pragma unroll
      for (int f = 0; f < 4; ++f) S.FY[f][fr][fc] = o[f];
    }
    if (bad) atomicOr(g.err, ERR_NONPHYSICAL);
    __syncthreads();
    // the differences read only FX and FY, which the next tile writes after its primitives' barrier
    for (int cell = tid; cell < CY * CX; cell += CHAR_THREADS) {
      const int tr = cell / CX, tc = cell - tr * CX;
      const int i = x0 + tc, j = y0 + tr;
      if (i < nx && j < ny) {
        const long long e = static_cast<long long>(j + GY) * pitch + i + GX;
        real* D = const_cast<real*>(g.ext_div);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const real dxf = Ar<real>::divided(S.FX[f][tr][tc + 1], S.FX[f][tr][tc], g.rdx, g.dx);
          const real dyf = Ar<real>::divided(S.FY[f][tr + 1][tc], S.FY[f][tr][tc], g.rdy, g.dy);
          D[f * fs + e] = Ar<real>::sum(dxf, dyf);
        }
      }
    }
  }
}

}  // namespace hydro
