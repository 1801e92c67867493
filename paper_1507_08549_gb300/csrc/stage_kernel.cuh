// stage_kernel.cuh -- fused SSP-RK3 stage of the WENO5 / global Lax-Friedrichs Euler update with the
// level-set scalar (Leung, Chu & Lin 2015, Sec. 2.1 Eq. euler2D and Sec. 2.2), for sm_103a.
//
// One CTA processes one 60 x TY tile per work item (persistent loop over items):
//   A. the (TY+6) x 68 halo box of every field is moved into shared memory by one TMA tensor copy
//      (cp.async.bulk.tensor.3d over (x, y, field) of the padded state, issued by one thread one tile
//      ahead, completion on an mbarrier);
//   B. primitive variables u, v, p at the box points (rcp of rho once per point);
//   C. x pass: each work item is (field, tile row, run of 15 cells); the split fluxes
//      f+- = (F +- alpha U)/2, the data of every point triplet and the 16 face fluxes of the run slide
//      through registers, so every point's split flux and every triplet's candidate values, smoothness
//      indicators and weights are formed once (FP32; FP64 keeps the textbook per-face order); the
//      level-set item forms the one-sided HJ-WENO5 derivatives the same way;
//   D. y pass: same on (field, tile column, run of 15 cells), adding dG/dy to dF/dx in shared memory;
//      the y pass of a hydro field waits only for that field's x-pass warps (named barrier);
//   E. per 3-cell group: L = -(dF/dx + dG/dy) + S and the level set's local Lax-Friedrichs
//      Hamiltonian, the RK blend a U^n + b (W + dt L), the stores, the ghost images the boundary
//      conditions ask for, and the reductions the next launches need: alpha_x, alpha_y of the output
//      (next stage), c + |u| + |v| (next step's dt), the conserved totals.
// Lane-to-item maps make every shared-memory access of the passes bank-conflict free (68 = 4 mod 32
// and 15 = 3 mod 4 spread the 32 lanes of an x-pass warp over all banks).
#pragma once
#include "hydro_internal.cuh"

namespace hydro {

// ------------------------------------------------------------------------------ precision traits

template <typename real>
struct RT;

template <>
struct RT<float> {
  static __device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ void atomic_max(float* a, float v) {
    atomicMax(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
  }
  static __device__ __forceinline__ bool finite(float v) { return isfinite(v); }
};

template <>
struct RT<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ void atomic_max(double* a, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(a), static_cast<unsigned long long>(__double_as_longlong(v)));
  }
  static __device__ __forceinline__ bool finite(double v) { return isfinite(v); }
};

// ------------------------------------------------------------------------------ TMA + mbarrier

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// One box of a 3-D tensor map (x innermost, then y, then field) into shared memory (TMA, tiled mode),
// completion on an mbarrier. The map lives in global memory (written from the host before the launch);
// dst is 128-byte aligned and x * sizeof(element) is a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Tensor store of one box of a 3-D tensor map from shared memory (src 128-byte aligned), tracked by the
// issuing thread's bulk async-group: commit after issuing, then wait until the source has been read
// (before the buffer is written again) or until the writes are done (before the CTA exits).
__device__ __forceinline__ void tma_store_3d(const void* tmap, const void* src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tmap),
               "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// L2 prefetch of one box of a 3-D tensor map (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_l2_3d(const void* tmap, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(tmap), "r"(x), "r"(y),
               "r"(z)
               : "memory");
}

// Barrier over `count` threads (whole warps) at named barrier ID (1..15; 0 is __syncthreads').
template <int ID>
__device__ __forceinline__ void named_barrier_sync(int count) {
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: false after `limit` polls or `max_ns` nanoseconds, whichever comes
// first (a poll of try_wait may suspend the thread for a while, so a poll count alone does not bound the
// time); the caller reports ERR_TIMEOUT.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, unsigned parity, unsigned limit,
                                                unsigned long long max_ns = ~0ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0u && global_ns() - t0 > max_ns) return false;
  }
  return false;
}

// The stage kernel's wait for a tile's copies: at most 2^28 polls and 2 seconds before giving up.
constexpr unsigned TILE_WAIT_POLLS = 1u << 28;
constexpr unsigned long long TILE_WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  return mbar_wait_limit(bar, parity, TILE_WAIT_POLLS, TILE_WAIT_NS);
}


// ------------------------------------------------------------------------------ WENO5 pieces

// Smoothness data of the point triplet (L, C, R) (Jiang & Shu 1996), already offset by eps:
//   m: eps + 13/12 s^2 + 1/4 (2s - t)^2  (the triplet as the leftmost stencil of a face),
//   t: eps + 13/12 s^2 + 1/4 t^2          (as the central stencil),
//   p: eps + 13/12 s^2 + 1/4 (2s + t)^2  (as the rightmost stencil),
// with s = (L + R) - 2C and t = L - R, evaluated as (s -+ t/2)^2 and (t/2)^2 (t/2 is exact). Mirroring
// the triplet keeps s and negates t, so the same data serve the reconstruction from the right.
template <typename real>
struct B3 {
  real m, t, p;
};

template <typename real>
__device__ __forceinline__ B3<real> betas(real L, real C, real R) {
  using T = RT<real>;
  const real s = T::fma_(real(-2), C, L + R);
  const real th = real(0.5) * (L - R);
  const real bs = T::fma_(real(13.0 / 12.0) * s, s, real(1e-6));
  const real mm = s - th;
  const real pp = s + th;
  B3<real> b;
  b.m = T::fma_(mm, mm, bs);
  b.t = T::fma_(th, th, bs);
  b.p = T::fma_(pp, pp, bs);
  return b;
}

// WENO5-JS value at the right face of c from (a, b, c, d, e) given D_k = eps + beta_k:
//   sum_k d_k q_k / (eps + beta_k)^2 / sum_k d_k / (eps + beta_k)^2,
// with the linear weights d = (1/10, 6/10, 3/10) and the 1/6 of the candidate values folded into the
// constants, so one reciprocal per weight and one for the normalisation remain.
template <typename real>
__device__ __forceinline__ real weno_side(real a, real b, real c, real d, real e, real D0, real D1, real D2) {
  using T = RT<real>;
  const real q0 = T::fma_(real(0.2), a, T::fma_(real(-0.7), b, real(1.1) * c));
  const real q1 = T::fma_(real(-0.6), b, T::fma_(real(3.0), c, real(1.2) * d));
  const real q2 = T::fma_(real(0.6), c, T::fma_(real(1.5), d, real(-0.3) * e));
  const real r0 = T::rcp(D0 * D0);
  const real r1 = T::rcp(D1 * D1);
  const real r2 = T::rcp(D2 * D2);
  const real num = T::fma_(r2, q2, T::fma_(r1, q1, r0 * q0));
  const real den = T::fma_(real(1.8), r2, T::fma_(real(3.6), r1, real(0.6) * r0));
  return num * T::rcp(den);
}

// FP32 line form: everything a face needs from one point triplet (L, C, R), formed once per triplet.
// With s = (L + R) - 2C and t = L - R (array order), the three candidate values a triplet serves are
//   C + 13/12 s -+ 3/4 t (as the upwind-most stencil: - from the left, + from the right),
//   C + s/12 - t/4 and C + s/12 + t/4 (the central and the downwind-most stencils),
// and its three smoothness indicators eps + beta are 13/12 s^2 + {(s - t/2)^2, (t/2)^2, (s + t/2)^2}
// (the Jiang-Shu beta_0, beta_1, beta_2 in these variables). All three indicators of a face are scaled by
// 12/13 (the weights only see their ratios), which removes the 13/12 multiply: D = s^2 + (12/13)(...)^2
// + (12/13) eps, with u = sqrt(12/13) t/2. Each role carries its reciprocal weight already multiplied by
// the linear weight (1, 6, 3 for the upwind-most, central and downwind-most stencil).
struct Role32 {
  float q, w;  // candidate value, d_k / D_k^2 (up to a factor common to the face)
};
struct Tri32 {
  Role32 up, mid, down;  // the triplet as the upwind-most, central, downwind-most stencil of a face
};

constexpr float TRI_KS = 0.96076892283052284f;  // sqrt(12/13)
constexpr float TRI_KU = 0.48038446141526142f;  // sqrt(12/13) / 2
constexpr float TRI_KQ = 0.52041649986653958f;  // sqrt(13/12) / 2: t/4 = KQ u
constexpr float TRI_EPS_SCALE = 12.0f / 13.0f;

// Smoothness data of a triplet, shared by both reconstruction directions.
struct TriD32 {
  float s, u, base, rm, rt6, rp;  // rm = 1/Dm^2, rt6 = 6/Dt^2, rp = 1/Dp^2
};
__device__ __forceinline__ TriD32 tri_data(float L, float C, float R, float eps_scaled) {
  using T = RT<float>;
  TriD32 d;
  d.s = T::fma_(-2.0f, C, L + R);
  d.u = T::mul_(TRI_KU, L - R);
  const float bs = T::fma_(d.s, d.s, eps_scaled);
  const float mm = T::fma_(TRI_KS, d.s, -d.u), pp = T::fma_(TRI_KS, d.s, d.u);
  const float Dm = T::fma_(mm, mm, bs), Dt = T::fma_(d.u, d.u, bs), Dp = T::fma_(pp, pp, bs);
  d.rm = T::rcp(T::mul_(Dm, Dm));
  d.rt6 = T::mul_(6.0f, T::rcp(T::mul_(Dt, Dt)));
  d.rp = T::rcp(T::mul_(Dp, Dp));
  d.base = T::fma_(1.0f / 12.0f, d.s, C);
  return d;
}
// The triplet's roles for the reconstruction from the left (left_to_right) or from the right. Mirroring
// the triplet keeps s, negates u and swaps Dm and Dp, so the two directions are mirror images bit for bit.
__device__ __forceinline__ Tri32 tri_roles(const TriD32& d, bool left_to_right) {
  using T = RT<float>;
  const float lo = T::fma_(-TRI_KQ, d.u, d.base), hi = T::fma_(TRI_KQ, d.u, d.base);
  const float bss = T::add_(d.base, d.s);
  Tri32 r;
  r.mid = {left_to_right ? lo : hi, d.rt6};
  if (left_to_right) {
    r.up = {T::fma_(-3.0f * TRI_KQ, d.u, bss), d.rm};
    r.down = {hi, T::mul_(3.0f, d.rp)};
  } else {
    r.up = {T::fma_(3.0f * TRI_KQ, d.u, bss), d.rp};
    r.down = {lo, T::mul_(3.0f, d.rm)};
  }
  return r;
}
// One face value from the upwind-most, central and downwind-most roles (the same expression for both
// directions, so mirrored data give mirrored values).
__device__ __forceinline__ float tri_face(const Role32& a, const Role32& b, const Role32& c) {
  using T = RT<float>;
  const float num = T::fma_(c.w, c.q, T::fma_(b.w, b.q, T::mul_(a.w, a.q)));
  const float den = T::add_(T::add_(a.w, b.w), c.w);
  return T::mul_(num, T::rcp(den));
}

// ------------------------------------------------------------------------------ arithmetic policy
//
// FP32 (the throughput path): fused multiply-adds, approximate reciprocals, smoothness indicators
// shared between the faces that use the same point triplet.
// FP64: every operation of the update is the one the plain definition writes, in its order, rounded
// once (explicit _rn intrinsics, so nothing is contracted or reordered): the same IEEE operations as a
// straightforward sequential implementation of Eq. euler2D / Sec. 2.2, so FP64 results are
// reproducible bit for bit by such an implementation.
template <typename real>
struct Ar;

template <>
struct Ar<float> {
  using T = RT<float>;
  static __device__ __forceinline__ void prims(float rho, float mx, float my, float E, float gm1, float& u,
                                               float& v, float& p) {
    const float rr = T::rcp(rho);
    u = mx * rr;
    v = my * rr;
    p = gm1 * T::fma_(-0.5f, T::add_(T::mul_(mx, u), T::mul_(my, v)), E);
  }
  static __device__ __forceinline__ void split(float F, float uu, float alpha, float& fp, float& fm) {
    const float hF = 0.5f * F, hal = 0.5f * alpha;
    fp = T::fma_(hal, uu, hF);
    fm = T::fma_(-hal, uu, hF);
  }
  static __device__ __forceinline__ float divided(float a, float b, float rd, double) { return T::mul_(a - b, rd); }
  static __device__ __forceinline__ float sum(float a, float b) { return T::add_(a, b); }
  // L = -(dF + dG) + S and the RK blend a U^n + b (W + dt L)
  static __device__ __forceinline__ float blend(bool use_un, float ra, float rb, float un, float w, float dt,
                                                float L) {
    const float inner = rb * T::fma_(dt, L, w);
    return use_un ? T::fma_(ra, un, inner) : inner;
  }
  // a further stage state's term of the five-stage scheme's blend
  static __device__ __forceinline__ float add_term(float out, float r, float x) { return T::fma_(r, x, out); }
  // cell-centre radius r_i = x0 + (i + 1/2) dx, in FP32
  template <typename G>
  static __device__ __forceinline__ float radius(const G& g, int i) {
    return T::fma_(static_cast<float>(i) + 0.5f, g.dx_r, g.x0_r);
  }
  static __device__ __forceinline__ float source(int f, bool rz, float grav, float rho, float mr, float mz, float E,
                                                float u, float v, float p, float r) {
    float S = 0.0f;
    if (rz) {  // -(1/r)(rho v_r, rho v_r^2, rho v_r v_z, (tau + p) v_r)
      const float rinv = T::rcp(r);
      S = (f == 0) ? -mr * rinv : (f == 1) ? -(mr * u) * rinv : (f == 2) ? -(mr * v) * rinv : -((E + p) * u) * rinv;
    }
    if (f == 2) S = T::fma_(rho, grav, S);  // -rho dPhi/dz with dPhi/dz = -g
    if (f == 3) S = T::fma_(mz, grav, S);   // -rho v_z dPhi/dz
    return S;
  }
  static __device__ __forceinline__ float lval(float D, float S) { return S - D; }
  static __device__ __forceinline__ float hamiltonian(float u, float v, float sf, float xm, float xp, float ym,
                                                     float yp) {
    const float gx = 0.5f * (xm + xp), gy = 0.5f * (ym + yp);
    const float adv = T::add_(T::mul_(u, gx), T::mul_(v, gy));
    const float nrm = T::sqrt_(T::add_(T::mul_(gx, gx), T::mul_(gy, gy)));
    const float H = T::fma_(-sf, nrm, adv);
    const float axl = fabsf(u) + sf, ayl = fabsf(v) + sf;
    return H - T::add_(T::mul_(0.5f * axl, xp - xm), T::mul_(0.5f * ayl, yp - ym));
  }
  // sound speed and the three signal speeds |u|+c, |v|+c, c+|u|+|v|
  static __device__ __forceinline__ void speeds(float rho, float mx, float my, float E, float gamma, float gm1,
                                                float& p, float& ax, float& ay, float& sm) {
    float u, v;
    prims(rho, mx, my, E, gm1, u, v, p);
    const float cs = T::sqrt_(gamma * p * T::rcp(rho));
    const float au = fabsf(u), av = fabsf(v);
    ax = au + cs;
    ay = av + cs;
    sm = T::add_(cs, T::add_(au, av));
  }
};

template <>
struct Ar<double> {
  static __device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ void prims(double rho, double mx, double my, double E, double gm1, double& u,
                                               double& v, double& p) {
    u = dv(mx, rho);
    v = dv(my, rho);
    p = ml(gm1, sb(E, ml(0.5, ad(ml(mx, u), ml(my, v)))));
  }
  static __device__ __forceinline__ double flux(int kind, double uu, double X, double vn, double p) {
    return kind == 0 ? X : (kind == 1) ? ad(ml(uu, vn), p) : (kind == 2) ? ml(uu, vn) : ml(ad(uu, p), vn);
  }
  static __device__ __forceinline__ void split(double F, double uu, double alpha, double& fp, double& fm) {
    fp = ml(0.5, ad(F, ml(alpha, uu)));
    fm = ml(0.5, sb(F, ml(alpha, uu)));
  }
  static __device__ __forceinline__ double divided(double a, double b, double, double h) { return dv(sb(a, b), h); }
  static __device__ __forceinline__ double sum(double a, double b) { return ad(a, b); }
  static __device__ __forceinline__ double blend(bool use_un, double ra, double rb, double un, double w, double dt,
                                                 double L) {
    const double inner = ml(rb, ad(w, ml(dt, L)));
    return use_un ? ad(ml(ra, un), inner) : inner;
  }
  static __device__ __forceinline__ double add_term(double out, double r, double x) { return ad(out, ml(r, x)); }
  // cell-centre radius r_i = x0 + (i + 1/2) dx, each operation rounded once
  template <typename G>
  static __device__ __forceinline__ double radius(const G& g, int i) {
    return ad(g.x0, ml(i + 0.5, g.dx));
  }
  static __device__ __forceinline__ double source(int f, bool rz, double grav, double rho, double mr, double mz,
                                                 double E, double u, double v, double p, double r) {
    double S = 0.0;
    if (rz) {
      S = (f == 0) ? dv(-mr, r) : (f == 1) ? dv(-ml(mr, u), r) : (f == 2) ? dv(-ml(mr, v), r) : dv(-ml(ad(E, p), u), r);
    }
    if (grav != 0.0) {
      if (f == 2) S = ad(S, ml(rho, grav));
      if (f == 3) S = ad(S, ml(mz, grav));
    }
    return S;
  }
  static __device__ __forceinline__ double lval(double D, double S) { return ad(-D, S); }
  static __device__ __forceinline__ double hamiltonian(double u, double v, double sf, double xm, double xp, double ym,
                                                       double yp) {
    const double gx = ml(0.5, ad(xm, xp)), gy = ml(0.5, ad(ym, yp));
    const double H = sb(ad(ml(u, gx), ml(v, gy)), ml(sf, __dsqrt_rn(ad(ml(gx, gx), ml(gy, gy)))));
    const double axl = ad(fabs(u), sf), ayl = ad(fabs(v), sf);
    return sb(H, ad(ml(ml(0.5, axl), sb(xp, xm)), ml(ml(0.5, ayl), sb(yp, ym))));
  }
  static __device__ __forceinline__ void speeds(double rho, double mx, double my, double E, double gamma,
                                                double gm1, double& p, double& ax, double& ay, double& sm) {
    double u, v;
    prims(rho, mx, my, E, gm1, u, v, p);
    const double cs = __dsqrt_rn(dv(ml(gamma, p), rho));
    ax = ad(fabs(u), cs);
    ay = ad(fabs(v), cs);
    sm = ad(ad(cs, fabs(u)), fabs(v));
  }
  // WENO5-JS in the textbook order (candidate values, smoothness indicators, normalised weights).
  static __device__ __forceinline__ double weno5(double a, double b, double c, double d, double e) {
    const double q0 = dv(ad(sb(ml(2.0, a), ml(7.0, b)), ml(11.0, c)), 6.0);
    const double q1 = dv(ad(ad(-b, ml(5.0, c)), ml(2.0, d)), 6.0);
    const double q2 = dv(sb(ad(ml(2.0, c), ml(5.0, d)), e), 6.0);
    const double k13 = 13.0 / 12.0;
    const double s0 = ad(sb(a, ml(2.0, b)), c), t0 = ad(sb(a, ml(4.0, b)), ml(3.0, c));
    const double s1 = ad(sb(b, ml(2.0, c)), d), t1 = sb(b, d);
    const double s2 = ad(sb(c, ml(2.0, d)), e), t2 = ad(sb(ml(3.0, c), ml(4.0, d)), e);
    const double b0 = ad(ml(ml(k13, s0), s0), ml(ml(0.25, t0), t0));
    const double b1 = ad(ml(ml(k13, s1), s1), ml(ml(0.25, t1), t1));
    const double b2 = ad(ml(ml(k13, s2), s2), ml(ml(0.25, t2), t2));
    const double e0 = ad(1e-6, b0), e1 = ad(1e-6, b1), e2 = ad(1e-6, b2);
    const double a0 = dv(0.1, ml(e0, e0)), a1 = dv(0.6, ml(e1, e1)), a2 = dv(0.3, ml(e2, e2));
    const double s = ad(ad(a0, a1), a2);
    const double ys = dv(1.0, s);  // the three quotients a_k / s share one correctly rounded reciprocal
    return ad(ad(ml(div_by(a0, s, ys), q0), ml(div_by(a1, s, ys), q1)), ml(div_by(a2, s, ys), q2));
  }
  // RN(a / b) from yb = RN(1 / b): q = RN(a yb), r = RN(a - q b) by a fused multiply-add, and one fused
  // correction q + r yb. Where a's significand is at least b's, q is within an ulp and Markstein's theorem
  // (IBM J. Res. Dev. 34, 1990) gives the correctly rounded quotient; otherwise q can be up to 1.5 ulps off
  // and r rounded, but the corrected value stays closer to a / b than any rounding midpoint is, except in
  // one corner (b's significand the largest below 2) that an exhaustive check covers. The result is the
  // double an IEEE division returns, for normal operands and quotients.
  static __device__ __forceinline__ double div_by(double a, double b, double yb) {
    const double q = __dmul_rn(a, yb);
    const double r = __fma_rn(-q, b, a);
    return __fma_rn(r, yb, q);
  }
};

// Flux kinds along a direction: 0 mass (flux = normal momentum), 1 normal momentum (m_n v_n + p),
// 2 tangential momentum (m_t v_n), 3 energy ((tau + p) v_n).
//
// One line of K cells: points m = 0 .. K+5 (cells -3 .. K+2 of the run), faces f = 0 .. K (left face
// of cell f). Writes (or adds) D[k] = (fhat_{k+1/2} - fhat_{k-1/2}) / h for k = 0 .. K-1, where
// fhat = W(f+ at the 5 points left-biased) + W(f- at the 5 points right-biased). The FP32 lines take their
// strides (points S, velocities VS, outputs DS) and the accumulate flag either as compile-time values (one
// instance per pass: every shared-memory access an immediate offset from the line's base pointers; used where
// one CTA per SM keeps the instruction footprint of the two instances affordable) or at run time (template
// values 0 and -1: one instance serves both passes).
//
// FP32 works on g+- = F +- alpha U = 2 f+- (the 1/2 goes into the final difference; eps scales by 4 with
// the squared differences, so the weights are those of f+-) through the triplet form above, and forms
// every flux kind as (U + c_E p) v_n + c_A p (c_E = 1 for energy, c_A = 1 for the normal momentum; the
// mass flux is rho v_n), so the line has no flux-kind branches.
template <int K, int CS = 0, int CVS = 0, int CDS = 0, int CACC = -1>
__device__ __forceinline__ void hydro_line_tri(const float* __restrict__ Uc, const float* __restrict__ vel,
                                               const float* __restrict__ pr, int S_rt, int VS_rt, int kind,
                                               float alpha, float rd, float* __restrict__ dst, int DS_rt,
                                               bool acc_rt) {
  using T = RT<float>;
  const int S = CS ? CS : S_rt, VS = CVS ? CVS : VS_rt, DS = CDS ? CDS : DS_rt;
  const bool accumulate = CACC >= 0 ? CACC != 0 : acc_rt;
  constexpr float EPS = 4e-6f * TRI_EPS_SCALE;
  const float rdh = T::mul_(0.5f, rd);
  const float cE = kind == 3 ? 1.0f : 0.0f, cA = kind == 1 ? 1.0f : 0.0f;
  float gp[K + 6], gm[K + 6];
  Tri32 tp[K + 6], tm[K + 6];
  float fh_prev = 0.0f;
#pragma unroll
  for (int m = 0; m < K + 6; ++m) {
    const float uu = Uc[m * S];
    const float pq = pr[m * S];
    const float F = T::fma_(T::fma_(cE, pq, uu), vel[m * VS], T::mul_(cA, pq));
    gp[m] = T::fma_(alpha, uu, F);
    gm[m] = T::fma_(-alpha, uu, F);
    if (m >= 2) {
      const int j = m - 1;
      if (j <= K + 3) tp[j] = tri_roles(tri_data(gp[j - 1], gp[j], gp[j + 1], EPS), true);
      if (j >= 2) tm[j] = tri_roles(tri_data(gm[j - 1], gm[j], gm[j + 1], EPS), false);
    }
    if (m >= 5) {
      const int f = m - 5;  // face f: the left face of run cell f
      const float plus = tri_face(tp[f + 1].up, tp[f + 2].mid, tp[f + 3].down);
      const float minus = tri_face(tm[f + 4].up, tm[f + 3].mid, tm[f + 2].down);
      const float fh = T::add_(plus, minus);
      if (f >= 1) {
        const float d = T::mul_(fh - fh_prev, rdh);
        float* o = dst + (f - 1) * DS;
        *o = accumulate ? T::add_(*o, d) : d;
      }
      fh_prev = fh;
    }
  }
}

// FP64: the textbook WENO5 per face side, in the plain definition's order.
template <int K>
__device__ __forceinline__ void hydro_line_f64(const double* __restrict__ Uc, const double* __restrict__ Xc,
                                               const double* __restrict__ vel, const double* __restrict__ pr, int S,
                                               int VS, int kind, double alpha, double h, double* __restrict__ dst,
                                               int DS, bool accumulate) {
  using A = Ar<double>;
  double fp[K + 6], fm[K + 6];
  double fh_prev = 0.0;
#pragma unroll
  for (int m = 0; m < K + 6; ++m) {
    const double uu = Uc[m * S];
    const double F = kind == 0 ? A::flux(0, uu, Xc[m * S], 0.0, 0.0) : A::flux(kind, uu, 0.0, vel[m * VS], pr[m * S]);
    A::split(F, uu, alpha, fp[m], fm[m]);
    if (m >= 5) {
      const int f = m - 5;
      const double plus = A::weno5(fp[f], fp[f + 1], fp[f + 2], fp[f + 3], fp[f + 4]);
      const double minus = A::weno5(fm[f + 5], fm[f + 4], fm[f + 3], fm[f + 2], fm[f + 1]);
      const double fh = A::sum(plus, minus);
      if (f >= 1) {
        const double d = A::divided(fh, fh_prev, 0.0, h);
        double* o = dst + (f - 1) * DS;
        *o = accumulate ? A::sum(*o, d) : d;
      }
      fh_prev = fh;
    }
  }
}

// One-sided HJ-WENO5 derivatives (Jiang & Peng 2000) of phi along a line of K cells from points
// m = 0 .. K+5: differences d_n = (phi_{n+1} - phi_n) / h, n = 0 .. K+4; cell k takes
// phi^- = W(d_k .. d_{k+4}) and phi^+ = W(d_{k+5} .. d_{k+1}), stored to om[k*DS], op[k*DS]. FP32 forms
// each difference triplet's smoothness data once for both derivatives.
template <int K, int CS = 0, int CDS = 0>
__device__ __forceinline__ void phi_line_tri(const float* __restrict__ ph, int S_rt, float rd, float* __restrict__ om,
                                             float* __restrict__ op, int DS_rt) {
  const int S = CS ? CS : S_rt, DS = CDS ? CDS : DS_rt;
  constexpr float EPS = 1e-6f * TRI_EPS_SCALE;
  float d[K + 5];
  Tri32 tl[K + 5], tr[K + 5];
  float prev = ph[0];
#pragma unroll
  for (int n = 0; n < K + 5; ++n) {
    const float nxt = ph[(n + 1) * S];
    d[n] = RT<float>::mul_(nxt - prev, rd);
    prev = nxt;
    if (n >= 2) {
      const int j = n - 1;
      const TriD32 td = tri_data(d[j - 1], d[j], d[j + 1], EPS);  // shared by both one-sided derivatives
      tl[j] = tri_roles(td, true);
      tr[j] = tri_roles(td, false);
    }
    if (n >= 5) {
      const int k = n - 5;
      om[k * DS] = tri_face(tl[k + 1].up, tl[k + 2].mid, tl[k + 3].down);
      op[k * DS] = tri_face(tr[k + 4].up, tr[k + 3].mid, tr[k + 2].down);
    }
  }
}

template <int K>
__device__ __forceinline__ void phi_line_f64(const double* __restrict__ ph, int S, double h, double* __restrict__ om,
                                             double* __restrict__ op, int DS) {
  using A = Ar<double>;
  double d[K + 5];
  double prev = ph[0];
#pragma unroll
  for (int n = 0; n < K + 5; ++n) {
    const double nxt = ph[(n + 1) * S];
    d[n] = A::divided(nxt, prev, 0.0, h);
    prev = nxt;
    if (n >= 5) {
      const int k = n - 5;
      om[k * DS] = A::weno5(d[k], d[k + 1], d[k + 2], d[k + 3], d[k + 4]);
      op[k * DS] = A::weno5(d[k + 5], d[k + 4], d[k + 3], d[k + 2], d[k + 1]);
    }
  }
}

// ------------------------------------------------------------------------------ small helpers

template <typename real>
__device__ __forceinline__ void load4(const real* p, real (&v)[4]) {
  if constexpr (sizeof(real) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

template <typename real>
__device__ __forceinline__ void store4(real* p, const real (&v)[4]) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

// The per-cell phase works on groups of EG = 3 neighbouring cells of a tile row: 20 groups per 60-cell
// row, 300 items for the 320 threads of a 15-row tile (4-cell groups left 95 threads idle and measured
// 4.6 % slower per launch despite their 16-byte vector accesses).
constexpr int EG = 3;
template <int G, typename real>
__device__ __forceinline__ void loadg(const real* p, real (&v)[G]) {
  if constexpr (G == 4) {
    load4(p, v);
  } else {
#pragma unroll
    for (int k = 0; k < G; ++k) v[k] = p[k];
  }
}
template <int G, typename real>
__device__ __forceinline__ void storeg(real* p, const real (&v)[G]) {
  if constexpr (G == 4) {
    store4(p, v);
  } else {
#pragma unroll
    for (int k = 0; k < G; ++k) p[k] = v[k];
  }
}

// Ghost images of interior cell (i, j) of a padded state: periodic wrap, transmissive copies of the
// edge cell, or mirror images with the normal momentum reversed (reflecting wall, symmetry axis).
// Corner ghosts are never read by the dimension-by-dimension stencil and are not written.
template <typename real, int NF>
__device__ __forceinline__ void write_ghost_images(real* out, long long fs, int pitch, int nx, int ny,
                                                   const int* bc, int i, int j, const real (&val)[NF]) {
  auto put = [&](int gi, int gj, bool fx, bool fy) {
    const long long off = static_cast<long long>(gj + GY) * pitch + gi + GX;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      real v = val[f];
      if ((f == 1 && fx) || (f == 2 && fy)) v = -v;
      out[f * fs + off] = v;
    }
  };
  if (i < 3 || i >= nx - 3) {
    const int bl = bc[0], bh = bc[1];
    if (bl == BC_PERIODIC) {
      if (i >= nx - 3) put(i - nx, j, false, false);
    } else if (bl == BC_TRANSMISSIVE) {
      if (i == 0) { put(-1, j, false, false); put(-2, j, false, false); put(-3, j, false, false); }
    } else if (i < 3) {
      put(-1 - i, j, true, false);
    }
    if (bh == BC_PERIODIC) {
      if (i < 3) put(nx + i, j, false, false);
    } else if (bh == BC_TRANSMISSIVE) {
      if (i == nx - 1) { put(nx, j, false, false); put(nx + 1, j, false, false); put(nx + 2, j, false, false); }
    } else if (i >= nx - 3) {
      put(2 * nx - 1 - i, j, true, false);
    }
  }
  if (j < 3 || j >= ny - 3) {
    const int bl = bc[2], bh = bc[3];
    if (bl == BC_PERIODIC) {
      if (j >= ny - 3) put(i, j - ny, false, false);
    } else if (bl == BC_TRANSMISSIVE) {
      if (j == 0) { put(i, -1, false, false); put(i, -2, false, false); put(i, -3, false, false); }
    } else if (j < 3) {
      put(i, -1 - j, false, true);
    }
    if (bh == BC_PERIODIC) {
      if (j < 3) put(i, ny + j, false, false);
    } else if (bh == BC_TRANSMISSIVE) {
      if (j == ny - 1) { put(i, ny, false, false); put(i, ny + 1, false, false); put(i, ny + 2, false, false); }
    } else if (j >= ny - 3) {
      put(i, 2 * ny - 1 - j, false, true);
    }
  }
}

// ------------------------------------------------------------------------------ tile geometry

// The FP32 kernel of one CTA per SM (640 threads, 60 x 30 tiles) has the shared memory to hold the tile's
// own cells of U^n: a TMA copy issued at the start of each tile, read by the per-cell phase (the other
// variants prefetch those cells into L2 instead).
template <typename real>
__host__ __device__ constexpr bool un_in_smem(int threads) { return sizeof(real) == 4 && threads >= 640; }

template <typename real, int NF, int TY, bool UNS = false>
struct Tile {
  static constexpr int TX = TILE_X, W = BOX_W, H = TY + 6, K = RUN, NQ = TX / RUN;
  static constexpr int NQY = TY / RUN;                   // y runs per column
  static constexpr int TYP = ((TY + 7) / 8) * 8;        // rows padded to whole 8-row lane groups
  static constexpr int XI_PER_C = TYP * NQ;             // x-pass items per field (multiple of 32)
  static constexpr int YI_PER_C = 64 * NQY;             // y-pass items per field (60 columns padded to 64)
  static constexpr int BOX = NF * H * W;                // elements of one halo box
  // shared-memory carve-up (elements of real); each box buffer starts on a 128-byte boundary (TMA)
  static constexpr int BOX_PAD = ((BOX * (int)sizeof(real) + 127) / 128) * 128 / (int)sizeof(real);
  static constexpr int OFF_U0 = 0;                      // [NF][H][W]   halo box, buffer 0
  static constexpr int OFF_U1 = OFF_U0 + BOX_PAD;       // [NF][H][W]   halo box, buffer 1
  static constexpr int OFF_PU = OFF_U1 + BOX_PAD;       // [TY][W]      u on the tile rows
  static constexpr int OFF_PV = OFF_PU + TY * W;        // [H][TX]      v on the tile columns
  static constexpr int OFF_PP = OFF_PV + H * TX;        // [H][W]       p
  // [NF][TY][TX] dF/dx + dG/dy, then the tile's outputs (the tensor store's source: 128-byte aligned)
  static constexpr int OFF_D = (((OFF_PP + H * W) * (int)sizeof(real) + 127) / 128) * 128 / (int)sizeof(real);
  static constexpr int OFF_X = OFF_D + NF * TY * TX;    // [4][TY][TX]  phi_x^-, phi_x^+, phi_y^-, phi_y^+
  static constexpr int END_X = OFF_X + (NF == 5 ? 4 * TY * TX : 0);
  static constexpr int OFF_UN = ((END_X * (int)sizeof(real) + 127) / 128) * 128 / (int)sizeof(real);  // [NF][TY][TX]
  static constexpr int ELEMS = UNS ? OFF_UN + NF * TY * TX : END_X;
  static constexpr unsigned UN_BYTES = NF * TY * TX * sizeof(real);
  // per-warp running slots (<= 20 warps): 3 maxima and 5 totals; FP32 adds 5 compensation terms (16 floats)
  static constexpr int RED_STRIDE = sizeof(real) == 4 ? 16 : 8;
  static constexpr int RED_ELEMS = 20 * RED_STRIDE;
  static constexpr size_t RED_OFF = ((ELEMS * sizeof(real) + 15) / 16) * 16;
  static constexpr size_t BYTES = RED_OFF + RED_ELEMS * sizeof(real) + 32;  // + 3 mbarriers
  static constexpr unsigned BOX_BYTES = BOX * sizeof(real);
  static_assert(TX % RUN == 0 && TY % RUN == 0, "tiles are whole runs");
  static_assert(TX % EG == 0, "tile rows are whole cell groups");
};

// The five-stage scheme's further stage states that a tile's blend adds (its own cells): into L2, when the
// interior maps' boxes are the launch's tiles.
template <typename real>
__device__ __forceinline__ void prefetch_stage_terms(const GridParams<real>* m, int x, int y, int TY) {
  if (m->tmap_ty != TY) return;
  if (m->tmap_ux0) tma_prefetch_l2_3d(m->tmap_ux0, x, y, 0);
  if (m->tmap_ux1) tma_prefetch_l2_3d(m->tmap_ux1, x, y, 0);
}

// Issue the TMA copy of one tile's halo box (one thread): arm the barrier with the box's bytes, then one
// tensor copy of the (68, TY + 6, NF) box at padded column tx * 60, row ty * TY. With prefetch_un, the
// tile's own cells of U^n (a (60, TY, NF) box) are prefetched into L2 for the tile's per-cell phase. m may
// point to shared memory.
template <typename real>
__device__ __forceinline__ void issue_box(const GridParams<real>* m, int tile, int TY, real* box, uint64_t* bar,
                                          unsigned bytes, bool prefetch_un) {
  const int tiles_x = m->tiles_x;
  const void* map = m->tmap_win;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  mbar_arrive_expect_tx(bar, bytes);
  tma_load_3d(box, map, tx * TILE_X, ty * TY, 0, bar);
  if (prefetch_un) tma_prefetch_l2_3d(m->tmap_un, tx * TILE_X + GX, ty * TY + GY, 0);  // the tile's own cells
  prefetch_stage_terms(m, tx * TILE_X + GX, ty * TY + GY, TY);
}

// ------------------------------------------------------------------------------ the stage kernel

template <typename real, int NF, int TY, int NT>
__global__ void __launch_bounds__(NT, (NT <= 320 && sizeof(real) == 4 ? 2 : 1))
    stage_kernel(const GridParams<real>* __restrict__ members, const WorkItem* __restrict__ work, int nwork,
                 StageCtl ctl) {
  using T = RT<real>;
  constexpr bool kUnSmem = un_in_smem<real>(NT);
  using TL = Tile<real, NF, TY, kUnSmem>;
  constexpr int TX = TL::TX, W = TL::W, H = TL::H, K = TL::K, NQ = TL::NQ;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* sm = reinterpret_cast<real*>(smem_raw);
  real* su = sm + TL::OFF_PU;
  real* sv = sm + TL::OFF_PV;
  real* sp = sm + TL::OFF_PP;
  real* sD = sm + TL::OFF_D;
  real* sX = sm + TL::OFF_X;
  real* red = reinterpret_cast<real*>(smem_raw + TL::RED_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + TL::RED_ELEMS);  // one barrier per box buffer, one for U^n
  real* sUn = sm + TL::OFF_UN;
  __shared__ GridParams<real> g;
  __shared__ int s_abort;
  // stage scalars, formed once per CTA and member (dt needs an FP64 division at stage 0; the FP64 pipe
  // is 1/64 of the FP32 rate, so no per-thread FP64 work stays in the tile loop of the FP32 kernel)
  __shared__ double s_dtd;
  __shared__ real s_dt, s_ra, s_rb, s_ax, s_ay, s_rx0, s_rx1;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;

  // compile-time line strides where one CTA runs per SM (its warps share one phase's code, so the two
  // instances' instruction footprint costs less than the address arithmetic they save: 2.87 -> 2.78 ms per
  // 8192^2 launch of the 640-thread variant; with two CTAs per SM the runtime-stride line measured faster)
  constexpr bool kCts = NT >= 640;
  // the 60x30 variant's level-set warps, whose lines are shorter than the hydro ones, also form the
  // Hamiltonian of their y-pass cells (after a barrier among themselves between their two passes); the
  // per-cell phase then reads it instead of the four one-sided derivatives and u, v
  constexpr bool kPhiH = kUnSmem && NF == 5;
  // the tensor copies write 128-byte aligned buffers: a launch that finds its dynamic shared memory
  // elsewhere reports it and returns before any copy (the same address for every thread)
  if ((smem_u32(smem_raw) & 127u) != 0u) {
    if (tid == 0 && nwork > 0) atomicOr(members[work ? work[0].member : 0].err, ERR_LAYOUT);
    return;
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    s_abort = 0;
  }
  for (int k = tid; k < TL::RED_ELEMS; k += NT) red[k] = real(0);
  __syncthreads();

  // the blend of stages 2 and 3 reads U^n in the per-cell phase: its tile box is prefetched into L2 with
  // the halo box, or (one CTA per SM, FP32) copied into shared memory at the start of the tile
  const bool blend_un = ctl.mode == 0 && ctl.rk_a != 0.0;
  const bool prefetch_un = blend_un && !kUnSmem;
  unsigned un_parity = 0u;
  // prologue: the first work item's box
  if (tid == 0 && static_cast<int>(blockIdx.x) < nwork) {
    const int w0 = blockIdx.x;
    const int m0 = work ? work[w0].member : 0;
    const int t0 = work ? work[w0].tile : ((sizeof(real) == 8 && ctl.mode == 2) ? w0 >> 2 : ctl.w0 + w0);
    issue_box<real>(members + m0, t0, TY, sm + TL::OFF_U0, &bar[0], TL::BOX_BYTES, prefetch_un);
  }

  unsigned parity[2] = {0u, 0u};
  int cur_member = -1;
  int it = 0;
  // The one-CTA-per-SM variant pipelines the per-cell phase of a tile with the next tile's box wait and
  // primitives (no barrier between them: the per-cell phase reads only the tile's box, sD, sX and the U^n
  // buffer, which also receives its outputs): the previous tile's tensor store and the next box are issued
  // after the primitives' barrier, and the tile's U^n copy after the store has read the buffer.
  bool prev_store = false;  // the previous tile's outputs wait in sUn for their tensor store
  const void* prev_map = nullptr;
  int prev_x = 0, prev_y = 0;
  // Reductions of the outputs (next stage's alpha, next step's dt, totals) accumulate per warp in
  // red[warp * RED_STRIDE + slot] across this CTA's tiles of one member (each tile: a warp shuffle, lane 0
  // updates its slots) and are flushed by each warp's lane 0 -- one atomic per slot, no barrier -- when
  // the member changes (batched launches change member almost every tile) and at the end. The FP32
  // kernel keeps its slots in FP32 (maxima are exact; each total is a compensated sum, value + error
  // term, as accurate as an FP64 running sum) so that its tile loop issues no FP64 instruction.
  auto flush = [&]() {  // per warp: lane 0 folds its own slots into the member's slots, then clears them
    if (ctl.mode != 0 || lane != 0) return;
    real* r = red + warp * TL::RED_STRIDE;
    if (g.alpha_out) {
      T::atomic_max(&g.alpha_out[0], r[0]);
      T::atomic_max(&g.alpha_out[1], r[1]);
    }
    if (ctl.last) T::atomic_max(g.smax, r[2]);
    if (g.totals) {
      if constexpr (sizeof(real) == 4) {  // the cell volume, applied once
        const double vol = g.geometry == 1 ? 6.283185307179586 * g.dx * g.dy : g.dx * g.dy;
        for (int f = 0; f < NF; ++f)
          atomicAdd(&g.totals[f], (static_cast<double>(r[3 + f]) + static_cast<double>(r[8 + f])) * vol);
      } else {
        for (int f = 0; f < NF; ++f) atomicAdd(&g.totals[f], r[3 + f]);
      }
    }
    for (int k = 0; k < TL::RED_STRIDE; ++k) r[k] = real(0);
  };
  for (int w = blockIdx.x; w < nwork; w += gridDim.x, ++it) {
    const int b = it & 1;
    real* sU = sm + (b ? TL::OFF_U1 : TL::OFF_U0);
    const int member = work ? work[w].member : 0;
    // mode 2 (field split, FP64 only): item w is field w & 3 of tile w >> 2
    constexpr bool kSplit = sizeof(real) == 8;
    const int tile = work ? work[w].tile : ((kSplit && ctl.mode == 2) ? w >> 2 : ctl.w0 + w);
    const int split_field = (kSplit && ctl.mode == 2) ? (w & 3) : -1;
    if (member != cur_member) {
      if (cur_member >= 0) flush();
      __syncthreads();
      if (tid == 0) {
        g = members[member];
        const double d = ctl.stage == 0 ? (g.dt_src ? *g.dt_src : g.cfl_delta / static_cast<double>(*g.smax))
                                        : *g.dt_cur;
        s_dtd = d;
        s_dt = static_cast<real>(d * ctl.rk_c);  // the stage's multiple of dt (1 in SSP-RK3)
        s_ra = static_cast<real>(ctl.rk_a);
        s_rb = static_cast<real>(ctl.rk_b);
        s_rx0 = static_cast<real>(ctl.rk_x0);
        s_rx1 = static_cast<real>(ctl.rk_x1);
        s_ax = g.alpha_in[0];  // the Lax-Friedrichs speeds, written by the previous launch
        s_ay = g.alpha_in[1];
      }
      __syncthreads();
      cur_member = member;
    }
    // prefetch the next item's box into the other buffer (free since the previous tile ended; pipelined:
    // after the primitives' barrier)
    const int wn = w + gridDim.x;
    if (!kUnSmem && tid == 0 && wn < nwork) {
      const int mn = work ? work[wn].member : 0;
      // the member's parameters come from the shared copy when the next item is of the same member
      issue_box<real>(mn == member ? &g : members + mn,
                      work ? work[wn].tile : ((kSplit && ctl.mode == 2) ? wn >> 2 : ctl.w0 + wn), TY,
                      sm + (b ? TL::OFF_U0 : TL::OFF_U1), &bar[b ^ 1], TL::BOX_BYTES, prefetch_un);
    }
    const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
    const int x0 = tx * TX, y0 = ty * TY;
    const long long fs = g.fstride;
    const int pitch = g.pitch;

    // stage scalars (overlap with the copies)
    const real ax = s_ax, ay = s_ay;
    if (tile == 0 && tid == 0 && ctl.mode == 0) {
      const double dtd = s_dtd;  // once per grid and stage
      if (ctl.stage == 0) {
        *g.dt_cur = dtd;
        *g.t_acc += dtd;
      }
      if (ctl.stage == 1) {
        *g.smax = real(0);
        if (g.totals_reset)
          for (int f = 0; f < 5; ++f) g.totals_reset[f] = 0.0;
      }
      if (g.alpha_zero) {
        g.alpha_zero[0] = real(0);
        g.alpha_zero[1] = real(0);
      }
      if (g.dt_log) {
        const int idx = *g.log_count;
        if (idx < g.log_cap) {
          if (ctl.stage == 0) g.dt_log[idx] = dtd;
          g.alpha_log[6 * idx + 2 * ctl.stage + 0] = static_cast<double>(ax);
          g.alpha_log[6 * idx + 2 * ctl.stage + 1] = static_cast<double>(ay);
        }
        if (ctl.last) *g.log_count = idx + 1;
      }
    }

    // ---- A. wait for this tile's halo box
    if (!mbar_wait_bounded(&bar[b], parity[b])) {
      atomicOr(g.err, ERR_TIMEOUT);
      s_abort = 1;
    }
    parity[b] ^= 1u;
    if constexpr (!kUnSmem) {
      __syncthreads();
      if (s_abort) {
        // a copy did not complete: before the CTA leaves (and its shared memory is reused), wait, again
        // with a limit, for the copies it still has in flight (this box and the prefetched next one)
        if (tid == 0) {
          mbar_wait_limit(&bar[b], parity[b] ^ 1u, TILE_WAIT_POLLS, TILE_WAIT_NS);
          if (wn < nwork) mbar_wait_limit(&bar[b ^ 1], parity[b ^ 1], TILE_WAIT_POLLS, TILE_WAIT_NS);
        }
        break;
      }
    }
    const bool maps_fit = g.tmap_ty == TY;  // the interior maps' boxes are this kernel's tiles
    // the tile's own cells of U^n, copied during the x pass
    const bool un_copy = kUnSmem && blend_un && maps_fit;

    // ---- B. primitive variables
    const real gm1 = g.gm1;
    for (int idx = tid; idx < H * W; idx += NT) {
      const int row = idx / W, col = idx - row * W;
      const bool irow = row >= 3 && row < TY + 3;
      const bool icol = col >= 4 && col < TX + 4;
      if (!irow && !icol) continue;
      real u, v, p;
      Ar<real>::prims(sU[0 * H * W + idx], sU[1 * H * W + idx], sU[2 * H * W + idx], sU[3 * H * W + idx], gm1, u,
                      v, p);
      sp[idx] = p;
      if (irow) su[(row - 3) * W + col] = u;
      if (icol) sv[row * TX + (col - 4)] = v;
    }
    if constexpr (kUnSmem) {
      if (prev_store) fence_proxy_async_smem();  // the previous tile's outputs, for its tensor store
      __syncthreads();
      if (s_abort) {
        // a copy did not complete: wait (with a limit) for the copies in flight -- this box, or the
        // previous tile's U^n -- before the CTA leaves; nothing else has been issued since
        if (tid == 0) {
          mbar_wait_limit(&bar[b], parity[b] ^ 1u, TILE_WAIT_POLLS, TILE_WAIT_NS);
          mbar_wait_limit(&bar[2], un_parity ^ 1u, TILE_WAIT_POLLS, TILE_WAIT_NS);
        }
        prev_store = false;
        break;
      }
      if (tid == 0) {
        fence_proxy_async_smem();  // everyone's reads of the previous tile's box and of sUn come first
        if (prev_store) {
          tma_store_3d(prev_map, sUn, prev_x, prev_y, 0);
          bulk_commit();
        }
        if (wn < nwork) {
          const int mn = work ? work[wn].member : 0;
          issue_box<real>(mn == member ? &g : members + mn, work ? work[wn].tile : ctl.w0 + wn, TY,
                          sm + (b ? TL::OFF_U0 : TL::OFF_U1), &bar[b ^ 1], TL::BOX_BYTES, false);
        }
      }
    } else {
      if (tid == 0) bulk_wait_read_all();  // the previous tile's tensor store has read sD
      __syncthreads();
    }

    // ---- C/D. x pass then y pass through the same line code: items (field, line, run of 15 cells)
    // Items [c per_c, (c+1) per_c) of both passes carry field c. When every item has its own thread, the
    // y pass of hydro field c (which adds to the rows of sD that field c's x pass wrote) only waits for
    // the warps of field c (named barrier 1 + c), and the level set's two passes share no data at all.
    constexpr bool kFieldSync = TL::XI_PER_C == TL::YI_PER_C && NF * TL::XI_PER_C <= NT && TL::XI_PER_C % 32 == 0;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const bool xp = pass == 0;
      const int per_c = xp ? TL::XI_PER_C : TL::YI_PER_C;
      const real alpha = xp ? ax : ay;
      const real rd = xp ? g.rdx : g.rdy;
      const double h = xp ? g.dx : g.dy;
      const int item0 = split_field >= 0 ? split_field * per_c : 0;
      const int item1 = split_field >= 0 ? item0 + per_c : NF * per_c;
      for (int item = item0 + tid; item < item1; item += NT) {
        const int c = item / per_c;
        const int rem = item - c * per_c;
        int trow, tcol, brow, bcol;
        if (xp) {  // lanes: 8 consecutive rows x 4 runs -> all 32 banks (68 = 4 mod 32, 15 = 3 mod 4)
          trow = (rem / (8 * NQ)) * 8 + (rem & 7);
          tcol = ((rem >> 3) % NQ) * K;
          if (trow >= TY) continue;
          brow = trow + 3;
          bcol = tcol + 1;
        } else {  // lanes: consecutive columns
          tcol = rem & 63;
          trow = (rem >> 6) * K;
          if (tcol >= TX) continue;
          brow = trow;
          bcol = tcol + 4;
        }
        const int S = xp ? 1 : W;
        const int DS = xp ? 1 : TX;
        if (c < 4) {
          // the divergence comes from another launch (char_div_kernel, or mode 2 of this kernel)
          if (g.ext_div && split_field < 0) continue;
          const int kind = (c == 0) ? 0 : (c == 3) ? 3 : ((c == 1) == xp) ? 1 : 2;
          const real* Uc = sU + (c * H + brow) * W + bcol;
          const real* Xc = sU + ((xp ? 1 : 2) * H + brow) * W + bcol;
          const real* vel = xp ? su + trow * W + bcol : sv + brow * TX + tcol;
          if constexpr (sizeof(real) == 4) {
            if constexpr (kCts) {
              if (xp)
                hydro_line_tri<K, 1, 1, 1, 0>(Uc, vel, sp + brow * W + bcol, 1, 1, kind, alpha, rd,
                                              sD + (c * TY + trow) * TX + tcol, 1, false);
              else
                hydro_line_tri<K, W, TX, TX, 1>(Uc, vel, sp + brow * W + bcol, W, TX, kind, alpha, rd,
                                                sD + (c * TY + trow) * TX + tcol, TX, true);
            } else {
              hydro_line_tri<K>(Uc, vel, sp + brow * W + bcol, S, xp ? 1 : TX, kind, alpha, rd,
                                sD + (c * TY + trow) * TX + tcol, DS, !xp);
            }
          } else
            hydro_line_f64<K>(Uc, Xc, vel, sp + brow * W + bcol, S, xp ? 1 : TX, kind, alpha, h,
                              sD + (c * TY + trow) * TX + tcol, DS, !xp);
        } else {
          real* om = sX + ((xp ? 0 : 2) * TY + trow) * TX + tcol;
          if constexpr (sizeof(real) == 4) {
            if constexpr (kCts) {
              if (xp)
                phi_line_tri<K, 1, 1>(sU + (4 * H + brow) * W + bcol, 1, rd, om, om + TY * TX, 1);
              else {
                phi_line_tri<K, W, TX>(sU + (4 * H + brow) * W + bcol, W, rd, om, om + TY * TX, TX);
                if constexpr (kPhiH) {
                  const real sf = g.flame_speed;
#pragma unroll
                  for (int k = 0; k < K; ++k) {
                    const int idx = (trow + k) * TX + tcol;
                    sX[idx] = Ar<real>::hamiltonian(su[(trow + k) * W + tcol + 4], sv[(trow + k + 3) * TX + tcol], sf,
                                                    sX[idx], sX[TY * TX + idx], sX[2 * TY * TX + idx],
                                                    sX[3 * TY * TX + idx]);
                  }
                }
              }
            } else {
              phi_line_tri<K>(sU + (4 * H + brow) * W + bcol, S, rd, om, om + TY * TX, DS);
            }
          } else
            phi_line_f64<K>(sU + (4 * H + brow) * W + bcol, S, h, om, om + TY * TX, DS);
        }
      }
      if (kUnSmem && xp && tid == 0) {
        bulk_wait_read_all();  // the previous tile's tensor store has read sUn
        if (un_copy) {
          mbar_arrive_expect_tx(&bar[2], TL::UN_BYTES);
          tma_load_3d(sUn, g.tmap_un, x0 + GX, y0 + GY, 0, &bar[2]);
        }
      }
      if (xp && kFieldSync && split_field < 0) {
        const int cm = tid / TL::XI_PER_C;  // the field whose lines this thread carries in both passes
        switch (cm) {  // warp-uniform
          case 0: named_barrier_sync<1>(TL::XI_PER_C); break;
          case 1: named_barrier_sync<2>(TL::XI_PER_C); break;
          case 2: named_barrier_sync<3>(TL::XI_PER_C); break;
          case 3: named_barrier_sync<4>(TL::XI_PER_C); break;
          default:
            if constexpr (kPhiH) named_barrier_sync<5>(TL::XI_PER_C);  // the level set's two passes
            break;
        }
      } else {
        __syncthreads();
      }
    }

    // ---- E. per cell: sources, RK blend, stores, ghost images, reductions
    // a whole tile inside the grid leaves through one tensor store of its outputs (written over its own
    // D values in sD); a ragged tile is stored cell by cell (a store of its box would reach the ghost frame)
    const bool tile_store = split_field < 0 && maps_fit && x0 + TX <= g.nx && y0 + TY <= g.ny;
    if (un_copy) {  // each thread waits for the U^n copy itself (its writes become visible)
      if (!mbar_wait_bounded(&bar[2], un_parity)) {
        atomicOr(g.err, ERR_TIMEOUT);
        s_abort = 1;  // this tile's outputs are void; the CTA leaves at the end of the tile
      }
      un_parity ^= 1u;
    }
    real amx = real(0), amy = real(0), smx = real(0);
    // totals: FP64 per cell in the FP64 kernel; the FP32 kernel sums U_f (times r in (r,z)) over a thread's
    // cells and then over its warp in FP32, the warp partials over the CTA's tiles as compensated FP32
    // sums and across the grid in FP64, with dV = dx dy (or 2 pi dr dz) applied once at the end
    double tot[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    real totr[5] = {real(0), real(0), real(0), real(0), real(0)};
    if (split_field >= 0) {  // field split: this CTA's field's dF/dx + dG/dy goes to the divergence buffer
      real* D = const_cast<real*>(g.ext_div) + split_field * fs;
      for (int idx = tid; idx < TY * TX; idx += NT) {
        const int row = idx / TX, col = idx - row * TX;
        const int i = x0 + col, j = y0 + row;
        if (i < g.nx && j < g.ny)
          D[static_cast<long long>(j + GY) * pitch + i + GX] = sD[(split_field * TY + row) * TX + col];
      }
    } else {
      const int nx = g.nx, ny = g.ny;
      const real gamma = g.gamma, grav = g.gravity, sf = g.flame_speed;
      const bool rz = g.geometry == 1;
      const real dt = s_dt;
      const real ra = s_ra, rb = s_rb;
      const bool use_un = blend_un;
      const real rx0 = s_rx0, rx1 = s_rx1;
      const bool use_x0 = g.ux0 != nullptr && ctl.mode == 0, use_x1 = g.ux1 != nullptr && ctl.mode == 0;
      constexpr int NG = TX / EG;
      for (int it2 = tid; it2 < TY * NG; it2 += NT) {
        const int row = it2 / NG, g4 = it2 - row * NG;
        const int j = y0 + row, ib = x0 + EG * g4;
        if (j >= ny || ib >= nx) continue;
        const int nvalid = min(EG, nx - ib);
        const long long gbase = static_cast<long long>(j + GY) * pitch + ib + GX;
        const int srow = row + 3, scol = 4 + EG * g4, tcol = EG * g4;
        real o[NF][EG];
        {
          real u4[EG], v4[EG], p4[EG], rr[EG];
          if (rz) {
#pragma unroll
            for (int e = 0; e < EG; ++e) rr[e] = Ar<real>::radius(g, ib + e);
          }
          const bool sources = rz || grav != real(0);
          if constexpr (kUnSmem) {  // pipelined: the next tile's primitives overwrite su, sv, sp meanwhile,
                                    // so the cell's own come from its box values (the same operations)
            if (sources || (NF == 5 && !kPhiH)) {
#pragma unroll
              for (int e = 0; e < EG; ++e) {
                const int c0 = srow * W + scol + e;
                Ar<real>::prims(sU[0 * H * W + c0], sU[1 * H * W + c0], sU[2 * H * W + c0], sU[3 * H * W + c0], gm1,
                                u4[e], v4[e], p4[e]);
              }
            }
          } else {
            if (sources || NF == 5) {  // the level set's Hamiltonian needs u and v, the sources p as well
              loadg<EG>(su + row * W + scol, u4);
              loadg<EG>(sv + srow * TX + tcol, v4);
            }
            if (sources) loadg<EG>(sp + srow * W + scol, p4);
          }
          // every U^n value of the group is loaded before any is used: one memory latency, not one per field
          real unv[NF][EG];
          if (un_copy) {  // columns past the grid hold ghost or fill values, never stored
#pragma unroll
            for (int f = 0; f < NF; ++f) loadg<EG>(sUn + (f * TY + row) * TX + tcol, unv[f]);
          } else if (use_un) {
            if (nvalid == EG) {
#pragma unroll
              for (int f = 0; f < NF; ++f) loadg<EG>(g.un + f * fs + gbase, unv[f]);
            } else {
#pragma unroll
              for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EG; ++e) unv[f][e] = (e < nvalid) ? g.un[f * fs + gbase + e] : real(0);
            }
          } else {
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
              for (int e = 0; e < EG; ++e) unv[f][e] = real(0);
          }

#pragma unroll
          for (int f = 0; f < NF; ++f) {
            real Uv[EG], Dv[EG];
            const real (&un)[EG] = unv[f];
            loadg<EG>(sU + (f * H + srow) * W + scol, Uv);
            if (f < 4) {
              if (g.ext_div) {
                loadg<EG>(g.ext_div + f * fs + gbase, Dv);
              } else {
                loadg<EG>(sD + (f * TY + row) * TX + tcol, Dv);
              }
            } else if constexpr (kPhiH) {  // level set: its Hamiltonian, formed in the y pass
              loadg<EG>(sX + (0 * TY + row) * TX + tcol, Dv);
            } else {  // level set: the local Lax-Friedrichs Hamiltonian from the four one-sided derivatives
              real xm[EG], xq[EG], ym[EG], yq[EG];
              loadg<EG>(sX + (0 * TY + row) * TX + tcol, xm);
              loadg<EG>(sX + (1 * TY + row) * TX + tcol, xq);
              loadg<EG>(sX + (2 * TY + row) * TX + tcol, ym);
              loadg<EG>(sX + (3 * TY + row) * TX + tcol, yq);
#pragma unroll
              for (int e = 0; e < EG; ++e) Dv[e] = Ar<real>::hamiltonian(u4[e], v4[e], sf, xm[e], xq[e], ym[e], yq[e]);
            }
#pragma unroll
            for (int e = 0; e < EG; ++e) {
              real S = real(0);
              if (f < 4 && (rz || grav != real(0))) {
                const real rho = sU[(0 * H + srow) * W + scol + e], mr = sU[(1 * H + srow) * W + scol + e];
                const real mz = sU[(2 * H + srow) * W + scol + e], E = sU[(3 * H + srow) * W + scol + e];
                S = Ar<real>::source(f, rz, grav, rho, mr, mz, E, u4[e], v4[e], p4[e], rr[e]);
              }
              const real L = (f < 4) ? Ar<real>::lval(Dv[e], S) : -Dv[e];
              o[f][e] = (ctl.mode == 1) ? L : Ar<real>::blend(use_un, ra, rb, un[e], Uv[e], dt, L);
            }
            // the five-stage scheme's further stage states (the cell's own values, like U^n)
            if (use_x0) {
#pragma unroll
              for (int e = 0; e < EG; ++e)
                if (e < nvalid) o[f][e] = Ar<real>::add_term(o[f][e], rx0, g.ux0[f * fs + gbase + e]);
            }
            if (use_x1) {
#pragma unroll
              for (int e = 0; e < EG; ++e)
                if (e < nvalid) o[f][e] = Ar<real>::add_term(o[f][e], rx1, g.ux1[f * fs + gbase + e]);
            }
          }
        }
        // the outputs: over the cells' own D values in sD (the tile's tensor store), or cell by cell into
        // the padded working state
        if (tile_store) {  // pipelined: over the cell's own U^n values in sUn, read above by this thread
#pragma unroll
          for (int f = 0; f < NF; ++f) storeg<EG>((kUnSmem ? sUn : sD) + (f * TY + row) * TX + tcol, o[f]);
        } else {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            real* dstp = g.out + f * fs + gbase;
            if (nvalid == EG) {
              storeg<EG>(dstp, o[f]);
            } else {
#pragma unroll
              for (int e = 0; e < EG; ++e)
                if (e < nvalid) dstp[e] = o[f][e];
            }
          }
        }
        if (ctl.mode == 1) continue;
        // ghost images and reductions
#pragma unroll
        for (int e = 0; e < EG; ++e) {
          if (e >= nvalid) break;
          const int i = ib + e;
          if (i < 3 || i >= nx - 3 || j < 3 || j >= ny - 3) {
            real val[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) val[f] = o[f][e];
            write_ghost_images<real, NF>(g.out, fs, pitch, nx, ny, g.bc, i, j, val);
          }
          // speeds of the output state (next stage's alpha, next step's dt) and validity
          const real rho = o[0][e], mx = o[1][e], my = o[2][e], E = o[3][e];
          real p, sx, sy, sm;
          Ar<real>::speeds(rho, mx, my, E, gamma, gm1, p, sx, sy, sm);
          // a non-finite momentum or energy makes p NaN or -inf, or c (hence c + |u| + |v|) infinite
          bool ok = rho > real(0) && p > real(0) && T::finite(sm);
          if (NF == 5) ok = ok && T::finite(o[NF - 1][e]);
          if (!ok) atomicOr(g.err, ERR_NONPHYSICAL);
          amx = fmax(amx, sx);
          amy = fmax(amy, sy);
          smx = fmax(smx, sm);
          if (g.totals) {
            if constexpr (sizeof(real) == 4) {
              const real wr = rz ? T::fma_(static_cast<real>(i) + real(0.5), g.dx_r, g.x0_r) : real(1);
#pragma unroll
              for (int f = 0; f < NF; ++f) totr[f] = T::fma_(o[f][e], wr, totr[f]);
            } else {
              const double dV = rz ? 6.283185307179586 * (g.x0 + (i + 0.5) * g.dx) * g.dx * g.dy : g.dx * g.dy;
#pragma unroll
              for (int f = 0; f < NF; ++f) tot[f] = fma(static_cast<double>(o[f][e]), dV, tot[f]);
            }
          }
        }
      }
    }

    // this tile's warp reductions into the warp's running slots
    if (ctl.mode == 0) {
      if constexpr (sizeof(real) == 4) {
        // the speed maxima are +0 .. +inf (fmax drops NaNs), whose bit patterns order as unsigned integers:
        // one warp reduction instruction each
        amx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(amx)));
        amy = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(amy)));
        smx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(smx)));
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          amx = fmax(amx, __shfl_xor_sync(0xffffffffu, amx, o));
          amy = fmax(amy, __shfl_xor_sync(0xffffffffu, amy, o));
          smx = fmax(smx, __shfl_xor_sync(0xffffffffu, smx, o));
        }
      }
      const bool want_tot = g.totals != nullptr;
      if (want_tot) {
        if constexpr (sizeof(real) == 4) {
#pragma unroll
          for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) totr[f] += __shfl_xor_sync(0xffffffffu, totr[f], o);
        } else {
#pragma unroll
          for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot[f] += __shfl_xor_sync(0xffffffffu, tot[f], o);
        }
      }
      if (lane == 0) {
        real* r = red + warp * TL::RED_STRIDE;
        r[0] = fmax(r[0], amx);
        r[1] = fmax(r[1], amy);
        r[2] = fmax(r[2], smx);
        if (want_tot) {
          if constexpr (sizeof(real) == 4) {
            for (int f = 0; f < NF; ++f) {  // Knuth's two-sum: r[3+f] + r[8+f] holds the running total
              const float a = r[3 + f], b = totr[f];
              const float sum = __fadd_rn(a, b);
              const float bb = __fsub_rn(sum, a);
              const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
              r[3 + f] = sum;
              r[8 + f] = __fadd_rn(r[8 + f], err);
            }
          } else {
            for (int f = 0; f < NF; ++f) r[3 + f] += tot[f];
          }
        }
      }
    }
    if constexpr (kUnSmem) {  // no barrier: the tensor store is issued after the next tile's primitives
      prev_store = tile_store;
      prev_map = g.tmap_out;
      prev_x = x0 + GX;
      prev_y = y0 + GY;
    } else {
      // the outputs in sD (generic-proxy writes) become visible to the tensor store: each writer fences,
      // then the barrier. The next copy overwrites the box that everyone has read: the barrier orders those
      // reads before the issuing thread's fence, which orders them before its copies.
      if (tile_store) fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) fence_proxy_async_smem();
      if (tile_store && tid == 0) {
        tma_store_3d(g.tmap_out, sD, x0 + GX, y0 + GY, 0);
        bulk_commit();
      }
    }
  }
  if constexpr (kUnSmem) {  // the last tile's tensor store, or (after a failed copy) the copies in flight
    if (prev_store) fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (s_abort) {
        mbar_wait_limit(&bar[2], un_parity ^ 1u, TILE_WAIT_POLLS, TILE_WAIT_NS);
      } else if (prev_store) {
        fence_proxy_async_smem();
        tma_store_3d(prev_map, sUn, prev_x, prev_y, 0);
        bulk_commit();
      }
    }
  }
  if (tid == 0) bulk_wait_all();  // the tensor stores are complete before the CTA exits
  if (cur_member >= 0) flush();
}

}  // namespace hydro
