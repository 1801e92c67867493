// poisson_kernel.cuh -- self-gravity potential (Leung, Chu & Lin 2015, Sec. 2.1), FP64.
//
// The potential solves (1/r) d/dr (r dPhi/dr) + d2Phi/dz2 = 4 pi G rho on the cell centres of an (r,z)
// grid by successive over-relaxation of red-black Gauss-Seidel sweeps. Per cell
//   Phi_GS = (aE Phi_E + aW Phi_W + aN Phi_N + aS Phi_S - 4 pi G rho) / (aE + aW + aN + aS),
//   aE = r_{i+1/2} / (r_i dr^2), aW = r_{i-1/2} / (r_i dr^2), aN = aS = 1 / dz^2,
//   Phi <- (1 - omega) Phi + omega Phi_GS,
// first on the red cells (i + j even), then on the black ones. A red update reads only black
// neighbours and the reverse, so one colour is a data-parallel pass and the sweep equals the
// lexicographic red-then-black order exactly. Inner boundaries reflect (the axis through aW = 0 at
// r = 0, the plane z = 0 by taking the cell's own value for the missing neighbour); outer ghost cells hold
// the Roche value -G M / sqrt(r^2 + z^2), M the mass (doubled for a z = 0 symmetry plane).
//
// Every operation is rounded once in the order written above (explicit _rn intrinsics, no contraction),
// so a sweep is bitwise reproducible against any IEEE FP64 evaluation in that order. The GPU's FP64 pipe
// (2 operations per SM per clock) bounds the sweep, so the kernel spends as few FP64 operations as
// that allows: 4 pi G rho is formed once per solve (one rounding, as in the definition); the division
// by the diagonal D is Markstein's correctly rounded quotient from the column's reciprocal y = RN(1/D)
// (q0 = RN(a y), r0 = RN(a - D q0), q1 = RN(q0 + r0 y) faithful, r1 = a - D q1 exact, q = RN(q1 + r1 y)
// = RN(a / D); P. Markstein, IBM J. Res. Dev. 34 (1990)), five fused operations in place of a full
// division; and the stopping test (every cell's relative change |Phi_new - Phi_old| / |Phi_new| below
// tol) compares exponents with integer operations, dividing only where the ratio is within a factor of
// four of tol, which takes the same decision as the rounded quotient.
//
// Convergence runs on the device: a sweep's kernels set flag[s % 3] when any cell did not converge; the
// red kernel of sweep s + 1 reads flag[s % 3] and, when it is clear, marks the solve done and every later
// kernel returns at once. The host replays a captured graph of SOR_CHUNK sweeps and reads the done flag
// between chunks, one chunk behind, so a solve needs no per-sweep synchronisation.
//
// The mass M = sum of rho 2 pi r dr dz is rounded once (correctly rounded sum): the terms are added
// exactly into a fixed-point accumulator of 32-bit digits held in 64-bit limbs (the long-accumulator
// idea of Kulisch, in the parallel carry-save form of Collange, Defour, Graillat and Iakymchuk 2015),
// and the final value is rounded to nearest-even once. The sum therefore does not depend on the order
// of the additions, i.e. on the launch configuration or the atomics' order.
#pragma once
#include "hydro_internal.cuh"

namespace hydro {

// ------------------------------------------------------------------------------ exact summation

// Adds x exactly to the limbs `acc` (shared or global memory) with atomics.
__device__ __forceinline__ void xs_add(unsigned long long* acc, int* nonfinite, double x) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ex = static_cast<int>((bits >> 52) & 0x7ff);
  if (ex == 0x7ff) {
    atomicOr(nonfinite, 1);
    return;
  }
  unsigned long long m = bits & ((1ull << 52) - 1);
  if (ex != 0) m |= 1ull << 52;
  if (m == 0) return;
  const int p = (ex == 0 ? -1074 : ex - 1075) + XS_BIAS;  // bit position of m's lowest bit, >= 14
  const int k = p >> 5, sh = p & 31;
  const unsigned __int128 w = static_cast<unsigned __int128>(m) << sh;  // < 2^84: three digits
  unsigned long long d0 = static_cast<unsigned long long>(w) & 0xffffffffull;
  unsigned long long d1 = static_cast<unsigned long long>(w >> 32) & 0xffffffffull;
  unsigned long long d2 = static_cast<unsigned long long>(w >> 64);
  if (bits >> 63) {
    d0 = 0ull - d0;
    d1 = 0ull - d1;
    d2 = 0ull - d2;
  }
  if (d0) atomicAdd(acc + k, d0);
  if (d1) atomicAdd(acc + k + 1, d1);
  if (d2) atomicAdd(acc + k + 2, d2);
}

// Block-level accumulation: threads add into shared limbs, then one atomic per limb to global.
__device__ __forceinline__ void xs_block_begin(unsigned long long* s) {
  for (int k = threadIdx.x; k < XS_LIMBS; k += blockDim.x) s[k] = 0ull;
  __syncthreads();
}

__device__ __forceinline__ void xs_block_end(const unsigned long long* s, ExactAcc* g) {
  __syncthreads();
  for (int k = threadIdx.x; k < XS_LIMBS; k += blockDim.x)
    if (s[k]) atomicAdd(&g->limb[k], s[k]);
}

// Correctly rounded (to nearest, ties to even) value of the accumulator; one thread.
__device__ inline double xs_round(const ExactAcc* a) {
  if (a->nonfinite) return __longlong_as_double(0x7ff8000000000000LL);
  // carry propagation to digits in [0, 2^32); the final carry is the sign (0 or -1)
  unsigned int dig[XS_LIMBS];
  __int128 carry = 0;
  for (int k = 0; k < XS_LIMBS; ++k) {
    const __int128 v = static_cast<__int128>(static_cast<long long>(a->limb[k])) + carry;
    dig[k] = static_cast<unsigned int>(static_cast<unsigned long long>(v) & 0xffffffffull);
    carry = v >> 32;  // arithmetic shift: floor division
  }
  const bool negative = carry < 0;
  if (negative) {  // magnitude = two's complement of the digit string
    unsigned long long c = 1;
    for (int k = 0; k < XS_LIMBS; ++k) {
      const unsigned long long v = static_cast<unsigned long long>(~dig[k]) + c;
      dig[k] = static_cast<unsigned int>(v);
      c = v >> 32;
    }
  }
  int t = XS_LIMBS - 1;
  while (t >= 0 && dig[t] == 0) --t;
  if (t < 0) return 0.0;
  // 96-bit window of the top three digits, sticky bit for everything below
  const unsigned __int128 W = (static_cast<unsigned __int128>(dig[t]) << 64) |
                              (static_cast<unsigned __int128>(t >= 1 ? dig[t - 1] : 0u) << 32) |
                              static_cast<unsigned __int128>(t >= 2 ? dig[t - 2] : 0u);
  bool sticky = false;
  for (int k = 0; k < t - 2; ++k) sticky |= dig[k] != 0;
  const int B = 32 * (t - 2) - XS_BIAS;                 // weight exponent of W's lowest bit
  const int L = 64 + (31 - __clz(static_cast<int>(dig[t])));  // W's leading bit, 64 .. 95
  const int E = B + L;                                  // value in [2^E, 2^(E+1))
  const int u = E - 52 > -1074 ? E - 52 : -1074;        // exponent of the result's last place
  const int sh = u - B;                                 // 12 .. 78 bits drop off W
  unsigned long long q = static_cast<unsigned long long>(W >> sh);
  const unsigned __int128 rem = W & ((static_cast<unsigned __int128>(1) << sh) - 1);
  const unsigned __int128 half = static_cast<unsigned __int128>(1) << (sh - 1);
  if (rem > half || (rem == half && (sticky || (q & 1)))) ++q;
  // q * 2^u with q <= 2^53: exponent field and mantissa add up in one integer (subnormals included);
  // u > 971 or a carry into exponent 2047 rounds beyond the largest double
  unsigned long long r = u > 971 ? 0x7ff0000000000000ull : (static_cast<unsigned long long>(u + 1074) << 52) + q;
  if (r > 0x7ff0000000000000ull) r = 0x7ff0000000000000ull;
  if (negative) r |= 1ull << 63;
  return __longlong_as_double(static_cast<long long>(r));
}

// sum of n device doubles
__global__ void __launch_bounds__(256) xs_array_kernel(const double* __restrict__ x, long long n, ExactAcc* acc) {
  __shared__ unsigned long long s[XS_LIMBS];
  xs_block_begin(s);
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<long long>(gridDim.x) * blockDim.x)
    xs_add(s, &acc->nonfinite, x[k]);
  xs_block_end(s, acc);
}

__global__ void xs_round_kernel(const ExactAcc* acc, double* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *out = xs_round(acc);
}

// ------------------------------------------------------------------------------ Poisson SOR

__device__ __forceinline__ double cell_r(const PoissonParams& P, double i_plus) {
  return __dadd_rn(P.x0, __dmul_rn(i_plus, P.dr));
}

__device__ __forceinline__ double roche(double G, double M, double r, double z) {
  return __ddiv_rn(__dmul_rn(-G, M), __dsqrt_rn(__dadd_rn(__dmul_rn(r, r), __dmul_rn(z, z))));
}

// mass terms rho 2 pi r dr dz, each rounded in that order, summed exactly
template <typename T>
__global__ void __launch_bounds__(256) poisson_mass_kernel(const PoissonParams* __restrict__ Pp, ExactAcc* acc) {
  __shared__ unsigned long long s[XS_LIMBS];
  const PoissonParams P = *Pp;
  xs_block_begin(s);
  const T* rho = static_cast<const T*>(P.rho);
  const long long n = static_cast<long long>(P.nx) * P.ny;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(k % P.nx);
    const double r = cell_r(P, i + 0.5);
    const double rk = static_cast<double>(rho[k]);
    const double term = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(rk, two_pi), r), P.dr), P.dz);
    xs_add(s, &acc->nonfinite, term);
    P.src[k] = __dmul_rn(P.four_pi_G, rk);
  }
  xs_block_end(s, acc);
}

// rounds the mass, then the per-column coefficients and the Roche ghost values
__global__ void __launch_bounds__(256) poisson_setup_kernel(PoissonParams* Pp, const ExactAcc* acc) {
  __shared__ double Ms;
  if (threadIdx.x == 0) {
    const double m = xs_round(acc);
    Ms = m;
    if (blockIdx.x == 0) {
      Pp->mass = m;
      Pp->aN = __ddiv_rn(1.0, __dmul_rn(Pp->dz, Pp->dz));
    }
  }
  __syncthreads();
  const PoissonParams P = *Pp;
  const double M = P.zsym ? __dmul_rn(2.0, Ms) : Ms;
  const double aN = __ddiv_rn(1.0, __dmul_rn(P.dz, P.dz));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.nx; i += gridDim.x * blockDim.x) {
    const double r = cell_r(P, i + 0.5), rp = cell_r(P, i + 1.0), rm = cell_r(P, static_cast<double>(i));
    const double den = __dmul_rn(__dmul_rn(r, P.dr), P.dr);
    const double aE = __ddiv_rn(rp, den), aW = __ddiv_rn(rm, den);
    P.cE[i] = aE;
    P.cW[i] = aW;
    const double D = __dadd_rn(__dadd_rn(__dadd_rn(aE, aW), aN), aN);
    P.cD[i] = D;
    P.cY[i] = __drcp_rn(D);
    const double ztop = __dadd_rn(P.y0, __dmul_rn(P.ny - 1 + 0.5, P.dz));
    const double zbot = __dadd_rn(P.y0, __dmul_rn(0.5, P.dz));
    P.gN[i] = roche(P.G, M, r, __dadd_rn(ztop, P.dz));
    P.gS[i] = roche(P.G, M, r, __dsub_rn(zbot, P.dz));
  }
  const double rlast = __dadd_rn(cell_r(P, P.nx - 1 + 1.0), __dmul_rn(0.5, P.dr));
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.ny; j += gridDim.x * blockDim.x)
    P.gE[j] = roche(P.G, M, rlast, __dadd_rn(P.y0, __dmul_rn(j + 0.5, P.dz)));
}

// One colour of one sweep. s_rel is the sweep's index within the chunk; the sweep is base + s_rel.
__global__ void __launch_bounds__(SOR_BX* SOR_BY) sor_color_kernel(const PoissonParams* __restrict__ Pp,
                                                                   SorCtl* ctl, int color, int s_rel) {
  const int s = ctl->base + s_rel;
  const int max_iters = Pp->max_iters;
  const double tol = Pp->tol;
  if (s >= max_iters || ctl->done) return;
  const bool first = blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0;
  if (tol > 0.0 && s > 0 && ctl->flag[(s + 2) % 3] == 0) {  // sweep s - 1 converged
    if (first) {
      ctl->done = 1;
      ctl->iters = s;
    }
    return;
  }
  if (color == 0 && first) ctl->flag[(s + 1) % 3] = 0;
  // (the exit above is uniform over the grid: nothing it reads changes while this kernel runs)
  const int nx = Pp->nx, ny = Pp->ny;
  const int j = blockIdx.y * SOR_BY + threadIdx.y;
  const int i = 2 * (blockIdx.x * SOR_BX + threadIdx.x) + ((j + color) & 1);
  bool unconv = false;
  if (j < ny && i < nx) {
    double* __restrict__ phi = Pp->phi;
    const long long g = static_cast<long long>(j) * nx + i;
    const double aN = Pp->aN;
    const double old = phi[g];
    const double pE = i + 1 < nx ? phi[g + 1] : Pp->gE[j];
    const double pW = i > 0 ? phi[g - 1] : old;  // aW = 0 on the axis; a reflecting inner face elsewhere
    const double pN = j + 1 < ny ? phi[g + nx] : Pp->gN[i];
    const double pS = j > 0 ? phi[g - nx] : (Pp->zsym ? old : Pp->gS[i]);
    double a = __dadd_rn(__dmul_rn(Pp->cE[i], pE), __dmul_rn(Pp->cW[i], pW));
    a = __dadd_rn(a, __dmul_rn(aN, pN));
    a = __dadd_rn(a, __dmul_rn(aN, pS));
    a = __dsub_rn(a, Pp->src[g]);
    // Markstein's correctly rounded a / D from y = RN(1/D)
    const double D = Pp->cD[i], y = Pp->cY[i];
    const double q0 = __dmul_rn(a, y);
    const double q1 = __fma_rn(__fma_rn(-q0, D, a), y, q0);
    const double gs = __fma_rn(__fma_rn(-q1, D, a), y, q1);
    const double nw = __dadd_rn(__dmul_rn(Pp->one_minus_omega, old), __dmul_rn(Pp->omega, gs));
    phi[g] = nw;
    if (tol > 0.0) {
      // decision fl(|d| / |nw|) >= tol (NaN: no). For normal d and nw with biased exponents ed, en and
      // mantissas Md, Mn in [1, 2), |d| / |nw| = (Md / Mn) 2^(ed - en) and tol = Mt 2^Et: with k = ed - en - Et
      // the ratio over tol is (Md / (Mn Mt)) 2^k. k <= -2 puts it below 1/2, k >= 2 at or above 2. Otherwise
      // an estimate from the leading 20 mantissa bits of d and nw (FP32 arithmetic, relative error below
      // 2^-18) decides unless it lies within 2^-14 of 1; only those cells divide. A ratio that clears 1 by
      // more than half an ulp rounds to the same side of tol, so every branch takes fl's decision.
      const double d = __dsub_rn(nw, old);
      const int hd = __double2hiint(d), hn = __double2hiint(nw);
      const int ed = (hd >> 20) & 0x7ff, en = (hn >> 20) & 0x7ff;
      if (d == 0.0) {
        unconv = false;  // 0 / |nw| = 0 < tol, or 0 / 0
      } else if (Pp->tol_screen && ed != 0 && ed != 0x7ff && en != 0 && en != 0x7ff) {
        const int k = ed - en - Pp->tol_exp;
        if (k >= 2) {
          unconv = true;
        } else if (k > -2) {
          const float fd = __int_as_float(0x3f800000 | ((hd & 0xfffff) << 3));
          const float fn = __int_as_float(0x3f800000 | ((hn & 0xfffff) << 3));
          const float est = __fdividef(fd, fn * Pp->tol_mant) * (k == 0 ? 1.0f : (k > 0 ? 2.0f : 0.5f));
          if (est >= 1.0f + 0x1p-14f)
            unconv = true;
          else if (est > 1.0f - 0x1p-14f)
            unconv = __ddiv_rn(fabs(d), fabs(nw)) >= tol;
        }
      } else {
        unconv = __ddiv_rn(fabs(d), fabs(nw)) >= tol;
      }
    }
  }
  if (__syncthreads_or(unconv) && threadIdx.x == 0 && threadIdx.y == 0) {
    int* f = &ctl->flag[s % 3];
    if (*reinterpret_cast<volatile int*>(f) == 0) *f = 1;
  }
}

__global__ void sor_advance_kernel(SorCtl* ctl, int n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->base += n;
}

}  // namespace hydro
