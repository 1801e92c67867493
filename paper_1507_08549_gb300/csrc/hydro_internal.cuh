// hydro_internal.cuh -- parameter blocks and device helpers shared by the stage kernels and the host
// runtime of the WENO5 / Lax-Friedrichs / SSP-RK3 Euler solver (Leung, Chu & Lin 2015, Sec. 2.1-2.2).
//
// Padded device layout of a working state (one plane per field, `fstride` elements apart):
//   cell (i, j) of the nx x ny interior sits at element (j + GY) * pitch + (i + GX)
// with GX = 4 ghost columns on the left (three are used; the fourth keeps every interior row 16-byte
// aligned, so tile boxes start on 16-byte boundaries for the TMA tensor copies and 4-wide vector stores
// line up) and GY = 3 ghost rows.
// pitch and the row count cover whole tiles plus the halo, so tile halo boxes never leave the
// allocation; cells beyond the grid are dead and masked.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hydro {

constexpr int GX = 4;        // ghost columns left of cell 0 (3 used + 1 alignment)
constexpr int GY = 3;        // ghost rows below row 0
constexpr int TILE_X = 60;   // cells per tile in x: halo box 68 = 60 + 8 wide (16-byte multiple)
constexpr int BOX_W = 68;    // smem row pitch; 68 = 4 (mod 32) makes the x-pass lanes conflict-free
constexpr int RUN = 15;      // cells per line work item, in x and in y (4 items per tile row)

enum Bc { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECT = 2, BC_AXIS = 3 };
// ERR_LAYOUT: a launch found its shared-memory buffers off the alignment the TMA copies need and did
// nothing (an internal error; no copy was issued)
enum ErrBits { ERR_NONPHYSICAL = 1, ERR_TIMEOUT = 2, ERR_LAYOUT = 4 };

// Tile variants: tile height TY (a multiple of the 15-cell run) and threads per CTA. Per field the
// x pass has 4 runs per row (rows padded to 8-row lane groups) and the y pass one run per 15 rows and
// column (columns padded to 64); 320 threads give about one item per thread for TY = 15.
struct Variant {
  int ty, threads;
};
constexpr int NUM_VARIANTS = 3;
constexpr int MAX_TY = 30;
constexpr Variant VARIANTS[NUM_VARIANTS] = {{15, 160}, {15, 320}, {30, 640}};

// Per-grid parameters of one stage launch (one ensemble member).
template <typename real>
struct GridParams {
  const real* win;   // stage input W (padded)
  const void* tmap_win;  // device CUtensorMap of win: (x, y, field) with one tile's halo box as its box
  const real* un;    // U^n (padded), read when rk_a != 0
  const void* tmap_un;   // device CUtensorMap of un's tile interiors (box 60 x TY x nfields)
  const void* tmap_out;  // device CUtensorMap of out's tile interiors (the tensor store of a whole tile)
  int tmap_ty;           // the tile height the tensor maps' boxes were built for
  const void* tmap_char; // device CUtensorMap of win with the characteristic kernel's box, else null
  const real* ux0;   // further stage states the blend adds (five-stage scheme), else null
  const real* ux1;
  const void* tmap_ux0;  // their tile-interior tensor maps (L2 prefetches), else null
  const void* tmap_ux1;
  real* out;         // stage output (padded) or L (mode RHS)
  long long fstride; // elements between field planes
  int nx, ny, pitch;
  int tiles_x, tiles_y;
  int bc[4];
  int geometry;
  real gamma, gm1, gravity, flame_speed;
  real rdx, rdy;       // 1/dx, 1/dy
  double dx, dy, x0;   // FP64 copies for geometry and totals
  real dx_r, x0_r;     // dx and x0 in the state precision (FP32 radii)
  double cfl_delta;    // c_cfl * min(dx, dy)
  // reduction slots (device)
  const real* alpha_in;   // (alpha_x, alpha_y) used by this stage
  real* alpha_out;        // max(|u|+c), max(|v|+c) of the output (next stage), may be null
  real* alpha_zero;       // slot to reset for the stage after next, may be null
  real* smax;             // CFL signal speed slot (read at stage 0, reset at 1, written at 2)
  double* dt_cur;         // dt of the running step (written at stage 0)
  const double* dt_src;   // frozen dt for this step (stage 0 of a frozen run), else null
  double* t_acc;          // FP64 time accumulator
  double* dt_log;         // recording: dt per step (null when not recording)
  double* alpha_log;      // recording: (alpha_x, alpha_y) per stage, 6 per step
  int* log_count;         // recording: steps logged so far (advanced by the last stage)
  int log_cap;            // recording: capacity in steps
  double* totals;         // 5 FP64 totals of the output (last stage), may be null
  double* totals_reset;   // totals array to clear (stage 1), may be null
  int* err;               // error bits
  const real* ext_div;    // characteristic scheme: D = dF/dx + dG/dy of the hydro fields (padded), else null
};

// Launch-wide stage control.
struct StageCtl {
  int stage;      // 0 .. stages-1
  int mode;       // 0 RK stage, 1 write L (no blending, no reductions), 2 field split: work item w computes
                  // dF/dx + dG/dy of hydro field w & 3 on tile w >> 2 into ext_div (FP64 grids with few tiles)
  double rk_a;    // out = a U^n + x0 ux0 + x1 ux1 + b (W + c dt L)
  double rk_b;
  int w0 = 0;     // first tile of the launch (row bands of one stage); work items w -> tile w0 + w
  double rk_c = 1.0;
  double rk_x0 = 0.0;
  double rk_x1 = 0.0;
  int last = 0;   // the step's last stage (writes the next step's CFL speed and the totals)
};

// Batched launch: a table of (member, tile) work items over an array of member parameters.
struct WorkItem {
  int member;
  int tile;
};

// Host-side launch entry points (one translation unit per precision). members_dev points to device
// GridParams (one per member; work_dev maps work item -> (member, tile), or is null for one grid whose
// tiles are the work items).
template <typename real>
cudaError_t launch_stage(int variant, int nfields, const GridParams<real>* members_dev, const WorkItem* work_dev,
                         int nwork, const StageCtl& ctl, int grid, cudaStream_t s);
template <typename real>
int stage_smem_bytes(int variant, int nfields);
template <typename real>
int stage_ctas_per_sm(int variant, int nfields);

// Copy an unpadded caller state into a padded working state, write its ghost images, and reduce its
// Lax-Friedrichs speeds and CFL signal speed into the given slots; sets *t_acc = t0 when t_acc != null.
template <typename real>
cudaError_t launch_pack(const real* U, const GridParams<real>& g, int nfields, real* alpha_slot, real* smax_slot,
                        double* t_acc, double t0, cudaStream_t s);
// Batched ensembles, one launch each over n members: pack every caller state U[m] with its first-stage
// parameters P[m] (into buffer A, reductions into its slots, *t_acc = t0[m]); unpack buffer A into U[m];
// zero (dst == null) or gather into dst the first `bytes` of every member's scratch record.
template <typename real>
cudaError_t launch_batch_pack(const GridParams<real>* P, const real* const* U, const double* t0, int n, int nfields,
                              long long max_cells, cudaStream_t s);
template <typename real>
cudaError_t launch_batch_unpack(const GridParams<real>* P, real* const* U, int n, int nfields, long long max_cells,
                                cudaStream_t s);
cudaError_t launch_batch_scratch(void* const* scratch, int n, int bytes, unsigned char* dst, cudaStream_t s);
// Copy every field's interior between a padded state and an unpadded [nf][ny][nx] one (one launch).
template <typename real>
cudaError_t launch_copy_state(real* dst, const real* src, int nx, int ny, int nf, int pitch, long long fstride,
                              bool to_padded, cudaStream_t s);
// Write frozen dt and stage alphas into device slots (frozen runs, adjoint).
template <typename real>
cudaError_t launch_set_frozen(double* dt_slot, double dt, real* alpha_slots, const double* alpha6, cudaStream_t s);
// FP64 conserved totals of an unpadded state: per-block partials, then a fixed-order final sum.
template <typename real>
cudaError_t launch_totals(const real* U, int nx, int ny, int nfields, int geometry, double x0, double dx,
                          double dy, double* partials, int nblocks, double* out, cudaStream_t s);

// Level-set reinitialisation (reinit_kernel.cuh): front points where phi changes sign between
// neighbouring cells (linear interpolation), minimum distance of every cell to them, tanh blend.
// Measured FMA throughput (FMAs per second) of the current device in precision real.
template <typename real>
cudaError_t run_fma_probe(int iters, cudaStream_t st, int num_sms, double* fma_per_s);

// One bounded device wait that nothing completes (polls polls), reporting ERR_TIMEOUT into *err.
cudaError_t launch_wait_selftest(unsigned polls, int* err, cudaStream_t s);

// Characteristic-wise flux divergence of p_dev->win into p_dev->ext_div (one launch per stage).
template <typename real>
cudaError_t launch_char_div(const GridParams<real>* p_dev, int nx, int ny, cudaStream_t s);

template <typename real>
cudaError_t launch_reinit(real* phi, int nx, int ny, int pitch, double x0, double y0, double dx, double dy,
                          real* front, int capacity, int* count, int* err, cudaStream_t s, int* launches);

// Discrete adjoint of one frozen RK stage (adjoint_kernel.cuh): point terms, line adjoints over the
// padded grid with its ghost frame, ghost fold and RK blend. Buffers are padded like the states.
template <typename real>
struct AdjParams;
template <typename real>
cudaError_t launch_adjoint_stage(const AdjParams<real>& P, int nfields, cudaStream_t s, int* launches);

// ------------------------------------------------------------------------------ device helpers

#ifdef __CUDACC__

// Source index and normal-momentum flip of ghost layer k (0 nearest) of a face of a line of n cells.
__host__ __device__ inline int ghost_src(int bc, bool hi, int k, int n, bool* flip) {
  *flip = false;
  if (bc == BC_PERIODIC) return hi ? k : n - 1 - k;
  if (bc == BC_TRANSMISSIVE) return hi ? n - 1 : 0;
  *flip = true;  // reflecting wall or axis: mirror image
  return hi ? n - 1 - k : k;
}

#endif

// ---- exact (correctly rounded) summation and the self-gravity Poisson solve (Sec. 2.1)

// limb k holds digits of weight 2^(32 k - XS_BIAS); a finite double's bits lie in [2^-1074, 2^1024),
// i.e. bit positions 14 .. 2111 above 2^-1088, limbs 0 .. 65; two more limbs absorb carries.
constexpr int XS_LIMBS = 68;
constexpr int XS_BIAS = 1088;
// every add puts less than 2^32 into a limb: at most 2^31 - 1 terms keep each 64-bit limb from overflowing
constexpr long long XS_MAX_TERMS = 0x7fffffffLL;

struct ExactAcc {
  unsigned long long limb[XS_LIMBS];  // two's complement digit sums
  int nonfinite;                      // a term was inf or NaN
};

struct PoissonParams {
  double* phi;        // [ny][nx], in/out
  const void* rho;    // density plane of the caller's state, [ny][nx] of the state dtype
  int nx, ny, zsym, max_iters;
  double x0, y0, dr, dz, G;
  double omega, one_minus_omega, tol;
  int tol_screen, tol_exp;  // tol normal and finite: its unbiased exponent Et (tol in [2^Et, 2^(Et+1)))
  float tol_mant;           // tol / 2^Et in [1, 2), rounded to FP32
  double four_pi_G;      // RN(RN(4 pi) G)
  double aN;             // set by poisson_setup_kernel
  double mass;           // grid mass (not doubled), set by poisson_setup_kernel
  double* cE;            // [nx] aE
  double* cW;            // [nx] aW
  double* cD;            // [nx] D = aE + aW + aN + aS
  double* cY;            // [nx] RN(1 / D)
  double* src;           // [ny][nx] RN(4 pi G rho), set by poisson_mass_kernel
  double* gE;            // [ny] Roche value of the ghost east of column nx - 1
  double* gN;            // [nx] Roche value of the ghost north of row ny - 1
  double* gS;            // [nx] Roche value of the ghost south of row 0 (unused with zsym)
};

struct SorCtl {
  int base;     // sweeps of the chunks already launched
  int done;     // convergence seen
  int iters;    // sweeps done when `done` was set
  int flag[3];  // flag[s % 3]: some cell of sweep s changed by tol or more
};

constexpr int SOR_CHUNK = 64;  // sweeps per captured graph
constexpr int SOR_BX = 128, SOR_BY = 2;

cudaError_t launch_exact_sum(const double* x, long long n, ExactAcc* acc, double* out, cudaStream_t s, int* launches);
template <typename T>
cudaError_t launch_poisson_setup(PoissonParams* P_dev, ExactAcc* acc, long long n, int nx, int ny, cudaStream_t s,
                                 int* launches);
cudaError_t launch_sor_chunk(const PoissonParams* P_dev, SorCtl* ctl, int nx, int ny, cudaStream_t s, int* launches);

}  // namespace hydro
