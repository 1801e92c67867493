// capi.cu -- host runtime behind the C ABI of include/hydro.h: contexts, the padded working states,
// the SSP-RK3 step loop (Leung, Chu & Lin 2015, Sec. 2.1) with CFL time steps (Sec. 5.4), CUDA-graph
// replay of a step's three stage launches, batched ensembles, the tile autotuner, totals, recording
// and the bounded host waits. All device work is issued on the context's stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>  // cuTensorMapEncodeTiled signature, CUtensorMap

#include "../../include/hydro.h"
#include "hydro_internal.cuh"
#include "adjoint_kernel.cuh"
#include "char_kernel.cuh"

using namespace hydro;

namespace {

template <typename real>
struct Scratch {
  real alpha[5][2];         // ring of (alpha_x, alpha_y) slots, one per stage of a step: stage k reads k,
                            // writes k+1, clears k+2 (mod the stage count)
  real smax;                // CFL signal speed of U^n
  real frozen_alpha[3][2];  // frozen runs
  real pad;
  double dt_cur, t_acc, frozen_dt;
  double totals[5];
  int err;
  int log_count;  // kept across calls while recording (not cleared with the rest)
};

double host_timeout_s() {
  const char* e = std::getenv("HYDRO_TIMEOUT_S");
  double v = e ? std::atof(e) : 0.0;
  return v > 0.0 ? v : 3600.0;
}

}  // namespace

struct hydro_ctx {
  hydro_config cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;  // private stream used only to capture graphs
  // host-buffer calls: the last stage runs in row bands; a copy stream moves each finished band's rows
  // to the caller's pinned state while the next band computes
  static constexpr int NBANDS = 8;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t band_ev[NBANDS] = {};
  cudaEvent_t copy_done = nullptr;
  int device = 0, num_sms = 0;
  int nf = 4;
  size_t esize = 4;
  int variant = 1;
  int uploaded_variant = -1;  // the variant the device parameters and tensor maps were built for
  // padded layout (sized for the tallest tile variant so every variant fits)
  int pitch = 0, rows = 0, tiles_x = 0, tiles_y = 0;
  long long fstride = 0;
  int ns = 3;  // stages per step: 3 (SSP-RK3) or 5 (the five-stage third-order scheme)
  // A = U^n / U^{n+1}, B = U^(1), C = U^(2) (and D = U^(3), E = U^(4) of the five-stage scheme)
  void* buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // device CUtensorMap[NTMAPS]: the working states' halo boxes for the current tile variant (0 .. ns-1)
  // and, from TMAP_INTERIOR on, the same states' tile interiors (U^n for the blend, the tensor stores)
  void* tmaps = nullptr;
  void* scratch = nullptr;
  void* params = nullptr;  // device GridParams[NPARAMS]: stages 0..ns-1, frozen stages P_FROZEN.., rhs P_RHS
  void* host_scratch = nullptr;  // pinned copy of Scratch
  double* partials = nullptr;
  int partial_blocks = 0;
  double* d_totals = nullptr;
  void* unpadded = nullptr;  // caller-layout device buffer (host entry, rhs output)
  // recording
  double* dt_log = nullptr;
  double* alpha_log = nullptr;
  int log_cap = 0;
  bool track_totals = true;
  // inside an adjoint sweep: the device error word accumulates over all its steps and is read once at
  // the end, so the sweep's steps need no host round trip
  bool defer_status = false;
  // graph of one step
  cudaGraphExec_t step_graph = nullptr;
  long long step_graph_launches = 0;
  // per-launch profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  cudaEvent_t done = nullptr;
  long long launches = 0;
  // adjoint: padded work buffers (nu ping-pong, mu, hb, accumulator), checkpoints, segment states
  void* adj_nu[2] = {nullptr, nullptr};
  void* adj_mu = nullptr;
  void* adj_hb = nullptr;
  int adj_in = 0;  // during a reverse sweep: 0 (adj_nu[0]) or 2 (adj_acc), the buffer holding the cotangent
  int adj_rows = 0;  // line-adjoint tile rows (hydro_set_adjoint_tile_rows), 0 for the size rule
  void* adj_acc = nullptr;
  void* ckpt = nullptr;
  size_t ckpt_cap = 0;
  void* seg = nullptr;
  size_t seg_cap = 0;
  int ck_nsteps = -1, ck_every = 0;
  // binomial (revolve) schedule: ck_mode 1 keeps only U^0 (slot 0 of rv_slots) and reverses with
  // rv_snapshots further state slots plus one recomputation buffer
  int ck_mode = 0;
  int rv_snapshots = 0;
  void* rv_slots = nullptr;
  size_t rv_cap = 0;
  // characteristic scheme: padded D = dF/dx + dG/dy of the 4 hydro fields, written per stage
  void* char_div = nullptr;
  // FP64 grids with fewer tiles than half the SMs: the same D, written per stage by a field-split launch
  // of the stage kernel (4 CTAs per tile) so that more SMs share the FP64 line work
  void* split_div = nullptr;
  // level-set reinitialisation: front points (x, y pairs) and their count
  void* front = nullptr;
  int* front_count = nullptr;
  int front_cap = 0;
  // self-gravity Poisson solve and exact sums: device PoissonDev block + coefficient arrays, pinned
  // host mirror of the control words, the captured graph of one chunk of sweeps
  void* pois = nullptr;
  void* pois_host = nullptr;
  cudaGraphExec_t sor_graph = nullptr;
  cudaEvent_t sor_ev[2] = {nullptr, nullptr};
  // identity of this context for batch plans: unique per process, never reused (a destroyed context's
  // address can come back from the allocator with other buffers behind it)
  unsigned long long uid = 0;
  // bumped whenever the device parameters are rebuilt (log buffers, tile variant ...): a batch plan holds
  // copies of its members' parameters and is valid only for the generations it was built from
  unsigned long long params_gen = 0;
  // batch plan (kept on the first member), keyed by the members' (uid, params_gen)
  std::vector<unsigned long long> plan_members;
  std::vector<unsigned long long> plan_gens;
  int plan_variant = -1;
  int plan_waves = 0, plan_layout = -1;  // the plan's grid size (CTA waves) and work-list layout
  int plan_grid = 0;
  void* plan_params = nullptr;  // device GridParams[3][nmembers]
  void* plan_work = nullptr;    // device WorkItem[nwork]
  int plan_nwork = 0;
  cudaGraphExec_t plan_graph = nullptr;
  // a batch call's per-member arguments (caller state and scratch pointers, start times) and the gathered
  // scratch records, on the device and in pinned host memory, for up to bio_cap members
  void* bio_dev = nullptr;
  void* bio_host = nullptr;
  int bio_cap = 0;
  // batch plan shape chosen by hydro_batch_autotune (on the first member): persistent CTAs in
  // batch_waves waves of (CTAs per SM x SMs), work-list layout (BatchLayout)
  int batch_waves = 1, batch_layout = 0;
  std::string err;
};

// ------------------------------------------------------------------------------------ helpers

static int fail(hydro_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static int cuda_fail(hydro_ctx* c, cudaError_t e, const char* what) {
  return fail(c, HYDRO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

static int validate_config(const hydro_config* g, std::string* why) {
  if (!g) { *why = "null config"; return HYDRO_EINVAL; }
  if (g->nx < 3 || g->ny < 3) { *why = "nx and ny must be >= 3"; return HYDRO_EINVAL; }
  if (g->nfields != 4 && g->nfields != 5) { *why = "nfields must be 4 or 5"; return HYDRO_EINVAL; }
  if (g->dtype != HYDRO_F32 && g->dtype != HYDRO_F64) { *why = "dtype must be HYDRO_F32 or HYDRO_F64"; return HYDRO_EINVAL; }
  if (!(g->x1 > g->x0) || !(g->y1 > g->y0)) { *why = "empty domain"; return HYDRO_EINVAL; }
  if (!(g->gamma > 1.0) || !(g->cfl > 0.0)) { *why = "gamma must be > 1 and cfl > 0"; return HYDRO_EINVAL; }
  if (g->geometry != 0 && g->geometry != 1) { *why = "geometry must be 0 or 1"; return HYDRO_EINVAL; }
  for (int k = 0; k < 4; ++k)
    if (g->bc[k] < HYDRO_BC_PERIODIC || g->bc[k] > HYDRO_BC_AXIS) { *why = "unknown boundary kind"; return HYDRO_EINVAL; }
  if ((g->bc[0] == HYDRO_BC_PERIODIC) != (g->bc[1] == HYDRO_BC_PERIODIC) ||
      (g->bc[2] == HYDRO_BC_PERIODIC) != (g->bc[3] == HYDRO_BC_PERIODIC)) {
    *why = "periodic faces must come in pairs";
    return HYDRO_EINVAL;
  }
  if (g->bc[1] == HYDRO_BC_AXIS || g->bc[2] == HYDRO_BC_AXIS || g->bc[3] == HYDRO_BC_AXIS ||
      (g->bc[0] == HYDRO_BC_AXIS && (g->geometry != 1 || g->x0 != 0.0))) {
    *why = "the axis boundary is the x-lo (r = 0) face of an (r,z) grid";
    return HYDRO_EINVAL;
  }
  if (g->geometry == 1 && g->x0 < 0.0) { *why = "(r,z) grids need r >= 0"; return HYDRO_EINVAL; }
  if (g->scheme != HYDRO_SCHEME_COMPONENT && g->scheme != HYDRO_SCHEME_CHARACTERISTIC) {
    *why = "scheme must be HYDRO_SCHEME_COMPONENT or HYDRO_SCHEME_CHARACTERISTIC";
    return HYDRO_EINVAL;
  }
  if (g->rk_stages != 0 && g->rk_stages != 3 && g->rk_stages != 5) {
    *why = "rk_stages must be 3 (or 0) or 5";
    return HYDRO_EINVAL;
  }
  if (!std::isfinite(g->gravity_y) || !std::isfinite(g->flame_speed) || g->flame_speed < 0.0) {
    *why = "gravity and flame speed must be finite, flame speed >= 0";
    return HYDRO_EINVAL;
  }
  return HYDRO_OK;
}

template <typename real>
static Scratch<real>* scr(hydro_ctx* c) {
  return static_cast<Scratch<real>*>(c->scratch);
}

template <typename real>
static real* bufp(hydro_ctx* c, int k) {
  return static_cast<real*>(c->buf[k]);
}

static int tile_ty(int variant) { return VARIANTS[variant].ty; }

// Device parameter table of a context: the step's stages (up to 5), the three frozen SSP-RK3 stages
// (recorded replays and the adjoint), the spatial operator.
constexpr int P_FROZEN = 5, P_RHS = 8, NPARAMS = 9;
constexpr int TMAP_INTERIOR = 5, TMAP_CHAR = 10, NTMAPS = 15;

// One stage of a step: W = buffer win, output buffer out, and out = a U^n + rx0 B[x0] + rx1 B[x1]
// + b (W + c dt L(W)) (x0, x1 = -1: no such term).
struct RkStage {
  int win, out, x0, x1;
  double a, b, c, rx0, rx1;
};

// SSP-RK3 (Sec. 2.1, the original prescription): U1 = U + dt L(U), U2 = 3/4 U + 1/4 (U1 + dt L(U1)),
// U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2)).
static const RkStage RK3_STAGES[3] = {{0, 1, -1, -1, 0.0, 1.0, 1.0, 0.0, 0.0},
                                      {1, 2, -1, -1, 0.75, 0.25, 1.0, 0.0, 0.0},
                                      {2, 0, -1, -1, 1.0 / 3.0, 2.0 / 3.0, 1.0, 0.0, 0.0}};
static const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};
static const double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};

// The five-stage third-order scheme (Sec. 2.1), read as Spiteri & Ruuth's SSP(5,3): Shu-Osher form
// u(i) = sum_k SO_A[i-1][k] u(k) + dt sum_k SO_B[i-1][k] L(u(k)), u(0) = U^n, U^{n+1} = u(5), with the
// published coefficients. Each stage here applies L to its newest input only: the terms dt L(u0) and
// dt L(u1) of the later stages are (u1 - u0) / b10 and (u2 - u1) / b21 exactly (stages 1 and 2), so
// their weights move onto u0, u1, u2 (the moved weights are below 0.01, so the rounding this adds is
// negligible).
static const double SO_A[5][5] = {{1.0, 0.0, 0.0, 0.0, 0.0},
                                  {0.0, 1.0, 0.0, 0.0, 0.0},
                                  {0.56656131914033, 0.0, 0.43343868085967, 0.0, 0.0},
                                  {0.09299483444413, 0.00002090369620, 0.0, 0.90698426185967, 0.0},
                                  {0.00736132260920, 0.20127980325145, 0.00182955389682, 0.0, 0.78952932024253}};
static const double SO_B[5][5] = {{0.37726891511710, 0.0, 0.0, 0.0, 0.0},
                                  {0.0, 0.37726891511710, 0.0, 0.0, 0.0},
                                  {0.0, 0.0, 0.16352294089771, 0.0, 0.0},
                                  {0.00071997378654, 0.0, 0.0, 0.34217696850008, 0.0},
                                  {0.00277719819460, 0.00001567934613, 0.0, 0.0, 0.29786487010104}};
static RkStage rk5_stage(int k) {
  const double b10 = SO_B[0][0], b21 = SO_B[1][1];
  switch (k) {
    case 0: return {0, 1, -1, -1, 0.0, SO_A[0][0], b10, 0.0, 0.0};
    case 1: return {1, 2, -1, -1, 0.0, SO_A[1][1], b21, 0.0, 0.0};
    case 2: return {2, 3, -1, -1, SO_A[2][0], SO_A[2][2], SO_B[2][2] / SO_A[2][2], 0.0, 0.0};
    case 3:
      return {3, 4, 1, -1, SO_A[3][0] - SO_B[3][0] / b10, SO_A[3][3], SO_B[3][3] / SO_A[3][3],
              SO_A[3][1] + SO_B[3][0] / b10, 0.0};
    default:
      return {4, 0, 1, 2, SO_A[4][0] - SO_B[4][0] / b10, SO_A[4][4], SO_B[4][4] / SO_A[4][4],
              SO_A[4][1] + SO_B[4][0] / b10 - SO_B[4][1] / b21, SO_A[4][2] + SO_B[4][1] / b21};
  }
}

static RkStage rk_stage(const hydro_ctx* c, int k, bool frozen) {
  return (c->ns == 5 && !frozen) ? rk5_stage(k) : RK3_STAGES[k];
}

// Launch control of stage k of a step (frozen: of the SSP-RK3 replay).
static StageCtl stage_ctl(const hydro_ctx* c, int k, bool frozen) {
  const RkStage r = rk_stage(c, k, frozen);
  StageCtl ctl{k, 0, r.a, r.b};
  ctl.rk_c = r.c;
  ctl.rk_x0 = r.rx0;
  ctl.rk_x1 = r.rx1;
  ctl.last = k == (frozen ? 3 : c->ns) - 1;
  return ctl;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link against libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Tensor map of one padded working state: dimensions (pitch, rows, nf) with strides pitch and fstride
// elements (multiples of 16 bytes: pitch is a multiple of 4), box (68, TY + 6, nf) = one tile's halo box.
// Tile boxes start at column tx * 60 (240 tx bytes in FP32, 480 tx in FP64: 16-byte aligned) and never
// leave the allocation (pitch and rows cover whole tiles plus the halo).
template <typename real>
static int encode_state_map(hydro_ctx* c, const void* base, int box_h, CUtensorMap* out, int box_w = BOX_W,
                            int box_z = 0) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return HYDRO_ECUDA;
  const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->rows, (cuuint64_t)c->nf};
  const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * sizeof(real), (cuuint64_t)c->fstride * sizeof(real)};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, (cuuint32_t)(box_z > 0 ? box_z : c->nf)};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult r =
      fn(out, sizeof(real) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
         const_cast<void*>(base), dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? HYDRO_OK : HYDRO_ECUDA;
}

// Stage parameters of this context for the current variant.
template <typename real>
static void build_params(hydro_ctx* c, GridParams<real> out[NPARAMS]) {
  const hydro_config& g = c->cfg;
  Scratch<real>* s = scr<real>(c);
  GridParams<real> base{};
  base.fstride = c->fstride;
  base.nx = g.nx;
  base.ny = g.ny;
  base.pitch = c->pitch;
  base.tiles_x = c->tiles_x;
  base.tiles_y = (g.ny + tile_ty(c->variant) - 1) / tile_ty(c->variant);
  for (int k = 0; k < 4; ++k) base.bc[k] = g.bc[k];
  base.geometry = g.geometry;
  base.gamma = static_cast<real>(g.gamma);
  base.gm1 = static_cast<real>(g.gamma - 1.0);
  base.gravity = static_cast<real>(g.gravity_y);
  base.flame_speed = static_cast<real>(g.flame_speed);
  base.dx = (g.x1 - g.x0) / g.nx;
  base.dy = (g.y1 - g.y0) / g.ny;
  base.rdx = static_cast<real>(1.0 / base.dx);
  base.rdy = static_cast<real>(1.0 / base.dy);
  base.x0 = g.x0;
  base.dx_r = static_cast<real>(base.dx);
  base.x0_r = static_cast<real>(g.x0);
  base.cfl_delta = g.cfl * std::min(base.dx, base.dy);
  base.smax = &s->smax;
  base.dt_cur = &s->dt_cur;
  base.t_acc = &s->t_acc;
  base.err = &s->err;
  base.ext_div = static_cast<const real*>(c->char_div ? c->char_div : c->split_div);
  base.tmap_ty = tile_ty(c->variant);
  real* A = bufp<real>(c, 0);
  real* B = bufp<real>(c, 1);
  const CUtensorMap* maps = static_cast<const CUtensorMap*>(c->tmaps);
  auto stage_params = [&](const RkStage& r, int k, int ns) {
    GridParams<real> p = base;
    p.win = bufp<real>(c, r.win);
    p.tmap_win = maps + r.win;
    p.tmap_un = maps + TMAP_INTERIOR;
    p.un = A;
    p.out = bufp<real>(c, r.out);
    p.tmap_out = maps + TMAP_INTERIOR + r.out;
    p.tmap_char = c->char_div ? maps + TMAP_CHAR + r.win : nullptr;
    p.ux0 = r.x0 >= 0 ? bufp<real>(c, r.x0) : nullptr;
    p.ux1 = r.x1 >= 0 ? bufp<real>(c, r.x1) : nullptr;
    p.tmap_ux0 = r.x0 >= 0 ? maps + TMAP_INTERIOR + r.x0 : nullptr;
    p.tmap_ux1 = r.x1 >= 0 ? maps + TMAP_INTERIOR + r.x1 : nullptr;
    p.alpha_in = s->alpha[k];
    p.alpha_out = s->alpha[(k + 1) % ns];
    p.alpha_zero = s->alpha[(k + 2) % ns];
    if (k == ns - 1 && c->track_totals) p.totals = s->totals;
    if (k == 1 && c->track_totals) p.totals_reset = s->totals;
    return p;
  };
  for (int k = 0; k < c->ns; ++k) {
    GridParams<real> p = stage_params(rk_stage(c, k, false), k, c->ns);
    if (c->log_cap > 0) {
      p.dt_log = c->dt_log;
      p.alpha_log = c->alpha_log;
      p.log_count = &s->log_count;
      p.log_cap = c->log_cap;
    }
    out[k] = p;
  }
  for (int k = c->ns; k < P_FROZEN; ++k) out[k] = out[0];  // unused slots
  for (int k = 0; k < 3; ++k) {  // frozen SSP-RK3: alphas and dt from the frozen slots
    GridParams<real> f = stage_params(RK3_STAGES[k], k, 3);
    f.alpha_in = s->frozen_alpha[k];
    f.dt_src = (k == 0) ? &s->frozen_dt : nullptr;
    out[P_FROZEN + k] = f;
  }
  GridParams<real> r = base;  // L(W) of buffer A into buffer B
  r.win = A;
  r.tmap_win = maps;
  r.tmap_un = maps + TMAP_INTERIOR;
  r.un = A;
  r.out = B;
  r.tmap_out = maps + TMAP_INTERIOR + 1;
  r.tmap_char = c->char_div ? maps + TMAP_CHAR : nullptr;
  r.alpha_in = s->frozen_alpha[0];
  r.dt_src = &s->frozen_dt;
  out[P_RHS] = r;
}

template <typename real>
static int upload_params(hydro_ctx* c) {
  GridParams<real> p[NPARAMS];
  build_params<real>(c, p);
  alignas(64) CUtensorMap maps[NTMAPS] = {};
  for (int k = 0; k < c->ns; ++k) {
    const int rc = encode_state_map<real>(c, c->buf[k], tile_ty(c->variant) + 2 * GY, &maps[k]);
    if (rc) return fail(c, rc, "cuTensorMapEncodeTiled failed for the working states");
  }
  // the tile interiors: box (60, TY, nf) at padded column tx * 60 + 4 (16-byte aligned), row ty * TY + 3
  for (int k = 0; k < c->ns; ++k)
    if (encode_state_map<real>(c, c->buf[k], tile_ty(c->variant), &maps[TMAP_INTERIOR + k], TILE_X))
      return fail(c, HYDRO_ECUDA, "cuTensorMapEncodeTiled failed for the tile interiors");
  // the characteristic kernel's boxes: (CHAR_BOX_W, CBH, 4 hydro fields) at padded column 32 bx, row CY by
  if (c->char_div)
    for (int k = 0; k < c->ns; ++k)
      if (encode_state_map<real>(c, c->buf[k], CharTile<real>::CBH, &maps[TMAP_CHAR + k], CHAR_BOX_W, 4))
        return fail(c, HYDRO_ECUDA, "cuTensorMapEncodeTiled failed for the characteristic boxes");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(c->tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->params, p, sizeof(p), cudaMemcpyHostToDevice));
  c->uploaded_variant = c->variant;
  ++c->params_gen;
  if (c->step_graph) {
    cudaGraphExecDestroy(c->step_graph);
    c->step_graph = nullptr;
  }
  return HYDRO_OK;
}

static int upload(hydro_ctx* c) {
  return c->cfg.dtype == HYDRO_F64 ? upload_params<double>(c) : upload_params<float>(c);
}

static int grid_for(hydro_ctx* c, int nwork) {
  int occ = c->cfg.dtype == HYDRO_F64 ? stage_ctas_per_sm<double>(c->variant, c->nf)
                                      : stage_ctas_per_sm<float>(c->variant, c->nf);
  if (occ < 1) occ = 1;
  return std::max(1, std::min(nwork, occ * c->num_sms));
}

static int wait_stream(hydro_ctx* c) {
  cudaError_t e = cudaEventRecord(c->done, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
  const double limit = host_timeout_s();
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    e = cudaEventQuery(c->done);
    if (e == cudaSuccess) return HYDRO_OK;
    if (e != cudaErrorNotReady) return cuda_fail(c, e, "stream wait");
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return fail(c, HYDRO_ETIMEOUT, "stream did not finish within HYDRO_TIMEOUT_S");
    std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
  }
}

template <typename real>
static int launch_ctl(hydro_ctx* c, int k, const StageCtl& ctl, cudaStream_t s) {
  const int stage = ctl.stage;
  const int nwork = c->tiles_x * ((c->cfg.ny + tile_ty(c->variant) - 1) / tile_ty(c->variant));
  const GridParams<real>* p = static_cast<const GridParams<real>*>(c->params) + k;
  const bool prof = c->profiling && s == c->stream;
  if (prof) {
    while ((int)c->ev.size() < c->ev_used + 2) {
      cudaEvent_t ev;
      CK(cudaEventCreate(&ev));
      c->ev.push_back(ev);
    }
    CK(cudaEventRecord(c->ev[c->ev_used], s));
  }
  if (c->char_div) {  // characteristic scheme: the hydro divergence of this stage's input first
    CK(launch_char_div<real>(p, c->cfg.nx, c->cfg.ny, s));
    c->launches++;
  } else if (c->split_div) {  // field split: one CTA per (tile, hydro field) writes the divergence first
    StageCtl split = ctl;
    split.mode = 2;
    CK(launch_stage<real>(c->variant, c->nf, p, nullptr, 4 * nwork, split, grid_for(c, 4 * nwork), s));
    c->launches++;
  }
  (void)stage;
  CK(launch_stage<real>(c->variant, c->nf, p, nullptr, nwork, ctl, grid_for(c, nwork), s));
  if (prof) {
    CK(cudaEventRecord(c->ev[c->ev_used + 1], s));
    c->ev_used += 2;
  }
  c->launches++;
  return HYDRO_OK;
}

template <typename real>
static int launch_step(hydro_ctx* c, bool frozen, cudaStream_t s) {
  const int ns = frozen ? 3 : c->ns;
  for (int k = 0; k < ns; ++k) {
    int rc = launch_ctl<real>(c, frozen ? P_FROZEN + k : k, stage_ctl(c, k, frozen), s);
    if (rc) return rc;
  }
  return HYDRO_OK;
}

template <typename real>
static int ensure_graph(hydro_ctx* c) {
  if (c->step_graph) return HYDRO_OK;
  cudaGraph_t gr = nullptr;
  CK(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
  const long long before = c->launches;
  int rc = launch_step<real>(c, false, c->capture);
  cudaError_t e = cudaStreamEndCapture(c->capture, &gr);
  c->step_graph_launches = c->launches - before;
  c->launches = before;  // captured, not launched
  if (rc) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->step_graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return HYDRO_OK;
}

template <typename real>
static int pack_state(hydro_ctx* c, const real* U, double t0) {
  Scratch<real>* s = scr<real>(c);
  CK(cudaMemsetAsync(s, 0, c->defer_status ? offsetof(Scratch<real>, err) : offsetof(Scratch<real>, log_count),
                     c->stream));
  GridParams<real> g{};
  GridParams<real> all[NPARAMS];
  build_params<real>(c, all);
  g = all[0];
  g.out = bufp<real>(c, 0);
  CK(launch_pack<real>(U, g, c->nf, s->alpha[0], &s->smax, &s->t_acc, t0, c->stream));
  c->launches++;
  return HYDRO_OK;
}

template <typename real>
static int unpack_state(hydro_ctx* c, real* U, int k) {
  CK(launch_copy_state<real>(U, bufp<real>(c, k), c->cfg.nx, c->cfg.ny, c->nf, c->pitch, c->fstride, false, c->stream));
  c->launches++;
  return HYDRO_OK;
}

template <typename real>
static int read_status(hydro_ctx* c, double* t_inout, double* dt_last) {
  CK(cudaMemcpyAsync(c->host_scratch, c->scratch, sizeof(Scratch<real>), cudaMemcpyDeviceToHost, c->stream));
  int rc = wait_stream(c);
  if (rc) return rc;
  const Scratch<real>* hs = static_cast<const Scratch<real>*>(c->host_scratch);
  if (t_inout) *t_inout = hs->t_acc;
  if (dt_last) *dt_last = hs->dt_cur;
  if (hs->err & ERR_LAYOUT) return fail(c, HYDRO_ECUDA, "internal: stage kernel shared memory not 128-byte aligned");
  if (hs->err & ERR_TIMEOUT) return fail(c, HYDRO_ETIMEOUT, "a device wait gave up (tile copy did not complete)");
  if (hs->err & ERR_NONPHYSICAL)
    return fail(c, HYDRO_ENONPHYSICAL, "non-finite value, rho <= 0 or p <= 0 in the state");
  return HYDRO_OK;
}

// Last stage of a host-buffer call: the stage kernel runs over row bands of tiles on the context's stream;
// after each band, the copy stream moves that band's interior rows (every field) from the padded state to
// the caller's dense pinned state, overlapping the copy engine with the next band's compute. The context's
// stream then waits for the last copy.
template <typename real>
static int last_stage_to_host(hydro_ctx* c, real* host_out) {
  const hydro_config& g = c->cfg;
  const int TY = tile_ty(c->variant);
  const int trows = (g.ny + TY - 1) / TY;
  const int nb = std::min(hydro_ctx::NBANDS, trows);
  const int last = c->ns - 1;
  const GridParams<real>* p = static_cast<const GridParams<real>*>(c->params) + last;
  const StageCtl last_ctl = stage_ctl(c, last, false);
  const real* A = bufp<real>(c, 0);
  const size_t es = sizeof(real);
  // an externally formed divergence (characteristic scheme, FP64 field split) first, for the whole grid
  if (c->char_div) {
    CK(launch_char_div<real>(p, g.nx, g.ny, c->stream));
    c->launches++;
  } else if (c->split_div) {
    const int nall = c->tiles_x * trows;
    StageCtl split = last_ctl;
    split.mode = 2;
    CK(launch_stage<real>(c->variant, c->nf, p, nullptr, 4 * nall, split, grid_for(c, 4 * nall), c->stream));
    c->launches++;
  }
  for (int b = 0; b < nb; ++b) {
    const int r0 = b * trows / nb, r1 = (b + 1) * trows / nb;
    StageCtl ctl = last_ctl;
    ctl.w0 = r0 * c->tiles_x;
    const int nwork = (r1 - r0) * c->tiles_x;
    CK(launch_stage<real>(c->variant, c->nf, p, nullptr, nwork, ctl, grid_for(c, nwork), c->stream));
    c->launches++;
    CK(cudaEventRecord(c->band_ev[b], c->stream));
    CK(cudaStreamWaitEvent(c->copy_stream, c->band_ev[b], 0));
    const int j0 = r0 * TY, j1 = std::min(g.ny, r1 * TY);
    for (int f = 0; f < c->nf; ++f) {
      const real* src = A + f * c->fstride + (long long)(j0 + GY) * c->pitch + GX;
      real* dst = host_out + (size_t)f * g.nx * g.ny + (size_t)j0 * g.nx;
      CK(cudaMemcpy2DAsync(dst, g.nx * es, src, c->pitch * es, g.nx * es, j1 - j0, cudaMemcpyDeviceToHost,
                           c->copy_stream));
    }
  }
  CK(cudaEventRecord(c->copy_done, c->copy_stream));
  CK(cudaStreamWaitEvent(c->stream, c->copy_done, 0));
  return HYDRO_OK;
}

template <typename real>
static int step_impl(hydro_ctx* c, real* U, int nsteps, double* t_inout, double* dt_last, const double* dtl,
                     const double* al, real* host_out = nullptr) {
  const bool frozen = dtl != nullptr;
  int rc = pack_state<real>(c, U, t_inout ? *t_inout : 0.0);
  if (rc) return rc;
  // host_out: U is the caller's state in mapped host memory (the pack above read it over the host link);
  // the last step's final stage writes the result straight back there, so no staging copies remain
  const bool direct = host_out != nullptr && !frozen && nsteps > 0;
  const int nloop = direct ? nsteps - 1 : nsteps;
  const bool use_graph = !frozen && !c->profiling && nloop > 1;
  if (use_graph) {
    rc = ensure_graph<real>(c);
    if (rc) return rc;
  }
  Scratch<real>* s = scr<real>(c);
  for (int st = 0; st < nloop; ++st) {
    if (frozen) {
      CK(launch_set_frozen<real>(&s->frozen_dt, dtl[st], &s->frozen_alpha[0][0], al + 6 * st, c->stream));
      c->launches++;
      rc = launch_step<real>(c, true, c->stream);
    } else if (use_graph) {
      CK(cudaGraphLaunch(c->step_graph, c->stream));
      c->launches += c->step_graph_launches;
    } else {
      rc = launch_step<real>(c, false, c->stream);
    }
    if (rc) return rc;
  }
  if (direct) {
    for (int k = 0; k + 1 < c->ns && !rc; ++k) rc = launch_ctl<real>(c, k, stage_ctl(c, k, false), c->stream);
    if (!rc) rc = last_stage_to_host<real>(c, host_out);
    if (rc) return rc;
  } else {
    rc = unpack_state<real>(c, U, 0);
    if (rc) return rc;
  }
  if (frozen) {
    double tt = t_inout ? *t_inout : 0.0;
    for (int st = 0; st < nsteps; ++st) tt += dtl[st];
    int r2 = c->defer_status ? HYDRO_OK : read_status<real>(c, nullptr, nullptr);
    if (t_inout) *t_inout = tt;
    if (dt_last && nsteps > 0) *dt_last = dtl[nsteps - 1];
    return r2;
  }
  return read_status<real>(c, t_inout, dt_last);
}

static int check_ctx(hydro_ctx* c) {
  if (!c) return HYDRO_EINVAL;
  c->err.clear();
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return HYDRO_OK;
}

// ------------------------------------------------------------------------------------ C ABI
// (the declarations in hydro.h carry the C linkage to these definitions)

int hydro_init(const hydro_config* cfg, void* stream, hydro_ctx** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  std::string why;
  int rc = validate_config(cfg, &why);
  if (rc) return rc;
  static std::atomic<unsigned long long> next_uid{1};
  hydro_ctx* c = new hydro_ctx();
  c->uid = next_uid.fetch_add(1);
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(stream);
  c->nf = cfg->nfields;
  c->esize = cfg->dtype == HYDRO_F64 ? 8 : 4;
  auto bail = [&](int code) {
    hydro_destroy(c);
    return code;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return bail(HYDRO_ECUDA);
  c->tiles_x = (cfg->nx + TILE_X - 1) / TILE_X;
  c->pitch = c->tiles_x * TILE_X + 8;
  c->rows = ((cfg->ny + MAX_TY - 1) / MAX_TY) * MAX_TY + 2 * GY;
  c->fstride = (long long)c->pitch * c->rows;
  const size_t bytes = (size_t)c->nf * c->fstride * c->esize;
  c->ns = cfg->rk_stages == 5 ? 5 : 3;
  for (int k = 0; k < c->ns; ++k) {
    if (cudaMalloc(&c->buf[k], bytes) != cudaSuccess) return bail(HYDRO_ECUDA);
    if (cudaMemsetAsync(c->buf[k], 0, bytes, c->stream) != cudaSuccess) return bail(HYDRO_ECUDA);
  }
  if (cfg->scheme == HYDRO_SCHEME_CHARACTERISTIC) {
    const size_t db = (size_t)4 * c->fstride * c->esize;
    if (cudaMalloc(&c->char_div, db) != cudaSuccess) return bail(HYDRO_ECUDA);
    if (cudaMemsetAsync(c->char_div, 0, db, c->stream) != cudaSuccess) return bail(HYDRO_ECUDA);
  }
  if (cfg->dtype == HYDRO_F64 && cfg->scheme == HYDRO_SCHEME_COMPONENT &&
      (long long)c->tiles_x * ((cfg->ny + 14) / 15) * 2 < c->num_sms) {
    const size_t db = (size_t)4 * c->fstride * c->esize;
    if (cudaMalloc(&c->split_div, db) != cudaSuccess) return bail(HYDRO_ECUDA);
    if (cudaMemsetAsync(c->split_div, 0, db, c->stream) != cudaSuccess) return bail(HYDRO_ECUDA);
  }
  const size_t sb = c->esize == 8 ? sizeof(Scratch<double>) : sizeof(Scratch<float>);
  if (cudaMalloc(&c->scratch, sb) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaMemsetAsync(c->scratch, 0, sb, c->stream) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaMallocHost(&c->host_scratch, sb) != cudaSuccess) return bail(HYDRO_ECUDA);
  const size_t pb = c->esize == 8 ? sizeof(GridParams<double>) * NPARAMS : sizeof(GridParams<float>) * NPARAMS;
  if (cudaMalloc(&c->params, pb) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaMalloc(&c->tmaps, NTMAPS * sizeof(CUtensorMap)) != cudaSuccess) return bail(HYDRO_ECUDA);
  c->partial_blocks = 4 * c->num_sms;
  if (cudaMalloc(&c->partials, sizeof(double) * 5 * c->partial_blocks) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaMalloc(&c->d_totals, sizeof(double) * 5) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(HYDRO_ECUDA);
  for (int b = 0; b < hydro_ctx::NBANDS; ++b)
    if (cudaEventCreateWithFlags(&c->band_ev[b], cudaEventDisableTiming) != cudaSuccess) return bail(HYDRO_ECUDA);
  if (cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming) != cudaSuccess) return bail(HYDRO_ECUDA);
  // default tile shape: component-wise FP32 grids with at least one 60 x 30 tile per SM take that variant
  // (one CTA of 640 threads per SM: 2.53 against 3.00 ms per 8192^2 stage, 0.325 against 0.339 ms per
  // 1024 x 2048 step); others 60 x 15 with 320 threads (the characteristic scheme's stage, whose hydro
  // divergence comes from its own kernel, measured 2 % faster there). hydro_autotune measures instead.
  const long long tiles30 = (long long)c->tiles_x * ((cfg->ny + 29) / 30);
  c->variant = (cfg->dtype == HYDRO_F32 && cfg->scheme == HYDRO_SCHEME_COMPONENT &&
                stage_ctas_per_sm<float>(2, c->nf) >= 1 && tiles30 >= c->num_sms)
                   ? 2
                   : 1;
  if (upload(c) != HYDRO_OK) return bail(HYDRO_ECUDA);
  *out = c;
  return HYDRO_OK;
}

void hydro_destroy(hydro_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
  if (c->plan_graph) cudaGraphExecDestroy(c->plan_graph);
  if (c->sor_graph) cudaGraphExecDestroy(c->sor_graph);
  for (cudaEvent_t e : c->sor_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->pois);
  if (c->pois_host) cudaFreeHost(c->pois_host);
  for (int k = 0; k < 5; ++k) cudaFree(c->buf[k]);
  cudaFree(c->scratch);
  cudaFree(c->params);
  cudaFree(c->tmaps);
  cudaFree(c->partials);
  cudaFree(c->d_totals);
  cudaFree(c->unpadded);
  cudaFree(c->dt_log);
  cudaFree(c->alpha_log);
  cudaFree(c->plan_params);
  cudaFree(c->plan_work);
  cudaFree(c->bio_dev);
  cudaFreeHost(c->bio_host);
  cudaFree(c->adj_nu[0]);
  cudaFree(c->adj_nu[1]);
  cudaFree(c->adj_mu);
  cudaFree(c->adj_hb);
  cudaFree(c->adj_acc);
  cudaFree(c->ckpt);
  cudaFree(c->seg);
  cudaFree(c->rv_slots);
  cudaFree(c->front);
  cudaFree(c->front_count);
  cudaFree(c->char_div);
  cudaFree(c->split_div);
  if (c->host_scratch) cudaFreeHost(c->host_scratch);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->done) cudaEventDestroy(c->done);
  if (c->capture) cudaStreamDestroy(c->capture);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (cudaEvent_t e : c->band_ev)
    if (e) cudaEventDestroy(e);
  if (c->copy_done) cudaEventDestroy(c->copy_done);
  delete c;
}

const char* hydro_last_error(hydro_ctx* c) { return c ? c->err.c_str() : "null context"; }

int hydro_set_stream(hydro_ctx* c, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->stream = static_cast<cudaStream_t>(stream);
  return HYDRO_OK;
}

int hydro_step(hydro_ctx* c, void* U, int nsteps, double* t_inout, double* dt_last) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || nsteps < 0) return fail(c, HYDRO_EINVAL, "null state or negative step count");
  if (c->cfg.dtype == HYDRO_F64) return step_impl<double>(c, (double*)U, nsteps, t_inout, dt_last, nullptr, nullptr);
  return step_impl<float>(c, (float*)U, nsteps, t_inout, dt_last, nullptr, nullptr);
}

static int ensure_unpadded(hydro_ctx* c) {
  if (c->unpadded) return HYDRO_OK;
  CK(cudaMalloc(&c->unpadded, (size_t)c->nf * c->cfg.nx * c->cfg.ny * c->esize));
  return HYDRO_OK;
}

int hydro_step_host(hydro_ctx* c, void* U_host, int nsteps, double* t_inout, double* dt_last) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U_host || nsteps < 0) return fail(c, HYDRO_EINVAL, "null state or negative step count");
  // pinned (page-locked, mapped) host memory: the kernels read and write it directly over the host link
  cudaPointerAttributes at{};
  const bool mapped = cudaPointerGetAttributes(&at, U_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      at.devicePointer != nullptr && nsteps > 0;
  if (!mapped) (void)cudaGetLastError();
  if (mapped) {
    if (c->cfg.dtype == HYDRO_F64) {
      double* dp = static_cast<double*>(at.devicePointer);
      return step_impl<double>(c, dp, nsteps, t_inout, dt_last, nullptr, nullptr, dp);
    }
    float* dp = static_cast<float*>(at.devicePointer);
    return step_impl<float>(c, dp, nsteps, t_inout, dt_last, nullptr, nullptr, dp);
  }
  // pageable memory: stage through a device copy
  rc = ensure_unpadded(c);
  if (rc) return rc;
  const size_t bytes = (size_t)c->nf * c->cfg.nx * c->cfg.ny * c->esize;
  CK(cudaMemcpyAsync(c->unpadded, U_host, bytes, cudaMemcpyHostToDevice, c->stream));
  rc = hydro_step(c, c->unpadded, nsteps, t_inout, dt_last);
  int rc2 = HYDRO_OK;
  cudaError_t e = cudaMemcpyAsync(U_host, c->unpadded, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) rc2 = cuda_fail(c, e, "copy back to host");
  else rc2 = wait_stream(c);
  return rc ? rc : rc2;
}

// Recording, frozen replays and the adjoint are of the three-stage scheme.
static int require_rk3(hydro_ctx* c) {
  return c->ns == 3 ? HYDRO_OK
                    : fail(c, HYDRO_EINVAL, "recording, frozen steps and the adjoint are of the 3-stage scheme");
}

int hydro_step_frozen(hydro_ctx* c, void* U, int nsteps, const double* dtl, const double* al) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = require_rk3(c))) return rc;
  if (!U || nsteps < 0 || (nsteps > 0 && (!dtl || !al))) return fail(c, HYDRO_EINVAL, "bad frozen-step arguments");
  if (c->cfg.dtype == HYDRO_F64) return step_impl<double>(c, (double*)U, nsteps, nullptr, nullptr, dtl, al);
  return step_impl<float>(c, (float*)U, nsteps, nullptr, nullptr, dtl, al);
}

template <typename real>
static int rhs_impl(hydro_ctx* c, const real* U, double ax, double ay, real* L) {
  int rc = pack_state<real>(c, U, 0.0);
  if (rc) return rc;
  Scratch<real>* s = scr<real>(c);
  const double a6[6] = {ax, ay, ax, ay, ax, ay};
  CK(launch_set_frozen<real>(&s->frozen_dt, 0.0, &s->frozen_alpha[0][0], a6, c->stream));
  c->launches++;
  StageCtl rhs_ctl{0, 1, 0.0, 1.0};
  rc = launch_ctl<real>(c, P_RHS, rhs_ctl, c->stream);
  if (rc) return rc;
  return unpack_state<real>(c, L, 1);
}

int hydro_rhs(hydro_ctx* c, const void* U, double ax, double ay, void* L) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !L || !(ax >= 0.0) || !(ay >= 0.0)) return fail(c, HYDRO_EINVAL, "bad rhs arguments");
  if (c->cfg.dtype == HYDRO_F64) return rhs_impl<double>(c, (const double*)U, ax, ay, (double*)L);
  return rhs_impl<float>(c, (const float*)U, ax, ay, (float*)L);
}

int conserved_totals(hydro_ctx* c, const void* U, double out[5]) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !out) return fail(c, HYDRO_EINVAL, "null argument");
  const hydro_config& g = c->cfg;
  const double dx = (g.x1 - g.x0) / g.nx, dy = (g.y1 - g.y0) / g.ny;
  cudaError_t e = g.dtype == HYDRO_F64
                      ? launch_totals<double>((const double*)U, g.nx, g.ny, c->nf, g.geometry, g.x0, dx, dy,
                                              c->partials, c->partial_blocks, c->d_totals, c->stream)
                      : launch_totals<float>((const float*)U, g.nx, g.ny, c->nf, g.geometry, g.x0, dx, dy,
                                             c->partials, c->partial_blocks, c->d_totals, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "totals kernels");
  c->launches += 2;
  CK(cudaMemcpyAsync(c->host_scratch, c->d_totals, sizeof(double) * 5, cudaMemcpyDeviceToHost, c->stream));
  rc = wait_stream(c);
  if (rc) return rc;
  std::memcpy(out, c->host_scratch, sizeof(double) * 5);
  return HYDRO_OK;
}

int hydro_last_totals(hydro_ctx* c, double out[5]) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out) return fail(c, HYDRO_EINVAL, "null argument");
  if (!c->track_totals) return fail(c, HYDRO_ESTATE, "totals tracking is off");
  const size_t off = c->esize == 8 ? offsetof(Scratch<double>, totals) : offsetof(Scratch<float>, totals);
  CK(cudaMemcpyAsync(c->host_scratch, static_cast<char*>(c->scratch) + off, sizeof(double) * 5,
                     cudaMemcpyDeviceToHost, c->stream));
  rc = wait_stream(c);
  if (rc) return rc;
  std::memcpy(out, c->host_scratch, sizeof(double) * 5);
  return HYDRO_OK;
}

int hydro_record(hydro_ctx* c, int max_steps) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (max_steps > 0 && (rc = require_rk3(c))) return rc;
  if (max_steps < 0) return fail(c, HYDRO_EINVAL, "negative capacity");
  CK(cudaStreamSynchronize(c->stream));
  cudaFree(c->dt_log);
  cudaFree(c->alpha_log);
  c->dt_log = nullptr;
  c->alpha_log = nullptr;
  c->log_cap = 0;
  if (max_steps > 0) {
    CK(cudaMalloc(&c->dt_log, sizeof(double) * max_steps));
    CK(cudaMalloc(&c->alpha_log, sizeof(double) * 6 * max_steps));
    c->log_cap = max_steps;
  }
  const size_t off = c->esize == 8 ? offsetof(Scratch<double>, log_count) : offsetof(Scratch<float>, log_count);
  CK(cudaMemset(static_cast<char*>(c->scratch) + off, 0, sizeof(int)));
  return upload(c);
}

int hydro_get_log(hydro_ctx* c, int n, double* dtl, double* al, int* n_recorded) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  int cnt = 0;
  const size_t off = c->esize == 8 ? offsetof(Scratch<double>, log_count) : offsetof(Scratch<float>, log_count);
  CK(cudaMemcpy(&cnt, static_cast<char*>(c->scratch) + off, sizeof(int), cudaMemcpyDeviceToHost));
  cnt = std::min(cnt, c->log_cap);
  if (n_recorded) *n_recorded = cnt;
  if (n < 0 || n > cnt) return fail(c, HYDRO_EINVAL, "more log entries requested than recorded");
  if (n > 0) {
    if (!dtl || !al) return fail(c, HYDRO_EINVAL, "null log buffer");
    CK(cudaMemcpy(dtl, c->dt_log, sizeof(double) * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(al, c->alpha_log, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost));
  }
  return HYDRO_OK;
}

// ---- tile variants, autotuner, profiling

int hydro_tile_variants(hydro_ctx* c, int* n, int* current) {
  if (!c) return HYDRO_EINVAL;
  if (n) *n = NUM_VARIANTS;
  if (current) *current = c->variant;
  return HYDRO_OK;
}

int hydro_set_tile_variant(hydro_ctx* c, int v) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (v < 0 || v >= NUM_VARIANTS) return fail(c, HYDRO_EINVAL, "no such tile variant");
  const int occ = c->cfg.dtype == HYDRO_F64 ? stage_ctas_per_sm<double>(v, c->nf) : stage_ctas_per_sm<float>(v, c->nf);
  if (occ < 1) return fail(c, HYDRO_EINVAL, "tile variant does not fit on this device");
  if (v == c->variant) return HYDRO_OK;
  c->variant = v;
  return upload(c);
}

int hydro_set_adjoint_tile_rows(hydro_ctx* c, int rows) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (rows != 0 && rows != 16 && !(rows == 32 && c->cfg.dtype == HYDRO_F32))
    return fail(c, HYDRO_EINVAL, "adjoint tile rows: 0 (by grid size), 16, or 32 (FP32)");
  c->adj_rows = rows;
  return HYDRO_OK;
}

int hydro_tile_info(hydro_ctx* c, int v, int* tx, int* ty, int* threads, int* smem) {
  if (!c || v < 0 || v >= NUM_VARIANTS) return HYDRO_EINVAL;
  if (tx) *tx = TILE_X;
  if (ty) *ty = VARIANTS[v].ty;
  if (threads) *threads = VARIANTS[v].threads;
  if (smem)
    *smem = c->cfg.dtype == HYDRO_F64 ? stage_smem_bytes<double>(v, c->nf) : stage_smem_bytes<float>(v, c->nf);
  return HYDRO_OK;
}

int hydro_profile(hydro_ctx* c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->profiling = enable != 0;
  c->ev_used = 0;
  return HYDRO_OK;
}

int hydro_stage_timing(hydro_ctx* c, int* launches, double* total_ms) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  for (int k = 0; k + 1 < c->ev_used; k += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
    tot += ms;
  }
  if (launches) *launches = c->ev_used / 2;
  if (total_ms) *total_ms = tot;
  return HYDRO_OK;
}

long long hydro_launch_count(hydro_ctx* c) { return c ? c->launches : -1; }

template <typename real>
static int autotune_impl(hydro_ctx* c, const real* U, int steps, double* ms_out) {
  const int keep = c->variant;
  double best = 1e300;
  int best_v = keep;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int v = 0; v < NUM_VARIANTS; ++v) {
    double ms_step = -1.0;
    if (stage_ctas_per_sm<real>(v, c->nf) >= 1) {
      c->variant = v;
      int rc = upload(c);
      if (!rc) rc = pack_state<real>(c, U, 0.0);
      if (!rc) rc = launch_step<real>(c, false, c->stream);  // warm-up step
      if (!rc) {
        cudaEventRecord(e0, c->stream);
        for (int s = 0; s < steps && !rc; ++s) rc = launch_step<real>(c, false, c->stream);
        cudaEventRecord(e1, c->stream);
      }
      if (!rc) rc = read_status<real>(c, nullptr, nullptr);
      if (rc && rc != HYDRO_ENONPHYSICAL) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->variant = keep;
        upload(c);
        return rc;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_step = ms / std::max(1, steps);
      if (ms_step < best) {
        best = ms_step;
        best_v = v;
      }
    }
    if (ms_out) ms_out[v] = ms_step;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->variant = best_v;
  return upload(c);
}

int hydro_autotune(hydro_ctx* c, const void* U, int steps, double* ms_out) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || steps < 1) return fail(c, HYDRO_EINVAL, "bad autotune arguments");
  if (c->cfg.dtype == HYDRO_F64) return autotune_impl<double>(c, (const double*)U, steps, ms_out);
  return autotune_impl<float>(c, (const float*)U, steps, ms_out);
}

// ---- batched ensembles

// Work-list layouts of a batch plan. The list of (member, tile) items is member-ordered; each persistent
// CTA takes a contiguous run of it (RUNS_ROWS: a member's tiles row by row; RUNS_COLUMNS: column by
// column, so that a CTA's consecutive tiles share halo rows), or the items are dealt out one by one
// (INTERLEAVED: CTA b takes items b, b + G, ...).
enum BatchLayout { BATCH_RUNS_ROWS = 0, BATCH_RUNS_COLUMNS = 1, BATCH_INTERLEAVED = 2, BATCH_LAYOUTS = 3 };
constexpr int BATCH_WAVES = 2;  // grid sizes tried: 1 or 2 waves of resident CTAs

// ms_graph != null: time the graph replays of the nsteps steps alone (events) into *ms_graph;
// writeback = false: the members' working states are stepped but U is neither written nor t updated.
template <typename real>
static int batch_impl(hydro_ctx* const* m, void* const* U, int n, int nsteps, double* t, bool writeback = true,
                      double* ms_graph = nullptr) {
  hydro_ctx* c = m[0];
  // every member (the first included) on the first member's tile variant, with device parameters and
  // tensor maps built for it
  for (int k = 0; k < n; ++k) {
    if (m[k]->variant != c->variant || m[k]->uploaded_variant != c->variant) {
      m[k]->variant = c->variant;
      int rc = upload(m[k]);
      if (rc) return fail(c, rc, "member " + std::to_string(k) + ": " + m[k]->err);
    }
  }
  bool same = (int)c->plan_members.size() == n && c->plan_variant == c->variant &&
              c->plan_waves == c->batch_waves && c->plan_layout == c->batch_layout;
  for (int k = 0; same && k < n; ++k) same = c->plan_members[k] == m[k]->uid && c->plan_gens[k] == m[k]->params_gen;
  if (!same) {
    if (c->plan_graph) {
      cudaGraphExecDestroy(c->plan_graph);
      c->plan_graph = nullptr;
    }
    cudaFree(c->plan_params);
    cudaFree(c->plan_work);
    c->plan_params = nullptr;
    c->plan_work = nullptr;
    c->plan_members.clear();  // no plan until the new one is complete (an error below leaves none)
    c->plan_gens.clear();
    c->plan_nwork = 0;
    std::vector<GridParams<real>> P(c->ns * (size_t)n);
    std::vector<WorkItem> W;
    for (int k = 0; k < n; ++k) {
      GridParams<real> p[NPARAMS];
      build_params<real>(m[k], p);
      for (int s = 0; s < c->ns; ++s) {
        P[(size_t)s * n + k] = p[s];
        P[(size_t)s * n + k].ext_div = nullptr;  // the batched launch computes every field itself
      }
    }
    // CTA b of the persistent launch takes items b, b + G, b + 2G, ...: with the RUNS layouts it gets a
    // contiguous run of the member-ordered tile list, so that it changes member (a flush and a parameter
    // reload) only at run boundaries; every CTA gets the same number of tiles (within one)
    std::vector<WorkItem> L;
    for (int k = 0; k < n; ++k) {
      const int tx_n = m[k]->tiles_x, ty_n = (m[k]->cfg.ny + tile_ty(c->variant) - 1) / tile_ty(c->variant);
      if (c->batch_layout == BATCH_RUNS_COLUMNS) {
        for (int tx = 0; tx < tx_n; ++tx)
          for (int ty = 0; ty < ty_n; ++ty) L.push_back(WorkItem{k, ty * tx_n + tx});
      } else {
        for (int t = 0; t < tx_n * ty_n; ++t) L.push_back(WorkItem{k, t});
      }
    }
    const int total = (int)L.size();
    const int G = std::max(1, std::min(total, grid_for(c, total) * std::max(1, c->batch_waves)));
    if (c->batch_layout == BATCH_INTERLEAVED) {
      W = L;
    } else {
      W.assign(total, WorkItem{0, 0});
      for (int b = 0, start = 0; b < G; ++b) {
        const int cnt = (total - b + G - 1) / G;  // items w = b + kG < total
        for (int k = 0; k < cnt; ++k) W[b + (size_t)k * G] = L[start + k];
        start += cnt;
      }
    }
    c->plan_grid = G;
    CK(cudaMalloc(&c->plan_params, sizeof(GridParams<real>) * P.size()));
    CK(cudaMalloc(&c->plan_work, sizeof(WorkItem) * W.size()));
    CK(cudaMemcpy(c->plan_params, P.data(), sizeof(GridParams<real>) * P.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->plan_work, W.data(), sizeof(WorkItem) * W.size(), cudaMemcpyHostToDevice));
    c->plan_nwork = total;
    for (int k = 0; k < n; ++k) {
      c->plan_members.push_back(m[k]->uid);
      c->plan_gens.push_back(m[k]->params_gen);
    }
    c->plan_variant = c->variant;
    c->plan_waves = c->batch_waves;
    c->plan_layout = c->batch_layout;
  }
  const int grid = c->plan_grid;
  const GridParams<real>* P = static_cast<const GridParams<real>*>(c->plan_params);
  // the members' arguments in one upload; their scratch records zeroed and their states packed (buffer A,
  // with the first stage's reductions) by one launch each for all members
  constexpr size_t SB = sizeof(Scratch<real>);  // one record per member, back to back
  const size_t args_bytes = 3 * sizeof(void*) * (size_t)n;
  if (c->bio_cap < n) {
    cudaFree(c->bio_dev);
    cudaFreeHost(c->bio_host);
    c->bio_dev = c->bio_host = nullptr;
    c->bio_cap = 0;
    CK(cudaMalloc(&c->bio_dev, args_bytes + SB * n));
    CK(cudaMallocHost(&c->bio_host, args_bytes + SB * n));
    c->bio_cap = n;
  }
  CK(cudaStreamSynchronize(c->stream));  // the pinned arguments of an earlier call are no longer in use
  void** hptr = static_cast<void**>(c->bio_host);
  long long max_cells = 0;
  for (int k = 0; k < n; ++k) {
    hptr[k] = U[k];
    hptr[n + k] = m[k]->scratch;
    reinterpret_cast<double*>(hptr + 2 * n)[k] = t ? t[k] : 0.0;
    max_cells = std::max(max_cells, (long long)m[k]->cfg.nx * m[k]->cfg.ny);
  }
  void** dptr = static_cast<void**>(c->bio_dev);
  unsigned char* gather_dev = static_cast<unsigned char*>(c->bio_dev) + args_bytes;
  const unsigned char* gather_host = static_cast<const unsigned char*>(c->bio_host) + args_bytes;
  CK(cudaMemcpyAsync(dptr, hptr, args_bytes, cudaMemcpyHostToDevice, c->stream));
  CK(launch_batch_scratch(dptr + n, n, (int)offsetof(Scratch<real>, log_count), nullptr, c->stream));
  CK(launch_batch_pack<real>(P, reinterpret_cast<const real* const*>(dptr), reinterpret_cast<const double*>(dptr + 2 * n),
                             n, c->nf, max_cells, c->stream));
  c->launches += 2;
  const WorkItem* W = static_cast<const WorkItem*>(c->plan_work);
  auto launch3 = [&](cudaStream_t s) -> int {
    for (int k = 0; k < c->ns; ++k) {
      const StageCtl ctl = stage_ctl(c, k, false);
      CK(launch_stage<real>(c->variant, c->nf, P + (size_t)k * n, W, c->plan_nwork, ctl, grid, s));
    }
    return HYDRO_OK;
  };
  if (!c->plan_graph) {
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
    int rc = launch3(c->capture);
    cudaError_t e = cudaStreamEndCapture(c->capture, &gr);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->plan_graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  cudaEvent_t g0 = nullptr, g1 = nullptr;
  if (ms_graph) {
    CK(cudaEventCreate(&g0));
    CK(cudaEventCreate(&g1));
    CK(cudaEventRecord(g0, c->stream));
  }
  for (int s = 0; s < nsteps; ++s) {
    CK(cudaGraphLaunch(c->plan_graph, c->stream));
    c->launches += c->ns;
  }
  if (ms_graph) CK(cudaEventRecord(g1, c->stream));
  int worst = HYDRO_OK;
  // every member's state back into its caller buffer, and every scratch record into one host copy
  if (writeback) {
    CK(launch_batch_unpack<real>(P, reinterpret_cast<real* const*>(dptr), n, c->nf, max_cells, c->stream));
    c->launches++;
  }
  CK(launch_batch_scratch(dptr + n, n, (int)SB, gather_dev, c->stream));
  c->launches++;
  CK(cudaMemcpyAsync(const_cast<unsigned char*>(gather_host), gather_dev, SB * n, cudaMemcpyDeviceToHost, c->stream));
  int rc = wait_stream(c);
  if (!rc)
    for (int k = 0; k < n; ++k) std::memcpy(m[k]->host_scratch, gather_host + SB * k, sizeof(Scratch<real>));
  if (ms_graph) {
    float ms = 0.f;
    if (!rc) cudaEventElapsedTime(&ms, g0, g1);
    *ms_graph = ms;
    cudaEventDestroy(g0);
    cudaEventDestroy(g1);
  }
  if (rc) return rc;
  for (int k = 0; k < n; ++k) {
    const Scratch<real>* hs = static_cast<const Scratch<real>*>(m[k]->host_scratch);
    if (t && writeback) t[k] = hs->t_acc;
    if (hs->err & ERR_LAYOUT) worst = fail(c, HYDRO_ECUDA, "internal: stage kernel shared memory not 128-byte aligned");
    else if (hs->err & ERR_TIMEOUT) worst = fail(c, HYDRO_ETIMEOUT, "member " + std::to_string(k) + ": device wait gave up");
    else if ((hs->err & ERR_NONPHYSICAL) && worst == HYDRO_OK)
      worst = fail(c, HYDRO_ENONPHYSICAL, "member " + std::to_string(k) + ": non-physical state");
  }
  return worst;
}

static int batch_check(hydro_ctx* const* members, void* const* U, int n) {
  hydro_ctx* c = members[0];
  for (int k = 0; k < n; ++k) {
    if (!members[k] || !U[k]) return fail(c, HYDRO_EINVAL, "null member or state");
    if (members[k]->cfg.dtype != c->cfg.dtype || members[k]->nf != c->nf || members[k]->device != c->device ||
        members[k]->ns != c->ns)
      return fail(c, HYDRO_EINVAL, "members must share dtype, nfields, time scheme and device");
    if (members[k]->cfg.scheme != HYDRO_SCHEME_COMPONENT)
      return fail(c, HYDRO_EINVAL, "batched steps take component-wise contexts (step characteristic ones one by one)");
  }
  return HYDRO_OK;
}

int hydro_batch_step(hydro_ctx* const* members, void* const* U, int n, int nsteps, double* t) {
  if (!members || !U || n < 1 || nsteps < 0) return HYDRO_EINVAL;
  hydro_ctx* c = members[0];
  int rc = check_ctx(c);
  if (rc) return rc;
  rc = batch_check(members, U, n);
  if (rc) return rc;
  if (c->cfg.dtype == HYDRO_F64) return batch_impl<double>(members, U, n, nsteps, t);
  return batch_impl<float>(members, U, n, nsteps, t);
}

int hydro_batch_autotune(hydro_ctx* const* members, void* const* U, int n, int steps, double* ms_out, int* best) {
  if (!members || !U || n < 1 || steps < 1) return HYDRO_EINVAL;
  hydro_ctx* c = members[0];
  int rc = check_ctx(c);
  if (rc) return rc;
  rc = batch_check(members, U, n);
  if (rc) return rc;
  const bool f64 = c->cfg.dtype == HYDRO_F64;
  const int keep_v = c->variant, keep_w = c->batch_waves, keep_l = c->batch_layout;
  double best_ms = 1e300;
  int best_i = -1;
  for (int v = 0; v < NUM_VARIANTS; ++v) {
    const bool fits = (f64 ? stage_ctas_per_sm<double>(v, c->nf) : stage_ctas_per_sm<float>(v, c->nf)) >= 1;
    for (int w = 0; w < BATCH_WAVES; ++w) {
      for (int l = 0; l < BATCH_LAYOUTS; ++l) {
        const int i = (v * BATCH_WAVES + w) * BATCH_LAYOUTS + l;
        double ms = -1.0;
        if (fits) {
          c->variant = v;
          c->batch_waves = w + 1;
          c->batch_layout = l;
          rc = upload(c);  // the first member's own parameters and tensor maps for this variant
          if (rc) {
            c->variant = keep_v;
            c->batch_waves = keep_w;
            c->batch_layout = keep_l;
            upload(c);
            return rc;
          }
          // one untimed step (plan, graph), then `steps` timed graph replays; U is only read
          rc = f64 ? batch_impl<double>(members, U, n, 1, nullptr, false) : batch_impl<float>(members, U, n, 1, nullptr, false);
          double g = 0.0;
          if (!rc || rc == HYDRO_ENONPHYSICAL)
            rc = f64 ? batch_impl<double>(members, U, n, steps, nullptr, false, &g)
                     : batch_impl<float>(members, U, n, steps, nullptr, false, &g);
          if (rc && rc != HYDRO_ENONPHYSICAL) {
            c->variant = keep_v;
            c->batch_waves = keep_w;
            c->batch_layout = keep_l;
            return rc;
          }
          ms = g / steps;
          if (ms < best_ms) {
            best_ms = ms;
            best_i = i;
          }
        }
        if (ms_out) ms_out[i] = ms;
      }
    }
  }
  if (best_i < 0) {
    c->variant = keep_v;
    c->batch_waves = keep_w;
    c->batch_layout = keep_l;
    return fail(c, HYDRO_EINVAL, "no tile variant fits the device");
  }
  c->variant = best_i / (BATCH_WAVES * BATCH_LAYOUTS);
  c->batch_waves = (best_i / BATCH_LAYOUTS) % BATCH_WAVES + 1;
  c->batch_layout = best_i % BATCH_LAYOUTS;
  if (best) *best = best_i;
  return upload(c);
}

// ---- discrete adjoint (frozen dt and stage alphas) and two-level checkpointing

static int ensure_adjoint_buffers(hydro_ctx* c) {
  if (c->adj_mu) return HYDRO_OK;
  const size_t bytes = (size_t)c->nf * c->fstride * c->esize;
  for (int k = 0; k < 2; ++k) {
    CK(cudaMalloc(&c->adj_nu[k], bytes));
    CK(cudaMemsetAsync(c->adj_nu[k], 0, bytes, c->stream));  // zero ghost frame, never written
  }
  CK(cudaMalloc(&c->adj_mu, bytes));
  CK(cudaMemsetAsync(c->adj_mu, 0, bytes, c->stream));
  CK(cudaMalloc(&c->adj_acc, bytes));
  CK(cudaMemsetAsync(c->adj_acc, 0, bytes, c->stream));
  const size_t hb = (size_t)4 * c->fstride * c->esize;
  CK(cudaMalloc(&c->adj_hb, hb));
  CK(cudaMemsetAsync(c->adj_hb, 0, hb, c->stream));  // zero frame: only interior cells are written
  return HYDRO_OK;
}

// caller-layout <-> padded-interior copies of a full state-shaped array
template <typename real>
static int copy_in(hydro_ctx* c, real* padded, const real* U) {
  CK(launch_copy_state<real>(padded, U, c->cfg.nx, c->cfg.ny, c->nf, c->pitch, c->fstride, true, c->stream));
  c->launches++;
  return HYDRO_OK;
}

template <typename real>
static int copy_out(hydro_ctx* c, real* U, const real* padded) {
  CK(launch_copy_state<real>(U, padded, c->cfg.nx, c->cfg.ny, c->nf, c->pitch, c->fstride, false, c->stream));
  c->launches++;
  return HYDRO_OK;
}

template <typename real>
// One adjoint step on padded cotangents (zero ghost frames): the cotangent of U^{n+1} in nu0, which is
// then reused as scratch; the result (dJ/dU^n) in acc; nu1 a third buffer for the middle stage.
static int adjoint_step_bufs(hydro_ctx* c, const real* Un, real* nu0, real* nu1, real* acc, double dt,
                             const double* alpha) {
  // stage states U^n (A), U^(1) (B), U^(2) (C) with the frozen alphas and dt
  int rc = pack_state<real>(c, Un, 0.0);
  if (rc) return rc;
  Scratch<real>* s = scr<real>(c);
  CK(launch_set_frozen<real>(&s->frozen_dt, dt, &s->frozen_alpha[0][0], alpha, c->stream));
  c->launches++;
  rc = launch_ctl<real>(c, P_FROZEN + 0, stage_ctl(c, 0, true), c->stream);
  if (!rc) rc = launch_ctl<real>(c, P_FROZEN + 1, stage_ctl(c, 1, true), c->stream);
  if (rc) return rc;
  real* nu[2] = {nu0, nu1};
  const hydro_config& g = c->cfg;
  AdjParams<real> P{};
  P.mu = static_cast<real*>(c->adj_mu);
  P.hb = static_cast<real*>(c->adj_hb);
  P.acc = acc;
  P.fstride = c->fstride;
  P.nx = g.nx;
  P.ny = g.ny;
  P.pitch = c->pitch;
  P.rows = c->rows;
  for (int k = 0; k < 4; ++k) P.bc[k] = g.bc[k];
  P.geometry = g.geometry;
  P.gamma = static_cast<real>(g.gamma);
  P.gravity = static_cast<real>(g.gravity_y);
  P.flame_speed = static_cast<real>(g.flame_speed);
  P.dx = (g.x1 - g.x0) / g.nx;
  P.dy = (g.y1 - g.y0) / g.ny;
  P.x0 = g.x0;
  P.dt = dt;
  P.rdx_r = static_cast<real>(1.0 / P.dx);
  P.rdy_r = static_cast<real>(1.0 / P.dy);
  P.dx_r = static_cast<real>(P.dx);
  P.x0_r = static_cast<real>(P.x0);
  P.dt_r = static_cast<real>(dt);
  P.tile_rows = c->adj_rows;
  // reverse stages 2, 1, 0
  const int order[3] = {2, 1, 0};
  for (int q = 0; q < 3; ++q) {
    const int k = order[q];
    P.W = bufp<real>(c, k);  // stage k's input: A, B, C
    P.nu = nu[q & 1];
    P.out = nu[(q + 1) & 1];
    P.ax = static_cast<real>(alpha[2 * k]);
    P.ay = static_cast<real>(alpha[2 * k + 1]);
    P.a = RK_A[k];
    P.b = RK_B[k];
    P.a_r = static_cast<real>(P.a);
    P.b_r = static_cast<real>(P.b);
    P.acc_mode = (q == 0) ? 0 : (q == 1) ? 1 : 2;
    int nl = 0;
    CK(launch_adjoint_stage<real>(P, c->nf, c->stream, &nl));
    c->launches += nl;
  }
  return HYDRO_OK;
}

// One adjoint step with an unpadded cotangent lam (in: of U^{n+1}; out: of U^n).
template <typename real>
static int adjoint_step_impl(hydro_ctx* c, const real* Un, real* lam, double dt, const double* alpha) {
  int rc = ensure_adjoint_buffers(c);
  if (rc) return rc;
  real* acc = static_cast<real*>(c->adj_acc);
  rc = copy_in<real>(c, static_cast<real*>(c->adj_nu[0]), lam);
  if (!rc) rc = adjoint_step_bufs<real>(c, Un, static_cast<real*>(c->adj_nu[0]), static_cast<real*>(c->adj_nu[1]), acc,
                                        dt, alpha);
  if (!rc) rc = copy_out<real>(c, lam, acc);
  if (rc) return rc;
  return c->defer_status ? HYDRO_OK : read_status<real>(c, nullptr, nullptr);
}

// A reverse sweep keeps its cotangent padded between steps: buffers adj_nu[0] and adj_acc alternate as the
// step's input and result (c->adj_in names the one holding the current cotangent), adj_nu[1] is the third.
template <typename real>
static int sweep_step(hydro_ctx* c, const real* Un, double dt, const double* alpha) {
  real* B[3] = {static_cast<real*>(c->adj_nu[0]), static_cast<real*>(c->adj_nu[1]), static_cast<real*>(c->adj_acc)};
  const int in = c->adj_in, out = 2 - in;
  const int rc = adjoint_step_bufs<real>(c, Un, B[in], B[1], B[out], dt, alpha);
  c->adj_in = out;
  return rc;
}

int hydro_adjoint_step(hydro_ctx* c, const void* U_n, void* lambda, double dt, const double alpha[6]) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = require_rk3(c))) return rc;
  if (!U_n || !lambda || !alpha || !(dt >= 0.0)) return fail(c, HYDRO_EINVAL, "bad adjoint arguments");
  if (c->cfg.scheme != HYDRO_SCHEME_COMPONENT)
    return fail(c, HYDRO_EINVAL, "the discrete adjoint is of the component-wise scheme");
  for (int k = 0; k < 6; ++k)
    if (!(alpha[k] >= 0.0) || !std::isfinite(alpha[k])) return fail(c, HYDRO_EINVAL, "alphas must be finite, >= 0");
  if (c->cfg.dtype == HYDRO_F64)
    return adjoint_step_impl<double>(c, (const double*)U_n, (double*)lambda, dt, alpha);
  return adjoint_step_impl<float>(c, (const float*)U_n, (float*)lambda, dt, alpha);
}

int hydro_forward_checkpointed(hydro_ctx* c, void* U, int nsteps, int every) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = require_rk3(c))) return rc;
  if (!U || nsteps < 1) return fail(c, HYDRO_EINVAL, "bad arguments");
  if (c->cfg.scheme != HYDRO_SCHEME_COMPONENT)
    return fail(c, HYDRO_EINVAL, "the discrete adjoint is of the component-wise scheme");
  if (every <= 0) every = std::max(1, (int)std::ceil(std::sqrt((double)nsteps)));
  every = std::min(every, nsteps);
  const int nseg = (nsteps + every - 1) / every;
  const size_t state = (size_t)c->nf * c->cfg.nx * c->cfg.ny * c->esize;
  if (c->ckpt_cap < (size_t)nseg) {
    cudaFree(c->ckpt);
    c->ckpt = nullptr;
    c->ckpt_cap = 0;
    CK(cudaMalloc(&c->ckpt, state * nseg));
    c->ckpt_cap = nseg;
  }
  rc = hydro_record(c, nsteps);
  if (rc) return rc;
  double t = 0.0;
  for (int sg = 0; sg < nseg; ++sg) {
    CK(cudaMemcpyAsync(static_cast<char*>(c->ckpt) + state * sg, U, state, cudaMemcpyDeviceToDevice, c->stream));
    const int n = std::min(every, nsteps - sg * every);
    rc = hydro_step(c, U, n, &t, nullptr);
    if (rc) return rc;
  }
  c->ck_nsteps = nsteps;
  c->ck_every = every;
  c->ck_mode = 0;
  return HYDRO_OK;
}

// ---- binomial checkpointing (revolve; Griewank 1992, Griewank & Walther 2000)
//
// Reversing n steps from a stored state with s free state slots: store the state at some m in a free
// slot, reverse [m, n) with s - 1 free slots, then [0, m) with s; with no free slot every step's state is
// recomputed from the start (n (n - 1) / 2 forward steps). With c = s + 1 slots counting the start's and
// t the least number of sweeps with C(c + t, c) >= n, the fewest forward steps any such schedule needs is
// P(n, s) = t n - C(c + 1 + t - 1, t - 1) (Griewank's bound); the split taken at each level is the m that
// minimises m + P(n - m, s - 1) + P(m, s), so the whole schedule attains P(n, s).

static long long rv_binom(int c, int t) {  // C(c + t, t), exact while it fits (saturates at 2^62)
  long long b = 1;
  const int k_max = std::min(c, t), big = std::max(c, t);
  for (int k = 1; k <= k_max; ++k) {
    if (b > (1LL << 62) / (big + k)) return 1LL << 62;
    b = b * (big + k) / k;
  }
  return b;
}

static long long rv_cost(int n, int s) {  // P(n, s)
  if (n <= 1) return 0;
  if (s == 0) return (long long)n * (n - 1) / 2;
  const int c = s + 1;
  int t = 0;
  while (rv_binom(c, t) < n) ++t;
  return (long long)t * n - rv_binom(c + 1, t - 1);
}

static int rv_split(int n, int s) {  // the checkpoint m (1 .. n-1) for n >= 2 and s >= 1
  long long best = -1;
  int bm = 1;
  for (int m = 1; m < n; ++m) {
    const long long v = m + rv_cost(n - m, s - 1) + rv_cost(m, s);
    if (best < 0 || v < best) {
      best = v;
      bm = m;
    }
  }
  return bm;
}

template <typename real>
static int rv_advance(hydro_ctx* c, real* U, int from, int to, const std::vector<double>& dtl,
                      const std::vector<double>& al) {
  for (int st = from; st < to; ++st) {
    const int rc = step_impl<real>(c, U, 1, nullptr, nullptr, &dtl[st], &al[6 * (size_t)st]);
    if (rc) return rc;
  }
  return HYDRO_OK;
}

// Reverse steps [a, b): slot `level` holds the state at a, slots level+1 .. nslots-1 are free, tmp is the
// recomputation buffer.
template <typename real>
static int rv_reverse(hydro_ctx* c, real* slots, int nslots, real* tmp, int level, int a, int b,
                      size_t elems, const std::vector<double>& dtl, const std::vector<double>& al) {
  const size_t state = elems * sizeof(real);
  real* Ua = slots + elems * (size_t)level;
  const int n = b - a, s = nslots - 1 - level;
  if (n == 1) return sweep_step<real>(c, Ua, dtl[a], &al[6 * (size_t)a]);
  if (s == 0) {
    for (int k = b - 1; k >= a; --k) {
      CK(cudaMemcpyAsync(tmp, Ua, state, cudaMemcpyDeviceToDevice, c->stream));
      int rc = rv_advance<real>(c, tmp, a, k, dtl, al);
      if (!rc) rc = sweep_step<real>(c, tmp, dtl[k], &al[6 * (size_t)k]);
      if (rc) return rc;
    }
    return HYDRO_OK;
  }
  const int m = a + rv_split(n, s);
  real* Um = slots + elems * (size_t)(level + 1);
  CK(cudaMemcpyAsync(Um, Ua, state, cudaMemcpyDeviceToDevice, c->stream));
  int rc = rv_advance<real>(c, Um, a, m, dtl, al);
  if (!rc) rc = rv_reverse<real>(c, slots, nslots, tmp, level + 1, m, b, elems, dtl, al);
  if (!rc) rc = rv_reverse<real>(c, slots, nslots, tmp, level, a, m, elems, dtl, al);
  return rc;
}

int hydro_forward_revolve(hydro_ctx* c, void* U, int nsteps, int snapshots, long long* sweep_forward_steps) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = require_rk3(c))) return rc;
  if (!U || nsteps < 1 || snapshots < 0 || snapshots > 4096) return fail(c, HYDRO_EINVAL, "bad arguments");
  if (c->cfg.scheme != HYDRO_SCHEME_COMPONENT)
    return fail(c, HYDRO_EINVAL, "the discrete adjoint is of the component-wise scheme");
  const size_t state = (size_t)c->nf * c->cfg.nx * c->cfg.ny * c->esize;
  const size_t need = (size_t)snapshots + 2;  // U^0, the snapshots, the recomputation buffer
  if (c->rv_cap < need) {
    cudaFree(c->rv_slots);
    c->rv_slots = nullptr;
    c->rv_cap = 0;
    CK(cudaMalloc(&c->rv_slots, state * need));
    c->rv_cap = need;
  }
  rc = hydro_record(c, nsteps);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->rv_slots, U, state, cudaMemcpyDeviceToDevice, c->stream));
  double t = 0.0;
  rc = hydro_step(c, U, nsteps, &t, nullptr);
  if (rc) return rc;
  c->ck_nsteps = nsteps;
  c->ck_mode = 1;
  c->rv_snapshots = snapshots;
  if (sweep_forward_steps) *sweep_forward_steps = rv_cost(nsteps, std::min(snapshots, nsteps));
  return HYDRO_OK;
}

template <typename real>
static int sweep_segments(hydro_ctx* c, real* seg, int nseg, int every, int N, size_t elems, size_t state,
                          const std::vector<double>& dtl, const std::vector<double>& al) {
  int rc = HYDRO_OK;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s0 = sg * every, s1 = std::min(N, s0 + every);
    // recompute the segment's states from its checkpoint with the recorded dt / alphas
    CK(cudaMemcpyAsync(seg, static_cast<const char*>(c->ckpt) + state * sg, state, cudaMemcpyDeviceToDevice,
                       c->stream));
    for (int st = s0; st + 1 < s1; ++st) {
      real* nxt = seg + elems * (st - s0 + 1);
      CK(cudaMemcpyAsync(nxt, seg + elems * (st - s0), state, cudaMemcpyDeviceToDevice, c->stream));
      rc = step_impl<real>(c, nxt, 1, nullptr, nullptr, &dtl[st], &al[6 * (size_t)st]);
      if (rc) return rc;
    }
    for (int st = s1 - 1; st >= s0; --st) {
      rc = sweep_step<real>(c, seg + elems * (st - s0), dtl[st], &al[6 * (size_t)st]);
      if (rc) return rc;
    }
  }
  return HYDRO_OK;
}

template <typename real>
static int sweep_impl(hydro_ctx* c, real* lam) {
  const int N = c->ck_nsteps, every = c->ck_every;
  std::vector<double> dtl(N), al(6 * (size_t)N);
  int got = 0;
  int rc = hydro_get_log(c, N, dtl.data(), al.data(), &got);
  if (rc) return rc;
  const size_t elems = (size_t)c->nf * c->cfg.nx * c->cfg.ny;
  const size_t state = elems * sizeof(real);
  // the cotangent stays padded for the whole sweep (copied in here, out at the end)
  if ((rc = ensure_adjoint_buffers(c))) return rc;
  if ((rc = copy_in<real>(c, static_cast<real*>(c->adj_nu[0]), lam))) return rc;
  c->adj_in = 0;
  auto finish = [&](int r) -> int {
    c->defer_status = false;
    if (r) return r;
    real* B[3] = {static_cast<real*>(c->adj_nu[0]), static_cast<real*>(c->adj_nu[1]), static_cast<real*>(c->adj_acc)};
    if ((r = copy_out<real>(c, lam, B[c->adj_in]))) return r;
    return read_status<real>(c, nullptr, nullptr);
  };
  if (c->ck_mode == 1) {  // binomial schedule from U^0
    real* slots = static_cast<real*>(c->rv_slots);
    const int nslots = c->rv_snapshots + 1;
    CK(cudaMemsetAsync(&scr<real>(c)->err, 0, sizeof(int), c->stream));
    c->defer_status = true;
    return finish(rv_reverse<real>(c, slots, nslots, slots + elems * (size_t)nslots, 0, 0, N, elems, dtl, al));
  }
  if (c->seg_cap < (size_t)every) {
    cudaFree(c->seg);
    c->seg = nullptr;
    c->seg_cap = 0;
    CK(cudaMalloc(&c->seg, state * every));
    c->seg_cap = every;
  }
  real* seg = static_cast<real*>(c->seg);
  const int nseg = (N + every - 1) / every;
  CK(cudaMemsetAsync(&scr<real>(c)->err, 0, sizeof(int), c->stream));
  c->defer_status = true;
  return finish(sweep_segments<real>(c, seg, nseg, every, N, elems, state, dtl, al));
}

int hydro_adjoint_sweep(hydro_ctx* c, void* lambda) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!lambda) return fail(c, HYDRO_EINVAL, "null lambda");
  if (c->ck_nsteps < 1 || (c->ck_mode == 0 && !c->ckpt) || (c->ck_mode == 1 && !c->rv_slots))
    return fail(c, HYDRO_ESTATE, "no checkpointed forward run to reverse");
  if (c->cfg.dtype == HYDRO_F64) return sweep_impl<double>(c, (double*)lambda);
  return sweep_impl<float>(c, (float*)lambda);
}

// ---- level-set reinitialisation (Sec. 2.2)

template <typename real>
static int reinit_impl(hydro_ctx* c, real* U) {
  const hydro_config& g = c->cfg;
  const long long n = (long long)g.nx * g.ny;
  if (!c->front) {
    // every cell pair can hold one front point: at most 2 n points
    const long long cap = 2 * n;
    if (cap > 0x7fffffffLL) return fail(c, HYDRO_EINVAL, "grid too large for the front point buffer");
    CK(cudaMalloc(&c->front, sizeof(real) * 2 * cap));
    CK(cudaMalloc(&c->front_count, sizeof(int)));
    c->front_cap = (int)cap;
  }
  Scratch<real>* s = scr<real>(c);
  CK(cudaMemsetAsync(&s->err, 0, sizeof(int), c->stream));
  const double dx = (g.x1 - g.x0) / g.nx, dy = (g.y1 - g.y0) / g.ny;
  int nl = 0;
  CK(launch_reinit<real>(U + 4 * n, g.nx, g.ny, g.nx, g.x0, g.y0, dx, dy, static_cast<real*>(c->front), c->front_cap,
                         c->front_count, &s->err, c->stream, &nl));
  c->launches += nl;
  return read_status<real>(c, nullptr, nullptr);
}

int hydro_reinit(hydro_ctx* c, void* U, int* npoints) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U) return fail(c, HYDRO_EINVAL, "null state");
  if (c->nf != 5) return fail(c, HYDRO_EINVAL, "reinitialisation needs the level-set field (nfields = 5)");
  rc = c->cfg.dtype == HYDRO_F64 ? reinit_impl<double>(c, (double*)U) : reinit_impl<float>(c, (float*)U);
  if (rc == HYDRO_OK && npoints) {
    cudaError_t e = cudaMemcpy(npoints, c->front_count, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "front count");
  }
  return rc;
}

// ---- self-gravity potential (Sec. 2.1) and exact sums

namespace {
struct PoissonDev {
  PoissonParams P;
  SorCtl ctl;
  ExactAcc acc;
  double sum_out;
};
struct PoissonHost {
  SorCtl ctl;
  int nonfinite;
  double mass, sum_out;
  int done[2];
};
}  // namespace

static int ensure_poisson(hydro_ctx* c) {
  if (c->pois) return HYDRO_OK;
  const size_t head = (sizeof(PoissonDev) + 255) / 256 * 256;
  const size_t arrays =
      sizeof(double) * (6 * (size_t)c->cfg.nx + (size_t)c->cfg.ny + (size_t)c->cfg.nx * (size_t)c->cfg.ny);
  CK(cudaMalloc(&c->pois, head + arrays));
  CK(cudaMallocHost(&c->pois_host, sizeof(PoissonHost)));
  for (cudaEvent_t& e : c->sor_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return HYDRO_OK;
}

static PoissonDev* pdev(hydro_ctx* c) { return static_cast<PoissonDev*>(c->pois); }
static PoissonHost* phost(hydro_ctx* c) { return static_cast<PoissonHost*>(c->pois_host); }

static int wait_event(hydro_ctx* c, cudaEvent_t ev) {
  const double limit = host_timeout_s();
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return HYDRO_OK;
    if (e != cudaErrorNotReady) return cuda_fail(c, e, "event wait");
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return fail(c, HYDRO_ETIMEOUT, "stream did not finish within HYDRO_TIMEOUT_S");
    std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
  }
}

static int ensure_sor_graph(hydro_ctx* c) {
  if (c->sor_graph) return HYDRO_OK;
  cudaGraph_t gr = nullptr;
  CK(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
  long long before = c->launches;
  int nl = 0;
  cudaError_t e1 = launch_sor_chunk(&pdev(c)->P, &pdev(c)->ctl, c->cfg.nx, c->cfg.ny, c->capture, &nl);
  cudaError_t e = cudaStreamEndCapture(c->capture, &gr);
  c->launches = before;  // captured, not launched
  if (e1 != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return cuda_fail(c, e1, "capture of the SOR sweeps");
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->sor_graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return HYDRO_OK;
}

template <typename T>
static int poisson_impl(hydro_ctx* c, const T* U, double G, double omega, double tol, int max_iters, double* phi,
                        int* iters, double* mass) {
  int rc = ensure_poisson(c);
  if (rc) return rc;
  const hydro_config& g = c->cfg;
  PoissonDev* d = pdev(c);
  double* arr = reinterpret_cast<double*>(static_cast<char*>(c->pois) + (sizeof(PoissonDev) + 255) / 256 * 256);
  PoissonParams hp{};
  hp.phi = phi;
  hp.rho = U;  // field 0 of the caller's state
  hp.nx = g.nx;
  hp.ny = g.ny;
  hp.zsym = g.bc[2] == HYDRO_BC_REFLECT ? 1 : 0;
  hp.max_iters = max_iters;
  hp.x0 = g.x0;
  hp.y0 = g.y0;
  hp.dr = (g.x1 - g.x0) / g.nx;
  hp.dz = (g.y1 - g.y0) / g.ny;
  hp.G = G;
  hp.omega = omega;
  hp.one_minus_omega = 1.0 - omega;
  hp.tol = tol;
  {
    int e2 = 0;
    const double m = std::frexp(tol, &e2);  // tol = m 2^e2, m in [1/2, 1)
    hp.tol_screen = std::isnormal(tol) && tol > 0.0 ? 1 : 0;
    hp.tol_exp = e2 - 1;
    hp.tol_mant = (float)(2.0 * m);
  }
  hp.four_pi_G = (4.0 * 3.14159265358979323846264338328) * G;
  hp.cE = arr;
  hp.cW = arr + g.nx;
  hp.cD = arr + 2 * g.nx;
  hp.gN = arr + 3 * g.nx;
  hp.gS = arr + 4 * g.nx;
  hp.gE = arr + 5 * g.nx;
  hp.cY = arr + 5 * g.nx + g.ny;
  hp.src = arr + 6 * g.nx + g.ny;
  CK(cudaMemcpyAsync(&d->P, &hp, sizeof(hp), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(&d->ctl, 0, sizeof(SorCtl), c->stream));
  int nl = 0;
  CK(launch_poisson_setup<T>(&d->P, &d->acc, (long long)g.nx * g.ny, g.nx, g.ny, c->stream, &nl));
  c->launches += nl;
  PoissonHost* h = phost(c);
  if (max_iters > 0) {
    rc = ensure_sor_graph(c);
    if (rc) return rc;
    const int nchunks = (int)(((long long)max_iters + SOR_CHUNK - 1) / SOR_CHUNK);
    for (int ch = 0; ch < nchunks; ++ch) {
      CK(cudaGraphLaunch(c->sor_graph, c->stream));
      c->launches += 2 * SOR_CHUNK + 1;
      if (tol > 0.0) {
        // read the done flag one chunk behind, so the GPU always has the next chunk queued
        CK(cudaMemcpyAsync(&h->done[ch & 1], &d->ctl.done, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaEventRecord(c->sor_ev[ch & 1], c->stream));
        if (ch >= 1) {
          rc = wait_event(c, c->sor_ev[(ch - 1) & 1]);
          if (rc) return rc;
          if (h->done[(ch - 1) & 1]) break;
        }
      }
    }
  }
  CK(cudaMemcpyAsync(&h->ctl, &d->ctl, sizeof(SorCtl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&h->nonfinite, &d->acc.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&h->mass, &d->P.mass, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  rc = wait_stream(c);
  if (rc) return rc;
  if (iters) *iters = h->ctl.done ? h->ctl.iters : max_iters;
  if (mass) *mass = h->mass;
  if (h->nonfinite) return fail(c, HYDRO_ENONPHYSICAL, "non-finite density in the mass sum");
  return HYDRO_OK;
}

int hydro_poisson(hydro_ctx* c, const void* U, double G, double omega, double tol, int max_iters, double* phi,
                  int* iters, double* mass) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !phi) return fail(c, HYDRO_EINVAL, "null state or potential");
  if (c->cfg.geometry != 1) return fail(c, HYDRO_EINVAL, "the Poisson solve is defined on an (r,z) grid (geometry 1)");
  if (!(omega > 0.0 && omega < 2.0)) return fail(c, HYDRO_EINVAL, "omega must lie in (0, 2)");
  if (max_iters < 0 || !std::isfinite(G) || std::isnan(tol)) return fail(c, HYDRO_EINVAL, "bad G, tol or max_iters");
  if ((c->cfg.nx + 1) / 2 > 0x7fffffff / 2 || (c->cfg.ny + SOR_BY - 1) / SOR_BY > 65535)
    return fail(c, HYDRO_EINVAL, "grid too tall for the SOR launch (ny <= 131070)");
  if ((long long)c->cfg.nx * c->cfg.ny > XS_MAX_TERMS) return fail(c, HYDRO_ESIZE, "more than 2^31 - 1 cells");
  if (c->cfg.dtype == HYDRO_F64)
    return poisson_impl<double>(c, static_cast<const double*>(U), G, omega, tol, max_iters, phi, iters, mass);
  return poisson_impl<float>(c, static_cast<const float*>(U), G, omega, tol, max_iters, phi, iters, mass);
}

int hydro_exact_sum(hydro_ctx* c, const double* x, long long n, double* out) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out || (n > 0 && !x) || n < 0) return fail(c, HYDRO_EINVAL, "null pointer or negative count");
  if (n > XS_MAX_TERMS) return fail(c, HYDRO_ESIZE, "more than 2^31 - 1 terms");
  rc = ensure_poisson(c);
  if (rc) return rc;
  PoissonDev* d = pdev(c);
  PoissonHost* h = phost(c);
  int nl = 0;
  CK(launch_exact_sum(x, n, &d->acc, &d->sum_out, c->stream, &nl));
  c->launches += nl;
  CK(cudaMemcpyAsync(&h->sum_out, &d->sum_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&h->nonfinite, &d->acc.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  rc = wait_stream(c);
  if (rc) return rc;
  *out = h->sum_out;
  if (h->nonfinite) return fail(c, HYDRO_ENONPHYSICAL, "a term is inf or NaN");
  return HYDRO_OK;
}

// ---- failure-path self-test

int hydro_wait_selftest(hydro_ctx* c, unsigned polls) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (polls == 0 || polls > (1u << 24)) return fail(c, HYDRO_EINVAL, "polls must be in 1 .. 2^24");
  int* err = c->cfg.dtype == HYDRO_F64 ? &scr<double>(c)->err : &scr<float>(c)->err;
  CK(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  CK(launch_wait_selftest(polls, err, c->stream));
  c->launches++;
  return c->cfg.dtype == HYDRO_F64 ? read_status<double>(c, nullptr, nullptr) : read_status<float>(c, nullptr, nullptr);
}

// ---- arithmetic peak probe

int hydro_fma_probe(hydro_ctx* c, int dtype, int iters, double* fma_per_s) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!fma_per_s || iters < 1 || (dtype != HYDRO_F32 && dtype != HYDRO_F64))
    return fail(c, HYDRO_EINVAL, "bad probe arguments");
  c->launches += 2;
  if (dtype == HYDRO_F64) CK(run_fma_probe<double>(iters, c->stream, c->num_sms, fma_per_s));
  else CK(run_fma_probe<float>(iters, c->stream, c->num_sms, fma_per_s));
  return HYDRO_OK;
}
