// stage_inst.cuh -- host launchers of the stage kernel variants and the small kernels for one
// precision (included by stage_f32.cu / stage_f64.cu with HYDRO_REAL defined).
#pragma once
#include "adjoint_kernel.cuh"
#include "reinit_kernel.cuh"
#include "char_kernel.cuh"
#include "aux_kernels.cuh"

namespace hydro {

namespace {

template <typename real, int NF, int V>
struct VariantLaunch {
  static constexpr int TY = VARIANTS[V].ty, NT = VARIANTS[V].threads;
  static constexpr size_t SMEM = Tile<real, NF, TY, un_in_smem<real>(NT)>::BYTES;
  static cudaError_t configure() {
    static cudaError_t once = [] {
      cudaError_t e = cudaFuncSetAttribute(stage_kernel<real, NF, TY, NT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
      if (e != cudaSuccess) (void)cudaGetLastError();  // a variant too large for the device: not sticky
      return e;
    }();
    return once;
  }
  static cudaError_t launch(const GridParams<real>* m, const WorkItem* w, int nwork, const StageCtl& ctl, int grid,
                            cudaStream_t s) {
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    stage_kernel<real, NF, TY, NT><<<grid, NT, SMEM, s>>>(m, w, nwork, ctl);
    return cudaGetLastError();
  }
  static int occupancy() {
    if (configure() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<real, NF, TY, NT>, NT, SMEM) != cudaSuccess)
      return 0;
    return n;
  }
};

template <typename real, int NF>
cudaError_t launch_nf(int variant, const GridParams<real>* m, const WorkItem* w, int nwork, const StageCtl& ctl,
                      int grid, cudaStream_t s) {
  switch (variant) {
    case 0: return VariantLaunch<real, NF, 0>::launch(m, w, nwork, ctl, grid, s);
    case 1: return VariantLaunch<real, NF, 1>::launch(m, w, nwork, ctl, grid, s);
    case 2: return VariantLaunch<real, NF, 2>::launch(m, w, nwork, ctl, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename real, int NF>
int occ_nf(int variant) {
  switch (variant) {
    case 0: return VariantLaunch<real, NF, 0>::occupancy();
    case 1: return VariantLaunch<real, NF, 1>::occupancy();
    case 2: return VariantLaunch<real, NF, 2>::occupancy();
    default: return 0;
  }
}

template <typename real, int NF>
int smem_nf(int variant) {
  switch (variant) {
    case 0: return (int)VariantLaunch<real, NF, 0>::SMEM;
    case 1: return (int)VariantLaunch<real, NF, 1>::SMEM;
    case 2: return (int)VariantLaunch<real, NF, 2>::SMEM;
    default: return 0;
  }
}

}  // namespace

template <>
cudaError_t launch_stage<HYDRO_REAL>(int variant, int nfields, const GridParams<HYDRO_REAL>* m, const WorkItem* w,
                                     int nwork, const StageCtl& ctl, int grid, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  return nfields == 5 ? launch_nf<HYDRO_REAL, 5>(variant, m, w, nwork, ctl, grid, s)
                      : launch_nf<HYDRO_REAL, 4>(variant, m, w, nwork, ctl, grid, s);
}

template <>
int stage_smem_bytes<HYDRO_REAL>(int variant, int nfields) {
  return nfields == 5 ? smem_nf<HYDRO_REAL, 5>(variant) : smem_nf<HYDRO_REAL, 4>(variant);
}

template <>
int stage_ctas_per_sm<HYDRO_REAL>(int variant, int nfields) {
  return nfields == 5 ? occ_nf<HYDRO_REAL, 5>(variant) : occ_nf<HYDRO_REAL, 4>(variant);
}

template <>
cudaError_t launch_pack<HYDRO_REAL>(const HYDRO_REAL* U, const GridParams<HYDRO_REAL>& g, int nfields,
                                    HYDRO_REAL* alpha_slot, HYDRO_REAL* smax_slot, double* t_acc, double t0,
                                    cudaStream_t s) {
  int dev = 0, sms = 132;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long n = static_cast<long long>(g.nx) * g.ny;
  const long long want = (n + 255) / 256;
  const int grid = static_cast<int>(want < 8LL * sms ? want : 8LL * sms);
  if (nfields == 5)
    pack_kernel<HYDRO_REAL, 5><<<grid, 256, 0, s>>>(U, g, alpha_slot, smax_slot, t_acc, t0);
  else
    pack_kernel<HYDRO_REAL, 4><<<grid, 256, 0, s>>>(U, g, alpha_slot, smax_slot, t_acc, t0);
  return cudaGetLastError();
}

template <>
cudaError_t launch_set_frozen<HYDRO_REAL>(double* dt_slot, double dt, HYDRO_REAL* alpha_slots, const double* a,
                                          cudaStream_t s) {
  set_frozen_kernel<HYDRO_REAL><<<1, 32, 0, s>>>(dt_slot, dt, alpha_slots, a[0], a[1], a[2], a[3], a[4], a[5]);
  return cudaGetLastError();
}

template <>
cudaError_t launch_totals<HYDRO_REAL>(const HYDRO_REAL* U, int nx, int ny, int nfields, int geometry, double x0,
                                      double dx, double dy, double* partials, int nblocks, double* out,
                                      cudaStream_t s) {
  if (nfields == 5)
    totals_partial_kernel<HYDRO_REAL, 5><<<nblocks, 256, 0, s>>>(U, nx, ny, geometry, x0, dx, dy, partials);
  else
    totals_partial_kernel<HYDRO_REAL, 4><<<nblocks, 256, 0, s>>>(U, nx, ny, geometry, x0, dx, dy, partials);
  totals_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, nfields, out);
  return cudaGetLastError();
}

namespace {
// blocks per member of the batched pack and unpack: enough for the largest member, about 8 per SM in all
inline int batch_blocks(int n, long long max_cells) {
  int dev = 0, sms = 132;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (max_cells + 255) / 256, cap = (8LL * sms + n - 1) / n;
  return static_cast<int>(want < cap ? (want > 0 ? want : 1) : (cap > 0 ? cap : 1));
}
}  // namespace

template <>
cudaError_t launch_copy_state<HYDRO_REAL>(HYDRO_REAL* dst, const HYDRO_REAL* src, int nx, int ny, int nf, int pitch,
                                          long long fstride, bool to_padded, cudaStream_t s) {
  int dev = 0, sms = 132;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (static_cast<long long>(nx) * ny * nf + 255) / 256;
  const int grid = static_cast<int>(want < 8LL * sms ? want : 8LL * sms);
  copy_state_kernel<HYDRO_REAL><<<grid, 256, 0, s>>>(dst, src, nx, ny, nf, pitch, fstride, to_padded);
  return cudaGetLastError();
}

template <>
cudaError_t launch_batch_pack<HYDRO_REAL>(const GridParams<HYDRO_REAL>* P, const HYDRO_REAL* const* U,
                                          const double* t0, int n, int nfields, long long max_cells, cudaStream_t s) {
  const dim3 grid(batch_blocks(n, max_cells), n);
  if (nfields == 5)
    batch_pack_kernel<HYDRO_REAL, 5><<<grid, 256, 0, s>>>(P, U, t0);
  else
    batch_pack_kernel<HYDRO_REAL, 4><<<grid, 256, 0, s>>>(P, U, t0);
  return cudaGetLastError();
}

template <>
cudaError_t launch_batch_unpack<HYDRO_REAL>(const GridParams<HYDRO_REAL>* P, HYDRO_REAL* const* U, int n, int nfields,
                                            long long max_cells, cudaStream_t s) {
  const dim3 grid(batch_blocks(n, max_cells), n);
  if (nfields == 5)
    batch_unpack_kernel<HYDRO_REAL, 5><<<grid, 256, 0, s>>>(P, U);
  else
    batch_unpack_kernel<HYDRO_REAL, 4><<<grid, 256, 0, s>>>(P, U);
  return cudaGetLastError();
}

#if HYDRO_REAL_IS_FLOAT  // precision-independent: in one translation unit only
// Byte-wise copies between the members' scratch records (blockIdx.x = member) and one contiguous array:
// zero the first `bytes` of each (dst == null), or gather `bytes` of each into dst[m * bytes].
__global__ void __launch_bounds__(128) batch_scratch_kernel(void* const* __restrict__ scratch, int bytes,
                                                            unsigned char* __restrict__ dst) {
  unsigned char* s = static_cast<unsigned char*>(scratch[blockIdx.x]);
  for (int i = threadIdx.x; i < bytes; i += blockDim.x) {
    if (dst)
      dst[static_cast<long long>(blockIdx.x) * bytes + i] = s[i];
    else
      s[i] = 0;
  }
}

cudaError_t launch_batch_scratch(void* const* scratch, int n, int bytes, unsigned char* dst, cudaStream_t s) {
  batch_scratch_kernel<<<n, 128, 0, s>>>(scratch, bytes, dst);
  return cudaGetLastError();
}
#endif

template <>
cudaError_t launch_char_div<HYDRO_REAL>(const GridParams<HYDRO_REAL>* p_dev, int nx, int ny, cudaStream_t s) {
  constexpr int CY = CharTile<HYDRO_REAL>::CY;
  constexpr int SMEM = static_cast<int>(CharLayout<HYDRO_REAL>::BYTES);
  // persistent CTAs: as many as are resident at once (the dynamic shared memory and the registers decide)
  static const int resident = []() -> int {
    int d = 0, n = 0, per = 0;
    if (cudaFuncSetAttribute(char_div_kernel<HYDRO_REAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) !=
            cudaSuccess ||
        cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, char_div_kernel<HYDRO_REAL>, CHAR_THREADS, SMEM) !=
            cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    return n * per;
  }();
  if (resident < 1) return cudaErrorInvalidConfiguration;
  const int tiles_x = (nx + CX - 1) / CX, ntiles = tiles_x * ((ny + CY - 1) / CY);
  const int grid = ntiles < resident ? ntiles : resident;
  char_div_kernel<HYDRO_REAL><<<grid, CHAR_THREADS, SMEM, s>>>(p_dev, tiles_x, ntiles);
  return cudaGetLastError();
}

template <>
cudaError_t launch_reinit<HYDRO_REAL>(HYDRO_REAL* phi, int nx, int ny, int pitch, double x0, double y0, double dx,
                                      double dy, HYDRO_REAL* front, int capacity, int* count, int* err,
                                      cudaStream_t s, int* launches) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  front_kernel<HYDRO_REAL><<<dim3((nx + 255) / 256, ny), 256, 0, s>>>(phi, nx, ny, pitch, x0, y0, dx, dy, front,
                                                                       capacity, count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = static_cast<long long>(nx) * ny;
#if HYDRO_REAL_IS_FLOAT
  distance_kernel_x2<HYDRO_REAL><<<static_cast<unsigned>((n + 511) / 512), 256, 0, s>>>(
      phi, nx, ny, pitch, x0, y0, dx, dy, dx < dy ? dx : dy, front, capacity, count, err);
#else
  distance_kernel<HYDRO_REAL><<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
      phi, nx, ny, pitch, x0, y0, dx, dy, dx < dy ? dx : dy, front, capacity, count, err);
#endif
  if (launches) *launches += 2;
  return cudaGetLastError();
}

namespace {
// the line adjoint over the tiles of the padded grid (columns 1 .. nx+6, rows 0 .. ny+5) in TY-row tiles
template <int NF, int TY>
cudaError_t adj_line(const AdjParams<HYDRO_REAL>& P, cudaStream_t s) {
  using TL = ATile<HYDRO_REAL, NF, TY>;
  const int tiles_x = (P.nx + 6 + ATX - 1) / ATX, tiles_y = (P.ny + 6 + TY - 1) / TY;
  static const cudaError_t cfg = [] {
    cudaError_t r = cudaFuncSetAttribute(adj_line_kernel<HYDRO_REAL, NF, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::BYTES);
    if (r != cudaSuccess) (void)cudaGetLastError();
    return r;
  }();
  if (cfg != cudaSuccess) return cfg;
  adj_line_kernel<HYDRO_REAL, NF, TY><<<tiles_x * tiles_y, adj_threads<HYDRO_REAL, NF, TY>(), TL::BYTES, s>>>(P, tiles_x);
  return cudaGetLastError();
}

template <int NF>
cudaError_t adj_nf(const AdjParams<HYDRO_REAL>& P, cudaStream_t s, int* launches) {
  dim3 pg((P.nx + 255) / 256, P.ny);
  adj_point_kernel<HYDRO_REAL, NF><<<pg, 256, 0, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
#if HYDRO_REAL_IS_FLOAT
  // 32-row tiles (one CTA per SM) where the grid has at least one per SM: 45.1 -> 43.8 ms per 8192^2
  // adjoint step; smaller grids keep two CTAs of 16-row tiles per SM
  static const int sms = [] {
    int d = 0, n = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
      (void)cudaGetLastError();
      return 1 << 30;
    }
    return n;
  }();
  const long long tiles32 = (long long)((P.nx + 6 + ATX - 1) / ATX) * ((P.ny + 6 + 31) / 32);
  const bool rows32 = P.tile_rows == 32 || (P.tile_rows == 0 && tiles32 >= sms);
  e = rows32 ? adj_line<NF, 32>(P, s) : adj_line<NF, 16>(P, s);
#else
  e = adj_line<NF, 16>(P, s);
#endif
  if (e != cudaSuccess) return e;
  adj_blend_kernel<HYDRO_REAL, NF><<<pg, 256, 0, s>>>(P);
  if (launches) *launches += 3;
  return cudaGetLastError();
}
}  // namespace

template <>
cudaError_t launch_adjoint_stage<HYDRO_REAL>(const AdjParams<HYDRO_REAL>& P, int nfields, cudaStream_t s,
                                             int* launches) {
  return nfields == 5 ? adj_nf<5>(P, s, launches) : adj_nf<4>(P, s, launches);
}

}  // namespace hydro
