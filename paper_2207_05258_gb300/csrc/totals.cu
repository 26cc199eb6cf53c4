// Conserved totals sum_i U_c(x_i) dx (dy) in FP64 with a fixed summation
// order: one CTA per tile writes its partial sums (a fixed-shape tree), then
// one thread per instance adds its tiles' partials in tile order. No floating
// point atomics, so the result has the same bits on every call.
#include "hweno.h"
#include "internal.h"

namespace hweno {
namespace {

constexpr int kThreads = 128;

template <class Real>
__global__ void __launch_bounds__(kThreads) k_totals_partial(int m, int dim, int tile,
                                                             const Real* U,
                                                             const int* tile_inst,
                                                             const int* tile_start,
                                                             const int* inst_n,
                                                             const long long* inst_off, int nx,
                                                             int ny, double* partial) {
  __shared__ double red[kThreads];
  const int b = blockIdx.x;
  long long base, stride;  // first element of component 0 of this tile, component stride
  int np;
  if (dim == 1) {
    const int k = tile_inst[b], s = tile_start[b], n = inst_n[k];
    np = min(tile, n - s);
    base = inst_off[k] * m + s;
    stride = n;
  } else {
    const int tiles_x = (nx + kTileX2D - 1) / kTileX2D;
    const int j = b / tiles_x, i0 = (b % tiles_x) * kTileX2D;
    np = min(kTileX2D, nx - i0);
    base = (long long)j * nx + i0;
    stride = (long long)nx * ny;
  }
  for (int c = 0; c < m; ++c) {
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) v += (double)U[base + c * stride + i];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)b * m + c] = red[0];
    __syncthreads();
  }
}

// One thread per instance; the tiles of an instance are consecutive.
__global__ void k_totals_final(int m, int batch, int ntiles, const int* tile_inst,
                               const double* partial, double cell, const double* inst_dx,
                               double* totals) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= batch) return;
  // first tile of instance k (tile table sorted by instance)
  int lo = 0, hi = ntiles;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (tile_inst[mid] < k) lo = mid + 1; else hi = mid;
  }
  const double h = inst_dx ? inst_dx[k] : cell;
  for (int c = 0; c < m; ++c) {
    double s = 0.0;
    for (int b = lo; b < ntiles && tile_inst[b] == k; ++b) s += partial[(long long)b * m + c];
    totals[k * m + c] = s * h;
  }
}

__global__ void k_totals_final_2d(int m, int ntiles, const double* partial, double cell,
                                  double* totals) {
  const int c = threadIdx.x;
  if (c >= m) return;
  double s = 0.0;
  for (int b = 0; b < ntiles; ++b) s += partial[(long long)b * m + c];
  totals[c] = s * cell;
}

}  // namespace

cudaError_t launch_totals(int m, bool fp32, int dim, const void* U, int ntiles, int tile,
                          const int* tile_inst, const int* tile_start, const int* inst_n,
                          const long long* inst_off, int batch, int nx, int ny, double cell,
                          const double* inst_dx, double* partial, double* totals,
                          cudaStream_t s) {
  if (fp32)
    k_totals_partial<float><<<ntiles, kThreads, 0, s>>>(m, dim, tile, static_cast<const float*>(U),
                                                        tile_inst, tile_start, inst_n, inst_off,
                                                        nx, ny, partial);
  else
    k_totals_partial<double><<<ntiles, kThreads, 0, s>>>(m, dim, tile, static_cast<const double*>(U),
                                                         tile_inst, tile_start, inst_n,
                                                         inst_off, nx, ny, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (dim == 1)
    k_totals_final<<<(batch + 127) / 128, 128, 0, s>>>(m, batch, ntiles, tile_inst, partial, cell,
                                                        inst_dx, totals);
  else
    k_totals_final_2d<<<1, 32, 0, s>>>(m, ntiles, partial, cell, totals);
  return cudaGetLastError();
}

}  // namespace hweno
