// Global Fourier amplitudes of a disk (paper, section on the gravitationally unstable
// disks, eq. of A_m(t)): A_m = |sum Sigma e^{i m phi}| / sum Sigma over the columns whose
// centre lies within R_f of the z axis, Sigma the column density (sum over z of rho h_z)
// and phi the polar angle of the column centre.
//
// One thread per column sums its rho in z order in FP64 (consecutive threads take
// consecutive x, so every load is coalesced), then adds Sigma, Sigma cos(m phi) and
// Sigma sin(m phi) for m = 1..m_max to its running sums, with cos / sin of m phi from the
// complex powers of (x + i y) / r.  Per-CTA partials and one folding block keep a fixed
// order (deterministic).  Geometry: column (i, j) is centred at
// ((i + 1/2 - nx/2) h_x, (j + 1/2 - ny/2) h_y); the grid is centred on the axis.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/ppml.h"
#include "ppml_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kModes = PPML_FOURIER_MAX_MODES;
constexpr int kSums = 2 * kModes + 1;  // Sigma, then (cos, sin) per mode
constexpr int kMaxBlocks = 1216;

// Warp then CTA sum of kSums values in a fixed shape; the result is valid in thread 0.
__device__ __forceinline__ void block_sum(double v[kSums], double (*sh)[kSums]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < kSums; q++) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int q = 0; q < kSums; q++) sh[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < kSums; q++) {
      double s = 0.0;
      for (int k = 0; k < kThreads / 32; k++) s += sh[k][q];
      v[q] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) fourier_kernel(const T* __restrict__ rho, int nx, int ny,
                                                           int nz, double hx, double hy, double hz,
                                                           double rf2, int m_max,
                                                           double* __restrict__ part) {
  double acc[kSums];
#pragma unroll
  for (int q = 0; q < kSums; q++) acc[q] = 0.0;
  const long long nxy = (long long)nx * ny;
  for (long long col = (long long)blockIdx.x * kThreads + threadIdx.x; col < nxy;
       col += (long long)gridDim.x * kThreads) {
    const int i = (int)(col % nx), j = (int)(col / nx);
    const double x = ((double)i + 0.5 - 0.5 * (double)nx) * hx;
    const double y = ((double)j + 0.5 - 0.5 * (double)ny) * hy;
    const double r2 = x * x + y * y;
    if (r2 > rf2) continue;
    double s = 0.0;
    for (int k = 0; k < nz; k++) s += (double)rho[col + nxy * k];
    s *= hz;
    acc[0] += s;
    const double r = sqrt(r2);
    const double c1 = r > 0.0 ? x / r : 1.0, s1 = r > 0.0 ? y / r : 0.0;  // phi(0, 0) = 0
    double cm = c1, sm = s1;
#pragma unroll
    for (int m = 1; m <= kModes; m++) {
      if (m <= m_max) {
        acc[2 * m - 1] += s * cm;
        acc[2 * m] += s * sm;
      }
      const double cn = cm * c1 - sm * s1;
      sm = sm * c1 + cm * s1;
      cm = cn;
    }
  }
  __shared__ double sh[kThreads / 32][kSums];
  block_sum(acc, sh);
  if (threadIdx.x == 0)
    for (int q = 0; q < kSums; q++) part[(size_t)blockIdx.x * kSums + q] = acc[q];
}

__global__ void __launch_bounds__(kThreads) fourier_fold_kernel(const double* __restrict__ part,
                                                                int nblk, double* __restrict__ out) {
  double acc[kSums];
#pragma unroll
  for (int q = 0; q < kSums; q++) acc[q] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads)
#pragma unroll
    for (int q = 0; q < kSums; q++) acc[q] += part[(size_t)b * kSums + q];
  __shared__ double sh[kThreads / 32][kSums];
  block_sum(acc, sh);
  if (threadIdx.x == 0)
    for (int q = 0; q < kSums; q++) out[q] = acc[q];
}

}  // namespace

struct FourierState {
  double* part;  // kMaxBlocks x kSums partials
  double* out;   // kSums folded sums
};

void ppml_fourier_free(FourierState* s) {
  if (!s) return;
  if (s->part) cudaFree(s->part);
  if (s->out) cudaFree(s->out);
  delete s;
}

int ppml_fourier_run(FourierState** state, const ppml_grid_desc* d, const void* rho, double r_f,
                     int m_max, double* a_out, cudaStream_t st) {
  if (!*state) {
    FourierState* s = new FourierState();
    if (cudaMalloc(&s->part, sizeof(double) * kSums * kMaxBlocks) != cudaSuccess ||
        cudaMalloc(&s->out, sizeof(double) * kSums) != cudaSuccess) {
      cudaGetLastError();
      ppml_fourier_free(s);
      return ppml_fail(PPML_E_NOMEM, "Fourier amplitude buffers");
    }
    *state = s;
  }
  FourierState* s = *state;
  const long long cols = (long long)d->nx * d->ny;
  long long nb = (cols + kThreads - 1) / kThreads;
  if (nb > kMaxBlocks) nb = kMaxBlocks;
  const double rf2 = r_f * r_f;
  if (d->dtype == PPML_F64)
    fourier_kernel<double><<<(int)nb, kThreads, 0, st>>>((const double*)rho, d->nx, d->ny, d->nz,
                                                         d->h[0], d->h[1], d->h[2], rf2, m_max,
                                                         s->part);
  else
    fourier_kernel<float><<<(int)nb, kThreads, 0, st>>>((const float*)rho, d->nx, d->ny, d->nz,
                                                        d->h[0], d->h[1], d->h[2], rf2, m_max,
                                                        s->part);
  int rc = ppml_check_launch("fourier_kernel");
  if (rc) return rc;
  fourier_fold_kernel<<<1, kThreads, 0, st>>>(s->part, (int)nb, s->out);
  if ((rc = ppml_check_launch("fourier_fold_kernel"))) return rc;
  double h[kSums];
  if (cudaMemcpyAsync(h, s->out, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "Fourier amplitudes: %s", cudaGetErrorString(cudaGetLastError()));
  if (!(h[0] > 0.0))
    return ppml_fail(PPML_E_INVAL, "no mass within r_f = %g of the axis", r_f);
  for (int m = 1; m <= m_max; m++) a_out[m - 1] = hypot(h[2 * m - 1], h[2 * m]) / h[0];
  return PPML_OK;
}
