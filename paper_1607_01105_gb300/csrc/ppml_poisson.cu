// Isolated-boundary Poisson solve of the paper's Sec. "The Poisson solver" (Stages 1-3 with
// the 27-point stencil, eq. stencil27point).
//
// Stage 1: the monopole and quadrupole moments of the cell masses about the coordinate
// centre (a deterministic FP64 reduction) give the potential on the shell of cells just
// outside the grid (MacCullagh's formula, with its factor 1/2); the shell values that enter
// the stencil of a boundary cell are moved to the right-hand side.  Stages 2-3: with
// Dirichlet data on the shell the 27-point operator is diagonal in the sine basis
// sin(pi j (i + 1) / (N + 1)), j = 1..N, so the exponential transform the paper prints is
// replaced by a type-I sine transform along each axis (odd extension to 2 (N + 1) points and
// a batched real-to-complex cuFFT), the amplitudes are divided by the operator's eigenvalue
// 6 (prod_a (1 - (2/3) sin^2(pi j_a / (2 (N_a + 1)))) - 1), and the same sine transform,
// scaled by prod_a 2 / (N_a + 1), brings the potential back.  The right-hand side is
// 4 pi G h^2 (rho + D7 rho / 12) (D7 the 7-point second difference, rho = 0 outside), which
// makes the 27-point solve fourth-order accurate as the paper states; the printed
// 4 pi G h^2 rho (second order) is available with PPML_POISSON_PRINTED_RHS.
//
// Geometry: cell (i, j, k) has its centre at ((i + 1/2 - nx/2) h, (j + 1/2 - ny/2) h,
// (k + 1/2 - nz/2) h), i.e. the grid is centred on the origin of the expansion.
//
// The potential array doubles as the work array of the transforms; the odd extension and
// the half spectrum live in buffers kept by the solver state between calls.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>

#include <vector>

#include "../../include/ppml.h"
#include "ppml_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMoments = 7;  // M, I_x, I_y, I_z, I_xy, I_xz, I_yz
constexpr int kMaxMomentBlocks = 1216;  // 8 per SM on 152 SMs

struct Dims {
  int n[3];
  long long nxy, ncell;
};

__device__ __forceinline__ double centre(int i, int n, double h) {
  return ((double)i + 0.5 - 0.5 * (double)n) * h;
}

// Stage 1a: per-block FP64 partial moments of the masses rho h^3, fixed block count and a
// fixed-shape tree, so the result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(kThreads) moment_kernel(const T* __restrict__ rho, Dims D,
                                                          double h, double* __restrict__ part) {
  double acc[kMoments] = {0, 0, 0, 0, 0, 0, 0};
  const double vol = h * h * h;
  for (long long idx = (long long)blockIdx.x * kThreads + threadIdx.x; idx < D.ncell;
       idx += (long long)gridDim.x * kThreads) {
    const int i = (int)(idx % D.n[0]);
    const long long r = idx / D.n[0];
    const int j = (int)(r % D.n[1]), k = (int)(r / D.n[1]);
    const double x = centre(i, D.n[0], h), y = centre(j, D.n[1], h), z = centre(k, D.n[2], h);
    const double m = (double)rho[idx] * vol;
    acc[0] += m;
    acc[1] += (z * z + y * y) * m;
    acc[2] += (x * x + z * z) * m;
    acc[3] += (x * x + y * y) * m;
    acc[4] += x * y * m;
    acc[5] += x * z * m;
    acc[6] += y * z * m;
  }
  __shared__ double s[kMoments][kThreads];
#pragma unroll
  for (int q = 0; q < kMoments; q++) s[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < kMoments; q++) s[q][threadIdx.x] += s[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kMoments) part[(size_t)blockIdx.x * kMoments + threadIdx.x] = s[threadIdx.x][0];
}

// Stage 1b: one block folds the partials in a fixed order.
__global__ void __launch_bounds__(kThreads) moment_final_kernel(const double* __restrict__ part,
                                                                int nblk, double* __restrict__ mom) {
  __shared__ double s[kMoments][kThreads];
  double acc[kMoments] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += kThreads)
#pragma unroll
    for (int q = 0; q < kMoments; q++) acc[q] += part[(size_t)b * kMoments + q];
#pragma unroll
  for (int q = 0; q < kMoments; q++) s[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < kMoments; q++) s[q][threadIdx.x] += s[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kMoments) mom[threadIdx.x] = s[threadIdx.x][0];
}

// Monopole + quadrupole potential at (x, y, z) (MacCullagh's formula).
__device__ double shell_potential(const double* __restrict__ mom, double x, double y, double z,
                                  double G) {
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  const double I0 = ((x * x * mom[1] + y * y * mom[2] + z * z * mom[3]) -
                     2.0 * (x * y * mom[4] + x * z * mom[5] + y * z * mom[6])) /
                    r2;
  return -G * mom[0] / r - 0.5 * G * (mom[1] + mom[2] + mom[3] - 3.0 * I0) / (r2 * r);
}

// Right-hand side: 4 pi G h^2 (rho [+ D7 rho / 12]) minus the stencil weights times the
// shell values next to boundary cells.  Written into the potential array (the work array).
template <typename T>
__global__ void __launch_bounds__(kThreads) rhs_kernel(const T* __restrict__ rho, T* __restrict__ out,
                                                       Dims D, double h, double G,
                                                       const double* __restrict__ mom, int printed) {
  const double c = 4.0 * M_PI * G * h * h;
  for (long long idx = (long long)blockIdx.x * kThreads + threadIdx.x; idx < D.ncell;
       idx += (long long)gridDim.x * kThreads) {
    const int i = (int)(idx % D.n[0]);
    const long long r = idx / D.n[0];
    const int j = (int)(r % D.n[1]), k = (int)(r / D.n[1]);
    const double rc = (double)rho[idx];
    double src = rc;
    if (!printed) {
      double lap = -6.0 * rc;
      if (i > 0) lap += (double)rho[idx - 1];
      if (i < D.n[0] - 1) lap += (double)rho[idx + 1];
      if (j > 0) lap += (double)rho[idx - D.n[0]];
      if (j < D.n[1] - 1) lap += (double)rho[idx + D.n[0]];
      if (k > 0) lap += (double)rho[idx - D.nxy];
      if (k < D.n[2] - 1) lap += (double)rho[idx + D.nxy];
      src = rc + lap / 12.0;
    }
    double v = c * src;
    const bool edge = i == 0 || j == 0 || k == 0 || i == D.n[0] - 1 || j == D.n[1] - 1 ||
                      k == D.n[2] - 1;
    if (edge) {
      for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
          for (int dx = -1; dx <= 1; dx++) {
            const int ii = i + dx, jj = j + dy, kk = k + dz;
            const bool outside = ii < 0 || jj < 0 || kk < 0 || ii >= D.n[0] || jj >= D.n[1] ||
                                 kk >= D.n[2];
            if (!outside) continue;
            const int nnz = (dx != 0) + (dy != 0) + (dz != 0);
            const double w = nnz == 1 ? 4.0 / 9.0 : (nnz == 2 ? 1.0 / 9.0 : 1.0 / 36.0);
            v -= w * shell_potential(mom, centre(ii, D.n[0], h), centre(jj, D.n[1], h),
                                     centre(kk, D.n[2], h), G);
          }
    }
    out[idx] = (T)v;
  }
}

// Odd extension of every line along `axis` to M = 2 (N + 1) points:
// (0, w_0 .. w_{N-1}, 0, -w_{N-1} .. -w_0).  Layout of the extension: axis 0 line-major
// (line * M + p); axes 1 and 2 position-major (p * B + b), b the line's index over the
// other two axes in memory order, so both the gather and the store are coalesced.
template <typename T>
__global__ void __launch_bounds__(kThreads) dst_pack_kernel(const T* __restrict__ w, T* __restrict__ ext,
                                                            Dims D, int axis) {
  const int N = D.n[axis];
  const int M = 2 * (N + 1);
  const long long B = D.ncell / N;
  const long long total = (long long)M * B;
  for (long long idx = (long long)blockIdx.x * kThreads + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * kThreads) {
    long long line;
    int p;
    if (axis == 0) {
      line = idx / M;
      p = (int)(idx % M);
    } else {
      p = (int)(idx / B);
      line = idx % B;
    }
    T v = T(0);
    if (p != 0 && p != N + 1) {
      const int q = p <= N ? p - 1 : 2 * N + 1 - p;  // position along the axis, 0..N-1
      long long src;
      if (axis == 0)
        src = line * D.n[0] + q;
      else if (axis == 1)
        src = (line / D.n[0]) * D.nxy + (long long)q * D.n[0] + line % D.n[0];
      else
        src = (long long)q * D.nxy + line;
      v = p <= N ? w[src] : -w[src];
    }
    ext[idx] = v;
  }
}

// Sine amplitudes back into the work array: S_k = -Im(Y_k) / 2, k = q + 1.
template <typename T>
__global__ void __launch_bounds__(kThreads) dst_unpack_kernel(const T* __restrict__ spec,
                                                              T* __restrict__ w, Dims D, int axis) {
  const int N = D.n[axis];
  const long long B = D.ncell / N;
  const long long half = N + 2;  // M / 2 + 1 complex values per line
  for (long long idx = (long long)blockIdx.x * kThreads + threadIdx.x; idx < D.ncell;
       idx += (long long)gridDim.x * kThreads) {
    const int i = (int)(idx % D.n[0]);
    const long long r = idx / D.n[0];
    const int j = (int)(r % D.n[1]), k = (int)(r / D.n[1]);
    long long ci;
    if (axis == 0)
      ci = r * half + (i + 1);
    else if (axis == 1)
      ci = (long long)(j + 1) * B + (long long)k * D.n[0] + i;
    else
      ci = (long long)(k + 1) * B + (long long)j * D.n[0] + i;
    w[idx] = (T)(-0.5 * (double)spec[2 * ci + 1]);
  }
}

// Divide the sine amplitudes by the eigenvalue 6 (prod - 1), with the inverse transform's
// scale prod_a 2 / (N_a + 1) folded in.
template <typename T>
__global__ void __launch_bounds__(kThreads) iso_symbol_kernel(T* __restrict__ w, Dims D,
                                                              const double* __restrict__ tab,
                                                              double scale) {
  const double* tx = tab;
  const double* ty = tx + D.n[0];
  const double* tz = ty + D.n[1];
  for (long long idx = (long long)blockIdx.x * kThreads + threadIdx.x; idx < D.ncell;
       idx += (long long)gridDim.x * kThreads) {
    const int i = (int)(idx % D.n[0]);
    const long long r = idx / D.n[0];
    const int j = (int)(r % D.n[1]), k = (int)(r / D.n[1]);
    const double lam = 6.0 * (tz[k] * ty[j] * tx[i] - 1.0);
    w[idx] = (T)((double)w[idx] * (scale / lam));
  }
}

int blocks_for(long long n) {
  const long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < 152LL * 16 ? (b > 0 ? b : 1) : 152LL * 16);
}

}  // namespace

struct PoissonIso {
  int n[3];
  int dtype;
  cufftHandle plan[3];
  int nplans;
  void* ext;
  void* spec;
  double* part;
  double* mom;
  double* tab;
};

void ppml_iso_free(PoissonIso* s) {
  if (!s) return;
  for (int a = 0; a < s->nplans; a++) cufftDestroy(s->plan[a]);
  if (s->ext) cudaFree(s->ext);
  if (s->spec) cudaFree(s->spec);
  if (s->part) cudaFree(s->part);
  if (s->mom) cudaFree(s->mom);
  if (s->tab) cudaFree(s->tab);
  delete s;
}

static int iso_create(const ppml_grid_desc* d, PoissonIso** out) {
  PoissonIso* s = new PoissonIso();
  s->n[0] = d->nx;
  s->n[1] = d->ny;
  s->n[2] = d->nz;
  s->dtype = d->dtype;
  const bool f64 = d->dtype == PPML_F64;
  const size_t elt = f64 ? sizeof(double) : sizeof(float);
  const long long ncell = (long long)d->nx * d->ny * d->nz;
  size_t ext_n = 0, spec_n = 0;
  for (int a = 0; a < 3; a++) {
    const long long N = s->n[a], B = ncell / N;
    if ((size_t)(2 * (N + 1) * B) > ext_n) ext_n = (size_t)(2 * (N + 1) * B);
    if ((size_t)((N + 2) * B) > spec_n) spec_n = (size_t)((N + 2) * B);
  }
  if (cudaMalloc(&s->ext, ext_n * elt) != cudaSuccess ||
      cudaMalloc(&s->spec, spec_n * 2 * elt) != cudaSuccess ||
      cudaMalloc(&s->part, sizeof(double) * kMoments * kMaxMomentBlocks) != cudaSuccess ||
      cudaMalloc(&s->mom, sizeof(double) * kMoments) != cudaSuccess ||
      cudaMalloc(&s->tab, sizeof(double) * (size_t)(s->n[0] + s->n[1] + s->n[2])) != cudaSuccess) {
    cudaGetLastError();
    ppml_iso_free(s);
    return ppml_fail(PPML_E_NOMEM, "isolated Poisson buffers (%zu + %zu elements)", ext_n,
                     2 * spec_n);
  }
  std::vector<double> tab;
  for (int a = 0; a < 3; a++)
    for (int q = 0; q < s->n[a]; q++) {
      const double sn = sin(M_PI * (double)(q + 1) / (2.0 * (double)(s->n[a] + 1)));
      tab.push_back(1.0 - (2.0 / 3.0) * sn * sn);
    }
  if (cudaMemcpy(s->tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    ppml_iso_free(s);
    return ppml_fail(PPML_E_CUDA, "isolated Poisson tables: %s",
                     cudaGetErrorString(cudaGetLastError()));
  }
  for (int a = 0; a < 3; a++) {
    int M = 2 * (s->n[a] + 1);
    int inembed[1] = {M}, onembed[1] = {M / 2 + 1};
    const int B = (int)(ncell / s->n[a]);
    const int istride = a == 0 ? 1 : B, idist = a == 0 ? M : 1;
    const int ostride = a == 0 ? 1 : B, odist = a == 0 ? M / 2 + 1 : 1;
    if (cufftPlanMany(&s->plan[a], 1, &M, inembed, istride, idist, onembed, ostride, odist,
                      f64 ? CUFFT_D2Z : CUFFT_R2C, B) != CUFFT_SUCCESS) {
      ppml_iso_free(s);
      return ppml_fail(PPML_E_CUDA, "cufftPlanMany for the sine transform along axis %d", a);
    }
    s->nplans = a + 1;
  }
  *out = s;
  return PPML_OK;
}

template <typename T>
static int iso_run(PoissonIso* s, const T* rho, T* phi, double h, double G, int printed,
                   cudaStream_t st) {
  Dims D;
  for (int a = 0; a < 3; a++) D.n[a] = s->n[a];
  D.nxy = (long long)D.n[0] * D.n[1];
  D.ncell = D.nxy * D.n[2];
  const int nb = blocks_for(D.ncell) < kMaxMomentBlocks ? blocks_for(D.ncell) : kMaxMomentBlocks;
  moment_kernel<T><<<nb, kThreads, 0, st>>>(rho, D, h, s->part);
  int rc = ppml_check_launch("moment_kernel");
  if (rc) return rc;
  moment_final_kernel<<<1, kThreads, 0, st>>>(s->part, nb, s->mom);
  if ((rc = ppml_check_launch("moment_final_kernel"))) return rc;
  rhs_kernel<T><<<blocks_for(D.ncell), kThreads, 0, st>>>(rho, phi, D, h, G, s->mom, printed);
  if ((rc = ppml_check_launch("rhs_kernel"))) return rc;
  double scale = 1.0;
  for (int a = 0; a < 3; a++) scale *= 2.0 / (double)(D.n[a] + 1);
  for (int pass = 0; pass < 2; pass++) {
    for (int a = 0; a < 3; a++) {
      const long long total = 2LL * (D.n[a] + 1) * (D.ncell / D.n[a]);
      dst_pack_kernel<T><<<blocks_for(total), kThreads, 0, st>>>(phi, (T*)s->ext, D, a);
      if ((rc = ppml_check_launch("dst_pack_kernel"))) return rc;
      if (cufftSetStream(s->plan[a], st) != CUFFT_SUCCESS)
        return ppml_fail(PPML_E_CUDA, "cufftSetStream failed");
      cufftResult r;
      if (sizeof(T) == sizeof(double))
        r = cufftExecD2Z(s->plan[a], (cufftDoubleReal*)s->ext, (cufftDoubleComplex*)s->spec);
      else
        r = cufftExecR2C(s->plan[a], (cufftReal*)s->ext, (cufftComplex*)s->spec);
      if (r != CUFFT_SUCCESS) return ppml_fail(PPML_E_CUDA, "cuFFT sine transform failed (%d)", (int)r);
      dst_unpack_kernel<T><<<blocks_for(D.ncell), kThreads, 0, st>>>((const T*)s->spec, phi, D, a);
      if ((rc = ppml_check_launch("dst_unpack_kernel"))) return rc;
    }
    if (pass == 0) {
      iso_symbol_kernel<T><<<blocks_for(D.ncell), kThreads, 0, st>>>(phi, D, s->tab, scale);
      if ((rc = ppml_check_launch("iso_symbol_kernel"))) return rc;
    }
  }
  return PPML_OK;
}

int ppml_iso_solve(PoissonIso** state, const ppml_grid_desc* d, const void* rho, void* phi,
                   double G, unsigned flags, cudaStream_t st) {
  if (!*state) {
    int rc = iso_create(d, state);
    if (rc) return rc;
  }
  PoissonIso* s = *state;
  const int printed = (flags & PPML_POISSON_PRINTED_RHS) != 0;
  if (d->dtype == PPML_F64)
    return iso_run<double>(s, (const double*)rho, (double*)phi, d->h[0], G, printed, st);
  return iso_run<float>(s, (const float*)rho, (float*)phi, d->h[0], G, printed, st);
}
