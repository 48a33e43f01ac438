// Definitions of the launchers for one precision PPML_REAL (included by
// ppml_kern_f32.cu / ppml_kern_f64.cu).
#include "../../include/ppml.h"
#include "ppml_internal.h"
#include "ppml_launch.h"

namespace ppml {

namespace {
// CTAs per SM the march kernels are compiled for (register budget per thread)
template <typename T>
struct MinBlocks;
template <>
struct MinBlocks<float> {
  static constexpr int value = 2;
};
template <>
struct MinBlocks<double> {
  static constexpr int value = 1;
};
}  // namespace

// Double-float states (low parts of rho, m, rho E) exist only in the FP32 path.
constexpr bool kHasDF = sizeof(PPML_REAL) == 4;

template <bool DF, bool INF>
cudaError_t set_stage_smem_one() {
  constexpr int MB = MinBlocks<PPML_REAL>::value;
  cudaError_t e = cudaFuncSetAttribute(lagrangian_tile<PPML_REAL, MB, DF, INF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(LagTileSmem<PPML_REAL>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eulerian_tile<PPML_REAL, MB, DF, INF>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EulTileSmem<PPML_REAL>));
  return e;
}
template <bool DF>
cudaError_t set_stage_smem() {
  cudaError_t e = set_stage_smem_one<DF, false>();
  if (e == cudaSuccess) e = set_stage_smem_one<DF, true>();
  return e;
}

template <>
int prepare_kernels<PPML_REAL>() {
  cudaError_t e = set_stage_smem<false>();
  if (e == cudaSuccess && kHasDF) e = set_stage_smem<kHasDF>();
  if (e != cudaSuccess) return ppml_fail(PPML_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  return PPML_OK;
}

template <>
int launch_eulerian<PPML_REAL>(const MarchArgs<PPML_REAL>& A, int nblk, cudaStream_t st) {
  constexpr int MB = MinBlocks<PPML_REAL>::value;
  constexpr size_t SM = sizeof(EulTileSmem<PPML_REAL>);
  const bool df = kHasDF && A.outlo[1];
  if (A.any_inflow) {
    if (df)
      eulerian_tile<PPML_REAL, MB, kHasDF, true><<<nblk, TN, SM, st>>>(A);
    else
      eulerian_tile<PPML_REAL, MB, false, true><<<nblk, TN, SM, st>>>(A);
  } else if (df) {
    eulerian_tile<PPML_REAL, MB, kHasDF, false><<<nblk, TN, SM, st>>>(A);
  } else {
    eulerian_tile<PPML_REAL, MB, false, false><<<nblk, TN, SM, st>>>(A);
  }
  return ppml_check_launch("eulerian_tile");
}

template <>
int launch_lagrangian<PPML_REAL>(const MarchArgs<PPML_REAL>& A, int nblk, cudaStream_t st) {
  constexpr int MB = MinBlocks<PPML_REAL>::value;
  constexpr size_t SM = sizeof(LagTileSmem<PPML_REAL>);
  const bool df = kHasDF && A.outlo[0];
  if (A.any_inflow) {
    if (df)
      lagrangian_tile<PPML_REAL, MB, kHasDF, true><<<nblk, TN, SM, st>>>(A);
    else
      lagrangian_tile<PPML_REAL, MB, false, true><<<nblk, TN, SM, st>>>(A);
  } else if (df) {
    lagrangian_tile<PPML_REAL, MB, kHasDF, false><<<nblk, TN, SM, st>>>(A);
  } else {
    lagrangian_tile<PPML_REAL, MB, false, false><<<nblk, TN, SM, st>>>(A);
  }
  return ppml_check_launch("lagrangian_tile");
}

template <>
int launch_diag<PPML_REAL>(const MarchArgs<PPML_REAL>& A, int nblk, cudaStream_t st) {
  diag_kernel<PPML_REAL><<<nblk, NT, 0, st>>>(A);
  return ppml_check_launch("diag_kernel");
}

namespace {
// Multiply the half spectrum (R2C layout: kx in [0, nx/2], ky, kz) by the inverse symbol of
// the 27-point stencil; tables hold 1 - (2/3) sin^2(pi k / N) per axis.
template <typename T>
__global__ void poisson_symbol_kernel(T* spec, const double* __restrict__ tx,
                                      const double* __restrict__ ty,
                                      const double* __restrict__ tz, int mx, int ny, int nz,
                                      double coef) {
  const long long n = (long long)mx * ny * nz;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(idx % mx);
    const long long r = idx / mx;
    const int ky = (int)(r % ny), kz = (int)(r / ny);
    const double den = 1.0 - tz[kz] * ty[ky] * tx[kx];
    const double f = idx == 0 ? 0.0 : coef / den;
    spec[2 * idx] = (T)(spec[2 * idx] * f);
    spec[2 * idx + 1] = (T)(spec[2 * idx + 1] * f);
  }
}
}  // namespace

template <>
int launch_poisson_symbol<PPML_REAL>(void* spec, const double* tx, const double* ty,
                                     const double* tz, int mx, int ny, int nz, double coef,
                                     cudaStream_t st) {
  const long long n = (long long)mx * ny * nz;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  poisson_symbol_kernel<PPML_REAL><<<blocks, 256, 0, st>>>((PPML_REAL*)spec, tx, ty, tz, mx, ny, nz,
                                                           coef);
  return ppml_check_launch("poisson_symbol_kernel");
}

namespace {
// Opt-in shared memory of a kernel, raised once to the largest size launched so far.
template <typename K>
int raise_smem(K kernel, size_t smem, size_t& configured) {
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    configured = smem;
  }
  return PPML_OK;
}

template <int NT, bool DF>
int launch_batch_ntd(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                     BatchLo<PPML_REAL> lo, InstDev* inst, const int* order, double gamma,
                     double cfl, int max_steps, int nmax, int ninst, size_t smem,
                     cudaStream_t st) {
  static size_t configured = 0;
  int rc = raise_smem(batch_kernel<PPML_REAL, NT, DF>, smem, configured);
  if (rc) return rc;
  batch_kernel<PPML_REAL, NT, DF><<<ninst, NT, smem, st>>>(rho, m, en, ei, lo, inst, order, gamma,
                                                           cfl, max_steps, nmax);
  return ppml_check_launch("batch_kernel");
}

template <int NT, bool DF>
int launch_cluster_ntd(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                       BatchLo<PPML_REAL> lo, InstDev* inst, const int2* items, double gamma,
                       double cfl, int max_steps, int nlmax, int nmax, int nitems, size_t smem,
                       cudaStream_t st) {
  static size_t configured = 0;
  int rc = raise_smem(batch_cluster_kernel<PPML_REAL, NT, DF>, smem, configured);
  if (rc) return rc;
  batch_cluster_kernel<PPML_REAL, NT, DF><<<2 * nitems, NT, smem, st>>>(
      rho, m, en, ei, lo, inst, items, gamma, cfl, max_steps, nlmax, nmax);
  return ppml_check_launch("batch_cluster_kernel");
}

// double-float launches (low parts given) exist only in FP32
template <int NT>
int launch_batch_nt(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                    BatchLo<PPML_REAL> lo, InstDev* inst, const int* order, double gamma,
                    double cfl, int max_steps, int nmax, int ninst, size_t smem, cudaStream_t st) {
  if (kHasDF && lo.p[0])
    return launch_batch_ntd<NT, kHasDF>(rho, m, en, ei, lo, inst, order, gamma, cfl, max_steps,
                                        nmax, ninst, smem, st);
  return launch_batch_ntd<NT, false>(rho, m, en, ei, lo, inst, order, gamma, cfl, max_steps, nmax,
                                     ninst, smem, st);
}

template <int NT>
int launch_cluster_nt(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                      BatchLo<PPML_REAL> lo, InstDev* inst, const int2* items, double gamma,
                      double cfl, int max_steps, int nlmax, int nmax, int nitems, size_t smem,
                      cudaStream_t st) {
  if (kHasDF && lo.p[0])
    return launch_cluster_ntd<NT, kHasDF>(rho, m, en, ei, lo, inst, items, gamma, cfl, max_steps,
                                          nlmax, nmax, nitems, smem, st);
  return launch_cluster_ntd<NT, false>(rho, m, en, ei, lo, inst, items, gamma, cfl, max_steps,
                                       nlmax, nmax, nitems, smem, st);
}
}  // namespace

template <>
int launch_batch_vacuum<PPML_REAL>(const PPML_REAL* rho, InstDev* inst, int ninst,
                                   cudaStream_t st) {
  // vacuum thresholds of instances not yet started (no-op for the others)
  batch_vacuum_kernel<PPML_REAL><<<ninst, 256, 0, st>>>(rho, inst);
  return ppml_check_launch("batch_vacuum_kernel");
}

template <>
int launch_batch_cluster<PPML_REAL>(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                                    BatchLo<PPML_REAL> lo, InstDev* inst, const int2* items,
                                    double gamma, double cfl, int max_steps, int nlmax, int nmax,
                                    int nitems, size_t smem, int threads, cudaStream_t st) {
  switch (threads) {
    case 256:
      return launch_cluster_nt<256>(rho, m, en, ei, lo, inst, items, gamma, cfl, max_steps, nlmax,
                                    nmax, nitems, smem, st);
    case 512:
      return launch_cluster_nt<512>(rho, m, en, ei, lo, inst, items, gamma, cfl, max_steps, nlmax,
                                    nmax, nitems, smem, st);
    case 1024:
      return launch_cluster_nt<1024>(rho, m, en, ei, lo, inst, items, gamma, cfl, max_steps, nlmax,
                                     nmax, nitems, smem, st);
    default:
      return ppml_fail(PPML_E_INVAL, "batch CTA size %d is not 256, 512 or 1024", threads);
  }
}

template <>
int launch_batch<PPML_REAL>(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                            BatchLo<PPML_REAL> lo, InstDev* inst, const int* order, double gamma,
                            double cfl, int max_steps, int nmax, int ninst, size_t smem,
                            int threads, cudaStream_t st) {
  switch (threads) {
    case 256:
      return launch_batch_nt<256>(rho, m, en, ei, lo, inst, order, gamma, cfl, max_steps, nmax, ninst,
                                  smem, st);
    case 512:
      return launch_batch_nt<512>(rho, m, en, ei, lo, inst, order, gamma, cfl, max_steps, nmax, ninst,
                                  smem, st);
    case 1024:
      return launch_batch_nt<1024>(rho, m, en, ei, lo, inst, order, gamma, cfl, max_steps, nmax,
                                   ninst, smem, st);
    default:
      return ppml_fail(PPML_E_INVAL, "batch CTA size %d is not 256, 512 or 1024", threads);
  }
}

}  // namespace ppml
