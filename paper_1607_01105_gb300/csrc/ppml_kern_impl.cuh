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

template <>
int prepare_kernels<PPML_REAL>() {
  constexpr int MB = MinBlocks<PPML_REAL>::value;
  cudaError_t e = cudaFuncSetAttribute(lagrangian_tile<PPML_REAL, MB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(LagTileSmem<PPML_REAL>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eulerian_tile<PPML_REAL, MB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EulTileSmem<PPML_REAL>));
  if (e != cudaSuccess) return ppml_fail(PPML_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  return PPML_OK;
}

template <>
int launch_eulerian<PPML_REAL>(const MarchArgs<PPML_REAL>& A, int nblk, cudaStream_t st) {
  constexpr int MB = MinBlocks<PPML_REAL>::value;
  eulerian_tile<PPML_REAL, MB><<<nblk, TN, sizeof(EulTileSmem<PPML_REAL>), st>>>(A);
  return ppml_check_launch("eulerian_tile");
}

template <>
int launch_lagrangian<PPML_REAL>(const MarchArgs<PPML_REAL>& A, int nblk, cudaStream_t st) {
  constexpr int MB = MinBlocks<PPML_REAL>::value;
  lagrangian_tile<PPML_REAL, MB><<<nblk, TN, sizeof(LagTileSmem<PPML_REAL>), st>>>(A);
  return ppml_check_launch("lagrangian_tile");
}

template <>
int launch_diag<PPML_REAL>(const MarchArgs<PPML_REAL>& A, int nblk, cudaStream_t st) {
  diag_kernel<PPML_REAL><<<nblk, NT, 0, st>>>(A);
  return ppml_check_launch("diag_kernel");
}

template <>
int launch_batch<PPML_REAL>(PPML_REAL* rho, PPML_REAL* m, PPML_REAL* en, PPML_REAL* ei,
                            InstDev* inst, const int* order, double gamma, double cfl,
                            int max_steps, int nmax, int ninst, size_t smem, cudaStream_t st) {
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<PPML_REAL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    configured = smem;
  }
  batch_kernel<PPML_REAL><<<ninst, kBatchThreads, smem, st>>>(rho, m, en, ei, inst, order, gamma,
                                                              cfl, max_steps, nmax);
  return ppml_check_launch("batch_kernel");
}

}  // namespace ppml
