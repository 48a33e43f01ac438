// Host-side launchers of the stencil kernels, instantiated once per precision in
// ppml_kern_f32.cu (FMA contraction on) and ppml_kern_f64.cu (contraction off, so the
// FP64 path evaluates every expression exactly as written).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "ppml_batch.cuh"
#include "ppml_tile.cuh"

namespace ppml {

template <typename T>
int prepare_kernels();  // opt-in shared-memory sizes; call outside stream capture
template <typename T>
int launch_eulerian(const MarchArgs<T>& A, int nblk, cudaStream_t st);
template <typename T>
int launch_lagrangian(const MarchArgs<T>& A, int nblk, cudaStream_t st);
template <typename T>
int launch_diag(const MarchArgs<T>& A, int nblk, cudaStream_t st);
template <typename T>
int launch_poisson_symbol(void* spec, const double* tx, const double* ty, const double* tz, int mx,
                          int ny, int nz, double coef, cudaStream_t st);
// Batched 1D problems: the vacuum thresholds of all ninst instances (instance = CTA index),
// then one CTA per instance of order[0 .. ninst), or one cluster of two CTAs per work item
// of items[0 .. nitems) (nlmax: the largest half of a split instance, nmax: the largest
// instance taken by one CTA).
template <typename T>
int launch_batch_vacuum(const T* rho, InstDev* inst, int ninst, cudaStream_t st);
template <typename T>
int launch_batch(T* rho, T* m, T* en, T* ei, BatchLo<T> lo, InstDev* inst, const int* order,
                 double gamma, double cfl, int max_steps, int nmax, int ninst, size_t smem,
                 int threads, cudaStream_t st);
template <typename T>
int launch_batch_cluster(T* rho, T* m, T* en, T* ei, BatchLo<T> lo, InstDev* inst,
                         const int2* items, double gamma, double cfl, int max_steps, int nlmax,
                         int nmax, int nitems, size_t smem, int threads, cudaStream_t st);

// Deterministic reduction of per-CTA partials into the step scalars (ppml_grid.cu).
int launch_finalize(const Partial* P, int nblk, DevScalars* S, double cfl, double hmin, double vol,
                    double t_end, int mode, const double* dt_dev, double dt_host, cudaStream_t st,
                    double* red);

// explicit specializations live in ppml_kern_f32.cu / ppml_kern_f64.cu
#define PPML_DECLARE_LAUNCHERS(R)                                                            \
  template <>                                                                                \
  int prepare_kernels<R>();                                                                  \
  template <>                                                                                \
  int launch_eulerian<R>(const MarchArgs<R>& A, int nblk, cudaStream_t st);                   \
  template <>                                                                                \
  int launch_lagrangian<R>(const MarchArgs<R>& A, int nblk, cudaStream_t st);                 \
  template <>                                                                                \
  int launch_diag<R>(const MarchArgs<R>& A, int nblk, cudaStream_t st);                       \
  template <>                                                                                \
  int launch_poisson_symbol<R>(void* spec, const double* tx, const double* ty,                 \
                               const double* tz, int mx, int ny, int nz, double coef,          \
                               cudaStream_t st);                                               \
  template <>                                                                                \
  int launch_batch_vacuum<R>(const R* rho, InstDev* inst, int ninst, cudaStream_t st);        \
  template <>                                                                                \
  int launch_batch<R>(R * rho, R * m, R * en, R * ei, BatchLo<R> lo, InstDev * inst,          \
                      const int* order, double gamma, double cfl, int max_steps, int nmax,     \
                      int ninst, size_t smem, int threads, cudaStream_t st);                   \
  template <>                                                                                \
  int launch_batch_cluster<R>(R * rho, R * m, R * en, R * ei, BatchLo<R> lo, InstDev * inst,  \
                              const int2* items, double gamma, double cfl, int max_steps,      \
                              int nlmax, int nmax, int nitems, size_t smem, int threads,       \
                              cudaStream_t st);
PPML_DECLARE_LAUNCHERS(float)
PPML_DECLARE_LAUNCHERS(double)
#undef PPML_DECLARE_LAUNCHERS

}  // namespace ppml
