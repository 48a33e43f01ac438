// ppml_step_noalloc: one full step without a handle and without allocating device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another part of the process
// is capturing a CUDA graph (allocation is not permitted then), plugins whose host
// application owns the device memory budget and its allocator, and real-time loops that
// must not allocate.  For them this entry point keeps the step's intermediate state U*,
// the per-CTA reduction partials and the step scalars in a fixed buffer of the library
// (the file-scope device array below), sized for grids of up to PPML_NOALLOC_MAX_CELLS
// cells.  The caller still passes the input and output states.
//
// Properties of the shared buffer: every GPU that loads the library holds it until the
// process exits; every call uses the same buffer and it keeps the last call's contents
// (the step scalars are cleared at the start of each call, the rest is fully rewritten
// before it is read); calls that overlap on the GPU (different streams, different host
// threads, no ordering between them) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/ppml.h"
#include "ppml_internal.h"
#include "ppml_launch.h"

using namespace ppml;

namespace {

// U* (five fields) in the widest element type, then the partials, then the scalars.
constexpr size_t kUstarBytes = 5ull * PPML_NOALLOC_MAX_CELLS * sizeof(double);
// A tile of 16^3 cells covers at least 16 cells of any grid, so the tile count of a grid
// of at most PPML_NOALLOC_MAX_CELLS cells is at most PPML_NOALLOC_MAX_CELLS / 16 + a few
// partial tiles per axis.
constexpr size_t kMaxPartials = PPML_NOALLOC_MAX_CELLS / 16 + 4096;
constexpr size_t kPartialBytes = kMaxPartials * sizeof(Partial);
constexpr size_t kScratchBytes = kUstarBytes + kPartialBytes + sizeof(DevScalars);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices];  // device address per device, set on first use

// Device address of the buffer on the current device (cudaGetSymbolAddress once per
// device, with that device current).  The host-side symbol is only a stand-in and must
// never be passed to a kernel.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ppml_fail(PPML_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return ppml_fail(PPML_E_INVAL, "device %d out of range", dev);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return ppml_fail(PPML_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_addr[dev];
  return PPML_OK;
}

template <typename T>
int step_noalloc(const ppml_grid_desc* d, const ppml_state* u_in, ppml_state* u_out, double dt,
                 double rho_mean, unsigned char* scratch, double* out9, cudaStream_t st) {
  int rc = prepare_kernels<T>();
  if (rc) return rc;
  const long long ncell = (long long)d->nx * d->ny * d->nz;
  T* ustar = (T*)scratch;
  Partial* partials = (Partial*)(scratch + kUstarBytes);
  DevScalars* S = (DevScalars*)(scratch + kUstarBytes + kPartialBytes);
  MarchArgs<T> A;
  memset(&A, 0, sizeof(A));
  A.g.n[0] = d->nx;
  A.g.n[1] = d->ny;
  A.g.n[2] = d->nz;
  for (int q = 0; q < 6; q++) {
    A.g.bc[q] = d->bc[q];
    A.any_reflect |= d->bc[q] == PPML_BC_REFLECT;
  }
  A.flags = d->flags;
  A.g.nxy = (long long)d->nx * d->ny;
  A.g.ncell = ncell;
  for (int a = 0; a < 3; a++) A.h[a] = d->h[a];
  A.gamma = d->gamma;
  A.dt_host = dt;
  A.dt_dev = nullptr;
  A.rho_vac = (d->vacuum_frac > 0.0 ? d->vacuum_frac : 1e-5) * rho_mean;
  A.partials = partials;
  A.tiles_x = (d->nx + TB - 1) / TB;
  A.tiles_y = (d->ny + TB - 1) / TB;
  const int tiles_z = (d->nz + TB - 1) / TB;
  A.tiles_z = tiles_z;
  A.tile_order = 0;
  const int nblk = A.tiles_x * A.tiles_y * tiles_z;
  if ((size_t)nblk > kMaxPartials)
    return ppml_fail(PPML_E_INVAL, "grid needs %d tiles (the fixed buffer holds %zu)", nblk,
                     kMaxPartials);
  double hmin = INFINITY;
  const int n[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; a++)
    if (n[a] > 1 && d->h[a] < hmin) hmin = d->h[a];
  if (!isfinite(hmin)) hmin = d->h[0];
  // the step scalars start from zero on every call
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(DevScalars), st);
  if (e != cudaSuccess) return ppml_fail(PPML_E_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  // Eulerian stage: U^n -> U* (rho is read from U^n by the Lagrangian stage)
  for (int f = 0; f < 6; f++) {
    A.u[f] = (const T*)u_in->f[f];
    A.out[f] = f == 0 ? nullptr : ustar + (size_t)(f - 1) * ncell;
  }
  rc = launch_eulerian<T>(A, nblk, st);
  if (rc) return rc;
  // Lagrangian stage and energy correction: U* -> U^{n+1}
  for (int f = 0; f < 6; f++) {
    A.u[f] = f == 0 ? (const T*)u_in->f[0] : ustar + (size_t)(f - 1) * ncell;
    A.out[f] = (T*)u_out->f[f];
  }
  rc = launch_lagrangian<T>(A, nblk, st);
  if (rc) return rc;
  rc = launch_finalize(partials, nblk, S, d->cfl, hmin, d->h[0] * d->h[1] * d->h[2], 0.0, 1,
                       nullptr, dt, st, nullptr);
  if (rc) return rc;
  if (out9) {
    DevScalars hs;
    if (cudaMemcpyAsync(&hs, S, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "step_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
    out9[0] = hs.dt;
    out9[1] = hs.vmax;
    out9[2] = hs.cmax;
    for (int f = 0; f < 6; f++) out9[3 + f] = hs.sums[f];
    if (hs.flags & PPML_FLAG_NONPHYSICAL)
      return ppml_fail(PPML_E_NONPHYSICAL, "non-physical cells in the output (%lld)", hs.n_bad);
  }
  return PPML_OK;
}

}  // namespace

extern "C" int ppml_step_noalloc(const ppml_grid_desc* d, const ppml_state* u_in,
                                 ppml_state* u_out, double dt, double rho_mean, double out[9],
                                 void* stream) {
  ppml_clear_error();
  int rc = ppml_validate_desc(d);
  if (rc) return rc;
  const long long ncell = (long long)d->nx * d->ny * d->nz;
  if (ncell > PPML_NOALLOC_MAX_CELLS)
    return ppml_fail(PPML_E_INVAL,
                     "grid of %lld cells exceeds the fixed buffer of ppml_step_noalloc (%d cells); "
                     "use ppml_init_grid / ppml_step",
                     ncell, PPML_NOALLOC_MAX_CELLS);
  rc = ppml_validate_state(u_in, "u_in");
  if (rc) return rc;
  rc = ppml_validate_state(u_out, "u_out");
  if (rc) return rc;
  if (ppml_state_has_lo(u_in) || ppml_state_has_lo(u_out))
    return ppml_fail(PPML_E_INVAL, "ppml_step_noalloc takes plain float or double states "
                                   "(no low parts)");
  if (d->t_end > 0.0)
    return ppml_fail(PPML_E_INVAL, "ppml_step_noalloc keeps no simulated time: t_end must be 0");
  if (ppml_desc_has_halo(d))
    return ppml_fail(PPML_E_INVAL, "ppml_step_noalloc: halo faces need the slab stage calls");
  for (int q = 0; q < 6; q++)
    if (d->bc[q] == PPML_BC_INFLOW)
      return ppml_fail(PPML_E_INVAL, "ppml_step_noalloc: inflow faces need a grid handle");
  for (int f = 0; f < 6; f++)
    for (int q = 0; q < 6; q++)
      if (u_in->f[f] == u_out->f[q]) return ppml_fail(PPML_E_INVAL, "u_in and u_out alias");
  if (!(dt > 0.0) || !isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt = %g must be > 0", dt);
  if (!(rho_mean > 0.0) || !isfinite(rho_mean))
    return ppml_fail(PPML_E_INVAL, "rho_mean = %g must be > 0", rho_mean);
  unsigned char* scratch = nullptr;
  rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  return d->dtype == PPML_F64 ? step_noalloc<double>(d, u_in, u_out, dt, rho_mean, scratch, out, st)
                              : step_noalloc<float>(d, u_in, u_out, dt, rho_mean, scratch, out, st);
}
