// Grid path of libppml.so: host side of one PPML operator-splitting step on a 3D uniform
// grid (Kulikov & Vorobyov, arXiv:1607.01105, Sec. 1).
//
// Per step, on the caller's stream:
//   eulerian_tile      Sec. 1.1/1.2: PPML parabolas of v and p, acoustic face solve,
//                      unsplit update of m, rho E, rho eps -> U* (library scratch)
//   lagrangian_tile    Sec. 1.3/1.4: 9-point velocity template, Roe-weighted face velocity,
//                      upwind parabola fluxes of all six fields, unsplit update, energy
//                      correction; per-CTA partial maxima and sums of U^{n+1}
//   finalize_kernel    deterministic reduction of the partials -> device-resident CFL step
//                      (Sec. 1.1), FP64 sums, time and flags
// No host synchronization inside a step, so consecutive steps can be captured in a CUDA
// graph (the step size stays on the device).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <cufft.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/ppml.h"
#include "ppml_internal.h"
#include "ppml_launch.h"

using namespace ppml;

namespace {

constexpr int kFinThreads = 512;

// The device scalars from the maxima, sums (times the cell volume) and counts of a state:
// advance: the state ends a step of tau (t += tau, clipped to t_end; steps + 1).  Then the
// next CFL step (Sec. 1.1) clipped to the remaining time, and the flags.
__device__ void apply_scalars(DevScalars* S, double vmax, double cmax, const double* sums,
                              double nvac, double nbad, int advance, double tau, double cfl,
                              double hmin, double t_end) {
  double tn = S->t;
  if (advance) {
    tn = S->t + tau;
    if (t_end > 0.0 && tn > t_end) tn = t_end;
    S->t = tn;
    S->steps += 1;
    S->n_vac = (long long)nvac;
  }
  S->vmax = vmax;
  S->cmax = cmax;
  for (int f = 0; f < 6; f++) S->sums[f] = sums[f];
  S->n_bad = (long long)nbad;
  double dt = cfl * hmin / (vmax + cmax);
  if (t_end > 0.0 && dt > t_end - tn) dt = t_end - tn;
  if (!(dt > 0.0)) {
    dt = 0.0;
    S->flags |= PPML_FLAG_DT_ZERO;
  }
  S->dt = dt;
  if (nbad > 0.0) S->flags |= PPML_FLAG_NONPHYSICAL;
}

// Reduce nblk partials in a fixed order (independent of scheduling).  mode 0: diagnostics
// of a state into the device scalars; 1: after a step; 2: only write the maxima, sums and
// counts to red[PPML_REDUCE_LEN] (a slab's share, for an all-reduce across slabs).
__global__ void __launch_bounds__(kFinThreads)
    finalize_kernel(const Partial* __restrict__ P, int nblk, DevScalars* S, double cfl,
                    double hmin, double vol, double t_end, int mode, const double* dt_dev,
                    double dt_host, double* red) {
  __shared__ double sh[kFinThreads][8];
  __shared__ unsigned long long shc[kFinThreads][2];
  const int t = threadIdx.x;
  double tau = 0.0;
  if (t == 0 && mode == 1) tau = dt_dev ? *dt_dev : dt_host;
  double s[6] = {0, 0, 0, 0, 0, 0}, vmax = 0.0, cmax = 0.0;
  unsigned long long nvac = 0, nbad = 0;
  for (int b = t; b < nblk; b += kFinThreads) {
    for (int f = 0; f < 6; f++) s[f] += P[b].s[f];
    vmax = fmax(vmax, P[b].vmax);
    cmax = fmax(cmax, P[b].cmax);
    nvac += P[b].nvac;
    nbad += P[b].nbad;
  }
  for (int f = 0; f < 6; f++) sh[t][f] = s[f];
  sh[t][6] = vmax;
  sh[t][7] = cmax;
  shc[t][0] = nvac;
  shc[t][1] = nbad;
  __syncthreads();
  for (int w = kFinThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      for (int f = 0; f < 6; f++) sh[t][f] += sh[t + w][f];
      sh[t][6] = fmax(sh[t][6], sh[t + w][6]);
      sh[t][7] = fmax(sh[t][7], sh[t + w][7]);
      shc[t][0] += shc[t + w][0];
      shc[t][1] += shc[t + w][1];
    }
    __syncthreads();
  }
  if (t == 0) {
    double sums[6];
    for (int f = 0; f < 6; f++) sums[f] = sh[0][f] * vol;
    if (mode == 2) {
      red[0] = sh[0][6];
      red[1] = sh[0][7];
      for (int f = 0; f < 6; f++) red[2 + f] = sums[f];
      red[8] = (double)shc[0][0];
      red[9] = (double)shc[0][1];
      return;
    }
    apply_scalars(S, sh[0][6], sh[0][7], sums, (double)shc[0][0], (double)shc[0][1], mode == 1,
                  tau, cfl, hmin, t_end);
  }
}

// The device scalars from an all-reduced red[PPML_REDUCE_LEN] (slab decomposition).
__global__ void apply_reduced_kernel(const double* __restrict__ red, DevScalars* S, int advance,
                                     const double* dt_dev, double dt_host, double cfl,
                                     double hmin, double t_end) {
  if (threadIdx.x != 0) return;
  const double tau = advance ? (dt_dev ? *dt_dev : dt_host) : 0.0;
  apply_scalars(S, red[0], red[1], red + 2, red[8], red[9], advance, tau, cfl, hmin, t_end);
}

}  // namespace

namespace ppml {
int launch_finalize(const Partial* P, int nblk, DevScalars* S, double cfl, double hmin, double vol,
                    double t_end, int mode, const double* dt_dev, double dt_host, cudaStream_t st,
                    double* red) {
  finalize_kernel<<<1, kFinThreads, 0, st>>>(P, nblk, S, cfl, hmin, vol, t_end, mode, dt_dev,
                                             dt_host, red);
  return ppml_check_launch("finalize_kernel");
}
}  // namespace ppml

struct ppml_grid {
  ppml_grid_desc d;
  GridGeom geom;
  size_t elt;
  void* ustar[6];  // [0] unused (rho is not changed by the Eulerian stage)
  void* ustar_lo[5];  // FP32: low parts of U*'s m and rho E ([0] unused)
  Partial* partials;
  void* inflow;  // 36 values of the state's type: the inflow faces' ghost states [face][field]
  int nblk_march, nblk_diag, npartials;  // tiles (partials of a step), diagnostics blocks
  int tiles_x, tiles_y, tiles_z;
  int tile_order;   // launch order of the stage kernels' tiles (ppml_grid_tune)
  int nblk_launch;  // blocks of a stage launch in that order
  DevScalars* dev;
  double rho_mean, rho_vac, hmin, vol;
  // measurement hook: events around each kernel of a step
  int profiling;
  static const int kEvSlots = 4096;
  cudaEvent_t* ev;  // kEvSlots * 4 events
  int ev_used;
  double ms[3];
  long long prof_steps;
  // periodic Poisson solve: cuFFT plans, half spectrum and per-axis symbol tables
  int fft_ready;
  cufftHandle fft_fwd, fft_inv;
  void* spec;
  double* tables;
  // isolated Poisson solve (ppml_poisson.cu)
  PoissonIso* iso;
  // disk Fourier amplitudes (ppml_fourier.cu)
  FourierState* fourier;
};

int ppml_validate_desc(const ppml_grid_desc* d) {
  if (!d) return ppml_fail(PPML_E_INVAL, "desc is NULL");
  const int n[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; a++) {
    if (n[a] < 1) return ppml_fail(PPML_E_INVAL, "axis %d has %d cells (need >= 1)", a, n[a]);
    if (!(d->h[a] > 0.0) || !isfinite(d->h[a]))
      return ppml_fail(PPML_E_INVAL, "h[%d] = %g must be positive", a, d->h[a]);
    const int lo = d->bc[2 * a], hi = d->bc[2 * a + 1];
    if (lo < 0 || lo > 4 || hi < 0 || hi > 4)
      return ppml_fail(PPML_E_INVAL, "bc of axis %d is not a ppml_bc", a);
    for (int side = 0; side < 2; side++) {
      if (d->bc[2 * a + side] != PPML_BC_INFLOW) continue;
      const double* s = d->inflow[2 * a + side];
      bool ok = s[0] > 0.0 && s[5] > 0.0;
      for (int f = 0; f < 6; f++) ok = ok && isfinite(s[f]);
      if (!ok) return ppml_fail(PPML_E_INVAL, "inflow state of face %d needs rho > 0, rho eps > 0, finite values", 2 * a + side);
    }
    if ((lo == PPML_BC_HALO || hi == PPML_BC_HALO) && (a != 2 || n[a] < 3))
      return ppml_fail(PPML_E_INVAL, "halo faces are z faces of an active z axis (axis %d)", a);
    if ((lo == PPML_BC_PERIODIC) != (hi == PPML_BC_PERIODIC))
      return ppml_fail(PPML_E_INVAL, "periodic bc on axis %d must be set on both faces", a);
    if (n[a] == 1 && (lo == PPML_BC_REFLECT || hi == PPML_BC_REFLECT))
      return ppml_fail(PPML_E_INVAL, "inactive axis %d cannot be reflecting", a);
    if (n[a] > 1 && n[a] < 3)
      return ppml_fail(PPML_E_INVAL, "axis %d has %d cells (active axes need >= 3)", a, n[a]);
  }
  bool has_inflow = false, has_reflect = false;
  for (int q = 0; q < 6; q++) {
    has_inflow = has_inflow || d->bc[q] == PPML_BC_INFLOW;
    has_reflect = has_reflect || d->bc[q] == PPML_BC_REFLECT;
  }
  if (has_inflow && has_reflect)
    return ppml_fail(PPML_E_INVAL, "inflow faces cannot be combined with reflecting faces");
  if (d->rho_ref < 0.0 || !isfinite(d->rho_ref))
    return ppml_fail(PPML_E_INVAL, "rho_ref = %g must be >= 0", d->rho_ref);
  if (!(d->gamma > 1.0) || !isfinite(d->gamma))
    return ppml_fail(PPML_E_INVAL, "gamma = %g must be > 1", d->gamma);
  if (!(d->cfl > 0.0 && d->cfl < 1.0)) return ppml_fail(PPML_E_INVAL, "cfl = %g not in (0,1)", d->cfl);
  if (d->dtype != PPML_F32 && d->dtype != PPML_F64)
    return ppml_fail(PPML_E_INVAL, "dtype %d is not a ppml_dtype", d->dtype);
  if (d->flags & ~(int)(PPML_FIRST_ORDER | PPML_VHAT_1PT))
    return ppml_fail(PPML_E_INVAL, "unknown flags 0x%x", d->flags);
  const long long nc = (long long)n[0] * n[1] * n[2];
  if (nc > (1ll << 31) - 1024) return ppml_fail(PPML_E_INVAL, "grid of %lld cells is too large", nc);
  return PPML_OK;
}

int ppml_validate_state(const ppml_state* u, const char* what) {
  if (!u) return ppml_fail(PPML_E_INVAL, "%s is NULL", what);
  for (int f = 0; f < 6; f++) {
    if (!u->f[f]) return ppml_fail(PPML_E_INVAL, "%s field %d is NULL", what, f);
    if (((uintptr_t)u->f[f]) & 15u)
      return ppml_fail(PPML_E_INVAL, "%s field %d is not 16-byte aligned", what, f);
  }
  const int nlo = ppml_state_has_lo(u);
  if (nlo != 0 && nlo != 5)
    return ppml_fail(PPML_E_INVAL, "%s has %d of 5 low-part pointers (all or none)", what, nlo);
  for (int f = 0; f < 5 && nlo; f++) {
    if (((uintptr_t)u->lo[f]) & 15u)
      return ppml_fail(PPML_E_INVAL, "%s low part %d is not 16-byte aligned", what, f);
    for (int q = 0; q < 6; q++)
      if (u->lo[f] == u->f[q]) return ppml_fail(PPML_E_INVAL, "%s low part %d aliases a field", what, f);
  }
  return PPML_OK;
}

int ppml_desc_has_halo(const ppml_grid_desc* d) {
  for (int q = 0; q < 6; q++)
    if (d->bc[q] == PPML_BC_HALO) return 1;
  return 0;
}

// Calls that step through the handle's own U* (which has no halo planes) refuse grids with
// halo faces: their Lagrangian stage would read U* beyond its first and last planes.
static int no_halo(const ppml_grid* g, const char* what) {
  if (ppml_desc_has_halo(&g->d))
    return ppml_fail(PPML_E_INVAL, "%s: the grid has halo faces (use the slab stage calls)", what);
  return PPML_OK;
}

int ppml_state_has_lo(const ppml_state* u) {
  int n = 0;
  for (int f = 0; f < 5; f++) n += u->lo[f] != nullptr;
  return n;
}

// A state of the grid's type: low parts only in FP32.
static int check_state_type(const ppml_grid_desc* d, const ppml_state* u, const char* what) {
  if (d->dtype == PPML_F64 && ppml_state_has_lo(u))
    return ppml_fail(PPML_E_INVAL, "%s: low parts are for FP32 states only", what);
  return PPML_OK;
}

namespace {

template <typename T>
MarchArgs<T> make_args(const ppml_grid* g, double dt_host, const double* dt_dev) {
  MarchArgs<T> A;
  memset(&A, 0, sizeof(A));
  A.g = g->geom;
  for (int a = 0; a < 3; a++) A.h[a] = g->d.h[a];
  A.gamma = g->d.gamma;
  A.dt_host = dt_host;
  A.dt_dev = dt_dev;
  A.rho_vac = g->rho_vac;
  A.partials = g->partials;
  A.tiles_x = g->tiles_x;
  A.tiles_y = g->tiles_y;
  A.tiles_z = g->tiles_z;
  A.tile_order = g->tile_order;
  A.any_reflect = 0;
  for (int q = 0; q < 6; q++) A.any_reflect |= g->d.bc[q] == PPML_BC_REFLECT;
  A.flags = g->d.flags;
  A.inflow = (const T*)g->inflow;
  A.any_inflow = 0;
  for (int q = 0; q < 6; q++) A.any_inflow |= g->d.bc[q] == PPML_BC_INFLOW;
  return A;
}

template <typename T>
int run_diag(ppml_grid* g, const ppml_state* u, cudaStream_t st) {
  MarchArgs<T> A = make_args<T>(g, 0.0, nullptr);
  for (int f = 0; f < 6; f++) A.u[f] = (const T*)u->f[f];
  for (int f = 0; f < 5; f++) A.ulo[f] = (const T*)u->lo[f];
  int rc = launch_diag<T>(A, g->nblk_diag, st);
  if (rc) return rc;
  return launch_finalize(g->partials, g->nblk_diag, g->dev, g->d.cfl, g->hmin, g->vol,
                         g->d.t_end, 0, nullptr, 0.0, st, nullptr);
}

template <typename T>
int run_eulerian(ppml_grid* g, const ppml_state* u, void* const out[6], void* const outlo[5],
                 const T* phi, double dt_host, const double* dt_dev, cudaStream_t st) {
  MarchArgs<T> A = make_args<T>(g, dt_host, dt_dev);
  for (int f = 0; f < 6; f++) {
    A.u[f] = (const T*)u->f[f];
    A.out[f] = (T*)out[f];
  }
  if (ppml_state_has_lo(u))
    for (int f = 0; f < 5; f++) {
      A.ulo[f] = (const T*)u->lo[f];
      A.outlo[f] = (T*)outlo[f];
    }
  A.phi = phi;
  return launch_eulerian<T>(A, g->nblk_launch, st);
}

// Fold the recorded events of finished steps into the per-kernel totals.
int fold_events(ppml_grid* g) {
  for (int s = 0; s < g->ev_used; s++) {
    cudaEvent_t* e = g->ev + 4 * s;
    for (int q = 0; q < 3; q++) {
      float ms = 0.f;
      if (cudaEventSynchronize(e[q + 1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e[q], e[q + 1]) != cudaSuccess)
        return ppml_fail(PPML_E_CUDA, "kernel timing: %s", cudaGetErrorString(cudaGetLastError()));
      g->ms[q] += ms;
    }
  }
  g->prof_steps += g->ev_used;
  g->ev_used = 0;
  return PPML_OK;
}

template <typename T>
int run_step(ppml_grid* g, const ppml_state* uin, ppml_state* uout, const T* phi,
             double dt_host, const double* dt_dev, cudaStream_t st) {
  cudaEvent_t* ev = nullptr;
  if (g->profiling) {
    if (g->ev_used == ppml_grid::kEvSlots) {
      int rc = fold_events(g);
      if (rc) return rc;
    }
    ev = g->ev + 4 * g->ev_used;
    g->ev_used++;
    cudaEventRecord(ev[0], st);
  }
  void* star[6] = {nullptr, g->ustar[1], g->ustar[2], g->ustar[3], g->ustar[4], g->ustar[5]};
  void* star_lo[5] = {nullptr, g->ustar_lo[1], g->ustar_lo[2], g->ustar_lo[3], g->ustar_lo[4]};
  int rc = run_eulerian<T>(g, uin, star, star_lo, phi, dt_host, dt_dev, st);
  if (rc) return rc;
  if (ev) cudaEventRecord(ev[1], st);
  MarchArgs<T> L = make_args<T>(g, dt_host, dt_dev);
  L.u[0] = (const T*)uin->f[0];
  for (int f = 1; f < 6; f++) L.u[f] = (const T*)g->ustar[f];
  for (int f = 0; f < 6; f++) L.out[f] = (T*)uout->f[f];
  if (ppml_state_has_lo(uin)) {
    L.ulo[0] = (const T*)uin->lo[0];
    for (int f = 1; f < 5; f++) L.ulo[f] = (const T*)g->ustar_lo[f];
    for (int f = 0; f < 5; f++) L.outlo[f] = (T*)uout->lo[f];
  }
  rc = launch_lagrangian<T>(L, g->nblk_launch, st);
  if (rc) return rc;
  if (ev) cudaEventRecord(ev[2], st);
  rc = launch_finalize(g->partials, g->nblk_march, g->dev, g->d.cfl, g->hmin, g->vol,
                       g->d.t_end, 1, dt_dev, dt_host, st, nullptr);
  if (ev) cudaEventRecord(ev[3], st);
  return rc;
}

}  // namespace

extern "C" int ppml_init_grid(const ppml_grid_desc* d, const ppml_state* u0, void* stream,
                              ppml_grid** out) {
  ppml_clear_error();
  if (!out) return ppml_fail(PPML_E_INVAL, "out is NULL");
  *out = nullptr;
  int rc = ppml_validate_desc(d);
  if (rc) return rc;
  rc = ppml_validate_state(u0, "u0");
  if (rc) return rc;
  rc = check_state_type(d, u0, "u0");
  if (rc) return rc;
  ppml_grid* g = new (std::nothrow) ppml_grid();
  if (!g) return ppml_fail(PPML_E_NOMEM, "host allocation failed");
  g->d = *d;
  if (!(g->d.vacuum_frac > 0.0)) g->d.vacuum_frac = 1e-5;
  g->geom.n[0] = d->nx;
  g->geom.n[1] = d->ny;
  g->geom.n[2] = d->nz;
  for (int q = 0; q < 6; q++) g->geom.bc[q] = d->bc[q];
  g->geom.nxy = (long long)d->nx * d->ny;
  g->geom.ncell = g->geom.nxy * d->nz;
  g->elt = d->dtype == PPML_F64 ? 8 : 4;
  g->tiles_x = (d->nx + TB - 1) / TB;
  g->tiles_y = (d->ny + TB - 1) / TB;
  g->tiles_z = (d->nz + TB - 1) / TB;
  g->nblk_march = g->tiles_x * g->tiles_y * g->tiles_z;
  g->tile_order = 0;
  g->nblk_launch = g->nblk_march;
  g->nblk_diag = (int)std::min<long long>((g->geom.ncell + NT - 1) / NT, 4 * 152);
  g->npartials = std::max(g->nblk_march, g->nblk_diag);
  g->hmin = INFINITY;
  const int n[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; a++)
    if (n[a] > 1 && d->h[a] < g->hmin) g->hmin = d->h[a];
  if (!isfinite(g->hmin)) g->hmin = d->h[0];
  g->vol = d->h[0] * d->h[1] * d->h[2];
  rc = d->dtype == PPML_F64 ? prepare_kernels<double>() : prepare_kernels<float>();
  if (rc) {
    delete g;
    return rc;
  }
  const size_t fbytes = (size_t)g->geom.ncell * g->elt;
  for (int f = 1; f < 6; f++) {
    if (cudaMalloc(&g->ustar[f], fbytes) != cudaSuccess) {
      ppml_free_grid(g);
      return ppml_fail(PPML_E_NOMEM, "cudaMalloc of U* (%zu bytes) failed", fbytes);
    }
  }
  for (int f = 1; f < 5 && d->dtype == PPML_F32; f++) {
    if (cudaMalloc(&g->ustar_lo[f], fbytes) != cudaSuccess) {
      ppml_free_grid(g);
      return ppml_fail(PPML_E_NOMEM, "cudaMalloc of U* low parts (%zu bytes) failed", fbytes);
    }
  }
  if (cudaMalloc(&g->partials, sizeof(Partial) * (size_t)g->npartials) != cudaSuccess ||
      cudaMalloc(&g->dev, sizeof(DevScalars)) != cudaSuccess ||
      cudaMalloc(&g->inflow, 36 * g->elt) != cudaSuccess) {
    ppml_free_grid(g);
    return ppml_fail(PPML_E_NOMEM, "cudaMalloc of reduction scratch failed");
  }
  cudaStream_t st = (cudaStream_t)stream;
  {  // the inflow states in the state's precision (zeros for faces that are not inflow)
    double hd[36];
    float hf[36];
    for (int q = 0; q < 6; q++)
      for (int f = 0; f < 6; f++) {
        hd[6 * q + f] = d->bc[q] == PPML_BC_INFLOW ? d->inflow[q][f] : 0.0;
        hf[6 * q + f] = (float)hd[6 * q + f];
      }
    if (cudaMemcpy(g->inflow, d->dtype == PPML_F64 ? (const void*)hd : (const void*)hf,
                   36 * g->elt, cudaMemcpyHostToDevice) != cudaSuccess) {
      ppml_free_grid(g);
      return ppml_fail(PPML_E_CUDA, "init: inflow states: %s", cudaGetErrorString(cudaGetLastError()));
    }
  }
  cudaMemsetAsync(g->dev, 0, sizeof(DevScalars), st);
  rc = d->dtype == PPML_F64 ? run_diag<double>(g, u0, st) : run_diag<float>(g, u0, st);
  if (rc) {
    ppml_free_grid(g);
    return rc;
  }
  DevScalars hs;
  if (cudaMemcpyAsync(&hs, g->dev, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    ppml_free_grid(g);
    return ppml_fail(PPML_E_CUDA, "init: %s", cudaGetErrorString(cudaGetLastError()));
  }
  g->rho_mean = g->d.rho_ref > 0.0 ? g->d.rho_ref : hs.sums[0] / (g->vol * (double)g->geom.ncell);
  g->rho_vac = g->d.vacuum_frac * g->rho_mean;
  *out = g;
  return PPML_OK;
}

extern "C" int ppml_free_grid(ppml_grid* g) {
  ppml_clear_error();
  if (!g) return PPML_OK;
  cudaDeviceSynchronize();
  for (int f = 0; f < 6; f++)
    if (g->ustar[f]) cudaFree(g->ustar[f]);
  for (int f = 0; f < 5; f++)
    if (g->ustar_lo[f]) cudaFree(g->ustar_lo[f]);
  if (g->partials) cudaFree(g->partials);
  if (g->inflow) cudaFree(g->inflow);
  if (g->dev) cudaFree(g->dev);
  if (g->ev) {
    for (int q = 0; q < 4 * ppml_grid::kEvSlots; q++) cudaEventDestroy(g->ev[q]);
    delete[] g->ev;
  }
  if (g->fft_ready) {
    cufftDestroy(g->fft_fwd);
    cufftDestroy(g->fft_inv);
  }
  if (g->spec) cudaFree(g->spec);
  if (g->tables) cudaFree(g->tables);
  ppml_iso_free(g->iso);
  ppml_fourier_free(g->fourier);
  delete g;
  return PPML_OK;
}

extern "C" int ppml_poisson_periodic(ppml_grid* g, const void* rho, void* phi, double G,
                                     void* stream) {
  ppml_clear_error();
  if (!g || !rho || !phi) return ppml_fail(PPML_E_INVAL, "grid, rho or phi is NULL");
  if (rho == phi) return ppml_fail(PPML_E_INVAL, "rho and phi alias");
  if (!isfinite(G)) return ppml_fail(PPML_E_INVAL, "G is not finite");
  if (ppml_desc_has_halo(&g->d)) return ppml_fail(PPML_E_INVAL, "Poisson solve on a slab");
  const int n[3] = {g->d.nx, g->d.ny, g->d.nz};
  for (int a = 1; a < 3; a++)
    if (n[a] > 1 && fabs(g->d.h[a] - g->d.h[0]) > 1e-12 * g->d.h[0])
      return ppml_fail(PPML_E_INVAL, "the 27-point solve needs equal cell sizes");
  cudaStream_t st = (cudaStream_t)stream;
  const bool f64 = g->d.dtype == PPML_F64;
  const int mx = n[0] / 2 + 1;
  if (!g->fft_ready) {
    const size_t cbytes = (size_t)mx * n[1] * n[2] * 2 * g->elt;
    if (cudaMalloc(&g->spec, cbytes) != cudaSuccess ||
        cudaMalloc(&g->tables, sizeof(double) * (size_t)(mx + n[1] + n[2])) != cudaSuccess)
      return ppml_fail(PPML_E_NOMEM, "Poisson buffers");
    std::vector<double> tab;
    const int len[3] = {mx, n[1], n[2]};
    for (int a = 0; a < 3; a++)
      for (int k = 0; k < len[a]; k++) {
        const double s = sin(M_PI * (double)k / (double)n[a]);
        tab.push_back(1.0 - (2.0 / 3.0) * s * s);
      }
    if (cudaMemcpy(g->tables, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "Poisson tables: %s", cudaGetErrorString(cudaGetLastError()));
    if (cufftPlan3d(&g->fft_fwd, n[2], n[1], n[0], f64 ? CUFFT_D2Z : CUFFT_R2C) != CUFFT_SUCCESS ||
        cufftPlan3d(&g->fft_inv, n[2], n[1], n[0], f64 ? CUFFT_Z2D : CUFFT_C2R) != CUFFT_SUCCESS)
      return ppml_fail(PPML_E_CUDA, "cufftPlan3d failed");
    g->fft_ready = 1;
  }
  if (cufftSetStream(g->fft_fwd, st) != CUFFT_SUCCESS || cufftSetStream(g->fft_inv, st) != CUFFT_SUCCESS)
    return ppml_fail(PPML_E_CUDA, "cufftSetStream failed");
  cufftResult r = f64 ? cufftExecD2Z(g->fft_fwd, (cufftDoubleReal*)rho, (cufftDoubleComplex*)g->spec)
                      : cufftExecR2C(g->fft_fwd, (cufftReal*)rho, (cufftComplex*)g->spec);
  if (r != CUFFT_SUCCESS) return ppml_fail(PPML_E_CUDA, "cuFFT forward failed (%d)", (int)r);
  const double h = g->d.h[0];
  const double coef = -(2.0 / 3.0) * M_PI * G * h * h / ((double)n[0] * n[1] * n[2]);
  const double* tx = g->tables;
  const double* ty = tx + mx;
  const double* tz = ty + n[1];
  int rc = f64 ? launch_poisson_symbol<double>(g->spec, tx, ty, tz, mx, n[1], n[2], coef, st)
               : launch_poisson_symbol<float>(g->spec, tx, ty, tz, mx, n[1], n[2], coef, st);
  if (rc) return rc;
  r = f64 ? cufftExecZ2D(g->fft_inv, (cufftDoubleComplex*)g->spec, (cufftDoubleReal*)phi)
          : cufftExecC2R(g->fft_inv, (cufftComplex*)g->spec, (cufftReal*)phi);
  if (r != CUFFT_SUCCESS) return ppml_fail(PPML_E_CUDA, "cuFFT inverse failed (%d)", (int)r);
  return PPML_OK;
}

extern "C" int ppml_poisson_isolated(ppml_grid* g, const void* rho, void* phi, double G,
                                     unsigned flags, void* stream) {
  ppml_clear_error();
  if (!g || !rho || !phi) return ppml_fail(PPML_E_INVAL, "grid, rho or phi is NULL");
  if (rho == phi) return ppml_fail(PPML_E_INVAL, "rho and phi alias");
  if (!isfinite(G)) return ppml_fail(PPML_E_INVAL, "G is not finite");
  if (flags & ~PPML_POISSON_PRINTED_RHS) return ppml_fail(PPML_E_INVAL, "unknown flags 0x%x", flags);
  if (ppml_desc_has_halo(&g->d)) return ppml_fail(PPML_E_INVAL, "Poisson solve on a slab");
  for (int a = 1; a < 3; a++)
    if (fabs(g->d.h[a] - g->d.h[0]) > 1e-12 * g->d.h[0])
      return ppml_fail(PPML_E_INVAL, "the 27-point solve needs equal cell sizes");
  return ppml_iso_solve(&g->iso, &g->d, rho, phi, G, flags, (cudaStream_t)stream);
}

extern "C" int ppml_fourier_amplitudes(ppml_grid* g, const void* rho, double r_f, int m_max,
                                       double* a_out, void* stream) {
  ppml_clear_error();
  if (!g || !rho || !a_out) return ppml_fail(PPML_E_INVAL, "grid, rho or a_out is NULL");
  if (!(r_f > 0.0) || !isfinite(r_f)) return ppml_fail(PPML_E_INVAL, "r_f = %g must be > 0", r_f);
  if (m_max < 1 || m_max > PPML_FOURIER_MAX_MODES)
    return ppml_fail(PPML_E_INVAL, "m_max = %d not in [1, %d]", m_max, PPML_FOURIER_MAX_MODES);
  return ppml_fourier_run(&g->fourier, &g->d, rho, r_f, m_max, a_out, (cudaStream_t)stream);
}

extern "C" int ppml_cfl_dt(ppml_grid* g, const ppml_state* u, double* dt_host, void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = ppml_validate_state(u, "u");
  if (rc) return rc;
  rc = check_state_type(&g->d, u, "u");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = g->d.dtype == PPML_F64 ? run_diag<double>(g, u, st) : run_diag<float>(g, u, st);
  if (rc) return rc;
  if (dt_host) {
    if (cudaMemcpyAsync(dt_host, &g->dev->dt, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "cfl_dt: %s", cudaGetErrorString(cudaGetLastError()));
  }
  return PPML_OK;
}

static int step_common(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out, const void* phi,
                       double dt, void* stream);

// An input and an output state of one call: the grid's type, low parts in both or neither,
// and no array of one in the other (rho_shared: b's rho and its low part may be a's).
static int check_state_pair(const ppml_grid_desc* d, const ppml_state* a, const ppml_state* b,
                            bool rho_shared = false) {
  int rc = check_state_type(d, a, "u_in");
  if (rc) return rc;
  rc = check_state_type(d, b, "u_out");
  if (rc) return rc;
  if ((ppml_state_has_lo(a) != 0) != (ppml_state_has_lo(b) != 0))
    return ppml_fail(PPML_E_INVAL, "u_in and u_out must both carry low parts or neither");
  const void* pa[11];
  const void* pb[11];
  for (int f = 0; f < 6; f++) {
    pa[f] = a->f[f];
    pb[f] = b->f[f];
  }
  for (int f = 0; f < 5; f++) {
    pa[6 + f] = a->lo[f];
    pb[6 + f] = b->lo[f];
  }
  for (int i = 0; i < 11; i++)
    for (int j = 0; j < 11; j++) {
      if (rho_shared && i == j && (i == 0 || i == 6)) continue;
      if (pa[i] && pa[i] == pb[j]) return ppml_fail(PPML_E_INVAL, "u_in and u_out alias");
    }
  return PPML_OK;
}

extern "C" int ppml_step(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out, double dt,
                         void* stream) {
  return step_common(g, u_in, u_out, nullptr, dt, stream);
}

extern "C" int ppml_step_phi(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out,
                             const void* phi, double dt, void* stream) {
  if (phi && (((uintptr_t)phi) & 15u)) {
    ppml_clear_error();
    return ppml_fail(PPML_E_INVAL, "phi is not 16-byte aligned");
  }
  return step_common(g, u_in, u_out, phi, dt, stream);
}

static int step_common(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out, const void* phi,
                       double dt, void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = no_halo(g, "ppml_step");
  if (rc) return rc;
  rc = ppml_validate_state(u_in, "u_in");
  if (rc) return rc;
  rc = ppml_validate_state(u_out, "u_out");
  if (rc) return rc;
  rc = check_state_pair(&g->d, u_in, u_out);
  if (rc) return rc;
  if (!isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt is not finite");
  const double* dt_dev = dt > 0.0 ? nullptr : &g->dev->dt;
  cudaStream_t st = (cudaStream_t)stream;
  return g->d.dtype == PPML_F64
             ? run_step<double>(g, u_in, u_out, (const double*)phi, dt, dt_dev, st)
             : run_step<float>(g, u_in, u_out, (const float*)phi, dt, dt_dev, st);
}

extern "C" int ppml_eulerian_stage(ppml_grid* g, const ppml_state* u_in, ppml_state* u_star,
                                   double dt, void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = ppml_validate_state(u_in, "u_in");
  if (rc) return rc;
  rc = ppml_validate_state(u_star, "u_star");
  if (rc) return rc;
  rc = check_state_pair(&g->d, u_in, u_star, true);
  if (rc) return rc;
  if (!isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt is not finite");
  const double* dt_dev = dt > 0.0 ? nullptr : &g->dev->dt;
  cudaStream_t st = (cudaStream_t)stream;
  // rho is not changed by the Eulerian stage: a shared rho array is left as it is
  void* out[6];
  void* outlo[5];
  for (int f = 0; f < 6; f++) out[f] = u_star->f[f];
  for (int f = 0; f < 5; f++) outlo[f] = u_star->lo[f];
  if (u_star->f[0] == u_in->f[0]) {
    out[0] = nullptr;
    outlo[0] = nullptr;
  }
  return g->d.dtype == PPML_F64
             ? run_eulerian<double>(g, u_in, out, outlo, nullptr, dt, dt_dev, st)
             : run_eulerian<float>(g, u_in, out, outlo, nullptr, dt, dt_dev, st);
}

extern "C" int ppml_conserved_sums(ppml_grid* g, const ppml_state* u, double out[6],
                                   void* stream) {
  ppml_clear_error();
  if (!g || !out) return ppml_fail(PPML_E_INVAL, "grid or out is NULL");
  int rc = ppml_validate_state(u, "u");
  if (rc) return rc;
  rc = check_state_type(&g->d, u, "u");
  if (rc) return rc;
  // Sums go through the same partial/finalize path; the handle's scalars are restored.
  DevScalars keep, hs;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&keep, g->dev, sizeof(keep), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "sums: %s", cudaGetErrorString(cudaGetLastError()));
  rc = g->d.dtype == PPML_F64 ? run_diag<double>(g, u, st) : run_diag<float>(g, u, st);
  if (rc) return rc;
  if (cudaMemcpyAsync(&hs, g->dev, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(g->dev, &keep, sizeof(keep), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "sums: %s", cudaGetErrorString(cudaGetLastError()));
  for (int f = 0; f < 6; f++) out[f] = hs.sums[f];
  return PPML_OK;
}

extern "C" int ppml_read_diag(ppml_grid* g, ppml_diag* out, void* stream) {
  ppml_clear_error();
  if (!g || !out) return ppml_fail(PPML_E_INVAL, "grid or out is NULL");
  DevScalars hs;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&hs, g->dev, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "read_diag: %s", cudaGetErrorString(cudaGetLastError()));
  out->t = hs.t;
  out->dt_next = hs.dt;
  out->vmax = hs.vmax;
  out->cmax = hs.cmax;
  for (int f = 0; f < 6; f++) out->sums[f] = hs.sums[f];
  out->steps = hs.steps;
  out->n_vacuum = hs.n_vac;
  out->n_bad = hs.n_bad;
  out->flags = hs.flags;
  if (hs.flags & PPML_FLAG_NONPHYSICAL)
    return ppml_fail(PPML_E_NONPHYSICAL, "non-physical cells seen (%lld in the last state)",
                     hs.n_bad);
  return PPML_OK;
}

extern "C" const double* ppml_dt_device(const ppml_grid* g) { return g ? &g->dev->dt : nullptr; }

extern "C" int ppml_profile(ppml_grid* g, int enable) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  if (enable && !g->ev) {
    g->ev = new (std::nothrow) cudaEvent_t[4 * ppml_grid::kEvSlots];
    if (!g->ev) return ppml_fail(PPML_E_NOMEM, "event pool");
    for (int q = 0; q < 4 * ppml_grid::kEvSlots; q++)
      if (cudaEventCreate(&g->ev[q]) != cudaSuccess)
        return ppml_fail(PPML_E_CUDA, "cudaEventCreate: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (g->ev_used) {
    int rc = fold_events(g);
    if (rc) return rc;
  }
  g->profiling = enable ? 1 : 0;
  g->ms[0] = g->ms[1] = g->ms[2] = 0.0;
  g->prof_steps = 0;
  return PPML_OK;
}

extern "C" int ppml_kernel_times(ppml_grid* g, double ms[3], long long* steps) {
  ppml_clear_error();
  if (!g || !ms) return ppml_fail(PPML_E_INVAL, "grid or ms is NULL");
  int rc = fold_events(g);
  if (rc) return rc;
  for (int q = 0; q < 3; q++) ms[q] = g->ms[q];
  if (steps) *steps = g->prof_steps;
  return PPML_OK;
}

extern "C" int ppml_grid_set_order(ppml_grid* g, int order) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  if (order < 0 || order >= kTileOrders)
    return ppml_fail(PPML_E_INVAL, "tile order %d not in [0, %d)", order, kTileOrders);
  const long long nb = order_blocks(order, g->tiles_x, g->tiles_y, g->tiles_z);
  if (nb > (1ll << 31) - 1) return ppml_fail(PPML_E_INVAL, "too many blocks for order %d", order);
  g->tile_order = order;
  g->nblk_launch = (int)nb;
  return PPML_OK;
}

extern "C" int ppml_grid_tune(ppml_grid* g, const ppml_state* u, int trial_steps, int* order_out,
                              double ms_out[PPML_TILE_ORDERS], void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = ppml_validate_state(u, "u");
  if (rc) return rc;
  rc = check_state_type(&g->d, u, "u");
  if (rc) return rc;
  if (trial_steps < 1) return ppml_fail(PPML_E_INVAL, "trial_steps = %d must be >= 1", trial_steps);
  rc = no_halo(g, "ppml_grid_tune");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t fbytes = (size_t)g->geom.ncell * g->elt;
  // two scratch states (the trials ping-pong between them from a copy of u's fields) and
  // the handle's step scalars, restored at the end
  void* buf[12] = {};
  DevScalars keep;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int prof = g->profiling, order0 = g->tile_order;
  g->profiling = 0;
  for (int q = 0; q < 12 && rc == PPML_OK; q++)
    if (cudaMalloc(&buf[q], fbytes) != cudaSuccess) rc = ppml_fail(PPML_E_NOMEM, "tuning scratch state");
  if (rc == PPML_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = ppml_fail(PPML_E_CUDA, "cudaEventCreate failed");
  if (rc == PPML_OK && (cudaMemcpyAsync(&keep, g->dev, sizeof(keep), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
    rc = ppml_fail(PPML_E_CUDA, "tuning: %s", cudaGetErrorString(cudaGetLastError()));
  ppml_state sa = {}, sb = {};
  for (int f = 0; f < 6; f++) {
    sa.f[f] = buf[f];
    sb.f[f] = buf[6 + f];
  }
  double best_ms = 0.0;
  int best = order0;
  for (int order = 0; order < kTileOrders && rc == PPML_OK; order++) {
    rc = ppml_grid_set_order(g, order);
    float best_k = 0.f;
    for (int rep = 0; rep < 2 && rc == PPML_OK; rep++) {  // the first repetition also warms up
      for (int f = 0; f < 6 && rc == PPML_OK; f++)
        if (cudaMemcpyAsync(sa.f[f], u->f[f], fbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          rc = ppml_fail(PPML_E_CUDA, "tuning copy: %s", cudaGetErrorString(cudaGetLastError()));
      if (rc == PPML_OK && cudaMemcpyAsync(g->dev, &keep, sizeof(keep), cudaMemcpyHostToDevice, st) !=
                               cudaSuccess)
        rc = ppml_fail(PPML_E_CUDA, "tuning copy: %s", cudaGetErrorString(cudaGetLastError()));
      if (rc) break;
      cudaEventRecord(e0, st);
      for (int k = 0; k < trial_steps && rc == PPML_OK; k++)
        rc = g->d.dtype == PPML_F64
                 ? run_step<double>(g, k % 2 ? &sb : &sa, k % 2 ? &sa : &sb, nullptr, 0.0, &g->dev->dt, st)
                 : run_step<float>(g, k % 2 ? &sb : &sa, k % 2 ? &sa : &sb, nullptr, 0.0, &g->dev->dt, st);
      if (rc) break;
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = ppml_fail(PPML_E_CUDA, "tuning timing: %s", cudaGetErrorString(cudaGetLastError()));
      if (rep == 0 || ms < best_k) best_k = ms;
    }
    if (rc) break;
    if (ms_out) ms_out[order] = best_k;
    if (order == 0 || best_k < best_ms) {
      best_ms = best_k;
      best = order;
    }
  }
  if (rc == PPML_OK &&
      (cudaMemcpyAsync(g->dev, &keep, sizeof(keep), cudaMemcpyHostToDevice, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = ppml_fail(PPML_E_CUDA, "tuning restore: %s", cudaGetErrorString(cudaGetLastError()));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int q = 0; q < 12; q++)
    if (buf[q]) cudaFree(buf[q]);
  g->profiling = prof;
  ppml_grid_set_order(g, rc == PPML_OK ? best : order0);
  if (rc) return rc;
  if (order_out) *order_out = best;
  return PPML_OK;
}

// ----------------------------------------------------------------- z-slab decomposition

extern "C" int ppml_local_reduce(ppml_grid* g, const ppml_state* u, double* red, void* stream) {
  ppml_clear_error();
  if (!g || !red) return ppml_fail(PPML_E_INVAL, "grid or red is NULL");
  int rc = ppml_validate_state(u, "u");
  if (rc) return rc;
  rc = check_state_type(&g->d, u, "u");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  MarchArgs<double> A64 = make_args<double>(g, 0.0, nullptr);
  MarchArgs<float> A32 = make_args<float>(g, 0.0, nullptr);
  for (int f = 0; f < 6; f++) {
    A64.u[f] = (const double*)u->f[f];
    A32.u[f] = (const float*)u->f[f];
  }
  for (int f = 0; f < 5; f++) A32.ulo[f] = (const float*)u->lo[f];
  rc = g->d.dtype == PPML_F64 ? launch_diag<double>(A64, g->nblk_diag, st)
                              : launch_diag<float>(A32, g->nblk_diag, st);
  if (rc) return rc;
  return launch_finalize(g->partials, g->nblk_diag, g->dev, g->d.cfl, g->hmin, g->vol,
                         g->d.t_end, 2, nullptr, 0.0, st, red);
}

extern "C" int ppml_lagrangian_stage(ppml_grid* g, const ppml_state* u_star, ppml_state* u_out,
                                     double dt, double* red, void* stream) {
  ppml_clear_error();
  if (!g || !red) return ppml_fail(PPML_E_INVAL, "grid or red is NULL");
  int rc = ppml_validate_state(u_star, "u_star");
  if (rc) return rc;
  rc = ppml_validate_state(u_out, "u_out");
  if (rc) return rc;
  rc = check_state_pair(&g->d, u_star, u_out);
  if (rc) return rc;
  if (!isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt is not finite");
  const double* dt_dev = dt > 0.0 ? nullptr : &g->dev->dt;
  cudaStream_t st = (cudaStream_t)stream;
  if (g->d.dtype == PPML_F64) {
    MarchArgs<double> L = make_args<double>(g, dt, dt_dev);
    for (int f = 0; f < 6; f++) {
      L.u[f] = (const double*)u_star->f[f];
      L.out[f] = (double*)u_out->f[f];
    }
    rc = launch_lagrangian<double>(L, g->nblk_launch, st);
  } else {
    MarchArgs<float> L = make_args<float>(g, dt, dt_dev);
    for (int f = 0; f < 6; f++) {
      L.u[f] = (const float*)u_star->f[f];
      L.out[f] = (float*)u_out->f[f];
    }
    if (ppml_state_has_lo(u_star))
      for (int f = 0; f < 5; f++) {
        L.ulo[f] = (const float*)u_star->lo[f];
        L.outlo[f] = (float*)u_out->lo[f];
      }
    rc = launch_lagrangian<float>(L, g->nblk_launch, st);
  }
  if (rc) return rc;
  return launch_finalize(g->partials, g->nblk_march, g->dev, g->d.cfl, g->hmin, g->vol,
                         g->d.t_end, 2, dt_dev, dt, st, red);
}

extern "C" int ppml_apply_reduced(ppml_grid* g, const double* red, int advance, double dt,
                                  void* stream) {
  ppml_clear_error();
  if (!g || !red) return ppml_fail(PPML_E_INVAL, "grid or red is NULL");
  if (!isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt is not finite");
  const double* dt_dev = dt > 0.0 ? nullptr : &g->dev->dt;
  apply_reduced_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(red, g->dev, advance ? 1 : 0, dt_dev, dt,
                                                           g->d.cfl, g->hmin, g->d.t_end);
  return ppml_check_launch("apply_reduced_kernel");
}
