// Grid path of libppml.so: one PPML operator-splitting step on a 3D uniform grid
// (Kulikov & Vorobyov, arXiv:1607.01105, Sec. 1), hand-written for sm_103a.
//
// Per step, on one stream:
//   eulerian_kernel    S0-S3: boundary-mapped loads of U^n, PPML parabolas of v and p per
//                      axis, acoustic face solve, unsplit update of m, rho E, rho eps -> U*
//   lagrangian_kernel  S4-S8 (+S10/S11 partials): boundary-mapped loads of U*, 9-point
//                      velocity template, Roe-weighted face velocity, upwind parabola
//                      fluxes of all six fields, unsplit update, energy correction, and
//                      per-block partial maxima / FP64 sums of U^{n+1}
//   finalize_kernel    deterministic reduction of the partials -> device-resident dt,
//                      sums, time and flags
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "../../include/ppml.h"
#include "ppml_device.cuh"
#include "ppml_internal.h"

using namespace ppml;

namespace {

constexpr int kThreads = 256;

struct Partial {
  double s[6];
  double vmax, cmax;
  unsigned long long nvac, nbad;
};

struct DevScalars {
  double t, dt, vmax, cmax, sums[6];
  long long steps, n_vac, n_bad;
  unsigned flags, pad;
};

template <typename T>
struct StepArgs {
  const T* u[6];   // U^n (or U* for the Lagrangian kernel: u[0] = rho^n, u[1..5] = U*)
  T* out[6];       // destination (out[0] may be NULL: rho is not rewritten)
  const T* phi;    // optional gravitational potential (Eulerian stage)
  GridGeom g;
  double h[3];
  double gamma;
  double dt_host;  // used when dt_dev == NULL
  const double* dt_dev;
  double rho_vac;
  Partial* partials;
};

__device__ __forceinline__ double step_tau(const double* dt_dev, double dt_host) {
  return dt_dev ? *dt_dev : dt_host;
}

__device__ __forceinline__ void cell_coords(long long idx, const GridGeom& g, int& i, int& j,
                                            int& k) {
  k = (int)(idx / g.nxy);
  long long r = idx - (long long)k * g.nxy;
  j = (int)(r / g.n[0]);
  i = (int)(r - (long long)j * g.n[0]);
}

// ------------------------------------------------------------------ block reduction

__device__ __forceinline__ void block_reduce_store(double s[6], double vmax, double cmax,
                                                   unsigned long long nvac,
                                                   unsigned long long nbad, Partial* out) {
  __shared__ double sh[kThreads / 32][8];
  __shared__ unsigned long long shc[kThreads / 32][2];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int f = 0; f < 6; f++) s[f] += __shfl_down_sync(0xffffffffu, s[f], o);
    vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    cmax = fmax(cmax, __shfl_down_sync(0xffffffffu, cmax, o));
    nvac += __shfl_down_sync(0xffffffffu, nvac, o);
    nbad += __shfl_down_sync(0xffffffffu, nbad, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    for (int f = 0; f < 6; f++) sh[w][f] = s[f];
    sh[w][6] = vmax;
    sh[w][7] = cmax;
    shc[w][0] = nvac;
    shc[w][1] = nbad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial p;
    for (int f = 0; f < 6; f++) p.s[f] = 0.0;
    p.vmax = 0.0;
    p.cmax = 0.0;
    p.nvac = 0;
    p.nbad = 0;
    for (int q = 0; q < kThreads / 32; q++) {
      for (int f = 0; f < 6; f++) p.s[f] += sh[q][f];
      p.vmax = fmax(p.vmax, sh[q][6]);
      p.cmax = fmax(p.cmax, sh[q][7]);
      p.nvac += shc[q][0];
      p.nbad += shc[q][1];
    }
    out[blockIdx.x] = p;
  }
}

// Per-cell diagnostics of an output state (S10/S11 and the non-physical check).
template <typename T>
__device__ __forceinline__ void cell_diag(const T u[6], double gamma, double s[6], double& vmax,
                                          double& cmax, unsigned long long& nbad) {
  const T rho = u[0];
  const T vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
  const T v = sqrt(vx * vx + vy * vy + vz * vz);
  const T p = T(gamma - 1.0) * u[5];
  const T c = sqrt(T(gamma) * p / rho);
  bool ok = rho > T(0) && u[5] > T(0);
#pragma unroll
  for (int f = 0; f < 6; f++) {
    s[f] += (double)u[f];
    ok = ok && isfinite((double)u[f]);
  }
  if (ok) {
    vmax = fmax(vmax, (double)v);
    cmax = fmax(cmax, (double)c);
  } else {
    nbad++;
  }
}

// ------------------------------------------------------------------ Eulerian stage

template <typename T>
__global__ void __launch_bounds__(kThreads) eulerian_kernel(StepArgs<T> A) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.g.ncell) return;
  int i, j, k;
  cell_coords(idx, A.g, i, j, k);
  const double tau = step_tau(A.dt_dev, A.dt_host);
  const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);
  const T rho0 = A.u[0][idx];
  T m0[3] = {A.u[1][idx], A.u[2][idx], A.u[3][idx]};
  const T en0 = A.u[4][idx], ei0 = A.u[5][idx];
  T dm[3] = {T(0), T(0), T(0)};
  T dpv = T(0), dv = T(0);
#pragma unroll 1
  for (int a = 0; a < 3; a++) {
    if (A.g.n[a] == 1) continue;
    const T th = T(tau / A.h[a]);
    T r[7], v[7], p[7];
#pragma unroll
    for (int o = -3; o <= 3; o++) {
      const int ci = i + (a == 0 ? o : 0), cj = j + (a == 1 ? o : 0), ck = k + (a == 2 ? o : 0);
      r[o + 3] = load_bc(A.u[0], 0, ci, cj, ck, A.g);
      v[o + 3] = load_bc(A.u[1 + a], 1 + a, ci, cj, ck, A.g) / r[o + 3];
      p[o + 3] = gm1 * load_bc(A.u[5], 5, ci, cj, ck, A.g);
    }
    Parab<T> Pv[3], Pp[3];
    window_parabolas(v, Pv);
    window_parabolas(p, Pp);
    T Vm, Pm, Vp, Pq;
    face_riemann(r[2], r[3], p[2], p[3], Pv[0], Pv[1], Pp[0], Pp[1], gamma, th, Vm, Pm);
    face_riemann(r[3], r[4], p[3], p[4], Pv[1], Pv[2], Pp[1], Pp[2], gamma, th, Vp, Pq);
    dm[a] = th * (Pq - Pm);
    dpv += th * (Pq * Vp - Pm * Vm);
    dv += th * (Vp - Vm);
  }
  T mo[3], eno = en0 - dpv;
#pragma unroll
  for (int a = 0; a < 3; a++) mo[a] = m0[a] - dm[a];
  if (A.phi) {
    // gravity source (central difference of Phi), from U^n
#pragma unroll 1
    for (int a = 0; a < 3; a++) {
      if (A.g.n[a] == 1) continue;
      const int di = a == 0, dj = a == 1, dk = a == 2;
      const T pp = load_bc(A.phi, -1, i + di, j + dj, k + dk, A.g);
      const T pm = load_bc(A.phi, -1, i - di, j - dj, k - dk, A.g);
      const T grad = (pp - pm) / T(2.0 * A.h[a]);
      mo[a] -= T(tau) * rho0 * grad;
      eno -= T(tau) * m0[a] * grad;
    }
  }
  if (A.out[0]) A.out[0][idx] = rho0;
  A.out[1][idx] = mo[0];
  A.out[2][idx] = mo[1];
  A.out[3][idx] = mo[2];
  A.out[4][idx] = eno;
  A.out[5][idx] = ei0 - gm1 * ei0 * dv;
}

// ---------------------------------------------------------------- Lagrangian stage

template <typename T>
__global__ void __launch_bounds__(kThreads) lagrangian_kernel(StepArgs<T> A) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s[6] = {0, 0, 0, 0, 0, 0};
  double vmax = 0.0, cmax = 0.0;
  unsigned long long nvac = 0, nbad = 0;
  if (idx < A.g.ncell) {
    int i, j, k;
    cell_coords(idx, A.g, i, j, k);
    const double tau = step_tau(A.dt_dev, A.dt_host);
    T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll 1
    for (int a = 0; a < 3; a++) {
      if (A.g.n[a] == 1) continue;
      const int b = (a + 1) % 3, c = (a + 2) % 3;
      const T th = T(tau / A.h[a]);
      // S5: 9-point template of v_a in the plane normal to a, at cells -1, 0, +1 along a
      T vt[3], sq[3];
#pragma unroll
      for (int o = -1; o <= 1; o++) {
        int base[3] = {i, j, k};
        base[a] += o;
        T vv[3][3];
#pragma unroll
        for (int db = -1; db <= 1; db++)
#pragma unroll
          for (int dc = -1; dc <= 1; dc++) {
            int cc[3] = {base[0], base[1], base[2]};
            cc[b] += db;
            cc[c] += dc;
            const T rr = load_bc(A.u[0], 0, cc[0], cc[1], cc[2], A.g);
            vv[db + 1][dc + 1] = load_bc(A.u[1 + a], 1 + a, cc[0], cc[1], cc[2], A.g) / rr;
            if (db == 0 && dc == 0) sq[o + 1] = sqrt(rr);
          }
        const T corners = vv[2][2] + vv[2][0] + vv[0][2] + vv[0][0];
        const T edges = vv[2][1] + vv[0][1] + vv[1][2] + vv[1][0];
        vt[o + 1] = corners * T(0.0625) + edges * T(0.125) + vv[1][1] * T(0.25);
      }
      const T vhm = (vt[1] * sq[1] + vt[0] * sq[0]) / (sq[1] + sq[0]);
      const T vhp = (vt[2] * sq[2] + vt[1] * sq[1]) / (sq[2] + sq[1]);
      // S6/S7: fluxes of every field along a
#pragma unroll 1
      for (int f = 0; f < 6; f++) {
        T q[7];
#pragma unroll
        for (int o = -3; o <= 3; o++) {
          int cc[3] = {i, j, k};
          cc[a] += o;
          q[o + 3] = load_bc(A.u[f], f, cc[0], cc[1], cc[2], A.g);
        }
        Parab<T> P[3];
        window_parabolas(q, P);
        const T Fm = upwind_flux(vhm, P[0], P[1], th);
        const T Fp = upwind_flux(vhp, P[1], P[2], th);
        acc[f] += th * (Fp - Fm);
      }
    }
    T un[6];
#pragma unroll
    for (int f = 0; f < 6; f++) un[f] = A.u[f][idx] - acc[f];
    // S8: energy consistency in double
    double ud[6];
#pragma unroll
    for (int f = 0; f < 6; f++) ud[f] = (double)un[f];
    nvac = energy_correction(ud, A.rho_vac);
#pragma unroll
    for (int f = 1; f < 6; f++) un[f] = (T)ud[f];
#pragma unroll
    for (int f = 0; f < 6; f++) A.out[f][idx] = un[f];
    cell_diag(un, A.gamma, s, vmax, cmax, nbad);
  }
  block_reduce_store(s, vmax, cmax, nvac, nbad, A.partials);
}

// ------------------------------------------------------------ standalone diagnostics

template <typename T>
__global__ void __launch_bounds__(kThreads) diag_kernel(StepArgs<T> A) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s[6] = {0, 0, 0, 0, 0, 0};
  double vmax = 0.0, cmax = 0.0;
  unsigned long long nbad = 0;
  if (idx < A.g.ncell) {
    T u[6];
#pragma unroll
    for (int f = 0; f < 6; f++) u[f] = A.u[f][idx];
    cell_diag(u, A.gamma, s, vmax, cmax, nbad);
  }
  block_reduce_store(s, vmax, cmax, 0ull, nbad, A.partials);
}

// Reduce nblk partials in a fixed order (independent of scheduling) and update the
// device scalars.  mode: 0 = diagnostics only (dt from state), 1 = after a step.
__global__ void __launch_bounds__(512) finalize_kernel(const Partial* __restrict__ P, int nblk,
                                                       DevScalars* S, double cfl, double hmin,
                                                       double vol, double t_end, int mode,
                                                       const double* dt_dev, double dt_host) {
  __shared__ double sh[512][8];
  __shared__ unsigned long long shc[512][2];
  const int t = threadIdx.x;
  double tau = 0.0;
  if (t == 0 && mode == 1) tau = dt_dev ? *dt_dev : dt_host;
  double s[6] = {0, 0, 0, 0, 0, 0}, vmax = 0.0, cmax = 0.0;
  unsigned long long nvac = 0, nbad = 0;
  for (int b = t; b < nblk; b += 512) {
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
  for (int w = 256; w > 0; w >>= 1) {
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
    double tn = S->t;
    if (mode == 1) {
      tn = S->t + tau;
      if (t_end > 0.0 && tn > t_end) tn = t_end;
      S->t = tn;
      S->steps += 1;
      S->n_vac = (long long)shc[0][0];
    }
    S->vmax = sh[0][6];
    S->cmax = sh[0][7];
    for (int f = 0; f < 6; f++) S->sums[f] = sh[0][f] * vol;
    S->n_bad = (long long)shc[0][1];
    double dt = cfl * hmin / (sh[0][6] + sh[0][7]);
    if (t_end > 0.0 && dt > t_end - tn) dt = t_end - tn;
    if (!(dt > 0.0)) {
      dt = 0.0;
      S->flags |= PPML_FLAG_DT_ZERO;
    }
    S->dt = dt;
    if (shc[0][1]) S->flags |= PPML_FLAG_NONPHYSICAL;
  }
}

}  // namespace

// ======================================================================= host side

struct ppml_grid {
  ppml_grid_desc d;
  GridGeom geom;
  size_t elt;
  void* ustar[6];  // [0] unused (rho is not changed by the Eulerian stage)
  Partial* partials;
  int nblk;
  DevScalars* dev;
  double rho_mean, rho_vac, hmin, vol;
  int device;
  // measurement hook: events around each kernel of a step (pairs per step, pooled)
  int profiling;
  static const int kEvSlots = 4096;
  cudaEvent_t* ev;      // kEvSlots * 4 events
  int ev_used;          // steps recorded but not yet folded into ms
  double ms[3];
  long long prof_steps;
};

namespace {

int validate_desc(const ppml_grid_desc* d) {
  if (!d) return ppml_fail(PPML_E_INVAL, "desc is NULL");
  const int n[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; a++) {
    if (n[a] < 1) return ppml_fail(PPML_E_INVAL, "axis %d has %d cells (need >= 1)", a, n[a]);
    if (!(d->h[a] > 0.0) || !isfinite(d->h[a]))
      return ppml_fail(PPML_E_INVAL, "h[%d] = %g must be positive", a, d->h[a]);
    const int lo = d->bc[2 * a], hi = d->bc[2 * a + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2)
      return ppml_fail(PPML_E_INVAL, "bc of axis %d is not a ppml_bc", a);
    if ((lo == PPML_BC_PERIODIC) != (hi == PPML_BC_PERIODIC))
      return ppml_fail(PPML_E_INVAL, "periodic bc on axis %d must be set on both faces", a);
    if (n[a] == 1 && (lo == PPML_BC_REFLECT || hi == PPML_BC_REFLECT))
      return ppml_fail(PPML_E_INVAL, "inactive axis %d cannot be reflecting", a);
    if (n[a] > 1 && n[a] < 3)
      return ppml_fail(PPML_E_INVAL, "axis %d has %d cells (active axes need >= 3)", a, n[a]);
  }
  if (!(d->gamma > 1.0) || !isfinite(d->gamma))
    return ppml_fail(PPML_E_INVAL, "gamma = %g must be > 1", d->gamma);
  if (!(d->cfl > 0.0 && d->cfl < 1.0)) return ppml_fail(PPML_E_INVAL, "cfl = %g not in (0,1)", d->cfl);
  if (d->dtype != PPML_F32 && d->dtype != PPML_F64)
    return ppml_fail(PPML_E_INVAL, "dtype %d is not a ppml_dtype", d->dtype);
  const long long nc = (long long)n[0] * n[1] * n[2];
  if (nc > (1ll << 31) - 1024) return ppml_fail(PPML_E_INVAL, "grid of %lld cells is too large", nc);
  return PPML_OK;
}

int validate_state(const ppml_grid* g, const ppml_state* u, const char* what, bool need_rho) {
  if (!u) return ppml_fail(PPML_E_INVAL, "%s is NULL", what);
  for (int f = 0; f < 6; f++) {
    if (f == 0 && !need_rho) continue;
    if (!u->f[f]) return ppml_fail(PPML_E_INVAL, "%s field %d is NULL", what, f);
    if (((uintptr_t)u->f[f]) & 15u)
      return ppml_fail(PPML_E_INVAL, "%s field %d is not 16-byte aligned", what, f);
  }
  (void)g;
  return PPML_OK;
}

template <typename T>
StepArgs<T> make_args(const ppml_grid* g, double dt_host, const double* dt_dev) {
  StepArgs<T> A;
  memset(&A, 0, sizeof(A));
  A.g = g->geom;
  for (int a = 0; a < 3; a++) A.h[a] = g->d.h[a];
  A.gamma = g->d.gamma;
  A.dt_host = dt_host;
  A.dt_dev = dt_dev;
  A.rho_vac = g->rho_vac;
  A.partials = g->partials;
  return A;
}

template <typename T>
int launch_diag(ppml_grid* g, const ppml_state* u, cudaStream_t st) {
  StepArgs<T> A = make_args<T>(g, 0.0, nullptr);
  for (int f = 0; f < 6; f++) A.u[f] = (const T*)u->f[f];
  diag_kernel<T><<<g->nblk, kThreads, 0, st>>>(A);
  finalize_kernel<<<1, 512, 0, st>>>(g->partials, g->nblk, g->dev, g->d.cfl, g->hmin, g->vol,
                                     g->d.t_end, 0, nullptr, 0.0);
  return ppml_check_launch("diagnostics");
}

template <typename T>
int launch_eulerian(ppml_grid* g, const ppml_state* u, void* const out[6], const T* phi,
                    double dt_host, const double* dt_dev, cudaStream_t st) {
  StepArgs<T> A = make_args<T>(g, dt_host, dt_dev);
  for (int f = 0; f < 6; f++) {
    A.u[f] = (const T*)u->f[f];
    A.out[f] = (T*)out[f];
  }
  A.phi = phi;
  eulerian_kernel<T><<<g->nblk, kThreads, 0, st>>>(A);
  return ppml_check_launch("eulerian_kernel");
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
int launch_step(ppml_grid* g, const ppml_state* uin, ppml_state* uout, double dt_host,
                const double* dt_dev, cudaStream_t st) {
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
  int rc = launch_eulerian<T>(g, uin, star, nullptr, dt_host, dt_dev, st);
  if (rc) return rc;
  if (ev) cudaEventRecord(ev[1], st);
  StepArgs<T> L = make_args<T>(g, dt_host, dt_dev);
  L.u[0] = (const T*)uin->f[0];
  for (int f = 1; f < 6; f++) L.u[f] = (const T*)g->ustar[f];
  for (int f = 0; f < 6; f++) L.out[f] = (T*)uout->f[f];
  lagrangian_kernel<T><<<g->nblk, kThreads, 0, st>>>(L);
  rc = ppml_check_launch("lagrangian_kernel");
  if (rc) return rc;
  if (ev) cudaEventRecord(ev[2], st);
  finalize_kernel<<<1, 512, 0, st>>>(g->partials, g->nblk, g->dev, g->d.cfl, g->hmin, g->vol,
                                     g->d.t_end, 1, dt_dev, dt_host);
  rc = ppml_check_launch("finalize_kernel");
  if (ev) cudaEventRecord(ev[3], st);
  return rc;
}

}  // namespace

extern "C" int ppml_init_grid(const ppml_grid_desc* d, const ppml_state* u0, void* stream,
                              ppml_grid** out) {
  ppml_clear_error();
  if (!out) return ppml_fail(PPML_E_INVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_desc(d);
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
  g->nblk = (int)((g->geom.ncell + kThreads - 1) / kThreads);
  g->hmin = INFINITY;
  const int n[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; a++)
    if (n[a] > 1 && d->h[a] < g->hmin) g->hmin = d->h[a];
  if (!isfinite(g->hmin)) g->hmin = d->h[0];
  g->vol = d->h[0] * d->h[1] * d->h[2];
  cudaGetDevice(&g->device);
  rc = validate_state(g, u0, "u0", true);
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
  if (cudaMalloc(&g->partials, sizeof(Partial) * (size_t)g->nblk) != cudaSuccess ||
      cudaMalloc(&g->dev, sizeof(DevScalars)) != cudaSuccess) {
    ppml_free_grid(g);
    return ppml_fail(PPML_E_NOMEM, "cudaMalloc of reduction scratch failed");
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(g->dev, 0, sizeof(DevScalars), st);
  rc = d->dtype == PPML_F64 ? launch_diag<double>(g, u0, st) : launch_diag<float>(g, u0, st);
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
  g->rho_mean = hs.sums[0] / (g->vol * (double)g->geom.ncell);
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
  if (g->partials) cudaFree(g->partials);
  if (g->dev) cudaFree(g->dev);
  if (g->ev) {
    for (int q = 0; q < 4 * ppml_grid::kEvSlots; q++) cudaEventDestroy(g->ev[q]);
    delete[] g->ev;
  }
  delete g;
  return PPML_OK;
}

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

extern "C" int ppml_cfl_dt(ppml_grid* g, const ppml_state* u, double* dt_host, void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = validate_state(g, u, "u", true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = g->d.dtype == PPML_F64 ? launch_diag<double>(g, u, st) : launch_diag<float>(g, u, st);
  if (rc) return rc;
  if (dt_host) {
    if (cudaMemcpyAsync(dt_host, &g->dev->dt, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "cfl_dt: %s", cudaGetErrorString(cudaGetLastError()));
  }
  return PPML_OK;
}

extern "C" int ppml_step(ppml_grid* g, const ppml_state* u_in, ppml_state* u_out, double dt,
                         void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = validate_state(g, u_in, "u_in", true);
  if (rc) return rc;
  rc = validate_state(g, u_out, "u_out", true);
  if (rc) return rc;
  for (int f = 0; f < 6; f++)
    for (int q = 0; q < 6; q++)
      if (u_in->f[f] == u_out->f[q]) return ppml_fail(PPML_E_INVAL, "u_in and u_out alias");
  if (!isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt is not finite");
  const double* dt_dev = dt > 0.0 ? nullptr : &g->dev->dt;
  cudaStream_t st = (cudaStream_t)stream;
  return g->d.dtype == PPML_F64 ? launch_step<double>(g, u_in, u_out, dt, dt_dev, st)
                                : launch_step<float>(g, u_in, u_out, dt, dt_dev, st);
}

extern "C" int ppml_eulerian_stage(ppml_grid* g, const ppml_state* u_in, ppml_state* u_star,
                                   double dt, void* stream) {
  ppml_clear_error();
  if (!g) return ppml_fail(PPML_E_INVAL, "grid is NULL");
  int rc = validate_state(g, u_in, "u_in", true);
  if (rc) return rc;
  rc = validate_state(g, u_star, "u_star", true);
  if (rc) return rc;
  if (!isfinite(dt)) return ppml_fail(PPML_E_INVAL, "dt is not finite");
  const double* dt_dev = dt > 0.0 ? nullptr : &g->dev->dt;
  cudaStream_t st = (cudaStream_t)stream;
  return g->d.dtype == PPML_F64
             ? launch_eulerian<double>(g, u_in, u_star->f, nullptr, dt, dt_dev, st)
             : launch_eulerian<float>(g, u_in, u_star->f, nullptr, dt, dt_dev, st);
}

extern "C" int ppml_conserved_sums(ppml_grid* g, const ppml_state* u, double out[6],
                                   void* stream) {
  ppml_clear_error();
  if (!g || !out) return ppml_fail(PPML_E_INVAL, "grid or out is NULL");
  // Sums go through the same partial/finalize path; the handle's dt and t are kept.
  DevScalars keep;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&keep, g->dev, sizeof(keep), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "sums: %s", cudaGetErrorString(cudaGetLastError()));
  int rc = validate_state(g, u, "u", true);
  if (rc) return rc;
  rc = g->d.dtype == PPML_F64 ? launch_diag<double>(g, u, st) : launch_diag<float>(g, u, st);
  if (rc) return rc;
  DevScalars hs;
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
