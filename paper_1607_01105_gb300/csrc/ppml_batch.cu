// Batched independent 1D problems (many shock tubes of uneven lengths) advanced by one
// persistent launch: each CTA owns one instance, keeps its four fields (rho, m, rho E,
// rho eps) resident in shared memory for all of its steps, takes its own CFL step from a
// CTA-local reduction (Sec. 1.1) and stops at its own end time.  The scheme per step is
// the 1D case of Sec. 1 (Eulerian face solve, upwind Lagrangian fluxes with
// v~ = v, energy correction of Sec. 1.4).  Outflow boundaries on both ends.  CTAs never
// wait on one another, so nothing can hang across the grid.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/ppml.h"
#include "ppml_device.cuh"
#include "ppml_internal.h"

using namespace ppml;

namespace {

constexpr int kBatchThreads = 512;
constexpr int kGhost = 3;

struct InstDev {
  long long off;   // first cell in the packed arrays
  int n;           // cells
  int steps;       // steps taken so far
  double h, t_end, t, rho_vac;
  int done, pad;
};

// Parabolas of the cells left and right of a face from the six values q[0..5] around it
// (face between q[2] and q[3]): Appendix Steps 1-3.
template <typename T>
__device__ __forceinline__ void pair_parabolas(const T q[6], Parab<T>& PL, Parab<T>& PR) {
  T d[4];
#pragma unroll
  for (int k = 1; k <= 4; k++) d[k - 1] = limited_slope(q[k - 1], q[k], q[k + 1]);
  const T f12 = face_value(q[1], q[2], d[0], d[1]);
  const T f23 = face_value(q[2], q[3], d[1], d[2]);
  const T f34 = face_value(q[3], q[4], d[2], d[3]);
  PL = parabola(q[2], f12, f23);
  PR = parabola(q[3], f23, f34);
}

template <typename T>
__device__ __forceinline__ void fill_ghosts(T* q, int n) {
  const int t = threadIdx.x;
  if (t < kGhost) q[t] = q[kGhost];
  else if (t < 2 * kGhost) q[n + kGhost + (t - kGhost)] = q[n + kGhost - 1];
}

template <typename T>
__device__ double block_max2(double a, double b, double* sh) {
  // returns max(a) + max(b) over the block (CFL denominator); sh holds 2*32 doubles
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[w] = a;
    sh[32 + w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
      A = fmax(A, sh[q]);
      B = fmax(B, sh[32 + q]);
    }
    sh[64] = A + B;
  }
  __syncthreads();
  const double r = sh[64];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(T* __restrict__ g_rho,
                                                              T* __restrict__ g_m,
                                                              T* __restrict__ g_en,
                                                              T* __restrict__ g_ei,
                                                              InstDev* __restrict__ inst,
                                                              const int* __restrict__ order,
                                                              int* __restrict__ done_count,
                                                              double gamma_d, double cfl,
                                                              int max_steps, int nmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[80];
  const int id = order[blockIdx.x];
  InstDev I = inst[id];
  if (I.done) return;
  const int n = I.n, np = n + 2 * kGhost;
  const int stride = nmax + 2 * kGhost;
  T* R = (T*)smem_raw;
  T* M = R + stride;
  T* E = M + stride;
  T* Ei = E + stride;
  T* FA = Ei + stride;       // face array A (V, then v hat)
  T* FB = FA + (nmax + 1);   // face array B (P, then fluxes)
  const int tid = threadIdx.x;
  for (int c = tid; c < n; c += blockDim.x) {
    R[c + kGhost] = g_rho[I.off + c];
    M[c + kGhost] = g_m[I.off + c];
    E[c + kGhost] = g_en[I.off + c];
    Ei[c + kGhost] = g_ei[I.off + c];
  }
  __syncthreads();
  const T gamma = T(gamma_d), gm1 = T(gamma_d - 1.0);
  if (I.steps == 0 && I.rho_vac < 0.0) {
    // vacuum threshold reference: the instance's mean initial density
    double s = 0.0;
    for (int c = tid; c < n; c += blockDim.x) s += (double)R[c + kGhost];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      double S = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); q++) S += red[q];
      red[79] = S / n;
    }
    __syncthreads();
    I.rho_vac = -I.rho_vac * red[79];  // stored negated fraction before the first call
    __syncthreads();
  }
  int s = 0;
  for (; s < max_steps; s++) {
    // CFL step of the current state (Sec. 1.1)
    double vm = 0.0, cm = 0.0;
    for (int c = tid; c < n; c += blockDim.x) {
      const T r = R[c + kGhost];
      const T v = M[c + kGhost] / r;
      const T cs = sqrt(gamma * gm1 * Ei[c + kGhost] / r);
      vm = fmax(vm, (double)tabs(v));
      cm = fmax(cm, (double)cs);
    }
    const double den = block_max2<T>(vm, cm, red);
    double dt = cfl * I.h / den;
    if (dt > I.t_end - I.t) dt = I.t_end - I.t;
    if (!(dt > 0.0)) {
      I.done = 1;
      break;
    }
    const T th = T(dt / I.h);
    fill_ghosts(R, n);
    fill_ghosts(M, n);
    fill_ghosts(E, n);
    fill_ghosts(Ei, n);
    __syncthreads();
    // Eulerian stage: faces f = 0..n between padded cells f+2 and f+3
    for (int f = tid; f <= n; f += blockDim.x) {
      T v[6], p[6];
#pragma unroll
      for (int q = 0; q < 6; q++) {
        v[q] = M[f + q] / R[f + q];
        p[q] = gm1 * Ei[f + q];
      }
      Parab<T> vL, vR, pL, pR;
      pair_parabolas(v, vL, vR);
      pair_parabolas(p, pL, pR);
      T V, P;
      face_riemann(R[f + 2], R[f + 3], p[2], p[3], vL, vR, pL, pR, gamma, th, V, P);
      FA[f] = V;
      FB[f] = P;
    }
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) {
      const int g = c + kGhost;
      const T Vm = FA[c], Vp = FA[c + 1], Pm = FB[c], Pp = FB[c + 1];
      const T ei0 = Ei[g];
      M[g] = M[g] - th * (Pp - Pm);
      E[g] = E[g] - th * (Pp * Vp - Pm * Vm);
      Ei[g] = ei0 - gm1 * ei0 * (th * (Vp - Vm));
    }
    __syncthreads();
    fill_ghosts(M, n);
    fill_ghosts(E, n);
    fill_ghosts(Ei, n);
    __syncthreads();
    // Lagrangian stage: v hat at faces (1D: v~ = v), then each field's flux and update
    for (int f = tid; f <= n; f += blockDim.x) {
      const T rl = R[f + 2], rr = R[f + 3];
      const T sl = sqrt(rl), sr = sqrt(rr);
      FA[f] = ((M[f + 3] / rr) * sr + (M[f + 2] / rl) * sl) / (sr + sl);
    }
    __syncthreads();
    T* fields[4] = {R, M, E, Ei};
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
      T* q = fields[k];
      for (int f = tid; f <= n; f += blockDim.x) {
        T w[6];
#pragma unroll
        for (int o = 0; o < 6; o++) w[o] = q[f + o];
        Parab<T> PL, PR;
        pair_parabolas(w, PL, PR);
        FB[f] = upwind_flux(FA[f], PL, PR, th);
      }
      __syncthreads();
      for (int c = tid; c < n; c += blockDim.x) q[c + kGhost] = q[c + kGhost] - th * (FB[c + 1] - FB[c]);
      __syncthreads();
    }
    // Sec. 1.4 energy consistency (double)
    for (int c = tid; c < n; c += blockDim.x) {
      const int g = c + kGhost;
      double u[6] = {(double)R[g], (double)M[g], 0.0, 0.0, (double)E[g], (double)Ei[g]};
      energy_correction(u, I.rho_vac);
      M[g] = (T)u[1];
      Ei[g] = (T)u[5];
    }
    __syncthreads();
    I.t = (I.t + dt > I.t_end) ? I.t_end : I.t + dt;
    I.steps += 1;
    if (I.t >= I.t_end) {
      I.done = 1;
      s++;
      break;
    }
  }
  (void)np;
  for (int c = tid; c < n; c += blockDim.x) {
    g_rho[I.off + c] = R[c + kGhost];
    g_m[I.off + c] = M[c + kGhost];
    g_en[I.off + c] = E[c + kGhost];
    g_ei[I.off + c] = Ei[c + kGhost];
  }
  if (tid == 0) {
    inst[id] = I;
    if (I.done) atomicAdd(done_count, 1);
  }
}

}  // namespace

struct ppml_batch {
  int n_inst, dtype, nmax;
  long long total;
  double gamma, cfl;
  InstDev* inst;
  int* order;
  int* done;
  size_t smem;
};

extern "C" int ppml_batch_init(int n_inst, const int* ncells, const double* h,
                               const double* t_end, double gamma, double cfl,
                               double vacuum_frac, int dtype, ppml_batch** out) {
  ppml_clear_error();
  if (!out) return ppml_fail(PPML_E_INVAL, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || !ncells || !h || !t_end)
    return ppml_fail(PPML_E_INVAL, "need n_inst >= 1 and non-NULL ncells, h, t_end");
  if (!(gamma > 1.0)) return ppml_fail(PPML_E_INVAL, "gamma = %g must be > 1", gamma);
  if (!(cfl > 0.0 && cfl < 1.0)) return ppml_fail(PPML_E_INVAL, "cfl = %g not in (0,1)", cfl);
  if (dtype != PPML_F32 && dtype != PPML_F64) return ppml_fail(PPML_E_INVAL, "bad dtype %d", dtype);
  if (!(vacuum_frac > 0.0)) vacuum_frac = 1e-5;
  const size_t elt = dtype == PPML_F64 ? 8 : 4;
  std::vector<InstDev> hi(n_inst);
  long long off = 0;
  int nmax = 0;
  for (int i = 0; i < n_inst; i++) {
    if (ncells[i] < 4) return ppml_fail(PPML_E_INVAL, "instance %d has %d cells (< 4)", i, ncells[i]);
    if (!(h[i] > 0.0) || !(t_end[i] > 0.0))
      return ppml_fail(PPML_E_INVAL, "instance %d: h and t_end must be positive", i);
    hi[i].off = off;
    hi[i].n = ncells[i];
    hi[i].steps = 0;
    hi[i].h = h[i];
    hi[i].t_end = t_end[i];
    hi[i].t = 0.0;
    hi[i].rho_vac = -vacuum_frac;  // fixed at the first step from the mean density
    hi[i].done = 0;
    hi[i].pad = 0;
    off += ncells[i];
    nmax = std::max(nmax, ncells[i]);
  }
  const size_t smem = (4 * (size_t)(nmax + 2 * kGhost) + 2 * (size_t)(nmax + 1)) * elt;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem + 1024 > (size_t)maxsm)
    return ppml_fail(PPML_E_INVAL, "largest instance (%d cells) needs %zu bytes of shared memory (> %d)",
                     nmax, smem, maxsm);
  // largest work first (work ~ n^2: cells x steps), so long instances start early
  std::vector<int> ord(n_inst);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return ncells[a] > ncells[b]; });
  ppml_batch* b = new (std::nothrow) ppml_batch();
  if (!b) return ppml_fail(PPML_E_NOMEM, "host allocation failed");
  b->n_inst = n_inst;
  b->dtype = dtype;
  b->nmax = nmax;
  b->total = off;
  b->gamma = gamma;
  b->cfl = cfl;
  b->smem = smem;
  if (cudaMalloc(&b->inst, sizeof(InstDev) * n_inst) != cudaSuccess ||
      cudaMalloc(&b->order, sizeof(int) * n_inst) != cudaSuccess ||
      cudaMalloc(&b->done, sizeof(int)) != cudaSuccess) {
    ppml_batch_free(b);
    return ppml_fail(PPML_E_NOMEM, "cudaMalloc of batch metadata failed");
  }
  if (cudaMemcpy(b->inst, hi.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->order, ord.data(), sizeof(int) * n_inst, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->done, 0, sizeof(int)) != cudaSuccess) {
    ppml_batch_free(b);
    return ppml_fail(PPML_E_CUDA, "batch init copy: %s", cudaGetErrorString(cudaGetLastError()));
  }
  cudaError_t e = dtype == PPML_F64
                      ? cudaFuncSetAttribute(batch_kernel<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(batch_kernel<float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    ppml_batch_free(b);
    return ppml_fail(PPML_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  }
  *out = b;
  return PPML_OK;
}

extern "C" int ppml_batch_step(ppml_batch* b, void* const state[4], int max_steps, int* done_host,
                               void* stream) {
  ppml_clear_error();
  if (!b || !state) return ppml_fail(PPML_E_INVAL, "batch or state is NULL");
  for (int f = 0; f < 4; f++) {
    if (!state[f]) return ppml_fail(PPML_E_INVAL, "state field %d is NULL", f);
    if (((uintptr_t)state[f]) & 15u) return ppml_fail(PPML_E_INVAL, "state field %d misaligned", f);
  }
  if (max_steps < 0) return ppml_fail(PPML_E_INVAL, "max_steps < 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(b->done, 0, sizeof(int), st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "memset: %s", cudaGetErrorString(cudaGetLastError()));
  if (b->dtype == PPML_F64)
    batch_kernel<double><<<b->n_inst, kBatchThreads, b->smem, st>>>(
        (double*)state[0], (double*)state[1], (double*)state[2], (double*)state[3], b->inst,
        b->order, b->done, b->gamma, b->cfl, max_steps, b->nmax);
  else
    batch_kernel<float><<<b->n_inst, kBatchThreads, b->smem, st>>>(
        (float*)state[0], (float*)state[1], (float*)state[2], (float*)state[3], b->inst, b->order,
        b->done, b->gamma, b->cfl, max_steps, b->nmax);
  int rc = ppml_check_launch("batch_kernel");
  if (rc) return rc;
  if (done_host) {
    // instances already finished before this call return early without counting: count
    // all finished instances from the metadata instead
    std::vector<InstDev> hi(b->n_inst);
    if (cudaMemcpyAsync(hi.data(), b->inst, sizeof(InstDev) * b->n_inst, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ppml_fail(PPML_E_CUDA, "batch status: %s", cudaGetErrorString(cudaGetLastError()));
    int d = 0;
    for (auto& x : hi) d += x.done;
    *done_host = d;
  }
  return PPML_OK;
}

extern "C" int ppml_batch_status(ppml_batch* b, double* t_host, int* steps_host, void* stream) {
  ppml_clear_error();
  if (!b) return ppml_fail(PPML_E_INVAL, "batch is NULL");
  std::vector<InstDev> hi(b->n_inst);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(hi.data(), b->inst, sizeof(InstDev) * b->n_inst, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "batch status: %s", cudaGetErrorString(cudaGetLastError()));
  for (int i = 0; i < b->n_inst; i++) {
    if (t_host) t_host[i] = hi[i].t;
    if (steps_host) steps_host[i] = hi[i].steps;
  }
  return PPML_OK;
}

extern "C" int ppml_batch_free(ppml_batch* b) {
  ppml_clear_error();
  if (!b) return PPML_OK;
  cudaDeviceSynchronize();
  if (b->inst) cudaFree(b->inst);
  if (b->order) cudaFree(b->order);
  if (b->done) cudaFree(b->done);
  delete b;
  return PPML_OK;
}
