// Shared pieces of the step kernels (Kulikov & Vorobyov, arXiv:1607.01105): kernel
// arguments, device-resident step scalars, deterministic per-CTA reductions of the CFL
// maxima (Sec. 1.1) and of the FP64 conservation sums, and the standalone
// diagnostics kernel.
#pragma once
#include "ppml_device.cuh"

namespace ppml {

constexpr int NT = 256;  // threads of the diagnostics kernel

struct Partial {
  double s[6];
  double vmax, cmax;
  unsigned long long nvac, nbad;
};

// Device-resident step scalars (one block per grid handle).
struct DevScalars {
  double t, dt, vmax, cmax, sums[6];
  long long steps, n_vac, n_bad;
  unsigned flags, pad;
};

template <typename T>
struct MarchArgs {
  const T* u[6];  // input fields
  T* out[6];      // output fields (out[0] NULL: rho is not written)
  // FP32 double-float states: low parts of rho, m_x, m_y, m_z, rho E of the input and the
  // output (all NULL for plain FP32 and FP64 states; outlo[0] NULL when out[0] is)
  const T* ulo[5];
  T* outlo[5];
  const T* phi;   // optional potential (Eulerian stage)
  GridGeom g;
  double h[3];
  double gamma;
  double dt_host;        // used when dt_dev == NULL
  const double* dt_dev;  // device-resident step
  double rho_vac;
  Partial* partials;      // per tile of the Lagrangian stage, at the tile's x-major index
  int tiles_x, tiles_y, tiles_z;  // tile grid of the stage kernels
  int tile_order;         // launch order of the tiles (TileOrder)
  int any_reflect;       // a reflecting wall exists (its sign flips need register copies)
  int flags;             // PPML_FIRST_ORDER, PPML_VHAT_1PT
  const T* inflow;       // [face][field]: the prescribed ghost states of inflow faces
  int any_inflow;        // an inflow face exists (selects the kernels that read them)
};

__device__ __forceinline__ double read_tau(const double* dt_dev, double dt_host) {
  return dt_dev ? *dt_dev : dt_host;
}

// The step size and tau / h per axis, formed by one thread of the CTA (three FP64
// divisions per CTA instead of per thread) and shared.  Contains a CTA barrier.
__device__ __forceinline__ void cta_step_constants(const double* dt_dev, double dt_host,
                                                   const double h[3], double out[4]) {
  __shared__ double s[4];
  if (threadIdx.x == 0) {
    const double tau = read_tau(dt_dev, dt_host);
    s[0] = tau;
    s[1] = tau / h[0];
    s[2] = tau / h[1];
    s[3] = tau / h[2];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; q++) out[q] = s[q];
}

// ------------------------------------------------------------------ block reduction

// Writes the CTA's partial to out[slot].
template <int NTHREADS>
__device__ __forceinline__ void block_reduce_store(double s[6], double vmax, double cmax,
                                                   unsigned long long nvac,
                                                   unsigned long long nbad, Partial* out,
                                                   int slot) {
  __shared__ double sh[NTHREADS / 32][8];
  __shared__ unsigned long long shc[NTHREADS / 32][2];
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
    for (int q = 0; q < NTHREADS / 32; q++) {
      for (int f = 0; f < 6; f++) p.s[f] += sh[q][f];
      p.vmax = fmax(p.vmax, sh[q][6]);
      p.cmax = fmax(p.cmax, sh[q][7]);
      p.nvac += shc[q][0];
      p.nbad += shc[q][1];
    }
    out[slot] = p;
  }
}

// (hi, lo) += (bh, bl) in double-float (TwoSum of the high parts, then renormalised).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

// block_reduce_store for the FP32 stage kernels: the warp level of the sums runs in
// double-float (FP32 operations only), the maxima in float (exact) and the counters in
// 32 bits; warp leaders convert to double and thread 0 folds the warps in a fixed order.
template <int NTHREADS>
__device__ __forceinline__ void block_reduce_store_f32(const float hi_in[6], const float lo_in[6],
                                                       float vmax, float cmax, unsigned nvac,
                                                       unsigned nbad, Partial* out, int slot) {
  float hi[6], lo[6];
#pragma unroll
  for (int f = 0; f < 6; f++) {
    hi[f] = hi_in[f];
    lo[f] = lo_in[f];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int f = 0; f < 6; f++) {
      const float bh = __shfl_down_sync(0xffffffffu, hi[f], o);
      const float bl = __shfl_down_sync(0xffffffffu, lo[f], o);
      ff_add(hi[f], lo[f], bh, bl);
    }
    vmax = fmaxf(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    cmax = fmaxf(cmax, __shfl_down_sync(0xffffffffu, cmax, o));
    nvac += __shfl_down_sync(0xffffffffu, nvac, o);
    nbad += __shfl_down_sync(0xffffffffu, nbad, o);
  }
  __shared__ double sh[NTHREADS / 32][8];
  __shared__ unsigned long long shc[NTHREADS / 32][2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    for (int f = 0; f < 6; f++) sh[w][f] = (double)hi[f] + (double)lo[f];
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
    for (int q = 0; q < NTHREADS / 32; q++) {
      for (int f = 0; f < 6; f++) p.s[f] += sh[q][f];
      p.vmax = fmax(p.vmax, sh[q][6]);
      p.cmax = fmax(p.cmax, sh[q][7]);
      p.nvac += shc[q][0];
      p.nbad += shc[q][1];
    }
    out[slot] = p;
  }
}

// Running per-thread sums of the six output fields: compensated float for the FP32
// path, plain double for the FP64 path.
template <typename T>
struct FieldSums;
template <>
struct FieldSums<float> {
  CompSum s[6];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int f = 0; f < 6; f++) s[f].init();
  }
  __device__ __forceinline__ void add(const float u[6]) {
#pragma unroll
    for (int f = 0; f < 6; f++) s[f].add(u[f]);
  }
  // low parts of a double-float state's fields 0..4 (below the sums' rounding: plain adds)
  __device__ __forceinline__ void add_lo(const float lo[5]) {
#pragma unroll
    for (int f = 0; f < 5; f++) s[f].lo += lo[f];
  }
  __device__ __forceinline__ void get(double out[6]) const {
#pragma unroll
    for (int f = 0; f < 6; f++) out[f] = s[f].value();
  }
};
template <>
struct FieldSums<double> {
  double s[6];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int f = 0; f < 6; f++) s[f] = 0.0;
  }
  __device__ __forceinline__ void add(const double u[6]) {
#pragma unroll
    for (int f = 0; f < 6; f++) s[f] += u[f];
  }
  __device__ __forceinline__ void get(double out[6]) const {
#pragma unroll
    for (int f = 0; f < 6; f++) out[f] = s[f];
  }
};

// Per-cell part of the CFL step (Sec. 1.1) and of the non-physical check, in T.
template <typename T>
__device__ __forceinline__ void cell_speeds(const T u[6], T gamma, T gm1, T& vmax, T& cmax,
                                            unsigned long long& nbad) {
  const T rho = u[0];
  const T vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
  const T v = sqrt(vx * vx + vy * vy + vz * vz);
  const T p = gm1 * u[5];
  const T c = sqrt(gamma * p / rho);
  bool ok = rho > T(0) && u[5] > T(0);
#pragma unroll
  for (int f = 0; f < 6; f++) ok = ok && isfinite(u[f]);
  if (ok) {
    vmax = fmax(vmax, v);
    cmax = fmax(cmax, c);
  } else {
    nbad++;
  }
}

// FP32 form for the stage kernels: one approximate reciprocal of rho, |v| = |m| / rho.
__device__ __forceinline__ void cell_speeds_f32(const float u[6], float gamma, float gm1,
                                                float& vmax, float& cmax,
                                                unsigned long long& nbad) {
  const float rho = u[0];
  const float ir = rcp_approx(rho);
  const float v = sqrt_approx(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * ir;
  const float c = sqrt_approx(gamma * gm1 * u[5] * ir);
  bool ok = rho > 0.f && u[5] > 0.f;
#pragma unroll
  for (int f = 0; f < 6; f++) ok = ok && isfinite(u[f]);
  if (ok) {
    vmax = fmaxf(vmax, v);
    cmax = fmaxf(cmax, c);
  } else {
    nbad++;
  }
}

// ------------------------------------------------------------------ standalone diagnostics

template <typename T>
__global__ void __launch_bounds__(NT) diag_kernel(MarchArgs<T> A) {
  const long long n = A.g.ncell;
  FieldSums<T> sums;
  sums.init();
  T vmax = T(0), cmax = T(0);
  unsigned long long nbad = 0;
  const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);
  for (long long idx = (long long)blockIdx.x * NT + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * NT) {
    T u[6];
#pragma unroll
    for (int f = 0; f < 6; f++) u[f] = A.u[f][idx];
    sums.add(u);
    if constexpr (sizeof(T) == 4) {
      if (A.ulo[0]) {  // double-float state: the sums take the low parts too
        float lo[5];
#pragma unroll
        for (int f = 0; f < 5; f++) lo[f] = A.ulo[f][idx];
        sums.add_lo(lo);
      }
    }
    cell_speeds<T>(u, gamma, gm1, vmax, cmax, nbad);
  }
  double sd[6];
  sums.get(sd);
  block_reduce_store<NT>(sd, (double)vmax, (double)cmax, 0ull, nbad, A.partials, blockIdx.x);
}

}  // namespace ppml
