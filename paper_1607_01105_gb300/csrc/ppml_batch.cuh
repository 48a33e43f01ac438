// Batched independent 1D problems (many shock tubes of uneven lengths) advanced by one
// persistent launch: each CTA owns one instance, keeps its four fields (rho, m, rho E,
// rho eps) resident in shared memory for all of its steps, takes its own CFL step from a
// CTA-local reduction (Sec. 1.1) and stops at its own end time.  The scheme per step is
// the 1D case of Sec. 1: Eulerian face solve, upwind Lagrangian fluxes, energy
// correction of Sec. 1.4.  In 1D the 9-point template (eq. veltemplate) runs on the cell
// itself (its transverse neighbours are the cell), evaluated term by term.  Outflow
// boundaries on both ends.  CTAs never wait on one another.  The CTA size (threads per
// instance) is a template parameter; the host picks it by timing the candidates on the
// actual batch (ppml_batch_tune).
#pragma once
#include "ppml_device.cuh"

namespace ppml {

constexpr int kBatchGhost = 3;

struct InstDev {
  long long off;  // first cell in the packed arrays
  int n;          // cells
  int steps;      // steps taken so far
  double h, t_end, t, rho_vac;
  int done, pad;
};

template <typename T>
__device__ __forceinline__ void fill_ghosts_1d(T* q, int n) {
  const int t = threadIdx.x;
  if (t < kBatchGhost)
    q[t] = q[kBatchGhost];
  else if (t < 2 * kBatchGhost)
    q[n + kBatchGhost + (t - kBatchGhost)] = q[n + kBatchGhost - 1];
}

// eq. veltemplate on a cell whose transverse neighbours are itself
template <typename T>
__device__ __forceinline__ T template_1d(T v) {
  const T four = v + v + v + v;
  return four / T(16) + four / T(8) + v / T(4);
}

// Parabolas of two quantities along a contiguous run of faces, streamed (Appendix Steps 1-3):
// for faces f = f0 .. f1 (face f between cells f-1 and f) calls
// on_face(f, a[f-1], a[f], Pa[f-1], Pa[f], b[f-1], b[f], Pb[f-1], Pb[f]).  qa(k), qb(k) give
// cell k's values for k = f0-3 .. f1+2.  Each slope, face value and parabola is formed once,
// with the same operations as per face.
template <typename T, typename QA, typename QB, typename OF>
__device__ __forceinline__ void stream_faces2(QA qa, QB qb, int f0, int f1, OF on_face) {
  T a0 = qa(f0 - 3), a1 = qa(f0 - 2), a2 = qa(f0 - 1), a3 = qa(f0), a4 = qa(f0 + 1);
  T b0 = qb(f0 - 3), b1 = qb(f0 - 2), b2 = qb(f0 - 1), b3 = qb(f0), b4 = qb(f0 + 1);
  const T da1 = limited_slope(a0, a1, a2), db1 = limited_slope(b0, b1, b2);  // cell f0-2
  T da2 = limited_slope(a1, a2, a3), db2 = limited_slope(b1, b2, b3);        // cell f0-1
  T da3 = limited_slope(a2, a3, a4), db3 = limited_slope(b2, b3, b4);        // cell f0
  const T fa1 = face_value(a1, a2, da1, da2), fb1 = face_value(b1, b2, db1, db2);  // face f0-1
  T fa2 = face_value(a2, a3, da2, da3), fb2 = face_value(b2, b3, db2, db3);        // face f0
  Parab<T> Pa = parabola(a2, fa1, fa2), Pb = parabola(b2, fb1, fb2);             // cell f0-1
  (void)da2;
  (void)db2;
#pragma unroll 2
  for (int f = f0; f <= f1; f++) {
    // window: a2 = cell f-1, a3 = cell f, a4 = cell f+1; da3 slope of f; fa2 face f
    const T an = qa(f + 2), bn = qb(f + 2);
    const T dan = limited_slope(a3, a4, an), dbn = limited_slope(b3, b4, bn);  // cell f+1
    const T fan = face_value(a3, a4, da3, dan), fbn = face_value(b3, b4, db3, dbn);  // face f+1
    const Parab<T> Qa = parabola(a3, fa2, fan), Qb = parabola(b3, fb2, fbn);       // cell f
    on_face(f, a2, a3, Pa, Qa, b2, b3, Pb, Qb);
    a2 = a3;
    a3 = a4;
    a4 = an;
    b2 = b3;
    b3 = b4;
    b4 = bn;
    da3 = dan;
    db3 = dbn;
    fa2 = fan;
    fb2 = fbn;
    Pa = Qa;
    Pb = Qb;
  }
}

// One quantity, as stream_faces2: on_face(f, Pq[f-1], Pq[f]).
template <typename T, typename QF, typename OF>
__device__ __forceinline__ void stream_faces(QF q, int f0, int f1, OF on_face) {
  T a0 = q(f0 - 3), a1 = q(f0 - 2), a2 = q(f0 - 1), a3 = q(f0), a4 = q(f0 + 1);
  const T d1 = limited_slope(a0, a1, a2);  // cell f0-2
  const T d2 = limited_slope(a1, a2, a3);  // cell f0-1
  T d3 = limited_slope(a2, a3, a4);        // cell f0
  const T f1v = face_value(a1, a2, d1, d2);  // face f0-1
  T f2v = face_value(a2, a3, d2, d3);        // face f0
  Parab<T> P = parabola(a2, f1v, f2v);       // cell f0-1
#pragma unroll 2
  for (int f = f0; f <= f1; f++) {
    const T an = q(f + 2);
    const T dn = limited_slope(a3, a4, an);
    const T fn = face_value(a3, a4, d3, dn);
    const Parab<T> Q = parabola(a3, f2v, fn);
    on_face(f, P, Q);
    a3 = a4;
    a4 = an;
    d3 = dn;
    f2v = fn;
    P = Q;
  }
}

// v = m / rho: approximate reciprocal in FP32 (as in the stage kernels), IEEE in FP64.
template <typename T>
__device__ __forceinline__ T vel_of(T m, T r) {
  if constexpr (sizeof(T) == 4)
    return m * rcp_approx(r);
  else
    return m / r;
}

// CFL step of the CTA's instance (Sec. 1.1): the CTA maxima a = max|v|, b = max c, then
// thread 0 forms dt = cfl h / (a + b), clipped to rem, and dt / h (the only FP64 divisions
// of the step) and shares them.
__device__ __forceinline__ void block_cfl_step(double a, double b, double cfl, double h,
                                               double rem, double* sh, double& dt, double& th) {
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
    const double den = A + B;
    double d = cfl * h / den;
    if (d > rem) d = rem;
    sh[64] = d;
    sh[65] = d / h;
  }
  __syncthreads();
  dt = sh[64];
  th = sh[65];
  __syncthreads();
}


// Vacuum threshold of every instance (Sec. 1.4: a fraction of the mean density; the
// fraction is stored negated until this kernel has run): the instance's mean initial
// density from a fixed 256-thread reduction, so the threshold does not depend on the CTA
// size of the stepping kernel.
template <typename T>
__global__ void __launch_bounds__(256) batch_vacuum_kernel(const T* __restrict__ g_rho,
                                                          InstDev* __restrict__ inst) {
  __shared__ double red[8];
  InstDev& I = inst[blockIdx.x];
  if (I.rho_vac >= 0.0) return;
  double s = 0.0;
  for (int c = threadIdx.x; c < I.n; c += 256) s += (double)g_rho[I.off + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    for (int q = 0; q < 8; q++) S += red[q];
    I.rho_vac = -I.rho_vac * (S / I.n);
  }
}

template <typename T, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS, 1) batch_kernel(T* __restrict__ g_rho,
                                                              T* __restrict__ g_m,
                                                              T* __restrict__ g_en,
                                                              T* __restrict__ g_ei,
                                                              InstDev* __restrict__ inst,
                                                              const int* __restrict__ order,
                                                              double gamma_d, double cfl,
                                                              int max_steps, int nmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[80];
  const int id = order[blockIdx.x];
  InstDev I = inst[id];
  if (I.done) return;
  const int n = I.n;
  const int stride = nmax + 2 * kBatchGhost;
  T* R = (T*)smem_raw;
  T* M = R + stride;
  T* E = M + stride;
  T* Ei = E + stride;
  T* FA = Ei + stride;      // face array A (V, then v hat)
  T* FB = FA + (nmax + 1);  // face array B (P, then fluxes)
  const int tid = threadIdx.x;
  for (int c = tid; c < n; c += blockDim.x) {
    R[c + kBatchGhost] = g_rho[I.off + c];
    M[c + kBatchGhost] = g_m[I.off + c];
    E[c + kBatchGhost] = g_en[I.off + c];
    Ei[c + kBatchGhost] = g_ei[I.off + c];
  }
  __syncthreads();
  const T gamma = T(gamma_d), gm1 = T(gamma_d - 1.0);
  // faces per streamed run: one run per thread covers all n + 1 faces; at least 9 (the
  // stream reads 3 extra cells on each side of its run) and odd, so that the runs of the
  // 32 lanes of a warp start on 32 different banks
  const int run = max(8, (n + 1 + NTHREADS - 1) / NTHREADS) | 1;
  const float rho_vac_up = __double2float_ru(I.rho_vac);  // set by batch_vacuum_kernel
  for (int s = 0; s < max_steps; s++) {
    // CFL step of the current state (Sec. 1.1), per cell in the checker's order
    T vm = T(0), cm = T(0);
    for (int c = tid; c < n; c += blockDim.x) {
      const T r = R[c + kBatchGhost];
      const T p = gm1 * Ei[c + kBatchGhost];
      T v, cs;
      if constexpr (sizeof(T) == 4) {
        const float ir = rcp_approx(r);
        v = fabsf(M[c + kBatchGhost] * ir);
        cs = sqrt_approx(gamma * p * ir);
      } else {
        const T vx = M[c + kBatchGhost] / r, vy = T(0) / r, vz = T(0) / r;
        v = sqrt(vx * vx + vy * vy + vz * vz);
        cs = sqrt(gamma * p / r);
      }
      vm = fmax(vm, v);
      cm = fmax(cm, cs);
    }
    double dt, thd;  // the maxima convert to double exactly
    block_cfl_step((double)vm, (double)cm, cfl, I.h, I.t_end - I.t, red, dt, thd);
    if (!(dt > 0.0)) {
      I.done = 1;
      break;
    }
    const T th = T(thd);
    fill_ghosts_1d(R, n);
    fill_ghosts_1d(M, n);
    fill_ghosts_1d(E, n);
    fill_ghosts_1d(Ei, n);
    __syncthreads();
    // Eulerian stage: faces f = 0..n (between cells f-1 and f, padded cells f+2 and f+3);
    // each thread streams one run of `run` consecutive faces
    {
      auto vq = [&](int k) { return vel_of(M[k + kBatchGhost], R[k + kBatchGhost]); };
      auto pq = [&](int k) { return gm1 * Ei[k + kBatchGhost]; };
      for (int f0 = tid * run; f0 <= n; f0 += NTHREADS * run) {
        const int f1 = min(f0 + run - 1, n);
        stream_faces2<T>(vq, pq, f0, f1,
                         [&](int f, T, T, const Parab<T>& vL, const Parab<T>& vR, T pl, T pr,
                             const Parab<T>& pL, const Parab<T>& pR) {
          const T rl = R[f + 2], rr = R[f + 3];
          T V, P;
          if constexpr (sizeof(T) == 4) {
            float lam, Z, hrz;
            face_constants_f32(rl, rr, sqrt_approx(rl), sqrt_approx(rr), pl, pr, gamma, lam, Z,
                               hrz);
            const float y = lam * th;
            const float vls = avg_right(vL.R, vL.D, vL.S, y), vrs = avg_left(vR.L, vR.D, vR.S, y);
            const float pls = avg_right(pL.R, pL.D, pL.S, y), prs = avg_left(pR.L, pR.D, pR.S, y);
            V = 0.5f * (vls + vrs) + (pls - prs) * hrz;
            P = 0.5f * (pls + prs) + 0.5f * Z * (vls - vrs);
          } else {
            T lam, Z;
            face_constants(rl, rr, pl, pr, gamma, lam, Z);
            const T y = Prec<T>::courant(lam, dt, I.h, th);
            riemann_vp(avg_right(vL.R, vL.D, vL.S, y), avg_left(vR.L, vR.D, vR.S, y),
                       avg_right(pL.R, pL.D, pL.S, y), avg_left(pR.L, pR.D, pR.S, y), Z, V, P);
          }
          FA[f] = V;
          FB[f] = P;
        });
      }
    }
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) {
      const int g = c + kBatchGhost;
      const T Vm = FA[c], Vp = FA[c + 1], Pm = FB[c], Pp = FB[c + 1];
      const T ei0 = Ei[g];
      M[g] = M[g] - th * (Pp - Pm);
      E[g] = E[g] - th * (Pp * Vp - Pm * Vm);
      Ei[g] = ei0 - gm1 * ei0 * (th * (Vp - Vm));
    }
    __syncthreads();
    fill_ghosts_1d(M, n);
    fill_ghosts_1d(E, n);
    fill_ghosts_1d(Ei, n);
    __syncthreads();
    // Lagrangian stage: v hat at faces, then each field's flux and update
    for (int f = tid; f <= n; f += blockDim.x) {
      const T rl = R[f + 2], rr = R[f + 3];
      const T vtl = template_1d(vel_of(M[f + 2], rl)), vtr = template_1d(vel_of(M[f + 3], rr));
      if constexpr (sizeof(T) == 4) {
        const float sl = sqrt_approx(rl), sr = sqrt_approx(rr);
        FA[f] = (vtr * sr + vtl * sl) * rcp_approx(sr + sl);
      } else {
        const T sl = sqrt(rl), sr = sqrt(rr);
        FA[f] = (vtr * sr + vtl * sl) / (sr + sl);
      }
    }
    __syncthreads();
    T* fields[4] = {R, M, E, Ei};
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
      T* q = fields[k];
      auto qq = [&](int c) { return q[c + kBatchGhost]; };
      for (int f0 = tid * run; f0 <= n; f0 += NTHREADS * run) {
        const int f1 = min(f0 + run - 1, n);
        stream_faces<T>(qq, f0, f1, [&](int f, const Parab<T>& PL, const Parab<T>& PR) {
          const T vh = FA[f];
          const T y = Prec<T>::courant(tabs(vh), dt, I.h, th);
          FB[f] = vh >= T(0) ? vh * avg_right(PL.R, PL.D, PL.S, y)
                             : vh * avg_left(PR.L, PR.D, PR.S, y);
        });
      }
      __syncthreads();
      for (int c = tid; c < n; c += blockDim.x)
        q[c + kBatchGhost] = q[c + kBatchGhost] - th * (FB[c + 1] - FB[c]);
      __syncthreads();
    }
    // Sec. 1.4 energy consistency
    for (int c = tid; c < n; c += blockDim.x) {
      const int g = c + kBatchGhost;
      T u[6] = {R[g], M[g], T(0), T(0), E[g], Ei[g]};
      if constexpr (sizeof(T) == 4)
        correct_energy_f32(u, rho_vac_up, I.rho_vac);
      else
        correct_energy<T>(u, I.rho_vac);
      M[g] = u[1];
      Ei[g] = u[5];
    }
    __syncthreads();
    I.t = (I.t + dt > I.t_end) ? I.t_end : I.t + dt;
    I.steps += 1;
    if (I.t >= I.t_end) {
      I.done = 1;
      break;
    }
  }
  for (int c = tid; c < n; c += blockDim.x) {
    g_rho[I.off + c] = R[c + kBatchGhost];
    g_m[I.off + c] = M[c + kBatchGhost];
    g_en[I.off + c] = E[c + kBatchGhost];
    g_ei[I.off + c] = Ei[c + kBatchGhost];
  }
  if (tid == 0) inst[id] = I;
}

}  // namespace ppml
