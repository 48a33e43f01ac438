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
// Face arrays of nmax + 1 values behind the four fields in shared memory.  FP32 holds the
// four Lagrangian fluxes of a step at once (one flux pass and one update pass per step);
// FP64 takes the fields in turn through two, so that 4096-cell instances fit in 227 KB.
template <typename T>
constexpr int kBatchFaceArrays = sizeof(T) == 4 ? 4 : 2;

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

// NQ quantities along a run of faces, as stream_faces2: on_face(f, l, r, PL, PR), where
// l[j], r[j] are quantity j in cells f-1 and f and PL[j], PR[j] its parabolas there;
// q(j, k) gives quantity j in cell k for k = f0-3 .. f1+2, each read one face ahead of its
// use (so that the read overlaps the previous face's stores).
template <typename T, int NQ, typename QN, typename OF>
__device__ __forceinline__ void stream_faces_n(QN q, int f0, int f1, OF on_face) {
  T a2[NQ], a3[NQ], a4[NQ], d3[NQ], fv[NQ];
  Parab<T> P[NQ];
#pragma unroll
  for (int j = 0; j < NQ; j++) {
    const T a0 = q(j, f0 - 3), a1 = q(j, f0 - 2);
    a2[j] = q(j, f0 - 1);
    a3[j] = q(j, f0);
    a4[j] = q(j, f0 + 1);
    const T d1 = limited_slope(a0, a1, a2[j]);      // cell f0-2
    const T d2 = limited_slope(a1, a2[j], a3[j]);   // cell f0-1
    d3[j] = limited_slope(a2[j], a3[j], a4[j]);     // cell f0
    const T fl = face_value(a1, a2[j], d1, d2);     // face f0-1
    fv[j] = face_value(a2[j], a3[j], d2, d3[j]);    // face f0
    P[j] = parabola(a2[j], fl, fv[j]);              // cell f0-1
  }
  T pa[NQ];  // cell f+2, read one face ahead
#pragma unroll
  for (int j = 0; j < NQ; j++) pa[j] = q(j, f0 + 2);
#pragma unroll 4
  for (int f = f0; f <= f1; f++) {
    T an[NQ], dn[NQ], fn[NQ];
    Parab<T> Q[NQ];
#pragma unroll
    for (int j = 0; j < NQ; j++) {
      an[j] = pa[j];
      if (f < f1) pa[j] = q(j, f + 3);
      dn[j] = limited_slope(a3[j], a4[j], an[j]);     // cell f+1
      fn[j] = face_value(a3[j], a4[j], d3[j], dn[j]);  // face f+1
      Q[j] = parabola(a3[j], fv[j], fn[j]);           // cell f
    }
    on_face(f, a2, a3, P, Q);
#pragma unroll
    for (int j = 0; j < NQ; j++) {
      a2[j] = a3[j];
      a3[j] = a4[j];
      a4[j] = an[j];
      d3[j] = dn[j];
      fv[j] = fn[j];
      P[j] = Q[j];
    }
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

// CFL step of the CTA's instance (Sec. 1.1) from the per-thread maxima a = max|v|,
// b = max c: warp maxima, then warp 0 folds the warps' (maxima in the state's precision;
// a maximum is exact in any).  Thread 0 alone keeps the instance's time (t, steps, done):
// it stops the CTA once t has reached t_end, else forms tau clipped to the remaining time
// and advances t.  FP64 forms tau = cfl h / (a + b) and tau / h as the checker does; FP32
// forms tau / h = cfl / (a + b) in FP32 and tau = (tau / h) h in FP64 (both divisions of
// the FP64 form, at the FP64 pipe's latency, would lie on every step's critical path).
// Returns whether the CTA takes the step (the same in every thread), with th = tau / h
// and, in FP64, dt = tau.  Two barriers; the caller puts at least one more between two
// calls, so the next call's writes to sh cannot overtake this call's reads.
template <typename T>
__device__ __forceinline__ bool block_cfl_step(T a, T b, double cfl, InstDev& I, double* sh,
                                               double& dt, T& th) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  T* shT = reinterpret_cast<T*>(sh);  // 32 + 32 warp maxima
  int* go_sh = reinterpret_cast<int*>(sh + 68);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    shT[w] = a;
    shT[32 + w] = b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x >> 5);
    T A = lane < nw ? shT[lane] : T(0), B = lane < nw ? shT[32 + lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      A = fmax(A, __shfl_down_sync(0xffffffffu, A, o));
      B = fmax(B, __shfl_down_sync(0xffffffffu, B, o));
    }
    if (lane == 0) {
      int go = 0;
      double d = 0.0;
      T q = T(0);
      if (!(I.t >= I.t_end)) {
        const double rem = I.t_end - I.t;
        if constexpr (sizeof(T) == 4) {
          q = (float)cfl / (A + B);
          d = (double)q * I.h;
          if (d > rem) {
            d = rem;
            q = (float)(rem / I.h);
          }
        } else {
          const double den = A + B;
          d = cfl * I.h / den;
          if (d > rem) d = rem;
          q = d / I.h;
        }
        go = d > 0.0;
      }
      if (go) {
        I.t = (I.t + d > I.t_end) ? I.t_end : I.t + d;
        I.steps += 1;
      } else {
        I.done = 1;
      }
      sh[64] = d;
      *reinterpret_cast<T*>(sh + 66) = q;
      *go_sh = go;
    }
  }
  __syncthreads();
  dt = sh[64];
  th = *reinterpret_cast<const T*>(sh + 66);
  return *go_sh != 0;
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
  T* FA = Ei + stride;      // face array A (V, then v hat or the rho flux)
  T* FB = FA + (nmax + 1);  // face array B (P, then fluxes)
  T* FC = FB + (nmax + 1);  // FP32 only: the rho E and rho eps fluxes
  T* FD = FC + (nmax + 1);
  const int tid = threadIdx.x;
  const T gamma = T(gamma_d), gm1 = T(gamma_d - 1.0);
  // faces per streamed run: one run per thread covers all n + 1 faces; at least 9 (the
  // stream reads 3 extra cells on each side of its run) and odd, so that the runs of the
  // 32 lanes of a warp start on 32 different banks
  const int run = max(8, (n + 1 + NTHREADS - 1) / NTHREADS) | 1;
  constexpr int kU = sizeof(T) == 4 ? 4 : 2;  // cells per thread per update pass
  const float rho_vac_up = __double2float_ru(I.rho_vac);  // set by batch_vacuum_kernel
  // Outflow ghosts of field q from its edge cells, written after a cell pass by the
  // threads that own those cells (cell c belongs to thread c mod NTHREADS in every cell
  // pass): they read back their own stores, so no barrier (and no pass) of its own.
  const int owner_last = (n - 1) % NTHREADS;
  auto edge_ghosts = [&](T* q) {
    if (tid == 0) {
      const T v = q[kBatchGhost];
#pragma unroll
      for (int k = 0; k < kBatchGhost; k++) q[k] = v;
    }
    if (tid == owner_last) {
      const T v = q[n + kBatchGhost - 1];
#pragma unroll
      for (int k = 0; k < kBatchGhost; k++) q[n + kBatchGhost + k] = v;
    }
  };
  // CFL maxima (Sec. 1.1) over the cells a thread owns, taken as each cell's final value
  // of a step is written: max |v| and max c, in the checker's per-cell operations
  T vm = T(0), cm = T(0);
  auto cfl_cell = [&](T r, T m, T ei, bool valid) {
    const T p = gm1 * ei;
    T v, cs;
    if constexpr (sizeof(T) == 4) {
      const float ir = rcp_approx(r);
      v = fabsf(m * ir);
      cs = sqrt_approx(gamma * p * ir);
    } else {
      const T vx = m / r, vy = T(0) / r, vz = T(0) / r;
      v = sqrt(vx * vx + vy * vy + vz * vz);
      cs = sqrt(gamma * p / r);
    }
    vm = valid ? fmax(vm, v) : vm;
    cm = valid ? fmax(cm, cs) : cm;
  };
  for (int c = tid; c < n; c += blockDim.x) {
    const int g = c + kBatchGhost;
    const T r = g_rho[I.off + c], m = g_m[I.off + c], en = g_en[I.off + c], ei = g_ei[I.off + c];
    R[g] = r;
    M[g] = m;
    E[g] = en;
    Ei[g] = ei;
    cfl_cell(r, m, ei, true);
  }
  edge_ghosts(R);
  edge_ghosts(M);
  edge_ghosts(E);
  edge_ghosts(Ei);
  // Upwind Lagrangian fluxes of one field at the faces of every thread's run (Sec. 1.3)
  auto lagrangian_fluxes = [&](const T* q, double dt, T th) {
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
  };
  // Barriers per step: two in the CFL reduction (the first also orders every field and
  // ghost write of the previous step), Eulerian faces, Eulerian update, then in FP32 one
  // after the Lagrangian flux pass; in FP64 one after v hat and two per Lagrangian field
  // but the last.  The last update pass also applies the energy correction, writes the
  // ghosts and takes the next step's CFL maxima.
  for (int s = 0; s < max_steps; s++) {
    double dt;
    T th;
    if (!block_cfl_step<T>(vm, cm, cfl, I, red, dt, th)) break;
    // Eulerian stage: faces f = 0..n (between cells f-1 and f, padded cells f+2 and f+3);
    // each thread streams one run of `run` consecutive faces
    {
      auto vq = [&](int k) { return vel_of(M[k + kBatchGhost], R[k + kBatchGhost]); };
      auto pq = [&](int k) { return gm1 * Ei[k + kBatchGhost]; };
      for (int f0 = tid * run; f0 <= n; f0 += NTHREADS * run) {
        const int f1 = min(f0 + run - 1, n);
        // rho and sqrt(rho) of the face's left cell, carried from the previous face
        T r_l = R[f0 + 2], s_l = T(0);
        if constexpr (sizeof(T) == 4) s_l = sqrt_approx(r_l);
        stream_faces2<T>(vq, pq, f0, f1,
                         [&](int f, T, T, const Parab<T>& vL, const Parab<T>& vR, T pl, T pr,
                             const Parab<T>& pL, const Parab<T>& pR) {
          const T rl = r_l, rr = R[f + 3];
          r_l = rr;
          T V, P;
          if constexpr (sizeof(T) == 4) {
            float lam, Z, hrz;
            const float sl = s_l, sr = sqrt_approx(rr);
            s_l = sr;
            face_constants_f32(rl, rr, sl, sr, pl, pr, gamma, lam, Z, hrz);
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
    // cells c0 + u NTHREADS, u < kU, per pass: every load of the pass ahead of its stores
    // (the compiler cannot move a load past a store into the same shared array)
    for (int c0 = tid; c0 < n; c0 += kU * NTHREADS) {
      T Vm[kU], Vp[kU], Pm[kU], Pp[kU], m0[kU], e0[kU], ei0[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int c = min(c0 + u * NTHREADS, n - 1), g = c + kBatchGhost;
        Vm[u] = FA[c];
        Vp[u] = FA[c + 1];
        Pm[u] = FB[c];
        Pp[u] = FB[c + 1];
        m0[u] = M[g];
        e0[u] = E[g];
        ei0[u] = Ei[g];
      }
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int c = c0 + u * NTHREADS, g = c + kBatchGhost;
        if (c < n) {
          const T m1 = m0[u] - th * (Pp[u] - Pm[u]);
          const T e1 = e0[u] - th * (Pp[u] * Vp[u] - Pm[u] * Vm[u]);
          const T ei1 = ei0[u] - gm1 * ei0[u] * (th * (Vp[u] - Vm[u]));
          M[g] = m1;
          E[g] = e1;
          Ei[g] = ei1;
        }
      }
    }
    edge_ghosts(M);
    edge_ghosts(E);
    edge_ghosts(Ei);
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // Lagrangian stage in one pass over each run of faces: v hat (eq. veltemplate with
      // the Roe weights, Sec. 1.3) from the streamed rho and m, each cell's template and
      // sqrt(rho) formed once and carried to the next face, then the upwind fluxes of all
      // four fields
      auto q4 = [&](int j, int k) {
        return (j == 0 ? R : j == 1 ? M : j == 2 ? E : Ei)[k + kBatchGhost];
      };
      for (int f0 = tid * run; f0 <= n; f0 += NTHREADS * run) {
        const int f1 = min(f0 + run - 1, n);
        const float r0 = R[f0 + 2];  // cell f0-1
        float vt_l = template_1d(vel_of(M[f0 + 2], r0)), s_l = sqrt_approx(r0);
        stream_faces_n<float, 4>(q4, f0, f1,
                                 [&](int f, const float*, const float* c, const Parab<float>* PL,
                                     const Parab<float>* PR) {
          const float vt_r = template_1d(vel_of(c[1], c[0])), s_r = sqrt_approx(c[0]);
          const float vh = (vt_r * s_r + vt_l * s_l) * rcp_approx(s_r + s_l);
          vt_l = vt_r;
          s_l = s_r;
          const float y = Prec<float>::courant(tabs(vh), dt, I.h, th);
          float F[4];
#pragma unroll
          for (int j = 0; j < 4; j++)
            F[j] = vh >= 0.0f ? vh * avg_right(PL[j].R, PL[j].D, PL[j].S, y)
                              : vh * avg_left(PR[j].L, PR[j].D, PR[j].S, y);
          FA[f] = F[0];
          FB[f] = F[1];
          FC[f] = F[2];
          FD[f] = F[3];
        });
      }
      __syncthreads();
      // every field's update, the Sec. 1.4 energy consistency, the ghosts and the next
      // step's CFL maxima, cell by cell
      vm = T(0);
      cm = T(0);
      for (int c0 = tid; c0 < n; c0 += kU * NTHREADS) {
        float q[kU][4];
#pragma unroll
        for (int u = 0; u < kU; u++) {
          const int c = min(c0 + u * NTHREADS, n - 1), g = c + kBatchGhost;
          q[u][0] = R[g] - th * (FA[c + 1] - FA[c]);
          q[u][1] = M[g] - th * (FB[c + 1] - FB[c]);
          q[u][2] = E[g] - th * (FC[c + 1] - FC[c]);
          q[u][3] = Ei[g] - th * (FD[c + 1] - FD[c]);
        }
        // Sec. 1.4: the dense branch for all kU cells without control flow (so that
        // their chains interleave), then the rare vacuum cells
        float w[kU][6];
        bool vac[kU], any_vac = false;
#pragma unroll
        for (int u = 0; u < kU; u++) {
          w[u][0] = q[u][0];
          w[u][1] = q[u][1];
          w[u][2] = 0.0f;
          w[u][3] = 0.0f;
          w[u][4] = q[u][2];
          w[u][5] = q[u][3];
          vac[u] = vacuum_cell_f32(w[u], rho_vac_up);
          any_vac |= vac[u];
          q[u][3] = dense_eps_f32(w[u]);
        }
        if (any_vac) {
#pragma unroll
          for (int u = 0; u < kU; u++)
            if (vac[u]) {
              vacuum_correct_f32(w[u], I.rho_vac);
              q[u][1] = w[u][1];
              q[u][3] = w[u][5];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
          const int c = c0 + u * NTHREADS, g = c + kBatchGhost;
          if (c < n) {
            R[g] = q[u][0];
            M[g] = q[u][1];
            E[g] = q[u][2];
            Ei[g] = q[u][3];
          }
        }
        // next step's CFL maxima over the valid cells (a clamped duplicate may have read
        // a cell its owner has already updated)
#pragma unroll
        for (int u = 0; u < kU; u++) cfl_cell(q[u][0], q[u][1], q[u][3], c0 + u * NTHREADS < n);
      }
      edge_ghosts(R);
      edge_ghosts(M);
      edge_ghosts(E);
      edge_ghosts(Ei);
    } else {
      // FP64 Lagrangian stage: v hat at faces, then each field's flux and update in turn
      for (int f = tid; f <= n; f += blockDim.x) {
        const T rl = R[f + 2], rr = R[f + 3];
        const T vtl = template_1d(vel_of(M[f + 2], rl)), vtr = template_1d(vel_of(M[f + 3], rr));
        const T sl = sqrt(rl), sr = sqrt(rr);
        FA[f] = (vtr * sr + vtl * sl) / (sr + sl);
      }
      __syncthreads();
      T* fields[3] = {R, M, E};
#pragma unroll 1
      for (int k = 0; k < 3; k++) {
        T* q = fields[k];
        lagrangian_fluxes(q, dt, th);
        __syncthreads();
        for (int c = tid; c < n; c += blockDim.x)
          q[c + kBatchGhost] = q[c + kBatchGhost] - th * (FB[c + 1] - FB[c]);
        __syncthreads();
      }
      lagrangian_fluxes(Ei, dt, th);
      __syncthreads();
      // rho eps update, then the Sec. 1.4 energy consistency, on the same cells
      vm = T(0);
      cm = T(0);
      for (int c = tid; c < n; c += blockDim.x) {
        const int g = c + kBatchGhost;
        const T r = R[g], en = E[g];
        T u[6] = {r, M[g], T(0), T(0), en, Ei[g] - th * (FB[c + 1] - FB[c])};
        correct_energy<T>(u, I.rho_vac);
        M[g] = u[1];
        Ei[g] = u[5];
        cfl_cell(r, u[1], u[5], true);
      }
      edge_ghosts(R);
      edge_ghosts(M);
      edge_ghosts(E);
      edge_ghosts(Ei);
    }
  }
  for (int c = tid; c < n; c += blockDim.x) {
    g_rho[I.off + c] = R[c + kBatchGhost];
    g_m[I.off + c] = M[c + kBatchGhost];
    g_en[I.off + c] = E[c + kBatchGhost];
    g_ei[I.off + c] = Ei[c + kBatchGhost];
  }
  if (tid == 0) {  // thread 0's copy holds the instance's time
    if (I.t >= I.t_end) I.done = 1;
    inst[id] = I;
  }
}

}  // namespace ppml
