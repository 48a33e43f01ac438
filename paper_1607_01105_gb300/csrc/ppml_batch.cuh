// Batched independent 1D problems (many shock tubes of uneven lengths) advanced by one
// persistent launch: each instance keeps its four fields (rho, m, rho E, rho eps) resident
// in shared memory for all of its steps, takes its own CFL step (Sec. 1.1) and stops at its
// own end time, or at the first step whose state has a cell with rho <= 0, rho eps <= 0 or
// a non-finite value (the instance is then flagged non-physical).  An FP32 batch given
// low-part arrays keeps rho, m and rho E as double-float pairs (the high parts feed the
// stencils, every update is added to the pair, and the Sec. 1.4 difference
// rho E - m^2 / (2 rho) is formed from both parts): FP64-class storage of the totals.  An instance is owned by one CTA, or -- the longest ones -- split over the
// two CTAs of a cluster, which exchange a halo and their CFL maxima once per step; no
// other CTAs wait on one another.  The scheme per step is the 1D case of Sec. 1: Eulerian
// face solve, upwind Lagrangian fluxes, energy correction of Sec. 1.4.  In 1D the 9-point
// template (eq. veltemplate) runs on the cell itself (its transverse neighbours are the
// cell), evaluated term by term.  Outflow boundaries on both ends.  The CTA size is a
// template parameter; the host picks it by timing the candidates on the actual batch
// (ppml_batch_tune).
#pragma once
#include <cooperative_groups.h>

#include "ppml_device.cuh"

namespace ppml {

constexpr int kBatchGhost = 3;
// Face arrays of nmax + 1 values behind the four fields in shared memory.  FP32 holds the
// four Lagrangian fluxes of a step at once (one flux pass and one update pass per step);
// FP64 takes the fields in turn through two, so that 4096-cell instances fit in 227 KB.
template <typename T>
constexpr int kBatchFaceArrays = sizeof(T) == 4 ? 4 : 2;
// A double-float FP32 batch keeps three more arrays of the instance's cells: the low parts
// of rho, m, rho E.
constexpr int kBatchLoArrays = 3;
// An instance split over a CTA pair: halo cells facing the partner, and the exchange slot
// (the kPairHalo edge cells of the four fields and, double-float, of the low parts, then
// the two CFL maxima and the non-physical flag).
constexpr int kPairHalo = 6;
constexpr int kPairFieldsMax = 4 + kBatchLoArrays;
constexpr int kPairSlot = kPairFieldsMax * kPairHalo + 3;

__device__ __forceinline__ unsigned cluster_rank() {
  return cooperative_groups::this_cluster().block_rank();
}
// barrier of all threads of the cluster (release / acquire of the cluster's shared memory)
__device__ __forceinline__ void cluster_sync() { cooperative_groups::this_cluster().sync(); }

struct InstDev {
  long long off;  // first cell in the packed arrays
  int n;          // cells
  int steps;      // steps taken so far
  double h, t_end, t, rho_vac;
  int done;  // stopped: t_end reached, the step underflowed, or non-physical
  int bad;   // a state of the instance had rho <= 0, rho eps <= 0 or a non-finite value
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

// Thread 0's CFL decision from the instance's maxima A = max|v|, B = max c (Sec. 1.1).
// Thread 0 alone keeps the instance's time (t, steps, done): it stops once t has reached
// t_end or when the current state is non-physical (bad: flagged, no step taken), else forms
// tau clipped to the remaining time and advances t.  FP64 forms tau =
// cfl h / (A + B) and tau / h as the checker does; FP32 forms tau / h = cfl / (A + B) in
// FP32 and tau = (tau / h) h in FP64 (both divisions of the FP64 form, at the FP64 pipe's
// latency, would lie on every step's critical path).  Publishes tau (sh[64]), tau / h
// (sh + 66) and the go flag (sh + 68).
template <typename T>
__device__ __forceinline__ void cfl_decide(T A, T B, bool bad, double cfl, InstDev& I,
                                           double* sh) {
  int go = 0;
  double d = 0.0;
  T q = T(0);
  if (bad) I.bad = 1;
  if (!bad && !(I.t >= I.t_end)) {
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
  *reinterpret_cast<int*>(sh + 68) = go;
}

// Warp maxima of (a, b) into sh (as T: slots 0..31 and 32..63); valid after a barrier.
template <typename T>
__device__ __forceinline__ void warp_maxima(T a, T b, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  T* shT = reinterpret_cast<T*>(sh);
  if ((threadIdx.x & 31) == 0) {
    shT[threadIdx.x >> 5] = a;
    shT[32 + (threadIdx.x >> 5)] = b;
  }
}

// Warp 0 folds the warp maxima (all 32 lanes take part); lane 0 receives A and B.
template <typename T>
__device__ __forceinline__ void fold_maxima(const double* sh, T& A, T& B) {
  const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
  const T* shT = reinterpret_cast<const T*>(sh);
  A = lane < nw ? shT[lane] : T(0);
  B = lane < nw ? shT[32 + lane] : T(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    A = fmax(A, __shfl_down_sync(0xffffffffu, A, o));
    B = fmax(B, __shfl_down_sync(0xffffffffu, B, o));
  }
}

// CFL step of the CTA's instance (Sec. 1.1) from the per-thread maxima a = max|v|,
// b = max c and non-physical flags: warp maxima, then warp 0 folds the warps' (maxima in
// the state's precision; a maximum is exact in any), the flags are OR-ed by the barrier,
// and thread 0 decides (cfl_decide).  Returns whether the CTA takes the step (the same in
// every thread), with th = tau / h and dt = tau.  Two barriers; the caller puts at least
// one more between two calls, so the next call's writes to sh cannot overtake this
// call's reads.
template <typename T>
__device__ __forceinline__ bool block_cfl_step(T a, T b, bool bad, double cfl, InstDev& I,
                                               double* sh, double& dt, T& th) {
  warp_maxima<T>(a, b, sh);
  const bool any_bad = __syncthreads_or(bad) != 0;
  if (threadIdx.x < 32) {
    T A, B;
    fold_maxima<T>(sh, A, B);
    if (threadIdx.x == 0) cfl_decide<T>(A, B, any_bad, cfl, I, sh);
  }
  __syncthreads();
  dt = sh[64];
  th = *reinterpret_cast<const T*>(sh + 66);
  return *reinterpret_cast<const int*>(sh + 68) != 0;
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

// The cells one CTA advances: the whole instance, or one half of it when the instance is
// split over the two CTAs of a cluster.  Local cell c is instance cell lo + c.
struct Part {
  int nl;       // own cells 0 .. nl-1
  int lo;       // instance index of local cell 0
  int fa, fb;   // Eulerian faces fa .. fb (face f between local cells f-1 and f)
  int ca, cb;   // Eulerian updates of local cells ca .. cb-1
  bool gl, gr;  // outflow ghosts left of cell 0 / right of cell nl-1 (the instance's ends)
};

// CFL step of an instance split over a CTA pair (Sec. 1.1), with the halo exchange.  Each
// CTA reduces its maxima and non-physical flags and publishes them, with its kPairHalo
// edge cells next to the partner of the four fields and (FP32) of the three low parts, in
// slot `par` of its shared memory; after the cluster barrier it copies the partner's edge
// cells into its halo through distributed shared memory, and thread 0 decides from the
// larger of the two CTAs' maxima and either flag (cfl_decide).  Both thread 0s hold the
// same time and see the same maxima and flags, so both CTAs take the same decisions and
// meet the same barriers.  The slots alternate with the step's parity: a slot is
// rewritten two steps later, after the next cluster barrier, which the partner passes
// only after its reads of this one.  q[0..NF) are the padded arrays (R, M, E, Ei, then
// RL, ML, EL for a double-float batch), padded by kPairHalo.
template <typename T, int NF>
__device__ __forceinline__ bool pair_cfl_step(T a, T b, bool bad, double cfl, InstDev& I,
                                              double* sh, T* xslot, int par, const Part& P,
                                              T* const* q, double& dt, T& th) {
  constexpr int G = kPairHalo;
  constexpr int SL = kPairSlot;
  warp_maxima<T>(a, b, sh);
  const bool any_bad = __syncthreads_or(bad) != 0;  // orders the step's last stores too
  T* slot = xslot + par * SL;
  if (threadIdx.x < NF * kPairHalo) {  // rank 0 publishes cells nl-6 .. nl-1, rank 1 0 .. 5
    const int f = threadIdx.x / kPairHalo, k = threadIdx.x % kPairHalo;
    slot[threadIdx.x] = q[f][G + (P.gl ? P.nl - kPairHalo : 0) + k];
  }
  if (threadIdx.x < 32) {
    T A, B;
    fold_maxima<T>(sh, A, B);
    if (threadIdx.x == 0) {
      slot[NF * kPairHalo] = A;
      slot[NF * kPairHalo + 1] = B;
      slot[NF * kPairHalo + 2] = any_bad ? T(1) : T(0);
    }
  }
  cluster_sync();
  const T* rslot = cooperative_groups::this_cluster().map_shared_rank(slot, cluster_rank() ^ 1u);
  if (threadIdx.x < NF * kPairHalo) {  // rank 0's halo is cells nl .. nl+5, rank 1's -6 .. -1
    const int f = threadIdx.x / kPairHalo, k = threadIdx.x % kPairHalo;
    q[f][G + (P.gl ? P.nl : -kPairHalo) + k] = rslot[threadIdx.x];
  }
  if (threadIdx.x == 0)
    cfl_decide<T>(fmax(slot[NF * kPairHalo], rslot[NF * kPairHalo]),
                  fmax(slot[NF * kPairHalo + 1], rslot[NF * kPairHalo + 1]),
                  slot[NF * kPairHalo + 2] != T(0) || rslot[NF * kPairHalo + 2] != T(0), cfl, I,
                  sh);
  __syncthreads();
  dt = sh[64];
  th = *reinterpret_cast<const T*>(sh + 66);
  return *reinterpret_cast<const int*>(sh + 68) != 0;
}

// One CTA's part of an instance advanced for up to max_steps steps (Sec. 1 in 1D).  PAIR:
// the part is half of an instance and the partner CTA of the cluster holds the other half
// (halo exchange and common CFL step in pair_cfl_step); else the part is the instance.
// Local arrays: four fields with G cells of padding on each side (the halo facing the
// partner, outflow ghosts at the instance's ends), face arrays indexed f + FO, and (DF,
// FP32 only) the low parts of rho, m, rho E padded like the fields, read from g_lo at the
// start and written back at the end.
template <typename T, int NTHREADS, bool PAIR, bool DF>
__device__ __forceinline__ void advance_part(T* __restrict__ g_rho, T* __restrict__ g_m,
                                             T* __restrict__ g_en, T* __restrict__ g_ei,
                                             T* const* g_lo, InstDev& I, const Part P, T* smem,
                                             int stride, int nface, double gamma_d, double cfl,
                                             int max_steps, double* red, T* xslot) {
  constexpr int G = PAIR ? kPairHalo : kBatchGhost;
  constexpr int FO = PAIR ? 3 : 0;
  static_assert(!DF || sizeof(T) == 4, "double-float states are FP32 only");
  const int nl = P.nl;
  T* R = smem;
  T* M = R + stride;
  T* E = M + stride;
  T* Ei = E + stride;
  T* FA = Ei + stride;  // face array A (V, then v hat or the rho flux)
  T* FB = FA + nface;   // face array B (P, then fluxes)
  T* FC = FB + nface;   // FP32 only: the rho E and rho eps fluxes
  T* FD = FC + nface;
  T* RL = FA + kBatchFaceArrays<T> * nface;  // DF: low parts of rho, m, rho E
  T* ML = RL + stride;
  T* EL = ML + stride;
  T* const fields[7] = {R, M, E, Ei, RL, ML, EL};
  const int tid = threadIdx.x;
  const T gamma = T(gamma_d), gm1 = T(gamma_d - 1.0);
  // faces per streamed run: one run per thread covers the pass's faces; at least 9 (the
  // stream reads 3 extra cells on each side of its run) and odd, so that the runs of the
  // 32 lanes of a warp start on 32 different banks
  const int run_e = max(8, (P.fb - P.fa + 1 + NTHREADS - 1) / NTHREADS) | 1;
  const int run = max(8, (nl + 1 + NTHREADS - 1) / NTHREADS) | 1;
  constexpr int kU = sizeof(T) == 4 ? 4 : 2;  // cells per thread per update pass
  const float rho_vac_up = __double2float_ru(I.rho_vac);  // set by batch_vacuum_kernel
  // Outflow ghosts of field q from the edge cells of the instance, written after a cell
  // pass that starts at cell `base` by the threads that own those cells in it (cell c
  // belongs to thread (c - base) mod NTHREADS): they read back their own stores, so no
  // barrier (and no pass) of its own.
  auto outer_ghosts = [&](T* q, int base) {
    if (P.gl && tid == (0 - base) % NTHREADS) {
      const T v = q[G];
#pragma unroll
      for (int k = 1; k <= kBatchGhost; k++) q[G - k] = v;
    }
    if (P.gr && tid == (nl - 1 - base) % NTHREADS) {
      const T v = q[G + nl - 1];
#pragma unroll
      for (int k = 0; k < kBatchGhost; k++) q[G + nl + k] = v;
    }
  };
  // CFL maxima (Sec. 1.1) over the cells a thread owns, taken as each cell's final value
  // of a step is written: max |v| and max c, in the checker's per-cell operations; and
  // whether one of them is non-physical (rho <= 0, rho eps <= 0 or a non-finite field)
  T vm = T(0), cm = T(0);
  bool bad = false;
  auto cfl_cell = [&](T r, T m, T en, T ei, bool valid) {
    const bool ok = r > T(0) && ei > T(0) && isfinite(r) && isfinite(m) && isfinite(en) &&
                    isfinite(ei);
    bad = bad || (valid && !ok);
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
  const long long off = I.off + P.lo;
  for (int c = tid; c < nl; c += NTHREADS) {
    const int g = c + G;
    const T r = g_rho[off + c], m = g_m[off + c], en = g_en[off + c], ei = g_ei[off + c];
    R[g] = r;
    M[g] = m;
    E[g] = en;
    Ei[g] = ei;
    if constexpr (DF) {
      RL[g] = g_lo[0][off + c];
      ML[g] = g_lo[1][off + c];
      EL[g] = g_lo[2][off + c];
    }
    cfl_cell(r, m, en, ei, true);
  }
  outer_ghosts(R, 0);
  outer_ghosts(M, 0);
  outer_ghosts(E, 0);
  outer_ghosts(Ei, 0);
  if constexpr (PAIR) {  // the initial halo: the partner's first cells, from the state
    const int h0 = P.gl ? nl : -kPairHalo;  // local index of the halo's first cell
    if (tid < kPairHalo) {
      const long long gi = off + h0 + tid;
      R[G + h0 + tid] = g_rho[gi];
      M[G + h0 + tid] = g_m[gi];
      E[G + h0 + tid] = g_en[gi];
      Ei[G + h0 + tid] = g_ei[gi];
      if constexpr (DF) {
        RL[G + h0 + tid] = g_lo[0][gi];
        ML[G + h0 + tid] = g_lo[1][gi];
        EL[G + h0 + tid] = g_lo[2][gi];
      }
    }
  }
  // Upwind Lagrangian fluxes of one field at the own faces 0 .. nl (Sec. 1.3)
  auto lagrangian_fluxes = [&](const T* q, double dt, T th) {
    auto qq = [&](int c) { return q[c + G]; };
    for (int f0 = tid * run; f0 <= nl; f0 += NTHREADS * run) {
      const int f1 = min(f0 + run - 1, nl);
      stream_faces<T>(qq, f0, f1, [&](int f, const Parab<T>& PL, const Parab<T>& PR) {
        const T vh = FA[f + FO];
        const T y = Prec<T>::courant(tabs(vh), dt, I.h, th);
        FB[f + FO] = vh >= T(0) ? vh * avg_right(PL.R, PL.D, PL.S, y)
                                : vh * avg_left(PR.L, PR.D, PR.S, y);
      });
    }
  };
  // Barriers per step: the CFL reduction (two; in a pair one CTA barrier, the cluster
  // barrier and one more CTA barrier), Eulerian faces, Eulerian update, then in FP32 one
  // after the Lagrangian flux pass; in FP64 one after v hat and two per Lagrangian field
  // but the last.  The last update pass also applies the energy correction, writes the
  // ghosts and takes the next step's CFL maxima.
  for (int s = 0; s < max_steps; s++) {
    double dt;
    T th;
    bool go;
    if constexpr (PAIR)
      go = pair_cfl_step<T, DF ? 7 : 4>(vm, cm, bad, cfl, I, red, xslot, s & 1, P, fields, dt,
                                        th);
    else
      go = block_cfl_step<T>(vm, cm, bad, cfl, I, red, dt, th);
    if (!go) break;
    // Eulerian stage: faces fa .. fb; each thread streams one run of consecutive faces
    {
      auto vq = [&](int k) { return vel_of(M[k + G], R[k + G]); };
      auto pq = [&](int k) { return gm1 * Ei[k + G]; };
      for (int f0 = P.fa + tid * run_e; f0 <= P.fb; f0 += NTHREADS * run_e) {
        const int f1 = min(f0 + run_e - 1, P.fb);
        // rho and sqrt(rho) of the face's left cell, carried from the previous face
        T r_l = R[f0 - 1 + G], s_l = T(0);
        if constexpr (sizeof(T) == 4) s_l = sqrt_approx(r_l);
        stream_faces2<T>(vq, pq, f0, f1,
                         [&](int f, T, T, const Parab<T>& vL, const Parab<T>& vR, T pl, T pr,
                             const Parab<T>& pL, const Parab<T>& pR) {
          const T rl = r_l, rr = R[f + G];
          r_l = rr;
          T V, Pf;
          if constexpr (sizeof(T) == 4) {
            float lam, Z, hrz;
            const float sl = s_l, sr = sqrt_approx(rr);
            s_l = sr;
            face_constants_f32(rl, rr, sl, sr, pl, pr, gamma, lam, Z, hrz);
            const float y = lam * th;
            const float vls = avg_right(vL.R, vL.D, vL.S, y), vrs = avg_left(vR.L, vR.D, vR.S, y);
            const float pls = avg_right(pL.R, pL.D, pL.S, y), prs = avg_left(pR.L, pR.D, pR.S, y);
            V = 0.5f * (vls + vrs) + (pls - prs) * hrz;
            Pf = 0.5f * (pls + prs) + 0.5f * Z * (vls - vrs);
          } else {
            T lam, Z;
            face_constants(rl, rr, pl, pr, gamma, lam, Z);
            const T y = Prec<T>::courant(lam, dt, I.h, th);
            riemann_vp(avg_right(vL.R, vL.D, vL.S, y), avg_left(vR.L, vR.D, vR.S, y),
                       avg_right(pL.R, pL.D, pL.S, y), avg_left(pR.L, pR.D, pR.S, y), Z, V, Pf);
          }
          FA[f + FO] = V;
          FB[f + FO] = Pf;
        });
      }
    }
    __syncthreads();
    // cells c0 + u NTHREADS, u < kU, per pass: every load of the pass ahead of its stores
    // (the compiler cannot move a load past a store into the same shared array)
    for (int c0 = P.ca + tid; c0 < P.cb; c0 += kU * NTHREADS) {
      T Vm[kU], Vp[kU], Pm[kU], Pp[kU], m0[kU], e0[kU], ei0[kU], ml0[kU], el0[kU];
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int c = min(c0 + u * NTHREADS, P.cb - 1), g = c + G;
        Vm[u] = FA[c + FO];
        Vp[u] = FA[c + 1 + FO];
        Pm[u] = FB[c + FO];
        Pp[u] = FB[c + 1 + FO];
        m0[u] = M[g];
        e0[u] = E[g];
        ei0[u] = Ei[g];
        if constexpr (DF) {
          ml0[u] = ML[g];
          el0[u] = EL[g];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; u++) {
        const int c = c0 + u * NTHREADS, g = c + G;
        if (c < P.cb) {
          const T dm = th * (Pp[u] - Pm[u]);
          const T de = th * (Pp[u] * Vp[u] - Pm[u] * Vm[u]);
          const T ei1 = ei0[u] - gm1 * ei0[u] * (th * (Vp[u] - Vm[u]));
          if constexpr (DF) {
            df_sub(m0[u], ml0[u], dm, M[g], ML[g]);
            df_sub(e0[u], el0[u], de, E[g], EL[g]);
          } else {
            M[g] = m0[u] - dm;
            E[g] = e0[u] - de;
          }
          Ei[g] = ei1;
        }
      }
    }
    outer_ghosts(M, P.ca);
    outer_ghosts(E, P.ca);
    outer_ghosts(Ei, P.ca);
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // Lagrangian stage in one pass over each run of faces: v hat (eq. veltemplate with
      // the Roe weights, Sec. 1.3) from the streamed rho and m, each cell's template and
      // sqrt(rho) formed once and carried to the next face, then the upwind fluxes of all
      // four fields
      auto q4 = [&](int j, int k) { return (j == 0 ? R : j == 1 ? M : j == 2 ? E : Ei)[k + G]; };
      for (int f0 = tid * run; f0 <= nl; f0 += NTHREADS * run) {
        const int f1 = min(f0 + run - 1, nl);
        const float r0 = R[f0 - 1 + G];  // cell f0-1
        float vt_l = template_1d(vel_of(M[f0 - 1 + G], r0)), s_l = sqrt_approx(r0);
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
          FA[f + FO] = F[0];
          FB[f + FO] = F[1];
          FC[f + FO] = F[2];
          FD[f + FO] = F[3];
        });
      }
      __syncthreads();
      // every field's update, the Sec. 1.4 energy consistency, the ghosts and the next
      // step's CFL maxima, cell by cell
      vm = T(0);
      cm = T(0);
      for (int c0 = tid; c0 < nl; c0 += kU * NTHREADS) {
        // every field's update (DF: rho, m, rho E added to their double-float pairs)
        float q[kU][4], ql[kU][3];
#pragma unroll
        for (int u = 0; u < kU; u++) {
          const int c = min(c0 + u * NTHREADS, nl - 1), g = c + G;
          const float d0 = th * (FA[c + 1 + FO] - FA[c + FO]);
          const float d1 = th * (FB[c + 1 + FO] - FB[c + FO]);
          const float d2 = th * (FC[c + 1 + FO] - FC[c + FO]);
          if constexpr (DF) {
            df_sub(R[g], RL[g], d0, q[u][0], ql[u][0]);
            df_sub(M[g], ML[g], d1, q[u][1], ql[u][1]);
            df_sub(E[g], EL[g], d2, q[u][2], ql[u][2]);
          } else {
            q[u][0] = R[g] - d0;
            q[u][1] = M[g] - d1;
            q[u][2] = E[g] - d2;
            ql[u][0] = ql[u][1] = ql[u][2] = 0.0f;
          }
          q[u][3] = Ei[g] - th * (FD[c + 1 + FO] - FD[c + FO]);
        }
        // Sec. 1.4: the dense branch for all kU cells without control flow (so that
        // their chains interleave), then the rare vacuum cells
        float w[kU][6], wl[kU][5];
        bool vac[kU], any_vac = false;
#pragma unroll
        for (int u = 0; u < kU; u++) {
          w[u][0] = q[u][0];
          w[u][1] = q[u][1];
          w[u][2] = 0.0f;
          w[u][3] = 0.0f;
          w[u][4] = q[u][2];
          w[u][5] = q[u][3];
          wl[u][0] = ql[u][0];
          wl[u][1] = ql[u][1];
          wl[u][2] = 0.0f;
          wl[u][3] = 0.0f;
          wl[u][4] = ql[u][2];
          vac[u] = vacuum_cell_f32(w[u], rho_vac_up);
          any_vac |= vac[u];
          q[u][3] = DF ? dense_eps_df(w[u], wl[u]) : dense_eps_f32(w[u]);
        }
        if (any_vac) {
#pragma unroll
          for (int u = 0; u < kU; u++)
            if (vac[u]) {
              if constexpr (DF)
                vacuum_correct_df(w[u], wl[u], I.rho_vac);
              else
                vacuum_correct_f32(w[u], I.rho_vac);
              q[u][1] = w[u][1];
              ql[u][1] = wl[u][1];
              q[u][3] = w[u][5];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
          const int c = c0 + u * NTHREADS, g = c + G;
          if (c < nl) {
            R[g] = q[u][0];
            M[g] = q[u][1];
            E[g] = q[u][2];
            Ei[g] = q[u][3];
            if constexpr (DF) {
              RL[g] = ql[u][0];
              ML[g] = ql[u][1];
              EL[g] = ql[u][2];
            }
          }
        }
        // next step's CFL maxima over the valid cells (a clamped duplicate may have read
        // a cell its owner has already updated)
#pragma unroll
        for (int u = 0; u < kU; u++)
          cfl_cell(q[u][0], q[u][1], q[u][2], q[u][3], c0 + u * NTHREADS < nl);
      }
    } else {
      // FP64 Lagrangian stage: v hat at faces, then each field's flux and update in turn
      for (int f = tid; f <= nl; f += NTHREADS) {
        const T rl = R[f - 1 + G], rr = R[f + G];
        const T vtl = template_1d(vel_of(M[f - 1 + G], rl)), vtr = template_1d(vel_of(M[f + G], rr));
        const T sl = sqrt(rl), sr = sqrt(rr);
        FA[f + FO] = (vtr * sr + vtl * sl) / (sr + sl);
      }
      __syncthreads();
      T* fields[3] = {R, M, E};
#pragma unroll 1
      for (int k = 0; k < 3; k++) {
        T* q = fields[k];
        lagrangian_fluxes(q, dt, th);
        __syncthreads();
        for (int c = tid; c < nl; c += NTHREADS)
          q[c + G] = q[c + G] - th * (FB[c + 1 + FO] - FB[c + FO]);
        __syncthreads();
      }
      lagrangian_fluxes(Ei, dt, th);
      __syncthreads();
      // rho eps update, then the Sec. 1.4 energy consistency, on the same cells
      vm = T(0);
      cm = T(0);
      for (int c = tid; c < nl; c += NTHREADS) {
        const int g = c + G;
        const T r = R[g], en = E[g];
        T u[6] = {r, M[g], T(0), T(0), en, Ei[g] - th * (FB[c + 1 + FO] - FB[c + FO])};
        correct_energy<T>(u, I.rho_vac);
        M[g] = u[1];
        Ei[g] = u[5];
        cfl_cell(r, u[1], en, u[5], true);
      }
    }
    outer_ghosts(R, 0);
    outer_ghosts(M, 0);
    outer_ghosts(E, 0);
    outer_ghosts(Ei, 0);
  }
  if constexpr (PAIR) cluster_sync();  // the partner may still read this CTA's slot
  for (int c = tid; c < nl; c += NTHREADS) {
    g_rho[off + c] = R[c + G];
    g_m[off + c] = M[c + G];
    g_en[off + c] = E[c + G];
    g_ei[off + c] = Ei[c + G];
    if constexpr (DF) {
      g_lo[0][off + c] = RL[c + G];
      g_lo[1][off + c] = ML[c + G];
      g_lo[2][off + c] = EL[c + G];
    }
  }
}

// Low parts of rho, m, rho E of a double-float FP32 batch in global memory.
template <typename T>
struct BatchLo {
  T* p[3];
};

template <typename T, int NTHREADS, bool DF>
__global__ void __launch_bounds__(NTHREADS, 1) batch_kernel(T* __restrict__ g_rho,
                                                              T* __restrict__ g_m,
                                                              T* __restrict__ g_en,
                                                              T* __restrict__ g_ei, BatchLo<T> lo,
                                                              InstDev* __restrict__ inst,
                                                              const int* __restrict__ order,
                                                              double gamma_d, double cfl,
                                                              int max_steps, int nmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[80];
  const int id = order[blockIdx.x];
  InstDev I = inst[id];
  if (I.done) return;
  const Part P{I.n, 0, 0, I.n, 0, I.n, true, true};
  advance_part<T, NTHREADS, false, DF>(g_rho, g_m, g_en, g_ei, lo.p, I, P, (T*)smem_raw,
                                       nmax + 2 * kBatchGhost, nmax + 1, gamma_d, cfl, max_steps,
                                       red, nullptr);
  if (threadIdx.x == 0) {  // thread 0's copy holds the instance's time
    if (I.t >= I.t_end) I.done = 1;
    inst[id] = I;
  }
}

// Work item of one cluster of two CTAs (the launch used when some instances are split):
// y == kItemSplit: instance x split over the pair (rank 0 owns cells [0, n/2), rank 1 the
// rest, each with a halo of kPairHalo cells on the side facing its partner); otherwise
// CTA 0 advances instance x and CTA 1 instance y (-1: none), each alone.  Items are
// ordered largest first, so the longest runs take SMs first.
constexpr int kItemSplit = -2;

// In a split instance each CTA forms the Eulerian faces and updates of its cells and of
// the 3 halo cells next to them (its Lagrangian stream reads 3 cells past its last face),
// then the Lagrangian stage of its own faces and cells; the face between the halves is
// formed by both from the same values.  The halo and the CFL maxima are exchanged once
// per step (pair_cfl_step).  Both CTAs of a split item take the same branch and the same
// decisions, so they meet the same cluster barriers; the CTAs of a two-instance item
// never wait on each other.  A split instance needs n >= 2 kPairHalo.
template <typename T, int NTHREADS, bool DF>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    batch_cluster_kernel(T* __restrict__ g_rho, T* __restrict__ g_m, T* __restrict__ g_en,
                         T* __restrict__ g_ei, BatchLo<T> lo, InstDev* __restrict__ inst,
                         const int2* __restrict__ items, double gamma_d, double cfl,
                         int max_steps, int nlmax, int nmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[80];
  __shared__ T xslot[2][kPairSlot];
  T* const* g_lo = lo.p;
  const int rank = (int)cluster_rank();
  const int2 item = items[blockIdx.x >> 1];
  if (item.y == kItemSplit) {
    const int id = item.x;
    InstDev I = inst[id];
    if (I.done) return;  // both CTAs of the pair read the same flag
    const int n = I.n, n0 = n / 2;
    const Part P = rank == 0 ? Part{n0, 0, 0, n0 + 3, 0, n0 + 3, true, false}
                             : Part{n - n0, n0, -3, n - n0, -3, n - n0, false, true};
    advance_part<T, NTHREADS, true, DF>(g_rho, g_m, g_en, g_ei, g_lo, I, P, (T*)smem_raw,
                                    nlmax + 2 * kPairHalo, nlmax + 8, gamma_d, cfl, max_steps,
                                    red, &xslot[0][0]);
    if (rank == 0 && threadIdx.x == 0) {  // both CTAs hold the same time; rank 0 stores it
      if (I.t >= I.t_end) I.done = 1;
      inst[id] = I;
    }
  } else {
    const int id = rank == 0 ? item.x : item.y;
    if (id < 0) return;
    InstDev I = inst[id];
    if (I.done) return;
    const Part P{I.n, 0, 0, I.n, 0, I.n, true, true};
    advance_part<T, NTHREADS, false, DF>(g_rho, g_m, g_en, g_ei, g_lo, I, P, (T*)smem_raw,
                                     nmax + 2 * kBatchGhost, nmax + 1, gamma_d, cfl, max_steps,
                                     red, nullptr);
    if (threadIdx.x == 0) {
      if (I.t >= I.t_end) I.done = 1;
      inst[id] = I;
    }
  }
}

}  // namespace ppml
