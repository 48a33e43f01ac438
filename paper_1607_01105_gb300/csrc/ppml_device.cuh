// Device building blocks of the PPML step (Kulikov & Vorobyov, arXiv:1607.01105),
// templated on the arithmetic type T (float or double).  Each helper states the passage
// it implements.  Readings of garbled or silent passages (identical to the ones the
// project's independent CPU checker takes):
//   * Delta q = q^R - q^L (Appendix prints q^L - q^R, contradicting eq. A1 and the
//     characteristic averages);
//   * rho_L, rho_R, p_L, p_R inside the Roe averages, lambda and the impedance are the
//     adjacent cell values; only v and p carrying (-+ lambda t) are parabola averages;
//   * the monotonicity step tests "flat" first, then applies at most one overshoot fix.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ppml {

template <typename T>
struct Parab {
  T L, R, D, S;  // q^L, q^R, Delta q = q^R - q^L, q^(6)
};

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Appendix, Step 1: limited slope delta_m q_i.
template <typename T>
__device__ __forceinline__ T limited_slope(T qm, T q0, T qp) {
  const T dq = T(0.5) * (qp - qm);
  const T r = qp - q0, l = q0 - qm;
  if (r * l > T(0)) {
    const T m = fmin(tabs(dq), fmin(T(2) * tabs(r), T(2) * tabs(l)));
    return dq > T(0) ? m : -m;
  }
  return T(0);
}

// Appendix, Step 1: 4th-order face value q_{i+1/2} from the cell values and limited slopes.
template <typename T>
__device__ __forceinline__ T face_value(T q0, T q1, T d0, T d1) {
  return T(0.5) * (q0 + q1) - (d1 - d0) * T(1.0 / 6.0);
}

// Appendix, Steps 2-3: parabola of a cell from its value and its two face values.
template <typename T>
__device__ __forceinline__ Parab<T> parabola(T q0, T L, T R) {
  if ((L - q0) * (q0 - R) <= T(0)) {
    L = q0;
    R = q0;
  } else {
    const T D = R - L;
    const T S = T(6) * (q0 - T(0.5) * (L + R));
    if (D * S > D * D)
      L = T(3) * q0 - T(2) * R;
    else if (D * S < -(D * D))
      R = T(3) * q0 - T(2) * L;
  }
  Parab<T> p;
  p.L = L;
  p.R = R;
  p.D = R - L;
  p.S = T(6) * (q0 - T(0.5) * (L + R));
  return p;
}

// Appendix, characteristic integrals: mean of the parabola over the right fraction y of
// the cell (q_L(-lambda t), y = lambda t / h) ...
template <typename T>
__device__ __forceinline__ T avg_right(const Parab<T>& p, T y) {
  return p.R - T(0.5) * y * (p.D - p.S * (T(1) - y * T(2.0 / 3.0)));
}
// ... and over its left fraction y (q_R(lambda t)).
template <typename T>
__device__ __forceinline__ T avg_left(const Parab<T>& p, T y) {
  return p.L + T(0.5) * y * (p.D + p.S * (T(1) - y * T(2.0 / 3.0)));
}

// Parabolas of the three middle cells (offsets -1, 0, +1) of a 7-cell window q[0..6].
template <typename T>
__device__ __forceinline__ void window_parabolas(const T q[7], Parab<T> P[3]) {
  T d[5];
#pragma unroll
  for (int k = 1; k <= 5; k++) d[k - 1] = limited_slope(q[k - 1], q[k], q[k + 1]);
  T f[4];  // faces between window cells k and k+1, k = 1..4
#pragma unroll
  for (int k = 1; k <= 4; k++) f[k - 1] = face_value(q[k], q[k + 1], d[k - 1], d[k]);
#pragma unroll
  for (int c = 0; c < 3; c++) P[c] = parabola(q[c + 2], f[c], f[c + 1]);
}

// Sec. 1.1/1.2: acoustic Riemann solution at a face.  rl, rr, pl, pr: adjacent cell values;
// the parabolas of v and p of the left and right cells; tau_h = tau / h.
template <typename T>
__device__ __forceinline__ void face_riemann(T rl, T rr, T pl, T pr, const Parab<T>& vL,
                                             const Parab<T>& vR, const Parab<T>& pL,
                                             const Parab<T>& pR, T gamma, T tau_h, T& V, T& P) {
  const T sl = sqrt(rl), sr = sqrt(rr);
  const T A = rl * sl + rr * sr;  // rho_L^{3/2} + rho_R^{3/2}
  const T B = pl * sl + pr * sr;  // p_L sqrt(rho_L) + p_R sqrt(rho_R)
  const T S = sl + sr;
  const T lam = sqrt(gamma * B / A);  // lambda = sqrt(gamma p^/rho^)
  const T y = lam * tau_h;
  const T vls = avg_right(vL, y), vrs = avg_left(vR, y);
  const T pls = avg_right(pL, y), prs = avg_left(pR, y);
  const T Z = sqrt(gamma * A * B / (S * S));  // impedance rho^ lambda
  V = T(0.5) * (vls + vrs) + (pls - prs) / (T(2) * Z);
  P = T(0.5) * (pls + prs) + T(0.5) * Z * (vls - vrs);
}

// Sec. 1.3, eq. fluxonlagrangestage: upwind flux through a face with velocity vh between
// the cells with parabolas PL and PR.
template <typename T>
__device__ __forceinline__ T upwind_flux(T vh, const Parab<T>& PL, const Parab<T>& PR, T tau_h) {
  const T y = tabs(vh) * tau_h;
  return vh >= T(0) ? vh * avg_right(PL, y) : vh * avg_left(PR, y);
}

// Sec. 1.4: energy consistency of one cell, in double.  u = {rho, mx, my, mz, rhoE, rhoeps}.
// Returns 1 if the cell took the vacuum branch.
__device__ __forceinline__ int energy_correction(double u[6], double rho_vac) {
  const double rho = u[0];
  const double m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  if (rho < rho_vac && m2 > 0.0) {
    const double de = u[4] - u[5];
    if (de < 0.0) {
      u[1] = u[2] = u[3] = 0.0;
      u[5] = u[4];
      return 1;
    }
    const double vnew = sqrt(2.0 * de / rho);
    const double vold = sqrt(m2) / rho;
    const double s = vnew / vold;
    u[1] *= s;
    u[2] *= s;
    u[3] *= s;
    return 1;
  }
  const double e = u[4] - m2 / (2.0 * rho);
  if (e > 0.0) u[5] = e;
  return 0;
}

// Boundary handling by index mapping: interior coordinate read for coordinate c of an
// axis with n cells (outflow: clamp; periodic: wrap; reflecting: mirror, flip = 1).
__device__ __forceinline__ int bc_map(int c, int n, int lo, int hi, int& flip) {
  flip = 0;
  if (c >= 0 && c < n) return c;
  const int bc = c < 0 ? lo : hi;
  if (bc == 1) {
    int r = c % n;
    return r < 0 ? r + n : r;
  }
  if (bc == 2) {
    flip = 1;
    int r = c < 0 ? -1 - c : 2 * n - 1 - c;
    return r < 0 ? 0 : (r > n - 1 ? n - 1 : r);
  }
  return c < 0 ? 0 : n - 1;
}

struct GridGeom {
  int n[3];
  int bc[6];
  long long nxy, ncell;
};

// Value of field `f` (0..5) at possibly out-of-domain cell (i, j, k), with the momentum
// component normal to a reflecting wall negated.
template <typename T>
__device__ __forceinline__ T load_bc(const T* __restrict__ q, int f, int i, int j, int k,
                                     const GridGeom& g) {
  int fx, fy, fz;
  const int ii = bc_map(i, g.n[0], g.bc[0], g.bc[1], fx);
  const int jj = bc_map(j, g.n[1], g.bc[2], g.bc[3], fy);
  const int kk = bc_map(k, g.n[2], g.bc[4], g.bc[5], fz);
  T v = __ldg(q + (long long)ii + (long long)g.n[0] * jj + g.nxy * kk);
  if ((f == 1 && fx) || (f == 2 && fy) || (f == 3 && fz)) v = -v;
  return v;
}

}  // namespace ppml
