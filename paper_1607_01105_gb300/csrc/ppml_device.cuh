// Device building blocks of the PPML step (Kulikov & Vorobyov, arXiv:1607.01105),
// templated on the arithmetic type T (float or double).  Each helper states the passage
// it implements.  Readings of garbled or silent passages (identical to the ones the
// project's independent CPU checker takes):
//   * Delta q = q^R - q^L (Appendix prints q^L - q^R, contradicting eq. A1 and the
//     characteristic averages);
//   * rho_L, rho_R, p_L, p_R inside the Roe averages, lambda and the impedance are the
//     adjacent cell values; only v and p carrying (-+ lambda t) are parabola averages;
//   * the monotonicity step tests "flat" first, then applies at most one overshoot fix.
//
// Precision policy.  The double instantiation is compiled without FMA contraction and
// evaluates every expression in the same order as the FP64 checker (x/6, 2y/3,
// (speed * tau) / h), so the FP64 path reproduces it bit for bit.  The float
// instantiation uses the cheaper forms (doubled slopes, x * (1/12), y * (2/3),
// speed * (tau/h)) and FMAs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ppml {

template <typename T>
struct Prec;

template <>
struct Prec<float> {
  static __device__ __forceinline__ float two_thirds(float y) { return y * (2.0f / 3.0f); }
  // Courant number of a signal speed s: s * tau / h with th = tau / h precomputed.
  static __device__ __forceinline__ float courant(float s, double /*tau*/, double /*h*/,
                                                  float th) {
    return s * th;
  }
};

template <>
struct Prec<double> {
  static __device__ __forceinline__ double two_thirds(double y) { return 2.0 * y / 3.0; }
  static __device__ __forceinline__ double courant(double s, double tau, double h,
                                                   double /*th*/) {
    return s * tau / h;
  }
};

template <typename T>
struct Parab {
  T L, R, D, S;  // q^L, q^R, Delta q = q^R - q^L, q^(6)
};

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Appendix, Step 1: limited slope delta_m q_i.  Branch-free: min(|dq|, 2 min(|r|, |l|))
// equals min(|dq|, 2|r|, 2|l|) exactly (doubling is exact), and r l > 0 implies q is
// strictly monotone, so dq != 0 (up to underflow to a zero of either sign) and the sign
// copy equals the test dq > 0; where r l <= 0 the result is +0 whatever the signs of the
// zeros inside, so fabs (an operand modifier) gives the values of the sign test.
// The FP32 instantiation returns twice the slope, min(|q+ - q-|, 4|r|, 4|l|) with its sign
// (every scaling exact), which face_value expects: the halving is folded into its 1/6.
template <typename T>
__device__ __forceinline__ T limited_slope(T qm, T q0, T qp) {
  const T r = qp - q0, l = q0 - qm;
  if constexpr (sizeof(T) == 8) {  // FP64: evaluate only what is used (same values)
    const T dq = T(0.5) * (qp - qm);
    if (!(r * l > T(0))) return T(0);
    const T m = fmin(fabs(dq), T(2) * fmin(fabs(r), fabs(l)));
    return copysign(m, dq);
  } else {
    const T dq2 = qp - qm;
    const T m2 = fmin(fabs(dq2), T(4) * fmin(fabs(r), fabs(l)));
    return r * l > T(0) ? copysign(m2, dq2) : T(0);
  }
}

// Appendix, Step 1: 4th-order face value q_{i+1/2} from the cell values and limited slopes
// (FP32: from the doubled slopes of limited_slope, (d1 - d0) / 12 = the (d1 - d0) / 6 of
// the halved values).
template <typename T>
__device__ __forceinline__ T face_value(T q0, T q1, T d0, T d1) {
  if constexpr (sizeof(T) == 8)
    return T(0.5) * (q0 + q1) - (d1 - d0) / 6.0;
  else
    return T(0.5) * (q0 + q1) - (d1 - d0) * (1.0f / 12.0f);
}

// Appendix, Steps 2-3: parabola of a cell from its value and its two face values.
// Branch-free: the overshoot tests are evaluated on the unflattened faces and only
// selected when the cell is not flattened, which gives the same values as the
// sequential form (flat test first, then at most one fix).
template <typename T>
__device__ __forceinline__ Parab<T> parabola(T q0, T L, T R) {
  const bool flat = (L - q0) * (q0 - R) <= T(0);
  if (sizeof(T) == 8 && flat) {  // FP64: skip the overshoot tests of a flattened cell
    Parab<T> p;
    p.L = q0;
    p.R = q0;
    p.D = q0 - q0;
    p.S = T(6) * (q0 - T(0.5) * (q0 + q0));
    return p;
  }
  const T D = R - L;
  const T S = T(6) * (q0 - T(0.5) * (L + R));
  // at most one fix: D S > D D >= 0 >= -(D D) excludes D S < -(D D)
  const bool fixL = D * S > D * D;
  const bool fixR = D * S < -(D * D);
  const T Ln = flat ? q0 : (fixL ? T(3) * q0 - T(2) * R : L);
  const T Rn = flat ? q0 : (fixR ? T(3) * q0 - T(2) * L : R);
  Parab<T> p;
  p.L = Ln;
  p.R = Rn;
  p.D = Rn - Ln;
  p.S = T(6) * (q0 - T(0.5) * (Ln + Rn));
  return p;
}

// Appendix, characteristic integrals: mean of the parabola over the right fraction y of
// the cell (q_L(-lambda t), y = lambda t / h) ...
template <typename T>
__device__ __forceinline__ T avg_right(T R, T D, T S, T y) {
  return R - T(0.5) * y * (D - S * (T(1) - Prec<T>::two_thirds(y)));
}
// ... and over its left fraction y (q_R(lambda t)).
template <typename T>
__device__ __forceinline__ T avg_left(T L, T D, T S, T y) {
  return L + T(0.5) * y * (D + S * (T(1) - Prec<T>::two_thirds(y)));
}

// Sec. 1.1/1.2: face constants of the acoustic Riemann problem from the adjacent cell
// values: lambda = sqrt(gamma p^/rho^) and the impedance Z = rho^ lambda.
template <typename T>
__device__ __forceinline__ void face_constants(T rl, T rr, T pl, T pr, T gamma, T& lam, T& Z) {
  const T sl = sqrt(rl), sr = sqrt(rr);
  const T A = rl * sl + rr * sr;  // rho_L^{3/2} + rho_R^{3/2}
  const T B = pl * sl + pr * sr;  // p_L sqrt(rho_L) + p_R sqrt(rho_R)
  const T S = sl + sr;
  lam = sqrt(gamma * B / A);
  Z = sqrt(gamma * A * B / (S * S));
}

// Upwind state of eq. fluxonlagrangestage: the left cell's mean over its right fraction y
// when the face velocity is >= 0, else the right cell's mean over its left fraction y.
// The selected operands go through one evaluation (same operations as avg_right /
// avg_left).
template <typename T>
__device__ __forceinline__ T upwind_state(bool from_left, T R_l, T D_l, T S_l, T L_r, T D_r,
                                          T S_r, T y) {
  const T D = from_left ? D_l : D_r;
  const T S = from_left ? S_l : S_r;
  const T t = S * (T(1) - Prec<T>::two_thirds(y));
  const T u = from_left ? D - t : D + t;
  const T w = T(0.5) * y * u;
  return from_left ? R_l - w : L_r + w;
}

// eqs. lowriemannvelocity / lowriemannpressure from the four characteristic averages.
template <typename T>
__device__ __forceinline__ void riemann_vp(T vls, T vrs, T pls, T prs, T Z, T& V, T& P) {
  V = T(0.5) * (vls + vrs) + (pls - prs) / (T(2) * Z);
  P = T(0.5) * (pls + prs) + T(0.5) * Z * (vls - vrs);
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

// ------------------------------------------------------- approximate FP32 operations
// PTX rcp.approx.f32 / sqrt.approx.f32 (relative error about 2^-23, one special-function
// instruction each).  The FP32 stage kernels use them where the result only feeds
// tolerance-checked FP32 arithmetic (velocities m / rho, Roe weights, the acoustic face
// constants, signal speeds); the FP64 instantiation never does.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP32 face constants (as face_constants) from the adjacent cell values and their square
// roots sl, sr (computed once per cell by the caller): lambda = sqrt(gamma B / A) and
// Z = sqrt(gamma A B) / S = lambda A / S.  Also returns 1 / (2 Z) for the velocity.
__device__ __forceinline__ void face_constants_f32(float rl, float rr, float sl, float sr,
                                                   float pl, float pr, float gamma, float& lam,
                                                   float& Z, float& half_rz) {
  const float A = rl * sl + rr * sr;
  const float B = pl * sl + pr * sr;
  const float S = sl + sr;
  lam = sqrt_approx(gamma * B * rcp_approx(A));
  Z = lam * A * rcp_approx(S);
  half_rz = 0.5f * rcp_approx(Z);
}

// ---------------------------------------------------------- compensated FP32 helpers
// Error-free transformations (Knuth TwoSum; FMA-based TwoProduct).  Used where the
// paper's quantity is a small difference of large totals so that the FP32 path keeps
// FP64-class accuracy without GB300's reduced-rate FP64 pipe.

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// rho eps = rho E - |m|^2 / (2 rho) evaluated in double-float (about 44 significant
// bits) and rounded once to float.  Sec. 1.4 (dense branch).
__device__ __forceinline__ float internal_energy_ff(float rho, float mx, float my, float mz,
                                                    float en) {
  const float p1 = mx * mx, e1 = fmaf(mx, mx, -p1);
  const float p2 = my * my, e2 = fmaf(my, my, -p2);
  const float p3 = mz * mz, e3 = fmaf(mz, mz, -p3);
  float s, t1, hi, t2;
  two_sum(p1, p2, s, t1);
  two_sum(s, p3, hi, t2);
  const float lo = ((t1 + t2) + (e1 + e2)) + e3;  // |m|^2 = hi + lo
  const float r2 = 2.0f * rho;
  const float ir2 = rcp_approx(r2);
  const float q = hi * ir2;
  const float rem = fmaf(-q, r2, hi) + lo;  // remainder of hi (exact to 2^-46) plus lo
  const float ql = rem * ir2;               // |m|^2/(2 rho) = q + ql
  float d, de;
  two_sum(en, -q, d, de);
  return d + (de - ql);
}

// ------------------------------------------------------------ double-float state values
// A field stored as an unevaluated float pair (hi, lo), |lo| <= ulp(hi) / 2, carries about
// 48 significant bits.  The FP32 path keeps rho, m and rho E this way when the caller
// supplies the low parts: the stencil arithmetic reads hi, and every update of a stored
// value and the Sec. 1.4 difference rho E - |m|^2 / (2 rho) use both parts.

// (hi, lo) = (h + l) - d, renormalised (TwoSum of h and -d, then the low terms).
__device__ __forceinline__ void df_sub(float h, float l, float d, float& hi, float& lo) {
  float s, e;
  two_sum(h, -d, s, e);
  e += l;
  hi = s + e;
  lo = e - (hi - s);
}

// Split a double into its float pair.
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// rho eps = (eh + el) - |m|^2 / (2 rho) with rho = rh + rl and m_a = mh_a + ml_a, in
// double-float (about 44 significant bits), rounded once to float.  Sec. 1.4 (dense
// branch) on double-float totals: the error of the difference does not grow with the
// ratio of kinetic to internal energy beyond the double-float rounding.
__device__ __forceinline__ float internal_energy_df(float rh, float rl, const float mh[3],
                                                    const float ml[3], float eh, float el) {
  float p[3], e[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    p[a] = mh[a] * mh[a];
    e[a] = fmaf(mh[a], mh[a], -p[a]) + 2.0f * mh[a] * ml[a];  // ml^2 is below 2^-48 |m|^2
  }
  float s, t1, hi, t2;
  two_sum(p[0], p[1], s, t1);
  two_sum(s, p[2], hi, t2);
  const float lo = ((t1 + t2) + (e[0] + e[1])) + e[2];  // |m|^2 = hi + lo
  const float r2 = 2.0f * rh, r2l = 2.0f * rl;            // 2 rho = r2 + r2l exactly
  const float ir2 = rcp_approx(r2);
  const float q = hi * ir2;
  const float rem = (fmaf(-q, r2, hi) - q * r2l) + lo;  // hi + lo - q (r2 + r2l)
  const float ql = rem * ir2;                           // |m|^2 / (2 rho) = q + ql
  float d, de;
  two_sum(eh, -q, d, de);
  return d + ((de + el) - ql);
}

// Neumaier-compensated running sum in float; value() = hi + lo in double.
struct CompSum {
  float hi, lo;
  __device__ __forceinline__ void init() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x;
    if (fabsf(hi) >= fabsf(x))
      lo += (hi - t) + x;
    else
      lo += (x - t) + hi;
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sec. 1.4 energy correction in the state's precision class: double computes it in
// double; float computes the dense branch in double-float and the (rare) vacuum branch
// in double.  Returns 1 for the vacuum branch.
template <typename T>
__device__ __forceinline__ int correct_energy(T u[6], double rho_vac);
template <>
__device__ __forceinline__ int correct_energy<double>(double u[6], double rho_vac) {
  return energy_correction(u, rho_vac);
}
// rho_vac_up = rho_vac rounded up to float: for any float x, x < rho_vac_up exactly when
// x < rho_vac (no float lies in [rho_vac, rho_vac_up) other than rho_vac itself).
// The two branches separately, for callers that batch cells: whether u takes the vacuum
// branch, the dense branch's rho eps, and the vacuum branch applied to u.
__device__ __forceinline__ bool vacuum_cell_f32(const float u[6], float rho_vac_up) {
  const float m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  return u[0] < rho_vac_up && m2 > 0.f;
}
__device__ __forceinline__ float dense_eps_f32(const float u[6]) {
  const float e = internal_energy_ff(u[0], u[1], u[2], u[3], u[4]);
  return e > 0.f ? e : u[5];
}
__device__ __forceinline__ void vacuum_correct_f32(float u[6], double rho_vac) {
  double d[6] = {u[0], u[1], u[2], u[3], u[4], u[5]};
  energy_correction(d, rho_vac);
  u[1] = (float)d[1];
  u[2] = (float)d[2];
  u[3] = (float)d[3];
  u[5] = (float)d[5];
}
// The same two branches on a double-float state (low parts ul of rho, m, rho E): the dense
// value of rho eps, and the vacuum branch in double on hi + lo (m's pairs and rho eps
// rewritten).
__device__ __forceinline__ float dense_eps_df(const float u[6], const float ul[5]) {
  const float mh[3] = {u[1], u[2], u[3]}, ml[3] = {ul[1], ul[2], ul[3]};
  const float e = internal_energy_df(u[0], ul[0], mh, ml, u[4], ul[4]);
  return e > 0.f ? e : u[5];
}
__device__ __forceinline__ void vacuum_correct_df(float u[6], float ul[5], double rho_vac) {
  double d[6];
#pragma unroll
  for (int f = 0; f < 5; f++) d[f] = (double)u[f] + (double)ul[f];
  d[5] = u[5];
  energy_correction(d, rho_vac);
#pragma unroll
  for (int a = 1; a <= 3; a++) df_split(d[a], u[a], ul[a]);
  u[5] = (float)d[5];
}
__device__ __forceinline__ int correct_energy_f32(float u[6], float rho_vac_up, double rho_vac) {
  if (vacuum_cell_f32(u, rho_vac_up)) {
    vacuum_correct_f32(u, rho_vac);
    return 1;
  }
  u[5] = dense_eps_f32(u);
  return 0;
}
template <>
__device__ __forceinline__ int correct_energy<float>(float u[6], double rho_vac) {
  return correct_energy_f32(u, __double2float_ru(rho_vac), rho_vac);
}

// Boundary handling by index mapping: interior coordinate read for coordinate c of an
// axis with n cells (outflow: clamp; periodic: wrap; reflecting: mirror, flip = 1; halo:
// the cell itself, stored up to kHaloCells beyond the face by the caller -- a neighbouring
// slab's cells).  Coordinates further than that outside the domain (only read for cells
// that produce no output) are clamped into range.
constexpr int kHaloCells = 3;
__device__ __forceinline__ int bc_map(int c, int n, int lo, int hi, int& flip) {
  flip = 0;
  if ((unsigned)c < (unsigned)n) return c;
  const int bc = c < 0 ? lo : hi;
  int r;
  if (bc == 1) {
    r = c < 0 ? c + n : c - n;
  } else if (bc == 2) {
    flip = 1;
    r = c < 0 ? -1 - c : 2 * n - 1 - c;
  } else if (bc == 3) {
    return c < 0 ? max(c, -kHaloCells) : min(c, n - 1 + kHaloCells);
  } else {
    r = c;
  }
  return min(max(r, 0), n - 1);
}

struct GridGeom {
  int n[3];
  int bc[6];
  long long nxy, ncell;
};

// Linear index of possibly out-of-domain cell (i, j, k) after boundary mapping; bit a of
// flips is set when axis a was mirrored (the a-momentum changes sign there).
__device__ __forceinline__ long long map_cell(int i, int j, int k, const GridGeom& g, int& flips) {
  int f0, f1, f2;
  const int ii = bc_map(i, g.n[0], g.bc[0], g.bc[1], f0);
  const int jj = bc_map(j, g.n[1], g.bc[2], g.bc[3], f1);
  const int kk = bc_map(k, g.n[2], g.bc[4], g.bc[5], f2);
  flips = f0 | (f1 << 1) | (f2 << 2);
  return (long long)ii + (long long)g.n[0] * jj + g.nxy * kk;
}

// Sign of field f (0..5; -1 for a scalar) at a cell reached through the mirrors in flips.
__device__ __forceinline__ bool field_flipped(int f, int flips) {
  return f >= 1 && f <= 3 && ((flips >> (f - 1)) & 1);
}

// Value of field `f` at possibly out-of-domain cell (i, j, k), with the momentum component
// normal to a reflecting wall negated.
template <typename T>
__device__ __forceinline__ T load_bc(const T* __restrict__ q, int f, int i, int j, int k,
                                     const GridGeom& g) {
  int fl;
  T v = __ldg(q + map_cell(i, j, k, g, fl));
  return field_flipped(f, fl) ? -v : v;
}

}  // namespace ppml
