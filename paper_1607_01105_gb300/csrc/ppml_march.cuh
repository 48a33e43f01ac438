// z-marching stencil kernels of one PPML step (Kulikov & Vorobyov, arXiv:1607.01105).
//
// Layout of the work: a CTA owns a TX x TY column tile of the (x, y) plane and marches a
// chunk of z planes.  Per output plane:
//   * z direction: a per-column register pipeline.  Each incoming plane (k+3) adds one
//     limited slope, one face value, one parabola and one face flux, so every quantity
//     along z is computed exactly once (Appendix Steps 1-3 and the characteristic
//     averages, eq. fluxonlagrangestage / lowriemann*).
//   * x and y directions: the plane with a 3-cell halo is staged in shared memory and the
//     same quantities are built in phases (slopes -> faces -> parabolas with their two
//     characteristic averages -> per-cell face fluxes), each computed once per cell or
//     face plus the halo.
//   * the 9-point velocity template (eq. veltemplate) reads a 3-plane ring of v = m/rho
//     over the tile plus a one-cell halo.
// Boundaries are index maps on every load (outflow / periodic / reflecting), so no ghost
// cells exist in memory.  Axes with a single cell are skipped (their fluxes are exactly
// zero).  The sum over axes of the updates is taken in the order x, y, z.
#pragma once
#include "ppml_device.cuh"

namespace ppml {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HALO = 3;
constexpr int RX = TX + 2 * HALO, RY = TY + 2 * HALO;  // staged plane, 38 x 14
constexpr int VXW = TX + 2, VYW = TY + 2;              // template region, 34 x 10
constexpr int VREG = VXW * VYW;

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
  const T* phi;   // optional potential (Eulerian stage)
  GridGeom g;
  double h[3];
  double gamma;
  double dt_host;        // used when dt_dev == NULL
  const double* dt_dev;  // device-resident step
  double rho_vac;
  Partial* partials;
  int tiles_x, tiles_y, nchunks, kc;
};

__device__ __forceinline__ double read_tau(const double* dt_dev, double dt_host) {
  return dt_dev ? *dt_dev : dt_host;
}

// ------------------------------------------------------------------ block reduction

template <int NTHREADS>
__device__ __forceinline__ void block_reduce_store(double s[6], double vmax, double cmax,
                                                   unsigned long long nvac,
                                                   unsigned long long nbad, Partial* out) {
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
    out[blockIdx.x] = p;
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

// Tile / chunk of a CTA (x tiles fastest, then y tiles, then z chunks).
struct TileInfo {
  int x0, y0, k0, k1;
};
__device__ __forceinline__ TileInfo tile_of(int b, int tiles_x, int tiles_y, int kc, int nz) {
  TileInfo t;
  const int txi = b % tiles_x;
  b /= tiles_x;
  const int tyi = b % tiles_y;
  const int ch = b / tiles_y;
  t.x0 = txi * TX;
  t.y0 = tyi * TY;
  t.k0 = ch * kc;
  t.k1 = min(t.k0 + kc, nz);
  return t;
}

__device__ __forceinline__ int ring3(int p) { return ((p % 3) + 3) % 3; }
__device__ __forceinline__ int ring2(int p) { return p & 1; }

// ===================================================================== Lagrangian stage

template <typename T>
struct LagSmem {
  T Q[6][RY][RX];         // plane k of U* with a 3-cell halo
  T DX[TY][TX + 4];       // x slopes, cells x in [-2, TX+1]
  T DY[TY + 4][TX];       // y slopes, cells y in [-2, TY+1]
  T FX[TY][TX + 3];       // x faces between x and x+1, x in [-2, TX]
  T FY[TY + 3][TX];       // y faces, y in [-2, TY]
  T AX[2][2][TY][TX + 2]; // [buf][R/L] averages, cells x in [-1, TX]
  T AY[2][2][TY + 2][TX]; // [buf][R/L] averages, cells y in [-1, TY]
  T VHX[TY][TX + 1];      // v hat on x faces, x in [-1, TX-1]
  T YX[TY][TX + 1];       // |v hat| tau / h_x
  T VHY[TY + 1][TX];      // v hat on y faces, y in [-1, TY-1]
  T YY[TY + 1][TX];
  T TVX[TY][TX + 2];      // v tilde_x, cells x in [-1, TX]
  T TVY[TY + 2][TX];      // v tilde_y, cells y in [-1, TY]
  T V[3][3][VYW][VXW];    // ring of v_x, v_y, v_z over the tile + 1 halo, planes k-1..k+1
  T SQ[2][VYW][VXW];      // ring of sqrt(rho), planes k, k+1
};

// z-pipeline state of one field for one column.
template <typename T>
struct ZPipe {
  T qa, qb;      // q(k+1), q(k+2) on entry of iteration k
  T da;          // slope at k+1
  T fa;          // face k+1/2
  T PR, PD, PS;  // parabola of cell k (R, Delta, q6)
  T Fa;          // flux at k-1/2
};

template <typename T, int MINB>
__global__ void __launch_bounds__(NT, MINB) lagrangian_march(MarchArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LagSmem<T>& S = *reinterpret_cast<LagSmem<T>*>(smem_raw);
  const GridGeom& g = A.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const bool ax = nx > 1, ay = ny > 1, az = nz > 1;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const TileInfo ti = tile_of(blockIdx.x, A.tiles_x, A.tiles_y, A.kc, nz);
  const int gx = ti.x0 + tx, gy = ti.y0 + ty;
  const bool own = gx < nx && gy < ny;
  const double tau = read_tau(A.dt_dev, A.dt_host);
  const T th[3] = {T(tau / A.h[0]), T(tau / A.h[1]), T(tau / A.h[2])};
  const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);

  ZPipe<T> zp[6];
  T vtz_c = T(0), sq_c = T(0), vhz = T(0), yz = T(0);
  FieldSums<T> sums;
  sums.init();
  T vmax = T(0), cmax = T(0);
  unsigned long long nvac = 0, nbad = 0;

  // column loads with boundary mapping (threads outside the domain read mapped cells)
  auto col_load = [&](int f, int k) -> T {
    const T* src = (f == 0) ? A.u[0] : A.u[f];
    return load_bc(src, f, gx, gy, k, g);
  };

  const int kstart = az ? ti.k0 - 4 : ti.k0;
  if (az) {
#pragma unroll
    for (int f = 0; f < 6; f++) {
      zp[f].qa = col_load(f, kstart + 1);  // q(k+1) for k = kstart
      zp[f].qb = col_load(f, kstart + 2);
      zp[f].da = T(0);
      zp[f].fa = T(0);
      zp[f].PR = zp[f].PD = zp[f].PS = T(0);
      zp[f].Fa = T(0);
    }
  }

  for (int k = kstart; k < ti.k1; k++) {
    // ---- template ring: plane k+1 (needed from k = k0-2 on); with a single plane in z
    //      every plane maps onto plane k itself, kept in the slot of k
    const int p1 = az ? k + 1 : k;
    if (k >= ti.k0 - 2 || !az) {
      const int sv = ring3(p1), ss = ring2(p1);
      for (int it = tid; it < VREG; it += NT) {
        const int ix = it % VXW, iy = it / VXW;
        int fl[3];
        const long long c = map_cell(ti.x0 - 1 + ix, ti.y0 - 1 + iy, p1, g, fl);
        const T r = A.u[0][c];
        T mx = A.u[1][c], my = A.u[2][c], mz = A.u[3][c];
        if (fl[0]) mx = -mx;
        if (fl[1]) my = -my;
        if (fl[2]) mz = -mz;
        S.V[0][sv][iy][ix] = mx / r;
        S.V[1][sv][iy][ix] = my / r;
        S.V[2][sv][iy][ix] = mz / r;
        S.SQ[ss][iy][ix] = sqrt(r);
      }
    }
    // ---- z-pipeline input q(k+3)
    T qn[6];
    if (az) {
#pragma unroll
      for (int f = 0; f < 6; f++) qn[f] = col_load(f, k + 3);
    }
    // ---- plane k staged with halo (only for output planes)
    const bool out_plane = k >= ti.k0;
    if (out_plane) {
      for (int it = tid; it < RX * RY; it += NT) {
        const int ix = it % RX, iy = it / RX;
        int fl[3];
        const long long c = map_cell(ti.x0 - HALO + ix, ti.y0 - HALO + iy, k, g, fl);
#pragma unroll
        for (int f = 0; f < 6; f++) {
          T v = A.u[f][c];
          if ((f == 1 && fl[0]) || (f == 2 && fl[1]) || (f == 3 && fl[2])) v = -v;
          S.Q[f][iy][ix] = v;
        }
      }
    }
    __syncthreads();

    // ---- z: template of v_z at plane k+1 for this column, face velocity at k+1/2
    if (az && k >= ti.k0 - 2) {
      const int sv = ring3(p1), ss = ring2(p1);
      const int cx = tx + 1, cy = ty + 1;
      // axis z: b = x, c = y (eq. veltemplate with the roles of the checker)
      const T corners = S.V[2][sv][cy + 1][cx + 1] + S.V[2][sv][cy - 1][cx + 1] +
                        S.V[2][sv][cy + 1][cx - 1] + S.V[2][sv][cy - 1][cx - 1];
      const T edges = S.V[2][sv][cy][cx + 1] + S.V[2][sv][cy][cx - 1] +
                      S.V[2][sv][cy + 1][cx] + S.V[2][sv][cy - 1][cx];
      const T vt = corners / T(16) + edges / T(8) + S.V[2][sv][cy][cx] / T(4);
      const T sq = S.SQ[ss][cy][cx];
      if (k >= ti.k0 - 1) {
        vhz = (vt * sq + vtz_c * sq_c) / (sq + sq_c);
        yz = Prec<T>::courant(tabs(vhz), tau, A.h[2], th[2]);
      }
      vtz_c = vt;
      sq_c = sq;
    }

    T divz[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (az) {
#pragma unroll
      for (int f = 0; f < 6; f++) {
        ZPipe<T>& z = zp[f];
        const T dn = limited_slope(z.qa, z.qb, qn[f]);             // slope at k+2
        const T fn = face_value(z.qa, z.qb, z.da, dn);             // face k+3/2
        const Parab<T> P = parabola(z.qa, z.fa, fn);               // cell k+1
        if (k >= ti.k0 - 1) {
          const T Fn = vhz >= T(0) ? vhz * avg_right(z.PR, z.PD, z.PS, yz)
                                   : vhz * avg_left(P.L, P.D, P.S, yz);  // face k+1/2
          if (k >= ti.k0) divz[f] = th[2] * (Fn - z.Fa);
          z.Fa = Fn;
        }
        z.qa = z.qb;
        z.qb = qn[f];
        z.da = dn;
        z.fa = fn;
        z.PR = P.R;
        z.PD = P.D;
        z.PS = P.S;
      }
    }
    if (!out_plane) {
      __syncthreads();
      continue;
    }

    // ---- in-plane templates: v tilde_x (cells x in [-1, TX], rows of the tile) and
    //      v tilde_y (cells y in [-1, TY]), from the v ring at planes k-1, k, k+1
    const int s0 = ring3(k);
    const int sm = az ? ring3(k - 1) : s0, sp = az ? ring3(k + 1) : s0;
    if (ax) {
      for (int it = tid; it < TY * (TX + 2); it += NT) {
        const int ix = it % (TX + 2), iy = it / (TX + 2);  // cell x = ix-1, y = iy
        const int cx = ix, cy = iy + 1;                      // template-region coords
        // axis x: b = y, c = z
        const T corners = S.V[0][sp][cy + 1][cx] + S.V[0][sm][cy + 1][cx] +
                          S.V[0][sp][cy - 1][cx] + S.V[0][sm][cy - 1][cx];
        const T edges = S.V[0][s0][cy + 1][cx] + S.V[0][s0][cy - 1][cx] +
                        S.V[0][sp][cy][cx] + S.V[0][sm][cy][cx];
        S.TVX[iy][ix] = corners / T(16) + edges / T(8) + S.V[0][s0][cy][cx] / T(4);
      }
    }
    if (ay) {
      for (int it = tid; it < (TY + 2) * TX; it += NT) {
        const int ix = it % TX, iy = it / TX;  // cell x = ix, y = iy-1
        const int cx = ix + 1, cy = iy;
        // axis y: b = z, c = x
        const T corners = S.V[1][sp][cy][cx + 1] + S.V[1][sp][cy][cx - 1] +
                          S.V[1][sm][cy][cx + 1] + S.V[1][sm][cy][cx - 1];
        const T edges = S.V[1][sp][cy][cx] + S.V[1][sm][cy][cx] +
                        S.V[1][s0][cy][cx + 1] + S.V[1][s0][cy][cx - 1];
        S.TVY[iy][ix] = corners / T(16) + edges / T(8) + S.V[1][s0][cy][cx] / T(4);
      }
    }
    __syncthreads();
    const int ssq = ring2(k);
    if (ax) {
      for (int it = tid; it < TY * (TX + 1); it += NT) {
        const int ix = it % (TX + 1), iy = it / (TX + 1);  // face between x = ix-1 and ix
        const T sl = S.SQ[ssq][iy + 1][ix], sr = S.SQ[ssq][iy + 1][ix + 1];
        const T vh = (S.TVX[iy][ix + 1] * sr + S.TVX[iy][ix] * sl) / (sr + sl);
        S.VHX[iy][ix] = vh;
        S.YX[iy][ix] = Prec<T>::courant(tabs(vh), tau, A.h[0], th[0]);
      }
    }
    if (ay) {
      for (int it = tid; it < (TY + 1) * TX; it += NT) {
        const int ix = it % TX, iy = it / TX;  // face between y = iy-1 and iy
        const T sl = S.SQ[ssq][iy][ix + 1], sr = S.SQ[ssq][iy + 1][ix + 1];
        const T vh = (S.TVY[iy + 1][ix] * sr + S.TVY[iy][ix] * sl) / (sr + sl);
        S.VHY[iy][ix] = vh;
        S.YY[iy][ix] = Prec<T>::courant(tabs(vh), tau, A.h[1], th[1]);
      }
    }
    // (the first field's slope phase below writes only DX/DY; the sync after it orders
    //  the VH/Y writes before their first reads in the parabola phase)

    T unew[6];
#pragma unroll 1
    for (int f = 0; f < 6; f++) {
      const int buf = f & 1;
      // phase A: limited slopes
      if (ax)
        for (int it = tid; it < TY * (TX + 4); it += NT) {
          const int ix = it % (TX + 4), iy = it / (TX + 4);  // cell x = ix-2
          const T* row = &S.Q[f][iy + HALO][0];
          const int c = ix - 2 + HALO;
          S.DX[iy][ix] = limited_slope(row[c - 1], row[c], row[c + 1]);
        }
      if (ay)
        for (int it = tid; it < (TY + 4) * TX; it += NT) {
          const int ix = it % TX, iy = it / TX;  // cell y = iy-2
          const int c = iy - 2 + HALO, cx = ix + HALO;
          S.DY[iy][ix] = limited_slope(S.Q[f][c - 1][cx], S.Q[f][c][cx], S.Q[f][c + 1][cx]);
        }
      __syncthreads();
      // phase B: face values
      if (ax)
        for (int it = tid; it < TY * (TX + 3); it += NT) {
          const int ix = it % (TX + 3), iy = it / (TX + 3);  // face between x = ix-2, ix-1
          const T* row = &S.Q[f][iy + HALO][0];
          const int c = ix - 2 + HALO;
          S.FX[iy][ix] = face_value(row[c], row[c + 1], S.DX[iy][ix], S.DX[iy][ix + 1]);
        }
      if (ay)
        for (int it = tid; it < (TY + 3) * TX; it += NT) {
          const int ix = it % TX, iy = it / TX;  // face between y = iy-2, iy-1
          const int c = iy - 2 + HALO, cx = ix + HALO;
          S.FY[iy][ix] = face_value(S.Q[f][c][cx], S.Q[f][c + 1][cx], S.DY[iy][ix], S.DY[iy + 1][ix]);
        }
      __syncthreads();
      // phase C: parabolas and their characteristic averages toward both faces
      if (ax)
        for (int it = tid; it < TY * (TX + 2); it += NT) {
          const int ix = it % (TX + 2), iy = it / (TX + 2);  // cell x = ix-1
          const T q0 = S.Q[f][iy + HALO][ix - 1 + HALO];
          const Parab<T> P = parabola(q0, S.FX[iy][ix], S.FX[iy][ix + 1]);
          // right face of cell x is face index x+1 = ix; left face is ix-1
          const T yr = ix <= TX ? S.YX[iy][ix] : T(0);
          const T yl = ix >= 1 ? S.YX[iy][ix - 1] : T(0);
          S.AX[buf][0][iy][ix] = avg_right(P.R, P.D, P.S, yr);
          S.AX[buf][1][iy][ix] = avg_left(P.L, P.D, P.S, yl);
        }
      if (ay)
        for (int it = tid; it < (TY + 2) * TX; it += NT) {
          const int ix = it % TX, iy = it / TX;  // cell y = iy-1
          const T q0 = S.Q[f][iy - 1 + HALO][ix + HALO];
          const Parab<T> P = parabola(q0, S.FY[iy][ix], S.FY[iy + 1][ix]);
          const T yr = iy <= TY ? S.YY[iy][ix] : T(0);
          const T yl = iy >= 1 ? S.YY[iy - 1][ix] : T(0);
          S.AY[buf][0][iy][ix] = avg_right(P.R, P.D, P.S, yr);
          S.AY[buf][1][iy][ix] = avg_left(P.L, P.D, P.S, yl);
        }
      __syncthreads();
      // phase D: upwind fluxes through the cell's faces and the unsplit update (x, y, z)
      T acc = T(0);
      if (ax) {
        const T vl = S.VHX[ty][tx], vr = S.VHX[ty][tx + 1];
        const T Fl = vl >= T(0) ? vl * S.AX[buf][0][ty][tx] : vl * S.AX[buf][1][ty][tx + 1];
        const T Fr = vr >= T(0) ? vr * S.AX[buf][0][ty][tx + 1] : vr * S.AX[buf][1][ty][tx + 2];
        acc = th[0] * (Fr - Fl);
      }
      if (ay) {
        const T vl = S.VHY[ty][tx], vr = S.VHY[ty + 1][tx];
        const T Fl = vl >= T(0) ? vl * S.AY[buf][0][ty][tx] : vl * S.AY[buf][1][ty + 1][tx];
        const T Fr = vr >= T(0) ? vr * S.AY[buf][0][ty + 1][tx] : vr * S.AY[buf][1][ty + 2][tx];
        acc = acc + th[1] * (Fr - Fl);
      }
      if (az) acc = acc + divz[f];
      unew[f] = S.Q[f][ty + HALO][tx + HALO] - acc;
    }

    if (own) {
      nvac += correct_energy<T>(unew, A.rho_vac);
      const long long c = (long long)gx + (long long)nx * gy + g.nxy * k;
#pragma unroll
      for (int f = 0; f < 6; f++) A.out[f][c] = unew[f];
      sums.add(unew);
      cell_speeds<T>(unew, gamma, gm1, vmax, cmax, nbad);
    }
    __syncthreads();  // the next plane overwrites the staged arrays
  }
  double sd[6];
  sums.get(sd);
  block_reduce_store<NT>(sd, (double)vmax, (double)cmax, nvac, nbad, A.partials);
}

// ====================================================================== Eulerian stage

template <typename T>
struct EulSmem {
  T R[RY][RX];             // rho, plane k with halo
  T VX[RY][RX];            // v_x
  T VY[RY][RX];            // v_y
  T P[RY][RX];             // p
  T DX[2][TY][TX + 4];     // x slopes of v_x, p
  T DY[2][TY + 4][TX];     // y slopes of v_y, p
  T FX[2][TY][TX + 3];     // x faces of v_x, p
  T FY[2][TY + 3][TX];     // y faces of v_y, p
  T CX[2][TY][TX + 1];     // x-face lambda*tau/h and impedance
  T CY[2][TY + 1][TX];
  T AX[2][2][TY][TX + 2];  // [v/p][R/L] averages, cells x in [-1, TX]
  T AY[2][2][TY + 2][TX];
};

template <typename T>
struct ZPipeE {
  T qa, qb, da, fa, PR, PD, PS;  // as ZPipe, for v_z and p
};

template <typename T, int MINB>
__global__ void __launch_bounds__(NT, MINB) eulerian_march(MarchArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EulSmem<T>& S = *reinterpret_cast<EulSmem<T>*>(smem_raw);
  const GridGeom& g = A.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const bool ax = nx > 1, ay = ny > 1, az = nz > 1;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const TileInfo ti = tile_of(blockIdx.x, A.tiles_x, A.tiles_y, A.kc, nz);
  const int gx = ti.x0 + tx, gy = ti.y0 + ty;
  const bool own = gx < nx && gy < ny;
  const double tau = read_tau(A.dt_dev, A.dt_host);
  const T th[3] = {T(tau / A.h[0]), T(tau / A.h[1]), T(tau / A.h[2])};
  const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);

  // z pipeline: v_z and p, plus the cell values rho, p around the z faces
  ZPipeE<T> zv, zq;
  T r1 = T(0), r2 = T(0), pz0 = T(0);  // rho(k+1), rho(k+2); p(k)
  T r0 = T(0);                         // rho(k)
  T Vz = T(0), Pz = T(0);              // face k-1/2 solution carried
  auto col = [&](int f, int k) -> T { return load_bc(A.u[f], f, gx, gy, k, g); };

  const int kstart = az ? ti.k0 - 4 : ti.k0;
  if (az) {
    const T ra = col(0, kstart + 1), rb = col(0, kstart + 2);
    zv.qa = col(3, kstart + 1) / ra;
    zv.qb = col(3, kstart + 2) / rb;
    zq.qa = gm1 * col(5, kstart + 1);
    zq.qb = gm1 * col(5, kstart + 2);
    r1 = ra;
    r2 = rb;
    r0 = col(0, kstart);
    pz0 = gm1 * col(5, kstart);
    zv.da = zv.fa = zv.PR = zv.PD = zv.PS = T(0);
    zq.da = zq.fa = zq.PR = zq.PD = zq.PS = T(0);
  }

  for (int k = kstart; k < ti.k1; k++) {
    const bool out_plane = k >= ti.k0;
    T dmz = T(0), dpvz = T(0), dvz = T(0);
    if (az) {
      const T r3 = col(0, k + 3);
      const T vn = col(3, k + 3) / r3;
      const T pn = gm1 * col(5, k + 3);
      // new slopes / faces / parabolas of cell k+1
      const T dnv = limited_slope(zv.qa, zv.qb, vn);
      const T fnv = face_value(zv.qa, zv.qb, zv.da, dnv);
      const Parab<T> Pv = parabola(zv.qa, zv.fa, fnv);
      const T dnp = limited_slope(zq.qa, zq.qb, pn);
      const T fnp = face_value(zq.qa, zq.qb, zq.da, dnp);
      const Parab<T> Pp = parabola(zq.qa, zq.fa, fnp);
      if (k >= ti.k0 - 1) {
        // face k+1/2 between cells k (carried parabola) and k+1
        T lam, Z;
        face_constants(r0, r1, pz0, zq.qa, gamma, lam, Z);
        const T y = Prec<T>::courant(lam, tau, A.h[2], th[2]);
        const T vls = avg_right(zv.PR, zv.PD, zv.PS, y), vrs = avg_left(Pv.L, Pv.D, Pv.S, y);
        const T pls = avg_right(zq.PR, zq.PD, zq.PS, y), prs = avg_left(Pp.L, Pp.D, Pp.S, y);
        T Vn, Pn;
        riemann_vp(vls, vrs, pls, prs, Z, Vn, Pn);
        if (out_plane) {
          dmz = th[2] * (Pn - Pz);
          dpvz = th[2] * (Pn * Vn - Pz * Vz);
          dvz = th[2] * (Vn - Vz);
        }
        Vz = Vn;
        Pz = Pn;
      }
      pz0 = zq.qa;
      r0 = r1;
      r1 = r2;
      r2 = r3;
      zv.qa = zv.qb;
      zv.qb = vn;
      zv.da = dnv;
      zv.fa = fnv;
      zv.PR = Pv.R;
      zv.PD = Pv.D;
      zv.PS = Pv.S;
      zq.qa = zq.qb;
      zq.qb = pn;
      zq.da = dnp;
      zq.fa = fnp;
      zq.PR = Pp.R;
      zq.PD = Pp.D;
      zq.PS = Pp.S;
    }
    if (!out_plane) continue;

    // ---- stage plane k: rho, v_x, v_y, p
    for (int it = tid; it < RX * RY; it += NT) {
      const int ix = it % RX, iy = it / RX;
      int fl[3];
      const long long c = map_cell(ti.x0 - HALO + ix, ti.y0 - HALO + iy, k, g, fl);
      const T r = A.u[0][c];
      T mx = A.u[1][c], my = A.u[2][c];
      if (fl[0]) mx = -mx;
      if (fl[1]) my = -my;
      S.R[iy][ix] = r;
      S.VX[iy][ix] = mx / r;
      S.VY[iy][ix] = my / r;
      S.P[iy][ix] = gm1 * A.u[5][c];
    }
    __syncthreads();
    // phase A: slopes (x: v_x, p; y: v_y, p) and face constants
    if (ax) {
      for (int it = tid; it < 2 * TY * (TX + 4); it += NT) {
        const int q = it / (TY * (TX + 4)), r = it % (TY * (TX + 4));
        const int ix = r % (TX + 4), iy = r / (TX + 4);
        const T* row = q == 0 ? &S.VX[iy + HALO][0] : &S.P[iy + HALO][0];
        const int c = ix - 2 + HALO;
        S.DX[q][iy][ix] = limited_slope(row[c - 1], row[c], row[c + 1]);
      }
      for (int it = tid; it < TY * (TX + 1); it += NT) {
        const int ix = it % (TX + 1), iy = it / (TX + 1);  // face between x = ix-1 and ix
        const int c = ix - 1 + HALO, cy = iy + HALO;
        T lam, Z;
        face_constants(S.R[cy][c], S.R[cy][c + 1], S.P[cy][c], S.P[cy][c + 1], gamma, lam, Z);
        S.CX[0][iy][ix] = Prec<T>::courant(lam, tau, A.h[0], th[0]);
        S.CX[1][iy][ix] = Z;
      }
    }
    if (ay) {
      for (int it = tid; it < 2 * (TY + 4) * TX; it += NT) {
        const int q = it / ((TY + 4) * TX), r = it % ((TY + 4) * TX);
        const int ix = r % TX, iy = r / TX;
        const int c = iy - 2 + HALO, cx = ix + HALO;
        if (q == 0)
          S.DY[0][iy][ix] = limited_slope(S.VY[c - 1][cx], S.VY[c][cx], S.VY[c + 1][cx]);
        else
          S.DY[1][iy][ix] = limited_slope(S.P[c - 1][cx], S.P[c][cx], S.P[c + 1][cx]);
      }
      for (int it = tid; it < (TY + 1) * TX; it += NT) {
        const int ix = it % TX, iy = it / TX;  // face between y = iy-1 and iy
        const int c = iy - 1 + HALO, cx = ix + HALO;
        T lam, Z;
        face_constants(S.R[c][cx], S.R[c + 1][cx], S.P[c][cx], S.P[c + 1][cx], gamma, lam, Z);
        S.CY[0][iy][ix] = Prec<T>::courant(lam, tau, A.h[1], th[1]);
        S.CY[1][iy][ix] = Z;
      }
    }
    __syncthreads();
    // phase B: faces
    if (ax)
      for (int it = tid; it < 2 * TY * (TX + 3); it += NT) {
        const int q = it / (TY * (TX + 3)), r = it % (TY * (TX + 3));
        const int ix = r % (TX + 3), iy = r / (TX + 3);
        const T* row = q == 0 ? &S.VX[iy + HALO][0] : &S.P[iy + HALO][0];
        const int c = ix - 2 + HALO;
        S.FX[q][iy][ix] = face_value(row[c], row[c + 1], S.DX[q][iy][ix], S.DX[q][iy][ix + 1]);
      }
    if (ay)
      for (int it = tid; it < 2 * (TY + 3) * TX; it += NT) {
        const int q = it / ((TY + 3) * TX), r = it % ((TY + 3) * TX);
        const int ix = r % TX, iy = r / TX;
        const int c = iy - 2 + HALO, cx = ix + HALO;
        const T a = q == 0 ? S.VY[c][cx] : S.P[c][cx];
        const T b = q == 0 ? S.VY[c + 1][cx] : S.P[c + 1][cx];
        S.FY[q][iy][ix] = face_value(a, b, S.DY[q][iy][ix], S.DY[q][iy + 1][ix]);
      }
    __syncthreads();
    // phase C: parabolas and characteristic averages with the face lambda
    if (ax)
      for (int it = tid; it < 2 * TY * (TX + 2); it += NT) {
        const int q = it / (TY * (TX + 2)), r = it % (TY * (TX + 2));
        const int ix = r % (TX + 2), iy = r / (TX + 2);  // cell x = ix-1
        const T q0 = q == 0 ? S.VX[iy + HALO][ix - 1 + HALO] : S.P[iy + HALO][ix - 1 + HALO];
        const Parab<T> P = parabola(q0, S.FX[q][iy][ix], S.FX[q][iy][ix + 1]);
        const T yr = ix <= TX ? S.CX[0][iy][ix] : T(0);
        const T yl = ix >= 1 ? S.CX[0][iy][ix - 1] : T(0);
        S.AX[q][0][iy][ix] = avg_right(P.R, P.D, P.S, yr);
        S.AX[q][1][iy][ix] = avg_left(P.L, P.D, P.S, yl);
      }
    if (ay)
      for (int it = tid; it < 2 * (TY + 2) * TX; it += NT) {
        const int q = it / ((TY + 2) * TX), r = it % ((TY + 2) * TX);
        const int ix = r % TX, iy = r / TX;  // cell y = iy-1
        const T q0 = q == 0 ? S.VY[iy - 1 + HALO][ix + HALO] : S.P[iy - 1 + HALO][ix + HALO];
        const Parab<T> P = parabola(q0, S.FY[q][iy][ix], S.FY[q][iy + 1][ix]);
        const T yr = iy <= TY ? S.CY[0][iy][ix] : T(0);
        const T yl = iy >= 1 ? S.CY[0][iy - 1][ix] : T(0);
        S.AY[q][0][iy][ix] = avg_right(P.R, P.D, P.S, yr);
        S.AY[q][1][iy][ix] = avg_left(P.L, P.D, P.S, yl);
      }
    __syncthreads();
    // phase D: face solutions at the cell's faces and the update (axes in order x, y, z)
    T dm[3] = {T(0), T(0), T(0)};
    T dpv = T(0), dv = T(0);
    if (ax) {
      T Vl, Pl, Vr, Pr;
      riemann_vp(S.AX[0][0][ty][tx], S.AX[0][1][ty][tx + 1], S.AX[1][0][ty][tx],
                 S.AX[1][1][ty][tx + 1], S.CX[1][ty][tx], Vl, Pl);
      riemann_vp(S.AX[0][0][ty][tx + 1], S.AX[0][1][ty][tx + 2], S.AX[1][0][ty][tx + 1],
                 S.AX[1][1][ty][tx + 2], S.CX[1][ty][tx + 1], Vr, Pr);
      dm[0] = th[0] * (Pr - Pl);
      dpv = th[0] * (Pr * Vr - Pl * Vl);
      dv = th[0] * (Vr - Vl);
    }
    if (ay) {
      T Vl, Pl, Vr, Pr;
      riemann_vp(S.AY[0][0][ty][tx], S.AY[0][1][ty + 1][tx], S.AY[1][0][ty][tx],
                 S.AY[1][1][ty + 1][tx], S.CY[1][ty][tx], Vl, Pl);
      riemann_vp(S.AY[0][0][ty + 1][tx], S.AY[0][1][ty + 2][tx], S.AY[1][0][ty + 1][tx],
                 S.AY[1][1][ty + 2][tx], S.CY[1][ty + 1][tx], Vr, Pr);
      dm[1] = th[1] * (Pr - Pl);
      dpv = dpv + th[1] * (Pr * Vr - Pl * Vl);
      dv = dv + th[1] * (Vr - Vl);
    }
    if (az) {
      dm[2] = dmz;
      dpv = dpv + dpvz;
      dv = dv + dvz;
    }
    if (own) {
      const long long c = (long long)gx + (long long)nx * gy + g.nxy * k;
      const T rho0 = A.u[0][c];
      T m[3] = {A.u[1][c] - dm[0], A.u[2][c] - dm[1], A.u[3][c] - dm[2]};
      T en = A.u[4][c] - dpv;
      const T ei0 = A.u[5][c];
      if (A.phi) {
        const T m0[3] = {A.u[1][c], A.u[2][c], A.u[3][c]};
#pragma unroll 1
        for (int a = 0; a < 3; a++) {
          if (g.n[a] == 1) continue;
          const int di = a == 0, dj = a == 1, dk = a == 2;
          const T pp = load_bc(A.phi, -1, gx + di, gy + dj, k + dk, g);
          const T pm = load_bc(A.phi, -1, gx - di, gy - dj, k - dk, g);
          const T grad = (pp - pm) / T(2.0 * A.h[a]);
          m[a] -= T(tau) * rho0 * grad;
          en -= T(tau) * m0[a] * grad;
        }
      }
      if (A.out[0]) A.out[0][c] = rho0;
      A.out[1][c] = m[0];
      A.out[2][c] = m[1];
      A.out[3][c] = m[2];
      A.out[4][c] = en;
      A.out[5][c] = ei0 - gm1 * ei0 * dv;
    }
    __syncthreads();
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
    cell_speeds<T>(u, gamma, gm1, vmax, cmax, nbad);
  }
  double sd[6];
  sums.get(sd);
  block_reduce_store<NT>(sd, (double)vmax, (double)cmax, 0ull, nbad, A.partials);
}

}  // namespace ppml
