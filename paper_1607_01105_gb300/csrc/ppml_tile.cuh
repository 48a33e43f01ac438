// Tiled line-sweep kernels of one PPML step (Kulikov & Vorobyov, arXiv:1607.01105).
//
// A CTA of 256 threads owns a 16^3 tile.  Thread t = a + 16 b owns one line per axis
// (x line (j, k) = (a, b); y line (i, k) = (a, b); z line (i, j) = (a, b)).  Each line is
// swept by a register pipeline (warm-up steps peeled, the steady steps a partly unrolled
// loop, its inputs loaded a step ahead): when position p arrives, the limited slope
// at p-1, the face value at p-3/2, the parabola of p-2 and the flux through the face
// p-5/2 are formed (Appendix Steps 1-3, characteristic averages), so every quantity along
// the line is computed once; the 3-cell halo costs 6 extra positions per 16 cells.
// Data is staged in shared memory (Lagrangian: one field box with a 3-cell cross-shaped
// halo; Eulerian: one slab per axis) with pitches that make every sweep's accesses
// bank-conflict free in FP32.  Boundaries are index maps on every load; tiles away from
// the domain faces take the unmapped fast path.  The unsplit sums over axes are taken in
// the order x, y, z.
#pragma once
#include <type_traits>

#include "../../include/ppml.h"
#include "ppml_common.cuh"

namespace ppml {

constexpr int TB = 16;           // tile edge
constexpr int TN = TB * TB;      // threads per CTA = lines per axis
constexpr int TH = 3;            // halo
constexpr int TW = TB + 2 * TH;  // 22 positions per line
// field box: (i, j, k) in [-3, 18]^3 (cross-shaped part used), pitches 23 and 528
constexpr int BRP = 23, BPP = 528, BOX = TW * BPP;
// accumulator over the tile: pitches 17 and 272
constexpr int ARP = 17, APP = 272, ACC = TB * APP;
// slab: position p in [-3, 18] times 256 transverse cells, pitch 257
constexpr int SLP = TN + 1, SLAB = TW * SLP;

__device__ __forceinline__ int box_at(int i, int j, int k) {
  return (i + TH) + BRP * (j + TH) + BPP * (k + TH);
}
__device__ __forceinline__ int acc_at(int i, int j, int k) { return i + ARP * j + APP * k; }

template <int V>
using IntC = std::integral_constant<int, V>;
template <bool V>
using BoolC = std::integral_constant<bool, V>;

struct TileGeom {
  int i0, j0, k0;
  int id;      // x-major index of the tile (its slot in the per-tile partials)
  bool valid;  // false for the padding blocks of a blocked order (no tile)
  bool fast;   // every cell within 3 of the tile is inside the domain on active axes
};

// Launch orders of the tiles (a systems choice, not the paper's: which tiles run
// concurrently, hence which halos the L2 holds).  Each tile computes the same values in any
// order, and the partials go to the tile's own slot.
//   0 x-major: x tile index fastest, then y, then z
//   1 z-major: z fastest, then y, then x
//   2, 3 blocked: blocks of 2^3 (4^3) tiles (fewer along axes with fewer tiles), x-major
//     within a block and over the blocks; blocks past the grid's edge are empty
constexpr int kTileOrders = 4;
static_assert(kTileOrders == PPML_TILE_ORDERS, "tile orders of the C ABI");

__host__ __device__ __forceinline__ int order_block(int order, int tiles) {
  const int s = order == 2 ? 2 : (order == 3 ? 4 : 1);
  return s < tiles ? s : tiles;
}

// Blocks launched for a tile grid in an order (the tile count, or more for padded blocks).
__host__ __device__ __forceinline__ long long order_blocks(int order, int tx, int ty, int tz) {
  const int sx = order_block(order, tx), sy = order_block(order, ty), sz = order_block(order, tz);
  return (long long)((tx + sx - 1) / sx * sx) * ((ty + sy - 1) / sy * sy) * ((tz + sz - 1) / sz * sz);
}

__device__ __forceinline__ TileGeom tile_geom(const GridGeom& g, const int tiles[3], int order) {
  TileGeom t;
  int b = blockIdx.x;
  int tc[3];
  if (order == 1) {
    tc[2] = b % tiles[2];
    b /= tiles[2];
    tc[1] = b % tiles[1];
    tc[0] = b / tiles[1];
  } else if (order >= 2) {
    int s[3], nsup[3];
    for (int a = 0; a < 3; a++) {
      s[a] = order_block(order, tiles[a]);
      nsup[a] = (tiles[a] + s[a] - 1) / s[a];
    }
    const int per = s[0] * s[1] * s[2];
    int sup = b / per, r = b % per;
    const int l0 = r % s[0];
    r /= s[0];
    const int l1 = r % s[1], l2 = r / s[1];
    const int S0 = sup % nsup[0];
    sup /= nsup[0];
    const int S1 = sup % nsup[1], S2 = sup / nsup[1];
    tc[0] = S0 * s[0] + l0;
    tc[1] = S1 * s[1] + l1;
    tc[2] = S2 * s[2] + l2;
  } else {
    tc[0] = b % tiles[0];
    b /= tiles[0];
    tc[1] = b % tiles[1];
    tc[2] = b / tiles[1];
  }
  t.valid = tc[0] < tiles[0] && tc[1] < tiles[1] && tc[2] < tiles[2];
  t.id = tc[0] + tiles[0] * (tc[1] + tiles[1] * tc[2]);
  t.i0 = tc[0] * TB;
  t.j0 = tc[1] * TB;
  t.k0 = tc[2] * TB;
  // fast: no cell within TH of the tile needs a map (halo faces hold their cells in the
  // arrays, at the same strides, so they count as inside)
  const int o[3] = {t.i0, t.j0, t.k0};
  bool f = true;
  for (int a = 0; a < 3; a++) {
    const bool lo_ok = o[a] - TH >= 0 || g.bc[2 * a] == 3;
    const bool hi_ok = o[a] + TB + TH <= g.n[a] || (g.bc[2 * a + 1] == 3 && o[a] + TB <= g.n[a]);
    f = f && g.n[a] > 1 && lo_ok && hi_ok;
  }
  t.fast = f;
  return t;
}

// Per-axis maps of the tile-relative coordinates -TH .. TB + TH - 1 to global offsets (the
// boundary-mapped coordinate times the axis stride, bc_map) and mirror flags (bit a for
// axis a), built once per CTA; a cell's offset is the sum of its three axis offsets and
// its flags the OR of the axis flags, which is map_cell without per-element arithmetic.
struct TileMaps {
  long long off[3][TW];
  int flip[3][TW];
  int inflow[3][TW];  // the inflow face whose ghost region the coordinate lies in, or -1
};

__device__ __forceinline__ void build_maps(TileMaps& M, const GridGeom& g, const TileGeom& t) {
  for (int e = threadIdx.x; e < 3 * TW; e += blockDim.x) {
    const int ax = e / TW, c = e % TW - TH;
    const int o = ax == 0 ? t.i0 : (ax == 1 ? t.j0 : t.k0);
    int fl;
    const int m = bc_map(o + c, g.n[ax], g.bc[2 * ax], g.bc[2 * ax + 1], fl);
    const long long stride = ax == 0 ? 1LL : (ax == 1 ? (long long)g.n[0] : g.nxy);
    M.off[ax][c + TH] = (long long)m * stride;
    M.flip[ax][c + TH] = fl << ax;
    // inflow ghosts only along active axes (an inactive axis has no ghost cells: its
    // coordinates are clamped onto the one cell)
    const int gc = o + c;
    const bool act = g.n[ax] > 1;
    M.inflow[ax][c + TH] = act && gc < 0 && g.bc[2 * ax] == PPML_BC_INFLOW
                               ? 2 * ax
                               : (act && gc >= g.n[ax] && g.bc[2 * ax + 1] == PPML_BC_INFLOW
                                      ? 2 * ax + 1
                                      : -1);
  }
}

// Whether the tile reads a ghost cell of an inflow face (uniform over the CTA).
__device__ __forceinline__ bool tile_inflow(const GridGeom& g, const TileGeom& t) {
  const int o[3] = {t.i0, t.j0, t.k0};
  bool r = false;
  for (int a = 0; a < 3; a++) {
    if (g.n[a] == 1) continue;
    r = r || (g.bc[2 * a] == PPML_BC_INFLOW && o[a] - TH < 0) ||
        (g.bc[2 * a + 1] == PPML_BC_INFLOW && o[a] + TB + TH > g.n[a]);
  }
  return r;
}

// The source of field f at tile-relative cell (i, j, k) whose mapped offset is off: an
// inflow face's prescribed value where the cell lies in that face's ghost region (the later
// axis deciding at edges and corners, as the ghost fill runs x, y, z), else the array.
template <typename T>
__device__ __forceinline__ const T* cell_src(const T* src, long long off, int f, const T* inflow,
                                             const TileMaps& M, bool tin, int i, int j, int k) {
  if (tin) {
    int face = M.inflow[2][k + TH];
    if (face < 0) face = M.inflow[1][j + TH];
    if (face < 0) face = M.inflow[0][i + TH];
    if (face >= 0) return inflow + 6 * face + f;
  }
  return src + off;
}

__device__ __forceinline__ long long map_off(const TileMaps& M, int i, int j, int k, int& fl) {
  fl = M.flip[0][i + TH] | M.flip[1][j + TH] | M.flip[2][k + TH];
  return M.off[0][i + TH] + M.off[1][j + TH] + M.off[2][k + TH];
}

// Field f at tile-relative cell (i, j, k) through the maps (momentum normal to a
// reflecting wall negated).
template <typename T>
__device__ __forceinline__ T load_mapped(const T* __restrict__ q, int f, const TileMaps& M, int i,
                                         int j, int k) {
  int fl;
  const T v = q[map_off(M, i, j, k, fl)];
  return field_flipped(f, fl) ? -v : v;
}

__device__ __forceinline__ bool in_domain(const GridGeom& g, const TileGeom& t, int i, int j,
                                          int k) {
  return t.i0 + i < g.n[0] && t.j0 + j < g.n[1] && t.k0 + k < g.n[2];
}

// Tile-relative coordinates of position p on the line (a, b) of axis ax.
__device__ __forceinline__ void line_cell(int ax, int p, int a, int b, int& i, int& j, int& k) {
  i = ax == 0 ? p : a;
  j = ax == 0 ? a : (ax == 1 ? p : b);
  k = ax == 2 ? p : b;
}

// ---------------------------------------------------------------- line pipelines

// The first-order variant's "parabola" of a cell: the constant cell value (Sec. 1.1).
template <typename T>
__device__ __forceinline__ Parab<T> flat_parabola(T q) {
  Parab<T> p;
  p.L = q;
  p.R = q;
  p.D = T(0);
  p.S = T(0);
  return p;
}

// Eulerian sweep along one line: v(p), pr(p), r(p) give v_a, p and rho at position p.
// emit(c, dm, dpv, dv) is called for cells c = 0..15 with dm = th (P+ - P-),
// dpv = th (P+V+ - P-V-), dv = th (V+ - V-).  hook(p) is called before step p = -1..18
// reads position p, and with p = 19 after the last step; positions below p - 3 are no
// longer read at that point (step p reads positions p, p - 2 and p - 3).
template <typename T, bool FLAT, typename VF, typename PF, typename RF, typename EF, typename HF>
__device__ __forceinline__ void sweep_eulerian(VF v, PF pr, RF r, T gamma, T th, double tau,
                                               double h, EF emit, HF hook) {
  T va = v(-3), vb = v(-2), pa = pr(-3), pb = pr(-2);
  T dva = T(0), fva = T(0), dpa = T(0), fpa = T(0);
  T vR = T(0), vD = T(0), vS = T(0), pR = T(0), pD = T(0), pS = T(0);
  T Vp = T(0), Pp = T(0);
  T rprev = T(0), pprev = T(0);  // rho, p of cell p-3
  T sprev = T(0);                // FP32: sqrt(rho) of cell p-3
  // step p; WARM: one of the first four steps (p constant), which skip the parts whose
  // inputs have not arrived; in FP32 the steady steps p = 3..18 run as a loop unrolled by
  // two (a smaller body for the instruction cache)
  auto step = [&](int p, auto warm_c) {
    constexpr bool W = decltype(warm_c)::value;
    hook(p);
    const T vn = v(p), pn = pr(p);
    const T dvn = limited_slope(va, vb, vn), dpn = limited_slope(pa, pb, pn);
    T fvn = T(0), fpn = T(0);
    if (!W || p >= 0) {
      fvn = face_value(va, vb, dva, dvn);
      fpn = face_value(pa, pb, dpa, dpn);
    }
    if (!W || p >= 1) {
      const Parab<T> Pv = FLAT ? flat_parabola(va) : parabola(va, fva, fvn);  // cell p-2
      const Parab<T> Pq = FLAT ? flat_parabola(pa) : parabola(pa, fpa, fpn);
      const T rc = r(p - 2);
      if constexpr (sizeof(T) == 4) {
        const float sc = sqrt_approx(rc);
        if (!W || p >= 2) {  // face between cells p-3 and p-2
          float lam, Z, hrz;
          face_constants_f32(rprev, rc, sprev, sc, pprev, pa, gamma, lam, Z, hrz);
          const float y = lam * th;
          const float vls = avg_right(vR, vD, vS, y), vrs = avg_left(Pv.L, Pv.D, Pv.S, y);
          const float pls = avg_right(pR, pD, pS, y), prs = avg_left(Pq.L, Pq.D, Pq.S, y);
          const float V = 0.5f * (vls + vrs) + (pls - prs) * hrz;
          const float P = 0.5f * (pls + prs) + 0.5f * Z * (vls - vrs);
          if (!W || p >= 3) emit(p - 3, th * (P - Pp), th * (P * V - Pp * Vp), th * (V - Vp));
          Vp = V;
          Pp = P;
        }
        sprev = sc;
      } else if (!W || p >= 2) {
        // face between cells p-3 and p-2
        T lam, Z;
        face_constants(rprev, rc, pprev, pa, gamma, lam, Z);
        const T y = Prec<T>::courant(lam, tau, h, th);
        T V, P;
        riemann_vp(avg_right(vR, vD, vS, y), avg_left(Pv.L, Pv.D, Pv.S, y),
                   avg_right(pR, pD, pS, y), avg_left(Pq.L, Pq.D, Pq.S, y), Z, V, P);
        if (!W || p >= 3) emit(p - 3, th * (P - Pp), th * (P * V - Pp * Vp), th * (V - Vp));
        Vp = V;
        Pp = P;
      }
      vR = Pv.R;
      vD = Pv.D;
      vS = Pv.S;
      pR = Pq.R;
      pD = Pq.D;
      pS = Pq.S;
      rprev = rc;
      pprev = pa;
    }
    va = vb;
    vb = vn;
    dva = dvn;
    fva = fvn;
    pa = pb;
    pb = pn;
    dpa = dpn;
    fpa = fpn;
  };
#pragma unroll
  for (int p = -1; p < 3; p++) step(p, BoolC<true>());
  if constexpr (sizeof(T) == 4) {
#pragma unroll 2
    for (int p = 3; p <= TB + 2; p++) step(p, BoolC<false>());
  } else {  // FP64 is bound by its FP64 pipe, not by instruction fetch: fully unrolled
#pragma unroll
    for (int p = 3; p <= TB + 2; p++) step(p, BoolC<false>());
  }
  hook(TB + 3);
}

// ===================================================================== Lagrangian stage

// Asynchronous global -> shared copies of one element (cp.async, completion awaited with
// cp.async.wait_all before the CTA barrier).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait until at most N committed groups of this thread are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Field storage of the Lagrangian tile: the 16^3 core (pitches 17, 272) and, per axis, the
// six halo positions -3..-1, 16..18 of every line (line-major, pitch 257).  Reused as a
// dense 18^3 box of v_a while the face velocities are formed.
constexpr int HALO_POS = 6;
constexpr int LAG_FIELD = ACC + 3 * HALO_POS * SLP;
static_assert(LAG_FIELD >= 18 * 18 * 18, "template box must fit in the field storage");

template <typename T>
struct LagTileSmem {
  T fld[LAG_FIELD];   // core (ACC) then halo[3][6][SLP]
  T acc[ACC];         // x + y part of the flux divergence
  T vh[3][TB + 1][TN];  // face velocities of every line, [axis][face][line]
};

__device__ __forceinline__ int halo_at(int ax, int h, int line) {
  return ACC + (ax * HALO_POS + h) * SLP + line;
}
__device__ __forceinline__ int tbox_at(int i, int j, int k) {  // dense 18^3, coords -1..16
  return (i + 1) + 18 * (j + 1) + 324 * (k + 1);
}

// One field over the dense 18^3 box (tile coordinates -1..16) of any tile, through the
// tile maps: asynchronous copies when async, else loads with the sign of component
// `flip_axis` of the momentum negated where that axis was mirrored (-1: no flip).
template <typename T>
__device__ __forceinline__ void stage_box_maps(T* box, const T* __restrict__ src,
                                               const TileMaps& M, int tid, int flip_axis,
                                               bool async, int field, const T* inflow,
                                               bool tin) {
  int i = tid % 18, j = (tid / 18) % 18, k = tid / 324;
  for (int it = tid; it < 18 * 18 * 18; it += TN) {
    int fl;
    const long long o = map_off(M, i - 1, j - 1, k - 1, fl);
    const T* p = tin ? cell_src(src, o, field, inflow, M, true, i - 1, j - 1, k - 1) : src + o;
    if (async) {
      cp_async_elem(&box[it], p);
    } else {
      const T v = *p;
      box[it] = (flip_axis >= 0 && ((fl >> flip_axis) & 1)) ? -v : v;
    }
    i += 4;
    if (i >= 18) {
      i -= 18;
      j++;
    }
    j += 14;
    if (j >= 18) {
      j -= 18;
      k++;
    }
  }
}

// Asynchronous copy of one field over the dense 18^3 box (tile coordinates -1..16) of an
// interior tile: thread tid copies elements tid, tid + 256, ...; the box coordinates and
// the global offset advance by 256 = 14 * 18 + 4 elements per copy with carries.
template <typename T>
__device__ __forceinline__ void stage_box_fast(T* box, const T* __restrict__ src,
                                               const GridGeom& g, const TileGeom& tg, int tid) {
  int i = tid % 18, j = (tid / 18) % 18;
  const long long nx = g.n[0];
  long long off = (long long)(tg.i0 - 1 + i) + nx * (tg.j0 - 1 + j) + g.nxy * (tg.k0 - 1 + tid / 324);
  for (int it = tid; it < 18 * 18 * 18; it += TN) {
    cp_async_elem(&box[it], src + off);
    i += 4;
    off += 4;
    if (i >= 18) {
      i -= 18;
      off += nx - 18;
      j++;
    }
    j += 14;
    off += 14 * nx;
    if (j >= 18) {
      j -= 18;
      off += g.nxy - 18 * nx;
    }
  }
}

// Face velocities as the sweeps read them.  FP64: v^ itself (the flux and the Courant
// number are formed as the checker forms them).  FP32: w = v^ th / 2 (th = tau / h), so
// that |w| is half the Courant number y and w times the upwind state is half of th times
// the flux (both exact rescalings of v^ th): the per-field products by th disappear, the
// sweeps accumulate half divergences and the update subtracts twice their sum.
__device__ __forceinline__ float vh_stored(float v, float th) { return v * (0.5f * th); }
__device__ __forceinline__ double vh_stored(double v, double) { return v; }
// The flux divergence summed over axes from what the sweeps accumulated (exact).
__device__ __forceinline__ float divergence_sum(float half_sum) { return 2.0f * half_sum; }
__device__ __forceinline__ double divergence_sum(double sum) { return sum; }

// FP32 flux through a face of eq. fluxonlagrangestage from w = v^ th / 2: w times the
// upwind state, the left cell's mean over its right fraction y when w >= 0, else the right
// cell's mean over its left fraction y, written as base + c1 D + c2 S with
// c1 = -+ y/2, c2 = (y/2)(1 - 2y/3) (the characteristic averages expanded).
__device__ __forceinline__ float half_flux_f32(float w, float R_l, float D_l, float S_l,
                                              float L_r, float D_r, float S_r) {
  const bool from_left = w >= 0.0f;
  const float hy = fabsf(w);
  const float c2 = hy * fmaf(-4.0f / 3.0f, hy, 1.0f);
  const float c1 = from_left ? -hy : hy;
  const float base = from_left ? R_l : L_r;
  const float D = from_left ? D_l : D_r;
  const float S = from_left ? S_l : S_r;
  return w * fmaf(c1, D, fmaf(c2, S, base));
}

// One line of the Lagrangian stage for any axis.  Field values: core[p cs] for p in
// [0, 16), halo[h SLP] for the positions -3..-1 (h = 0..2) and 16..18 (h = 3..5).  Face
// velocities vh[c TN], c = 0..16 (face between cells c-1 and c).  MODE 0: acc = div;
// 1: acc += div; 2: dst[c gs] = core - (acc + div) for c < nvalid (acc only if have_acc).
// The pipeline forms, when position p arrives, the slope at p-1, the face at p-3/2, the
// parabola of cell p-2 and the flux through face p-5/2; the warm-up positions -1..2 are
// peeled and the steady state is a loop unrolled by four.  DF (MODE 2): when dstlo is
// non-NULL the field is a double-float value whose low part srclo[c gs] is read and the
// update is added in double-float (dst the high part, dstlo the low part).  CS: the core
// stride of the sweep axis as a compile-time constant (immediate shared-memory offsets).
template <typename T, int MODE, bool FLAT, bool DF, int CS>
__device__ __forceinline__ void lag_line(const T* core, const T* halo, const T* vh, T th,
                                         double tau, double h, T* acc, bool have_acc,
                                         T* __restrict__ dst, long long gs, int nvalid,
                                         const T* __restrict__ srclo = nullptr,
                                         T* __restrict__ dstlo = nullptr) {
  constexpr int cs = CS;
  T qa = halo[0], qb = halo[SLP];  // q(p-2), q(p-1)
  T qn = halo[2 * SLP];            // p = -1
  T da = limited_slope(qa, qb, qn);
  qa = qb;
  qb = qn;
  qn = core[0];  // p = 0
  T dn = limited_slope(qa, qb, qn);
  T fa = face_value(qa, qb, da, dn);
  qa = qb;
  qb = qn;
  da = dn;
  qn = core[cs];  // p = 1
  dn = limited_slope(qa, qb, qn);
  T fn = face_value(qa, qb, da, dn);
  Parab<T> P = FLAT ? flat_parabola(qa) : parabola(qa, fa, fn);  // cell -1
  T PR = P.R, PD = P.D, PS = P.S;
  qa = qb;
  qb = qn;
  da = dn;
  fa = fn;
  qn = core[2 * cs];  // p = 2
  dn = limited_slope(qa, qb, qn);
  fn = face_value(qa, qb, da, dn);
  P = FLAT ? flat_parabola(qa) : parabola(qa, fa, fn);  // cell 0
  T Fp;
  if constexpr (sizeof(T) == 4) {
    Fp = half_flux_f32(vh[0], PR, PD, PS, P.L, P.D, P.S);
  } else {
    const T v = vh[0];
    const T y = Prec<T>::courant(tabs(v), tau, h, th);
    Fp = v * upwind_state(v >= T(0), PR, PD, PS, P.L, P.D, P.S, y);
  }
  PR = P.R;
  PD = P.D;
  PS = P.S;
  T qc = qa;  // q(c) for c = 0: cell c's value, the base of its update (MODE 2)
  qa = qb;
  qb = qn;
  da = dn;
  fa = fn;
  // steady state: p = 3..18 emits cell c = p-3
  auto step = [&](T qnew, T vv, int c) {
    const T dnn = limited_slope(qa, qb, qnew);
    const T fnn = face_value(qa, qb, da, dnn);
    const Parab<T> Pn = FLAT ? flat_parabola(qa) : parabola(qa, fa, fnn);  // cell c+1
    T F, d;  // through the face between cells c and c+1
    if constexpr (sizeof(T) == 4) {
      F = half_flux_f32(vv, PR, PD, PS, Pn.L, Pn.D, Pn.S);
      d = F - Fp;  // half of th (F+ - F-)
    } else {
      const T yy = Prec<T>::courant(tabs(vv), tau, h, th);
      F = vv * upwind_state(vv >= T(0), PR, PD, PS, Pn.L, Pn.D, Pn.S, yy);
      d = th * (F - Fp);
    }
    const int o = c * cs;
    if (MODE == 0) {
      acc[o] = d;
    } else if (MODE == 1) {
      acc[o] = acc[o] + d;
    } else if (c < nvalid) {
      const T upd = divergence_sum(have_acc ? acc[o] + d : d);
      if constexpr (DF) {
        if (dstlo) {
          float hi, lo;
          df_sub(qc, srclo[gs * c], upd, hi, lo);
          dst[gs * c] = hi;
          dstlo[gs * c] = lo;
        } else {
          dst[gs * c] = qc - upd;
        }
      } else {
        dst[gs * c] = qc - upd;
      }
    }
    qc = qa;
    Fp = F;
    PR = Pn.R;
    PD = Pn.D;
    PS = Pn.S;
    qa = qb;
    qb = qnew;
    da = dnn;
    fa = fnn;
  };
  // inputs one step ahead: position c + 3 and face c + 1 of step c are loaded in step c - 1
  T q_in = core[3 * cs], v_in = vh[TN];
#pragma unroll 4
  for (int c = 0; c < TB - 4; c++) {
    const T q = q_in, v = v_in;
    q_in = core[(c + 4) * cs];
    v_in = vh[(c + 2) * TN];
    step(q, v, c);
  }
#pragma unroll 1
  for (int c = TB - 4; c < TB - 1; c++) {
    const T q = q_in, v = v_in;
    q_in = halo[(c - TB + 7) * SLP];  // positions 16..18
    v_in = vh[(c + 2) * TN];          // faces 14..16
    step(q, v, c);
  }
  step(q_in, v_in, TB - 1);
}

// Face velocities v^ of line (a, b) along axis ax (faces 0..16, face c between cells c-1
// and c) from the dense 18^3 boxes of v_ax and rho: the 9-point template in the plane normal
// to ax (eq. veltemplate; the cell's own v in the one-point variant) and the sqrt(rho)
// weighted average of the two adjacent cells (eq. modspaceaveragevelocitylagrange).
template <typename T>
__device__ __forceinline__ void line_face_velocities(const T* vb, const T* rb, int ax, int a,
                                                     int b, bool one_point, T out[TB + 1]) {
  // transverse roles of eq. veltemplate: axis x -> (y, z), y -> (z, x), z -> (x, y)
  const int s_ax = ax == 0 ? 1 : (ax == 1 ? 18 : 324);
  const int s_b = ax == 0 ? 18 : (ax == 1 ? 324 : 1);
  const int s_c = ax == 0 ? 324 : (ax == 1 ? 1 : 18);
  int li, lj, lk;
  line_cell(ax, 0, a, b, li, lj, lk);
  const int base = tbox_at(li, lj, lk);
  T vt_prev = T(0), sq_prev = T(0);
#pragma unroll
  for (int p = -1; p <= TB; p++) {
    const int o = base + p * s_ax;
    const T corners = vb[o + s_b + s_c] + vb[o + s_b - s_c] + vb[o - s_b + s_c] + vb[o - s_b - s_c];
    const T edges = vb[o + s_b] + vb[o - s_b] + vb[o + s_c] + vb[o - s_c];
    const T vt = one_point ? vb[o] : corners / T(16) + edges / T(8) + vb[o] / T(4);
    T sq;
    if constexpr (sizeof(T) == 4) {
      sq = sqrt_approx(rb[o]);
      if (p >= 0) out[p] = (vt * sq + vt_prev * sq_prev) * rcp_approx(sq + sq_prev);
    } else {
      sq = sqrt(rb[o]);
      if (p >= 0) out[p] = (vt * sq + vt_prev * sq_prev) / (sq + sq_prev);
    }
    vt_prev = vt;
    sq_prev = sq;
  }
}

// DF: the state is double-float (A.ulo / A.outlo give the low parts of rho, m, rho E).
// INF: the grid has an inflow face (its ghost reads take the prescribed states; without
// one the kernel carries none of that code).
template <typename T, int MINB, bool DF, bool INF>
__global__ void __launch_bounds__(TN, MINB) lagrangian_tile(MarchArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LagTileSmem<T>& S = *reinterpret_cast<LagTileSmem<T>*>(smem_raw);
  const GridGeom& g = A.g;
  const bool act[3] = {g.n[0] > 1, g.n[1] > 1, g.n[2] > 1};
  const int tid = threadIdx.x, a = tid % TB, b = tid / TB;
  const int tiles[3] = {A.tiles_x, A.tiles_y, A.tiles_z};
  const TileGeom tg = tile_geom(g, tiles, A.tile_order);
  if (!tg.valid) return;  // a padding block of a blocked order (uniform over the CTA)
  const bool async_ok = !A.any_reflect;  // reflecting walls flip signs: copy through registers
  const bool fast_async = async_ok && tg.fast;
  const bool tin = INF && tile_inflow(g, tg);  // some copy of this tile reads an inflow ghost
  T* const smem_t = reinterpret_cast<T*>(smem_raw);  // fld and acc are contiguous
  T* const vspace = &S.vh[0][0][0];
  // template boxes: rho, then m_a (turned into v_a in place)
  T* rbox = smem_t;  // rho, dense 18^3
  auto vbox = [&](int ax) { return ax == 0 ? smem_t + 5832 : vspace + (ax - 1) * 5832; };
  // interior tiles issue the template copies first, so that they are in flight while the
  // per-CTA constants are formed
  if (fast_async) {
    stage_box_fast(rbox, A.u[0], g, tg, tid);
#pragma unroll 1
    for (int ax = 0; ax < 3; ax++)
      if (act[ax]) stage_box_fast(vbox(ax), A.u[1 + ax], g, tg, tid);
  }
  __shared__ TileMaps maps;
  if (!fast_async) build_maps(maps, g, tg);  // ordered by the barrier below
  double stc[4];
  cta_step_constants(A.dt_dev, A.dt_host, A.h, stc);
  const double tau = stc[0];
  const T th[3] = {T(stc[1]), T(stc[2]), T(stc[3])};
  const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);
  const bool first_order = (A.flags & PPML_FIRST_ORDER) != 0;
  const bool one_point = (A.flags & PPML_VHAT_1PT) != 0;
  const bool line_ok = in_domain(g, tg, a, b, 0);
  const int nvalid_z = line_ok ? min(TB, g.n[2] - tg.k0) : 0;
  const long long zline0 =
      (long long)(tg.i0 + a) + (long long)g.n[0] * (tg.j0 + b) + g.nxy * tg.k0;

  // ---- face velocities of every line (eqs. veltemplate, modspaceaveragevelocitylagrange)
  // rho and the three momenta over [-1, 16]^3 are staged at once -- rho and m_x in the
  // field + accumulator space, m_y and m_z in the face-velocity space, free until written --
  // and turned into velocities in place.  The y and z lines keep their face velocities in
  // registers until every thread has read the y and z boxes; then the x lines write theirs
  // and all three sets are stored.
  static_assert(2 * 5832 <= LAG_FIELD + ACC, "template boxes must fit in fld + acc");
  static_assert(2 * 5832 <= 3 * (TB + 1) * TN, "two boxes must fit in the face-velocity space");
  if (!fast_async) {
    // boundary tiles through the maps; rho never changes sign: always asynchronous
    stage_box_maps(rbox, A.u[0], maps, tid, -1, true, 0, A.inflow, tin);
#pragma unroll 1
    for (int ax = 0; ax < 3; ax++)
      if (act[ax])
        stage_box_maps(vbox(ax), A.u[1 + ax], maps, tid, ax, async_ok, 1 + ax, A.inflow, tin);
  }
  cp_async_wait_all();
  __syncthreads();
  for (int it = tid; it < 18 * 18 * 18; it += TN) {
    const T r = rbox[it];
    if constexpr (sizeof(T) == 4) {
      const float ir = rcp_approx(r);
#pragma unroll
      for (int ax = 0; ax < 3; ax++)
        if (act[ax]) vbox(ax)[it] = vbox(ax)[it] * ir;
    } else {
#pragma unroll
      for (int ax = 0; ax < 3; ax++)
        if (act[ax]) vbox(ax)[it] = vbox(ax)[it] / r;
    }
  }
  __syncthreads();
  T vh1[TB + 1], vh2[TB + 1];
  if (act[1]) line_face_velocities(vbox(1), rbox, 1, a, b, one_point, vh1);
  if (act[2]) line_face_velocities(vbox(2), rbox, 2, a, b, one_point, vh2);
  __syncthreads();  // the y and z boxes are read; the face-velocity space is free
  if (act[0]) {
    T vh0[TB + 1];
    line_face_velocities(vbox(0), rbox, 0, a, b, one_point, vh0);
#pragma unroll
    for (int q = 0; q <= TB; q++) S.vh[0][q][tid] = vh_stored(vh0[q], th[0]);
  }
#pragma unroll
  for (int q = 0; q <= TB; q++) {
    if (act[1]) S.vh[1][q][tid] = vh_stored(vh1[q], th[1]);
    if (act[2]) S.vh[2][q][tid] = vh_stored(vh2[q], th[2]);
  }
  __syncthreads();

  // ---- per field: stage, sweep x, y (into acc), z (finish into the output)
#pragma unroll 1
  for (int f = 0; f < 6; f++) {
    const T* __restrict__ src = A.u[f];
    if (fast_async) {
      // interior tile: thread (a, b) copies the z column (a, b, *) of the core and the six
      // halo positions of its x, y and z lines
      const T* col = src + zline0;
      T* dcore = &S.fld[acc_at(a, b, 0)];
#pragma unroll 4
      for (int s = 0; s < TB; s++) cp_async_elem(dcore + s * APP, col + g.nxy * s);
      const long long nx = g.n[0];
      const T* xl = src + (long long)tg.i0 + nx * (tg.j0 + a) + g.nxy * (tg.k0 + b);
      const T* yl = src + (long long)(tg.i0 + a) + nx * tg.j0 + g.nxy * (tg.k0 + b);
#pragma unroll
      for (int h = 0; h < HALO_POS; h++) {
        const int p = h < 3 ? h - 3 : TB + h - 3;
        if (act[0]) cp_async_elem(&S.fld[halo_at(0, h, tid)], xl + p);
      }
      cp_async_commit();
#pragma unroll
      for (int h = 0; h < HALO_POS; h++) {
        const int p = h < 3 ? h - 3 : TB + h - 3;
        if (act[1]) cp_async_elem(&S.fld[halo_at(1, h, tid)], yl + nx * p);
      }
      cp_async_commit();
#pragma unroll
      for (int h = 0; h < HALO_POS; h++) {
        const int p = h < 3 ? h - 3 : TB + h - 3;
        if (act[2]) cp_async_elem(&S.fld[halo_at(2, h, tid)], col + g.nxy * p);
      }
      cp_async_commit();
    } else if (async_ok) {
      // boundary tile, through the tile maps: the z column (a, b, *) of the core and the
      // halo positions of the thread's lines on active axes, in the same three commit
      // groups as on interior tiles.  The thread's line bases (the sum of the two
      // transverse map entries) are formed once, so each copy adds one map entry.
      const long long bx = maps.off[0][a + TH], by = maps.off[1][b + TH];
      const long long base_z = bx + by;  // z line (a, b): x = a, y = b
      if (tin) {
#pragma unroll 4
        for (int s = 0; s < TB; s++)
          cp_async_elem(&S.fld[acc_at(a, b, s)],
                        cell_src(src, base_z + maps.off[2][s + TH], f, A.inflow, maps, true, a, b, s));
      } else {
#pragma unroll 4
        for (int s = 0; s < TB; s++)
          cp_async_elem(&S.fld[acc_at(a, b, s)], src + (base_z + maps.off[2][s + TH]));
      }
#pragma unroll 1
      for (int ax = 0; ax < 3; ax++) {
        if (act[ax]) {
          // line (a, b) of axis ax: x line (y = a, z = b), y line (x = a, z = b), z line
          const long long base = ax == 0 ? maps.off[1][a + TH] + maps.off[2][b + TH]
                                         : (ax == 1 ? bx + maps.off[2][b + TH] : base_z);
          if (tin) {
#pragma unroll
            for (int h = 0; h < HALO_POS; h++) {
              const int p = h < 3 ? h - 3 : TB + h - 3;
              int i, j, k;
              line_cell(ax, p, a, b, i, j, k);
              cp_async_elem(&S.fld[halo_at(ax, h, tid)],
                            cell_src(src, base + maps.off[ax][p + TH], f, A.inflow, maps, true, i, j, k));
            }
          } else {
#pragma unroll
            for (int h = 0; h < HALO_POS; h++) {
              const int p = h < 3 ? h - 3 : TB + h - 3;
              cp_async_elem(&S.fld[halo_at(ax, h, tid)], src + (base + maps.off[ax][p + TH]));
            }
          }
        }
        cp_async_commit();  // same three groups as on interior tiles
      }
    } else {
      // reflecting walls somewhere: copies through registers with the mirror signs
#pragma unroll 4
      for (int s = 0; s < TB; s++) S.fld[acc_at(a, b, s)] = load_mapped(src, f, maps, a, b, s);
#pragma unroll 1
      for (int ax = 0; ax < 3; ax++) {
        if (!act[ax]) continue;
#pragma unroll
        for (int h = 0; h < HALO_POS; h++) {
          const int p = h < 3 ? h - 3 : TB + h - 3;
          int i, j, k;
          line_cell(ax, p, a, b, i, j, k);
          S.fld[halo_at(ax, h, tid)] = load_mapped(src, f, maps, i, j, k);
        }
      }
    }
    // three commit groups when asynchronous: core + x halo, y halo, z halo; each sweep
    // waits only for the group it reads, so the later copies overlap the earlier sweeps.
    // Every thread stages its own core column and halo rows, and the halo rows are read
    // by their owner alone: the halo waits need no barrier, and the barrier below (which
    // publishes the core) also orders this field's acc writes after the previous field's
    // z sweep, so no barrier ends a field.
    if (async_ok) cp_async_wait_group<2>();
    __syncthreads();
    int mode = 0;
#pragma unroll 1
    for (int ax = 0; ax < 3; ax++) {
      if (!act[ax]) continue;
      if (async_ok && ax == 1) cp_async_wait_group<1>();  // the thread's own y halo
      if (async_ok && ax == 2) cp_async_wait_group<0>();  // and z halo
      int li, lj, lk;
      line_cell(ax, 0, a, b, li, lj, lk);
      const int cb = acc_at(li, lj, lk);
      const T* halo = &S.fld[halo_at(ax, 0, tid)];
      const T* vhl = &S.vh[ax][0][tid];
      const T* srclo = DF && f < 5 ? A.ulo[f] + zline0 : nullptr;
      T* dstlo = DF && f < 5 ? A.outlo[f] + zline0 : nullptr;
      const T* core = &S.fld[cb];
      T* acc = &S.acc[cb];
      // one instantiation per (axis, mode): x is always the first sweep (mode 0), y the
      // first or the second, z the last (MODE 2: finish into the output)
      auto sweep = [&](auto mode_c, auto flat_c, auto cs_c) {
        constexpr int M = decltype(mode_c)::value;
        constexpr bool FL = decltype(flat_c)::value;
        constexpr int C = decltype(cs_c)::value;
        if constexpr (M == 2)
          lag_line<T, 2, FL, DF, C>(core, halo, vhl, th[2], tau, A.h[2], acc, mode == 1,
                                    A.out[f] + zline0, g.nxy, nvalid_z, srclo, dstlo);
        else
          lag_line<T, M, FL, false, C>(core, halo, vhl, th[ax], tau, A.h[ax], acc, false,
                                       nullptr, 0, 0);
      };
      auto sweep_ax = [&](auto flat_c) {
        if (ax == 2)
          sweep(IntC<2>(), flat_c, IntC<APP>());
        else if (ax == 1 && mode == 1)
          sweep(IntC<1>(), flat_c, IntC<ARP>());
        else if (ax == 1)
          sweep(IntC<0>(), flat_c, IntC<ARP>());
        else
          sweep(IntC<0>(), flat_c, IntC<1>());
      };
      if (first_order)
        sweep_ax(BoolC<true>());
      else
        sweep_ax(BoolC<false>());
      mode = 1;
      if (ax < 2) __syncthreads();
    }
    if (!act[2]) {  // no z sweep: finish from the x/y part
      for (int c = 0; c < nvalid_z; c++) {
        const int o = acc_at(a, b, c);
        const long long idx = zline0 + g.nxy * c;
        const T upd = mode == 1 ? divergence_sum(S.acc[o]) : T(0);
        if constexpr (DF) {
          if (f < 5) {
            float hi, lo;
            df_sub(S.fld[o], A.ulo[f][idx], upd, hi, lo);
            A.out[f][idx] = hi;
            A.outlo[f][idx] = lo;
            continue;
          }
        }
        A.out[f][idx] = S.fld[o] - upd;
      }
    }
  }

  // ---- energy correction (Sec. 1.4), CFL maxima and sums of the thread's z line
  FieldSums<T> sums;
  sums.init();
  T vmax = T(0), cmax = T(0);
  unsigned long long nvac = 0, nbad = 0;
  const float rho_vac_up = __double2float_ru(A.rho_vac);
  // groups of FB cells: all loads of a group are issued before its first store.  The
  // correction changes m only in vacuum cells, so only those store m back.
  constexpr int FB = 4;
#pragma unroll 1
  for (int c0 = 0; c0 < nvalid_z; c0 += FB) {
    T u[FB][6];
    T ul[FB][5];  // low parts (double-float states)
#pragma unroll
    for (int q = 0; q < FB; q++) {
      const long long idx = zline0 + g.nxy * (c0 + q);
      const bool ok = c0 + q < nvalid_z;
#pragma unroll
      for (int f = 0; f < 6; f++) u[q][f] = ok ? A.out[f][idx] : T(1);
#pragma unroll
      for (int f = 0; f < 5; f++) ul[q][f] = DF && ok ? A.outlo[f][idx] : T(0);
    }
    bool vac[FB];
    if constexpr (sizeof(T) == 4) {
      // the dense branch for every cell of the group without control flow (so that the
      // cells' chains interleave), then the rare vacuum cells on their stored values
      bool any_vac = false;
#pragma unroll
      for (int q = 0; q < FB; q++) {
        vac[q] = c0 + q < nvalid_z && vacuum_cell_f32(u[q], rho_vac_up);
        any_vac |= vac[q];
        const float e = DF ? dense_eps_df(u[q], ul[q]) : dense_eps_f32(u[q]);
        u[q][5] = vac[q] ? u[q][5] : e;
      }
      if (any_vac) {
#pragma unroll
        for (int q = 0; q < FB; q++)
          if (vac[q]) {
            if constexpr (DF)
              vacuum_correct_df(u[q], ul[q], A.rho_vac);
            else
              vacuum_correct_f32(u[q], A.rho_vac);
            nvac++;
          }
      }
    } else {
#pragma unroll
      for (int q = 0; q < FB; q++) {
        vac[q] = false;
        if (c0 + q < nvalid_z) {
          vac[q] = correct_energy<T>(u[q], A.rho_vac) != 0;
          nvac += vac[q];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < FB; q++) {
      if (c0 + q >= nvalid_z) break;
      const long long idx = zline0 + g.nxy * (c0 + q);
      if (vac[q]) {
#pragma unroll
        for (int f = 1; f <= 3; f++) {
          A.out[f][idx] = u[q][f];
          if constexpr (DF) A.outlo[f][idx] = ul[q][f];
        }
      }
      A.out[5][idx] = u[q][5];
      sums.add(u[q]);
      if constexpr (DF) sums.add_lo(ul[q]);
      if constexpr (sizeof(T) == 4)
        cell_speeds_f32(u[q], gamma, gm1, vmax, cmax, nbad);
      else
        cell_speeds<T>(u[q], gamma, gm1, vmax, cmax, nbad);
    }
  }
  if constexpr (sizeof(T) == 4) {
    float hi[6], lo[6];
#pragma unroll
    for (int f = 0; f < 6; f++) {
      hi[f] = sums.s[f].hi;
      lo[f] = sums.s[f].lo;
    }
    block_reduce_store_f32<TN>(hi, lo, vmax, cmax, (unsigned)nvac, (unsigned)nbad, A.partials,
                               tg.id);
  } else {
    double sd[6];
    sums.get(sd);
    block_reduce_store<TN>(sd, (double)vmax, (double)cmax, nvac, nbad, A.partials, tg.id);
  }
}

// ====================================================================== Eulerian stage

// eq. SCHintenEulerian: rho eps - (gamma - 1) rho eps th (V+ - V-), one rounding order for
// every code path (FP32: one FMA; FP64: as written, the checker's order).
__device__ __forceinline__ float eps_update(float ei, float gm1, float dv) {
  return fmaf(-(gm1 * ei), dv, ei);
}
__device__ __forceinline__ double eps_update(double ei, double gm1, double dv) {
  return ei - gm1 * ei * dv;
}

template <typename T>
struct EulTileSmem {
  T r[SLAB];   // rho along the sweep axis
  T m[SLAB];   // m_a along the sweep axis
  T p[SLAB];   // rho eps along the sweep axis (p = (gamma - 1) rho eps when read)
  T apv[ACC];  // sum over axes of th (PV+ - PV-)
  T av[ACC];   // sum over axes of th (V+ - V-)
};

__device__ __forceinline__ int slab_at(int p, int a, int b) { return (p + TH) * SLP + a + TB * b; }

// DF: the state is double-float (A.ulo / A.outlo give the low parts of rho, m, rho E); the
// momentum and total-energy updates are added in double-float.
template <typename T, int MINB, bool DF, bool INF>
__global__ void __launch_bounds__(TN, MINB) eulerian_tile(MarchArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EulTileSmem<T>& S = *reinterpret_cast<EulTileSmem<T>*>(smem_raw);
  const GridGeom& g = A.g;
  const bool act[3] = {g.n[0] > 1, g.n[1] > 1, g.n[2] > 1};
  const int tid = threadIdx.x, a = tid % TB, b = tid / TB;
  const int tiles[3] = {A.tiles_x, A.tiles_y, A.tiles_z};
  const TileGeom tg = tile_geom(g, tiles, A.tile_order);
  if (!tg.valid) return;  // a padding block of a blocked order (uniform over the CTA)
  const bool async_ok = !A.any_reflect;  // reflecting walls flip signs: copy through registers
  const bool tin = INF && tile_inflow(g, tg);  // some copy of this tile reads an inflow ghost
  __shared__ TileMaps maps;
  build_maps(maps, g, tg);  // ordered by the barrier below
  double stc[4];
  cta_step_constants(A.dt_dev, A.dt_host, A.h, stc);
  const double tau = stc[0];
  const T th[3] = {T(stc[1]), T(stc[2]), T(stc[3])};
  const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);

  const long long zline0e =
      (long long)(tg.i0 + a) + (long long)g.n[0] * (tg.j0 + b) + g.nxy * tg.k0;
  bool first = true;
  // With asynchronous copies a sweep fetches the next active axis's slab entries of its own
  // line into the slots it no longer reads (every line's entries are read by its owner
  // alone): positions -3..5, 6..11 and 12..18 in three commit groups, awaited before the
  // next sweep, before its step 6 and before its step 12.
  bool staged = false;  // this axis's entries were fetched during the previous sweep
#pragma unroll 1
  for (int ax = 0; ax < 3; ax++) {
    if (!act[ax]) continue;
    // stage rho, m_ax, rho eps along the axis: position p in [-3, 18], transverse
    // (s % 16, s / 16); on interior tiles the y and z lines are copied by their owners
    // (lanes consecutive in x), the x slab walks x fastest
    if (staged) {
      cp_async_wait_group<2>();
    } else if (async_ok && tg.fast && ax > 0) {
      int li, lj, lk;
      line_cell(ax, 0, a, b, li, lj, lk);
      const long long lb =
          (long long)(tg.i0 + li) + (long long)g.n[0] * (tg.j0 + lj) + g.nxy * (tg.k0 + lk);
      const long long st = ax == 0 ? 1 : (ax == 1 ? (long long)g.n[0] : g.nxy);
      const T* rl = A.u[0] + lb;
      const T* ml = A.u[1 + ax] + lb;
      const T* el = A.u[5] + lb;
#pragma unroll 2
      for (int p = -TH; p < TB + TH; p++) {
        const int o = slab_at(p, a, b);
        cp_async_elem(&S.r[o], rl + st * p);
        cp_async_elem(&S.m[o], ml + st * p);
        cp_async_elem(&S.p[o], el + st * p);
      }
    } else
    for (int it = tid; it < TW * TN; it += TN) {
      int p, s;
      if (ax == 0) {  // x fastest in memory: walk p fastest
        p = it % TW - TH;
        s = it / TW;
      } else {
        s = it % TN;
        p = it / TN - TH;
      }
      int i, j, k;
      line_cell(ax, p, s % TB, s / TB, i, j, k);
      int fl;
      const long long c = map_off(maps, i, j, k, fl);
      const int o = slab_at(p, s % TB, s / TB);
      if (async_ok && tin) {
        cp_async_elem(&S.r[o], cell_src(A.u[0], c, 0, A.inflow, maps, true, i, j, k));
        cp_async_elem(&S.m[o], cell_src(A.u[1 + ax], c, 1 + ax, A.inflow, maps, true, i, j, k));
        cp_async_elem(&S.p[o], cell_src(A.u[5], c, 5, A.inflow, maps, true, i, j, k));
      } else if (async_ok) {
        cp_async_elem(&S.r[o], A.u[0] + c);
        cp_async_elem(&S.m[o], A.u[1 + ax] + c);
        cp_async_elem(&S.p[o], A.u[5] + c);
      } else {
        T m = A.u[1 + ax][c];
        if ((fl >> ax) & 1) m = -m;
        S.r[o] = A.u[0][c];
        S.m[o] = m;
        S.p[o] = A.u[5][c];
      }
    }
    if (async_ok && !staged) cp_async_wait_all();
    __syncthreads();
    // the next active axis, fetched during this sweep
    int nax = -1;
    for (int q = 2; q > ax; q--)
      if (act[q]) nax = q;
    // (tiles that read an inflow face's ghosts stage every axis at its start instead)
    const bool pf = async_ok && nax >= 0 && !tin;
    long long nbase = 0, nst = 0;
    if (pf) {
      int ni, nj, nk;
      line_cell(nax, 0, a, b, ni, nj, nk);
      if (tg.fast) {
        nbase = (long long)(tg.i0 + ni) + (long long)g.n[0] * (tg.j0 + nj) + g.nxy * (tg.k0 + nk);
        nst = nax == 1 ? (long long)g.n[0] : g.nxy;
      } else {  // the two transverse map entries of the line
        nbase = (nax == 0 ? 0 : maps.off[0][ni + TH]) + (nax == 1 ? 0 : maps.off[1][nj + TH]) +
                (nax == 2 ? 0 : maps.off[2][nk + TH]);
      }
    }
    auto fetch = [&](int q) {  // position q of the thread's line along nax
      const long long go = tg.fast ? nbase + nst * q : nbase + maps.off[nax][q + TH];
      const int o = slab_at(q, a, b);
      cp_async_elem(&S.r[o], A.u[0] + go);
      cp_async_elem(&S.m[o], A.u[1 + nax] + go);
      cp_async_elem(&S.p[o], A.u[5] + go);
    };
    const bool was_staged = staged;
    auto hook = [&](int p) {
      if (was_staged) {
        if (p == 6) cp_async_wait_group<1>();
        if (p == 12) {
          if (pf)
            cp_async_wait_group<1>();
          else
            cp_async_wait_group<0>();
        }
      }
      if (pf) {
        if (p >= 1 && p <= TB + 2) fetch(p - 4);
        if (p == 9 || p == 15) cp_async_commit();
        if (p == TB + 3) {
#pragma unroll
          for (int q = TB - 1; q < TB + TH; q++) fetch(q);
          cp_async_commit();
        }
      }
    };
    staged = pf;
    // the thread's line along ax: accumulator base and stride, global offset and stride,
    // and the number of its cells inside the domain, formed once per axis
    int li, lj, lk;
    line_cell(ax, 0, a, b, li, lj, lk);
    const int acc0 = acc_at(li, lj, lk);
    const int acs = ax == 0 ? 1 : (ax == 1 ? ARP : APP);
    const long long gst = ax == 0 ? 1 : (ax == 1 ? (long long)g.n[0] : g.nxy);
    const long long gbase =
        (long long)(tg.i0 + li) + (long long)g.n[0] * (tg.j0 + lj) + g.nxy * (tg.k0 + lk);
    const int lo_ax = ax == 0 ? tg.i0 : (ax == 1 ? tg.j0 : tg.k0);
    const int nvalid = in_domain(g, tg, li, lj, lk) ? min(TB, g.n[ax] - lo_ax) : 0;
    T* const om = A.out[1 + ax] + gbase;
    auto emit = [&](int c, T dm, T dpv, T dv) {
      const int ai = acc0 + c * acs;
      S.apv[ai] = first ? dpv : S.apv[ai] + dpv;
      S.av[ai] = first ? dv : S.av[ai] + dv;
      if (c < nvalid) {
        const long long off = gst * c;
        if constexpr (DF) {
          float hi, lo;
          df_sub(S.m[slab_at(c, a, b)], A.ulo[1 + ax][gbase + off], dm, hi, lo);
          om[off] = hi;
          A.outlo[1 + ax][gbase + off] = lo;
        } else {
          om[off] = S.m[slab_at(c, a, b)] - dm;
        }
      }
    };
    auto vq = [&](int p) {
      const int o = slab_at(p, a, b);
      if constexpr (sizeof(T) == 4)
        return S.m[o] * rcp_approx(S.r[o]);
      else
        return S.m[o] / S.r[o];
    };
    auto pq = [&](int p) { return gm1 * S.p[slab_at(p, a, b)]; };
    auto rq = [&](int p) { return S.r[slab_at(p, a, b)]; };
    if (A.flags & PPML_FIRST_ORDER)
      sweep_eulerian<T, true>(vq, pq, rq, gamma, th[ax], tau, A.h[ax], emit, hook);
    else
      sweep_eulerian<T, false>(vq, pq, rq, gamma, th[ax], tau, A.h[ax], emit, hook);
    first = false;
    __syncthreads();
  }
  // momentum of inactive axes is unchanged
#pragma unroll 1
  for (int ax = 0; ax < 3; ax++) {
    if (act[ax]) continue;
    for (int c = 0; c < TB; c++) {
      if (!in_domain(g, tg, a, b, c)) continue;
      const long long idx = (long long)(tg.i0 + a) + (long long)g.n[0] * (tg.j0 + b) + g.nxy * (tg.k0 + c);
      A.out[1 + ax][idx] = A.u[1 + ax][idx];
      if constexpr (DF) A.outlo[1 + ax][idx] = A.ulo[1 + ax][idx];
    }
  }
  __syncthreads();
  // rho E, rho eps (and the optional gravity source), cells of the thread's z line
  if (tg.fast && !A.phi && !A.out[0]) {  // interior tile: loads of 8 cells in flight
    constexpr int EB = 8;
#pragma unroll 1
    for (int c0 = 0; c0 < TB; c0 += EB) {
      T en[EB], ei[EB], el[EB];
#pragma unroll
      for (int q = 0; q < EB; q++) {
        const long long idx = zline0e + g.nxy * (c0 + q);
        en[q] = A.u[4][idx];
        ei[q] = A.u[5][idx];
        if constexpr (DF) el[q] = A.ulo[4][idx];
      }
#pragma unroll
      for (int q = 0; q < EB; q++) {
        const long long idx = zline0e + g.nxy * (c0 + q);
        const int ai = acc_at(a, b, c0 + q);
        if constexpr (DF) {
          float hi, lo;
          df_sub(en[q], el[q], S.apv[ai], hi, lo);
          A.out[4][idx] = hi;
          A.outlo[4][idx] = lo;
        } else {
          A.out[4][idx] = en[q] - S.apv[ai];
        }
        A.out[5][idx] = eps_update(ei[q], gm1, S.av[ai]);
      }
    }
    return;
  }
  for (int c = 0; c < TB; c++) {
    if (!in_domain(g, tg, a, b, c)) continue;
    const int gi = tg.i0 + a, gj = tg.j0 + b, gk = tg.k0 + c;
    const long long idx = (long long)gi + (long long)g.n[0] * gj + g.nxy * gk;
    const T rho0 = A.u[0][idx];
    const T ei0 = A.u[5][idx];
    const T dpvs = first ? T(0) : S.apv[acc_at(a, b, c)];
    const T dvs = first ? T(0) : S.av[acc_at(a, b, c)];
    T en = A.u[4][idx] - dpvs;
    T den = dpvs;  // DF: the whole FP32 decrement of rho E, added to the pair once
    if (A.phi) {
      GridGeom gp = g;  // Phi: zero-gradient at reflecting walls and inflow faces, as at outflow
      for (int q = 0; q < 6; q++)
        if (gp.bc[q] == 2 || gp.bc[q] == 3 || gp.bc[q] == PPML_BC_INFLOW) gp.bc[q] = 0;
      T m[3] = {A.out[1][idx], A.out[2][idx], A.out[3][idx]};
      const T m0[3] = {A.u[1][idx], A.u[2][idx], A.u[3][idx]};
#pragma unroll 1
      for (int ax = 0; ax < 3; ax++) {
        if (!act[ax]) continue;
        const int di = ax == 0, dj = ax == 1, dk = ax == 2;
        const T pp = load_bc(A.phi, -1, gi + di, gj + dj, gk + dk, gp);
        const T pm = load_bc(A.phi, -1, gi - di, gj - dj, gk - dk, gp);
        const T grad = (pp - pm) / T(2.0 * A.h[ax]);
        if constexpr (DF) {
          float hi, lo;
          df_sub(m[ax], A.outlo[1 + ax][idx], T(tau) * rho0 * grad, hi, lo);
          m[ax] = hi;
          A.outlo[1 + ax][idx] = lo;
          den += T(tau) * m0[ax] * grad;
        } else {
          m[ax] -= T(tau) * rho0 * grad;
          en -= T(tau) * m0[ax] * grad;
        }
      }
      A.out[1][idx] = m[0];
      A.out[2][idx] = m[1];
      A.out[3][idx] = m[2];
    }
    if (A.out[0]) {
      A.out[0][idx] = rho0;
      if constexpr (DF) A.outlo[0][idx] = A.ulo[0][idx];
    }
    if constexpr (DF) {
      float hi, lo;
      df_sub(A.u[4][idx], A.ulo[4][idx], den, hi, lo);
      A.out[4][idx] = hi;
      A.outlo[4][idx] = lo;
    } else {
      A.out[4][idx] = en;
    }
    A.out[5][idx] = eps_update(ei0, gm1, dvs);
  }
}

}  // namespace ppml
