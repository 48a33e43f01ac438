/*
 * Plain FP64 CPU oracle of one PPML operator-splitting step (Kulikov & Vorobyov,
 * arXiv:1607.01105).  TEST INFRASTRUCTURE ONLY: the GPU library never links, calls
 * or includes this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark use it.
 *
 * It follows the paper's algorithm step by step, cell by cell, on ghost-padded
 * arrays, in the order the paper states it:
 *   S0  ghost fill of U^n (outflow / periodic / reflecting / inflow, axes in order x, y, z)
 *   S1  PPML parabolas of v_a and p                 (Appendix, Steps 1-3, eq. A1)
 *   S2  face Riemann solve with modified Roe averages and parabola averages
 *                                                   (Sec. "Low-dissipation hydrodynamic
 *                                                    solver at the Eulerian step",
 *                                                    eqs. lowriemannvelocity/-pressure)
 *   S3  Eulerian update of rho v, rho E, rho eps    (eqs. SCHdensEulerian..SCHintenEulerian),
 *       all three axes from U^n (unsplit)
 *   S4  ghost fill of U*
 *   S5  9-point transverse velocity template and Roe-weighted face velocity
 *                                                   (eqs. veltemplate,
 *                                                    modspaceaveragevelocitylagrange)
 *   S6  upwind parabola-average fluxes               (eq. fluxonlagrangestage)
 *   S7  unsplit Lagrangian update                    (Sec. "Hydrodynamic solver at the
 *                                                    Lagrangian step", Cartesian form)
 *   S8  total-energy consistency                     (Sec. "The conservation of total energy")
 *   S10 CFL time step                                (Sec. 1.1, CFL condition)
 *   S11 FP64 conservation sums
 * Readings of garbled or silent passages (kept identical in the GPU library, which
 * shares no code with this file):
 *   - Delta q = q^R - q^L (the Appendix prints q^L - q^R, which contradicts eq. A1 and
 *     the characteristic averages of the same Appendix);
 *   - rho_L, rho_R, p_L, p_R inside the Roe averages, lambda and the impedance are the
 *     adjacent cell values; only v and p carrying the (-+ lambda t) argument are
 *     parabola averages;
 *   - the Eulerian stage is unsplit (all axes from U^n), like the Lagrangian formula;
 *   - the monotonicity step tests "flat" first, then applies at most one overshoot fix;
 *   - energy correction: vacuum cells (rho < vacuum_frac * mean initial density) keep
 *     eps and the direction of v and rescale |v| = sqrt(2(E - eps)); |v| = 0 falls back
 *     to the dense formula; E - eps < 0 sets m = 0, eps = E.  Dense cells take
 *     rho eps = rho E - |m|^2/(2 rho) unless that is <= 0, in which case the advected
 *     rho eps is kept;
 *   - CFL: tau = CFL * min_a h_a / (max|v| + max c), the two maxima taken separately,
 *     |v| the Euclidean norm, axes with one cell excluded from min h_a;
 *   - boundaries: outflow = zero-gradient copy, periodic = wrap, reflecting = mirror
 *     with the normal momentum negated; edges and corners by filling x, then y, then z;
 *   - gravity (optional): cell-centred central difference of Phi, m -= tau rho grad Phi,
 *     rho E -= tau m . grad Phi, both from U^n.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (OpenMP only splits
 * independent cells/lines; reductions are serial in index order, so results do not
 * depend on the thread count).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NG 3           /* ghost layers per side */
#define NFIELD 6       /* rho, m_x, m_y, m_z, rho E, rho eps */
enum { F_RHO = 0, F_MX = 1, F_MY = 2, F_MZ = 3, F_EN = 4, F_EI = 5 };
enum { BC_OUTFLOW = 0, BC_PERIODIC = 1, BC_REFLECT = 2, BC_INFLOW = 4 };

typedef struct {
  int n[3];            /* interior cells per axis (x fastest in memory) */
  int bc[6];           /* -x, +x, -y, +y, -z, +z */
  double h[3];         /* cell size per axis */
  double gamma;        /* ratio of specific heats */
  double vacuum_frac;  /* vacuum threshold relative to rho_mean */
  double rho_mean;     /* mean initial density */
  int flags;           /* ORACLE_FIRST_ORDER: piecewise-constant states (Sec. 1.1);
                          ORACLE_VHAT_1PT: face velocity from the line only (no 9-point
                          template, the 1-point variant the paper compares against) */
  double inflow[6][NFIELD]; /* per face: the prescribed state of its ghost cells (rho,
                               m_x, m_y, m_z, rho E, rho eps), read where bc is BC_INFLOW */
} oracle_desc;
#define ORACLE_FIRST_ORDER 1
#define ORACLE_VHAT_1PT 2

typedef struct {
  double dt_cfl;       /* CFL step of the output state for the given cfl number */
  double vmax, cmax;   /* the two maxima entering the CFL step */
  double sums[6];      /* sum of each field over interior cells times the cell volume */
  long long n_vacuum;  /* cells that took the vacuum branch of the energy correction */
  long long n_keep_e;  /* dense cells whose corrected rho eps would be <= 0 */
  long long n_zero_m;  /* vacuum cells with rho E - rho eps < 0 (momentum set to zero) */
  long long n_nonphys; /* output cells with rho <= 0, rho eps <= 0 or non-finite values */
} oracle_diag;

/* ------------------------------------------------------------------ grid helpers */

typedef struct {
  int n[3], N[3];
  int g[3];     /* ghost layers per side: NG on axes with more than one cell, else 0 */
  size_t cells; /* N0*N1*N2 */
} gshape;

static gshape make_shape(const oracle_desc* d) {
  gshape s;
  s.cells = 1;
  for (int a = 0; a < 3; a++) {
    s.n[a] = d->n[a];
    s.g[a] = d->n[a] > 1 ? NG : 0; /* nothing reads ghosts along a single-cell axis */
    s.N[a] = d->n[a] + 2 * s.g[a];
    s.cells *= (size_t)s.N[a];
  }
  return s;
}

static size_t gidx(const gshape* s, int i, int j, int k) {
  return (size_t)i + (size_t)s->N[0] * ((size_t)j + (size_t)s->N[1] * (size_t)k);
}

static size_t axis_stride(const gshape* s, int a) {
  if (a == 0) return 1;
  if (a == 1) return (size_t)s->N[0];
  return (size_t)s->N[0] * (size_t)s->N[1];
}

/* copy interior-only field (n0*n1*n2, x fastest) into a ghost-padded array */
static void scatter_interior(const gshape* s, const double* src, double* dst) {
  for (int k = 0; k < s->n[2]; k++)
    for (int j = 0; j < s->n[1]; j++)
      for (int i = 0; i < s->n[0]; i++)
        dst[gidx(s, i + s->g[0], j + s->g[1], k + s->g[2])] =
            src[(size_t)i + (size_t)s->n[0] * ((size_t)j + (size_t)s->n[1] * (size_t)k)];
}

static void gather_interior(const gshape* s, const double* src, double* dst) {
  for (int k = 0; k < s->n[2]; k++)
    for (int j = 0; j < s->n[1]; j++)
      for (int i = 0; i < s->n[0]; i++)
        dst[(size_t)i + (size_t)s->n[0] * ((size_t)j + (size_t)s->n[1] * (size_t)k)] =
            src[gidx(s, i + s->g[0], j + s->g[1], k + s->g[2])];
}

/* Interior coordinate that a ghost coordinate c (c < 0 or c >= n) copies from, and the
 * sign applied to the momentum component normal to the boundary (reflecting walls). */
static int bc_source(int c, int n, int bc_lo, int bc_hi, int* flip) {
  *flip = 0;
  if (c >= 0 && c < n) return c;
  int bc = (c < 0) ? bc_lo : bc_hi;
  if (bc == BC_PERIODIC) return ((c % n) + n) % n;
  if (bc == BC_REFLECT) {
    *flip = 1;
    int r = (c < 0) ? (-1 - c) : (2 * n - 1 - c);
    if (r < 0) r = 0;
    if (r > n - 1) r = n - 1;
    return r;
  }
  return (c < 0) ? 0 : n - 1; /* outflow: zero-gradient copy */
}

/* S0 / S4: fill the NG ghost layers of one field, axes in order x, y, z; each axis pass
 * runs over the full padded extent of the other axes so edges and corners are filled.
 * An inflow face's ghost layers take its prescribed state (field >= 0; a potential,
 * field -1, is filled with the boundaries of its own descriptor).  At an edge or a corner
 * a later axis's pass overwrites an earlier one's ghosts. */
static void fill_ghosts(const gshape* s, const oracle_desc* d, double* q, int field) {
  for (int a = 0; a < 3; a++) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    size_t st = axis_stride(s, a);
    for (int ic = 0; ic < s->N[c]; ic++)
      for (int ib = 0; ib < s->N[b]; ib++) {
        int idx[3];
        idx[a] = 0; idx[b] = ib; idx[c] = ic;
        size_t base = gidx(s, idx[0], idx[1], idx[2]);
        for (int g = 0; g < s->g[a]; g++) {
          int ghosts[2] = {g - s->g[a], s->n[a] + g}; /* interior coords of a low and a high ghost */
          for (int side = 0; side < 2; side++) {
            const size_t dst = base + st * (size_t)(ghosts[side] + s->g[a]);
            if (d->bc[2 * a + side] == BC_INFLOW && field >= 0) {
              q[dst] = d->inflow[2 * a + side][field];
              continue;
            }
            int flip;
            int src = bc_source(ghosts[side], s->n[a], d->bc[2 * a], d->bc[2 * a + 1], &flip);
            double v = q[base + st * (size_t)(src + s->g[a])];
            if (flip && field == F_MX + a) v = -v;
            q[dst] = v;
          }
        }
      }
  }
}

/* The two axes transverse to a, ordered (inner, outer) by memory stride, so that threads
 * splitting the outer axis write disjoint planes or rows (no false sharing). */
static void transverse(int a, int* inner, int* outer) {
  int b = (a + 1) % 3, c = (a + 2) % 3;
  *inner = b < c ? b : c;
  *outer = b < c ? c : b;
}

/* ---------------------------------------------------------------- PPML parabolas */

/* Appendix, Step 1: limited slope delta_m q_i of a cell from its two neighbours. */
static double limited_slope(double qm, double q0, double qp) {
  double dq = 0.5 * (qp - qm);
  double r = qp - q0, l = q0 - qm;
  if (r * l > 0.0) {
    double m = fmin(fabs(dq), fmin(2.0 * fabs(r), 2.0 * fabs(l)));
    return (dq > 0.0) ? m : -m;
  }
  return 0.0;
}

/* Appendix, Steps 1-3, on one line q[0..N-1] (ghost-padded).  Outputs the parabola
 * (qL, qR, dq = qR - qL, q6) of every cell c in [2, N-3]; other entries are untouched.
 * work must hold N doubles for delta_m q and N for the face values. */
static void line_parabolas_ex(const double* q, int N, double* work, double* qL, double* qR,
                              double* dq, double* q6, int first_order);
static void line_parabolas(const double* q, int N, double* work, double* qL, double* qR,
                           double* dq, double* q6) {
  line_parabolas_ex(q, N, work, qL, qR, dq, q6, 0);
}

/* First-order variant (Sec. 1.1, piecewise-constant initial data of the face problems):
 * every cell's "parabola" is the constant cell value. */
static void line_flat(const double* q, int N, double* qL, double* qR, double* dq, double* q6) {
  for (int c = 2; c <= N - 3; c++) {
    qL[c] = q[c];
    qR[c] = q[c];
    dq[c] = 0.0;
    q6[c] = 0.0;
  }
}

static void line_parabolas_ex(const double* q, int N, double* work, double* qL, double* qR,
                              double* dq, double* q6, int first_order) {
  if (first_order) {
    line_flat(q, N, qL, qR, dq, q6);
    return;
  }
  double* dm = work;
  double* face = work + N; /* face[c] = q_{c+1/2} */
  for (int c = 1; c <= N - 2; c++) dm[c] = limited_slope(q[c - 1], q[c], q[c + 1]);
  for (int c = 1; c <= N - 3; c++)
    face[c] = 0.5 * (q[c] + q[c + 1]) - (dm[c + 1] - dm[c]) / 6.0;
  for (int c = 2; c <= N - 3; c++) {
    double L = face[c - 1], R = face[c], q0 = q[c];
    /* Step 2: a cell that is a local extremum becomes flat; otherwise remove overshoot */
    if ((L - q0) * (q0 - R) <= 0.0) {
      L = q0;
      R = q0;
    } else {
      double D = R - L;
      double S = 6.0 * (q0 - 0.5 * (L + R));
      if (D * S > D * D)
        L = 3.0 * q0 - 2.0 * R;
      else if (D * S < -(D * D))
        R = 3.0 * q0 - 2.0 * L;
    }
    /* Step 3 */
    qL[c] = L;
    qR[c] = R;
    dq[c] = R - L;
    q6[c] = 6.0 * (q0 - 0.5 * (L + R));
  }
}

/* Average of a cell's parabola over the right fraction y of the cell (the state left of
 * the cell's right face, q_L(-lambda t) with y = lambda t / h). */
static double avg_right_part(double qR, double dq, double q6, double y) {
  return qR - 0.5 * y * (dq - q6 * (1.0 - 2.0 * y / 3.0));
}

/* Average over the left fraction y of the cell (the state right of the cell's left face,
 * q_R(lambda t)). */
static double avg_left_part(double qL, double dq, double q6, double y) {
  return qL + 0.5 * y * (dq + q6 * (1.0 - 2.0 * y / 3.0));
}

/* S2: face solution (V, P) of the acoustic Riemann problem with modified Roe averages.
 * rl, rr, pl, pr are the adjacent cell values; vls, vrs, pls, prs the parabola averages
 * over the domains of dependence. */
static void face_riemann(double rl, double rr, double pl, double pr, double vls, double vrs,
                         double pls, double prs, double gamma, double* V, double* P) {
  double sl = sqrt(rl), sr = sqrt(rr);
  double A = rl * sl + rr * sr;    /* rho_L^{3/2} + rho_R^{3/2} */
  double B = pl * sl + pr * sr;    /* p_L sqrt(rho_L) + p_R sqrt(rho_R) */
  double S = sl + sr;
  double Z = sqrt(gamma * A * B / (S * S));
  *V = 0.5 * (vls + vrs) + (pls - prs) / (2.0 * Z);
  *P = 0.5 * (pls + prs) + 0.5 * Z * (vls - vrs);
}

/* lambda = sqrt(gamma p^ / rho^) of a face */
static double face_lambda(double rl, double rr, double pl, double pr, double gamma) {
  double sl = sqrt(rl), sr = sqrt(rr);
  return sqrt(gamma * (pl * sl + pr * sr) / (rl * sl + rr * sr));
}

/* ------------------------------------------------------------------ line buffers */

typedef struct {
  double *q, *q2, *r, *work, *L, *R, *D, *S, *L2, *R2, *D2, *S2, *Vf, *Pf, *Ff, *y;
} linebuf;

static void* xmalloc(size_t n) {
  void* p = malloc(n ? n : 1);
  return p;
}

static int lb_alloc(linebuf* b, int N) {
  size_t sz = (size_t)N * sizeof(double);
  double* blk = (double*)xmalloc(17 * sz);
  if (!blk) return -1;
  b->q = blk; b->q2 = blk + N; b->r = blk + 2 * N; b->work = blk + 3 * N;
  b->L = blk + 5 * N; b->R = blk + 6 * N; b->D = blk + 7 * N; b->S = blk + 8 * N;
  b->L2 = blk + 9 * N; b->R2 = blk + 10 * N; b->D2 = blk + 11 * N; b->S2 = blk + 12 * N;
  b->Vf = blk + 13 * N; b->Pf = blk + 14 * N; b->Ff = blk + 15 * N; b->y = blk + 16 * N;
  return 0;
}

static void lb_free(linebuf* b) { free(b->q); }

/* ---------------------------------------------------------------- Eulerian stage */

/* S1-S3 on ghost-filled U (padded); writes U* interior (padded layout, ghosts untouched).
 * phi (padded, ghost-filled) may be NULL. */
static int eulerian_stage(const gshape* s, const oracle_desc* d, double* const U[NFIELD],
                          double* const Us[NFIELD], const double* phi, double tau) {
  const double gm1 = d->gamma - 1.0;
  size_t nc = s->cells;
  double* vel[3];
  double* p = (double*)xmalloc(nc * sizeof(double));
  double* dmom[3];
  double* dPV = (double*)calloc(nc, sizeof(double));
  double* dV = (double*)calloc(nc, sizeof(double));
  for (int a = 0; a < 3; a++) {
    vel[a] = (double*)xmalloc(nc * sizeof(double));
    dmom[a] = (double*)calloc(nc, sizeof(double));
  }
  /* primitives on every padded cell */
  for (size_t c = 0; c < nc; c++) {
    for (int a = 0; a < 3; a++) vel[a][c] = U[F_MX + a][c] / U[F_RHO][c];
    p[c] = gm1 * U[F_EI][c];
  }
  for (int a = 0; a < 3; a++) {
    if (s->n[a] == 1) continue; /* a single cell along an axis gives exactly zero fluxes */
    int b, cax;
    transverse(a, &b, &cax);
    size_t st = axis_stride(s, a);
    int N = s->N[a];
    double rk = tau / d->h[a];
#pragma omp parallel
    {
      linebuf lb;
      lb_alloc(&lb, N);
#pragma omp for schedule(static)
      for (int ic = s->g[cax]; ic < s->g[cax] + s->n[cax]; ic++)
        for (int ib = s->g[b]; ib < s->g[b] + s->n[b]; ib++) {
          int idx[3];
          idx[a] = 0; idx[b] = ib; idx[cax] = ic;
          size_t base = gidx(s, idx[0], idx[1], idx[2]);
          for (int c = 0; c < N; c++) {
            lb.q[c] = vel[a][base + st * c];
            lb.q2[c] = p[base + st * c];
            lb.r[c] = U[F_RHO][base + st * c];
          }
          const int fo = d->flags & ORACLE_FIRST_ORDER;
          line_parabolas_ex(lb.q, N, lb.work, lb.L, lb.R, lb.D, lb.S, fo);
          line_parabolas_ex(lb.q2, N, lb.work, lb.L2, lb.R2, lb.D2, lb.S2, fo);
          /* faces c+1/2 for c in [NG-1, NG+n-1] */
          for (int c = NG - 1; c <= NG + s->n[a] - 1; c++) {
            double rl = lb.r[c], rr = lb.r[c + 1], pl = lb.q2[c], pr = lb.q2[c + 1];
            double lam = face_lambda(rl, rr, pl, pr, d->gamma);
            double y = lam * tau / d->h[a];
            double vls = avg_right_part(lb.R[c], lb.D[c], lb.S[c], y);
            double vrs = avg_left_part(lb.L[c + 1], lb.D[c + 1], lb.S[c + 1], y);
            double pls = avg_right_part(lb.R2[c], lb.D2[c], lb.S2[c], y);
            double prs = avg_left_part(lb.L2[c + 1], lb.D2[c + 1], lb.S2[c + 1], y);
            face_riemann(rl, rr, pl, pr, vls, vrs, pls, prs, d->gamma, &lb.Vf[c], &lb.Pf[c]);
          }
          for (int c = NG; c < NG + s->n[a]; c++) {
            size_t g = base + st * c;
            dmom[a][g] = rk * (lb.Pf[c] - lb.Pf[c - 1]);
            dPV[g] += rk * (lb.Pf[c] * lb.Vf[c] - lb.Pf[c - 1] * lb.Vf[c - 1]);
            dV[g] += rk * (lb.Vf[c] - lb.Vf[c - 1]);
          }
        }
      lb_free(&lb);
    }
  }
  /* S3 update of the interior */
#pragma omp parallel for schedule(static)
  for (int k = s->g[2]; k < s->g[2] + s->n[2]; k++)
    for (int j = s->g[1]; j < s->g[1] + s->n[1]; j++)
      for (int i = s->g[0]; i < s->g[0] + s->n[0]; i++) {
        size_t g = gidx(s, i, j, k);
        double rho = U[F_RHO][g];
        double m[3], en = U[F_EN][g] - dPV[g];
        for (int a = 0; a < 3; a++) m[a] = U[F_MX + a][g] - dmom[a][g];
        if (phi) {
          for (int a = 0; a < 3; a++) {
            if (s->n[a] == 1) continue;
            size_t st = axis_stride(s, a);
            double grad = (phi[g + st] - phi[g - st]) / (2.0 * d->h[a]);
            m[a] -= tau * rho * grad;
            en -= tau * U[F_MX + a][g] * grad;
          }
        }
        Us[F_RHO][g] = rho;
        for (int a = 0; a < 3; a++) Us[F_MX + a][g] = m[a];
        Us[F_EN][g] = en;
        Us[F_EI][g] = U[F_EI][g] - gm1 * U[F_EI][g] * dV[g];
      }
  free(p);
  free(dPV);
  free(dV);
  for (int a = 0; a < 3; a++) {
    free(vel[a]);
    free(dmom[a]);
  }
  return 0;
}

/* -------------------------------------------------------------- Lagrangian stage */

/* S5 along axis a on ghost-filled U* (padded): v_a = m_a / rho on every padded cell,
 * the 9-point template v tilde in the plane normal to a (eq. veltemplate: 1/16 at the
 * four corners, 1/8 at the four edge neighbours, 1/4 at the cell itself; the cell's own
 * v in the one-point variant) on every cell whose transverse neighbours exist (a
 * single-cell transverse axis uses the cell itself, which makes the template the 1D / 2D
 * marginal), and the sqrt(rho)-weighted face velocity v hat of eq.
 * modspaceaveragevelocitylagrange at faces c+1/2, c in [NG-1, NG+n-1], of every interior
 * line, stored at the index of the face's left cell. */
static void face_velocities(const gshape* s, const oracle_desc* d, double* const Us[NFIELD],
                            int a, double* vel, double* vt, double* vhat) {
  size_t nc = s->cells;
  int b = (a + 1) % 3, cax = (a + 2) % 3; /* template roles (eq. veltemplate) */
  int li, lo;                             /* loop order (memory strides) */
  transverse(a, &li, &lo);
  size_t st = axis_stride(s, a), sb = axis_stride(s, b), sc = axis_stride(s, cax);
  int N = s->N[a];
  for (size_t c = 0; c < nc; c++) vel[c] = Us[F_MX + a][c] / Us[F_RHO][c];
#pragma omp parallel for schedule(static)
  for (int io = 0; io < s->N[lo]; io++)
    for (int ii = 0; ii < s->N[li]; ii++) {
      int idx[3];
      idx[lo] = io; idx[li] = ii;
      int ib = idx[b], ic = idx[cax];
      int bm = (s->n[b] == 1) ? 0 : 1, cm = (s->n[cax] == 1) ? 0 : 1;
      if (ib - bm < 0 || ib + bm >= s->N[b] || ic - cm < 0 || ic + cm >= s->N[cax]) continue;
      for (int ia = 0; ia < N; ia++) {
        idx[a] = ia;
        size_t g = gidx(s, idx[0], idx[1], idx[2]);
        size_t db = sb * (size_t)bm, dc = sc * (size_t)cm;
        if (d->flags & ORACLE_VHAT_1PT) {
          vt[g] = vel[g];
          continue;
        }
        double corners = vel[g + db + dc] + vel[g + db - dc] + vel[g - db + dc] + vel[g - db - dc];
        double edges = vel[g + db] + vel[g - db] + vel[g + dc] + vel[g - dc];
        vt[g] = corners / 16.0 + edges / 8.0 + vel[g] / 4.0;
      }
    }
#pragma omp parallel for schedule(static)
  for (int io = s->g[lo]; io < s->g[lo] + s->n[lo]; io++)
    for (int ii = s->g[li]; ii < s->g[li] + s->n[li]; ii++) {
      int idx[3];
      idx[a] = 0; idx[lo] = io; idx[li] = ii;
      size_t base = gidx(s, idx[0], idx[1], idx[2]);
      for (int c = NG - 1; c <= NG + s->n[a] - 1; c++) {
        size_t gl = base + st * c, gr = gl + st;
        double sl = sqrt(Us[F_RHO][gl]), sr = sqrt(Us[F_RHO][gr]);
        vhat[gl] = (vt[gr] * sr + vt[gl] * sl) / (sr + sl);
      }
    }
}

/* S5-S7 on ghost-filled U* (padded); writes U^{n+1} into Un (padded, interior only). */
static int lagrangian_stage(const gshape* s, const oracle_desc* d, double* const Us[NFIELD],
                            double* const Un[NFIELD], double tau) {
  size_t nc = s->cells;
  double* vel = (double*)xmalloc(nc * sizeof(double));
  double* vt = (double*)xmalloc(nc * sizeof(double));   /* v tilde */
  double* vhat = (double*)xmalloc(nc * sizeof(double)); /* v hat at face c+1/2 along a */
  double* div[NFIELD];
  for (int f = 0; f < NFIELD; f++) div[f] = (double*)calloc(nc, sizeof(double));

  for (int a = 0; a < 3; a++) {
    if (s->n[a] == 1) continue;
    int li, lo; /* loop order (memory strides) */
    transverse(a, &li, &lo);
    size_t st = axis_stride(s, a);
    int N = s->N[a];
    double rk = tau / d->h[a];
    face_velocities(s, d, Us, a, vel, vt, vhat); /* S5 */
    /* S6: fluxes of every field; S7 accumulation */
#pragma omp parallel
    {
      linebuf lb;
      lb_alloc(&lb, N);
#pragma omp for schedule(static)
      for (int io = s->g[lo]; io < s->g[lo] + s->n[lo]; io++)
        for (int ii = s->g[li]; ii < s->g[li] + s->n[li]; ii++) {
          int idx[3];
          idx[a] = 0; idx[lo] = io; idx[li] = ii;
          size_t base = gidx(s, idx[0], idx[1], idx[2]);
          for (int f = 0; f < NFIELD; f++) {
            for (int c = 0; c < N; c++) lb.q[c] = Us[f][base + st * c];
            line_parabolas_ex(lb.q, N, lb.work, lb.L, lb.R, lb.D, lb.S,
                              d->flags & ORACLE_FIRST_ORDER);
            for (int c = NG - 1; c <= NG + s->n[a] - 1; c++) {
              double vh = vhat[base + st * c];
              double y = fabs(vh) * tau / d->h[a];
              double fs;
              if (vh >= 0.0)
                fs = avg_right_part(lb.R[c], lb.D[c], lb.S[c], y);
              else
                fs = avg_left_part(lb.L[c + 1], lb.D[c + 1], lb.S[c + 1], y);
              lb.Ff[c] = vh * fs;
            }
            for (int c = NG; c < NG + s->n[a]; c++)
              div[f][base + st * c] += rk * (lb.Ff[c] - lb.Ff[c - 1]);
          }
        }
      lb_free(&lb);
    }
  }
#pragma omp parallel for schedule(static)
  for (int k = s->g[2]; k < s->g[2] + s->n[2]; k++)
    for (int j = s->g[1]; j < s->g[1] + s->n[1]; j++)
      for (int i = s->g[0]; i < s->g[0] + s->n[0]; i++) {
        size_t g = gidx(s, i, j, k);
        for (int f = 0; f < NFIELD; f++) Un[f][g] = Us[f][g] - div[f][g];
      }
  free(vel);
  free(vt);
  free(vhat);
  for (int f = 0; f < NFIELD; f++) free(div[f]);
  return 0;
}

/* ---------------------------------------------------------- S8 energy correction */

/* One cell; u = {rho, mx, my, mz, rhoE, rhoeps}, modified in place.  Returns a code:
 * 0 dense, 1 vacuum, 2 dense with rho eps kept, 3 vacuum with momentum set to zero. */
static int energy_correction(double* u, double rho_vac) {
  double rho = u[F_RHO];
  double m2 = u[F_MX] * u[F_MX] + u[F_MY] * u[F_MY] + u[F_MZ] * u[F_MZ];
  if (rho < rho_vac && m2 > 0.0) {
    double de = u[F_EN] - u[F_EI];
    if (de < 0.0) {
      u[F_MX] = u[F_MY] = u[F_MZ] = 0.0;
      u[F_EI] = u[F_EN];
      return 3;
    }
    double vnew = sqrt(2.0 * de / rho);
    double vold = sqrt(m2) / rho;
    double scale = vnew / vold;
    u[F_MX] *= scale;
    u[F_MY] *= scale;
    u[F_MZ] *= scale;
    return 1;
  }
  double e = u[F_EN] - m2 / (2.0 * rho);
  if (e > 0.0) {
    u[F_EI] = e;
    return 0;
  }
  return 2;
}

/* ------------------------------------------------------------------ public API */

static void diag_of(const oracle_desc* d, double* const u[NFIELD], double cfl, oracle_diag* dg) {
  /* interior-only arrays; serial in index order */
  size_t n = (size_t)d->n[0] * d->n[1] * d->n[2];
  double vol = d->h[0] * d->h[1] * d->h[2];
  double vmax = 0.0, cmax = 0.0, sums[6] = {0, 0, 0, 0, 0, 0};
  long long bad = 0;
  for (size_t c = 0; c < n; c++) {
    double rho = u[F_RHO][c];
    double vx = u[F_MX][c] / rho, vy = u[F_MY][c] / rho, vz = u[F_MZ][c] / rho;
    double v = sqrt(vx * vx + vy * vy + vz * vz);
    double pr = (d->gamma - 1.0) * u[F_EI][c];
    double cs = sqrt(d->gamma * pr / rho);
    if (v > vmax) vmax = v;
    if (cs > cmax) cmax = cs;
    int ok = (rho > 0.0) && (u[F_EI][c] > 0.0);
    for (int f = 0; f < NFIELD; f++) {
      sums[f] += u[f][c];
      if (!isfinite(u[f][c])) ok = 0;
    }
    if (!ok) bad++;
  }
  double hmin = INFINITY;
  for (int a = 0; a < 3; a++)
    if (d->n[a] > 1 && d->h[a] < hmin) hmin = d->h[a];
  if (!isfinite(hmin)) hmin = d->h[0];
  dg->vmax = vmax;
  dg->cmax = cmax;
  dg->dt_cfl = cfl * hmin / (vmax + cmax);
  for (int f = 0; f < NFIELD; f++) dg->sums[f] = sums[f] * vol;
  dg->n_nonphys = bad;
}

/* S10 + S11 of a state given as six interior-only arrays. */
void oracle_diagnostics(const oracle_desc* d, double* const u[NFIELD], double cfl, oracle_diag* out) {
  memset(out, 0, sizeof(*out));
  diag_of(d, u, cfl, out);
}

/* Parabolas of one ghost-padded line (exposed for unit tests). */
void oracle_line_parabolas(const double* q, int N, double* qL, double* qR, double* dq, double* q6) {
  double* work = (double*)xmalloc(2 * (size_t)N * sizeof(double));
  line_parabolas(q, N, work, qL, qR, dq, q6);
  free(work);
}

double oracle_avg_right_part(double qR, double dq, double q6, double y) { return avg_right_part(qR, dq, q6, y); }
double oracle_avg_left_part(double qL, double dq, double q6, double y) { return avg_left_part(qL, dq, q6, y); }

void oracle_face_riemann(double rl, double rr, double pl, double pr, double vls, double vrs,
                         double pls, double prs, double gamma, double* V, double* P) {
  face_riemann(rl, rr, pl, pr, vls, vrs, pls, prs, gamma, V, P);
}

double oracle_face_lambda(double rl, double rr, double pl, double pr, double gamma) {
  return face_lambda(rl, rr, pl, pr, gamma);
}

int oracle_energy_correction(double* u6, double rho_vac) { return energy_correction(u6, rho_vac); }

/* S5 alone: the face velocities v hat along axis a (0..2, an active axis) of the state
 * u_star (six interior-only arrays, ghost-filled here with the descriptor's boundaries).
 * vhat_out holds the faces of every line along a: (n_a + 1) faces, face c between
 * interior cells c-1 and c, the other axes as in the state (x fastest).  Returns 0, or -1
 * for an inactive axis or a failed allocation. */
int oracle_face_velocities(const oracle_desc* d, double* const u_star[NFIELD], int a,
                           double* vhat_out) {
  if (a < 0 || a > 2 || d->n[a] == 1) return -1;
  gshape s = make_shape(d);
  double* Us[NFIELD];
  for (int f = 0; f < NFIELD; f++) {
    Us[f] = (double*)calloc(s.cells, sizeof(double));
    if (!Us[f]) return -1;
    scatter_interior(&s, u_star[f], Us[f]);
    fill_ghosts(&s, d, Us[f], f);
  }
  double* vel = (double*)xmalloc(s.cells * sizeof(double));
  double* vt = (double*)xmalloc(s.cells * sizeof(double));
  double* vhat = (double*)xmalloc(s.cells * sizeof(double));
  face_velocities(&s, d, Us, a, vel, vt, vhat);
  int m[3] = {d->n[0], d->n[1], d->n[2]};
  m[a] += 1;
  for (int k = 0; k < m[2]; k++)
    for (int j = 0; j < m[1]; j++)
      for (int i = 0; i < m[0]; i++) {
        int c[3] = {i, j, k};
        c[a] -= 1; /* face c[a] + 1/2 of interior cell c[a] - 1 */
        vhat_out[(size_t)i + (size_t)m[0] * ((size_t)j + (size_t)m[1] * (size_t)k)] =
            vhat[gidx(&s, c[0] + s.g[0], c[1] + s.g[1], c[2] + s.g[2])];
      }
  free(vel);
  free(vt);
  free(vhat);
  for (int f = 0; f < NFIELD; f++) free(Us[f]);
  return 0;
}

/* S4-S11 alone: the Lagrangian stage, the energy correction and the diagnostics of a given
 * U* (six interior-only arrays, ghost-filled here with the descriptor's boundaries), as the
 * second half of oracle_step.  Used to check a decomposition of the step over z slabs,
 * whose U* is exchanged between the stages. */
int oracle_lagrangian_step(const oracle_desc* d, double* const u_star[NFIELD],
                           double* const u_out[NFIELD], double tau, double cfl, oracle_diag* diag) {
  gshape s = make_shape(d);
  double* Us[NFIELD];
  double* Un[NFIELD];
  for (int f = 0; f < NFIELD; f++) {
    Us[f] = (double*)calloc(s.cells, sizeof(double));
    Un[f] = (double*)calloc(s.cells, sizeof(double));
    if (!Us[f] || !Un[f]) return -1;
    scatter_interior(&s, u_star[f], Us[f]);
    fill_ghosts(&s, d, Us[f], f); /* S4 */
  }
  lagrangian_stage(&s, d, Us, Un, tau); /* S5-S7 */
  double rho_vac = d->vacuum_frac * d->rho_mean;
  long long cnt[4] = {0, 0, 0, 0};
  for (int k = s.g[2]; k < s.g[2] + s.n[2]; k++)
    for (int j = s.g[1]; j < s.g[1] + s.n[1]; j++)
      for (int i = s.g[0]; i < s.g[0] + s.n[0]; i++) {
        size_t g = gidx(&s, i, j, k);
        double u[NFIELD];
        for (int f = 0; f < NFIELD; f++) u[f] = Un[f][g];
        cnt[energy_correction(u, rho_vac)]++; /* S8 */
        for (int f = 0; f < NFIELD; f++) Un[f][g] = u[f];
      }
  for (int f = 0; f < NFIELD; f++) gather_interior(&s, Un[f], u_out[f]);
  if (diag) {
    memset(diag, 0, sizeof(*diag));
    diag_of(d, u_out, cfl, diag); /* S10, S11 */
    diag->n_vacuum = cnt[1] + cnt[3];
    diag->n_keep_e = cnt[2];
    diag->n_zero_m = cnt[3];
  }
  for (int f = 0; f < NFIELD; f++) {
    free(Us[f]);
    free(Un[f]);
  }
  return 0;
}

/* One full step.  u_in, u_out: six interior-only arrays each (may alias: the output is
 * written only at the end).  u_star (optional, may be NULL): receives U* interior.
 * phi (optional): interior-only potential, ghost-filled with the state's boundaries
 * (reflecting walls treated as zero-gradient for Phi).  cfl: used only for diag. */
int oracle_step(const oracle_desc* d, double* const u_in[NFIELD], double* const u_out[NFIELD],
                double* const u_star[NFIELD], const double* phi_in, double tau, double cfl,
                oracle_diag* diag) {
  gshape s = make_shape(d);
  double* U[NFIELD];
  double* Us[NFIELD];
  double* Un[NFIELD];
  double* phi = NULL;
  for (int f = 0; f < NFIELD; f++) {
    U[f] = (double*)calloc(s.cells, sizeof(double));
    Us[f] = (double*)calloc(s.cells, sizeof(double));
    Un[f] = (double*)calloc(s.cells, sizeof(double));
    if (!U[f] || !Us[f] || !Un[f]) return -1;
    scatter_interior(&s, u_in[f], U[f]);
    fill_ghosts(&s, d, U[f], f); /* S0 */
  }
  if (phi_in) {
    oracle_desc dphi = *d;
    for (int q = 0; q < 6; q++)
      if (dphi.bc[q] == BC_REFLECT || dphi.bc[q] == BC_INFLOW) dphi.bc[q] = BC_OUTFLOW;
    phi = (double*)calloc(s.cells, sizeof(double));
    scatter_interior(&s, phi_in, phi);
    fill_ghosts(&s, &dphi, phi, -1);
  }
  eulerian_stage(&s, d, U, Us, phi, tau); /* S1-S3 */
  for (int f = 0; f < NFIELD; f++) {
    fill_ghosts(&s, d, Us[f], f); /* S4 */
    if (u_star) gather_interior(&s, Us[f], u_star[f]);
  }
  lagrangian_stage(&s, d, Us, Un, tau); /* S5-S7 */
  /* S8, serial counters */
  double rho_vac = d->vacuum_frac * d->rho_mean;
  long long cnt[4] = {0, 0, 0, 0};
  for (int k = s.g[2]; k < s.g[2] + s.n[2]; k++)
    for (int j = s.g[1]; j < s.g[1] + s.n[1]; j++)
      for (int i = s.g[0]; i < s.g[0] + s.n[0]; i++) {
        size_t g = gidx(&s, i, j, k);
        double u[NFIELD];
        for (int f = 0; f < NFIELD; f++) u[f] = Un[f][g];
        cnt[energy_correction(u, rho_vac)]++;
        for (int f = 0; f < NFIELD; f++) Un[f][g] = u[f];
      }
  for (int f = 0; f < NFIELD; f++) gather_interior(&s, Un[f], u_out[f]);
  if (diag) {
    memset(diag, 0, sizeof(*diag));
    diag_of(d, u_out, cfl, diag); /* S10, S11 */
    diag->n_vacuum = cnt[1] + cnt[3];
    diag->n_keep_e = cnt[2];
    diag->n_zero_m = cnt[3];
  }
  for (int f = 0; f < NFIELD; f++) {
    free(U[f]);
    free(Us[f]);
    free(Un[f]);
  }
  free(phi);
  return 0;
}
