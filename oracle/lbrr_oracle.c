/*
 * FP64 CPU oracle of the recursive-regularized (RR) BGK lattice Boltzmann step
 * of Malaspinas, "Increasing stability and accuracy of the lattice Boltzmann
 * scheme: recursivity and regularization" (arXiv:1505.06900).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header,
 * table or helper with the CUDA library: it carries its own lattice tables and
 * follows the paper's formulas one by one, in the paper's order:
 *
 *   moments rho, rho*u            (Sec. 2, eq_def_rho / eq_def_j)
 *   equilibrium f0                (Sec. 3.2, eq_fzero_d2q9 / eq_fzero_d3q27)
 *   a1^(2) = Pi^(1)               (Sec. 2, P^(1) = a1^(2); projection of f - f0)
 *   a1^(3..6) by the recursion    (Sec. 3.1 eq_rel_a1, written out in Appendix B,
 *                                  with the starred O(Ma^(n+1)) terms dropped)
 *   f1                            (Sec. 3.2, eq_fone_d2q9 / eq_fone_d3q27)
 *   f_post = f0 + (1 - 1/tau) f1  (Sec. 3.5, eq_discr_bgk_reg; tau is the
 *                                  shifted relaxation time tau-bar of Sec. 3.4)
 *   streaming f_i(x + xi_i, t+1)  (eq_discr_bgk_reg), periodic wrap, with a
 *                                  plain two-array pull update.
 *
 * No-slip walls (Sec. 3.7, boundary conditions): the regularized Dirichlet
 * procedure with u_bc = 0 on boundary nodes that lie on the walls (rho from
 * the lattice symmetries, f0(rho, u_bc), Pi^(1) from the symmetries,
 * f1 = w / (2 cs^4) H2 : Pi^(1), all populations replaced by f0 + f1), then
 * the usual collision; see wall_regularize.
 *
 * The order-2 regularized model of Sec. 3.8.1 (eq_feq_2) is the comparator
 * variant ORA_REG2; ORA_BGK is the plain BGK update of Sec. 3.4
 * (eq_full_discr_bgk) with the same full-basis equilibrium. Everything is plain loops in double precision; no
 * blocking, fusion or reordering beyond the formulas. Population arrays are
 * laid out f[i][z][y][x] (x fastest), i = (cx+1) + 3(cy+1) + 9(cz+1).
 *
 * D3Q19 (the paper leaves its recursion open, Sec. 5): the D3Q27 velocities
 * without the eight corners, weights 1/3, 1/18, 1/36. That rule integrates
 * polynomials up to degree five exactly, so orders 0..2 keep their Hermite
 * norms; order-3 products have degree six and are not exact there:
 * <H_xxy, H_yzz> = -cs^6 on D3Q19 (0 on D3Q27), xyz vanishes on every D3Q19
 * velocity, and the order-4 members are not orthogonal to order 2
 * (<H_xxyy, H_zz> = -cs^6). The basis kept is therefore 1, xi, H2 and, for
 * each odd index b with even pair (a, c), H_aab + H_bcc and H_aab - H_bcc,
 * which D3Q19 keeps orthogonal to each other and to the lower orders with
 * norms 2 cs^6 and 6 cs^6. f0 and f1 are the expansions on that basis
 * whose coefficients are the projections of the Hermite coefficients
 * (a_aab +- a_bcc) given by Sec. 2 (f0) and by the recursion (f1); with the
 * sum and the difference both kept, every order-3 Hermite moment except xyz
 * is reproduced.
 *
 * Readings of the paper that this file depends on:
 *  - lattice weights and c_s^2 = 1/3: the paper names D2Q9/D3Q27 Gauss-Hermite
 *    quadratures (Sec. 3.2) without printing them; the tensor products of the
 *    D1Q3 rule {2/3, 1/6, 1/6} at {0, +-1} are used.
 *  - Hermite polynomials: the paper defers to Grad; the standard tensor
 *    Hermite polynomials with variance c_s^2 are used (H_xxy = (x^2-cs2) y ...).
 *  - Appendix B, 2D a1^(4)_xxyy: the printed "a^(3)_xxy" is read as a1^(3)_xxy.
 *  - Walls: populations of a buried link (a population and its opposite both
 *    streaming in from outside, on edges and corners) are taken at
 *    equilibrium when rho is formed; boundary nodes start at rest; the
 *    enstrophy with walls is the trapezoidal rule over the nodes with
 *    second-order one-sided differences on the wall planes.
 *  - The initial non-equilibrium stress uses a1^(2) = -2 c_s^2 rho tau S
 *    (Sec. 3.3 CE result) with tau the scheme's tau-bar, S by periodic second
 *    order central differences.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_D2Q9 9
#define ORA_D3Q27 27
#define ORA_D3Q19 19
#define ORA_RR 0
#define ORA_REG2 1
#define ORA_BGK 2
#define ORA_INIT_EQ 0
#define ORA_INIT_EQ_NEQ_FD 1

static const double cs2 = 1.0 / 3.0; /* lattice speed of sound squared */

typedef struct {
  int d, q;
  int c[27][3];
  double w[27];
} ora_lattice;

/* Gauss-Hermite quadrature of Sec. 3.2: tensor product of the D1Q3 rule. */
static int make_lattice(int lattice, ora_lattice *L) {
  static const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
  if (lattice == ORA_D2Q9) {
    L->d = 2;
    L->q = 9;
  } else if (lattice == ORA_D3Q27) {
    L->d = 3;
    L->q = 27;
  } else if (lattice == ORA_D3Q19) {
    /* D3Q27 order without the corners; weights by |xi|^2 = 0, 1, 2 */
    static const double w19[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    L->d = 3;
    L->q = 19;
    int k = 0;
    for (int i = 0; i < 27; ++i) {
      const int c[3] = {i % 3 - 1, (i / 3) % 3 - 1, i / 9 - 1};
      const int m = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
      if (m == 3) continue;
      for (int a = 0; a < 3; ++a) L->c[k][a] = c[a];
      L->w[k] = w19[m];
      ++k;
    }
    return 0;
  } else {
    return -1;
  }
  for (int i = 0; i < L->q; ++i) {
    int ix = i % 3, iy = (i / 3) % 3, iz = i / 9;
    L->c[i][0] = ix - 1;
    L->c[i][1] = iy - 1;
    L->c[i][2] = (L->d == 3) ? iz - 1 : 0;
    L->w[i] = w1[ix] * w1[iy] * (L->d == 3 ? w1[iz] : 1.0);
  }
  return 0;
}

/* Hermite coefficients of orders 2..6 kept by the D3Q27 basis (Sec. 3.2);
 * D2Q9 uses the subset xx, xy, yy, xxy, xyy, xxyy. */
typedef struct {
  double xx, xy, xz, yy, yz, zz;
  double xxy, xxz, xyy, xzz, yzz, yyz, xyz;
  double xxyy, xxzz, yyzz, xyzz, xyyz, xxyz;
  double xxyzz, xxyyz, xyyzz;
  double xxyyzz;
} hcoef;

/* one-dimensional Hermite factor of degree two, xi^2 - c_s^2 */
static double h2(double x) { return x * x - cs2; }

/* Hermite expansion of a population set, Sec. 3.2 (the expansion of f_i for
 * D2Q9 and for D3Q27; D3Q19 on the basis described in the header):
 * f_i = w_i ( c0 + xi.c1/cs2 + H2:a2/(2cs4) + ... ).
 * c0 is the order-0 coefficient, c1 the order-1 coefficient, a the orders 2..6.
 */
static double hermite_sum(const ora_lattice *L, int i, double c0, const double c1[3],
                          const hcoef *a) {
  const double x = L->c[i][0], y = L->c[i][1], z = L->c[i][2];
  const double cs4 = cs2 * cs2, cs6 = cs4 * cs2, cs8 = cs6 * cs2;
  const double cs10 = cs8 * cs2, cs12 = cs10 * cs2;
  double s = c0;
  if (L->d == 2) {
    s += (x * c1[0] + y * c1[1]) / cs2;
    s += (h2(x) * a->xx + 2.0 * x * y * a->xy + h2(y) * a->yy) / (2.0 * cs4);
    s += (h2(x) * y * a->xxy + x * h2(y) * a->xyy) / (2.0 * cs6);
    s += h2(x) * h2(y) * a->xxyy / (4.0 * cs8);
  } else if (L->q == 19) {
    s += (x * c1[0] + y * c1[1] + z * c1[2]) / cs2;
    s += (h2(x) * a->xx + h2(y) * a->yy + h2(z) * a->zz +
          2.0 * (x * y * a->xy + x * z * a->xz + y * z * a->yz)) /
         (2.0 * cs4);
    /* order 3 on D3Q19: H_aab + H_bcc (norm 2 cs^6), H_aab - H_bcc (6 cs^6) */
    s += (x * (h2(y) + h2(z)) * (a->xyy + a->xzz) + y * (h2(x) + h2(z)) * (a->xxy + a->yzz) +
          z * (h2(x) + h2(y)) * (a->xxz + a->yyz)) /
         (2.0 * cs6);
    s += (x * (y * y - z * z) * (a->xyy - a->xzz) + y * (x * x - z * z) * (a->xxy - a->yzz) +
          z * (x * x - y * y) * (a->xxz - a->yyz)) /
         (6.0 * cs6);
  } else {
    s += (x * c1[0] + y * c1[1] + z * c1[2]) / cs2;
    s += (h2(x) * a->xx + h2(y) * a->yy + h2(z) * a->zz +
          2.0 * (x * y * a->xy + x * z * a->xz + y * z * a->yz)) /
         (2.0 * cs4);
    s += (h2(x) * y * a->xxy + h2(x) * z * a->xxz + x * h2(y) * a->xyy +
          x * h2(z) * a->xzz + y * h2(z) * a->yzz + h2(y) * z * a->yyz +
          2.0 * x * y * z * a->xyz) /
         (2.0 * cs6);
    s += (h2(x) * h2(y) * a->xxyy + h2(x) * h2(z) * a->xxzz + h2(y) * h2(z) * a->yyzz +
          2.0 * (x * y * h2(z) * a->xyzz + x * h2(y) * z * a->xyyz +
                 h2(x) * y * z * a->xxyz)) /
         (4.0 * cs8);
    s += (h2(x) * y * h2(z) * a->xxyzz + h2(x) * h2(y) * z * a->xxyyz +
          x * h2(y) * h2(z) * a->xyyzz) /
         (4.0 * cs10);
    s += h2(x) * h2(y) * h2(z) * a->xxyyzz / (8.0 * cs12);
  }
  return L->w[i] * s;
}

/* Equilibrium Hermite coefficients a0^(n) = rho u...u (Sec. 2, and the
 * recursion a0^(n) = a0^(n-1) u of Sec. 3.1), orders 2..6. */
static void equilibrium_coefficients(double rho, const double u[3], hcoef *a) {
  const double ux = u[0], uy = u[1], uz = u[2];
  a->xx = rho * ux * ux;
  a->xy = rho * ux * uy;
  a->xz = rho * ux * uz;
  a->yy = rho * uy * uy;
  a->yz = rho * uy * uz;
  a->zz = rho * uz * uz;
  a->xxy = a->xx * uy;
  a->xxz = a->xx * uz;
  a->xyy = a->xy * uy;
  a->xzz = a->xz * uz;
  a->yzz = a->yz * uz;
  a->yyz = a->yy * uz;
  a->xyz = a->xy * uz;
  a->xxyy = a->xxy * uy;
  a->xxzz = a->xxz * uz;
  a->yyzz = a->yyz * uz;
  a->xyzz = a->xyz * uz;
  a->xyyz = a->xyy * uz;
  a->xxyz = a->xxy * uz;
  a->xxyzz = a->xxyz * uz;
  a->xxyyz = a->xxyy * uz;
  a->xyyzz = a->xyyz * uz;
  a->xxyyzz = a->xxyyz * uz;
}

/* f0_i of eq_fzero_d2q9 / eq_fzero_d3q27. With variant ORA_REG2 the series is
 * cut at order two (eq_feq_2). */
static double feq(const ora_lattice *L, int variant, int i, double rho, const double u[3]) {
  hcoef a;
  if (variant == ORA_BGK) variant = ORA_RR;
  double j[3] = {rho * u[0], rho * u[1], rho * u[2]};
  equilibrium_coefficients(rho, u, &a);
  if (variant == ORA_REG2) {
    hcoef a2;
    memset(&a2, 0, sizeof a2);
    a2.xx = a.xx; a2.xy = a.xy; a2.xz = a.xz;
    a2.yy = a.yy; a2.yz = a.yz; a2.zz = a.zz;
    return hermite_sum(L, i, rho, j, &a2);
  }
  return hermite_sum(L, i, rho, j, &a);
}

/* Off-equilibrium coefficients of order 3..6 from a1^(2) and u by the
 * recursion eq_rel_a1, as written out in Appendix B (2D and 3D), with the
 * starred O(Ma^(n+1)) terms ignored as Appendix B prescribes. a->xx..zz must
 * hold a1^(2) on entry. */
static void recursive_coefficients(int d, const double u[3], hcoef *a) {
  const double ux = u[0], uy = u[1], uz = u[2];
  if (d == 2) {
    a->xyy = ux * a->yy + 2.0 * uy * a->xy;
    a->xxy = 2.0 * ux * a->xy + uy * a->xx;
    a->xxyy = uy * a->xxy + ux * ux * a->yy + 2.0 * ux * uy * a->xy;
    return;
  }
  /* n = 3 */
  a->xxy = 2.0 * ux * a->xy + uy * a->xx;
  a->xxz = 2.0 * ux * a->xz + uz * a->xx;
  a->xyy = ux * a->yy + 2.0 * uy * a->xy;
  a->xzz = ux * a->zz + 2.0 * uz * a->xz;
  a->yzz = uy * a->zz + 2.0 * uz * a->yz;
  a->yyz = 2.0 * uy * a->yz + uz * a->yy;
  a->xyz = ux * a->yz + uy * a->xz + uz * a->xy;
  /* n = 4 */
  a->xxyy = ux * ux * a->yy + 2.0 * ux * uy * a->xy + uy * a->xxy;
  a->xxzz = ux * ux * a->zz + 2.0 * ux * uz * a->xz + uz * a->xxz;
  a->yyzz = uy * uy * a->zz + 2.0 * uy * uz * a->yz + uz * a->yyz;
  a->xyzz = ux * uy * a->zz + ux * uz * a->yz + uy * uz * a->xz + uz * a->xyz;
  a->xyyz = 2.0 * ux * uy * a->yz + uy * uy * a->xz + uz * a->xyy;
  a->xxyz = ux * ux * a->yz + 2.0 * ux * uy * a->xz + uz * a->xxy;
  /* n = 5 */
  a->xxyzz = ux * ux * uy * a->zz + ux * ux * uz * a->yz + 2.0 * ux * uy * uz * a->xz +
             uz * a->xxyz;
  a->xxyyz = 2.0 * ux * ux * uy * a->yz + 2.0 * ux * uy * uy * a->xz + uz * a->xxyy;
  a->xyyzz = ux * uy * uy * a->zz + 2.0 * ux * uy * uz * a->yz + uy * uy * uz * a->xz +
             uz * a->xyyz;
  /* n = 6 */
  a->xxyyzz = ux * ux * uy * uy * a->zz + 2.0 * ux * ux * uy * uz * a->yz +
              2.0 * ux * uy * uy * uz * a->xz + uz * a->xxyyz;
}

/* f1_i of eq_fone_d2q9 / eq_fone_d3q27 from the coefficients a1. With variant
 * ORA_REG2 only the order-two term is kept (Sec. 3.8.1). */
static double fneq(const ora_lattice *L, int variant, int i, const hcoef *a1) {
  const double zero[3] = {0.0, 0.0, 0.0};
  if (variant == ORA_BGK) variant = ORA_RR;
  if (variant == ORA_REG2) {
    hcoef a2;
    memset(&a2, 0, sizeof a2);
    a2.xx = a1->xx; a2.xy = a1->xy; a2.xz = a1->xz;
    a2.yy = a1->yy; a2.yz = a1->yz; a2.zz = a1->zz;
    return hermite_sum(L, i, 0.0, zero, &a2);
  }
  return hermite_sum(L, i, 0.0, zero, a1);
}

/* rho = sum f, rho u = sum xi f (eq_def_rho, eq_def_j on the lattice). */
static void density_velocity(const ora_lattice *L, const double *f, double *rho, double u[3]) {
  double r = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < L->q; ++i) {
    r += f[i];
    for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * f[i];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* a1^(2) = P^(1): the order-two Hermite coefficient of f1 = f - f0 (Sec. 2),
 * i.e. sum_i H2_i (f_i - f0_i). */
static void neq_stress(const ora_lattice *L, int variant, const double *f, double rho,
                       const double u[3], hcoef *a1) {
  double s[3][3] = {{0}};
  for (int i = 0; i < L->q; ++i) {
    double fn = f[i] - feq(L, variant, i, rho, u);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        s[a][b] += (L->c[i][a] * L->c[i][b] - (a == b ? cs2 : 0.0)) * fn;
  }
  memset(a1, 0, sizeof *a1);
  a1->xx = s[0][0];
  a1->xy = s[0][1];
  a1->yy = s[1][1];
  if (L->d == 3) {
    a1->xz = s[0][2];
    a1->yz = s[1][2];
    a1->zz = s[2][2];
  }
}

/* Regularized collision of one cell, eq_reg and eq_discr_bgk_reg:
 * f_post_i = f0_i + (1 - 1/tau) f1_i. */
static void collide_cell(const ora_lattice *L, int variant, double tau, const double *f,
                         double *fpost) {
  double rho, u[3];
  hcoef a1;
  density_velocity(L, f, &rho, u);
  if (variant == ORA_BGK) {
    /* eq_full_discr_bgk: f_post = f - (f - f0) / tau */
    for (int i = 0; i < L->q; ++i) fpost[i] = f[i] - (f[i] - feq(L, ORA_RR, i, rho, u)) / tau;
    return;
  }
  neq_stress(L, variant, f, rho, u, &a1);
  recursive_coefficients(L->d, u, &a1);
  for (int i = 0; i < L->q; ++i)
    fpost[i] = feq(L, variant, i, rho, u) + (1.0 - 1.0 / tau) * fneq(L, variant, i, &a1);
}

static long wrap(long a, long n) { return ((a % n) + n) % n; }

/* ------------------------------------------------------------------------ */
/* exported entry points (all arrays double precision, x fastest)            */

int ora_lattice_tables(int lattice, int *d, int *q, int *c /* q*3 */, double *w /* q */) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  *d = L.d;
  *q = L.q;
  for (int i = 0; i < L.q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
  }
  return 0;
}

/* Values of the kept Hermite polynomials at each velocity, and the paper's
 * prefactor of each in the expansion of f (Sec. 3.2). Rows follow the order
 * 1, x, y, (z), xx, xy, (xz), yy, (yz), (zz), then order 3..6 as in hcoef.
 * mult[k] is the number of index orderings of member k, so that the expansion
 * term is w_i * pref[k] * H_k,i * a_k with pref = mult/(n! cs^(2n)).
 * D3Q19: 16 rows, 1, x, y, z, the six of order 2, then H_xyy + H_xzz,
 * H_xxy + H_yzz, H_xxz + H_yyz (pref 1/(2 cs^6)) and the three differences
 * (pref 1/(6 cs^6)), a_k being the sum or difference of the two Hermite
 * coefficients; the remaining rows are left untouched. */
int ora_hermite_basis(int lattice, double *H /* q*q */, double *pref /* q */) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  for (int i = 0; i < L.q; ++i) {
    double x = L.c[i][0], y = L.c[i][1], z = L.c[i][2];
    int k = 0;
    const double cs4 = cs2 * cs2, cs6 = cs4 * cs2, cs8 = cs6 * cs2;
    const double cs10 = cs8 * cs2, cs12 = cs10 * cs2;
#define ROW(val, p)              \
  do {                           \
    H[k * L.q + i] = (val);      \
    pref[k] = (p);               \
    ++k;                         \
  } while (0)
    ROW(1.0, 1.0);
    ROW(x, 1.0 / cs2);
    ROW(y, 1.0 / cs2);
    if (L.q == 19) {
      ROW(z, 1.0 / cs2);
      ROW(h2(x), 1.0 / (2.0 * cs4));
      ROW(x * y, 2.0 / (2.0 * cs4));
      ROW(x * z, 2.0 / (2.0 * cs4));
      ROW(h2(y), 1.0 / (2.0 * cs4));
      ROW(y * z, 2.0 / (2.0 * cs4));
      ROW(h2(z), 1.0 / (2.0 * cs4));
      ROW(x * (h2(y) + h2(z)), 1.0 / (2.0 * cs6));
      ROW(y * (h2(x) + h2(z)), 1.0 / (2.0 * cs6));
      ROW(z * (h2(x) + h2(y)), 1.0 / (2.0 * cs6));
      ROW(x * (y * y - z * z), 1.0 / (6.0 * cs6));
      ROW(y * (x * x - z * z), 1.0 / (6.0 * cs6));
      ROW(z * (x * x - y * y), 1.0 / (6.0 * cs6));
    } else if (L.d == 2) {
      ROW(h2(x), 1.0 / (2.0 * cs4));
      ROW(x * y, 2.0 / (2.0 * cs4));
      ROW(h2(y), 1.0 / (2.0 * cs4));
      ROW(h2(x) * y, 1.0 / (2.0 * cs6));
      ROW(x * h2(y), 1.0 / (2.0 * cs6));
      ROW(h2(x) * h2(y), 1.0 / (4.0 * cs8));
    } else {
      ROW(z, 1.0 / cs2);
      ROW(h2(x), 1.0 / (2.0 * cs4));
      ROW(x * y, 2.0 / (2.0 * cs4));
      ROW(x * z, 2.0 / (2.0 * cs4));
      ROW(h2(y), 1.0 / (2.0 * cs4));
      ROW(y * z, 2.0 / (2.0 * cs4));
      ROW(h2(z), 1.0 / (2.0 * cs4));
      ROW(h2(x) * y, 1.0 / (2.0 * cs6));
      ROW(h2(x) * z, 1.0 / (2.0 * cs6));
      ROW(x * h2(y), 1.0 / (2.0 * cs6));
      ROW(x * h2(z), 1.0 / (2.0 * cs6));
      ROW(y * h2(z), 1.0 / (2.0 * cs6));
      ROW(h2(y) * z, 1.0 / (2.0 * cs6));
      ROW(x * y * z, 2.0 / (2.0 * cs6));
      ROW(h2(x) * h2(y), 1.0 / (4.0 * cs8));
      ROW(h2(x) * h2(z), 1.0 / (4.0 * cs8));
      ROW(h2(y) * h2(z), 1.0 / (4.0 * cs8));
      ROW(x * y * h2(z), 2.0 / (4.0 * cs8));
      ROW(x * h2(y) * z, 2.0 / (4.0 * cs8));
      ROW(h2(x) * y * z, 2.0 / (4.0 * cs8));
      ROW(h2(x) * y * h2(z), 1.0 / (4.0 * cs10));
      ROW(h2(x) * h2(y) * z, 1.0 / (4.0 * cs10));
      ROW(x * h2(y) * h2(z), 1.0 / (4.0 * cs10));
      ROW(h2(x) * h2(y) * h2(z), 1.0 / (8.0 * cs12));
    }
#undef ROW
  }
  return 0;
}

/* Equilibrium populations of one cell (eq_fzero_*; variant 1: eq_feq_2). */
int ora_feq_cell(int lattice, int variant, double rho, const double *u, double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  double uu[3] = {u[0], u[1], L.d == 3 ? u[2] : 0.0};
  for (int i = 0; i < L.q; ++i) out[i] = feq(&L, variant, i, rho, uu);
  return 0;
}

/* Off-equilibrium coefficients a1^(2..n) from u and a1^(2) (Appendix B).
 * pi1 holds xx, xy, yy (2D) or xx, xy, xz, yy, yz, zz (3D). out receives the
 * coefficients in the row order of ora_hermite_basis from order 2 on
 * (3 + 3 = 6 values in 2D, 6 + 7 + 6 + 3 + 1 = 23 in 3D). */
int ora_a1_coefficients(int lattice, const double *u, const double *pi1, double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  hcoef a;
  memset(&a, 0, sizeof a);
  double uu[3] = {u[0], u[1], L.d == 3 ? u[2] : 0.0};
  if (L.d == 2) {
    a.xx = pi1[0]; a.xy = pi1[1]; a.yy = pi1[2];
  } else {
    a.xx = pi1[0]; a.xy = pi1[1]; a.xz = pi1[2];
    a.yy = pi1[3]; a.yz = pi1[4]; a.zz = pi1[5];
  }
  recursive_coefficients(L.d, uu, &a);
  if (L.d == 2) {
    double v[6] = {a.xx, a.xy, a.yy, a.xxy, a.xyy, a.xxyy};
    memcpy(out, v, sizeof v);
  } else {
    double v[23] = {a.xx,   a.xy,   a.xz,   a.yy,   a.yz,    a.zz,    a.xxy,  a.xxz,
                    a.xyy,  a.xzz,  a.yzz,  a.yyz,  a.xyz,   a.xxyy,  a.xxzz, a.yyzz,
                    a.xyzz, a.xyyz, a.xxyz, a.xxyzz, a.xxyyz, a.xyyzz, a.xxyyzz};
    memcpy(out, v, sizeof v);
  }
  return 0;
}

/* Off-equilibrium populations f1 of one cell (eq_fone_*; variant 1: order 2
 * only) from u and a1^(2), higher orders by the recursion. */
int ora_fneq_cell(int lattice, int variant, const double *u, const double *pi1, double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  hcoef a;
  memset(&a, 0, sizeof a);
  double uu[3] = {u[0], u[1], L.d == 3 ? u[2] : 0.0};
  if (L.d == 2) {
    a.xx = pi1[0]; a.xy = pi1[1]; a.yy = pi1[2];
  } else {
    a.xx = pi1[0]; a.xy = pi1[1]; a.xz = pi1[2];
    a.yy = pi1[3]; a.yz = pi1[4]; a.zz = pi1[5];
  }
  recursive_coefficients(L.d, uu, &a);
  for (int i = 0; i < L.q; ++i) out[i] = fneq(&L, variant, i, &a);
  return 0;
}

/* Moments of one cell: rho, u (D), a1^(2) (3 or 6 values). */
int ora_moments_cell(int lattice, int variant, const double *f, double *rho, double *u,
                     double *pi1) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  double uu[3];
  hcoef a;
  density_velocity(&L, f, rho, uu);
  neq_stress(&L, variant, f, *rho, uu, &a);
  for (int k = 0; k < L.d; ++k) u[k] = uu[k];
  if (L.d == 2) {
    pi1[0] = a.xx; pi1[1] = a.xy; pi1[2] = a.yy;
  } else {
    pi1[0] = a.xx; pi1[1] = a.xy; pi1[2] = a.xz;
    pi1[3] = a.yy; pi1[4] = a.yz; pi1[5] = a.zz;
  }
  return 0;
}

/* Post-collision populations of one cell (eq_discr_bgk_reg before streaming). */
int ora_collide_cell(int lattice, int variant, double tau, const double *f, double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  collide_cell(&L, variant, tau, f, out);
  return 0;
}

/* Post-collision populations of one D3Q27 cell with a learned correction
 * delta[17] added to the recursion's off-equilibrium coefficients of orders
 * 3..6 (in the order xxy, xxz, xyy, xzz, yzz, yyz, xyz, xxyy, xxzz, yyzz,
 * xyzz, xyyz, xxyz, xxyzz, xxyyz, xyyzz, xxyyzz) before the (1 - 1/tau)
 * relaxation of eq_discr_bgk_reg. delta = 0 is the RR collision. */
int ora_collide_cell_closure(double tau, const double *f, const double *delta, double *out) {
  ora_lattice L;
  make_lattice(ORA_D3Q27, &L);
  double rho, u[3];
  hcoef a1;
  density_velocity(&L, f, &rho, u);
  neq_stress(&L, ORA_RR, f, rho, u, &a1);
  recursive_coefficients(3, u, &a1);
  double *hi[17] = {&a1.xxy,  &a1.xxz,  &a1.xyy,  &a1.xzz,   &a1.yzz,   &a1.yyz,
                    &a1.xyz,  &a1.xxyy, &a1.xxzz, &a1.yyzz,  &a1.xyzz,  &a1.xyyz,
                    &a1.xxyz, &a1.xxyzz, &a1.xxyyz, &a1.xyyzz, &a1.xxyyzz};
  for (int k = 0; k < 17; ++k) *hi[k] += delta[k];
  for (int i = 0; i < L.q; ++i)
    out[i] = feq(&L, ORA_RR, i, rho, u) + (1.0 - 1.0 / tau) * fneq(&L, ORA_RR, i, &a1);
  return 0;
}

/* nsteps full updates of eq_discr_bgk_reg on a periodic nx*ny*nz grid:
 * collide every cell, then pull-stream f_i(x) <- f_post_i(x - xi_i).
 * f is updated in place (a scratch array of the same size is allocated). */
int ora_step(int lattice, int variant, int nx, int ny, int nz, double tau, double *f,
             int nsteps) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  if (nx <= 0 || ny <= 0 || nz <= 0 || (L.d == 2 && nz != 1) || nsteps < 0) return -1;
  const long n = (long)nx * ny * nz;
  double *post = (double *)malloc(sizeof(double) * L.q * n);
  if (!post) return -2;
  for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < n; ++cell) {
      double fc[27], fp[27];
      for (int i = 0; i < L.q; ++i) fc[i] = f[i * n + cell];
      collide_cell(&L, variant, tau, fc, fp);
      for (int i = 0; i < L.q; ++i) post[i * n + cell] = fp[i];
    }
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < n; ++cell) {
      long x = cell % nx, y = (cell / nx) % ny, z = cell / ((long)nx * ny);
      for (int i = 0; i < L.q; ++i) {
        long xs = wrap(x - L.c[i][0], nx), ys = wrap(y - L.c[i][1], ny);
        long zs = wrap(z - L.c[i][2], nz);
        f[i * n + cell] = post[i * n + (zs * ny + ys) * nx + xs];
      }
    }
  }
  free(post);
  return 0;
}

/* Periodic second-order central difference d u_comp / d x_axis at a cell. */
static double central_diff(const double *u, int comp, int axis, long x, long y, long z, int nx,
                           int ny, int nz) {
  const long n = (long)nx * ny * nz;
  long p[3] = {x, y, z}, m[3] = {x, y, z};
  const long dims[3] = {nx, ny, nz};
  p[axis] = wrap(p[axis] + 1, dims[axis]);
  m[axis] = wrap(m[axis] - 1, dims[axis]);
  const double *uc = u + comp * n;
  return 0.5 * (uc[(p[2] * ny + p[1]) * nx + p[0]] - uc[(m[2] * ny + m[1]) * nx + m[0]]);
}

/* Initial populations from rho [n] and u [d][n]. mode ORA_INIT_EQ: f = f0.
 * mode ORA_INIT_EQ_NEQ_FD: f = f0 + f1 with a1^(2) = -2 cs2 rho tau S, where
 * S = (grad u + grad u^T)/2 by periodic central differences (Sec. 3.3) and
 * higher orders by the recursion. */
int ora_init(int lattice, int variant, int nx, int ny, int nz, double tau, int mode,
             const double *rho, const double *u, double *f) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  if (nx <= 0 || ny <= 0 || nz <= 0 || (L.d == 2 && nz != 1)) return -1;
  const long n = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long cell = 0; cell < n; ++cell) {
    long x = cell % nx, y = (cell / nx) % ny, z = cell / ((long)nx * ny);
    double uu[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < L.d; ++a) uu[a] = u[a * n + cell];
    hcoef a1;
    memset(&a1, 0, sizeof a1);
    if (mode == ORA_INIT_EQ_NEQ_FD) {
      double S[3][3] = {{0}};
      for (int a = 0; a < L.d; ++a)
        for (int b = 0; b < L.d; ++b)
          S[a][b] = 0.5 * (central_diff(u, b, a, x, y, z, nx, ny, nz) +
                           central_diff(u, a, b, x, y, z, nx, ny, nz));
      const double k = -2.0 * cs2 * rho[cell] * tau;
      a1.xx = k * S[0][0];
      a1.xy = k * S[0][1];
      a1.yy = k * S[1][1];
      if (L.d == 3) {
        a1.xz = k * S[0][2];
        a1.yz = k * S[1][2];
        a1.zz = k * S[2][2];
      }
      recursive_coefficients(L.d, uu, &a1);
    }
    for (int i = 0; i < L.q; ++i) {
      double v = feq(&L, variant, i, rho[cell], uu);
      if (mode == ORA_INIT_EQ_NEQ_FD) v += fneq(&L, variant, i, &a1);
      f[i * n + cell] = v;
    }
  }
  return 0;
}

/* Macroscopic fields of every cell: rho [n], u [d][n], a1^(2) [3 or 6][n]. */
int ora_fields(int lattice, int variant, int nx, int ny, int nz, const double *f, double *rho,
               double *u, double *pi1) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  const long n = (long)nx * ny * nz;
  const int np = L.d == 2 ? 3 : 6;
#pragma omp parallel for schedule(static)
  for (long cell = 0; cell < n; ++cell) {
    double fc[27], r, uu[3], p[6];
    for (int i = 0; i < L.q; ++i) fc[i] = f[i * n + cell];
    ora_moments_cell(lattice, variant, fc, &r, uu, p);
    rho[cell] = r;
    for (int a = 0; a < L.d; ++a) u[a * n + cell] = uu[a];
    for (int k = 0; k < np; ++k) pi1[k * n + cell] = p[k];
  }
  return 0;
}

/* Global diagnostics, serial sums: out = mass, momentum[d], kinetic energy
 * 0.5 sum rho |u|^2. */
int ora_diagnostics(int lattice, int nx, int ny, int nz, const double *f, double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  const long n = (long)nx * ny * nz;
  double mass = 0.0, mom[3] = {0.0, 0.0, 0.0}, ke = 0.0;
  for (long cell = 0; cell < n; ++cell) {
    double fc[27], rho, u[3];
    for (int i = 0; i < L.q; ++i) fc[i] = f[i * n + cell];
    density_velocity(&L, fc, &rho, u);
    mass += rho;
    for (int a = 0; a < L.d; ++a) mom[a] += rho * u[a];
    ke += 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  }
  out[0] = mass;
  for (int a = 0; a < L.d; ++a) out[1 + a] = mom[a];
  out[1 + L.d] = ke;
  return 0;
}

/* Enstrophy 0.5 sum |curl u|^2 with periodic central differences (the
 * enstrophy of Sec. 4.1 summed over cells; 2D: omega = dx uy - dy ux). */
int ora_enstrophy(int lattice, int nx, int ny, int nz, const double *f, double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  const long n = (long)nx * ny * nz;
  double *u = (double *)malloc(sizeof(double) * 3 * n);
  if (!u) return -2;
  for (long cell = 0; cell < n; ++cell) {
    double fc[27], rho, uu[3];
    for (int i = 0; i < L.q; ++i) fc[i] = f[i * n + cell];
    density_velocity(&L, fc, &rho, uu);
    for (int a = 0; a < 3; ++a) u[a * n + cell] = uu[a];
  }
  double s = 0.0;
  for (long cell = 0; cell < n; ++cell) {
    long x = cell % nx, y = (cell / nx) % ny, z = cell / ((long)nx * ny);
    double wx = 0.0, wy = 0.0, wz;
    wz = central_diff(u, 1, 0, x, y, z, nx, ny, nz) - central_diff(u, 0, 1, x, y, z, nx, ny, nz);
    if (L.d == 3) {
      wx = central_diff(u, 2, 1, x, y, z, nx, ny, nz) - central_diff(u, 1, 2, x, y, z, nx, ny, nz);
      wy = central_diff(u, 0, 2, x, y, z, nx, ny, nz) - central_diff(u, 2, 0, x, y, z, nx, ny, nz);
    }
    s += 0.5 * (wx * wx + wy * wy + wz * wz);
  }
  free(u);
  *out = s;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* No-slip walls (Sec. 3.7, the boundary-conditions subsection)               */
/*                                                                          */
/* walls: bit a set = axis a is bounded by no-slip walls that pass through   */
/* its first and last node planes (the boundary nodes lie on the walls and   */
/* carry u_bc = 0); the other axes stay periodic. A population of a node is  */
/* unknown when the node it streams from, x - xi_i, lies outside the domain.  */

/* 1 if node p has unknown populations; unknown[i] marks them. */
static int unknown_set(const ora_lattice *L, int walls, const long p[3], const long dims[3],
                       int *unknown) {
  int any = 0;
  for (int i = 0; i < L->q; ++i) {
    unknown[i] = 0;
    for (int a = 0; a < L->d; ++a) {
      if (!((walls >> a) & 1)) continue;
      const long s = p[a] - L->c[i][a];
      if (s < 0 || s >= dims[a]) unknown[i] = 1;
    }
    any |= unknown[i];
  }
  return any;
}

/* The regularized Dirichlet procedure with u_bc = 0, step by step as the
 * paper describes it (after Latt et al. 2008):
 *  1. rho from the lattice symmetries: with zero wall velocity the unknown
 *     populations carry as much mass as their known opposites, so
 *     rho = sum of the known populations whose opposite is known
 *         + 2 x sum of the known populations whose opposite is unknown.
 *     Reading for buried links (a population and its opposite both unknown,
 *     on edges and corners): they are taken at equilibrium, w_i rho, so the
 *     sum above equals rho (1 - sum of their weights).
 *  2. f0_i(rho, u_bc) (eq_fzero with u = 0).
 *  3. Pi^(1) from the symmetries: the off-equilibrium part of an unknown
 *     population is that of its opposite (zero for buried links), and
 *     Pi^(1) = sum_i H2_i f1_i.
 *  4. f1_i = w_i / (2 cs^4) H2_i : Pi^(1), which is eq_fone at u = 0 (the
 *     recursion's higher orders vanish there).
 *  5. every population of the node is replaced by f0_i + f1_i (eq_reg).
 * freg receives the regularized populations. */
static void wall_regularize(const ora_lattice *L, int variant, const double *f,
                            const int *unknown, double *freg) {
  const double zero[3] = {0.0, 0.0, 0.0};
  double s = 0.0, wb = 0.0;
  for (int i = 0; i < L->q; ++i) {
    const int o = L->q - 1 - i;
    if (!unknown[i])
      s += unknown[o] ? 2.0 * f[i] : f[i];
    else if (unknown[o])
      wb += L->w[i];
  }
  const double rho = s / (1.0 - wb);
  double f1[27];
  for (int i = 0; i < L->q; ++i) {
    const int o = L->q - 1 - i;
    if (!unknown[i])
      f1[i] = f[i] - feq(L, variant, i, rho, zero);
    else if (!unknown[o])
      f1[i] = f[o] - feq(L, variant, o, rho, zero);
    else
      f1[i] = 0.0;
  }
  double S[3][3] = {{0}};
  for (int i = 0; i < L->q; ++i)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        S[a][b] += (L->c[i][a] * L->c[i][b] - (a == b ? cs2 : 0.0)) * f1[i];
  hcoef a1;
  memset(&a1, 0, sizeof a1);
  a1.xx = S[0][0];
  a1.xy = S[0][1];
  a1.yy = S[1][1];
  if (L->d == 3) {
    a1.xz = S[0][2];
    a1.yz = S[1][2];
    a1.zz = S[2][2];
  }
  recursive_coefficients(L->d, zero, &a1);
  for (int i = 0; i < L->q; ++i) freg[i] = feq(L, variant, i, rho, zero) + fneq(L, variant, i, &a1);
}

static int check_walls(const ora_lattice *L, int walls, int nx, int ny, int nz) {
  const int dims[3] = {nx, ny, nz};
  if (walls < 0 || walls >= (1 << L->d)) return -1;
  for (int a = 0; a < L->d; ++a)
    if (((walls >> a) & 1) && dims[a] < 3) return -1;
  return 0;
}

/* nsteps updates of eq_discr_bgk_reg with no-slip walls on the axes in
 * `walls`: every boundary node is regularized (wall_regularize) and then
 * collided like any other node; the pull streaming leaves the populations
 * that would come from outside the domain undefined (NaN), to be rebuilt by
 * the next regularization. */
int ora_step_walls(int lattice, int variant, int nx, int ny, int nz, double tau, int walls,
                   double *f, int nsteps) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  if (nx <= 0 || ny <= 0 || nz <= 0 || (L.d == 2 && nz != 1) || nsteps < 0) return -1;
  if (check_walls(&L, walls, nx, ny, nz)) return -1;
  const long n = (long)nx * ny * nz;
  const long dims[3] = {nx, ny, nz};
  double *post = (double *)malloc(sizeof(double) * L.q * n);
  if (!post) return -2;
  for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < n; ++cell) {
      const long p[3] = {cell % nx, (cell / nx) % ny, cell / ((long)nx * ny)};
      double fc[27], fr[27], fp[27];
      int unknown[27];
      for (int i = 0; i < L.q; ++i) fc[i] = f[i * n + cell];
      if (unknown_set(&L, walls, p, dims, unknown)) {
        wall_regularize(&L, variant, fc, unknown, fr);
        collide_cell(&L, variant, tau, fr, fp);
      } else {
        collide_cell(&L, variant, tau, fc, fp);
      }
      for (int i = 0; i < L.q; ++i) post[i * n + cell] = fp[i];
    }
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < n; ++cell) {
      const long p[3] = {cell % nx, (cell / nx) % ny, cell / ((long)nx * ny)};
      for (int i = 0; i < L.q; ++i) {
        long q[3];
        int out = 0;
        for (int a = 0; a < 3; ++a) {
          q[a] = p[a] - L.c[i][a];
          if ((walls >> a) & 1)
            out |= q[a] < 0 || q[a] >= dims[a];
          else
            q[a] = wrap(q[a], dims[a]);
        }
        f[i * n + cell] = out ? NAN : post[i * n + (q[2] * ny + q[1]) * nx + q[0]];
      }
    }
  }
  free(post);
  return 0;
}

/* Initial populations with walls: as ora_init for the nodes off the walls
 * (their central differences never cross a wall); the boundary nodes start
 * at rest, f = f0(rho, 0). */
int ora_init_walls(int lattice, int variant, int nx, int ny, int nz, double tau, int mode,
                   int walls, const double *rho, const double *u, double *f) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  if (check_walls(&L, walls, nx, ny, nz)) return -1;
  int rc = ora_init(lattice, variant, nx, ny, nz, tau, mode, rho, u, f);
  if (rc) return rc;
  const long n = (long)nx * ny * nz;
  const long dims[3] = {nx, ny, nz};
  const double zero[3] = {0.0, 0.0, 0.0};
  for (long cell = 0; cell < n; ++cell) {
    const long p[3] = {cell % nx, (cell / nx) % ny, cell / ((long)nx * ny)};
    int unknown[27];
    if (unknown_set(&L, walls, p, dims, unknown))
      for (int i = 0; i < L.q; ++i) f[i * n + cell] = feq(&L, variant, i, rho[cell], zero);
  }
  return 0;
}

/* Macroscopic fields with walls: a boundary node reports those of its
 * regularized populations (rho of the symmetry rule, u = u_bc = 0, Pi^(1)). */
int ora_fields_walls(int lattice, int variant, int nx, int ny, int nz, int walls, const double *f,
                     double *rho, double *u, double *pi1) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  if (check_walls(&L, walls, nx, ny, nz)) return -1;
  const long n = (long)nx * ny * nz;
  const long dims[3] = {nx, ny, nz};
  const int np = L.d == 2 ? 3 : 6;
#pragma omp parallel for schedule(static)
  for (long cell = 0; cell < n; ++cell) {
    const long p[3] = {cell % nx, (cell / nx) % ny, cell / ((long)nx * ny)};
    double fc[27], fr[27], r, uu[3], pp[6];
    int unknown[27];
    for (int i = 0; i < L.q; ++i) fc[i] = f[i * n + cell];
    if (unknown_set(&L, walls, p, dims, unknown)) {
      wall_regularize(&L, variant, fc, unknown, fr);
      memcpy(fc, fr, sizeof fr);
    }
    ora_moments_cell(lattice, variant, fc, &r, uu, pp);
    rho[cell] = r;
    for (int a = 0; a < L.d; ++a) u[a * n + cell] = uu[a];
    for (int k = 0; k < np; ++k) pi1[k * n + cell] = pp[k];
  }
  return 0;
}

/* d u_comp / d x_axis at node p with walls: second-order one-sided
 * differences on the wall planes of a walled axis, central differences
 * elsewhere (periodic across the faces of periodic axes). */
static double wall_at(const double *uc, int axis, const long p[3], const long dims[3], long k) {
  long q[3] = {p[0], p[1], p[2]};
  q[axis] = k;
  return uc[(q[2] * dims[1] + q[1]) * dims[0] + q[0]];
}

static double wall_diff(const double *u, int comp, int axis, const long p[3], const long dims[3],
                        int walls) {
  const long n = dims[0] * dims[1] * dims[2];
  const double *uc = u + comp * n;
  const long m = dims[axis], a = p[axis];
  if ((walls >> axis) & 1) {
    if (a == 0)
      return 0.5 * (-3.0 * wall_at(uc, axis, p, dims, 0) + 4.0 * wall_at(uc, axis, p, dims, 1) -
                    wall_at(uc, axis, p, dims, 2));
    if (a == m - 1)
      return 0.5 * (3.0 * wall_at(uc, axis, p, dims, m - 1) -
                    4.0 * wall_at(uc, axis, p, dims, m - 2) + wall_at(uc, axis, p, dims, m - 3));
    return 0.5 * (wall_at(uc, axis, p, dims, a + 1) - wall_at(uc, axis, p, dims, a - 1));
  }
  return 0.5 * (wall_at(uc, axis, p, dims, wrap(a + 1, m)) -
                wall_at(uc, axis, p, dims, wrap(a - 1, m)));
}

/* Enstrophy with walls, the trapezoidal rule of 0.5 |curl u|^2 over the
 * nodes (weight 1/2 on each wall plane a node lies on), velocities of
 * ora_fields_walls, derivatives of wall_diff. In lattice units: the
 * dimensionless 0.5 int omega^2 dA of Sec. 4.1 is this sum / U_lb^2. */
int ora_enstrophy_walls(int lattice, int nx, int ny, int nz, int walls, const double *f,
                        double *out) {
  ora_lattice L;
  if (make_lattice(lattice, &L)) return -1;
  if (check_walls(&L, walls, nx, ny, nz)) return -1;
  const long n = (long)nx * ny * nz;
  const long dims[3] = {nx, ny, nz};
  double *rho = (double *)malloc(sizeof(double) * n);
  double *u = (double *)calloc(3 * n, sizeof(double));
  double *pi = (double *)malloc(sizeof(double) * 6 * n);
  if (!rho || !u || !pi) {
    free(rho);
    free(u);
    free(pi);
    return -2;
  }
  ora_fields_walls(lattice, ORA_RR, nx, ny, nz, walls, f, rho, u, pi);
  double s = 0.0;
  for (long cell = 0; cell < n; ++cell) {
    const long p[3] = {cell % nx, (cell / nx) % ny, cell / ((long)nx * ny)};
    double wgt = 1.0;
    for (int a = 0; a < L.d; ++a)
      if (((walls >> a) & 1) && (p[a] == 0 || p[a] == dims[a] - 1)) wgt *= 0.5;
    double wx = 0.0, wy = 0.0;
    const double wz = wall_diff(u, 1, 0, p, dims, walls) - wall_diff(u, 0, 1, p, dims, walls);
    if (L.d == 3) {
      wx = wall_diff(u, 2, 1, p, dims, walls) - wall_diff(u, 1, 2, p, dims, walls);
      wy = wall_diff(u, 0, 2, p, dims, walls) - wall_diff(u, 2, 0, p, dims, walls);
    }
    s += wgt * 0.5 * (wx * wx + wy * wy + wz * wz);
  }
  free(rho);
  free(u);
  free(pi);
  *out = s;
  return 0;
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
