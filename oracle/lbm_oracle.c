/*
 * Plain FP64 CPU oracle of the D2Q9 lattice Boltzmann step for isotropic
 * linear elastic solids (Escande, Kolluru, Cleon, Sagaut, arXiv 2009.06404).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is compared against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may build, load or
 * call it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every routine below follows one passage of the paper, cited beside it, and
 * takes the algorithm's steps in the paper's order:
 *
 *   lattice          D2Q9 velocities/weights, b^2 = 1/3      Sec. 2 (after Eq. 12), Eq. 27
 *   equilibrium      f_i^eq(rho, j, P^n)                    Eqs. 14-15
 *   forcing          S_i = w_i c_i.S / b^2                  Eq. 11
 *   elastic source   S = (mu - lambda)/rho0 grad(rho) + F   Eqs. 9-10
 *   absorbing layer  -A j treated as a forcing              Sec. 6.4, Eq. 44
 *   LBGK update      f* = f - (f - f^eq)/tau + (1-1/(2tau)) S_i   Eq. 18
 *   streaming        pull form of the left side of Eq. 18
 *   rigid wall       half-way bounce-back                   Sec. 6.1, Eq. 36
 *   free surface     anti-bounce-back with extrapolated rho_air, P_air
 *                                                           Sec. 6.2, Eqs. 37-42
 *   Ricker x Gaussian body force                            Sec. 5 (first paragraph)
 *
 * Readings of passages that are silent or garbled (each one is also listed in
 * the design notes of the repository):
 *   - The first-moment line of Eq. 12 prints sum f^eq c = j - S/2; this
 *     contradicts the solvability condition Eq. 22 (sum f^neq c = -S/2) together
 *     with sum f^eq c = j.  The oracle uses the consistent reading: the physical
 *     flux is j = sum f c + S/2 and f^eq is built from that j.
 *   - Populations are deviations from a rest state with rho_r = 0 (the step is
 *     linear-affine, so this is exact).
 *   - The absorbing term -A j enters S and the S/2 shift implicitly:
 *     j = (m + (G + F)/2) / (1 + A/2), S = G + F - A j, with G the elastic
 *     force.  A(x) = A_max (d/L)^2, d the depth into a layer of thickness L
 *     (d = 0 on the first interior cell); corners take the largest value.
 *     A_max <= 0 selects 12.8/L for each layer.
 *   - Free surface: "t + Delta x" in the ABB formula is read as t + Delta t;
 *     the other stress components of P_air are zero (P_air n = 0) and the
 *     tangential diagonal stress is kept.  rho and P of the post-collision
 *     populations equal those of the pre-collision ones (the collision conserves
 *     both), so they are taken from f* at time t.  Two extrapolations to the
 *     wall: fs_order = 1 is the paper's linear one, rho_air = 1.5 rho_b -
 *     0.5 rho_in and the same for the tangential stress (Eq. 39); fs_order = 0
 *     takes the boundary cell's own rho and stress.  The linear one has growing
 *     modes at every tangential wavenumber (|eig| up to 1.046 per step at
 *     tau = 1, 1.009 at tau = 0.55), the constant one none.
 *   - grad(rho) at a wall uses a ghost value: free surface 2 rho_b - rho_in
 *     (fs_order = 1) or rho_b (fs_order = 0), rigid wall rho_b; periodic axes
 *     wrap.  The rigid ghost makes the wall a mirror plane (a field uniform
 *     along the wall evolves as half of its mirror-extended periodic
 *     domain); the free-surface ghost makes the force summed over the solid
 *     equal to the surface term of the divergence theorem with the wall
 *     density of Eq. 39's order.
 *   - A diagonal link that leaves the domain through both a horizontal and a
 *     vertical wall takes the rule of the horizontal (top/bottom) wall.
 *   - Source: g(x) = exp(-|x - x_s|^2 / (2 sigma^2)) for |x - x_s| <= r_cut,
 *     else 0 (minimum-image distance on periodic axes); Ricker
 *     r(t) = (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2); the force of
 *     step n is evaluated at t = n.
 *   - Displacement u^{n+1} = u^n + j^n / rho0 (Delta t = 1); receivers record
 *     (u^{n+1}, j^n / rho0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9

/* D2Q9 lattice (Sec. 2, "the widely used D2Q9 lattice"): c_0 = 0, then the
 * four axis links, then the four diagonals, counter-clockwise. */
static const int ex[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double wt[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* b^2 = v_S^2 = 1/3 for regular lattices (Sec. 2, after Eq. 12). */
static const double bb = 1.0 / 3.0;

static int opposite(int i) {
  int k;
  for (k = 0; k < NQ; k++)
    if (ex[k] == -ex[i] && ey[k] == -ey[i]) return k;
  return -1;
}

enum { BC_PERIODIC = 0, BC_FREE = 1, BC_RIGID = 2 };

typedef struct {
  int nx, ny;
  double tau;
  int bc_top, bc_bottom, bc_left, bc_right;
  int sp_top, sp_bottom, sp_left, sp_right;
  double sp_amax;
  int fs_order; /* free-surface extrapolation: 1 linear (Eq. 39), 0 constant */
  const double *rho0, *lam, *mu; /* [ny][nx] each */
  int nsrc;
  const double *src; /* 9 per source: x y sigma dir_x dir_y amplitude f_peak t0 r_cut */
  int nrec;
  const int *rec; /* 2 per receiver: x y */
  int nthreads;
} oracle_problem;

/* ---------------------------------------------------------------- lattice */

void oracle_lattice(int *cx, int *cy, double *w, double *b2) {
  int i;
  for (i = 0; i < NQ; i++) {
    cx[i] = ex[i];
    cy[i] = ey[i];
    w[i] = wt[i];
  }
  *b2 = bb;
}

/* Eq. 14 with Eq. 15: f_i^eq = w_i (rho + j.c_i/b^2 + P^n:(c_i c_i - b^2 I)/(2 b^4)),
 * P^n = P - rho b^2 I. */
void oracle_equilibrium(double rho, double jx, double jy, double pxx,
                        double pxy, double pyy, double *feq) {
  double pnxx = pxx - rho * bb, pnyy = pyy - rho * bb, pnxy = pxy;
  int i;
  for (i = 0; i < NQ; i++) {
    double cx = ex[i], cy = ey[i];
    double cj = cx * jx + cy * jy;
    double hxx = cx * cx - bb, hyy = cy * cy - bb, hxy = cx * cy;
    double pn_h = pnxx * hxx + 2.0 * pnxy * hxy + pnyy * hyy;
    feq[i] = wt[i] * (rho + cj / bb + pn_h / (2.0 * bb * bb));
  }
}

/* Eq. 11: S_i = w_i c_i.S / b^2. */
void oracle_forcing(double sx, double sy, double *si) {
  int i;
  for (i = 0; i < NQ; i++) si[i] = wt[i] * (ex[i] * sx + ey[i] * sy) / bb;
}

/* Ricker wavelet of peak frequency f centred on t0 (Sec. 5). */
double oracle_ricker(double t, double f, double t0) {
  double a = M_PI * M_PI * f * f * (t - t0) * (t - t0);
  return (1.0 - 2.0 * a) * exp(-a);
}

/* ---------------------------------------------------------------- helpers */

static double *plane(double *f, const oracle_problem *p, int i) {
  return f + (size_t)i * p->nx * p->ny;
}
static const double *cplane(const double *f, const oracle_problem *p, int i) {
  return f + (size_t)i * p->nx * p->ny;
}

/* Moments of the nine populations of one cell: rho = sum f, m = sum f c,
 * P = sum f c c (Eq. 12 applied to f). */
static void cell_moments(const double *f, const oracle_problem *p, int x,
                         int y, double *rho, double *mx, double *my,
                         double *pxx, double *pxy, double *pyy) {
  size_t c = (size_t)y * p->nx + x;
  int i;
  *rho = *mx = *my = *pxx = *pxy = *pyy = 0.0;
  for (i = 0; i < NQ; i++) {
    double v = cplane(f, p, i)[c];
    *rho += v;
    *mx += v * ex[i];
    *my += v * ey[i];
    *pxx += v * ex[i] * ex[i];
    *pxy += v * ex[i] * ey[i];
    *pyy += v * ey[i] * ey[i];
  }
}

/* Wall rule for the incoming population i at boundary cell (x, y).
 * nxo, nyo is the outward unit normal of the wall crossed by the link.
 * Rigid wall: Eq. 36, f_ibar(x_b, t+1) = f*_i(x_b, t).
 * Free surface: Eqs. 37-42, anti-bounce-back with rho_air and P_air
 * extrapolated from x_b and x_in = x_b - n. */
static double wall_value(const double *fs, const oracle_problem *p, int bc,
                         int nxo, int nyo, int i, int x, int y) {
  int k = opposite(i); /* the population that left x_b through the wall */
  size_t c = (size_t)y * p->nx + x;
  double fk = cplane(fs, p, k)[c];
  if (bc == BC_RIGID) return fk;
  {
    double rb, mxb, myb, pxxb, pxyb, pyyb;
    double ri, mxi, myi, pxxi, pxyi, pyyi;
    double rho_air, pxx_air = 0.0, pyy_air = 0.0;
    double pnxx, pnyy, pnxy, hxx, hyy, hxy, cx, cy;
    cell_moments(fs, p, x, y, &rb, &mxb, &myb, &pxxb, &pxyb, &pyyb);
    cell_moments(fs, p, x - nxo, y - nyo, &ri, &mxi, &myi, &pxxi, &pxyi,
                 &pyyi);
    if (p->fs_order == 1) {
      /* linear extrapolation to the wall half a cell out (Eq. 39) */
      rho_air = 1.5 * rb - 0.5 * ri;
      if (nyo != 0) /* horizontal wall: the tangential stress is P_xx */
        pxx_air = 1.5 * pxxb - 0.5 * pxxi;
      else /* vertical wall: the tangential stress is P_yy */
        pyy_air = 1.5 * pyyb - 0.5 * pyyi;
    } else {
      /* constant extrapolation: the values of the boundary cell */
      rho_air = rb;
      if (nyo != 0)
        pxx_air = pxxb;
      else
        pyy_air = pyyb;
    }
    pnxx = pxx_air - bb * rho_air;
    pnyy = pyy_air - bb * rho_air;
    pnxy = 0.0;
    cx = ex[k];
    cy = ey[k];
    hxx = cx * cx - bb;
    hyy = cy * cy - bb;
    hxy = cx * cy;
    return -fk + 2.0 * wt[k] *
                     (rho_air + (pnxx * hxx + 2.0 * pnxy * hxy + pnyy * hyy) /
                                    (2.0 * bb * bb));
  }
}

/* Pull streaming (left side of Eq. 18 read backwards): the population i
 * arriving at (x, y) left x - c_i one step earlier. */
static double pull(const double *fs, const oracle_problem *p, int i, int x,
                   int y) {
  int sx = x - ex[i], sy = y - ey[i];
  if (sy < 0 || sy >= p->ny) {
    if (p->bc_top == BC_PERIODIC) {
      sy = (sy + p->ny) % p->ny;
    } else if (sy < 0) {
      return wall_value(fs, p, p->bc_top, 0, -1, i, x, y);
    } else {
      return wall_value(fs, p, p->bc_bottom, 0, 1, i, x, y);
    }
  }
  if (sx < 0 || sx >= p->nx) {
    if (p->bc_left == BC_PERIODIC) {
      sx = (sx + p->nx) % p->nx;
    } else if (sx < 0) {
      return wall_value(fs, p, p->bc_left, -1, 0, i, x, y);
    } else {
      return wall_value(fs, p, p->bc_right, 1, 0, i, x, y);
    }
  }
  return cplane(fs, p, i)[(size_t)sy * p->nx + sx];
}

/* rho at (x, y), where (x, y) may lie one cell outside the domain: periodic
 * axes wrap, walls use the ghost values of the reading above. */
static double rho_ghost(const double *rho, const oracle_problem *p, int x,
                        int y) {
  if (y < 0 || y >= p->ny) {
    int yb = y < 0 ? 0 : p->ny - 1, yin = y < 0 ? 1 : p->ny - 2;
    int bc = y < 0 ? p->bc_top : p->bc_bottom;
    if (bc == BC_PERIODIC) return rho[(size_t)((y + p->ny) % p->ny) * p->nx + x];
    if (bc == BC_FREE && p->fs_order == 1)
      return 2.0 * rho[(size_t)yb * p->nx + x] - rho[(size_t)yin * p->nx + x];
    return rho[(size_t)yb * p->nx + x];
  }
  if (x < 0 || x >= p->nx) {
    int xb = x < 0 ? 0 : p->nx - 1, xin = x < 0 ? 1 : p->nx - 2;
    int bc = x < 0 ? p->bc_left : p->bc_right;
    if (bc == BC_PERIODIC) return rho[(size_t)y * p->nx + (x + p->nx) % p->nx];
    if (bc == BC_FREE && p->fs_order == 1)
      return 2.0 * rho[(size_t)y * p->nx + xb] - rho[(size_t)y * p->nx + xin];
    return rho[(size_t)y * p->nx + xb];
  }
  return rho[(size_t)y * p->nx + x];
}

/* Absorbing-layer coefficient A(x) (Sec. 6.4; profile is a reading). */
static double sponge_coeff(const oracle_problem *p, int x, int y) {
  double a = 0.0;
  int L[4] = {p->sp_top, p->sp_bottom, p->sp_left, p->sp_right};
  int d[4];
  int s;
  d[0] = p->sp_top - y;
  d[1] = y - (p->ny - 1 - p->sp_bottom);
  d[2] = p->sp_left - x;
  d[3] = x - (p->nx - 1 - p->sp_right);
  for (s = 0; s < 4; s++) {
    if (L[s] > 0 && d[s] > 0) {
      double amax = p->sp_amax > 0.0 ? p->sp_amax : 12.8 / L[s];
      double r = (double)d[s] / L[s];
      double v = amax * r * r;
      if (v > a) a = v;
    }
  }
  return a;
}

/* Body force of step n at (x, y): sum over sources of
 * amplitude * dir * g(x) * r(n) (Sec. 5). */
static void body_force(const oracle_problem *p, int x, int y, long n,
                       double *fx, double *fy) {
  int s;
  *fx = *fy = 0.0;
  for (s = 0; s < p->nsrc; s++) {
    const double *q = p->src + 9 * s;
    double dx = x - q[0], dy = y - q[1];
    double r2, g, r;
    if (p->bc_left == BC_PERIODIC) dx -= p->nx * floor(dx / p->nx + 0.5);
    if (p->bc_top == BC_PERIODIC) dy -= p->ny * floor(dy / p->ny + 0.5);
    r2 = dx * dx + dy * dy;
    if (r2 > q[8] * q[8]) continue;
    g = exp(-r2 / (2.0 * q[2] * q[2]));
    r = oracle_ricker((double)n, q[6], q[7]);
    *fx += q[5] * q[3] * g * r;
    *fy += q[5] * q[4] * g * r;
  }
}

static int check_problem(const oracle_problem *p) {
  if (p->nx < 3 || p->ny < 3) return -1;
  if ((p->bc_top == BC_PERIODIC) != (p->bc_bottom == BC_PERIODIC)) return -1;
  if ((p->bc_left == BC_PERIODIC) != (p->bc_right == BC_PERIODIC)) return -1;
  if (!(p->tau > 0.5)) return -1;
  return 0;
}

/* Physical flux, source and post-collision populations of one cell, from the
 * streamed populations f[9], its density gradient and the local coefficients
 * (Eqs. 9, 11, 12 with the reading above, 14, 15, 18, 44). */
static void collide(const double *f, double gx_rho, double gy_rho,
                    double Lambda, double A, double Fx, double Fy, double tau,
                    double *fstar, double *jx_out, double *jy_out) {
  double rho = 0, mx = 0, my = 0, pxx = 0, pxy = 0, pyy = 0;
  double Gx, Gy, jx, jy, Sx, Sy;
  double feq[NQ], si[NQ];
  int i;
  for (i = 0; i < NQ; i++) {
    rho += f[i];
    mx += f[i] * ex[i];
    my += f[i] * ey[i];
    pxx += f[i] * ex[i] * ex[i];
    pxy += f[i] * ex[i] * ey[i];
    pyy += f[i] * ey[i] * ey[i];
  }
  /* elastic force (mu - lambda)/rho0 grad rho = Lambda b^2 grad rho (Eq. 9) */
  Gx = Lambda * bb * gx_rho;
  Gy = Lambda * bb * gy_rho;
  /* half-force shift with the absorbing term taken implicitly */
  jx = (mx + 0.5 * (Gx + Fx)) / (1.0 + 0.5 * A);
  jy = (my + 0.5 * (Gy + Fy)) / (1.0 + 0.5 * A);
  Sx = Gx + Fx - A * jx;
  Sy = Gy + Fy - A * jy;
  oracle_equilibrium(rho, jx, jy, pxx, pxy, pyy, feq);
  oracle_forcing(Sx, Sy, si);
  for (i = 0; i < NQ; i++)
    fstar[i] = f[i] - (f[i] - feq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * si[i];
  *jx_out = jx;
  *jy_out = jy;
}

/* Streams fs (post-collision state of step n-1) into fcur and computes rho. */
static void stream_all(const oracle_problem *p, const double *fs, double *fcur,
                       double *rho) {
  int y;
#ifdef _OPENMP
#pragma omp parallel for num_threads(p->nthreads > 0 ? p->nthreads : 1)
#endif
  for (y = 0; y < p->ny; y++) {
    int x, i;
    for (x = 0; x < p->nx; x++) {
      size_t c = (size_t)y * p->nx + x;
      double r = 0.0;
      for (i = 0; i < NQ; i++) {
        double v = pull(fs, p, i, x, y);
        plane(fcur, p, i)[c] = v;
        r += v;
      }
      rho[c] = r;
    }
  }
}

/*
 * Advances the state by nsteps time steps.
 *   fs      [9][ny][nx]  post-collision populations f* of step n0-1 (in/out)
 *   u       [2][ny][nx]  displacement u^{n0} (in/out)
 *   traces  [nsteps][nrec][4] (ux, uy, vx, vy) after each step, or NULL
 * Returns 0, or -1 for an invalid problem.
 */
int oracle_run(const oracle_problem *p, double *fs, double *u, long n0,
               int nsteps, double *traces) {
  size_t cells = (size_t)p->nx * p->ny;
  double *fcur, *rho, *vx, *vy;
  int s;
  if (check_problem(p)) return -1;
  if (nsteps <= 0) return 0;
  fcur = (double *)malloc(sizeof(double) * cells * NQ);
  rho = (double *)malloc(sizeof(double) * cells);
  vx = (double *)malloc(sizeof(double) * cells);
  vy = (double *)malloc(sizeof(double) * cells);
  for (s = 0; s < nsteps; s++) {
    long n = n0 + s;
    int y, r;
    stream_all(p, fs, fcur, rho);
#ifdef _OPENMP
#pragma omp parallel for num_threads(p->nthreads > 0 ? p->nthreads : 1)
#endif
    for (y = 0; y < p->ny; y++) {
      int x, i;
      for (x = 0; x < p->nx; x++) {
        size_t c = (size_t)y * p->nx + x;
        double f[NQ], fst[NQ];
        double gx = 0.5 * (rho_ghost(rho, p, x + 1, y) - rho_ghost(rho, p, x - 1, y));
        double gy = 0.5 * (rho_ghost(rho, p, x, y + 1) - rho_ghost(rho, p, x, y - 1));
        double Lambda = (p->mu[c] - p->lam[c]) / (p->rho0[c] * bb);
        double A = sponge_coeff(p, x, y);
        double Fx, Fy, jx, jy;
        body_force(p, x, y, n, &Fx, &Fy);
        for (i = 0; i < NQ; i++) f[i] = plane(fcur, p, i)[c];
        collide(f, gx, gy, Lambda, A, Fx, Fy, p->tau, fst, &jx, &jy);
        for (i = 0; i < NQ; i++) plane(fs, p, i)[c] = fst[i];
        vx[c] = jx / p->rho0[c];
        vy[c] = jy / p->rho0[c];
        u[c] += vx[c];
        u[cells + c] += vy[c];
      }
    }
    if (traces) {
      for (r = 0; r < p->nrec; r++) {
        size_t c = (size_t)p->rec[2 * r + 1] * p->nx + p->rec[2 * r];
        double *t = traces + ((size_t)s * p->nrec + r) * 4;
        t[0] = u[c];
        t[1] = u[cells + c];
        t[2] = vx[c];
        t[3] = vy[c];
      }
    }
  }
  free(fcur);
  free(rho);
  free(vx);
  free(vy);
  return 0;
}

/*
 * Macroscopic fields of the state reached after n steps (fs = f* of step n-1):
 * the quantities step n would compute before its collision.
 *   out [8][ny][nx] = ux, uy, vx, vy, rho, Pxx, Pxy, Pyy  with v = j/rho0.
 */
int oracle_fields(const oracle_problem *p, const double *fs, const double *u,
                  long n, double *out) {
  size_t cells = (size_t)p->nx * p->ny;
  double *fcur, *rho;
  int y;
  if (check_problem(p)) return -1;
  fcur = (double *)malloc(sizeof(double) * cells * NQ);
  rho = (double *)malloc(sizeof(double) * cells);
  stream_all(p, fs, fcur, rho);
  for (y = 0; y < p->ny; y++) {
    int x, i;
    for (x = 0; x < p->nx; x++) {
      size_t c = (size_t)y * p->nx + x;
      double f[NQ], fst[NQ];
      double gx = 0.5 * (rho_ghost(rho, p, x + 1, y) - rho_ghost(rho, p, x - 1, y));
      double gy = 0.5 * (rho_ghost(rho, p, x, y + 1) - rho_ghost(rho, p, x, y - 1));
      double Lambda = (p->mu[c] - p->lam[c]) / (p->rho0[c] * bb);
      double A = sponge_coeff(p, x, y);
      double Fx, Fy, jx, jy, r = 0, pxx = 0, pxy = 0, pyy = 0;
      body_force(p, x, y, n, &Fx, &Fy);
      for (i = 0; i < NQ; i++) {
        f[i] = plane(fcur, p, i)[c];
        r += f[i];
        pxx += f[i] * ex[i] * ex[i];
        pxy += f[i] * ex[i] * ey[i];
        pyy += f[i] * ey[i] * ey[i];
      }
      collide(f, gx, gy, Lambda, A, Fx, Fy, p->tau, fst, &jx, &jy);
      out[0 * cells + c] = u[c];
      out[1 * cells + c] = u[cells + c];
      out[2 * cells + c] = jx / p->rho0[c];
      out[3 * cells + c] = jy / p->rho0[c];
      out[4 * cells + c] = r;
      out[5 * cells + c] = pxx;
      out[6 * cells + c] = pxy;
      out[7 * cells + c] = pyy;
    }
  }
  free(fcur);
  free(rho);
  return 0;
}

/* Pre-collision populations f^n = stream(f*^{n-1}) (for unit tests of the
 * streaming and wall rules). out [9][ny][nx]. */
int oracle_stream(const oracle_problem *p, const double *fs, double *out) {
  size_t cells = (size_t)p->nx * p->ny;
  double *rho;
  if (check_problem(p)) return -1;
  rho = (double *)malloc(sizeof(double) * cells);
  stream_all(p, fs, out, rho);
  free(rho);
  return 0;
}

/* A(x) over the whole grid, out [ny][nx]. */
void oracle_sponge(const oracle_problem *p, double *out) {
  int x, y;
  for (y = 0; y < p->ny; y++)
    for (x = 0; x < p->nx; x++) out[(size_t)y * p->nx + x] = sponge_coeff(p, x, y);
}

/* Body force of step n over the whole grid, out [2][ny][nx]. */
void oracle_force(const oracle_problem *p, long n, double *out) {
  size_t cells = (size_t)p->nx * p->ny;
  int x, y;
  for (y = 0; y < p->ny; y++)
    for (x = 0; x < p->nx; x++) {
      size_t c = (size_t)y * p->nx + x;
      body_force(p, x, y, n, &out[c], &out[cells + c]);
    }
}

int oracle_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}
