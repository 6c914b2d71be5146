/*
 * FP64 CPU oracle for the double-distribution-function (DDF) lattice Boltzmann
 * scheme with local vorticity recovery (Hajabdollahi & Premnath, arXiv 1908.06742).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no source, header, table or helper with the CUDA
 * path.  It is deliberately plain: every node is processed with 9x9 matrix-vector
 * products built from the paper's definitions, in double precision, in the order
 * the paper states the algorithm (collide in moment space, then stream).
 *
 * State convention: the arrays f[9][ny][nx] and g[9][ny][nx] hold the
 * PRE-collision populations f(x,t), g(x,t) (full values, not deviations).
 * Node (i,j) sits at x=i, y=j.  Lattice units dx = dt = 1 (Sec. 5).
 *
 * Boundary kinds:
 *   0 periodic in x and y                                        (Sec. 5.2)
 *   1 cavity: half-way walls on all four sides, the top one moving (Sec. 5.4)
 *   2 channel: periodic in x, half-way walls at the bottom (static) and top
 *     (moving with u_lid)                                         (Sec. 5.1, 5.3)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* D2Q9 particle velocities, Eq. (particlevelocities). */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

typedef struct {
  int32_t nx, ny, bc, storage;  /* storage: 0 exact FP64, 1 FP32, 2 FP16, 3 BF16 emulation */
  double lam[Q];                /* flow relaxation diag(0,0,0,w3..w8), Eq. (relaxationtimematrix_fluidmotion) */
  double lam_phi[Q];            /* scalar relaxation diag(0,w1..w8), Eq. (relaxationtimematrix_CDE) */
  double beta1, beta2;          /* anisotropy of the third-order scalar equilibria, Eq. (eqmrawmoment_CDE) */
  double cs2, cs2_phi;          /* squared sound speeds c_s^2, c_sphi^2 */
  double rho0, phi0;            /* reference state: wall density and storage offsets */
  double u_lid, phi_lid, phi_wall;
  double phi_min;               /* |phi| below this: cross derivatives and vorticity are NaN */
  double scale_f, scale_g;      /* storage scale for the rounding emulation */
  double fx, fy;                /* constant body force (Sec. 2, F in Eq. momentumeqn) */
  double f_omega;               /* force modulation cos(f_omega t); 0 = steady */
  int32_t scalar_model;         /* scalar collision: 0 MRT (Sec. 3), 1 SRT (App. B),
                                   2 cascaded central moments (App. C),
                                   3 non-cascaded central moments (App. D) */
  int32_t pad_;
} orc_params;

/* ---------------------------------------------------------------------------
 * Moment basis T (Eqs. basisvectors, transformationmatrix) evaluated from the
 * basis polynomials on the lattice velocities, and its inverse by Gaussian
 * elimination with partial pivoting.
 * ------------------------------------------------------------------------- */
static double T_[Q * Q], TI_[Q * Q];
static int basis_ready = 0;

static double basis_poly(int k, double ex, double ey) {
  switch (k) {
    case 0: return 1.0;
    case 1: return ex;
    case 2: return ey;
    case 3: return ex * ex + ey * ey;
    case 4: return ex * ex - ey * ey;
    case 5: return ex * ey;
    case 6: return ex * ex * ey;
    case 7: return ex * ey * ey;
    default: return ex * ex * ey * ey;
  }
}

static int invert(const double* A, double* Ainv, int n) {
  double M[Q][2 * Q];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c)
      M[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (fabs(M[piv][c]) < 1e-300) return -1;
    if (piv != c)
      for (int k = 0; k < 2 * n; ++k) {
        double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t;
      }
    double d = M[c][c];
    for (int k = 0; k < 2 * n; ++k) M[c][k] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double fac = M[r][c];
      if (fac != 0.0)
        for (int k = 0; k < 2 * n; ++k) M[r][k] -= fac * M[c][k];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r][n + c];
  return 0;
}

static void ensure_basis(void) {
  if (basis_ready) return;
  for (int k = 0; k < Q; ++k)
    for (int a = 0; a < Q; ++a) T_[k * Q + a] = basis_poly(k, EX[a], EY[a]);
  invert(T_, TI_, Q);
  basis_ready = 1;
}

static void matvec(const double* A, const double* x, double* y) {
  for (int r = 0; r < Q; ++r) {
    double s = 0.0;
    for (int c = 0; c < Q; ++c) s += A[r * Q + c] * x[c];
    y[r] = s;
  }
}

/* ---------------------------------------------------------------------------
 * Moment equilibria.
 * Flow: Eq. (eqmrawmoment), arranged as m = (k0, kx, ky, kxx+kyy, kxx-kyy, kxy,
 * kxxy, kxyy, kxxyy).  Scalar: Eq. (eqmrawmoment_CDE), same with rho -> phi,
 * c_s -> c_sphi, and beta1, beta2 on the scalar flux inside kxxy, kxyy.
 * ------------------------------------------------------------------------- */
static void raw_to_m(double k0, double kx, double ky, double kxx, double kyy, double kxy,
                     double kxxy, double kxyy, double kxxyy, double* m) {
  m[0] = k0; m[1] = kx; m[2] = ky; m[3] = kxx + kyy; m[4] = kxx - kyy;
  m[5] = kxy; m[6] = kxxy; m[7] = kxyy; m[8] = kxxyy;
}

static void eq_flow(double rho, double ux, double uy, double cs2, double* meq) {
  raw_to_m(rho, rho * ux, rho * uy,
           cs2 * rho + rho * ux * ux, cs2 * rho + rho * uy * uy, rho * ux * uy,
           cs2 * rho * uy + rho * ux * ux * uy, cs2 * rho * ux + rho * ux * uy * uy,
           cs2 * cs2 * rho + cs2 * rho * (ux * ux + uy * uy) + rho * ux * ux * uy * uy, meq);
}

static void eq_scalar(double phi, double ux, double uy, double cs2p, double b1, double b2,
                      double* neq) {
  raw_to_m(phi, phi * ux, phi * uy,
           cs2p * phi + phi * ux * ux, cs2p * phi + phi * uy * uy, phi * ux * uy,
           b1 * cs2p * phi * uy + phi * ux * ux * uy, b2 * cs2p * phi * ux + phi * ux * uy * uy,
           cs2p * cs2p * phi + cs2p * phi * (ux * ux + uy * uy) + phi * ux * ux * uy * uy, neq);
}

/* Rest weights: populations of the equilibrium at u = 0 per unit density. */
static void rest_weights(double cs2, double* w) {
  double meq[Q];
  eq_flow(1.0, 0.0, 0.0, cs2, meq);
  matvec(TI_, meq, w);
}

/* ---------------------------------------------------------------------------
 * Storage-rounding emulation: IEEE round-to-nearest-even of the stored
 * deviation (value - w*ref) * scale to binary32, binary16 or bfloat16, written
 * from the format definitions (significand bits, minimum exponent).
 * ------------------------------------------------------------------------- */
static double round_bits(double v, int sig_bits, int min_q, double max_finite) {
  if (v == 0.0 || !isfinite(v)) return v;
  double a = fabs(v);
  int e;
  frexp(a, &e);              /* a = m * 2^e, 0.5 <= m < 1 */
  int q = e - sig_bits;      /* exponent of one unit in the last place */
  if (q < min_q) q = min_q;  /* subnormal range */
  double r = ldexp(nearbyint(ldexp(a, -q)), q);
  if (r > max_finite) r = INFINITY;
  return copysign(r, v);
}

static double round_storage(int storage, double v) {
  switch (storage) {
    case 1: return (double)(float)v;
    case 2: return round_bits(v, 11, -24, 65504.0);
    case 3: return round_bits(v, 8, -133, 3.3895313892515355e38);
    default: return v;
  }
}

static double emulate(const orc_params* p, double v, double wref, double scale) {
  if (p->storage == 0) return v;
  double d = (v - wref) * scale;
  return round_storage(p->storage, d) / scale + wref;
}

/* ---------------------------------------------------------------------------
 * Collision at one node: m = T f, n = T g; rho, u (Eq. hydrodynamic_fields,
 * F = 0); phi = sum g; relax in moment space; back to velocity space by T^-1
 * (Eqs. MRT-LBEfluidmotion_transformed, MRT-LBECDE).
 * ------------------------------------------------------------------------- */
/* Source moments of the body force F = (Fx, Fy) at velocity u (Sec. 2, the
 * moments sigma' listed after Eq. eqmrawmoment), arranged like m. */
static void source_m(double Fx, double Fy, double ux, double uy, double* S) {
  raw_to_m(0.0, Fx, Fy, 2.0 * Fx * ux, 2.0 * Fy * uy, Fx * uy + Fy * ux,
           Fy * ux * ux + 2.0 * Fx * ux * uy, Fx * uy * uy + 2.0 * Fy * uy * ux,
           2.0 * (Fx * ux * uy * uy + Fy * uy * ux * ux), S);
}

/* Force acting at node c at time t: constant part plus optional field, times
 * cos(f_omega t) when f_omega != 0 (pulsatile driving, Sec. 5.3). */
static void node_force(const orc_params* p, const double* field, size_t N, size_t c, int64_t t,
                       double* Fx, double* Fy) {
  const double mod = p->f_omega != 0.0 ? cos(p->f_omega * (double)t) : 1.0;
  *Fx = (p->fx + (field ? field[c] : 0.0)) * mod;
  *Fy = (p->fy + (field ? field[N + c] : 0.0)) * mod;
}

/* ---------------------------------------------------------------------------
 * Alternative scalar collision models (Apps. B-D).
 * ------------------------------------------------------------------------- */

/* Bare raw-moment basis P of App. B (Eq. basisvectors1): rows |e_x^m e_y^n> for
 * (m, n) = (0,0) (1,0) (0,1) (2,0) (0,2) (1,1) (2,1) (1,2) (2,2); the same orders
 * index the central moments of Eq. (centralmomentdefinitions_CDE). */
static const int MO[Q] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int NO[Q] = {0, 0, 1, 0, 2, 1, 1, 2, 2};

static double ipow(double v, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= v;
  return r;
}

/* Rows of sum_a (.) (e_ax - ux)^m (e_ay - uy)^n: the raw moments for u = 0. */
static void central_matrix(double ux, double uy, double* C) {
  for (int j = 0; j < Q; ++j)
    for (int a = 0; a < Q; ++a) C[j * Q + a] = ipow(EX[a] - ux, MO[j]) * ipow(EY[a] - uy, NO[j]);
}

/* Raw-moment equilibria of Eq. (eqmrawmoment_CDE) in the bare order of App. B. */
static void raw_eq_bare(const orc_params* p, double phi, double ux, double uy, double* q) {
  const double c = p->cs2_phi;
  q[0] = phi;
  q[1] = phi * ux;
  q[2] = phi * uy;
  q[3] = c * phi + phi * ux * ux;
  q[4] = c * phi + phi * uy * uy;
  q[5] = phi * ux * uy;
  q[6] = p->beta1 * c * phi * uy + phi * ux * ux * uy;
  q[7] = p->beta2 * c * phi * ux + phi * ux * uy * uy;
  q[8] = c * c * phi + c * phi * (ux * ux + uy * uy) + phi * ux * ux * uy * uy;
}

/* Central-moment equilibria, Eq. (eqmcentralmoment_CDE): the local Maxwellian's,
 * with (beta - 1) anisotropy in the third-order ones. */
static void central_eq(const orc_params* p, double phi, double ux, double uy, double* e) {
  const double c = p->cs2_phi;
  e[0] = phi;
  e[1] = 0.0;
  e[2] = 0.0;
  e[3] = c * phi;
  e[4] = c * phi;
  e[5] = 0.0;
  e[6] = (p->beta1 - 1.0) * c * phi * uy;
  e[7] = (p->beta2 - 1.0) * c * phi * ux;
  e[8] = c * c * phi;
}

/* Solve C g = rhs for g (9 x 9, Gaussian elimination through invert()). */
static void solve9(const double* C, const double* rhs, double* g) {
  double Ci[Q * Q];
  invert(C, Ci, Q);
  matvec(Ci, rhs, g);
}

/* App. B: single relaxation time, g~ = g - (g - g^eq)/tau_phi with g^eq = P^-1 q^eq
 * and 1/tau_phi = lam_phi[1]. */
static void scalar_srt(const orc_params* p, const double* g, double phi, double ux, double uy,
                       double* gs) {
  double P[Q * Q], q[Q], geq[Q];
  central_matrix(0.0, 0.0, P);
  raw_eq_bare(p, phi, ux, uy, q);
  solve9(P, q, geq);
  const double w = p->lam_phi[1];
  for (int a = 0; a < Q; ++a) gs[a] = g[a] - w * (g[a] - geq[a]);
}

/* App. D: every central moment relaxes to its equilibrium at its own rate (the
 * pair xx, yy through their sum at lam_phi[3] and difference at lam_phi[4]);
 * the post-collision populations are the ones with those central moments. */
static void scalar_central(const orc_params* p, const double* g, double phi, double ux,
                           double uy, double* gs) {
  double C[Q * Q], k[Q], e[Q], kt[Q];
  central_matrix(ux, uy, C);
  matvec(C, g, k);
  central_eq(p, phi, ux, uy, e);
  const double* w = p->lam_phi;
  kt[0] = k[0];
  kt[1] = k[1] + w[1] * (e[1] - k[1]);
  kt[2] = k[2] + w[2] * (e[2] - k[2]);
  const double sum = (k[3] + k[4]) + w[3] * ((e[3] + e[4]) - (k[3] + k[4]));
  const double dif = (k[3] - k[4]) + w[4] * ((e[3] - e[4]) - (k[3] - k[4]));
  kt[3] = 0.5 * (sum + dif);
  kt[4] = 0.5 * (sum - dif);
  for (int j = 5; j < Q; ++j) kt[j] = k[j] + w[j] * (e[j] - k[j]);
  solve9(C, kt, gs);
}

/* App. C: cascaded collision.  The changes h_0..h_8 of the moments are found
 * order by order so that each central moment relaxes at its rate, then
 * g~ = g + K h with the orthogonal basis K of Eq. (orthogonalbasisvectors).
 * Reading: the printed K6 = |e_x^2 e_y>, K7 = |e_x e_y^2> are not orthogonal to
 * K2, K1 and contradict the printed inner products (<e_x|K h> = 6 h1,
 * <e_x^2 e_y|K h> = 4 h2 - 4 h6) and the printed expansion of g~; all three are
 * met by the orthogonal K6 = 2|e_y> - 3|e_x^2 e_y>, K7 = 2|e_x> - 3|e_x e_y^2>. */
static double kbasis(int j, int ex, int ey) {
  const double x2 = ex * ex, y2 = ey * ey;
  switch (j) {
    case 0: return 1.0;
    case 1: return ex;
    case 2: return ey;
    case 3: return 3.0 * (x2 + y2) - 4.0;
    case 4: return x2 - y2;
    case 5: return (double)(ex * ey);
    case 6: return 2.0 * ey - 3.0 * x2 * ey;
    case 7: return 2.0 * ex - 3.0 * ex * y2;
    default: return 9.0 * x2 * y2 - 6.0 * (x2 + y2) + 4.0;
  }
}

static void scalar_cascaded(const orc_params* p, const double* g, double phi, double ux,
                            double uy, double* gs) {
  double C[Q * Q], k[Q], e[Q], h[Q];
  central_matrix(ux, uy, C);
  matvec(C, g, k);            /* pre-collision central moments */
  central_eq(p, phi, ux, uy, e);
  const double* w = p->lam_phi;
  const double ux2 = ux * ux, uy2 = uy * uy;
  h[0] = 0.0;
  h[1] = w[1] / 6.0 * (e[1] - k[1]);
  h[2] = w[2] / 6.0 * (e[2] - k[2]);
  h[3] = w[3] / 12.0 * ((e[3] + e[4]) - (k[3] + k[4])) + (ux * h[1] + uy * h[2]);
  h[4] = w[4] / 4.0 * ((e[3] - e[4]) - (k[3] - k[4])) + 3.0 * (ux * h[1] - uy * h[2]);
  h[5] = w[5] / 4.0 * (e[5] - k[5]) + 1.5 * (ux * h[2] + uy * h[1]);
  h[6] = -w[6] / 4.0 * (e[6] - k[6]) - 2.0 * ux * h[5] - 0.5 * uy * h[4] - 1.5 * uy * h[3] +
         (1.0 + 1.5 * ux2) * h[2] + 3.0 * ux * uy * h[1];
  h[7] = -w[7] / 4.0 * (e[7] - k[7]) - 2.0 * uy * h[5] + 0.5 * ux * h[4] - 1.5 * ux * h[3] +
         3.0 * ux * uy * h[2] + (1.0 + 1.5 * uy2) * h[1];
  h[8] = w[8] / 4.0 * (e[8] - k[8]) - 2.0 * ux * h[7] - 2.0 * uy * h[6] - 4.0 * ux * uy * h[5] +
         0.5 * (ux2 - uy2) * h[4] - (2.0 + 1.5 * (ux2 + uy2)) * h[3] +
         (2.0 + 3.0 * ux2) * uy * h[2] + (2.0 + 3.0 * uy2) * ux * h[1];
  for (int a = 0; a < Q; ++a) {
    double d = 0.0;
    for (int j = 0; j < Q; ++j) d += kbasis(j, EX[a], EY[a]) * h[j];
    gs[a] = g[a] + d;
  }
}

/* Scalar relaxation rate j as the model uses it (SRT: the single rate lam_phi[1]). */
static double wphi(const orc_params* p, int j) {
  return p->scalar_model == 1 ? p->lam_phi[1] : p->lam_phi[j];
}

/* The populations held are f-bar = f - S/2 (the transformation that makes the
 * trapezoidal source explicit, Sec. 2), so u = (sum f-bar e + F/2) / rho
 * (Eq. hydrodynamic_fields) and the collision of Eq.
 * MRT-LBEfluidmotion_transformed is m* = m - Lambda (m - m^eq) + (I - Lambda/2) S. */
static void collide_node(const orc_params* p, const double* f, const double* g,
                         double* fs, double* gs, double Fx, double Fy) {
  double m[Q], n[Q], meq[Q], neq[Q], ms[Q], ns[Q], S[Q];
  matvec(T_, f, m);
  matvec(T_, g, n);
  double rho = m[0], ux = (m[1] + 0.5 * Fx) / rho, uy = (m[2] + 0.5 * Fy) / rho, phi = n[0];
  eq_flow(rho, ux, uy, p->cs2, meq);
  eq_scalar(phi, ux, uy, p->cs2_phi, p->beta1, p->beta2, neq);
  source_m(Fx, Fy, ux, uy, S);
  for (int k = 0; k < Q; ++k) {
    ms[k] = m[k] - p->lam[k] * (m[k] - meq[k]) + (1.0 - 0.5 * p->lam[k]) * S[k];
    ns[k] = n[k] - p->lam_phi[k] * (n[k] - neq[k]);
  }
  matvec(TI_, ms, fs);
  switch (p->scalar_model) {
    case 1: scalar_srt(p, g, phi, ux, uy, gs); break;
    case 2: scalar_cascaded(p, g, phi, ux, uy, gs); break;
    case 3: scalar_central(p, g, phi, ux, uy, gs); break;
    default: matvec(TI_, ns, gs);
  }
}

static int opposite(int a) {
  for (int b = 0; b < Q; ++b)
    if (EX[b] == -EX[a] && EY[b] == -EY[a]) return b;
  return -1;
}

/* One time step: collide every node, then pull-stream with the wall rules.
 * Periodic directions wrap.  A link whose upstream node lies outside a wall:
 *   flow   f_a(x,t+1) =  f*_abar(x,t) + 2 w_a rho0 (e_a . u_w) / c_s^2
 *   scalar g_a(x,t+1) = -g*_abar(x,t) + 2 w^phi_a phi_w
 * with u_w = (u_lid, 0), phi_w = phi_lid when the upstream node is above the
 * top row, else u_w = 0, phi_w = phi_wall (Sec. 5: half-way bounce-back,
 * moving-lid momentum term, fixed scalar value on the walls). */
static void step_once(const orc_params* p, double* f, double* g, double* fs, double* gs,
                      const double* force, int64_t t) {
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
  double w[Q], wp[Q];
  rest_weights(p->cs2, w);
  rest_weights(p->cs2_phi, wp);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      double fl[Q], gl[Q], fo[Q], go[Q], Fx, Fy;
      for (int a = 0; a < Q; ++a) { fl[a] = f[a * N + c]; gl[a] = g[a * N + c]; }
      node_force(p, force, N, c, t, &Fx, &Fy);
      collide_node(p, fl, gl, fo, go, Fx, Fy);
      for (int a = 0; a < Q; ++a) {
        fs[a * N + c] = emulate(p, fo[a], w[a] * p->rho0, p->scale_f);
        gs[a * N + c] = emulate(p, go[a], wp[a] * p->phi0, p->scale_g);
      }
    }
  const int wrap_x = 1, wrap_y = (p->bc == 0);
  const int walls_x = (p->bc == 1);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      for (int a = 0; a < Q; ++a) {
        int si = i - EX[a], sj = j - EY[a];
        int out_x = si < 0 || si >= nx, out_y = sj < 0 || sj >= ny;
        int solid = (out_x && walls_x) || (out_y && !wrap_y);
        if (!solid) {
          if (wrap_x) si = (si + nx) % nx;
          if (wrap_y) sj = (sj + ny) % ny;
          size_t s = (size_t)sj * nx + si;
          f[a * N + c] = fs[a * N + s];
          g[a * N + c] = gs[a * N + s];
        } else {
          int b = opposite(a);
          int lid = sj >= ny;
          double uw = lid ? p->u_lid : 0.0;
          double phw = lid ? p->phi_lid : p->phi_wall;
          f[a * N + c] = fs[b * N + c] + 2.0 * w[a] * p->rho0 * (EX[a] * uw) / p->cs2;
          g[a * N + c] = -gs[b * N + c] + 2.0 * wp[a] * phw;
        }
      }
    }
  (void)wrap_x;
}

/* ======================== exported entry points ======================== */

/* Lattice tables for tests: T, T^-1, velocities and rest weights. */
int orc_lattice(double cs2, double* T, double* Tinv, int32_t* ex, int32_t* ey, double* w) {
  ensure_basis();
  memcpy(T, T_, sizeof T_);
  memcpy(Tinv, TI_, sizeof TI_);
  for (int a = 0; a < Q; ++a) { ex[a] = EX[a]; ey[a] = EY[a]; }
  rest_weights(cs2, w);
  return 0;
}

/* Equilibrium moments of both lattices at one state (tests). */
void orc_equilibria(const orc_params* p, double rho, double ux, double uy, double phi,
                    double* meq, double* neq) {
  ensure_basis();
  eq_flow(rho, ux, uy, p->cs2, meq);
  eq_scalar(phi, ux, uy, p->cs2_phi, p->beta1, p->beta2, neq);
}

/* Collision of one node in isolation (tests). */
void orc_collide_node(const orc_params* p, const double* f, const double* g, double* fs,
                      double* gs) {
  ensure_basis();
  collide_node(p, f, g, fs, gs, 0.0, 0.0);
}

/* Initial populations from macroscopic fields.
 * f = T^-1 (m^eq + m^(1)), g = T^-1 (n^eq + n^(1)), with the Chapman-Enskog
 * non-equilibrium parts of Eqs. (strainratexxpyy)-(strainratexy) for the flow
 * and Eqs. (1stnoneqmmomentx_CDE), (1stnoneqmmomenty_CDE),
 * (offdiagonal2ndnoneqmmoment_CDE) for the scalar; all other non-equilibrium
 * moments are zero.  grads = 6 planes (dxux, dyux, dxuy, dyuy, dxphi, dyphi) or
 * NULL for the pure equilibrium.  With a body force the flow populations held
 * are f-bar = f - S/2 (force at t = 0). */
void orc_init(const orc_params* p, const double* rho, const double* ux, const double* uy,
              const double* phi, const double* grads, double* f, double* g,
              const double* force) {
  ensure_basis();
  const size_t N = (size_t)p->nx * p->ny;
  const double cs2 = p->cs2, cp2 = p->cs2_phi;
  double w[Q], wp[Q];
  rest_weights(p->cs2, w);
  rest_weights(p->cs2_phi, wp);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < (long)N; ++c) {
    double m[Q], n[Q], fl[Q], gl[Q], S[Q], Fx, Fy;
    double r = rho[c], vx = ux[c], vy = uy[c], ph = phi[c];
    eq_flow(r, vx, vy, cs2, m);
    node_force(p, force, N, (size_t)c, 0, &Fx, &Fy);
    source_m(Fx, Fy, vx, vy, S);
    for (int k = 0; k < Q; ++k) m[k] -= 0.5 * S[k];
    eq_scalar(ph, vx, vy, cp2, p->beta1, p->beta2, n);
    /* central-moment models: the equilibrium is the raw image of the central
     * equilibria, and the first-order non-equilibrium parts are those of the
     * central moments (reading: the Chapman-Enskog expansion of a central-moment
     * collision gives eta_x^(1), eta_y^(1) as for the MRT and
     * eta_xy^(1) = -(c/w5)[phi N^phi + (b1 - 1) uy dxphi + (b2 - 1) ux dyphi]) */
    double e[Q];
    const int central = p->scalar_model >= 2;
    if (central) central_eq(p, ph, vx, vy, e);
    if (grads) {
      double dxux = grads[0 * N + c], dyux = grads[1 * N + c];
      double dxuy = grads[2 * N + c], dyuy = grads[3 * N + c];
      double dxph = grads[4 * N + c], dyph = grads[5 * N + c];
      m[3] += -(2.0 * cs2 * r / p->lam[3]) * (dxux + dyuy);
      m[4] += -(2.0 * cs2 * r / p->lam[4]) * (dxux - dyuy);
      m[5] += -(cs2 * r / p->lam[5]) * (dxuy + dyux);
      const double Nphi = ph * (p->beta1 * dxuy + p->beta2 * dyux);
      if (central) {
        e[1] += -(cp2 / wphi(p, 1)) * dxph;
        e[2] += -(cp2 / wphi(p, 2)) * dyph;
        e[5] += -(cp2 / wphi(p, 5)) *
                (Nphi + (p->beta1 - 1.0) * vy * dxph + (p->beta2 - 1.0) * vx * dyph);
      } else {
        n[1] += -(cp2 / wphi(p, 1)) * dxph;
        n[2] += -(cp2 / wphi(p, 2)) * dyph;
        n[5] += -(cp2 / wphi(p, 5)) * (Nphi + p->beta1 * vy * dxph + p->beta2 * vx * dyph);
      }
    }
    matvec(TI_, m, fl);
    if (central) {
      double C[Q * Q];
      central_matrix(vx, vy, C);
      solve9(C, e, gl);
    } else {
      matvec(TI_, n, gl);
    }
    for (int a = 0; a < Q; ++a) {
      f[a * N + c] = emulate(p, fl[a], w[a] * p->rho0, p->scale_f);
      g[a * N + c] = emulate(p, gl[a], wp[a] * p->phi0, p->scale_g);
    }
  }
}

/* Advance nsteps; f, g hold the pre-collision state on entry and exit.
 * fs, gs are caller scratch of the same size. */
void orc_step(const orc_params* p, double* f, double* g, double* fs, double* gs,
              int64_t nsteps, const double* force, int64_t t0) {
  ensure_basis();
  for (int64_t t = t0; t < t0 + nsteps; ++t) step_once(p, f, g, fs, gs, force, t);
}

/* Local kinematics from the current (pre-collision) populations, Sec. 4:
 * out planes (rho, ux, uy, phi, Sxx, Sxy, Syy, omega_z).  If extra != NULL it
 * receives 6 more planes (dxux, dyux, dxuy, dyuy, N_xy, N^phi_xy) and, after
 * them, (dxphi, dyphi). */
void orc_fields(const orc_params* p, const double* f, const double* g, double* out,
                double* extra, const double* force, int64_t t) {
  ensure_basis();
  const size_t N = (size_t)p->nx * p->ny;
  const double cs2 = p->cs2, cp2 = p->cs2_phi, b1 = p->beta1, b2 = p->beta2;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < (long)N; ++c) {
    double fl[Q], gl[Q], m[Q], n[Q], S[Q], Fx, Fy;
    for (int a = 0; a < Q; ++a) { fl[a] = f[a * N + c]; gl[a] = g[a * N + c]; }
    matvec(T_, fl, m);
    matvec(T_, gl, n);
    node_force(p, force, N, (size_t)c, t, &Fx, &Fy);
    double rho = m[0], ux = (m[1] + 0.5 * Fx) / rho, uy = (m[2] + 0.5 * Fy) / rho, phi = n[0];
    /* moments of f = f-bar + S/2 (reading: the non-equilibrium moments of Sec. 4
     * are those of the distribution f itself) */
    source_m(Fx, Fy, ux, uy, S);
    for (int k = 3; k < Q; ++k) m[k] += 0.5 * S[k];
    /* non-equilibrium moments, Sec. 4 (local evaluation) */
    double m3 = m[3] - (2.0 * cs2 * rho + rho * (ux * ux + uy * uy));
    double m4 = m[4] - rho * (ux * ux - uy * uy);
    double m5 = m[5] - rho * ux * uy;
    double n1 = n[1] - phi * ux, n2 = n[2] - phi * uy;
    double n5 = n[5] - phi * ux * uy;
    /* scalar gradient from the first-order non-equilibrium moments */
    double dxph = -wphi(p, 1) / cp2 * n1;
    double dyph = -wphi(p, 2) / cp2 * n2;
    /* N_xy and N^phi_xy, Eqs. (crossderivativeRHS1), (crossderivativeRHS2) */
    double Nxy = -p->lam[5] / (rho * cs2) * m5;
    double dxuy = NAN, dyux = NAN, om = NAN, Nph = NAN;
    if (fabs(phi) >= p->phi_min) {
      if (p->scalar_model >= 2) {
        /* central-moment models (reading, see orc_init): the central xy moment,
         * whose equilibrium is zero, with (beta - 1) in the correction term */
        double C[Q * Q], k[Q];
        central_matrix(ux, uy, C);
        matvec(C, gl, k);
        Nph = -wphi(p, 5) / (phi * cp2) * k[5] -
              ((b1 - 1.0) * uy * dxph + (b2 - 1.0) * ux * dyph) / phi;
      } else {
        Nph = -wphi(p, 5) / (phi * cp2) * n5 - (b1 * uy * dxph + b2 * ux * dyph) / phi;
      }
      dxuy = (Nph - b2 * Nxy) / (b1 - b2);      /* Eq. (offdiagvelderivativeresult1) */
      dyux = (b1 * Nxy - Nph) / (b1 - b2);      /* Eq. (offdiagvelderivativeresult2) */
      om = (2.0 * Nph - (b1 + b2) * Nxy) / (b1 - b2); /* Eq. (vorticityexpression) */
    }
    /* diagonal derivatives, Eqs. (diagvelderivativeresult1), (...2) */
    double dxux = -(p->lam[3] * m3 + p->lam[4] * m4) / (4.0 * cs2 * rho);
    double dyuy = -(p->lam[3] * m3 - p->lam[4] * m4) / (4.0 * cs2 * rho);
    out[0 * N + c] = rho;
    out[1 * N + c] = ux;
    out[2 * N + c] = uy;
    out[3 * N + c] = phi;
    out[4 * N + c] = dxux;
    out[5 * N + c] = 0.5 * Nxy; /* S_xy = (dxuy + dyux)/2 = N_xy/2 */
    out[6 * N + c] = dyuy;
    out[7 * N + c] = om;
    if (extra) {
      extra[0 * N + c] = dxux;
      extra[1 * N + c] = dyux;
      extra[2 * N + c] = dxuy;
      extra[3 * N + c] = dyuy;
      extra[4 * N + c] = Nxy;
      extra[5 * N + c] = Nph;
      extra[6 * N + c] = dxph;
      extra[7 * N + c] = dyph;
    }
  }
}

/* Global sums over the pre-collision state: (sum rho, sum phi, sum |u|^2).
 * Row sums in parallel, then rows added in order (deterministic). */
void orc_sums(const orc_params* p, const double* f, const double* g, double* out3,
              const double* force, int64_t t) {
  ensure_basis();
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
  double* rows = (double*)calloc((size_t)ny * 3, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    double sr = 0, sp = 0, su = 0;
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      double fl[Q], gl[Q], m[Q], n[Q], Fx, Fy;
      for (int a = 0; a < Q; ++a) { fl[a] = f[a * N + c]; gl[a] = g[a * N + c]; }
      matvec(T_, fl, m);
      matvec(T_, gl, n);
      node_force(p, force, N, c, t, &Fx, &Fy);
      double ux = (m[1] + 0.5 * Fx) / m[0], uy = (m[2] + 0.5 * Fy) / m[0];
      sr += m[0];
      sp += n[0];
      su += ux * ux + uy * uy;
    }
    rows[3 * j] = sr; rows[3 * j + 1] = sp; rows[3 * j + 2] = su;
  }
  out3[0] = out3[1] = out3[2] = 0;
  for (int j = 0; j < ny; ++j) {
    out3[0] += rows[3 * j]; out3[1] += rows[3 * j + 1]; out3[2] += rows[3 * j + 2];
  }
  free(rows);
}

/* Number of OpenMP threads the oracle runs with (0 = not built with OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(int set) {
  if (set > 0) omp_set_num_threads(set);
  return omp_get_max_threads();
}
#else
int orc_threads(int set) { (void)set; return 0; }
#endif

/* Storage rounding of n values in place (tests of the emulation itself). */
void orc_round(int32_t storage, double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i) v[i] = round_storage(storage, v[i]);
}
