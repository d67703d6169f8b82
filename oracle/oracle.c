/*
 * FP64 CPU oracle for the AlGDock binding-potential-of-mean-force (BPMF) hot path
 * (Minh, "Alchemical Grid Dock (AlGDock)", arXiv:1507.03703).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, deliberately unoptimised restatement of
 * what the method computes, written to check the CUDA library against.  It shares no code,
 * header, table or constant with that library; only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg load it.  Nothing in the product path may call it.
 *
 * Units: A, kcal/mol, amu, fs, K, elementary charge.  Build with -ffp-contract=off so that every
 * floating-point operation rounds as written (needed for the bit-exact exchange comparison).
 *
 * Contents and the passages they follow (paper sections / equations):
 *   philox4x32_10          Salmon et al., SC'11 (counter-based generator, published definition)
 *   grid_direct_sum        Methodology, "Thermodynamic Cycle": electrostatic and van der Waals
 *                          grids, here computed by direct summation over receptor atoms
 *   prepare_lattices       same section: power-4 transform of the repulsive grid and the soft
 *                          (tanh-capped) repulsive and electrostatic grids
 *   interp                 same section: trilinear interpolation, with its analytic gradient
 *   restraint              Eq. (binding_site): flat-bottom harmonic restraint on the centre of mass
 *   ligand_ff              "Thermodynamic Cycle": GAFF-like sampling force field of the ligand
 *   state weights          Eq. (protocol): alpha_sg, alpha_g and the reduced potential u_alpha
 *   hmc                    "Sampling": HMC with velocity Verlet and the Metropolis criterion
 *   exchange               "Sampling", Eq. (repXacc): Hamiltonian replica exchange sweeps over
 *                          pairs 1..min(5, K-1) states apart
 *   reduced_energies       "Estimation": u_kn for MBAR
 *   mbar                   "Estimation": MBAR (Shirts & Chodera 2008) self-consistent iteration
 *   statistical_inefficiency  "Equilibration and production" (Chodera 2016)
 *   learned proposal       an extension of "Sampling" (not in the paper): network, mixture, move
 *   external_moves         "Sampling": external-coordinate MCMC (random rotation about the centre
 *                          of mass, Gaussian translation, Metropolis) for states with alpha < 0.01
 *   detect_equilibration   "Equilibration and production": the start that maximises N / g
 *   protocol pieces        "Initialization": state statistics, thermodynamic-length steps in T and
 *                          alpha, importance-resampled seeds, mean p_acc, the time-step rule
 *   target_interaction     "Thermodynamic Cycle": the target force field's receptor-ligand energy,
 *                          computed directly (the postprocessing of milestone D samples)
 *
 * Parity unpinned: nothing in this file is left without a pin; see the tests.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ---------------------------------------------------------------- constants (own copy) */
static const double O_KB = 0.0019872043;            /* kcal / (mol K) */
static const double O_COULOMB = 332.0637;           /* kcal A / (mol e^2) */
static const double O_MV2_TO_KCAL = 1.0 / 4.184e-4; /* 1 amu A^2 / fs^2 in kcal/mol */
static const double O_LJR_NODE_CAP = 1.0e10;        /* cap of raw repulsive node values */
static const double O_R_MIN = 0.01;                 /* A, smallest distance in the repulsive sum */
static const double O_R_MIN_ATT = 2.0;              /* A, smallest distance in the attractive and
                                                       electrostatic sums */

enum { O_PURPOSE_MOMENTUM = 1, O_PURPOSE_ACCEPT = 2, O_PURPOSE_EXCHANGE = 3 };

/* ---------------------------------------------------------------- Philox4x32-10 */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t o[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, o);
}

/* Uniform on [0, 1) with 53 random bits: 27 bits of a, 26 bits of b. */
double oracle_u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* Box-Muller pair from two words: u1 in (0,1] via 23 bits + 1/2, u2 in [0,1) via 23 bits. */
static void box_muller(uint32_t a, uint32_t b, double* z0, double* z1) {
  double u1 = ((double)(a >> 9) + 0.5) * (1.0 / 8388608.0);
  double u2 = (double)(b >> 9) * (1.0 / 8388608.0);
  double r = sqrt(-2.0 * log(u1));
  double th = 2.0 * M_PI * u2;
  *z0 = r * cos(th);
  *z1 = r * sin(th);
}

/* ---------------------------------------------------------------- per-atom LJ factors */
/* Receptor-ligand LJ uses geometric combining of A = eps (2R*)^12 and B = 2 eps (2R*)^6, so that
 * an atom's grid energy is sqrt(A_i) * LJr(p) + sqrt(B_i) * LJa(p). */
static double sqrtA_of(double rstar, double eps) { return sqrt(eps * pow(2.0 * rstar, 12.0)); }
static double sqrtB_of(double rstar, double eps) { return sqrt(2.0 * eps * pow(2.0 * rstar, 6.0)); }

/* ---------------------------------------------------------------- grids by direct sum */
typedef struct {
  int n_rec;
  const double *xyz, *sA, *sB, *q;
  const double* pts;
  int64_t n_pts;
  double *ljr, *lja, *elec;
  int64_t begin, end;
} grid_job;

static void grid_point(const grid_job* J, const double p[3], double* vr, double* va, double* ve) {
  double sr = 0.0, sa = 0.0, se = 0.0;
  for (int j = 0; j < J->n_rec; ++j) {
    double dx = p[0] - J->xyz[3 * j], dy = p[1] - J->xyz[3 * j + 1], dz = p[2] - J->xyz[3 * j + 2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double rr = r < O_R_MIN ? O_R_MIN : r;
    double ra = r < O_R_MIN_ATT ? O_R_MIN_ATT : r;
    double ir2 = 1.0 / (rr * rr), ia2 = 1.0 / (ra * ra);
    double ir6 = ir2 * ir2 * ir2, ia6 = ia2 * ia2 * ia2;
    sr += J->sA[j] * (ir6 * ir6); /* 1/r^12 */
    sa -= J->sB[j] * ia6;         /* 1/r^6 */
    se += J->q[j] * ia2 / 4.0;    /* distance-dependent dielectric eps(r) = 4 r */
  }
  *vr = sr;
  *va = sa;
  *ve = O_COULOMB * se;
}

static void* grid_worker(void* arg) {
  grid_job* J = (grid_job*)arg;
  for (int64_t i = J->begin; i < J->end; ++i)
    grid_point(J, J->pts + 3 * i, J->ljr + i, J->lja + i, J->elec + i);
  return NULL;
}

static int n_threads_default(int n) {
  if (n > 0) return n;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

/* Raw grid values at arbitrary points: LJr = sum sqrt(A_j)/r^12, LJa = -sum sqrt(B_j)/r^6,
 * elec = 332.0637 sum q_j / (4 r^2).  The repulsive sum takes r >= 0.01 A; the attractive and
 * electrostatic sums take r >= 2 A, where one receptor atom's repulsion on any ligand atom already
 * exceeds ~80 kcal/mol: without that bound, trilinear interpolation between a node inside a
 * receptor atom and its neighbours opens attractive holes of up to ~1e9 kcal/mol, because the
 * repulsive lattice is interpolated in its 4th root and the others linearly.
 * Returns the number of threads used. */
int oracle_grid_points(int n_rec, const double* rec_xyz, const double* rec_rstar, const double* rec_eps,
                       const double* rec_q, int64_t n_pts, const double* pts, double* ljr, double* lja,
                       double* elec, int n_threads) {
  double* sA = (double*)malloc(sizeof(double) * (size_t)(n_rec > 0 ? n_rec : 1));
  double* sB = (double*)malloc(sizeof(double) * (size_t)(n_rec > 0 ? n_rec : 1));
  for (int j = 0; j < n_rec; ++j) {
    sA[j] = sqrtA_of(rec_rstar[j], rec_eps[j]);
    sB[j] = sqrtB_of(rec_rstar[j], rec_eps[j]);
  }
  int T = n_threads_default(n_threads);
  if (T > n_pts) T = n_pts > 0 ? (int)n_pts : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)T);
  grid_job* jobs = (grid_job*)malloc(sizeof(grid_job) * (size_t)T);
  for (int t = 0; t < T; ++t) {
    grid_job J = {n_rec, rec_xyz, sA, sB, rec_q, pts, n_pts, ljr, lja, elec,
                  n_pts * t / T, n_pts * (t + 1) / T};
    jobs[t] = J;
    pthread_create(&th[t], NULL, grid_worker, &jobs[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  free(th); free(jobs); free(sA); free(sB);
  return T;
}

/* Raw grids on the lattice origin + h*(i,j,k), x fastest. */
int oracle_grid_direct_sum(int n_rec, const double* rec_xyz, const double* rec_rstar, const double* rec_eps,
                           const double* rec_q, const double origin[3], double h, const int n[3],
                           double* ljr, double* lja, double* elec, int n_threads) {
  int64_t nn = (int64_t)n[0] * n[1] * n[2];
  double* pts = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int64_t p = ((int64_t)k * n[1] + j) * n[0] + i;
        pts[3 * p] = origin[0] + h * i;
        pts[3 * p + 1] = origin[1] + h * j;
        pts[3 * p + 2] = origin[2] + h * k;
      }
  int T = oracle_grid_points(n_rec, rec_xyz, rec_rstar, rec_eps, rec_q, nn, pts, ljr, lja, elec, n_threads);
  free(pts);
  return T;
}

/* Soft electrostatic cap: v_e = v_r * min over charged atoms of sqrt(A_i)/|q_i|, so that
 * |q_i| v_e <= sqrt(A_i) v_r for every ligand atom. */
double oracle_soft_elec_cap(double vmax_r, int n_atoms, const double* rstar, const double* eps, const double* q) {
  double best = INFINITY;
  for (int i = 0; i < n_atoms; ++i) {
    if (q[i] == 0.0) continue;
    double r = sqrtA_of(rstar[i], eps[i]) / fabs(q[i]);
    if (r < best) best = r;
  }
  return vmax_r * best;
}

/* Transformed lattices: repulsive stored as its 4th root; soft grids v_max tanh(v / v_max). */
void oracle_prepare_lattices(int64_t n_nodes, const double* ljr, const double* elec, double vmax_r, double vmax_e,
                             double* ljr_t, double* sljr_t, double* selec) {
  for (int64_t p = 0; p < n_nodes; ++p) {
    double v = ljr[p];
    if (v > O_LJR_NODE_CAP) v = O_LJR_NODE_CAP;
    if (v < 0.0) v = 0.0;
    ljr_t[p] = pow(v, 0.25);
    sljr_t[p] = isinf(vmax_r) ? pow(v, 0.25) : pow(vmax_r * tanh(v / vmax_r), 0.25);
    /* an infinite cap (no charged ligand atom) leaves the grid unchanged: v tanh(e/v) -> e */
    selec[p] = isinf(vmax_e) ? elec[p] : vmax_e * tanh(elec[p] / vmax_e);
  }
}

/* ---------------------------------------------------------------- trilinear interpolation */
/* Value and gradient of the trilinear interpolant of lattice L at x.  A coordinate outside the
 * lattice is clamped to its boundary; there the gradient component along it is zero. */
void oracle_interp(const double* L, const int n[3], const double o[3], double h, const double x[3], double* v,
                   double g[3]) {
  int c[3], inside[3];
  double t[3];
  for (int d = 0; d < 3; ++d) {
    double u = (x[d] - o[d]) / h;
    inside[d] = 1;
    if (!(u >= 0.0)) { u = 0.0; inside[d] = 0; } /* also catches NaN */
    if (u > (double)(n[d] - 1)) { u = (double)(n[d] - 1); inside[d] = 0; }
    int ci = (int)floor(u);
    if (ci > n[d] - 2) ci = n[d] - 2;
    c[d] = ci;
    t[d] = u - ci;
  }
  double val = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int e = 0; e < 2; ++e) {
        double node = L[((int64_t)(c[2] + e) * n[1] + (c[1] + b)) * n[0] + (c[0] + a)];
        double wx = a ? t[0] : 1.0 - t[0], dwx = a ? 1.0 : -1.0;
        double wy = b ? t[1] : 1.0 - t[1], dwy = b ? 1.0 : -1.0;
        double wz = e ? t[2] : 1.0 - t[2], dwz = e ? 1.0 : -1.0;
        val += wx * wy * wz * node;
        gx += dwx * wy * wz * node;
        gy += wx * dwy * wz * node;
        gz += wx * wy * dwz * node;
      }
  *v = val;
  g[0] = inside[0] ? gx / h : 0.0;
  g[1] = inside[1] ? gy / h : 0.0;
  g[2] = inside[2] ? gz / h : 0.0;
}

/* ---------------------------------------------------------------- the system */
typedef struct oracle_system {
  /* lattices */
  int n[3];
  double o[3], h;
  double *Lr, *La, *Le, *Lsr, *Lse;
  /* restraint */
  double site[3], k_rest, d0;
  /* ligand */
  int na;
  double *mass, *q, *sA, *sB, *rstar, *eps;
  int nb, nang, ntor, npair;
  int *bonds, *angles, *tors, *pairs;
  double *bk, *br0, *ak, *at0, *tV, *tg, *pscale_lj, *pscale_el;
  /* states */
  int K;
  double *T, *alpha, *dt, *w_sg, *w_g, *beta;
} oracle_system;

static double* dup_d(const double* s, int64_t n) {
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (n > 0) memcpy(d, s, sizeof(double) * (size_t)n);
  return d;
}
static int* dup_i(const int* s, int64_t n) {
  int* d = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (n > 0) memcpy(d, s, sizeof(int) * (size_t)n);
  return d;
}

/* Protocol weights, Eq. (protocol): alpha_sg = 1 - (2a-1)^2, alpha_g = (2a-1)^2 / (1 + e^{-1000(a-1/2)}).
 * The logistic is evaluated in the form that cannot overflow.  alpha = NaN marks a state without
 * receptor grids (the warming leg). */
double oracle_alpha_sg(double a) {
  if (isnan(a)) return 0.0;
  double s = 2.0 * a - 1.0;
  return 1.0 - s * s;
}
double oracle_alpha_g(double a) {
  if (isnan(a)) return 0.0;
  double s = 2.0 * a - 1.0;
  double z = 1000.0 * (a - 0.5);
  double logistic = z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
  return s * s * logistic;
}
double oracle_beta(double T) { return 1.0 / (O_KB * T); }

oracle_system* oracle_system_create(const int n[3], const double origin[3], double h, const double* ljr,
                                    const double* lja, const double* elec, double vmax_r, double vmax_e,
                                    const double site[3], double k_rest, double d0, int na, const double* mass,
                                    const double* q, const double* rstar, const double* eps, int nb,
                                    const int* bonds, const double* bk, const double* br0, int nang,
                                    const int* angles, const double* ak, const double* at0, int ntor,
                                    const int* tors, const double* tV, const double* tg, int K, const double* T,
                                    const double* alpha, const double* dt) {
  oracle_system* s = (oracle_system*)calloc(1, sizeof(oracle_system));
  int64_t nn = (int64_t)n[0] * n[1] * n[2];
  for (int d = 0; d < 3; ++d) { s->n[d] = n[d]; s->o[d] = origin[d]; s->site[d] = site[d]; }
  s->h = h;
  s->Lr = (double*)malloc(sizeof(double) * (size_t)nn);
  s->Lsr = (double*)malloc(sizeof(double) * (size_t)nn);
  s->Lse = (double*)malloc(sizeof(double) * (size_t)nn);
  s->La = dup_d(lja, nn);
  s->Le = dup_d(elec, nn);
  oracle_prepare_lattices(nn, ljr, elec, vmax_r, vmax_e, s->Lr, s->Lsr, s->Lse);
  s->k_rest = k_rest;
  s->d0 = d0;
  s->na = na;
  s->mass = dup_d(mass, na);
  s->q = dup_d(q, na);
  s->rstar = dup_d(rstar, na);
  s->eps = dup_d(eps, na);
  s->sA = (double*)malloc(sizeof(double) * (size_t)(na > 0 ? na : 1));
  s->sB = (double*)malloc(sizeof(double) * (size_t)(na > 0 ? na : 1));
  for (int i = 0; i < na; ++i) { s->sA[i] = sqrtA_of(rstar[i], eps[i]); s->sB[i] = sqrtB_of(rstar[i], eps[i]); }
  s->nb = nb; s->bonds = dup_i(bonds, 2 * (int64_t)nb); s->bk = dup_d(bk, nb); s->br0 = dup_d(br0, nb);
  s->nang = nang; s->angles = dup_i(angles, 3 * (int64_t)nang); s->ak = dup_d(ak, nang); s->at0 = dup_d(at0, nang);
  s->ntor = ntor; s->tors = dup_i(tors, 4 * (int64_t)ntor); s->tV = dup_d(tV, 3 * (int64_t)ntor);
  s->tg = dup_d(tg, 3 * (int64_t)ntor);
  /* Nonbonded pairs: graph distance >= 3 (1-2 and 1-3 excluded); 1-4 pairs scaled by 1/2 (LJ)
   * and 1/1.2 (Coulomb).  Graph distances by breadth-first search over the bonds. */
  int* dist = (int*)malloc(sizeof(int) * (size_t)(na > 0 ? na * na : 1));
  int* queue = (int*)malloc(sizeof(int) * (size_t)(na > 0 ? na : 1));
  for (int i = 0; i < na; ++i) {
    for (int j = 0; j < na; ++j) dist[i * na + j] = -1;
    dist[i * na + i] = 0;
    int head = 0, tail = 0;
    queue[tail++] = i;
    while (head < tail) {
      int u = queue[head++];
      for (int b = 0; b < nb; ++b) {
        int v = -1;
        if (bonds[2 * b] == u) v = bonds[2 * b + 1];
        else if (bonds[2 * b + 1] == u) v = bonds[2 * b];
        if (v >= 0 && dist[i * na + v] < 0) { dist[i * na + v] = dist[i * na + u] + 1; queue[tail++] = v; }
      }
    }
  }
  int cnt = 0;
  for (int i = 0; i < na; ++i)
    for (int j = i + 1; j < na; ++j) {
      int dij = dist[i * na + j];
      if (dij < 0 || dij >= 3) ++cnt;
    }
  s->npair = cnt;
  s->pairs = (int*)malloc(sizeof(int) * 2 * (size_t)(cnt > 0 ? cnt : 1));
  s->pscale_lj = (double*)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
  s->pscale_el = (double*)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
  cnt = 0;
  for (int i = 0; i < na; ++i)
    for (int j = i + 1; j < na; ++j) {
      int dij = dist[i * na + j];
      if (dij < 0 || dij >= 3) {
        s->pairs[2 * cnt] = i;
        s->pairs[2 * cnt + 1] = j;
        s->pscale_lj[cnt] = dij == 3 ? 1.0 / 2.0 : 1.0;
        s->pscale_el[cnt] = dij == 3 ? 1.0 / 1.2 : 1.0;
        ++cnt;
      }
    }
  free(dist);
  free(queue);
  s->K = K;
  s->T = dup_d(T, K);
  s->alpha = dup_d(alpha, K);
  s->dt = dup_d(dt, K);
  s->w_sg = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  s->w_g = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  s->beta = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  for (int k = 0; k < K; ++k) {
    s->w_sg[k] = oracle_alpha_sg(alpha[k]);
    s->w_g[k] = oracle_alpha_g(alpha[k]);
    s->beta[k] = oracle_beta(T[k]);
  }
  return s;
}

/* Replaces the state table (used while a protocol is built state by state). */
void oracle_system_set_states(oracle_system* s, int K, const double* T, const double* alpha, const double* dt) {
  free(s->T); free(s->alpha); free(s->dt); free(s->w_sg); free(s->w_g); free(s->beta);
  s->K = K;
  s->T = dup_d(T, K);
  s->alpha = dup_d(alpha, K);
  s->dt = dup_d(dt, K);
  s->w_sg = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  s->w_g = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  s->beta = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  for (int k = 0; k < K; ++k) {
    s->w_sg[k] = oracle_alpha_sg(alpha[k]);
    s->w_g[k] = oracle_alpha_g(alpha[k]);
    s->beta[k] = oracle_beta(T[k]);
  }
}

void oracle_system_destroy(oracle_system* s) {
  if (!s) return;
  free(s->Lr); free(s->La); free(s->Le); free(s->Lsr); free(s->Lse);
  free(s->mass); free(s->q); free(s->sA); free(s->sB); free(s->rstar); free(s->eps);
  free(s->bonds); free(s->bk); free(s->br0); free(s->angles); free(s->ak); free(s->at0);
  free(s->tors); free(s->tV); free(s->tg); free(s->pairs); free(s->pscale_lj); free(s->pscale_el);
  free(s->T); free(s->alpha); free(s->dt); free(s->w_sg); free(s->w_g); free(s->beta);
  free(s);
}

int oracle_system_npairs(const oracle_system* s) { return s->npair; }
void oracle_system_pairs(const oracle_system* s, int* pairs, double* scale_lj, double* scale_el) {
  for (int p = 0; p < s->npair; ++p) {
    pairs[2 * p] = s->pairs[2 * p];
    pairs[2 * p + 1] = s->pairs[2 * p + 1];
    scale_lj[p] = s->pscale_lj[p];
    scale_el[p] = s->pscale_el[p];
  }
}
void oracle_state_weights(const oracle_system* s, double* w_sg, double* w_g, double* beta) {
  for (int k = 0; k < s->K; ++k) { w_sg[k] = s->w_sg[k]; w_g[k] = s->w_g[k]; beta[k] = s->beta[k]; }
}

/* ---------------------------------------------------------------- energy terms */
/* Grid interaction: psi[0] = Psi_sg (soft repulsive + soft electrostatic), psi[1] = Psi_g
 * (repulsive + attractive + electrostatic).  grad_sg / grad_g (may be NULL) receive dPsi/dx. */
void oracle_grid_terms(const oracle_system* s, const double* x, double psi[2], double* grad_sg, double* grad_g) {
  double Psg = 0.0, Pg = 0.0;
  for (int i = 0; i < s->na; ++i) {
    const double* xi = x + 3 * i;
    double vr, va, ve, vsr, vse, gr[3], ga[3], ge[3], gsr[3], gse[3];
    oracle_interp(s->Lr, s->n, s->o, s->h, xi, &vr, gr);
    oracle_interp(s->La, s->n, s->o, s->h, xi, &va, ga);
    oracle_interp(s->Le, s->n, s->o, s->h, xi, &ve, ge);
    oracle_interp(s->Lsr, s->n, s->o, s->h, xi, &vsr, gsr);
    oracle_interp(s->Lse, s->n, s->o, s->h, xi, &vse, gse);
    Pg += s->sA[i] * pow(vr, 4.0) + s->sB[i] * va + s->q[i] * ve;
    Psg += s->sA[i] * pow(vsr, 4.0) + s->q[i] * vse;
    for (int d = 0; d < 3; ++d) {
      if (grad_g) grad_g[3 * i + d] = 4.0 * s->sA[i] * pow(vr, 3.0) * gr[d] + s->sB[i] * ga[d] + s->q[i] * ge[d];
      if (grad_sg) grad_sg[3 * i + d] = 4.0 * s->sA[i] * pow(vsr, 3.0) * gsr[d] + s->q[i] * gse[d];
    }
  }
  psi[0] = Psg;
  psi[1] = Pg;
}

/* Flat-bottom harmonic restraint of the centre of mass, Eq. (binding_site); F receives -dU/dx. */
double oracle_restraint(const oracle_system* s, const double* x, double* F) {
  double M = 0.0, com[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < s->na; ++i) {
    M += s->mass[i];
    for (int d = 0; d < 3; ++d) com[d] += s->mass[i] * x[3 * i + d];
  }
  double r[3], dd = 0.0;
  for (int d = 0; d < 3; ++d) { com[d] /= M; r[d] = com[d] - s->site[d]; dd += r[d] * r[d]; }
  double dist = sqrt(dd);
  if (F) for (int i = 0; i < 3 * s->na; ++i) F[i] = 0.0;
  if (dist <= s->d0) return 0.0;
  double ex = dist - s->d0;
  if (F)
    for (int i = 0; i < s->na; ++i)
      for (int d = 0; d < 3; ++d) F[3 * i + d] = -s->k_rest * ex * (r[d] / dist) * (s->mass[i] / M);
  return 0.5 * s->k_rest * ex * ex;
}

static void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Ligand intramolecular energy.  terms[0..3] = bonds, angles, torsions, nonbonded (may be NULL).
 * F (may be NULL) receives -dU/dx.
 *   bonds     k (r - r0)^2
 *   angles    k (theta - theta0)^2
 *   torsions  sum_{n=1..3} V_n/2 (1 + cos(n phi - gamma_n))
 *   pairs     eps_ij [(R_ij/r)^12 - 2 (R_ij/r)^6] + 332.0637 q_i q_j / r, Lorentz-Berthelot
 *             (eps_ij = sqrt(eps_i eps_j), R_ij = R*_i + R*_j), 1-4 scaled. */
double oracle_ligand_ff(const oracle_system* s, const double* x, double* F, double* terms) {
  double Eb = 0.0, Ea = 0.0, Et = 0.0, En = 0.0;
  if (F) for (int i = 0; i < 3 * s->na; ++i) F[i] = 0.0;
  for (int b = 0; b < s->nb; ++b) {
    int i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
    double d[3];
    sub3(x + 3 * i, x + 3 * j, d);
    double r = sqrt(dot3(d, d));
    double dr = r - s->br0[b];
    Eb += s->bk[b] * dr * dr;
    if (F) {
      double c = -2.0 * s->bk[b] * dr / r;
      for (int e = 0; e < 3; ++e) { F[3 * i + e] += c * d[e]; F[3 * j + e] -= c * d[e]; }
    }
  }
  for (int a = 0; a < s->nang; ++a) {
    int i = s->angles[3 * a], j = s->angles[3 * a + 1], k = s->angles[3 * a + 2];
    double u[3], w[3];
    sub3(x + 3 * i, x + 3 * j, u);
    sub3(x + 3 * k, x + 3 * j, w);
    double lu = sqrt(dot3(u, u)), lw = sqrt(dot3(w, w));
    double c = dot3(u, w) / (lu * lw);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double dth = th - s->at0[a];
    Ea += s->ak[a] * dth * dth;
    if (F) {
      double sn = sqrt(1.0 - c * c);
      if (sn < 1e-12) sn = 1e-12;
      double dEdth = 2.0 * s->ak[a] * dth;
      for (int e = 0; e < 3; ++e) {
        /* dtheta/dx = -1/sin(theta) dcos/dx */
        double dci = w[e] / (lu * lw) - c * u[e] / (lu * lu);
        double dck = u[e] / (lu * lw) - c * w[e] / (lw * lw);
        double fi = dEdth * dci / sn; /* -dE/dx_i = -dEdth * (-dci/sn) */
        double fk = dEdth * dck / sn;
        F[3 * i + e] += fi;
        F[3 * k + e] += fk;
        F[3 * j + e] -= fi + fk;
      }
    }
  }
  for (int t = 0; t < s->ntor; ++t) {
    int i = s->tors[4 * t], j = s->tors[4 * t + 1], k = s->tors[4 * t + 2], l = s->tors[4 * t + 3];
    double b1[3], b2[3], b3[3], n1[3], n2[3], m[3];
    sub3(x + 3 * j, x + 3 * i, b1);
    sub3(x + 3 * k, x + 3 * j, b2);
    sub3(x + 3 * l, x + 3 * k, b3);
    cross3(b1, b2, n1);
    cross3(b2, b3, n2);
    double lb2 = sqrt(dot3(b2, b2));
    cross3(n1, b2, m);
    /* phi = atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3)) */
    double y = lb2 * dot3(b1, n2);
    double xx = dot3(n1, n2);
    double phi = atan2(y, xx);
    double dEdphi = 0.0;
    for (int nn = 1; nn <= 3; ++nn) {
      double V = s->tV[3 * t + nn - 1], g = s->tg[3 * t + nn - 1];
      Et += 0.5 * V * (1.0 + cos(nn * phi - g));
      dEdphi += -0.5 * V * nn * sin(nn * phi - g);
    }
    if (F) {
      double n1s = dot3(n1, n1), n2s = dot3(n2, n2);
      double dpi[3], dpl[3];
      for (int e = 0; e < 3; ++e) { dpi[e] = -lb2 * n1[e] / n1s; dpl[e] = lb2 * n2[e] / n2s; }
      double p = dot3(b1, b2) / (lb2 * lb2), r = dot3(b3, b2) / (lb2 * lb2);
      for (int e = 0; e < 3; ++e) {
        double dpj = -(1.0 + p) * dpi[e] + r * dpl[e];
        double dpk = p * dpi[e] - (1.0 + r) * dpl[e];
        F[3 * i + e] -= dEdphi * dpi[e];
        F[3 * j + e] -= dEdphi * dpj;
        F[3 * k + e] -= dEdphi * dpk;
        F[3 * l + e] -= dEdphi * dpl[e];
      }
    }
  }
  for (int p = 0; p < s->npair; ++p) {
    int i = s->pairs[2 * p], j = s->pairs[2 * p + 1];
    double d[3];
    sub3(x + 3 * i, x + 3 * j, d);
    double r = sqrt(dot3(d, d));
    double eij = sqrt(s->eps[i] * s->eps[j]);
    double Rij = s->rstar[i] + s->rstar[j];
    double sr6 = pow(Rij / r, 6.0);
    double elj = s->pscale_lj[p] * eij * (sr6 * sr6 - 2.0 * sr6);
    double eel = s->pscale_el[p] * O_COULOMB * s->q[i] * s->q[j] / r;
    En += elj + eel;
    if (F) {
      /* dE/dr = lj: eps (-12 sr12 + 12 sr6)/r ; el: -eel/r */
      double dEdr = s->pscale_lj[p] * eij * (-12.0 * sr6 * sr6 + 12.0 * sr6) / r - eel / r;
      for (int e = 0; e < 3; ++e) {
        double f = -dEdr * d[e] / r;
        F[3 * i + e] += f;
        F[3 * j + e] -= f;
      }
    }
  }
  if (terms) { terms[0] = Eb; terms[1] = Ea; terms[2] = Et; terms[3] = En; }
  return Eb + Ea + Et + En;
}

/* All components at x: comps = {U_L, U_I, Psi_sg, Psi_g}.  If F is given, it receives the force
 * of the state with grid weights (w_sg, w_g). */
void oracle_energy_force(const oracle_system* s, const double* x, double w_sg, double w_g, double* F,
                         double comps[4]) {
  int n3 = 3 * s->na;
  double* f1 = F ? (double*)malloc(sizeof(double) * (size_t)n3) : NULL;
  double* f2 = F ? (double*)malloc(sizeof(double) * (size_t)n3) : NULL;
  double* gs = F ? (double*)malloc(sizeof(double) * (size_t)n3) : NULL;
  double* gg = F ? (double*)malloc(sizeof(double) * (size_t)n3) : NULL;
  double psi[2];
  comps[0] = oracle_ligand_ff(s, x, f1, NULL);
  comps[1] = oracle_restraint(s, x, f2);
  oracle_grid_terms(s, x, psi, gs, gg);
  comps[2] = psi[0];
  comps[3] = psi[1];
  if (F) {
    /* a zero weight means the term is absent (it is not evaluated as 0 * Psi) */
    for (int i = 0; i < n3; ++i) {
      double f = f1[i] + f2[i];
      if (w_sg != 0.0) f -= w_sg * gs[i];
      if (w_g != 0.0) f -= w_g * gg[i];
      F[i] = f;
    }
    free(f1); free(f2); free(gs); free(gg);
  }
}

/* Reduced potential of components c at a state: beta * (((U_L + U_I) + w_sg Psi_sg) + w_g Psi_g),
 * a term with weight exactly 0 omitted. */
static double weighted_energy(double w_sg, double w_g, const double* c) {
  double e = c[0] + c[1];
  if (w_sg != 0.0) e = e + w_sg * c[2];
  if (w_g != 0.0) e = e + w_g * c[3];
  return e;
}
static double reduced(double beta, double w_sg, double w_g, const double* c) {
  return beta * weighted_energy(w_sg, w_g, c);
}

/* ---------------------------------------------------------------- velocity Verlet */
/* n_steps of velocity Verlet at fixed grid weights: v += dt/2 F/m; x += dt v; F(x); v += dt/2 F/m.
 * x, v in place (A, A/fs); H[0..n_steps] (may be NULL) receives K + U after each step, H[0] before
 * the first.  This is the integrator inside the HMC trial ("Sampling"). */
void oracle_vv(const oracle_system* s, double* x, double* v, double w_sg, double w_g, double dt, int n_steps,
               double* H) {
  int na = s->na, n3 = 3 * na;
  double* F = (double*)malloc(sizeof(double) * (size_t)n3);
  double c[4];
  oracle_energy_force(s, x, w_sg, w_g, F, c);
  for (int st = 0; st <= n_steps; ++st) {
    if (st > 0) {
      for (int i = 0; i < na; ++i)
        for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * 4.184e-4 / s->mass[i];
      for (int j = 0; j < n3; ++j) x[j] += dt * v[j];
      oracle_energy_force(s, x, w_sg, w_g, F, c);
      for (int i = 0; i < na; ++i)
        for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * 4.184e-4 / s->mass[i];
    }
    if (H) {
      double Kin = 0.0;
      for (int i = 0; i < na; ++i)
        for (int d = 0; d < 3; ++d) Kin += 0.5 * s->mass[i] * v[3 * i + d] * v[3 * i + d] * O_MV2_TO_KCAL;
      H[st] = Kin + weighted_energy(w_sg, w_g, c);
    }
  }
  free(F);
}

/* ---------------------------------------------------------------- HMC */
typedef struct {
  const oracle_system* s;
  int64_t begin, end;
  const int* state_of;
  int64_t rep_offset;
  double* x;
  double* comps;
  double* dH;
  unsigned char* acc;
  int n_steps;
  uint64_t seed, cycle;
} hmc_job;

/* One HMC trial per replica: momenta ~ N(0, kT/m), n_steps of velocity Verlet, then Metropolis on
 * the total energy H = K + U_k.  Replica r draws from Philox counters
 * {atom, r, cycle, MOMENTUM} (three normals per atom from one block) and {0, r, cycle, ACCEPT}. */
static void hmc_one(const oracle_system* s, int64_t r, const hmc_job* J) {
  int na = s->na, n3 = 3 * na;
  int k = J->state_of[r];
  double kT = O_KB * s->T[k];
  double dt = s->dt[k];
  double wsg = s->w_sg[k], wg = s->w_g[k];
  double* x = J->x + (int64_t)n3 * r;
  double* x0 = (double*)malloc(sizeof(double) * (size_t)n3);
  double* v = (double*)malloc(sizeof(double) * (size_t)n3);
  double* F = (double*)malloc(sizeof(double) * (size_t)n3);
  memcpy(x0, x, sizeof(double) * (size_t)n3);
  double c0[4], c1[4];
  oracle_energy_force(s, x, wsg, wg, F, c0);
  uint32_t rid = (uint32_t)(J->rep_offset + r);
  double K0 = 0.0;
  for (int i = 0; i < na; ++i) {
    uint32_t o[4];
    philox(J->seed, (uint32_t)i, rid, (uint32_t)J->cycle, O_PURPOSE_MOMENTUM, o);
    double z0, z1, z2, z3;
    box_muller(o[0], o[1], &z0, &z1);
    box_muller(o[2], o[3], &z2, &z3);
    double sd = sqrt(kT * 4.184e-4 / s->mass[i]);
    v[3 * i] = z0 * sd;
    v[3 * i + 1] = z1 * sd;
    v[3 * i + 2] = z2 * sd;
    for (int d = 0; d < 3; ++d) K0 += 0.5 * s->mass[i] * v[3 * i + d] * v[3 * i + d] * O_MV2_TO_KCAL;
  }
  double U0 = weighted_energy(wsg, wg, c0);
  for (int st = 0; st < J->n_steps; ++st) {
    for (int i = 0; i < na; ++i)
      for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * 4.184e-4 / s->mass[i];
    for (int j = 0; j < n3; ++j) x[j] += dt * v[j];
    oracle_energy_force(s, x, wsg, wg, F, c1);
    for (int i = 0; i < na; ++i)
      for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * dt * F[3 * i + d] * 4.184e-4 / s->mass[i];
  }
  if (J->n_steps == 0) memcpy(c1, c0, sizeof(c0));
  double K1 = 0.0;
  for (int i = 0; i < na; ++i)
    for (int d = 0; d < 3; ++d) K1 += 0.5 * s->mass[i] * v[3 * i + d] * v[3 * i + d] * O_MV2_TO_KCAL;
  double U1 = weighted_energy(wsg, wg, c1);
  double dH = (K1 + U1) - (K0 + U0);
  uint32_t o[4];
  philox(J->seed, 0u, rid, (uint32_t)J->cycle, O_PURPOSE_ACCEPT, o);
  double u = oracle_u53(o[0], o[1]);
  int accept = u < exp(-dH / kT);
  if (!accept) {
    memcpy(x, x0, sizeof(double) * (size_t)n3);
    memcpy(c1, c0, sizeof(c0));
  }
  if (J->comps) memcpy(J->comps + 4 * r, c1, sizeof(c1));
  if (J->dH) J->dH[r] = dH;
  if (J->acc) J->acc[r] = (unsigned char)accept;
  free(x0); free(v); free(F);
}

static void* hmc_worker(void* arg) {
  hmc_job* J = (hmc_job*)arg;
  for (int64_t r = J->begin; r < J->end; ++r) hmc_one(J->s, r, J);
  return NULL;
}

/* Returns the number of threads used. */
int oracle_hmc(const oracle_system* s, int64_t n_rep, const int* state_of, int64_t rep_offset, double* x,
               double* comps, double* dH, unsigned char* acc, int n_steps, uint64_t seed, uint64_t cycle,
               int n_threads) {
  int T = n_threads_default(n_threads);
  if (T > n_rep) T = n_rep > 0 ? (int)n_rep : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)T);
  hmc_job* jobs = (hmc_job*)malloc(sizeof(hmc_job) * (size_t)T);
  for (int t = 0; t < T; ++t) {
    hmc_job J = {s, n_rep * t / T, n_rep * (t + 1) / T, state_of, rep_offset, x, comps, dH, acc, n_steps,
                 seed, cycle};
    jobs[t] = J;
    pthread_create(&th[t], NULL, hmc_worker, &jobs[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  free(th); free(jobs);
  return T;
}

/* ---------------------------------------------------------------- replica exchange */
/* Sweeps of Hamiltonian replica exchange on each ladder, Eq. (repXacc).  config_of[l*K + k] is the
 * slot (row of comps) whose configuration is at state k of ladder l; comps[(l*K + i)*4 + c] are the
 * components of slot i.  One sweep: for separations s = 1..min(max_sep, K-1), colour 0 then 1,
 * attempt every pair (a, a+s) with floor(a/s) % 2 == colour (pairs of one colour are disjoint).
 * The uniform of attempt (sweep, s, a) comes from Philox counter
 * {(sweep*max_sep + s-1)*65536 + a, ladder_offset + l, cycle, EXCHANGE}.
 * attempts / accepts are [max_sep][K] counters indexed by (s-1, a), accumulated. */
void oracle_exchange(int n_ladders, int K, const double* T, const double* alpha, const double* comps,
                     int* config_of, int n_sweeps, int max_sep, uint64_t seed, uint64_t cycle,
                     int64_t ladder_offset, int64_t* attempts, int64_t* accepts) {
  double* beta = (double*)malloc(sizeof(double) * (size_t)K);
  double* wsg = (double*)malloc(sizeof(double) * (size_t)K);
  double* wg = (double*)malloc(sizeof(double) * (size_t)K);
  double* u = (double*)malloc(sizeof(double) * (size_t)K * (size_t)K);
  for (int k = 0; k < K; ++k) { beta[k] = oracle_beta(T[k]); wsg[k] = oracle_alpha_sg(alpha[k]); wg[k] = oracle_alpha_g(alpha[k]); }
  int smax = max_sep < K - 1 ? max_sep : K - 1;
  for (int l = 0; l < n_ladders; ++l) {
    const double* C = comps + (int64_t)l * K * 4;
    int* cfg = config_of + (int64_t)l * K;
    for (int k = 0; k < K; ++k)
      for (int i = 0; i < K; ++i) u[k * K + i] = reduced(beta[k], wsg[k], wg[k], C + 4 * i);
    for (int sw = 0; sw < n_sweeps; ++sw)
      for (int sep = 1; sep <= smax; ++sep)
        for (int colour = 0; colour < 2; ++colour)
          for (int a = 0; a + sep < K; ++a) {
            if ((a / sep) % 2 != colour) continue;
            int b = a + sep;
            int xi = cfg[a], yi = cfg[b];
            double d = u[a * K + yi] + u[b * K + xi];
            d = d - u[a * K + xi];
            d = d - u[b * K + yi];
            uint32_t o[4];
            philox(seed, (uint32_t)((sw * max_sep + sep - 1) * 65536 + a), (uint32_t)(ladder_offset + l),
                   (uint32_t)cycle, O_PURPOSE_EXCHANGE, o);
            double un = oracle_u53(o[0], o[1]);
            if (attempts) attempts[(int64_t)(sep - 1) * K + a] += 1;
            if (un < exp(-d)) {
              cfg[a] = yi;
              cfg[b] = xi;
              if (accepts) accepts[(int64_t)(sep - 1) * K + a] += 1;
            }
          }
  }
  free(beta); free(wsg); free(wg); free(u);
}

/* ---------------------------------------------------------------- u_kn */
/* Components of N configurations (energy only) and u_kn[k*N + n] for every state of the system. */
void oracle_reduced_energies(const oracle_system* s, int64_t N, const double* x, double* u_kn, double* comps) {
  for (int64_t n = 0; n < N; ++n) {
    double c[4];
    oracle_energy_force(s, x + (int64_t)3 * s->na * n, 0.0, 0.0, NULL, c);
    if (comps) memcpy(comps + 4 * n, c, sizeof(c));
    if (u_kn)
      for (int k = 0; k < s->K; ++k) u_kn[(int64_t)k * N + n] = reduced(s->beta[k], s->w_sg[k], s->w_g[k], c);
  }
}

/* u_kn from stored components for an explicit state table. */
void oracle_ukn_from_comps(int K, const double* T, const double* alpha, int64_t N, const double* comps,
                           double* u_kn) {
  for (int k = 0; k < K; ++k) {
    double b = oracle_beta(T[k]), ws = oracle_alpha_sg(alpha[k]), wg = oracle_alpha_g(alpha[k]);
    for (int64_t n = 0; n < N; ++n) u_kn[(int64_t)k * N + n] = reduced(b, ws, wg, comps + 4 * n);
  }
}

/* ---------------------------------------------------------------- MBAR */
/* Self-consistent MBAR iteration (Shirts & Chodera 2008), in log-sum-exp form:
 *   log D_n  = ln sum_k N_k exp(f_k - u_kn)
 *   f_i_new  = -ln sum_n exp(-u_in - log D_n),   then f_new -= f_new[0]
 * starting from f = 0, until max_i |f_new - f| < tol.  Returns iterations used, or -1 if max_iter
 * was reached (f then holds the last iterate). */
int oracle_mbar(int K, int64_t N, const double* u_kn, const int64_t* N_k, double tol, int max_iter, double* f) {
  double* logD = (double*)malloc(sizeof(double) * (size_t)N);
  double* fn = (double*)malloc(sizeof(double) * (size_t)K);
  for (int k = 0; k < K; ++k) f[k] = 0.0;
  int result = -1;
  for (int it = 1; it <= max_iter; ++it) {
    for (int64_t n = 0; n < N; ++n) {
      double m = -INFINITY;
      for (int k = 0; k < K; ++k) {
        if (N_k[k] == 0) continue;
        double a = log((double)N_k[k]) + f[k] - u_kn[(int64_t)k * N + n];
        if (a > m) m = a;
      }
      double sum = 0.0;
      for (int k = 0; k < K; ++k) {
        if (N_k[k] == 0) continue;
        sum += exp(log((double)N_k[k]) + f[k] - u_kn[(int64_t)k * N + n] - m);
      }
      logD[n] = m + log(sum);
    }
    for (int i = 0; i < K; ++i) {
      double m = -INFINITY;
      for (int64_t n = 0; n < N; ++n) {
        double a = -u_kn[(int64_t)i * N + n] - logD[n];
        if (a > m) m = a;
      }
      double sum = 0.0;
      for (int64_t n = 0; n < N; ++n) sum += exp(-u_kn[(int64_t)i * N + n] - logD[n] - m);
      fn[i] = -(m + log(sum));
    }
    double f0 = fn[0], delta = 0.0;
    for (int i = 0; i < K; ++i) {
      fn[i] -= f0;
      double dd = fabs(fn[i] - f[i]);
      if (dd > delta) delta = dd;
      f[i] = fn[i];
    }
    if (delta < tol) { result = it; break; }
  }
  free(logD);
  free(fn);
  return result;
}

/* ---------------------------------------------------------------- statistical inefficiency */
/* g = 1 + 2 sum_{t=1}^{N-1} (1 - t/N) C(t), C the normalised autocorrelation of a, summed until
 * C(t) first drops to zero or below; g >= 1.  Effective samples N/g. */
double oracle_statistical_inefficiency(int64_t N, const double* a) {
  if (N < 2) return 1.0;
  double mu = 0.0;
  for (int64_t i = 0; i < N; ++i) mu += a[i];
  mu /= (double)N;
  double var = 0.0;
  for (int64_t i = 0; i < N; ++i) var += (a[i] - mu) * (a[i] - mu);
  var /= (double)N;
  if (var == 0.0) return 1.0;
  double g = 1.0;
  for (int64_t t = 1; t < N; ++t) {
    double c = 0.0;
    for (int64_t i = 0; i + t < N; ++i) c += (a[i] - mu) * (a[i + t] - mu);
    c /= (double)(N - t) * var;
    if (c <= 0.0) break;
    g += 2.0 * c * (1.0 - (double)t / (double)N);
  }
  return g < 1.0 ? 1.0 : g;
}

/* ================================================================ learned pose proposal
 * Not a step of the paper: a learned proposal of rigid-body and torsion moves, made exact by the
 * Metropolis-Hastings test of an involution.  It generalises the paper's external-coordinate moves
 * ("Sampling": a random rotation about the centre of mass and a Gaussian translation).
 *
 *  torsion tree   root atom 0; a bond is rotatable if both its atoms have two or more neighbours;
 *                 the first 16 rotatable bonds (bond-list order) are moved; each moves the atoms
 *                 on its side away from the root, about the axis proximal -> distal atom.
 *  move           Apply(x, d) = Rigid(d_r / 2) o Tor(d_tau) o Rigid(d_r / 2), Rigid(t, w) = rotate
 *                 about the centre of mass by exp(w) (axis-angle), then translate by t.  Torsion
 *                 rotations commute (each changes one dihedral, the root side fixed), so
 *                 Apply(Apply(x, d), -d) = x; every factor preserves volume (unit Jacobian).
 *  network        64 features -> 256 -> 256 -> 256 (ReLU) -> 360 outputs: an 8-component diagonal
 *                 Gaussian mixture over d = (t[3] A, w[3] rad, d_tau[T] rad); log sigma =
 *                 -2 + 4 tanh(raw / 4).
 *  acceptance     min(1, exp(-(u(x') - u(x))) q(-d | x') / q(d | x)).
 * Random numbers: Philox counter {draw, replica, cycle * n_moves + move, 4}: draw d < 22 gives the
 * normal of dimension d (first Box-Muller output), draw 100 the component uniform, draw 101 the
 * acceptance uniform. */
#define O_TMAX 16
#define O_NFEAT 64
#define O_NCOMP 8
#define O_DMAX (6 + O_TMAX)
#define O_NOUT (O_NCOMP * (1 + 2 * O_DMAX))
#define O_HID 256
enum { O_PURPOSE_LEARNED = 4 };

typedef struct {
  int T;
  int prox[O_TMAX], dist[O_TMAX];
  int dih[O_TMAX][4];
  unsigned char* moved; /* [T][na] */
} o_tree;

static void o_tree_build(const oracle_system* s, o_tree* t) {
  int na = s->na;
  int* deg = (int*)calloc((size_t)(na > 0 ? na : 1), sizeof(int));
  for (int b = 0; b < s->nb; ++b) { deg[s->bonds[2 * b]]++; deg[s->bonds[2 * b + 1]]++; }
  t->T = 0;
  t->moved = (unsigned char*)calloc((size_t)O_TMAX * (size_t)(na > 0 ? na : 1), 1);
  int* seen = (int*)malloc(sizeof(int) * (size_t)(na > 0 ? na : 1));
  int* queue = (int*)malloc(sizeof(int) * (size_t)(na > 0 ? na : 1));
  for (int b = 0; b < s->nb && t->T < O_TMAX; ++b) {
    int j = s->bonds[2 * b], k = s->bonds[2 * b + 1];
    if (deg[j] < 2 || deg[k] < 2) continue;
    /* atoms reachable from the root without crossing bond b */
    for (int i = 0; i < na; ++i) seen[i] = 0;
    int h = 0, tl = 0;
    seen[0] = 1;
    queue[tl++] = 0;
    while (h < tl) {
      int u = queue[h++];
      for (int c = 0; c < s->nb; ++c) {
        if (c == b) continue;
        int v = -1;
        if (s->bonds[2 * c] == u) v = s->bonds[2 * c + 1];
        else if (s->bonds[2 * c + 1] == u) v = s->bonds[2 * c];
        if (v >= 0 && !seen[v]) { seen[v] = 1; queue[tl++] = v; }
      }
    }
    int prox = seen[j] ? j : k, dist = seen[j] ? k : j;
    int T = t->T;
    t->prox[T] = prox;
    t->dist[T] = dist;
    for (int i = 0; i < na; ++i) t->moved[(size_t)T * na + i] = (unsigned char)(seen[i] ? 0 : 1);
    t->moved[(size_t)T * na + dist] = 0; /* on the axis */
    int ii = -1, ll = -1;
    for (int c = 0; c < s->nb; ++c) {
      int a0 = s->bonds[2 * c], a1 = s->bonds[2 * c + 1];
      int v;
      if (a0 == prox || a1 == prox) {
        v = a0 == prox ? a1 : a0;
        if (v != dist && (ii < 0 || v < ii)) ii = v;
      }
      if (a0 == dist || a1 == dist) {
        v = a0 == dist ? a1 : a0;
        if (v != prox && (ll < 0 || v < ll)) ll = v;
      }
    }
    t->dih[T][0] = ii; t->dih[T][1] = prox; t->dih[T][2] = dist; t->dih[T][3] = ll;
    t->T++;
  }
  free(deg); free(seen); free(queue);
}

int oracle_learned_ntorsions(const oracle_system* s) {
  o_tree t;
  o_tree_build(s, &t);
  free(t.moved);
  return t.T;
}

static double o_dihedral(const double* x, const int* a) {
  double b1[3], b2[3], b3[3], n1[3], n2[3];
  sub3(x + 3 * a[1], x + 3 * a[0], b1);
  sub3(x + 3 * a[2], x + 3 * a[1], b2);
  sub3(x + 3 * a[3], x + 3 * a[2], b3);
  cross3(b1, b2, n1);
  cross3(b2, b3, n2);
  return atan2(sqrt(dot3(b2, b2)) * dot3(b1, n2), dot3(n1, n2));
}

static void o_com(const oracle_system* s, const double* x, double c[3]) {
  double M = 0.0;
  c[0] = c[1] = c[2] = 0.0;
  for (int i = 0; i < s->na; ++i) {
    M += s->mass[i];
    for (int d = 0; d < 3; ++d) c[d] += s->mass[i] * x[3 * i + d];
  }
  for (int d = 0; d < 3; ++d) c[d] /= M;
}

/* Features of a pose at state k (comps = {U_L, U_I, Psi_sg, Psi_g} of x). */
void oracle_features(const oracle_system* s, const double* x, const double comps[4], int k, double* f) {
  o_tree t;
  o_tree_build(s, &t);
  for (int i = 0; i < O_NFEAT; ++i) f[i] = 0.0;
  double c[3];
  o_com(s, x, c);
  for (int d = 0; d < 3; ++d) f[d] = (c[d] - s->site[d]) / s->d0;
  int ref[2] = {0, s->na - 1};
  for (int r = 0; r < 2; ++r) {
    double v[3];
    sub3(x + 3 * ref[r], c, v);
    double n = sqrt(dot3(v, v));
    if (n < 1e-6) n = 1e-6;
    for (int d = 0; d < 3; ++d) f[3 + 3 * r + d] = v[d] / n;
  }
  for (int q = 0; q < t.T; ++q) {
    double tau = o_dihedral(x, t.dih[q]);
    f[9 + 2 * q] = cos(tau);
    f[10 + 2 * q] = sin(tau);
  }
  f[41] = s->w_sg[k];
  f[42] = s->w_g[k];
  f[43] = 300.0 / s->T[k];
  for (int i = 0; i < 4; ++i) f[44 + i] = asinh(comps[i] / 10.0);
  free(t.moved);
}

static void o_rotate(double* v, const double w[3]) {
  /* v <- exp([w]x) v (Rodrigues) */
  double th = sqrt(dot3(w, w));
  double a, b;
  if (th < 1e-8) { a = 1.0 - th * th / 6.0; b = 0.5 - th * th / 24.0; }
  else { a = sin(th) / th; b = (1.0 - cos(th)) / (th * th); }
  double wv[3], wwv[3];
  cross3(w, v, wv);
  cross3(w, wv, wwv);
  for (int d = 0; d < 3; ++d) v[d] = v[d] + a * wv[d] + b * wwv[d];
}

static void o_rigid(const oracle_system* s, double* x, const double t[3], const double w[3]) {
  double c[3];
  o_com(s, x, c);
  for (int i = 0; i < s->na; ++i) {
    double v[3];
    sub3(x + 3 * i, c, v);
    o_rotate(v, w);
    for (int d = 0; d < 3; ++d) x[3 * i + d] = c[d] + v[d] + t[d];
  }
}

/* y = Apply(x, d), d = (t[3], w[3], d_tau[T]). */
void oracle_apply(const oracle_system* s, const double* x, const double* dl, double* y) {
  o_tree t;
  o_tree_build(s, &t);
  memcpy(y, x, sizeof(double) * 3 * (size_t)s->na);
  double ht[3] = {0.5 * dl[0], 0.5 * dl[1], 0.5 * dl[2]}, hw[3] = {0.5 * dl[3], 0.5 * dl[4], 0.5 * dl[5]};
  o_rigid(s, y, ht, hw);
  for (int q = 0; q < t.T; ++q) {
    double ax[3];
    sub3(y + 3 * t.dist[q], y + 3 * t.prox[q], ax);
    double n = sqrt(dot3(ax, ax));
    double w[3] = {ax[0] / n * dl[6 + q], ax[1] / n * dl[6 + q], ax[2] / n * dl[6 + q]};
    const double* p = y + 3 * t.prox[q];
    double pc[3] = {p[0], p[1], p[2]};
    for (int i = 0; i < s->na; ++i) {
      if (!t.moved[(size_t)q * s->na + i]) continue;
      double v[3];
      sub3(y + 3 * i, pc, v);
      o_rotate(v, w);
      for (int d = 0; d < 3; ++d) y[3 * i + d] = pc[d] + v[d];
    }
  }
  o_rigid(s, y, ht, hw);
  free(t.moved);
}

/* Training target: the move taking pose x to pose y (translation of the centre of mass, rotation
 * of the frame of reference atoms 0 and n-1, wrapped torsion differences). */
void oracle_pose_delta(const oracle_system* s, const double* x, const double* y, double* dl) {
  o_tree t;
  o_tree_build(s, &t);
  double cx[3], cy[3];
  o_com(s, x, cx);
  o_com(s, y, cy);
  for (int d = 0; d < 3; ++d) dl[d] = cy[d] - cx[d];
  double F[2][3][3];
  const double* P[2] = {x, y};
  const double* C[2] = {cx, cy};
  for (int p = 0; p < 2; ++p) {
    double e1[3], e2[3], e3[3];
    sub3(P[p] + 0, C[p], e1);
    double n = sqrt(dot3(e1, e1));
    if (n < 1e-9) { e1[0] = 1; e1[1] = 0; e1[2] = 0; n = 1; }
    for (int d = 0; d < 3; ++d) e1[d] /= n;
    sub3(P[p] + 3 * (s->na - 1), C[p], e2);
    double pr = dot3(e2, e1);
    for (int d = 0; d < 3; ++d) e2[d] -= pr * e1[d];
    n = sqrt(dot3(e2, e2));
    if (n < 1e-9) { double a[3] = {0, 0, 1}; if (fabs(e1[2]) > 0.9) { a[1] = 1; a[2] = 0; } cross3(e1, a, e2); n = sqrt(dot3(e2, e2)); }
    for (int d = 0; d < 3; ++d) e2[d] /= n;
    cross3(e1, e2, e3);
    for (int d = 0; d < 3; ++d) { F[p][d][0] = e1[d]; F[p][d][1] = e2[d]; F[p][d][2] = e3[d]; }
  }
  double R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      R[a][b] = 0.0;
      for (int c = 0; c < 3; ++c) R[a][b] += F[1][a][c] * F[0][b][c];
    }
  double tr = R[0][0] + R[1][1] + R[2][2];
  double ct = 0.5 * (tr - 1.0);
  if (ct > 1.0) ct = 1.0;
  if (ct < -1.0) ct = -1.0;
  double th = acos(ct);
  double v[3] = {R[2][1] - R[1][2], R[0][2] - R[2][0], R[1][0] - R[0][1]};
  double sn = sin(th);
  double f = th < 1e-8 ? 0.5 : (sn > 1e-8 ? th / (2.0 * sn) : 0.0);
  if (th > 1e-8 && sn <= 1e-8) { /* rotation by pi: axis from the symmetric part */
    double ax[3] = {sqrt(fmax(0.0, 0.5 * (R[0][0] + 1))), sqrt(fmax(0.0, 0.5 * (R[1][1] + 1))),
                    sqrt(fmax(0.0, 0.5 * (R[2][2] + 1)))};
    if (R[0][1] < 0) ax[1] = -ax[1];
    if (R[0][2] < 0) ax[2] = -ax[2];
    for (int d = 0; d < 3; ++d) dl[3 + d] = th * ax[d];
  } else {
    for (int d = 0; d < 3; ++d) dl[3 + d] = f * v[d];
  }
  for (int q = 0; q < t.T; ++q) {
    double d = o_dihedral(y, t.dih[q]) - o_dihedral(x, t.dih[q]);
    while (d > M_PI) d -= 2.0 * M_PI;
    while (d <= -M_PI) d += 2.0 * M_PI;
    dl[6 + q] = d;
  }
  free(t.moved);
}

/* ---------------- MLP (weights row-major [out][in]); activations kept for the backward pass */
static void o_dense(int B, int nin, int nout, const double* W, const double* b, const double* X, double* Y, int relu) {
  for (int r = 0; r < B; ++r)
    for (int o = 0; o < nout; ++o) {
      double acc = b[o];
      for (int i = 0; i < nin; ++i) acc += W[(size_t)o * nin + i] * X[(size_t)r * nin + i];
      Y[(size_t)r * nout + o] = relu ? (acc > 0.0 ? acc : 0.0) : acc;
    }
}

/* With BF16 emulation on, the network's input and hidden activations are rounded to BF16 (round
 * to nearest even), as a BF16 tensor-core implementation stores them; off (the default), FP64. */
static int o_bf16_act = 0;
void oracle_set_bf16_activations(int on) { o_bf16_act = on; }

static double o_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
  }
  memcpy(&f, &u, 4);
  return (double)f;
}

void oracle_mlp_forward(const double* W1, const double* b1, const double* W2, const double* b2, const double* W3,
                        const double* b3, const double* W4, const double* b4, int B, const double* X, double* out,
                        double* h1, double* h2, double* h3) {
  double* a1 = h1 ? h1 : (double*)malloc(sizeof(double) * (size_t)B * O_HID);
  double* a2 = h2 ? h2 : (double*)malloc(sizeof(double) * (size_t)B * O_HID);
  double* a3 = h3 ? h3 : (double*)malloc(sizeof(double) * (size_t)B * O_HID);
  const double* in = X;
  double* xr = NULL;
  if (o_bf16_act) {
    xr = (double*)malloc(sizeof(double) * (size_t)B * O_NFEAT);
    for (size_t i = 0; i < (size_t)B * O_NFEAT; ++i) xr[i] = o_bf16(X[i]);
    in = xr;
  }
  o_dense(B, O_NFEAT, O_HID, W1, b1, in, a1, 1);
  if (o_bf16_act) for (size_t i = 0; i < (size_t)B * O_HID; ++i) a1[i] = o_bf16(a1[i]);
  o_dense(B, O_HID, O_HID, W2, b2, a1, a2, 1);
  if (o_bf16_act) for (size_t i = 0; i < (size_t)B * O_HID; ++i) a2[i] = o_bf16(a2[i]);
  o_dense(B, O_HID, O_HID, W3, b3, a2, a3, 1);
  if (o_bf16_act) for (size_t i = 0; i < (size_t)B * O_HID; ++i) a3[i] = o_bf16(a3[i]);
  o_dense(B, O_HID, O_NOUT, W4, b4, a3, out, 0);
  free(xr);
  if (!h1) free(a1);
  if (!h2) free(a2);
  if (!h3) free(a3);
}

/* Gradients (summed over the batch) of sum_r <dout_r, out_r> with respect to all parameters. */
void oracle_mlp_backward(const double* W2, const double* W3, const double* W4, int B, const double* X,
                         const double* h1, const double* h2, const double* h3, const double* dout, double* gW1,
                         double* gb1, double* gW2, double* gb2, double* gW3, double* gb3, double* gW4,
                         double* gb4) {
  double* d3 = (double*)calloc((size_t)B * O_HID, sizeof(double));
  double* d2 = (double*)calloc((size_t)B * O_HID, sizeof(double));
  double* d1 = (double*)calloc((size_t)B * O_HID, sizeof(double));
  memset(gW1, 0, sizeof(double) * O_HID * O_NFEAT); memset(gb1, 0, sizeof(double) * O_HID);
  memset(gW2, 0, sizeof(double) * O_HID * O_HID); memset(gb2, 0, sizeof(double) * O_HID);
  memset(gW3, 0, sizeof(double) * O_HID * O_HID); memset(gb3, 0, sizeof(double) * O_HID);
  memset(gW4, 0, sizeof(double) * O_NOUT * O_HID); memset(gb4, 0, sizeof(double) * O_NOUT);
  for (int r = 0; r < B; ++r) {
    const double* g = dout + (size_t)r * O_NOUT;
    for (int o = 0; o < O_NOUT; ++o) {
      gb4[o] += g[o];
      for (int i = 0; i < O_HID; ++i) gW4[(size_t)o * O_HID + i] += g[o] * h3[(size_t)r * O_HID + i];
    }
    for (int i = 0; i < O_HID; ++i) {
      double acc = 0.0;
      for (int o = 0; o < O_NOUT; ++o) acc += g[o] * W4[(size_t)o * O_HID + i];
      d3[(size_t)r * O_HID + i] = h3[(size_t)r * O_HID + i] > 0.0 ? acc : 0.0;
    }
    const double* g3 = d3 + (size_t)r * O_HID;
    for (int o = 0; o < O_HID; ++o) {
      gb3[o] += g3[o];
      for (int i = 0; i < O_HID; ++i) gW3[(size_t)o * O_HID + i] += g3[o] * h2[(size_t)r * O_HID + i];
    }
    for (int i = 0; i < O_HID; ++i) {
      double acc = 0.0;
      for (int o = 0; o < O_HID; ++o) acc += g3[o] * W3[(size_t)o * O_HID + i];
      d2[(size_t)r * O_HID + i] = h2[(size_t)r * O_HID + i] > 0.0 ? acc : 0.0;
    }
    const double* g2 = d2 + (size_t)r * O_HID;
    for (int o = 0; o < O_HID; ++o) {
      gb2[o] += g2[o];
      for (int i = 0; i < O_HID; ++i) gW2[(size_t)o * O_HID + i] += g2[o] * h1[(size_t)r * O_HID + i];
    }
    for (int i = 0; i < O_HID; ++i) {
      double acc = 0.0;
      for (int o = 0; o < O_HID; ++o) acc += g2[o] * W2[(size_t)o * O_HID + i];
      d1[(size_t)r * O_HID + i] = h1[(size_t)r * O_HID + i] > 0.0 ? acc : 0.0;
    }
    const double* g1 = d1 + (size_t)r * O_HID;
    for (int o = 0; o < O_HID; ++o) {
      gb1[o] += g1[o];
      for (int i = 0; i < O_NFEAT; ++i) gW1[(size_t)o * O_NFEAT + i] += g1[o] * X[(size_t)r * O_NFEAT + i];
    }
  }
  free(d1); free(d2); free(d3);
}

/* log q(d) of the mixture encoded by one output row o[360], over the first D dimensions; g (may be
 * NULL) receives d log q / d o. */
double oracle_mixture_logq(const double* o, int D, const double* dl, double* g) {
  double lw[O_NCOMP], lp[O_NCOMP];
  double m = -INFINITY;
  for (int c = 0; c < O_NCOMP; ++c) if (o[c] > m) m = o[c];
  double z = 0.0;
  for (int c = 0; c < O_NCOMP; ++c) z += exp(o[c] - m);
  double lz = m + log(z);
  for (int c = 0; c < O_NCOMP; ++c) {
    lw[c] = o[c] - lz;
    double s = lw[c];
    for (int d = 0; d < D; ++d) {
      double mu = o[O_NCOMP + c * O_DMAX + d];
      double ls = -2.0 + 4.0 * tanh(o[O_NCOMP + O_NCOMP * O_DMAX + c * O_DMAX + d] / 4.0);
      double zz = (dl[d] - mu) / exp(ls);
      s += -0.5 * zz * zz - ls - 0.5 * log(2.0 * M_PI);
    }
    lp[c] = s;
  }
  double mm = -INFINITY;
  for (int c = 0; c < O_NCOMP; ++c) if (lp[c] > mm) mm = lp[c];
  double ss = 0.0;
  for (int c = 0; c < O_NCOMP; ++c) ss += exp(lp[c] - mm);
  double lq = mm + log(ss);
  if (g) {
    for (int i = 0; i < O_NOUT; ++i) g[i] = 0.0;
    for (int c = 0; c < O_NCOMP; ++c) {
      double r = exp(lp[c] - lq);
      g[c] += r;
      for (int c2 = 0; c2 < O_NCOMP; ++c2) g[c2] -= r * exp(lw[c2]);
      for (int d = 0; d < D; ++d) {
        double mu = o[O_NCOMP + c * O_DMAX + d];
        double raw = o[O_NCOMP + O_NCOMP * O_DMAX + c * O_DMAX + d];
        double th = tanh(raw / 4.0);
        double ls = -2.0 + 4.0 * th;
        double sg = exp(ls);
        double zz = (dl[d] - mu) / sg;
        g[O_NCOMP + c * O_DMAX + d] += r * zz / sg;
        g[O_NCOMP + O_NCOMP * O_DMAX + c * O_DMAX + d] += r * (zz * zz - 1.0) * (1.0 - th * th);
      }
    }
  }
  return lq;
}

/* Draw d ~ q(. | o) with the replica's Philox stream. */
void oracle_mixture_sample(const double* o, int D, uint64_t seed, uint32_t rep, uint32_t ctr, double* dl) {
  double m = -INFINITY;
  for (int c = 0; c < O_NCOMP; ++c) if (o[c] > m) m = o[c];
  double w[O_NCOMP], z = 0.0;
  for (int c = 0; c < O_NCOMP; ++c) { w[c] = exp(o[c] - m); z += w[c]; }
  uint32_t r4[4];
  philox(seed, 100u, rep, ctr, O_PURPOSE_LEARNED, r4);
  double u = oracle_u53(r4[0], r4[1]) * z;
  int comp = O_NCOMP - 1;
  double cum = 0.0;
  for (int c = 0; c < O_NCOMP; ++c) {
    cum += w[c];
    if (u < cum) { comp = c; break; }
  }
  for (int d = 0; d < D; ++d) {
    philox(seed, (uint32_t)d, rep, ctr, O_PURPOSE_LEARNED, r4);
    double z0, z1;
    box_muller(r4[0], r4[1], &z0, &z1);
    double mu = o[O_NCOMP + comp * O_DMAX + d];
    double ls = -2.0 + 4.0 * tanh(o[O_NCOMP + O_NCOMP * O_DMAX + comp * O_DMAX + d] / 4.0);
    dl[d] = mu + exp(ls) * z0;
  }
}

/* n_moves learned proposals per replica at its state, each accepted with the involutive MH test.
 * x [R][na][3] and comps [R][4] (components of x) are updated in place; acc [R] counts accepts;
 * logratio [R] (may be NULL) receives the last move's log acceptance ratio. */
void oracle_learned_mh(const oracle_system* s, const double* W1, const double* b1, const double* W2, const double* b2,
                       const double* W3, const double* b3, const double* W4, const double* b4, int64_t n_rep,
                       const int* state_of, int64_t rep_offset, double* x, double* comps, int n_moves,
                       int n_torsions, uint64_t seed, uint64_t cycle, int* acc, double* logratio) {
  /* n_torsions limits the moved torsions to the first min(T, n_torsions) (negative: all); the
   * other increments are zero and the mixture uses 6 + that many dimensions. */
  int na = s->na, T = oracle_learned_ntorsions(s);
  if (n_torsions >= 0 && n_torsions < T) T = n_torsions;
  int D = 6 + T;
  double f[O_NFEAT], o[O_NOUT], dl[O_DMAX], ndl[O_DMAX], c1[4];
  for (int d = 0; d < O_DMAX; ++d) dl[d] = ndl[d] = 0.0;
  double* y = (double*)malloc(sizeof(double) * 3 * (size_t)na);
  for (int64_t r = 0; r < n_rep; ++r) {
    int k = state_of[r];
    double* xr = x + (size_t)3 * na * r;
    double* cr = comps + 4 * r;
    uint32_t rid = (uint32_t)(rep_offset + r);
    acc[r] = 0;
    for (int mv = 0; mv < n_moves; ++mv) {
      uint32_t ctr = (uint32_t)(cycle * (uint64_t)n_moves + (uint64_t)mv);
      oracle_features(s, xr, cr, k, f);
      oracle_mlp_forward(W1, b1, W2, b2, W3, b3, W4, b4, 1, f, o, NULL, NULL, NULL);
      oracle_mixture_sample(o, D, seed, rid, ctr, dl);
      double lqf = oracle_mixture_logq(o, D, dl, NULL);
      oracle_apply(s, xr, dl, y);
      oracle_energy_force(s, y, 0.0, 0.0, NULL, c1);
      oracle_features(s, y, c1, k, f);
      oracle_mlp_forward(W1, b1, W2, b2, W3, b3, W4, b4, 1, f, o, NULL, NULL, NULL);
      for (int d = 0; d < D; ++d) ndl[d] = -dl[d];
      double lqr = oracle_mixture_logq(o, D, ndl, NULL);
      double du = s->beta[k] * (weighted_energy(s->w_sg[k], s->w_g[k], c1) - weighted_energy(s->w_sg[k], s->w_g[k], cr));
      double lr = (lqr - lqf) - du;
      uint32_t r4[4];
      philox(seed, 101u, rid, ctr, O_PURPOSE_LEARNED, r4);
      double u = oracle_u53(r4[0], r4[1]);
      if (logratio) logratio[r] = lr;
      if (u < exp(lr)) {
        memcpy(xr, y, sizeof(double) * 3 * (size_t)na);
        memcpy(cr, c1, sizeof(c1));
        acc[r] += 1;
      }
    }
  }
  free(y);
}

/* ---------------------------------------------------------------- external-coordinate moves
 * "Sampling": for states with alpha below a threshold (the paper: 0.01, on the coupling leg), a
 * move rotates the ligand about its centre of mass by a uniformly random rotation (from a random
 * unit quaternion) and translates it by a Gaussian step (0.6 A per dimension in the paper); the
 * Metropolis criterion on the state's energy accepts it.  The proposal is symmetric, so the test
 * is u < exp(-beta (U_k(x') - U_k(x))).
 *
 * Random numbers: Philox counter {d, replica, cycle * n_moves + move, 5}
 *   d = 0: three 23-bit uniforms (words 0..2) for the quaternion;
 *   d = 1: the translation, Box-Muller on words (0, 1) for x and y, (2, 3) for z;
 *   d = 2: the accept uniform (53 bits from words 0, 1). */
enum { O_PURPOSE_EXTERNAL = 5 };

/* Rotation matrix (row-major) of the unit quaternion made from three uniforms by Shoemake's
 * construction ("Uniform random rotations", Graphics Gems III, 1992), which is uniform over the
 * rotation group. */
void oracle_random_rotation(uint32_t a, uint32_t b, uint32_t c, double R[9]) {
  double u1 = (double)(a >> 9) * (1.0 / 8388608.0);
  double u2 = (double)(b >> 9) * (1.0 / 8388608.0);
  double u3 = (double)(c >> 9) * (1.0 / 8388608.0);
  double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
  double qx = s1 * sin(2.0 * M_PI * u2), qy = s1 * cos(2.0 * M_PI * u2);
  double qz = s2 * sin(2.0 * M_PI * u3), qw = s2 * cos(2.0 * M_PI * u3);
  R[0] = 1.0 - 2.0 * (qy * qy + qz * qz);
  R[1] = 2.0 * (qx * qy - qz * qw);
  R[2] = 2.0 * (qx * qz + qy * qw);
  R[3] = 2.0 * (qx * qy + qz * qw);
  R[4] = 1.0 - 2.0 * (qx * qx + qz * qz);
  R[5] = 2.0 * (qy * qz - qx * qw);
  R[6] = 2.0 * (qx * qz - qy * qw);
  R[7] = 2.0 * (qy * qz + qx * qw);
  R[8] = 1.0 - 2.0 * (qx * qx + qy * qy);
}

/* n_moves external-coordinate moves per replica whose state has alpha < alpha_max (the warming
 * leg's alpha = NaN never qualifies).  x [R][na][3] and comps [R][4] are updated in place; acc [R]
 * counts accepted moves (0 for replicas without moves); logratio [R] (may be NULL) receives the
 * last attempted move's log acceptance ratio -beta dU (0 for replicas without moves). */
void oracle_external_moves(const oracle_system* s, int64_t n_rep, const int* state_of, int64_t rep_offset,
                           double* x, double* comps, int n_moves, double alpha_max, double sigma, uint64_t seed,
                           uint64_t cycle, int* acc, double* logratio) {
  int na = s->na;
  double* y = (double*)malloc(sizeof(double) * 3 * (size_t)na);
  for (int64_t r = 0; r < n_rep; ++r) {
    acc[r] = 0;
    if (logratio) logratio[r] = 0.0;
    int k = state_of[r];
    if (k < 0 || k >= s->K || !(s->alpha[k] < alpha_max)) continue;
    double* xr = x + (size_t)3 * na * r;
    double* cr = comps + 4 * r;
    uint32_t rid = (uint32_t)(rep_offset + r);
    for (int mv = 0; mv < n_moves; ++mv) {
      uint32_t ctr = (uint32_t)(cycle * (uint64_t)n_moves + (uint64_t)mv);
      uint32_t r4[4];
      double R[9], t[3], zz, c[3], c1[4];
      philox(seed, 0u, rid, ctr, O_PURPOSE_EXTERNAL, r4);
      oracle_random_rotation(r4[0], r4[1], r4[2], R);
      philox(seed, 1u, rid, ctr, O_PURPOSE_EXTERNAL, r4);
      box_muller(r4[0], r4[1], &t[0], &t[1]);
      box_muller(r4[2], r4[3], &t[2], &zz);
      for (int d = 0; d < 3; ++d) t[d] *= sigma;
      o_com(s, xr, c);
      for (int i = 0; i < na; ++i) {
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = xr[3 * i + d] - c[d];
        for (int d = 0; d < 3; ++d) y[3 * i + d] = c[d] + (R[3 * d] * v[0] + R[3 * d + 1] * v[1] + R[3 * d + 2] * v[2]) + t[d];
      }
      oracle_energy_force(s, y, 0.0, 0.0, NULL, c1);
      double du = s->beta[k] * (weighted_energy(s->w_sg[k], s->w_g[k], c1) - weighted_energy(s->w_sg[k], s->w_g[k], cr));
      philox(seed, 2u, rid, ctr, O_PURPOSE_EXTERNAL, r4);
      double u = oracle_u53(r4[0], r4[1]);
      if (logratio) logratio[r] = -du;
      if (u < exp(-du)) {
        memcpy(xr, y, sizeof(double) * 3 * (size_t)na);
        memcpy(cr, c1, sizeof(c1));
        acc[r] += 1;
      }
    }
  }
  free(y);
}

/* ---------------------------------------------------------------- equilibration detection
 * "Equilibration and production": the statistical inefficiency g of a series measures how many
 * correlated samples make one independent one.  Automated detection (Chodera 2016, "A simple
 * method for automated equilibration detection in molecular simulations") discards the start t0
 * that maximises the effective sample count of the rest, N_eff(t0) = (T - t0) / g(a[t0:]).
 * Candidates t0 = c * stride, c < n_cand; g_out[c] receives g of each tail; the best t0 (the
 * earliest on ties) and its N_eff are returned. */
void oracle_detect_equilibration(int64_t T, const double* a, int64_t stride, int n_cand, double* g_out,
                                 int64_t* t0_best, double* neff_best) {
  double best = -1.0;
  int64_t bt = 0;
  for (int c = 0; c < n_cand; ++c) {
    int64_t t0 = (int64_t)c * stride;
    double g = oracle_statistical_inefficiency(T - t0, a + t0);
    g_out[c] = g;
    double neff = (double)(T - t0) / g;
    if (neff > best) {
      best = neff;
      bt = t0;
    }
  }
  *t0_best = bt;
  *neff_best = best;
}

/* ---------------------------------------------------------------- protocol initialization
 * "Initialization": states are placed one after another at even steps of thermodynamic length,
 * Delta lambda = s / sigma_0[d l / d lambda], with seeds resampled from the previous state, a time
 * step adapted to the Metropolis acceptance, and a check on the mean exchange probability.  The
 * pieces below are the per-state arithmetic; the driver that runs them in order is in the Python
 * part of the oracle (it samples with oracle_hmc). */

/* Population standard deviations over n samples (components c [n][4]) at state k:
 * out = {sigma[U_L + U_I], sigma[Psi_sg], sigma[Psi_g], sigma[u_k]}, u_k the reduced energy. */
void oracle_state_statistics(const oracle_system* s, int64_t n, const double* comps, int k, double out[4]) {
  double mean[4] = {0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    const double* c = comps + 4 * i;
    double v[4] = {c[0] + c[1], c[2], c[3], reduced(s->beta[k], s->w_sg[k], s->w_g[k], c)};
    for (int q = 0; q < 4; ++q) mean[q] += v[q];
  }
  for (int q = 0; q < 4; ++q) mean[q] /= (double)n;
  double var[4] = {0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    const double* c = comps + 4 * i;
    double v[4] = {c[0] + c[1], c[2], c[3], reduced(s->beta[k], s->w_sg[k], s->w_g[k], c)};
    for (int q = 0; q < 4; ++q) var[q] += (v[q] - mean[q]) * (v[q] - mean[q]);
  }
  for (int q = 0; q < 4; ++q) out[q] = sqrt(var[q] / (double)n);
}

/* Warming leg: l = -U_S/(k_B T) - ln Z, so sigma[dl/dT] = sigma[U_S] / (k_B T^2) and the next
 * temperature is T + speed k_B T^2 / sigma[U_S], not past T_end. */
double oracle_next_temperature(double T, double sigma_U, double speed, double T_end) {
  double Tn = T + speed * O_KB * T * T / sigma_U;
  return Tn > T_end ? T_end : Tn;
}

/* Derivatives of the protocol weights of Eq. (protocol) with respect to alpha. */
static double d_alpha_sg(double a) { return -4.0 * (2.0 * a - 1.0); }
static double d_alpha_g(double a) {
  double s = 2.0 * a - 1.0;
  double z = 1000.0 * (a - 0.5);
  double L = z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
  return 4.0 * s * L + s * s * 1000.0 * L * (1.0 - L);
}

/* Coupling leg, T(alpha) = (T_T - T_H) alpha + T_H: the next alpha is
 * alpha + speed / (|d alpha_sg/d alpha| sigma[Psi_sg] / (k_B T) + |d alpha_g/d alpha| sigma[Psi_g] / (k_B T)
 *                  + |T_T - T_H| sigma[u_alpha] / T), not past 1. */
double oracle_next_alpha(double a, double sigma_sg, double sigma_g, double sigma_u, double speed, double T_T,
                         double T_H) {
  double T = (T_T - T_H) * a + T_H;
  double rate = fabs(d_alpha_sg(a)) * sigma_sg / (O_KB * T) + fabs(d_alpha_g(a)) * sigma_g / (O_KB * T) +
                fabs(T_T - T_H) * sigma_u / T;
  double an = a + speed / rate;
  return an > 1.0 ? 1.0 : an;
}

/* Sampling importance resampling: n_out indices drawn with replacement from n samples with weights
 * proportional to exp(logw_i); draw j takes the 53-bit uniform of Philox counter {j, 0, ctr, 6}
 * and the first index whose cumulative weight exceeds u times the total (weights relative to the
 * largest, summed in index order). */
void oracle_resample(int64_t n, const double* logw, int n_out, uint64_t seed, uint32_t ctr, int64_t* idx) {
  double m = -INFINITY;
  for (int64_t i = 0; i < n; ++i) if (logw[i] > m) m = logw[i];
  double* cum = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double tot = 0.0;
  for (int64_t i = 0; i < n; ++i) { tot += exp(logw[i] - m); cum[i] = tot; }
  for (int j = 0; j < n_out; ++j) {
    uint32_t r4[4];
    philox(seed, (uint32_t)j, 0u, ctr, 6u, r4);
    double u = oracle_u53(r4[0], r4[1]) * tot;
    int64_t pick = n - 1;
    for (int64_t i = 0; i < n; ++i) if (u < cum[i]) { pick = i; break; }
    idx[j] = pick;
  }
  free(cum);
}

/* Mean exchange probability of Eq. (repXacc) over n pairs (the i-th sample of state a with the
 * i-th of state b): min(1, exp(u_a(x_a) + u_b(x_b) - u_a(x_b) - u_b(x_a))). */
double oracle_mean_pacc(const oracle_system* s, int64_t n, const double* comps_a, const double* comps_b, int ka,
                        int kb) {
  double tot = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double* ca = comps_a + 4 * i;
    const double* cb = comps_b + 4 * i;
    double d = reduced(s->beta[ka], s->w_sg[ka], s->w_g[ka], ca) + reduced(s->beta[kb], s->w_sg[kb], s->w_g[kb], cb) -
               reduced(s->beta[ka], s->w_sg[ka], s->w_g[ka], cb) - reduced(s->beta[kb], s->w_sg[kb], s->w_g[kb], ca);
    tot += d >= 0.0 ? 1.0 : exp(d);
  }
  return tot / (double)n;
}

/* Time-step rule of the sampling-and-adaptation step: acceptance > 0.8: +0.125 fs; < 0.1: -0.5 fs;
 * < 0.4: -0.25 fs; kept in [0.1, 5] fs. */
double oracle_adapt_dt(double dt, double acc) {
  if (acc > 0.8) dt += 0.125;
  else if (acc < 0.1) dt -= 0.5;
  else if (acc < 0.4) dt -= 0.25;
  if (dt < 0.1) dt = 0.1;
  if (dt > 5.0) dt = 5.0;
  return dt;
}

/* ---------------------------------------------------------------- target force field (end points) */
/* Receptor-ligand interaction of the target force field ("Thermodynamic Cycle": the target force
 * field computes receptor-ligand interactions directly rather than by grid interpolation).  The
 * same sums that define the grids are taken at each ligand atom's own position and weighted by
 * that atom's factors:  Psi_T = sum_i sqrt(A_i) LJr(x_i) + sqrt(B_i) LJa(x_i) + q_i elec(x_i).
 * x holds n_samples configurations [n_samples][n_lig][3]; out [n_samples].
 * Returns the number of threads used. */
int oracle_target_interaction(int n_rec, const double* rec_xyz, const double* rec_rstar, const double* rec_eps,
                              const double* rec_q, int n_lig, const double* lig_rstar, const double* lig_eps,
                              const double* lig_q, int64_t n_samples, const double* x, double* out, int n_threads) {
  int64_t np_ = n_samples * n_lig;
  double* ljr = (double*)malloc(sizeof(double) * (size_t)(np_ > 0 ? np_ : 1));
  double* lja = (double*)malloc(sizeof(double) * (size_t)(np_ > 0 ? np_ : 1));
  double* elec = (double*)malloc(sizeof(double) * (size_t)(np_ > 0 ? np_ : 1));
  int T = 1;
  if (np_ > 0)
    T = oracle_grid_points(n_rec, rec_xyz, rec_rstar, rec_eps, rec_q, np_, x, ljr, lja, elec, n_threads);
  for (int64_t s = 0; s < n_samples; ++s) {
    double psi = 0.0;
    for (int i = 0; i < n_lig; ++i) {
      int64_t p = s * n_lig + i;
      psi += sqrtA_of(lig_rstar[i], lig_eps[i]) * ljr[p] + sqrtB_of(lig_rstar[i], lig_eps[i]) * lja[p] +
             lig_q[i] * elec[p];
    }
    out[s] = psi;
  }
  free(ljr); free(lja); free(elec);
  return T;
}
