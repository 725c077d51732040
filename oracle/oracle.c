/*
 * oracle.c — plain, slow FP64 CPU reference of the D3Q19 LBGK step over a
 * sparse lattice, and its discrete adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the GPU solver: it keeps its own velocity tables, neighbour search and
 * boundary arithmetic, stores populations as an array of structures (one
 * 19-vector per site, as in the CPU code of the paper, Section 3.2.3, Fig. 2)
 * and streams in push order (collide, then scatter, Section 3.1).
 *
 * What it computes (arXiv 2202.11770):
 *   - D3Q19 velocities and weights 1/3, 1/18, 1/36 (Section 2.2).
 *   - Density and momentum as zeroth and first moments (Eqs. 5-6).
 *   - Equilibrium: second order in u (Eq. 4).  The printed Eq. 4 lacks the
 *     factors 1/2 on the quadratic terms; without them the second moment of
 *     f^eq would be rho c_s^2 I + 2 rho u u instead of the Navier-Stokes
 *     momentum flux rho c_s^2 I + rho u u, so the standard form
 *       f^eq_i = w_i rho [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)]
 *     is used (reading c2).
 *   - BGK collision f' = f - (f - f^eq)/tau (Eq. 3a, dt = 1) and streaming
 *     f_i(x + c_i, t+1) = f'_i(x, t) (Eq. 3b).
 *   - Walls: mid-link bounce-back (Section 2.3.1): a population that would
 *     stream into a solid node returns to its own site reversed.
 *   - Velocity iolets: Ladd's bounce-back with the correction
 *     -2 w_i rho (u_w . c_i)/cs2 (Section 2.3.2), rho the site's density at
 *     the collision (reading c3), u_w = a_g * w(t) * W(x_m) * n, W = 1 - r^2/R^2
 *     at the link midpoint x_m (clamped at 0): each inlet point carries a
 *     weight from its position in the cross-section (Section 6).
 *   - Pressure iolets: the unknown population is set from a ghost density,
 *     the target pressure's density p/cs2 (Section 2.3.2, Eq. 7); it is the
 *     equilibrium of that density at the ghost velocity (u.n) n, the site's
 *     velocity projected on the iolet normal (reading c4; option: u itself).
 *   - Wall shear stress (not in the paper): stress
 *     sigma = -(1 - 1/(2 tau)) sum_i (f_i - f^eq_i) c_i c_i, traction
 *     t = sigma n, WSS = |t - (t.n) n| at sites with a wall link.
 *   - Adjoint: the exact transpose of the linearised step above, by explicit
 *     per-site 19x19 Jacobians, for an objective averaging squared deviations
 *     of the axial velocity at probe sites from a target.
 *   - Iolet waveforms: constant, cosine, or a table of samples evenly spaced
 *     over one period, interpolated linearly and periodically (the paper's
 *     Section 6 drives its pipe with such a measured one-beat profile).
 *   - Windkessel outlets (not the paper's method; its Section 7 names outlet
 *     resistance models as future work): see wk_t.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
static const int CV[Q][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
static const double CS2 = 1.0 / 3.0;

static double weight(int i) {
  if (i == 0) return 1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* opposite direction: the one with c = -c_i, found by search once */
static int OPP[Q];
static int opp_ready = 0;
static void init_opposite(void) {
  if (opp_ready) return;
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j)
      if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) OPP[i] = j;
  opp_ready = 1;
}
static int opposite(int i) { return OPP[i]; }

static char g_err[256];
const char* ora_last_error(void) { return g_err; }
static int fail(const char* m) { snprintf(g_err, sizeof g_err, "%s", m); return -1; }

/* ---------------- waveforms ---------------- */
typedef struct {
  int kind;        /* 0 constant, 1 cosine, 2 table */
  double mean, rel, period, phase;
  int nsamp;
  double* samp;
} wave_t;

static double wave_at(const wave_t* w, double t) {
  if (w->kind == 0) return w->mean;
  if (w->kind == 1) return w->mean * (1.0 + w->rel * cos(2.0 * M_PI * t / w->period + w->phase));
  /* table: nsamp samples evenly spaced over one period, linear, periodic */
  double x = fmod(t, w->period);
  if (x < 0) x += w->period;
  double pos = x / w->period * w->nsamp;
  int j = (int)floor(pos);
  double fr = pos - j;
  j %= w->nsamp;
  int j1 = (j + 1) % w->nsamp;
  return w->mean * ((1.0 - fr) * w->samp[j] + fr * w->samp[j1]);
}

/* ---------------- oracle object ---------------- */
/* Three-element Windkessel outlet (resistance Rp, compliance C, resistance
 * Rd to a distal density rho_d), coupled explicitly: the ghost density used
 * to produce f(m+1) is rho_c(m) + Rp q(m), with q(m) the volumetric outflow
 * (minus the mass flux) of the step that produced f(m); after that step
 * rho_c(m+1) = rho_c(m) + (q(m+1) - (rho_c(m) - rho_d) / Rd) / C.  C = 0
 * means no compliance: ghost density rho_d + (Rp + Rd) q(m). */
typedef struct {
  int on;
  double Rp, C, Rd, rho_d;
  double rho_c, q;   /* state: compliance density, outflow of the last step */
  double rho_used;   /* ghost density used in the last step */
} wk_t;

typedef struct {
  int kind; /* 0 velocity, 1 pressure */
  double c[3], nrm[3], R;
  int ngroups, goff;
  wave_t wave;
  wk_t wk;
} iolet_t;

typedef struct {
  int64_t n;
  int nio, ngroups_total;
  int32_t* xyz;   /* [n][3] */
  int32_t* dest;  /* [n][Q] push destination or link code */
  int32_t* group; /* [n] */
  double *f, *fn; /* [n][Q] pre-collision state, next state */
  iolet_t* io;
  double* amp;    /* [ngroups_total] */
  double tau;
  int64_t t;
  int ladd_rho_one;  /* 1: use rho = 1 in the Ladd term instead of local rho */
  int ghost_full_u;  /* 1: ghost velocity = u instead of (u.n) n */
  double* flux;      /* [nio] mass entering through each iolet in the last step */
  int threads;       /* host threads a step uses (1: serial) */
} ora_t;

/* ---------------- coordinate hash ---------------- */
typedef struct { uint64_t* key; int64_t* val; uint64_t mask; } hash_t;
static uint64_t pack(int x, int y, int z) {
  return ((uint64_t)(x + (1 << 20)) << 42) | ((uint64_t)(y + (1 << 20)) << 21) | (uint64_t)(z + (1 << 20));
}
static uint64_t mix(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
  return k;
}
static int hash_init(hash_t* h, int64_t n) {
  uint64_t cap = 16;
  while (cap < (uint64_t)n * 2) cap <<= 1;
  h->mask = cap - 1;
  h->key = (uint64_t*)malloc(cap * sizeof(uint64_t));
  h->val = (int64_t*)malloc(cap * sizeof(int64_t));
  if (!h->key || !h->val) return -1;
  memset(h->key, 0xff, cap * sizeof(uint64_t));
  return 0;
}
static void hash_put(hash_t* h, uint64_t k, int64_t v) {
  uint64_t s = mix(k) & h->mask;
  while (h->key[s] != ~0ull) s = (s + 1) & h->mask;
  h->key[s] = k;
  h->val[s] = v;
}
static int64_t hash_get(const hash_t* h, uint64_t k) {
  uint64_t s = mix(k) & h->mask;
  while (h->key[s] != ~0ull) {
    if (h->key[s] == k) return h->val[s];
    s = (s + 1) & h->mask;
  }
  return -1;
}

void ora_free(ora_t* o) {
  if (!o) return;
  free(o->xyz); free(o->dest); free(o->group); free(o->f); free(o->fn);
  if (o->io) for (int k = 0; k < o->nio; ++k) free(o->io[k].wave.samp);
  free(o->io); free(o->amp); free(o->flux);
  free(o);
}

/*
 * Create from a lattice.  xyz[n][3] gives the sites; the push destination of
 * each link is found from the coordinates.  For links whose end is not a
 * fluid site the kind (wall or iolet k) is read from the lattice's pull-source
 * code of the reverse direction at the same site: src[(j-1)*n + x] with
 * c_j = -c_i, -1 = wall, -(2+k) = iolet k.  Fluid entries of src must agree
 * with the coordinates.
 */
int ora_create(int64_t n, const int32_t* xyz, const int32_t* src, int nio, const int32_t* kind,
               const double* centre, const double* normal, const double* radius,
               const int32_t* ngroups, const int32_t* group, ora_t** out) {
  *out = NULL;
  if (n <= 0) return fail("n must be positive");
  if (nio < 0 || nio > 256) return fail("at most 256 iolets");
  init_opposite();
  ora_t* o = (ora_t*)calloc(1, sizeof *o);
  o->n = n;
  o->nio = nio;
  o->tau = 1.0;
  o->xyz = (int32_t*)malloc((size_t)n * 3 * sizeof(int32_t));
  o->dest = (int32_t*)malloc((size_t)n * Q * sizeof(int32_t));
  o->group = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  o->f = (double*)malloc((size_t)n * Q * sizeof(double));
  o->fn = (double*)malloc((size_t)n * Q * sizeof(double));
  o->io = (iolet_t*)calloc((size_t)(nio > 0 ? nio : 1), sizeof(iolet_t));
  o->flux = (double*)calloc((size_t)(nio > 0 ? nio : 1), sizeof(double));
  if (!o->xyz || !o->dest || !o->group || !o->f || !o->fn || !o->io || !o->flux) {
    ora_free(o); return fail("out of memory");
  }
  memcpy(o->xyz, xyz, (size_t)n * 3 * sizeof(int32_t));
  if (group) memcpy(o->group, group, (size_t)n * sizeof(int32_t));
  int goff = 0;
  for (int k = 0; k < nio; ++k) {
    iolet_t* io = &o->io[k];
    io->kind = kind[k];
    for (int a = 0; a < 3; ++a) { io->c[a] = centre[3 * k + a]; io->nrm[a] = normal[3 * k + a]; }
    io->R = radius[k];
    io->ngroups = ngroups ? ngroups[k] : 1;
    /* amplitude groups are numbered over the velocity iolets only */
    io->goff = io->kind == 0 ? goff : -1;
    if (io->kind == 0) goff += io->ngroups;
    io->wave.kind = 0;
    io->wave.mean = io->kind == 1 ? 1.0 : 0.0;
  }
  o->ngroups_total = goff;
  o->amp = (double*)calloc((size_t)(goff > 0 ? goff : 1), sizeof(double));
  for (int g = 0; g < goff; ++g) o->amp[g] = 1.0;

  hash_t h;
  if (hash_init(&h, n)) { ora_free(o); return fail("out of memory"); }
  for (int64_t x = 0; x < n; ++x) hash_put(&h, pack(xyz[3 * x], xyz[3 * x + 1], xyz[3 * x + 2]), x);
  int bad = 0;
  for (int64_t x = 0; x < n && !bad; ++x) {
    o->dest[x * Q] = (int32_t)x;
    for (int i = 1; i < Q; ++i) {
      int64_t y = hash_get(&h, pack(xyz[3 * x] + CV[i][0], xyz[3 * x + 1] + CV[i][1], xyz[3 * x + 2] + CV[i][2]));
      int j = opposite(i);
      int32_t code = src[(int64_t)(j - 1) * n + x]; /* pull source of x along c_j = x - c_j = x + c_i */
      if (y >= 0) {
        if (code != (int32_t)y) bad = 1;
        o->dest[x * Q + i] = (int32_t)y;
      } else {
        if (code >= 0 || code < -(2 + nio - 1)) bad = 2;
        else if (code <= -2 && o->io[-code - 2].kind == 0 &&
                 (o->group[x] < 0 || o->group[x] >= o->io[-code - 2].ngroups)) bad = 3;
        o->dest[x * Q + i] = code;
      }
    }
  }
  free(h.key);
  free(h.val);
  if (bad) {
    ora_free(o);
    return fail(bad == 1 ? "src table disagrees with coordinates"
                         : bad == 2 ? "bad link code" : "amplitude group out of range");
  }
  *out = o;
  return 0;
}

void ora_set_tau(ora_t* o, double tau) { o->tau = tau; }
/* Host threads of ora_step (default 1); the state is the same for any count. */
void ora_set_threads(ora_t* o, int threads) { o->threads = threads > 1 ? threads : 1; }
void ora_set_options(ora_t* o, int ladd_rho_one, int ghost_full_u) {
  o->ladd_rho_one = ladd_rho_one;
  o->ghost_full_u = ghost_full_u;
}

static int set_wave(wave_t* w, int kind, double mean, double rel, double period, double phase,
                    int nsamp, const double* samp) {
  free(w->samp);
  w->samp = NULL;
  w->kind = kind; w->mean = mean; w->rel = rel; w->period = period; w->phase = phase; w->nsamp = 0;
  if (kind == 2) {
    if (nsamp < 1 || !samp) return fail("table waveform needs samples");
    w->samp = (double*)malloc((size_t)nsamp * sizeof(double));
    memcpy(w->samp, samp, (size_t)nsamp * sizeof(double));
    w->nsamp = nsamp;
  }
  if (kind != 0 && !(period > 0)) return fail("waveform period must be positive");
  return 0;
}

/* Velocity iolet k: u_w = amps[g] * w(t) * W * n. */
int ora_set_velocity(ora_t* o, int k, const double* amps, int ngroups, int kind, double mean,
                     double rel, double period, double phase, int nsamp, const double* samp) {
  if (k < 0 || k >= o->nio || o->io[k].kind != 0) return fail("not a velocity iolet");
  if (ngroups != o->io[k].ngroups) return fail("group count mismatch");
  for (int g = 0; g < ngroups; ++g) o->amp[o->io[k].goff + g] = amps[g];
  return set_wave(&o->io[k].wave, kind, mean, rel, period, phase, nsamp, samp);
}
/* Pressure iolet k becomes a Windkessel outlet (Rp, C, Rd >= 0) with
 * compliance density rho_c0 and no outflow history.  With C > 0 the
 * explicit update of rho_c multiplies its distance to the fixed point by
 * 1 - 1/(Rd C) per step, so Rd C >= 1 is required (no overshoot). */
int ora_set_windkessel(ora_t* o, int k, double Rp, double C, double Rd, double rho_d, double rho_c0) {
  if (k < 0 || k >= o->nio || o->io[k].kind != 1) return fail("not a pressure iolet");
  if (!(Rp >= 0) || !(C >= 0) || !(Rd >= 0) || (C > 0 && !(Rd * C >= 1))) return fail("bad Windkessel parameters");
  wk_t* m = &o->io[k].wk;
  m->on = 1; m->Rp = Rp; m->C = C; m->Rd = Rd; m->rho_d = rho_d;
  m->rho_c = C > 0 ? rho_c0 : rho_d;
  m->q = 0;
  m->rho_used = NAN;
  return 0;
}
/* Ghost density iolet k used in the last step (Windkessel outlets), and the
 * compliance density now. */
double ora_windkessel_rho(const ora_t* o, int k) { return o->io[k].wk.rho_used; }
double ora_windkessel_rho_c(const ora_t* o, int k) { return o->io[k].wk.rho_c; }

/* Value of iolet k's waveform at time t (test access to wave_at). */
double ora_wave_value(const ora_t* o, int k, double t) {
  if (k < 0 || k >= o->nio) return NAN;
  return wave_at(&o->io[k].wave, t);
}
/* Pressure iolet k: ghost density rho(t) = w(t). */
int ora_set_pressure(ora_t* o, int k, int kind, double mean, double rel, double period,
                     double phase, int nsamp, const double* samp) {
  if (k < 0 || k >= o->nio || o->io[k].kind != 1) return fail("not a pressure iolet");
  o->io[k].wk.on = 0;
  return set_wave(&o->io[k].wave, kind, mean, rel, period, phase, nsamp, samp);
}

/* Equilibrium, Eq. 4 with the factors 1/2 (reading c2). */
void ora_feq(double rho, const double* u, double* feq) {
  const double a = 1.0 / CS2, b = 1.0 / (2.0 * CS2 * CS2), c = 1.0 / (2.0 * CS2);
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    feq[i] = weight(i) * rho * (1.0 + cu * a + cu * cu * b - uu * c);
  }
}

static void moments(const double* f, double* rho, double* u) {
  double r = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) {
    r += f[i];
    for (int a = 0; a < 3; ++a) j[a] += f[i] * CV[i][a];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* Ladd weight at the midpoint of link (x, i) for iolet io. */
static double ladd_weight(const iolet_t* io, const int32_t* p, int i) {
  double m[3], v[3];
  for (int a = 0; a < 3; ++a) m[a] = p[a] + 0.5 * CV[i][a];
  for (int a = 0; a < 3; ++a) v[a] = m[a] - io->c[a];
  double s = v[0] * io->nrm[0] + v[1] * io->nrm[1] + v[2] * io->nrm[2];
  double r2 = 0;
  for (int a = 0; a < 3; ++a) { double w = v[a] - s * io->nrm[a]; r2 += w * w; }
  double W = 1.0 - r2 / (io->R * io->R);
  return W > 0 ? W : 0;
}

void ora_init_equilibrium(ora_t* o, double rho0, const double* u0) {
  double zero[3] = {0, 0, 0};
  for (int64_t x = 0; x < o->n; ++x) ora_feq(rho0, u0 ? &u0[3 * x] : zero, &o->f[x * Q]);
  o->t = 0;
  for (int k = 0; k < o->nio; ++k) {
    o->flux[k] = 0;
    o->io[k].wk.q = 0;  /* no outflow history; the compliance density is kept */
  }
}

/* Collide site x and push its populations (with the boundary values of its
 * wall and iolet links) into the next state; adds the mass each iolet link
 * lets in to flux[k]. */
static void site_step(ora_t* o, int64_t x, const double* wk, double* flux) {
  const double* f = &o->f[x * Q];
  double rho, u[3], feq[Q], fp[Q];
  moments(f, &rho, u);
  ora_feq(rho, u, feq);
  const double omega = 1.0 / o->tau;
  for (int i = 0; i < Q; ++i) fp[i] = f[i] - (f[i] - feq[i]) * omega;
  for (int i = 0; i < Q; ++i) {
    int32_t y = o->dest[x * Q + i];
    if (y >= 0) {
      o->fn[(int64_t)y * Q + i] = fp[i];
      continue;
    }
    int ib = opposite(i);
    double val;
    if (y == -1) {
      val = fp[i];
    } else {
      int k = -y - 2;
      const iolet_t* io = &o->io[k];
      if (io->kind == 0) {
        double W = ladd_weight(io, &o->xyz[3 * x], i);
        double A = o->amp[io->goff + o->group[x]] * wk[k];
        double cu_w = A * W * (CV[i][0] * io->nrm[0] + CV[i][1] * io->nrm[1] + CV[i][2] * io->nrm[2]);
        double r = o->ladd_rho_one ? 1.0 : rho;
        val = fp[i] - 2.0 * weight(i) * r * cu_w / CS2;
      } else {
        double ug[3], geq[Q];
        if (o->ghost_full_u) {
          memcpy(ug, u, sizeof ug);
        } else {
          double un = u[0] * io->nrm[0] + u[1] * io->nrm[1] + u[2] * io->nrm[2];
          for (int a = 0; a < 3; ++a) ug[a] = un * io->nrm[a];
        }
        ora_feq(wk[k], ug, geq);
        val = geq[ib];
      }
      flux[k] += val - fp[i];
    }
    o->fn[x * Q + ib] = val;
  }
}

/* One time step: collide every site, push to neighbours, apply BCs (Section
 * 3.1).  Sites may be split over threads (ora_set_threads): every slot of the
 * next state has exactly one writer, so the state does not depend on the
 * thread count; each thread sums its own iolet fluxes over a contiguous block
 * of sites and the blocks are added in thread order. */
static void step_once(ora_t* o) {
  const int64_t n = o->n;
  const double t = (double)o->t;
  double wk[256];
  for (int k = 0; k < o->nio && k < 256; ++k) {
    const wk_t* m = &o->io[k].wk;
    if (m->on)
      wk[k] = m->C > 0 ? m->rho_c + m->Rp * m->q : m->rho_d + (m->Rp + m->Rd) * m->q;
    else
      wk[k] = wave_at(&o->io[k].wave, t);
    o->io[k].wk.rho_used = wk[k];
  }
  const int nt = o->threads > 1 ? o->threads : 1;
  const int nk = o->nio > 0 ? o->nio : 1;
  double* part = (double*)calloc((size_t)nt * nk, sizeof(double));
  if (nt == 1) {
    for (int64_t x = 0; x < n; ++x) site_step(o, x, wk, part);
  } else {
#pragma omp parallel num_threads(nt)
    {
      const int tid = omp_get_thread_num(), cnt = omp_get_num_threads();
      const int64_t b = n * tid / cnt, e = n * (tid + 1) / cnt;
      for (int64_t x = b; x < e; ++x) site_step(o, x, wk, part + (size_t)tid * nk);
    }
  }
  for (int k = 0; k < o->nio; ++k) {
    o->flux[k] = 0;
    for (int th = 0; th < nt; ++th) o->flux[k] += part[(size_t)th * nk + k];
  }
  free(part);
  double* tmp = o->f;
  o->f = o->fn;
  o->fn = tmp;
  o->t += 1;
  for (int k = 0; k < o->nio; ++k) {
    wk_t* m = &o->io[k].wk;
    if (!m->on) continue;
    m->q = -o->flux[k];
    if (m->C > 0) m->rho_c += (m->q - (m->rho_c - m->rho_d) / m->Rd) / m->C;
  }
}

void ora_step(ora_t* o, int64_t nsteps) {
  for (int64_t s = 0; s < nsteps; ++s) step_once(o);
}

int64_t ora_time(const ora_t* o) { return o->t; }

void ora_get_state(const ora_t* o, double* f) { memcpy(f, o->f, (size_t)o->n * Q * sizeof(double)); }
void ora_set_state(ora_t* o, const double* f, int64_t t) {
  memcpy(o->f, f, (size_t)o->n * Q * sizeof(double));
  o->t = t;
}

/* Total mass (sum of all populations of the current state). */
double ora_mass(const ora_t* o) {
  double m = 0;
  for (int64_t x = 0; x < o->n; ++x)
    for (int i = 0; i < Q; ++i) m += o->f[x * Q + i];
  return m;
}
void ora_flux(const ora_t* o, double* out) { memcpy(out, o->flux, (size_t)o->nio * sizeof(double)); }

/*
 * Density, velocity and wall shear stress of the current state.  wss is NaN at
 * sites without a wall link.  wall_normal[3][n] (unit, into the fluid) may be
 * NULL: the normal then falls back to the normalised sum of -c_i over the
 * site's wall links.  Any output pointer may be NULL.
 */
void ora_macros(const ora_t* o, double* rho_out, double* u_out, double* wss_out,
                const float* wall_normal) {
  const int64_t n = o->n;
  for (int64_t x = 0; x < n; ++x) {
    const double* f = &o->f[x * Q];
    double rho, u[3];
    moments(f, &rho, u);
    if (rho_out) rho_out[x] = rho;
    if (u_out) for (int a = 0; a < 3; ++a) u_out[3 * x + a] = u[a];
    if (!wss_out) continue;
    int has_wall = 0;
    double nsum[3] = {0, 0, 0};
    for (int i = 1; i < Q; ++i)
      if (o->dest[x * Q + i] == -1) {
        has_wall = 1;
        for (int a = 0; a < 3; ++a) nsum[a] -= CV[i][a];
      }
    if (!has_wall) { wss_out[x] = NAN; continue; }
    double nv[3];
    if (wall_normal) {
      for (int a = 0; a < 3; ++a) nv[a] = wall_normal[(int64_t)a * n + x];
    } else {
      double l = sqrt(nsum[0] * nsum[0] + nsum[1] * nsum[1] + nsum[2] * nsum[2]);
      for (int a = 0; a < 3; ++a) nv[a] = l > 0 ? nsum[a] / l : 0;
    }
    double feq[Q], sig[3][3] = {{0}};
    ora_feq(rho, u, feq);
    for (int i = 0; i < Q; ++i)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          sig[a][b] += -(1.0 - 1.0 / (2.0 * o->tau)) * (f[i] - feq[i]) * CV[i][a] * CV[i][b];
    double tr[3], tn = 0;
    for (int a = 0; a < 3; ++a) tr[a] = sig[a][0] * nv[0] + sig[a][1] * nv[1] + sig[a][2] * nv[2];
    for (int a = 0; a < 3; ++a) tn += tr[a] * nv[a];
    double s = 0;
    for (int a = 0; a < 3; ++a) { double w = tr[a] - tn * nv[a]; s += w * w; }
    wss_out[x] = sqrt(s);
  }
}

/* ---------------- objective and adjoint ---------------- */
typedef struct {
  int64_t np;
  const int64_t* site;
  const double* target;
  double axis[3];
  int64_t nsteps;
} objective_t;

static double objective_at(const ora_t* o, const objective_t* ob) {
  double s = 0;
  for (int64_t p = 0; p < ob->np; ++p) {
    double rho, u[3];
    moments(&o->f[ob->site[p] * Q], &rho, u);
    double ua = u[0] * ob->axis[0] + u[1] * ob->axis[1] + u[2] * ob->axis[2];
    s += (ua - ob->target[p]) * (ua - ob->target[p]);
  }
  return s / (double)ob->nsteps;
}

/* J = (1/N) sum_{t=1..N} sum_p (u(p,t).axis - target_p)^2 over N steps from
 * the current state (which is advanced by N steps). */
double ora_objective(ora_t* o, int64_t nsteps, int64_t np, const int64_t* site,
                     const double* target, const double* axis) {
  objective_t ob = {np, site, target, {axis[0], axis[1], axis[2]}, nsteps};
  double J = 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    step_once(o);
    J += objective_at(o, &ob);
  }
  return J;
}

/* d feq_i / d u_a at (rho, u) */
static void dfeq_du(double rho, const double* u, double out[Q][3]) {
  for (int i = 0; i < Q; ++i) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    for (int a = 0; a < 3; ++a)
      out[i][a] = weight(i) * rho * (CV[i][a] / CS2 + cu * CV[i][a] / (CS2 * CS2) - u[a] / CS2);
  }
}

/*
 * Discrete adjoint over N steps from the current state.  Stores every state
 * (memory n*19*8*(N+1) bytes; small cases only), then sweeps backwards.
 * Outputs J, dJ/dtau and dJ/da_g for every amplitude group of every velocity
 * iolet (global group order: iolet by iolet).  The state is advanced by N.
 */
int ora_adjoint(ora_t* o, int64_t nsteps, int64_t np, const int64_t* site, const double* target,
                const double* axis, double* J_out, double* dtau_out, double* damp_out) {
  const int64_t n = o->n;
  const size_t S = (size_t)n * Q;
  objective_t ob = {np, site, target, {axis[0], axis[1], axis[2]}, nsteps};
  double* F = (double*)malloc(S * (size_t)(nsteps + 1) * sizeof(double));
  double* mu = (double*)calloc(S, sizeof(double));
  double* mu_prev = (double*)calloc(S, sizeof(double));
  if (!F || !mu || !mu_prev) { free(F); free(mu); free(mu_prev); return fail("out of memory for adjoint states"); }
  const int64_t t0 = o->t;
  memcpy(F, o->f, S * sizeof(double));
  double J = 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    step_once(o);
    memcpy(F + S * (size_t)(s + 1), o->f, S * sizeof(double));
    J += objective_at(o, &ob);
  }
  for (int g = 0; g < o->ngroups_total; ++g) damp_out[g] = 0;
  double dtau = 0;
  const double tau = o->tau;

  /* objective derivative w.r.t. the state f(s) at step index s (s >= 1) */
#define ADD_OBJ(mu_arr, s_idx)                                                             \
  for (int64_t p = 0; p < np; ++p) {                                                       \
    const double* fs = F + S * (size_t)(s_idx) + (size_t)site[p] * Q;                      \
    double rho, u[3];                                                                      \
    moments(fs, &rho, u);                                                                  \
    double ua = u[0] * axis[0] + u[1] * axis[1] + u[2] * axis[2];                          \
    double g = 2.0 * (ua - target[p]) / (double)nsteps;                                    \
    for (int j = 0; j < Q; ++j) {                                                          \
      double cj = CV[j][0] * axis[0] + CV[j][1] * axis[1] + CV[j][2] * axis[2];            \
      mu_arr[(size_t)site[p] * Q + j] += g * (cj - ua) / rho;                              \
    }                                                                                      \
  }

  memset(mu, 0, S * sizeof(double));
  ADD_OBJ(mu, nsteps);
  for (int64_t s = nsteps - 1; s >= 0; --s) {
    const double tt = (double)(t0 + s);
    double wk[256];
    for (int k = 0; k < o->nio && k < 256; ++k) wk[k] = wave_at(&o->io[k].wave, tt);
    memset(mu_prev, 0, S * sizeof(double));
    const double* Fs = F + S * (size_t)s;
    for (int64_t x = 0; x < n; ++x) {
      const double* f = &Fs[x * Q];
      double rho, u[3], feq[Q], lam[Q], du[Q][3];
      moments(f, &rho, u);
      ora_feq(rho, u, feq);
      dfeq_du(rho, u, du);
      double arho = 0, au[3] = {0, 0, 0}; /* adjoints of rho and u via direct BC dependence */
      for (int i = 0; i < Q; ++i) {
        int32_t y = o->dest[x * Q + i];
        int ib = opposite(i);
        if (y >= 0) { lam[i] = mu[(size_t)y * Q + i]; continue; }
        double m = mu[(size_t)x * Q + ib];
        if (y == -1) { lam[i] = m; continue; }
        const iolet_t* io = &o->io[-y - 2];
        if (io->kind == 0) {
          lam[i] = m;
          double W = ladd_weight(io, &o->xyz[3 * x], i);
          double cn = CV[i][0] * io->nrm[0] + CV[i][1] * io->nrm[1] + CV[i][2] * io->nrm[2];
          int g = io->goff + o->group[x];
          double A = o->amp[g] * wk[-y - 2];
          double r = o->ladd_rho_one ? 1.0 : rho;
          if (!o->ladd_rho_one) arho += m * (-2.0 * weight(i) * A * W * cn / CS2);
          damp_out[g] += m * (-2.0 * weight(i) * r * wk[-y - 2] * W * cn / CS2);
        } else {
          lam[i] = 0;
          double ug[3], dg[Q][3];
          double un = u[0] * io->nrm[0] + u[1] * io->nrm[1] + u[2] * io->nrm[2];
          for (int a = 0; a < 3; ++a) ug[a] = o->ghost_full_u ? u[a] : un * io->nrm[a];
          dfeq_du(wk[-y - 2], ug, dg);
          double aug[3];
          for (int b = 0; b < 3; ++b) aug[b] = m * dg[ib][b];
          if (o->ghost_full_u) {
            for (int a = 0; a < 3; ++a) au[a] += aug[a];
          } else {
            double s2 = aug[0] * io->nrm[0] + aug[1] * io->nrm[1] + aug[2] * io->nrm[2];
            for (int a = 0; a < 3; ++a) au[a] += s2 * io->nrm[a];
          }
        }
      }
      /* collision Jacobian: dfp_i/df_j = delta_ij (1 - 1/tau) + (1/tau) dfeq_i/df_j,
       * dfeq_i/df_j = feq_i/rho + sum_a du[i][a] (c_ja - u_a)/rho */
      for (int j = 0; j < Q; ++j) {
        double acc = lam[j] * (1.0 - 1.0 / tau);
        for (int i = 0; i < Q; ++i) {
          double d = feq[i] / rho;
          for (int a = 0; a < 3; ++a) d += du[i][a] * (CV[j][a] - u[a]) / rho;
          acc += lam[i] * d / tau;
        }
        acc += arho;
        for (int a = 0; a < 3; ++a) acc += au[a] * (CV[j][a] - u[a]) / rho;
        mu_prev[(size_t)x * Q + j] = acc;
      }
      for (int i = 0; i < Q; ++i) dtau += lam[i] * (f[i] - feq[i]) / (tau * tau);
    }
    if (s >= 1) ADD_OBJ(mu_prev, s);
    double* tmp = mu; mu = mu_prev; mu_prev = tmp;
  }
#undef ADD_OBJ
  *J_out = J;
  *dtau_out = dtau;
  free(F); free(mu); free(mu_prev);
  return 0;
}

int ora_n_groups(const ora_t* o) { return o->ngroups_total; }
