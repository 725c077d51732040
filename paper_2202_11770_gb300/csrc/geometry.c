/*
 * geometry.c — seeded synthetic sparse lattices for the D3Q19 solver and its
 * oracle.  Input generation only: voxelisation, neighbour search and link
 * classification.  No lattice Boltzmann arithmetic lives here.
 *
 * Paper context (arXiv 2202.11770): Section 3.2.1 (the solver starts from a
 * sparse list of fluid sites with streaming indices and wall/iolet link
 * information), Section 3.2.2 (six site types), Section 2.2 (D3Q19 set).
 * The paper's vascular geometries come from patient scans; the straight pipe
 * and the seeded bifurcating tree built here stand in for them.
 */
#include "../../include/hlb_geometry.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* errors                                                              */
/* ------------------------------------------------------------------ */
static __thread char g_err[256];
static int fail(const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return -1;
}
const char* hlbg_last_error(void) { return g_err; }

/* D3Q19 directions in the order documented in hlb_geometry.h. */
static const int C[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double* a) {
  double l = sqrt(dot3(a, a));
  if (l > 0) { a[0] /= l; a[1] /= l; a[2] /= l; }
}
/* Rotate v about unit axis k by angle th (Rodrigues). */
static void rotate3(const double* v, const double* k, double th, double* o) {
  double c = cos(th), s = sin(th), kv = dot3(k, v), kxv[3];
  cross3(k, v, kxv);
  for (int a = 0; a < 3; ++a) o[a] = v[a] * c + kxv[a] * s + k[a] * kv * (1 - c);
}

/* ------------------------------------------------------------------ */
/* seeded random numbers: SplitMix64 (Steele, Lea & Flood 2014)        */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t s; } rng_t;
static uint64_t rng_next(rng_t* r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
/* uniform in [0,1) with 53 random bits */
static double rng_uniform(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------ */
/* segments                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
  double a[3], b[3], d[3]; /* start, end, unit direction */
  double r, len;
  int flat_a, flat_b;      /* flat (iolet) ends instead of spherical caps */
  int leaf, depth;
  double lo[3], hi[3];     /* bounding box of the solid segment */
} seg_t;

static void seg_bbox(seg_t* s) {
  for (int a = 0; a < 3; ++a) {
    double m = fmin(s->a[a], s->b[a]), M = fmax(s->a[a], s->b[a]);
    s->lo[a] = m - s->r;
    s->hi[a] = M + s->r;
  }
}

/* Is point p strictly inside segment s (radius inflated by `grow`)? */
static int seg_inside(const seg_t* s, const double* p, double grow) {
  double v[3] = {p[0] - s->a[0], p[1] - s->a[1], p[2] - s->a[2]};
  double t = dot3(v, s->d), q[3];
  if (t < 0) {
    if (s->flat_a) return 0;
    t = 0;
  } else if (t > s->len) {
    if (s->flat_b) return 0;
    t = s->len;
  }
  for (int a = 0; a < 3; ++a) q[a] = s->a[a] + t * s->d[a];
  double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
  double rr = s->r + grow;
  return dx * dx + dy * dy + dz * dz < rr * rr;
}

/* Closest axis point of s to p (clamped to the segment). */
static void seg_axis_point(const seg_t* s, const double* p, double* q) {
  double v[3] = {p[0] - s->a[0], p[1] - s->a[1], p[2] - s->a[2]};
  double t = dot3(v, s->d);
  if (t < 0) t = 0;
  if (t > s->len) t = s->len;
  for (int a = 0; a < 3; ++a) q[a] = s->a[a] + t * s->d[a];
}

/* ------------------------------------------------------------------ */
/* lattice object                                                      */
/* ------------------------------------------------------------------ */
struct hlbg_lattice {
  int64_t n;
  int32_t* xyz;
  int32_t* src;
  uint8_t* type;
  float* wall_normal;
  int32_t* amp_group;
  int32_t n_iolets;
  hlbg_iolet* iolets;
  int32_t* iolet_seg; /* segment owning each iolet */
  double info[8];
};

void hlbg_free(hlbg_lattice* L) {
  if (!L) return;
  free(L->xyz);
  free(L->src);
  free(L->type);
  free(L->wall_normal);
  free(L->amp_group);
  free(L->iolets);
  free(L->iolet_seg);
  free(L);
}
int64_t hlbg_n_sites(const hlbg_lattice* L) { return L->n; }
const int32_t* hlbg_xyz(const hlbg_lattice* L) { return L->xyz; }
const int32_t* hlbg_src(const hlbg_lattice* L) { return L->src; }
const uint8_t* hlbg_type(const hlbg_lattice* L) { return L->type; }
const float* hlbg_wall_normal(const hlbg_lattice* L) { return L->wall_normal; }
const int32_t* hlbg_amp_group(const hlbg_lattice* L) { return L->amp_group; }
int32_t hlbg_n_iolets(const hlbg_lattice* L) { return L->n_iolets; }
const hlbg_iolet* hlbg_iolets(const hlbg_lattice* L) { return L->iolets; }
void hlbg_info(const hlbg_lattice* L, double info[8]) { memcpy(info, L->info, sizeof L->info); }

/* ------------------------------------------------------------------ */
/* voxelisation of a union of segments                                 */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t* pts; /* x,y,z triples */
  int64_t n, cap;
} ptbuf_t;

static int ptbuf_push(ptbuf_t* b, int x, int y, int z) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? b->cap * 2 : 4096;
    int32_t* np = (int32_t*)realloc(b->pts, (size_t)nc * 3 * sizeof(int32_t));
    if (!np) return -1;
    b->pts = np;
    b->cap = nc;
  }
  b->pts[3 * b->n + 0] = x;
  b->pts[3 * b->n + 1] = y;
  b->pts[3 * b->n + 2] = z;
  b->n++;
  return 0;
}

static int boxes_overlap(const seg_t* A, const seg_t* B, double pad) {
  for (int a = 0; a < 3; ++a)
    if (A->hi[a] + pad < B->lo[a] || B->hi[a] + pad < A->lo[a]) return 0;
  return 1;
}

/* Voxelise: every integer point strictly inside at least one segment is
 * emitted once, by the lowest-numbered segment containing it.  If `bufs` is
 * NULL only the count is returned. */
static int64_t voxelise(const seg_t* segs, int ns, ptbuf_t* bufs, int* err) {
  int64_t total = 0;
  *err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
  for (int k = 0; k < ns; ++k) {
    const seg_t* s = &segs[k];
    int prior[512], np = 0;
    for (int j = 0; j < k && np < 512; ++j)
      if (boxes_overlap(s, &segs[j], 1.0)) prior[np++] = j;
    int x0 = (int)floor(s->lo[0]), x1 = (int)ceil(s->hi[0]);
    int y0 = (int)floor(s->lo[1]), y1 = (int)ceil(s->hi[1]);
    int z0 = (int)floor(s->lo[2]), z1 = (int)ceil(s->hi[2]);
    int64_t cnt = 0;
    for (int z = z0; z <= z1; ++z)
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
          double p[3] = {x, y, z};
          if (!seg_inside(s, p, 0.0)) continue;
          int owned = 1;
          for (int q = 0; q < np; ++q)
            if (seg_inside(&segs[prior[q]], p, 0.0)) { owned = 0; break; }
          if (!owned) continue;
          ++cnt;
          if (bufs && ptbuf_push(&bufs[k], x, y, z)) {
#pragma omp atomic write
            *err = 1;
          }
        }
    total += cnt;
  }
  return total;
}

/* LSD radix sort of 64-bit keys carrying a 64-bit payload index. */
static int radix_sort(uint64_t* key, int64_t* idx, int64_t n, int nbits) {
  uint64_t* k2 = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  int64_t* i2 = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!k2 || !i2) { free(k2); free(i2); return -1; }
  int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
  for (int shift = 0; shift < nbits; shift += 16) {
    memset(cnt, 0, 65536 * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cnt[(key[i] >> shift) & 0xFFFF]++;
    int64_t run = 0;
    for (int b = 0; b < 65536; ++b) { int64_t c = cnt[b]; cnt[b] = run; run += c; }
    for (int64_t i = 0; i < n; ++i) {
      int64_t o = cnt[(key[i] >> shift) & 0xFFFF]++;
      k2[o] = key[i];
      i2[o] = idx[i];
    }
    memcpy(key, k2, (size_t)n * sizeof(uint64_t));
    memcpy(idx, i2, (size_t)n * sizeof(int64_t));
  }
  free(cnt);
  free(k2);
  free(i2);
  return 0;
}

/* Row-indexed lookup of fluid sites sorted by (z, y, x). */
typedef struct {
  int lo[3], dim[3];
  int64_t* row_start; /* dim[1]*dim[2] + 1 */
  const int32_t* xyz;
} finder_t;

static int64_t find_site(const finder_t* F, int x, int y, int z) {
  int ry = y - F->lo[1], rz = z - F->lo[2];
  if (x < F->lo[0] || x >= F->lo[0] + F->dim[0]) return -1;
  if (ry < 0 || ry >= F->dim[1] || rz < 0 || rz >= F->dim[2]) return -1;
  int64_t r = (int64_t)rz * F->dim[1] + ry;
  int64_t a = F->row_start[r], b = F->row_start[r + 1];
  while (a < b) {
    int64_t m = (a + b) >> 1;
    int xm = F->xyz[3 * m];
    if (xm == x) return m;
    if (xm < x) a = m + 1; else b = m;
  }
  return -1;
}

/* ------------------------------------------------------------------ */
/* lattice assembly from segments + iolets                             */
/* ------------------------------------------------------------------ */
static int classify_link(const hlbg_lattice* L, const int32_t* p, int i) {
  double m[3] = {p[0] + 0.5 * C[i][0], p[1] + 0.5 * C[i][1], p[2] + 0.5 * C[i][2]};
  for (int k = 0; k < L->n_iolets; ++k) {
    const hlbg_iolet* io = &L->iolets[k];
    double v[3] = {m[0] - io->centre[0], m[1] - io->centre[1], m[2] - io->centre[2]};
    double s = dot3(v, io->normal);
    if (s > 0 || s < -1.0) continue;
    double w[3] = {v[0] - s * io->normal[0], v[1] - s * io->normal[1], v[2] - s * io->normal[2]};
    if (dot3(w, w) <= io->radius * io->radius) return -(2 + k);
  }
  return -1;
}

static void iolet_basis(const hlbg_iolet* io, double* e1, double* e2) {
  double ref[3] = {1, 0, 0};
  if (fabs(io->normal[0]) > 0.9) { ref[0] = 0; ref[1] = 1; }
  double s = dot3(ref, io->normal);
  for (int a = 0; a < 3; ++a) e1[a] = ref[a] - s * io->normal[a];
  normalize3(e1);
  cross3(io->normal, e1, e2);
}

static int assemble(hlbg_lattice* L, const seg_t* segs, int ns, int n_sectors, int n_rings) {
  int err = 0;
  ptbuf_t* bufs = (ptbuf_t*)calloc((size_t)ns, sizeof(ptbuf_t));
  if (!bufs) return fail("out of host memory");
  int64_t n = voxelise(segs, ns, bufs, &err);
  if (err) { for (int k = 0; k < ns; ++k) free(bufs[k].pts); free(bufs); return fail("out of host memory"); }
  if (n <= 0 || n >= (int64_t)1 << 31) { for (int k = 0; k < ns; ++k) free(bufs[k].pts); free(bufs); return fail("site count out of range"); }

  /* bounding box of the sites */
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int k = 0; k < ns; ++k)
    for (int64_t q = 0; q < bufs[k].n; ++q)
      for (int a = 0; a < 3; ++a) {
        int v = bufs[k].pts[3 * q + a];
        if (v < lo[a]) lo[a] = v;
        if (v > hi[a]) hi[a] = v;
      }
  int dim[3] = {hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};

  /* gather + sort by (z, y, x) */
  int32_t* raw = (int32_t*)malloc((size_t)n * 3 * sizeof(int32_t));
  uint64_t* key = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  int64_t* idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!raw || !key || !idx) { free(raw); free(key); free(idx); return fail("out of host memory"); }
  int64_t off = 0;
  for (int k = 0; k < ns; ++k) {
    memcpy(raw + 3 * off, bufs[k].pts, (size_t)bufs[k].n * 3 * sizeof(int32_t));
    off += bufs[k].n;
    free(bufs[k].pts);
  }
  free(bufs);
  uint64_t X = (uint64_t)dim[0], XY = X * (uint64_t)dim[1];
  for (int64_t q = 0; q < n; ++q) {
    key[q] = (uint64_t)(raw[3 * q + 2] - lo[2]) * XY + (uint64_t)(raw[3 * q + 1] - lo[1]) * X +
             (uint64_t)(raw[3 * q] - lo[0]);
    idx[q] = q;
  }
  uint64_t maxkey = XY * (uint64_t)dim[2];
  int nbits = 0;
  while (nbits < 64 && (maxkey >> nbits)) nbits += 16;
  if (radix_sort(key, idx, n, nbits)) { free(raw); free(key); free(idx); return fail("out of host memory"); }
  free(key);

  L->n = n;
  L->xyz = (int32_t*)malloc((size_t)n * 3 * sizeof(int32_t));
  L->src = (int32_t*)malloc((size_t)n * 18 * sizeof(int32_t));
  L->type = (uint8_t*)malloc((size_t)n);
  L->wall_normal = (float*)calloc((size_t)n * 3, sizeof(float));
  L->amp_group = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!L->xyz || !L->src || !L->type || !L->wall_normal || !L->amp_group) {
    free(raw); free(idx); return fail("out of host memory");
  }
  for (int64_t q = 0; q < n; ++q)
    for (int a = 0; a < 3; ++a) L->xyz[3 * q + a] = raw[3 * idx[q] + a];
  free(raw);
  free(idx);

  /* row starts */
  finder_t F;
  memcpy(F.lo, lo, sizeof lo);
  memcpy(F.dim, dim, sizeof dim);
  F.xyz = L->xyz;
  int64_t nrows = (int64_t)dim[1] * dim[2];
  F.row_start = (int64_t*)calloc((size_t)nrows + 1, sizeof(int64_t));
  if (!F.row_start) return fail("out of host memory");
  for (int64_t q = 0; q < n; ++q) {
    int64_t r = (int64_t)(L->xyz[3 * q + 2] - lo[2]) * dim[1] + (L->xyz[3 * q + 1] - lo[1]);
    F.row_start[r + 1]++;
  }
  for (int64_t r = 0; r < nrows; ++r) F.row_start[r + 1] += F.row_start[r];

  /* pull-source table, types, wall normals, amplitude groups */
  double (*e1)[3] = (double(*)[3])malloc(sizeof(double[3]) * (size_t)(L->n_iolets + 1));
  double (*e2)[3] = (double(*)[3])malloc(sizeof(double[3]) * (size_t)(L->n_iolets + 1));
  for (int k = 0; k < L->n_iolets; ++k) iolet_basis(&L->iolets[k], e1[k], e2[k]);

#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* p = &L->xyz[3 * q];
    int has_wall = 0, first_iolet = -1;
    double lsum[3] = {0, 0, 0};
    for (int i = 1; i < 19; ++i) {
      int64_t s = find_site(&F, p[0] - C[i][0], p[1] - C[i][1], p[2] - C[i][2]);
      int32_t code;
      if (s >= 0) {
        code = (int32_t)s;
      } else {
        /* link from p along -c_i leaves the fluid */
        int j = (i & 1) ? i + 1 : i - 1; /* opposite of i: c_j = -c_i */
        code = classify_link(L, p, j);
        if (code == -1) {
          has_wall = 1;
          for (int a = 0; a < 3; ++a) lsum[a] -= C[j][a];
        } else if (first_iolet < 0) {
          first_iolet = -code - 2;
        }
      }
      L->src[(int64_t)(i - 1) * n + q] = code;
    }
    uint8_t t = HLBG_INNER;
    if (first_iolet >= 0) {
      int outlet = L->iolets[first_iolet].role == 1;
      t = outlet ? (has_wall ? HLBG_OUTLET_WALL : HLBG_OUTLET) : (has_wall ? HLBG_INLET_WALL : HLBG_INLET);
    } else if (has_wall) {
      t = HLBG_WALL;
    }
    L->type[q] = t;

    if (has_wall) {
      double pp[3] = {p[0], p[1], p[2]}, nrm[3] = {0, 0, 0};
      int owner = -1, count = 0;
      for (int k = 0; k < ns; ++k)
        if (seg_inside(&segs[k], pp, 0.0)) { owner = k; ++count; }
      if (count == 1) {
        double qa[3];
        seg_axis_point(&segs[owner], pp, qa);
        for (int a = 0; a < 3; ++a) nrm[a] = qa[a] - pp[a];
      }
      if (dot3(nrm, nrm) < 1e-12) memcpy(nrm, lsum, sizeof nrm);
      normalize3(nrm);
      for (int a = 0; a < 3; ++a) L->wall_normal[(int64_t)a * n + q] = (float)nrm[a];
    }

    if (first_iolet >= 0) {
      /* group from the first velocity iolet this site links to */
      for (int i = 1; i < 19; ++i) {
        int32_t code = L->src[(int64_t)(i - 1) * n + q];
        if (code > -2) continue;
        int k = -code - 2;
        const hlbg_iolet* io = &L->iolets[k];
        if (io->kind != HLBG_END_VELOCITY || io->n_groups <= 1) continue;
        double v[3] = {p[0] - io->centre[0], p[1] - io->centre[1], p[2] - io->centre[2]};
        double a1 = dot3(v, e1[k]), a2 = dot3(v, e2[k]);
        double r2 = (a1 * a1 + a2 * a2) / (io->radius * io->radius);
        int ring = (int)floor(r2 * n_rings);
        if (ring < 0) ring = 0;
        if (ring >= n_rings) ring = n_rings - 1;
        double phi = atan2(a2, a1); /* (-pi, pi] */
        int sector = (int)floor((phi + M_PI) / (2 * M_PI) * n_sectors);
        if (sector < 0) sector = 0;
        if (sector >= n_sectors) sector = n_sectors - 1;
        L->amp_group[q] = ring * n_sectors + sector;
        break;
      }
    }
  }
  free(e1);
  free(e2);
  free(F.row_start);
  L->info[1] = (double)n / ((double)dim[0] * dim[1] * dim[2]);
  L->info[2] = dim[0];
  L->info[3] = dim[1];
  L->info[4] = dim[2];
  L->info[5] = ns;
  return 0;
}

/* ------------------------------------------------------------------ */
/* pipe                                                                */
/* ------------------------------------------------------------------ */
int hlbg_pipe(double radius, int32_t length, int32_t inlet_kind, int32_t outlet_kind,
              hlbg_lattice** out) {
  if (!out) return fail("null output pointer");
  *out = NULL;
  if (!(radius > 0.5) || length < 1) return fail("pipe radius must exceed 0.5 and length >= 1");
  if (inlet_kind < 0 || inlet_kind > 2 || outlet_kind < 0 || outlet_kind > 2)
    return fail("end kind must be velocity (0), pressure (1) or wall (2)");
  hlbg_lattice* L = (hlbg_lattice*)calloc(1, sizeof *L);
  if (!L) return fail("out of host memory");
  seg_t s;
  memset(&s, 0, sizeof s);
  s.a[2] = -0.5;
  s.b[2] = length - 0.5;
  s.d[2] = 1;
  s.r = radius;
  s.len = length;
  s.flat_a = s.flat_b = 1;
  s.leaf = 1;
  seg_bbox(&s);
  L->iolets = (hlbg_iolet*)calloc(2, sizeof(hlbg_iolet));
  L->iolet_seg = (int32_t*)calloc(2, sizeof(int32_t));
  int k = 0;
  if (inlet_kind != HLBG_END_WALL) {
    hlbg_iolet* io = &L->iolets[k++];
    io->kind = inlet_kind; io->role = 0;
    io->centre[2] = -0.5; io->normal[2] = 1; io->radius = radius; io->n_groups = 1;
  }
  if (outlet_kind != HLBG_END_WALL) {
    hlbg_iolet* io = &L->iolets[k++];
    io->kind = outlet_kind; io->role = 1;
    io->centre[2] = length - 0.5; io->normal[2] = -1; io->radius = radius; io->n_groups = 1;
  }
  L->n_iolets = k;
  L->info[0] = radius;
  L->info[7] = length;
  if (assemble(L, &s, 1, 1, 1)) { hlbg_free(L); return -1; }
  *out = L;
  return 0;
}

/* ------------------------------------------------------------------ */
/* seeded bifurcating tree                                             */
/* ------------------------------------------------------------------ */
typedef struct {
  double a[3], d[3], p[3]; /* start (unit-scale), direction, bifurcation-plane normal */
  double r;                /* radius relative to the root */
  int depth, leaf;
} shape_seg_t;

static void draw_shape(rng_t* rng, int depth, double lratio, shape_seg_t* out, int* count) {
  /* breadth-first in a fixed order: segment k's daughters are 2k+1, 2k+2 */
  int total = (1 << (depth + 1)) - 1;
  const double murray = pow(2.0, -1.0 / 3.0);
  shape_seg_t* root = &out[0];
  memset(root, 0, sizeof *root);
  root->d[2] = 1;
  root->p[0] = 1; /* initial bifurcation plane normal */
  root->r = 1;
  root->depth = 0;
  root->a[2] = 0;
  for (int k = 0; k < total; ++k) {
    shape_seg_t* s = &out[k];
    s->leaf = s->depth == depth;
    if (s->leaf) continue;
    double theta = (30.0 + 40.0 * rng_uniform(rng)) * M_PI / 180.0; /* full angle */
    double turn0 = (90.0 + (40.0 * rng_uniform(rng) - 20.0)) * M_PI / 180.0;
    double turn1 = (90.0 + (40.0 * rng_uniform(rng) - 20.0)) * M_PI / 180.0;
    double end[3];
    for (int a = 0; a < 3; ++a) end[a] = s->a[a] + lratio * s->r * s->d[a];
    for (int c = 0; c < 2; ++c) {
      shape_seg_t* ch = &out[2 * k + 1 + c];
      memset(ch, 0, sizeof *ch);
      double sgn = c == 0 ? 0.5 : -0.5;
      rotate3(s->d, s->p, sgn * theta, ch->d);
      normalize3(ch->d);
      double pn[3];
      rotate3(s->p, ch->d, c == 0 ? turn0 : turn1, pn);
      /* keep the plane normal perpendicular to the daughter axis */
      double pd = dot3(pn, ch->d);
      for (int a = 0; a < 3; ++a) pn[a] -= pd * ch->d[a];
      normalize3(pn);
      memcpy(ch->p, pn, sizeof pn);
      memcpy(ch->a, end, sizeof end);
      ch->r = s->r * murray;
      ch->depth = s->depth + 1;
    }
  }
  *count = total;
}

static void scale_shape(const shape_seg_t* sh, int ns, double R0, double lratio, seg_t* segs) {
  /* The unit-scale shape uses root radius 1; lengths are lratio * r.  Scale
   * about the root start, which sits on the plane z = -1/2. */
  for (int k = 0; k < ns; ++k) {
    seg_t* s = &segs[k];
    memset(s, 0, sizeof *s);
    for (int a = 0; a < 3; ++a) s->a[a] = sh[k].a[a] * R0;
    s->a[2] -= 0.5;
    memcpy(s->d, sh[k].d, sizeof s->d);
    s->r = sh[k].r * R0;
    s->len = lratio * s->r;
    for (int a = 0; a < 3; ++a) s->b[a] = s->a[a] + s->len * s->d[a];
    s->flat_a = k == 0;
    s->flat_b = sh[k].leaf;
    s->leaf = sh[k].leaf;
    s->depth = sh[k].depth;
    seg_bbox(s);
  }
}

/* Reject shapes where another segment reaches into the neighbourhood of an
 * iolet plane (where links would be mis-classified). */
static int iolets_clear(const seg_t* segs, int ns) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int k = 0; k < ns; ++k) {
    const seg_t* s = &segs[k];
    if (!(k == 0 || s->leaf)) continue;
    /* iolet plane: root start (normal +d) or leaf end (normal -d) */
    double c[3], nrm[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = k == 0 ? s->a[a] : s->b[a];
      nrm[a] = k == 0 ? s->d[a] : -s->d[a];
    }
    double e1[3], e2[3];
    hlbg_iolet tmp;
    memset(&tmp, 0, sizeof tmp);
    memcpy(tmp.normal, nrm, sizeof nrm);
    iolet_basis(&tmp, e1, e2);
    double R = s->r + 2.0;
    for (int j = 0; j < ns && !bad; ++j) {
      if (j == k) continue;
      /* quick reject by distance between bounding boxes and the disc */
      int far = 0;
      for (int a = 0; a < 3; ++a)
        if (c[a] + R + 2.0 < segs[j].lo[a] || segs[j].hi[a] < c[a] - R - 2.0) far = 1;
      if (far) continue;
      for (double h = -2.0; h <= 1.0 && !bad; h += 0.5)
        for (double u = -R; u <= R && !bad; u += 0.5)
          for (double v = -R; v <= R && !bad; v += 0.5) {
            if (u * u + v * v > R * R) continue;
            double p[3];
            for (int a = 0; a < 3; ++a) p[a] = c[a] + h * nrm[a] + u * e1[a] + v * e2[a];
            if (seg_inside(&segs[j], p, 1.5)) bad = 1;
          }
    }
  }
  return !bad;
}

int hlbg_tree(int32_t depth, uint64_t seed, int64_t target_sites, double root_radius,
              double length_ratio, int32_t n_sectors, int32_t n_rings, hlbg_lattice** out) {
  if (!out) return fail("null output pointer");
  *out = NULL;
  if (depth < 0 || depth > 10) return fail("tree depth must be in 0..10");
  if (!(length_ratio >= 2.0)) return fail("length_ratio must be >= 2");
  if (n_sectors < 1 || n_rings < 1) return fail("n_sectors and n_rings must be >= 1");
  if (target_sites <= 0 && !(root_radius > 1.0)) return fail("give target_sites > 0 or root_radius > 1");
  int ns = (1 << (depth + 1)) - 1;
  shape_seg_t* shape = (shape_seg_t*)calloc((size_t)ns, sizeof(shape_seg_t));
  seg_t* segs = (seg_t*)calloc((size_t)ns, sizeof(seg_t));
  if (!shape || !segs) { free(shape); free(segs); return fail("out of host memory"); }
  rng_t rng = {seed};
  int rejected = 0, cnt = 0;
  double R0 = root_radius;
  /* analytic volume per unit root radius: each segment is pi r^2 len + caps */
  for (int attempt = 0; attempt < 200; ++attempt) {
    draw_shape(&rng, depth, length_ratio, shape, &cnt);
    if (target_sites > 0) {
      double vol = 0;
      for (int k = 0; k < ns; ++k) vol += M_PI * shape[k].r * shape[k].r * length_ratio * shape[k].r;
      R0 = cbrt((double)target_sites / vol);
      int err = 0;
      for (int it = 0; it < 12; ++it) {
        scale_shape(shape, ns, R0, length_ratio, segs);
        int64_t c = voxelise(segs, ns, NULL, &err);
        double ratio = (double)target_sites / (double)(c > 0 ? c : 1);
        if (fabs(ratio - 1.0) < 0.005) break;
        R0 *= cbrt(ratio);
      }
    }
    scale_shape(shape, ns, R0, length_ratio, segs);
    if (iolets_clear(segs, ns)) break;
    ++rejected;
    if (attempt == 199) { free(shape); free(segs); return fail("no admissible tree shape in 200 draws"); }
  }
  hlbg_lattice* L = (hlbg_lattice*)calloc(1, sizeof *L);
  int nleaf = 1 << depth;
  L->n_iolets = 1 + nleaf;
  L->iolets = (hlbg_iolet*)calloc((size_t)L->n_iolets, sizeof(hlbg_iolet));
  L->iolet_seg = (int32_t*)calloc((size_t)L->n_iolets, sizeof(int32_t));
  if (!L || !L->iolets || !L->iolet_seg) { hlbg_free(L); free(shape); free(segs); return fail("out of host memory"); }
  hlbg_iolet* in = &L->iolets[0];
  in->kind = HLBG_END_VELOCITY;
  in->role = 0;
  memcpy(in->centre, segs[0].a, sizeof in->centre);
  memcpy(in->normal, segs[0].d, sizeof in->normal);
  in->radius = segs[0].r;
  in->n_groups = n_sectors * n_rings;
  int k = 1;
  for (int s = 0; s < ns; ++s) {
    if (!segs[s].leaf) continue;
    hlbg_iolet* io = &L->iolets[k];
    io->kind = HLBG_END_PRESSURE;
    io->role = 1;
    memcpy(io->centre, segs[s].b, sizeof io->centre);
    for (int a = 0; a < 3; ++a) io->normal[a] = -segs[s].d[a];
    io->radius = segs[s].r;
    io->n_groups = 1;
    L->iolet_seg[k] = s;
    ++k;
  }
  L->info[0] = R0;
  L->info[6] = rejected;
  L->info[7] = segs[0].len;
  int rc = assemble(L, segs, ns, n_sectors, n_rings);
  free(shape);
  free(segs);
  if (rc) { hlbg_free(L); return -1; }
  *out = L;
  return 0;
}
