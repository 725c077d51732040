// hlb_common.cuh — device-side building blocks of the D3Q19 sparse-lattice
// solver: velocity tables, shifted-population storage traits, link records,
// kernel parameters, and the per-site gather (streaming + boundaries) and
// BGK collision shared by the forward, readback and adjoint kernels.
//
// Method (arXiv 2202.11770): Section 2.2 (D3Q19, Eqs. 3a-3b, 4-6),
// Section 2.3 (bounce-back walls, Ladd velocity iolets, ghost-density
// pressure iolets), Section 3.2.3 (structure-of-arrays populations).
// Streaming is done as a pull (gather) through the streaming-index table,
// the ordering the paper's future-work list (Section 7, item 3) expects to
// be faster than its push kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlb {

constexpr int Q = 19;

// Velocity set (Section 2.2) in the order documented in hemegb.h.
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[i];
}
// Opposite pairs are adjacent: 1<->2, 3<->4, ..., 17<->18.
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// Weights 1/3, 1/18, 1/36 (Section 2.2).
template <typename R>
__host__ __device__ constexpr R wgt(int i) {
  return i == 0 ? R(1) / R(3) : (i <= 6 ? R(1) / R(18) : R(1) / R(36));
}

// ---------------------------------------------------------------------------
// Storage traits: populations are stored shifted, h = f - w.
// ---------------------------------------------------------------------------
template <typename S> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

__device__ __forceinline__ float to_real(float v) { return v; }
__device__ __forceinline__ double to_real(double v) { return v; }
__device__ __forceinline__ float to_real(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_real(__half v) { return __half2float(v); }

template <typename S> __device__ __forceinline__ S from_real(float v);
template <> __device__ __forceinline__ float from_real<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_real<__half>(float v) { return __float2half_rn(v); }
template <typename S> __device__ __forceinline__ S from_real(double v);
template <> __device__ __forceinline__ double from_real<double>(double v) { return v; }

// Programmatic dependent launch (sm_90 and later).  A step kernel lets the
// next kernel of its stream be scheduled as soon as all of its own blocks are
// resident (pdl_trigger), and waits for the previous kernel to complete, its
// memory visible, before it reads anything that kernel wrote (pdl_wait).  The
// next kernel's blocks then fill the SMs that the tail of this one frees,
// instead of waiting for the launch after it ends.  Without the launch
// attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Cached load of a population (read-only for the whole kernel).
template <typename S>
__device__ __forceinline__ typename Real<S>::type ldpop(const S* p) {
  return to_real(__ldg(p));
}
// Streaming load of the index table (read once per step, evict first).
__device__ __forceinline__ int32_t ldidx(const int32_t* p) { return __ldcs(p); }
// Streaming store of a population (next read is a full sweep later).
template <typename S>
__device__ __forceinline__ void stpop(S* p, typename Real<S>::type v) {
  __stcs(p, from_real<S>(v));
}

// ---------------------------------------------------------------------------
// Boundary links and per-launch parameters.
// ---------------------------------------------------------------------------
// One record per (site, pull direction) whose source crosses an iolet.  In
// the device index table such a link carries the code -(2 + record index).
struct LinkRec {
  int32_t site;
  int8_t dir;      // pull direction j: the source x - c_j is beyond the iolet
  int8_t kind;     // 0 velocity, 1 pressure
  int16_t iolet;
  int32_t group;   // global amplitude group (velocity), -1 otherwise
  float coef_f;    // (float) coef, rounded on the host
  double coef;     // velocity: 6 w_j W(x_m) (c_j . n); pressure: unused
};
static_assert(sizeof(LinkRec) == 24, "LinkRec is 24 bytes");

constexpr int MAX_IOLETS = 128;

// Parameters are carried in double and rounded to the compute type at use,
// so that FP64 storage sees no FP32-rounded coefficient anywhere.
struct IoletParam {
  double nx, ny, nz;
  double val;  // velocity iolet: waveform factor w(t); pressure iolet: rho(t) - 1
  float nxf, nyf, nzf, valf;  // the same rounded to float on the host
};

struct StepParams {
  int64_t n;
  int64_t sn;           // row stride of the index table: n rounded up to a multiple of 4
  double omega;         // 1 / tau
  int32_t n_iolets;
  int32_t ladd_rho_one;
  int32_t ghost_full_u;
  float omegaf;         // (float) omega, rounded on the host: FP64 arithmetic is slow on GB300
                        // (1/64 of the FP32 rate), so FP32 kernels convert no double per thread
  uint64_t coupled[MAX_IOLETS / 64];  // bit k: iolet k's value lives in ioval[k] (Windkessel outlet)
  const double* ioval;                // device, [n_iolets]: rho - 1 of coupled outlets
  const float* ampf;                  // device, [amplitude groups]: the amplitudes rounded to float
  IoletParam io[MAX_IOLETS];
};
static_assert(MAX_IOLETS % 64 == 0, "coupling mask words");

// Division of a block number b < 2^31 by a fixed divisor d without an
// integer divide in the kernel: q = (b >> s) for d a power of two (m = 0),
// else q = umulhi(b, m) >> s with l = ceil(log2 d), m = ceil(2^(31+l) / d),
// s = l - 1, which is exact for all b < 2^31 (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994: m d lies in
// [2^(31+l), 2^(31+l) + 2^l]).
struct BlockDiv {
  uint32_t d, m, s;
};
inline BlockDiv make_block_div(uint32_t d) {
  BlockDiv r{d, 0u, 0u};
  if ((d & (d - 1)) == 0) {
    while ((1u << r.s) < d) ++r.s;
    return r;
  }
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;  // ceil(log2 d)
  r.m = (uint32_t)((((uint64_t)1 << (31 + l)) + d - 1) / d);
  r.s = l - 1;
  return r;
}
__device__ __forceinline__ uint32_t block_div(uint32_t b, const BlockDiv& q) {
  return q.m == 0 ? (b >> q.s) : (__umulhi(b, q.m) >> q.s);
}

// Relaxation rate 1/tau in the arithmetic type of a kernel.
template <typename R> __device__ __forceinline__ R omega_of(const StepParams& p);
template <> __device__ __forceinline__ float omega_of<float>(const StepParams& p) { return p.omegaf; }
template <> __device__ __forceinline__ double omega_of<double>(const StepParams& p) { return p.omega; }

// Boundary value of iolet k for this launch: the host waveform, or for a
// Windkessel outlet the ghost density the device-side model last produced.
__device__ __forceinline__ double io_val(const StepParams& p, int k) {
  return ((p.coupled[k >> 6] >> (k & 63)) & 1ull) ? p.ioval[k] : p.io[k].val;
}

// Boundary data in the arithmetic type R of a kernel.  FP32 kernels read
// copies rounded to float on the host (or, for a Windkessel outlet's ghost
// density, once on the device): the value is the one R(x) would give, without
// a conversion from double per use (FP64 arithmetic runs at 1/64 of the FP32
// rate on GB300).
template <typename R> struct BC;
template <> struct BC<float> {
  static __device__ __forceinline__ float val(const StepParams& p, int k) {
    return ((p.coupled[k >> 6] >> (k & 63)) & 1ull) ? (float)p.ioval[k] : p.io[k].valf;
  }
  static __device__ __forceinline__ float coef(const LinkRec& L) { return L.coef_f; }
  static __device__ __forceinline__ float amp(const StepParams& p, const double*, int g) { return p.ampf[g]; }
  static __device__ __forceinline__ float nx(const IoletParam& q) { return q.nxf; }
  static __device__ __forceinline__ float ny(const IoletParam& q) { return q.nyf; }
  static __device__ __forceinline__ float nz(const IoletParam& q) { return q.nzf; }
};
template <> struct BC<double> {
  static __device__ __forceinline__ double val(const StepParams& p, int k) { return io_val(p, k); }
  static __device__ __forceinline__ double coef(const LinkRec& L) { return L.coef; }
  static __device__ __forceinline__ double amp(const StepParams&, const double* a, int g) { return a[g]; }
  static __device__ __forceinline__ double nx(const IoletParam& q) { return q.nx; }
  static __device__ __forceinline__ double ny(const IoletParam& q) { return q.ny; }
  static __device__ __forceinline__ double nz(const IoletParam& q) { return q.nz; }
};

// ---------------------------------------------------------------------------
// Moments and equilibrium in shifted form.
//   rho = 1 + drho, drho = sum h_i;  j = sum h_i c_i;  u = j / rho
//   f^eq_i - w_i = w_i (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u))
// which is Eq. 4 with the factors 1/2 (cs2 = 1/3).
// ---------------------------------------------------------------------------
template <typename R>
struct Macro {
  R drho, rho, ux, uy, uz;
};

template <typename R>
__device__ __forceinline__ Macro<R> moments(const R* h) {
  R d = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    d += h[i];
    if (cx(i)) jx += cx(i) > 0 ? h[i] : -h[i];
    if (cy(i)) jy += cy(i) > 0 ? h[i] : -h[i];
    if (cz(i)) jz += cz(i) > 0 ? h[i] : -h[i];
  }
  Macro<R> m;
  m.drho = d;
  m.rho = R(1) + d;
  R inv = R(1) / m.rho;
  m.ux = jx * inv;
  m.uy = jy * inv;
  m.uz = jz * inv;
  return m;
}

template <typename R>
__device__ __forceinline__ R cdotu(int i, R ux, R uy, R uz) {
  R s = R(0);
  if (cx(i)) s += cx(i) > 0 ? ux : -ux;
  if (cy(i)) s += cy(i) > 0 ? uy : -uy;
  if (cz(i)) s += cz(i) > 0 ? uz : -uz;
  return s;
}

// Shifted equilibrium of direction i at (drho, rho, u).
template <typename R>
__device__ __forceinline__ R heq(int i, R drho, R rho, R ux, R uy, R uz, R usq15) {
  R cu = cdotu<R>(i, ux, uy, uz);
  return wgt<R>(i) * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - usq15));
}

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// BGK collision (Eq. 3a, dt = 1): h'_i = h_i + omega (heq_i - h_i), handed to
// emit(i, h'_i) direction by direction as each value is final.  Arranged by
// opposite pairs (2p+1, 2p+2), whose c.u differ in sign only:
//  * pair sums and differences give drho = h_0 + sum (h_2p+1 + h_2p+2) and
//    j = sum (h_2p+1 - h_2p+2) c_{2p+1};
//  * a pair shares a = 4.5 (c.u)^2 - 1.5 u.u, and its two equilibria are
//    w (drho + rho (a +- 3 c.u));
//  * h' = (1 - omega) h + omega heq, with omega w rho and omega w drho formed
//    once per weight class, is two fused multiply-adds per direction.
// About 140 FP32 instructions a site against 210 for the direction-by-
// direction form, in kernels whose 16-bit variants are issue-bound; emitting
// each pair as soon as it is final lets a kernel store it and free its
// registers.
template <typename R, typename Emit>
__device__ __forceinline__ void collide_emit(const R* h, R omega, Emit&& emit) {
  R drho = h[0], jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const int i = 2 * p + 1;
    const R sp = h[i] + h[i + 1], dp = h[i] - h[i + 1];
    drho += sp;
    if (cx(i)) jx = cx(i) > 0 ? jx + dp : jx - dp;
    if (cy(i)) jy = cy(i) > 0 ? jy + dp : jy - dp;
    if (cz(i)) jz = cz(i) > 0 ? jz + dp : jz - dp;
  }
  const R rho = R(1) + drho;
  const R inv = R(1) / rho;
  const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
  const R usq15 = R(1.5) * fmadd(uz, uz, fmadd(uy, uy, ux * ux));
  const R om1 = R(1) - omega;
  R wr[3], wd[3];  // omega w rho, omega w drho for w = 1/3, 1/18, 1/36
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R ow = omega * wgt<R>(c == 0 ? 0 : (c == 1 ? 1 : 7));
    wr[c] = ow * rho;
    wd[c] = ow * drho;
  }
  emit(0, fmadd(om1, h[0], fmadd(-wr[0], usq15, wd[0])));
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const int i = 2 * p + 1, c = i <= 6 ? 1 : 2;
    const R cu = cdotu<R>(i, ux, uy, uz);
    const R a = fmadd(R(4.5) * cu, cu, -usq15);
    emit(i, fmadd(om1, h[i], fmadd(wr[c], fmadd(R(3), cu, a), wd[c])));
    emit(i + 1, fmadd(om1, h[i + 1], fmadd(wr[c], fmadd(R(-3), cu, a), wd[c])));
  }
}

// The collision in place.
template <typename R>
__device__ __forceinline__ void collide(R* h, R omega) {
  R out[Q];
  collide_emit<R>(h, omega, [&](int i, R v) { out[i] = v; });
#pragma unroll
  for (int i = 0; i < Q; ++i) h[i] = out[i];
}

// ---------------------------------------------------------------------------
// Gather of the pre-collision state f(t) at site x from the post-collision
// state s'(t-1) (pull streaming, Eq. 3b) with boundaries:
//   fluid source:   h_i = s'_i(x - c_i)
//   wall link:      h_i = s'_ibar(x)                         (bounce-back)
//   velocity iolet: h_i = s'_ibar(x) + coef rho_s A          (Ladd)
//   pressure iolet: h_i = f^eq_i(rho_k, u_g) - w_i           (ghost density)
// rho_s, u_s are the moments of s'(t-1) at x: BGK conserves mass and
// momentum, so they equal the pre-collision moments at time t-1 that the
// paper's push formulation uses for these boundaries.
// Returns whether the site has an iolet link.
// ---------------------------------------------------------------------------
template <typename S>
__device__ __forceinline__ bool gather_site(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                            int64_t n, int64_t sn, int64_t x, typename Real<S>::type* h) {
  h[0] = ldpop(fin + x);
  bool any_iolet = false;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int32_t s = ldidx(src + (int64_t)(i - 1) * sn + x);
    int64_t a = s >= 0 ? (int64_t)i * n + s : (int64_t)opp(i) * n + x;
    h[i] = ldpop(fin + a);
    any_iolet |= s <= -2;
  }
  return any_iolet;
}

// Boundary values of iolet links at site x (rare: only iolet sites).  On
// entry h[i] of an iolet link already holds s'_ibar(x) (the gather selects
// the own opposite slot for every non-fluid source).  All index codes and
// link records are loaded up front, independently of each other, so the
// loads overlap instead of forming a chain per direction.
template <typename S>
__device__ __forceinline__ void iolet_fixup(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                            const LinkRec* __restrict__ links, const double* __restrict__ amp,
                                            const StepParams& p, int64_t x, typename Real<S>::type* h) {
  using R = typename Real<S>::type;
  const int64_t n = p.n;
  int32_t code[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) code[i] = src[(int64_t)(i - 1) * p.sn + x];
  // moments of the site's own post-collision state s'(t-1)
  R d = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R v = ldpop(fin + (int64_t)i * n + x);
    d += v;
    if (cx(i)) jx += cx(i) > 0 ? v : -v;
    if (cy(i)) jy += cy(i) > 0 ? v : -v;
    if (cz(i)) jz += cz(i) > 0 ? v : -v;
  }
  const R rho_s = R(1) + d;
  const R ux = jx / rho_s, uy = jy / rho_s, uz = jz / rho_s;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const bool io = code[i] <= -2;
    const LinkRec L = links[io ? -code[i] - 2 : 0];       // record 0 exists whenever a site has an iolet link
    const R a = BC<R>::amp(p, amp, L.kind == 0 && L.group >= 0 ? L.group : 0);
    if (!io) continue;
    const IoletParam& iop = p.io[L.iolet];
    if (L.kind == 0) {
      R rho = p.ladd_rho_one ? R(1) : rho_s;
      h[i] += BC<R>::coef(L) * rho * a * BC<R>::val(p, L.iolet);
    } else {
      R gx = ux, gy = uy, gz = uz;
      if (!p.ghost_full_u) {
        R un = gx * BC<R>::nx(iop) + gy * BC<R>::ny(iop) + gz * BC<R>::nz(iop);
        gx = un * BC<R>::nx(iop);
        gy = un * BC<R>::ny(iop);
        gz = un * BC<R>::nz(iop);
      }
      R drho = BC<R>::val(p, L.iolet);
      R usq15 = R(1.5) * (gx * gx + gy * gy + gz * gz);
      h[i] = heq<R>(i, drho, R(1) + drho, gx, gy, gz, usq15);
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-cooperative boundary sites: a lane per direction (the adjoint: one
// warp a site, lanes 19..31 idle; the forward kernels: a half-warp a site,
// three lanes holding two directions).  Moments are summed by a shuffle loop
// in direction order with exactly the operations of the per-thread code
// above, so a site gets bit-identical values whichever path processes it.
// ---------------------------------------------------------------------------
constexpr unsigned FULL_MASK = 0xffffffffu;
static __constant__ int8_t k_cx[32] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static __constant__ int8_t k_cy[32] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static __constant__ int8_t k_cz[32] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

__device__ __forceinline__ int lane_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <typename R>
__device__ __forceinline__ R lane_w(int i) {
  return i == 0 ? R(1) / R(3) : (i <= 6 ? R(1) / R(18) : R(1) / R(36));
}
template <typename R>
__device__ __forceinline__ R lane_cdotu(int i, R ux, R uy, R uz) {
  R s = R(0);
  if (k_cx[i]) s += k_cx[i] > 0 ? ux : -ux;
  if (k_cy[i]) s += k_cy[i] > 0 ? uy : -uy;
  if (k_cz[i]) s += k_cz[i] > 0 ? uz : -uz;
  return s;
}
template <typename R>
__device__ __forceinline__ R lane_heq(int i, R drho, R rho, R ux, R uy, R uz, R usq15) {
  R cu = lane_cdotu<R>(i, ux, uy, uz);
  return lane_w<R>(i) * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - usq15));
}
// (sum v, sum v c) over lanes 0..18 in direction order; sgn = -1 sums -v c
template <typename R>
__device__ __forceinline__ void lane_moment_sums(R v, R sgn, R* d, R* jx, R* jy, R* jz) {
  R a = R(0), x = R(0), y = R(0), z = R(0);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const R vk = __shfl_sync(FULL_MASK, v, k);
    a += vk;
    if (cx(k)) x += (cx(k) > 0) == (sgn > R(0)) ? vk : -vk;
    if (cy(k)) y += (cy(k) > 0) == (sgn > R(0)) ? vk : -vk;
    if (cz(k)) z += (cz(k) > 0) == (sgn > R(0)) ? vk : -vk;
  }
  *d = a; *jx = x; *jy = y; *jz = z;
}
// Boundary value of the lane's iolet link (as iolet_fixup computes it):
// `out` = s'_ibar(x); rho_s, u_s the moments of the stored post-collision state.
template <typename R>
__device__ __forceinline__ R lane_iolet_value(int i, const LinkRec& L, R out, R rho_s, R ux, R uy, R uz, R a,
                                              const StepParams& p) {
  const IoletParam& iop = p.io[L.iolet];
  if (L.kind == 0) {
    R rho = p.ladd_rho_one ? R(1) : rho_s;
    return out + BC<R>::coef(L) * rho * a * BC<R>::val(p, L.iolet);
  }
  R gx = ux, gy = uy, gz = uz;
  if (!p.ghost_full_u) {
    R un = gx * BC<R>::nx(iop) + gy * BC<R>::ny(iop) + gz * BC<R>::nz(iop);
    gx = un * BC<R>::nx(iop);
    gy = un * BC<R>::ny(iop);
    gz = un * BC<R>::nz(iop);
  }
  R drho = BC<R>::val(p, L.iolet);
  R usq15 = R(1.5) * (gx * gx + gy * gy + gz * gz);
  return lane_heq<R>(i, drho, R(1) + drho, gx, gy, gz, usq15);
}

// ---------------------------------------------------------------------------
// Reading f(t) from a population buffer (read modes of hlb_internal.h:
// 0 = in place, 1 = pull A-B gather with boundaries, 2 = AA gather).
// ---------------------------------------------------------------------------
// Address of slot i of site x in an odd step (and in an AA read-back): the
// population arriving along c_i was written by the source x - c_i into its
// opposite slot, or, for a non-fluid source, by x itself into slot i.
__device__ __forceinline__ int64_t aa_addr(int i, int32_t s, int64_t n, int64_t x) {
  return s >= 0 ? (int64_t)opp(i) * n + s : (int64_t)i * n + x;
}

template <typename S, int MODE>
__device__ __forceinline__ void load_state(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                           const LinkRec* __restrict__ links, const double* __restrict__ amp,
                                           const StepParams& p, int64_t x, typename Real<S>::type* h) {
  if (MODE == 1) {
    if (gather_site<S>(fin, src, p.n, p.sn, x, h)) iolet_fixup<S>(fin, src, links, amp, p, x, h);
  } else if (MODE == 2) {
    h[0] = ldpop(fin + x);
#pragma unroll
    for (int i = 1; i < Q; ++i) h[i] = ldpop(fin + aa_addr(i, src[(int64_t)(i - 1) * p.sn + x], p.n, x));
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldpop(fin + (int64_t)i * p.n + x);
  }
}

// ---------------------------------------------------------------------------
// Offsets of the hot kernels.  A thread keeps up to 18 slot offsets in
// registers, so they are 32-bit.  With WIDE = false (19 x the index row
// stride below 2^32, about 226M sites) an offset is the element offset from
// the array base.  With WIDE = true it is the offset within the direction
// pair (2p-1, 2p), p = (i + 1) / 2, whose two rows are contiguous and start
// at element (2p - 1) n: every gather or store of a step touches only
// direction i and opp(i), both in that pair, and offsets there stay below
// 2n < 2^32 for any lattice of fewer than 2^31 sites.  The 64-bit pair start
// is added when the address is formed.
// ---------------------------------------------------------------------------
// offset of row `row` (i or opp(i), i >= 1) at site e
template <bool WIDE>
__device__ __forceinline__ uint32_t slot(int row, uint32_t n, uint32_t e) {
  return WIDE ? ((row & 1) ? e : n + e) : (uint32_t)row * n + e;
}
// address of a slot of direction i's pair
template <bool WIDE, typename T>
__device__ __forceinline__ T* at(T* a, int i, uint32_t n, uint32_t off) {
  return WIDE ? a + ((uint64_t)(2 * ((i + 1) >> 1) - 1) * n + off) : a + off;
}
// index code of direction i >= 1 at site x (rows of stride sn)
template <bool WIDE>
__device__ __forceinline__ const int32_t* idx_at(const int32_t* src, int i, uint32_t sn, uint32_t x) {
  return WIDE ? src + ((uint64_t)(i - 1) * sn + x) : src + (uint32_t)(i - 1) * sn + x;
}

// ---------------------------------------------------------------------------
// Compact index table.  The lattice is ordered lexicographically by (z, y, x)
// and x - c_i keeps that order, so over a tile of CT_TILE consecutive sites
// the fluid sources of one direction increase with the site index, and in
// vessel lattices they span a few hundred sites.  Per tile and direction the
// table keeps the smallest fluid source (tbase[tile][i - 1], CT_BASES int32
// entries a tile, the last two unused), and per site and direction a 16-bit
// offset from it, or CT_WALL / CT_IOLET for a link without a fluid source.
// Directions 2p + 1 (low half) and 2p + 2 (high half) share one 32-bit word
// in row p of ctab (rows of stride sn): 36 bytes a site instead of the 72 of
// the 32-bit table.  A lattice with a span above CT_MAX_SPAN uses the 32-bit
// table (the same kernels with CT = false).
// ---------------------------------------------------------------------------
constexpr uint32_t CT_WALL = 0xffffu, CT_IOLET = 0xfffeu, CT_MAX_SPAN = 0xfffdu;
constexpr int CT_TILE = 256, CT_BASES = 20;

// How a kernel loads its index entries: read-only cached, streaming (read
// once, evict first), or cached in L1 for a re-read by the same thread.
enum { LD_NC = 0, LD_STREAM = 1, LD_L1 = 2 };
template <int LD, typename T>
__device__ __forceinline__ T ld_index(const T* p) {
  return LD == LD_STREAM ? __ldcs(p) : (LD == LD_L1 ? __ldca(p) : __ldg(p));
}

// The 18 index codes s[i - 1] of site x (tile `tile` of the compact table):
// a fluid source's index, -1 across a wall, and for an iolet link the
// re-coded record (32-bit table) or -2 (compact table).
template <bool CT, bool WIDE, int LD>
__device__ __forceinline__ void load_codes(const int32_t* __restrict__ src, const uint32_t* __restrict__ ctab,
                                           const int32_t* __restrict__ tbase, uint32_t sn, uint32_t x,
                                           uint32_t tile, int32_t* s) {
  if (CT) {
    uint32_t w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = ld_index<LD>(WIDE ? ctab + ((uint64_t)q * sn + x) : ctab + (uint32_t)q * sn + x);
    const int4* tb = reinterpret_cast<const int4*>(tbase + (uint64_t)tile * CT_BASES);
    int b[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int4 v = __ldg(tb + q);
      b[4 * q] = v.x;
      b[4 * q + 1] = v.y;
      b[4 * q + 2] = v.z;
      b[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t o = (i & 1) ? (w[(i - 1) >> 1] & 0xffffu) : (w[(i - 1) >> 1] >> 16);
      s[i - 1] = o < CT_IOLET ? (int32_t)((uint32_t)b[i - 1] + o) : (o == CT_WALL ? -1 : -2);
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) s[i - 1] = ld_index<LD>(idx_at<WIDE>(src, i, sn, x));
  }
}

// The 18 population offsets a bulk step kernel gathers from at site x (off[i],
// i = 1..18): for a fluid source s the slot of row i at s (pull; AAODD: row
// opp(i) at s), otherwise row opp(i) at x itself (AAODD: row i at x), which is
// bounce-back (iolet links get their values elsewhere).  From the compact
// table a link is fluid exactly when its offset is below CT_IOLET, so the
// offset goes straight into the slot without forming a signed code.
template <bool CT, bool WIDE, int LD, bool AAODD>
__device__ __forceinline__ void load_offsets(const int32_t* __restrict__ src, const uint32_t* __restrict__ ctab,
                                             const int32_t* __restrict__ tbase, uint32_t sn, uint32_t n, uint32_t x,
                                             uint32_t tile, uint32_t* off) {
  if (CT) {
    uint32_t w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = ld_index<LD>(WIDE ? ctab + ((uint64_t)q * sn + x) : ctab + (uint32_t)q * sn + x);
    const int4* tb = reinterpret_cast<const int4*>(tbase + (uint64_t)tile * CT_BASES);
    int b[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int4 v = __ldg(tb + q);
      b[4 * q] = v.x;
      b[4 * q + 1] = v.y;
      b[4 * q + 2] = v.z;
      b[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t o = (i & 1) ? (w[(i - 1) >> 1] & 0xffffu) : (w[(i - 1) >> 1] >> 16);
      off[i] = o < CT_IOLET ? slot<WIDE>(AAODD ? opp(i) : i, n, (uint32_t)b[i - 1] + o)
                            : slot<WIDE>(AAODD ? i : opp(i), n, x);
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int32_t s = ld_index<LD>(idx_at<WIDE>(src, i, sn, x));
      off[i] = s >= 0 ? slot<WIDE>(AAODD ? opp(i) : i, n, (uint32_t)s) : slot<WIDE>(AAODD ? i : opp(i), n, x);
    }
  }
}

}  // namespace hlb
