// hlb_adjoint.cu — discrete adjoint of the fused step with sqrt(N)
// checkpointing (no counterpart in arXiv 2202.11770; it differentiates the
// paper's LBGK step, Eqs. 3a-3b and 4-6, with its Section 2.3 boundaries).
//
// Forward map (pull form, as run by k_step):
//   s'(t)   = C(f(t))                 BGK collision, Eq. 3a
//   f(t+1)  = G_t(s'(t))              gather through the index table with
//                                     bounce-back / Ladd / pressure values
//   J       = (1/N) sum_{t=1..N} sum_p (u(x_p, t).axis - target_p)^2
// Adjoint (mu = dJ/df, lam = dJ/ds'):
//   lam(t)  = G_t^T mu(t+1)
//   mu(t)   = C'(f(t))^T lam(t) + dJ/df(t)
//   dJ/dtau = sum_t lam(t) . dC/dtau = sum_t omega^2 lam(t) . (f(t) - feq)
//   dJ/da_g = sum_t mu(t+1) . dG_t/da_g
// G_t^T is itself a gather: s'_i(x) is read by the site x + c_i, whose
// index is src[opp(i)][x], or (boundary link) by x itself in direction
// opp(i).  One kernel per reverse step reads the index table and gathers
// both mu(t+1) and s'(t-1) (to recompute f(t)), from one decode of the
// index (the compact table when the lattice fits it).  J itself is summed in
// the reverse sweep too, where f(t)'s moments are at hand, so the forward
// sweep runs the plain step kernels of the solver's scheme and nothing else.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "hlb_internal.h"

using namespace hlb;

namespace {

constexpr int BLOCK = 256;
inline unsigned grid_for(int64_t n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

// Probe sites as a bit mask over sites plus per-32-site prefix counts: site
// x is probe k when bit x of mask is set, k = base[x / 32] + popcount(mask
// bits of its word below x).  Lets the reverse kernels evaluate the
// objective and add dJ/df(t) at the probes without launches of their own.
struct ProbeMap {
  const uint32_t* mask;
  const int32_t* base;
  const double* target;  // ordered by site
  double* jp;            // per-probe objective accumulators, ordered by site
  double ax, ay, az;
  double inv_n;          // 1 / N
  float axf, ayf, azf;   // the axis rounded to float on the host (FP32 kernels)
};

// The probe axis in the arithmetic type of a kernel.
template <typename R> __device__ __forceinline__ void probe_axis(const ProbeMap& pm, R* a);
template <> __device__ __forceinline__ void probe_axis<float>(const ProbeMap& pm, float* a) {
  a[0] = pm.axf; a[1] = pm.ayf; a[2] = pm.azf;
}
template <> __device__ __forceinline__ void probe_axis<double>(const ProbeMap& pm, double* a) {
  a[0] = pm.ax; a[1] = pm.ay; a[2] = pm.az;
}

// At a probe, with d = u(t).axis - target: J gains d^2 / N (when add_j) and
// dJ/df_j(t) = pg (c_j . axis - u_ax) with pg = 2 d / (N rho).  pg = 0 off
// the probes.
template <typename R>
__device__ __forceinline__ R probe_term(const ProbeMap& pm, int64_t x, const Macro<R>& m, R* uax, bool add_j) {
  const uint32_t word = pm.mask[x >> 5];
  const uint32_t bit = (uint32_t)(x & 31);
  *uax = R(0);
  if (!((word >> bit) & 1u)) return R(0);
  const int k = pm.base[x >> 5] + __popc(word & ((1u << bit) - 1u));
  const double ua = (double)m.ux * pm.ax + (double)m.uy * pm.ay + (double)m.uz * pm.az;
  const double d = ua - pm.target[k];
  if (add_j) pm.jp[k] += d * d * pm.inv_n;
  *uax = R(ua);
  return R(2.0 * pm.inv_n * d) / m.rho;
}

struct AdjParams {
  StepParams prev;            // boundary data of G_{t-1} (recomputing f(t))
  double val_cur[MAX_IOLETS];  // waveform values of G_t (velocity w, pressure rho - 1)
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  __syncthreads();
  return r;
}

// Sum over a block in the arithmetic type R (fixed order): warp xor
// butterflies, then thread 0 adds the warps' sums in order.  Valid in thread 0.
template <typename R>
__device__ __forceinline__ R block_sum_r(R v, R* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  R r = R(0);
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;
}

// Offsets of the two gathers of a reverse step at site x.  off[i] is the
// slot f_i(x, t) is gathered from: row i at the fluid source s = x - c_i, or
// row opp(i) at x itself (boundary link); bit i of *fluid says which.  The
// adjoint gather of mu(t+1) reads, for direction i, row opp(i) at s (fluid)
// or row i at x: in both offset forms that is off[i] + n when the link is
// fluid and i is odd or the link is not fluid and i is even, and off[i] - n
// otherwise (mu_offset), so one decode of the index serves both gathers.
template <bool CT, bool WIDE>
__device__ __forceinline__ void reverse_offsets(const int32_t* __restrict__ src, const uint32_t* __restrict__ ctab,
                                                const int32_t* __restrict__ tbase, uint32_t sn, uint32_t n,
                                                uint32_t x, uint32_t tile, uint32_t* off, uint32_t* fluid) {
  uint32_t fl = 0;
  if (CT) {
    uint32_t w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = __ldg(WIDE ? ctab + ((uint64_t)q * sn + x) : ctab + (uint32_t)q * sn + x);
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
      const bool f = o < CT_IOLET;
      off[i] = f ? slot<WIDE>(i, n, (uint32_t)b[i - 1] + o) : slot<WIDE>(opp(i), n, x);
      fl |= f ? 1u << i : 0u;
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int32_t s = __ldg(idx_at<WIDE>(src, i, sn, x));
      off[i] = s >= 0 ? slot<WIDE>(i, n, (uint32_t)s) : slot<WIDE>(opp(i), n, x);
      fl |= s >= 0 ? 1u << i : 0u;
    }
  }
  *fluid = fl;
}
__device__ __forceinline__ uint32_t mu_offset(uint32_t off, uint32_t fluid, int i, uint32_t n) {
  return (((fluid >> i) & 1u) == (uint32_t)(i & 1)) ? off + n : off - n;
}

// Bulk reverse step over all sites without iolet links, one site per
// thread.  f(t) is gathered from s'(t-1) first (GPREV; otherwise it is read
// in place from a checkpoint); its moments are kept and its non-equilibrium
// parts h_i - heq_i are parked in shared memory, so that the 19 gathered
// values of mu(t+1) can reuse the registers.  Then lam = G_t^T mu(t+1) and
// mu_j(t) = (1 - omega) lam_j + omega (S0 + (c_j - u).B) plus the probe term,
// with S0 = sum lam_i feq_i / rho, B = sum lam_i w_i (3 + 9 c_i.u) c_i - 3 u L,
// L = sum lam_i w_i.  Like the forward collision, the sums run over opposite
// pairs, whose c.u differ in sign only: a pair adds w (s (1 + a) + 3 c.u d) to
// S0, w s to L and w (3 d + 9 c.u s) c to B, with s and d the pair's sum and
// difference of lam.  The index is decoded once for both gathers
// (reverse_offsets).  Measured and dropped: both gathers issued at once as
// asynchronous copies into shared memory (5 instead of 4 blocks per SM, no
// faster), both gathers in registers (no parked parts, 3 or 2 blocks per SM),
// and the index rows staged in shared memory with bulk copies.
template <typename S, bool GPREV, bool WIDE, bool CT>
__device__ __forceinline__ typename Real<S>::type adjoint_site(const S* __restrict__ prev, const S* __restrict__ mu_next,
                                                               S* __restrict__ mu_out, const int32_t* __restrict__ src,
                                                               const uint32_t* __restrict__ ctab,
                                                               const int32_t* __restrict__ tbase,
                                                               const uint32_t* __restrict__ imask,
                                                               const AdjParams& ap, const ProbeMap& pm, int store,
                                                               int64_t x, uint32_t tile,
                                                               typename Real<S>::type (*neq)[BLOCK]) {
  using R = typename Real<S>::type;
  const uint32_t n = (uint32_t)ap.prev.n, sn = (uint32_t)ap.prev.sn, xi = (uint32_t)x;
  const R omega = omega_of<R>(ap.prev);
  if (x >= ap.prev.n) return R(0);
  if ((__ldg(imask + (xi >> 5)) >> (xi & 31)) & 1u) return R(0);  // iolet sites: adjoint_iolet_site
  uint32_t off[Q], fluid;
  reverse_offsets<CT, WIDE>(src, ctab, tbase, sn, n, xi, tile, off, &fluid);
  pdl_wait();  // the states below were written by the kernels before this one
  pdl_trigger();
  R drho, rho, ux, uy, uz, usq15;
  {
    R h[Q];
    h[0] = ldpop(prev + xi);
#pragma unroll
    for (int i = 1; i < Q; ++i) h[i] = ldpop(at<WIDE>(prev, i, n, GPREV ? off[i] : slot<WIDE>(i, n, xi)));
    drho = h[0];
    R jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int i = 2 * p + 1;
      const R dp = h[i] - h[i + 1];
      drho += h[i] + h[i + 1];
      if (cx(i)) jx = cx(i) > 0 ? jx + dp : jx - dp;
      if (cy(i)) jy = cy(i) > 0 ? jy + dp : jy - dp;
      if (cz(i)) jz = cz(i) > 0 ? jz + dp : jz - dp;
    }
    rho = R(1) + drho;
    const R inv = R(1) / rho;
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
    usq15 = R(1.5) * fmadd(uz, uz, fmadd(uy, uy, ux * ux));
    neq[0][threadIdx.x] = h[0] - wgt<R>(0) * fmadd(-rho, usq15, drho);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int i = 2 * p + 1;
      const R w = wgt<R>(i), cu = cdotu<R>(i, ux, uy, uz);
      const R a = fmadd(R(4.5) * cu, cu, -usq15);
      neq[i][threadIdx.x] = h[i] - w * fmadd(rho, fmadd(R(3), cu, a), drho);
      neq[i + 1][threadIdx.x] = h[i + 1] - w * fmadd(rho, fmadd(R(-3), cu, a), drho);
    }
  }
  R lam[Q];
  lam[0] = ldpop(mu_next + xi);
#pragma unroll
  for (int i = 1; i < Q; ++i) lam[opp(i)] = ldpop(at<WIDE>(mu_next, i, n, mu_offset(off[i], fluid, i, n)));
  // sums per weight class (1: axis pairs, 2: diagonal pairs)
  R S1 = R(0), S2 = R(0), L1 = R(0), L2 = R(0), B1x = R(0), B1y = R(0), B1z = R(0), B2x = R(0), B2y = R(0),
    B2z = R(0), dt = lam[0] * neq[0][threadIdx.x];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const int i = 2 * p + 1;
    const R sp = lam[i] + lam[i + 1], dp = lam[i] - lam[i + 1];
    const R cu = cdotu<R>(i, ux, uy, uz);
    const R a = fmadd(R(4.5) * cu, cu, -usq15);
    const R sv = fmadd(R(3) * cu, dp, sp * (R(1) + a));
    const R q = fmadd(R(9) * cu, sp, R(3) * dp);
    dt = fmadd(lam[i], neq[i][threadIdx.x], dt);
    dt = fmadd(lam[i + 1], neq[i + 1][threadIdx.x], dt);
    if (i <= 6) {
      S1 += sv;
      L1 += sp;
      if (cx(i)) B1x += cx(i) > 0 ? q : -q;
      if (cy(i)) B1y += cy(i) > 0 ? q : -q;
      if (cz(i)) B1z += cz(i) > 0 ? q : -q;
    } else {
      S2 += sv;
      L2 += sp;
      if (cx(i)) B2x += cx(i) > 0 ? q : -q;
      if (cy(i)) B2y += cy(i) > 0 ? q : -q;
      if (cz(i)) B2z += cz(i) > 0 ? q : -q;
    }
  }
  const R w0 = wgt<R>(0), w1 = wgt<R>(1), w2 = wgt<R>(7);
  const R S0 = fmadd(w0 * lam[0], R(1) - usq15, fmadd(w1, S1, w2 * S2));
  const R Lw = fmadd(w0, lam[0], fmadd(w1, L1, w2 * L2));
  const R Bx = fmadd(w1, B1x, w2 * B2x) - R(3) * ux * Lw;
  const R By = fmadd(w1, B1y, w2 * B2y) - R(3) * uy * Lw;
  const R Bz = fmadd(w1, B1z, w2 * B2z) - R(3) * uz * Lw;
  const R dtau_local = omega * omega * dt;
  if (store) {
    // mu_j = (1-omega) lam_j + omega (S0 + (c_j - u).B) + pg (c_j - u).axis
    //      = (1-omega) lam_j + T0 + c_j.E
    R uax, ax[3];
    probe_axis<R>(pm, ax);
    Macro<R> m;
    m.drho = drho;
    m.rho = rho;
    m.ux = ux;
    m.uy = uy;
    m.uz = uz;
    const R pg = probe_term<R>(pm, x, m, &uax, true);
    const R Ex = omega * Bx + pg * ax[0], Ey = omega * By + pg * ax[1], Ez = omega * Bz + pg * ax[2];
    const R T0 = omega * (S0 - ux * Bx - uy * By - uz * Bz) - pg * uax;
    const R om1 = R(1) - omega;
    *(mu_out + xi) = from_real<S>(fmadd(om1, lam[0], T0));
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int i = 2 * p + 1;
      const R ce = cdotu<R>(i, Ex, Ey, Ez);
      *at<WIDE>(mu_out, i, n, slot<WIDE>(i, n, xi)) = from_real<S>(fmadd(om1, lam[i], T0 + ce));
      *at<WIDE>(mu_out, i, n, slot<WIDE>(i + 1, n, xi)) = from_real<S>(fmadd(om1, lam[i + 1], T0 - ce));
    }
  }
  return dtau_local;
}

// Warp sums for the iolet-site reverse kernel: xor butterflies (5 shuffles a
// sum).  Each level adds the same two partials on both lanes of a pair, so
// every lane ends with identical bits.  Lanes 19..31 must hold 0.
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}
// (sum v, sum v c) with lane i holding v for direction i
template <typename R>
__device__ __forceinline__ void warp_moment_sums(R v, int i, R* d, R* jx, R* jy, R* jz) {
  R a = v, x = k_cx[i] ? (k_cx[i] > 0 ? v : -v) : R(0), y = k_cy[i] ? (k_cy[i] > 0 ? v : -v) : R(0),
    z = k_cz[i] ? (k_cz[i] > 0 ? v : -v) : R(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(FULL_MASK, a, o);
    x += __shfl_xor_sync(FULL_MASK, x, o);
    y += __shfl_xor_sync(FULL_MASK, y, o);
    z += __shfl_xor_sync(FULL_MASK, z, o);
  }
  *d = a; *jx = x; *jy = y; *jz = z;
}

// Reverse step of the sites with iolet links: one warp per site, lane i =
// direction i.  Recomputes f(t) with the boundary values of G_{t-1} (as the
// forward computed them), forms lam = G_t^T mu(t+1) including the transposes
// of the Ladd and ghost-density boundaries of G_t (which read the moments of
// s'(t) at the site), applies the collision transpose, and accumulates the
// per-link amplitude derivatives (each link record belongs to one lane).
template <typename S, bool GPREV>
__device__ __forceinline__ typename Real<S>::type adjoint_iolet_site(const S* __restrict__ prev, const S* __restrict__ cur,
                                                     const S* __restrict__ mu_next, S* __restrict__ mu_out,
                                                     const int32_t* __restrict__ src,
                                                     const LinkRec* __restrict__ links,
                                                     const double* __restrict__ amp, const AdjParams& ap,
                                                     const ProbeMap& pm, const int32_t* __restrict__ sites,
                                                     int64_t nsites, double* __restrict__ dlink, int store,
                                                     int64_t w) {
  using R = typename Real<S>::type;
  const StepParams& p = ap.prev;
  const int i = threadIdx.x & 31;
  const bool dir = i < Q;
  R dtau_local = R(0);
  if (w < nsites) {  // uniform across the warp
    const int64_t n = p.n, x = sites[w];
    const int32_t code = (dir && i > 0) ? src[(int64_t)(i - 1) * p.sn + x] : 0;
    pdl_wait();  // the states below were written by the kernels before this one
    pdl_trigger();
    // f(t) at x: gathered from s'(t-1) with the boundary values of G_{t-1}
    R h = R(0);
    if (GPREV) {
      R own = R(0);
      if (dir) {
        h = ldpop(prev + (i == 0 ? x : (code >= 0 ? (int64_t)i * n + code : (int64_t)lane_opp(i) * n + x)));
        own = ldpop(prev + (int64_t)i * n + x);
      }
      R d, jx, jy, jz;  // summed in the forward's order: f(t) gets the forward's bits
      lane_moment_sums<R>(own, R(1), &d, &jx, &jy, &jz);
      const R rp = R(1) + d;
      const R ux = jx / rp, uy = jy / rp, uz = jz / rp;
      if (code <= -2) {
        const LinkRec L = links[-code - 2];
        const R a = BC<R>::amp(p, amp, L.kind == 0 && L.group >= 0 ? L.group : 0);
        h = lane_iolet_value<R>(i, L, h, rp, ux, uy, uz, a, p);
      }
    } else if (dir) {
      h = ldpop(prev + (int64_t)i * n + x);
    }
    // lane i loads lam_opp(i): s'_opp(i)(x) is read by x - c_i in direction
    // opp(i), or by x itself in direction i across a boundary
    R lo = R(0);
    if (dir) lo = ldpop(mu_next + (i == 0 ? x : (code >= 0 ? (int64_t)lane_opp(i) * n + code : (int64_t)i * n + x)));
    // boundary transposes of G_t (moments of s'(t) at x)
    const R c = dir ? ldpop(cur + (int64_t)i * n + x) : R(0);
    R d, jx, jy, jz;
    warp_moment_sums<R>(c, i, &d, &jx, &jy, &jz);
    const R rho_s = R(1) + d;
    const R usx = jx / rho_s, usy = jy / rho_s, usz = jz / rho_s;
    R gs = R(0), gx = R(0), gy = R(0), gz = R(0);
    if (code <= -2) {
      const int64_t r = -code - 2;
      const LinkRec L = links[r];
      const R a = ldpop(mu_next + (int64_t)i * n + x);  // adjoint of f_i(x, t+1)
      const R val = R(ap.val_cur[L.iolet]);
      if (L.kind == 0) {
        const R rho = p.ladd_rho_one ? R(1) : rho_s;
        if (!p.ladd_rho_one) gs = a * R(L.coef) * R(amp[L.group]) * val;
        dlink[r] += (double)(a * R(L.coef) * rho * val);
      } else {
        lo = R(0);  // the ghost value does not read s'_opp(i)(x)
        const IoletParam io = p.io[L.iolet];
        R ex = usx, ey = usy, ez = usz;
        if (!p.ghost_full_u) {
          const R un = ex * R(io.nx) + ey * R(io.ny) + ez * R(io.nz);
          ex = un * R(io.nx);
          ey = un * R(io.ny);
          ez = un * R(io.nz);
        }
        const R rho_k = R(1) + val;
        const R cu = lane_cdotu<R>(i, ex, ey, ez);
        const R k3 = a * lane_w<R>(i) * rho_k;
        // d f^eq_i / d u_g = w_i rho_k (3 c_i + 9 (c_i . u_g) c_i - 3 u_g)
        R vx = k3 * (R(3) * k_cx[i] + R(9) * cu * k_cx[i] - R(3) * ex);
        R vy = k3 * (R(3) * k_cy[i] + R(9) * cu * k_cy[i] - R(3) * ey);
        R vz = k3 * (R(3) * k_cz[i] + R(9) * cu * k_cz[i] - R(3) * ez);
        if (!p.ghost_full_u) {
          const R vn = vx * R(io.nx) + vy * R(io.ny) + vz * R(io.nz);
          vx = vn * R(io.nx);
          vy = vn * R(io.ny);
          vz = vn * R(io.nz);
        }
        gx = vx;
        gy = vy;
        gz = vz;
      }
    }
    const R gsum = warp_sum<R>(gs), gux = warp_sum<R>(gx), guy = warp_sum<R>(gy), guz = warp_sum<R>(gz);
    // lam_i, with d u_s / d s'_j = (c_j - u_s) / rho_s and d rho_s / d s'_j = 1
    R lam = __shfl_sync(FULL_MASK, lo, lane_opp(i < Q ? i : 0));
    lam += gsum + ((R(k_cx[i]) - usx) * gux + (R(k_cy[i]) - usy) * guy + (R(k_cz[i]) - usz) * guz) / rho_s;
    if (!dir) lam = R(0);
    // collision transpose at f(t) = h
    Macro<R> m;
    {
      R jx, jy, jz;
      warp_moment_sums<R>(h, i, &m.drho, &jx, &jy, &jz);
      m.rho = R(1) + m.drho;
      const R inv = R(1) / m.rho;
      m.ux = jx * inv;
      m.uy = jy * inv;
      m.uz = jz * inv;
    }
    const R usq15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    const R omega = omega_of<R>(p);
    const R cu = lane_cdotu<R>(i, m.ux, m.uy, m.uz);
    const R wi = lane_w<R>(i);
    const R b = lam * wi * (R(3) + R(9) * cu);
    const R S0 = warp_sum<R>(lam * wi * (R(1) + R(3) * cu + R(4.5) * cu * cu - usq15));
    const R Lw = warp_sum<R>(lam * wi);
    R Bx = warp_sum<R>(b * R(k_cx[i])), By = warp_sum<R>(b * R(k_cy[i])), Bz = warp_sum<R>(b * R(k_cz[i]));
    const R dt = warp_sum<R>(dir ? lam * (h - lane_heq<R>(i, m.drho, m.rho, m.ux, m.uy, m.uz, usq15)) : R(0));
    Bx -= R(3) * m.ux * Lw;
    By -= R(3) * m.uy * Lw;
    Bz -= R(3) * m.uz * Lw;
    if (i == 0) dtau_local = omega * omega * dt;
    if (store && dir) {
      R uax;
      const R pg = probe_term<R>(pm, x, m, &uax, i == 0);
      R v = (R(1) - omega) * lam +
            omega * (S0 + (R(k_cx[i]) - m.ux) * Bx + (R(k_cy[i]) - m.uy) * By + (R(k_cz[i]) - m.uz) * Bz);
      R ax[3];
      probe_axis<R>(pm, ax);
      v += pg * (R(k_cx[i]) * ax[0] + R(k_cy[i]) * ax[1] + R(k_cz[i]) * ax[2] - uax);
      mu_out[(int64_t)i * n + x] = from_real<S>(v);
    }
  }
  return dtau_local;
}

// One reverse step in one launch.  Every stride-th block (the first
// n_iolet_blocks of them) takes eight iolet sites, a warp each; the others
// take 256 bulk sites, a thread each.  Spreading the short, latency-bound
// iolet blocks through the grid lets them run beside the bulk blocks instead
// of ahead of them.  Block b's dJ/dtau partial goes to part[b] (fixed order).
// WIDE: offsets within direction pairs (lattices above ~226M sites); the
// offsets stay 32-bit either way, which keeps the 38 gather addresses from
// spilling.
template <typename S, bool GPREV, bool WIDE, bool CT>
__global__ void __launch_bounds__(BLOCK, sizeof(typename Real<S>::type) == 8 ? 2 : 4)
    k_adjoint(const S* __restrict__ prev, const S* __restrict__ cur, const S* __restrict__ mu_next,
              S* __restrict__ mu_out, const int32_t* __restrict__ src, const uint32_t* __restrict__ ctab,
              const int32_t* __restrict__ tbase, const uint32_t* __restrict__ imask,
              const LinkRec* __restrict__ links, const double* __restrict__ amp, const AdjParams ap,
              const ProbeMap pm, const int32_t* __restrict__ sites, int64_t nsites, unsigned n_iolet_blocks,
              const BlockDiv stride, double* __restrict__ part, double* __restrict__ dlink, int store) {
  using R = typename Real<S>::type;
  __shared__ R neq[Q][BLOCK];
  __shared__ R sh[BLOCK / 32];
  const unsigned b = blockIdx.x, j = block_div(b, stride);
  R d;
  if (b == j * stride.d && j < n_iolet_blocks) {
    d = adjoint_iolet_site<S, GPREV>(prev, cur, mu_next, mu_out, src, links, amp, ap, pm, sites, nsites, dlink,
                                     store, ((int64_t)j * BLOCK + threadIdx.x) >> 5);
  } else {
    const unsigned k = b - min(n_iolet_blocks, j + 1);  // bulk block: blocks before b that are not iolet blocks
    d = adjoint_site<S, GPREV, WIDE, CT>(prev, mu_next, mu_out, src, ctab, tbase, imask, ap, pm, store,
                                         (int64_t)k * BLOCK + threadIdx.x, k, neq);
  }
  // block sum of the dJ/dtau terms in the kernel's arithmetic type (FP64 on
  // GB300 runs at 1/64 of the FP32 rate), accumulated per block in FP64
  // across the reverse steps (threads without a site have not waited yet)
  pdl_wait();
  pdl_trigger();
  const R bs = block_sum_r<R>(d, sh);
  if (threadIdx.x == 0) part[b] += (double)bs;
}

// The objective's last term, t = N: J gains (u.axis - target)^2 / N and
// mu(N) = dJ/df(N), dJ/df_j = (2/N) (u.axis - target) (c_j.axis - u.axis) / rho
// (added to mu, which holds zeros).
template <typename S, int MODE>
__global__ void k_probe_adj(const S* __restrict__ fin, const int32_t* __restrict__ src,
                            const LinkRec* __restrict__ links, const double* __restrict__ amp, const StepParams p,
                            const int64_t* __restrict__ sites, const double* __restrict__ target, double ax,
                            double ay, double az, double invN, int64_t np, S* __restrict__ mu,
                            double* __restrict__ jp) {
  using R = typename Real<S>::type;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int64_t x = sites[q];
  R h[Q];
  load_state<S, MODE>(fin, src, links, amp, p, x, h);
  const Macro<R> m = moments<R>(h);
  const double uad = (double)m.ux * ax + (double)m.uy * ay + (double)m.uz * az;
  const double dd = uad - target[q];
  jp[q] += dd * dd * invN;
  const R ua = R(uad);
  const R g = R(2.0 * invN * dd) / m.rho;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const R cj = R(cx(j)) * R(ax) + R(cy(j)) * R(ay) + R(cz(j)) * R(az);
    S* a = mu + (int64_t)j * p.n + x;
    *a = from_real<S>(to_real(*a) + g * (cj - ua));
  }
}

// Final sums in a fixed order: out[0] = J, out[1] = dJ/dtau, out[2+g] = dJ/da_g.
__global__ void k_adj_finish(const double* __restrict__ jp, int64_t np, const double* __restrict__ dtau_part,
                             int64_t nb, const double* __restrict__ dlink, const int64_t* __restrict__ gbegin,
                             int ngroups, double* __restrict__ out) {
  __shared__ double sh[32];
  const int task = blockIdx.x;  // 0: J, 1: dtau, 2+g: group g
  const double* arr;
  int64_t b, e;
  if (task == 0) { arr = jp; b = 0; e = np; }
  else if (task == 1) { arr = dtau_part; b = 0; e = nb; }
  else { arr = dlink; b = gbegin[task - 2]; e = gbegin[task - 1]; }
  double v = 0;
  for (int64_t k = b + threadIdx.x; k < e; k += blockDim.x) v += arr[k];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) out[task] = v;
  (void)ngroups;
}


template <typename S>
cudaError_t launch_adjoint(const hlb_solver* h, const void* prev, bool gprev, const void* cur, const void* mu_next,
                           void* mu_out, int64_t tb_prev, int64_t tb_cur, const ProbeMap& pm, double* dtau_part,
                           double* dlink, bool store, cudaStream_t st) {
  AdjParams ap;
  ap.prev = h->params(tb_prev);
  StepParams pc = h->params(tb_cur);
  for (int k = 0; k < MAX_IOLETS; ++k) ap.val_cur[k] = k < h->n_iolets ? pc.io[k].val : 0.0;
  const int st_ = store ? 1 : 0;
  const unsigned gi = (unsigned)((h->n_iolet_sites + 7) / 8);  // one warp per iolet site
  const unsigned grid = gi + grid_for(h->n);
  const unsigned stride = gi ? grid / gi : 1;  // gi * stride <= grid
  const bool off32 = h->off32, ct = h->compact;
  auto pick = [&](auto gp) {
    constexpr bool G = decltype(gp)::value;
    return ct ? (off32 ? k_adjoint<S, G, false, true> : k_adjoint<S, G, true, true>)
              : (off32 ? k_adjoint<S, G, false, false> : k_adjoint<S, G, true, false>);
  };
  auto kernel = gprev ? pick(std::true_type{}) : pick(std::false_type{});
  // programmatic dependent launch: the index decode overlaps the previous
  // kernel's tail (the reverse steps and the segment recomputes alternate)
  return launch_pdl(kernel, grid, BLOCK, st, (const S*)prev, (const S*)cur, (const S*)mu_next, (S*)mu_out, h->d_src,
                    h->d_ctab, h->d_tbase, h->d_imask, h->d_links, h->d_amp, ap, pm, h->d_iolet_sites,
                    h->n_iolet_sites, gi, make_block_div(stride), dtau_part, dlink, st_);
}

struct Probe {
  const int64_t* sites;
  const double* target;
  double ax, ay, az, invN;
  int64_t np;
};

#define PROBE_MODE_SWITCH(mode, LAUNCH)                                    \
  switch (mode) {                                                         \
    case 1: { constexpr int M = 1; LAUNCH; break; }                       \
    case 2: { constexpr int M = 2; LAUNCH; break; }                       \
    default: { constexpr int M = 0; LAUNCH; break; }                      \
  }

template <typename S>
cudaError_t launch_probe_adj(const hlb_solver* h, const void* fin, int mode, int64_t tb, const Probe& pr, void* mu,
                             double* jp, cudaStream_t st) {
  if (pr.np == 0) return cudaSuccess;
  StepParams p = h->params(tb);
  const unsigned g = (unsigned)((pr.np + 127) / 128);
  PROBE_MODE_SWITCH(mode, (k_probe_adj<S, M><<<g, 128, 0, st>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p,
                                                                 pr.sites, pr.target, pr.ax, pr.ay, pr.az, pr.invN,
                                                                 pr.np, (S*)mu, jp)));
  return cudaGetLastError();
}

// Workspace of one adjoint run.  The minimum (`total`) holds the sqrt(N)
// checkpoints, one segment of states and the adjoint buffers.  A larger
// workspace keeps, in `keep`, the post-collision states of `n_keep` whole
// segments from the forward sweep, so that the reverse sweep need not
// recompute them: segments [nck - 1 - n_keep, nck - 1) (never the last one,
// which runs in the solver's own scheme so that the run ends exactly as N
// plain steps would).
struct AdjLayout {
  int64_t K = 1, nck = 1, nseg = 2, n_keep = 0;
  size_t ck = 0, seg = 0, mu = 0, dtau = 0, dlink = 0, sites = 0, target = 0, jp = 0, gbegin = 0, pmask = 0,
         pbase = 0, out = 0, keep = 0, total = 0, used = 0;
};

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

AdjLayout adj_layout(const hlb_solver* h, int64_t N, int64_t np, size_t ws_bytes = 0) {
  AdjLayout y;
  // AA checkpoints are taken after odd steps, so the interval is even
  y.K = (int64_t)ceil(sqrt((double)N));
  if (y.K < 2) y.K = 2;
  if (y.K & 1) ++y.K;
  y.nck = (N + y.K - 1) / y.K;
  y.nseg = std::max<int64_t>(y.K, 2);
  const size_t st = al256(h->state_bytes());
  size_t off = 0;
  y.ck = off; off += st * (size_t)y.nck;
  y.seg = off; off += st * (size_t)y.nseg;
  y.mu = off; off += st * 2;
  y.dtau = off; off += al256(sizeof(double) * (grid_for(h->n) + (size_t)(h->n_iolet_sites + 7) / 8));
  y.dlink = off; off += al256(sizeof(double) * (size_t)std::max<int64_t>(h->n_links, 1));
  y.sites = off; off += al256(sizeof(int64_t) * (size_t)std::max<int64_t>(np, 1));
  y.target = off; off += al256(sizeof(double) * (size_t)std::max<int64_t>(np, 1));
  y.jp = off; off += al256(sizeof(double) * (size_t)std::max<int64_t>(np, 1));
  y.gbegin = off; off += al256(sizeof(int64_t) * (size_t)(h->n_groups_total + 1));
  y.pmask = off; off += al256(sizeof(uint32_t) * (size_t)((h->n + 31) / 32));
  y.pbase = off; off += al256(sizeof(int32_t) * (size_t)((h->n + 31) / 32));
  y.out = off; off += al256(sizeof(double) * (size_t)(2 + h->n_groups_total));
  y.total = off;
  y.keep = off;
  if (ws_bytes > y.total && y.nck > 1)
    y.n_keep = std::min<int64_t>(y.nck - 1, (int64_t)((ws_bytes - y.total) / (st * (size_t)y.K)));
  y.used = y.total + st * (size_t)y.K * (size_t)y.n_keep;
  return y;
}

template <typename S>
int run_adjoint(hlb_solver* h, int64_t N, const hlb_objective* obj, char* ws, const AdjLayout& y, double* J,
                double* dtau_out, double* damp) {
  cudaStream_t st = h->stream;
  const size_t stb = al256(h->state_bytes());
  auto ck = [&](int64_t c) -> void* { return ws + y.ck + stb * (size_t)c; };
  auto sg = [&](int64_t j) -> void* { return ws + y.seg + stb * (size_t)j; };
  void* mu[2] = {ws + y.mu, ws + y.mu + stb};
  double* dtau_part = (double*)(ws + y.dtau);
  double* dlink = (double*)(ws + y.dlink);
  int64_t* d_sites = (int64_t*)(ws + y.sites);
  double* d_target = (double*)(ws + y.target);
  double* jp = (double*)(ws + y.jp);
  int64_t* gbegin = (int64_t*)(ws + y.gbegin);
  double* out = (double*)(ws + y.out);
  const int64_t nb = grid_for(h->n) + (h->n_iolet_sites + 7) / 8;  // bulk + iolet-site partials
  const int64_t np = obj->n_probe;
  const int G = h->n_groups_total;

#define TRY(expr)                                          \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return hlb_cuda_fail(_e, #expr); \
  } while (0)

  // starting pre-collision state f(t0) into checkpoint 0
  if (h->phase == HLB_READ_LOCAL)
    TRY(cudaMemcpyAsync(ck(0), h->f[h->cur], h->state_bytes(), cudaMemcpyDeviceToDevice, st));
  else
    TRY(hlb_launch_state(h, h->f[h->cur], h->phase, h->t - 1, ck(0), -1, st));
  const int64_t t0 = h->t;
  TRY(cudaMemsetAsync(dtau_part, 0, sizeof(double) * nb, st));
  TRY(cudaMemsetAsync(dlink, 0, sizeof(double) * std::max<int64_t>(h->n_links, 1), st));
  TRY(cudaMemsetAsync(jp, 0, sizeof(double) * std::max<int64_t>(np, 1), st));
  // probes ordered by site, and their bit mask with per-word prefix counts
  std::vector<int64_t> order((size_t)np);
  for (int64_t k = 0; k < np; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int64_t a_, int64_t b_) { return obj->sites[a_] < obj->sites[b_]; });
  std::vector<int64_t> ssites((size_t)np);
  std::vector<double> starget((size_t)np);
  for (int64_t k = 0; k < np; ++k) {
    ssites[k] = obj->sites[order[k]];
    starget[k] = obj->target[order[k]];
  }
  const int64_t nw = (h->n + 31) / 32;
  std::vector<uint32_t> mask((size_t)nw, 0u);
  std::vector<int32_t> base((size_t)nw, 0);
  for (int64_t k = 0; k < np; ++k) mask[ssites[k] >> 5] |= 1u << (ssites[k] & 31);
  for (int64_t wd = 1; wd < nw; ++wd) base[wd] = base[wd - 1] + __builtin_popcount(mask[wd - 1]);
  uint32_t* d_mask = (uint32_t*)(ws + y.pmask);
  int32_t* d_base = (int32_t*)(ws + y.pbase);
  if (np > 0) {
    TRY(cudaMemcpyAsync(d_sites, ssites.data(), sizeof(int64_t) * np, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(d_target, starget.data(), sizeof(double) * np, cudaMemcpyHostToDevice, st));
  }
  TRY(cudaMemcpyAsync(d_mask, mask.data(), sizeof(uint32_t) * nw, cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(d_base, base.data(), sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st));
  const ProbeMap pm{d_mask, d_base, d_target, jp, obj->axis[0], obj->axis[1], obj->axis[2], 1.0 / (double)N,
                    (float)obj->axis[0], (float)obj->axis[1], (float)obj->axis[2]};
  TRY(cudaMemcpyAsync(gbegin, h->group_link_begin.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, st));
  Probe pr{d_sites, d_target, obj->axis[0], obj->axis[1], obj->axis[2], 1.0 / (double)N, np};

  // ---- forward sweep, segment by segment.  A kept segment runs pull steps
  // that write its post-collision states into its kept slots; every other
  // segment runs the solver's own scheme (the faster one for the lattice size
  // when it was created with AUTO).  Checkpoint c is taken at the start of
  // segment c: f(cK) in natural layout (checkpoint 0, and after an AA odd
  // step) or s'(cK - 1), from which the segment's first step gathers f(cK)
  // (ckg[c]). ----
  const int64_t K = y.K, nck = y.nck, A = nck - 1 - y.n_keep;  // kept: [A, nck - 1)
  const bool ab = h->scheme == HLB_PULL_AB;
  auto kept = [&](int64_t c) { return c >= A && c < nck - 1; };
  auto kp = [&](int64_t c, int64_t j) -> void* { return ws + y.keep + stb * (size_t)((c - A) * K + j); };
  std::vector<char> ckg((size_t)nck, 0);
  void* W = sg(0);                  // AA working buffer
  const void* in = ck(0);           // pull: f(t) in place (gather false) or s'(t - 1)
  bool gather = false, in_aa = false, swapped = false;
  for (int64_t c = 0; c < nck; ++c) {
    const int64_t sb = c * K, se = std::min<int64_t>(N, (c + 1) * K);
    const bool aa_mode = !ab && !kept(c);
    if (c > 0) {
      TRY(cudaMemcpyAsync(ck(c), in_aa ? W : in, h->state_bytes(), cudaMemcpyDeviceToDevice, st));
      ckg[(size_t)c] = in_aa ? 0 : 1;
    }
    if (aa_mode && !in_aa) {
      // f(sb) in natural layout, with the boundary values the AA pass would have written
      if (c == 0)
        TRY(cudaMemcpyAsync(W, ck(0), h->state_bytes(), cudaMemcpyDeviceToDevice, st));
      else
        TRY(hlb_launch_state(h, in, HLB_READ_GATHER_AB, t0 + sb - 1, W, -1, st));
      in_aa = true;
      swapped = false;
    } else if (!aa_mode && in_aa) {
      in = W;  // f(sb) in place after an AA odd step (K is even)
      gather = false;
      in_aa = false;
    }
    for (int64_t s = sb; s < se; ++s) {
      if (aa_mode) {
        TRY(hlb_launch_aa(h, W, swapped, t0 + s, st));
        swapped = !swapped;
      } else {
        // pull A-B: two working buffers (segment slots 0 and 1) or the kept
        // slots; the final s'(t0 + N - 1) goes straight into the solver's
        // buffer 0, free during the run (the start state is checkpoint 0)
        void* out_ = kept(c) ? kp(c, s - sb) : (s == N - 1 ? h->f[0] : sg(s & 1));
        TRY(hlb_launch_step(h, in, out_, gather, t0 + s - 1, st));
        in = out_;
        gather = true;
      }
    }
  }
  int fin_mode;
  if (in_aa) {
    // the final state f(t0 + N) in the AA layout it ended in
    TRY(cudaMemcpyAsync(h->f[0], W, h->state_bytes(), cudaMemcpyDeviceToDevice, st));
    fin_mode = swapped ? HLB_READ_GATHER_AA : HLB_READ_LOCAL;
  } else {
    fin_mode = HLB_READ_GATHER_AB;
  }
  const void* fin_state = h->f[0];

  // ---- reverse: recompute each segment's post-collision states with the
  // pull kernels from its checkpoint (kept segments need none), then sweep
  // it backwards ----
  int a = 0;  // mu[a] holds mu(t+1)
  TRY(cudaMemsetAsync(mu[a], 0, h->state_bytes(), st));
  TRY(launch_probe_adj<S>(h, fin_state, fin_mode, t0 + N - 1, pr, mu[a], jp, st));
  for (int64_t c = nck - 1; c >= 0; --c) {
    const int64_t sb = c * K, se = std::min<int64_t>(N, (c + 1) * K);
    const bool ck_gather = ckg[(size_t)c] != 0;  // checkpoint holds s'(cK - 1)
    auto slot = [&](int64_t j) -> void* { return kept(c) ? kp(c, j) : sg(j); };
    if (!kept(c)) {
      const void* rin = ck(c);
      bool rg = ck_gather;
      for (int64_t s = sb; s < se; ++s) {
        TRY(hlb_launch_step(h, rin, sg(s - sb), rg, t0 + s - 1, st));
        rin = sg(s - sb);
        rg = true;
      }
    }
    for (int64_t s = se - 1; s >= sb; --s) {
      const void* prev = s == sb ? ck(c) : slot(s - sb - 1);
      const bool gprev = s != sb || ck_gather;  // f(s) gathered from s'(s - 1), or a checkpoint in place
      // mu(s) = C^T G^T mu(s+1) + dJ/df(s) at the probes (s >= 1), in one pass
      TRY(launch_adjoint<S>(h, prev, gprev, slot(s - sb), mu[a], mu[a ^ 1], t0 + s - 1, t0 + s, pm, dtau_part, dlink,
                            s >= 1, st));
      a ^= 1;
    }
  }
  k_adj_finish<<<2 + G, 256, 0, st>>>(jp, np, dtau_part, nb, dlink, gbegin, G, out);
  TRY(cudaGetLastError());

  std::vector<double> host(2 + G);
  TRY(cudaMemcpyAsync(host.data(), out, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
#undef TRY
  h->cur = 0;
  h->phase = fin_mode;
  h->stepped = true;  // the final state came from a step of the solver's scheme
  h->t = t0 + N;
  if (J) *J = host[0];
  if (dtau_out) *dtau_out = host[1];
  if (damp)
    for (int k = 0; k < G; ++k) damp[k] = host[2 + k];
  if (!std::isfinite(host[0]) || !std::isfinite(host[1])) return hlb_fail(HLB_ERR_DIVERGED, "non-finite adjoint");
  return HLB_OK;
}

int check_objective(const hlb_solver* h, int64_t N, const hlb_objective* obj) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (h->precision != HLB_FP32 && h->precision != HLB_FP64)
    return hlb_fail(HLB_ERR_ARG, "the adjoint needs FP32 or FP64 storage");
  if (N < 1) return hlb_fail(HLB_ERR_ARG, "nsteps must be >= 1");
  if (!obj) return hlb_fail(HLB_ERR_ARG, "null objective");
  if (obj->n_probe < 0 || (obj->n_probe > 0 && (!obj->sites || !obj->target)))
    return hlb_fail(HLB_ERR_ARG, "bad probe arrays");
  std::vector<int64_t> s(obj->sites, obj->sites + obj->n_probe);
  std::sort(s.begin(), s.end());
  for (size_t k = 0; k < s.size(); ++k) {
    if (s[k] < 0 || s[k] >= h->n) return hlb_fail(HLB_ERR_ARG, "probe site out of range");
    if (k && s[k] == s[k - 1]) return hlb_fail(HLB_ERR_ARG, "probe sites must be distinct");
  }
  return HLB_OK;
}

}  // namespace

extern "C" int hlb_adjoint_workspace_bytes(const hlb_solver* h, int64_t nsteps, int64_t n_probe, size_t* bytes) {
  if (!h || !bytes) return hlb_fail(HLB_ERR_ARG, "null argument");
  if (nsteps < 1 || n_probe < 0) return hlb_fail(HLB_ERR_ARG, "nsteps must be >= 1 and n_probe >= 0");
  *bytes = adj_layout(h, nsteps, n_probe).total;
  return HLB_OK;
}

extern "C" int hlb_adjoint_plan(const hlb_solver* h, int64_t nsteps, int64_t n_probe, size_t ws_bytes,
                                int64_t* interval, int64_t* kept_segments, int64_t* recomputed_steps,
                                size_t* bytes_used) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (nsteps < 1 || n_probe < 0) return hlb_fail(HLB_ERR_ARG, "nsteps must be >= 1 and n_probe >= 0");
  const AdjLayout y = adj_layout(h, nsteps, n_probe, ws_bytes);
  if (ws_bytes < y.total) return hlb_fail(HLB_ERR_WS, "workspace below the minimum of hlb_adjoint_workspace_bytes");
  if (interval) *interval = y.K;
  if (kept_segments) *kept_segments = y.n_keep;
  if (recomputed_steps) *recomputed_steps = nsteps - y.n_keep * y.K;
  if (bytes_used) *bytes_used = y.used;
  return HLB_OK;
}

static int adjoint_run_impl(hlb_solver* h, int64_t nsteps, const hlb_objective* obj, void* ws, size_t ws_bytes,
                            double* J, double* dtau, double* damp) {
  int rc = check_objective(h, nsteps, obj);
  if (rc) return rc;
  if (h->any_wk()) return hlb_fail(HLB_ERR_ARG, "the adjoint does not differentiate Windkessel outlets");
  AdjLayout y = adj_layout(h, nsteps, obj->n_probe, ws_bytes);
  if (!ws || ((uintptr_t)ws & 255)) return hlb_fail(HLB_ERR_WS, "adjoint workspace missing or not 256-byte aligned");
  if (ws_bytes < y.total)
    return hlb_fail(HLB_ERR_WS, "adjoint workspace too small: need " + std::to_string(y.total) + " bytes");
  if (h->precision == HLB_FP64) return run_adjoint<double>(h, nsteps, obj, (char*)ws, y, J, dtau, damp);
  return run_adjoint<float>(h, nsteps, obj, (char*)ws, y, J, dtau, damp);
}

extern "C" int hlb_adjoint_run(hlb_solver* h, int64_t nsteps, const hlb_objective* obj, void* ws, size_t ws_bytes,
                               double* J, double* dtau, double* damp) {
  return hlb_no_throw([&] { return adjoint_run_impl(h, nsteps, obj, ws, ws_bytes, J, dtau, damp); });
}
