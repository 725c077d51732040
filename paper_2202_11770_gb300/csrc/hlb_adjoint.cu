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
// opp(i).  One kernel per reverse step reads the index table once and
// gathers both mu(t+1) and s'(t-1) (to recompute f(t)).
#include <math.h>

#include <algorithm>
#include <vector>

#include "hlb_internal.h"

using namespace hlb;

namespace {

constexpr int BLOCK = 256;
inline unsigned grid_for(int64_t n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

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

// Adjoint of one reverse step at site x (GPREV: f(t) is gathered from
// s'(t-1); false only at t = 0 where prev holds f(0) itself).  With
// IOLET = false the site is skipped (returns false) when it has an iolet
// link; those sites go through the IOLET = true instantiation, which adds
// the boundary transposes.  Returns the site's dJ/dtau contribution in *dtau.
template <typename S, bool GPREV, bool IOLET>
__device__ __forceinline__ bool adjoint_site(const S* __restrict__ prev, const S* __restrict__ cur,
                                             const S* __restrict__ mu_next, S* __restrict__ mu_out,
                                             const int32_t* __restrict__ src, const LinkRec* __restrict__ links,
                                             const double* __restrict__ amp, const AdjParams& ap,
                                             double* __restrict__ dlink, int store, int64_t x, double* dtau) {
  using R = typename Real<S>::type;
  const StepParams& p = ap.prev;
  const int64_t n = p.n;
  R h[Q], lam[Q];
  bool any_iolet = false;
  h[0] = ldpop(prev + x);
  lam[0] = ldpop(mu_next + x);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int32_t s = ldidx(src + (int64_t)(i - 1) * n + x);
    if (GPREV) h[i] = ldpop(prev + (s >= 0 ? (int64_t)i * n + s : (int64_t)opp(i) * n + x));
    else h[i] = ldpop(prev + (int64_t)i * n + x);
    // s'_opp(i)(x) is read by x - c_i = x + c_opp(i) in direction opp(i),
    // or by x itself in direction i when that source is not fluid
    lam[opp(i)] = ldpop(mu_next + (s >= 0 ? (int64_t)opp(i) * n + s : (int64_t)i * n + x));
    any_iolet |= s <= -2;
  }
  if (!IOLET && any_iolet) return false;
  if (IOLET) {
    if (GPREV) iolet_fixup<S>(prev, src, links, amp, p, x, h);
    // boundary terms of G_t, which reads the moments of s'(t) at x
    R d = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R v = ldpop(cur + (int64_t)i * n + x);
      d += v;
      if (cx(i)) jx += cx(i) > 0 ? v : -v;
      if (cy(i)) jy += cy(i) > 0 ? v : -v;
      if (cz(i)) jz += cz(i) > 0 ? v : -v;
    }
    const R rho_s = R(1) + d;
    const R ux = jx / rho_s, uy = jy / rho_s, uz = jz / rho_s;
    R gsum = R(0), gux = R(0), guy = R(0), guz = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int32_t s = src[(int64_t)(i - 1) * n + x];
      if (s > -2) continue;
      const int64_t r = -s - 2;
      const LinkRec L = links[r];
      const R a = ldpop(mu_next + (int64_t)i * n + x);  // adjoint of f_i(x, t+1)
      const R val = R(ap.val_cur[L.iolet]);
      if (L.kind == 0) {
        const R rho = p.ladd_rho_one ? R(1) : rho_s;
        if (!p.ladd_rho_one) gsum += a * R(L.coef) * R(amp[L.group]) * val;
        dlink[r] += (double)(a * R(L.coef) * rho * val);
      } else {
        lam[opp(i)] = R(0);  // the ghost value does not read s'_opp(i)(x)
        const IoletParam io = p.io[L.iolet];
        R gx = ux, gy = uy, gz = uz;
        if (!p.ghost_full_u) {
          const R un = gx * R(io.nx) + gy * R(io.ny) + gz * R(io.nz);
          gx = un * R(io.nx);
          gy = un * R(io.ny);
          gz = un * R(io.nz);
        }
        const R rho_k = R(1) + val;
        const R cu = cdotu<R>(i, gx, gy, gz);
        const R k3 = a * wgt<R>(i) * rho_k;
        // d f^eq_i / d u_g = w_i rho_k (3 c_i + 9 (c_i . u_g) c_i - 3 u_g)
        R vx = k3 * (R(3) * cx(i) + R(9) * cu * cx(i) - R(3) * gx);
        R vy = k3 * (R(3) * cy(i) + R(9) * cu * cy(i) - R(3) * gy);
        R vz = k3 * (R(3) * cz(i) + R(9) * cu * cz(i) - R(3) * gz);
        if (!p.ghost_full_u) {
          const R vn = vx * R(io.nx) + vy * R(io.ny) + vz * R(io.nz);
          vx = vn * R(io.nx);
          vy = vn * R(io.ny);
          vz = vn * R(io.nz);
        }
        gux += vx;
        guy += vy;
        guz += vz;
      }
    }
    // d u_s / d s'_j = (c_j - u_s) / rho_s;  d rho_s / d s'_j = 1
#pragma unroll
    for (int j = 0; j < Q; ++j)
      lam[j] += gsum + ((R(cx(j)) - ux) * gux + (R(cy(j)) - uy) * guy + (R(cz(j)) - uz) * guz) / rho_s;
  }
  // collision adjoint at f(t) = h
  const Macro<R> m = moments<R>(h);
  const R usq15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
  const R omega = R(p.omega);
  R S0 = R(0), Lw = R(0), Bx = R(0), By = R(0), Bz = R(0), dt = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R cu = cdotu<R>(i, m.ux, m.uy, m.uz);
    const R w = wgt<R>(i);
    S0 += lam[i] * w * (R(1) + R(3) * cu + R(4.5) * cu * cu - usq15);  // feq_i / rho
    Lw += lam[i] * w;
    const R b = lam[i] * w * (R(3) + R(9) * cu);
    if (cx(i)) Bx += cx(i) > 0 ? b : -b;
    if (cy(i)) By += cy(i) > 0 ? b : -b;
    if (cz(i)) Bz += cz(i) > 0 ? b : -b;
    dt += lam[i] * (h[i] - heq<R>(i, m.drho, m.rho, m.ux, m.uy, m.uz, usq15));
  }
  // (1/rho) d feq_i/d u_a summed with lam: B_a - 3 u_a Lw
  Bx -= R(3) * m.ux * Lw;
  By -= R(3) * m.uy * Lw;
  Bz -= R(3) * m.uz * Lw;
  *dtau = (double)(omega * omega * dt);
  if (store) {
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const R v = (R(1) - omega) * lam[j] +
                  omega * (S0 + (R(cx(j)) - m.ux) * Bx + (R(cy(j)) - m.uy) * By + (R(cz(j)) - m.uz) * Bz);
      mu_out[(int64_t)j * n + x] = from_real<S>(v);
    }
  }
  return true;
}

// Bulk reverse step over all sites without iolet links.
template <typename S, bool GPREV>
__global__ void __launch_bounds__(BLOCK) k_adjoint(const S* __restrict__ prev, const S* __restrict__ mu_next,
                                                   S* __restrict__ mu_out, const int32_t* __restrict__ src,
                                                   const AdjParams ap, double* __restrict__ dtau_part, int store) {
  __shared__ double sh[BLOCK / 32];
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  double dtau_local = 0;
  if (x < ap.prev.n)
    adjoint_site<S, GPREV, false>(prev, nullptr, mu_next, mu_out, src, nullptr, nullptr, ap, nullptr, store, x,
                                  &dtau_local);
  const double bs = block_sum(dtau_local, sh);
  if (threadIdx.x == 0) dtau_part[blockIdx.x] += bs;
}

// Reverse step of the sites with iolet links (one thread per site).
template <typename S, bool GPREV>
__global__ void __launch_bounds__(128) k_adjoint_iolet(const S* __restrict__ prev, const S* __restrict__ cur,
                                                       const S* __restrict__ mu_next, S* __restrict__ mu_out,
                                                       const int32_t* __restrict__ src,
                                                       const LinkRec* __restrict__ links,
                                                       const double* __restrict__ amp, const AdjParams ap,
                                                       const int32_t* __restrict__ sites, int64_t nsites,
                                                       double* __restrict__ dtau_part, double* __restrict__ dlink,
                                                       int store) {
  __shared__ double sh[4];
  const int64_t q = (int64_t)blockIdx.x * 128 + threadIdx.x;
  double dtau_local = 0;
  if (q < nsites)
    adjoint_site<S, GPREV, true>(prev, cur, mu_next, mu_out, src, links, amp, ap, dlink, store, sites[q],
                                 &dtau_local);
  const double bs = block_sum(dtau_local, sh);
  if (threadIdx.x == 0) dtau_part[blockIdx.x] += bs;
}

// Objective term at time t for every probe: accumulate (u.axis - target)^2 / N.
template <typename S, bool GATHER>
__global__ void k_probe_obj(const S* __restrict__ fin, const int32_t* __restrict__ src,
                            const LinkRec* __restrict__ links, const double* __restrict__ amp, const StepParams p,
                            const int64_t* __restrict__ sites, const double* __restrict__ target, double ax,
                            double ay, double az, double invN, int64_t np, double* __restrict__ jp) {
  using R = typename Real<S>::type;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int64_t x = sites[q];
  R h[Q];
  if (GATHER) {
    if (gather_site<S>(fin, src, p.n, x, h)) iolet_fixup<S>(fin, src, links, amp, p, x, h);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldpop(fin + (int64_t)i * p.n + x);
  }
  const Macro<R> m = moments<R>(h);
  const double ua = (double)m.ux * ax + (double)m.uy * ay + (double)m.uz * az;
  const double d = ua - target[q];
  jp[q] += d * d * invN;
}

// Objective derivative at time t added to mu(t) at the probes:
// dJ/df_j = (2/N) (u.axis - target) (c_j.axis - u.axis) / rho.
template <typename S, bool GATHER>
__global__ void k_probe_adj(const S* __restrict__ fin, const int32_t* __restrict__ src,
                            const LinkRec* __restrict__ links, const double* __restrict__ amp, const StepParams p,
                            const int64_t* __restrict__ sites, const double* __restrict__ target, double ax,
                            double ay, double az, double invN, int64_t np, S* __restrict__ mu) {
  using R = typename Real<S>::type;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int64_t x = sites[q];
  R h[Q];
  if (GATHER) {
    if (gather_site<S>(fin, src, p.n, x, h)) iolet_fixup<S>(fin, src, links, amp, p, x, h);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldpop(fin + (int64_t)i * p.n + x);
  }
  const Macro<R> m = moments<R>(h);
  const R ua = m.ux * R(ax) + m.uy * R(ay) + m.uz * R(az);
  const R g = R(2.0 * invN) * (ua - R(target[q])) / m.rho;
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

__global__ void k_fill(double* p, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) p[i] = 0;
}

template <typename S>
cudaError_t launch_adjoint(const hlb_solver* h, const void* prev, bool gprev, const void* cur, const void* mu_next,
                           void* mu_out, int64_t tb_prev, int64_t tb_cur, double* dtau_part, double* dlink,
                           bool store, cudaStream_t st) {
  AdjParams ap;
  ap.prev = h->params(tb_prev);
  StepParams pc = h->params(tb_cur);
  for (int k = 0; k < MAX_IOLETS; ++k) ap.val_cur[k] = k < h->n_iolets ? pc.io[k].val : 0.0;
  const int st_ = store ? 1 : 0;
  double* part_i = dtau_part + grid_for(h->n);  // partials of the iolet-site kernel
  const unsigned gi = (unsigned)((h->n_iolet_sites + 127) / 128);
  if (gprev) {
    k_adjoint<S, true><<<grid_for(h->n), BLOCK, 0, st>>>((const S*)prev, (const S*)mu_next, (S*)mu_out, h->d_src, ap,
                                                         dtau_part, st_);
    if (gi)
      k_adjoint_iolet<S, true><<<gi, 128, 0, st>>>((const S*)prev, (const S*)cur, (const S*)mu_next, (S*)mu_out,
                                                   h->d_src, h->d_links, h->d_amp, ap, h->d_iolet_sites,
                                                   h->n_iolet_sites, part_i, dlink, st_);
  } else {
    k_adjoint<S, false><<<grid_for(h->n), BLOCK, 0, st>>>((const S*)prev, (const S*)mu_next, (S*)mu_out, h->d_src, ap,
                                                          dtau_part, st_);
    if (gi)
      k_adjoint_iolet<S, false><<<gi, 128, 0, st>>>((const S*)prev, (const S*)cur, (const S*)mu_next, (S*)mu_out,
                                                    h->d_src, h->d_links, h->d_amp, ap, h->d_iolet_sites,
                                                    h->n_iolet_sites, part_i, dlink, st_);
  }
  return cudaGetLastError();
}

struct Probe {
  const int64_t* sites;
  const double* target;
  double ax, ay, az, invN;
  int64_t np;
};

template <typename S>
cudaError_t launch_probe_obj(const hlb_solver* h, const void* fin, bool gather, int64_t tb, const Probe& pr, double* jp,
                             cudaStream_t st) {
  if (pr.np == 0) return cudaSuccess;
  StepParams p = h->params(tb);
  const unsigned g = (unsigned)((pr.np + 127) / 128);
  if (gather)
    k_probe_obj<S, true><<<g, 128, 0, st>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, pr.sites, pr.target,
                                            pr.ax, pr.ay, pr.az, pr.invN, pr.np, jp);
  else
    k_probe_obj<S, false><<<g, 128, 0, st>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, pr.sites, pr.target,
                                             pr.ax, pr.ay, pr.az, pr.invN, pr.np, jp);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_probe_adj(const hlb_solver* h, const void* fin, bool gather, int64_t tb, const Probe& pr, void* mu,
                             cudaStream_t st) {
  if (pr.np == 0) return cudaSuccess;
  StepParams p = h->params(tb);
  const unsigned g = (unsigned)((pr.np + 127) / 128);
  if (gather)
    k_probe_adj<S, true><<<g, 128, 0, st>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, pr.sites, pr.target,
                                            pr.ax, pr.ay, pr.az, pr.invN, pr.np, (S*)mu);
  else
    k_probe_adj<S, false><<<g, 128, 0, st>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, pr.sites, pr.target,
                                             pr.ax, pr.ay, pr.az, pr.invN, pr.np, (S*)mu);
  return cudaGetLastError();
}

struct AdjLayout {
  int64_t K = 1, nck = 1, nseg = 2;
  size_t ck = 0, seg = 0, mu = 0, dtau = 0, dlink = 0, sites = 0, target = 0, jp = 0, gbegin = 0, out = 0, total = 0;
};

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

AdjLayout adj_layout(const hlb_solver* h, int64_t N, int64_t np) {
  AdjLayout y;
  y.K = (int64_t)ceil(sqrt((double)N));
  if (y.K < 1) y.K = 1;
  y.nck = (N + y.K - 1) / y.K;
  y.nseg = std::max<int64_t>(y.K, 2);
  const size_t st = al256(h->state_bytes());
  size_t off = 0;
  y.ck = off; off += st * (size_t)y.nck;
  y.seg = off; off += st * (size_t)y.nseg;
  y.mu = off; off += st * 2;
  y.dtau = off; off += al256(sizeof(double) * (grid_for(h->n) + (size_t)(h->n_iolet_sites + 127) / 128));
  y.dlink = off; off += al256(sizeof(double) * (size_t)std::max<int64_t>(h->n_links, 1));
  y.sites = off; off += al256(sizeof(int64_t) * (size_t)std::max<int64_t>(np, 1));
  y.target = off; off += al256(sizeof(double) * (size_t)std::max<int64_t>(np, 1));
  y.jp = off; off += al256(sizeof(double) * (size_t)std::max<int64_t>(np, 1));
  y.gbegin = off; off += al256(sizeof(int64_t) * (size_t)(h->n_groups_total + 1));
  y.out = off; off += al256(sizeof(double) * (size_t)(2 + h->n_groups_total));
  y.total = off;
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
  const int64_t nb = grid_for(h->n) + (h->n_iolet_sites + 127) / 128;  // bulk + iolet-site partials
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
  if (np > 0) {
    TRY(cudaMemcpyAsync(d_sites, obj->sites, sizeof(int64_t) * np, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(d_target, obj->target, sizeof(double) * np, cudaMemcpyHostToDevice, st));
  }
  TRY(cudaMemcpyAsync(gbegin, h->group_link_begin.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, st));
  Probe pr{d_sites, d_target, obj->axis[0], obj->axis[1], obj->axis[2], 1.0 / (double)N, np};

  // ---- forward: checkpoints every K steps, last segment kept whole ----
  const int64_t K = y.K, nck = y.nck;
  const int64_t last_begin = (nck - 1) * K;
  const void* in = ck(0);
  bool g = false;
  int scratch = 0;
  for (int64_t s = 0; s < N; ++s) {
    void* o;
    if (s >= last_begin) {
      o = sg(s - last_begin);
    } else if ((s + 1) % K == 0) {
      o = ck((s + 1) / K);
    } else {
      o = sg(scratch);
      scratch ^= 1;
    }
    TRY(hlb_launch_step(h, in, o, g, t0 + s - 1, st));
    TRY(launch_probe_obj<S>(h, o, true, t0 + s, pr, jp, st));
    in = o;
    g = true;
  }

  // ---- reverse ----
  int a = 0;  // mu[a] holds mu(t+1)
  TRY(cudaMemsetAsync(mu[a], 0, h->state_bytes(), st));
  TRY(launch_probe_adj<S>(h, in, true, t0 + N - 1, pr, mu[a], st));
  for (int64_t c = nck - 1; c >= 0; --c) {
    const int64_t sb = c * K, se = std::min<int64_t>(N, (c + 1) * K);
    if (c != nck - 1) {
      const void* rin = ck(c);
      bool rg = c > 0;
      for (int64_t s = sb; s < se; ++s) {
        TRY(hlb_launch_step(h, rin, sg(s - sb), rg, t0 + s - 1, st));
        rin = sg(s - sb);
        rg = true;
      }
    }
    for (int64_t s = se - 1; s >= sb; --s) {
      const void* prev = s == sb ? ck(c) : sg(s - sb - 1);
      const bool gprev = s != 0;
      TRY(launch_adjoint<S>(h, prev, gprev, sg(s - sb), mu[a], mu[a ^ 1], t0 + s - 1, t0 + s, dtau_part, dlink,
                            s >= 1, st));
      if (s >= 1) TRY(launch_probe_adj<S>(h, prev, gprev, t0 + s - 1, pr, mu[a ^ 1], st));
      a ^= 1;
    }
  }
  k_adj_finish<<<2 + G, 256, 0, st>>>(jp, np, dtau_part, nb, dlink, gbegin, G, out);
  TRY(cudaGetLastError());

  // leave the solver at t0 + N: A-B keeps the last post-collision state,
  // AA receives the gathered pre-collision state f(t0 + N) in place
  const void* last = sg(N - 1 - last_begin);
  if (h->scheme == HLB_AA)
    TRY(hlb_launch_state(h, last, HLB_READ_GATHER_AB, t0 + N - 1, h->f[0], -1, st));
  else
    TRY(cudaMemcpyAsync(h->f[0], last, h->state_bytes(), cudaMemcpyDeviceToDevice, st));
  std::vector<double> host(2 + G);
  TRY(cudaMemcpyAsync(host.data(), out, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
#undef TRY
  h->cur = 0;
  h->phase = h->scheme == HLB_AA ? HLB_READ_LOCAL : HLB_READ_GATHER_AB;
  h->stepped = h->scheme != HLB_AA;
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

extern "C" int hlb_adjoint_run(hlb_solver* h, int64_t nsteps, const hlb_objective* obj, void* ws, size_t ws_bytes,
                               double* J, double* dtau, double* damp) {
  int rc = check_objective(h, nsteps, obj);
  if (rc) return rc;
  AdjLayout y = adj_layout(h, nsteps, obj->n_probe);
  if (!ws || ((uintptr_t)ws & 255)) return hlb_fail(HLB_ERR_WS, "adjoint workspace missing or not 256-byte aligned");
  if (ws_bytes < y.total)
    return hlb_fail(HLB_ERR_WS, "adjoint workspace too small: need " + std::to_string(y.total) + " bytes");
  if (h->precision == HLB_FP64) return run_adjoint<double>(h, nsteps, obj, (char*)ws, y, J, dtau, damp);
  return run_adjoint<float>(h, nsteps, obj, (char*)ws, y, J, dtau, damp);
}
