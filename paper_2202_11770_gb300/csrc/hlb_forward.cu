// hlb_forward.cu — forward kernels of the D3Q19 sparse-lattice solver.
//
// k_step: the fused stream-collide-boundary kernel (arXiv 2202.11770,
//   Section 3.2.2: load f, compute rho and u (Eqs. 5-6), f^eq (Eq. 4),
//   collide (Eq. 3a), stream (Eq. 3b) with wall and iolet boundaries, store).
//   One thread per fluid site over the whole site list; the paper's six
//   per-site-type kernels become one kernel in which boundary links are
//   branch-free address selects (walls) plus a rare per-site fix-up (iolets).
// k_macros: the property cache of Section 3.2.2 step 7 (rho, u) plus WSS.
// k_mass / k_flux / k_finish: FP64 reductions in a fixed order.
#include <math.h>

#include "hlb_internal.h"

using namespace hlb;

namespace {

constexpr int BLOCK = 256;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

// ---------------------------------------------------------------------------
// Fused step.  GATHER = false: the buffer holds the pre-collision state f(t)
// (right after initialisation or set_state); GATHER = true: it holds the
// post-collision state s'(t-1) and f(t) is gathered from it.
// ---------------------------------------------------------------------------
template <typename S, bool GATHER>
__global__ void __launch_bounds__(BLOCK) k_step(const S* __restrict__ fin, S* __restrict__ fout,
                                                const int32_t* __restrict__ src,
                                                const LinkRec* __restrict__ links,
                                                const double* __restrict__ amp, const StepParams p) {
  using R = typename Real<S>::type;
  const int64_t n = p.n;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (x >= n) return;
  R h[Q];
  if (GATHER) {
    if (gather_site<S>(fin, src, n, x, h)) iolet_fixup<S>(fin, src, links, amp, p, x, h);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldpop(fin + (int64_t)i * n + x);
  }
  collide<R>(h, R(p.omega));
#pragma unroll
  for (int i = 0; i < Q; ++i) stpop<S>(fout + (int64_t)i * n + x, h[i]);
}

template <typename S, bool GATHER>
__device__ __forceinline__ void load_state(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                           const LinkRec* __restrict__ links, const double* __restrict__ amp,
                                           const StepParams& p, int64_t x, typename Real<S>::type* h) {
  if (GATHER) {
    if (gather_site<S>(fin, src, p.n, x, h)) iolet_fixup<S>(fin, src, links, amp, p, x, h);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = ldpop(fin + (int64_t)i * p.n + x);
  }
}

// ---------------------------------------------------------------------------
// Density, velocity and wall shear stress of f(t).
// ---------------------------------------------------------------------------
template <typename S, bool GATHER>
__global__ void __launch_bounds__(BLOCK) k_macros(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                  const LinkRec* __restrict__ links,
                                                  const double* __restrict__ amp,
                                                  const float* __restrict__ normal, const StepParams p,
                                                  float* __restrict__ rho_out, float* __restrict__ u_out,
                                                  float* __restrict__ wss_out) {
  using R = typename Real<S>::type;
  const int64_t n = p.n;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (x >= n) return;
  R h[Q];
  load_state<S, GATHER>(fin, src, links, amp, p, x, h);
  Macro<R> m = moments<R>(h);
  if (rho_out) rho_out[x] = (float)m.rho;
  if (u_out) {
    u_out[x] = (float)m.ux;
    u_out[n + x] = (float)m.uy;
    u_out[2 * n + x] = (float)m.uz;
  }
  if (!wss_out) return;
  // wall links and the fallback normal (sum of c_j over pull wall directions)
  bool wall = false;
  R nx = 0, ny = 0, nz = 0;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (src[(int64_t)(i - 1) * n + x] == -1) {
      wall = true;
      nx += R(cx(i));
      ny += R(cy(i));
      nz += R(cz(i));
    }
  }
  if (!wall) {
    wss_out[x] = __int_as_float(0x7fc00000);  // NaN
    return;
  }
  if (normal) {
    nx = R(normal[x]);
    ny = R(normal[n + x]);
    nz = R(normal[2 * n + x]);
  } else {
    R l = sqrt(nx * nx + ny * ny + nz * nz);
    nx /= l; ny /= l; nz /= l;
  }
  R usq15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
  R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    R d = h[i] - heq<R>(i, m.drho, m.rho, m.ux, m.uy, m.uz, usq15);
    pxx += cx(i) * cx(i) * d;
    pyy += cy(i) * cy(i) * d;
    pzz += cz(i) * cz(i) * d;
    pxy += cx(i) * cy(i) * d;
    pxz += cx(i) * cz(i) * d;
    pyz += cy(i) * cz(i) * d;
  }
  R k = -(R(1) - R(0.5) * R(p.omega));
  R tx = k * (pxx * nx + pxy * ny + pxz * nz);
  R ty = k * (pxy * nx + pyy * ny + pyz * nz);
  R tz = k * (pxz * nx + pyz * ny + pzz * nz);
  R tn = tx * nx + ty * ny + tz * nz;
  tx -= tn * nx;
  ty -= tn * ny;
  tz -= tn * nz;
  wss_out[x] = (float)sqrt(tx * tx + ty * ty + tz * tz);
}

// Shifted pre-collision state f(t) - w into out [19][n].
template <typename S, bool GATHER>
__global__ void __launch_bounds__(BLOCK) k_state(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                 const LinkRec* __restrict__ links,
                                                 const double* __restrict__ amp, const StepParams p,
                                                 S* __restrict__ out) {
  using R = typename Real<S>::type;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (x >= p.n) return;
  R h[Q];
  load_state<S, GATHER>(fin, src, links, amp, p, x, h);
#pragma unroll
  for (int i = 0; i < Q; ++i) out[(int64_t)i * p.n + x] = from_real<S>(h[i]);
}

// f = f^eq(rho0, u0) (Section 3.1 step 1), stored shifted.
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_init(S* __restrict__ f, int64_t n, double rho0,
                                                const float* __restrict__ u0) {
  using R = typename Real<S>::type;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (x >= n) return;
  R ux = 0, uy = 0, uz = 0;
  if (u0) {
    ux = R(u0[x]);
    uy = R(u0[n + x]);
    uz = R(u0[2 * n + x]);
  }
  R drho = R(rho0 - 1.0);
  R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
#pragma unroll
  for (int i = 0; i < Q; ++i) f[(int64_t)i * n + x] = from_real<S>(heq<R>(i, drho, R(1) + drho, ux, uy, uz, usq15));
}

// ---------------------------------------------------------------------------
// FP64 reductions.
// ---------------------------------------------------------------------------
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
  return r;  // valid in thread 0
}

// Per-block sums of drho (mass - n) into part[blockIdx.x].
template <typename S, bool GATHER>
__global__ void __launch_bounds__(BLOCK) k_mass(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                const LinkRec* __restrict__ links,
                                                const double* __restrict__ amp, const StepParams p,
                                                double* __restrict__ part) {
  using R = typename Real<S>::type;
  __shared__ double sh[BLOCK / 32];
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  double d = 0;
  if (x < p.n) {
    R h[Q];
    load_state<S, GATHER>(fin, src, links, amp, p, x, h);
#pragma unroll
    for (int i = 0; i < Q; ++i) d += (double)h[i];
  }
  double s = block_sum(d, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Per-iolet flux: one block per iolet over its link records, in order.
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_flux(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                const LinkRec* __restrict__ links,
                                                const double* __restrict__ amp, const StepParams p,
                                                const int64_t* __restrict__ begin, double* __restrict__ out) {
  using R = typename Real<S>::type;
  __shared__ double sh[BLOCK / 32];
  const int k = blockIdx.x;
  const int64_t n = p.n;
  double acc = 0;
  for (int64_t r = begin[k] + threadIdx.x; r < begin[k + 1]; r += BLOCK) {
    const LinkRec L = links[r];
    const int64_t x = L.site;
    R own[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) own[i] = ldpop(fin + (int64_t)i * n + x);
    const int j = L.dir;
    // incoming boundary value minus the post-collision population leaving
    // through the iolet (own[opp(j)]):
    R contrib;
    if (L.kind == 0) {
      Macro<R> ms = moments<R>(own);
      R rho = p.ladd_rho_one ? R(1) : ms.rho;
      contrib = R(L.coef) * rho * R(amp[L.group]) * R(p.io[k].val);
    } else {
      Macro<R> ms = moments<R>(own);
      R gx = ms.ux, gy = ms.uy, gz = ms.uz;
      const IoletParam io = p.io[k];
      if (!p.ghost_full_u) {
        R un = gx * R(io.nx) + gy * R(io.ny) + gz * R(io.nz);
        gx = un * R(io.nx);
        gy = un * R(io.ny);
        gz = un * R(io.nz);
      }
      R drho = R(io.val);
      R usq15 = R(1.5) * (gx * gx + gy * gy + gz * gz);
      R hin = R(0);
      // direction j is a runtime value: evaluate the equilibrium by a switch-free loop
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (i == j) hin = heq<R>(i, drho, R(1) + drho, gx, gy, gz, usq15);
      R hout = R(0);
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (i == opp(j)) hout = own[i];
      contrib = hin - hout;
    }
    acc += (double)contrib;
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[1 + k] = s;
}

// out[0] = n + sum of the per-block partials (fixed order).
__global__ void __launch_bounds__(1024) k_finish(const double* __restrict__ part, int64_t nb, int64_t n,
                                                 double* __restrict__ out) {
  __shared__ double sh[32];
  double v = 0;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    out[0] = (double)n + r;
  }
}

__global__ void k_zero(double* p, int64_t m) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) p[i] = 0;
}

// ---------------------------------------------------------------------------
// dispatch helpers
// ---------------------------------------------------------------------------
template <template <typename> class F, typename... A>
cudaError_t dispatch(int precision, A... a) {
  switch (precision) {
    case HLB_FP32: return F<float>::run(a...);
    case HLB_BF16: return F<__nv_bfloat16>::run(a...);
    case HLB_FP16: return F<__half>::run(a...);
    case HLB_FP64: return F<double>::run(a...);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
struct StepOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, void* fout, bool gather, int64_t tb,
                         cudaStream_t s) {
    StepParams p = h->params(tb);
    if (gather)
      k_step<S, true><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, (S*)fout, h->d_src, h->d_links, h->d_amp, p);
    else
      k_step<S, false><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, (S*)fout, h->d_src, h->d_links, h->d_amp, p);
    return cudaGetLastError();
  }
};

template <typename S>
struct MacroOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, bool gather, int64_t tb, float* rho, float* u,
                         float* wss, cudaStream_t s) {
    StepParams p = h->params(tb);
    const float* nrm = h->has_normals ? h->d_normal : nullptr;
    if (gather)
      k_macros<S, true><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, nrm, p,
                                                         rho, u, wss);
    else
      k_macros<S, false><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, nrm, p,
                                                          rho, u, wss);
    return cudaGetLastError();
  }
};

template <typename S>
struct StateOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, bool gather, int64_t tb, void* out, cudaStream_t s) {
    StepParams p = h->params(tb);
    if (gather)
      k_state<S, true><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, (S*)out);
    else
      k_state<S, false><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, (S*)out);
    return cudaGetLastError();
  }
};

template <typename S>
struct InitOp {
  static cudaError_t run(const hlb_solver* h, void* f, double rho0, const float* u0, cudaStream_t s) {
    k_init<S><<<grid_for(h->n), BLOCK, 0, s>>>((S*)f, h->n, rho0, u0);
    return cudaGetLastError();
  }
};

template <typename S>
struct ReduceOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, bool gather, int64_t tb, double* out,
                         cudaStream_t s) {
    StepParams p = h->params(tb);
    const int64_t nb = grid_for(h->n);
    double* part = h->d_red;
    if (gather)
      k_mass<S, true><<<(unsigned)nb, BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, part);
    else
      k_mass<S, false><<<(unsigned)nb, BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, part);
    k_finish<<<1, 1024, 0, s>>>(part, nb, h->n, out);
    if (h->n_iolets > 0) {
      if (gather) {
        const int64_t* begin = (const int64_t*)(h->d_red + nb);  // link ranges stored after the partials
        k_flux<S><<<(unsigned)h->n_iolets, BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links, h->d_amp, p, begin,
                                                          out);
      } else {
        k_zero<<<1, 256, 0, s>>>(out + 1, h->n_iolets);
      }
    }
    return cudaGetLastError();
  }
};

}  // namespace

int64_t hlb_reduce_slots(int64_t n, int32_t n_iolets) {
  // per-block partials, iolet link ranges (int64, n_iolets + 1), final outputs (1 + n_iolets)
  return (int64_t)grid_for(n) + (n_iolets + 1) + (1 + n_iolets);
}

cudaError_t hlb_launch_step(const hlb_solver* h, const void* fin, void* fout, bool gather, int64_t tb,
                            cudaStream_t s) {
  return dispatch<StepOp>(h->precision, h, fin, fout, gather, tb, s);
}
cudaError_t hlb_launch_macros(const hlb_solver* h, const void* fin, bool gather, int64_t tb, float* rho, float* u,
                              float* wss, cudaStream_t s) {
  return dispatch<MacroOp>(h->precision, h, fin, gather, tb, rho, u, wss, s);
}
cudaError_t hlb_launch_state(const hlb_solver* h, const void* fin, bool gather, int64_t tb, void* out,
                             cudaStream_t s) {
  return dispatch<StateOp>(h->precision, h, fin, gather, tb, out, s);
}
cudaError_t hlb_launch_init(const hlb_solver* h, void* f, double rho0, const float* u0, cudaStream_t s) {
  return dispatch<InitOp>(h->precision, h, f, rho0, u0, s);
}
cudaError_t hlb_launch_reduce(const hlb_solver* h, const void* fin, bool gather, int64_t tb, double* out_dev,
                              cudaStream_t s) {
  return dispatch<ReduceOp>(h->precision, h, fin, gather, tb, out_dev, s);
}
