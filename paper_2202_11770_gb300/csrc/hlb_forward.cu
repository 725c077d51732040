// hlb_forward.cu — forward kernels of the D3Q19 sparse-lattice solver.
//
// The step (arXiv 2202.11770, Section 3.2.2: load f, compute rho and u
// (Eqs. 5-6), f^eq (Eq. 4), collide (Eq. 3a), stream (Eq. 3b) with wall and
// iolet boundaries, store) runs as one fused kernel per time step over the
// whole site list; the paper's six per-site-type kernels become one kernel in
// which wall links are branch-free address selects and iolet links a rare
// per-site fix-up.  Two streaming schemes:
//
//  * pull A-B (k_step): read buffer A by gathering through the index table,
//    write buffer B; 188 B per FP32 site update with the compact index
//    table (224 B with the int32 one).
//  * AA pattern (k_aa_even / k_aa_odd, then k_aa_fix over iolet sites): one
//    buffer.  Even steps read a site's 19 slots and write them back swapped
//    (no index table); odd steps read 19 slots through the index table and
//    write the results to the very same 19 slots.  152 B (even) + 188 B
//    (odd; 224 B with the int32 table) per FP32 update.
//
// The bulk kernels take the index from its compact form (hlb_common.cuh,
// built by k_ctab_build) unless the lattice does not fit it; iolet-site
// paths and read-back kernels use the int32 table.
//
// Read modes of the readback kernels: LOCAL (the buffer holds f(t) in place),
// GATHER_AB (the buffer holds s'(t-1); boundaries applied while gathering),
// GATHER_AA (AA buffer after an even step; boundaries already written).
//
// k_macros: the property cache of Section 3.2.2 step 7 (rho, u) plus WSS.
// k_mass / k_flux / k_finish: FP64 reductions in a fixed order.
#include <math.h>

#include "hlb_internal.h"

using namespace hlb;

namespace {

constexpr int BLOCK = 256;
// Lanes a site for the iolet sites: a site's 19 directions spread over them,
// up to ceil(19 / lanes) a lane.  Measured on the 20M-site tree: the pull
// step's iolet sites 8 lanes (BF16 step 411 -> 405 us against 16, 418 at 32),
// the AA iolet pass 16 (8 lanes 1-2 us slower a step, 32 lanes 3 us slower).
constexpr int kStepIoletLanes = 8;
constexpr int kFixLanes = 16;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

// L2 prefetch hint: `bytes` (a multiple of 16) from a 16-byte aligned address.
__device__ __forceinline__ void l2_prefetch(const void* q, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(q)), "r"(bytes)
               : "memory");
}

// Called by the first warp of a bulk block: prefetch into L2 what the block
// that takes tile `tile` (about a wave of resident blocks later) reads
// first, so that its loads find L2 instead of waiting on DRAM.  Lanes 0-8:
// the tile's compact index words (row q, 256 sites).  With POPS, lanes
// 9-26: for direction i = lane - 8, the population row its gathers read
// (ROWOPP: row opp(i), as the AA odd step reads; else row i) from the
// tile's base for i, 320 sites wide (the sources of a tile span about 255
// sites on vessel lattices).  Every range is clamped to its array: ctab
// holds 9 rows of sn words, A 19 rows of n populations.
template <typename S, bool POPS, bool ROWOPP>
__device__ __forceinline__ void prefetch_tile(const S* A, const uint32_t* __restrict__ ctab,
                                              const int32_t* __restrict__ tbase, uint32_t n, uint32_t sn,
                                              uint32_t tile) {
  const uint32_t ntiles = (n + BLOCK - 1) / BLOCK;
  const int l = threadIdx.x & 31;
  if (tile >= ntiles) return;
  const uint64_t x0 = (uint64_t)tile * BLOCK;
  if (l < 9) {
    const uint64_t e = x0 + BLOCK < (uint64_t)sn ? x0 + BLOCK : (uint64_t)sn;  // sn: a multiple of 4
    l2_prefetch(ctab + (uint64_t)l * sn + x0, (uint32_t)((e - x0) * 4));
  } else if (POPS && l < 9 + Q - 1) {
    const int i = l - 8;
    const uint64_t b = (uint32_t)__ldg(tbase + (uint64_t)tile * CT_BASES + (i - 1));  // < n
    const uint64_t r = ROWOPP ? (uint64_t)lane_opp(i) : (uint64_t)i;
    const uint64_t e = b + 320 < (uint64_t)n ? b + 320 : (uint64_t)n;
    const uint64_t total = ((uint64_t)Q * n * sizeof(S) + 15) & ~15ull;  // within the 256-aligned section
    const uint64_t lo = ((r * n + b) * sizeof(S)) & ~15ull;
    const uint64_t hr = ((r * n + e) * sizeof(S) + 15) & ~15ull;
    const uint64_t hi = hr < total ? hr : total;
    if (hi > lo) l2_prefetch(reinterpret_cast<const char*>(A) + lo, (uint32_t)(hi - lo));
  }
}

// ---------------------------------------------------------------------------
// Pull A-B step from f(t) held in place (the first step after initialisation
// or set_state): no gather.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_step_local(const S* __restrict__ fin, S* __restrict__ fout,
                                                      const StepParams p) {
  using R = typename Real<S>::type;
  const int64_t n = p.n;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (x >= n) return;
  R h[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) h[i] = ldpop(fin + (int64_t)i * n + x);
  collide_emit<R>(h, omega_of<R>(p), [&](int i, R v) { stpop<S>(fout + (int64_t)i * n + x, v); });
}

// Post-collision population of direction i from the site's sums, with the
// operations of collide_emit.
template <typename R>
__device__ __forceinline__ R iolet_lane_out(int i, R h, R omega, R drho, R rho, R ux, R uy, R uz, R usq15) {
  const R om1 = R(1) - omega;
  if (i == 0) {
    const R ow = omega * wgt<R>(0);
    return fmadd(om1, h, fmadd(-(ow * rho), usq15, ow * drho));
  }
  const int ip = 2 * ((i - 1) >> 1) + 1;
  const R ow = omega * (ip <= 6 ? wgt<R>(1) : wgt<R>(7));
  const R cu = lane_cdotu<R>(ip, ux, uy, uz);
  const R a = fmadd(R(4.5) * cu, cu, -usq15);
  return fmadd(om1, h, fmadd(ow * rho, fmadd((i & 1) ? R(3) : R(-3), cu, a), ow * drho));
}
// The same step for the sites with iolet links, kStepIoletLanes lanes a
// site, lane h holding directions h, h + lanes, ... (gather, boundary value,
// collision).  Moments and collision sums run over the directions in the
// order of the per-thread code (collide_emit, and the read-back path
// iolet_fixup), so every value equals it bit for bit.  w is the lane
// group's site; a group past the end shadows site 0 and stores nothing (all
// 32 lanes take part in the shuffles).
template <typename S>
__device__ __forceinline__ void step_iolet_site(const S* __restrict__ fin, S* __restrict__ fout,
                                                const int32_t* __restrict__ src, const LinkRec* __restrict__ links,
                                                const double* __restrict__ amp, const int32_t* __restrict__ sites,
                                                int64_t nsites, const StepParams& p, int64_t w) {
  using R = typename Real<S>::type;
  constexpr int W = kStepIoletLanes, NE = (Q + W - 1) / W;
  const bool live = w < nsites;
  const int hl = threadIdx.x & (W - 1);
  const int64_t n = p.n, x = sites[live ? w : 0];
  int32_t c[NE];
  LinkRec L[NE];
  R h[NE], own[NE], a[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int i = e * W + hl;
    c[e] = (i >= 1 && i < Q) ? src[(int64_t)(i - 1) * p.sn + x] : 0;
    // link records and amplitudes load beside the populations, not after
    // them (record 0 exists whenever a site has an iolet link)
    L[e] = links[c[e] <= -2 ? -c[e] - 2 : 0];
    h[e] = own[e] = R(0);
    if (i < Q) {
      h[e] = ldpop(fin + (i == 0 ? x : (c[e] >= 0 ? (int64_t)i * n + c[e] : (int64_t)lane_opp(i) * n + x)));
      own[e] = ldpop(fin + (int64_t)i * n + x);
    }
    a[e] = BC<R>::amp(p, amp, L[e].kind == 0 && L[e].group >= 0 ? L[e].group : 0);
  }
  // moments of the stored s'(t-1) at x, in direction order
  R d = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const R vk = __shfl_sync(FULL_MASK, own[k / W], k % W, W);
    d += vk;
    if (cx(k)) jx += cx(k) > 0 ? vk : -vk;
    if (cy(k)) jy += cy(k) > 0 ? vk : -vk;
    if (cz(k)) jz += cz(k) > 0 ? vk : -vk;
  }
  const R rho_s = R(1) + d;
  const R ux = jx / rho_s, uy = jy / rho_s, uz = jz / rho_s;
#pragma unroll
  for (int e = 0; e < NE; ++e)
    if (c[e] <= -2) h[e] = lane_iolet_value<R>(e * W + hl, L[e], h[e], rho_s, ux, uy, uz, a[e], p);
  // collision: sums over opposite pairs as collide_emit forms them
  const R omega = omega_of<R>(p);
  R drho = __shfl_sync(FULL_MASK, h[0], 0, W), cjx = R(0), cjy = R(0), cjz = R(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int ip = 2 * q + 1;
    const R va = __shfl_sync(FULL_MASK, h[ip / W], ip % W, W), vb = __shfl_sync(FULL_MASK, h[(ip + 1) / W], (ip + 1) % W, W);
    const R sp = va + vb, dp = va - vb;
    drho += sp;
    if (cx(ip)) cjx = cx(ip) > 0 ? cjx + dp : cjx - dp;
    if (cy(ip)) cjy = cy(ip) > 0 ? cjy + dp : cjy - dp;
    if (cz(ip)) cjz = cz(ip) > 0 ? cjz + dp : cjz - dp;
  }
  const R rho = R(1) + drho;
  const R inv = R(1) / rho;
  const R cux = cjx * inv, cuy = cjy * inv, cuz = cjz * inv;
  const R usq15 = R(1.5) * fmadd(cuz, cuz, fmadd(cuy, cuy, cux * cux));
  if (!live) return;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int i = e * W + hl;
    if (i < Q) stpop<S>(fout + (int64_t)i * n + x, iolet_lane_out<R>(i, h[e], omega, drho, rho, cux, cuy, cuz, usq15));
  }
}

// Pull A-B step from s'(t-1) in one launch: gather f(t) through the index
// table (walls: the site's own opposite slot), collide, store coalesced.
// Every stride-th block (the first n_iolet_blocks of them) takes 32 iolet
// sites, 8 lanes each (step_iolet_site); the others take 256 bulk sites,
// a thread each, and leave iolet sites alone.  The iolet blocks, spread
// through the grid, run beside the bulk blocks instead of after them.
// WIDE: offsets within direction pairs (lattices above ~226M sites).  CT:
// bulk codes from the compact index table (iolet warps read the 32-bit one),
// and an L2 prefetch of the bulk tile `pf` tiles ahead, as in k_aa_odd.
template <typename S, bool WIDE, bool CT>
__global__ void __launch_bounds__(BLOCK, 5) k_step(const S* __restrict__ fin, S* __restrict__ fout,
                                                const int32_t* __restrict__ src, const uint32_t* __restrict__ ctab,
                                                const int32_t* __restrict__ tbase, const LinkRec* __restrict__ links,
                                                const double* __restrict__ amp, const int32_t* __restrict__ sites,
                                                int64_t nsites, unsigned n_iolet_blocks, const BlockDiv stride,
                                                const uint32_t* __restrict__ imask, uint32_t pf, uint32_t tile0,
                                                const StepParams p) {
  using R = typename Real<S>::type;
  const unsigned b = blockIdx.x, j = block_div(b, stride);
  if (b == j * stride.d && j < n_iolet_blocks) {
    pdl_wait();
    pdl_trigger();
    step_iolet_site<S>(fin, fout, src, links, amp, sites, nsites, p, ((int64_t)j * BLOCK + threadIdx.x) / kStepIoletLanes);
    return;
  }
  const uint32_t n = (uint32_t)p.n, sn = (uint32_t)p.sn;
  const uint32_t tile = tile0 + b - min(n_iolet_blocks, j + 1);
  const uint32_t x = tile * BLOCK + threadIdx.x;
  if (CT && pf && threadIdx.x < 32) prefetch_tile<S, sizeof(S) >= 4, false>(fin, ctab, tbase, n, sn, tile + pf);
  uint32_t off[Q];
  const bool live = x < n;
  // sites with an iolet link are stepped by the iolet warps (one 32-bit mask
  // word per warp instead of a test of each of the 18 codes)
  bool skip = true;
  if (live) {
    load_offsets<CT, WIDE, LD_STREAM, false>(src, ctab, tbase, sn, n, x, tile, off);
    skip = (__ldg(imask + (x >> 5)) >> (x & 31)) & 1u;
  }
  pdl_wait();
  pdl_trigger();
  if (skip) return;
  R h[Q];
  h[0] = ldpop(fin + x);
  // fluid source: row i at s; otherwise row opp(i) at x (bounce-back)
#pragma unroll
  for (int i = 1; i < Q; ++i) h[i] = ldpop(at<WIDE>(fin, i, n, off[i]));
  collide<R>(h, omega_of<R>(p));
  if (WIDE) {
    stpop<S>(fout + x, h[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) stpop<S>(at<WIDE>(fout, i, n, slot<WIDE>(i, n, x)), h[i]);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) stpop<S>(fout + (uint32_t)i * n + x, h[i]);
  }
}

// ---------------------------------------------------------------------------
// AA pattern.
// ---------------------------------------------------------------------------
// Even step: f(t) in place -> collide -> s'(t) stored swapped (slot ibar).
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_aa_even(S* A, const StepParams p) {
  using R = typename Real<S>::type;
  const int64_t n = p.n;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (x >= n) return;
  R h[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) h[i] = to_real(A[(int64_t)i * n + x]);
  collide<R>(h, omega_of<R>(p));
#pragma unroll
  for (int i = 0; i < Q; ++i) stpop<S>(A + (int64_t)opp(i) * n + x, h[i]);
}

// Even step for 16-bit storage, two neighbouring sites per thread with 4-byte
// accesses (rows are 4-byte aligned when n is even).  The two collisions run
// in paired FP32 instructions (collide2), which halves the arithmetic
// instructions of a kernel whose 16-bit traffic leaves instruction issue as
// a limit.  Four blocks per SM (64 registers, a few bytes of spill) measured
// 4-5 % faster than the scalar collisions, and than three blocks without
// the spill.
template <typename S> struct Pair;
template <> struct Pair<__nv_bfloat16> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ float2 to(T v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ T from(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <> struct Pair<__half> {
  using T = __half2;
  static __device__ __forceinline__ float2 to(T v) { return __half22float2(v); }
  static __device__ __forceinline__ T from(float a, float b) { return __floats2half2_rn(a, b); }
};
template <> struct Pair<float> {
  using T = float2;
  static __device__ __forceinline__ float2 to(T v) { return v; }
  static __device__ __forceinline__ T from(float a, float b) { return make_float2(a, b); }
};

// Paired FP32 arithmetic (sm_100 and later): one instruction applies the
// operation to .x and .y, each rounded as the scalar operation is.
__device__ __forceinline__ float2 p_splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// collide() of two sites at once, h[i] = (site x, site x + 1).  Directions
// 2p-1 and 2p are opposite, so each pair shares c.u and 4.5 (c.u)^2 - 1.5 u.u
// and differs only in the sign of the 3 c.u term.
__device__ __forceinline__ void collide2(float2* h, float omega) {
  float2 d = h[0];
#pragma unroll
  for (int i = 1; i < Q; ++i) d = p_add(d, h[i]);
  // momentum: each component is the sum over the pairs that move along it
  float2 jx = p_sub(h[1], h[2]), jy = p_sub(h[3], h[4]), jz = p_sub(h[5], h[6]);
#pragma unroll
  for (int i = 7; i < Q; ++i) {
    if (cx(i)) jx = cx(i) > 0 ? p_add(jx, h[i]) : p_sub(jx, h[i]);
    if (cy(i)) jy = cy(i) > 0 ? p_add(jy, h[i]) : p_sub(jy, h[i]);
    if (cz(i)) jz = cz(i) > 0 ? p_add(jz, h[i]) : p_sub(jz, h[i]);
  }
  const float2 rho = p_add(p_splat(1.f), d);
  const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
  const float2 ux = p_mul(jx, inv), uy = p_mul(jy, inv), uz = p_mul(jz, inv);
  const float2 nusq = p_mul(p_splat(-1.5f), p_fma(uz, uz, p_fma(uy, uy, p_mul(ux, ux))));
  const float2 om = p_splat(omega);
  {  // rest population: c.u = 0
    const float2 heq = p_mul(p_splat(1.f / 3.f), p_fma(rho, nusq, d));
    h[0] = p_fma(om, p_sub(heq, h[0]), h[0]);
  }
#pragma unroll
  for (int q = 1; q < 10; ++q) {
    const int i = 2 * q - 1;  // c_i has a positive first nonzero component
    float2 cu = cx(i) ? ux : uy;
    if (cx(i) && cy(i)) cu = cy(i) > 0 ? p_add(ux, uy) : p_sub(ux, uy);
    if (cx(i) && cz(i)) cu = cz(i) > 0 ? p_add(ux, uz) : p_sub(ux, uz);
    if (!cx(i) && cz(i)) cu = cy(i) ? (cz(i) > 0 ? p_add(uy, uz) : p_sub(uy, uz)) : uz;
    const float2 a = p_fma(p_mul(p_splat(4.5f), cu), cu, nusq);
    const float2 tp = p_fma(p_splat(3.f), cu, a), tm = p_fma(p_splat(-3.f), cu, a);
    const float2 w = p_splat(wgt<float>(i));
    const float2 ep = p_mul(w, p_fma(rho, tp, d)), em = p_mul(w, p_fma(rho, tm, d));
    h[i] = p_fma(om, p_sub(ep, h[i]), h[i]);
    h[i + 1] = p_fma(om, p_sub(em, h[i + 1]), h[i + 1]);
  }
}

template <typename S>
__global__ void __launch_bounds__(BLOCK, 4) k_aa_even2(S* A, const StepParams p) {
  using P = Pair<S>;
  using T = typename P::T;
  const int64_t n = p.n;
  const int64_t x = 2 * ((int64_t)blockIdx.x * BLOCK + threadIdx.x);
  pdl_wait();
  pdl_trigger();
  if (x >= n) return;
  T* A2 = reinterpret_cast<T*>(A);
  const int64_t n2 = n / 2, x2 = x / 2;
  float2 h[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) h[i] = P::to(A2[(int64_t)i * n2 + x2]);
  collide2(h, p.omegaf);
#pragma unroll
  for (int i = 0; i < Q; ++i) __stcs(A2 + (int64_t)opp(i) * n2 + x2, P::from(h[i].x, h[i].y));
}

// collide_emit() of two sites at once, h[i] = (site x, site x + 1): the same
// operations in the same order, each pair of scalar operations one paired
// FP32 instruction (rounded as the scalar one), so each site gets the bits
// of the per-thread collision.
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_cdotu(int i, float2 ux, float2 uy, float2 uz) {
  float2 s = p_splat(0.f);
  if (cx(i)) s = p_add(s, cx(i) > 0 ? ux : p_neg(ux));
  if (cy(i)) s = p_add(s, cy(i) > 0 ? uy : p_neg(uy));
  if (cz(i)) s = p_add(s, cz(i) > 0 ? uz : p_neg(uz));
  return s;
}
template <typename Emit>
__device__ __forceinline__ void collide_pair(const float2* h, float omega, Emit&& emit) {
  float2 drho = h[0], jx = p_splat(0.f), jy = p_splat(0.f), jz = p_splat(0.f);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const int i = 2 * p + 1;
    const float2 sp = p_add(h[i], h[i + 1]), dp = p_sub(h[i], h[i + 1]);
    drho = p_add(drho, sp);
    if (cx(i)) jx = cx(i) > 0 ? p_add(jx, dp) : p_sub(jx, dp);
    if (cy(i)) jy = cy(i) > 0 ? p_add(jy, dp) : p_sub(jy, dp);
    if (cz(i)) jz = cz(i) > 0 ? p_add(jz, dp) : p_sub(jz, dp);
  }
  const float2 rho = p_add(p_splat(1.f), drho);
  const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
  const float2 ux = p_mul(jx, inv), uy = p_mul(jy, inv), uz = p_mul(jz, inv);
  const float2 usq15 = p_mul(p_splat(1.5f), p_fma(uz, uz, p_fma(uy, uy, p_mul(ux, ux))));
  const float2 om1 = p_splat(1.f - omega);
  float2 wr[3], wd[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float ow = omega * wgt<float>(c == 0 ? 0 : (c == 1 ? 1 : 7));
    wr[c] = p_mul(p_splat(ow), rho);
    wd[c] = p_mul(p_splat(ow), drho);
  }
  emit(0, p_fma(om1, h[0], p_fma(p_neg(wr[0]), usq15, wd[0])));
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const int i = 2 * p + 1, c = i <= 6 ? 1 : 2;
    const float2 cu = p_cdotu(i, ux, uy, uz);
    const float2 a = p_fma(p_mul(p_splat(4.5f), cu), cu, p_neg(usq15));
    emit(i, p_fma(om1, h[i], p_fma(wr[c], p_fma(p_splat(3.f), cu, a), wd[c])));
    emit(i + 1, p_fma(om1, h[i + 1], p_fma(wr[c], p_fma(p_splat(-3.f), cu, a), wd[c])));
  }
}

// Pull A-B step (k_step) with two neighbouring sites x, x + 1 per thread (n
// even, compact table, 32-bit offsets; FP32 or 16-bit storage): the index
// words of both in one 8-byte load per row, the two collisions in paired
// FP32 instructions (collide_pair: the bits of k_step) and one store of the
// pair per direction; the gathers stay one per site and direction.  A block
// takes two tiles.  A pair with one iolet site stores only its other site.
// Three blocks per SM (80 registers), on the 20M-site tree: BF16 447 -> 419
// us (four blocks, 64 registers with spills: 485 us), FP32 577 -> 567 us.
// The same pairing in the AA odd step, whose stores scatter, was slower
// (463 -> 563 us BF16).
template <typename S>
__global__ void __launch_bounds__(BLOCK, 3) k_step2(const S* __restrict__ fin, S* __restrict__ fout,
                                                 const int32_t* __restrict__ src, const uint32_t* __restrict__ ctab,
                                                 const int32_t* __restrict__ tbase, const LinkRec* __restrict__ links,
                                                 const double* __restrict__ amp, const int32_t* __restrict__ sites,
                                                 int64_t nsites, unsigned n_iolet_blocks, const BlockDiv stride,
                                                 const uint32_t* __restrict__ imask, uint32_t pf,
                                                 const StepParams p) {
  using P = Pair<S>;
  using T = typename P::T;
  const unsigned b = blockIdx.x, j = block_div(b, stride);
  if (b == j * stride.d && j < n_iolet_blocks) {
    pdl_wait();
    pdl_trigger();
    step_iolet_site<S>(fin, fout, src, links, amp, sites, nsites, p, ((int64_t)j * BLOCK + threadIdx.x) / kStepIoletLanes);
    return;
  }
  const uint32_t n = (uint32_t)p.n, sn = (uint32_t)p.sn;
  const uint32_t k = b - min(n_iolet_blocks, j + 1);  // bulk block: tiles 2k, 2k + 1
  const uint32_t x = 2 * (k * BLOCK + threadIdx.x);
  const uint32_t tile = x / CT_TILE;
  if (pf && threadIdx.x < 64) prefetch_tile<S, false, false>(fin, ctab, tbase, n, sn, 2 * (k + pf) + (threadIdx.x >> 5));
  uint32_t m = 3u;  // bit 0: x is stepped elsewhere (iolet warps, or x >= n), bit 1: x + 1
  uint32_t off[2][Q];
  if (x < n) {
    m = (__ldg(imask + (x >> 5)) >> (x & 31)) & 3u;  // x even: both bits in one word
    uint2 w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = __ldcs(reinterpret_cast<const uint2*>(ctab + (uint32_t)q * sn + x));
    const int4* tb = reinterpret_cast<const int4*>(tbase + (uint64_t)tile * CT_BASES);
    int bs[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int4 v = __ldg(tb + q);
      bs[4 * q] = v.x;
      bs[4 * q + 1] = v.y;
      bs[4 * q + 2] = v.z;
      bs[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t wa = w[(i - 1) >> 1].x, wb = w[(i - 1) >> 1].y;
      const uint32_t oa = (i & 1) ? (wa & 0xffffu) : (wa >> 16), ob = (i & 1) ? (wb & 0xffffu) : (wb >> 16);
      off[0][i] = oa < CT_IOLET ? (uint32_t)i * n + (uint32_t)bs[i - 1] + oa : (uint32_t)opp(i) * n + x;
      off[1][i] = ob < CT_IOLET ? (uint32_t)i * n + (uint32_t)bs[i - 1] + ob : (uint32_t)opp(i) * n + x + 1;
    }
  }
  pdl_wait();
  pdl_trigger();
  if (m == 3u) return;
  const T* fin2 = reinterpret_cast<const T*>(fin);
  float2 h[Q];
  h[0] = P::to(__ldg(fin2 + x / 2));
#pragma unroll
  for (int i = 1; i < Q; ++i) h[i] = make_float2(ldpop(fin + off[0][i]), ldpop(fin + off[1][i]));
  if (m == 0u) {
    T* fout2 = reinterpret_cast<T*>(fout);
    collide_pair(h, p.omegaf, [&](int i, float2 v) { __stcs(fout2 + ((uint32_t)i * n + x) / 2, P::from(v.x, v.y)); });
  } else {
    const uint32_t y = m == 1u ? x + 1 : x;  // the pair's site without iolet links
    collide_pair(h, p.omegaf,
                 [&](int i, float2 v) { stpop<S>(fout + (uint32_t)i * n + y, m == 1u ? v.y : v.x); });
  }
}

// Boundary value of iolet link (pull direction i, record L) at a site whose
// pre-collision moments at time t are (drho, u) and whose outgoing
// post-collision population is `out` (= s'_ibar): incoming f_i(t+1) - w_i.
template <typename R>
__device__ __forceinline__ R iolet_value(int i, const LinkRec& L, R out, R rho, R ux, R uy, R uz,
                                         const double* __restrict__ amp, const StepParams& p) {
  const IoletParam& io = p.io[L.iolet];
  if (L.kind == 0) {
    R r = p.ladd_rho_one ? R(1) : rho;
    return out + BC<R>::coef(L) * r * BC<R>::amp(p, amp, L.group) * BC<R>::val(p, L.iolet);
  }
  R gx = ux, gy = uy, gz = uz;
  if (!p.ghost_full_u) {
    R un = gx * BC<R>::nx(io) + gy * BC<R>::ny(io) + gz * BC<R>::nz(io);
    gx = un * BC<R>::nx(io);
    gy = un * BC<R>::ny(io);
    gz = un * BC<R>::nz(io);
  }
  R drho = BC<R>::val(p, L.iolet);
  R usq15 = R(1.5) * (gx * gx + gy * gy + gz * gz);
  return heq<R>(i, drho, R(1) + drho, gx, gy, gz, usq15);
}

// After an AA step at time t: overwrite the slots that the iolet links of
// each iolet site read in the next step with their boundary values, and
// record the mass each link lets in.  A lane's codes, stored values and (iolet
// links) link records are one load each, so the pass is a few rounds of
// loads whatever the site's number of iolet links; records and amplitudes
// load before the wait for the step kernel.  The site's stored post-collision
// populations s'_ibar(x) sit in slot i of x after an even step, and in the
// slot it read direction i from after an odd step; an iolet link's slot is
// slot i of x in both cases.  Boundary values use the moments of these
// stored values, as the A-B gather does, summed over s'_0, s'_1, ... in the
// order of the A-B warp path, so the two schemes give the same bits.
// icode[q][i - 1] is the index code of direction i at iolet site q: 72
// contiguous bytes a site.  Two iolet sites a warp: 16 lanes a site, lane h
// holding direction h and, for h < 3, also direction 16 + h (32 registers,
// 8 blocks per SM).  Against one warp a site it runs in half the warps: the
// 54k iolet sites of the 20M-site tree in 2.8 waves instead of 5.6, about
// 3 us less a step.
template <typename S, bool ODD>
__global__ void __launch_bounds__(256, 8) k_aa_fix(S* A, const int32_t* __restrict__ icode,
                                                 const LinkRec* __restrict__ links, const double* __restrict__ amp,
                                                 const int32_t* __restrict__ sites, int64_t nsites,
                                                 const StepParams p, double* __restrict__ lflux) {
  using R = typename Real<S>::type;
  constexpr int W = kFixLanes, NE = (Q + W - 1) / W;
  const int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
  const bool live = q0 < nsites;
  const int64_t q = live ? q0 : 0;  // lanes past the end shadow site 0 and store nothing
  const int hl = threadIdx.x & (W - 1);
  const int64_t x = __ldg(sites + q);
  int32_t c[NE];
  LinkRec L[NE];
  R a[NE], v[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int i = e * W + hl;
    c[e] = (i >= 1 && i < Q) ? __ldg(icode + q * (Q - 1) + (i - 1)) : 0;
    // link records and amplitudes do not change between steps: loaded before
    // the wait for the step kernel (record 0 exists whenever there are iolet sites)
    L[e] = links[c[e] <= -2 ? -c[e] - 2 : 0];
    a[e] = BC<R>::amp(p, amp, L[e].kind == 0 && L[e].group >= 0 ? L[e].group : 0);
  }
  pdl_wait();
  pdl_trigger();
  const int64_t n = p.n;
  // s'_ibar(x): the value in the slot the link of direction i reads
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int i = e * W + hl;
    v[e] = R(0);
    if (i < Q) v[e] = to_real(A[i == 0 ? x : (ODD ? aa_addr(i, c[e], n, x) : (int64_t)i * n + x)]);
  }
  // rho = 1 + sum s'_k, j = sum s'_k c_k in direction order; s'_k sits with direction opp(k)
  R d = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int o = opp(k);
    const R vk = __shfl_sync(FULL_MASK, v[o / W], o % W, W);
    d += vk;
    if (cx(k)) jx += cx(k) > 0 ? vk : -vk;
    if (cy(k)) jy += cy(k) > 0 ? vk : -vk;
    if (cz(k)) jz += cz(k) > 0 ? vk : -vk;
  }
  const R rho = R(1) + d;
  const R ux = jx / rho, uy = jy / rho, uz = jz / rho;
  if (!live) return;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int i = e * W + hl;
    if (c[e] <= -2) {
      const R val = lane_iolet_value<R>(i, L[e], v[e], rho, ux, uy, uz, a[e], p);
      lflux[-c[e] - 2] = (double)val - (double)v[e];
      A[(int64_t)i * n + x] = from_real<S>(val);
    }
  }
}

// Odd step: gather f(t) through the index table, collide, and write each
// post-collision population into the slot it came from, where the site
// downstream (or, across a wall or iolet, the site itself) reads it in the
// next (even) step.  Iolet links get their boundary values from k_aa_fix.
// The 18 slot offsets (32-bit) are computed once and held in registers for
// the stores, so the index row is read once.  Five resident blocks per SM
// (48 registers, a few bytes of spill in FP32) measured fastest.  WIDE:
// offsets within direction pairs (lattices above ~226M sites), which need a
// few more registers: four blocks per SM (64 registers) measured 8 % faster
// than five with their spills.  CT: codes from the compact index table, and
// the first warp prefetches into L2 the tile `pf` blocks ahead (0: none):
// index words, and for 4- and 8-byte storage the gathered rows (for 16-bit
// storage the rows measured slower).  With 32-bit offsets pf is 3 blocks per
// SM, 0.6 of a wave: FP32 odd step 608 us at one wave, 599 us at 0.6, 615 us
// at 0.2 (16-bit unchanged); the wide form keeps one wave (4 blocks per SM).
template <typename S, bool WIDE, bool CT>
__global__ void __launch_bounds__(BLOCK, WIDE ? 4 : 5) k_aa_odd(S* A, const int32_t* __restrict__ src,
                                                               const uint32_t* __restrict__ ctab,
                                                               const int32_t* __restrict__ tbase, uint32_t pf,
                                                               const StepParams p) {
  using R = typename Real<S>::type;
  const uint32_t n = (uint32_t)p.n, sn = (uint32_t)p.sn;
  const uint32_t x = blockIdx.x * BLOCK + threadIdx.x;
  if (CT && pf && threadIdx.x < 32) prefetch_tile<S, sizeof(S) >= 4, true>(A, ctab, tbase, n, sn, blockIdx.x + pf);
  int32_t code[Q - 1];
  if (x < n) load_codes<CT, WIDE, LD_NC>(src, ctab, tbase, sn, x, blockIdx.x, code);
  pdl_wait();
  pdl_trigger();
  if (x >= n) return;
  uint32_t off[Q];
  R h[Q];
  h[0] = to_real(A[x]);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int32_t s = code[i - 1];
    // slot opp(i) of the source, or slot i of x itself across a wall or iolet
    off[i] = s >= 0 ? slot<WIDE>(opp(i), n, (uint32_t)s) : slot<WIDE>(i, n, x);
    h[i] = to_real(*at<WIDE>(A, i, n, off[i]));
  }
  collide<R>(h, omega_of<R>(p));
  stpop<S>(A + x, h[0]);
#pragma unroll
  for (int i = 1; i < Q; ++i) stpop<S>(at<WIDE>(A, i, n, off[i]), h[opp(i)]);
}

// ---------------------------------------------------------------------------
// Compact index table (layout in hlb_common.cuh), built once from the 32-bit
// table: one block per tile.  Per direction the block finds the smallest and
// largest fluid source of its sites (warp min/max, then across the eight
// warps), writes the base, and each thread its offset; pairs of directions
// share a word.  Padding entries (n <= x < sn) read as walls.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CT_TILE) k_ctab_build(const int32_t* __restrict__ src, int64_t n, int64_t sn,
                                                        uint32_t* __restrict__ ctab, int32_t* __restrict__ tbase,
                                                        int32_t* __restrict__ misfit) {
  static_assert(CT_TILE == 256, "eight warps a tile");
  __shared__ uint32_t smin[8], smax[8];
  const int64_t x = (int64_t)blockIdx.x * CT_TILE + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t word = 0;
  for (int i = 1; i < Q; ++i) {
    const int32_t s = x < n ? src[(int64_t)(i - 1) * sn + x] : -1;
    uint32_t lo = __reduce_min_sync(0xffffffffu, s >= 0 ? (uint32_t)s : 0xffffffffu);
    uint32_t hi = __reduce_max_sync(0xffffffffu, s >= 0 ? (uint32_t)s : 0u);
    if (lane == 0) {
      smin[wid] = lo;
      smax[wid] = hi;
    }
    __syncthreads();
    lo = smin[0];
    hi = smax[0];
    for (int k = 1; k < 8; ++k) {
      lo = min(lo, smin[k]);
      hi = max(hi, smax[k]);
    }
    __syncthreads();
    const bool any = lo != 0xffffffffu;  // some site of the tile has a fluid source
    const uint32_t base = any ? lo : 0u;
    if (threadIdx.x == 0) {
      tbase[(int64_t)blockIdx.x * CT_BASES + (i - 1)] = (int32_t)base;
      if (any && hi - lo > CT_MAX_SPAN) atomicOr(misfit, 1);
    }
    const uint32_t o = s >= 0 ? ((uint32_t)s - base) & 0xffffu : (s == -1 ? CT_WALL : CT_IOLET);
    if (i & 1) {
      word = o;
    } else {
      word |= o << 16;
      if (x < sn) ctab[(int64_t)(i / 2 - 1) * sn + x] = word;
    }
  }
  if (threadIdx.x < CT_BASES - (Q - 1)) tbase[(int64_t)blockIdx.x * CT_BASES + (Q - 1) + threadIdx.x] = 0;
}

// ---------------------------------------------------------------------------
// Read-back kernels.
// ---------------------------------------------------------------------------
// Density, velocity and wall shear stress of f(t).
template <typename S, int MODE>
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
  load_state<S, MODE>(fin, src, links, amp, p, x, h);
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
    if (src[(int64_t)(i - 1) * p.sn + x] == -1) {
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
  R k = -(R(1) - R(0.5) * omega_of<R>(p));
  R tx = k * (pxx * nx + pxy * ny + pxz * nz);
  R ty = k * (pxy * nx + pyy * ny + pyz * nz);
  R tz = k * (pxz * nx + pyz * ny + pzz * nz);
  R tn = tx * nx + ty * ny + tz * nz;
  tx -= tn * nx;
  ty -= tn * ny;
  tz -= tn * nz;
  wss_out[x] = (float)sqrt(tx * tx + ty * ty + tz * tz);
}

// Shifted pre-collision state f(t) - w into out [19][n] (row < 0), or only
// direction `row` into out [n].
template <typename S, int MODE>
__global__ void __launch_bounds__(BLOCK) k_state(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                 const LinkRec* __restrict__ links,
                                                 const double* __restrict__ amp, const StepParams p,
                                                 S* __restrict__ out, int row) {
  using R = typename Real<S>::type;
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (x >= p.n) return;
  R h[Q];
  load_state<S, MODE>(fin, src, links, amp, p, x, h);
  if (row >= 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (i == row) out[x] = from_real<S>(h[i]);
    return;
  }
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

// Per-block sums of drho (mass - sites) over the sites [lo, hi) into
// part[blockIdx.x].
template <typename S, int MODE>
__global__ void __launch_bounds__(BLOCK) k_mass(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                const LinkRec* __restrict__ links,
                                                const double* __restrict__ amp, const StepParams p, int64_t lo,
                                                int64_t hi, double* __restrict__ part) {
  using R = typename Real<S>::type;
  __shared__ double sh[BLOCK / 32];
  const int64_t x = lo + (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  double d = 0;
  if (x < hi) {
    R h[Q];
    load_state<S, MODE>(fin, src, links, amp, p, x, h);
#pragma unroll
    for (int i = 0; i < Q; ++i) d += (double)h[i];
  }
  double s = block_sum(d, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Per-iolet flux of the A-B scheme: one block per iolet over its link
// records, in order, recomputed from the post-collision state s'(t-1).
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_flux(const S* __restrict__ fin, const LinkRec* __restrict__ links,
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
    const Macro<R> ms = moments<R>(own);
    const int j = L.dir;
    R out = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (i == opp(j)) out = own[i];
    R val = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (i == j) val = iolet_value<R>(i, L, out, ms.rho, ms.ux, ms.uy, ms.uz, amp, p);
    acc += (double)val - (double)out;
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[1 + k] = s;
}

// Per-iolet flux of the AA scheme: sum of the per-link values the last step
// recorded, one block per iolet, in order.
__global__ void __launch_bounds__(BLOCK) k_flux_sum(const double* __restrict__ lflux,
                                                    const int64_t* __restrict__ begin, double* __restrict__ out) {
  __shared__ double sh[BLOCK / 32];
  const int k = blockIdx.x;
  double acc = 0;
  for (int64_t r = begin[k] + threadIdx.x; r < begin[k + 1]; r += BLOCK) acc += lflux[r];
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
// dispatch
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

// One pull A-B gather step over the bulk tiles [tile0, tile0 + ntiles) and,
// with `iolets`, the iolet sites (the whole step: tile0 = 0, all tiles).
template <typename S>
cudaError_t launch_gather(const hlb_solver* h, const void* fin, void* fout, const StepParams& p, uint32_t tile0,
                          uint32_t ntiles, bool iolets, cudaStream_t s) {
  constexpr unsigned per_block = BLOCK / kStepIoletLanes;  // iolet sites a block
  const unsigned gi = iolets ? (unsigned)((h->n_iolet_sites + per_block - 1) / per_block) : 0u;
  const unsigned grid = gi + ntiles;
  if (grid == 0) return cudaSuccess;
  if constexpr (sizeof(S) <= 4) {
    if (h->compact && h->off32 && h->n % 2 == 0 && tile0 == 0 && ntiles == grid_for(h->n)) {
      const unsigned g2 = gi + (unsigned)((h->n + 2 * BLOCK - 1) / (2 * BLOCK));
      return launch_pdl(k_step2<S>, g2, BLOCK, s, (const S*)fin, (S*)fout, h->d_src, h->d_ctab, h->d_tbase,
                        h->d_links, h->d_amp, h->d_iolet_sites, h->n_iolet_sites, gi,
                        make_block_div(gi ? g2 / gi : 1), h->d_imask, (uint32_t)h->n_sm * 3u, p);
    }
  }
  auto kernel = h->compact ? (h->off32 ? k_step<S, false, true> : k_step<S, true, true>)
                           : (h->off32 ? k_step<S, false, false> : k_step<S, true, false>);
  return launch_pdl(kernel, grid, BLOCK, s, (const S*)fin, (S*)fout, h->d_src, h->d_ctab, h->d_tbase, h->d_links,
                    h->d_amp, h->d_iolet_sites, h->n_iolet_sites, gi, make_block_div(gi ? grid / gi : 1), h->d_imask,
                    (uint32_t)h->n_sm * 5u, tile0, p);
}

template <typename S>
struct StepOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, void* fout, bool gather, int64_t tb,
                         cudaStream_t s) {
    StepParams p = h->params(tb);
    if (gather) return launch_gather<S>(h, fin, fout, p, 0, grid_for(h->n), true, s);
    return launch_pdl(k_step_local<S>, grid_for(h->n), BLOCK, s, (const S*)fin, (S*)fout, p);
  }
};

template <typename S>
struct StepRangeOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, void* fout, int64_t tb, int64_t tile0,
                         int64_t ntiles, bool iolets, cudaStream_t s) {
    StepParams p = h->params(tb);
    return launch_gather<S>(h, fin, fout, p, (uint32_t)tile0, (uint32_t)ntiles, iolets, s);
  }
};

template <typename S>
cudaError_t aa_even(const hlb_solver* h, S* A, const StepParams& p, cudaStream_t s) {
  return launch_pdl(k_aa_even<S>, grid_for(h->n), BLOCK, s, A, p);
}
template <typename S>
cudaError_t aa_even_pairs(const hlb_solver* h, S* A, const StepParams& p, cudaStream_t s) {
  if (h->n % 2 == 0) return launch_pdl(k_aa_even2<S>, grid_for(h->n / 2), BLOCK, s, A, p);
  return launch_pdl(k_aa_even<S>, grid_for(h->n), BLOCK, s, A, p);
}
template <>
cudaError_t aa_even<__nv_bfloat16>(const hlb_solver* h, __nv_bfloat16* A, const StepParams& p, cudaStream_t s) {
  return aa_even_pairs<__nv_bfloat16>(h, A, p, s);
}
template <>
cudaError_t aa_even<__half>(const hlb_solver* h, __half* A, const StepParams& p, cudaStream_t s) {
  return aa_even_pairs<__half>(h, A, p, s);
}

template <typename S>
struct AAOp {
  static cudaError_t run(const hlb_solver* h, void* A, bool odd, int64_t t, cudaStream_t s) {
    StepParams p = h->params(t);
    cudaError_t e;
    if (odd)
      e = launch_pdl(h->compact ? (h->off32 ? k_aa_odd<S, false, true> : k_aa_odd<S, true, true>)
                                : (h->off32 ? k_aa_odd<S, false, false> : k_aa_odd<S, true, false>),
                     grid_for(h->n), BLOCK, s, (S*)A, h->d_src, h->d_ctab, h->d_tbase,
                     (uint32_t)h->n_sm * (h->off32 ? 3u : 4u), p);
    else
      e = aa_even<S>(h, (S*)A, p, s);
    if (e != cudaSuccess || h->n_iolet_sites == 0) return e;
    constexpr int per_block = 256 / kFixLanes;  // iolet sites a block
    const unsigned g = (unsigned)((h->n_iolet_sites + per_block - 1) / per_block);
    return launch_pdl(odd ? k_aa_fix<S, true> : k_aa_fix<S, false>, g, 256, s, (S*)A, h->d_icode, h->d_links,
                      h->d_amp, h->d_iolet_sites, h->n_iolet_sites, p, h->d_lflux);
  }
};

#define HLB_MODE_SWITCH(mode, KERNEL_LAUNCH)                  \
  switch (mode) {                                              \
    case HLB_READ_GATHER_AB: { constexpr int M = HLB_READ_GATHER_AB; KERNEL_LAUNCH; break; } \
    case HLB_READ_GATHER_AA: { constexpr int M = HLB_READ_GATHER_AA; KERNEL_LAUNCH; break; } \
    default: { constexpr int M = HLB_READ_LOCAL; KERNEL_LAUNCH; break; }                      \
  }

template <typename S>
struct MacroOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, int mode, int64_t tb, float* rho, float* u,
                         float* wss, cudaStream_t s) {
    StepParams p = h->params(tb);
    const float* nrm = h->has_normals ? h->d_normal : nullptr;
    HLB_MODE_SWITCH(mode, (k_macros<S, M><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links,
                                                                             h->d_amp, nrm, p, rho, u, wss)));
    return cudaGetLastError();
  }
};

// Per-iolet monitor of f(t): block k walks the sites with a link to iolet k
// (ilist[ioff[k] .. ioff[k+1])) and writes out[k] = max |u| and
// out[K + k] = mean rho over them.  Per-thread partial sums run in a fixed
// stride order and the block combines them in a fixed tree, so the result
// does not depend on scheduling.
template <typename S, int MODE>
__global__ void __launch_bounds__(256) k_iolet_monitor(const S* __restrict__ fin, const int32_t* __restrict__ src,
                                                       const LinkRec* __restrict__ links,
                                                       const double* __restrict__ amp, const StepParams p,
                                                       const int64_t* __restrict__ ioff,
                                                       const int32_t* __restrict__ ilist, double* __restrict__ out) {
  using R = typename Real<S>::type;
  __shared__ double smax[256], ssum[256];
  const int k = blockIdx.x;
  const int64_t b = ioff[k], e = ioff[k + 1];
  double umax = 0.0, rsum = 0.0;
  for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) {
    R h[Q];
    load_state<S, MODE>(fin, src, links, amp, p, ilist[q], h);
    const Macro<R> m = moments<R>(h);
    const double u2 = (double)m.ux * m.ux + (double)m.uy * m.uy + (double)m.uz * m.uz;
    umax = fmax(umax, sqrt(u2));
    rsum += (double)m.rho;
  }
  smax[threadIdx.x] = umax;
  ssum[threadIdx.x] = rsum;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
      ssum[threadIdx.x] += ssum[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[k] = smax[0];
    out[gridDim.x + k] = e > b ? ssum[0] / (double)(e - b) : 0.0;
  }
}

// Windkessel outlets after a step (block k = iolet k; other iolets return).
// q = -(mass that enters through outlet k to produce the current state f):
//  * AA: the fix-up pass has just written f's boundary values with ioval[k]
//    and recorded the per-link masses; q is their sum.
//  * A-B: f's boundary values are applied by the next gather.  That gather
//    uses the value computed one update earlier (iovnext[k]), which `shift`
//    moves into ioval[k]; q is then recomputed from the post-collision state
//    `fin` with it, exactly as the gather will see it.
// Then rho_c <- rho_c + (q - (rho_c - rho_d) / Rd) / C and the next ghost
// density rho_c + Rp q (C = 0: rho_d + (Rp + Rd) q) goes to ioval[k] (AA) or
// iovnext[k] (A-B), minus 1.
template <typename S, bool AA>
__global__ void __launch_bounds__(BLOCK) k_wk_update(const S* __restrict__ fin, const LinkRec* __restrict__ links,
                                                     const double* __restrict__ amp, const StepParams p,
                                                     const int64_t* __restrict__ begin,
                                                     const double* __restrict__ lflux,
                                                     const double* __restrict__ par, double* __restrict__ state,
                                                     double* ioval, double* __restrict__ iovnext, int shift) {
  using R = typename Real<S>::type;
  __shared__ double sh[BLOCK / 32];
  const int k = blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (!((p.coupled[k >> 6] >> (k & 63)) & 1ull)) return;  // uniform per block
  if (!AA && shift) {
    if (threadIdx.x == 0) ioval[k] = iovnext[k];
    __syncthreads();  // io_val(p, k) below reads it (p.ioval == ioval)
  }
  const int64_t n = p.n;
  double acc = 0;
  for (int64_t r = begin[k] + threadIdx.x; r < begin[k + 1]; r += BLOCK) {
    if (AA) {
      acc += lflux[r];
    } else {
      const LinkRec L = links[r];
      const int64_t x = L.site;
      R own[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) own[i] = ldpop(fin + (int64_t)i * n + x);
      const Macro<R> ms = moments<R>(own);
      const int j = L.dir;
      R out = R(0), val = R(0);
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (i == opp(j)) out = own[i];
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (i == j) val = iolet_value<R>(i, L, out, ms.rho, ms.ux, ms.uy, ms.uz, amp, p);
      acc += (double)val - (double)out;
    }
  }
  const double flux = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double Rp = par[4 * k], C = par[4 * k + 1], Rd = par[4 * k + 2], rho_d = par[4 * k + 3];
    const double q = -flux;
    double rho_c = state[2 * k], ghost;
    if (C > 0) {
      rho_c += (q - (rho_c - rho_d) / Rd) / C;
      ghost = rho_c + Rp * q;
    } else {
      ghost = rho_d + (Rp + Rd) * q;
    }
    state[2 * k] = rho_c;
    state[2 * k + 1] = q;
    (AA ? ioval : iovnext)[k] = ghost - 1.0;
  }
}

// Windkessel outlets at initialisation: no outflow history.
__global__ void k_wk_reset(int32_t n_iolets, const StepParams p, const double* __restrict__ par,
                           double* __restrict__ state, double* __restrict__ ioval, double* __restrict__ iovnext) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_iolets || !((p.coupled[k >> 6] >> (k & 63)) & 1ull)) return;
  const double C = par[4 * k + 1], rho_d = par[4 * k + 3];
  if (!(C > 0)) state[2 * k] = rho_d;
  state[2 * k + 1] = 0.0;
  ioval[k] = iovnext[k] = state[2 * k] - 1.0;
}

template <typename S>
struct WkOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, int64_t tb, bool shift, cudaStream_t s) {
    StepParams p = h->params(tb);
    const int64_t nb = grid_for(h->n);
    const int64_t* begin = (const int64_t*)(h->d_red + nb);  // link ranges stored after the reduction partials
    if (h->scheme == HLB_AA)
      return launch_pdl(k_wk_update<S, true>, (unsigned)h->n_iolets, BLOCK, s, (const S*)nullptr, h->d_links,
                        h->d_amp, p, begin, h->d_lflux, h->d_wkpar, h->d_wkstate, h->d_ioval, h->d_iovnext, 0);
    return launch_pdl(k_wk_update<S, false>, (unsigned)h->n_iolets, BLOCK, s, (const S*)fin, h->d_links, h->d_amp,
                      p, begin, (const double*)nullptr, h->d_wkpar, h->d_wkstate, h->d_ioval, h->d_iovnext,
                      shift ? 1 : 0);
  }
};

template <typename S>
struct MonitorOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, int mode, int64_t tb, double* out, cudaStream_t s) {
    if (h->n_iolets == 0) return cudaSuccess;
    StepParams p = h->params(tb);
    HLB_MODE_SWITCH(mode, (k_iolet_monitor<S, M><<<h->n_iolets, 256, 0, s>>>(
                              (const S*)fin, h->d_src, h->d_links, h->d_amp, p, h->d_ioff, h->d_ilist, out)));
    return cudaGetLastError();
  }
};

template <typename S>
struct StateOp {
  static cudaError_t run(const hlb_solver* h, const void* fin, int mode, int64_t tb, void* out, int row,
                         cudaStream_t s) {
    StepParams p = h->params(tb);
    HLB_MODE_SWITCH(mode, (k_state<S, M><<<grid_for(h->n), BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links,
                                                                            h->d_amp, p, (S*)out, row)));
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
  static cudaError_t run(const hlb_solver* h, const void* fin, int mode, int64_t tb, bool have_flux, double* out,
                         cudaStream_t s) {
    StepParams p = h->params(tb);
    const int64_t nb = grid_for(h->n);
    const int64_t lo = h->owned_lo, hi = h->owned_hi, nbo = grid_for(hi - lo);
    double* part = h->d_red;
    HLB_MODE_SWITCH(mode, (k_mass<S, M><<<(unsigned)nbo, BLOCK, 0, s>>>((const S*)fin, h->d_src, h->d_links,
                                                                          h->d_amp, p, lo, hi, part)));
    k_finish<<<1, 1024, 0, s>>>(part, nbo, hi - lo, out);
    if (h->n_iolets > 0) {
      const int64_t* begin = (const int64_t*)(h->d_red + nb);  // link ranges stored after the partials
      if (!have_flux)
        k_zero<<<1, 256, 0, s>>>(out + 1, h->n_iolets);
      else if (h->scheme == HLB_AA)
        k_flux_sum<<<(unsigned)h->n_iolets, BLOCK, 0, s>>>(h->d_lflux, begin, out);
      else
        k_flux<S><<<(unsigned)h->n_iolets, BLOCK, 0, s>>>((const S*)fin, h->d_links, h->d_amp, p, begin, out);
    }
    return cudaGetLastError();
  }
};

}  // namespace

int64_t hlb_reduce_partials(int64_t n) { return (int64_t)grid_for(n); }

int64_t hlb_reduce_slots(int64_t n, int32_t n_iolets) {
  // per-block partials, iolet link ranges (int64, n_iolets + 1), final outputs (1 + n_iolets)
  return (int64_t)grid_for(n) + (n_iolets + 1) + (1 + n_iolets);
}

cudaError_t hlb_launch_step(const hlb_solver* h, const void* fin, void* fout, bool gather, int64_t tb,
                            cudaStream_t s) {
  return dispatch<StepOp>(h->precision, h, fin, fout, gather, tb, s);
}
cudaError_t hlb_launch_step_range(const hlb_solver* h, const void* fin, void* fout, int64_t tb, int64_t tile0,
                                  int64_t ntiles, bool iolets, cudaStream_t s) {
  return dispatch<StepRangeOp>(h->precision, h, fin, fout, tb, tile0, ntiles, iolets, s);
}
cudaError_t hlb_launch_aa(const hlb_solver* h, void* A, bool odd, int64_t t, cudaStream_t s) {
  return dispatch<AAOp>(h->precision, h, A, odd, t, s);
}
cudaError_t hlb_launch_macros(const hlb_solver* h, const void* fin, int mode, int64_t tb, float* rho, float* u,
                              float* wss, cudaStream_t s) {
  return dispatch<MacroOp>(h->precision, h, fin, mode, tb, rho, u, wss, s);
}
cudaError_t hlb_launch_wk_update(const hlb_solver* h, const void* fin, int64_t tb, bool shift, cudaStream_t s) {
  return dispatch<WkOp>(h->precision, h, fin, tb, shift, s);
}
cudaError_t hlb_launch_wk_reset(const hlb_solver* h, cudaStream_t s) {
  StepParams p = h->params(h->t);
  k_wk_reset<<<(unsigned)((h->n_iolets + 127) / 128), 128, 0, s>>>(h->n_iolets, p, h->d_wkpar, h->d_wkstate,
                                                                   h->d_ioval, h->d_iovnext);
  return cudaGetLastError();
}
cudaError_t hlb_launch_monitor(const hlb_solver* h, const void* fin, int mode, int64_t tb, double* out,
                               cudaStream_t s) {
  return dispatch<MonitorOp>(h->precision, h, fin, mode, tb, out, s);
}
cudaError_t hlb_launch_state(const hlb_solver* h, const void* fin, int mode, int64_t tb, void* out, int row,
                             cudaStream_t s) {
  return dispatch<StateOp>(h->precision, h, fin, mode, tb, out, row, s);
}
cudaError_t hlb_launch_ctab(const hlb_solver* h, int32_t* misfit, cudaStream_t s) {
  const int64_t tiles = (h->sn + CT_TILE - 1) / CT_TILE;
  k_ctab_build<<<(unsigned)tiles, CT_TILE, 0, s>>>(h->d_src, h->n, h->sn, h->d_ctab, h->d_tbase, misfit);
  return cudaGetLastError();
}
cudaError_t hlb_launch_init(const hlb_solver* h, void* f, double rho0, const float* u0, cudaStream_t s) {
  return dispatch<InitOp>(h->precision, h, f, rho0, u0, s);
}
cudaError_t hlb_launch_reduce(const hlb_solver* h, const void* fin, int mode, int64_t tb, bool have_flux,
                              double* out_dev, cudaStream_t s) {
  return dispatch<ReduceOp>(h->precision, h, fin, mode, tb, have_flux, out_dev, s);
}
