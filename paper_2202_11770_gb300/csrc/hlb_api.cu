// hlb_api.cu — C ABI of libhemegb: validation, workspace layout, set-up of
// the device tables (the GPU initialisation of arXiv 2202.11770,
// Section 3.2.1), time bookkeeping and readback.  All compute runs in the
// kernels of hlb_forward.cu / hlb_adjoint.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "hlb_internal.h"

using namespace hlb;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

int hlb_fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int hlb_cuda_fail(cudaError_t e, const char* where) {
  return hlb_fail(HLB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CUDA_TRY(expr)                                     \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return hlb_cuda_fail(_e, #expr); \
  } while (0)

extern "C" const char* hlb_last_error(void) { return g_err.c_str(); }

extern "C" int hlb_version(void) { return 10200; }

// ---------------------------------------------------------------------------
// waveforms
// ---------------------------------------------------------------------------
double HostWave::at(double t) const {
  if (kind == HLB_WAVE_CONST) return mean;
  if (kind == HLB_WAVE_COSINE) return mean * (1.0 + rel * cos(2.0 * M_PI * t / period + phase));
  double x = fmod(t, period);
  if (x < 0) x += period;
  const int ns = (int)samples.size();
  double pos = x / period * ns;
  int j = (int)floor(pos);
  double fr = pos - j;
  j %= ns;
  return mean * ((1.0 - fr) * samples[j] + fr * samples[(j + 1) % ns]);
}

static int parse_wave(const hlb_waveform* w, HostWave* out) {
  if (!w) return hlb_fail(HLB_ERR_ARG, "null waveform");
  HostWave hw;
  hw.kind = w->kind;
  hw.mean = w->mean;
  hw.rel = w->rel_amp;
  hw.period = w->period;
  hw.phase = w->phase;
  if (w->kind != HLB_WAVE_CONST && w->kind != HLB_WAVE_COSINE && w->kind != HLB_WAVE_TABLE)
    return hlb_fail(HLB_ERR_ARG, "unknown waveform kind");
  if (w->kind != HLB_WAVE_CONST && !(w->period > 0)) return hlb_fail(HLB_ERR_ARG, "waveform period must be > 0");
  if (w->kind == HLB_WAVE_TABLE) {
    if (w->n_samples < 1 || !w->samples) return hlb_fail(HLB_ERR_ARG, "table waveform needs samples");
    hw.samples.assign(w->samples, w->samples + w->n_samples);
  }
  if (!std::isfinite(hw.mean)) return hlb_fail(HLB_ERR_ARG, "non-finite waveform mean");
  *out = hw;
  return HLB_OK;
}

// ---------------------------------------------------------------------------
// solver helpers
// ---------------------------------------------------------------------------
size_t hlb_solver::elem_bytes() const {
  switch (precision) {
    case HLB_FP32: return 4;
    case HLB_BF16: return 2;
    case HLB_FP16: return 2;
    default: return 8;
  }
}

StepParams hlb_solver::params(int64_t tb) const {
  StepParams p;
  memset(&p, 0, sizeof p);
  p.n = n;
  p.sn = sn;
  p.omega = 1.0 / tau;
  p.omegaf = (float)p.omega;
  p.n_iolets = n_iolets;
  p.ladd_rho_one = ladd_rho_one;
  p.ghost_full_u = ghost_full_u;
  p.ioval = d_ioval;
  for (int k = 0; k < n_iolets; ++k)
    if (k < (int)wk_on.size() && wk_on[k]) p.coupled[k >> 6] |= 1ull << (k & 63);
  p.ampf = d_ampf;
  for (int k = 0; k < n_iolets; ++k) {
    p.io[k].nx = iolets[k].normal[0];
    p.io[k].ny = iolets[k].normal[1];
    p.io[k].nz = iolets[k].normal[2];
    double w = wave[k].at((double)tb);
    p.io[k].val = iolets[k].kind == HLB_VELOCITY ? w : w - 1.0;
    p.io[k].nxf = (float)p.io[k].nx;
    p.io[k].nyf = (float)p.io[k].ny;
    p.io[k].nzf = (float)p.io[k].nz;
    p.io[k].valf = (float)p.io[k].val;
  }
  return p;
}

// ---------------------------------------------------------------------------
// lattice validation and workspace layout
// ---------------------------------------------------------------------------
namespace {

struct Layout {
  size_t f0 = 0, f1 = 0, src = 0, ctab = 0, tbase = 0, ctflag = 0, links = 0, amp = 0, ampf = 0, normal = 0, stage = 0, red = 0, lflux = 0, isites = 0, icode = 0, imask = 0, ioff = 0,
         ilist = 0, mon = 0, wkpar = 0, wkstate = 0,
         ioval = 0, iovnext = 0, total = 0;
  int64_t n_links = 0;
  int32_t n_groups = 0;
};

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }
// Index rows are padded to a multiple of 4 entries, so every row starts on
// a 16-byte boundary.
int64_t row_stride(int64_t n) { return (n + 3) & ~(int64_t)3; }

// An iolet link of the caller's table: site x, pull direction dir.
struct LinkRef {
  int32_t x;
  int32_t dir;
};

// Checks of one direction row, run on its own thread: the first error in
// site order, per-iolet link counts and the row's iolet links.
struct RowCheck {
  int code = HLB_OK;
  const char* msg = nullptr;
  std::vector<int64_t> per;
  std::vector<LinkRef> links;
};

void check_row(const hlb_lattice* L, int i, RowCheck* out) {
  const int64_t n = L->n_sites;
  const int32_t* row = L->src + (int64_t)(i - 1) * n;
  out->per.assign((size_t)std::max(1, (int)L->n_iolets), 0);
  for (int64_t x = 0; x < n; ++x) {
    const int32_t s = row[x];
    if (s >= 0) {
      if (s >= n) { out->code = HLB_ERR_ARG; out->msg = "src index out of range"; return; }
    } else if (s <= -2) {
      const int k = -s - 2;
      if (k >= L->n_iolets) { out->code = HLB_ERR_ARG; out->msg = "link code names a missing iolet"; return; }
      if (L->iolets[k].kind == HLB_VELOCITY && L->amp_group) {
        const int g = L->amp_group[x];
        if (g < 0 || g >= L->iolets[k].n_groups) { out->code = HLB_ERR_ARG; out->msg = "amplitude group out of range"; return; }
      }
      out->per[(size_t)k]++;
      out->links.push_back({(int32_t)x, i});
    }
  }
}

int validate(const hlb_lattice* L, const hlb_options* o, std::vector<int64_t>* per_iolet_links,
             int64_t* n_iolet_sites, std::vector<LinkRef>* links_out = nullptr) {
  if (!L || !o) return hlb_fail(HLB_ERR_ARG, "null lattice or options");
  if (L->n_sites < 1 || L->n_sites >= ((int64_t)1 << 31)) return hlb_fail(HLB_ERR_ARG, "n_sites must be in [1, 2^31)");
  if (!L->src || !L->xyz) return hlb_fail(HLB_ERR_ARG, "lattice needs xyz and src");
  if (L->n_iolets < 0 || L->n_iolets > HLB_MAX_IOLETS) return hlb_fail(HLB_ERR_ARG, "n_iolets out of range");
  if (L->n_iolets > 0 && !L->iolets) return hlb_fail(HLB_ERR_ARG, "null iolet array");
  if (o->precision < HLB_FP32 || o->precision > HLB_FP64) return hlb_fail(HLB_ERR_ARG, "unknown precision");
  if (o->scheme != HLB_SCHEME_AUTO && o->scheme != HLB_PULL_AB && o->scheme != HLB_AA)
    return hlb_fail(HLB_ERR_ARG, "unknown scheme");
  for (int k = 0; k < L->n_iolets; ++k) {
    const hlb_iolet& io = L->iolets[k];
    if (io.kind != HLB_VELOCITY && io.kind != HLB_PRESSURE) return hlb_fail(HLB_ERR_ARG, "bad iolet kind");
    double nn = io.normal[0] * io.normal[0] + io.normal[1] * io.normal[1] + io.normal[2] * io.normal[2];
    if (!(fabs(nn - 1.0) < 1e-6)) return hlb_fail(HLB_ERR_ARG, "iolet normal must be a unit vector");
    if (!(io.radius > 0)) return hlb_fail(HLB_ERR_ARG, "iolet radius must be > 0");
    if (io.n_groups < 1) return hlb_fail(HLB_ERR_ARG, "iolet n_groups must be >= 1");
  }
  const int64_t n = L->n_sites;
  // the 18 rows in parallel (one thread each); errors and links merged in row order
  std::vector<RowCheck> rows(Q - 1);
  {
    std::vector<std::thread> pool;
    pool.reserve(Q - 1);
    for (int i = 1; i < Q; ++i) pool.emplace_back(check_row, L, i, &rows[(size_t)(i - 1)]);
    for (auto& t : pool) t.join();
  }
  per_iolet_links->assign((size_t)std::max(1, (int)L->n_iolets), 0);
  for (const RowCheck& r : rows)
    if (r.code != HLB_OK) return hlb_fail(r.code, r.msg);
  std::vector<uint8_t> iolet_site((size_t)n, 0);
  *n_iolet_sites = 0;
  for (const RowCheck& r : rows) {
    for (size_t k = 0; k < r.per.size(); ++k) (*per_iolet_links)[k] += r.per[k];
    for (const LinkRef& l : r.links)
      if (!iolet_site[(size_t)l.x]) {
        iolet_site[(size_t)l.x] = 1;
        ++*n_iolet_sites;
      }
    if (links_out) links_out->insert(links_out->end(), r.links.begin(), r.links.end());
  }
  return HLB_OK;
}

// AUTO resolves to the scheme measured faster on GB300 for the lattice size.
// The AA pattern moves 170 B per FP32 site update against 188 B for pull
// A-B (compact index table), but needs a second launch per step for its
// iolet-site pass.  Measured per step (seeded vessel trees, FP32 / BF16):
// 0.5M sites A-B 13.4 / 12.0 us, AA 14.8 / 12.6 us (the state fits in L2);
// 1.0M sites A-B 32.4 / 23.8 us, AA 29.8 / 19.9 us; 2.0M 67.7 / 49.4 against
// 61.7 / 42.3 us; 8.0M 256 / 188 against 229 / 145 us.  AA from 750k sites.
constexpr int64_t AA_MIN_SITES = 750000;
int32_t resolve_scheme(int32_t scheme, int64_t n) {
  if (scheme != HLB_SCHEME_AUTO) return scheme;
  return n >= AA_MIN_SITES ? HLB_AA : HLB_PULL_AB;
}

Layout layout(const hlb_lattice* L, const hlb_options* o, const std::vector<int64_t>& per_iolet,
              int64_t n_iolet_sites) {
  Layout y;
  const int64_t n = L->n_sites;
  size_t eb = o->precision == HLB_FP64 ? 8 : (o->precision == HLB_FP32 ? 4 : 2);
  size_t state = align_up(eb * 19 * (size_t)n);
  for (int k = 0; k < L->n_iolets; ++k) y.n_links += per_iolet[k];
  for (int k = 0; k < L->n_iolets; ++k)
    if (L->iolets[k].kind == HLB_VELOCITY) y.n_groups += L->iolets[k].n_groups;
  size_t off = 0;
  y.f0 = off; off += state;
  y.f1 = off; off += resolve_scheme(o->scheme, n) == HLB_AA ? 0 : state;
  y.src = off; off += align_up(sizeof(int32_t) * 18 * (size_t)row_stride(n));
  y.ctab = off; off += align_up(sizeof(uint32_t) * 9 * (size_t)row_stride(n));
  y.tbase = off; off += align_up(sizeof(int32_t) * hlb::CT_BASES * (size_t)((n + hlb::CT_TILE - 1) / hlb::CT_TILE));
  y.ctflag = off; off += align_up(sizeof(int32_t));
  y.links = off; off += align_up(sizeof(LinkRec) * (size_t)std::max<int64_t>(y.n_links, 1));
  y.amp = off; off += align_up(sizeof(double) * (size_t)std::max(y.n_groups, 1));
  y.ampf = off; off += align_up(sizeof(float) * (size_t)std::max(y.n_groups, 1));
  y.normal = off; off += L->wall_normal ? align_up(sizeof(float) * 3 * (size_t)n) : 0;
  y.stage = off; off += align_up(sizeof(float) * 5 * (size_t)n);
  y.red = off; off += align_up(sizeof(double) * (size_t)hlb_reduce_slots(n, L->n_iolets));
  y.lflux = off; off += align_up(sizeof(double) * (size_t)std::max<int64_t>(y.n_links, 1));
  y.isites = off; off += align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(n_iolet_sites, 1));
  y.icode = off; off += align_up(sizeof(int32_t) * 18 * (size_t)std::max<int64_t>(n_iolet_sites, 1));
  y.imask = off; off += align_up(sizeof(uint32_t) * (size_t)((n + 31) / 32));
  y.ioff = off; off += align_up(sizeof(int64_t) * (size_t)(L->n_iolets + 1));
  y.ilist = off; off += align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(y.n_links, 1));  // >= sites per iolet
  y.mon = off; off += align_up(sizeof(double) * 2 * (size_t)std::max(L->n_iolets, 1));
  y.wkpar = off; off += align_up(sizeof(double) * 4 * (size_t)std::max(L->n_iolets, 1));
  y.wkstate = off; off += align_up(sizeof(double) * 2 * (size_t)std::max(L->n_iolets, 1));
  y.ioval = off; off += align_up(sizeof(double) * (size_t)std::max(L->n_iolets, 1));
  y.iovnext = off; off += align_up(sizeof(double) * (size_t)std::max(L->n_iolets, 1));
  y.total = off;
  return y;
}

}  // namespace

static int workspace_bytes_impl(const hlb_lattice* L, const hlb_options* o, size_t* bytes) {
  if (!bytes) return hlb_fail(HLB_ERR_ARG, "null output");
  std::vector<int64_t> per;
  int64_t nis = 0;
  int rc = validate(L, o, &per, &nis);
  if (rc) return rc;
  *bytes = layout(L, o, per, nis).total;
  return HLB_OK;
}

extern "C" int hlb_workspace_bytes(const hlb_lattice* L, const hlb_options* o, size_t* bytes) {
  return hlb_no_throw([&] { return workspace_bytes_impl(L, o, bytes); });
}

namespace {

// Iolet links re-coded to their records at create: record r (site x,
// direction j) gets the code -(2 + r) in row j - 1.
__global__ void k_recode(int32_t* __restrict__ src, int64_t sn, const LinkRec* __restrict__ links, int64_t nlinks) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nlinks) return;
  const LinkRec L = links[r];
  src[(int64_t)(L.dir - 1) * sn + L.site] = -(int32_t)(2 + r);
}

// The 18 codes of each iolet site, contiguous: icode[q][i - 1].
__global__ void k_icode(const int32_t* __restrict__ src, int64_t sn, const int32_t* __restrict__ sites, int64_t nsites,
                        int32_t* __restrict__ icode) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsites * (Q - 1)) return;
  const int64_t q = k / (Q - 1);
  const int i = (int)(k - q * (Q - 1));
  icode[k] = src[(int64_t)i * sn + sites[q]];
}

}  // namespace

cudaError_t hlb_launch_recode(const hlb_solver* h, cudaStream_t s) {
  k_recode<<<(unsigned)((h->n_links + 255) / 256), 256, 0, s>>>(h->d_src, h->sn, h->d_links, h->n_links);
  return cudaGetLastError();
}
cudaError_t hlb_launch_icode(const hlb_solver* h, cudaStream_t s) {
  const int64_t k = h->n_iolet_sites * (Q - 1);
  k_icode<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(h->d_src, h->sn, h->d_iolet_sites, h->n_iolet_sites, h->d_icode);
  return cudaGetLastError();
}
static int create_impl(const hlb_lattice* L, const hlb_options* o, void* ws, size_t ws_bytes, hlb_stream stream,
                       hlb_solver** out, std::unique_ptr<hlb_solver>* owner) {
  if (!out) return hlb_fail(HLB_ERR_ARG, "null output");
  *out = nullptr;
  std::vector<int64_t> per;
  int64_t nis = 0;
  std::vector<LinkRef> links;
  int rc = validate(L, o, &per, &nis, &links);
  if (rc) return rc;
  Layout y = layout(L, o, per, nis);
  if (!ws) return hlb_fail(HLB_ERR_WS, "null workspace");
  if (((uintptr_t)ws & 255) != 0) return hlb_fail(HLB_ERR_WS, "workspace must be 256-byte aligned");
  if (ws_bytes < y.total)
    return hlb_fail(HLB_ERR_WS, "workspace too small: need " + std::to_string(y.total) + " bytes");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ws) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return hlb_fail(HLB_ERR_WS, "workspace is not device memory");
  }

  owner->reset(new hlb_solver());
  hlb_solver* h = owner->get();
  const int64_t n = L->n_sites;
  h->n = n;
  h->sn = row_stride(n);
  h->owned_lo = 0;
  h->owned_hi = n;
  h->n_iolets = L->n_iolets;
  h->iolets.assign(L->iolets, L->iolets + L->n_iolets);
  h->precision = o->precision;
  h->scheme = resolve_scheme(o->scheme, n);
  h->ladd_rho_one = o->ladd_rho_one ? 1 : 0;
  h->ghost_full_u = o->ghost_full_u ? 1 : 0;
  h->off32 = !o->wide_offsets && (uint64_t)Q * (uint64_t)h->sn <= 0xffffffffull;
  h->stream = (cudaStream_t)stream;
  h->device = attr.device;
  if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, attr.device) != cudaSuccess) {
    cudaGetLastError();
    h->n_sm = 0;  // no prefetch distance: the kernels skip the prefetch
  }
  h->has_normals = L->wall_normal != nullptr;
  h->wave.resize(h->n_iolets);
  h->group_offset.assign(h->n_iolets, -1);
  int32_t g = 0;
  for (int k = 0; k < h->n_iolets; ++k) {
    if (h->iolets[k].kind == HLB_VELOCITY) {
      h->group_offset[k] = g;
      g += h->iolets[k].n_groups;
      h->wave[k].mean = 0.0;
    } else {
      h->wave[k].mean = 1.0;
    }
  }
  h->n_groups_total = g;
  h->amp.assign(g, 0.0);

  char* base = (char*)ws;
  h->f[0] = base + y.f0;
  h->f[1] = h->scheme == HLB_AA ? nullptr : base + y.f1;
  h->d_src = (int32_t*)(base + y.src);
  h->d_ctab = (uint32_t*)(base + y.ctab);
  h->d_tbase = (int32_t*)(base + y.tbase);
  int32_t* d_misfit = (int32_t*)(base + y.ctflag);
  h->d_links = (LinkRec*)(base + y.links);
  h->d_amp = (double*)(base + y.amp);
  h->d_ampf = (float*)(base + y.ampf);
  h->d_normal = L->wall_normal ? (float*)(base + y.normal) : nullptr;
  h->d_stage = (float*)(base + y.stage);
  h->d_red = (double*)(base + y.red);
  h->red_slots = hlb_reduce_slots(n, h->n_iolets);
  h->d_lflux = (double*)(base + y.lflux);
  h->d_iolet_sites = (int32_t*)(base + y.isites);
  h->d_icode = (int32_t*)(base + y.icode);
  h->d_imask = (uint32_t*)(base + y.imask);
  h->d_ioff = (int64_t*)(base + y.ioff);
  h->d_ilist = (int32_t*)(base + y.ilist);
  h->d_mon = (double*)(base + y.mon);
  h->d_wkpar = (double*)(base + y.wkpar);
  h->d_wkstate = (double*)(base + y.wkstate);
  h->d_ioval = (double*)(base + y.ioval);
  h->d_iovnext = (double*)(base + y.iovnext);
  h->wk_on.assign((size_t)h->n_iolets, 0);
  h->n_iolet_sites = nis;

  // link records sorted by (iolet, group, site, direction), from the links
  // validate() collected (no further pass over the table)
  std::vector<int64_t> bucket_base(h->n_iolets + 1, 0);
  for (int k = 0; k < h->n_iolets; ++k)
    bucket_base[k + 1] = bucket_base[k] + (h->iolets[k].kind == HLB_VELOCITY ? h->iolets[k].n_groups : 1);
  auto group_of = [&](int k, int64_t x) -> int {
    return (h->iolets[k].kind == HLB_VELOCITY && L->amp_group) ? L->amp_group[x] : 0;
  };
  auto code_of = [&](const LinkRef& l) { return L->src[(int64_t)(l.dir - 1) * n + l.x]; };
  auto bucket_of = [&](const LinkRef& l) {
    const int k = -code_of(l) - 2;
    return bucket_base[k] + group_of(k, l.x);
  };
  std::sort(links.begin(), links.end(), [&](const LinkRef& a, const LinkRef& b) {
    const int64_t ba = bucket_of(a), bb = bucket_of(b);
    if (ba != bb) return ba < bb;
    if (a.x != b.x) return a.x < b.x;
    return a.dir < b.dir;
  });
  std::vector<int64_t> count(bucket_base[h->n_iolets] + 1, 0);
  for (const LinkRef& l : links) count[bucket_of(l) + 1]++;
  for (size_t b = 1; b < count.size(); ++b) count[b] += count[b - 1];
  h->n_links = y.n_links;
  h->link_begin.resize(h->n_iolets + 1);
  for (int k = 0; k <= h->n_iolets; ++k) h->link_begin[k] = count[bucket_base[k]];
  h->group_link_begin.assign(g + 1, 0);
  for (int k = 0; k < h->n_iolets; ++k) {
    if (h->iolets[k].kind != HLB_VELOCITY) continue;
    for (int gl = 0; gl < h->iolets[k].n_groups; ++gl) {
      h->group_link_begin[h->group_offset[k] + gl] = count[bucket_base[k] + gl];
      h->group_link_begin[h->group_offset[k] + gl + 1] = count[bucket_base[k] + gl + 1];
    }
  }
  std::vector<LinkRec> recs((size_t)std::max<int64_t>(y.n_links, 1));
  const int64_t sn = h->sn;
  for (int64_t r = 0; r < (int64_t)links.size(); ++r) {
    const int64_t x = links[(size_t)r].x;
    const int j = links[(size_t)r].dir;
    {
      const int k = -code_of(links[(size_t)r]) - 2;
      const hlb_iolet& io = h->iolets[k];
      const int gl = group_of(k, x);
      LinkRec& R = recs[(size_t)r];
      R.site = (int32_t)x;
      R.dir = (int8_t)j;
      R.kind = (int8_t)io.kind;
      R.iolet = (int16_t)k;
      R.group = io.kind == HLB_VELOCITY ? h->group_offset[k] + gl : -1;
      R.coef = 0.0;
      if (io.kind == HLB_VELOCITY) {
        // Ladd weight at the link midpoint x - c_j / 2
        double m[3] = {L->xyz[3 * x] - 0.5 * cx(j), L->xyz[3 * x + 1] - 0.5 * cy(j), L->xyz[3 * x + 2] - 0.5 * cz(j)};
        double v[3] = {m[0] - io.centre[0], m[1] - io.centre[1], m[2] - io.centre[2]};
        double an = v[0] * io.normal[0] + v[1] * io.normal[1] + v[2] * io.normal[2];  // axial coordinate
        double r2 = 0;
        for (int a = 0; a < 3; ++a) {
          double w = v[a] - an * io.normal[a];
          r2 += w * w;
        }
        double W = std::max(0.0, 1.0 - r2 / (io.radius * io.radius));
        double cn = cx(j) * io.normal[0] + cy(j) * io.normal[1] + cz(j) * io.normal[2];
        // f_j(x) = f'_jbar(x) - 2 w rho (c_jbar . u_w) / cs2 = f'_jbar(x) + 6 w_j rho A W (c_j . n)
        R.coef = 6.0 * wgt<double>(j) * W * cn;
      }
      R.coef_f = (float)R.coef;
    }
  }

  cudaStream_t st = h->stream;
  int64_t nb = hlb_reduce_partials(n);
  std::vector<int64_t> begin(h->link_begin);
  std::vector<double> ampf(std::max(g, 1), 0.0);
  std::vector<int32_t> isites;
  isites.reserve(links.size());
  for (const LinkRef& l : links) isites.push_back(l.x);
  std::sort(isites.begin(), isites.end());
  isites.erase(std::unique(isites.begin(), isites.end()), isites.end());
  cudaError_t e = cudaSuccess;
  // the caller's rows straight into the padded device table (no host copy of
  // the table), padding entries (never gathered) -1, then the iolet links
  // re-coded to their records on the device
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(h->d_src, sizeof(int32_t) * (size_t)sn, L->src, sizeof(int32_t) * (size_t)n,
                          sizeof(int32_t) * (size_t)n, 18, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && sn > n)
    e = cudaMemset2DAsync(h->d_src + n, sizeof(int32_t) * (size_t)sn, 0xff, sizeof(int32_t) * (size_t)(sn - n), 18, st);
  if (e == cudaSuccess && y.n_links > 0)
    e = cudaMemcpyAsync(h->d_links, recs.data(), sizeof(LinkRec) * (size_t)y.n_links, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && y.n_links > 0) e = hlb_launch_recode(h, st);
  // compact index table from the re-coded one; the fit flag comes back with
  // the final synchronisation
  int32_t misfit = 1;
  if (e == cudaSuccess) e = cudaMemsetAsync(d_misfit, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = hlb_launch_ctab(h, d_misfit, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&misfit, d_misfit, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_amp, ampf.data(), sizeof(double) * ampf.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_ampf, 0, sizeof(float) * ampf.size(), st);
  if (e == cudaSuccess && h->d_normal)
    e = cudaMemcpyAsync(h->d_normal, L->wall_normal, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_red + nb, begin.data(), sizeof(int64_t) * begin.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nis > 0)
    e = cudaMemcpyAsync(h->d_iolet_sites, isites.data(), sizeof(int32_t) * (size_t)nis, cudaMemcpyHostToDevice, st);
  // index codes of the iolet sites (the library's own re-coded table), 18 per site
  if (e == cudaSuccess && nis > 0) e = hlb_launch_icode(h, st);
  // bit mask of the sites with an iolet link (bulk threads of k_step leave them to the iolet warps)
  std::vector<uint32_t> imask((size_t)((n + 31) / 32), 0u);
  for (int32_t x : isites) imask[(size_t)x >> 5] |= 1u << (x & 31);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_imask, imask.data(), sizeof(uint32_t) * imask.size(), cudaMemcpyHostToDevice, st);
  // sites of each iolet (a link to it), ascending, as ranges of one list
  std::vector<std::vector<int32_t>> per_io((size_t)h->n_iolets);
  for (int32_t x : isites) {
    for (int i = 1; i < Q; ++i) {
      const int32_t c = L->src[(int64_t)(i - 1) * n + x];
      if (c > -2) continue;
      const int k = -c - 2;
      bool seen = false;
      for (int j = 1; j < i && !seen; ++j) seen = L->src[(int64_t)(j - 1) * n + x] == c;
      if (!seen) per_io[(size_t)k].push_back(x);
    }
  }
  std::vector<int64_t> ioff((size_t)h->n_iolets + 1, 0);
  std::vector<int32_t> ilist;
  for (int k = 0; k < h->n_iolets; ++k) {
    ilist.insert(ilist.end(), per_io[(size_t)k].begin(), per_io[(size_t)k].end());
    ioff[(size_t)k + 1] = (int64_t)ilist.size();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_ioff, ioff.data(), sizeof(int64_t) * ioff.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !ilist.empty())
    e = cudaMemcpyAsync(h->d_ilist, ilist.data(), sizeof(int32_t) * ilist.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_lflux, 0, sizeof(double) * (size_t)std::max<int64_t>(y.n_links, 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, h->state_bytes(), st);  // rest: h = f - w = 0
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hlb_cuda_fail(e, "hlb_create upload");  // the owner frees h
  h->compact = !o->full_index && misfit == 0;
  h->cur = 0;
  h->phase = 0;
  h->t = 0;
  *out = owner->release();
  return HLB_OK;
}

extern "C" int hlb_create(const hlb_lattice* L, const hlb_options* o, void* ws, size_t ws_bytes, hlb_stream stream,
                          hlb_solver** out) {
  std::unique_ptr<hlb_solver> owner;
  return hlb_no_throw([&] { return create_impl(L, o, ws, ws_bytes, stream, out, &owner); });
}

extern "C" int hlb_destroy(hlb_solver* h) {
  delete h;
  return HLB_OK;
}

extern "C" int hlb_set_stream(hlb_solver* h, hlb_stream s) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  h->stream = (cudaStream_t)s;
  return HLB_OK;
}

extern "C" int64_t hlb_n_sites(const hlb_solver* h) { return h ? h->n : -1; }
extern "C" int hlb_compact_index(const hlb_solver* h) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  return h->compact ? 1 : 0;
}
extern "C" int hlb_n_amp_groups(const hlb_solver* h) { return h ? h->n_groups_total : -1; }

extern "C" int hlb_set_tau(hlb_solver* h, double tau) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (!(tau > 0.5) || !std::isfinite(tau)) return hlb_fail(HLB_ERR_ARG, "tau must be > 1/2");
  h->tau = tau;
  return HLB_OK;
}

static int hlb_set_velocity_waveform_impl(hlb_solver* h, int32_t k, const double* amp, int32_t n_groups,
                                         const hlb_waveform* w) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (k < 0 || k >= h->n_iolets || h->iolets[k].kind != HLB_VELOCITY)
    return hlb_fail(HLB_ERR_ARG, "not a velocity iolet");
  if (n_groups != h->iolets[k].n_groups || !amp) return hlb_fail(HLB_ERR_ARG, "amplitude count mismatch");
  HostWave hw;
  int rc = parse_wave(w, &hw);
  if (rc) return rc;
  for (int gi = 0; gi < n_groups; ++gi)
    if (!std::isfinite(amp[gi])) return hlb_fail(HLB_ERR_ARG, "non-finite amplitude");
  h->wave[k] = hw;
  std::vector<float> af((size_t)n_groups);
  for (int gi = 0; gi < n_groups; ++gi) {
    h->amp[h->group_offset[k] + gi] = amp[gi];
    af[(size_t)gi] = (float)amp[gi];
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_amp + h->group_offset[k], amp, sizeof(double) * n_groups,
                           cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_ampf + h->group_offset[k], af.data(), sizeof(float) * n_groups,
                           cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return HLB_OK;
}

extern "C" int hlb_set_velocity_waveform(hlb_solver* h, int32_t k, const double* amp, int32_t n_groups,
                                         const hlb_waveform* w) {
  return hlb_no_throw([&] { return hlb_set_velocity_waveform_impl(h, k, amp, n_groups, w); });
}

static int hlb_set_pressure_impl(hlb_solver* h, int32_t k, const hlb_waveform* w) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (k < 0 || k >= h->n_iolets || h->iolets[k].kind != HLB_PRESSURE)
    return hlb_fail(HLB_ERR_ARG, "not a pressure iolet");
  HostWave hw;
  int rc = parse_wave(w, &hw);
  if (rc) return rc;
  h->wave[k] = hw;
  h->wk_on[k] = 0;
  return HLB_OK;
}

extern "C" int hlb_set_pressure(hlb_solver* h, int32_t k, const hlb_waveform* w) {
  return hlb_no_throw([&] { return hlb_set_pressure_impl(h, k, w); });
}

extern "C" int hlb_set_windkessel(hlb_solver* h, int32_t k, double Rp, double C, double Rd, double rho_d,
                                  double rho_c0) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (k < 0 || k >= h->n_iolets || h->iolets[k].kind != HLB_PRESSURE)
    return hlb_fail(HLB_ERR_ARG, "not a pressure iolet");
  if (!(Rp >= 0) || !(C >= 0) || !(Rd >= 0) || (C > 0 && !(Rd * C >= 1)) || !(rho_d > 0) ||
      (C > 0 && !(rho_c0 > 0)))
    return hlb_fail(HLB_ERR_ARG, "Windkessel needs Rp, C, Rd >= 0, Rd C >= 1 when C > 0, positive densities");
  const double par[4] = {Rp, C, Rd, rho_d};
  const double rho_c = C > 0 ? rho_c0 : rho_d;
  const double state[2] = {rho_c, 0.0};
  const double val = rho_c - 1.0;  // ghost density before any outflow: rho_c + Rp * 0
  CUDA_TRY(cudaMemcpyAsync(h->d_wkpar + 4 * k, par, sizeof par, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_wkstate + 2 * k, state, sizeof state, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_ioval + k, &val, sizeof val, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_iovnext + k, &val, sizeof val, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->wk_on[k] = 1;
  return HLB_OK;
}

extern "C" int hlb_windkessel_state(hlb_solver* h, int32_t k, double* rho_ghost, double* rho_c, double* q) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (k < 0 || k >= h->n_iolets || !h->wk_on[k]) return hlb_fail(HLB_ERR_ARG, "not a Windkessel outlet");
  double state[2], val;
  CUDA_TRY(cudaMemcpyAsync(state, h->d_wkstate + 2 * k, sizeof state, cudaMemcpyDeviceToHost, h->stream));
  // the ghost density that produces the next state: AA has already applied
  // the current one, pull A-B applies it at the next gather
  const double* g = h->scheme == HLB_AA ? h->d_ioval : h->d_iovnext;
  CUDA_TRY(cudaMemcpyAsync(&val, g + k, sizeof val, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (rho_ghost) *rho_ghost = 1.0 + val;
  if (rho_c) *rho_c = state[0];
  if (q) *q = state[1];
  return HLB_OK;
}

extern "C" int hlb_init_equilibrium(hlb_solver* h, double rho0, const float* u0, int32_t where) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (!(rho0 > 0) || !std::isfinite(rho0)) return hlb_fail(HLB_ERR_ARG, "rho0 must be positive");
  const float* du = u0;
  if (u0 && where == HLB_HOST) {
    CUDA_TRY(cudaMemcpyAsync(h->d_stage, u0, sizeof(float) * 3 * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
    du = h->d_stage;
  }
  CUDA_TRY(hlb_launch_init(h, h->f[0], rho0, du, h->stream));
  if (h->any_wk()) CUDA_TRY(hlb_launch_wk_reset(h, h->stream));
  h->cur = 0;
  h->phase = HLB_READ_LOCAL;
  h->t = 0;
  h->stepped = false;
  if (u0 && where == HLB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream));
  return HLB_OK;
}

extern "C" int hlb_step(hlb_solver* h, int64_t nsteps) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (nsteps < 0) return hlb_fail(HLB_ERR_ARG, "negative step count");
  if (h->midstep) return hlb_fail(HLB_ERR_STATE, "a partial step (hlb_step_range) is not finished");
  for (int64_t s = 0; s < nsteps; ++s) {
    if (h->scheme == HLB_AA) {
      // even step from f(t) in place, odd step from the swapped buffer
      const bool odd = h->phase == HLB_READ_GATHER_AA;
      CUDA_TRY(hlb_launch_aa(h, h->f[0], odd, h->t, h->stream));
      if (h->any_wk()) CUDA_TRY(hlb_launch_wk_update(h, nullptr, h->t, false, h->stream));
      h->phase = odd ? HLB_READ_LOCAL : HLB_READ_GATHER_AA;
    } else {
      const bool gather = h->phase == HLB_READ_GATHER_AB;
      CUDA_TRY(hlb_launch_step(h, h->f[h->cur], h->f[h->cur ^ 1], gather, h->t - 1, h->stream));
      // outflow into f(t+1) = G(s'(t)): the new s'(t) with the ghost density the next gather uses
      if (h->any_wk()) CUDA_TRY(hlb_launch_wk_update(h, h->f[h->cur ^ 1], h->t, gather, h->stream));
      h->cur ^= 1;
      h->phase = HLB_READ_GATHER_AB;
    }
    h->t += 1;
    h->stepped = true;
  }
  return HLB_OK;
}

extern "C" int hlb_time(const hlb_solver* h, int64_t* t) {
  if (!h || !t) return hlb_fail(HLB_ERR_ARG, "null argument");
  *t = h->t;
  return HLB_OK;
}

extern "C" int hlb_read_macros(hlb_solver* h, float* rho, float* u, float* wss, int32_t where) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  const int64_t n = h->n;
  if (where == HLB_DEVICE) {
    CUDA_TRY(hlb_launch_macros(h, h->f[h->cur], h->phase, h->t - 1, rho, u, wss, h->stream));
    return HLB_OK;
  }
  float* sr = rho ? h->d_stage : nullptr;
  float* su = u ? h->d_stage + n : nullptr;
  float* sw = wss ? h->d_stage + 4 * n : nullptr;
  CUDA_TRY(hlb_launch_macros(h, h->f[h->cur], h->phase, h->t - 1, sr, su, sw, h->stream));
  if (rho) CUDA_TRY(cudaMemcpyAsync(rho, sr, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
  if (u) CUDA_TRY(cudaMemcpyAsync(u, su, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  if (wss) CUDA_TRY(cudaMemcpyAsync(wss, sw, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return HLB_OK;
}

static int hlb_reduce_impl(hlb_solver* h, double* mass, double* flux) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  const int64_t nb = hlb_reduce_partials(h->n);
  double* out = h->d_red + nb + (h->n_iolets + 1);
  CUDA_TRY(hlb_launch_reduce(h, h->f[h->cur], h->phase, h->t - 1, h->stepped, out, h->stream));
  std::vector<double> host(1 + h->n_iolets);
  CUDA_TRY(cudaMemcpyAsync(host.data(), out, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (mass) *mass = host[0];
  if (flux)
    for (int k = 0; k < h->n_iolets; ++k) flux[k] = host[1 + k];
  if (!std::isfinite(host[0])) return hlb_fail(HLB_ERR_DIVERGED, "mass is not finite");
  return HLB_OK;
}

extern "C" int hlb_reduce(hlb_solver* h, double* mass, double* flux) {
  return hlb_no_throw([&] { return hlb_reduce_impl(h, mass, flux); });
}

static int hlb_iolet_monitor_impl(hlb_solver* h, double* flux, double* u_max, double* rho_mean) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  const int K = h->n_iolets;
  if (K == 0) return HLB_OK;
  if (flux) {
    std::vector<double> fl((size_t)K);
    int rc = hlb_reduce(h, nullptr, fl.data());
    if (rc) return rc;
    for (int k = 0; k < K; ++k) flux[k] = fl[(size_t)k];
  }
  if (!u_max && !rho_mean) return HLB_OK;
  CUDA_TRY(hlb_launch_monitor(h, h->f[h->cur], h->phase, h->t - 1, h->d_mon, h->stream));
  std::vector<double> host(2 * (size_t)K);
  CUDA_TRY(cudaMemcpyAsync(host.data(), h->d_mon, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < K; ++k) {
    if (u_max) u_max[k] = host[(size_t)k];
    if (rho_mean) rho_mean[k] = host[(size_t)(K + k)];
  }
  return HLB_OK;
}

extern "C" int hlb_iolet_monitor(hlb_solver* h, double* flux, double* u_max, double* rho_mean) {
  return hlb_no_throw([&] { return hlb_iolet_monitor_impl(h, flux, u_max, rho_mean); });
}

extern "C" int hlb_get_state(hlb_solver* h, void* f, int32_t where, int64_t* t) {
  if (!h || !f) return hlb_fail(HLB_ERR_ARG, "null argument");
  const size_t bytes = h->state_bytes();
  if (h->phase == HLB_READ_LOCAL) {
    CUDA_TRY(cudaMemcpyAsync(f, h->f[h->cur], bytes, where == HLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             h->stream));
  } else if (where == HLB_DEVICE) {
    CUDA_TRY(hlb_launch_state(h, h->f[h->cur], h->phase, h->t - 1, f, -1, h->stream));
  } else if (h->scheme != HLB_AA) {
    // the spare population buffer is free until the next step
    void* spare = h->f[h->cur ^ 1];
    CUDA_TRY(hlb_launch_state(h, h->f[h->cur], h->phase, h->t - 1, spare, -1, h->stream));
    CUDA_TRY(cudaMemcpyAsync(f, spare, bytes, cudaMemcpyDeviceToHost, h->stream));
  } else {
    // one direction at a time through the read-back staging area
    const size_t row = h->elem_bytes() * (size_t)h->n;
    for (int i = 0; i < 19; ++i) {
      CUDA_TRY(hlb_launch_state(h, h->f[0], h->phase, h->t - 1, h->d_stage, i, h->stream));
      CUDA_TRY(cudaMemcpyAsync((char*)f + row * i, h->d_stage, row, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (t) *t = h->t;
  if (where == HLB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream));
  return HLB_OK;
}

extern "C" int hlb_set_state(hlb_solver* h, const void* f, int32_t where, int64_t t) {
  if (!h || !f) return hlb_fail(HLB_ERR_ARG, "null argument");
  if (t < 0) return hlb_fail(HLB_ERR_ARG, "negative time");
  CUDA_TRY(cudaMemcpyAsync(h->f[0], f, h->state_bytes(),
                           where == HLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
  if (where == HLB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->cur = 0;
  h->phase = HLB_READ_LOCAL;
  h->t = t;
  h->stepped = false;
  return HLB_OK;
}
