// hlb_partition.cu — slab decomposition of a sparse lattice, the halo lists
// between its parts, and the device pack / unpack of the halo populations
// (include/hlb_partition.h).
//
// The paper splits the lattice over MPI ranks and exchanges the populations
// that stream across domain edges every step (arXiv 2202.11770, Section 3.1;
// on the GPU, Section 3.2.2, GPU_StreamReceivedDistr scatters the received
// populations into the local arrays).  Here each part keeps ghost copies of
// the remote sites its owned sites pull from, so that a part is an ordinary
// lattice for hlb_create, and the exchange writes the owners' post-collision
// values into the ghosts' slots between steps.
#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "hlb_internal.h"
#include "hlb_partition.h"

using namespace hlb;

struct hlb_part {
  struct Local {
    std::vector<int64_t> global;   // local -> global site, ascending
    int64_t lo = 0, hi = 0;        // owned sites, local indexing
    std::vector<int32_t> xyz, src, group;
    std::vector<float> normal;
  };
  int32_t P = 0;
  int64_t n = 0;
  bool has_normal = false, has_group = false;
  std::vector<int64_t> bound;      // [P + 1] first global site of each part
  std::vector<Local> parts;
  std::vector<hlb_iolet> iolets;
  // [q * P + p]: halo slots (post-collision values p pulls from q) and ghost sites
  std::vector<std::vector<int64_t>> hsrc, hdst, gsrc, gdst;

  int32_t owner(int64_t g) const {
    return (int32_t)(std::upper_bound(bound.begin(), bound.end(), g) - bound.begin()) - 1;
  }
  static int64_t local_of(const Local& L, int64_t g) {
    const auto it = std::lower_bound(L.global.begin(), L.global.end(), g);
    return (it != L.global.end() && *it == g) ? (int64_t)(it - L.global.begin()) : -1;
  }
};

namespace {

int plan_impl(const hlb_lattice* L, int32_t P, hlb_part** out) {
  if (!out) return hlb_fail(HLB_ERR_ARG, "null output");
  *out = nullptr;
  if (!L || !L->src || !L->xyz) return hlb_fail(HLB_ERR_ARG, "lattice needs xyz and src");
  const int64_t n = L->n_sites;
  if (n < 1 || n >= ((int64_t)1 << 31)) return hlb_fail(HLB_ERR_ARG, "n_sites must be in [1, 2^31)");
  if (P < 1 || P > n) return hlb_fail(HLB_ERR_ARG, "n_parts must be in [1, n_sites]");
  if (L->n_iolets < 0 || L->n_iolets > HLB_MAX_IOLETS || (L->n_iolets > 0 && !L->iolets))
    return hlb_fail(HLB_ERR_ARG, "bad iolet list");
  for (int64_t k = 0; k < (int64_t)Q - 1; ++k)
    for (int64_t x = 0; x < n; ++x) {
      const int32_t s = L->src[k * n + x];
      if (s >= n || (s < -1 && -(int64_t)s - 2 >= L->n_iolets)) return hlb_fail(HLB_ERR_ARG, "src entry out of range");
    }
  std::unique_ptr<hlb_part> plan(new hlb_part());
  hlb_part& H = *plan;
  H.P = P;
  H.n = n;
  H.has_normal = L->wall_normal != nullptr;
  H.has_group = L->amp_group != nullptr;
  H.iolets.assign(L->iolets, L->iolets + L->n_iolets);
  H.bound.resize((size_t)P + 1);
  for (int32_t p = 0; p <= P; ++p) H.bound[(size_t)p] = (int64_t)((__int128)n * p / P);
  H.parts.resize((size_t)P);
  const int64_t* B = H.bound.data();
  auto S = [&](int i, int64_t g) { return L->src[(int64_t)(i - 1) * n + g]; };

  // local site lists: ghosts below the slab, the slab, ghosts above
  for (int32_t p = 0; p < P; ++p) {
    hlb_part::Local& T = H.parts[(size_t)p];
    std::vector<int64_t> ghosts;
    for (int64_t g = B[p]; g < B[p + 1]; ++g)
      for (int i = 1; i < Q; ++i) {
        const int32_t s = S(i, g);
        if (s >= 0 && (s < B[p] || s >= B[p + 1])) ghosts.push_back(s);
      }
    std::sort(ghosts.begin(), ghosts.end());
    ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
    const auto mid = std::lower_bound(ghosts.begin(), ghosts.end(), B[p]);
    T.global.assign(ghosts.begin(), mid);
    T.lo = (int64_t)T.global.size();
    for (int64_t g = B[p]; g < B[p + 1]; ++g) T.global.push_back(g);
    T.hi = (int64_t)T.global.size();
    T.global.insert(T.global.end(), mid, ghosts.end());
  }
  // local lattices
  for (int32_t p = 0; p < P; ++p) {
    hlb_part::Local& T = H.parts[(size_t)p];
    const int64_t m = (int64_t)T.global.size();
    T.xyz.resize((size_t)m * 3);
    T.src.resize((size_t)m * 18);
    if (H.has_group) T.group.resize((size_t)m);
    if (H.has_normal) T.normal.resize((size_t)m * 3);
    for (int64_t l = 0; l < m; ++l) {
      const int64_t g = T.global[(size_t)l];
      const bool owned = l >= T.lo && l < T.hi;
      for (int a = 0; a < 3; ++a) T.xyz[(size_t)(3 * l + a)] = L->xyz[3 * g + a];
      if (H.has_group) T.group[(size_t)l] = L->amp_group[g];
      if (H.has_normal)
        for (int a = 0; a < 3; ++a) T.normal[(size_t)(a * m + l)] = L->wall_normal[a * n + g];
      for (int i = 1; i < Q; ++i) {
        const int32_t s = S(i, g);
        int32_t v;
        if (s >= 0) {
          const int64_t ls = owned && s >= B[p] && s < B[p + 1] ? s - B[p] + T.lo : hlb_part::local_of(T, s);
          v = ls >= 0 ? (int32_t)ls : -1;  // a ghost's source outside the part: a wall (never read)
        } else {
          v = owned ? s : -1;              // a ghost carries no iolet link
        }
        T.src[(size_t)((i - 1) * m + l)] = v;
      }
    }
  }
  // halo lists: the post-collision populations s'_i(y) that p's owned sites pull from q's site y
  H.hsrc.assign((size_t)P * P, {});
  H.hdst.assign((size_t)P * P, {});
  H.gsrc.assign((size_t)P * P, {});
  H.gdst.assign((size_t)P * P, {});
  for (int32_t p = 0; p < P; ++p) {
    const hlb_part::Local& T = H.parts[(size_t)p];
    const int64_t m = (int64_t)T.global.size();
    for (int64_t g = B[p]; g < B[p + 1]; ++g)
      for (int i = 1; i < Q; ++i) {
        const int32_t s = S(i, g);
        if (s < 0 || (s >= B[p] && s < B[p + 1])) continue;
        const int32_t q = H.owner(s);
        const hlb_part::Local& U = H.parts[(size_t)q];
        const int64_t mq = (int64_t)U.global.size();
        H.hsrc[(size_t)q * P + p].push_back((int64_t)i * mq + (s - B[q] + U.lo));
        H.hdst[(size_t)q * P + p].push_back((int64_t)i * m + hlb_part::local_of(T, s));
      }
    for (int64_t l = 0; l < m; ++l) {
      if (l >= T.lo && l < T.hi) continue;
      const int64_t g = T.global[(size_t)l];
      const int32_t q = H.owner(g);
      H.gsrc[(size_t)q * P + p].push_back(g - B[q] + H.parts[(size_t)q].lo);
      H.gdst[(size_t)q * P + p].push_back(l);
    }
  }
  *out = plan.release();
  return HLB_OK;
}

constexpr int BLOCK = 256;

template <typename T>
__global__ void k_halo_pack(const T* __restrict__ f, const int64_t* __restrict__ slots, int64_t n, T* __restrict__ buf) {
  const int64_t k = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (k < n) buf[k] = f[slots[k]];
}
template <typename T>
__global__ void k_halo_unpack(T* __restrict__ f, const int64_t* __restrict__ slots, int64_t n, const T* __restrict__ buf) {
  const int64_t k = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (k < n) f[slots[k]] = buf[k];
}

template <typename T>
cudaError_t halo_copy(bool pack, void* f, const int64_t* slots, int64_t n, void* buf, cudaStream_t st) {
  const unsigned g = (unsigned)((n + BLOCK - 1) / BLOCK);
  if (pack)
    k_halo_pack<T><<<g, BLOCK, 0, st>>>((const T*)f, slots, n, (T*)buf);
  else
    k_halo_unpack<T><<<g, BLOCK, 0, st>>>((T*)f, slots, n, (const T*)buf);
  return cudaGetLastError();
}

int halo_impl(hlb_solver* h, const int64_t* slots, int64_t n, void* buf, bool pack) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  // pack / unpack address the post-collision state of the step in progress
  // (mid-step) or of the last step
  if (n < 0 || (n > 0 && (!slots || !buf))) return hlb_fail(HLB_ERR_ARG, "bad halo arrays");
  if (h->scheme != HLB_PULL_AB || h->phase != HLB_READ_GATHER_AB)
    return hlb_fail(HLB_ERR_STATE, "halo exchange needs a pull A-B solver after a step");
  if (n == 0) return HLB_OK;
  void* f = h->f[h->midstep ? h->cur ^ 1 : h->cur];  // mid-step: the state being written
  cudaError_t e;
  switch (h->elem_bytes()) {
    case 2: e = halo_copy<uint16_t>(pack, f, slots, n, buf, h->stream); break;
    case 4: e = halo_copy<uint32_t>(pack, f, slots, n, buf, h->stream); break;
    default: e = halo_copy<uint64_t>(pack, f, slots, n, buf, h->stream); break;
  }
  if (e != cudaSuccess) return hlb_cuda_fail(e, pack ? "hlb_halo_pack" : "hlb_halo_unpack");
  return HLB_OK;
}

}  // namespace

extern "C" int hlb_part_create(const hlb_lattice* lat, int32_t n_parts, hlb_part** out) {
  return hlb_no_throw([&] { return plan_impl(lat, n_parts, out); });
}

extern "C" int hlb_part_destroy(hlb_part* plan) {
  delete plan;
  return HLB_OK;
}

extern "C" int32_t hlb_part_count(const hlb_part* plan) { return plan ? plan->P : -1; }

extern "C" int hlb_part_local(const hlb_part* plan, int32_t p, hlb_lattice* local, int64_t* owned_lo,
                              int64_t* owned_hi, const int64_t** global) {
  if (!plan || p < 0 || p >= plan->P) return hlb_fail(HLB_ERR_ARG, "no such part");
  const hlb_part::Local& T = plan->parts[(size_t)p];
  if (local) {
    local->n_sites = (int64_t)T.global.size();
    local->xyz = T.xyz.data();
    local->src = T.src.data();
    local->wall_normal = plan->has_normal ? T.normal.data() : nullptr;
    local->amp_group = plan->has_group ? T.group.data() : nullptr;
    local->n_iolets = (int32_t)plan->iolets.size();
    local->iolets = plan->iolets.data();
  }
  if (owned_lo) *owned_lo = T.lo;
  if (owned_hi) *owned_hi = T.hi;
  if (global) *global = T.global.data();
  return HLB_OK;
}

extern "C" int hlb_part_halo(const hlb_part* plan, int32_t q, int32_t p, int64_t* n, const int64_t** src_slots,
                             const int64_t** dst_slots) {
  if (!plan || p < 0 || q < 0 || p >= plan->P || q >= plan->P || p == q || !n)
    return hlb_fail(HLB_ERR_ARG, "bad part pair");
  const size_t k = (size_t)q * plan->P + p;
  *n = (int64_t)plan->hsrc[k].size();
  if (src_slots) *src_slots = plan->hsrc[k].data();
  if (dst_slots) *dst_slots = plan->hdst[k].data();
  return HLB_OK;
}

extern "C" int hlb_part_ghosts(const hlb_part* plan, int32_t q, int32_t p, int64_t* n, const int64_t** src_sites,
                               const int64_t** dst_sites) {
  if (!plan || p < 0 || q < 0 || p >= plan->P || q >= plan->P || p == q || !n)
    return hlb_fail(HLB_ERR_ARG, "bad part pair");
  const size_t k = (size_t)q * plan->P + p;
  *n = (int64_t)plan->gsrc[k].size();
  if (src_sites) *src_sites = plan->gsrc[k].data();
  if (dst_sites) *dst_sites = plan->gdst[k].data();
  return HLB_OK;
}

extern "C" int hlb_halo_pack(hlb_solver* h, const int64_t* slots, int64_t n, void* buf) {
  return halo_impl(h, slots, n, buf, true);
}

extern "C" int hlb_halo_unpack(hlb_solver* h, const int64_t* slots, int64_t n, const void* buf) {
  return halo_impl(h, slots, n, const_cast<void*>(buf), false);
}

extern "C" int hlb_set_owned_range(hlb_solver* h, int64_t lo, int64_t hi) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (lo < 0 || hi > h->n || lo >= hi) return hlb_fail(HLB_ERR_ARG, "owned range must satisfy 0 <= lo < hi <= n");
  h->owned_lo = lo;
  h->owned_hi = hi;
  return HLB_OK;
}

extern "C" int hlb_step_range(hlb_solver* h, int64_t first_tile, int64_t n_tiles, int32_t iolet_sites,
                              int32_t finish) {
  if (!h) return hlb_fail(HLB_ERR_ARG, "null solver");
  if (h->scheme != HLB_PULL_AB || h->phase != HLB_READ_GATHER_AB)
    return hlb_fail(HLB_ERR_STATE, "a partial step needs a pull A-B solver after a step");
  if (h->any_wk()) return hlb_fail(HLB_ERR_STATE, "a partial step does not update Windkessel outlets");
  const int64_t tiles = (h->n + 255) / 256;
  if (first_tile < 0 || n_tiles < 0 || first_tile + n_tiles > tiles) return hlb_fail(HLB_ERR_ARG, "tile range out of bounds");
  const cudaError_t e = hlb_launch_step_range(h, h->f[h->cur], h->f[h->cur ^ 1], h->t - 1, first_tile, n_tiles,
                                              iolet_sites != 0, h->stream);
  if (e != cudaSuccess) return hlb_cuda_fail(e, "hlb_step_range");
  h->midstep = !finish;
  if (finish) {
    h->cur ^= 1;
    h->t += 1;
    h->stepped = true;
  }
  return HLB_OK;
}
