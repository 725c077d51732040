// hlb_internal.h — host-side solver object and kernel launchers shared by
// the translation units of libhemegb.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>
#include <vector>

#include "hemegb.h"
#include "hlb_common.cuh"

// How read-back kernels obtain f(t) from a population buffer.
enum { HLB_READ_LOCAL = 0, HLB_READ_GATHER_AB = 1, HLB_READ_GATHER_AA = 2 };

struct HostWave {
  int32_t kind = HLB_WAVE_CONST;
  double mean = 0, rel = 0, period = 1, phase = 0;
  std::vector<double> samples;
  double at(double t) const;
};

struct hlb_solver {
  // lattice
  int64_t n = 0;
  int64_t sn = 0;                     // index-table row stride: n rounded up to a multiple of 4
  int64_t owned_lo = 0, owned_hi = 0; // sites counted by the mass reduction (a part's own sites)
  int32_t n_iolets = 0;
  std::vector<hlb_iolet> iolets;
  std::vector<int32_t> group_offset;  // per iolet: first global amplitude group (-1: pressure)
  int32_t n_groups_total = 0;
  std::vector<int64_t> link_begin;    // per iolet: first link record (records sorted by iolet, group)
  std::vector<int64_t> group_link_begin;  // per global amplitude group: first record; [G] = end of the last
  int64_t n_links = 0;
  bool has_normals = false;

  // options
  int32_t precision = HLB_FP32;
  int32_t scheme = HLB_PULL_AB;
  int32_t ladd_rho_one = 0;
  int32_t ghost_full_u = 0;
  bool off32 = true;  // 32-bit element offsets in the step/adjoint kernels (19 x sn fits)

  // state
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 0;                       // SMs of the device: one wave = n_sm x resident blocks per SM
  void* f[2] = {nullptr, nullptr};    // population buffers [19][n] (storage precision); AA uses f[0]
  int cur = 0;                        // buffer holding the current state
  int phase = 0;                      // HLB_READ_LOCAL: f(t) in place; GATHER_AB: s'(t-1); GATHER_AA: AA after an even step
  int64_t t = 0;
  bool stepped = false;               // f(t) came from a step (iolet fluxes defined)
  bool midstep = false;               // between the calls of one hlb_step_range step: f[cur ^ 1] is being written
  double tau = 1.0;
  std::vector<HostWave> wave;         // per iolet
  std::vector<double> amp;            // per global group

  // device tables (inside the caller's workspace)
  int32_t* d_src = nullptr;           // [18][n], iolet links re-coded to -(2 + record)
  uint32_t* d_ctab = nullptr;         // compact index table [9][sn] (hlb_common.cuh)
  int32_t* d_tbase = nullptr;         // its per-tile bases [tiles][CT_BASES]
  bool compact = false;               // bulk step and adjoint codes from the compact table
  hlb::LinkRec* d_links = nullptr;
  double* d_amp = nullptr;            // [n_groups_total]
  float* d_ampf = nullptr;            // [n_groups_total] the same rounded to float (FP32 kernels)
  float* d_normal = nullptr;          // [3][n] or null
  float* d_stage = nullptr;           // [5][n] staging for host readback
  double* d_red = nullptr;            // reduction scratch
  double* d_lflux = nullptr;          // [n_links] mass let in by each iolet link in the last AA step
  int32_t* d_iolet_sites = nullptr;   // sites with at least one iolet link (AA boundary fix-up)
  int32_t* d_icode = nullptr;         // [n_iolet_sites][18] their index codes
  uint32_t* d_imask = nullptr;        // [(n + 31) / 32] bit x % 32 of word x / 32: site x has an iolet link
  int64_t* d_ioff = nullptr;          // [n_iolets + 1] ranges of d_ilist per iolet
  int32_t* d_ilist = nullptr;         // sites with a link to iolet k, ascending, iolet by iolet
  double* d_mon = nullptr;            // [2][n_iolets] monitor outputs
  // Windkessel outlets: host flags, device parameters, model state and the
  // ghost densities the kernels read (io_val)
  std::vector<int> wk_on;             // per iolet
  double* d_wkpar = nullptr;          // [n_iolets][4] Rp, C, Rd, rho_d
  double* d_wkstate = nullptr;        // [n_iolets][2] rho_c, q (outflow of the last step)
  double* d_ioval = nullptr;          // [n_iolets] ghost density - 1 the kernels read (io_val)
  double* d_iovnext = nullptr;        // [n_iolets] pull A-B: the one after it (boundaries lag a step)
  bool any_wk() const {
    for (int v : wk_on)
      if (v) return true;
    return false;
  }
  int64_t n_iolet_sites = 0;
  int64_t red_slots = 0;

  size_t elem_bytes() const;
  size_t state_bytes() const { return elem_bytes() * 19 * (size_t)n; }
  // kernel parameters for a launch that gathers with boundary data at time tb
  hlb::StepParams params(int64_t tb) const;
};

// thread-local error text
int hlb_fail(int code, const std::string& msg);
// HLB_ERR_CUDA with the runtime's message for e (and where it happened).
int hlb_cuda_fail(cudaError_t e, const char* where);

// Runs an entry point's body; host allocation or thread failures become
// HLB_ERR_NOMEM instead of exceptions crossing the C ABI.
template <typename F>
int hlb_no_throw(F f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return hlb_fail(HLB_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return hlb_fail(HLB_ERR_NOMEM, std::string("host resource failure: ") + e.what());
  }
}

// Launch of a step-sequence kernel with programmatic stream serialisation
// (pdl_trigger / pdl_wait in hlb_common.cuh): it may be scheduled while the
// previous kernel of the stream finishes, and waits for it in pdl_wait.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- launchers (hlb_forward.cu) ----
// One pull A-B time step from fin into fout (gather: fin holds s'(t-1)).
cudaError_t hlb_launch_step(const hlb_solver* h, const void* fin, void* fout, bool gather, int64_t tb,
                            cudaStream_t s);
// Part of a pull A-B gather step: bulk tiles [tile0, tile0 + ntiles) of 256
// sites and, with `iolets`, the iolet sites.
cudaError_t hlb_launch_step_range(const hlb_solver* h, const void* fin, void* fout, int64_t tb, int64_t tile0,
                                  int64_t ntiles, bool iolets, cudaStream_t s);
// One AA time step at time t on buffer A (odd: the buffer is in the swapped phase).
cudaError_t hlb_launch_aa(const hlb_solver* h, void* A, bool odd, int64_t t, cudaStream_t s);
// rho, u [3][n], wss of the current state, device outputs (any may be null).
cudaError_t hlb_launch_macros(const hlb_solver* h, const void* fin, int mode, int64_t tb, float* rho, float* u,
                              float* wss, cudaStream_t s);
// Windkessel outlets after a step: the outflow that produces the current
// state (AA: recorded per-link masses; A-B: recomputed from `fin`, the
// post-collision state the next gather reads, with parameters at tb and,
// after `shift`, the ghost density computed one update earlier), the model
// update, and the next ghost densities.
cudaError_t hlb_launch_wk_update(const hlb_solver* h, const void* fin, int64_t tb, bool shift, cudaStream_t s);
// Windkessel outlets: forget the outflow history (q = 0) and reset the ghost
// densities to the compliance state.
cudaError_t hlb_launch_wk_reset(const hlb_solver* h, cudaStream_t s);
// Per-iolet max |u| (out[k]) and mean rho (out[K + k]) over the sites linked to iolet k.
cudaError_t hlb_launch_monitor(const hlb_solver* h, const void* fin, int mode, int64_t tb, double* out,
                               cudaStream_t s);
// Shifted pre-collision state into out [19][n] (row < 0) or direction `row` into out [n].
cudaError_t hlb_launch_state(const hlb_solver* h, const void* fin, int mode, int64_t tb, void* out, int row,
                             cudaStream_t s);
// Iolet links of d_src re-coded to -(2 + record) from the uploaded link
// records (d_links: site, direction).
cudaError_t hlb_launch_recode(const hlb_solver* h, cudaStream_t s);
// d_icode[q][i - 1] = d_src[i - 1][d_iolet_sites[q]]: the 18 codes of every
// iolet site, contiguous (after hlb_launch_recode).
cudaError_t hlb_launch_icode(const hlb_solver* h, cudaStream_t s);
// Compact index table from d_src; *misfit (device, zeroed by the caller)
// becomes nonzero if some tile's sources span more than a 16-bit offset.
cudaError_t hlb_launch_ctab(const hlb_solver* h, int32_t* misfit, cudaStream_t s);
// Equilibrium initialisation; u0 [3][n] device or null.
cudaError_t hlb_launch_init(const hlb_solver* h, void* f, double rho0, const float* u0, cudaStream_t s);
// Mass (out[0]) and per-iolet flux (out[1..]) in FP64.
cudaError_t hlb_launch_reduce(const hlb_solver* h, const void* fin, int mode, int64_t tb, bool have_flux,
                              double* out_dev, cudaStream_t s);
int64_t hlb_reduce_slots(int64_t n, int32_t n_iolets);
// Number of per-block mass partials at the start of the reduction scratch.
int64_t hlb_reduce_partials(int64_t n);
