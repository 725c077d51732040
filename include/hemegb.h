/*
 * hemegb.h — C ABI of the GB300 D3Q19 LBGK sparse-lattice solver.
 *
 * The method is the lattice Boltzmann step of arXiv 2202.11770: D3Q19 BGK
 * collision and streaming (Section 2.2, Eqs. 3a-3b, 4-6), mid-link
 * bounce-back walls (Section 2.3.1), Ladd velocity iolets and ghost-density
 * pressure iolets (Section 2.3.2), over a compact list of fluid sites reached
 * through a per-site, per-direction streaming-index table (Section 3.2.1),
 * with populations stored as a structure of arrays (Section 3.2.3, Fig. 3).
 * The equilibrium is the standard second-order form (the printed Eq. 4 lacks
 * the factors 1/2 on its quadratic terms).
 *
 * Conventions
 *  - Every call returns int: HLB_OK (0) or a negative hlb_status.  The text
 *    of the last error on the calling thread is hlb_last_error().  Nothing
 *    throws across this boundary.
 *  - Host inputs are copied during the call; the caller keeps ownership.
 *  - The library allocates no device memory.  hlb_workspace_bytes() reports
 *    the size of the device workspace that the caller allocates and passes to
 *    hlb_create(); it is borrowed until hlb_destroy().  Same for the adjoint
 *    workspace.
 *  - All GPU work is enqueued on the stream given at creation (or by
 *    hlb_set_stream).  Calls writing into device pointers are asynchronous;
 *    calls writing into host pointers synchronise that stream.
 *  - Populations are stored shifted, h_i = f_i - w_i, which keeps the
 *    significant digits of the small deviations from rest (exactly zero at
 *    rest).  The storage precision is FP32, BF16, FP16 or FP64; arithmetic is
 *    FP32 (FP64 for HLB_FP64).
 *  - D3Q19 directions, with opposite pairs adjacent (ibar = i+1 for odd i,
 *    i-1 for even i >= 2):
 *      0: (0,0,0)
 *      1..6:  (+1,0,0) (-1,0,0) (0,+1,0) (0,-1,0) (0,0,+1) (0,0,-1)
 *      7..18: (+1,+1,0) (-1,-1,0) (+1,-1,0) (-1,+1,0) (+1,0,+1) (-1,0,-1)
 *             (+1,0,-1) (-1,0,+1) (0,+1,+1) (0,-1,-1) (0,+1,-1) (0,-1,+1)
 *    weights 1/3, 1/18 (1..6), 1/36 (7..18) (Section 2.2).
 *  - Time: the solver holds the pre-collision state f(t) at integer t.  One
 *    step collides f(t) and streams it, applying boundary values computed with
 *    the waveforms evaluated at t, giving f(t+1).
 */
#ifndef HEMEGB_H
#define HEMEGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hlb_solver hlb_solver;
/* A cudaStream_t (pass 0 for the legacy default stream). */
typedef void* hlb_stream;

enum hlb_status {
  HLB_OK = 0,
  HLB_ERR_ARG = -1,      /* invalid argument or inconsistent lattice          */
  HLB_ERR_WS = -2,       /* workspace missing, too small or misaligned        */
  HLB_ERR_CUDA = -3,     /* a CUDA runtime call failed                        */
  HLB_ERR_STATE = -4,    /* call not valid in the solver's current state      */
  HLB_ERR_DIVERGED = -5, /* non-finite mass: the run has blown up             */
  HLB_ERR_NOMEM = -6     /* host allocation failed                            */
};
enum hlb_precision { HLB_FP32 = 0, HLB_BF16 = 1, HLB_FP16 = 2, HLB_FP64 = 3 };
enum hlb_scheme { HLB_SCHEME_AUTO = 0, HLB_PULL_AB = 1, HLB_AA = 2 };
enum hlb_iolet_kind { HLB_VELOCITY = 0, HLB_PRESSURE = 1 };
enum hlb_wave_kind { HLB_WAVE_CONST = 0, HLB_WAVE_COSINE = 1, HLB_WAVE_TABLE = 2 };
enum hlb_where { HLB_HOST = 0, HLB_DEVICE = 1 };
enum hlb_site_type { HLB_INNER = 0, HLB_WALLSITE = 1, HLB_INLET = 2, HLB_OUTLET = 3,
                     HLB_INLET_WALL = 4, HLB_OUTLET_WALL = 5 };

#define HLB_MAX_IOLETS 128

/* An inlet or outlet plane (Section 3.2.1: iolet count, site ranges and
 * normals are part of the GPU initialisation). */
typedef struct {
  int32_t kind;       /* HLB_VELOCITY or HLB_PRESSURE                        */
  double centre[3];   /* a point of the plane on the vessel axis             */
  double normal[3];   /* unit normal pointing into the fluid                 */
  double radius;      /* vessel radius R: Ladd weight W = max(0, 1 - r^2/R^2) */
  int32_t n_groups;   /* amplitude groups of a velocity iolet (>= 1)         */
} hlb_iolet;

/* A sparse lattice (all arrays host memory, read during hlb_create only).
 *  n_sites      number of fluid sites N, 1 <= N < 2^31
 *  xyz          int32 [N][3] integer site coordinates
 *  src          int32 [18][N]: src[(i-1)*N + s] for direction i = 1..18 is
 *               the index of the fluid site at x_s - c_i (streaming index,
 *               Section 3.2.1), or -1 (wall link: x_s - c_i is solid), or
 *               -(2+k) (the link crosses iolet k)
 *  wall_normal  float [3][N], optional (NULL): unit normal into the fluid at
 *               sites with a wall link, used by the wall shear stress;
 *               without it the normal is the normalised sum of c_i over the
 *               site's wall links (pull directions)
 *  amp_group    int32 [N], optional: amplitude group (0..n_groups-1 of the
 *               iolet) of every site with a link through a velocity iolet
 *  iolets       n_iolets (<= HLB_MAX_IOLETS) descriptors
 */
typedef struct {
  int64_t n_sites;
  const int32_t* xyz;
  const int32_t* src;
  const float* wall_normal;
  const int32_t* amp_group;
  int32_t n_iolets;
  const hlb_iolet* iolets;
} hlb_lattice;

/* precision: HLB_FP32 / HLB_BF16 / HLB_FP16 / HLB_FP64 storage.
 * scheme: HLB_PULL_AB (two population buffers, pull gather) or HLB_AA
 *   (one buffer, alternating in-place even/odd steps); AUTO picks the
 *   scheme measured faster for the lattice size: pull A-B below 750k sites
 *   (one launch per step; such states fit in the GPU's L2 cache), AA from
 *   750k sites on (fewer bytes per site).
 * ladd_rho_one: 1 = use rho = 1 in the Ladd correction instead of the
 *   site's density (the paper does not say which density).
 * ghost_full_u: 1 = pressure-iolet ghost velocity u instead of (u.n) n.
 * wide_offsets: 1 = always use the large-lattice addressing of the step
 *   and adjoint kernels.  They keep per-site offsets in 32 bits: measured
 *   from the array base while 19 x the index row stride fits (up to about
 *   226M sites), and from the start of the direction pair (rows 2p-1, 2p)
 *   above that, which covers any lattice below 2^31 sites.  This flag selects
 *   the second form at any size, so that it can be checked on small
 *   lattices.  Results are identical either way.
 * full_index: 1 = the step and adjoint kernels read the 32-bit streaming
 *   index table.  By default (0) they read a compact copy built at create:
 *   per 256-site tile and direction the smallest fluid source, and per site
 *   and direction a 16-bit offset from it (36 instead of 72 bytes a site).
 *   The lattice's sources are ordered as its sites, so in a vessel lattice
 *   the sources of one direction over a tile span a few hundred sites; if
 *   some tile's span does not fit 16 bits the library uses the 32-bit table
 *   (hlb_compact_index reports which).  Results are identical either way. */
typedef struct {
  int32_t precision;
  int32_t scheme;
  int32_t ladd_rho_one;
  int32_t ghost_full_u;
  int32_t wide_offsets;
  int32_t full_index;
} hlb_options;

/* Time-dependent scalar w(t):
 *   CONST   w = mean
 *   COSINE  w = mean * (1 + rel_amp * cos(2 pi t / period + phase))
 *   TABLE   w = mean * linear interpolation of n_samples values spaced
 *           period / n_samples apart, periodic (copied by the library). */
typedef struct {
  int32_t kind;
  double mean, rel_amp, period, phase;
  int32_t n_samples;
  const double* samples;
} hlb_waveform;

/* Objective of the adjoint: J = (1/N) sum_{t=1..N} sum_p (u(x_p, t).axis -
 * target_p)^2 over the N steps run (host arrays, copied). */
typedef struct {
  int64_t n_probe;
  const int64_t* sites;
  const double* target;
  double axis[3];
} hlb_objective;

const char* hlb_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int hlb_version(void);

/* Device workspace size for a lattice and options (Section 3.2.1: the
 * populations f_old/f_new, streaming indices, boundary-link data and iolet
 * data the GPU initialisation allocates).  HLB_ERR_ARG on a bad lattice. */
int hlb_workspace_bytes(const hlb_lattice* lat, const hlb_options* opt, size_t* bytes);

/* Validate the lattice, lay out the workspace (256-byte aligned device
 * pointer of at least hlb_workspace_bytes), upload tables and set the state
 * to rest (f = w, t = 0), tau = 1, velocity amplitudes 0 and pressure
 * densities 1.  Errors: HLB_ERR_ARG (index out of range, link code naming a
 * missing iolet, group out of range, bad option), HLB_ERR_WS, HLB_ERR_CUDA. */
int hlb_create(const hlb_lattice* lat, const hlb_options* opt, void* dev_ws, size_t ws_bytes,
               hlb_stream stream, hlb_solver** out);
int hlb_destroy(hlb_solver* h);
int hlb_set_stream(hlb_solver* h, hlb_stream stream);
int64_t hlb_n_sites(const hlb_solver* h);
/* 1 if the step and adjoint kernels read the compact index table, 0 if the
 * 32-bit one (see hlb_options.full_index); HLB_ERR_ARG for a null handle. */
int hlb_compact_index(const hlb_solver* h);

/* Relaxation time tau (Eq. 3a, Delta t = 1); viscosity nu = (tau - 1/2)/3
 * (Eq. 8).  HLB_ERR_ARG unless tau > 1/2. */
int hlb_set_tau(hlb_solver* h, double tau);

/* Velocity iolet k (Section 2.3.2, Section 6): the wall velocity at a link
 * midpoint x_m is u_w = amp[g] * w(t) * W(x_m) * n, g the site's amplitude
 * group, W the parabolic cross-section weight.  n_groups must equal the
 * iolet's.  HLB_ERR_ARG if k is not a velocity iolet. */
int hlb_set_velocity_waveform(hlb_solver* h, int32_t k, const double* amp, int32_t n_groups,
                              const hlb_waveform* w);

/* Pressure iolet k (Section 2.3.2, Eq. 7): ghost density rho(t) = w(t)
 * (= p(t)/cs^2).  HLB_ERR_ARG if k is not a pressure iolet.  Turns a
 * Windkessel outlet back into a waveform outlet. */
int hlb_set_pressure(hlb_solver* h, int32_t k, const hlb_waveform* w);

/* Pressure iolet k as a three-element Windkessel outlet: the downstream
 * resistance model that the paper's Section 7 names as future work (not part
 * of its method).  The ghost density becomes state of the device:
 *   ghost density for the next step = rho_c + Rp q,
 *   rho_c <- rho_c + (q - (rho_c - rho_d) / Rd) / C   after each step,
 * q being the outflow (minus the mass flux of hlb_reduce) of the step that
 * produced the current state; C = 0 is a pure resistance, ghost density
 * rho_d + (Rp + Rd) q.  The coupling is explicit (one step of lag) and runs
 * one extra small kernel per step.  rho_c starts at rho_c0 (C > 0) and the
 * outflow history at 0; hlb_init_equilibrium clears the history again.
 * Densities are lattice densities (pressure = rho / 3).  HLB_ERR_ARG if k
 * is not a pressure iolet, a parameter is negative, rho_d or rho_c0 is not
 * positive, or C > 0 with Rd C < 1 (the explicit update would overshoot).
 * hlb_adjoint_run refuses a solver with Windkessel outlets. */
int hlb_set_windkessel(hlb_solver* h, int32_t k, double Rp, double C, double Rd, double rho_d, double rho_c0);

/* Model state of Windkessel outlet k (synchronises): the ghost density the
 * next boundary evaluation uses, rho_c and the last outflow q (any NULL). */
int hlb_windkessel_state(hlb_solver* h, int32_t k, double* rho_ghost, double* rho_c, double* q);

/* Set f = f^eq(rho0, u0) everywhere and t = 0 (Section 3.1 step 1).  u0 is
 * float [3][N] (host or device per `where`) or NULL for u = 0. */
int hlb_init_equilibrium(hlb_solver* h, double rho0, const float* u0, int32_t where);

/* Advance n >= 0 time steps (Section 3.1 steps 2-5), asynchronously: per
 * step one fused collide-stream-boundary kernel launch (pull A-B: iolet
 * sites included), plus for the AA scheme the boundary pass over the iolet
 * sites, plus one small update kernel when Windkessel outlets are set. */
int hlb_step(hlb_solver* h, int64_t n);
int hlb_time(const hlb_solver* h, int64_t* t);

/* Density rho [N], velocity u [3][N] and wall shear stress wss [N] of the
 * current state f(t) (Eqs. 5-6; the paper's property cache).  WSS (not in the
 * paper): traction t = sigma n of the viscous stress
 * sigma = -(1 - 1/(2 tau)) sum_i (f_i - f^eq_i) c_i c_i, WSS = |t - (t.n) n|,
 * NaN at sites without a wall link.  Any output may be NULL.  Device outputs
 * are asynchronous; host outputs synchronise. */
int hlb_read_macros(hlb_solver* h, float* rho, float* u, float* wss, int32_t where);

/* FP64 reductions of the current state (synchronises): total mass
 * sum_x sum_i f_i(x, t), and per iolet the mass that entered through it in
 * the step that produced f(t) (incoming boundary populations minus the
 * post-collision populations that left), so that
 * mass(t) - mass(t-1) = sum_k flux_k(t).  iolet_flux may be NULL.
 * HLB_ERR_DIVERGED if the mass is not finite. */
int hlb_reduce(hlb_solver* h, double* mass, double* iolet_flux);

/* Iolet monitor of the current state f(t), the quantities of the paper's
 * pipe validation (Section 6: volumetric flow rate, maximum velocity and
 * pressure at the inlet and the outlet), per iolet k, each array
 * [n_iolets] on the host, any of them NULL:
 *   flux[k]     mass that entered through iolet k in the step that produced
 *               f(t), as hlb_reduce reports it (flow rate x density);
 *   u_max[k]    max |u| over the sites with a link to iolet k;
 *   rho_mean[k] mean density over those sites (pressure = rho_mean / 3).
 * FP64, deterministic; synchronises the solver's stream. */
int hlb_iolet_monitor(hlb_solver* h, double* flux, double* u_max, double* rho_mean);

/* Shifted pre-collision state h_i = f_i(t) - w_i as [19][N] in the storage
 * precision (host or device per `where`), and its time t.  set_state
 * resumes from such a state. */
int hlb_get_state(hlb_solver* h, void* f, int32_t where, int64_t* t);
int hlb_set_state(hlb_solver* h, const void* f, int32_t where, int64_t t);

/* Discrete adjoint (no counterpart in the paper): from the current state,
 * run N steps, evaluate the objective, and back-propagate through the exact
 * transpose of every step (collision, streaming, bounce-back, Ladd and
 * pressure boundaries), recomputing states from sqrt(N)-spaced checkpoints.
 * Outputs J, dJ/dtau and dJ/da_g for every amplitude group of every velocity
 * iolet (iolet order, then group).  The forward sweep runs the solver's own
 * scheme; the state is left at t + N as that scheme's step leaves it.  FP32
 * and FP64 storage only.  hlb_adjoint_workspace_bytes gives the device workspace
 * (checkpoints + one segment of states + adjoint buffers). */
int hlb_adjoint_workspace_bytes(const hlb_solver* h, int64_t nsteps, int64_t n_probe,
                                size_t* bytes);
/* A workspace larger than that minimum trades memory for recomputation: the
 * run then keeps the post-collision states of whole checkpoint segments from
 * its forward sweep (K more states each, K = 2 ceil(ceil(sqrt N) / 2) the
 * checkpoint interval, every segment but the last) and recomputes only the
 * others; results are identical.  hlb_adjoint_plan reports, for a workspace
 * of ws_bytes, the interval K, the kept segments, the steps still recomputed
 * and the bytes the run uses (any output may be NULL); HLB_ERR_WS below the
 * minimum. */
int hlb_adjoint_plan(const hlb_solver* h, int64_t nsteps, int64_t n_probe, size_t ws_bytes, int64_t* interval,
                     int64_t* kept_segments, int64_t* recomputed_steps, size_t* bytes_used);
int hlb_adjoint_run(hlb_solver* h, int64_t nsteps, const hlb_objective* obj, void* dev_ws,
                    size_t ws_bytes, double* J, double* dJ_dtau, double* dJ_damp);
int hlb_n_amp_groups(const hlb_solver* h);

/* Total mass without any allocation (the paper has no counterpart).  For
 * callers that cannot allocate device memory where they need this number:
 * a host framework whose allocator owns all device memory, or a
 * time-critical loop where cudaMalloc's implicit synchronisation is not
 * acceptable.  Sums a shifted population array f [19][n_sites] (device
 * memory, storage `precision`, e.g. written by hlb_get_state with
 * HLB_DEVICE) into *mass (one double in device memory) as
 * n_sites + sum of all entries, in FP64, asynchronously on `stream`.  For
 * FP32 and FP64 storage, and for AA-scheme states in any precision, the
 * result equals hlb_reduce's mass of the same state.  A 16-bit state that
 * hlb_get_state reads back after a pull A-B step carries the boundary values
 * of the iolet links rounded to the storage format, which hlb_reduce sums
 * unrounded: the two masses then differ by at most the sum of half an ulp of
 * each of those values.  Its per-block partial
 * sums live in a fixed 2 MiB device array inside the library (one copy per
 * GPU that loads the library, held until the process exits), so n_sites may
 * not exceed HLB_STATIC_MAX_SITES: larger sizes return HLB_ERR_ARG.  The
 * first call on a device looks up that array's device address (with the
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture.  cudaDeviceReset ends the device's context
 * and with it that address: do not call this entry point on a device after
 * resetting it.  Every
 * call shares the array and leaves its partial sums there; nothing in it
 * needs to start at zero.  Calls that overlap on the GPU (two streams, or two
 * host threads) race on it and must be serialised by the caller.  No
 * cudaMalloc, cudaFree or allocating library routine is called. */
#define HLB_STATIC_MAX_SITES 67108864
int hlb_mass_static(const void* f, int32_t precision, int64_t n_sites, double* mass, hlb_stream stream);

#ifdef __cplusplus
}
#endif
#endif
